// smcx_energy_noalloc: the lattice energy for callers that cannot allocate
// device memory.
//
// Some callers must not call cudaMalloc at all: code running inside another
// allocator's arena (a framework that owns every byte of device memory and
// would be confused by a foreign allocation), real-time loops that may not
// block on the driver's allocator, or callers that only hold a device pointer
// to a configuration and no smcx handle.  smcx_energy (the handle-based call)
// keeps its pair-count histogram in memory the handle allocated; this entry
// point instead keeps that histogram, the EPI table and the result in one
// file-scope device array of fixed size, so it allocates nothing.
//
// The array lives in every GPU that loads this library until the process
// exits.  Its device address is looked up once per device (with that device
// current) the first time this entry point runs there; make that first call
// before any stream capture.  Every call uses the same array: the histogram
// is cleared at the start of each call, and calls whose GPU work overlaps
// (two streams, two host threads) race on it and give wrong results.
#include <mutex>

#include "smcx_device.cuh"

namespace smcx {

// Scratch capacity: K*M*M histogram words, one energy word, the int32 EPI
// table packed two per word.  16 KiB holds K*M*M <= 1300.
constexpr int kNoAllocWords = 2048;
constexpr int kNoAllocMaxKMM = 1300;
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocWords];

namespace {

std::mutex g_noalloc_mu;
unsigned long long* g_noalloc_ptr[64] = {nullptr};

unsigned long long* scratch_for_current_device() {
  int dev = 0;
  check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= 64) fail(SMCX_E_UNSUPPORTED, "device ordinal above 63");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    check_cuda(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(noalloc scratch)");
    g_noalloc_ptr[dev] = static_cast<unsigned long long*>(p);
  }
  return g_noalloc_ptr[dev];
}

}  // namespace
}  // namespace smcx

using namespace smcx;

extern "C" int smcx_energy_noalloc(int kind, int nx, int ny, int nz, int M, int storage, int K, const int32_t* V,
                                   const void* d_sites, int64_t* E, void* stream) {
  try {
    set_error("");
    if (!V || !d_sites || !E) fail(SMCX_E_INVALID_ARG, "NULL argument");
    if (kind != kBCC && kind != kFCC) fail(SMCX_E_INVALID_ARG, "kind must be SMCX_BCC or SMCX_FCC");
    if (nx < 1 || ny < 1 || nz < 1) fail(SMCX_E_INVALID_ARG, "dimensions must be >= 1");
    if (storage != SMCX_INT8 && storage != SMCX_PACKED4) fail(SMCX_E_INVALID_ARG, "unknown storage");
    if (M < 1 || M > (storage == SMCX_PACKED4 ? 15 : 127)) fail(SMCX_E_INVALID_ARG, "species count out of range");
    const Shells S = make_shells(kind, K);  // validates K
    {
      const int n3[3] = {nx, ny, nz};
      check_reach(S, n3);
    }
    const int KMM = K * M * M;
    if (KMM > kNoAllocMaxKMM)
      fail(SMCX_E_INVALID_ARG, "K*M*M = " + std::to_string(KMM) + " exceeds the fixed scratch of this entry point (" +
                                   std::to_string(kNoAllocMaxKMM) + ")");
    for (int k = 0; k < K; k++)
      for (int p = 0; p < M; p++)
        for (int q = 0; q < M; q++)
          if (V[(k * M + p) * M + q] != V[(k * M + q) * M + p])
            fail(SMCX_E_INVALID_ARG, "EPI table is not symmetric");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned long long* scratch = scratch_for_current_device();
    unsigned long long* counts = scratch;
    long long* energy = reinterpret_cast<long long*>(scratch + KMM);
    int32_t* dV = reinterpret_cast<int32_t*>(scratch + KMM + 1);

    SweepParams P;
    memset(&P, 0, sizeof(P));
    P.sites = const_cast<uint8_t*>(static_cast<const uint8_t*>(d_sites));
    P.M = M;
    P.storage = storage;
    P.n[0] = nx;
    P.n[1] = ny;
    P.n[2] = nz;
    for (int b = 0; b < S.m; b++) {
      int B[3];
      basis_of(kind, b, B);
      for (int j = 0; j < S.nv; j++) {
        int d[3], r[3];
        for (int a = 0; a < 3; a++) {
          const int p = B[a] + S.v[j][a];
          d[a] = (p >= 0) ? p / 2 : -((-p + 1) / 2);
          r[a] = p - 2 * d[a];
        }
        P.gd[b][j][0] = (signed char)d[0];
        P.gd[b][j][1] = (signed char)d[1];
        P.gd[b][j][2] = (signed char)d[2];
        P.gd[b][j][3] = (signed char)basis_index(kind, r[0], r[1], r[2]);
      }
    }
    check_cuda(cudaMemsetAsync(counts, 0, (size_t)KMM * sizeof(unsigned long long), st), "clear scratch histogram");
    // pageable source: staged before cudaMemcpyAsync returns
    check_cuda(cudaMemcpyAsync(dV, V, (size_t)KMM * sizeof(int32_t), cudaMemcpyHostToDevice, st), "EPI upload");
    pair_counts_raw(kind, K, P, (long long)nx * ny * nz, KMM, counts, st);
    energy_raw(counts, dV, KMM, energy, st);
    long long e = 0;
    check_cuda(cudaMemcpyAsync(&e, energy, sizeof(e), cudaMemcpyDeviceToHost, st), "energy download");
    check_cuda(cudaStreamSynchronize(st), "energy sync");
    *E = e;
    return SMCX_OK;
  } catch (const SmcxException& ex) {
    set_error(ex.msg);
    return ex.code;
  } catch (...) {
    set_error("unknown failure");
    return SMCX_E_INVALID_ARG;
  }
}
