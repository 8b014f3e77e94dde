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
// before any stream capture.  The looked-up address is kept for the life of
// the process: after cudaDeviceReset it may be stale, so a process that
// resets a device must not call this entry point on it again.  Every call
// uses the same array: the histogram and the bad-id flag are cleared at the
// start of each call, and calls whose GPU work overlaps (two streams, two
// host threads) race on it and give wrong results.
//
// The configuration arrives as a bare device pointer that no handle has
// validated, so this entry point counts pairs with its own kernel, which
// checks every species id against M: an id outside 0..M-1 is not counted (it
// would index past the shared-memory histogram), sets a flag word in the
// scratch array, and the call returns SMCX_E_INVALID_ARG.
#include <mutex>

#include "smcx_device.cuh"

namespace smcx {

// Scratch capacity: K*M*M histogram words, one energy word, the int32 EPI
// table packed two per word, and (last word of the array) the bad-id flag.
// 16 KiB holds K*M*M <= 1300: 1300 + 1 + 650 words, below the flag word.
constexpr int kNoAllocWords = 2048;
constexpr int kNoAllocMaxKMM = 1300;
constexpr int kNoAllocFlagWord = kNoAllocWords - 1;
static_assert(kNoAllocMaxKMM + 1 + (kNoAllocMaxKMM + 1) / 2 <= kNoAllocFlagWord, "scratch layout");
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocWords];

// Ordered pair counts C[k][p][q] (Eq. Total_EPI, pair form) of a store that
// no handle validated: ids outside 0..M-1 are skipped and flagged in *bad.
template <int KIND, int K>
__global__ void __launch_bounds__(256) k_noalloc_pair_counts(const SweepParams P, unsigned long long* counts,
                                                             unsigned long long* bad) {
  constexpr int m = cell_sites(KIND);
  extern __shared__ unsigned int hist[];
  const int M = P.M, KMM = K * P.M * P.M;
  for (int i = threadIdx.x; i < KMM; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
  const long long ncell = (long long)nx * ny * nz;
  int seen_bad = 0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % nx);
    const long long r = c / nx;
    const int y = (int)(r % ny), z = (int)(r / ny);
    for (int b = 0; b < m; b++) {
      const int p = load_site(P.sites, c * m + b, P.storage);
      if (p >= M) {
        seen_bad = 1;
        continue;
      }
      int j = 0;
#pragma unroll
      for (int k = 0; k < K; k++) {
        for (int v = 0; v < shell_size(KIND, k); v++, j++) {
          const signed char* d = P.gd[b][j];
          const long long t =
              (((long long)wrap_add(z, d[2], nz) * ny + wrap_add(y, d[1], ny)) * nx + wrap_add(x, d[0], nx)) * m +
              d[3];
          const int q = load_site(P.sites, t, P.storage);
          if (q >= M) {
            seen_bad = 1;
            continue;
          }
          atomicAdd(&hist[(k * M + p) * M + q], 1u);
        }
      }
    }
  }
  if (__syncthreads_or(seen_bad) && threadIdx.x == 0) atomicOr(bad, 1ull);
  for (int i = threadIdx.x; i < KMM; i += blockDim.x)
    if (hist[i]) atomicAdd(&counts[i], (unsigned long long)hist[i]);
}

static void noalloc_pair_counts(int kind, int K, const SweepParams& P, long long ncell, int KMM,
                                unsigned long long* counts, unsigned long long* bad, cudaStream_t st) {
  int dev = 0, nsm = 0;
  check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  check_cuda(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "SM count");
  const int grid = (int)std::min<long long>((ncell + 255) / 256, (long long)nsm * 8);
  const size_t sm = (size_t)KMM * sizeof(unsigned int);
  if (kind == kBCC) {
    switch (K) {
      case 1: k_noalloc_pair_counts<kBCC, 1><<<grid, 256, sm, st>>>(P, counts, bad); break;
      case 2: k_noalloc_pair_counts<kBCC, 2><<<grid, 256, sm, st>>>(P, counts, bad); break;
      case 3: k_noalloc_pair_counts<kBCC, 3><<<grid, 256, sm, st>>>(P, counts, bad); break;
      default: k_noalloc_pair_counts<kBCC, 4><<<grid, 256, sm, st>>>(P, counts, bad); break;
    }
  } else {
    switch (K) {
      case 1: k_noalloc_pair_counts<kFCC, 1><<<grid, 256, sm, st>>>(P, counts, bad); break;
      case 2: k_noalloc_pair_counts<kFCC, 2><<<grid, 256, sm, st>>>(P, counts, bad); break;
      default: k_noalloc_pair_counts<kFCC, 3><<<grid, 256, sm, st>>>(P, counts, bad); break;
    }
  }
  check_cuda(cudaGetLastError(), "no-alloc pair-count launch");
}

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
    {
      // a host or unregistered pointer would fault in the kernel
      cudaPointerAttributes attr;
      if (cudaPointerGetAttributes(&attr, d_sites) != cudaSuccess) {
        cudaGetLastError();
        fail(SMCX_E_INVALID_ARG, "configuration pointer is not known to CUDA");
      }
      if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
        fail(SMCX_E_INVALID_ARG, "configuration pointer is not device memory");
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned long long* scratch = scratch_for_current_device();
    unsigned long long* bad = scratch + kNoAllocFlagWord;
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
    check_cuda(cudaMemsetAsync(bad, 0, sizeof(unsigned long long), st), "clear bad-id flag");
    // pageable source: staged before cudaMemcpyAsync returns
    check_cuda(cudaMemcpyAsync(dV, V, (size_t)KMM * sizeof(int32_t), cudaMemcpyHostToDevice, st), "EPI upload");
    noalloc_pair_counts(kind, K, P, (long long)nx * ny * nz, KMM, counts, bad, st);
    energy_raw(counts, dV, KMM, energy, st);
    long long e = 0;
    unsigned long long flag = 0;
    check_cuda(cudaMemcpyAsync(&e, energy, sizeof(e), cudaMemcpyDeviceToHost, st), "energy download");
    check_cuda(cudaMemcpyAsync(&flag, bad, sizeof(flag), cudaMemcpyDeviceToHost, st), "flag download");
    check_cuda(cudaStreamSynchronize(st), "energy sync");
    if (flag) fail(SMCX_E_INVALID_ARG, "configuration holds species ids outside 0..M-1");
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
