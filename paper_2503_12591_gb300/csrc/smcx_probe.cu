// Measured on-chip roof for the sweep kernels: the shared-memory byte-load
// rate of this GPU.  Every lane of every warp issues independent LDS.U8 at
// addresses that put the 32 lanes on 32 different banks (one wavefront per
// warp load), so the kernel runs at the shared-memory pipe's peak: lane-loads
// per second = (loads per thread) x (threads) / time.  The sweep kernels'
// roofline fraction is their algorithmic lane-loads per second over this.
#include "smcx_internal.h"

namespace smcx {
namespace {

constexpr int kProbeBytes = 16384;
constexpr int kProbeIters = 2048;  // 16 loads each

__global__ void __launch_bounds__(256) k_lds_probe(unsigned* out) {
  __shared__ unsigned char buf[kProbeBytes];
  for (int i = threadIdx.x; i < kProbeBytes; i += blockDim.x) buf[i] = (unsigned char)(i * 131u);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // lane l reads byte 4 l of a 128-byte line: bank l
  unsigned base = (unsigned)(warp * 512 + 4 * lane);
  unsigned acc = 0;
  for (int it = 0; it < kProbeIters; it++) {
#pragma unroll
    for (int u = 0; u < 16; u++) acc += buf[(base + (unsigned)u * 128u) & (kProbeBytes - 1)];
    base = (base + 2048u + (acc & 0u)) & (kProbeBytes - 1);
  }
  if (acc == 0xFFFFFFFFu) out[0] = acc;  // keeps the loads live
}

}  // namespace
}  // namespace smcx

using namespace smcx;

extern "C" int smcx_probe_lds_rate(double* lane_loads_per_s, void* stream) {
  return guarded_call([&] {
    if (!lane_loads_per_s) fail(SMCX_E_INVALID_ARG, "NULL argument");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0, per_sm = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    check_cuda(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "SM count");
    check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lds_probe, 256, 0), "occupancy");
    const int grid = nsm * per_sm;
    unsigned* d_out = nullptr;
    check_cuda(cudaMalloc(&d_out, sizeof(unsigned)), "probe output");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    check_cuda(cudaEventCreate(&e0), "event");
    check_cuda(cudaEventCreate(&e1), "event");
    k_lds_probe<<<grid, 256, 0, st>>>(d_out);  // warm-up
    check_cuda(cudaEventRecord(e0, st), "event");
    const int reps = 4;
    for (int r = 0; r < reps; r++) k_lds_probe<<<grid, 256, 0, st>>>(d_out);
    check_cuda(cudaEventRecord(e1, st), "event");
    check_cuda(cudaEventSynchronize(e1), "event sync");
    check_cuda(cudaGetLastError(), "probe launch");
    float ms = 0;
    check_cuda(cudaEventElapsedTime(&ms, e0, e1), "event time");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_out);
    const double loads = (double)reps * grid * 256.0 * kProbeIters * 16.0;
    *lane_loads_per_s = loads / (ms * 1e-3);
  });
}
