// Differentiation kernels for fitting and for thermodynamic derivatives.
//
// Energy model (Method, Eq. Total_EPI, pair form):
//   E(sigma; V) = 1/2 sum_{k,p,q} V_k[p][q] C_k[p][q](sigma),
// linear in V, so dE/dV_k[p][q] = C_k[p][q] / 2 with the entries of V taken
// as independent (the paper fits V by back-propagation, Results "Energy
// model"; the pair-count histograms are the whole backward pass).
//
// Thermal averages under the Boltzmann weight exp(-beta E) (Supplementary
// "Statistical mechanics") obey
//   d<A>/dV_i = -beta (<A dE/dV_i> - <A><dE/dV_i>),
// so an estimator needs sum(1), sum(A), sum(C), sum(A C^T) over samples; they
// are accumulated on the device in FP64 (weighted, so that exact enumeration
// can feed Boltzmann weights through the same code).
#include "smcx_device.cuh"

namespace smcx {

// One CTA per configuration: stage the configuration's species ids in shared
// memory, count ordered pairs per shell into a shared histogram, write it out.
template <int KIND, int K>
__global__ void __launch_bounds__(256) k_pair_counts_batch(const int8_t* __restrict__ cfg, long long B, int nx,
                                                           int ny, int nz, int M, SweepParams P,
                                                           long long* __restrict__ out) {
  constexpr int m = cell_sites(KIND);
  extern __shared__ __align__(16) unsigned char smem[];
  const int KMM = K * M * M;
  unsigned int* hist = reinterpret_cast<unsigned int*>(smem);
  int8_t* s = reinterpret_cast<int8_t*>(hist + KMM);
  const long long N = (long long)nx * ny * nz * m;
  for (long long b = blockIdx.x; b < B; b += gridDim.x) {
    for (int i = threadIdx.x; i < KMM; i += blockDim.x) hist[i] = 0;
    const int8_t* c = cfg + b * N;
    int bad = 0;
    for (long long i = threadIdx.x; i < N; i += blockDim.x) {
      const int8_t v = c[i];
      s[i] = v;
      bad |= (v < 0 || v >= M);
    }
    // a configuration holding an id outside 0..M-1 is not counted (its bins
    // would lie outside the histogram); all its counts are set to -1
    bad = __syncthreads_or(bad);
    for (long long cell = threadIdx.x; !bad && cell < (long long)nx * ny * nz; cell += blockDim.x) {
      const int x = (int)(cell % nx), y = (int)((cell / nx) % ny), z = (int)(cell / ((long long)nx * ny));
#pragma unroll
      for (int bsub = 0; bsub < m; bsub++) {
        const int p = s[cell * m + bsub];
        int j = 0;
#pragma unroll
        for (int k = 0; k < K; k++) {
#pragma unroll
          for (int q = 0; q < shell_size(KIND, k); q++, j++) {
            const signed char* d = P.gd[bsub][j];
            const long long t =
                (((long long)wrap_add(z, d[2], nz) * ny + wrap_add(y, d[1], ny)) * nx + wrap_add(x, d[0], nx)) * m +
                d[3];
            atomicAdd(&hist[(k * M + p) * M + s[t]], 1u);
          }
        }
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < KMM; i += blockDim.x) out[b * KMM + i] = bad ? -1ll : (long long)hist[i];
    __syncthreads();
  }
}

// E_b = 1/2 sum_i V_i C_bi (FP64 sum, FP32 result): one warp per config.
__global__ void k_epi_energy(const float* __restrict__ V, const long long* __restrict__ C, long long B, int KMM,
                             float* __restrict__ E) {
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= B) return;
  double s = 0.0;
  for (int i = lane; i < KMM; i += 32) s += (double)V[i] * (double)C[w * KMM + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) E[w] = (float)(0.5 * s);
}

// grad_i = 1/2 sum_b g_b C_bi (FP64 sum, FP32 result): one CTA per entry i.
__global__ void k_epi_grad(const float* __restrict__ g, const long long* __restrict__ C, long long B, int KMM,
                           float* __restrict__ grad) {
  __shared__ double part[32];
  const int i = blockIdx.x;
  double s = 0.0;
  for (long long b = threadIdx.x; b < B; b += blockDim.x) s += (double)g[b] * (double)C[b * KMM + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; w++) t += part[w];
    grad[i] = (float)(0.5 * t);
  }
}

// Accumulate B weighted samples (w == NULL: weight 1).  A = Warren-Cowley
// alpha of shell `sh` from the counts (species numbers from the shell-0 row
// sums / z_0):
//   acc[0] += sum w; acc[1 + a] += sum w A_a; acc[1 + MM + i] += sum w C_i;
//   acc[1 + MM + KMM + a * KMM + i] += sum w A_a C_i.
// Each thread owns fixed entries and sums samples in order (deterministic).
constexpr int kFluctOwn = 8;
// With acc_stride > 0, CTA r takes sample r alone into acc + r acc_stride
// (one accumulator per replica) and, for N <= 0, the site count of that
// sample from its shell-1 counts (sum_pq C_1[p][q] = z_1 N).
__global__ void k_fluct_accumulate(const long long* __restrict__ C, long long B, const double* __restrict__ w, int K,
                                   int M, int sh, int z0, int zs, double N, double* __restrict__ acc,
                                   long long acc_stride) {
  extern __shared__ double sA[];  // MM
  const int MM = M * M, KMM = K * MM;
  const int total = 1 + MM + KMM + MM * KMM;
  double loc[kFluctOwn];
#pragma unroll
  for (int j = 0; j < kFluctOwn; j++) loc[j] = 0.0;
  long long b_lo = 0, b_hi = B;
  if (acc_stride > 0) {
    b_lo = blockIdx.x;
    b_hi = b_lo + 1;
    acc += b_lo * acc_stride;
  }
  for (long long b = b_lo; b < b_hi; b++) {
    const long long* Cb = C + b * KMM;
    if (N <= 0.0) {
      double n1 = 0.0;
      for (int i = 0; i < MM; i++) n1 += (double)Cb[i];
      N = n1 / z0;
    }
    for (int a = threadIdx.x; a < MM; a += blockDim.x) {
      const int p = a / M, q = a % M;
      double Np = 0.0, Nq = 0.0;
      for (int r = 0; r < M; r++) {
        Np += (double)Cb[p * M + r];
        Nq += (double)Cb[q * M + r];
      }
      Np /= z0;
      Nq /= z0;
      const double denom = (double)zs * Np * (Nq / N);
      sA[a] = denom > 0.0 ? 1.0 - (double)Cb[(size_t)sh * MM + a] / denom : 0.0;
    }
    __syncthreads();
    const double wb = w ? w[b] : 1.0;
#pragma unroll
    for (int j = 0; j < kFluctOwn; j++) {
      const int t = threadIdx.x + j * blockDim.x;
      if (t >= total) continue;
      double v;
      if (t == 0) v = 1.0;
      else if (t < 1 + MM) v = sA[t - 1];
      else if (t < 1 + MM + KMM) v = (double)Cb[t - 1 - MM];
      else {
        const int u = t - 1 - MM - KMM;
        v = sA[u / KMM] * (double)Cb[u % KMM];
      }
      loc[j] += wb * v;
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < kFluctOwn; j++) {
    const int t = threadIdx.x + j * blockDim.x;
    if (t < total) acc[t] += loc[j];
  }
}

// d<A_a>/dV_i = -beta (<A_a C_i/2> - <A_a><C_i/2>), beta in 1/meV: the
// gradient with respect to V in meV.
__global__ void k_fluct_gradient(const double* __restrict__ acc, int MM, int KMM, double beta,
                                 double* __restrict__ grad) {
  const double W = acc[0];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < MM * KMM; t += gridDim.x * blockDim.x) {
    const int a = t / KMM, i = t % KMM;
    const double EA = acc[1 + a] / W, EC = 0.5 * acc[1 + MM + i] / W;
    const double EAC = 0.5 * acc[1 + MM + KMM + t] / W;
    grad[t] = -beta * (EAC - EA * EC);
  }
}

void fill_offsets_kind(int kind, const Shells& S, SweepParams& P) {
  for (int b = 0; b < S.m; b++) {
    int Bv[3];
    basis_of(kind, b, Bv);
    for (int j = 0; j < S.nv; j++) {
      int d[3], r[3];
      for (int a = 0; a < 3; a++) {
        const int p = Bv[a] + S.v[j][a];
        d[a] = (p >= 0) ? p / 2 : -((-p + 1) / 2);
        r[a] = p - 2 * d[a];
      }
      P.gd[b][j][0] = (signed char)d[0];
      P.gd[b][j][1] = (signed char)d[1];
      P.gd[b][j][2] = (signed char)d[2];
      P.gd[b][j][3] = (signed char)basis_index(kind, r[0], r[1], r[2]);
    }
  }
}

}  // namespace smcx

using namespace smcx;

extern "C" {

int smcx_pair_counts_batch(int kind, int nx, int ny, int nz, int M, int K, const int8_t* d_configs, int64_t B,
                           int64_t* d_counts, void* stream) {
  return guarded_call([&] {
    if (!d_configs || !d_counts || B < 0) fail(SMCX_E_INVALID_ARG, "bad arguments");
    if (nx < 1 || ny < 1 || nz < 1 || M < 1 || M > 127) fail(SMCX_E_INVALID_ARG, "bad geometry");
    const Shells S = make_shells(kind, K);
    {
      const int n3[3] = {nx, ny, nz};
      check_reach(S, n3);
    }
    const long long N = (long long)nx * ny * nz * S.m;
    const int KMM = K * M * M;
    const size_t smem = (size_t)KMM * 4 + (size_t)N;
    if (smem > 200 * 1024) fail(SMCX_E_UNSUPPORTED, "configurations above ~200k sites: use smcx_pair_counts");
    if (B == 0) return;
    SweepParams P;
    memset(&P, 0, sizeof(P));
    fill_offsets_kind(kind, S, P);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int grid = (int)std::min<long long>(B, 65535);
    auto go = [&](auto kern) {
      check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "smem attr");
      kern<<<grid, 256, smem, st>>>(d_configs, B, nx, ny, nz, M, P, reinterpret_cast<long long*>(d_counts));
    };
    if (kind == kBCC) {
      if (K == 1) go(k_pair_counts_batch<kBCC, 1>);
      else if (K == 2) go(k_pair_counts_batch<kBCC, 2>);
      else if (K == 3) go(k_pair_counts_batch<kBCC, 3>);
      else go(k_pair_counts_batch<kBCC, 4>);
    } else {
      if (K == 1) go(k_pair_counts_batch<kFCC, 1>);
      else if (K == 2) go(k_pair_counts_batch<kFCC, 2>);
      else go(k_pair_counts_batch<kFCC, 3>);
    }
    check_cuda(cudaGetLastError(), "pair-count batch launch");
  });
}

int smcx_epi_energy_batch(const float* d_V, const int64_t* d_counts, int64_t B, int KMM, float* d_E, void* stream) {
  return guarded_call([&] {
    if (!d_V || !d_counts || !d_E || B < 0 || KMM < 1) fail(SMCX_E_INVALID_ARG, "bad arguments");
    if (B == 0) return;
    const long long warps = B;
    const int grid = (int)((warps * 32 + 255) / 256);
    k_epi_energy<<<grid, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        d_V, reinterpret_cast<const long long*>(d_counts), B, KMM, d_E);
    check_cuda(cudaGetLastError(), "energy batch launch");
  });
}

int smcx_epi_grad_batch(const float* d_g, const int64_t* d_counts, int64_t B, int KMM, float* d_grad, void* stream) {
  return guarded_call([&] {
    if (!d_g || !d_counts || !d_grad || B < 0 || KMM < 1) fail(SMCX_E_INVALID_ARG, "bad arguments");
    k_epi_grad<<<KMM, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        d_g, reinterpret_cast<const long long*>(d_counts), B, KMM, d_grad);
    check_cuda(cudaGetLastError(), "grad batch launch");
  });
}

}  // extern "C"

static void fluct_launch(const long long* C, long long B, const double* w, int K, int M, int shell, int z0, int zs,
                         double N, double* acc, cudaStream_t st) {
  const int MM = M * M, KMM = K * MM;
  const int total = 1 + MM + KMM + MM * KMM;
  const int threads = std::min(1024, std::max(128, ((total + kFluctOwn - 1) / kFluctOwn + 31) / 32 * 32));
  if ((long long)threads * kFluctOwn < total) fail(SMCX_E_UNSUPPORTED, "K*M*M too large for the accumulator");
  k_fluct_accumulate<<<1, threads, MM * sizeof(double), st>>>(C, B, w, K, M, shell, z0, zs, N, acc, 0);
  check_cuda(cudaGetLastError(), "fluctuation accumulate launch");
}

// One accumulator per sample: sample r of C [R][K][M][M] into acc + r * (1 +
// MM + KMM + MM KMM), each with its own site count.
void fluct_launch_per_sample(const long long* C, long long R, int K, int M, int shell, int z0, int zs, double* acc,
                             cudaStream_t st) {
  const int MM = M * M, KMM = K * MM;
  const long long total = 1 + MM + KMM + (long long)MM * KMM;
  const int threads = std::min(1024, std::max(128, (int)((total + kFluctOwn - 1) / kFluctOwn + 31) / 32 * 32));
  if ((long long)threads * kFluctOwn < total) fail(SMCX_E_UNSUPPORTED, "K*M*M too large for the accumulator");
  if (R == 0) return;
  k_fluct_accumulate<<<(unsigned)R, threads, MM * sizeof(double), st>>>(C, R, nullptr, K, M, shell, z0, zs, 0.0, acc,
                                                                        total);
  check_cuda(cudaGetLastError(), "fluctuation accumulate launch");
}

extern "C" {

int smcx_fluct_accumulate(const int64_t* d_counts, int64_t B, const double* d_weights, int kind, int K, int M,
                          int shell, int64_t n_sites, double* d_acc, void* stream) {
  return guarded_call([&] {
    if (!d_counts || !d_acc || n_sites < 1 || B < 0) fail(SMCX_E_INVALID_ARG, "bad arguments");
    const Shells S = make_shells(kind, K);
    if (shell < 0 || shell >= K) fail(SMCX_E_INVALID_ARG, "shell out of range");
    if (B == 0) return;
    fluct_launch(reinterpret_cast<const long long*>(d_counts), B, d_weights, K, M, shell, S.z[0], S.z[shell],
                 (double)n_sites, d_acc, reinterpret_cast<cudaStream_t>(stream));
  });
}

int smcx_lattice_fluct_accumulate(smcx_lattice* h, int shell, double* d_acc) {
  return guarded_call([&] {
    if (!h || !d_acc) fail(SMCX_E_INVALID_ARG, "NULL argument");
    if (!h->have_epi) fail(SMCX_E_NO_EPI, "call smcx_set_epi first");
    if (shell < 0 || shell >= h->shells.K) fail(SMCX_E_INVALID_ARG, "shell out of range");
    pair_counts_device(h);
    fluct_launch(reinterpret_cast<const long long*>(h->d_counts), 1, nullptr, h->shells.K, h->M, shell,
                 h->shells.z[0], h->shells.z[shell], (double)h->N, d_acc, h->stream);
  });
}

int smcx_fluct_gradient(const double* d_acc, int K, int M, double T, double* d_grad, void* stream) {
  return guarded_call([&] {
    if (!d_acc || !d_grad || !(T > 0.0)) fail(SMCX_E_INVALID_ARG, "bad arguments");
    const int MM = M * M, KMM = K * MM;
    k_fluct_gradient<<<(MM * KMM + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        d_acc, MM, KMM, 1.0 / (kBoltzmannMeV * T), d_grad);
    check_cuda(cudaGetLastError(), "fluctuation gradient launch");
  });
}

}  // extern "C"
