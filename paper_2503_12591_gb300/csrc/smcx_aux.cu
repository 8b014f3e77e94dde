// Observables, initial configuration and host<->device configuration I/O.
//
//  * k_pair_counts: ordered pair counts C[k][p][q] over every site and shell
//    vector (the pair fractions of Method Eq. quadratic_local_SRO summed over
//    the lattice), privatised per CTA in shared memory, merged with 64-bit
//    atomics.  The energy E = 1/2 sum V C (Eq. Total_EPI, pair form) and the
//    Warren-Cowley SRO follow from C.
//  * initial configuration: 64-bit Philox key per site, stable radix sort of
//    (key, site id), species by rank at the exact composition.
#include <cub/device/device_radix_sort.cuh>

#include "smcx_device.cuh"

namespace smcx {

template <int KIND, int K>
__global__ void __launch_bounds__(256) k_pair_counts(const SweepParams P, unsigned long long* counts) {
  constexpr int m = cell_sites(KIND);
  extern __shared__ unsigned int hist[];
  const int M = P.M, KMM = K * P.M * P.M;
  for (int i = threadIdx.x; i < KMM; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
  const long long ncell = (long long)nx * ny * nz;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % nx);
    const long long r = c / nx;
    const int y = (int)(r % ny), z = (int)(r / ny);
#pragma unroll
    for (int b = 0; b < m; b++) {
      const int p = load_site(P.sites, c * m + b, P.storage);
      int j = 0;
#pragma unroll
      for (int k = 0; k < K; k++) {
#pragma unroll
        for (int q = 0; q < shell_size(KIND, k); q++, j++) {
          const signed char* d = P.gd[b][j];
          const long long t =
              (((long long)wrap_add(z, d[2], nz) * ny + wrap_add(y, d[1], ny)) * nx + wrap_add(x, d[0], nx)) * m +
              d[3];
          const int bin = (k * M + p) * M + load_site(P.sites, t, P.storage);
#ifdef SMCX_DEBUG
          if (!dbg::in_bounds(bin, KMM, kDbgPairHist)) continue;
#endif
          atomicAdd(&hist[bin], 1u);
        }
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < KMM; i += blockDim.x)
    if (hist[i]) atomicAdd(&counts[i], (unsigned long long)hist[i]);
}

// E = 1/2 sum_{k,p,q} V_k[p][q] C_k[p][q]; the sum over ordered pairs is even
// for a symmetric V, so E is exact.
__global__ void k_energy(const unsigned long long* C, const int32_t* V, int KMM, long long* E) {
  __shared__ long long part[32];
  long long s = 0;
  for (int i = threadIdx.x; i < KMM; i += blockDim.x) s += (long long)V[i] * (long long)C[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; w++) t += part[w];
    *E = t / 2;
  }
}

void fill_offsets_global(const smcx_lattice* hd, SweepParams& P);

template <int KIND, int K>
static void launch_counts(smcx_lattice* hd, const SweepParams& P) {
  const int KMM = K * hd->M * hd->M;
  int dev = 0, nsm = 0;
  check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  check_cuda(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "SM count");
  const long long ncell = (long long)hd->n[0] * hd->n[1] * hd->n[2];
  long long want = (ncell + 255) / 256;
  const int grid = (int)std::min<long long>(want, (long long)nsm * 8);
  k_pair_counts<KIND, K><<<grid, 256, KMM * sizeof(unsigned int), hd->stream>>>(P, hd->d_counts);
}

void pair_counts_device(smcx_lattice* hd) {
  SweepParams P;
  memset(&P, 0, sizeof(P));
  P.sites = hd->d_sites;
  P.M = hd->M;
  P.storage = hd->storage;
  for (int a = 0; a < 3; a++) P.n[a] = hd->n[a];
  fill_offsets_global(hd, P);
  const int KMM = hd->shells.K * hd->M * hd->M;
  check_cuda(cudaMemsetAsync(hd->d_counts, 0, KMM * sizeof(unsigned long long), hd->stream), "memset counts");
  int nt[3];
  if (hd->kernel_choice != SMCX_KERNEL_GENERIC && bcc_counts_usable(hd, nt)) {
    pair_counts_bcc_tiled(hd, nt);
    return;
  }
  const int K = hd->shells.K;
  if (hd->kind == kBCC) {
    switch (K) {
      case 1: launch_counts<kBCC, 1>(hd, P); break;
      case 2: launch_counts<kBCC, 2>(hd, P); break;
      case 3: launch_counts<kBCC, 3>(hd, P); break;
      case 4: launch_counts<kBCC, 4>(hd, P); break;
    }
  } else {
    switch (K) {
      case 1: launch_counts<kFCC, 1>(hd, P); break;
      case 2: launch_counts<kFCC, 2>(hd, P); break;
      case 3: launch_counts<kFCC, 3>(hd, P); break;
    }
  }
  check_cuda(cudaGetLastError(), "pair-count launch");
}

void energy_device(smcx_lattice* hd) {
  const int KMM = hd->shells.K * hd->M * hd->M;
  // device table layout: W[a][b][k][c] (M*M*K*M), X[a][b] (M*M), V[k][p][q]
  const int32_t* dV = hd->d_wtab + (size_t)hd->M * hd->M * hd->shells.K * hd->M + hd->M * hd->M;
  k_energy<<<1, 256, 0, hd->stream>>>(hd->d_counts, dV, KMM, hd->d_energy);
  check_cuda(cudaGetLastError(), "energy launch");
}

// Launchers on caller-provided buffers (used by the non-allocating entry point).
void pair_counts_raw(int kind, int K, const SweepParams& P, long long ncell, int KMM, unsigned long long* counts,
                     cudaStream_t st) {
  int dev = 0, nsm = 0;
  check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  check_cuda(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "SM count");
  const int grid = (int)std::min<long long>((ncell + 255) / 256, (long long)nsm * 8);
  const size_t sm = (size_t)KMM * sizeof(unsigned int);
  if (kind == kBCC) {
    switch (K) {
      case 1: k_pair_counts<kBCC, 1><<<grid, 256, sm, st>>>(P, counts); break;
      case 2: k_pair_counts<kBCC, 2><<<grid, 256, sm, st>>>(P, counts); break;
      case 3: k_pair_counts<kBCC, 3><<<grid, 256, sm, st>>>(P, counts); break;
      default: k_pair_counts<kBCC, 4><<<grid, 256, sm, st>>>(P, counts); break;
    }
  } else {
    switch (K) {
      case 1: k_pair_counts<kFCC, 1><<<grid, 256, sm, st>>>(P, counts); break;
      case 2: k_pair_counts<kFCC, 2><<<grid, 256, sm, st>>>(P, counts); break;
      default: k_pair_counts<kFCC, 3><<<grid, 256, sm, st>>>(P, counts); break;
    }
  }
  check_cuda(cudaGetLastError(), "pair-count launch");
}

void energy_raw(const unsigned long long* C, const int32_t* V, int KMM, long long* E, cudaStream_t st) {
  k_energy<<<1, 256, 0, st>>>(C, V, KMM, E);
  check_cuda(cudaGetLastError(), "energy launch");
}

// ---------------------------------------------------------------------------
// Initial configuration.
// ---------------------------------------------------------------------------
__global__ void k_init_keys(unsigned long long* keys, uint32_t* ids, long long N, uint32_t s_lo, uint32_t s_hi) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)((unsigned long long)i >> 32), 0u, 0x80000000u),
                                  make_uint2(s_lo, s_hi));
    keys[i] = ((unsigned long long)r.x << 32) | r.y;
    ids[i] = (uint32_t)i;
  }
}

struct Prefix {
  long long end[16];  // end[p] = first rank after species p
};

__global__ void k_assign(const uint32_t* ids, long long N, Prefix pf, int M, uint8_t* sites, int storage) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < N; r += (long long)gridDim.x * blockDim.x) {
    int p = 0;
    while (p < M - 1 && r >= pf.end[p]) p++;
    const uint32_t i = ids[r];
    if (storage == SMCX_INT8) {
      sites[i] = (uint8_t)p;
    } else {
      unsigned int* w = reinterpret_cast<unsigned int*>(sites) + (i >> 3);
      atomicOr(w, (unsigned int)p << (4 * (i & 7)));
    }
  }
}

void init_config_device(smcx_lattice* hd, const double* comp, uint64_t seed) {
  const long long N = hd->N;
  if (N > 0xFFFFFFFFll) fail(SMCX_E_UNSUPPORTED, "initial placement supports up to 2^32-1 sites");
  int64_t counts[16];
  species_counts(hd->M, comp, N, counts);
  Prefix pf;
  long long acc = 0;
  for (int p = 0; p < 16; p++) {
    acc += (p < hd->M) ? counts[p] : 0;
    pf.end[p] = acc;
  }
  cudaStream_t st = hd->stream;
  unsigned long long *k_in = nullptr, *k_out = nullptr;
  uint32_t *v_in = nullptr, *v_out = nullptr;
  void* temp = nullptr;
  size_t temp_bytes = 0;
  auto cleanup = [&]() {
    cudaFree(k_in);
    cudaFree(k_out);
    cudaFree(v_in);
    cudaFree(v_out);
    cudaFree(temp);
  };
  try {
    check_cuda(cudaMalloc(&k_in, N * 8), "init keys");
    check_cuda(cudaMalloc(&k_out, N * 8), "init keys");
    check_cuda(cudaMalloc(&v_in, N * 4), "init ids");
    check_cuda(cudaMalloc(&v_out, N * 4), "init ids");
    check_cuda(cub::DeviceRadixSort::SortPairs(nullptr, temp_bytes, k_in, k_out, v_in, v_out, (long long)N, 0, 64, st),
               "radix sort sizing");
    check_cuda(cudaMalloc(&temp, temp_bytes), "radix sort temp");
    k_init_keys<<<1024, 256, 0, st>>>(k_in, v_in, N, (uint32_t)seed, (uint32_t)(seed >> 32));
    check_cuda(cudaGetLastError(), "init keys launch");
    check_cuda(cub::DeviceRadixSort::SortPairs(temp, temp_bytes, k_in, k_out, v_in, v_out, (long long)N, 0, 64, st),
               "radix sort");
    check_cuda(cudaMemsetAsync(hd->d_sites, 0, hd->site_bytes, st), "clear sites");
    k_assign<<<1024, 256, 0, st>>>(v_out, N, pf, hd->M, hd->d_sites, hd->storage);
    check_cuda(cudaGetLastError(), "assign launch");
    check_cuda(cudaStreamSynchronize(st), "init sync");
  } catch (...) {
    cleanup();
    throw;
  }
  cleanup();
}

// ---------------------------------------------------------------------------
// Configuration I/O between int8 staging buffers and the lattice store.
// `first` is even for PACKED4 so each thread owns whole bytes.
// ---------------------------------------------------------------------------
__global__ void k_validate(const int8_t* ids, long long count, int M, int* flag) {
  int bad = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const int v = ids[i];
    bad |= (v < 0 || v >= M);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

__global__ void k_pack(const int8_t* ids, long long first, long long count, uint8_t* sites, int storage) {
  if (storage == SMCX_INT8) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
      sites[first + i] = (uint8_t)ids[i];
  } else {
    const long long nb = (count + 1) / 2;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nb;
         q += (long long)gridDim.x * blockDim.x) {
      const int lo = ids[2 * q];
      const int hi = (2 * q + 1 < count) ? ids[2 * q + 1] : 0;
      sites[(first >> 1) + q] = (uint8_t)((lo & 15) | ((hi & 15) << 4));
    }
  }
}

__global__ void k_unpack(const uint8_t* sites, long long first, long long count, int8_t* ids, int storage) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    ids[i] = (int8_t)load_site(sites, first + i, storage);
}

__global__ void k_validate_store(const uint8_t* sites, long long count, int storage, int M, int* flag) {
  int bad = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    bad |= (load_site(sites, i, storage) >= M);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

void validate_store(smcx_lattice* hd) { validate_store_at(hd, hd->d_sites); }

// E_i = E_0 + (accepted dE sum now) - (accepted dE sum at the start): one
// thread, enqueued after each sweep of smcx_sweep_energies.
__global__ void k_record_energy(const long long* E0, const unsigned long long* stats, const long long* dsum0,
                                long long* out) {
  *out = *E0 + (long long)stats[3] - *dsum0;
}

void record_energy(smcx_lattice* hd, const long long* d_dsum0, long long* d_out) {
  k_record_energy<<<1, 1, 0, hd->stream>>>(hd->d_energy, hd->d_stats, d_dsum0, d_out);
  check_cuda(cudaGetLastError(), "energy record launch");
}

// FP64 moments of a recorded energy trace and the specific heat from its
// fluctuation (Results, Fig. C_V; Method "MC simulation"):
// C_V / (N k_B) = Var(E) / (N (k_B T)^2), E converted from 0.01 meV to meV.
// One CTA, two passes over the trace (mean, then mean squared deviation),
// each a strided per-thread sum and a block reduction.
__device__ double block_sum(double v, double* part) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += part[w];
  return t;
}

__global__ void __launch_bounds__(512) k_energy_moments(const long long* E, long long n, long long N, double T,
                                                        double* out) {
  __shared__ double part[16];
  __shared__ double s_mean;
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) s += (double)E[i];
  s = block_sum(s, part);
  if (threadIdx.x == 0) s_mean = s / (double)n;
  __syncthreads();
  const double mean = s_mean;
  double q = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const double d = (double)E[i] - mean;
    q += d * d;
  }
  q = block_sum(q, part);
  if (threadIdx.x == 0) {
    const double var = q / (double)n;
    const double kT = kBoltzmannMeV * T;
    out[0] = mean;
    out[1] = var;
    out[2] = var * 1e-4 / ((double)N * kT * kT);
  }
}

void energy_moments(smcx_lattice* hd, const long long* d_E, long long n, double T, double* d_out) {
  k_energy_moments<<<1, 512, 0, hd->stream>>>(d_E, n, hd->N, T, d_out);
  check_cuda(cudaGetLastError(), "energy moments launch");
}

void validate_store_at(smcx_lattice* hd, const uint8_t* d_store) {
  k_validate_store<<<1024, 256, 0, hd->stream>>>(d_store, hd->N, hd->storage, hd->M, hd->d_flag);
  check_cuda(cudaGetLastError(), "validate launch");
}

void validate_int8(smcx_lattice* hd, const int8_t* d_ids, int64_t count) {
  k_validate<<<1024, 256, 0, hd->stream>>>(d_ids, count, hd->M, hd->d_flag);
  check_cuda(cudaGetLastError(), "validate launch");
}

void pack_from_int8(smcx_lattice* hd, const int8_t* d_ids, int64_t first, int64_t count) {
  k_pack<<<1024, 256, 0, hd->stream>>>(d_ids, first, count, hd->d_sites, hd->storage);
  check_cuda(cudaGetLastError(), "pack launch");
}

void unpack_to_int8(smcx_lattice* hd, int8_t* d_ids, int64_t first, int64_t count) {
  k_unpack<<<1024, 256, 0, hd->stream>>>(hd->d_sites, first, count, d_ids, hd->storage);
  check_cuda(cudaGetLastError(), "unpack launch");
}

// neighbour deltas (cell dx, dy, dz and target sublattice) for the global-
// memory kernels
void fill_offsets_global(const smcx_lattice* hd, SweepParams& P) {
  const Shells& S = hd->shells;
  for (int b = 0; b < hd->m; b++) {
    int B[3];
    basis_of(hd->kind, b, B);
    for (int j = 0; j < S.nv; j++) {
      int d[3], r[3];
      for (int a = 0; a < 3; a++) {
        int p = B[a] + S.v[j][a];
        d[a] = (p >= 0) ? p / 2 : -((-p + 1) / 2);
        r[a] = p - 2 * d[a];
      }
      P.gd[b][j][0] = (signed char)d[0];
      P.gd[b][j][1] = (signed char)d[1];
      P.gd[b][j][2] = (signed char)d[2];
      P.gd[b][j][3] = (signed char)basis_index(hd->kind, r[0], r[1], r[2]);
    }
  }
}

}  // namespace smcx
