// Local-energy field and clusters (Results, FeCoNiAlTi one-billion-atom
// section; Method "MC simulation": the local energy of every site is
// computed, an energy threshold decides which neighbouring sites belong to
// one set, and union-find collects the sets).
//
//  * e2[i] = 2 E_i = sum_k sum_{v in shell k} V_k[s_i][s_{i+v}] (Eq.
//    Linear_EPI without the bias terms, each bond counted at both ends, so
//    sum_i e2[i] = 2 E), plus 2 sum_k W_k[s_i] n_k(i)^2 under the qSRO model
//    (Eq. quadratic_local_SRO); one thread per cell, neighbours gathered from
//    the lattice store with periodic wrap.
//  * class(i) = e2[i] < thr2.  Two shell-1 neighbours of one class are in
//    one cluster.  Concurrent union-find over int32 parents: a root is only
//    ever linked below a smaller root with a compare-and-swap, so parents
//    decrease along every path, paths can be halved with plain stores, and
//    the final root of a cluster is its smallest site id (a unique label).
//    Parents are read with volatile loads (L2, coherent across SMs).  Every
//    find and union loop has an iteration limit that raises an error flag.
//  * Summary: cluster sizes by warp-aggregated atomics on the labels, the
//    clusters of at least min_size sites listed on the device, sorted on the
//    host, and species counts of the largest ones.
#include <algorithm>
#include <vector>

#include "smcx_device.cuh"

namespace smcx {

void fill_offsets_global(const smcx_lattice* hd, SweepParams& P);

namespace {

constexpr int kFindLimit = 1 << 22;
constexpr int kUnionLimit = 1 << 20;

// Half of shell 1 (first nonzero half-unit component positive), per centre
// sublattice: global (dx, dy, dz, b').
struct HalfShell {
  signed char d[4][8][4];
  int n;
};

__device__ __forceinline__ long long nb_gid(const SweepParams& P, int x, int y, int z, const signed char* d, int m) {
  return (((long long)wrap_add(z, d[2], P.n[2]) * P.n[1] + wrap_add(y, d[1], P.n[1])) * P.n[0] +
          wrap_add(x, d[0], P.n[0])) * m + d[3];
}

// qSRO weights W[k][c] (on = 0: pair model)
struct QsroWeights {
  int32_t w[kMaxShells * kMaxSweepM];
  int on;
};

template <int KIND, int K>
__global__ void __launch_bounds__(256) k_local_energy2(const SweepParams P, const int32_t* __restrict__ dV,
                                                       const QsroWeights QW, int32_t* e2, uint8_t* cls,
                                                       long long thr2) {
  constexpr int m = cell_sites(KIND);
  __shared__ int32_t sV[kMaxShells * kMaxSweepM * kMaxSweepM];
  __shared__ int32_t sW[kMaxShells * kMaxSweepM];
  const int M = P.M;
  for (int i = threadIdx.x; i < K * M * M; i += blockDim.x) sV[i] = dV[i];
  for (int i = threadIdx.x; i < K * M; i += blockDim.x) sW[i] = QW.on ? QW.w[i] : 0;
  __syncthreads();
  const long long ncell = (long long)P.n[0] * P.n[1] * P.n[2];
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % P.n[0]);
    const long long r = c / P.n[0];
    const int y = (int)(r % P.n[1]), z = (int)(r / P.n[1]);
    for (int b = 0; b < m; b++) {
      const int p = load_site(P.sites, c * m + b, P.storage);
      int acc = 0;
      int j = 0;
#pragma unroll
      for (int k = 0; k < K; k++) {
        const int32_t* row = sV + (k * M + p) * M;
        int n = 0;
#pragma unroll 4
        for (int q = 0; q < shell_size(KIND, k); q++, j++) {
          const int c = load_site(P.sites, nb_gid(P, x, y, z, P.gd[b][j], m), P.storage);
          acc += row[c];
          n += (c == p);
        }
        acc += 2 * sW[k * M + p] * n * n;  // qSRO term (W = 0 for the pair model)
      }
      if (e2) e2[c * m + b] = acc;
      if (cls) cls[c * m + b] = (uint8_t)((long long)acc < thr2);
    }
  }
}

__global__ void k_label_init(int32_t* lab, long long N) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    lab[i] = (int32_t)i;
}

__device__ __forceinline__ int find_root(int32_t* lab, int x, int* flag) {
  volatile int32_t* p = lab;
  for (int it = 0; it < kFindLimit; it++) {
    const int px = p[x];
    if (px == x) return x;
    const int gx = p[px];
    if (gx != px) p[x] = gx;  // halving: gx < px < x, still an ancestor
    x = gx;
  }
  atomicOr(flag, 1);
  return x;
}

__device__ __forceinline__ void unite(int32_t* lab, int a, int b, int* flag) {
  for (int it = 0; it < kUnionLimit; it++) {
    a = find_root(lab, a, flag);
    b = find_root(lab, b, flag);
    if (a == b) return;
    if (a < b) {
      const int t = a;
      a = b;
      b = t;
    }
    if (atomicCAS(&lab[a], a, b) == a) return;  // a was a root: now below b
  }
  atomicOr(flag, 2);
}

template <int KIND>
__global__ void __launch_bounds__(256) k_hook(const SweepParams P, const HalfShell H, const uint8_t* cls, int32_t* lab,
                                              int* flag) {
  constexpr int m = cell_sites(KIND);
  const long long ncell = (long long)P.n[0] * P.n[1] * P.n[2];
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % P.n[0]);
    const long long r = c / P.n[0];
    const int y = (int)(r % P.n[1]), z = (int)(r / P.n[1]);
#pragma unroll
    for (int b = 0; b < m; b++) {
      const long long i = c * m + b;
      const uint8_t ci = cls[i];
      for (int j = 0; j < H.n; j++) {
        const long long t = nb_gid(P, x, y, z, H.d[b][j], m);
        if (cls[t] == ci && t != i) unite(lab, (int)i, (int)t, flag);
      }
    }
    if (*(volatile int*)flag) return;
  }
}

// Root without writing: every pointer read is an ancestor, so the walk ends
// at the root whatever other threads write meanwhile, as long as they write
// ancestors too.
__device__ __forceinline__ int find_root_ro(const int32_t* lab, int x, int* flag) {
  const volatile int32_t* p = lab;
  for (int it = 0; it < kFindLimit; it++) {
    const int px = p[x];
    if (px == x) return x;
    x = px;
  }
  atomicOr(flag, 1);
  return x;
}

// Labels to roots in two launches.  The first shortens the paths (halving)
// and points every site at its root; a concurrent halving step elsewhere can
// still overwrite such a final write with an intermediate ancestor.  The
// second walks without halving, so every write is a root and stays one, and
// counts the roots.
template <bool FINAL>
__global__ void k_compress(int32_t* lab, long long N, int* flag, unsigned long long* n_roots) {
  unsigned long long roots = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int r = FINAL ? find_root_ro(lab, (int)i, flag) : find_root(lab, (int)i, flag);
    lab[i] = r;
    roots += (r == (int)i);
  }
  if (FINAL) {
    for (int o = 16; o > 0; o >>= 1) roots += __shfl_down_sync(0xffffffffu, roots, o);
    if ((threadIdx.x & 31) == 0 && roots) atomicAdd(n_roots, roots);
  }
}

// size[label]++ with one atomic per distinct label in a warp
__global__ void k_sizes(const int32_t* lab, long long N, int32_t* size) {
  for (long long i0 = (long long)blockIdx.x * blockDim.x; i0 < N; i0 += (long long)gridDim.x * blockDim.x) {
    const long long i = i0 + threadIdx.x;
    const bool ok = i < N;
    const int l = ok ? lab[i] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, l);
    if (ok && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&size[l], __popc(peers));
  }
}

__global__ void k_select(const int32_t* size, long long N, long long min_size, int32_t* out, long long cap,
                         unsigned long long* count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    if (size[i] > 0 && size[i] >= min_size) {
      const unsigned long long k = atomicAdd(count, 1ull);
      if ((long long)k < cap) out[k] = (int32_t)i;
    }
  }
}

__global__ void k_gather(const int32_t* src, const int32_t* idx, long long n, int32_t* out) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[j] = src[idx[j]];
}

__global__ void k_mark(const int32_t* roots, int n, int32_t* size) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) size[roots[j]] = -(j + 1);
}

__global__ void k_species(const int32_t* lab, const int32_t* size, const uint8_t* sites, int storage, long long N, int M,
                          unsigned long long* counts) {
  for (long long i0 = (long long)blockIdx.x * blockDim.x; i0 < N; i0 += (long long)gridDim.x * blockDim.x) {
    const long long i = i0 + threadIdx.x;
    int key = -1;
    if (i < N) {
      const int v = size[lab[i]];
      if (v < 0) key = (-v - 1) * M + load_site(sites, i, storage);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (key >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&counts[key], (unsigned long long)__popc(peers));
  }
}

int grid_for(long long work) {
  int dev = 0, nsm = 0;
  check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  check_cuda(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "SM count");
  return (int)std::max<long long>(1, std::min<long long>((work + 255) / 256, (long long)nsm * 16));
}

void setup_params(const smcx_lattice* hd, SweepParams& P) {
  memset(&P, 0, sizeof(P));
  P.sites = hd->d_sites;
  P.M = hd->M;
  P.storage = hd->storage;
  for (int a = 0; a < 3; a++) P.n[a] = hd->n[a];
  fill_offsets_global(hd, P);
}

void need_epi(const smcx_lattice* hd) {
  if (!hd->have_epi) fail(SMCX_E_NO_EPI, "smcx_set_epi first");
  // |2 E_i| <= sum_k z_k max |V_k|
  long long bound = 0;
  const int M = hd->M;
  for (int k = 0; k < hd->shells.K; k++) {
    long long vmax = 0;
    for (int i = 0; i < M * M; i++) vmax = std::max(vmax, std::llabs((long long)hd->V[k * M * M + i]));
    bound += vmax * hd->shells.z[k];
    if (!hd->Wq.empty()) {
      long long wmax = 0;
      for (int p = 0; p < M; p++) wmax = std::max(wmax, std::llabs((long long)hd->Wq[k * M + p]));
      bound += 2 * wmax * hd->shells.z[k] * hd->shells.z[k];
    }
  }
  if (bound > 2147483647ll) fail(SMCX_E_RANGE, "local energies do not fit int32 for this EPI table");
}

void launch_local_energy(smcx_lattice* hd, int32_t* e2, uint8_t* cls, long long thr2) {
  need_epi(hd);
  SweepParams P;
  setup_params(hd, P);
  // the plain V table sits after W[a][b][k][c] and X[a][b] in the device EPI table
  const int32_t* dV = hd->d_wtab + (size_t)hd->M * hd->M * hd->shells.K * hd->M + hd->M * hd->M;
  QsroWeights QW;
  memset(&QW, 0, sizeof(QW));
  QW.on = hd->Wq.empty() ? 0 : 1;
  for (size_t i = 0; i < hd->Wq.size(); i++) QW.w[i] = hd->Wq[i];
  const long long ncell = (long long)hd->n[0] * hd->n[1] * hd->n[2];
  const int grid = grid_for(ncell);
  const int K = hd->shells.K;
  auto go = [&](auto kern) { kern<<<grid, 256, 0, hd->stream>>>(P, dV, QW, e2, cls, thr2); };
  if (hd->kind == kBCC) {
    switch (K) {
      case 1: go(k_local_energy2<kBCC, 1>); break;
      case 2: go(k_local_energy2<kBCC, 2>); break;
      case 3: go(k_local_energy2<kBCC, 3>); break;
      default: go(k_local_energy2<kBCC, 4>); break;
    }
  } else {
    switch (K) {
      case 1: go(k_local_energy2<kFCC, 1>); break;
      case 2: go(k_local_energy2<kFCC, 2>); break;
      default: go(k_local_energy2<kFCC, 3>); break;
    }
  }
  check_cuda(cudaGetLastError(), "local energy launch");
}

HalfShell half_shell(const smcx_lattice* hd) {
  HalfShell H;
  memset(&H, 0, sizeof(H));
  const Shells& S = hd->shells;
  int n = 0;
  for (int j = 0; j < S.z[0]; j++) {
    const int* v = S.v[j];
    const bool half = v[0] > 0 || (v[0] == 0 && (v[1] > 0 || (v[1] == 0 && v[2] > 0)));
    if (!half) continue;
    for (int b = 0; b < hd->m; b++) {
      int B[3], d[3], r[3];
      basis_of(hd->kind, b, B);
      for (int a = 0; a < 3; a++) {
        const int p = B[a] + v[a];
        d[a] = (p >= 0) ? p / 2 : -((-p + 1) / 2);
        r[a] = p - 2 * d[a];
      }
      H.d[b][n][0] = (signed char)d[0];
      H.d[b][n][1] = (signed char)d[1];
      H.d[b][n][2] = (signed char)d[2];
      H.d[b][n][3] = (signed char)basis_index(hd->kind, r[0], r[1], r[2]);
    }
    n++;
  }
  H.n = n;
  return H;
}

template <typename T>
struct DevBuf {
  T* p = nullptr;
  explicit DevBuf(size_t n) { check_cuda(cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)), "cluster scratch"); }
  ~DevBuf() { cudaFree(p); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
};

}  // namespace

void local_energy_device(smcx_lattice* hd, int32_t* d_e2) { launch_local_energy(hd, d_e2, nullptr, 0); }

void clusters_device(smcx_lattice* hd, long long thr2, int32_t* d_lab, int64_t* n_clusters) {
  if (hd->N > 2147483647ll) fail(SMCX_E_RANGE, "cluster labels are int32: at most 2^31 - 1 sites");
  DevBuf<uint8_t> cls((size_t)hd->N);
  DevBuf<unsigned long long> roots(1);
  launch_local_energy(hd, nullptr, cls.p, thr2);
  const int grid = grid_for(hd->N);
  k_label_init<<<grid, 256, 0, hd->stream>>>(d_lab, hd->N);
  check_cuda(cudaMemsetAsync(hd->d_flag, 0, sizeof(int), hd->stream), "clear flag");
  check_cuda(cudaMemsetAsync(roots.p, 0, sizeof(unsigned long long), hd->stream), "clear root count");
  SweepParams P;
  setup_params(hd, P);
  const HalfShell H = half_shell(hd);
  const long long ncell = (long long)hd->n[0] * hd->n[1] * hd->n[2];
  if (hd->kind == kBCC)
    k_hook<kBCC><<<grid_for(ncell), 256, 0, hd->stream>>>(P, H, cls.p, d_lab, hd->d_flag);
  else
    k_hook<kFCC><<<grid_for(ncell), 256, 0, hd->stream>>>(P, H, cls.p, d_lab, hd->d_flag);
  k_compress<false><<<grid, 256, 0, hd->stream>>>(d_lab, hd->N, hd->d_flag, roots.p);
  k_compress<true><<<grid, 256, 0, hd->stream>>>(d_lab, hd->N, hd->d_flag, roots.p);
  check_cuda(cudaGetLastError(), "cluster launches");
  int flag = 0;
  unsigned long long nr = 0;
  check_cuda(cudaMemcpyAsync(&flag, hd->d_flag, sizeof(int), cudaMemcpyDeviceToHost, hd->stream), "flag download");
  check_cuda(cudaMemcpyAsync(&nr, roots.p, sizeof(nr), cudaMemcpyDeviceToHost, hd->stream), "root count download");
  check_cuda(cudaStreamSynchronize(hd->stream), "cluster sync");
  if (flag) fail(SMCX_E_TIMEOUT, "union-find exceeded its iteration limit");
  if (n_clusters) *n_clusters = (int64_t)nr;
}

void cluster_summary_device(smcx_lattice* hd, const int32_t* d_lab, long long min_size, int max_out, int64_t* roots,
                            int64_t* sizes, int64_t* counts, int* n_out) {
  if (hd->N > 2147483647ll) fail(SMCX_E_RANGE, "cluster labels are int32: at most 2^31 - 1 sites");
  const long long N = hd->N;
  const int grid = grid_for(N);
  DevBuf<int32_t> size((size_t)N);
  DevBuf<unsigned long long> cnt(1);
  check_cuda(cudaMemsetAsync(size.p, 0, (size_t)N * sizeof(int32_t), hd->stream), "clear sizes");
  check_cuda(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long), hd->stream), "clear count");
  k_sizes<<<grid, 256, 0, hd->stream>>>(d_lab, N, size.p);
  k_select<<<grid, 256, 0, hd->stream>>>(size.p, N, std::max(1ll, min_size), nullptr, 0, cnt.p);
  unsigned long long n_big = 0;
  check_cuda(cudaMemcpyAsync(&n_big, cnt.p, sizeof(n_big), cudaMemcpyDeviceToHost, hd->stream), "count download");
  check_cuda(cudaStreamSynchronize(hd->stream), "summary sync");
  if (n_big > (1ull << 26)) fail(SMCX_E_RANGE, "more than 2^26 clusters of min_size sites: raise min_size");
  DevBuf<int32_t> list((size_t)n_big);
  check_cuda(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long), hd->stream), "clear count");
  k_select<<<grid, 256, 0, hd->stream>>>(size.p, N, std::max(1ll, min_size), list.p, (long long)n_big, cnt.p);
  std::vector<int32_t> r(n_big), s(n_big);
  check_cuda(cudaMemcpyAsync(r.data(), list.p, n_big * sizeof(int32_t), cudaMemcpyDeviceToHost, hd->stream),
             "list download");
  check_cuda(cudaStreamSynchronize(hd->stream), "summary sync");
  // sizes of the listed roots, gathered on the device
  {
    DevBuf<int32_t> sz((size_t)n_big);
    if (n_big) {
      k_gather<<<(int)((n_big + 255) / 256), 256, 0, hd->stream>>>(size.p, list.p, (long long)n_big, sz.p);
      check_cuda(cudaMemcpyAsync(s.data(), sz.p, n_big * sizeof(int32_t), cudaMemcpyDeviceToHost, hd->stream),
                 "size download");
    }
    check_cuda(cudaStreamSynchronize(hd->stream), "summary sync");
  }
  std::vector<size_t> order(n_big);
  for (size_t j = 0; j < n_big; j++) order[j] = j;
  std::sort(order.begin(), order.end(), [&](size_t a, size_t b) { return s[a] != s[b] ? s[a] > s[b] : r[a] < r[b]; });
  const int n = (int)std::min<unsigned long long>(n_big, (unsigned long long)std::max(0, max_out));
  std::vector<int32_t> top(n);
  for (int j = 0; j < n; j++) {
    top[j] = r[order[j]];
    roots[j] = top[j];
    sizes[j] = s[order[j]];
  }
  *n_out = n;
  if (n == 0 || !counts) return;
  const int M = hd->M;
  DevBuf<int32_t> d_top((size_t)n);
  DevBuf<unsigned long long> d_counts((size_t)n * M);
  check_cuda(cudaMemcpyAsync(d_top.p, top.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, hd->stream),
             "top upload");
  check_cuda(cudaMemsetAsync(d_counts.p, 0, (size_t)n * M * sizeof(unsigned long long), hd->stream), "clear counts");
  k_mark<<<(n + 255) / 256, 256, 0, hd->stream>>>(d_top.p, n, size.p);
  k_species<<<grid, 256, 0, hd->stream>>>(d_lab, size.p, hd->d_sites, hd->storage, N, M, d_counts.p);
  check_cuda(cudaGetLastError(), "summary launches");
  std::vector<unsigned long long> h((size_t)n * M);
  check_cuda(cudaMemcpyAsync(h.data(), d_counts.p, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                             hd->stream),
             "counts download");
  check_cuda(cudaStreamSynchronize(hd->stream), "summary sync");
  for (size_t j = 0; j < h.size(); j++) counts[j] = (int64_t)h[j];
}

}  // namespace smcx

using namespace smcx;

extern "C" {

int smcx_local_energy(smcx_lattice* h, int32_t* d_e2) {
  return guarded_call([&] {
    if (!h || !d_e2) fail(SMCX_E_INVALID_ARG, "NULL argument");
    local_energy_device(h, d_e2);
  });
}

int smcx_clusters(smcx_lattice* h, int64_t thr2, int32_t* d_labels, int64_t* n_clusters) {
  return guarded_call([&] {
    if (!h || !d_labels) fail(SMCX_E_INVALID_ARG, "NULL argument");
    clusters_device(h, thr2, d_labels, n_clusters);
  });
}

int smcx_cluster_summary(smcx_lattice* h, const int32_t* d_labels, int64_t min_size, int max_out, int64_t* roots,
                         int64_t* sizes, int64_t* counts, int* n_out) {
  return guarded_call([&] {
    if (!h || !d_labels || !n_out || (max_out > 0 && (!roots || !sizes)))
      fail(SMCX_E_INVALID_ARG, "NULL argument");
    if (max_out < 0) fail(SMCX_E_INVALID_ARG, "max_out must be >= 0");
    cluster_summary_device(h, d_labels, min_size, max_out, roots, sizes, counts, n_out);
  });
}

}  // extern "C"
