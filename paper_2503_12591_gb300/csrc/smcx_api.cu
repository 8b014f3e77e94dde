// C ABI entry points (include/smcx.h).  Every entry point converts internal
// failures into an SMCX_E_* status and a per-thread message.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "smcx_internal.h"

using namespace smcx;

namespace {

template <class F>
int guarded(F&& f) {
  try {
    set_error("");
    f();
    return SMCX_OK;
  } catch (const SmcxException& e) {
    set_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return SMCX_E_OOM;
  } catch (const std::exception& e) {
    set_error(e.what());
    return SMCX_E_INVALID_ARG;
  } catch (...) {
    set_error("unknown failure");
    return SMCX_E_INVALID_ARG;
  }
}

void need(bool ok, int code, const char* msg) {
  if (!ok) fail(code, msg);
}

int kind_max_shells(int kind) { return kind == kBCC ? 4 : 3; }

void release(smcx_lattice* h) {
  if (h->owns_sites) cudaFree(h->d_sites);
  cudaFree(h->d_stats);
  cudaFree(h->d_counts);
  cudaFree(h->d_energy);
  cudaFree(h->d_thr);
  cudaFree(h->d_wtab);
  cudaFree(h->d_flag);
  cudaFree(h->d_stage);
  cudaFree(h->d_qcnt);
}

// One int8 id per site, allocated on first configuration transfer and kept.
void ensure_stage(smcx_lattice* h) {
  if (!h->d_stage) {
    check_cuda(cudaMalloc(&h->d_stage, (size_t)h->N), "staging buffer");
    h->stage_bytes = (size_t)h->N;
  }
}

// Shells against which a schedule is validated: the EPI's, or before
// set_epi the largest shell count this lattice kind supports.
Shells sched_shells(const smcx_lattice* h) {
  return h->have_epi ? h->shells : make_shells(h->kind, kind_max_shells(h->kind));
}

// An explicit schedule must be valid; the library's choice may be "none"
// (L = 0) for lattices too small for any checkerboard: such a handle can be
// created, read and written, but smcx_sweep returns SMCX_E_SCHEDULE.
void apply_schedule(smcx_lattice* h, const smcx_sched* s) {
  Shells S = sched_shells(h);
  smcx_sched sc;
  if (s == nullptr || s->L == 0) {
    sc = choose_schedule(S, h->n);
    h->sched_auto = true;
  } else {
    sc = *s;
    h->sched_auto = false;
    std::string why = schedule_problem(S, h->n, sc);
    if (!why.empty()) fail(SMCX_E_SCHEDULE, "schedule rejected: " + why);
  }
  h->sched = sc;
}

void upload_thresholds(smcx_lattice* h, double T) {
  if (T == h->thr_T) return;
  std::vector<uint32_t> tab(kNA + kNB);
  int nA = 0;
  threshold_tables(T, tab.data(), &nA, tab.data() + kNA);
  // pageable source: the copy is staged before cudaMemcpyAsync returns
  check_cuda(cudaMemcpyAsync(h->d_thr, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, h->stream),
             "threshold upload");
  check_cuda(cudaStreamSynchronize(h->stream), "threshold upload sync");
  h->thr_T = T;
  h->thr_nA = nA;
}

}  // namespace

#include <nvtx3/nvToolsExt.h>

namespace smcx {

// Debug build: host readers of the per-translation-unit status words (see
// smcx_device.cuh); registered by static initialisers when the library loads.
namespace dbg {
static std::vector<int (*)(unsigned long long*)>& readers() {
  static std::vector<int (*)(unsigned long long*)> r;
  return r;
}
int register_reader(int (*reader)(unsigned long long*)) {
  readers().push_back(reader);
  return (int)readers().size();
}
}  // namespace dbg

NvtxRange::NvtxRange(const char* name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }
void upload_thresholds_for(smcx_lattice* h, double T) { upload_thresholds(h, T); }
}  // namespace smcx

extern "C" {

const char* smcx_last_error(void) { return last_error().c_str(); }

int smcx_version(void) { return 10000; }

int smcx_threshold_tables(double T, uint32_t* A, int* nA, uint32_t* B) {
  return guarded([&] {
    need(A && nA && B, SMCX_E_INVALID_ARG, "NULL output");
    need(T > 0.0, SMCX_E_INVALID_ARG, "temperature must be > 0");
    threshold_tables(T, A, nA, B);
  });
}

// Geometry, schedule and every buffer except the lattice store.
static void setup_handle(smcx_lattice* h, int kind, int nx, int ny, int nz, int M, int storage,
                         const smcx_sched* sched, void* stream) {
  h->kind = kind;
  h->m = sites_per_cell(kind);
  h->M = M;
  h->storage = storage;
  h->n[0] = nx;
  h->n[1] = ny;
  h->n[2] = nz;
  h->N = (int64_t)nx * ny * nz * h->m;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  apply_schedule(h, sched);
  int dev_count = 0;
  check_cuda(cudaGetDeviceCount(&dev_count), "no CUDA device");
  check_cuda(cudaMalloc(&h->d_stats, 4 * sizeof(unsigned long long)), "stats");  // trials, accepts, same, sum dE
  check_cuda(cudaMalloc(&h->d_counts, (size_t)kMaxShells * M * M * sizeof(unsigned long long)), "counts");
  check_cuda(cudaMalloc(&h->d_energy, sizeof(long long)), "energy");
  check_cuda(cudaMalloc(&h->d_thr, (kNA + kNB) * sizeof(uint32_t)), "threshold table");
  const size_t nw = (size_t)M * M * kMaxShells * M + (size_t)M * M + (size_t)kMaxShells * M * M;
  check_cuda(cudaMalloc(&h->d_wtab, nw * sizeof(int32_t)), "EPI table");
  check_cuda(cudaMalloc(&h->d_flag, sizeof(int)), "flag");
  check_cuda(cudaMemsetAsync(h->d_stats, 0, 4 * sizeof(unsigned long long), h->stream), "clear stats");
  check_cuda(cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream), "clear flag");
}

static void check_create_args(smcx_lattice** out, int kind, int nx, int ny, int nz, int M, int storage) {
  need(out != nullptr, SMCX_E_INVALID_ARG, "NULL handle pointer");
  *out = nullptr;
  need(kind == kBCC || kind == kFCC, SMCX_E_INVALID_ARG, "kind must be SMCX_BCC or SMCX_FCC");
  need(nx >= 1 && ny >= 1 && nz >= 1, SMCX_E_INVALID_ARG, "dimensions must be >= 1");
  need(storage == SMCX_INT8 || storage == SMCX_PACKED4, SMCX_E_INVALID_ARG, "unknown storage");
  need(M >= 1 && M <= (storage == SMCX_PACKED4 ? 15 : 127), SMCX_E_INVALID_ARG,
       "species count out of range for the storage");
}

int smcx_lattice_create(smcx_lattice** out, int kind, int nx, int ny, int nz, int M, const double* comp,
                        uint64_t init_seed, int storage, const smcx_sched* sched, void* stream) {
  return guarded([&] {
    check_create_args(out, kind, nx, ny, nz, M, storage);
    need(comp != nullptr, SMCX_E_INVALID_ARG, "NULL composition");
    smcx_lattice* h = new smcx_lattice();
    try {
      setup_handle(h, kind, nx, ny, nz, M, storage, sched, stream);
      h->site_bytes = (size_t)(storage == SMCX_INT8 ? h->N : (h->N + 1) / 2);
      h->site_bytes = (h->site_bytes + 15) & ~(size_t)15;
      check_cuda(cudaMalloc(&h->d_sites, h->site_bytes), "lattice store");
      init_config_device(h, comp, init_seed);
    } catch (...) {
      release(h);
      delete h;
      throw;
    }
    *out = h;
  });
}

int smcx_lattice_wrap(smcx_lattice** out, int kind, int nx, int ny, int nz, int M, void* d_sites, size_t bytes,
                      int storage, const smcx_sched* sched, void* stream) {
  return guarded([&] {
    check_create_args(out, kind, nx, ny, nz, M, storage);
    need(d_sites != nullptr, SMCX_E_INVALID_ARG, "NULL lattice store");
    cudaPointerAttributes attr;
    check_cuda(cudaPointerGetAttributes(&attr, d_sites), "pointer attributes");
    need(attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged, SMCX_E_INVALID_ARG,
         "lattice store is not device memory");
    need(reinterpret_cast<uintptr_t>(d_sites) % 16 == 0, SMCX_E_INVALID_ARG,
         "lattice store must be 16-byte aligned");
    smcx_lattice* h = new smcx_lattice();
    try {
      h->owns_sites = false;
      h->d_sites = static_cast<uint8_t*>(d_sites);
      setup_handle(h, kind, nx, ny, nz, M, storage, sched, stream);
      h->site_bytes = (size_t)(storage == SMCX_INT8 ? h->N : (h->N + 1) / 2);
      need(bytes >= h->site_bytes, SMCX_E_INVALID_ARG, "lattice store smaller than the lattice");
      validate_store(h);
      int flag = 0;
      check_cuda(cudaMemcpyAsync(&flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "flag download");
      check_cuda(cudaStreamSynchronize(h->stream), "validate sync");
      need(flag == 0, SMCX_E_INVALID_ARG, "lattice store holds species ids outside 0..M-1");
    } catch (...) {
      release(h);
      delete h;
      throw;
    }
    *out = h;
  });
}

int smcx_lattice_destroy(smcx_lattice* h) {
  if (!h) return SMCX_OK;
  return guarded([&] {
    cudaStreamSynchronize(h->stream);
    release(h);
    delete h;
  });
}

int smcx_set_epi(smcx_lattice* h, int K, const int32_t* V) {
  return guarded([&] {
    need(h && V, SMCX_E_INVALID_ARG, "NULL argument");
    need(K >= 1 && K <= kind_max_shells(h->kind), SMCX_E_INVALID_ARG, "shell count out of range");
    const int M = h->M;
    need(M <= kMaxSweepM, SMCX_E_UNSUPPORTED, "sweep kernels of this library run at most 8 species");
    for (int k = 0; k < K; k++)
      for (int p = 0; p < M; p++)
        for (int q = 0; q < M; q++)
          need(V[(k * M + p) * M + q] == V[(k * M + q) * M + p], SMCX_E_INVALID_ARG, "EPI table is not symmetric");
    Shells S = make_shells(h->kind, K);
    check_reach(S, h->n);
    // largest |dE|: every neighbour of both sites changes by at most the
    // largest species difference of its shell, plus the s-s' bond term
    long long bound = 0;
    for (int k = 0; k < K; k++) {
      long long dmax = 0;
      for (int a = 0; a < M; a++)
        for (int b = 0; b < M; b++)
          for (int c = 0; c < M; c++)
            dmax = std::max(dmax, std::llabs((long long)V[(k * M + b) * M + c] - V[(k * M + a) * M + c]));
      bound += 2LL * S.z[k] * dmax;
    }
    long long vmax = 0;
    for (int i = 0; i < K * M * M; i++) vmax = std::max(vmax, std::llabs((long long)V[i]));
    bound += 4 * vmax;
    need(bound < (1LL << 31) - 1, SMCX_E_RANGE, "EPI values too large: |dE| could overflow int32");
    // the schedule must still separate trials for the new reach
    smcx_sched sc = h->sched_auto ? choose_schedule(S, h->n) : h->sched;
    if (sc.L != 0) {
      std::string why = schedule_problem(S, h->n, sc);
      if (!why.empty()) fail(SMCX_E_SCHEDULE, "schedule too small for this EPI: " + why);
    }
    // device table: W[a][b][k][c] = V_k[b][c] - V_k[a][c]; X[a][b]; V
    std::vector<int32_t> tab((size_t)M * M * K * M + M * M + (size_t)K * M * M);
    size_t o = 0;
    for (int a = 0; a < M; a++)
      for (int b = 0; b < M; b++)
        for (int k = 0; k < K; k++)
          for (int c = 0; c < M; c++) tab[o++] = V[(k * M + b) * M + c] - V[(k * M + a) * M + c];
    for (int a = 0; a < M; a++)
      for (int b = 0; b < M; b++) tab[o++] = 2 * V[(0 * M + a) * M + b] - V[a * M + a] - V[b * M + b];
    for (int i = 0; i < K * M * M; i++) tab[o++] = V[i];
    check_cuda(cudaMemcpyAsync(h->d_wtab, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, h->stream),
               "EPI upload");
    check_cuda(cudaStreamSynchronize(h->stream), "EPI upload sync");
    h->V.assign(V, V + (size_t)K * M * M);
    h->Wq.clear();  // a new pair table returns the handle to the pair model
    h->shells = S;
    h->sched = sc;
    h->have_epi = true;
  });
}

int smcx_set_qsro(smcx_lattice* h, const int32_t* W) {
  return guarded([&] {
    need(h != nullptr, SMCX_E_INVALID_ARG, "NULL handle");
    need(h->have_epi, SMCX_E_NO_EPI, "call smcx_set_epi first");
    Shells S = h->shells;
    const int K = S.K, M = h->M;
    if (W == nullptr) {
      S.model = 0;
    } else {
      S.model = 1;
      // |dE| bound: the pair part (checked by smcx_set_epi) plus, for s and
      // s', their whole quadratic terms, and for every other site of the two
      // environments at most two shells changing by one neighbour
      long long pair = 0, q = 0, vmax = 0;
      for (int k = 0; k < K; k++) {
        long long dmax = 0, wmax = 0;
        for (int a = 0; a < M; a++)
          for (int b = 0; b < M; b++)
            for (int c = 0; c < M; c++)
              dmax = std::max(dmax, std::llabs((long long)h->V[(k * M + b) * M + c] - h->V[(k * M + a) * M + c]));
        for (int p = 0; p < M; p++) wmax = std::max(wmax, std::llabs((long long)W[k * M + p]));
        pair += 2LL * S.z[k] * dmax;
        q += 4 * wmax * S.z[k] * S.z[k] + 2LL * S.nv * 2 * wmax * (2 * S.z[k] + 1);
      }
      for (int i = 0; i < K * M * M; i++) vmax = std::max(vmax, std::llabs((long long)h->V[i]));
      need(pair + 4 * vmax + q < (1LL << 31) - 1, SMCX_E_RANGE, "qSRO weights too large: |dE| could overflow int32");
    }
    smcx_sched sc = h->sched_auto ? choose_schedule(S, h->n) : h->sched;
    if (sc.L != 0) {
      std::string why = schedule_problem(S, h->n, sc);
      if (!why.empty()) fail(SMCX_E_SCHEDULE, "schedule too small for this model: " + why);
    }
    if (W == nullptr) h->Wq.clear();
    else h->Wq.assign(W, W + (size_t)K * M);
    h->shells = S;
    h->sched = sc;
  });
}

int smcx_set_kernel(smcx_lattice* h, int which) {
  return guarded([&] {
    need(h != nullptr, SMCX_E_INVALID_ARG, "NULL handle");
    need(which == SMCX_KERNEL_AUTO || which == SMCX_KERNEL_GENERIC, SMCX_E_INVALID_ARG, "unknown kernel family");
    h->kernel_choice = which;
  });
}

int smcx_set_replica(smcx_lattice* h, int replica) {
  return guarded([&] {
    need(h != nullptr, SMCX_E_INVALID_ARG, "NULL handle");
    need(replica >= 0 && replica < 65536, SMCX_E_INVALID_ARG, "replica id must be in 0..65535");
    h->replica = replica;
  });
}

int smcx_set_proposal(smcx_lattice* h, int mode) {
  return guarded([&] {
    need(h != nullptr, SMCX_E_INVALID_ARG, "NULL handle");
    need(mode == SMCX_PROPOSAL_SITE || mode == SMCX_PROPOSAL_TILE || mode == SMCX_PROPOSAL_BLOCK,
         SMCX_E_INVALID_ARG, "unknown proposal mode");
    h->proposal = mode;
  });
}

int smcx_set_block(smcx_lattice* h, int threads) {
  return guarded([&] {
    need(h != nullptr, SMCX_E_INVALID_ARG, "NULL handle");
    need(threads == 0 || (threads >= 32 && threads <= 512 && threads % 32 == 0), SMCX_E_INVALID_ARG,
         "threads must be 0 or a multiple of 32 in 32..512");
    h->bcc_threads = threads;
  });
}

int smcx_set_schedule(smcx_lattice* h, const smcx_sched* sched) {
  return guarded([&] {
    need(h != nullptr, SMCX_E_INVALID_ARG, "NULL handle");
    apply_schedule(h, sched);
  });
}

int smcx_get_schedule(const smcx_lattice* h, smcx_sched* out) {
  return guarded([&] {
    need(h && out, SMCX_E_INVALID_ARG, "NULL argument");
    *out = h->sched;
  });
}

int smcx_sweep(smcx_lattice* h, double T, int64_t n_sweeps, uint64_t seed) {
  NvtxRange nvtx_range("smcx_sweep");
  return guarded([&] {
    need(h != nullptr, SMCX_E_INVALID_ARG, "NULL handle");
    need(h->have_epi, SMCX_E_NO_EPI, "call smcx_set_epi before smcx_sweep");
    need(h->sched.L != 0, SMCX_E_SCHEDULE, "no checkerboard schedule fits this lattice");
    need(T > 0.0 && isfinite(T), SMCX_E_INVALID_ARG, "temperature must be finite and > 0");
    need(n_sweeps >= 0, SMCX_E_INVALID_ARG, "negative sweep count");
    need(h->sweep_cum + (uint64_t)n_sweeps < (1ull << 63), SMCX_E_INVALID_ARG, "sweep counter overflow");
    if (n_sweeps == 0) return;
    upload_thresholds(h, T);
    sweep_device(h, h->thr_nA, seed, n_sweeps);
    h->sweep_cum += (uint64_t)n_sweeps;
  });
}

// Times `trial` sweeps for every candidate schedule (link cell from the
// model's minimum to 5, tiles of about 10..20 cells) and, for the BCC tile
// kernel, block size, on a snapshot of the configuration; restores the
// configuration, statistics and sweep counter and installs the fastest.
int smcx_autotune(smcx_lattice* h, double T, int trial, smcx_sched* out, int* threads) {
  NvtxRange nvtx_range("smcx_autotune");
  return guarded([&] {
    need(h != nullptr, SMCX_E_INVALID_ARG, "NULL handle");
    need(h->have_epi, SMCX_E_NO_EPI, "call smcx_set_epi first");
    need(T > 0.0 && isfinite(T), SMCX_E_INVALID_ARG, "temperature must be finite and > 0");
    need(trial >= 1 && trial <= 64, SMCX_E_INVALID_ARG, "trial sweeps must be 1..64");
    uint8_t* d_copy = nullptr;
    check_cuda(cudaMalloc(&d_copy, h->site_bytes), "autotune snapshot");
    unsigned long long st[4];
    check_cuda(cudaMemcpyAsync(d_copy, h->d_sites, h->site_bytes, cudaMemcpyDeviceToDevice, h->stream),
               "autotune snapshot copy");
    check_cuda(cudaMemcpyAsync(st, h->d_stats, sizeof(st), cudaMemcpyDeviceToHost, h->stream), "stats snapshot");
    check_cuda(cudaStreamSynchronize(h->stream), "autotune snapshot sync");
    const smcx_sched sched0 = h->sched;
    const bool auto0 = h->sched_auto;
    const int threads0 = h->bcc_threads;
    const uint64_t sweep0 = h->sweep_cum;
    double best = 1e300;
    smcx_sched best_sc = sched0;
    int best_th = threads0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    // put back the configuration, statistics and settings whatever happens
    auto restore = [&]() {
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      cudaMemcpyAsync(h->d_sites, d_copy, h->site_bytes, cudaMemcpyDeviceToDevice, h->stream);
      cudaMemcpyAsync(h->d_stats, st, sizeof(st), cudaMemcpyHostToDevice, h->stream);
      cudaStreamSynchronize(h->stream);
      cudaFree(d_copy);
      h->sweep_cum = sweep0;
      h->sched = sched0;
      h->sched_auto = auto0;
      h->bcc_threads = threads0;
    };
    try {
      upload_thresholds(h, T);
      check_cuda(cudaEventCreate(&e0), "event");
      check_cuda(cudaEventCreate(&e1), "event");
      const int Lmin = min_link_cell(h->shells);
      for (int L = Lmin; L <= std::max(Lmin, 5); L++)
        for (int target : {10, 12, 14, 15, 16, 18, 19, 20})
          for (int th : {0, 128, 256}) {
            smcx_sched sc;
            sc.L = L;
            for (int a = 0; a < 3; a++) {
              int nt = 2;
              while ((h->n[a] + nt - 1) / nt > target) nt += 2;
              sc.nt[a] = nt;
            }
            if (!schedule_problem(h->shells, h->n, sc).empty()) continue;
            h->sched = sc;
            h->bcc_threads = th;
            const bool fast = h->kernel_choice != 1 && h->Wq.empty() && bcc_fast_usable(h);
            if (th != 0 && !fast) continue;  // block size only matters to the BCC tile kernel
            float ms = 0;
            try {
              sweep_device(h, h->thr_nA, 0x5eedull, 1);
              check_cuda(cudaEventRecord(e0, h->stream), "event");
              sweep_device(h, h->thr_nA, 0x5eedull, trial);
              check_cuda(cudaEventRecord(e1, h->stream), "event");
              check_cuda(cudaEventSynchronize(e1), "event sync");
              check_cuda(cudaEventElapsedTime(&ms, e0, e1), "event time");
            } catch (const SmcxException&) {
              continue;
            }
            if (ms < best) {
              best = ms;
              best_sc = sc;
              best_th = th;
            }
          }
    } catch (...) {
      restore();
      throw;
    }
    restore();
    if (best >= 1e300) fail(SMCX_E_SCHEDULE, "no autotuner candidate fits this lattice");
    h->sched = best_sc;
    h->sched_auto = false;
    h->bcc_threads = best_th;
    if (out) *out = best_sc;
    if (threads) *threads = best_th;
  });
}

// n_sweeps sweeps at T with the exact energy after each one recorded on the
// device; then optionally the trace (E, host) and its FP64 moments and
// specific heat (moments, host [3]).
static void sweep_recorded(smcx_lattice* h, double T, int64_t n_sweeps, uint64_t seed, int64_t* E,
                           double* moments, const char* who) {
  need(h != nullptr, SMCX_E_INVALID_ARG, "NULL handle");
  need(h->have_epi, SMCX_E_NO_EPI, (std::string("call smcx_set_epi before ") + who).c_str());
  need(h->sched.L != 0, SMCX_E_SCHEDULE, "no checkerboard schedule fits this lattice");
  need(T > 0.0 && isfinite(T), SMCX_E_INVALID_ARG, "temperature must be finite and > 0");
  need(n_sweeps >= 0 && n_sweeps <= (1 << 24), SMCX_E_INVALID_ARG, "n_sweeps must be 0..2^24");
  need(n_sweeps == 0 || E != nullptr || moments != nullptr, SMCX_E_INVALID_ARG, "NULL output buffer");
  need(h->sweep_cum + (uint64_t)n_sweeps < (1ull << 63), SMCX_E_INVALID_ARG, "sweep counter overflow");
  if (n_sweeps == 0) return;
  // start energy into d_energy, accepted-dE sum at the start beside it
  if (!energy_bcc_direct(h)) {
    pair_counts_device(h);
    energy_device(h);
  }
  if (!h->Wq.empty()) qsro_energy_add(h);
  // d_buf: dE-sum snapshot, the n_sweeps energies, then 3 doubles of moments
  long long* d_buf = nullptr;
  check_cuda(cudaMalloc(&d_buf, (size_t)(n_sweeps + 1 + 3) * sizeof(long long)), "energy trace");
  try {
    check_cuda(cudaMemcpyAsync(d_buf, h->d_stats + 3, sizeof(long long), cudaMemcpyDeviceToDevice, h->stream),
               "dE sum snapshot");
    upload_thresholds(h, T);
    for (int64_t i = 0; i < n_sweeps; i++) {
      sweep_device(h, h->thr_nA, seed, 1);
      h->sweep_cum += 1;
      record_energy(h, d_buf, d_buf + 1 + i);
    }
    double* d_mom = reinterpret_cast<double*>(d_buf + 1 + n_sweeps);
    if (moments) energy_moments(h, d_buf + 1, n_sweeps, T, d_mom);
    if (E)
      check_cuda(cudaMemcpyAsync(E, d_buf + 1, (size_t)n_sweeps * sizeof(long long), cudaMemcpyDeviceToHost,
                                 h->stream),
                 "energy trace download");
    if (moments)
      check_cuda(cudaMemcpyAsync(moments, d_mom, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
                 "moments download");
    check_cuda(cudaStreamSynchronize(h->stream), "energy trace sync");
  } catch (...) {
    cudaFree(d_buf);
    throw;
  }
  cudaFree(d_buf);
}

int smcx_sweep_energies(smcx_lattice* h, double T, int64_t n_sweeps, uint64_t seed, int64_t* E) {
  NvtxRange nvtx_range("smcx_sweep_energies");
  return guarded([&] {
    need(n_sweeps == 0 || E != nullptr, SMCX_E_INVALID_ARG, "NULL energy buffer");
    sweep_recorded(h, T, n_sweeps, seed, E, nullptr, "smcx_sweep_energies");
  });
}

int smcx_sweep_cv(smcx_lattice* h, double T, int64_t n_sweeps, uint64_t seed, int64_t* E, double* moments) {
  NvtxRange nvtx_range("smcx_sweep_cv");
  return guarded([&] {
    need(n_sweeps >= 1, SMCX_E_INVALID_ARG, "the specific heat needs n_sweeps >= 1");
    need(moments != nullptr, SMCX_E_INVALID_ARG, "NULL moments buffer");
    sweep_recorded(h, T, n_sweeps, seed, E, moments, "smcx_sweep_cv");
  });
}

int smcx_sweep_partial(smcx_lattice* h, double T, uint64_t seed, int n_colours) {
  NvtxRange nvtx_range("smcx_sweep_partial");
  return guarded([&] {
    need(h != nullptr, SMCX_E_INVALID_ARG, "NULL handle");
    need(h->have_epi, SMCX_E_NO_EPI, "call smcx_set_epi before smcx_sweep_partial");
    need(h->sched.L != 0, SMCX_E_SCHEDULE, "no checkerboard schedule fits this lattice");
    need(T > 0.0 && isfinite(T), SMCX_E_INVALID_ARG, "temperature must be finite and > 0");
    need(n_colours >= 0 && n_colours <= 8, SMCX_E_INVALID_ARG, "n_colours must be in 0..8");
    if (n_colours == 0) return;
    upload_thresholds(h, T);
    sweep_device(h, h->thr_nA, seed, 1, n_colours);
  });
}

int smcx_pair_counts(smcx_lattice* h, int64_t* C) {
  return guarded([&] {
    need(h && C, SMCX_E_INVALID_ARG, "NULL argument");
    need(h->have_epi, SMCX_E_NO_EPI, "pair counts need the shell count: call smcx_set_epi first");
    pair_counts_device(h);
    const int KMM = h->shells.K * h->M * h->M;
    check_cuda(cudaMemcpyAsync(C, h->d_counts, KMM * 8, cudaMemcpyDeviceToHost, h->stream), "counts download");
    check_cuda(cudaStreamSynchronize(h->stream), "counts sync");
  });
}

int smcx_energy(smcx_lattice* h, int64_t* E) {
  NvtxRange nvtx_range("smcx_energy");
  return guarded([&] {
    need(h && E, SMCX_E_INVALID_ARG, "NULL argument");
    need(h->have_epi, SMCX_E_NO_EPI, "call smcx_set_epi first");
    if (!energy_bcc_direct(h)) {
      pair_counts_device(h);
      energy_device(h);
    }
    if (!h->Wq.empty()) qsro_energy_add(h);
    long long e = 0;
    check_cuda(cudaMemcpyAsync(&e, h->d_energy, 8, cudaMemcpyDeviceToHost, h->stream), "energy download");
    check_cuda(cudaStreamSynchronize(h->stream), "energy sync");
    *E = e;
  });
}

int smcx_sro(smcx_lattice* h, double* alpha) {
  return guarded([&] {
    need(h && alpha, SMCX_E_INVALID_ARG, "NULL argument");
    need(h->have_epi, SMCX_E_NO_EPI, "call smcx_set_epi first");
    const int K = h->shells.K, M = h->M;
    std::vector<int64_t> C((size_t)K * M * M);
    pair_counts_device(h);
    check_cuda(cudaMemcpyAsync(C.data(), h->d_counts, C.size() * 8, cudaMemcpyDeviceToHost, h->stream),
               "counts download");
    check_cuda(cudaStreamSynchronize(h->stream), "counts sync");
    // species counts from the shell-1 row sums: sum_q C_1[p][q] = z_1 N_p
    std::vector<double> Np(M);
    for (int p = 0; p < M; p++) {
      int64_t r = 0;
      for (int q = 0; q < M; q++) r += C[(size_t)p * M + q];
      Np[p] = (double)(r / h->shells.z[0]);
    }
    const double N = (double)h->N;
    for (int k = 0; k < K; k++)
      for (int p = 0; p < M; p++)
        for (int q = 0; q < M; q++) {
          const double denom = (double)h->shells.z[k] * Np[p] * (Np[q] / N);
          alpha[((size_t)k * M + p) * M + q] =
              denom > 0.0 ? 1.0 - (double)C[((size_t)k * M + p) * M + q] / denom : 0.0;
        }
  });
}

int smcx_get_config(smcx_lattice* h, int8_t* host) {
  return guarded([&] {
    need(h && host, SMCX_E_INVALID_ARG, "NULL argument");
    ensure_stage(h);
    unpack_to_int8(h, reinterpret_cast<int8_t*>(h->d_stage), 0, h->N);
    check_cuda(cudaMemcpyAsync(host, h->d_stage, (size_t)h->N, cudaMemcpyDeviceToHost, h->stream),
               "config download");
    check_cuda(cudaStreamSynchronize(h->stream), "config download sync");
  });
}

static size_t store_bytes(const smcx_lattice* h) {
  return (size_t)(h->storage == SMCX_INT8 ? h->N : (h->N + 1) / 2);
}

int smcx_store_bytes(const smcx_lattice* h, size_t* bytes) {
  return guarded([&] {
    need(h && bytes, SMCX_E_INVALID_ARG, "NULL argument");
    *bytes = store_bytes(h);
  });
}

int smcx_get_config_store(smcx_lattice* h, uint8_t* host, size_t bytes) {
  return guarded([&] {
    need(h && host, SMCX_E_INVALID_ARG, "NULL argument");
    need(bytes == store_bytes(h), SMCX_E_INVALID_ARG, "buffer size must equal the store size");
    check_cuda(cudaMemcpyAsync(host, h->d_sites, bytes, cudaMemcpyDeviceToHost, h->stream), "store download");
    check_cuda(cudaStreamSynchronize(h->stream), "store download sync");
  });
}

int smcx_set_config_store(smcx_lattice* h, const uint8_t* host, size_t bytes) {
  return guarded([&] {
    need(h && host, SMCX_E_INVALID_ARG, "NULL argument");
    need(bytes == store_bytes(h), SMCX_E_INVALID_ARG, "buffer size must equal the store size");
    ensure_stage(h);  // N bytes >= the store size
    check_cuda(cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream), "clear flag");
    check_cuda(cudaMemcpyAsync(h->d_stage, host, bytes, cudaMemcpyHostToDevice, h->stream), "store upload");
    validate_store_at(h, h->d_stage);
    int flag = 0;
    check_cuda(cudaMemcpyAsync(&flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "flag download");
    check_cuda(cudaStreamSynchronize(h->stream), "store upload sync");
    need(flag == 0, SMCX_E_INVALID_ARG, "configuration holds species ids outside 0..M-1");
    check_cuda(cudaMemcpyAsync(h->d_sites, h->d_stage, bytes, cudaMemcpyDeviceToDevice, h->stream), "store copy");
  });
}

int smcx_set_config(smcx_lattice* h, const int8_t* host) {
  return guarded([&] {
    need(h && host, SMCX_E_INVALID_ARG, "NULL argument");
    ensure_stage(h);
    // ids are checked on the device before the lattice store is touched, so
    // a rejected configuration leaves the lattice unchanged
    check_cuda(cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream), "clear flag");
    check_cuda(cudaMemcpyAsync(h->d_stage, host, (size_t)h->N, cudaMemcpyHostToDevice, h->stream), "config upload");
    validate_int8(h, reinterpret_cast<const int8_t*>(h->d_stage), h->N);
    int flag = 0;
    check_cuda(cudaMemcpyAsync(&flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "flag download");
    check_cuda(cudaStreamSynchronize(h->stream), "config upload sync");
    need(flag == 0, SMCX_E_INVALID_ARG, "configuration holds species ids outside 0..M-1");
    pack_from_int8(h, reinterpret_cast<const int8_t*>(h->d_stage), 0, h->N);
  });
}

int smcx_get_state(smcx_lattice* h, uint64_t* sweep_cum, int64_t* stats) {
  return guarded([&] {
    need(h != nullptr, SMCX_E_INVALID_ARG, "NULL handle");
    if (sweep_cum) *sweep_cum = h->sweep_cum;
    if (stats) {
      unsigned long long s[4];
      check_cuda(cudaMemcpyAsync(s, h->d_stats, sizeof(s), cudaMemcpyDeviceToHost, h->stream), "stats download");
      check_cuda(cudaStreamSynchronize(h->stream), "stats sync");
      for (int i = 0; i < 4; i++) stats[i] = (int64_t)s[i];
    }
  });
}

int smcx_set_sweep_counter(smcx_lattice* h, uint64_t sweep_cum) {
  return guarded([&] {
    need(h != nullptr, SMCX_E_INVALID_ARG, "NULL handle");
    need(sweep_cum < (1ull << 63), SMCX_E_INVALID_ARG, "sweep counter must be < 2^63");
    h->sweep_cum = sweep_cum;
  });
}

int smcx_device_buffer(const smcx_lattice* h, void** ptr, size_t* bytes) {
  return guarded([&] {
    need(h && ptr && bytes, SMCX_E_INVALID_ARG, "NULL argument");
    *ptr = h->d_sites;
    *bytes = (size_t)(h->storage == SMCX_INT8 ? h->N : (h->N + 1) / 2);
  });
}

int smcx_synchronize(smcx_lattice* h) {
  return guarded([&] {
    need(h != nullptr, SMCX_E_INVALID_ARG, "NULL handle");
    check_cuda(cudaStreamSynchronize(h->stream), "stream synchronize");
  });
}

int smcx_lattice_info(const smcx_lattice* h, int* kind, int* dims, int* M, int* K, int* storage, int64_t* n_sites) {
  return guarded([&] {
    need(h != nullptr, SMCX_E_INVALID_ARG, "NULL handle");
    if (kind) *kind = h->kind;
    if (dims)
      for (int a = 0; a < 3; a++) dims[a] = h->n[a];
    if (M) *M = h->M;
    if (K) *K = h->have_epi ? h->shells.K : 0;
    if (storage) *storage = h->storage;
    if (n_sites) *n_sites = h->N;
  });
}

}  // extern "C"

int smcx_debug_status(uint64_t* info) {
  return guarded([&] {
    need(info != nullptr, SMCX_E_INVALID_ARG, "NULL argument");
#ifdef SMCX_DEBUG
    check_cuda(cudaDeviceSynchronize(), "debug status sync");
    info[0] = 0;
    info[1] = 0;
    for (auto rd : dbg::readers()) {
      unsigned long long w[2] = {0ull, 0ull};
      if (rd(w) != 0) fail(SMCX_E_CUDA, "debug status read failed");
      if (info[0] == 0 && w[0] != 0) {
        info[0] = w[0];
        info[1] = w[1];
      }
    }
#else
    fail(SMCX_E_UNSUPPORTED, "not a debug build (build with SMCX_DEBUG=1)");
#endif
  });
}
