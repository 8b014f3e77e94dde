// Batched replicas: many independent BCC lattices (uneven sizes, one
// temperature each, shared EPI) swept in ONE persistent cooperative launch.
//
// Temperature parallelism is one of the paper's parallel opportunities
// (Supplementary "Parallelization opportunities": simulations at different
// temperatures are independent); the paper runs them on separate GPUs, here
// they share one GPU and one launch.  Every replica keeps its own schedule,
// sweep counter and Philox replica id, so its trajectory is bit-identical to
// sweeping it alone through smcx_sweep, in either proposal mode.
//
// The kernel (smcx_batch_body.cuh) loops over sweeps and tile colours; in
// each colour the CTAs take the pooled list of (replica, tile) work items of
// that colour, then meet at a grid barrier.  The barrier waits at most
// `timeout_ns`: a CTA that gives up writes SMCX_E_TIMEOUT into a device status
// word and returns, and so does every other CTA once it sees the status, so
// the context stays usable.
#include <algorithm>
#include <cmath>
#include <map>

#include "smcx_batch_body.cuh"

struct smcx_batch {
  std::vector<smcx_lattice*> lat;
  cudaStream_t stream = nullptr;
  smcx::bccfast::LatDesc* d_desc = nullptr;
  int2* d_items = nullptr;  // (replica, tile index within its colour)
  int n_items = 0;
  unsigned* d_bar = nullptr;
  int* d_status = nullptr;
  int threads = 0, slots = 1;
  long long timeout_ns = 2000000000ll;
  int skip_cta = -1;  // fault injection: this CTA never arrives at the barrier
  bool use_graph = true;
  std::map<long long, cudaGraphExec_t> graphs;  // keyed by (sweeps, table size)
  std::vector<int32_t> graph_V;                 // EPI baked into the graphs
  bool items_dirty = true;
  int items_proposal = -1;  // proposal mode the work list and block shape were built for
  int last_grid = 0;
  bool last_graph = false;
  // fluctuation accumulation: per-replica descriptors, (replica, tile) items, counts
  smcx::bccfast::LatDesc* d_fdesc = nullptr;
  int2* d_fitems = nullptr;
  unsigned long long* d_fcounts = nullptr;
  size_t fitems_cap = 0;
};

void fluct_launch_per_sample(const long long* C, long long R, int K, int M, int shell, int z0, int zs, double* acc,
                             cudaStream_t st);

namespace smcx {

int build_planes(const smcx_lattice* hd, bccfast::Planes* Q, int min_planes);


namespace {

void check_batch(const smcx_batch* b) {
  if (b->lat.empty()) fail(SMCX_E_INVALID_ARG, "empty batch");
  const smcx_lattice* h0 = b->lat[0];
  for (const smcx_lattice* h : b->lat) {
    if (!h->have_epi) fail(SMCX_E_NO_EPI, "every replica needs smcx_set_epi");
    if (h->kind != kBCC) fail(SMCX_E_UNSUPPORTED, "batched sweeps run BCC lattices");
    if (h->M != h0->M || h->shells.K != h0->shells.K || h->V != h0->V)
      fail(SMCX_E_INVALID_ARG, "replicas must share M and the EPI table");
    if (h->stream != b->stream) fail(SMCX_E_INVALID_ARG, "replicas must share the batch stream");
    if (h->proposal != h0->proposal) fail(SMCX_E_INVALID_ARG, "replicas must share the proposal mode");
    if (!bcc_fast_usable(h, 256))
      fail(SMCX_E_UNSUPPORTED, "replica schedule needs tiles of at most 20 cells (BCC, M <= 8)");
  }
  if (h0->shells.K != 4) fail(SMCX_E_UNSUPPORTED, "batched sweeps run 4-shell EPI tables");
}

void rebuild_items(smcx_batch* b) {
  std::vector<int2> items;
  int nq = 0;
  for (size_t r = 0; r < b->lat.size(); r++) {
    const smcx_lattice* h = b->lat[r];
    const int per_colour = (h->sched.nt[0] / 2) * (h->sched.nt[1] / 2) * (h->sched.nt[2] / 2);
    for (int j = 0; j < per_colour; j++) items.push_back(make_int2((int)r, j));
    nq = std::max(nq, bcc_slots_per_axis(h->n, h->sched));
  }
  // largest replicas first, so the tail of each colour pass holds small tiles
  std::stable_sort(items.begin(), items.end(), [&](const int2& a, const int2& c) {
    const smcx_lattice* ha = b->lat[a.x];
    const smcx_lattice* hc = b->lat[c.x];
    return (long long)ha->N / ((long long)ha->sched.nt[0] * ha->sched.nt[1] * ha->sched.nt[2]) >
           (long long)hc->N / ((long long)hc->sched.nt[0] * hc->sched.nt[1] * hc->sched.nt[2]);
  });
  cudaFree(b->d_items);
  b->d_items = nullptr;
  check_cuda(cudaMalloc(&b->d_items, items.size() * sizeof(int2)), "batch work list");
  check_cuda(cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice,
                             b->stream),
             "batch work list upload");
  check_cuda(cudaStreamSynchronize(b->stream), "batch work list sync");
  b->n_items = (int)items.size();
  int threads, slots;
  // shared-direction proposals run one slot per thread: tiles of more than
  // 128 slots take 256-thread CTAs unless 128 threads were asked for
  const bool dir = b->lat[0]->proposal != 0;
  if (b->threads == 256 || (dir && b->threads != 128 && nq * nq * nq > 128)) {
    threads = 256;  // one slot per thread
    slots = 1;
    if (nq * nq * nq > 256) fail(SMCX_E_UNSUPPORTED, "256-thread CTAs take tiles of at most 256 link-cell slots");
  } else {
    bcc_block_shape(nq, b->threads, &threads, &slots);
  }
  if (slots > 2) fail(SMCX_E_UNSUPPORTED, "batched tiles need at most 256 link-cell slots");
  b->threads = threads;
  b->slots = slots;
  b->items_proposal = b->lat[0]->proposal;
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.second);
  b->graphs.clear();
  b->items_dirty = false;
}

using bccfast::BatchKernelFn;

BatchKernelFn pick_kernel(int nw, int pl, int slots, int threads, int proposal) {
  using namespace bccfast;
  if (proposal != 0) {
    // shared-direction proposals: one compiled variant (M <= 4, |V| < 2^15)
    if (nw != 1 || pl != 2 || slots != 1)
      fail(SMCX_E_UNSUPPORTED, "shared-direction batches need M <= 4, |V| < 2^15 and one slot per thread");
    return batch_dir_kernel(threads);
  }
#define SMCX_PICK(NW_, PL_)                                    \
  return threads == 256 ? k_bcc_batch256<4, NW_, PL_, 0>       \
         : slots == 1   ? k_bcc_batch<4, NW_, PL_, 1, 0> \
                        : k_bcc_batch<4, NW_, PL_, 2, 0>
  if (nw == 1 && pl == 2) SMCX_PICK(1, 2);
  if (nw == 1) SMCX_PICK(1, 3);
  if (pl == 2) SMCX_PICK(2, 2);
  SMCX_PICK(2, 3);
#undef SMCX_PICK
}

}  // namespace

void upload_thresholds_for(smcx_lattice* h, double T);  // smcx_api.cu

// Enqueue n sweeps of every replica (temperatures T[r]); returns after the
// launch completed and its status was read.
static void batch_sweep_launch(smcx_batch* b, const double* T, int64_t n_sweeps, uint64_t seed);

void batch_sweep(smcx_batch* b, const double* T, int64_t n_sweeps, uint64_t seed) {
  check_batch(b);
  // at most 2^16 sweeps per launch keep the barrier counter far from overflow
  for (int64_t done = 0; done < n_sweeps;) {
    const int64_t n = std::min<int64_t>(n_sweeps - done, 1 << 16);
    batch_sweep_launch(b, T, n, seed);
    done += n;
  }
}

static void batch_sweep_launch(smcx_batch* b, const double* T, int64_t n_sweeps, uint64_t seed) {
  if (b->items_dirty || b->items_proposal != b->lat[0]->proposal) rebuild_items(b);
  const size_t R = b->lat.size();
  std::vector<bccfast::LatDesc> desc(R);
  int max_nA = 0;
  for (size_t r = 0; r < R; r++) {
    smcx_lattice* h = b->lat[r];
    if (!(T[r] > 0.0) || !std::isfinite(T[r])) fail(SMCX_E_INVALID_ARG, "temperatures must be finite and > 0");
    if (h->sweep_cum + (uint64_t)n_sweeps >= (1ull << 63)) fail(SMCX_E_INVALID_ARG, "sweep counter overflow");
    upload_thresholds_for(h, T[r]);
    bccfast::LatDesc& D = desc[r];
    memset(&D, 0, sizeof(D));
    D.sites = h->d_sites;
    D.thr = h->d_thr;
    D.stats = h->d_stats;
    for (int a = 0; a < 3; a++) {
      D.n[a] = h->n[a];
      D.nt[a] = h->sched.nt[a];
    }
    D.L = h->sched.L;
    D.NQ = bcc_slots_per_axis(h->n, h->sched);
    D.nA = h->thr_nA;
    D.storage = h->storage;
    D.replica = h->replica;
    D.seed_lo = (uint32_t)seed;
    D.seed_hi = (uint32_t)(seed >> 32);
    D.sweep = h->sweep_cum;
    D.proposal = h->proposal;
    max_nA = std::max(max_nA, D.nA);
  }
  if (!b->d_desc) check_cuda(cudaMalloc(&b->d_desc, R * sizeof(bccfast::LatDesc)), "batch descriptors");
  check_cuda(cudaMemcpyAsync(b->d_desc, desc.data(), R * sizeof(bccfast::LatDesc), cudaMemcpyHostToDevice, b->stream),
             "batch descriptor upload");
  bccfast::Planes Q;
  const int PL = build_planes(b->lat[0], &Q, 2);
  const int nw = b->lat[0]->M <= 4 ? 1 : 2;
  BatchKernelFn fn = pick_kernel(nw, PL, b->slots, b->threads, b->lat[0]->proposal);
  // shared memory for the largest table of this call, rounded up so that a
  // graph instantiated for it serves nearby temperature sets as well
  const int nA_cap = std::min(kNA, ((max_nA + 255) / 256) * 256);
  const size_t smem = bccfast::smem_bytes(nA_cap);
  check_cuda(cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
             "batch smem attribute");
  int dev = 0, nsm = 0, per_sm = 0;
  check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  check_cuda(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "SM count");
  check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)fn, b->threads, smem), "occupancy");
  if (per_sm < 1) fail(SMCX_E_UNSUPPORTED, "batch kernel does not fit an SM");
  const int grid = std::min(b->n_items, per_sm * nsm);
  if (!b->d_bar) {
    check_cuda(cudaMalloc(&b->d_bar, sizeof(unsigned)), "barrier word");
    check_cuda(cudaMalloc(&b->d_status, sizeof(int)), "status word");
  }
  int n_int = (int)n_sweeps;
  int max_nA_arg = nA_cap;
  void* args[] = {(void*)&Q, (void*)&b->d_desc, (void*)&b->d_items, (void*)&b->n_items, (void*)&n_int,
                  (void*)&b->d_bar, (void*)&b->d_status, (void*)&b->timeout_ns, (void*)&b->skip_cta,
                  (void*)&max_nA_arg};
  if (b->graph_V != b->lat[0]->V) {
    for (auto& g : b->graphs) cudaGraphExecDestroy(g.second);
    b->graphs.clear();
    b->graph_V = b->lat[0]->V;
  }
  auto enqueue = [&]() {
    check_cuda(cudaMemsetAsync(b->d_bar, 0, sizeof(unsigned), b->stream), "barrier reset");
    check_cuda(cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream), "status reset");
    check_cuda(cudaLaunchCooperativeKernel((const void*)fn, dim3(grid), dim3(b->threads), args, smem, b->stream),
               "batch cooperative launch");
  };
  bool launched = false;
  if (b->use_graph && b->skip_cta < 0) {
    // one instantiated graph per sweep count; planes, seed and descriptors
    // are read from memory or baked parameters that do not change between
    // calls of one batch (the EPI is fixed once the batch sweeps)
    const long long key = (long long)n_sweeps * 8192 + nA_cap;
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      bool ok = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        cudaMemsetAsync(b->d_bar, 0, sizeof(unsigned), b->stream);
        cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream);
        cudaLaunchCooperativeKernel((const void*)fn, dim3(grid), dim3(b->threads), args, smem, b->stream);
        ok = cudaStreamEndCapture(b->stream, &g) == cudaSuccess && g != nullptr;
      }
      if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();  // clear a failed capture's sticky-free error
      if (ok) it = b->graphs.emplace(key, ge).first;
      else b->use_graph = false;
    }
    if (b->use_graph) {
      check_cuda(cudaGraphLaunch(it->second, b->stream), "batch graph launch");
      launched = true;
    }
  }
  if (!launched) enqueue();
  b->last_grid = grid;
  b->last_graph = launched;
  int status = 0;
  check_cuda(cudaMemcpyAsync(&status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->stream), "status read");
  check_cuda(cudaStreamSynchronize(b->stream), "batch sync");
  if (status != 0) fail(status, "batched sweep stopped: a grid barrier timed out");
  for (smcx_lattice* h : b->lat) h->sweep_cum += (uint64_t)n_sweeps;
}

void batch_release(smcx_batch* b) {
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.second);
  cudaFree(b->d_desc);
  cudaFree(b->d_items);
  cudaFree(b->d_fdesc);
  cudaFree(b->d_fitems);
  cudaFree(b->d_fcounts);
  cudaFree(b->d_bar);
  cudaFree(b->d_status);
}

// Autotuner: for each candidate (link cell L, tile target, threads per CTA)
// assign every replica the schedule the candidate implies, time `trial`
// batched sweeps on a copy of the configurations, restore them, and keep the
// fastest candidate.  The schedule defines the trajectory, so the choice is
// reported (smcx_get_schedule on each replica) and a run can be reproduced.
void batch_autotune(smcx_batch* b, const double* T, int trial, int* best_threads) {
  check_batch(b);
  const size_t R = b->lat.size();
  struct Saved {
    uint8_t* d_copy = nullptr;
    smcx_sched sched;
    uint64_t sweep;
    unsigned long long stats[4];
  };
  std::vector<Saved> saved(R);
  for (size_t r = 0; r < R; r++) {
    smcx_lattice* h = b->lat[r];
    check_cuda(cudaMalloc(&saved[r].d_copy, h->site_bytes), "autotune snapshot");
    check_cuda(cudaMemcpyAsync(saved[r].d_copy, h->d_sites, h->site_bytes, cudaMemcpyDeviceToDevice, b->stream),
               "autotune snapshot copy");
    check_cuda(cudaMemcpyAsync(saved[r].stats, h->d_stats, sizeof(saved[r].stats), cudaMemcpyDeviceToHost, b->stream),
               "autotune stats snapshot");
    saved[r].sched = h->sched;
    saved[r].sweep = h->sweep_cum;
  }
  check_cuda(cudaStreamSynchronize(b->stream), "autotune snapshot sync");
  struct Cand {
    int L, target, threads;
  };
  std::vector<Cand> cands;
  // a tile pass takes 2 L^3 phase steps whatever the tile's size, so the
  // candidates trade tile size (lanes busy per step) against the number of
  // items per colour (CTA rounds); shapes a kernel does not take are skipped
  for (int L : {3, 4})
    for (int target : {12, 13, 14, 15, 16, 17, 18, 20})
      for (int th : {128, 256}) cands.push_back({L, target, th});
  double best = 1e300;
  Cand bestc = cands[0];
  std::vector<smcx_sched> best_sched(R);
  cudaEvent_t e0, e1;
  check_cuda(cudaEventCreate(&e0), "event");
  check_cuda(cudaEventCreate(&e1), "event");
  for (const Cand& c : cands) {
    bool ok = true;
    std::vector<smcx_sched> sc(R);
    for (size_t r = 0; r < R && ok; r++) {
      smcx_lattice* h = b->lat[r];
      sc[r].L = c.L;
      for (int a = 0; a < 3; a++) {
        int nt = 2;
        while ((h->n[a] + nt - 1) / nt > c.target) nt += 2;
        sc[r].nt[a] = nt;
      }
      if (!schedule_problem(h->shells, h->n, sc[r]).empty()) ok = false;
    }
    if (!ok) continue;
    for (size_t r = 0; r < R; r++) b->lat[r]->sched = sc[r];
    b->threads = c.threads;
    b->items_dirty = true;
    bool usable = true;
    for (size_t r = 0; r < R; r++) usable = usable && bcc_fast_usable(b->lat[r], 256);
    if (!usable) continue;
    try {
      batch_sweep(b, T, 1, 0x5eedull);  // warm-up: instantiate, load tables
      check_cuda(cudaEventRecord(e0, b->stream), "event");
      batch_sweep(b, T, trial, 0x5eedull);
      check_cuda(cudaEventRecord(e1, b->stream), "event");
      check_cuda(cudaEventSynchronize(e1), "event sync");
    } catch (const SmcxException&) {
      continue;
    }
    float ms = 0;
    check_cuda(cudaEventElapsedTime(&ms, e0, e1), "event time");
    if (ms < best) {
      best = ms;
      bestc = c;
      best_sched = sc;
    }
    // restore configurations and counters before the next candidate
    for (size_t r = 0; r < R; r++) {
      smcx_lattice* h = b->lat[r];
      check_cuda(cudaMemcpyAsync(h->d_sites, saved[r].d_copy, h->site_bytes, cudaMemcpyDeviceToDevice, b->stream),
                 "autotune restore");
      h->sweep_cum = saved[r].sweep;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (size_t r = 0; r < R; r++) {
    smcx_lattice* h = b->lat[r];
    check_cuda(cudaMemcpyAsync(h->d_sites, saved[r].d_copy, h->site_bytes, cudaMemcpyDeviceToDevice, b->stream),
               "autotune restore");
    check_cuda(cudaMemcpyAsync(h->d_stats, saved[r].stats, sizeof(saved[r].stats), cudaMemcpyHostToDevice, b->stream),
               "autotune stats restore");
    h->sweep_cum = saved[r].sweep;
    h->sched = best < 1e300 ? best_sched[r] : saved[r].sched;
    h->sched_auto = false;
  }
  check_cuda(cudaStreamSynchronize(b->stream), "autotune restore sync");
  for (auto& s : saved) cudaFree(s.d_copy);
  if (best >= 1e300) fail(SMCX_E_SCHEDULE, "no autotuner candidate fits these lattices");
  b->threads = bestc.threads;
  b->items_dirty = true;
  if (best_threads) *best_threads = bestc.threads;
}

// Replica exchange (Supplementary "Parallelization opportunities": the
// configurations at different temperatures are exchanged by a rule that
// keeps detailed balance).  A round sweeps every replica at the temperature
// of its slot, then proposes swaps of the slot pairs (t, t+1), t = round mod
// 2, +2, ...; the swap of replicas a (slot t) and c (slot t+1) is accepted
// when x = (beta_t - beta_{t+1})(E_a - E_c) >= 0, else when u <
// floor(2^32 exp(x)) (capped at 2^32 - 1), u = word 0 of Philox(counter (t,
// round lo, round hi, 0xC0000000), key = seed).  Energies are exact: the
// start energy of each replica plus its accumulated accepted dE.  The O(R)
// decision runs on the host in double, like the acceptance tables.
void batch_exchange(smcx_batch* b, const double* T_slot, int32_t* slot_rep, int64_t n_rounds,
                    int64_t sweeps_per_round, uint64_t seed, uint64_t* round_ctr, int64_t* accepts) {
  check_batch(b);
  const int R = (int)b->lat.size();
  const smcx_lattice* h0 = b->lat[0];
  for (const smcx_lattice* h : b->lat)
    if (h->n[0] != h0->n[0] || h->n[1] != h0->n[1] || h->n[2] != h0->n[2])
      fail(SMCX_E_INVALID_ARG, "replica exchange needs replicas of one lattice shape");
  std::vector<int> seen(R, 0);
  for (int t = 0; t < R; t++) {
    if (!(T_slot[t] > 0.0) || !std::isfinite(T_slot[t])) fail(SMCX_E_INVALID_ARG, "temperatures must be finite and > 0");
    if (slot_rep[t] < 0 || slot_rep[t] >= R || seen[slot_rep[t]]++)
      fail(SMCX_E_INVALID_ARG, "slot_rep must be a permutation of the replicas");
  }
  std::vector<long long> E(R), d0(R), dcur(R);
  for (int r = 0; r < R; r++) {
    int64_t e = 0;
    int rc = smcx_energy(b->lat[r], &e);
    if (rc != SMCX_OK) fail(rc, last_error());
    E[r] = e;
  }
  auto read_dsum = [&](std::vector<long long>& out) {
    for (int r = 0; r < R; r++)
      check_cuda(cudaMemcpyAsync(&out[r], b->lat[r]->d_stats + 3, sizeof(long long), cudaMemcpyDeviceToHost, b->stream),
                 "stats download");
    check_cuda(cudaStreamSynchronize(b->stream), "stats sync");
  };
  read_dsum(d0);
  std::vector<double> T(R);
  const double kB = 8.617333262e-2;  // meV / K
  for (int64_t i = 0; i < n_rounds; i++) {
    for (int t = 0; t < R; t++) T[slot_rep[t]] = T_slot[t];
    batch_sweep(b, T.data(), sweeps_per_round, seed);
    read_dsum(dcur);
    const uint64_t rnd = *round_ctr;
    for (int t = (int)(rnd & 1); t + 1 < R; t += 2) {
      const int a = slot_rep[t], c = slot_rep[t + 1];
      const long long Ea = E[a] + dcur[a] - d0[a], Ec = E[c] + dcur[c] - d0[c];
      const double bt = 1.0 / (kB * T_slot[t]);
      const double bu = 1.0 / (kB * T_slot[t + 1]);
      const double x = (bt - bu) * ((double)(Ea - Ec) * 0.01);
      const uint4 w = philox4x32_10(make_uint4((uint32_t)t, (uint32_t)rnd, (uint32_t)(rnd >> 32), 0xC0000000u),
                                    make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
      bool accept;
      if (x >= 0.0) {
        accept = true;
      } else {
        const double v = std::exp(x) * 4294967296.0;
        const uint32_t thr = v >= 4294967295.0 ? 4294967295u : (uint32_t)v;
        accept = w.x < thr;
      }
      if (accept) {
        slot_rep[t] = c;
        slot_rep[t + 1] = a;
        if (accepts) accepts[t]++;
      }
    }
    *round_ctr = rnd + 1;
  }
}

void pair_counts_bcc_multi(const bccfast::LatDesc* d_descs, const int2* d_items, int n_items, int K, int M,
                           unsigned long long* d_counts, cudaStream_t st);  // smcx_reduce_bcc.cu

// Fluctuation sums of every replica in two launches: the tiled pair counts of
// all replicas' tiles in one grid, then one accumulator CTA per replica
// (d_acc [R][1 + MM + KMM + MM KMM]).
void batch_fluct_accumulate(smcx_batch* b, int shell, double* d_acc) {
  check_batch(b);
  const int R = (int)b->lat.size();
  const smcx_lattice* h0 = b->lat[0];
  const int K = h0->shells.K, M = h0->M;
  if (shell < 0 || shell >= K) fail(SMCX_E_INVALID_ARG, "shell out of range");
  if (M > 4) fail(SMCX_E_UNSUPPORTED, "batched fluctuation sums run M <= 4 (use smcx_lattice_fluct_accumulate)");
  std::vector<bccfast::LatDesc> desc(R);
  std::vector<int2> items;
  for (int r = 0; r < R; r++) {
    const smcx_lattice* h = b->lat[r];
    bccfast::LatDesc& D = desc[r];
    memset(&D, 0, sizeof(D));
    D.sites = h->d_sites;
    D.storage = h->storage;
    D.M = M;
    int ntiles = 1;
    for (int a = 0; a < 3; a++) {
      D.n[a] = h->n[a];
      D.nt[a] = h->sched.nt[a];
      if (D.nt[a] < 2 || h->n[a] < 6 || (h->n[a] + D.nt[a] - 1) / D.nt[a] + 4 > bccfast::BOX)
        fail(SMCX_E_UNSUPPORTED, "replica tiles do not fit the tiled pair counts");
      ntiles *= D.nt[a];
    }
    for (int t = 0; t < ntiles; t++) items.push_back(make_int2(r, t));
  }
  if (!b->d_fdesc) {
    check_cuda(cudaMalloc(&b->d_fdesc, R * sizeof(bccfast::LatDesc)), "fluctuation descriptors");
    check_cuda(cudaMalloc(&b->d_fcounts, (size_t)R * kMaxShells * 16 * sizeof(unsigned long long)),
               "fluctuation counts");
  }
  if (items.size() > b->fitems_cap) {
    cudaFree(b->d_fitems);
    b->d_fitems = nullptr;
    check_cuda(cudaMalloc(&b->d_fitems, items.size() * sizeof(int2)), "fluctuation items");
    b->fitems_cap = items.size();
  }
  check_cuda(cudaMemcpyAsync(b->d_fdesc, desc.data(), R * sizeof(bccfast::LatDesc), cudaMemcpyHostToDevice,
                             b->stream),
             "fluctuation descriptor upload");
  check_cuda(cudaMemcpyAsync(b->d_fitems, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice,
                             b->stream),
             "fluctuation item upload");
  const int kmm = K * M * M;
  check_cuda(cudaMemsetAsync(b->d_fcounts, 0, (size_t)R * kmm * sizeof(unsigned long long), b->stream),
             "clear counts");
  pair_counts_bcc_multi(b->d_fdesc, b->d_fitems, (int)items.size(), K, M, b->d_fcounts, b->stream);
  fluct_launch_per_sample(reinterpret_cast<const long long*>(b->d_fcounts), R, K, M, shell, h0->shells.z[0],
                          h0->shells.z[shell], d_acc, b->stream);
  // the host descriptor and item arrays are pageable: wait before they go
  check_cuda(cudaStreamSynchronize(b->stream), "fluctuation sync");
}

}  // namespace smcx

namespace {
void need_(bool ok, int code, const char* msg) {
  if (!ok) smcx::fail(code, msg);
}
}  // namespace

using namespace smcx;

extern "C" {

int smcx_batch_create(smcx_batch** out, int R, smcx_lattice* const* lattices, void* stream) {
  return guarded_call([&] {
    need_(out && lattices && R >= 1, SMCX_E_INVALID_ARG, "bad batch arguments");
    *out = nullptr;
    smcx_batch* b = new smcx_batch();
    b->stream = reinterpret_cast<cudaStream_t>(stream);
    for (int r = 0; r < R; r++) {
      if (!lattices[r]) {
        delete b;
        fail(SMCX_E_INVALID_ARG, "NULL lattice in batch");
      }
      b->lat.push_back(lattices[r]);
    }
    *out = b;
  });
}

int smcx_batch_destroy(smcx_batch* b) {
  if (!b) return SMCX_OK;
  return guarded_call([&] {
    cudaStreamSynchronize(b->stream);
    batch_release(b);
    delete b;
  });
}

int smcx_batch_sweep(smcx_batch* b, const double* T, int64_t n_sweeps, uint64_t seed) {
  NvtxRange nvtx_range("smcx_batch_sweep");
  return guarded_call([&] {
    need_(b && T, SMCX_E_INVALID_ARG, "NULL argument");
    need_(n_sweeps >= 0, SMCX_E_INVALID_ARG, "negative sweep count");
    batch_sweep(b, T, n_sweeps, seed);
  });
}

int smcx_batch_autotune(smcx_batch* b, const double* T, int trial_sweeps, int* threads) {
  NvtxRange nvtx_range("smcx_batch_autotune");
  return guarded_call([&] {
    need_(b && T, SMCX_E_INVALID_ARG, "NULL argument");
    need_(trial_sweeps >= 1, SMCX_E_INVALID_ARG, "trial_sweeps must be >= 1");
    batch_autotune(b, T, trial_sweeps, threads);
  });
}

int smcx_batch_energy(smcx_batch* b, int64_t* E) {
  return guarded_call([&] {
    need_(b && E, SMCX_E_INVALID_ARG, "NULL argument");
    for (size_t r = 0; r < b->lat.size(); r++) {
      int rc = smcx_energy(b->lat[r], E + r);
      if (rc != SMCX_OK) fail(rc, last_error());
    }
  });
}

int smcx_batch_exchange(smcx_batch* b, const double* T_slot, int32_t* slot_rep, int64_t n_rounds,
                        int64_t sweeps_per_round, uint64_t seed, uint64_t* round_ctr, int64_t* accepts) {
  NvtxRange nvtx_range("smcx_batch_exchange");
  return guarded_call([&] {
    need_(b && T_slot && slot_rep && round_ctr, SMCX_E_INVALID_ARG, "NULL argument");
    need_(n_rounds >= 0 && sweeps_per_round >= 0, SMCX_E_INVALID_ARG, "negative round or sweep count");
    batch_exchange(b, T_slot, slot_rep, n_rounds, sweeps_per_round, seed, round_ctr, accepts);
  });
}

int smcx_batch_fluct_accumulate(smcx_batch* b, int shell, double* d_acc) {
  NvtxRange nvtx_range("smcx_batch_fluct_accumulate");
  return guarded_call([&] {
    need_(b && d_acc, SMCX_E_INVALID_ARG, "NULL argument");
    batch_fluct_accumulate(b, shell, d_acc);
  });
}

int smcx_batch_info(const smcx_batch* b, int* grid, int* threads, int* used_graph) {
  return guarded_call([&] {
    need_(b != nullptr, SMCX_E_INVALID_ARG, "NULL batch");
    if (grid) *grid = b->last_grid;
    if (threads) *threads = b->threads;
    if (used_graph) *used_graph = b->last_graph ? 1 : 0;
  });
}

int smcx_batch_set_block(smcx_batch* b, int threads) {
  return guarded_call([&] {
    need_(b != nullptr, SMCX_E_INVALID_ARG, "NULL batch");
    need_(threads == 0 || threads == 128 || threads == 256, SMCX_E_INVALID_ARG, "threads must be 0, 128 or 256");
    b->threads = threads;
    b->items_dirty = true;
  });
}

int smcx_batch_set_fault(smcx_batch* b, int skip_cta, int timeout_ms) {
  return guarded_call([&] {
    need_(b != nullptr, SMCX_E_INVALID_ARG, "NULL batch");
    need_(timeout_ms >= 1 && timeout_ms <= 60000, SMCX_E_INVALID_ARG, "timeout must be 1..60000 ms");
    b->skip_cta = skip_cta < 0 ? -1 : skip_cta;
    b->timeout_ns = (long long)timeout_ms * 1000000ll;
    for (auto& g : b->graphs) cudaGraphExecDestroy(g.second);
    b->graphs.clear();
  });
}

}  // extern "C"
