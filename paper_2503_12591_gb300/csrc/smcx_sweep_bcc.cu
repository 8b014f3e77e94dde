// Single-lattice BCC sweep on the specialised tile pass (smcx_bcc_tile.cuh):
// one launch per tile colour, one CTA per tile of that colour.
#include "smcx_bcc_tile.cuh"

namespace smcx {


// Byte planes of V: the fewest that hold every entry (2 at least, which
// covers |V| < 2^15), or more if the caller asks (min_planes).  Planes below
// the top one hold unsigned bytes, the top plane the signed high byte.
int build_planes(const smcx_lattice* hd, bccfast::Planes* Q, int min_planes) {
  memset(Q, 0, sizeof(*Q));
  const int K = hd->shells.K, M = hd->M;
  long long vmax = 0;
  for (int32_t v : hd->V) vmax = std::max(vmax, std::llabs((long long)v));
  const int PL = std::max(min_planes, vmax < 32768 ? 2 : 3);
  // V-difference rows for shared-direction trials (M <= 4, 4 shells)
  Q->rows = (M <= 4 && K == 4) ? 1 : 0;
  for (int a = 0; a < 4 && Q->rows; a++)
    for (int b = 0; b < 4 && Q->rows; b++)
      for (int k = 0; k < 4 && Q->rows; k++)
        for (int c = 0; c < 4; c++) {
          const long long vb = (b < M && c < M) ? hd->V[((size_t)k * M + b) * M + c] : 0;
          const long long va = (a < M && c < M) ? hd->V[((size_t)k * M + a) * M + c] : 0;
          const long long T = vb - va;
          if (T < -32768 || T > 32767) {
            Q->rows = 0;
            break;
          }
          Q->R[a * 4 + b][k] |= (uint32_t)(T & 0xFF) << (8 * c);
          Q->R[a * 4 + b][4 + k] |= (uint32_t)((T >> 8) & 0xFF) << (8 * c);
        }
  for (int k = 0; k < K; k++)
    for (int p = 0; p < M; p++)
      for (int c = 0; c < M; c++) {
        const uint32_t v = (uint32_t)hd->V[((size_t)k * M + p) * M + c];
        const int w = c / 4, sh = 8 * (c % 4);
        for (int j = 0; j < PL; j++) Q->P[j][k][p][w] |= ((v >> (8 * j)) & 0xFFu) << sh;
      }
  return PL;
}

// Usable when the lattice is BCC, M <= 8, |V| < 2^23, the tiles fit the
// 24^3 box and two link-cell slots per thread cover a tile.
bool bcc_fast_usable(const smcx_lattice* hd, int dir_slots) {
  const smcx_sched& sc = hd->sched;
  if (hd->kind != kBCC || hd->M > kMaxSweepM || !hd->have_epi) return false;
  if (hd->proposal != 0) {
    // one compiled variant: 4 shells, M <= 4, |V| < 2^15, one slot per thread
    if (hd->shells.K != 4 || hd->M > 4) return false;
    for (int32_t v : hd->V)
      if (v >= 32768 || v <= -32768) return false;
  }
  if (sc.L == 0 || (sc.nt[0] == 1 && sc.nt[1] == 1 && sc.nt[2] == 1)) return false;
  if (halo_cells(hd->shells) != 2 || ring_cells(hd->shells) != 1) return false;
  for (int32_t v : hd->V)
    if (v >= (1 << 23) || v <= -(1 << 23)) return false;  // three byte planes at most
  int nq = 0;
  for (int a = 0; a < 3; a++) {
    const int tmax = (hd->n[a] + sc.nt[a] - 1) / sc.nt[a];
    if (tmax + 4 > bccfast::BOX) return false;
    nq = std::max(nq, (tmax + sc.L - 1) / sc.L);
  }
  if (hd->proposal != 0 && nq * nq * nq > dir_slots) return false;  // one slot per thread
  // four slots per thread are compiled for 4 shells, M <= 4, two planes only
  if (nq * nq * nq > 256) {
    if (hd->shells.K != 4 || hd->M > 4) return false;
    for (int32_t v : hd->V)
      if (v >= 32768 || v <= -32768) return false;
  }
  return nq * nq * nq <= 512;
}

int bcc_slots_per_axis(const int n[3], const smcx_sched& sc) {
  int nq = 0;
  for (int a = 0; a < 3; a++) nq = std::max(nq, ((n[a] + sc.nt[a] - 1) / sc.nt[a] + sc.L - 1) / sc.L);
  return nq;
}

// Threads per CTA (at most 128, the kernels' launch bound) and link-cell
// slots per thread (1, 2 or 4) for NQ^3 slots: the handle's tuned block
// size if set, else the fewest threads that need no more slots.
void bcc_block_shape(int nq, int tuned_threads, int* threads, int* slots) {
  const int ns = nq * nq * nq;
  int t = tuned_threads > 0 ? std::min(128, tuned_threads) : std::min(128, ((ns + 31) / 32) * 32);
  int s = (ns + t - 1) / t;
  s = s <= 1 ? 1 : (s <= 2 ? 2 : 4);
  if (tuned_threads <= 0) t = std::min(128, ((ns + s - 1) / s + 31) / 32 * 32);
  if ((long long)t * s < ns) fail(SMCX_E_UNSUPPORTED, "tile needs more than 512 link-cell slots");
  *threads = t;
  *slots = s;
}


void sweep_bcc_dir(smcx_lattice* hd, bccfast::LatDesc& D, const bccfast::Planes& Q, int threads, int64_t n,
                   int nc);  // smcx_sweep_bcc_dir.cu

static void dispatch(smcx_lattice* hd, bccfast::LatDesc& D, const bccfast::Planes& Q, int nw, int pl,
                     int threads, int slots, int64_t n, int nc) {
  const int K = hd->shells.K;
  if (D.proposal != 0) return sweep_bcc_dir(hd, D, Q, threads, n, nc);
  if (K == 4) {
    if (nw == 1 && pl == 2) {
      if (slots == 1) return launch_bcc<4, 1, 2, 1>(hd, D, Q, threads, n, nc);
      if (slots == 2) return launch_bcc<4, 1, 2, 2>(hd, D, Q, threads, n, nc);
      return launch_bcc<4, 1, 2, 4>(hd, D, Q, threads, n, nc);
    }
    if (slots == 4) fail(SMCX_E_UNSUPPORTED, "block shape");
    if (nw == 1) return slots == 1 ? launch_bcc<4, 1, 3, 1>(hd, D, Q, threads, n, nc)
                                   : launch_bcc<4, 1, 3, 2>(hd, D, Q, threads, n, nc);
    if (pl == 2) return slots == 1 ? launch_bcc<4, 2, 2, 1>(hd, D, Q, threads, n, nc)
                                   : launch_bcc<4, 2, 2, 2>(hd, D, Q, threads, n, nc);
    return slots == 1 ? launch_bcc<4, 2, 3, 1>(hd, D, Q, threads, n, nc) : launch_bcc<4, 2, 3, 2>(hd, D, Q, threads, n, nc);
  }
  // fewer shells: one counter word and two planes (M <= 4, |V| < 2^15), or
  // the general variant (any M <= 8, two words, three planes)
  if (slots == 4) fail(SMCX_E_UNSUPPORTED, "block shape");
  if (nw == 1 && pl == 2) {
    if (K == 3) return slots == 1 ? launch_bcc<3, 1, 2, 1>(hd, D, Q, threads, n, nc) : launch_bcc<3, 1, 2, 2>(hd, D, Q, threads, n, nc);
    if (K == 2) return slots == 1 ? launch_bcc<2, 1, 2, 1>(hd, D, Q, threads, n, nc) : launch_bcc<2, 1, 2, 2>(hd, D, Q, threads, n, nc);
  }
  if (K == 3) return slots == 1 ? launch_bcc<3, 2, 3, 1>(hd, D, Q, threads, n, nc) : launch_bcc<3, 2, 3, 2>(hd, D, Q, threads, n, nc);
  if (K == 2) return slots == 1 ? launch_bcc<2, 2, 3, 1>(hd, D, Q, threads, n, nc) : launch_bcc<2, 2, 3, 2>(hd, D, Q, threads, n, nc);
  return slots == 1 ? launch_bcc<1, 2, 3, 1>(hd, D, Q, threads, n, nc) : launch_bcc<1, 2, 3, 2>(hd, D, Q, threads, n, nc);
}

void sweep_bcc_fast(smcx_lattice* hd, int nA, uint64_t seed, int64_t n_sweeps, int n_colours) {
  bccfast::LatDesc D;
  memset(&D, 0, sizeof(D));
  const smcx_sched& sc = hd->sched;
  D.sites = hd->d_sites;
  D.thr = hd->d_thr;
  D.stats = hd->d_stats;
  for (int a = 0; a < 3; a++) {
    D.n[a] = hd->n[a];
    D.nt[a] = sc.nt[a];
  }
  D.L = sc.L;
  D.NQ = bcc_slots_per_axis(hd->n, sc);
  D.nA = nA;
  D.storage = hd->storage;
  D.replica = hd->replica;
  D.seed_lo = (uint32_t)seed;
  D.seed_hi = (uint32_t)(seed >> 32);
  D.sweep = hd->sweep_cum;
  D.proposal = hd->proposal;
  bccfast::Planes Q;
  // 4 shells: every (words, planes) pair is compiled.  2 or 3 shells: one
  // counter word and two planes (M <= 4, |V| < 2^15), else the general
  // variant (two words, three planes); 1 shell: the general variant.
  const int K = hd->shells.K;
  int nw = hd->M <= 4 ? 1 : 2;
  int PL = build_planes(hd, &Q, 2);
  if (K < 4 && !(nw == 1 && PL == 2 && K >= 2)) {
    nw = 2;
    PL = build_planes(hd, &Q, 3);
  }
  int threads, slots;
  bcc_block_shape(D.NQ, hd->bcc_threads, &threads, &slots);

  dispatch(hd, D, Q, nw, PL, threads, slots, n_sweeps, n_colours);
}

}  // namespace smcx
