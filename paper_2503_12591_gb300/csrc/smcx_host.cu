// Host-side geometry, schedule rules, acceptance tables and error plumbing.
#include <math.h>

#include <algorithm>
#include <array>
#include <cstdlib>
#include <stdexcept>

#include "smcx_internal.h"

namespace smcx {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
const std::string& last_error() { return g_last_error; }

void fail(int code, const std::string& msg) { throw SmcxException{code, msg}; }

void check_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return;
  int code = (e == cudaErrorMemoryAllocation) ? SMCX_E_OOM : SMCX_E_CUDA;
  fail(code, std::string(what) + ": " + cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// Lattices.  Positions in half-lattice-constant units; a site is a cubic cell
// (x, y, z) plus a basis vector.
// ---------------------------------------------------------------------------
int sites_per_cell(int kind) { return kind == kBCC ? 2 : (kind == kFCC ? 4 : 0); }

void basis_of(int kind, int b, int out[3]) {
  static const int bcc[2][3] = {{0, 0, 0}, {1, 1, 1}};
  static const int fcc[4][3] = {{0, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
  const int* p = kind == kBCC ? bcc[b] : fcc[b];
  out[0] = p[0];
  out[1] = p[1];
  out[2] = p[2];
}

int basis_index(int kind, int rx, int ry, int rz) {
  for (int b = 0; b < sites_per_cell(kind); b++) {
    int B[3];
    basis_of(kind, b, B);
    if (B[0] == rx && B[1] == ry && B[2] == rz) return b;
  }
  return -1;
}

// The global-memory kernels wrap a neighbour's cell coordinate once; that is
// exact while every shell vector moves at most n[a] cells along axis a.
void check_reach(const Shells& S, const int n[3]) {
  for (int b = 0; b < S.m; b++) {
    int B[3];
    basis_of(S.kind, b, B);
    for (int j = 0; j < S.nv; j++)
      for (int a = 0; a < 3; a++) {
        const int p = B[a] + S.v[j][a];
        const int d = (p >= 0) ? p / 2 : -((-p + 1) / 2);
        if (d > n[a] || -d > n[a]) fail(SMCX_E_INVALID_ARG, "lattice edge shorter than the reach of the shells");
      }
  }
}

Shells make_shells(int kind, int K) {
  Shells s;
  s.kind = kind;
  s.m = sites_per_cell(kind);
  if (s.m == 0) fail(SMCX_E_INVALID_ARG, "unknown lattice kind");
  int kmax = kind == kBCC ? 4 : 3;
  if (K < 1 || K > kmax) fail(SMCX_E_INVALID_ARG, "shell count out of range for this lattice");
  // every lattice vector within 3 cells, keyed by (|v|^2, vx, vy, vz)
  std::vector<std::array<int, 4>> all;
  for (int cx = -3; cx <= 3; cx++)
    for (int cy = -3; cy <= 3; cy++)
      for (int cz = -3; cz <= 3; cz++)
        for (int b = 0; b < s.m; b++) {
          int B[3];
          basis_of(kind, b, B);
          int x = 2 * cx + B[0], y = 2 * cy + B[1], z = 2 * cz + B[2];
          int d2 = x * x + y * y + z * z;
          if (d2) all.push_back({d2, x, y, z});
        }
  std::sort(all.begin(), all.end());
  int shell = -1, prev = 0;
  for (auto& e : all) {
    if (e[0] != prev) {
      shell++;
      prev = e[0];
      if (shell == K) break;
    }
    s.v[s.nv][0] = e[1];
    s.v[s.nv][1] = e[2];
    s.v[s.nv][2] = e[3];
    s.shell_of[s.nv] = shell;
    s.z[shell]++;
    s.nv++;
  }
  s.K = K;
  for (int i = 0; i < s.nv; i++)
    for (int c = 0; c < 3; c++) {
      int a = std::abs(s.v[i][c]);
      s.RK = std::max(s.RK, a);
      if (s.shell_of[i] == 0) s.R1 = std::max(s.R1, a);
    }
  return s;
}

// Two trials whose centres are 2L half-units apart on one axis cannot touch
// each other's read sets when 2L > 2 R1 + RK (each partner moves <= R1, a
// pair-model read reaches <= R1 + RK from the centre).  Under the qSRO model
// a trial also reads the environments of every site whose local energy it
// changes, R1 + 2 RK from its centre, so 2L > 2 R1 + 2 RK.  Across a whole
// tile of g cells the centres are at least 2g + 1 half-units apart.
static int reach_half_units(const Shells& s) { return s.model == 1 ? 2 * s.R1 + 2 * s.RK : 2 * s.R1 + s.RK; }
int min_link_cell(const Shells& s) { return reach_half_units(s) / 2 + 1; }
int min_tile(const Shells& s) { return (reach_half_units(s) - 1) / 2 + 1; }
int halo_cells(const Shells& s) { return (s.R1 + (s.model == 1 ? 2 * s.RK : s.RK) + 1) / 2; }
int ring_cells(const Shells& s) { return (s.R1 + 1) / 2; }

std::string schedule_problem(const Shells& s, const int n[3], const smcx_sched& sc) {
  if (sc.L < min_link_cell(s))
    return "link cell L=" + std::to_string(sc.L) + " is below the interaction reach (needs >= " +
           std::to_string(min_link_cell(s)) + ")";
  bool all_one = sc.nt[0] == 1 && sc.nt[1] == 1 && sc.nt[2] == 1;
  for (int a = 0; a < 3; a++) {
    if (all_one) {
      if (n[a] % sc.L) return "link-cell schedule needs every edge to be a multiple of L";
      // shell vectors must not alias: edges >= 2 R_K / 2 + 1 avoid it
      if (2 * n[a] <= 2 * s.RK) return "lattice edge too small for the link-cell kernel";
    } else {
      if (sc.nt[a] < 2 || sc.nt[a] % 2)
        return "tile counts must be even (>= 2) on every axis, or 1 on all axes";
      if (n[a] / sc.nt[a] < min_tile(s))
        return "tiles thinner than the interaction reach (needs >= " +
               std::to_string(min_tile(s)) + " cells)";
    }
  }
  return "";
}

// Library choice: link cell of 4 (BCC) or the minimum size (FCC); tiles of at most 20 cells (15 for the FCC pair model)
// (the sweep kernel stages (tile + 2 halo)^3 cells in shared memory).  When
// the lattice is too small to tile, the paper's link-cell schedule with the
// smallest L that divides every edge; L = 0 when neither exists.
smcx_sched choose_schedule(const Shells& s, const int n[3]) {
  smcx_sched sc;
  // BCC: L = 4 gives 5^3 = 125 link-cell slots per 20-cell tile (one 128-thread
  // CTA); measured faster than L = 3 on GB300.  FCC keeps the smallest valid L.
  sc.L = s.kind == kBCC ? std::max(min_link_cell(s), 4) : std::max(min_link_cell(s), 3);
  // FCC pair model: tiles of at most 15 cells fit the FCC tile kernel's box
  const int target = (s.kind == kFCC && s.model == 0) ? 15 : 20;
  bool ok = true;
  for (int a = 0; a < 3; a++) {
    int nt = std::max(2, (n[a] + target - 1) / target);  // tiles of at most `target` cells
    if (nt % 2) nt++;
    while (nt > 2 && n[a] / nt < std::max(min_tile(s), 4)) nt -= 2;
    if (n[a] / nt < min_tile(s)) ok = false;
    sc.nt[a] = nt;
  }
  if (ok) return sc;
  sc.nt[0] = sc.nt[1] = sc.nt[2] = 1;
  for (int L = min_link_cell(s); L <= std::min(n[0], std::min(n[1], n[2])); L++) {
    sc.L = L;
    if (schedule_problem(s, n, sc).empty()) return sc;
  }
  sc.L = 0;
  return sc;
}

// F(d) = min(2^32 - 1, floor(2^32 exp(-d * 0.01 meV / (k_B T)))).
static uint32_t boltzmann_fixed(long long d, double beta_q) {
  double e = exp(-((double)d * beta_q));
  double v = e * 4294967296.0;
  if (v >= 4294967295.0) return 4294967295u;
  return (uint32_t)v;
}

int threshold_tables(double T, uint32_t* A, int* nA, uint32_t* B) {
  if (!(T > 0.0)) return -1;
  double beta_q = 0.01 / (kBoltzmannMeV * T);
  int n = 0;
  for (int h = 0; h < kNA; h++) {
    A[h] = boltzmann_fixed((long long)h * kNB, beta_q);
    if (A[h] == 0) {
      for (int r = h + 1; r < kNA; r++) A[r] = 0;
      break;
    }
    n = h + 1;
  }
  for (int l = 0; l < kNB; l++) B[l] = boltzmann_fixed(l, beta_q);
  *nA = n;
  return 0;
}

void species_counts(int M, const double* comp, int64_t N, int64_t* counts) {
  double sum = 0;
  for (int p = 0; p < M; p++) {
    if (!(comp[p] >= 0.0)) fail(SMCX_E_INVALID_ARG, "negative or NaN composition");
    sum += comp[p];
  }
  if (fabs(sum - 1.0) > 1e-9) fail(SMCX_E_INVALID_ARG, "composition does not sum to 1");
  std::vector<double> rem(M);
  int64_t given = 0;
  for (int p = 0; p < M; p++) {
    double x = comp[p] * (double)N;
    double f = floor(x);
    counts[p] = (int64_t)f;
    rem[p] = x - f;
    given += counts[p];
  }
  // largest remainders get the leftover sites; equal remainders favour the
  // lower species index
  for (int64_t left = N - given; left > 0; left--) {
    int best = 0;
    for (int p = 1; p < M; p++)
      if (rem[p] > rem[best]) best = p;
    counts[best]++;
    rem[best] = -1.0;
  }
  for (int64_t left = N - given; left < 0; left++) {
    int best = -1;
    for (int p = 0; p < M; p++)
      if (counts[p] > 0 && (best < 0 || rem[p] < rem[best])) best = p;
    counts[best]--;
    rem[best] = 2.0;
  }
}

}  // namespace smcx
