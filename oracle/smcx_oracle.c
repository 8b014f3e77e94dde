/*
 * smcx_oracle.c -- plain serial CPU reference of the swap-sweep method.
 *
 * TEST INFRASTRUCTURE ONLY (see smcx_oracle.h).  Written for a reader who
 * checks it against the paper by eye: no blocking, no tables beyond what the
 * definitions name, neighbours recomputed from coordinates on every use.
 */
#include "smcx_oracle.h"

#include <math.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <string.h>

/* ------------------------------------------------------------------ */
/* Geometry                                                            */
/* ------------------------------------------------------------------ */

static const int BASIS_BCC[2][3] = {{0, 0, 0}, {1, 1, 1}};
static const int BASIS_FCC[4][3] = {{0, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};

int orc_sites_per_cell(int kind) {
  if (kind == ORC_BCC) return 2;
  if (kind == ORC_FCC) return 4;
  return 0;
}

static const int* basis_vec(int kind, int b) {
  return kind == ORC_BCC ? BASIS_BCC[b] : BASIS_FCC[b];
}

/* basis index of a parity residual (rx,ry,rz) in {0,1}^3, or -1 */
static int basis_index(int kind, int rx, int ry, int rz) {
  int m = orc_sites_per_cell(kind);
  for (int b = 0; b < m; b++) {
    const int* B = basis_vec(kind, b);
    if (B[0] == rx && B[1] == ry && B[2] == rz) return b;
  }
  return -1;
}

typedef struct {
  int v[3];
  int d2;
} hvec;

static int cmp_hvec(const void* pa, const void* pb) {
  const hvec* a = (const hvec*)pa;
  const hvec* b = (const hvec*)pb;
  if (a->d2 != b->d2) return a->d2 < b->d2 ? -1 : 1;
  for (int i = 0; i < 3; i++)
    if (a->v[i] != b->v[i]) return a->v[i] < b->v[i] ? -1 : 1;
  return 0;
}

/* All lattice vectors 2c + basis_b with |c_i| <= 4, sorted by length then
 * lexicographically; the first K distinct lengths are the K shells. */
int orc_shells(int kind, int K, int* z, int* vecs, int max_vecs) {
  int m = orc_sites_per_cell(kind);
  if (m == 0 || K < 1 || K > ORC_KMAX) return -1;
  const int R = 4;
  int cap = (2 * R + 1) * (2 * R + 1) * (2 * R + 1) * m;
  hvec* all = (hvec*)malloc(sizeof(hvec) * (size_t)cap);
  int n = 0;
  for (int cx = -R; cx <= R; cx++)
    for (int cy = -R; cy <= R; cy++)
      for (int cz = -R; cz <= R; cz++)
        for (int b = 0; b < m; b++) {
          const int* B = basis_vec(kind, b);
          hvec h;
          h.v[0] = 2 * cx + B[0];
          h.v[1] = 2 * cy + B[1];
          h.v[2] = 2 * cz + B[2];
          h.d2 = h.v[0] * h.v[0] + h.v[1] * h.v[1] + h.v[2] * h.v[2];
          if (h.d2 == 0) continue;
          all[n++] = h;
        }
  qsort(all, (size_t)n, sizeof(hvec), cmp_hvec);
  int shell = 0, total = 0, prev = -1;
  for (int i = 0; i < n; i++) {
    if (all[i].d2 != prev) {
      if (prev != -1) shell++;
      prev = all[i].d2;
      if (shell >= K) break;
      z[shell] = 0;
    }
    if (total >= max_vecs) {
      free(all);
      return -1;
    }
    vecs[3 * total + 0] = all[i].v[0];
    vecs[3 * total + 1] = all[i].v[1];
    vecs[3 * total + 2] = all[i].v[2];
    z[shell]++;
    total++;
  }
  free(all);
  return total;
}

static int wrapi(int p, int n) {
  int r = p % n;
  return r < 0 ? r + n : r;
}

int64_t orc_neighbour(int kind, int nx, int ny, int nz, int64_t s, const int v[3]) {
  int m = orc_sites_per_cell(kind);
  int b = (int)(s % m);
  int64_t c = s / m;
  int x = (int)(c % nx);
  c /= nx;
  int y = (int)(c % ny);
  int zz = (int)(c / ny);
  const int* B = basis_vec(kind, b);
  int px = wrapi(2 * x + B[0] + v[0], 2 * nx);
  int py = wrapi(2 * y + B[1] + v[1], 2 * ny);
  int pz = wrapi(2 * zz + B[2] + v[2], 2 * nz);
  int bb = basis_index(kind, px & 1, py & 1, pz & 1);
  if (bb < 0) return -1; /* not a lattice vector */
  return (((int64_t)(pz >> 1) * ny + (py >> 1)) * nx + (px >> 1)) * m + bb;
}

/* Shell table of one (kind, K), built on demand. */
typedef struct {
  int K;
  int z[ORC_KMAX];
  int start[ORC_KMAX + 1];
  int v[512][3];
} shells_t;

static int load_shells(int kind, int K, shells_t* S) {
  int tot = orc_shells(kind, K, S->z, &S->v[0][0], 512);
  if (tot < 0) return -1;
  S->K = K;
  S->start[0] = 0;
  for (int k = 0; k < K; k++) S->start[k + 1] = S->start[k] + S->z[k];
  return 0;
}

int orc_check_geometry(int kind, int nx, int ny, int nz, int K) {
  shells_t S;
  if (orc_sites_per_cell(kind) == 0 || nx < 1 || ny < 1 || nz < 1) return -1;
  if (load_shells(kind, K, &S)) return -1;
  for (int i = 0; i < S.start[K]; i++) {
    if (wrapi(S.v[i][0], 2 * nx) == 0 && wrapi(S.v[i][1], 2 * ny) == 0 &&
        wrapi(S.v[i][2], 2 * nz) == 0)
      return -2; /* a shell vector maps every site onto itself */
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random  */
/* numbers: as easy as 1, 2, 3"), written from the published round:   */
/* two 32x32->64 multiplies by M0, M1, a word permutation with key     */
/* xor, and a Weyl key schedule between rounds.                        */
/* ------------------------------------------------------------------ */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; r++) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * c0;
    uint64_t p1 = (uint64_t)M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* Counter of one attempt: pair index j = site >> 1 (words 0..1, replica in
 * the top half of word 1), cumulative sweep index (words 2..3); key = seed.
 * The even site of the pair uses outputs (0,1), the odd site (2,3). */
void orc_attempt_words(uint64_t seed, uint64_t sweep, int replica, int64_t site,
                       uint32_t* rd, uint32_t* ru) {
  uint64_t j = (uint64_t)site >> 1;
  uint32_t ctr[4], key[2], out[4];
  ctr[0] = (uint32_t)j;
  ctr[1] = (uint32_t)(j >> 32) | ((uint32_t)replica << 16);
  ctr[2] = (uint32_t)sweep;
  ctr[3] = (uint32_t)(sweep >> 32);
  key[0] = (uint32_t)seed;
  key[1] = (uint32_t)(seed >> 32);
  orc_philox4x32_10(ctr, key, out);
  if (site & 1) {
    *rd = out[2];
    *ru = out[3];
  } else {
    *rd = out[0];
    *ru = out[1];
  }
}

/* ------------------------------------------------------------------ */
/* Initial configuration: exact composition (largest remainder), then  */
/* species by rank of a 64-bit Philox key per site (ties by site id).  */
/* ------------------------------------------------------------------ */

int orc_species_counts(int M, const double* comp, int64_t N, int64_t* counts) {
  if (M < 1 || M > ORC_MMAX || N < 0) return -1;
  double sum = 0.0;
  for (int p = 0; p < M; p++) {
    if (!(comp[p] >= 0.0)) return -1;
    sum += comp[p];
  }
  if (fabs(sum - 1.0) > 1e-9) return -1;
  double frac[ORC_MMAX];
  int64_t assigned = 0;
  for (int p = 0; p < M; p++) {
    double r = comp[p] * (double)N;
    double f = floor(r);
    counts[p] = (int64_t)f;
    frac[p] = r - f;
    assigned += counts[p];
  }
  int64_t left = N - assigned;
  while (left > 0) {
    int best = -1;
    for (int p = 0; p < M; p++)
      if (best < 0 || frac[p] > frac[best]) best = p; /* ties: lower index */
    counts[best]++;
    frac[best] = -1.0;
    left--;
  }
  while (left < 0) { /* only reachable through rounding of sum != 1 */
    int best = -1;
    for (int p = 0; p < M; p++)
      if (counts[p] > 0 && (best < 0 || frac[p] < frac[best])) best = p;
    counts[best]--;
    frac[best] = 2.0;
    left++;
  }
  return 0;
}

typedef struct {
  uint64_t key;
  int64_t id;
} keyed_t;

static int cmp_keyed(const void* pa, const void* pb) {
  const keyed_t* a = (const keyed_t*)pa;
  const keyed_t* b = (const keyed_t*)pb;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  if (a->id != b->id) return a->id < b->id ? -1 : 1;
  return 0;
}

int orc_init_config(int kind, int nx, int ny, int nz, int M, const double* comp,
                    uint64_t seed, int8_t* sigma) {
  int m = orc_sites_per_cell(kind);
  if (m == 0 || nx < 1 || ny < 1 || nz < 1) return -1;
  int64_t N = (int64_t)nx * ny * nz * m;
  int64_t counts[ORC_MMAX];
  if (orc_species_counts(M, comp, N, counts)) return -1;
  keyed_t* a = (keyed_t*)malloc(sizeof(keyed_t) * (size_t)N);
  if (!a) return -1;
  for (int64_t i = 0; i < N; i++) {
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)((uint64_t)i >> 32), 0u, 0x80000000u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    a[i].key = ((uint64_t)out[0] << 32) | out[1];
    a[i].id = i;
  }
  qsort(a, (size_t)N, sizeof(keyed_t), cmp_keyed);
  int64_t r = 0;
  for (int p = 0; p < M; p++)
    for (int64_t c = 0; c < counts[p]; c++) sigma[a[r++].id] = (int8_t)p;
  free(a);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Energy model (EPI, pair form)                                        */
/* ------------------------------------------------------------------ */

int orc_pair_counts(int kind, int nx, int ny, int nz, int M, int K,
                    const int8_t* sigma, int64_t* C) {
  shells_t S;
  int m = orc_sites_per_cell(kind);
  if (m == 0 || load_shells(kind, K, &S)) return -1;
  int64_t N = (int64_t)nx * ny * nz * m;
  memset(C, 0, sizeof(int64_t) * (size_t)K * M * M);
  for (int64_t s = 0; s < N; s++) {
    int p = sigma[s];
    for (int k = 0; k < K; k++)
      for (int i = S.start[k]; i < S.start[k + 1]; i++) {
        int64_t t = orc_neighbour(kind, nx, ny, nz, s, S.v[i]);
        C[((int64_t)k * M + p) * M + sigma[t]]++;
      }
  }
  return 0;
}

/* E = 1/2 sum over sites i, shells k and vectors v of V_k[s_i][s_{i+v}]:
 * every unordered pair of the pair model counted once (Eq. Total_EPI with
 * the single-site and bias terms dropped at fixed composition). */
int64_t orc_energy(int kind, int nx, int ny, int nz, int M, int K,
                   const int32_t* V, const int8_t* sigma) {
  shells_t S;
  int m = orc_sites_per_cell(kind);
  if (m == 0 || load_shells(kind, K, &S)) return INT64_MIN;
  int64_t N = (int64_t)nx * ny * nz * m;
  int64_t twice = 0;
  for (int64_t s = 0; s < N; s++)
    for (int k = 0; k < K; k++)
      for (int i = S.start[k]; i < S.start[k + 1]; i++) {
        int64_t t = orc_neighbour(kind, nx, ny, nz, s, S.v[i]);
        twice += V[((int64_t)k * M + sigma[s]) * M + sigma[t]];
      }
  return twice / 2;
}

/* Energy change of swapping site s (species a) with its shell-1 neighbour
 * along direction dir (species b), from the environments of the two sites
 * only: for every pair model the other sites' local energies change by the
 * same bond terms, so the change is the bond sum around s and s'. */
static int64_t delta_e_local(int kind, int nx, int ny, int nz, int M, const shells_t* S,
                             const int32_t* V, const int8_t* sigma, int64_t s, int64_t sp) {
  int a = sigma[s], b = sigma[sp];
  int64_t d = 0;
  for (int k = 0; k < S->K; k++)
    for (int i = S->start[k]; i < S->start[k + 1]; i++) {
      int64_t t = orc_neighbour(kind, nx, ny, nz, s, S->v[i]);
      if (t == s || t == sp) continue;
      int c = sigma[t];
      d += (int64_t)V[((int64_t)k * M + b) * M + c] - V[((int64_t)k * M + a) * M + c];
    }
  for (int k = 0; k < S->K; k++)
    for (int i = S->start[k]; i < S->start[k + 1]; i++) {
      int64_t t = orc_neighbour(kind, nx, ny, nz, sp, S->v[i]);
      if (t == s || t == sp) continue;
      int c = sigma[t];
      d += (int64_t)V[((int64_t)k * M + a) * M + c] - V[((int64_t)k * M + b) * M + c];
    }
  return d;
}

int64_t orc_delta_e(int kind, int nx, int ny, int nz, int M, int K,
                    const int32_t* V, const int8_t* sigma, int64_t s, int dir) {
  shells_t S;
  if (load_shells(kind, K, &S)) return INT64_MIN;
  if (dir < 0 || dir >= S.z[0]) return INT64_MIN;
  int64_t sp = orc_neighbour(kind, nx, ny, nz, s, S.v[dir]);
  return delta_e_local(kind, nx, ny, nz, M, &S, V, sigma, s, sp);
}

/* ------------------------------------------------------------------ */
/* qSRO model (Method "The EPI and qSRO model", Eq. quadratic_local_SRO): */
/* the pair terms plus, per site, W_k[s_i] (n_k(i))^2 over the shells,    */
/* where n_k(i) is the number of shell-k neighbours of i with i's own     */
/* species (the same-element pair fraction pi_m^{pp} times z_k).  W is in */
/* 0.01 meV with the 1/z_k^2 of the pair fraction folded in, so every     */
/* energy stays an integer; the regularisation term of the equation is   */
/* a constant for the sampler.                                          */
/* ------------------------------------------------------------------ */
static int64_t qsro_site(int kind, int nx, int ny, int nz, int M, const shells_t* S, const int32_t* W,
                         const int8_t* sigma, int64_t i) {
  int c = sigma[i];
  int64_t q = 0;
  for (int k = 0; k < S->K; k++) {
    int64_t n = 0;
    for (int j = S->start[k]; j < S->start[k + 1]; j++)
      if (sigma[orc_neighbour(kind, nx, ny, nz, i, S->v[j])] == c) n++;
    q += (int64_t)W[k * M + c] * n * n;
  }
  return q;
}

/* The quadratic part of the energy change of swapping s and sp: the sites
 * whose term can change are s, sp and their neighbours over all K shells
 * (each listed once); their terms are summed before and after the swap. */
static int64_t delta_q_local(int kind, int nx, int ny, int nz, int M, const shells_t* S, const int32_t* W,
                             int8_t* sigma, int64_t s, int64_t sp) {
  int64_t U[2 + 2 * 512];
  int nu = 0;
  int64_t cand[2] = {s, sp};
  for (int e = 0; e < 2; e++) {
    int64_t list[1 + 512];
    int nl = 0;
    list[nl++] = cand[e];
    for (int j = 0; j < S->start[S->K]; j++) list[nl++] = orc_neighbour(kind, nx, ny, nz, cand[e], S->v[j]);
    for (int a = 0; a < nl; a++) {
      int dup = 0;
      for (int b = 0; b < nu; b++)
        if (U[b] == list[a]) {
          dup = 1;
          break;
        }
      if (!dup) U[nu++] = list[a];
    }
  }
  int64_t before = 0, after = 0;
  for (int a = 0; a < nu; a++) before += qsro_site(kind, nx, ny, nz, M, S, W, sigma, U[a]);
  int8_t t = sigma[s];
  sigma[s] = sigma[sp];
  sigma[sp] = t;
  for (int a = 0; a < nu; a++) after += qsro_site(kind, nx, ny, nz, M, S, W, sigma, U[a]);
  sigma[sp] = sigma[s];
  sigma[s] = t;
  return after - before;
}

int64_t orc_energy_qsro(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, const int32_t* W,
                        const int8_t* sigma) {
  shells_t S;
  int m = orc_sites_per_cell(kind);
  if (m == 0 || load_shells(kind, K, &S)) return INT64_MIN;
  int64_t N = (int64_t)nx * ny * nz * m;
  int64_t e = orc_energy(kind, nx, ny, nz, M, K, V, sigma);
  for (int64_t i = 0; i < N; i++) e += qsro_site(kind, nx, ny, nz, M, &S, W, sigma, i);
  return e;
}

int64_t orc_delta_e_qsro(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, const int32_t* W,
                         int8_t* sigma, int64_t s, int dir) {
  shells_t S;
  if (load_shells(kind, K, &S)) return INT64_MIN;
  if (dir < 0 || dir >= S.z[0]) return INT64_MIN;
  int64_t sp = orc_neighbour(kind, nx, ny, nz, s, S.v[dir]);
  return delta_e_local(kind, nx, ny, nz, M, &S, V, sigma, s, sp) +
         delta_q_local(kind, nx, ny, nz, M, &S, W, sigma, s, sp);
}

/* Warren-Cowley SRO over ordered pairs: alpha = 1 - C_k[p][q]/(z_k N_p c_q),
 * c_q = N_q/N; 0 where a species is absent. */
int orc_sro(int kind, int nx, int ny, int nz, int M, int K, const int8_t* sigma,
            double* alpha) {
  shells_t S;
  int m = orc_sites_per_cell(kind);
  if (m == 0 || load_shells(kind, K, &S)) return -1;
  int64_t N = (int64_t)nx * ny * nz * m;
  int64_t* C = (int64_t*)malloc(sizeof(int64_t) * (size_t)K * M * M);
  int64_t Np[ORC_MMAX] = {0};
  for (int64_t s = 0; s < N; s++) Np[sigma[s]]++;
  orc_pair_counts(kind, nx, ny, nz, M, K, sigma, C);
  for (int k = 0; k < K; k++)
    for (int p = 0; p < M; p++)
      for (int q = 0; q < M; q++) {
        double denom = (double)S.z[k] * (double)Np[p] * ((double)Np[q] / (double)N);
        double v = 0.0;
        if (denom > 0.0) v = 1.0 - (double)C[((int64_t)k * M + p) * M + q] / denom;
        alpha[((int64_t)k * M + p) * M + q] = v;
      }
  free(C);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Metropolis acceptance: P = 1 for dE <= 0, exp(-beta dE) otherwise,   */
/* realised as u < thr(dE) with a 32-bit uniform u and                 */
/*   F(d)    = min(2^32-1, floor(2^32 exp(-d * 0.01 meV / (kB T))))    */
/*   thr(dE) = (A[dE >> 10] * B[dE & 1023]) >> 32,                     */
/*   A[h] = F(1024 h), B[l] = F(l); thr = 0 once A reaches 0.          */
/* ------------------------------------------------------------------ */

static uint32_t fixed_boltzmann(int64_t d, double beta_q) {
  double e = exp(-((double)d * beta_q));
  double v = e * 4294967296.0;
  if (v >= 4294967295.0) return 4294967295u;
  return (uint32_t)v;
}

int orc_threshold_tables(double T, uint32_t* A, int* nA, uint32_t* B) {
  if (!(T > 0.0)) return -1;
  double beta_q = 0.01 / (ORC_KB_MEV * T);
  int n = 0;
  for (int h = 0; h < ORC_NA_MAX; h++) {
    uint32_t a = fixed_boltzmann((int64_t)h * ORC_NB, beta_q);
    A[h] = a;
    if (a == 0) break;
    n = h + 1;
  }
  for (int h = n; h < ORC_NA_MAX; h++) A[h] = 0;
  for (int l = 0; l < ORC_NB; l++) B[l] = fixed_boltzmann(l, beta_q);
  *nA = n;
  return 0;
}

uint32_t orc_threshold(const uint32_t* A, int nA, const uint32_t* B, int64_t dE) {
  if (dE < 0) return 0xFFFFFFFFu;
  int64_t h = dE >> 10;
  if (h >= nA) return 0;
  return (uint32_t)(((uint64_t)A[h] * (uint64_t)B[dE & (ORC_NB - 1)]) >> 32);
}

/* ------------------------------------------------------------------ */
/* Schedule: generalized checkerboard.                                  */
/*   Each axis is cut into nt tiles (sizes differ by at most one, the   */
/*   first n % nt tiles one larger).  Tile colour = parity of the tile  */
/*   index on each axis (8 colours).  Inside a tile, the intra colour   */
/*   of a site is ((z-z0) mod L, (y-y0) mod L, (x-x0) mod L, b), i.e.   */
/*   its place in an L^3 link cell measured from the tile origin.  A    */
/*   sweep visits tile colours 0..7, and inside each the n_A = L^3 m    */
/*   intra colours in the order ic = ((cz L + cy) L + cx) m + b.  With  */
/*   one tile on every axis this is the paper's link-cell schedule.     */
/* ------------------------------------------------------------------ */

/* Largest |component| over shell-1 vectors (R1) and over shells 1..K (RK). */
static void reaches(const shells_t* S, int* R1, int* RK) {
  *R1 = 0;
  *RK = 0;
  for (int i = 0; i < S->start[S->K]; i++)
    for (int c = 0; c < 3; c++) {
      int a = abs(S->v[i][c]);
      if (a > *RK) *RK = a;
      if (i < S->z[0] && a > *R1) *R1 = a;
    }
}

/* model 0 (pair model): a trial reads the sites within R1 + RK of its
 * centre; model 1 (qSRO): within R1 + 2 RK (the environments of every site
 * whose local energy the swap changes).  A concurrent trial writes within R1
 * of its own centre, so two trials of one phase must be more than
 * reach = 2 R1 + RK (model 0) or 2 R1 + 2 RK (model 1) half units apart
 * along some axis. */
int orc_schedule_check_model(int kind, int nx, int ny, int nz, int K, int L, int ntx, int nty, int ntz, int model) {
  shells_t S;
  if (orc_sites_per_cell(kind) == 0 || load_shells(kind, K, &S)) return -1;
  if (orc_check_geometry(kind, nx, ny, nz, K)) return -1;
  if (model != 0 && model != 1) return -1;
  if (L == 0) return 0; /* serial */
  int R1, RK;
  reaches(&S, &R1, &RK);
  int reach = model == 1 ? 2 * R1 + 2 * RK : 2 * R1 + RK;
  /* same intra colour: half-unit separation >= 2L on some axis */
  int Lmin = reach / 2 + 1;
  /* same tile colour, different tiles: a whole tile of g cells between
   * them, half-unit separation >= 2g + 1. */
  int gmin = (reach - 1) / 2 + 1;
  if (L < Lmin) return -2;
  int n[3] = {nx, ny, nz}, nt[3] = {ntx, nty, ntz};
  for (int a = 0; a < 3; a++) {
    if (nt[a] < 1) return -2;
    if (nt[a] == 1) {
      if (n[a] % L) return -2;
    } else {
      if (nt[a] % 2) return -2;
      if (n[a] / nt[a] < gmin) return -2;
    }
  }
  return 0;
}

int orc_schedule_check(int kind, int nx, int ny, int nz, int K, int L,
                       int ntx, int nty, int ntz) {
  return orc_schedule_check_model(kind, nx, ny, nz, K, L, ntx, nty, ntz, 0);
}

static void tile_bounds(int n, int nt, int i, int* start, int* size) {
  int base = n / nt, rem = n % nt;
  *size = base + (i < rem ? 1 : 0);
  *start = i * base + (i < rem ? i : rem);
}

static int tile_of(int n, int nt, int x) {
  for (int i = 0; i < nt; i++) {
    int st, sz;
    tile_bounds(n, nt, i, &st, &sz);
    if (x >= st && x < st + sz) return i;
  }
  return -1;
}

int64_t orc_phase_of(int kind, int nx, int ny, int nz, int L, int ntx, int nty,
                     int ntz, int64_t s, int* tile) {
  int m = orc_sites_per_cell(kind);
  if (L == 0) return -1;
  int b = (int)(s % m);
  int64_t c = s / m;
  int x = (int)(c % nx);
  c /= nx;
  int y = (int)(c % ny);
  int z = (int)(c / ny);
  int ix = tile_of(nx, ntx, x), iy = tile_of(ny, nty, y), iz = tile_of(nz, ntz, z);
  int x0, y0, z0, sz;
  tile_bounds(nx, ntx, ix, &x0, &sz);
  tile_bounds(ny, nty, iy, &y0, &sz);
  tile_bounds(nz, ntz, iz, &z0, &sz);
  int tc = (ix & 1) | ((iy & 1) << 1) | ((iz & 1) << 2);
  int64_t nA = (int64_t)L * L * L * m;
  int64_t ic = ((((int64_t)((z - z0) % L) * L + (y - y0) % L) * L + (x - x0) % L) * m) + b;
  if (tile) {
    tile[0] = ix;
    tile[1] = iy;
    tile[2] = iz;
  }
  return tc * nA + ic;
}

typedef struct {
  int kind, nx, ny, nz, m, M;
  const shells_t* S;
  const int32_t* V;
  int8_t* sigma;
  const uint32_t *A, *B;
  int nA;
  uint64_t seed, sweep;
  int replica;
  int64_t* stats;
  const int32_t* W; /* qSRO weights [K][M], NULL for the pair model */
} attempt_ctx;

/* One canonical swap trial at site s (Supplementary "Monte Carlo
 * Simulation Algorithms"): partner = a uniformly chosen shell-1 neighbour,
 * energy change from the two sites' environments, Metropolis acceptance. */
static void attempt_dir(attempt_ctx* c, int64_t s, int forced_dir) {
  uint32_t rd, ru;
  orc_attempt_words(c->seed, c->sweep, c->replica, s, &rd, &ru);
  int z1 = c->S->z[0];
  int dir = forced_dir >= 0 ? forced_dir : (int)(((uint64_t)rd * (uint64_t)z1) >> 32);
  int64_t sp = orc_neighbour(c->kind, c->nx, c->ny, c->nz, s, c->S->v[dir]);
  c->stats[0]++;
  int a = c->sigma[s], b = c->sigma[sp];
  if (a == b) {
    c->stats[2]++;
    return;
  }
  int64_t dE = delta_e_local(c->kind, c->nx, c->ny, c->nz, c->M, c->S, c->V, c->sigma, s, sp);
  if (c->W) dE += delta_q_local(c->kind, c->nx, c->ny, c->nz, c->M, c->S, c->W, c->sigma, s, sp);
  int accept = 0;
  if (dE <= 0)
    accept = 1;
  else if (ru < orc_threshold(c->A, c->nA, c->B, dE))
    accept = 1;
  if (accept) {
    c->sigma[s] = (int8_t)b;
    c->sigma[sp] = (int8_t)a;
    c->stats[1]++;
    c->stats[3] += dE;
  }
}

static void attempt(attempt_ctx* c, int64_t s) { attempt_dir(c, s, -1); }

/* Shared-direction proposals: one shell-1 direction per (sweep, tile, intra
 * colour ic), drawn from Philox with counter (tile index, (ic >> 1) |
 * replica << 16, sweep lo, sweep hi | 2^30) and key = seed, output word 0 for
 * even ic and word 2 for odd ic; the acceptance uniforms stay per site.
 * Every trial of a phase is still a symmetric proposal (the swap along a
 * fixed vector is its own inverse), so each phase keeps detailed balance. */
int orc_phase_direction(uint64_t seed, uint64_t sweep, int replica, int64_t tile, int ic, int z1) {
  uint32_t ctr[4] = {(uint32_t)tile, ((uint32_t)ic >> 1) | ((uint32_t)replica << 16), (uint32_t)sweep,
                     (uint32_t)(sweep >> 32) | 0x40000000u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t o[4];
  orc_philox4x32_10(ctr, key, o);
  return (int)(((uint64_t)((ic & 1) ? o[2] : o[0]) * (uint64_t)z1) >> 32);
}

/* Block-shared proposals (mode 2): one shell-1 direction per (sweep, tile
 * colour tc, block, intra colour ic), where a block is a pair of tiles of one
 * colour: the tiles of colour tc are numbered j = (jz * ncy + jy) * ncx + jx
 * with j_a = tile index >> 1 and nc_a the colour's tile count on axis a, and
 * block = j >> 1 (the last block of an odd count holds one tile).  Philox
 * counter (block | tc << 28, (ic >> 1) | replica << 16, sweep lo, sweep hi |
 * 2^29), key = seed; word 0 for even ic, word 2 for odd ic.  As in mode 1,
 * every trial is a symmetric proposal along a state-independent vector. */
int orc_block_direction(uint64_t seed, uint64_t sweep, int replica, int tc, int64_t block, int ic, int z1) {
  uint32_t ctr[4] = {(uint32_t)block | ((uint32_t)tc << 28), ((uint32_t)ic >> 1) | ((uint32_t)replica << 16),
                     (uint32_t)sweep, (uint32_t)(sweep >> 32) | 0x20000000u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t o[4];
  orc_philox4x32_10(ctr, key, o);
  return (int)(((uint64_t)((ic & 1) ? o[2] : o[0]) * (uint64_t)z1) >> 32);
}

/* block index (mode 2) of tile (ix, iy, iz) among the tiles of its colour */
static int64_t tile_block(int ntx, int nty, int ix, int iy, int iz) {
  const int ncx = (ntx + 1 - (ix & 1)) / 2, ncy = (nty + 1 - (iy & 1)) / 2;
  const int64_t j = ((int64_t)(iz >> 1) * ncy + (iy >> 1)) * ncx + (ix >> 1);
  return j >> 1;
}

/* forced direction of a phase of tile (ix, iy, iz), or -1 (mode 0) */
static int phase_dir(int proposal, uint64_t seed, uint64_t sweep, int replica, int ntx, int nty, int ix, int iy,
                     int iz, int ic, int z1) {
  const int tc = (ix & 1) | ((iy & 1) << 1) | ((iz & 1) << 2);
  if (proposal == 1) return orc_phase_direction(seed, sweep, replica, ((int64_t)iz * nty + iy) * ntx + ix, ic, z1);
  if (proposal == 2) return orc_block_direction(seed, sweep, replica, tc, tile_block(ntx, nty, ix, iy, iz), ic, z1);
  return -1;
}

/* All intra-colour phases of ONE tile (tile indices tx, ty, tz) of sweep
 * `sweep`: the part of the sweep loop below that belongs to this tile.  Tiles
 * of one colour never interact, so on that tile (and its partner ring) the
 * result equals the whole colour pass. */
static int tile_pass_impl(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, const int32_t* W,
                          int8_t* sigma, double T, uint64_t seed, uint64_t sweep, int replica, int L, int ntx,
                          int nty, int ntz, int tx, int ty, int tz, int64_t* stats, int proposal);

int orc_tile_pass(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V,
                  int8_t* sigma, double T, uint64_t seed, uint64_t sweep, int replica,
                  int L, int ntx, int nty, int ntz, int tx, int ty, int tz, int64_t* stats) {
  return tile_pass_impl(kind, nx, ny, nz, M, K, V, NULL, sigma, T, seed, sweep, replica, L, ntx, nty, ntz, tx, ty,
                        tz, stats, 0);
}

/* orc_tile_pass with proposal mode 0, 1 or 2. */
int orc_tile_pass_proposal(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, int8_t* sigma,
                           double T, uint64_t seed, uint64_t sweep, int replica, int L, int ntx, int nty, int ntz,
                           int tx, int ty, int tz, int64_t* stats, int proposal) {
  if (proposal < 0 || proposal > 2) return -2;
  return tile_pass_impl(kind, nx, ny, nz, M, K, V, NULL, sigma, T, seed, sweep, replica, L, ntx, nty, ntz, tx, ty,
                        tz, stats, proposal);
}

/* orc_tile_pass for the qSRO model (W [K][M]). */
int orc_tile_pass_qsro(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, const int32_t* W,
                       int8_t* sigma, double T, uint64_t seed, uint64_t sweep, int replica, int L, int ntx, int nty,
                       int ntz, int tx, int ty, int tz, int64_t* stats) {
  return tile_pass_impl(kind, nx, ny, nz, M, K, V, W, sigma, T, seed, sweep, replica, L, ntx, nty, ntz, tx, ty, tz,
                        stats, 0);
}

static int tile_pass_impl(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, const int32_t* W,
                          int8_t* sigma, double T, uint64_t seed, uint64_t sweep, int replica, int L, int ntx,
                          int nty, int ntz, int tx, int ty, int tz, int64_t* stats, int proposal) {
  shells_t S;
  int m = orc_sites_per_cell(kind);
  if (m == 0 || load_shells(kind, K, &S)) return -1;
  if (orc_schedule_check_model(kind, nx, ny, nz, K, L, ntx, nty, ntz, W ? 1 : 0) || L == 0) return -2;
  if (tx < 0 || tx >= ntx || ty < 0 || ty >= nty || tz < 0 || tz >= ntz) return -1;
  uint32_t* A = (uint32_t*)malloc(sizeof(uint32_t) * ORC_NA_MAX);
  uint32_t* B = (uint32_t*)malloc(sizeof(uint32_t) * ORC_NB);
  int nA;
  if (!A || !B || orc_threshold_tables(T, A, &nA, B)) {
    free(A);
    free(B);
    return -1;
  }
  attempt_ctx c;
  c.kind = kind;
  c.nx = nx;
  c.ny = ny;
  c.nz = nz;
  c.m = m;
  c.M = M;
  c.S = &S;
  c.V = V;
  c.sigma = sigma;
  c.A = A;
  c.B = B;
  c.nA = nA;
  c.seed = seed;
  c.replica = replica;
  c.stats = stats;
  c.W = W;
  c.sweep = sweep;
  stats[0] = stats[1] = stats[2] = stats[3] = 0;
  int x0, sx, y0, sy, z0, sz;
  tile_bounds(nx, ntx, tx, &x0, &sx);
  tile_bounds(ny, nty, ty, &y0, &sy);
  tile_bounds(nz, ntz, tz, &z0, &sz);
  for (int ic = 0; ic < L * L * L * m; ic++) {
    int b = ic % m;
    int cx = (ic / m) % L, cy = (ic / m / L) % L, cz = ic / m / L / L;
    const int fd = phase_dir(proposal, seed, sweep, replica, ntx, nty, tx, ty, tz, ic, S.z[0]);
    for (int z = z0 + cz; z < z0 + sz; z += L)
      for (int y = y0 + cy; y < y0 + sy; y += L)
        for (int x = x0 + cx; x < x0 + sx; x += L) attempt_dir(&c, (((int64_t)z * ny + y) * nx + x) * m + b, fd);
  }
  free(A);
  free(B);
  return 0;
}

/* Species of sampled sites in the initial configuration of a lattice too
 * large to sort here: each sample's rank among all N keys (ties by id) is
 * counted in one pass and mapped through the species counts. */
int orc_init_sample(int kind, int nx, int ny, int nz, int M, const double* comp, uint64_t seed,
                    const int64_t* ids, int n_ids, int8_t* out) {
  int m = orc_sites_per_cell(kind);
  if (m == 0 || n_ids < 1 || n_ids > 64) return -1;
  int64_t N = (int64_t)nx * ny * nz * m;
  int64_t counts[ORC_MMAX];
  if (orc_species_counts(M, comp, N, counts)) return -1;
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint64_t skey[64];
  int64_t rank[64];
  for (int j = 0; j < n_ids; j++) {
    uint32_t ctr[4] = {(uint32_t)ids[j], (uint32_t)((uint64_t)ids[j] >> 32), 0u, 0x80000000u};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    skey[j] = ((uint64_t)o[0] << 32) | o[1];
    rank[j] = 0;
  }
  for (int64_t i = 0; i < N; i++) {
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)((uint64_t)i >> 32), 0u, 0x80000000u};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    uint64_t k = ((uint64_t)o[0] << 32) | o[1];
    for (int j = 0; j < n_ids; j++)
      if (k < skey[j] || (k == skey[j] && i < ids[j])) rank[j]++;
  }
  for (int j = 0; j < n_ids; j++) {
    int64_t r = rank[j], acc = 0;
    int p = 0;
    for (p = 0; p < M; p++) {
      acc += counts[p];
      if (r < acc) break;
    }
    out[j] = (int8_t)p;
  }
  return 0;
}

static int sweep_impl(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V,
                      int8_t* sigma, double T, int64_t n_sweeps, uint64_t seed,
                      uint64_t sweep0, int replica, int L, int ntx, int nty, int ntz,
                      int64_t* stats, int proposal, int n_threads, const int32_t* W);

int orc_sweep(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V,
              int8_t* sigma, double T, int64_t n_sweeps, uint64_t seed,
              uint64_t sweep0, int replica, int L, int ntx, int nty, int ntz,
              int64_t* stats) {
  return sweep_impl(kind, nx, ny, nz, M, K, V, sigma, T, n_sweeps, seed, sweep0, replica, L, ntx, nty, ntz,
                    stats, 0, 1, NULL);
}

int orc_sweep_proposal(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V,
                       int8_t* sigma, double T, int64_t n_sweeps, uint64_t seed,
                       uint64_t sweep0, int replica, int L, int ntx, int nty, int ntz,
                       int64_t* stats, int proposal) {
  if (proposal != 0 && ((proposal != 1 && proposal != 2) || L == 0)) return -2;
  return sweep_impl(kind, nx, ny, nz, M, K, V, sigma, T, n_sweeps, seed, sweep0, replica, L, ntx, nty, ntz,
                    stats, proposal, 1, NULL);
}

/* The same sweep with the sites of each phase split across n_threads OpenMP
 * threads (n_threads <= 0: the OpenMP default).  Sites of one phase are
 * independent, so the result equals the serial sweep's bit for bit.  The
 * serial schedule (L = 0) stays serial.  Returns the thread count used in
 * *used (1 when built without OpenMP). */
int orc_sweep_parallel(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V,
                       int8_t* sigma, double T, int64_t n_sweeps, uint64_t seed,
                       uint64_t sweep0, int replica, int L, int ntx, int nty, int ntz,
                       int64_t* stats, int n_threads, int* used) {
#ifdef _OPENMP
  int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#else
  int nt = 1;
  (void)n_threads;
#endif
  if (L == 0) nt = 1;
  if (used) *used = nt;
  return sweep_impl(kind, nx, ny, nz, M, K, V, sigma, T, n_sweeps, seed, sweep0, replica, L, ntx, nty, ntz,
                    stats, 0, nt, NULL);
}

/* orc_sweep_parallel with proposal mode 0, 1 or 2 (identical to the serial
 * orc_sweep_proposal). */
int orc_sweep_parallel_proposal(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, int8_t* sigma,
                                double T, int64_t n_sweeps, uint64_t seed, uint64_t sweep0, int replica, int L,
                                int ntx, int nty, int ntz, int64_t* stats, int n_threads, int* used, int proposal) {
#ifdef _OPENMP
  int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#else
  int nt = 1;
  (void)n_threads;
#endif
  if (proposal < 0 || proposal > 2 || (proposal != 0 && L == 0)) return -2;
  if (L == 0) nt = 1;
  if (used) *used = nt;
  return sweep_impl(kind, nx, ny, nz, M, K, V, sigma, T, n_sweeps, seed, sweep0, replica, L, ntx, nty, ntz,
                    stats, proposal, nt, NULL);
}

/* Sweep of the qSRO model (W [K][M], see qsro_site); the schedule is checked
 * against the qSRO read reach. */
int orc_sweep_qsro(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, const int32_t* W,
                   int8_t* sigma, double T, int64_t n_sweeps, uint64_t seed, uint64_t sweep0, int replica, int L,
                   int ntx, int nty, int ntz, int64_t* stats) {
  return sweep_impl(kind, nx, ny, nz, M, K, V, sigma, T, n_sweeps, seed, sweep0, replica, L, ntx, nty, ntz,
                    stats, 0, 1, W);
}

/* One sweep of the link-cell / tile schedule with each phase's sites listed
 * in the serial loop's order and split across threads; every thread keeps its
 * own statistics, summed at the end (integer sums: order-free). */
static void sweep_phases_parallel(const attempt_ctx* c0, int L, int ntx, int nty, int ntz, uint64_t sweep0,
                                  int64_t n_sweeps, int n_threads, int proposal) {
  const int m = c0->m, nx = c0->nx, ny = c0->ny, nz = c0->nz;
  const int64_t N = (int64_t)nx * ny * nz * m;
  int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
  int8_t* fdir = (int8_t*)malloc((size_t)(N > 0 ? N : 1));
  int64_t tot[4] = {0, 0, 0, 0};
  int nA_ic = L * L * L * m;
  for (int64_t n = 0; n < n_sweeps; n++) {
    uint64_t sw = sweep0 + (uint64_t)n;
    for (int tc = 0; tc < 8; tc++)
      for (int ic = 0; ic < nA_ic; ic++) {
        int b = ic % m;
        int cx = (ic / m) % L, cy = (ic / m / L) % L, cz = ic / m / L / L;
        int64_t cnt = 0;
        for (int iz = 0; iz < ntz; iz++)
          for (int iy = 0; iy < nty; iy++)
            for (int ix = 0; ix < ntx; ix++) {
              if (((ix & 1) | ((iy & 1) << 1) | ((iz & 1) << 2)) != tc) continue;
              int x0, sx, y0, sy, z0, sz;
              tile_bounds(nx, ntx, ix, &x0, &sx);
              tile_bounds(ny, nty, iy, &y0, &sy);
              tile_bounds(nz, ntz, iz, &z0, &sz);
              const int fd = phase_dir(proposal, c0->seed, sw, c0->replica, ntx, nty, ix, iy, iz, ic, c0->S->z[0]);
              for (int z = z0 + cz; z < z0 + sz; z += L)
                for (int y = y0 + cy; y < y0 + sy; y += L)
                  for (int x = x0 + cx; x < x0 + sx; x += L) {
                    fdir[cnt] = (int8_t)fd;
                    list[cnt++] = (((int64_t)z * ny + y) * nx + x) * m + b;
                  }
            }
        int64_t t0 = 0, t1 = 0, t2 = 0, t3 = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(n_threads) reduction(+ : t0, t1, t2, t3)
#endif
        {
          attempt_ctx c = *c0;
          int64_t st[4] = {0, 0, 0, 0};
          c.stats = st;
          c.sweep = sw;
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
          for (int64_t i = 0; i < cnt; i++) attempt_dir(&c, list[i], fdir[i]);
          t0 += st[0];
          t1 += st[1];
          t2 += st[2];
          t3 += st[3];
        }
        tot[0] += t0;
        tot[1] += t1;
        tot[2] += t2;
        tot[3] += t3;
      }
  }
  for (int i = 0; i < 4; i++) c0->stats[i] += tot[i];
  free(list);
  free(fdir);
}

static int sweep_impl(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V,
                      int8_t* sigma, double T, int64_t n_sweeps, uint64_t seed,
                      uint64_t sweep0, int replica, int L, int ntx, int nty, int ntz,
                      int64_t* stats, int proposal, int n_threads, const int32_t* W) {
  shells_t S;
  int m = orc_sites_per_cell(kind);
  if (m == 0 || load_shells(kind, K, &S)) return -1;
  if (orc_schedule_check_model(kind, nx, ny, nz, K, L, ntx, nty, ntz, W ? 1 : 0)) return -2;
  uint32_t* A = (uint32_t*)malloc(sizeof(uint32_t) * ORC_NA_MAX);
  uint32_t* B = (uint32_t*)malloc(sizeof(uint32_t) * ORC_NB);
  int nA;
  if (!A || !B || orc_threshold_tables(T, A, &nA, B)) {
    free(A);
    free(B);
    return -1;
  }
  attempt_ctx c;
  c.kind = kind;
  c.nx = nx;
  c.ny = ny;
  c.nz = nz;
  c.m = m;
  c.M = M;
  c.S = &S;
  c.V = V;
  c.sigma = sigma;
  c.A = A;
  c.B = B;
  c.nA = nA;
  c.seed = seed;
  c.replica = replica;
  c.stats = stats;
  c.W = W;
  stats[0] = stats[1] = stats[2] = stats[3] = 0;
  int64_t N = (int64_t)nx * ny * nz * m;
  if (n_threads > 1) {
    sweep_phases_parallel(&c, L, ntx, nty, ntz, sweep0, n_sweeps, n_threads, proposal);
    free(A);
    free(B);
    return 0;
  }
  for (int64_t n = 0; n < n_sweeps; n++) {
    c.sweep = sweep0 + (uint64_t)n;
    if (L == 0) {
      for (int64_t s = 0; s < N; s++) attempt(&c, s);
      continue;
    }
    int nA_ic = L * L * L * m;
    for (int tc = 0; tc < 8; tc++)
      for (int ic = 0; ic < nA_ic; ic++) {
        int b = ic % m;
        int cx = (ic / m) % L, cy = (ic / m / L) % L, cz = ic / m / L / L;
        for (int iz = 0; iz < ntz; iz++)
          for (int iy = 0; iy < nty; iy++)
            for (int ix = 0; ix < ntx; ix++) {
              if (((ix & 1) | ((iy & 1) << 1) | ((iz & 1) << 2)) != tc) continue;
              int x0, sx, y0, sy, z0, sz;
              tile_bounds(nx, ntx, ix, &x0, &sx);
              tile_bounds(ny, nty, iy, &y0, &sy);
              tile_bounds(nz, ntz, iz, &z0, &sz);
              const int fd = phase_dir(proposal, seed, c.sweep, replica, ntx, nty, ix, iy, iz, ic, S.z[0]);
              for (int z = z0 + cz; z < z0 + sz; z += L)
                for (int y = y0 + cy; y < y0 + sy; y += L)
                  for (int x = x0 + cx; x < x0 + sx; x += L)
                    attempt_dir(&c, (((int64_t)z * ny + y) * nx + x) * m + b, fd);
            }
      }
  }
  free(A);
  free(B);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Replica exchange between temperature slots (Supplementary           */
/* "Parallelization opportunities": configurations at different        */
/* temperatures are exchanged with a rule that keeps detailed balance). */
/*   Slot t holds temperature T_slot[t] and replica slot_rep[t].  Round */
/*   r pairs the slots (t, t+1) with t = r mod 2, r mod 2 + 2, ...  The */
/*   swap of the replicas a (slot t) and c (slot t+1) multiplies the    */
/*   joint Boltzmann weight by exp(x), x = (beta_t - beta_{t+1})        */
/*   (E_a - E_c), beta = 1/(k_B T); it is accepted when x >= 0, else    */
/*   when u < floor(2^32 exp(x)) (capped at 2^32 - 1), with u word 0 of */
/*   Philox(counter (t, r lo, r hi, 0xC0000000), key = seed).  Energies */
/*   are in 0.01 meV.                                                   */
/* ------------------------------------------------------------------ */
int orc_exchange_round(int R, const double* T_slot, const int64_t* E, int32_t* slot_rep, uint64_t round,
                       uint64_t seed, int64_t* accepts) {
  for (int t = 0; t < R; t++)
    if (!(T_slot[t] > 0.0)) return -1;
  for (int t = (int)(round & 1); t + 1 < R; t += 2) {
    int a = slot_rep[t], c = slot_rep[t + 1];
    double bt = 1.0 / (ORC_KB_MEV * T_slot[t]);
    double bu = 1.0 / (ORC_KB_MEV * T_slot[t + 1]);
    double x = (bt - bu) * ((double)(E[a] - E[c]) * 0.01);
    uint32_t ctr[4] = {(uint32_t)t, (uint32_t)round, (uint32_t)(round >> 32), 0xC0000000u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    int accept = 0;
    if (x >= 0.0) {
      accept = 1;
    } else {
      double v = exp(x) * 4294967296.0;
      uint32_t thr = v >= 4294967295.0 ? 4294967295u : (uint32_t)v;
      accept = o[0] < thr;
    }
    if (accept) {
      slot_rep[t] = c;
      slot_rep[t + 1] = a;
      if (accepts) accepts[t]++;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Local-energy field and clusters (Results, FeCoNiAlTi one-billion-    */
/* atom section; Method "MC simulation": the local energy of every site */
/* is computed, an energy threshold decides which sites go together,    */
/* and union-find collects the clusters).                               */
/*   e2[i] = 2 E_i = sum_k sum_{v in shell k} V_k[s_i][s_{i+v}], so the  */
/*   local energies (Eq. Linear_EPI without bias terms) add up to E.    */
/*   Site class = (e2[i] < thr2).  Two shell-1 neighbours of one class  */
/*   are in one cluster; a cluster is labelled by its smallest site id. */
/* ------------------------------------------------------------------ */
int orc_local_energy2(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, const int8_t* sigma,
                      int64_t* e2) {
  shells_t S;
  int m = orc_sites_per_cell(kind);
  if (m == 0 || load_shells(kind, K, &S)) return -1;
  int64_t N = (int64_t)nx * ny * nz * m;
  for (int64_t s = 0; s < N; s++) {
    int64_t acc = 0;
    for (int k = 0; k < K; k++)
      for (int i = S.start[k]; i < S.start[k + 1]; i++) {
        int64_t t = orc_neighbour(kind, nx, ny, nz, s, S.v[i]);
        acc += V[((int64_t)k * M + sigma[s]) * M + sigma[t]];
      }
    e2[s] = acc;
  }
  return 0;
}

/* Under the qSRO model the local energy also carries the site's quadratic
 * term: e2[i] += 2 sum_k W[k][s_i] n_k(i)^2, so that sum_i e2[i] = 2 E
 * still holds for the qSRO energy. */
int orc_local_energy2_qsro(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, const int32_t* W,
                           const int8_t* sigma, int64_t* e2) {
  shells_t S;
  int m = orc_sites_per_cell(kind);
  if (m == 0 || load_shells(kind, K, &S)) return -1;
  if (orc_local_energy2(kind, nx, ny, nz, M, K, V, sigma, e2)) return -1;
  int64_t N = (int64_t)nx * ny * nz * m;
  for (int64_t i = 0; i < N; i++) e2[i] += 2 * qsro_site(kind, nx, ny, nz, M, &S, W, sigma, i);
  return 0;
}

/* e2 of the sites ids[0..n-1] only (same definition, for lattices too large
 * to evaluate whole). */
int orc_local_energy2_sample(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, const int8_t* sigma,
                             const int64_t* ids, int64_t n, int64_t* e2) {
  shells_t S;
  int m = orc_sites_per_cell(kind);
  if (m == 0 || load_shells(kind, K, &S)) return -1;
  for (int64_t j = 0; j < n; j++) {
    int64_t s = ids[j];
    int64_t acc = 0;
    for (int k = 0; k < K; k++)
      for (int i = S.start[k]; i < S.start[k + 1]; i++) {
        int64_t t = orc_neighbour(kind, nx, ny, nz, s, S.v[i]);
        acc += V[((int64_t)k * M + sigma[s]) * M + sigma[t]];
      }
    e2[j] = acc;
  }
  return 0;
}

/* Breadth-first search from every unvisited site in increasing id order:
 * the start of each search is the smallest id of its cluster. */
static int clusters_impl(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, const int32_t* W,
                         const int8_t* sigma, int64_t thr2, int64_t* labels, int64_t* n_clusters) {
  shells_t S;
  int m = orc_sites_per_cell(kind);
  if (m == 0 || load_shells(kind, K, &S)) return -1;
  int64_t N = (int64_t)nx * ny * nz * m;
  int64_t* e2 = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
  int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
  if (!e2 || !queue) {
    free(e2);
    free(queue);
    return -1;
  }
  if (W)
    orc_local_energy2_qsro(kind, nx, ny, nz, M, K, V, W, sigma, e2);
  else
    orc_local_energy2(kind, nx, ny, nz, M, K, V, sigma, e2);
  for (int64_t s = 0; s < N; s++) labels[s] = -1;
  int64_t nc = 0;
  for (int64_t s0 = 0; s0 < N; s0++) {
    if (labels[s0] >= 0) continue;
    nc++;
    int cls = e2[s0] < thr2;
    int64_t head = 0, tail = 0;
    queue[tail++] = s0;
    labels[s0] = s0;
    while (head < tail) {
      int64_t s = queue[head++];
      for (int i = S.start[0]; i < S.start[1]; i++) {
        int64_t t = orc_neighbour(kind, nx, ny, nz, s, S.v[i]);
        if (labels[t] >= 0 || (e2[t] < thr2) != cls) continue;
        labels[t] = s0;
        queue[tail++] = t;
      }
    }
  }
  *n_clusters = nc;
  free(e2);
  free(queue);
  return 0;
}

int orc_clusters(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, const int8_t* sigma,
                 int64_t thr2, int64_t* labels, int64_t* n_clusters) {
  return clusters_impl(kind, nx, ny, nz, M, K, V, NULL, sigma, thr2, labels, n_clusters);
}

/* Clusters from the qSRO local energies. */
int orc_clusters_qsro(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, const int32_t* W,
                      const int8_t* sigma, int64_t thr2, int64_t* labels, int64_t* n_clusters) {
  return clusters_impl(kind, nx, ny, nz, M, K, V, W, sigma, thr2, labels, n_clusters);
}

/* ------------------------------------------------------------------ */
/* Specific heat from energy fluctuations                              */
/* ------------------------------------------------------------------ */

/* C_V / (N k_B) = Var(E) / (N (k_B T)^2) with E converted from 0.01 meV to
 * meV and k_B in meV/K (Results, Fig. C_V; Method "MC simulation"). */
int orc_specific_heat(const int64_t* E, const double* w, int64_t n, int64_t N, double T, double* out) {
  if (n < 1 || N < 1 || !(T > 0.0)) return -1;
  double wsum = 0.0, mean = 0.0;
  for (int64_t i = 0; i < n; i++) {
    const double wi = w ? w[i] : 1.0;
    wsum += wi;
    mean += wi * (double)E[i];
  }
  if (!(wsum > 0.0)) return -1;
  mean /= wsum;
  double var = 0.0;
  for (int64_t i = 0; i < n; i++) {
    const double wi = w ? w[i] : 1.0;
    const double d = (double)E[i] - mean;
    var += wi * d * d;
  }
  var /= wsum;
  const double var_mev2 = var * 0.01 * 0.01;
  const double kT = ORC_KB_MEV * T;
  out[0] = mean;
  out[1] = var;
  out[2] = var_mev2 / ((double)N * kT * kT);
  return 0;
}
