/*
 * smcx_oracle.h -- plain serial CPU reference of the swap-sweep method.
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists so that the CUDA path can be
 * checked against an independent, obviously-correct implementation.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or constant generator with the CUDA
 * library: the geometry, the Philox generator, the Metropolis threshold table,
 * the schedule and the energy arithmetic are all written out again here.
 *
 * Paper: Liu et al., "Revealing Nanostructures in High-Entropy Alloys via
 * Machine-Learning Accelerated Scalable Monte Carlo Simulation" (SMC-X).
 *   - EPI energy model: Method "The EPI and qSRO model", Eqs. Linear_EPI and
 *     Total_EPI.
 *   - Pairwise energy change of a swap from the two swapped sites only:
 *     same section, the paragraph after Eq. Total_EPI.
 *   - Metropolis acceptance and canonical swap trial: Supplementary
 *     "Monte Carlo Simulation Algorithms" (acceptance equation).
 *   - Sweep = one trial per lattice site: same section; also Method
 *     "Theoretical speedup".
 *   - Link-cell generalized checkerboard: Results "Performance of the SMC-X
 *     algorithm" and Method "Implementation of SMC-GPU" (link-cell size item).
 *
 * Parity status of every function is stated beside it.  Every function is
 * pinned by a test under tests/ against something other than itself.
 *
 * Conventions (readings of the paper, all listed in the design notes):
 *   - positions in half-lattice-constant integer units; BCC basis (0,0,0),
 *     (1,1,1); FCC basis (0,0,0),(1,1,0),(1,0,1),(0,1,1);
 *   - canonical site id = ((z*ny + y)*nx + x)*m + b;
 *   - shells: lattice vectors grouped by length, ascending; within a shell
 *     in ascending lexicographic (vx, vy, vz) order;
 *   - V is int32 in units of 0.01 meV, [K][M][M], symmetric;
 *   - E = 1/2 sum_i sum_k sum_{v in shell k} V_k[s_i][s_{i+v}]  (exact int64).
 */
#ifndef SMCX_ORACLE_H
#define SMCX_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_BCC 0
#define ORC_FCC 1
#define ORC_KMAX 8
#define ORC_MMAX 15
#define ORC_NA_MAX 4096      /* high-part entries of the acceptance table */
#define ORC_NB 1024          /* low-part entries (10 bits) */

/* Boltzmann constant in meV/K (exact SI value 1.380649e-23 J/K). */
#define ORC_KB_MEV 8.617333262e-2

/* ---- geometry (pinned: textbook coordination numbers, closed-form energies) */
int orc_sites_per_cell(int kind);
/* Enumerate the first K shells; z[k] = size of shell k, vecs = concatenated
 * (vx,vy,vz) triples (half units).  Returns total vector count, or -1. */
int orc_shells(int kind, int K, int* z, int* vecs, int max_vecs);
/* Neighbour of site s along half-unit vector v with periodic wrap. */
int64_t orc_neighbour(int kind, int nx, int ny, int nz, int64_t s, const int v[3]);
/* 0 if no shell vector of the first K shells maps a site onto itself. */
int orc_check_geometry(int kind, int nx, int ny, int nz, int K);

/* ---- Philox4x32-10 (pinned: ATen's philox_engine run on the same inputs) */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Random words of one attempt at `site` (direction word rd, uniform word ru). */
void orc_attempt_words(uint64_t seed, uint64_t sweep, int replica, int64_t site,
                       uint32_t* rd, uint32_t* ru);

/* ---- initial configuration (pinned: numpy lexsort of the same keys) */
int orc_species_counts(int M, const double* comp, int64_t N, int64_t* counts);
int orc_init_config(int kind, int nx, int ny, int nz, int M, const double* comp,
                    uint64_t seed, int8_t* sigma);

/* ---- energy model (pinned: B2 / L1_2 / pure-element closed forms,
 *      row-sum identity, brute-force E(after)-E(before)) */
int orc_pair_counts(int kind, int nx, int ny, int nz, int M, int K,
                    const int8_t* sigma, int64_t* C /*[K][M][M]*/);
int64_t orc_energy(int kind, int nx, int ny, int nz, int M, int K,
                   const int32_t* V, const int8_t* sigma);
int64_t orc_delta_e(int kind, int nx, int ny, int nz, int M, int K,
                    const int32_t* V, const int8_t* sigma, int64_t s, int dir);
int orc_sro(int kind, int nx, int ny, int nz, int M, int K, const int8_t* sigma,
            double* alpha /*[K][M][M]*/);

/* ---- acceptance table (pinned: closed-form exp and its limits) */
int orc_threshold_tables(double T, uint32_t* A /*[ORC_NA_MAX]*/, int* nA,
                         uint32_t* B /*[ORC_NB]*/);
uint32_t orc_threshold(const uint32_t* A, int nA, const uint32_t* B, int64_t dE);

/* ---- schedule and sweep (pinned: exact enumeration of the canonical
 *      distribution, split-sweep identity, brute-force phase independence) */
/* L == 0 selects the serial schedule (canonical site order). */
int orc_schedule_check(int kind, int nx, int ny, int nz, int K, int L,
                       int ntx, int nty, int ntz);
int orc_sweep(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V,
              int8_t* sigma, double T, int64_t n_sweeps, uint64_t seed,
              uint64_t sweep0, int replica, int L, int ntx, int nty, int ntz,
              int64_t* stats /*[4]: attempts, accepts, same-species,
                                 sum of accepted dE*/);
/* Sweep with a proposal mode: 0 = a uniform shell-1 direction per trial
 * (orc_sweep), 1 = one shared direction per (sweep, tile, intra colour),
 * see orc_phase_direction.  Mode 1 needs a checkerboard schedule (L > 0). */
int orc_sweep_proposal(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V,
                       int8_t* sigma, double T, int64_t n_sweeps, uint64_t seed,
                       uint64_t sweep0, int replica, int L, int ntx, int nty, int ntz,
                       int64_t* stats, int proposal);

/* orc_sweep with each phase split across OpenMP threads (identical result;
 * n_threads <= 0 = OpenMP default; *used = threads used, 1 without OpenMP
 * or for the serial schedule L = 0). */
int orc_sweep_parallel(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V,
                       int8_t* sigma, double T, int64_t n_sweeps, uint64_t seed,
                       uint64_t sweep0, int replica, int L, int ntx, int nty, int ntz,
                       int64_t* stats, int n_threads, int* used);
int orc_phase_direction(uint64_t seed, uint64_t sweep, int replica, int64_t tile, int ic, int z1);
/* All phases of one tile (tx, ty, tz) of sweep `sweep` (stats as orc_sweep). */
int orc_tile_pass(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V,
                  int8_t* sigma, double T, uint64_t seed, uint64_t sweep, int replica,
                  int L, int ntx, int nty, int ntz, int tx, int ty, int tz, int64_t* stats);
/* Initial species of up to 64 sampled sites of a lattice too large to sort
 * (one pass over all N keys). */
int orc_init_sample(int kind, int nx, int ny, int nz, int M, const double* comp, uint64_t seed,
                    const int64_t* ids, int n_ids, int8_t* out);
/* Phase id of a site under schedule (L, nt*): tile colour * nA + intra colour,
 * or -1 for the serial schedule.  Used by the independence test. */
int64_t orc_phase_of(int kind, int nx, int ny, int nz, int L, int ntx, int nty,
                     int ntz, int64_t s, int* tile /*[3] out, may be NULL*/);

/* One replica-exchange round: slot pairs (t, t+1), t = round mod 2, +2, ...;
 * slot_rep [R] in/out (replica at each slot), E [R] energies by replica
 * (0.01 meV), accepts [R-1] incremented per accepted slot pair. */
int orc_exchange_round(int R, const double* T_slot, const int64_t* E, int32_t* slot_rep, uint64_t round,
                       uint64_t seed, int64_t* accepts);

/* Twice the local energy of every site, e2 [N] (0.01 meV):
 * e2[i] = sum_k sum_{v in shell k} V_k[s_i][s_{i+v}]; sum_i e2[i] = 2 E. */
int orc_local_energy2(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, const int8_t* sigma,
                      int64_t* e2);

/* e2 under the qSRO model: the pair value + 2 sum_k W[k][s_i] n_k(i)^2. */
int orc_local_energy2_qsro(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, const int32_t* W,
                           const int8_t* sigma, int64_t* e2);

/* orc_clusters with the qSRO local energies. */
int orc_clusters_qsro(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, const int32_t* W,
                      const int8_t* sigma, int64_t thr2, int64_t* labels, int64_t* n_clusters);

/* e2 of the listed sites only: e2 [n] for ids [n]. */
int orc_local_energy2_sample(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, const int8_t* sigma,
                             const int64_t* ids, int64_t n, int64_t* e2);

/* Clusters: class(i) = e2[i] < thr2; shell-1 neighbours of one class are
 * connected; labels [N] = smallest site id of the cluster; *n_clusters. */
int orc_clusters(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, const int8_t* sigma,
                 int64_t thr2, int64_t* labels, int64_t* n_clusters);

/* qSRO model (Eq. quadratic_local_SRO, integer form): E = pair energy +
 * sum_i sum_k W[k][s_i] n_k(i)^2, n_k(i) = shell-k neighbours of i with i's
 * species; W [K][M] in 0.01 meV. */
int64_t orc_energy_qsro(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, const int32_t* W,
                        const int8_t* sigma);
/* Energy change of swapping s with its shell-1 neighbour dir (sigma is
 * restored before returning). */
int64_t orc_delta_e_qsro(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, const int32_t* W,
                         int8_t* sigma, int64_t s, int dir);
/* Schedule check for model 0 (pair) or 1 (qSRO: larger read reach). */
int orc_schedule_check_model(int kind, int nx, int ny, int nz, int K, int L, int ntx, int nty, int ntz, int model);
/* orc_tile_pass for the qSRO model. */
int orc_tile_pass_qsro(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, const int32_t* W,
                       int8_t* sigma, double T, uint64_t seed, uint64_t sweep, int replica, int L, int ntx, int nty,
                       int ntz, int tx, int ty, int tz, int64_t* stats);
/* orc_sweep for the qSRO model. */
int orc_sweep_qsro(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, const int32_t* W,
                   int8_t* sigma, double T, int64_t n_sweeps, uint64_t seed, uint64_t sweep0, int replica, int L,
                   int ntx, int nty, int ntz, int64_t* stats);

/* Block-shared proposals (mode 2): the shell-1 direction shared by the tiles
 * of one block (a pair of consecutive tiles of colour tc) in phase ic. */
int orc_block_direction(uint64_t seed, uint64_t sweep, int replica, int tc, int64_t block, int ic, int z1);
/* orc_tile_pass / orc_sweep_parallel with a proposal mode (0, 1, 2). */
int orc_tile_pass_proposal(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, int8_t* sigma,
                           double T, uint64_t seed, uint64_t sweep, int replica, int L, int ntx, int nty, int ntz,
                           int tx, int ty, int tz, int64_t* stats, int proposal);
int orc_sweep_parallel_proposal(int kind, int nx, int ny, int nz, int M, int K, const int32_t* V, int8_t* sigma,
                                double T, int64_t n_sweeps, uint64_t seed, uint64_t sweep0, int replica, int L,
                                int ntx, int nty, int ntz, int64_t* stats, int n_threads, int* used, int proposal);

/* Specific heat from energy fluctuations (Results, Fig. C_V; Method "MC
 * simulation"; Supplementary "Statistical mechanics" for the canonical
 * average).  The canonical fluctuation formula
 *   C_V / (N k_B) = (<E^2> - <E>^2) / (N (k_B T)^2),
 * where <.> averages the n energies E[i] (0.01 meV units) with weights w[i]
 * (w = NULL: weight 1 each, the time average over a recorded trace; else,
 * e.g., Boltzmann weights of enumerated states; they need not sum to 1).
 * Two passes in double: the weighted mean, then the weighted mean squared
 * deviation from it.  out[0] = <E> (0.01 meV), out[1] = <E^2> - <E>^2
 * ((0.01 meV)^2), out[2] = C_V / (N k_B) (per site, k_B units).
 * Returns 0, or -1 for n < 1, N < 1, T <= 0 or a non-positive weight sum.
 * Pinned: equals d<E>/dT / (N k_B) of an exactly enumerated canonical
 * average (16-site box) and the two-level closed form. */
int orc_specific_heat(const int64_t* E, const double* w, int64_t n, int64_t N, double T, double* out);

#ifdef __cplusplus
}
#endif
#endif
