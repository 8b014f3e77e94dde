/*
 * smcx.h -- C ABI of the GB300 (sm_103a) swap-sweep library for SMC-X.
 *
 * Method: Liu et al., "Revealing Nanostructures in High-Entropy Alloys via
 * Machine-Learning Accelerated Scalable Monte Carlo Simulation" (SMC-X,
 * SMC-GPU).  The library runs the canonical-ensemble (fixed composition)
 * Metropolis swap sweep of an effective-pair-interaction (EPI) lattice model
 * on one GPU:
 *   - energy model: EPI over K neighbour shells (Method "The EPI and qSRO
 *     model", Eq. Linear_EPI, Eq. Total_EPI), pair form
 *       E = 1/2 sum_i sum_k sum_{v in shell k} V_k[s_i][s_{i+v}],
 *     V in int32 units of 0.01 meV, so every energy is an exact integer;
 *   - trial: swap a site with a uniformly chosen nearest neighbour (Results
 *     "Performance of the SMC-X algorithm"; Supplementary "Monte Carlo
 *     Simulation Algorithms", canonical swap);
 *   - energy change from the two swapped sites' environments only (Method
 *     "The EPI and qSRO model", paragraph after Eq. Total_EPI);
 *   - Metropolis acceptance P = min(1, exp(-beta dE)) (Supplementary, the
 *     acceptance equation), realised as u < thr(dE) with a 32-bit uniform u
 *     and an integer table thr computed on the host in double precision:
 *       F(d) = min(2^32-1, floor(2^32 exp(-d 0.01 meV / (k_B T)))),
 *       thr(d) = (A[d >> 10] * B[d & 1023]) >> 32, A[h] = F(1024 h), B[l] = F(l);
 *   - sweep = one trial per site (Supplementary, sweep definition), ordered by
 *     the generalized checkerboard (Results "Performance of the SMC-X
 *     algorithm"; Method "Implementation of SMC-GPU", link-cell item) in its
 *     tiled form described at smcx_sched;
 *   - trial random numbers: Philox4x32-10 (the paper uses cuRAND, Method
 *     "Implementation of SMC-GPU", random-number item) with counter
 *     (pair index j = site >> 1, replica << 16 | j >> 32, sweep lo, sweep hi)
 *     and key = seed; the even site of a pair uses outputs (0,1), the odd
 *     site (2,3); direction = floor(word0 * z1 / 2^32), u = word1.
 *
 * Conventions
 *   - Lattices: SMCX_BCC (2 sites per cubic cell, basis (0,0,0),(1/2,1/2,1/2))
 *     and SMCX_FCC (4 sites, basis (0,0,0),(1/2,1/2,0),(1/2,0,1/2),(0,1/2,1/2));
 *     dimensions "nx x ny x nz x m" as in Tab. models_summary; periodic.
 *   - Canonical site id = ((z*ny + y)*nx + x)*m + b.
 *   - Shells: lattice vectors grouped by length; inside a shell in ascending
 *     lexicographic order of the half-lattice-unit components.
 *   - Every call returns an int status: SMCX_OK (0) or a negative SMCX_E_*
 *     code; smcx_last_error() gives a message for the calling thread.  No
 *     C++ exception crosses the ABI.
 *   - Ownership: a lattice handle owns all device memory it allocates; host
 *     arrays passed in are owned by the caller and read or written only
 *     during the call.  Work is ordered on the handle's CUDA stream; calls
 *     that return host data synchronise that stream before returning;
 *     smcx_sweep only enqueues.  A handle must not be used by two threads at
 *     once.
 *   - No CPU fallback: every compute call runs CUDA kernels and fails with
 *     SMCX_E_CUDA when no device is usable.
 */
#ifndef SMCX_H
#define SMCX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define SMCX_OK 0
#define SMCX_E_INVALID_ARG (-1) /* a bad argument value or a NULL pointer      */
#define SMCX_E_NO_EPI (-2)      /* sweep/energy before smcx_set_epi            */
#define SMCX_E_SCHEDULE (-3)    /* no valid checkerboard for this lattice      */
#define SMCX_E_CUDA (-4)        /* a CUDA runtime error (message has details)  */
#define SMCX_E_OOM (-5)         /* device allocation failed                    */
#define SMCX_E_TIMEOUT (-6)     /* a bounded device wait gave up               */
#define SMCX_E_RANGE (-7)       /* |dE| of this EPI table may overflow int32   */
#define SMCX_E_UNSUPPORTED (-8) /* valid request this library does not run     */

/* ---- enumerations ---------------------------------------------------- */
#define SMCX_BCC 0
#define SMCX_FCC 1
#define SMCX_INT8 0    /* one int8 species id per site                        */
#define SMCX_PACKED4 1 /* two 4-bit ids per byte, byte = site pair (id >> 1)  */
#define SMCX_NA_MAX 4096 /* entries of the high-part acceptance table A       */
#define SMCX_NB 1024     /* entries of the low-part acceptance table B        */

/*
 * Checkerboard schedule (Results "Performance of the SMC-X algorithm":
 * link cells of n_A sites; trials at the same i_A in different link cells are
 * independent when the link cell is larger than the interaction reach).
 *
 * Each axis is cut into nt[a] tiles whose sizes differ by at most one (the
 * first n % nt tiles are one cell larger).  Tile colour = parity of the tile
 * index on each axis.  Inside a tile, a site's intra colour is its place in
 * an L^3 link cell counted from the tile origin, ic = ((cz L + cy) L + cx) m + b.
 * A sweep runs tile colours 0..7 in order and, inside each, the L^3 m intra
 * colours in order; all trials of one (tile colour, intra colour) phase are
 * independent, and trials in different tiles of one tile colour are
 * independent whatever their intra colour, so tiles of one colour may run
 * concurrently at different intra colours.
 *   - nt = {1,1,1}: the paper's link-cell schedule (n_A sequential steps of
 *     n_C parallel trials); every n must be a multiple of L.
 *   - otherwise every nt must be even (>= 2) and every tile at least as thick
 *     as the interaction reach requires (3 cells for BCC <= 4 shells).
 * L must exceed the reach: L >= 3 for BCC with 2..4 shells and FCC with 2..3.
 * Passing NULL (or L == 0) asks the library to choose; its choice is L == 0
 * ("none") for lattices too small for any valid schedule, in which case the
 * handle works for configuration I/O and observables but smcx_sweep returns
 * SMCX_E_SCHEDULE.
 */
typedef struct smcx_sched {
  int32_t L;
  int32_t nt[3];
} smcx_sched;

typedef struct smcx_lattice smcx_lattice;

/* Message of the last failed call on this thread ("" if none).  The string is
 * owned by the library and valid until the next call on this thread. */
const char* smcx_last_error(void);

/* ABI version (major * 10000 + minor * 100 + patch). */
int smcx_version(void);

/*
 * Create a lattice with an exact-composition initial configuration.
 *   kind      SMCX_BCC or SMCX_FCC;  nx, ny, nz >= 1 cubic cells.
 *   M         species count, 1 <= M <= 15 (PACKED4) or 127 (INT8); the sweep
 *             kernels of this library run M <= 8.
 *   comp      [M] fractions summing to 1; counts are floor(c_p N) plus one for
 *             the largest remainders (ties to the lower index).
 *   init_seed species are placed by the rank of a 64-bit Philox key per site
 *             (counter (id lo, id hi, 0, 2^31), key init_seed; ties by id): the
 *             paper's random initial configuration (Results, FeCoNiAlTi
 *             section), made exactly reproducible.
 *   storage   SMCX_INT8 or SMCX_PACKED4.
 *   sched     schedule (see smcx_sched) or NULL for the library's choice.
 *   stream    a cudaStream_t (NULL = legacy default stream) that orders all
 *             work of the handle.
 * Returns SMCX_E_SCHEDULE if no valid schedule exists for these dimensions,
 * SMCX_E_OOM if the device buffers cannot be allocated.
 */
int smcx_lattice_create(smcx_lattice** out, int kind, int nx, int ny, int nz, int M,
                        const double* comp, uint64_t init_seed, int storage,
                        const smcx_sched* sched, void* stream);

/*
 * Make a handle over a lattice store the caller already holds on the device
 * (e.g. the storage of a framework tensor), without copying it.
 *   d_sites   16-byte aligned device (or managed) pointer to the species of the N sites in
 *             canonical site order, in the layout of `storage`: one byte per
 *             site (SMCX_INT8) or two sites per byte, the even site in the
 *             low nibble (SMCX_PACKED4).  The caller keeps ownership; the
 *             buffer must outlive the handle, and nothing else may write it
 *             while the handle's stream has work queued on it.
 *   bytes     size of the buffer; at least N (INT8) or N/2 (PACKED4) bytes.
 *   other arguments as for smcx_lattice_create (no composition or seed: the
 *   configuration is the buffer's).
 * Every stored id is checked on the device: SMCX_E_INVALID_ARG if one is
 * >= M, if the buffer is too small or is not device memory.  The handle
 * sweeps, measures and reads/writes the configuration in place;
 * smcx_lattice_destroy frees the handle's own buffers, not d_sites.
 */
int smcx_lattice_wrap(smcx_lattice** out, int kind, int nx, int ny, int nz, int M, void* d_sites,
                      size_t bytes, int storage, const smcx_sched* sched, void* stream);

/* Release the handle and its device memory (synchronises its stream). */
int smcx_lattice_destroy(smcx_lattice* h);

/*
 * Set the EPI table V[K][M][M] (int32, 0.01 meV units), copied by the call.
 * V must be symmetric in its species indices (Eq. Total_EPI sums unordered
 * pairs).  K ranges over 1..4 (BCC) or 1..3 (FCC).  Returns SMCX_E_RANGE when
 * the largest possible |dE| would not fit int32, SMCX_E_SCHEDULE when the
 * handle's schedule is too small for the new interaction reach.
 */
int smcx_set_epi(smcx_lattice* h, int K, const int32_t* V);

/*
 * qSRO model (Method "The EPI and qSRO model", Eq. quadratic_local_SRO), in
 * integer form: E = the pair energy of smcx_set_epi + sum_i sum_k
 * W[k][s_i] n_k(i)^2, where n_k(i) is the number of shell-k neighbours of
 * site i with i's own species (the same-element pair fraction of the
 * equation times z_k; W carries the 1/z_k^2) and W [K][M] is in 0.01 meV,
 * K the shell count of the current EPI table.  The equation's regularisation
 * term is a constant for the sampler and is not represented.
 *   W = NULL returns to the pair model; smcx_set_epi also does.
 * A trial then reads R1 + 2 R_K around its centre (the environments of every
 * site whose term it changes), so the schedule needs larger link cells and
 * tiles (FCC, 3 shells: L >= 4); the automatic schedule is re-chosen, an
 * explicit one re-checked (SMCX_E_SCHEDULE).  qSRO sweeps run tiled
 * schedules (>= 2 tiles per axis) with per-trial directions; smcx_energy
 * includes the quadratic term.  SMCX_E_NO_EPI before smcx_set_epi;
 * SMCX_E_RANGE if |dE| could overflow int32.
 */
int smcx_set_qsro(smcx_lattice* h, const int32_t* W);

/* Kernel family used by smcx_sweep.  SMCX_KERNEL_AUTO (default) picks the
 * fastest kernel that supports the lattice (the shared-memory BCC kernel for
 * BCC with M <= 8 and tiles <= 20 cells); SMCX_KERNEL_GENERIC forces the
 * generic tiled kernel (or the link-cell kernel for the paper's schedule).
 * Both give bit-identical trajectories. */
#define SMCX_KERNEL_AUTO 0
#define SMCX_KERNEL_GENERIC 1
int smcx_set_kernel(smcx_lattice* h, int which);

/* Philox replica id of the handle (0..65535, default 0): counter word 1
 * carries it in bits 16..31, so replicas with equal seeds draw independent
 * streams.  A handle swept alone with replica id r follows exactly the
 * trajectory it follows as replica r of a batch. */
int smcx_set_replica(smcx_lattice* h, int replica);

/* Proposal mode.  SMCX_PROPOSAL_SITE (default): every trial draws its own
 * shell-1 direction (the reading of the paper: a random nearest neighbour per
 * trial).  SMCX_PROPOSAL_TILE: one direction per (sweep, tile, intra
 * colour ic), drawn from Philox with counter (tile index, (ic >> 1) |
 * replica << 16, sweep lo, sweep hi | 2^30) and key = seed, output word 0 for
 * even ic and word 2 for odd ic, where tile index = (tz * nt[1] + ty) * nt[0]
 * + tx (0 for the link-cell schedule); acceptance uniforms stay per trial.  Each trial is still a symmetric proposal, so every
 * phase keeps detailed balance and the canonical distribution is unchanged;
 * trials of a phase move along the same vector, which lets the BCC kernel
 * fetch the two environments as one compile-time union.
 * SMCX_PROPOSAL_BLOCK: one direction per (sweep, tile colour tc, block, intra
 * colour ic), where a block is a pair of consecutive tiles of colour tc (the
 * colour's tiles numbered j = (jz * ncy + jy) * ncx + jx, j_a = tile index >>
 * 1, nc_a = the colour's tile count on axis a; block = j >> 1): Philox counter
 * (block | tc << 28, (ic >> 1) | replica << 16, sweep lo, sweep hi | 2^29),
 * key = seed, word 0 for even ic and word 2 for odd ic.  The proposals are
 * keyed by (seed, sweep, colour, block); the two tiles of a block share their
 * directions (each tile still runs in its own CTA).  The shared-direction
 * modes run on the BCC tile kernels (single-lattice and batched) when the
 * table has 4 shells, M <= 4 and |V| < 2^15, on the FCC tile kernel when it
 * has 3 shells and M = 5, or M <= 4 with |V| < 2^15, else on the generic
 * tile kernel; qSRO sweeps run SMCX_PROPOSAL_SITE only. */
#define SMCX_PROPOSAL_SITE 0
#define SMCX_PROPOSAL_TILE 1
#define SMCX_PROPOSAL_BLOCK 2
int smcx_set_proposal(smcx_lattice* h, int mode);

/* Threads per CTA of the BCC shared-memory kernel (0 = one thread per
 * link-cell slot; else a multiple of 32 up to 512).  Performance only. */
int smcx_set_block(smcx_lattice* h, int threads);

/* Replace the schedule (NULL = library's choice).  The trajectory depends on
 * it: equal schedules give bit-identical results. */
int smcx_set_schedule(smcx_lattice* h, const smcx_sched* sched);
int smcx_get_schedule(const smcx_lattice* h, smcx_sched* out);

/*
 * Enqueue n_sweeps >= 0 sweeps at temperature T (kelvin, > 0) with Philox
 * seed `seed`.  The Philox counter uses the handle's cumulative sweep index,
 * so sweep(T, a, s); sweep(T, b, s) equals sweep(T, a + b, s).  Asynchronous.
 */
int smcx_sweep(smcx_lattice* h, double T, int64_t n_sweeps, uint64_t seed);

/*
 * Pick the fastest schedule for this lattice and model by measurement: for
 * link cells from the model's minimum to 5 and tiles of about 10..20 cells
 * (and, for the BCC tile kernel, 0/128/256 threads per CTA), time `trial`
 * (1..64) sweeps at temperature T on a snapshot of the configuration.  The
 * configuration, statistics and sweep counter are restored; the fastest
 * schedule and block size are installed (as if set explicitly) and returned
 * in *out / *threads (either may be NULL).  Small lattices leave most SMs idle
 * with the default 20-cell tiles; this is the remedy.  Needs N bytes of
 * temporary device memory.  SMCX_E_SCHEDULE if no candidate fits.
 */
int smcx_autotune(smcx_lattice* h, double T, int trial, smcx_sched* out, int* threads);

/*
 * n_sweeps sweeps as smcx_sweep, recording the exact energy after each one in
 * E [n_sweeps] (host, int64, 0.01 meV) -- the series that energy-fluctuation
 * observables such as the specific heat C_V = Var(E) / (k_B T^2) (Results,
 * Fig. C_V) are computed from.  One energy pass at the start; after every
 * sweep a one-thread kernel writes E_0 + (accepted dE since the start) into a
 * device buffer that is read once at the end, so the host never waits
 * between sweeps.  n_sweeps <= 2^24; temporary device memory 8 (n_sweeps + 1)
 * bytes.
 */
int smcx_sweep_energies(smcx_lattice* h, double T, int64_t n_sweeps, uint64_t seed, int64_t* E);

/*
 * Specific heat from energy fluctuations (Results, Fig. C_V; Method "MC
 * simulation": C_V from the energies recorded over the sweeps at one
 * temperature).  Runs n_sweeps (1..2^24) sweeps as smcx_sweep_energies,
 * recording the exact energy after each one on the device, and reduces that
 * trace on the device in FP64 (two passes: mean, then mean squared deviation)
 * to the canonical fluctuation formula
 *   moments[0] = <E>                  (0.01 meV),
 *   moments[1] = <E^2> - <E>^2        ((0.01 meV)^2),
 *   moments[2] = C_V / (N k_B) = (<E^2> - <E>^2) / (N (k_B T)^2)
 * with E in meV and k_B = 8.617333262e-2 meV/K; <.> is the average over the
 * n_sweeps recorded energies.  moments: host double[3], required.  E: host
 * int64[n_sweeps] receiving the trace, or NULL.  Synchronous on return.
 * Temporary device memory 8 (n_sweeps + 4) bytes.  Errors as
 * smcx_sweep_energies; SMCX_E_INVALID_ARG for n_sweeps < 1 or NULL moments.
 */
int smcx_sweep_cv(smcx_lattice* h, double T, int64_t n_sweeps, uint64_t seed, int64_t* E, double* moments);

/* Verification hook: run tile colours 0..n_colours-1 (0..8) of sweep number
 * `cumulative sweep index` without advancing the index, i.e. the first part
 * of the next smcx_sweep.  Tiles of one colour never interact, so after one
 * colour every tile of colour 0 can be compared with an independent
 * single-tile computation even on a lattice too large to sweep elsewhere.
 * Needs a tiled schedule (SMCX_E_UNSUPPORTED for the link-cell schedule). */
int smcx_sweep_partial(smcx_lattice* h, double T, uint64_t seed, int n_colours);

/* Exact total energy (0.01 meV units) of the current configuration. */
int smcx_energy(smcx_lattice* h, int64_t* E);

/* Ordered pair counts C[k][p][q] = #{(i, v in shell k): s_i = p, s_{i+v} = q}
 * (int64, K*M*M entries, symmetric); E = 1/2 sum V*C. */
int smcx_pair_counts(smcx_lattice* h, int64_t* C);

/* Warren-Cowley SRO over ordered pairs, alpha_k[p][q] = 1 - C_k[p][q] /
 * (z_k N_p c_q), c_q = N_q / N (0 where a species is absent); the local
 * fraction of Method Eq. quadratic_local_SRO summed over the lattice. */
int smcx_sro(smcx_lattice* h, double* alpha);

/*
 * Local-energy field and clusters (Results, FeCoNiAlTi one-billion-atom
 * section; Method "MC simulation": the local energy of every site, an energy
 * threshold, union-find over neighbouring sites).  Need smcx_set_epi; the
 * local energies must fit int32 (sum_k z_k max|V_k| < 2^31, else
 * SMCX_E_RANGE).  All three are enqueued on the handle's stream and return
 * after it has finished.
 *
 * smcx_local_energy: d_e2 (device, [N] int32, caller-owned) receives twice
 *   the local energy of every site, 2 E_i = sum_k sum_{v in shell k}
 *   V_k[s_i][s_{i+v}] (0.01 meV; Eq. Linear_EPI without bias terms, each bond
 *   at both ends, so sum_i 2 E_i = 2 E), canonical site order.  Under the
 *   qSRO model (smcx_set_qsro) 2 E_i also carries 2 sum_k W[k][s_i]
 *   n_k(i)^2, and the clusters use these local energies.
 * smcx_clusters: a site's class is (2 E_i < thr2); two shell-1 neighbours of
 *   one class are in one cluster.  d_labels (device, [N] int32, caller-owned)
 *   receives for every site the smallest site id of its cluster (a unique
 *   labelling); *n_clusters (may be NULL) the number of clusters.  Needs N <
 *   2^31 (SMCX_E_RANGE); temporary device memory N bytes.  SMCX_E_TIMEOUT if
 *   the union-find exceeded its iteration limit (labels then undefined).
 * smcx_cluster_summary: from labels made by smcx_clusters on this handle's
 *   current configuration, the clusters of at least min_size sites, largest
 *   first (ties: smaller label first), at most max_out of them: roots [max_out]
 *   (labels), sizes [max_out], counts [max_out][M] (species counts, may be
 *   NULL); *n_out = number written.  Temporary device memory 4 N bytes.
 *   SMCX_E_RANGE if more than 2^26 clusters reach min_size.
 */
int smcx_local_energy(smcx_lattice* h, int32_t* d_e2);
int smcx_clusters(smcx_lattice* h, int64_t thr2, int32_t* d_labels, int64_t* n_clusters);
int smcx_cluster_summary(smcx_lattice* h, const int32_t* d_labels, int64_t min_size, int max_out, int64_t* roots,
                         int64_t* sizes, int64_t* counts, int* n_out);

/* Copy the configuration out / in as int8 species ids in canonical site
 * order (N = nx*ny*nz*m entries).  set_config checks ids < M and keeps the
 * sweep counter; it does not require the old composition. */
int smcx_get_config(smcx_lattice* h, int8_t* host);
int smcx_set_config(smcx_lattice* h, const int8_t* host);

/* The same in the lattice store's own layout (no conversion on either side):
 * smcx_store_bytes gives its size, N bytes for SMCX_INT8 and N/2 for
 * SMCX_PACKED4 (two sites per byte, the even site of each pair in the low
 * nibble).  set_config_store checks every id < M on the device before the
 * store is touched (SMCX_E_INVALID_ARG otherwise, lattice unchanged); `bytes`
 * must equal the store size. */
int smcx_store_bytes(const smcx_lattice* h, size_t* bytes);
int smcx_get_config_store(smcx_lattice* h, uint8_t* host, size_t bytes);
int smcx_set_config_store(smcx_lattice* h, const uint8_t* host, size_t bytes);

/* Cumulative sweep index and trial statistics since creation (int64[4]):
 * stats[0] = trials, stats[1] = accepted swaps, stats[2] = proposals whose
 * two sites held the same species (no-ops; counted as trials), stats[3] =
 * sum of the energy changes of accepted swaps (0.01 meV), so that
 * E(now) = E(creation or last set_config) + stats[3] - (stats[3] then). */
int smcx_get_state(smcx_lattice* h, uint64_t* sweep_cum, int64_t* stats);
int smcx_set_sweep_counter(smcx_lattice* h, uint64_t sweep_cum);

/* Device pointer and size in bytes of the species buffer (INT8: N bytes;
 * PACKED4: ceil(N/2) bytes).  Owned by the handle. */
int smcx_device_buffer(const smcx_lattice* h, void** ptr, size_t* bytes);

/* Block until all work enqueued on the handle's stream is done. */
int smcx_synchronize(smcx_lattice* h);

/* Total sites N and the handle's geometry. */
int smcx_lattice_info(const smcx_lattice* h, int* kind, int* dims /*[3]*/, int* M,
                      int* K, int* storage, int64_t* n_sites);

/*
 * Host-only helper: the acceptance tables this library uses at temperature T
 * (A[SMCX_NA_MAX], B[SMCX_NB], nA = entries of A before the first zero).
 * Needs no GPU.
 */
int smcx_threshold_tables(double T, uint32_t* A, int* nA, uint32_t* B);

/*
 * Batched replicas (temperature parallelism, Supplementary "Parallelization
 * opportunities"): independent BCC lattices of any sizes, each at its own
 * temperature and with its own schedule, sweep counter and replica id, swept
 * together in one persistent cooperative launch (captured in a CUDA graph and
 * replayed on later calls with the same sweep count).  Every replica's
 * trajectory equals the one smcx_sweep gives it alone.
 *   smcx_batch_create   references R existing handles (not owned; they must
 *                       outlive the batch), which must share M, the EPI table
 *                       (4 shells, set with smcx_set_epi), the proposal mode
 *                       and `stream`, and have schedules with tiles of at most
 *                       20 cells.  Shared-direction modes also need M <= 4,
 *                       |V| < 2^15 and tiles of at most 256 link cells (one
 *                       slot per thread).
 *   smcx_batch_sweep    n_sweeps at temperatures T[R] with Philox seed `seed`;
 *                       returns after the launch has finished; SMCX_E_TIMEOUT
 *                       if a grid barrier waited longer than its limit.
 *   smcx_batch_autotune times `trial_sweeps` batched sweeps for every
 *                       candidate (link cell 3 or 4, tiles of at most 12-20
 *                       cells, 128- or 256-thread CTAs) on snapshots of the
 *                       configurations, restores them, and installs the
 *                       fastest candidate's schedules (read them back with
 *                       smcx_get_schedule) and block size (*threads).
 *   smcx_batch_energy   E[R], one smcx_energy per replica.
 *   smcx_batch_info     grid size, threads per CTA and whether the last call
 *                       replayed a graph.
 *   smcx_batch_set_block threads per CTA of the next sweeps: 0 (the fewest
 *                       128-thread-or-smaller CTAs that cover a tile's link
 *                       cells with at most 2 slots per thread; 256 threads for
 *                       tiles of more than 128 link cells under a
 *                       shared-direction mode), 128, or 256
 *                       (one slot per thread; SMCX_E_UNSUPPORTED at the next
 *                       sweep if a tile has more than 256 link cells).
 *                       SMCX_E_INVALID_ARG for other values.
 *   smcx_batch_set_fault test hook: CTA `skip_cta` (>= 0) skips the first grid
 *                       barrier, which then times out after timeout_ms and the
 *                       next smcx_batch_sweep returns SMCX_E_TIMEOUT; -1 turns
 *                       it off.  timeout_ms (1..60000, default 2000) bounds
 *                       every barrier wait.
 */
typedef struct smcx_batch smcx_batch;
int smcx_batch_create(smcx_batch** out, int R, smcx_lattice* const* lattices, void* stream);
int smcx_batch_destroy(smcx_batch* b);
int smcx_batch_sweep(smcx_batch* b, const double* T, int64_t n_sweeps, uint64_t seed);
int smcx_batch_autotune(smcx_batch* b, const double* T, int trial_sweeps, int* threads);
int smcx_batch_energy(smcx_batch* b, int64_t* E);

/*
 * Replica exchange between temperature slots (Supplementary "Parallelization
 * opportunities": configurations at different temperatures are exchanged by
 * a rule that keeps detailed balance).  Needs replicas of one lattice shape.
 *   T_slot      [R] temperature of each slot (K, > 0).
 *   slot_rep    [R] in/out: the replica at each slot, a permutation of 0..R-1.
 *   n_rounds    rounds to run; each sweeps every replica sweeps_per_round
 *               times at its slot's temperature (one batched launch), then
 *               proposes swaps of the slot pairs (t, t+1), t = round mod 2,
 *               round mod 2 + 2, ...
 *   round_ctr   in/out cumulative round counter (selects the pairing and the
 *               random numbers; split calls equal one call).
 *   accepts     [R-1] in/out, may be NULL: accepted swaps per slot pair.
 * The swap of replicas a (slot t) and c (slot t+1) is accepted when x =
 * (beta_t - beta_{t+1}) (E_a - E_c) >= 0, beta = 1/(k_B T), E in 0.01 meV,
 * else when u < floor(2^32 exp(x)) (capped at 2^32 - 1), u = word 0 of
 * Philox4x32-10(counter (t, round lo, round hi, 0xC0000000), key = seed).
 * The energies are exact (start energy + accepted dE).  Configurations stay
 * in their replica; only the temperature assignment moves.
 */
int smcx_batch_exchange(smcx_batch* b, const double* T_slot, int32_t* slot_rep, int64_t n_rounds,
                        int64_t sweeps_per_round, uint64_t seed, uint64_t* round_ctr, int64_t* accepts);

/*
 * smcx_lattice_fluct_accumulate for every replica of the batch in two launches
 * (the tiled pair counts of all replicas' tiles, then one FP64 accumulator per
 * replica): d_acc is a device array [R][1 + M^2 + K M^2 + M^2 K M^2], replica
 * r's sums at offset r times that size, laid out as for
 * smcx_fluct_accumulate (each replica with its own site count).  Needs
 * M <= 4 (SMCX_E_UNSUPPORTED otherwise).  Returns after the sums are done.
 */
int smcx_batch_fluct_accumulate(smcx_batch* b, int shell, double* d_acc);
int smcx_batch_info(const smcx_batch* b, int* grid, int* threads, int* used_graph);
int smcx_batch_set_block(smcx_batch* b, int threads);
int smcx_batch_set_fault(smcx_batch* b, int skip_cta, int timeout_ms);

/*
 * Differentiation (all pointers are device pointers owned by the caller;
 * work is enqueued on `stream`, nothing is synchronised).
 *
 * The pair energy is linear in V (Eq. Total_EPI): E = 1/2 sum V_i C_i, so
 * dE/dV_i = C_i / 2 -- the backward pass of fitting V to reference energies
 * by back-propagation (Results "Energy model").
 *   smcx_pair_counts_batch  C[B][K][M][M] (int64) of B configurations of one
 *                           geometry (int8 ids [B][N], canonical order; N up
 *                           to ~200k sites).  A configuration holding an id
 *                           outside 0..M-1 is not counted: all its K*M*M
 *                           counts are set to -1.
 *   smcx_epi_energy_batch   E[b] = 1/2 sum_i V[i] C[b][i] (float V, FP64 sum,
 *                           float E), KMM = K*M*M.
 *   smcx_epi_grad_batch     grad[i] = 1/2 sum_b g[b] C[b][i] (float).
 * Thermal derivative of an observable A (Supplementary "Statistical
 * mechanics": <O> under exp(-beta E)):
 *   d<A>/dV_i = -beta (<A C_i/2> - <A><C_i/2>),  beta = 1 / (k_B T) in 1/meV.
 *   smcx_fluct_accumulate   adds B weighted samples (weights d_weights[B], or
 *                           1 when NULL) of A = the Warren-Cowley alpha of
 *                           shell `shell` (M*M) and C to d_acc (FP64),
 *                           layout [1 + MM + KMM + MM*KMM]: sum w, sum w A,
 *                           sum w C, sum w A C^T (row-major [a][i]).
 *   smcx_lattice_fluct_accumulate  one sample (weight 1) of the handle's
 *                           current configuration, on the handle's stream.
 *   smcx_fluct_gradient     grad[MM][KMM] = d<A_a>/dV_i in 1/meV from d_acc.
 */
int smcx_pair_counts_batch(int kind, int nx, int ny, int nz, int M, int K, const int8_t* d_configs, int64_t B,
                           int64_t* d_counts, void* stream);
int smcx_epi_energy_batch(const float* d_V, const int64_t* d_counts, int64_t B, int KMM, float* d_E, void* stream);
int smcx_epi_grad_batch(const float* d_g, const int64_t* d_counts, int64_t B, int KMM, float* d_grad, void* stream);
int smcx_fluct_accumulate(const int64_t* d_counts, int64_t B, const double* d_weights, int kind, int K, int M,
                          int shell, int64_t n_sites, double* d_acc, void* stream);
int smcx_lattice_fluct_accumulate(smcx_lattice* h, int shell, double* d_acc);
int smcx_fluct_gradient(const double* d_acc, int K, int M, double T, double* d_grad, void* stream);

/*
 * Energy of a device-resident configuration without allocating device memory.
 * The paper has no counterpart: this entry point exists for callers that may
 * not call cudaMalloc -- code that runs inside another framework's memory
 * arena, latency-critical loops that must not wait on the allocator, or
 * callers holding only a device pointer to a configuration (for instance from
 * smcx_device_buffer) and no handle.
 *   kind, nx, ny, nz, M, storage  describe d_sites exactly as for
 *                                 smcx_lattice_create (canonical site order);
 *   K, V                          EPI table V[K][M][M] on the host (symmetric);
 *   d_sites                       device (or managed) pointer to the species
 *                                 ids, read only; a host pointer is rejected;
 *   E                             host output, exact energy in 0.01 meV;
 *   stream                        cudaStream_t ordering the work (NULL = default).
 * The histogram, the EPI table, the result and a bad-id flag live in one fixed
 * device array of 16 KiB inside the library (held by every GPU that loads it
 * until the process exits): K*M*M must not exceed 1300, otherwise
 * SMCX_E_INVALID_ARG.  Species ids are checked as they are read: an id outside
 * 0..M-1 is not counted and the call returns SMCX_E_INVALID_ARG.  The first
 * call on a device looks up that array's address with the device current;
 * make that first call before any stream capture.  The address is kept for the
 * life of the process and does not survive cudaDeviceReset: do not call this
 * entry point on a device after resetting it.  All calls share the array: it
 * is cleared at the start of each call, and calls whose GPU work overlaps
 * (several streams or host threads) race and return wrong energies.
 * Synchronises `stream` before returning.
 */
int smcx_energy_noalloc(int kind, int nx, int ny, int nz, int M, int storage, int K, const int32_t* V,
                        const void* d_sites, int64_t* E, void* stream);

/*
 * Measured shared-memory byte-load rate of the current device (entry point
 * outside the paper: the denominator of the sweep kernels' on-chip roofline).
 * Runs a conflict-free LDS.U8 stream on every SM (a few milliseconds,
 * enqueued on `stream` and waited for) and returns lane-loads per second.
 */
int smcx_probe_lds_rate(double* lane_loads_per_s, void* stream);

/*
 * Bounds-check status of the debug build (entry point outside the paper).
 * The library built with SMCX_DEBUG=1 (paper_2503_12591_gb300/_build/
 * libsmcx_debug.so) checks the index of its shared-memory box accesses,
 * tile staging and write-back, and pair-count bins against their extents;
 * an out-of-range index skips that access and records a tag (the access
 * kind, SMCX_DEBUG_* in smcx_device.cuh order: 1 BCC box, 2 BCC staging,
 * 3 BCC write-back, 4 BCC phase directions, 5 generic tile box, 6 FCC box,
 * 7 pair-count bin, 8 lattice store) and the index.  Nothing traps.  This call
 * synchronises the device, writes info[0] = the first tag recorded since the
 * last call (0: none), info[1] = its index, and clears the record.
 * SMCX_E_UNSUPPORTED in the normal build.
 */
int smcx_debug_status(uint64_t* info);

#ifdef __cplusplus
}
#endif
#endif /* SMCX_H */
