// Internal declarations of the smcx library (CUDA sm_103a).
//
// Geometry, schedule, acceptance tables and the Philox generator are written
// here for the GPU path; the CPU oracle under oracle/ carries its own
// independent copies, so that a mistake in one is caught by the other.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/smcx.h"

namespace smcx {

constexpr int kBCC = SMCX_BCC;
constexpr int kFCC = SMCX_FCC;
constexpr int kMaxShells = 4;     // BCC 1..4, FCC 1..3
constexpr int kMaxVec = 64;       // neighbour vectors of all shells in use
constexpr int kMaxZ1 = 12;        // shell-1 size (BCC 8, FCC 12)
constexpr int kMaxSweepM = 8;     // species supported by the sweep kernels
constexpr double kBoltzmannMeV = 8.617333262e-2;  // k_B in meV/K (exact SI)

// ---------------------------------------------------------------------------
// NVTX: every sweep-type entry point opens a range named after itself for the
// whole call (argument checks included), so that a profiler or an NVTX
// injection library sees where each call's GPU work was enqueued.  Header-only
// NVTX v3: without an attached tool every push and pop is a no-op.
// ---------------------------------------------------------------------------
struct NvtxRange {
  explicit NvtxRange(const char* name);
  ~NvtxRange();
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------------------
// Status plumbing: every C entry point catches and converts to an SMCX_E_*.
// ---------------------------------------------------------------------------
struct SmcxException {
  int code;
  std::string msg;
};
void set_error(const std::string& msg);
const std::string& last_error();
[[noreturn]] void fail(int code, const std::string& msg);
void check_cuda(cudaError_t e, const char* what);

// Run f, turning failures into an SMCX_E_* status and a per-thread message.
template <class F>
int guarded_call(F&& f) {
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
  } catch (...) {
    set_error("unknown failure");
    return SMCX_E_INVALID_ARG;
  }
}

// ---------------------------------------------------------------------------
// Host geometry.
// ---------------------------------------------------------------------------
struct Shells {
  int kind = 0;
  int m = 0;          // sites per cubic cell
  int K = 0;          // shells in use
  int z[kMaxShells] = {0};
  int nv = 0;         // total neighbour vectors
  int v[kMaxVec][3];  // half-lattice-unit vectors, shell-major, lexicographic
  int shell_of[kMaxVec];
  int R1 = 0, RK = 0; // max |component| of shell-1 vectors and of shells 1..K
  int model = 0;      // 0: pair model; 1: qSRO (a trial reads R1 + 2 RK around its centre)
};

int sites_per_cell(int kind);
void basis_of(int kind, int b, int out[3]);
int basis_index(int kind, int rx, int ry, int rz);
Shells make_shells(int kind, int K);
void check_reach(const Shells& S, const int n[3]);  // SMCX_E_INVALID_ARG if an edge < reach
// smallest link-cell edge and tile thickness for which the checkerboard
// phases are independent (see smcx_sched)
int min_link_cell(const Shells& s);
int min_tile(const Shells& s);
int halo_cells(const Shells& s);   // staging halo around a tile (cells)
int ring_cells(const Shells& s);   // cells outside a tile a partner can reach

// Validates a schedule; returns "" if valid, else a reason.
std::string schedule_problem(const Shells& s, const int n[3], const smcx_sched& sc);
smcx_sched choose_schedule(const Shells& s, const int n[3]);

// Acceptance tables: A[kNA], B[kNB], nA.
constexpr int kNA = SMCX_NA_MAX;
constexpr int kNB = SMCX_NB;
int threshold_tables(double T, uint32_t* A, int* nA, uint32_t* B);

// ---------------------------------------------------------------------------
// Lattice handle.
// ---------------------------------------------------------------------------
}  // namespace smcx

struct smcx_batch;  // smcx_batch.cu

struct smcx_lattice {
  int kind = 0, m = 0, M = 0, storage = 0;
  int n[3] = {0, 0, 0};
  int64_t N = 0;
  smcx::Shells shells;  // shells of the EPI in use (K = 0 before set_epi)
  bool have_epi = false;
  std::vector<int32_t> V;
  std::vector<int32_t> Wq;  // qSRO weights [K][M] (0.01 meV); empty: pair model
  smcx_sched sched{0, {0, 0, 0}};
  bool sched_auto = true;
  cudaStream_t stream = nullptr;

  uint8_t* d_sites = nullptr;
  size_t site_bytes = 0;
  bool owns_sites = true;                 // false for a handle made by smcx_lattice_wrap
  unsigned long long* d_stats = nullptr;  // [4] trials, accepts, same, sum dE
  unsigned long long* d_counts = nullptr; // [K*M*M] reduction output
  long long* d_energy = nullptr;          // [1]
  uint32_t* d_thr = nullptr;              // A[kNA] then B[kNB]
  int32_t* d_wtab = nullptr;              // W[a][b][k][c], then X[a][b]
  int* d_flag = nullptr;                  // device error flag
  uint8_t* d_stage = nullptr;             // host<->device staging (int8 ids)
  uint16_t* d_qcnt = nullptr;             // qSRO same-species counts, one word per site (FCC sweeps)
  size_t stage_bytes = 0;

  int kernel_choice = 0;  // 0 = fastest usable, 1 = generic tile/link-cell kernels
  int replica = 0;        // Philox replica id (counter word 1, bits 16..31)
  int proposal = 0;       // SMCX_PROPOSAL_SITE or SMCX_PROPOSAL_TILE
  int bcc_threads = 0;    // tuned block size of the BCC tile kernel (0 = default)
  double thr_T = -1.0;
  int thr_nA = 0;
  uint64_t sweep_cum = 0;
};

namespace smcx {

// Kernels' host launchers (implemented in the .cu files).
void init_config_device(smcx_lattice* h, const double* comp, uint64_t seed);
void validate_int8(smcx_lattice* h, const int8_t* d_ids, int64_t count);  // sets d_flag
void validate_store(smcx_lattice* h);  // every stored id < M, else sets d_flag
void validate_store_at(smcx_lattice* h, const uint8_t* d_store);  // same for a buffer in the store layout
void record_energy(smcx_lattice* h, const long long* d_dsum0, long long* d_out);  // d_energy + stats[3] - dsum0
void energy_moments(smcx_lattice* h, const long long* d_E, long long n, double T, double* d_out);  // mean, var, C_V/(N k_B)
void local_energy_device(smcx_lattice* h, int32_t* d_e2);
void sweep_qsro_device(smcx_lattice* h, int nA, uint64_t seed, int64_t n_sweeps, int n_colours);
bool fcc_fast_usable(const smcx_lattice* h);
void sweep_fcc_fast(smcx_lattice* h, int nA, uint64_t seed, int64_t n_sweeps, int n_colours);
void qsro_energy_add(smcx_lattice* h);
bool energy_bcc_direct(smcx_lattice* h);  // pair energy into d_energy; false if not applicable  // adds sum_i sum_k W[k][s_i] n_k(i)^2 to d_energy
void clusters_device(smcx_lattice* h, long long thr2, int32_t* d_labels, int64_t* n_clusters);
void cluster_summary_device(smcx_lattice* h, const int32_t* d_labels, long long min_size, int max_out,
                            int64_t* roots, int64_t* sizes, int64_t* counts, int* n_out);
void pack_from_int8(smcx_lattice* h, const int8_t* d_ids, int64_t first, int64_t count);
void unpack_to_int8(smcx_lattice* h, int8_t* d_ids, int64_t first, int64_t count);
void pair_counts_device(smcx_lattice* h);          // fills h->d_counts
void energy_device(smcx_lattice* h);               // fills h->d_energy (needs counts)
void sweep_device(smcx_lattice* h, int nA, uint64_t seed, int64_t n_sweeps, int n_colours = 8);
// dir_slots: the most link-cell slots a tile may have under shared-direction
// proposals (one slot per thread: 128 for the single-lattice kernel, 256 for
// the batched kernel's 256-thread CTAs).
bool bcc_fast_usable(const smcx_lattice* h, int dir_slots = 128);
bool bcc_counts_usable(const smcx_lattice* h, int nt[3]);
void pair_counts_bcc_tiled(smcx_lattice* h, const int nt[3]);
int bcc_slots_per_axis(const int n[3], const smcx_sched& sc);
void bcc_block_shape(int nq, int tuned_threads, int* threads, int* slots);
void sweep_bcc_fast(smcx_lattice* h, int nA, uint64_t seed, int64_t n_sweeps, int n_colours);
void species_counts(int M, const double* comp, int64_t N, int64_t* counts);

struct SweepParams;
void pair_counts_raw(int kind, int K, const SweepParams& P, long long ncell, int KMM, unsigned long long* counts,
                     cudaStream_t st);
void energy_raw(const unsigned long long* C, const int32_t* V, int KMM, long long* E, cudaStream_t st);

}  // namespace smcx
