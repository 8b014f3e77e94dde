// BCC sweep with shared-direction proposals (SMCX_PROPOSAL_TILE and
// SMCX_PROPOSAL_BLOCK), single-lattice and batched: the one compiled variant
// (4 shells, M <= 4, two byte planes, one link-cell slot per thread).  The
// direction of a phase is the same for every lane, so the union of the s and
// s' environments is read with offsets from a constant-memory table (one row
// per sublattice and direction) and the shells of every entry are
// compile-time constants.
#include "smcx_batch_body.cuh"

namespace smcx {

namespace bccfast {

__constant__ UnionOffsets c_union = make_union_offsets();

template <int B, int K, int NW, int PL>
__device__ void trial_shared_dir(uint8_t* box, int s, int dir, uint32_t ru, const Planes& P, const uint32_t* s_rows,
                                 int nA, const uint32_t* sA, const uint32_t* sB, unsigned& acc, unsigned& same,
                                 long long& dsum) {
  constexpr UTable T = make_union7<K>();
  const int sp = s + c_union.poff[B][dir];
  const uint32_t a8 = ld_chk(box, s, 2 * SUB, kDbgBccBox), b8 = ld_chk(box, sp, 2 * SUB, kDbgBccBox);
  if (a8 == b8) {
    same++;
    return;
  }
  uint32_t h[kMaxShells][2];
#pragma unroll
  for (int k = 0; k < kMaxShells; k++) h[k][0] = h[k][1] = 0x80808080u;
  const int* off = c_union.off[B][dir];
#pragma unroll
  for (int j = 0; j < T.n; j++) {
    const uint32_t v = ld_chk(box, s + off[j], 2 * SUB, kDbgBccBox);
    uint32_t one;
    asm("shl.b32 %0, 1, %1;" : "=r"(one) : "r"(v));
    if (T.e[j].k1 >= 0) h[T.e[j].k1][0] += one;
    if (T.e[j].k2 >= 0) h[T.e[j].k2][0] -= one;
  }
  if (P.rows)
    finish_trial_rows<K>(box, s, sp, a8, b8, h, ru, s_rows, nA, sA, sB, acc, dsum);
  else
    finish_trial<K, NW, PL>(box, s, sp, a8, b8, h, ru, P, nA, sA, sB, acc, dsum);
}

}  // namespace bccfast

bccfast::BatchKernelFn batch_dir_kernel(int threads) {
  return threads == 256 ? bccfast::k_bcc_batch256<4, 1, 2, 1> : bccfast::k_bcc_batch<4, 1, 2, 1, 1>;
}

void sweep_bcc_dir(smcx_lattice* hd, bccfast::LatDesc& D, const bccfast::Planes& Q, int threads, int64_t n,
                   int nc) {
  const int nq = D.NQ;
  if (nq * nq * nq > threads) fail(SMCX_E_UNSUPPORTED, "shared-direction kernel runs one slot per thread");
  launch_bcc<4, 1, 2, 1, 1>(hd, D, Q, threads, n, nc);
}

}  // namespace smcx
