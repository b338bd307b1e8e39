// k_grad_tc.cu -- tcgen05 / TMEM / TMA kernel for one fold-masked gradient
// evaluation of a flat model (logistic; Gaussian linear and AR with the
// GAUSS instantiations) for all chains, fused with the leapfrog update
// (Section 3.3; masks of eq. mask-log-prob / mask-log-pred, Appendix B).
// The two contractions of the masked likelihood gradient are tensor-core
// GEMMs in BF16 with FP32 accumulation:
//
//   S = Theta_tile . X_chunk^T      (128 chains x 128 rows, K = p + 3)  -> TMEM
//   R = mask .* (1 - tanh(S))       (epilogue, FP32, rounded to BF16)   -> TMEM
//       (Gaussian: mask .* (-2 S) / sigma^2, S = (eta - y) / 2)
//   G += R . X_chunk                (128 chains x p, K = 128 rows)      -> TMEM
//
// Logistic model: row n of the stored design matrix is s_n x_n with
// s_n = 2 y_n - 1, so S = s eta / 2 and, as y - sigmoid(eta) =
// s (1 - tanh(s eta / 2)) / 2, the likelihood gradient is G / 2 with no
// response in the epilogue; 1 - tanh keeps its relative precision for rows
// the model already predicts well.  The log likelihood of a row is
// -softplus(-s eta).
//
// Gaussian models: the folded columns hold (eta_ref - y) / 2, so S =
// (eta - y) / 2 and the residual needs no response either.
//
// R is the A operand of the second GEMM straight from TMEM, so shared memory
// carries only Theta and X: with both operands of both GEMMs in SMEM the
// MMAs alone saturate its bandwidth.
//
// The tensor cores see theta centred on a reference theta_ref (the mean of
// the full-data draws, or of the positions a caller sets) and scaled by 1/2:
// the shadows hold (theta - theta_ref) / 2 in bf16 hi + lo parts.  The
// row's eta_ref / 2 = x . theta_ref / 2 enters the same GEMM: three more K
// columns of X hold it as hi + mid + lo bf16 parts and the hi shadow holds 1
// there, so S is eta / 2 (logistic: s eta / 2) straight from the tensor
// cores and the epilogue needs no per-row addition.  The same SMEM X tile is the
// K-major B operand of the first GEMM and the MN-major B operand of the
// second.  Launches that need log densities accumulate hi + lo (an
// FP32-accurate eta for the Metropolis test); the kick-drift launches use
// the hi part only once a reference is set.  Centred, the bf16 rounding of
// theta - theta_ref is ~0.4 % of a posterior standard deviation (of theta
// itself it was a few percent, enough to slow mixing); HMC stays exact
// because the accept test uses the accurate log density.
// Where log densities are needed (last leapfrog step, evaluations) the
// epilogue also sums softplus(-s eta) over the fold's training and test
// rows.
//
// Work: persistent CTAs (one per SM) take equal contiguous ranges of the
// flattened (chain tile, row chunk) units ("stream-K").  A CTA flushes its G
// partial for each tile segment to a workspace; the last CTA of a tile
// (atomic ticket, no spinning) sums the segments in order and applies priors
// and the momentum / position update.
//
// Roles: warpgroup 0 holds the producers: warp 0 issues TMA loads, warp 1
// allocates TMEM and issues the first GEMM (one thread), warp 2 issues the
// second GEMM (one thread, so that waiting for the epilogue never delays the
// first GEMM of later chunks).  Warpgroups 1 and 2 run the epilogue on
// alternate chunks (thread = TMEM lane = chain; two warps per SM
// sub-partition so TMEM-load and barrier latencies overlap); they take the
// registers the producers give up (setmaxnreg) and read a chunk's S row
// whole, releasing S before computing R (32 rows at a time); each 64-row
// half of R is handed to the second GEMM as soon as its TMEM stores have
// completed.
// Every mbarrier wait is bounded: on time-out the kernel sets an error flag,
// stops issuing work and exits after freeing TMEM.
#include <cuda.h>

#include <utility>

#include "pcv_internal.cuh"
#include "tc_ptx.cuh"

namespace pcv {

constexpr int kTN = 128;        // rows per chunk
constexpr int kTM = 128;        // chains per tile
constexpr int kTcThreads = 384; // 12 warps: TMA, GEMM1 MMA, GEMM2 MMA, idle, 8 epilogue
// Registers per thread after the split (setmaxnreg): the producer warpgroup
// gives registers up so that the epilogue can hold a whole S row.  The
// split must fit in what the CTA was launched with: checked on the host
// against the compiled register count before any launch.
constexpr int kTcRegsProducer = 64, kTcRegsEpilogue = 208;
constexpr int kTcMaxStages = 8; // X pipeline stages (as many as fit in shared memory)


// --------------------------------------------------------------------------
// KS (GEMM1 K steps of 16, = ceil(p / 16)) is a template parameter so that
// every MMA group is straight-line code: MMAs issued from a runtime-count
// loop between commits measured up to 3x slower on sm_103a.
//
// TF (the TF32 operand form): kind::tf32 MMAs (K = 8 per instruction) on
// FP32 shadows of theta and an FP32 copy of X, both rounded to TF32, hi part
// only; chunks of 64 rows (so that the FP32 tiles fit in shared memory and
// TMEM); the second GEMM reads X^T (a K-major copy, loaded with each chunk
// through tm_lo, which the TF form does not otherwise use) so that both
// GEMMs take K-major operands; the residual goes to TMEM as TF32, one
// element per column.
// MS: several kick-drift steps in one launch (BF16, one CTA per tile,
// ta.steps of them); a separate instantiation so that the one-step kernel's
// code is not touched by it
template <int KS, bool ACC, bool GAUSS, bool TF = false, bool MS = false>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_grad_tc(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_hi,
              const __grid_constant__ CUtensorMap tm_lo, Problem pb, GradArgs a, TcArgs ta) {
  constexpr int TN = TF ? 64 : kTN;                // rows per chunk
  constexpr int AE = TF ? 32 : 64;                 // operand elements per 128-byte K atom
  constexpr int NQ = TN / 32;                      // 32-row quarters per chunk
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned base, by an offset into the shared array (so that the
  // compiler keeps shared-memory loads for y)
  uint8_t *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const int KA = ta.KP / AE;                       // 128-byte K atoms
  // theta in shared memory (the TF32 form keeps it in TMEM instead)
  const uint32_t th_bytes = TF ? 0u : (uint32_t)KA * kTM * 128;
  const uint32_t x_bytes = (uint32_t)KA * TN * 128;             // K-major X chunk
  // TF32: the chunk's X^T (two 32-row column blocks of PN feature rows) in a
  // ring of its own, so that an X slot is free again once the first GEMM is
  // done with it while the X^T slot waits for the epilogue and second GEMM
  const uint32_t xt_bytes = TF ? 2u * ta.PN * 128u : 0u;
  const int NS = ta.NS, NT = TF ? ta.NT : 0;
  uint8_t *th_hi = sm;
  uint8_t *th_lo = th_hi + th_bytes;
  uint8_t *xs = th_lo + (ta.need_lo ? th_bytes : 0);
  uint8_t *xts = xs + (size_t)NS * x_bytes;
  uint64_t *bars = reinterpret_cast<uint64_t *>(xts + (size_t)NT * xt_bytes + 64);
  // barrier slots (up to kTcMaxStages X stages)
  uint64_t *x_full = bars, *x_empty = bars + kTcMaxStages;
  // r_part[4 b + h], h < 2: half h (64 rows) of R buffer b is in TMEM, so the
  // second GEMM starts on a chunk while its epilogue is still computing
  // (slots h = 2, 3 are unused)
  uint64_t *s_full = bars + 2 * kTcMaxStages, *s_empty = s_full + 2;
  uint64_t *r_part = s_full + 4, *r_empty = s_full + 12, *th_full = s_full + 14, *th_empty = s_full + 15;
  uint64_t *g_full = s_full + 16, *g_empty = s_full + 17;
  uint32_t *tmem_base_slot = reinterpret_cast<uint32_t *>(s_full + 18);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(s_full + 19);
  volatile int *last_flag = reinterpret_cast<volatile int *>(s_full + 20);
  uint64_t *flush_bar = s_full + 21, *decide_bar = s_full + 22;   // epilogue-internal sync
  // several steps per launch: the finish of a step is done (its theta,
  // momentum and shadows written), so the next step may load theta
  uint64_t *th_ready = s_full + 23;
  uint64_t *xt_full = s_full + 24, *xt_empty = xt_full + kTcMaxStages;   // X^T ring (TF32)

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long U = (long long)ta.T * ta.J;
  const long long u0 = (long long)blockIdx.x * U / ta.n_cta;
  const long long u1 = (long long)(blockIdx.x + 1) * U / ta.n_cta;
  // MS (kick-drift, one CTA per tile): the CTA carries its tile
  // through that many leapfrog steps, its J units once per step
  const int per = (int)(u1 - u0);
  const int nunits = MS ? per * ta.steps : per;
  // Order of the CTA's units: a range that ends in a later tile than it
  // starts in runs its last piece (chunks 0 .. of that tile) first, then the
  // rest in order.  Every CTA's range is about U / n_cta units, so at any
  // time all CTAs work on rows within J - U / n_cta chunks of one another
  // and the X chunks in use stay resident in L2 (in plain order the CTAs
  // start at chunks spread over all of X).  All roles walk this order; the
  // ownership of tile segments and the finish do not depend on it.
  const long long ls = (u1 - 1) / ta.J * ta.J;     // start of the last unit's tile
  const int rot = (nunits > 0 && ls > u0) ? (int)(u1 - ls) : 0;
  auto unit_of = [&](const int i) -> long long { return i < rot ? ls + i : u0 + (MS ? (i - rot) % per : i - rot); };
  // the chunk index j of unit i, walked incrementally by the single-thread
  // issuers (no 64-bit division per unit): j of unit 0, and the step
  const int j_u0 = (int)(u0 % ta.J);
  const int j_first = rot > 0 ? 0 : j_u0;
  auto j_step = [&](const int i, const int j) { return i + 1 == rot ? j_u0 : (j + 1 == ta.J ? 0 : j + 1); };
  // segment boundaries in this order
  auto seg_first = [&](const int i, const int j) { return i == 0 || i == rot || j == 0; };
  auto seg_last = [&](const int i, const int j) { return i == nunits - 1 || i == rot - 1 || j == ta.J - 1; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) { mbar_init(smem_u32(&x_full[s]), 1); mbar_init(smem_u32(&x_empty[s]), 1); }
    for (int s = 0; s < NT; ++s) { mbar_init(smem_u32(&xt_full[s]), 1); mbar_init(smem_u32(&xt_empty[s]), 1); }
    for (int s = 0; s < 2; ++s) {
      mbar_init(smem_u32(&s_full[s]), 1); mbar_init(smem_u32(&s_empty[s]), 4);
      for (int qq = 0; qq < 2; ++qq) mbar_init(smem_u32(&r_part[4 * s + qq]), 4);
      mbar_init(smem_u32(&r_empty[s]), 1);
    }
    // th_full: the TMA load of theta (bf16), or the eight epilogue warps'
    // TMEM stores of it (TF32)
    mbar_init(smem_u32(th_full), TF ? 8 : 1); mbar_init(smem_u32(th_empty), 1);
    mbar_init(smem_u32(g_full), 1); mbar_init(smem_u32(g_empty), 4);
    mbar_init(smem_u32(flush_bar), 8); mbar_init(smem_u32(decide_bar), 1);
    if (MS) mbar_init(smem_u32(th_ready), 8);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // TMEM, bf16: S[0] 0-127, S[1] 128-255, G 256-383, R[0] 384-447, R[1] 448-511;
  // TF32: S[0] 0-63, S[1] 64-127, G 128-255, R[0] 256-319, R[1] 320-383,
  // theta 384-511 (the first GEMM's A operand, K steps of 8 columns)
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_base_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_base_slot;

  // S[b] at tmem + TN b; G after them; R[b] (64 columns: 128 rows as
  // bf16x2, or 64 rows as TF32) after G
  const uint32_t tmem_G = tmem + 2 * TN;
  const uint32_t tmem_R = tmem_G + 128;
  const uint32_t tmem_T = tmem_R + 128;            // TF32 only

  if (warp < 4) {
  // register split: warpgroup 0 (producers) gives registers up ...
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kTcRegsProducer));
  if (warp == 0) {
    // ------------------------------ TMA producer ---------------------------
    if (lane == 0) {
      int seg = 0, th_issued = -1;
      int last_round[kTcMaxStages];
#pragma unroll
      for (int s2 = 0; s2 < kTcMaxStages; ++s2) last_round[s2] = -1;
      // theta of the segment starting at unit i (the chain tile's shadow)
      auto load_theta = [&](const int i) -> bool {
        const int t = (int)(unit_of(i) / ta.J);
        if (!mbar_wait_fast(smem_u32(th_empty), (seg & 1) ^ 1, abort_flag, ta.err)) return false;
        // the next step of the same tile: its theta comes from the last
        // step's finish
        if (MS && seg > 0 && !mbar_wait_fast(smem_u32(th_ready), (seg - 1) & 1, abort_flag, ta.err)) return false;
        mbar_expect_tx(smem_u32(th_full), th_bytes * (ta.need_lo ? 2 : 1));
        for (int kb = 0; kb < KA; ++kb) {
          tma_load_2d(smem_u32(th_hi + kb * kTM * 128), &tm_hi, kb * AE, t * kTM, smem_u32(th_full));
          if (!TF && ta.need_lo)
            tma_load_2d(smem_u32(th_lo + kb * kTM * 128), &tm_lo, kb * AE, t * kTM, smem_u32(th_full));
        }
        th_issued = seg;
        ++seg;
        return true;
      };
      // the X chunk of unit i (chunk j) into its ring slot
      auto load_x = [&](const int i, const int j) -> bool {
        const int st = i % NS, rnd = i / NS;
        if (!mbar_wait_fast(smem_u32(&x_empty[st]), (rnd & 1) ^ 1, abort_flag, ta.err)) return false;
        mbar_expect_tx(smem_u32(&x_full[st]), x_bytes);
        uint8_t *xb = xs + (size_t)st * x_bytes;
        for (int kb = 0; kb < KA; ++kb)
          tma_load_2d(smem_u32(xb + kb * TN * 128), &tm_x, kb * AE, j * TN, smem_u32(&x_full[st]));
        last_round[st] = rnd;
        return true;
      };
      for (int i = 0, j = j_first; i < nunits; j = j_step(i, j), ++i) {
        const bool sf = !TF && seg_first(i, j);
        if (MS && sf && seg > 0) {
          // the next step's first chunk does not depend on the last step's
          // finish: load it before waiting for the new theta
          if (!load_x(i, j) || !load_theta(i)) break;
          continue;
        }
        if (sf && !load_theta(i)) break;
        if (!load_x(i, j)) break;
      }
      // on abort: let copies already issued land before the CTA exits
      if (*abort_flag) {
        for (int s = 0; s < NS; ++s)
          if (last_round[s] >= 0) mbar_wait_quiet(smem_u32(&x_full[s]), last_round[s] & 1);
        if (th_issued >= 0) mbar_wait_quiet(smem_u32(th_full), th_issued & 1);
      }
    }
  } else if (warp == 1) {
    // ------------------------------ GEMM1 issuer ---------------------------
    // Per unit i: S[i & 1] = Theta . X_chunk^T (hi + lo).  (tile, chunk), stage
    // and parities are tracked incrementally.
    if (lane == 0) {
      const uint32_t id1 = TF ? idesc_tf32(kTM, TN) : idesc_bf16(kTM, kTN, false);
      const uint64_t hd0 = sdesc_sw128(smem_u32(th_hi), 16, 1024);
      const uint64_t ld0 = sdesc_sw128(smem_u32(th_lo), 16, 1024);
      const uint64_t xd_k = sdesc_sw128(smem_u32(xs), 16, 1024);   // K-major view, stage 0
      const uint64_t x_step = (uint64_t)(x_bytes >> 4);
      int seg1 = 0, st = 0, xph = 0;
      for (int i = 0, j = j_first; i < nunits; j = j_step(i, j), ++i) {
        const bool first = seg_first(i, j);
        const bool last = seg_last(i, j);
        if (first && !mbar_wait_fast(smem_u32(th_full), seg1 & 1, abort_flag, ta.err)) break;
        if (!mbar_wait_fast(smem_u32(&x_full[st]), xph, abort_flag, ta.err)) break;
        const int sb = i & 1;
        if (!mbar_wait_fast(smem_u32(&s_empty[sb]), ((i >> 1) & 1) ^ 1, abort_flag, ta.err)) break;
        tc_fence_after();
        const uint64_t xd0 = xd_k + (uint64_t)st * x_step;
        const uint32_t dS = tmem + sb * TN;
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
          // K step ks: 32 bytes into 128-byte atom ks / 4 (16 bf16 or 8 TF32)
          const uint64_t off = (uint64_t)((((ks >> 2) * kTM * 128) + (ks & 3) * 32) >> 4);
          const uint64_t offx = (uint64_t)((((ks >> 2) * TN * 128) + (ks & 3) * 32) >> 4);
          if constexpr (TF) tc_mma_tf32_ta(dS, tmem_T + 8 * ks, xd0 + offx, id1, ks > 0 ? 1u : 0u);
          else tc_mma_bf16(dS, hd0 + off, xd0 + offx, id1, ks > 0 ? 1u : 0u);
        }
        if (!TF && ta.need_lo) {
#pragma unroll
          for (int ks = 0; ks < KS; ++ks) {
            const uint64_t off = (uint64_t)((((ks >> 2) * kTM * 128) + (ks & 3) * 32) >> 4);
            const uint64_t offx = (uint64_t)((((ks >> 2) * kTN * 128) + (ks & 3) * 32) >> 4);
            tc_mma_bf16(dS, ld0 + off, xd0 + offx, id1, 1u);
          }
        }
        tc_commit(smem_u32(&s_full[sb]));
        if constexpr (TF) tc_commit(smem_u32(&x_empty[st]));   // X slot read: free it
        if (last) { tc_commit(smem_u32(th_empty)); ++seg1; }
        if (++st == NS) { st = 0; xph ^= 1; }
      }
    }
  } else if (warp == 2) {
    // ------------------------------ GEMM2 issuer ---------------------------
    // Per unit i: G += R[i & 1] . X_chunk, four K steps (64 rows) per half
    // of R as the epilogue produces it.
    if (lane == 0) {
      const uint32_t id2 = TF ? idesc_tf32(kTM, ta.PN) : idesc_bf16(kTM, ta.PN, true);
      // bf16: X chunk as the MN-major B operand; TF: X^T chunk, K-major, from
      // its own ring
      const uint64_t xd_mn = TF ? sdesc_sw128(smem_u32(xts), 16, 1024)
                                : sdesc_sw128(smem_u32(xs), kTN * 128, 1024);
      const uint64_t x_step = (uint64_t)((TF ? xt_bytes : x_bytes) >> 4);
      const int nring = TF ? NT : NS;
      int seg2 = 0, st = 0, tph = 0;
      for (int i = 0, j = j_first; i < nunits; j = j_step(i, j), ++i) {
        const bool first = seg_first(i, j);
        const bool last = seg_last(i, j);
        const int rb = i & 1;
        const uint32_t a0 = tmem_R + 64 * rb;       // K step ks: 8 columns (16 bf16) at a0 + 8 ks
        const uint64_t bd0 = xd_mn + (uint64_t)st * x_step;
        bool ok = true;
#pragma unroll
        for (int qq = 0; qq < 2 && ok; ++qq) {
          ok = mbar_wait_fast(smem_u32(&r_part[4 * rb + qq]), (i >> 1) & 1, abort_flag, ta.err);
          if (ok && qq == 0 && first) ok = mbar_wait_fast(smem_u32(g_empty), (seg2 & 1) ^ 1, abort_flag, ta.err);
          if (TF && ok && qq == 0) ok = mbar_wait_fast(smem_u32(&xt_full[st]), tph, abort_flag, ta.err);
          if (!ok) break;
          tc_fence_after();
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const int ks = 4 * qq + kk;
            if constexpr (TF)   // 8 rows per K step: 32 bytes into 128-byte atom ks / 4 of X^T
              tc_mma_tf32_ta(tmem_G, a0 + 8 * ks,
                             bd0 + (uint64_t)((((ks >> 2) * ta.PN * 128) + (ks & 3) * 32) >> 4), id2,
                             (first && ks == 0) ? 0u : 1u);
            else                // 16 rows per K step: 2048 bytes of the MN-major X chunk
              tc_mma_bf16_ta(tmem_G, a0 + 8 * ks, bd0 + (uint64_t)((ks * 2048) >> 4), id2,
                             (first && ks == 0) ? 0u : 1u);
          }
        }
        if (!ok) break;
        tc_commit(smem_u32(&r_empty[rb]));
        tc_commit(smem_u32(TF ? &xt_empty[st] : &x_empty[st]));
        if (last) { tc_commit(smem_u32(g_full)); ++seg2; }
        if (++st == nring) { st = 0; tph ^= 1; }
      }
    }
  } else if (warp == 3) {
    // ---------------------------- TMA producer, X^T ------------------------
    // (TF32 form only; idle otherwise)
    if (TF && lane == 0) {
      int last_round[kTcMaxStages];
#pragma unroll
      for (int s2 = 0; s2 < kTcMaxStages; ++s2) last_round[s2] = -1;
      const int nt = TF ? NT : 1;
      for (int i = 0, j = j_first; i < nunits; j = j_step(i, j), ++i) {
        const int st = i % nt, rnd = i / nt;
        if (!mbar_wait_fast(smem_u32(&xt_empty[st]), (rnd & 1) ^ 1, abort_flag, ta.err)) break;
        mbar_expect_tx(smem_u32(&xt_full[st]), xt_bytes);
        uint8_t *xb = xts + (size_t)st * xt_bytes;
        // X^T of the chunk: two 32-row column blocks of PN feature rows
        for (int h = 0; h < 2; ++h)
          tma_load_2d(smem_u32(xb + h * ta.PN * 128), &tm_lo, j * TN + 32 * h, 0, smem_u32(&xt_full[st]));
        last_round[st] = rnd;
      }
      if (*abort_flag)
        for (int s = 0; s < NT; ++s)
          if (last_round[s] >= 0) mbar_wait_quiet(smem_u32(&xt_full[s]), last_round[s] & 1);
    }
  }
  } else {
    // ... and warpgroups 1-2 (epilogue) take them
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kTcRegsEpilogue));
    // ------------------------------ epilogue -------------------------------
    const int ew = warp - 4;                        // epilogue warp 0..7
    const int eg = ew >> 2;                         // warpgroup: units with (i & 1) == eg
    const int q = warp & 3;                         // TMEM lane quarter of this warp
    const int m = q * 32 + lane;                    // chain row within the tile
    const int et = ew * 32 + lane;                  // 0..255
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    constexpr bool accurate = ACC;                  // log densities (a separate instantiation)
    const int wstride = ta.PN + kTcSlots;           // workspace rows per segment
    const int sb = eg, rb = eg;                     // this group's S and R buffers
    int nseg_done = 0;
    bool aborted = false;
    // TF32 form: theta of chain tile tt as the first GEMM's A operand in
    // TMEM, written by the epilogue warps from the shadow array (row m of
    // the tile in TMEM lane m; group eg writes the K steps of its parity).
    // Segment sgi's theta may be written once the first GEMMs of segment
    // sgi - 1 have completed (th_empty); the first GEMM waits for all eight
    // warps (th_full).  Tile rows up to the padded chain count are
    // allocated, so the loads stay in bounds.
    auto theta_to_tmem = [&](const int tt, const int sgi) -> bool {
      if (!warp_wait(smem_u32(th_empty), (sgi & 1) ^ 1, abort_flag, ta.err)) return false;
      tc_fence_after();
      const float *row = ta.shadow32 + ((size_t)tt * kTM + m) * (size_t)ta.KP;
#pragma unroll
      for (int ks = eg; ks < KS; ks += 2) {
        const float4 lo4 = __ldcg(reinterpret_cast<const float4 *>(row + 8 * ks));
        const float4 hi4 = __ldcg(reinterpret_cast<const float4 *>(row + 8 * ks + 4));
        uint32_t v[8] = {__float_as_uint(lo4.x), __float_as_uint(lo4.y), __float_as_uint(lo4.z),
                         __float_as_uint(lo4.w), __float_as_uint(hi4.x), __float_as_uint(hi4.y),
                         __float_as_uint(hi4.z), __float_as_uint(hi4.w)};
        PCV_TMEM_ST8(tmem_T + 8 * ks + lane_off, v);
        tmem_wait_st();
        tmem_fence_regs(v);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(th_full));
      return true;
    };
    // walk the CTA's segments (maximal runs of units in one tile)
    if constexpr (TF) {
      if (nunits > 0 && !theta_to_tmem((int)(unit_of(0) / ta.J), 0)) aborted = true;
    }
    for (int ib = 0; ib < nunits && !aborted; ) {
      const long long ub = unit_of(ib);
      const int t = (int)(ub / ta.J), j0 = (int)(ub - (long long)t * ta.J);
      // segment [ib, ie): the rotated first piece, or up to the tile's end
      const int ie = ib < rot ? rot : min(nunits, ib + (ta.J - j0));
      const int c = t * kTM + m;
      const bool valid = c < a.C;
      FoldDesc fd = {0, 0, 0, 0};
      if (valid) fd = pb.folds[fold_of_chain(a, c)];
      // per-chain sums over the fold's training and test rows: softplus(eta)
      // (logistic) or squared residuals (Gaussian models)
      // (each as an FP32 pair hi + lo kept exact by TwoSum: FP64 arithmetic
      // is slow on this part, and a per-quarter FP64 add paced the
      // log-density launch)
      float tr_hi = 0.0f, tr_lo = 0.0f, te_hi = 0.0f, te_lo = 0.0f;
      // Gaussian models: 1 / sigma^2 of the chain (sigma known, or exp of the
      // log sigma coordinate after beta; theta only moves in the finish)
      float inv_s2 = 1.0f;
      if constexpr (GAUSS) {
        if (pb.variant == MV_GAUSS_LOGSIG)
          inv_s2 = valid ? expf(-2.0f * a.theta[(size_t)c * a.ld_theta + pb.p]) : 1.0f;
        else
          inv_s2 = 1.0f / (pb.sigma_known * pb.sigma_known);
      }
      const bool need_e2 = GAUSS && (ACC || pb.variant == MV_GAUSS_LOGSIG);
      for (int i = ib + ((ib & 1) != eg ? 1 : 0); i < ie; i += 2) {
        const int j = j0 + (i - ib);
        if (!warp_wait(smem_u32(&s_full[sb]), (i >> 1) & 1, abort_flag, ta.err)) { aborted = true; break; }
        tc_fence_after();
        // residuals r of quarter qq (32 rows) of the chunk from v = S (FP32,
        // the fold's excluded rows not yet masked), plus the log-likelihood
        // or squared-residual sums
        auto quarter = [&](const int qq, const uint32_t (&v)[32], float (&r)[32]) {
          const int n0 = j * TN + 32 * qq;
          if constexpr (!GAUSS) {
            // 1 - tanh(S) in FP32 (twice the residual along the sign-folded
            // row), rounded to bf16 (or TF32) for the second GEMM.  A bf16x2
            // tanh here would bias the gradient: its error is a smooth
            // function of eta, so it adds up over rows instead of averaging
            // out (a force error of ~6 % of the posterior scale per dimension
            // at N = 1e5, which shrinks the adapted step size).
#pragma unroll
            for (int k = 0; k < 32; ++k) r[k] = 1.0f - tanh_f32(__uint_as_float(v[k]));
            if constexpr (accurate) {
              // log likelihood y eta - softplus(eta) = -softplus(-2 S) with
              // the sign-folded S: softplus(-2 S) = max(-2 S, 0) +
              // log(1 + exp(-|2 S|)) is summed here, in FP32 per quarter and
              // as an exact FP32 pair across quarters.
              // Quarters clear of the fold's excluded rows and of the
              // padding need no per-row mask; there the logs of eight rows
              // are taken at once, as the log of the product of their
              // factors 1 + exp(-|eta|) (each in (1, 2], so the product stays
              // below 2^8): one lg2 per eight rows instead of one per row
              // (the log-density launch is bound by its MUFU and issue
              // slots).  Against an FP64 sum this moves log pi by a constant
              // 4e-8 per row, the same at every theta, so H1 - H0 keeps its
              // accuracy.
              if (n0 + 32 <= pb.N && (n0 + 32 <= fd.excl_lo || n0 >= fd.excl_hi)) {
                float pr[4] = {1.0f, 1.0f, 1.0f, 1.0f}, mx[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                  const float s = __uint_as_float(v[k]);
                  pr[k & 3] = fmaf(pr[k & 3], exp_neg_abs_eta(s), pr[k & 3]);
                  mx[k & 3] += fmaxf(-s, 0.0f);
                }
                float lg[4];
#pragma unroll
                for (int g = 0; g < 4; ++g) lg[g] = log2_approx(pr[g]);
                two_sum_add(tr_hi, tr_lo, fmaf((lg[0] + lg[1]) + (lg[2] + lg[3]), 0.6931471805599453f,
                                               2.0f * ((mx[0] + mx[1]) + (mx[2] + mx[3]))));
              } else {
                // rare (the quarter meets the fold's excluded rows or the
                // padding): a rolled loop over a local copy keeps this
                // path's code small, which the instruction cache of the
                // log-density launch needs
                float sq[32];
#pragma unroll
                for (int k = 0; k < 32; ++k) sq[k] = __uint_as_float(v[k]);
                float tr = 0.0f, te = 0.0f;
#pragma unroll 1
                for (int k = 0; k < 32; ++k) {
                  const int n = n0 + k;
                  const float sp = softplus_half(-sq[k]);
                  if (n < pb.N && (n < fd.excl_lo || n >= fd.excl_hi)) tr += sp;
                  if (n >= fd.test_lo && n < fd.test_hi) te += sp;
                }
                two_sum_add(tr_hi, tr_lo, tr);
                two_sum_add(te_hi, te_lo, te);
              }
            }
          } else {
            // Gaussian: residual (y - eta) / sigma^2 = -2 S / sigma^2; the
            // squared residuals of the fold's training and test rows feed the
            // log sigma gradient and the log densities
            float e[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) {
              e[k] = -2.0f * __uint_as_float(v[k]);
              r[k] = e[k] * inv_s2;
            }
            if (need_e2) {
              if (n0 + 32 <= pb.N && (n0 + 32 <= fd.excl_lo || n0 >= fd.excl_hi)) {
                float acc4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int k = 0; k < 32; ++k) acc4[k & 3] = fmaf(e[k], e[k], acc4[k & 3]);
                two_sum_add(tr_hi, tr_lo, (acc4[0] + acc4[1]) + (acc4[2] + acc4[3]));
              } else {
                float sq[32];                      // rolled, as for the softplus sums
#pragma unroll
                for (int k = 0; k < 32; ++k) sq[k] = e[k];
                float tr = 0.0f, te = 0.0f;
#pragma unroll 1
                for (int k = 0; k < 32; ++k) {
                  const int n = n0 + k;
                  const float e2 = sq[k] * sq[k];
                  if (n < pb.N && (n < fd.excl_lo || n >= fd.excl_hi)) tr += e2;
                  if (n >= fd.test_lo && n < fd.test_hi) te += e2;
                }
                two_sum_add(tr_hi, tr_lo, tr);
                two_sum_add(te_hi, te_lo, te);
              }
            }
          }
        };
        // the bf16 form of quarter qq: 16 bf16x2 (rows 2c, 2c + 1 in column c),
        // the fold's excluded rows zeroed
        auto pack16 = [&](const int qq, const float (&r)[32], uint32_t (&pk)[16]) {
#pragma unroll
          for (int k = 0; k < 16; ++k) pk[k] = bf16x2_from(r[2 * k], r[2 * k + 1]);
          const int n0 = j * TN + 32 * qq;
          if (valid && n0 < fd.excl_hi && n0 + 32 > fd.excl_lo) {
#pragma unroll
            for (int k = 0; k < 32; ++k) {
              const int n = n0 + k;
              if (n >= fd.excl_lo && n < fd.excl_hi) pk[k >> 1] &= (k & 1) ? 0x0000FFFFu : 0xFFFF0000u;
            }
          }
        };
        // the TF32 form: one element per column, the excluded rows zeroed
        auto pack32 = [&](const int qq, const float (&r)[32], uint32_t (&pk)[32]) {
#pragma unroll
          for (int k = 0; k < 32; ++k) pk[k] = tf32_bits(r[k]);
          const int n0 = j * TN + 32 * qq;
          if (valid && n0 < fd.excl_hi && n0 + 32 > fd.excl_lo) {
#pragma unroll
            for (int k = 0; k < 32; ++k) {
              const int n = n0 + k;
              if (n >= fd.excl_lo && n < fd.excl_hi) pk[k] = 0u;
            }
          }
        };
        if constexpr (ACC || TF) {
          // a rolled loop over the quarters, each loaded from TMEM on its own:
          // the log-density launch (one of L_f per iteration: small code for
          // the instruction cache) and the TF32 form (two quarters per
          // chunk); S is released after the last quarter's load, and each
          // stored half of R (TF32: each quarter) is handed to the second
          // GEMM at once
          const uint32_t rbuf = tmem_R + 64 * rb + lane_off;
#pragma unroll 1
          for (int qq = 0; qq < NQ; ++qq) {
            uint32_t v[32];
            float r[32];
            PCV_TMEM_LD32(tmem + sb * TN + lane_off + 32 * qq, v);
            tmem_wait_ld();
            tmem_fence_regs(v);
            if (qq == NQ - 1) {
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(smem_u32(&s_empty[sb]));
            }
            quarter(qq, v, r);
            if (qq == 0) {
              if (!warp_wait(smem_u32(&r_empty[rb]), ((i >> 1) & 1) ^ 1, abort_flag, ta.err)) {
                aborted = true;
                break;
              }
              tc_fence_after();
            }
            if constexpr (TF) {
              uint32_t pk[32];
              pack32(qq, r, pk);
              PCV_TMEM_ST32(rbuf + 32 * qq, pk);
              tmem_wait_st();
              tmem_fence_regs(pk);
            } else {
              uint32_t pk[16];
              pack16(qq, r, pk);
              PCV_TMEM_ST16(rbuf + 16 * qq, pk);
              tmem_wait_st();
              tmem_fence_regs(pk);
            }
            if (TF || (qq & 1)) {
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(smem_u32(&r_part[4 * rb + (TF ? qq : qq >> 1)]));
            }
          }
          if (aborted) break;
          continue;
        }
        uint32_t sv[128], p0[16], p1[16], p2[16], p3[16];
        PCV_TMEM_LD128(tmem + sb * TN + lane_off, sv);   // one load: ~2 % faster than four x32
        tmem_wait_ld();
        tmem_fence_regs(sv);
        // the four 32-row quarters of the row (constant indices: registers)
        const uint32_t (&v0)[32] = *reinterpret_cast<const uint32_t (*)[32]>(&sv[0]);
        const uint32_t (&v1)[32] = *reinterpret_cast<const uint32_t (*)[32]>(&sv[32]);
        const uint32_t (&v2)[32] = *reinterpret_cast<const uint32_t (*)[32]>(&sv[64]);
        const uint32_t (&v3)[32] = *reinterpret_cast<const uint32_t (*)[32]>(&sv[96]);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&s_empty[sb]));   // S fully read: release it
        {
          float r[32];
          quarter(0, v0, r);
          pack16(0, r, p0);
        }
        if (!warp_wait(smem_u32(&r_empty[rb]), ((i >> 1) & 1) ^ 1, abort_flag, ta.err)) { aborted = true; break; }
        tc_fence_after();
        // R row m (TMEM lane m): chunk rows 2c, 2c + 1 in bf16x2 column c
        const uint32_t rbuf = tmem_R + 64 * rb + lane_off;
        // a half's stores complete while the next quarter is computed; then
        // the second GEMM may take it (handing R over by quarters measured
        // 0.556 ms per launch, by halves 0.541, whole 0.543)
        auto quarter_stored = [&](int qq) {
          tmem_wait_st();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&r_part[4 * rb + qq]));
        };
        PCV_TMEM_ST16(rbuf, p0);
        {
          float r[32];
          quarter(1, v1, r);
          pack16(1, r, p1);
        }
        PCV_TMEM_ST16(rbuf + 16, p1);
        {
          float r[32];
          quarter(2, v2, r);
          pack16(2, r, p2);
        }
        quarter_stored(0);
        tmem_fence_regs(p0);
        tmem_fence_regs(p1);
        PCV_TMEM_ST16(rbuf + 32, p2);
        {
          float r[32];
          quarter(3, v3, r);
          pack16(3, r, p3);
        }
        PCV_TMEM_ST16(rbuf + 48, p3);
        quarter_stored(1);
        tmem_fence_regs(p2);
        tmem_fence_regs(p3);
      }
      if (aborted) break;
      // TF32: the next segment's theta goes to TMEM before this
      // segment's finish, so that its first GEMMs need not wait for it
      // (several steps per launch: the next segment is this tile's next
      // step, whose theta comes from this finish, so it goes after it)
      if constexpr (TF && !MS) {
        if (ie < nunits && !theta_to_tmem((int)(unit_of(ie) / ta.J), nseg_done + 1)) break;
      }
      // ---- segment end (both groups): the group that owns the segment's
      // last unit flushes this tile's G partial; both write their ll sums
      const int owner = (ie - 1) & 1;
      const int fl = nseg_done++;
      const int b0 = owner_cta((long long)t * ta.J, U, ta.n_cta);
      const int sidx = blockIdx.x - b0;
      // workspace rows are chain-major ([chain][PN + slots]) so that the
      // finish reads them in the layout of theta / grad (coalesced)
      float *wsp = ta.ws + ((size_t)t * ta.max_seg + sidx) * (size_t)wstride * kTM;
      float *wrow = wsp + (size_t)m * wstride;
      if (eg == owner) {
        if (!warp_wait(smem_u32(g_full), fl & 1, abort_flag, ta.err)) break;
        tc_fence_after();
        for (int cb = 0; cb < ta.PN; cb += 16) {
          uint32_t gv[16];
          PCV_TMEM_LD16(tmem_G + cb + lane_off, gv);
          tmem_wait_ld();
#pragma unroll
          for (int k = 0; k < 16; k += 4)
            __stcg(reinterpret_cast<float4 *>(wrow + cb + k),
                   make_float4(__uint_as_float(gv[k]), __uint_as_float(gv[k + 1]),
                               __uint_as_float(gv[k + 2]), __uint_as_float(gv[k + 3])));
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(g_empty));
      }
      {
        __stcg(reinterpret_cast<float4 *>(wrow + ta.PN + 4 * eg), make_float4(tr_hi, tr_lo, te_hi, te_lo));
      }
      __threadfence();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(flush_bar));
      if (!warp_wait(smem_u32(flush_bar), fl & 1, abort_flag, ta.err)) break;
      const int nseg = owner_cta((long long)t * ta.J + ta.J - 1, U, ta.n_cta) - b0 + 1;
      if (et == 0) {
        if constexpr (MS) {
          *last_flag = 1;                           // the CTA is the tile's only owner
        } else {
          __threadfence();
          const unsigned prev = atomicAdd(ta.tickets + t, 1u);
          *last_flag = (prev == (unsigned)nseg - 1);
          if (prev == (unsigned)nseg - 1) ta.tickets[t] = 0u;
        }
        mbar_arrive(smem_u32(decide_bar));
      }
      if (!warp_wait(smem_u32(decide_bar), fl & 1, abort_flag, ta.err)) break;
      if (*last_flag) {
        // ---- last segment of tile t: sum the segments in order, priors,
        // leapfrog update.  No shared memory is involved, so the epilogue
        // warps need no barrier inside the finish.
        __threadfence();
        const float *base = ta.ws + (size_t)t * ta.max_seg * (size_t)wstride * kTM;
        const size_t seg_stride = (size_t)wstride * kTM;
        const float eps = a.mode != MODE_NONE ? *a.eps : 0.0f;
        const float kick = a.mode == MODE_LAST_KICK ? 0.5f * eps : eps;
        // (chain, 4 dimensions) items spread over all 256 epilogue threads,
        // kFinU items per thread at a time with all their loads issued before
        // any arithmetic: a serial item loop waited on every load in turn and
        // took ~50 us per tile.  Consecutive items are consecutive
        // dimensions of one chain (coalesced float4 accesses).
        const int p_ = pb.p;
        const bool vec = ((a.ld_theta | a.ld_grad) & 3) == 0 &&
                         ((reinterpret_cast<uintptr_t>(a.theta) | reinterpret_cast<uintptr_t>(a.grad) |
                           reinterpret_cast<uintptr_t>(a.r)) & 15) == 0;
        const int nq = vec ? p_ >> 2 : 0;           // whole quads per chain
        const bool kd = a.mode == MODE_KICK_DRIFT;
        constexpr int kFinU = 4;
        for (int i0 = et; i0 < kTM * nq; i0 += 256 * kFinU) {
          float4 tv[kFinU], gs[kFinU], rv[kFinU], mv[kFinU], rf[kFinU];
          int cc_[kFinU], jj_[kFinU];
          bool ok[kFinU];
#pragma unroll
          for (int u = 0; u < kFinU; ++u) {
            const int it = i0 + 256 * u;
            const int mm = it / max(nq, 1);
            jj_[u] = 4 * (it - mm * nq);
            cc_[u] = t * kTM + mm;
            ok[u] = it < kTM * nq && cc_[u] < a.C;
            tv[u] = gs[u] = rv[u] = mv[u] = rf[u] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (ok[u]) {
              tv[u] = *reinterpret_cast<const float4 *>(a.theta + (size_t)cc_[u] * a.ld_theta + jj_[u]);
              for (int s2 = 0; s2 < nseg; ++s2) {
                const float4 w = __ldcg(reinterpret_cast<const float4 *>(base + s2 * seg_stride +
                                                                         (size_t)mm * wstride + jj_[u]));
                gs[u].x += w.x; gs[u].y += w.y; gs[u].z += w.z; gs[u].w += w.w;
              }
              if (a.mode != MODE_NONE)
                rv[u] = *reinterpret_cast<const float4 *>(a.r + (size_t)cc_[u] * a.ld_theta + jj_[u]);
              if (kd) {
                mv[u] = *reinterpret_cast<const float4 *>(minv_row(a.minv, cc_[u], a.minv_every, a.minv_ld) + jj_[u]);
                rf[u] = *reinterpret_cast<const float4 *>(ta.theta_ref + jj_[u]);
              }
            }
          }
#pragma unroll
          for (int u = 0; u < kFinU; ++u) {
            if (!ok[u]) continue;
            const float gsc = GAUSS ? 1.0f : 0.5f;   // logistic: the likelihood gradient is G / 2
            const float4 g = make_float4(fmaf(gsc, gs[u].x, -tv[u].x * pb.beta_prec),
                                         fmaf(gsc, gs[u].y, -tv[u].y * pb.beta_prec),
                                         fmaf(gsc, gs[u].z, -tv[u].z * pb.beta_prec),
                                         fmaf(gsc, gs[u].w, -tv[u].w * pb.beta_prec));
            *reinterpret_cast<float4 *>(a.grad + (size_t)cc_[u] * a.ld_grad + jj_[u]) = g;
            if (a.mode == MODE_NONE) continue;
            const float4 r4 = make_float4(rv[u].x + kick * g.x, rv[u].y + kick * g.y, rv[u].z + kick * g.z,
                                          rv[u].w + kick * g.w);
            *reinterpret_cast<float4 *>(a.r + (size_t)cc_[u] * a.ld_theta + jj_[u]) = r4;
            if (!kd) continue;
            const float4 tn = make_float4(tv[u].x + eps * mv[u].x * r4.x, tv[u].y + eps * mv[u].y * r4.y,
                                          tv[u].z + eps * mv[u].z * r4.z, tv[u].w + eps * mv[u].w * r4.w);
            *reinterpret_cast<float4 *>(const_cast<float *>(a.theta) + (size_t)cc_[u] * a.ld_theta + jj_[u]) = tn;
            // shadows hold (theta - ref) / 2 as bf16 hi + lo (TF32: one part)
            const float h0 = 0.5f * (tn.x - rf[u].x), h1 = 0.5f * (tn.y - rf[u].y);
            const float h2 = 0.5f * (tn.z - rf[u].z), h3 = 0.5f * (tn.w - rf[u].w);
            if constexpr (TF) {
              *reinterpret_cast<uint4 *>(ta.shadow32 + (size_t)cc_[u] * a.ld_shadow + jj_[u]) =
                  make_uint4(tf32_bits(h0), tf32_bits(h1), tf32_bits(h2), tf32_bits(h3));
              continue;
            }
            const uint32_t hi01 = bf16x2_from(h0, h1), hi23 = bf16x2_from(h2, h3);
            const float l0 = h0 - __uint_as_float(hi01 << 16), l1 = h1 - __uint_as_float(hi01 & 0xFFFF0000u);
            const float l2 = h2 - __uint_as_float(hi23 << 16), l3 = h3 - __uint_as_float(hi23 & 0xFFFF0000u);
            const size_t so = (size_t)cc_[u] * a.ld_shadow + jj_[u];
            *reinterpret_cast<uint2 *>(a.shadow_hi + so) = make_uint2(hi01, hi23);
            *reinterpret_cast<uint2 *>(a.shadow_lo + so) = make_uint2(bf16x2_from(l0, l1), bf16x2_from(l2, l3));
          }
        }
        // the remaining dimensions (p mod 4 of every chain, or all of them
        // when the caller's layout does not allow float4 access), one by one
        const int j_s = 4 * nq, n_rem = p_ - j_s;
        for (int it = et; it < kTM * n_rem; it += 256) {
          const int mm = it / n_rem, jj = j_s + (it - mm * n_rem);
          const int cc = t * kTM + mm;
          if (cc >= a.C) break;
          float *th = const_cast<float *>(a.theta) + (size_t)cc * a.ld_theta;
          const float tv = th[jj];
          float gs = 0.0f;
          for (int s2 = 0; s2 < nseg; ++s2) gs += __ldcg(base + s2 * seg_stride + (size_t)mm * wstride + jj);
          const float g = fmaf(GAUSS ? 1.0f : 0.5f, gs, -tv * pb.beta_prec);
          a.grad[(size_t)cc * a.ld_grad + jj] = g;
          if (a.mode != MODE_NONE) {
            float *rr = a.r + (size_t)cc * a.ld_theta;
            const float rj = rr[jj] + kick * g;
            rr[jj] = rj;
            if (kd) {
              const float tn = tv + eps * minv_row(a.minv, cc, a.minv_every, a.minv_ld)[jj] * rj;
              th[jj] = tn;
              const float half = 0.5f * (tn - ta.theta_ref[jj]);   // shadows hold (theta - ref) / 2
              if constexpr (TF) {
                ta.shadow32[(size_t)cc * a.ld_shadow + jj] = __uint_as_float(tf32_bits(half));
                continue;
              }
              const __nv_bfloat16 hi = __float2bfloat16_rn(half);
              a.shadow_hi[(size_t)cc * a.ld_shadow + jj] = hi;
              a.shadow_lo[(size_t)cc * a.ld_shadow + jj] = __float2bfloat16_rn(half - __bfloat162float(hi));
            }
          }
        }
        // per-chain row sums of the segments (softplus or squared residuals)
        const bool need_sums = a.need_ll || (GAUSS && pb.variant == MV_GAUSS_LOGSIG);
        double s0 = 0.0, s1 = 0.0;                  // over the training / test rows
        const int cc = t * kTM + et;
        if (need_sums && et < kTM && cc < a.C) {
          for (int s2 = 0; s2 < nseg; ++s2) {
            const float *ws2 = base + s2 * seg_stride + (size_t)et * wstride + ta.PN;
#pragma unroll
            for (int g2 = 0; g2 < 2; ++g2) {
              s0 += (double)__ldcg(ws2 + 4 * g2 + 0) + (double)__ldcg(ws2 + 4 * g2 + 1);
              s1 += (double)__ldcg(ws2 + 4 * g2 + 2) + (double)__ldcg(ws2 + 4 * g2 + 3);
            }
          }
        }
        if constexpr (GAUSS) {
          // log sigma (after beta), sigma ~ half-N(0, sd^2):
          // d/dlog sigma = sum_train (e^2 / sigma^2 - 1) - sigma^2 / sd^2 + 1
          if (pb.variant == MV_GAUSS_LOGSIG && et < kTM && cc < a.C) {
            const FoldDesc f = pb.folds[fold_of_chain(a, cc)];
            const double n_tr = (double)(pb.N - (f.excl_hi - f.excl_lo));
            float *th = const_cast<float *>(a.theta) + (size_t)cc * a.ld_theta;
            const float ls = th[pb.p];
            const float s2v = expf(2.0f * ls), is2 = expf(-2.0f * ls);
            const float g = (float)((double)is2 * s0 - n_tr) - s2v * pb.sigma_prec + 1.0f;
            a.grad[(size_t)cc * a.ld_grad + pb.p] = g;
            if (a.mode != MODE_NONE) {
              float *rr = a.r + (size_t)cc * a.ld_theta;
              const float rj = rr[pb.p] + kick * g;
              rr[pb.p] = rj;
              if (kd) th[pb.p] = ls + eps * minv_row(a.minv, cc, a.minv_every, a.minv_ld)[pb.p] * rj;
            }
          }
        }
        if (a.need_ll && et < kTM && cc < a.C) {
          // (theta is not moved on the steps that need log densities, so it
          // is the evaluation point)
          const float *th = a.theta + (size_t)cc * a.ld_theta;
          if constexpr (!GAUSS) {
            // the log prior, in a fixed order; the likelihood sums are -s0, -s1
            double q = 0.0;
#pragma unroll 4
            for (int jj = 0; jj < pb.p; ++jj) q = fma((double)th[jj], (double)th[jj], q);
            const double lprior = (double)pb.p * (-0.5 * kLog2PiD - (double)pb.log_beta_sd) - 0.5 * pb.beta_prec * q;
            a.logp[cc] = lprior - s0;
            a.shat[cc] = -s1;
          } else {
            // sum of -log(2 pi)/2 - log sigma - e^2 / (2 sigma^2) over the
            // fold's training / test rows, and the log priors
            double q = 0.0;
#pragma unroll 4
            for (int jj = 0; jj < pb.p; ++jj) q = fma((double)th[jj], (double)th[jj], q);
            double lprior = (double)pb.p * (-0.5 * kLog2PiD - (double)pb.log_beta_sd) - 0.5 * pb.beta_prec * q;
            double ls, is2;
            if (pb.variant == MV_GAUSS_LOGSIG) {
              const float lsf = th[pb.p];
              const float s2v = expf(2.0f * lsf);
              ls = (double)lsf;
              is2 = (double)expf(-2.0f * lsf);
              lprior += kLog2D - 0.5 * kLog2PiD - pb.log_sigma_sd - 0.5 * (double)s2v * pb.sigma_prec + ls;
            } else {
              ls = (double)logf(pb.sigma_known);
              is2 = (double)(1.0f / (pb.sigma_known * pb.sigma_known));
            }
            const FoldDesc f = pb.folds[fold_of_chain(a, cc)];
            const double n_tr = (double)(pb.N - (f.excl_hi - f.excl_lo)), n_te = (double)(f.test_hi - f.test_lo);
            a.logp[cc] = -0.5 * is2 * s0 - n_tr * (0.5 * kLog2PiD + ls) + lprior;
            a.shat[cc] = -0.5 * is2 * s1 - n_te * (0.5 * kLog2PiD + ls);
          }
        }
      }
      // several steps per launch: every epilogue thread's finish writes
      // (theta, momentum, gradient, shadows) precede the next step, both
      // the producer's TMA load of the new shadow (async proxy: hence the
      // proxy fence) and the epilogue's own reads of theta
      if constexpr (MS) {
        asm volatile("fence.proxy.async.global;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(th_ready));
        if (!warp_wait(smem_u32(th_ready), fl & 1, abort_flag, ta.err)) break;
        // TF32: the new theta into TMEM for the next step's first GEMMs
        if constexpr (TF) {
          if (ie < nunits && !theta_to_tmem((int)(unit_of(ie) / ta.J), nseg_done)) break;
        }
      }
      ib = ie;
    }
    // back to the producers' count, so that all warps meet the teardown alike
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kTcRegsProducer));
  }

  // teardown: every role has left its loop (normally or by abort)
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
size_t tc_smem_bytes(int KP, int NS, int NT, int need_lo, int p, int tf32, int PN) {
  (void)p;
  size_t b;
  if (tf32) {   // NS 64-row X chunks and NT X^T chunks (2 x PN rows of 128 B); theta is in TMEM
    const size_t KA = KP / 32;
    b = (size_t)NS * KA * 64 * 128 + (size_t)NT * 2 * PN * 128;
  } else {
    const size_t KA = KP / 64;
    b = KA * kTM * 128 * (need_lo ? 2 : 1) + (size_t)NS * KA * kTN * 128;
  }
  b += 64 + (4 * kTcMaxStages + 24) * 8;   // barrier / flag slots
  return b + 1024;                          // alignment slack
}

int tc_max_stages() { return kTcMaxStages; }

int tc_segments_per_tile(int T, int J, int n_cta) {
  const long long U = (long long)T * J;
  int mx = 1;
  for (int t = 0; t < T; ++t) {
    const int b0 = owner_cta((long long)t * J, U, n_cta);
    const int b1 = owner_cta((long long)t * J + J - 1, U, n_cta);
    mx = mx > b1 - b0 + 1 ? mx : b1 - b0 + 1;
  }
  return mx;
}

template <int KS, bool TF>
static cudaError_t set_smem_attr() {
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t r[6] = {cudaFuncSetAttribute(k_grad_tc<KS, false, false, TF>, at, 227 * 1024),
                      cudaFuncSetAttribute(k_grad_tc<KS, true, false, TF>, at, 227 * 1024),
                      cudaFuncSetAttribute(k_grad_tc<KS, false, true, TF>, at, 227 * 1024),
                      cudaFuncSetAttribute(k_grad_tc<KS, true, true, TF>, at, 227 * 1024),
                      cudaSuccess, cudaSuccess};
  // the several-steps kick-drift kernels
  r[4] = cudaFuncSetAttribute(k_grad_tc<KS, false, false, TF, true>, at, 227 * 1024);
  r[5] = cudaFuncSetAttribute(k_grad_tc<KS, false, true, TF, true>, at, 227 * 1024);
  for (cudaError_t x : r)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}

// setmaxnreg.inc waits until the CTA's register pool can grant the request:
// the pool is what the CTA was launched with (threads x the compiled register
// count), so a split larger than that would never be granted.  Every
// instantiation is checked once; launches are refused if any fails.
static bool g_tc_regs_ok = false;
template <int KS, bool TF>
static bool regs_fit() {
  const long need = 128L * kTcRegsProducer + 256L * kTcRegsEpilogue;
  cudaFuncAttributes fa[6];
  if (cudaFuncGetAttributes(&fa[0], k_grad_tc<KS, false, false, TF>) != cudaSuccess ||
      cudaFuncGetAttributes(&fa[1], k_grad_tc<KS, true, false, TF>) != cudaSuccess ||
      cudaFuncGetAttributes(&fa[2], k_grad_tc<KS, false, true, TF>) != cudaSuccess ||
      cudaFuncGetAttributes(&fa[3], k_grad_tc<KS, true, true, TF>) != cudaSuccess)
    return false;
  if (cudaFuncGetAttributes(&fa[4], k_grad_tc<KS, false, false, TF, true>) != cudaSuccess ||
      cudaFuncGetAttributes(&fa[5], k_grad_tc<KS, false, true, TF, true>) != cudaSuccess)
    return false;
  for (const cudaFuncAttributes &f : fa)
    if ((long)f.numRegs * kTcThreads < need) return false;
  return true;
}

template <int... K>
static bool all_prepared(std::integer_sequence<int, K...>) {
  bool ok = true;
  ((ok = ok && set_smem_attr<K + 1, false>() == cudaSuccess && regs_fit<K + 1, false>()), ...);
  return ok;
}
template <int... K>
static bool all_prepared_tf(std::integer_sequence<int, K...>) {
  bool ok = true;
  ((ok = ok && set_smem_attr<K + 1, true>() == cudaSuccess && regs_fit<K + 1, true>()), ...);
  return ok;
}

// once per context (outside any stream capture): allow the large dynamic SMEM
// (bf16 form: K steps 1 .. 9, p <= 128; TF32 form: 1 .. 15, p <= 112)
cudaError_t tc_prepare() {
  g_tc_regs_ok = all_prepared(std::make_integer_sequence<int, 9>{}) &&
                 all_prepared_tf(std::make_integer_sequence<int, 15>{});
  return g_tc_regs_ok ? cudaSuccess : cudaErrorInvalidConfiguration;
}

template <int K, bool TF>
static void launch_k(bool gauss, bool accurate, const CUtensorMap &tm_x, const CUtensorMap &tm_hi,
                     const CUtensorMap &tm_lo, const Problem &pb, const GradArgs &a, const TcArgs &ta, size_t smem,
                     cudaStream_t st) {
  if (ta.steps > 1) {   // several kick-drift steps (the caller checked the grid)
    if (gauss) k_grad_tc<K, false, true, TF, true><<<ta.n_cta, kTcThreads, smem, st>>>(tm_x, tm_hi, tm_lo, pb, a, ta);
    else k_grad_tc<K, false, false, TF, true><<<ta.n_cta, kTcThreads, smem, st>>>(tm_x, tm_hi, tm_lo, pb, a, ta);
    return;
  }
  if (gauss) {
    if (accurate) k_grad_tc<K, true, true, TF><<<ta.n_cta, kTcThreads, smem, st>>>(tm_x, tm_hi, tm_lo, pb, a, ta);
    else k_grad_tc<K, false, true, TF><<<ta.n_cta, kTcThreads, smem, st>>>(tm_x, tm_hi, tm_lo, pb, a, ta);
  } else {
    if (accurate) k_grad_tc<K, true, false, TF><<<ta.n_cta, kTcThreads, smem, st>>>(tm_x, tm_hi, tm_lo, pb, a, ta);
    else k_grad_tc<K, false, false, TF><<<ta.n_cta, kTcThreads, smem, st>>>(tm_x, tm_hi, tm_lo, pb, a, ta);
  }
}

template <bool TF, int... K>
static bool launch_ks(int ks, std::integer_sequence<int, K...>, bool gauss, bool accurate, const CUtensorMap &tm_x,
                      const CUtensorMap &tm_hi, const CUtensorMap &tm_lo, const Problem &pb, const GradArgs &a,
                      const TcArgs &ta, size_t smem, cudaStream_t st) {
  bool done = false;
  ((ks == K + 1 ? (launch_k<K + 1, TF>(gauss, accurate, tm_x, tm_hi, tm_lo, pb, a, ta, smem, st), done = true)
                : false), ...);
  return done;
}

cudaError_t launch_grad_tc(const CUtensorMap &tm_x, const CUtensorMap &tm_hi, const CUtensorMap &tm_lo,
                           const Problem &pb, const GradArgs &a, const TcArgs &ta, cudaStream_t st) {
  const size_t smem = tc_smem_bytes(ta.KP, ta.NS, ta.NT, ta.need_lo, pb.p, ta.tf32, ta.PN);
  if (ta.NS < 1 || ta.NS > kTcMaxStages || (ta.tf32 && (ta.NT < 1 || ta.NT > kTcMaxStages)))
    return cudaErrorInvalidValue;
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  if (!g_tc_regs_ok) return cudaErrorInvalidConfiguration;   // tc_prepare not run, or the split does not fit
  if (pb.variant == MV_HIER) return cudaErrorInvalidValue;
  if (ta.tf32 && ta.need_lo) return cudaErrorInvalidValue;    // the TF32 form has no lo part
  // several steps per launch: kick-drift steps, one CTA per tile
  if (ta.steps > 1 && (ta.n_cta != ta.T || a.mode != MODE_KICK_DRIFT || a.need_ll))
    return cudaErrorInvalidValue;
  const bool gauss = pb.variant == MV_GAUSS_KNOWN || pb.variant == MV_GAUSS_LOGSIG;
  const bool ok = ta.tf32 ? launch_ks<true>(ta.KS, std::make_integer_sequence<int, 15>{}, gauss, ta.accurate != 0,
                                           tm_x, tm_hi, tm_lo, pb, a, ta, smem, st)
                          : launch_ks<false>(ta.KS, std::make_integer_sequence<int, 9>{}, gauss, ta.accurate != 0,
                                             tm_x, tm_hi, tm_lo, pb, a, ta, smem, st);
  if (!ok) return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace pcv
