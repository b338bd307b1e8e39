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

#include "pcv_internal.cuh"

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


// softplus(eta) for eta = 2 s (the first GEMM yields s = eta / 2):
// max(eta, 0) + ln 2 * log2(1 + 2^(-|eta| log2 e)) with the PTX ex2 / lg2
// approximations
__device__ __forceinline__ float exp_neg_abs_eta(float s) {   // e^-|eta|, eta = 2 s
  float e;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(fabsf(s) * -2.8853900817779268f));
  return e;
}
__device__ __forceinline__ float log2_approx(float x) {
  float l;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(x));
  return l;
}
__device__ __forceinline__ float softplus_half(float s) {
  const float m = fmaxf(s, 0.0f);
  return fmaf(log2_approx(1.0f + exp_neg_abs_eta(s)), 0.6931471805599453f, m + m);
}

// ----------------------------- PTX helpers --------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait (2 s of wall time).  Returns false on time-out or abort.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                       unsigned int *err) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (global_ns() - t0 > 2000000000ull) {
      atomicOr(err, 1u);
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Non-blocking check first (cheap when the phase has completed), then the
// bounded blocking wait.
__device__ __forceinline__ bool mbar_wait_fast(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                               unsigned int *err) {
  return mbar_test(bar, parity) || mbar_wait(bar, parity, abort_flag, err);
}
// Warp-uniform bounded wait: lane 0 waits, the outcome is broadcast, and
// __syncwarp orders the other lanes after lane 0's acquire.  Keeps the
// warp converged for the .sync.aligned tcgen05 instructions that follow.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                          unsigned int *err) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait_fast(bar, parity, abort_flag, err) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  return ok != 0;
}
// Bounded wait that ignores the abort flag (draining copies in flight).
__device__ __forceinline__ void mbar_wait_quiet(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > 2000000000ull) return;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *tm, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
  // Keep consecutive MMAs of an unrolled group apart: without an instruction
  // between them, the last MMA of a short unrolled group (4 MMAs) was
  // measured to accumulate a wrong product on sm_103a.
  __syncwarp(1u);
}
__device__ __forceinline__ void tc_mma_bf16_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                               uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
  __syncwarp(1u);   // see tc_mma_bf16
}
#define PCV_TMEM_ST32(taddr, v)                                                                  \
  asm volatile(                                                                                  \
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13," \
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"            \
      ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), \
        "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]),         \
        "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]),       \
        "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),       \
        "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])                                            \
      : "memory")
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
#define PCV_TMEM_LD32(taddr, v)                                                                  \
  asm volatile(                                                                                  \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"  \
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"      \
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),    \
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), \
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),          \
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),          \
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])           \
      : "r"(taddr))
#define PCV_TMEM_LD16(taddr, v)                                                                  \
  asm volatile(                                                                                  \
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"  \
      "%14,%15}, [%16];"                                                                         \
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),    \
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), \
        "=r"(v[14]), "=r"(v[15])                                                                 \
      : "r"(taddr))
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// one TMEM load of 128 consecutive columns (a whole S row of the thread's lane)
#define PCV_TMEM_LD128(taddr, v)                                                     \
  asm volatile(                                                                      \
      "tcgen05.ld.sync.aligned.32x32b.x128.b32 {"                                    \
      "%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15," \
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31," \
      "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47," \
      "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63," \
      "%64,%65,%66,%67,%68,%69,%70,%71,%72,%73,%74,%75,%76,%77,%78,%79," \
      "%80,%81,%82,%83,%84,%85,%86,%87,%88,%89,%90,%91,%92,%93,%94,%95," \
      "%96,%97,%98,%99,%100,%101,%102,%103,%104,%105,%106,%107,%108,%109,%110,%111," \
      "%112,%113,%114,%115,%116,%117,%118,%119,%120,%121,%122,%123,%124,%125,%126,%127" \
      "}, [%128];"                                                                  \
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), \
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), \
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), \
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]), \
        "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]), "=r"(v[37]), "=r"(v[38]), "=r"(v[39]), \
        "=r"(v[40]), "=r"(v[41]), "=r"(v[42]), "=r"(v[43]), "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]), \
        "=r"(v[48]), "=r"(v[49]), "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]), "=r"(v[55]), \
        "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]), "=r"(v[61]), "=r"(v[62]), "=r"(v[63]), \
        "=r"(v[64]), "=r"(v[65]), "=r"(v[66]), "=r"(v[67]), "=r"(v[68]), "=r"(v[69]), "=r"(v[70]), "=r"(v[71]), \
        "=r"(v[72]), "=r"(v[73]), "=r"(v[74]), "=r"(v[75]), "=r"(v[76]), "=r"(v[77]), "=r"(v[78]), "=r"(v[79]), \
        "=r"(v[80]), "=r"(v[81]), "=r"(v[82]), "=r"(v[83]), "=r"(v[84]), "=r"(v[85]), "=r"(v[86]), "=r"(v[87]), \
        "=r"(v[88]), "=r"(v[89]), "=r"(v[90]), "=r"(v[91]), "=r"(v[92]), "=r"(v[93]), "=r"(v[94]), "=r"(v[95]), \
        "=r"(v[96]), "=r"(v[97]), "=r"(v[98]), "=r"(v[99]), "=r"(v[100]), "=r"(v[101]), "=r"(v[102]), "=r"(v[103]), \
        "=r"(v[104]), "=r"(v[105]), "=r"(v[106]), "=r"(v[107]), "=r"(v[108]), "=r"(v[109]), "=r"(v[110]), "=r"(v[111]), \
        "=r"(v[112]), "=r"(v[113]), "=r"(v[114]), "=r"(v[115]), "=r"(v[116]), "=r"(v[117]), "=r"(v[118]), "=r"(v[119]), \
        "=r"(v[120]), "=r"(v[121]), "=r"(v[122]), "=r"(v[123]), "=r"(v[124]), "=r"(v[125]), "=r"(v[126]), "=r"(v[127]) \
      : "r"(taddr))
#define PCV_TMEM_ST16(taddr, v)                                                                  \
  asm volatile(                                                                                  \
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13," \
      "%14,%15,%16};" ::"r"(taddr),                                                              \
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),    \
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]) \
      : "memory")
// The compiler does not know that a TMEM load writes its registers until the
// wait, nor that a TMEM store may read its sources until the wait: an empty
// asm that "modifies" the registers, placed right after the wait, keeps
// every use of loaded values after it and every source register alive (not
// reused for temporaries) up to it.
template <int Nr>
__device__ __forceinline__ void tmem_fence_regs(uint32_t (&v)[Nr]) {
#pragma unroll
  for (int k = 0; k < Nr; ++k) asm volatile("" : "+r"(v[k]));
}

// Shared-memory matrix descriptor (tcgen05): start >> 4 at bits 0-13, leading
// byte offset >> 4 at 16-29, stride byte offset >> 4 at 32-45, the fixed
// version 0b001 at 46-48, 128-byte swizzle (value 2) at 61-63.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), A K-major, B K-major or MN-major (bit 16),
// N >> 3 at 17-22, M >> 4 at 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool b_mn_major) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((b_mn_major ? 1u : 0u) << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t bf16x2_from(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
// hi + lo += v with the rounding error of the sum kept in lo (Knuth's
// TwoSum: exact for any magnitudes)
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float v) {
  const float s = hi + v;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (v - bp);
  hi = s;
}
__device__ __forceinline__ float tanh_f32(float x) {
  float r;
  asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// CTA owning flattened unit u when U units are split over n CTAs as
// [floor(b U / n), floor((b+1) U / n)).
__host__ __device__ inline int owner_cta(long long u, long long U, long long n) {
  return (int)(((u + 1) * n + U - 1) / U - 1);
}

// --------------------------------------------------------------------------
// KS (GEMM1 K steps of 16, = ceil(p / 16)) is a template parameter so that
// every MMA group is straight-line code: MMAs issued from a runtime-count
// loop between commits measured up to 3x slower on sm_103a.
template <int KS, bool ACC, bool GAUSS>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_grad_tc(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_hi,
              const __grid_constant__ CUtensorMap tm_lo, Problem pb, GradArgs a, TcArgs ta) {
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned base, by an offset into the shared array (so that the
  // compiler keeps shared-memory loads for y)
  uint8_t *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const int KA = ta.KP / 64;                       // 128-byte K atoms
  const uint32_t th_bytes = (uint32_t)KA * kTM * 128;
  const uint32_t x_bytes = (uint32_t)KA * kTN * 128;
  const int NS = ta.NS;
  uint8_t *th_hi = sm;
  uint8_t *th_lo = th_hi + th_bytes;
  uint8_t *xs = th_lo + (ta.need_lo ? th_bytes : 0);
  uint64_t *bars = reinterpret_cast<uint64_t *>(xs + (size_t)NS * x_bytes + 64);
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

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long U = (long long)ta.T * ta.J;
  const long long u0 = (long long)blockIdx.x * U / ta.n_cta;
  const long long u1 = (long long)(blockIdx.x + 1) * U / ta.n_cta;
  const int nunits = (int)(u1 - u0);

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) { mbar_init(smem_u32(&x_full[s]), 1); mbar_init(smem_u32(&x_empty[s]), 1); }
    for (int s = 0; s < 2; ++s) {
      mbar_init(smem_u32(&s_full[s]), 1); mbar_init(smem_u32(&s_empty[s]), 4);
      for (int qq = 0; qq < 2; ++qq) mbar_init(smem_u32(&r_part[4 * s + qq]), 4);
      mbar_init(smem_u32(&r_empty[s]), 1);
    }
    mbar_init(smem_u32(th_full), 1); mbar_init(smem_u32(th_empty), 1);
    mbar_init(smem_u32(g_full), 1); mbar_init(smem_u32(g_empty), 4);
    mbar_init(smem_u32(flush_bar), 8); mbar_init(smem_u32(decide_bar), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {   // TMEM: S[0] 0-127, S[1] 128-255, G 256-383, R[0] 384-447, R[1] 448-511
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_base_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_base_slot;

  const uint32_t tmem_G = tmem + 256;
  const uint32_t tmem_R = tmem + 384;              // R[b] at tmem_R + 64 b (bf16x2 per column)

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
      for (int i = 0; i < nunits; ++i) {
        const long long u = u0 + i;
        const int t = (int)(u / ta.J), j = (int)(u - (long long)t * ta.J);
        if (i == 0 || j == 0) {
          if (!mbar_wait_fast(smem_u32(th_empty), (seg & 1) ^ 1, abort_flag, ta.err)) break;
          mbar_expect_tx(smem_u32(th_full), th_bytes * (ta.need_lo ? 2 : 1));
          for (int kb = 0; kb < KA; ++kb) {
            tma_load_2d(smem_u32(th_hi + kb * kTM * 128), &tm_hi, kb * 64, t * kTM, smem_u32(th_full));
            if (ta.need_lo)
              tma_load_2d(smem_u32(th_lo + kb * kTM * 128), &tm_lo, kb * 64, t * kTM, smem_u32(th_full));
          }
          th_issued = seg;
          ++seg;
        }
        const int st = i % NS, rnd = i / NS;
        if (!mbar_wait_fast(smem_u32(&x_empty[st]), (rnd & 1) ^ 1, abort_flag, ta.err)) break;
        mbar_expect_tx(smem_u32(&x_full[st]), x_bytes);
        uint8_t *xb = xs + (size_t)st * x_bytes;
        for (int kb = 0; kb < KA; ++kb)
          tma_load_2d(smem_u32(xb + kb * kTN * 128), &tm_x, kb * 64, j * kTN, smem_u32(&x_full[st]));
        last_round[st] = rnd;
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
      const uint32_t id1 = idesc_bf16(kTM, kTN, false);
      const uint64_t hd0 = sdesc_sw128(smem_u32(th_hi), 16, 1024);
      const uint64_t ld0 = sdesc_sw128(smem_u32(th_lo), 16, 1024);
      const uint64_t xd_k = sdesc_sw128(smem_u32(xs), 16, 1024);   // K-major view, stage 0
      const uint64_t x_step = (uint64_t)(x_bytes >> 4);
      int j = (int)(u0 % ta.J);
      int seg1 = 0, st = 0, xph = 0;
      for (int i = 0; i < nunits; ++i) {
        const bool first = (i == 0 || j == 0);
        const bool last = (i == nunits - 1 || j == ta.J - 1);
        if (first && !mbar_wait_fast(smem_u32(th_full), seg1 & 1, abort_flag, ta.err)) break;
        if (!mbar_wait_fast(smem_u32(&x_full[st]), xph, abort_flag, ta.err)) break;
        const int sb = i & 1;
        if (!mbar_wait_fast(smem_u32(&s_empty[sb]), ((i >> 1) & 1) ^ 1, abort_flag, ta.err)) break;
        tc_fence_after();
        const uint64_t xd0 = xd_k + (uint64_t)st * x_step;
        const uint32_t dS = tmem + sb * 128;
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
          const uint64_t off = (uint64_t)((((ks >> 2) * kTM * 128) + (ks & 3) * 32) >> 4);
          const uint64_t offx = (uint64_t)((((ks >> 2) * kTN * 128) + (ks & 3) * 32) >> 4);
          tc_mma_bf16(dS, hd0 + off, xd0 + offx, id1, ks > 0 ? 1u : 0u);
        }
        if (ta.need_lo) {
#pragma unroll
          for (int ks = 0; ks < KS; ++ks) {
            const uint64_t off = (uint64_t)((((ks >> 2) * kTM * 128) + (ks & 3) * 32) >> 4);
            const uint64_t offx = (uint64_t)((((ks >> 2) * kTN * 128) + (ks & 3) * 32) >> 4);
            tc_mma_bf16(dS, ld0 + off, xd0 + offx, id1, 1u);
          }
        }
        tc_commit(smem_u32(&s_full[sb]));
        if (last) { tc_commit(smem_u32(th_empty)); ++seg1; }
        if (++j == ta.J) j = 0;
        if (++st == NS) { st = 0; xph ^= 1; }
      }
    }
  } else if (warp == 2) {
    // ------------------------------ GEMM2 issuer ---------------------------
    // Per unit i: G += R[i & 1] . X_chunk, four K steps (64 rows) per half
    // of R as the epilogue produces it.
    if (lane == 0) {
      const uint32_t id2 = idesc_bf16(kTM, ta.PN, true);
      const uint64_t xd_mn = sdesc_sw128(smem_u32(xs), kTN * 128, 1024);  // MN-major view, stage 0
      const uint64_t x_step = (uint64_t)(x_bytes >> 4);
      int j = (int)(u0 % ta.J);
      int seg2 = 0, st = 0;
      for (int i = 0; i < nunits; ++i) {
        const bool first = (i == 0 || j == 0);
        const bool last = (i == nunits - 1 || j == ta.J - 1);
        const int rb = i & 1;
        const uint32_t a0 = tmem_R + 64 * rb;       // K step ks: 8 columns (16 bf16) at a0 + 8 ks
        const uint64_t bd0 = xd_mn + (uint64_t)st * x_step;
        bool ok = true;
#pragma unroll
        for (int qq = 0; qq < 2 && ok; ++qq) {
          ok = mbar_wait_fast(smem_u32(&r_part[4 * rb + qq]), (i >> 1) & 1, abort_flag, ta.err);
          if (ok && qq == 0 && first) ok = mbar_wait_fast(smem_u32(g_empty), (seg2 & 1) ^ 1, abort_flag, ta.err);
          if (!ok) break;
          tc_fence_after();
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const int ks = 4 * qq + kk;
            tc_mma_bf16_ta(tmem_G, a0 + 8 * ks, bd0 + (uint64_t)((ks * 2048) >> 4), id2,
                           (first && ks == 0) ? 0u : 1u);
          }
        }
        if (!ok) break;
        tc_commit(smem_u32(&r_empty[rb]));
        tc_commit(smem_u32(&x_empty[st]));
        if (last) { tc_commit(smem_u32(g_full)); ++seg2; }
        if (++j == ta.J) j = 0;
        if (++st == NS) st = 0;
      }
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
    // walk the CTA's segments (maximal runs of units in one tile)
    int t = (int)(u0 / ta.J), j0 = (int)(u0 - (long long)t * ta.J);
    for (int ib = 0; ib < nunits && !aborted; ) {
      const int ie = min(nunits, ib + (ta.J - j0));   // segment [ib, ie)
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
        // residual of quarter qq (32 rows) of the chunk from v = S into pk
        // (16 bf16x2), plus the log-likelihood sums when ACC
        auto quarter = [&](const int qq, const uint32_t (&v)[32], uint32_t (&pk)[16]) {
          const int n0 = j * kTN + 32 * qq;
          if constexpr (!GAUSS) {
            // 1 - tanh(S) in FP32 (twice the residual along the sign-folded
            // row), rounded to bf16 for the second GEMM.  A bf16x2 tanh here
            // would bias the gradient: its error is a smooth function of eta,
            // so it adds up over rows instead of averaging out (a force error
            // of ~6 % of the posterior scale per dimension at N = 1e5, which
            // shrinks the adapted step size).
#pragma unroll
            for (int k = 0; k < 16; ++k)
              pk[k] = bf16x2_from(1.0f - tanh_f32(__uint_as_float(v[2 * k])),
                                  1.0f - tanh_f32(__uint_as_float(v[2 * k + 1])));
            if (valid && n0 < fd.excl_hi && n0 + 32 > fd.excl_lo) {
#pragma unroll
              for (int k = 0; k < 32; ++k) {
                const int n = n0 + k;
                if (n >= fd.excl_lo && n < fd.excl_hi) pk[k >> 1] &= (k & 1) ? 0x0000FFFFu : 0xFFFF0000u;
              }
            }
            if constexpr (accurate) {
              // log likelihood y eta - softplus(eta) = -softplus(-2 S) with
              // the sign-folded S: softplus(-2 S) = max(-2 S, 0) +
              // log(1 + exp(-|2 S|)) is summed here, in FP32 per quarter and
              // FP64 across quarters.
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
            // Gaussian: residual (y - eta) / sigma^2 = -2 S / sigma^2, rounded
            // to bf16; the squared residuals of the fold's training and test
            // rows feed the log sigma gradient and the log densities
            float e[32];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              e[2 * k] = -2.0f * __uint_as_float(v[2 * k]);
              e[2 * k + 1] = -2.0f * __uint_as_float(v[2 * k + 1]);
              pk[k] = bf16x2_from(e[2 * k] * inv_s2, e[2 * k + 1] * inv_s2);
            }
            if (valid && n0 < fd.excl_hi && n0 + 32 > fd.excl_lo) {
#pragma unroll
              for (int k = 0; k < 32; ++k) {
                const int n = n0 + k;
                if (n >= fd.excl_lo && n < fd.excl_hi) pk[k >> 1] &= (k & 1) ? 0x0000FFFFu : 0xFFFF0000u;
              }
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
        // The whole S tile row (128 columns) comes into registers at once and
        // S is released before any arithmetic, so the first GEMM of unit
        // i + 2 waits only for the TMEM loads of unit i.  The four R quarters
        // go out as 16-column stores; each store's wait comes after the
        // next quarter's arithmetic (TMEM round trips are several hundred
        // cycles while the MMAs run), and each completed quarter is handed
        // to the second GEMM at once.  Loaded registers are used only after
        // the load wait, and store sources stay allocated until their store
        // wait (tmem_fence_regs pins both).
        if constexpr (ACC) {
          // log-density launch (one of L_f per iteration): a rolled loop
          // over the quarters, each loaded from TMEM on its own, keeps this
          // instantiation's code small (the unrolled form below, with the
          // softplus sums, overflowed the instruction cache); S is released
          // after the last quarter's load
          const uint32_t rbuf = tmem_R + 64 * rb + lane_off;
#pragma unroll 1
          for (int qq = 0; qq < 4; ++qq) {
            uint32_t v[32], pk[16];
            PCV_TMEM_LD32(tmem + sb * 128 + lane_off + 32 * qq, v);
            tmem_wait_ld();
            tmem_fence_regs(v);
            if (qq == 3) {
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(smem_u32(&s_empty[sb]));
            }
            quarter(qq, v, pk);
            if (qq == 0) {
              if (!warp_wait(smem_u32(&r_empty[rb]), ((i >> 1) & 1) ^ 1, abort_flag, ta.err)) {
                aborted = true;
                break;
              }
              tc_fence_after();
            }
            PCV_TMEM_ST16(rbuf + 16 * qq, pk);
            tmem_wait_st();
            tmem_fence_regs(pk);
            if (qq & 1) {                                   // a 64-row half of R is in TMEM
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(smem_u32(&r_part[4 * rb + (qq >> 1)]));
            }
          }
          if (aborted) break;
          continue;
        }
        uint32_t sv[128], p0[16], p1[16], p2[16], p3[16];
        PCV_TMEM_LD128(tmem + sb * 128 + lane_off, sv);   // one load: ~2 % faster than four x32
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
        quarter(0, v0, p0);
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
        quarter(1, v1, p1);
        PCV_TMEM_ST16(rbuf + 16, p1);
        quarter(2, v2, p2);
        quarter_stored(0);
        tmem_fence_regs(p0);
        tmem_fence_regs(p1);
        PCV_TMEM_ST16(rbuf + 32, p2);
        quarter(3, v3, p3);
        PCV_TMEM_ST16(rbuf + 48, p3);
        quarter_stored(1);
        tmem_fence_regs(p2);
        tmem_fence_regs(p3);
      }
      if (aborted) break;
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
        __threadfence();
        const unsigned prev = atomicAdd(ta.tickets + t, 1u);
        *last_flag = (prev == (unsigned)nseg - 1);
        if (prev == (unsigned)nseg - 1) ta.tickets[t] = 0u;
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
                mv[u] = *reinterpret_cast<const float4 *>(a.minv + jj_[u]);
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
            // shadows hold (theta - ref) / 2 as bf16 hi + lo
            const float h0 = 0.5f * (tn.x - rf[u].x), h1 = 0.5f * (tn.y - rf[u].y);
            const float h2 = 0.5f * (tn.z - rf[u].z), h3 = 0.5f * (tn.w - rf[u].w);
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
              const float tn = tv + eps * a.minv[jj] * rj;
              th[jj] = tn;
              const float half = 0.5f * (tn - ta.theta_ref[jj]);   // shadows hold (theta - ref) / 2
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
              if (kd) th[pb.p] = ls + eps * a.minv[pb.p] * rj;
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
      // next segment starts at chunk 0 of the next tile
      ib = ie;
      ++t;
      j0 = 0;
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
size_t tc_smem_bytes(int KP, int NS, int need_lo, int p) {
  (void)p;
  const size_t KA = KP / 64;
  size_t b = KA * kTM * 128 * (need_lo ? 2 : 1) + (size_t)NS * KA * kTN * 128 +
             64 + (2 * kTcMaxStages + 23) * 8;   // barrier / flag slots
  return b + 1024;   // alignment slack
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

template <int KS>
static cudaError_t set_smem_attr() {
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t r[4] = {cudaFuncSetAttribute(k_grad_tc<KS, false, false>, at, 227 * 1024),
                      cudaFuncSetAttribute(k_grad_tc<KS, true, false>, at, 227 * 1024),
                      cudaFuncSetAttribute(k_grad_tc<KS, false, true>, at, 227 * 1024),
                      cudaFuncSetAttribute(k_grad_tc<KS, true, true>, at, 227 * 1024)};
  for (cudaError_t x : r)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}

// setmaxnreg.inc waits until the CTA's register pool can grant the request:
// the pool is what the CTA was launched with (threads x the compiled register
// count), so a split larger than that would never be granted.  Every
// instantiation is checked once; launches are refused if any fails.
static bool g_tc_regs_ok = false;
template <int KS>
static bool regs_fit() {
  const long need = 128L * kTcRegsProducer + 256L * kTcRegsEpilogue;
  cudaFuncAttributes fa[4];
  if (cudaFuncGetAttributes(&fa[0], k_grad_tc<KS, false, false>) != cudaSuccess ||
      cudaFuncGetAttributes(&fa[1], k_grad_tc<KS, true, false>) != cudaSuccess ||
      cudaFuncGetAttributes(&fa[2], k_grad_tc<KS, false, true>) != cudaSuccess ||
      cudaFuncGetAttributes(&fa[3], k_grad_tc<KS, true, true>) != cudaSuccess)
    return false;
  for (const cudaFuncAttributes &f : fa)
    if ((long)f.numRegs * kTcThreads < need) return false;
  return true;
}

// once per context (outside any stream capture): allow the large dynamic SMEM
cudaError_t tc_prepare() {
  cudaError_t e = cudaSuccess;
  cudaError_t r[9] = {set_smem_attr<1>(), set_smem_attr<2>(), set_smem_attr<3>(), set_smem_attr<4>(), set_smem_attr<5>(),
                      set_smem_attr<6>(), set_smem_attr<7>(), set_smem_attr<8>(), set_smem_attr<9>()};
  for (cudaError_t x : r)
    if (x != cudaSuccess) e = x;
  g_tc_regs_ok = regs_fit<1>() && regs_fit<2>() && regs_fit<3>() && regs_fit<4>() && regs_fit<5>() &&
                 regs_fit<6>() && regs_fit<7>() && regs_fit<8>() && regs_fit<9>();
  if (e == cudaSuccess && !g_tc_regs_ok) e = cudaErrorInvalidConfiguration;
  return e;
}

cudaError_t launch_grad_tc(const CUtensorMap &tm_x, const CUtensorMap &tm_hi, const CUtensorMap &tm_lo,
                           const Problem &pb, const GradArgs &a, const TcArgs &ta, cudaStream_t st) {
  const size_t smem = tc_smem_bytes(ta.KP, ta.NS, ta.need_lo, pb.p);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  if (!g_tc_regs_ok) return cudaErrorInvalidConfiguration;   // tc_prepare not run, or the split does not fit
  if (pb.variant == MV_HIER) return cudaErrorInvalidValue;
  const bool gauss = pb.variant == MV_GAUSS_KNOWN || pb.variant == MV_GAUSS_LOGSIG;
  switch (ta.KS) {
#define PCV_TC_CASE(K)                                                                          \
  case K:                                                                                       \
    if (gauss) {                                                                                \
      if (ta.accurate) k_grad_tc<K, true, true><<<ta.n_cta, kTcThreads, smem, st>>>(tm_x, tm_hi, tm_lo, pb, a, ta); \
      else k_grad_tc<K, false, true><<<ta.n_cta, kTcThreads, smem, st>>>(tm_x, tm_hi, tm_lo, pb, a, ta);           \
    } else {                                                                                    \
      if (ta.accurate) k_grad_tc<K, true, false><<<ta.n_cta, kTcThreads, smem, st>>>(tm_x, tm_hi, tm_lo, pb, a, ta); \
      else k_grad_tc<K, false, false><<<ta.n_cta, kTcThreads, smem, st>>>(tm_x, tm_hi, tm_lo, pb, a, ta);           \
    }                                                                                           \
    break;
    PCV_TC_CASE(1) PCV_TC_CASE(2) PCV_TC_CASE(3) PCV_TC_CASE(4)
    PCV_TC_CASE(5) PCV_TC_CASE(6) PCV_TC_CASE(7) PCV_TC_CASE(8) PCV_TC_CASE(9)
#undef PCV_TC_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace pcv
