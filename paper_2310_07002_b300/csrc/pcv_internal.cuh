// pcv_internal.cuh -- device-side data layout and helpers shared by the PCV
// kernels (sm_103a).  Product code: nothing here is shared with the oracle.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace pcv {

// model variants the kernels are specialised on
enum ModelVariant : int {
  MV_GAUSS_KNOWN = 0,   // Gaussian, sigma known
  MV_GAUSS_LOGSIG = 1,  // Gaussian (linear or AR design), log sigma sampled
  MV_LOGISTIC = 2,
  MV_HIER = 3           // varying intercept tau*z_g, log tau, log sigma
};

// Philox stream tags (the counter's last word)
enum Stream : uint32_t {
  ST_MOM = 0, ST_ACC = 1, ST_INIT = 2, ST_JIT = 3, ST_SHUF = 4, ST_PRED = 5, ST_FD_MOM = 16, ST_FD_ACC = 17, ST_FD_INIT = 18
};

// Row ranges of one fold in the library's sorted row order (the Appendix B
// masks restated as ranges): test rows [test_lo, test_hi); training rows are
// the rows outside [excl_lo, excl_hi) (the test block widened by the h(v)-block
// buffer).  The full-data pseudo-fold (id K) has empty ranges.
struct FoldDesc {
  int test_lo, test_hi, excl_lo, excl_hi;
};

// Device view of the data (rows sorted so that test blocks and groups are
// contiguous).
struct Problem {
  int variant;            // ModelVariant
  int N;                  // rows
  int p;                  // regressors
  int p_pad;              // row stride of X (multiple of 4)
  int d;                  // dimension of theta
  int d_pad;              // row stride of chain vectors (multiple of 4)
  int G;                  // groups (HIER)
  int K;                  // folds; fold id K is the full data set
  const float *X;         // N x p_pad, zero padded columns
  const float *y;         // N
  const int *grp_off;     // G + 1 row offsets of the group segments (HIER)
  const int *seg_grp;     // G: group id of each segment (HIER)
  const int *grp_seg;     // G: segment of each group (HIER)
  const FoldDesc *folds;  // K + 1
  float beta_prec;        // 1 / beta_prior_sd^2
  float log_beta_sd;
  float sigma_known;      // GAUSS_KNOWN
  float sigma_prec;       // 1 / sigma_prior_sd^2
  float log_sigma_sd;
  float tau_prec;         // 1 / tau_prior_sd^2
  float log_tau_sd;
};

enum { MODE_NONE = 0, MODE_KICK_DRIFT = 1, MODE_LAST_KICK = 2 };

// Arguments of one gradient evaluation (optionally fused with a leapfrog
// update) for a batch of chain positions.
// Two models in one context (covariate masks M_A, M_B; Appendix B): chains
// [0, K L) are model A's, [K L, 2 K L) model B's, and each model has its own
// row of the inverse mass (B's is A's with B's inactive coefficients at 0).
__host__ __device__ inline const float *minv_row(const float *minv, int c, int every, int ld) {
  return every > 0 ? minv + (size_t)(c / every) * ld : minv;
}

struct GradArgs {
  int C;                  // positions
  int L;                  // chains per fold (fold = fold_base + c / L) if fold_of == nullptr
  int fold_base;
  const int *fold_of;     // optional explicit fold per position
  const float *theta;     // C x ld_theta (read; updated in place by MODE_KICK_DRIFT)
  int ld_theta;
  float *grad;            // C x ld_grad (out)
  int ld_grad;
  double *logp;           // C (out) when need_ll
  double *shat;           // C (out) when need_ll
  int need_ll;
  int mode;               // MODE_NONE, MODE_KICK_DRIFT, MODE_LAST_KICK
  float *r;               // C x ld_theta momenta (updated by the modes)
  const float *eps;       // device scalar step size
  const float *minv;      // inverse mass diagonal (d_pad), one row per model
  int minv_every, minv_ld;   // chains per row and row stride (minv_every 0: one row)
  // split-N cross-CTA combine
  int splits;             // row splits per chain tile
  float *ws;              // workspace: tiles x splits x 32 x ws_stride floats
  int ws_stride;
  unsigned int *tickets;  // one per chain tile, zero between launches
  // bf16 hi/lo shadow of theta for the tensor-core path (written by updates)
  __nv_bfloat16 *shadow_hi, *shadow_lo;
  int ld_shadow;
};

// Per-chain online accumulator state, structure of arrays, FP64.
struct Accum {
  int C;
  int M;                  // autocovariance lag cap (0 = off)
  int max_batches;
  int b;                  // batch size
  double *Ux, *Ux2, *Zx;  // sums of exp(s - em), exp(2 (s - em)), and exp(s - em) in the current batch
  double *em, *emean, *eM2;   // log-shifted Welford of exp(s) over draws (em: the running max of s)
  double *vm, *vmean, *vM2;   // log-shifted Welford of batch means
  double *wmean, *wM2;        // Welford of s over draws
  double *bmean_cur, *bM2_cur;// Welford of s in the current batch
  double *bmean, *bM2;        // per closed batch [max_batches x C]
  double *c0, *xsum;          // acov centring constant (first draw), sum of x
  double *lagsum;             // [C x (M+1)]
  double *first;              // [C x M]
  double *ring;               // [C x M]
  long long *div, *acc;       // divergences, accepts (sampling only)
  double *draws;              // optional stored draws [C x draw_cap]
  int draw_cap;
};

// Iteration counters and adaptation state kept in device memory so that
// CUDA graph replays need no parameter updates.
struct IterState {
  unsigned int iter;        // fold-chain Philox iteration counter
  unsigned int fd_iter;     // full-data iteration counter
  long long n_draws;        // draws accumulated so far
  unsigned int ticket;      // last-block election in the accept kernel
  unsigned int error;       // device error flags
  float eps;                // nominal step size (adapted in the full-data warm-up)
  float eps_iter;           // this iteration's step size (eps, jittered for fold chains)
  double da_mu, da_hbar, da_logeps, da_logeps_bar;
  long long da_t;
  double mass_n;            // Welford count of the mass window
};

// Philox4x32-10 (Salmon et al., SC 2011): 10 rounds of the 4x32 bijection,
// key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    if (i) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
    const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
    uint32_t hi0 = __umulhi(m0, c.x), lo0 = m0 * c.x;
    uint32_t hi1 = __umulhi(m1, c.z), lo1 = m1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ uint4 philox_at(unsigned long long seed, uint32_t block, uint32_t chain,
                                           uint32_t iter, uint32_t stream) {
  return philox4x32_10(make_uint4(block, chain, iter, stream),
                       make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

__device__ __forceinline__ double unit_from_word(uint32_t a) {
  return ((double)a + 0.5) * 2.3283064365386963e-10;
}

// Box-Muller on two words: (sqrt(-2 ln u1) cos 2 pi u2, sqrt(-2 ln u1) sin 2 pi u2),
// u = (w + 1/2) 2^-32 in (0, 1).  FP32 throughout (FP64 is slow on this
// part), with the complements taken from the integer words so that they
// keep their relative precision: ln u1 = log1p(-(1 - u1)) when u1 >= 1/2,
// else log(u1); the angle 2 pi u2 as 2 pi (u2 - 1) when u2 >= 1/2 (the same
// point of the circle).  The result is within ~1e-7 relative of the FP64
// transform.
__device__ __forceinline__ float2 box_muller(uint32_t a, uint32_t b) {
  const float k = 2.3283064365386963e-10f;            // 2^-32
  const float l = a >= 0x80000000u ? log1pf(-(((float)(0xFFFFFFFFu - a) + 0.5f) * k))
                                   : logf(((float)a + 0.5f) * k);
  const float t = b >= 0x80000000u ? -2.0f * (((float)(0xFFFFFFFFu - b) + 0.5f) * k)
                                   : 2.0f * (((float)b + 0.5f) * k);
  const float rad = sqrtf(-2.0f * l);
  float s, c;
  sincospif(t, &s, &c);
  return make_float2(rad * c, rad * s);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// A sum of FP32 products carried as an unevaluated pair hi + lo of floats
// with error-free transformations: Knuth's TwoSum for each addition and the
// FMA TwoProduct for each product (the Dot2 scheme of Ogita, Rump and Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 2005).  The pair holds
// the sum to about twice FP32's precision (~2^-48 relative for the positive
// kinetic-energy terms) without FP64 arithmetic, whose pipe on this part
// takes ~32 cycles of an SM per warp instruction; it becomes one double at
// the end (hi + lo).
struct F2 {
  float hi, lo;
};
// (the _rn intrinsics keep the compiler from contracting a product and a
// sum into one FMA, which would break the exact error terms)
__device__ __forceinline__ void f2_add(F2 &s, float x) {
  const float t = __fadd_rn(s.hi, x);
  const float z = __fsub_rn(t, s.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, z)), __fsub_rn(x, z)));
  s.hi = t;
}
// s += m r^2: m r = p1 + p2 exactly, p1 r = q1 + q2 exactly, p2 r rounded
__device__ __forceinline__ void f2_add_mr2(F2 &s, float m, float r) {
  const float p1 = __fmul_rn(m, r), p2 = __fmaf_rn(m, r, -p1);
  const float q1 = __fmul_rn(p1, r), q2 = __fmaf_rn(p1, r, -q1);
  f2_add(s, q1);
  s.lo = __fadd_rn(s.lo, __fmaf_rn(p2, r, q2));
}
// the pair summed over the lanes of an aligned group of gsz lanes (xor tree)
__device__ __forceinline__ double f2_group_sum(F2 s, int gsz) {
  for (int o = gsz >> 1; o > 0; o >>= 1) {
    const float h = __shfl_xor_sync(0xffffffffu, s.hi, o), l = __shfl_xor_sync(0xffffffffu, s.lo, o);
    f2_add(s, h);
    s.lo = __fadd_rn(s.lo, l);
  }
  return (double)s.hi + (double)s.lo;
}

__device__ __forceinline__ int fold_of_chain(const GradArgs &a, int c) {
  return a.fold_of ? a.fold_of[c] : a.fold_base + c / a.L;
}

// log(1 + e^x) without overflow
__device__ __forceinline__ float softplusf(float x) {
  return fmaxf(x, 0.0f) + log1pf(__expf(-fabsf(x)));
}

constexpr float kLog2Pi = 1.8378770664093453f;
constexpr double kLog2PiD = 1.8378770664093454835606594728112;
constexpr double kLog2D = 0.69314718055994530942;

// The hierarchical model's held-out group (leave-one-group-out):
// log N(e | 0, s^2 I + t^2 1 1') of a group of m rows with residuals e
// (intercept integrated out), from S1 = sum e and S2 = sum e^2:
//   det = s^(2(m-1)) (s^2 + m t^2),
//   e' inv e = (S2 - t^2 S1^2 / (s^2 + m t^2)) / s^2
__device__ __forceinline__ double new_group_log_pred(float S1, float S2, int m, float logsig, float logtau) {
  const double s2 = exp(2.0 * (double)logsig), t2 = exp(2.0 * (double)logtau);
  const double den = s2 + (double)m * t2;
  const double q = ((double)S2 - t2 * (double)S1 * (double)S1 / den) / s2;
  return -0.5 * (double)m * kLog2PiD - 0.5 * ((double)(m - 1) * log(s2) + log(den)) - 0.5 * q;
}

// tensor-core path (k_grad_tc.cu)
// workspace rows per tile segment beyond the PN gradient rows: per
// warpgroup the training and test softplus sums, each as an FP32 hi + lo pair
constexpr int kTcSlots = 8;
// Tensor-core operand columns p .. p + kEtaCols - 1: X holds eta_ref / 2 of
// its row split into kEtaCols bf16 parts (hi, mid, lo), the theta shadows hold
// 1 (hi) and 0 (lo) there, so the first GEMM yields eta / 2 itself.
constexpr int kEtaCols = 3;

struct TcArgs {
  int KP;                 // padded K in SMEM / global (a multiple of 64, >= 16 KS)
  int KS;                 // GEMM1 K steps of 16 (ceil((p + kEtaCols) / 16)): the p
                          // covariates and the eta_ref / 2 columns
  int PN;                 // GEMM2 N (16 * ceil(p / 16))
  int N_pad;              // rows padded to a multiple of the 128-row chunk
  int J;                  // chunks per tile
  int T;                  // chain tiles of 128
  int n_cta;              // grid size
  int max_seg;            // workspace segments per tile
  int NS;                 // X pipeline stages
  int NT;                 // X^T pipeline stages (TF32 form)
  int need_lo;            // accumulate the theta lo part too (FP32-accurate eta)
  int accurate;           // FP32 epilogue with log densities (else the bf16x2 fast path)
  const float *theta_ref; // d: the shadows hold (theta - theta_ref) / 2
  float *ws;              // T x max_seg x (PN + kTcSlots) x 128
  unsigned int *tickets;  // T
  unsigned int *err;      // error flags (bit 0: wait time-out)
  int tf32;               // TF32 operands (kind::tf32, 64-row chunks, X^T for the second GEMM)
  float *shadow32;        // TF32 path: (theta - theta_ref) / 2 rounded to TF32 [C_pad x KP]
  int steps;              // kick-drift steps in this launch (> 1: one CTA per tile)
};

// launchers (k_grad_simt.cu)
int simt_flat_pp(int p);
size_t bigp_smem_bytes(int pp);
int simt_chain_tile(int p);   // chains per CTA tile of the FP32 gradient kernels
size_t hier_smem_bytes(int PP, int G, int splits);
cudaError_t launch_grad_simt(const Problem &pb, const GradArgs &a, cudaStream_t st);

// ---------------------------------------------------------------------------
// per-chain HMC kernels (k_hmc.cu)
// ---------------------------------------------------------------------------
struct BeginArgs {
  int C, d, ld;
  unsigned long long seed;
  unsigned int stream;
  const unsigned int *iter;     // device iteration counter
  const float *theta, *grad;    // current state
  const double *logp;
  float *theta_p, *r;           // proposal position and momentum (out)
  double *H0;                   // out
  const float *eps, *minv;      // nominal step size, inverse mass (one row per model)
  int minv_every, minv_ld;      // chains per inverse-mass row, row stride (0: one row)
  float jitter;                 // eps_iter = eps (1 + jitter (2u - 1)), u from stream ST_JIT
  int chain_base;               // Philox chain id = chain_base + c (global fold-chain id)
  float *eps_iter;              // out (written by block 0): the step size of this iteration
  const float *r_given;         // optional start momenta instead of drawing (C x ld)
  __nv_bfloat16 *shadow_hi, *shadow_lo;
  float *shadow32;              // TF32 form: (theta_p - theta_ref) / 2 rounded to TF32
  int ld_shadow;
  int shadow_d;                 // leading coordinates with a shadow (beta: p)
  const float *theta_ref;       // shadows hold (theta_p - theta_ref) / 2
};

// A whole leapfrog trajectory per chain in one launch (k_traj_small.cu):
// the momentum draw and first half step of k_begin, then L_f gradient
// evaluations with their kicks and drifts, writing the same proposal state
// as k_begin + L_f gradient launches.
struct TrajArgs {
  int C, L, fold_base, ld;
  unsigned long long seed;
  unsigned int stream;
  int chain_base;
  const unsigned int *iter;     // device iteration counter
  const float *eps;             // nominal step size
  float *eps_iter;              // out (chain 0): this iteration's step size
  float jitter;
  const float *minv;
  int minv_every, minv_ld;      // chains per inverse-mass row, row stride (0: one row)
  const float *theta, *grad;    // current state
  const double *logp;
  const float *r_given;         // optional start momenta (C x ld)
  float *theta_p, *r, *grad_p;  // proposal (out)
  double *logp_p, *shat_p, *H0; // out
  int Lf;
  const __nv_bfloat16 *X16;     // BF16 form: N x PP copy of X, zero-padded to a multiple of
                                // 16 bytes (else nullptr: FP32 X)
  int eval_only;                // 1: gradient and log densities at theta only, into
                                // grad_p, logp_p, shat_p (no momentum, no update)
  int smem_rows;                // set by the launcher: X (or X16) and y staged in shared memory
  int part_offset;              // set by the launcher: byte offset of the team partial sums
  int wpc;                      // warps per chain (1, 2, 4, 8): a chain's rows are split over them
  // accept mode: the Metropolis test and the draw's accumulators follow in
  // the same launch (as k_accept), the proposal stays in registers
  int accept;
  unsigned int acc_stream;      // Philox stream of the accept uniforms
  IterState *st;
  int fd;                       // full-data chains (fd_iter counter, no accumulators)
  int accumulate;
  Accum acc;
  double *accept_prob;          // per chain, or null
  float *theta_w, *grad_w;      // the chains' state, updated on acceptance
  double *logp_w, *shat_w;
};
int traj_default_wpc(int C);
int traj_max_wpc(const Problem &pb);
bool traj_small_supported(const Problem &pb);
int traj_small_row_width(int p);
cudaError_t launch_traj_small(const Problem &pb, const TrajArgs &t, cudaStream_t st);
__global__ void k_x_bf16_compact(long long N, int PP, int p_pad, const float *X, __nv_bfloat16 *X16);

struct AcceptArgs {
  int C, d, ld;
  int chain_base;               // Philox chain id = chain_base + c
  unsigned long long seed;
  unsigned int stream;
  IterState *st;
  int fd;                          // 1: full-data chains (fd_iter counter)
  float *theta, *grad;
  double *logp, *shat;
  const float *theta_p, *r, *grad_p;
  const double *logp_p, *shat_p, *H0;
  const float *minv;
  int minv_every, minv_ld;         // chains per inverse-mass row, row stride (0: one row)
  int accumulate;                  // 1: sampling phase
  Accum acc;
  double *accept_prob;             // per chain, or null
};

struct FdAdaptArgs {
  IterState *st;
  int n_adapt, w0, w1, w2;     // mass windows [w0, w1) and [w1, w2)
  float eps_cap;              // final step size cap (trajectory length / L_f); <= 0: none
  const float *active;        // d: 1 / 0 covariate-selection mask (nullptr: all active)
  int adapt_eps, adapt_mass;
  int C, d, ld;
  const float *theta;
  const double *accept_prob;
  float *minv;
  double *wmean, *wM2;        // d each
  float *pool;                // n_keep*C x ld
  int n_keep;
};

enum { F_ELPD, F_MCSE, F_SIG2BM, F_S2, F_ESSBM, F_RHAT, F_SRHAT, F_ESSAC, F_DIV, F_ACTRUNC,
       F_ACCRATE, F_NFIELDS };
enum { T_ELPD, T_MCSE, T_SEEPI, T_RHATMAX, T_ESSTOT, T_SRHATMAX, T_DIV, T_NFIELDS };

__global__ void k_begin(BeginArgs a);
__global__ void k_normals(int C, int d, int ld, unsigned long long seed, unsigned int iter,
                          unsigned int stream, float scale, float *out);
__global__ void k_init_from_pool(int C, int d, int ld, unsigned long long seed, const float *pool,
                                 int n_pool, float *theta, int chain_base);
__global__ void k_shadow(int C, int d, int ld, const float *theta, const float *theta_ref,
                         __nv_bfloat16 *hi, __nv_bfloat16 *lo, int ld_shadow);
// Hyvarinen / Dawid-Sebastiani accumulators (Algorithms A3, A4): per chain
// sums over draws of xi1 = sum_i [d2 + d1^2], of d1_i, of a predictive draw
// ytil_i and of ytil ytil' (T = the largest test set)
struct Extra {
  int flags, T;
  double *hs1, *hs2, *dsum, *douter;   // C, C x T, C x T, C x T x T
};
__global__ void k_extra_push(Problem pb, GradArgs a, Extra E, const unsigned int *iter,
                             unsigned long long seed, int chain_base);
__global__ void k_extra_finalize(Problem pb, Extra E, int K, int L, double n, double *hs, double *dss);
__global__ void k_block_stats(Accum A, int a, int D, double *blk);
__global__ void k_mask_positions(int C, int d, int ld, const float *active, float *theta);
__global__ void k_compare(const double *fo_a, const double *fo_b, int K, double *out);
__global__ void k_rhat_shuffle(const double *blk, int K, int L, int D, int R, unsigned long long seed,
                               unsigned long long *out_max, double *out_all, int first_fold);
__global__ void k_theta_ref(int n, int d, int ld, const float *src, float *theta_ref);
__global__ void k_eta_ref(int N, int N_pad, int p, int KP, const __nv_bfloat16 *X16, const float *theta_ref,
                          float *eta_half);
__global__ void k_eta_fold(int N_pad, int p, int KP, const float *eta_half, const float *y,
                           __nv_bfloat16 *X16);
__global__ void k_gather_rows(long long N, int p, int p_pad, const int *perm, const float *xraw, float *X);
__global__ void k_x_bf16(long long N, int p, int p_pad, int KP, const float *X, const float *ysign,
                         __nv_bfloat16 *X16);
__global__ void k_shadow_ones(int C_pad, int p, int KP, __nv_bfloat16 *hi);
__global__ void k_x_tf32(long long N, int p, int p_pad, int KP, int N_pad, const float *X, const float *ysign,
                         float *X32, float *XT32);
__global__ void k_eta_ref32(int N, int N_pad, int p, int KP, const float *X32, const float *theta_ref,
                            float *eta_half);
__global__ void k_eta_fold32(int N_pad, int p, int KP, const float *eta_half, const float *y, float *X32);
__global__ void k_shadow32(int C, int d, int ld, const float *theta, const float *theta_ref, float *s32, int ld_s);
__global__ void k_shadow_ones32(int C_pad, int p, int KP, float *hi);
// k_begin: a chain takes this many lanes (the power of two that covers its
// ceil(d/4) coordinate quads, at most 32), so small models pack 32 / that
// many chains per warp; 8 warps per block
__host__ __device__ inline int begin_lanes_per_chain(int d) {
  const int nq = (d + 3) / 4;
  int g = 1;
  while (g < nq && g < 32) g <<= 1;
  return g;
}
inline int begin_blocks(int C, int d) {
  const int per_block = 8 * (32 / begin_lanes_per_chain(d));
  return (C + per_block - 1) / per_block;
}
constexpr int kAccChains = 32;   // chains per block of the accept / accumulate kernels
constexpr int kAccWarps = 8;     // warps per block of the accept kernel (each takes 4 chains' vector work)
__global__ void k_accept(AcceptArgs a);
__global__ void k_accumulate_given(Accum A, const double *s, int n, long long n0);
__global__ void k_fd_adapt(FdAdaptArgs a);
__global__ void k_fd_init_state(IterState *st, float eps0, int adapt);
__global__ void k_fd_final_eps(IterState *st, float eps_cap);
__global__ void k_copy_eps(IterState *st);
__global__ void k_finalize(Accum A, int K, int L, long long n, double *out, double *scratch);
__global__ void k_totals(const double *fo, int K, double Ln, double *tot);

}  // namespace pcv
