// pcv_api.cu -- host side of the PCV C ABI (include/pcv.h): validation, the
// sorted row layout and fold ranges, device buffers, and the orchestration
// of warm-up reuse (Section 3.1) and lock-step sampling (Section 3.3,
// Algorithm A2).  Each HMC iteration is one momentum kernel, L_f fused
// gradient+update kernels and one accept/accumulate kernel; iterations are
// captured once as CUDA graphs and replayed, with all counters in device
// memory.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "../../include/pcv.h"
#include "pcv_internal.cuh"

namespace pcv {
size_t tc_smem_bytes(int KP, int NS, int NT, int need_lo, int p, int tf32, int PN);
int tc_max_stages();
int tc_segments_per_tile(int T, int J, int n_cta);
cudaError_t tc_prepare();
cudaError_t launch_grad_tc(const CUtensorMap &tm_x, const CUtensorMap &tm_hi, const CUtensorMap &tm_lo,
                           const Problem &pb, const GradArgs &a, const TcArgs &ta, cudaStream_t st);
}  // namespace pcv


using namespace pcv;

namespace {

constexpr int kNumFdChains = 4;
constexpr int kTargetCtas = 148 * 4;

struct ChainBufs {
  int C = 0, L = 1, fold_base = 0;
  float *theta = nullptr, *grad = nullptr, *theta_p = nullptr, *r = nullptr, *grad_p = nullptr;
  double *logp = nullptr, *shat = nullptr, *logp_p = nullptr, *shat_p = nullptr, *H0 = nullptr;
  double *accept_prob = nullptr;
  // tensor-core path: bf16 hi / lo of theta / 2 [C_pad x KP] and their TMA maps
  int C_pad = 0;
  __nv_bfloat16 *shadow_hi = nullptr, *shadow_lo = nullptr;
  CUtensorMap tm_hi{}, tm_lo{};
  float *shadow32 = nullptr;        // TF32 form: one FP32 shadow (TF32 values), map in tm_hi
};

enum CtxState { ST_CREATED = 0, ST_WARMED = 1, ST_SAMPLED = 2 };

}  // namespace

struct pcv_ctx {
  std::string err;
  pcv_options opt;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev0 = nullptr, ev1 = nullptr;
  int kind = 0, variant = 0, p = 0, p_pad = 0, d = 0, d_pad = 0, K = 0, L = 0, C = 0, G = 0;
  int64_t N = 0;
  int h = 0, Lf = 16, b = 50, M = 64, max_batches = 1024, n_fd_draws = 250;
  int chain_base = 0;             // Philox chain id of fold-chain 0 (first_fold * L)
  double traj_len = 0.0;          // effective trajectory length (0: no cap)
  float jitter = 0.0f;            // effective step-size jitter of the fold chains
  Problem pb{};
  std::vector<void *> allocs;
  // device buffers
  float *X = nullptr, *y = nullptr, *minv = nullptr, *pool = nullptr;
  int *seg_off = nullptr, *seg_grp = nullptr, *grp_seg = nullptr;
  FoldDesc *folds = nullptr;
  IterState *st = nullptr;
  ChainBufs fold_cb, fd_cb, traj_cb;
  Accum acc{};
  float *ws = nullptr;
  size_t ws_floats = 0;
  unsigned int *tickets = nullptr;
  size_t n_tickets = 0;
  double *wmean = nullptr, *wM2 = nullptr;
  double *fold_out = nullptr, *tot_out = nullptr, *fin_scratch = nullptr;
  // host
  std::vector<int64_t> perm;
  int state = ST_CREATED;
  long long n_sampled = 0;
  double last_ms = 0.0;
  bool finalized = false;
  std::vector<double> h_fold, h_tot;
  // graphs
  cudaGraphExec_t g_sample_b = nullptr, g_fold_1 = nullptr, g_fd_1 = nullptr;
  // kernels issued by iterations: kernel nodes of each instantiated graph,
  // and the running count (exact while every iteration ran from a graph)
  std::map<cudaGraphExec_t, long long> graph_kernels;
  long long kernels_issued = 0;
  bool kernels_exact = true;
  int fd_n_adapt = 0;
  // tensor-core path
  bool tc = false;
  bool tc32 = false;              // the tensor-core path with TF32 operands (64-row chunks)
  int KP = 0, KS = 0, PN = 0, N_pad = 0, J = 0, n_sm = 148;
  int TN = 128;                   // rows per chunk of the tensor-core path
  float *X32 = nullptr, *XT32 = nullptr;   // TF32 form: X [N_pad x KP] and X^T [PN x N_pad]
  CUtensorMap tm_xt{};
  __nv_bfloat16 *X16 = nullptr;
  float *ycf = nullptr;           // tensor-core path: y per row (N_pad; folded into X16 for Gaussian models)
  CUtensorMap tm_x{};
  float *ws_tc = nullptr;
  float *theta_ref = nullptr;     // tensor-core path: centring reference (d_pad)
  float *eta_half = nullptr;      // tensor-core path: x . theta_ref / 2 per row (N_pad)
  bool centered = false;          // a reference has been set
  // autotuned launch configurations: split-N count of the FP32 gradient
  // kernels per chain count; X stages of the tensor-core kernel per
  // (chain count, theta lo used)
  std::map<int, int> tuned_splits;
  std::map<std::pair<int, int>, int> tuned_ns;
  std::map<int, int> tuned_ncta;          // tensor-core grid per chain count (one CTA per tile or one per SM)
  std::vector<std::string> tune_log;
  // host wall clock spent autotuning and capturing / instantiating graphs
  // (both inside pcv_warmup / pcv_sample; reported apart from them)
  double tune_ms = 0.0, capture_ms = 0.0;
  // Hyvarinen / Dawid-Sebastiani accumulators
  Extra extra{};
  double *extra_out = nullptr;
  // covariate-selection mask (d_pad floats 1 / 0; nullptr: every covariate)
  float *active_d = nullptr;
  std::vector<float> active_h;
  // two models in one context (pcv_model.active_covariates_b, Appendix B):
  // folds [K_model, 2 K_model) are model B's copies of folds [0, K_model),
  // chains [K_model L, 2 K_model L) its chains, and minv holds a second row
  // (model A's inverse mass with B's inactive coefficients at 0)
  bool pair = false;
  int K_model = 0;
  float *active_b_d = nullptr;
  std::vector<float> active_b_h;
  double *cmp_out = nullptr;
  size_t cmp_n = 0;
  // R-hat_max benchmark scratch
  double *shuf_blk = nullptr, *shuf_all = nullptr;
  unsigned long long *shuf_max = nullptr;
  size_t shuf_blk_n = 0, shuf_all_n = 0, shuf_max_n = 0;
  size_t ws_tc_floats = 0;
  unsigned int *tickets_tc = nullptr;
  size_t n_tickets_tc = 0;
  ChainBufs ld_cb;          // positions of pcv_log_density calls (tensor-core path)
  int ld_cap = 0;
  float *rstart = nullptr;
  // whole trajectories in one launch (k_traj_small) for small problems:
  // possible at all, the choice per chain count, and the BF16 form's copy
  // of X
  bool traj_ok = false;
  std::map<int, int> tuned_fused;
  __nv_bfloat16 *X16c = nullptr;
};

namespace {

pcv_status fail(pcv_ctx *x, pcv_status s, const std::string &msg) {
  if (x) x->err = msg;
  return s;
}

pcv_status fail_cuda(pcv_ctx *x, const char *what, cudaError_t e) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(x, e == cudaErrorMemoryAllocation ? PCV_E_OOM : PCV_E_CUDA, m);
}

#define CK(call)                                             \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return fail_cuda(x, #call, e_);   \
  } while (0)

void *dalloc(pcv_ctx *x, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  void *ptr = nullptr;
  if (x->opt.device_alloc) {
    ptr = x->opt.device_alloc(bytes, x->opt.alloc_user);
  } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
    ptr = nullptr;
  }
  if (ptr) {
    x->allocs.push_back(ptr);
    cudaMemsetAsync(ptr, 0, bytes, x->stream);
  }
  return ptr;
}

template <class T>
bool dalloc_n(pcv_ctx *x, T **out, size_t n) {
  *out = static_cast<T *>(dalloc(x, n * sizeof(T)));
  return *out != nullptr;
}

void free_all(pcv_ctx *x) {
  if (x->stream) cudaStreamSynchronize(x->stream);
  for (void *p : x->allocs) {
    if (x->opt.device_free) x->opt.device_free(p, x->opt.alloc_user);
    else cudaFree(p);
  }
  x->allocs.clear();
}

// chains per CTA tile and workspace row stride of the CUDA-core gradient
// kernels (split-N partials)
int chain_tile(const pcv_ctx *x) { return simt_chain_tile(x->p); }
int ws_stride_of(const pcv_ctx *x) {
  const int s = std::max(x->d_pad, std::max(0, simt_flat_pp(x->p)));
  return s + 4;
}

// chains per inverse-mass row (two models: one row per model; else one row)
int minv_every_of(const pcv_ctx *x) { return x->pair ? x->K_model * x->L : 0; }

// model B's inverse-mass row: model A's (row 0) with B's inactive
// coefficients at 0 (B's covariates are a subset of A's)
pcv_status sync_minv_b(pcv_ctx *x) {
  if (!x->pair) return PCV_OK;
  CK(cudaMemcpyAsync(x->minv + x->d_pad, x->minv, sizeof(float) * x->d_pad, cudaMemcpyDeviceToDevice, x->stream));
  k_mask_positions<<<(unsigned)((x->d + 255) / 256), 256, 0, x->stream>>>(1, x->d, x->d_pad, x->active_b_d,
                                                                          x->minv + x->d_pad);
  CK(cudaGetLastError());
  return PCV_OK;
}

int splits_cap(const pcv_ctx *x) {
  return x->variant == MV_HIER ? std::max(1, x->G / 4) : std::max(1, (int)(x->N / 256));
}

// fixed rule: enough CTAs to fill 4 per SM, at most the cap
int splits_rule(const pcv_ctx *x, int C) {
  const int tw = x->tc ? 32 : chain_tile(x);
  const int tiles = (C + tw - 1) / tw;
  const int s = (kTargetCtas + tiles - 1) / tiles;
  return std::max(1, std::min(s, splits_cap(x)));
}

int splits_for(const pcv_ctx *x, int C) {
  auto it = x->tuned_splits.find(C);
  return it != x->tuned_splits.end() ? it->second : splits_rule(x, C);
}

pcv_status ensure_ws(pcv_ctx *x, int C, int splits) {
  const int tw = chain_tile(x);
  const int tiles = (C + tw - 1) / tw;
  const int stride = ws_stride_of(x);
  const size_t need = (size_t)tiles * splits * tw * stride;
  if (need > x->ws_floats) {
    float *w;
    if (!dalloc_n(x, &w, need)) return fail(x, PCV_E_OOM, "workspace allocation failed");
    x->ws = w;
    x->ws_floats = need;
  }
  if ((size_t)tiles > x->n_tickets) {
    unsigned *t;
    if (!dalloc_n(x, &t, (size_t)tiles)) return fail(x, PCV_E_OOM, "ticket allocation failed");
    x->tickets = t;
    x->n_tickets = tiles;
  }
  return PCV_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void *ptr = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }
  return fn;
}

// 2-D bf16 tensor [rows x cols] row-major, 128 x 64 boxes, 128-byte swizzle
bool encode_bf16_map(CUtensorMap *m, const void *base, int rows, int cols) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {64, 128};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 2-D FP32 tensor [rows x cols] row-major, boxes of box_rows x 32 columns
// (128 bytes), 128-byte swizzle
bool encode_f32_map(CUtensorMap *m, const void *base, int rows, int cols, int box_rows) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 4};
  cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

pcv_status alloc_shadows(pcv_ctx *x, ChainBufs &cb, int C) {
  cb.C_pad = (C + 127) / 128 * 128;
  if (x->tc32) {
    // TF32 form: one FP32 shadow, 1 in the eta_ref / 2 columns
    if (!dalloc_n(x, &cb.shadow32, (size_t)cb.C_pad * x->KP)) return fail(x, PCV_E_OOM, "shadow allocation failed");
    CK(cudaMemsetAsync(cb.shadow32, 0, sizeof(float) * (size_t)cb.C_pad * x->KP, x->stream));
    if (!encode_f32_map(&cb.tm_hi, cb.shadow32, cb.C_pad, x->KP, 128))
      return fail(x, PCV_E_CUDA, "cuTensorMapEncodeTiled failed for the parameter shadow");
    k_shadow_ones32<<<(cb.C_pad * kEtaCols + 255) / 256, 256, 0, x->stream>>>(cb.C_pad, x->p, x->KP, cb.shadow32);
    CK(cudaGetLastError());
    return PCV_OK;
  }
  if (!dalloc_n(x, &cb.shadow_hi, (size_t)cb.C_pad * x->KP) || !dalloc_n(x, &cb.shadow_lo, (size_t)cb.C_pad * x->KP))
    return fail(x, PCV_E_OOM, "shadow allocation failed");
  if (!encode_bf16_map(&cb.tm_hi, cb.shadow_hi, cb.C_pad, x->KP) ||
      !encode_bf16_map(&cb.tm_lo, cb.shadow_lo, cb.C_pad, x->KP))
    return fail(x, PCV_E_CUDA, "cuTensorMapEncodeTiled failed for the parameter shadows");
  // the eta_ref / 2 columns: 1 in hi for every chain row (also the padding)
  k_shadow_ones<<<(cb.C_pad * kEtaCols + 255) / 256, 256, 0, x->stream>>>(cb.C_pad, x->p, x->KP, cb.shadow_hi);
  CK(cudaGetLastError());
  return PCV_OK;
}

// X stages that fit (the TF32 form: with as many X^T stages)
int tc_max_fit_stages(const pcv_ctx *x, int need_lo) {
  for (int ns = tc_max_stages(); ns > 2; --ns)
    if (tc_smem_bytes(x->KP, ns, x->tc32 ? ns : 0, need_lo, x->p, x->tc32 ? 1 : 0, x->PN) <= 227 * 1024) return ns;
  return 2;
}

// TF32 form: the X^T stages beside ns X stages (as many as fit)
int tc_xt_stages(const pcv_ctx *x, int ns) {
  int nt = ns;
  while (nt < tc_max_stages() && tc_smem_bytes(x->KP, ns, nt + 1, 0, x->p, 1, x->PN) <= 227 * 1024) ++nt;
  return nt;
}

TcArgs tc_args(pcv_ctx *x, int C, bool need_ll) {
  TcArgs t{};
  t.KP = x->KP; t.KS = x->KS; t.PN = x->PN; t.N_pad = x->N_pad; t.J = x->J;
  t.T = (C + 127) / 128;   // (the chain tiles; J = N_pad / TN chunks of rows)
  const long long U = (long long)t.T * t.J;
  t.n_cta = (int)std::min<long long>(x->n_sm, U);
  // the autotuner may choose one CTA per chain tile instead (no tile split
  // across CTAs: better for short tiles, worse when tiles are long)
  auto itn = x->tuned_ncta.find(C);
  if (itn != x->tuned_ncta.end()) t.n_cta = (int)std::min<long long>(itn->second, U);
  if (x->opt.tc_grid == 1) t.n_cta = (int)std::min<long long>(x->n_sm, U);   // fixed by the caller
  else if (x->opt.tc_grid == 2) t.n_cta = t.T;
  t.max_seg = tc_segments_per_tile(t.T, t.J, t.n_cta);
  // theta hi + lo where log densities are needed or no centring reference
  // is set yet; the kick-drift launches of centred chains use hi only
  t.need_lo = (need_ll || !x->centered) ? 1 : 0;
  t.accurate = need_ll ? 1 : 0;
  // the deepest X pipeline that fits in shared memory (without the theta
  // lo buffer, hi-only launches have room for one or two more stages),
  // unless the autotuner chose another depth for this chain count
  t.NS = tc_max_fit_stages(x, t.need_lo);
  auto it = x->tuned_ns.find(std::make_pair(C, t.need_lo));
  if (it != x->tuned_ns.end()) t.NS = it->second;
  t.theta_ref = x->theta_ref;
  t.ws = x->ws_tc;
  t.tickets = x->tickets_tc;
  t.err = &x->st->error;
  t.tf32 = x->tc32 ? 1 : 0;
  if (x->tc32) t.need_lo = 0;       // one TF32 part (centred)
  t.NT = x->tc32 ? tc_xt_stages(x, t.NS) : 0;
  return t;
}

pcv_status ensure_ws_tc(pcv_ctx *x, int C) {
  TcArgs t = tc_args(x, C, false);
  // sized for the larger of the default grid (one CTA per SM) and the tuned
  // one, so that either can run without a reallocation
  const int seg_default = tc_segments_per_tile(t.T, t.J, (int)std::min<long long>(x->n_sm, (long long)t.T * t.J));
  const size_t need = (size_t)t.T * std::max(t.max_seg, seg_default) * (t.PN + kTcSlots) * 128;
  if (need > x->ws_tc_floats) {
    float *w;
    if (!dalloc_n(x, &w, need)) return fail(x, PCV_E_OOM, "workspace allocation failed");
    x->ws_tc = w;
    x->ws_tc_floats = need;
  }
  if ((size_t)t.T > x->n_tickets_tc) {
    unsigned *tk;
    if (!dalloc_n(x, &tk, (size_t)t.T)) return fail(x, PCV_E_OOM, "ticket allocation failed");
    x->tickets_tc = tk;
    x->n_tickets_tc = t.T;
  }
  return PCV_OK;
}

GradArgs grad_args(pcv_ctx *x, const ChainBufs &cb, bool proposal) {
  GradArgs a{};
  a.C = cb.C;
  a.L = cb.L;
  a.fold_base = cb.fold_base;
  a.fold_of = nullptr;
  a.theta = proposal ? cb.theta_p : cb.theta;
  a.ld_theta = x->d_pad;
  a.grad = proposal ? cb.grad_p : cb.grad;
  a.ld_grad = x->d_pad;
  a.logp = proposal ? cb.logp_p : cb.logp;
  a.shat = proposal ? cb.shat_p : cb.shat;
  a.need_ll = 1;
  a.mode = MODE_NONE;
  a.r = cb.r;
  a.eps = &x->st->eps_iter;
  a.minv = x->minv;
  a.minv_every = minv_every_of(x); a.minv_ld = x->d_pad;
  a.splits = splits_for(x, cb.C);
  a.ws = x->ws;
  a.ws_stride = ws_stride_of(x);
  a.tickets = x->tickets;
  a.shadow_hi = x->tc ? cb.shadow_hi : nullptr;
  a.shadow_lo = x->tc ? cb.shadow_lo : nullptr;
  a.ld_shadow = x->tc ? x->KP : 0;
  return a;
}

pcv_status launch_grad(pcv_ctx *x, GradArgs a, const ChainBufs *cb = nullptr, int steps = 1) {
  if (x->tc) {
    if (!cb) return fail(x, PCV_E_UNSUPPORTED, "internal: tensor-core launch without a chain set");
    pcv_status s = ensure_ws_tc(x, a.C);
    if (s != PCV_OK) return s;
    TcArgs t = tc_args(x, a.C, a.need_ll != 0);
    t.shadow32 = cb->shadow32;
    t.steps = steps;
    // TF32 form: the X^T map goes where the bf16 form's lo shadow map goes
    CK(launch_grad_tc(x->tm_x, cb->tm_hi, x->tc32 ? x->tm_xt : cb->tm_lo, x->pb, a, t, x->stream));
    return PCV_OK;
  }
  pcv_status s = ensure_ws(x, a.C, a.splits);
  if (s != PCV_OK) return s;
  a.ws = x->ws;
  a.tickets = x->tickets;
  CK(launch_grad_simt(x->pb, a, x->stream));
  return PCV_OK;
}

// Kick-drift steps per tensor-core launch for a chain set: all L_f - 1 of
// them where each 128-chain tile has a CTA of its own, else one.
int tc_steps_per_launch(pcv_ctx *x, int C) {
  if (!x->tc || x->opt.tc_steps_per_launch == 1 || x->Lf < 3) return 1;
  const TcArgs t = tc_args(x, C, false);
  return t.n_cta == t.T ? x->Lf - 1 : 1;
}

// Whole trajectories in one launch: warps per chain (1, 2, 4, 8), or 0 for
// k_begin + L_f gradient launches.  Where the autotuner has not decided for
// a chain count, small problems (rows x register width <= 32 Ki) take it.
int fused_for(const pcv_ctx *x, int C) {
  if (!x->traj_ok) return 0;
  const int wmax = traj_max_wpc(x->pb);           // the hierarchical kernel: one warp per chain
  if (x->opt.fused_trajectory > 0) return std::min(x->opt.fused_trajectory, wmax);
  auto it = x->tuned_fused.find(C);
  if (it != x->tuned_fused.end()) return it->second;
  return x->N * (int64_t)traj_small_row_width(x->p) <= 32768 ? std::min(traj_default_wpc(C), wmax) : 0;
}

TrajArgs traj_args(pcv_ctx *x, ChainBufs &cb, bool fd, const float *r_given, float jitter, int wpc) {
  TrajArgs t{};
  t.wpc = wpc;
  t.C = cb.C; t.L = cb.L; t.fold_base = cb.fold_base; t.ld = x->d_pad;
  t.seed = x->opt.seed;
  t.stream = fd ? ST_FD_MOM : ST_MOM;
  t.chain_base = fd ? 0 : x->chain_base;
  t.iter = fd ? &x->st->fd_iter : &x->st->iter;
  t.eps = &x->st->eps;
  t.eps_iter = &x->st->eps_iter;
  t.jitter = jitter;
  t.minv = x->minv;
  t.minv_every = minv_every_of(x); t.minv_ld = x->d_pad;
  t.theta = cb.theta; t.grad = cb.grad; t.logp = cb.logp;
  t.r_given = r_given;
  t.theta_p = cb.theta_p; t.r = cb.r; t.grad_p = cb.grad_p;
  t.logp_p = cb.logp_p; t.shat_p = cb.shat_p; t.H0 = cb.H0;
  t.Lf = x->Lf;
  t.X16 = x->X16c;
  t.eval_only = 0;
  return t;
}

// The proposal of one HMC transition for every chain of a set (Section
// 3.3): momentum draw, half kick and drift, then L_f gradient evaluations
// with their kicks and drifts; as one launch per trajectory where fused
// (force: -1 the chain set's choice, 0 separate launches, w > 0 fused with w
// warps per chain), else k_begin and L_f gradient launches.
pcv_status launch_proposal(pcv_ctx *x, ChainBufs &cb, bool fd, const float *r_given, float jitter,
                           int force = -1) {
  const int wpc = force < 0 ? fused_for(x, cb.C) : force;
  if (wpc > 0) {
    CK(launch_traj_small(x->pb, traj_args(x, cb, fd, r_given, jitter, wpc), x->stream));
    return PCV_OK;
  }
  BeginArgs ba{};
  ba.C = cb.C; ba.d = x->d; ba.ld = x->d_pad;
  ba.seed = x->opt.seed;
  ba.stream = fd ? ST_FD_MOM : ST_MOM;
  ba.iter = fd ? &x->st->fd_iter : &x->st->iter;
  ba.theta = cb.theta; ba.grad = cb.grad; ba.logp = cb.logp;
  ba.theta_p = cb.theta_p; ba.r = cb.r; ba.H0 = cb.H0;
  ba.eps = &x->st->eps; ba.minv = x->minv;
  ba.minv_every = minv_every_of(x); ba.minv_ld = x->d_pad;
  ba.jitter = jitter;
  ba.eps_iter = &x->st->eps_iter;
  ba.chain_base = fd ? 0 : x->chain_base;
  ba.r_given = r_given;
  ba.shadow_hi = x->tc && !x->tc32 ? cb.shadow_hi : nullptr;
  ba.shadow_lo = x->tc && !x->tc32 ? cb.shadow_lo : nullptr;
  ba.shadow32 = x->tc32 ? cb.shadow32 : nullptr;
  ba.ld_shadow = x->KP;
  ba.shadow_d = x->p;
  ba.theta_ref = x->theta_ref;
  k_begin<<<begin_blocks(cb.C, x->d), 256, 0, x->stream>>>(ba);
  CK(cudaGetLastError());
  GradArgs ga = grad_args(x, cb, true);
  // the kick-drift steps: one launch each, or all in one launch where each
  // tile has a CTA of its own (BF16 form); then the last step with the log
  // densities
  const int per_launch = tc_steps_per_launch(x, cb.C);
  for (int s = 1; s <= x->Lf;) {
    const bool last = s == x->Lf;
    const int k = last ? 1 : std::min(per_launch, x->Lf - s);
    ga.mode = last ? MODE_LAST_KICK : MODE_KICK_DRIFT;
    ga.need_ll = last;
    pcv_status st = launch_grad(x, ga, &cb, k);
    if (st != PCV_OK) return st;
    s += k;
  }
  return PCV_OK;
}

pcv_status refresh(pcv_ctx *x, ChainBufs &cb);

// the fused-trajectory choice for a chain set: one launch per trajectory
// with 1, 2, 4 or 8 warps per chain against k_begin + L_f gradient
// launches, each timed (1 warm-up + 3) on the proposal buffers, which are
// scratch between iterations
pcv_status tune_fused(pcv_ctx *x, ChainBufs &cb) {
  const int C = cb.C;
  if (!x->traj_ok || !x->opt.autotune || x->opt.fused_trajectory > 0 || C < 1 || x->tuned_fused.count(C))
    return PCV_OK;
  const int before = fused_for(x, C);
  const bool fd = &cb == &x->fd_cb;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int cand[5] = {0, 1, 2, 4, 8};
  float best_ms = 1e30f;
  int best = 0;
  std::string log = "trajectory for " + std::to_string(C) + " chains:";
  for (int f : cand) {
    if (f > traj_max_wpc(x->pb)) continue;
    float ms = 0.0f;
    pcv_status s = launch_proposal(x, cb, fd, nullptr, 0.0f, f);
    if (s == PCV_OK) s = cudaEventRecord(e0, x->stream) == cudaSuccess ? PCV_OK : PCV_E_CUDA;
    for (int r = 0; r < 3 && s == PCV_OK; ++r) s = launch_proposal(x, cb, fd, nullptr, 0.0f, f);
    if (s == PCV_OK && (cudaEventRecord(e1, x->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      s = fail(x, PCV_E_CUDA, "autotuner timing failed");
    if (s != PCV_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return s; }
    log += (f == 0 ? std::string(" separate launches=") : " fused " + std::to_string(f) + " warps/chain=") +
           std::to_string(ms / 3.0f) + "ms";
    if (ms < best_ms) { best_ms = ms; best = f; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  x->tuned_fused[C] = best;
  x->tune_log.push_back(log + " -> " + (best == 0 ? std::string("separate") : "fused " + std::to_string(best)));
  // the cached gradients and log densities come from the chosen path
  if ((best != 0) != (before != 0)) return refresh(x, cb);
  return PCV_OK;
}

// Autotuner: time the gradient launch of a chain set (no leapfrog update;
// the proposal buffers are scratch between iterations) under a few launch
// configurations and keep the fastest for this chain count.
pcv_status tune(pcv_ctx *x, ChainBufs &cb) {
  if (!x->opt.autotune || cb.C < 1) return PCV_OK;
  const int C = cb.C;
  const int need_lo = x->centered ? 0 : 1;
  if (x->tc ? x->tuned_ns.count(std::make_pair(C, need_lo)) > 0 : x->tuned_splits.count(C) > 0)
    return tune_fused(x, cb);
  const auto w0 = std::chrono::steady_clock::now();
  struct AddWall {   // adds the wall time of this call on every return path
    double *acc;
    std::chrono::steady_clock::time_point t0;
    ~AddWall() { *acc += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count(); }
  } add_wall{&x->tune_ms, w0};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto time_launch = [&](float *ms) -> pcv_status {
    GradArgs a = grad_args(x, cb, true);
    a.mode = MODE_NONE;
    a.need_ll = 0;
    pcv_status s = launch_grad(x, a, &cb);                       // warm-up
    if (s != PCV_OK) return s;
    CK(cudaEventRecord(e0, x->stream));
    for (int r = 0; r < 3 && s == PCV_OK; ++r) s = launch_grad(x, a, &cb);
    if (s != PCV_OK) return s;
    CK(cudaEventRecord(e1, x->stream));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(ms, e0, e1));
    return PCV_OK;
  };
  std::vector<int> cand;
  if (x->tc) {
    for (int ns = 2; ns <= tc_max_fit_stages(x, need_lo); ++ns) cand.push_back(ns);
  } else {
    const int s0 = splits_rule(x, C), cap = splits_cap(x);
    for (int v : {s0 / 4, s0 / 2, s0, 2 * s0})
      if (v >= 1 && v <= cap && std::find(cand.begin(), cand.end(), v) == cand.end()) cand.push_back(v);
  }
  int best = cand.back();
  float best_ms = 1e30f;
  std::string log = std::string(x->tc ? "tensor-core X stages" : "FP32 split-N count") + " for " +
                    std::to_string(C) + " chains:";
  for (int v : cand) {
    if (x->tc) x->tuned_ns[std::make_pair(C, need_lo)] = v;
    else x->tuned_splits[C] = v;
    float ms = 0.0f;
    pcv_status s = time_launch(&ms);
    if (s != PCV_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return s; }
    log += " " + std::to_string(v) + "=" + std::to_string(ms / 3.0f) + "ms";
    if (ms < best_ms) { best_ms = ms; best = v; }
  }
  if (x->tc) x->tuned_ns[std::make_pair(C, need_lo)] = best;
  else x->tuned_splits[C] = best;
  x->tune_log.push_back(log + " -> " + std::to_string(best));
  if (x->tc && x->opt.tc_grid == 0 && x->tuned_ncta.count(C) == 0) {
    // grid: one CTA per SM (tiles split across CTAs, stream-K) or, when
    // there are fewer tiles than SMs, one CTA per tile
    const int T = (C + 127) / 128;
    if (T < x->n_sm) {
      x->tuned_ncta[C] = T;
      float ms = 0.0f;
      pcv_status s = time_launch(&ms);
      if (s != PCV_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return s; }
      const bool per_tile = ms < best_ms;
      x->tune_log.push_back("tensor-core grid for " + std::to_string(C) + " chains: " + std::to_string(x->n_sm) +
                            " CTAs=" + std::to_string(best_ms / 3.0f) + "ms " + std::to_string(T) + " CTAs=" +
                            std::to_string(ms / 3.0f) + "ms -> " + std::to_string(per_tile ? T : x->n_sm));
      x->tuned_ncta[C] = per_tile ? T : x->n_sm;
    } else {
      x->tuned_ncta[C] = x->n_sm;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return tune_fused(x, cb);
}

// write the bf16 shadow of a chain set's current positions (tensor-core path)
pcv_status write_shadow(pcv_ctx *x, ChainBufs &cb, const float *theta, int ld) {
  if (!x->tc) return PCV_OK;
  const long long T = (long long)cb.C * x->p;
  // beta only: a log sigma coordinate has no tensor-core operand column
  if (x->tc32) {
    k_shadow32<<<(unsigned)((T + 255) / 256), 256, 0, x->stream>>>(cb.C, x->p, ld, theta, x->theta_ref, cb.shadow32,
                                                                  x->KP);
    CK(cudaGetLastError());
    return PCV_OK;
  }
  k_shadow<<<(unsigned)((T + 255) / 256), 256, 0, x->stream>>>(cb.C, x->p, ld, theta, x->theta_ref, cb.shadow_hi,
                                                              cb.shadow_lo, x->KP);
  CK(cudaGetLastError());
  return PCV_OK;
}

// eta_ref / 2 (eta_half) into the operand columns of the bf16 design matrix
pcv_status fold_eta(pcv_ctx *x) {
  if (x->tc32) {
    k_eta_fold32<<<(x->N_pad + 255) / 256, 256, 0, x->stream>>>(x->N_pad, x->p, x->KP, x->eta_half,
                                                               x->kind == PCV_LOGISTIC ? nullptr : x->ycf, x->X32);
    CK(cudaGetLastError());
    return PCV_OK;
  }
  // Gaussian models fold -y / 2 into the same columns (zero-padded y)
  k_eta_fold<<<(x->N_pad + 255) / 256, 256, 0, x->stream>>>(x->N_pad, x->p, x->KP, x->eta_half,
                                                           x->kind == PCV_LOGISTIC ? nullptr : x->ycf, x->X16);
  CK(cudaGetLastError());
  return PCV_OK;
}

// tensor-core path: centre on the mean of n parameter vectors (ld apart)
pcv_status set_reference(pcv_ctx *x, const float *src, int n, int ld) {
  if (!x->tc) return PCV_OK;
  k_theta_ref<<<(x->d + 127) / 128, 128, 0, x->stream>>>(n, x->d, ld, src, x->theta_ref);
  CK(cudaGetLastError());
  if (x->tc32)
    k_eta_ref32<<<(x->N_pad + 255) / 256, 256, 0, x->stream>>>((int)x->N, x->N_pad, x->p, x->KP, x->X32,
                                                              x->theta_ref, x->eta_half);
  else
  k_eta_ref<<<(x->N_pad + 255) / 256, 256, 0, x->stream>>>((int)x->N, x->N_pad, x->p, x->KP, x->X16, x->theta_ref,
                                                          x->eta_half);
  CK(cudaGetLastError());
  const pcv_status s = fold_eta(x);
  if (s == PCV_OK) x->centered = true;
  return s;
}

// evaluate gradient, logp and shat at the current positions of a chain set
pcv_status refresh(pcv_ctx *x, ChainBufs &cb) {
  pcv_status s = write_shadow(x, cb, cb.theta, x->d_pad);
  if (s != PCV_OK) return s;
  if (const int wpc = fused_for(x, cb.C)) {
    // the same gradient as the fused trajectories (no momentum, no update)
    TrajArgs t = traj_args(x, cb, false, nullptr, 0.0f, wpc);
    t.eval_only = 1;
    t.eps_iter = nullptr;
    t.grad_p = cb.grad; t.logp_p = cb.logp; t.shat_p = cb.shat;
    CK(launch_traj_small(x->pb, t, x->stream));
    return PCV_OK;
  }
  GradArgs a = grad_args(x, cb, false);
  return launch_grad(x, a, &cb);
}

pcv_status launch_fd_adapt(pcv_ctx *x, ChainBufs &cb);

// one HMC transition for every chain of a set (Section 3.3)
pcv_status launch_iteration(pcv_ctx *x, ChainBufs &cb, bool fd, bool accumulate) {
  const int wpc = fused_for(x, cb.C);
  const bool extra = accumulate && x->extra.flags;
  if (wpc > 0 && !extra) {
    // the whole iteration in one launch: trajectory, Metropolis test and
    // the draw's accumulators (the proposal never leaves the registers)
    TrajArgs t = traj_args(x, cb, fd, nullptr, fd ? 0.0f : x->jitter, wpc);
    t.accept = 1;
    t.acc_stream = fd ? ST_FD_ACC : ST_ACC;
    t.st = x->st;
    t.fd = fd ? 1 : 0;
    t.accumulate = accumulate ? 1 : 0;
    t.acc = x->acc;
    t.accept_prob = cb.accept_prob;
    t.theta_w = cb.theta; t.grad_w = cb.grad; t.logp_w = cb.logp; t.shat_w = cb.shat;
    CK(launch_traj_small(x->pb, t, x->stream));
    return fd ? launch_fd_adapt(x, cb) : PCV_OK;
  }
  pcv_status sp = launch_proposal(x, cb, fd, nullptr, fd ? 0.0f : x->jitter);
  if (sp != PCV_OK) return sp;
  AcceptArgs aa{};
  aa.C = cb.C; aa.d = x->d; aa.ld = x->d_pad;
  aa.seed = x->opt.seed;
  aa.stream = fd ? ST_FD_ACC : ST_ACC;
  aa.chain_base = fd ? 0 : x->chain_base;
  aa.st = x->st;
  aa.fd = fd ? 1 : 0;
  aa.theta = cb.theta; aa.grad = cb.grad; aa.logp = cb.logp; aa.shat = cb.shat;
  aa.theta_p = cb.theta_p; aa.r = cb.r; aa.grad_p = cb.grad_p;
  aa.logp_p = cb.logp_p; aa.shat_p = cb.shat_p; aa.H0 = cb.H0;
  aa.minv = x->minv;
  aa.minv_every = minv_every_of(x); aa.minv_ld = x->d_pad;
  aa.accumulate = accumulate ? 1 : 0;
  aa.acc = x->acc;
  aa.accept_prob = cb.accept_prob;
  k_accept<<<(cb.C + kAccChains - 1) / kAccChains, kAccWarps * 32, 0, x->stream>>>(aa);
  CK(cudaGetLastError());
  if (accumulate && x->extra.flags) {
    k_extra_push<<<(cb.C + 7) / 8, 256, sizeof(double) * 8 * x->extra.T, x->stream>>>(
        x->pb, grad_args(x, cb, false), x->extra, &x->st->iter, x->opt.seed, x->chain_base);
    CK(cudaGetLastError());
  }
  return fd ? launch_fd_adapt(x, cb) : PCV_OK;
}

// the full-data adaptation after an iteration of the full-data chains
pcv_status launch_fd_adapt(pcv_ctx *x, ChainBufs &cb) {
  {
    FdAdaptArgs fa{};
    fa.st = x->st;
    fa.n_adapt = x->fd_n_adapt;
    fa.w0 = x->fd_n_adapt / 4;
    fa.w1 = x->fd_n_adapt / 2;
    fa.w2 = (7 * x->fd_n_adapt) / 8;
    fa.adapt_eps = !(x->opt.step_size > 0);
    fa.adapt_mass = fa.adapt_eps && x->opt.inv_mass_diag == nullptr;
    fa.C = cb.C; fa.d = x->d; fa.ld = x->d_pad;
    fa.theta = cb.theta;
    fa.accept_prob = cb.accept_prob;
    fa.minv = x->minv;
    fa.wmean = x->wmean; fa.wM2 = x->wM2;
    fa.pool = x->pool;
    fa.active = x->active_d;
    fa.n_keep = x->n_fd_draws;
    k_fd_adapt<<<1, 128, 0, x->stream>>>(fa);
    CK(cudaGetLastError());
  }
  return PCV_OK;
}

// run `count` iterations, through a captured graph of `per_graph` iterations
pcv_status run_iterations(pcv_ctx *x, ChainBufs &cb, bool fd, bool accumulate, long long count,
                          cudaGraphExec_t *cache, int per_graph) {
  if (count <= 0) return PCV_OK;
  if (!x->opt.use_graphs) {
    x->kernels_exact = false;          // launches outside a graph are not counted
    for (long long i = 0; i < count; ++i) {
      pcv_status s = launch_iteration(x, cb, fd, accumulate);
      if (s != PCV_OK) return s;
    }
    return PCV_OK;
  }
  // make sure workspaces exist before capture (no allocation inside a capture)
  pcv_status s0 = x->tc ? ensure_ws_tc(x, cb.C) : ensure_ws(x, cb.C, splits_for(x, cb.C));
  if (s0 != PCV_OK) return s0;
  if (!*cache) {
    const auto w0 = std::chrono::steady_clock::now();
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(x->stream, cudaStreamCaptureModeThreadLocal));
    pcv_status s = PCV_OK;
    for (int i = 0; i < per_graph && s == PCV_OK; ++i) s = launch_iteration(x, cb, fd, accumulate);
    cudaError_t e = cudaStreamEndCapture(x->stream, &g);
    if (s != PCV_OK) return s;
    if (e != cudaSuccess) return fail_cuda(x, "cudaStreamEndCapture", e);
    // the graph's kernel nodes: the kernels each replay issues
    long long nk = 0;
    {
      size_t nn = 0;
      if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
        std::vector<cudaGraphNode_t> nodes(nn);
        if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
          for (size_t k = 0; k < nn; ++k) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nodes[k], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
          }
      }
    }
    e = cudaGraphInstantiate(cache, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail_cuda(x, "cudaGraphInstantiate", e);
    x->graph_kernels[*cache] = nk;
    x->capture_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
  }
  long long full = count / per_graph, rest = count - full * per_graph;
  for (long long i = 0; i < full; ++i) CK(cudaGraphLaunch(*cache, x->stream));
  {
    const auto it = x->graph_kernels.find(*cache);
    if (it == x->graph_kernels.end() || (rest > 0 && it->second % per_graph != 0)) x->kernels_exact = false;
    else x->kernels_issued += full * it->second + rest * (it->second / per_graph);
  }
  for (long long i = 0; i < rest; ++i) {
    pcv_status s = launch_iteration(x, cb, fd, accumulate);
    if (s != PCV_OK) return s;
  }
  return PCV_OK;
}

pcv_status alloc_chains(pcv_ctx *x, ChainBufs &cb, int C, int L, int fold_base) {
  cb.C = C; cb.L = L; cb.fold_base = fold_base;
  const size_t n = (size_t)C * x->d_pad;
  bool ok = dalloc_n(x, &cb.theta, n) && dalloc_n(x, &cb.grad, n) && dalloc_n(x, &cb.theta_p, n) &&
            dalloc_n(x, &cb.r, n) && dalloc_n(x, &cb.grad_p, n) && dalloc_n(x, &cb.logp, (size_t)C) &&
            dalloc_n(x, &cb.shat, (size_t)C) && dalloc_n(x, &cb.logp_p, (size_t)C) &&
            dalloc_n(x, &cb.shat_p, (size_t)C) && dalloc_n(x, &cb.H0, (size_t)C) &&
            dalloc_n(x, &cb.accept_prob, (size_t)C);
  if (!ok) return fail(x, PCV_E_OOM, "chain state allocation failed");
  return x->tc ? alloc_shadows(x, cb, C) : PCV_OK;
}

pcv_status alloc_accum(pcv_ctx *x) {
  Accum &A = x->acc;
  const size_t C = (size_t)x->C;
  A.C = x->C; A.M = x->M; A.max_batches = x->max_batches; A.b = x->b;
  bool ok = true;
  double **scal[] = {&A.Ux, &A.Ux2, &A.Zx, &A.em, &A.emean, &A.eM2, &A.vm, &A.vmean, &A.vM2,
                     &A.wmean, &A.wM2, &A.bmean_cur, &A.bM2_cur, &A.c0, &A.xsum};
  for (double **pp : scal) ok = ok && dalloc_n(x, pp, C);
  ok = ok && dalloc_n(x, &A.bmean, C * x->max_batches) && dalloc_n(x, &A.bM2, C * x->max_batches);
  ok = ok && dalloc_n(x, &A.lagsum, C * (x->M + 1)) && dalloc_n(x, &A.first, C * std::max(1, x->M)) &&
       dalloc_n(x, &A.ring, C * std::max(1, x->M));
  ok = ok && dalloc_n(x, &A.div, C) && dalloc_n(x, &A.acc, C);
  A.draw_cap = x->opt.store_draws > 0 ? x->opt.store_draws : 0;
  A.draws = nullptr;
  if (A.draw_cap > 0) ok = ok && dalloc_n(x, &A.draws, C * A.draw_cap);
  if (!ok) return fail(x, PCV_E_OOM, "accumulator allocation failed");
  // the shifts start at -inf (A2 "initial entries -inf"); the shifted sums
  // U_x, U_x^2, Z_x and the Welford states start at 0 (allocations are zeroed)
  std::vector<double> ninf(C, -INFINITY);
  for (double *p : {A.em, A.vm})
    CK(cudaMemcpyAsync(p, ninf.data(), C * sizeof(double), cudaMemcpyHostToDevice, x->stream));
  CK(cudaStreamSynchronize(x->stream));
  return PCV_OK;
}

// order the legacy default stream and the private stream (NULL stream option)
void enter(pcv_ctx *x) {
  if (x->own_stream) {
    cudaEventRecord(x->ev_in, cudaStreamLegacy);
    cudaStreamWaitEvent(x->stream, x->ev_in, 0);
  }
}
void leave(pcv_ctx *x) {
  if (x->own_stream) {
    cudaEventRecord(x->ev_out, x->stream);
    cudaStreamWaitEvent(cudaStreamLegacy, x->ev_out, 0);
  }
}

pcv_status finalize(pcv_ctx *x) {
  if (x->finalized) return PCV_OK;
  if (x->n_sampled < 2LL * x->b)
    return fail(x, PCV_E_BAD_STATE, "need at least two batches of draws (pcv_sample)");
  k_finalize<<<(x->K + 127) / 128, 128, 0, x->stream>>>(x->acc, x->K, x->L, x->n_sampled,
                                                          x->fold_out, x->fin_scratch);
  CK(cudaGetLastError());
  k_totals<<<1, 256, 0, x->stream>>>(x->fold_out, x->K, (double)x->L * x->n_sampled, x->tot_out);
  CK(cudaGetLastError());
  x->h_fold.resize((size_t)x->K * F_NFIELDS);
  x->h_tot.resize(T_NFIELDS);
  CK(cudaMemcpyAsync(x->h_fold.data(), x->fold_out, x->h_fold.size() * sizeof(double),
                     cudaMemcpyDeviceToHost, x->stream));
  CK(cudaMemcpyAsync(x->h_tot.data(), x->tot_out, x->h_tot.size() * sizeof(double),
                     cudaMemcpyDeviceToHost, x->stream));
  CK(cudaStreamSynchronize(x->stream));
  x->finalized = true;
  return PCV_OK;
}

// message of the calling thread's last failed pcv_create (there is no
// context to hold it)
std::string &create_error() {
  static thread_local std::string m = "null context";
  return m;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void pcv_default_options(pcv_options *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->seed = 0;
  o->leapfrog_steps = 16;
  o->step_size = -1.0;
  o->inv_mass_diag = nullptr;
  o->batch_size = 50;
  o->hv_buffer = 0;
  o->precision = PCV_FP32_SIMT;
  o->cuda_stream = nullptr;
  o->store_draws = 0;
  o->acov_max_lag = 64;
  o->max_batches = 1024;
  o->n_fulldata_draws = 250;
  o->init_scale = 1.0;
  o->use_graphs = 1;
  o->trajectory_length = -1.0;
  o->step_jitter = -1.0;
  o->autotune = 1;
  o->extra_scores = 0;
  o->first_fold = 0;
  o->fused_trajectory = -1;
  o->tc_steps_per_launch = 0;
  o->tc_grid = 0;
}

pcv_status pcv_create(const pcv_model *model, const float *X, const float *y,
                      const int32_t *fold_assignment, int64_t N, int32_t p, int32_t chains_per_fold,
                      const pcv_options *opt, pcv_ctx **out) {
  auto invalid = [](const char *m) {
    create_error() = m;
    return PCV_E_INVALID_ARG;
  };
  if (!out) return invalid("out is NULL");
  *out = nullptr;
  if (!model || !X || !y || !fold_assignment || !opt) return invalid("a required pointer is NULL");
  if (N < 1 || p < 1 || chains_per_fold < 2 || N > (int64_t)1 << 30)
    return invalid("need 1 <= N <= 2^30, p >= 1 and chains_per_fold >= 2");
  if (opt->leapfrog_steps < 1 || opt->batch_size < 1 || opt->hv_buffer < 0 ||
      opt->acov_max_lag < 0 || opt->max_batches < 1 || opt->n_fulldata_draws < 1 ||
      !(opt->step_jitter < 1.0) || !std::isfinite(opt->trajectory_length) || opt->first_fold < 0 ||
      (opt->fused_trajectory != -1 && opt->fused_trajectory != 0 && opt->fused_trajectory != 1 &&
       opt->fused_trajectory != 2 && opt->fused_trajectory != 4 && opt->fused_trajectory != 8) ||
      (opt->tc_steps_per_launch != 0 && opt->tc_steps_per_launch != 1) || opt->tc_grid < 0 || opt->tc_grid > 2)
    return invalid("an option is out of range");
  if (model->kind < PCV_GAUSS_LINEAR || model->kind > PCV_AR_GAUSS) return invalid("unknown model kind");
  if (!(model->beta_prior_sd > 0)) return invalid("beta_prior_sd must be > 0");

  pcv_ctx *x = new pcv_ctx();
  x->opt = *opt;
  x->kind = model->kind;
  x->N = N; x->p = p; x->L = chains_per_fold;
  x->h = opt->hv_buffer; x->Lf = opt->leapfrog_steps; x->b = opt->batch_size;
  x->M = opt->acov_max_lag; x->max_batches = opt->max_batches; x->n_fd_draws = opt->n_fulldata_draws;
  {
    // trajectory length (cap of the adapted step size) and step-size jitter:
    // < 0 selects the defaults, which apply when the step size is adapted
    const bool adapted = !(opt->step_size > 0);
    x->traj_len = opt->trajectory_length < 0 ? (adapted ? 1.5707963267948966 : 0.0) : opt->trajectory_length;
    x->jitter = (float)(opt->step_jitter < 0 ? (adapted ? 0.5 : 0.0) : opt->step_jitter);
  }
  auto bail = [&](pcv_status s, const std::string &m) {
    // creation failed: release everything; the message stays with the
    // calling thread for pcv_last_error(NULL)
    create_error() = m;
    free_all(x);
    if (x->own_stream && x->stream) cudaStreamDestroy(x->stream);
    delete x;
    return s;
  };
  if (opt->precision < PCV_FP32_SIMT || opt->precision > PCV_BF16) return bail(PCV_E_INVALID_ARG, "bad precision");
  // BF16 and TF32 run on the tensor-core path (tcgen05), TF32 with 32-bit
  // operands
  x->tc = opt->precision == PCV_BF16 || opt->precision == PCV_TF32;
  x->tc32 = opt->precision == PCV_TF32;
  if (x->tc32 && (model->kind == PCV_HIER_GAUSS || p > 112))
    return bail(PCV_E_UNSUPPORTED, "the TF32 path covers the flat models (logistic, Gaussian linear, AR) with p <= 112");
  if (x->tc && (model->kind == PCV_HIER_GAUSS || p > 128))
    return bail(PCV_E_UNSUPPORTED, "the BF16 tensor-core path covers the flat models (logistic, Gaussian linear, "
                                   "AR) with p <= 128");
  // model variant and dimension
  if (x->kind == PCV_LOGISTIC) { x->variant = MV_LOGISTIC; x->d = p; }
  else if (x->kind == PCV_HIER_GAUSS) {
    if (!model->group || model->n_groups < 1) return bail(PCV_E_INVALID_ARG, "HIER_GAUSS needs groups");
    if (x->h > 0) return bail(PCV_E_UNSUPPORTED, "hv_buffer with HIER_GAUSS");
    x->variant = MV_HIER; x->G = model->n_groups; x->d = p + x->G + 2;
  } else if (x->kind == PCV_GAUSS_LINEAR && model->sigma_known > 0) {
    x->variant = MV_GAUSS_KNOWN; x->d = p;
  } else {
    x->variant = MV_GAUSS_LOGSIG; x->d = p + 1;
  }
  if ((x->variant == MV_GAUSS_LOGSIG || x->variant == MV_HIER) && !(model->sigma_prior_sd > 0))
    return bail(PCV_E_INVALID_ARG, "sigma_prior_sd must be > 0");
  if (x->variant == MV_HIER && !(model->tau_prior_sd > 0)) return bail(PCV_E_INVALID_ARG, "tau_prior_sd must be > 0");
  const int PP = simt_flat_pp(p);
  if (!x->tc && (p > 128 || (PP < 0 && x->variant == MV_HIER)))
    return bail(PCV_E_UNSUPPORTED, "FP32 path: p <= 128 (flat models) or p <= 32 (hierarchical)");
  x->p_pad = PP > 0 ? PP : (p + 3) / 4 * 4;
  if (x->tc) {
    // the first GEMM's K covers the p covariates and the eta_ref / 2 columns
    // (K steps of 16 bf16 or 8 TF32 values; 128-byte K atoms of 64 or 32)
    const int kstep = x->tc32 ? 8 : 16, atom = x->tc32 ? 32 : 64;
    x->TN = x->tc32 ? 64 : 128;
    x->KS = (p + kEtaCols + kstep - 1) / kstep;
    x->KP = (kstep * x->KS + atom - 1) / atom * atom;
    x->PN = 16 * ((p + 15) / 16);
    x->N_pad = (int)((N + x->TN - 1) / x->TN * x->TN);
    x->J = x->N_pad / x->TN;
  }
  x->d_pad = (x->d + 3) / 4 * 4;

  // data checks
  {
    // exponent all ones = Inf or NaN; a branch-free pass the compiler vectorises
    uint32_t bad = 0;
    for (int64_t i = 0; i < N * p; ++i) {
      uint32_t u;
      std::memcpy(&u, X + i, sizeof(u));
      bad |= (uint32_t)((u & 0x7f800000u) == 0x7f800000u);
    }
    if (bad) return bail(PCV_E_NUMERIC, "non-finite X");
  }
  for (int64_t i = 0; i < N; ++i) {
    if (!std::isfinite(y[i])) return bail(PCV_E_NUMERIC, "non-finite y");
    if (x->kind == PCV_LOGISTIC && y[i] != 0.0f && y[i] != 1.0f)
      return bail(PCV_E_INVALID_ARG, "LOGISTIC needs y in {0, 1}");
  }
  int K = 0;
  for (int64_t i = 0; i < N; ++i) {
    const int f = fold_assignment[i];
    if (f < -1) return bail(PCV_E_INVALID_ARG, "fold ids must be >= -1");
    K = std::max(K, f + 1);
  }
  if (K < 1) return bail(PCV_E_INVALID_ARG, "no folds");
  x->K = K;
  x->K_model = K;
  x->pair = model->active_covariates_b != nullptr;
  if (x->pair) {
    if (opt->first_fold != 0) return bail(PCV_E_UNSUPPORTED, "two models in one context: first_fold must be 0");
    x->K = 2 * K;     // model B's folds follow model A's
  }
  x->C = x->K * x->L;
  x->chain_base = opt->first_fold * x->L;
  if (x->variant == MV_HIER)
    for (int64_t i = 0; i < N; ++i)
      if (model->group[i] < 0 || model->group[i] >= x->G) return bail(PCV_E_INVALID_ARG, "group id out of range");

  // row order: sort by (fold, group) unless an h(v) buffer needs time order
  x->perm.resize(N);
  std::iota(x->perm.begin(), x->perm.end(), 0);
  auto fkey = [&](int64_t i) { return fold_assignment[i] < 0 ? K : fold_assignment[i]; };
  if (x->h == 0) {
    // stable counting sorts (the keys are small integers): by group first
    // (hierarchical model), then by fold, so rows end up ordered by
    // (fold, group) and by original index within equal keys
    auto counting_pass = [&](int nkeys, auto key) {
      std::vector<int64_t> start((size_t)nkeys + 1, 0);
      for (int64_t r = 0; r < N; ++r) start[(size_t)key(x->perm[r]) + 1]++;
      for (int k = 0; k < nkeys; ++k) start[(size_t)k + 1] += start[(size_t)k];
      std::vector<int64_t> out((size_t)N);
      for (int64_t r = 0; r < N; ++r) out[(size_t)start[(size_t)key(x->perm[r])]++] = x->perm[r];
      x->perm.swap(out);
    };
    if (x->variant == MV_HIER) counting_pass(x->G, [&](int64_t i) { return model->group[i]; });
    counting_pass(K + 1, fkey);
  }
  std::vector<FoldDesc> fds(K + 1, FoldDesc{0, 0, 0, 0});
  std::vector<int64_t> cnt(K, 0), lo(K, -1), hi(K, -1);
  for (int64_t r = 0; r < N; ++r) {
    const int f = fold_assignment[x->perm[r]];
    if (f < 0) continue;
    cnt[f]++;
    if (lo[f] < 0) lo[f] = r;
    hi[f] = r + 1;
  }
  for (int k = 0; k < K; ++k) {
    if (cnt[k] == 0) return bail(PCV_E_INVALID_ARG, "fold " + std::to_string(k) + " has no test rows");
    if (hi[k] - lo[k] != cnt[k])
      return bail(PCV_E_INVALID_ARG, "fold " + std::to_string(k) + " test rows are not contiguous");
    const int64_t elo = std::max<int64_t>(0, lo[k] - x->h), ehi = std::min<int64_t>(N, hi[k] + x->h);
    if (N - (ehi - elo) < 1) return bail(PCV_E_INVALID_ARG, "fold " + std::to_string(k) + " has no training rows");
    fds[k] = FoldDesc{(int)lo[k], (int)hi[k], (int)elo, (int)ehi};
  }
  if (x->pair) {   // model B's folds: the same rows; the full-data descriptor last
    std::vector<FoldDesc> two(fds.begin(), fds.begin() + K);
    two.insert(two.end(), fds.begin(), fds.end());
    fds.swap(two);
  }
  // hierarchical segments: one contiguous row run per group
  std::vector<int> seg_off, seg_grp, grp_seg;
  if (x->variant == MV_HIER) {
    grp_seg.assign(x->G, -1);
    for (int64_t r = 0; r < N; ++r) {
      const int g = model->group[x->perm[r]];
      if (r == 0 || g != model->group[x->perm[r - 1]]) {
        if (grp_seg[g] >= 0) return bail(PCV_E_UNSUPPORTED, "a group spans several folds");
        grp_seg[g] = (int)seg_grp.size();
        seg_grp.push_back(g);
        seg_off.push_back((int)r);
      }
    }
    seg_off.push_back((int)N);
    for (int g = 0; g < x->G; ++g)
      if (grp_seg[g] < 0) return bail(PCV_E_INVALID_ARG, "every group needs at least one row");
  }

  // stream and events
  if (opt->cuda_stream) {
    x->stream = (cudaStream_t)opt->cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&x->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(PCV_E_CUDA, "cudaStreamCreate failed");
    x->own_stream = true;
  }
  cudaEventCreateWithFlags(&x->ev_in, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&x->ev_out, cudaEventDisableTiming);
  cudaEventCreate(&x->ev0);
  cudaEventCreate(&x->ev1);
  enter(x);

  // device data
  // y and the row permutation on the host; X goes to the device as the
  // caller laid it out and is gathered into the fold-sorted layout there
  // (as are its bf16 copy and the per-fold sums of the tensor-core path)
  std::vector<float> hy(N);
  std::vector<int> hperm(N);
  for (int64_t r = 0; r < N; ++r) {
    const int64_t i = x->perm[r];
    hy[r] = y[i];
    hperm[r] = (int)i;
  }
  if (!dalloc_n(x, &x->X, (size_t)N * x->p_pad) || !dalloc_n(x, &x->y, (size_t)N) ||
      !dalloc_n(x, &x->folds, (size_t)x->K + 1) || !dalloc_n(x, &x->minv, (size_t)x->d_pad * (x->pair ? 2 : 1)) ||
      !dalloc_n(x, &x->st, 1) || !dalloc_n(x, &x->wmean, (size_t)x->d) || !dalloc_n(x, &x->wM2, (size_t)x->d) ||
      !dalloc_n(x, &x->pool, (size_t)x->n_fd_draws * kNumFdChains * x->d_pad) ||
      !dalloc_n(x, &x->fold_out, (size_t)x->K * F_NFIELDS) || !dalloc_n(x, &x->tot_out, (size_t)T_NFIELDS) ||
      !dalloc_n(x, &x->fin_scratch, (size_t)x->K * (4 * x->L + 2 * (x->M + 2))))
    return bail(PCV_E_OOM, "device allocation failed");
  {
    float *xraw = nullptr;
    int *dperm = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void **>(&xraw), sizeof(float) * (size_t)N * p, x->stream) != cudaSuccess)
      return bail(PCV_E_OOM, "staging allocation failed");
    if (cudaMallocAsync(reinterpret_cast<void **>(&dperm), sizeof(int) * (size_t)N, x->stream) != cudaSuccess) {
      cudaFreeAsync(xraw, x->stream);
      return bail(PCV_E_OOM, "staging allocation failed");
    }
    cudaMemcpyAsync(xraw, X, sizeof(float) * (size_t)N * p, cudaMemcpyHostToDevice, x->stream);
    cudaMemcpyAsync(dperm, hperm.data(), sizeof(int) * (size_t)N, cudaMemcpyHostToDevice, x->stream);
    const long long items = (long long)N * p;
    k_gather_rows<<<(unsigned)((items + 255) / 256), 256, 0, x->stream>>>(N, p, x->p_pad, dperm, xraw, x->X);
    cudaFreeAsync(xraw, x->stream);
    cudaFreeAsync(dperm, x->stream);
    if (cudaGetLastError() != cudaSuccess) return bail(PCV_E_CUDA, "row gather failed");
  }
  cudaMemcpyAsync(x->y, hy.data(), hy.size() * sizeof(float), cudaMemcpyHostToDevice, x->stream);
  cudaMemcpyAsync(x->folds, fds.data(), fds.size() * sizeof(FoldDesc), cudaMemcpyHostToDevice, x->stream);
  if (x->tc) {
    // the operand copy of the design matrix: bf16 [N_pad x KP] (round to
    // nearest even), or for the TF32 form X [N_pad x KP] and X^T [PN x N_pad]
    // rounded to TF32; padding rows and columns stay 0.  y on the device
    // (zero-padded), which the Gaussian models fold into the eta_ref columns
    std::vector<float> hyc((size_t)x->N_pad, 0.0f);
    for (int64_t r = 0; r < N; ++r) hyc[r] = hy[r];
    if (!dalloc_n(x, &x->ycf, hyc.size()) || !dalloc_n(x, &x->theta_ref, (size_t)x->d_pad) ||
        !dalloc_n(x, &x->eta_half, (size_t)x->N_pad))
      return bail(PCV_E_OOM, "device allocation failed");
    const long long items = (long long)N * p;
    // logistic model: rows signed by 2 y - 1 (the kernel's residual and log
    // likelihood are written for that form)
    const float *ysign = x->kind == PCV_LOGISTIC ? x->y : nullptr;
    if (x->tc32) {
      if (!dalloc_n(x, &x->X32, (size_t)x->N_pad * x->KP) || !dalloc_n(x, &x->XT32, (size_t)x->PN * x->N_pad))
        return bail(PCV_E_OOM, "device allocation failed");
      cudaMemsetAsync(x->X32, 0, sizeof(float) * (size_t)x->N_pad * x->KP, x->stream);
      cudaMemsetAsync(x->XT32, 0, sizeof(float) * (size_t)x->PN * x->N_pad, x->stream);
      k_x_tf32<<<(unsigned)((items + 255) / 256), 256, 0, x->stream>>>(N, p, x->p_pad, x->KP, x->N_pad, x->X, ysign,
                                                                        x->X32, x->XT32);
    } else {
      if (!dalloc_n(x, &x->X16, (size_t)x->N_pad * x->KP)) return bail(PCV_E_OOM, "device allocation failed");
      k_x_bf16<<<(unsigned)((items + 255) / 256), 256, 0, x->stream>>>(N, p, x->p_pad, x->KP, x->X, ysign, x->X16);
    }
    cudaMemcpyAsync(x->ycf, hyc.data(), hyc.size() * sizeof(float), cudaMemcpyHostToDevice, x->stream);
    // no reference yet (eta_ref = 0): the folded columns hold -y / 2
    // (Gaussian models) or 0
    cudaMemsetAsync(x->eta_half, 0, sizeof(float) * x->N_pad, x->stream);
    if (fold_eta(x) != PCV_OK) return bail(PCV_E_CUDA, "upload failed");
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(x->stream) != cudaSuccess)
      return bail(PCV_E_CUDA, "upload failed");
    if (x->tc32 ? !(encode_f32_map(&x->tm_x, x->X32, x->N_pad, x->KP, 64) &&
                    encode_f32_map(&x->tm_xt, x->XT32, x->PN, x->N_pad, x->PN))
                : !encode_bf16_map(&x->tm_x, x->X16, x->N_pad, x->KP))
      return bail(PCV_E_CUDA, "cuTensorMapEncodeTiled failed for X");
    if (tc_prepare() != cudaSuccess) return bail(PCV_E_CUDA, "cudaFuncSetAttribute failed");
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&x->n_sm, cudaDevAttrMultiProcessorCount, dev);
  }
  std::vector<float> hm(x->d_pad, 1.0f);
  if (opt->inv_mass_diag)
    for (int j = 0; j < x->d; ++j) {
      if (!(opt->inv_mass_diag[j] > 0)) return bail(PCV_E_INVALID_ARG, "inverse mass must be > 0");
      hm[j] = (float)opt->inv_mass_diag[j];
    }
  if (model->active_covariates) {
    // covariate-selection mask: inactive coefficients are held at zero
    x->active_h.assign(x->d_pad, 1.0f);
    for (int j = 0; j < p; ++j) {
      const int32_t a = model->active_covariates[j];
      if (a != 0 && a != 1) return bail(PCV_E_INVALID_ARG, "active_covariates must hold 0 or 1");
      x->active_h[j] = (float)a;
      if (!a) hm[j] = 0.0f;
    }
    if (!dalloc_n(x, &x->active_d, (size_t)x->d_pad)) return bail(PCV_E_OOM, "device allocation failed");
    cudaMemcpyAsync(x->active_d, x->active_h.data(), sizeof(float) * x->d_pad, cudaMemcpyHostToDevice, x->stream);
  }
  if (x->pair) {
    // model B's mask: a subset of model A's covariates (B nested in A), so
    // that B's inverse mass is A's adapted one restricted to B's covariates
    x->active_b_h.assign(x->d_pad, 1.0f);
    for (int j = 0; j < p; ++j) {
      const int32_t a = model->active_covariates_b[j];
      if (a != 0 && a != 1) return bail(PCV_E_INVALID_ARG, "active_covariates_b must hold 0 or 1");
      if (a && !(x->active_h.empty() || x->active_h[j] > 0))
        return bail(PCV_E_INVALID_ARG, "active_covariates_b must select a subset of model A's covariates");
      x->active_b_h[j] = (float)a;
    }
    if (!dalloc_n(x, &x->active_b_d, (size_t)x->d_pad)) return bail(PCV_E_OOM, "device allocation failed");
    cudaMemcpyAsync(x->active_b_d, x->active_b_h.data(), sizeof(float) * x->d_pad, cudaMemcpyHostToDevice,
                    x->stream);
  }
  cudaMemcpyAsync(x->minv, hm.data(), hm.size() * sizeof(float), cudaMemcpyHostToDevice, x->stream);
  if (x->pair) {
    std::vector<float> hb(hm);
    for (int j = 0; j < x->d_pad; ++j) hb[j] *= x->active_b_h[j];
    cudaMemcpyAsync(x->minv + x->d_pad, hb.data(), hb.size() * sizeof(float), cudaMemcpyHostToDevice, x->stream);
  }
  if (x->variant == MV_HIER) {
    if (!dalloc_n(x, &x->seg_off, seg_off.size()) || !dalloc_n(x, &x->seg_grp, seg_grp.size()) ||
        !dalloc_n(x, &x->grp_seg, grp_seg.size()))
      return bail(PCV_E_OOM, "device allocation failed");
    cudaMemcpyAsync(x->seg_off, seg_off.data(), seg_off.size() * sizeof(int), cudaMemcpyHostToDevice, x->stream);
    cudaMemcpyAsync(x->seg_grp, seg_grp.data(), seg_grp.size() * sizeof(int), cudaMemcpyHostToDevice, x->stream);
    cudaMemcpyAsync(x->grp_seg, grp_seg.data(), grp_seg.size() * sizeof(int), cudaMemcpyHostToDevice, x->stream);
  }
  IterState hst{};
  hst.eps = opt->step_size > 0 ? (float)opt->step_size : 0.1f;
  hst.eps_iter = hst.eps;
  cudaMemcpyAsync(x->st, &hst, sizeof(hst), cudaMemcpyHostToDevice, x->stream);

  Problem &pb = x->pb;
  pb.variant = x->variant; pb.N = (int)N; pb.p = p; pb.p_pad = x->p_pad; pb.d = x->d; pb.d_pad = x->d_pad;
  pb.G = x->G; pb.K = x->K; pb.X = x->X; pb.y = x->y; pb.grp_off = x->seg_off; pb.folds = x->folds;
  pb.seg_grp = x->seg_grp; pb.grp_seg = x->grp_seg;
  pb.beta_prec = (float)(1.0 / (model->beta_prior_sd * model->beta_prior_sd));
  pb.log_beta_sd = (float)std::log(model->beta_prior_sd);
  pb.sigma_known = (float)(model->sigma_known > 0 ? model->sigma_known : 1.0);
  const double ssd = model->sigma_prior_sd > 0 ? model->sigma_prior_sd : 1.0;
  const double tsd = model->tau_prior_sd > 0 ? model->tau_prior_sd : 1.0;
  pb.sigma_prec = (float)(1.0 / (ssd * ssd));
  pb.log_sigma_sd = (float)std::log(ssd);
  pb.tau_prec = (float)(1.0 / (tsd * tsd));
  pb.log_tau_sd = (float)std::log(tsd);

  // whole trajectories in one launch for the flat models with p <= 32 (FP32
  // and the BF16 form, which reads a bf16 copy of X)
  x->traj_ok = opt->fused_trajectory != 0 && !x->tc32 && traj_small_supported(pb);
  if (x->traj_ok && x->tc) {   // (the BF16 form)
    const int PP = traj_small_row_width(p);
    const size_t n16 = ((size_t)N * PP + 7) / 8 * 8;     // whole 16-byte units (the kernel copies by 16 bytes)
    if (!dalloc_n(x, &x->X16c, n16)) return bail(PCV_E_OOM, "device allocation failed");
    cudaMemsetAsync(x->X16c, 0, n16 * sizeof(__nv_bfloat16), x->stream);
    const long long items = (long long)N * PP;
    k_x_bf16_compact<<<(unsigned)((items + 255) / 256), 256, 0, x->stream>>>(N, PP, x->p_pad, x->X, x->X16c);
    if (cudaGetLastError() != cudaSuccess) return bail(PCV_E_CUDA, "bf16 copy of X failed");
  }
  pcv_status s;
  if ((s = alloc_chains(x, x->fold_cb, x->C, x->L, 0)) != PCV_OK) return bail(s, x->err);
  // full-data chains: the fold descriptor after the last fold (no rows excluded)
  if ((s = alloc_chains(x, x->fd_cb, kNumFdChains, kNumFdChains, x->K)) != PCV_OK) return bail(s, x->err);
  if ((s = alloc_accum(x)) != PCV_OK) return bail(s, x->err);
  if (opt->extra_scores) {
    // Hyvarinen / Dawid-Sebastiani accumulators (Gaussian models whose rows
    // are conditionally independent given theta)
    if (opt->extra_scores & ~3) return bail(PCV_E_INVALID_ARG, "extra_scores: bits 0 (HS) and 1 (DSS) only");
    if (x->variant != MV_GAUSS_KNOWN && x->variant != MV_GAUSS_LOGSIG &&
        !(x->variant == MV_LOGISTIC && opt->extra_scores == 2))
      return bail(PCV_E_UNSUPPORTED, "HS needs a Gaussian linear or AR model; DSS a Gaussian or logistic one");
    int T = 0;
    for (int k = 0; k < K; ++k) T = std::max(T, fds[k].test_hi - fds[k].test_lo);
    if ((opt->extra_scores & 2) && T > 64) return bail(PCV_E_UNSUPPORTED, "DSS needs test sets of at most 64 rows");
    Extra &E = x->extra;
    E.flags = opt->extra_scores;
    E.T = T;
    const size_t C = (size_t)x->C;
    if (!dalloc_n(x, &E.hs1, C) || !dalloc_n(x, &E.hs2, C * T) || !dalloc_n(x, &E.dsum, C * T) ||
        !dalloc_n(x, &E.douter, C * T * T))
      return bail(PCV_E_OOM, "accumulator allocation failed");
  }
  if (x->tc) {
    if ((s = ensure_ws_tc(x, x->C)) != PCV_OK) return bail(s, x->err);
  } else {
    if ((s = ensure_ws(x, x->C, splits_for(x, x->C))) != PCV_OK) return bail(s, x->err);
    if ((s = ensure_ws(x, kNumFdChains, splits_for(x, kNumFdChains))) != PCV_OK) return bail(s, x->err);
  }
  if (cudaStreamSynchronize(x->stream) != cudaSuccess) return bail(PCV_E_CUDA, "upload failed");
  leave(x);
  *out = x;
  return PCV_OK;
}

pcv_status pcv_warmup(pcv_ctx *x, int32_t n_fd, int32_t n_wu) {
  if (!x) return PCV_E_INVALID_ARG;
  if (x->state != ST_CREATED) return fail(x, PCV_E_BAD_STATE, "pcv_warmup may be called once, before sampling");
  if (n_fd < 0 || n_wu < 0) return fail(x, PCV_E_INVALID_ARG, "negative iteration count");
  enter(x);
  const bool adapt = !(x->opt.step_size > 0);
  const float eps0 = adapt ? 0.1f : (float)x->opt.step_size;
  x->fd_n_adapt = n_fd;
  k_fd_init_state<<<1, 1, 0, x->stream>>>(x->st, eps0, adapt ? 1 : 0);
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(x->wmean, 0, sizeof(double) * x->d, x->stream));
  CK(cudaMemsetAsync(x->wM2, 0, sizeof(double) * x->d, x->stream));
  // full-data chains: init_scale * N(0, I) from stream ST_FD_INIT
  {
    const int nq = (x->d + 3) / 4;
    const long long T = (long long)kNumFdChains * nq;
    k_normals<<<(unsigned)((T + 255) / 256), 256, 0, x->stream>>>(
        kNumFdChains, x->d, x->d_pad, x->opt.seed, 0u, ST_FD_INIT, (float)x->opt.init_scale, x->fd_cb.theta);
    CK(cudaGetLastError());
    if (x->active_d) {
      const long long Tm = (long long)kNumFdChains * x->d;
      k_mask_positions<<<(unsigned)((Tm + 255) / 256), 256, 0, x->stream>>>(kNumFdChains, x->d, x->d_pad,
                                                                          x->active_d, x->fd_cb.theta);
      CK(cudaGetLastError());
    }
  }
  pcv_status s = refresh(x, x->fd_cb);
  if (s != PCV_OK) return s;
  if ((s = tune(x, x->fd_cb)) != PCV_OK) return s;
  s = run_iterations(x, x->fd_cb, true, false, n_fd, &x->g_fd_1, 1);
  if (s != PCV_OK) return s;
  if (adapt && n_fd > 0) {
    k_fd_final_eps<<<1, 1, 0, x->stream>>>(x->st, x->traj_len > 0 ? (float)(x->traj_len / x->Lf) : 0.0f);
    CK(cudaGetLastError());
  }
  s = run_iterations(x, x->fd_cb, true, false, x->n_fd_draws, &x->g_fd_1, 1);
  if (s != PCV_OK) return s;
  // tensor-core path: centre on the mean of the full-data draws
  s = set_reference(x, x->pool, x->n_fd_draws * kNumFdChains, x->d_pad);
  if (s != PCV_OK) return s;
  // two models: B's inverse mass from A's adaptation
  if ((s = sync_minv_b(x)) != PCV_OK) return s;
  // fold chains start from full-data draws (Algorithm 1); model B's chains
  // with B's inactive coefficients at 0
  {
    const long long T = (long long)x->C * x->d;
    k_init_from_pool<<<(unsigned)((T + 255) / 256), 256, 0, x->stream>>>(
        x->C, x->d, x->d_pad, x->opt.seed, x->pool, x->n_fd_draws * kNumFdChains, x->fold_cb.theta,
        x->chain_base);
    CK(cudaGetLastError());
    if (x->pair) {
      const int cb = x->K_model * x->L;
      const long long Tm = (long long)cb * x->d;
      k_mask_positions<<<(unsigned)((Tm + 255) / 256), 256, 0, x->stream>>>(
          cb, x->d, x->d_pad, x->active_b_d, x->fold_cb.theta + (size_t)cb * x->d_pad);
      CK(cudaGetLastError());
    }
  }
  s = refresh(x, x->fold_cb);
  if (s != PCV_OK) return s;
  if ((s = tune(x, x->fold_cb)) != PCV_OK) return s;
  s = run_iterations(x, x->fold_cb, false, false, n_wu, &x->g_fold_1, 1);
  if (s != PCV_OK) return s;
  CK(cudaStreamSynchronize(x->stream));
  {
    unsigned int derr = 0;
    CK(cudaMemcpy(&derr, &x->st->error, sizeof(derr), cudaMemcpyDeviceToHost));
    if (derr) return fail(x, PCV_E_TIMEOUT, "a device-side wait timed out (error flags " + std::to_string(derr) + ")");
  }
  leave(x);
  x->state = ST_WARMED;
  return PCV_OK;
}

pcv_status pcv_sample(pcv_ctx *x, int32_t n_draws) {
  if (!x) return PCV_E_INVALID_ARG;
  if (x->state == ST_CREATED) return fail(x, PCV_E_BAD_STATE, "pcv_sample before pcv_warmup / pcv_set_positions");
  if (n_draws <= 0 || n_draws % x->b != 0)
    return fail(x, PCV_E_INVALID_ARG, "n_draws must be a positive multiple of batch_size");
  if ((x->n_sampled + n_draws) / x->b > x->max_batches)
    return fail(x, PCV_E_INVALID_ARG, "more batches than max_batches");
  enter(x);
  pcv_status s = tune(x, x->fold_cb);               // outside the timed region
  if (s != PCV_OK) return s;
  CK(cudaEventRecord(x->ev0, x->stream));
  s = run_iterations(x, x->fold_cb, false, true, n_draws, &x->g_sample_b, x->b);
  if (s != PCV_OK) return s;
  CK(cudaEventRecord(x->ev1, x->stream));
  CK(cudaEventSynchronize(x->ev1));
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, x->ev0, x->ev1);
  x->last_ms = ms;
  {
    unsigned int derr = 0;
    CK(cudaMemcpy(&derr, &x->st->error, sizeof(derr), cudaMemcpyDeviceToHost));
    if (derr) return fail(x, PCV_E_TIMEOUT, "a device-side wait timed out (error flags " + std::to_string(derr) + ")");
  }
  x->n_sampled += n_draws;
  x->finalized = false;
  x->state = ST_SAMPLED;
  leave(x);
  return PCV_OK;
}

pcv_status pcv_scores(pcv_ctx *x, double *elpd_k, double *mcse_k, double *elpd_total, double *mcse_total,
                      double *se_epistemic) {
  if (!x) return PCV_E_INVALID_ARG;
  if (x->state != ST_SAMPLED) return fail(x, PCV_E_BAD_STATE, "pcv_scores before pcv_sample");
  pcv_status s = finalize(x);
  if (s != PCV_OK) return s;
  for (int k = 0; k < x->K; ++k) {
    if (elpd_k) elpd_k[k] = x->h_fold[(size_t)k * F_NFIELDS + F_ELPD];
    if (mcse_k) mcse_k[k] = x->h_fold[(size_t)k * F_NFIELDS + F_MCSE];
  }
  if (elpd_total) *elpd_total = x->h_tot[T_ELPD];
  if (mcse_total) *mcse_total = x->h_tot[T_MCSE];
  if (se_epistemic) *se_epistemic = x->h_tot[T_SEEPI];
  return PCV_OK;
}

pcv_status pcv_diagnostics(pcv_ctx *x, double *rhat_k, double *split_rhat_k, double *ess_bm_k,
                           double *ess_acov_k, int64_t *divergences_k, double *rhat_max, double *ess_total) {
  if (!x) return PCV_E_INVALID_ARG;
  if (x->state != ST_SAMPLED) return fail(x, PCV_E_BAD_STATE, "pcv_diagnostics before pcv_sample");
  pcv_status s = finalize(x);
  if (s != PCV_OK) return s;
  for (int k = 0; k < x->K; ++k) {
    const double *o = &x->h_fold[(size_t)k * F_NFIELDS];
    if (rhat_k) rhat_k[k] = o[F_RHAT];
    if (split_rhat_k) split_rhat_k[k] = o[F_SRHAT];
    if (ess_bm_k) ess_bm_k[k] = o[F_ESSBM];
    if (ess_acov_k) ess_acov_k[k] = o[F_ESSAC];
    if (divergences_k) divergences_k[k] = (int64_t)o[F_DIV];
  }
  if (rhat_max) *rhat_max = x->h_tot[T_RHATMAX];
  if (ess_total) *ess_total = x->h_tot[T_ESSTOT];
  return PCV_OK;
}

int32_t pcv_num_folds(const pcv_ctx *x) { return x ? x->K : -1; }
int32_t pcv_num_chains(const pcv_ctx *x) { return x ? x->C : -1; }
int32_t pcv_dim(const pcv_ctx *x) { return x ? x->d : -1; }
const char *pcv_last_error(const pcv_ctx *x) { return x ? x->err.c_str() : create_error().c_str(); }

void pcv_destroy(pcv_ctx *x) {
  if (!x) return;
  free_all(x);
  for (cudaGraphExec_t g : {x->g_sample_b, x->g_fold_1, x->g_fd_1})
    if (g) cudaGraphExecDestroy(g);
  for (cudaEvent_t e : {x->ev_in, x->ev_out, x->ev0, x->ev1})
    if (e) cudaEventDestroy(e);
  if (x->own_stream && x->stream) cudaStreamDestroy(x->stream);
  delete x;
}

pcv_status pcv_set_positions(pcv_ctx *x, const double *theta, double step_size, const double *inv_mass) {
  if (!x || !theta) return fail(x, PCV_E_INVALID_ARG, "null argument");
  if (x->state == ST_SAMPLED) return fail(x, PCV_E_BAD_STATE, "positions cannot be reset after sampling");
  enter(x);
  std::vector<float> h((size_t)x->C * x->d_pad, 0.0f);
  for (int c = 0; c < x->C; ++c)
    for (int j = 0; j < x->d; ++j) {
      const double v = theta[(size_t)c * x->d + j];
      if (!std::isfinite(v)) return fail(x, PCV_E_NUMERIC, "non-finite position");
      // masked coefficients (the chain's model's mask) are held at 0
      const bool in_b = x->pair && c >= x->K_model * x->L;
      const float m = in_b ? x->active_b_h[j] : x->active_d ? x->active_h[j] : 1.0f;
      h[(size_t)c * x->d_pad + j] = (float)v * m;
    }
  CK(cudaMemcpyAsync(x->fold_cb.theta, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, x->stream));
  {
    // tensor-core path: centre on the mean of the given positions
    pcv_status sr = set_reference(x, x->fold_cb.theta, x->C, x->d_pad);
    if (sr != PCV_OK) return sr;
  }
  if (step_size > 0) {
    const float e[2] = {(float)step_size, (float)step_size};   // eps, eps_iter
    static_assert(offsetof(IterState, eps_iter) == offsetof(IterState, eps) + sizeof(float), "layout");
    CK(cudaMemcpyAsync(&x->st->eps, e, sizeof(e), cudaMemcpyHostToDevice, x->stream));
  }
  if (inv_mass) {
    std::vector<float> hm(x->d_pad, 1.0f);
    for (int j = 0; j < x->d; ++j) {
      if (!(inv_mass[j] > 0)) return fail(x, PCV_E_INVALID_ARG, "inverse mass must be > 0");
      hm[j] = (float)inv_mass[j] * (x->active_d ? x->active_h[j] : 1.0f);
    }
    CK(cudaMemcpyAsync(x->minv, hm.data(), hm.size() * sizeof(float), cudaMemcpyHostToDevice, x->stream));
    pcv_status sb = sync_minv_b(x);
    if (sb != PCV_OK) return sb;
  }
  pcv_status s = refresh(x, x->fold_cb);
  if (s != PCV_OK) return s;
  CK(cudaStreamSynchronize(x->stream));
  leave(x);
  x->state = ST_WARMED;
  return PCV_OK;
}

pcv_status pcv_get_positions(pcv_ctx *x, double *theta, double *logp, double *shat) {
  if (!x) return PCV_E_INVALID_ARG;
  enter(x);
  std::vector<float> h((size_t)x->C * x->d_pad);
  std::vector<double> lp(x->C), sh(x->C);
  CK(cudaMemcpyAsync(h.data(), x->fold_cb.theta, h.size() * sizeof(float), cudaMemcpyDeviceToHost, x->stream));
  CK(cudaMemcpyAsync(lp.data(), x->fold_cb.logp, lp.size() * sizeof(double), cudaMemcpyDeviceToHost, x->stream));
  CK(cudaMemcpyAsync(sh.data(), x->fold_cb.shat, sh.size() * sizeof(double), cudaMemcpyDeviceToHost, x->stream));
  CK(cudaStreamSynchronize(x->stream));
  leave(x);
  for (int c = 0; c < x->C; ++c) {
    if (theta)
      for (int j = 0; j < x->d; ++j) theta[(size_t)c * x->d + j] = h[(size_t)c * x->d_pad + j];
    if (logp) logp[c] = lp[c];
    if (shat) shat[c] = sh[c];
  }
  return PCV_OK;
}

pcv_status pcv_get_adaptation(pcv_ctx *x, double *step_size, double *inv_mass) {
  if (!x) return PCV_E_INVALID_ARG;
  enter(x);
  IterState hs;
  std::vector<float> hm(x->d_pad);
  CK(cudaMemcpyAsync(&hs, x->st, sizeof(hs), cudaMemcpyDeviceToHost, x->stream));
  CK(cudaMemcpyAsync(hm.data(), x->minv, hm.size() * sizeof(float), cudaMemcpyDeviceToHost, x->stream));
  CK(cudaStreamSynchronize(x->stream));
  leave(x);
  if (step_size) *step_size = hs.eps;
  if (inv_mass)
    for (int j = 0; j < x->d; ++j) inv_mass[j] = hm[j];
  return PCV_OK;
}

pcv_status pcv_get_pool(pcv_ctx *x, double *pool, int32_t *n_pool) {
  if (!x || !n_pool) return fail(x, PCV_E_INVALID_ARG, "null argument");
  if (x->state == ST_CREATED) return fail(x, PCV_E_BAD_STATE, "the pool is filled by pcv_warmup");
  const int n = x->n_fd_draws * kNumFdChains;
  *n_pool = n;
  if (!pool) return PCV_OK;
  enter(x);
  std::vector<float> h((size_t)n * x->d_pad);
  CK(cudaMemcpyAsync(h.data(), x->pool, h.size() * sizeof(float), cudaMemcpyDeviceToHost, x->stream));
  CK(cudaStreamSynchronize(x->stream));
  leave(x);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < x->d; ++j) pool[(size_t)i * x->d + j] = h[(size_t)i * x->d_pad + j];
  return PCV_OK;
}

pcv_status pcv_adapt_trace(pcv_ctx *x, int32_t n_adapt, const double *accept, const float *draws, double eps0,
                           int32_t adapt_mass, double *eps_out, double *minv_out, double *eps_final) {
  if (!x) return PCV_E_INVALID_ARG;
  if (!accept || !draws || !eps_out || !minv_out || !eps_final || n_adapt < 1 || !(eps0 > 0))
    return fail(x, PCV_E_INVALID_ARG, "bad argument");
  if (x->state != ST_CREATED) return fail(x, PCV_E_BAD_STATE, "pcv_adapt_trace runs before pcv_warmup");
  enter(x);
  const int nc = kNumFdChains, d = x->d, ld = x->d_pad;
  ChainBufs &cb = x->fd_cb;
  // the context's inverse mass is restored afterwards
  std::vector<float> minv_keep(ld);
  CK(cudaMemcpyAsync(minv_keep.data(), x->minv, sizeof(float) * ld, cudaMemcpyDeviceToHost, x->stream));
  k_fd_init_state<<<1, 1, 0, x->stream>>>(x->st, (float)eps0, 1);
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(x->wmean, 0, sizeof(double) * d, x->stream));
  CK(cudaMemsetAsync(x->wM2, 0, sizeof(double) * d, x->stream));
  FdAdaptArgs fa{};
  fa.st = x->st;
  fa.n_adapt = n_adapt;
  fa.w0 = n_adapt / 4;
  fa.w1 = n_adapt / 2;
  fa.w2 = (7 * n_adapt) / 8;
  fa.adapt_eps = 1;
  fa.adapt_mass = adapt_mass ? 1 : 0;
  fa.C = nc; fa.d = d; fa.ld = ld;
  fa.theta = cb.theta;
  fa.accept_prob = cb.accept_prob;
  fa.minv = x->minv;
  fa.wmean = x->wmean; fa.wM2 = x->wM2;
  fa.pool = x->pool;
  fa.active = x->active_d;
  fa.n_keep = 0;
  std::vector<float> th((size_t)nc * ld, 0.0f), hm(ld);
  for (int i = 0; i < n_adapt; ++i) {
    for (int c = 0; c < nc; ++c)
      for (int j = 0; j < d; ++j) th[(size_t)c * ld + j] = draws[((size_t)i * nc + c) * d + j];
    const unsigned it = (unsigned)i + 1;      // the adaptation reads "the iteration just completed"
    CK(cudaMemcpyAsync(cb.theta, th.data(), th.size() * sizeof(float), cudaMemcpyHostToDevice, x->stream));
    CK(cudaMemcpyAsync(cb.accept_prob, accept + (size_t)i * nc, sizeof(double) * nc, cudaMemcpyHostToDevice,
                       x->stream));
    CK(cudaMemcpyAsync(&x->st->fd_iter, &it, sizeof(it), cudaMemcpyHostToDevice, x->stream));
    k_fd_adapt<<<1, 128, 0, x->stream>>>(fa);
    CK(cudaGetLastError());
    IterState hs;
    CK(cudaMemcpyAsync(&hs, x->st, sizeof(hs), cudaMemcpyDeviceToHost, x->stream));
    CK(cudaMemcpyAsync(hm.data(), x->minv, sizeof(float) * ld, cudaMemcpyDeviceToHost, x->stream));
    CK(cudaStreamSynchronize(x->stream));
    eps_out[i] = hs.eps;
    for (int j = 0; j < d; ++j) minv_out[(size_t)i * d + j] = hm[j];
  }
  k_fd_final_eps<<<1, 1, 0, x->stream>>>(x->st, 0.0f);
  CK(cudaGetLastError());
  IterState hs;
  CK(cudaMemcpyAsync(&hs, x->st, sizeof(hs), cudaMemcpyDeviceToHost, x->stream));
  CK(cudaMemcpyAsync(x->minv, minv_keep.data(), sizeof(float) * ld, cudaMemcpyHostToDevice, x->stream));
  CK(cudaStreamSynchronize(x->stream));
  *eps_final = hs.eps;
  leave(x);
  return PCV_OK;
}

pcv_status pcv_log_density(pcv_ctx *x, const float *theta, const int32_t *fold, int32_t n, int32_t precision,
                           double *logp, float *grad, double *shat) {
  if (!x) return PCV_E_INVALID_ARG;
  if (!theta || !fold || !logp || !grad || !shat || n < 1) return fail(x, PCV_E_INVALID_ARG, "bad argument");
  if (precision != x->opt.precision)
    return fail(x, PCV_E_UNSUPPORTED, "precision not available for this context");
  enter(x);
  ChainBufs cb;
  cb.C = n; cb.L = 1; cb.fold_base = 0;
  if (x->tc) {
    if (n > x->ld_cap) {                     // grow the shadow buffers of evaluated positions
      pcv_status s0 = alloc_shadows(x, x->ld_cb, n);
      if (s0 != PCV_OK) return s0;
      x->ld_cap = x->ld_cb.C_pad;
    }
    cb.C_pad = x->ld_cb.C_pad; cb.shadow_hi = x->ld_cb.shadow_hi; cb.shadow_lo = x->ld_cb.shadow_lo;
    cb.shadow32 = x->ld_cb.shadow32;
    cb.tm_hi = x->ld_cb.tm_hi; cb.tm_lo = x->ld_cb.tm_lo;
    pcv_status s0 = write_shadow(x, cb, theta, x->d);
    if (s0 != PCV_OK) return s0;
  }
  GradArgs a = grad_args(x, cb, false);
  a.fold_of = fold;
  a.theta = theta; a.ld_theta = x->d;
  a.grad = grad; a.ld_grad = x->d;
  a.logp = logp; a.shat = shat;
  a.need_ll = 1;
  a.mode = MODE_NONE;
  a.r = nullptr;
  pcv_status s = launch_grad(x, a, &cb);
  if (s != PCV_OK) return s;
  leave(x);
  return PCV_OK;
}

pcv_status pcv_trajectory(pcv_ctx *x, const float *theta0, const float *r0, int32_t precision, float *theta1,
                          float *r1, double *logp1, double *shat1) {
  if (!x) return PCV_E_INVALID_ARG;
  if (!theta0 || !r0 || !theta1 || !r1 || !logp1 || !shat1) return fail(x, PCV_E_INVALID_ARG, "null argument");
  if (precision != x->opt.precision)
    return fail(x, PCV_E_UNSUPPORTED, "precision not available for this context");
  enter(x);
  if (!x->traj_cb.theta) {
    pcv_status s = alloc_chains(x, x->traj_cb, x->C, x->L, 0);
    if (s != PCV_OK) return s;
    if (!dalloc_n(x, &x->rstart, (size_t)x->C * x->d_pad)) return fail(x, PCV_E_OOM, "allocation failed");
  }
  ChainBufs &cb = x->traj_cb;
  float *rstart = x->rstart;
  const size_t row = sizeof(float) * x->d, pitch = sizeof(float) * x->d_pad;
  CK(cudaMemcpy2DAsync(cb.theta, pitch, theta0, row, row, x->C, cudaMemcpyDeviceToDevice, x->stream));
  CK(cudaMemcpy2DAsync(rstart, pitch, r0, row, row, x->C, cudaMemcpyDeviceToDevice, x->stream));
  pcv_status s = refresh(x, cb);
  if (s != PCV_OK) return s;
  s = launch_proposal(x, cb, false, rstart, 0.0f);
  if (s != PCV_OK) return s;
  CK(cudaMemcpy2DAsync(theta1, row, cb.theta_p, pitch, row, x->C, cudaMemcpyDeviceToDevice, x->stream));
  CK(cudaMemcpy2DAsync(r1, row, cb.r, pitch, row, x->C, cudaMemcpyDeviceToDevice, x->stream));
  CK(cudaMemcpyAsync(logp1, cb.logp_p, sizeof(double) * x->C, cudaMemcpyDeviceToDevice, x->stream));
  CK(cudaMemcpyAsync(shat1, cb.shat_p, sizeof(double) * x->C, cudaMemcpyDeviceToDevice, x->stream));
  CK(cudaStreamSynchronize(x->stream));
  leave(x);
  return PCV_OK;
}

pcv_status pcv_draw_normals(pcv_ctx *x, uint32_t iteration, uint32_t stream, float *out) {
  if (!x) return PCV_E_INVALID_ARG;
  if (!out) return fail(x, PCV_E_INVALID_ARG, "null argument");
  enter(x);
  const int nq = (x->d + 3) / 4;
  const long long T = (long long)x->C * nq;
  k_normals<<<(unsigned)((T + 255) / 256), 256, 0, x->stream>>>(x->C, x->d, x->d, x->opt.seed, iteration,
                                                                stream, 1.0f, out);
  CK(cudaGetLastError());
  leave(x);
  return PCV_OK;
}

pcv_status pcv_accumulate(pcv_ctx *x, const double *shat, int32_t n) {
  if (!x) return PCV_E_INVALID_ARG;
  if (!shat || n <= 0 || n % x->b != 0) return fail(x, PCV_E_INVALID_ARG, "n must be a positive multiple of batch_size");
  if (x->state == ST_CREATED) return fail(x, PCV_E_BAD_STATE, "accumulate before positions are set");
  if ((x->n_sampled + n) / x->b > x->max_batches) return fail(x, PCV_E_INVALID_ARG, "more batches than max_batches");
  enter(x);
  k_accumulate_given<<<(x->C + kAccChains - 1) / kAccChains, kAccChains * 32, 0, x->stream>>>(x->acc, shat, n,
                                                                                              x->n_sampled);
  CK(cudaGetLastError());
  x->n_sampled += n;
  const long long nd = x->n_sampled;
  CK(cudaMemcpyAsync(&x->st->n_draws, &nd, sizeof(nd), cudaMemcpyHostToDevice, x->stream));
  CK(cudaStreamSynchronize(x->stream));
  leave(x);
  x->finalized = false;
  x->state = ST_SAMPLED;
  return PCV_OK;
}

pcv_status pcv_get_draws(pcv_ctx *x, double *shat, int32_t *n_stored) {
  if (!x) return PCV_E_INVALID_ARG;
  if (!x->acc.draws) return fail(x, PCV_E_BAD_STATE, "store_draws was not enabled");
  const int n = (int)std::min<long long>(x->n_sampled, x->acc.draw_cap);
  if (n_stored) *n_stored = n;
  if (!shat) return PCV_OK;
  enter(x);
  std::vector<double> h((size_t)x->C * x->acc.draw_cap);
  CK(cudaMemcpyAsync(h.data(), x->acc.draws, h.size() * sizeof(double), cudaMemcpyDeviceToHost, x->stream));
  CK(cudaStreamSynchronize(x->stream));
  leave(x);
  for (int c = 0; c < x->C; ++c)
    std::memcpy(shat + (size_t)c * n, &h[(size_t)c * x->acc.draw_cap], sizeof(double) * n);
  return PCV_OK;
}

pcv_status pcv_accept_rate(pcv_ctx *x, double *accept_k) {
  if (!x || !accept_k) return fail(x, PCV_E_INVALID_ARG, "null argument");
  if (x->state != ST_SAMPLED) return fail(x, PCV_E_BAD_STATE, "no draws yet");
  pcv_status s = finalize(x);
  if (s != PCV_OK) return s;
  for (int k = 0; k < x->K; ++k) accept_k[k] = x->h_fold[(size_t)k * F_NFIELDS + F_ACCRATE];
  return PCV_OK;
}

pcv_status pcv_time_leapfrog_kernel(pcv_ctx *x, int32_t reps, double *ms_per_launch) {
  if (!x || !ms_per_launch || reps < 1) return fail(x, PCV_E_INVALID_ARG, "bad argument");
  if (x->state == ST_CREATED) return fail(x, PCV_E_BAD_STATE, "positions not set");
  enter(x);
  ChainBufs &cb = x->fold_cb;
  {
    pcv_status st = tune(x, cb);
    if (st != PCV_OK) return st;
  }
  const size_t n = sizeof(float) * (size_t)cb.C * x->d_pad;
  CK(cudaMemcpyAsync(cb.theta_p, cb.theta, n, cudaMemcpyDeviceToDevice, x->stream));
  CK(cudaMemsetAsync(cb.r, 0, n, x->stream));
  pcv_status s = write_shadow(x, cb, cb.theta_p, x->d_pad);
  if (s != PCV_OK) return s;
  GradArgs ga = grad_args(x, cb, true);
  ga.mode = MODE_KICK_DRIFT;
  ga.need_ll = 0;
  s = launch_grad(x, ga, &cb);                            // warm-up launch
  if (s != PCV_OK) return s;
  CK(cudaEventRecord(x->ev0, x->stream));
  for (int i = 0; i < reps; ++i) {
    s = launch_grad(x, ga, &cb);
    if (s != PCV_OK) return s;
  }
  CK(cudaEventRecord(x->ev1, x->stream));
  CK(cudaEventSynchronize(x->ev1));
  float ms = 0.0f;
  CK(cudaEventElapsedTime(&ms, x->ev0, x->ev1));
  *ms_per_launch = ms / reps;
  leave(x);
  return PCV_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint / resume: the O(C) state that the next iterations read, in a
// fixed order behind a header that identifies the problem and the options.
// ---------------------------------------------------------------------------
namespace {
struct CkptHeader {
  char magic[8];
  int32_t version;
  int32_t precision, variant, p, d, d_pad, K, L, C, M, max_batches, b, draw_cap, Lf, N_pad;
  int64_t N;
  uint64_t seed;
  int64_t n_sampled;
  int32_t state, centered;
  int32_t tuned_splits, tuned_ns0, tuned_ns1, tuned_ncta, tuned_fused;
  int32_t first_fold;
  float jitter;
  double traj_len;
  int64_t payload;
};
constexpr char kCkptMagic[8] = {'P', 'C', 'V', 'C', 'K', 'P', 'T', '1'};

struct Seg { void *dev; size_t bytes; };

std::vector<Seg> ckpt_segments(pcv_ctx *x) {
  const size_t C = (size_t)x->C;
  std::vector<Seg> v;
  Accum &A = x->acc;
  v.push_back({x->st, sizeof(IterState)});
  v.push_back({x->minv, sizeof(float) * x->d_pad * (x->pair ? 2 : 1)});
  v.push_back({x->fold_cb.theta, sizeof(float) * C * x->d_pad});
  v.push_back({x->fold_cb.grad, sizeof(float) * C * x->d_pad});
  v.push_back({x->fold_cb.logp, sizeof(double) * C});
  v.push_back({x->fold_cb.shat, sizeof(double) * C});
  if (x->tc) {
    v.push_back({x->theta_ref, sizeof(float) * x->d_pad});
    v.push_back({x->eta_half, sizeof(float) * x->N_pad});
  }
  for (double *p : {A.Ux, A.Ux2, A.Zx, A.em, A.emean, A.eM2, A.vm, A.vmean, A.vM2, A.wmean, A.wM2,
                    A.bmean_cur, A.bM2_cur, A.c0, A.xsum})
    v.push_back({p, sizeof(double) * C});
  v.push_back({A.bmean, sizeof(double) * C * x->max_batches});
  v.push_back({A.bM2, sizeof(double) * C * x->max_batches});
  v.push_back({A.lagsum, sizeof(double) * C * (x->M + 1)});
  v.push_back({A.first, sizeof(double) * C * std::max(1, x->M)});
  v.push_back({A.ring, sizeof(double) * C * std::max(1, x->M)});
  v.push_back({A.div, sizeof(long long) * C});
  v.push_back({A.acc, sizeof(long long) * C});
  if (A.draw_cap > 0) v.push_back({A.draws, sizeof(double) * C * A.draw_cap});
  if (x->extra.flags) {
    const size_t T = (size_t)x->extra.T;
    v.push_back({x->extra.hs1, sizeof(double) * C});
    v.push_back({x->extra.hs2, sizeof(double) * C * T});
    v.push_back({x->extra.dsum, sizeof(double) * C * T});
    v.push_back({x->extra.douter, sizeof(double) * C * T * T});
  }
  return v;
}

CkptHeader ckpt_header(pcv_ctx *x) {
  CkptHeader h{};
  std::memcpy(h.magic, kCkptMagic, 8);
  h.version = 3;
  h.precision = x->opt.precision; h.variant = x->variant; h.p = x->p; h.d = x->d; h.d_pad = x->d_pad;
  h.K = x->K; h.L = x->L; h.C = x->C; h.M = x->M; h.max_batches = x->max_batches; h.b = x->b;
  h.draw_cap = x->acc.draw_cap; h.Lf = x->Lf; h.N_pad = x->N_pad; h.N = x->N; h.seed = x->opt.seed;
  h.jitter = x->jitter; h.traj_len = x->traj_len; h.first_fold = x->opt.first_fold;
  size_t payload = 0;
  for (const Seg &g : ckpt_segments(x)) payload += g.bytes;
  h.payload = (int64_t)payload;
  return h;
}
}  // namespace

pcv_status pcv_checkpoint_size(pcv_ctx *x, int64_t *bytes) {
  if (!x) return PCV_E_INVALID_ARG;
  if (!bytes) return fail(x, PCV_E_INVALID_ARG, "null argument");
  *bytes = (int64_t)sizeof(CkptHeader) + ckpt_header(x).payload;
  return PCV_OK;
}

pcv_status pcv_checkpoint_save(pcv_ctx *x, void *buf, int64_t bytes) {
  if (!x) return PCV_E_INVALID_ARG;
  if (!buf) return fail(x, PCV_E_INVALID_ARG, "null buffer");
  if (x->state == ST_CREATED) return fail(x, PCV_E_BAD_STATE, "nothing to checkpoint before warm-up");
  CkptHeader h = ckpt_header(x);
  if (bytes < (int64_t)sizeof(h) + h.payload) return fail(x, PCV_E_INVALID_ARG, "checkpoint buffer too small");
  h.n_sampled = x->n_sampled;
  h.state = x->state;
  h.centered = x->centered ? 1 : 0;
  auto ts = x->tuned_splits.find(x->C);
  h.tuned_splits = ts != x->tuned_splits.end() ? ts->second : -1;
  auto n0 = x->tuned_ns.find(std::make_pair(x->C, 0)), n1 = x->tuned_ns.find(std::make_pair(x->C, 1));
  h.tuned_ns0 = n0 != x->tuned_ns.end() ? n0->second : -1;
  h.tuned_ns1 = n1 != x->tuned_ns.end() ? n1->second : -1;
  auto nc = x->tuned_ncta.find(x->C);
  h.tuned_ncta = nc != x->tuned_ncta.end() ? nc->second : -1;
  auto tf = x->tuned_fused.find(x->C);
  h.tuned_fused = tf != x->tuned_fused.end() ? tf->second : -1;
  enter(x);
  uint8_t *out = static_cast<uint8_t *>(buf);
  std::memcpy(out, &h, sizeof(h));
  size_t off = sizeof(h);
  for (const Seg &g : ckpt_segments(x)) {
    CK(cudaMemcpyAsync(out + off, g.dev, g.bytes, cudaMemcpyDeviceToHost, x->stream));
    off += g.bytes;
  }
  CK(cudaStreamSynchronize(x->stream));
  leave(x);
  return PCV_OK;
}

pcv_status pcv_checkpoint_load(pcv_ctx *x, const void *buf, int64_t bytes) {
  if (!x) return PCV_E_INVALID_ARG;
  if (!buf || bytes < (int64_t)sizeof(CkptHeader)) return fail(x, PCV_E_INVALID_ARG, "no checkpoint");
  CkptHeader h;
  std::memcpy(&h, buf, sizeof(h));
  const CkptHeader mine = ckpt_header(x);
  if (std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != 3)
    return fail(x, PCV_E_INVALID_ARG, "not a PCV checkpoint");
  if (h.precision != mine.precision || h.variant != mine.variant || h.p != mine.p || h.d != mine.d ||
      h.K != mine.K || h.L != mine.L || h.C != mine.C || h.M != mine.M || h.max_batches != mine.max_batches ||
      h.b != mine.b || h.draw_cap != mine.draw_cap || h.Lf != mine.Lf || h.N != mine.N || h.seed != mine.seed ||
      h.jitter != mine.jitter || h.traj_len != mine.traj_len || h.payload != mine.payload ||
      h.first_fold != mine.first_fold)
    return fail(x, PCV_E_INVALID_ARG, "the checkpoint belongs to another problem or other options");
  if (bytes < (int64_t)sizeof(h) + h.payload) return fail(x, PCV_E_INVALID_ARG, "truncated checkpoint");
  if (h.state != ST_WARMED && h.state != ST_SAMPLED) return fail(x, PCV_E_INVALID_ARG, "bad checkpoint state");
  enter(x);
  const uint8_t *in = static_cast<const uint8_t *>(buf);
  size_t off = sizeof(h);
  for (const Seg &g : ckpt_segments(x)) {
    CK(cudaMemcpyAsync(g.dev, in + off, g.bytes, cudaMemcpyHostToDevice, x->stream));
    off += g.bytes;
  }
  x->n_sampled = h.n_sampled;
  x->state = h.state;
  x->finalized = false;
  x->centered = h.centered != 0;
  if (h.tuned_splits > 0) x->tuned_splits[x->C] = h.tuned_splits;
  if (h.tuned_ns0 > 0) x->tuned_ns[std::make_pair(x->C, 0)] = h.tuned_ns0;
  if (h.tuned_ns1 > 0) x->tuned_ns[std::make_pair(x->C, 1)] = h.tuned_ns1;
  if (h.tuned_ncta > 0) x->tuned_ncta[x->C] = h.tuned_ncta;
  if (h.tuned_fused >= 0) x->tuned_fused[x->C] = h.tuned_fused;
  // the bf16 shadows and the eta_ref columns of X follow from the restored
  // positions and reference
  pcv_status s = write_shadow(x, x->fold_cb, x->fold_cb.theta, x->d_pad);
  if (s != PCV_OK) return s;
  if (x->tc && (s = fold_eta(x)) != PCV_OK) return s;
  CK(cudaStreamSynchronize(x->stream));
  leave(x);
  return PCV_OK;
}

pcv_status pcv_scores_extra(pcv_ctx *x, double *hs_k, double *dss_k, double *hs_total, double *dss_total) {
  if (!x) return PCV_E_INVALID_ARG;
  if (!x->extra.flags) return fail(x, PCV_E_UNSUPPORTED, "extra_scores was not enabled");
  if (x->state != ST_SAMPLED || x->n_sampled < 2) return fail(x, PCV_E_BAD_STATE, "pcv_scores_extra before pcv_sample");
  const int K = x->K, T = x->extra.T;
  if (!x->extra_out && !dalloc_n(x, &x->extra_out, (size_t)2 * K)) return fail(x, PCV_E_OOM, "allocation failed");
  enter(x);
  const size_t smem = sizeof(double) * ((size_t)T * T + 2 * (size_t)T);
  k_extra_finalize<<<K, 128, smem, x->stream>>>(x->pb, x->extra, K, x->L, (double)x->L * (double)x->n_sampled,
                                              x->extra_out, x->extra_out + K);
  CK(cudaGetLastError());
  std::vector<double> h((size_t)2 * K);
  CK(cudaMemcpyAsync(h.data(), x->extra_out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, x->stream));
  CK(cudaStreamSynchronize(x->stream));
  leave(x);
  double th = 0.0, td = 0.0;
  for (int k = 0; k < K; ++k) { th += h[k]; td += h[K + k]; }
  const bool has_hs = x->extra.flags & 1, has_dss = x->extra.flags & 2;
  if (hs_k && has_hs) std::memcpy(hs_k, h.data(), sizeof(double) * K);
  if (dss_k && has_dss) std::memcpy(dss_k, h.data() + K, sizeof(double) * K);
  if (hs_total) *hs_total = has_hs ? th : NAN;
  if (dss_total) *dss_total = has_dss ? td : NAN;
  return PCV_OK;
}

pcv_status pcv_compare(pcv_ctx *a, pcv_ctx *b, double *delta_k, double *mcse_k, double *out) {
  if (!a || !b) return PCV_E_INVALID_ARG;
  pcv_ctx *x = a;   // the context that reports errors (CK)
  if (!delta_k || !mcse_k || !out) return fail(a, PCV_E_INVALID_ARG, "null argument");
  if (a->N != b->N || a->K != b->K) return fail(a, PCV_E_INVALID_ARG, "the two contexts have different data or folds");
  if (a->state != ST_SAMPLED || b->state != ST_SAMPLED) return fail(a, PCV_E_BAD_STATE, "pcv_compare before pcv_sample");
  pcv_status s = finalize(b);
  if (s != PCV_OK) return fail(a, s, std::string("model B: ") + b->err);
  enter(a);
  if ((s = finalize(a)) != PCV_OK) return s;
  const int K = a->K;
  if ((size_t)(2 * K + 4) > a->cmp_n) {
    if (!dalloc_n(a, &a->cmp_out, (size_t)(2 * K + 4))) return fail(a, PCV_E_OOM, "allocation failed");
    a->cmp_n = (size_t)(2 * K + 4);
  }
  k_compare<<<1, 256, 0, a->stream>>>(a->fold_out, b->fold_out, K, a->cmp_out);
  CK(cudaGetLastError());
  std::vector<double> h((size_t)(2 * K + 4));
  CK(cudaMemcpyAsync(h.data(), a->cmp_out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, a->stream));
  CK(cudaStreamSynchronize(a->stream));
  std::memcpy(delta_k, h.data(), sizeof(double) * K);
  std::memcpy(mcse_k, h.data() + K, sizeof(double) * K);
  std::memcpy(out, h.data() + 2 * K, sizeof(double) * 4);
  leave(a);
  return PCV_OK;
}

pcv_status pcv_kernel_launches(pcv_ctx *x, int64_t *n) {
  if (!x || !n) return fail(x, PCV_E_INVALID_ARG, "null argument");
  if (!x->kernels_exact) return fail(x, PCV_E_UNSUPPORTED, "iterations ran outside CUDA graphs (use_graphs = 0)");
  *n = x->kernels_issued;
  return PCV_OK;
}

pcv_status pcv_compare_pair(pcv_ctx *x, double *delta_k, double *mcse_k, double *out) {
  if (!x) return PCV_E_INVALID_ARG;
  if (!delta_k || !mcse_k || !out) return fail(x, PCV_E_INVALID_ARG, "null argument");
  if (!x->pair) return fail(x, PCV_E_INVALID_ARG, "the context holds one model (no active_covariates_b)");
  if (x->state != ST_SAMPLED) return fail(x, PCV_E_BAD_STATE, "pcv_compare_pair before pcv_sample");
  enter(x);
  pcv_status s = finalize(x);
  if (s != PCV_OK) return s;
  const int K = x->K_model;
  if ((size_t)(2 * K + 4) > x->cmp_n) {
    if (!dalloc_n(x, &x->cmp_out, (size_t)(2 * K + 4))) return fail(x, PCV_E_OOM, "allocation failed");
    x->cmp_n = (size_t)(2 * K + 4);
  }
  // model A's folds [0, K), model B's [K, 2 K): the fold outputs are fold-major
  k_compare<<<1, 256, 0, x->stream>>>(x->fold_out, x->fold_out + (size_t)K * F_NFIELDS, K, x->cmp_out);
  CK(cudaGetLastError());
  std::vector<double> h((size_t)(2 * K + 4));
  CK(cudaMemcpyAsync(h.data(), x->cmp_out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, x->stream));
  CK(cudaStreamSynchronize(x->stream));
  std::memcpy(delta_k, h.data(), sizeof(double) * K);
  std::memcpy(mcse_k, h.data() + K, sizeof(double) * K);
  std::memcpy(out, h.data() + 2 * K, sizeof(double) * 4);
  leave(x);
  return PCV_OK;
}

pcv_status pcv_rhat_shuffle(pcv_ctx *x, int32_t n_blocks, int32_t n_reps, double *rhat_max_rep,
                            double *rhat_fold_rep) {
  if (!x) return PCV_E_INVALID_ARG;
  if (!rhat_max_rep || n_blocks < 1 || n_reps < 1) return fail(x, PCV_E_INVALID_ARG, "bad argument");
  if (x->state != ST_SAMPLED) return fail(x, PCV_E_BAD_STATE, "pcv_rhat_shuffle before pcv_sample");
  const long long a = x->n_sampled / x->b;
  if (a < n_blocks) return fail(x, PCV_E_INVALID_ARG, "fewer batches than blocks");
  if (a > x->max_batches) return fail(x, PCV_E_INVALID_ARG, "more batches than max_batches were stored");
  const size_t nb = (size_t)x->C * n_blocks * 3, na = (size_t)n_reps * x->K;
  if (nb > x->shuf_blk_n) {
    if (!dalloc_n(x, &x->shuf_blk, nb)) return fail(x, PCV_E_OOM, "allocation failed");
    x->shuf_blk_n = nb;
  }
  if (rhat_fold_rep && na > x->shuf_all_n) {
    if (!dalloc_n(x, &x->shuf_all, na)) return fail(x, PCV_E_OOM, "allocation failed");
    x->shuf_all_n = na;
  }
  if ((size_t)n_reps > x->shuf_max_n) {
    if (!dalloc_n(x, &x->shuf_max, (size_t)n_reps)) return fail(x, PCV_E_OOM, "allocation failed");
    x->shuf_max_n = (size_t)n_reps;
  }
  enter(x);
  const long long T1 = (long long)x->C * n_blocks;
  k_block_stats<<<(unsigned)((T1 + 255) / 256), 256, 0, x->stream>>>(x->acc, (int)a, n_blocks, x->shuf_blk);
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(x->shuf_max, 0, sizeof(unsigned long long) * n_reps, x->stream));
  const long long T2 = (long long)n_reps * x->K;
  k_rhat_shuffle<<<(unsigned)((T2 + 255) / 256), 256, 0, x->stream>>>(
      x->shuf_blk, x->K, x->L, n_blocks, n_reps, x->opt.seed, x->shuf_max, rhat_fold_rep ? x->shuf_all : nullptr,
      x->opt.first_fold);
  CK(cudaGetLastError());
  std::vector<unsigned long long> hm(n_reps);
  CK(cudaMemcpyAsync(hm.data(), x->shuf_max, sizeof(unsigned long long) * n_reps, cudaMemcpyDeviceToHost, x->stream));
  if (rhat_fold_rep)
    CK(cudaMemcpyAsync(rhat_fold_rep, x->shuf_all, sizeof(double) * na, cudaMemcpyDeviceToHost, x->stream));
  CK(cudaStreamSynchronize(x->stream));
  for (int r = 0; r < n_reps; ++r) std::memcpy(&rhat_max_rep[r], &hm[r], sizeof(double));
  leave(x);
  return PCV_OK;
}

pcv_status pcv_tuning_info(const pcv_ctx *x, char *buf, int32_t len) {
  if (!x || !buf || len < 1) return PCV_E_INVALID_ARG;
  std::string s;
  for (const std::string &l : x->tune_log) s += l + "\n";
  std::snprintf(buf, (size_t)len, "%s", s.c_str());
  return PCV_OK;
}

pcv_status pcv_setup_ms(const pcv_ctx *x, double *autotune_ms, double *graph_capture_ms) {
  if (!x || !autotune_ms || !graph_capture_ms) return PCV_E_INVALID_ARG;
  *autotune_ms = x->tune_ms;
  *graph_capture_ms = x->capture_ms;
  return PCV_OK;
}

pcv_status pcv_last_sample_ms(pcv_ctx *x, double *ms) {
  if (!x || !ms) return PCV_E_INVALID_ARG;
  *ms = x->last_ms;
  return PCV_OK;
}

}  // extern "C"

// ===========================================================================
// Allocation-free gradient evaluation.
//
// Some callers must not allocate device memory at call time: a process that
// hands the GPU's memory to another framework's pool, or a latency-bound
// serving loop where cudaMalloc could stall or synchronise the device at an
// unpredictable moment.  For them the split-N workspace and tickets of the
// gradient kernels live in fixed file-scope device arrays instead of the
// context's (growable) workspace.  Every GPU that loads this library keeps
// these arrays (kNoAllocScratchFloats floats = 16 MiB, plus kNoAllocTickets
// counters) until the process exits.
// ===========================================================================
namespace {

constexpr size_t kNoAllocScratchFloats = (size_t)4 << 20;   // 16 MiB of FP32 partials
constexpr int kNoAllocTickets = 8192;                        // chain tiles (32 or 64 chains)

static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];
static __device__ __align__(256) unsigned int g_noalloc_tickets[kNoAllocTickets];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
float *g_noalloc_ws[kMaxDevices] = {};
unsigned int *g_noalloc_tk[kMaxDevices] = {};

// Device addresses of the arrays on the current device, looked up once per
// device (host code cannot use the symbols' names as device pointers).
cudaError_t noalloc_addresses(float **ws, unsigned int **tk) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ws[dev]) {
    void *p = nullptr, *q = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress(&q, g_noalloc_tickets);
    if (e != cudaSuccess) return e;
    g_noalloc_ws[dev] = static_cast<float *>(p);
    g_noalloc_tk[dev] = static_cast<unsigned int *>(q);
  }
  *ws = g_noalloc_ws[dev];
  *tk = g_noalloc_tk[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" pcv_status pcv_log_density_noalloc(pcv_ctx *x, const float *theta, const int32_t *fold,
                                              int32_t n, int32_t precision, double *logp,
                                              float *grad, double *shat) {
  if (!x) return PCV_E_INVALID_ARG;
  if (!theta || !fold || !logp || !grad || !shat || n < 1) return fail(x, PCV_E_INVALID_ARG, "bad argument");
  if (precision != PCV_FP32_SIMT) return fail(x, PCV_E_UNSUPPORTED, "precision not available for this context");
  const int tw = simt_chain_tile(x->p);
  const int tiles = (n + tw - 1) / tw;
  const int stride = std::max(x->d_pad, simt_flat_pp(x->p)) + 4;
  const std::string what = "pcv_log_density_noalloc: n = " + std::to_string(n) + " positions of dimension " +
                           std::to_string(x->d) + " need " + std::to_string(tiles) + " chain tiles of " +
                           std::to_string(tw);
  if (tiles > kNoAllocTickets)
    return fail(x, PCV_E_INVALID_ARG,
                what + ", more than the fixed ticket array's " + std::to_string(kNoAllocTickets) +
                    " tiles; use pcv_log_density");
  if ((size_t)tiles * tw * stride > kNoAllocScratchFloats)
    return fail(x, PCV_E_INVALID_ARG,
                what + " x " + std::to_string(stride) + " partial sums = " +
                    std::to_string((size_t)tiles * tw * stride) + " floats, more than the fixed scratch's " +
                    std::to_string(kNoAllocScratchFloats) + "; use pcv_log_density");
  float *ws = nullptr;
  unsigned int *tk = nullptr;
  CK(noalloc_addresses(&ws, &tk));
  // largest split count that fits the fixed scratch, at most the usual choice
  ChainBufs cb;
  cb.C = n; cb.L = 1; cb.fold_base = 0;
  GradArgs a = grad_args(x, cb, false);
  const size_t per_split = (size_t)tiles * tw * stride;
  a.splits = std::max(1, std::min(a.splits, (int)(kNoAllocScratchFloats / per_split)));
  a.fold_of = fold;
  a.theta = theta; a.ld_theta = x->d;
  a.grad = grad; a.ld_grad = x->d;
  a.logp = logp; a.shat = shat;
  a.need_ll = 1;
  a.mode = MODE_NONE;
  a.r = nullptr;
  a.ws = ws;
  a.ws_stride = stride;
  a.tickets = tk;
  enter(x);
  // tickets must start at zero: a previous call that failed part-way could
  // have left some set (clearing is a memset, not an allocation)
  CK(cudaMemsetAsync(tk, 0, sizeof(unsigned int) * (size_t)tiles, x->stream));
  CK(launch_grad_simt(x->pb, a, x->stream));
  leave(x);
  return PCV_OK;
}
