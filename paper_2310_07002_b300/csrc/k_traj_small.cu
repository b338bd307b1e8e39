// k_traj_small.cu -- a whole leapfrog trajectory of every chain in one
// launch, for problems small enough that one warp can sweep all rows of a
// chain at every step (the latency-bound configurations: a few thousand rows
// and p <= 32).  Lock-step HMC (Section 3.3) needs no synchronisation between
// chains, so a warp owns one chain for the whole trajectory:
//   momentum draw r ~ N(0, M) (Philox4x32-10 + Box-Muller), H0, the first
//   half kick and drift (as k_begin), then L_f gradient evaluations of the
//   fold-masked log posterior (eq. mask-log-prob / mask-log-pred,
//   Appendix B), each followed by its kick and drift, the last one by the
//   final half kick and the log densities log pi_k(theta') and
//   s_k(theta') = sum over the fold's test rows of log p(y_n | theta').
// In accept mode the same warp then takes the Metropolis decision and updates
// the chain's FP64 accumulators (what k_accept does), so an iteration is one
// launch; otherwise k_accept runs after it.  The hierarchical model has a
// kernel of its own below (k_traj_hier: z lives in shared memory).
//
// Layout: lanes stride over rows; each lane keeps the whole position and
// momentum in registers, the gradient sums are reduced with warp shuffles
// (xor tree: every lane ends with the totals) and every lane applies the
// same update, so the steps need no block synchronisation.  Rows are sorted
// by fold, so a chain's training rows are the two ranges around its fold's
// excluded block and its test rows one range: the masks of Appendix B become
// loop bounds.  Every warp re-reads the whole design matrix at every step,
// so where it fits (with y) the CTA first copies it into shared memory;
// otherwise the rows come through the L1 cache.  The BF16 form reads a bf16
// copy of X (half the bytes; products and sums in FP32).
//
// Gaussian models accumulate sum_n e_n x_n and sum_n e_n^2 (e = y - eta) and
// apply 1 / sigma^2 once after the reduction: the gradient, the log sigma
// term and both log densities follow from them.
#include "pcv_internal.cuh"
#include "pcv_accum.cuh"

namespace pcv {

constexpr int kTrajWarps = 8;
constexpr size_t kTrajSmemMax = 100 * 1024;   // rows staged in shared memory up to this size

// Where the rows come from: FP32 X or its bf16 copy (row stride `stride`
// elements), and y, in shared memory or global memory.  Rows are read in
// 16-byte (FP32) / 8-byte (bf16) pieces when PP is a multiple of 4, else in
// pairs.
template <int PP, bool XB16>
struct Rows {
  const float *X;
  const __nv_bfloat16 *X16;
  const float *y;
  int stride;
  __device__ __forceinline__ void load(int n, float (&x)[PP]) const {
    if constexpr (XB16) {
      if constexpr (PP % 4 == 0) {
        const uint2 *xr = reinterpret_cast<const uint2 *>(X16 + (size_t)n * stride);
#pragma unroll
        for (int q = 0; q < PP / 4; ++q) {
          const uint2 v = xr[q];
          x[4 * q] = __uint_as_float(v.x << 16);
          x[4 * q + 1] = __uint_as_float(v.x & 0xFFFF0000u);
          x[4 * q + 2] = __uint_as_float(v.y << 16);
          x[4 * q + 3] = __uint_as_float(v.y & 0xFFFF0000u);
        }
      } else {
        const uint32_t *xr = reinterpret_cast<const uint32_t *>(X16 + (size_t)n * stride);
#pragma unroll
        for (int q = 0; q < PP / 2; ++q) {
          const uint32_t v = xr[q];
          x[2 * q] = __uint_as_float(v << 16);
          x[2 * q + 1] = __uint_as_float(v & 0xFFFF0000u);
        }
      }
    } else {
      if constexpr (PP % 4 == 0) {
        const float4 *xr = reinterpret_cast<const float4 *>(X + (size_t)n * stride);
#pragma unroll
        for (int q = 0; q < PP / 4; ++q) {
          const float4 v = xr[q];
          x[4 * q] = v.x; x[4 * q + 1] = v.y; x[4 * q + 2] = v.z; x[4 * q + 3] = v.w;
        }
      } else {
        const float2 *xr = reinterpret_cast<const float2 *>(X + (size_t)n * stride);
#pragma unroll
        for (int q = 0; q < PP / 2; ++q) {
          const float2 v = xr[q];
          x[2 * q] = v.x; x[2 * q + 1] = v.y;
        }
      }
    }
  }
};

// One row's contribution at position th: logistic w = y - sigmoid(eta) and
// (LL) y eta - softplus(eta) into ll; Gaussian w = e = y - eta and e^2 into
// e2; then (GRAD) w x into acc.
template <int PP, int MV, bool GRAD, bool LL>
__device__ __forceinline__ void row_terms(const float (&th)[PP], const float (&x)[PP], float yv, float (&acc)[PP],
                                          float &e2, float &ll) {
  float eta = 0.0f;
#pragma unroll
  for (int j = 0; j < PP; ++j) eta = fmaf(th[j], x[j], eta);
  float w;
  if constexpr (MV == MV_LOGISTIC) {
    w = yv - 1.0f / (1.0f + __expf(-eta));
    if (LL) ll += yv * eta - softplusf(eta);
  } else {
    w = yv - eta;
    e2 = fmaf(w, w, e2);
  }
  if (GRAD) {
#pragma unroll
    for (int j = 0; j < PP; ++j) acc[j] = fmaf(w, x[j], acc[j]);
  }
}

// One lane's sums over rows [lo, hi): rows lo + first + i * step (first =
// this thread's place in the chain's team of warps, step = the team's
// threads); several rows per pass so that their loads are in flight together.
template <int PP, int MV, bool XB16, bool GRAD, bool LL>
__device__ __forceinline__ void range_sums(const Rows<PP, XB16> &R, int lo, int hi, int first, int step,
                                           const float (&th)[PP], float (&acc)[PP], float &e2, float &ll) {
  constexpr int U = PP <= 8 ? 4 : PP <= 16 ? 2 : 1;
  int n = lo + first;
  for (; n + step * (U - 1) < hi; n += step * U) {
    float x[U][PP], yv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      R.load(n + step * u, x[u]);
      yv[u] = R.y[n + step * u];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) row_terms<PP, MV, GRAD, LL>(th, x[u], yv[u], acc, e2, ll);
  }
  for (; n < hi; n += step) {
    float x[PP];
    R.load(n, x);
    row_terms<PP, MV, GRAD, LL>(th, x, R.y[n], acc, e2, ll);
  }
}

// The warps that share one chain (wpc of them, consecutive in the CTA): each
// sums its share of the rows; the partial sums meet in shared memory (two
// buffers, alternating by evaluation, so one barrier per evaluation
// suffices) and every warp adds them in the same order, so all hold the same
// totals and apply the same update.
struct Team {
  int wpc, wic, lane, warp;  // warps per chain, this warp's place in it, lane, warp in the CTA
  int bar;                   // named barrier of the team (1 + chain within the CTA)
  float *fpart;              // [2][8 warps][PP + 2] floats
  double *dpart;             // [2][8 warps][2] doubles
  int parity;
};

__device__ __forceinline__ void team_sync(const Team &tm) {
  asm volatile("bar.sync %0, %1;" ::"r"(tm.bar), "r"(32 * tm.wpc) : "memory");
}

// One gradient evaluation of the chain's fold-masked log posterior at th
// (ls: log sigma for the LOGSIG variant): the gradient in g / gls (every
// lane of every warp of the team) and, with LL, the log likelihoods of the
// training and test rows.
template <int PP, int MV, bool XB16, bool LL>
__device__ __forceinline__ void evaluate(const Problem &pb, const Rows<PP, XB16> &R, const FoldDesc &fd, Team &tm,
                                         const float (&th)[PP], float ls, float (&g)[PP], float &gls,
                                         double &ll_tr, double &ll_te) {
  constexpr bool GAUSS = MV != MV_LOGISTIC;
  const int first = tm.wic * 32 + tm.lane, step = 32 * tm.wpc;
  float acc[PP];
#pragma unroll
  for (int j = 0; j < PP; ++j) acc[j] = 0.0f;
  float e2 = 0.0f, ll = 0.0f;
  range_sums<PP, MV, XB16, true, LL>(R, 0, fd.excl_lo, first, step, th, acc, e2, ll);
  range_sums<PP, MV, XB16, true, LL>(R, fd.excl_hi, pb.N, first, step, th, acc, e2, ll);
  float e2t = 0.0f, llt = 0.0f;
  if (LL) range_sums<PP, MV, XB16, false, true>(R, fd.test_lo, fd.test_hi, first, step, th, acc, e2t, llt);
#pragma unroll
  for (int j = 0; j < PP; ++j) acc[j] = warp_sum(acc[j]);
  if (GAUSS) e2 = warp_sum(e2);
  double dl = 0.0, dlt = 0.0;
  if (LL) {
    if (GAUSS) e2t = warp_sum(e2t);
    else { dl = warp_sum_d((double)ll); dlt = warp_sum_d((double)llt); }
  }
  if (tm.wpc > 1) {
    float *fp = tm.fpart + ((size_t)tm.parity * 8 + tm.warp) * (PP + 2);
    double *dp = tm.dpart + ((size_t)tm.parity * 8 + tm.warp) * 2;
    if (tm.lane == 0) {
#pragma unroll
      for (int j = 0; j < PP; ++j) fp[j] = acc[j];
      fp[PP] = e2;
      fp[PP + 1] = e2t;
      dp[0] = dl;
      dp[1] = dlt;
    }
    team_sync(tm);
    const int w0 = tm.warp - tm.wic;                 // the team's first warp
#pragma unroll
    for (int j = 0; j < PP; ++j) acc[j] = 0.0f;
    e2 = 0.0f; e2t = 0.0f; dl = 0.0; dlt = 0.0;
    for (int w = 0; w < tm.wpc; ++w) {
      const float *q = tm.fpart + ((size_t)tm.parity * 8 + w0 + w) * (PP + 2);
      const double *qd = tm.dpart + ((size_t)tm.parity * 8 + w0 + w) * 2;
#pragma unroll
      for (int j = 0; j < PP; ++j) acc[j] += q[j];
      e2 += q[PP];
      e2t += q[PP + 1];
      dl += qd[0];
      dlt += qd[1];
    }
    tm.parity ^= 1;
  }
  float logsig = 0.0f, inv_s2 = 1.0f;
  if (MV == MV_GAUSS_KNOWN) {
    logsig = logf(pb.sigma_known);
    inv_s2 = 1.0f / (pb.sigma_known * pb.sigma_known);
  } else if (MV == MV_GAUSS_LOGSIG) {
    logsig = ls;
    inv_s2 = expf(-2.0f * ls);
  }
  const float wscale = GAUSS ? inv_s2 : 1.0f;
#pragma unroll
  for (int j = 0; j < PP; ++j) g[j] = fmaf(wscale, acc[j], -th[j] * pb.beta_prec);
  const int n_tr = pb.N - (fd.excl_hi - fd.excl_lo);
  if (MV == MV_GAUSS_LOGSIG)   // d/dlog sigma: sum_train (e^2 / sigma^2 - 1) - sigma^2 / sd^2 + 1
    gls = (inv_s2 * e2 - (float)n_tr) - __expf(2.0f * ls) * pb.sigma_prec + 1.0f;
  if (LL) {
    if (GAUSS) {
      const double c0 = 0.5 * kLog2PiD + (double)logsig;
      ll_tr = -(double)n_tr * c0 - 0.5 * (double)inv_s2 * (double)e2;
      ll_te = -(double)(fd.test_hi - fd.test_lo) * c0 - 0.5 * (double)inv_s2 * (double)e2t;
    } else {
      ll_tr = dl;
      ll_te = dlt;
    }
  }
}

// Accept mode: the Metropolis tests and scalar accumulators of the CTA's
// chains, one lane per chain in the CTA's first warp (as k_accept's phase
// B): an FP64 warp instruction, ~32 cycles of an SM on this part, then
// serves every chain of the CTA instead of one.  Every warp of the CTA calls
// it exactly once (it holds two CTA barriers); slot is the chain's place in
// the CTA (its lane 0 reports dH, finiteness and the proposal's log
// densities), -1 for a warp with nothing to report.  Returns whether the
// chain was accepted and, in s_draw, the draw's held-out value; on
// acceptance the chain's log densities are the proposal's.
constexpr int kBatchMax = 16;   // chains per CTA at most (k_traj_hier: 16 warps)

__device__ __forceinline__ bool accept_batch(const TrajArgs &t, int slot, int lane, int c0, int nch, double dH,
                                             bool finite, double logp1, double ll_te, double &s_draw) {
  __shared__ double b_dh[kBatchMax], b_lp[kBatchMax], b_te[kBatchMax], b_s[kBatchMax];
  __shared__ int b_fl[kBatchMax];
  if (slot >= 0 && lane == 0) {
    b_dh[slot] = dH;
    b_lp[slot] = logp1;
    b_te[slot] = ll_te;
    b_fl[slot] = finite ? 1 : 0;
  }
  __syncthreads();
  if (threadIdx.x < nch) {
    const int l = threadIdx.x, cc = c0 + l;
    const uint4 w = philox_at(t.seed, 0u, (uint32_t)(t.chain_base + cc), *t.iter, t.acc_stream);
    const double lu = log(unit_from_word(w.x));
    const double d = b_dh[l];
    const bool fin = b_fl[l] != 0;
    const bool acc = fin && (lu < -d);
    const bool div = !fin || d > 1000.0;
    const double sd = acc ? b_te[l] : t.shat_w[cc];
    if (acc) {
      t.logp_w[cc] = b_lp[l];
      t.shat_w[cc] = b_te[l];
    }
    if (t.accept_prob) t.accept_prob[cc] = fin ? (d <= 0.0 ? 1.0 : exp(-d)) : 0.0;
    if (t.accumulate) {
      const long long n_before = t.st->n_draws;
      t.acc.div[cc] += div ? 1 : 0;
      t.acc.acc[cc] += acc ? 1 : 0;
      accum_scalar(t.acc, cc, sd, n_before);
      if (t.acc.draws && n_before < t.acc.draw_cap) t.acc.draws[(size_t)cc * t.acc.draw_cap + n_before] = sd;
    }
    b_fl[l] = acc ? 1 : 0;
    b_s[l] = sd;
  }
  __syncthreads();
  if (slot < 0) return false;
  s_draw = b_s[slot];
  return b_fl[slot] != 0;
}

// One chain's trajectory (and, in accept mode, its Metropolis test and
// accumulators), carried by its team of warps.
template <int PP, int MV, bool XB16>
__device__ __forceinline__ void traj_team(const Problem &pb, const TrajArgs &t, const Rows<PP, XB16> &R, Team &tm,
                                          int c) {
  constexpr bool LOGSIG = MV == MV_GAUSS_LOGSIG;
  const int lane = tm.lane;
  const bool writer = tm.wic == 0;                // the team's first warp writes the results
  const int p = pb.p, d = pb.d;
  const unsigned it = *t.iter;
  // this iteration's step size (nominal, or jittered by one uniform shared
  // by every chain: Philox stream ST_JIT at chain 0)
  float eps = *t.eps;
  if (t.jitter > 0.0f) {
    const uint4 w = philox_at(t.seed, 0u, 0u, it, ST_JIT);
    eps = (float)((double)eps * (1.0 + (double)t.jitter * (2.0 * unit_from_word(w.x) - 1.0)));
  }
  if (!t.eval_only && c == 0 && writer && lane == 0 && t.eps_iter) *t.eps_iter = eps;
  const FoldDesc fd = pb.folds[t.fold_base + c / t.L];
  const float *mvr = minv_row(t.minv, c, t.minv_every, t.minv_ld);   // this chain's model's inverse mass
  const float *th0 = t.theta + (size_t)c * t.ld;

  // position and momentum in registers (every lane holds all of them); for
  // the LOGSIG variant log sigma is coordinate p, kept apart (ls, rls)
  float th[PP], rr[PP], g[PP];
  float ls = LOGSIG ? th0[p] : 0.0f, rls = 0.0f, gls = 0.0f;
#pragma unroll
  for (int j = 0; j < PP; ++j) { th[j] = j < p ? th0[j] : 0.0f; rr[j] = 0.0f; }
  double ll_tr = 0.0, ll_te = 0.0, H0 = 0.0;
  if (t.eval_only) {
    // one evaluation at the current position (no momentum, no update)
    evaluate<PP, MV, XB16, true>(pb, R, fd, tm, th, ls, g, gls, ll_tr, ll_te);
  } else {
    // momentum: lane q draws the normals of coordinate quad q (the same
    // Philox words and Box-Muller as k_begin), then they are broadcast;
    // kinetic energy in FP64 across coordinates, first half kick and drift
    const int nq = (d + 3) / 4;
    float z0 = 0.0f, z1 = 0.0f, z2 = 0.0f, z3 = 0.0f;
    if (!t.r_given && lane < nq) {
      const uint4 w = philox_at(t.seed, (uint32_t)lane, (uint32_t)(t.chain_base + c), it, t.stream);
      const float2 a0 = box_muller(w.x, w.y), a1 = box_muller(w.z, w.w);
      z0 = a0.x; z1 = a0.y; z2 = a1.x; z3 = a1.y;
    }
    const float *g0 = t.grad + (size_t)c * t.ld;
    float kterm = 0.0f;     // this lane's kinetic-energy terms (coordinates j with j % 32 == lane)
    // coordinate jj's momentum r0 (its normal from lane jj / 4), kinetic
    // term, half kick and drift of the start value v
    auto start = [&](int jj, float v, float &tn, float &rh) {
      const int k = jj & 3;
      const float zq = k == 0 ? z0 : k == 1 ? z1 : k == 2 ? z2 : z3;
      const float zj = __shfl_sync(0xffffffffu, zq, jj >> 2);
      const float m = mvr[jj];
      const float r0 = t.r_given ? t.r_given[(size_t)c * t.ld + jj] : (m > 0.0f ? zj / sqrtf(m) : 0.0f);
      if (lane == (jj & 31)) kterm = fmaf(m * r0, r0, kterm);
      rh = r0 + 0.5f * eps * g0[jj];
      tn = v + eps * m * rh;
    };
#pragma unroll
    for (int j = 0; j < PP; ++j) {
      if (j < p) {
        float tn, rh;
        start(j, th[j], tn, rh);
        th[j] = tn;
        rr[j] = rh;
      }
    }
    if (LOGSIG) {
      float tn, rh;
      start(p, ls, tn, rh);
      ls = tn;
      rls = rh;
    }
    H0 = -t.logp[c] + 0.5 * warp_sum_d((double)kterm);
    if (!t.accept && writer && lane == 0) t.H0[c] = H0;
    for (int s = 1; s <= t.Lf; ++s) {
      const bool last = s == t.Lf;
      if (last) evaluate<PP, MV, XB16, true>(pb, R, fd, tm, th, ls, g, gls, ll_tr, ll_te);
      else evaluate<PP, MV, XB16, false>(pb, R, fd, tm, th, ls, g, gls, ll_tr, ll_te);
      // kick, and drift except after the last gradient (every lane alike)
      const float kick = last ? 0.5f * eps : eps;
#pragma unroll
      for (int j = 0; j < PP; ++j) {
        if (j < p) {
          rr[j] += kick * g[j];
          if (!last) th[j] += eps * mvr[j] * rr[j];
        }
      }
      if (LOGSIG) {
        rls += kick * gls;
        if (!last) ls += eps * mvr[p] * rls;
      }
    }
  }
  const int cpc = kTrajWarps / t.wpc, c0 = blockIdx.x * cpc, nch = min(cpc, t.C - c0);
  if (!writer) {
    double sd;
    if (t.accept) accept_batch(t, -1, lane, c0, nch, 0.0, false, 0.0, 0.0, sd);
    return;
  }
  // log prior: this lane's coordinates in FP32, summed across lanes in FP64
  float lpt = 0.0f;
#pragma unroll
  for (int j = 0; j < PP; ++j)
    if (j < p && lane == (j & 31))
      lpt += -0.5f * kLog2Pi - pb.log_beta_sd - 0.5f * th[j] * th[j] * pb.beta_prec;
  if (LOGSIG && lane == (p & 31)) {
    const float s2 = __expf(2.0f * ls);
    lpt += (float)kLog2D - 0.5f * kLog2Pi - pb.log_sigma_sd - 0.5f * s2 * pb.sigma_prec + ls;
  }
  const double logp1 = ll_tr + warp_sum_d((double)lpt);
  if (!t.accept) {
    // proposal state out (lane j writes coordinate j), gradient, log densities
    float *thp = t.theta_p + (size_t)c * t.ld, *rp = t.r + (size_t)c * t.ld, *gp = t.grad_p + (size_t)c * t.ld;
#pragma unroll
    for (int j = 0; j < PP; ++j)
      if (j < p && lane == (j & 31)) {
        if (!t.eval_only) { thp[j] = th[j]; rp[j] = rr[j]; }
        gp[j] = g[j];
      }
    if (LOGSIG && lane == (p & 31)) {
      if (!t.eval_only) { thp[p] = ls; rp[p] = rls; }
      gp[p] = gls;
    }
    if (lane == 0) {
      t.logp_p[c] = logp1;
      t.shat_p[c] = ll_te;
    }
    return;
  }
  // ---- accept mode: the Metropolis test in FP64 (as k_accept): H1 from
  // the momentum at the end of the trajectory, u from the accept stream;
  // a divergence when H1 is not finite or H1 - H0 > 1000; on acceptance the
  // chain's state becomes the proposal, else it stays
  float kt = 0.0f;
#pragma unroll
  for (int j = 0; j < PP; ++j)
    if (j < p && lane == (j & 31)) kt = fmaf(mvr[j] * rr[j], rr[j], kt);
  if (LOGSIG && lane == (p & 31)) kt = fmaf(mvr[p] * rls, rls, kt);
  const double H1 = -logp1 + 0.5 * warp_sum_d((double)kt);
  const double dH = H1 - H0;
  const bool finite = isfinite(H1) && isfinite(dH);
  double s_draw = 0.0;
  const bool acc = accept_batch(t, tm.warp / t.wpc, lane, c0, nch, dH, finite, logp1, ll_te, s_draw);
  float *thw = t.theta_w + (size_t)c * t.ld, *gw = t.grad_w + (size_t)c * t.ld;
  if (acc) {
#pragma unroll
    for (int j = 0; j < PP; ++j)
      if (j < p && lane == (j & 31)) { thw[j] = th[j]; gw[j] = g[j]; }
    if (LOGSIG && lane == (p & 31)) { thw[p] = ls; gw[p] = gls; }
  }
  if (t.accumulate) {
    const long long n_before = t.st->n_draws;
    accum_lags(t.acc, c, acov_x(t.acc, c, s_draw, n_before), n_before, lane);
  }
}

// Accept mode, at the end of the kernel (every thread of the CTA): once all
// teams of this CTA are done, the last CTA advances the iteration counters
// (every CTA has read them by now).
__device__ __forceinline__ void advance_counters(const TrajArgs &t) {
  __shared__ int is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&t.st->ticket, 1u);
    is_last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (is_last && threadIdx.x == 0) {
    __threadfence();
    t.st->ticket = 0u;
    if (t.fd) t.st->fd_iter += 1u;
    else {
      t.st->iter += 1u;
      if (t.accumulate) t.st->n_draws += 1;
    }
  }
}

template <int PP, int MV, bool XB16>
__global__ void __launch_bounds__(kTrajWarps * 32, PP <= 12 ? 2 : 1) k_traj_small(Problem pb, TrajArgs t) {
  extern __shared__ __align__(16) uint8_t traj_smem[];
  // rows: staged into shared memory (compact, PP elements per row) when the
  // host sized it for them
  Rows<PP, XB16> R{pb.X, t.X16, pb.y, XB16 ? PP : pb.p_pad};
  if (t.smem_rows) {
    const size_t xbytes = ((size_t)pb.N * PP * (XB16 ? 2 : 4) + 15) / 16 * 16;
    if constexpr (XB16) {
      // the bf16 copy is compact already, allocated and zero-padded to a
      // multiple of 16 bytes
      const uint4 *src = reinterpret_cast<const uint4 *>(t.X16);
      uint4 *dst = reinterpret_cast<uint4 *>(traj_smem);
      for (size_t i = threadIdx.x; i < xbytes / 16; i += blockDim.x) dst[i] = __ldg(src + i);
    } else {
      // FP32 rows of p_pad floats, PP of them kept (pairs)
      float2 *dst = reinterpret_cast<float2 *>(traj_smem);
      const int np2 = PP / 2;
      for (int i = threadIdx.x; i < pb.N * np2; i += blockDim.x) {
        const int n = i / np2, q = i - n * np2;
        dst[i] = __ldg(reinterpret_cast<const float2 *>(pb.X + (size_t)n * pb.p_pad) + q);
      }
    }
    float *ys = reinterpret_cast<float *>(traj_smem + xbytes);
    for (int i = threadIdx.x; i < pb.N; i += blockDim.x) ys[i] = __ldg(pb.y + i);
    __syncthreads();
    R.X = reinterpret_cast<const float *>(traj_smem);
    R.X16 = reinterpret_cast<const __nv_bfloat16 *>(traj_smem);
    R.y = ys;
    R.stride = PP;
  }
  // the team of warps of this chain; partial sums live after the staged rows
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Team tm;
  tm.wpc = t.wpc;
  tm.wic = warp % t.wpc;
  tm.lane = lane;
  tm.warp = warp;
  tm.bar = 1 + warp / t.wpc;
  tm.dpart = reinterpret_cast<double *>(traj_smem + t.part_offset);
  tm.fpart = reinterpret_cast<float *>(tm.dpart + 2 * kTrajWarps * 2);
  tm.parity = 0;
  const int c = blockIdx.x * (kTrajWarps / t.wpc) + warp / t.wpc;
  // a team past the last chain does nothing, but (accept mode) still meets
  // the CTA barriers of the batched accept and of the counter advance
  if (c < t.C) {
    traj_team<PP, MV, XB16>(pb, t, R, tm, c);
  } else if (t.accept) {
    const int cpc = kTrajWarps / t.wpc, c0 = blockIdx.x * cpc;
    double sd;
    accept_batch(t, -1, lane, c0, min(cpc, t.C - c0), 0.0, false, 0.0, 0.0, sd);
  }
  if (t.accept) advance_counters(t);
}

// ---------------------------------------------------------------------------
// The hierarchical model in one launch per iteration (varying intercepts,
// non-centred alpha_g = tau z_g; theta = [beta (p), z (G), log tau,
// log sigma]): one warp per chain.  beta, log tau and log sigma live in
// every lane's registers (every lane applies the same update to them); z,
// its momentum and its gradient live in the chain's slice of shared memory.
// Rows are sorted by group, so lane l owns the row segments l, l + 32, ...
// (one group each): the sums for d/dz_g need no atomics, and a group's z is
// read, kicked and drifted by its own lane only (no barrier between steps).
// The gradient and the log densities are those of k_grad_hier with
// finish_chain<MV_HIER>: a training row adds e x / sigma^2 to beta's
// gradient, e / sigma^2 to its segment's sum seg_g (d/dz_g = tau seg_g,
// d/dlog tau = sum_g seg_g tau z_g) and e^2 / sigma^2 - 1 to d/dlog sigma;
// a group held out by the fold is scored by the group-level predictive with
// its intercept integrated out.
// ---------------------------------------------------------------------------
template <int PP, bool LL>
__device__ __forceinline__ void eval_hier(const Problem &pb, const Rows<PP, false> &R, const FoldDesc &fd,
                                          int lane, const float (&bt)[PP], float lt, float ls, const float *zs,
                                          float *gz, float (&g)[PP], float &glt, float &gls, double &ll_tr,
                                          double &ll_te) {
  const int p = pb.p, G = pb.G;
  const float tau = expf(lt), inv_s2 = expf(-2.0f * ls);
  float acc[PP];
#pragma unroll
  for (int j = 0; j < PP; ++j) acc[j] = 0.0f;
  float dls = 0.0f, dlt = 0.0f, llt = 0.0f;
  double lte = 0.0;
  for (int gg = lane; gg < G; gg += 32) {
    const int gid = pb.seg_grp[gg];
    const float z = zs[gid], off = tau * z;
    const int n0 = pb.grp_off[gg], n1 = pb.grp_off[gg + 1];
    const bool test_seg = LL && n1 > n0 && n0 >= fd.test_lo && n1 <= fd.test_hi;
    float seg = 0.0f, s1 = 0.0f, s2 = 0.0f;
    auto row = [&](const float (&x)[PP], float yv, int n) {
      float eta = off;
#pragma unroll
      for (int j = 0; j < PP; ++j) eta = fmaf(bt[j], x[j], eta);
      const float e = yv - eta;
      const float tr = (n < fd.excl_lo || n >= fd.excl_hi) ? 1.0f : 0.0f;
      const float wv = e * inv_s2 * tr;
#pragma unroll
      for (int j = 0; j < PP; ++j) acc[j] = fmaf(wv, x[j], acc[j]);
      seg += wv;
      dls = fmaf(tr, e * e * inv_s2 - 1.0f, dls);
      if (LL) {
        llt = fmaf(tr, -0.5f * kLog2Pi - ls - 0.5f * e * e * inv_s2, llt);
        if (test_seg) {
          const float e0 = e + off;
          s1 += e0;
          s2 = fmaf(e0, e0, s2);
        }
      }
    };
    // several rows per pass, their loads issued before any arithmetic
    constexpr int U = PP <= 8 ? 4 : PP <= 16 ? 3 : 2;
    int n = n0;
    for (; n + U <= n1; n += U) {
      float x[U][PP], yv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        R.load(n + u, x[u]);
        yv[u] = R.y[n + u];
      }
#pragma unroll
      for (int u = 0; u < U; ++u) row(x[u], yv[u], n + u);
    }
    for (; n < n1; ++n) {
      float x[PP];
      R.load(n, x);
      row(x, R.y[n], n);
    }
    if (test_seg) lte += new_group_log_pred(s1, s2, n1 - n0, ls, lt);
    gz[gid] = tau * seg - z;                        // the likelihood's, then z_g ~ N(0, 1)
    dlt = fmaf(seg, off, dlt);
  }
#pragma unroll
  for (int j = 0; j < PP; ++j) g[j] = j < p ? warp_sum(acc[j]) - bt[j] * pb.beta_prec : 0.0f;
  dls = warp_sum(dls);
  dlt = warp_sum(dlt);
  glt = dlt - __expf(2.0f * lt) * pb.tau_prec + 1.0f;   // tau ~ half-N, with the log-Jacobian
  gls = dls - __expf(2.0f * ls) * pb.sigma_prec + 1.0f; // sigma ~ half-N, with the log-Jacobian
  if (LL) {
    ll_tr = warp_sum_d((double)llt);
    ll_te = warp_sum_d(lte);
  }
}

// One chain's trajectory of the hierarchical model (and, in accept mode,
// its Metropolis test and accumulators); zsh: the chain's shared-memory
// slice [z (G) | momentum (G) | gradient (G) | normals (d_pad)].
template <int PP>
__device__ __forceinline__ void traj_hier(const Problem &pb, const TrajArgs &t, const Rows<PP, false> &R, int c,
                                          int lane, float *zsh) {
  const int p = pb.p, G = pb.G, d = pb.d;
  const int jt = p + G, js = p + G + 1;            // log tau, log sigma
  float *zs = zsh, *rz = zsh + G, *gz = rz + G, *nrm = gz + G;
  const unsigned it = *t.iter;
  float eps = *t.eps;
  if (t.jitter > 0.0f) {
    const uint4 w = philox_at(t.seed, 0u, 0u, it, ST_JIT);
    eps = (float)((double)eps * (1.0 + (double)t.jitter * (2.0 * unit_from_word(w.x) - 1.0)));
  }
  if (!t.eval_only && c == 0 && lane == 0 && t.eps_iter) *t.eps_iter = eps;
  const FoldDesc fd = pb.folds[t.fold_base + c / t.L];
  const float *mvr = minv_row(t.minv, c, t.minv_every, t.minv_ld);
  const float *th0 = t.theta + (size_t)c * t.ld;
  float bt[PP], rb[PP], g[PP];
#pragma unroll
  for (int j = 0; j < PP; ++j) { bt[j] = j < p ? th0[j] : 0.0f; rb[j] = 0.0f; }
  float lt = th0[jt], ls = th0[js], rlt = 0.0f, rls = 0.0f, glt = 0.0f, gls = 0.0f;
  for (int gg = lane; gg < G; gg += 32) {          // each lane its own groups' z
    const int gid = pb.seg_grp[gg];
    zs[gid] = th0[p + gid];
  }
  double ll_tr = 0.0, ll_te = 0.0, H0 = 0.0;
  if (t.eval_only) {
    eval_hier<PP, true>(pb, R, fd, lane, bt, lt, ls, zs, gz, g, glt, gls, ll_tr, ll_te);
  } else {
    // momentum: the normals of coordinate quad q (Philox block q, as
    // k_begin) drawn by lane q mod 32 into shared memory, read by the
    // coordinate's lane; kinetic energy in FP64, first half kick and drift
    if (!t.r_given) {
      for (int q = lane; q < (d + 3) / 4; q += 32) {
        const uint4 w = philox_at(t.seed, (uint32_t)q, (uint32_t)(t.chain_base + c), it, t.stream);
        const float2 a0 = box_muller(w.x, w.y), a1 = box_muller(w.z, w.w);
        nrm[4 * q] = a0.x; nrm[4 * q + 1] = a0.y; nrm[4 * q + 2] = a1.x; nrm[4 * q + 3] = a1.y;
      }
      __syncwarp();
    }
    const float *g0 = t.grad + (size_t)c * t.ld;
    auto start = [&](int j, float v, float &tn, float &rh) -> float {
      const float m = mvr[j];
      const float r0 = t.r_given ? t.r_given[(size_t)c * t.ld + j] : (m > 0.0f ? nrm[j] / sqrtf(m) : 0.0f);
      rh = r0 + 0.5f * eps * g0[j];
      tn = v + eps * m * rh;
      return m * r0 * r0;
    };
    float kterm = 0.0f;     // this lane's kinetic-energy terms
#pragma unroll
    for (int j = 0; j < PP; ++j)
      if (j < p) {
        float tn, rh;
        const float k = start(j, bt[j], tn, rh);
        bt[j] = tn;
        rb[j] = rh;
        if (lane == (j & 31)) kterm += k;
      }
    {
      float tn, rh;
      const float k = start(jt, lt, tn, rh);
      lt = tn;
      rlt = rh;
      if (lane == (jt & 31)) kterm += k;
    }
    {
      float tn, rh;
      const float k = start(js, ls, tn, rh);
      ls = tn;
      rls = rh;
      if (lane == (js & 31)) kterm += k;
    }
    for (int gg = lane; gg < G; gg += 32) {
      const int gid = pb.seg_grp[gg];
      float tn, rh;
      kterm += start(p + gid, zs[gid], tn, rh);
      zs[gid] = tn;
      rz[gid] = rh;
    }
    H0 = -t.logp[c] + 0.5 * warp_sum_d((double)kterm);
    if (!t.accept && lane == 0) t.H0[c] = H0;
    for (int s = 1; s <= t.Lf; ++s) {
      const bool last = s == t.Lf;
      if (last) eval_hier<PP, true>(pb, R, fd, lane, bt, lt, ls, zs, gz, g, glt, gls, ll_tr, ll_te);
      else eval_hier<PP, false>(pb, R, fd, lane, bt, lt, ls, zs, gz, g, glt, gls, ll_tr, ll_te);
      const float kick = last ? 0.5f * eps : eps;
#pragma unroll
      for (int j = 0; j < PP; ++j)
        if (j < p) {
          rb[j] += kick * g[j];
          if (!last) bt[j] += eps * mvr[j] * rb[j];
        }
      rlt += kick * glt;
      rls += kick * gls;
      if (!last) {
        lt += eps * mvr[jt] * rlt;
        ls += eps * mvr[js] * rls;
      }
      for (int gg = lane; gg < G; gg += 32) {
        const int gid = pb.seg_grp[gg];
        rz[gid] += kick * gz[gid];
        if (!last) zs[gid] += eps * mvr[p + gid] * rz[gid];
      }
    }
  }
  // log prior (finish_chain<MV_HIER>'s terms): this lane's coordinates in
  // FP32, summed across lanes in FP64
  float lpt = 0.0f;
#pragma unroll
  for (int j = 0; j < PP; ++j)
    if (j < p && lane == (j & 31)) lpt += -0.5f * kLog2Pi - pb.log_beta_sd - 0.5f * bt[j] * bt[j] * pb.beta_prec;
  for (int gg = lane; gg < G; gg += 32) {
    const float z = zs[pb.seg_grp[gg]];
    lpt += -0.5f * kLog2Pi - 0.5f * z * z;
  }
  if (lane == (jt & 31))
    lpt += (float)kLog2D - 0.5f * kLog2Pi - pb.log_tau_sd - 0.5f * __expf(2.0f * lt) * pb.tau_prec + lt;
  if (lane == (js & 31))
    lpt += (float)kLog2D - 0.5f * kLog2Pi - pb.log_sigma_sd - 0.5f * __expf(2.0f * ls) * pb.sigma_prec + ls;
  const double logp1 = ll_tr + warp_sum_d((double)lpt);
  // every coordinate of a state out: beta, log tau, log sigma by lane j mod
  // 32, each z by its group's lane
  auto put = [&](float *th_o, float *r_o, float *g_o) {
    float *tho = th_o ? th_o + (size_t)c * t.ld : nullptr, *ro = r_o ? r_o + (size_t)c * t.ld : nullptr;
    float *go = g_o + (size_t)c * t.ld;
#pragma unroll
    for (int j = 0; j < PP; ++j)
      if (j < p && lane == (j & 31)) {
        if (tho) tho[j] = bt[j];
        if (ro) ro[j] = rb[j];
        go[j] = g[j];
      }
    if (lane == (jt & 31)) {
      if (tho) tho[jt] = lt;
      if (ro) ro[jt] = rlt;
      go[jt] = glt;
    }
    if (lane == (js & 31)) {
      if (tho) tho[js] = ls;
      if (ro) ro[js] = rls;
      go[js] = gls;
    }
    for (int gg = lane; gg < G; gg += 32) {
      const int gid = pb.seg_grp[gg];
      if (tho) tho[p + gid] = zs[gid];
      if (ro) ro[p + gid] = rz[gid];
      go[p + gid] = gz[gid];
    }
  };
  if (!t.accept) {
    if (t.eval_only) put(nullptr, nullptr, t.grad_p);
    else put(t.theta_p, t.r, t.grad_p);
    if (lane == 0) {
      t.logp_p[c] = logp1;
      t.shat_p[c] = ll_te;
    }
    return;
  }
  // accept mode: the Metropolis test in FP64 (as k_accept)
  float kt = 0.0f;
#pragma unroll
  for (int j = 0; j < PP; ++j)
    if (j < p && lane == (j & 31)) kt = fmaf(mvr[j] * rb[j], rb[j], kt);
  if (lane == (jt & 31)) kt = fmaf(mvr[jt] * rlt, rlt, kt);
  if (lane == (js & 31)) kt = fmaf(mvr[js] * rls, rls, kt);
  for (int gg = lane; gg < G; gg += 32) {
    const int gid = pb.seg_grp[gg];
    kt = fmaf(mvr[p + gid] * rz[gid], rz[gid], kt);
  }
  const double H1 = -logp1 + 0.5 * warp_sum_d((double)kt);
  const double dH = H1 - H0;
  const bool finite = isfinite(H1) && isfinite(dH);
  const int nw = blockDim.x >> 5, c0 = blockIdx.x * nw;
  double s_draw = 0.0;
  const bool acc = accept_batch(t, c - c0, lane, c0, min(nw, t.C - c0), dH, finite, logp1, ll_te, s_draw);
  if (acc) put(t.theta_w, nullptr, t.grad_w);
  if (t.accumulate) {
    const long long n_before = t.st->n_draws;
    accum_lags(t.acc, c, acov_x(t.acc, c, s_draw, n_before), n_before, lane);
  }
}

// Every chain reads every row at every step, so the CTA first copies X (PP
// columns per row), y and the group tables (segment offsets and groups)
// into shared memory when they fit beside the chains' slices (t.smem_rows;
// t.part_offset: bytes of the staged rows);
// the warps of a CTA (blockDim.x / 32, up to hier_warps_max(PP): 16 where
// the registers of a wider row would not fit) are its chains.
constexpr int hier_warps_max(int PP) { return PP <= 12 ? 16 : 8; }

template <int PP>
__global__ void __launch_bounds__(hier_warps_max(PP) * 32, 1) k_traj_hier(Problem pb, TrajArgs t) {
  extern __shared__ __align__(16) uint8_t hier_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  Rows<PP, false> R{pb.X, nullptr, pb.y, pb.p_pad};
  Problem pl = pb;
  if (t.smem_rows) {
    float *xs = reinterpret_cast<float *>(hier_smem);
    for (int i = threadIdx.x; i < pb.N * PP; i += blockDim.x) {
      const int n = i / PP, q = i - n * PP;
      xs[i] = __ldg(pb.X + (size_t)n * pb.p_pad + q);
    }
    float *ys = xs + (size_t)pb.N * PP;
    for (int i = threadIdx.x; i < pb.N; i += blockDim.x) ys[i] = __ldg(pb.y + i);
    // the group tables too: each segment's row loop waits on them
    int *go = reinterpret_cast<int *>(ys + pb.N), *sg = go + pb.G + 1;
    for (int i = threadIdx.x; i <= pb.G; i += blockDim.x) go[i] = __ldg(pb.grp_off + i);
    for (int i = threadIdx.x; i < pb.G; i += blockDim.x) sg[i] = __ldg(pb.seg_grp + i);
    __syncthreads();
    R.X = xs;
    R.y = ys;
    R.stride = PP;
    pl.grp_off = go;
    pl.seg_grp = sg;
  }
  float *zsh = reinterpret_cast<float *>(hier_smem + t.part_offset) + (size_t)warp * (3 * pb.G + pb.d_pad);
  const int c = blockIdx.x * nw + warp;
  if (c < t.C) {
    traj_hier<PP>(pl, t, R, c, lane, zsh);
  } else if (t.accept) {   // no chain: still meets the batched accept's barriers
    double sd;
    accept_batch(t, -1, lane, blockIdx.x * nw, min(nw, t.C - (int)blockIdx.x * nw), 0.0, false, 0.0, 0.0, sd);
  }
  if (t.accept) advance_counters(t);
}

// which register width PP serves p (p <= 32)
static int traj_pp(int p) {
  if (p <= 2) return 2;
  if (p <= 4) return 4;
  if (p <= 6) return 6;
  if (p <= 8) return 8;
  if (p <= 12) return 12;
  if (p <= 16) return 16;
  if (p <= 24) return 24;
  if (p <= 32) return 32;
  return -1;
}

// shared memory of the hierarchical kernel per chain: z, its momentum and
// gradient (G each) and the normals (d_pad)
static size_t traj_hier_slice(const Problem &pb) {
  return (3 * (size_t)pb.G + (size_t)pb.d_pad) * sizeof(float);
}
static size_t traj_hier_smem(const Problem &pb) { return (size_t)kTrajWarps * traj_hier_slice(pb); }
constexpr size_t kHierSmemMax = 227 * 1024 - 1024;   // opt-in shared memory per CTA, less the static part

bool traj_small_supported(const Problem &pb) {
  const bool rows = traj_pp(pb.p) > 0 && pb.p_pad >= traj_pp(pb.p) && pb.p_pad % 4 == 0;
  if (pb.variant == MV_HIER) return rows && traj_hier_smem(pb) <= kTrajSmemMax;
  return rows;
}

// the hierarchical kernel runs one warp per chain
int traj_max_wpc(const Problem &pb) { return pb.variant == MV_HIER ? 1 : 8; }

int traj_small_row_width(int p) { return traj_pp(p); }

// warps per chain without tuning: split each chain's rows until about eight
// warps per SM sub-partition are busy (148 SMs x 4), at most 8 per chain
int traj_default_wpc(int C) {
  int w = 1;
  while (w < 8 && (long long)C * w < 148LL * 4 * 8) w <<= 1;
  return w;
}

// shared memory of the staged rows (0: rows are read from global memory)
static size_t traj_rows_bytes(const Problem &pb, bool b16) {
  const size_t b = ((size_t)pb.N * traj_pp(pb.p) * (b16 ? 2 : 4) + 15) / 16 * 16 + (size_t)pb.N * 4;
  return b <= kTrajSmemMax ? b : 0;
}

template <int PP, int MV, bool XB16>
static cudaError_t launch_one(const Problem &pb, TrajArgs t, cudaStream_t st) {
  static bool attr_set = false;   // per process: the attribute belongs to the function
  if (t.wpc != 1 && t.wpc != 2 && t.wpc != 4 && t.wpc != 8) return cudaErrorInvalidValue;
  const size_t rows = traj_rows_bytes(pb, XB16);
  t.smem_rows = rows > 0 ? 1 : 0;
  t.part_offset = (int)((rows + 15) / 16 * 16);
  const size_t smem = (size_t)t.part_offset + 2 * kTrajWarps * 2 * sizeof(double) +
                      2 * kTrajWarps * (PP + 2) * sizeof(float);
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_traj_small<PP, MV, XB16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kTrajSmemMax + 4096));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int per_cta = kTrajWarps / t.wpc;
  const int grid = (t.C + per_cta - 1) / per_cta;
  k_traj_small<PP, MV, XB16><<<grid, kTrajWarps * 32, smem, st>>>(pb, t);
  return cudaGetLastError();
}

template <int PP>
static cudaError_t launch_hier(const Problem &pb, TrajArgs t, cudaStream_t st) {
  static bool attr_set = false;
  if (t.wpc != 1 || t.X16) return cudaErrorInvalidValue;
  // warps (chains) per CTA: enough for one wave over the 148 SMs, at most 16
  int nw = (int)std::min<long long>(hier_warps_max(PP), std::max<long long>(1, ((long long)t.C + 147) / 148));
  const size_t rows = ((size_t)pb.N * PP * sizeof(float) + (size_t)pb.N * sizeof(float) +
                       (2 * (size_t)pb.G + 1) * sizeof(int) + 15) / 16 * 16;
  const size_t slice = traj_hier_slice(pb);
  t.smem_rows = rows + (size_t)nw * slice <= kHierSmemMax ? 1 : 0;
  if (!t.smem_rows) nw = kTrajWarps;          // rows from global memory: 8 chains per CTA
  t.part_offset = t.smem_rows ? (int)rows : 0;
  const size_t smem = (size_t)t.part_offset + (size_t)nw * slice;
  if (smem > kHierSmemMax) return cudaErrorInvalidValue;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_traj_hier<PP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kHierSmemMax);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int grid = (t.C + nw - 1) / nw;
  k_traj_hier<PP><<<grid, nw * 32, smem, st>>>(pb, t);
  return cudaGetLastError();
}

template <int MV, bool XB16>
static cudaError_t launch_mv(const Problem &pb, const TrajArgs &t, cudaStream_t st) {
  switch (traj_pp(pb.p)) {
    case 2: return launch_one<2, MV, XB16>(pb, t, st);
    case 4: return launch_one<4, MV, XB16>(pb, t, st);
    case 6: return launch_one<6, MV, XB16>(pb, t, st);
    case 8: return launch_one<8, MV, XB16>(pb, t, st);
    case 12: return launch_one<12, MV, XB16>(pb, t, st);
    case 16: return launch_one<16, MV, XB16>(pb, t, st);
    case 24: return launch_one<24, MV, XB16>(pb, t, st);
    case 32: return launch_one<32, MV, XB16>(pb, t, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_traj_small(const Problem &pb, const TrajArgs &t, cudaStream_t st) {
  if (!traj_small_supported(pb) || t.C < 1) return cudaErrorInvalidValue;
  const bool b16 = t.X16 != nullptr;
  switch (pb.variant) {
    case MV_GAUSS_KNOWN: return b16 ? launch_mv<MV_GAUSS_KNOWN, true>(pb, t, st) : launch_mv<MV_GAUSS_KNOWN, false>(pb, t, st);
    case MV_GAUSS_LOGSIG: return b16 ? launch_mv<MV_GAUSS_LOGSIG, true>(pb, t, st) : launch_mv<MV_GAUSS_LOGSIG, false>(pb, t, st);
    case MV_LOGISTIC: return b16 ? launch_mv<MV_LOGISTIC, true>(pb, t, st) : launch_mv<MV_LOGISTIC, false>(pb, t, st);
    case MV_HIER:
      switch (traj_pp(pb.p)) {
        case 2: return launch_hier<2>(pb, t, st);
        case 4: return launch_hier<4>(pb, t, st);
        case 6: return launch_hier<6>(pb, t, st);
        case 8: return launch_hier<8>(pb, t, st);
        case 12: return launch_hier<12>(pb, t, st);
        case 16: return launch_hier<16>(pb, t, st);
        case 24: return launch_hier<24>(pb, t, st);
        case 32: return launch_hier<32>(pb, t, st);
        default: return cudaErrorInvalidValue;
      }
    default: return cudaErrorInvalidValue;
  }
}

// the BF16 form's copy of the design matrix: the first PP columns of X
// (FP32, row stride p_pad) rounded to bf16 once, row stride PP
__global__ void k_x_bf16_compact(long long N, int PP, int p_pad, const float *X, __nv_bfloat16 *X16) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N * PP) return;
  const long long n = i / PP;
  X16[i] = __float2bfloat16_rn(X[n * p_pad + (i - n * PP)]);
}

}  // namespace pcv
