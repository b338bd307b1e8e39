// k_grad_simt.cu -- FP32 CUDA-core kernels for one fold-masked log-posterior
// gradient evaluation of many chains, fused with the leapfrog momentum and
// position update (Section 3.3; masks of eq. mask-log-prob / mask-log-pred,
// Appendix B; the gradient is written by hand, no autodiff).
//
// Layout: a CTA owns a tile of 32 chains (lane = chain) and one of `splits`
// row ranges; its 8 warps stride over the rows of that range, so every X row
// is a warp-wide broadcast load and the per-chain masks are register compares
// against the chain's fold ranges.  Per-warp partial sums are reduced through
// shared memory; with several splits the partials go to a workspace and the
// last CTA of a tile (atomic ticket, no spinning) sums them in split order
// (deterministic) and applies the update.
#include "pcv_internal.cuh"

namespace pcv {

constexpr int kWarps = 8;

// Priors, gradient write-back and the leapfrog update for one chain.  `tot`
// holds the chain's likelihood-gradient sums indexed like theta; ll sums are
// passed in FP64.  Executed by one warp; lanes stride over dimensions.
template <int MV>
__device__ __forceinline__ void finish_chain(const Problem &pb, const GradArgs &a, int c,
                                             const float *tot, double ll_tr, double ll_te,
                                             int lane) {
  float *th = const_cast<float *>(a.theta) + (size_t)c * a.ld_theta;
  float *gr = a.grad + (size_t)c * a.ld_grad;
  float *rr = a.r ? a.r + (size_t)c * a.ld_theta : nullptr;
  const float eps = a.mode != MODE_NONE ? *a.eps : 0.0f;
  const float kick = a.mode == MODE_LAST_KICK ? 0.5f * eps : eps;
  double lp = 0.0;
  const int p = pb.p;
  for (int j = lane; j < pb.d; j += 32) {
    const float t = th[j];
    float g;
    if (j < p) {                                     // beta ~ N(0, sd^2)
      g = tot[j] - t * pb.beta_prec;
      lp += -0.5 * kLog2PiD - (double)pb.log_beta_sd - 0.5 * (double)t * t * pb.beta_prec;
    } else if (MV == MV_GAUSS_LOGSIG) {              // log sigma, sigma ~ half-N
      const float s2 = __expf(2.0f * t);
      g = tot[j] - s2 * pb.sigma_prec + 1.0f;
      lp += kLog2D - 0.5 * kLog2PiD - pb.log_sigma_sd - 0.5 * (double)s2 * pb.sigma_prec + t;
    } else {                                         // hierarchical extras
      const int G = pb.G;
      if (j < p + G) {                               // z_g ~ N(0, 1)
        g = tot[j] - t;
        lp += -0.5 * kLog2PiD - 0.5 * (double)t * t;
      } else if (j == p + G) {                       // log tau, tau ~ half-N
        const float v2 = __expf(2.0f * t);
        g = tot[j] - v2 * pb.tau_prec + 1.0f;
        lp += kLog2D - 0.5 * kLog2PiD - pb.log_tau_sd - 0.5 * (double)v2 * pb.tau_prec + t;
      } else {                                       // log sigma, sigma ~ half-N
        const float v2 = __expf(2.0f * t);
        g = tot[j] - v2 * pb.sigma_prec + 1.0f;
        lp += kLog2D - 0.5 * kLog2PiD - pb.log_sigma_sd - 0.5 * (double)v2 * pb.sigma_prec + t;
      }
    }
    gr[j] = g;
    if (a.mode != MODE_NONE) {
      const float rj = rr[j] + kick * g;
      rr[j] = rj;
      if (a.mode == MODE_KICK_DRIFT) {
        const float tn = t + eps * minv_row(a.minv, c, a.minv_every, a.minv_ld)[j] * rj;
        th[j] = tn;
        if (a.shadow_hi) {
          const __nv_bfloat16 hi = __float2bfloat16_rn(tn);
          a.shadow_hi[(size_t)c * a.ld_shadow + j] = hi;
          a.shadow_lo[(size_t)c * a.ld_shadow + j] = __float2bfloat16_rn(tn - __bfloat162float(hi));
        }
      }
    }
  }
  if (a.need_ll) {
    lp = warp_sum_d(lp);
    if (lane == 0) {
      a.logp[c] = ll_tr + lp;
      a.shat[c] = ll_te;
    }
  }
}

// ---------------------------------------------------------------------------
// Flat models (Gaussian linear / AR, logistic): theta = beta[p] (+ log sigma)
// ---------------------------------------------------------------------------
template <int PP, int MV>
__global__ void __launch_bounds__(kWarps * 32) k_grad_flat(Problem pb, GradArgs a) {
  constexpr int S = PP + 4;               // slots: PP grads, dlogsig, ll_tr, ll_te, pad
  __shared__ float red[kWarps][32][S + 1];
  __shared__ double lls[2][32];
  __shared__ int is_last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x / a.splits, split = blockIdx.x - tile * a.splits;
  const int c = tile * 32 + lane;
  const bool valid = c < a.C;
  const int p = pb.p;

  float th[PP];
  const float *tp = a.theta + (size_t)(valid ? c : 0) * a.ld_theta;
#pragma unroll
  for (int j = 0; j < PP; ++j) th[j] = (valid && j < p) ? tp[j] : 0.0f;
  float logsig = 0.0f, inv_s2 = 1.0f;
  if (MV == MV_GAUSS_KNOWN) {
    logsig = logf(pb.sigma_known);
    inv_s2 = 1.0f / (pb.sigma_known * pb.sigma_known);
  } else if (MV == MV_GAUSS_LOGSIG) {
    logsig = valid ? tp[p] : 0.0f;
    inv_s2 = expf(-2.0f * logsig);
  }
  FoldDesc fd = {0, 0, 0, 0};
  if (valid) fd = pb.folds[fold_of_chain(a, c)];

  const int r0 = (int)((long long)pb.N * split / a.splits);
  const int r1 = (int)((long long)pb.N * (split + 1) / a.splits);
  float g[PP];
#pragma unroll
  for (int j = 0; j < PP; ++j) g[j] = 0.0f;
  float ll_tr = 0.0f, ll_te = 0.0f, dls = 0.0f;

  for (int n = r0 + warp; n < r1; n += kWarps) {
    float x[PP];
    const float4 *xr = reinterpret_cast<const float4 *>(pb.X + (size_t)n * pb.p_pad);
#pragma unroll
    for (int q = 0; q < PP / 4; ++q) {
      const float4 v = __ldg(xr + q);
      x[4 * q] = v.x; x[4 * q + 1] = v.y; x[4 * q + 2] = v.z; x[4 * q + 3] = v.w;
    }
    float eta = 0.0f;
#pragma unroll
    for (int j = 0; j < PP; ++j) eta = fmaf(th[j], x[j], eta);
    const float yv = __ldg(pb.y + n);
    const float tr = (n < fd.excl_lo || n >= fd.excl_hi) ? 1.0f : 0.0f;
    float ll = 0.0f, dll;
    if (MV == MV_LOGISTIC) {
      dll = yv - 1.0f / (1.0f + __expf(-eta));
      if (a.need_ll) ll = yv * eta - softplusf(eta);
    } else {
      const float e = yv - eta;
      dll = e * inv_s2;
      if (a.need_ll) ll = -0.5f * kLog2Pi - logsig - 0.5f * e * e * inv_s2;
      if (MV == MV_GAUSS_LOGSIG) dls = fmaf(tr, e * e * inv_s2 - 1.0f, dls);
    }
    const float wv = dll * tr;
#pragma unroll
    for (int j = 0; j < PP; ++j) g[j] = fmaf(wv, x[j], g[j]);
    if (a.need_ll) {
      const float te = (n >= fd.test_lo && n < fd.test_hi) ? 1.0f : 0.0f;
      ll_tr = fmaf(tr, ll, ll_tr);
      ll_te = fmaf(te, ll, ll_te);
    }
  }
#pragma unroll
  for (int j = 0; j < PP; ++j) red[warp][lane][j] = g[j];
  red[warp][lane][PP] = dls;
  red[warp][lane][PP + 1] = ll_tr;
  red[warp][lane][PP + 2] = ll_te;
  red[warp][lane][PP + 3] = 0.0f;
  __syncthreads();
  // sum over warps: thread t handles (chain t / S, slot t % S)
  for (int t = threadIdx.x; t < 32 * S; t += blockDim.x) {
    const int cl = t / S, sl = t - cl * S;
    float s = 0.0f;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += red[w][cl][sl];
    red[0][cl][sl] = s;
  }
  __syncthreads();

  if (a.splits > 1) {
    float *mine = a.ws + ((size_t)tile * a.splits + split) * 32 * a.ws_stride;
    for (int t = threadIdx.x; t < 32 * S; t += blockDim.x) {
      const int cl = t / S, sl = t - cl * S;
      mine[cl * a.ws_stride + sl] = red[0][cl][sl];
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned prev = atomicAdd(a.tickets + tile, 1u);
      is_last = (prev == (unsigned)a.splits - 1);
      if (is_last) a.tickets[tile] = 0u;   // ready for the next launch
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    const float *base = a.ws + (size_t)tile * a.splits * 32 * a.ws_stride;
    for (int t = threadIdx.x; t < 32 * S; t += blockDim.x) {
      const int cl = t / S, sl = t - cl * S;
      if (sl == PP + 1 || sl == PP + 2) {
        double s = 0.0;
        for (int q = 0; q < a.splits; ++q)
          s += (double)__ldcg(base + ((size_t)q * 32 + cl) * a.ws_stride + sl);
        lls[sl - PP - 1][cl] = s;
      } else {
        float s = 0.0f;
        for (int q = 0; q < a.splits; ++q) s += __ldcg(base + ((size_t)q * 32 + cl) * a.ws_stride + sl);
        red[0][cl][sl] = s;
      }
    }
  } else if (threadIdx.x < 32) {
    lls[0][threadIdx.x] = (double)red[0][threadIdx.x][PP + 1];
    lls[1][threadIdx.x] = (double)red[0][threadIdx.x][PP + 2];
  }
  __syncthreads();
  for (int cl = warp; cl < 32; cl += kWarps) {
    const int cc = tile * 32 + cl;
    if (cc >= a.C) continue;
    float tot[PP + 1];
#pragma unroll
    for (int j = 0; j < PP; ++j) tot[j] = red[0][cl][j];
    tot[PP] = 0.0f;
    if (MV == MV_GAUSS_LOGSIG) tot[p] = red[0][cl][PP];   // d/dlog sigma of the likelihood
    finish_chain<MV>(pb, a, cc, tot, lls[0][cl], lls[1][cl], lane);
  }
}

// ---------------------------------------------------------------------------
// Hierarchical varying-intercept model: theta = beta[p], z[G], log tau,
// log sigma.  Rows are sorted so that each group is one contiguous segment;
// splits and warps own whole segments, so the segmented sums over a group's
// rows need no atomics.
//
// Every CTA writes its partial in theta layout into the workspace
// (ws_stride = d_pad + 4; slot d_pad / d_pad+1 = ll_tr / ll_te); z slots are
// written only for the groups the CTA owns.  The finishing CTA sums the
// shared slots over splits and takes each z slot from its owner split.
template <int PP>
__global__ void __launch_bounds__(kWarps * 32) k_grad_hier(Problem pb, GradArgs a) {
  constexpr int S = PP + 4;        // beta grads, dlogtau, dlogsig, ll_tr, ll_te
  extern __shared__ float smem[];
  float *red = smem;                                  // [kWarps][32][S]
  __shared__ int is_last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x / a.splits, split = blockIdx.x - tile * a.splits;
  const int c = tile * 32 + lane;
  const bool valid = c < a.C;
  const int p = pb.p, G = pb.G, dp = pb.d_pad;
  const int g0 = (int)((long long)G * split / a.splits);
  const int g1 = (int)((long long)G * (split + 1) / a.splits);
  float *mine = a.ws + ((size_t)tile * a.splits + split) * 32 * a.ws_stride;

  float th[PP];
  const float *tp = a.theta + (size_t)(valid ? c : 0) * a.ld_theta;
#pragma unroll
  for (int j = 0; j < PP; ++j) th[j] = (valid && j < p) ? tp[j] : 0.0f;
  const float logtau = valid ? tp[p + G] : 0.0f;
  const float logsig = valid ? tp[p + G + 1] : 0.0f;
  const float tau = expf(logtau);
  const float inv_s2 = expf(-2.0f * logsig);
  FoldDesc fd = {0, 0, 0, 0};
  if (valid) fd = pb.folds[fold_of_chain(a, c)];

  float g[PP];
#pragma unroll
  for (int j = 0; j < PP; ++j) g[j] = 0.0f;
  float ll_tr = 0.0f, ll_te = 0.0f, dls = 0.0f, dlt = 0.0f;

  for (int gg = g0 + warp; gg < g1; gg += kWarps) {   // gg: row segment of one group
    const int gid = __ldg(pb.seg_grp + gg);
    const float z = valid ? tp[p + gid] : 0.0f;
    const float off = tau * z;
    const int n0 = __ldg(pb.grp_off + gg), n1 = __ldg(pb.grp_off + gg + 1);
    // a group held out by this chain's fold has no training rows there: it
    // is a new group, scored by the group-level predictive (eq. group-marg)
    // from the sums of e0 = y - x beta over its rows
    const bool test_seg = a.need_ll && valid && n1 > n0 && n0 >= fd.test_lo && n1 <= fd.test_hi;
    float s1 = 0.0f, s2 = 0.0f;
    float seg = 0.0f;
    for (int n = n0; n < n1; ++n) {
      float x[PP];
      const float4 *xr = reinterpret_cast<const float4 *>(pb.X + (size_t)n * pb.p_pad);
#pragma unroll
      for (int q = 0; q < PP / 4; ++q) {
        const float4 v = __ldg(xr + q);
        x[4 * q] = v.x; x[4 * q + 1] = v.y; x[4 * q + 2] = v.z; x[4 * q + 3] = v.w;
      }
      float eta = off;
#pragma unroll
      for (int j = 0; j < PP; ++j) eta = fmaf(th[j], x[j], eta);
      const float e = __ldg(pb.y + n) - eta;
      const float tr = (n < fd.excl_lo || n >= fd.excl_hi) ? 1.0f : 0.0f;
      const float wv = e * inv_s2 * tr;
#pragma unroll
      for (int j = 0; j < PP; ++j) g[j] = fmaf(wv, x[j], g[j]);
      seg += wv;
      dls = fmaf(tr, e * e * inv_s2 - 1.0f, dls);
      if (a.need_ll) {
        const float ll = -0.5f * kLog2Pi - logsig - 0.5f * e * e * inv_s2;
        ll_tr = fmaf(tr, ll, ll_tr);
        if (test_seg) {
          const float e0 = e + off;
          s1 += e0;
          s2 = fmaf(e0, e0, s2);
        }
      }
    }
    if (test_seg) ll_te += (float)new_group_log_pred(s1, s2, n1 - n0, logsig, logtau);
    mine[lane * a.ws_stride + p + gid] = tau * seg;  // d/dz_g of the likelihood
    dlt = fmaf(seg, off, dlt);                        // d/dlog tau: sum_g seg_g tau z_g
  }
  float *rw = red + (warp * 32 + lane) * S;
#pragma unroll
  for (int j = 0; j < PP; ++j) rw[j] = g[j];
  rw[PP] = dlt;
  rw[PP + 1] = dls;
  rw[PP + 2] = ll_tr;
  rw[PP + 3] = ll_te;
  __syncthreads();
  for (int t = threadIdx.x; t < 32 * S; t += blockDim.x) {
    const int cl = t / S, sl = t - cl * S;
    if (sl < PP && sl >= p) continue;
    float s = 0.0f;
    for (int w = 0; w < kWarps; ++w) s += red[(w * 32 + cl) * S + sl];
    const int dst = sl < PP ? sl : (sl == PP ? p + G : sl == PP + 1 ? p + G + 1 : dp + (sl - PP - 2));
    mine[cl * a.ws_stride + dst] = s;
  }
  __threadfence();
  __syncthreads();
  if (a.splits > 1) {
    if (threadIdx.x == 0) {
      const unsigned prev = atomicAdd(a.tickets + tile, 1u);
      is_last = (prev == (unsigned)a.splits - 1);
      if (is_last) a.tickets[tile] = 0u;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
  }
  float *base = a.ws + (size_t)tile * a.splits * 32 * a.ws_stride;
  for (int cl = warp; cl < 32; cl += kWarps) {
    const int cc = tile * 32 + cl;
    if (cc >= a.C) continue;
    float *row0 = base + (size_t)cl * a.ws_stride;
    double ltr = 0.0, lte = 0.0;
    if (a.splits > 1) {
      for (int j = lane; j < dp; j += 32) {
        if (j >= p && j < p + G) {
          // owner split of the group's segment sg: the largest s with
          // floor(G s / splits) <= sg
          const int sg = __ldg(pb.grp_seg + (j - p));
          int s = (int)(((long long)(sg + 1) * a.splits + G - 1) / G) - 1;
          if (s > a.splits - 1) s = a.splits - 1;
          if (s != 0) row0[j] = __ldcg(base + ((size_t)s * 32 + cl) * a.ws_stride + j);
        } else if (j < p || j == p + G || j == p + G + 1) {
          float s = __ldcg(row0 + j);
          for (int q = 1; q < a.splits; ++q) s += __ldcg(base + ((size_t)q * 32 + cl) * a.ws_stride + j);
          row0[j] = s;
        }
      }
      for (int q = lane; q < a.splits; q += 32) {
        ltr += (double)__ldcg(base + ((size_t)q * 32 + cl) * a.ws_stride + dp);
        lte += (double)__ldcg(base + ((size_t)q * 32 + cl) * a.ws_stride + dp + 1);
      }
      ltr = warp_sum_d(ltr);
      lte = warp_sum_d(lte);
      __syncwarp();
    } else {
      ltr = (double)__ldcg(row0 + dp);
      lte = (double)__ldcg(row0 + dp + 1);
    }
    __threadfence_block();
    finish_chain<MV_HIER>(pb, a, cc, row0, ltr, lte, lane);
  }
}


// ---------------------------------------------------------------------------
// Large p (33..128), flat models, FP32 CUDA cores.  A CTA owns a tile of 64
// chains and one of `splits` row ranges; per 64-row chunk it computes
//   S = Theta_tile . X_chunk^T   (4 chains x 4 rows per thread, float4 loads along K)
//   R = mask .* dlogp/deta       (shared memory)
//   G += R . X_chunk             (4 chains x 8 dims per thread, kept for the range)
// then combines split-N partials like the kernels above.  Rows of the
// shared tiles are 132 floats (528 B = 16 mod 128 B): the float4 loads of
// 8 consecutive rows, or of 8 consecutive dim groups, hit distinct banks.
// ---------------------------------------------------------------------------
constexpr int kBigTileC = 64, kBigRows = 64, kBigLd = 132, kBigLdr = 68;

template <int MV>
__global__ void __launch_bounds__(256) k_grad_bigp(Problem pb, GradArgs a, int pp) {
  extern __shared__ __align__(16) float sm_big[];
  float *th_s = sm_big;                             // [64][132] theta (0 beyond p)
  float *xs = th_s + kBigTileC * kBigLd;            // [64][132] X chunk (0 beyond p and nr)
  float *rs = xs + kBigRows * kBigLd;               // [64][68]  residual, chains x rows
  float *ys = rs + kBigTileC * kBigLdr;             // [64]
  float *lls = ys + kBigRows;                       // [3][64][16]: ll_tr, ll_te, dlogsig partials
  __shared__ int is_last;
  __shared__ double lld[2][kBigTileC];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int tile = blockIdx.x / a.splits, split = blockIdx.x - tile * a.splits;
  const int c0 = tile * kBigTileC;
  const int p = pb.p;
  for (int q = t; q < kBigTileC * 32; q += 256) {
    const int cl = q >> 5, j4 = (q & 31) * 4;
    const int c = c0 + cl;
    float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (c < a.C) {
      const float *tp = a.theta + (size_t)c * a.ld_theta;
      if (j4 < p) v.x = tp[j4];
      if (j4 + 1 < p) v.y = tp[j4 + 1];
      if (j4 + 2 < p) v.z = tp[j4 + 2];
      if (j4 + 3 < p) v.w = tp[j4 + 3];
    }
    *reinterpret_cast<float4 *>(th_s + cl * kBigLd + j4) = v;
  }
  // thread roles: chains 4 cg .. 4 cg + 3 in both GEMMs; rows rg + 16 j
  // (j < 4) in the first, dims 4 dg .. 4 dg + 3 and 64 + 4 dg .. in the second
  const int cg = t >> 4, rg = t & 15, dg = t & 15;
  float logsig[4], inv_s2[4];
  FoldDesc fd[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int c = c0 + 4 * cg + i;
    const bool valid = c < a.C;
    fd[i] = valid ? pb.folds[fold_of_chain(a, c)] : FoldDesc{0, 0, 0, 0};
    logsig[i] = 0.0f;
    inv_s2[i] = 1.0f;
    if (MV == MV_GAUSS_KNOWN) {
      logsig[i] = logf(pb.sigma_known);
      inv_s2[i] = 1.0f / (pb.sigma_known * pb.sigma_known);
    } else if (MV == MV_GAUSS_LOGSIG) {
      logsig[i] = valid ? a.theta[(size_t)c * a.ld_theta + p] : 0.0f;
      inv_s2[i] = expf(-2.0f * logsig[i]);
    }
  }
  float acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[i][k] = 0.0f;
  float ll_tr[4] = {0.0f, 0.0f, 0.0f, 0.0f}, ll_te[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  float dls[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  const int r0 = (int)((long long)pb.N * split / a.splits);
  const int r1 = (int)((long long)pb.N * (split + 1) / a.splits);
  __syncthreads();
  for (int n0 = r0; n0 < r1; n0 += kBigRows) {
    const int nr = min(kBigRows, r1 - n0);
    for (int q = t; q < kBigRows * 32; q += 256) {
      const int rr = q >> 5, j4 = (q & 31) * 4;
      float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (rr < nr && j4 < pb.p_pad) v = *reinterpret_cast<const float4 *>(pb.X + (size_t)(n0 + rr) * pb.p_pad + j4);
      *reinterpret_cast<float4 *>(xs + rr * kBigLd + j4) = v;
    }
    if (t < kBigRows) ys[t] = t < nr ? pb.y[n0 + t] : 0.0f;
    __syncthreads();
    // ---- S: chains 4 cg + i, rows rg + 16 j
    float sv[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) sv[i][j] = 0.0f;
    for (int k = 0; k < pp; k += 4) {
      float4 av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = *reinterpret_cast<const float4 *>(th_s + (4 * cg + i) * kBigLd + k);
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = *reinterpret_cast<const float4 *>(xs + (rg + 16 * j) * kBigLd + k);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float v = sv[i][j];
          v = fmaf(av[i].x, bv[j].x, v);
          v = fmaf(av[i].y, bv[j].y, v);
          v = fmaf(av[i].z, bv[j].z, v);
          sv[i][j] = fmaf(av[i].w, bv[j].w, v);
        }
    }
    // ---- masked residual dlogp/deta (and log likelihoods on evaluation steps)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int rr = rg + 16 * j, n = n0 + rr;
        const float eta = sv[i][j], yv = ys[rr];
        const bool in_rows = rr < nr;
        const float tr = (in_rows && (n < fd[i].excl_lo || n >= fd[i].excl_hi)) ? 1.0f : 0.0f;
        float dll, ll = 0.0f;
        if (MV == MV_LOGISTIC) {
          dll = yv - 1.0f / (1.0f + __expf(-eta));
          if (a.need_ll) ll = yv * eta - softplusf(eta);
        } else {
          const float e = yv - eta;
          dll = e * inv_s2[i];
          if (a.need_ll) ll = -0.5f * kLog2Pi - logsig[i] - 0.5f * e * e * inv_s2[i];
          if (MV == MV_GAUSS_LOGSIG) dls[i] = fmaf(tr, e * e * inv_s2[i] - 1.0f, dls[i]);
        }
        rs[(4 * cg + i) * kBigLdr + rr] = dll * tr;
        if (a.need_ll) {
          const float te = (in_rows && n >= fd[i].test_lo && n < fd[i].test_hi) ? 1.0f : 0.0f;
          ll_tr[i] = fmaf(tr, ll, ll_tr[i]);
          ll_te[i] = fmaf(te, ll, ll_te[i]);
        }
      }
    }
    __syncthreads();
    // ---- G[4 cg + i][dims] += R[4 cg + i][row] X[row][dims] (rows beyond nr
    // carry R = 0 and X = 0)
    for (int row = 0; row < kBigRows; row += 4) {
      float4 rv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) rv[i] = *reinterpret_cast<const float4 *>(rs + (4 * cg + i) * kBigLdr + row);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 x0 = *reinterpret_cast<const float4 *>(xs + (row + u) * kBigLd + 4 * dg);
        const float4 x1 = *reinterpret_cast<const float4 *>(xs + (row + u) * kBigLd + 64 + 4 * dg);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float r = u == 0 ? rv[i].x : u == 1 ? rv[i].y : u == 2 ? rv[i].z : rv[i].w;
          acc[i][0] = fmaf(r, x0.x, acc[i][0]);
          acc[i][1] = fmaf(r, x0.y, acc[i][1]);
          acc[i][2] = fmaf(r, x0.z, acc[i][2]);
          acc[i][3] = fmaf(r, x0.w, acc[i][3]);
          acc[i][4] = fmaf(r, x1.x, acc[i][4]);
          acc[i][5] = fmaf(r, x1.y, acc[i][5]);
          acc[i][6] = fmaf(r, x1.z, acc[i][6]);
          acc[i][7] = fmaf(r, x1.w, acc[i][7]);
        }
      }
    }
    __syncthreads();
  }
  // per-chain likelihood sums: the 16 threads of a chain group leave their
  // partials in shared memory; one thread per chain adds them in order
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int cl = 4 * cg + i;
    lls[(0 * kBigTileC + cl) * 16 + rg] = ll_tr[i];
    lls[(1 * kBigTileC + cl) * 16 + rg] = ll_te[i];
    lls[(2 * kBigTileC + cl) * 16 + rg] = dls[i];
  }
  __syncthreads();
  float sums[3] = {0.0f, 0.0f, 0.0f};
  if (t < kBigTileC) {
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int v = 0; v < 16; ++v) sums[q] += lls[(q * kBigTileC + t) * 16 + v];
  }
  // partial of this CTA: [64 chains][ws_stride]: grads, slot pp dlogsig,
  // pp+1 ll_tr, pp+2 ll_te
  float *mine = a.ws + ((size_t)tile * a.splits + split) * kBigTileC * a.ws_stride;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int dim = (k < 4 ? 4 * dg : 64 + 4 * dg) + (k & 3);
      if (dim < pp) mine[(4 * cg + i) * a.ws_stride + dim] = acc[i][k];
    }
  if (t < kBigTileC) {
    mine[t * a.ws_stride + pp] = sums[2];
    mine[t * a.ws_stride + pp + 1] = sums[0];
    mine[t * a.ws_stride + pp + 2] = sums[1];
  }
  __threadfence();
  __syncthreads();
  if (a.splits > 1) {
    if (t == 0) {
      const unsigned prev = atomicAdd(a.tickets + tile, 1u);
      is_last = (prev == (unsigned)a.splits - 1);
      if (is_last) a.tickets[tile] = 0u;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
  }
  // sum the splits' partials in split order; likelihood sums in FP64
  float *tot = xs;                                  // [64][pp + 4], reuses the X tile
  const int ts = pp + 4;
  const float *base = a.ws + (size_t)tile * a.splits * kBigTileC * a.ws_stride;
  for (int q = t; q < kBigTileC * (pp + 3); q += 256) {
    const int cl = q / (pp + 3), j = q - cl * (pp + 3);
    if (j > pp) {
      double sacc = 0.0;
      for (int s2 = 0; s2 < a.splits; ++s2)
        sacc += (double)__ldcg(base + ((size_t)s2 * kBigTileC + cl) * a.ws_stride + j);
      lld[j - pp - 1][cl] = sacc;
    } else {
      float sacc = 0.0f;
      for (int s2 = 0; s2 < a.splits; ++s2) sacc += __ldcg(base + ((size_t)s2 * kBigTileC + cl) * a.ws_stride + j);
      tot[cl * ts + j] = sacc;
    }
  }
  __syncthreads();
  for (int cl = warp; cl < kBigTileC; cl += 8) {
    const int c = c0 + cl;
    if (c >= a.C) continue;
    float *row = tot + cl * ts;
    if (MV == MV_GAUSS_LOGSIG) {
      const float d = row[pp];
      __syncwarp();
      if (lane == 0) row[p] = d;                    // d/dlog sigma at index p
      __syncwarp();
    }
    finish_chain<MV>(pb, a, c, row, lld[0][cl], lld[1][cl], lane);
  }
}

int simt_chain_tile(int p) { return simt_flat_pp(p) > 0 ? 32 : kBigTileC; }

size_t bigp_smem_bytes(int pp) {
  (void)pp;
  return sizeof(float) * ((size_t)kBigTileC * kBigLd + (size_t)kBigRows * kBigLd + (size_t)kBigTileC * kBigLdr +
                          kBigRows + 3 * kBigTileC * 16);
}

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------
template <int MV>
static cudaError_t launch_flat_mv(const Problem &pb, const GradArgs &a, int PP, cudaStream_t st) {
  const int tiles = (a.C + 31) / 32;
  dim3 grid(tiles * a.splits), block(kWarps * 32);
  switch (PP) {
    case 4: k_grad_flat<4, MV><<<grid, block, 0, st>>>(pb, a); break;
    case 8: k_grad_flat<8, MV><<<grid, block, 0, st>>>(pb, a); break;
    case 12: k_grad_flat<12, MV><<<grid, block, 0, st>>>(pb, a); break;
    case 16: k_grad_flat<16, MV><<<grid, block, 0, st>>>(pb, a); break;
    case 24: k_grad_flat<24, MV><<<grid, block, 0, st>>>(pb, a); break;
    case 32: k_grad_flat<32, MV><<<grid, block, 0, st>>>(pb, a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int simt_flat_pp(int p) {
  if (p <= 4) return 4;
  if (p <= 8) return 8;
  if (p <= 12) return 12;
  if (p <= 16) return 16;
  if (p <= 24) return 24;
  if (p <= 32) return 32;
  return -1;
}

size_t hier_smem_bytes(int PP, int, int) {
  return (size_t)kWarps * 32 * (PP + 4) * sizeof(float);
}

template <int MV>
static cudaError_t launch_bigp_mv(const Problem &pb, const GradArgs &a, cudaStream_t st) {
  const int pp = (pb.p + 3) / 4 * 4;
  const int tiles = (a.C + kBigTileC - 1) / kBigTileC;
  const size_t sm = bigp_smem_bytes(pp);
  cudaError_t e = cudaFuncSetAttribute(k_grad_bigp<MV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_grad_bigp<MV><<<tiles * a.splits, 256, sm, st>>>(pb, a, pp);
  return cudaGetLastError();
}

cudaError_t launch_grad_simt(const Problem &pb, const GradArgs &a, cudaStream_t st) {
  const int PP = simt_flat_pp(pb.p);
  if (PP < 0) {
    if (pb.p > 128) return cudaErrorInvalidValue;
    switch (pb.variant) {
      case MV_GAUSS_KNOWN: return launch_bigp_mv<MV_GAUSS_KNOWN>(pb, a, st);
      case MV_GAUSS_LOGSIG: return launch_bigp_mv<MV_GAUSS_LOGSIG>(pb, a, st);
      case MV_LOGISTIC: return launch_bigp_mv<MV_LOGISTIC>(pb, a, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (pb.variant) {
    case MV_GAUSS_KNOWN: return launch_flat_mv<MV_GAUSS_KNOWN>(pb, a, PP, st);
    case MV_GAUSS_LOGSIG: return launch_flat_mv<MV_GAUSS_LOGSIG>(pb, a, PP, st);
    case MV_LOGISTIC: return launch_flat_mv<MV_LOGISTIC>(pb, a, PP, st);
    case MV_HIER: {
      const int tiles = (a.C + 31) / 32;
      dim3 grid(tiles * a.splits), block(kWarps * 32);
      const size_t sm = hier_smem_bytes(PP, pb.G, a.splits);
      switch (PP) {
        case 4: k_grad_hier<4><<<grid, block, sm, st>>>(pb, a); break;
        case 8: k_grad_hier<8><<<grid, block, sm, st>>>(pb, a); break;
        case 12: k_grad_hier<12><<<grid, block, sm, st>>>(pb, a); break;
        case 16: k_grad_hier<16><<<grid, block, sm, st>>>(pb, a); break;
        case 24: k_grad_hier<24><<<grid, block, sm, st>>>(pb, a); break;
        case 32: k_grad_hier<32><<<grid, block, sm, st>>>(pb, a); break;
        default: return cudaErrorInvalidValue;
      }
      return cudaGetLastError();
    }
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pcv
