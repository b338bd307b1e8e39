// k_hmc.cu -- per-chain HMC kernels around the fused gradient step:
//   k_begin     momentum draw (Philox4x32-10 + Box-Muller), H0, first
//               half-kick and drift of the leapfrog (Section 3.3)
//   k_accept    FP64 Hamiltonian difference and Metropolis accept, the
//               divergence count, and the online accumulators of
//               Algorithm A2 (Appendix A.1) updated in place
//   k_fd_adapt  full-data dual averaging of the step size and the windowed
//               diagonal mass estimate (warm-up reuse, Section 3.1)
//   k_finalize  per-fold estimators: elpd, MCSE (eq. bmvar, mc-var), ESS
//               (Section 4.1), R-hat / split R-hat (eq. rhat), Geyer ESS
// All accept-test and accumulator arithmetic is FP64.
#include "pcv_internal.cuh"
#include "pcv_accum.cuh"

namespace pcv {

// FP32 rounded to TF32 (nearest, ties away from zero)
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// ---------------------------------------------------------------------------
// k_begin: one warp per chain
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_begin(BeginArgs a) {
  __shared__ float eps_s;
  const int lane = threadIdx.x & 31;
  const int gsz = begin_lanes_per_chain(a.d), sl = lane & (gsz - 1);
  const int c = (blockIdx.x * 8 + (threadIdx.x >> 5)) * (32 / gsz) + lane / gsz;
  const unsigned it = *a.iter;
  // this iteration's step size: the nominal one, or (fold chains) jittered
  // by one uniform per iteration shared by every chain (stream ST_JIT);
  // formed once per block (FP64 work is slow on this part)
  if (threadIdx.x == 0) {
    float e = *a.eps;
    if (a.jitter > 0.0f) {
      const uint4 w = philox_at(a.seed, 0u, 0u, it, ST_JIT);
      e = (float)((double)e * (1.0 + (double)a.jitter * (2.0 * unit_from_word(w.x) - 1.0)));
    }
    eps_s = e;
    if (a.eps_iter && blockIdx.x == 0) *a.eps_iter = e;
  }
  __syncthreads();
  const bool valid = c < a.C;
  const float eps = eps_s;
  const float *th = a.theta + (size_t)c * a.ld;
  const float *g = a.grad + (size_t)c * a.ld;
  F2 kin = {0.0f, 0.0f};                    // kinetic energy r' M^-1 r, as an FP32 pair
  for (int q = sl; valid && 4 * q < a.d; q += gsz) {
    float z[4];
    if (a.r_given) {
#pragma unroll
      for (int e = 0; e < 4; ++e) z[e] = 0.0f;
    } else {
      const uint4 w = philox_at(a.seed, (uint32_t)q, (uint32_t)(a.chain_base + c), it, a.stream);
      const float2 p0 = box_muller(w.x, w.y), p1 = box_muller(w.z, w.w);
      z[0] = p0.x; z[1] = p0.y; z[2] = p1.x; z[3] = p1.y;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int j = 4 * q + e;
      if (j >= a.d) break;
      const float mv = minv_row(a.minv, c, a.minv_every, a.minv_ld)[j];
      // a coordinate with inverse mass 0 (masked covariate) is held: r = 0
      const float r0 = a.r_given ? a.r_given[(size_t)c * a.ld + j] : (mv > 0.0f ? z[e] / sqrtf(mv) : 0.0f);
      f2_add_mr2(kin, mv, r0);
      const float rh = r0 + 0.5f * eps * g[j];
      const float tn = th[j] + eps * mv * rh;
      a.r[(size_t)c * a.ld + j] = rh;
      a.theta_p[(size_t)c * a.ld + j] = tn;
      if (a.shadow32 && j < a.shadow_d)      // TF32 form of the tensor-core operand
        a.shadow32[(size_t)c * a.ld_shadow + j] = to_tf32(0.5f * (tn - a.theta_ref[j]));
      if (a.shadow_hi && j < a.shadow_d) {   // bf16 hi + lo of theta / 2 (tensor-core operand)
        const float half = 0.5f * (tn - a.theta_ref[j]);
        const __nv_bfloat16 hi = __float2bfloat16_rn(half);
        a.shadow_hi[(size_t)c * a.ld_shadow + j] = hi;
        a.shadow_lo[(size_t)c * a.ld_shadow + j] = __float2bfloat16_rn(half - __bfloat162float(hi));
      }
    }
  }
  // sum over the chain's lanes (xor tree within the group), then FP64
  const double K0 = f2_group_sum(kin, gsz);
  if (valid && sl == 0) a.H0[c] = -a.logp[c] + 0.5 * K0;
}

// standard normals for (iteration, stream) into out[C x ld] (scaled)
__global__ void __launch_bounds__(256) k_normals(int C, int d, int ld, unsigned long long seed,
                                                 unsigned int iter, unsigned int stream,
                                                 float scale, float *out) {
  const int nq = (d + 3) / 4;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)C * nq) return;
  const int c = (int)(t / nq), q = (int)(t - (long long)c * nq);
  const uint4 w = philox_at(seed, (uint32_t)q, (uint32_t)c, iter, stream);
  const float2 p0 = box_muller(w.x, w.y), p1 = box_muller(w.z, w.w);
  const float z[4] = {p0.x, p0.y, p1.x, p1.y};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int j = 4 * q + e;
    if (j < d) out[(size_t)c * ld + j] = scale * z[e];
  }
}

// fold chains start from full-data draws chosen uniformly with replacement:
// index = floor(w0 * n_pool / 2^32) from Philox stream ST_INIT (Algorithm 1)
__global__ void k_init_from_pool(int C, int d, int ld, unsigned long long seed, const float *pool,
                                 int n_pool, float *theta, int chain_base) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)C * d) return;
  const int c = (int)(t / d), j = (int)(t - (long long)c * d);
  const uint4 w = philox_at(seed, 0u, (uint32_t)(chain_base + c), 0u, ST_INIT);
  const unsigned idx = (unsigned)(((unsigned long long)w.x * (unsigned long long)n_pool) >> 32);
  theta[(size_t)c * ld + j] = pool[(size_t)idx * ld + j];
}

__global__ void k_shadow(int C, int d, int ld, const float *theta, const float *theta_ref,
                         __nv_bfloat16 *hi, __nv_bfloat16 *lo, int ld_shadow) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)C * d) return;
  const int c = (int)(t / d), j = (int)(t - (long long)c * d);
  const float v = 0.5f * (theta[(size_t)c * ld + j] - theta_ref[j]);   // shadows hold (theta - ref) / 2
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  hi[(size_t)c * ld_shadow + j] = h;
  lo[(size_t)c * ld_shadow + j] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// ---------------------------------------------------------------------------
// k_accept: 32 chains per block.  B300's FP64 pipe takes ~32 cycles of an SM
// per warp instruction, so the FP64 work runs one lane per chain (a warp
// instruction serves 32 chains) and the vector work a warp per chain:
//   A) a warp per chain: the kinetic energy of the proposal as an FP32 pair
//      (error-free sums, no FP64);
//   B) one lane per chain (warp 0): log u, H1, dH, the Metropolis test in
//      FP64, the kept log density and held-out value, the scalar
//      accumulators;
//   C) a warp per chain: the accept copies and the lag sums;
// the last block advances the counters.  A block has kAccWarps warps, each
// taking kAccChains / kAccWarps chains in A and C, so that several blocks
// (several phase-B warps) share an SM and hide the FP64 latency.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kAccWarps * 32) k_accept(AcceptArgs a) {
  __shared__ float khi_s[kAccChains], klo_s[kAccChains];
  __shared__ double s_s[kAccChains];
  __shared__ int flag_s[kAccChains];         // 1: accepted
  __shared__ int is_last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cb0 = blockIdx.x * kAccChains;
  const unsigned it = a.fd ? a.st->fd_iter : a.st->iter;
  const long long n_before = a.st->n_draws;
  // A) kinetic energy r' M^-1 r of the proposal
  for (int wc = warp; wc < kAccChains; wc += kAccWarps) {
    const int c = cb0 + wc;
    if (c < a.C) {
      F2 k2 = {0.0f, 0.0f};
      const float *mvr = minv_row(a.minv, c, a.minv_every, a.minv_ld);
      for (int j = lane; j < a.d; j += 32) f2_add_mr2(k2, mvr[j], a.r[(size_t)c * a.ld + j]);
      for (int o = 16; o > 0; o >>= 1) {
        const float h = __shfl_xor_sync(0xffffffffu, k2.hi, o), l = __shfl_xor_sync(0xffffffffu, k2.lo, o);
        f2_add(k2, h);
        k2.lo = __fadd_rn(k2.lo, l);
      }
      if (lane == 0) { khi_s[wc] = k2.hi; klo_s[wc] = k2.lo; }
    }
  }
  __syncthreads();
  // B) one lane per chain: FP64 Hamiltonian difference, Metropolis test with
  // the uniform of stream a.stream, the kept state's log density and
  // held-out value, the scalar accumulators
  if (warp == 0 && cb0 + lane < a.C) {
    const int c = cb0 + lane;
    const uint4 w = philox_at(a.seed, 0u, (uint32_t)(a.chain_base + c), it, a.stream);
    const double lu = log(unit_from_word(w.x));
    const double kin = (double)khi_s[lane] + (double)klo_s[lane];
    const double H1 = -a.logp_p[c] + 0.5 * kin;
    const double dH = H1 - a.H0[c];
    const bool finite = isfinite(H1) && isfinite(dH);
    const bool acc = finite && (lu < -dH);
    const bool div = !finite || dH > 1000.0;
    double s;
    if (acc) {
      s = a.shat_p[c];
      a.logp[c] = a.logp_p[c];
      a.shat[c] = s;
    } else {
      s = a.shat[c];
    }
    flag_s[lane] = acc ? 1 : 0;
    s_s[lane] = s;
    if (a.accept_prob) a.accept_prob[c] = finite ? (dH <= 0.0 ? 1.0 : exp(-dH)) : 0.0;
    if (a.accumulate) {
      a.acc.div[c] += div ? 1 : 0;
      a.acc.acc[c] += acc ? 1 : 0;
      accum_scalar(a.acc, c, s, n_before);
      if (a.acc.draws && n_before < a.acc.draw_cap) a.acc.draws[(size_t)c * a.acc.draw_cap + n_before] = s;
    }
  }
  __syncthreads();
  // C) a warp per chain: restore-or-keep (theta and gradient of the proposal
  // when accepted) and the lag sums of the held-out value
  for (int wc = warp; wc < kAccChains; wc += kAccWarps) {
    const int c = cb0 + wc;
    if (c < a.C) {
      if (flag_s[wc] & 1) {
        for (int j = lane; j < a.d; j += 32) {
          a.theta[(size_t)c * a.ld + j] = a.theta_p[(size_t)c * a.ld + j];
          a.grad[(size_t)c * a.ld + j] = a.grad_p[(size_t)c * a.ld + j];
        }
      }
      if (a.accumulate) accum_lags(a.acc, c, acov_x(a.acc, c, s_s[wc], n_before), n_before, lane);
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&a.st->ticket, 1u);
    is_last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (is_last && threadIdx.x == 0) {
    __threadfence();
    a.st->ticket = 0u;
    if (a.fd) a.st->fd_iter += 1u;
    else {
      a.st->iter += 1u;
      if (a.accumulate) a.st->n_draws += 1;
    }
  }
}

// push given draws (test entry), 32 chains per block: per draw the scalar
// accumulators (one lane per chain), then the lag sums (one warp per chain)
__global__ void __launch_bounds__(kAccChains * 32) k_accumulate_given(Accum A, const double *s, int n,
                                                                     long long n0) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cb0 = blockIdx.x * kAccChains;
  for (int t = 0; t < n; ++t) {
    if (warp == 0 && cb0 + lane < A.C) {
      const int cc = cb0 + lane;
      const double v = s[(size_t)cc * n + t];
      accum_scalar(A, cc, v, n0 + t);
      if (A.draws && n0 + t < A.draw_cap) A.draws[(size_t)cc * A.draw_cap + n0 + t] = v;
    }
    __syncthreads();
    const int c = cb0 + warp;
    if (c < A.C) accum_lags(A, c, acov_x(A, c, s[(size_t)c * n + t], n0 + t), n0 + t, lane);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// full-data adaptation (one block), run after each full-data iteration
// ---------------------------------------------------------------------------

__device__ void da_reset(IterState *st, double eps) {
  st->da_mu = log(10.0 * eps);
  st->da_hbar = 0.0;
  st->da_logeps = log(eps);
  st->da_logeps_bar = 0.0;
  st->da_t = 0;
}

__global__ void k_fd_adapt(FdAdaptArgs a) {
  const int i = (int)a.st->fd_iter - 1;          // iteration just completed
  if (i < a.n_adapt) {
    if (a.adapt_eps && threadIdx.x == 0) {
      // Nesterov dual averaging (Hoffman & Gelman 2014): delta 0.8, gamma 0.05,
      // t0 10, kappa 0.75
      double asum = 0.0;
      for (int c = 0; c < a.C; ++c) asum += a.accept_prob[c];
      IterState *st = a.st;
      st->da_t += 1;
      const double t = (double)st->da_t;
      const double wgt = 1.0 / (t + 10.0);
      st->da_hbar = (1.0 - wgt) * st->da_hbar + wgt * (0.8 - asum / a.C);
      st->da_logeps = st->da_mu - sqrt(t) / 0.05 * st->da_hbar;
      const double eta = pow(t, -0.75);
      st->da_logeps_bar = eta * st->da_logeps + (1.0 - eta) * st->da_logeps_bar;
      st->eps = (float)exp(st->da_logeps);
    }
    __syncthreads();
    if (a.adapt_mass && i >= a.w0 && i < a.w2) {
      const double n0 = a.st->mass_n;
      for (int j = threadIdx.x; j < a.d; j += blockDim.x) {
        double m = a.wmean[j], M2 = a.wM2[j];
        for (int c = 0; c < a.C; ++c) {
          const double v = a.theta[(size_t)c * a.ld + j];
          const double dl = v - m;
          m += dl / (n0 + c + 1);
          M2 += dl * (v - m);
        }
        a.wmean[j] = m;
        a.wM2[j] = M2;
      }
      __syncthreads();
      if (threadIdx.x == 0) a.st->mass_n = n0 + a.C;
      __syncthreads();
      const double wn = a.st->mass_n;
      if ((i == a.w1 - 1 || i == a.w2 - 1) && wn > 1.0) {
        // end of a mass window: regularised variance, restart dual
        // averaging, and start the next window's Welford sums afresh
        const double w = wn / (wn + 5.0);
        for (int j = threadIdx.x; j < a.d; j += blockDim.x) {
          a.minv[j] = (float)(w * (a.wM2[j] / (wn - 1.0)) + 1e-3 * (1.0 - w));
          if (a.active) a.minv[j] *= a.active[j];          // masked covariates stay held
          a.wmean[j] = 0.0;
          a.wM2[j] = 0.0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          da_reset(a.st, (double)a.st->eps);
          a.st->mass_n = 0.0;
        }
      }
    }
  } else {
    const int k = i - a.n_adapt;
    if (k < a.n_keep) {
      for (int t = threadIdx.x; t < a.C * a.d; t += blockDim.x) {
        const int c = t / a.d, j = t - c * a.d;
        a.pool[((size_t)k * a.C + c) * a.ld + j] = a.theta[(size_t)c * a.ld + j];
      }
    }
  }
}

__global__ void k_fd_init_state(IterState *st, float eps0, int adapt) {
  st->eps = eps0;
  st->eps_iter = eps0;
  da_reset(st, (double)eps0);
  st->mass_n = 0.0;
  st->fd_iter = 0u;
  (void)adapt;
}

// the dual-averaged step size, capped so that L_f steps span at most the
// trajectory length (eps_cap = trajectory length / L_f; <= 0: no cap)
__global__ void k_fd_final_eps(IterState *st, float eps_cap) {
  float e = (float)exp(st->da_logeps_bar);
  if (eps_cap > 0.0f && e > eps_cap) e = eps_cap;
  st->eps = e;
  st->eps_iter = e;
}

__global__ void k_copy_eps(IterState *st) { st->eps_iter = st->eps; }

// ---------------------------------------------------------------------------
// per-fold estimators
// ---------------------------------------------------------------------------

struct Welf { double n, mean, M2; };
__device__ __forceinline__ void welf_merge(Welf &x, double n2, double m2, double M22) {
  const double nt = x.n + n2;
  if (nt == 0.0) return;
  const double dl = m2 - x.mean;
  x.mean += dl * n2 / nt;
  x.M2 += M22 + dl * dl * x.n * n2 / nt;
  x.n = nt;
}

// eq. rhat from sequence summaries: sqrt(((n-1)/n W + B/n) / W)
__device__ double rhat_eq(int nseq, double n, const double *mean, const double *M2) {
  double Wv = 0.0, gm = 0.0;
  for (int l = 0; l < nseq; ++l) { Wv += M2[l] / (n - 1.0); gm += mean[l]; }
  Wv /= nseq; gm /= nseq;
  double B = 0.0;
  for (int l = 0; l < nseq; ++l) B += (mean[l] - gm) * (mean[l] - gm);
  B *= n / (nseq - 1.0);
  return sqrt((((n - 1.0) / n) * Wv + B / n) / Wv);
}

// one thread per fold; scratch: per-thread arrays in a global buffer
__global__ void k_finalize(Accum A, int K, int L, long long n, double *out, double *scratch) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const int b = A.b;
  const long long a = n / b;
  const int c0 = k * L;
  double *o = out + (size_t)k * F_NFIELDS;
  double *mean = scratch + (size_t)k * (4 * L + 2 * (A.M + 2));
  double *M2 = mean + 2 * L;
  double *rho = M2 + 2 * L;
  // f_k by log-sum-exp of the per-chain U_x (A2 final step); a chain keeps
  // U_x as the sum of exp(s - em) on its shift em
  double lse = -INFINITY;
  for (int l = 0; l < L; ++l) lse = log_add_exp(lse, A.em[c0 + l] + log(A.Ux[c0 + l]));
  const double Ln = (double)L * (double)n;
  o[F_ELPD] = lse - log(Ln);
  // pooled log-shifted Welford of exp(s) (sample variance s^2)
  double sh = -INFINITY;
  for (int l = 0; l < L; ++l) sh = fmax(sh, A.em[c0 + l]);
  Welf pe = {0.0, 0.0, 0.0};
  for (int l = 0; l < L; ++l) {
    const double sc = exp(A.em[c0 + l] - sh);
    welf_merge(pe, (double)n, A.emean[c0 + l] * sc, A.eM2[c0 + l] * sc * sc);
  }
  const double s2_rel = (pe.M2 / (pe.n - 1.0)) / (pe.mean * pe.mean);
  // pooled batch means (eq. bmvar), centred on the grand mean f_k
  double vsh = -INFINITY;
  for (int l = 0; l < L; ++l) vsh = fmax(vsh, A.vm[c0 + l]);
  Welf pv = {0.0, 0.0, 0.0};
  for (int l = 0; l < L; ++l) {
    const double sc = exp(A.vm[c0 + l] - vsh);
    welf_merge(pv, (double)a, A.vmean[c0 + l] * sc, A.vM2[c0 + l] * sc * sc);
  }
  const double sig2_rel = ((double)b * pv.M2 / ((double)L * (double)a - 1.0)) / (pv.mean * pv.mean);
  o[F_SIG2BM] = sig2_rel;
  o[F_S2] = s2_rel;
  o[F_MCSE] = sqrt(sig2_rel / Ln);                 // delta method, eq. mc-var
  o[F_ESSBM] = Ln * s2_rel / sig2_rel;
  // R-hat on s (eq. rhat)
  for (int l = 0; l < L; ++l) { mean[l] = A.wmean[c0 + l]; M2[l] = A.wM2[c0 + l]; }
  o[F_RHAT] = rhat_eq(L, (double)n, mean, M2);
  // split R-hat: halves of whole batches (middle batch dropped if a is odd)
  const long long half = a / 2;
  if (half >= 1 && a <= A.max_batches) {
    for (int l = 0; l < L; ++l) {
      for (int hh = 0; hh < 2; ++hh) {
        Welf w = {0.0, 0.0, 0.0};
        const long long h0 = hh == 0 ? 0 : a - half;
        for (long long h = h0; h < h0 + half; ++h)
          welf_merge(w, (double)b, A.bmean[(size_t)h * A.C + c0 + l], A.bM2[(size_t)h * A.C + c0 + l]);
        mean[2 * l + hh] = w.mean;
        M2[2 * l + hh] = w.M2;
      }
    }
    o[F_SRHAT] = rhat_eq(2 * L, (double)(half * b), mean, M2);
  } else {
    o[F_SRHAT] = NAN;
  }
  // multi-chain autocorrelation ESS of s with Geyer's initial monotone sequence
  int trunc = 0;
  double ess = NAN;
  if (A.M > 0) {
    const int Mu = (int)(A.M < n - 1 ? A.M : n - 1);
    double Wv = 0.0, gm = 0.0, B = 0.0;
    for (int l = 0; l < L; ++l) { Wv += A.wM2[c0 + l] / (double)(n - 1); gm += A.wmean[c0 + l]; }
    Wv /= L; gm /= L;
    for (int l = 0; l < L; ++l) B += (A.wmean[c0 + l] - gm) * (A.wmean[c0 + l] - gm);
    B *= (double)n / (L - 1.0);
    const double varplus = ((double)(n - 1) / n) * Wv + B / n;
    for (int m = 0; m <= Mu; ++m) rho[m] = 0.0;
    for (int l = 0; l < L; ++l) {
      const int c = c0 + l;
      const double xbar = A.xsum[c] / (double)n;
      double head = 0.0, tail = 0.0;
      for (int m = 0; m <= Mu; ++m) {
        if (m > 0) {
          head += A.first[(size_t)c * A.M + (m - 1)];
          tail += A.ring[(size_t)c * A.M + (int)((n - m) % A.M)];
        }
        const double P = A.xsum[c] - head, Q = A.xsum[c] - tail;
        const double gam = A.lagsum[(size_t)c * (A.M + 1) + m] - xbar * (P + Q) +
                           (double)(n - m) * xbar * xbar;
        rho[m] += gam / (double)n;
      }
    }
    for (int m = 0; m <= Mu; ++m) rho[m] = 1.0 - (Wv - rho[m] / L) / varplus;
    rho[0] = 1.0;
    double tau = -1.0, prev = INFINITY;
    trunc = 1;
    for (int kk = 0; 2 * kk + 1 <= Mu; ++kk) {
      double P = rho[2 * kk] + rho[2 * kk + 1];
      if (!(P > 0.0)) { trunc = 0; break; }
      if (P > prev) P = prev;
      prev = P;
      tau += 2.0 * P;
    }
    if (tau < 1e-12) tau = 1e-12;
    ess = Ln / tau;
  }
  o[F_ESSAC] = ess;
  o[F_ACTRUNC] = trunc;
  double dv = 0.0, ac = 0.0;
  for (int l = 0; l < L; ++l) { dv += (double)A.div[c0 + l]; ac += (double)A.acc[c0 + l]; }
  o[F_DIV] = dv;
  o[F_ACCRATE] = ac / Ln;
}

// totals over folds (one block)
__global__ void k_totals(const double *fo, int K, double Ln, double *tot) {
  __shared__ double sh[7][256];
  double e = 0, m2 = 0, rmax = -INFINITY, srmax = -INFINITY, s2 = 0, sg = 0, dv = 0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const double *o = fo + (size_t)k * F_NFIELDS;
    e += o[F_ELPD];
    m2 += o[F_MCSE] * o[F_MCSE];
    rmax = fmax(rmax, o[F_RHAT]);
    srmax = fmax(srmax, o[F_SRHAT]);
    s2 += o[F_S2];
    sg += o[F_SIG2BM];
    dv += o[F_DIV];
  }
  sh[0][threadIdx.x] = e; sh[1][threadIdx.x] = m2; sh[2][threadIdx.x] = rmax;
  sh[3][threadIdx.x] = srmax; sh[4][threadIdx.x] = s2; sh[5][threadIdx.x] = sg;
  sh[6][threadIdx.x] = dv;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      for (int f = 0; f < 7; ++f) {
        if (f == 2 || f == 3) sh[f][threadIdx.x] = fmax(sh[f][threadIdx.x], sh[f][threadIdx.x + s]);
        else sh[f][threadIdx.x] += sh[f][threadIdx.x + s];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double mean = sh[0][0] / K;
    double v = 0.0;
    for (int k = 0; k < K; ++k) {
      const double dd = fo[(size_t)k * F_NFIELDS + F_ELPD] - mean;
      v += dd * dd;
    }
    v = K > 1 ? v / (K - 1) : 0.0;
    tot[T_ELPD] = sh[0][0];
    tot[T_MCSE] = sqrt(sh[1][0]);
    tot[T_SEEPI] = sqrt(K * v);
    tot[T_RHATMAX] = sh[2][0];
    tot[T_ESSTOT] = Ln * sh[4][0] / sh[5][0];
    tot[T_SRHATMAX] = sh[3][0];
    tot[T_DIV] = sh[6][0];
  }
}

}  // namespace pcv

namespace pcv {
// centring reference for the tensor-core path: theta_ref = mean of n rows
// of src (ld floats apart), then eta_half[n] = x16_n . theta_ref / 2 for
// every row (bf16 X as the tensor cores see it, FP64 sums, 0 on padding)
__global__ void k_theta_ref(int n, int d, int ld, const float *src, float *theta_ref) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d; j += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += (double)src[(size_t)i * ld + j];
    theta_ref[j] = (float)(s / n);
  }
}
__global__ void k_eta_ref(int N, int N_pad, int p, int KP, const __nv_bfloat16 *X16, const float *theta_ref,
                          float *eta_half) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N_pad) return;
  double s = 0.0;
  if (n < N)
    for (int j = 0; j < p; ++j) s += (double)__bfloat162float(X16[(size_t)n * KP + j]) * (double)theta_ref[j];
  eta_half[n] = (float)(0.5 * s);
}
// ---------------------------------------------------------------------------
// data set-up on the device (pcv_create): the caller's X rows gathered into
// the fold-sorted layout and its bf16 copy for the tensor cores (logistic
// rows signed by 2 y - 1)
// ---------------------------------------------------------------------------
__global__ void k_gather_rows(long long N, int p, int p_pad, const int *perm, const float *xraw, float *X) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * p) return;
  const long long r = t / p;
  const int j = (int)(t - r * p);
  X[r * p_pad + j] = xraw[(long long)perm[r] * p + j];
}
// bf16 copy of X; with ysign (logistic model) row r is multiplied by
// s_r = 2 y_r - 1 (exact in bf16), so that the first GEMM yields s eta / 2
__global__ void k_x_bf16(long long N, int p, int p_pad, int KP, const float *X, const float *ysign,
                         __nv_bfloat16 *X16) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * p) return;
  const long long r = t / p;
  const int j = (int)(t - r * p);
  const float v = X[r * p_pad + j];
  X16[r * KP + j] = __float2bfloat16_rn(ysign && ysign[r] == 0.0f ? -v : v);
}

// eta_ref / 2 of every row into the operand columns p .. p + kEtaCols - 1 of
// the bf16 design matrix, as a sum of kEtaCols bf16 parts (each part rounds
// what the previous ones left: 24 significant bits, the precision of eta_half)
__global__ void k_eta_fold(int N_pad, int p, int KP, const float *eta_half, const float *y,
                           __nv_bfloat16 *X16) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N_pad) return;
  // Gaussian models (y given): (eta_ref - y) / 2, so that the first GEMM
  // yields (eta - y) / 2 and the epilogue needs no response
  float rest = y ? eta_half[n] - 0.5f * y[n] : eta_half[n];
#pragma unroll
  for (int k = 0; k < kEtaCols; ++k) {
    const __nv_bfloat16 part = __float2bfloat16_rn(rest);
    X16[(size_t)n * KP + p + k] = part;
    rest -= __bfloat162float(part);
  }
}
// the constant 1 of the eta_ref columns in a chain set's hi shadow (the lo
// shadow keeps 0 there, so launches that add hi and lo count it once)
// ---- the TF32 operand form of the tensor-core path: FP32 arrays whose
// values are rounded to TF32 (to_tf32), as the MMAs read them
// X [N_pad x KP] (logistic: rows signed by 2 y - 1) and X^T [PN x N_pad]
__global__ void k_x_tf32(long long N, int p, int p_pad, int KP, int N_pad, const float *X, const float *ysign,
                         float *X32, float *XT32) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * p) return;
  const long long r = t / p;
  const int j = (int)(t - r * p);
  const float v = X[r * p_pad + j];
  const float x = to_tf32(ysign && ysign[r] == 0.0f ? -v : v);
  X32[r * KP + j] = x;
  XT32[(size_t)j * N_pad + r] = x;
}
__global__ void k_eta_ref32(int N, int N_pad, int p, int KP, const float *X32, const float *theta_ref,
                            float *eta_half) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N_pad) return;
  double s = 0.0;
  if (n < N)
    for (int j = 0; j < p; ++j) s += (double)X32[(size_t)n * KP + j] * (double)theta_ref[j];
  eta_half[n] = (float)(0.5 * s);
}
// eta_ref / 2 (Gaussian: (eta_ref - y) / 2) as three TF32 parts
__global__ void k_eta_fold32(int N_pad, int p, int KP, const float *eta_half, const float *y, float *X32) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N_pad) return;
  float rest = y ? eta_half[n] - 0.5f * y[n] : eta_half[n];
#pragma unroll
  for (int k = 0; k < kEtaCols; ++k) {
    const float part = to_tf32(rest);
    X32[(size_t)n * KP + p + k] = part;
    rest -= part;
  }
}
__global__ void k_shadow32(int C, int d, int ld, const float *theta, const float *theta_ref, float *s32, int ld_s) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)C * d) return;
  const int c = (int)(t / d), j = (int)(t - (long long)c * d);
  s32[(size_t)c * ld_s + j] = to_tf32(0.5f * (theta[(size_t)c * ld + j] - theta_ref[j]));
}
__global__ void k_shadow_ones32(int C_pad, int p, int KP, float *hi) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= C_pad * kEtaCols) return;
  const int c = t / kEtaCols, k = t - c * kEtaCols;
  hi[(size_t)c * KP + p + k] = 1.0f;
}

__global__ void k_shadow_ones(int C_pad, int p, int KP, __nv_bfloat16 *hi) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= C_pad * kEtaCols) return;
  const int c = t / kEtaCols, k = t - c * kEtaCols;
  hi[(size_t)c * KP + p + k] = __float2bfloat16_rn(1.0f);
}
}  // namespace pcv

namespace pcv {
// ---------------------------------------------------------------------------
// R-hat_max benchmark by block shuffling (Section 4.2; the shuffle loop of
// Algorithm A2).  Chains are cut into D contiguous blocks of whole batches
// (block d holds batches [d a / D, (d+1) a / D)); replicate r rebuilds
// every chain slot of every fold from blocks of chains drawn uniformly with
// replacement and takes the R-hat (eq. rhat) of the rebuilt chains.
// ---------------------------------------------------------------------------
// Welford state (count, mean, M2) of each (chain, block): [C x D] x 3
__global__ void k_block_stats(Accum A, int a, int D, double *blk) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)A.C * D) return;
  const int c = (int)(t / D), d = (int)(t - (long long)c * D);
  Welf w{0.0, 0.0, 0.0};
  const int h0 = (int)((long long)d * a / D), h1 = (int)((long long)(d + 1) * a / D);
  for (int h = h0; h < h1; ++h) welf_merge(w, (double)A.b, A.bmean[(size_t)h * A.C + c], A.bM2[(size_t)h * A.C + c]);
  blk[3 * t] = w.n;
  blk[3 * t + 1] = w.mean;
  blk[3 * t + 2] = w.M2;
}

// one thread per (replicate r, fold k): the picks are word t % 4 of Philox
// (block t / 4, chain k, iteration r, stream ST_SHUF) for t = l D + d,
// l' = floor(w L / 2^32); out_max[r] = max over folds (bit pattern of a
// non-negative double, so an integer max orders it), out_all[r K + k]
__global__ void k_rhat_shuffle(const double *blk, int K, int L, int D, int R, unsigned long long seed,
                               unsigned long long *out_max, double *out_all, int first_fold) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)R * K) return;
  const int r = (int)(t / K), k = (int)(t - (long long)r * K);
  double wsum = 0.0, nn = 0.0;
  Welf means{0.0, 0.0, 0.0};                      // Welford of the slot means
  for (int l = 0; l < L; ++l) {
    Welf w{0.0, 0.0, 0.0};
    for (int d = 0; d < D; ++d) {
      const int q = l * D + d;
      const uint4 wd = philox_at(seed, (uint32_t)(q >> 2), (uint32_t)(first_fold + k), (uint32_t)r, ST_SHUF);
      const uint32_t word = (q & 3) == 0 ? wd.x : (q & 3) == 1 ? wd.y : (q & 3) == 2 ? wd.z : wd.w;
      const int src = (int)(((unsigned long long)word * (unsigned long long)L) >> 32);
      const double *b3 = blk + 3 * ((size_t)(k * L + src) * D + d);
      welf_merge(w, b3[0], b3[1], b3[2]);
    }
    nn = w.n;
    wsum += w.M2 / (w.n - 1.0);
    welf_merge(means, 1.0, w.mean, 0.0);
  }
  const double Wv = wsum / L;
  const double B = nn * means.M2 / (L - 1.0);
  const double rh = sqrt((((nn - 1.0) / nn) * Wv + B / nn) / Wv);
  if (out_all) out_all[t] = rh;
  atomicMax(out_max + r, (unsigned long long)__double_as_longlong(rh));
}
}  // namespace pcv

namespace pcv {
// zero the masked coordinates of C positions
__global__ void k_mask_positions(int C, int d, int ld, const float *active, float *theta) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)C * d) return;
  const int c = (int)(t / d), j = (int)(t - (long long)c * d);
  theta[(size_t)c * ld + j] *= active[j];
}

// pairwise model selection from two contexts' fold results (eq. sel-cv,
// eq. norm-approx, eq. mc-var): out = [delta_k (K) | mcse_k (K) | delta, se,
// mcse, Pr(A better than B)]; one block, fixed reduction order
__global__ void k_compare(const double *fo_a, const double *fo_b, int K, double *out) {
  __shared__ double sh[2][256];
  double s = 0.0, m2 = 0.0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const double dk = fo_a[(size_t)k * F_NFIELDS + F_ELPD] - fo_b[(size_t)k * F_NFIELDS + F_ELPD];
    const double ma = fo_a[(size_t)k * F_NFIELDS + F_MCSE], mb = fo_b[(size_t)k * F_NFIELDS + F_MCSE];
    const double mk2 = ma * ma + mb * mb;
    out[k] = dk;
    out[K + k] = sqrt(mk2);
    s += dk;
    m2 += mk2;
  }
  sh[0][threadIdx.x] = s;
  sh[1][threadIdx.x] = m2;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double sum = sh[0][0], mean = sum / K;
    double v = 0.0;
    for (int k = 0; k < K; ++k) v += (out[k] - mean) * (out[k] - mean);
    const double se = sqrt(K * (v / (K - 1.0)));
    out[2 * K] = sum;
    out[2 * K + 1] = se;
    out[2 * K + 2] = sqrt(sh[1][0]);
    out[2 * K + 3] = 0.5 * erfc(-(sum / se) * 0.70710678118654752440);
  }
}
}  // namespace pcv

namespace pcv {
// ---------------------------------------------------------------------------
// Hyvarinen (Algorithm A3) and Dawid-Sebastiani (Algorithm A4) scores for
// the Gaussian models with conditionally independent rows.  One warp per
// chain after the accept of a sampling iteration: for the fold's test rows,
// mu_i = x_i . beta, d1_i = -(y_i - mu_i) / sigma^2, d2 = -1 / sigma^2 and a
// predictive draw ytil_i = mu_i + sigma z_i (z: Philox stream ST_PRED,
// element i of (chain, iteration) as for the momenta).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_extra_push(Problem pb, GradArgs a, Extra E, const unsigned int *iter,
                                                    unsigned long long seed, int chain_base) {
  extern __shared__ double ysh[];                    // [8 warps][T]
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int c = blockIdx.x * 8 + wib;
  if (c >= a.C) return;
  const unsigned it = *iter - 1u;                     // the iteration just accepted
  const FoldDesc fd = pb.folds[fold_of_chain(a, c)];
  const int m = fd.test_hi - fd.test_lo;
  const float *th = a.theta + (size_t)c * a.ld_theta;
  double *yt = ysh + (size_t)wib * E.T;
  if (pb.variant == MV_LOGISTIC) {
    // a predictive draw ytil_i ~ Bernoulli(sigmoid(eta_i)) (DSS only): 1
    // iff u_i < sigmoid(eta_i), u_i from word i % 4 of Philox block i / 4;
    // the comparison in FP64
    for (int i = lane; i < m; i += 32) {
      const int n = fd.test_lo + i;
      double eta = 0.0;
      for (int j = 0; j < pb.p; ++j) eta += (double)pb.X[(size_t)n * pb.p_pad + j] * (double)th[j];
      const uint4 w = philox_at(seed, (uint32_t)(i >> 2), (uint32_t)(chain_base + c), it, ST_PRED);
      const uint32_t word = (i & 3) == 0 ? w.x : (i & 3) == 1 ? w.y : (i & 3) == 2 ? w.z : w.w;
      const double pr = eta >= 0.0 ? 1.0 / (1.0 + exp(-eta)) : exp(eta) / (1.0 + exp(eta));
      yt[i] = unit_from_word(word) < pr ? 1.0 : 0.0;
    }
  } else {
  const double sigma = pb.variant == MV_GAUSS_KNOWN ? (double)pb.sigma_known : exp((double)th[pb.p]);
  const double s2 = sigma * sigma;
  double xi1 = 0.0;
  for (int i = lane; i < m; i += 32) {
    const int n = fd.test_lo + i;
    double mu = 0.0;
    for (int j = 0; j < pb.p; ++j) mu += (double)pb.X[(size_t)n * pb.p_pad + j] * (double)th[j];
    const double d1 = -((double)pb.y[n] - mu) / s2;
    xi1 += -1.0 / s2 + d1 * d1;
    if (E.flags & 1) E.hs2[(size_t)c * E.T + i] += d1;
    // element i of the standard normals of (chain, iteration): Philox block
    // i / 4, Box-Muller pair (words 0, 1) or (2, 3)
    const uint4 w = philox_at(seed, (uint32_t)(i >> 2), (uint32_t)(chain_base + c), it, ST_PRED);
    const float2 z2 = (i & 2) ? box_muller(w.z, w.w) : box_muller(w.x, w.y);
    const double z = (i & 1) ? (double)z2.y : (double)z2.x;
    yt[i] = mu + sigma * z;
  }
  xi1 = warp_sum_d(xi1);
  if ((E.flags & 1) && lane == 0) E.hs1[c] += xi1;
  }
  __syncwarp();
  if (E.flags & 2) {
    for (int i = lane; i < m; i += 32) E.dsum[(size_t)c * E.T + i] += yt[i];
    for (int q = lane; q < m * m; q += 32) {
      const int i = q / m, j = q - i * m;
      E.douter[((size_t)c * E.T + i) * E.T + j] += yt[i] * yt[j];
    }
  }
}

// per fold (one block each): HS_k = sum_i [-2 E(d2 + d1^2)... as the pooled
// means over L chains x n draws; DSS_k = -log|S| - (y - m)' S^-1 (y - m) by
// a Cholesky factorisation of the pooled predictive covariance (thread 0)
__global__ void k_extra_finalize(Problem pb, Extra E, int K, int L, double n, double *hs, double *dss) {
  extern __shared__ double sm[];                     // A [T x T], mu [T], w [T]
  const int k = blockIdx.x;
  if (k >= K) return;
  const FoldDesc fd = pb.folds[k];
  const int m = fd.test_hi - fd.test_lo, T = E.T;
  double *A = sm, *mu = sm + (size_t)T * T, *w = mu + T;
  if (E.flags & 2) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      double sum = 0.0;
      for (int l = 0; l < L; ++l) sum += E.dsum[(size_t)(k * L + l) * T + i];
      mu[i] = sum / n;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < m * m; q += blockDim.x) {
      const int i = q / m, j = q - i * m;
      double so = 0.0;
      for (int l = 0; l < L; ++l) so += E.douter[((size_t)(k * L + l) * T + i) * T + j];
      A[i * m + j] = (so - n * mu[i] * mu[j]) / (n - 1.0);
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  if (E.flags & 1) {
    double e1 = 0.0;
    for (int l = 0; l < L; ++l) e1 += E.hs1[k * L + l];
    double h = -2.0 * e1 / n;
    for (int i = 0; i < m; ++i) {
      double e2 = 0.0;
      for (int l = 0; l < L; ++l) e2 += E.hs2[(size_t)(k * L + l) * T + i];
      h += (e2 / n) * (e2 / n);
    }
    hs[k] = h;
  }
  if (E.flags & 2) {
    double ld = 0.0;
    for (int j = 0; j < m; ++j) {
      double v = A[j * m + j];
      for (int q = 0; q < j; ++q) v -= A[j * m + q] * A[j * m + q];
      const double ljj = sqrt(v);
      A[j * m + j] = ljj;
      ld += 2.0 * log(ljj);
      for (int i = j + 1; i < m; ++i) {
        double u = A[i * m + j];
        for (int q = 0; q < j; ++q) u -= A[i * m + q] * A[j * m + q];
        A[i * m + j] = u / ljj;
      }
    }
    double quad = 0.0;
    for (int i = 0; i < m; ++i) {
      double u = (double)pb.y[fd.test_lo + i] - mu[i];
      for (int q = 0; q < i; ++q) u -= A[i * m + q] * w[q];
      w[i] = u / A[i * m + i];
      quad += w[i] * w[i];
    }
    dss[k] = -ld - quad;
  }
}
}  // namespace pcv
