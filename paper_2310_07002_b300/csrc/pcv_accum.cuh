// pcv_accum.cuh -- the online accumulators of one draw (Algorithm A2 with
// the readings: log-shifted Welford instead of centred log-space sums), used
// by the accept kernel and by the one-launch iteration of small problems.
#pragma once
#include "pcv_internal.cuh"

namespace pcv {

// ---------------------------------------------------------------------------
// online accumulators (Algorithm A2 with the readings: log-shifted Welford
// instead of centred log-space sums)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double log_add_exp(double a, double b) {
  if (a == -INFINITY) return b;
  if (b == -INFINITY) return a;
  const double m = fmax(a, b);
  return m + log1p(exp(-fabs(a - b)));
}

// running (shift, mean, M2) of exp(lv - shift) values; count_after >= 1
__device__ __forceinline__ void lshift_push(double &shift, double &mean, double &M2,
                                            long long count_after, double lv) {
  if (lv > shift) {
    if (shift != -INFINITY) {
      const double sc = exp(shift - lv);
      mean *= sc;
      M2 *= sc * sc;
    }
    shift = lv;
  }
  const double v = exp(lv - shift);
  const double delta = v - mean;
  mean += delta / (double)count_after;
  M2 += delta * (v - mean);
}

// The accumulators of one draw are split by the shape of their work: the
// scalar ones (the log-sum-exps, the log-shifted Welford of exp(s), Welford
// of s, batch means) are FP64 chains, run one thread per chain so that a warp
// instruction serves 32 chains (B300's FP64 pipe is narrow: a warp
// instruction of it takes ~32 cycles of an SM); the lag sums of the
// autocovariance are a warp per chain, lanes over lags.
//
// The log-sum-exps of Algorithm A2 (U_x, U_x^2 and the batch's Z_x) share the
// shift of the log-shifted Welford of exp(s): m = em, the chain's running
// maximum of s.  They are kept as plain FP64 sums of exp(s - m),
// exp(2 (s - m)) and (within the batch) exp(s - m), rescaled when m moves,
// so that a draw costs one FP64 exp (v = exp(s - m), or the rescale factor
// exp(m_old - s) when s is the new maximum and v = 1) instead of one exp and
// one log1p per log-sum-exp; U_x = m + log(sum) is formed in the finalize and
// Z_x at the batch's close.

// x_t = s_t - c0 (c0: the chain's first draw), the autocovariance variable
__device__ __forceinline__ double acov_x(const Accum &A, int c, double s, long long n_before) {
  return n_before == 0 ? 0.0 : s - A.c0[c];
}

// scalar accumulators of draw s (0-based index n_before) of chain c; one thread
__device__ __forceinline__ void accum_scalar(const Accum &A, int c, double s, long long n_before) {
  const long long n = n_before + 1;
  const int b = A.b;
  const int in_batch = (int)(n_before % b) + 1;
  const double rn = 1.0 / (double)n;
  // the shared shift m (running maximum of s) and v = exp(s - m)
  double m = A.em[c], sc = 1.0, v;
  if (s > m) {
    sc = m == -INFINITY ? 0.0 : exp(m - s);
    m = s;
    v = 1.0;
  } else {
    v = s == -INFINITY ? 0.0 : exp(s - m);   // (m = s = -inf: no mass yet)
  }
  A.em[c] = m;
  A.Ux[c] = A.Ux[c] * sc + v;                        // sum exp(s - m)
  A.Ux2[c] = A.Ux2[c] * (sc * sc) + v * v;           // sum exp(2 (s - m))
  const double zs = (in_batch == 1 ? 0.0 : A.Zx[c] * sc) + v;   // this batch's sum exp(s - m)
  A.Zx[c] = zs;
  if (in_batch == b) {                       // the batch closes (A2 batch loop end)
    const long long na = n / b;
    const double z = m + log(zs / (double)b);   // log of the batch mean, eq. bmean
    double vm = A.vm[c], vmean = A.vmean[c], vM2 = A.vM2[c];
    lshift_push(vm, vmean, vM2, na, z);
    A.vm[c] = vm; A.vmean[c] = vmean; A.vM2[c] = vM2;
  }
  {
    // log-shifted Welford of exp(s) on the shift m (as lshift_push, with v shared)
    double emean = A.emean[c] * sc, eM2 = A.eM2[c] * (sc * sc);
    const double delta = v - emean;
    emean += delta * rn;
    eM2 += delta * (v - emean);
    A.emean[c] = emean; A.eM2[c] = eM2;
  }
  double wm = A.wmean[c], wM2 = A.wM2[c];
  double dl = s - wm;
  wm += dl * rn;
  wM2 += dl * (s - wm);
  A.wmean[c] = wm; A.wM2[c] = wM2;
  double bm = in_batch == 1 ? 0.0 : A.bmean_cur[c], b2 = in_batch == 1 ? 0.0 : A.bM2_cur[c];
  dl = s - bm;
  bm += dl / (double)in_batch;
  b2 += dl * (s - bm);
  A.bmean_cur[c] = bm; A.bM2_cur[c] = b2;
  if (n_before == 0) A.c0[c] = s;
  A.xsum[c] += acov_x(A, c, s, n_before);
  if (in_batch == b) {
    const long long na = n / b;
    if (na <= A.max_batches) {
      A.bmean[(size_t)(na - 1) * A.C + c] = bm;
      A.bM2[(size_t)(na - 1) * A.C + c] = b2;
    }
  }
}

// lag sums sum_t x_t x_{t-m}, m = 0..M, and the ring of the last M values of
// x; one warp per chain, lanes over lags (t = n_before)
__device__ __forceinline__ void accum_lags(const Accum &A, int c, double x, long long t, int lane) {
  if (A.M == 0) return;
  const int tr = (int)(t % A.M);             // ring slot of this draw
  double *lag = A.lagsum + (size_t)c * (A.M + 1);
  double *ring = A.ring + (size_t)c * A.M;
  for (int m = lane; m <= A.M; m += 32) {
    if (m == 0) lag[0] += x * x;
    else if (m <= t) {
      int slot = tr - m;                     // (t - m) mod M, as 0 <= tr < M and m <= M
      if (slot < 0) slot += A.M;
      lag[m] += x * ring[slot];
    }
  }
  __syncwarp();
  if (lane == 0) {
    ring[tr] = x;
    if (t < A.M) A.first[(size_t)c * A.M + t] = x;
  }
}

}  // namespace pcv
