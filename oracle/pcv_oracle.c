/*
 * pcv_oracle.c -- FP64 CPU oracle for parallel Bayesian cross-validation (PCV).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * It is a plain, slow, sequential-per-chain restatement of the method of
 * "Bayesian cross-validation by parallel Markov chain Monte Carlo"
 * (arXiv 2310.07002), in double precision throughout:
 *
 *   - fold-masked log joint density and log predictive, eq. (mask-log-prob)
 *     and eq. (mask-log-pred) of Appendix B, with the training mask read as
 *     the complement of the test mask (the masked code listing of
 *     Appendix B uses fold_index != fold_id for training);
 *   - lock-step HMC with a fold identifier, Section 3.3, with a fixed
 *     number of leapfrog steps and a Metropolis accept;
 *   - warm-up reuse (Section 3.1; Algorithm 1): full-data chains adapt a
 *     step size (Nesterov dual averaging, Hoffman & Gelman 2014) and a
 *     diagonal inverse mass; fold chains start from full-data draws and run a
 *     short discarded warm-up;
 *   - the online accumulators of Algorithm A2 (Appendix A.1/A.2): log-sum-exp
 *     of the held-out log predictive draws, batch means (eq. bmean), the
 *     batch-means variance (eq. bmvar), Welford sums for R-hat (eq. rhat),
 *     plus autocovariance lag sums for a Geyer (1992) ESS;
 *   - the per-fold and total estimators: elpd, MCSE by the delta method
 *     (eq. mc-var), ESS (Section 4.1), R-hat and R-hat_max (eq. rhat,
 *     eq. rhat-max).
 *
 * Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror & Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC 2011), written here from
 * its published definition; normals by the Box-Muller transform.
 *
 * Counter layout (shared *definition* with the GPU path, not shared code):
 *   key     = (seed low 32 bits, seed high 32 bits)
 *   counter = (block, chain, iteration, stream)
 *   block   = element index / 4 (each Philox call yields 4 words)
 *   streams: 0 fold-chain momentum, 1 fold-chain accept uniform,
 *            2 fold-chain init index, 3 step-size jitter (chain 0: one
 *            value per iteration, shared by all chains), 16 full-data momentum,
 *            17 full-data accept uniform, 18 full-data init position.
 *
 * Parity pins: see tests/test_oracle_*.py.  Every function here is pinned
 * by closed forms, finite differences, brute force or published values.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TWO_PI 6.283185307179586476925286766559
#define ORC_LOG_2PI 1.8378770664093454835606594728112

enum { ORC_GAUSS = 0, ORC_LOGISTIC = 1, ORC_HIER = 2, ORC_AR = 3 };
enum { ST_MOM = 0, ST_ACC = 1, ST_INIT = 2, ST_JIT = 3, ST_FD_MOM = 16, ST_FD_ACC = 17, ST_FD_INIT = 18 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10                                                             */
/* ------------------------------------------------------------------------ */
void orc_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    /* multipliers and Weyl key increments from the Philox definition */
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t prod0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox_at(uint64_t seed, uint32_t block, uint32_t chain, uint32_t iter,
                      uint32_t stream, uint32_t out[4])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {block, chain, iter, stream};
    orc_philox(ctr, key, out);
}

/* u32 -> uniform on the open interval (0, 1) */
static double u32_to_unit(uint32_t u) { return ((double)u + 0.5) * (1.0 / 4294967296.0); }

/* n standard normals for (chain, iter, stream): element i uses Philox block
 * i/4; words (0,1) give a Box-Muller pair (cos, sin), words (2,3) the next. */
void orc_normals(uint64_t seed, uint32_t chain, uint32_t iter, uint32_t stream,
                 int32_t n, double *z)
{
    for (int32_t b = 0; 4 * b < n; ++b) {
        uint32_t w[4];
        philox_at(seed, (uint32_t)b, chain, iter, stream, w);
        for (int pr = 0; pr < 2; ++pr) {
            double u1 = u32_to_unit(w[2 * pr]), u2 = u32_to_unit(w[2 * pr + 1]);
            double rad = sqrt(-2.0 * log(u1));
            int i0 = 4 * b + 2 * pr;
            if (i0 < n) z[i0] = rad * cos(ORC_TWO_PI * u2);
            if (i0 + 1 < n) z[i0 + 1] = rad * sin(ORC_TWO_PI * u2);
        }
    }
}

double orc_uniform(uint64_t seed, uint32_t chain, uint32_t iter, uint32_t stream)
{
    uint32_t w[4];
    philox_at(seed, 0, chain, iter, stream, w);
    return u32_to_unit(w[0]);
}

/* uniform index in [0, n) from one Philox word: floor(u * n / 2^32), exact */
uint32_t orc_index(uint64_t seed, uint32_t chain, uint32_t iter, uint32_t stream, uint32_t n)
{
    uint32_t w[4];
    philox_at(seed, 0, chain, iter, stream, w);
    return (uint32_t)(((uint64_t)w[0] * (uint64_t)n) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Problem and fold masks                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t kind;
    int32_t p;
    int64_t N;
    const double *X;        /* N x p, row-major */
    const double *y;        /* N */
    const int32_t *fold;    /* N: fold id 0..K-1, or -1 (in no test set) */
    int32_t K;
    int32_t h;              /* h(v)-block buffer rows on each side of a test block */
    const int32_t *group;   /* N (hierarchical only) */
    int32_t G;
    double beta_sd;
    double sigma_known;     /* > 0: known noise sd */
    double sigma_sd;        /* half-normal prior scale of sigma */
    double tau_sd;          /* half-normal prior scale of tau */
    const int32_t *active;  /* p flags, 1 = covariate in the model (NULL: all);
                             * Appendix B's selection mask M_j: an inactive
                             * coefficient is held at 0 (inverse mass 0), so it
                             * drops out of the likelihood and the predictive */
} orc_problem;

int32_t orc_dim(const orc_problem *P)
{
    if (P->kind == ORC_LOGISTIC) return P->p;
    if (P->kind == ORC_HIER) return P->p + P->G + 2;
    if (P->kind == ORC_GAUSS && P->sigma_known > 0) return P->p;
    return P->p + 1;
}

/* first and last test row of fold k (for the h-block buffer) */
static void test_extent(const orc_problem *P, int32_t k, int64_t *first, int64_t *last)
{
    *first = -1; *last = -2;
    for (int64_t n = 0; n < P->N; ++n)
        if (P->fold[n] == k) { if (*first < 0) *first = n; *last = n; }
}

/* The masks of Appendix B: test_k(n) = [fold(n) == k]; train_k(n) =
 * [fold(n) != k], minus h rows on each side of the test block for h(v)-block
 * CV.  k < 0 is the full-data posterior: every row trains, none tests. */
static void fold_masks(const orc_problem *P, int32_t k, unsigned char *train, unsigned char *test)
{
    if (k < 0) {
        for (int64_t n = 0; n < P->N; ++n) { train[n] = 1; test[n] = 0; }
        return;
    }
    int64_t first, last;
    test_extent(P, k, &first, &last);
    for (int64_t n = 0; n < P->N; ++n) {
        test[n] = (P->fold[n] == k);
        int tr = (P->fold[n] != k);
        if (P->h > 0 && first >= 0 && n >= first - P->h && n <= last + P->h) tr = 0;
        train[n] = (unsigned char)tr;
    }
}

/* ------------------------------------------------------------------------ */
/* Log densities and analytic gradients                                      */
/* ------------------------------------------------------------------------ */
static double softplus(double x) { return x > 0 ? x + log1p(exp(-x)) : log1p(exp(x)); }
static double sigmoid(double x) { return x >= 0 ? 1.0 / (1.0 + exp(-x)) : exp(x) / (1.0 + exp(x)); }

/* log N(v | 0, s^2) for a normal prior */
static double lnorm(double v, double s) { return -0.5 * ORC_LOG_2PI - log(s) - 0.5 * v * v / (s * s); }
/* log half-normal(v | s) density of v > 0, with the log-Jacobian log(v) of
 * the v = exp(u) transform: returns log p(v) + u where u = log v */
static double lhalfnorm_logscale(double u, double s)
{
    double v = exp(u);
    return log(2.0) - 0.5 * ORC_LOG_2PI - log(s) - 0.5 * v * v / (s * s) + u;
}

/*
 * log N(e | 0, s2 I + t2 1 1') for a vector e of length m: the density of a
 * group's rows after its intercept tau z ~ N(0, tau^2) is integrated out.
 * Written out with a dense m x m Cholesky factor (plain on purpose).
 */
static double lmvn_compound(const double *e, int64_t m, double s2, double t2)
{
    double *A = (double *)malloc(sizeof(double) * (size_t)(m * m));
    double *w = (double *)malloc(sizeof(double) * (size_t)m);
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < m; ++j) A[i * m + j] = t2 + (i == j ? s2 : 0.0);
    double logdet = 0.0;
    for (int64_t j = 0; j < m; ++j) {              /* A = L L', L stored in the lower half */
        double v = A[j * m + j];
        for (int64_t q = 0; q < j; ++q) v -= A[j * m + q] * A[j * m + q];
        const double ljj = sqrt(v);
        A[j * m + j] = ljj;
        logdet += 2.0 * log(ljj);
        for (int64_t i = j + 1; i < m; ++i) {
            double u = A[i * m + j];
            for (int64_t q = 0; q < j; ++q) u -= A[i * m + q] * A[j * m + q];
            A[i * m + j] = u / ljj;
        }
    }
    double quad = 0.0;                             /* solve L w = e, quad = w'w */
    for (int64_t i = 0; i < m; ++i) {
        double u = e[i];
        for (int64_t q = 0; q < i; ++q) u -= A[i * m + q] * w[q];
        w[i] = u / A[i * m + i];
        quad += w[i] * w[i];
    }
    free(A); free(w);
    return -0.5 * (double)m * ORC_LOG_2PI - 0.5 * logdet - 0.5 * quad;
}

/*
 * Evaluate, for fold k and parameters theta (dimension orc_dim):
 *   logp = sum over training rows of log p(y_n | theta) + log prior(theta)
 *          (+ log-Jacobians of the log-scale parameters)      eq. mask-log-prob
 *   shat = sum over test rows of log p(y_n | theta)            eq. mask-log-pred
 *   grad = d logp / d theta
 * Hierarchical model: a group none of whose rows trains in fold k is a new
 * group for that fold, and its test rows are scored by the group-level
 * predictive of eq. group-marg, the intercept tau z integrated over
 * z ~ N(0, 1): log N(y_g | X_g beta, sigma^2 I + tau^2 1 1').  Test rows of
 * a group that also has training rows use the sampled z.
 * Masks are built per call from the fold array (slow on purpose).
 */
int orc_log_density(const orc_problem *P, int32_t k, const double *theta,
                    double *logp_out, double *grad, double *shat_out)
{
    const int64_t N = P->N;
    const int32_t p = P->p, d = orc_dim(P);
    unsigned char *train = (unsigned char *)malloc((size_t)N);
    unsigned char *test = (unsigned char *)malloc((size_t)N);
    if (!train || !test) { free(train); free(test); return -1; }
    fold_masks(P, k, train, test);
    for (int32_t j = 0; j < d; ++j) grad[j] = 0.0;

    double logp = 0.0, shat = 0.0;
    const double *beta = theta;
    double sigma = 1.0, log_sigma = 0.0, tau = 0.0, log_tau = 0.0;
    const double *z = NULL;
    if (P->kind == ORC_GAUSS || P->kind == ORC_AR) {
        if (P->kind == ORC_GAUSS && P->sigma_known > 0) { sigma = P->sigma_known; log_sigma = log(sigma); }
        else { log_sigma = theta[p]; sigma = exp(log_sigma); }
    } else if (P->kind == ORC_HIER) {
        z = theta + p;
        log_tau = theta[p + P->G];
        log_sigma = theta[p + P->G + 1];
        tau = exp(log_tau);
        sigma = exp(log_sigma);
    }
    const double inv_s2 = 1.0 / (sigma * sigma);
    double d_logsigma = 0.0, d_logtau = 0.0;

    for (int64_t n = 0; n < N; ++n) {
        if (!train[n] && !test[n]) continue;
        const double *x = P->X + n * p;
        double eta = 0.0;
        for (int32_t j = 0; j < p; ++j) eta += x[j] * beta[j];
        int32_t g = 0;
        if (P->kind == ORC_HIER) { g = P->group[n]; eta += tau * z[g]; }
        double ll, dll_deta;
        if (P->kind == ORC_LOGISTIC) {
            ll = P->y[n] * eta - softplus(eta);
            dll_deta = P->y[n] - sigmoid(eta);
        } else {
            double e = P->y[n] - eta;
            ll = -0.5 * ORC_LOG_2PI - log_sigma - 0.5 * e * e * inv_s2;
            dll_deta = e * inv_s2;
            if (train[n]) d_logsigma += -1.0 + e * e * inv_s2;
        }
        if (test[n] && P->kind != ORC_HIER) shat += ll;
        if (train[n]) {
            logp += ll;
            for (int32_t j = 0; j < p; ++j) grad[j] += dll_deta * x[j];
            if (P->kind == ORC_HIER) {
                grad[p + g] += dll_deta * tau;
                d_logtau += dll_deta * tau * z[g];
            }
        }
    }
    if (P->kind == ORC_HIER) {
        double *e = (double *)malloc(sizeof(double) * (size_t)N);
        for (int32_t g = 0; g < P->G; ++g) {
            int64_t m = 0, n_train = 0;
            for (int64_t n = 0; n < N; ++n) {
                if (P->group[n] != g) continue;
                if (train[n]) ++n_train;
                if (test[n]) {
                    double eta = 0.0;
                    for (int32_t j = 0; j < p; ++j) eta += P->X[n * p + j] * beta[j];
                    e[m++] = P->y[n] - eta;
                }
            }
            if (m == 0) continue;
            if (n_train == 0) {
                shat += lmvn_compound(e, m, sigma * sigma, tau * tau);
            } else {
                for (int64_t i = 0; i < m; ++i) {
                    const double ei = e[i] - tau * z[g];
                    shat += -0.5 * ORC_LOG_2PI - log_sigma - 0.5 * ei * ei * inv_s2;
                }
            }
        }
        free(e);
    }
    /* priors */
    for (int32_t j = 0; j < p; ++j) {
        logp += lnorm(beta[j], P->beta_sd);
        grad[j] += -beta[j] / (P->beta_sd * P->beta_sd);
    }
    if (P->kind == ORC_HIER) {
        for (int32_t g = 0; g < P->G; ++g) { logp += lnorm(z[g], 1.0); grad[p + g] += -z[g]; }
        logp += lhalfnorm_logscale(log_tau, P->tau_sd);
        grad[p + P->G] = d_logtau - tau * tau / (P->tau_sd * P->tau_sd) + 1.0;
        logp += lhalfnorm_logscale(log_sigma, P->sigma_sd);
        grad[p + P->G + 1] = d_logsigma - sigma * sigma / (P->sigma_sd * P->sigma_sd) + 1.0;
    } else if (d == p + 1) {
        logp += lhalfnorm_logscale(log_sigma, P->sigma_sd);
        grad[p] = d_logsigma - sigma * sigma / (P->sigma_sd * P->sigma_sd) + 1.0;
    }
    *logp_out = logp;
    if (shat_out) *shat_out = shat;
    free(train); free(test);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Leapfrog trajectory and one HMC transition (Section 3.3)                 */
/* ------------------------------------------------------------------------ */
/*
 * Leapfrog with diagonal inverse mass minv:
 *   r += eps/2 * grad(theta);  repeat Lf times { theta += eps * minv .* r;
 *   grad = grad(theta); r += eps * grad }, with the last momentum update a
 *   half step.  The gradient at the start is passed in (cached from the
 *   previous transition), so a trajectory costs Lf gradient evaluations.
 * On return theta, r, grad hold the end point; logp/shat its densities.
 */
int orc_trajectory(const orc_problem *P, int32_t k, double eps, int32_t Lf,
                   const double *minv, double *theta, double *r, double *grad,
                   double *logp, double *shat)
{
    const int32_t d = orc_dim(P);
    for (int32_t j = 0; j < d; ++j) r[j] += 0.5 * eps * grad[j];
    for (int32_t s = 1; s <= Lf; ++s) {
        for (int32_t j = 0; j < d; ++j) theta[j] += eps * minv[j] * r[j];
        if (orc_log_density(P, k, theta, logp, grad, shat) != 0) return -1;
        double w = (s == Lf) ? 0.5 * eps : eps;
        for (int32_t j = 0; j < d; ++j) r[j] += w * grad[j];
    }
    return 0;
}

static double kinetic(int32_t d, const double *minv, const double *r)
{
    double kin = 0.0;
    for (int32_t j = 0; j < d; ++j) kin += minv[j] * r[j] * r[j];
    return 0.5 * kin;
}

typedef struct {
    double *theta, *grad;   /* d each */
    double logp, shat;
} orc_chain;

/*
 * One HMC transition for a chain: momentum r ~ N(0, M) with M = diag(1/minv),
 * leapfrog, accept iff log u < H(start) - H(end), with H = -logp + r'M^{-1}r/2.
 * A non-finite end energy is a reject.  A transition is divergent when the
 * end energy is non-finite or exceeds the start by more than 1000.
 * Returns the acceptance probability min(1, exp(H0 - H1)) (0 if non-finite).
 */
static double hmc_transition(const orc_problem *P, int32_t k, uint64_t seed, uint32_t chain,
                             uint32_t iter, uint32_t st_mom, uint32_t st_acc, double eps,
                             int32_t Lf, const double *minv, orc_chain *c, double *work,
                             int *accepted, int *divergent)
{
    const int32_t d = orc_dim(P);
    double *r = work, *th = work + d, *gr = work + 2 * d;
    orc_normals(seed, chain, iter, st_mom, d, r);
    for (int32_t j = 0; j < d; ++j) r[j] = minv[j] > 0 ? r[j] / sqrt(minv[j]) : 0.0;   /* held coordinates: r = 0 */
    double H0 = -c->logp + kinetic(d, minv, r);
    memcpy(th, c->theta, sizeof(double) * (size_t)d);
    memcpy(gr, c->grad, sizeof(double) * (size_t)d);
    double logp1 = -INFINITY, shat1 = 0.0;
    orc_trajectory(P, k, eps, Lf, minv, th, r, gr, &logp1, &shat1);
    double H1 = -logp1 + kinetic(d, minv, r);
    double dH = H1 - H0;
    double logu = log(orc_uniform(seed, chain, iter, st_acc));
    int finite = isfinite(H1) && isfinite(dH);
    int acc = finite && (logu < -dH);
    *divergent = (!finite) || (dH > 1000.0);
    *accepted = acc;
    if (acc) {
        memcpy(c->theta, th, sizeof(double) * (size_t)d);
        memcpy(c->grad, gr, sizeof(double) * (size_t)d);
        c->logp = logp1;
        c->shat = shat1;
    }
    if (!finite) return 0.0;
    return dH <= 0 ? 1.0 : exp(-dH);
}

/* ------------------------------------------------------------------------ */
/* Online accumulators (Algorithm A2, Appendix A.1)                          */
/* ------------------------------------------------------------------------ */
static double logaddexp(double a, double b)
{
    if (a == -INFINITY) return b;
    if (b == -INFINITY) return a;
    double m = a > b ? a : b;
    return m + log1p(exp(-fabs(a - b)));
}

typedef struct {
    int64_t n;            /* draws so far */
    double Ux, Ux2;       /* log sum exp(s), log sum exp(2 s)          (A2: U_x, U_x^2) */
    double Zx;            /* log sum exp(s) over the current batch        (A2: Z_x) */
    int32_t in_batch;     /* draws in the current batch */
    /* log-shifted Welford of exp(s) over draws: values exp(s - em) */
    double em, emean, eM2;
    /* log-shifted Welford of batch means exp(Zx - log b): values exp(z - vm) */
    int64_t a;
    double vm, vmean, vM2;
    /* Welford of s over all draws (R-hat) and over the current batch */
    double wmean, wM2, bmean_cur, bM2_cur;
    double *bmean, *bM2;  /* per completed batch: Welford mean / M2 of s */
    int32_t max_batches;
    /* autocovariance lag sums of x_t = s_t - c (c = first draw) */
    int32_t M;
    double c, xsum;
    double *lagsum;       /* M+1: sum_{t>m} x_t x_{t-m} */
    double *first;        /* first M values of x */
    double *ring;         /* last M values of x (ring buffer) */
    int64_t divergences, accepts;
} orc_accum;

static void accum_init(orc_accum *A, int32_t M, int32_t max_batches)
{
    memset(A, 0, sizeof(*A));
    A->Ux = A->Ux2 = A->Zx = -INFINITY;
    A->em = A->vm = -INFINITY;
    A->M = M;
    A->max_batches = max_batches;
    A->bmean = (double *)calloc((size_t)max_batches, sizeof(double));
    A->bM2 = (double *)calloc((size_t)max_batches, sizeof(double));
    A->lagsum = (double *)calloc((size_t)M + 1, sizeof(double));
    A->first = (double *)calloc((size_t)(M > 0 ? M : 1), sizeof(double));
    A->ring = (double *)calloc((size_t)(M > 0 ? M : 1), sizeof(double));
}

static void accum_free(orc_accum *A)
{
    free(A->bmean); free(A->bM2); free(A->lagsum); free(A->first); free(A->ring);
}

/* Welford update of a log-shifted running (shift, mean, M2) with a value given
 * by its logarithm lv: the stored values are exp(lv - shift). */
static void lshift_welford(double *shift, double *mean, double *M2, int64_t count_after, double lv)
{
    if (lv > *shift) {
        if (*shift != -INFINITY) {
            double sc = exp(*shift - lv);
            *mean *= sc;
            *M2 *= sc * sc;
        }
        *shift = lv;
    }
    double v = exp(lv - *shift);
    double delta = v - *mean;
    *mean += delta / (double)count_after;
    *M2 += delta * (v - *mean);
}

/* one draw s of the held-out log predictive (batch size b) */
static void accum_push(orc_accum *A, double s, int32_t b)
{
    A->n += 1;
    A->Ux = logaddexp(A->Ux, s);
    A->Ux2 = logaddexp(A->Ux2, 2.0 * s);
    A->Zx = logaddexp(A->Zx, s);
    lshift_welford(&A->em, &A->emean, &A->eM2, A->n, s);
    /* Welford of s (all draws, and this batch) */
    double delta = s - A->wmean;
    A->wmean += delta / (double)A->n;
    A->wM2 += delta * (s - A->wmean);
    A->in_batch += 1;
    double db = s - A->bmean_cur;
    A->bmean_cur += db / (double)A->in_batch;
    A->bM2_cur += db * (s - A->bmean_cur);
    /* autocovariance lag sums */
    if (A->M >= 0) {
        if (A->n == 1) A->c = s;
        double x = s - A->c;
        int64_t t = A->n - 1;              /* 0-based time index */
        A->lagsum[0] += x * x;
        for (int32_t m = 1; m <= A->M && m <= t; ++m)
            A->lagsum[m] += x * A->ring[(t - m) % A->M];
        if (A->M > 0) {
            if (t < A->M) A->first[t] = x;
            A->ring[t % A->M] = x;
        }
        A->xsum += x;
    }
    if (A->in_batch == b) {               /* close the batch (A2 batch loop end) */
        double z = A->Zx - log((double)b);   /* log of the batch mean, eq. bmean */
        A->a += 1;
        lshift_welford(&A->vm, &A->vmean, &A->vM2, A->a, z);
        if (A->a <= A->max_batches) {
            A->bmean[A->a - 1] = A->bmean_cur;
            A->bM2[A->a - 1] = A->bM2_cur;
        }
        A->Zx = -INFINITY;
        A->in_batch = 0;
        A->bmean_cur = 0.0;
        A->bM2_cur = 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* Per-fold estimators                                                       */
/* ------------------------------------------------------------------------ */
enum { F_ELPD, F_MCSE, F_SIG2BM, F_S2, F_ESSBM, F_RHAT, F_SRHAT, F_ESSAC, F_DIV,
       F_ACTRUNC, F_ACCRATE, F_NFIELDS };
enum { T_ELPD, T_MCSE, T_SEEPI, T_RHATMAX, T_ESSTOT, T_SRHATMAX, T_DIV, T_NFIELDS };

int32_t orc_n_fold_fields(void) { return F_NFIELDS; }
int32_t orc_n_total_fields(void) { return T_NFIELDS; }

/* R-hat of eq. (rhat) from per-sequence (count n, mean, M2); L sequences */
static double rhat_from(int32_t L, const double *n, const double *mean, const double *M2)
{
    double nn = n[0];
    double W = 0.0, gm = 0.0;
    for (int32_t l = 0; l < L; ++l) { W += M2[l] / (nn - 1.0); gm += mean[l]; }
    W /= L; gm /= L;
    double B = 0.0;
    for (int32_t l = 0; l < L; ++l) B += (mean[l] - gm) * (mean[l] - gm);
    B *= nn / (L - 1.0);
    return sqrt((((nn - 1.0) / nn) * W + B / nn) / W);
}

/* Pooled (count, mean, M2) merge of Welford states (Chan et al. 1979). */
static void welford_merge(double *n, double *mean, double *M2, double n2, double mean2, double M22)
{
    double nt = *n + n2;
    if (nt == 0) return;
    double delta = mean2 - *mean;
    *mean += delta * n2 / nt;
    *M2 += M22 + delta * delta * (*n) * n2 / nt;
    *n = nt;
}

/*
 * Multi-chain autocorrelation ESS (reading of Section 4.1 with Geyer 1992):
 * per-chain autocovariances gamma_m (1/n normalisation) from the lag sums,
 * rho_m = 1 - (W - mean_l gamma_{m,l}) / var+, var+ = (n-1)/n W + B/n,
 * Geyer's initial positive sequence of pair sums rho_{2k}+rho_{2k+1},
 * made monotone, tau = -1 + 2 sum pair sums, ESS = L n / tau.
 * Sets *trunc = 1 when the sequence reached the lag cap M.
 */
static double ess_acov_fold(const orc_accum *Ac, int32_t L, double *rho_work, int *trunc)
{
    const int64_t n = Ac[0].n;
    const int32_t M = Ac[0].M;
    int32_t Mu = (int32_t)(M < n - 1 ? M : n - 1);
    double W = 0.0, gm = 0.0, B = 0.0;
    for (int32_t l = 0; l < L; ++l) {
        W += Ac[l].wM2 / (double)(n - 1);
        gm += Ac[l].wmean;
    }
    W /= L; gm /= L;
    for (int32_t l = 0; l < L; ++l) B += (Ac[l].wmean - gm) * (Ac[l].wmean - gm);
    B *= (double)n / (L - 1.0);
    double varplus = ((double)(n - 1) / n) * W + B / n;
    for (int32_t m = 0; m <= Mu; ++m) {
        double gsum = 0.0;
        for (int32_t l = 0; l < L; ++l) {
            const orc_accum *A = &Ac[l];
            double xbar = A->xsum / (double)n;
            double head = 0.0, tail = 0.0;   /* first m and last m values of x */
            for (int32_t i = 0; i < m; ++i) {
                head += A->first[i];
                tail += A->ring[(n - 1 - i) % A->M];
            }
            double P = A->xsum - head;        /* sum_{t=m}^{n-1} x_t   (0-based) */
            double Q = A->xsum - tail;        /* sum_{t=0}^{n-1-m} x_t */
            double g = A->lagsum[m] - xbar * (P + Q) + (double)(n - m) * xbar * xbar;
            gsum += g / (double)n;
        }
        rho_work[m] = 1.0 - (W - gsum / L) / varplus;
    }
    rho_work[0] = 1.0;                        /* lag-0 autocorrelation by definition */
    double tau = -1.0, prev = INFINITY;
    *trunc = 1;
    for (int32_t kk = 0; 2 * kk + 1 <= Mu; ++kk) {
        double P = rho_work[2 * kk] + rho_work[2 * kk + 1];
        if (!(P > 0.0)) { *trunc = 0; break; }
        if (P > prev) P = prev;
        prev = P;
        tau += 2.0 * P;
    }
    if (tau < 1e-12) tau = 1e-12;
    return (double)L * (double)n / tau;
}

/*
 * Per-fold results from L chains' accumulators (all with the same n, a):
 *   f_k   = (1/(Ln)) sum exp(s)                  elpd_k = log f_k (A2 final step)
 *   sig2  = b/(La-1) sum_l sum_h (mbar_lh - f_k)^2                 eq. bmvar
 *   s2    = 1/(Ln-1) sum (exp(s) - f_k)^2
 *   mcse  = sqrt(sig2/(Ln)) / f_k                          eq. mc-var (delta)
 *   ess   = Ln s2 / sig2                                        Section 4.1
 *   rhat  = eq. rhat on s; split-rhat = eq. rhat on 2L half chains (halves
 *           made of whole batches; the middle batch is dropped if a is odd).
 * sig2 and s2 are returned divided by f_k^2 (scale-free).
 */
static void fold_estimates(const orc_accum *Ac, int32_t L, int32_t b, double *out, double *rho_work)
{
    const int64_t n = Ac[0].n;
    const int64_t a = Ac[0].a;
    /* f_k via log-sum-exp of per-chain U_x */
    double lse = -INFINITY;
    for (int32_t l = 0; l < L; ++l) lse = logaddexp(lse, Ac[l].Ux);
    double logf = lse - log((double)L * (double)n);
    /* pooled log-shifted Welford of exp(s) over draws */
    double sh = -INFINITY;
    for (int32_t l = 0; l < L; ++l) if (Ac[l].em > sh) sh = Ac[l].em;
    double pn = 0, pmean = 0, pM2 = 0;
    for (int32_t l = 0; l < L; ++l) {
        double sc = exp(Ac[l].em - sh);
        welford_merge(&pn, &pmean, &pM2, (double)n, Ac[l].emean * sc, Ac[l].eM2 * sc * sc);
    }
    double fscaled = pmean;                   /* = f_k * exp(-sh) */
    double s2_rel = (pM2 / (pn - 1.0)) / (fscaled * fscaled);
    /* pooled log-shifted Welford of batch means */
    double vsh = -INFINITY;
    for (int32_t l = 0; l < L; ++l) if (Ac[l].vm > vsh) vsh = Ac[l].vm;
    double qn = 0, qmean = 0, qM2 = 0;
    for (int32_t l = 0; l < L; ++l) {
        double sc = exp(Ac[l].vm - vsh);
        welford_merge(&qn, &qmean, &qM2, (double)a, Ac[l].vmean * sc, Ac[l].vM2 * sc * sc);
    }
    /* grand mean of batch means equals f_k when every draw is in a batch */
    double fb = qmean;                        /* = f_k * exp(-vsh) */
    double sig2_rel = ((double)b * qM2 / ((double)L * (double)a - 1.0)) / (fb * fb);
    out[F_ELPD] = logf;
    out[F_SIG2BM] = sig2_rel;
    out[F_S2] = s2_rel;
    out[F_MCSE] = sqrt(sig2_rel / ((double)L * (double)n));
    out[F_ESSBM] = (double)L * (double)n * s2_rel / sig2_rel;
    /* R-hat on s */
    double *cnt = (double *)malloc(sizeof(double) * 6 * (size_t)L);
    double *mean = cnt + 2 * L, *M2 = cnt + 4 * L;
    for (int32_t l = 0; l < L; ++l) { cnt[l] = (double)n; mean[l] = Ac[l].wmean; M2[l] = Ac[l].wM2; }
    out[F_RHAT] = rhat_from(L, cnt, mean, M2);
    /* split R-hat from per-batch Welford states */
    int64_t half = a / 2;
    if (half >= 1 && a <= Ac[0].max_batches) {
        for (int32_t l = 0; l < L; ++l) {
            for (int hh = 0; hh < 2; ++hh) {
                double hn = 0, hm = 0, hM2 = 0;
                int64_t h0 = hh == 0 ? 0 : a - half;
                for (int64_t h = h0; h < h0 + half; ++h)
                    welford_merge(&hn, &hm, &hM2, (double)b, Ac[l].bmean[h], Ac[l].bM2[h]);
                cnt[2 * l + hh] = hn; mean[2 * l + hh] = hm; M2[2 * l + hh] = hM2;
            }
        }
        out[F_SRHAT] = rhat_from(2 * L, cnt, mean, M2);
    } else {
        out[F_SRHAT] = NAN;
    }
    int trunc = 0;
    out[F_ESSAC] = Ac[0].M > 0 ? ess_acov_fold(Ac, L, rho_work, &trunc) : NAN;
    out[F_ACTRUNC] = trunc;
    double dv = 0, ac = 0;
    for (int32_t l = 0; l < L; ++l) { dv += (double)Ac[l].divergences; ac += (double)Ac[l].accepts; }
    out[F_DIV] = dv;
    out[F_ACCRATE] = ac / ((double)L * (double)n);
    free(cnt);
}

/* totals over folds: elpd = sum, MCSE = sqrt(sum MCSE_k^2) (eq. mc-var),
 * se_epistemic = sqrt(K var_k(elpd_k)) (eq. norm-approx for one model),
 * R-hat_max (eq. rhat-max), aggregate ESS = Ln sum s2_k / sum sig2_k. */
static void totals(const double *fold_out, int32_t K, double Ln, double *tot)
{
    double e = 0, m2 = 0, rmax = -INFINITY, srmax = -INFINITY, s2 = 0, sg = 0, dv = 0;
    for (int32_t k = 0; k < K; ++k) {
        const double *o = fold_out + (size_t)k * F_NFIELDS;
        e += o[F_ELPD];
        m2 += o[F_MCSE] * o[F_MCSE];
        if (o[F_RHAT] > rmax) rmax = o[F_RHAT];
        if (o[F_SRHAT] > srmax) srmax = o[F_SRHAT];
        s2 += o[F_S2];
        sg += o[F_SIG2BM];
        dv += o[F_DIV];
    }
    double mean = e / K, v = 0;
    for (int32_t k = 0; k < K; ++k) {
        double dd = fold_out[(size_t)k * F_NFIELDS + F_ELPD] - mean;
        v += dd * dd;
    }
    v = K > 1 ? v / (K - 1) : 0.0;
    tot[T_ELPD] = e;
    tot[T_MCSE] = sqrt(m2);
    tot[T_SEEPI] = sqrt(K * v);
    tot[T_RHATMAX] = rmax;
    tot[T_ESSTOT] = Ln * s2 / sg;
    tot[T_SRHATMAX] = srmax;
    tot[T_DIV] = dv;
}

/*
 * Feed a given sequence of held-out log predictive draws s[C x n] (chain c
 * belongs to fold c / L) through the online accumulators and the estimators.
 * Used to pin the online path against batch formulas and to drive the GPU
 * accumulators and this oracle with identical inputs.
 */
int orc_accumulate_series(int32_t C, int32_t L, int32_t n, const double *s, int32_t b,
                          int32_t M, int32_t max_batches, double *fold_out, double *tot)
{
    if (C % L != 0 || n < 2 || b < 1) return -1;
    const int32_t K = C / L;
    orc_accum *A = (orc_accum *)calloc((size_t)C, sizeof(orc_accum));
    double *rho = (double *)malloc(sizeof(double) * ((size_t)M + 2));
    for (int32_t c = 0; c < C; ++c) {
        accum_init(&A[c], M, max_batches);
        for (int32_t t = 0; t < n; ++t) accum_push(&A[c], s[(size_t)c * n + t], b);
    }
    for (int32_t k = 0; k < K; ++k) fold_estimates(A + (size_t)k * L, L, b, fold_out + (size_t)k * F_NFIELDS, rho);
    totals(fold_out, K, (double)L * n, tot);
    for (int32_t c = 0; c < C; ++c) accum_free(&A[c]);
    free(A); free(rho);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Pairwise model selection (eq. sel-cv, eq. norm-approx, eq. mc-var)        */
/* ------------------------------------------------------------------------ */
/*
 * From the per-fold elpd and MCSE of models A and B on the same folds:
 *   delta_k = elpd_A,k - elpd_B,k,  delta = sum_k delta_k          eq. sel-cv
 *   sigma2  = 1/(K-1) sum_k (delta_k - delta/K)^2
 *   se      = sqrt(K sigma2),  Pr(A > B) = Phi(delta / se)     eq. norm-approx
 *   mcse_k  = sqrt(MCSE_A,k^2 + MCSE_B,k^2), mcse = sqrt(sum_k mcse_k^2)
 *                                     (MC variance summed over models, eq. mc-var)
 * out = {delta, se, mcse, prob}; delta_k, mcse_k per fold.
 */
int orc_compare(int32_t K, const double *elpd_a, const double *mcse_a, const double *elpd_b,
                const double *mcse_b, double *delta_k, double *mcse_k, double *out)
{
    if (K < 2) return -1;
    double sum = 0.0, mc2 = 0.0;
    for (int32_t k = 0; k < K; ++k) {
        delta_k[k] = elpd_a[k] - elpd_b[k];
        mcse_k[k] = sqrt(mcse_a[k] * mcse_a[k] + mcse_b[k] * mcse_b[k]);
        sum += delta_k[k];
        mc2 += mcse_k[k] * mcse_k[k];
    }
    double var = 0.0;
    for (int32_t k = 0; k < K; ++k) var += (delta_k[k] - sum / K) * (delta_k[k] - sum / K);
    var /= (K - 1.0);
    const double se = sqrt(K * var);
    out[0] = sum;
    out[1] = se;
    out[2] = sqrt(mc2);
    out[3] = 0.5 * erfc(-(sum / se) / sqrt(2.0));   /* Phi(delta / se) */
    return 0;
}

/* ------------------------------------------------------------------------ */
/* R-hat_max benchmark by block shuffling (Section 4.2; the shuffle loop of  */
/* Algorithm A2)                                                              */
/* ------------------------------------------------------------------------ */
/*
 * Each chain's draws are cut into D contiguous blocks of whole batches
 * (block d holds batches [d a / D, (d+1) a / D)).  A replicate rebuilds, for
 * every chain slot l of a fold, a sequence whose block d is block d of chain
 * picks[l * D + d]; its R-hat (eq. rhat) is computed from the Welford states
 * of those blocks.  With picks[l * D + d] = l the result is the fold's R-hat.
 */
double orc_rhat_from_picks_accum(const orc_accum *Ac, int32_t L, int32_t D, const int32_t *picks)
{
    const int64_t a = Ac[0].a;
    double *cnt = (double *)calloc(3 * (size_t)L, sizeof(double));
    double *mean = cnt + L, *M2 = cnt + 2 * L;
    for (int32_t l = 0; l < L; ++l) {
        for (int32_t d = 0; d < D; ++d) {
            const orc_accum *src = &Ac[picks[l * D + d]];
            int64_t h0 = (int64_t)d * a / D, h1 = (int64_t)(d + 1) * a / D;
            for (int64_t h = h0; h < h1; ++h)
                welford_merge(&cnt[l], &mean[l], &M2[l], (double)(src->n / a), src->bmean[h], src->bM2[h]);
        }
    }
    double r = rhat_from(L, cnt, mean, M2);
    free(cnt);
    return r;
}

/* The chain picks of replicate r for fold k: pick t = l D + d uses word t % 4
 * of Philox (block t / 4, chain k, iteration r, stream 4) and l' = floor(w L
 * / 2^32), a chain drawn uniformly with replacement. */
#define ST_SHUF 4u
static void shuffle_picks(uint64_t seed, int32_t k, int32_t r, int32_t L, int32_t D, int32_t *picks)
{
    for (int32_t t = 0; t < L * D; ++t) {
        uint32_t w[4];
        philox_at(seed, (uint32_t)(t / 4), (uint32_t)k, (uint32_t)r, ST_SHUF, w);
        picks[t] = (int32_t)(((uint64_t)w[t % 4] * (uint64_t)L) >> 32);
    }
}

/* R replicates of R-hat_max: out_max[r] = max over folds of the replicate's
 * R-hat; out_all[r * K + k] (optional) the per-fold values. */
static int rhat_shuffle_accums(const orc_accum *A, int32_t K, int32_t L, int32_t D, int32_t R, uint64_t seed,
                               double *out_max, double *out_all)
{
    if (D < 1 || R < 1 || A[0].a < D || A[0].a > A[0].max_batches) return -1;
    int32_t *picks = (int32_t *)malloc(sizeof(int32_t) * (size_t)L * D);
    for (int32_t r = 0; r < R; ++r) {
        double mx = -INFINITY;
        for (int32_t k = 0; k < K; ++k) {
            shuffle_picks(seed, k, r, L, D, picks);
            double v = orc_rhat_from_picks_accum(A + (size_t)k * L, L, D, picks);
            if (out_all) out_all[(size_t)r * K + k] = v;
            if (v > mx) mx = v;
        }
        out_max[r] = mx;
    }
    free(picks);
    return 0;
}

/* Drivers on a given series s[C x n] of held-out log predictive draws. */
int orc_shuffle_series(int32_t C, int32_t L, int32_t n, const double *s, int32_t b, int32_t max_batches,
                       int32_t D, int32_t R, uint64_t seed, double *out_max, double *out_all)
{
    if (C % L != 0 || n < 2 || b < 1) return -1;
    orc_accum *A = (orc_accum *)calloc((size_t)C, sizeof(orc_accum));
    for (int32_t c = 0; c < C; ++c) {
        accum_init(&A[c], 0, max_batches);
        for (int32_t t = 0; t < n; ++t) accum_push(&A[c], s[(size_t)c * n + t], b);
    }
    int rc = rhat_shuffle_accums(A, C / L, L, D, R, seed, out_max, out_all);
    for (int32_t c = 0; c < C; ++c) accum_free(&A[c]);
    free(A);
    return rc;
}
int orc_rhat_from_picks_series(int32_t L, int32_t n, const double *s, int32_t b, int32_t D, const int32_t *picks,
                               double *out)
{
    orc_accum *A = (orc_accum *)calloc((size_t)L, sizeof(orc_accum));
    for (int32_t c = 0; c < L; ++c) {
        accum_init(&A[c], 0, n / b + 1);
        for (int32_t t = 0; t < n; ++t) accum_push(&A[c], s[(size_t)c * n + t], b);
    }
    *out = orc_rhat_from_picks_accum(A, L, D, picks);
    for (int32_t c = 0; c < L; ++c) accum_free(&A[c]);
    free(A);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The PCV run: warm-up reuse (Section 3.1) and sampling (Algorithm A2)      */
/* ------------------------------------------------------------------------ */
typedef struct {
    orc_problem P;
    int32_t L, C, d, Lf, b, M, max_batches, store_draws, n_threads;
    uint64_t seed;
    double eps;
    int adapt_eps;
    double traj_len;          /* < 0: pi/2 when eps is adapted; 0: no cap */
    double jitter;            /* < 0: 0.5 when eps is adapted, else 0 */
    double *minv;             /* d */
    int user_minv;
    double init_scale;
    orc_chain *chains;        /* C */
    double *thbuf, *grbuf;    /* C x d */
    orc_accum *acc;           /* C */
    uint32_t iter;            /* fold-chain transition counter */
    int32_t n_sampled;
    double *draws;            /* C x draw_cap (store_draws) */
    int32_t draw_cap;
    double *pool;             /* full-data draws: n_pool x d */
    int32_t n_pool;
    int warmed;
    /* per-parameter accumulators (conjugate-model pin): running sum of theta,
     * current-batch sum, and a Welford of the batch means, C x d each */
    double *th_sum, *th_bsum, *th_bmean, *th_bM2;
    int64_t th_a;
    /* Hyvarinen and Dawid-Sebastiani scores (Algorithms A3, A4), Gaussian
     * models with conditionally independent rows: per chain, sums over draws
     * of xi1 = sum_i [d2 log p / dy_i^2 + (d log p / dy_i)^2] and of
     * xi2_i = d log p / dy_i (test row i), and of a predictive draw ytil and
     * its outer product (plain sums: the oracle favours the obvious form) */
    int32_t extra, T;         /* extra: 1 HS, 2 DSS; T: largest test set */
    double *hs1, *hs2, *dsum, *douter;   /* C, C x T, C x T, C x T x T */
    double fd_tail_accept;    /* mean acceptance statistic since the last dual-averaging start */
    double fd_keep_accept;    /* mean acceptance statistic of the pool draws */
    uint32_t chain_base;      /* Philox chain id of fold chain c: chain_base + c */
} orc_pcv;

orc_pcv *orc_pcv_create(const orc_problem *P, int32_t L, uint64_t seed, int32_t Lf, double eps,
                        const double *minv, int32_t b, int32_t M, int32_t max_batches,
                        int32_t store_draws, int32_t n_threads, double init_scale)
{
    orc_pcv *S = (orc_pcv *)calloc(1, sizeof(orc_pcv));
    S->P = *P;
    S->L = L; S->C = P->K * L; S->d = orc_dim(P);
    S->Lf = Lf; S->b = b; S->M = M; S->max_batches = max_batches;
    S->store_draws = store_draws; S->n_threads = n_threads > 0 ? n_threads : 1;
    S->seed = seed;
    S->eps = eps; S->adapt_eps = !(eps > 0);
    S->traj_len = -1.0; S->jitter = -1.0;
    S->init_scale = init_scale > 0 ? init_scale : 1.0;
    S->minv = (double *)malloc(sizeof(double) * (size_t)S->d);
    S->user_minv = minv != NULL;
    for (int32_t j = 0; j < S->d; ++j) S->minv[j] = minv ? minv[j] : 1.0;
    if (P->active)
        for (int32_t j = 0; j < P->p; ++j) if (!P->active[j]) S->minv[j] = 0.0;
    S->chains = (orc_chain *)calloc((size_t)S->C, sizeof(orc_chain));
    S->thbuf = (double *)calloc((size_t)S->C * S->d, sizeof(double));
    S->grbuf = (double *)calloc((size_t)S->C * S->d, sizeof(double));
    S->acc = (orc_accum *)calloc((size_t)S->C, sizeof(orc_accum));
    S->th_sum = (double *)calloc((size_t)S->C * S->d, sizeof(double));
    S->th_bsum = (double *)calloc((size_t)S->C * S->d, sizeof(double));
    S->th_bmean = (double *)calloc((size_t)S->C * S->d, sizeof(double));
    S->th_bM2 = (double *)calloc((size_t)S->C * S->d, sizeof(double));
    for (int32_t c = 0; c < S->C; ++c) {
        S->chains[c].theta = S->thbuf + (size_t)c * S->d;
        S->chains[c].grad = S->grbuf + (size_t)c * S->d;
        accum_init(&S->acc[c], M, max_batches);
    }
    return S;
}

void orc_pcv_destroy(orc_pcv *S)
{
    if (!S) return;
    for (int32_t c = 0; c < S->C; ++c) accum_free(&S->acc[c]);
    free(S->acc); free(S->chains); free(S->thbuf); free(S->grbuf);
    free(S->minv); free(S->draws); free(S->pool);
    free(S->th_sum); free(S->th_bsum); free(S->th_bmean); free(S->th_bM2);
    free(S->hs1); free(S->hs2); free(S->dsum); free(S->douter);
    free(S);
}

/* test rows of fold k in the problem's row order */
static int64_t fold_test_rows(const orc_problem *P, int32_t k, int64_t *rows)
{
    int64_t m = 0;
    for (int64_t n = 0; n < P->N; ++n) if (P->fold[n] == k) rows[m++] = n;
    return m;
}

int orc_pcv_enable_extra(orc_pcv *S, int32_t flags)
{
    const orc_problem *P = &S->P;
    /* HS needs a density in y (Gaussian rows); the DSS needs only predictive
     * draws, which the logistic model has too (Bernoulli) */
    if (P->kind != ORC_GAUSS && P->kind != ORC_AR && !(P->kind == ORC_LOGISTIC && flags == 2)) return -1;
    int64_t *rows = (int64_t *)malloc(sizeof(int64_t) * (size_t)P->N);
    int32_t T = 0;
    for (int32_t k = 0; k < P->K; ++k) {
        int64_t m = fold_test_rows(P, k, rows);
        if (m > T) T = (int32_t)m;
    }
    free(rows);
    S->extra = flags;
    S->T = T;
    S->hs1 = (double *)calloc((size_t)S->C, sizeof(double));
    S->hs2 = (double *)calloc((size_t)S->C * T, sizeof(double));
    S->dsum = (double *)calloc((size_t)S->C * T, sizeof(double));
    S->douter = (double *)calloc((size_t)S->C * T * T, sizeof(double));
    return 0;
}

/* one sampling draw of chain c (fold k) at iteration it */
static void extra_push(orc_pcv *S, int32_t c, int32_t k, uint32_t it, const double *theta, int64_t *rows,
                       double *ytil)
{
    const orc_problem *P = &S->P;
    const int64_t m = fold_test_rows(P, k, rows);
    if (P->kind == ORC_LOGISTIC) {
        /* a predictive draw ytil_i ~ Bernoulli(sigmoid(x_i' theta)): ytil_i = 1
         * iff u_i < sigmoid(eta_i), u_i from word i % 4 of Philox block i / 4
         * of stream 5 */
        for (int64_t i = 0; i < m; ++i) {
            const int64_t n = rows[i];
            double eta = 0.0;
            for (int32_t j = 0; j < P->p; ++j) eta += P->X[n * P->p + j] * theta[j];
            uint32_t w[4];
            philox_at(S->seed, (uint32_t)(i / 4), S->chain_base + (uint32_t)c, it, 5u, w);
            ytil[i] = u32_to_unit(w[i % 4]) < sigmoid(eta) ? 1.0 : 0.0;
        }
        for (int64_t i = 0; i < m; ++i) {
            S->dsum[(size_t)c * S->T + i] += ytil[i];
            for (int64_t j2 = 0; j2 < m; ++j2)
                S->douter[((size_t)c * S->T + i) * S->T + j2] += ytil[i] * ytil[j2];
        }
        return;
    }
    const double sigma = (P->kind == ORC_GAUSS && P->sigma_known > 0) ? P->sigma_known : exp(theta[P->p]);
    const double s2 = sigma * sigma;
    orc_normals(S->seed, S->chain_base + (uint32_t)c, it, 5u, (int32_t)m, ytil);   /* stream 5: predictive draws */
    double xi1 = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        const int64_t n = rows[i];
        double mu = 0.0;
        for (int32_t j = 0; j < P->p; ++j) mu += P->X[n * P->p + j] * theta[j];
        const double d1 = -(P->y[n] - mu) / s2;        /* d log N(y | mu, s2) / dy */
        const double d2 = -1.0 / s2;                     /* d2 log N / dy2 */
        xi1 += d2 + d1 * d1;
        S->hs2[(size_t)c * S->T + i] += d1;
        ytil[i] = mu + sigma * ytil[i];                  /* a draw from p(y_i | theta) */
    }
    S->hs1[c] += xi1;
    for (int64_t i = 0; i < m; ++i) {
        S->dsum[(size_t)c * S->T + i] += ytil[i];
        for (int64_t j2 = 0; j2 < m; ++j2)
            S->douter[((size_t)c * S->T + i) * S->T + j2] += ytil[i] * ytil[j2];
    }
}

/* log det and quadratic form (y - mu)' A^{-1} (y - mu) of an m x m SPD matrix
 * by a dense Cholesky factorisation (A is overwritten) */
static void chol_logdet_quad(double *A, int64_t m, const double *r, double *logdet, double *quad)
{
    double *w = (double *)malloc(sizeof(double) * (size_t)m);
    *logdet = 0.0;
    for (int64_t j = 0; j < m; ++j) {
        double v = A[j * m + j];
        for (int64_t q = 0; q < j; ++q) v -= A[j * m + q] * A[j * m + q];
        const double ljj = sqrt(v);
        A[j * m + j] = ljj;
        *logdet += 2.0 * log(ljj);
        for (int64_t i = j + 1; i < m; ++i) {
            double u = A[i * m + j];
            for (int64_t q = 0; q < j; ++q) u -= A[i * m + q] * A[j * m + q];
            A[i * m + j] = u / ljj;
        }
    }
    *quad = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        double u = r[i];
        for (int64_t q = 0; q < i; ++q) u -= A[i * m + q] * w[q];
        w[i] = u / A[i * m + i];
        *quad += w[i] * w[i];
    }
    free(w);
}

/*
 * Per fold, from the L chains' sums over n draws each:
 *   HS_k  = sum_i [ -2 E(d2_i + d1_i^2) + (E d1_i)^2 ]   (Algorithm A3, per
 *           test observation; positively oriented as in the score table)
 *   DSS_k = -log|S| - (y - m)' S^{-1} (y - m), m and S the sample mean and
 *           covariance (LN - 1 dof) of the predictive draws (Algorithm A4)
 */
int orc_pcv_extra_results(orc_pcv *S, double *hs, double *dss)
{
    if (!S->extra || S->n_sampled < 2) return -1;
    const orc_problem *P = &S->P;
    const int32_t L = S->L, T = S->T;
    const double n = (double)S->n_sampled * L;
    int64_t *rows = (int64_t *)malloc(sizeof(int64_t) * (size_t)P->N);
    double *mu = (double *)malloc(sizeof(double) * (size_t)T), *A = (double *)malloc(sizeof(double) * (size_t)T * T);
    double *r = (double *)malloc(sizeof(double) * (size_t)T);
    for (int32_t k = 0; k < P->K; ++k) {
        const int64_t m = fold_test_rows(P, k, rows);
        double e1 = 0.0;
        for (int32_t l = 0; l < L; ++l) e1 += S->hs1[k * L + l];
        double h = -2.0 * e1 / n;
        for (int64_t i = 0; i < m; ++i) {
            double e2 = 0.0;
            for (int32_t l = 0; l < L; ++l) e2 += S->hs2[(size_t)(k * L + l) * T + i];
            h += (e2 / n) * (e2 / n);
        }
        hs[k] = (S->extra & 1) ? h : NAN;               /* HS only where it was accumulated */
        for (int64_t i = 0; i < m; ++i) {
            double sm = 0.0;
            for (int32_t l = 0; l < L; ++l) sm += S->dsum[(size_t)(k * L + l) * T + i];
            mu[i] = sm / n;
        }
        for (int64_t i = 0; i < m; ++i)
            for (int64_t j2 = 0; j2 < m; ++j2) {
                double so = 0.0;
                for (int32_t l = 0; l < L; ++l) so += S->douter[((size_t)(k * L + l) * T + i) * T + j2];
                A[i * m + j2] = (so - n * mu[i] * mu[j2]) / (n - 1.0);
            }
        for (int64_t i = 0; i < m; ++i) r[i] = P->y[rows[i]] - mu[i];
        double ld, q;
        chol_logdet_quad(A, m, r, &ld, &q);
        dss[k] = -ld - q;
    }
    free(rows); free(mu); free(A); free(r);
    return 0;
}

static void chain_refresh(const orc_problem *P, int32_t k, orc_chain *c)
{
    orc_log_density(P, k, c->theta, &c->logp, c->grad, &c->shat);
}

/* Trajectory length and step-size jitter (Section 3.1 reuses the full-data
 * step size and trajectory length for every fold).  With L_f fixed, the
 * adapted step size is capped at traj_len / L_f (traj_len in units of the
 * adapted inverse mass, default pi/2), and the fold chains draw, once per
 * iteration, eps_i = eps (1 + j (2u - 1)) with u from stream 3 (Neal 2011:
 * a randomised step size breaks the periodicity of a fixed trajectory). */
int orc_pcv_set_tuning(orc_pcv *S, double traj_len, double jitter)
{
    S->traj_len = traj_len;
    S->jitter = jitter;
    return 0;
}
/* The fold chains' Philox chain ids start at chain_base (default 0): with
 * base K L the run replays the chains of a second model whose chains follow
 * the K L chains of the first in one run (Appendix B's two-model runs). */
int orc_pcv_set_chain_base(orc_pcv *S, int64_t chain_base)
{
    if (chain_base < 0 || chain_base > 0x7fffffff) return -1;
    S->chain_base = (uint32_t)chain_base;
    return 0;
}
static double eff_traj_len(const orc_pcv *S) { return S->traj_len < 0 ? 1.5707963267948966 : S->traj_len; }
static double eff_jitter(const orc_pcv *S) { return S->jitter < 0 ? (S->adapt_eps ? 0.5 : 0.0) : S->jitter; }
static double iter_eps(const orc_pcv *S, uint32_t iter)
{
    const double j = eff_jitter(S);
    if (!(j > 0)) return S->eps;
    const double u = orc_uniform(S->seed, 0, iter, ST_JIT);
    return S->eps * (1.0 + j * (2.0 * u - 1.0));
}

/* Nesterov dual averaging of the log step size (Hoffman & Gelman 2014,
 * Section 3.2.1), target acceptance delta = 0.8, gamma = 0.05, t0 = 10,
 * kappa = 0.75. */
typedef struct { double mu, hbar, logeps, logeps_bar; int64_t t; } dual_avg;
static void da_reset(dual_avg *D, double eps)
{
    D->mu = log(10.0 * eps); D->hbar = 0; D->logeps = log(eps); D->logeps_bar = 0; D->t = 0;
}
static void da_update(dual_avg *D, double accept_stat)
{
    const double delta = 0.8, gamma = 0.05, t0 = 10.0, kappa = 0.75;
    D->t += 1;
    double t = (double)D->t;
    double w = 1.0 / (t + t0);
    D->hbar = (1.0 - w) * D->hbar + w * (delta - accept_stat);
    D->logeps = D->mu - sqrt(t) / gamma * D->hbar;
    double eta = pow(t, -kappa);
    D->logeps_bar = eta * D->logeps + (1.0 - eta) * D->logeps_bar;
}

/*
 * The full-data warm-up adaptation (warm-up reuse, Section 3.1), one call per
 * completed adaptation iteration i = 0 .. n-1 (n = n_adapt):
 *   - the step size follows dual averaging on the chains' mean acceptance
 *     statistic (if it is adapted);
 *   - when the inverse mass is adapted too, the positions of iterations
 *     [n/4, n/2) form the first window and those of [n/2, 7n/8) the second;
 *     at the end of each window the diagonal inverse mass becomes
 *       minv_j = w var_j + 1e-3 (1 - w),  w = m / (m + 5)
 *     (var_j the sample variance of coordinate j over the m = chains x
 *     iterations draws of the window, m - 1 degrees of freedom), masked
 *     covariates stay at 0, and dual averaging restarts from the current
 *     step size.
 */
typedef struct {
    int32_t d, p, adapt_eps, adapt_mass, w0, w1, w2;
    const int32_t *active;    /* p flags or NULL */
    dual_avg D;
    double eps;               /* current step size */
    double *minv;             /* d, caller-owned */
    double wn, *wmean, *wM2;  /* Welford sums of the open window */
} warm_adapt;

static void wa_init(warm_adapt *A, int32_t n_adapt, int32_t d, int32_t p, const int32_t *active,
                    int adapt_eps, int adapt_mass, double eps0, double *minv)
{
    A->d = d; A->p = p; A->active = active;
    A->adapt_eps = adapt_eps; A->adapt_mass = adapt_eps && adapt_mass;
    A->w0 = n_adapt / 4; A->w1 = n_adapt / 2; A->w2 = (7 * n_adapt) / 8;
    A->eps = eps0;
    da_reset(&A->D, eps0);
    A->minv = minv;
    A->wn = 0.0;
    A->wmean = (double *)calloc((size_t)d, sizeof(double));
    A->wM2 = (double *)calloc((size_t)d, sizeof(double));
}
static void wa_free(warm_adapt *A) { free(A->wmean); free(A->wM2); }

/* after adaptation iteration i: mean acceptance statistic of the chains and
 * their positions theta[c] (nc chains); returns 1 if minv changed */
static int wa_step(warm_adapt *A, int32_t i, double mean_accept, int32_t nc, const double *const *theta)
{
    if (A->adapt_eps) {
        da_update(&A->D, mean_accept);
        A->eps = exp(A->D.logeps);
    }
    if (!A->adapt_mass || i < A->w0 || i >= A->w2) return 0;
    for (int32_t c = 0; c < nc; ++c) {
        A->wn += 1.0;
        for (int32_t j = 0; j < A->d; ++j) {
            double dl = theta[c][j] - A->wmean[j];
            A->wmean[j] += dl / A->wn;
            A->wM2[j] += dl * (theta[c][j] - A->wmean[j]);
        }
    }
    if ((i != A->w1 - 1 && i != A->w2 - 1) || !(A->wn > 1)) return 0;
    double w = A->wn / (A->wn + 5.0);
    for (int32_t j = 0; j < A->d; ++j) A->minv[j] = w * (A->wM2[j] / (A->wn - 1.0)) + 1e-3 * (1.0 - w);
    if (A->active)
        for (int32_t j = 0; j < A->p; ++j) if (!A->active[j]) A->minv[j] = 0.0;
    da_reset(&A->D, A->eps);
    A->wn = 0.0;                                  /* the next window starts afresh */
    for (int32_t j = 0; j < A->d; ++j) { A->wmean[j] = 0.0; A->wM2[j] = 0.0; }
    return 1;
}

/* the step size after adaptation: the dual-averaged exp(logeps_bar), capped
 * at cap (<= 0: no cap) */
static double wa_final_eps(const warm_adapt *A, double cap)
{
    double e = exp(A->D.logeps_bar);
    return (cap > 0 && e > cap) ? cap : e;
}

/*
 * The adaptation driven by given inputs instead of HMC transitions (for the
 * tests): accept[i] is the mean acceptance statistic after iteration i and
 * draws[(i nc + c) d + j] the position of chain c after it.  Outputs: the
 * step size after each iteration (eps_out, n_adapt), the inverse mass after
 * each iteration (minv_out, n_adapt x d, starting from minv0) and the final
 * step size with no cap.
 */
int orc_adapt_trace(int32_t n_adapt, int32_t nc, int32_t d, const double *accept, const double *draws,
                    double eps0, int32_t adapt_eps, int32_t adapt_mass, const double *minv0,
                    const int32_t *active, int32_t p, double *eps_out, double *minv_out, double *eps_final)
{
    warm_adapt A;
    double *minv = (double *)malloc(sizeof(double) * (size_t)d);
    const double **th = (const double **)malloc(sizeof(double *) * (size_t)nc);
    for (int32_t j = 0; j < d; ++j) minv[j] = minv0[j];
    wa_init(&A, n_adapt, d, p, active, adapt_eps, adapt_mass, eps0, minv);
    for (int32_t i = 0; i < n_adapt; ++i) {
        for (int32_t c = 0; c < nc; ++c) th[c] = draws + ((size_t)i * nc + c) * d;
        wa_step(&A, i, accept[i], nc, th);
        eps_out[i] = A.eps;
        memcpy(minv_out + (size_t)i * d, minv, sizeof(double) * (size_t)d);
    }
    *eps_final = wa_final_eps(&A, 0.0);
    wa_free(&A);
    free(minv); free(th);
    return 0;
}

/*
 * Full-data step (Step 1 of the workflow, as far as PCV needs it):
 * NFD = 4 full-data chains start from init_scale * N(0,1) (stream 18) and
 * run n_adapt iterations under the adaptation above (the step size when none
 * was given, from eps0; the inverse mass as well when neither was given).
 * The final step size is the dual-averaged one, capped at traj_len / L_f.
 * Then n_keep iterations at fixed settings give the pool of 4 n_keep
 * full-data draws (Algorithm 1, "draw from {theta^(fd)}").  The mean
 * acceptance statistics of the last dual-averaging phase and of the kept
 * draws are recorded for the tests.
 */
#define NFD 4
int orc_pcv_fulldata(orc_pcv *S, int32_t n_adapt, int32_t n_keep, double eps0)
{
    const orc_problem *P = &S->P;
    const int32_t d = S->d;
    orc_chain ch[NFD];
    const double *th[NFD];
    double *buf = (double *)calloc((size_t)NFD * 2 * d, sizeof(double));
    double *work = (double *)malloc(sizeof(double) * 3 * (size_t)d);
    for (int32_t c = 0; c < NFD; ++c) {
        ch[c].theta = buf + (size_t)c * 2 * d;
        ch[c].grad = ch[c].theta + d;
        th[c] = ch[c].theta;
        orc_normals(S->seed, (uint32_t)c, 0, ST_FD_INIT, d, ch[c].theta);
        for (int32_t j = 0; j < d; ++j) ch[c].theta[j] *= S->init_scale;
        if (P->active)
            for (int32_t j = 0; j < P->p; ++j) if (!P->active[j]) ch[c].theta[j] = 0.0;
        chain_refresh(P, -1, &ch[c]);
    }
    if (S->adapt_eps) S->eps = eps0 > 0 ? eps0 : 0.1;
    warm_adapt A;
    wa_init(&A, n_adapt, d, P->p, P->active, S->adapt_eps, !S->user_minv, S->eps, S->minv);
    uint32_t it = 0;
    double tail_sum = 0.0;
    int32_t tail_n = 0;
    for (int32_t i = 0; i < n_adapt; ++i, ++it) {
        double asum = 0.0;
        for (int32_t c = 0; c < NFD; ++c) {
            int acc, div;
            asum += hmc_transition(P, -1, S->seed, (uint32_t)c, it, ST_FD_MOM, ST_FD_ACC, S->eps,
                                   S->Lf, S->minv, &ch[c], work, &acc, &div);
        }
        if (wa_step(&A, i, asum / NFD, NFD, th)) {
            for (int32_t c = 0; c < NFD; ++c) chain_refresh(P, -1, &ch[c]);
            tail_sum = 0.0;                       /* dual averaging restarted */
            tail_n = 0;
        } else {
            tail_sum += asum / NFD;
            tail_n += 1;
        }
        S->eps = A.eps;
    }
    S->fd_tail_accept = tail_n > 0 ? tail_sum / tail_n : 0.0;
    if (S->adapt_eps && n_adapt > 0) {
        const double T = eff_traj_len(S);
        S->eps = wa_final_eps(&A, T > 0 ? T / S->Lf : 0.0);
    }
    wa_free(&A);
    free(S->pool);
    S->n_pool = NFD * n_keep;
    S->pool = (double *)malloc(sizeof(double) * (size_t)S->n_pool * d);
    double keep_acc = 0.0;
    for (int32_t i = 0; i < n_keep; ++i, ++it) {
        for (int32_t c = 0; c < NFD; ++c) {
            int acc, div;
            keep_acc += hmc_transition(P, -1, S->seed, (uint32_t)c, it, ST_FD_MOM, ST_FD_ACC, S->eps, S->Lf,
                                       S->minv, &ch[c], work, &acc, &div);
            memcpy(S->pool + ((size_t)i * NFD + c) * d, ch[c].theta, sizeof(double) * (size_t)d);
        }
    }
    S->fd_keep_accept = n_keep > 0 ? keep_acc / (NFD * (double)n_keep) : 0.0;
    free(buf); free(work);
    return 0;
}

/* mean acceptance statistics of the full-data chains: over the adaptation
 * iterations since dual averaging last (re)started, and over the draws kept
 * in the pool */
int orc_pcv_fulldata_accept(const orc_pcv *S, double *tail, double *keep)
{
    *tail = S->fd_tail_accept;
    *keep = S->fd_keep_accept;
    return 0;
}

/* Fold chains start from full-data draws chosen uniformly with replacement
 * (Algorithm 1, stream 2), then run n_wu discarded transitions (Step 2). */
int orc_pcv_fold_warmup(orc_pcv *S, int32_t n_wu)
{
    if (!S->pool || S->n_pool < 1) return -1;
    const orc_problem *P = &S->P;
    const int32_t d = S->d;
    for (int32_t c = 0; c < S->C; ++c) {
        uint32_t idx = orc_index(S->seed, S->chain_base + (uint32_t)c, 0, ST_INIT, (uint32_t)S->n_pool);
        memcpy(S->chains[c].theta, S->pool + (size_t)idx * d, sizeof(double) * (size_t)d);
    }
#pragma omp parallel for schedule(dynamic, 1) num_threads(S->n_threads)
    for (int32_t c = 0; c < S->C; ++c) {
        int32_t k = c / S->L;
        double *work = (double *)malloc(sizeof(double) * 3 * (size_t)d);
        chain_refresh(P, k, &S->chains[c]);
        for (int32_t i = 0; i < n_wu; ++i) {
            int acc, div;
            const uint32_t it = S->iter + (uint32_t)i;
            hmc_transition(P, k, S->seed, S->chain_base + (uint32_t)c, it, ST_MOM, ST_ACC, iter_eps(S, it),
                           S->Lf, S->minv, &S->chains[c], work, &acc, &div);
        }
        free(work);
    }
    S->iter += (uint32_t)n_wu;
    S->warmed = 1;
    return 0;
}

/* Set positions directly (C x d) instead of warming up, e.g. in tests. */
int orc_pcv_set_state(orc_pcv *S, const double *theta, double eps, const double *minv)
{
    if (eps > 0) S->eps = eps;
    if (minv) for (int32_t j = 0; j < S->d; ++j) S->minv[j] = minv[j];
#pragma omp parallel for schedule(dynamic, 1) num_threads(S->n_threads)
    for (int32_t c = 0; c < S->C; ++c) {
        memcpy(S->chains[c].theta, theta + (size_t)c * S->d, sizeof(double) * (size_t)S->d);
        chain_refresh(&S->P, c / S->L, &S->chains[c]);
    }
    S->warmed = 1;
    return 0;
}

/* Sampling (Algorithm A2 without the shuffle benchmark): n_draws transitions
 * per chain, each followed by the accumulator updates with s = log p(y_test |
 * theta) at the chain's current state.  n_draws must be a multiple of b. */
int orc_pcv_sample(orc_pcv *S, int32_t n_draws)
{
    if (!S->warmed || n_draws % S->b != 0) return -1;
    const orc_problem *P = &S->P;
    const int32_t d = S->d;
    if (S->store_draws) {
        int32_t cap = S->n_sampled + n_draws;
        double *nd = (double *)calloc((size_t)S->C * cap, sizeof(double));
        for (int32_t c = 0; c < S->C && S->draws; ++c)
            memcpy(nd + (size_t)c * cap, S->draws + (size_t)c * S->draw_cap, sizeof(double) * (size_t)S->n_sampled);
        free(S->draws);
        S->draws = nd;
        S->draw_cap = cap;
    }
#pragma omp parallel for schedule(dynamic, 1) num_threads(S->n_threads)
    for (int32_t c = 0; c < S->C; ++c) {
        int32_t k = c / S->L;
        double *work = (double *)malloc(sizeof(double) * 3 * (size_t)d);
        int64_t *xrows = S->extra ? (int64_t *)malloc(sizeof(int64_t) * (size_t)P->N) : NULL;
        double *xy = S->extra ? (double *)malloc(sizeof(double) * ((size_t)S->T + 4)) : NULL;
        for (int32_t i = 0; i < n_draws; ++i) {
            int acc, div;
            const uint32_t it = S->iter + (uint32_t)i;
            hmc_transition(P, k, S->seed, S->chain_base + (uint32_t)c, it, ST_MOM, ST_ACC, iter_eps(S, it),
                           S->Lf, S->minv, &S->chains[c], work, &acc, &div);
            S->acc[c].divergences += div;
            S->acc[c].accepts += acc;
            accum_push(&S->acc[c], S->chains[c].shat, S->b);
            if (S->extra) extra_push(S, c, k, S->iter + (uint32_t)i, S->chains[c].theta, xrows, xy);
            {
                double *ts = S->th_sum + (size_t)c * d, *tb = S->th_bsum + (size_t)c * d;
                for (int32_t j = 0; j < d; ++j) { ts[j] += S->chains[c].theta[j]; tb[j] += S->chains[c].theta[j]; }
                if (S->acc[c].in_batch == 0) {          /* a batch just closed */
                    double aa = (double)S->acc[c].a;
                    double *bm = S->th_bmean + (size_t)c * d, *b2 = S->th_bM2 + (size_t)c * d;
                    for (int32_t j = 0; j < d; ++j) {
                        double v = tb[j] / S->b, dl = v - bm[j];
                        bm[j] += dl / aa;
                        b2[j] += dl * (v - bm[j]);
                        tb[j] = 0.0;
                    }
                }
            }
            if (S->store_draws) S->draws[(size_t)c * S->draw_cap + S->n_sampled + i] = S->chains[c].shat;
        }
        free(work); free(xrows); free(xy);
    }
    S->iter += (uint32_t)n_draws;
    S->n_sampled += n_draws;
    return 0;
}

int orc_pcv_results(orc_pcv *S, double *fold_out, double *tot)
{
    if (S->n_sampled < 2 * S->b) return -1;
    double *rho = (double *)malloc(sizeof(double) * ((size_t)S->M + 2));
    for (int32_t k = 0; k < S->P.K; ++k)
        fold_estimates(S->acc + (size_t)k * S->L, S->L, S->b, fold_out + (size_t)k * F_NFIELDS, rho);
    totals(fold_out, S->P.K, (double)S->L * S->n_sampled, tot);
    free(rho);
    return 0;
}

int orc_pcv_rhat_shuffle(orc_pcv *S, int32_t D, int32_t R, double *out_max)
{
    return rhat_shuffle_accums(S->acc, S->P.K, S->L, D, R, S->seed, out_max, NULL);
}

int orc_pcv_get_draws(orc_pcv *S, double *out)
{
    if (!S->store_draws) return -1;
    for (int32_t c = 0; c < S->C; ++c)
        memcpy(out + (size_t)c * S->n_sampled, S->draws + (size_t)c * S->draw_cap, sizeof(double) * (size_t)S->n_sampled);
    return 0;
}

/* positions [C x d], step size and inverse mass [d] */
int orc_pcv_get_state(orc_pcv *S, double *theta, double *eps, double *minv, double *logp, double *shat)
{
    for (int32_t c = 0; c < S->C; ++c) {
        if (theta) memcpy(theta + (size_t)c * S->d, S->chains[c].theta, sizeof(double) * (size_t)S->d);
        if (logp) logp[c] = S->chains[c].logp;
        if (shat) shat[c] = S->chains[c].shat;
    }
    if (eps) *eps = S->eps;
    if (minv) memcpy(minv, S->minv, sizeof(double) * (size_t)S->d);
    return 0;
}

int orc_pcv_get_pool(orc_pcv *S, double *out, int32_t *n_pool)
{
    *n_pool = S->n_pool;
    if (out && S->pool) memcpy(out, S->pool, sizeof(double) * (size_t)S->n_pool * S->d);
    return 0;
}

/* per chain: posterior mean of theta, and (mean, M2) of its batch means */
int orc_pcv_theta_stats(orc_pcv *S, double *mean, double *bmean, double *bM2)
{
    if (S->n_sampled < 1) return -1;
    for (size_t i = 0; i < (size_t)S->C * S->d; ++i) {
        mean[i] = S->th_sum[i] / S->n_sampled;
        bmean[i] = S->th_bmean[i];
        bM2[i] = S->th_bM2[i];
    }
    return 0;
}
