/*
 * dpmm_oracle.c -- plain, slow FP64 CPU reference of the sub-cluster split/merge
 * Dirichlet-process mixture sampler (Dinari et al., arXiv 2204.08988, Sec. 2.3 and
 * Sec. 4.1; sampler of Chang & Fisher III, NIPS 2013).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load this library.  It shares no code, header,
 * table or constant generator with the CUDA library; both implement the same
 * written specification of the random streams (below) independently.
 *
 * Everything is double precision, single-threaded, written as straight loops in
 * the order of the paper's algorithm (Sec. 4.1 steps (a)-(f), then splits and
 * merges), so that it can be checked against the paper by eye.
 *
 * Random streams (our specification; the paper uses std::mt19937 and a
 * "C algorithm" for categorical draws, which no counter-based design can match):
 *   Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  key = (seed lo32, seed hi32),
 *   counter = (c0 = entity, c1 = sweep index lo32, c2 = (tag << 24) | block, c3 = problem).
 *   Uniform in (0,1) from words (a, b): m = ((a >> 6) << 26) | (b >> 6) (52 bits),
 *   u = (2m + 1) * 2^-53.  Reduced-precision paths use u32 = (2(a >> 9) + 1) * 2^-24.
 *   Normal number q of a stream starting at block B: Box-Muller on block B + q/2,
 *   u1 from words (0,1), u2 from words (2,3); cos branch for even q, sin for odd q.
 *   Gamma variate with base block B: Marsaglia & Tsang (2000) in log space; attempt r
 *   takes its normal from block B + 2r (cos branch) and its uniform from block
 *   B + 2r + 1 (words 0,1); at most 31 attempts; shape < 1 uses the boost
 *   G(a) = G(a + 1) U^(1/a) with U from block B + 63 (words 0,1).
 *   Tags: INIT 1, WEIGHT 2, SUBW 3, PARAM 4, Z 5, ZBAR 6, SPLIT 7, MERGE 8, RESUB 9.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_INIT 1u
#define ORC_WEIGHT 2u
#define ORC_SUBW 3u
#define ORC_PARAM 4u
#define ORC_Z 5u
#define ORC_ZBAR 6u
#define ORC_SPLIT 7u
#define ORC_MERGE 8u
#define ORC_RESUB 9u

#define ORC_NIW 0
#define ORC_DIRICHLET 1

/* ------------------------------------------------------------------ Philox */

/* Philox4x32 with 10 rounds, as published by Salmon et al. (SC'11): two 32x32->64
 * multiplications per round, Weyl-sequence key schedule. */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)M0 * x0;
        uint64_t p1 = (uint64_t)M1 * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0; k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

double orc_u01(uint32_t a, uint32_t b)
{
    uint64_t m = ((uint64_t)(a >> 6) << 26) | (uint64_t)(b >> 6);
    return (double)(2 * m + 1) * 0x1p-53;
}

float orc_u01_f32(uint32_t a)
{
    return (float)(2u * (a >> 9) + 1u) * 0x1p-24f;
}

typedef struct {
    uint64_t seed;
    uint32_t iter;
    uint32_t problem;
} orc_key;

static void orc_block(const orc_key* k, uint32_t c0, uint32_t tag, uint32_t blk, uint32_t w[4])
{
    uint32_t ctr[4] = {c0, k->iter, (tag << 24) | (blk & 0xFFFFFFu), k->problem};
    uint32_t key[2] = {(uint32_t)k->seed, (uint32_t)(k->seed >> 32)};
    orc_philox4x32_10(ctr, key, w);
}

static double orc_uniform(const orc_key* k, uint32_t c0, uint32_t tag, uint32_t blk)
{
    uint32_t w[4];
    orc_block(k, c0, tag, blk, w);
    return orc_u01(w[0], w[1]);
}

static double orc_normal(const orc_key* k, uint32_t c0, uint32_t tag, uint32_t base, uint32_t q)
{
    uint32_t w[4];
    orc_block(k, c0, tag, base + q / 2, w);
    double u1 = orc_u01(w[0], w[1]);
    double u2 = orc_u01(w[2], w[3]);
    double r = sqrt(-2.0 * log(u1));
    double ang = 2.0 * M_PI * u2;
    return (q % 2 == 0) ? r * cos(ang) : r * sin(ang);
}

/* log of a Gamma(a, 1) variate, Marsaglia & Tsang (ACM TOMS 26(3), 2000). */
double orc_log_gamma_variate(uint64_t seed, uint32_t iter, uint32_t problem, uint32_t c0,
                             uint32_t tag, uint32_t base, double a)
{
    orc_key k = {seed, iter, problem};
    double boost = 0.0;
    if (a < 1.0) {
        double U = orc_uniform(&k, c0, tag, base + 63);
        boost = log(U) / a;
        a = a + 1.0;
    }
    double dd = a - 1.0 / 3.0;
    double c = 1.0 / sqrt(9.0 * dd);
    for (uint32_t r = 0; r < 31; ++r) {
        double x = orc_normal(&k, c0, tag, base + 2 * r, 0);
        double v = 1.0 + c * x;
        if (v <= 0.0) continue;
        v = v * v * v;
        double u = orc_uniform(&k, c0, tag, base + 2 * r + 1);
        if (log(u) < 0.5 * x * x + dd - dd * v + dd * log(v)) return log(dd) + log(v) + boost;
    }
    return log(dd) + boost; /* unreachable in practice: 31 rejections in a row */
}

double orc_normal_variate(uint64_t seed, uint32_t iter, uint32_t problem, uint32_t c0,
                          uint32_t tag, uint32_t base, uint32_t q)
{
    orc_key k = {seed, iter, problem};
    return orc_normal(&k, c0, tag, base, q);
}

/* ------------------------------------------------------ small dense algebra */

/* Cholesky A = L L^T (A symmetric positive definite, row-major d x d).  Returns 0
 * on success, -1 if A is not positive definite.  L is lower-triangular. */
static int orc_cholesky(const double* A, double* L, int d)
{
    memset(L, 0, sizeof(double) * d * d);
    for (int i = 0; i < d; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = A[i * d + j];
            for (int m = 0; m < j; ++m) s -= L[i * d + m] * L[j * d + m];
            if (i == j) {
                if (!(s > 0.0)) return -1;
                L[i * d + i] = sqrt(s);
            } else {
                L[i * d + j] = s / L[j * d + j];
            }
        }
    }
    return 0;
}

/* log det of an SPD matrix via its Cholesky factor. */
static double orc_logdet_spd(const double* A, int d, int* ok)
{
    double* L = (double*)malloc(sizeof(double) * d * d);
    int r = orc_cholesky(A, L, d);
    double s = 0.0;
    for (int i = 0; i < d; ++i) s += log(L[i * d + i]);
    free(L);
    if (ok) *ok = (r == 0);
    return 2.0 * s;
}

/* log of the multivariate Gamma function Gamma_d(a). */
static double orc_lmvgamma(double a, int d)
{
    double s = 0.25 * d * (d - 1) * log(M_PI);
    for (int j = 1; j <= d; ++j) s += lgamma(a + 0.5 * (1 - j));
    return s;
}

/* ------------------------------------------------------------ the sampler */

typedef struct {
    int kind, d, K_max, init_K, burn_out;
    double alpha;
    /* NIW prior (Sec. 2.2): kappa0 > 0, m0 in R^d, nu0 > d - 1, Psi0 SPD */
    double kappa0, nu0;
    double *m0, *psi0;
    /* Dirichlet prior on multinomial parameters */
    double* beta;

    int64_t N;
    double* X; /* N x d row-major */

    int initialized;
    uint32_t iter; /* sweep counter t */
    int K;
    int32_t* z;
    uint8_t* zbar;
    int* age;

    /* sufficient statistics per slot s = 3k + {0: cluster, 1: sub l, 2: sub r} */
    double* n;   /* 3 K_max */
    double* sx;  /* 3 K_max x d */
    double* sxx; /* 3 K_max x d x d (Gaussian only) */

    /* parameters per slot */
    double* logw;    /* log pi_k for clusters, log pibar_kh for sub-clusters */
    double* mu;      /* Gaussian mean */
    double* W;       /* precision factor: Lambda = W W^T, W upper-triangular */
    double* logdetW; /* sum_j log W_jj = (1/2) log det Lambda */
    double* logtheta;/* multinomial log-probabilities */
    int params_valid;

    /* last sweep's split/merge accounting */
    int n_split, n_merge, n_split_rejected_kmax, n_removed;
} orc_state;

static int orc_stat_slots(const orc_state* o) { return 3 * o->K_max; }

orc_state* orc_create(int kind, int d, int K_max, double alpha, double kappa0, const double* m0,
                      double nu0, const double* psi0, const double* beta, int init_K, int burn_out)
{
    if (d < 1 || K_max < 1 || !(alpha > 0) || init_K < 1 || init_K > K_max) return NULL;
    orc_state* o = (orc_state*)calloc(1, sizeof(orc_state));
    o->kind = kind; o->d = d; o->K_max = K_max; o->alpha = alpha;
    o->init_K = init_K; o->burn_out = burn_out;
    o->kappa0 = kappa0; o->nu0 = nu0;
    o->m0 = (double*)calloc(d, sizeof(double));
    /* the d x d arrays exist for the Gaussian model only (a multinomial d can be 20,000) */
    const size_t dd = kind == ORC_NIW ? (size_t)d * d : 1;
    o->psi0 = (double*)calloc(dd, sizeof(double));
    o->beta = (double*)calloc(d, sizeof(double));
    if (kind == ORC_NIW) {
        memcpy(o->m0, m0, sizeof(double) * d);
        memcpy(o->psi0, psi0, sizeof(double) * d * d);
    } else {
        memcpy(o->beta, beta, sizeof(double) * d);
    }
    int S = orc_stat_slots(o);
    o->age = (int*)calloc(K_max, sizeof(int));
    o->n = (double*)calloc(S, sizeof(double));
    o->sx = (double*)calloc((size_t)S * d, sizeof(double));
    o->sxx = (double*)calloc((size_t)S * dd, sizeof(double));
    o->logw = (double*)calloc(S, sizeof(double));
    o->mu = (double*)calloc((size_t)S * d, sizeof(double));
    o->W = (double*)calloc((size_t)S * dd, sizeof(double));
    o->logdetW = (double*)calloc(S, sizeof(double));
    o->logtheta = (double*)calloc((size_t)S * d, sizeof(double));
    return o;
}

void orc_destroy(orc_state* o)
{
    if (!o) return;
    free(o->m0); free(o->psi0); free(o->beta); free(o->X); free(o->z); free(o->zbar);
    free(o->age); free(o->n); free(o->sx); free(o->sxx); free(o->logw); free(o->mu);
    free(o->W); free(o->logdetW); free(o->logtheta);
    free(o);
}

int orc_set_data(orc_state* o, const double* X, int64_t N)
{
    if (N < 1) return -1;
    free(o->X); free(o->z); free(o->zbar);
    o->N = N;
    o->X = (double*)malloc(sizeof(double) * N * o->d);
    memcpy(o->X, X, sizeof(double) * N * o->d);
    o->z = (int32_t*)calloc(N, sizeof(int32_t));
    o->zbar = (uint8_t*)calloc(N, sizeof(uint8_t));
    o->initialized = 0;
    o->iter = 0;
    o->params_valid = 0;
    return 0;
}

/* Sufficient statistics from the labels, by definition: counts, sums and sums of
 * outer products of the points of every sub-cluster; a cluster's statistics are the
 * sum of its two sub-clusters' (Sec. 4.4, "updating the sufficient statistics"). */
static void orc_compute_stats(orc_state* o)
{
    int d = o->d, S = orc_stat_slots(o);
    memset(o->n, 0, sizeof(double) * S);
    memset(o->sx, 0, sizeof(double) * S * d);
    if (o->kind == ORC_NIW) memset(o->sxx, 0, sizeof(double) * S * d * d);
    for (int64_t i = 0; i < o->N; ++i) {
        const double* x = o->X + i * d;
        int s = 3 * o->z[i] + 1 + o->zbar[i];
        o->n[s] += 1.0;
        for (int j = 0; j < d; ++j) o->sx[(size_t)s * d + j] += x[j];
        if (o->kind == ORC_NIW)
            for (int j = 0; j < d; ++j)
                for (int l = 0; l < d; ++l) o->sxx[((size_t)s * d + j) * d + l] += x[j] * x[l];
    }
    for (int k = 0; k < o->K; ++k) {
        int c = 3 * k, a = c + 1, b = c + 2;
        o->n[c] = o->n[a] + o->n[b];
        for (int j = 0; j < d; ++j) o->sx[(size_t)c * d + j] = o->sx[(size_t)a * d + j] + o->sx[(size_t)b * d + j];
        if (o->kind == ORC_NIW)
            for (int j = 0; j < d * d; ++j)
                o->sxx[(size_t)c * d * d + j] = o->sxx[(size_t)a * d * d + j] + o->sxx[(size_t)b * d * d + j];
    }
}

/* second moments of slot s (Gaussian), NULL for the multinomial model */
static const double* orc_sxx(const orc_state* o, int s)
{
    return o->kind == ORC_NIW ? o->sxx + (size_t)s * o->d * o->d : NULL;
}

int orc_set_state(orc_state* o, int K, const int32_t* z, const uint8_t* zbar)
{
    if (K < 1 || K > o->K_max) return -1;
    for (int64_t i = 0; i < o->N; ++i)
        if (z[i] < 0 || z[i] >= K || zbar[i] > 1) return -1;
    o->K = K;
    memcpy(o->z, z, sizeof(int32_t) * o->N);
    memcpy(o->zbar, zbar, o->N);
    for (int k = 0; k < o->K_max; ++k) o->age[k] = 0;
    o->initialized = 1;
    orc_compute_stats(o);
    return 0;
}

/* NIW posterior given (n, sum x, sum x x^T) -- the textbook conjugate update
 * (Gelman et al., BDA 3rd ed., Sec. 3.6; the paper's Eq. (sample_params) refers to it):
 * kappa_n = kappa0 + n, nu_n = nu0 + n, m_n = (kappa0 m0 + n xbar)/kappa_n,
 * Psi_n = Psi0 + S + (kappa0 n / kappa_n)(xbar - m0)(xbar - m0)^T with S the scatter. */
void orc_niw_posterior(const orc_state* o, double n, const double* sx, const double* sxx,
                       double* kn, double* mn, double* nun, double* psin)
{
    int d = o->d;
    *kn = o->kappa0 + n;
    *nun = o->nu0 + n;
    double* xbar = (double*)calloc(d, sizeof(double));
    if (n > 0)
        for (int j = 0; j < d; ++j) xbar[j] = sx[j] / n;
    for (int j = 0; j < d; ++j) mn[j] = (o->kappa0 * o->m0[j] + n * xbar[j]) / *kn;
    for (int j = 0; j < d; ++j)
        for (int l = 0; l < d; ++l) {
            double scatter = (n > 0) ? sxx[j * d + l] - n * xbar[j] * xbar[l] : 0.0;
            psin[j * d + l] = o->psi0[j * d + l] + scatter +
                              (o->kappa0 * n / *kn) * (xbar[j] - o->m0[j]) * (xbar[l] - o->m0[l]);
        }
    free(xbar);
}

/* log marginal likelihood f_x(C; lambda) of a set of points under the NIW prior:
 * the textbook closed form the paper defers to (Sec. 2.3, below Eq. HastingsRatioSplit). */
double orc_niw_log_marginal(const orc_state* o, double n, const double* sx, const double* sxx)
{
    int d = o->d;
    double kn, nun;
    double* mn = (double*)malloc(sizeof(double) * d);
    double* psin = (double*)malloc(sizeof(double) * d * d);
    orc_niw_posterior(o, n, sx, sxx, &kn, mn, &nun, psin);
    int ok0, okn;
    double ld0 = orc_logdet_spd(o->psi0, d, &ok0);
    double ldn = orc_logdet_spd(psin, d, &okn);
    double L = -0.5 * n * d * log(M_PI) + orc_lmvgamma(0.5 * nun, d) - orc_lmvgamma(0.5 * o->nu0, d) +
               0.5 * o->nu0 * ld0 - 0.5 * nun * ldn + 0.5 * d * (log(o->kappa0) - log(kn));
    free(mn); free(psin);
    return L;
}

/* Dirichlet-multinomial log marginal (the per-point multinomial coefficients are
 * left out: they are the same in every partition and cancel in every ratio). */
double orc_dirmult_log_marginal(const orc_state* o, const double* counts)
{
    int d = o->d;
    double sb = 0.0, sc = 0.0, L = 0.0;
    for (int j = 0; j < d; ++j) {
        sb += o->beta[j];
        sc += counts[j];
        L += lgamma(o->beta[j] + counts[j]) - lgamma(o->beta[j]);
    }
    return L + lgamma(sb) - lgamma(sb + sc);
}

static double orc_log_marginal_slot(const orc_state* o, double n, const double* sx, const double* sxx)
{
    if (o->kind == ORC_NIW) return orc_niw_log_marginal(o, n, sx, sxx);
    return orc_dirmult_log_marginal(o, sx);
}

/* Draw (mu, Lambda) ~ NIW posterior.  Lambda ~ Wishart(nu_n, Psi_n^-1) by the Bartlett
 * decomposition written with an upper-triangular factor B (B B^T ~ Wishart(nu_n, I),
 * B_jj^2 ~ chi^2(nu_n - d + j), j = 1..d, entries above the diagonal N(0,1)), and
 * W = U^-T B where Psi_n = U U^T; then Lambda = W W^T.  mu = m_n + W^-T eps / sqrt(kappa_n). */
void orc_niw_draw(const orc_state* o, uint64_t seed, uint32_t iter, uint32_t problem, uint32_t slot,
                  double kn, const double* mn, double nun, const double* psin,
                  double* W, double* mu, double* logdetW)
{
    int d = o->d;
    orc_key key = {seed, iter, problem};
    uint32_t NB = 64u * (uint32_t)d; /* first normal block of the slot's PARAM stream */
    double* U = (double*)malloc(sizeof(double) * d * d);
    double* B = (double*)calloc((size_t)d * d, sizeof(double));
    orc_cholesky(psin, U, d);
    for (int j = 0; j < d; ++j) {
        double df = nun - d + (j + 1);
        double lg = orc_log_gamma_variate(seed, iter, problem, slot, ORC_PARAM, 64u * j, 0.5 * df);
        B[j * d + j] = sqrt(2.0 * exp(lg));
        for (int l = j + 1; l < d; ++l) B[j * d + l] = orc_normal(&key, slot, ORC_PARAM, NB, (uint32_t)(j * d + l));
    }
    /* solve U^T W = B column by column (U^T upper-triangular: back substitution) */
    for (int c = 0; c < d; ++c) {
        for (int r = d - 1; r >= 0; --r) {
            double s = B[r * d + c];
            for (int m = r + 1; m < d; ++m) s -= U[m * d + r] * W[m * d + c];
            W[r * d + c] = s / U[r * d + r];
        }
    }
    /* mu = m_n + v / sqrt(kappa_n), W^T v = eps (W^T lower-triangular: forward substitution) */
    double* v = (double*)malloc(sizeof(double) * d);
    for (int j = 0; j < d; ++j) {
        double s = orc_normal(&key, slot, ORC_PARAM, NB, (uint32_t)(d * d + j));
        for (int m = 0; m < j; ++m) s -= W[m * d + j] * v[m];
        v[j] = s / W[j * d + j];
    }
    for (int j = 0; j < d; ++j) mu[j] = mn[j] + v[j] / sqrt(kn);
    free(v);
    double ld = 0.0;
    for (int j = 0; j < d; ++j) ld += log(W[j * d + j]);
    *logdetW = ld;
    free(U); free(B);
}

/* theta ~ Dir(beta + counts), kept as log theta (log-space Gamma draws). */
void orc_dirichlet_draw(const orc_state* o, uint64_t seed, uint32_t iter, uint32_t problem, uint32_t slot,
                        const double* counts, double* logtheta)
{
    int d = o->d;
    double mx = -INFINITY;
    for (int j = 0; j < d; ++j) {
        logtheta[j] = orc_log_gamma_variate(seed, iter, problem, slot, ORC_PARAM, 64u * j, o->beta[j] + counts[j]);
        if (logtheta[j] > mx) mx = logtheta[j];
    }
    double s = 0.0;
    for (int j = 0; j < d; ++j) s += exp(logtheta[j] - mx);
    double lse = mx + log(s);
    for (int j = 0; j < d; ++j) logtheta[j] -= lse;
}

/* Steps (a)-(d) of Sec. 4.1: weights, sub-weights, cluster and sub-cluster parameters. */
static void orc_draw_params(orc_state* o, uint64_t seed, uint32_t problem)
{
    int d = o->d, K = o->K;
    uint32_t t = o->iter;
    /* (a) (pi_1..pi_K, pi~_{K+1}) ~ Dir(N_1, ..., N_K, alpha) */
    double* lg = (double*)malloc(sizeof(double) * (K + 1));
    for (int k = 0; k < K; ++k) lg[k] = orc_log_gamma_variate(seed, t, problem, (uint32_t)k, ORC_WEIGHT, 0, o->n[3 * k]);
    lg[K] = orc_log_gamma_variate(seed, t, problem, 0xFFFFFFFFu, ORC_WEIGHT, 0, o->alpha);
    double mx = -INFINITY;
    for (int k = 0; k <= K; ++k) if (lg[k] > mx) mx = lg[k];
    double s = 0.0;
    for (int k = 0; k <= K; ++k) s += exp(lg[k] - mx);
    double lse = mx + log(s);
    for (int k = 0; k < K; ++k) o->logw[3 * k] = lg[k] - lse;
    free(lg);
    /* (b) (pibar_kl, pibar_kr) ~ Dir(N_kl + alpha/2, N_kr + alpha/2) */
    for (int k = 0; k < K; ++k) {
        double gl = orc_log_gamma_variate(seed, t, problem, (uint32_t)k, ORC_SUBW, 0, o->n[3 * k + 1] + 0.5 * o->alpha);
        double gr = orc_log_gamma_variate(seed, t, problem, (uint32_t)k, ORC_SUBW, 64, o->n[3 * k + 2] + 0.5 * o->alpha);
        double m = gl > gr ? gl : gr;
        double l2 = m + log(exp(gl - m) + exp(gr - m));
        o->logw[3 * k + 1] = gl - l2;
        o->logw[3 * k + 2] = gr - l2;
    }
    /* (c), (d) theta_k and thetabar_kh from their posteriors */
    double* mn = (double*)malloc(sizeof(double) * d);
    double* psin = (double*)malloc(sizeof(double) * (o->kind == ORC_NIW ? (size_t)d * d : 1));
    for (int s3 = 0; s3 < 3 * K; ++s3) {
        const double* sx = o->sx + (size_t)s3 * d;
        if (o->kind == ORC_NIW) {
            double kn, nun;
            orc_niw_posterior(o, o->n[s3], sx, o->sxx + (size_t)s3 * d * d, &kn, mn, &nun, psin);
            orc_niw_draw(o, seed, t, problem, (uint32_t)s3, kn, mn, nun, psin, o->W + (size_t)s3 * d * d,
                         o->mu + (size_t)s3 * d, o->logdetW + s3);
        } else {
            orc_dirichlet_draw(o, seed, t, problem, (uint32_t)s3, sx, o->logtheta + (size_t)s3 * d);
        }
    }
    free(mn); free(psin);
    o->params_valid = 1;
}

/* log f_x(x; theta_s) for slot s.  Gaussian: log N(x; mu, Lambda^-1) =
 * -(d/2) log 2pi + (1/2) log det Lambda - (1/2) ||W^T (x - mu)||^2.
 * Multinomial: sum_j x_j log theta_j (multinomial coefficient dropped: it is the
 * same for every k and cannot change a draw). */
static double orc_loglik(const orc_state* o, int s, const double* x)
{
    int d = o->d;
    if (o->kind == ORC_NIW) {
        const double* W = o->W + (size_t)s * d * d;
        const double* mu = o->mu + (size_t)s * d;
        double q = 0.0;
        for (int j = 0; j < d; ++j) {
            double y = 0.0;
            for (int l = 0; l < d; ++l) y += W[l * d + j] * (x[l] - mu[l]);
            q += y * y;
        }
        return -0.5 * d * log(2.0 * M_PI) + o->logdetW[s] - 0.5 * q;
    }
    const double* lt = o->logtheta + (size_t)s * d;
    double a = 0.0;
    for (int j = 0; j < d; ++j) a += x[j] * lt[j];
    return a;
}

/* Gumbel-max draw: argmax_k (score_k + G_k), G_k = -log(-log u_k). */
static double orc_gumbel(double u) { return -log(-log(u)); }

/* Steps (e) and (f) of Sec. 4.1 for point i: its cluster label, then its sub-cluster
 * label, each a Gumbel-max draw over log pi + log f with uniforms keyed by the point. */
static void orc_label_point(const orc_state* o, const orc_key* key, int64_t i, int32_t* zi, uint8_t* zbi)
{
    int d = o->d, K = o->K;
    const double* x = o->X + i * d;
    double best = -INFINITY;
    int zb = 0;
    for (int k = 0; k < K; ++k) {
        uint32_t w[4];
        orc_block(key, (uint32_t)i, ORC_Z, (uint32_t)(k / 2), w);
        double u = (k % 2 == 0) ? orc_u01(w[0], w[1]) : orc_u01(w[2], w[3]);
        double v = o->logw[3 * k] + orc_loglik(o, 3 * k, x) + orc_gumbel(u);
        if (v > best) { best = v; zb = k; }
    }
    *zi = zb;
    uint32_t w[4];
    orc_block(key, (uint32_t)i, ORC_ZBAR, 0, w);
    double vl = o->logw[3 * zb + 1] + orc_loglik(o, 3 * zb + 1, x) + orc_gumbel(orc_u01(w[0], w[1]));
    double vr = o->logw[3 * zb + 2] + orc_loglik(o, 3 * zb + 2, x) + orc_gumbel(orc_u01(w[2], w[3]));
    *zbi = (vr > vl) ? 1 : 0;
}

/* Steps (e) and (f) of Sec. 4.1 for every point. */
static void orc_draw_labels(orc_state* o, uint64_t seed, uint32_t problem)
{
    orc_key key = {seed, o->iter, problem};
    for (int64_t i = 0; i < o->N; ++i) orc_label_point(o, &key, i, &o->z[i], &o->zbar[i]);
}

static void orc_compact(orc_state* o, const int* dead);

/* Initial labels: K = init_K, z uniform over the K clusters, zbar a fair coin. */
static void orc_init_labels(orc_state* o, uint64_t seed, uint32_t problem)
{
    orc_key key = {seed, 0, problem};
    o->K = o->init_K;
    for (int64_t i = 0; i < o->N; ++i) {
        uint32_t w[4];
        orc_block(&key, (uint32_t)i, ORC_INIT, 0, w);
        int k = (int)(orc_u01(w[0], w[1]) * o->init_K);
        if (k >= o->init_K) k = o->init_K - 1;
        o->z[i] = k;
        o->zbar[i] = orc_u01(w[2], w[3]) < 0.5 ? 0 : 1;
    }
    for (int k = 0; k < o->K_max; ++k) o->age[k] = 0;
    o->initialized = 1;
    orc_compute_stats(o);
    int* dead = (int*)calloc(o->K, sizeof(int));
    int any = 0;
    for (int k = 0; k < o->K; ++k) if (o->n[3 * k] == 0) { dead[k] = 1; any = 1; }
    if (any) { orc_compact(o, dead); orc_compute_stats(o); }
    free(dead);
}

/* Stable removal of empty clusters: the survivors keep their order. */
static void orc_compact(orc_state* o, const int* dead)
{
    int* newid = (int*)malloc(sizeof(int) * o->K);
    int Kn = 0;
    for (int k = 0; k < o->K; ++k) newid[k] = dead[k] ? -1 : Kn++;
    for (int64_t i = 0; i < o->N; ++i) o->z[i] = newid[o->z[i]];
    for (int k = 0; k < o->K; ++k)
        if (newid[k] >= 0) o->age[newid[k]] = o->age[k];
    o->K = Kn;
    free(newid);
}

/* Splits (Eq. sample_splits) then merges (Eq. sample_merges); then relabelling. */
static void orc_split_merge(orc_state* o, uint64_t seed, uint32_t problem)
{
    int d = o->d, K = o->K;
    orc_key key = {seed, o->iter, problem};
    double la = log(o->alpha);
    int S = K; /* number of slots after splits */
    int* split_to = (int*)malloc(sizeof(int) * o->K_max);   /* new slot of sub r, or -1 */
    int* touched = (int*)calloc(o->K_max, sizeof(int));
    int* merged_into = (int*)malloc(sizeof(int) * o->K_max);/* -1, or k1 for an absorbed k2 */
    int* merge_head = (int*)calloc(o->K_max, sizeof(int));
    for (int k = 0; k < o->K_max; ++k) { split_to[k] = -1; merged_into[k] = -1; }

    for (int k = 0; k < K; ++k) {
        double nl = o->n[3 * k + 1], nr = o->n[3 * k + 2], nk = o->n[3 * k];
        if (o->age[k] < o->burn_out || nl < 1 || nr < 1) continue;
        double lH = la + lgamma(nl) + orc_log_marginal_slot(o, nl, o->sx + (size_t)(3 * k + 1) * d, orc_sxx(o, 3 * k + 1)) +
                    lgamma(nr) + orc_log_marginal_slot(o, nr, o->sx + (size_t)(3 * k + 2) * d, orc_sxx(o, 3 * k + 2)) -
                    lgamma(nk) - orc_log_marginal_slot(o, nk, o->sx + (size_t)(3 * k) * d, orc_sxx(o, 3 * k));
        double u = orc_uniform(&key, (uint32_t)k, ORC_SPLIT, 0);
        if (log(u) < lH) {
            if (S >= o->K_max) { o->n_split_rejected_kmax++; continue; }
            split_to[k] = S;
            touched[k] = 1;
            touched[S] = 1;
            S++;
            o->n_split++;
        }
    }

    double* sxm = (double*)malloc(sizeof(double) * d);
    double* sxxm = o->kind == ORC_NIW ? (double*)malloc(sizeof(double) * d * d) : NULL;
    for (int k1 = 0; k1 < K; ++k1) {
        if (touched[k1] || merged_into[k1] >= 0 || merge_head[k1]) continue;
        for (int k2 = k1 + 1; k2 < K; ++k2) {
            if (touched[k2] || merged_into[k2] >= 0 || merge_head[k2]) continue;
            double n1 = o->n[3 * k1], n2 = o->n[3 * k2], nm = n1 + n2;
            for (int j = 0; j < d; ++j) sxm[j] = o->sx[(size_t)3 * k1 * d + j] + o->sx[(size_t)3 * k2 * d + j];
            if (sxxm)
                for (int j = 0; j < d * d; ++j) sxxm[j] = o->sxx[(size_t)3 * k1 * d * d + j] + o->sxx[(size_t)3 * k2 * d * d + j];
            double lH = lgamma(nm) - la - lgamma(n1) - lgamma(n2) +
                        orc_log_marginal_slot(o, nm, sxm, sxxm) -
                        orc_log_marginal_slot(o, n1, o->sx + (size_t)3 * k1 * d, orc_sxx(o, 3 * k1)) -
                        orc_log_marginal_slot(o, n2, o->sx + (size_t)3 * k2 * d, orc_sxx(o, 3 * k2)) +
                        lgamma(o->alpha) - lgamma(o->alpha + nm) + lgamma(0.5 * o->alpha + n1) +
                        lgamma(0.5 * o->alpha + n2) - 2.0 * lgamma(0.5 * o->alpha);
            double u = orc_uniform(&key, (uint32_t)k1, ORC_MERGE, (uint32_t)k2);
            if (log(u) < lH) {
                merged_into[k2] = k1;
                merge_head[k1] = 1;
                o->n_merge++;
                break; /* k1 takes part in one merge only (Sec. 4.3) */
            }
        }
    }
    free(sxm); free(sxxm);

    int changed = (o->n_split + o->n_merge) > 0;
    if (changed) {
        for (int64_t i = 0; i < o->N; ++i) {
            int k = o->z[i];
            if (split_to[k] >= 0) {
                if (o->zbar[i] == 1) o->z[i] = split_to[k];
                o->zbar[i] = orc_uniform(&key, (uint32_t)i, ORC_RESUB, 0) < 0.5 ? 0 : 1;
            } else if (merged_into[k] >= 0) {
                o->z[i] = merged_into[k];
                o->zbar[i] = 1;
            } else if (merge_head[k]) {
                o->zbar[i] = 0;
            }
        }
        for (int k = 0; k < K; ++k) {
            if (split_to[k] >= 0) { o->age[k] = -1; o->age[split_to[k]] = -1; }
            if (merge_head[k]) o->age[k] = -1;
        }
        o->K = S;
        int* dead = (int*)calloc(S, sizeof(int));
        for (int k = 0; k < K; ++k) dead[k] = merged_into[k] >= 0;
        orc_compact(o, dead);
        free(dead);
    }
    free(split_to); free(touched); free(merged_into); free(merge_head);
}

/* One sweep of Sec. 4.1: (a)-(d) parameters, (e)-(f) labels, statistics, removal of
 * clusters the restricted step emptied, splits, merges, statistics again.
 * step_mask bit 0: draw parameters (else keep the injected ones); bit 1: labels;
 * bit 2: splits and merges. */
static void orc_one_sweep(orc_state* o, uint64_t seed, uint32_t problem, unsigned mask)
{
    o->n_split = o->n_merge = o->n_split_rejected_kmax = o->n_removed = 0;
    if (mask & 1u) orc_draw_params(o, seed, problem);
    if (mask & 2u) {
        orc_draw_labels(o, seed, problem);
        orc_compute_stats(o);
        int* dead = (int*)calloc(o->K, sizeof(int));
        int any = 0;
        for (int k = 0; k < o->K; ++k) if (o->n[3 * k] == 0) { dead[k] = 1; any = 1; o->n_removed++; }
        if (any) { orc_compact(o, dead); orc_compute_stats(o); }
        free(dead);
    }
    if (mask & 4u) {
        orc_split_merge(o, seed, problem);
        orc_compute_stats(o);
    }
    for (int k = 0; k < o->K; ++k) o->age[k] += 1;
    o->iter += 1;
}

int orc_sweep(orc_state* o, int iters, uint64_t seed, uint32_t problem, unsigned mask)
{
    if (!o->X) return -1;
    if (!o->initialized) orc_init_labels(o, seed, problem);
    for (int it = 0; it < iters; ++it) {
        if ((mask & 2u) && !(mask & 1u) && !o->params_valid) return -2;
        orc_one_sweep(o, seed, problem, mask);
    }
    return 0;
}

/* Parameters only (steps (a)-(d)) at the current sweep index; the sweep counter
 * does not move.  Used to hand identical parameters to another implementation. */
int orc_draw_params_only(orc_state* o, uint64_t seed, uint32_t problem)
{
    if (!o->X) return -1;
    if (!o->initialized) orc_init_labels(o, seed, problem);
    orc_draw_params(o, seed, problem);
    return 0;
}

int orc_get_K(const orc_state* o) { return o->K; }
uint32_t orc_get_iter(const orc_state* o) { return o->iter; }
void orc_set_iter(orc_state* o, uint32_t t) { o->iter = t; }

void orc_get_labels(const orc_state* o, int32_t* z, uint8_t* zbar)
{
    memcpy(z, o->z, sizeof(int32_t) * o->N);
    memcpy(zbar, o->zbar, o->N);
}

/* Statistics of the 3K slots (s = 3k + {0,1,2}); sxx may be NULL. */
void orc_get_stats(const orc_state* o, double* n, double* sx, double* sxx)
{
    int d = o->d, S = 3 * o->K;
    memcpy(n, o->n, sizeof(double) * S);
    memcpy(sx, o->sx, sizeof(double) * S * d);
    if (sxx && o->kind == ORC_NIW) memcpy(sxx, o->sxx, sizeof(double) * S * d * d);
}

void orc_get_params(const orc_state* o, double* logw, double* mu, double* W, double* logdetW, double* logtheta)
{
    int d = o->d, S = 3 * o->K;
    if (logw) memcpy(logw, o->logw, sizeof(double) * S);
    if (mu) memcpy(mu, o->mu, sizeof(double) * S * d);
    if (W && o->kind == ORC_NIW) memcpy(W, o->W, sizeof(double) * S * d * d);
    if (logdetW) memcpy(logdetW, o->logdetW, sizeof(double) * S);
    if (logtheta) memcpy(logtheta, o->logtheta, sizeof(double) * S * d);
}

void orc_get_counters(const orc_state* o, int* out4)
{
    out4[0] = o->n_split; out4[1] = o->n_merge; out4[2] = o->n_split_rejected_kmax; out4[3] = o->n_removed;
}

void orc_get_ages(const orc_state* o, int* age) { memcpy(age, o->age, sizeof(int) * o->K); }

/* Labels (steps (e)-(f)) that the current parameters would give at sweep index
 * `iter`, without touching the chain's state.  Used by the pins on the categorical
 * draws. */
void orc_label_probe(orc_state* o, uint64_t seed, uint32_t iter, uint32_t problem, int32_t* z, uint8_t* zbar)
{
    uint32_t keep = o->iter;
    int32_t* zk = o->z;
    uint8_t* zbk = o->zbar;
    o->iter = iter;
    o->z = z;
    o->zbar = zbar;
    orc_draw_labels(o, seed, problem);
    o->z = zk;
    o->zbar = zbk;
    o->iter = keep;
}

/* The same labels as orc_label_probe, for the listed points only (idx[0..n), global
 * point indices, so the random streams are those of the whole data set).  Used where
 * the data set is too large for the whole label step to run in seconds. */
void orc_label_probe_points(const orc_state* o, uint64_t seed, uint32_t iter, uint32_t problem, const int64_t* idx,
                            int64_t n, int32_t* z, uint8_t* zbar)
{
    orc_key key = {seed, iter, problem};
    for (int64_t q = 0; q < n; ++q) orc_label_point(o, &key, idx[q], &z[q], &zbar[q]);
}
