/*
 * Plain FP64 oracle for PCDM1 on LASSO (Richtarik & Takac, "Parallel Coordinate
 * Descent Methods for Big Data Optimization", arXiv:1212.0873).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path calls this file: only
 * the tests, the smoke check and the CPU-baseline leg of the benchmark load it.
 * It shares no code, header or constant table with the CUDA library; the two
 * meet only through the seeded instance generator and the written spec of the
 * sampler (Philox4x32-10 keyed Feistel permutation, restated below).
 *
 * Everything is single-threaded, in IEEE double, in the order the paper states
 * the steps.  Build with -ffp-contract=off so x86 and Arm hosts agree bit for
 * bit.
 *
 * Functions and the passage each one follows:
 *   pcdm_oracle_philox4x32_10   Salmon, Moraes, Dror, Shaw, SC'11 (Philox-4x32, 10 rounds)
 *   pcdm_oracle_sample          tau-nice sampling, Sec. 4.1 item 3 (every tau-subset
 *                               equally likely), realised by the keyed permutation
 *                               spec below (Philox round keys, 12 Feistel rounds)
 *   pcdm_oracle_col_sqnorms     L_i = ||a_i||^2, Sec. 3 item "Partial separability"
 *   pcdm_oracle_omega           omega = max_j ||A_j||_0, Sec. 1 "Examples of partially
 *                               separable functions"
 *   pcdm_oracle_beta_nice       beta = 1 + (omega-1)(tau-1)/max(1,n-1), Theorem ESO-nice
 *                               (eq. inequalityToGetZeta), Table ESO
 *   pcdm_oracle_iteration       Algorithm 1 (PCDM1), step 4, with h(x) from eq. (h(x))
 *                               and H_{beta,w} (eq. H_{beta,w}) for Omega = lambda*||.||_1, w = L
 *   pcdm_oracle_residual        g = A x - b (the gradient of f is A^T g)
 *   pcdm_oracle_gap             LASSO duality gap at the dual point theta = s*g
 *   pcdm_oracle_objective       F(x) = 1/2 ||Ax-b||^2 + lambda ||x||_1  (eq. P with LASSO, Sec. 8.1)
 *   pcdm_oracle_run             K iterations of Algorithm 1 with the residual refreshed
 *                               every refresh_every iterations
 *   pcdm_oracle_sample_independent   tau-independent sampling (Sec. 4.1, item 4): tau iid
 *                               uniform picks; a block picked more than once is updated
 *                               once (the first pick), the others are idle
 *   pcdm_oracle_binomial_keep   (tau, p_b)-binomial sampling (Sec. 4.1, item 5, case 2):
 *                               the tau-nice positions, each kept with probability p_b
 *   pcdm_oracle_q_independent   the paper's q_k = C(n,k) c_k recursion for item 4
 *   pcdm_oracle_moments         E|S| and E|S|^2 of the three samplings
 *   pcdm_oracle_beta_du         beta of Theorem ESO-DU from E|S| and E|S|^2
 *   pcdm_oracle_run_sampling    pcdm_oracle_run with the sampling chosen by `kind`
 *
 * Sampler spec (shared in words only):
 *   w = smallest even integer >= 2 with 2^w >= n;  hb = w/2;  mask = 2^hb - 1
 *   round keys of iteration k: K[4c .. 4c+3] = Philox4x32-10(counter = (c, 0, lo32(k), hi32(k)),
 *                                                 key = (lo32(seed), hi32(seed))),  c = 0, 1, 2
 *   F_r(R) = fmix32(R xor K[r]) & mask, fmix32 the 32-bit finalizer of MurmurHash3
 *            (h ^= h>>16; h *= 0x85EBCA6B; h ^= h>>13; h *= 0xC2B2AE35; h ^= h>>16)
 *   pi(v): L = v >> hb, R = v & mask; for r = 0..11: (L, R) <- (R, L xor F_r(R));
 *          return (L << hb) | R
 *   S_k[j] = first element below n of pi(j), pi(pi(j)), ...   (cycle walking)
 * pi is a bijection of [0, 2^w), so cycle walking yields a bijection of [0, n)
 * and S_k[0..tau-1] are tau distinct coordinates.  All randomness comes from
 * Philox; the Feistel rounds only mix it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

/* Twelve rounds: with four to eight, the distribution of sampled subsets on
 * small domains (n <= 64) fails a chi-square test against the uniform law; with
 * twelve the p-values over many small domains are uniformly distributed. */
#define ORACLE_FEISTEL_ROUNDS 12

/* ---------------------------------------------------------------------- */
/* Philox4x32-10 (SC'11 Sec. 4): ten rounds of two 32x32->64 multiplies,   */
/* a word permutation and xor with a Weyl-sequence key schedule.           */
/* ---------------------------------------------------------------------- */
void pcdm_oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Half width of the Feistel domain for a given n (see spec above). */
static int feistel_half_bits(int64_t n)
{
    int w = 2;
    while (((int64_t)1 << w) < n) w += 2;
    return w / 2;
}

/* MurmurHash3's 32-bit finalizer (Appleby): a bijective avalanche mix. */
static uint32_t fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

/* The 12 round keys of iteration k: three Philox4x32-10 blocks. */
static void round_keys(uint64_t seed, uint64_t k, uint32_t K[12])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (uint32_t c = 0; c < 3; ++c) {
        uint32_t ctr[4] = {c, 0u, (uint32_t)k, (uint32_t)(k >> 32)};
        pcdm_oracle_philox4x32_10(ctr, key, K + 4 * c);
    }
}

static uint32_t feistel_permute(uint32_t v, int hb, const uint32_t K[12])
{
    uint32_t mask = (hb >= 32) ? 0xFFFFFFFFu : (((uint32_t)1 << hb) - 1u);
    uint32_t left = v >> hb, right = v & mask;
    for (uint32_t r = 0; r < ORACLE_FEISTEL_ROUNDS; ++r) {
        uint32_t f = fmix32(right ^ K[r]) & mask;
        uint32_t new_right = left ^ f;
        left = right;
        right = new_right;
    }
    return (left << hb) | right;
}

/* Positions j0 .. j1-1 of the tau-nice sample of iteration k: S[j0..j1-1].
 * Returns 0, or -1 on bad sizes. */
int pcdm_oracle_sample_range(uint64_t seed, int64_t k, int64_t n, int64_t j0, int64_t j1, int32_t *S)
{
    if (n < 1 || n > 2147483647LL || j0 < 0 || j1 < j0 || j1 > n || k < 0) return -1;
    int hb = feistel_half_bits(n);
    uint32_t K[12];
    round_keys(seed, (uint64_t)k, K);
    for (int64_t j = j0; j < j1; ++j) {
        uint32_t v = feistel_permute((uint32_t)j, hb, K);
        while ((int64_t)v >= n) v = feistel_permute(v, hb, K);
        S[j] = (int32_t)v;
    }
    return 0;
}

/* tau-nice sample of iteration k: S[0..tau-1].  Returns 0, or -1 on bad sizes. */
int pcdm_oracle_sample(uint64_t seed, int64_t k, int64_t n, int64_t tau, int32_t *S)
{
    if (tau < 0 || tau > n) return -1;
    return pcdm_oracle_sample_range(seed, k, n, 0, tau, S);
}

/* Samples of iterations k0 .. k0+K-1, row after row, into out[K*tau]. */
int pcdm_oracle_sample_many(uint64_t seed, int64_t k0, int64_t K, int64_t n, int64_t tau, int32_t *out)
{
    for (int64_t q = 0; q < K; ++q)
        if (pcdm_oracle_sample(seed, k0 + q, n, tau, out + q * tau) != 0) return -1;
    return 0;
}

/* Number of Feistel rounds of the spec, exported so tests can report it. */
int pcdm_oracle_feistel_rounds(void) { return ORACLE_FEISTEL_ROUNDS; }

/* ---------------------------------------------------------------------- */
/* Problem constants                                                       */
/* ---------------------------------------------------------------------- */

/* L_i = sum_r a_ri^2, summed in storage order. */
void pcdm_oracle_col_sqnorms(int64_t n, const int64_t *col_ptr, const double *val, double *L)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t p = col_ptr[i]; p < col_ptr[i + 1]; ++p) s += val[p] * val[p];
        L[i] = s;
    }
}

/* omega = largest number of nonzeros in a row of A (0 when A has none). */
int64_t pcdm_oracle_omega(int64_t m, int64_t n, const int64_t *col_ptr, const int32_t *row_idx)
{
    int64_t *count = (int64_t *)calloc((size_t)(m > 0 ? m : 1), sizeof(int64_t));
    if (!count) return -1;
    for (int64_t p = col_ptr[0]; p < col_ptr[n]; ++p) count[row_idx[p]] += 1;
    int64_t omega = 0;
    for (int64_t r = 0; r < m; ++r)
        if (count[r] > omega) omega = count[r];
    free(count);
    return omega;
}

/* beta for the tau-nice sampling (Theorem ESO-nice).  omega is taken as at
 * least 1 so that an all-zero A still gives beta = 1. */
double pcdm_oracle_beta_nice(int64_t omega, int64_t tau, int64_t n)
{
    double om = (double)(omega < 1 ? 1 : omega);
    double denom = (double)(n - 1 > 1 ? n - 1 : 1);
    return 1.0 + (om - 1.0) * ((double)tau - 1.0) / denom;
}

/* ---------------------------------------------------------------------- */
/* The method                                                              */
/* ---------------------------------------------------------------------- */

static double soft_threshold(double u, double t)
{
    if (u > t) return u - t;
    if (u < -t) return u + t;
    return 0.0;
}

/*
 * One PCDM1 iteration on the set S (tau distinct coordinates), Jacobi style:
 * every h_i is computed from the same x_k and the same residual g = A x_k - b,
 * and only then are x and g moved.
 *   grad_i = a_i^T g
 *   h_i    = argmin_t grad_i t + (beta L_i / 2) t^2 + lambda |x_i + t|
 *          = soft(x_i - grad_i/(beta L_i), lambda/(beta L_i)) - x_i
 * A column with L_i = 0 leaves only lambda |x_i + t|, minimised by t = -x_i.
 * The new coordinate is stored as the soft-threshold value itself and the
 * residual moves by a_i * (x_new - x_old).
 * hbuf and xbuf are scratch arrays of length tau.
 *
 * pcdm_oracle_steps is the first half for positions t0 .. t1-1 (x_new and h
 * into xbuf[t], hbuf[t]; it only reads x and g), pcdm_oracle_apply the second;
 * pcdm_oracle_iteration is the one followed by the other over all positions.
 */
void pcdm_oracle_steps(const int64_t *col_ptr, const int32_t *row_idx, const double *val, const double *L,
                       double lambda, double beta, int64_t t0, int64_t t1, const int32_t *S,
                       double *x, double *g, double *hbuf, double *xbuf)
{
    for (int64_t t = t0; t < t1; ++t) {
        int64_t i = S[t];
        double grad = 0.0;
        for (int64_t p = col_ptr[i]; p < col_ptr[i + 1]; ++p) grad += val[p] * g[row_idx[p]];
        double x_new;
        if (L[i] > 0.0) {
            double bl = beta * L[i];
            x_new = soft_threshold(x[i] - grad / bl, lambda / bl);
        } else {
            x_new = 0.0;
        }
        xbuf[t] = x_new;
        hbuf[t] = x_new - x[i];
    }
}

/* x_i = xbuf[t], then g += a_i h_t, for t = 0 .. tau-1 in turn. */
void pcdm_oracle_apply(const int64_t *col_ptr, const int32_t *row_idx, const double *val, int64_t tau,
                       const int32_t *S, double *x, double *g, const double *hbuf, const double *xbuf)
{
    for (int64_t t = 0; t < tau; ++t) {
        int64_t i = S[t];
        x[i] = xbuf[t];
        double h = hbuf[t];
        if (h == 0.0) continue;
        for (int64_t p = col_ptr[i]; p < col_ptr[i + 1]; ++p) g[row_idx[p]] += val[p] * h;
    }
}

void pcdm_oracle_iteration(int64_t m, int64_t n, const int64_t *col_ptr, const int32_t *row_idx,
                           const double *val, const double *L, double lambda, double beta,
                           int64_t tau, const int32_t *S, double *x, double *g,
                           double *hbuf, double *xbuf)
{
    (void)m; (void)n;
    pcdm_oracle_steps(col_ptr, row_idx, val, L, lambda, beta, 0, tau, S, x, g, hbuf, xbuf);
    pcdm_oracle_apply(col_ptr, row_idx, val, tau, S, x, g, hbuf, xbuf);
}

/* g = A x - b. */
void pcdm_oracle_residual(int64_t m, int64_t n, const int64_t *col_ptr, const int32_t *row_idx,
                          const double *val, const double *b, const double *x, double *g)
{
    for (int64_t r = 0; r < m; ++r) g[r] = -b[r];
    for (int64_t i = 0; i < n; ++i) {
        if (x[i] == 0.0) continue;
        for (int64_t p = col_ptr[i]; p < col_ptr[i + 1]; ++p) g[row_idx[p]] += val[p] * x[i];
    }
}

/* F(x) = 1/2 ||Ax - b||^2 + lambda ||x||_1, computed from scratch. */
double pcdm_oracle_objective(int64_t m, int64_t n, const int64_t *col_ptr, const int32_t *row_idx,
                             const double *val, const double *b, const double *x, double lambda)
{
    double *r = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    if (!r) return NAN;
    pcdm_oracle_residual(m, n, col_ptr, row_idx, val, b, x, r);
    double rr = 0.0, l1 = 0.0;
    for (int64_t q = 0; q < m; ++q) rr += r[q] * r[q];
    for (int64_t i = 0; i < n; ++i) l1 += fabs(x[i]);
    free(r);
    return 0.5 * rr + lambda * l1;
}

/*
 * Duality gap of LASSO at x, with r = A x - b supplied by the caller.
 *   c = A^T r,  s = min(1, lambda/||c||_inf)  (s = 1 when c = 0),  theta = s r
 *   P = 1/2 ||r||^2 + lambda ||x||_1
 *   D = -1/2 ||theta||^2 - b^T theta           (dual of LASSO, feasible: ||A^T theta||_inf <= lambda)
 *   gap = 1/2 (1-s)^2 ||r||^2 + sum_i (lambda |x_i| + s x_i c_i)
 * The last line equals P - D when r = A x - b exactly (b^T r = x^T c - ||r||^2) and
 * every summand is >= 0, so it is free of cancellation.
 * out = {P, D, gap, ||c||_inf, s, ||r||^2, b^T r, ||x||_1, x^T c}
 */
void pcdm_oracle_gap(int64_t m, int64_t n, const int64_t *col_ptr, const int32_t *row_idx,
                     const double *val, const double *b, const double *x, const double *r,
                     double lambda, double *out)
{
    double *c = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!c) {
        for (int q = 0; q < 9; ++q) out[q] = NAN;
        return;
    }
    double cinf = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t p = col_ptr[i]; p < col_ptr[i + 1]; ++p) s += val[p] * r[row_idx[p]];
        c[i] = s;
        if (fabs(s) > cinf) cinf = fabs(s);
    }
    double s = 1.0;
    if (cinf > 0.0 && lambda / cinf < 1.0) s = lambda / cinf;
    double rr = 0.0, br = 0.0;
    for (int64_t q = 0; q < m; ++q) {
        rr += r[q] * r[q];
        br += b[q] * r[q];
    }
    double l1 = 0.0, xc = 0.0, terms = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        l1 += fabs(x[i]);
        xc += x[i] * c[i];
        terms += lambda * fabs(x[i]) + s * x[i] * c[i];
    }
    free(c);
    out[0] = 0.5 * rr + lambda * l1;
    out[1] = -0.5 * s * s * rr - s * br;
    out[2] = 0.5 * (1.0 - s) * (1.0 - s) * rr + terms;
    out[3] = cinf;
    out[4] = s;
    out[5] = rr;
    out[6] = br;
    out[7] = l1;
    out[8] = xc;
}

/*
 * Iterations k0 .. k0+iters-1 of Algorithm 1 from the state (x, g), with
 * S_k drawn by pcdm_oracle_sample(seed, k, n, tau).  After iteration k, when
 * refresh_every > 0 and (k+1) % refresh_every == 0, g is recomputed as A x - b.
 * Returns 0, or -1 on allocation failure or bad sizes.
 */
int pcdm_oracle_run(int64_t m, int64_t n, const int64_t *col_ptr, const int32_t *row_idx,
                    const double *val, const double *b, const double *L, double lambda,
                    double beta, int64_t tau, uint64_t seed, int64_t k0, int64_t iters,
                    int64_t refresh_every, double *x, double *g)
{
    if (tau < 1 || tau > n) return -1;
    int32_t *S = (int32_t *)malloc((size_t)tau * sizeof(int32_t));
    double *hbuf = (double *)malloc((size_t)tau * sizeof(double));
    double *xbuf = (double *)malloc((size_t)tau * sizeof(double));
    if (!S || !hbuf || !xbuf) {
        free(S); free(hbuf); free(xbuf);
        return -1;
    }
    int rc = 0;
    for (int64_t it = 0; it < iters; ++it) {
        int64_t k = k0 + it;
        if (pcdm_oracle_sample(seed, k, n, tau, S) != 0) { rc = -1; break; }
        pcdm_oracle_iteration(m, n, col_ptr, row_idx, val, L, lambda, beta, tau, S, x, g, hbuf, xbuf);
        if (refresh_every > 0 && (k + 1) % refresh_every == 0)
            pcdm_oracle_residual(m, n, col_ptr, row_idx, val, b, x, g);
    }
    free(S); free(hbuf); free(xbuf);
    return rc;
}


/* ---------------------------------------------------------------------- */
/* Other doubly uniform samplings (Sec. 4.1 items 4 and 5) and their beta  */
/* (Theorem ESO-DU).  Sampling kinds: 0 tau-nice, 1 tau-independent,      */
/* 2 (tau, p_b)-binomial.                                                  */
/* Spec (shared in words only):                                            */
/*   independent: W_j = w0 | w1 << 32 of Philox4x32-10(counter = (j, 1,    */
/*     lo32(k), hi32(k)), key = (lo32(seed), hi32(seed))); pick_j =        */
/*     floor(W_j * n / 2^64); position j is active iff no position j' < j  */
/*     picked the same block.                                              */
/*   binomial: positions j < tau of the tau-nice S_k; position j is kept   */
/*     iff word 0 of Philox4x32-10(counter = (j, 2, lo32(k), hi32(k)),     */
/*     same key) is below T = min(2^32, floor(p_b * 2^32)).                */
/* ---------------------------------------------------------------------- */
static void philox_block(uint64_t seed, uint32_t c0, uint32_t c1, uint64_t k, uint32_t out[4])
{
    const uint32_t ctr[4] = {c0, c1, (uint32_t)k, (uint32_t)(k >> 32)};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    pcdm_oracle_philox4x32_10(ctr, key, out);
}

int pcdm_oracle_sample_independent(uint64_t seed, int64_t k, int64_t n, int64_t tau, int32_t *S,
                                   uint8_t *active)
{
    if (n < 1 || n > 2147483647LL || tau < 0 || k < 0) return -1;
    uint8_t *seen = (uint8_t *)calloc((size_t)n, 1);
    if (!seen) return -1;
    for (int64_t j = 0; j < tau; ++j) {
        uint32_t w[4];
        philox_block(seed, (uint32_t)j, 1u, (uint64_t)k, w);
        const uint64_t W = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
        const int64_t pick = (int64_t)(((unsigned __int128)W * (unsigned __int128)(uint64_t)n) >> 64);
        S[j] = (int32_t)pick;
        active[j] = seen[pick] ? 0 : 1;
        seen[pick] = 1;
    }
    free(seen);
    return 0;
}

static uint64_t keep_threshold(double p_b)
{
    if (p_b >= 1.0) return (uint64_t)1 << 32;
    if (p_b <= 0.0) return 0;
    return (uint64_t)floor(p_b * 4294967296.0);
}

void pcdm_oracle_binomial_keep(uint64_t seed, int64_t k, int64_t tau, double p_b, uint8_t *active)
{
    const uint64_t T = keep_threshold(p_b);
    for (int64_t j = 0; j < tau; ++j) {
        uint32_t w[4];
        philox_block(seed, (uint32_t)j, 2u, (uint64_t)k, w);
        active[j] = (uint64_t)w[0] < T ? 1 : 0;
    }
}

/* q_k = C(n, k) c_k, c_1 = (1/n)^tau, c_k = (k/n)^tau - sum_{i<k} C(k, i) c_i
 * (Sec. 4.1 item 4), k = 1 .. tau, written to q[k]; q[0] = 0.  Small n and tau only. */
void pcdm_oracle_q_independent(int64_t n, int64_t tau, double *q)
{
    double *c = (double *)calloc((size_t)(tau + 1), sizeof(double));
    q[0] = 0.0;
    for (int64_t kk = 1; kk <= tau; ++kk) {
        double ck = pow((double)kk / (double)n, (double)tau);
        double binom = 1.0;                       /* C(kk, i), built up over i */
        for (int64_t i = 1; i < kk; ++i) {
            binom = binom * (double)(kk - i + 1) / (double)i;
            ck -= binom * c[i];
        }
        c[kk] = ck;
        double cnk = 1.0;                         /* C(n, kk) */
        for (int64_t i = 1; i <= kk; ++i) cnk = cnk * (double)(n - kk + i) / (double)i;
        q[kk] = cnk * ck;
    }
    free(c);
}

/* E|S| and E|S|^2.  nice: tau, tau^2.  independent: with a = (1 - 1/n)^tau and
 * b2 = (1 - 2/n)^tau, E|S| = n (1 - a), E|S|^2 = E|S| + n (n-1) (1 - 2a + b2)
 * (inclusion of one block, of two blocks).  binomial: tau p_b and
 * tau p_b (1 + tau p_b - p_b) as printed with its definition. */
void pcdm_oracle_moments(int kind, int64_t n, int64_t tau, double p_b, double *e1, double *e2)
{
    const double t = (double)tau, nn = (double)n;
    if (kind == 1) {
        const double a = exp(t * log1p(-1.0 / nn));
        const double b2 = n > 1 ? exp(t * log1p(-2.0 / nn)) : 0.0;
        *e1 = nn * (1.0 - a);
        *e2 = *e1 + nn * (nn - 1.0) * (1.0 - 2.0 * a + b2);
    } else if (kind == 2) {
        *e1 = t * p_b;
        *e2 = t * p_b * (1.0 + t * p_b - p_b);
    } else {
        *e1 = t;
        *e2 = t * t;
    }
}

/* beta = 1 + (omega - 1)(E|S|^2 / E|S| - 1) / max(1, n - 1)  (Theorem ESO-DU). */
double pcdm_oracle_beta_du(int64_t omega, double e1, double e2, int64_t n)
{
    const double om = (double)(omega < 1 ? 1 : omega);
    const double denom = (double)(n - 1 > 1 ? n - 1 : 1);
    if (!(e1 > 0.0)) return 1.0;
    return 1.0 + (om - 1.0) * (e2 / e1 - 1.0) / denom;
}

/* Iterations of Algorithm 1 with the sampling `kind`: the positions of the
 * drawn list that are active form S_k (inactive ones are idle); the step and
 * update are those of pcdm_oracle_iteration, applied to the active positions
 * in list order. */
int pcdm_oracle_run_sampling(int64_t m, int64_t n, const int64_t *col_ptr, const int32_t *row_idx,
                             const double *val, const double *b, const double *L, double lambda,
                             double beta, int kind, double p_b, int64_t tau, uint64_t seed, int64_t k0,
                             int64_t iters, int64_t refresh_every, double *x, double *g)
{
    if (tau < 1 || tau > n || kind < 0 || kind > 2) return -1;
    int32_t *S = (int32_t *)malloc((size_t)tau * sizeof(int32_t));
    int32_t *Sa = (int32_t *)malloc((size_t)tau * sizeof(int32_t));
    uint8_t *act = (uint8_t *)malloc((size_t)tau);
    double *hbuf = (double *)malloc((size_t)tau * sizeof(double));
    double *xbuf = (double *)malloc((size_t)tau * sizeof(double));
    int rc = 0;
    if (!S || !Sa || !act || !hbuf || !xbuf) rc = -1;
    for (int64_t it = 0; rc == 0 && it < iters; ++it) {
        const int64_t k = k0 + it;
        if (kind == 1) {
            if (pcdm_oracle_sample_independent(seed, k, n, tau, S, act) != 0) { rc = -1; break; }
        } else {
            if (pcdm_oracle_sample(seed, k, n, tau, S) != 0) { rc = -1; break; }
            if (kind == 2)
                pcdm_oracle_binomial_keep(seed, k, tau, p_b, act);
            else
                for (int64_t j = 0; j < tau; ++j) act[j] = 1;
        }
        int64_t na = 0;
        for (int64_t j = 0; j < tau; ++j)
            if (act[j]) Sa[na++] = S[j];
        pcdm_oracle_iteration(m, n, col_ptr, row_idx, val, L, lambda, beta, na, Sa, x, g, hbuf, xbuf);
        if (refresh_every > 0 && (k + 1) % refresh_every == 0)
            pcdm_oracle_residual(m, n, col_ptr, row_idx, val, b, x, g);
    }
    free(S); free(Sa); free(act); free(hbuf); free(xbuf);
    return rc;
}
