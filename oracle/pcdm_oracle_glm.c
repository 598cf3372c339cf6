/*
 * Plain FP64 oracle for PCDM1 on the two other objectives the paper runs:
 * the dual of the L2-regularised hinge-loss SVM (Sec. 8.3) and L2-regularised
 * logistic regression (Sec. 8.4), both with blocks of size 1.
 *
 * TEST INFRASTRUCTURE ONLY, like pcdm_oracle.c: nothing in the product path
 * calls this file.  It shares no code with the CUDA library and meets it only
 * through the seeded instance generator and the written sampler spec (the
 * tau-nice sample comes from pcdm_oracle_sample of the same oracle library).
 * Single-threaded IEEE double, steps in the paper's order, built with
 * -ffp-contract=off.
 *
 * problem = 1, SVM dual (Sec. 8.3).  Data: A in R^{d x n}, column i the
 * example A_i; labels y in {-1,+1}^n; lambda > 0.
 *   f(x)   = 1/(2 lambda n^2) x^T Z x - (1/n) sum_i x_i,  Z_ij = y_i y_j <A_i, A_j>
 *   Psi(x) = 0 on the box [0,1]^n, +infinity outside
 * The oracle keeps u = sum_i y_i x_i A_i (a d-vector), so x^T Z x = ||u||^2 and
 *   grad_i f = y_i <A_i, u> / (lambda n^2) - 1/n,   L_i = ||A_i||^2 / (lambda n^2).
 * f is a sum over features r of terms in u_r (each touching the examples that
 * have feature r) plus a separable part, so omega = the largest number of
 * examples sharing a feature (row counts of A), as the paper states for rcv1.
 * Step (eq. (h(x)) with this Psi): h_i = clip(x_i - grad_i/(beta L_i), 0, 1) - x_i.
 * An all-zero example (L_i = 0) leaves f = -x_i/n along x_i: x_i goes to 1.
 * Primal point w = u/(lambda n) and hinge-loss primal
 *   P(w) = (1/n) sum_i max(0, 1 - y_i <w, A_i>) + (lambda/2) ||w||^2;
 * dual value D(x) = -f(x); gap = P(w(x)) - D(x).
 *
 * problem = 2, logistic regression (Sec. 8.4).  Data: A in R^{m x n}, row j the
 * example A_j; labels y in {-1,+1}^m; lambda > 0.
 *   f(x) = sum_j log(1 + exp(-y_j A_j^T x)),   Psi(x) = lambda ||x||^2 = sum_i lambda x_i^2
 * The oracle keeps z = A x, so
 *   grad_i f = -sum_j y_j a_ji / (1 + exp(y_j z_j)),   L_i = ||a_i||^2 / 4
 * (the second derivative of t -> log(1 + exp(-t)) is at most 1/4), and
 *   h_i = argmin_t grad_i t + (beta L_i / 2) t^2 + lambda (x_i + t)^2
 *       = -(grad_i + 2 lambda x_i) / (beta L_i + 2 lambda).
 * Fenchel dual at alpha_j = 1/(1 + exp(y_j z_j)) in (0, 1):
 *   D(alpha) = -sum_j [alpha_j log alpha_j + (1 - alpha_j) log(1 - alpha_j)]
 *              - ||sum_j alpha_j y_j A_j||^2 / (4 lambda);
 * gap = F(x) - D(alpha(x)).
 *
 * Functions:
 *   pcdm_oracle_glm_lipschitz   L_i of the problem (above)
 *   pcdm_oracle_glm_residual    u (SVM) or z (logistic) from x
 *   pcdm_oracle_glm_gradient    grad f (all n coordinates) from the kept vector
 *   pcdm_oracle_glm_objective   F = f + Psi at x (from scratch; +inf outside the SVM box)
 *   pcdm_oracle_glm_gap         {P, D, gap} at x (from scratch)
 *   pcdm_oracle_glm_iteration   Algorithm 1, step 4, Jacobi, on the set S
 *   pcdm_oracle_glm_run         iterations k0 .. k0+iters-1 with the tau-nice sampling
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

int pcdm_oracle_sample(uint64_t seed, int64_t k, int64_t n, int64_t tau, int32_t *S);

enum { GLM_SVM_DUAL = 1, GLM_LOGISTIC = 2 };

/* log(1 + exp(t)) without overflow. */
static double softplus(double t)
{
    if (t > 0.0) return t + log1p(exp(-t));
    return log1p(exp(t));
}

void pcdm_oracle_glm_lipschitz(int problem, int64_t n, const int64_t *col_ptr, const double *val, double lambda,
                               double *L)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t p = col_ptr[i]; p < col_ptr[i + 1]; ++p) s += val[p] * val[p];
        if (problem == GLM_SVM_DUAL)
            L[i] = s / (lambda * (double)n * (double)n);
        else
            L[i] = s / 4.0;
    }
}

/* SVM: v = u = sum_i y_i x_i A_i (d = m entries).  Logistic: v = z = A x. */
void pcdm_oracle_glm_residual(int problem, int64_t m, int64_t n, const int64_t *col_ptr, const int32_t *row_idx,
                              const double *val, const double *y, const double *x, double *v)
{
    for (int64_t r = 0; r < m; ++r) v[r] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (x[i] == 0.0) continue;
        const double c = problem == GLM_SVM_DUAL ? y[i] * x[i] : x[i];
        for (int64_t p = col_ptr[i]; p < col_ptr[i + 1]; ++p) v[row_idx[p]] += val[p] * c;
    }
}

/* grad_i f for one coordinate from the kept vector v. */
static double coord_grad(int problem, int64_t n, const int64_t *col_ptr, const int32_t *row_idx, const double *val,
                         const double *y, const double *v, double lambda, int64_t i)
{
    double s = 0.0;
    if (problem == GLM_SVM_DUAL) {
        for (int64_t p = col_ptr[i]; p < col_ptr[i + 1]; ++p) s += val[p] * v[row_idx[p]];
        return y[i] * s / (lambda * (double)n * (double)n) - 1.0 / (double)n;
    }
    for (int64_t p = col_ptr[i]; p < col_ptr[i + 1]; ++p) {
        const int32_t j = row_idx[p];
        s += -y[j] * val[p] / (1.0 + exp(y[j] * v[j]));
    }
    return s;
}

void pcdm_oracle_glm_gradient(int problem, int64_t m, int64_t n, const int64_t *col_ptr, const int32_t *row_idx,
                              const double *val, const double *y, const double *v, double lambda, double *grad)
{
    (void)m;
    for (int64_t i = 0; i < n; ++i) grad[i] = coord_grad(problem, n, col_ptr, row_idx, val, y, v, lambda, i);
}

double pcdm_oracle_glm_objective(int problem, int64_t m, int64_t n, const int64_t *col_ptr, const int32_t *row_idx,
                                 const double *val, const double *y, const double *x, double lambda)
{
    double *v = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    if (!v) return NAN;
    pcdm_oracle_glm_residual(problem, m, n, col_ptr, row_idx, val, y, x, v);
    double F;
    if (problem == GLM_SVM_DUAL) {
        double uu = 0.0, sx = 0.0;
        int inside = 1;
        for (int64_t r = 0; r < m; ++r) uu += v[r] * v[r];
        for (int64_t i = 0; i < n; ++i) {
            sx += x[i];
            if (!(x[i] >= 0.0 && x[i] <= 1.0)) inside = 0;
        }
        F = inside ? uu / (2.0 * lambda * (double)n * (double)n) - sx / (double)n : INFINITY;
    } else {
        double loss = 0.0, xx = 0.0;
        for (int64_t j = 0; j < m; ++j) loss += softplus(-y[j] * v[j]);
        for (int64_t i = 0; i < n; ++i) xx += x[i] * x[i];
        F = loss + lambda * xx;
    }
    free(v);
    return F;
}

/* out = {P, D, gap}. */
void pcdm_oracle_glm_gap(int problem, int64_t m, int64_t n, const int64_t *col_ptr, const int32_t *row_idx,
                         const double *val, const double *y, const double *x, double lambda, double *out)
{
    double *v = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    double *w = (double *)malloc((size_t)((m > n ? m : n) > 0 ? (m > n ? m : n) : 1) * sizeof(double));
    if (!v || !w) {
        free(v);
        free(w);
        out[0] = out[1] = out[2] = NAN;
        return;
    }
    pcdm_oracle_glm_residual(problem, m, n, col_ptr, row_idx, val, y, x, v);
    if (problem == GLM_SVM_DUAL) {
        const double nn = (double)n;
        for (int64_t r = 0; r < m; ++r) w[r] = v[r] / (lambda * nn);
        double hinge = 0.0, ww = 0.0, uu = 0.0, sx = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double wa = 0.0;
            for (int64_t p = col_ptr[i]; p < col_ptr[i + 1]; ++p) wa += w[row_idx[p]] * val[p];
            const double margin = 1.0 - y[i] * wa;
            hinge += margin > 0.0 ? margin : 0.0;
            sx += x[i];
        }
        for (int64_t r = 0; r < m; ++r) {
            ww += w[r] * w[r];
            uu += v[r] * v[r];
        }
        out[0] = hinge / nn + 0.5 * lambda * ww;
        out[1] = sx / nn - uu / (2.0 * lambda * nn * nn);
    } else {
        double loss = 0.0, xx = 0.0, ent = 0.0;
        for (int64_t i = 0; i < n; ++i) w[i] = 0.0;
        for (int64_t j = 0; j < m; ++j) {
            const double t = y[j] * v[j];
            loss += softplus(-t);
            /* alpha = 1/(1+e^t): log alpha = -softplus(t), log(1-alpha) = -softplus(-t) */
            const double alpha = 1.0 / (1.0 + exp(t));
            ent += -alpha * softplus(t) - (1.0 - alpha) * softplus(-t);
        }
        for (int64_t i = 0; i < n; ++i) {
            double s = 0.0;   /* (sum_j alpha_j y_j A_j)_i */
            for (int64_t p = col_ptr[i]; p < col_ptr[i + 1]; ++p) {
                const int32_t j = row_idx[p];
                s += y[j] * val[p] / (1.0 + exp(y[j] * v[j]));
            }
            w[i] = s;
            xx += x[i] * x[i];
        }
        double ss = 0.0;
        for (int64_t i = 0; i < n; ++i) ss += w[i] * w[i];
        out[0] = loss + lambda * xx;
        out[1] = -ent - ss / (4.0 * lambda);
    }
    out[2] = out[0] - out[1];
    free(v);
    free(w);
}

/*
 * One Jacobi iteration on S: every step from the same x_k and the same kept
 * vector v, then x and v move.  SVM: u += y_i h_i A_i.  Logistic: z += h_i a_i.
 */
void pcdm_oracle_glm_iteration(int problem, int64_t m, int64_t n, const int64_t *col_ptr, const int32_t *row_idx,
                               const double *val, const double *y, const double *L, double lambda, double beta,
                               int64_t tau, const int32_t *S, double *x, double *v, double *hbuf, double *xbuf)
{
    (void)m;
    for (int64_t t = 0; t < tau; ++t) {
        const int64_t i = S[t];
        const double grad = coord_grad(problem, n, col_ptr, row_idx, val, y, v, lambda, i);
        double x_new;
        if (problem == GLM_SVM_DUAL) {
            if (L[i] > 0.0) {
                x_new = x[i] - grad / (beta * L[i]);
                if (x_new < 0.0) x_new = 0.0;
                if (x_new > 1.0) x_new = 1.0;
            } else {
                x_new = 1.0;
            }
        } else {
            x_new = x[i] - (grad + 2.0 * lambda * x[i]) / (beta * L[i] + 2.0 * lambda);
        }
        xbuf[t] = x_new;
        hbuf[t] = x_new - x[i];
    }
    for (int64_t t = 0; t < tau; ++t) {
        const int64_t i = S[t];
        x[i] = xbuf[t];
        const double h = hbuf[t];
        if (h == 0.0) continue;
        const double c = problem == GLM_SVM_DUAL ? y[i] * h : h;
        for (int64_t p = col_ptr[i]; p < col_ptr[i + 1]; ++p) v[row_idx[p]] += val[p] * c;
    }
}

/* Iterations k0 .. k0+iters-1 (tau-nice S_k from pcdm_oracle_sample), v recomputed
 * from x after iteration k when refresh_every > 0 and (k+1) % refresh_every == 0. */
int pcdm_oracle_glm_run(int problem, int64_t m, int64_t n, const int64_t *col_ptr, const int32_t *row_idx,
                        const double *val, const double *y, const double *L, double lambda, double beta, int64_t tau,
                        uint64_t seed, int64_t k0, int64_t iters, int64_t refresh_every, double *x, double *v)
{
    if (tau < 1 || tau > n) return -1;
    int32_t *S = (int32_t *)malloc((size_t)tau * sizeof(int32_t));
    double *hb = (double *)malloc((size_t)tau * sizeof(double));
    double *xb = (double *)malloc((size_t)tau * sizeof(double));
    int rc = 0;
    if (!S || !hb || !xb) rc = -1;
    for (int64_t k = k0; rc == 0 && k < k0 + iters; ++k) {
        if (pcdm_oracle_sample(seed, k, n, tau, S) != 0) {
            rc = -1;
            break;
        }
        pcdm_oracle_glm_iteration(problem, m, n, col_ptr, row_idx, val, y, L, lambda, beta, tau, S, x, v, hb, xb);
        if (refresh_every > 0 && (k + 1) % refresh_every == 0)
            pcdm_oracle_glm_residual(problem, m, n, col_ptr, row_idx, val, y, x, v);
    }
    free(S);
    free(hb);
    free(xb);
    return rc;
}
