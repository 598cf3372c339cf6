/*
 * Threaded timing mode of the FP64 oracle (TEST INFRASTRUCTURE: only the tests
 * and the benchmark's CPU-baseline legs load it; nothing in the product path).
 *
 * pcdm_oracle_run_threads runs the same iterations as pcdm_oracle_run
 * (Algorithm 1 with the tau-nice sampling, Jacobi, the residual refreshed every
 * refresh_every iterations) on T host threads:
 *   1. every thread draws its share of the positions of S_k
 *      (pcdm_oracle_sample_range);
 *   2. every thread computes x_new and h for its share (pcdm_oracle_steps),
 *      reading only x_k and g_k;
 *   3. one thread applies the iteration (pcdm_oracle_apply: x_i = x_new, then
 *      g += a_i h in position order) and refreshes g when due.
 * The per-position arithmetic and the order of every update to g are those of
 * the single-threaded run, so the result equals it bit for bit; the
 * single-threaded run stays the parity reference and this mode is its timed
 * multicore form.  POSIX threads and barriers only.
 */
#define _POSIX_C_SOURCE 200809L
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

int pcdm_oracle_sample_range(uint64_t seed, int64_t k, int64_t n, int64_t j0, int64_t j1, int32_t *S);
void pcdm_oracle_steps(const int64_t *col_ptr, const int32_t *row_idx, const double *val, const double *L,
                       double lambda, double beta, int64_t t0, int64_t t1, const int32_t *S,
                       double *x, double *g, double *hbuf, double *xbuf);
void pcdm_oracle_apply(const int64_t *col_ptr, const int32_t *row_idx, const double *val, int64_t tau,
                       const int32_t *S, double *x, double *g, const double *hbuf, const double *xbuf);
void pcdm_oracle_residual(int64_t m, int64_t n, const int64_t *col_ptr, const int32_t *row_idx,
                          const double *val, const double *b, const double *x, double *g);

struct mt_shared {
    int64_t m, n;
    const int64_t *col_ptr;
    const int32_t *row_idx;
    const double *val, *b, *L;
    double lambda, beta;
    int64_t tau;
    uint64_t seed;
    int64_t k0, iters, refresh_every;
    double *x, *g;
    int32_t *S;
    double *hbuf, *xbuf;
    int threads;
    pthread_barrier_t bar;
    int failed;
    /* start gate: workers wait until every thread exists (or a start failed) */
    pthread_mutex_t gate_mu;
    pthread_cond_t gate_cv;
    int gate_open, start_failed;
};

struct mt_worker {
    struct mt_shared *sh;
    int id;
};

static void *mt_run(void *arg)
{
    struct mt_worker *w = (struct mt_worker *)arg;
    struct mt_shared *c = w->sh;
    pthread_mutex_lock(&c->gate_mu);
    while (!c->gate_open) pthread_cond_wait(&c->gate_cv, &c->gate_mu);
    const int skip = c->start_failed;
    pthread_mutex_unlock(&c->gate_mu);
    if (skip) return NULL;
    const int64_t t0 = c->tau * w->id / c->threads, t1 = c->tau * (w->id + 1) / c->threads;
    for (int64_t it = 0; it < c->iters; ++it) {
        const int64_t k = c->k0 + it;
        if (pcdm_oracle_sample_range(c->seed, k, c->n, t0, t1, c->S) != 0) c->failed = 1;
        pthread_barrier_wait(&c->bar);
        if (c->failed) break;
        pcdm_oracle_steps(c->col_ptr, c->row_idx, c->val, c->L, c->lambda, c->beta, t0, t1, c->S, c->x, c->g,
                          c->hbuf, c->xbuf);
        pthread_barrier_wait(&c->bar);
        if (w->id == 0) {
            pcdm_oracle_apply(c->col_ptr, c->row_idx, c->val, c->tau, c->S, c->x, c->g, c->hbuf, c->xbuf);
            if (c->refresh_every > 0 && (k + 1) % c->refresh_every == 0)
                pcdm_oracle_residual(c->m, c->n, c->col_ptr, c->row_idx, c->val, c->b, c->x, c->g);
        }
        pthread_barrier_wait(&c->bar);
    }
    return NULL;
}

/* The arguments of pcdm_oracle_run plus the thread count (>= 1).  Returns 0, or
 * -1 on bad sizes or a failed allocation or thread start. */
int pcdm_oracle_run_threads(int64_t m, int64_t n, const int64_t *col_ptr, const int32_t *row_idx,
                            const double *val, const double *b, const double *L, double lambda,
                            double beta, int64_t tau, uint64_t seed, int64_t k0, int64_t iters,
                            int64_t refresh_every, double *x, double *g, int threads)
{
    if (tau < 1 || tau > n || threads < 1 || iters < 0) return -1;
    if (threads > tau) threads = (int)tau;
    struct mt_shared c;
    c.m = m; c.n = n; c.col_ptr = col_ptr; c.row_idx = row_idx; c.val = val; c.b = b; c.L = L;
    c.lambda = lambda; c.beta = beta; c.tau = tau; c.seed = seed; c.k0 = k0; c.iters = iters;
    c.refresh_every = refresh_every; c.x = x; c.g = g; c.threads = threads; c.failed = 0;
    c.gate_open = 0; c.start_failed = 0;
    c.S = (int32_t *)malloc((size_t)tau * sizeof(int32_t));
    c.hbuf = (double *)malloc((size_t)tau * sizeof(double));
    c.xbuf = (double *)malloc((size_t)tau * sizeof(double));
    struct mt_worker *w = (struct mt_worker *)malloc((size_t)threads * sizeof(struct mt_worker));
    pthread_t *tid = (pthread_t *)malloc((size_t)threads * sizeof(pthread_t));
    int rc = 0;
    if (!c.S || !c.hbuf || !c.xbuf || !w || !tid || pthread_barrier_init(&c.bar, NULL, (unsigned)threads) != 0) {
        free(c.S); free(c.hbuf); free(c.xbuf); free(w); free(tid);
        return -1;
    }
    pthread_mutex_init(&c.gate_mu, NULL);
    pthread_cond_init(&c.gate_cv, NULL);
    int started = 1;
    for (int q = 0; q < threads; ++q) {
        w[q].sh = &c;
        w[q].id = q;
    }
    for (int q = 1; q < threads; ++q) {
        if (pthread_create(&tid[q], NULL, mt_run, &w[q]) != 0) break;
        started += 1;
    }
    /* open the gate: with every thread started all of them run (the main thread
       as worker 0); otherwise the started ones leave without touching the barrier */
    pthread_mutex_lock(&c.gate_mu);
    c.start_failed = started != threads;
    c.gate_open = 1;
    pthread_cond_broadcast(&c.gate_cv);
    pthread_mutex_unlock(&c.gate_mu);
    if (started == threads) {
        mt_run(&w[0]);
        if (c.failed) rc = -1;
    } else {
        rc = -1;
    }
    for (int q = 1; q < started; ++q) pthread_join(tid[q], NULL);
    pthread_barrier_destroy(&c.bar);
    pthread_cond_destroy(&c.gate_cv);
    pthread_mutex_destroy(&c.gate_mu);
    free(c.S); free(c.hbuf); free(c.xbuf); free(w); free(tid);
    return rc;
}
