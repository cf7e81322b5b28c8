/*
 * Relay-BP oracle: a plain, slow, step-by-step CPU implementation of Relay
 * decoding, used as TEST INFRASTRUCTURE ONLY.  Only tests, the package smoke
 * check and the CPU-baseline leg of the benchmark may load it; the decoder
 * library never does, and this file shares no code with it.
 *
 * What it computes (paper Sec. 2.3, "Relay decoding"):
 *   initialisation     nu_{j->i}(0) = lambda_j(0) = Lambda_j(0) = w_j = log((1-p_j)/p_j)
 *   memory update      lambda_j(t) = (1-gamma_j) lambda_j(0) + gamma_j Lambda_j(t-1)
 *   check -> fault     mu_{i->j}(t) = (-1)^{sigma_i} prod_{j' in N(i)\j} sign(nu_{j'->i}(t-1))
 *                                      * min_{j' in N(i)\j} |nu_{j'->i}(t-1)|
 *   fault -> check     nu_{j->i}(t) = lambda_j(t) + sum_{i' in N(j)\i} mu_{i'->j}(t)
 *   marginal           Lambda_j(t) = lambda_j(t) + sum_{i' in N(j)} mu_{i'->j}(t)
 *   decision           F_j(t) = 1 iff Lambda_j(t) < 0
 *   convergence        H F(t) = sigma
 *   relay chaining     leg r >= 2 starts from Lambda^{(r)}(0) = Lambda^{(r-1)}(T_{r-1}),
 *                      lambda^{(r)}(0) = Lambda^{(r)}(0), nu^{(r)}(0) = lambda^{(r)}(0)
 *   stopping           a leg ends at its first valid correction or after T_r
 *                      iterations; decoding stops after S solutions or after the
 *                      last leg, keeping the lowest-weight solution.
 * Parameters of App. A.3: T_1 = 80, T_r = 60, R = 300 legs after the first,
 * gamma_0 = 0.125 on the first leg, later gammas drawn uniformly (the draws are
 * an input table here).
 *
 * Readings where the paper is silent (each is also listed in the design notes):
 *   - sign(x) = -1 iff x < 0, so sign(0) = +1; F_j = 1 iff Lambda_j < 0.
 *   - every message and marginal is clamped to [-clip, clip] after it is
 *     computed, and the minimum over an empty set is clip.
 *   - the weight of a solution is W = sum_j F_j w_j, compared exactly: the sum
 *     is accumulated in double, which is exact for float32 w_j of magnitude
 *     >= 2^-10 (and for w_j = 0) over up to 2^13 faults.  A new solution
 *     replaces the kept one only if its weight is strictly lower.
 *   - convergence is tested after every iteration t >= 1; the iteration budget
 *     (max_total_iters > 0) is tested after the convergence test.
 *   - warm_mode 0 is the paper's chaining above; warm_mode 1 keeps
 *     lambda^{(r)}(0) = w and nu^{(r)}(0) = w while Lambda^{(r)}(0) still
 *     takes the previous leg's terminal marginals.
 *
 * Precision: REAL is double by default.  Built with -DREAL=float it is the
 * single-precision mirror (same operations, same order), and with
 * -DMSG_FP16 every fault->check message is also rounded to binary16 when
 * stored.  All builds use -ffp-contract=off, so every + and * rounds once.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef REAL
#define REAL double
#endif

#ifdef MSG_FP16
#define STORE_MSG(x) ((REAL)(_Float16)(x))
#else
#define STORE_MSG(x) ((REAL)(x))
#endif

typedef struct {
    int M, N, E;
    const int32_t *row_ptr; /* [M+1], edges of check i are row_ptr[i] .. row_ptr[i+1]-1 */
    const int32_t *col_idx; /* [E], fault of edge e */
    int32_t *var_ptr;       /* [N+1] */
    int32_t *var_edges;     /* [E], edges of fault j in increasing edge (= check) order */
} tanner;

typedef struct {
    REAL *nu, *mu;          /* [E] fault->check and check->fault messages */
    REAL *Lam, *lam0, *lam; /* [N] marginals, memory anchor lambda(0), bias lambda(t) */
    uint8_t *F, *best;      /* [N] current decision, kept solution */
} state;

static REAL clampv(REAL x, REAL c) { return x > c ? c : (x < -c ? -c : x); }

static int tanner_build(tanner *g, int M, int N, const int32_t *row_ptr, const int32_t *col_idx)
{
    g->M = M; g->N = N; g->E = row_ptr[M];
    g->row_ptr = row_ptr; g->col_idx = col_idx;
    g->var_ptr = (int32_t *)calloc((size_t)N + 1, sizeof(int32_t));
    g->var_edges = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->E > 0 ? g->E : 1));
    if (!g->var_ptr || !g->var_edges) return -1;
    for (int e = 0; e < g->E; ++e) {
        if (col_idx[e] < 0 || col_idx[e] >= N) return -1;
        g->var_ptr[col_idx[e] + 1]++;
    }
    for (int j = 0; j < N; ++j) g->var_ptr[j + 1] += g->var_ptr[j];
    int32_t *fill = (int32_t *)calloc((size_t)N, sizeof(int32_t));
    if (!fill) return -1;
    for (int e = 0; e < g->E; ++e) {          /* e increasing => per-fault lists sorted */
        int j = col_idx[e];
        g->var_edges[g->var_ptr[j] + fill[j]++] = e;
    }
    free(fill);
    return 0;
}

static void tanner_free(tanner *g) { free(g->var_ptr); free(g->var_edges); }

static int state_alloc(state *s, int N, int E)
{
    size_t e = (size_t)(E > 0 ? E : 1), n = (size_t)(N > 0 ? N : 1);
    s->nu = (REAL *)malloc(e * sizeof(REAL));
    s->mu = (REAL *)malloc(e * sizeof(REAL));
    s->Lam = (REAL *)malloc(n * sizeof(REAL));
    s->lam0 = (REAL *)malloc(n * sizeof(REAL));
    s->lam = (REAL *)malloc(n * sizeof(REAL));
    s->F = (uint8_t *)calloc(n, 1);
    s->best = (uint8_t *)calloc(n, 1);
    return (s->nu && s->mu && s->Lam && s->lam0 && s->lam && s->F && s->best) ? 0 : -1;
}

static void state_free(state *s)
{
    free(s->nu); free(s->mu); free(s->Lam); free(s->lam0); free(s->lam); free(s->F); free(s->best);
}

/* nu_{j->i}(0) = lambda_j(0) on every edge. */
static void init_messages(const tanner *g, state *s)
{
    for (int e = 0; e < g->E; ++e) s->nu[e] = STORE_MSG(s->lam0[g->col_idx[e]]);
}

/* One DMem-BP iteration: memory update, check->fault, fault->check, marginals, decision. */
static void dmem_iteration(const tanner *g, const uint8_t *sigma, const REAL *gamma, REAL clip,
                           state *s)
{
    /* memory update, Lambda_j(t-1) is the marginal held in s->Lam */
    for (int j = 0; j < g->N; ++j)
        s->lam[j] = (1 - gamma[j]) * s->lam0[j] + gamma[j] * s->Lam[j];

    /* check -> fault, written literally as a loop over the excluded set */
    for (int i = 0; i < g->M; ++i) {
        for (int e = g->row_ptr[i]; e < g->row_ptr[i + 1]; ++e) {
            int negative = sigma[i] ? 1 : 0;
            REAL m = clip;
            for (int e2 = g->row_ptr[i]; e2 < g->row_ptr[i + 1]; ++e2) {
                if (e2 == e) continue;
                REAL v = s->nu[e2];
                if (v < 0) negative ^= 1;
                REAL a = v < 0 ? -v : v;
                if (a < m) m = a;
            }
            s->mu[e] = negative ? -m : m;
        }
    }

    /* fault -> check, marginals and decision */
    for (int j = 0; j < g->N; ++j) {
        int b = g->var_ptr[j], d = g->var_ptr[j + 1] - b;
        REAL L = s->lam[j];
        for (int k = 0; k < d; ++k) L += s->mu[g->var_edges[b + k]];
        s->Lam[j] = clampv(L, clip);
        for (int k = 0; k < d; ++k) {
            REAL v = s->lam[j];
            for (int k2 = 0; k2 < d; ++k2)
                if (k2 != k) v += s->mu[g->var_edges[b + k2]];
            s->nu[g->var_edges[b + k]] = STORE_MSG(clampv(v, clip));
        }
        s->F[j] = s->Lam[j] < 0 ? 1 : 0;
    }
}

/* H F = sigma (mod 2)? */
static int syndrome_ok(const tanner *g, const uint8_t *sigma, const uint8_t *F)
{
    for (int i = 0; i < g->M; ++i) {
        int par = sigma[i] ? 1 : 0;
        for (int e = g->row_ptr[i]; e < g->row_ptr[i + 1]; ++e) par ^= F[g->col_idx[e]];
        if (par) return 0;
    }
    return 1;
}

typedef struct {
    int R, T_first, T_later, S, warm_mode;
    int64_t max_total_iters;
    REAL clip;
} relay_params;

static void relay_one(const tanner *g, const REAL *w, const double *gamma_tab,
                      const relay_params *prm, const uint8_t *sigma, state *s, REAL *gbuf,
                      uint8_t *corr, int32_t *legs_out, uint8_t *conv_out, int64_t *iters_out,
                      double *final_Lam)
{
    const int N = g->N;
    for (int j = 0; j < N; ++j) { s->lam0[j] = w[j]; s->Lam[j] = s->lam0[j]; s->F[j] = 0; }
    init_messages(g, s);

    int leg = 0, sols = 0, have = 0;
    int64_t iters = 0;
    double best_w = 0;
    for (;;) {
        int T = leg == 0 ? prm->T_first : prm->T_later;
        for (int j = 0; j < N; ++j) gbuf[j] = (REAL)gamma_tab[(size_t)leg * N + j];
        for (int t = 1; t <= T; ++t) {
            dmem_iteration(g, sigma, gbuf, prm->clip, s);
            iters++;
            if (syndrome_ok(g, sigma, s->F)) {
                double W = 0;
                for (int j = 0; j < N; ++j) if (s->F[j]) W += (double)w[j];
                if (!have || W < best_w) {
                    memcpy(s->best, s->F, (size_t)N);
                    best_w = W;
                    have = 1;
                }
                sols++;
                break;
            }
            if (prm->max_total_iters > 0 && iters >= prm->max_total_iters) break;
        }
        int budget_spent = prm->max_total_iters > 0 && iters >= prm->max_total_iters;
        if (sols >= prm->S || leg == prm->R || budget_spent) break;
        /* warm start of the next leg */
        leg++;
        for (int j = 0; j < N; ++j) s->lam0[j] = prm->warm_mode == 0 ? s->Lam[j] : w[j];
        init_messages(g, s);
    }
    memcpy(corr, have ? s->best : s->F, (size_t)N);
    if (final_Lam)
        for (int j = 0; j < N; ++j) final_Lam[j] = (double)s->Lam[j];
    *legs_out = leg + 1;
    *conv_out = (uint8_t)have;
    *iters_out = iters;
}

static int priors_to_llr(int N, const double *priors, REAL *w)
{
    for (int j = 0; j < N; ++j) {
        double p = priors[j];
        if (!(p > 0.0 && p < 1.0)) return -1;
        w[j] = (REAL)log((1.0 - p) / p);
    }
    return 0;
}

/*
 * Decode B syndromes (sigma: uint8 [B][M], one byte per check) with Relay.
 * Outputs: corr uint8 [B][N], legs int32 [B] (legs run), conv uint8 [B]
 * (1 iff at least one valid correction was found), iters int64 [B], and when
 * not NULL final_Lam float64 [B][N], the marginals of the last iteration run.
 * gamma: float64 [(R+1)][N] memory strengths, row r used by leg r+1.
 * Returns 0, or -1 on invalid input.
 */
int oracle_relay_decode(int32_t M, int32_t N, const int32_t *row_ptr, const int32_t *col_idx,
                        const double *priors, const double *gamma, int32_t R, int32_t T_first,
                        int32_t T_later, int64_t max_total_iters, int32_t S, int32_t warm_mode,
                        double clip, const uint8_t *sigma, int64_t B, uint8_t *corr,
                        int32_t *legs, uint8_t *conv, int64_t *iters, double *final_Lam,
                        int32_t nthreads)
{
    if (M < 0 || N < 0 || B < 0 || R < 0 || T_first < 1 || T_later < 1 || S < 1 || !(clip > 0))
        return -1;
    tanner g;
    if (tanner_build(&g, M, N, row_ptr, col_idx)) { tanner_free(&g); return -1; }
    REAL *w = (REAL *)malloc(sizeof(REAL) * (size_t)(N > 0 ? N : 1));
    if (!w || priors_to_llr(N, priors, w)) { free(w); tanner_free(&g); return -1; }
    relay_params prm = {R, T_first, T_later, S, warm_mode, max_total_iters, (REAL)clip};
    int err = 0;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        state s;
        REAL *gbuf = (REAL *)malloc(sizeof(REAL) * (size_t)(N > 0 ? N : 1));
        int ok = state_alloc(&s, N, g.E) == 0 && gbuf;
        if (!ok) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t b = 0; b < B; ++b) {
            if (!ok) continue;
            relay_one(&g, w, gamma, &prm, sigma + (size_t)b * M, &s, gbuf,
                      corr + (size_t)b * N, legs + b, conv + b, iters + b,
                      final_Lam ? final_Lam + (size_t)b * N : NULL);
        }
        state_free(&s);
        free(gbuf);
    }
    free(w);
    tanner_free(&g);
    return err ? -1 : 0;
}

/*
 * Run T iterations of the first leg (memory strengths gamma_row [N]) with no
 * early exit and record every iteration: Lambda [B][T][N], and when not NULL
 * nu [B][T][E] and mu [B][T][E] in CSR edge order.  Returns 0 or -1.
 */
int oracle_dmem_trace(int32_t M, int32_t N, const int32_t *row_ptr, const int32_t *col_idx,
                      const double *priors, const double *gamma_row, double clip,
                      const uint8_t *sigma, int64_t B, int32_t T, double *Lam_out,
                      double *nu_out, double *mu_out, int32_t nthreads)
{
    if (M < 0 || N < 0 || B < 0 || T < 0 || !(clip > 0)) return -1;
    tanner g;
    if (tanner_build(&g, M, N, row_ptr, col_idx)) { tanner_free(&g); return -1; }
    REAL *w = (REAL *)malloc(sizeof(REAL) * (size_t)(N > 0 ? N : 1));
    REAL *gr = (REAL *)malloc(sizeof(REAL) * (size_t)(N > 0 ? N : 1));
    if (!w || !gr || priors_to_llr(N, priors, w)) { free(w); free(gr); tanner_free(&g); return -1; }
    for (int j = 0; j < N; ++j) gr[j] = (REAL)gamma_row[j];
    int err = 0;
    const int E = g.E;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        state s;
        int ok = state_alloc(&s, N, E) == 0;
        if (!ok) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t b = 0; b < B; ++b) {
            if (!ok) continue;
            const uint8_t *sg = sigma + (size_t)b * M;
            for (int j = 0; j < N; ++j) { s.lam0[j] = w[j]; s.Lam[j] = s.lam0[j]; }
            init_messages(&g, &s);
            for (int t = 0; t < T; ++t) {
                dmem_iteration(&g, sg, gr, (REAL)clip, &s);
                size_t o = ((size_t)b * T + t);
                for (int j = 0; j < N; ++j) Lam_out[o * N + j] = (double)s.Lam[j];
                if (nu_out) for (int e = 0; e < E; ++e) nu_out[o * E + e] = (double)s.nu[e];
                if (mu_out) for (int e = 0; e < E; ++e) mu_out[o * E + e] = (double)s.mu[e];
            }
        }
        state_free(&s);
    }
    free(w); free(gr);
    tanner_free(&g);
    return err ? -1 : 0;
}
