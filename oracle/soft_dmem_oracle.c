/*
 * Soft DMem-BP oracle: one unrolled leg of disordered-memory belief propagation
 * with the sum-product check rule, its loss and its gradient, in FP64.
 * TEST INFRASTRUCTURE ONLY: only tests, the package smoke check and the CPU
 * baseline of the benchmark may load it; it shares no code with the library.
 *
 * Relay's memory rule and message structure (paper Sec. 2.3, "Relay decoding")
 * with the min-sum check rule replaced by sum-product, a per-iteration scale
 * alpha_t and trainable per-fault memory strengths gamma_j (the paper trains
 * nothing; these readings are the design notes' S1-S5):
 *   t = 0           nu_e(0) = Lambda_j(0) = w_j = log((1-p_j)/p_j)  (j = fault of e)
 *   memory          lambda_j(t) = (1-gamma_j) w_j + gamma_j Lambda_j(t-1)
 *   check -> fault  P_e = prod_{e' in row(e), e' != e} tanh(nu_e'(t-1)/2), clamped
 *                   to [-(1-eps), 1-eps];  mu_e(t) = alpha_t (-1)^sigma_i 2 atanh(P_e)
 *   fault -> check  nu_e(t) = lambda_j(t) + sum_{e' in col(j), e' != e} mu_e'(t)
 *   marginal        Lambda_j(t) = lambda_j(t) + sum_{e in col(j)} mu_e(t)
 *   loss            L = mean over shots b and faults j of BCE(sigmoid(-Lambda_j(T)), F_j)
 *                     = F_j softplus(Lambda_j) + (1 - F_j) softplus(-Lambda_j)
 * The gradient is a plain reverse pass over the fully stored trajectory (no
 * checkpointing), written out step by step below; a clamped product passes no
 * gradient.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int M, N, E;
    const int32_t *row_ptr, *col_idx;
    int32_t *row_of;    /* [E] check of edge e */
    int32_t *var_ptr;   /* [N+1] */
    int32_t *var_edges; /* [E] edges of fault j, increasing order */
} graph;

static int graph_build(graph *g, int M, int N, const int32_t *row_ptr, const int32_t *col_idx)
{
    g->M = M; g->N = N; g->E = row_ptr[M];
    g->row_ptr = row_ptr; g->col_idx = col_idx;
    size_t e = (size_t)(g->E > 0 ? g->E : 1);
    g->row_of = (int32_t *)malloc(e * sizeof(int32_t));
    g->var_ptr = (int32_t *)calloc((size_t)N + 1, sizeof(int32_t));
    g->var_edges = (int32_t *)malloc(e * sizeof(int32_t));
    int32_t *fill = (int32_t *)calloc((size_t)N + 1, sizeof(int32_t));
    if (!g->row_of || !g->var_ptr || !g->var_edges || !fill) { free(fill); return -1; }
    for (int i = 0; i < M; ++i)
        for (int e2 = row_ptr[i]; e2 < row_ptr[i + 1]; ++e2) {
            if (col_idx[e2] < 0 || col_idx[e2] >= N) { free(fill); return -1; }
            g->row_of[e2] = i;
            g->var_ptr[col_idx[e2] + 1]++;
        }
    for (int j = 0; j < N; ++j) g->var_ptr[j + 1] += g->var_ptr[j];
    for (int e2 = 0; e2 < g->E; ++e2) {
        int j = col_idx[e2];
        g->var_edges[g->var_ptr[j] + fill[j]++] = e2;
    }
    free(fill);
    return 0;
}

static void graph_free(graph *g) { free(g->row_of); free(g->var_ptr); free(g->var_edges); }

static double softplus(double x) { return x > 0 ? x + log1p(exp(-x)) : log1p(exp(x)); }
static double sigmoid(double x) { return x >= 0 ? 1.0 / (1.0 + exp(-x)) : exp(x) / (1.0 + exp(x)); }

/*
 * One shot: forward over T iterations storing everything, the loss sum over its
 * faults, and (when grad_gamma / grad_alpha are given) the gradient of that sum
 * added into them.  Work arrays: nu [(T+1)*E], mu [(T+1)*E], P [(T+1)*E],
 * clamped [(T+1)*E], Lam [(T+1)*N], lam [(T+1)*N], and adjoints.
 */
typedef struct {
    double *nu, *mu, *P, *Lam, *lam;
    uint8_t *clamped;
    double *nub, *mub, *Lamb, *lamb, *taub;
} work;

static double shot(const graph *g, const double *w, int T, const double *gamma,
                   const double *alpha, double eps, const uint8_t *sigma, const uint8_t *F,
                   work *s, double *grad_gamma, double *grad_alpha, double *marg)
{
    const int N = g->N, E = g->E;
    /* t = 0 */
    for (int j = 0; j < N; ++j) s->Lam[j] = w[j];
    for (int e = 0; e < E; ++e) s->nu[e] = w[g->col_idx[e]];
    for (int t = 1; t <= T; ++t) {
        const double *nu0 = s->nu + (size_t)(t - 1) * E;
        const double *L0 = s->Lam + (size_t)(t - 1) * N;
        double *nu1 = s->nu + (size_t)t * E, *mu1 = s->mu + (size_t)t * E;
        double *P1 = s->P + (size_t)t * E, *L1 = s->Lam + (size_t)t * N;
        double *lam1 = s->lam + (size_t)t * N;
        uint8_t *cl1 = s->clamped + (size_t)t * E;
        for (int j = 0; j < N; ++j) lam1[j] = (1 - gamma[j]) * w[j] + gamma[j] * L0[j];
        for (int i = 0; i < g->M; ++i)
            for (int e = g->row_ptr[i]; e < g->row_ptr[i + 1]; ++e) {
                double prod = 1.0;
                for (int e2 = g->row_ptr[i]; e2 < g->row_ptr[i + 1]; ++e2)
                    if (e2 != e) prod *= tanh(nu0[e2] / 2);
                cl1[e] = 0;
                if (prod > 1 - eps) { prod = 1 - eps; cl1[e] = 1; }
                if (prod < -(1 - eps)) { prod = -(1 - eps); cl1[e] = 1; }
                P1[e] = prod;
                mu1[e] = alpha[t - 1] * (sigma[i] ? -1.0 : 1.0) * 2 * atanh(prod);
            }
        for (int j = 0; j < N; ++j) {
            double L = lam1[j];
            for (int k = g->var_ptr[j]; k < g->var_ptr[j + 1]; ++k) L += mu1[g->var_edges[k]];
            L1[j] = L;
            for (int k = g->var_ptr[j]; k < g->var_ptr[j + 1]; ++k) {
                double v = lam1[j];
                for (int k2 = g->var_ptr[j]; k2 < g->var_ptr[j + 1]; ++k2)
                    if (k2 != k) v += mu1[g->var_edges[k2]];
                nu1[g->var_edges[k]] = v;
            }
        }
    }
    const double *LT = s->Lam + (size_t)T * N;
    double loss = 0;
    for (int j = 0; j < N; ++j) {
        loss += F[j] ? softplus(LT[j]) : softplus(-LT[j]);
        if (marg) marg[j] = LT[j];
    }
    if (!grad_gamma && !grad_alpha) return loss;

    /* reverse pass: adjoints of Lambda(T) from the loss sum */
    for (int j = 0; j < N; ++j) s->Lamb[j] = sigmoid(LT[j]) - (F[j] ? 0.0 : 1.0);
    for (int e = 0; e < E; ++e) s->nub[e] = 0;   /* nu(T) does not reach the loss */
    for (int t = T; t >= 1; --t) {
        const double *nu0 = s->nu + (size_t)(t - 1) * E;
        const double *L0 = s->Lam + (size_t)(t - 1) * N;
        const double *P1 = s->P + (size_t)t * E;
        const uint8_t *cl1 = s->clamped + (size_t)t * E;
        /* nu_e(t) = lambda_j + sum_{e' != e} mu_e';  Lambda_j(t) = lambda_j + sum mu */
        for (int j = 0; j < N; ++j) {
            double sum_nub = 0;
            for (int k = g->var_ptr[j]; k < g->var_ptr[j + 1]; ++k) sum_nub += s->nub[g->var_edges[k]];
            s->lamb[j] = s->Lamb[j] + sum_nub;
            for (int k = g->var_ptr[j]; k < g->var_ptr[j + 1]; ++k) {
                int e = g->var_edges[k];
                double acc = s->Lamb[j];
                for (int k2 = g->var_ptr[j]; k2 < g->var_ptr[j + 1]; ++k2)
                    if (k2 != k) acc += s->nub[g->var_edges[k2]];
                s->mub[e] = acc;
            }
        }
        /* mu_e = alpha_t s_i 2 atanh(P_e);  P_e = prod_{e' != e} tanh(nu_e'(t-1)/2) */
        for (int e = 0; e < E; ++e) s->taub[e] = 0;
        for (int i = 0; i < g->M; ++i) {
            double sgn = sigma[i] ? -1.0 : 1.0;
            for (int e = g->row_ptr[i]; e < g->row_ptr[i + 1]; ++e) {
                if (grad_alpha) grad_alpha[t - 1] += s->mub[e] * sgn * 2 * atanh(P1[e]);
                if (cl1[e]) continue;
                double Pb = s->mub[e] * alpha[t - 1] * sgn * 2 / (1 - P1[e] * P1[e]);
                for (int e2 = g->row_ptr[i]; e2 < g->row_ptr[i + 1]; ++e2) {
                    if (e2 == e) continue;
                    double rest = 1.0;   /* prod over the row without e and e2 */
                    for (int e3 = g->row_ptr[i]; e3 < g->row_ptr[i + 1]; ++e3)
                        if (e3 != e && e3 != e2) rest *= tanh(nu0[e3] / 2);
                    s->taub[e2] += Pb * rest;
                }
            }
        }
        /* tau = tanh(nu(t-1)/2): d tau / d nu = (1 - tau^2) / 2 */
        for (int e = 0; e < E; ++e) {
            double tau = tanh(nu0[e] / 2);
            s->nub[e] = (t - 1 >= 1) ? s->taub[e] * (1 - tau * tau) / 2 : 0.0;
        }
        /* lambda_j(t) = (1 - gamma_j) w_j + gamma_j Lambda_j(t-1) */
        for (int j = 0; j < N; ++j) {
            if (grad_gamma) grad_gamma[j] += s->lamb[j] * (L0[j] - w[j]);
            s->Lamb[j] = (t - 1 >= 1) ? s->lamb[j] * gamma[j] : 0.0;
        }
    }
    return loss;
}

/*
 * Loss (mean over B shots and N faults) and, when the pointers are not NULL, its
 * gradient with respect to gamma [N] and alpha [T], and the final marginals
 * Lambda(T) [B][N].  sigma uint8 [B][M], F uint8 [B][N] (true faults).
 * eps: product clamp (the check rule's |prod| <= 1 - eps).  Returns 0 or -1.
 */
int oracle_soft_dmem(int32_t M, int32_t N, const int32_t *row_ptr, const int32_t *col_idx,
                     const double *priors, int32_t T, const double *gamma, const double *alpha,
                     double eps, const uint8_t *sigma, const uint8_t *F, int64_t B,
                     double *loss, double *grad_gamma, double *grad_alpha, double *marg,
                     int32_t nthreads)
{
    if (M < 0 || N < 1 || T < 1 || B < 1 || !(eps > 0)) return -1;
    graph g;
    if (graph_build(&g, M, N, row_ptr, col_idx)) { graph_free(&g); return -1; }
    double *w = (double *)malloc(sizeof(double) * (size_t)N);
    if (!w) { graph_free(&g); return -1; }
    for (int j = 0; j < N; ++j) {
        if (!(priors[j] > 0 && priors[j] < 1)) { free(w); graph_free(&g); return -1; }
        w[j] = log((1 - priors[j]) / priors[j]);
    }
    const int E = g.E;
    double total = 0;
    int err = 0;
    if (grad_gamma) memset(grad_gamma, 0, sizeof(double) * (size_t)N);
    if (grad_alpha) memset(grad_alpha, 0, sizeof(double) * (size_t)T);
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1) reduction(+ : total)
    {
        work s;
        size_t te = (size_t)(T + 1) * (E > 0 ? E : 1), tn = (size_t)(T + 1) * N;
        s.nu = (double *)malloc(te * sizeof(double));
        s.mu = (double *)calloc(te, sizeof(double));
        s.P = (double *)calloc(te, sizeof(double));
        s.clamped = (uint8_t *)calloc(te, 1);
        s.Lam = (double *)malloc(tn * sizeof(double));
        s.lam = (double *)calloc(tn, sizeof(double));
        s.nub = (double *)malloc(sizeof(double) * (E > 0 ? E : 1));
        s.mub = (double *)malloc(sizeof(double) * (E > 0 ? E : 1));
        s.taub = (double *)malloc(sizeof(double) * (E > 0 ? E : 1));
        s.Lamb = (double *)malloc(sizeof(double) * N);
        s.lamb = (double *)malloc(sizeof(double) * N);
        double *gg = grad_gamma ? (double *)calloc((size_t)N, sizeof(double)) : NULL;
        double *ga = grad_alpha ? (double *)calloc((size_t)T, sizeof(double)) : NULL;
        int ok = s.nu && s.mu && s.P && s.clamped && s.Lam && s.lam && s.nub && s.mub && s.taub &&
                 s.Lamb && s.lamb && (!grad_gamma || gg) && (!grad_alpha || ga);
        if (!ok) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t b = 0; b < B; ++b) {
            if (!ok) continue;
            total += shot(&g, w, T, gamma, alpha, eps, sigma + (size_t)b * M, F + (size_t)b * N,
                          &s, gg, ga, marg ? marg + (size_t)b * N : NULL);
        }
#pragma omp critical
        {
            if (ok && gg) for (int j = 0; j < N; ++j) grad_gamma[j] += gg[j];
            if (ok && ga) for (int t = 0; t < T; ++t) grad_alpha[t] += ga[t];
        }
        free(s.nu); free(s.mu); free(s.P); free(s.clamped); free(s.Lam); free(s.lam);
        free(s.nub); free(s.mub); free(s.taub); free(s.Lamb); free(s.lamb); free(gg); free(ga);
    }
    const double scale = 1.0 / ((double)B * N);
    *loss = total * scale;
    if (grad_gamma) for (int j = 0; j < N; ++j) grad_gamma[j] *= scale;
    if (grad_alpha) for (int t = 0; t < T; ++t) grad_alpha[t] *= scale;
    free(w);
    graph_free(&g);
    return err ? -1 : 0;
}
