// Soft DMem-BP: one unrolled leg of disordered-memory belief propagation with the
// sum-product check rule, its BCE loss and a hand-written adjoint (reverse mode)
// with checkpointing.  The memory rule and message structure are Relay's (paper
// Sec. 2.3, "Relay decoding"); the sum-product rule, the per-iteration scale
// alpha_t, the trainable gamma_j and the loss are this library's readings:
//   nu_e(0) = Lambda_j(0) = w_j
//   lambda_j(t) = (1 - gamma_j) w_j + gamma_j Lambda_j(t-1)
//   P_e = prod_{e' in row, e' != e} tanh(nu_e'(t-1)/2) clamped to |P_e| <= 1 - eps
//   mu_e(t) = alpha_t (-1)^sigma_i 2 atanh(P_e)
//   nu_e(t) = lambda_j(t) + sum_{e' in col(j), e' != e} mu_e'(t);  Lambda_j(t) = lambda_j(t) + sum mu
//   loss = mean_{b, j} [F_j softplus(Lambda_j(T)) + (1 - F_j) softplus(-Lambda_j(T))]
//
// One block per shot.  The forward keeps nu (edge order of the CSR) and Lambda in
// shared memory and stores them every K iterations (checkpoints).  The adjoint
// walks the checkpoint segments backwards: it recomputes the segment's forward from
// its checkpoint, keeping what each reverse step needs of the state before iteration
// t (the rows' tanh(nu(t-1)/2) and Lambda(t-1)) in a global segment buffer, then runs
// the reverse iterations.  Only the last segment runs its final iteration again (for
// Lambda(T)); in the others the recompute forms only the tanh rows of that iteration's
// input.  Per-shot gradients are summed over shots in a fixed order, so results are
// deterministic.
#include "soft_internal.h"

namespace qldpc {
namespace {

// Threads per block of the forward and of the adjoint, and the adjoint's resident blocks
// per SM (float32 rows of up to 8 edges; its register budget follows from them).
#ifndef SOFT_FWD_THREADS
#define SOFT_FWD_THREADS 512
#endif
#ifndef SOFT_BWD_THREADS
#define SOFT_BWD_THREADS 384
#endif
#ifndef SOFT_BWD_MINB
#define SOFT_BWD_MINB 4
#endif
constexpr unsigned FULL = 0xffffffffu;

template <typename T>
struct RM;
// float32: tanh(x/2) and atanh from the hardware exponential and logarithm and an
// approximate division (absolute errors of a few 1e-7, far inside the float32 path's
// tolerance against the FP64 oracle); FP64 keeps the library functions.
template <>
struct RM<float> {
    // tanh(x/2) = 1 - 2/(1 + e^x); e^x = inf gives 1 and e^x = 0 gives -1
    static __device__ __forceinline__ float tanh_half(float x) {
        return 1.0f - __fdividef(2.0f, 1.0f + __expf(x));
    }
    // atanh(x) = log((1 + x)/(1 - x)) / 2, for |x| <= 1 - 2^-23 (products are clamped)
    static __device__ __forceinline__ float atanh_(float x) {
        return 0.5f * __logf(__fdividef(1.0f + x, 1.0f - x));
    }
    static __device__ __forceinline__ float div(float x, float y) { return __fdividef(x, y); }
    static __device__ __forceinline__ float softplus(float x) {
        return x > 0.0f ? x + log1pf(expf(-x)) : log1pf(expf(x));
    }
    static __device__ __forceinline__ float sigmoid(float x) {
        return x >= 0.0f ? 1.0f / (1.0f + expf(-x)) : expf(x) / (1.0f + expf(x));
    }
};
template <>
struct RM<double> {
    static __device__ __forceinline__ double tanh_half(double x) { return tanh(x / 2.0); }
    static __device__ __forceinline__ double atanh_(double x) { return atanh(x); }
    static __device__ __forceinline__ double div(double x, double y) { return x / y; }
    static __device__ __forceinline__ double softplus(double x) {
        return x > 0.0 ? x + log1p(exp(-x)) : log1p(exp(x));
    }
    static __device__ __forceinline__ double sigmoid(double x) {
        return x >= 0.0 ? 1.0 / (1.0 + exp(-x)) : exp(x) / (1.0 + exp(x));
    }
};

template <typename T>
struct SoftArgs {
    SoftGraph g;
    int T_it, K, nck;
    T eps;
    const uint64_t *syn, *faults;
    int B;
    const T *gamma, *alpha, *w;
    T *ckpt;       // [B][nck][sst] states (nu then Lambda, stride sst)
    T *seg;        // [B][K][sst]
    T *shot_loss;  // [B]
    T *shot_gg;    // [B][N]
    T *shot_ga;    // [B][T]
    T *shot_adj;   // [B][sst] nb and Lb between segments (backward scratch)
    T *marg;       // [B][N] or nullptr
    int sst;       // values per stored state: E + N rounded up to a multiple of 4
};

__device__ __forceinline__ uint32_t bit_of(const uint64_t *v, int i) {
    return (uint32_t)((v[i >> 6] >> (i & 63)) & 1ull);
}

// Sum of one value per thread in a fixed order (warp shuffles, then warp 0):
// deterministic.  Every thread must call it; thread 0 gets the total.
template <int NT, typename T>
__device__ __forceinline__ T block_sum(T v, T *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    T s = 0;
    if (threadIdx.x == 0)
        for (int q = 0; q < NT / 32; ++q) s += red[q];
    __syncthreads();
    return s;
}

// Rows of the edge arrays.  float32 with rows of at most 8 edges (the library pads
// them: row i holds slots 8 i .. 8 i + 7, its degree in row_deg): two 16-byte halves,
// read and written in an order that alternates with i / 4, so that the 8 lanes of a
// quarter warp (8 consecutive rows) meet 32 distinct banks.  Otherwise the CSR row,
// element by element.  Slots k >= d are read as 0 and not written.
template <typename T, int DCM>
__host__ __device__ constexpr bool padded_rows() { return sizeof(T) == 4 && DCM == 8; }

template <typename T, int DCM>
__device__ __forceinline__ void load_row(const T *row, int i, int d, T (&v)[DCM]) {
    if constexpr (padded_rows<T, DCM>()) {
        const bool h = (i >> 2) & 1;
        const float4 a = reinterpret_cast<const float4 *>(row)[h ? 1 : 0];
        const float4 b = reinterpret_cast<const float4 *>(row)[h ? 0 : 1];
        const float4 lo = h ? b : a, hi = h ? a : b;
        v[0] = lo.x; v[1] = lo.y; v[2] = lo.z; v[3] = lo.w;
        v[4] = hi.x; v[5] = hi.y; v[6] = hi.z; v[7] = hi.w;
    } else {
#pragma unroll
        for (int k = 0; k < DCM; ++k) v[k] = k < d ? row[k] : T(0);
    }
}

template <typename T, int DCM>
__device__ __forceinline__ void store_row(T *row, int i, int d, const T (&v)[DCM]) {
    if constexpr (padded_rows<T, DCM>()) {
        const bool h = (i >> 2) & 1;
        const float4 lo = make_float4(v[0], v[1], v[2], v[3]);
        const float4 hi = make_float4(v[4], v[5], v[6], v[7]);
        reinterpret_cast<float4 *>(row)[h ? 1 : 0] = h ? hi : lo;
        reinterpret_cast<float4 *>(row)[h ? 0 : 1] = h ? lo : hi;
    } else {
#pragma unroll
        for (int k = 0; k < DCM; ++k)
            if (k < d) row[k] = v[k];
    }
}

__device__ __forceinline__ void row_span(const SoftGraph &g, int i, int &e0, int &d) {
    if (g.row_deg) {  // padded rows: row i is slots 8 i .. 8 i + 7
        e0 = 8 * i;
        d = g.row_deg[i];
    } else {
        e0 = g.row_ptr[i];
        d = g.row_ptr[i + 1] - e0;
    }
}

// Degree d of fault j and, for degrees 2 and 3, its slots e0, e1, e2 (increasing slot
// order; e2 only for degree 3); b = its first var_edges entry, set for the other degrees
// only (the generic loops).  One 8-byte record when the graph has them, else var_ptr
// and var_edges.
__device__ __forceinline__ void fault_slots(const SoftGraph &g, int j, int &d, int &b, int &e0,
                                            int &e1, int &e2) {
    if (g.fault_rec) {
        const uint2 r = __ldg(g.fault_rec + j);
        e0 = (int)(r.x & 0xffffu);
        e1 = (int)(r.x >> 16);
        e2 = (int)(r.y & 0xffffu);
        d = (int)(r.y >> 16);
        b = (d == 3 || d == 2) ? 0 : g.var_ptr[j];
    } else {
        b = g.var_ptr[j];
        d = g.var_ptr[j + 1] - b;
        e0 = e1 = e2 = 0;
        if (d == 3 || d == 2) {
            e0 = g.var_edges[b];
            e1 = g.var_edges[b + 1];
            if (d == 3) e2 = g.var_edges[b + 2];
        }
    }
}

// tau_k = tanh(nu_k/2) of one row of d <= DCM edges (values v); 1 on slots k >= d.
template <typename T, int DCM>
__device__ __forceinline__ void row_tanh(const T (&v)[DCM], int d, T (&tau)[DCM]) {
#pragma unroll
    for (int k = 0; k < DCM; ++k) tau[k] = k < d ? RM<T>::tanh_half(v[k]) : T(1);
}

// Check products of one row: P_k = prod_{l != k} tau_l, clamped (cl_k: it was).  The
// row has d <= DCM edges and tau = 1 on slots k >= d.  float32 forms them from prefix
// and suffix products (O(d)); FP64 multiplies in increasing l, as the oracle does.
template <typename T, int DCM>
__device__ __forceinline__ void row_products(const T (&tau)[DCM], int d, T eps, T (&P)[DCM],
                                             bool (&cl)[DCM]) {
    T suf[DCM];
    if constexpr (sizeof(T) == 4) {
        suf[DCM - 1] = T(1);
#pragma unroll
        for (int k = DCM - 2; k >= 0; --k) suf[k] = suf[k + 1] * tau[k + 1];
    }
    T pre = T(1);
#pragma unroll
    for (int k = 0; k < DCM; ++k) {
        T prod = T(1);
        if constexpr (sizeof(T) == 4) {
            prod = pre * suf[k];
            pre *= tau[k];
        } else {
#pragma unroll
            for (int l = 0; l < DCM; ++l)
                if (l != k && l < d) prod *= tau[l];
        }
        cl[k] = false;
        if (prod > T(1) - eps) {
            prod = T(1) - eps;
            cl[k] = true;
        }
        if (prod < -(T(1) - eps)) {
            prod = -(T(1) - eps);
            cl[k] = true;
        }
        P[k] = prod;
    }
}

// One forward iteration t (1-based) on the shared state nu[E], Lam[N] (in place).  With
// tau_out, the check pass also stores each row's tanh(nu(t-1)/2) there (the adjoint's
// saved state; padded rows whole, with 1 on the padding slots).
template <int NT, typename T, int DCM>
__device__ __forceinline__ void soft_iteration(const SoftArgs<T> &a, const uint64_t *sy, int t,
                                               T *nu, T *Lam, T *tau_out = nullptr) {
    const SoftGraph &g = a.g;
    const T at = a.alpha[t - 1];
    for (int i = threadIdx.x; i < g.M; i += NT) {
        int e0, d;
        row_span(g, i, e0, d);
        T v[DCM], tau[DCM], P[DCM];
        bool cl[DCM];
        load_row<T, DCM>(nu + e0, i, d, v);
        row_tanh<T, DCM>(v, d, tau);
        if (tau_out) store_row<T, DCM>(tau_out + e0, i, d, tau);
        row_products<T, DCM>(tau, d, a.eps, P, cl);
        const T s = bit_of(sy, i) ? T(-2) : T(2);
#pragma unroll
        for (int k = 0; k < DCM; ++k) v[k] = k < d ? at * s * RM<T>::atanh_(P[k]) : T(0);
        store_row<T, DCM>(nu + e0, i, d, v);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < g.N; j += NT) {
        int d, b, e0, e1, e2;
        fault_slots(g, j, d, b, e0, e1, e2);
        const T lam = (T(1) - a.gamma[j]) * a.w[j] + a.gamma[j] * Lam[j];
        // degrees 3 and 2 in registers, with the generic loop's order of additions
        if (d == 3 || d == 2) {
            const T m0 = nu[e0], m1 = nu[e1];
            if (d == 3) {
                const T m2 = nu[e2];
                Lam[j] = lam + m0 + m1 + m2;
                nu[e0] = lam + m1 + m2;
                nu[e1] = lam + m0 + m2;
                nu[e2] = lam + m0 + m1;
            } else {
                Lam[j] = lam + m0 + m1;
                nu[e0] = lam + m1;
                nu[e1] = lam + m0;
            }
            continue;
        }
        T mu[8];
        for (int k = 0; k < d; ++k) mu[k] = nu[g.var_edges[b + k]];
        T L = lam;
        for (int k = 0; k < d; ++k) L += mu[k];
        Lam[j] = L;
        for (int k = 0; k < d; ++k) {
            T v = lam;
            for (int k2 = 0; k2 < d; ++k2)
                if (k2 != k) v += mu[k2];
            nu[g.var_edges[b + k]] = v;
        }
    }
    __syncthreads();
}

// tanh(nu/2) of every row of the shared nu, stored to tau_out as in soft_iteration.
template <int NT, typename T, int DCM>
__device__ __forceinline__ void tau_pass(const SoftGraph &g, const T *nu, T *tau_out) {
    for (int i = threadIdx.x; i < g.M; i += NT) {
        int e0, d;
        row_span(g, i, e0, d);
        T v[DCM], tau[DCM];
        load_row<T, DCM>(nu + e0, i, d, v);
        row_tanh<T, DCM>(v, d, tau);
        store_row<T, DCM>(tau_out + e0, i, d, tau);
    }
}

template <int NT, typename T>
__device__ __forceinline__ void init_state(const SoftArgs<T> &a, T *nu, T *Lam) {
    const SoftGraph &g = a.g;
    for (int j = threadIdx.x; j < g.N; j += NT) Lam[j] = a.w[j];
    for (int e = threadIdx.x; e < g.E; e += NT) nu[e] = a.w[g.col_idx[e]];
    __syncthreads();
}

// Bulk prefetch of bytes (a multiple of 16) at a 16-byte aligned global address into L2.
__device__ __forceinline__ void prefetch_l2(const void *p, size_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"((unsigned)bytes)
                 : "memory");
}

// Copy of n values (a state: nu then Lambda, contiguous in both places, or nu or its
// adjoint alone).  float32 moves 16-byte vectors: every state starts on a 16-byte
// boundary (the stride a.sst is a multiple of 4 values, the workspace is 16-byte
// aligned) and n is a multiple of 4.
template <int NT, typename T>
__device__ __forceinline__ void copy_state(const T *src, T *dst, int n) {
    if constexpr (sizeof(T) == 4) {
        const float4 *s4 = reinterpret_cast<const float4 *>(src);
        float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll 4
        for (int q = threadIdx.x; q < n / 4; q += NT) d4[q] = s4[q];
    } else {
        for (int e = threadIdx.x; e < n; e += NT) dst[e] = src[e];
    }
}

// Forward.  Shared memory: nu[E], Lam[N] (a.sst values).  The state before iterations
// 1, K + 1, 2K + 1, ... is stored as a checkpoint.
template <typename T, int DCM>
__global__ void __launch_bounds__(SOFT_FWD_THREADS) soft_forward(SoftArgs<T> a) {
    constexpr int NT = SOFT_FWD_THREADS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SoftGraph &g = a.g;
    T *nu = reinterpret_cast<T *>(smem_raw);
    T *Lam = nu + g.E;
    __shared__ T red[NT / 32];
    const int b = blockIdx.x;
    const uint64_t *sy = a.syn + (size_t)b * g.syn_words;
    const uint64_t *fy = a.faults + (size_t)b * g.cor_words;
    const size_t S = (size_t)a.sst;
    init_state<NT>(a, nu, Lam);
    for (int t = 1; t <= a.T_it; ++t) {
        if ((t - 1) % a.K == 0) {
            copy_state<NT>(nu, a.ckpt + ((size_t)b * a.nck + (t - 1) / a.K) * S, (int)S);
            __syncthreads();  // copied before the check pass overwrites nu
        }
        soft_iteration<NT, T, DCM>(a, sy, t, nu, Lam);
    }
    T part = 0;
    for (int j = threadIdx.x; j < g.N; j += NT) {
        part += bit_of(fy, j) ? RM<T>::softplus(Lam[j]) : RM<T>::softplus(-Lam[j]);
        if (a.marg) a.marg[(size_t)b * g.N + j] = Lam[j];
    }
    const T tot = block_sum<NT>(part, red);
    if (threadIdx.x == 0) a.shot_loss[b] = tot;
}

// Adjoint.  Shared memory holds a.sst + T values, as much as the forward's state, so
// the adjoint runs as many blocks per SM as the forward:
//   * the recompute of a segment runs the forward iterations on nu[E], Lam[N] and
//     stores, for each of the segment's iterations, what its reverse step needs of the
//     state before it in the segment buffer: tanh(nu/2) of every row (written by the
//     check pass that computes it) and Lambda;
//   * the reverse steps keep nb[E] (adjoint of nu(t), then of mu(t)) in nu's place and
//     Lb[N] (adjoint of Lambda) in Lam's place, and read the saved states from the
//     segment buffer (the next step's state is prefetched into L2 by one bulk prefetch);
//     during a recompute nb and Lb wait in global scratch (shot_adj);
//   * as[T] (alpha gradient of the shot) follows the state.
// The gamma gradient of fault j is touched only by the thread that owns j, so it stays
// in global memory (shot_gg: coalesced, cached).
template <typename T, int DCM>
__global__ void __launch_bounds__(SOFT_BWD_THREADS, padded_rows<T, DCM>() ? SOFT_BWD_MINB : 1)
    soft_backward(SoftArgs<T> a) {
    constexpr int NT = SOFT_BWD_THREADS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SoftGraph &g = a.g;
    T *nu = reinterpret_cast<T *>(smem_raw);
    T *Lam = nu + g.E;
    T *nb = nu;
    T *Lb = Lam;
    T *as = nu + a.sst;
    __shared__ T red[NT / 32];
    const int b = blockIdx.x;
    T *gs = a.shot_gg + (size_t)b * g.N;
    const uint64_t *sy = a.syn + (size_t)b * g.syn_words;
    const uint64_t *fy = a.faults + (size_t)b * g.cor_words;
    const size_t S = (size_t)a.sst;
    T *segb = a.seg + (size_t)b * a.K * S;
    T *adj = a.shot_adj + (size_t)b * S;
    for (int j = threadIdx.x; j < g.N; j += NT) gs[j] = 0;
    for (int t = threadIdx.x; t < a.T_it; t += NT) as[t] = 0;

    for (int s = a.nck - 1; s >= 0; --s) {
        const int t0 = s * a.K, t1 = min(a.T_it, t0 + a.K);
        const bool last = s == a.nck - 1;
        T *ck = a.ckpt + ((size_t)b * a.nck + s) * S;
        if (!last) {  // nb and Lb of the segment after this one wait in global scratch
            copy_state<NT>(nu, adj, (int)S);
            __syncthreads();
        }
        copy_state<NT>(ck, nu, (int)S);  // nu, then Lam = nu + E
        __syncthreads();
        // the saved states before iterations t0+1 .. t1 (tanh rows, then Lambda); iteration
        // t1 itself runs only in the last segment, whose Lambda(T) seeds the adjoint (in the
        // others only its tanh rows are formed).  Lam[j] is copied and later updated by the
        // thread that owns j, so the copy needs no barrier.
        for (int t = t0 + 1; t <= t1; ++t) {
            T *st = segb + (size_t)(t - t0 - 1) * S;
            for (int j = threadIdx.x; j < g.N; j += NT) st[g.E + j] = Lam[j];
            if (t < t1 || last)
                soft_iteration<NT, T, DCM>(a, sy, t, nu, Lam, st);
            else
                tau_pass<NT, T, DCM>(g, nu, st);
        }
        if (last) {  // Lambda(T) is in Lam: Lb = adjoint of the loss sum, in place; nb = 0
            for (int j = threadIdx.x; j < g.N; j += NT)
                Lb[j] = RM<T>::sigmoid(Lam[j]) - (bit_of(fy, j) ? T(0) : T(1));
            for (int e = threadIdx.x; e < g.E; e += NT) nb[e] = 0;
        } else {
            __syncthreads();  // the tanh pass has read nu
            copy_state<NT>(adj, nu, (int)S);
        }
        __syncthreads();
        for (int t = t1; t > t0; --t) {
            // the saved state before iteration t, from the segment buffer
            const T *tau_prev = segb + (size_t)(t - t0 - 1) * S;
            const T *L_prev = tau_prev + g.E;
            if (threadIdx.x == 0 && t > t0 + 1) prefetch_l2(tau_prev - S, S * sizeof(T));
            const bool inner = t - 1 >= 1;
            // fault adjoint: lambda_bar = Lb + sum nb;  mu_bar_e = lambda_bar - nb_e
            for (int j = threadIdx.x; j < g.N; j += NT) {
                int d, e0, f0, f1, f2;
                fault_slots(g, j, d, e0, f0, f1, f2);
                T lb;
                if (d == 3 || d == 2) {  // in registers, same order of additions
                    const T n0 = nb[f0], n1 = nb[f1];
                    const T n2 = d == 3 ? nb[f2] : T(0);
                    lb = Lb[j] + (d == 3 ? T(0) + n0 + n1 + n2 : T(0) + n0 + n1);
                    nb[f0] = lb - n0;
                    nb[f1] = lb - n1;
                    if (d == 3) nb[f2] = lb - n2;
                } else {
                    T sum = 0;
                    for (int k = 0; k < d; ++k) sum += nb[g.var_edges[e0 + k]];
                    lb = Lb[j] + sum;
                    for (int k = 0; k < d; ++k) {
                        const int e = g.var_edges[e0 + k];
                        nb[e] = lb - nb[e];
                    }
                }
                gs[j] += lb * (L_prev[j] - a.w[j]);
                Lb[j] = inner ? lb * a.gamma[j] : T(0);
            }
            __syncthreads();
            // check adjoint: mu_e = alpha_t s 2 atanh(P_e)
            const T at = a.alpha[t - 1];
            T apart = 0;
            for (int i = threadIdx.x; i < g.M; i += NT) {
                int e0, d;
                row_span(g, i, e0, d);
                T tau[DCM], P[DCM], Pb[DCM], mbv[DCM];
                bool cl[DCM];
                load_row<T, DCM>(tau_prev + e0, i, d, tau);
                if constexpr (!padded_rows<T, DCM>()) {  // slots k >= d were read as 0
#pragma unroll
                    for (int k = 0; k < DCM; ++k)
                        if (k >= d) tau[k] = T(1);
                }
                row_products<T, DCM>(tau, d, a.eps, P, cl);
                load_row<T, DCM>(nb + e0, i, d, mbv);
                const T s2 = bit_of(sy, i) ? T(-2) : T(2);
#pragma unroll
                for (int k = 0; k < DCM; ++k) {
                    Pb[k] = 0;
                    if (k < d) {
                        const T mb = mbv[k];
                        apart += mb * s2 * RM<T>::atanh_(P[k]);
                        if (!cl[k]) Pb[k] = RM<T>::div(mb * at * s2, T(1) - P[k] * P[k]);
                    }
                }
                // tau_bar_k = sum_{m != k} Pb_m prod_{l != m, k} tau_l in O(d), without
                // division: with pre_k = prod_{l < k} tau_l and suf_k = prod_{l > k} tau_l,
                // the terms m > k are pre_k X_k and the terms m < k are Y_k suf_k, where
                // X_k = Pb_{k+1} suf_{k+1} + tau_{k+1} X_{k+1} and
                // Y_k = Pb_{k-1} pre_{k-1} + tau_{k-1} Y_{k-1}.
                T pre[DCM], suf[DCM];
                pre[0] = T(1);
#pragma unroll
                for (int k = 1; k < DCM; ++k) pre[k] = pre[k - 1] * tau[k - 1];
                suf[DCM - 1] = T(1);
#pragma unroll
                for (int k = DCM - 2; k >= 0; --k) suf[k] = suf[k + 1] * tau[k + 1];
                // slots k >= d hold tau = 1 and Pb = 0, so the full-width recurrences give
                // the row's values for k < d
                T X[DCM], Y = T(0);
                X[DCM - 1] = T(0);
#pragma unroll
                for (int k = DCM - 2; k >= 0; --k) X[k] = Pb[k + 1] * suf[k + 1] + tau[k + 1] * X[k + 1];
#pragma unroll
                for (int k = 0; k < DCM; ++k) {
                    if (k > 0) Y = Pb[k - 1] * pre[k - 1] + tau[k - 1] * Y;
                    mbv[k] = T(0);
                    if (k < d) {
                        const T tb = pre[k] * X[k] + Y * suf[k];
                        mbv[k] = inner ? tb * (T(1) - tau[k] * tau[k]) / T(2) : T(0);
                    }
                }
                store_row<T, DCM>(nb + e0, i, d, mbv);
            }
            const T asum = block_sum<NT>(apart, red);  // includes the barrier
            if (threadIdx.x == 0) as[t - 1] += asum;
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < a.T_it; t += NT) a.shot_ga[(size_t)b * a.T_it + t] = as[t];
}

// out[c] = scale * upstream * sum_b in[b][c], summed over b in order.
template <typename T>
__global__ void reduce_shots(const T *in, int B, int n, T scale, const T *upstream, T *out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    T s = 0;
    for (int b = 0; b < B; ++b) s += in[(size_t)b * n + c];
    out[c] = s * scale * (upstream ? *upstream : T(1));
}

template <typename T>
size_t fwd_smem(const SoftGraph &g) { return sizeof(T) * (size_t)soft_state_values(g); }
template <typename T>
size_t bwd_smem(const SoftGraph &g, int Tit) {
    return sizeof(T) * ((size_t)soft_state_values(g) + Tit);
}

template <typename T, int DCM>
cudaError_t run_forward_t(const SoftLaunch &L, cudaStream_t st) {
    SoftArgs<T> a{};
    a.g = L.g;
    a.T_it = L.T_it;
    a.K = L.K;
    a.nck = (L.T_it + L.K - 1) / L.K;
    a.eps = (T)L.eps;
    a.syn = L.syn;
    a.faults = L.faults;
    a.B = L.B;
    a.gamma = static_cast<const T *>(L.gamma);
    a.alpha = static_cast<const T *>(L.alpha);
    a.w = static_cast<const T *>(L.w);
    a.ckpt = static_cast<T *>(L.ckpt);
    a.seg = static_cast<T *>(L.seg);
    a.shot_loss = static_cast<T *>(L.shot_loss);
    a.shot_gg = static_cast<T *>(L.shot_gg);
    a.shot_ga = static_cast<T *>(L.shot_ga);
    a.marg = static_cast<T *>(L.marg);
    a.sst = soft_state_values(L.g);
    const size_t sm = fwd_smem<T>(L.g);
    cudaError_t e = cudaFuncSetAttribute(soft_forward<T, DCM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    soft_forward<T, DCM><<<L.B, SOFT_FWD_THREADS, sm, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const T scale = T(1) / ((T)L.B * (T)L.g.N);
    reduce_shots<T><<<1, 32, 0, st>>>(a.shot_loss, L.B, 1, scale, nullptr,
                                      static_cast<T *>(L.loss));
    return cudaGetLastError();
}

template <typename T, int DCM>
cudaError_t run_backward_t(const SoftLaunch &L, cudaStream_t st) {
    SoftArgs<T> a{};
    a.g = L.g;
    a.T_it = L.T_it;
    a.K = L.K;
    a.nck = (L.T_it + L.K - 1) / L.K;
    a.eps = (T)L.eps;
    a.syn = L.syn;
    a.faults = L.faults;
    a.B = L.B;
    a.gamma = static_cast<const T *>(L.gamma);
    a.alpha = static_cast<const T *>(L.alpha);
    a.w = static_cast<const T *>(L.w);
    a.ckpt = static_cast<T *>(L.ckpt);
    a.seg = static_cast<T *>(L.seg);
    a.shot_loss = static_cast<T *>(L.shot_loss);
    a.shot_gg = static_cast<T *>(L.shot_gg);
    a.shot_ga = static_cast<T *>(L.shot_ga);
    a.shot_adj = static_cast<T *>(L.shot_adj);
    a.sst = soft_state_values(L.g);
    const size_t sm = bwd_smem<T>(L.g, L.T_it);
    cudaError_t e = cudaFuncSetAttribute(soft_backward<T, DCM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    soft_backward<T, DCM><<<L.B, SOFT_BWD_THREADS, sm, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const T scale = T(1) / ((T)L.B * (T)L.g.N);
    const T *up = static_cast<const T *>(L.upstream);
    reduce_shots<T><<<(L.g.N + 127) / 128, 128, 0, st>>>(a.shot_gg, L.B, L.g.N, scale, up,
                                                         static_cast<T *>(L.grad_gamma));
    reduce_shots<T><<<(L.T_it + 127) / 128, 128, 0, st>>>(a.shot_ga, L.B, L.T_it, scale, up,
                                                          static_cast<T *>(L.grad_alpha));
    return cudaGetLastError();
}

}  // namespace

size_t soft_smem_forward(const SoftGraph &g, int fp64) {
    return fp64 ? fwd_smem<double>(g) : fwd_smem<float>(g);
}
size_t soft_smem_backward(const SoftGraph &g, int T_it, int fp64) {
    return fp64 ? bwd_smem<double>(g, T_it) : bwd_smem<float>(g, T_it);
}

cudaError_t soft_run_forward(const SoftLaunch &L, cudaStream_t st) {
    if (L.fp64) return L.dc_max <= 8 ? run_forward_t<double, 8>(L, st) : run_forward_t<double, 32>(L, st);
    return L.dc_max <= 8 ? run_forward_t<float, 8>(L, st) : run_forward_t<float, 32>(L, st);
}

cudaError_t soft_run_backward(const SoftLaunch &L, cudaStream_t st) {
    if (L.fp64) return L.dc_max <= 8 ? run_backward_t<double, 8>(L, st) : run_backward_t<double, 32>(L, st);
    return L.dc_max <= 8 ? run_backward_t<float, 8>(L, st) : run_backward_t<float, 32>(L, st);
}

}  // namespace qldpc
