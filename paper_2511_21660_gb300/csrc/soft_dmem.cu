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
// its checkpoint, keeping each iteration's nu(t-1), Lambda(t-1) in a global
// segment buffer, then runs the reverse iterations.  Only the last segment runs its
// final iteration again (for Lambda(T)); in the others the recompute stops one
// iteration short, and the state it ends on is the first reverse step's input.  Per-shot gradients are summed
// over shots in a fixed order, so results are deterministic.
#include "soft_internal.h"

namespace qldpc {
namespace {

constexpr int SOFT_THREADS = 256;
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
    T *ckpt;       // [B][nck][E+N]
    T *seg;        // [B][K][E+N]
    T *shot_loss;  // [B]
    T *shot_gg;    // [B][N]
    T *shot_ga;    // [B][T]
    T *shot_lb;    // [B][N] adjoint of Lambda (backward scratch)
    T *marg;       // [B][N] or nullptr
};

__device__ __forceinline__ uint32_t bit_of(const uint64_t *v, int i) {
    return (uint32_t)((v[i >> 6] >> (i & 63)) & 1ull);
}

// Sum of one value per thread in a fixed order (warp shuffles, then warp 0):
// deterministic.  Every thread must call it; thread 0 gets the total.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    T s = 0;
    if (threadIdx.x == 0)
        for (int q = 0; q < SOFT_THREADS / 32; ++q) s += red[q];
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
    e0 = g.row_ptr[i];
    d = g.row_deg ? g.row_deg[i] : g.row_ptr[i + 1] - e0;
}

// Check products of one row: P_k = prod_{l != k} tanh(nu_l/2), clamped.  The row
// has d <= DCM edges (values v).  float32 forms them from prefix and suffix products
// (O(d)); FP64 multiplies in increasing l, as the oracle does.
template <typename T, int DCM>
__device__ __forceinline__ void row_products(const T (&v)[DCM], int d, T eps, T (&tau)[DCM],
                                             T (&P)[DCM], bool (&cl)[DCM]) {
#pragma unroll
    for (int k = 0; k < DCM; ++k) tau[k] = k < d ? RM<T>::tanh_half(v[k]) : T(1);
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

// One forward iteration t (1-based) on the shared state nu[E], Lam[N] (in place).
template <typename T, int DCM>
__device__ __forceinline__ void soft_iteration(const SoftArgs<T> &a, const uint64_t *sy, int t,
                                               T *nu, T *Lam) {
    const SoftGraph &g = a.g;
    const T at = a.alpha[t - 1];
    for (int i = threadIdx.x; i < g.M; i += SOFT_THREADS) {
        int e0, d;
        row_span(g, i, e0, d);
        T v[DCM], tau[DCM], P[DCM];
        bool cl[DCM];
        load_row<T, DCM>(nu + e0, i, d, v);
        row_products<T, DCM>(v, d, a.eps, tau, P, cl);
        const T s = bit_of(sy, i) ? T(-2) : T(2);
#pragma unroll
        for (int k = 0; k < DCM; ++k) v[k] = k < d ? at * s * RM<T>::atanh_(P[k]) : T(0);
        store_row<T, DCM>(nu + e0, i, d, v);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < g.N; j += SOFT_THREADS) {
        const int b = g.var_ptr[j], d = g.var_ptr[j + 1] - b;
        const T lam = (T(1) - a.gamma[j]) * a.w[j] + a.gamma[j] * Lam[j];
        // degrees 3 and 2 in registers, with the generic loop's order of additions
        if (d == 3 || d == 2) {
            const int e0 = g.var_edges[b], e1 = g.var_edges[b + 1];
            const T m0 = nu[e0], m1 = nu[e1];
            if (d == 3) {
                const int e2 = g.var_edges[b + 2];
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

template <typename T>
__device__ __forceinline__ void init_state(const SoftArgs<T> &a, T *nu, T *Lam) {
    const SoftGraph &g = a.g;
    for (int j = threadIdx.x; j < g.N; j += SOFT_THREADS) Lam[j] = a.w[j];
    for (int e = threadIdx.x; e < g.E; e += SOFT_THREADS) nu[e] = a.w[g.col_idx[e]];
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ void copy_state(const T *src_nu, const T *src_L, T *dst, int E, int N) {
    for (int e = threadIdx.x; e < E; e += SOFT_THREADS) dst[e] = src_nu[e];
    for (int j = threadIdx.x; j < N; j += SOFT_THREADS) dst[E + j] = src_L[j];
}

template <typename T, int DCM>
__global__ void __launch_bounds__(SOFT_THREADS) soft_forward(SoftArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SoftGraph &g = a.g;
    T *nu = reinterpret_cast<T *>(smem_raw);
    T *Lam = nu + g.E;
    __shared__ T red[SOFT_THREADS / 32];
    const int b = blockIdx.x;
    const uint64_t *sy = a.syn + (size_t)b * g.syn_words;
    const uint64_t *fy = a.faults + (size_t)b * g.cor_words;
    const size_t EN = (size_t)g.E + g.N;
    init_state(a, nu, Lam);
    for (int t = 1; t <= a.T_it; ++t) {
        if ((t - 1) % a.K == 0)
            copy_state(nu, Lam, a.ckpt + ((size_t)b * a.nck + (t - 1) / a.K) * EN, g.E, g.N);
        soft_iteration<T, DCM>(a, sy, t, nu, Lam);
    }
    T part = 0;
    for (int j = threadIdx.x; j < g.N; j += SOFT_THREADS) {
        part += bit_of(fy, j) ? RM<T>::softplus(Lam[j]) : RM<T>::softplus(-Lam[j]);
        if (a.marg) a.marg[(size_t)b * g.N + j] = Lam[j];
    }
    const T tot = block_sum(part, red);
    if (threadIdx.x == 0) a.shot_loss[b] = tot;
}

// Adjoint.  Shared memory: nu[E], Lam[N] (forward recompute, then each reverse step's
// saved state), nb[E] (adjoint of nu(t), then of mu(t)), as[T] (alpha gradient of the
// shot).  The adjoint of Lambda and the gamma gradient of fault j are touched only by
// the thread that owns j, so they stay in global memory (shot_lb, shot_gg: coalesced,
// cached), which keeps the block's shared state small enough for 3 blocks per SM.
template <typename T, int DCM>
__global__ void __launch_bounds__(SOFT_THREADS) soft_backward(SoftArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SoftGraph &g = a.g;
    T *nu = reinterpret_cast<T *>(smem_raw);
    T *Lam = nu + g.E;
    T *nb = Lam + g.N;
    T *as = nb + g.E;
    __shared__ T red[SOFT_THREADS / 32];
    const int b = blockIdx.x;
    T *Lb = a.shot_lb + (size_t)b * g.N;
    T *gs = a.shot_gg + (size_t)b * g.N;
    const uint64_t *sy = a.syn + (size_t)b * g.syn_words;
    const uint64_t *fy = a.faults + (size_t)b * g.cor_words;
    const size_t EN = (size_t)g.E + g.N;
    T *segb = a.seg + (size_t)b * a.K * EN;
    for (int j = threadIdx.x; j < g.N; j += SOFT_THREADS) gs[j] = 0;
    for (int t = threadIdx.x; t < a.T_it; t += SOFT_THREADS) as[t] = 0;

    for (int s = a.nck - 1; s >= 0; --s) {
        const int t0 = s * a.K, t1 = min(a.T_it, t0 + a.K);
        const bool last = s == a.nck - 1;
        const T *ck = a.ckpt + ((size_t)b * a.nck + s) * EN;
        for (int e = threadIdx.x; e < g.E; e += SOFT_THREADS) nu[e] = ck[e];
        for (int j = threadIdx.x; j < g.N; j += SOFT_THREADS) Lam[j] = ck[g.E + j];
        __syncthreads();
        // states before iterations t0+1 .. t1; iteration t1 itself runs only in the last
        // segment, whose Lambda(T) seeds the adjoint; elsewhere the state before t1 stays
        // in shared memory for the first reverse step
        for (int t = t0 + 1; t <= (last ? t1 : t1 - 1); ++t) {
            copy_state(nu, Lam, segb + (size_t)(t - t0 - 1) * EN, g.E, g.N);
            soft_iteration<T, DCM>(a, sy, t, nu, Lam);
        }
        if (last) {  // Lambda(T) is in Lam: adjoint of the loss sum
            for (int j = threadIdx.x; j < g.N; j += SOFT_THREADS)
                Lb[j] = RM<T>::sigmoid(Lam[j]) - (bit_of(fy, j) ? T(0) : T(1));
            for (int e = threadIdx.x; e < g.E; e += SOFT_THREADS) nb[e] = 0;
        }
        __syncthreads();
        for (int t = t1; t > t0; --t) {
            // the state before iteration t, staged in the forward arrays (free here; it is
            // already there for the first reverse step of a segment that is not the last)
            if (t < t1 || last)
                copy_state(segb + (size_t)(t - t0 - 1) * EN,
                           segb + (size_t)(t - t0 - 1) * EN + g.E, nu, g.E, g.N);
            __syncthreads();
            const T *nu_prev = nu;
            const T *L_prev = Lam;
            const bool inner = t - 1 >= 1;
            // fault adjoint: lambda_bar = Lb + sum nb;  mu_bar_e = lambda_bar - nb_e
            for (int j = threadIdx.x; j < g.N; j += SOFT_THREADS) {
                const int e0 = g.var_ptr[j], d = g.var_ptr[j + 1] - e0;
                T lb;
                if (d == 3 || d == 2) {  // in registers, same order of additions
                    const int f0 = g.var_edges[e0], f1 = g.var_edges[e0 + 1];
                    const int f2 = d == 3 ? g.var_edges[e0 + 2] : f1;
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
            for (int i = threadIdx.x; i < g.M; i += SOFT_THREADS) {
                int e0, d;
                row_span(g, i, e0, d);
                T v[DCM], tau[DCM], P[DCM], Pb[DCM], mbv[DCM];
                bool cl[DCM];
                load_row<T, DCM>(nu_prev + e0, i, d, v);
                row_products<T, DCM>(v, d, a.eps, tau, P, cl);
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
            const T asum = block_sum(apart, red);  // includes the barrier
            if (threadIdx.x == 0) as[t - 1] += asum;
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < a.T_it; t += SOFT_THREADS) a.shot_ga[(size_t)b * a.T_it + t] = as[t];
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
size_t fwd_smem(const SoftGraph &g) { return sizeof(T) * ((size_t)g.E + g.N); }
template <typename T>
size_t bwd_smem(const SoftGraph &g, int Tit) {
    return sizeof(T) * (2 * (size_t)g.E + g.N + Tit);
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
    a.shot_lb = static_cast<T *>(L.shot_lb);
    a.marg = static_cast<T *>(L.marg);
    const size_t sm = fwd_smem<T>(L.g);
    cudaError_t e = cudaFuncSetAttribute(soft_forward<T, DCM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    soft_forward<T, DCM><<<L.B, SOFT_THREADS, sm, st>>>(a);
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
    a.shot_lb = static_cast<T *>(L.shot_lb);
    const size_t sm = bwd_smem<T>(L.g, L.T_it);
    cudaError_t e = cudaFuncSetAttribute(soft_backward<T, DCM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    soft_backward<T, DCM><<<L.B, SOFT_THREADS, sm, st>>>(a);
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
