// Plain float32 Relay-BP kernel: one thread block per syndrome (paper Sec. 2.3,
// "Relay decoding"; App. A.3).
//
// The reference point for the fused kernel.  It is a direct GPU rendering of the
// algorithm: dense edge-ordered message arrays nu[E] and mu[E] plus the per-fault
// arrays in shared memory, one pass per equation with a block barrier between
// them, and the CSR / CSC index arrays read from global memory.  Arithmetic is
// the same as the fused kernel and the single-precision oracle (every + and *
// rounded separately, same summation order), so all three agree bit for bit.
#include "qldpc_internal.h"

namespace qldpc {
namespace {

constexpr int BASE_THREADS = 256;
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float clampc(float x, float c) { return fminf(fmaxf(x, -c), c); }

struct BaseSmem {
    float *nu, *mu, *Lam, *lam0, *lam;
    uint8_t *F, *sig;
};

__device__ __forceinline__ BaseSmem base_layout(const BaseGraph &g, unsigned char *raw) {
    BaseSmem s;
    size_t o = 0;
    s.nu = reinterpret_cast<float *>(raw + o);
    o += sizeof(float) * g.E;
    s.mu = reinterpret_cast<float *>(raw + o);
    o += sizeof(float) * g.E;
    s.Lam = reinterpret_cast<float *>(raw + o);
    o += sizeof(float) * g.N;
    s.lam0 = reinterpret_cast<float *>(raw + o);
    o += sizeof(float) * g.N;
    s.lam = reinterpret_cast<float *>(raw + o);
    o += sizeof(float) * g.N;
    s.F = raw + o;
    o += g.N;
    s.sig = raw + o;
    return s;
}

// Weight of a decided fault in 2^-33 units with integer operations only (exact
// for float32 |w| >= 2^-10): |w| = m * 2^(e-23) -> m * 2^(e+10).
__device__ __forceinline__ long long base_wfix(float w) {
    const uint32_t b = __float_as_uint(w);
    const int e = (int)((b >> 23) & 0xffu) - 127;
    const long long m = (long long)((b & 0x7fffffu) | 0x800000u);
    const long long a = e >= -10 ? (m << (e + 10)) : (e > -34 ? (m >> (-10 - e)) : 0ll);
    return (b >> 31) ? -a : a;
}

// W = sum_j F_j w_j in 2^-33 units: per-warp partial sums into part[], added up by
// every thread after a barrier (exact, independent of the order).
__device__ void base_weight(const BaseGraph &g, const uint8_t *F, long long *part) {
    long long s = 0;
    for (int j = threadIdx.x; j < g.N; j += BASE_THREADS)
        if (F[j]) s += base_wfix(g.w[j]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
}

__global__ void __launch_bounds__(BASE_THREADS) baseline_decode(BaseGraph g, DevParams p,
                                                                const uint64_t *__restrict__ syn,
                                                                DecodeOut out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const BaseSmem s = base_layout(g, smem_raw);
    __shared__ long long s_Wpart[BASE_THREADS / 32];
    const int shot = blockIdx.x;
    const int tid = threadIdx.x;
    const float C = p.clip;
    const uint64_t *sy = syn + (size_t)shot * g.syn_words;
    uint64_t *cor = out.corr + (size_t)shot * g.cor_words;

    for (int i = tid; i < g.M; i += BASE_THREADS) s.sig[i] = (sy[i >> 6] >> (i & 63)) & 1u;
    for (int j = tid; j < g.N; j += BASE_THREADS) {
        s.lam0[j] = g.w[j];
        s.Lam[j] = s.lam0[j];
    }
    __syncthreads();
    for (int e = tid; e < g.E; e += BASE_THREADS) s.nu[e] = s.lam0[g.col_idx[e]];
    __syncthreads();

    int leg = 0, sols = 0;
    long long iters = 0, Wbest = 0;
    bool have = false;
    for (;;) {
        const int T = leg == 0 ? p.T1 : p.T2;
        const float *gam = g.gamma + (size_t)leg * g.N;
        for (int t = 1; t <= T; ++t) {
            // memory update
            for (int j = tid; j < g.N; j += BASE_THREADS)
                s.lam[j] = __fadd_rn(__fmul_rn(__fsub_rn(1.0f, gam[j]), s.lam0[j]),
                                     __fmul_rn(gam[j], s.Lam[j]));
            // check -> fault
            for (int i = tid; i < g.M; i += BASE_THREADS) {
                const int e0 = g.row_ptr[i], e1 = g.row_ptr[i + 1];
                float m1 = C, m2 = C;
                int am = -1;
                uint32_t neg = s.sig[i];
                for (int e = e0; e < e1; ++e) {
                    const float v = s.nu[e];
                    const float a = fabsf(v);
                    neg ^= v < 0.0f ? 1u : 0u;
                    if (a < m1) {
                        m2 = m1;
                        m1 = a;
                        am = e;
                    } else if (a < m2) {
                        m2 = a;
                    }
                }
                for (int e = e0; e < e1; ++e) {
                    const float v = s.nu[e];
                    const float mag = (e == am) ? m2 : m1;
                    s.mu[e] = (neg ^ (v < 0.0f ? 1u : 0u)) ? -mag : mag;
                }
            }
            __syncthreads();
            // fault -> check, marginals, decisions
            for (int j = tid; j < g.N; j += BASE_THREADS) {
                const int b = g.var_ptr[j], d = g.var_ptr[j + 1] - b;
                float L = s.lam[j];
                for (int k = 0; k < d; ++k) L = __fadd_rn(L, s.mu[g.var_edges[b + k]]);
                L = clampc(L, C);
                s.Lam[j] = L;
                for (int k = 0; k < d; ++k) {
                    float v = s.lam[j];
                    for (int k2 = 0; k2 < d; ++k2)
                        if (k2 != k) v = __fadd_rn(v, s.mu[g.var_edges[b + k2]]);
                    s.nu[g.var_edges[b + k]] = clampc(v, C);
                }
                s.F[j] = L < 0.0f ? 1 : 0;
            }
            __syncthreads();
            ++iters;
            // H F = sigma ?
            int bad = 0;
            for (int i = tid; i < g.M; i += BASE_THREADS) {
                uint32_t par = s.sig[i];
                for (int e = g.row_ptr[i]; e < g.row_ptr[i + 1]; ++e) par ^= s.F[g.col_idx[e]];
                bad |= (int)par;
            }
            if (!__syncthreads_or(bad)) {
                base_weight(g, s.F, s_Wpart);
                __syncthreads();
                long long W = 0;
                for (int w = 0; w < BASE_THREADS / 32; ++w) W += s_Wpart[w];
                if (!have || W < Wbest) {
                    for (int q = tid; q < g.cor_words; q += BASE_THREADS) {
                        uint64_t word = 0;
                        for (int b = 0; b < 64; ++b) {
                            const int j = 64 * q + b;
                            if (j < g.N && s.F[j]) word |= 1ull << b;
                        }
                        cor[q] = word;
                    }
                    have = true;
                    Wbest = W;
                }
                ++sols;
                break;
            }
            if (p.max_iters > 0 && iters >= p.max_iters) break;
        }
        const bool spent = p.max_iters > 0 && iters >= p.max_iters;
        if (sols >= p.S || leg == p.R || spent) break;
        ++leg;
        __syncthreads();
        for (int j = tid; j < g.N; j += BASE_THREADS)
            s.lam0[j] = p.warm_mode == 0 ? s.Lam[j] : g.w[j];
        __syncthreads();
        for (int e = tid; e < g.E; e += BASE_THREADS) s.nu[e] = s.lam0[g.col_idx[e]];
        __syncthreads();
    }
    if (!have) {
        for (int q = tid; q < g.cor_words; q += BASE_THREADS) {
            uint64_t word = 0;
            for (int b = 0; b < 64; ++b) {
                const int j = 64 * q + b;
                if (j < g.N && s.F[j]) word |= 1ull << b;
            }
            cor[q] = word;
        }
    }
    if (tid == 0) {
        if (out.legs) out.legs[shot] = leg + 1;
        if (out.conv) out.conv[shot] = have ? 1 : 0;
        if (out.iters) out.iters[shot] = (int32_t)iters;
    }
}

}  // namespace

size_t baseline_smem_bytes(int M, int N, int E) {
    return sizeof(float) * (2 * (size_t)E + 3 * (size_t)N) + (size_t)N + (size_t)M + 16;
}

const void *baseline_fn() { return (const void *)baseline_decode; }

cudaError_t launch_baseline(int B, int threads, size_t smem, cudaStream_t st, const BaseGraph &g,
                            const DevParams &p, const uint64_t *syn, DecodeOut out) {
    (void)threads;
    baseline_decode<<<B, BASE_THREADS, smem, st>>>(g, p, syn, out);
    return cudaGetLastError();
}

}  // namespace qldpc
