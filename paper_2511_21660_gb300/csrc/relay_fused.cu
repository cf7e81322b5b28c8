// Fused persistent Relay-BP kernel (paper Sec. 2.3 "Relay decoding", App. A.3).
//
// One thread block decodes one syndrome at a time and pulls the next one from a
// global work counter when it finishes (per-shot early exit, no idle blocks
// behind slow shots).  Per shot:
//   * the message of every edge lives in shared memory in one slot, overwritten
//     in place: the check pass turns nu(t-1) into mu(t), the fault pass turns
//     mu(t) into nu(t).  Slot (k, i) = k*Mp + i is the k-th edge of check i, so
//     the check pass reads and writes whole warps of consecutive addresses and
//     only the fault pass gathers;
//   * the per-fault state (Lambda_j, (1-gamma_j) lambda_j(0), gamma_j) lives in
//     registers: fault j belongs to thread j mod NT for the whole shot;
//   * decisions F_j = [Lambda_j < 0] are packed by warp ballots into a bitmap in
//     shared memory, and H F = sigma is tested by XOR over each check's slots.
// All float arithmetic rounds every + and * separately (__fadd_rn/__fmul_rn), in
// the same order as the single-precision oracle, so results are bit-identical.
//
// This translation unit is compiled once per (message precision, max check
// degree DC, max fault degree DV), selected by QL_MSG_F16, QL_DC and QL_DV.
#include <cuda_fp16.h>

#include "qldpc_internal.h"

#ifndef QL_MSG_F16
#define QL_MSG_F16 0
#endif
#ifndef QL_DC
#define QL_DC 8
#endif
#ifndef QL_DV
#define QL_DV 4
#endif

namespace qldpc {
namespace {

constexpr unsigned FULL = 0xffffffffu;

template <typename MT>
struct Msg;
template <>
struct Msg<float> {
    static __device__ __forceinline__ float ld(const float *p) { return *p; }
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};
template <>
struct Msg<__half> {
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
};

__device__ __forceinline__ float clampc(float x, float c) { return fminf(fmaxf(x, -c), c); }

// Per-fault edge list: DV slot indices, the first one carrying the fault degree
// in its top byte (slot indices are below 2^24).
template <int DV>
__device__ __forceinline__ int load_slots(const FusedGraph &g, int j, int (&sl)[DV]) {
    const int4 *p = reinterpret_cast<const int4 *>(g.var_slot + (size_t)j * DV);
    const int4 v = __ldg(p);
    sl[0] = v.x & 0xffffff;
    sl[1] = v.y;
    sl[2] = v.z;
    sl[3] = v.w;
    const int deg = (int)((unsigned)v.x >> 24);
#pragma unroll
    for (int q = 1; q < DV / 4; ++q) {
        if (deg > 4 * q) {
            const int4 u = __ldg(p + q);
            sl[4 * q] = u.x;
            sl[4 * q + 1] = u.y;
            sl[4 * q + 2] = u.z;
            sl[4 * q + 3] = u.w;
        } else {
            sl[4 * q] = sl[4 * q + 1] = sl[4 * q + 2] = sl[4 * q + 3] = 0;
        }
    }
    return deg;
}

// Messages are stored with zeros canonicalised to +0 (x + 0 = x for x != 0 and
// -0 + 0 = +0), so that the check pass may take the sign of a stored message from
// its sign bit: sign(x) = -1 iff x < 0 then holds bit for bit.
__device__ __forceinline__ float canon(float x) { return __fadd_rn(x, 0.0f); }

// Start of a leg: lambda(0), Lambda(0), nu(0) and the leg's memory strengths.
//   leg 0:  lambda(0) = Lambda(0) = w
//   leg r:  Lambda(0) = previous terminal marginals; lambda(0) = Lambda(0)
//           (warm_mode 0) or w (warm_mode 1); nu(0) = lambda(0)
// bb holds (1 - gamma_j) * lambda_j(0), rounded, which is the first product of
// the memory update and is constant within a leg.
template <typename MT, int NT, int VPT, int DV>
__device__ __forceinline__ void leg_init(const FusedGraph &g, const DevParams &p, int leg, MT *msg,
                                         float (&Lam)[VPT], float (&bb)[VPT], float (&gg)[VPT]) {
    const float *grow = g.gamma + (size_t)leg * g.N;
#pragma unroll
    for (int r = 0; r < VPT; ++r) {
        const int j = threadIdx.x + r * NT;
        if (j < g.N) {
            const float lam0 = (leg == 0 || p.warm_mode == 1) ? __ldg(g.w + j) : Lam[r];
            if (leg == 0) Lam[r] = lam0;
            const float gm = __ldg(grow + j);
            gg[r] = gm;
            bb[r] = __fmul_rn(__fsub_rn(1.0f, gm), lam0);
            int sl[DV];
            const int deg = load_slots<DV>(g, j, sl);
            const float nu0 = canon(lam0);
#pragma unroll
            for (int k = 0; k < DV; ++k)
                if (k < deg) Msg<MT>::st(msg + sl[k], nu0);
        }
    }
}

// Check pass, float32 messages: mu_{i->j}(t) from nu(t-1) for every check, in place.
// (m1, m2) = the two smallest magnitudes of the check's slots (with multiplicity),
// so the min over the excluded set of slot k is m2 if |nu_k| = m1, else m1.
// Padding slots hold C, which is also the min over an empty set, and are never
// written.  The sign is (-1)^sigma_i times the product of all signs times sign(nu_k).
template <int NT, int DC>
__device__ __forceinline__ void check_pass(const FusedGraph &g, float *msg, const uint32_t *sg,
                                           float C) {
    for (int i = threadIdx.x; i < g.M; i += NT) {
        const int deg = g.chk_deg[i];
        uint32_t sx = sg[i >> 5] << (31 - (i & 31));
        float v[DC];
#pragma unroll
        for (int k = 0; k < DC; ++k) v[k] = msg[k * g.Mp + i];
        float m1 = C, m2 = C;
#pragma unroll
        for (int k = 0; k < DC; ++k) {
            const float a = fabsf(v[k]);
            m2 = fminf(m2, fmaxf(m1, a));
            m1 = fminf(m1, a);
            sx ^= __float_as_uint(v[k]);
        }
        sx &= 0x80000000u;
#pragma unroll
        for (int k = 0; k < DC; ++k) {
            if (k < deg) {
                const float mag = (fabsf(v[k]) <= m1) ? m2 : m1;
                msg[k * g.Mp + i] = __uint_as_float(__float_as_uint(mag) |
                                                    ((sx ^ __float_as_uint(v[k])) & 0x80000000u));
            }
        }
    }
}

// Check pass, binary16 messages: two checks (2q, 2q+1) per thread with half2
// arithmetic (min, max and sign manipulation are exact in any format).  A 32-bit
// word of slot k holds both checks; a per-pair mask keeps C in padding lanes.
template <int NT, int DC>
__device__ __forceinline__ void check_pass(const FusedGraph &g, __half *msg, const uint32_t *sg,
                                           float C) {
    uint32_t *w32 = reinterpret_cast<uint32_t *>(msg);
    const int Mp2 = g.Mp >> 1, M2 = (g.M + 1) >> 1;
    const __half2 C2 = __float2half2_rn(C);
    const uint32_t c2 = *reinterpret_cast<const uint32_t *>(&C2);
    for (int q = threadIdx.x; q < M2; q += NT) {
        const int i = 2 * q;
        const uint32_t sb = (sg[i >> 5] >> (i & 31)) & 3u;
        uint32_t sx = ((sb & 1u) << 15) | ((sb & 2u) << 30);
        uint32_t v[DC];
#pragma unroll
        for (int k = 0; k < DC; ++k) v[k] = w32[k * Mp2 + q];
        __half2 m1 = C2, m2 = C2;
#pragma unroll
        for (int k = 0; k < DC; ++k) {
            const __half2 a = __habs2(*reinterpret_cast<const __half2 *>(&v[k]));
            m2 = __hmin2(m2, __hmax2(m1, a));
            m1 = __hmin2(m1, a);
            sx ^= v[k];
        }
        sx &= 0x80008000u;
        const uint32_t u1 = *reinterpret_cast<const uint32_t *>(&m1);
        const uint32_t u2 = *reinterpret_cast<const uint32_t *>(&m2);
        const uint4 *pm4 = reinterpret_cast<const uint4 *>(g.pad_mask + (size_t)q * DC);
        uint32_t pm[DC];
#pragma unroll
        for (int k4 = 0; k4 < DC / 4; ++k4) {
            const uint4 t = __ldg(pm4 + k4);
            pm[4 * k4] = t.x;
            pm[4 * k4 + 1] = t.y;
            pm[4 * k4 + 2] = t.z;
            pm[4 * k4 + 3] = t.w;
        }
#pragma unroll
        for (int k = 0; k < DC; ++k) {
            const __half2 a = __habs2(*reinterpret_cast<const __half2 *>(&v[k]));
            const uint32_t eq = __hle2_mask(a, m1);
            const uint32_t mag = (u2 & eq) | (u1 & ~eq);
            const uint32_t o = mag | ((sx ^ v[k]) & 0x80008000u);
            w32[k * Mp2 + q] = (o & ~pm[k]) | (c2 & pm[k]);
        }
    }
}

// Fault update for one fault: memory term, marginal, excluded sums (increasing check
// order, one rounding per addition, exactly as written in the oracle).
template <typename MT, int DV>
__device__ __forceinline__ float fault_update(MT *msg, const int (&sl)[DV], int deg, float lam,
                                              float C) {
    if (deg == 3) {
        const float mu0 = Msg<MT>::ld(msg + sl[0]), mu1 = Msg<MT>::ld(msg + sl[1]),
                    mu2 = Msg<MT>::ld(msg + sl[2]);
        const float s0 = __fadd_rn(lam, mu0), s01 = __fadd_rn(s0, mu1);
        Msg<MT>::st(msg + sl[0], canon(clampc(__fadd_rn(__fadd_rn(lam, mu1), mu2), C)));
        Msg<MT>::st(msg + sl[1], canon(clampc(__fadd_rn(s0, mu2), C)));
        Msg<MT>::st(msg + sl[2], canon(clampc(s01, C)));
        return clampc(__fadd_rn(s01, mu2), C);
    }
    if (deg == 2) {
        const float mu0 = Msg<MT>::ld(msg + sl[0]), mu1 = Msg<MT>::ld(msg + sl[1]);
        const float s0 = __fadd_rn(lam, mu0);
        Msg<MT>::st(msg + sl[0], canon(clampc(__fadd_rn(lam, mu1), C)));
        Msg<MT>::st(msg + sl[1], canon(clampc(s0, C)));
        return clampc(__fadd_rn(s0, mu1), C);
    }
    float mu[DV];
#pragma unroll
    for (int k = 0; k < DV; ++k) mu[k] = (k < deg) ? Msg<MT>::ld(msg + sl[k]) : 0.0f;
    float L = lam;
#pragma unroll
    for (int k = 0; k < DV; ++k)
        if (k < deg) L = __fadd_rn(L, mu[k]);
#pragma unroll
    for (int k = 0; k < DV; ++k) {
        if (k < deg) {
            float v = lam;
#pragma unroll
            for (int k2 = 0; k2 < DV; ++k2)
                if (k2 != k && k2 < deg) v = __fadd_rn(v, mu[k2]);
            Msg<MT>::st(msg + sl[k], canon(clampc(v, C)));
        }
    }
    return clampc(L, C);
}

// Fault pass: memory update, marginals, fault->check messages, decisions into the bitmap.
template <typename MT, int NT, int VPT, int DV>
__device__ __forceinline__ void fault_pass(const FusedGraph &g, MT *msg, uint32_t *fw,
                                           float (&Lam)[VPT], const float (&bb)[VPT],
                                           const float (&gg)[VPT], float C) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < VPT; ++r) {
        const int j = threadIdx.x + r * NT;
        const bool valid = j < g.N;
        float L = 0.0f;
        if (valid) {
            const float lam = __fadd_rn(bb[r], __fmul_rn(gg[r], Lam[r]));
            int sl[DV];
            const int deg = load_slots<DV>(g, j, sl);
            L = fault_update<MT, DV>(msg, sl, deg, lam, C);
            Lam[r] = L;
        }
        const uint32_t bal = __ballot_sync(FULL, valid && L < 0.0f);
        const int jb = threadIdx.x - lane + r * NT;
        if (lane == 0 && jb < g.N) fw[jb >> 5] = bal;
    }
}

// H F = sigma ?  Returns true (in every thread) when some check is unsatisfied.
// Padding slots name fault N, whose decision bit is always 0.
template <int NT, int DC>
__device__ __forceinline__ bool syndrome_unsat(const FusedGraph &g, const uint32_t *fw,
                                               const uint32_t *sg) {
    uint32_t bad = 0;
    for (int i = threadIdx.x; i < g.M; i += NT) {
        uint32_t par = sg[i >> 5] >> (i & 31);
        const int4 *c4 = reinterpret_cast<const int4 *>(g.chk_col + (size_t)i * DC);
#pragma unroll
        for (int q = 0; q < DC / 4; ++q) {
            const int4 c = __ldg(c4 + q);
            const uint32_t wx = fw[c.x >> 5], wy = fw[c.y >> 5], wz = fw[c.z >> 5],
                           ww = fw[c.w >> 5];
            par ^= __funnelshift_r(wx, wx, c.x) ^ __funnelshift_r(wy, wy, c.y) ^
                   __funnelshift_r(wz, wz, c.z) ^ __funnelshift_r(ww, ww, c.w);
        }
        bad |= par & 1u;
    }
    return __syncthreads_or(bad) != 0;
}

// W = sum_j F_j w_j in increasing j, one rounding per addition (called by one
// whole warp; every lane returns the same value).
__device__ __forceinline__ float solution_weight(const FusedGraph &g, const uint32_t *fw) {
    const int lane = threadIdx.x & 31;
    const int nw = (g.N + 31) >> 5;
    float W = 0.0f;
    for (int q0 = 0; q0 < nw; q0 += 32) {
        const uint32_t mine = (q0 + lane < nw) ? fw[q0 + lane] : 0u;
        uint32_t any = __ballot_sync(FULL, mine != 0u);
        while (any) {
            const int l = __ffs(any) - 1;
            any &= any - 1;
            uint32_t wd = __shfl_sync(FULL, mine, l);
            while (wd) {
                const int b = __ffs(wd) - 1;
                wd &= wd - 1;
                W = __fadd_rn(W, __ldg(g.w + ((q0 + l) << 5) + b));
            }
        }
    }
    return W;
}

template <int NT>
__device__ __forceinline__ void store_bits(uint64_t *dst, const uint32_t *fw, int words) {
    for (int q = threadIdx.x; q < words; q += NT)
        dst[q] = (uint64_t)fw[2 * q] | ((uint64_t)fw[2 * q + 1] << 32);
}

template <typename MT, int DC>
__device__ __forceinline__ void smem_layout(const FusedGraph &g, unsigned char *raw, MT *&msg,
                                            uint32_t *&fw, uint32_t *&sg) {
    msg = reinterpret_cast<MT *>(raw);
    const size_t mb = ((size_t)DC * g.Mp * sizeof(MT) + 15) & ~(size_t)15;
    fw = reinterpret_cast<uint32_t *>(raw + mb);
    sg = fw + g.f_words;
}

template <typename MT, int NT, int DC>
__device__ __forceinline__ void block_setup(const FusedGraph &g, MT *msg, uint32_t *fw, float C) {
    for (int q = threadIdx.x; q < g.f_words; q += NT) fw[q] = 0u;
    for (int i = threadIdx.x; i < g.Mp; i += NT) {
        const int deg = g.chk_deg[i];
        for (int k = deg; k < DC; ++k) Msg<MT>::st(msg + k * g.Mp + i, C);
    }
}

template <int NT>
__device__ __forceinline__ void load_syndrome(const FusedGraph &g, const uint64_t *sy,
                                              uint32_t *sg) {
    for (int q = threadIdx.x; q < g.syn_words; q += NT) {
        const uint64_t v = __ldg(sy + q);
        sg[2 * q] = (uint32_t)v;
        sg[2 * q + 1] = (uint32_t)(v >> 32);
    }
}

template <typename MT, int NT, int VPT, int MINB, int DC, int DV>
__global__ void __launch_bounds__(NT, MINB) fused_decode(FusedGraph g, DevParams p,
                                                   const uint64_t *__restrict__ syn, int B,
                                                   DecodeOut out, unsigned int *counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MT *msg;
    uint32_t *fw, *sg;
    smem_layout<MT, DC>(g, smem_raw, msg, fw, sg);
    __shared__ int s_shot;
    __shared__ float s_W;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float C = p.clip;
    block_setup<MT, NT, DC>(g, msg, fw, C);

    float Lam[VPT], bb[VPT], gg[VPT];
#pragma unroll
    for (int r = 0; r < VPT; ++r) Lam[r] = bb[r] = gg[r] = 0.0f;

    for (;;) {
        __syncthreads();  // the previous shot is done with shared memory and s_shot
        if (tid == 0) s_shot = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int shot = s_shot;
        if (shot >= B) break;
        load_syndrome<NT>(g, syn + (size_t)shot * g.syn_words, sg);
        uint64_t *cor = out.corr + (size_t)shot * g.cor_words;

        int leg = 0, sols = 0;
        long long iters = 0;
        bool have = false;
        float Wbest = 0.0f;
        leg_init<MT, NT, VPT, DV>(g, p, 0, msg, Lam, bb, gg);
        __syncthreads();
        for (;;) {
            const int T = leg == 0 ? p.T1 : p.T2;
            for (int t = 1; t <= T; ++t) {
                check_pass<NT, DC>(g, msg, sg, C);
                __syncthreads();
                fault_pass<MT, NT, VPT, DV>(g, msg, fw, Lam, bb, gg, C);
                __syncthreads();
                ++iters;
                if (!syndrome_unsat<NT, DC>(g, fw, sg)) {
                    if (warp == 0) {
                        const float W = solution_weight(g, fw);
                        if (lane == 0) s_W = W;
                    }
                    __syncthreads();
                    const float W = s_W;
                    if (!have || W < Wbest) {
                        store_bits<NT>(cor, fw, g.cor_words);
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
            leg_init<MT, NT, VPT, DV>(g, p, leg, msg, Lam, bb, gg);
            __syncthreads();
        }
        if (!have) store_bits<NT>(cor, fw, g.cor_words);
        if (tid == 0) {
            if (out.legs) out.legs[shot] = leg + 1;
            if (out.conv) out.conv[shot] = have ? 1 : 0;
            if (out.iters) out.iters[shot] = (int32_t)iters;
        }
    }
}

// First leg without early exit, every iteration recorded (one shot per block).
template <typename MT, int NT, int VPT, int DC, int DV>
__global__ void __launch_bounds__(NT) fused_trace(FusedGraph g, DevParams p,
                                                  const uint64_t *__restrict__ syn, int B, int T,
                                                  int E, float *marg, float *nu, float *mu) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MT *msg;
    uint32_t *fw, *sg;
    smem_layout<MT, DC>(g, smem_raw, msg, fw, sg);
    const int shot = blockIdx.x;
    const float C = p.clip;
    block_setup<MT, NT, DC>(g, msg, fw, C);
    load_syndrome<NT>(g, syn + (size_t)shot * g.syn_words, sg);
    float Lam[VPT], bb[VPT], gg[VPT];
#pragma unroll
    for (int r = 0; r < VPT; ++r) Lam[r] = bb[r] = gg[r] = 0.0f;
    __syncthreads();
    leg_init<MT, NT, VPT, DV>(g, p, 0, msg, Lam, bb, gg);
    __syncthreads();
    const int nslots = DC * g.Mp;
    for (int t = 0; t < T; ++t) {
        const size_t o = (size_t)t * B + shot;
        check_pass<NT, DC>(g, msg, sg, C);
        __syncthreads();
        if (mu)
            for (int s = threadIdx.x; s < nslots; s += NT) {
                const int e = g.slot_edge[s];
                if (e >= 0) mu[o * E + e] = Msg<MT>::ld(msg + s);
            }
        __syncthreads();
        fault_pass<MT, NT, VPT, DV>(g, msg, fw, Lam, bb, gg, C);
        __syncthreads();
        if (marg) {
#pragma unroll
            for (int r = 0; r < VPT; ++r) {
                const int j = threadIdx.x + r * NT;
                if (j < g.N) marg[o * g.N + j] = Lam[r];
            }
        }
        if (nu)
            for (int s = threadIdx.x; s < nslots; s += NT) {
                const int e = g.slot_edge[s];
                if (e >= 0) nu[o * E + e] = Msg<MT>::ld(msg + s);
            }
        __syncthreads();
    }
}

template <typename MT, int NT, int VPT, int MINB, int DC, int DV>
cudaError_t launch_decode(dim3 grid, size_t smem, cudaStream_t st, const FusedGraph &g,
                          const DevParams &p, const uint64_t *syn, int B, DecodeOut out,
                          unsigned int *counter) {
    fused_decode<MT, NT, VPT, MINB, DC, DV><<<grid, NT, smem, st>>>(g, p, syn, B, out, counter);
    return cudaGetLastError();
}

template <typename MT, int NT, int VPT, int DC, int DV>
cudaError_t launch_trace(dim3 grid, size_t smem, cudaStream_t st, const FusedGraph &g,
                         const DevParams &p, const uint64_t *syn, int B, int T, float *marg,
                         float *nu, float *mu) {
    fused_trace<MT, NT, VPT, DC, DV><<<grid, NT, smem, st>>>(g, p, syn, B, T, g.E, marg, nu, mu);
    return cudaGetLastError();
}

#if QL_MSG_F16
using MsgT = __half;
#else
using MsgT = float;
#endif

template <int NT, int VPT, int MINB, bool TRACE>
FusedKernel entry() {
    FusedKernel k;
    k.msg_fp16 = QL_MSG_F16;
    k.threads = NT;
    k.min_blocks = MINB;
    k.vpt = VPT;
    k.dc = QL_DC;
    k.dv = QL_DV;
    k.decode_fn = (const void *)fused_decode<MsgT, NT, VPT, MINB, QL_DC, QL_DV>;
    k.launch_decode = &launch_decode<MsgT, NT, VPT, MINB, QL_DC, QL_DV>;
    if constexpr (TRACE) {
        k.trace_fn = (const void *)fused_trace<MsgT, NT, VPT, QL_DC, QL_DV>;
        k.launch_trace = &launch_trace<MsgT, NT, VPT, QL_DC, QL_DV>;
    } else {
        k.trace_fn = nullptr;
        k.launch_trace = nullptr;
    }
    return k;
}

}  // namespace

#define QL_CAT2(P, DC, DV) fused_table_##P##_##DC##_##DV
#define QL_EXPAND(P, DC, DV) QL_CAT2(P, DC, DV)
#if QL_MSG_F16
#define QL_P f16
#else
#define QL_P f32
#endif

void QL_EXPAND(QL_P, QL_DC, QL_DV)(const FusedKernel **out, int *n) {
    // (threads, faults per thread, min resident blocks): the first entry whose
    // threads * vpt >= N is used unless the caller asks for a block size; the last
    // entry also serves the trace kernel.
    static const FusedKernel table[] = {
        entry<256, 4, 4, false>(),
        entry<512, 6, 2, false>(),
        entry<256, 12, 3, false>(),
        entry<512, 16, 1, false>(),
        entry<512, 32, 1, true>(),
    };
    *out = table;
    *n = (int)(sizeof(table) / sizeof(table[0]));
}

}  // namespace qldpc
