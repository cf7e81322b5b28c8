// Device building blocks of the fused Relay-BP kernels (paper Sec. 2.3, "Relay
// decoding"): message access, the check pass, the fault pass with decisions and
// syndrome parity, convergence and weight reductions, leg initialisation and the
// shared-memory layout.  Included by the Relay kernels and by the filtered-OSD
// kernel, whose plain-BP stage is the same passes with every gamma_j = 0.
#pragma once

#include <cuda_fp16.h>

#include "qldpc_internal.h"

namespace qldpc {
namespace {

constexpr unsigned FULL = 0xffffffffu;

template <typename MT>
struct Msg;
template <>
struct Msg<float> {
    static __device__ __forceinline__ float ld(const unsigned char *base, int off) {
        return *reinterpret_cast<const float *>(base + off);
    }
    static __device__ __forceinline__ void st(unsigned char *base, int off, float v) {
        *reinterpret_cast<float *>(base + off) = v;
    }
};
template <>
struct Msg<__half> {
    static __device__ __forceinline__ float ld(const unsigned char *base, int off) {
        return __half2float(*reinterpret_cast<const __half *>(base + off));
    }
    static __device__ __forceinline__ void st(unsigned char *base, int off, float v) {
        *reinterpret_cast<__half *>(base + off) = __float2half_rn(v);
    }
};

__device__ __forceinline__ float clampc(float x, float c) { return fminf(fmaxf(x, -c), c); }

// Binary16 store with saturation at the largest finite value, 65504: for every finite x
// it equals rounding min(max(x, -65504), 65504) to nearest, i.e. the clamp to C = 65504
// followed by the store.
__device__ __forceinline__ void st_half_sat(unsigned char *base, int off, float v) {
    unsigned short h;
    asm("cvt.rn.satfinite.f16.f32 %0, %1;" : "=h"(h) : "f"(v));
    *reinterpret_cast<unsigned short *>(base + off) = h;
}

__device__ __forceinline__ unsigned short ld_half_bits(const unsigned char *base, int off) {
    return *reinterpret_cast<const unsigned short *>(base + off);
}

// x + h for a binary16 operand h in one float32 addition (the widening of h is exact,
// so this is __fadd_rn(x, __half2float(h)) without a separate conversion).
__device__ __forceinline__ float add_f16(float x, unsigned short h) {
    float d;
    asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(h), "f"(x));
    return d;
}

// x + 0 = x for x != 0 and -0 + 0 = +0.  Applied to lambda(0) and to
// (1 - gamma) lambda(0) at the start of a leg, it guarantees that lambda(t) and
// therefore every stored message nu (a sum starting from lambda(t)) is never -0,
// so the check pass may read sign(nu) = -1 iff nu < 0 straight off the sign bit.
// A zero's sign never changes a comparison or a non-zero result, so this leaves
// every decision and every non-zero value as in the oracle.
__device__ __forceinline__ float canon(float x) { return __fadd_rn(x, 0.0f); }

// Weight of a decided fault in 2^-33 units, from the float's fields with integer
// operations only: |w| = m * 2^(e-23) -> m * 2^(e+10).  Exact for |w| >= 2^-10
// (smaller magnitudes are truncated); |w| < 2^20 keeps it below 2^54.
__device__ __forceinline__ long long wfix(float w) {
    const uint32_t b = __float_as_uint(w);
    const int e = (int)((b >> 23) & 0xffu) - 127;
    const long long m = (long long)((b & 0x7fffffu) | 0x800000u);
    const long long a = e >= -10 ? (m << (e + 10)) : (e > -34 ? (m >> (-10 - e)) : 0ll);
    return (b >> 31) ? -a : a;
}

// Per-fault edge list: DV byte offsets of the fault's slots (increasing check
// order); entry 0 carries the fault degree in its top byte.
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

// Swizzle of the slots inside a check (or check pair): physical position p holds
// logical slot p ^ swz(i); with 32/DC checks per 128-byte row, this spreads a
// fixed logical slot of 32 consecutive rows over 32 banks.
template <int DC>
__device__ __forceinline__ int swz(int i) {
    constexpr int sh = DC >= 32 ? 0 : (DC == 16 ? 1 : 2);
    return (i >> sh) & (DC - 1);
}

// Start of a leg: lambda(0), Lambda(0), nu(0) and the leg's memory strengths.
//   leg 0:  lambda(0) = Lambda(0) = w
//   leg r:  Lambda(0) = previous terminal marginals; lambda(0) = Lambda(0)
//           (warm_mode 0) or w (warm_mode 1); nu(0) = lambda(0)
// bb holds (1 - gamma_j) * lambda_j(0), rounded, which is the first product of
// the memory update and is constant within a leg.
template <typename MT, int NT, int VPT, int DV, bool SKIP = false>
__device__ __forceinline__ void leg_init(const FusedGraph &g, const DevParams &p, int leg,
                                         unsigned char *msg, const float *ws, float (&Lam)[VPT],
                                         float (&bb)[VPT], float (&gg)[VPT]) {
    const float *grow = g.gamma + (size_t)leg * g.N;
#pragma unroll
    for (int r = 0; r < VPT; ++r) {
        if (SKIP && r * NT >= g.N) break;  // the block's remaining fault slots are empty
        const int j = threadIdx.x + r * NT;
        if (j < g.N) {
            const float lam0 = canon((leg == 0 || p.warm_mode == 1) ? ws[j] : Lam[r]);
            if (leg == 0) Lam[r] = lam0;
            const float gm = __ldg(grow + j);
            gg[r] = gm;
            bb[r] = canon(__fmul_rn(__fsub_rn(1.0f, gm), lam0));
            int sl[DV];
            const int deg = load_slots<DV>(g, j, sl);
#pragma unroll
            for (int k = 0; k < DV; ++k)
                if (k < deg) Msg<MT>::st(msg, sl[k], lam0);
        }
    }
}

// Two smallest of n values (with multiplicity) by a pairwise tree: sorted pairs, then
// merges of sorted pairs, (l, h) = (min(l1, l2), min(max(l1, l2), min(h1, h2))).  min
// and max are exact, so the result is the one a sequential scan gives, in log2(n)
// dependent steps instead of n.  V is float or __half2 (two checks at once).
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ __half2 vmin(__half2 a, __half2 b) { return __hmin2(a, b); }
__device__ __forceinline__ __half2 vmax(__half2 a, __half2 b) { return __hmax2(a, b); }

// Rows wider than 8 slots keep the sequential scan (the tree's live values would spill).
template <int n, typename V>
__device__ __forceinline__ void two_smallest(const V (&a)[n], V &m1, V &m2) {
    static_assert(n >= 2 && (n & (n - 1)) == 0, "power-of-two row capacity");
    if constexpr (n > 8) {
        m1 = vmin(a[0], a[1]);
        m2 = vmax(a[0], a[1]);
#pragma unroll
        for (int k = 2; k < n; ++k) {
            m2 = vmin(m2, vmax(m1, a[k]));
            m1 = vmin(m1, a[k]);
        }
        return;
    }
    V lo[n / 2], hi[n / 2];
#pragma unroll
    for (int k = 0; k < n / 2; ++k) {
        lo[k] = vmin(a[2 * k], a[2 * k + 1]);
        hi[k] = vmax(a[2 * k], a[2 * k + 1]);
    }
#pragma unroll
    for (int w = n / 2; w > 1; w >>= 1) {
#pragma unroll
        for (int k = 0; k < w / 2; ++k) {
            const V l = vmin(lo[2 * k], lo[2 * k + 1]);
            hi[k] = vmin(vmax(lo[2 * k], lo[2 * k + 1]), vmin(hi[2 * k], hi[2 * k + 1]));
            lo[k] = l;
        }
    }
    m1 = lo[0];
    m2 = hi[0];
}

// Check pass, float32 messages: mu_{i->j}(t) from nu(t-1) for every check, in place.
// (m1, m2) = the two smallest magnitudes of the check's slots (with multiplicity) and
// of {C, C}, so the min over the excluded set of slot k is m2 if |nu_k| = m1, else m1.
// Padding slots hold C, which is also the min over an empty set, and keep it.
// The sign is (-1)^sigma_i times the product of all signs times sign(nu_k).
// Slots are processed in physical order: the rule does not depend on the order.
// Lanes read and write their row's 16-byte chunks in the order k4 ^ cs: rows are
// 4*DC bytes apart, and cs = (row / rows per 128-byte line) mod chunks per row makes
// each 128-bit access of a warp touch every bank equally often (no bank conflict).
template <int NT, int DC>
__device__ __forceinline__ void check_pass(const FusedGraph &g, float *msg, const uint32_t *sg,
                                           uint32_t *par_zero, float C) {
    for (int q = threadIdx.x; q < g.m_words; q += NT) par_zero[q] = 0u;
    for (int i = threadIdx.x; i < g.M; i += NT) {
        const int deg = g.chk_deg[i];
        uint32_t sx = sg[i >> 5] << (31 - (i & 31));
        float4 *row = reinterpret_cast<float4 *>(msg + (size_t)i * DC);
        const int cs = (i / (DC >= 32 ? 1 : 32 / DC)) & (DC / 4 - 1);  // chunk order
        float v[DC];
#pragma unroll
        for (int k4 = 0; k4 < DC / 4; ++k4) {
            const float4 t = row[k4 ^ cs];
            v[4 * k4] = t.x;
            v[4 * k4 + 1] = t.y;
            v[4 * k4 + 2] = t.z;
            v[4 * k4 + 3] = t.w;
        }
        float a[DC], m1, m2;
        uint32_t x[DC / 2];
#pragma unroll
        for (int k = 0; k < DC; ++k) a[k] = fabsf(v[k]);
        two_smallest<DC>(a, m1, m2);
        m1 = fminf(m1, C);
        m2 = fminf(m2, C);
#pragma unroll
        for (int k = 0; k < DC / 2; ++k)
            x[k] = __float_as_uint(v[2 * k]) ^ __float_as_uint(v[2 * k + 1]);
#pragma unroll
        for (int w = DC / 2; w > 1; w >>= 1)
#pragma unroll
            for (int k = 0; k < w / 2; ++k) x[k] = x[2 * k] ^ x[2 * k + 1];
        sx = (sx ^ x[0]) & 0x80000000u;
        // Slot k holds a smallest magnitude iff |nu_k| <= m1 (no |nu_k| is below m1);
        // its excluded minimum is then m2 (= m1 on a tie), else m1.  Both candidates
        // carry the sign of the whole product; one XOR takes the slot's own sign out.
        const uint32_t s1 = __float_as_uint(m1) | sx, s2 = __float_as_uint(m2) | sx;
        float o[DC];
#pragma unroll
        for (int k = 0; k < DC; ++k) {
            const uint32_t c = a[k] <= m1 ? s2 : s1;
            o[k] = __uint_as_float(c ^ (__float_as_uint(v[k]) & 0x80000000u));
        }
        if (deg < DC) {  // v[k] is physical slot k ^ 4cs, logical slot k ^ 4cs ^ swz(i)
            const int f = swz<DC>(i) ^ (cs << 2);
#pragma unroll
            for (int k = 0; k < DC; ++k)
                if ((k ^ f) >= deg) o[k] = C;
        }
#pragma unroll
        for (int k4 = 0; k4 < DC / 4; ++k4)
            row[k4 ^ cs] = make_float4(o[4 * k4], o[4 * k4 + 1], o[4 * k4 + 2], o[4 * k4 + 3]);
    }
}

// Check pass, binary16 messages: checks 2q and 2q+1 share each 32-bit word (low
// and high half), processed together with half2 arithmetic; min, max and sign
// manipulation are exact in any format.  A per-pair mask keeps C in padding halves.
// Row chunks are visited in the order k4 ^ cs as in the float32 pass (rows of check
// pairs are 4*DC bytes apart too); only the padding mask follows the order.
template <int NT, int DC>
__device__ __forceinline__ void check_pass(const FusedGraph &g, __half *msg, const uint32_t *sg,
                                           uint32_t *par_zero, float C) {
    for (int q = threadIdx.x; q < g.m_words; q += NT) par_zero[q] = 0u;
    const __half2 C2 = __float2half2_rn(C);
    const uint32_t c2 = *reinterpret_cast<const uint32_t *>(&C2);
    const int M2 = (g.M + 1) >> 1;
    for (int q = threadIdx.x; q < M2; q += NT) {
        const int i = 2 * q;
        const uint32_t sb = (sg[i >> 5] >> (i & 31)) & 3u;
        uint32_t sx = ((sb & 1u) << 15) | ((sb & 2u) << 30);
        const bool full = g.chk_deg[i] == DC && g.chk_deg[i + 1] == DC;
        uint4 *row = reinterpret_cast<uint4 *>(msg + (size_t)q * 2 * DC);
        const int cs = (q / (DC >= 32 ? 1 : 32 / DC)) & (DC / 4 - 1);
        uint32_t v[DC];
#pragma unroll
        for (int k4 = 0; k4 < DC / 4; ++k4) {
            const uint4 t = row[k4 ^ cs];
            v[4 * k4] = t.x;
            v[4 * k4 + 1] = t.y;
            v[4 * k4 + 2] = t.z;
            v[4 * k4 + 3] = t.w;
        }
        __half2 a[DC], m1, m2;
        uint32_t x[DC / 2];
#pragma unroll
        for (int k = 0; k < DC; ++k) a[k] = __habs2(*reinterpret_cast<const __half2 *>(&v[k]));
        two_smallest<DC>(a, m1, m2);
        m1 = __hmin2(m1, C2);
        m2 = __hmin2(m2, C2);
#pragma unroll
        for (int k = 0; k < DC / 2; ++k) x[k] = v[2 * k] ^ v[2 * k + 1];
#pragma unroll
        for (int w = DC / 2; w > 1; w >>= 1)
#pragma unroll
            for (int k = 0; k < w / 2; ++k) x[k] = x[2 * k] ^ x[2 * k + 1];
        sx = (sx ^ x[0]) & 0x80008000u;
        const uint32_t u1 = *reinterpret_cast<const uint32_t *>(&m1);
        const uint32_t u2 = *reinterpret_cast<const uint32_t *>(&m2);
        const uint32_t s1 = u1 | sx, s2 = u2 | sx;  // candidates with the product's sign
        uint32_t o[DC];
#pragma unroll
        for (int k = 0; k < DC; ++k) {
            const uint32_t eq = __hle2_mask(a[k], m1);
            o[k] = ((s2 & eq) | (s1 & ~eq)) ^ (v[k] & 0x80008000u);
        }
        if (!full) {
            const uint4 *pm4 = reinterpret_cast<const uint4 *>(g.pad_mask + (size_t)q * DC);
#pragma unroll
            for (int k4 = 0; k4 < DC / 4; ++k4) {
                const uint4 t = __ldg(pm4 + (k4 ^ cs));
                o[4 * k4] = (o[4 * k4] & ~t.x) | (c2 & t.x);
                o[4 * k4 + 1] = (o[4 * k4 + 1] & ~t.y) | (c2 & t.y);
                o[4 * k4 + 2] = (o[4 * k4 + 2] & ~t.z) | (c2 & t.z);
                o[4 * k4 + 3] = (o[4 * k4 + 3] & ~t.w) | (c2 & t.w);
            }
        }
#pragma unroll
        for (int k4 = 0; k4 < DC / 4; ++k4)
            row[k4 ^ cs] = make_uint4(o[4 * k4], o[4 * k4 + 1], o[4 * k4 + 2], o[4 * k4 + 3]);
    }
}

// Fault update for one fault: memory term, marginal, excluded sums (increasing check
// order, one rounding per addition, exactly as written in the oracle).
template <typename MT, int DV>
__device__ __forceinline__ float fault_update(unsigned char *msg, const int (&sl)[DV], int deg,
                                              float lam, float C) {
    // binary16 storage with C = 65504 (its default): the saturating store clamps the
    // messages, so only the marginal needs an explicit clamp
    // the binary16 operands enter the float32 sums through mixed-precision additions
    if constexpr (sizeof(MT) == 2) {
        if (C == 65504.0f && (deg == 3 || deg == 2)) {
            const unsigned short mu0 = ld_half_bits(msg, sl[0]), mu1 = ld_half_bits(msg, sl[1]);
            const float s0 = add_f16(lam, mu0);
            if (deg == 3) {
                const unsigned short mu2 = ld_half_bits(msg, sl[2]);
                const float s01 = add_f16(s0, mu1);
                st_half_sat(msg, sl[0], add_f16(add_f16(lam, mu1), mu2));
                st_half_sat(msg, sl[1], add_f16(s0, mu2));
                st_half_sat(msg, sl[2], s01);
                return clampc(add_f16(s01, mu2), C);
            }
            st_half_sat(msg, sl[0], add_f16(lam, mu1));
            st_half_sat(msg, sl[1], s0);
            return clampc(add_f16(s0, mu1), C);
        }
    }
    // The clamp is the identity unless some value exceeds C in magnitude, so it is
    // applied only then (same values either way).  Binary16 storage with another C takes
    // the generic loop (less code in the persistent kernel; the same sums and clamps).
    if (sizeof(MT) == 4 && deg == 3) {
        const float mu0 = Msg<MT>::ld(msg, sl[0]), mu1 = Msg<MT>::ld(msg, sl[1]),
                    mu2 = Msg<MT>::ld(msg, sl[2]);
        const float s0 = __fadd_rn(lam, mu0), s01 = __fadd_rn(s0, mu1);
        float n0 = __fadd_rn(__fadd_rn(lam, mu1), mu2), n1 = __fadd_rn(s0, mu2), n2 = s01;
        float L = __fadd_rn(s01, mu2);
        if (fmaxf(fmaxf(fabsf(n0), fabsf(n1)), fmaxf(fabsf(n2), fabsf(L))) > C) {
            n0 = clampc(n0, C);
            n1 = clampc(n1, C);
            n2 = clampc(n2, C);
            L = clampc(L, C);
        }
        Msg<MT>::st(msg, sl[0], n0);
        Msg<MT>::st(msg, sl[1], n1);
        Msg<MT>::st(msg, sl[2], n2);
        return L;
    }
    if (sizeof(MT) == 4 && deg == 2) {
        const float mu0 = Msg<MT>::ld(msg, sl[0]), mu1 = Msg<MT>::ld(msg, sl[1]);
        const float s0 = __fadd_rn(lam, mu0);
        float n0 = __fadd_rn(lam, mu1), n1 = s0, L = __fadd_rn(s0, mu1);
        if (fmaxf(fmaxf(fabsf(n0), fabsf(n1)), fabsf(L)) > C) {
            n0 = clampc(n0, C);
            n1 = clampc(n1, C);
            L = clampc(L, C);
        }
        Msg<MT>::st(msg, sl[0], n0);
        Msg<MT>::st(msg, sl[1], n1);
        return L;
    }
    float mu[DV];
#pragma unroll
    for (int k = 0; k < DV; ++k) mu[k] = (k < deg) ? Msg<MT>::ld(msg, sl[k]) : 0.0f;
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
            Msg<MT>::st(msg, sl[k], clampc(v, C));
        }
    }
    return clampc(L, C);
}

// Fault pass: memory update, marginals, fault->check messages, decisions into the
// bitmap fw, and the syndrome of the decision: every fault with F_j = 1 flips the
// parity bits of its checks in par (zeroed by the preceding check pass).  Decisions
// are sparse, so this costs a few atomics per shot instead of a pass over all edges.
// Returns the thread's decided faults (bit r: fault threadIdx.x + r*NT has F_j = 1).
template <typename MT, int NT, int VPT, int DV, bool SKIP = false>
__device__ __forceinline__ uint32_t fault_pass(const FusedGraph &g, unsigned char *msg, uint32_t *fw,
                                           uint32_t *par, float (&Lam)[VPT],
                                           const float (&bb)[VPT], const float (&gg)[VPT],
                                           float C) {
    static_assert(VPT <= 32, "one decision bit per fault of the thread");
    const int lane = threadIdx.x & 31;
    uint32_t dmask = 0u;  // bit r: this thread's fault r is decided (F_j = 1)
#pragma unroll
    for (int r = 0; r < VPT; ++r) {
        if (SKIP && r * NT >= g.N) break;  // the block's remaining fault slots are empty
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
        const bool dec = valid && L < 0.0f;
        const uint32_t bal = __ballot_sync(FULL, dec);
        const int jb = threadIdx.x - lane + r * NT;
        if (lane == 0 && jb < g.N) fw[jb >> 5] = bal;
        dmask |= (dec ? 1u : 0u) << r;
    }
    // Decided faults are few: flip their checks' parity after the loop, so that the
    // per-fault body carries no divergent branch and no live edge state.
    const uint32_t decided = dmask;
    while (dmask) {
        const int r = __ffs(dmask) - 1;
        dmask &= dmask - 1u;
        const int j = threadIdx.x + r * NT;
        const int deg = (int)((uint32_t)__ldg(g.var_slot + (size_t)j * DV) >> 24);
        const int *ck = g.var_chk + (size_t)j * DV;
        for (int k = 0; k < deg; ++k) {
            const int c = __ldg(ck + k);
            atomicXor(par + (c >> 5), 1u << (c & 31));
        }
    }
    return decided;
}

// H F = sigma ?  Each warp compares the parity words with the syndrome on its own
// (no block barrier); every warp reaches the same answer.
__device__ __forceinline__ bool warp_converged(const uint32_t *par, const uint32_t *sg, int nw) {
    uint32_t bad = 0;
    for (int q = threadIdx.x & 31; q < nw; q += 32) bad |= par[q] ^ sg[q];
    return !__any_sync(FULL, bad != 0u);
}

// Adds this thread's share of the solution weight sum_j F_j w_j (2^-33 units) to the
// block's accumulator: only the few threads with decided faults (mask dm from the
// fault pass) issue an atomic.  Integer addition makes the total exact and
// independent of the order.
template <int NT>
__device__ __forceinline__ void add_weight(const float *ws, uint32_t dm, long long *acc) {
    long long w = 0;
    for (uint32_t m = dm; m; m &= m - 1u) w += wfix(ws[threadIdx.x + (__ffs(m) - 1) * NT]);
    if (w != 0)
        atomicAdd(reinterpret_cast<unsigned long long *>(acc), (unsigned long long)w);
}

template <int NT>
__device__ __forceinline__ void store_bits(uint64_t *dst, const uint32_t *fw, int words) {
    for (int q = threadIdx.x; q < words; q += NT)
        dst[q] = (uint64_t)fw[2 * q] | ((uint64_t)fw[2 * q + 1] << 32);
}

// Kept solution: the output row and the shared copy used by warp_same_solution.
template <int NT>
__device__ __forceinline__ void keep_solution(uint64_t *dst, const uint32_t *fw, uint32_t *fb,
                                              int words) {
    for (int q = threadIdx.x; q < words; q += NT) {
        const uint32_t lo = fw[2 * q], hi = fw[2 * q + 1];
        fb[2 * q] = lo;
        fb[2 * q + 1] = hi;
        dst[q] = (uint64_t)lo | ((uint64_t)hi << 32);
    }
}

// Shared memory: messages [msg_bytes], decision bitmap fw [f_words], kept solution
// fb [f_words], syndrome sg [2*syn_words] (bits past M cleared), two parity buffers
// par [2][m_words], prior LLRs ws [N] (read by the weight sum and leg initialisation).
__device__ __forceinline__ void smem_layout(const FusedGraph &g, unsigned char *raw,
                                            uint32_t *&fw, uint32_t *&fb, uint32_t *&sg,
                                            uint32_t *&par, float *&ws) {
    const size_t mb = ((size_t)g.msg_bytes + 15) & ~(size_t)15;
    fw = reinterpret_cast<uint32_t *>(raw + mb);
    fb = fw + g.f_words;
    sg = fb + g.f_words;
    par = sg + 2 * g.syn_words;
    ws = reinterpret_cast<float *>(par + 2 * g.m_words);
}

// Plain min-sum BP (paper Sec. 2.3, "Belief propagation decoding"): DMem-BP with every
// gamma_j = 0, which the graph's gamma row (all zeros) provides, from the priors, for
// `iters` iterations without early exit; the marginals end in Lam.  Re-stages the
// padding slots and priors first (callers reuse the message area between shots).
// Called by every thread of the block.
template <int NT, int VPT, int DC, int DV>
__device__ __forceinline__ void plain_bp(const FusedGraph &g, const DevParams &p, int iters,
                                         const uint64_t *sy, unsigned char *msg, uint32_t *fw,
                                         uint32_t *sg, uint32_t *par, float *ws,
                                         float (&Lam)[VPT], float (&bb)[VPT], float (&gg)[VPT]);

// Is the decision bitmap equal to the kept solution (its first `words` words)?  Each
// warp decides on its own, comparing 128 bits per lane: fw and fb are 16-byte aligned,
// f_words is a multiple of 4 and the words past the last fault are zero in both.
__device__ __forceinline__ bool warp_same_solution(const uint32_t *fw, const uint32_t *fb,
                                                   int words) {
    const uint4 *a = reinterpret_cast<const uint4 *>(fw), *b = reinterpret_cast<const uint4 *>(fb);
    uint32_t diff = 0;
    for (int q = threadIdx.x & 31; 4 * q < words; q += 32) {
        const uint4 x = a[q], y = b[q];
        diff |= (x.x ^ y.x) | (x.y ^ y.y) | (x.z ^ y.z) | (x.w ^ y.w);
    }
    return !__any_sync(FULL, diff != 0u);
}

// Padding slots of every check hold C for good (the check pass writes C back).
template <typename MT, int NT, int DC>
__device__ __forceinline__ void block_setup(const FusedGraph &g, unsigned char *msg, uint32_t *fw,
                                            float *ws, float C) {
    for (int q = threadIdx.x; q < 2 * g.f_words; q += NT) fw[q] = 0u;  // fw and fb
    for (int j = threadIdx.x; j < g.N; j += NT) ws[j] = __ldg(g.w + j);
    for (int i = threadIdx.x; i < g.Mp; i += NT) {
        const int deg = g.chk_deg[i];
        const bool half = sizeof(MT) == 2;
        const int f = half ? swz<DC>(i >> 1) : swz<DC>(i);
        for (int k = deg; k < DC; ++k) {
            const int p = k ^ f;
            const int off = half ? (((i >> 1) * DC + p) * 4 + (i & 1) * 2) : ((i * DC + p) * 4);
            Msg<MT>::st(msg, off, C);
        }
    }
}

template <int NT>
__device__ __forceinline__ void load_syndrome(const FusedGraph &g, const uint64_t *sy,
                                              uint32_t *sg) {
    for (int q = threadIdx.x; q < g.syn_words; q += NT) {
        uint64_t v = __ldg(sy + q);
        const int hi = g.M - 64 * q;  // padding bits of the last word are ignored
        if (hi < 64) v &= (1ull << hi) - 1ull;
        sg[2 * q] = (uint32_t)v;
        sg[2 * q + 1] = (uint32_t)(v >> 32);
    }
}


template <int NT, int VPT, int DC, int DV>
__device__ __forceinline__ void plain_bp(const FusedGraph &g, const DevParams &p, int iters,
                                         const uint64_t *sy, unsigned char *msg, uint32_t *fw,
                                         uint32_t *sg, uint32_t *par, float *ws,
                                         float (&Lam)[VPT], float (&bb)[VPT], float (&gg)[VPT]) {
    block_setup<float, NT, DC>(g, msg, fw, ws, p.clip);
    load_syndrome<NT>(g, sy, sg);
    __syncthreads();
    leg_init<float, NT, VPT, DV>(g, p, 0, msg, ws, Lam, bb, gg);
    __syncthreads();
    for (int t = 0; t < iters; ++t) {
        check_pass<NT, DC>(g, reinterpret_cast<float *>(msg), sg, par, p.clip);
        __syncthreads();
        fault_pass<float, NT, VPT, DV>(g, msg, fw, par, Lam, bb, gg, p.clip);
        __syncthreads();
    }
}

}  // namespace
}  // namespace qldpc
