// GF(2) elimination by one warp for the systems the post-processors solve (filtered-OSD:
// H_R x = sigma, paper Sec. 5; a cluster's system, Sec. 6): the streaming ("lifted")
// elimination of Sec. 4 (Algorithm "Lifted Gauss-Jordan over F_2"), as the systolic
// solvers of Sec. 5 and Sec. 6 apply it.  Rows arrive in a stream; each is reduced by
// stored pivot rows, one per step (the stored row whose pivot column is the row's leading
// 1), until its leading 1 lies in a column no stored row has taken, where it is stored
// with its right-hand side; a row that reduces to 0 with right-hand side 1 means no
// solution.  Back substitution over the pivot columns, from the right, gives x with every
// free column 0.
//
// Columns are positions 0..ncols-1 (ncols <= 1024).  Pivot row c is a bitset of `stride`
// >= ceil(ncols / 32) 32-bit words at up[c * stride]; when a solver returns, the
// pivot-column bitmap and the pivot rows' right-hand-side bits are lockw and specw, one
// word per lane (lane l: columns 32 l .. 32 l + 31).
//
// Several rows are in flight at once.  The stored rows do not change while rows are
// reduced; then, for each free column that reduced rows lead with, one of them is stored,
// and the others go back for more reduction.  Every stored row still has a
// leading column of its own, so the stored rows are an echelon basis of the rows seen, as
// with one row at a time.  The pivot columns (the leading positions of any echelon basis
// of the span), the inconsistency (a row in the span of the stored rows with the other
// right-hand side) and the solution with free columns 0 are properties of the system, so
// they are the same whatever the order in which rows are stored.
//   stream_rows_lanes: one row per lane, held in registers (up to NWR words), so that a
//     lane reduces its row without the other lanes;
//   stream_rows: lane groups of GW >= ceil(ncols / 32) lanes, lane q of a group holding
//     word q of the group's row (any width up to 32 words).
// rowpos(r, s) is the position of the s-th entry of row r (s < DC; -1: none; positions
// distinct), rowspec(r) its right-hand side.
#pragma once

#include <stdint.h>

namespace qldpc {
namespace gf2 {

constexpr unsigned kFull = 0xffffffffu;

// x over the columns (lane l: word l) with every unlocked column 0: for locked columns
// from the right, x_c = spec_c + <pivot row c, x> (the pivot row's bits left of c are 0).
__device__ __forceinline__ uint32_t back_substitute(uint32_t lockw, uint32_t specw,
                                                    const uint32_t *up, int stride, int ncols) {
    const int lane = threadIdx.x & 31;
    uint32_t xw = 0u;
    for (int pc = ncols - 1; pc >= 0; --pc) {
        const int wl = pc >> 5, bit = pc & 31;
        if (!((__shfl_sync(kFull, lockw, wl) >> bit) & 1u)) continue;
        const uint32_t t = lane < stride ? (up[(size_t)pc * stride + lane] & xw) : 0u;
        const uint32_t parity = __popc(__ballot_sync(kFull, __popc(t) & 1u)) & 1u;
        const uint32_t xp = ((__shfl_sync(kFull, specw, wl) >> bit) & 1u) ^ parity;
        if (xp && lane == wl) xw |= 1u << bit;
    }
    return xw;
}

// One row per lane (ceil(ncols / 32) <= NWR).  Rounds: every lane with a row reduces it
// until it is 0 or its leading 1 is a free column; zero rows retire (right-hand side 1:
// no solution); of the other rows, the lowest lane's row for each leading column is
// stored; lanes whose row was stored or retired take the next rows of the stream.  lk and
// sw are 32-word shared arrays for the pivot bitmaps.
template <int DC, int NWR, typename RowPos, typename RowSpec>
__device__ __forceinline__ bool stream_rows_lanes(int R, int ncols, uint32_t *up, int stride,
                                                  uint32_t *lk, uint32_t *sw, uint32_t &lockw,
                                                  uint32_t &specw, RowPos rowpos,
                                                  RowSpec rowspec) {
    const int lane = threadIdx.x & 31;
    const int nw = (ncols + 31) >> 5;
    if (lane < nw) lk[lane] = sw[lane] = 0u;
    __syncwarp();
    int cur = lane < R ? lane : -1;  // the lane's row (-1: none)
    int next = 32;                   // next row of the stream
    bool fresh = true, ok = true;
    uint32_t r[NWR];
    uint32_t spec = 0u;
    // every round stores or retires at least one row (each leading column met is free
    // and one row per such column is stored), so R + 1 rounds suffice
    for (int round = 0; round <= R; ++round) {
        if (fresh) {
#pragma unroll
            for (int q = 0; q < NWR; ++q) r[q] = 0u;
            spec = 0u;
            if (cur >= 0) {
#pragma unroll 8
                for (int k = 0; k < DC; ++k) {
                    const int p = rowpos(cur, k);
                    const uint32_t bit = p >= 0 ? 1u << (p & 31) : 0u;
#pragma unroll
                    for (int q = 0; q < NWR; ++q)
                        if (q == (p >> 5)) r[q] ^= bit;
                }
                spec = rowspec(cur) & 1u;
            }
            fresh = false;
        }
        const unsigned active = __ballot_sync(kFull, cur >= 0);
        if (!active) break;
        // reduce the lane's row; its leading 1 moves right at every step
        int lead = -1;
        if (cur >= 0) {
            for (int step = 0; step <= ncols; ++step) {
                int w = -1;
                uint32_t v = 0u;
#pragma unroll
                for (int q = NWR - 1; q >= 0; --q)
                    if (r[q] != 0u) {
                        w = q;
                        v = r[q];
                    }
                if (w < 0) {
                    lead = -1;
                    break;
                }
                const int b = __ffs(v) - 1;
                lead = 32 * w + b;
                if (!((lk[w] >> b) & 1u)) break;  // a free column
                const uint32_t *pr = up + (size_t)lead * stride;
#pragma unroll
                for (int q = 0; q < NWR; ++q)
                    if (q < nw) r[q] ^= pr[q];
                spec ^= (sw[w] >> b) & 1u;
            }
        }
        const bool zero = cur >= 0 && lead < 0;
        if (__any_sync(kFull, zero && spec)) {
            ok = false;
            break;
        }
        // store: of the rows that share a leading column, the lowest lane's (the others
        // reduce again by it next round); rows with distinct leading columns are stored
        // side by side
        const bool pend = cur >= 0 && lead >= 0;
        const unsigned same = __match_any_sync(kFull, pend ? lead : -1 - lane);
        const bool store = pend && (same & ((1u << lane) - 1u)) == 0u;
        if (store) {
            uint32_t *pr = up + (size_t)lead * stride;
#pragma unroll
            for (int q = 0; q < NWR; ++q)
                if (q < nw) pr[q] = r[q];
            atomicOr(lk + (lead >> 5), 1u << (lead & 31));
            if (spec) atomicOr(sw + (lead >> 5), 1u << (lead & 31));
        }
        const unsigned retired = __ballot_sync(kFull, zero || store);
        if ((retired >> lane) & 1u) {
            const int k = __popc(retired & ((1u << lane) - 1u));
            cur = next + k < R ? next + k : -1;
            fresh = true;
        }
        next += __popc(retired);
        __syncwarp();
    }
    lockw = lane < nw ? lk[lane] : 0u;
    specw = lane < nw ? sw[lane] : 0u;
    return ok;
}

// Lane groups.  With nw = ceil(ncols / 32), the warp splits into G = 32 / GW groups of GW
// lanes (GW the power of two >= nw); lane q of a group holds word q of that group's row,
// and every group holds a copy of the pivot bitmaps (lane q: words q of lockw and specw).
// Rounds alternate a reduce phase (the groups side by side) and a commit phase (the
// groups in order, as in stream_rows_lanes).
template <int DC, typename RowPos, typename RowSpec>
__device__ __forceinline__ bool stream_rows(int R, int ncols, uint32_t *up, int stride,
                                            uint32_t &lockw, uint32_t &specw, RowPos rowpos,
                                            RowSpec rowspec) {
    const int lane = threadIdx.x & 31;
    const int nw = (ncols + 31) >> 5;
    int GW = 1;
    while (GW < nw) GW <<= 1;
    const int G = 32 / GW, g = lane / GW, q = lane % GW, gb = g * GW;
    const uint32_t low = GW == 32 ? kFull : ((1u << GW) - 1u);
    lockw = specw = 0u;
    int cur = g < R ? g : -1;  // the group's row (-1: none)
    int next = G;              // next row of the stream
    bool fresh = true;         // the group's row is to be built
    uint32_t row = 0u, spec = 0u;
    for (int round = 0; round <= R; ++round) {
        // build the rows of the groups that took a new one (every lane takes part)
        uint32_t built = 0u;
        for (int s0 = 0; s0 < DC; s0 += GW) {
            const int ps = (fresh && cur >= 0 && s0 + q < DC) ? rowpos(cur, s0 + q) : -1;
            for (int t = 0; t < GW && s0 + t < DC; ++t) {
                const int pt = __shfl_sync(kFull, ps, gb + t);
                if (pt >= 0 && (pt >> 5) == q) built ^= 1u << (pt & 31);
            }
        }
        if (fresh) {
            row = built;
            spec = cur >= 0 ? (rowspec(cur) & 1u) : 0u;
            fresh = false;
        }
        if (!__any_sync(kFull, cur >= 0)) return true;
        // reduce: the leading 1 moves right at every step, so at most ncols steps
        for (int step = 0; step <= ncols; ++step) {
            const bool nz = row != 0u;
            const int bl = nz ? __ffs(row) - 1 : 0;
            const uint32_t info = nz ? ((uint32_t)bl | (((lockw >> bl) & 1u) << 5) |
                                        (((specw >> bl) & 1u) << 6))
                                     : 0u;
            const uint32_t gbal = (__ballot_sync(kFull, nz) >> gb) & low;
            const int wl = gbal ? __ffs(gbal) - 1 : 0;
            const uint32_t li = __shfl_sync(kFull, info, gb + wl);
            const bool act = cur >= 0 && gbal != 0u && ((li >> 5) & 1u);
            if (!__any_sync(kFull, act)) break;
            if (act) {
                if (q < nw) row ^= up[(size_t)(32 * wl + (li & 31)) * stride + q];
                spec ^= (li >> 6) & 1u;
            }
        }
        // commit, group by group
        const uint32_t bal = __ballot_sync(kFull, row != 0u);
        for (int h = 0; h < G; ++h) {
            const int hb = h * GW;
            if (__shfl_sync(kFull, cur, hb) < 0) continue;
            const uint32_t hbal = (bal >> hb) & low;
            const uint32_t hspec = __shfl_sync(kFull, spec, hb);
            if (hbal != 0u) {
                const int wl = __ffs(hbal) - 1;
                const int bit = __ffs(__shfl_sync(kFull, row, hb + wl)) - 1;
                if ((__shfl_sync(kFull, lockw, wl) >> bit) & 1u) continue;  // taken: next round
                if (g == h && q < nw) up[(size_t)(32 * wl + bit) * stride + q] = row;
                if (q == wl) {
                    lockw |= 1u << bit;
                    specw |= hspec << bit;
                }
            } else if (hspec) {
                return false;
            }
            if (g == h) {
                cur = next < R ? next : -1;
                fresh = true;
            }
            ++next;
        }
        __syncwarp();
    }
    return true;
}

// Either solver by the row width: registers per lane when ceil(ncols / 32) <= 16.  The
// pivot rows are stored with stride ceil(ncols / 32).
template <int DC, typename RowPos, typename RowSpec>
__device__ __forceinline__ bool solve_stream(int R, int ncols, uint32_t *up, uint32_t *lk,
                                             uint32_t *sw, uint32_t &lockw, uint32_t &specw,
                                             RowPos rowpos, RowSpec rowspec) {
    const int nw = (ncols + 31) >> 5;
    if (nw <= 8)
        return stream_rows_lanes<DC, 8>(R, ncols, up, nw, lk, sw, lockw, specw, rowpos, rowspec);
    if (nw <= 16)
        return stream_rows_lanes<DC, 16>(R, ncols, up, nw, lk, sw, lockw, specw, rowpos, rowspec);
    return stream_rows<DC>(R, ncols, up, nw, lockw, specw, rowpos, rowspec);
}

}  // namespace gf2
}  // namespace qldpc
