// Streaming ("lifted") Gauss-Jordan elimination over GF(2) by one warp (paper Sec. 4,
// Algorithm "Lifted Gauss-Jordan over F_2", as the systolic solvers of Sec. 5 and Sec. 6
// apply it to H_R x = sigma and to a cluster's system).
//
// Columns are positions 0..ncols-1 (ncols <= 32 * W <= 1024).  A pivot row is a W-word
// bitset over the columns held in shared memory (up[column][W]); in registers, lane l
// owns word l of a row, of the locked-column bitmap `lockw` and of the pivot rows'
// right-hand-side bits `specw`.  Rows are streamed one at a time; the solution with
// every non-pivot column 0 follows by back substitution.
#pragma once

#include <stdint.h>

namespace qldpc {
namespace gf2 {

constexpr unsigned kFull = 0xffffffffu;

// Row (lane l: word l) with a 1 at each position held by lanes 0..nslots-1 (-1: none).
__device__ __forceinline__ uint32_t row_from_positions(int pos, int nslots) {
    const int lane = threadIdx.x & 31;
    uint32_t row = 0u;
    for (int s = 0; s < nslots; ++s) {
        const int ps = __shfl_sync(kFull, pos, s);
        if (ps >= 0 && (ps >> 5) == lane) row |= 1u << (ps & 31);
    }
    return row;
}

// Reduces `row` (right-hand side `spec`) by the locked pivot rows until its leftmost 1
// is an unlocked column, where it is stored and that column locked.  Returns false when
// the row reduces to zero with right-hand side 1: the system has no solution.  Every
// reduction clears the row's leading column, so at most ncols + 1 steps run.
__device__ __forceinline__ bool insert_row(uint32_t row, uint32_t spec, uint32_t &lockw,
                                           uint32_t &specw, uint32_t *up, int W, int ncols) {
    const int lane = threadIdx.x & 31;
    for (int step = 0; step <= ncols; ++step) {
        const uint32_t nz = __ballot_sync(kFull, row != 0u);
        if (nz == 0u) return spec == 0u;
        const int wl = __ffs(nz) - 1;
        const int bit = __ffs(__shfl_sync(kFull, row, wl)) - 1;
        const int pc = 32 * wl + bit;
        const uint32_t lk = __shfl_sync(kFull, lockw, wl);
        if ((lk >> bit) & 1u) {
            if (lane < W) row ^= up[(size_t)pc * W + lane];
            spec ^= (__shfl_sync(kFull, specw, wl) >> bit) & 1u;
        } else {
            if (lane < W) up[(size_t)pc * W + lane] = row;
            if (lane == wl) {
                lockw |= 1u << bit;
                specw |= spec << bit;
            }
            return true;
        }
    }
    return true;
}

// x over the columns (lane l: word l) with every unlocked column 0: for locked columns
// from the right, x_c = spec_c + <pivot row c, x> (the pivot row's bits left of c are 0).
__device__ __forceinline__ uint32_t back_substitute(uint32_t lockw, uint32_t specw,
                                                    const uint32_t *up, int W, int ncols) {
    const int lane = threadIdx.x & 31;
    uint32_t xw = 0u;
    for (int pc = ncols - 1; pc >= 0; --pc) {
        const int wl = pc >> 5, bit = pc & 31;
        if (!((__shfl_sync(kFull, lockw, wl) >> bit) & 1u)) continue;
        const uint32_t t = lane < W ? (up[(size_t)pc * W + lane] & xw) : 0u;
        const uint32_t parity = __popc(__ballot_sync(kFull, __popc(t) & 1u)) & 1u;
        const uint32_t xp = ((__shfl_sync(kFull, specw, wl) >> bit) & 1u) ^ parity;
        if (xp && lane == wl) xw |= 1u << bit;
    }
    return xw;
}

}  // namespace gf2
}  // namespace qldpc
