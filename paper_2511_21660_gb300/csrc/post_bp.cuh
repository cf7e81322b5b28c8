// Plain min-sum BP of the post-processors (paper Sec. 2.3, "Belief propagation
// decoding"; the pre-decoder set-up of Sec. 7.1): DMem-BP with every gamma_j = 0, run from
// the priors for a fixed number of iterations without early exit.  The post-processors
// use only the marginals, so this form keeps two values per fault in registers: with
// gamma_j = 0 the memory term of every iteration is lambda_j(t) = w_j, so Lambda_j and w_j
// are all the fault state there is (no memory strength, no product to form), and the
// fault pass forms no decisions (no ballots, no parity atomics).  Every float
// operation is the decoding kernels' (relay_device.cuh) in the same order: there
// lambda = (1 - 0) w + 0 Lambda, which equals w exactly (Lambda is finite, w carries no
// negative zero), so the marginals are bit-identical to theirs.
#pragma once

#include "relay_device.cuh"

namespace qldpc {
namespace {

// Marginals of plain BP after `iters` iterations into Lam (fault threadIdx.x + r NT in
// Lam[r]).  Shared memory: the float32 message slots (msg), the staged syndrome (sg) and
// one parity buffer (par, zeroed by each check pass and otherwise unused).  Re-stages the
// padding slots first (callers reuse the message area between shots).  Called by every
// thread of the block; ends with a barrier.
template <int NT, int VPT, int DC, int DV>
__device__ __forceinline__ void plain_bp_marginals(const FusedGraph &g, float C, int iters,
                                                   const uint64_t *sy, unsigned char *msg,
                                                   uint32_t *sg, uint32_t *par,
                                                   float (&Lam)[VPT]) {
    // padding slots hold C for good (the check pass writes C back)
    for (int i = threadIdx.x; i < g.Mp; i += NT) {
        const int deg = g.chk_deg[i], f = swz<DC>(i);
        for (int k = deg; k < DC; ++k) Msg<float>::st(msg, (i * DC + (k ^ f)) * 4, C);
    }
    load_syndrome<NT>(g, sy, sg);
    // nu(0) = lambda(0) = w on every edge, Lambda(0) = w
    float wr[VPT];
#pragma unroll
    for (int r = 0; r < VPT; ++r) {
        const int j = threadIdx.x + r * NT;
        wr[r] = 0.0f;
        if (j < g.N) {
            const float w = canon(__ldg(g.w + j));
            wr[r] = w;
            Lam[r] = w;
            int sl[DV];
            const int deg = load_slots<DV>(g, j, sl);
#pragma unroll
            for (int k = 0; k < DV; ++k)
                if (k < deg) Msg<float>::st(msg, sl[k], w);
        }
    }
    __syncthreads();
    for (int t = 0; t < iters; ++t) {
        check_pass<NT, DC>(g, reinterpret_cast<float *>(msg), sg, par, C);
        __syncthreads();
#pragma unroll
        for (int r = 0; r < VPT; ++r) {
            const int j = threadIdx.x + r * NT;
            if (j < g.N) {
                int sl[DV];
                const int deg = load_slots<DV>(g, j, sl);
                Lam[r] = fault_update<float, DV>(msg, sl, deg, wr[r], C);
            }
        }
        __syncthreads();
    }
}

}  // namespace
}  // namespace qldpc
