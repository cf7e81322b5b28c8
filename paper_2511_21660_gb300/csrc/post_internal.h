// Internal declarations of the post-processors (filtered-OSD, paper Sec. 5; the cluster
// decoder, Sec. 2.5 and Sec. 6), shared by their kernels and their host API.
#pragma once

#include "qldpc_internal.h"

namespace qldpc {

// Filtered-OSD post-processor (paper Sec. 5): plain min-sum BP on the fused layout
// (the graph's gamma row is all zeros), then ranking, submatrix and GF(2) solve.
constexpr int kOsdMaxCandidates = 1024;
struct OsdArgs {
    const int32_t *chk_var;  // [Mp][DC] fault of the k-th edge of check i, -1 past its degree
    int bp_iters;            // plain BP iterations before the ranking
    float llr_conf;          // keep faults with Lambda_j < llr_conf
    int max_cand;            // |R|_max, 1..kOsdMaxCandidates
    int W;                   // 32-bit words of a pivot row: ceil(max_cand / 32)
    int KP;                  // sort capacity: the power of two >= max_cand
};
struct OsdOut {
    uint64_t *corr;    // [B][cor_words], written for solved shots only
    int32_t *status;   // [B] 0 skipped, 1 solved, -1 too many candidates, -2 no solution
    int32_t *ncand;    // [B] |R| (may be NULL)
};
struct OsdKernel {
    int threads, vpt, dc, dv;
    const void *fn;
    cudaError_t (*launch)(dim3 grid, size_t smem, cudaStream_t st, const FusedGraph &g,
                          const DevParams &p, const OsdArgs &o, const uint64_t *syn,
                          const int32_t *list, int B, OsdOut out, unsigned int *counter);
};
void osd_table(const OsdKernel **out, int *n);
// The OSD stage reuses the message area: the inverse ranking [N] i16, then one region
// that holds the sort keys [KP] u64 and, once the inverse ranking is built, the pivot
// rows [max_cand][W] u32, then the list of touched checks [M] i16.
struct OsdLayout {
    size_t pos, region, region_bytes, rows, total;
};
__host__ __device__ inline OsdLayout osd_layout(const FusedGraph &g, const OsdArgs &o) {
    auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
    const size_t keys = 8 * (size_t)o.KP, rows = 4 * (size_t)o.max_cand * o.W;
    OsdLayout L;
    size_t x = 0;
    L.pos = x;    x = al(x + 2 * (size_t)g.N);
    L.region = x; L.region_bytes = al(keys > rows ? keys : rows); x += L.region_bytes;
    L.rows = x;   x = al(x + 2 * (size_t)g.M);
    L.total = x;
    return L;
}
__host__ __device__ inline size_t osd_union_bytes(const FusedGraph &g, const OsdArgs &o) {
    const size_t msg = ((size_t)g.msg_bytes + 15) & ~(size_t)15;
    const size_t osd = osd_layout(g, o).total;
    return msg > osd ? msg : osd;
}
inline size_t osd_smem_bytes(const FusedGraph &g, const OsdArgs &o) {
    return osd_union_bytes(g, o) + 8 * (size_t)g.f_words + 8 * (size_t)g.syn_words +
           8 * (size_t)g.m_words + 64;
}

// Cluster decoder (paper Sec. 2.5 and Sec. 6) after plain BP: partial correction,
// erasures, union-find growth and merging of per-vertex cluster labels, validity by the
// streaming GF(2) solver of one warp.  Vertices are checks 0..M-1 then faults M..M+N-1.
constexpr int kClusterMaxColumns = 512;   // interior faults of one cluster (solver width)
constexpr int kClusterMaxClusters = 4096; // initial clusters (16-bit labels)
struct ClusterArgs {
    const int32_t *chk_var;  // [Mp][DC] fault of the k-th edge of check i, -1 past its degree
    int bp_iters;
    float llr_accept;        // Lambda_j <= llr_accept: partial correction
    float llr_erase;         // llr_accept < Lambda_j <= llr_erase: erasure
    int max_clusters;        // 1..kClusterMaxClusters
    int max_cols;            // 1..kClusterMaxColumns
    int W;                   // ceil(max_cols / 32)
};
struct ClusterOut {
    uint64_t *corr;    // [B][cor_words], written for decoded shots only
    int32_t *status;   // [B] 0 skipped, 1 decoded, -1 cluster too large, -2 too many clusters
    int32_t *steps;    // [B] growth steps (may be NULL)
};
struct ClusterKernel {
    int threads, vpt, dc, dv;
    const void *fn;
    cudaError_t (*launch)(dim3 grid, size_t smem, cudaStream_t st, const FusedGraph &g,
                          const DevParams &p, const ClusterArgs &a, const uint64_t *syn,
                          const int32_t *list, int B, ClusterOut out, unsigned int *counter);
};
void cluster_table(const ClusterKernel **out, int *n);
// The cluster stage reuses the message area: labels [M+N] i16, the grown-vertex bitmap,
// interior / partial-correction / erasure / correction bitmaps over faults, their word
// prefix counts, the updated syndrome, per-cluster flags and queue, pivot rows, the
// list of the cluster's checks [M] i16.
struct ClusterLayout {
    size_t label, grown, intr, wpre, fpre, fera, fout, sp, spre, flags, queue, up, rows, total;
};
__host__ __device__ inline ClusterLayout cluster_layout(const FusedGraph &g, const ClusterArgs &a) {
    auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
    // fault bitmaps padded to whole 64-bit words (the correction's layout)
    const size_t V = (size_t)g.M + g.N, VW = (V + 31) / 32, NW = 2 * (size_t)g.cor_words;
    const size_t MW = (size_t)g.m_words;
    ClusterLayout L;
    size_t o = 0;
    L.label = o; o = al(o + 2 * V);
    L.grown = o; o = al(o + 4 * VW);
    L.intr = o;  o = al(o + 4 * NW);
    L.wpre = o;  o = al(o + 4 * NW);
    L.fpre = o;  o = al(o + 4 * NW);
    L.fera = o;  o = al(o + 4 * NW);
    L.fout = o;  o = al(o + 4 * NW);
    L.sp = o;    o = al(o + 4 * MW);
    L.spre = o;  o = al(o + 4 * (MW > NW ? MW : NW));
    L.flags = o; o = al(o + 2 * (size_t)a.max_clusters);   // merge flag, alive flag
    L.queue = o; o = al(o + 2 * (size_t)a.max_clusters);
    L.up = o;    o = al(o + 4 * (size_t)a.max_cols * a.W);
    L.rows = o;  o = al(o + 2 * (size_t)g.M);
    L.total = o;
    return L;
}
__host__ __device__ inline size_t cluster_union_bytes(const FusedGraph &g, const ClusterArgs &a) {
    const size_t msg = ((size_t)g.msg_bytes + 15) & ~(size_t)15;
    const size_t c = cluster_layout(g, a).total;
    return msg > c ? msg : c;
}
inline size_t cluster_smem_bytes(const FusedGraph &g, const ClusterArgs &a) {
    return cluster_union_bytes(g, a) + 8 * (size_t)g.f_words + 8 * (size_t)g.syn_words +
           8 * (size_t)g.m_words + 4 * (size_t)g.N + 64;
}

}  // namespace qldpc
