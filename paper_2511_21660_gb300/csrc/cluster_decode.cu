// Cluster decoder after plain BP (paper Sec. 2.5, "Cluster decoding" and "BP-UF
// decoding"; its FPGA form in Sec. 6; pre-decoder set-up of Sec. 7.1), one thread block
// per shot at a time:
//
//   1. plain min-sum BP for bp_iters iterations from the priors (relay_device.cuh);
//   2. input (Sec. 6.2): faults with Lambda_j <= llr_accept form the partial correction
//      F_pre, faults with llr_accept < Lambda_j <= llr_erase the erasure set;
//      sigma <- sigma + H F_pre by parity atomics;
//   3. initialisation (Sec. 6.3): one cluster per syndrome check and per erased fault,
//      numbered in seed-extraction order (right-most bit of the initialisation bitmap
//      first: decreasing check index, then decreasing fault index); the single-check
//      clusters are the invalid list, the erased-fault clusters start valid (no check,
//      no interior fault);
//   4. update loop (Sec. 6.4-6.7): the first invalid cluster c is grown by every
//      neighbour of its vertices, every cluster the grown set meets is merged into c
//      (and leaves the invalid list), the interior faults of c are found, and c is
//      tested by the streaming GF(2) solver of one warp (gf2_warp.cuh, several rows in
//      flight) on its checks (rows, increasing index) and interior faults (columns,
//      increasing index); an invalid c goes to the end of the list;
//   5. output (Sec. 6.8): each surviving cluster's solution with free columns 0; the
//      correction is F_pre + the union of those.
//
// Clusters are kept as one 16-bit label per vertex (checks 0..M-1, faults M..M+N-1)
// instead of one bitmap per cluster: growth, merge detection and relabelling are then
// three block-wide passes over the vertices, whatever the number of clusters.
#include "gf2_warp.cuh"
#include "post_internal.h"
#include "relay_device.cuh"

namespace qldpc {
namespace {

// Exclusive prefix of the popcounts of words[0..nw) into pre[], by one warp; returns
// the total on every lane.
__device__ __forceinline__ int warp_word_prefix(const uint32_t *words, uint32_t *pre, int nw) {
    const int lane = threadIdx.x & 31;
    const int ch = (nw + 31) / 32;
    const int w0 = lane * ch, w1 = min(nw, w0 + ch);
    int local = 0;
    for (int w = w0; w < w1; ++w) local += __popc(words[w]);
    int incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    int run = incl - local;
    for (int w = w0; w < w1; ++w) {
        pre[w] = (uint32_t)run;
        run += __popc(words[w]);
    }
    return __shfl_sync(FULL, incl, 31);
}

// Set bits of words at or below position b of its word.
__device__ __forceinline__ uint32_t mask_upto(int b) {
    return b == 31 ? 0xffffffffu : ((2u << b) - 1u);
}

__device__ __forceinline__ void set_bit(uint32_t *bm, int v) {
    atomicOr(bm + (v >> 5), 1u << (v & 31));
}

__device__ __forceinline__ bool get_bit(const uint32_t *bm, int v) {
    return (bm[v >> 5] >> (v & 31)) & 1u;
}

template <int DV>
__device__ __forceinline__ int fault_degree(const FusedGraph &g, int j) {
    return (int)((uint32_t)__ldg(g.var_slot + (size_t)j * DV) >> 24);
}

// Fault j belongs to cluster `lab` and so does each of its checks.
template <int DV>
__device__ __forceinline__ bool interior_of(const FusedGraph &g, const int16_t *label, int j,
                                            int lab) {
    if (label[g.M + j] != lab) return false;
    const int deg = fault_degree<DV>(g, j);
    for (int k = 0; k < deg; ++k)
        if (label[__ldg(g.var_chk + (size_t)j * DV + k)] != lab) return false;
    return true;
}

// Solves the system of cluster `lab` (rows: its checks, increasing index; columns: its
// interior faults, bitmap intr with word prefix wpre) by one warp, streaming the rows
// (gf2_warp.cuh); lab < 0 takes the checks of every cluster.  Returns consistency; with
// `want_x`, lane l's word of the solution (free columns 0) goes to *x.
template <int DC>
__device__ __forceinline__ bool solve_cluster(const FusedGraph &g, const ClusterArgs &a,
                                              const ClusterLayout &L, unsigned char *smem,
                                              const int16_t *label, int lab,
                                              const uint32_t *intr, const uint32_t *wpre,
                                              const uint32_t *sp, int ncols, bool want_x,
                                              uint32_t *x) {
    const int lane = threadIdx.x & 31;
    uint32_t *up = reinterpret_cast<uint32_t *>(smem + L.up);
    int16_t *rows = reinterpret_cast<int16_t *>(smem + L.rows);
    // the cluster's checks: lane l lists those of the contiguous range [i0, i1)
    const int ch = (g.M + 31) / 32, i0 = min(g.M, lane * ch), i1 = min(g.M, i0 + ch);
    int local = 0;
    auto member = [&](int i) { return lab < 0 ? label[i] >= 0 : label[i] == lab; };
    bool odd = false;  // a row with syndrome bit 1
    for (int i = i0; i < i1; ++i)
        if (member(i)) {
            ++local;
            odd |= (sp[i >> 5] >> (i & 31)) & 1u;
        }
    // no syndrome bit: x = 0 solves it (and is the solution with free columns 0); no
    // column: only the zero syndrome is in the image
    const bool any_odd = __any_sync(FULL, odd);
    if (!any_odd || ncols == 0) {
        if (want_x) *x = 0u;
        return !any_odd;
    }
    int incl = local;
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += t;
    }
    const int R = __shfl_sync(FULL, incl, 31);
    int r = incl - local;
    for (int i = i0; i < i1; ++i)
        if (member(i)) rows[r++] = (int16_t)i;
    __syncwarp();
    __shared__ uint32_t s_lk[32], s_sw[32];
    uint32_t lockw, specw;
    const bool ok = gf2::solve_stream<DC>(
        R, ncols, up, s_lk, s_sw, lockw, specw,
        [&](int rr, int k) {
            const int jv = __ldg(a.chk_var + (size_t)rows[rr] * DC + k);
            if (jv < 0 || !get_bit(intr, jv)) return -1;
            return (int)wpre[jv >> 5] + __popc(intr[jv >> 5] & ((1u << (jv & 31)) - 1u));
        },
        [&](int rr) {
            const int c = rows[rr];
            return (sp[c >> 5] >> (c & 31)) & 1u;
        });
    if (want_x) *x = ok ? gf2::back_substitute(lockw, specw, up, (ncols + 31) >> 5, ncols) : 0u;
    return ok;
}

// Two blocks per SM where the kernel fits in 64 registers without spilling (8 faults
// per thread, rows of up to 16 slots): the single-warp stages of one shot then overlap
// the other block's work.
template <int NT, int VPT, int DC, int DV>
__global__ void __launch_bounds__(NT, VPT <= 8 && DC <= 16 ? 2 : 1) cluster_decode(FusedGraph g, DevParams p, ClusterArgs a,
                                                        const uint64_t *__restrict__ syn,
                                                        const int32_t *__restrict__ list, int B,
                                                        ClusterOut out, unsigned int *counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *msg = smem_raw;
    const ClusterLayout L = cluster_layout(g, a);
    int16_t *label = reinterpret_cast<int16_t *>(smem_raw + L.label);
    uint32_t *grown = reinterpret_cast<uint32_t *>(smem_raw + L.grown);
    uint32_t *intr = reinterpret_cast<uint32_t *>(smem_raw + L.intr);
    uint32_t *wpre = reinterpret_cast<uint32_t *>(smem_raw + L.wpre);
    uint32_t *fpre = reinterpret_cast<uint32_t *>(smem_raw + L.fpre);
    uint32_t *fera = reinterpret_cast<uint32_t *>(smem_raw + L.fera);
    uint32_t *fout = reinterpret_cast<uint32_t *>(smem_raw + L.fout);
    uint32_t *sp = reinterpret_cast<uint32_t *>(smem_raw + L.sp);
    uint32_t *spre = reinterpret_cast<uint32_t *>(smem_raw + L.spre);
    uint8_t *mflag = smem_raw + L.flags;
    int16_t *queue = reinterpret_cast<int16_t *>(smem_raw + L.queue);
    uint32_t *fw = reinterpret_cast<uint32_t *>(smem_raw + cluster_union_bytes(g, a));
    uint32_t *fb = fw + g.f_words;
    uint32_t *sg = fb + g.f_words;
    uint32_t *par = sg + 2 * g.syn_words;
    float *ws = reinterpret_cast<float *>(par + 2 * g.m_words);
    __shared__ int s_shot, s_ns, s_ne, s_status, s_c, s_head, s_count, s_steps, s_nint, s_valid;
    __shared__ uint32_t s_x[32];
    // the shots: list[0 .. counter[1]) (the host's compaction of a skip mask), else 0 .. B-1
    const int n_work = list ? (int)counter[1] : B;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int V = g.M + g.N, VW = (V + 31) / 32, NW = (g.N + 31) / 32;
    const int NWp = 2 * g.cor_words;  // fault bitmaps padded to whole 64-bit words
    const int MW = g.m_words, KC = a.max_clusters;

    for (;;) {
        // per-shot registers, declared here so that nothing of them lives across shots
        float Lam[VPT], bb[VPT], gg[VPT];
#pragma unroll
        for (int r = 0; r < VPT; ++r) Lam[r] = bb[r] = gg[r] = 0.0f;
        __syncthreads();  // the previous shot is done with shared memory
        if (tid == 0) s_shot = (int)atomicAdd(counter, 1u);
        __syncthreads();
        if (s_shot >= n_work) break;
        const int shot = list ? list[s_shot] : s_shot;

        // 1. plain BP
        if (tid == 0) {
            s_status = 1;
            s_steps = 0;
        }
        plain_bp<NT, VPT, DC, DV>(g, p, a.bp_iters, syn + (size_t)shot * g.syn_words, msg, fw,
                                  sg, par, ws, Lam, bb, gg);

        // 2. partial correction and erasures; sigma + H F_pre
        uint32_t pmask = 0u;
#pragma unroll
        for (int r = 0; r < VPT; ++r) {
            const int j = tid + r * NT;
            const bool valid = j < g.N;
            const float x = Lam[r];
            const bool pre = valid && x <= a.llr_accept;
            const bool era = valid && x > a.llr_accept && x <= a.llr_erase;
            const uint32_t bp_ = __ballot_sync(FULL, pre), be = __ballot_sync(FULL, era);
            const int jb = tid - lane + r * NT;
            if (lane == 0 && jb < g.N) {
                fpre[jb >> 5] = bp_;
                fera[jb >> 5] = be;
            }
            pmask |= (pre ? 1u : 0u) << r;
        }
        if (tid == 0)
            for (int q = NW; q < NWp; ++q) fpre[q] = fera[q] = 0u;
        for (int q = tid; q < MW; q += NT) sp[q] = sg[q];
        __syncthreads();
        while (pmask) {
            const int r = __ffs(pmask) - 1;
            pmask &= pmask - 1u;
            const int j = tid + r * NT;
            const int deg = fault_degree<DV>(g, j);
            for (int k = 0; k < deg; ++k) {
                const int c = __ldg(g.var_chk + (size_t)j * DV + k);
                atomicXor(sp + (c >> 5), 1u << (c & 31));
            }
        }
        __syncthreads();

        // 3. seeds, numbered right-most first: checks, then erased faults
        if (warp == 0) {
            const int ns = warp_word_prefix(sp, spre, MW);
            if (lane == 0) s_ns = ns;
        } else if (warp == 1) {
            const int ne = warp_word_prefix(fera, wpre, NWp);
            if (lane == 0) s_ne = ne;
        }
        __syncthreads();
        const int ns = s_ns, ne = s_ne;
        if (ns + ne > KC) {
            if (tid == 0) {
                out.status[shot] = -2;
                if (out.steps) out.steps[shot] = 0;
            }
            continue;
        }
        for (int v = tid; v < V; v += NT) {
            int16_t lab = -1;
            if (v < g.M) {
                if (get_bit(sp, v))
                    lab = (int16_t)(ns - (int)spre[v >> 5] -
                                    __popc(sp[v >> 5] & mask_upto(v & 31)));
            } else {
                const int j = v - g.M;
                if (get_bit(fera, j))
                    lab = (int16_t)(ns + ne - (int)wpre[j >> 5] -
                                    __popc(fera[j >> 5] & mask_upto(j & 31)));
            }
            label[v] = lab;
        }
        for (int q = tid; q < KC; q += NT) {
            mflag[q] = 0;
            queue[q] = (int16_t)q;  // the invalid list starts as the check seeds 0..ns-1
        }
        if (tid == 0) {
            s_head = 0;
            s_count = ns;
        }
        __syncthreads();

        // 4. update loop: every step adds a vertex to a cluster, so at most V steps
        for (;;) {
            if (tid == 0) {
                if (s_count == 0 || s_steps >= V) {
                    s_c = -1;
                    if (s_count != 0) s_status = -3;
                } else {
                    s_c = queue[s_head];
                    s_head = s_head + 1 == KC ? 0 : s_head + 1;
                    --s_count;
                    ++s_steps;
                }
            }
            for (int q = tid; q < VW; q += NT) grown[q] = 0u;
            __syncthreads();
            const int c = s_c;
            if (c < 0) break;
            // grow: every vertex of c and its neighbours; a neighbour in another cluster
            // flags that cluster for merging (labels do not change in this pass)
            for (int q = tid; q < NWp; q += NT) intr[q] = 0u;
            for (int v = tid; v < V; v += NT) {
                if (label[v] != c) continue;
                set_bit(grown, v);
                if (v < g.M) {
                    for (int k = 0; k < DC; ++k) {
                        const int jv = __ldg(a.chk_var + (size_t)v * DC + k);
                        if (jv < 0) break;
                        const int lu = label[g.M + jv];
                        set_bit(grown, g.M + jv);
                        if (lu >= 0 && lu != c) mflag[lu] = 1;
                    }
                } else {
                    const int j = v - g.M, deg = fault_degree<DV>(g, j);
                    for (int k = 0; k < deg; ++k) {
                        const int u = __ldg(g.var_chk + (size_t)j * DV + k);
                        const int lu = label[u];
                        set_bit(grown, u);
                        if (lu >= 0 && lu != c) mflag[lu] = 1;
                    }
                }
            }
            __syncthreads();
            // merge: the grown set and the flagged clusters join c
            for (int v = tid; v < V; v += NT) {
                const int lab = label[v];
                if (get_bit(grown, v) || (lab >= 0 && mflag[lab])) label[v] = (int16_t)c;
            }
            if (warp == NT / 32 - 1) {  // merged clusters leave the invalid list, in order
                const int cnt = s_count, head = s_head;
                int kept = 0;
                for (int q0 = 0; q0 < cnt; q0 += 32) {
                    const int q = q0 + lane;
                    const int at = head + q >= KC ? head + q - KC : head + q;
                    const int id = q < cnt ? queue[at] : 0;
                    const bool keep = q < cnt && !mflag[id];
                    const unsigned bal = __ballot_sync(FULL, keep);
                    if (keep) {
                        const int to = head + kept + __popc(bal & ((1u << lane) - 1u));
                        queue[to >= KC ? to - KC : to] = (int16_t)id;
                    }
                    kept += __popc(bal);
                    __syncwarp();
                }
                if (lane == 0) s_count = kept;
            }
            __syncthreads();
            for (int q = tid; q < ns + ne; q += NT) mflag[q] = 0;  // next read after two barriers
            // interior faults of c
            for (int j = tid; j < g.N; j += NT)
                if (interior_of<DV>(g, label, j, c)) set_bit(intr, j);
            __syncthreads();
            if (warp == 0) {
                const int n = warp_word_prefix(intr, wpre, NWp);
                if (lane == 0) s_nint = n;
            }
            __syncthreads();
            const int n = s_nint;
            if (n > a.max_cols) {
                if (tid == 0) s_status = -1;
                break;
            }
            // validity of c by warp 0
            if (warp == 0) {
                const bool ok = solve_cluster<DC>(g, a, L, smem_raw, label, c, intr, wpre, sp, n,
                                                  false, nullptr);
                if (lane == 0) s_valid = ok;
            }
            __syncthreads();
            if (tid == 0 && !s_valid) {
                queue[(s_head + s_count) % KC] = (int16_t)c;
                ++s_count;
            }
        }
        __syncthreads();
        if (s_status != 1) {
            if (tid == 0) {
                out.status[shot] = s_status;
                if (out.steps) out.steps[shot] = s_steps;
            }
            continue;
        }

        // 5. solutions of the clusters that own an interior fault.  The clusters are
        // disjoint and the checks of an interior fault all lie in its cluster, so the
        // clusters' systems are the diagonal blocks of one system (rows: the checks of
        // every cluster; columns: every interior fault).  A column is independent of the
        // columns left of it exactly when it is so within its block, so the pivot columns
        // are the blocks' together and the solution with free columns 0 is the blocks'
        // side by side: one solve serves every cluster when the interior faults fit the
        // solver's width; otherwise the clusters are solved one by one.
        for (int q = tid; q < NWp; q += NT) fout[q] = intr[q] = 0u;
        __syncthreads();
        for (int j = tid; j < g.N; j += NT) {
            const int lab = label[g.M + j];
            if (lab >= 0 && interior_of<DV>(g, label, j, lab)) {
                mflag[lab] = 1;
                set_bit(intr, j);
            }
        }
        __syncthreads();
        if (warp == 0) {
            const int n = warp_word_prefix(intr, wpre, NWp);
            if (lane == 0) s_nint = n;
        }
        __syncthreads();
        const bool joint = s_nint <= a.max_cols;
        if (joint) {
            if (warp == 0) {
                uint32_t xw = 0u;
                solve_cluster<DC>(g, a, L, smem_raw, label, -1, intr, wpre, sp, s_nint, true,
                                  &xw);
                s_x[lane] = xw;
            }
            __syncthreads();
            for (int j = tid; j < g.N; j += NT) {
                if (!get_bit(intr, j)) continue;
                const int pc = (int)wpre[j >> 5] + __popc(intr[j >> 5] & ((1u << (j & 31)) - 1u));
                if ((s_x[pc >> 5] >> (pc & 31)) & 1u) set_bit(fout, j);
            }
            __syncthreads();
        }
        for (int id = 0; id < (joint ? 0 : ns + ne); ++id) {
            if (!mflag[id]) continue;  // uniform: every thread reads the same flag
            for (int q = tid; q < NWp; q += NT) intr[q] = 0u;
            __syncthreads();
            for (int j = tid; j < g.N; j += NT)
                if (interior_of<DV>(g, label, j, id)) set_bit(intr, j);
            __syncthreads();
            if (warp == 0) {
                const int n = warp_word_prefix(intr, wpre, NWp);
                uint32_t xw = 0u;
                solve_cluster<DC>(g, a, L, smem_raw, label, id, intr, wpre, sp, n, true, &xw);
                s_x[lane] = xw;
            }
            __syncthreads();
            for (int j = tid; j < g.N; j += NT) {
                if (!get_bit(intr, j)) continue;
                const int pc = (int)wpre[j >> 5] + __popc(intr[j >> 5] & ((1u << (j & 31)) - 1u));
                if ((s_x[pc >> 5] >> (pc & 31)) & 1u) set_bit(fout, j);
            }
            __syncthreads();
        }
        for (int q = tid; q < g.cor_words; q += NT)
            out.corr[(size_t)shot * g.cor_words + q] =
                (uint64_t)(fout[2 * q] ^ fpre[2 * q]) |
                ((uint64_t)(fout[2 * q + 1] ^ fpre[2 * q + 1]) << 32);
        if (tid == 0) {
            out.status[shot] = 1;
            if (out.steps) out.steps[shot] = s_steps;
        }
    }
}

template <int NT, int VPT, int DC, int DV>
cudaError_t launch_cluster(dim3 grid, size_t smem, cudaStream_t st, const FusedGraph &g,
                           const DevParams &p, const ClusterArgs &a, const uint64_t *syn,
                           const int32_t *list, int B, ClusterOut out, unsigned int *counter) {
    cluster_decode<NT, VPT, DC, DV><<<grid, NT, smem, st>>>(g, p, a, syn, list, B, out, counter);
    return cudaGetLastError();
}

template <int NT, int VPT, int DC, int DV>
ClusterKernel cluster_entry() {
    ClusterKernel k;
    k.threads = NT;
    k.vpt = VPT;
    k.dc = DC;
    k.dv = DV;
    k.fn = (const void *)cluster_decode<NT, VPT, DC, DV>;
    k.launch = &launch_cluster<NT, VPT, DC, DV>;
    return k;
}

}  // namespace

void cluster_table(const ClusterKernel **out, int *n) {
    // per (DC, DV) family of the fused layout: the first entry with threads * vpt >= N
    static const ClusterKernel table[] = {
        cluster_entry<512, 8, 8, 4>(),  cluster_entry<512, 16, 8, 4>(),
        cluster_entry<512, 8, 16, 8>(), cluster_entry<512, 16, 16, 8>(),
        cluster_entry<512, 8, 32, 8>(), cluster_entry<512, 16, 32, 8>(),
    };
    *out = table;
    *n = (int)(sizeof(table) / sizeof(table[0]));
}

}  // namespace qldpc
