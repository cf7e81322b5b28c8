// Filtered-OSD post-processor (paper Sec. 5, "Filtered ordered statistics decoding",
// with the pre-decoder set-up of Sec. 7.1), one thread block per shot at a time:
//
//   1. plain min-sum BP (Sec. 2.3, "Belief propagation decoding") for bp_iters
//      iterations from the priors: the Relay check and fault passes with every
//      gamma_j = 0, no early exit; Lambda stays in registers;
//   2. filtered ranking (Sec. 5, "Filtered column ranking"): the faults with
//      Lambda_j < llr_conf are compacted by warp ballots and sorted by (Lambda_j, j)
//      with a bitonic network in shared memory; more than max_cand is a failure;
//   3. submatrix (Sec. 5, "Extracting submatrix and filtering out zero rows"): the
//      checks touched by R are marked; an untouched check with sigma_i = 1 makes the
//      system unsolvable; only touched rows are streamed;
//   4. solver (Sec. 4, Algorithm "Lifted Gauss-Jordan over F_2", as the paper's
//      systolic solver applies it; gf2_warp.cuh): one warp streams the touched rows in
//      check order; a row is reduced by locked pivot rows until its leftmost 1 (in
//      ranking order) is an unlocked column, where it is stored with its syndrome bit;
//      a row reduced to zero with syndrome bit 1 means no solution.  Several rows are
//      reduced at a time (one per lane, or one per lane group for wide rows).  Back
//      substitution over the locked columns, from the right, gives x with free columns 0;
//   5. F_j = x_r for j = R_r (Sec. 5, "Algorithm output").
//
// A row is a bitset over ranking positions, 32 columns per word.
#include "gf2_warp.cuh"
#include "post_internal.h"
#include "post_bp.cuh"

namespace qldpc {
namespace {

// Order-preserving map of a float (not NaN, not -0) onto uint32.
__device__ __forceinline__ uint32_t sortable(float x) {
    const uint32_t u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

template <int NT>
__device__ __forceinline__ void bitonic_sort(uint64_t *keys, int n) {
    for (int k = 2; k <= n; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int i = threadIdx.x; i < n; i += NT) {
                const int ixj = i ^ jj;
                if (ixj > i) {
                    const uint64_t a = keys[i], b = keys[ixj];
                    const bool ascending = (i & k) == 0;
                    if ((a > b) == ascending) {
                        keys[i] = b;
                        keys[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Several blocks per SM (256 threads x 12 faults: 5 blocks in 48 registers, the plain BP
// holding only Lambda_j and w_j per fault; 512 x 8 with rows of up to 16 slots: 2 in 64):
// the single-warp stages and barriers of one shot then overlap the other blocks' work.
template <int NT, int VPT, int DC, int DV>
__global__ void __launch_bounds__(NT, NT == 256 ? 5 : (VPT <= 8 && DC <= 16 ? 2 : 1)) osd_decode(FusedGraph g, DevParams p, OsdArgs o,
                                                    const uint64_t *__restrict__ syn,
                                                    const int32_t *__restrict__ list, int B,
                                                    OsdOut out, unsigned int *counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *msg = smem_raw;
    const OsdLayout L = osd_layout(g, o);
    int16_t *pos = reinterpret_cast<int16_t *>(smem_raw + L.pos);
    uint64_t *keys = reinterpret_cast<uint64_t *>(smem_raw + L.region);
    uint32_t *up = reinterpret_cast<uint32_t *>(smem_raw + L.region);  // after the sort
    int16_t *rows = reinterpret_cast<int16_t *>(smem_raw + L.rows);
    uint32_t *fw = reinterpret_cast<uint32_t *>(smem_raw + osd_union_bytes(g, o));
    uint32_t *fb = fw + g.f_words;
    uint32_t *sg = fb + g.f_words;
    uint32_t *par = sg + 2 * g.syn_words;
    __shared__ int s_shot, s_cnt, s_bad, s_rows;
    // the shots: list[0 .. counter[1]) (the host's compaction of a skip mask), else 0 .. B-1
    const int n_work = list ? (int)counter[1] : B;
    __shared__ uint32_t s_x[32], s_lk[32], s_sw[32];
    const int tid = threadIdx.x, lane = tid & 31;

    for (;;) {
        // per-shot registers, declared here so that nothing of them lives across shots
        float Lam[VPT];
#pragma unroll
        for (int r = 0; r < VPT; ++r) Lam[r] = 0.0f;
        __syncthreads();  // the previous shot is done with shared memory
        if (tid == 0) s_shot = (int)atomicAdd(counter, 1u);
        __syncthreads();
        if (s_shot >= n_work) break;
        const int shot = list ? list[s_shot] : s_shot;

        // 1. plain BP: lambda_j(t) = w_j (gamma row of zeros), Lambda from the priors
        if (tid == 0) {
            s_cnt = 0;
            s_bad = 0;
            s_rows = 0;
        }
        plain_bp_marginals<NT, VPT, DC, DV>(g, p.clip, o.bp_iters, syn + (size_t)shot * g.syn_words,
                                            msg, sg, par, Lam);

        // 2. ranking: candidates Lambda_j < llr_conf, keys (Lambda_j, j)
#pragma unroll
        for (int r = 0; r < VPT; ++r) {
            const int j = tid + r * NT;
            const bool valid = j < g.N;
            const float x = valid ? canon(Lam[r]) : 0.0f;
            const bool cand = valid && x < o.llr_conf;
            const uint32_t bal = __ballot_sync(FULL, cand);
            if (bal) {
                const int leader = __ffs(bal) - 1;
                int base = 0;
                if (lane == leader) base = atomicAdd(&s_cnt, __popc(bal));
                base = __shfl_sync(FULL, base, leader);
                if (cand) {
                    const int idx = base + __popc(bal & ((1u << lane) - 1u));
                    if (idx < o.KP) keys[idx] = ((uint64_t)sortable(x) << 32) | (uint32_t)j;
                }
            }
        }
        __syncthreads();
        const int n = s_cnt;
        if (n > o.max_cand) {
            if (tid == 0) {
                out.status[shot] = -1;
                if (out.ncand) out.ncand[shot] = n;
            }
            continue;
        }
        int np2 = 1;
        while (np2 < n) np2 <<= 1;
        for (int q = n + tid; q < np2; q += NT) keys[q] = ~0ull;
        __syncthreads();
        bitonic_sort<NT>(keys, np2);

        // 3. inverse ranking and the checks touched by R (par reused as the bitmap)
        for (int j = tid; j < g.N; j += NT) pos[j] = -1;
        for (int q = tid; q < g.m_words; q += NT) par[q] = 0u;
        __syncthreads();
        for (int r = tid; r < n; r += NT) {
            const int j = (int)(uint32_t)keys[r];
            pos[j] = (int16_t)r;
            const int deg = (int)((uint32_t)__ldg(g.var_slot + (size_t)j * DV) >> 24);
            for (int k = 0; k < deg; ++k) {
                const int c = __ldg(g.var_chk + (size_t)j * DV + k);
                atomicOr(par + (c >> 5), 1u << (c & 31));
            }
        }
        __syncthreads();
        for (int q = tid; q < g.m_words; q += NT)
            if (sg[q] & ~par[q]) s_bad = 1;  // a syndrome bit on a row H_R leaves empty
        __syncthreads();

        // 4. the touched checks (the rows of H_R), listed by the whole block in any order
        // (the elimination's result does not depend on it), with each row's ranking
        // positions in a table after the pivot rows' space when it fits there
        const int nw = (n + 31) >> 5;
        const size_t piv_words = ((size_t)n * nw + 3) & ~(size_t)3;
        int16_t *tab = reinterpret_cast<int16_t *>(up + piv_words);
        const size_t piv_bytes = 4 * piv_words;  // <= region_bytes, as n <= max_cand
        const int tab_rows =
            piv_bytes < L.region_bytes ? (int)((L.region_bytes - piv_bytes) / (2 * DC)) : 0;
        if (!s_bad)
            for (int c = tid; c < g.M; c += NT) {
                if (!((par[c >> 5] >> (c & 31)) & 1u)) continue;
                const int r = atomicAdd(&s_rows, 1);
                rows[r] = (int16_t)c;
                if (r < tab_rows)
                    for (int k = 0; k < DC; ++k) {
                        const int jv = __ldg(o.chk_var + (size_t)c * DC + k);
                        tab[r * DC + k] = jv >= 0 ? pos[jv] : (int16_t)-1;
                    }
            }
        __syncthreads();

        // 5. elimination by warp 0
        if (tid < 32 && !s_bad) {
            const int R = s_rows;
            const bool in_tab = R <= tab_rows;
            uint32_t lockw, specw;
            const bool ok = gf2::solve_stream<DC>(
                R, n, up, s_lk, s_sw, lockw, specw,
                [&](int rr, int k) {
                    if (in_tab) return (int)tab[rr * DC + k];
                    const int jv = __ldg(o.chk_var + (size_t)rows[rr] * DC + k);
                    return jv >= 0 ? (int)pos[jv] : -1;
                },
                [&](int rr) {
                    const int c = rows[rr];
                    return (sg[c >> 5] >> (c & 31)) & 1u;
                });
            const bool bad = !ok;
            const uint32_t xw = ok ? gf2::back_substitute(lockw, specw, up, nw, n) : 0u;
            s_x[lane] = xw;
            if (lane == 0 && bad) s_bad = 1;
        }
        __syncthreads();

        // 6. scatter x to the faults of R
        if (s_bad) {
            if (tid == 0) {
                out.status[shot] = -2;
                if (out.ncand) out.ncand[shot] = n;
            }
            continue;
        }
        for (int q = tid; q < 2 * g.cor_words; q += NT) fw[q] = 0u;
        __syncthreads();
        for (int j = tid; j < g.N; j += NT) {
            const int r = pos[j];
            if (r >= 0 && ((s_x[r >> 5] >> (r & 31)) & 1u)) atomicOr(fw + (j >> 5), 1u << (j & 31));
        }
        __syncthreads();
        store_bits<NT>(out.corr + (size_t)shot * g.cor_words, fw, g.cor_words);
        if (tid == 0) {
            out.status[shot] = 1;
            if (out.ncand) out.ncand[shot] = n;
        }
    }
}

template <int NT, int VPT, int DC, int DV>
cudaError_t launch_osd(dim3 grid, size_t smem, cudaStream_t st, const FusedGraph &g,
                       const DevParams &p, const OsdArgs &o, const uint64_t *syn,
                       const int32_t *list, int B, OsdOut out, unsigned int *counter) {
    osd_decode<NT, VPT, DC, DV><<<grid, NT, smem, st>>>(g, p, o, syn, list, B, out, counter);
    return cudaGetLastError();
}

template <int NT, int VPT, int DC, int DV>
OsdKernel osd_entry() {
    OsdKernel k;
    k.threads = NT;
    k.vpt = VPT;
    k.dc = DC;
    k.dv = DV;
    k.fn = (const void *)osd_decode<NT, VPT, DC, DV>;
    k.launch = &launch_osd<NT, VPT, DC, DV>;
    return k;
}

}  // namespace

void osd_table(const OsdKernel **out, int *n) {
    // per (DC, DV) family of the fused layout: the first entry with threads * vpt >= N
    static const OsdKernel table[] = {
        osd_entry<256, 12, 8, 4>(), osd_entry<512, 8, 8, 4>(),  osd_entry<512, 16, 8, 4>(),
        osd_entry<512, 8, 16, 8>(), osd_entry<512, 16, 16, 8>(),
        osd_entry<512, 8, 32, 8>(), osd_entry<512, 16, 32, 8>(),
    };
    *out = table;
    *n = (int)(sizeof(table) / sizeof(table[0]));
}

}  // namespace qldpc
