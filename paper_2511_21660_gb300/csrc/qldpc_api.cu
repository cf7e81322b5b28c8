// Host side of the Relay decoder's C ABI (include/qldpc.h): input validation, graph
// layout for the kernels, kernel selection, launches and buffer staging.  The soft
// DMem-BP leg's entry points are in soft_api.cu, the post-processors' in post_api.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_fp16.h>

#include "api_common.h"

using namespace qldpc;

namespace qldpc {

static thread_local std::string g_last_error;

std::string &last_error() { return g_last_error; }

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int validate_graph(int32_t M, int32_t N, const int32_t *row_ptr, const int32_t *col_idx,
                   const double *priors) {
    if (M < 1 || N < 1) return fail(QLDPC_ERR_INVALID_ARG, "need M >= 1 and N >= 1 (got %d, %d)", M, N);
    if (!row_ptr || !priors) return fail(QLDPC_ERR_INVALID_ARG, "row_ptr and priors must not be NULL");
    if (row_ptr[0] != 0) return fail(QLDPC_ERR_INVALID_ARG, "row_ptr[0] must be 0");
    for (int i = 0; i < M; ++i)
        if (row_ptr[i + 1] < row_ptr[i])
            return fail(QLDPC_ERR_INVALID_ARG, "row_ptr decreases at row %d", i);
    const int64_t E = row_ptr[M];
    if (E > 0 && !col_idx) return fail(QLDPC_ERR_INVALID_ARG, "col_idx must not be NULL");
    for (int i = 0; i < M; ++i)
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            if (col_idx[e] < 0 || col_idx[e] >= N)
                return fail(QLDPC_ERR_INVALID_ARG, "col_idx[%d] = %d outside [0, %d)", e, col_idx[e], N);
            if (e > row_ptr[i] && col_idx[e] <= col_idx[e - 1])
                return fail(QLDPC_ERR_INVALID_ARG, "columns of row %d are not strictly increasing", i);
        }
    for (int j = 0; j < N; ++j)
        if (!(priors[j] > 0.0 && priors[j] < 1.0))
            return fail(QLDPC_ERR_INVALID_ARG, "prior %d = %g outside (0, 1)", j, priors[j]);
    return QLDPC_OK;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int check_batch(const qldpc_decoder *d, const void *syn, int64_t B, const void *corr) {
    if (!d) return fail(QLDPC_ERR_INVALID_ARG, "decoder handle is NULL");
    if (B < 0 || B > 0x7fffffffLL) return fail(QLDPC_ERR_INVALID_ARG, "batch size %lld out of range", (long long)B);
    if (B > 0 && (!syn || !corr)) return fail(QLDPC_ERR_INVALID_ARG, "syndromes and corrections must not be NULL");
    return QLDPC_OK;
}

}  // namespace qldpc


namespace {
int lookup_static_scratch(qldpc_decoder *d);
}

namespace {


int validate_params(const qldpc_relay_params *p, int N) {
    if (!p) return fail(QLDPC_ERR_INVALID_ARG, "params must not be NULL");
    if (p->legs_after_first < 0) return fail(QLDPC_ERR_INVALID_ARG, "legs_after_first < 0");
    if (p->iters_first < 1 || p->iters_later < 1)
        return fail(QLDPC_ERR_INVALID_ARG, "iteration limits must be >= 1");
    if (p->stop_after_solutions < 1) return fail(QLDPC_ERR_INVALID_ARG, "stop_after_solutions < 1");
    if (p->warm_start_mode != 0 && p->warm_start_mode != 1)
        return fail(QLDPC_ERR_INVALID_ARG, "warm_start_mode must be 0 or 1");
    if (p->msg_precision != QLDPC_MSG_FP32 && p->msg_precision != QLDPC_MSG_FP16)
        return fail(QLDPC_ERR_INVALID_ARG, "unknown msg_precision %d", p->msg_precision);
    if (p->kernel < QLDPC_KERNEL_AUTO || p->kernel > QLDPC_KERNEL_FUSED)
        return fail(QLDPC_ERR_INVALID_ARG, "unknown kernel %d", p->kernel);
    if (p->block_threads < 0) return fail(QLDPC_ERR_INVALID_ARG, "block_threads < 0");
    if (!(std::isfinite(p->llr_clip))) return fail(QLDPC_ERR_INVALID_ARG, "llr_clip is not finite");
    if (p->msg_precision == QLDPC_MSG_FP16 && p->llr_clip > 0.0f &&
        __half2float(__float2half_rn(p->llr_clip)) != p->llr_clip)
        return fail(QLDPC_ERR_INVALID_ARG, "llr_clip must be a binary16 value (<= 65504)");
    if (!p->gamma_table) return fail(QLDPC_ERR_INVALID_ARG, "gamma_table must not be NULL");
    const size_t n = (size_t)(p->legs_after_first + 1) * N;
    for (size_t q = 0; q < n; ++q)
        if (!std::isfinite(p->gamma_table[q]))
            return fail(QLDPC_ERR_INVALID_ARG, "gamma_table[%zu] is not finite", q);
    return QLDPC_OK;
}


// Picks the compiled fused-kernel family for the graph's degrees.
int pick_family(int dc, int dv, int fp16, const FusedKernel **tab, int *n) {
    if (dc <= 8 && dv <= 4) {
        if (fp16) fused_table_f16_8_4(tab, n); else fused_table_f32_8_4(tab, n);
    } else if (dc <= 16 && dv <= 8) {
        if (fp16) fused_table_f16_16_8(tab, n); else fused_table_f32_16_8(tab, n);
    } else if (dc <= 32 && dv <= 8) {
        if (fp16) fused_table_f16_32_8(tab, n); else fused_table_f32_32_8(tab, n);
    } else {
        return fail(QLDPC_ERR_UNSUPPORTED,
                    "check degree %d / fault degree %d above the supported 32 / 8", dc, dv);
    }
    return QLDPC_OK;
}

// Places each check's edges on the check's real slots (padding keeps its slots) so that
// the fault pass's warp-wide accesses spread over the 32 shared-memory banks.  A warp
// takes 32 consecutive faults and accesses, for each k, the message of each fault's
// k-th edge: that is one access group, whose cost is its most crowded bank (the
// wavefronts it takes), with the sum of squared bank counts as the tie-breaker.  The
// check rule does not depend on where an edge sits in its check, so every placement
// gives the same messages.  Local search: swap two edges of one check when that
// lowers the cost (equal-cost swaps are taken now and then, from a fixed LCG stream,
// to leave plateaus); at most 8 sweeps, and fewer on large graphs so that a create call
// evaluates about 4 million swaps at most.  bank(i, k) = bank of logical slot k of check
// i; pos[e] = the logical slot of edge e.
template <typename BankFn>
void place_edges(int M, int N, int DV, const int32_t *row_ptr, const int32_t *col_idx,
                 BankFn bank, std::vector<int> &pos) {
    const int E = row_ptr[M];
    std::vector<int> cnt(N, 0), grp(E);
    const size_t G = (size_t)(N + 31) / 32 * DV;
    std::vector<int> hist(G * 32, 0);
    pos.resize(E);
    for (int i = 0; i < M; ++i)
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int j = col_idx[e];
            pos[e] = e - row_ptr[i];
            grp[e] = (j >> 5) * DV + cnt[j]++;  // rows ascending => the fault's k-th edge
            ++hist[(size_t)grp[e] * 32 + bank(i, pos[e])];
        }
    auto cost = [&](int g) {
        const int *h = &hist[(size_t)g * 32];
        int mx = 0, sq = 0;
        for (int b = 0; b < 32; ++b) {
            mx = std::max(mx, h[b]);
            sq += h[b] * h[b];
        }
        return mx * 65536 + sq;
    };
    auto move = [&](int g, int from, int to) {
        --hist[(size_t)g * 32 + from];
        ++hist[(size_t)g * 32 + to];
    };
    long long pairs = 0;
    for (int i = 0; i < M; ++i) {
        const long long d = row_ptr[i + 1] - row_ptr[i];
        pairs += d * (d - 1) / 2;
    }
    const int sweeps = (int)std::max(1LL, std::min(8LL, 4000000LL / std::max(1LL, pairs)));
    uint32_t lcg = 12345u;
    for (int sweep = 0; sweep < sweeps; ++sweep) {
        int improved = 0;
        for (int i = 0; i < M; ++i)
            for (int a = row_ptr[i]; a < row_ptr[i + 1]; ++a)
                for (int b = a + 1; b < row_ptr[i + 1]; ++b) {
                    const int ga = grp[a], gb = grp[b];
                    const int ba = bank(i, pos[a]), bb = bank(i, pos[b]);
                    if (ba == bb) continue;
                    const int before = cost(ga) + (gb != ga ? cost(gb) : 0);
                    move(ga, ba, bb);
                    move(gb, bb, ba);
                    const int after = cost(ga) + (gb != ga ? cost(gb) : 0);
                    lcg = lcg * 1664525u + 1013904223u;
                    if (after < before || (after == before && (lcg >> 30) == 0u)) {
                        std::swap(pos[a], pos[b]);
                        improved += after < before;
                    } else {
                        move(ga, bb, ba);
                        move(gb, ba, bb);
                    }
                }
        if (!improved) break;
    }
}

// Tail continuation: the resuming launch runs the compiled 1024-thread shape with the
// fewest faults per thread that holds N (one block per SM; none holds it: no
// continuation); 4 records per SM.  tail_cut < 0 turns it off, 0 picks T_1 + 8 T_r.
int setup_tail(qldpc_decoder *d, const FusedKernel *tab, int ntab, int tail_cut) {
    if (tail_cut < 0) return QLDPC_OK;
    for (int q = 0; q < ntab; ++q)
        if (tab[q].resume_fn && (long long)tab[q].threads * tab[q].vpt >= d->N &&
            (!d->fk_tail || tab[q].vpt < d->fk_tail->vpt))
            d->fk_tail = &tab[q];
    if (!d->fk_tail) return QLDPC_OK;  // no resuming shape holds the graph
    QL_CUDA(cudaFuncSetAttribute(d->fk_tail->resume_fn,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d->smem));
    int bps = 0;
    QL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, d->fk_tail->resume_fn,
                                                          d->fk_tail->threads, d->smem));
    if (bps < 1) {  // not resident: no continuation
        d->fk_tail = nullptr;
        return QLDPC_OK;
    }
    d->tail_grid = d->num_sms * bps;
    TailCont &tc = d->tail;
    tc.cap = 4 * d->num_sms;
    tc.cut = tail_cut > 0 ? tail_cut : (long long)d->prm.T1 + 8LL * d->prm.T2;
    const size_t rec_bytes = align_up(sizeof(TailRecord) * (size_t)tc.cap, 256);
    QL_CUDA(cudaMalloc(&d->tail_arena, rec_bytes + sizeof(float) * (size_t)tc.cap * d->N));
    tc.rec = static_cast<TailRecord *>(d->tail_arena);
    tc.lam = reinterpret_cast<float *>(static_cast<char *>(d->tail_arena) + rec_bytes);
    tc.count = d->counter + 1;
    tc.mode = 1;
    return QLDPC_OK;
}

int setup_fused(qldpc_decoder *d, const int32_t *row_ptr, const int32_t *col_idx,
                const std::vector<float> &w, const float *gamma, int block_threads,
                int tail_cut) {
    const int M = d->M, N = d->N, E = d->E;
    const FusedKernel *tab = nullptr;
    int ntab = 0;
    int rc = pick_family(d->dc_max, d->dv_max, d->msg_fp16, &tab, &ntab);
    if (rc) return rc;
    const int DC = tab[0].dc, DV = tab[0].dv;
    for (int q = 0; q < ntab && !d->fk; ++q)
        if ((long long)tab[q].threads * tab[q].vpt >= N &&
            (block_threads == 0 || tab[q].threads == block_threads))
            d->fk = &tab[q];
    if (!d->fk)
        return fail(QLDPC_ERR_UNSUPPORTED, "no compiled kernel for N = %d with %d threads", N,
                    block_threads);
    if ((long long)tab[ntab - 1].threads * tab[ntab - 1].vpt >= N) d->fk_trace = &tab[ntab - 1];

    FusedGraph &g = d->fg;
    g.M = M;
    g.N = N;
    g.E = E;
    g.Mp = (M + 31) / 32 * 32;
    g.syn_words = (M + 63) / 64;
    g.cor_words = (N + 63) / 64;
    g.f_words = (2 * g.cor_words + 2 + 3) & ~3;  // whole 16-byte groups
    g.m_words = (M + 31) / 32;

    // message layout (see FusedGraph): rows of DC slots, swizzled inside a row
    const bool half = d->msg_fp16 != 0;
    const int sh = DC >= 32 ? 0 : (DC == 16 ? 1 : 2);
    auto swz = [&](int x) { return (x >> sh) & (DC - 1); };
    auto byte_off = [&](int i, int k) {
        return half ? (((i >> 1) * DC + (k ^ swz(i >> 1))) * 4 + (i & 1) * 2)
                    : ((i * DC + (k ^ swz(i))) * 4);
    };
    const int msg_size = half ? 2 : 4;
    g.msg_bytes = g.Mp * DC * msg_size;
    if ((long long)g.Mp * DC * msg_size >= (1LL << 24))
        return fail(QLDPC_ERR_UNSUPPORTED, "message array above 16 MB");

    std::vector<uint8_t> chk_deg(g.Mp, 0);
    std::vector<int> var_deg(N, 0);
    std::vector<int32_t> var_chk((size_t)N * DV, 0), var_slot((size_t)N * DV, 0);
    std::vector<int32_t> slot_edge((size_t)g.Mp * DC, -1);
    std::vector<uint32_t> pad_mask((size_t)(g.Mp / 2) * DC, 0);
    std::vector<int> pos;
    place_edges(M, N, DV, row_ptr, col_idx,
                [&](int i, int k) { return (byte_off(i, k) >> 2) & 31; }, pos);
    for (int i = 0; i < M; ++i) {
        chk_deg[i] = (uint8_t)(row_ptr[i + 1] - row_ptr[i]);
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int k = pos[e], j = col_idx[e];
            const int off = byte_off(i, k);
            slot_edge[off / msg_size] = e;
            var_chk[(size_t)j * DV + var_deg[j]] = i;
            var_slot[(size_t)j * DV + var_deg[j]++] = off;  // rows ascending => checks ascending
        }
    }
    for (int j = 0; j < N; ++j) var_slot[(size_t)j * DV] |= var_deg[j] << 24;
    for (int i = 0; i < g.Mp; ++i)
        for (int k = chk_deg[i]; k < DC; ++k) {
            const int p = k ^ swz(i >> 1);
            pad_mask[(size_t)(i / 2) * DC + p] |= (i & 1) ? 0xffff0000u : 0x0000ffffu;
        }

    d->smem = fused_smem_bytes(g.msg_bytes, g.f_words, g.syn_words, g.m_words, N);
    int optin = 0;
    QL_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, d->device));
    QL_CUDA(cudaDeviceGetAttribute(&d->num_sms, cudaDevAttrMultiProcessorCount, d->device));
    if (d->smem > (size_t)optin)
        return fail(QLDPC_ERR_UNSUPPORTED, "per-shot state needs %zu B of shared memory, above %d",
                    d->smem, optin);
    QL_CUDA(cudaFuncSetAttribute(d->fk->decode_fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)d->smem));
    QL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d->blocks_per_sm, d->fk->decode_fn,
                                                          d->fk->threads, d->smem));
    if (d->blocks_per_sm < 1)
        return fail(QLDPC_ERR_UNSUPPORTED, "the decode kernel cannot be resident on an SM");
    if (d->fk_trace) {
        d->trace_smem = d->smem;
        QL_CUDA(cudaFuncSetAttribute(d->fk_trace->trace_fn,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d->smem));
    }
    d->block_threads = d->fk->threads;
    d->grid = d->num_sms * d->blocks_per_sm;

    // one device arena for every graph array
    const size_t R1 = (size_t)d->prm.R + 1;
    size_t off[8], o = 0;
    const size_t sizes[8] = {(size_t)g.Mp, sizeof(int32_t) * N * DV, sizeof(uint32_t) * pad_mask.size(),
                             sizeof(int32_t) * N * DV, sizeof(float) * N, sizeof(float) * R1 * N,
                             sizeof(int32_t) * slot_edge.size(), sizeof(unsigned int) * 4};
    for (int q = 0; q < 8; ++q) {
        off[q] = o;
        o = align_up(o + sizes[q], 256);
    }
    QL_CUDA(cudaMalloc(&d->arena, o));
    char *base = static_cast<char *>(d->arena);
    const void *src[7] = {chk_deg.data(), var_chk.data(), pad_mask.data(), var_slot.data(),
                          w.data(), gamma, slot_edge.data()};
    for (int q = 0; q < 7; ++q)
        QL_CUDA(cudaMemcpy(base + off[q], src[q], sizes[q], cudaMemcpyHostToDevice));
    g.chk_deg = reinterpret_cast<const uint8_t *>(base + off[0]);
    g.var_chk = reinterpret_cast<const int32_t *>(base + off[1]);
    g.pad_mask = reinterpret_cast<const uint32_t *>(base + off[2]);
    g.var_slot = reinterpret_cast<const int32_t *>(base + off[3]);
    g.w = reinterpret_cast<const float *>(base + off[4]);
    g.gamma = reinterpret_cast<const float *>(base + off[5]);
    g.slot_edge = reinterpret_cast<const int32_t *>(base + off[6]);
    d->counter = reinterpret_cast<unsigned int *>(base + off[7]);
    QL_CUDA(cudaMemset(d->counter, 0, sizeof(unsigned int) * 4));
    return setup_tail(d, tab, ntab, tail_cut);
}

int setup_baseline(qldpc_decoder *d, const int32_t *row_ptr, const int32_t *col_idx,
                   const std::vector<float> &w, const float *gamma) {
    const int M = d->M, N = d->N, E = d->E;
    if (d->msg_fp16) return fail(QLDPC_ERR_UNSUPPORTED, "the baseline kernel stores float32 messages");
    std::vector<int32_t> var_ptr(N + 1, 0), var_edges(std::max(E, 1)), fill(N, 0);
    for (int e = 0; e < E; ++e) var_ptr[col_idx[e] + 1]++;
    for (int j = 0; j < N; ++j) var_ptr[j + 1] += var_ptr[j];
    for (int e = 0; e < E; ++e) {
        const int j = col_idx[e];
        var_edges[var_ptr[j] + fill[j]++] = e;
    }
    d->smem = baseline_smem_bytes(M, N, E);
    int optin = 0;
    QL_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, d->device));
    QL_CUDA(cudaDeviceGetAttribute(&d->num_sms, cudaDevAttrMultiProcessorCount, d->device));
    if (d->smem > (size_t)optin)
        return fail(QLDPC_ERR_UNSUPPORTED, "baseline kernel needs %zu B of shared memory, above %d",
                    d->smem, optin);
    QL_CUDA(cudaFuncSetAttribute(baseline_fn(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)d->smem));
    QL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d->blocks_per_sm, baseline_fn(), 256,
                                                          d->smem));
    d->block_threads = 256;
    d->grid = 0;
    const size_t R1 = (size_t)d->prm.R + 1;
    size_t off[6], o = 0;
    const size_t sizes[6] = {sizeof(int32_t) * (M + 1), sizeof(int32_t) * std::max(E, 1),
                             sizeof(int32_t) * (N + 1), sizeof(int32_t) * std::max(E, 1),
                             sizeof(float) * N, sizeof(float) * R1 * N};
    for (int q = 0; q < 6; ++q) {
        off[q] = o;
        o = align_up(o + sizes[q], 256);
    }
    QL_CUDA(cudaMalloc(&d->arena, o));
    char *base = static_cast<char *>(d->arena);
    const void *src[6] = {row_ptr, E > 0 ? (const void *)col_idx : (const void *)var_edges.data(),
                          var_ptr.data(), var_edges.data(), w.data(), gamma};
    for (int q = 0; q < 6; ++q)
        QL_CUDA(cudaMemcpy(base + off[q], src[q], sizes[q], cudaMemcpyHostToDevice));
    BaseGraph &g = d->bg;
    g.M = M;
    g.N = N;
    g.E = E;
    g.syn_words = (M + 63) / 64;
    g.cor_words = (N + 63) / 64;
    g.row_ptr = reinterpret_cast<const int32_t *>(base + off[0]);
    g.col_idx = reinterpret_cast<const int32_t *>(base + off[1]);
    g.var_ptr = reinterpret_cast<const int32_t *>(base + off[2]);
    g.var_edges = reinterpret_cast<const int32_t *>(base + off[3]);
    g.w = reinterpret_cast<const float *>(base + off[4]);
    g.gamma = reinterpret_cast<const float *>(base + off[5]);
    return QLDPC_OK;
}

// The persistent decode over the shots of `map`, with the tail continuation when the
// handle has one: the first launch (work counter `counter`, zeroed here) suspends long
// shots into the handle's records, the second launch (one block per SM of the tail
// shape) finishes them.  Both on `st`, so the pair can be captured in a CUDA graph.
int launch_persistent(const qldpc_decoder *d, const uint64_t *syn, int64_t B, DecodeOut out,
                      unsigned int *counter, ShotMap map, cudaStream_t st) {
    const bool tail = d->fk_tail != nullptr;
    QL_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned int), st));
    if (tail) QL_CUDA(cudaMemsetAsync(d->counter + 1, 0, 2 * sizeof(unsigned int), st));
    const int grid = (int)std::min<int64_t>(d->grid, B);
    QL_CUDA(d->fk->launch_decode(dim3(grid), d->smem, st, d->fg, d->prm, syn, (int)B, out,
                                 counter, map, d->tail));
    if (tail)
        QL_CUDA(d->fk_tail->launch_resume(dim3(std::min(d->tail_grid, d->tail.cap)), d->smem, st,
                                          d->fg, d->prm, syn, (int)B, out, d->counter + 2, map,
                                          d->tail));
    return QLDPC_OK;
}

int launch(qldpc_decoder *d, const uint64_t *syn, int64_t B, DecodeOut out, cudaStream_t st) {
    if (d->kernel == QLDPC_KERNEL_BASELINE) {
        QL_CUDA(launch_baseline((int)B, d->block_threads, d->smem, st, d->bg, d->prm, syn, out));
        return QLDPC_OK;
    }
    return launch_persistent(d, syn, B, out, d->counter,
                             ShotMap{nullptr, nullptr, d->fg.syn_words, d->fg.cor_words}, st);
}


}  // namespace

extern "C" {

int qldpc_create(qldpc_decoder **out, int32_t M, int32_t N, const int32_t *row_ptr,
                 const int32_t *col_idx, const double *priors, const qldpc_relay_params *prm,
                 int device) {
    g_last_error.clear();
    if (!out) return fail(QLDPC_ERR_INVALID_ARG, "out must not be NULL");
    *out = nullptr;
    int rc = validate_graph(M, N, row_ptr, col_idx, priors);
    if (rc) return rc;
    rc = validate_params(prm, N);
    if (rc) return rc;
    int ndev = 0;
    QL_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(QLDPC_ERR_INVALID_ARG, "device %d of %d", device, ndev);
    DeviceGuard guard(device);
    QL_CUDA(guard.err);

    qldpc_decoder *d = new (std::nothrow) qldpc_decoder();
    if (!d) return fail(QLDPC_ERR_OOM, "host allocation failed");
    d->device = device;
    d->M = M;
    d->N = N;
    d->E = row_ptr[M];
    std::vector<int> vdeg(N, 0);
    for (int e = 0; e < d->E; ++e) vdeg[col_idx[e]]++;
    for (int i = 0; i < M; ++i) d->dc_max = std::max(d->dc_max, row_ptr[i + 1] - row_ptr[i]);
    for (int j = 0; j < N; ++j) d->dv_max = std::max(d->dv_max, vdeg[j]);
    d->msg_fp16 = prm->msg_precision == QLDPC_MSG_FP16;
    d->kernel = prm->kernel == QLDPC_KERNEL_BASELINE ? QLDPC_KERNEL_BASELINE : QLDPC_KERNEL_FUSED;
    d->prm.R = prm->legs_after_first;
    d->prm.T1 = prm->iters_first;
    d->prm.T2 = prm->iters_later;
    d->prm.S = prm->stop_after_solutions;
    d->prm.warm_mode = prm->warm_start_mode;
    d->prm.max_iters = prm->max_total_iters;
    d->prm.clip = prm->llr_clip > 0.0f ? prm->llr_clip : (d->msg_fp16 ? 65504.0f : 1e30f);

    // prior LLRs w_j = log((1 - p_j) / p_j), computed in double and rounded once
    std::vector<float> w(N);
    for (int j = 0; j < N; ++j) w[j] = (float)std::log((1.0 - priors[j]) / priors[j]);

    rc = d->kernel == QLDPC_KERNEL_BASELINE
             ? setup_baseline(d, row_ptr, col_idx, w, prm->gamma_table)
             : setup_fused(d, row_ptr, col_idx, w, prm->gamma_table, prm->block_threads,
                           prm->tail_cut_iters);
    if (rc == QLDPC_OK) {
        cudaError_t e = cudaStreamCreateWithFlags(&d->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) rc = fail(QLDPC_ERR_CUDA, "stream creation failed: %s", cudaGetErrorString(e));
    }
    if (rc == QLDPC_OK && d->kernel == QLDPC_KERNEL_FUSED) rc = lookup_static_scratch(d);
    if (rc != QLDPC_OK) {
        std::string msg = g_last_error;
        qldpc_destroy(d);
        g_last_error = msg;
        return rc;
    }
    *out = d;
    return QLDPC_OK;
}

int qldpc_decode_batch(qldpc_decoder *d, const uint64_t *syndromes, int64_t B,
                       uint64_t *corrections, int32_t *legs_used, uint8_t *converged,
                       int32_t *iters, void *stream) {
    g_last_error.clear();
    int rc = check_batch(d, syndromes, B, corrections);
    if (rc) return rc;
    if (B == 0) return QLDPC_OK;
    DeviceGuard guard(d->device);
    QL_CUDA(guard.err);
    const void *ptrs[5] = {syndromes, corrections, legs_used, converged, iters};
    for (int q = 0; q < 5; ++q)
        if (ptrs[q] && !is_device_ptr(ptrs[q]))
            return fail(QLDPC_ERR_INVALID_ARG, "argument %d is not device memory", q);
    return launch(d, syndromes, B, DecodeOut{corrections, legs_used, converged, iters},
                  static_cast<cudaStream_t>(stream));
}

int qldpc_decode_batch_host(qldpc_decoder *d, const uint64_t *syndromes, int64_t B,
                            uint64_t *corrections, int32_t *legs_used, uint8_t *converged,
                            int32_t *iters) {
    g_last_error.clear();
    int rc = check_batch(d, syndromes, B, corrections);
    if (rc) return rc;
    if (B == 0) return QLDPC_OK;
    DeviceGuard guard(d->device);
    QL_CUDA(guard.err);
    const int sw = (d->M + 63) / 64, cw = (d->N + 63) / 64;
    const size_t s_syn = align_up(8 * (size_t)sw * B, 256), s_cor = align_up(8 * (size_t)cw * B, 256);
    const size_t s_i32 = align_up(4 * (size_t)B, 256), s_u8 = align_up((size_t)B, 256);
    if (B > d->stage_B) {
        if (d->stage) QL_CUDA(cudaFree(d->stage));
        d->stage = nullptr;
        d->stage_B = 0;
        QL_CUDA(cudaMalloc(&d->stage, s_syn + s_cor + 2 * s_i32 + s_u8));
        d->stage_B = B;
    }
    char *base = static_cast<char *>(d->stage);
    uint64_t *dsyn = reinterpret_cast<uint64_t *>(base);
    uint64_t *dcor = reinterpret_cast<uint64_t *>(base + s_syn);
    int32_t *dlegs = reinterpret_cast<int32_t *>(base + s_syn + s_cor);
    int32_t *diters = reinterpret_cast<int32_t *>(base + s_syn + s_cor + s_i32);
    uint8_t *dconv = reinterpret_cast<uint8_t *>(base + s_syn + s_cor + 2 * s_i32);
    cudaStream_t st = d->stream;
    QL_CUDA(cudaMemcpyAsync(dsyn, syndromes, 8 * (size_t)sw * B, cudaMemcpyHostToDevice, st));
    rc = launch(d, dsyn, B, DecodeOut{dcor, legs_used ? dlegs : nullptr, converged ? dconv : nullptr,
                                      iters ? diters : nullptr}, st);
    if (rc) return rc;
    QL_CUDA(cudaMemcpyAsync(corrections, dcor, 8 * (size_t)cw * B, cudaMemcpyDeviceToHost, st));
    if (legs_used) QL_CUDA(cudaMemcpyAsync(legs_used, dlegs, 4 * (size_t)B, cudaMemcpyDeviceToHost, st));
    if (iters) QL_CUDA(cudaMemcpyAsync(iters, diters, 4 * (size_t)B, cudaMemcpyDeviceToHost, st));
    if (converged) QL_CUDA(cudaMemcpyAsync(converged, dconv, (size_t)B, cudaMemcpyDeviceToHost, st));
    QL_CUDA(cudaStreamSynchronize(st));
    return QLDPC_OK;
}

}  // extern "C"

// ---- host-buffer decode without any allocation ------------------------------------
//
// qldpc_decode_batch_host stages batches in device buffers that it allocates on
// first use and whenever a batch is larger than any before.  Callers that must not
// allocate device memory while decoding (a real-time loop with a fixed memory
// budget, a process whose device memory belongs to another allocator) use
// qldpc_decode_batch_host_static instead: its staging area and the fused kernel's
// work counter live in the file-scope array below, which every GPU that loads the
// library holds until the process exits.

static __device__ __align__(256) unsigned char g_static_scratch[QLDPC_STATIC_SCRATCH_BYTES];

namespace {

// Device address of g_static_scratch in the context current at set-up (qldpc_create,
// with the handle's device current).  Host code must not hand the symbol itself to a
// kernel: on the host it is only a stand-in.  Keeping the address in the handle ties it
// to the context the handle lives in; a handle does not outlive a cudaDeviceReset.
int lookup_static_scratch(qldpc_decoder *d) {
    void *p = nullptr;
    QL_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
    d->static_scratch = static_cast<unsigned char *>(p);
    return QLDPC_OK;
}

// Bytes of the static array a batch of B shots takes: the work counter, then syndromes,
// corrections, legs, iterations and converged flags, each 256-byte aligned.
size_t static_need(int sw, int cw, int64_t B) {
    return 256 + align_up(8 * (size_t)sw * B, 256) + align_up(8 * (size_t)cw * B, 256) +
           2 * align_up(4 * (size_t)B, 256) + align_up((size_t)B, 256);
}

// Largest batch that fits the static array (static_need grows with B).
int64_t static_max_shots(int sw, int cw) {
    int64_t lo = 0, hi = (int64_t)QLDPC_STATIC_SCRATCH_BYTES;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        if (static_need(sw, cw, mid) <= (size_t)QLDPC_STATIC_SCRATCH_BYTES) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace

extern "C" int qldpc_decode_batch_host_static(qldpc_decoder *d, const uint64_t *syndromes,
                                              int64_t B, uint64_t *corrections,
                                              int32_t *legs_used, uint8_t *converged,
                                              int32_t *iters) {
    g_last_error.clear();
    int rc = check_batch(d, syndromes, B, corrections);
    if (rc) return rc;
    if (d->kernel != QLDPC_KERNEL_FUSED)
        return fail(QLDPC_ERR_UNSUPPORTED, "the static-scratch path runs the fused kernel only");
    if (B == 0) return QLDPC_OK;
    const int sw = (d->M + 63) / 64, cw = (d->N + 63) / 64;
    const size_t s_cnt = 256, s_syn = align_up(8 * (size_t)sw * B, 256);
    const size_t s_cor = align_up(8 * (size_t)cw * B, 256);
    const size_t s_i32 = align_up(4 * (size_t)B, 256);
    const size_t need = static_need(sw, cw, B);
    if (need > (size_t)QLDPC_STATIC_SCRATCH_BYTES)
        return fail(QLDPC_ERR_INVALID_ARG,
                    "a batch of %lld shots needs %zu bytes of static scratch, above the %d-byte "
                    "maximum (at most %lld shots of this code per call)",
                    (long long)B, need, QLDPC_STATIC_SCRATCH_BYTES,
                    (long long)static_max_shots(sw, cw));
    if (!d->static_scratch)
        return fail(QLDPC_ERR_UNSUPPORTED, "the handle has no static scratch address");
    DeviceGuard guard(d->device);
    QL_CUDA(guard.err);
    unsigned char *base = d->static_scratch;
    unsigned int *counter = reinterpret_cast<unsigned int *>(base);
    uint64_t *dsyn = reinterpret_cast<uint64_t *>(base + s_cnt);
    uint64_t *dcor = reinterpret_cast<uint64_t *>(base + s_cnt + s_syn);
    int32_t *dlegs = reinterpret_cast<int32_t *>(base + s_cnt + s_syn + s_cor);
    int32_t *diters = reinterpret_cast<int32_t *>(base + s_cnt + s_syn + s_cor + s_i32);
    uint8_t *dconv = reinterpret_cast<uint8_t *>(base + s_cnt + s_syn + s_cor + 2 * s_i32);
    cudaStream_t st = d->stream;
    QL_CUDA(cudaMemcpyAsync(dsyn, syndromes, 8 * (size_t)sw * B, cudaMemcpyHostToDevice, st));
    rc = launch_persistent(d, dsyn, B,
                           DecodeOut{dcor, legs_used ? dlegs : nullptr, converged ? dconv : nullptr,
                                     iters ? diters : nullptr},
                           counter, ShotMap{nullptr, nullptr, sw, cw}, st);
    if (rc) return rc;
    QL_CUDA(cudaMemcpyAsync(corrections, dcor, 8 * (size_t)cw * B, cudaMemcpyDeviceToHost, st));
    if (legs_used) QL_CUDA(cudaMemcpyAsync(legs_used, dlegs, 4 * (size_t)B, cudaMemcpyDeviceToHost, st));
    if (iters) QL_CUDA(cudaMemcpyAsync(iters, diters, 4 * (size_t)B, cudaMemcpyDeviceToHost, st));
    if (converged) QL_CUDA(cudaMemcpyAsync(converged, dconv, (size_t)B, cudaMemcpyDeviceToHost, st));
    QL_CUDA(cudaStreamSynchronize(st));
    return QLDPC_OK;
}

extern "C" {

int qldpc_decode_batch_multi(qldpc_decoder *const *decoders, int32_t n_codes,
                              const int32_t *code_of_shot, const uint64_t *syndromes,
                              int32_t syndrome_stride, int64_t B, uint64_t *corrections,
                              int32_t correction_stride, int32_t *legs_used, uint8_t *converged,
                              int32_t *iters, void *stream) {
    g_last_error.clear();
    if (!decoders || n_codes < 1 || n_codes > kMaxMultiCodes)
        return fail(QLDPC_ERR_INVALID_ARG, "need 1..%d decoders", kMaxMultiCodes);
    if (B < 0 || B > 0x7fffffffLL) return fail(QLDPC_ERR_INVALID_ARG, "batch size out of range");
    if (B == 0) return QLDPC_OK;
    if (!code_of_shot || !syndromes || !corrections)
        return fail(QLDPC_ERR_INVALID_ARG, "code_of_shot, syndromes and corrections are required");
    const qldpc_decoder *d0 = decoders[0];
    int max_sw = 0, max_cw = 0, big = 0;
    for (int c = 0; c < n_codes; ++c) {
        const qldpc_decoder *d = decoders[c];
        if (!d) return fail(QLDPC_ERR_INVALID_ARG, "decoder %d is NULL", c);
        if (d->kernel != QLDPC_KERNEL_FUSED)
            return fail(QLDPC_ERR_UNSUPPORTED, "mixed batches need fused-kernel decoders");
        if (d->device != d0->device || d->msg_fp16 != d0->msg_fp16 || d->fk->dc != d0->fk->dc ||
            d->fk->dv != d0->fk->dv)
            return fail(QLDPC_ERR_UNSUPPORTED,
                        "decoders of a mixed batch must share device, message precision and "
                        "degree family (decoder %d differs)", c);
        max_sw = std::max(max_sw, d->fg.syn_words);
        max_cw = std::max(max_cw, d->fg.cor_words);
        if (d->fg.N > decoders[big]->fg.N) big = c;
    }
    if (syndrome_stride < max_sw || correction_stride < max_cw)
        return fail(QLDPC_ERR_INVALID_ARG, "row strides %d/%d below the widest code's %d/%d words",
                    syndrome_stride, correction_stride, max_sw, max_cw);
    DeviceGuard guard(d0->device);
    QL_CUDA(guard.err);
    const void *ptrs[6] = {code_of_shot, syndromes, corrections, legs_used, converged, iters};
    for (int q = 0; q < 6; ++q)
        if (ptrs[q] && !is_device_ptr(ptrs[q]))
            return fail(QLDPC_ERR_INVALID_ARG, "argument %d is not device memory", q);
    // the kernel instance of the code with the most faults serves every code
    const qldpc_decoder *db = decoders[big];
    const FusedKernel *fk = db->fk;
    MultiTable tab{};
    tab.n = n_codes;
    size_t smem = 0;
    for (int c = 0; c < n_codes; ++c) {
        tab.g[c] = decoders[c]->fg;
        tab.p[c] = decoders[c]->prm;
        smem = std::max(smem, decoders[c]->smem);
    }
    QL_CUDA(cudaFuncSetAttribute(fk->multi_fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    int bps = 0;
    QL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fk->multi_fn, fk->threads, smem));
    if (bps < 1) return fail(QLDPC_ERR_UNSUPPORTED, "mixed-batch kernel cannot be resident");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    QL_CUDA(cudaMemsetAsync(d0->counter, 0, sizeof(unsigned int), st));
    const int grid = (int)std::min<int64_t>((int64_t)db->num_sms * bps, B);
    QL_CUDA(fk->launch_multi(dim3(grid), smem, st, tab, code_of_shot, syndromes, syndrome_stride,
                             correction_stride, (int)B,
                             DecodeOut{corrections, legs_used, converged, iters}, d0->counter));
    return QLDPC_OK;
}

}  // extern "C"

namespace {

// Shots of a mixed batch sorted into one index list per code ([n_codes][B], in any
// order within a code; counts[c] = length of list c).  Shots with an unknown code id
// get legs 0, converged 0 and iters -1, as in the single-launch mixed kernel.
__global__ void partition_shots(const int32_t *__restrict__ code_of_shot, int B, int n_codes,
                                int32_t *counts, int32_t *lists, DecodeOut out) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
        const int c = code_of_shot[b];
        if (c >= 0 && c < n_codes) {
            const int k = atomicAdd(counts + c, 1);
            lists[(size_t)c * B + k] = b;
        } else {
            if (out.legs) out.legs[b] = 0;
            if (out.conv) out.conv[b] = 0;
            if (out.iters) out.iters[b] = -1;
        }
    }
}

}  // namespace

extern "C" {

uint64_t qldpc_grouped_workspace_bytes(int32_t n_codes, int64_t B) {
    if (n_codes < 1 || B < 0) return 0;
    return (uint64_t)align_up(sizeof(int32_t) * (size_t)n_codes, 256) +
           sizeof(int32_t) * (uint64_t)n_codes * (uint64_t)B;
}

int qldpc_decode_batch_grouped(qldpc_decoder *const *decoders, int32_t n_codes,
                               const int32_t *code_of_shot, const uint64_t *syndromes,
                               int32_t syndrome_stride, int64_t B, uint64_t *corrections,
                               int32_t correction_stride, int32_t *legs_used,
                               uint8_t *converged, int32_t *iters, void *workspace,
                               uint64_t workspace_bytes, void *stream) {
    g_last_error.clear();
    if (!decoders || n_codes < 1 || n_codes > kMaxMultiCodes)
        return fail(QLDPC_ERR_INVALID_ARG, "need 1..%d decoders", kMaxMultiCodes);
    if (B < 0 || B > 0x7fffffffLL) return fail(QLDPC_ERR_INVALID_ARG, "batch size out of range");
    if (B == 0) return QLDPC_OK;
    if (!code_of_shot || !syndromes || !corrections || !workspace)
        return fail(QLDPC_ERR_INVALID_ARG,
                    "code_of_shot, syndromes, corrections and workspace are required");
    if (workspace_bytes < qldpc_grouped_workspace_bytes(n_codes, B))
        return fail(QLDPC_ERR_INVALID_ARG, "workspace of %llu bytes below the %llu needed",
                    (unsigned long long)workspace_bytes,
                    (unsigned long long)qldpc_grouped_workspace_bytes(n_codes, B));
    const qldpc_decoder *d0 = decoders[0];
    for (int c = 0; c < n_codes; ++c) {
        const qldpc_decoder *d = decoders[c];
        if (!d) return fail(QLDPC_ERR_INVALID_ARG, "decoder %d is NULL", c);
        if (d->kernel != QLDPC_KERNEL_FUSED)
            return fail(QLDPC_ERR_UNSUPPORTED, "grouped batches need fused-kernel decoders");
        if (d->device != d0->device)
            return fail(QLDPC_ERR_UNSUPPORTED, "decoders of a batch must share the device");
        for (int c2 = 0; c2 < c; ++c2)
            if (decoders[c2] == d)
                return fail(QLDPC_ERR_INVALID_ARG, "decoder %d appears twice", c);
        if (syndrome_stride < d->fg.syn_words || correction_stride < d->fg.cor_words)
            return fail(QLDPC_ERR_INVALID_ARG, "row strides %d/%d below code %d's %d/%d words",
                        syndrome_stride, correction_stride, c, d->fg.syn_words, d->fg.cor_words);
    }
    DeviceGuard guard(d0->device);
    QL_CUDA(guard.err);
    const void *ptrs[7] = {code_of_shot, syndromes, corrections, legs_used, converged, iters,
                           workspace};
    for (int q = 0; q < 7; ++q)
        if (ptrs[q] && !is_device_ptr(ptrs[q]))
            return fail(QLDPC_ERR_INVALID_ARG, "argument %d is not device memory", q);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t *counts = static_cast<int32_t *>(workspace);
    int32_t *lists = reinterpret_cast<int32_t *>(static_cast<char *>(workspace) +
                                                 align_up(sizeof(int32_t) * n_codes, 256));
    const DecodeOut out{corrections, legs_used, converged, iters};
    QL_CUDA(cudaMemsetAsync(counts, 0, sizeof(int32_t) * n_codes, st));
    const int pgrid = (int)std::min<int64_t>((B + 255) / 256, (int64_t)d0->num_sms * 8);
    partition_shots<<<pgrid, 256, 0, st>>>(code_of_shot, (int)B, n_codes, counts, lists, out);
    QL_CUDA(cudaGetLastError());
    // each code with its own kernel shape, largest code first
    int order[kMaxMultiCodes];
    for (int c = 0; c < n_codes; ++c) order[c] = c;
    std::sort(order, order + n_codes,
              [&](int a, int b) { return decoders[a]->fg.E > decoders[b]->fg.E; });
    for (int q = 0; q < n_codes; ++q) {
        const int c = order[q];
        qldpc_decoder *d = decoders[c];
        const int rc = launch_persistent(d, syndromes, B, out, d->counter,
                                         ShotMap{lists + (size_t)c * B, counts + c,
                                                 syndrome_stride, correction_stride},
                                         st);
        if (rc) return rc;
    }
    return QLDPC_OK;
}

int qldpc_trace_first_leg(qldpc_decoder *d, const uint64_t *syndromes, int64_t B, int32_t T,
                          float *marginals, float *nu, float *mu, void *stream) {
    g_last_error.clear();
    if (!d) return fail(QLDPC_ERR_INVALID_ARG, "decoder handle is NULL");
    if (d->kernel != QLDPC_KERNEL_FUSED || !d->fk_trace)
        return fail(QLDPC_ERR_UNSUPPORTED, "tracing needs the fused kernel");
    if (B < 0 || B > 0x7fffffffLL || T < 0) return fail(QLDPC_ERR_INVALID_ARG, "bad B or T");
    if (B == 0 || T == 0) return QLDPC_OK;
    if (!syndromes) return fail(QLDPC_ERR_INVALID_ARG, "syndromes must not be NULL");
    DeviceGuard guard(d->device);
    QL_CUDA(guard.err);
    const void *ptrs[4] = {syndromes, marginals, nu, mu};
    for (int q = 0; q < 4; ++q)
        if (ptrs[q] && !is_device_ptr(ptrs[q]))
            return fail(QLDPC_ERR_INVALID_ARG, "argument %d is not device memory", q);
    QL_CUDA(d->fk_trace->launch_trace(dim3((unsigned)B), d->trace_smem,
                                      static_cast<cudaStream_t>(stream), d->fg, d->prm,
                                      syndromes, (int)B, T, marginals, nu, mu));
    return QLDPC_OK;
}

int qldpc_get_info(const qldpc_decoder *d, qldpc_info *info) {
    if (!d || !info) return fail(QLDPC_ERR_INVALID_ARG, "NULL argument");
    info->M = d->M;
    info->N = d->N;
    info->E = d->E;
    info->max_check_degree = d->dc_max;
    info->max_fault_degree = d->dv_max;
    info->kernel = d->kernel;
    info->msg_precision = d->msg_fp16 ? QLDPC_MSG_FP16 : QLDPC_MSG_FP32;
    info->block_threads = d->block_threads;
    info->blocks_per_sm = d->blocks_per_sm;
    info->num_sms = d->num_sms;
    info->grid_blocks = d->grid;
    info->smem_bytes = (int32_t)d->smem;
    info->syndrome_words = (d->M + 63) / 64;
    info->correction_words = (d->N + 63) / 64;
    info->tail_cut_iters = d->fk_tail ? (int32_t)d->tail.cut : -1;
    info->tail_block_threads = d->fk_tail ? d->fk_tail->threads : 0;
    info->tail_records = d->fk_tail ? d->tail.cap : 0;
    return QLDPC_OK;
}

void qldpc_destroy(qldpc_decoder *d) {
    if (!d) return;
    DeviceGuard guard(d->device);
    if (d->stream) {
        cudaStreamSynchronize(d->stream);
        cudaStreamDestroy(d->stream);
    }
    if (d->arena) cudaFree(d->arena);  // cudaFree waits for work that may still use it
    if (d->tail_arena) cudaFree(d->tail_arena);
    if (d->stage) cudaFree(d->stage);
    delete d;
}

const char *qldpc_status_string(int status) {
    switch (status) {
        case QLDPC_OK: return "ok";
        case QLDPC_ERR_INVALID_ARG: return "invalid argument";
        case QLDPC_ERR_CUDA: return "CUDA error";
        case QLDPC_ERR_OOM: return "out of memory";
        case QLDPC_ERR_UNSUPPORTED: return "unsupported graph or configuration";
        default: return "unknown status";
    }
}

const char *qldpc_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

