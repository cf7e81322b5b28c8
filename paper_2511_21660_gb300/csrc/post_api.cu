// Host side of the post-processors' C ABI (include/qldpc.h: qldpc_osd_*, qldpc_cluster_*):
// the fused-layout graph of their plain BP, the check-to-fault table, kernel choice and
// residency, the list of shots to post-process, launches.
#include <algorithm>
#include <cmath>
#include <vector>

#include "api_common.h"
#include "post_internal.h"

using namespace qldpc;

// ---- filtered-OSD post-processor ----------------------------------------------------

namespace {

// The faults of each check in CSR order, -1 past the check's degree: [Mp][DC].
std::vector<int32_t> check_faults(int M, int Mp, int DC, const int32_t *row_ptr,
                                  const int32_t *col_idx) {
    std::vector<int32_t> cv((size_t)Mp * DC, -1);
    for (int i = 0; i < M; ++i)
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            cv[(size_t)i * DC + (e - row_ptr[i])] = col_idx[e];
    return cv;
}

// The graph of a post-processor: a fused-layout decoder whose single gamma row is all
// zeros, so that its first leg is plain min-sum BP of `bp_iters` iterations.
int create_plain_bp(qldpc_decoder **out, int32_t M, int32_t N, const int32_t *row_ptr,
                    const int32_t *col_idx, const double *priors, int bp_iters, int device) {
    std::vector<float> zeros((size_t)N, 0.0f);
    qldpc_relay_params rp{};
    rp.tail_cut_iters = -1;
    rp.legs_after_first = 0;
    rp.iters_first = bp_iters > 0 ? bp_iters : 1;
    rp.iters_later = 1;
    rp.max_total_iters = 0;
    rp.stop_after_solutions = 1;
    rp.warm_start_mode = 0;
    rp.msg_precision = QLDPC_MSG_FP32;
    rp.kernel = QLDPC_KERNEL_FUSED;
    rp.block_threads = 0;
    rp.llr_clip = 0.0f;
    rp.gamma_table = zeros.data();
    return qldpc_create(out, M, N, row_ptr, col_idx, priors, &rp, device);
}

// Shared memory attribute, occupancy and grid of a post-processing kernel.
cudaError_t configure_kernel(const void *fn, int threads, size_t smem, int device, int num_sms,
                             int *grid, bool *fits) {
    int optin = 0, bps = 0;
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    *fits = e == cudaSuccess && smem <= (size_t)optin;
    if (e != cudaSuccess || !*fits) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, threads, smem);
    *fits = e == cudaSuccess && bps >= 1;
    *grid = num_sms * std::max(bps, 1);
    return e;
}

}  // namespace

// The shots a post-processor is to take: the indices b with skip[b] == 0, in any order
// (each shot's result depends on its own inputs only), appended to list by warp-wide
// ballots; count ends as their number.  Skipped shots get their status (and the extra
// per-shot output) 0 here, so the post-processor visits only the listed shots.
__global__ void compact_active(const uint8_t *__restrict__ skip, int B, int32_t *list,
                               unsigned int *count, int32_t *status, int32_t *extra) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = b < B && !skip[b];
    if (b < B && !act) {
        status[b] = 0;
        if (extra) extra[b] = 0;
    }
    const unsigned m = __ballot_sync(0xffffffffu, act);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(count, (unsigned)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (act) list[base + __popc(m & ((1u << lane) - 1u))] = b;
}

// Post-processor work list: with a skip mask, the listed shots (the list grows with B on
// the host, which then waits for the device); without one, every shot.  counter[0] is
// the work counter, counter[1] the list's length.
struct WorkList {
    int32_t *list = nullptr;
    int64_t cap = 0;
};

static cudaError_t prepare_work(WorkList &w, const uint8_t *skip, int64_t B, int32_t *status,
                                int32_t *extra, unsigned int *counter, cudaStream_t st,
                                const int32_t **list) {
    cudaError_t e = cudaMemsetAsync(counter, 0, 2 * sizeof(unsigned int), st);
    *list = nullptr;
    if (e != cudaSuccess || !skip) return e;
    if (B > w.cap) {
        if (w.list) {
            e = cudaStreamSynchronize(st);
            if (e == cudaSuccess) e = cudaFree(w.list);
            w.list = nullptr;
            w.cap = 0;
            if (e != cudaSuccess) return e;
        }
        e = cudaMalloc(&w.list, sizeof(int32_t) * (size_t)B);
        if (e != cudaSuccess) return e;
        w.cap = B;
    }
    compact_active<<<(unsigned)((B + 255) / 256), 256, 0, st>>>(skip, (int)B, w.list, counter + 1,
                                                               status, extra);
    *list = w.list;
    return cudaGetLastError();
}

struct qldpc_osd {
    int device = 0;
    qldpc_decoder *bp = nullptr;  // fused graph of H (float32 messages, gamma row of zeros)
    const OsdKernel *k = nullptr;
    OsdArgs args{};
    void *arena = nullptr;        // chk_var and the work counters
    unsigned int *counter = nullptr;
    WorkList work;
    size_t smem = 0;
    int grid = 0;
};

extern "C" {

int qldpc_osd_create(qldpc_osd **out, int32_t M, int32_t N, const int32_t *row_ptr,
                     const int32_t *col_idx, const double *priors,
                     const qldpc_osd_params *params, int device) {
    last_error().clear();
    if (!out) return fail(QLDPC_ERR_INVALID_ARG, "out must not be NULL");
    *out = nullptr;
    if (!params) return fail(QLDPC_ERR_INVALID_ARG, "params must not be NULL");
    if (params->bp_iters < 0) return fail(QLDPC_ERR_INVALID_ARG, "bp_iters < 0");
    if (!std::isfinite(params->llr_confident))
        return fail(QLDPC_ERR_INVALID_ARG, "llr_confident is not finite");
    if (params->max_candidates < 1 || params->max_candidates > kOsdMaxCandidates)
        return fail(QLDPC_ERR_INVALID_ARG, "max_candidates %d outside 1..%d",
                    params->max_candidates, kOsdMaxCandidates);
    int rc = validate_graph(M, N, row_ptr, col_idx, priors);
    if (rc) return rc;
    if (N > 32767) return fail(QLDPC_ERR_UNSUPPORTED, "N = %d above 32767", N);
    if (M > 32767) return fail(QLDPC_ERR_UNSUPPORTED, "M = %d above 32767", M);

    qldpc_osd *o = new (std::nothrow) qldpc_osd();
    if (!o) return fail(QLDPC_ERR_OOM, "host allocation failed");
    o->device = device;
    rc = create_plain_bp(&o->bp, M, N, row_ptr, col_idx, priors, params->bp_iters, device);
    if (rc) {
        delete o;
        return rc;
    }
    DeviceGuard guard(device);
    const qldpc_decoder *d = o->bp;
    const int DC = d->fk->dc, DV = d->fk->dv;
    const OsdKernel *tab = nullptr;
    int ntab = 0;
    osd_table(&tab, &ntab);
    for (int q = 0; q < ntab && !o->k; ++q)
        if (tab[q].dc == DC && tab[q].dv == DV && (long long)tab[q].threads * tab[q].vpt >= N)
            o->k = &tab[q];
    auto bail = [&](int code) {
        std::string msg = last_error();
        qldpc_osd_destroy(o);
        last_error() = msg;
        return code;
    };
    if (!o->k) {
        fail(QLDPC_ERR_UNSUPPORTED, "no compiled OSD kernel for N = %d", N);
        return bail(QLDPC_ERR_UNSUPPORTED);
    }
    OsdArgs &a = o->args;
    a.bp_iters = params->bp_iters;
    a.llr_conf = params->llr_confident;
    a.max_cand = params->max_candidates;
    a.W = (a.max_cand + 31) / 32;
    a.KP = 1;
    while (a.KP < a.max_cand) a.KP <<= 1;

    const std::vector<int32_t> chk_var = check_faults(M, d->fg.Mp, DC, row_ptr, col_idx);
    const size_t cv_bytes = align_up(sizeof(int32_t) * chk_var.size(), 256);
    cudaError_t e = cudaMalloc(&o->arena, cv_bytes + 256);
    if (e != cudaSuccess) {
        fail(QLDPC_ERR_OOM, "cudaMalloc failed: %s", cudaGetErrorString(e));
        return bail(QLDPC_ERR_OOM);
    }
    e = cudaMemcpy(o->arena, chk_var.data(), sizeof(int32_t) * chk_var.size(),
                   cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        a.chk_var = static_cast<const int32_t *>(o->arena);
        o->counter = reinterpret_cast<unsigned int *>(static_cast<char *>(o->arena) + cv_bytes);
        o->smem = osd_smem_bytes(d->fg, a);
        bool fits = false;
        e = configure_kernel(o->k->fn, o->k->threads, o->smem, device, d->num_sms, &o->grid,
                             &fits);
        if (e == cudaSuccess && !fits) {
            fail(QLDPC_ERR_UNSUPPORTED, "the OSD stage (%zu B of shared memory) cannot be resident",
                 o->smem);
            return bail(QLDPC_ERR_UNSUPPORTED);
        }
    }
    if (e != cudaSuccess) {
        fail(QLDPC_ERR_CUDA, "OSD set-up failed: %s", cudaGetErrorString(e));
        return bail(QLDPC_ERR_CUDA);
    }
    *out = o;
    return QLDPC_OK;
}

int qldpc_osd_decode_batch(qldpc_osd *o, const uint64_t *syndromes, int64_t B,
                           const uint8_t *skip, uint64_t *corrections, int32_t *status,
                           int32_t *n_candidates, void *stream) {
    last_error().clear();
    if (!o) return fail(QLDPC_ERR_INVALID_ARG, "OSD handle is NULL");
    int rc = check_batch(o->bp, syndromes, B, corrections);
    if (rc) return rc;
    if (B > 0 && !status) return fail(QLDPC_ERR_INVALID_ARG, "status must not be NULL");
    if (B == 0) return QLDPC_OK;
    DeviceGuard guard(o->device);
    QL_CUDA(guard.err);
    const void *ptrs[5] = {syndromes, skip, corrections, status, n_candidates};
    for (int q = 0; q < 5; ++q)
        if (ptrs[q] && !is_device_ptr(ptrs[q]))
            return fail(QLDPC_ERR_INVALID_ARG, "argument %d is not device memory", q);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int32_t *list = nullptr;
    QL_CUDA(prepare_work(o->work, skip, B, status, n_candidates, o->counter, st, &list));
    const int grid = (int)std::min<int64_t>(o->grid, B);
    QL_CUDA(o->k->launch(dim3(grid), o->smem, st, o->bp->fg, o->bp->prm, o->args, syndromes,
                         list, (int)B, OsdOut{corrections, status, n_candidates}, o->counter));
    return QLDPC_OK;
}

void qldpc_osd_destroy(qldpc_osd *o) {
    if (!o) return;
    {
        DeviceGuard guard(o->device);
        if (o->arena) cudaFree(o->arena);  // waits for work that may still use it
        if (o->work.list) cudaFree(o->work.list);
    }
    qldpc_destroy(o->bp);
    delete o;
}

}  // extern "C"

// ---- cluster decoder ------------------------------------------------------------------

struct qldpc_cluster {
    int device = 0;
    qldpc_decoder *bp = nullptr;  // fused graph of H (float32 messages, gamma row of zeros)
    const ClusterKernel *k = nullptr;
    ClusterArgs args{};
    void *arena = nullptr;        // chk_var and the work counters
    unsigned int *counter = nullptr;
    WorkList work;
    size_t smem = 0;
    int grid = 0;
};

extern "C" {

int qldpc_cluster_create(qldpc_cluster **out, int32_t M, int32_t N, const int32_t *row_ptr,
                         const int32_t *col_idx, const double *priors,
                         const qldpc_cluster_params *params, int device) {
    last_error().clear();
    if (!out) return fail(QLDPC_ERR_INVALID_ARG, "out must not be NULL");
    *out = nullptr;
    if (!params) return fail(QLDPC_ERR_INVALID_ARG, "params must not be NULL");
    if (params->bp_iters < 0) return fail(QLDPC_ERR_INVALID_ARG, "bp_iters < 0");
    if (!std::isfinite(params->llr_accept) || !std::isfinite(params->llr_erase) ||
        params->llr_erase < params->llr_accept)
        return fail(QLDPC_ERR_INVALID_ARG, "need finite llr_accept <= llr_erase");
    if (params->max_clusters < 1 || params->max_clusters > kClusterMaxClusters)
        return fail(QLDPC_ERR_INVALID_ARG, "max_clusters %d outside 1..%d", params->max_clusters,
                    kClusterMaxClusters);
    if (params->max_cluster_faults < 1 || params->max_cluster_faults > kClusterMaxColumns)
        return fail(QLDPC_ERR_INVALID_ARG, "max_cluster_faults %d outside 1..%d",
                    params->max_cluster_faults, kClusterMaxColumns);
    int rc = validate_graph(M, N, row_ptr, col_idx, priors);
    if (rc) return rc;
    if (M + N > 32767) return fail(QLDPC_ERR_UNSUPPORTED, "M + N = %d above 32767", M + N);
    qldpc_cluster *o = new (std::nothrow) qldpc_cluster();
    if (!o) return fail(QLDPC_ERR_OOM, "host allocation failed");
    o->device = device;
    rc = create_plain_bp(&o->bp, M, N, row_ptr, col_idx, priors, params->bp_iters, device);
    if (rc) {
        delete o;
        return rc;
    }
    DeviceGuard guard(device);
    const qldpc_decoder *d = o->bp;
    const int DC = d->fk->dc, DV = d->fk->dv;
    auto bail = [&](int code) {
        std::string msg = last_error();
        qldpc_cluster_destroy(o);
        last_error() = msg;
        return code;
    };
    const ClusterKernel *tab = nullptr;
    int ntab = 0;
    cluster_table(&tab, &ntab);
    for (int q = 0; q < ntab && !o->k; ++q)
        if (tab[q].dc == DC && tab[q].dv == DV && (long long)tab[q].threads * tab[q].vpt >= N)
            o->k = &tab[q];
    if (!o->k) {
        fail(QLDPC_ERR_UNSUPPORTED, "no compiled cluster kernel for N = %d", N);
        return bail(QLDPC_ERR_UNSUPPORTED);
    }
    ClusterArgs &a = o->args;
    a.bp_iters = params->bp_iters;
    a.llr_accept = params->llr_accept;
    a.llr_erase = params->llr_erase;
    a.max_clusters = params->max_clusters;
    a.max_cols = params->max_cluster_faults;
    a.W = (a.max_cols + 31) / 32;
    const std::vector<int32_t> chk_var = check_faults(M, d->fg.Mp, DC, row_ptr, col_idx);
    const size_t cv_bytes = align_up(sizeof(int32_t) * chk_var.size(), 256);
    cudaError_t e = cudaMalloc(&o->arena, cv_bytes + 256);
    if (e != cudaSuccess) {
        fail(QLDPC_ERR_OOM, "cudaMalloc failed: %s", cudaGetErrorString(e));
        return bail(QLDPC_ERR_OOM);
    }
    e = cudaMemcpy(o->arena, chk_var.data(), sizeof(int32_t) * chk_var.size(),
                   cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        a.chk_var = static_cast<const int32_t *>(o->arena);
        o->counter = reinterpret_cast<unsigned int *>(static_cast<char *>(o->arena) + cv_bytes);
        o->smem = cluster_smem_bytes(d->fg, a);
        bool fits = false;
        e = configure_kernel(o->k->fn, o->k->threads, o->smem, device, d->num_sms, &o->grid,
                             &fits);
        if (e == cudaSuccess && !fits) {
            fail(QLDPC_ERR_UNSUPPORTED,
                 "the cluster stage (%zu B of shared memory) cannot be resident", o->smem);
            return bail(QLDPC_ERR_UNSUPPORTED);
        }
    }
    if (e != cudaSuccess) {
        fail(QLDPC_ERR_CUDA, "cluster set-up failed: %s", cudaGetErrorString(e));
        return bail(QLDPC_ERR_CUDA);
    }
    *out = o;
    return QLDPC_OK;
}

int qldpc_cluster_decode_batch(qldpc_cluster *o, const uint64_t *syndromes, int64_t B,
                               const uint8_t *skip, uint64_t *corrections, int32_t *status,
                               int32_t *steps, void *stream) {
    last_error().clear();
    if (!o) return fail(QLDPC_ERR_INVALID_ARG, "cluster handle is NULL");
    int rc = check_batch(o->bp, syndromes, B, corrections);
    if (rc) return rc;
    if (B > 0 && !status) return fail(QLDPC_ERR_INVALID_ARG, "status must not be NULL");
    if (B == 0) return QLDPC_OK;
    DeviceGuard guard(o->device);
    QL_CUDA(guard.err);
    const void *ptrs[5] = {syndromes, skip, corrections, status, steps};
    for (int q = 0; q < 5; ++q)
        if (ptrs[q] && !is_device_ptr(ptrs[q]))
            return fail(QLDPC_ERR_INVALID_ARG, "argument %d is not device memory", q);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int32_t *list = nullptr;
    QL_CUDA(prepare_work(o->work, skip, B, status, steps, o->counter, st, &list));
    const int grid = (int)std::min<int64_t>(o->grid, B);
    QL_CUDA(o->k->launch(dim3(grid), o->smem, st, o->bp->fg, o->bp->prm, o->args, syndromes,
                         list, (int)B, ClusterOut{corrections, status, steps}, o->counter));
    return QLDPC_OK;
}

void qldpc_cluster_destroy(qldpc_cluster *o) {
    if (!o) return;
    {
        DeviceGuard guard(o->device);
        if (o->arena) cudaFree(o->arena);  // waits for work that may still use it
        if (o->work.list) cudaFree(o->work.list);
    }
    qldpc_destroy(o->bp);
    delete o;
}

}  // extern "C"
