// Host side of the soft DMem-BP leg's C ABI (include/qldpc.h: qldpc_soft_*): graph layout
// for the soft kernels (float32 rows of up to 8 edges padded to 8 slots), workspace
// layout, argument checks and launches.
#include <algorithm>
#include <cmath>
#include <vector>

#include "api_common.h"
#include "soft_internal.h"

using namespace qldpc;

// ---- soft DMem-BP (sum-product leg with trainable gamma_j, alpha_t) -------------------

struct qldpc_soft {
    int device = 0;
    int M = 0, N = 0, E = 0, dc_max = 0, dv_max = 0;
    int T = 0, K = 0, fp64 = 0;
    double eps = 0;
    SoftGraph g{};
    void *arena = nullptr;
    void *w = nullptr;  // prior LLRs in the working precision
};

namespace {

// Workspace arrays: checkpoints [B][nck][S], segment buffer [B][K][S] (S values per
// state), per-shot loss [B], gamma gradient [B][N], alpha gradient [B][T], and the
// adjoint state (of nu, then of Lambda) between segments [B][S].
size_t soft_workspace_layout(const qldpc_soft *s, int64_t B, size_t off[6]) {
    const size_t rs = s->fp64 ? 8 : 4, S = (size_t)soft_state_values(s->g);
    const int nck = (s->T + s->K - 1) / s->K;
    const size_t sz[6] = {(size_t)B * nck * S * rs, (size_t)B * s->K * S * rs, (size_t)B * rs,
                          (size_t)B * s->N * rs,     (size_t)B * s->T * rs,     (size_t)B * S * rs};
    size_t o = 0;
    for (int q = 0; q < 6; ++q) {
        off[q] = o;
        o = align_up(o + sz[q], 256);
    }
    return o;
}

int soft_check_call(const qldpc_soft *s, const uint64_t *syn, const uint64_t *faults, int64_t B,
                    const void *gamma, const void *alpha, void *ws, uint64_t ws_bytes,
                    size_t off[6]) {
    if (!s) return fail(QLDPC_ERR_INVALID_ARG, "soft handle is NULL");
    if (B < 1 || B > 0x7fffffffLL) return fail(QLDPC_ERR_INVALID_ARG, "batch size out of range");
    if (!syn || !faults || !gamma || !alpha || !ws)
        return fail(QLDPC_ERR_INVALID_ARG, "syndromes, faults, gamma, alpha and workspace are required");
    if (reinterpret_cast<uintptr_t>(ws) % 16 != 0)
        return fail(QLDPC_ERR_INVALID_ARG, "workspace must be 16-byte aligned");
    const size_t need = soft_workspace_layout(s, B, off);
    if (ws_bytes < need)
        return fail(QLDPC_ERR_INVALID_ARG, "workspace of %llu bytes, %zu needed",
                    (unsigned long long)ws_bytes, need);
    const void *ptrs[5] = {syn, faults, gamma, alpha, ws};
    for (int q = 0; q < 5; ++q)
        if (!is_device_ptr(ptrs[q]))
            return fail(QLDPC_ERR_INVALID_ARG, "argument %d is not device memory", q);
    return QLDPC_OK;
}

SoftLaunch soft_launch(const qldpc_soft *s, const uint64_t *syn, const uint64_t *faults,
                       int64_t B, const void *gamma, const void *alpha, void *ws,
                       const size_t off[6]) {
    SoftLaunch L{};
    char *base = static_cast<char *>(ws);
    L.g = s->g;
    L.fp64 = s->fp64;
    L.dc_max = s->dc_max;
    L.T_it = s->T;
    L.K = s->K;
    L.B = (int)B;
    L.eps = s->eps;
    L.syn = syn;
    L.faults = faults;
    L.gamma = gamma;
    L.alpha = alpha;
    L.w = s->w;
    L.ckpt = base + off[0];
    L.seg = base + off[1];
    L.shot_loss = base + off[2];
    L.shot_gg = base + off[3];
    L.shot_ga = base + off[4];
    L.shot_adj = base + off[5];
    return L;
}

}  // namespace

extern "C" {

int qldpc_soft_create(qldpc_soft **out, int32_t M, int32_t N, const int32_t *row_ptr,
                      const int32_t *col_idx, const double *priors, int32_t iterations,
                      int32_t checkpoint_every, int32_t real_type, int device) {
    last_error().clear();
    if (!out) return fail(QLDPC_ERR_INVALID_ARG, "out must not be NULL");
    *out = nullptr;
    int rc = validate_graph(M, N, row_ptr, col_idx, priors);
    if (rc) return rc;
    if (iterations < 1) return fail(QLDPC_ERR_INVALID_ARG, "iterations must be >= 1");
    if (checkpoint_every < 1 || checkpoint_every > iterations)
        return fail(QLDPC_ERR_INVALID_ARG, "checkpoint_every must be in [1, iterations]");
    if (real_type != QLDPC_REAL_FP32 && real_type != QLDPC_REAL_FP64)
        return fail(QLDPC_ERR_INVALID_ARG, "unknown real_type %d", real_type);
    int ndev = 0;
    QL_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(QLDPC_ERR_INVALID_ARG, "device %d of %d", device, ndev);
    DeviceGuard guard(device);
    QL_CUDA(guard.err);
    qldpc_soft *s = new (std::nothrow) qldpc_soft();
    if (!s) return fail(QLDPC_ERR_OOM, "host allocation failed");
    s->device = device;
    s->M = M;
    s->N = N;
    s->E = row_ptr[M];
    s->T = iterations;
    s->K = checkpoint_every;
    s->fp64 = real_type == QLDPC_REAL_FP64;
    s->eps = s->fp64 ? 1e-15 : 1.1920928955078125e-07;  // |product| <= 1 - eps
    for (int i = 0; i < M; ++i) s->dc_max = std::max(s->dc_max, row_ptr[i + 1] - row_ptr[i]);
    // float32 rows of at most 8 edges are padded to 8 slots (row i: slots 8 i .. 8 i + 7),
    // which the kernels read and write as 16-byte halves
    const bool pad = !s->fp64 && s->dc_max <= 8;
    const int slots = pad ? 8 * M : s->E;
    std::vector<int32_t> rp(M + 1), deg(std::max(M, 1)), ci(std::max(slots, 1));
    for (int i = 0; i < M; ++i) {
        const int d = row_ptr[i + 1] - row_ptr[i];
        rp[i] = pad ? 8 * i : row_ptr[i];
        deg[i] = d;
        for (int k = 0; k < (pad ? 8 : d); ++k)  // padding slots: the row's first fault (0 if none)
            ci[rp[i] + k] = d > 0 ? col_idx[row_ptr[i] + (k < d ? k : 0)] : 0;
    }
    rp[M] = slots;
    std::vector<int32_t> var_ptr(N + 1, 0), var_edges(std::max(slots, 1)), fill(N, 0);
    for (int e = 0; e < s->E; ++e) var_ptr[col_idx[e] + 1]++;
    for (int j = 0; j < N; ++j) {
        s->dv_max = std::max(s->dv_max, var_ptr[j + 1]);
        var_ptr[j + 1] += var_ptr[j];
    }
    for (int i = 0; i < M; ++i)
        for (int k = 0; k < deg[i]; ++k) {
            const int j = col_idx[row_ptr[i] + k];
            var_edges[var_ptr[j] + fill[j]++] = rp[i] + k;
        }
    auto cleanup = [&](int code) {
        std::string msg = last_error();
        qldpc_soft_destroy(s);
        last_error() = msg;
        return code;
    };
    if (s->dc_max > 32 || s->dv_max > 8)
        return cleanup(fail(QLDPC_ERR_UNSUPPORTED, "check degree %d / fault degree %d above 32 / 8",
                            s->dc_max, s->dv_max));
    SoftGraph &g = s->g;
    g.M = M;
    g.N = N;
    g.E = slots;
    g.syn_words = (M + 63) / 64;
    g.cor_words = (N + 63) / 64;
    int optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e != cudaSuccess) return cleanup(fail(QLDPC_ERR_CUDA, "%s", cudaGetErrorString(e)));
    if (soft_smem_backward(g, s->T, s->fp64) > (size_t)optin)
        return cleanup(fail(QLDPC_ERR_UNSUPPORTED, "soft state needs %zu B of shared memory, above %d",
                            soft_smem_backward(g, s->T, s->fp64), optin));
    // one 8-byte record per fault (its first three slots and its degree) replaces the two
    // dependent reads of var_ptr and var_edges in the kernels' fault loops
    const bool rec = pad && slots < 65536;
    std::vector<uint32_t> frec(2 * (size_t)std::max(N, 1), 0u);
    if (rec)
        for (int j = 0; j < N; ++j) {
            const int b = var_ptr[j], d = var_ptr[j + 1] - b;
            uint32_t sl[3];
            for (int k = 0; k < 3; ++k) sl[k] = (uint32_t)(d > 0 ? var_edges[b + (k < d ? k : 0)] : 0);
            frec[2 * j] = sl[0] | (sl[1] << 16);
            frec[2 * j + 1] = sl[2] | ((uint32_t)d << 16);
        }
    const size_t rs = s->fp64 ? 8 : 4;
    const size_t sizes[7] = {sizeof(int32_t) * (M + 1), sizeof(int32_t) * std::max(slots, 1),
                             sizeof(int32_t) * (N + 1), sizeof(int32_t) * std::max(slots, 1),
                             rs * N, sizeof(int32_t) * std::max(M, 1),
                             sizeof(uint32_t) * frec.size()};
    size_t off[7], o = 0;
    for (int q = 0; q < 7; ++q) {
        off[q] = o;
        o = align_up(o + sizes[q], 256);
    }
    e = cudaMalloc(&s->arena, o);
    if (e != cudaSuccess) return cleanup(fail(QLDPC_ERR_OOM, "cudaMalloc: %s", cudaGetErrorString(e)));
    std::vector<double> w64(N);
    std::vector<float> w32(N);
    for (int j = 0; j < N; ++j) {
        w64[j] = std::log((1.0 - priors[j]) / priors[j]);
        w32[j] = (float)w64[j];
    }
    char *base = static_cast<char *>(s->arena);
    const void *src[7] = {rp.data(), ci.data(), var_ptr.data(), var_edges.data(),
                          s->fp64 ? (const void *)w64.data() : (const void *)w32.data(),
                          deg.data(), frec.data()};
    for (int q = 0; q < 7; ++q) {
        e = cudaMemcpy(base + off[q], src[q], sizes[q], cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cleanup(fail(QLDPC_ERR_CUDA, "cudaMemcpy: %s", cudaGetErrorString(e)));
    }
    g.row_ptr = reinterpret_cast<const int32_t *>(base + off[0]);
    g.col_idx = reinterpret_cast<const int32_t *>(base + off[1]);
    g.var_ptr = reinterpret_cast<const int32_t *>(base + off[2]);
    g.var_edges = reinterpret_cast<const int32_t *>(base + off[3]);
    g.row_deg = pad ? reinterpret_cast<const int32_t *>(base + off[5]) : nullptr;
    g.fault_rec = rec ? reinterpret_cast<const uint2 *>(base + off[6]) : nullptr;
    s->w = base + off[4];
    *out = s;
    return QLDPC_OK;
}

int qldpc_soft_workspace_bytes(const qldpc_soft *s, int64_t B, uint64_t *bytes) {
    if (!s || !bytes || B < 0) return fail(QLDPC_ERR_INVALID_ARG, "bad argument");
    size_t off[6];
    *bytes = soft_workspace_layout(s, B, off);
    return QLDPC_OK;
}

int qldpc_soft_forward(qldpc_soft *s, const uint64_t *syndromes, const uint64_t *faults, int64_t B,
                       const void *gamma, const void *alpha, void *loss, void *marginals,
                       void *workspace, uint64_t workspace_bytes, void *stream) {
    last_error().clear();
    size_t off[6];
    int rc = soft_check_call(s, syndromes, faults, B, gamma, alpha, workspace, workspace_bytes, off);
    if (rc) return rc;
    if (!loss || !is_device_ptr(loss)) return fail(QLDPC_ERR_INVALID_ARG, "loss must be device memory");
    if (marginals && !is_device_ptr(marginals))
        return fail(QLDPC_ERR_INVALID_ARG, "marginals must be device memory");
    DeviceGuard guard(s->device);
    QL_CUDA(guard.err);
    SoftLaunch L = soft_launch(s, syndromes, faults, B, gamma, alpha, workspace, off);
    L.loss = loss;
    L.marg = marginals;
    QL_CUDA(soft_run_forward(L, static_cast<cudaStream_t>(stream)));
    return QLDPC_OK;
}

int qldpc_soft_backward(qldpc_soft *s, const uint64_t *syndromes, const uint64_t *faults,
                        int64_t B, const void *gamma, const void *alpha, const void *loss_grad,
                        void *grad_gamma, void *grad_alpha, void *workspace,
                        uint64_t workspace_bytes, void *stream) {
    last_error().clear();
    size_t off[6];
    int rc = soft_check_call(s, syndromes, faults, B, gamma, alpha, workspace, workspace_bytes, off);
    if (rc) return rc;
    if (!grad_gamma || !grad_alpha || !is_device_ptr(grad_gamma) || !is_device_ptr(grad_alpha))
        return fail(QLDPC_ERR_INVALID_ARG, "grad_gamma and grad_alpha must be device memory");
    if (loss_grad && !is_device_ptr(loss_grad))
        return fail(QLDPC_ERR_INVALID_ARG, "loss_grad must be device memory");
    DeviceGuard guard(s->device);
    QL_CUDA(guard.err);
    SoftLaunch L = soft_launch(s, syndromes, faults, B, gamma, alpha, workspace, off);
    L.upstream = loss_grad;
    L.grad_gamma = grad_gamma;
    L.grad_alpha = grad_alpha;
    QL_CUDA(soft_run_backward(L, static_cast<cudaStream_t>(stream)));
    return QLDPC_OK;
}

void qldpc_soft_destroy(qldpc_soft *s) {
    if (!s) return;
    DeviceGuard guard(s->device);
    if (s->arena) cudaFree(s->arena);
    delete s;
}

}  // extern "C"

