// Host-side pieces shared by the C-ABI translation units: qldpc_api.cu (the Relay
// decoder), soft_api.cu (the soft DMem-BP leg) and post_api.cu (filtered-OSD and the
// cluster decoder).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "qldpc.h"
#include "qldpc_internal.h"

namespace qldpc {

// The calling thread's last error message (qldpc_last_error), and a failure return that
// sets it (printf-style message) and returns `code`.
std::string &last_error();
int fail(int code, const char *fmt, ...);

// Makes `dev` current for the scope and restores the caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) err = cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Checks of a CSR graph with its priors (the rules of qldpc_create); sets the error.
int validate_graph(int32_t M, int32_t N, const int32_t *row_ptr, const int32_t *col_idx,
                   const double *priors);

// Whether p is device (or managed) memory.
bool is_device_ptr(const void *p);

}  // namespace qldpc

// A failed CUDA call returns QLDPC_ERR_OOM or QLDPC_ERR_CUDA with the call in the message.
#define QL_CUDA(call)                                                                    \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            int code_ = e_ == cudaErrorMemoryAllocation ? QLDPC_ERR_OOM : QLDPC_ERR_CUDA; \
            return ::qldpc::fail(code_, "%s failed: %s", #call, cudaGetErrorString(e_)); \
        }                                                                                \
    } while (0)

// The decoder handle of the C ABI (an opaque type in qldpc.h).
struct qldpc_decoder {
    int device = 0;
    int M = 0, N = 0, E = 0, dc_max = 0, dv_max = 0;
    qldpc::DevParams prm{};
    int kernel = QLDPC_KERNEL_FUSED;
    int msg_fp16 = 0;
    const qldpc::FusedKernel *fk = nullptr;        // decode kernel
    const qldpc::FusedKernel *fk_trace = nullptr;  // trace kernel
    size_t trace_smem = 0;
    int block_threads = 0, blocks_per_sm = 0, num_sms = 0, grid = 0;
    size_t smem = 0;
    qldpc::FusedGraph fg{};
    qldpc::BaseGraph bg{};
    void *arena = nullptr;
    unsigned int *counter = nullptr;  // [0] work counter, [1] tail records, [2] records taken
    // tail continuation (fused kernel): the resuming launch's kernel and grid, the records
    const qldpc::FusedKernel *fk_tail = nullptr;
    int tail_grid = 0;
    qldpc::TailCont tail{};  // mode 0 when off
    void *tail_arena = nullptr;
    cudaStream_t stream = nullptr;  // internal stream of the host-buffer entry point
    void *stage = nullptr;
    int64_t stage_B = 0;
    unsigned char *static_scratch = nullptr;  // device address of the static staging array
};

namespace qldpc {

// The batch arguments every decode entry point checks; sets the error.
int check_batch(const qldpc_decoder *d, const void *syn, int64_t B, const void *corr);

}  // namespace qldpc
