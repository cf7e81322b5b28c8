/*
 * qldpc.h — C ABI of the GB300 batched Relay-BP decoder (libqldpc.so).
 *
 * Relay decoding (paper Sec. 2.3, "Relay decoding"; parameters App. A.3) of many
 * syndromes of one decoding problem (H, p) (paper Sec. 2.1, "Noise and decoding").
 * For each syndrome sigma the decoder runs legs of disordered-memory min-sum
 * belief propagation (DMem-BP):
 *     lambda_j(t) = (1 - gamma_j) lambda_j(0) + gamma_j Lambda_j(t-1)
 *     mu_{i->j}(t) = (-1)^{sigma_i} prod_{j' in N(i)\j} sign(nu_{j'->i}(t-1)) min |nu_{j'->i}(t-1)|
 *     nu_{j->i}(t) = lambda_j(t) + sum_{i' in N(j)\i} mu_{i'->j}(t)
 *     Lambda_j(t) = lambda_j(t) + sum_{i in N(j)} mu_{i->j}(t),  F_j = [Lambda_j < 0]
 * until H F = sigma (a solution) or T_r iterations; leg r >= 2 is warm-started from
 * the previous leg's terminal marginals; decoding stops after S solutions or after
 * the last leg and returns the lowest-weight solution (W = sum_j F_j w_j).
 *
 * Conventions for every entry point:
 *   - Return value: QLDPC_OK (0) or a negative QLDPC_ERR_* code; qldpc_last_error()
 *     then describes the failure for the calling thread.  Nothing aborts or traps.
 *   - Bit vectors are packed little-endian into uint64 words: bit k of word w is
 *     entry 64*w + k.  Padding bits of syndromes are ignored; padding bits of
 *     corrections are written as zero.
 *   - A decoder handle may be used by one host thread at a time, and its decode
 *     calls must not overlap on the GPU (they share the handle's work counter).
 *   - "device" pointers are CUDA device (or managed) memory of the handle's device;
 *     "host" pointers are ordinary (preferably pinned) host memory.
 */
#ifndef QLDPC_H
#define QLDPC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QLDPC_OK 0
#define QLDPC_ERR_INVALID_ARG (-1)  /* a pointer, size or value is outside its contract   */
#define QLDPC_ERR_CUDA (-2)         /* a CUDA runtime call failed                         */
#define QLDPC_ERR_OOM (-3)          /* a device or host allocation failed                 */
#define QLDPC_ERR_UNSUPPORTED (-4)  /* the graph exceeds what the kernels are built for   */

/* Message storage precision (variable-node sums are always float32). */
#define QLDPC_MSG_FP32 0
#define QLDPC_MSG_FP16 1

/* Kernel selection. */
#define QLDPC_KERNEL_AUTO 0      /* the fused persistent kernel                          */
#define QLDPC_KERNEL_BASELINE 1  /* plain one-shot-per-block float32 kernel (reference)  */
#define QLDPC_KERNEL_FUSED 2     /* fused persistent kernel                              */

/* Relay parameters (paper App. A.3 gives T_1 = 80, T_r = 60, R = 300, S = 1). */
typedef struct {
    int32_t legs_after_first;     /* R >= 0: relay legs after the first leg                 */
    int32_t iters_first;          /* T_1 >= 1: iteration limit of the first leg             */
    int32_t iters_later;          /* T_r >= 1: iteration limit of legs 2..R+1               */
    int64_t max_total_iters;      /* iteration budget per shot over all legs; <= 0: none    */
    int32_t stop_after_solutions; /* S >= 1                                                 */
    int32_t warm_start_mode;      /* 0: lambda(0) <- previous terminal marginals (paper);
                                     1: lambda(0) = nu(0) = w, Lambda(0) carried over       */
    int32_t msg_precision;        /* QLDPC_MSG_FP32 or QLDPC_MSG_FP16                       */
    int32_t kernel;               /* QLDPC_KERNEL_*                                         */
    int32_t block_threads;        /* threads per block; 0 = chosen by the library          */
    float llr_clip;               /* saturation bound C of messages and marginals;
                                     <= 0: 65504 (FP16 storage) or 1e30 (FP32)              */
    const float *gamma_table;     /* host, [(R+1)][N] row-major: row r holds the memory
                                     strengths gamma_j of leg r+1 (row 0 = first leg).
                                     Copied at create time; finite values required.        */
    int32_t tail_cut_iters;       /* tail continuation of the fused kernel: a shot that has
                                     run this many iterations when a leg ends, with a next
                                     leg to run, is handed to a second launch with one
                                     1024-thread block per SM (same results, lower latency
                                     for the few very long shots).  0: T_1 + 8 T_r;
                                     < 0: off                                              */
} qldpc_relay_params;

typedef struct qldpc_decoder qldpc_decoder; /* opaque */

/* Facts about a created decoder (for tests, tuning and reports). */
typedef struct {
    int32_t M, N, E;              /* checks, faults, edges of H                              */
    int32_t max_check_degree, max_fault_degree;
    int32_t kernel;               /* QLDPC_KERNEL_BASELINE or QLDPC_KERNEL_FUSED             */
    int32_t msg_precision;
    int32_t block_threads;
    int32_t blocks_per_sm;        /* resident blocks per SM of the chosen kernel             */
    int32_t num_sms;
    int32_t grid_blocks;          /* persistent grid size (fused kernel)                     */
    int32_t smem_bytes;           /* dynamic shared memory per block                         */
    int32_t syndrome_words;       /* ceil(M/64): uint64 words per syndrome                   */
    int32_t correction_words;     /* ceil(N/64): uint64 words per correction                 */
    int32_t tail_cut_iters;       /* iterations before a shot may move to the second launch
                                     (-1: no tail continuation)                             */
    int32_t tail_block_threads;   /* block size of the second launch                        */
    int32_t tail_records;         /* shots the second launch can take per call; later long
                                     shots finish in the first launch                       */
} qldpc_info;

/*
 * Create a decoder for H (M x N, given as CSR: row_ptr[M+1], col_idx[E], columns
 * strictly increasing within a row, 0 <= col < N) with fault probabilities
 * priors[N] in (0, 1) (paper Sec. 2.1) and Relay parameters *prm.  All inputs are
 * host memory and are copied; the caller may free them on return.  device: CUDA
 * device ordinal.  *out receives the handle (NULL on failure).
 * Errors: INVALID_ARG (malformed CSR, prior outside (0,1), bad parameter),
 * UNSUPPORTED (a check degree above 32, a fault degree above 8, or a graph whose
 * state does not fit in shared memory), OOM, CUDA.
 */
int qldpc_create(qldpc_decoder **out, int32_t M, int32_t N, const int32_t *row_ptr,
                 const int32_t *col_idx, const double *priors, const qldpc_relay_params *prm,
                 int device);

/*
 * Decode B syndromes.  syndromes: device, [B][ceil(M/64)] uint64.  Outputs, all
 * device: corrections [B][ceil(N/64)] uint64 (the kept solution, or the last
 * iteration's decision when no solution was found); legs_used [B] int32 (legs run);
 * converged [B] uint8 (1 iff at least one valid correction was found); iters [B]
 * int32 (DMem-BP iterations run over all legs).  legs_used, converged and iters may
 * be NULL.  stream: a cudaStream_t (NULL = legacy default stream).  The call is
 * asynchronous on stream: it returns after the launch is queued.  B = 0 is a no-op.
 * Errors: INVALID_ARG (NULL handle, NULL syndromes/corrections with B > 0, B < 0 or
 * above 2^31-1, a pointer that is not device memory), CUDA (launch failure).
 */
int qldpc_decode_batch(qldpc_decoder *d, const uint64_t *syndromes, int64_t B,
                       uint64_t *corrections, int32_t *legs_used, uint8_t *converged,
                       int32_t *iters, void *stream);

/*
 * Same as qldpc_decode_batch with HOST buffers: copies the syndromes to device
 * buffers owned by the handle (grown on demand), decodes on the handle's internal
 * stream, copies the results back and waits for completion.  Pinned host memory
 * gives full copy bandwidth.  legs_used, converged, iters may be NULL.
 * Errors: as qldpc_decode_batch, plus OOM when the staging buffers cannot grow.
 */
int qldpc_decode_batch_host(qldpc_decoder *d, const uint64_t *syndromes, int64_t B,
                            uint64_t *corrections, int32_t *legs_used, uint8_t *converged,
                            int32_t *iters);

/*
 * Decode a mixed batch of shots of several codes in one persistent launch.
 * decoders[0..n_codes-1] (1 <= n_codes <= 8): fused-kernel decoders created on one
 * device with the same message precision and degree family (max check degree <= 8
 * and max fault degree <= 4 for all, or the same wider family).  Each keeps its own
 * graph, priors, gamma table and Relay parameters.  Device arrays:
 * code_of_shot [B] int32 (index into decoders), syndromes [B][syndrome_stride] and
 * corrections [B][correction_stride] uint64 rows (strides >= the widest code's
 * ceil(M/64) and ceil(N/64); each shot uses the first words of its row), legs_used,
 * converged, iters [B] as in qldpc_decode_batch (may be NULL).  A shot whose code id
 * is out of range is skipped and gets iters = -1, legs = 0, converged = 0.  Uses the
 * work counter of decoders[0]: do not overlap with other calls on that handle.
 * Asynchronous on stream.  Errors: INVALID_ARG, UNSUPPORTED (mixed families or
 * precisions, baseline decoders), CUDA.
 */
int qldpc_decode_batch_multi(qldpc_decoder *const *decoders, int32_t n_codes,
                             const int32_t *code_of_shot, const uint64_t *syndromes,
                             int32_t syndrome_stride, int64_t B, uint64_t *corrections,
                             int32_t correction_stride, int32_t *legs_used, uint8_t *converged,
                             int32_t *iters, void *stream);

/*
 * The same mixed batch decoded per code: the shots are sorted into one index list per
 * code on the device, then each code's shots run in one persistent launch of that
 * decoder's own kernel shape (largest code first), all on `stream` (capturable in a
 * CUDA graph).  Results equal qldpc_decode_batch_multi's.  Decoders may differ in
 * message precision and degree family but must be distinct and on one device; each
 * decoder's work counter is used.  workspace: device memory of at least
 * qldpc_grouped_workspace_bytes(n_codes, B) bytes, caller-owned, not touched by other
 * work meanwhile.  Errors: INVALID_ARG, UNSUPPORTED (baseline decoders, two devices),
 * CUDA.
 */
uint64_t qldpc_grouped_workspace_bytes(int32_t n_codes, int64_t B);
int qldpc_decode_batch_grouped(qldpc_decoder *const *decoders, int32_t n_codes,
                               const int32_t *code_of_shot, const uint64_t *syndromes,
                               int32_t syndrome_stride, int64_t B, uint64_t *corrections,
                               int32_t correction_stride, int32_t *legs_used,
                               uint8_t *converged, int32_t *iters, void *workspace,
                               uint64_t workspace_bytes, void *stream);

/*
 * Size of the static scratch area used by qldpc_decode_batch_host_static: 8 MiB of
 * device memory that every GPU loading this library holds until the process exits.
 */
#define QLDPC_STATIC_SCRATCH_BYTES (8 * 1024 * 1024)

/*
 * qldpc_decode_batch_host with no allocation at all.  (The paper has no
 * counterpart: this serves callers that cannot allocate device memory while they
 * decode, such as a real-time loop with a fixed memory budget or a process whose
 * device memory is owned by another allocator; qldpc_decode_batch_host allocates
 * its staging buffers on first use and whenever the batch grows.)
 * The syndromes, outputs and the kernel's work counter are staged in one static
 * device array of QLDPC_STATIC_SCRATCH_BYTES; a batch must fit in it (for the gross
 * code, 936 x 2736, 17,732 shots per call), else INVALID_ARG names the exact limit.
 * Host pointers as in qldpc_decode_batch_host; synchronous on the handle's internal
 * stream.  qldpc_create looks up the array's device address in the context current
 * at creation (the first create on a device makes the driver load the array there)
 * and keeps it in the handle, so calls themselves load and allocate nothing; like
 * every handle, one created before a cudaDeviceReset must not be used after it.
 * Every call on a device shares the one array, which keeps the previous call's
 * contents (the work counter is cleared by each call): calls that overlap on the GPU,
 * from any handle, race.  Fused kernel only (UNSUPPORTED for the baseline kernel).
 */
int qldpc_decode_batch_host_static(qldpc_decoder *d, const uint64_t *syndromes, int64_t B,
                                   uint64_t *corrections, int32_t *legs_used,
                                   uint8_t *converged, int32_t *iters);

/*
 * Run T iterations of the first leg (memory strengths = row 0 of the gamma table)
 * on B syndromes with no early exit, recording every iteration, for checking
 * message precision.  Outputs (device, float32, may be NULL):
 * marginals [T][B][N] = Lambda(t); nu [T][B][E] and mu [T][B][E] = the two message
 * directions after iteration t, in CSR edge order (edge e = position in col_idx).
 * Uses the decoder's message precision and kernel family (fused kernel only).
 * Asynchronous on stream.  Errors: INVALID_ARG, UNSUPPORTED (baseline kernel), CUDA.
 */
int qldpc_trace_first_leg(qldpc_decoder *d, const uint64_t *syndromes, int64_t B, int32_t T,
                          float *marginals, float *nu, float *mu, void *stream);

/* ---- Soft DMem-BP: differentiable unrolled leg for tuning memory strengths ---------
 *
 * One leg of Relay's DMem-BP (paper Sec. 2.3, "Relay decoding": memory rule
 * lambda_j(t) = (1-gamma_j) w_j + gamma_j Lambda_j(t-1), fault->check and marginal
 * sums as in Relay) with the min-sum check rule replaced by sum-product and scaled per
 * iteration (the paper trains nothing; these are this library's choices):
 *     mu_e(t) = alpha_t (-1)^sigma_i 2 atanh(prod_{e' != e} tanh(nu_e'(t-1)/2)),
 * with the product clamped to |.| <= 1 - eps (eps = 2^-23 in FP32, 1e-15 in FP64),
 * run for `iterations` iterations from nu(0) = Lambda(0) = w with no early exit.
 * Loss: mean over shots b and faults j of
 *     F_bj softplus(Lambda_bj(T)) + (1 - F_bj) softplus(-Lambda_bj(T)),
 * i.e. binary cross-entropy of sigmoid(-Lambda) against the true faults F.
 * The backward pass is a hand-written adjoint that recomputes each segment of
 * checkpoint_every iterations from the checkpoints stored by the forward pass.
 */
#define QLDPC_REAL_FP32 0
#define QLDPC_REAL_FP64 1

typedef struct qldpc_soft qldpc_soft; /* opaque */

/* Create for H (CSR, host, copied) and priors (host, in (0,1)); fault degree <= 8,
 * check degree <= 32.  real_type: QLDPC_REAL_FP32 or QLDPC_REAL_FP64 (the type of
 * every real array passed to forward/backward).  Errors: INVALID_ARG, UNSUPPORTED
 * (degrees, or state above the shared-memory limit), OOM, CUDA. */
int qldpc_soft_create(qldpc_soft **out, int32_t M, int32_t N, const int32_t *row_ptr,
                      const int32_t *col_idx, const double *priors, int32_t iterations,
                      int32_t checkpoint_every, int32_t real_type, int device);

/* Bytes of device workspace a batch of B shots needs (checkpoints, segment buffer,
 * per-shot partial results, the adjoint's per-shot scratch).  The caller allocates it,
 * 16-byte aligned (forward and backward refuse another alignment with INVALID_ARG). */
int qldpc_soft_workspace_bytes(const qldpc_soft *s, int64_t B, uint64_t *bytes);

/* Forward.  Device pointers: syndromes [B][ceil(M/64)] uint64, faults [B][ceil(N/64)]
 * uint64 (the true F for the loss), gamma [N], alpha [iterations], loss [1], marginals
 * [B][N] (Lambda(T), may be NULL), workspace (>= qldpc_soft_workspace_bytes).  Stores
 * the checkpoints for qldpc_soft_backward in the workspace.  Asynchronous on stream.
 * Errors: INVALID_ARG, CUDA. */
int qldpc_soft_forward(qldpc_soft *s, const uint64_t *syndromes, const uint64_t *faults,
                       int64_t B, const void *gamma, const void *alpha, void *loss,
                       void *marginals, void *workspace, uint64_t workspace_bytes,
                       void *stream);

/* Backward: grad_gamma [N] = loss_grad * dloss/dgamma, grad_alpha [iterations] =
 * loss_grad * dloss/dalpha (device; loss_grad is a device scalar, NULL means 1).
 * Must follow qldpc_soft_forward with the same inputs and workspace.  Gradients are
 * summed over shots in a fixed order (deterministic).  Errors: INVALID_ARG, CUDA. */
int qldpc_soft_backward(qldpc_soft *s, const uint64_t *syndromes, const uint64_t *faults,
                        int64_t B, const void *gamma, const void *alpha, const void *loss_grad,
                        void *grad_gamma, void *grad_alpha, void *workspace,
                        uint64_t workspace_bytes, void *stream);

/* Free the soft handle (syncs through cudaFree).  NULL is ignored. */
void qldpc_soft_destroy(qldpc_soft *s);

/* ---- Filtered-OSD post-processor (paper Sec. 5, pre-decoder set-up of Sec. 7.1) ----
 *
 * For each shot not marked in `skip` (typically the shots whose first Relay leg did
 * not converge; the paper's pre-decoder is that leg, T_1 = 80 with gamma_0):
 *   1. bp_iters iterations of plain min-sum BP (Sec. 2.3, "Belief propagation
 *      decoding") from the priors, no early exit, give the marginals Lambda;
 *   2. R = the faults with Lambda_j < llr_confident (a float32 compare), sorted by
 *      increasing Lambda_j, ties by increasing j; |R| > max_candidates fails;
 *   3. x solves H_R x = sigma with x supported on the leftmost linearly independent
 *      columns of H_R (free columns 0), found by the streaming ("lifted") Gauss-Jordan
 *      elimination of Sec. 4; no solution fails;
 *   4. F_j = x_r for j = R_r.
 * The paper fixes bp_iters = 25 and |R|_max = 500 (Sec. 7.1, App. A.1);
 * it gives no value for Lambda_confident. */
typedef struct qldpc_osd qldpc_osd;

typedef struct {
    int32_t bp_iters;        /* >= 0 plain BP iterations before the ranking (paper 25)        */
    float llr_confident;     /* finite; keep faults with Lambda_j < llr_confident              */
    int32_t max_candidates;  /* |R|_max, 1..1024 (paper 500)                                   */
} qldpc_osd_params;

#define QLDPC_OSD_SKIPPED 0        /* skip[b] != 0: nothing written                           */
#define QLDPC_OSD_SOLVED 1         /* corrections[b] holds the OSD correction                 */
#define QLDPC_OSD_TOO_MANY (-1)    /* |R| > max_candidates; corrections[b] untouched          */
#define QLDPC_OSD_NO_SOLUTION (-2) /* H_R x = sigma has no solution; corrections[b] untouched */

/* Copy H (CSR as in qldpc_create, M <= 32767, N <= 32767, check degree <= 32, fault
 * degree <= 8) and the priors to `device`.  Errors: INVALID_ARG, UNSUPPORTED, CUDA, OOM. */
int qldpc_osd_create(qldpc_osd **out, int32_t M, int32_t N, const int32_t *row_ptr,
                     const int32_t *col_idx, const double *priors,
                     const qldpc_osd_params *params, int device);

/* Post-process B shots (device pointers): syndromes [B][ceil(M/64)] u64; skip [B] u8
 * or NULL (post-process every shot); corrections [B][ceil(N/64)] u64, written only for
 * solved shots (pass the pre-decoder's corrections to keep them elsewhere); status [B]
 * int32 (QLDPC_OSD_*); n_candidates [B] int32 |R| or NULL.  Asynchronous on `stream`
 * (cudaStream_t, NULL = legacy default stream), except that with a skip mask the handle
 * lists the shots to post-process in a device array of B entries, allocated on the first
 * such call and whenever B grows (the call then waits for the device).  One call at a
 * time per handle.  Errors: INVALID_ARG, CUDA. */
int qldpc_osd_decode_batch(qldpc_osd *o, const uint64_t *syndromes, int64_t B,
                           const uint8_t *skip, uint64_t *corrections, int32_t *status,
                           int32_t *n_candidates, void *stream);

/* Wait for the handle's work, then free it.  NULL is ignored. */
void qldpc_osd_destroy(qldpc_osd *o);

/* ---- Cluster decoder (paper Sec. 2.5 "Cluster decoding" / "BP-UF decoding", Sec. 6,
 * pre-decoder set-up of Sec. 7.1) ----
 *
 * For each shot not marked in `skip` (typically those the first Relay leg leaves
 * unconverged):
 *   1. bp_iters iterations of plain min-sum BP from the priors give Lambda;
 *   2. faults with Lambda_j <= llr_accept form a partial correction F_pre, faults with
 *      llr_accept < Lambda_j <= llr_erase the erasure set; sigma <- sigma + H F_pre;
 *   3. one cluster per syndrome check and per erased fault, taken in decreasing node
 *      index (checks before faults); clusters are vertex sets of the Tanner graph;
 *   4. while a cluster is invalid (its syndrome is not in the image of H restricted to
 *      its checks and interior faults), the first invalid one is grown by all neighbours
 *      of its vertices, merged with every cluster it meets, re-tested, and queued last
 *      if still invalid;
 *   5. the correction is F_pre + each cluster's solution on its interior faults (free
 *      columns 0, columns in increasing fault index).
 * The paper gives N_clus = 50 / 100 and solver sizes up to 144 x 288 / 576 x 1152
 * (App. A.2) and no values for the cutoffs. */
typedef struct qldpc_cluster qldpc_cluster;

typedef struct {
    int32_t bp_iters;           /* >= 0 plain BP iterations (paper 25)                       */
    float llr_accept;           /* Lambda_j <= llr_accept: partial correction (finite)      */
    float llr_erase;            /* llr_accept < Lambda_j <= llr_erase: erasure (finite)     */
    int32_t max_clusters;       /* 1..4096 initial clusters; more fails                     */
    int32_t max_cluster_faults; /* 1..512 interior faults of one cluster; more fails        */
} qldpc_cluster_params;

#define QLDPC_CLUSTER_SKIPPED 0       /* skip[b] != 0: nothing written                       */
#define QLDPC_CLUSTER_DECODED 1       /* every cluster valid; corrections[b] written         */
#define QLDPC_CLUSTER_TOO_LARGE (-1)  /* a cluster exceeded max_cluster_faults               */
#define QLDPC_CLUSTER_TOO_MANY (-2)   /* more than max_clusters initial clusters             */
#define QLDPC_CLUSTER_STALLED (-3)    /* the update loop exceeded M + N steps (not expected)  */

/* Copy H (CSR as in qldpc_create, M + N <= 32767, check degree <= 32, fault degree <= 8)
 * and the priors to `device`.  Errors: INVALID_ARG, UNSUPPORTED, CUDA, OOM. */
int qldpc_cluster_create(qldpc_cluster **out, int32_t M, int32_t N, const int32_t *row_ptr,
                         const int32_t *col_idx, const double *priors,
                         const qldpc_cluster_params *params, int device);

/* Decode B shots (device pointers): syndromes [B][ceil(M/64)] u64; skip [B] u8 or NULL;
 * corrections [B][ceil(N/64)] u64, written only for decoded shots; status [B] int32
 * (QLDPC_CLUSTER_*); steps [B] int32 growth steps or NULL.  Asynchronous on `stream`,
 * with the same list of shots as qldpc_osd_decode_batch when skip is given (allocated on
 * the first such call and whenever B grows).  One call at a time per handle.
 * Errors: INVALID_ARG, CUDA. */
int qldpc_cluster_decode_batch(qldpc_cluster *c, const uint64_t *syndromes, int64_t B,
                               const uint8_t *skip, uint64_t *corrections, int32_t *status,
                               int32_t *steps, void *stream);

/* Wait for the handle's work, then free it.  NULL is ignored. */
void qldpc_cluster_destroy(qldpc_cluster *c);

/* Fill *info.  Errors: INVALID_ARG. */
int qldpc_get_info(const qldpc_decoder *d, qldpc_info *info);

/* Wait for the handle's work, then free everything it owns.  NULL is ignored. */
void qldpc_destroy(qldpc_decoder *d);

/* Static description of a status code. */
const char *qldpc_status_string(int status);

/* Thread-local description of the last failure on this thread ("" if none). */
const char *qldpc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* QLDPC_H */
