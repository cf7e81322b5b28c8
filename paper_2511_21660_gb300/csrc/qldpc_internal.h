// Internal declarations shared by the host API and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qldpc {

// Relay parameters as the kernels see them (paper App. A.3 naming).
struct DevParams {
    int R;                 // relay legs after the first
    int T1, T2;            // iteration limits of the first and later legs
    int S;                 // stop after S solutions
    int warm_mode;         // 0: lambda(0) <- terminal marginals; 1: lambda(0) = w
    long long max_iters;   // budget over all legs (<= 0: none)
    float clip;            // saturation bound C
};

// Tanner graph in the layouts of the fused kernel.
//   The edges of check i sit on its logical slots k = 0..deg-1 (slots deg..DC-1 are
//   padding); which edge takes which slot is chosen at create time to spread the fault
//   pass's accesses over the shared-memory banks.  Logical slot k of check i is the
//   physical position p = k ^ swz(i) of the check's DC-slot row:
//     float32:  element i*DC + p                      (byte offset 4 * element)
//     binary16: checks 2q, 2q+1 share the 32-bit words q*DC + p, low half for even
//               i (byte offset 4 * word + 2 * (i & 1)), swizzled by swz(q)
//   with swz(x) = (x >> log2(32/DC)) & (DC-1).  Mp = M rounded up to 32.
struct FusedGraph {
    int M, N, E, Mp;
    int msg_bytes;        // bytes of the message array (Mp * DC * message size)
    int syn_words;        // ceil(M/64) uint64 words per syndrome
    int cor_words;        // ceil(N/64) uint64 words per correction
    int f_words;          // uint32 words of the decision bitmap (2*cor_words + 2, rounded
                          // up to a multiple of 4)
    int m_words;          // ceil(M/32) uint32 words of a parity bitmap
    const uint8_t *chk_deg;   // [Mp] check degrees (0 for rows M..Mp-1)
    const int32_t *var_chk;   // [N][DV] checks of fault j, increasing order
    const int32_t *var_slot;  // [N][DV] byte offsets of the messages of fault j's edges,
                              // increasing check order; top byte of entry 0 = degree
    const uint32_t *pad_mask; // [Mp/2][DC] binary16 only: 0xffff in each half of the
                              // pair's physical word p that holds a padding slot
    const float *w;           // [N] prior LLRs
    const float *gamma;       // [(R+1)][N]
    const int32_t *slot_edge; // [Mp*DC] CSR edge id of each message element, -1 for padding
};

// CSR/CSC graph of the plain baseline kernel.
struct BaseGraph {
    int M, N, E;
    int syn_words, cor_words;
    const int32_t *row_ptr;    // [M+1]
    const int32_t *col_idx;    // [E]
    const int32_t *var_ptr;    // [N+1]
    const int32_t *var_edges;  // [E] edges of fault j in increasing edge order
    const float *w;            // [N]
    const float *gamma;        // [(R+1)][N]
};

// Per-code graphs and parameters of a mixed batch, passed by value to the kernel.
constexpr int kMaxMultiCodes = 8;
struct MultiTable {
    int n;
    FusedGraph g[kMaxMultiCodes];
    DevParams p[kMaxMultiCodes];
};

struct DecodeOut {
    uint64_t *corr;
    int32_t *legs;
    uint8_t *conv;
    int32_t *iters;
};

// Which shots a decode launch takes: all B in order (order == nullptr), or the *count
// shots order[0..*count) of a batch; rows of the syndrome / correction arrays are
// syn_stride / cor_stride 64-bit words apart.
struct ShotMap {
    const int32_t *order;
    const int32_t *count;
    int syn_stride, cor_stride;
};

// Tail continuation of a persistent decode (two launches on one stream).  The first
// launch (mode 1) suspends a shot at a leg boundary once it has run `cut` iterations and
// a next leg would start: the shot's Relay state at that boundary goes to record k of
// the list (k from *count; at most cap records, later candidates go on decoding in the
// first launch) and its outputs are left to the second launch (mode 2), which takes the
// records in turn with a wider block shape, restores the state and finishes the shots.
// The kept solution of a suspended shot is already in its correction row.  Mode 0: no
// continuation.  A leg boundary holds the whole state of Relay, so both paths give the
// same results.  The second launch runs the kernel's RESUME instance.
struct TailRecord {
    int32_t shot;
    int32_t leg;          // the leg that starts when the shot resumes
    int32_t sols;         // solutions found so far
    int32_t have;         // 1: a solution is kept (in the shot's correction row)
    long long iters;      // iterations run so far
    long long Wbest;      // weight of the kept solution (2^-33 units)
};
struct TailCont {
    int mode;             // 0 none, 1 suspend long shots (the second launch ignores it)
    int cap;              // records available
    long long cut;        // iterations before a shot may be suspended (mode 1)
    TailRecord *rec;      // [cap]
    float *lam;           // [cap][N] Lambda of each suspended shot at its boundary
    unsigned int *count;  // suspension candidates so far (records used: min(count, cap))
};

// One compiled instance of the fused kernel.
struct FusedKernel {
    int msg_fp16;   // 0 float32 storage, 1 binary16 storage
    int threads;    // NT
    int min_blocks; // launch-bounds residency target
    int vpt;        // faults per thread (register-resident)
    int dc, dv;     // max check / fault degree supported
    const void *decode_fn;   // __global__ symbol of the decode kernel
    cudaError_t (*launch_decode)(dim3 grid, size_t smem, cudaStream_t st, const FusedGraph &g,
                                 const DevParams &p, const uint64_t *syn, int B, DecodeOut out,
                                 unsigned int *counter, ShotMap map, TailCont tc);
    const void *resume_fn;   // __global__ symbol of the resuming instance (nullptr if none)
    cudaError_t (*launch_resume)(dim3 grid, size_t smem, cudaStream_t st, const FusedGraph &g,
                                 const DevParams &p, const uint64_t *syn, int B, DecodeOut out,
                                 unsigned int *counter, ShotMap map, TailCont tc);
    const void *multi_fn;    // __global__ symbol of the mixed-batch kernel
    cudaError_t (*launch_multi)(dim3 grid, size_t smem, cudaStream_t st, const MultiTable &tab,
                                const int32_t *code_of_shot, const uint64_t *syn,
                                int syn_stride, int cor_stride, int B, DecodeOut out,
                                unsigned int *counter);
    const void *trace_fn;    // __global__ symbol of the trace kernel (nullptr if none)
    cudaError_t (*launch_trace)(dim3 grid, size_t smem, cudaStream_t st, const FusedGraph &g,
                                const DevParams &p, const uint64_t *syn, int B, int T,
                                float *marg, float *nu, float *mu);
};

// Shared memory of the fused kernels for a graph (bytes).
inline size_t fused_smem_bytes(int msg_bytes, int f_words, int syn_words, int m_words, int N) {
    size_t msg = ((size_t)msg_bytes + 15) & ~(size_t)15;
    return msg + 8 * (size_t)f_words + 8 * (size_t)syn_words + 8 * (size_t)m_words +
           4 * (size_t)N + 64;
}

// Tables of compiled fused kernels, one per (precision, DC, DV) translation unit.
#define QLDPC_DECLARE_TABLE(P, DC, DV) \
    void fused_table_##P##_##DC##_##DV(const FusedKernel **out, int *n);
QLDPC_DECLARE_TABLE(f32, 8, 4)
QLDPC_DECLARE_TABLE(f32, 16, 8)
QLDPC_DECLARE_TABLE(f32, 32, 8)
QLDPC_DECLARE_TABLE(f16, 8, 4)
QLDPC_DECLARE_TABLE(f16, 16, 8)
QLDPC_DECLARE_TABLE(f16, 32, 8)
#undef QLDPC_DECLARE_TABLE

// Baseline kernel (float32, one shot per block).
size_t baseline_smem_bytes(int M, int N, int E);
const void *baseline_fn();
cudaError_t launch_baseline(int B, int threads, size_t smem, cudaStream_t st, const BaseGraph &g,
                            const DevParams &p, const uint64_t *syn, DecodeOut out);

}  // namespace qldpc
