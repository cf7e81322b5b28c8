// Internal declarations of the soft DMem-BP leg, shared by its kernels and its host API.
#pragma once

#include "qldpc_internal.h"

namespace qldpc {

// CSR / CSC graph of the soft kernels (device pointers).
struct SoftGraph {
    int M, N, E;               // E: edge slots (8 M when the rows are padded)
    int syn_words, cor_words;
    const int32_t *row_ptr;    // [M+1] first slot of each row
    const int32_t *row_deg;    // [M] row degrees when the rows are padded to 8 slots, else null
    const int32_t *col_idx;    // [E] fault of each slot (padding slots: the row's first fault)
    const int32_t *var_ptr;    // [N+1]
    const int32_t *var_edges;  // [E] slots of fault j in increasing slot order
    const uint2 *fault_rec;    // [N] padded rows with E < 2^16 only, else null: the first
                               // three slots of fault j and its degree as 16-bit fields
                               // (x = s0 | s1 << 16, y = s2 | deg << 16; unused slots = s0)
};

// Everything one soft forward or backward launch needs (device pointers; real
// arrays are float or double according to fp64).
struct SoftLaunch {
    SoftGraph g;
    int fp64, dc_max, T_it, K, B;
    double eps;
    const uint64_t *syn, *faults;
    const void *gamma, *alpha, *w, *upstream;
    void *ckpt, *seg, *shot_loss, *shot_gg, *shot_ga, *shot_adj;
    void *loss, *marg, *grad_gamma, *grad_alpha;
};

// Values of one stored state (nu then Lambda): E + N rounded up to a multiple of 4, so
// that every state of a 16-byte aligned workspace starts on a 16-byte boundary.
inline int soft_state_values(const SoftGraph &g) { return (g.E + g.N + 3) & ~3; }

size_t soft_smem_forward(const SoftGraph &g, int fp64);
size_t soft_smem_backward(const SoftGraph &g, int T_it, int fp64);
cudaError_t soft_run_forward(const SoftLaunch &L, cudaStream_t st);
cudaError_t soft_run_backward(const SoftLaunch &L, cudaStream_t st);

}  // namespace qldpc
