// Fused persistent Relay-BP kernel (paper Sec. 2.3 "Relay decoding", App. A.3).
//
// One thread block decodes one syndrome at a time and pulls the next one from a
// global work counter when it finishes (per-shot early exit, no idle blocks
// behind slow shots).  Per shot:
//   * every edge's message lives in shared memory in one slot, overwritten in
//     place: the check pass turns nu(t-1) into mu(t), the fault pass turns mu(t)
//     into nu(t).  The DC slots of a check are contiguous (128-bit loads and
//     stores in the check pass), with their order inside the check XOR-swizzled
//     by the check index so that the fault pass's gathers and scatters over
//     consecutive checks fall into distinct banks;
//   * the per-fault state (Lambda_j, (1-gamma_j) lambda_j(0), gamma_j) lives in
//     registers: fault j belongs to thread j mod NT for the whole shot;
//   * decisions F_j = [Lambda_j < 0] are packed by warp ballots into a bitmap, and
//     the syndrome H F is accumulated by the (few) faults with F_j = 1.
// All float arithmetic rounds every + and * separately (__fadd_rn/__fmul_rn), in
// the same order as the single-precision oracle, so results are bit-identical.
//
// This translation unit is compiled once per (message precision, max check
// degree DC, max fault degree DV), selected by QL_MSG_F16, QL_DC and QL_DV.
#include "relay_device.cuh"

#ifndef QL_MSG_F16
#define QL_MSG_F16 0
#endif
#ifndef QL_DC
#define QL_DC 8
#endif
#ifndef QL_DV
#define QL_DV 4
#endif

namespace qldpc {
namespace {

// Relay on one shot: the leg schedule around the check and fault passes.  Per
// iteration: check pass | barrier | fault pass | barrier | per-warp convergence
// test.  A leg end adds the weight sum, the next leg's initialisation and one
// barrier.  Called by every thread of the block with block-uniform arguments.
// SKIP: the shot's code may use only part of the block's fault slots (mixed batches),
// so the per-fault loops stop at the code's last slot.
// wacc[2]: the block's weight accumulators, used in turn (ab selects the one the next
// new solution adds into); the other one is zeroed after each use, at least two
// barriers before it is added into again.  Both start at zero and ab persists across
// the block's shots.
// Tail continuation (TailCont): with tc.mode 1 a shot that reaches a leg boundary after
// tc.cut iterations, with a next leg to run, may be suspended (its state saved in a
// record, no outputs written); rec >= 0 resumes the shot of record rec at its boundary.
// s_slot: a shared int that broadcasts the record taken for a suspension.
template <typename MT, int NT, int VPT, int DC, int DV, bool SKIP = false, bool RESUME = false>
__device__ __forceinline__ void decode_shot(const FusedGraph &g, const DevParams &p, int shot,
                                            const uint64_t *sy, uint64_t *cor, DecodeOut out,
                                            unsigned char *msg, uint32_t *fw, uint32_t *fb,
                                            uint32_t *sg, uint32_t *par, float *ws,
                                            long long *wacc,
                                            float (&Lam)[VPT], float (&bb)[VPT],
                                            float (&gg)[VPT], int &ab, const TailCont &tc,
                                            int rec, int *s_slot) {
    const int tid = threadIdx.x;
    const float C = p.clip;
    load_syndrome<NT>(g, sy, sg);
    int leg = 0, sols = 0, t = 0, pb = 0;
    long long iters = 0, Wbest = 0;
    bool have = false;
    if (RESUME) {  // resume at the boundary where the first launch stopped the shot
        const TailRecord r = tc.rec[rec];
        leg = r.leg;
        sols = r.sols;
        have = r.have != 0;
        iters = r.iters;
        Wbest = r.Wbest;
        const float *lr = tc.lam + (size_t)rec * g.N;
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            const int j = threadIdx.x + q * NT;
            if (j < g.N) Lam[q] = lr[j];
        }
        if (have)  // the kept solution, for the same-solution test
            for (int q = tid; q < g.cor_words; q += NT) {
                const uint64_t v = cor[q];
                fb[2 * q] = (uint32_t)v;
                fb[2 * q + 1] = (uint32_t)(v >> 32);
            }
    }
    leg_init<MT, NT, VPT, DV, SKIP>(g, p, leg, msg, ws, Lam, bb, gg);
    __syncthreads();
    for (;;) {
        uint32_t *pc = par + pb * g.m_words;
        check_pass<NT, DC>(g, reinterpret_cast<MT *>(msg), sg, pc, C);
        __syncthreads();
        const uint32_t dm = fault_pass<MT, NT, VPT, DV, SKIP>(g, msg, fw, pc, Lam, bb, gg, C);
        __syncthreads();
        ++iters;
        ++t;
        pb ^= 1;
        const bool conv = warp_converged(pc, sg, g.m_words);
        const bool spent = p.max_iters > 0 && iters >= p.max_iters;
        const bool leg_end = conv || spent || t == (leg == 0 ? p.T1 : p.T2);
        if (!leg_end) continue;
        // a solution equal to the kept one has its weight and cannot replace it
        const bool fresh = conv && !(have && warp_same_solution(fw, fb, 2 * g.cor_words));
        if (conv) ++sols;
        if (fresh) add_weight<NT>(ws, dm, wacc + ab);
        const bool done = sols >= p.S || leg == p.R || spent;
        if (!done) {
            ++leg;
            t = 0;
            leg_init<MT, NT, VPT, DV, SKIP>(g, p, leg, msg, ws, Lam, bb, gg);
        }
        // a long shot with a next leg to run is suspended if a record is free (the next
        // leg's initialisation is redone on resumption from the same state); thread 0
        // decides and takes the record, *s_slot tells the block (-1: go on)
        if (!RESUME && tid == 0) {
            int k = -1;
            if (!done && tc.mode == 1 && iters >= tc.cut) {
                const unsigned int c = atomicAdd(tc.count, 1u);
                if (c < (unsigned int)tc.cap) k = (int)c;
            }
            *s_slot = k;
        }
        __syncthreads();  // the weight and the next leg's initial messages are visible
        if (fresh) {
            const long long W = wacc[ab];
            if (!have || W < Wbest) {
                keep_solution<NT>(cor, fw, fb, g.cor_words);
                have = true;
                Wbest = W;
            }
            if (tid == 0) wacc[ab ^ 1] = 0;
            ab ^= 1;
        }
        if (!RESUME && *s_slot >= 0) break;
        if (done) break;
    }
    const int slot = RESUME ? -1 : *s_slot;  // this shot's last leg end set it
    if (slot >= 0) {  // suspended: the state at this boundary; the next leg runs on resumption
        float *lr = tc.lam + (size_t)slot * g.N;
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            const int j = threadIdx.x + q * NT;
            if (j < g.N) lr[j] = Lam[q];
        }
        if (tid == 0) tc.rec[slot] = TailRecord{shot, leg, sols, have ? 1 : 0, iters, Wbest};
        return;
    }
    if (!have) store_bits<NT>(cor, fw, g.cor_words);
    if (tid == 0) {
        if (out.legs) out.legs[shot] = leg + 1;
        if (out.conv) out.conv[shot] = have ? 1 : 0;
        if (out.iters) out.iters[shot] = (int32_t)iters;
    }
}

// One block per shot at a time; shots come from a global counter (through the shot
// map's index list when it has one).
// RESUME: the second launch of the tail continuation; shots come from the records of the
// first launch (counter then numbers the records taken).
template <typename MT, int NT, int VPT, int MINB, int DC, int DV, bool RESUME = false>
__global__ void __launch_bounds__(NT, MINB) fused_decode(FusedGraph g, DevParams p,
                                                   const uint64_t *__restrict__ syn, int B,
                                                   DecodeOut out, unsigned int *counter,
                                                   ShotMap map, TailCont tc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *msg = smem_raw;
    uint32_t *fw, *fb, *sg, *par;
    float *ws;
    smem_layout(g, smem_raw, fw, fb, sg, par, ws);
    __shared__ int s_shot, s_rec, s_slot;
    __shared__ long long s_wacc[2];
    block_setup<MT, NT, DC>(g, msg, fw, ws, p.clip);

    float Lam[VPT], bb[VPT], gg[VPT];
#pragma unroll
    for (int r = 0; r < VPT; ++r) Lam[r] = bb[r] = gg[r] = 0.0f;
    int ab = 0;
    if (threadIdx.x < 2) s_wacc[threadIdx.x] = 0;

    const int limit = RESUME ? (int)min(*tc.count, (unsigned int)tc.cap)
                             : (map.order ? min(*map.count, B) : B);
    for (;;) {
        __syncthreads();  // the previous shot is done with shared memory and s_shot
        if (threadIdx.x == 0) {
            const int k = (int)atomicAdd(counter, 1u);
            if (RESUME) {
                s_rec = k < limit ? k : -1;
                s_shot = k < limit ? tc.rec[k].shot : -1;
            } else {
                s_rec = -1;
                s_shot = k < limit ? (map.order ? map.order[k] : k) : -1;
            }
        }
        __syncthreads();
        const int shot = s_shot;
        if (shot < 0) break;
        decode_shot<MT, NT, VPT, DC, DV, false, RESUME>(g, p, shot,
                                         syn + (size_t)shot * map.syn_stride,
                                         out.corr + (size_t)shot * map.cor_stride, out, msg, fw,
                                         fb, sg, par, ws, s_wacc, Lam, bb, gg, ab, tc, s_rec,
                                         &s_slot);
    }
}

// Mixed batch: shot b belongs to code code_of_shot[b] of the table; syndromes and
// corrections are rows of fixed strides.  A block re-initialises its shared state
// (padding slots, priors) whenever it moves to a shot of another code.
template <typename MT, int NT, int VPT, int MINB, int DC, int DV>
__global__ void __launch_bounds__(NT, MINB) fused_decode_multi(MultiTable tab,
                                                         const int32_t *__restrict__ code_of_shot,
                                                         const uint64_t *__restrict__ syn,
                                                         int syn_stride, int cor_stride, int B,
                                                         DecodeOut out, unsigned int *counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *msg = smem_raw;
    __shared__ FusedGraph s_g;
    __shared__ DevParams s_p;
    __shared__ int s_shot, s_code, s_slot;
    __shared__ long long s_wacc[2];
    int cur = -1;

    float Lam[VPT], bb[VPT], gg[VPT];
#pragma unroll
    for (int r = 0; r < VPT; ++r) Lam[r] = bb[r] = gg[r] = 0.0f;
    int ab = 0;
    if (threadIdx.x < 2) s_wacc[threadIdx.x] = 0;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int shot = (int)atomicAdd(counter, 1u);
            s_shot = shot;
            int c = shot < B ? code_of_shot[shot] : 0;
            if (c < 0 || c >= tab.n) c = -1;  // invalid code id: the shot is skipped
            s_code = c;
            if (c >= 0 && c != cur) {
                s_g = tab.g[c];
                s_p = tab.p[c];
            }
        }
        __syncthreads();
        const int shot = s_shot, code = s_code;
        if (shot >= B) break;
        if (code < 0) {  // not a code of the table: marked by iters = -1
            if (threadIdx.x == 0) {
                if (out.legs) out.legs[shot] = 0;
                if (out.conv) out.conv[shot] = 0;
                if (out.iters) out.iters[shot] = -1;
            }
            continue;
        }
        uint32_t *fw, *fb, *sg, *par;
        float *ws;
        smem_layout(s_g, smem_raw, fw, fb, sg, par, ws);
        if (code != cur) {
            block_setup<MT, NT, DC>(s_g, msg, fw, ws, s_p.clip);
            cur = code;
            __syncthreads();
        }
        decode_shot<MT, NT, VPT, DC, DV, true>(s_g, s_p, shot, syn + (size_t)shot * syn_stride,
                                         out.corr + (size_t)shot * cor_stride, out, msg, fw, fb,
                                         sg, par, ws, s_wacc, Lam, bb, gg, ab, TailCont{},
                                         -1, &s_slot);
    }
}

// First leg without early exit, every iteration recorded (one shot per block).
template <typename MT, int NT, int VPT, int DC, int DV>
__global__ void __launch_bounds__(NT) fused_trace(FusedGraph g, DevParams p,
                                                  const uint64_t *__restrict__ syn, int B, int T,
                                                  int E, float *marg, float *nu, float *mu) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *msg = smem_raw;
    uint32_t *fw, *fb, *sg, *par;
    float *ws;
    smem_layout(g, smem_raw, fw, fb, sg, par, ws);
    const int shot = blockIdx.x;
    const float C = p.clip;
    block_setup<MT, NT, DC>(g, msg, fw, ws, C);
    load_syndrome<NT>(g, syn + (size_t)shot * g.syn_words, sg);
    float Lam[VPT], bb[VPT], gg[VPT];
#pragma unroll
    for (int r = 0; r < VPT; ++r) Lam[r] = bb[r] = gg[r] = 0.0f;
    __syncthreads();
    leg_init<MT, NT, VPT, DV>(g, p, 0, msg, ws, Lam, bb, gg);
    __syncthreads();
    const int nslots = g.msg_bytes / (int)sizeof(MT);
    for (int t = 0; t < T; ++t) {
        const size_t o = (size_t)t * B + shot;
        check_pass<NT, DC>(g, reinterpret_cast<MT *>(msg), sg, par, C);
        __syncthreads();
        if (mu)
            for (int s = threadIdx.x; s < nslots; s += NT) {
                const int e = g.slot_edge[s];
                if (e >= 0) mu[o * E + e] = Msg<MT>::ld(msg, s * (int)sizeof(MT));
            }
        __syncthreads();
        fault_pass<MT, NT, VPT, DV>(g, msg, fw, par, Lam, bb, gg, C);
        __syncthreads();
        if (marg) {
#pragma unroll
            for (int r = 0; r < VPT; ++r) {
                const int j = threadIdx.x + r * NT;
                if (j < g.N) marg[o * g.N + j] = Lam[r];
            }
        }
        if (nu)
            for (int s = threadIdx.x; s < nslots; s += NT) {
                const int e = g.slot_edge[s];
                if (e >= 0) nu[o * E + e] = Msg<MT>::ld(msg, s * (int)sizeof(MT));
            }
        __syncthreads();
    }
}

template <typename MT, int NT, int VPT, int MINB, int DC, int DV, bool RESUME>
cudaError_t launch_decode(dim3 grid, size_t smem, cudaStream_t st, const FusedGraph &g,
                          const DevParams &p, const uint64_t *syn, int B, DecodeOut out,
                          unsigned int *counter, ShotMap map, TailCont tc) {
    fused_decode<MT, NT, VPT, MINB, DC, DV, RESUME><<<grid, NT, smem, st>>>(g, p, syn, B, out,
                                                                            counter, map, tc);
    return cudaGetLastError();
}

template <typename MT, int NT, int VPT, int MINB, int DC, int DV>
cudaError_t launch_multi(dim3 grid, size_t smem, cudaStream_t st, const MultiTable &tab,
                         const int32_t *code_of_shot, const uint64_t *syn, int syn_stride,
                         int cor_stride, int B, DecodeOut out, unsigned int *counter) {
    fused_decode_multi<MT, NT, VPT, MINB, DC, DV><<<grid, NT, smem, st>>>(
        tab, code_of_shot, syn, syn_stride, cor_stride, B, out, counter);
    return cudaGetLastError();
}

template <typename MT, int NT, int VPT, int DC, int DV>
cudaError_t launch_trace(dim3 grid, size_t smem, cudaStream_t st, const FusedGraph &g,
                         const DevParams &p, const uint64_t *syn, int B, int T, float *marg,
                         float *nu, float *mu) {
    fused_trace<MT, NT, VPT, DC, DV><<<grid, NT, smem, st>>>(g, p, syn, B, T, g.E, marg, nu, mu);
    return cudaGetLastError();
}

#if QL_MSG_F16
using MsgT = __half;
#else
using MsgT = float;
#endif

template <int NT, int VPT, int MINB, bool TRACE>
FusedKernel entry() {
    FusedKernel k;
    k.msg_fp16 = QL_MSG_F16;
    k.threads = NT;
    k.min_blocks = MINB;
    k.vpt = VPT;
    k.dc = QL_DC;
    k.dv = QL_DV;
    k.decode_fn = (const void *)fused_decode<MsgT, NT, VPT, MINB, QL_DC, QL_DV>;
    k.launch_decode = &launch_decode<MsgT, NT, VPT, MINB, QL_DC, QL_DV, false>;
    if constexpr (NT == 1024) {  // the shapes of the tail continuation's second launch
        k.resume_fn = (const void *)fused_decode<MsgT, NT, VPT, MINB, QL_DC, QL_DV, true>;
        k.launch_resume = &launch_decode<MsgT, NT, VPT, MINB, QL_DC, QL_DV, true>;
    } else {
        k.resume_fn = nullptr;
        k.launch_resume = nullptr;
    }
    k.multi_fn = (const void *)fused_decode_multi<MsgT, NT, VPT, MINB, QL_DC, QL_DV>;
    k.launch_multi = &launch_multi<MsgT, NT, VPT, MINB, QL_DC, QL_DV>;
    if constexpr (TRACE) {
        k.trace_fn = (const void *)fused_trace<MsgT, NT, VPT, QL_DC, QL_DV>;
        k.launch_trace = &launch_trace<MsgT, NT, VPT, QL_DC, QL_DV>;
    } else {
        k.trace_fn = nullptr;
        k.launch_trace = nullptr;
    }
    return k;
}

}  // namespace

#define QL_CAT2(P, DC, DV) fused_table_##P##_##DC##_##DV
#define QL_EXPAND(P, DC, DV) QL_CAT2(P, DC, DV)
#if QL_MSG_F16
#define QL_P f16
#else
#define QL_P f32
#endif

void QL_EXPAND(QL_P, QL_DC, QL_DV)(const FusedKernel **out, int *n) {
    // (threads, faults per thread, min resident blocks): the first entry whose
    // threads * vpt >= N is used unless the caller asks for a block size; the last
    // entry also serves the trace kernel; the 1024-thread entries serve the resuming
    // launch of the tail continuation.
    static const FusedKernel table[] = {
        entry<256, 4, 4, false>(),
        entry<512, 6, 2, false>(),
        entry<256, 12, 4, false>(),
        entry<384, 8, 3, false>(),
        entry<640, 5, 2, false>(),
        entry<768, 4, 2, false>(),
        entry<1024, 3, 1, false>(),
        entry<1024, 8, 1, false>(),
        entry<512, 16, 1, false>(),
        entry<512, 32, 1, true>(),
    };
    *out = table;
    *n = (int)(sizeof(table) / sizeof(table[0]));
}

}  // namespace qldpc
