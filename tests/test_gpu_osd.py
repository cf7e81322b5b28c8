"""Parity of the CUDA filtered-OSD post-processor (through the C ABI) with the oracle.

The plain-BP marginals are float32 on both sides (the oracle's single-precision
mirror), so the ranking, and with it the GF(2) system and its solution, must match bit
for bit: status, |R| and the correction of every shot.
"""
import numpy as np
import pytest

from oracle.osd import OSDParams, bp_llrs, filtered_osd, first_leg_then_osd as oracle_pipeline
from workloads import (BB72, BB144, BB288, gamma_table, pack_bits, phenomenological_dem,
                       sample_faults, syndromes_of, unpack_bits)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2511_21660_gb300 import (FilteredOSD, QLDPC_OSD_SKIPPED, QLDPC_OSD_SOLVED,  # noqa: E402
                                    RelayConfig, RelayDecoder, first_leg_then_osd)

def _shots(P, n, seed):
    F = sample_faults(P.p, seed, n)
    return F, syndromes_of(P.row_ptr, P.col_idx, F)


def _gpu_osd(P, sig, prm, skip=None, init=None):
    osd = FilteredOSD(P.row_ptr, P.col_idx, P.p, prm.bp_iters, prm.llr_confident,
                      prm.max_candidates)
    try:
        syn = torch.from_numpy(pack_bits(sig).view(np.int64)).cuda()
        B = sig.shape[0]
        cor = (torch.from_numpy(pack_bits(init).view(np.int64)).cuda() if init is not None
               else torch.zeros((B, osd.correction_words), dtype=torch.int64, device="cuda"))
        sk = torch.from_numpy(skip.astype(np.uint8)).cuda() if skip is not None else None
        st, nc = osd.decode(syn, cor, skip=sk)
        torch.cuda.synchronize()
        return (unpack_bits(cor.cpu().numpy().view(np.uint64), P.N), st.cpu().numpy(),
                nc.cpu().numpy())
    finally:
        osd.close()


def _oracle_osd(P, sig, prm):
    L = bp_llrs(P.row_ptr, P.col_idx, P.p, sig, prm.bp_iters, precision="f32")
    out = [filtered_osd(P.H, sig[b], L[b], prm) for b in range(sig.shape[0])]
    return (np.array([o[0] for o in out]), np.array([o[1] for o in out]),
            np.array([o[2] for o in out]))


def _assert_same(got, ref, label):
    cor, st, nc = got
    rcor, rst, rnc = ref
    assert (st == rst).all(), (label, np.nonzero(st != rst)[0][:5], st[st != rst][:5],
                               rst[st != rst][:5])
    assert (nc == rnc).all(), (label, nc[nc != rnc][:5], rnc[nc != rnc][:5])
    ok = st == QLDPC_OSD_SOLVED
    assert (cor[ok] == rcor[ok]).all(), (label, np.nonzero((cor[ok] != rcor[ok]).any(1))[0][:5])


# (code, rounds, p, shots, llr_confident, max_candidates): the 512-thread kernel with 8
# faults per thread (N = 720, 2736) and with 16 (N = 8064); |R|_max 500 and 1024
CASES = [(BB72, 6, 0.04, 300, 4.0, 500),
         (BB144, 12, 0.02, 300, 8.0, 500),
         (BB144, 12, 0.02, 120, 12.0, 1024),
         (BB288, 18, 0.012, 60, 10.0, 500)]


@pytest.mark.parametrize("code,T,p,n,conf,rmax", CASES)
def test_osd_matches_oracle_on_every_shot(code, T, p, n, conf, rmax):
    P = phenomenological_dem(code, T, p)
    F, sig = _shots(P, n, 11)
    prm = OSDParams(bp_iters=25, llr_confident=conf, max_candidates=rmax)
    got = _gpu_osd(P, sig, prm)
    ref = _oracle_osd(P, sig, prm)
    _assert_same(got, ref, f"{code.n} T={T}")
    st = got[1]
    assert (st == QLDPC_OSD_SOLVED).sum() >= n // 3
    if rmax == 1024:  # every width of the eliminated rows: 8 or 16 words in registers, lane groups
        nc = got[2]
        for lo, hi in ((1, 256), (257, 512), (513, rmax)):
            assert ((nc >= lo) & (nc <= hi)).any(), (lo, hi)
    ok = st == QLDPC_OSD_SOLVED
    assert (((got[0][ok].astype(np.int64) @ P.H.T.astype(np.int64)) % 2) == sig[ok]).all()


def test_edge_cases_cap_empty_ranking_zero_syndrome_and_skip():
    P = phenomenological_dem(BB144, 12, 0.02)
    F, sig = _shots(P, 64, 5)
    sig[:4] = 0                                         # zero syndromes
    # tiny cap: most shots have too many candidates
    prm = OSDParams(25, 8.0, 3)
    _assert_same(_gpu_osd(P, sig, prm), _oracle_osd(P, sig, prm), "cap")
    # threshold below every marginal: R empty; only zero syndromes are solvable
    prm = OSDParams(25, -1e6, 500)
    got = _gpu_osd(P, sig, prm)
    _assert_same(got, _oracle_osd(P, sig, prm), "empty")
    assert (got[1][:4] == QLDPC_OSD_SOLVED).all() and not got[0][:4].any()
    assert (got[1][4:] == -2).all()
    # no BP iteration: the ranking is by priors alone
    prm = OSDParams(0, 8.0, 1024)
    _assert_same(_gpu_osd(P, sig, prm), _oracle_osd(P, sig, prm), "bp0")
    # skipped shots keep their corrections and report status 0
    prm = OSDParams(25, 8.0, 500)
    skip = np.zeros(64, bool)
    skip[::3] = True
    init = np.zeros((64, P.N), np.uint8)
    init[:, 7] = 1
    cor, st, nc = _gpu_osd(P, sig, prm, skip=skip, init=init)
    assert (st[skip] == QLDPC_OSD_SKIPPED).all() and (nc[skip] == 0).all()
    assert (cor[skip] == init[skip]).all()
    ref = _oracle_osd(P, sig[~skip], prm)
    _assert_same((cor[~skip], st[~skip], nc[~skip]), ref, "skip")
    failed = ~skip & (st != QLDPC_OSD_SOLVED)
    assert (cor[failed] == init[failed]).all()


def test_first_leg_then_osd_pipeline_matches_oracle():
    P = phenomenological_dem(BB144, 12, 0.02)
    F, sig = _shots(P, 8000, 21)
    g0 = gamma_table(P.N, 0, 0.125, -0.24, 0.66, 3)
    first = RelayDecoder(P.row_ptr, P.col_idx, P.p, g0,
                         RelayConfig(legs_after_first=0, stop_after_solutions=1))
    prm = OSDParams(25, 8.0, 500)
    osd = FilteredOSD(P.row_ptr, P.col_idx, P.p, prm.bp_iters, prm.llr_confident,
                      prm.max_candidates)
    syn = torch.from_numpy(pack_bits(sig).view(np.int64)).cuda()
    cor, st, nc, conv = first_leg_then_osd(first, osd, syn)
    torch.cuda.synchronize()
    cor = unpack_bits(cor.cpu().numpy().view(np.uint64), P.N)
    st, nc, conv = st.cpu().numpy(), nc.cpu().numpy(), conv.cpu().numpy()
    first.close()
    osd.close()
    todo = np.nonzero(conv == 0)[0]
    assert todo.size >= 20
    Fo, sto, nco = oracle_pipeline(P.H, P.row_ptr, P.col_idx, P.p, g0[0], sig[todo], prm)
    assert (st[todo] == sto).all() and (nc[todo] == nco).all()
    assert (cor[todo] == Fo).all()
    assert (st[conv == 1] == QLDPC_OSD_SKIPPED).all()


def test_full_size_post_processing_sampled_parity():
    """The benchmark's post-processing workload: 10^5 gross shots at p = 0.02, first Relay
    leg, then filtered-OSD and the cluster decoder on the unconverged shots; sampled
    unconverged shots against the oracle."""
    from oracle.cluster import ClusterParams, bp_uf
    from paper_2511_21660_gb300 import ClusterDecoder
    P = phenomenological_dem(BB144, 12, 0.02)
    F, sig = _shots(P, 100000, 2)
    g0 = gamma_table(P.N, 0, 0.125, -0.24, 0.66, 2)
    first = RelayDecoder(P.row_ptr, P.col_idx, P.p, g0,
                         RelayConfig(legs_after_first=0, stop_after_solutions=1))
    osd = FilteredOSD(P.row_ptr, P.col_idx, P.p, 25, 8.0, 500)
    cl = ClusterDecoder(P.row_ptr, P.col_idx, P.p, 25, -0.5, 4.5, 4096, 512)
    syn = torch.from_numpy(pack_bits(sig).view(np.int64)).cuda()
    cor, _, conv, _ = first.decode(syn)
    cor_cl = cor.clone()
    st, nc = osd.decode(syn, cor, skip=conv)
    stc, steps = cl.decode(syn, cor_cl, skip=conv)
    torch.cuda.synchronize()
    conv = conv.cpu().numpy()
    cor = unpack_bits(cor.cpu().numpy().view(np.uint64), P.N)
    cor_cl = unpack_bits(cor_cl.cpu().numpy().view(np.uint64), P.N)
    st, nc, stc, steps = (x.cpu().numpy() for x in (st, nc, stc, steps))
    for d in (first, osd, cl):
        d.close()
    todo = np.nonzero(conv == 0)[0]
    assert todo.size >= 300
    pick = np.random.default_rng(1).choice(todo, 40, replace=False)
    L = bp_llrs(P.row_ptr, P.col_idx, P.p, sig[pick], 25, precision="f32")
    for k, b in enumerate(pick):
        f, s_, n = filtered_osd(P.H, sig[b], L[k], OSDParams(25, 8.0, 500))
        assert st[b] == s_ and nc[b] == n
        if s_ == 1:
            assert (cor[b] == f).all()
        f, s_, n = bp_uf(P.H, sig[b], L[k], ClusterParams(25, -0.5, 4.5, 512, 4096))
        assert stc[b] == s_ and steps[b] == n
        if s_ == 1:
            assert (cor_cl[b] == f).all()


@pytest.mark.parametrize("dc_wide", [(9, 17), (17, 33)])
def test_osd_and_cluster_on_wider_check_families(dc_wide):
    """Random graphs whose widest checks put them in the 16- and 32-slot families."""
    from oracle.cluster import ClusterParams, bp_uf
    from paper_2511_21660_gb300 import ClusterDecoder
    from workloads import DecodingProblem
    rng = np.random.default_rng(31 + dc_wide[0])
    M, N = 150, 300
    H = np.zeros((M, N), dtype=np.uint8)
    for j in range(N):
        H[rng.choice(M, int(rng.integers(1, 5)), replace=False), j] = 1
    for i in rng.choice(M, 6, replace=False):
        H[i, :] = 0
        free = np.nonzero(H.sum(0) < 4)[0]
        H[i, rng.choice(free, int(rng.integers(*dc_wide)), replace=False)] = 1
    assert dc_wide[0] <= H.sum(1).max() < dc_wide[1]
    p = rng.uniform(0.01, 0.08, N)
    P = DecodingProblem("wide", H, np.zeros((1, N), np.uint8), p, {"code": "bb72"})
    F = (rng.random((60, N)) < p).astype(np.uint8)
    sig = ((F.astype(np.int64) @ H.T.astype(np.int64)) % 2).astype(np.uint8)
    prm = OSDParams(25, 4.0, 300)
    _assert_same(_gpu_osd(P, sig, prm), _oracle_osd(P, sig, prm), f"osd {dc_wide}")
    cp = ClusterParams(25, -0.5, 3.0, 512, 4096)
    cl = ClusterDecoder(P.row_ptr, P.col_idx, P.p, 25, -0.5, 3.0, 4096, 512)
    syn = torch.from_numpy(pack_bits(sig).view(np.int64)).cuda()
    cor = torch.zeros((60, cl.correction_words), dtype=torch.int64, device="cuda")
    st, steps = cl.decode(syn, cor)
    torch.cuda.synchronize()
    cl.close()
    cor = unpack_bits(cor.cpu().numpy().view(np.uint64), N)
    st, steps = st.cpu().numpy(), steps.cpu().numpy()
    L = bp_llrs(P.row_ptr, P.col_idx, P.p, sig, 25, precision="f32")
    for b in range(60):
        f, s_, n = bp_uf(H, sig[b], L[b], cp)
        assert st[b] == s_ and steps[b] == n, (b, st[b], s_, steps[b], n)
        if s_ == 1:
            assert (cor[b] == f).all()


def test_one_handle_with_skip_masks_of_growing_and_shrinking_batches():
    """The handle's list of shots to post-process is allocated on the first masked call
    and reallocated when a batch grows: masked calls of 40, 300, 90 and 16 shots on one
    handle, one with every shot skipped and one with none, against the oracle."""
    P = phenomenological_dem(BB72, 6, 0.04)
    prm = OSDParams(25, 4.0, 500)
    osd = FilteredOSD(P.row_ptr, P.col_idx, P.p, prm.bp_iters, prm.llr_confident,
                      prm.max_candidates)
    try:
        rng = np.random.default_rng(9)
        for k, n in enumerate((40, 300, 90, 16, 16)):
            F, sig = _shots(P, n, 30 + k)
            skip = rng.random(n) < 0.5
            if k == 3:
                skip[:] = True
            if k == 4:
                skip[:] = False
            syn = torch.from_numpy(pack_bits(sig).view(np.int64)).cuda()
            cor = torch.zeros((n, osd.correction_words), dtype=torch.int64, device="cuda")
            st, nc = osd.decode(syn, cor, skip=torch.from_numpy(skip.astype(np.uint8)).cuda())
            torch.cuda.synchronize()
            st, nc = st.cpu().numpy(), nc.cpu().numpy()
            got = unpack_bits(cor.cpu().numpy().view(np.uint64), P.N)
            assert (st[skip] == QLDPC_OSD_SKIPPED).all() and (nc[skip] == 0).all()
            if (~skip).any():
                ref = _oracle_osd(P, sig[~skip], prm)
                _assert_same((got[~skip], st[~skip], nc[~skip]), ref, f"call {k}")
    finally:
        osd.close()
