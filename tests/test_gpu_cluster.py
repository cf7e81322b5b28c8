"""Parity of the CUDA cluster decoder (through the C ABI) with the oracle.

The plain-BP marginals are float32 on both sides, so the partial correction, the
erasures, every growth and merge step and every cluster solution must match: status,
growth-step count and the correction of every shot, bit for bit.
"""
import numpy as np
import pytest

from oracle.cluster import ClusterParams, bp_uf, first_leg_then_cluster as oracle_pipeline
from oracle.osd import bp_llrs
from workloads import (BB72, BB144, BB288, gamma_table, pack_bits, phenomenological_dem,
                       sample_faults, syndromes_of, unpack_bits)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2511_21660_gb300 import (QLDPC_CLUSTER_DECODED, QLDPC_CLUSTER_SKIPPED,  # noqa: E402
                                    ClusterDecoder, RelayConfig, RelayDecoder,
                                    first_leg_then_cluster)


def _shots(P, n, seed):
    F = sample_faults(P.p, seed, n)
    return F, syndromes_of(P.row_ptr, P.col_idx, F)


def _gpu(P, sig, prm, skip=None, init=None):
    dec = ClusterDecoder(P.row_ptr, P.col_idx, P.p, prm.bp_iters, prm.llr_accept, prm.llr_erase,
                         prm.max_clusters, prm.max_cluster_faults)
    try:
        syn = torch.from_numpy(pack_bits(sig).view(np.int64)).cuda()
        B = sig.shape[0]
        cor = (torch.from_numpy(pack_bits(init).view(np.int64)).cuda() if init is not None
               else torch.zeros((B, dec.correction_words), dtype=torch.int64, device="cuda"))
        sk = torch.from_numpy(skip.astype(np.uint8)).cuda() if skip is not None else None
        st, steps = dec.decode(syn, cor, skip=sk)
        torch.cuda.synchronize()
        return (unpack_bits(cor.cpu().numpy().view(np.uint64), P.N), st.cpu().numpy(),
                steps.cpu().numpy())
    finally:
        dec.close()


def _oracle(P, sig, prm):
    L = bp_llrs(P.row_ptr, P.col_idx, P.p, sig, prm.bp_iters, precision="f32")
    out = [bp_uf(P.H, sig[b], L[b], prm) for b in range(sig.shape[0])]
    return (np.array([o[0] for o in out]), np.array([o[1] for o in out]),
            np.array([o[2] for o in out]))


def _assert_same(got, ref, label):
    cor, st, steps = got
    rcor, rst, rsteps = ref
    assert (st == rst).all(), (label, np.nonzero(st != rst)[0][:5], st[st != rst][:5],
                               rst[st != rst][:5])
    assert (steps == rsteps).all(), (label, np.nonzero(steps != rsteps)[0][:5])
    ok = st == QLDPC_CLUSTER_DECODED
    assert (cor[ok] == rcor[ok]).all(), (label, np.nonzero((cor[ok] != rcor[ok]).any(1))[0][:5])


# (code, rounds, p, shots, accept, erase): 512 threads x 8 faults (N = 720, 2736) and
# x 16 faults (N = 8064)
CASES = [(BB72, 6, 0.04, 60, -0.5, 3.5),
         (BB144, 12, 0.02, 60, -0.5, 4.5),
         (BB144, 12, 0.02, 30, -4.5, 8.5),
         (BB288, 18, 0.012, 12, -0.5, 5.0)]


@pytest.mark.parametrize("code,T,p,n,acc,era", CASES)
def test_cluster_matches_oracle_on_every_shot(code, T, p, n, acc, era):
    P = phenomenological_dem(code, T, p)
    F, sig = _shots(P, n, 13)
    prm = ClusterParams(25, acc, era, max_cluster_faults=512, max_clusters=4096)
    got = _gpu(P, sig, prm)
    _assert_same(got, _oracle(P, sig, prm), f"{code.n} T={T}")
    ok = got[1] == QLDPC_CLUSTER_DECODED
    assert ok.sum() >= n // 2
    assert (((got[0][ok].astype(np.int64) @ P.H.T.astype(np.int64)) % 2) == sig[ok]).all()


def test_caps_and_skip():
    P = phenomenological_dem(BB144, 12, 0.02)
    F, sig = _shots(P, 40, 17)
    for prm in (ClusterParams(25, -0.5, 4.5, max_cluster_faults=512, max_clusters=6),
                ClusterParams(25, -0.5, 4.5, max_cluster_faults=6, max_clusters=4096)):
        got = _gpu(P, sig, prm)
        _assert_same(got, _oracle(P, sig, prm), "cap")
        assert (got[1] < 0).sum() >= 3
    prm = ClusterParams(25, -0.5, 4.5, max_cluster_faults=512, max_clusters=4096)
    skip = np.zeros(40, bool)
    skip[1::4] = True
    init = np.zeros((40, P.N), np.uint8)
    init[:, 3] = 1
    cor, st, steps = _gpu(P, sig, prm, skip=skip, init=init)
    assert (st[skip] == QLDPC_CLUSTER_SKIPPED).all() and (cor[skip] == init[skip]).all()
    _assert_same((cor[~skip], st[~skip], steps[~skip]), _oracle(P, sig[~skip], prm), "skip")


def test_first_leg_then_cluster_pipeline_matches_oracle():
    P = phenomenological_dem(BB144, 12, 0.02)
    F, sig = _shots(P, 6000, 23)
    g0 = gamma_table(P.N, 0, 0.125, -0.24, 0.66, 3)
    first = RelayDecoder(P.row_ptr, P.col_idx, P.p, g0,
                         RelayConfig(legs_after_first=0, stop_after_solutions=1))
    prm = ClusterParams(25, -0.5, 4.5, max_cluster_faults=512, max_clusters=4096)
    cl = ClusterDecoder(P.row_ptr, P.col_idx, P.p, prm.bp_iters, prm.llr_accept, prm.llr_erase,
                        prm.max_clusters, prm.max_cluster_faults)
    syn = torch.from_numpy(pack_bits(sig).view(np.int64)).cuda()
    cor, st, steps, conv = first_leg_then_cluster(first, cl, syn)
    torch.cuda.synchronize()
    cor = unpack_bits(cor.cpu().numpy().view(np.uint64), P.N)
    st, steps, conv = st.cpu().numpy(), steps.cpu().numpy(), conv.cpu().numpy()
    first.close()
    cl.close()
    todo = np.nonzero(conv == 0)[0]
    assert todo.size >= 15
    Fo, sto, stepso = oracle_pipeline(P.H, P.row_ptr, P.col_idx, P.p, g0[0], sig[todo], prm)
    assert (st[todo] == sto).all() and (steps[todo] == stepso).all()
    assert (cor[todo] == Fo).all()
    assert (st[conv == 1] == QLDPC_CLUSTER_SKIPPED).all()


def test_one_handle_with_skip_masks_of_growing_and_shrinking_batches():
    """The handle's list of shots to post-process is allocated on the first masked call
    and reallocated when a batch grows: masked calls of 30, 200, 70 and 12 shots on one
    handle, one with every shot skipped and one with none, against the oracle."""
    P = phenomenological_dem(BB72, 6, 0.04)
    prm = ClusterParams(25, -0.5, 3.5, max_cluster_faults=512, max_clusters=4096)
    dec = ClusterDecoder(P.row_ptr, P.col_idx, P.p, prm.bp_iters, prm.llr_accept, prm.llr_erase,
                         prm.max_clusters, prm.max_cluster_faults)
    try:
        rng = np.random.default_rng(4)
        for k, n in enumerate((30, 200, 70, 12, 12)):
            F, sig = _shots(P, n, 50 + k)
            skip = rng.random(n) < 0.5
            if k == 3:
                skip[:] = True
            if k == 4:
                skip[:] = False
            syn = torch.from_numpy(pack_bits(sig).view(np.int64)).cuda()
            cor = torch.zeros((n, dec.correction_words), dtype=torch.int64, device="cuda")
            st, steps = dec.decode(syn, cor, skip=torch.from_numpy(skip.astype(np.uint8)).cuda())
            torch.cuda.synchronize()
            st, steps = st.cpu().numpy(), steps.cpu().numpy()
            got = unpack_bits(cor.cpu().numpy().view(np.uint64), P.N)
            assert (st[skip] == QLDPC_CLUSTER_SKIPPED).all() and (got[skip] == 0).all()
            if (~skip).any():
                ref = _oracle(P, sig[~skip], prm)
                _assert_same((got[~skip], st[~skip], steps[~skip]), ref, f"call {k}")
    finally:
        dec.close()
