"""Soft DMem-BP on the GPU (forward, adjoint, autograd) against the FP64 oracle and
against finite differences.

The adjoint is checked in FP64 on the [[72,12,6]] code: against the oracle's own
reverse pass and against central finite differences of the GPU forward (1e-6
relative).  FP64 runs on the GPU only in these gradient checks; decoding never
uses it.
"""
import numpy as np
import pytest

from oracle.soft import soft_dmem
from workloads import BB72, BB144, code_capacity_dem, pack_bits, phenomenological_dem, \
    sample_faults, syndromes_of

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2511_21660_gb300 import SoftDMem, soft_dmem_loss  # noqa: E402

EPS32 = 2.0 ** -23


def _case(seed=5, B=12, T=25):
    P = code_capacity_dem(BB72, 0.05)
    F = sample_faults(P.p, seed, B)
    s = syndromes_of(P.row_ptr, P.col_idx, F)
    rng = np.random.default_rng(seed)
    gam = rng.uniform(0.0, 0.3, P.N)
    alpha = rng.uniform(0.25, 0.4, T)   # unsaturated: no product reaches the clamp
    return P, F, s, gam, alpha


def _dev(P, F, s, gam, alpha, dtype):
    syn = torch.from_numpy(pack_bits(s).view(np.int64)).cuda()
    flt = torch.from_numpy(pack_bits(F).view(np.int64)).cuda()
    g = torch.tensor(gam, dtype=dtype, device="cuda")
    a = torch.tensor(alpha, dtype=dtype, device="cuda")
    return syn, flt, g, a


def test_fp64_forward_and_adjoint_match_oracle():
    P, F, s, gam, alpha = _case()
    L_ref, gg_ref, ga_ref, m_ref = soft_dmem(P.row_ptr, P.col_idx, P.p, gam, alpha, s, F,
                                             marginals=True)
    soft = SoftDMem(P.row_ptr, P.col_idx, P.p, iterations=25, checkpoint_every=5,
                    dtype=torch.float64)
    syn, flt, g, a = _dev(P, F, s, gam, alpha, torch.float64)
    loss, marg, ws = soft.forward(syn, flt, g, a, marginals=True)
    gg, ga = soft.backward(syn, flt, g, a, ws)
    torch.cuda.synchronize()
    assert abs(loss.item() - L_ref) <= 1e-12 * L_ref
    np.testing.assert_allclose(marg.cpu().numpy(), m_ref, rtol=1e-11, atol=1e-11)
    assert np.abs(gg.cpu().numpy() - gg_ref).max() <= 1e-9 * np.abs(gg_ref).max()
    assert np.abs(ga.cpu().numpy() - ga_ref).max() <= 1e-9 * np.abs(ga_ref).max()
    soft.close()


def test_fp64_adjoint_matches_finite_differences_72_qubit_code():
    """Every component of d loss / d gamma (72) and d loss / d alpha (25), h = 1e-6."""
    P, F, s, gam, alpha = _case(seed=9)
    soft = SoftDMem(P.row_ptr, P.col_idx, P.p, iterations=25, checkpoint_every=5,
                    dtype=torch.float64)
    syn, flt, g, a = _dev(P, F, s, gam, alpha, torch.float64)
    ws = soft.workspace(syn.shape[0])
    soft.forward(syn, flt, g, a, workspace=ws)
    gg, ga = soft.backward(syn, flt, g, a, ws)
    gg, ga = gg.cpu().numpy(), ga.cpu().numpy()
    h = 1e-6

    def loss(gv, av):
        return soft.forward(syn, flt, gv, av, workspace=ws)[0].item()

    fd_g = np.array([(loss(g + h * e, a) - loss(g - h * e, a)) / (2 * h)
                     for e in torch.eye(P.N, dtype=torch.float64, device="cuda")])
    fd_a = np.array([(loss(g, a + h * e) - loss(g, a - h * e)) / (2 * h)
                     for e in torch.eye(25, dtype=torch.float64, device="cuda")])
    assert np.abs(fd_g - gg).max() <= 1e-6 * np.abs(gg).max()
    assert np.abs(fd_a - ga).max() <= 1e-6 * np.abs(ga).max()
    soft.close()


def test_checkpoint_interval_does_not_change_the_gradient():
    P, F, s, gam, alpha = _case(seed=2, T=12)
    out = []
    for K in (1, 5, 12):
        soft = SoftDMem(P.row_ptr, P.col_idx, P.p, iterations=12, checkpoint_every=K,
                        dtype=torch.float64)
        syn, flt, g, a = _dev(P, F, s, gam, alpha, torch.float64)
        loss, _, ws = soft.forward(syn, flt, g, a)
        gg, ga = soft.backward(syn, flt, g, a, ws)
        out.append((loss.item(), gg.cpu().numpy(), ga.cpu().numpy()))
        soft.close()
    for o in out[1:]:
        assert o[0] == out[0][0]
        assert np.array_equal(o[1], out[0][1]) and np.array_equal(o[2], out[0][2])


def test_fp32_tracks_fp64_oracle():
    P, F, s, gam, alpha = _case(seed=4)
    L_ref, gg_ref, ga_ref, m_ref = soft_dmem(P.row_ptr, P.col_idx, P.p, gam, alpha, s, F,
                                             eps=EPS32, marginals=True)
    soft = SoftDMem(P.row_ptr, P.col_idx, P.p, iterations=25, checkpoint_every=5)
    syn, flt, g, a = _dev(P, F, s, gam.astype(np.float32), alpha.astype(np.float32),
                          torch.float32)
    loss, marg, ws = soft.forward(syn, flt, g, a, marginals=True)
    gg, ga = soft.backward(syn, flt, g, a, ws)
    torch.cuda.synchronize()
    # float32 inputs are the rounded gamma/alpha: compare with the oracle on those
    L_ref, gg_ref, ga_ref, m_ref = soft_dmem(P.row_ptr, P.col_idx, P.p,
                                             gam.astype(np.float32).astype(np.float64),
                                             alpha.astype(np.float32).astype(np.float64), s, F,
                                             eps=EPS32, marginals=True)
    err = np.abs(marg.cpu().numpy() - m_ref) / np.maximum(1.0, np.abs(m_ref))
    assert err.max() <= 1e-4, err.max()
    assert abs(loss.item() - L_ref) <= 1e-4 * L_ref
    assert np.abs(gg.cpu().numpy() - gg_ref).max() <= 1e-3 * np.abs(gg_ref).max()
    assert np.abs(ga.cpu().numpy() - ga_ref).max() <= 1e-3 * np.abs(ga_ref).max()
    soft.close()


def test_autograd_function_matches_direct_backward():
    P, F, s, gam, alpha = _case(seed=6, T=10)
    soft = SoftDMem(P.row_ptr, P.col_idx, P.p, iterations=10, checkpoint_every=5,
                    dtype=torch.float64)
    syn, flt, g, a = _dev(P, F, s, gam, alpha, torch.float64)
    g.requires_grad_(True)
    a.requires_grad_(True)
    loss = soft_dmem_loss(soft, syn, flt, g, a)
    (3.0 * loss).backward()
    loss2, _, ws = soft.forward(syn, flt, g.detach(), a.detach())
    gg, ga = soft.backward(syn, flt, g.detach(), a.detach(), ws)
    assert torch.allclose(g.grad, 3.0 * gg, rtol=1e-14, atol=0)
    assert torch.allclose(a.grad, 3.0 * ga, rtol=1e-14, atol=0)
    assert loss.item() == loss2.item()
    soft.close()


def test_gross_code_training_steps_reduce_the_loss():
    """Batch 4096 of gross-code T=12 syndromes at p = 0.003, float32, 25 iterations."""
    P = phenomenological_dem(BB144, 12, 0.003)
    F = sample_faults(P.p, 20, 4096)
    s = syndromes_of(P.row_ptr, P.col_idx, F)
    soft = SoftDMem(P.row_ptr, P.col_idx, P.p, iterations=25, checkpoint_every=5)
    syn = torch.from_numpy(pack_bits(s).view(np.int64)).cuda()
    flt = torch.from_numpy(pack_bits(F).view(np.int64)).cuda()
    g = torch.full((P.N,), 0.125, device="cuda", requires_grad=True)
    a = torch.full((25,), 1.0, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([g, a], lr=0.01)
    losses = []
    for _ in range(6):
        opt.zero_grad()
        loss = soft_dmem_loss(soft, syn, flt, g, a)
        loss.backward()
        opt.step()
        losses.append(loss.item())
    assert np.isfinite(losses).all()
    assert losses[-1] < losses[0], losses
    soft.close()


def test_fp32_tracks_fp64_oracle_on_the_gross_code():
    """The benchmark's graph (gross T = 12, 936 x 2736, p = 0.003), 16 shots, 25 iterations.

    The loss and the gradients keep the 72-qubit tolerances.  Single marginals get 1e-3
    relative: with prior LLRs near 5.8 the check products approach +-1, where
    atanh amplifies float32 rounding of the product by 1/(1 - P^2); the largest marginal
    error measured here is 2.9e-4 whether tanh/atanh come from the hardware exponential
    and logarithm or from the accurate library functions, i.e. it is the format's.
    """
    P = phenomenological_dem(BB144, 12, 0.003)
    F = sample_faults(P.p, 21, 16)
    s = syndromes_of(P.row_ptr, P.col_idx, F)
    rng = np.random.default_rng(21)
    gam = rng.uniform(0.0, 0.3, P.N).astype(np.float32).astype(np.float64)
    alpha = rng.uniform(0.25, 0.4, 25).astype(np.float32).astype(np.float64)
    L_ref, gg_ref, ga_ref, m_ref = soft_dmem(P.row_ptr, P.col_idx, P.p, gam, alpha, s, F,
                                             eps=EPS32, marginals=True)
    soft = SoftDMem(P.row_ptr, P.col_idx, P.p, iterations=25, checkpoint_every=5)
    syn, flt, g, a = _dev(P, F, s, gam, alpha, torch.float32)
    loss, marg, ws = soft.forward(syn, flt, g, a, marginals=True)
    gg, ga = soft.backward(syn, flt, g, a, ws)
    torch.cuda.synchronize()
    err = np.abs(marg.cpu().numpy() - m_ref) / np.maximum(1.0, np.abs(m_ref))
    assert err.max() <= 1e-3, err.max()
    assert abs(loss.item() - L_ref) <= 1e-4 * L_ref
    assert np.abs(gg.cpu().numpy() - gg_ref).max() <= 1e-3 * np.abs(gg_ref).max()
    assert np.abs(ga.cpu().numpy() - ga_ref).max() <= 1e-3 * np.abs(ga_ref).max()
    soft.close()


def test_fp32_tracks_fp64_oracle_on_a_14_round_gross_graph():
    """Gross code, 14 rounds (1080 x 3168, more faults than 12 per thread): the float32
    forward and adjoint against the FP64 oracle, with the 12-round graph's tolerances."""
    P = phenomenological_dem(BB144, 14, 0.003)
    F = sample_faults(P.p, 23, 8)
    s = syndromes_of(P.row_ptr, P.col_idx, F)
    rng = np.random.default_rng(23)
    gam = rng.uniform(0.0, 0.3, P.N).astype(np.float32).astype(np.float64)
    alpha = rng.uniform(0.25, 0.4, 25).astype(np.float32).astype(np.float64)
    L_ref, gg_ref, ga_ref, m_ref = soft_dmem(P.row_ptr, P.col_idx, P.p, gam, alpha, s, F,
                                             eps=EPS32, marginals=True)
    soft = SoftDMem(P.row_ptr, P.col_idx, P.p, iterations=25, checkpoint_every=5)
    syn, flt, g, a = _dev(P, F, s, gam, alpha, torch.float32)
    loss, marg, ws = soft.forward(syn, flt, g, a, marginals=True)
    gg, ga = soft.backward(syn, flt, g, a, ws)
    torch.cuda.synchronize()
    err = np.abs(marg.cpu().numpy() - m_ref) / np.maximum(1.0, np.abs(m_ref))
    assert err.max() <= 1e-3, err.max()
    assert abs(loss.item() - L_ref) <= 1e-4 * L_ref
    assert np.abs(gg.cpu().numpy() - gg_ref).max() <= 1e-3 * np.abs(gg_ref).max()
    assert np.abs(ga.cpu().numpy() - ga_ref).max() <= 1e-3 * np.abs(ga_ref).max()
    soft.close()


def test_fp32_padded_rows_with_empty_and_short_checks():
    """float32 pads check rows to 8 slots; rows of degree 0 and of degree below 8 (the
    72-qubit code-capacity rows have 6) keep their padding slots out of every product:
    the 72-qubit case with an empty check appended first and last, against the oracle."""
    P, F, s, gam, alpha = _case(seed=8)
    rp = np.concatenate([[0], P.row_ptr, [P.row_ptr[-1]]]).astype(np.int32)
    s2 = np.concatenate([np.zeros((s.shape[0], 1), s.dtype), s,
                         np.zeros((s.shape[0], 1), s.dtype)], axis=1)
    g32 = gam.astype(np.float32).astype(np.float64)
    a32 = alpha.astype(np.float32).astype(np.float64)
    L_ref, gg_ref, ga_ref, m_ref = soft_dmem(rp, P.col_idx, P.p, g32, a32, s2, F, eps=EPS32,
                                             marginals=True)
    soft = SoftDMem(rp, P.col_idx, P.p, iterations=25, checkpoint_every=5)
    syn, flt, g, a = _dev(P, F, s2, g32, a32, torch.float32)
    loss, marg, ws = soft.forward(syn, flt, g, a, marginals=True)
    gg, ga = soft.backward(syn, flt, g, a, ws)
    torch.cuda.synchronize()
    err = np.abs(marg.cpu().numpy() - m_ref) / np.maximum(1.0, np.abs(m_ref))
    assert err.max() <= 1e-4, err.max()
    assert abs(loss.item() - L_ref) <= 1e-4 * L_ref
    assert np.abs(gg.cpu().numpy() - gg_ref).max() <= 1e-3 * np.abs(gg_ref).max()
    assert np.abs(ga.cpu().numpy() - ga_ref).max() <= 1e-3 * np.abs(ga_ref).max()
    soft.close()


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_odd_state_size_generic_fault_degrees_and_partial_last_segment(dtype):
    """A 73-fault graph (the 72-qubit code-capacity matrix without its first column, plus
    a fault of degree 1 and one of degree 4): a state of E + N values that is not a
    multiple of 4, faults outside the degree-2/3 fast paths, and 23 iterations in
    checkpoint segments of 5 (the last one of 3), against the oracle.  The adjoint leaves
    the forward's checkpoints as they were (a second backward on the same workspace gives
    the same gradients, bit for bit), and a workspace that does not start on a 16-byte
    boundary is refused."""
    P, F0, s0, gam0, alpha = _case(seed=6, B=16, T=23)
    H = P.H[:, 1:].astype(np.uint8)
    extra = np.zeros((H.shape[0], 2), np.uint8)
    extra[4, 0] = 1
    extra[:4, 1] = 1
    H = np.concatenate([H, extra], axis=1)
    N = H.shape[1]
    rp = np.concatenate([[0], np.cumsum(H.sum(1))]).astype(np.int32)
    ci = np.concatenate([np.nonzero(r)[0] for r in H]).astype(np.int32)
    assert (N + 8 * H.shape[0]) % 4 != 0 and H.sum(1).max() <= 8
    pr = np.concatenate([P.p[1:], [0.05, 0.05]])
    F = sample_faults(pr, 6, 16)
    s = syndromes_of(rp, ci, F)
    gam = np.random.default_rng(6).uniform(0.0, 0.3, N)
    tdt = getattr(torch, dtype)
    if dtype == "float32":
        gam = gam.astype(np.float32).astype(np.float64)
        alpha = alpha.astype(np.float32).astype(np.float64)
    L_ref, gg_ref, ga_ref, m_ref = soft_dmem(rp, ci, pr, gam, alpha, s, F,
                                             eps=EPS32 if dtype == "float32" else 1e-15,
                                             marginals=True)
    soft = SoftDMem(rp, ci, pr, iterations=23, checkpoint_every=5, dtype=tdt)
    syn, flt, g, a = _dev(None, F, s, gam, alpha, tdt)
    loss, marg, ws = soft.forward(syn, flt, g, a, marginals=True)
    gg, ga = soft.backward(syn, flt, g, a, ws)
    gg2, ga2 = soft.backward(syn, flt, g, a, ws)
    torch.cuda.synchronize()
    tol_m, tol_g = (1e-4, 1e-3) if dtype == "float32" else (1e-11, 1e-9)
    err = np.abs(marg.cpu().numpy() - m_ref) / np.maximum(1.0, np.abs(m_ref))
    assert err.max() <= tol_m, err.max()
    assert abs(loss.item() - L_ref) <= tol_m * L_ref
    assert np.abs(gg.cpu().numpy() - gg_ref).max() <= tol_g * np.abs(gg_ref).max()
    assert np.abs(ga.cpu().numpy() - ga_ref).max() <= tol_g * np.abs(ga_ref).max()
    assert torch.equal(gg, gg2) and torch.equal(ga, ga2)
    big = torch.empty(ws.numel() + 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(Exception, match="16-byte aligned"):
        soft.forward(syn, flt, g, a, workspace=big[8:])
    soft.close()
