"""Mixed-code batches in one persistent launch, and CUDA-graph capture of a decode.

A mixed batch ([[72,12,6]] T=6, gross T=12, [[288,12,18]] T=18 in a 1:2:1 mix,
interleaved at random) must decode every shot exactly as the single-code decoder
of its code does, and as the oracle's float32 mirror.
"""
import numpy as np
import pytest

from oracle.relay import RelayParams, relay_decode
from workloads import pack_bits, unpack_bits

from _cases import gamma_for, problem, shots

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2511_21660_gb300 import (QLDPC_MSG_FP16, RelayConfig, RelayDecoder,  # noqa: E402
                                    decode_grouped, decode_mixed)


def test_mixed_batch_matches_single_code_decoders():
    names = ["bb72_T6", "bb144_T12", "bb288_T18"]
    probs = [problem(n) for n in names]
    gams = [gamma_for(P, seed=2) for P in probs]
    cfg = RelayConfig(stop_after_solutions=5)
    decs = [RelayDecoder(P.row_ptr, P.col_idx, P.p, g, cfg) for P, g in zip(probs, gams)]
    rng = np.random.default_rng(3)
    counts = [400, 800, 400]
    code = rng.permutation(np.repeat(np.arange(3), counts)).astype(np.int32)
    sw = max(d.syndrome_words for d in decs)
    rows = np.zeros((code.size, sw), dtype=np.uint64)
    sigs = []
    for c, (P, n) in enumerate(zip(probs, counts)):
        F, s = shots(P, n, 40 + c)
        sigs.append(s)
        packed = pack_bits(s)
        rows[np.nonzero(code == c)[0], :packed.shape[1]] = packed
    code0 = code.copy()
    code[7] = 9                                        # not a code of the table
    cor, legs, conv, iters = decode_mixed(decs, torch.from_numpy(code).cuda(),
                                          torch.from_numpy(rows.view(np.int64)).cuda())
    torch.cuda.synchronize()
    cor, legs, conv, iters = (x.cpu().numpy() for x in (cor, legs, conv, iters))
    assert iters[7] == -1 and legs[7] == 0 and conv[7] == 0
    for c, (P, d, s) in enumerate(zip(probs, decs, sigs)):
        rows_c = np.nonzero(code0 == c)[0]             # batch rows of code c, in shot order
        live = rows_c != 7
        syn = torch.from_numpy(pack_bits(s).view(np.int64)).cuda()
        rc, rl, rv, ri = (x.cpu().numpy() for x in d.decode(syn))
        got = unpack_bits(cor[rows_c].view(np.uint64)[:, :d.correction_words], P.N)
        ref_c = unpack_bits(rc.view(np.uint64), P.N)
        assert (got[live] == ref_c[live]).all()
        assert (legs[rows_c][live] == rl[live]).all() and (conv[rows_c][live] == rv[live]).all()
        assert (iters[rows_c][live] == ri[live]).all()
        pick = np.arange(1, s.shape[0], 13)
        ref = relay_decode(P.row_ptr, P.col_idx, P.p, gams[c], s[pick],
                           RelayParams(stop_after_solutions=5), precision="f32")
        ok = live[pick]
        assert (got[pick][ok] == ref.corrections[ok]).all()
        assert (iters[rows_c][pick][ok] == ref.iters[ok]).all()
    for d in decs:
        d.close()


def test_decode_is_capturable_in_a_cuda_graph():
    P = problem("bb144_T12")
    F, s = shots(P, 3000, 8)
    gam = gamma_for(P, seed=8)
    dec = RelayDecoder(P.row_ptr, P.col_idx, P.p, gam, RelayConfig(stop_after_solutions=5))
    syn = torch.from_numpy(pack_bits(s).view(np.int64)).cuda()
    ref = [x.clone() for x in dec.decode(syn)]
    out = dec.outputs(syn.shape[0])
    for x in out:
        x.zero_()
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        dec.decode(syn, out=out, stream=stream)
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    for a, b in zip(out, ref):
        assert torch.equal(a, b)
    dec.close()


def _mixed_rows(probs, counts, seed):
    rng = np.random.default_rng(seed)
    code = rng.permutation(np.repeat(np.arange(len(probs)), counts)).astype(np.int32)
    sw = max((P.M + 63) // 64 for P in probs)
    rows = np.zeros((code.size, sw), dtype=np.uint64)
    for c, (P, n) in enumerate(zip(probs, counts)):
        F, s = shots(P, n, 60 + c)
        rows[np.nonzero(code == c)[0], :(P.M + 63) // 64] = pack_bits(s)
    return code, rows


def test_grouped_batch_equals_single_launch_and_per_code_decoders():
    names = ["bb72_T6", "bb144_T12", "bb288_T18"]
    probs = [problem(n) for n in names]
    gams = [gamma_for(P, seed=4) for P in probs]
    cfg = RelayConfig(stop_after_solutions=5)
    decs = [RelayDecoder(P.row_ptr, P.col_idx, P.p, g, cfg) for P, g in zip(probs, gams)]
    code, rows = _mixed_rows(probs, [500, 1000, 500], 5)
    code[11] = -3                                       # not a code of the table
    code_t = torch.from_numpy(code).cuda()
    rows_t = torch.from_numpy(rows.view(np.int64)).cuda()
    a = decode_mixed(decs, code_t, rows_t)
    b = decode_grouped(decs, code_t, rows_t)
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    assert b[3][11].item() == -1 and b[1][11].item() == 0
    # graph capture of the grouped call
    ws = torch.empty(4 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        out = decode_grouped(decs, code_t, rows_t, workspace=ws, stream=stream)
    graph.replay()
    torch.cuda.synchronize()
    for x, y in zip(out, b):
        assert torch.equal(x, y)
    for d in decs:
        d.close()


def test_grouped_batch_with_mixed_precisions():
    """Per-code decoders may differ in message precision: each shot equals its own
    decoder's single-code result."""
    names = ["bb72_T6", "bb144_T12"]
    probs = [problem(n) for n in names]
    gams = [gamma_for(P, seed=6) for P in probs]
    cfgs = [RelayConfig(stop_after_solutions=5),
            RelayConfig(stop_after_solutions=5, msg_precision=QLDPC_MSG_FP16)]
    decs = [RelayDecoder(P.row_ptr, P.col_idx, P.p, g, c) for P, g, c in zip(probs, gams, cfgs)]
    code, rows = _mixed_rows(probs, [300, 600], 7)
    cor, legs, conv, iters = decode_grouped(decs, torch.from_numpy(code).cuda(),
                                            torch.from_numpy(rows.view(np.int64)).cuda())
    torch.cuda.synchronize()
    cor, iters = cor.cpu().numpy(), iters.cpu().numpy()
    for c, (P, d) in enumerate(zip(probs, decs)):
        sel = np.nonzero(code == c)[0]
        syn = torch.from_numpy(np.ascontiguousarray(
            rows[sel, :(P.M + 63) // 64]).view(np.int64)).cuda()
        rc, rl, rv, ri = (x.cpu().numpy() for x in d.decode(syn))
        assert (cor[sel, :d.correction_words] == rc).all() and (iters[sel] == ri).all()
    for d in decs:
        d.close()
