"""The autotuner's cache key (CPU) and a tuning run with a cache hit (GPU)."""
import numpy as np
import pytest

from paper_2511_21660_gb300 import RelayConfig
from paper_2511_21660_gb300.autotune import problem_key

from _cases import gamma_for, problem


def _base():
    P = problem("bb72_T6")
    return P, gamma_for(P, R=300, seed=1)


def test_key_separates_problems_of_equal_size():
    P, gam = _base()
    cfg = RelayConfig(stop_after_solutions=5)
    k0 = problem_key(P.row_ptr, P.col_idx, P.p, gam, cfg, "GB300")
    assert k0 == problem_key(P.row_ptr.copy(), P.col_idx.copy(), P.p.copy(), gam.copy(), cfg,
                             "GB300")
    ci = P.col_idx.copy()
    i = int(np.argmax(np.diff(P.row_ptr)))            # a row with room to move an edge
    cols = set(ci[P.row_ptr[i]:P.row_ptr[i + 1]])
    free = next(j for j in range(P.N) if j not in cols and j > ci[P.row_ptr[i + 1] - 1])
    ci[P.row_ptr[i + 1] - 1] = free                   # same sizes, another graph
    p2 = P.p.copy()
    p2[0] *= 1.5
    g2 = gam.copy()
    g2[3, 7] += 0.01
    others = [problem_key(P.row_ptr, ci, P.p, gam, cfg, "GB300"),
              problem_key(P.row_ptr, P.col_idx, p2, gam, cfg, "GB300"),
              problem_key(P.row_ptr, P.col_idx, P.p, g2, cfg, "GB300"),
              problem_key(P.row_ptr, P.col_idx, P.p, gam, RelayConfig(stop_after_solutions=1),
                          "GB300"),
              problem_key(P.row_ptr, P.col_idx, P.p, gam,
                          RelayConfig(stop_after_solutions=5, max_total_iters=100), "GB300"),
              problem_key(P.row_ptr, P.col_idx, P.p, gam, cfg, "another GPU")]
    assert len(set(others + [k0])) == len(others) + 1


@pytest.mark.gpu
def test_tune_times_the_candidates_and_reuses_the_cache(tmp_path, monkeypatch):
    torch = pytest.importorskip("torch")
    from paper_2511_21660_gb300 import autotune
    from workloads import pack_bits

    from _cases import shots
    P, gam = _base()
    F, sig = shots(P, 3000, 4)
    syn = torch.from_numpy(pack_bits(sig).view(np.int64)).cuda()
    cfg = RelayConfig(stop_after_solutions=5)
    cache = str(tmp_path / "tuning.json")
    (bt, tail), ms = autotune.tune(P.row_ptr, P.col_idx, P.p, gam, cfg, syn, repeats=1,
                                   cache=cache, block_sizes=(256, 384), tail_options=(0, -1))
    assert set(ms) == {"256/0", "256/-1", "384/0", "384/-1"}
    assert ms[f"{bt}/{tail}"] == min(ms.values())

    class NoDecoder:
        def __init__(self, *a, **k):
            raise AssertionError("a cache hit must not build decoders")
    monkeypatch.setattr(autotune, "RelayDecoder", NoDecoder)
    again = autotune.tune(P.row_ptr, P.col_idx, P.p, gam, cfg, syn, repeats=1, cache=cache,
                          block_sizes=(256, 384), tail_options=(0, -1))
    assert again == ((bt, tail), ms)
    # another gamma table of the same size is a miss (and so builds decoders)
    g2 = gam.copy()
    g2[1, 0] += 0.01
    with pytest.raises(AssertionError):
        autotune.tune(P.row_ptr, P.col_idx, P.p, g2, cfg, syn, repeats=1, cache=cache,
                      block_sizes=(256, 384), tail_options=(0, -1))
    monkeypatch.undo()
    assert autotune.tune_block_threads(P.row_ptr, P.col_idx, P.p, gam,
                                       RelayConfig(stop_after_solutions=5, tail_cut_iters=-1),
                                       syn, repeats=1, cache=None)[0] in autotune.CANDIDATES
