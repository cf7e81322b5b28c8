"""Pick the fused kernel's launch configuration for a decoding problem by timing the
compiled candidates on a sample batch, with a JSON cache keyed by GPU, problem and options.

The library compiles several (threads per block, faults per thread, resident blocks)
shapes, and its tail continuation (a second launch that finishes the few very long
shots) pays when those shots fit about one wave of that launch; which is fastest
depends on the code, the message precision, the noise and the Relay schedule, so it is
measured rather than guessed.  The cache key holds a digest of the graph, the priors and
the gamma table, so two problems of equal size do not share an entry.
"""
from __future__ import annotations

import dataclasses
import hashlib
import json
import os

import numpy as np

from .qldpc import QldpcError, RelayConfig, RelayDecoder

CANDIDATES = (256, 384, 512, 640, 768, 1024)
TAIL_OPTIONS = (0, -1)   # the library default (continuation after T_1 + 8 T_r), off
CACHE = os.path.join(os.path.expanduser("~"), ".cache", "qldpc", "tuning.json")


def problem_key(row_ptr, col_idx, priors, gamma_table, cfg: RelayConfig, device_name: str,
                sample_digest: str = "") -> str:
    """Cache key: device, sizes, a digest of H (CSR), the priors and the gamma table, the
    options that change the work (precision, schedule, budget, clip, warm mode) and the
    sample's digest."""
    h = hashlib.sha1()
    for a, dt in ((row_ptr, np.int32), (col_idx, np.int32), (priors, np.float64),
                  (gamma_table, np.float32)):
        h.update(np.ascontiguousarray(a, dtype=dt).tobytes())
    M, N, E = len(row_ptr) - 1, len(priors), int(row_ptr[-1])
    return (f"{device_name.replace('|', ' ')}|M{M}|N{N}|E{E}|{h.hexdigest()[:20]}"
            f"|msg{cfg.msg_precision}|S{cfg.stop_after_solutions}|R{cfg.legs_after_first}"
            f"|T{cfg.iters_first},{cfg.iters_later}|budget{cfg.max_total_iters}"
            f"|warm{cfg.warm_start_mode}|clip{cfg.llr_clip}|{sample_digest}")


def _sample_digest(syndromes) -> str:
    import torch
    s = syndromes.detach()
    return f"B{s.shape[0]}:{int(torch.sum(s.to(torch.float64) * 1e-9).item() * 1e6)}"


def tune(row_ptr, col_idx, priors, gamma_table, config: RelayConfig, syndromes,
         repeats: int = 3, cache: str | None = CACHE, block_sizes=CANDIDATES,
         tail_options=TAIL_OPTIONS):
    """Time every compiled block size with each tail setting on `syndromes` (int64 CUDA
    tensor [B, words]).  Returns ((block_threads, tail_cut_iters), {"bt/tail": ms}).
    Shapes the graph does not fit are skipped (block size 0: the library's choice); the
    answer is cached per key."""
    import torch
    key = problem_key(row_ptr, col_idx, priors, gamma_table, config,
                      torch.cuda.get_device_name(), _sample_digest(syndromes)) + \
        f"|bt{','.join(map(str, block_sizes))}|tail{','.join(map(str, tail_options))}"
    if cache and os.path.exists(cache):
        try:
            hit = json.load(open(cache)).get(key)
            if hit:
                return (int(hit["best"][0]), int(hit["best"][1])), dict(hit["ms"])
        except (OSError, ValueError, KeyError, TypeError):
            pass
    timings = {}
    for bt in block_sizes:
        for tail in tail_options:
            cfg = dataclasses.replace(config, block_threads=bt, tail_cut_iters=tail)
            try:
                dec = RelayDecoder(row_ptr, col_idx, priors, gamma_table, cfg)
            except QldpcError:
                continue
            if bt and dec.info.block_threads != bt:  # 0: the library's own choice
                dec.close()
                continue
            out = dec.outputs(syndromes.shape[0])
            dec.decode(syndromes, out=out)
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record()
            for _ in range(repeats):
                dec.decode(syndromes, out=out)
            ev[1].record()
            torch.cuda.synchronize()
            timings[f"{bt}/{tail}"] = ev[0].elapsed_time(ev[1]) / repeats
            dec.close()
    if not timings:
        raise RuntimeError("no compiled block shape fits this problem")
    best_key = min(timings, key=timings.get)
    best = tuple(int(x) for x in best_key.split("/"))
    if cache:
        try:
            os.makedirs(os.path.dirname(cache), exist_ok=True)
            data = json.load(open(cache)) if os.path.exists(cache) else {}
            data[key] = {"best": list(best), "ms": timings}
            json.dump(data, open(cache, "w"), indent=1)
        except (OSError, ValueError):
            pass
    return best, timings


def tune_block_threads(row_ptr, col_idx, priors, gamma_table, config: RelayConfig,
                       syndromes, repeats: int = 3, cache: str | None = CACHE):
    """The block size alone (the config's tail setting kept).  Returns (best
    block_threads, {block_threads: ms})."""
    (bt, _), timings = tune(row_ptr, col_idx, priors, gamma_table, config, syndromes,
                            repeats=repeats, cache=cache,
                            tail_options=(config.tail_cut_iters,))
    return bt, {int(k.split("/")[0]): v for k, v in timings.items()}
