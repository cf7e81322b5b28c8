"""Pick the fused kernel's block shape for a decoding problem by timing the compiled
candidates on a sample batch, with a JSON cache keyed by GPU, problem and options.

The library compiles several (threads per block, faults per thread, resident blocks)
shapes; which is fastest depends on the code size, the message precision and the
Relay schedule, so it is measured rather than guessed.
"""
from __future__ import annotations

import dataclasses
import json
import os

from .qldpc import QldpcError, RelayConfig, RelayDecoder

CANDIDATES = (256, 384, 512, 640, 768, 1024)
CACHE = os.path.join(os.path.expanduser("~"), ".cache", "qldpc", "tuning.json")


def _key(M, N, E, cfg: RelayConfig) -> str:
    import torch
    name = torch.cuda.get_device_name().replace("|", " ")
    return (f"{name}|M{M}|N{N}|E{E}|msg{cfg.msg_precision}|S{cfg.stop_after_solutions}"
            f"|R{cfg.legs_after_first}|T{cfg.iters_first},{cfg.iters_later}")


def tune_block_threads(row_ptr, col_idx, priors, gamma_table, config: RelayConfig,
                       syndromes, repeats: int = 3, cache: str | None = CACHE):
    """Time every compiled block size on `syndromes` (int64 CUDA tensor [B, words]).

    Returns (best block_threads, {block_threads: ms}).  Shapes the graph does not fit
    are skipped.  The answer is cached per (GPU, problem size, options).
    """
    import torch
    E = int(row_ptr[-1])
    M, N = len(row_ptr) - 1, len(priors)
    key = _key(M, N, E, config)
    if cache and os.path.exists(cache):
        try:
            hit = json.load(open(cache)).get(key)
            if hit:
                return int(hit["best"]), {int(k): v for k, v in hit["ms"].items()}
        except (OSError, ValueError):
            pass
    timings = {}
    for bt in CANDIDATES:
        cfg = dataclasses.replace(config, block_threads=bt)
        try:
            dec = RelayDecoder(row_ptr, col_idx, priors, gamma_table, cfg)
        except QldpcError:
            continue
        if dec.info.block_threads != bt:
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
        timings[bt] = ev[0].elapsed_time(ev[1]) / repeats
        dec.close()
    if not timings:
        raise RuntimeError("no compiled block shape fits this problem")
    best = min(timings, key=timings.get)
    if cache:
        try:
            os.makedirs(os.path.dirname(cache), exist_ok=True)
            data = json.load(open(cache)) if os.path.exists(cache) else {}
            data[key] = {"best": best, "ms": timings}
            json.dump(data, open(cache, "w"), indent=1)
        except (OSError, ValueError):
            pass
    return best, timings
