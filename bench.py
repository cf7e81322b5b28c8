"""Benchmark: Relay-BP syndromes/s on one GB300, gross code [[144,12,12]], 12 noisy rounds.

Workload: the phenomenological detector model of the gross code (936 detectors x 2736
faults, 7344 edges), 12 noisy rounds plus one perfect round, i.i.d. faults with
p = 0.003, 10^5 syndromes per step, Relay with the App. A.3 leg schedule
(T_1 = 80, T_r = 60, R = 300, gamma_0 = 0.125, gamma ~ U[-0.24, 0.66]) and S = 5
solutions, float32 messages.  A step decodes the whole batch with one call.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  --impl reference times the CPU oracle (FP64, all
host cores) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import BB144, gamma_table, pack_bits, phenomenological_dem, sample_faults, \
    syndromes_of  # noqa: E402

WORKLOAD = "gross [[144,12,12]] phenomenological T=12 + 1 perfect round, 936x2736, p=0.003"
SHOTS = 100_000
SEED = 1
S_SOLUTIONS = 5
METRIC = "Relay-BP syndromes/s on 1 GB300 (gross code, 12 rds) and % of roofline"


def make_inputs(n_shots: int, seed: int, first_shot: int = 0, device=None):
    """The benchmark workload: gross T=12 detector model, shots first_shot.. of the stream.

    With a CUDA device the same seeded stream is sampled there (bit-identical to the
    host sampler) and the syndromes are returned on the host.
    """
    P = phenomenological_dem(BB144, 12, 0.003)
    if device is not None:
        from workloads.torch_sampling import sample_faults_t, syndromes_t
        F = sample_faults_t(P.p, seed, n_shots, first_shot=first_shot, device=device)
        sig = syndromes_t(P.H, F).cpu().numpy()
        del F
    else:
        F = sample_faults(P.p, seed, n_shots, first_shot=first_shot)
        sig = syndromes_of(P.row_ptr, P.col_idx, F)
    gam = gamma_table(P.N, 300, 0.125, -0.24, 0.66, seed)
    return P, sig, gam


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard_first_shot(rank: int, shots_per_rank: int) -> int:
    """Weak scaling: rank r decodes shots [r*S, (r+1)*S) of the counter-based shot stream."""
    return rank * shots_per_rank


def reduce_max_ms(ms: float, ws: int, device) -> float:
    """Slowest rank's step time (the only collective of the benchmark; none on the data path)."""
    if ws == 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(ws: int, shots_per_rank: int, ms: float) -> float:
    """Whole-job syndromes/s: every rank's shots over the slowest rank's step time."""
    return ws * shots_per_rank / (ms / 1e3)


# ---------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = os.path.join("/tmp", f"qldpc_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return self
        # the timed region starts once the sampler is writing (at most 3 s of waiting)
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
            self.fh.flush()
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)
        self.skip = self._lines()
        return self

    def _lines(self):
        try:
            with open(self.path) as f:
                return sum(1 for _ in f)
        except OSError:
            return 0

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for k, line in enumerate(open(self.path)):
            parts = [x.strip() for x in line.split(",")]
            if k >= getattr(self, "skip", 0) and len(parts) >= 9:
                rows.append(parts)   # samples taken after the timed region started
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------------------
# the reference arm: the CPU oracle on a bounded sample
# ---------------------------------------------------------------------------------------
ORACLE_TIMED_BUILD = "gcc -O3 -ffp-contract=off -fno-fast-math -fopenmp (oracle/build.py, f64_O3)"


def cpu_oracle_rate(P, sig, gam, target_s: float = 8.0, precision: str = "f64_O3"):
    """The FP64 oracle (the -O3 build of the same source, same values as the parity
    build) timed on this host's cores twice: OpenMP over shots on every core, and on one
    thread.  Each leg decodes a prefix of the benchmark's syndromes sized, from a short
    calibration run, for about target_s seconds."""
    from oracle import build as oracle_build
    from oracle.relay import RelayParams, relay_decode
    oracle_build.build()
    prm = RelayParams(stop_after_solutions=S_SOLUTIONS)
    cores = os.cpu_count() or 1

    def leg(nthreads, cal):
        cal = min(cal, sig.shape[0])
        t0 = time.perf_counter()
        relay_decode(P.row_ptr, P.col_idx, P.p, gam, sig[:cal], prm, precision=precision,
                     nthreads=nthreads)
        dt = time.perf_counter() - t0
        n = int(min(sig.shape[0], max(cal, cal * target_s / max(dt, 1e-6))))
        t0 = time.perf_counter()
        r = relay_decode(P.row_ptr, P.col_idx, P.p, gam, sig[:n], prm, precision=precision,
                         nthreads=nthreads)
        dt = time.perf_counter() - t0
        return n, dt, float(P.E * r.iters.sum() / dt)

    n, dt, eu = leg(cores, 2000)
    n1, dt1, eu1 = leg(1, 200)
    return {"value": n / dt, "unit": "syndromes/s", "cores": cores, "kind": "oracle",
            "sample": f"first {n} of the {sig.shape[0]} syndromes, FP64 oracle, OpenMP over "
                      f"shots on {cores} host threads, {dt:.1f} s",
            "edge_updates_per_s": eu, "build": ORACLE_TIMED_BUILD,
            "single_thread": {"value": n1 / dt1, "unit": "syndromes/s", "cores": 1,
                              "sample": f"first {n1} syndromes on one thread, {dt1:.1f} s",
                              "edge_updates_per_s": eu1}}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    P, sig, gam = make_inputs(SHOTS, SEED)
    from oracle import build as oracle_build
    from oracle.relay import RelayParams, relay_decode
    oracle_build.build()
    cores = os.cpu_count() or 1
    prm = RelayParams(stop_after_solutions=S_SOLUTIONS)
    # a bounded sample per step so that warm-up + steps end within a few minutes
    per_step = int(os.environ.get("QLDPC_REF_SHOTS", "2000"))
    times = []
    off = 0
    for k in range(args.warmup + args.steps):
        s = sig[off:off + per_step]
        off = (off + per_step) % (SHOTS - per_step)
        t0 = time.perf_counter()
        relay_decode(P.row_ptr, P.col_idx, P.p, gam, s, prm, precision="f64_O3",
                     nthreads=cores)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = per_step / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "syndromes/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "shots_per_step": per_step, "S": S_SOLUTIONS,
                       "parallelism": "OpenMP over shots", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "syndromes/s", "cores": cores,
                             "kind": "oracle", "build": ORACLE_TIMED_BUILD,
                             "sample": f"{per_step} syndromes per step of the same workload"},
            "e2e": {"value": value, "unit": "syndromes/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------
KERNEL_SOURCES = ("relay_device.cuh", "relay_fused.cu", "qldpc_internal.h", "qldpc_api.cu")


def kernel_source_sha1() -> str:
    """sha1 (12 hex digits) of the fused decode kernel's sources and of the host code that
    lays out its graph (edge placement, shared-memory layout), in that order."""
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2511_21660_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


PROFILE_FP32 = "fused_decode_gross_T12.md"
PROFILE_FP16 = "fused_decode_gross_T12_fp16.md"


def profile_field(name: str, profile: str = PROFILE_FP32):
    """A value recorded in a committed ncu summary of the decode kernel (float32 by
    default), or None when the summary is absent or was taken on a different kernel
    source."""
    path = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(path):
        return None
    same, val = False, None
    for line in open(path):
        if line.startswith("| kernel source sha1"):
            same = line.split("|")[2].strip() == kernel_source_sha1()
        elif line.startswith(f"| {name} |"):
            val = float(line.split("|")[2])
    return val if same else None


def traffic_per_launch(args, profile: str = PROFILE_FP32):
    """DRAM bytes (read + write) of one decode launch, from the committed ncu summary.

    profiles/fused_decode_gross_T12.md records dram__bytes_read.sum and
    dram__bytes_write.sum for a 20,000-shot launch of the same kernel; DRAM traffic
    (syndromes in, corrections out, graph and gamma rows) grows with the shot count,
    so it is scaled to the benchmark's shots.  None when the summary is absent or
    was taken on a different kernel source (the sha1 of KERNEL_SOURCES is recorded in the
    summary).
    """
    path = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(path):
        return None
    sha = kernel_source_sha1()
    rd = wr = shots = None
    same_source = False
    for line in open(path):
        if line.startswith("| kernel source sha1"):
            same_source = line.split("|")[2].strip() == sha
        elif line.startswith("| dram__bytes_read.sum"):
            rd = float(line.split("|")[2])
        elif line.startswith("| dram__bytes_write.sum"):
            wr = float(line.split("|")[2])
        elif line.startswith("| shots per launch"):
            shots = float(line.split("|")[2])
    if not same_source or rd is None or wr is None or not shots:
        return None
    return (rd + wr) * SHOTS / shots


def sm_max_mhz() -> float:
    """Maximum SM clock measured on this machine (MEASURED_PEAKS.json), else the nominal
    2070 MHz."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"])
    except (OSError, ValueError, KeyError, TypeError):
        return 2070.0


# Algorithmic work of one DMem-BP iteration of one shot (paper Sec. 2.3), per edge and
# per fault: every edge's message is read and written by the check pass and by the fault
# pass (4 accesses of the message size), every fault reads lambda(0), gamma and Lambda
# and writes Lambda (16 B).  13 lane operations per edge: check node |nu|, two-smallest
# update (3), sign parity, magnitude select, sign apply; fault node marginal add,
# excluded-sum add, two clamp operations, the memory rule's share; the syndrome XOR.
OPS_PER_EDGE_ITER = 13


def smem_bytes_per_shot_iter(E: int, N: int, msg: str) -> int:
    return (4 * (2 if msg == "fp16" else 4)) * E + 16 * N


def decode_roofline(E, N, iters, ms, msg, sms, mhz, traffic=None):
    """Roofline of a decode launch.  Shared memory moves 128 B/clock/SM and the SM
    issues 128 lane-instructions/clock (4 schedulers x 32 lanes), at the maximum SM
    clock: the smem roof is that bandwidth over the algorithmic bytes per edge-update,
    the issue roof that rate over 13 operations per edge-update.  `frac` divides the
    measured edge-updates/s by the lower roof (the smem roof for both message sizes),
    i.e. algorithmic bytes/s over the shared-memory bandwidth."""
    per_iter = smem_bytes_per_shot_iter(E, N, msg)
    eu = E * iters / (ms / 1e3)
    smem_peak = 128 * sms * mhz * 1e6                        # B/s
    issue_peak = 128 * sms * mhz * 1e6                       # lane-instructions/s
    smem_roof = smem_peak / (per_iter / E)
    issue_roof = issue_peak / OPS_PER_EDGE_ITER
    roof = min(smem_roof, issue_roof)
    achieved = per_iter * iters / (ms / 1e3) / 1e9
    ops = OPS_PER_EDGE_ITER * E * iters / (ms / 1e3)
    # 9 of the 13 operations (two-smallest 3, sign parity, magnitude select, sign apply,
    # two clamp ops, syndrome XOR) run on the ALU pipe, which issues 64 lanes/clock/SM
    alu_ceiling = OPS_PER_EDGE_ITER / 9 * 64 * sms * mhz * 1e6
    return {"bound": "smem" if smem_roof <= issue_roof else "alu",
            "achieved": achieved, "peak": smem_peak / 1e9, "unit": "GB/s",
            "frac": eu / roof, "traffic": traffic,
            "peak_kind": "derived: 128 B/clk/SM x %d SMs x %.0f MHz (max SM clock)" % (sms, mhz),
            "algorithmic": f"{per_iter} B per shot-iteration ({msg} messages: "
                           f"{per_iter / E:.2f} B per edge-update) x {iters} iterations",
            "edge_updates_per_s": eu, "smem_roof_edge_updates_per_s": smem_roof,
            "issue_roof_edge_updates_per_s": issue_roof,
            "issue_view": {"achieved_Tops": ops / 1e12, "peak_Tops": issue_peak / 1e12,
                           "frac": ops / issue_peak,
                           "basis": f"{OPS_PER_EDGE_ITER} algorithmic lane operations per "
                                    "edge-update against 128 lanes/clk/SM"},
            "alu_pipe_ceiling": {"peak_Tops": alu_ceiling / 1e12, "frac": ops / alu_ceiling,
                                 "basis": "9 of 13 ops per edge-update on the ALU pipe at "
                                          "64 lanes/clk/SM"}}


def timed_decode(dec, syn, out, steps, warmup, stream, flush):
    """Per-step CUDA-event times (ms) of the decode call, L2 flushed between steps."""
    import torch
    for _ in range(warmup):
        dec.decode(syn, out=out, stream=stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev[k][0].record(stream)
        dec.decode(syn, out=out, stream=stream)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def run_decode_only(args):
    """Profiling driver: decode args.shots syndromes with one kernel configuration."""
    import torch

    from paper_2511_21660_gb300 import (QLDPC_KERNEL_BASELINE, QLDPC_KERNEL_FUSED,
                                        QLDPC_MSG_FP16, QLDPC_MSG_FP32, RelayConfig, RelayDecoder)
    dev = torch.device("cuda", 0)
    P, sig, gam = make_inputs(args.shots, SEED, device=dev)
    syn = torch.from_numpy(pack_bits(sig).view(np.int64)).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    cfg = RelayConfig(stop_after_solutions=args.solutions,
                      msg_precision=QLDPC_MSG_FP16 if args.msg == "fp16" else QLDPC_MSG_FP32,
                      kernel=QLDPC_KERNEL_BASELINE if args.kernel == "baseline"
                      else QLDPC_KERNEL_FUSED, block_threads=args.block_threads)
    dec = RelayDecoder(P.row_ptr, P.col_idx, P.p, gam, cfg)
    out = dec.outputs(args.shots)
    times = timed_decode(dec, syn, out, args.steps, args.warmup, stream, flush)
    iters = int(out[3].sum().item())
    legs = int(out[1].sum().item())
    ms = sum(times) / len(times)
    print(json.dumps({"mode": "decode-only", "kernel": args.kernel, "msg": args.msg,
                      "S": args.solutions,
                      "shots": args.shots, "ms_per_step": ms,
                      "syndromes_per_s": args.shots / (ms / 1e3),
                      "iterations": iters, "legs": legs, "block_threads": dec.info.block_threads,
                      "blocks_per_sm": dec.info.blocks_per_sm, "grid": dec.info.grid_blocks,
                      "smem_bytes": dec.info.smem_bytes}), flush=True)
    dec.close()


def timed_post(post, syn, base_cor, skip, stream, flush, steps=3, warmup=3):
    """CUDA-event ms of a post-processor launch (corrections reset before each)."""
    import torch
    cor = torch.empty_like(base_cor)
    n = syn.shape[0]
    status = torch.empty(n, dtype=torch.int32, device=syn.device)
    extra = torch.empty(n, dtype=torch.int32, device=syn.device)
    times = []
    for k in range(warmup + steps):
        cor.copy_(base_cor)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            post.decode(syn, cor, skip, status, extra, stream=stream)
            e1.record(stream)
        torch.cuda.synchronize()
        if k >= warmup:
            times.append(e0.elapsed_time(e1))
    return sum(times) / len(times), cor, status, extra


def post_processing_variants(args, dev, stream, flush, block_threads=0):
    """First Relay leg + filtered-OSD (paper Sec. 5) and first Relay leg + BP + cluster
    decoding (Sec. 2.5, Sec. 6), the paper's two post-processed decoders (Sec. 7.1),
    against full Relay on the gross 12-round model at p = 0.02, where the first leg
    leaves about 1% of the shots unconverged: each post-processor's time on those
    shots, its outcomes, and the three decoders' logical error rates on the same 10^5
    shots."""
    import torch

    from paper_2511_21660_gb300 import (QLDPC_CLUSTER_DECODED, QLDPC_OSD_NO_SOLUTION,
                                        QLDPC_OSD_SOLVED, QLDPC_OSD_TOO_MANY, ClusterDecoder,
                                        FilteredOSD, RelayConfig, RelayDecoder)
    from paper_2511_21660_gb300 import latency_tail
    from workloads.torch_sampling import pack_bits_t, sample_faults_t, syndromes_t
    p, n, conf, rmax = 0.02, SHOTS, 8.0, 500
    P = phenomenological_dem(BB144, 12, p)
    F = sample_faults_t(P.p, 2, n, device=dev)
    syn = pack_bits_t(syndromes_t(P.H, F))
    gam = gamma_table(P.N, 300, 0.125, -0.24, 0.66, 2)
    first = RelayDecoder(P.row_ptr, P.col_idx, P.p, gam[:1],
                         RelayConfig(legs_after_first=0, stop_after_solutions=1,
                                     block_threads=block_threads), device=dev.index)
    # full Relay: the tail continuation on or off, whichever is faster on this batch
    from paper_2511_21660_gb300.autotune import tune
    rcfg = RelayConfig(stop_after_solutions=S_SOLUTIONS, block_threads=block_threads)
    (_, tail), tail_ms = tune(P.row_ptr, P.col_idx, P.p, gam, rcfg, syn, repeats=1, cache=None,
                              block_sizes=(block_threads,), tail_options=(0, -1))
    rcfg.tail_cut_iters = tail
    relay = RelayDecoder(P.row_ptr, P.col_idx, P.p, gam, rcfg, device=dev.index)
    osd = FilteredOSD(P.row_ptr, P.col_idx, P.p, 25, conf, rmax, device=dev.index)
    accept, erase = -0.5, 4.5
    cluster = ClusterDecoder(P.row_ptr, P.col_idx, P.p, 25, accept, erase, 4096, 512,
                             device=dev.index)
    fo = first.outputs(n)
    ms_first = sum(timed_decode(first, syn, fo, 3, 3, stream, flush)) / 3
    ro = relay.outputs(n)
    ms_relay = sum(timed_decode(relay, syn, ro, 3, 2, stream, flush)) / 3
    it_relay = ro[3].to(torch.int64)
    # the paper's gross cutoff (Sec. 7.2): T_max = 6000 FPGA cycles = 3000 iterations at
    # 2 cycles per iteration; a shot without a solution by then fails
    cut = RelayDecoder(P.row_ptr, P.col_idx, P.p, gam,
                       RelayConfig(stop_after_solutions=S_SOLUTIONS, max_total_iters=3000,
                                   block_threads=block_threads), device=dev.index)
    co = cut.outputs(n)
    ms_cut = sum(timed_decode(cut, syn, co, 3, 2, stream, flush)) / 3
    skip = fo[2]
    ms_osd, cor, status, ncand = timed_post(osd, syn, fo[0], skip, stream, flush)
    ms_cl, cor_cl, st_cl, steps_cl = timed_post(cluster, syn, fo[0], skip, stream, flush)
    A = torch.from_numpy(P.A.astype(np.float32)).to(dev)
    shifts = torch.arange(64, dtype=torch.int64, device=dev)

    def logical(c):
        bits = ((c[:, :, None] >> shifts) & 1).reshape(n, -1)[:, :P.N].to(torch.uint8)
        return ((F ^ bits).to(torch.float32) @ A.T).to(torch.int64).remainder(2).any(1)
    fail_first = (logical(cor) | ((skip == 0) & (status != QLDPC_OSD_SOLVED))).sum().item()
    fail_relay = (logical(ro[0]) | (ro[2] == 0)).sum().item()
    fail_cut = (logical(co[0]) | (co[2] == 0)).sum().item()
    fail_cl = (logical(cor_cl) | ((skip == 0) & (st_cl != QLDPC_CLUSTER_DECODED))).sum().item()
    todo = int((skip == 0).sum().item())
    st = status[skip == 0]
    stc = st_cl[skip == 0]
    out = {"workload": "gross [[144,12,12]] phenomenological T=12, p=0.02, 10^5 shots",
           "osd": f"25 plain BP iterations, Lambda_confident={conf}, |R|_max={rmax}",
           "first_leg_ms": ms_first, "first_leg_failures": todo,
           "osd_ms": ms_osd, "osd_shots_per_s": todo / (ms_osd / 1e3) if todo else None,
           # the BP share of the launch: its 25 float32 iterations per post-processed shot
           # against the shared-memory roof (the ranking, the sort and the elimination are
           # not counted, so this is a lower bound on the launch's use of the SM)
           "osd_bp_roofline": decode_roofline(P.E, P.N, 25 * todo, ms_osd, "fp32",
                                              first.info.num_sms, sm_max_mhz()),
           "osd_status": {"solved": int((st == QLDPC_OSD_SOLVED).sum().item()),
                          "too_many": int((st == QLDPC_OSD_TOO_MANY).sum().item()),
                          "no_solution": int((st == QLDPC_OSD_NO_SOLUTION).sum().item())},
           "mean_candidates": float(ncand[skip == 0].float().mean().item()) if todo else 0.0,
           "ler_first_leg_plus_osd": fail_first / n, "ler_relay_S5": fail_relay / n,
           "relay_ms": ms_relay,
           "relay_tail_continuation": {"cut_iterations": relay.info.tail_cut_iters,
                                       "resume_block_threads": relay.info.tail_block_threads,
                                       "ms_by_block_and_cut": tail_ms},
           "relay_iterations_per_shot": {"mean": float(it_relay.double().mean().item()),
                                         "p99": float(torch.quantile(it_relay.double(), 0.99)),
                                         "max": int(it_relay.max().item()),
                                         "shots_at_the_18080_bound":
                                             int((it_relay >= 80 + 300 * 60).sum().item())},
           # the same decode's roofline (the hard regime: many iterations per leg end)
           "relay_roofline": decode_roofline(P.E, P.N, int(it_relay.sum().item()), ms_relay,
                                             "fp32", relay.info.num_sms, sm_max_mhz()),
           "ler_relay_S5_cutoff_3000_iterations": fail_cut / n,
           # the same decode under the gross cutoff: a shot gets at most 3000 iterations
           "relay_cutoff_3000_ms": ms_cut,
           # Sec. 2.2 / 7.2 conditions on full Relay's measured iteration counts at this
           # noise rate, in FPGA cycles at 2 per iteration (T_ref 500, T_gen 1000, 6000)
           "relay_latency_tail": {k: v for k, v in latency_tail.report(
               ro[3].cpu().numpy(), t_ref=500, t_gen=1000, t_max=6000, C=10,
               cycles_per_iter=2).items()
               if k in ("eps", "L", "holds", "max_code_blocks", "slowdown_bound")},
           "cluster": {"decoder": f"25 plain BP iterations, Lambda_accept={accept}, "
                                  f"Lambda_erase={erase}, clusters <= 4096, "
                                  f"interior faults <= 512",
                       "ms": ms_cl,
                       "shots_per_s": todo / (ms_cl / 1e3) if todo else None,
                       # the BP share, as for filtered-OSD (growth steps and validity
                       # tests not counted)
                       "bp_roofline": decode_roofline(P.E, P.N, 25 * todo, ms_cl, "fp32",
                                                      first.info.num_sms, sm_max_mhz()),
                       "decoded": int((stc == QLDPC_CLUSTER_DECODED).sum().item()),
                       "failed": int((stc < 0).sum().item()),
                       "mean_growth_steps": float(steps_cl[skip == 0].float().mean().item())
                       if todo else 0.0,
                       "ler_first_leg_plus_cluster": fail_cl / n}}
    if args.cpu_baseline and todo:
        from oracle.osd import OSDParams, bp_llrs, filtered_osd
        idx = torch.nonzero(skip == 0).flatten()[:40].cpu().numpy()
        sig = syndromes_t(P.H, F[torch.from_numpy(idx).to(dev)]).cpu().numpy()
        t0 = time.perf_counter()
        L = bp_llrs(P.row_ptr, P.col_idx, P.p, sig, 25)
        t_bp = time.perf_counter() - t0
        for b in range(sig.shape[0]):
            filtered_osd(P.H, sig[b], L[b], OSDParams(25, conf, rmax))
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": sig.shape[0] / dt, "unit": "post-processed shots/s",
                               "cores": os.cpu_count(), "kind": "oracle",
                               "sample": f"the first {sig.shape[0]} unconverged shots"}
    if args.cpu_baseline and todo:
        from oracle.cluster import ClusterParams, bp_uf
        t0 = time.perf_counter()
        for b in range(sig.shape[0]):
            bp_uf(P.H, sig[b], L[b], ClusterParams(25, accept, erase, 512, 4096))
        dt = time.perf_counter() - t0 + t_bp
        out["cluster"]["cpu_baseline"] = {
            "value": sig.shape[0] / dt, "unit": "post-processed shots/s",
            "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"the first {sig.shape[0]} unconverged shots"}
    for d in (first, relay, cut, osd, cluster):
        d.close()
    return out


def mixed_batch_variant(args, dev, stream, flush):
    """The uneven-batch workload: 2^18 shots of the [[72,12,6]] T=6, gross T=12 and
    [[288,12,18]] T=18 detector models (p = 0.003) in a 1:2:1 mix, interleaved at random,
    decoded by one persistent launch replayed from a CUDA graph; the block size is chosen
    by timing the compiled shapes that hold the largest code.  Also times each code's
    shots decoded on their own (with its autotuned block size) for comparison."""
    import torch

    from paper_2511_21660_gb300 import RelayConfig, RelayDecoder, decode_mixed
    from paper_2511_21660_gb300.autotune import CANDIDATES, tune_block_threads
    from workloads import BB72, BB288
    from workloads.torch_sampling import pack_bits_t, sample_faults_t, syndromes_t
    codes = [(BB72, 6, (-0.24, 0.66)), (BB144, 12, (-0.24, 0.66)), (BB288, 18, (-0.161, 0.815))]
    counts = [65536, 131072, 65536]
    B = sum(counts)
    probs = [phenomenological_dem(c, T, 0.003) for c, T, _ in codes]
    gams = [gamma_table(P.N, 300, 0.125, lo, hi, 3) for P, (_, _, (lo, hi)) in zip(probs, codes)]
    stride = max((P.M + 63) // 64 for P in probs)
    rng = np.random.default_rng(3)
    code = rng.permutation(np.repeat(np.arange(3), counts)).astype(np.int32)
    code_t = torch.from_numpy(code).to(dev)
    rows = torch.zeros((B, stride), dtype=torch.int64, device=dev)
    per_code = []
    for c, (P, n) in enumerate(zip(probs, counts)):
        syn_c = pack_bits_t(syndromes_t(P.H, sample_faults_t(P.p, 30 + c, n, device=dev)))
        per_code.append(syn_c)
        idx = torch.from_numpy(np.nonzero(code == c)[0]).to(dev)
        rows[idx, :syn_c.shape[1]] = syn_c
    cfg = RelayConfig(stop_after_solutions=S_SOLUTIONS)
    timings = {}
    best = None
    for bt in CANDIDATES:
        try:
            big = RelayDecoder(probs[2].row_ptr, probs[2].col_idx, probs[2].p, gams[2],
                               RelayConfig(stop_after_solutions=S_SOLUTIONS, block_threads=bt),
                               device=dev.index)
        except Exception:
            continue
        if big.info.block_threads != bt:
            big.close()
            continue
        decs = [RelayDecoder(P.row_ptr, P.col_idx, P.p, g, cfg, device=dev.index)
                for P, g in zip(probs[:2], gams[:2])] + [big]
        out = decode_mixed(decs, code_t, rows, stream=stream)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            out = decode_mixed(decs, code_t, rows, stream=stream)
        times = []
        for k in range(8):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                graph.replay()
                e1.record(stream)
            torch.cuda.synchronize()
            if k >= 3:
                times.append(e0.elapsed_time(e1))
        timings[bt] = sum(times) / len(times)
        if best is None or timings[bt] < timings[best[0]]:
            best = (bt, out[3].clone(), out[2].clone())
        for d in decs:
            d.close()
    bt, iters, conv = best
    ms = timings[bt]
    # the same batch decoded per code in one call (each code's own autotuned shape)
    from paper_2511_21660_gb300 import decode_grouped
    from paper_2511_21660_gb300.qldpc import qldpc_grouped_workspace_bytes
    gdecs = []
    for P, g in zip(probs, gams):
        tb, _ = tune_block_threads(P.row_ptr, P.col_idx, P.p, g, cfg,
                                   per_code[len(gdecs)][:20000], cache=None)
        gdecs.append(RelayDecoder(P.row_ptr, P.col_idx, P.p, g,
                                  RelayConfig(stop_after_solutions=S_SOLUTIONS, block_threads=tb),
                                  device=dev.index))
    ws = torch.empty(qldpc_grouped_workspace_bytes(3, B), dtype=torch.uint8, device=dev)
    gout = decode_grouped(gdecs, code_t, rows, workspace=ws, stream=stream)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        gout = decode_grouped(gdecs, code_t, rows, workspace=ws, stream=stream)
    gtimes = []
    for k in range(8):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            graph.replay()
            e1.record(stream)
        torch.cuda.synchronize()
        if k >= 3:
            gtimes.append(e0.elapsed_time(e1))
    gms = sum(gtimes) / len(gtimes)
    grouped_same = bool(torch.equal(gout[3], iters) and torch.equal(gout[2], conv))
    for d in gdecs:
        d.close()
    alone = {}
    for c, (P, g, syn_c) in enumerate(zip(probs, gams, per_code)):
        tb, _ = tune_block_threads(P.row_ptr, P.col_idx, P.p, g, cfg, syn_c[:20000], cache=None)
        d = RelayDecoder(P.row_ptr, P.col_idx, P.p, g,
                         RelayConfig(stop_after_solutions=S_SOLUTIONS, block_threads=tb),
                         device=dev.index)
        o = d.outputs(syn_c.shape[0])
        t = timed_decode(d, syn_c, o, 3, 2, stream, flush)
        alone[f"{P.meta['code']}_T{[6, 12, 18][c]}"] = {"shots": int(syn_c.shape[0]),
                                                        "ms": sum(t) / len(t),
                                                        "block_threads": tb}
        d.close()
    it = iters.cpu().numpy()
    return {"workload": "[[72,12,6]] T=6 : gross T=12 : [[288,12,18]] T=18 = 1:2:1, "
                        "2^18 shots interleaved, p=0.003, S=5",
            "value": B / (ms / 1e3), "unit": "syndromes/s", "ms_per_launch": ms,
            "launch": "one persistent launch, CUDA-graph replay",
            "block_threads": bt, "tuning_ms": {str(k): round(v, 3) for k, v in timings.items()},
            "converged_fraction": float(conv.float().mean().item()),
            "iterations_per_shot": {f"code{c}": float(it[code == c].mean()) for c in range(3)},
            "grouped": {"value": B / (gms / 1e3), "unit": "syndromes/s", "ms_per_call": gms,
                        "launch": "one call: device partition by code, then one persistent "
                                  "launch per code with its own block shape, CUDA-graph replay",
                        "identical_to_single_launch": grouped_same},
            "codes_decoded_separately": alone,
            "separate_total_ms": sum(v["ms"] for v in alone.values())}


# Special-function (MUFU) operations per edge per iteration of the float32 soft kernels:
# forward tanh(nu/2) = 1 - 2/(1 + e^nu) (exponential, reciprocal) and
# atanh(P) = log((1+P)/(1-P))/2 (reciprocal, logarithm).  The adjoint's recompute stores
# each iteration's tanh(nu/2) rows, so a reverse step evaluates only atanh (2) and one
# reciprocal for 1/(1 - P^2); the recompute runs the forward (4) of every iteration but
# the last of each checkpoint segment other than the final one, and for those the tanh
# rows alone (2).
SOFT_XU_OPS_FORWARD = 4
SOFT_XU_OPS_REVERSE = 3
SOFT_XU_OPS_TANH = 2


def soft_backward_ops_per_edge_iter(T, K):
    """Special-function operations per edge per iteration of the adjoint, averaged over
    the T iterations (checkpoints every K): 3 T reverse, 4 (T - ceil(T/K) + 1) recomputed
    iterations and 2 (ceil(T/K) - 1) tanh passes."""
    nck = (T + K - 1) // K
    return (SOFT_XU_OPS_REVERSE * T + SOFT_XU_OPS_FORWARD * (T - nck + 1)
            + SOFT_XU_OPS_TANH * (nck - 1)) / T


def soft_roofline(edge_iters, ms, ops_per_edge_iter, sms):
    """The soft kernels' special-function roof: one warp-instruction per clock per SM on
    the XU pipe (32 results/clock/SM; ncu's XU utilisation of the forward, 10.9% at 24.8M
    XU warp-instructions over 1.50M active cycles per SM, gives the same peak) at the
    maximum SM clock."""
    mhz = sm_max_mhz()
    peak = 32 * sms * mhz * 1e6
    ops = ops_per_edge_iter * edge_iters / (ms / 1e3)
    return {"bound": "xu", "achieved": ops / 1e12, "peak": peak / 1e12, "unit": "Tops/s",
            "frac": ops / peak,
            "peak_kind": "derived: 32 special-function results/clk/SM x %d SMs x %.0f MHz"
                         % (sms, mhz),
            "algorithmic": f"{ops_per_edge_iter:.3g} special-function operations per edge per "
                           f"iteration x {edge_iters} edge-iterations"}


def soft_dmem_variant(args, dev, stream, flush, B=4096):
    """One training step of the differentiable leg: unrolled soft DMem-BP (25 iterations,
    trainable gamma_j and alpha_t, BCE loss, checkpoints every 5 iterations, float32) on
    a batch of B (4096) gross T=12 shots at p = 0.003: forward and adjoint times."""
    import torch

    from paper_2511_21660_gb300 import SoftDMem
    from workloads.torch_sampling import pack_bits_t, sample_faults_t, syndromes_t
    P = phenomenological_dem(BB144, 12, 0.003)
    T = 25
    F = sample_faults_t(P.p, 20, B, device=dev)
    syn = pack_bits_t(syndromes_t(P.H, F))
    faults = pack_bits_t(F)
    gamma = torch.full((P.N,), 0.125, dtype=torch.float32, device=dev)
    alpha = torch.ones(T, dtype=torch.float32, device=dev)

    def time_step(K):
        soft = SoftDMem(P.row_ptr, P.col_idx, P.p, T, K, torch.float32, device=dev.index)
        ws = soft.workspace(B)
        fwd, bwd = [], []
        for k in range(8):
            flush.zero_()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            with torch.cuda.stream(stream):
                e[0].record(stream)
                loss, _, _ = soft.forward(syn, faults, gamma, alpha, ws, stream=stream)
                e[1].record(stream)
                gg, ga = soft.backward(syn, faults, gamma, alpha, ws, stream=stream)
                e[2].record(stream)
            torch.cuda.synchronize()
            if k >= 3:
                fwd.append(e[0].elapsed_time(e[1]))
                bwd.append(e[1].elapsed_time(e[2]))
        nbytes = ws.numel()
        soft.close()
        return sum(fwd) / len(fwd), sum(bwd) / len(bwd), loss, gg, nbytes

    # every state stored (no recompute in the adjoint): 25 checkpoints per shot
    f1_ms, b1_ms, _, _, ws1 = time_step(1)
    f_ms, b_ms, loss, gg, ws5 = time_step(5)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    out = {"workload": f"gross T=12 p=0.003, batch {B}, 25 iterations, checkpoint every 5, "
                       "float32, gamma_j (2736) and alpha_t (25) trainable",
           "forward_ms": f_ms, "backward_ms": b_ms,
           "step_shots_per_s": B / ((f_ms + b_ms) / 1e3),
           "forward_edge_iterations_per_s": B * T * P.E / (f_ms / 1e3),
           "roofline": soft_roofline(P.E * T * B, f_ms, SOFT_XU_OPS_FORWARD, sms),
           "backward_roofline": soft_roofline(P.E * T * B, b_ms,
                                              soft_backward_ops_per_edge_iter(T, 5), sms),
           "loss": float(loss.item()),
           "grad_gamma_norm": float(gg.norm().item()),
           "workspace_bytes": ws5,
           # the same step with every state a checkpoint: the forward stores 25 states per
           # shot, the adjoint recomputes nothing
           "checkpoint_every_1": {"forward_ms": f1_ms, "backward_ms": b1_ms,
                                  "step_shots_per_s": B / ((f1_ms + b1_ms) / 1e3),
                                  "workspace_bytes": ws1,
                                  "backward_roofline": soft_roofline(
                                      P.E * T * B, b1_ms, soft_backward_ops_per_edge_iter(T, 1),
                                      sms)}}
    if args.cpu_baseline:
        from oracle.soft import soft_dmem
        n = 64
        sig = syndromes_t(P.H, F[:n]).cpu().numpy()
        Fh = F[:n].cpu().numpy()
        t0 = time.perf_counter()
        soft_dmem(P.row_ptr, P.col_idx, P.p, np.full(P.N, 0.125), np.ones(T), sig, Fh)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": n / dt, "unit": "shots/s (forward + gradient)",
                               "cores": os.cpu_count(), "kind": "oracle",
                               "sample": f"{n} shots, FP64, full trajectory stored"}
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2511_21660_gb300 import (QLDPC_KERNEL_BASELINE, QLDPC_KERNEL_FUSED,
                                        QLDPC_MSG_FP16, QLDPC_MSG_FP32, RelayConfig, RelayDecoder)
    from paper_2511_21660_gb300 import latency_tail
    from paper_2511_21660_gb300 import qldpc as Q

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    # weak scaling: each rank decodes its own 10^5 shots (shard `rank` of the shot stream)
    P, sig, gam = make_inputs(SHOTS, SEED, first_shot=shard_first_shot(rank, SHOTS), device=dev)
    packed = pack_bits(sig)
    syn = torch.from_numpy(packed.view(np.int64)).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB of L2
    stream = torch.cuda.Stream(device=dev)

    # block shape chosen by timing the compiled candidates on a 20,000-shot sample
    from paper_2511_21660_gb300.autotune import tune_block_threads
    cfg = RelayConfig(stop_after_solutions=S_SOLUTIONS, msg_precision=QLDPC_MSG_FP32,
                      kernel=QLDPC_KERNEL_FUSED)
    bt, tuning = tune_block_threads(P.row_ptr, P.col_idx, P.p, gam, cfg, syn[:50000], cache=None)
    cfg.block_threads = bt
    dec = RelayDecoder(P.row_ptr, P.col_idx, P.p, gam, cfg, device=local)
    out = dec.outputs(SHOTS)

    # the headline measurement
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        times = timed_decode(dec, syn, out, args.steps, args.warmup, stream, flush)
        t_wall = time.perf_counter() - t_wall
    torch.cuda.synchronize()
    ms = reduce_max_ms(sum(times) / len(times), ws, dev)
    if ws > 1:
        dist.barrier()
    iters = out[3].cpu().numpy().astype(np.int64)
    conv = out[2].cpu().numpy()
    total_iters = int(iters.sum())
    value = aggregate_rate(ws, SHOTS, ms)

    if rank != 0:
        dec.close()
        if ws > 1:
            dist.destroy_process_group()
        return

    # roofline of the decode kernel (shared-memory roof of the algorithmic message and
    # fault-state bytes, the lower of the two roofs; issue and ALU-pipe views beside it)
    sms = dec.info.num_sms
    mhz = sm_max_mhz()
    roofline = decode_roofline(P.E, P.N, total_iters, ms, "fp32", sms, mhz,
                               traffic=traffic_per_launch(args))
    roofline["issue_slots_used_frac"] = (lambda v: v / 100.0 if v is not None else None)(
        profile_field("smsp__issue_active.avg.pct_of_peak_sustained_active"))

    # variants measured in the same run: FP16 messages and the plain baseline kernel
    variants = {}
    cfg16 = RelayConfig(stop_after_solutions=S_SOLUTIONS, msg_precision=QLDPC_MSG_FP16,
                        kernel=QLDPC_KERNEL_FUSED)
    cfg16.block_threads, tuning16 = tune_block_threads(P.row_ptr, P.col_idx, P.p, gam, cfg16,
                                                       syn[:50000], cache=None)
    # S = 1: stop at the first solution (the workload's variant), the headline's shape
    cfg_s1 = RelayConfig(stop_after_solutions=1, msg_precision=QLDPC_MSG_FP32,
                         kernel=QLDPC_KERNEL_FUSED, block_threads=dec.info.block_threads)
    for name, vcfg in (("fused_fp16", cfg16),
                       ("baseline_fp32", RelayConfig(stop_after_solutions=S_SOLUTIONS,
                                                     msg_precision=QLDPC_MSG_FP32,
                                                     kernel=QLDPC_KERNEL_BASELINE)),
                       ("fused_fp32_S1", cfg_s1)):
        vd = RelayDecoder(P.row_ptr, P.col_idx, P.p, gam, vcfg, device=local)
        vo = vd.outputs(SHOTS)
        vt = timed_decode(vd, syn, vo, max(3, min(args.steps, 5)), 3, stream, flush)
        vms = sum(vt) / len(vt)
        same = bool(torch.equal(vo[0], out[0]) and torch.equal(vo[3], out[3]))
        variants[name] = {"value": SHOTS / (vms / 1e3), "unit": "syndromes/s",
                          "ms_per_step": vms, "block_threads": vd.info.block_threads,
                          "blocks_per_sm": vd.info.blocks_per_sm,
                          "identical_to_fp32_fused": same}
        if name == "fused_fp16":
            it16 = int(vo[3].to(torch.int64).sum().item())
            r16 = decode_roofline(P.E, P.N, it16, vms, "fp16", sms, mhz,
                                  traffic=traffic_per_launch(args, PROFILE_FP16))
            r16["issue_slots_used_frac"] = (lambda v: v / 100.0 if v is not None else None)(
                profile_field("smsp__issue_active.avg.pct_of_peak_sustained_active",
                              PROFILE_FP16))
            variants[name]["roofline"] = r16
            variants[name]["speedup_vs_fused_fp32"] = ms / vms
        if name == "fused_fp32_S1":
            it1 = vo[3].to(torch.int64)
            variants[name]["identical_to_fp32_fused"] = None  # a different stopping rule
            variants[name]["iterations_per_shot"] = float(it1.double().mean().item())
            variants[name]["legs_per_shot"] = float(vo[1].double().mean().item())
            variants[name]["roofline"] = decode_roofline(P.E, P.N, int(it1.sum().item()), vms,
                                                         "fp32", sms, mhz)
        vd.close()
    variants["fused_fp32_speedup_vs_baseline"] = (value / ws) / variants["baseline_fp32"]["value"]

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    sw, cw = dec.syndrome_words, dec.correction_words
    h_syn = torch.from_numpy(packed.view(np.int64)).pin_memory()
    h_cor = torch.empty((SHOTS, cw), dtype=torch.int64).pin_memory()
    h_legs = torch.empty(SHOTS, dtype=torch.int32).pin_memory()
    h_conv = torch.empty(SHOTS, dtype=torch.uint8).pin_memory()
    h_it = torch.empty(SHOTS, dtype=torch.int32).pin_memory()

    def host_call():
        Q.qldpc_decode_batch_host(dec.handle, ctypes.c_void_p(h_syn.data_ptr()), SHOTS,
                                  ctypes.c_void_p(h_cor.data_ptr()),
                                  ctypes.c_void_p(h_legs.data_ptr()),
                                  ctypes.c_void_p(h_conv.data_ptr()),
                                  ctypes.c_void_p(h_it.data_ptr()))
    for _ in range(max(1, args.warmup)):
        host_call()
    e2e_t = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        host_call()
        e2e_t.append(time.perf_counter() - t0)
    e2e = {"value": SHOTS / (sum(e2e_t) / len(e2e_t)), "unit": "syndromes/s",
           "h2d_bytes_per_step": int(SHOTS * sw * 8),
           "d2h_bytes_per_step": int(SHOTS * (cw * 8 + 4 + 1 + 4))}
    assert np.array_equal(h_cor.numpy(), out[0].cpu().numpy()), "host path differs"

    # the gross code's autotuned block size serves the p = 0.02 decodes too
    variants["first_leg_then_post_processing"] = post_processing_variants(
        args, dev, stream, flush, block_threads=dec.info.block_threads)
    variants["mixed_batch"] = mixed_batch_variant(args, dev, stream, flush)
    variants["soft_dmem_training_step"] = soft_dmem_variant(args, dev, stream, flush)
    cpu = cpu_oracle_rate(P, sig, gam) if args.cpu_baseline else None
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": "syndromes/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "shots_per_step": SHOTS, "S": S_SOLUTIONS,
                   "relay": "T1=80 T2=60 R=300 gamma0=0.125 gamma~U[-0.24,0.66]",
                   "messages": "float32", "kernel": "fused persistent",
                   "block_threads": dec.info.block_threads,
                   "blocks_per_sm": dec.info.blocks_per_sm, "grid": dec.info.grid_blocks,
                   "autotune_ms_50k_shots": {str(k): round(v, 3) for k, v in tuning.items()},
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "l2": "flushed between steps (256 MB write)"},
        "edge_updates_per_s": ws * P.E * total_iters / (ms / 1e3),
        "iterations_per_shot": {"mean": total_iters / SHOTS, "max": int(iters.max()),
                                "p99": float(np.percentile(iters, 99))},
        # Sec. 7.2's latency-tail analysis applied to the measured iteration counts, in
        # FPGA cycles at 2 cycles per iteration: T_ref 500, T_gen 1000, gross cutoff 6000
        "latency_tail": {k: v for k, v in latency_tail.report(
            iters, t_ref=500, t_gen=1000, t_max=6000, C=10, cycles_per_iter=2).items()
            if k in ("eps", "L", "holds", "max_code_blocks", "slowdown_bound")},
        "converged_fraction": float(conv.mean()),
        # context only: the paper's FPGA cost-model figures for Relay (other hardware,
        # circuit-level noise; Sec. 7.1-7.2, App. A.3), not a target for this metric
        "paper_context": {"device": "AMD VU19P FPGA cost model", "cycles_per_iteration": 2,
                          "clock_ns": 12, "iteration_ns": 24,
                          "gross_cutoff_cycles": 6000, "gross_ler_at_cutoff": 4e-7,
                          "tail_fraction_beyond_500_cycles_gross": 5e-5,
                          "single_instance_syndromes_per_s_upper_bound": 1.7e5},
        "roofline": roofline,
        # the same kernel in the hard regime (p = 0.02, full Relay, S = 5, 10^5 shots)
        "roofline_hard_regime": {
            "workload": "gross T=12 phenomenological p=0.02, 10^5 shots, S=5, float32",
            **variants["first_leg_then_post_processing"]["relay_roofline"]},
        "variants": variants, "e2e": e2e, "cpu_baseline": cpu,
        "clocks": clocks, "gpu_launches": args.steps,
        "wall_s_timed_region": t_wall,
    }
    print(json.dumps(line), flush=True)
    dec.close()
    if ws > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--shots", type=int, default=SHOTS,
                    help="syndromes per step (profiling runs use fewer)")
    ap.add_argument("--only-decode", action="store_true",
                    help="time the decode kernel only (no variants, e2e or CPU baseline)")
    ap.add_argument("--kernel", choices=["fused", "baseline"], default="fused")
    ap.add_argument("--msg", choices=["fp32", "fp16"], default="fp32")
    ap.add_argument("--block-threads", type=int, default=0)
    ap.add_argument("--solutions", type=int, default=S_SOLUTIONS,
                    help="S of a decode-only run")
    ap.add_argument("--only-post", action="store_true",
                    help="profiling driver: the p = 0.02 first-leg, full-Relay, filtered-OSD and "
                         "cluster-decoder comparison only")
    ap.add_argument("--only-soft", type=int, default=0, metavar="B",
                    help="profiling driver: one soft DMem-BP training-step measurement on a "
                         "batch of B gross shots (no decode, e2e or CPU baseline)")
    args = ap.parse_args()
    if args.only_soft:
        import torch
        dev = torch.device("cuda", 0)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        args.cpu_baseline = False
        r = soft_dmem_variant(args, dev, torch.cuda.Stream(dev), flush, B=args.only_soft)
        print(json.dumps({"mode": "soft-only", **r}))
        return
    if args.only_post:
        import torch
        dev = torch.device("cuda", 0)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        args.cpu_baseline = False
        r = post_processing_variants(args, dev, torch.cuda.Stream(dev), flush,
                                     block_threads=args.block_threads)
        print(json.dumps({"mode": "post-only", **r}))
        return
    if (args.shots != SHOTS or args.kernel != "fused" or args.msg != "fp32"
            or args.block_threads or args.solutions != S_SOLUTIONS):
        args.only_decode = True
    if args.impl == "reference":
        run_reference(args)
    elif args.only_decode:
        run_decode_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
