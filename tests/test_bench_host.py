"""Host logic of the benchmark that its JSON line depends on (CPU only): the clock record
taken during the timed region, and the fields read from the committed ncu summary, which
must go null as soon as the kernel's sources differ from the ones the summary was taken on.
"""
import hashlib
import os

import pytest

import bench


class _Running:
    """Stands in for the nvidia-smi process (summary() only checks that one existed)."""


def _sampler(tmp_path, lines, skip):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    s.proc = _Running()
    s.skip = skip
    return s


def _row(mhz, max_mhz=2070, hw="Not Active", sw_pc="Not Active", thermal="Not Active"):
    return f"0, {mhz}, {max_mhz}, 900.0, 0x0, {hw}, {thermal}, Not Active, {sw_pc}"


def test_clock_summary_uses_samples_of_the_timed_region_only(tmp_path):
    # the first two lines predate the timed region; one idle sample is ignored as unloaded
    lines = [_row(345, hw="Active"), _row(345)] + [_row(2070)] * 5 + [_row(510)] + [_row(2055)]
    s = _sampler(tmp_path, lines, skip=2)
    out = s.summary()
    assert out["samples"] == 7
    assert out["sm_max_mhz"] == 2070.0
    assert out["sm_mhz"] == 2070.0           # median of the loaded samples
    assert out["reasons"] == []              # hw_slowdown was active before the region only
    assert not os.path.exists(s.path)


def test_clock_summary_reports_throttle_reasons(tmp_path):
    lines = [_row(1900, hw="Active"), _row(2070, sw_pc="Active"), _row(2070, thermal="Active")]
    out = _sampler(tmp_path, lines, skip=0).summary()
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap"]


def test_clock_summary_without_samples(tmp_path):
    out = _sampler(tmp_path, [_row(2070)], skip=1).summary()
    assert out["sm_mhz"] is None and out["reasons"] == ["no samples"]


def _fake_tree(root, shots, rd, wr, issue):
    csrc = root / "paper_2511_21660_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for k, name in enumerate(bench.KERNEL_SOURCES):
        (csrc / name).write_text(f"// source {k}\n")
    h = hashlib.sha1()
    for name in bench.KERNEL_SOURCES:
        h.update((csrc / name).read_bytes())
    (root / "profiles").mkdir()
    (root / "profiles" / "fused_decode_gross_T12.md").write_text(
        "| metric | value | unit |\n|---|---|---|\n"
        f"| kernel source sha1 (sources) | {h.hexdigest()[:12]} | |\n"
        f"| shots per launch | {shots} | shots |\n"
        f"| dram__bytes_read.sum | {rd} | byte |\n"
        f"| dram__bytes_write.sum | {wr} | byte |\n"
        f"| smsp__issue_active.avg.pct_of_peak_sustained_active | {issue} | % |\n")
    return csrc


def test_profile_fields_follow_the_kernel_source_hash(tmp_path, monkeypatch):
    csrc = _fake_tree(tmp_path, 20000, 2_600_000, 4000, 75.5)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_field("smsp__issue_active.avg.pct_of_peak_sustained_active") == 75.5
    # DRAM bytes scale from the summary's 20,000 shots to the benchmark's launch
    assert bench.traffic_per_launch(None) == pytest.approx(2_604_000 * bench.SHOTS / 20000)
    (csrc / bench.KERNEL_SOURCES[-1]).write_text("// changed\n")
    assert bench.profile_field("smsp__issue_active.avg.pct_of_peak_sustained_active") is None
    assert bench.traffic_per_launch(None) is None


def test_profile_fields_absent_summary(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_field("anything") is None
    assert bench.traffic_per_launch(None) is None


def _run_reference(rank, tmp_path):
    import json
    import subprocess
    import sys
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
               QLDPC_REF_SHOTS="40")
    r = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl",
                        "reference", "--steps", "1", "--warmup", "0", "--gpus", "2"],
                       capture_output=True, text=True, env=env, cwd=str(tmp_path), timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [json.loads(line) for line in r.stdout.splitlines() if line.startswith("{")]


def test_reference_arm_prints_one_line_on_rank_0(tmp_path):
    lines = _run_reference(0, tmp_path)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["unit"] == "syndromes/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "syndromes/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["n_gpus"] == 2


def test_reference_arm_other_ranks_exit_without_work(tmp_path):
    assert _run_reference(1, tmp_path) == []


def test_decode_roofline_follows_the_shared_memory_and_issue_roofs():
    """Gross T=12 (E = 7344, N = 2736), 561,398 iterations in 7.718 ms on 152 SMs at
    2070 MHz: 161,280 B per shot-iteration in float32 (16 B per edge, 16 B per fault), so
    the smem roof is 40.27 TB/s / 21.96 B = 1.834e12 edge-updates/s, below the issue roof
    of 40.27e12 / 13 = 3.098e12; binary16 moves 102,528 B and its smem roof is 2.885e12."""
    r = bench.decode_roofline(7344, 2736, 561398, 7.718, "fp32", 152, 2070.0)
    assert bench.smem_bytes_per_shot_iter(7344, 2736, "fp32") == 161280
    assert bench.smem_bytes_per_shot_iter(7344, 2736, "fp16") == 102528
    assert r["bound"] == "smem" and r["unit"] == "GB/s"
    assert r["peak"] == pytest.approx(40273.92)
    assert r["smem_roof_edge_updates_per_s"] == pytest.approx(40.27392e12 / (161280 / 7344))
    assert r["issue_roof_edge_updates_per_s"] == pytest.approx(40.27392e12 / 13)
    eu = 7344 * 561398 / 7.718e-3
    assert r["edge_updates_per_s"] == pytest.approx(eu)
    assert r["frac"] == pytest.approx(eu / r["smem_roof_edge_updates_per_s"])
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert 0.28 < r["frac"] < 0.30
    assert r["issue_view"]["frac"] == pytest.approx(13 * eu / 40.27392e12)
    h = bench.decode_roofline(7344, 2736, 561515, 7.42, "fp16", 152, 2070.0)
    assert h["bound"] == "smem" and h["smem_roof_edge_updates_per_s"] == pytest.approx(
        40.27392e12 / (102528 / 7344))
    assert h["frac"] == pytest.approx(h["achieved"] / h["peak"])


def test_cpu_baseline_reports_all_cores_and_one_thread():
    P, sig, gam = bench.make_inputs(400, 1)
    r = bench.cpu_oracle_rate(P, sig, gam, target_s=0.05)
    assert r["kind"] == "oracle" and r["cores"] == (os.cpu_count() or 1) and r["value"] > 0
    assert "-O3" in r["build"] and "-ffp-contract=off" in r["build"]
    one = r["single_thread"]
    assert one["cores"] == 1 and one["value"] > 0 and one["edge_updates_per_s"] > 0


def test_soft_roofline_counts_special_function_operations():
    """4 (forward) special-function operations per edge-iteration against 32 results per
    clock per SM: batch 4096, E = 7344, 25 iterations in 2.78 ms.  The adjoint with
    checkpoints every 5 iterations: 3 per reverse step (the recompute keeps the tanh
    values), 4 for each of the 21 recomputed iterations (25 less the last of the first
    four segments) and 2 for the tanh rows of each of those four last iterations."""
    ei = 7344 * 25 * 4096
    r = bench.soft_roofline(ei, 2.78, bench.SOFT_XU_OPS_FORWARD, 152)
    peak = 32 * 152 * bench.sm_max_mhz() * 1e6
    assert r["bound"] == "xu" and r["peak"] == pytest.approx(peak / 1e12)
    assert r["frac"] == pytest.approx(4 * ei / 2.78e-3 / peak)
    assert bench.soft_backward_ops_per_edge_iter(25, 5) == pytest.approx((3 * 25 + 4 * 21 + 2 * 4) / 25)
    assert bench.soft_backward_ops_per_edge_iter(25, 25) == pytest.approx(7)
    assert bench.soft_backward_ops_per_edge_iter(25, 1) == pytest.approx(3 + 4 / 25 + 2 * 24 / 25)
