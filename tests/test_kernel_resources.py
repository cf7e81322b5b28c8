"""Register budget of the fused decode kernel's launch shapes (CPU only: reads the
`-Xptxas -v` report that the build keeps beside each object).

The persistent kernel keeps 3 x VPT per-fault values in registers; at the shapes the
autotuner picks for the gross code (384 threads x 8 faults x 3 blocks per SM, 56
registers) a few bytes of local-memory spill inside the iteration loop cost several
per cent, and small source changes can bring one in.  The float32 shapes below must
compile without spills.
"""
import os
import re

import pytest

from paper_2511_21660_gb300 import build as lib_build

SPILL_FREE_F32 = [(384, 8, 3), (512, 6, 2), (1024, 8, 1), (512, 16, 1)]


def ptxas_report(unit):
    lib_build.build()
    path = os.path.join(lib_build.BUILD, unit + ".ptxas.txt")
    if not os.path.exists(path):
        pytest.skip("no ptxas report (library built by another route)")
    return open(path).read()


def fused_resources(report):
    """{(threads, faults per thread, blocks per SM): (registers, spill store bytes,
    spill load bytes)} of the fused_decode entry points in one ptxas report."""
    out, cur = {}, None
    for line in report.splitlines():
        m = re.search(r"(?:Compiling entry function|Function properties for) '?(\S+?)'?$", line)
        if m:
            cur = m.group(1)
            continue
        if cur is None or "fused_decode" not in cur or "multi" in cur:
            continue
        t = re.search(r"fused_decodeI\w+?Li(\d+)ELi(\d+)ELi(\d+)E", cur)
        if not t:
            continue
        key = tuple(int(x) for x in t.groups())
        regs, st, ld = out.get(key, (None, 0, 0))
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m:
            st, ld = int(m.group(1)), int(m.group(2))
        m = re.search(r"Used (\d+) registers", line)
        if m:
            regs = int(m.group(1))
        out[key] = (regs, st, ld)
    return out


def test_report_parser_reads_every_shape():
    res = fused_resources(ptxas_report("relay_fused_f32_8_4"))
    for shape in SPILL_FREE_F32[:3]:
        assert shape in res and res[shape][0] is not None, (shape, sorted(res))


@pytest.mark.parametrize("unit,shapes", [("relay_fused_f32_8_4", SPILL_FREE_F32[:3]),
                                         ("relay_fused_f32_16_8", SPILL_FREE_F32[3:])])
def test_float32_autotuned_shapes_do_not_spill(unit, shapes):
    res = fused_resources(ptxas_report(unit))
    for shape in shapes:
        regs, st, ld = res[shape]
        assert st == 0 and ld == 0, f"{unit} {shape}: {regs} registers, spill {st}/{ld} bytes"
