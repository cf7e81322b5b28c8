"""The C ABI library loads, exports every declared entry point and rejects bad input.

These tests make no compute calls, so they run without a GPU.
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2511_21660_gb300 import build
    build.build()
    from paper_2511_21660_gb300 import qldpc
    return qldpc.load_library()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "qldpc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qldpc_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert "qldpc_create" in names and "qldpc_decode_batch" in names and "qldpc_destroy" in names
    for n in names:
        assert hasattr(lib, n), n
    from paper_2511_21660_gb300 import qldpc
    assert set(names) == set(qldpc.EXPORTED)


def test_status_strings(lib):
    from paper_2511_21660_gb300 import qldpc
    assert qldpc.status_string(0) == "ok"
    assert qldpc.status_string(-1) == "invalid argument"
    assert qldpc.status_string(-4).startswith("unsupported")
    assert qldpc.status_string(99) == "unknown status"


def _params(N, R=2, gamma=None, **kw):
    from paper_2511_21660_gb300 import qldpc
    g = np.full((R + 1, N), 0.125, dtype=np.float32) if gamma is None else gamma
    p = qldpc.qldpc_relay_params(R, 80, 60, 0, 1, 0, 0, 0, 0, 0.0, g.ctypes.data)
    for k, v in kw.items():
        setattr(p, k, v)
    return p, g


def _create(M, N, row_ptr, col_idx, priors, prm):
    from paper_2511_21660_gb300 import qldpc
    lib = qldpc.load_library()
    h = ctypes.c_void_p()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    pr = np.ascontiguousarray(priors, dtype=np.float64)
    rc = lib.qldpc_create(ctypes.byref(h), M, N, rp.ctypes.data, ci.ctypes.data, pr.ctypes.data,
                          ctypes.byref(prm), 0)
    return rc, h


def test_create_rejects_malformed_input(lib):
    from paper_2511_21660_gb300 import qldpc
    rp, ci, pr = [0, 2, 4], [0, 1, 1, 2], [0.1, 0.1, 0.1]
    prm, _g = _params(3)
    cases = [
        (2, 3, [1, 2, 4], ci, pr, prm),                 # row_ptr[0] != 0
        (2, 3, [0, 3, 2], ci, pr, prm),                 # decreasing row_ptr
        (2, 3, rp, [0, 3, 1, 2], pr, prm),              # column out of range
        (2, 3, rp, [1, 0, 1, 2], pr, prm),              # unsorted row
        (2, 3, rp, [0, 0, 1, 2], pr, prm),              # duplicate column
        (2, 3, rp, ci, [0.1, 0.0, 0.1], prm),           # p = 0
        (2, 3, rp, ci, [0.1, 1.0, 0.1], prm),           # p = 1
        (2, 3, rp, ci, [0.1, np.nan, 0.1], prm),        # NaN prior
        (0, 3, [0], [], pr, prm),                       # empty graph
    ]
    for M, N, r, c, p, prm_ in cases:
        rc, h = _create(M, N, r, c, p, prm_)
        assert rc == qldpc.QLDPC_ERR_INVALID_ARG, (r, c, p, rc)
        assert not h.value
        assert qldpc.last_error() != ""
    bad_gamma = np.full((3, 3), 0.125, dtype=np.float32)
    bad_gamma[1, 1] = np.inf
    for kw in ({"stop_after_solutions": 0}, {"iters_first": 0}, {"warm_start_mode": 2},
               {"msg_precision": 7}, {"legs_after_first": -1}, {"gamma_table": None}):
        prm_, _g2 = _params(3, **kw)
        assert _create(2, 3, rp, ci, pr, prm_)[0] == qldpc.QLDPC_ERR_INVALID_ARG, kw
    prm_, _g3 = _params(3, gamma=bad_gamma)
    assert _create(2, 3, rp, ci, pr, prm_)[0] == qldpc.QLDPC_ERR_INVALID_ARG
    prm_, _g4 = _params(3, msg_precision=1, llr_clip=1e6)
    assert _create(2, 3, rp, ci, pr, prm_)[0] == qldpc.QLDPC_ERR_INVALID_ARG


def test_decode_rejects_null_handle(lib):
    from paper_2511_21660_gb300 import qldpc
    assert lib.qldpc_decode_batch(None, None, 0, None, None, None, None, None) == \
        qldpc.QLDPC_ERR_INVALID_ARG
    assert lib.qldpc_decode_batch_host(None, None, 1, None, None, None, None) == \
        qldpc.QLDPC_ERR_INVALID_ARG
    lib.qldpc_destroy(None)   # ignored


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.mark.skipif(_has_gpu(), reason="checks the no-GPU error path")
def test_create_without_gpu_reports_cuda_error(lib):
    from paper_2511_21660_gb300 import qldpc
    prm, _g = _params(3)
    rc, h = _create(2, 3, [0, 2, 4], [0, 1, 1, 2], [0.1, 0.1, 0.1], prm)
    assert rc == qldpc.QLDPC_ERR_CUDA and not h.value
    assert "cudaGetDeviceCount" in qldpc.last_error()


def test_product_path_has_no_cpu_fallback():
    """The package never imports the oracle and fails loudly without its library."""
    import subprocess
    import sys
    code = ("import paper_2511_21660_gb300.qldpc as q\n"
            "try:\n    q.load_library('/nonexistent/libqldpc.so')\nexcept ImportError:\n"
            "    print('raised')\n")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT)
    assert "raised" in out.stdout, out.stderr
    pkg = os.path.join(ROOT, "paper_2511_21660_gb300")
    for dirpath, _d, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"(import|from)\s+oracle|oracle/|liboracle", src), f


def test_post_processor_and_grouped_entry_points_reject_bad_input(lib):
    from paper_2511_21660_gb300 import qldpc
    rp = np.ascontiguousarray([0, 2, 4], dtype=np.int32)
    ci = np.ascontiguousarray([0, 1, 1, 2], dtype=np.int32)
    pr = np.ascontiguousarray([0.1, 0.1, 0.1])
    h = ctypes.c_void_p()
    for bp, conf, rmax in ((-1, 4.0, 500), (25, float("nan"), 500), (25, 4.0, 0),
                           (25, 4.0, 1025)):
        prm = qldpc.qldpc_osd_params(bp, conf, rmax)
        rc = lib.qldpc_osd_create(ctypes.byref(h), 2, 3, rp.ctypes.data, ci.ctypes.data,
                                  pr.ctypes.data, ctypes.byref(prm), 0)
        assert rc == qldpc.QLDPC_ERR_INVALID_ARG and not h.value, (bp, conf, rmax)
    for bp, acc, era, nc, nf in ((-1, -1.0, 1.0, 10, 10), (25, 1.0, -1.0, 10, 10),
                                 (25, -1.0, float("inf"), 10, 10), (25, -1.0, 1.0, 0, 10),
                                 (25, -1.0, 1.0, 4097, 10), (25, -1.0, 1.0, 10, 0),
                                 (25, -1.0, 1.0, 10, 513)):
        prm = qldpc.qldpc_cluster_params(bp, acc, era, nc, nf)
        rc = lib.qldpc_cluster_create(ctypes.byref(h), 2, 3, rp.ctypes.data, ci.ctypes.data,
                                      pr.ctypes.data, ctypes.byref(prm), 0)
        assert rc == qldpc.QLDPC_ERR_INVALID_ARG and not h.value, (bp, acc, era, nc, nf)
    assert lib.qldpc_osd_decode_batch(None, None, 1, None, None, None, None, None) == \
        qldpc.QLDPC_ERR_INVALID_ARG
    assert lib.qldpc_cluster_decode_batch(None, None, 1, None, None, None, None, None) == \
        qldpc.QLDPC_ERR_INVALID_ARG
    assert lib.qldpc_decode_batch_grouped(None, 0, None, None, 1, 1, None, 1, None, None,
                                          None, None, 0, None) == qldpc.QLDPC_ERR_INVALID_ARG
    assert qldpc.qldpc_grouped_workspace_bytes(3, 100) == 256 + 4 * 3 * 100
    assert qldpc.qldpc_grouped_workspace_bytes(0, 100) == 0
    lib.qldpc_osd_destroy(None)
    lib.qldpc_cluster_destroy(None)
