"""Latency-tail conditions (paper Sec. 2.2 equations, Sec. 7.2 numbers)."""
import json
import math
import os

import numpy as np
import pytest

from paper_2511_21660_gb300 import latency_tail as lt

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_layers_and_requirement_follow_the_equation():
    # L = ceil((T_max - T_ref) / (T_gen - T_ref))
    assert lt.layers(500, 1000, 6000) == 11
    assert lt.layers(600, 1000, 6000) == 14
    assert lt.layers(500, 1000, 36160) == 72
    ok, L, g = lt.condition(5e-5, 1000, 500, 1000, 6000)
    assert ok and L == 11 and abs(g - 0.55) < 1e-12
    assert not lt.condition(5e-5, 2000, 500, 1000, 6000)[0]
    C = lt.max_code_blocks(5e-5, 500, 1000, 6000)
    assert 5e-5 * C * 11 < 1 <= 5e-5 * (C + 1) * 11
    with pytest.raises(ValueError):
        lt.layers(1000, 1000, 6000)
    # no tail: every number of code blocks satisfies the requirement
    assert lt.max_code_blocks(0.0, 500, 1000, 6000) is None
    # the requirement fails: the derivation gives no slowdown bound
    assert lt.slowdown_bound(5e-5, 2000, 500, 1000, 6000) is None


def test_slowdown_bound_with_no_tail_is_the_paper_value():
    # Sec. 7.2: with eps = 0 every run finishes within T_ref = 600 of T_gen = 1000: R = 1.6
    assert lt.slowdown_bound(0.0, 10, 600, 1000, 6000) == pytest.approx(1.6)


def test_slowdown_bound_dominates_its_first_order_form_and_the_probability_bound():
    g = json.load(open(os.path.join(GOLDEN, "relay_parameters_appA3.json")))
    tmax = g["two_gross_max_runtime_cycles"]
    for eps in (1e-6, 1e-5, 8e-5):
        ok, L, gamma = lt.condition(eps, 10, 500, 1000, tmax)
        assert ok
        b = lt.slowdown_bound(eps, 10, 500, 1000, tmax)
        assert b >= 1 + 0.5 + 2 * gamma          # 2 gamma / (1 - gamma) >= 2 gamma
        # the derivation's 1 - (1 - x)^n <= x n
        n = 2 * 10
        assert 1 - (1 - eps) ** n <= eps * n


def test_report_from_iteration_counts():
    iters = np.array([1] * 9990 + [300] * 10)
    r = lt.report(iters, t_ref=250, t_gen=1000, t_max=18080, C=10)
    assert r["eps"] == pytest.approx(1e-3)
    assert r["L"] == math.ceil((18080 - 250) / 750)
    assert r["holds"] == (1e-3 * 10 * r["L"] < 1)
