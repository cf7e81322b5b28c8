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


def _sec72():
    return json.load(open(os.path.join(GOLDEN, "latency_tail_sec72.json")))


def _c_bound(eps, L):
    """The requirement eps * C * L < 1 as a bound on C: C < 1 / (eps * L)."""
    return 1.0 / (eps * L)


@pytest.mark.parametrize("code", ["gross", "two_gross"])
def test_printed_code_block_limits_follow_from_t_ref_600_and_one_more_layer(code):
    """Sec. 7.2 prints C < 1333 (gross) and C < 138 (two-gross).  Neither T_ref reading
    with the equation's L reproduces both; T_ref = 600 (the value of the paper's eps = 0
    sentence) with L + 1 layers reproduces both exactly, as floor(1 / (eps (L + 1)))."""
    g = _sec72()
    c = g[code]
    tgen, tmax, eps = g["T_gen_cycles"], c["T_max_cycles"], c["eps_upper"]
    L600 = lt.layers(600, tgen, tmax)
    assert math.floor(_c_bound(eps, L600 + 1)) == c["printed_max_code_blocks_exclusive"]
    # the equation as written reproduces neither number at either T_ref
    for t_ref in (g["T_ref_stated_cycles"], 600):
        L = lt.layers(t_ref, tgen, tmax)
        assert math.floor(_c_bound(eps, L)) != c["printed_max_code_blocks_exclusive"]
        # and its own limit is what max_code_blocks returns
        C = lt.max_code_blocks(eps, t_ref, tgen, tmax)
        assert eps * C * L < 1 <= eps * (C + 1) * L


def test_printed_slowdown_bounds_gross_full_two_gross_first_order():
    """C = 10: the gross bound <R> < 1.62 holds with the full Eq. latency-tail-slowdown at
    T_ref = 600 (1.614; 1.615 with L + 1); the two-gross 1.74 is the first-order form
    1 + T_ref/T_gen + 2 gamma at T_ref = 600 (1.742; 1.744 with L + 1), which the full
    bound (1.753 / 1.755) exceeds.  At the stated T_ref = 500 the equations give 1.511
    and 1.622, neither printed value."""
    g = _sec72()
    tgen, C = g["T_gen_cycles"], g["C_for_the_slowdown_estimate"]
    gr, tg = g["gross"], g["two_gross"]

    def first_order(eps, t_ref, tmax, extra=0):
        L = lt.layers(t_ref, tgen, tmax) + extra
        return 1 + t_ref / tgen + 2 * eps * C * L

    def full(eps, t_ref, tmax, extra=0):
        gamma = eps * C * (lt.layers(t_ref, tgen, tmax) + extra)
        return 1 + t_ref / tgen + 2 * gamma / (1 - gamma)

    # gross: both forms and both layer counts at T_ref = 600 are below the printed 1.62
    b = lt.slowdown_bound(gr["eps_upper"], C, 600, tgen, gr["T_max_cycles"])
    assert b == pytest.approx(full(gr["eps_upper"], 600, gr["T_max_cycles"]))
    assert b == pytest.approx(1.6141, abs=1e-4) and b < gr["printed_slowdown_upper"]
    assert full(gr["eps_upper"], 600, gr["T_max_cycles"], 1) < gr["printed_slowdown_upper"]
    # two-gross: the printed 1.74 is the first-order value truncated to two decimals
    for extra in (0, 1):
        fo = first_order(tg["eps_upper"], 600, tg["T_max_cycles"], extra)
        assert math.floor(fo * 100) / 100 == tg["printed_slowdown_upper"]
        assert full(tg["eps_upper"], 600, tg["T_max_cycles"], extra) > tg["printed_slowdown_upper"]
    assert lt.slowdown_bound(tg["eps_upper"], C, 600, tgen, tg["T_max_cycles"]) == pytest.approx(
        1.7533, abs=1e-4)
    # the stated T_ref = 500 reproduces neither printed bound
    t500 = g["T_ref_stated_cycles"]
    assert lt.slowdown_bound(gr["eps_upper"], C, t500, tgen, gr["T_max_cycles"]) == pytest.approx(
        1.5111, abs=1e-4)
    assert lt.slowdown_bound(tg["eps_upper"], C, t500, tgen, tg["T_max_cycles"]) == pytest.approx(
        1.6222, abs=1e-4)
    # the eps = 0 sentence
    assert lt.slowdown_bound(0.0, C, 600, tgen, gr["T_max_cycles"]) == pytest.approx(
        g["printed_slowdown_at_eps0"])
