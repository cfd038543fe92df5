"""Binary template bank (Sec. V.B, Eq. (30)-(32)) and explicit-bank problems, host side.

The oracle's bank (oracle/bank.py) is pinned to what the paper fixes: the
spacings of Eq. (30)-(32) evaluated where they are smallest, coverage of the
region, and the paper's template-count scaling (the binary part of
dN ~ T_c^6 T_obs f^5 Omega^4 a_p^2 is T_c^3 f^3 T_obs).  The library's
generator (bsh_template_bank) must then produce the very same bank, entry for
entry.  An explicit bank that lists a grid's templates in grid order gives the
oracle the grid's counts exactly.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import bank as obank
from paper_1904_04873_gb300 import bsh, synth
from _common import oracle_inputs, oracle_problem

DAY = synth.DAY


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1904_04873_gb300 import build
    build.build()


def spec(**kw):
    s = dict(f=200.1, T_c=900.0, T_obs=synth.YEAR_SID, t_mid=0.0, ap_min=3.0, ap_max=13.0, P_min=10 * DAY,
             P_max=20 * DAY, m_a=1.6, m_Om=1.6, m_t=1.6, ap_block=1.0)
    s.update(kw)
    return s


@pytest.mark.parametrize("res", ["oracle", "library"])
def test_resolution_scalings(res):
    # the dependence on each variable that Eq. (30)-(32) fix
    fn = obank.resolution if res == "oracle" else bsh.binary_resolution
    f, T_c, T_obs, a, Om = 200.1, 900.0, 3.0e7, 5.0, 2 * math.pi / (15 * DAY)
    d_ap, d_Om, d_t = fn(f, T_c, T_obs, a, Om, 1.0, 1.0, 1.0)
    base = (d_ap, d_Om, d_t)
    assert np.allclose(fn(2 * f, T_c, T_obs, a, Om, 1, 1, 1), np.array(base) / 2, rtol=1e-14)
    assert np.allclose(fn(f, 2 * T_c, T_obs, a, Om, 1, 1, 1), np.array(base) / 2, rtol=1e-14)
    assert np.allclose(fn(f, T_c, T_obs, 2 * a, Om, 1, 1, 1), (d_ap, d_Om / 2, d_t / 2), rtol=1e-14)
    assert np.allclose(fn(f, T_c, T_obs, a, 2 * Om, 1, 1, 1), (d_ap / 2, d_Om / 4, d_t / 4), rtol=1e-14)
    assert np.allclose(fn(f, T_c, 2 * T_obs, a, Om, 1, 1, 1), (d_ap, d_Om / 2, d_t), rtol=1e-14)
    assert np.allclose(fn(f, T_c, T_obs, a, Om, 4.0, 9.0, 16.0), (2 * d_ap, 3 * d_Om, 4 * d_t), rtol=1e-14)
    # the product of the three spacings: the binary part of the paper's template density
    vol = d_ap * d_Om * d_t
    assert vol * (T_c * f) ** 3 * a ** 2 * Om ** 4 * T_obs == pytest.approx(
        math.sqrt(6.0 * 72.0 * 6.0) / math.pi ** 3, rel=1e-13)


def _golden_points():
    """Rows of tests/golden/bank_resolution.txt: (inputs, expected spacings), the expected values
    evaluated from the closed forms written there."""
    import os
    from fractions import Fraction
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "bank_resolution.txt")
    env = {"pi": math.pi, "sqrt": math.sqrt, "__builtins__": {}}
    rows = []
    for line in open(path):
        if not line.strip() or line.startswith("#"):
            continue
        lhs, rhs = line.split("|")
        name, *vals = lhs.split()
        f, T_c, T_obs, a, Om = (float(x) for x in vals[:5])
        m = [float(Fraction(x)) for x in vals[5:8]]
        exp = [eval(x, env) for x in rhs.split()]
        rows.append((name, (f, T_c, T_obs, a, Om, *m), exp))
    return rows


@pytest.mark.parametrize("res", ["oracle", "library"])
def test_resolution_hand_worked_points(res):
    # each spacing separately, at points worked by hand (tests/golden/bank_resolution.txt)
    fn = obank.resolution if res == "oracle" else bsh.binary_resolution
    rows = _golden_points()
    assert [r[0] for r in rows] == ["A", "B"]
    for name, args, exp in rows:
        got = fn(*args)
        for k, (g, e) in enumerate(zip(got, exp)):
            assert g == pytest.approx(e, rel=1e-13), (name, ("d_ap", "d_Om", "d_t")[k], g, e)


def test_bank_layout_and_spacings():
    sp = spec(ap_block=1.5)
    orbit, bo, ba = obank.template_bank(**sp)
    assert orbit.shape[0] > 100 and ba.size >= orbit.shape[0]
    assert np.all(np.diff(bo) >= 0) and bo[0] == 0 and bo[-1] == orbit.shape[0] - 1
    assert np.all(orbit[:, 2:] == 0.0)
    Oms = np.unique(orbit[:, 0])
    assert Oms[0] == pytest.approx(2 * math.pi / sp["P_max"], rel=1e-15)
    assert Oms[-1] <= 2 * math.pi / sp["P_min"]
    for k in range(len(Oms) - 1):
        _, d_Om, _ = obank.resolution(sp["f"], sp["T_c"], sp["T_obs"], sp["ap_max"], Oms[k], 1.6, 1.6, 1.6)
        assert Oms[k + 1] - Oms[k] == pytest.approx(d_Om, rel=1e-9)
    # one Omega: a_p steps, blocks, t_asc grids over one period
    Om = Oms[len(Oms) // 2]
    rows = np.nonzero(orbit[:, 0] == Om)[0]
    d_ap, _, _ = obank.resolution(sp["f"], sp["T_c"], sp["T_obs"], 5.0, Om, 1.6, 1.6, 1.6)
    aps = np.unique(ba[np.isin(bo, rows)])
    assert aps[0] == sp["ap_min"] and aps[-1] <= sp["ap_max"] < aps[-1] + d_ap
    assert np.allclose(np.diff(aps), d_ap, rtol=1e-9)
    P = 2 * math.pi / Om
    for r in rows:
        a_row = ba[bo == r]
        assert a_row.max() <= sp["ap_block"] * a_row.min() + 1e-12
    ts = orbit[rows, 1]
    assert ts.min() == pytest.approx(-P / 2) and ts.max() < P / 2


def test_bank_covers_the_region():
    # every point lies within half a spacing (evaluated at the point) of a template in each
    # parameter -- checked for the nearest Omega, a_p and t_asc templates
    sp = spec(ap_block=1.3, m_a=4.0, m_Om=4.0, m_t=4.0)
    orbit, bo, ba = obank.template_bank(**sp)
    rng = np.random.default_rng(5)
    Oms = np.unique(orbit[:, 0])
    for _ in range(200):
        Om = rng.uniform(2 * math.pi / sp["P_max"], 2 * math.pi / sp["P_min"])
        a = rng.uniform(sp["ap_min"], sp["ap_max"])
        t = rng.uniform(-math.pi / Om, math.pi / Om)
        d_ap, d_Om, d_t = obank.resolution(sp["f"], sp["T_c"], sp["T_obs"], a, Om, 4.0, 4.0, 4.0)
        k = np.searchsorted(Oms, Om) - 1
        k = min(max(k, 0), len(Oms) - 1)
        assert Om - Oms[k] <= d_Om * 1.0000001
        rows = np.nonzero(orbit[:, 0] == Oms[k])[0]
        sel = np.isin(bo, rows)
        aps = np.unique(ba[sel])
        j = np.searchsorted(aps, a) - 1
        assert 0 <= a - aps[max(j, 0)] <= d_ap * 1.0000001 * (Om / Oms[k])
        # t_asc rows of the block holding the first a_p at or above a (its spacing is the
        # one at an a_p >= a, so at most the spacing at the point)
        a_up = aps[min(j + 1, aps.size - 1)]
        blk_rows = np.unique(bo[sel & (ba == a_up)])
        tt = np.sort(orbit[blk_rows, 1])
        P = 2 * math.pi / Oms[k]
        i = np.searchsorted(tt, t) - 1
        gap = (t - tt[i]) if i >= 0 else (t + P - tt[-1])
        assert 0 <= gap <= d_t * (Om / Oms[k]) ** 2 * 1.0000001 + 1e-9


@pytest.mark.parametrize("what,factor,expect", [("f", 2.0, 8.0), ("T_c", 2.0, 8.0), ("T_obs", 2.0, 2.0)])
def test_bank_size_follows_the_template_count_scaling(what, factor, expect):
    # ranges many spacings wide in every dimension: the bank is near its continuum limit
    sp = spec(m_a=0.4, m_Om=6.4, m_t=6.4, ap_min=20.0, ap_max=30.0, P_min=12 * DAY, P_max=13 * DAY)
    n0 = obank.template_bank(**sp)[2].size
    sp2 = dict(sp)
    sp2[what] = sp[what] * factor
    n1 = obank.template_bank(**sp2)[2].size
    assert n1 / n0 == pytest.approx(expect, rel=0.05)


@pytest.mark.parametrize("kw", [dict(), dict(ap_block=1.5), dict(ap_block=3.0, m_a=0.4, m_Om=6.4, m_t=1.0),
                                dict(f=1200.0, T_c=300.0, P_min=2 * DAY, P_max=3 * DAY, ap_min=0.5, ap_max=1.5)])
def test_library_bank_equals_the_oracle_bank(kw):
    sp = spec(**kw)
    lo, lb, la = bsh.template_bank(**sp)
    oo, ob, oa = obank.template_bank(**sp)
    assert lo.shape == oo.shape and lb.size == ob.size
    assert np.array_equal(lo, oo) and np.array_equal(lb, ob) and np.array_equal(la, oa)


def test_bank_argument_errors():
    with pytest.raises(bsh.BshError):
        bsh.template_bank(**spec(P_min=600.0))          # P_min <= T_c
    with pytest.raises(bsh.BshError):
        bsh.template_bank(**spec(ap_block=0.5))
    with pytest.raises(bsh.BshError):
        bsh.template_bank(**spec(ap_min=-1.0))


def test_oracle_grid_written_as_bank_counts_the_same():
    pr = synth.mid(n_sky=3, n_per_det=60, n_ap=3, n_P=2, n_T=2, patch_size=3)
    rho, bits, w = oracle_inputs(pr)
    a = oracle_problem(pr, bits, w).count_dense()
    bank = synth.grid_as_bank(pr)
    assert bank.B == pr.B
    b = oracle_problem(bank, bits, w).count_dense()
    assert np.array_equal(a["n_unw"], b["n_unw"]) and np.array_equal(a["n_w"], b["n_w"])


def test_debug_windows_of_a_bank_problem():
    # the kernels' fixed-point window code on a metric bank (host build) against the oracle's bins
    from test_track_fixedpoint import _check
    pr = synth.metric(n_sky=64, n_per_det=300)
    pr = synth.attach_bank(pr, *obank.template_bank(**synth.metric_spec(pr, m=6.4)))
    _check(pr, 3000, 7)
