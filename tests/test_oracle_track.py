"""Pins for the oracle's frequency track (Eq. (15) times T_c, rounded to a bin).

The oracle's FP64 value is compared with a 50-digit mpmath evaluation of
F (1 + v.n - a_p Omega cos(Omega (t - t_asc))): the bins agree everywhere
outside the tie band, and the band is much wider than the largest FP64
deviation seen.  Special cases: a_p = 0 and v = 0 (k = round(F)), a_p = 0
(isolated-star Doppler shift, Sec. IV.B), v = 0 (pure binary modulation),
invariance under t_asc -> t_asc + P, and exact ties.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1904_04873_gb300 import synth

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 50


def _x_exact(F, v, n, ap, Om, Ta, t):
    mp = mpmath.mpf
    vn = mp(v[0]) * mp(n[0]) + mp(v[1]) * mp(n[1]) + mp(v[2]) * mp(n[2])
    return mp(F) * (1 + vn - mp(ap) * mp(Om) * mpmath.cos(mp(Om) * (mp(t) - mp(Ta))))


def _random_terms(rng, m, F_lo=9.0e4, F_hi=2.8e5):
    pr = synth.mid(n_sky=64, n_per_det=200, n_ap=4, n_P=4, n_T=4)
    for _ in range(m):
        i = rng.integers(pr.N)
        s = rng.integers(pr.S)
        F = float(rng.integers(int(F_lo), int(F_hi))) + (0.5 if rng.random() < 0.3 else 0.0)
        ap = rng.uniform(0.0, 15.0)
        P = rng.uniform(10.0, 60.0) * synth.DAY
        Om = 2 * math.pi / P
        Ta = rng.uniform(-P / 2, P / 2)
        yield F, pr.v[i], pr.sky[s], ap, Om, Ta, float(pr.t[i])


def test_matches_high_precision_outside_tie_band():
    rng = np.random.default_rng(21)
    worst = 0.0
    n_checked = 0
    for F, v, n, ap, Om, Ta, t in _random_terms(rng, 3000):
        x = oracle.track_x(F, v, n, ap, Om, Ta, t)
        xe = _x_exact(F, v, n, ap, Om, Ta, t)
        worst = max(worst, abs(float(mpmath.mpf(x) - xe)))
        k, tie = oracle.track_bin(F, v, n, ap, Om, Ta, t)
        ke = int(mpmath.floor(xe + mpmath.mpf(0.5)))
        if not tie:
            assert k == ke
            n_checked += 1
    assert n_checked > 2900
    # FP64 evaluation error (|x| ~ 3e5 bins) is far inside the 1e-9 tie band
    assert worst < oracle.TIE_BAND / 10


def test_isolated_and_static_limits():
    rng = np.random.default_rng(22)
    for F, v, n, ap, Om, Ta, t in _random_terms(rng, 500):
        # a_p = 0, v = 0: the bin is F itself (integer F) or F + 1/2 (half-integer F)
        k, _ = oracle.track_bin(F, np.zeros(3), n, 0.0, Om, Ta, t)
        assert k == math.floor(F + 0.5)
        # a_p = 0: isolated-star Doppler, f = f0 (1 + v.n)
        k, tie = oracle.track_bin(F, v, n, 0.0, Om, Ta, t)
        xe = mpmath.mpf(F) * (1 + sum(mpmath.mpf(a) * mpmath.mpf(b) for a, b in zip(v, n)))
        if not tie:
            assert k == int(mpmath.floor(xe + mpmath.mpf(0.5)))
        # v = 0: pure binary modulation, f = f0 (1 - a_p Omega cos(Omega (t - t_asc)))
        k, tie = oracle.track_bin(F, np.zeros(3), n, ap, Om, Ta, t)
        xe = mpmath.mpf(F) * (1 - mpmath.mpf(ap) * mpmath.mpf(Om) *
                              mpmath.cos(mpmath.mpf(Om) * (mpmath.mpf(t) - mpmath.mpf(Ta))))
        if not tie:
            assert k == int(mpmath.floor(xe + mpmath.mpf(0.5)))


def test_period_shift_of_t_asc():
    rng = np.random.default_rng(23)
    for F, v, n, ap, Om, Ta, t in _random_terms(rng, 1000):
        P = 2 * math.pi / Om
        k1, t1 = oracle.track_bin(F, v, n, ap, Om, Ta, t)
        k2, t2 = oracle.track_bin(F, v, n, ap, Om, Ta + P, t)
        if not (t1 or t2):
            assert k1 == k2


def test_exact_forced_ties():
    # half-integer F, a_p = 0 and n perpendicular to v: x = F exactly, so
    # x + 1/2 is an integer and both roundings agree on k = F + 1/2.
    pr = synth.precision_stress(n_sky=8, n_per_det=50, n_ap=4, n_P=4, n_T=4)
    pole = pr.sky[0]
    assert pole[2] == 1.0 and np.all(pr.v[:, 2] == 0.0)
    F = pr.F0 + 7
    assert F - math.floor(F) == 0.5
    for i in range(pr.N):
        x = oracle.track_x(F, pr.v[i], pole, 0.0, pr.Omega[0], pr.T_asc[0, 0], pr.t[i])
        assert x == F
        k, tie = oracle.track_bin(F, pr.v[i], pole, 0.0, pr.Omega[0], pr.T_asc[0, 0], pr.t[i])
        assert tie and k == F + 0.5


def test_modulation_depth_bound():
    # |k - F| never exceeds F (max|v| + a_p Omega) + 1 bins (Sec. V.F band margin)
    rng = np.random.default_rng(24)
    for F, v, n, ap, Om, Ta, t in _random_terms(rng, 2000):
        k, _ = oracle.track_bin(F, v, n, ap, Om, Ta, t)
        assert abs(k - F) <= F * (np.linalg.norm(v) + ap * Om) + 1.0
