"""Pins for the oracle's low-eccentricity (ELL1) track, Eq. (14) times T_c.

The ELL1 frequency is the first-order expansion in e of the exact Keplerian
orbit of Eq. (6)-(10), so the pins compare it with that orbit, solved here
independently (Kepler's equation by Newton iteration, the projected radius of
Eq. (9) differentiated analytically): the difference is O(e^2) a_p Omega F,
while an error in the first-order terms (a wrong sign of kappa or eta, a
missing factor 2 in the harmonic, kappa and eta swapped) leaves an O(e)
difference and fails.  Further pins: kappa = eta = 0 reproduces the circular
track bit for bit, invariance under t_asc -> t_asc + P, and the dense count
of a (kappa, eta) grid equals the counts of the single-orbit problems it is
made of (the template layout).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1904_04873_gb300 import synth
from _common import oracle_inputs, oracle_problem


def _kepler_E(M, e):
    """Eccentric anomaly from the mean anomaly M = E - e sin E (Newton, to 1e-15)."""
    E = M + e * np.sin(M)
    for _ in range(50):
        dE = (E - e * np.sin(E) - M) / (1.0 - e * np.cos(E))
        E = E - dE
        if np.max(np.abs(dE)) < 1e-15:
            break
    return E


def _exact_x(F, vn, ap, Om, Ta, e, w, t):
    """F (1 + v.n - d(R/c)/dt) for the Keplerian orbit of Eq. (6)-(10).

    R/c = a_p [sin w (cos E - e) + cos w sin E sqrt(1 - e^2)] with the mean
    anomaly Omega (t - tau_p) = E - e sin E and tau_p = t_asc + w / Omega.
    dE/dt = Omega / (1 - e cos E).
    """
    tp = Ta + w / Om
    E = _kepler_E(Om * (t - tp), e)
    dE = Om / (1.0 - e * np.cos(E))
    dR = ap * (-math.sin(w) * np.sin(E) + math.cos(w) * np.cos(E) * math.sqrt(1.0 - e * e)) * dE
    return F * (1.0 + vn - dR)


def _ell1_x(F, v, n, ap, Om, Ta, e, w, ts):
    kap, eta = e * math.cos(w), e * math.sin(w)
    return np.array([oracle.track_x_ell1(F, v, n, ap, Om, Ta, kap, eta, t) for t in ts])


@pytest.mark.parametrize("e", [1e-3, 1e-2, 3e-2])
def test_first_order_agreement_with_keplerian_orbit(e):
    rng = np.random.default_rng(31)
    v = np.zeros(3)
    n = np.array([0.0, 0.0, 1.0])
    for _ in range(20):
        F = float(rng.integers(90000, 280000))
        ap = rng.uniform(0.5, 15.0)
        P = rng.uniform(10.0, 60.0) * synth.DAY
        Om = 2.0 * math.pi / P
        Ta = rng.uniform(-P / 2, P / 2)
        w = rng.uniform(0.0, 2.0 * math.pi)
        ts = np.linspace(-P, P, 257)
        xe = _exact_x(F, 0.0, ap, Om, Ta, e, w, ts)
        xa = _ell1_x(F, v, n, ap, Om, Ta, e, w, ts)
        scale = F * ap * Om
        # second-order remainder: |d/dt of the O(e^2) terms of R/c| <= 4 e^2 a_p Omega
        assert np.max(np.abs(xa - xe)) <= 4.0 * e * e * scale
        # and the first-order terms matter: the circular track misses them by O(e)
        xc = np.array([oracle.track_x(F, v, n, ap, Om, Ta, t) for t in ts])
        assert np.max(np.abs(xc - xe)) >= 0.5 * e * scale


def test_wrong_first_order_terms_are_detected():
    # The pin above separates the ELL1 form from each plausible mistake in it.
    e, w = 1e-2, 0.3
    F, ap, Om, Ta = 2.0e5, 8.0, 2.0 * math.pi / (20.0 * synth.DAY), 1234.0
    ts = np.linspace(-2e6, 2e6, 513)
    xe = _exact_x(F, 0.0, ap, Om, Ta, e, w, ts)
    scale = F * ap * Om
    kap, eta = e * math.cos(w), e * math.sin(w)
    ph = Om * (ts - Ta)
    good = F * (1.0 - ap * Om * (np.cos(ph) + kap * np.cos(2 * ph) + eta * np.sin(2 * ph)))
    assert np.max(np.abs(good - xe)) <= 4.0 * e * e * scale
    for g in (np.cos(ph) + kap * np.cos(2 * ph) - eta * np.sin(2 * ph),     # eta sign as printed
              np.cos(ph) - kap * np.cos(2 * ph) + eta * np.sin(2 * ph),     # kappa sign
              np.cos(ph) + eta * np.cos(2 * ph) + kap * np.sin(2 * ph),     # swapped
              np.cos(ph) + kap * np.cos(ph) + eta * np.sin(ph)):            # first harmonic
        bad = F * (1.0 - ap * Om * g)
        assert np.max(np.abs(bad - xe)) > 0.2 * e * scale    # 5x the second-order bound


def test_circular_limit_is_bitwise():
    rng = np.random.default_rng(32)
    pr = synth.mid(n_sky=16, n_per_det=50, n_ap=2, n_P=2, n_T=2)
    for _ in range(2000):
        i, s = rng.integers(pr.N), rng.integers(pr.S)
        F = float(rng.integers(90000, 280000))
        ap = rng.uniform(0.0, 15.0)
        Om = 2 * math.pi / (rng.uniform(10.0, 60.0) * synth.DAY)
        Ta = rng.uniform(-1e6, 1e6)
        a = oracle.track_x(F, pr.v[i], pr.sky[s], ap, Om, Ta, pr.t[i])
        b = oracle.track_x_ell1(F, pr.v[i], pr.sky[s], ap, Om, Ta, 0.0, 0.0, pr.t[i])
        assert a == b


def test_period_shift_of_t_asc():
    rng = np.random.default_rng(33)
    pr = synth.mid(n_sky=16, n_per_det=50, n_ap=2, n_P=2, n_T=2)
    for _ in range(500):
        i, s = rng.integers(pr.N), rng.integers(pr.S)
        F = float(rng.integers(90000, 280000))
        ap = rng.uniform(0.0, 15.0)
        P = rng.uniform(10.0, 60.0) * synth.DAY
        Om = 2 * math.pi / P
        Ta = rng.uniform(-P / 2, P / 2)
        kap, eta = rng.uniform(-0.05, 0.05, 2)
        a = oracle.track_x_ell1(F, pr.v[i], pr.sky[s], ap, Om, Ta, kap, eta, pr.t[i])
        b = oracle.track_x_ell1(F, pr.v[i], pr.sky[s], ap, Om, Ta + P, kap, eta, pr.t[i])
        assert abs(a - b) < 1e-6


def test_grid_layout_matches_single_orbit_problems():
    kappa = np.array([-0.02, 0.0, 0.03])
    eta = np.array([0.01, -0.025])
    pr = synth.make_problem("ecc-small", n_per_det=40, dets=["H1", "L1"], T_sft=900.0, span=synth.YEAR_SID,
                            random_times=True, f_lo=200.0, n_f0=40, half_bin=False,
                            sky=synth.fibonacci_sky(3), patch_size=3, a_p=np.array([2.0, 9.0]),
                            P_days=np.array([15.0, 30.0]), n_T=2, power_kind="exp", kappa=kappa, eta=eta)
    rho, bits, w = oracle_inputs(pr)
    d = oracle_problem(pr, bits, w).count_dense()
    n_ap, n_T = pr.a_p.size, pr.T_asc.shape[1]
    assert d["n_unw"].shape == (pr.S, pr.B, pr.n_f0)
    assert pr.B == n_ap * pr.T_asc.size * kappa.size * eta.size
    for ik in range(kappa.size):
        for ie in range(eta.size):
            one = oracle.OracleProblem(bits=bits, w=w, v=pr.v, t=pr.t, F0=pr.F0, n_f0=pr.n_f0, sky=pr.sky,
                                       a_p=pr.a_p, Omega=pr.Omega, T_asc=pr.T_asc, k_lo=pr.k_lo, K=pr.K,
                                       kappa=kappa[ik:ik + 1], eta=eta[ie:ie + 1]).count_dense()
            for ot in range(pr.T_asc.size):
                for iap in range(n_ap):
                    b_full = ((ot * kappa.size + ik) * eta.size + ie) * n_ap + iap
                    b_one = ot * n_ap + iap
                    assert np.array_equal(d["n_unw"][:, b_full], one["n_unw"][:, b_one])
                    assert np.array_equal(d["n_w"][:, b_full], one["n_w"][:, b_one])
    # the circular grid is the kappa = eta = 0 slice
    circ = oracle.OracleProblem(bits=bits, w=w, v=pr.v, t=pr.t, F0=pr.F0, n_f0=pr.n_f0, sky=pr.sky,
                                a_p=pr.a_p, Omega=pr.Omega, T_asc=pr.T_asc, k_lo=pr.k_lo, K=pr.K).count_dense()
    zero = oracle.OracleProblem(bits=bits, w=w, v=pr.v, t=pr.t, F0=pr.F0, n_f0=pr.n_f0, sky=pr.sky,
                                a_p=pr.a_p, Omega=pr.Omega, T_asc=pr.T_asc, k_lo=pr.k_lo, K=pr.K,
                                kappa=[0.0], eta=[0.0]).count_dense()
    assert np.array_equal(circ["n_unw"], zero["n_unw"]) and np.array_equal(circ["n_w"], zero["n_w"])
