"""Pins for the oracle's look-up-table (LUT) approximation of stage 1 (Sec. IV.B).

In a block of L contiguous f0 templates the LUT reuses the modulation F_ref D
of the block's middle template: k_j = floor(F_ref + F_ref D + 1/2) + (j - j_ref).
Pins: L = 1 and D = 0 reduce to the exact track; the reference template's
count is the exact one; a LUT count equals the exact count of the reference
template on the peakgram shifted by the f0 offset (the shift's direction);
and the fraction of SFTs whose LUT bin leaves the exact track matches the
probability |(j - j_ref) D| that the exact argument F_j + F_j D + 1/2 and the
LUT argument F_j + F_ref D + 1/2, which differ by (j - j_ref) D, straddle an
integer (D computed here with numpy from Eq. (15)).  A reference taken at the
block's first template would double that fraction; a shift of the wrong sign
would leave the track almost everywhere.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1904_04873_gb300 import synth
from _common import oracle_inputs, oracle_problem, orbit_of, pack_bits


def lut_block(n_f0):
    """Blocks of at most 32 f0 templates, as even as possible."""
    nb = -(-n_f0 // 32)
    return -(-n_f0 // nb)


def j_ref(j, L, n_f0):
    q = j // L
    return q * L + (min(L, n_f0 - q * L) - 1) // 2


def _fast_binaries():
    # a_p Omega up to 4e-3 so that LUT departures are frequent enough to count
    return synth.make_problem("lut", n_per_det=300, dets=["H1", "L1"], T_sft=900.0, span=synth.YEAR_SID,
                              random_times=True, f_lo=200.0, n_f0=90, half_bin=False,
                              sky=synth.fibonacci_sky(4), patch_size=4, a_p=np.array([60.0, 100.0]),
                              P_days=np.array([1.5, 2.0]), n_T=2, power_kind="exp")


def _op(pr, bits, w, L):
    return oracle.OracleProblem(bits=bits, w=w, v=pr.v, t=pr.t, F0=pr.F0, n_f0=pr.n_f0, sky=pr.sky,
                                a_p=pr.a_p, Omega=pr.Omega, T_asc=pr.T_asc, k_lo=pr.k_lo, K=pr.K,
                                kappa=pr.kappa, eta=pr.eta, lut_block=L)


def test_block_of_one_is_exact():
    pr = synth.mid(n_sky=3, n_per_det=60, n_ap=3, n_P=2, n_T=2, patch_size=3)
    rho, bits, w = oracle_inputs(pr)
    a = oracle_problem(pr, bits, w).count_dense()
    b = _op(pr, bits, w, 1).count_dense()
    assert np.array_equal(a["n_unw"], b["n_unw"]) and np.array_equal(a["n_w"], b["n_w"])


def test_zero_modulation_is_exact():
    pr = synth.mid(n_sky=3, n_per_det=60, n_ap=3, n_P=2, n_T=2, patch_size=3)
    pr.v = np.zeros_like(pr.v)
    pr.a_p = np.zeros_like(pr.a_p)
    rho, bits, w = oracle_inputs(pr)
    a = oracle_problem(pr, bits, w).count_dense()
    b = _op(pr, bits, w, lut_block(pr.n_f0)).count_dense()
    assert np.array_equal(a["n_unw"], b["n_unw"]) and np.array_equal(a["n_w"], b["n_w"])


def test_reference_templates_are_exact_and_shift_direction():
    pr = _fast_binaries()
    L = lut_block(pr.n_f0)
    rho, bits, w = oracle_inputs(pr)
    ex = oracle_problem(pr, bits, w)
    lut = _op(pr, bits, w, L)
    on = ((bits[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(pr.N, -1)[:, :pr.K].astype(bool)
    rng = np.random.default_rng(41)
    for _ in range(12):
        s, b = int(rng.integers(pr.S)), int(rng.integers(pr.B))
        j = int(rng.integers(pr.n_f0))
        jr = j_ref(j, L, pr.n_f0)
        cr = ex.count_one(s, b, jr)
        assert lut.count_one(s, b, jr)["n_unw"] == cr["n_unw"]
        # LUT template j on P  ==  exact template j_ref on P shifted by (j - j_ref) bins
        d = j - jr
        sh = np.zeros_like(on)
        if d >= 0:
            sh[:, :pr.K - d] = on[:, d:]
        else:
            sh[:, -d:] = on[:, :pr.K + d]
        shifted = oracle_problem(pr, pack_bits(sh, pr.W), w)
        assert lut.count_one(s, b, j)["n_unw"] == shifted.count_one(s, b, jr)["n_unw"]


def test_departure_rate_matches_its_probability():
    pr = _fast_binaries()
    L = lut_block(pr.n_f0)
    w = np.ones((pr.S, pr.N))
    rng = np.random.default_rng(42)
    observed = expected = expected_first = 0.0
    for _ in range(100):
        s, b = int(rng.integers(pr.S)), int(rng.integers(pr.B))
        j = int(rng.integers(pr.n_f0))
        ap, Om, Ta, kap, eta = orbit_of(pr, b)
        # peakgram with one bit per SFT, on the exact track of template j
        ks = np.array([oracle.track_bin_ell1(pr.F0 + j, pr.v[i], pr.sky[s], ap, Om, Ta, kap, eta, pr.t[i])[0]
                       for i in range(pr.N)])
        one = np.zeros((pr.N, pr.K), bool)
        one[np.arange(pr.N), ks - pr.k_lo] = True
        c = _op(pr, pack_bits(one, pr.W), w, L).count_one(s, b, j)
        observed += pr.N - c["n_unw"]
        D = pr.v @ pr.sky[s] - ap * Om * np.cos(Om * (pr.t - Ta))
        expected += np.abs((j - j_ref(j, L, pr.n_f0)) * D).sum()
        expected_first += np.abs((j - (j // L) * L) * D).sum()
    sigma = math.sqrt(expected)
    assert expected > 800
    assert abs(observed - expected) < 5 * sigma, (observed, expected, expected_first)
    assert expected_first > expected + 10 * sigma
