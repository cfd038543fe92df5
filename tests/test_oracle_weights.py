"""Pins for the oracle's antenna patterns and weights (Eq. (1), Eq. (22)) and
for its weight quantisation.

Closed forms for simple geometries, invariance of F+^2 + Fx^2 under the
polarisation angle, the 2/5 sky average of a 90-degree interferometer
(checked by Gauss-Legendre quadrature over the sphere), the [0, 1] range,
the sum-to-N normalisation, and rounding against numpy casts and exact
rational arithmetic.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1904_04873_gb300 import synth

X = np.array([1.0, 0.0, 0.0])
Y = np.array([0.0, 1.0, 0.0])
Z = np.array([0.0, 0.0, 1.0])


def _f2(n, u, v, psi=0.0):
    Fp, Fc = oracle.antenna(n, u, v, psi)
    return Fp * Fp + Fc * Fc


def test_closed_forms():
    # source overhead of an L-shaped detector: full response
    assert abs(_f2(Z, X, Y) - 1.0) < 1e-15
    # source along one arm: D:e+ = -1/2, D:ex = 0
    assert abs(_f2(X, X, Y) - 0.25) < 1e-15
    assert abs(_f2(-Y, X, Y) - 0.25) < 1e-15
    # source in the detector plane along the bisector: blind direction
    b = np.array([1.0, 1.0, 0.0]) / math.sqrt(2.0)
    assert _f2(b, X, Y) < 1e-30


def _random_detector(rng):
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    return q[:, 0], q[:, 1]


def test_psi_invariance_and_rotation():
    rng = np.random.default_rng(11)
    for _ in range(200):
        u, v = _random_detector(rng)
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        psi = rng.uniform(0, math.pi)
        Fp0, Fc0 = oracle.antenna(n, u, v, 0.0)
        Fp1, Fc1 = oracle.antenna(n, u, v, psi)
        assert abs((Fp0 ** 2 + Fc0 ** 2) - (Fp1 ** 2 + Fc1 ** 2)) < 1e-14
        # (F+, Fx) turns by 2 psi (spin-2 polarisation)
        a0, a1 = math.atan2(Fc0, Fp0), math.atan2(Fc1, Fp1)
        d = (a1 - a0) % (2 * math.pi)
        assert min(abs(d - (-2 * psi) % (2 * math.pi)), abs(d - (2 * psi) % (2 * math.pi)),
                   2 * math.pi - abs(d - (2 * psi) % (2 * math.pi))) < 1e-9 or (Fp0 ** 2 + Fc0 ** 2) < 1e-20


def test_range_zero_one():
    rng = np.random.default_rng(12)
    for _ in range(500):
        u, v = _random_detector(rng)
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        f = _f2(n, u, v)
        assert -1e-15 <= f <= 1.0 + 1e-14


def test_sky_average_two_fifths():
    # <F+^2 + Fx^2> over the sphere = 2/5 for perpendicular arms.
    rng = np.random.default_rng(13)
    u, v = _random_detector(rng)
    xg, wg = np.polynomial.legendre.leggauss(12)
    nphi = 24
    acc = 0.0
    for ct, wct in zip(xg, wg):
        st = math.sqrt(1.0 - ct * ct)
        for k in range(nphi):
            ph = 2 * math.pi * k / nphi
            n = np.array([st * math.cos(ph), st * math.sin(ph), ct])
            acc += wct * (2 * math.pi / nphi) * _f2(n, u, v)
    assert abs(acc / (4 * math.pi) - 0.4) < 1e-12


def test_weights_normalisation_and_proportionality():
    pr = synth.tiny()
    sky = synth.fibonacci_sky(5)
    Sn = np.linspace(1.0, 1.5, pr.N)
    w = oracle.weights(sky, pr.arms, Sn, norm=True)
    assert np.allclose(w.sum(axis=1), pr.N, rtol=1e-13)
    raw = oracle.weights(sky, pr.arms, Sn, norm=False)
    for s in range(5):
        f2 = np.array([_f2(sky[s], pr.arms[i, :3], pr.arms[i, 3:]) for i in range(pr.N)])
        assert np.allclose(raw[s], f2 / Sn, rtol=1e-13, atol=1e-300)
        ratio = w[s] / raw[s]
        assert np.allclose(ratio, ratio[0], rtol=1e-13)
    # the detector turns with the Earth: weights vary over the run
    assert np.ptp(w[0]) > 0.1


def test_quantize_f32_and_f16_match_numpy():
    rng = np.random.default_rng(14)
    x = np.concatenate([rng.uniform(0, 8, 20000), rng.uniform(0, 1e-4, 2000),
                        rng.uniform(0, 1e-7, 2000), [65504.0, 65519.9, 6.0e-8, 2.98e-8]])
    q16 = oracle.quantize(x, "f16")
    assert np.array_equal(q16, x.astype(np.float16).astype(np.float64))
    q32 = oracle.quantize(x, "f32")
    assert np.array_equal(q32, x.astype(np.float32).astype(np.float64))
    # exact ties between neighbouring halves go to the even mantissa
    a = np.float16(1.0)
    b = np.nextafter(a, np.float16(2.0))
    mid = (float(a) + float(b)) / 2.0
    assert oracle.quantize(np.array([mid]), "f16")[0] == float(a)


def _bf16_exact(x: float) -> float:
    # round to 8 significant bits, ties to even, with exact rationals
    if x == 0.0:
        return 0.0
    fx = Fraction(x)
    e = math.floor(math.log2(x))
    while Fraction(2) ** e > fx:
        e -= 1
    while Fraction(2) ** (e + 1) <= fx:
        e += 1
    e = max(e, -126)
    q = Fraction(2) ** (e - 7)
    r = fx / q
    lo = math.floor(r)
    rem = r - lo
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and lo % 2 == 1):
        lo += 1
    return float(lo * q)


def test_quantize_bf16_exact_rational():
    rng = np.random.default_rng(15)
    x = np.concatenate([rng.uniform(0, 8, 3000), rng.uniform(0, 1e-3, 500)])
    ties = [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 3.0 * (1.0 + 2.0 ** -8)]
    x = np.concatenate([x, ties])
    q = oracle.quantize(x, "bf16")
    ref = np.array([_bf16_exact(float(v)) for v in x])
    assert np.array_equal(q, ref)
