"""Pins for the oracle's peakgram (Eq. (20)-(21) and the rho_th threshold, Sec. IV.A).

The running median is checked against numpy.median on the same shifted
101-bin windows; the threshold against closed forms (constant rows, single
spikes) and against the Exp(1) peak density exp(-1.6) that the paper uses
for rho_F (Eq. (47)).
"""
import math

import numpy as np
import pytest

import oracle


def _unpack(bits, K):
    N, W = bits.shape
    b = np.unpackbits(bits.view(np.uint8).reshape(N, W, 4)[:, :, ::-1].reshape(N, W * 4), axis=1,
                      bitorder="big")
    # per word: bytes reversed -> big-endian bit order of the 32-bit word
    b = b.reshape(N, W, 32)[:, :, ::-1].reshape(N, W * 32)
    return b[:, :K].astype(bool)


def test_unpack_helper_roundtrip():
    bits = np.array([[0x00000001, 0x80000000]], dtype=np.uint32)
    u = _unpack(bits, 64)
    assert u[0, 0] and u[0, 63] and u.sum() == 2


@pytest.mark.parametrize("K", [101, 150, 333])
def test_running_median_matches_numpy(K):
    rng = np.random.default_rng(K)
    row = rng.exponential(size=K).astype(np.float32)
    for k in range(K):
        a = min(max(k - 50, 0), K - 101)
        ref = float(np.median(row[a:a + 101]))
        assert oracle.running_median(row, 101, k) == ref


def test_constant_row_and_spike():
    K = 200
    row = np.full((1, K), 3.0, np.float32)
    rho, bits = oracle.peakgram(row, 101, 1.6)
    # median = 3 -> <n>^2 = 3/ln2 -> rho = ln 2 everywhere, below threshold
    assert np.allclose(rho, math.log(2.0), rtol=1e-7)
    assert bits.sum() == 0
    row[0, 77] = 30.0
    rho, bits = oracle.peakgram(row, 101, 1.6)
    assert abs(rho[0, 77] - 10.0 * math.log(2.0)) < 1e-5
    on = _unpack(bits, K)[0]
    assert on[77] and on.sum() == 1


def test_bits_agree_with_rho_threshold():
    rng = np.random.default_rng(5)
    P = rng.exponential(size=(20, 257)).astype(np.float32) * 4.0
    rho, bits = oracle.peakgram(P, 101, 1.6)
    on = _unpack(bits, 257)
    far = np.abs(rho.astype(np.float64) - 1.6) > 1e-6
    assert np.array_equal(on[far], (rho > 1.6)[far])


def test_given_rho_mode_passes_through():
    rng = np.random.default_rng(6)
    r = rng.exponential(size=(7, 90)).astype(np.float32)
    rho, bits = oracle.peakgram(r, 0, 1.6)
    assert np.array_equal(rho, r)
    assert np.array_equal(_unpack(bits, 90), r.astype(np.float64) > 1.6)


def test_exp1_peak_density():
    # P(rho > rho_th) = exp(-rho_th) for Exp(1) powers (Sec. V.F, rho_F)
    rng = np.random.default_rng(1904)
    r = (-np.log1p(-rng.random((400, 2500)))).astype(np.float32)
    _, bits = oracle.peakgram(r, 0, 1.6, W=79)
    frac = _unpack(bits, 2500).mean()
    p = math.exp(-1.6)
    sigma = math.sqrt(p * (1 - p) / r.size)
    assert abs(frac - p) < 5 * sigma


def test_median_normalised_density_and_scale_invariance():
    # With the running-median normalisation the density stays near exp(-1.6)
    # whatever the noise level, and rho does not depend on the noise scale.
    rng = np.random.default_rng(7)
    P = rng.exponential(size=(200, 600)).astype(np.float32)
    rho1, b1 = oracle.peakgram(P, 101, 1.6)
    rho2, b2 = oracle.peakgram(P * np.float32(8.0), 101, 1.6)   # power-of-two scale: exact
    assert np.array_equal(b1, b2)
    assert np.array_equal(rho1, rho2)
    frac = _unpack(b1, 600).mean()
    assert abs(frac - math.exp(-1.6)) < 0.01
