"""CPU check of the kernels' fixed-point track (host build of the same code).

bsh_debug_track_windows evaluates, on the host, the exact functions the
count kernel uses to turn a (sky point, binary template, SFT, f0 block) into
a 32-bit peak window: fixed-point tables, the fast single-cell test, the
crossing path and the exact FP64 fallback.  Every window bit must equal the
peakgram bit at the oracle's track bin (Eq. (14)/(15)) of that f0 template,
except where the oracle flags a tie.
"""
import numpy as np
import pytest

import oracle
from paper_1904_04873_gb300 import bsh, synth
from _common import orbit_of

pytest.importorskip("ctypes")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1904_04873_gb300 import build
    build.build()


def _check(pr, n_q, seed, force=None):
    rng = np.random.default_rng(seed)
    nfb_block = 32
    queries, rows, expect, ties = [], [], [], []
    for e in range(n_q):
        if force is not None:
            s, b = force
        else:
            s = int(rng.integers(pr.S))
            b = int(rng.integers(pr.B))
        i = int(rng.integers(pr.N))
        nb = -(-pr.n_f0 // nfb_block)
        JB = -(-pr.n_f0 // nb)
        j0 = int(rng.integers(nb)) * JB
        row = rng.integers(0, 2 ** 32, size=pr.W, dtype=np.uint64).astype(np.uint32)
        ap, Om, Ta, kap, eta = orbit_of(pr, b)
        bits = np.zeros(32, np.uint32)
        tie = np.zeros(32, bool)
        for j in range(32):
            k, t = oracle.track_bin_ell1(pr.F0 + j0 + j, pr.v[i], pr.sky[s], ap, Om, Ta, kap, eta, pr.t[i])
            col = k - pr.k_lo
            assert 0 <= col < 32 * pr.W
            bits[j] = (row[col >> 5] >> np.uint32(col & 31)) & 1
            tie[j] = t
        queries.append((s, b, i, j0))
        rows.append(row)
        expect.append(bits)
        ties.append(tie)
    out, path = bsh.debug_track_windows(pr, np.array(queries), np.array(rows))
    got = ((out[:, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(np.uint32)
    expect = np.array(expect)
    ties = np.array(ties)
    mism = (got != expect) & ~ties
    assert not mism.any(), f"{mism.sum()} mismatching bits; paths {np.bincount(path + 1)}"
    assert (path >= 0).all()
    return path, ties


def test_mid_band_windows():
    pr = synth.mid(n_sky=200, n_per_det=300, n_ap=8, n_P=8, n_T=8)
    path, _ = _check(pr, 4000, 1)
    # the common case takes the fast path; crossings are resolved without FP64
    assert (path == 0).mean() > 0.9
    assert (path == 1).sum() > 0


def test_full_band_windows_high_frequency():
    pr = synth.full(n_sky=500, n_per_det=300, n_f0=9000, patch_size=169)
    _check(pr, 3000, 2)


def test_tiny_windows():
    pr = synth.tiny()
    _check(pr, 2000, 3)


def test_forced_exact_ties_use_fp64_fallback():
    pr = synth.precision_stress(n_sky=8, n_per_det=100, n_ap=4, n_P=4, n_T=4)
    # pole sky point (index 0) and a_p = 0 (binary index with iap = 0)
    path, ties = _check(pr, 200, 4, force=(0, 0))
    assert ties.all()
    assert (path == 2).all()


def test_half_bin_grid_windows():
    pr = synth.precision_stress(n_sky=64, n_per_det=300, n_ap=8, n_P=8, n_T=8)
    _check(pr, 3000, 5)


def test_eccentric_grid_windows():
    # kappa, eta in [-0.05, 0.05]: the fixed-point scales widen to Omega (1 + |kappa| + |eta|)
    pr = synth.eccentric(n_sky=64, n_per_det=300, n_ap=6, n_P=4, n_T=4, n_kap=3, n_eta=3, e_max=0.05)
    path, _ = _check(pr, 4000, 6)
    assert (path == 0).mean() > 0.9
