"""Pins for the oracle's post-processing (Sec. V.E, Eq. (44)).

Distances: zero at a point, symmetric, one bin per resolution step along f and a_p
(whose resolutions are the same at both ends), Pythagoras across parameters.
Clusters: against scipy's connected components of the same threshold graph, chains
that link (spacing below the threshold) or break (above it).  Option-B cut, centroid
weights, the band's best cluster and coincidences on constructed configurations.
Ecliptic projection: the ecliptic pole maps to the origin, the ecliptic to the unit
circle.
"""
import math

import numpy as np
import pytest

from oracle import postprocess as pp_

scipy_graph = pytest.importorskip("scipy.sparse.csgraph")
sparse = pytest.importorskip("scipy.sparse")

OBL = math.radians(23.4393)
PP = dict(T_c=900.0, T_obs=3.15e7, v_over_c=1e-4, P_F=2.0, m_a=1.6, m_Om=1.6, m_t=1.6)
D_CL = math.sqrt(14.0)


def base_point(f=200.05):
    return np.array([f, 0.3, -0.2, 8.0, 2 * math.pi / (15 * 86400.0), 1.0e5])


def test_distance_basics():
    p = base_point()
    r = pp_.resolutions(p[None], PP)[0]
    assert pp_.distance2(p, r, p, r) == 0.0
    rng = np.random.default_rng(1)
    for _ in range(50):
        q = p + rng.normal(size=6) * r
        rq = pp_.resolutions(q[None], PP)[0]
        assert pp_.distance2(p, r, q, rq) == pp_.distance2(q, rq, p, r)
    # k bins along f (delta f = 1/T_c at every point)
    for k in (1, 3, 7):
        q = p.copy()
        q[0] = (200.05 * 900.0 + k) / 900.0
        rq = pp_.resolutions(q[None], PP)[0]
        # only f (and the f-dependent resolutions) change; x, y etc. coincide
        assert math.sqrt(pp_.distance2(p, r, q, rq)) == pytest.approx(k, rel=1e-9)
    # one a_p resolution step (delta a_p does not depend on a_p), then Pythagoras with f
    q = p.copy()
    q[3] += r[3]
    rq = pp_.resolutions(q[None], PP)[0]
    assert rq[3] == r[3]
    assert math.sqrt(pp_.distance2(p, r, q, rq)) == pytest.approx(1.0, rel=1e-12)
    q2 = q.copy()
    q2[0] = (200.05 * 900.0 + 1) / 900.0
    rq2 = pp_.resolutions(q2[None], PP)[0]
    # (the f step changes delta a_p by 1/(f T_c) = 5.6e-6 relative, hence the tolerance)
    assert math.sqrt(pp_.distance2(p, r, q2, rq2)) == pytest.approx(math.sqrt(2.0), rel=1e-5)


def _random_cloud(n, seed, spread):
    rng = np.random.default_rng(seed)
    p0 = base_point()
    r0 = pp_.resolutions(p0[None], PP)[0]
    return p0 + rng.normal(size=(n, 6)) * r0 * spread


@pytest.mark.parametrize("seed,spread", [(2, 3.0), (3, 6.0), (4, 12.0)])
def test_components_match_scipy(seed, spread):
    p = _random_cloud(120, seed, spread)
    valid = np.ones(len(p), bool)
    valid[::17] = False
    label, r = pp_.components(p, valid, PP, D_CL)
    n = len(p)
    rows, cols = [], []
    for i in range(n):
        for j in range(n):
            if i != j and valid[i] and valid[j] and pp_.distance2(p[i], r[i], p[j], r[j]) < D_CL * D_CL:
                rows.append(i)
                cols.append(j)
    g = sparse.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    nc, lab = scipy_graph.connected_components(g, directed=False)
    for i in range(n):
        for j in range(n):
            if valid[i] and valid[j]:
                assert (label[i] == label[j]) == (lab[i] == lab[j])
    assert np.all(label[~valid] == -1)
    for i in np.nonzero(valid)[0]:
        assert label[i] == np.min(np.nonzero(label == label[i])[0])


@pytest.mark.parametrize("step,expect", [(0.9, 1), (1.1, 6)])
def test_chains_link_or_break(step, expect):
    p = np.repeat(base_point()[None], 6, axis=0)
    for k in range(6):
        p[k, 0] = (200.05 * 900.0 + k * step * D_CL) / 900.0
    label, _ = pp_.components(p, np.ones(6, bool), PP, D_CL)
    assert len(np.unique(label)) == expect


def test_cut_centroid_and_best():
    # cluster A: a strong centre at f0 with members 1, 2, 3 bins above and below; cluster B far away
    p = np.repeat(base_point()[None], 9, axis=0)
    offs = [0, 1, -1, 2, -2, 3, -3]
    for e, k in enumerate(offs):
        p[e, 0] = (200.05 * 900.0 + k) / 900.0
    p[7, 0] = (200.05 * 900.0 + 40) / 900.0
    p[8, 0] = (200.05 * 900.0 + 41) / 900.0
    sig = np.array([10.0, 2, 2, 1, 1, 0.5, 0.5, 4.0, 3.0])
    valid = np.ones(9, bool)
    label, keep, cen, csig, best = pp_.cluster(p, sig, valid, PP, D_CL, 2.5)
    assert list(label) == [0] * 7 + [7, 7]
    assert list(keep) == [1, 1, 1, 1, 1, 0, 0, 1, 1]
    # symmetric weights about the centre: the centroid is the centre
    assert cen[0, 0] == pytest.approx(p[0, 0], rel=1e-15)
    assert csig[0] == pytest.approx(16.0) and csig[7] == pytest.approx(7.0)
    assert best == 0
    assert cen[7, 0] == pytest.approx((4.0 * p[7, 0] + 3.0 * p[8, 0]) / 7.0, rel=1e-15)
    assert np.isnan(cen[1]).all()
    # no cut keeps everyone; a single member is its own centroid
    label, keep, cen, csig, best = pp_.cluster(p[:1], sig[:1], valid[:1], PP, D_CL, 0.0)
    assert keep[0] == 1 and np.array_equal(cen[0], p[0]) and csig[0] == 10.0
    # weights are max(significance, 0); all-zero weights give the plain mean
    label, keep, cen, csig, best = pp_.cluster(p[7:9], np.array([-1.0, -2.0]), valid[:2], PP, D_CL, 0.0)
    assert cen[0, 0] == pytest.approx(0.5 * (p[7, 0] + p[8, 0]), rel=1e-15)
    assert csig[0] == -3.0


def test_coincidences():
    a = np.repeat(base_point()[None], 3, axis=0)
    b = np.repeat(base_point()[None], 2, axis=0)
    for e, k in enumerate((0, 10, 20)):
        a[e, 0] = (200.05 * 900.0 + k) / 900.0
    for e, k in enumerate((1, 30)):
        b[e, 0] = (200.05 * 900.0 + k) / 900.0
    out = pp_.coincidences(a, np.array([2.0, 1.0, 1.0]), b, np.array([2.0, 5.0]), PP, 3.0)
    assert [(i, j) for i, j, _, _ in out] == [(0, 0)]
    i, j, c, s = out[0]
    assert c[0] == pytest.approx(0.5 * (a[0, 0] + b[0, 0]), rel=1e-15) and s == 4.0


def test_ecliptic_projection():
    pole = np.array([0.0, -math.sin(OBL), math.cos(OBL)])
    x, y = pp_.ecliptic_xy(pole, OBL)
    assert abs(x[0]) < 1e-16 and abs(y[0]) < 1e-16
    lam = np.linspace(0, 2 * math.pi, 13)
    # points on the ecliptic, written in equatorial coordinates
    ecl = np.stack([np.cos(lam), np.sin(lam) * math.cos(OBL), np.sin(lam) * math.sin(OBL)], axis=1)
    x, y = pp_.ecliptic_xy(ecl, OBL)
    assert np.allclose(x * x + y * y, 1.0, rtol=1e-15)
    assert np.allclose(x, np.cos(lam), atol=1e-15) and np.allclose(y, np.sin(lam), atol=1e-15)
