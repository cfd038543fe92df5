"""Pins for the oracle's number count, significance (Eq. (25)), toplist and
power sum (Eq. (26)).

All-ones / all-zeros peakgrams, single-bit peakgrams (the count is 1 exactly
for the templates whose track hits that bit), linearity over disjoint
peakgrams, invariance under a permutation of the SFTs, the noise-only mean
p * sum(w), the Monte-Carlo mean and variance of s_H, an injected template
that collects every weight and ranks first, the toplist against a full
numpy sort, and the power sum against closed forms.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1904_04873_gb300 import synth
from _common import (P_TH, inject_on_track, oracle_dense_parallel, oracle_inputs, oracle_problem, pack_bits,
                     small_mid, template_of, track_bins)


@pytest.fixture(scope="module")
def prob():
    pr = small_mid()
    rho, bits, w = oracle_inputs(pr)
    return pr, rho, bits, w


def test_all_ones_and_all_zeros(prob):
    pr, rho, bits, w = prob
    ones = pack_bits(np.ones((pr.N, pr.K), bool), pr.W)
    d = oracle_problem(pr, ones, w).count_dense()
    assert np.all(d["n_unw"] == pr.N)
    sw = w.sum(axis=1)
    assert np.allclose(d["n_w"], sw[:, None, None], rtol=1e-13)
    d0 = oracle_problem(pr, np.zeros_like(ones), w).count_dense()
    assert np.all(d0["n_unw"] == 0) and np.all(d0["n_w"] == 0.0)


def test_single_bit_hits(prob):
    pr, rho, bits, w = prob
    rng = np.random.default_rng(31)
    for _ in range(3):
        i0 = int(rng.integers(pr.N))
        col0 = int(rng.integers(pr.K // 3, 2 * pr.K // 3))
        on = np.zeros((pr.N, pr.K), bool)
        on[i0, col0] = True
        d = oracle_problem(pr, pack_bits(on, pr.W), w).count_dense()
        expect = np.zeros_like(d["n_unw"])
        for s in range(pr.S):
            for b in range(pr.B):
                ap, Om, Ta = template_of(pr, b)
                for j in range(pr.n_f0):
                    k, _ = oracle.track_bin(pr.F0 + j, pr.v[i0], pr.sky[s], ap, Om, Ta, pr.t[i0])
                    expect[s, b, j] = int(k - pr.k_lo == col0)
        assert np.array_equal(d["n_unw"], expect)
        assert expect.sum() > 0
        assert np.allclose(d["n_w"], expect * w[:, i0][:, None, None])


def test_linearity_over_disjoint_peakgrams(prob):
    pr, rho, bits, w = prob
    rng = np.random.default_rng(32)
    on = rng.random((pr.N, pr.K)) < 0.3
    split = rng.random((pr.N, pr.K)) < 0.5
    a = oracle_problem(pr, pack_bits(on & split, pr.W), w).count_dense()
    b = oracle_problem(pr, pack_bits(on & ~split, pr.W), w).count_dense()
    c = oracle_problem(pr, pack_bits(on, pr.W), w).count_dense()
    assert np.array_equal(a["n_unw"] + b["n_unw"], c["n_unw"])
    assert np.allclose(a["n_w"] + b["n_w"], c["n_w"], rtol=1e-12)


def test_sft_permutation_invariance(prob):
    pr, rho, bits, w = prob
    perm = np.random.default_rng(33).permutation(pr.N)
    ref = oracle_problem(pr, bits, w).count_dense()
    op = oracle.OracleProblem(bits=bits[perm], w=w[:, perm], v=pr.v[perm], t=pr.t[perm], F0=pr.F0,
                              n_f0=pr.n_f0, sky=pr.sky, a_p=pr.a_p, Omega=pr.Omega, T_asc=pr.T_asc,
                              k_lo=pr.k_lo, K=pr.K)
    got = op.count_dense()
    assert np.array_equal(got["n_unw"], ref["n_unw"])
    assert np.allclose(got["n_w"], ref["n_w"], rtol=1e-12)


def test_noise_mean_count(prob):
    pr, rho, bits, w = prob
    d = oracle_problem(pr, bits, w).count_dense()
    sw = w.sum(axis=1)
    sw2 = (w * w).sum(axis=1)
    for s in range(pr.S):
        m = d["n_w"][s].mean()
        # templates share bits, so bound the spread by the single-template sigma
        assert abs(m - P_TH * sw[s]) < 5 * math.sqrt(P_TH * (1 - P_TH) * sw2[s])
    # over all sky points and templates the mean is much tighter
    tot = d["n_w"].mean()
    assert abs(tot - P_TH * sw.mean()) < 0.05 * P_TH * sw.mean()


def test_significance_monte_carlo():
    # n = sum_i w_i b_i with b_i ~ Bernoulli(exp(-1.6)): s_H has mean 0, variance 1.
    rng = np.random.default_rng(34)
    w = rng.uniform(0.2, 2.0, 300)
    b = rng.random((40000, 300)) < P_TH
    n = (b * w).sum(axis=1)
    s = oracle.significance(n, w.sum(), (w * w).sum())
    assert abs(s.mean()) < 5 / math.sqrt(s.size)
    assert abs(s.var() - 1.0) < 5 * math.sqrt(2.0 / s.size)


def test_injection_collects_all_weight_and_ranks_first():
    pr = synth.tiny()
    rho, bits, w = oracle_inputs(pr)
    inj = synth.TINY_INJECTION
    b_inj = (inj["Om_index"] * pr.T_asc.shape[1] + inj["T_index"]) * pr.a_p.size + inj["ap_index"]
    rho_i = inject_on_track(pr, pr.power, inj["sky"], b_inj, inj["f0_index"], inj["excess"])
    _, bits_i = oracle.peakgram(rho_i, 0, 1.6, W=pr.W)
    op = oracle_problem(pr, bits_i, w)
    c = op.count_one(inj["sky"], b_inj, inj["f0_index"])
    assert c["n_unw"] == pr.N
    assert abs(c["n_w"] - w[inj["sky"]].sum()) < 1e-9
    d = op.count_dense()
    sw, sw2 = w.sum(axis=1), (w * w).sum(axis=1)
    sH = oracle.significance(d["n_w"], sw[:, None, None], sw2[:, None, None])
    ids, _ = oracle.topk(sH.ravel(), 5)
    assert ids[0] == (inj["sky"] * pr.B + b_inj) * pr.n_f0 + inj["f0_index"]


def test_out_of_band_is_an_error(prob):
    pr, rho, bits, w = prob
    op = oracle.OracleProblem(bits=bits, w=w, v=pr.v, t=pr.t, F0=pr.F0, n_f0=pr.n_f0, sky=pr.sky,
                              a_p=pr.a_p, Omega=pr.Omega, T_asc=pr.T_asc, k_lo=pr.k_lo + 40, K=pr.K)
    with pytest.raises(ValueError):
        op.count_dense()


def test_topk_matches_full_sort():
    rng = np.random.default_rng(35)
    sc = np.round(rng.standard_normal(5000), 2)   # many exact ties
    ids, vals = oracle.topk(sc, 300)
    order = np.lexsort((np.arange(sc.size), -sc))[:300]
    assert np.array_equal(ids, order)
    assert np.array_equal(vals, sc[order])
    ids, _ = oracle.topk(sc[:10], 300)
    assert ids.size == 10


def test_power_sum_closed_forms(prob):
    pr, rho, bits, w = prob
    ones = np.ones((pr.N, pr.K), np.float32)
    op = oracle_problem(pr, bits, w, rho=ones)
    for (s, b, j) in [(0, 0, 0), (2, 5, 40), (5, pr.B - 1, pr.n_f0 - 1)]:
        assert abs(op.power_sum(s, b, j) - w[s].sum()) < 1e-10
    # rho = delta at one (SFT, bin): P = w_i if the track passes there, else 0
    s, b, j = 1, 3, 17
    ks, _ = track_bins(pr, s, b, j)
    i0 = 7
    delta = np.zeros((pr.N, pr.K), np.float32)
    delta[i0, ks[i0] - pr.k_lo] = 2.0
    op = oracle_problem(pr, bits, w, rho=delta)
    assert abs(op.power_sum(s, b, j) - 2.0 * w[s, i0]) < 1e-12
    # linearity in rho
    r1 = np.random.default_rng(36).exponential(size=(pr.N, pr.K)).astype(np.float32)
    r2 = np.random.default_rng(37).exponential(size=(pr.N, pr.K)).astype(np.float32)
    p1 = oracle_problem(pr, bits, w, rho=r1).power_sum(s, b, j)
    p2 = oracle_problem(pr, bits, w, rho=r2).power_sum(s, b, j)
    p12 = oracle_problem(pr, bits, w, rho=r1 + r2).power_sum(s, b, j)
    assert abs(p1 + p2 - p12) < 1e-7 * p12   # r1 + r2 is rounded to float32
    assert abs(oracle.power_significance(w[s].sum(), w[s].sum(), (w[s] ** 2).sum())) < 1e-15


def test_parallel_dense_equals_the_oracle_dense():
    # the process-sharded dense count used by the full-size GPU test splits only the work
    pr = small_mid(n_sky=5, n_per_det=40, n_ap=3, n_P=4, n_T=2)
    rho, bits, w = oracle_inputs(pr, "f16")
    ref = oracle_problem(pr, bits, w).count_dense(1, 5)
    got = oracle_dense_parallel(pr, bits, w, [1, 2, 3, 4], procs=2)
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k
    got = oracle_dense_parallel(pr, bits, w, [3], procs=2)
    for k in ref:
        assert np.array_equal(got[k][0], ref[k][2]), k
