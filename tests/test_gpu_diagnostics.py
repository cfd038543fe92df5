"""Track diagnostics and the precision-stress experiment on the GPU.

The fixed-point bins of the batched kernels agree with the exact FP64 bins
for every term outside the tie band, while the same expression evaluated in
single precision disagrees (f T_c ~ 1e5 bins leaves FP32 with 1/64-bin
resolution).  The exact bins of listed templates equal the oracle's.
"""
import numpy as np
import pytest

import oracle
from paper_1904_04873_gb300 import bsh, experiments, synth
from _common import template_of

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1904_04873_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def test_fixed_point_bins_match_fp64_single_precision_does_not():
    pr = synth.mid(n_sky=40, n_per_det=400, n_ap=16, n_P=8, n_T=8)
    dp = bsh.DeviceProblem(pr, w_dtype="f16")
    dp.prepare()
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=10)
    terms, single, fixed, ties = plan.track_precision(0, 0, 8)
    assert bsh.sync_status() == bsh.OK
    assert terms == 8 * pr.B * pr.N * pr.n_f0
    assert fixed == 0
    assert single > terms // 1000          # single precision flips bins
    plan.close()


def test_forced_ties_are_in_the_tie_band():
    pr = synth.precision_stress(n_sky=16, n_per_det=100, n_ap=4, n_P=3, n_T=3)
    dp = bsh.DeviceProblem(pr, w_dtype="f16")
    dp.prepare()
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=10)
    terms, single, fixed, ties = plan.track_precision(0, 0, 1)     # the pole
    assert bsh.sync_status() == bsh.OK
    # a_p = 0 templates (1 in 4) at the pole sit exactly on ties in every SFT and f0
    assert ties >= terms // 4
    assert fixed == 0
    plan.close()


def test_track_bins_equal_oracle():
    pr = synth.mid(n_sky=12, n_per_det=100, n_ap=4, n_P=4, n_T=4)
    dp = bsh.DeviceProblem(pr, w_dtype="f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=10)
    rng = np.random.default_rng(3)
    ids = rng.integers(0, pr.n_templates, 20)
    bins = plan.track_bins(torch.as_tensor(ids, device="cuda")).cpu().numpy()
    assert bsh.sync_status() == bsh.OK
    per_s = pr.B * pr.n_f0
    for q, tid in enumerate(ids):
        s, rem = divmod(int(tid), per_s)
        b, j = divmod(rem, pr.n_f0)
        ap, Om, Ta = template_of(pr, b)
        for i in range(0, pr.N, 7):
            k, tie = oracle.track_bin(pr.F0 + j, pr.v[i], pr.sky[s], ap, Om, Ta, pr.t[i])
            assert tie or bins[q, i] == k
    plan.close()


def test_precision_experiment_small():
    r = experiments.precision(n_sky=40, n_sky_terms=1, n_sky_dense=2)
    assert r["tracks"]["sample"]["fixed_point_mismatch_outside_tie_band"] == 0
    assert r["tracks"]["sky0"]["tie_band_terms"] > 0
    for dt in ("f32", "f16", "bf16"):
        e = r["weights"][dt]
        assert e["accumulation_max_rel_err"] < 1e-5
        assert e["unweighted_equal_to_plain"]
    assert r["weights"]["f32"]["quantisation_max_rel_err_vs_f64_weights"] < 1e-6
    assert r["weights"]["bf16"]["quantisation_rms_rel_err_vs_f64_weights"] > \
        r["weights"]["f16"]["quantisation_rms_rel_err_vs_f64_weights"]
