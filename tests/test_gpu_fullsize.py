"""Full-size parity on the benchmark workload (mid: 2 x 2000 SFTs, 2000 sky
points in 40 patches, 32^3 binary templates, 90 f0 bins, top-1000), in the
launch configuration bench.py times (autotuned batched plan), end to end (the
GPU forms the peakgram and the weights itself; they must equal the oracle's),
and on the shapes of the other workloads (full scale with stage 2, multi-band
batching, the eccentric grid, a metric template bank).

The oracle cannot count all 5.9e9 templates.  It counts two whole sky points
densely (2 x 32768 x 90 templates over all 4000 SFTs, in spawned processes),
compared element by element with the kernel's dense counts in the same tile
shape, and their toplist with the oracle's full sort; and it recomputes
sampled outputs of the full run one template at a time: toplist entries
(counts, s_H, P), random templates outside the lists, whose oracle s_H must
not exceed the list's k-th score (the toplist property), and, for the two
densely counted sky points, every template of theirs above that k-th score.
"""
import numpy as np
import pytest

import oracle
from paper_1904_04873_gb300 import bsh, synth
from _common import oracle_dense_parallel
from gpu_common import REL_TOL, check_dense, check_toplists, device_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def run():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1904_04873_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    pr = synth.mid()
    # end to end: the GPU forms the peakgram, rho and fp16 weights from the raw inputs
    dp, op, wq = device_problem(pr, "f16", oracle_fed=False)
    assert bsh.sync_status() == bsh.OK
    assert np.array_equal(dp.bits.cpu().numpy().view(np.uint32), op.bits)
    assert np.array_equal(dp.rho.cpu().numpy(), op.rho)
    assert np.array_equal(dp.w.double().cpu().numpy(), wq)
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    tile = plan.autotune()
    plan.number_count()
    cands, n = plan.toplist()
    plan.power_sum(100)
    assert bsh.sync_status() == bsh.OK
    lists = bsh.cands_to_numpy(cands, n)
    plan.close()
    return pr, op, wq, lists, tile


DENSE_SKY = [0, 1]


@pytest.fixture(scope="module")
def dense(run):
    """The oracle's dense counts of sky points 0 and 1 at full size, with their s_H."""
    pr, op, wq, _, _ = run
    d = oracle_dense_parallel(pr, op.bits, wq, DENSE_SKY)
    sw = wq[DENSE_SKY].sum(axis=1)
    sw2 = (wq[DENSE_SKY] ** 2).sum(axis=1)
    p = np.exp(-pr.rho_th)
    sc = (d["n_w"] - p * sw[:, None, None]) / np.sqrt(p * (1 - p) * sw2)[:, None, None]
    return d, sc


def test_dense_slice_full_size(run, dense):
    # sky points 0 and 1 at the full B x F x N of the bench workload, searched as one patch by
    # a plan in the bench's tile shape; every count against the oracle, then the patch's
    # toplist against the oracle's full sort of all 5.9e6 scores
    pr, op, wq, _, tile = run
    d, sc = dense
    sub = synth.mid(sky=pr.sky[DENSE_SKY], patch_size=len(DENSE_SKY))
    dp = bsh.DeviceProblem(sub, w_dtype="f16")
    dp.prepare()
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k, threads=tile["threads"], sft_chunk=tile["sft_chunk"])
    plan.set_direct(tile["direct"])
    plan.set_accumulate(tile["accumulate"])
    t = plan.tile()
    assert (t["threads"], t["sft_chunk"], t["direct"], t["accumulate"]) == \
        (tile["threads"], tile["sft_chunk"], tile["direct"], tile["accumulate"])
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    check_dense(gu[0], gw[0], d)
    plan.number_count()
    check_toplists(plan, dp, 0, [sc], pr.top_k, 2e-4)
    assert bsh.sync_status() == bsh.OK
    plan.close()


def test_full_run_toplist_complete_on_dense_sky_points(run, dense):
    # patch 0 of the full run holds sky points 0-49: every template of sky points 0 and 1 whose
    # oracle s_H clears the list's k-th score by the score tolerance is in the list, and every
    # list entry of theirs has the oracle's counts
    pr, op, wq, lists, _ = run
    d, sc = dense
    g = lists[0]
    kth = float(g["s_h"][-1])
    per_s = pr.B * pr.n_f0
    in_list = {int(x) for x in g["template_id"]}
    for k, s in enumerate(DENSE_SKY):
        above = np.flatnonzero(sc[k].ravel() > kth + 2e-4)
        missing = [int(x) for x in above if s * per_s + int(x) not in in_list]
        assert not missing, (s, missing[:5])
    for c in g:
        s, rem = divmod(int(c["template_id"]), per_s)
        if s not in DENSE_SKY:
            continue
        k = DENSE_SKY.index(s)
        b, j = divmod(rem, pr.n_f0)
        assert d["unw_lo"][k, b, j] <= int(c["n_unw"]) <= d["unw_hi"][k, b, j]
        assert abs(float(c["n_w"]) - d["n_w"][k, b, j]) <= REL_TOL * d["n_w"][k, b, j]
        assert abs(float(c["s_h"]) - sc[k, b, j]) < 2e-4


def _score(op, wq, s, b, j):
    c = op.count_one(s, b, j)
    sH = oracle.significance(c["n_w"], wq[s].sum(), (wq[s] ** 2).sum())
    return c, float(sH)


def test_sampled_toplist_entries(run):
    pr, op, wq, lists, _ = run
    rng = np.random.default_rng(8)
    per_s = pr.B * pr.n_f0
    patches = [0, len(lists) - 1] + list(rng.choice(len(lists), 2, replace=False))
    for p in patches:
        g = lists[p]
        assert g.size == pr.top_k
        assert np.all(np.diff(g["s_h"]) <= 0)
        pick = list(range(10)) + list(rng.choice(np.arange(10, g.size), 20, replace=False))
        for e in pick:
            c = g[e]
            s, rem = divmod(int(c["template_id"]), per_s)
            b, j = divmod(rem, pr.n_f0)
            assert pr.patch_start[p] <= s < pr.patch_start[p + 1]
            ref, sH = _score(op, wq, s, b, j)
            assert ref["unw_lo"] <= int(c["n_unw"]) <= ref["unw_hi"]
            assert abs(float(c["n_w"]) - ref["n_w"]) <= REL_TOL * ref["n_w"]
            assert abs(float(c["s_h"]) - sH) < 2e-4
            if e < 10:
                P = op.power_sum(s, b, j) if op.rho is not None else None
                if P is not None:
                    assert abs(float(c["power"]) - P) <= REL_TOL * P


def test_random_templates_respect_the_kth_score(run):
    pr, op, wq, lists, _ = run
    rng = np.random.default_rng(9)
    per_s = pr.B * pr.n_f0
    for p in rng.choice(len(lists), 3, replace=False):
        g = lists[p]
        kth = float(g["s_h"][-1])
        ids = set(int(x) for x in g["template_id"])
        s0, s1 = pr.patch_start[p], pr.patch_start[p + 1]
        for _ in range(150):
            s = int(rng.integers(s0, s1))
            b = int(rng.integers(pr.B))
            j = int(rng.integers(pr.n_f0))
            tid = (s * pr.B + b) * pr.n_f0 + j
            if tid in ids:
                continue
            _, sH = _score(op, wq, s, b, j)
            assert sH <= kth + 2e-4, (p, s, b, j, sH, kth)


def _sampled_check(pr, op, wq, lists, first_region, rng, n_patch_check=2, n_entries=25, n_random=100):
    per_s = pr.B * pr.n_f0
    n_patch = len(pr.patch_start) - 1
    for p in rng.choice(n_patch, min(n_patch_check, n_patch), replace=False):
        g = lists[first_region + p]
        s0, s1 = pr.patch_start[p], pr.patch_start[p + 1]
        assert g.size == min(pr.top_k, (s1 - s0) * per_s)
        assert np.all(np.diff(g["s_h"]) <= 0)
        for e in list(range(5)) + list(rng.choice(np.arange(5, g.size), n_entries - 5, replace=False)):
            c = g[e]
            s, rem = divmod(int(c["template_id"]), per_s)
            b, j = divmod(rem, pr.n_f0)
            assert s0 <= s < s1
            ref, sH = _score(op, wq, s, b, j)
            assert ref["unw_lo"] <= int(c["n_unw"]) <= ref["unw_hi"]
            assert abs(float(c["n_w"]) - ref["n_w"]) <= REL_TOL * ref["n_w"]
            assert abs(float(c["s_h"]) - sH) < 2e-4
            P = op.power_sum(s, b, j)
            assert abs(float(c["power"]) - P) <= REL_TOL * P
        kth = float(g["s_h"][-1])
        ids = set(int(x) for x in g["template_id"])
        for _ in range(n_random):
            s = int(rng.integers(s0, s1))
            b = int(rng.integers(pr.B))
            j = int(rng.integers(pr.n_f0))
            if (s * pr.B + b) * pr.n_f0 + j in ids:
                continue
            _, sH = _score(op, wq, s, b, j)
            assert sH <= kth + 2e-4


def test_full_scale_shape_with_stage2():
    # config-5 shape: 2 x 4000 SFTs over 1 yr, 9000 f0 bins at 300 Hz, 8^3 binaries, patches of
    # 169 sky points, top-10000, stage-2 power sums; 6 patches of the sky (rho given directly)
    pr = synth.full(n_sky=1014, power_kind="exp")
    dp, op, wq = device_problem(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    plan.autotune()
    plan.number_count()
    cands, n = plan.toplist()
    plan.power_sum(1000)
    assert bsh.sync_status() == bsh.OK
    lists = bsh.cands_to_numpy(cands, n)
    plan.close()
    _sampled_check(pr, op, wq, lists, 0, np.random.default_rng(11))


def test_batching_shape_multi_band():
    # config-3 shape: four 1 Hz bands (T_c = 900/600/450/360 s), 2 x 500 SFTs each, 8^3 binaries,
    # uneven patches; one persistent launch over all bands
    probs = synth.batching(n_patch=4, size_lo=20, size_hi=60, power_kind="exp")
    dps = [device_problem(p, "f16") for p in probs]
    plan = bsh.Plan([d[0] for d in dps], bsh.MODE_BATCHED, top_k=1000)
    plan.autotune()
    plan.number_count()
    cands, n = plan.toplist()
    plan.power_sum(100)
    assert bsh.sync_status() == bsh.OK
    lists = bsh.cands_to_numpy(cands, n)
    rng = np.random.default_rng(12)
    for q, (dp, op, wq) in enumerate(dps):
        _sampled_check(dp.pr, op, wq, lists, plan.first_region(q), rng, n_patch_check=1, n_entries=15,
                       n_random=40)
    plan.close()


def test_eccentric_workload_shape():
    # the eccentric bench workload's construction (16^3 x 3 x 3 ELL1 grid), 4 patches of its sky
    pr = synth.eccentric(n_sky=200, patch_size=50)
    dp, op, wq = device_problem(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    plan.autotune()
    plan.number_count()
    cands, n = plan.toplist()
    plan.power_sum(100)
    assert bsh.sync_status() == bsh.OK
    lists = bsh.cands_to_numpy(cands, n)
    plan.close()
    _sampled_check(pr, op, wq, lists, 0, np.random.default_rng(13), n_patch_check=2, n_entries=20, n_random=60)


def test_metric_bank_workload_shape():
    # the metric experiment's bank (a_p 3-13 ls, P 10-20 d, mismatch 6.4, one a_p block per Omega)
    from oracle import bank as obank
    pr = synth.metric(n_sky=150, patch_size=50)
    pr = synth.attach_bank(pr, *obank.template_bank(**synth.metric_spec(pr, m=6.4)))
    dp, op, wq = device_problem(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    plan.autotune()
    plan.number_count()
    cands, n = plan.toplist()
    plan.power_sum(100)
    assert bsh.sync_status() == bsh.OK
    lists = bsh.cands_to_numpy(cands, n)
    plan.close()
    _sampled_check(pr, op, wq, lists, 0, np.random.default_rng(14), n_patch_check=2, n_entries=20, n_random=60)
