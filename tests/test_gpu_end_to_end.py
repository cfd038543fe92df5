"""End to end on the GPU against an oracle that computes every step itself.

The GPU path takes the raw inputs (SFT powers, detector arms and velocities,
noise levels, sky and binary grids) and runs every step of the hot path in its
kernels: peakgram and rho (Sec. IV.A, Eq. (20)-(21)), weights (Eq. (22))
quantised to the stored dtype, the FP64 track tables, the number count
(Sec. IV.C, Eq. (15), (25)), the fused toplist, the stage-2 power sum
(Eq. (26)) and the re-rank.  The oracle computes its own peakgram, rho and
weights from the same raw inputs and its own counts from those; nothing is
copied from one side to the other.

Bar: peakgram bits, rho and quantised weights bit-exact (both sides evaluate
the same definitions in the same order, each operation rounded on its own);
unweighted counts exact outside the oracle's tie band; weighted counts and
power sums within 1e-5 relative of the oracle's FP64 sums; toplists equal to
the oracle's full sort up to entries within the score error of the k-th.
"""
import numpy as np
import pytest

import oracle
from paper_1904_04873_gb300 import bsh, synth
from _common import oracle_inputs, oracle_problem, small_mid
from gpu_common import REL_TOL, check_dense, check_toplists, oracle_scores

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1904_04873_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _gpu_and_oracle(pr, dtype):
    """The GPU's own inputs (prepare() from the raw arrays) and the oracle's own, checked equal."""
    dp = bsh.DeviceProblem(pr, w_dtype=dtype)
    dp.prepare()
    assert bsh.sync_status() == bsh.OK
    orho, obits, ow = oracle_inputs(pr, dtype)
    assert np.array_equal(dp.bits.cpu().numpy().view(np.uint32), obits)
    assert np.array_equal(dp.rho.cpu().numpy(), orho)
    assert np.array_equal(dp.w.double().cpu().numpy(), ow)
    return dp, oracle_problem(pr, obits, ow, rho=orho), ow


def _patches(pr, sc):
    return [sc[pr.patch_start[p]:pr.patch_start[p + 1]] for p in range(len(pr.patch_start) - 1)]


def _check_stage2(pr, op, ow, cands, n, final, nf, n_cf):
    lists = bsh.cands_to_numpy(cands, n)
    per_s = pr.B * pr.n_f0
    for g in lists:
        for c in g:
            s, rem = divmod(int(c["template_id"]), per_s)
            b, j = divmod(rem, pr.n_f0)
            P = op.power_sum(s, b, j)
            assert abs(float(c["power"]) - P) <= REL_TOL * P
            sP = oracle.power_significance(P, ow[s].sum(), (ow[s] ** 2).sum())
            assert abs(float(c["s_p"]) - sP) < 1e-4
    for g, f in zip(lists, bsh.cands_to_numpy(final, nf)):
        assert f.size == min(n_cf, g.size)
        order = np.lexsort((g["template_id"], -g["s_p"].astype(np.float64)))[:n_cf]
        assert np.array_equal(f["template_id"], g["template_id"][order])


@pytest.mark.parametrize("dtype", ["f16", "bf16", "f32"])
def test_end_to_end_batched(dtype):
    # the mid construction at reduced size: 2 x 300 SFTs (five 128-SFT stages, the last
    # ragged), 60 binary templates (a ragged tile), 90 f0 (three blocks of 30), 6 sky points
    # in 2 patches, Gaussian-noise powers through the running median
    pr = small_mid(n_sky=6, n_per_det=300, n_ap=5, n_P=4, n_T=3, patch_size=3, top_k=60)
    dp, op, ow = _gpu_and_oracle(pr, dtype)
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    d, sc = oracle_scores(op, ow)
    check_dense(gu[0], gw[0], d)
    plan.number_count()
    check_toplists(plan, dp, 0, _patches(pr, sc), pr.top_k, tol=2e-4)
    cands, n = plan.toplist()
    final, nf = plan.power_sum(12)
    assert bsh.sync_status() == bsh.OK
    _check_stage2(pr, op, ow, cands, n, final, nf, 12)
    plan.close()


def test_end_to_end_graph_step():
    # the captured step (count, toplist, stage 2 in one CUDA graph) after prepare(), twice
    pr = small_mid(n_sky=8, n_per_det=200, n_ap=6, n_P=3, n_T=3, patch_size=4, top_k=40)
    dp, op, ow = _gpu_and_oracle(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    _, sc = oracle_scores(op, ow)
    for _ in range(2):
        dp.prepare()
        final, nf = plan.graph_launch(10)
        assert bsh.sync_status() == bsh.OK
        _check_stage2(pr, op, ow, plan.cands, plan.n_cands, final, nf, 10)
        check_toplists(plan, dp, 0, _patches(pr, sc), pr.top_k, tol=2e-4)   # (merges again)
    plan.close()


def test_end_to_end_plain_fp64():
    # the plain form with FP64 weights formed on the GPU: the weighted sums follow the oracle's
    # order (SFTs ascending, FP64), so they are exact
    pr = small_mid(n_sky=4, n_per_det=150, n_ap=4, n_P=3, n_T=3, patch_size=2, top_k=30)
    dp, op, ow = _gpu_and_oracle(pr, "f64")
    plan = bsh.Plan([dp], bsh.MODE_PLAIN, top_k=pr.top_k)
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    d, sc = oracle_scores(op, ow)
    check_dense(gu[0], gw[0], d, exact_w=True)
    plan.number_count()
    check_toplists(plan, dp, 0, _patches(pr, sc), pr.top_k, tol=2e-4)
    plan.close()


def test_end_to_end_injection_tiny():
    # the tiny workload with its injected binary: GPU path from the raw powers, the oracle's
    # own inputs; the injected template collects every SFT and heads its patch after stage 2
    pr = synth.tiny()
    inj = synth.TINY_INJECTION
    n_ap, n_T = pr.a_p.size, pr.T_asc.shape[1]
    b_inj = (inj["Om_index"] * n_T + inj["T_index"]) * n_ap + inj["ap_index"]
    ap, Om, Ta = pr.a_p[inj["ap_index"]], pr.Omega[inj["Om_index"]], pr.T_asc[inj["Om_index"], inj["T_index"]]
    rho = pr.power.copy()
    for i in range(pr.N):
        k, _ = oracle.track_bin(pr.F0 + inj["f0_index"], pr.v[i], pr.sky[inj["sky"]], ap, Om, Ta, pr.t[i])
        rho[i, k - pr.k_lo] += np.float32(inj["excess"])
    pr.power = rho
    dp, op, ow = _gpu_and_oracle(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    plan.number_count()
    cands, n = plan.toplist()
    final, nf = plan.power_sum(10)
    assert bsh.sync_status() == bsh.OK
    want = (inj["sky"] * pr.B + b_inj) * pr.n_f0 + inj["f0_index"]
    top = bsh.cands_to_numpy(cands, n)[0]
    assert int(top[0]["template_id"]) == want and int(top[0]["n_unw"]) == pr.N
    assert abs(float(top[0]["n_w"]) - ow[inj["sky"]].sum()) <= REL_TOL * ow[inj["sky"]].sum()
    assert int(bsh.cands_to_numpy(final, nf)[0][0]["template_id"]) == want
    _check_stage2(pr, op, ow, cands, n, final, nf, 10)
    _, sc = oracle_scores(op, ow)
    check_toplists(plan, dp, 0, _patches(pr, sc), pr.top_k, tol=2e-4)
    plan.close()
