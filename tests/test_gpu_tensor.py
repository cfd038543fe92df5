"""The tensor-core accumulation of the batched count (acc_mode 2, count_tc.cu).

The weighted and unweighted counts are a matrix product of the 0/1 peak matrix
(templates x SFTs) with the weights' fixed-point digits and a column of ones,
accumulated in FP32 on the tensor cores with no rounding.  So against the
oracle's FP64 sums of the same fp16 weights the weighted counts are the
correctly rounded FP32 values (within half an FP32 ulp, not merely within the
1e-5 bar), and the unweighted counts are exact outside the tie band; toplists
match the oracle's full sort.  Shapes: several SFT chunks with a ragged last
one, ragged binary tiles (64 binary templates per item), ragged f0 blocks,
both ways of forming the binary term, multi-problem batches, forced exact ties.
"""
import numpy as np
import pytest

from paper_1904_04873_gb300 import bsh, synth
from _common import small_mid
from gpu_common import check_dense, check_toplists, device_problem, oracle_scores

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HALF_ULP = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1904_04873_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def tc_plan(dps, top_k, chunk=0, direct=0):
    plan = bsh.Plan(dps, bsh.MODE_BATCHED, top_k=top_k, threads=256, sft_chunk=chunk)
    plan.set_direct(direct)
    plan.set_accumulate(2)
    t = plan.tile()
    assert t["accumulate"] == 2 and t["direct"] == direct and t["threads"] == 256
    return plan


def check_rounded(gw, d):
    """Weighted counts equal the oracle's FP64 sums rounded once to FP32 (ties excluded)."""
    gw = gw.cpu().numpy().astype(np.float64)
    notie = d["n_tie"] == 0
    ref = d["n_w"]
    err = np.abs(gw - ref)
    assert np.all(err[notie] <= HALF_ULP * np.abs(ref[notie]) + 1e-30), \
        f"max rel err {np.max(err[notie] / np.maximum(np.abs(ref[notie]), 1e-30)):.3e}"


@pytest.mark.parametrize("direct", [0, 1])
@pytest.mark.parametrize("chunk", [64, 128])
def test_tensor_dense_counts(direct, chunk):
    # 2 x 170 SFTs (ragged last chunk), 100 binaries (two 64-template tiles, the second ragged),
    # 90 f0 in three blocks of 30, 5 sky points in 2 patches
    pr = small_mid(n_sky=5, n_per_det=170, n_ap=5, n_P=5, n_T=4, patch_size=3, top_k=50)
    dp, op, wq = device_problem(pr, "f16")
    plan = tc_plan([dp], pr.top_k, chunk, direct)
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    d = op.count_dense()
    check_dense(gu[0], gw[0], d)
    check_rounded(gw[0], d)
    plan.number_count()
    assert bsh.sync_status() == bsh.OK
    _, sc = oracle_scores(op, wq)
    by_patch = [sc[pr.patch_start[p]:pr.patch_start[p + 1]] for p in range(len(pr.patch_start) - 1)]
    check_toplists(plan, dp, 0, by_patch, pr.top_k, tol=2e-4)
    plan.close()


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_tensor_other_weight_dtypes(dtype):
    # weights other than fp16 enter in fixed point with a 2^-24 quantum: within the 1e-5 bar
    pr = small_mid(n_sky=3, n_per_det=100, n_ap=4, n_P=3, n_T=3, patch_size=3, top_k=20)
    dp, op, wq = device_problem(pr, dtype)
    plan = tc_plan([dp], pr.top_k)
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    check_dense(gu[0], gw[0], op.count_dense())
    plan.close()


def test_tensor_multi_problem_batch_and_stage2():
    probs = synth.batching(n_patch=3, size_lo=2, size_hi=4, n_per_det=70, n_bin=5)
    for p in probs:
        p.n_f0 = 40
    dps = [device_problem(p, "f16") for p in probs]
    plan = tc_plan([d[0] for d in dps], 15, direct=1)
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    for q, (dp, op, wq) in enumerate(dps):
        d = op.count_dense()
        check_dense(gu[q], gw[q], d)
        check_rounded(gw[q], d)
    plan.number_count()
    cands, n = plan.toplist()
    plan.power_sum(5)
    assert bsh.sync_status() == bsh.OK
    for q, (dp, op, wq) in enumerate(dps):
        _, sc = oracle_scores(op, wq)
        pr = dp.pr
        by_patch = [sc[pr.patch_start[p]:pr.patch_start[p + 1]] for p in range(len(pr.patch_start) - 1)]
        check_toplists(plan, dp, q, by_patch, 15, tol=2e-4)
    plan.close()


def test_tensor_forced_exact_ties():
    pr = synth.precision_stress(n_sky=4, n_per_det=100, n_ap=4, n_P=3, n_T=3)
    dp, op, wq = device_problem(pr, "f32")
    plan = tc_plan([dp], 10)
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    d = op.count_dense()
    assert np.array_equal(gu[0].cpu().numpy()[0, ::4], d["n_unw"][0, ::4])
    check_dense(gu[0], gw[0], d)
    plan.close()


def test_tensor_graph_replay_matches_eager():
    pr = small_mid(n_sky=6, n_per_det=150, n_ap=4, n_P=3, n_T=3, patch_size=3, top_k=40)
    dp, op, wq = device_problem(pr, "f16")
    plan = tc_plan([dp], pr.top_k)
    plan.number_count()
    c1, n1 = plan.toplist()
    f1, nf1 = plan.power_sum(8)
    ref = (c1.clone(), n1.clone(), f1.clone(), nf1.clone())
    for _ in range(3):
        f2, nf2 = plan.graph_launch(8)
    assert bsh.sync_status() == bsh.OK
    assert torch.equal(plan.cands, ref[0]) and torch.equal(plan.n_cands, ref[1])
    assert torch.equal(f2, ref[2]) and torch.equal(nf2, ref[3])
    plan.close()
