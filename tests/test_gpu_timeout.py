"""Failure detection of the batched count: a bounded staging wait that expires.

The batched kernel stages each SFT chunk through a shared-memory buffer and
waits on a barrier for its copies.  bsh_plan_set_wait's test hook leaves one
stage per CTA unissued, so nothing ever completes that barrier phase (a flag
that nothing sets): every CTA's wait on it gives up after the poll limit, the
kernel records BSH_ERR_TIMEOUT, waits (bounded) for the copies it still has in
flight, frees its tensor memory and returns.  Nothing faults or hangs; the
context stays usable, and the next launch on the same plan -- which needs the
tensor memory back -- counts exactly as the oracle does.
"""
import numpy as np
import pytest

from paper_1904_04873_gb300 import bsh
from _common import small_mid
from gpu_common import check_dense, check_toplists, device_problem, oracle_scores

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1904_04873_gb300 import build
    build.build()
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def prob():
    # 2 x 300 SFTs: five 128-SFT stages per item (ten of 64), so every CTA with work has them
    pr = small_mid(n_sky=6, n_per_det=300, n_ap=5, n_P=4, n_T=3, patch_size=3, top_k=40)
    dp, op, wq = device_problem(pr, "f16")
    d, sc = oracle_scores(op, wq)
    return pr, dp, d, sc


@pytest.mark.parametrize("threads,direct,acc", [(256, 0, 0), (128, 0, 0), (256, 1, 0), (256, 0, 2), (256, 1, 2)])
def test_expired_wait_reports_timeout_then_recovers(prob, threads, direct, acc):
    # acc 2: the tensor-core kernel, whose exit path also waits for its MMAs in flight
    pr, dp, d, sc = prob
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k, threads=threads, sft_chunk=128)
    plan.set_direct(direct)
    plan.set_accumulate(acc)
    assert plan.tile()["accumulate"] == acc
    chunk = plan.tile()["sft_chunk"]          # 128, or 64 where the shared memory asks for it
    stages = -(-pr.N // chunk)                # stages of a CTA's first item
    assert stages >= 5
    for skip in (1, 0, stages - 1):           # a middle stage, the first, the item's last
        plan.set_wait(polls=1 << 14, skip_stage=skip)
        plan.number_count()
        assert bsh.sync_status() == bsh.ERR_TIMEOUT
        assert bsh.sync_status() == bsh.OK      # the status word was cleared
    # the default limit and no skipped stage: the same plan counts as the oracle does
    plan.set_wait(0, -1)
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    check_dense(gu[0], gw[0], d)
    plan.number_count()
    assert bsh.sync_status() == bsh.OK
    by_patch = [sc[pr.patch_start[p]:pr.patch_start[p + 1]] for p in range(len(pr.patch_start) - 1)]
    check_toplists(plan, dp, 0, by_patch, pr.top_k, tol=2e-4)
    plan.close()


def test_skip_past_the_last_stage_changes_nothing(prob):
    # a stage number that no CTA reaches: every copy is issued and the count completes
    pr, dp, d, _ = prob
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k, sft_chunk=128)
    plan.set_wait(polls=0, skip_stage=1 << 20)
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    check_dense(gu[0], gw[0], d)
    plan.close()
