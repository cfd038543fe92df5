"""The batched kernels' pooled walk over the item list, against the FP64 oracle.

Items are ordered sky point, binary tile, f0 block.  CTAs c + m C/4 (m < 4) share a pool: a
contiguous range of items that they take one at a time, in the pool's walk order.  A pool
holding more than one sky point's items (P of them) walks them in sweeps of P, each started at
the first binary tile of the next sky point and wrapped round.  These problems have few items
per sky point and many sky points, so most pools walk rotated sweeps: every item must still be
counted exactly once (dense counts), a range that holds a sky-patch boundary meets the two
patches in turn (up to four runs, each with one toplist visit per CTA of the pool), and the
visits must merge to the oracle's per-patch toplists, the same on every launch however the
pool's CTAs split the items.
"""
import dataclasses
import math

import numpy as np
import pytest

from _common import oracle_dense_parallel, small_mid
from gpu_common import check_dense, check_toplists, device_problem, oracle_scores
from paper_1904_04873_gb300 import bsh, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1904_04873_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _sky_many(patch_size):
    # 400 sky points, 64 SFTs, 8 binaries (one tile), 90 f0 templates (3 blocks of 30):
    # P = 3 items per sky point, 1200 items over at most 304 CTAs (76 pools)
    return small_mid(n_sky=400, n_per_det=32, n_ap=2, n_P=2, n_T=2, patch_size=patch_size, top_k=20)


@pytest.fixture(scope="module", params=[3, 1, 7], ids=lambda p: f"patch{p}")
def many_sky(request):
    pr = _sky_many(request.param)
    dp, op, wq = device_problem(pr, "f16")
    return pr, dp, op, wq


def _pool_ranges_exceed_sweep(pr, plan):
    tile = plan.tile()
    tb = 64 if tile["accumulate"] == 2 else tile["threads"]
    P = math.ceil(pr.B / tb) * math.ceil(pr.n_f0 / 32)   # f0 blocks of at most 32 templates
    items = pr.S * P
    assert 2 * items / tile["ctas"] > P, "sizes must give pool ranges longer than one sky point"


@pytest.mark.parametrize("acc", [0, 1, 2])
def test_dense_counts_every_item_once(many_sky, acc):
    pr, dp, op, _ = many_sky
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k, threads=256)
    plan.set_direct(0)
    plan.set_accumulate(acc)
    assert plan.tile()["accumulate"] == acc
    _pool_ranges_exceed_sweep(pr, plan)
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    check_dense(gu[0], gw[0], op.count_dense())
    plan.close()


@pytest.mark.parametrize("acc", [0, 2])
def test_toplists_merge_over_revisited_patches(many_sky, acc):
    pr, dp, op, wq = many_sky
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k, threads=256)
    plan.set_accumulate(acc)
    _pool_ranges_exceed_sweep(pr, plan)
    plan.number_count()
    assert bsh.sync_status() == bsh.OK
    _, sc = oracle_scores(op, wq)
    by_patch = [sc[pr.patch_start[p]:pr.patch_start[p + 1]] for p in range(len(pr.patch_start) - 1)]
    check_toplists(plan, dp, 0, by_patch, pr.top_k, tol=2e-4)
    plan.close()


def test_pooled_ctas_give_the_same_toplists_every_launch(many_sky):
    # the CTAs of a pool split its items differently from launch to launch (whichever takes
    # the next item first); the toplists (sorted by score, then template id) must not
    pr, dp, _, _ = many_sky
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k, threads=256)
    first = None
    for _ in range(4):
        plan.number_count()
        cands, n = plan.toplist()
        assert bsh.sync_status() == bsh.OK
        lists = bsh.cands_to_numpy(cands, n)
        got = [(l["template_id"].copy(), l["s_h"].copy()) for l in lists]
        if first is None:
            first = got
            continue
        for (ia, sa), (ib, sb) in zip(first, got):
            assert np.array_equal(ia, ib) and np.array_equal(sa, sb)
    plan.close()


def test_pairs_for_a_large_orbit_table_count_every_item_once():
    # 4 200 orbit rows (70 Omega x 60 t_asc, one a_p) over 2 x 2 048 SFTs: a 69 MB fixed-point
    # orbit table, more than half the L2, so the plan pools its CTAs in pairs (visits 2j + m);
    # two sky points in patches of one, 32 f0 templates: 1.1e9 terms for the oracle
    pr = synth.mid(n_sky=2, n_per_det=2048, n_ap=1, n_P=70, n_T=60, patch_size=1, top_k=20)
    pr = dataclasses.replace(pr, n_f0=32)
    dp, op, wq = device_problem(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    assert bsh.debug_pool_walk(plan.h)[1] == 2
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    d = oracle_dense_parallel(pr, op.bits, wq, [0, 1])
    check_dense(gu[0], gw[0], d)
    plan.number_count()
    assert bsh.sync_status() == bsh.OK
    p = math.exp(-pr.rho_th)
    sw, sw2 = wq.sum(axis=1), (wq * wq).sum(axis=1)
    sc = (d["n_w"] - p * sw[:, None, None]) / np.sqrt(p * (1 - p) * sw2)[:, None, None]
    check_toplists(plan, dp, 0, [sc[0:1], sc[1:2]], pr.top_k, tol=2e-4)
    plan.close()
