"""The batched schedule on the host (no GPU): pools, walks and their alignment.

bsh_plan_create builds the schedule without touching a GPU; bsh_debug_pool_walk returns each
pool's item order.  Items of a problem run sky point, binary tile, f0 block, so item i sits at
offset i mod P of its sky point, P = (binary tiles) x (f0 blocks).  The properties checked:
every item is in exactly one pool and each pool's walk is a permutation of a contiguous range;
in its whole sweeps a pool is at offset k mod P at step k, so all pools meet a binary tile
together; in the last, partial sweep the pools sit on at most ceil(P / m) + 2 offsets at any
step (m the sweep's length); and a plan uses pools of four CTAs unless its fixed-point orbit
table (rows x SFTs padded to 256 x 4 bytes) exceeds half the L2.
"""
import math

import numpy as np
import pytest

from paper_1904_04873_gb300 import bsh, synth
from test_abi_host import FakeProblem, create


def _walks(h):
    n_pools, psize, _ = bsh.debug_pool_walk(h)
    return n_pools, psize, [bsh.debug_pool_walk(h, q)[2] for q in range(n_pools)]


@pytest.fixture(scope="module")
def grid():
    # 2000 sky points in patches of 50, 16^3 binaries (16 tiles of 256), 90 f0 (3 blocks): P = 48
    pr = synth.mid(n_sky=2000, n_per_det=32, n_ap=16, n_P=16, n_T=16, patch_size=50)
    fp = FakeProblem(pr)
    rc, h = create([fp.d])
    assert rc == bsh.OK
    yield pr, h
    bsh.lib().bsh_plan_destroy(h)


def test_pools_partition_the_items(grid):
    pr, h = grid
    n_pools, psize, walks = _walks(h)
    assert psize == 4 and n_pools == math.ceil(2 * 152 / 4)
    P = math.ceil(pr.B / 256) * math.ceil(pr.n_f0 / 32)
    allitems = np.concatenate(walks)
    assert np.array_equal(np.sort(allitems), np.arange(pr.S * P))
    for w in walks:
        assert np.array_equal(np.sort(w), np.arange(w.min(), w.min() + w.size))


def test_whole_sweeps_are_aligned_across_pools(grid):
    pr, h = grid
    _, _, walks = _walks(h)
    P = math.ceil(pr.B / 256) * math.ceil(pr.n_f0 / 32)
    for w in walks:
        assert w.size > P                       # every pool holds more than one sky point
        full = (w.size // P) * P
        k = np.arange(full)
        assert np.array_equal(w[:full] % P, k % P), "a whole sweep left the common tile order"


def test_last_partial_sweep_stays_on_few_tiles(grid):
    pr, h = grid
    _, _, walks = _walks(h)
    P = math.ceil(pr.B / 256) * math.ceil(pr.n_f0 / 32)
    tails = [w[(w.size // P) * P:] for w in walks]
    m = min(t.size for t in tails)
    assert m > 0
    for x in range(m):
        offsets = {int(t[x] % P) for t in tails if t.size == m}
        assert len(offsets) <= math.ceil(P / m) + 2


def test_pairs_for_an_orbit_table_beyond_half_the_l2():
    # the metric bank of Eq. (30)-(32) over 2 x 1000 SFTs: 8 517 orbit rows x 2 048 padded SFTs x
    # 4 B = 70 MB; the same bank over 2 x 40 SFTs: 8.7 MB
    from oracle import bank as obank
    sizes = {}
    for n_per_det in (40, 1000):
        pr = synth.metric(n_sky=4, n_per_det=n_per_det, patch_size=2)
        orbit, bo, ba = obank.template_bank(**synth.metric_spec(pr, m=6.4))
        fb = FakeProblem(pr, n_orbit=orbit.shape[0], orbit=orbit.ctypes.data, n_bank=bo.size,
                         bank_orbit=bo.ctypes.data, bank_ap=ba.ctypes.data)
        rc, h = create([fb.d])
        assert rc == bsh.OK
        n_pools, psize, walks = _walks(h)
        assert np.array_equal(np.sort(np.concatenate(walks)), np.arange(sum(w.size for w in walks)))
        table = orbit.shape[0] * (-(-pr.N // 256) * 256) * 4
        sizes[n_per_det] = (table, psize)
        bsh.lib().bsh_plan_destroy(h)
    assert sizes[40][0] < 64 << 20 and sizes[40][1] == 4
    assert sizes[1000][0] > 64 << 20 and sizes[1000][1] == 2


def test_plain_plans_have_no_pools(grid):
    pr, _ = grid
    rc, h = create([FakeProblem(pr).d], mode=bsh.MODE_PLAIN)
    assert rc == bsh.OK
    assert bsh.lib().bsh_debug_pool_walk(h, 0, None, 0, None, None, None) == bsh.ERR_STATE
    bsh.lib().bsh_plan_destroy(h)
