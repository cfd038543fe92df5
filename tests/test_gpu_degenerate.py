"""Degenerate and ragged-edge shapes through the C ABI against the FP64 oracle: a single
template over two SFTs, and binary tiles, SFT chunks and patches that end with a remainder
(one template, 12 SFTs, one sky point) next to uneven f0 blocks."""
import numpy as np
import pytest

import oracle
from paper_1904_04873_gb300 import bsh, synth
from gpu_common import REL_TOL, check_dense, check_toplists, device_problem, oracle_scores

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1904_04873_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _problem(n_per_det, n_f0, a_p, n_sky, patch_size, top_k):
    return synth.make_problem("degenerate", n_per_det=n_per_det, dets=["H1", "L1"], T_sft=900.0,
                              span=synth.YEAR_SID, random_times=True, f_lo=200.0, n_f0=n_f0, half_bin=False,
                              sky=synth.fibonacci_sky(n_sky), patch_size=patch_size, a_p=np.asarray(a_p),
                              P_days=np.array([20.0]), n_T=1, power_kind="gauss", top_k=top_k)


def one_template():
    # one sky point, one binary template, one f0 bin, one SFT per detector
    return _problem(n_per_det=1, n_f0=1, a_p=[2.0], n_sky=1, patch_size=1, top_k=1)


def ragged_edges():
    # 257 binaries (a full 256-thread tile + 1), 33 f0 bins (uneven blocks of 17 and 16),
    # 2 x 70 SFTs (a 128-SFT stage + 12), 3 sky points in patches of 2 and 1
    return _problem(n_per_det=70, n_f0=33, a_p=np.linspace(0.5, 10.0, 257), n_sky=3, patch_size=2, top_k=7)


@pytest.mark.parametrize("mode", [bsh.MODE_BATCHED, bsh.MODE_PLAIN])
def test_one_template(mode):
    pr = one_template()
    assert (pr.S, pr.B, pr.n_f0, pr.N) == (1, 1, 1, 2)
    dp, op, wq = device_problem(pr, "f64" if mode == bsh.MODE_PLAIN else "f16")
    plan = bsh.Plan([dp], mode, top_k=pr.top_k)
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    check_dense(gu[0], gw[0], op.count_dense(), exact_w=mode == bsh.MODE_PLAIN)
    plan.number_count()
    cands, n = plan.toplist()
    final, nf = plan.power_sum(1)
    assert bsh.sync_status() == bsh.OK
    lists = bsh.cands_to_numpy(cands, n)
    assert len(lists) == 1 and lists[0].size == 1 and int(lists[0][0]["template_id"]) == 0
    P = op.power_sum(0, 0, 0)
    fin = bsh.cands_to_numpy(final, nf)[0]
    assert fin.size == 1 and abs(fin[0]["power"] - P) <= REL_TOL * abs(P)
    plan.close()


@pytest.mark.parametrize("direct", [0, 1])
def test_ragged_edges_batched(direct):
    pr = ragged_edges()
    assert (pr.S, pr.B, pr.n_f0, pr.N) == (3, 257, 33, 140)
    dp, op, wq = device_problem(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k, threads=256, sft_chunk=128)
    assert plan.set_direct(direct) == direct
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    check_dense(gu[0], gw[0], op.count_dense())
    plan.number_count()
    assert bsh.sync_status() == bsh.OK
    _, sc = oracle_scores(op, wq)
    by_patch = [sc[pr.patch_start[p]:pr.patch_start[p + 1]] for p in range(len(pr.patch_start) - 1)]
    check_toplists(plan, dp, 0, by_patch, pr.top_k, tol=2e-4)
    plan.close()


def test_ragged_edges_lut():
    pr = ragged_edges()
    dp, op, wq = device_problem(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_LUT, top_k=pr.top_k, threads=256, sft_chunk=128)
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    nb = -(-pr.n_f0 // 32)
    lut = oracle.OracleProblem(bits=op.bits, w=op.w, v=pr.v, t=pr.t, F0=pr.F0, n_f0=pr.n_f0, sky=pr.sky,
                               a_p=pr.a_p, Omega=pr.Omega, T_asc=pr.T_asc, k_lo=pr.k_lo, K=pr.K,
                               lut_block=-(-pr.n_f0 // nb))
    check_dense(gu[0], gw[0], lut.count_dense())
    plan.close()
