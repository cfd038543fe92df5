"""GPU parity of the look-up-table (LUT) number count (Sec. IV.B) against the FP64 oracle.

BSH_MODE_LUT reuses, within each f0 block, the modulation of the block's
middle template.  The oracle evaluates the same definition template by
template; bar as for the exact count (bins and unweighted counts bit-exact
outside the tie band of the reference template, weighted counts within 1e-5).
Stage 2 of a LUT plan keeps the exact track.
"""
import numpy as np
import pytest

import oracle
from paper_1904_04873_gb300 import bsh, synth
from _common import small_mid
from gpu_common import REL_TOL, check_dense, check_toplists, device_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1904_04873_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def lut_block(n_f0):
    nb = -(-n_f0 // 32)
    return -(-n_f0 // nb)


def lut_oracle(pr, op):
    return oracle.OracleProblem(bits=op.bits, w=op.w, v=pr.v, t=pr.t, F0=pr.F0, n_f0=pr.n_f0, sky=pr.sky,
                                a_p=pr.a_p, Omega=pr.Omega, T_asc=pr.T_asc, k_lo=pr.k_lo, K=pr.K,
                                rho=op.rho, kappa=pr.kappa, eta=pr.eta, lut_block=lut_block(pr.n_f0))


def _fast_binaries(n_f0=90, top_k=30):
    # large a_p Omega so that the LUT departs from the exact track often; 2 patches, ragged tiles
    return synth.make_problem("lut", n_per_det=150, dets=["H1", "L1"], T_sft=900.0, span=synth.YEAR_SID,
                              random_times=True, f_lo=200.0, n_f0=n_f0, half_bin=False,
                              sky=synth.fibonacci_sky(6), patch_size=3, a_p=np.array([10.0, 30.0, 60.0]),
                              P_days=np.array([1.5, 2.0, 3.0]), n_T=3, power_kind="exp", top_k=top_k)


@pytest.mark.parametrize("dtype", ["f16", "f32"])
@pytest.mark.parametrize("n_f0", [90, 77])
def test_count_dense_lut(dtype, n_f0):
    pr = _fast_binaries(n_f0=n_f0)
    dp, op, wq = device_problem(pr, dtype)
    lo = lut_oracle(pr, op)
    plan = bsh.Plan([dp], bsh.MODE_LUT, top_k=pr.top_k)
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    d_lut = lo.count_dense()
    check_dense(gu[0], gw[0], d_lut)
    # the approximation is visible: the exact count differs on some templates
    d_ex = op.count_dense()
    notie = (d_lut["n_tie"] == 0) & (d_ex["n_tie"] == 0)
    assert (d_lut["n_unw"][notie] != d_ex["n_unw"][notie]).mean() > 0.01
    plan.close()


def test_lut_tile_shapes_and_accumulation():
    pr = _fast_binaries()
    dp, op, wq = device_problem(pr, "f16")
    d_lut = lut_oracle(pr, op).count_dense()
    for threads, chunk, acc, direct in ((128, 64, 1, 0), (256, 256, 0, 0), (256, 64, 0, 1)):
        plan = bsh.Plan([dp], bsh.MODE_LUT, top_k=pr.top_k, threads=threads, sft_chunk=chunk)
        plan.set_direct(direct)
        plan.set_accumulate(acc)
        assert plan.tile()["accumulate"] == acc and plan.tile()["direct"] == direct
        gu, gw = plan.count_dense()
        assert bsh.sync_status() == bsh.OK
        check_dense(gu[0], gw[0], d_lut)
        plan.close()


def test_lut_toplist_and_exact_stage2():
    pr = _fast_binaries()
    dp, op, wq = device_problem(pr, "f16")
    lo = lut_oracle(pr, op)
    plan = bsh.Plan([dp], bsh.MODE_LUT, top_k=pr.top_k)
    plan.autotune()
    plan.number_count()
    assert bsh.sync_status() == bsh.OK
    d = lo.count_dense()
    sw = wq.sum(axis=1)
    sw2 = (wq ** 2).sum(axis=1)
    p = np.exp(-1.6)
    sc = (d["n_w"] - p * sw[:, None, None]) / np.sqrt(p * (1 - p) * sw2)[:, None, None]
    by_patch = [sc[pr.patch_start[q]:pr.patch_start[q + 1]] for q in range(len(pr.patch_start) - 1)]
    check_toplists(plan, dp, 0, by_patch, pr.top_k, tol=2e-4)
    cands, n = plan.toplist()
    plan.power_sum(8)
    assert bsh.sync_status() == bsh.OK
    per_s = pr.B * pr.n_f0
    for g in bsh.cands_to_numpy(cands, n):
        for c in g[:10]:
            s, rem = divmod(int(c["template_id"]), per_s)
            b, j = divmod(rem, pr.n_f0)
            P = op.power_sum(s, b, j)          # exact track
            assert abs(c["power"] - P) <= REL_TOL * P
    plan.close()


def test_lut_with_eccentric_grid():
    pr = synth.eccentric(n_sky=4, n_per_det=100, n_ap=3, n_P=2, n_T=2, n_kap=2, n_eta=2, e_max=0.1,
                         patch_size=2, top_k=10)
    dp, op, wq = device_problem(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_LUT, top_k=10)
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    check_dense(gu[0], gw[0], lut_oracle(pr, op).count_dense())
    plan.close()


def test_lut_equals_exact_on_the_mid_grid_mostly():
    # on the mid grid (a_p Omega <= 5e-5) the LUT bins leave the exact track rarely
    pr = small_mid(n_sky=6, n_per_det=150, n_ap=4, n_P=3, n_T=3, patch_size=3, top_k=40)
    dp, op, wq = device_problem(pr, "f16")
    a = bsh.Plan([dp], bsh.MODE_LUT, top_k=40)
    lu, lw = a.count_dense()
    b = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=40)
    eu, ew = b.count_dense()
    assert bsh.sync_status() == bsh.OK
    diff = (lu[0] != eu[0]).float().mean().item()
    assert 0.0 < diff < 0.2
    a.close()
    b.close()
