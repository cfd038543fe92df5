"""GPU parity of searches over an explicit binary bank (Sec. V.B) against the FP64 oracle.

A grid written out as a bank must give the grid's counts bit for bit; a metric
bank (spacings of Eq. (30)-(32), from the oracle's bank generator) is checked
like any problem: bins and unweighted counts exact outside the tie band,
weighted counts and power sums within 1e-5, toplists equal up to ties.
"""
import numpy as np
import pytest

from oracle import bank as obank
from paper_1904_04873_gb300 import bsh, synth
from _common import small_mid
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


def metric_slice(n_sky=4, n_per_det=100, rows=(0, 600), m=6.4, ap_block=2.0, top_k=30):
    """A metric() problem over a contiguous slice of its metric bank's orbit rows."""
    pr = synth.metric(n_sky=n_sky, n_per_det=n_per_det, patch_size=2, top_k=top_k)
    orbit, bo, ba = obank.template_bank(**synth.metric_spec(pr, m=m, ap_block=ap_block))
    r0, r1 = rows
    sel = (bo >= r0) & (bo < r1)
    return synth.attach_bank(pr, orbit[r0:r1], bo[sel] - r0, ba[sel])


def _dense(pr, dtype="f16", mode=bsh.MODE_BATCHED, **kw):
    dp, op, wq = device_problem(pr, dtype)
    plan = bsh.Plan([dp], mode, top_k=pr.top_k, **kw)
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    plan.close()
    return gu[0], gw[0], op, wq


@pytest.mark.parametrize("ecc", [False, True])
def test_grid_written_as_bank_is_bitwise_the_grid(ecc):
    if ecc:
        pr = synth.eccentric(n_sky=6, n_per_det=150, n_ap=4, n_P=2, n_T=2, n_kap=3, n_eta=2, e_max=0.05,
                             patch_size=3, top_k=40)
    else:
        pr = small_mid(n_sky=6, n_per_det=150, n_ap=4, n_P=3, n_T=3, patch_size=3, top_k=40)
    gu, gw, _, _ = _dense(pr)
    bu, bw, _, _ = _dense(synth.grid_as_bank(pr))
    assert torch.equal(gu, bu) and torch.equal(gw, bw)


@pytest.mark.parametrize("dtype", ["f16", "f32"])
def test_metric_bank_dense(dtype):
    pr = metric_slice()
    assert pr.B > 256 and pr.orbit.shape[0] == 600
    gu, gw, op, wq = _dense(pr, dtype)
    check_dense(gu, gw, op.count_dense())


def test_metric_bank_tile_shapes_and_plain():
    pr = metric_slice(rows=(1000, 1400))
    gu, gw, op, wq = _dense(pr, "f16", threads=128, sft_chunk=64)
    d = op.count_dense()
    check_dense(gu, gw, d)
    pu, pw, op64, _ = _dense(pr, "f64", mode=bsh.MODE_PLAIN)
    check_dense(pu, pw, op64.count_dense(), exact_w=True)


def test_metric_bank_toplist_and_power_sum():
    pr = metric_slice(rows=(200, 700))
    dp, op, wq = device_problem(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    plan.autotune()
    plan.number_count()
    assert bsh.sync_status() == bsh.OK
    _, sc = oracle_scores(op, wq)
    by_patch = [sc[pr.patch_start[p]:pr.patch_start[p + 1]] for p in range(len(pr.patch_start) - 1)]
    check_toplists(plan, dp, 0, by_patch, pr.top_k, tol=2e-4)
    cands, n = plan.toplist()
    plan.power_sum(10)
    assert bsh.sync_status() == bsh.OK
    per_s = pr.B * pr.n_f0
    for g in bsh.cands_to_numpy(cands, n):
        for c in g[:10]:
            s, rem = divmod(int(c["template_id"]), per_s)
            b, j = divmod(rem, pr.n_f0)
            P = op.power_sum(s, b, j)
            assert abs(c["power"] - P) <= REL_TOL * P
    plan.close()


def test_library_bank_drives_the_same_search():
    # the library's generator gives the oracle's bank, so a plan over it counts the same
    pr = synth.metric(n_sky=2, n_per_det=60, patch_size=2, top_k=10)
    spec = synth.metric_spec(pr, m=6.4, ap_block=2.0)
    lib_bank = bsh.template_bank(**spec)
    orc_bank = obank.template_bank(**spec)
    for x, y in zip(lib_bank, orc_bank):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("kind", ["grid", "bank"])
@pytest.mark.parametrize("direct", [0, 1])
def test_per_term_and_per_warp_binary_terms(kind, direct):
    # both ways of forming the fixed-point binary term, on a grid (many templates per orbit row)
    # and on a metric bank (few)
    if kind == "grid":
        pr = small_mid(n_sky=6, n_per_det=150, n_ap=4, n_P=3, n_T=3, patch_size=3, top_k=40)
    else:
        pr = metric_slice(rows=(300, 700))
    dp, op, wq = device_problem(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
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


def test_one_cta_per_sm_keeps_the_stage():
    # ctas_per_sm = 1 keeps the asked-for stage, which two CTAs per SM would not fit (up to 128
    # orbit rows per tile of this slice), and gives the same counts
    chunk = 64
    pr = metric_slice(rows=(100, 500))
    dp, op, wq = device_problem(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k, threads=256, sft_chunk=chunk, ctas_per_sm=1)
    t = plan.tile()
    assert t["sft_chunk"] == chunk and t["ctas"] <= torch.cuda.get_device_properties(0).multi_processor_count
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    check_dense(gu[0], gw[0], op.count_dense())
    plan.close()


def test_bank_defaults_to_per_term_terms():
    pr = metric_slice(rows=(0, 600), ap_block=2.0)
    dp, _, _ = device_problem(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    assert plan.tile()["direct"] == 1
    plan.close()
    pr = small_mid(n_sky=6, n_per_det=150, n_ap=32, n_P=2, n_T=2, patch_size=3, top_k=40)
    dp, _, _ = device_problem(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    assert plan.tile()["direct"] == 0
    plan.close()


def test_per_term_binary_terms_with_the_lut():
    import oracle
    pr = metric_slice(rows=(300, 700))
    dp, op, wq = device_problem(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_LUT, top_k=pr.top_k)
    assert plan.tile()["direct"] == 1
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    nb = -(-pr.n_f0 // 32)
    lut = oracle.OracleProblem(bits=op.bits, w=op.w, v=pr.v, t=pr.t, F0=pr.F0, n_f0=pr.n_f0, sky=pr.sky,
                               a_p=pr.a_p, Omega=pr.Omega, T_asc=pr.T_asc, k_lo=pr.k_lo, K=pr.K, orbit=pr.orbit,
                               bank_orbit=pr.bank_orbit, bank_ap=pr.bank_ap, lut_block=-(-pr.n_f0 // nb))
    check_dense(gu[0], gw[0], lut.count_dense())
    plan.close()
