"""GPU parity of the low-eccentricity (ELL1, Eq. (14)) search against the FP64 oracle.

The eccentric grid adds kappa = e cos(omega) and eta = e sin(omega) to each
circular orbit; the kernels see it only through the per-orbit track tables,
so the bar is the circular one: bins and unweighted counts bit-exact outside
the tie band, weighted counts and power sums within 1e-5 relative, toplists
equal up to entries within the score error of the k-th.
"""
import numpy as np
import pytest

import oracle
from paper_1904_04873_gb300 import bsh, synth
from _common import inject_on_track, orbit_of, small_mid
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


def _ecc_small(top_k=40, e_max=0.05):
    # 6 sky points in 2 patches, 300 SFTs (ragged chunks), B = 4 a_p x 2 x 2 x 3 kappa x 2 eta = 96
    # (ragged binary tile), 90 f0 templates (3 blocks)
    return synth.eccentric(n_sky=6, n_per_det=150, n_ap=4, n_P=2, n_T=2, n_kap=3, n_eta=2, e_max=e_max,
                           patch_size=3, top_k=top_k)


@pytest.mark.parametrize("dtype", ["f16", "f32"])
def test_count_dense_batched(dtype):
    pr = _ecc_small()
    assert pr.B == 96
    dp, op, wq = device_problem(pr, dtype)
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    check_dense(gu[0], gw[0], op.count_dense())
    plan.close()


def test_count_dense_plain_is_fp64_exact():
    pr = _ecc_small()
    dp, op, wq = device_problem(pr, "f64")
    plan = bsh.Plan([dp], bsh.MODE_PLAIN, top_k=pr.top_k)
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    check_dense(gu[0], gw[0], op.count_dense(), exact_w=True)
    plan.close()


def test_zero_eccentricity_grid_equals_circular():
    pr = small_mid(n_sky=6, n_per_det=150, n_ap=4, n_P=3, n_T=3, patch_size=3, top_k=40)
    dp, _, _ = device_problem(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=40)
    gu, gw = plan.count_dense()
    plan.close()
    pr.kappa = np.zeros(1)
    pr.eta = np.zeros(1)
    dz, _, _ = device_problem(pr, "f16")
    plan = bsh.Plan([dz], bsh.MODE_BATCHED, top_k=40)
    zu, zw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    assert torch.equal(gu[0], zu[0]) and torch.equal(gw[0], zw[0])
    plan.close()


def test_toplist_and_power_sum():
    pr = _ecc_small()
    dp, op, wq = device_problem(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    plan.autotune()
    plan.number_count()
    assert bsh.sync_status() == bsh.OK
    _, sc = oracle_scores(op, wq)
    by_patch = [sc[pr.patch_start[p]:pr.patch_start[p + 1]] for p in range(len(pr.patch_start) - 1)]
    lists = check_toplists(plan, dp, 0, by_patch, pr.top_k, tol=2e-4)
    cands, n = plan.toplist()
    plan.power_sum(10)
    assert bsh.sync_status() == bsh.OK
    per_s = pr.B * pr.n_f0
    for g in bsh.cands_to_numpy(cands, n):
        for c in g[:15]:
            s, rem = divmod(int(c["template_id"]), per_s)
            b, j = divmod(rem, pr.n_f0)
            P = op.power_sum(s, b, j)
            assert abs(c["power"] - P) <= REL_TOL * P
    assert len(lists) == 2
    plan.close()


def test_track_bins_equal_oracle():
    pr = synth.eccentric(n_sky=12, n_per_det=100, n_ap=4, n_P=3, n_T=3, n_kap=3, n_eta=3, e_max=0.1)
    dp = bsh.DeviceProblem(pr, w_dtype="f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=10)
    rng = np.random.default_rng(4)
    ids = rng.integers(0, pr.n_templates, 24)
    bins = plan.track_bins(torch.as_tensor(ids, device="cuda")).cpu().numpy()
    assert bsh.sync_status() == bsh.OK
    per_s = pr.B * pr.n_f0
    n_ecc = 0
    for q, tid in enumerate(ids):
        s, rem = divmod(int(tid), per_s)
        b, j = divmod(rem, pr.n_f0)
        ap, Om, Ta, kap, eta = orbit_of(pr, b)
        n_ecc += (kap != 0.0 or eta != 0.0)
        for i in range(0, pr.N, 5):
            k, tie = oracle.track_bin_ell1(pr.F0 + j, pr.v[i], pr.sky[s], ap, Om, Ta, kap, eta, pr.t[i])
            assert tie or bins[q, i] == k
    assert n_ecc > 0
    plan.close()


def test_eccentric_injection_ranks_first_and_needs_the_eccentric_terms():
    # an injection on an e = 0.1 track: found by its own template with every SFT hit; the
    # circular template of the same (a_p, Omega, t_asc, f0) misses part of the track
    pr = synth.eccentric(n_sky=4, n_per_det=150, n_ap=3, n_P=2, n_T=2, n_kap=3, n_eta=3, e_max=0.1,
                         patch_size=4, top_k=20)
    pr.power = synth.exp_rho(pr.N, pr.K, np.random.default_rng(5))
    pr.median_window = 0
    ik, ie = 2, 0                       # kappa = +0.1, eta = -0.1
    # P = 15 d, a_p = 10 ls at F = 180045: F a_p Omega = 8.7 bins, so e = 0.14 moves the track by ~1 bin
    b_inj = (((0 * pr.T_asc.shape[1] + 1) * pr.kappa.size + ik) * pr.eta.size + ie) * pr.a_p.size + 2
    s_inj, j_inj = 2, 45
    pr.power = inject_on_track(pr, pr.power, s_inj, b_inj, j_inj, excess=3.0)
    dp = bsh.DeviceProblem(pr, w_dtype="f32")
    dp.prepare()
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    plan.number_count()
    cands, n = plan.toplist()
    gu, _ = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    top = bsh.cands_to_numpy(cands, n)[0]
    assert top[0]["template_id"] == (s_inj * pr.B + b_inj) * pr.n_f0 + j_inj
    assert top[0]["n_unw"] == pr.N
    b_circ = (((0 * pr.T_asc.shape[1] + 1) * pr.kappa.size + 1) * pr.eta.size + 1) * pr.a_p.size + 2
    assert orbit_of(pr, b_circ)[3:] == (0.0, 0.0)
    assert int(gu[0][s_inj, b_circ, j_inj]) < pr.N
    plan.close()


def test_mixed_circular_and_eccentric_batch():
    circ = small_mid(n_sky=5, n_per_det=70, n_ap=3, n_P=2, n_T=3, patch_size=2, top_k=12)
    ecc = synth.eccentric(n_sky=5, n_per_det=70, n_ap=3, n_P=2, n_T=2, n_kap=2, n_eta=3, e_max=0.03,
                          patch_size=3, top_k=12)
    dps = [device_problem(p, "f16") for p in (circ, ecc)]
    plan = bsh.Plan([d[0] for d in dps], bsh.MODE_BATCHED, top_k=12)
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    for q, (dp, op, wq) in enumerate(dps):
        check_dense(gu[q], gw[q], op.count_dense())
    plan.number_count()
    assert bsh.sync_status() == bsh.OK
    for q, (dp, op, wq) in enumerate(dps):
        _, sc = oracle_scores(op, wq)
        pr = dp.pr
        by_patch = [sc[pr.patch_start[p]:pr.patch_start[p + 1]] for p in range(len(pr.patch_start) - 1)]
        check_toplists(plan, dp, q, by_patch, 12, tol=2e-4)
    plan.close()
