"""bsh_power_sum_static against bsh_power_sum and the oracle, through the C ABI.

bsh_power_sum_static is for callers that cannot allocate device memory (no
cudaMalloc and no caching allocator available where they run): it needs no
plan and no workspace and keeps its track tables in a fixed-size static
device array inside the library.  Its P and s_P must match the plan-based
power sum of the same candidates, and the FP64 oracle's Eq. (26) sums, within
the stage-2 tolerance, on two calls in a row (the second call reuses, and must
fully rewrite, the static array).  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
from paper_1904_04873_gb300 import bsh
from _common import small_mid
from gpu_common import REL_TOL, device_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1904_04873_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _reference(dp, top_k):
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=top_k)
    plan.number_count()
    cands, n = plan.toplist()
    plan.power_sum(min(8, top_k))
    assert bsh.sync_status() == bsh.OK
    lists = bsh.cands_to_numpy(cands, n)
    plan.close()
    return np.concatenate(lists)


def _check(dp, ref, op, wq):
    ids = torch.as_tensor(ref["template_id"], dtype=torch.int64, device="cuda")
    power, s_p = bsh.power_sum_static(dp, ids)
    assert bsh.sync_status() == bsh.OK
    power = power.cpu().numpy()
    s_p = s_p.cpu().numpy()
    # against the plan's bsh_power_sum of the same templates
    P = ref["power"].astype(np.float64)
    assert np.all(np.abs(power - P) <= REL_TOL * np.abs(P))
    assert np.all(np.abs(s_p - ref["s_p"]) < 1e-4)
    # against the oracle's FP64 sums (Eq. (26)) along the exact track
    pr = dp.pr
    per_s = pr.B * pr.n_f0
    for e, tid in enumerate(ref["template_id"]):
        s, rem = divmod(int(tid), per_s)
        b, j = divmod(rem, pr.n_f0)
        Po = op.power_sum(s, b, j)
        assert abs(float(power[e]) - Po) <= REL_TOL * Po
        sPo = oracle.power_significance(Po, wq[s].sum(), (wq[s] ** 2).sum())
        assert abs(float(s_p[e]) - sPo) < 1e-4


def test_static_power_sum_matches_plan_twice():
    pr1 = small_mid(n_sky=6, n_per_det=150, n_ap=4, n_P=3, n_T=3, patch_size=3, top_k=30)
    pr2 = small_mid(n_sky=9, n_per_det=100, n_ap=8, n_P=2, n_T=4, patch_size=3, top_k=20, seed=77)
    dp1, op1, wq1 = device_problem(pr1, "f16")
    dp2, op2, wq2 = device_problem(pr2, "f32")
    ref1 = _reference(dp1, 30)
    ref2 = _reference(dp2, 20)
    _check(dp1, ref1, op1, wq1)      # first call on this device sets up the static scratch
    _check(dp2, ref2, op2, wq2)      # second call, different problem: the array is rewritten
    _check(dp1, ref1, op1, wq1)


def test_static_power_sum_eccentric_grid():
    # the ELL1 orbit rows (kappa, eta of Eq. (14)) are expanded in the static tables too
    from paper_1904_04873_gb300 import synth
    pr = synth.eccentric(n_sky=6, n_per_det=150, n_ap=4, n_P=2, n_T=2, n_kap=3, n_eta=2, e_max=0.05,
                         patch_size=3, top_k=25)
    dp, op, wq = device_problem(pr, "f16")
    ref = _reference(dp, 25)
    _check(dp, ref, op, wq)


def test_static_power_sum_explicit_bank():
    # an explicit (metric) bank is staged in the static array as given
    from test_gpu_bank import metric_slice
    pr = metric_slice(rows=(0, 300), top_k=20)
    dp, op, wq = device_problem(pr, "f16")
    ref = _reference(dp, 20)
    _check(dp, ref, op, wq)


def test_static_power_sum_rejects_oversized_problem():
    pr = small_mid(n_sky=2, n_per_det=64, n_ap=2, n_P=2, n_T=2, patch_size=2, top_k=5)
    dp, _, _ = device_problem(pr, "f16")
    d = dp.descriptor()
    # 2 x 6000 Omega-T rows of 256 SFTs need 12000 x 256 x 12 bytes > 32 MiB of tables
    big_T = np.ascontiguousarray(np.tile(pr.T_asc, (1, 3000)))
    d.n_T = big_T.shape[1]
    d.T_asc = big_T.ctypes.data
    ids = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = torch.empty(1, dtype=torch.float32, device="cuda")
    rc = bsh.lib().bsh_power_sum_static(d, ids.data_ptr(), 1, out.data_ptr(), out.data_ptr(),
                                        bsh._stream())
    assert rc == bsh.ERR_WORKSPACE
