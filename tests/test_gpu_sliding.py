"""Stage 2 with the sliding SFTs of Sec. IV.C, through the C ABI.

Both SFT sets come from one seeded time series (synth.sliding_problems): stage 1 counts
over the whole SFTs of the data, stage 2 sums powers over those plus the SFTs that start
T_c/2 later.  The stage-2 power sums of stage 1's candidates must equal the oracle's
power sums over the combined set (1e-5 relative, s_P 1e-4), a plan over other templates
is refused, and an injected signal gains significance from the extra SFTs.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1904_04873_gb300 import bsh, synth
from _common import orbit_of
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


def test_sliding_stage2_matches_oracle():
    pr1, pr2, ts = synth.sliding_problems()
    assert pr2.N > 1.8 * pr1.N
    d1, o1, w1 = device_problem(pr1, "f16")
    d2, o2, w2 = device_problem(pr2, "f16")
    p1 = bsh.Plan([d1], bsh.MODE_BATCHED, top_k=pr1.top_k)
    p2 = bsh.Plan([d2], bsh.MODE_BATCHED, top_k=pr1.top_k)
    p1.number_count()
    cands, n = p1.toplist()
    final, nf = p2.power_sum_sft(p1, 20)
    assert bsh.sync_status() == bsh.OK
    lists = bsh.cands_to_numpy(cands, n)
    finals = bsh.cands_to_numpy(final, nf)
    per_s = pr1.B * pr1.n_f0
    for r, g in enumerate(lists):
        assert g.size == pr1.top_k
        for c in g:
            s, rem = divmod(int(c["template_id"]), per_s)
            b, j = divmod(rem, pr1.n_f0)
            P = o2.power_sum(s, b, j)
            assert abs(c["power"] - P) <= REL_TOL * P
            sP = oracle.power_significance(P, w2[s].sum(), (w2[s] ** 2).sum())
            assert abs(c["s_p"] - sP) < 1e-4
        f = finals[r]
        assert f.size == 20
        assert np.array_equal(np.sort(f["s_p"])[::-1], np.sort(g["s_p"])[::-1][:20])
    p1.close()
    p2.close()


def test_plans_over_other_templates_are_refused():
    pr1, pr2, ts = synth.sliding_problems()
    other = synth.sliding_problems(n_f0=60)[1]
    d1, _, _ = device_problem(pr1, "f16")
    dx, _, _ = device_problem(other, "f16")
    p1 = bsh.Plan([d1], bsh.MODE_BATCHED, top_k=pr1.top_k)
    px = bsh.Plan([dx], bsh.MODE_BATCHED, top_k=pr1.top_k)
    p1.number_count()
    p1.toplist()
    with pytest.raises(bsh.BshError):
        px.power_sum_sft(p1, 10)
    assert bsh.sync_status() == bsh.OK
    p1.close()
    px.close()


def test_injection_gains_significance_from_the_sliding_sfts():
    s_inj, b_inj, j_inj = 2, 5, 40

    def inject(ts, pr):
        ap, Om, Ta, kap, eta = orbit_of(pr, b_inj)
        F = pr.F0 + j_inj
        n = pr.sky[s_inj]

        def freq(d, t):
            v = synth.detector_velocity(t, ts.dets[d])
            return np.array([oracle.track_x_ell1(F, v[i], n, ap, Om, Ta, kap, eta, t[i]) for i in range(t.size)])
        synth.inject_series(ts, freq, amp=1.0)

    pr1, pr2, ts = synth.sliding_problems(inject=inject)
    d1 = bsh.DeviceProblem(pr1, w_dtype="f16")
    d1.prepare()
    d2 = bsh.DeviceProblem(pr2, w_dtype="f16")
    d2.prepare()
    p1 = bsh.Plan([d1], bsh.MODE_BATCHED, top_k=pr1.top_k)
    p2 = bsh.Plan([d2], bsh.MODE_BATCHED, top_k=pr1.top_k)
    p1.number_count()
    cands, n = p1.toplist()
    f1, n1 = p1.power_sum(10)
    g1 = bsh.cands_to_numpy(cands, n)
    tid = (s_inj * pr1.B + b_inj) * pr1.n_f0 + j_inj
    patch = int(np.searchsorted(pr1.patch_start, s_inj, side="right") - 1)
    e = np.nonzero(g1[patch]["template_id"] == tid)[0]
    assert e.size == 1
    sp1 = float(g1[patch]["s_p"][e[0]])
    cands, n = p1.toplist()
    p2.power_sum_sft(p1, 10)
    assert bsh.sync_status() == bsh.OK
    g2 = bsh.cands_to_numpy(cands, n)
    e2 = np.nonzero(g2[patch]["template_id"] == tid)[0]
    sp2 = float(g2[patch]["s_p"][e2[0]])
    # twice the SFTs: the signal sum doubles while the noise variance grows about threefold
    # (each shifted SFT shares half its data with two neighbours): s_P gains about 2/sqrt(3)
    assert sp2 > sp1 > 3.0
    p1.close()
    p2.close()
