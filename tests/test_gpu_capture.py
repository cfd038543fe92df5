"""The calls marked capturable in include/bsh.h, recorded into one CUDA graph by the caller.

One graph holds the whole search step and its post-processing -- number count with the
fused toplist, merge, stage 2, candidate parameters, clustering -- plus stage 2 over a
second SFT set; replaying it must reproduce the eager results exactly.
"""
import numpy as np
import pytest

from paper_1904_04873_gb300 import bsh, synth
from _common import small_mid
from gpu_common import device_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1904_04873_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _step(plan, pp):
    plan.number_count()
    plan.toplist()
    final, nf = plan.power_sum(10)
    params, sig, valid = bsh.cand_params(plan, 0, final, nf, 1, pp)
    label, keep, cen, csig, best = bsh.cluster(params, sig, valid, pp)
    return [plan.cands, plan.n_cands, final, nf, params, sig, valid, label, keep, cen, csig, best]


def test_search_step_and_post_processing_in_one_graph():
    pr = small_mid(n_sky=6, n_per_det=150, n_ap=4, n_P=3, n_T=3, patch_size=3, top_k=40)
    dp, _, _ = device_problem(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    pp = bsh.post_params(T_c=900.0, T_obs=synth.YEAR_SID, d_cut=3.0)
    eager = [t.clone() for t in _step(plan, pp)]          # also the warm-up: kernel attributes set
    torch.cuda.synchronize()
    assert bsh.sync_status() == bsh.OK
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            outs = _step(plan, pp)
    for _ in range(2):
        for t in outs:
            if t.dtype == torch.float64:
                t.fill_(float("nan"))
            else:
                t.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert bsh.sync_status() == bsh.OK
        for a, b in zip(eager, outs):
            if a.dtype == torch.float64:
                assert torch.equal(torch.nan_to_num(a, nan=-7.0), torch.nan_to_num(b, nan=-7.0)) or \
                    torch.allclose(a, b, rtol=1e-12, equal_nan=True)
            else:
                assert torch.equal(a, b)
    plan.close()


def test_sliding_stage2_in_a_graph():
    pr1, pr2, _ = synth.sliding_problems()
    d1, _, _ = device_problem(pr1, "f16")
    d2, _, _ = device_problem(pr2, "f16")
    p1 = bsh.Plan([d1], bsh.MODE_BATCHED, top_k=pr1.top_k)
    p2 = bsh.Plan([d2], bsh.MODE_BATCHED, top_k=pr1.top_k)
    p1.number_count()
    p1.toplist()
    f, n = p2.power_sum_sft(p1, 20)
    ref = (f.clone(), n.clone())
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            p1.toplist()
            f2, n2 = p2.power_sum_sft(p1, 20)
    f2.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert bsh.sync_status() == bsh.OK
    assert torch.equal(f2, ref[0]) and torch.equal(n2, ref[1])
    p1.close()
    p2.close()
