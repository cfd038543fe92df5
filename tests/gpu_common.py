"""Helpers for the GPU parity tests: device problems fed with oracle inputs."""
import numpy as np

import oracle
from paper_1904_04873_gb300 import bsh, synth
from _common import oracle_inputs, oracle_problem

# Weighted-count and power-sum tolerance against FP64 (relative), from the
# stated accuracy of the FP32 Kahan-compensated sums.
REL_TOL = 1e-5


def device_problem(pr, w_dtype="f16", oracle_fed=True):
    """DeviceProblem whose peakgram, rho and weights come from the oracle
    (so that count parity isolates the count) or from the GPU kernels."""
    import torch
    dp = bsh.DeviceProblem(pr, w_dtype=w_dtype)
    rho, bits, wq = oracle_inputs(pr, w_dtype)
    if oracle_fed:
        dp.bits.copy_(torch.from_numpy(bits.view(np.int32)))
        dp.rho.copy_(torch.from_numpy(rho))
        tdt = dp.w.dtype
        dp.w.copy_(torch.from_numpy(wq).to(tdt))
        dp.sum_w.copy_(torch.from_numpy(wq.sum(axis=1)))
        dp.sum_w2.copy_(torch.from_numpy((wq * wq).sum(axis=1)))
    else:
        dp.prepare()
    return dp, oracle_problem(pr, bits, wq, rho=rho), wq


def oracle_scores(op, wq, rho_th=1.6, s_begin=0, s_end=None):
    d = op.count_dense(s_begin, s_end)
    s_end = op.S if s_end is None else s_end
    sw = wq[s_begin:s_end].sum(axis=1)
    sw2 = (wq[s_begin:s_end] ** 2).sum(axis=1)
    p = np.exp(-rho_th)
    sc = (d["n_w"] - p * sw[:, None, None]) / np.sqrt(p * (1 - p) * sw2)[:, None, None]
    return d, sc


def check_dense(gu, gw, d, rel=REL_TOL, exact_w=False):
    """GPU dense counts against oracle counts (with tie ranges)."""
    gu = gu.cpu().numpy()
    gw = gw.cpu().numpy()
    assert gu.shape == d["n_unw"].shape
    notie = d["n_tie"] == 0
    assert np.array_equal(gu[notie], d["n_unw"][notie]), \
        f"unweighted mismatch in {(gu[notie] != d['n_unw'][notie]).sum()} templates"
    assert np.all((gu >= d["unw_lo"]) & (gu <= d["unw_hi"]))
    ref = d["n_w"]
    if exact_w:
        assert np.array_equal(gw[notie], ref[notie].astype(np.float32))
    else:
        err = np.abs(gw.astype(np.float64) - ref)
        scale = np.maximum(np.abs(ref), 1e-30)
        bad = notie & (err > rel * scale)
        assert not bad.any(), f"weighted mismatch: max rel err {np.max(err[notie] / scale[notie]):.3e}"
    return gu, gw


def check_toplists(plan, dp, q, scores_by_patch, k, tol):
    """GPU toplists of problem q against the oracle's full sort of its scores."""
    cands, n = plan.toplist()
    lists = bsh.cands_to_numpy(cands, n)
    pr = dp.pr
    r0 = plan.first_region(q)
    per_s = pr.B * pr.n_f0
    for p in range(len(pr.patch_start) - 1):
        sc = scores_by_patch[p].ravel()
        g = lists[r0 + p]
        m = min(k, sc.size)
        assert g.size == m
        base = pr.patch_start[p] * per_s
        gid = g["template_id"] - base
        assert np.all(gid >= 0) and np.all(gid < sc.size)
        # GPU scores agree with the oracle's
        assert np.max(np.abs(g["s_h"] - sc[gid])) < tol
        # sorted by (s_H desc, id asc)
        order = np.lexsort((gid, -g["s_h"].astype(np.float64)))
        assert np.array_equal(order, np.arange(g.size))
        ids, osc = oracle.topk(sc, m)
        kth = osc[-1]
        sym = set(ids.tolist()) ^ set(gid.tolist())
        for t in sym:
            assert abs(sc[t] - kth) < 2 * tol, (p, t, sc[t], kth)
    return lists
