"""Workload experiments through the public API (one JSON document each).

    python -m paper_1904_04873_gb300.experiments precision [--sky N]
    python -m paper_1904_04873_gb300.experiments batching [--patches P] [--steps K]
    python -m paper_1904_04873_gb300.experiments full [--sky N] [--injections M]
    python -m paper_1904_04873_gb300.experiments lut [--sky N]
    python -m paper_1904_04873_gb300.experiments metric [--sky N] [--injections M] [--mismatch m]

precision  Half-bin f0 grid with forced exact ties: the fixed-point track of the
           batched kernels against the exact FP64 bins for every term of a sky
           subset, the same expression in single precision (which must disagree),
           and the weighted-count error of fp16 / bf16 / fp32 weights against
           FP64 weights (plain FP64 form as the reference).
batching   Uneven sky patches searched in four bands with different T_c in one
           persistent launch per step, replayed as a CUDA graph; terms/s.
full       2 x 4000 SFTs, 10 Hz at 300 Hz, patches of 169 sky points, 8^3 binary
           templates, top-10000, stage-2 power sum; seeded injections placed on
           their exact tracks; recovery = a toplist entry within one grid step of
           the injection in every parameter.
metric     A search over a binary template bank with the spacings of Eq. (30)-(32)
           (the BS3 ranges of Sec. VI.A: a_p 3-13 ls, P 10-20 d) with seeded
           injections, stage 2, and the post-processing of Sec. V.E on the GPU:
           clusters of each band's final lists, and recovery = a kept cluster's
           centroid within 13 bins (Eq. (44)) of the injection, the criterion of
           Sec. VI.A.
lut        Exact track against the look-up-table approximation of Sec. IV.B
           (BSH_MODE_LUT) on the mid workload and on a fast-binary variant
           (P = 1.5-3 d, a_p = 10-60 ls): number-count throughput of both, the
           fraction of templates whose count changes, the change of s_H, and the
           overlap of the per-patch toplists.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import sys
import time

import numpy as np

from . import bsh, synth


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def precision(n_sky: int = 2000, n_sky_terms: int = 2, n_sky_dense: int = 4) -> dict:
    """Fixed-point vs FP64 vs single-precision bins, and weight-dtype errors."""
    import torch
    pr = synth.precision_stress(n_sky=n_sky)
    out = {"workload": f"precision stress: {pr.N} SFTs, half-bin f0 grid (F0 = {pr.F0}), {pr.S} sky points "
                       f"(pole included), a_p grid with 0, {pr.B} binaries, {pr.n_f0} f0", "tracks": {}}
    dp = bsh.DeviceProblem(pr, w_dtype="f16")
    dp.prepare()
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=100)
    # forced-tie sky point (the pole, index 0) plus one ordinary sky point
    for s0 in (0, 1):
        c = plan.track_precision(0, s0, s0 + 1)
        out["tracks"][f"sky{s0}"] = {"terms": c[0], "single_precision_mismatch": c[1],
                                     "fixed_point_mismatch_outside_tie_band": c[2], "tie_band_terms": c[3]}
    c = plan.track_precision(0, 2, 2 + n_sky_terms)
    out["tracks"]["sample"] = {"sky_points": n_sky_terms, "terms": c[0], "single_precision_mismatch": c[1],
                               "fixed_point_mismatch_outside_tie_band": c[2], "tie_band_terms": c[3]}
    assert bsh.sync_status() == bsh.OK
    plan.close()
    # weighted-count error by weight dtype, on a few sky points
    sub = synth.precision_stress(n_sky=n_sky)
    sub.sky = sub.sky[:n_sky_dense]
    sub.patch_start = np.array([0, n_sky_dense])
    ref = bsh.DeviceProblem(sub, w_dtype="f64")
    ref.prepare()
    pplan = bsh.Plan([ref], bsh.MODE_PLAIN, top_k=10)
    ru, rw = pplan.count_dense()
    rw64 = rw[0].double().cpu().numpy()
    pplan.close()
    errs = {}
    for dt in ("f32", "f16", "bf16"):
        d = bsh.DeviceProblem(sub, w_dtype=dt)
        d.prepare()
        # the same quantised weights summed exactly (FP64) by the plain form
        q = bsh.DeviceProblem(sub, w_dtype="f64")
        q.prepare()
        q.w.copy_(d.w.double())
        q.sum_w.copy_(d.sum_w)
        q.sum_w2.copy_(d.sum_w2)
        qp = bsh.Plan([q], bsh.MODE_PLAIN, top_k=10)
        _, qw = qp.count_dense()
        qp.close()
        bp = bsh.Plan([d], bsh.MODE_BATCHED, top_k=10)
        bu, bw = bp.count_dense()
        bp.close()
        g = bw[0].double().cpu().numpy()
        e = qw[0].double().cpu().numpy()
        nz = rw64 > 0
        errs[dt] = {"accumulation_max_rel_err": float(np.max(np.abs(g[nz] - e[nz]) / e[nz])),
                    "quantisation_max_rel_err_vs_f64_weights": float(np.max(np.abs(g[nz] - rw64[nz]) / rw64[nz])),
                    "quantisation_rms_rel_err_vs_f64_weights":
                        float(np.sqrt(np.mean(((g[nz] - rw64[nz]) / rw64[nz]) ** 2))),
                    "unweighted_equal_to_plain": bool(np.array_equal(bu[0].cpu().numpy(), ru[0].cpu().numpy()))}
    assert bsh.sync_status() == bsh.OK
    out["weights"] = errs
    out["dense_templates"] = int(n_sky_dense * sub.B * sub.n_f0)
    return out


def batching(n_patch: int = 64, steps: int = 2, warmup: int = 1, size_lo: int = 500, size_hi: int = 5000) -> dict:
    """Four bands x uneven patches in one persistent launch, graph-replayed."""
    import torch
    probs = synth.batching(n_patch=n_patch, size_lo=size_lo, size_hi=size_hi)
    dps = [bsh.DeviceProblem(p, w_dtype="f16") for p in probs]
    for d in dps:
        d.prepare()
    plan = bsh.Plan(dps, bsh.MODE_BATCHED, top_k=1000)
    tile = plan.autotune()
    for _ in range(warmup):
        plan.graph_launch(100)
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    for _ in range(steps):
        plan.graph_launch(100)
    e1.record()
    torch.cuda.synchronize()
    assert bsh.sync_status() == bsh.OK
    dt = e0.elapsed_time(e1) / 1e3 / steps
    terms = sum(p.n_terms for p in probs)
    sizes = np.diff(probs[0].patch_start)
    plan.close()
    return {"workload": f"batching: {n_patch} patches of {sizes.min()}-{sizes.max()} sky points "
                        f"({probs[0].S} total) x 4 bands (T_c = 900/600/450/360 s, 1 Hz each), "
                        f"{probs[0].N} SFTs per band, 8^3 binaries", "terms_per_step": int(terms),
            "s_per_step": dt, "terms_per_s": terms / dt, "tile": tile, "graph": True, "launches": "1 count kernel per step"}


def full(n_sky: int = 100048, n_inj: int = 100, depth_amp: float = 0.5, top_k: int = 10000,
         n_f0: int = 9000, seed: int = synth.SEED_INJ) -> dict:
    """Full-scale search with seeded injections and the stage-2 power sum."""
    import torch
    pr = synth.full(n_sky=n_sky, n_f0=n_f0)
    rng = np.random.default_rng(seed)
    # injections: random sky point, binary template and f0 away from the band edges
    inj = []
    for _ in range(n_inj):
        s = int(rng.integers(pr.S))
        b = int(rng.integers(pr.B))
        j = int(rng.integers(2, pr.n_f0 - 2))
        inj.append((s * pr.B + b) * pr.n_f0 + j)
    dp = bsh.DeviceProblem(pr, w_dtype="f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=top_k)
    # exact track bins of the injections (GPU), then a complex amplitude added in the SFT
    # domain at those bins: |n + A|^2 with n the noise of the bin
    ids = torch.as_tensor(np.array(inj, dtype=np.int64), device="cuda")
    bins = plan.track_bins(ids).cpu().numpy()
    power = pr.power.copy()
    srng = np.random.default_rng(seed + 1)
    for q in range(n_inj):
        cols = bins[q] - pr.k_lo
        ph = srng.uniform(0, 2 * math.pi)
        amp = depth_amp * np.sqrt(pr.Sn)
        # re-draw the noise of the affected bins so that signal and noise add coherently
        re = srng.standard_normal(pr.N) * np.sqrt(0.5 * pr.Sn) + amp * math.cos(ph)
        im = srng.standard_normal(pr.N) * np.sqrt(0.5 * pr.Sn) + amp * math.sin(ph)
        power[np.arange(pr.N), cols] = (re * re + im * im).astype(np.float32)
    dp.power.copy_(torch.as_tensor(power))
    dp.prepare()
    tile = plan.autotune()
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    plan.number_count()
    e1.record()
    cands, n = plan.toplist()
    final, nf = plan.power_sum(100)
    torch.cuda.synchronize()
    assert bsh.sync_status() == bsh.OK
    t_count = e0.elapsed_time(e1) / 1e3
    lists = bsh.cands_to_numpy(cands, n)
    # recovery: an entry of the injection's patch within one grid step in every parameter
    per_s = pr.B * pr.n_f0
    n_ap, n_T = pr.a_p.size, pr.T_asc.shape[1]

    def params(tid):
        s, rem = divmod(int(tid), per_s)
        b, j = divmod(rem, pr.n_f0)
        iap = b % n_ap
        r = b // n_ap
        return s, iap, r % n_T, r // n_T, j

    sky = pr.sky
    step = math.acos(max(-1.0, min(1.0, 1 - 2.0 / pr.S))) * 2.5     # ~ grid spacing of the Fibonacci sky
    rec = 0
    for q, tid in enumerate(inj):
        s, iap, iT, iOm, j = params(tid)
        patch = int(np.searchsorted(pr.patch_start, s, side="right") - 1)
        g = lists[patch]
        ok = False
        for c in g["template_id"]:
            s2, a2, t2, o2, j2 = params(c)
            if abs(a2 - iap) <= 1 and abs(t2 - iT) <= 1 and abs(o2 - iOm) <= 1 and abs(j2 - j) <= 1:
                if math.acos(max(-1.0, min(1.0, float(sky[s] @ sky[s2])))) <= step:
                    ok = True
                    break
        rec += ok
    E = rec / n_inj
    plan.close()
    return {"workload": f"full: {pr.N} SFTs (2 det, 1 yr), {pr.n_f0} f0 bins at 300 Hz, {pr.S} sky points in "
                        f"{len(pr.patch_start) - 1} patches, {pr.B} binaries, top-{top_k}",
            "terms": int(pr.n_terms), "count_s": t_count, "terms_per_s": pr.n_terms / t_count, "tile": tile,
            "injections": n_inj, "amplitude_over_sqrt_Sn": depth_amp, "recovered": rec, "efficiency": E,
            "efficiency_error": math.sqrt(E * (1 - E) / n_inj)}


def metric(n_sky: int = 2000, n_inj: int = 20, depth_amp: float = 0.5, m: float = 6.4, ap_block=None,
           n_cf: int = 100, seed: int = synth.SEED_INJ) -> dict:
    """Bank search with injections, stage 2 and GPU post-processing."""
    import torch
    pr = synth.metric(n_sky=n_sky)
    spec = synth.metric_spec(pr, m=m, ap_block=ap_block)
    pr = synth.attach_bank(pr, *bsh.template_bank(**spec))
    rng = np.random.default_rng(seed)
    inj = []
    for _ in range(n_inj):
        s = int(rng.integers(pr.S))
        b = int(rng.integers(pr.B))
        j = int(rng.integers(2, pr.n_f0 - 2))
        inj.append((s * pr.B + b) * pr.n_f0 + j)
    dp = bsh.DeviceProblem(pr, w_dtype="f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    ids = torch.as_tensor(np.array(inj, dtype=np.int64), device="cuda")
    bins = plan.track_bins(ids).cpu().numpy()
    power = pr.power.copy()
    srng = np.random.default_rng(seed + 1)
    for q in range(n_inj):
        cols = bins[q] - pr.k_lo
        ph = srng.uniform(0, 2 * math.pi)
        amp = depth_amp * np.sqrt(pr.Sn)
        re = srng.standard_normal(pr.N) * np.sqrt(0.5 * pr.Sn) + amp * math.cos(ph)
        im = srng.standard_normal(pr.N) * np.sqrt(0.5 * pr.Sn) + amp * math.sin(ph)
        power[np.arange(pr.N), cols] = (re * re + im * im).astype(np.float32)
    dp.power.copy_(torch.as_tensor(power))
    dp.prepare()
    tile = plan.autotune()
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    plan.number_count()
    e1.record()
    cands, n = plan.toplist()
    final, nf = plan.power_sum(n_cf)
    torch.cuda.synchronize()
    t_count = e0.elapsed_time(e1) / 1e3
    # post-processing of the band's final lists (s_P), on the GPU
    pp = bsh.post_params(T_c=pr.T_sft, T_obs=spec["T_obs"], m_a=m, m_Om=m, m_t=m, d_cut=math.sqrt(14.0))
    c0, c1 = _events()
    c0.record()
    params, sig, valid = bsh.cand_params(plan, 0, final, nf, 1, pp)
    label, keep, cen, csig, best = bsh.cluster(params, sig, valid, pp)
    c1.record()
    torch.cuda.synchronize()
    assert bsh.sync_status() == bsh.OK
    t_post = c0.elapsed_time(c1) / 1e3
    lab = label.cpu().numpy()
    roots = np.nonzero(lab == np.arange(lab.size))[0]
    # recovery: a cluster centroid within 13 bins of the injection (GPU coincidences of the
    # injections' true parameters against the centroids)
    ones = torch.ones(n_inj, dtype=torch.int32, device="cuda")
    true_p, _, _ = bsh.cand_params(plan, 0, *_id_lists(plan, pr, inj), 0, pp)
    tp = true_p.cpu().numpy()
    truth = torch.as_tensor(np.stack([tp[q] for q in _rows_of(plan, pr, inj)]), device="cuda")
    croot = cen[torch.as_tensor(roots, device="cuda")].contiguous()
    pr13 = bsh.post_params(T_c=pr.T_sft, T_obs=spec["T_obs"], m_a=m, m_Om=m, m_t=m, d_coinc=13.0)
    pairs, _, _, npair = bsh.coincidences(truth, ones.double(), ones, croot,
                                          torch.ones(roots.size, dtype=torch.float64, device="cuda"),
                                          torch.ones(roots.size, dtype=torch.int32, device="cuda"), pr13,
                                          cap=n_inj * max(1, roots.size))
    npair = int(npair.item())
    found = set(int(i) for i in pairs[:npair, 0].cpu().numpy())
    rec = len(found)
    E = rec / n_inj
    plan.close()
    return {"workload": f"metric bank: {pr.N} SFTs (2 det, 1 yr), 0.1 Hz at 200 Hz, {pr.S} sky points in "
                        f"{len(pr.patch_start) - 1} patches, a_p 3-13 ls, P 10-20 d, mismatch {m}, "
                        f"{pr.B} binary templates on {pr.orbit.shape[0]} orbit rows",
            "terms": int(pr.n_terms), "count_s": t_count, "terms_per_s": pr.n_terms / t_count, "tile": tile,
            "ap_block": spec["ap_block"], "post_s": t_post, "candidates": int(valid.sum().item()), "clusters": int(roots.size),
            "injections": n_inj, "amplitude_over_sqrt_Sn": depth_amp, "recovered_within_13_bins": rec,
            "efficiency": E, "efficiency_error": math.sqrt(E * (1 - E) / n_inj)}


def _id_lists(plan, pr, ids):
    """Candidate lists holding the given template ids at rank 0 of their patches' regions
    (one id per region slot; later ids of the same patch go to further ranks)."""
    import torch
    regions = plan.regions
    per = max(1, len(ids))
    raw = np.zeros((regions, per), dtype=bsh.CAND_DTYPE)
    cnt = np.zeros(regions, np.int32)
    per_s = pr.B * pr.n_f0
    for tid in ids:
        s = tid // per_s
        r = int(np.searchsorted(pr.patch_start, s, side="right") - 1)
        raw[r, cnt[r]]["template_id"] = tid
        cnt[r] += 1
    return (torch.as_tensor(raw.view(np.uint8).reshape(regions, per, 32), device="cuda"),
            torch.as_tensor(cnt, device="cuda"))


def _rows_of(plan, pr, ids):
    """Row of each id in the output of cand_params over _id_lists(ids)."""
    per = max(1, len(ids))
    per_s = pr.B * pr.n_f0
    cnt = {}
    rows = []
    for tid in ids:
        s = tid // per_s
        r = int(np.searchsorted(pr.patch_start, s, side="right") - 1)
        k = cnt.get(r, 0)
        cnt[r] = k + 1
        rows.append(r * per + k)
    return rows


def _lut_case(pr, n_sky_dense: int, steps: int) -> dict:
    import torch
    dp = bsh.DeviceProblem(pr, w_dtype="f16")
    dp.prepare()
    out = {"modes": {}}
    lists = {}
    for name, mode in (("exact", bsh.MODE_BATCHED), ("lut", bsh.MODE_LUT)):
        plan = bsh.Plan([dp], mode, top_k=pr.top_k)
        tile = plan.autotune()
        plan.number_count()
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record()
        for _ in range(steps):
            plan.number_count()
        e1.record()
        torch.cuda.synchronize()
        dt = e0.elapsed_time(e1) / 1e3 / steps
        cands, n = plan.toplist()
        assert bsh.sync_status() == bsh.OK
        lists[name] = bsh.cands_to_numpy(cands, n)
        out["modes"][name] = {"s_per_count": dt, "terms_per_s": pr.n_terms / dt, "tile": tile}
        plan.close()
    ov = [len(set(a["template_id"].tolist()) & set(b["template_id"].tolist())) / max(1, a.size)
          for a, b in zip(lists["exact"], lists["lut"])]
    out["toplist_overlap"] = {"mean": float(np.mean(ov)), "min": float(np.min(ov))}
    out["lut_speedup"] = out["modes"]["exact"]["s_per_count"] / out["modes"]["lut"]["s_per_count"]
    # dense counts of both on the first sky points
    sub = dataclasses.replace(pr, sky=pr.sky[:n_sky_dense], patch_start=np.array([0, n_sky_dense]))
    ds = bsh.DeviceProblem(sub, w_dtype="f16")
    ds.prepare()
    res = {}
    for name, mode in (("exact", bsh.MODE_BATCHED), ("lut", bsh.MODE_LUT)):
        plan = bsh.Plan([ds], mode, top_k=10)
        gu, gw = plan.count_dense()
        assert bsh.sync_status() == bsh.OK
        res[name] = (gu[0].cpu().numpy(), gw[0].double().cpu().numpy())
        plan.close()
    p = math.exp(-pr.rho_th)
    sig = np.sqrt(p * (1 - p) * ds.sum_w2.cpu().numpy())[:, None, None]
    dsh = (res["lut"][1] - res["exact"][1]) / sig
    out["dense"] = {"sky_points": n_sky_dense, "templates": int(res["exact"][0].size),
                    "count_changed_fraction": float((res["lut"][0] != res["exact"][0]).mean()),
                    "mean_unweighted_change": float((res["lut"][0] - res["exact"][0]).mean()),
                    "s_h_change_mean": float(dsh.mean()), "s_h_change_rms": float(np.sqrt((dsh ** 2).mean())),
                    "s_h_change_max_abs": float(np.abs(dsh).max())}
    return out


def lut(n_sky: int = 2000, steps: int = 3, n_sky_dense: int = 4) -> dict:
    """Exact track vs the LUT approximation: throughput and count deviation."""
    mid = synth.mid(n_sky=n_sky)
    fast = synth.mid(n_sky=n_sky, a_p=np.linspace(10.0, 60.0, 32), P_days=np.linspace(1.5, 3.0, 32))
    return {"mid": {"workload": f"mid: {mid.N} SFTs, {mid.S} sky points, 32^3 binaries (a_p 0.5-10 ls, "
                                f"P 15-45 d), 90 f0"} | _lut_case(mid, n_sky_dense, steps),
            "fast": {"workload": f"fast binaries: the mid construction with a_p 10-60 ls, P 1.5-3 d "
                                 f"({fast.K} loaded bins)"} | _lut_case(fast, n_sky_dense, steps)}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["precision", "batching", "full", "lut", "metric"])
    ap.add_argument("--mismatch", type=float, default=6.4)
    ap.add_argument("--ap-block", type=float, default=None)
    ap.add_argument("--sky", type=int, default=0)
    ap.add_argument("--patches", type=int, default=64)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--injections", type=int, default=100)
    ap.add_argument("--amp", type=float, default=0.5)
    ap.add_argument("--f0", type=int, default=9000)
    a = ap.parse_args(argv)
    import torch
    from . import build
    from .clocks import ClockSampler
    build.build()
    torch.cuda.set_device(0)
    sampler = ClockSampler(0).start()
    if a.what == "precision":
        r = precision(n_sky=a.sky or 2000)
    elif a.what == "batching":
        r = batching(n_patch=a.patches, steps=a.steps)
    elif a.what == "lut":
        r = lut(n_sky=a.sky or 2000)
    elif a.what == "metric":
        r = metric(n_sky=a.sky or 2000, n_inj=a.injections if a.injections != 100 else 20, depth_amp=a.amp,
                   m=a.mismatch, ap_block=a.ap_block)
    else:
        r = full(n_sky=a.sky or 100048, n_inj=a.injections, depth_amp=a.amp, n_f0=a.f0)
    # SM clocks and throttle reasons over the whole experiment (a rate measured under a thermal
    # or hardware slowdown, or at a clock stuck below its maximum, is not a valid measurement)
    r["clocks"] = sampler.stop()
    print(json.dumps(r))


if __name__ == "__main__":
    main()
