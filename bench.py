#!/usr/bin/env python3
"""Benchmark of the BinarySkyHough number count on one GB300 (or N, one process each).

Metric: template-SFT terms per second (one term = one template x one SFT, the
unit of the paper's stage-1 cost C1, Eq. (47)) over one pass of the whole hot
path -- peakgram, weights, FP64 track tables, number count with the fused
per-patch toplist, toplist merge, stage-2 power sum -- on the mid workload:
2 detectors x 2000 SFTs (T_c = 900 s, 1 yr), 0.1 Hz at 200 Hz, 2000 sky points
in 40 patches of 50, 32 a_p x 32 P x 32 t_asc, 90 f0 bins, top-1000 per patch,
fp16 weights.  Synthetic, seeded inputs resident in HBM.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "template-SFT terms/sec and % of gather roofline, batched vs plain, on 1 GB300"
UNIT = "terms/s"
KERNELS_PER_STEP = 8   # peakgram, weights, 2 table kernels, count, merge, power, rerank


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["mid", "small", "eccentric", "metric", "metric-small"], default="mid")
    ap.add_argument("--graph", action="store_true", help="replay count+toplist+power as one CUDA graph")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--no-tune", action="store_true", help="skip the tile-shape autotuner")
    ap.add_argument("--track", choices=["exact", "lut"], default="exact",
                    help="exact track (default) or the look-up-table approximation of Sec. IV.B")
    return ap.parse_args()


def make_problem(kind: str, rank: int, bank_fn=None):
    """The workload's problem; `bank_fn(**spec)` generates the metric workloads' binary bank
    (the library's generator on the GPU arm, the oracle's in the reference arm)."""
    from paper_1904_04873_gb300 import synth
    sky = rank_sky(synth.fibonacci_sky(200 if kind in ("small", "metric-small") else 2000), rank)
    if kind == "mid":
        return synth.mid(sky=sky)
    if kind == "eccentric":
        return synth.eccentric(sky=sky)
    if kind in ("metric", "metric-small"):
        return metric_problem(sky, bank_fn)
    return synth.mid(n_sky=200, n_per_det=500, n_ap=16, n_P=16, n_T=16, sky=sky)


def metric_problem(sky: np.ndarray, bank_fn):
    """The mid construction over a_p 3-13 ls, P 10-20 d searching the template bank of
    Eq. (30)-(32) at mismatch 6.4, one a_p block per Omega."""
    from paper_1904_04873_gb300 import synth
    pr = synth.metric(sky=sky)
    return synth.attach_bank(pr, *bank_fn(**synth.metric_spec(pr, m=6.4)))


def plain_sample(kind: str, sky: np.ndarray, bank_fn=None):
    """The first 4 sky points of the workload, for the plain-form sample."""
    from paper_1904_04873_gb300 import synth
    if kind == "mid":
        return synth.mid(sky=sky[:4], patch_size=50)
    if kind == "eccentric":
        return synth.eccentric(sky=sky[:4])
    if kind in ("metric", "metric-small"):
        return metric_problem(sky[:4], bank_fn)
    return synth.mid(n_sky=4, n_per_det=500, n_ap=16, n_P=16, n_T=16, sky=sky[:4])


def rank_sky(sky: np.ndarray, rank: int) -> np.ndarray:
    """The sky grid searched by `rank`: rotated about z by a rank-dependent angle."""
    if not rank:
        return sky
    a = 2.399963 * rank
    c, s = math.cos(a), math.sin(a)
    return sky @ np.array([[c, s, 0.0], [-s, c, 0.0], [0.0, 0.0, 1.0]])


def rank_env():
    """(world, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, device=None) -> float:
    """Largest value over ranks (control path only); x itself without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(terms_per_rank: float, world: int, t_max: float) -> float:
    """Whole-job throughput: every rank's terms over the slowest rank's time."""
    return terms_per_rank * world / t_max


def workload_config(pr, kind):
    if pr.bank_orbit is not None:
        binary = (f"metric bank (Eq. (30)-(32), mismatch 6.4, a_p {pr.a_p.min():g}-{pr.a_p.max():g} ls, "
                  f"P {2 * math.pi / pr.Omega.max() / 86400:.0f}-{2 * math.pi / pr.Omega.min() / 86400:.0f} d) "
                  f"of {pr.B} binaries on {pr.orbit.shape[0]} orbit rows")
    else:
        binary = f"{pr.a_p.size}x{pr.Omega.size}x{pr.T_asc.shape[1]}"
        if pr.kappa is not None:
            binary += (f"x{pr.kappa.size}x{pr.eta.size} ELL1 (kappa, eta in +-{float(np.max(np.abs(pr.kappa))):g})")
        binary += " binary"
    return {"workload": f"{kind}: {pr.N} SFTs (2 det, T_c=900 s, 1 yr), band {pr.F0 / 900.0:.1f}-"
                        f"{(pr.F0 + pr.n_f0) / 900.0:.1f} Hz, {pr.S} sky pts in patches of 50, "
                        f"{binary}, {pr.n_f0} f0, top-{pr.top_k}",
            "templates": int(pr.n_templates), "terms_per_step": int(pr.n_terms), "weights": "fp16",
            "l2": "256 MiB L2 flush write between steps"}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        try:
            rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
            os.unlink(self.path)
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if sm:
            out = {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def code_only(text: str) -> str:
    """C/CUDA source with comments removed and whitespace runs collapsed."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_sha(root: str = ROOT) -> str:
    """Short hash of the count kernel's sources with comments and whitespace removed, so
    that only code changes invalidate a summary (matches the ncu summaries' stamp)."""
    import hashlib
    src = os.path.join(root, "paper_1904_04873_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("count.cu", "bsh_internal.cuh", "select.cuh"):
        h.update(code_only(open(os.path.join(src, f), encoding="utf-8").read()).encode())
    return h.hexdigest()[:16]


def profile_value(name: str, key: str, root: str = ROOT):
    """A figure recorded in a committed ncu summary, with its source; None when the
    summary is missing or was taken on other kernel sources."""
    path = os.path.join(root, "profiles", name)
    try:
        txt = open(path).read()
    except OSError:
        return None, None
    vals = dict(l.split(":", 1) for l in txt.splitlines() if l.startswith((key + ":", "kernel_source_sha256_16:")))
    if vals.get("kernel_source_sha256_16", "").strip() != kernel_sha(root) or key not in vals:
        return None, f"profiles/{name} (stale: kernel changed since)"
    return float(vals[key]), f"profiles/{name}"


def profiled_traffic(kind: str):
    """DRAM bytes per count launch from the committed ncu summary of this workload."""
    if kind == "mid":
        return profile_value("count_batched_mid.md", "traffic_bytes_per_launch")
    if kind == "metric":
        return profile_value("count_batched_metric_bank.md", "traffic_bytes_per_launch")
    if kind == "metric-small":
        return profile_value("count_batched_metric_bank.md", "traffic_bytes_per_launch_small")
    return None, None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _oracle_worker(args):
    """Spawned process: time the oracle on binary templates [b0, b1) of sky point 0."""
    kw, b0, b1 = args
    import sys
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle
    op = oracle.OracleProblem(**kw)
    t0 = time.perf_counter()
    for b in range(b0, b1):
        for j in range(kw["n_f0"]):
            op.count_one(0, b, j)
    return time.perf_counter() - t0


def _oracle_inputs(pr) -> dict:
    """The oracle's problem for sky point 0 of `pr`: its own peakgram and fp16 weights."""
    import oracle
    rho, bits = oracle.peakgram(pr.power, pr.median_window, pr.rho_th, W=pr.W)
    w = oracle.quantize(oracle.weights(pr.sky[:1], pr.arms, pr.Sn, norm=True), "f16")
    return dict(bits=bits, w=w, v=pr.v, t=pr.t, F0=pr.F0, n_f0=pr.n_f0, sky=pr.sky[:1], a_p=pr.a_p,
                Omega=pr.Omega, T_asc=pr.T_asc, k_lo=pr.k_lo, K=pr.K, kappa=pr.kappa, eta=pr.eta,
                orbit=pr.orbit, bank_orbit=pr.bank_orbit, bank_ap=pr.bank_ap)


def cpu_baseline_sample(pr, budget_s: float = 12.0, procs: int = 0):
    """Time the FP64 oracle on whole templates of sky point 0 (all SFTs, all f0
    bins, a block of binary templates per process), with one process per host
    core; returns (terms/s, cores, sample text)."""
    import multiprocessing as mp
    procs = procs or (os.cpu_count() or 1)
    base = _oracle_inputs(pr)
    per_b = _oracle_worker((base, 0, 2)) / 2          # calibration, in this process
    nb = max(1, min(pr.B // procs, int(budget_s / max(per_b, 1e-6))))
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        times = pool.map(_oracle_worker, [(base, q * nb, (q + 1) * nb) for q in range(procs)])
    dt = max(times)
    terms = procs * nb * pr.n_f0 * pr.N
    return terms / dt, procs, (f"oracle count of sky point 0 x {procs * nb} binary templates x {pr.n_f0} f0 x "
                               f"{pr.N} SFTs ({terms:.3g} terms), {procs} spawned processes of {nb} binaries "
                               f"each, slowest {dt:.1f} s")


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, on every host core
    (spawned processes sharded by binary template), a bounded sample per step."""
    import multiprocessing as mp
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import bank as obank
    pr = make_problem(args.workload, 0, obank.template_bank)
    procs = os.cpu_count() or 1
    base = _oracle_inputs(pr)
    per_b = _oracle_worker((base, 0, 1))
    nb = max(1, min(pr.B // (procs * max(1, args.steps + args.warmup)), int(1.5 / max(per_b, 1e-6))))

    def shards(step):
        b0 = step * procs * nb
        return [(base, b0 + q * nb, b0 + (q + 1) * nb) for q in range(procs)]

    with mp.get_context("spawn").Pool(procs) as pool:
        for k in range(args.warmup):
            pool.map(_oracle_worker, shards(k))
        t0 = time.perf_counter()
        for k in range(args.steps):
            pool.map(_oracle_worker, shards(args.warmup + k))
        dt = time.perf_counter() - t0
    terms = args.steps * procs * nb * pr.n_f0 * pr.N
    v = terms / dt
    sample = (f"per step: oracle count of sky point 0 x {procs * nb} binary templates x {pr.n_f0} f0 x {pr.N} SFTs "
              f"on {procs} spawned processes")
    print(json.dumps({"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "impl": "reference", "config": workload_config(pr, args.workload),
                      "cpu_baseline": {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample},
                      "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist
    from paper_1904_04873_gb300 import build as _build
    from paper_1904_04873_gb300 import bsh

    world, rank, local = rank_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    bsh.lib()

    pr = make_problem(args.workload, rank, bsh.template_bank)
    stream = torch.cuda.current_stream()
    dp = bsh.DeviceProblem(pr, w_dtype="f16")
    mode = bsh.MODE_LUT if args.track == "lut" else bsh.MODE_BATCHED
    plan = bsh.Plan([dp], mode, top_k=pr.top_k, threads=args.threads, sft_chunk=args.chunk)
    n_cf = 100
    dp.prepare()
    tile = plan.tile() if args.no_tune else plan.autotune()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]

    def step(k=None):
        flush.fill_(k if k is not None else 0)
        dp.prepare()
        if k is not None:
            ev[k][0].record(stream)
        plan.number_count()
        if k is not None:
            ev[k][1].record(stream)
        if args.graph:
            plan.graph_launch(n_cf)
        else:
            plan.toplist()
            if k is not None:
                ev2[k][0].record(stream)
            plan.power_sum(n_cf)
            if k is not None:
                ev2[k][1].record(stream)

    for _ in range(max(args.warmup, 0)):
        step()
    st = bsh.sync_status()
    if st != bsh.OK:
        raise SystemExit(f"device status {st} after warm-up")

    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        step(k)
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    elapsed = t_start.elapsed_time(t_end) / 1e3
    count_ms = [a.elapsed_time(b) for a, b in ev]
    count_s = sum(count_ms) / 1e3 / args.steps
    stage2 = None
    if not args.graph:
        # stage 2 (power_kernel + rerank_kernel): every toplist entry of every patch over all SFTs
        s2_ms = sum(a.elapsed_time(b) for a, b in ev2) / args.steps
        n_c = int(plan.n_cands.sum().item())
        stage2 = {"candidates": n_c, "terms": n_c * pr.N, "ms": s2_ms,
                  "terms_per_s": n_c * pr.N / (s2_ms * 1e-3) if s2_ms > 0 else None}
    st = bsh.sync_status()
    if st != bsh.OK:
        raise SystemExit(f"device status {st} in timed region")

    t_max = max_over_ranks(elapsed, "cuda")
    terms_rank = pr.n_terms * args.steps
    value = weak_value(terms_rank, world, t_max)

    # ---- end to end through the public API: pinned host inputs -> device -> toplists -> host
    e2e = None
    if not args.no_e2e:
        host = {k: torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for k, a in
                dict(power=pr.power, v=pr.v, t=pr.t, arms=pr.arms, Sn=pr.Sn, sky=pr.sky).items()}
        h2d = sum(t.numel() * t.element_size() for t in host.values())
        out_host = torch.empty_like(plan.cands, device="cpu").pin_memory()
        n_host = torch.empty_like(plan.n_cands, device="cpu").pin_memory()
        fin_host = None

        def e2e_step():
            nonlocal fin_host
            dp.power.copy_(host["power"], non_blocking=True)
            dp.v.copy_(host["v"], non_blocking=True)
            dp.t.copy_(host["t"], non_blocking=True)
            dp.arms.copy_(host["arms"], non_blocking=True)
            dp.Sn.copy_(host["Sn"], non_blocking=True)
            dp.sky.copy_(host["sky"], non_blocking=True)
            dp.prepare()
            plan.number_count()
            plan.toplist()
            fin, nf = plan.power_sum(n_cf)
            if fin_host is None:
                fin_host = torch.empty_like(fin, device="cpu").pin_memory()
            fin_host.copy_(fin, non_blocking=True)
            n_host.copy_(nf, non_blocking=True)
            return fin.numel() * fin.element_size() + nf.numel() * nf.element_size()

        e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        ke = max(1, min(args.steps, 3))
        a0.record(stream)
        for _ in range(ke):
            d2h = e2e_step()
        a1.record(stream)
        torch.cuda.synchronize()
        te = max_over_ranks(a0.elapsed_time(a1) / 1e3, "cuda")
        e2e = {"value": weak_value(pr.n_terms * ke, world, te), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    # ---- plain form (FP64 track per term, FP64 weights, one launch per patch) on a bounded sample
    plain = None
    if not args.no_plain and rank == 0:
        sub = plain_sample(args.workload, pr.sky, bsh.template_bank)
        dps = bsh.DeviceProblem(sub, w_dtype="f64")
        dps.prepare()
        pplan = bsh.Plan([dps], bsh.MODE_PLAIN, top_k=pr.top_k)
        pplan.number_count()
        torch.cuda.synchronize()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        pplan.number_count()
        b1.record(stream)
        torch.cuda.synchronize()
        tp = b0.elapsed_time(b1) / 1e3
        plain = {"value": sub.n_terms / tp, "unit": UNIT, "sample": f"plain form on {sub.S} sky points x "
                 f"{sub.B} binaries x {sub.n_f0} f0 x {sub.N} SFTs (one launch per patch)", "ms": tp * 1e3}
        pplan.close()

    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    count_rate = pr.n_terms / count_s
    achieved_gbs = count_rate * 4.0 / 1e9
    peak_gbs = n_sm * 128.0 * f_max / 1e9
    traffic, traffic_src = profiled_traffic(args.workload)
    roofline = {"bound": "smem", "achieved": achieved_gbs, "peak": peak_gbs, "unit": "GB/s",
                "frac": achieved_gbs / peak_gbs, "traffic": traffic, "traffic_source": traffic_src,
                "kernel": "bsh_number_count (track tables + count_batched)",
                "peak_source": f"derived: {n_sm} SMs x 32 banks x 4 B/clk x {f_max / 1e6:.0f} MHz "
                               f"(MEASURED_PEAKS sm_max_mhz); one 32-bit word per term",
                "terms_per_s": count_rate, "count_ms": count_s * 1e3,
                "count_ms_median": float(np.median(count_ms)) if count_ms else None}
    if clocks.get("sm_mhz"):
        roofline["frac_at_observed_clock"] = count_rate / (n_sm * 32.0 * clocks["sm_mhz"] * 1e6)
    # the bit-level ceiling: one peakgram bit (1/8 B) of shared memory per term
    roofline["bit_ceiling"] = {"terms_per_s": n_sm * 128.0 * 8.0 * f_max,
                               "frac": count_rate / (n_sm * 128.0 * 8.0 * f_max)}
    # the binding ceiling of this kernel is ALU issue: 128 lanes x f_SM per SM, at the thread
    # instructions per term that ncu measured for this kernel variant
    ipt, ipt_src = profile_value("count_batched_metric_bank.md" if args.workload.startswith("metric")
                                 else "count_batched_small_full.md",
                                 "lut_instr_per_term" if args.track == "lut" else "instr_per_term")
    if ipt:
        roofline["alu"] = {"ceiling_terms_per_s": n_sm * 128.0 * f_max / ipt, "instr_per_term": ipt,
                           "frac": count_rate / (n_sm * 128.0 * f_max / ipt), "source": ipt_src}
    else:
        roofline["alu"] = {"ceiling_terms_per_s": None, "instr_per_term": None, "frac": None, "source": ipt_src}
    # the word-gather roofline is the metric's denominator, not a hard limit of this kernel (one
    # shared-memory word serves 32 terms); the ceilings that bind are ALU issue, then the bit level
    roofline["binding"] = "alu" if ipt else None

    cpu = None
    if not args.no_cpu and rank == 0:
        v, cores, sample = cpu_baseline_sample(pr)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32+f32", "data": "synthetic",
                "config": workload_config(pr, args.workload) | {"parallelism": f"replicas x{world}",
                                                                  "graph": bool(args.graph), "tile": tile,
                                                                  "track": args.track},
                "clocks": {k: clocks.get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons")},
                "e2e": e2e, "gpu_launches": KERNELS_PER_STEP * args.steps, "roofline": roofline, "stage2": stage2,
                "plain": plain, "cpu_baseline": cpu}
        print(json.dumps(line))
    plan.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
