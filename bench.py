#!/usr/bin/env python3
"""Benchmark of the BinarySkyHough number count on one GB300 (or N, one process each).

Metric: template-SFT terms per second (one term = one template x one SFT, the
unit of the paper's stage-1 cost C1, Eq. (47)) over one pass of the whole hot
path -- peakgram, weights, FP64 track tables, number count with the fused
per-patch toplist, toplist merge, stage-2 power sum and re-rank -- with the
count, toplist and stage 2 replayed as one captured CUDA graph.

Default workload (batching): 64 sky patches of uneven size (500-5000 points,
seeded) searched in four 1 Hz bands at 100/200/300/400 Hz with T_c =
900/600/450/360 s (2 x 500 SFTs over 30 days per band, all f0 bins), an
8 x 8 x 8 binary grid, top-1000 per patch, fp16 weights.  The patches are
dealt into 8 groups of about equal sky count; step k searches group k mod 8 in
all four bands in one persistent launch, so 8 steps cover the whole
configuration.  Synthetic, seeded inputs resident in HBM.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle instead.
With --gpus N > 1 outside torchrun, the script relaunches itself under
torch.distributed.run with N ranks (replicas, one GPU each).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import socket
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "template-SFT terms/sec and % of gather roofline, batched vs plain, on 1 GB300"
UNIT = "terms/s"
WORKLOADS = ("batching", "batching-small", "mid", "small", "eccentric", "metric", "metric-small", "full")
N_GROUPS = 8                         # batching: patch groups, one per step
FULL_PATCHES = (0, 148, 296, 444)    # full: the fixed slice of patches searched per step
N_CF = 100                           # stage-2 survivors per patch


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=WORKLOADS, default="batching")
    ap.add_argument("--eager", action="store_true",
                    help="launch count, toplist and stage 2 one by one instead of replaying the captured graph")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--no-tune", action="store_true", help="skip the tile-shape autotuner")
    ap.add_argument("--ctas", type=int, default=0, help="CTAs per SM of the persistent grid (0: the plan's choice)")
    ap.add_argument("--direct", type=int, choices=[-1, 0, 1], default=-1,
                    help="binary term per warp (0) or per term (1); -1 leaves it to the plan / autotuner")
    ap.add_argument("--acc", type=int, choices=[-1, 0, 1, 2], default=-1,
                    help="weighted accumulation (0 predicated adds, 1 byte table, 2 tensor cores); -1: plan / autotuner")
    ap.add_argument("--track", choices=["exact", "lut"], default="exact",
                    help="exact track (default) or the look-up-table approximation of Sec. IV.B")
    return ap.parse_args(argv)


# ------------------------------------------------------------------ workloads

def make_problem(kind: str, rank: int, bank_fn=None):
    """The single-problem workloads; `bank_fn(**spec)` generates the metric workloads'
    binary bank (the library's generator on the GPU arm, the oracle's in the reference arm)."""
    from paper_1904_04873_gb300 import synth
    sky = rank_sky(synth.fibonacci_sky(200 if kind in ("small", "metric-small") else 2000), rank)
    if kind == "mid":
        return synth.mid(sky=sky)
    if kind == "eccentric":
        return synth.eccentric(sky=sky)
    if kind in ("metric", "metric-small"):
        return metric_problem(sky, bank_fn)
    if kind == "small":
        return synth.mid(n_sky=200, n_per_det=500, n_ap=16, n_P=16, n_T=16, sky=sky)
    raise ValueError(kind)


def metric_problem(sky: np.ndarray, bank_fn):
    """The mid construction over a_p 3-13 ls, P 10-20 d searching the template bank of
    Eq. (30)-(32) at mismatch 6.4, one a_p block per Omega."""
    from paper_1904_04873_gb300 import synth
    pr = synth.metric(sky=sky)
    return synth.attach_bank(pr, *bank_fn(**synth.metric_spec(pr, m=6.4)))


def workload_batches(kind: str, rank: int, bank_fn=None):
    """The workload as a list of step batches, each a list of problems searched together in
    one plan (one persistent launch); step k runs batch k mod len(batches)."""
    from paper_1904_04873_gb300 import synth
    if kind == "batching":
        probs = [dataclasses.replace(p, sky=rank_sky(p.sky, rank)) for p in synth.batching()]
        groups = synth.patch_groups(probs[0].patch_start, N_GROUPS)
        return [[synth.select_patches(p, g) for p in probs] for g in groups]
    if kind == "batching-small":
        # the batching construction at profiling size: 8 patches of 20-60 sky points, one step group
        return [[dataclasses.replace(p, sky=rank_sky(p.sky, rank))
                 for p in synth.batching(n_patch=8, size_lo=20, size_hi=60)]]
    if kind == "full":
        pr = synth.full()
        pr = dataclasses.replace(pr, sky=rank_sky(pr.sky, rank))
        return [[synth.select_patches(pr, FULL_PATCHES)]]
    return [[make_problem(kind, rank, bank_fn)]]


def first_points(pr, n: int = 4):
    """The problem restricted to its first n sky points, as one patch."""
    return dataclasses.replace(pr, sky=np.ascontiguousarray(pr.sky[:n]), patch_start=np.array([0, n], np.int64))


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


def free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def launcher_command(n: int, argv, port: int):
    """torch.distributed.run command that starts this script as n ranks on this node."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
            "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__), *argv]


def relaunch(n: int, argv) -> int:
    """Run this script as n ranks (one process per GPU); returns the launcher's exit code."""
    return subprocess.call(launcher_command(n, list(argv), free_port()))


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


def binary_text(pr) -> str:
    if pr.bank_orbit is not None:
        return (f"metric bank (Eq. (30)-(32), mismatch 6.4, a_p {pr.a_p.min():g}-{pr.a_p.max():g} ls, "
                f"P {2 * math.pi / pr.Omega.max() / 86400:.0f}-{2 * math.pi / pr.Omega.min() / 86400:.0f} d) "
                f"of {pr.B} binaries on {pr.orbit.shape[0]} orbit rows")
    out = f"{pr.a_p.size}x{pr.Omega.size}x{pr.T_asc.shape[1]}"
    if pr.kappa is not None:
        out += f"x{pr.kappa.size}x{pr.eta.size} ELL1 (kappa, eta in +-{float(np.max(np.abs(pr.kappa))):g})"
    return out + " binary"


def workload_config(batches, kind: str) -> dict:
    """The `config` object of the JSON line (identical on both arms)."""
    pr = batches[0][0]
    per_step = [sum(p.n_terms for p in b) for b in batches]
    tmpl = [sum(p.n_templates for p in b) for b in batches]
    if kind == "batching":
        S = sum(b[0].S for b in batches)
        text = (f"batching: 64 sky patches of 500-5000 points ({S} sky points) x 4 bands (100/200/300/400 Hz, "
                f"1 Hz each, T_c 900/600/450/360 s, all f0 bins), 2 x 500 SFTs over 30 d per band, "
                f"{binary_text(pr)}, top-{pr.top_k} per patch; patches dealt into {len(batches)} groups of about "
                f"equal sky count, step k searches group k mod {len(batches)} in all 4 bands in one persistent "
                f"launch ({len(batches)} steps cover the configuration)")
    elif kind == "batching-small":
        text = (f"batching-small: the batching construction at profiling size, 8 patches of 20-60 sky points "
                f"({pr.S} sky points) x 4 bands, {binary_text(pr)}, one step group")
    elif kind == "full":
        text = (f"full: {pr.N} SFTs (2 det, T_c=900 s, 1 yr), band {pr.F0 / 900.0:.0f}-"
                f"{(pr.F0 + pr.n_f0) / 900.0:.0f} Hz ({pr.n_f0} f0), {binary_text(pr)}, top-{pr.top_k}; "
                f"per step the fixed slice of patches {', '.join(str(p) for p in FULL_PATCHES)} of the 592 "
                f"patches of 169 sky points ({pr.S} of 100048 sky points)")
    else:
        text = (f"{kind}: {pr.N} SFTs (2 det, T_c=900 s, 1 yr), band {pr.F0 / 900.0:.1f}-"
                f"{(pr.F0 + pr.n_f0) / 900.0:.1f} Hz, {pr.S} sky pts in patches of 50, "
                f"{binary_text(pr)}, {pr.n_f0} f0, top-{pr.top_k}")
    return {"workload": text, "templates_per_step": int(round(np.mean(tmpl))),
            "terms_per_step": int(round(np.mean(per_step))), "terms_per_cycle": int(sum(per_step)),
            "steps_per_cycle": len(batches), "weights": "fp16",
            "l2": "256 MiB L2 flush write between steps"}


def launches_per_step(batch) -> int:
    """Kernels of this library per step: peakgram + weights per problem, the two track-table
    kernels per problem, the count, the merge, the power sum and the re-rank."""
    return 4 * len(batch) + 4


# ------------------------------------------------------------------ clocks

from paper_1904_04873_gb300.clocks import ClockSampler, summarize_clocks  # noqa: E402,F401


# ------------------------------------------------------------------ committed ncu summaries

def code_only(text: str) -> str:
    """C/CUDA source with comments removed and whitespace runs collapsed."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_sha(root: str = ROOT) -> str:
    """Short hash of the count kernels' sources with comments and whitespace removed, so
    that only code changes invalidate a summary (matches the ncu summaries' stamp)."""
    import hashlib
    src = os.path.join(root, "paper_1904_04873_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("count.cu", "count_tc.cu", "count_common.cuh", "bsh_internal.cuh", "select.cuh"):
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


# per workload, where the committed ncu summaries hold the count kernel's thread instructions
# per term ("ipt") and its DRAM bytes per launch ("traffic"): (file, key)
PROFILES = {"batching": {"ipt": ("count_batched_batching.md", "instr_per_term"),
                         "traffic": ("count_batched_batching.md", "traffic_bytes_per_launch")},
            "mid": {"ipt": ("count_batched_mid.md", "instr_per_term"),
                    "traffic": ("count_batched_mid.md", "traffic_bytes_per_launch")},
            "metric": {"ipt": ("count_batched_metric_bank.md", "instr_per_term"),
                       "traffic": ("count_batched_metric_bank.md", "traffic_bytes_per_launch")},
            "metric-small": {"ipt": ("count_batched_metric_bank.md", "instr_per_term"),
                             "traffic": ("count_batched_metric_bank.md", "traffic_bytes_per_launch_small")}}


def profiled(kind: str, what: str, track: str = "exact"):
    ent = PROFILES.get(kind, {}).get(what)
    if ent is None:
        return None, None
    name, key = ent
    if what == "ipt" and track == "lut":
        key = "lut_" + key
    return profile_value(name, key)


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------------ the oracle (CPU legs only)

def _oracle_worker(args):
    """Spawned process: time the oracle on binary templates [b0, b1) (mod B) of sky point 0."""
    kw, b0, b1 = args
    import sys
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle
    op = oracle.OracleProblem(**kw)
    t0 = time.perf_counter()
    for b in range(b0, b1):
        for j in range(kw["n_f0"]):
            op.count_one(0, b % op.B, j)
    return time.perf_counter() - t0


def oracle_sample_problem(pr, max_f0: int = 900):
    """The part of a problem the CPU sample needs: sky point 0 and at most max_f0 f0 bins, with
    the loaded band cut to the bins those templates read (so that the oracle's running median
    runs over that band only)."""
    if pr.n_f0 <= max_f0:
        return pr
    from paper_1904_04873_gb300 import synth
    margin = int(pr.F0) - pr.k_lo
    K = min(pr.K, margin + max_f0 + margin + 1)
    K = max(K, 101)
    W = -(-(-(-K // 32)) // 4) * 4
    return dataclasses.replace(pr, n_f0=max_f0, K=K, W=W, power=np.ascontiguousarray(pr.power[:, :K]))


def _oracle_inputs(pr) -> dict:
    """The oracle's problem for sky point 0 of `pr`: its own peakgram and fp16 weights."""
    import oracle
    pr = oracle_sample_problem(pr)
    rho, bits = oracle.peakgram(pr.power, pr.median_window, pr.rho_th, W=pr.W)
    w = oracle.quantize(oracle.weights(pr.sky[:1], pr.arms, pr.Sn, norm=True), "f16")
    return dict(bits=bits, w=w, v=pr.v, t=pr.t, F0=pr.F0, n_f0=pr.n_f0, sky=pr.sky[:1], a_p=pr.a_p,
                Omega=pr.Omega, T_asc=pr.T_asc, k_lo=pr.k_lo, K=pr.K, kappa=pr.kappa, eta=pr.eta,
                orbit=pr.orbit, bank_orbit=pr.bank_orbit, bank_ap=pr.bank_ap)


def cpu_baseline_sample(pr, budget_s: float = 12.0, procs: int = 0):
    """Time the FP64 oracle on whole templates of sky point 0 (all SFTs, all f0
    bins up to 900, a block of binary templates per process), with one process per
    host core; returns (terms/s, cores, sample text)."""
    import multiprocessing as mp
    procs = procs or (os.cpu_count() or 1)
    base = _oracle_inputs(pr)
    per_b = _oracle_worker((base, 0, 2)) / 2          # calibration, in this process
    B = pr.B
    nb = max(1, min(max(1, B // procs), int(budget_s / max(per_b, 1e-6))))
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        times = pool.map(_oracle_worker, [(base, q * nb, (q + 1) * nb) for q in range(procs)])
    dt = max(times)
    terms = procs * nb * base["n_f0"] * pr.N
    return terms / dt, procs, (f"oracle count of sky point 0 of the {pr.name} band x {procs * nb} binary "
                               f"templates x {base['n_f0']} f0 x {pr.N} SFTs ({terms:.3g} terms), {procs} "
                               f"spawned processes of {nb} binaries each, slowest {dt:.1f} s")


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, on every host core (spawned
    processes sharded by binary template), a bounded sample of the workload per step
    (step k samples sky point 0 of problem k mod n of the first batch)."""
    import multiprocessing as mp
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import bank as obank
    batches = workload_batches(args.workload, 0, obank.template_bank)
    probs = batches[0]
    procs = os.cpu_count() or 1
    bases = [_oracle_inputs(p) for p in probs]
    per_b = _oracle_worker((bases[0], 0, 1))
    nb = max(1, min(max(1, probs[0].B // procs), int(1.0 / max(per_b, 1e-6))))

    def shards(step):
        base = bases[step % len(bases)]
        b0 = (step // len(bases)) * procs * nb
        return [(base, b0 + q * nb, b0 + (q + 1) * nb) for q in range(procs)]

    terms = 0
    with mp.get_context("spawn").Pool(procs) as pool:
        for k in range(args.warmup):
            pool.map(_oracle_worker, shards(k))
        t0 = time.perf_counter()
        for k in range(args.steps):
            pool.map(_oracle_worker, shards(args.warmup + k))
            i = (args.warmup + k) % len(bases)
            terms += procs * nb * bases[i]["n_f0"] * probs[i].N
        dt = time.perf_counter() - t0
    v = terms / dt
    sample = (f"per step: oracle count of sky point 0 x {procs * nb} binary templates x all f0 (up to 900) x all "
              f"SFTs of one problem of the first batch (in turn), on {procs} spawned processes")
    cfg = workload_config(batches, args.workload) | {"parallelism": f"replicas x{args.gpus}", "track": args.track}
    print(json.dumps({"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(1, args.steps), "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "impl": "reference", "config": cfg,
                      "cpu_baseline": {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample},
                      "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# ------------------------------------------------------------------ the GPU arm

def main(argv=None):
    args = parse(argv)
    world, rank, local = rank_env()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        raise SystemExit(relaunch(args.gpus, sys.argv[1:] if argv is None else argv))
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist
    from paper_1904_04873_gb300 import build as _build
    from paper_1904_04873_gb300 import bsh

    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    bsh.lib()

    batches = workload_batches(args.workload, rank, bsh.template_bank)
    G = len(batches)
    stream = torch.cuda.current_stream()
    dps = [[bsh.DeviceProblem(p, w_dtype="f16") for p in b] for b in batches]
    mode = bsh.MODE_LUT if args.track == "lut" else bsh.MODE_BATCHED
    plans, tiles = [], []
    for dpb in dps:
        for dp in dpb:
            dp.prepare()
        plan = bsh.Plan(dpb, mode, top_k=dpb[0].pr.top_k, threads=args.threads, sft_chunk=args.chunk,
                        ctas_per_sm=args.ctas)
        if args.direct >= 0:
            plan.set_direct(args.direct)
        if args.acc >= 0:
            plan.set_accumulate(args.acc)
        tiles.append(plan.tile() if args.no_tune else plan.autotune())
        plans.append(plan)
    terms = [sum(p.n_terms for p in b) for b in batches]
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def launch(g):
        """Count + toplist + stage 2 of group g: the captured graph (or eager launches)."""
        plan = plans[g]
        if args.eager:
            plan.number_count()
            plan.toplist()
            return plan.power_sum(N_CF)
        return plan.graph_launch(N_CF)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]

    def step(k, timed=False):
        g = k % G
        flush.fill_(k & 255)
        for dp in dps[g]:
            dp.prepare()
        if timed:
            ev[k][0].record(stream)
        launch(g)
        if timed:
            ev[k][1].record(stream)

    for g in range(G):            # set-up: records every group's graph (untimed)
        step(g)
    for k in range(max(args.warmup, 0)):
        step(k)
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
        step(k, timed=True)
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    elapsed = t_start.elapsed_time(t_end) / 1e3
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    st = bsh.sync_status()
    if st != bsh.OK:
        raise SystemExit(f"device status {st} in timed region")
    terms_rank = sum(terms[k % G] for k in range(args.steps))
    t_max = max_over_ranks(elapsed, "cuda")
    value = weak_value(terms_rank, world, t_max)

    # ---- stage 2 on its own (one eager pass of group 0 after the timed region)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plans[0].number_count()
    plans[0].toplist()
    s0.record(stream)
    plans[0].power_sum(N_CF)
    s1.record(stream)
    torch.cuda.synchronize()
    s2_ms = s0.elapsed_time(s1)
    n_c = int(plans[0].n_cands.sum().item())
    n_sft = batches[0][0].N
    stage2 = {"candidates": n_c, "terms": n_c * n_sft, "ms": s2_ms,
              "terms_per_s": n_c * n_sft / (s2_ms * 1e-3) if s2_ms > 0 else None,
              "measured": "one eager bsh_power_sum (power_kernel + rerank_kernel) of step group 0 after the "
                          "timed region"}

    # ---- end to end through the public API, every step: pinned host inputs -> device -> lists -> host
    e2e = None
    if not args.no_e2e:
        host = [[{k: torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for k, a in
                  dict(power=dp.pr.power, v=dp.pr.v, t=dp.pr.t, arms=dp.pr.arms, Sn=dp.pr.Sn,
                       sky=dp.pr.sky).items()} for dp in dpb] for dpb in dps]
        fin_host = [torch.empty_like(p.final, device="cpu").pin_memory() for p in plans]   # (set up above)
        nf_host = [torch.empty_like(p.n_final, device="cpu").pin_memory() for p in plans]

        def e2e_step(k):
            g = k % G
            for dp, h in zip(dps[g], host[g]):
                for name, t in h.items():
                    getattr(dp, name).copy_(t, non_blocking=True)
            for dp in dps[g]:
                dp.prepare()
            fin, nf = launch(g)
            fin_host[g].copy_(fin, non_blocking=True)
            nf_host[g].copy_(nf, non_blocking=True)

        h2d = [sum(t.numel() * t.element_size() for h in hb for t in h.values()) for hb in host]
        d2h = [fin_host[g].numel() * fin_host[g].element_size() + nf_host[g].numel() * nf_host[g].element_size()
               for g in range(G)]
        for g in range(G):
            e2e_step(g)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for k in range(args.steps):
            e2e_step(k)
        a1.record(stream)
        torch.cuda.synchronize()
        te = max_over_ranks(a0.elapsed_time(a1) / 1e3, "cuda")
        e2e = {"value": weak_value(terms_rank, world, te), "unit": UNIT,
               "h2d_bytes_per_step": int(round(np.mean([h2d[k % G] for k in range(args.steps)]))),
               "d2h_bytes_per_step": int(round(np.mean([d2h[k % G] for k in range(args.steps)]))),
               "steps": args.steps}

    # ---- plain form (FP64 track per term, FP64 weights, one launch per patch) on a bounded sample
    plain = None
    if not args.no_plain and rank == 0:
        subs = [first_points(p) for p in batches[0]]
        dps_p = [bsh.DeviceProblem(s, w_dtype="f64") for s in subs]
        for d in dps_p:
            d.prepare()
        pplan = bsh.Plan(dps_p, bsh.MODE_PLAIN, top_k=subs[0].top_k)
        pplan.number_count()
        torch.cuda.synchronize()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        pplan.number_count()
        b1.record(stream)
        torch.cuda.synchronize()
        tp = b0.elapsed_time(b1) / 1e3
        pt = sum(s.n_terms for s in subs)
        plain = {"value": pt / tp, "unit": UNIT, "ms": tp * 1e3,
                 "sample": f"plain form on the first 4 sky points of step group 0 in each of its {len(subs)} "
                           f"problem(s), all binaries, f0 and SFTs ({pt:.3g} terms; one launch per patch)"}
        pplan.close()

    # ---- roofline of the count kernel
    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    launch_s = sum(launch_ms) / 1e3
    count_rate = terms_rank / launch_s
    achieved_gbs = count_rate * 4.0 / 1e9
    peak_gbs = n_sm * 128.0 * f_max / 1e9
    traffic, traffic_src = profiled(args.workload, "traffic")
    roofline = {"bound": "smem", "achieved": achieved_gbs, "peak": peak_gbs, "unit": "GB/s",
                "frac": achieved_gbs / peak_gbs, "traffic": traffic, "traffic_source": traffic_src,
                "kernel": "count_batched (with the track-table kernels, the toplist merge and stage 2 of the "
                          "same launch: the timed unit is the graph)" if not args.eager else
                          "count_batched (with the track-table kernels, the toplist merge and stage 2)",
                "peak_source": f"derived: {n_sm} SMs x 32 banks x 4 B/clk x {f_max / 1e6:.0f} MHz "
                               f"(MEASURED_PEAKS sm_max_mhz); one 32-bit shared-memory word per term",
                "terms_per_s": count_rate, "launch_ms_mean": 1e3 * launch_s / args.steps,
                "launch_ms_median": float(np.median(launch_ms)) if launch_ms else None}
    if clocks.get("sm_mhz"):
        roofline["frac_at_observed_clock"] = count_rate / (n_sm * 32.0 * clocks["sm_mhz"] * 1e6)
    # the bit-level ceiling: one peakgram bit (1/8 B) of shared memory per term
    roofline["bit_ceiling"] = {"terms_per_s": n_sm * 128.0 * 8.0 * f_max,
                               "frac": count_rate / (n_sm * 128.0 * 8.0 * f_max)}
    # issue ceilings: 128 thread instructions per SM and clock, at the kernel's measured
    # instructions per term, and at one per term (the FP32 add of the weighted sum)
    ipt, ipt_src = profiled(args.workload, "ipt", args.track)
    issue = n_sm * 128.0 * f_max
    roofline["alu"] = {"ceiling_terms_per_s": issue / ipt if ipt else None, "instr_per_term": ipt,
                       "frac": count_rate * ipt / issue if ipt else None, "source": ipt_src,
                       "one_instr_per_term": {"terms_per_s": issue, "frac": count_rate / issue}}
    roofline["binding"] = "alu" if ipt else None

    cpu = None
    if not args.no_cpu and rank == 0:
        v, cores, sample = cpu_baseline_sample(batches[0][0])
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        cfg = workload_config(batches, args.workload) | {"parallelism": f"replicas x{world}", "track": args.track}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32+f32", "data": "synthetic",
                "config": cfg,
                "launch": {"graph": not args.eager, "groups": G, "tile": tiles[0],
                           "same_tile_all_groups": all(t == tiles[0] for t in tiles)},
                "clocks": {k: clocks.get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons")},
                "e2e": e2e, "gpu_launches": sum(launches_per_step(batches[k % G]) for k in range(args.steps)),
                "roofline": roofline, "stage2": stage2, "plain": plain, "cpu_baseline": cpu}
        print(json.dumps(line))
    for p in plans:
        p.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
