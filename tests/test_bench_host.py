"""Host logic of bench.py (no GPU): the summary stamp, workload descriptions, the
reference arm's JSON line."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from oracle import bank as obank  # noqa: E402


def test_code_only_ignores_comments_and_layout():
    a = "int f(int x) {  // doubles x\n    return 2 * x; /* no\n overflow */ }\n"
    b = "int f(int x) { return 2 * x; }"
    assert bench.code_only(a) == bench.code_only(b)
    assert bench.code_only(a) != bench.code_only("int f(int x) { return 3 * x; }")


def _fake_tree(tmp_path, body="int k;"):
    src = tmp_path / "paper_1904_04873_gb300" / "csrc"
    src.mkdir(parents=True)
    for f in ("count.cu", "count_tc.cu", "count_common.cuh", "bsh_internal.cuh", "select.cuh"):
        (src / f).write_text(f"// {f}\n{body}\n")
    (tmp_path / "profiles").mkdir()
    return src


def test_profile_value_follows_the_kernel_sources(tmp_path):
    src = _fake_tree(tmp_path)
    root = str(tmp_path)
    sha = bench.kernel_sha(root)
    (tmp_path / "profiles" / "k.md").write_text(f"# k\nkernel_source_sha256_16: {sha}\ninstr_per_term: 3.5\n")
    assert bench.profile_value("k.md", "instr_per_term", root) == (3.5, "profiles/k.md")
    assert bench.profile_value("k.md", "missing_key", root)[0] is None
    assert bench.profile_value("absent.md", "instr_per_term", root) == (None, None)
    # a comment edit keeps the stamp, a code edit makes the summary stale
    (src / "count.cu").write_text("// reworded\nint k;   \n")
    assert bench.kernel_sha(root) == sha
    (src / "count.cu").write_text("int k2;\n")
    v, why = bench.profile_value("k.md", "instr_per_term", root)
    assert v is None and "stale" in why


def test_committed_summaries_hold_the_figures_bench_reads():
    # (whether their stamp matches the current kernel is bench.py's business: a stale
    # summary gives null figures there, not a failure)
    for name, key in [e for ent in bench.PROFILES.values() for e in ent.values()]:
        text = open(os.path.join(ROOT, "profiles", name)).read()
        vals = dict(l.split(":", 1) for l in text.splitlines() if ":" in l and not l.startswith(("|", " ")))
        assert len(vals.get("kernel_source_sha256_16", "").strip()) == 16, name
        assert float(vals[key]) > 0, (name, key)


@pytest.mark.parametrize("kind", ["mid", "small", "eccentric", "metric-small"])
def test_workload_config(kind):
    batches = bench.workload_batches(kind, 0, obank.template_bank)
    assert len(batches) == 1 and len(batches[0]) == 1
    pr = batches[0][0]
    cfg = bench.workload_config(batches, kind)
    assert cfg["workload"].startswith(kind + ":")
    assert cfg["terms_per_step"] == cfg["terms_per_cycle"] == pr.n_terms == pr.S * pr.B * pr.n_f0 * pr.N
    if kind.startswith("metric"):
        assert "metric bank" in cfg["workload"] and pr.orbit is not None
    sub = bench.first_points(pr)
    assert sub.S == 4 and sub.B == pr.B and sub.N == pr.N and list(sub.patch_start) == [0, 4]
    assert bench.launches_per_step(batches[0]) == 8


def test_batching_workload_covers_the_configuration():
    # the default workload: the 64 uneven patches x 4 bands of the batching construction, dealt
    # into 8 step groups of about equal sky count that together hold every patch once
    from paper_1904_04873_gb300 import synth
    full = synth.batching()
    batches = bench.workload_batches("batching", 0)
    assert len(batches) == bench.N_GROUPS and all(len(b) == 4 for b in batches)
    sizes = np.diff(full[0].patch_start)
    assert sizes.size == 64 and sizes.min() >= 500 and sizes.max() <= 5000
    got = []
    for b in batches:
        for q, p in enumerate(b):
            assert p.N == full[q].N and p.n_f0 == full[q].n_f0 and p.B == full[q].B == 512
            assert np.array_equal(p.patch_start, b[0].patch_start)
        got.append(b[0].sky)
    sky = np.concatenate(got)
    assert sky.shape == full[0].sky.shape
    # every sky point of the construction exactly once
    key = lambda a: np.round(a, 12).view([("x", a.dtype), ("y", a.dtype), ("z", a.dtype)]).ravel()
    assert np.array_equal(np.sort(key(sky)), np.sort(key(full[0].sky)))
    S = np.array([b[0].S for b in batches])
    assert S.max() / S.min() < 1.1
    cfg = bench.workload_config(batches, "batching")
    assert cfg["terms_per_cycle"] == sum(p.n_terms for p in full)
    assert cfg["steps_per_cycle"] == 8 and cfg["workload"].startswith("batching:")
    assert bench.launches_per_step(batches[0]) == 20


def test_patch_groups_and_selection():
    from paper_1904_04873_gb300 import synth
    ps = np.array([0, 5, 7, 20, 21, 30])
    groups = synth.patch_groups(ps, 2)
    assert sorted(p for g in groups for p in g) == [0, 1, 2, 3, 4]
    pr = synth.mid(n_sky=30, n_per_det=20, n_ap=2, n_P=2, n_T=2, patch_size=30)
    import dataclasses
    pr = dataclasses.replace(pr, patch_start=ps)
    sub = synth.select_patches(pr, [2, 4])
    assert list(sub.patch_start) == [0, 13, 22]
    assert np.array_equal(sub.sky, np.concatenate([pr.sky[7:20], pr.sky[21:30]]))


def test_launcher_command():
    cmd = bench.launcher_command(4, ["--steps", "3"], 29555)
    assert cmd[1:4] == ["-m", "torch.distributed.run", "--nnodes=1"]
    assert "--nproc-per-node=4" in cmd and "--master-addr=127.0.0.1" in cmd and "--master-port=29555" in cmd
    assert cmd[-3:] == [os.path.join(ROOT, "bench.py"), "--steps", "3"]


def test_clock_summary():
    rows = [["0", "2070", "2070", "400", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
            ["0", "1980", "2070", "900", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
            ["0", "[N/A]", "2070"]]
    c = bench.summarize_clocks(rows)
    assert c["sm_mhz"] == 2025.0 and c["sm_max_mhz"] == 2070.0 and c["reasons"] == ["sw_power_cap"]
    assert c["samples"] == 2


def test_ranks_search_rotated_skies():
    pr0 = bench.make_problem("small", 0)
    pr1 = bench.make_problem("small", 1)
    b1 = bench.workload_batches("batching", 1)
    assert not np.allclose(b1[0][0].sky, bench.workload_batches("batching", 0)[0][0].sky)
    assert pr0.sky.shape == pr1.sky.shape and not np.allclose(pr0.sky, pr1.sky)
    assert np.allclose(np.linalg.norm(pr1.sky, axis=1), 1.0)


def test_reference_arm_prints_its_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "small", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "terms/s"
    assert line["metric"] == bench.METRIC and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "terms/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_relaunches_itself_for_two_ranks():
    # --gpus 2 outside torchrun: bench.py starts itself as two ranks (torch.distributed.run);
    # rank 0 times the oracle and prints the one line, rank 1 exits without work
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "small", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=900,
                       env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["config"]["parallelism"] == "replicas x2"
