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
    for f in ("count.cu", "bsh_internal.cuh", "select.cuh"):
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
    for name, key in (("count_batched_mid.md", "traffic_bytes_per_launch"),
                      ("count_batched_small_full.md", "instr_per_term"),
                      ("count_batched_small_full.md", "lut_instr_per_term"),
                      ("count_batched_metric_bank.md", "instr_per_term"),
                      ("count_batched_metric_bank.md", "traffic_bytes_per_launch"),
                      ("count_batched_metric_bank.md", "traffic_bytes_per_launch_small")):
        text = open(os.path.join(ROOT, "profiles", name)).read()
        vals = dict(l.split(":", 1) for l in text.splitlines() if ":" in l and not l.startswith(("|", " ")))
        assert len(vals.get("kernel_source_sha256_16", "").strip()) == 16, name
        assert float(vals[key]) > 0, (name, key)


@pytest.mark.parametrize("kind", ["mid", "small", "eccentric", "metric-small"])
def test_workload_config(kind):
    pr = bench.make_problem(kind, 0, obank.template_bank)
    cfg = bench.workload_config(pr, kind)
    assert cfg["workload"].startswith(kind + ":")
    assert cfg["terms_per_step"] == pr.n_terms == pr.S * pr.B * pr.n_f0 * pr.N
    if kind.startswith("metric"):
        assert "metric bank" in cfg["workload"] and pr.orbit is not None
    sub = bench.plain_sample(kind, pr.sky, obank.template_bank)
    assert sub.S == 4 and sub.B == pr.B and sub.N == pr.N


def test_ranks_search_rotated_skies():
    pr0 = bench.make_problem("small", 0)
    pr1 = bench.make_problem("small", 1)
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
