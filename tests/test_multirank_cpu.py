"""The N > 1 benchmark path on CPU: two gloo ranks, each searching its own
sky (the grid rotated by a rank-dependent angle) with the oracle, timing
reduced by max over ranks, and the whole-job value from all ranks' terms.
The shards share no template and together give the union of both searches.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_1904_04873_gb300 import synth
    w, r, lr = bench.rank_env()
    assert (w, r, lr) == (world, rank, rank)
    sky = bench.rank_sky(synth.fibonacci_sky(4), rank)
    pr = synth.mid(n_sky=4, n_per_det=30, n_ap=2, n_P=2, n_T=2, sky=sky, patch_size=2)
    rho, bits = oracle.peakgram(pr.power, pr.median_window, pr.rho_th, W=pr.W)
    wq = oracle.quantize(oracle.weights(pr.sky, pr.arms, pr.Sn), "f16")
    op = oracle.OracleProblem(bits=bits, w=wq, v=pr.v, t=pr.t, F0=pr.F0, n_f0=pr.n_f0, sky=pr.sky, a_p=pr.a_p,
                              Omega=pr.Omega, T_asc=pr.T_asc, k_lo=pr.k_lo, K=pr.K)
    d = op.count_dense()
    elapsed = 1.0 + rank                       # a stand-in per-rank time
    t_max = bench.max_over_ranks(elapsed)
    value = bench.weak_value(pr.n_terms, world, t_max)
    # gather the ranks' sky points (no data-path collective is used by the bench itself)
    allsky = [None] * world
    dist.all_gather_object(allsky, pr.sky.tolist())
    out[rank] = dict(t_max=t_max, value=value, terms=pr.n_terms, sky=allsky, n=int(d["n_unw"].sum()))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    r0, r1 = out[0], out[1]
    assert r0["t_max"] == r1["t_max"] == 2.0
    assert r0["value"] == pytest.approx(r0["terms"] * world / 2.0)
    s0, s1 = np.array(r0["sky"][0]), np.array(r0["sky"][1])
    assert not np.allclose(s0, s1)                      # distinct shards
    assert np.allclose(np.linalg.norm(s1, axis=1), 1.0)
    assert r0["n"] > 0 and r1["n"] > 0
