"""C-ABI host logic, no GPU: exports, status strings, argument validation,
band / fixed-point range checks, workspace sizing and call-order errors."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1904_04873_gb300 import bsh, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1904_04873_gb300 import build
    build.build()


def header_functions():
    src = open(os.path.join(ROOT, "include", "bsh.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bsh_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_function():
    names = header_functions()
    assert len(names) >= 15
    L = bsh.lib()
    for n in names:
        assert hasattr(L, n), n


def test_version_and_strings():
    L = bsh.lib()
    assert L.bsh_version() >= 10000
    for code in range(7):
        assert len(L.bsh_error_string(code)) > 0


class FakeProblem:
    """Descriptor with fake (never dereferenced) device pointers, for plan_create."""

    def __init__(self, pr, **over):
        self.pr = pr
        self.ps = np.ascontiguousarray(pr.patch_start, np.int64)
        self.ap = np.ascontiguousarray(pr.a_p)
        self.Om = np.ascontiguousarray(pr.Omega)
        self.Ta = np.ascontiguousarray(pr.T_asc)
        fake = 1 << 20
        kw = dict(N=pr.N, k_lo=pr.k_lo, K=pr.K, W=pr.W, bits=fake, rho=fake, w=fake, w_dtype=bsh.F16,
                  sum_w=fake, sum_w2=fake, v=fake, t=fake,
                  v_max=float(np.max(np.linalg.norm(pr.v, axis=1))) * (1 + 1e-9), F0=pr.F0, n_f0=pr.n_f0,
                  S=pr.S, sky=fake, n_patch=len(self.ps) - 1, patch_start=self.ps.ctypes.data,
                  n_ap=self.ap.size, a_p=self.ap.ctypes.data, n_Om=self.Om.size, Omega=self.Om.ctypes.data,
                  n_T=self.Ta.shape[1], T_asc=self.Ta.ctypes.data, rho_th=1.6)
        kw.update(over)
        self.d = bsh.Problem(**kw)


def create(descs, **opt):
    o = dict(mode=bsh.MODE_BATCHED, top_k=100, threads=0, sft_chunk=0, ctas_per_sm=0)
    o.update(opt)
    arr = (bsh.Problem * len(descs))(*descs)
    h = ctypes.c_void_p()
    rc = bsh.lib().bsh_plan_create(arr, len(descs), ctypes.byref(bsh.CountOptions(**o)), ctypes.byref(h))
    return rc, h


@pytest.fixture(scope="module")
def small():
    return synth.mid(n_sky=20, n_per_det=40, n_ap=4, n_P=4, n_T=4, patch_size=5)


def test_valid_plan_and_workspace(small):
    fp = FakeProblem(small)
    rc, h = create([fp.d])
    assert rc == bsh.OK
    L = bsh.lib()
    ws = L.bsh_plan_workspace_size(h)
    assert ws > small.S * small.N * 8
    assert L.bsh_plan_num_regions(h) == 4
    assert L.bsh_plan_first_region(h, 0) == 0
    # call-order and workspace errors need no device
    assert L.bsh_number_count(h, None) == bsh.ERR_STATE
    assert L.bsh_plan_bind(h, None, ws, None) == bsh.ERR_WORKSPACE
    L.bsh_plan_destroy(h)


def test_wait_limit_arguments(small):
    fp = FakeProblem(small)
    rc, h = create([fp.d])
    assert rc == bsh.OK
    L = bsh.lib()
    assert L.bsh_plan_set_wait(h, -1, -1) == bsh.ERR_ARG
    assert L.bsh_plan_set_wait(h, 0, -2) == bsh.ERR_ARG
    assert L.bsh_plan_set_wait(h, 4096, 1) == bsh.OK
    assert L.bsh_plan_set_wait(h, 0, -1) == bsh.OK
    assert L.bsh_plan_set_wait(None, 0, -1) == bsh.ERR_ARG
    L.bsh_plan_destroy(h)


def test_tensor_accumulation_needs_the_exact_batched_256_thread_plan(small):
    L = bsh.lib()
    fp = FakeProblem(small)
    rc, h = create([fp.d])
    assert rc == bsh.OK and L.bsh_plan_set_accumulate(h, 2) == bsh.OK and L.bsh_plan_accumulate(h) == 2
    assert L.bsh_plan_set_accumulate(h, 3) == bsh.ERR_ARG
    L.bsh_plan_destroy(h)
    for opt in (dict(threads=128), dict(mode=bsh.MODE_LUT), dict(mode=bsh.MODE_PLAIN)):
        rc, h = create([fp.d], **opt)
        assert rc == bsh.OK
        assert L.bsh_plan_set_accumulate(h, 2) == bsh.ERR_ARG
        L.bsh_plan_destroy(h)


def test_plain_plan(small):
    fp = FakeProblem(small)
    rc, h = create([fp.d], mode=bsh.MODE_PLAIN)
    assert rc == bsh.OK
    bsh.lib().bsh_plan_destroy(h)


@pytest.mark.parametrize("field,value", [("W", 3), ("K", 0), ("N", 0), ("w_dtype", 7), ("F0", 1000.25),
                                         ("bits", 1 << 20 | 4), ("n_f0", 0), ("v_max", -1.0)])
def test_argument_errors(small, field, value):
    fp = FakeProblem(small, **{field: value})
    rc, _ = create([fp.d])
    assert rc == bsh.ERR_ARG


def test_options_errors(small):
    fp = FakeProblem(small)
    assert create([fp.d], top_k=0)[0] == bsh.ERR_ARG
    assert create([fp.d], top_k=20000)[0] == bsh.ERR_ARG
    assert create([fp.d], threads=96)[0] == bsh.ERR_ARG
    assert create([fp.d], sft_chunk=100)[0] == bsh.ERR_ARG
    assert create([fp.d], mode=5)[0] == bsh.ERR_ARG
    assert create([], top_k=10)[0] == bsh.ERR_ARG


def test_band_too_narrow_is_range_error(small):
    fp = FakeProblem(small, k_lo=small.k_lo + 10)
    assert create([fp.d])[0] == bsh.ERR_RANGE
    fp = FakeProblem(small, K=small.K - 12)
    assert create([fp.d])[0] == bsh.ERR_RANGE


def test_bad_patch_starts(small):
    fp = FakeProblem(small)
    bad = np.array([0, 7, 3, 20], np.int64)
    fp.d.patch_start = bad.ctypes.data
    fp.d.n_patch = 3
    assert create([fp.d])[0] == bsh.ERR_ARG
    bad2 = np.array([0, 10, 19], np.int64)
    fp.d.patch_start = bad2.ctypes.data
    fp.d.n_patch = 2
    assert create([fp.d])[0] == bsh.ERR_ARG


def test_multi_problem_regions():
    probs = synth.batching(n_patch=6, size_lo=5, size_hi=20, n_per_det=20, n_bin=2)
    fps = [FakeProblem(p) for p in probs]
    rc, h = create([f.d for f in fps])
    assert rc == bsh.OK
    L = bsh.lib()
    assert L.bsh_plan_num_regions(h) == 24
    assert [L.bsh_plan_first_region(h, q) for q in range(4)] == [0, 6, 12, 18]
    L.bsh_plan_destroy(h)


def test_peakgram_and_weights_argument_errors():
    L = bsh.lib()
    assert L.bsh_make_peakgram(None, 4, 100, 101, 1.6, None, 1 << 20, 4, None) == bsh.ERR_ARG
    assert L.bsh_make_peakgram(1 << 20, 4, 100, 0, 1.6, None, 1 << 20, 3, None) == bsh.ERR_ARG
    assert L.bsh_make_peakgram(1 << 20, 4, 200, 100, 1.6, None, 1 << 20, 8, None) == bsh.ERR_ARG
    assert L.bsh_weights(1 << 20, 3, 1 << 20, 1 << 20, 10, 1, 9, 1 << 20, None, None, None) == bsh.ERR_ARG


def test_bank_and_eccentric_plans_on_the_host(small):
    # explicit banks and eccentric grids are validated and planned without a GPU
    from oracle import bank as obank
    fp = FakeProblem(small)
    kap = np.array([-0.05, 0.0, 0.05])
    fk = FakeProblem(small, n_kappa=3, kappa=kap.ctypes.data, n_eta=1, eta=kap[1:2].ctypes.data)
    rc, h = create([fk.d])
    assert rc == bsh.OK
    bsh.lib().bsh_plan_destroy(h)
    bad = np.array([0.7])
    rc, _ = create([FakeProblem(small, n_kappa=1, kappa=bad.ctypes.data).d])
    assert rc == bsh.ERR_ARG
    pr = synth.metric(n_sky=4, n_per_det=40, patch_size=2)
    orbit, bo, ba = obank.template_bank(**synth.metric_spec(pr, m=6.4))
    fb = FakeProblem(pr, n_orbit=orbit.shape[0], orbit=orbit.ctypes.data, n_bank=bo.size,
                     bank_orbit=bo.ctypes.data, bank_ap=ba.ctypes.data)
    rc, h = create([fb.d])
    assert rc == bsh.OK
    L = bsh.lib()
    assert L.bsh_plan_direct(h) == 1          # warps span many orbit rows
    assert L.bsh_plan_set_direct(h, 2) == bsh.ERR_ARG
    assert L.bsh_plan_set_direct(h, 0) == bsh.OK and L.bsh_plan_direct(h) == 0
    L.bsh_plan_destroy(h)
    # a bank whose rows decrease, or that points past its rows, is refused
    bo2 = bo.copy()
    bo2[[0, 1]] = bo2[[1, 0]] + np.array([5, 0], np.int32)
    fb2 = FakeProblem(pr, n_orbit=orbit.shape[0], orbit=orbit.ctypes.data, n_bank=bo2.size,
                      bank_orbit=bo2.ctypes.data, bank_ap=ba.ctypes.data)
    assert create([fb2.d])[0] == bsh.ERR_ARG
    bo3 = bo.copy()
    bo3[-1] = orbit.shape[0]
    fb3 = FakeProblem(pr, n_orbit=orbit.shape[0], orbit=orbit.ctypes.data, n_bank=bo3.size,
                      bank_orbit=bo3.ctypes.data, bank_ap=ba.ctypes.data)
    assert create([fb3.d])[0] == bsh.ERR_ARG


def test_post_processing_argument_errors():
    # argument checks happen on the host before anything is enqueued
    L = bsh.lib()
    pp = bsh.post_params()
    fake = ctypes.c_void_p(1 << 20)
    assert L.bsh_cluster(fake, fake, fake, (1 << 20) + 1, ctypes.byref(pp), fake, 1 << 30, fake, fake, fake,
                         fake, fake, None) == bsh.ERR_ARG
    assert L.bsh_cluster(fake, fake, fake, 10, None, fake, 1 << 30, fake, fake, fake, fake, fake,
                         None) == bsh.ERR_ARG
    assert L.bsh_cluster(fake, fake, fake, 10, ctypes.byref(pp), fake, 16, fake, fake, fake, fake, fake,
                         None) == bsh.ERR_WORKSPACE
    bad = bsh.post_params(T_c=-1.0)
    assert L.bsh_coincidences(fake, fake, fake, 5, fake, fake, fake, 5, ctypes.byref(bad), fake, 1 << 20, fake,
                              fake, fake, 10, fake, None) == bsh.ERR_ARG
    assert L.bsh_cluster_workspace(1000) >= 1000 * 120
    assert L.bsh_coincidence_workspace(10, 20) >= 30 * 48
    assert L.bsh_cand_params(None, 0, fake, fake, 10, 0, ctypes.byref(pp), fake, fake, fake, None) == \
        bsh.ERR_STATE
    assert L.bsh_power_sum_sft(None, None, fake, fake, 10, fake, fake, None) == bsh.ERR_STATE
