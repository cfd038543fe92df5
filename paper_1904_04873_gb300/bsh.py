"""Thin ctypes binding to libbsh (include/bsh.h): argument marshalling only.

Device memory comes from PyTorch tensors; every step of the hot path runs in
the library's CUDA kernels.  Loading fails loudly when the library has not
been built (``python -m paper_1904_04873_gb300.build`` or
``__graft_entry__.build()``): there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbsh.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_RANGE, ERR_TIMEOUT, ERR_CUDA, ERR_WORKSPACE, ERR_STATE = range(7)
F64, F32, F16, BF16 = range(4)
MODE_BATCHED, MODE_PLAIN, MODE_LUT = 0, 1, 2
DTYPE_CODES = {"f64": F64, "f32": F32, "f16": F16, "bf16": BF16}


class BshError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = lib().bsh_error_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} (status {code})")


class Problem(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int), ("k_lo", ctypes.c_int), ("K", ctypes.c_int), ("W", ctypes.c_int),
        ("bits", ctypes.c_void_p), ("rho", ctypes.c_void_p), ("w", ctypes.c_void_p),
        ("w_dtype", ctypes.c_int),
        ("sum_w", ctypes.c_void_p), ("sum_w2", ctypes.c_void_p), ("v", ctypes.c_void_p),
        ("t", ctypes.c_void_p), ("v_max", ctypes.c_double), ("F0", ctypes.c_double),
        ("n_f0", ctypes.c_int), ("S", ctypes.c_int), ("sky", ctypes.c_void_p),
        ("n_patch", ctypes.c_int), ("patch_start", ctypes.c_void_p),
        ("n_ap", ctypes.c_int), ("a_p", ctypes.c_void_p),
        ("n_Om", ctypes.c_int), ("Omega", ctypes.c_void_p),
        ("n_T", ctypes.c_int), ("T_asc", ctypes.c_void_p),
        ("rho_th", ctypes.c_double),
        ("n_kappa", ctypes.c_int), ("kappa", ctypes.c_void_p),
        ("n_eta", ctypes.c_int), ("eta", ctypes.c_void_p),
        ("n_orbit", ctypes.c_int), ("orbit", ctypes.c_void_p),
        ("n_bank", ctypes.c_int), ("bank_orbit", ctypes.c_void_p), ("bank_ap", ctypes.c_void_p),
    ]


def _ecc_fields(pr, keep: dict) -> dict:
    """The eccentric grid (n_kappa / kappa / n_eta / eta) and the explicit bank
    (n_orbit / orbit / n_bank / bank_orbit / bank_ap) of a problem, as HOST
    arrays kept alive in ``keep``."""
    out = {}
    for name in ("kappa", "eta"):
        a = getattr(pr, name, None)
        if a is None:
            out["n_" + name], out[name] = 0, None
        else:
            keep[name] = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
            out["n_" + name], out[name] = keep[name].size, keep[name].ctypes.data
    orbit = getattr(pr, "orbit", None)
    if orbit is None:
        out.update(n_orbit=0, orbit=None, n_bank=0, bank_orbit=None, bank_ap=None)
    else:
        keep["orbit"] = np.ascontiguousarray(orbit, dtype=np.float64).reshape(-1, 4)
        keep["bank_orbit"] = np.ascontiguousarray(pr.bank_orbit, dtype=np.int32).reshape(-1)
        keep["bank_ap"] = np.ascontiguousarray(pr.bank_ap, dtype=np.float64).reshape(-1)
        out.update(n_orbit=keep["orbit"].shape[0], orbit=keep["orbit"].ctypes.data,
                   n_bank=keep["bank_ap"].size, bank_orbit=keep["bank_orbit"].ctypes.data,
                   bank_ap=keep["bank_ap"].ctypes.data)
    return out


class CountOptions(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("top_k", ctypes.c_int), ("threads", ctypes.c_int),
                ("sft_chunk", ctypes.c_int), ("ctas_per_sm", ctypes.c_int)]


class Cand(ctypes.Structure):
    _fields_ = [("template_id", ctypes.c_int64), ("s_h", ctypes.c_float), ("n_w", ctypes.c_float),
                ("n_unw", ctypes.c_int32), ("power", ctypes.c_float), ("s_p", ctypes.c_float),
                ("region", ctypes.c_int32)]


CAND_DTYPE = np.dtype([("template_id", "<i8"), ("s_h", "<f4"), ("n_w", "<f4"), ("n_unw", "<i4"),
                       ("power", "<f4"), ("s_p", "<f4"), ("region", "<i4")])
assert CAND_DTYPE.itemsize == ctypes.sizeof(Cand) == 32

_SIGS = {
    "bsh_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "bsh_version": (ctypes.c_int, []),
    "bsh_sync_status": (ctypes.c_int, [ctypes.c_void_p]),
    "bsh_make_peakgram": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "bsh_weights": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p]),
    "bsh_plan_create": (ctypes.c_int, [ctypes.POINTER(Problem), ctypes.c_int, ctypes.POINTER(CountOptions),
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "bsh_plan_destroy": (None, [ctypes.c_void_p]),
    "bsh_plan_workspace_size": (ctypes.c_size_t, [ctypes.c_void_p]),
    "bsh_plan_num_regions": (ctypes.c_int, [ctypes.c_void_p]),
    "bsh_plan_first_region": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "bsh_plan_bind": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "bsh_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "bsh_plan_set_accumulate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "bsh_plan_accumulate": (ctypes.c_int, [ctypes.c_void_p]),
    "bsh_plan_tile": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int)]),
    "bsh_number_count": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "bsh_count_dense": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "bsh_toplist": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "bsh_power_sum": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "bsh_graph_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "bsh_graph_reset": (ctypes.c_int, [ctypes.c_void_p]),
    "bsh_track_precision": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_void_p, ctypes.c_void_p]),
    "bsh_track_bins": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                      ctypes.c_void_p, ctypes.c_void_p]),
    "bsh_power_sum_static": (ctypes.c_int, [ctypes.POINTER(Problem), ctypes.c_void_p, ctypes.c_int,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "bsh_debug_track_windows": (ctypes.c_int, [ctypes.POINTER(Problem), ctypes.c_void_p, ctypes.c_int,
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "bsh_binary_resolution": (ctypes.c_int, [ctypes.c_double] * 8 + [ctypes.c_void_p] * 3),
    "bsh_plan_set_direct": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "bsh_plan_direct": (ctypes.c_int, [ctypes.c_void_p]),
    "bsh_plan_set_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "bsh_debug_pool_walk": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "bsh_cand_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "bsh_cluster_workspace": (ctypes.c_size_t, [ctypes.c_int]),
    "bsh_power_sum_sft": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "bsh_cluster": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "bsh_coincidence_workspace": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int]),
    "bsh_coincidences": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "bsh_template_bank": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
}


class PostParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("T_c", "T_obs", "v_over_c", "P_F", "m_a", "m_Om", "m_t", "obliquity",
                                               "d_cluster", "d_cut", "d_coinc")]


def post_params(**kw) -> PostParams:
    """bsh_post_params with the values of Sec. VI as defaults (clustering window sqrt(14)
    bins, coincidence window 3 bins, v/c = 1e-4, pixel factor 2, no cut)."""
    d = dict(T_c=900.0, T_obs=3.15e7, v_over_c=1e-4, P_F=2.0, m_a=1.0, m_Om=1.0, m_t=1.0,
             obliquity=0.40909280422232897, d_cluster=14.0 ** 0.5, d_cut=0.0, d_coinc=3.0)
    d.update(kw)
    return PostParams(**{k: float(v) for k, v in d.items()})


class BankSpec(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("f", "T_c", "T_obs", "t_mid", "ap_min", "ap_max", "P_min", "P_max",
                                               "m_a", "m_Om", "m_t", "ap_block")]


def lib():
    """Load libbsh.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libbsh.so not built ({LIB_PATH}); run paper_1904_04873_gb300/build.py")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != OK:
        raise BshError(rc, where)


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def sync_status(stream=None) -> int:
    """Synchronise the stream and return (and clear) the device status code."""
    return lib().bsh_sync_status(_stream(stream))


# ------------------------------------------------------------ (i) peakgram

def make_peakgram(power, median_window: int, rho_th: float = 1.6, W: Optional[int] = None,
                  want_rho: bool = True, out_bits=None, out_rho=None, stream=None):
    import torch
    assert power.is_cuda and power.dtype == torch.float32 and power.is_contiguous()
    N, K = power.shape
    if W is None:
        W = -(-K // 32)
        W = -(-W // 4) * 4
    bits = out_bits if out_bits is not None else torch.empty((N, W), dtype=torch.int32, device=power.device)
    rho = None
    if want_rho:
        rho = out_rho if out_rho is not None else torch.empty((N, K), dtype=torch.float32, device=power.device)
    _check(lib().bsh_make_peakgram(_ptr(power), N, K, median_window, float(rho_th), _ptr(rho), _ptr(bits), W,
                                   _stream(stream)), "bsh_make_peakgram")
    return rho, bits


# ------------------------------------------------------------- (ii) weights

def weights(sky, arms, Sn, normalize: bool = True, dtype: str = "f16", out=None, stream=None):
    import torch
    tdt = {"f64": torch.float64, "f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[dtype]
    S, N = sky.shape[0], Sn.shape[0]
    if out is None:
        w = torch.empty((S, N), dtype=tdt, device=sky.device)
        sw = torch.empty(S, dtype=torch.float64, device=sky.device)
        sw2 = torch.empty(S, dtype=torch.float64, device=sky.device)
    else:
        w, sw, sw2 = out
    _check(lib().bsh_weights(_ptr(sky), S, _ptr(arms), _ptr(Sn), N, int(normalize), DTYPE_CODES[dtype], _ptr(w),
                             _ptr(sw), _ptr(sw2), _stream(stream)), "bsh_weights")
    return w, sw, sw2


# -------------------------------------------------------- problems and plans

class DeviceProblem:
    """A synth.Problem resident on the GPU, with its peakgram and weights buffers."""

    def __init__(self, pr, device="cuda", w_dtype: str = "f16"):
        import torch
        self.pr = pr
        self.device = device
        f64 = dict(dtype=torch.float64, device=device)
        self.t = torch.as_tensor(pr.t, **f64)
        self.v = torch.as_tensor(pr.v, **f64).contiguous()
        self.arms = torch.as_tensor(pr.arms, **f64).contiguous()
        self.Sn = torch.as_tensor(pr.Sn, **f64)
        self.sky = torch.as_tensor(pr.sky, **f64).contiguous()
        self.power = torch.as_tensor(pr.power, dtype=torch.float32, device=device).contiguous()
        self.w_dtype = w_dtype
        self.v_max = float(np.max(np.linalg.norm(pr.v, axis=1))) * (1.0 + 1e-9)
        N, K, W, S = pr.N, pr.K, pr.W, pr.S
        self.bits = torch.empty((N, W), dtype=torch.int32, device=device)
        self.rho = torch.empty((N, K), dtype=torch.float32, device=device)
        tdt = {"f64": torch.float64, "f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[w_dtype]
        self.w = torch.empty((S, N), dtype=tdt, device=device)
        self.sum_w = torch.empty(S, **f64)
        self.sum_w2 = torch.empty(S, **f64)

    def prepare(self, stream=None):
        """Rows (i) and (ii): peakgram and weights from the resident inputs."""
        pr = self.pr
        make_peakgram(self.power, pr.median_window, pr.rho_th, pr.W, out_bits=self.bits, out_rho=self.rho,
                      stream=stream)
        weights(self.sky, self.arms, self.Sn, True, self.w_dtype, out=(self.w, self.sum_w, self.sum_w2),
                stream=stream)

    def descriptor(self) -> Problem:
        pr = self.pr
        self._ps = np.ascontiguousarray(pr.patch_start, dtype=np.int64)
        self._ap = np.ascontiguousarray(pr.a_p, dtype=np.float64)
        self._Om = np.ascontiguousarray(pr.Omega, dtype=np.float64)
        self._Ta = np.ascontiguousarray(pr.T_asc, dtype=np.float64)
        self._ecc = {}
        ecc = _ecc_fields(pr, self._ecc)
        return Problem(N=pr.N, k_lo=pr.k_lo, K=pr.K, W=pr.W, bits=_ptr(self.bits), rho=_ptr(self.rho),
                       w=_ptr(self.w), w_dtype=DTYPE_CODES[self.w_dtype], sum_w=_ptr(self.sum_w),
                       sum_w2=_ptr(self.sum_w2), v=_ptr(self.v), t=_ptr(self.t), v_max=self.v_max,
                       F0=float(pr.F0), n_f0=pr.n_f0, S=pr.S, sky=_ptr(self.sky),
                       n_patch=len(self._ps) - 1, patch_start=self._ps.ctypes.data,
                       n_ap=self._ap.size, a_p=self._ap.ctypes.data, n_Om=self._Om.size,
                       Omega=self._Om.ctypes.data, n_T=self._Ta.shape[1], T_asc=self._Ta.ctypes.data,
                       rho_th=float(pr.rho_th), **ecc)


class Plan:
    """bsh_plan with its workspace (a torch uint8 tensor) and output buffers."""

    def __init__(self, problems: Sequence[DeviceProblem], mode: int = MODE_BATCHED, top_k: int = 1000,
                 threads: int = 0, sft_chunk: int = 0, ctas_per_sm: int = 0, stream=None):
        import torch
        self.problems = list(problems)
        descs = (Problem * len(self.problems))(*[p.descriptor() for p in self.problems])
        self._descs = descs
        opt = CountOptions(mode=mode, top_k=top_k, threads=threads, sft_chunk=sft_chunk, ctas_per_sm=ctas_per_sm)
        h = ctypes.c_void_p()
        _check(lib().bsh_plan_create(descs, len(self.problems), ctypes.byref(opt), ctypes.byref(h)),
               "bsh_plan_create")
        self.h = h
        self.top_k = top_k
        self.mode = mode
        dev = self.problems[0].device
        self.ws_bytes = lib().bsh_plan_workspace_size(h)
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=dev)
        base = self.ws.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        _check(lib().bsh_plan_bind(h, ctypes.c_void_p(self._ws_ptr), self.ws_bytes, _stream(stream)), "bsh_plan_bind")
        self.regions = lib().bsh_plan_num_regions(h)
        self.cands = torch.zeros((self.regions, top_k, 32), dtype=torch.uint8, device=dev)
        self.n_cands = torch.zeros(self.regions, dtype=torch.int32, device=dev)
        self.final = None
        self.n_final = None

    def first_region(self, q: int) -> int:
        return lib().bsh_plan_first_region(self.h, q)

    def number_count(self, stream=None):
        _check(lib().bsh_number_count(self.h, _stream(stream)), "bsh_number_count")

    def count_dense(self, stream=None):
        import torch
        outs_u, outs_w = [], []
        for p in self.problems:
            pr = p.pr
            outs_u.append(torch.full((pr.S, pr.B, pr.n_f0), -1, dtype=torch.int32, device=p.device))
            outs_w.append(torch.full((pr.S, pr.B, pr.n_f0), float("nan"), dtype=torch.float32, device=p.device))
        pu = (ctypes.c_void_p * len(outs_u))(*[o.data_ptr() for o in outs_u])
        pw = (ctypes.c_void_p * len(outs_w))(*[o.data_ptr() for o in outs_w])
        _check(lib().bsh_count_dense(self.h, pu, pw, _stream(stream)), "bsh_count_dense")
        return outs_u, outs_w

    def toplist(self, stream=None):
        _check(lib().bsh_toplist(self.h, _ptr(self.cands), _ptr(self.n_cands), _stream(stream)), "bsh_toplist")
        return self.cands, self.n_cands

    def _final_buffers(self, n_cf):
        import torch
        if self.final is None or self.final.shape[1] != n_cf:
            dev = self.problems[0].device
            self.final = torch.zeros((self.regions, n_cf, 32), dtype=torch.uint8, device=dev)
            self.n_final = torch.zeros(self.regions, dtype=torch.int32, device=dev)

    def power_sum(self, n_cf: int, stream=None):
        self._final_buffers(n_cf)
        _check(lib().bsh_power_sum(self.h, _ptr(self.cands), _ptr(self.n_cands), n_cf, _ptr(self.final),
                                   _ptr(self.n_final), _stream(stream)), "bsh_power_sum")
        return self.final, self.n_final

    def power_sum_sft(self, stage1: "Plan", n_cf: int, stream=None):
        """bsh_power_sum_sft: stage 2 of stage1's lists with this plan's SFTs (the sliding set)."""
        self._final_buffers(n_cf)
        _check(lib().bsh_power_sum_sft(self.h, stage1.h, _ptr(stage1.cands), _ptr(stage1.n_cands), n_cf,
                                       _ptr(self.final), _ptr(self.n_final), _stream(stream)), "bsh_power_sum_sft")
        return self.final, self.n_final

    def graph_launch(self, n_cf: int, stream=None):
        self._final_buffers(n_cf)
        _check(lib().bsh_graph_launch(self.h, _ptr(self.cands), _ptr(self.n_cands), n_cf, _ptr(self.final),
                                      _ptr(self.n_final), _stream(stream)), "bsh_graph_launch")
        return self.final, self.n_final

    def set_direct(self, mode: int):
        """bsh_plan_set_direct: -1 automatic, 0 per-warp C values, 1 per-term C values."""
        _check(lib().bsh_plan_set_direct(self.h, mode), "bsh_plan_set_direct")
        return lib().bsh_plan_direct(self.h)

    def set_wait(self, polls: int = 0, skip_stage: int = -1):
        """bsh_plan_set_wait: the staging-barrier poll limit (0 = default) and the test hook
        that leaves one stage per CTA unissued (-1 = none)."""
        _check(lib().bsh_plan_set_wait(self.h, polls, skip_stage), "bsh_plan_set_wait")

    def autotune(self, stream=None):
        _check(lib().bsh_autotune(self.h, _stream(stream)), "bsh_autotune")
        return self.tile()

    def tile(self):
        t, c, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().bsh_plan_tile(self.h, ctypes.byref(t), ctypes.byref(c), ctypes.byref(g)), "bsh_plan_tile")
        return {"threads": t.value, "sft_chunk": c.value, "ctas": g.value,
                "accumulate": lib().bsh_plan_accumulate(self.h), "direct": lib().bsh_plan_direct(self.h)}

    def set_accumulate(self, variant: int):
        _check(lib().bsh_plan_set_accumulate(self.h, variant), "bsh_plan_set_accumulate")

    def track_precision(self, problem: int = 0, s_begin: int = 0, s_end: Optional[int] = None, stream=None):
        """Counts of (terms, single-precision bin mismatches, fixed-point mismatches, tie-band terms)."""
        import torch
        if s_end is None:
            s_end = self.problems[problem].pr.S
        c = torch.zeros(4, dtype=torch.int64, device=self.problems[problem].device)
        _check(lib().bsh_track_precision(self.h, problem, s_begin, s_end, _ptr(c), _stream(stream)),
               "bsh_track_precision")
        return [int(x) for x in c.cpu().tolist()]

    def track_bins(self, template_ids, problem: int = 0, stream=None):
        """Exact bins [n][N] of the listed templates (device int32)."""
        import torch
        ids = template_ids.contiguous()
        out = torch.empty((ids.numel(), self.problems[problem].pr.N), dtype=torch.int32, device=ids.device)
        _check(lib().bsh_track_bins(self.h, problem, _ptr(ids), ids.numel(), _ptr(out), _stream(stream)),
               "bsh_track_bins")
        return out

    def close(self):
        if self.h:
            lib().bsh_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def power_sum_static(dp: "DeviceProblem", template_ids, stream=None):
    """bsh_power_sum_static: P and s_P for a device int64 list of template ids,
    with the library's static scratch instead of a plan workspace."""
    import torch
    ids = template_ids.contiguous()
    n = ids.numel()
    power = torch.empty(n, dtype=torch.float32, device=ids.device)
    s_p = torch.empty(n, dtype=torch.float32, device=ids.device)
    d = dp.descriptor()
    _check(lib().bsh_power_sum_static(ctypes.byref(d), _ptr(ids), n, _ptr(power), _ptr(s_p), _stream(stream)),
           "bsh_power_sum_static")
    return power, s_p


def cands_to_numpy(cands, n) -> List[np.ndarray]:
    """Device toplists -> one structured numpy array per region."""
    raw = cands.cpu().numpy()
    nn = n.cpu().numpy()
    return [raw[r, :nn[r]].copy().view(CAND_DTYPE).reshape(-1) for r in range(raw.shape[0])]


def debug_track_windows(pr, queries: np.ndarray, rows: np.ndarray):
    """Host evaluation of the kernels' fixed-point windows (no GPU needed)."""
    q = np.ascontiguousarray(queries, dtype=np.int32)
    rows = np.ascontiguousarray(rows, dtype=np.uint32)
    n = q.shape[0]
    out = np.zeros(n, np.uint32)
    path = np.zeros(n, np.int32)
    arrs = dict(v=np.ascontiguousarray(pr.v), t=np.ascontiguousarray(pr.t), sky=np.ascontiguousarray(pr.sky),
                ap=np.ascontiguousarray(pr.a_p), Om=np.ascontiguousarray(pr.Omega),
                Ta=np.ascontiguousarray(pr.T_asc))
    v_max = float(np.max(np.linalg.norm(pr.v, axis=1))) * (1.0 + 1e-9)
    d = Problem(N=pr.N, k_lo=pr.k_lo, K=pr.K, W=pr.W, v=arrs["v"].ctypes.data, t=arrs["t"].ctypes.data,
                v_max=v_max, F0=float(pr.F0), n_f0=pr.n_f0, S=pr.S, sky=arrs["sky"].ctypes.data, n_patch=1,
                n_ap=arrs["ap"].size, a_p=arrs["ap"].ctypes.data, n_Om=arrs["Om"].size,
                Omega=arrs["Om"].ctypes.data, n_T=arrs["Ta"].shape[1], T_asc=arrs["Ta"].ctypes.data,
                rho_th=float(pr.rho_th), **_ecc_fields(pr, arrs))
    _check(lib().bsh_debug_track_windows(ctypes.byref(d), q.ctypes.data, n, rows.ctypes.data, out.ctypes.data,
                                         path.ctypes.data), "bsh_debug_track_windows")
    return out, path


def debug_pool_walk(plan_handle, pool: int = -1):
    """The batched schedule of a plan (a handle from bsh_plan_create): (number of pools, CTAs
    per pool, pool `pool`'s item indices in walk order, or None for pool -1).  No GPU needed."""
    npools, psize, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
    rc = lib().bsh_debug_pool_walk(plan_handle, max(pool, 0), None, 0, ctypes.byref(n), ctypes.byref(npools),
                                   ctypes.byref(psize))
    if pool < 0:
        if rc not in (OK, ERR_ARG):
            _check(rc, "bsh_debug_pool_walk")
        return npools.value, psize.value, None
    _check(rc, "bsh_debug_pool_walk")
    items = np.zeros(max(n.value, 1), np.int64)
    _check(lib().bsh_debug_pool_walk(plan_handle, pool, items.ctypes.data, items.size, ctypes.byref(n), None, None),
           "bsh_debug_pool_walk")
    return npools.value, psize.value, items[:n.value]


def binary_resolution(f, T_c, T_obs, a_p, Omega, m_a, m_Om, m_t):
    """bsh_binary_resolution: (d_ap, d_Om, d_t) of Eq. (30)-(32)."""
    out = [ctypes.c_double() for _ in range(3)]
    _check(lib().bsh_binary_resolution(f, T_c, T_obs, a_p, Omega, m_a, m_Om, m_t, *[ctypes.byref(o) for o in out]),
           "bsh_binary_resolution")
    return tuple(o.value for o in out)


def template_bank(**spec):
    """bsh_template_bank: (orbit [R][4], bank_orbit [B], bank_ap [B]) for a BankSpec."""
    sp = BankSpec(**{k: float(v) for k, v in spec.items()})
    nr, nb = ctypes.c_int(), ctypes.c_int()
    _check(lib().bsh_template_bank(ctypes.byref(sp), ctypes.byref(nr), None, 0, ctypes.byref(nb), None, None, 0),
           "bsh_template_bank")
    orbit = np.zeros((nr.value, 4))
    bo = np.zeros(nb.value, np.int32)
    ba = np.zeros(nb.value)
    _check(lib().bsh_template_bank(ctypes.byref(sp), ctypes.byref(nr), orbit.ctypes.data, orbit.shape[0],
                                   ctypes.byref(nb), bo.ctypes.data, ba.ctypes.data, bo.size), "bsh_template_bank")
    return orbit, bo, ba


def cand_params(plan: "Plan", problem: int, cands, n_cands, stat: int, pp: PostParams, stream=None):
    """bsh_cand_params: (params [n][6], sig [n], valid [n]) device tensors for one problem's lists."""
    import torch
    per_region = cands.shape[1]
    n_patch = len(plan.problems[problem].pr.patch_start) - 1
    n = n_patch * per_region
    dev = cands.device
    params = torch.empty((n, 6), dtype=torch.float64, device=dev)
    sig = torch.empty(n, dtype=torch.float64, device=dev)
    valid = torch.empty(n, dtype=torch.int32, device=dev)
    _check(lib().bsh_cand_params(plan.h, problem, _ptr(cands), _ptr(n_cands), per_region, stat, ctypes.byref(pp),
                                 _ptr(params), _ptr(sig), _ptr(valid), _stream(stream)), "bsh_cand_params")
    return params, sig, valid


def cluster(params, sig, valid, pp: PostParams, stream=None):
    """bsh_cluster: (label, keep, centroid, csig, best) device tensors."""
    import torch
    n = params.shape[0]
    dev = params.device
    work = torch.empty(max(1, lib().bsh_cluster_workspace(n)), dtype=torch.uint8, device=dev)
    label = torch.empty(n, dtype=torch.int32, device=dev)
    keep = torch.empty(n, dtype=torch.int32, device=dev)
    centroid = torch.empty((n, 6), dtype=torch.float64, device=dev)
    csig = torch.empty(n, dtype=torch.float64, device=dev)
    best = torch.empty(1, dtype=torch.int32, device=dev)
    _check(lib().bsh_cluster(_ptr(params), _ptr(sig), _ptr(valid), n, ctypes.byref(pp), _ptr(work), work.numel(),
                             _ptr(label), _ptr(keep), _ptr(centroid), _ptr(csig), _ptr(best), _stream(stream)),
           "bsh_cluster")
    return label, keep, centroid, csig, best


def coincidences(pa, sa, va, pb, sb, vb, pp: PostParams, cap: int, stream=None):
    """bsh_coincidences: (pairs [cap][2], centroid [cap][6], sig [cap], n_pairs [1]) device tensors."""
    import torch
    dev = pa.device
    na, nb = pa.shape[0], pb.shape[0]
    work = torch.empty(max(1, lib().bsh_coincidence_workspace(na, nb)), dtype=torch.uint8, device=dev)
    pairs = torch.empty((cap, 2), dtype=torch.int32, device=dev)
    cen = torch.empty((cap, 6), dtype=torch.float64, device=dev)
    sig = torch.empty(cap, dtype=torch.float64, device=dev)
    n_pairs = torch.zeros(1, dtype=torch.int32, device=dev)
    _check(lib().bsh_coincidences(_ptr(pa), _ptr(sa), _ptr(va), na, _ptr(pb), _ptr(sb), _ptr(vb), nb,
                                  ctypes.byref(pp), _ptr(work), work.numel(), _ptr(pairs), _ptr(cen), _ptr(sig),
                                  cap, _ptr(n_pairs), _stream(stream)), "bsh_coincidences")
    return pairs, cen, sig, n_pairs
