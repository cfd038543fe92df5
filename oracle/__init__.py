"""FP64 CPU oracle for the BinarySkyHough number count -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It is a
thin ctypes wrapper around ``bsh_oracle.c`` (plain C, double precision,
``-ffp-contract=off``), which computes every quantity from the paper's
definitions template by template.  It shares no code with the CUDA path.

Parity status per function (each pinned by ``tests/test_oracle_*.py``):
  peakgram        pinned (numpy sliding median; Exp(1) peak density e^-1.6)
  antenna/weights pinned (closed forms, psi invariance, sky average 2/5, range)
  quantize        pinned (numpy float16, exact rational rounding)
  track           pinned (50-digit mpmath evaluation; a_p = 0 / v = 0 special cases;
                  period shift of t_asc; exact forced ties)
  ELL1 track      pinned (exact Keplerian orbit of Eq. (6)-(10) solved independently:
                  agreement to O(e^2); circular limit bitwise; t_asc period shift;
                  grid layout against single-orbit problems)
  count           pinned (all-ones / all-zeros peakgrams, single-bit hits, linearity,
                  SFT-permutation invariance, noise mean and variance, injection)
  significance    pinned (Monte-Carlo mean / variance of Bernoulli peakgrams)
  toplist         pinned (full numpy lexsort)
  power sum       pinned (rho = 1 gives sum w; linearity; single-bin rho)
  LUT count       pinned (block of one and zero modulation reduce to the exact track;
                  reference templates exact; shift direction; departure rate vs |(j - j_ref) D|)
  explicit banks  pinned (a grid written out as a bank counts the same)
  bank.py         pinned (Eq. (30)-(32) scalings, layout and spacings, coverage, the
                  paper's template-count scaling)
  postprocess.py  pinned (distance identities, scipy connected components, chains, cut /
                  centroid / best cluster, coincidences, ecliptic projection)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bsh_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile bsh_oracle.c into _build/liboracle.so (gcc, -ffp-contract=off)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Problem(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int), ("k_lo", ctypes.c_int), ("K", ctypes.c_int), ("W", ctypes.c_int),
        ("bits", ctypes.c_void_p), ("rho", ctypes.c_void_p), ("w", ctypes.c_void_p),
        ("v", ctypes.c_void_p), ("t", ctypes.c_void_p), ("F0", ctypes.c_double),
        ("n_f0", ctypes.c_int), ("S", ctypes.c_int), ("sky", ctypes.c_void_p),
        ("n_ap", ctypes.c_int), ("ap", ctypes.c_void_p), ("n_Om", ctypes.c_int),
        ("Om", ctypes.c_void_p), ("n_T", ctypes.c_int), ("Tasc", ctypes.c_void_p),
        ("rho_th", ctypes.c_double), ("tie_band", ctypes.c_double),
        ("n_kap", ctypes.c_int), ("kap", ctypes.c_void_p), ("n_eta", ctypes.c_int), ("eta", ctypes.c_void_p),
        ("lut_block", ctypes.c_int),
        ("n_orbit", ctypes.c_int), ("orbit", ctypes.c_void_p), ("n_bank", ctypes.c_int64),
        ("bank_orbit", ctypes.c_void_p), ("bank_ap", ctypes.c_void_p),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            d, i, i64, vp = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
            P = ctypes.POINTER(Problem)
            L.orc_running_median.restype = d
            L.orc_running_median.argtypes = [vp, i, i, i]
            L.orc_peakgram.restype = i
            L.orc_peakgram.argtypes = [vp, i, i, i, d, vp, vp, i]
            L.orc_antenna.restype = None
            L.orc_antenna.argtypes = [vp, vp, vp, d, vp, vp]
            L.orc_weights.restype = i
            L.orc_weights.argtypes = [vp, i, vp, vp, i, i, vp]
            L.orc_quantize.restype = None
            L.orc_quantize.argtypes = [vp, vp, ctypes.c_size_t, i]
            for name in ("orc_round_f16", "orc_round_bf16", "orc_round_f32"):
                getattr(L, name).restype = d
                getattr(L, name).argtypes = [d]
            L.orc_track_x.restype = d
            L.orc_track_x.argtypes = [d, vp, vp, d, d, d, d]
            L.orc_track_bin.restype = i64
            L.orc_track_bin.argtypes = [d, vp, vp, d, d, d, d, d, vp]
            L.orc_track_x_ell1.restype = d
            L.orc_track_x_ell1.argtypes = [d, vp, vp, d, d, d, d, d, d]
            L.orc_track_bin_ell1.restype = i64
            L.orc_track_bin_ell1.argtypes = [d, vp, vp, d, d, d, d, d, d, d, vp]
            L.orc_count_one.restype = i
            L.orc_count_one.argtypes = [P, i, i64, i, vp, vp, vp, vp, vp, vp, vp]
            L.orc_count_dense.restype = i
            L.orc_count_dense.argtypes = [P, i, i, vp, vp, vp, vp, vp, vp, vp]
            L.orc_significance.restype = d
            L.orc_significance.argtypes = [d, d, d, d]
            L.orc_topk.restype = i64
            L.orc_topk.argtypes = [vp, i64, i64, vp, vp]
            L.orc_power_sum.restype = i
            L.orc_power_sum.argtypes = [P, i, i64, i, vp]
            L.orc_power_significance.restype = d
            L.orc_power_significance.argtypes = [d, d, d]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


DTYPES = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}
TIE_BAND = 1e-9


# ---------------------------------------------------------------- peakgram

def peakgram(power, window: int, rho_th: float = 1.6, W: int | None = None):
    """Eq. (20): rho and the bit-packed 1/0 peakgram (uint32 rows of W words)."""
    power = _c(power, np.float32)
    N, K = power.shape
    if W is None:
        W = -(-K // 32)
    rho = np.empty((N, K), np.float32)
    bits = np.zeros((N, W), np.uint32)
    rc = lib().orc_peakgram(_ptr(power), N, K, window, rho_th, _ptr(rho), _ptr(bits), W)
    if rc:
        raise ValueError(f"orc_peakgram rc={rc}")
    return rho, bits


def running_median(row, window: int, k: int) -> float:
    row = _c(row, np.float32)
    return lib().orc_running_median(_ptr(row), row.size, window, k)


# ----------------------------------------------------------------- weights

def antenna(n, u, v, psi: float = 0.0):
    Fp, Fc = ctypes.c_double(), ctypes.c_double()
    n, u, v = (_c(x, np.float64) for x in (n, u, v))
    lib().orc_antenna(_ptr(n), _ptr(u), _ptr(v), psi, ctypes.byref(Fp), ctypes.byref(Fc))
    return Fp.value, Fc.value


def weights(sky, arms, Sn, norm: bool = True):
    """Eq. (22) FP64 weights [S][N]."""
    sky, arms, Sn = _c(sky, np.float64), _c(arms, np.float64), _c(Sn, np.float64)
    S, N = sky.shape[0], Sn.size
    w = np.empty((S, N))
    rc = lib().orc_weights(_ptr(sky), S, _ptr(arms), _ptr(Sn), N, int(norm), _ptr(w))
    if rc:
        raise ValueError(f"orc_weights rc={rc}")
    return w


def quantize(w, dtype: str):
    """Round FP64 weights to f32/f16/bf16 (ties to even); returns float64 values."""
    w = _c(w, np.float64)
    out = np.empty_like(w)
    lib().orc_quantize(_ptr(w), _ptr(out), w.size, DTYPES[dtype])
    return out


# ------------------------------------------------------------------- track

def track_x(F, v, n, ap, Om, Tasc, t) -> float:
    v, n = _c(v, np.float64), _c(n, np.float64)
    return lib().orc_track_x(F, _ptr(v), _ptr(n), ap, Om, Tasc, t)


def track_bin(F, v, n, ap, Om, Tasc, t, tie_band: float = TIE_BAND):
    v, n = _c(v, np.float64), _c(n, np.float64)
    tie = ctypes.c_int()
    k = lib().orc_track_bin(F, _ptr(v), _ptr(n), ap, Om, Tasc, t, tie_band, ctypes.byref(tie))
    return int(k), bool(tie.value)


def track_x_ell1(F, v, n, ap, Om, Tasc, kap, eta, t) -> float:
    v, n = _c(v, np.float64), _c(n, np.float64)
    return lib().orc_track_x_ell1(F, _ptr(v), _ptr(n), ap, Om, Tasc, kap, eta, t)


def track_bin_ell1(F, v, n, ap, Om, Tasc, kap, eta, t, tie_band: float = TIE_BAND):
    v, n = _c(v, np.float64), _c(n, np.float64)
    tie = ctypes.c_int()
    k = lib().orc_track_bin_ell1(F, _ptr(v), _ptr(n), ap, Om, Tasc, kap, eta, t, tie_band, ctypes.byref(tie))
    return int(k), bool(tie.value)


# ----------------------------------------------------------------- counting

class OracleProblem:
    """Holds contiguous arrays alive for the ctypes struct."""

    def __init__(self, *, bits, w, v, t, F0, n_f0, sky, a_p, Omega, T_asc, k_lo, K, rho=None,
                 rho_th: float = 1.6, tie_band: float = TIE_BAND, kappa=None, eta=None, lut_block: int = 0,
                 orbit=None, bank_orbit=None, bank_ap=None):
        """Binary templates: the a_p x Omega x t_asc (x kappa x eta) grid, or with
        ``orbit`` ([R][4]: Omega, t_asc, kappa, eta) an explicit bank where template b
        has a_p = bank_ap[b] on orbit row bank_orbit[b] (then a_p / Omega / T_asc are
        not used and may be empty)."""
        self.bits = _c(bits, np.uint32)
        self.w = _c(w, np.float64)
        self.v = _c(v, np.float64)
        self.t = _c(t, np.float64)
        self.sky = _c(sky, np.float64)
        self.ap = _c(a_p, np.float64)
        self.Om = _c(Omega, np.float64)
        self.Tasc = _c(T_asc, np.float64)
        self.rho = None if rho is None else _c(rho, np.float32)
        N, W = self.bits.shape
        self.n_T = self.Tasc.shape[1] if self.Tasc.ndim == 2 else self.Tasc.size // self.Om.size
        self.kap = None if kappa is None else _c(kappa, np.float64)
        self.eta = None if eta is None else _c(eta, np.float64)
        nk = 1 if self.kap is None else self.kap.size
        ne = 1 if self.eta is None else self.eta.size
        self.B = self.ap.size * self.Om.size * self.n_T * nk * ne
        self.orbit = None if orbit is None else _c(orbit, np.float64).reshape(-1, 4)
        self.bank_orbit = None if bank_orbit is None else _c(bank_orbit, np.int32)
        self.bank_ap = None if bank_ap is None else _c(bank_ap, np.float64)
        if self.orbit is not None:
            self.B = self.bank_ap.size
        self.S = self.sky.shape[0]
        self.n_f0 = int(n_f0)
        self.N = N
        self.rho_th = rho_th
        self.c = Problem(N=N, k_lo=int(k_lo), K=int(K), W=W, bits=self.bits.ctypes.data,
                         rho=None if self.rho is None else self.rho.ctypes.data, w=self.w.ctypes.data,
                         v=self.v.ctypes.data, t=self.t.ctypes.data, F0=float(F0), n_f0=self.n_f0,
                         S=self.S, sky=self.sky.ctypes.data, n_ap=self.ap.size, ap=self.ap.ctypes.data,
                         n_Om=self.Om.size, Om=self.Om.ctypes.data, n_T=self.n_T,
                         Tasc=self.Tasc.ctypes.data, rho_th=float(rho_th), tie_band=float(tie_band),
                         n_kap=0 if self.kap is None else self.kap.size,
                         kap=None if self.kap is None else self.kap.ctypes.data,
                         n_eta=0 if self.eta is None else self.eta.size,
                         eta=None if self.eta is None else self.eta.ctypes.data,
                         lut_block=int(lut_block),
                         n_orbit=0 if self.orbit is None else self.orbit.shape[0],
                         orbit=None if self.orbit is None else self.orbit.ctypes.data,
                         n_bank=0 if self.orbit is None else self.bank_ap.size,
                         bank_orbit=None if self.orbit is None else self.bank_orbit.ctypes.data,
                         bank_ap=None if self.orbit is None else self.bank_ap.ctypes.data)

    def count_one(self, s: int, b: int, j: int):
        nu, nw, nt = ctypes.c_int32(), ctypes.c_double(), ctypes.c_int32()
        lo, hi, wl, wh = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double(), ctypes.c_double()
        rc = lib().orc_count_one(ctypes.byref(self.c), s, b, j, ctypes.byref(nu), ctypes.byref(nw),
                                 ctypes.byref(nt), ctypes.byref(lo), ctypes.byref(hi),
                                 ctypes.byref(wl), ctypes.byref(wh))
        if rc:
            raise ValueError(f"orc_count_one rc={rc}")
        return dict(n_unw=nu.value, n_w=nw.value, n_tie=nt.value, unw_lo=lo.value,
                    unw_hi=hi.value, w_lo=wl.value, w_hi=wh.value)

    def count_dense(self, s_begin: int = 0, s_end: int | None = None):
        """All templates of sky points [s_begin, s_end) -> dict of [S', B, n_f0] arrays."""
        if s_end is None:
            s_end = self.S
        shape = (s_end - s_begin, self.B, self.n_f0)
        n = int(np.prod(shape))
        out = dict(n_unw=np.empty(n, np.int32), n_w=np.empty(n), n_tie=np.empty(n, np.int32),
                   unw_lo=np.empty(n, np.int32), unw_hi=np.empty(n, np.int32),
                   w_lo=np.empty(n), w_hi=np.empty(n))
        rc = lib().orc_count_dense(ctypes.byref(self.c), s_begin, s_end, *[_ptr(out[k]) for k in
                                   ("n_unw", "n_w", "n_tie", "unw_lo", "unw_hi", "w_lo", "w_hi")])
        if rc:
            raise ValueError(f"orc_count_dense rc={rc}")
        return {k: a.reshape(shape) for k, a in out.items()}

    def power_sum(self, s: int, b: int, j: int) -> float:
        P = ctypes.c_double()
        rc = lib().orc_power_sum(ctypes.byref(self.c), s, b, j, ctypes.byref(P))
        if rc:
            raise ValueError(f"orc_power_sum rc={rc}")
        return P.value


def significance(n, sum_w, sum_w2, rho_th: float = 1.6):
    """Eq. (25) elementwise (n array, sums broadcast)."""
    n = np.asarray(n, dtype=np.float64)
    sw = np.broadcast_to(np.asarray(sum_w, dtype=np.float64), n.shape)
    sw2 = np.broadcast_to(np.asarray(sum_w2, dtype=np.float64), n.shape)
    f = lib().orc_significance
    return np.array([f(float(a), float(b), float(c), rho_th) for a, b, c in
                     zip(n.ravel(), sw.ravel(), sw2.ravel())]).reshape(n.shape)


def power_significance(P, sum_w, sum_w2):
    return lib().orc_power_significance(float(P), float(sum_w), float(sum_w2))


def topk(scores, k: int):
    """Per-patch toplist: ids (template order within the patch) and scores."""
    scores = _c(scores, np.float64).ravel()
    ids = np.empty(min(k, scores.size), np.int64)
    sc = np.empty(ids.size)
    m = lib().orc_topk(_ptr(scores), scores.size, k, _ptr(ids), _ptr(sc))
    return ids[:m], sc[:m]
