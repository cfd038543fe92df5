"""Seeded synthetic inputs for the BinarySkyHough number count.

This module only *makes inputs*: SFT mid-times, detector velocities and arm
orientations from an analytic Earth orbit + spin model, sky grids, binary
template grids, noise spectrograms and the loaded frequency band.  It holds
none of the method's arithmetic (no track, no peakgram, no weights, no
count), so both the CUDA path and the CPU oracle can draw on it.

The paper's searches run on LIGO O1 SFTs (Sec. VI); those data are not
available here, so every workload is synthetic, with the shapes the paper
uses: T_c = 900 s SFTs spread over the run (Sec. IV.A), 0.1 Hz bands,
sky patches of 49 or 169 points (Sec. V.F, Table I), and circular-orbit
binary parameters (a_p, P = 2*pi/Omega, t_asc) with t_asc restricted to
one period around the mid-time (Eq. (35)).

Units: times in seconds relative to the run mid-time, velocities in units
of c, a_p in light-seconds, Omega in rad/s, frequencies expressed as bin
numbers F = f * T_c.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

C_LIGHT = 299792458.0
AU = 1.495978707e11
DAY = 86400.0
YEAR_SID = 365.256363004 * DAY
OMEGA_EARTH = 7.2921150e-5          # sidereal rotation rate, rad/s
R_EARTH = 6.371e6
OBLIQUITY = math.radians(23.4393)

SEED_NOISE = 1904
SEED_INJ = 4873
SEED_SKY = 473

# Site latitude / longitude (deg) and arm azimuths (deg, from North
# through East).  Approximations of the two LIGO sites; synthetic data.
SITES = {
    "H1": dict(lat=46.455, lon=-119.408, az_x=324.0, az_y=234.0),
    "L1": dict(lat=30.563, lon=-90.774, az_x=252.3, az_y=162.3),
}


# --------------------------------------------------------------------------
# time stamps, velocities, arms
# --------------------------------------------------------------------------

def sft_mid_times(n: int, T_sft: float, span: float, rng: Optional[np.random.Generator] = None) -> np.ndarray:
    """Mid-times of ``n`` SFTs over ``span`` seconds centred on t = 0.

    With ``rng`` None the SFTs are evenly spread; otherwise start times are
    drawn uniformly (seeded) and sorted, as for a real duty-cycled run.
    """
    if rng is None:
        step = span / n
        return (np.arange(n) + 0.5) * step - 0.5 * span
    starts = np.sort(rng.uniform(-0.5 * span, 0.5 * span - T_sft, size=n))
    return starts + 0.5 * T_sft


def _site_angle(t: np.ndarray, site: dict, theta0: float) -> np.ndarray:
    return theta0 + OMEGA_EARTH * t + math.radians(site["lon"])


def detector_velocity(t: np.ndarray, site_name: str, lam0: float = 0.3, theta0: float = 1.1,
                      orbit_only: bool = False) -> np.ndarray:
    """Detector velocity / c in the equatorial frame at times ``t``.

    Circular Earth orbit of radius 1 AU (sidereal year) rotated by the
    obliquity, plus the site's rotational velocity.  With ``orbit_only`` the
    ecliptic-frame orbital velocity is returned unrotated and without spin,
    so every vector lies in the xy-plane (used to force exact bin ties).
    """
    t = np.asarray(t, dtype=np.float64)
    site = SITES[site_name]
    v_orb = 2.0 * math.pi * AU / YEAR_SID / C_LIGHT
    lam = lam0 + 2.0 * math.pi * t / YEAR_SID
    ex, ey = -np.sin(lam) * v_orb, np.cos(lam) * v_orb
    out = np.zeros((t.size, 3))
    if orbit_only:
        out[:, 0], out[:, 1] = ex, ey
        return out
    ce, se = math.cos(OBLIQUITY), math.sin(OBLIQUITY)
    out[:, 0] = ex
    out[:, 1] = ey * ce
    out[:, 2] = ey * se
    lat = math.radians(site["lat"])
    th = _site_angle(t, site, theta0)
    v_rot = OMEGA_EARTH * R_EARTH * math.cos(lat) / C_LIGHT
    out[:, 0] += -np.sin(th) * v_rot
    out[:, 1] += np.cos(th) * v_rot
    return out


def detector_arms(t: np.ndarray, site_name: str, theta0: float = 1.1) -> np.ndarray:
    """Unit vectors of the x and y arms in the equatorial frame: [N][6]."""
    t = np.asarray(t, dtype=np.float64)
    site = SITES[site_name]
    lat = math.radians(site["lat"])
    th = _site_angle(t, site, theta0)
    east = np.stack([-np.sin(th), np.cos(th), np.zeros_like(th)], axis=1)
    north = np.stack([-math.sin(lat) * np.cos(th), -math.sin(lat) * np.sin(th),
                      np.full_like(th, math.cos(lat))], axis=1)
    out = np.empty((t.size, 6))
    for k, key in enumerate(("az_x", "az_y")):
        az = math.radians(site[key])
        out[:, 3 * k:3 * k + 3] = math.cos(az) * north + math.sin(az) * east
    return out


def fibonacci_sky(S: int) -> np.ndarray:
    """Near-uniform sky grid of S unit vectors (declination-ordered)."""
    k = np.arange(S, dtype=np.float64)
    z = 1.0 - (2.0 * k + 1.0) / S
    phi = k * math.pi * (3.0 - math.sqrt(5.0))
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


# --------------------------------------------------------------------------
# spectrogram powers
# --------------------------------------------------------------------------

def exp_rho(N: int, K: int, rng: np.random.Generator) -> np.ndarray:
    """Normalised powers rho ~ Exp(1) (Gaussian noise, Sec. V.F), float32."""
    return (-np.log1p(-rng.random((N, K)))).astype(np.float32)


def gaussian_power(Sn: np.ndarray, K: int, rng: np.random.Generator) -> np.ndarray:
    """|x~|^2 of complex Gaussian noise with variance Sn[i] per SFT, float32."""
    N = Sn.size
    re = rng.standard_normal((N, K))
    im = rng.standard_normal((N, K))
    return (0.5 * (re * re + im * im) * Sn[:, None]).astype(np.float32)


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Problem:
    """One frequency band searched over a sky set and a binary grid."""
    name: str
    T_sft: float
    t: np.ndarray            # [N] SFT mid-times (s, relative to the run mid-time)
    v: np.ndarray            # [N][3] detector velocity / c
    arms: np.ndarray         # [N][6] x- and y-arm unit vectors
    Sn: np.ndarray           # [N] noise level per SFT
    det: np.ndarray          # [N] detector index
    sky: np.ndarray          # [S][3]
    patch_start: np.ndarray  # [P+1]
    a_p: np.ndarray          # [n_ap] (light-s)
    Omega: np.ndarray        # [n_Om] (rad/s)
    T_asc: np.ndarray        # [n_Om][n_T] (s)
    F0: float                # first f0 template, bins (integer or half-integer)
    n_f0: int
    k_lo: int
    K: int
    W: int
    power: np.ndarray        # [N][K] float32 input powers (or rho when median_window == 0)
    median_window: int       # 101, or 0 when ``power`` already holds rho
    rho_th: float = 1.6
    top_k: int = 1000
    kappa: Optional[np.ndarray] = None   # [n_kap] e cos(omega) (Eq. (14)); None: circular orbits
    eta: Optional[np.ndarray] = None     # [n_eta] e sin(omega)
    # explicit binary bank (replaces the grid above when set): orbit rows [R][4]
    # (Omega, t_asc, kappa, eta) and, per binary template, its row and a_p
    orbit: Optional[np.ndarray] = None
    bank_orbit: Optional[np.ndarray] = None
    bank_ap: Optional[np.ndarray] = None

    @property
    def N(self) -> int:
        return int(self.t.size)

    @property
    def S(self) -> int:
        return int(self.sky.shape[0])

    @property
    def B(self) -> int:
        if self.orbit is not None:
            return int(np.size(self.bank_ap))
        nk = 1 if self.kappa is None else int(np.size(self.kappa))
        ne = 1 if self.eta is None else int(np.size(self.eta))
        return int(self.a_p.size * self.T_asc.size * nk * ne)

    @property
    def n_templates(self) -> int:
        return self.S * self.B * self.n_f0

    @property
    def n_terms(self) -> int:
        return self.n_templates * self.N


def band_for(F_min: float, F_max: float, v_max: float, ap_max: float, Om_max: float,
             min_K: int = 0, ecc_max: float = 0.0):
    """Loaded band [k_lo, k_lo+K) covering every track, plus words per row.

    The margin bounds |F*(v.n - a_p*Omega*g)| + 2 bins with |g| <= 1 + ecc_max
    (ecc_max = max|kappa| + max|eta|); K is widened to at least ``min_K`` (the
    running-median window) and W padded to 4 words.
    """
    margin = int(math.ceil(F_max * (v_max + ap_max * Om_max * (1.0 + ecc_max)))) + 2
    k_lo = int(math.floor(F_min)) - margin
    k_hi = int(math.floor(F_max)) + 1 + margin
    K = k_hi - k_lo + 1
    if K < min_K:
        extra = min_K - K
        k_lo -= extra // 2
        K = min_K
    W = -(-K // 32)
    W = -(-W // 4) * 4
    return k_lo, K, W


def _tasc_grid(Omega: np.ndarray, n_T: int) -> np.ndarray:
    P = 2.0 * math.pi / Omega
    j = np.arange(n_T, dtype=np.float64)
    return -0.5 * P[:, None] + j[None, :] * (P[:, None] / n_T)


def _patches(S: int, size: int) -> np.ndarray:
    edges = list(range(0, S, size)) + [S]
    return np.asarray(edges, dtype=np.int64)


def make_problem(name: str, *, n_per_det: int, dets: List[str], T_sft: float, span: float,
                 random_times: bool, f_lo: float, n_f0: int, half_bin: bool,
                 sky: np.ndarray, patch_size: int, a_p: np.ndarray, P_days: np.ndarray,
                 n_T: int, power_kind: str, seed: int = SEED_NOISE, top_k: int = 1000,
                 orbit_only: bool = False, sn_ratio: Optional[float] = None,
                 patch_start: Optional[np.ndarray] = None, kappa: Optional[np.ndarray] = None,
                 eta: Optional[np.ndarray] = None) -> Problem:
    rng = np.random.default_rng(seed)
    ts, vs, arms, Sns, detidx = [], [], [], [], []
    if sn_ratio is None:
        sn_ratio = float(rng.uniform(1.0, 1.5))
    for d, dn in enumerate(dets):
        t = sft_mid_times(n_per_det, T_sft, span, rng if random_times else None)
        ts.append(t)
        vs.append(detector_velocity(t, dn, orbit_only=orbit_only))
        arms.append(detector_arms(t, dn))
        Sns.append(np.full(t.size, 1.0 if d == 0 else sn_ratio))
        detidx.append(np.full(t.size, d, dtype=np.int32))
    t = np.concatenate(ts)
    v = np.concatenate(vs)
    arm = np.concatenate(arms)
    Sn = np.concatenate(Sns)
    det = np.concatenate(detidx)
    Omega = 2.0 * math.pi / (np.asarray(P_days, dtype=np.float64) * DAY)
    T_asc = _tasc_grid(Omega, n_T)
    F0 = math.floor(f_lo * T_sft) + (0.5 if half_bin else 0.0)
    v_max = float(np.max(np.linalg.norm(v, axis=1)))
    ecc_max = (0.0 if kappa is None else float(np.max(np.abs(kappa)))) + \
        (0.0 if eta is None else float(np.max(np.abs(eta))))
    k_lo, K, W = band_for(F0, F0 + n_f0 - 1, v_max, float(np.max(a_p)), float(np.max(Omega)),
                          min_K=101 if power_kind == "gauss" else 0, ecc_max=ecc_max)
    prng = np.random.default_rng(seed + 17)
    if power_kind == "exp":
        power = exp_rho(t.size, K, prng)
        mw = 0
    elif power_kind == "gauss":
        power = gaussian_power(Sn, K, prng)
        mw = 101
    else:
        raise ValueError(power_kind)
    if patch_start is None:
        patch_start = _patches(sky.shape[0], patch_size)
    return Problem(name=name, T_sft=T_sft, t=t, v=v, arms=arm, Sn=Sn, det=det, sky=sky,
                   patch_start=np.asarray(patch_start, dtype=np.int64), a_p=np.asarray(a_p, dtype=np.float64),
                   Omega=Omega, T_asc=T_asc, F0=float(F0), n_f0=int(n_f0), k_lo=k_lo, K=K, W=W,
                   power=power, median_window=mw, top_k=top_k,
                   kappa=None if kappa is None else np.asarray(kappa, dtype=np.float64),
                   eta=None if eta is None else np.asarray(eta, dtype=np.float64))


def grid_as_bank(pr: Problem) -> Problem:
    """The same problem with its binary grid written out as an explicit bank, in the
    grid's template order b = (((iOm * n_T + iT) * n_kap + ik) * n_eta + ie) * n_ap + iap."""
    kap = np.zeros(1) if pr.kappa is None else np.asarray(pr.kappa, dtype=np.float64)
    eta = np.zeros(1) if pr.eta is None else np.asarray(pr.eta, dtype=np.float64)
    n_T = pr.T_asc.shape[1]
    rows = []
    for iOm in range(pr.Omega.size):
        for iT in range(n_T):
            for k in kap:
                for e in eta:
                    rows.append((pr.Omega[iOm], pr.T_asc[iOm, iT], k, e))
    orbit = np.array(rows, dtype=np.float64)
    n_ap = pr.a_p.size
    bank_orbit = np.repeat(np.arange(orbit.shape[0], dtype=np.int32), n_ap)
    bank_ap = np.tile(np.asarray(pr.a_p, dtype=np.float64), orbit.shape[0])
    return dataclasses.replace(pr, orbit=orbit, bank_orbit=bank_orbit, bank_ap=bank_ap)


def tiny(seed: int = SEED_NOISE) -> Problem:
    """Plain method, tiny: 1 detector, 200 SFTs of 900 s over 30 days, rho ~ Exp(1),
    band 100.0-100.1 Hz, 8 sky x 4 a_p x 4 Omega x 4 t_asc x 90 f0."""
    sky = fibonacci_sky(8)
    return make_problem("tiny", n_per_det=200, dets=["H1"], T_sft=900.0, span=30 * DAY,
                        random_times=False, f_lo=100.0, n_f0=90, half_bin=False, sky=sky,
                        patch_size=8, a_p=np.array([1.0, 2.0, 3.0, 4.0]),
                        P_days=np.array([15.0, 20.0, 25.0, 30.0]), n_T=4, power_kind="exp",
                        seed=seed, top_k=100)


TINY_INJECTION = dict(sky=3, ap_index=1, Om_index=1, T_index=1, f0_index=45, excess=3.0)


def mid(n_sky: int = 2000, n_per_det: int = 2000, n_ap: int = 32, n_P: int = 32, n_T: int = 32,
        half_bin: bool = False, seed: int = SEED_NOISE, patch_size: int = 50, top_k: int = 1000,
        orbit_only: bool = False, sky: Optional[np.ndarray] = None, a_p: Optional[np.ndarray] = None,
        P_days: Optional[np.ndarray] = None) -> Problem:
    """Plain method, mid: 2 detectors x 2000 SFTs of 900 s over 1 yr (random
    starts), Gaussian noise with a 1-1.5 S_n ratio between detectors, 0.1 Hz
    band at 200 Hz, 2000 sky points in patches of 50, a_p 0.5-10 ls (32),
    P 15-45 d (32), 32 t_asc per period, all 90 f0 bins, top-1000 per patch.
    Smaller variants keep the same construction."""
    if sky is None:
        sky = fibonacci_sky(n_sky)
    if a_p is None:
        a_p = np.linspace(0.5, 10.0, n_ap)
    if P_days is None:
        P_days = np.linspace(15.0, 45.0, n_P)
    return make_problem("mid", n_per_det=n_per_det, dets=["H1", "L1"], T_sft=900.0, span=YEAR_SID,
                        random_times=True, f_lo=200.0, n_f0=90, half_bin=half_bin, sky=sky,
                        patch_size=patch_size, a_p=a_p, P_days=P_days,
                        n_T=n_T, power_kind="gauss", seed=seed, top_k=top_k, orbit_only=orbit_only)


def eccentric(n_sky: int = 2000, n_per_det: int = 2000, n_ap: int = 16, n_P: int = 16, n_T: int = 16,
              n_kap: int = 3, n_eta: int = 3, e_max: float = 0.1, seed: int = SEED_NOISE,
              patch_size: int = 50, top_k: int = 1000, sky: Optional[np.ndarray] = None) -> Problem:
    """Low-eccentricity search (Eq. (14)): the mid construction (2 x 2000 SFTs over 1 yr,
    200 Hz, patches of 50) with a 16^3 circular grid widened by kappa, eta in
    [-e_max, e_max] (3 x 3), so B = 16^3 * 9 = 36864 binary templates.  e up to
    0.14 passes the circular model's limit 1/(2 T_c f0 a_p Omega) (0.057 at
    a_p = 10 ls, P = 15 d) while e^2 T_c f0 a_p Omega stays below one bin."""
    if sky is None:
        sky = fibonacci_sky(n_sky)
    return make_problem("eccentric", n_per_det=n_per_det, dets=["H1", "L1"], T_sft=900.0, span=YEAR_SID,
                        random_times=True, f_lo=200.0, n_f0=90, half_bin=False, sky=sky,
                        patch_size=patch_size, a_p=np.linspace(0.5, 10.0, n_ap),
                        P_days=np.linspace(15.0, 45.0, n_P), n_T=n_T, power_kind="gauss", seed=seed,
                        top_k=top_k, kappa=np.linspace(-e_max, e_max, n_kap),
                        eta=np.linspace(-e_max, e_max, n_eta))


def metric(n_sky: int = 2000, n_per_det: int = 2000, ap_range=(3.0, 13.0), P_days=(10.0, 20.0),
           seed: int = SEED_NOISE, patch_size: int = 50, top_k: int = 1000, sky: Optional[np.ndarray] = None) -> Problem:
    """Search over a binary template bank: the mid construction (2 x 2000 SFTs over 1 yr,
    0.1 Hz at 200 Hz, patches of 50) over the BS3 ranges of the paper's simulations
    (Sec. VI.A: a_p 3-13 ls, P 10-20 d).  The grid fields hold only the range's corners
    (they size the loaded band); attach the bank with attach_bank()."""
    if sky is None:
        sky = fibonacci_sky(n_sky)
    return make_problem("metric", n_per_det=n_per_det, dets=["H1", "L1"], T_sft=900.0, span=YEAR_SID,
                        random_times=True, f_lo=200.0, n_f0=90, half_bin=False, sky=sky,
                        patch_size=patch_size, a_p=np.array(ap_range, dtype=np.float64),
                        P_days=np.array([P_days[1], P_days[0]], dtype=np.float64), n_T=1, power_kind="gauss",
                        seed=seed, top_k=top_k)


def metric_spec(pr: Problem, m: float = 6.4, ap_block: Optional[float] = None) -> dict:
    """Bank parameters for a metric() problem: spacings at the band's top frequency,
    T_obs the span of the SFTs, t_asc around the mid-time (t = 0), equal mismatch
    parameters m for a_p, Omega and t_asc; ap_block None = one a_p block per Omega
    (every a_p of an Omega shares its t_asc grid)."""
    f_top = (pr.F0 + pr.n_f0 - 1) / pr.T_sft
    T_obs = float(pr.t.max() - pr.t.min()) + pr.T_sft
    a0, a1 = float(pr.a_p.min()), float(pr.a_p.max())
    return dict(f=f_top, T_c=pr.T_sft, T_obs=T_obs, t_mid=0.0, ap_min=a0, ap_max=a1,
                P_min=2.0 * math.pi / float(pr.Omega.max()), P_max=2.0 * math.pi / float(pr.Omega.min()),
                m_a=m, m_Om=m, m_t=m, ap_block=(a1 / a0) if ap_block is None else ap_block)


def attach_bank(pr: Problem, orbit, bank_orbit, bank_ap) -> Problem:
    """The problem searching the given explicit binary bank."""
    return dataclasses.replace(pr, orbit=np.asarray(orbit, dtype=np.float64).reshape(-1, 4),
                               bank_orbit=np.asarray(bank_orbit, dtype=np.int32),
                               bank_ap=np.asarray(bank_ap, dtype=np.float64))


@dataclasses.dataclass
class TimeSeries:
    """Complex baseband data of one band for each detector, in contiguous segments.

    Sample n of a segment starting at t0 is taken at t0 + n T_sft / M; M = 2 K samples
    per SFT length, so that a T_sft / 2 offset is a whole number of samples.  The
    discrete Fourier transform of M consecutive samples puts band bin k_lo + m at
    index m (m < K).  Noise: complex white Gaussian with E|x|^2 = S_n / M, so that an
    SFT bin has mean power S_n.
    """
    T_sft: float
    k_lo: int
    K: int
    M: int
    dets: List[str]
    Sn: List[float]
    seg_start: List[np.ndarray]     # per detector: start time of each segment (s)
    seg_len: List[np.ndarray]       # per detector: whole SFTs in each segment
    x: List[List[np.ndarray]]       # per detector, per segment: samples [seg_len * M]

    def sample_times(self, d: int, g: int) -> np.ndarray:
        return self.seg_start[d][g] + np.arange(self.x[d][g].size) * (self.T_sft / self.M)


def time_series(n_per_det: int, dets: List[str], T_sft: float, span: float, k_lo: int, K: int,
                seg_sfts=(8, 40), seed: int = SEED_NOISE, sn_ratio: float = 1.25) -> TimeSeries:
    """Seeded noise data: each detector's n_per_det SFT lengths of data cut into contiguous
    segments of seg_sfts SFTs (uniform), placed at random over the span without overlap."""
    rng = np.random.default_rng(seed)
    M = 2 * K
    starts, lens, xs, Sns = [], [], [], []
    for d, _ in enumerate(dets):
        L = []
        left = n_per_det
        while left > 0:
            m = int(min(left, rng.integers(seg_sfts[0], seg_sfts[1] + 1)))
            L.append(m)
            left -= m
        L = np.array(L, dtype=np.int64)
        total = float(L.sum()) * T_sft
        gaps = rng.random(L.size + 1)
        gaps *= (span - total) / gaps.sum()
        st = -0.5 * span + np.cumsum(gaps[:-1]) + np.concatenate([[0.0], np.cumsum(L[:-1] * T_sft)])
        Sn = 1.0 if d == 0 else sn_ratio
        seg = []
        for m in L:
            n = int(m) * M
            seg.append((rng.standard_normal(n) + 1j * rng.standard_normal(n)) * math.sqrt(Sn / (2.0 * M)))
        starts.append(st)
        lens.append(L)
        xs.append(seg)
        Sns.append(Sn)
    return TimeSeries(T_sft=T_sft, k_lo=k_lo, K=K, M=M, dets=list(dets), Sn=Sns, seg_start=starts, seg_len=lens,
                      x=xs)


def inject_series(ts: TimeSeries, freq_bins, amp: float, phase: float = 0.0) -> None:
    """Adds a unit-amplitude-per-SFT-bin signal whose instantaneous frequency, in bins, is
    freq_bins(d, t) (detector index, times); amp scales its SFT-bin amplitude to amp sqrt(S_n)."""
    for d in range(len(ts.dets)):
        A = amp * math.sqrt(ts.Sn[d]) / ts.M
        for g in range(len(ts.x[d])):
            t = ts.sample_times(d, g)
            f = np.asarray(freq_bins(d, t), dtype=np.float64) - ts.k_lo
            ph = phase + 2.0 * math.pi * np.concatenate([[0.0], np.cumsum(f[:-1])]) / ts.M
            ts.x[d][g] = ts.x[d][g] + A * np.exp(1j * ph)


def _sfts(ts: TimeSeries, sliding: bool):
    """(mid-times, detector index, powers [n][K]) of the SFTs of the data: every whole SFT of
    each segment, or with sliding=True the SFTs starting T_sft/2 later (where a whole SFT
    length of data follows)."""
    tm, det, pw = [], [], []
    off = ts.M // 2 if sliding else 0
    for d in range(len(ts.dets)):
        for g, L in enumerate(ts.seg_len[d]):
            x = ts.x[d][g]
            for k in range(int(L) - (1 if sliding else 0)):
                a = k * ts.M + off
                X = np.fft.fft(x[a:a + ts.M])
                pw.append((X[:ts.K].real ** 2 + X[:ts.K].imag ** 2).astype(np.float32))
                tm.append(ts.seg_start[d][g] + (k + 0.5) * ts.T_sft + off * ts.T_sft / ts.M)
                det.append(d)
    return np.array(tm), np.array(det, dtype=np.int32), np.array(pw)


def sliding_problems(n_per_det: int = 120, n_sky: int = 6, patch_size: int = 3, n_ap: int = 3, n_P: int = 2,
                     n_T: int = 2, f_lo: float = 200.0, n_f0: int = 90, span: float = 30 * DAY,
                     T_sft: float = 900.0, seg_sfts=(6, 20), seed: int = SEED_NOISE, top_k: int = 50,
                     inject=None):
    """Stage-1 and stage-2 SFT sets from one time series (Sec. IV.C): the stage-1 problem
    holds every whole SFT of the data, the stage-2 problem those plus the SFTs shifted by
    T_sft / 2.  Both search the same sky (patches of patch_size), binary grid (a_p 0.5-10 ls,
    P 15-45 d) and f0 bins.  inject(ts, pr1) may add signals to the data before the SFTs
    are taken.  Returns (pr1, pr2, ts)."""
    dets = ["H1", "L1"]
    sky = fibonacci_sky(n_sky)
    a_p = np.linspace(0.5, 10.0, n_ap)
    Omega = 2.0 * math.pi / (np.linspace(15.0, 45.0, n_P) * DAY)
    F0 = math.floor(f_lo * T_sft)
    tt = np.linspace(-0.5 * span, 0.5 * span, 4001)
    v_max = max(float(np.max(np.linalg.norm(detector_velocity(tt, d), axis=1))) for d in dets) * (1 + 1e-9)
    k_lo, K, W = band_for(F0, F0 + n_f0 - 1, v_max, float(a_p.max()), float(Omega.max()), min_K=101)
    ts = time_series(n_per_det, dets, T_sft, span, k_lo, K, seg_sfts=seg_sfts, seed=seed)

    def problem(name, tm, det, pw):
        v = np.concatenate([detector_velocity(tm[det == d], dn) for d, dn in enumerate(dets)])
        arms = np.concatenate([detector_arms(tm[det == d], dn) for d, dn in enumerate(dets)])
        order = np.concatenate([np.nonzero(det == d)[0] for d in range(len(dets))])
        Sn = np.array([ts.Sn[d] for d in det[order]])
        return Problem(name=name, T_sft=T_sft, t=tm[order], v=v, arms=arms, Sn=Sn, det=det[order], sky=sky,
                       patch_start=_patches(sky.shape[0], patch_size), a_p=a_p, Omega=Omega,
                       T_asc=_tasc_grid(Omega, n_T), F0=float(F0), n_f0=int(n_f0), k_lo=k_lo, K=K, W=W,
                       power=pw[order], median_window=101, top_k=top_k)

    tm0, det0, _ = _sfts(ts, False)
    if inject is not None:
        inject(ts, problem("plan", tm0, det0, np.zeros((tm0.size, K), np.float32)))
    tm1, det1, pw1 = _sfts(ts, False)
    tm2, det2, pw2 = _sfts(ts, True)
    pr1 = problem("stage1", tm1, det1, pw1)
    pr2 = problem("stage2", np.concatenate([tm1, tm2]), np.concatenate([det1, det2]), np.concatenate([pw1, pw2]))
    return pr1, pr2, ts


def precision_stress(n_sky: int = 2000, n_per_det: int = 2000, n_ap: int = 32, n_P: int = 32,
                     n_T: int = 32, seed: int = SEED_NOISE) -> Problem:
    """Mid workload on the half-bin f0 grid (F = k + 1/2), detector velocities
    restricted to the xy-plane, the pole among the sky points and a_p = 0 in
    the grid, so that (pole, a_p = 0) templates sit exactly on bin ties."""
    sky = fibonacci_sky(n_sky)
    sky[0] = np.array([0.0, 0.0, 1.0])
    a_p = np.concatenate([[0.0], np.linspace(0.5, 10.0, n_ap - 1)])
    return mid(n_sky=n_sky, n_per_det=n_per_det, n_ap=n_ap, n_P=n_P, n_T=n_T, half_bin=True,
               seed=seed, orbit_only=True, sky=sky, a_p=a_p)


def batching(n_patch: int = 64, size_lo: int = 500, size_hi: int = 5000, n_per_det: int = 500,
             seed: int = SEED_NOISE, n_bin: int = 8, power_kind: str = "gauss") -> List[Problem]:
    """Batching: 64 sky patches of uneven size (500-5000 points, seeded) searched
    in four 1 Hz bands at 100/200/300/400 Hz with T_c = 900/600/450/360 s;
    2 x 500 SFTs over 30 days per band; 8 x 8 x 8 binary grid."""
    rng = np.random.default_rng(SEED_SKY)
    sizes = rng.integers(size_lo, size_hi + 1, size=n_patch)
    ps = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    sky = fibonacci_sky(int(ps[-1]))
    out = []
    for f, T in ((100.0, 900.0), (200.0, 600.0), (300.0, 450.0), (400.0, 360.0)):
        out.append(make_problem(f"batch{int(f)}", n_per_det=n_per_det, dets=["H1", "L1"], T_sft=T,
                                span=30 * DAY, random_times=True, f_lo=f, n_f0=int(round(T)),
                                half_bin=False, sky=sky, patch_size=0, a_p=np.linspace(0.5, 5.0, n_bin),
                                P_days=np.linspace(15.0, 45.0, n_bin), n_T=n_bin, power_kind=power_kind,
                                seed=seed + int(f), top_k=1000, patch_start=ps))
    return out


def patch_groups(patch_start, n_groups: int) -> List[List[int]]:
    """The patches of a problem dealt into n_groups groups of about equal sky count:
    largest patch first, in a snake order over the groups; each group lists its
    patches in their original order."""
    ps = np.asarray(patch_start, dtype=np.int64)
    sizes = np.diff(ps)
    order = sorted(range(sizes.size), key=lambda p: (-int(sizes[p]), p))
    groups: List[List[int]] = [[] for _ in range(n_groups)]
    for k, p in enumerate(order):
        r, c = divmod(k, n_groups)
        groups[c if r % 2 == 0 else n_groups - 1 - c].append(p)
    return [sorted(g) for g in groups if g]


def select_patches(pr: Problem, patches: Sequence[int]) -> Problem:
    """The problem restricted to the listed patches: their sky points in the listed
    order, one patch each (band, SFTs, powers and binary templates unchanged)."""
    ps = np.asarray(pr.patch_start, dtype=np.int64)
    sky = np.concatenate([pr.sky[ps[p]:ps[p + 1]] for p in patches], axis=0)
    sizes = [int(ps[p + 1] - ps[p]) for p in patches]
    new_ps = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return dataclasses.replace(pr, sky=np.ascontiguousarray(sky), patch_start=new_ps)


def full(n_sky: int = 100048, n_per_det: int = 4000, n_f0: int = 9000, seed: int = SEED_NOISE,
         patch_size: int = 169, power_kind: str = "gauss") -> Problem:
    """Full scale: 2 x 4000 SFTs over 1 yr, 10 Hz band at 300 Hz, ~1e5 sky points
    in patches of 169, a_p 0.5-15 ls, P 10-60 d (8 x 8 x 8), top-10000."""
    return make_problem("full", n_per_det=n_per_det, dets=["H1", "L1"], T_sft=900.0, span=YEAR_SID,
                        random_times=True, f_lo=300.0, n_f0=n_f0, half_bin=False,
                        sky=fibonacci_sky(n_sky), patch_size=patch_size,
                        a_p=np.linspace(0.5, 15.0, 8), P_days=np.linspace(10.0, 60.0, 8), n_T=8,
                        power_kind=power_kind, seed=seed, top_k=10000)
