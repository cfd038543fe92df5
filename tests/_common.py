"""Shared test helpers: small seeded problems and oracle views of them."""
import math

import numpy as np

import oracle
from paper_1904_04873_gb300 import synth


def small_mid(n_sky=6, n_per_det=60, n_ap=4, n_P=3, n_T=3, seed=synth.SEED_NOISE, patch_size=3,
              half_bin=False, top_k=50):
    return synth.mid(n_sky=n_sky, n_per_det=n_per_det, n_ap=n_ap, n_P=n_P, n_T=n_T, seed=seed,
                     patch_size=patch_size, half_bin=half_bin, top_k=top_k)


def oracle_inputs(pr, dtype="f64"):
    """Oracle peakgram (rho, bits) and quantised weights for a synth problem."""
    rho, bits = oracle.peakgram(pr.power, pr.median_window, pr.rho_th, W=pr.W)
    w = oracle.quantize(oracle.weights(pr.sky, pr.arms, pr.Sn, norm=True), dtype)
    return rho, bits, w


def oracle_problem(pr, bits, w, rho=None):
    return oracle.OracleProblem(bits=bits, w=w, v=pr.v, t=pr.t, F0=pr.F0, n_f0=pr.n_f0, sky=pr.sky,
                                a_p=pr.a_p, Omega=pr.Omega, T_asc=pr.T_asc, k_lo=pr.k_lo, K=pr.K,
                                rho=rho, rho_th=pr.rho_th, kappa=pr.kappa, eta=pr.eta, orbit=pr.orbit,
                                bank_orbit=pr.bank_orbit, bank_ap=pr.bank_ap)


def pack_bits(on, W):
    """Pack a bool [N][K] array into uint32 rows (bit k of word k//32)."""
    N, K = on.shape
    out = np.zeros((N, W), np.uint32)
    for k in range(K):
        out[:, k >> 5] |= (on[:, k].astype(np.uint32) << np.uint32(k & 31))
    return out


def orbit_of(pr, b):
    """(a_p, Omega, t_asc, kappa, eta) of binary index b:
    b = (((iOm * n_T + iT) * n_kap + ik) * n_eta + ie) * n_ap + iap, or the bank's entry b."""
    if pr.orbit is not None:
        Om, Ta, kap, eta = pr.orbit[pr.bank_orbit[b]]
        return pr.bank_ap[b], Om, Ta, float(kap), float(eta)
    nk = 1 if pr.kappa is None else pr.kappa.size
    ne = 1 if pr.eta is None else pr.eta.size
    iap = b % pr.a_p.size
    r = b // pr.a_p.size
    ie = r % ne
    r //= ne
    ik = r % nk
    r //= nk
    iT = r % pr.T_asc.shape[1]
    iOm = r // pr.T_asc.shape[1]
    kap = 0.0 if pr.kappa is None else float(pr.kappa[ik])
    eta = 0.0 if pr.eta is None else float(pr.eta[ie])
    return pr.a_p[iap], pr.Omega[iOm], pr.T_asc[iOm, iT], kap, eta


def template_of(pr, b):
    """(a_p, Omega, t_asc) of binary index b of a circular-orbit problem."""
    assert pr.kappa is None and pr.eta is None and pr.orbit is None
    return orbit_of(pr, b)[:3]


def track_bins(pr, s, b, j):
    """Oracle bins (and tie flags) of one template in every SFT."""
    ap, Om, Ta, kap, eta = orbit_of(pr, b)
    F = pr.F0 + j
    ks, ties = [], []
    for i in range(pr.N):
        k, t = oracle.track_bin_ell1(F, pr.v[i], pr.sky[s], ap, Om, Ta, kap, eta, pr.t[i])
        ks.append(k)
        ties.append(t)
    return np.array(ks), np.array(ties)


def inject_on_track(pr, rho, s, b, j, excess=3.0):
    """Add `excess` to rho at the template's track bin in every SFT (config 1 injection)."""
    ks, _ = track_bins(pr, s, b, j)
    out = rho.copy()
    out[np.arange(pr.N), ks - pr.k_lo] += np.float32(excess)
    return out


P_TH = math.exp(-1.6)
