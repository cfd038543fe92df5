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


def _dense_shard(args):
    """Spawned process: the oracle's dense counts of the s-th listed sky point for the binary
    templates of one Omega of a circular grid (contiguous b = iOm * n_T * n_ap + b')."""
    import oracle as _orc
    kw, s, iOm = args
    sub = dict(kw)
    sub["sky"] = kw["sky"][s:s + 1]
    sub["w"] = kw["w"][s:s + 1]
    sub["Omega"] = kw["Omega"][iOm:iOm + 1]
    sub["T_asc"] = kw["T_asc"][iOm:iOm + 1]
    return s, iOm, _orc.OracleProblem(**sub).count_dense()


def oracle_dense_parallel(pr, bits, w, sky_points, procs=0):
    """The oracle's dense counts ([len(sky_points), B, n_f0] per field, as count_dense) of
    a circular-grid problem, computed in spawned processes, one (sky point, Omega) shard each.
    The arithmetic is the oracle's count_one, unchanged; only the work is split."""
    import multiprocessing as mp
    import os
    assert pr.kappa is None and pr.eta is None and pr.orbit is None
    sel = np.asarray(sky_points, dtype=np.int64)
    kw = dict(bits=bits, w=np.ascontiguousarray(w[sel]), v=pr.v, t=pr.t, F0=pr.F0, n_f0=pr.n_f0,
              sky=np.ascontiguousarray(pr.sky[sel]), a_p=pr.a_p, Omega=pr.Omega, T_asc=pr.T_asc, k_lo=pr.k_lo,
              K=pr.K, rho_th=pr.rho_th)
    n_Om = pr.Omega.size
    per_Om = pr.B // n_Om
    shape = (len(sky_points), pr.B, pr.n_f0)
    out = dict(n_unw=np.empty(shape, np.int32), n_w=np.empty(shape), n_tie=np.empty(shape, np.int32),
               unw_lo=np.empty(shape, np.int32), unw_hi=np.empty(shape, np.int32),
               w_lo=np.empty(shape), w_hi=np.empty(shape))
    tasks = [(kw, s, k) for s in range(sel.size) for k in range(n_Om)]
    with mp.get_context("spawn").Pool(procs or os.cpu_count() or 1) as pool:
        for s, iOm, d in pool.imap_unordered(_dense_shard, tasks):
            for f, a in d.items():
                out[f][s, iOm * per_Om:(iOm + 1) * per_Om] = a[0]
    return out
