"""Post-processing of the toplists (Sec. V.E) -- TEST INFRASTRUCTURE (oracle).

Plain numpy in double precision, following the paper's steps:
  * candidate parameters: f (Hz), x, y (the sky direction in ecliptic Cartesian
    coordinates, projected onto the ecliptic plane), a_p, Omega, t_asc;
  * the parameter-space distance of Eq. (44), each resolution taken as the mean of
    its values at the two candidates: delta f = 1/T_c, delta theta = c / (v T_c f P_F)
    (Sec. V.B) for x and y, and delta a_p, delta Omega, delta t_asc of Eq. (30)-(32);
  * coincidences between two lists (option A): pairs closer than a threshold, each
    replaced by its significance-weighted centroid carrying the summed significance;
  * clustering: the connected components of the graph whose edges join candidates
    closer than the clustering threshold (a candidate joins every cluster it is close
    to, and clusters that share a candidate are one cluster);
  * option B: members farther than a cut distance from the cluster's most significant
    member (ties: the first in list order) are removed;
  * centroids: significance-weighted means of the remaining members; the cluster's
    significance is the sum over them; the band keeps its most significant cluster.
Readings (where the paper is silent): distances are strict for the thresholds
(d < d_cluster, d < d_coinc) and inclusive for the cut (kept if d <= d_cut); weights
are max(significance, 0), and a cluster whose weights sum to 0 gets the plain mean;
t_asc differences are plain differences.

Every floating-point expression is written in the order the CUDA path uses, so that
the threshold decisions (which are integer outcomes) are taken on identical values.
"""
from __future__ import annotations

import math
from collections import deque

import numpy as np

from .bank import resolution as binary_resolution

# parameter columns
F, X, Y, AP, OM, TA = range(6)


def ecliptic_xy(n, obliquity):
    """Equatorial unit vector(s) -> (x, y) in the ecliptic plane (rotation about x)."""
    n = np.atleast_2d(np.asarray(n, dtype=np.float64))
    ce, se = math.cos(obliquity), math.sin(obliquity)
    return n[:, 0].copy(), ce * n[:, 1] + se * n[:, 2]


def resolutions(params, pp):
    """[n][6] resolutions at each candidate: (delta f, delta theta, delta theta, delta a_p,
    delta Omega, delta t_asc)."""
    p = np.asarray(params, dtype=np.float64)
    out = np.empty_like(p)
    for i in range(p.shape[0]):
        f = p[i, F]
        d_th = 1.0 / (pp["v_over_c"] * pp["T_c"] * f * pp["P_F"])
        d_ap, d_Om, d_t = binary_resolution(f, pp["T_c"], pp["T_obs"], p[i, AP], p[i, OM], pp["m_a"], pp["m_Om"],
                                            pp["m_t"])
        out[i] = (1.0 / pp["T_c"], d_th, d_th, d_ap, d_Om, d_t)
    return out


def distance2(pi, ri, pj, rj):
    """Squared Eq. (44) distance between candidates with parameters p and resolutions r
    (the mean of the two resolutions for each parameter)."""
    d2 = 0.0
    for k in range(6):
        r = 0.5 * (ri[k] + rj[k])
        q = (pi[k] - pj[k]) / r
        d2 = d2 + q * q
    return d2


def _d2_row(p, r, i):
    """distance2 of candidate i to every candidate, vectorised over j, same operation order."""
    d2 = np.zeros(p.shape[0])
    for k in range(6):
        rk = 0.5 * (r[i, k] + r[:, k])
        q = (p[i, k] - p[:, k]) / rk
        d2 = d2 + q * q
    return d2


def components(params, valid, pp, d_cluster):
    """label[i] = smallest index of i's connected component (edges: d < d_cluster); -1 if invalid."""
    p = np.asarray(params, dtype=np.float64)
    r = resolutions(p, pp)
    n = p.shape[0]
    D2 = d_cluster * d_cluster
    adj = []
    for i in range(n):
        if not valid[i]:
            adj.append(np.zeros(0, dtype=np.int64))
            continue
        d2 = _d2_row(p, r, i)
        nb = np.nonzero((d2 < D2) & valid)[0]
        adj.append(nb[nb != i])
    label = np.full(n, -1, dtype=np.int64)
    for i in range(n):
        if not valid[i] or label[i] >= 0:
            continue
        # breadth-first search from the smallest unlabelled index: it is the component's minimum
        label[i] = i
        q = deque([i])
        while q:
            u = q.popleft()
            for v in adj[u]:
                if label[v] < 0:
                    label[v] = i
                    q.append(v)
    return label, r


def cluster(params, sig, valid, pp, d_cluster, d_cut):
    """Clusters of one band: (label, keep, centroid [n][6] at root rows, csig [n] at root rows, best).

    label as in components(); keep[i] = 1 when i survives the option-B cut (d_cut <= 0:
    no cut); centroid / csig are filled at the rows of the roots (label == index), NaN / 0
    elsewhere; best = root of the cluster with the largest csig (ties: smallest root), -1 if none.
    """
    p = np.asarray(params, dtype=np.float64)
    s = np.asarray(sig, dtype=np.float64)
    valid = np.asarray(valid, dtype=bool)
    label, r = components(p, valid, pp, d_cluster)
    n = p.shape[0]
    keep = np.zeros(n, dtype=np.int32)
    centroid = np.full((n, 6), np.nan)
    csig = np.zeros(n)
    best, best_s = -1, -math.inf
    for root in np.unique(label[label >= 0]):
        mem = np.nonzero(label == root)[0]
        # most significant member, first in list order on ties
        top = mem[0]
        for m in mem:
            if s[m] > s[top]:
                top = m
        if d_cut > 0.0:
            C2 = d_cut * d_cut
            kept = [m for m in mem if distance2(p[top], r[top], p[m], r[m]) <= C2]
        else:
            kept = list(mem)
        keep[kept] = 1
        w = np.maximum(s[kept], 0.0)
        sw = 0.0
        for x in w:
            sw = sw + x
        acc = np.zeros(6)
        if sw > 0.0:
            for m, x in zip(kept, w):
                acc = acc + x * p[m]
            centroid[root] = acc / sw
        else:
            for m in kept:
                acc = acc + p[m]
            centroid[root] = acc / float(len(kept))
        tot = 0.0
        for m in kept:
            tot = tot + s[m]
        csig[root] = tot
        if tot > best_s:
            best, best_s = int(root), tot
    return label, keep, centroid, csig, best


def coincidences(pa, sa, pb, sb, pp, d_coinc):
    """Option A: every pair (i in A, j in B) with d < d_coinc, as (i, j, centroid [6], summed
    significance), sorted by (i, j); the centroid weights are max(significance, 0)."""
    pa = np.asarray(pa, dtype=np.float64)
    pb = np.asarray(pb, dtype=np.float64)
    ra, rb = resolutions(pa, pp), resolutions(pb, pp)
    D2 = d_coinc * d_coinc
    out = []
    for i in range(pa.shape[0]):
        for j in range(pb.shape[0]):
            if distance2(pa[i], ra[i], pb[j], rb[j]) < D2:
                wa, wb = max(sa[i], 0.0), max(sb[j], 0.0)
                sw = wa + wb
                c = (wa * pa[i] + wb * pb[j]) / sw if sw > 0.0 else 0.5 * (pa[i] + pb[j])
                out.append((i, j, c, sa[i] + sb[j]))
    return out


def candidate_params(ids, F0, n_f0, B, T_c, sky, obliquity, binary_of):
    """Parameters [n][6] of templates id = ((s * B + b) * n_f0 + j): f = (F0 + j) / T_c,
    (x, y) of sky[s], and (a_p, Omega, t_asc) = binary_of(b)."""
    out = np.empty((len(ids), 6))
    ce, se = math.cos(obliquity), math.sin(obliquity)
    for e, tid in enumerate(ids):
        s, rem = divmod(int(tid), B * n_f0)
        b, j = divmod(rem, n_f0)
        n = sky[s]
        a_p, Om, Ta = binary_of(b)
        out[e] = ((F0 + float(j)) / T_c, n[0], ce * n[1] + se * n[2], a_p, Om, Ta)
    return out
