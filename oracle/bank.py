"""Binary template bank of Sec. V.B -- TEST INFRASTRUCTURE (oracle).

Plain Python floats (IEEE double), written from the resolutions of
Eq. (30)-(32) and the t_asc range of Eq. (35):

    delta a_p     = sqrt(6 m_a) / (pi T_c f Omega)
    delta Omega   = sqrt(72 m_Omega) / (pi T_c f a_p Omega T_obs)
    delta t_asc   = sqrt(6 m_t) / (pi T_c f a_p Omega^2)

The paper gives the spacings, not the lattice.  Reading taken here: every
spacing is evaluated where it is smallest over the cell it spans, so the bank
is nowhere coarser than the metric asks for --
  * Omega runs from 2 pi / P_max upwards; each step is delta Omega at the
    largest a_p of the range, evaluated at the current Omega; it stops once past
    2 pi / P_min;
  * at each Omega, a_p runs from a_min upwards in steps of delta a_p(Omega) while
    it does not exceed a_max;
  * the a_p values are cut, in order, into blocks whose largest value is at most
    ap_block times their smallest; each block gets one t_asc grid, spaced by
    delta t_asc at the block's largest a_p, from t_mid - P/2 while below
    t_mid + P/2 (P = 2 pi / Omega).
Output: orbit rows (Omega, t_asc, 0, 0) and, per template, its row and a_p, rows
in the order built, a block's templates in increasing a_p.
"""
from __future__ import annotations

import math

import numpy as np


def resolution(f, T_c, T_obs, a_p, Om, m_a, m_Om, m_t):
    """Eq. (30)-(32): (delta a_p, delta Omega, delta t_asc) at (f, a_p, Omega)."""
    d_ap = math.sqrt(6.0 * m_a) / (math.pi * T_c * f * Om)
    d_Om = math.sqrt(72.0 * m_Om) / (math.pi * T_c * f * a_p * Om * T_obs)
    d_t = math.sqrt(6.0 * m_t) / (math.pi * T_c * f * a_p * Om * Om)
    return d_ap, d_Om, d_t


def template_bank(f, T_c, T_obs, t_mid, ap_min, ap_max, P_min, P_max, m_a, m_Om, m_t, ap_block):
    """The bank described in the module docstring: (orbit [R][4], bank_orbit [B], bank_ap [B])."""
    Om_lo = 2.0 * math.pi / P_max
    Om_hi = 2.0 * math.pi / P_min
    orbit, rows_of, aps_of = [], [], []
    Om = Om_lo
    while True:
        d_ap, d_Om, _ = resolution(f, T_c, T_obs, ap_max, Om, m_a, m_Om, m_t)
        aps = []
        k = 0
        while True:
            a = ap_min + float(k) * d_ap
            if a > ap_max:
                break
            aps.append(a)
            k += 1
        P = 2.0 * math.pi / Om
        i0 = 0
        while i0 < len(aps):
            i1 = i0 + 1
            while i1 < len(aps) and aps[i1] <= ap_block * aps[i0]:
                i1 += 1
            _, _, d_t = resolution(f, T_c, T_obs, aps[i1 - 1], Om, m_a, m_Om, m_t)
            k = 0
            while True:
                t = (t_mid - 0.5 * P) + float(k) * d_t
                if not (t < t_mid + 0.5 * P):
                    break
                r = len(orbit)
                orbit.append((Om, t, 0.0, 0.0))
                for i in range(i0, i1):
                    rows_of.append(r)
                    aps_of.append(aps[i])
                k += 1
            i0 = i1
        Om = Om + d_Om
        if Om > Om_hi:
            break
    return (np.array(orbit, dtype=np.float64).reshape(-1, 4), np.array(rows_of, dtype=np.int32),
            np.array(aps_of, dtype=np.float64))
