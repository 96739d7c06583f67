"""Amplitude spaces, partitions, the mixed-triples slice and the initial guess.

Spin-adapted storage (Supporting Information, Sec. S1): for a singlet only
t1[i,a] = t_{i alpha}^{a alpha}, t2[i,j,a,b] = t_{i alpha j beta}^{a alpha b beta}
and t3[i,j,k,a,b,c] = t_{i alpha j beta k beta}^{a alpha b beta c beta} are
unique.  A full spin flip leaves an amplitude unchanged; same-spin amplitudes
follow from Eqs. S1-S2:
    t_{i a j a}^{a a b a}          = t2[i,j,a,b] - t2[j,i,a,b]
    t_{i a j a k a}^{a a b a c a}  = t3[k,i,j,c,a,b] - t3[k,i,j,b,a,c] + t3[k,i,j,a,b,c]
Cluster operators, with a^+ / a spin-orbital creation / annihilation:
    T1 = sum t1[i,a] (a+_{a up} a_{i up} + a+_{a dn} a_{i dn})
    T2 = sum_{ijab} t2[i,j,a,b] a+_{a up} a+_{b dn} a_{j dn} a_{i up} + same-spin parts
    T3 = 1/4 sum t3[i,j,k,a,b,c] a+_{a up} a+_{b dn} a+_{c dn} a_{k dn} a_{j dn} a_{i up}
         + spin flip + same-spin parts.
t2 obeys t2[i,j,a,b] = t2[j,i,b,a]; t3 is antisymmetric in (j,k) and in (b,c).

Primary orbitals (Sec. II.B): the hole h (occupied index) and the particle p
(virtual index) of S.  An amplitude is primary (P) when every spatial index is
primary, non-primary (N) when none is, and mixed (M) otherwise (Eq. pnm split).

Mixed-triples slice T3' (Sec. II.B.1): the alpha-beta-beta triples whose
spin-orbital index set holds at least three of {h up, h dn, p up, p dn}.  A
same-spin triple holds at most one primary hole and one primary particle, so
T3' has no alpha-alpha-alpha part; the alpha-alpha-beta part is the spin flip.
"""
from __future__ import annotations

import numpy as np

SQRT_HALF = 1.0 / np.sqrt(2.0)


# ---------------------------------------------------------------- partitions
def t1_class_masks(o, v, hole, particle):
    """Boolean masks (P, M, N) over t1[i,a]."""
    ip = np.zeros(o, bool); ip[hole] = True
    ap = np.zeros(v, bool); ap[particle] = True
    cnt = ip[:, None].astype(int) + ap[None, :].astype(int)
    return cnt == 2, cnt == 1, cnt == 0


def t2_class_masks(o, v, hole, particle):
    """Boolean masks (P, M, N) over t2[i,j,a,b] by the count of primary spatial indices."""
    ip = np.zeros(o, int); ip[hole] = 1
    ap = np.zeros(v, int); ap[particle] = 1
    cnt = (ip[:, None, None, None] + ip[None, :, None, None]
           + ap[None, None, :, None] + ap[None, None, None, :])
    return cnt == 4, (cnt > 0) & (cnt < 4), cnt == 0


# ------------------------------------------------------------- T3' slice
def t3p_index(o, v, hole, particle):
    """Index list [N, 6] of the unique T3' amplitudes (i, j, k, a, b, c).

    Only j < k and b < c are listed; the primary spin-orbital count
    [i=h] + [h in {j,k}] + [a=p] + [p in {b,c}] is at least 3.  Rows are in
    lexicographic order of (i, j, k, a, b, c).
    """
    if hole is None:
        return np.zeros((0, 6), dtype=np.int64)
    h, p = hole, particle
    rows = []
    for i in range(o):
        for j in range(o):
            for k in range(j + 1, o):
                occ = int(i == h) + int(h in (j, k))
                if occ == 0:
                    continue
                for a in range(v):
                    need = 3 - occ - int(a == p)
                    if need > 1:
                        continue
                    if need <= 0:
                        for b in range(v):
                            for c in range(b + 1, v):
                                rows.append((i, j, k, a, b, c))
                    else:  # exactly one more: p must be in {b, c}
                        for b in range(v):
                            for c in range(b + 1, v):
                                if b == p or c == p:
                                    rows.append((i, j, k, a, b, c))
    return np.array(rows, dtype=np.int64).reshape(-1, 6)


def t3_dense(idx, vals, o, v):
    """Dense alpha-beta-beta array [o,o,o,v,v,v] (antisymmetric in jk and bc) from the slice."""
    t = np.zeros((o, o, o, v, v, v))
    if len(idx) == 0:
        return t
    i, j, k, a, b, c = idx.T
    t[i, j, k, a, b, c] = vals
    t[i, k, j, a, b, c] = -vals
    t[i, j, k, a, c, b] = -vals
    t[i, k, j, a, c, b] = vals
    return t


def t3_gather(t, idx):
    """Values of a dense alpha-beta-beta array at the slice positions."""
    if len(idx) == 0:
        return np.zeros(0)
    i, j, k, a, b, c = idx.T
    return t[i, j, k, a, b, c].copy()


# ------------------------------------------------------------ initial guess
def initial_guess(o, v, hole=None, particle=None, beta=1.0, n_t3=0, xsign=1.0):
    """Zeroth-order amplitudes (Eq. TP-guess): T^P = beta S + gamma S^2, gamma = -beta^2/2.

    S = (1/sqrt2)(p+_up h_up + p+_dn h_dn) gives t1[h,p] = beta/sqrt2 and, since
    S^2 = a+_{p up} a+_{p dn} a_{h dn} a_{h up}, t2[h,h,p,p] = gamma.  All other
    amplitudes (T^M, T^N, T3') start at zero.  The ground state starts at zero.
    xsign = -1 is the same guess written for S -> -S (the second ansatz).
    """
    t1 = np.zeros((o, v)); t2 = np.zeros((o, o, v, v)); t3 = np.zeros(n_t3)
    if hole is not None:
        t1[hole, particle] = xsign * beta * SQRT_HALF
        t2[hole, hole, particle, particle] = -0.5 * beta * beta
    return t1, t2, t3


def beta_from_alpha(alpha: float):
    """The two ansatz choices of Sec. II.D for an Aufbau weight alpha.

    With gamma = -beta^2/2 the reference becomes ((1-beta)/beta) phi0 + S phi0,
    so (1-beta)/beta = alpha gives beta = 1/(1+alpha); flipping the sign of
    the hole orbital flips alpha, giving the second choice 1/(1-alpha).
    """
    return 1.0 / (1.0 + alpha), 1.0 / (1.0 - alpha)


# ----------------------------------------------------------- spin relations
def t2_same_spin(t2):
    """t_{i up j up}^{a up b up} = t2[i,j,a,b] - t2[j,i,a,b] (Eq. S1)."""
    return t2 - t2.transpose(1, 0, 2, 3)


def t3_same_spin(t3):
    """t_{i up j up k up}^{a up b up c up} from alpha-beta-beta amplitudes (Eq. S2).

    Value at (i,j,k,a,b,c) = t3[k,i,j,c,a,b] - t3[k,i,j,b,a,c] + t3[k,i,j,a,b,c].
    """
    # r[i,j,k,a,b,c] = t3[k,i,j,...] with the named virtual orders
    s = t3.transpose(1, 2, 0, 3, 4, 5)          # s[i,j,k,x,y,z] = t3[k,i,j,x,y,z]
    return (s.transpose(0, 1, 2, 4, 5, 3)       # t3[k,i,j,c,a,b]
            - s.transpose(0, 1, 2, 4, 3, 5)     # t3[k,i,j,b,a,c]
            + s)                                # t3[k,i,j,a,b,c]
