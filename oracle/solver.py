"""Diagonal-Jacobian (Jacobi) amplitude iteration with DIIS (test infrastructure).

The paper drives ASCC with the diagonal approximate Jacobian update plus DIIS
used by ground-state CCSD codes (Sec. III.B) and stops when the largest
residual and the energy change fall below thresholds (Sec. III.A).  The
paper does not spell out the DIIS details; the rules below are the ones this
project fixes, and the CUDA solver follows the same rules:

* denominators from orbital energies:
    D1[i,a] = e_i - e_a,  D2[i,j,a,b] = e_i + e_j - e_a - e_b,
    D3[i,j,k,a,b,c] = e_i + e_j + e_k - e_a - e_b - e_c,
  with the bare e for the ground state; for a one-CSF state both primary
  orbitals take the mean (e_h + e_p)/2, since in the excited reference S phi0
  the hole and the particle are each half occupied (this zeroth-order
  diagonal matches the measured diagonal of the Jacobian);
* Jacobi step t' = t + R / D, except, for a one-CSF state, the pairs
  (t1[i,a], t2[i,h,a,p]) (with t2[h,i,p,a] = t2[i,h,a,p]).  Through the
  zeroth-order T^P these pairs are coupled at O(1): R1[i,a] depends on
  t2[i,h,a,p] through F_hp and, when i = h or a = p, R2[i,h,a,p] depends on
  t1[i,a] through F_ph, where F is the Fock matrix of exp(-T1) Hbar exp(T1).
  Their step solves the 2 x 2 model Jacobian
      J = [[-D1[i,a], c F_hp], [q, -D2[i,h,a,p]]],   (dt1, dt2) = -J^-1 (R1[i,a], R2[i,h,a,p]),
  c = 2, q = 0 for i != h and a != p; c = 1, q = F_ph when i = h or a = p
  (not both); for the primary pair (h, p) J = [[0, F_hp], [2 F_hp, 0]] (its
  mean-energy diagonal vanishes).  A near-singular J (|det| < 1e-12 max|J|^2)
  falls back to the diagonal step (bare denominators for the primary pair);
* DIIS over the vector (t1, t2, t3'): the error is e = t' - t, the history
  keeps the last `diis_dim` (default 16) pairs (t', e); once it holds `diis_start` pairs
  the new amplitudes are sum_k c_k t'_k with c solving the bordered system
  [[G, 1], [1, 0]] [c; l] = [0; 1], G_kl = e_k . e_l scaled by 1/max diag G
  plus a 1e-12 ridge, solved by Gaussian elimination with partial pivoting;
  a non-finite or degenerate solve empties the history but the newest pair;
* converged when max|R| <= r_tol and |E - E_previous| <= e_tol, checked on
  the residual of the current amplitudes before any update.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class SolveResult:
    energy: float
    iterations: int
    max_resid: float
    converged: bool
    t1: np.ndarray
    t2: np.ndarray
    t3: np.ndarray
    history: list = field(default_factory=list)


def bordered_solve(G: np.ndarray):
    """DIIS coefficients from the Gram matrix G (see module docstring)."""
    m = G.shape[0]
    scale = np.max(np.abs(np.diag(G)))
    if not np.isfinite(scale) or scale <= 0.0:
        return None
    A = np.zeros((m + 1, m + 1))
    A[:m, :m] = G / scale + 1e-12 * np.eye(m)
    A[:m, m] = 1.0
    A[m, :m] = 1.0
    b = np.zeros(m + 1); b[m] = 1.0
    # Gaussian elimination with partial pivoting
    n = m + 1
    for c in range(n):
        piv = c + int(np.argmax(np.abs(A[c:, c])))
        if abs(A[piv, c]) < 1e-300:
            return None
        if piv != c:
            A[[c, piv]] = A[[piv, c]]; b[[c, piv]] = b[[piv, c]]
        for r in range(c + 1, n):
            f = A[r, c] / A[c, c]
            A[r, c:] -= f * A[c, c:]
            b[r] -= f * b[c]
    x = np.zeros(n)
    for r in range(n - 1, -1, -1):
        x[r] = (b[r] - A[r, r + 1:] @ x[r + 1:]) / A[r, r]
    if not np.all(np.isfinite(x)):
        return None
    return x[:m]


def _raw_denominators(eps, o, t3_idx):
    eo, ev = eps[:o], eps[o:]
    D1 = eo[:, None] - ev[None, :]
    D2 = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    if t3_idx is None or len(t3_idx) == 0:
        D3 = np.zeros(0)
    else:
        i, j, k, a, b, c = t3_idx.T
        D3 = eo[i] + eo[j] + eo[k] - ev[a] - ev[b] - ev[c]
    return D1, D2, D3


def denominators(eps, o, t3_idx=None, hole=None, particle=None):
    """Diagonal denominators; for a one-CSF state the primary amplitudes t1[h,p]
    and t2[h,h,p,p] (zero with the mean energies) keep the bare values, which
    only serve when their pair step falls back to the diagonal."""
    if hole is None:
        return _raw_denominators(eps, o, t3_idx)
    e = np.array(eps, dtype=float)
    m = 0.5 * (e[hole] + e[o + particle])
    e[hole] = m
    e[o + particle] = m
    D1, D2, D3 = _raw_denominators(e, o, t3_idx)
    B1, B2, _ = _raw_denominators(eps, o, None)
    h, p = hole, particle
    D1[h, p] = B1[h, p]
    D2[h, h, p, p] = B2[h, h, p, p]
    return D1, D2, D3


def jacobi_step(R1, R2, R3, D1, D2, D3, hole=None, particle=None, fock=None):
    """Update (dt1, dt2, dt3) of one iteration (see the module docstring)."""
    d1 = R1 / D1
    d2 = R2 / D2
    d3 = R3 / D3 if R3.size else np.zeros(0)
    if hole is None:
        return d1, d2, d3
    o, v = R1.shape
    h, p = hole, particle
    fhp, fph = fock
    for i in range(o):
        for a in range(v):
            if i == h and a == p:
                # both mean-energy diagonals vanish for the primary pair
                J = np.array([[0.0, fhp], [2.0 * fhp, 0.0]])
            else:
                c, q = (1.0, fph) if (i == h or a == p) else (2.0, 0.0)
                J = np.array([[-D1[i, a], c * fhp], [q, -D2[i, h, a, p]]])
            det = J[0, 0] * J[1, 1] - J[0, 1] * J[1, 0]
            if abs(det) <= 1e-12 * np.max(np.abs(J)) ** 2:
                continue
            r1, r2 = R1[i, a], R2[i, h, a, p]
            x1 = (J[1, 1] * r1 - J[0, 1] * r2) / det
            x2 = (-J[1, 0] * r1 + J[0, 0] * r2) / det
            d1[i, a] = -x1
            d2[i, h, a, p] = -x2
            d2[h, i, p, a] = -x2
    return d1, d2, d3


def solve(resid_fn, eps, o, t1, t2, t3, t3_idx=None, r_tol=1e-8, e_tol=1e-10,
          max_iter=200, diis_dim=16, diis_start=3, verbose=False, hole=None, particle=None,
          fock_fn=None):
    """Iterate resid_fn(t1, t2, t3) -> (E, R1, R2, R3) to convergence.

    hole/particle: the primary orbitals of a one-CSF state (None for the
    ground state), which select the update described above; fock_fn(t1)
    returns (F_hp, F_ph) of exp(-T1) Hbar exp(T1) for the pair step.
    """
    D1, D2, D3 = denominators(eps, o, t3_idx, hole, particle)
    shapes = [t1.shape, t2.shape, t3.shape]
    sizes = [t1.size, t2.size, t3.size]

    def pack(a, b, c):
        return np.concatenate([a.ravel(), b.ravel(), c.ravel()])

    def unpack(x):
        p = np.cumsum([0] + sizes)
        return [x[p[k]:p[k + 1]].reshape(shapes[k]) for k in range(3)]

    hist_t, hist_e = [], []
    e_prev = None
    log = []
    for it in range(max_iter + 1):
        En, R1, R2, R3 = resid_fn(t1, t2, t3)
        rmax = max(np.max(np.abs(R1)) if R1.size else 0.0, np.max(np.abs(R2)),
                   np.max(np.abs(R3)) if R3 is not None and R3.size else 0.0)
        log.append((it, En, rmax))
        if verbose:
            print(f"it {it:3d}  E {En:.12f}  max|R| {rmax:.3e}")
        if not np.isfinite(En) or not np.isfinite(rmax):
            return SolveResult(En, it, rmax, False, t1, t2, t3, log)
        if e_prev is not None and rmax <= r_tol and abs(En - e_prev) <= e_tol:
            return SolveResult(En, it, rmax, True, t1, t2, t3, log)
        if it == max_iter:
            break
        e_prev = En
        R3v = R3 if R3 is not None else np.zeros(0)
        fock = fock_fn(t1) if (hole is not None and fock_fn is not None) else None
        d1, d2, d3 = jacobi_step(R1, R2, R3v, D1, D2, D3, hole if fock else None, particle, fock)
        tn = pack(t1 + d1, t2 + d2, t3 + (d3 if R3v.size else 0.0))
        err = tn - pack(t1, t2, t3)
        hist_t.append(tn); hist_e.append(err)
        if len(hist_t) > diis_dim:
            hist_t.pop(0); hist_e.pop(0)
        if len(hist_t) >= diis_start:
            Emat = np.array(hist_e)
            c = bordered_solve(Emat @ Emat.T)
            if c is None:
                hist_t = hist_t[-1:]; hist_e = hist_e[-1:]
            else:
                tn = c @ np.array(hist_t)
        t1, t2, t3 = unpack(tn)
    return SolveResult(En, max_iter, rmax, False, t1, t2, t3, log)
