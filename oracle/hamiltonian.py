"""Hamiltonian construction for the oracle (test infrastructure).

Conventions
  * spatial orbitals 0..o-1 occupied, o..o+v-1 virtual;
  * (pq|rs) = sum_P B[P,p,q] B[P,r,s] in chemists' notation with p and r the
    creation indices:  H = sum h_pq E_pq + 1/2 sum (pq|rs)(E_pq E_rs - d_qr E_ps);
  * the synthetic reference is canonical Hartree-Fock by construction: the
    Fock matrix f_pq = h_pq + sum_i [2(pq|ii) - (pi|iq)] equals diag(eps),
    which fixes h.  No nuclear repulsion term.

Similarity transform (Sec. II.A, Eqs. 1CSF-S and sim).  For the one-CSF state
with hole h and particle p, S = (1/sqrt2)(p_up^+ h_up + p_dn^+ h_dn), so
S^+ = sum_pq x_pq E_pq with the single element x[h, p] = 1/sqrt2.  For a
one-body generator K = sum kappa_pq E_pq,
    exp(K) a_q^+ exp(-K) = sum_p a_p^+ [exp(kappa)]_pq,
    exp(K) a_q   exp(-K) = sum_p [exp(-kappa)]_qp a_p,
so H-bar keeps the two-body form with h-bar = U h U^-1 and
B-bar^P = U B^P U^-1, U = exp(x) = 1 + x (x^2 = 0 because h != p).  H-bar is
not Hermitian; only (pq|rs)-bar = (rs|pq)-bar survives.

T1 dressing.  exp(-T1) H-bar exp(T1) is again an orbital transform with
kappa = -t1 (t1 as an n x n matrix with entries t1[a, i]), i.e.
U = 1 - t1, U^-1 = 1 + t1.
"""
from __future__ import annotations

import numpy as np

SQRT_HALF = 1.0 / np.sqrt(2.0)


def eri_from_df(B: np.ndarray) -> np.ndarray:
    """Full (pq|rs) = sum_P B[P,p,q] B[P,r,s]."""
    naux, n, _ = B.shape
    Bm = B.reshape(naux, n * n)
    return (Bm.T @ Bm).reshape(n, n, n, n)


def bare_hamiltonian(eps: np.ndarray, B: np.ndarray, o: int):
    """Core Hamiltonian h that makes diag(eps) the Fock matrix, and E_HF.

    h = diag(eps) - sum_i [2 (pq|ii) - (pi|iq)],  E_HF = sum_i (h_ii + eps_i).
    """
    J = np.einsum('Ppq,Pii->pq', B, B[:, :o, :o])
    K = np.einsum('Ppi,Piq->pq', B[:, :, :o], B[:, :o, :])
    h = np.diag(eps) - (2.0 * J - K)
    e_hf = float(np.sum(np.diag(h)[:o]) + np.sum(eps[:o]))
    return h, e_hf


def suppression_generator(n: int, o: int, hole: int | None, particle: int | None,
                          amplitude: float = SQRT_HALF) -> np.ndarray:
    """Matrix x of S^+ (Eq. 1CSF-S): x[h, o+p] = 1/sqrt2; zero for the ground state."""
    x = np.zeros((n, n))
    if hole is not None:
        x[hole, o + particle] = amplitude
    return x


def transform(h: np.ndarray, B: np.ndarray, U: np.ndarray, Uinv: np.ndarray):
    """Integrals of exp(K) H exp(-K) for U = exp(kappa): U h U^-1 and U B^P U^-1."""
    hbar = U @ h @ Uinv
    Bbar = np.einsum('pq,Pqr,rs->Pps', U, B, Uinv, optimize=True)
    return hbar, Bbar


def similarity_transform(h: np.ndarray, B: np.ndarray, o: int, hole=None, particle=None,
                         xsign: float = 1.0):
    """H-bar = exp(S^+) H exp(-S^+) (Eq. sim) as (h-bar, B-bar); xsign = -1 uses -S."""
    n = h.shape[0]
    x = suppression_generator(n, o, hole, particle, xsign * SQRT_HALF)
    eye = np.eye(n)
    return transform(h, B, eye + x, eye - x)


def t1_matrix(t1: np.ndarray, n: int) -> np.ndarray:
    """n x n matrix with entries [o+a, i] = t1[i, a]."""
    o, v = t1.shape
    m = np.zeros((n, n))
    m[o:, :o] = t1.T
    return m


def t1_dress(hbar: np.ndarray, Bbar: np.ndarray, t1: np.ndarray):
    """Integrals of exp(-T1) H-bar exp(T1): U = 1 - t1, U^-1 = 1 + t1."""
    n = hbar.shape[0]
    m = t1_matrix(t1, n)
    eye = np.eye(n)
    return transform(hbar, Bbar, eye - m, eye + m)


def fock(h: np.ndarray, g: np.ndarray, o: int) -> np.ndarray:
    """f_pq = h_pq + sum_k [2 (pq|kk) - (pk|kq)] for a general (non-Hermitian) H."""
    return h + 2.0 * np.einsum('pqkk->pq', g[:, :, :o, :o]) - np.einsum('pkkq->pq', g[:, :o, :o, :])


def reference_energy(h: np.ndarray, g: np.ndarray, o: int) -> float:
    """<phi0|H|phi0> = sum_i 2 h_ii + sum_ij [2 (ii|jj) - (ij|ji)]."""
    occ = slice(0, o)
    return float(2.0 * np.trace(h[occ, occ])
                 + 2.0 * np.einsum('iijj->', g[occ, occ, occ, occ])
                 - np.einsum('ijji->', g[occ, occ, occ, occ]))
