"""O-SA: spin-adapted closed-shell ASCC residual (test infrastructure).

This is the oracle the CUDA path is compared against.  It evaluates the
projected equations (Eqs. energy, amp) over H-bar = exp(S^+) H exp(-S^+)
(Eq. sim) for the singlet amplitudes t1[i,a], t2[i,j,a,b] (Sec. S1).

T1 is absorbed exactly by the orbital transform H-hat = exp(-T1) H-bar exp(T1)
(hamiltonian.t1_dress), applied to the density-fitting factor: B-hat^P =
U B-bar^P U^-1 and g-hat = (pq|rs)-hat = sum_P B-hat^P_pq B-hat^P_rs.  What
remains are the closed-shell CCSD doubles-only equations of a general
(non-Hermitian) spin-free two-body Hamiltonian; for real integrals that keep
only (pq|rs) = (rs|pq) they read, with u[i,j,a,b] = 2 t2[i,j,a,b] - t2[j,i,a,b],
L_pqrs = 2 g_pqrs - g_psrq and F the Fock matrix of H-hat:

  R1[i,a] = F_ai + sum_kcd u[k,i,c,d] g_adkc - sum_klc u[k,l,a,c] g_kilc
            + sum_kc u[i,k,a,c] F_kc
  R2 = A + B + P(C + D + E),  (P X)[i,j,a,b] = X[i,j,a,b] + X[j,i,b,a]
    A = g_aibj + sum_cd t[i,j,c,d] g_acbd                      (particle-particle ladder)
    B = sum_kl t[k,l,a,b] (g_kilj + sum_cd t[i,j,c,d] g_kcld)   (hole-hole ladder)
    C = -1/2 sum_kc t[k,j,b,c] (g_kiac - 1/2 sum_ld t[l,i,a,d] g_kdlc)
        -    sum_kc t[k,i,b,c] (g_kjac - 1/2 sum_ld t[l,j,a,d] g_kdlc)   (crossed ring)
    D = 1/2 sum_kc u[j,k,b,c] (L_aikc + 1/2 sum_ld u[i,l,a,d] L_ldkc)   (ring)
    E = sum_c t[i,j,a,c] (F_bc - sum_kld u[k,l,b,d] g_ldkc)
        - sum_k t[i,k,a,b] (F_kj + sum_lcd u[l,j,c,d] g_kdlc)           (Fock-like)
  E = <phi0|H-hat|phi0> + sum t[i,j,a,b] L_iajb.

R1 is the alpha-single projection and R2 the alpha-beta double projection.
Partial linearisation (Sec. II.C): the terms bilinear in T2 are collected in
quad(t, t); PLASCC subtracts quad(m, m) with m = T2^M (mixed doubles).

The mixed-triples slice (Sec. II.B.1) is evaluated on the slice by
t3slice.residual (the spin-orbital terms of spinorb, one spin case at a time
on spatial blocks).
"""
from __future__ import annotations

import numpy as np

from . import amplitudes as amp
from . import hamiltonian as ham

def E(*args, **kw):
    kw.setdefault("optimize", True)
    return np.einsum(*args, **kw)


class Blocks:
    """Blocks of the T1-dressed H-bar, built from the dressed DF factor."""

    def __init__(self, hh, Bh, o):
        self.o = o
        self.B = Bh
        n = hh.shape[0]
        self.n = n
        self.sl = {'o': slice(0, o), 'v': slice(o, n)}
        self._cache = {}
        # Fock matrix of H-hat: f_pq = h_pq + sum_k [2 (pq|kk) - (pk|kq)]
        J = E('Ppq,P->pq', Bh, E('Pkk->P', Bh[:, :o, :o]))
        K = E('Ppk,Pkq->pq', Bh[:, :, :o], Bh[:, :o, :])
        self.F = hh + 2.0 * J - K
        self.h = hh

    def g(self, key):
        if key not in self._cache:
            s = [self.sl[c] for c in key]
            B1 = self.B[:, s[0], s[1]]
            B2 = self.B[:, s[2], s[3]]
            naux = B1.shape[0]
            m = B1.reshape(naux, -1).T @ B2.reshape(naux, -1)
            self._cache[key] = m.reshape(B1.shape[1], B1.shape[2], B2.shape[1], B2.shape[2])
        return self._cache[key]

    def L(self, key):
        """L_pqrs = 2 g_pqrs - g_psrq for the block named by (p,q,r,s) spaces."""
        swapped = key[0] + key[3] + key[2] + key[1]
        return 2.0 * self.g(key) - self.g(swapped).transpose(0, 3, 2, 1)

    def reference_energy(self):
        o = self.o
        g = self.g('oooo')
        return float(2.0 * np.trace(self.h[:o, :o]) + 2.0 * E('iijj->', g) - E('ijji->', g))


def dressed_blocks(h, B, o, t1):
    """Blocks of exp(-T1) H exp(T1) for integrals (h, B) (B: DF factor of H)."""
    n = h.shape[0]
    m = ham.t1_matrix(t1, n)
    U = np.eye(n) - m
    Ui = np.eye(n) + m
    hh = U @ h @ Ui
    Bh = E('pq,Pqr,rs->Pps', U, B, Ui, optimize=True)
    return Blocks(hh, Bh, o)


def sym(X):
    return X + X.transpose(1, 0, 3, 2)


def tilde(t):
    """u[i,j,a,b] = 2 t[i,j,a,b] - t[j,i,a,b]."""
    return 2.0 * t - t.transpose(1, 0, 2, 3)


def quad(t, s, blk):
    """Doubles terms bilinear in T2: first factor t, second factor s."""
    ut, us = tilde(t), tilde(s)
    g_ovov = blk.g('ovov'); L_ovov = blk.L('ovov')
    # hole-hole ladder: sum_kl s[k,l,a,b] sum_cd t[i,j,c,d] g_kcld
    Wq = E('ijcd,kcld->klij', t, g_ovov)
    Bq = E('klab,klij->ijab', s, Wq)
    # crossed ring
    Xq = -0.5 * E('liad,kdlc->kiac', t, g_ovov)           # sum_ld t[l,i,a,d] g_kdlc
    Cq = -0.5 * E('kjbc,kiac->ijab', s, Xq) - E('kibc,kjac->ijab', s, Xq)
    # ring
    Yq = 0.5 * E('ilad,ldkc->aikc', ut, L_ovov)
    Dq = 0.5 * E('jkbc,aikc->ijab', us, Yq)
    # Fock-like
    Fvv = -E('klbd,ldkc->bc', ut, g_ovov)
    Foo = E('ljcd,kdlc->kj', ut, g_ovov)
    Eq = E('ijac,bc->ijab', s, Fvv) - E('ikab,kj->ijab', s, Foo)
    return Bq + sym(Cq + Dq + Eq)


def linear(t, blk):
    """Doubles terms independent of or linear in T2 (plus the driver term)."""
    o = blk.o
    u = tilde(t)
    F = blk.F
    Fov = F[:o, o:]; Fvv = F[o:, o:]; Foo = F[:o, :o]
    A = blk.g('vovo').transpose(1, 3, 0, 2) + E('ijcd,acbd->ijab', t, blk.g('vvvv'))
    Bl = E('klab,kilj->ijab', t, blk.g('oooo'))
    Cl = -0.5 * E('kjbc,kiac->ijab', t, blk.g('oovv')) - E('kibc,kjac->ijab', t, blk.g('oovv'))
    Dl = 0.5 * E('jkbc,aikc->ijab', u, blk.L('voov'))
    El = E('ijac,bc->ijab', t, Fvv) - E('ikab,kj->ijab', t, Foo)
    return A + Bl + sym(Cl + Dl + El)


def singles(t, blk):
    o = blk.o
    u = tilde(t)
    F = blk.F
    R1 = F[o:, :o].T.copy()
    R1 += E('kicd,adkc->ia', u, blk.g('vvov'))
    R1 -= E('klac,kilc->ia', u, blk.g('ooov'))
    R1 += E('ikac,kc->ia', u, F[:o, o:])
    return R1


def energy_from_blocks(t, blk):
    return blk.reference_energy() + float(E('ijab,iajb->', t, blk.L('ovov')))


def residual(hbar, Bbar, o, t1, t2, linearize=False, hole=None, particle=None,
             t3_idx=None, t3_vals=None):
    """Spin-adapted (E, R1, R2, R3) over H-bar integrals (hbar, Bbar).

    linearize=True gives PLASCC with the mixed/non-mixed split defined by
    (hole, particle); t3_idx/t3_vals carry the T3' slice (small systems only).
    """
    v = t1.shape[1]
    blk = dressed_blocks(hbar, Bbar, o, t1)
    R1 = singles(t2, blk)
    R2 = linear(t2, blk) + quad(t2, t2, blk)
    if linearize:
        _, M2, _ = amp.t2_class_masks(o, v, hole, particle)
        m = np.where(M2, t2, 0.0)
        R2 -= quad(m, m, blk)
    En = energy_from_blocks(t2, blk)
    R3 = None
    if t3_idx is not None and len(t3_idx):
        from . import t3slice
        r1x, r2x, R3 = t3slice.residual(blk, t2, t3_idx, t3_vals, hole, particle,
                                        linearize=linearize)
        R1 += r1x; R2 += r2x
    return En, R1, R2, R3
