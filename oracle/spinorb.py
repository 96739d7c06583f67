"""O-SO: spin-orbital residual of the ASCC equations (test infrastructure).

The working equations are the ground-state ones over H-bar's integrals
(Sec. II.A, Eqs. energy/amp/sim).  T1 enters through the exact identity
exp(-T) H-bar exp(T) = exp(-T2-T3) H-hat exp(T2+T3), H-hat = exp(-T1) H-bar exp(T1),
which is again a two-body Hamiltonian with transformed integrals (see
hamiltonian.t1_dress).  With T1 absorbed, the projected equations are

  E   = <0| H-hat + [H-hat,T2] |0>
  R1  = <S| H-hat + [H-hat,T2] + [H-hat,T3] |0>
  R2  = <D| H-hat + [H-hat,T2] + 1/2[[H-hat,T2],T2] + [H-hat,T3] |0>
  R3  = <T| [H-hat,T2] + 1/2[[H-hat,T2],T2] + [H-hat,T3] + [[H-hat,T2],T3] |0>

(a two-body operator lowers the excitation rank by at most two, so no other
term survives).  The terms below are the Wick contractions of these
commutators for a general, non-Hermitian two-body H:  H = sum f_pq {p+ q} +
1/4 sum <pq||rs> {p+ q+ s r}, with p, q the creation indices.  Spin orbitals
are used throughout, with T2 and T3 as full antisymmetric tensors built from
the spin-adapted amplitudes (Eqs. S1, S2 and the spin flip).

Partial linearisation (Sec. II.C) removes every term with two or more factors
from T2^M and T3' (T1 is never counted); here those are the T2^M T2^M part of
the quadratic terms (R2, R3) and the T2^M T3' part of R3.
"""
from __future__ import annotations

import numpy as np

from . import amplitudes as amp
from . import hamiltonian as ham

E = np.einsum


class SpinOrbitals:
    """Index bookkeeping: occupied spin orbitals (i up..., i dn...), then virtual."""

    def __init__(self, o, v):
        self.o, self.v, self.n = o, v, o + v
        self.O, self.V = 2 * o, 2 * v
        occ = [(i, 0) for i in range(o)] + [(i, 1) for i in range(o)]
        vir = [(o + a, 0) for a in range(v)] + [(o + a, 1) for a in range(v)]
        self.orb = np.array([p for p, _ in occ + vir])
        self.spin = np.array([s for _, s in occ + vir])

    def one_body(self, f):
        same = self.spin[:, None] == self.spin[None, :]
        return f[np.ix_(self.orb, self.orb)] * same

    def two_body(self, g):
        """<PQ||RS> (P, Q creation) from spatial chemists' g[p,q,r,s] = (pq|rs)."""
        o = self.orb; s = self.spin
        # <PQ|RS> = (PR|QS) = g[p, r, q, s] delta(sP, sR) delta(sQ, sS)
        gg = g[np.ix_(o, o, o, o)].transpose(0, 2, 1, 3)
        d = (s[:, None, None, None] == s[None, None, :, None]) & (s[None, :, None, None] == s[None, None, None, :])
        phys = gg * d
        return phys - phys.transpose(0, 1, 3, 2)

    def t2(self, t2):
        o, v = self.o, self.v
        O, V = self.O, self.V
        X = np.zeros((O, O, V, V))
        X[:o, o:, :v, v:] = t2                                  # alpha beta alpha beta
        ss = amp.t2_same_spin(t2) / 4.0
        X[:o, :o, :v, :v] = ss
        X[o:, o:, v:, v:] = ss
        return (X - X.transpose(1, 0, 2, 3) - X.transpose(0, 1, 3, 2) + X.transpose(1, 0, 3, 2))

    def t3(self, t3):
        """Full antisymmetric spin-orbital triples from the dense alpha-beta-beta array."""
        o, v = self.o, self.v
        O, V = self.O, self.V
        X = np.zeros((O, O, O, V, V, V))
        X[:o, o:, o:, :v, v:, v:] = t3 / 4.0                      # alpha beta beta
        X[o:, :o, :o, v:, :v, :v] = t3 / 4.0                      # spin flip
        ss = amp.t3_same_spin(t3) / 36.0
        X[:o, :o, :o, :v, :v, :v] = ss
        X[o:, o:, o:, v:, v:, v:] = ss
        perms = [((0, 1, 2), 1), ((1, 0, 2), -1), ((0, 2, 1), -1), ((2, 1, 0), -1), ((1, 2, 0), 1), ((2, 0, 1), 1)]
        out = np.zeros_like(X)
        for po, so in perms:
            for pv, sv in perms:
                out += so * sv * X.transpose(*po, *(3 + q for q in pv))
        return out


def so_blocks(sob, h, g):
    """Fock matrix and <pq||rs> in spin orbitals, sliced into o/v blocks."""
    O = sob.O
    f = sob.one_body(ham.fock(h, g, sob.o))
    w = sob.two_body(g)
    o_, v_ = slice(0, O), slice(O, None)
    sl = {'o': o_, 'v': v_}
    blk = lambda key: w[tuple(sl[c] for c in key)]
    return f, blk, o_, v_


def quad2(t, u, blk):
    """Doubles terms bilinear in T2 (first factor t, second u), T1 = 0."""
    w = blk('oovv')
    r = np.zeros_like(t)
    r += E('ilad,jmbe,lmde->ijab', t, u, w)
    r += 0.5 * E('jlde,imab,lmde->ijab', t, u, w)
    r -= E('jlad,imbe,lmde->ijab', t, u, w)
    r -= 0.5 * E('ilde,jmab,lmde->ijab', t, u, w)
    r -= 0.5 * E('ijad,lmbe,lmde->ijab', t, u, w)
    r -= 0.5 * E('lmad,ijbe,lmde->ijab', t, u, w)
    r += 0.25 * E('ijde,lmab,lmde->ijab', t, u, w)
    return r


def residual(h, g, t1, t2, t3=None, linearize=False, hole=None, particle=None,
             triples_only=False):
    """Spin-orbital (E, R1, R2, R3) for H-bar integrals (h, g) and spin-adapted amplitudes.

    h, g: spatial H-bar integrals (g[p,q,r,s] = (pq|rs), non-Hermitian);
    t3: dense alpha-beta-beta array or None.  Returns E, R1[i,a] (alpha
    single), R2[i,j,a,b] (alpha-beta double) and, if t3 is given, the dense
    alpha-beta-beta R3.  With triples_only=True, R1 and R2 hold only the
    contributions of T3 (used by the spin-adapted oracle).
    """
    o, v = t1.shape
    sob = SpinOrbitals(o, v)
    hh, gg = _dress_full(h, g, t1)
    f, blk, oo, vv = so_blocks(sob, hh, gg)
    T = sob.t2(t2)
    T3 = sob.t3(t3) if t3 is not None else None
    fov, foo, fvv = f[oo, vv], f[oo, oo], f[vv, vv]
    Tm = None
    if linearize:
        _, M2, _ = amp.t2_class_masks(o, v, hole, particle)
        Tm = sob.t2(np.where(M2, t2, 0.0))

    e_ref = float(np.trace(sob.one_body(hh)[oo, oo]) + 0.5 * E('ijij->', blk('oooo')))
    E_ = e_ref + 0.25 * E('lmde,lmde->', T, blk('oovv'))

    R1 = np.zeros((sob.O, sob.V))
    R2 = np.zeros((sob.O, sob.O, sob.V, sob.V))
    if not triples_only:
        R1 += f[vv, oo].T
        R1 += E('ld,ilad->ia', fov, T)
        R1 += 0.5 * E('ilde,alde->ia', T, blk('vovv'))
        R1 -= 0.5 * E('lmad,lmid->ia', T, blk('ooov'))

        R2 += blk('vvoo').transpose(2, 3, 0, 1)
        R2 += E('bd,ijad->ijab', fvv, T)
        R2 -= E('ad,ijbd->ijab', fvv, T)
        R2 += E('li,jlab->ijab', foo, T)
        R2 -= E('lj,ilab->ijab', foo, T)
        R2 += E('ilad,bljd->ijab', T, blk('voov'))
        R2 += E('jlbd,alid->ijab', T, blk('voov'))
        R2 -= E('jlad,blid->ijab', T, blk('voov'))
        R2 -= E('ilbd,aljd->ijab', T, blk('voov'))
        R2 += 0.5 * E('lmab,lmij->ijab', T, blk('oooo'))
        R2 += 0.5 * E('ijde,abde->ijab', T, blk('vvvv'))
        R2 += quad2(T, T, blk)
        if Tm is not None:
            R2 -= quad2(Tm, Tm, blk)

    R3 = None
    if T3 is not None:
        R1 += 0.25 * E('ilmade,lmde->ia', T3, blk('oovv'))
        R2 += E('ld,ijlabd->ijab', fov, T3)
        R2 += 0.5 * E('jlmabd,lmid->ijab', T3, blk('ooov'))
        R2 -= 0.5 * E('ilmabd,lmjd->ijab', T3, blk('ooov'))
        R2 += 0.5 * E('ijlade,blde->ijab', T3, blk('vovv'))
        R2 -= 0.5 * E('ijlbde,alde->ijab', T3, blk('vovv'))
        R3full = triples_residual(T, T3, f, blk, oo, vv, Tm)
        R3 = R3full[:o, o:, o:, :v, v:, v:]
    return E_, R1[:o, :v], R2[:o, o:, :v, v:], R3


def _dress_full(h, g, t1):
    """T1-dressed spatial integrals from full (h, g): U = 1 - t1, U^-1 = 1 + t1."""
    n = h.shape[0]
    m = ham.t1_matrix(t1, n)
    U = np.eye(n) - m; Ui = np.eye(n) + m
    hh = U @ h @ Ui
    gg = E('pa,abcd,bq,rc,ds->pqrs', U, g, Ui, U, Ui, optimize=True)
    return hh, gg


def triples_residual(T, T3, f, blk, oo, vv, Tm=None):
    """Triples projection from the generated Wick terms (so_triples_terms).

    With Tm (the mixed doubles) given, the partially linearised form drops
    the Tm x Tm part of 1/2[[H,T2],T2] and the Tm x T3 part of [[H,T2],T3].
    """
    from .so_triples_terms import TERMS
    sl = {'o': oo, 'v': vv}

    def operand(key, t2):
        name, b = key.split(':')
        if name == 'f':
            return f[sl[b[0]], sl[b[1]]]
        if name == 'v':
            return blk(b)
        if name == 't2':
            return t2
        return T3

    def group(name, t2):
        acc = 0.0
        for coef, spec, ops in TERMS[name]:
            acc = acc + coef * np.einsum(spec, *[operand(k, t2) for k in ops], optimize=True)
        return acc

    R3 = group('H_T2', T) + group('H_T2_T2', T) + group('H_T3', T)
    if Tm is None:
        R3 = R3 + group('H_T2_T3', T)
    else:
        R3 = R3 - group('H_T2_T2', Tm) + group('H_T2_T3', T - Tm)
    return R3
