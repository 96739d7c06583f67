"""O-BF: brute-force determinant-space definition of the ASCC equations.

Test infrastructure (oracle).  For tiny systems this module applies
exp(-T) H-bar exp(T) to the Aufbau determinant in the full space of
determinants with o alpha and o beta electrons and reads off

    E     = <phi0| exp(-T) H-bar exp(T) |phi0>          (Eq. energy)
    R_mu  = <mu|   exp(-T) H-bar exp(T) |phi0>          (Eq. amp)

for mu = alpha singles, alpha-beta doubles and alpha-beta-beta triples of the
T3' slice.  T is nilpotent, so exp(+-T) are finite Taylor series.  H-bar is
applied in second quantisation from its integrals (Eq. sim).  Partial
linearisation (Sec. II.C) is evaluated from its definition: with the mixed
doubles and T3' scaled by lambda, R(lambda) is a polynomial of degree <= 4;
PLASCC keeps its lambda^0 and lambda^1 coefficients, recovered here from five
evaluations.  FCI energies of H and H-bar come from the same Hamiltonian
matrix.

Spin orbitals: P = p (alpha) or n + p (beta).  A determinant is a bit mask;
|D> = a+_{P1} a+_{P2} ... |vac> with P1 < P2 < ...
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from . import amplitudes as amp


def _sign_below(det: int, P: int) -> int:
    return -1 if bin(det & ((1 << P) - 1)).count("1") & 1 else 1


def apply_ops(det: int, ops):
    """Apply a product of operators (listed left to right) to a determinant.

    ops: sequence of (P, is_creation).  Returns (sign, det') or None.
    """
    sign = 1
    for P, cre in reversed(ops):
        bit = 1 << P
        if cre:
            if det & bit:
                return None
            sign *= _sign_below(det, P)
            det |= bit
        else:
            if not det & bit:
                return None
            sign *= _sign_below(det, P)
            det &= ~bit
    return sign, det


class DetSpace:
    """Determinants with o alpha and o beta electrons in n spatial orbitals."""

    def __init__(self, o: int, v: int):
        self.o, self.v, self.n = o, v, o + v
        n = self.n
        alpha = [sum(1 << q for q in c) for c in itertools.combinations(range(n), o)]
        self.dets = [a | (b << n) for a in alpha for b in alpha]
        self.index = {d: k for k, d in enumerate(self.dets)}
        self.dim = len(self.dets)
        self.ref = self.index[sum(1 << q for q in range(o)) | (sum(1 << q for q in range(o)) << n)]
        self._E = None

    def spin_orb(self, p: int, beta: int) -> int:
        return p + beta * self.n

    def string_matrix(self, strings):
        """Sparse matrix of sum_k c_k * (operator string k)."""
        rows, cols, vals = [], [], []
        for coef, ops in strings:
            if coef == 0.0:
                continue
            for col, d in enumerate(self.dets):
                r = apply_ops(d, ops)
                if r is None:
                    continue
                s, d2 = r
                row = self.index.get(d2)
                if row is None:
                    continue
                rows.append(row); cols.append(col); vals.append(coef * s)
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.dim, self.dim))

    def E_ops(self):
        """Spin-free excitation operators E_pq = sum_sigma a+_{p sigma} a_{q sigma}."""
        if self._E is None:
            n = self.n
            self._E = [[self.string_matrix([(1.0, [(self.spin_orb(p, s), True), (self.spin_orb(q, s), False)])
                                            for s in (0, 1)])
                        for q in range(n)] for p in range(n)]
        return self._E

    # ----------------------------------------------------------- H-bar
    def apply_h(self, hbar: np.ndarray, V: np.ndarray, psi: np.ndarray) -> np.ndarray:
        """H psi for H = sum h_pq E_pq + 1/2 sum V_pqrs (E_pq E_rs - d_qr E_ps)."""
        n = self.n
        E = self.E_ops()
        Ev = np.array([[E[r][s] @ psi for s in range(n)] for r in range(n)]).reshape(n * n, -1)
        W = (V.reshape(n * n, n * n) @ Ev)
        k1 = hbar - 0.5 * np.einsum('pqqs->ps', V)
        out = np.zeros_like(psi)
        for p in range(n):
            for q in range(n):
                out += E[p][q] @ (0.5 * W[p * n + q] + k1[p, q] * psi)
        return out

    def hamiltonian_matrix(self, hbar: np.ndarray, V: np.ndarray) -> np.ndarray:
        return np.array([self.apply_h(hbar, V, e) for e in np.eye(self.dim)]).T

    def s2_matrix(self) -> np.ndarray:
        """S^2 = S_z^2 + S_z + S_- S_+ on this space (S_z = 0 here)."""
        n = self.n
        Sp = self.string_matrix([(1.0, [(self.spin_orb(p, 0), True), (self.spin_orb(p, 1), False)])
                                 for p in range(n)])
        return (Sp.T @ Sp).toarray()

    # ------------------------------------------------------- cluster operator
    def cluster_strings(self, t1, t2, t3_idx=None, t3_vals=None):
        """Spin-orbital operator strings of T1 + T2 + T3 from spin-adapted amplitudes."""
        o, v = self.o, self.v
        A = lambda a, s: self.spin_orb(o + a, s)
        I = lambda i, s: self.spin_orb(i, s)
        out = []
        for i in range(o):
            for a in range(v):
                for s in (0, 1):
                    out.append((t1[i, a], [(A(a, s), True), (I(i, s), False)]))
        for i, j, a, b in itertools.product(range(o), range(o), range(v), range(v)):
            out.append((t2[i, j, a, b], [(A(a, 0), True), (A(b, 1), True), (I(j, 1), False), (I(i, 0), False)]))
        t2ss = amp.t2_same_spin(t2)
        for i, j in itertools.combinations(range(o), 2):
            for a, b in itertools.combinations(range(v), 2):
                for s in (0, 1):
                    out.append((t2ss[i, j, a, b], [(A(a, s), True), (A(b, s), True), (I(j, s), False), (I(i, s), False)]))
        if t3_idx is not None and len(t3_idx):
            t3 = amp.t3_dense(t3_idx, t3_vals, o, v)
            for i in range(o):
                for j, k in itertools.combinations(range(o), 2):
                    for a in range(v):
                        for b, c in itertools.combinations(range(v), 2):
                            val = t3[i, j, k, a, b, c]
                            if val != 0.0:
                                # alpha-beta-beta
                                out.append((val, [(A(a, 0), True), (A(b, 1), True), (A(c, 1), True),
                                                  (I(k, 1), False), (I(j, 1), False), (I(i, 0), False)]))
            # alpha-alpha-beta: t_{i a j a k b}^{a a b a c b} = t3[k,i,j,c,a,b] (spin flip)
            for i, j in itertools.combinations(range(o), 2):
                for k in range(o):
                    for a, b in itertools.combinations(range(v), 2):
                        for c in range(v):
                            val = t3[k, i, j, c, a, b]
                            if val != 0.0:
                                out.append((val, [(A(a, 0), True), (A(b, 0), True), (A(c, 1), True),
                                                  (I(k, 1), False), (I(j, 0), False), (I(i, 0), False)]))
            t3ss = amp.t3_same_spin(t3)
            for i, j, k in itertools.combinations(range(o), 3):
                for a, b, c in itertools.combinations(range(v), 3):
                    val = t3ss[i, j, k, a, b, c]
                    if val != 0.0:
                        for s in (0, 1):
                            out.append((val, [(A(a, s), True), (A(b, s), True), (A(c, s), True),
                                              (I(k, s), False), (I(j, s), False), (I(i, s), False)]))
        return out

    def exp_apply(self, T, psi, sign=1.0):
        """exp(sign*T) psi as a terminating Taylor series."""
        out = psi.copy(); term = psi.copy(); k = 1
        while True:
            term = sign * (T @ term) / k
            if not np.any(np.abs(term) > 0.0):
                break
            out += term
            k += 1
            if k > 4 * self.o + 2:
                break
        return out

    # ----------------------------------------------------------- projections
    def coefficient(self, psi, ops):
        r = apply_ops(self.dets[self.ref], ops)
        s, d = r
        return s * psi[self.index[d]]

    def project(self, psi, t3_idx=None):
        o, v = self.o, self.v
        A = lambda a, s: self.spin_orb(o + a, s)
        I = lambda i, s: self.spin_orb(i, s)
        E = psi[self.ref]
        R1 = np.zeros((o, v)); R2 = np.zeros((o, o, v, v))
        for i in range(o):
            for a in range(v):
                R1[i, a] = self.coefficient(psi, [(A(a, 0), True), (I(i, 0), False)])
        for i, j, a, b in itertools.product(range(o), range(o), range(v), range(v)):
            R2[i, j, a, b] = self.coefficient(psi, [(A(a, 0), True), (A(b, 1), True), (I(j, 1), False), (I(i, 0), False)])
        R3 = np.zeros(0 if t3_idx is None else len(t3_idx))
        if t3_idx is not None:
            for q, (i, j, k, a, b, c) in enumerate(t3_idx):
                R3[q] = self.coefficient(psi, [(A(a, 0), True), (A(b, 1), True), (A(c, 1), True),
                                               (I(k, 1), False), (I(j, 1), False), (I(i, 0), False)])
        return E, R1, R2, R3


def transformed_psi(space, hbar, V, strings):
    T = space.string_matrix(strings)
    ref = np.zeros(space.dim); ref[space.ref] = 1.0
    psi = space.exp_apply(T, ref, +1.0)
    psi = space.apply_h(hbar, V, psi)
    return space.exp_apply(T, psi, -1.0)


def projected_equations(space, hbar, V, t1, t2, t3_idx=None, t3_vals=None,
                        linearize=False, hole=None, particle=None):
    """(E, R1, R2, R3) of exp(-T) H-bar exp(T) projected (Eqs. energy, amp).

    With linearize=True, the mixed doubles and all of T3' carry a factor
    lambda and only the lambda^0 + lambda^1 part is kept (Sec. II.C).  The
    ground state uses the same (hole, particle) labels for this split.
    """
    o, v = space.o, space.v
    if not linearize:
        psi = transformed_psi(space, hbar, V, space.cluster_strings(t1, t2, t3_idx, t3_vals))
        return space.project(psi, t3_idx)
    _, M2, _ = amp.t2_class_masks(o, v, hole, particle)
    t2M = np.where(M2, t2, 0.0); t2R = t2 - t2M
    lams = [0.0, 1.0, -1.0, 2.0, -2.0]
    outs = []
    for lam in lams:
        tv = None if t3_vals is None else lam * t3_vals
        psi = transformed_psi(space, hbar, V, space.cluster_strings(t1, t2R + lam * t2M, t3_idx, tv))
        outs.append(space.project(psi, t3_idx))
    Vm = np.vander(np.array(lams), 5, increasing=True)
    coef = np.linalg.solve(Vm, np.eye(5))       # rows: polynomial coefficient k
    res = []
    for part in range(4):
        stack = np.array([np.atleast_1d(np.asarray(x[part], dtype=float)).ravel() for x in outs])
        c = coef @ stack
        val = c[0] + c[1]
        res.append(val.reshape(np.shape(outs[0][part])))
    E = float(res[0]) if np.ndim(res[0]) == 0 else float(res[0].ravel()[0])
    return E, res[1], res[2], res[3]


def fci_energies(space, h, V):
    """All eigenvalues of H on the space, with <S^2> of each eigenvector."""
    H = space.hamiltonian_matrix(h, V)
    w, U = np.linalg.eig(H)
    S2 = space.s2_matrix()
    s2 = np.real(np.einsum('ik,ij,jk->k', U.conj(), S2, U) / np.einsum('ik,ik->k', U.conj(), U))
    order = np.argsort(w.real)
    return w[order], s2[order]
