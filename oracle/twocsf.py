"""O-BF for two-CSF ASCC (Sec. II.B.2): brute-force determinant-space definition.

Test infrastructure (oracle): only tests and the benchmark's CPU leg call it.

The excited-state reference of Eq. 2csf is a(phi_{h1}^{p1} + phi_{h1b}^{p1b})
+ b(phi_{h2}^{p2} + phi_{h2b}^{p2b}) with 2a^2 + 2b^2 = 1, and S = T1^{P(0)}
is the one-body operator that makes it from phi0:

    S = a sum_sigma a+_{p1 sigma} a_{h1 sigma} + b sum_sigma a+_{p2 sigma} a_{h2 sigma}.

As in the one-CSF case (Sec. II.A) the Hamiltonian is H-bar = exp(S+) H
exp(-S+), the wave function exp(-S+) exp(T) phi0, and the equations are the
projections of exp(-T) H-bar exp(T) phi0 on phi0 (energy) and on the
determinants of the amplitude space (residuals).

Amplitude space (Sec. II.B.2, the two-CSF amplitude choices): the primary
spin orbitals are h1, h2, p1, p2 in both spins.  Singles and doubles are
kept whole; triples with at least three primary spin-orbital indices (T3'),
quadruples with at least five (T4') and, for the excited state, quintuples
with at least seven (T5').  The ground state keeps T1 + T2 + T3' + T4' with
the same primary labels and S = 0.  Amplitudes are spin-orbital (one per
excitation with equal numbers of alpha electrons removed and added), so no
spin-adaptation relation enters; the space is closed under spin rotations
(primary is a property of the spatial orbital), and the solution is a
singlet.

Initial guess: T^{P(0)} must make exp(-S+) exp(T^{P(0)}) phi0 equal the
reference.  Since S+ S phi0 = (2a^2 + 2b^2) phi0 = phi0 and S+ phi0 = 0,
exp(-S+)(1 + S) phi0 = S phi0, so exp(T^{P(0)}) phi0 = (1 + S) phi0 and
T^{P(0)} = ln(1 + S) = S - S^2/2 + S^3/3 - S^4/4 (excitation operators
commute; S^5 phi0 = 0): all-primary singles to quadruples, as the section
states.

Partial linearisation (Sec. II.C) applies as in the one-CSF case: with
T = T^P + T^N + T1^M + lambda T^M_{>=2} (an excitation is P when every index
is primary, N when none is, M otherwise; all-primary triples and quadruples
are T^P here), PLASCC keeps the lambda^0 + lambda^1 part of the projections,
the ground state with the same primary labels.

The equations are solved by Newton's method with the exact Jacobian
dR_mu/dt_nu = <mu| exp(-T) [H-bar, X_nu] exp(T) |phi0> (X_nu commutes with T).
The paper obtains the reference from ESMF (Sec. III.A); cis_two_csf stands in
for it with the two largest CSFs of a singlet CIS vector.

Pins (tests/test_twocsf_oracle.py): the guess reproduces the reference
exactly; with every orbital primary (o = v = 2) the energies are FCI
eigenvalues; with b = 0 and one primary pair the energy is the one-CSF
ASCC / PLASCC + T3' oracle's; the example determinants the section prints belong to
T4' and T5'; the converged state is a singlet; the CIS matrix is H on
the singlet singles.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from . import hamiltonian as ham
from .bruteforce import DetSpace, apply_ops

# minimum number of primary spin-orbital indices per excitation rank
EXCITED_RULE = {1: 0, 2: 0, 3: 3, 4: 5, 5: 7}
GROUND_RULE = {1: 0, 2: 0, 3: 3, 4: 5}


def excitations(space: DetSpace, prim_occ, prim_vir, rule):
    """Spin-orbital excitations (occupied tuple, virtual tuple), each sorted,
    with as many alpha electrons removed as added, kept by `rule` (rank ->
    minimum count of primary spin orbitals; a rank absent from it is
    dropped).  prim_occ / prim_vir: primary spatial orbitals, 0-based within
    the occupied / virtual block."""
    o, v, n = space.o, space.v, space.n
    occ = [space.spin_orb(i, s) for s in (0, 1) for i in range(o)]
    vir = [space.spin_orb(o + a, s) for s in (0, 1) for a in range(v)]
    p_occ = {space.spin_orb(i, s) for i in prim_occ for s in (0, 1)}
    p_vir = {space.spin_orb(o + a, s) for a in prim_vir for s in (0, 1)}
    out = []
    for r in sorted(rule):
        for I in itertools.combinations(occ, r):
            na = sum(1 for q in I if q < n)
            for A in itertools.combinations(vir, r):
                if sum(1 for q in A if q < n) != na:
                    continue
                prim = sum(1 for q in I if q in p_occ) + sum(1 for q in A if q in p_vir)
                if prim >= rule[r]:
                    out.append((I, A))
    return out


def excitation_ops(I, A):
    """a+_{A1} ... a+_{Ar} a_{Ir} ... a_{I1}: the operator string whose
    coefficient in T is the amplitude of (I, A)."""
    return [(q, True) for q in A] + [(q, False) for q in reversed(I)]


class TwoCSF:
    """One two-CSF state (or the ground state with the same primary labels)
    of a tiny system, in the full determinant space with o alpha and o beta
    electrons."""

    def __init__(self, eps, B, o, h1, p1, h2, p2, a, b, excited=True, prim_occ=None,
                 prim_vir=None, linearize=False):
        v = len(eps) - o
        self.space = sp_ = DetSpace(o, v)
        self.o, self.v = o, v
        h, self.e_hf = ham.bare_hamiltonian(np.asarray(eps, float), np.asarray(B, float), o)
        V = ham.eri_from_df(np.asarray(B, float))
        H = sp_.hamiltonian_matrix(h, V)
        self.H = H
        self.prim_occ = sorted({h1, h2}) if prim_occ is None else sorted(prim_occ)
        self.prim_vir = sorted({p1, p2}) if prim_vir is None else sorted(prim_vir)
        self.excited = excited
        so = sp_.spin_orb
        if excited:
            strings = [(a, [(so(o + p1, s), True), (so(h1, s), False)]) for s in (0, 1)]
            strings += [(b, [(so(o + p2, s), True), (so(h2, s), False)]) for s in (0, 1)]
            S = sp_.string_matrix(strings).toarray()
        else:
            S = np.zeros((sp_.dim, sp_.dim))
        self.S = S
        Sd = S.T.copy()                                   # S+ (real coefficients)
        eSd = self._exp(Sd, +1.0)
        emSd = self._exp(Sd, -1.0)
        self.Hbar = eSd @ H @ emSd                        # Sec. II.A form, Eq. sim
        self.ref = np.zeros(sp_.dim)
        self.ref[sp_.ref] = 1.0
        rule = EXCITED_RULE if excited else GROUND_RULE
        self.exc = excitations(sp_, self.prim_occ, self.prim_vir, rule)
        self.X = [sp_.string_matrix([(1.0, excitation_ops(I, A))]).tocsr() for I, A in self.exc]
        # determinant and phase of each excitation applied to phi0
        self.pos, self.sgn = [], []
        for I, A in self.exc:
            s, d = apply_ops(sp_.dets[sp_.ref], excitation_ops(I, A))
            self.pos.append(sp_.index[d])
            self.sgn.append(float(s))
        self.pos = np.array(self.pos)
        self.sgn = np.array(self.sgn)
        # partial linearisation (Sec. II.C): T = T^P + T^N + T1^M + lambda T^M_{>=2},
        # an excitation being P if all its indices are primary, N if none is
        p_so = ({sp_.spin_orb(i, s_) for i in self.prim_occ for s_ in (0, 1)}
                | {sp_.spin_orb(o + a_, s_) for a_ in self.prim_vir for s_ in (0, 1)})
        nprim = np.array([sum(q in p_so for q in I + A) for I, A in self.exc])
        rank = np.array([len(I) for I, _ in self.exc])
        self.scaled = (nprim > 0) & (nprim < 2 * rank) & (rank >= 2)
        self.linearize = linearize

    # ------------------------------------------------------------ helpers
    def _exp(self, M, sign):
        """exp(sign M) for a nilpotent M, as its terminating Taylor series."""
        out = np.eye(M.shape[0])
        term = np.eye(M.shape[0])
        for k in range(1, 4 * self.o + 3):
            term = sign * (M @ term) / k
            if not np.any(term):
                break
            out = out + term
        return out

    def _exp_apply(self, T, X, sign):
        out = X.copy()
        term = X.copy()
        for k in range(1, 4 * self.o + 3):
            term = sign * (T @ term) / k
            if not np.any(term):
                break
            out = out + term
        return out

    def cluster(self, t):
        T = sp.csr_matrix((self.space.dim, self.space.dim))
        for c, X in zip(t, self.X):
            if c != 0.0:
                T = T + c * X
        return T

    def amplitudes_of(self, psi):
        """Amplitudes of the excitations that make psi from phi0 (coefficient
        of the excitation's determinant, in the phase of its operator string)."""
        return self.sgn * psi[self.pos]

    # ------------------------------------------------------------ equations
    def reference_state(self):
        """The reference of Eq. 2csf (phi0-free), S phi0."""
        return self.S @ self.ref

    def guess(self):
        """T^{P(0)} = ln(1 + S) applied to phi0, read off as amplitudes."""
        if not self.excited:
            return np.zeros(len(self.exc))
        Sphi = [self.ref]
        for _ in range(4):
            Sphi.append(self.S @ Sphi[-1])
        tphi = sum(((-1.0) ** (k + 1) / k) * Sphi[k] for k in range(1, 5))
        return self.amplitudes_of(tphi)

    def wavefunction(self, t):
        """exp(-S+) exp(T) phi0."""
        T = self.cluster(t)
        u = self._exp_apply(T, self.ref, +1.0)
        return self._exp(self.S.T.copy(), -1.0) @ u

    # with the mixed amplitudes of rank >= 2 scaled by lambda, the projections
    # are polynomials of degree <= 4 in lambda (a two-body H-bar); PLASCC keeps
    # their lambda^0 + lambda^1 coefficients, taken from five evaluations
    _LAMS = np.array([0.0, 1.0, -1.0, 2.0, -2.0])

    def _linear_part(self, f, t):
        coef = np.linalg.solve(np.vander(self._LAMS, 5, increasing=True), np.eye(5))
        vals = [f(np.where(self.scaled, lam * t, t), lam) for lam in self._LAMS]
        return [sum((coef[0, q] + coef[1, q]) * vals[q][k] for q in range(5))
                for k in range(len(vals[0]))]

    def equations(self, t):
        """(E, R): projections of exp(-T) H-bar exp(T) phi0 (Eqs. energy, amp);
        with linearize, their lambda^0 + lambda^1 part (Sec. II.C)."""
        if self.linearize:
            E, R = self._linear_part(lambda tl, lam: self._equations(tl), t)
            return float(E), R
        return self._equations(t)

    def _equations(self, t):
        T = self.cluster(t)
        u = self._exp_apply(T, self.ref, +1.0)
        psi = self._exp_apply(T, self.Hbar @ u, -1.0)
        return float(psi[self.space.ref]), self.amplitudes_of(psi)

    def jacobian(self, t):
        """dR_mu / dt_nu = <mu| exp(-T) (H-bar X_nu - X_nu H-bar) exp(T) |phi0>;
        with linearize, of the lambda^0 + lambda^1 part (a scaled amplitude's
        column carries the factor lambda)."""
        if self.linearize:
            return self._linear_part(
                lambda tl, lam: (self._jacobian(tl) * np.where(self.scaled, lam, 1.0)[None, :],),
                t)[0]
        return self._jacobian(t)

    def _jacobian(self, t):
        T = self.cluster(t)
        u = self._exp_apply(T, self.ref, +1.0)
        Hu = self.Hbar @ u
        C = np.stack([X @ u for X in self.X], axis=1)
        D = np.stack([X @ Hu for X in self.X], axis=1)
        W = self._exp_apply(T, self.Hbar @ C - D, -1.0)
        return self.sgn[:, None] * W[self.pos, :]

    def solve(self, r_tol=1e-11, max_iter=60):
        """Newton's method from the guess, each step halved until |R| drops
        (a full step can overshoot from the zeroth-order guess); returns
        (E, t, iterations).  The fixed point does not depend on the solver."""
        t = self.guess()
        E, R = self.equations(t)
        for it in range(max_iter):
            if np.abs(R).max() <= r_tol:
                return E, t, it
            d = np.linalg.solve(self.jacobian(t), R)
            r0 = np.linalg.norm(R)
            lam = 1.0
            while True:
                tn = t - lam * d
                En, Rn = self.equations(tn)
                if np.linalg.norm(Rn) < (1.0 - 1e-4 * lam) * r0 or lam < 1e-4:
                    break
                lam *= 0.5
            t, E, R = tn, En, Rn
        if np.abs(R).max() > r_tol:
            raise RuntimeError("two-CSF Newton iteration did not converge")
        return E, t, max_iter


def cis_singlet_matrix(eps, B, o):
    """Singlet CIS matrix over the CSFs (phi_i^a + phi_ib^ab)/sqrt(2), row
    i * v + a: A[ia, jb] = delta_ij delta_ab (e_a - e_i) + 2 (ia|jb) - (ij|ab)."""
    eps = np.asarray(eps, float)
    v = len(eps) - o
    g = ham.eri_from_df(np.asarray(B, float))
    A = np.zeros((o * v, o * v))
    for i, a in itertools.product(range(o), range(v)):
        for j, b in itertools.product(range(o), range(v)):
            A[i * v + a, j * v + b] = ((i == j) * (a == b) * (eps[o + a] - eps[i])
                                       + 2.0 * g[i, o + a, j, o + b] - g[i, j, o + a, o + b])
    return A


def cis_two_csf(eps, B, o, root):
    """A two-CSF reference from a singlet CIS vector (stand-in for the ESMF
    wave function of Sec. III.A, which is CIS with orbital relaxation): the two
    largest singlet CSF coefficients c1 (h1 -> p1) and c2 (h2 -> p2) of CIS
    root `root`, scaled to 2a^2 + 2b^2 = 1 (Eq. 2csf).  Returns (h1, p1, h2,
    p2, a, b, weights of the three largest CSFs)."""
    v = len(eps) - o
    _, U = np.linalg.eigh(cis_singlet_matrix(eps, B, o))
    c = U[:, root]
    order = np.argsort(-np.abs(c))
    (h1, p1), (h2, p2) = divmod(int(order[0]), v), divmod(int(order[1]), v)
    nrm = np.sqrt(2.0 * (c[order[0]] ** 2 + c[order[1]] ** 2))
    return h1, p1, h2, p2, c[order[0]] / nrm, c[order[1]] / nrm, np.abs(c[order[:3]])
