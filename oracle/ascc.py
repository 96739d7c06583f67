"""Oracle entry points: one ASCC / PLASCC / ground-state solve (test infrastructure).

A state is the ground state (hole = None: S = 0, CCSD or its partially
linearised form with the primary labels (pl_hole, pl_particle), Sec. II.C) or
a one-CSF excited state (hole, particle) with S of Eq. 1CSF-S.  The
excitation energy is E(excited) - E(ground) (Sec. II.B.1).
"""
from __future__ import annotations

import numpy as np

from . import amplitudes as amp
from . import hamiltonian as ham
from . import solver
from . import spinadapted as sa


def prepare(eps, B, o, hole=None, particle=None, xsign=1.0):
    h, e_hf = ham.bare_hamiltonian(eps, B, o)
    hbar, Bbar = ham.similarity_transform(h, B, o, hole, particle, xsign)
    return hbar, Bbar, e_hf


def ansatz_beta(alpha, ansatz):
    """(beta, sign of S) of the two ansatz choices for Aufbau weight alpha (Sec. II.D).

    ansatz 0: beta = 1/(1+alpha) with S as given.  ansatz 1: the hole orbital
    with flipped sign, which turns alpha into -alpha (beta = 1/(1-alpha));
    written in the original orbitals this is S -> -S, i.e. exp(+S^+) exp(T)
    with T^P(0) = -beta S + gamma S^2.
    """
    lo, hi = amp.beta_from_alpha(alpha)
    return (lo, 1.0) if ansatz == 0 else (hi, -1.0)


def solve_state(eps, B, o, hole=None, particle=None, linearize=True, triples=False,
                pl_hole=None, pl_particle=None, beta=1.0, r_tol=1e-8, e_tol=1e-10,
                max_iter=200, diis_dim=16, diis_start=3, verbose=False, xsign=1.0):
    v = len(eps) - o
    hbar, Bbar, _ = prepare(eps, B, o, hole, particle, xsign)
    lh, lp = (hole, particle) if hole is not None else (pl_hole, pl_particle)
    if lh is None:
        linearize = False
    idx = amp.t3p_index(o, v, hole, particle) if (triples and hole is not None) else np.zeros((0, 6), np.int64)
    t1, t2, t3 = amp.initial_guess(o, v, hole, particle, beta, len(idx), xsign)

    def fn(a, b, c):
        E, R1, R2, R3 = sa.residual(hbar, Bbar, o, a, b, linearize=linearize, hole=lh,
                                    particle=lp, t3_idx=idx if len(idx) else None, t3_vals=c)
        return E, R1, R2, (R3 if R3 is not None else np.zeros(0))

    def fock(a):
        F = sa.dressed_blocks(hbar, Bbar, o, a).F
        return F[hole, o + particle], F[o + particle, hole]

    res = solver.solve(fn, eps, o, t1, t2, t3, t3_idx=idx, r_tol=r_tol, e_tol=e_tol,
                       max_iter=max_iter, diis_dim=diis_dim, diis_start=diis_start,
                       verbose=verbose, hole=hole, particle=particle,
                       fock_fn=fock if hole is not None else None)
    return res
