"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws random numbers.  It holds none of the method's
arithmetic: no Hamiltonian, no Fock matrix, no amplitude equation.  Both the
CPU oracle and the CUDA path consume the arrays it returns.

The paper's molecules (QUEST, charge-transfer set, water clusters; Sec. III.A)
need basis sets, ESMF orbitals and integral codes that are not available, so a
synthetic closed-shell system stands in for them:

* orbital energies: occupied uniform in [-1.5, -0.3] Eh, virtual uniform in
  [0.1, 2.5] Eh, each block sorted ascending;
* a density-fitting factor B[P, p, q], P < Naux = 3 (o + v), symmetric in
  (p, q), every element N(0, sigma^2): the upper triangle is drawn and mirrored.
  (pq|rs) = sum_P B[P,p,q] B[P,r,s] then has 8-fold permutational symmetry and
  is positive semidefinite.

Integral scale.  With sigma = 0.05 for every size, every exchange integral
(pq|pq) is about Naux sigma^2 and the systems are far more strongly
correlated than the paper's molecules: at o=20, v=200 the MP2 energy is about
-3.3e4 Eh and CCSD diverges.  The default therefore fixes the coupling
kappa = 3 (o+v) v^2 sigma^4 -- the sum over virtual pairs of the mean squared
(ia|jb) for one occupied pair, which sets the size of an MP2 pair energy -- at
KAPPA = 2e-3 Eh^2, i.e. sigma = (KAPPA / (3 (o+v) v^2))^(1/4).  Passing
sigma=0.05 gives the literal distribution.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = ["System", "make_system", "random_amplitudes", "batch_workload",
           "serving_trace"]


@dataclass
class System:
    o: int                 # occupied spatial orbitals
    v: int                 # virtual spatial orbitals
    naux: int              # rank of the density-fitting factor
    eps: np.ndarray        # [o+v] orbital energies (float64)
    B: np.ndarray          # [naux, n, n] symmetric DF factor (float64, C order)
    seed: int = 0
    sigma: float = 0.0

    @property
    def n(self) -> int:
        return self.o + self.v


KAPPA = 2e-3
LITERAL_SIGMA = 0.05


def default_sigma(o: int, v: int, kappa: float = KAPPA) -> float:
    """sigma with 3 (o+v) v^2 sigma^4 = kappa (see the module docstring)."""
    return float((kappa / (3.0 * (o + v) * v * v)) ** 0.25)


def make_system(o: int, v: int, seed: int = 0, naux: int | None = None,
                sigma: float | None = None) -> System:
    """Draw one synthetic closed-shell system of o occupied and v virtual orbitals."""
    n = o + v
    if naux is None:
        naux = 3 * n
    if sigma is None:
        sigma = default_sigma(o, v)
    rng = np.random.default_rng(seed)
    eps_o = np.sort(rng.uniform(-1.5, -0.3, o))
    eps_v = np.sort(rng.uniform(0.1, 2.5, v))
    G = rng.normal(0.0, sigma, (naux, n, n))
    up = np.triu(G)
    B = up + np.transpose(np.triu(G, 1), (0, 2, 1))
    return System(o=o, v=v, naux=naux,
                  eps=np.ascontiguousarray(np.concatenate([eps_o, eps_v])),
                  B=np.ascontiguousarray(B), seed=seed, sigma=float(sigma))


def random_amplitudes(o: int, v: int, seed: int = 1, scale: float = 0.05,
                      n_t3: int = 0):
    """Random spin-adapted amplitudes for residual parity tests.

    t1[i,a] and t2[i,j,a,b] with the closed-shell pair symmetry
    t2[i,j,a,b] = t2[j,i,b,a]; when n_t3 > 0, also n_t3 random values for the
    mixed-triples slice (its element order is defined by the method code).
    """
    rng = np.random.default_rng(seed)
    t1 = scale * rng.standard_normal((o, v))
    x = scale * rng.standard_normal((o, o, v, v))
    t2 = 0.5 * (x + x.transpose(1, 0, 3, 2))
    t3 = scale * rng.standard_normal(n_t3) if n_t3 else None
    return t1, t2, t3


def batch_workload(n_problems: int = 64):
    """Batched workload: one molecule per seed 0..n-1.

    o uniform in [4, 16], v uniform in [40, 160], one to three distinct
    excitations (h in [o-3, o), p in [0, 3)) drawn from a second stream.
    Returns a list of dicts {seed, o, v, excitations=[(h, p), ...]}.
    """
    out = []
    for seed in range(n_problems):
        r = np.random.default_rng(seed)
        o = int(r.integers(4, 17))
        v = int(r.integers(40, 161))
        k = int(r.integers(1, 4))
        r2 = np.random.default_rng([seed, 1])
        pairs = [(h, p) for h in range(o - 3, o) for p in range(3)]
        pick = r2.choice(len(pairs), size=k, replace=False)
        out.append(dict(seed=seed, o=o, v=v,
                        excitations=[pairs[int(q)] for q in sorted(pick)]))
    return out


def serving_trace(n_requests: int = 500, seed: int = 12345, rate: float = 1.0,
                  o_range=(5, 40), v_range=(50, 400), max_states: int = 4):
    """Poisson arrival trace of solve requests.

    o and v are log-uniform on the given ranges (rounded), 1..max_states
    excited states per molecule (HOMO-side holes, LUMO-side particles), and
    exponential inter-arrival times of mean 1/rate seconds.
    """
    r = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for q in range(n_requests):
        t += float(r.exponential(1.0 / rate))
        o = int(round(math.exp(r.uniform(math.log(o_range[0]), math.log(o_range[1])))))
        v = int(round(math.exp(r.uniform(math.log(v_range[0]), math.log(v_range[1])))))
        k = int(r.integers(1, max_states + 1))
        pairs = [(o - 1 - (s % 2), s // 2) for s in range(k)]
        reqs.append(dict(id=q, arrival=t, seed=int(r.integers(0, 2**31 - 1)),
                         o=o, v=v, excitations=pairs))
    return reqs
