"""Writes tests/golden/c2_t3_residual.txt: the CPU oracle's PLASCC residual with
the mixed-triples slice T3' (Sec. II.B.1) at o=20, v=200 (seed 0, excitation
19 -> 3), at seeded random amplitudes added to the zeroth-order guess.

Only oracle/ and synth/ are called.  The file holds the energy, the 2-norms
and max-norms of R1, R2 and R3', and a seeded sample of their entries (flat
index, value), so that a GPU test can check the full-size residual element by
element at the sampled positions.  Run from the repository root (about half
an hour on 8 cores, ~40 GB of host memory):

    python tests/golden/make_c2_t3_residual.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import amplitudes as amp  # noqa: E402
from oracle import ascc  # noqa: E402
from oracle import spinadapted as sa  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_t3_residual.txt")
O, V, SEED, HOLE, PART = 20, 200, 0, 19, 3
AMP_SEED, AMP_SCALE = 21, 0.01
SAMPLE_SEED, N_SAMPLE = 5, 400


def amplitudes():
    """The amplitudes of the check: the zeroth-order guess plus seeded noise."""
    idx = amp.t3p_index(O, V, HOLE, PART)
    t1, t2, t3 = synth.random_amplitudes(O, V, seed=AMP_SEED, scale=AMP_SCALE, n_t3=len(idx))
    g1, g2, _ = amp.initial_guess(O, V, HOLE, PART)
    return idx, t1 + g1, t2 + g2, t3


def sample_positions(n1, n2, n3):
    rng = np.random.default_rng(SAMPLE_SEED)
    return (np.sort(rng.choice(n1, N_SAMPLE, replace=False)),
            np.sort(rng.choice(n2, N_SAMPLE, replace=False)),
            np.sort(rng.choice(n3, N_SAMPLE, replace=False)))


def main():
    s = synth.make_system(O, V, seed=SEED)
    hbar, Bbar, _ = ascc.prepare(s.eps, s.B, O, HOLE, PART)
    idx, t1, t2, t3 = amplitudes()
    t0 = time.time()
    E, R1, R2, R3 = sa.residual(hbar, Bbar, O, t1, t2, linearize=True, hole=HOLE, particle=PART,
                                t3_idx=idx, t3_vals=t3)
    p1, p2, p3 = sample_positions(R1.size, R2.size, R3.size)
    with open(OUT, "w") as f:
        f.write("# oracle PLASCC+T3' residual at o=20 v=200 seed 0, excitation 19->3, amplitudes =\n")
        f.write(f"# guess + synth.random_amplitudes(seed={AMP_SEED}, scale={AMP_SCALE}); "
                "written by tests/golden/make_c2_t3_residual.py\n")
        f.write(f"energy {E:.15e}\n")
        for name, R in (("r1", R1), ("r2", R2), ("r3", R3)):
            f.write(f"norm {name} {np.linalg.norm(R):.15e} {np.abs(R).max():.15e}\n")
        for name, R, pos in (("r1", R1.ravel(), p1), ("r2", R2.ravel(), p2), ("r3", R3, p3)):
            for q in pos:
                f.write(f"{name} {int(q)} {R[q]:.17e}\n")
    print(f"wrote {OUT} in {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
