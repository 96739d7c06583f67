"""Writes tests/golden/reference_energies.txt with the CPU oracle's converged energies.

Only oracle/ and synth/ are called.  Each line: name o v seed hole particle
method energy iterations; a method ending in +T3' includes the mixed-triples
slice (Sec. II.B.1).  Run from the repository root:

    python tests/golden/make_reference_energies.py [name ...]
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import ascc  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "reference_energies.txt")

CASES = {
    # name: (o, v, seed, hole, particle, linearize, pl_hole, pl_particle[, triples])
    "c2_plascc_excited": (20, 200, 0, 19, 3, True, None, None),
    "c2_plascc_ground": (20, 200, 0, None, None, True, 19, 3),
    "c1_plascc_excited": (4, 20, 0, 3, 0, True, None, None),
    "c1_plascc_ground": (4, 20, 0, None, None, True, 3, 0),
    "c1_plascc_excited_t3": (4, 20, 0, 3, 0, True, None, None, True),
    "c1_ascc_excited_t3": (4, 20, 0, 3, 0, False, None, None, True),
    "mid_plascc_excited_t3": (9, 70, 3, 8, 2, True, None, None, True),
    "c2_plascc_excited_t3": (20, 200, 0, 19, 3, True, None, None, True),
}


def main(names):
    lines = []
    if os.path.exists(OUT):
        lines = [l for l in open(OUT) if l.strip() and not l.startswith("#")]
    done = {l.split()[0]: l for l in lines}
    for name in names:
        o, v, seed, h, p, lin, lh, lp = CASES[name][:8]
        t3 = len(CASES[name]) > 8 and CASES[name][8]
        s = synth.make_system(o, v, seed=seed)
        t0 = time.time()
        r = ascc.solve_state(s.eps, s.B, o, h, p, linearize=lin, pl_hole=lh, pl_particle=lp,
                             triples=t3, max_iter=400, verbose=True)
        assert r.converged, name
        method = ('PLASCC' if lin else 'ASCC') + ("+T3'" if t3 else '')
        done[name] = (f"{name} {o} {v} {seed} {h if h is not None else -1} "
                      f"{p if p is not None else -1} {method} "
                      f"{r.energy:.12f} {r.iterations}\n")
        print(name, r.energy, r.iterations, f"{time.time() - t0:.0f}s", flush=True)
        with open(OUT, "w") as f:
            f.write("# oracle energies (Eh), written by tests/golden/make_reference_energies.py\n")
            f.write("# name o v seed hole particle method energy iterations\n")
            for k in sorted(done):
                f.write(done[k])


if __name__ == "__main__":
    main(sys.argv[1:] or list(CASES))
