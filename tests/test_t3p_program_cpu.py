"""The generated T3' program (paper_2501_10515_gb300/csrc/t3p_program.inc,
written by csrc/gen_t3p.py) executed op by op with numpy, each intermediate
in its own array and the stacks as row blocks, against the spin-orbital
oracle's T3' contributions to R1 and R2 and its R3' (Sec. II.B.1, and the
partial linearisation of Sec. II.C).  This checks the generator's algebra on
the CPU, independently of the GPU executor's placement and streams (which
tests/test_t3p_plan.py checks)."""
import os
import re

import numpy as np
import pytest

import synth
from oracle import amplitudes as amp, hamiltonian as ham, spinadapted as sa, spinorb as so

INC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2501_10515_gb300", "csrc", "t3p_program.inc")
BASES = ("F", "B", "t2", "ts", "TA", "TB", "TC", "TD", "r1", "r2", "RA", "RB", "RC", "RD")
BDIMS = {"F": "nn", "B": "Pnn", "t2": "oovv", "ts": "oovv", "TA": "ovv", "TB": "ovv",
         "TC": "oov", "TD": "oov", "r1": "ov", "r2": "oovv", "RA": "ovv", "RB": "ovv",
         "RC": "oov", "RD": "oov"}


def _table():
    src = open(INC).read()
    head, ops_part = src.split("kT3pOps[]")
    tens = re.findall(r'\{(\d+), (-?\d+), "([^"]*)", "([^"]*)", (\d+), "([^"]*)"\},', head)
    ops = re.findall(r'\{(\d+), (\d+), (-?\d+), (-?\d+), (-?\d+), "([^"]*)", ([^,]+), (-?\d+), '
                     r'"([^"]*)", (-?\d+)\},', ops_part)
    return tens, ops


def _run_program(o, v, naux, hole, part, blk, t2, tm, t3d, linearize):
    tens, ops = _table()
    n = o + v
    D = {"o": o, "v": v, "P": naux}
    TA = t3d[hole, hole, :, part, :, :].copy(); TA[hole] = 0
    TB = t3d[hole, hole, :, :, part, :].copy(); TB[hole] = 0; TB[:, part, :] = 0; TB[:, :, part] = 0
    TC = t3d[hole, :, :, part, part, :].copy(); TC[hole] = 0; TC[:, hole] = 0; TC[:, :, part] = 0
    TD = t3d[:, hole, :, part, part, :].copy(); TD[hole] = 0; TD[:, hole] = 0; TD[:, :, part] = 0
    base = {"F": blk.F, "B": blk.B, "TA": TA, "TB": TB, "TC": TC, "TD": TD,
            "r1": np.zeros((o, v)), "r2": np.zeros((o, o, v, v)), "RA": np.zeros((o, v, v)),
            "RB": np.zeros((o, v, v)), "RC": np.zeros((o, o, v)), "RD": np.zeros((o, o, v))}

    def select(name, spec):
        sl = []
        for d, c in zip(BDIMS[name], spec):
            full = d == "n"
            if c == "h":
                sl.append(hole)
            elif c == "p":
                sl.append((o if full else 0) + part)
            elif c == "o":
                sl.append(slice(0, o))
            elif c == "v":
                sl.append(slice(o, n) if full else slice(0, v))
            else:
                sl.append(slice(None))
        return tuple(sl)

    def rows_of(rows):
        return [int(np.prod([D[c] for c in r])) if r else 1 for r in rows.split("+")]

    def shape_of(t):
        kind, b, spec, dims, sec, rows = tens[t]
        return [sum(rows_of(rows)) if c == "#" else D[c] for c in dims]

    val = {}  # intermediates (later sections read those of earlier ones)

    def run(section, t2b, scale):
        base["t2"] = t2b
        base["ts"] = t2b - t2b.transpose(1, 0, 2, 3)

        def get(t):
            kind, b = tens[t][0], int(tens[t][1])
            return base[BASES[b]] if kind == "0" else val[t]

        for sec, kind, out, a, b, spec, alpha, ob, ospec, member in ops:
            if int(sec) != section:
                continue
            kind, out, a, b = int(kind), int(out), int(a), int(b)
            alpha, member = float(alpha), int(member)
            if kind == 0:
                nm = BASES[int(ob)]
                val[out] = np.array(base[nm][select(nm, tens[out][2])], copy=True)
            elif kind == 1:
                val[out] = alpha * np.einsum(spec, get(a), get(b))
            elif kind == 2:
                nm = BASES[int(ob)]
                base[nm][select(nm, ospec)] += scale * alpha * np.einsum(spec, get(a), get(b))
            elif kind == 3:
                lhs, rhs = spec.split("->")
                rows = rows_of(tens[out][5])
                off = sum(rows[:member])
                if out not in val:
                    val[out] = np.zeros(shape_of(out))
                y = np.einsum(f"{lhs}->{rhs}", get(a))
                val[out][off:off + rows[member]] = y.reshape((rows[member],) + val[out].shape[1:])
            else:
                lhs, rhs = spec.split("->")
                w = get(a)
                rows = rows_of(tens[a][5])
                off = sum(rows[:member])
                gdims = tens[a][5].split("+")[member]
                fshape = list(w.shape[:-1])
                wm = w[..., off:off + rows[member]].reshape(fshape + [D[c] for c in gdims])
                res = np.einsum(f"{lhs}->{rhs}", wm)
                if out >= 0:
                    val[out] = alpha * res
                else:
                    nm = BASES[int(ob)]
                    base[nm][select(nm, ospec)] += scale * alpha * res

    run(0, t2, 1.0)
    run(1, t2, 1.0)
    run(2, t2, 1.0)
    if linearize:
        run(2, tm, -1.0)
        run(3, t2 - tm, 1.0)
    else:
        run(3, t2, 1.0)
    return base


def _gather_blocks(base, idx, hole, part):
    got = np.zeros(len(idx))
    for q, (i, j, k, a, b, c) in enumerate(idx):
        sg = 1
        if i == hole and (j == hole or k == hole):
            if j != hole:
                j, k, sg = k, j, -sg
            if a == part:
                got[q] = sg * base["RA"][k, b, c]
            else:
                if b != part:
                    b, c, sg = c, b, -sg
                got[q] = sg * base["RB"][k, a, c]
        elif i == hole:
            if b != part:
                b, c, sg = c, b, -sg
            got[q] = sg * base["RC"][j, k, c]
        else:
            if j != hole:
                j, k, sg = k, j, -sg
            if b != part:
                b, c, sg = c, b, -sg
            got[q] = sg * base["RD"][i, k, c]
    return got


@pytest.mark.parametrize("o,v,hole,part,linearize", [(3, 6, 2, 1, True), (3, 6, 1, 0, False),
                                                     (4, 7, 3, 2, True)])
def test_generated_program_matches_spin_orbital_oracle(o, v, hole, part, linearize):
    s = synth.make_system(o, v, seed=4, sigma=0.2)
    h, _ = ham.bare_hamiltonian(s.eps, s.B, o)
    hb, Bb = ham.similarity_transform(h, s.B, o, hole, part)
    idx = amp.t3p_index(o, v, hole, part)
    t1, t2, t3v = synth.random_amplitudes(o, v, seed=11, scale=0.1, n_t3=len(idx))
    blk = sa.dressed_blocks(hb, Bb, o, t1)
    t3d = amp.t3_dense(idx, t3v, o, v)
    _, M2, _ = amp.t2_class_masks(o, v, hole, part)
    tm = np.where(M2, t2, 0.0)
    base = _run_program(o, v, s.naux, hole, part, blk, t2, tm, t3d, linearize)
    _, r1x, r2x, r3 = so.residual(hb, ham.eri_from_df(Bb), t1, t2, t3d, linearize=linearize,
                                  hole=hole, particle=part, triples_only=True)
    want = amp.t3_gather(r3, idx)
    got = _gather_blocks(base, idx, hole, part)
    rel = lambda x, y: np.abs(x - y).max() / max(np.abs(y).max(), 1e-300)
    assert rel(base["r1"], r1x) < 1e-10
    assert rel(base["r2"], r2x) < 1e-10
    assert rel(got, want) < 1e-10
