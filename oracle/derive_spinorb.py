"""Regenerates oracle/so_triples_terms.py (test infrastructure; needs sympy).

Wick's theorem for the triples projection of the T1-free commutator series

    <T| [H,T2] + 1/2 [[H,T2],T2] + [H,T3] + [[H,T2],T3] |0>

for a general two-body H = sum f_pq {p+ q} + 1/4 sum v_pqrs {p+ q+ s r}
(upper indices of v are the creation indices; nothing assumes hermiticity),
evaluated with sympy.physics.secondquant as a library step, then written out
as einsum terms grouped by commutator.  Run:  python -m oracle.derive_spinorb
"""
from __future__ import annotations

import re
import sys


def derive(group: int):
    from sympy import Dummy, Rational, expand, symbols
    from sympy.physics.secondquant import (AntiSymmetricTensor, Commutator, F, Fd, NO,
                                           evaluate_deltas, substitute_dummies, wicks)
    p, q, r, s = symbols('p,q,r,s', cls=Dummy)
    H = (AntiSymmetricTensor('f', (p,), (q,)) * NO(Fd(p) * F(q))
         + Rational(1, 4) * AntiSymmetricTensor('v', (p, q), (r, s)) * NO(Fd(p) * Fd(q) * F(s) * F(r)))

    def T2():
        i, j = symbols('i,j', below_fermi=True, cls=Dummy)
        a, b = symbols('a,b', above_fermi=True, cls=Dummy)
        return Rational(1, 4) * AntiSymmetricTensor('t', (a, b), (i, j)) * NO(Fd(a) * Fd(b) * F(j) * F(i))

    def T3():
        i, j, k = symbols('i,j,k', below_fermi=True, cls=Dummy)
        a, b, c = symbols('a,b,c', above_fermi=True, cls=Dummy)
        return (Rational(1, 36) * AntiSymmetricTensor('u', (a, b, c), (i, j, k))
                * NO(Fd(a) * Fd(b) * Fd(c) * F(k) * F(j) * F(i)))

    i, j, k = symbols('i,j,k', below_fermi=True)
    a, b, c = symbols('a,b,c', above_fermi=True)
    bra = NO(Fd(i) * Fd(j) * Fd(k) * F(c) * F(b) * F(a))
    C1 = Commutator(H, T2())
    term = [C1, Rational(1, 2) * Commutator(C1, T2()), Commutator(H, T3()), Commutator(C1, T3())][group]
    pretty = {'above': 'defg', 'below': 'lmno', 'general': 'pqrstu'}
    e = wicks(bra * term.doit(), simplify_kronecker_deltas=True, keep_only_fully_contracted=True)
    e = substitute_dummies(evaluate_deltas(e), new_indices=True, pretty_indices=pretty)
    return [str(x) for x in expand(e).args]


TENSOR = re.compile(r"AntiSymmetricTensor\((\w), \(([^)]*)\), \(([^)]*)\)\)")


def to_einsum(term: str):
    coef = 1.0
    s = term.strip()
    if s.startswith('-'):
        coef = -1.0; s = s[1:]
    m = re.match(r"^(\d+)\*", s)
    if m:
        coef *= float(m.group(1)); s = s[m.end():]
    m = re.search(r"/(\d+)$", s)
    if m:
        coef /= float(m.group(1)); s = s[:m.start()]
    ops, subs = [], []
    for name, up, lo in TENSOR.findall(s):
        up = [x.strip().lstrip('_') for x in up.split(',') if x.strip()]
        lo = [x.strip().lstrip('_') for x in lo.split(',') if x.strip()]
        if name == 'f':
            key, idx = 'f', up + lo
        elif name == 'v':
            key, idx = 'v', up + lo
        elif name == 't':
            key, idx = 't2', lo + up
        elif name == 'u':
            key, idx = 't3', lo + up
        else:
            raise ValueError(name)
        blk = ''.join('o' if x in 'ijklmno' else 'v' for x in idx)
        ops.append(f"{key}:{blk}")
        subs.append(''.join(idx))
    return coef, ','.join(subs) + '->ijkabc', ops


def main():
    out = ['"""Spin-orbital triples-projection terms (generated by oracle/derive_spinorb.py).',
           '',
           'Each entry is (coefficient, einsum subscripts, operands) of one Wick term of',
           '<T_ijk^abc| G |0> for the commutator group G named by the key; operands are',
           'f:<block> (Fock), v:<block> (<pq||rs>, creation indices first), t2:oovv and',
           't3:ooovvv amplitudes stored [occupied..., virtual...].',
           '"""', '', 'TERMS = {']
    names = ['H_T2', 'H_T2_T2', 'H_T3', 'H_T2_T3']
    for g, name in enumerate(names):
        out.append(f"    {name!r}: [")
        for t in derive(g):
            coef, spec, ops = to_einsum(t)
            out.append(f"        ({coef!r}, {spec!r}, {ops!r}),")
        out.append("    ],")
    out.append('}')
    sys.stdout.write('\n'.join(out) + '\n')


if __name__ == '__main__':
    main()
