"""Generates t3p_program.inc: the mixed-triples (T3') part of the residual as
a list of dense spatial-orbital contractions for the engine's einsum planner.

Run from the repository root (needs sympy):
    python -m paper_2501_10515_gb300.csrc.gen_t3p > paper_2501_10515_gb300/csrc/t3p_program.inc

What it computes (arXiv 2501.10515, Sec. II.B.1 and Sec. II.C).  A one-CSF
ASCC state carries, beside T1 and T2, the alpha-beta-beta triples with at
least three primary spin-orbital indices (h-up, h-down, p-up, p-down).  With
T1 absorbed into the orbital-dressed Hamiltonian H-hat (a general two-body
operator), the triples enter

    R1 += <S| [H,T3] |0>,   R2 += <D| [H,T3] |0>,
    R3  = <T| [H,T2] + 1/2 [[H,T2],T2] + [H,T3] + [[H,T2],T3] |0>,

and the partially linearised form drops the T2^M T2^M and T2^M T3' parts of
R3 (T3' is all mixed).  No other commutator reaches these projections.

Steps:
 1. Wick's theorem (sympy.physics.secondquant, a library step) gives the
    spin-orbital terms of each projection for a non-Hermitian two-body H.
 2. Every spin-orbital index is given a spin.  The output spins are fixed by
    the projection (singles alpha; doubles alpha-beta; triples
    alpha-beta-beta), summed indices take both; each factor becomes the
    spatial block of that spin case:
      f_pq            -> F[p][q] (same spin)
      <pq||rs>        -> (pr|qs) d(sp,sr) d(sq,ss) - (ps|qr) d(sp,ss) d(sq,sr)
      t_ij^ab         -> t2[i,j,a,b] (ab,ab), -t2[i,j,b,a] (ab,ba),
                         ts[i,j,a,b] = t2[i,j,a,b] - t2[j,i,a,b] (same spin)
      t_ijk^abc       -> +-t3[I,J,K,A,B,C], the index of the odd spin first
    (the spin-flip partner has the same spatial value).
 3. The slice t3 is stored as four dense blocks that partition it (the
    exact set of primary spin orbitals an element holds decides its block):
      TA[k][b][c] = t3[h,h,k,p,b,c]              (h-up h-dn p-up [+ p-dn])
      TB[k][a][c] = t3[h,h,k,a,p,c],  a != p     (h-up h-dn p-dn)
      TC[j][k][c] = t3[h,j,k,p,p,c],  j,k != h   (h-up p-up p-dn)
      TD[i][k][c] = t3[i,h,k,p,p,c],  i != h     (h-dn p-up p-dn)
    zero at k = h, c = p and the other excluded positions, so
      t3[I,J,K,A,B,C] = [I=h][J=h][A=p] TA[K,B,C] - [I=h][K=h][A=p] TA[J,B,C]
        + [I=h][J=h][B=p] TB[K,A,C] - [I=h][K=h][B=p] TB[J,A,C]
        - [I=h][J=h][C=p] TB[K,A,B] + [I=h][K=h][C=p] TB[J,A,B]
        + [I=h][A=p][B=p] TC[J,K,C] - [I=h][A=p][C=p] TC[J,K,B]
        + [J=h][A=p][B=p] TD[I,K,C] - [K=h][A=p][B=p] TD[I,J,C]
        - [J=h][A=p][C=p] TD[I,K,B] + [K=h][A=p][C=p] TD[I,J,B].
    The triples residual is produced in the same four blocks (RA..RD).  A
    Kronecker factor fixes the index it names: a summed index becomes the
    constant h or p, an output index restricts the term to that slice of
    the output (dropped where the block is not read).
 4. Terms are brought to a canonical form (index symmetries of t2, ts, the
    blocks and (pq|rs) = (rs|pq)) and merged.
 5. Integrals: a block with a fixed index, or with at most two virtual
    indices, is formed from the dressed density-fitting factor once per
    residual; (ov|vv)-type and (vv|vv) blocks stay factorised as
    sum_P B[P][.][.] B[P][.][.].  Each term is contracted pairwise in the
    order of fewest flops (sizes o = 20, v = 200, naux = 660), and equal
    intermediates are computed once.
 6. Contractions of a section that share a large operand (>= 10^6
    elements) with the same indices contracted are stacked into one product:
    their other operands are copied into the rows of a stack S (member by
    member), W = X . S^T is one GEMM, and each member's result is copied out
    of its columns of W (stacks capped at 6.4 10^7 elements of W).  The ops
    are re-ordered so that each stack's members are ready when it is formed.
 7. The op table (tensors with their kind, base operand, selector and
    dimensions; ops with section, kind, operands, einsum labels, weight and
    output selector) is written for the C++ executor (t3p.cu), which places
    the intermediates in one workspace by lifetime, plans the streams and
    runs each section with its t2 binding.
"""
from __future__ import annotations

import itertools
import sys
from fractions import Fraction

OCC, VIR = 'o', 'v'
EXTERNAL = {'I': 'i', 'J': 'j', 'K': 'k', 'A': 'a', 'B': 'b', 'C': 'c'}


# ----------------------------------------------------------------- 1. Wick terms
def wick_terms():
    from sympy import Add, Dummy, Rational, expand, symbols
    from sympy.physics.secondquant import (AntiSymmetricTensor, Commutator, F, Fd, NO,
                                           evaluate_deltas, substitute_dummies, wicks)

    def gen(cls_kw, names):
        return symbols(names, cls=Dummy, **cls_kw)

    p, q, r, s = symbols('p,q,r,s', cls=Dummy)
    H = (AntiSymmetricTensor('f', (p,), (q,)) * NO(Fd(p) * F(q))
         + Rational(1, 4) * AntiSymmetricTensor('v', (p, q), (r, s))
         * NO(Fd(p) * Fd(q) * F(s) * F(r)))

    def T2():
        i, j = gen({'below_fermi': True}, 'i,j')
        a, b = gen({'above_fermi': True}, 'a,b')
        return (Rational(1, 4) * AntiSymmetricTensor('t', (a, b), (i, j))
                * NO(Fd(a) * Fd(b) * F(j) * F(i)))

    def T3():
        i, j, k = gen({'below_fermi': True}, 'i,j,k')
        a, b, c = gen({'above_fermi': True}, 'a,b,c')
        return (Rational(1, 36) * AntiSymmetricTensor('u', (a, b, c), (i, j, k))
                * NO(Fd(a) * Fd(b) * Fd(c) * F(k) * F(j) * F(i)))

    I, J, K = symbols('I,J,K', below_fermi=True)
    A, B, C = symbols('A,B,C', above_fermi=True)
    bras = {1: NO(Fd(I) * F(A)), 2: NO(Fd(I) * Fd(J) * F(B) * F(A)),
            3: NO(Fd(I) * Fd(J) * Fd(K) * F(C) * F(B) * F(A))}
    HT2 = Commutator(H, T2())
    groups = {
        'R1_T3': (1, Commutator(H, T3())),
        'R2_T3': (2, Commutator(H, T3())),
        'R3_T2': (3, HT2),
        'R3_T2T2': (3, Rational(1, 2) * Commutator(HT2, T2())),
        'R3_T3': (3, Commutator(H, T3())),
        'R3_T2T3': (3, Commutator(HT2, T3())),
    }
    out = {}
    for name, (rank, op) in groups.items():
        e = wicks(bras[rank] * op.doit(), simplify_kronecker_deltas=True,
                  keep_only_fully_contracted=True)
        e = substitute_dummies(evaluate_deltas(e), new_indices=True)
        terms = []
        for term in Add.make_args(expand(e)) if e != 0 else []:
            coef = Fraction(1)
            factors = []
            rename = {}

            def lab(x):
                nm = str(x)
                if nm in EXTERNAL:
                    return EXTERNAL[nm]
                if nm not in rename:
                    sp = OCC if x.assumptions0.get('below_fermi') else VIR
                    rename[nm] = f"{sp}{len(rename)}"
                return rename[nm]

            for fac in term.as_ordered_factors():
                if isinstance(fac, AntiSymmetricTensor):
                    sym = str(fac.symbol)
                    up = [lab(x) for x in fac.upper]
                    lo = [lab(x) for x in fac.lower]
                    if sym == 'f':
                        factors.append(('f', (up[0], lo[0])))
                    elif sym == 'v':
                        factors.append(('v', (up[0], up[1], lo[0], lo[1])))
                    elif sym == 't':
                        factors.append(('t', (lo[0], lo[1], up[0], up[1])))
                    elif sym == 'u':
                        factors.append(('u', tuple(lo) + tuple(up)))
                    else:
                        raise ValueError(sym)
                else:
                    coef *= Fraction(str(fac))
            terms.append((coef, factors))
        out[name] = terms
    return out


def space(label):
    if label in ('i', 'j', 'k') or label.startswith(OCC):
        return OCC
    return VIR


# ---------------------------------------------------------------- 2. spin cases
ALPHA, BETA = 0, 1


def spin_factor(name, labs, sp):
    """Spatial blocks of one spin-orbital factor: [(coef, name, labels)]."""
    s = [sp[x] for x in labs]
    if name == 'f':
        return [(1, 'F', labs)] if s[0] == s[1] else []
    if name == 'v':
        p, q, r, t = labs
        out = []
        if s[0] == s[2] and s[1] == s[3]:
            out.append((1, 'g', (p, r, q, t)))
        if s[0] == s[3] and s[1] == s[2]:
            out.append((-1, 'g', (p, t, q, r)))
        return out
    if name == 't':
        i, j, a, b = labs
        if s[0] == s[1] == s[2] == s[3]:
            return [(1, 'ts', (i, j, a, b))]
        if s[0] != s[1] and s[0] == s[2] and s[1] == s[3]:
            return [(1, 't2', (i, j, a, b))]
        if s[0] != s[1] and s[0] == s[3] and s[1] == s[2]:
            return [(-1, 't2', (i, j, b, a))]
        return []
    if name == 'u':
        occ, vir = labs[:3], labs[3:]
        so, sv = s[:3], s[3:]
        na_o, na_v = so.count(ALPHA), sv.count(ALPHA)
        if na_o != na_v or na_o not in (1, 2):
            return []
        odd = ALPHA if na_o == 1 else BETA
        po, pv = so.index(odd), sv.index(odd)
        sign = (-1) ** (po + pv)
        oo = (occ[po],) + tuple(x for n_, x in enumerate(occ) if n_ != po)
        vv = (vir[pv],) + tuple(x for n_, x in enumerate(vir) if n_ != pv)
        return [(sign, 't3', oo + vv)]
    raise ValueError(name)


def t3_blocks(labs):
    """Block expansion of the spatial slice t3[I,J,K,A,B,C]: [(sign, block, labels, pins)]."""
    I, J, K, A, B, C = labs
    H, P = 'h', 'p'
    return [
        (+1, 'TA', (K, B, C), {I: H, J: H, A: P}),
        (-1, 'TA', (J, B, C), {I: H, K: H, A: P}),
        (+1, 'TB', (K, A, C), {I: H, J: H, B: P}),
        (-1, 'TB', (J, A, C), {I: H, K: H, B: P}),
        (-1, 'TB', (K, A, B), {I: H, J: H, C: P}),
        (+1, 'TB', (J, A, B), {I: H, K: H, C: P}),
        (+1, 'TC', (J, K, C), {I: H, A: P, B: P}),
        (-1, 'TC', (J, K, B), {I: H, A: P, C: P}),
        (+1, 'TD', (I, K, C), {J: H, A: P, B: P}),
        (-1, 'TD', (I, J, C), {K: H, A: P, B: P}),
        (-1, 'TD', (I, K, B), {J: H, A: P, C: P}),
        (+1, 'TD', (I, J, B), {K: H, A: P, C: P}),
    ]


# positions at which a block tensor vanishes when fixed to the primary index
BLOCK_ZERO = {'TA': (0,), 'TB': (0, 1, 2), 'TC': (0, 1, 2), 'TD': (0, 1, 2)}
# antisymmetric index pairs (a repeated fixed value there gives zero)
ANTISYM = {'TA': [(1, 2)], 'TC': [(0, 1)], 'ts': [(0, 1), (2, 3)]}

# outputs: name, labels, spins, fixed indices, output indices that may be fixed
OUTPUTS = {
    'R1_T3': [('r1', ('i', 'a'), {'i': ALPHA, 'a': ALPHA}, {}, {'i', 'a'})],
    'R2_T3': [('r2', ('i', 'j', 'a', 'b'),
               {'i': ALPHA, 'j': BETA, 'a': ALPHA, 'b': BETA}, {}, {'i', 'j', 'a', 'b'})],
}
_S3 = {'i': ALPHA, 'j': BETA, 'k': BETA, 'a': ALPHA, 'b': BETA, 'c': BETA}
R3_OUT = [
    ('RA', ('k', 'b', 'c'), _S3, {'i': 'h', 'j': 'h', 'a': 'p'}, {'b', 'c'}),
    ('RB', ('k', 'a', 'c'), _S3, {'i': 'h', 'j': 'h', 'b': 'p'}, set()),
    ('RC', ('j', 'k', 'c'), _S3, {'i': 'h', 'a': 'p', 'b': 'p'}, set()),
    ('RD', ('i', 'k', 'c'), _S3, {'j': 'h', 'a': 'p', 'b': 'p'}, set()),
]
for g in ('R3_T2', 'R3_T2T2', 'R3_T3', 'R3_T2T3'):
    OUTPUTS[g] = R3_OUT


def spin_expand(group, terms):
    """Spatial terms (coef, out_name, out_slots, factors) with fixed slots 'h'/'p'."""
    res = []
    for out_name, out_labs, out_spin, out_fix, may_fix in OUTPUTS[group]:
        for coef, factors in terms:
            labels = sorted({x for _, labs in factors for x in labs})
            summed = [x for x in labels if x not in out_spin]
            for spins in itertools.product((ALPHA, BETA), repeat=len(summed)):
                sp = dict(out_spin)
                sp.update(zip(summed, spins))
                choices = [spin_factor(nm, labs, sp) for nm, labs in factors]
                if any(not c for c in choices):
                    continue
                for combo in itertools.product(*choices):
                    # expand the t3 factors into blocks
                    parts = [[]]
                    for c_, nm, labs in combo:
                        if nm == 't3':
                            parts = [pp + [(c_ * s2, bl, bl_labs, pins)]
                                     for pp in parts for s2, bl, bl_labs, pins in t3_blocks(labs)]
                        else:
                            parts = [pp + [(c_, nm, labs, {})] for pp in parts]
                    for pp in parts:
                        t = fix_term(coef, pp, out_name, out_labs, out_fix, may_fix)
                        if t is not None:
                            res.append(t)
    return res


def fix_term(coef, parts, out_name, out_labs, out_fix, may_fix):
    fix = dict(out_fix)
    c = Fraction(coef)
    for c_, _, _, pins in parts:
        c *= c_
        for lab_, val in pins.items():
            if lab_ in fix:
                if fix[lab_] != val:
                    return None
                continue
            if lab_ in out_labs and lab_ not in may_fix:
                return None
            fix[lab_] = val
    if c == 0:
        return None
    factors = []
    for _, nm, labs, _ in parts:
        slots = tuple(fix.get(x, x) for x in labs)
        for pos in BLOCK_ZERO.get(nm, ()):
            if slots[pos] in ('h', 'p'):
                return None
        for a_, b_ in ANTISYM.get(nm, ()):
            if slots[a_] == slots[b_]:
                return None
        factors.append((nm, slots))
    out_slots = tuple(fix.get(x, x) for x in out_labs)
    # output block positions that are never read: RA's k = h
    if out_name == 'RA' and out_slots[0] == 'h':
        return None
    if out_name == 'RA' and out_slots[1] == out_slots[2] == 'p':
        return None
    return (c, out_name, out_slots, tuple(factors))


# ------------------------------------------------------------- 3. canonical form
SYMS = {
    't2': [((1, 0, 3, 2), 1)],
    'ts': [((1, 0, 2, 3), -1), ((0, 1, 3, 2), -1)],
    'g': [((2, 3, 0, 1), 1)],
    'TA': [((0, 2, 1), -1)],
    'TC': [((1, 0, 2), -1)],
}


def factor_variants(nm, slots):
    """All (sign, slots) equal to the factor under its index symmetries."""
    seen = {tuple(slots): 1}
    todo = [tuple(slots)]
    while todo:
        cur = todo.pop()
        for perm, sg in SYMS.get(nm, []):
            nxt = tuple(cur[q] for q in perm)
            s_ = seen[cur] * sg
            if nxt not in seen:
                seen[nxt] = s_
                todo.append(nxt)
    return [(s_, sl) for sl, s_ in seen.items()]


FIXED = ('h', 'p')


def canonical(term):
    """(sign, key) of a term; key is independent of summed-label names."""
    c, out_name, out_slots, factors = term
    outs = set(x for x in out_slots if x not in FIXED)
    best = None
    variants = [factor_variants(nm, sl) for nm, sl in factors]
    for order in itertools.permutations(range(len(factors))):
        for choice in itertools.product(*[variants[k] for k in order]):
            ren = {}
            sign = 1
            items = []
            for k, (s_, sl) in zip(order, choice):
                sign *= s_
                lab = []
                for x in sl:
                    if x in FIXED or x in outs:
                        lab.append(x)
                    else:
                        if x not in ren:
                            ren[x] = f"#{space(x)}{len(ren)}"
                        lab.append(ren[x])
                items.append((factors[k][0], tuple(lab)))
            key = (out_name, out_slots, tuple(items))
            if best is None or key < best[1]:
                best = (sign, key)
    return best


def merge(terms):
    acc = {}
    for t in terms:
        sign, key = canonical(t)
        acc[key] = acc.get(key, Fraction(0)) + sign * t[0]
    return [(c, k) for k, c in acc.items() if c != 0]


# ---------------------------------------------------------- 5. contraction plan
PLAN_SIZE = {'o': 20, 'v': 200, 'P': 660, '#': 1}
# base tensors: name -> spaces of their dimensions ('n': all orbitals, 'P': DF index)
BASE_DIMS = {'F': 'nn', 'B': 'Pnn', 't2': 'oovv', 'ts': 'oovv', 'TA': 'ovv', 'TB': 'ovv',
             'TC': 'oov', 'TD': 'oov', 'r1': 'ov', 'r2': 'oovv', 'RA': 'ovv', 'RB': 'ovv',
             'RC': 'oov', 'RD': 'oov'}
T2_BASES = ('t2', 'ts')
# integral blocks up to this size at the planning sizes are formed once per
# residual; larger ones ((vv|vv)) stay factorised through the DF index
MAX_G_ELEMENTS = 2.0e8
GROUPS = ('R1_T3', 'R2_T3', 'R3_T2', 'R3_T2T2', 'R3_T3', 'R3_T2T3')
# which amplitudes the t2 / ts operands of a group are bound to at run time
GROUP_SECTION = {'R1_T3': 'pro', 'R2_T3': 'pro', 'R3_T3': 'pro', 'R3_T2': 'lin',
                 'R3_T2T2': 'quad', 'R3_T2T3': 'mix'}


def lab_space(x):
    if x.startswith('P'):
        return 'P'
    if x in ('i', 'j', 'k') or x.startswith('#o') or x.startswith(OCC):
        return OCC
    return VIR


def size_of(labels):
    r = 1.0
    for x in labels:
        r *= PLAN_SIZE[lab_space(x)]
    return r


def leaf_spec(nm, slots):
    """Per-dimension selector of a base tensor: 'h', 'p', or the space of the label."""
    out = []
    for d, x in zip(BASE_DIMS[nm], slots):
        if x in FIXED:
            out.append(x)
        else:
            sp = lab_space(x)
            assert d in ('n', sp), (nm, slots)
            out.append(sp)
    return ''.join(out)


def leaves_of(items):
    """Leaf operands of a term; an integral is a formed block ('g') or two DF factors."""
    out = []
    for k, (nm, slots) in enumerate(items):
        if nm == 'g':
            free = [x for x in slots if x not in FIXED]
            if size_of(free) <= MAX_G_ELEMENTS:
                out.append(('g', slots))
            else:
                P = f"P{k}"
                out.append(('B', (P,) + tuple(slots[:2])))
                out.append(('B', (P,) + tuple(slots[2:])))
        else:
            out.append((nm, tuple(slots)))
    return out


def node_canonical(leaves, externals):
    """Canonical (sign, key, ext_order) of a product of leaves with the given
    external labels: summed labels renamed '#..', external ones '@..' by first
    appearance; ext_order lists the external labels in '@' order."""
    best = None
    variants = [factor_variants(nm, sl) if nm != 'B' else [(1, sl)] for nm, sl in leaves]
    order0 = sorted(range(len(leaves)), key=lambda k: leaves[k][0])
    names = [leaves[k][0] for k in order0]
    # only orders that keep the leaves sorted by tensor name
    perms = set()
    for perm in itertools.permutations(order0):
        if [leaves[k][0] for k in perm] == names:
            perms.add(perm)
    for perm in perms:
        for choice in itertools.product(*[variants[k] for k in perm]):
            ren, ext = {}, []
            sign = 1
            items = []
            for k, (s_, sl) in zip(perm, choice):
                sign *= s_
                lab = []
                for x in sl:
                    if x in FIXED:
                        lab.append(x)
                        continue
                    if x not in ren:
                        if x in externals:
                            ren[x] = f"@{lab_space(x)}{len(ext)}"
                            ext.append(x)
                        else:
                            ren[x] = f"#{lab_space(x)}{len(ren) - len(ext)}"
                    lab.append(ren[x])
                items.append((leaves[k][0], tuple(lab)))
            key = tuple(items)
            if best is None or key < best[1]:
                best = (sign, key, tuple(ext))
    return best


class Program:
    def __init__(self):
        self.tensors = []     # dict(kind, dims, section, ...)
        self.index = {}
        self.ops = {s: [] for s in ('pro', 'lin', 'quad', 'mix')}
        self.flops = {s: 0.0 for s in self.ops}
        self.counts = {}

    def _new(self, key, info, section, op):
        if key in self.index:
            return self.index[key], False
        tid = len(self.tensors)
        info = dict(info)
        info['section'] = section
        self.tensors.append(info)
        self.index[key] = tid
        if op is not None:
            op = dict(op)
            op['out'] = tid
            self.ops[section].append(op)
        return tid, True

    def leaf(self, nm, slots, section):
        """(tensor id, labels in its dimension order)."""
        if nm == 'g':
            return self.gblock(slots)
        sec = section if nm in T2_BASES else 'pro'
        spec = leaf_spec(nm, slots)
        labels = [x for x in slots if x not in FIXED]
        if all(c in ('o', 'v', 'P') for c in spec) and (
                BASE_DIMS[nm] == spec):
            tid, _ = self._new(('base', nm, sec), {'kind': 'base', 'base': nm, 'dims': spec},
                               sec, None)
            return tid, labels
        dims = ''.join(c for c in spec if c not in FIXED)
        tid, _ = self._new(('slice', nm, spec, sec),
                           {'kind': 'slice', 'base': nm, 'spec': spec, 'dims': dims}, sec,
                           {'kind': 'slice', 'base': nm, 'spec': spec})
        return tid, labels

    def gblock(self, slots):
        # (wx|yz) = (yz|wx): the block is formed once, with the smaller
        # selector string first
        slots = tuple(slots)
        sw = slots[2:] + slots[:2]
        spec_of = lambda sl: ''.join(x if x in FIXED else lab_space(x) for x in sl)
        if spec_of(sw) < spec_of(slots):
            slots = sw
        spec = spec_of(slots)
        free = [x for x in slots if x not in FIXED]
        key = ('gblk', spec)
        if key in self.index:
            return self.index[key], free
        a, la = self.leaf('B', ('Pq',) + tuple(slots[:2]), 'pro')
        b, lb = self.leaf('B', ('Pq',) + tuple(slots[2:]), 'pro')
        dims = ''.join(lab_space(x) for x in free)
        self.flops['pro'] += 2 * size_of(set(la) | set(lb))
        tid, _ = self._new(key, {'kind': 'inter', 'dims': dims}, 'pro',
                           {'kind': 'ctr', 'a': a, 'b': b, 'spec': letters(la, lb, free),
                            'alpha': 1.0})
        return tid, free

    def node(self, leaves, externals, section, sub):
        """Tensor id, labels (dimension order) and sign of a product of leaves.
        sub: (node_a, node_b) leaf subsets of the chosen pairwise split."""
        if len(leaves) == 1:
            nm, slots = leaves[0]
            tid, labels = self.leaf(nm, slots, section)
            return tid, labels, 1
        sec = section if any(nm in T2_BASES for nm, _ in leaves) else 'pro'
        sign, key, ext = node_canonical(leaves, externals)
        full = ('node', key, sec)
        if full in self.index:
            return self.index[full], list(ext), sign
        (la_leaves, la_ext, la_sub), (lb_leaves, lb_ext, lb_sub) = sub
        a, la, sa = self.node(la_leaves, la_ext, section, la_sub)
        b, lb, sb = self.node(lb_leaves, lb_ext, section, lb_sub)
        dims = ''.join(lab_space(x) for x in ext)
        self.flops[sec] += 2 * size_of(set(la) | set(lb))
        tid, _ = self._new(full, {'kind': 'inter', 'dims': dims}, sec,
                           {'kind': 'ctr', 'a': a, 'b': b, 'spec': letters(la, lb, list(ext)),
                            'alpha': float(sa * sb * sign)})
        return tid, list(ext), sign

    def term(self, coef, key, group):
        out_name, out_slots, items = key
        section = GROUP_SECTION[group]
        leaves = leaves_of(items)
        outl = [x for x in out_slots if x not in FIXED]
        best = plan_pairs(leaves, outl)
        (a_sub, b_sub) = best
        a, la, sa = self.node(a_sub[0], a_sub[1], section, a_sub[2])
        b, lb, sb = self.node(b_sub[0], b_sub[1], section, b_sub[2])
        out_spec = leaf_spec(out_name, out_slots)
        sec = section
        self.flops[sec] += 2 * size_of(set(la) | set(lb))
        self.ops[sec].append({'kind': 'acc', 'a': a, 'b': b, 'spec': letters(la, lb, outl),
                              'alpha': float(coef) * sa * sb, 'outbase': out_name,
                              'outspec': out_spec})


def plan_pairs(leaves, outl):
    """Best pairwise contraction tree (fewest flops at the planning sizes) as
    nested (leaves, externals, sub) for the two children of the root."""
    memo = {}

    def ext_of(subset):
        inside = set(x for k in subset for x in leaves[k][1] if x not in FIXED)
        outside = set(outl)
        for k in range(len(leaves)):
            if k not in subset:
                outside |= set(x for x in leaves[k][1] if x not in FIXED)
        return [x for x in dict.fromkeys(x for k in sorted(subset) for x in leaves[k][1])
                if x not in FIXED and x in outside and x in inside]

    def best(subset):
        subset = tuple(sorted(subset))
        if subset in memo:
            return memo[subset]
        if len(subset) == 1:
            memo[subset] = (0.0, None)
            return memo[subset]
        res = None
        items = list(subset)
        for r in range(1, len(items)):
            for left in itertools.combinations(items, r):
                if items[0] not in left:
                    continue
                right = tuple(x for x in items if x not in left)
                la, lb = ext_of(left), ext_of(right)
                c = best(left)[0] + best(right)[0] + 2 * size_of(set(la) | set(lb))
                if res is None or c < res[0]:
                    res = (c, (left, right))
        memo[subset] = res
        return res

    def build(subset):
        subset = tuple(sorted(subset))
        lv = [leaves[k] for k in subset]
        ext = ext_of(subset)
        if len(subset) == 1:
            return (lv, ext, None)
        left, right = best(subset)[1]
        return (lv, ext, (build(left), build(right)))

    root = tuple(range(len(leaves)))
    if len(leaves) == 1:
        raise ValueError("single-factor term")
    left, right = best(root)[1]
    return (build(left), build(right))


def letters(*label_lists):
    """einsum spec with one letter per label: 'abc,cd->abd'."""
    m = {}
    for ll in label_lists:
        for x in ll:
            if x not in m:
                m[x] = 'abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ'[len(m)]
    parts = [''.join(m[x] for x in ll) for ll in label_lists]
    return ','.join(parts[:-1]) + '->' + parts[-1]


def build_program(w):
    prog = Program()
    for g in GROUPS:
        for c, key in sorted(merge(spin_expand(g, w[g])), key=lambda t: repr(t[1])):
            prog.term(c, key, g)
    return prog


SECTIONS = ('pro', 'lin', 'quad', 'mix')
BASES = ('F', 'B', 't2', 'ts', 'TA', 'TB', 'TC', 'TD', 'r1', 'r2', 'RA', 'RB', 'RC', 'RD')

# ------------------------------------------------ 6. shared-operand stacking
# Contractions that read the same large operand X with the same indices of X
# contracted (an integral block, t2, a DF slice against many small operands)
# are run as one: the small operands Y_i are stacked as rows of S[#][K],
# W[F][#] = X . S^T is one GEMM, and each result is copied (or accumulated)
# out of its columns of W.  X is then prepared and read once per group.
FUSE_MIN = 1.0e6   # elements of X at the planning sizes
FUSE_MAX_W = 6.4e7  # elements of a stacked product W (and of S) at the planning sizes


def dims_size(dims):
    r = 1.0
    for c in dims:
        r *= PLAN_SIZE[c]
    return r


def fuse_candidate(prog, op):
    """((X, roles), (lx, Y, ly)) for a contraction that may share operand X."""
    if op['kind'] not in ('ctr', 'acc'):
        return None
    lhs, c = op['spec'].split('->')
    la, lb = lhs.split(',')
    if any(x in la and x in lb for x in c):
        return None
    best = None
    for X, lx, Y, ly in ((op['a'], la, op['b'], lb), (op['b'], lb, op['a'], la)):
        dims = prog.tensors[X]['dims']
        if '#' in dims or dims_size(dims) < FUSE_MIN or len(ly) == 0:
            continue
        roles = tuple('K' if (x in ly and x not in c) else 'F' for x in lx)
        if 'K' not in roles:
            continue
        size = dims_size(dims)
        if best is None or size > best[2]:
            best = ((X, roles), (lx, Y, ly), size)
    return None if best is None else best[:2]


def fuse_shared_operands(prog):
    for sec in SECTIONS:
        ops = prog.ops[sec]
        producer = {}
        for i, op in enumerate(ops):
            if op['kind'] in ('slice', 'ctr'):
                producer[op['out']] = i
        deps = []
        for op in ops:
            d = set()
            for t in (op.get('a'), op.get('b')):
                if t is not None and t in producer:
                    d.add(producer[t])
            deps.append(d)
        cand = [fuse_candidate(prog, op) for op in ops]
        count = {}
        for cnd in cand:
            if cnd is not None:
                count[cnd[0]] = count.get(cnd[0], 0) + 1
        emitted, out, remaining = set(), [], list(range(len(ops)))
        while remaining:
            ready = [i for i in remaining if deps[i] <= emitted]
            plain = [i for i in ready if cand[i] is None or count[cand[i][0]] < 2]
            if plain:
                take = plain
                out.extend(ops[i] for i in take)
            else:
                by = {}
                for i in ready:
                    by.setdefault(cand[i][0], []).append(i)
                key, take = max(by.items(), key=lambda kv: (len(kv[1]), -kv[1][0]))
                for chunk in size_chunks(prog, key, [(ops[i], cand[i][1]) for i in take]):
                    if len(chunk) == 1:
                        out.append(chunk[0][0])
                    else:
                        out.extend(stacked_ops(prog, sec, key, chunk))
            emitted.update(take)
            tk = set(take)
            remaining = [i for i in remaining if i not in tk]
        prog.ops[sec] = out


def size_chunks(prog, key, members):
    """Members in order, cut so that no stack product W or stack S exceeds FUSE_MAX_W."""
    X, roles = key
    xdims = prog.tensors[X]['dims']
    f = dims_size(''.join(d for d, r in zip(xdims, roles) if r == 'F'))
    kk = dims_size(''.join(d for d, r in zip(xdims, roles) if r == 'K'))
    chunks, cur, rows = [], [], 0.0
    for op, (lx, Y, ly) in members:
        c = op['spec'].split('->')[1]
        ydims = prog.tensors[Y]['dims']
        n = dims_size(''.join(ydims[ly.index(x)] for x in c if x in ly))
        if cur and max(f, kk) * (rows + n) > FUSE_MAX_W:
            chunks.append(cur)
            cur, rows = [], 0.0
        cur.append((op, (lx, Y, ly)))
        rows += n
    if cur:
        chunks.append(cur)
    return chunks


def stacked_ops(prog, sec, key, members):
    X, roles = key
    xdims = prog.tensors[X]['dims']
    kdims = ''.join(d for d, r in zip(xdims, roles) if r == 'K')
    fdims = ''.join(d for d, r in zip(xdims, roles) if r == 'F')
    rows, stacks, unstacks = [], [], []
    for m, (op, (lx, Y, ly)) in enumerate(members):
        c = op['spec'].split('->')[1]
        kl = ''.join(x for x, r in zip(lx, roles) if r == 'K')
        fl = ''.join(x for x, r in zip(lx, roles) if r == 'F')
        gl = ''.join(x for x in c if x in ly)
        ydims = prog.tensors[Y]['dims']
        rows.append(''.join(ydims[ly.index(x)] for x in gl))
        stacks.append({'kind': 'stack', 'a': Y, 'spec': f"{ly}->{gl}{kl}", 'member': m})
        u = {'kind': 'unstack', 'spec': f"{fl}{gl}->{c}", 'alpha': op['alpha'], 'member': m}
        if op['kind'] == 'ctr':
            u['out'] = op['out']
        else:
            u['outbase'], u['outspec'] = op['outbase'], op['outspec']
        unstacks.append(u)
    rs = '+'.join(rows)
    S = len(prog.tensors)
    prog.tensors.append({'kind': 'inter', 'dims': '#' + kdims, 'rows': rs, 'section': sec})
    W = len(prog.tensors)
    prog.tensors.append({'kind': 'inter', 'dims': fdims + '#', 'rows': rs, 'section': sec})
    for st in stacks:
        st['out'] = S
    for u in unstacks:
        u['a'] = W
    lx = ''.join('abcdefghijklmnopqrstuvwxy'[q] for q in range(len(xdims)))
    klet = ''.join(x for x, r in zip(lx, roles) if r == 'K')
    flet = ''.join(x for x, r in zip(lx, roles) if r == 'F')
    ctr = {'kind': 'ctr', 'a': X, 'b': S, 'out': W, 'spec': f"{lx},Z{klet}->{flet}Z", 'alpha': 1.0}
    return stacks + [ctr] + unstacks


def emit(prog, out):
    """Writes the program as C++ tables (included by t3p.cu)."""
    w = out.write
    w("// Generated by gen_t3p.py from the spin-orbital triples equations; do not edit.\n")
    w("// Tensors: kind 0 = base operand, 1 = slice of a base operand, 2 = intermediate;\n")
    w("// dims use o (occupied), v (virtual), P (density-fitting index) and # (the rows of\n")
    w("// a stack: the sum over its members of the products of the '+'-separated dims);\n")
    w("// a slice selector has one character per base dimension: o / v / P (range),\n")
    w("// h / p (fixed).  Ops: kind 0 = slice, 1 = contraction into an intermediate,\n")
    w("// 2 = contraction accumulated into an output block (selector outspec),\n")
    w("// 3 = copy of a member operand into its rows of a stack, 4 = copy of a\n")
    w("// member's columns of a stacked product into its intermediate or output.\n")
    w(f"static const int kT3pTensorCount = {len(prog.tensors)};\n")
    w("static const T3pTensor kT3pTensors[] = {\n")
    for t in prog.tensors:
        kind = {'base': 0, 'slice': 1, 'inter': 2}[t['kind']]
        base = BASES.index(t['base']) if 'base' in t else -1
        w(f'    {{{kind}, {base}, "{t.get("spec", "")}", "{t["dims"]}", '
          f'{SECTIONS.index(t["section"])}, "{t.get("rows", "")}"}},\n')
    w("};\n")
    n = sum(len(v) for v in prog.ops.values())
    w(f"static const int kT3pOpCount = {n};\n")
    w("static const T3pOp kT3pOps[] = {\n")
    for sec in SECTIONS:
        sid = SECTIONS.index(sec)
        for op in prog.ops[sec]:
            k = op['kind']
            if k == 'slice':
                w(f'    {{{sid}, 0, {op["out"]}, -1, -1, "{op["spec"]}", 1.0, '
                  f'{BASES.index(op["base"])}, "", -1}},\n')
            elif k == 'ctr':
                w(f'    {{{sid}, 1, {op["out"]}, {op["a"]}, {op["b"]}, '
                  f'"{op["spec"]}", {op["alpha"]!r}, -1, "", -1}},\n')
            elif k == 'acc':
                w(f'    {{{sid}, 2, -1, {op["a"]}, {op["b"]}, "{op["spec"]}", '
                  f'{op["alpha"]!r}, {BASES.index(op["outbase"])}, "{op["outspec"]}", -1}},\n')
            elif k == 'stack':
                w(f'    {{{sid}, 3, {op["out"]}, {op["a"]}, -1, "{op["spec"]}", 1.0, -1, "", '
                  f'{op["member"]}}},\n')
            else:
                ob = BASES.index(op['outbase']) if 'outbase' in op else -1
                w(f'    {{{sid}, 4, {op.get("out", -1)}, {op["a"]}, -1, "{op["spec"]}", '
                  f'{op["alpha"]!r}, {ob}, "{op.get("outspec", "")}", {op["member"]}}},\n')
    w("};\n")


def main():
    import os
    import pickle
    cache = os.environ.get('T3P_WICK_CACHE')
    w = pickle.load(open(cache, 'rb')) if cache and os.path.exists(cache) else wick_terms()
    prog = build_program(w)
    fuse_shared_operands(prog)
    for s in SECTIONS:
        print(s, len(prog.ops[s]), f"{prog.flops[s]:.3e} flops at o=20 v=200 (before stacking)",
              file=sys.stderr)
    emit(prog, sys.stdout)


if __name__ == '__main__':
    main()
