"""O-SL: the T3' terms of the residual on the slice itself (test infrastructure).

The same projections as spinorb.residual's triples part -- R1 and R2 from
[H,T3'], and R3' from [H,T2] + 1/2[[H,T2],T2] + [H,T3'] + [[H,T2],T3'] with
the partial linearisation of Sec. II.C -- for H-hat = exp(-T1) H-bar exp(T1),
but evaluated without spin-orbital tensors, so that it reaches o = 20,
v = 200:

* the spin-orbital Wick terms are the oracle's own (so_triples_terms for R3',
  the five [H,T3] terms of spinorb.residual for R1 and R2);
* each spin-orbital index is given a spin (output indices: singles alpha,
  doubles alpha-beta, triples alpha-beta-beta; summed indices: both), and
  every factor is replaced by its spatial block for that spin case:
    f_pq             F[p,q] if the spins agree
    <pq||rs>         (pr|qs) [sp=sr][sq=ss] - (ps|qr) [sp=ss][sq=sr]
    t_ij^ab          t2[i,j,a,b] (spins a b a b), -t2[i,j,b,a] (a b b a), and
                     t2[i,j,a,b] - t2[j,i,a,b] for equal spins (Eq. S1)
    t_ijk^abc        +- t3[I,J,K,A,B,C]: the occupied and the virtual index of
                     the odd spin moved to the front, one sign per swap (the
                     spin-flipped triple has the same value);
* t3 lives only on the slice (Sec. II.B.1), so t3[I,J,K,A,B,C] is read from
  four dense blocks that partition it by the primary spin orbitals an element
  holds,
    XA[k,b,c] = t3[h,h,k,p,b,c]            XB[k,a,c] = t3[h,h,k,a,p,c], a != p
    XC[j,k,c] = t3[h,j,k,p,p,c], j,k != h  XD[i,k,c] = t3[i,h,k,p,p,c], i != h
  (zero elsewhere): each placement of h into the I or the J/K slots and of p
  into the A or the B/C slots that one of the blocks covers fixes those
  indices (function slice_value below lists them);
* R3' is produced in the same four blocks (output indices fixed likewise) and
  gathered at the slice positions.

The integral blocks are those of spinadapted.Blocks, (pq|rs) = sum_P
B[P,p,q] B[P,r,s] of the dressed DF factor, formed once per residual.

Pinned to spinorb.residual (itself pinned to the brute-force projections) in
tests/test_oracle_pins.py.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import amplitudes as amp
from .so_triples_terms import TERMS

ALPHA, BETA = 'a', 'b'

# [H,T3] on singles and doubles (spinorb.residual): (coef, subscripts, operand keys)
R1_T3 = [(0.25, 'ilmade,lmde->ia', ['t3:ooovvv', 'v:oovv'])]
R2_T3 = [(1.0, 'ld,ijlabd->ijab', ['f:ov', 't3:ooovvv']),
         (0.5, 'jlmabd,lmid->ijab', ['t3:ooovvv', 'v:ooov']),
         (-0.5, 'ilmabd,lmjd->ijab', ['t3:ooovvv', 'v:ooov']),
         (0.5, 'ijlade,blde->ijab', ['t3:ooovvv', 'v:vovv']),
         (-0.5, 'ijlbde,alde->ijab', ['t3:ooovvv', 'v:vovv'])]


class Operands:
    """Spatial arrays of one residual evaluation: the Fock matrix, the integral
    blocks (pq|rs) of spinadapted.Blocks (formed once and cached there) and the
    slice blocks."""

    def __init__(self, blk, hole, part, t3_blocks):
        self.blk, self.F, self.o = blk, blk.F, blk.o
        self.h, self.p = hole, part
        self.n = blk.F.shape[0]
        self.X = t3_blocks   # dict XA..XD

    def index(self, space, fixed):
        """Index into an all-orbital dimension: a range or the fixed primary."""
        if fixed == 'h':
            return self.h
        if fixed == 'p':
            return self.o + self.p
        return slice(0, self.o) if space == 'o' else slice(self.o, self.n)

    def block_index(self, space, fixed):
        """Index into an occupied or virtual block dimension."""
        if fixed == 'h':
            return self.h
        if fixed == 'p':
            return self.p
        return slice(None)


def slice_value(I, J, K, A, B, C):
    """t3[I,J,K,A,B,C] on the slice as (sign, block, block labels, fixed labels)."""
    return [(+1, 'XA', (K, B, C), {I: 'h', J: 'h', A: 'p'}),
            (-1, 'XA', (J, B, C), {I: 'h', K: 'h', A: 'p'}),
            (+1, 'XB', (K, A, C), {I: 'h', J: 'h', B: 'p'}),
            (-1, 'XB', (J, A, C), {I: 'h', K: 'h', B: 'p'}),
            (-1, 'XB', (K, A, B), {I: 'h', J: 'h', C: 'p'}),
            (+1, 'XB', (J, A, B), {I: 'h', K: 'h', C: 'p'}),
            (+1, 'XC', (J, K, C), {I: 'h', A: 'p', B: 'p'}),
            (-1, 'XC', (J, K, B), {I: 'h', A: 'p', C: 'p'}),
            (+1, 'XD', (I, K, C), {J: 'h', A: 'p', B: 'p'}),
            (-1, 'XD', (I, J, C), {K: 'h', A: 'p', B: 'p'}),
            (-1, 'XD', (I, K, B), {J: 'h', A: 'p', C: 'p'}),
            (+1, 'XD', (I, J, B), {K: 'h', A: 'p', C: 'p'})]


def spin_blocks(kind, labels, spin):
    """[(coef, tensor, labels)] of one spin-orbital factor for given spins."""
    s = [spin[x] for x in labels]
    if kind == 'f':
        return [(1.0, 'F', labels)] if s[0] == s[1] else []
    if kind == 'v':
        p, q, r, t = labels
        out = []
        if s[0] == s[2] and s[1] == s[3]:
            out.append((1.0, 'g', (p, r, q, t)))
        if s[0] == s[3] and s[1] == s[2]:
            out.append((-1.0, 'g', (p, t, q, r)))
        return out
    if kind == 't2':
        i, j, a, b = labels
        if s[0] == s[1] == s[2] == s[3]:
            return [(1.0, 't2', (i, j, a, b)), (-1.0, 't2', (j, i, a, b))]
        if s[0] != s[1] and (s[0], s[1]) == (s[2], s[3]):
            return [(1.0, 't2', (i, j, a, b))]
        if s[0] != s[1] and (s[0], s[1]) == (s[3], s[2]):
            return [(-1.0, 't2', (i, j, b, a))]
        return []
    if kind == 't3':
        occ, vir = list(labels[:3]), list(labels[3:])
        so, sv = s[:3], s[3:]
        if sorted(so) != sorted(sv) or len(set(so)) == 1:
            return []
        odd = ALPHA if so.count(ALPHA) == 1 else BETA
        io, iv = so.index(odd), sv.index(odd)
        sign = (-1.0) ** (io + iv)
        occ = [occ[io]] + occ[:io] + occ[io + 1:]
        vir = [vir[iv]] + vir[:iv] + vir[iv + 1:]
        return [(sign, 't3', tuple(occ + vir))]
    raise ValueError(kind)


BLOCK_SPACES = {'XA': 'ovv', 'XB': 'ovv', 'XC': 'oov', 'XD': 'oov'}


def evaluate(term_list, outputs, ops, t2, acc, scale=1.0):
    """Adds every spin case of every term of term_list to the output arrays in acc.

    outputs: [(name, labels, spins, fixed)] -- fixed output indices of a block.
    """
    for out_name, out_labels, out_spin, out_fixed in outputs:
        for coef, subs, keys in term_list:
            lhs, _ = subs.split('->')
            facs = [(k.split(':')[0], tuple(sub)) for k, sub in zip(keys, lhs.split(','))]
            summed = sorted({x for _, ls in facs for x in ls} - set(out_spin))
            for spins in itertools.product((ALPHA, BETA), repeat=len(summed)):
                spin = dict(out_spin)
                spin.update(zip(summed, spins))
                expansions = [spin_blocks(kind, ls, spin) for kind, ls in facs]
                for combo in itertools.product(*expansions):
                    c = coef * np.prod([x[0] for x in combo])
                    _add_product(c * scale, combo, out_name, out_labels, out_fixed, ops, t2, acc)


def _add_product(c, combo, out_name, out_labels, out_fixed, ops, t2, acc):
    """One spin case: read the t3 factor from the slice blocks and contract."""
    t3_at = [k for k, x in enumerate(combo) if x[1] == 't3']
    placements = [slice_value(*combo[k][2]) for k in t3_at]
    for sel in itertools.product(*placements):
        fixed = dict(out_fixed)
        sign = 1.0
        ok = True
        for s_, blk, bl, fx in sel:
            sign *= s_
            for lab, val in fx.items():
                ok = ok and fixed.get(lab, val) == val
                fixed[lab] = val
        if not ok:
            continue
        factors = []
        placed = iter(sel)
        for cf, name, ls in combo:
            if name == 't3':
                _, blk, bl, _ = next(placed)
                factors.append((blk, bl))
            else:
                factors.append((name, ls))
        _contract(c * sign, factors, fixed, out_name, out_labels, ops, t2, acc)


def _space(lab):
    return 'o' if lab in 'ijklmno' else 'v'


def _contract(c, factors, fixed, out_name, out_labels, ops, t2, acc):
    arrays, subs = [], []
    letters = {}

    def L(x):
        if x not in letters:
            letters[x] = 'ABCDEFGHIJKLMNOPQRSTUVWXYZ'[len(letters)]
        return letters[x]

    for name, ls in factors:
        if name == 'F':
            idx = tuple(ops.index(_space(x), fixed.get(x)) for x in ls)
            arrays.append(ops.F[idx])
            subs.append(''.join(L(x) for x in ls if x not in fixed))
            continue
        if name == 'g':
            # (pq|rs) block of the spaces of the four labels, fixed ones sliced
            g = ops.blk.g(''.join(_space(x) for x in ls))
            idx = tuple(ops.block_index(_space(x), fixed.get(x)) for x in ls)
            arrays.append(g[idx])
            subs.append(''.join(L(x) for x in ls if x not in fixed))
            continue
        if name == 't2':
            arr = t2
            spaces = 'oovv'
        else:
            arr = ops.X[name]
            spaces = BLOCK_SPACES[name]
        idx = []
        for x, sp in zip(ls, spaces):
            if x in fixed:
                idx.append(ops.h if fixed[x] == 'h' else ops.p)
            else:
                idx.append(slice(None))
        arrays.append(arr[tuple(idx)])
        subs.append(''.join(L(x) for x in ls if x not in fixed))
    free_out = [x for x in out_labels if x not in fixed]
    val = np.einsum(','.join(subs) + '->' + ''.join(L(x) for x in free_out), *arrays,
                    optimize=True)
    dst = acc[out_name]
    sel = tuple((ops.h if fixed[x] == 'h' else ops.p) if x in fixed else slice(None)
                for x in out_labels)
    dst[sel] += c * val


def blocks_from_slice(idx, vals, o, v, hole, part):
    """The four dense blocks XA..XD of the slice (zero outside their part)."""
    h, p = hole, part
    X = {'XA': np.zeros((o, v, v)), 'XB': np.zeros((o, v, v)),
         'XC': np.zeros((o, o, v)), 'XD': np.zeros((o, o, v))}
    for (i, j, k, a, b, c), x in zip(idx, vals):
        reg, key, partner = _locate(i, j, k, a, b, c, h, p)
        s, blk = reg
        X[blk][key] = s * x
        if partner is not None:
            X[blk][partner] = -s * x
    return X


def _locate(i, j, k, a, b, c, h, p):
    """Block, position and antisymmetric partner position of slice element (i,j<k,a,b<c)."""
    s = 1.0
    if i == h and h in (j, k):
        if j != h:
            j, k, s = k, j, -s
        if a == p:
            return (s, 'XA'), (k, b, c), (k, c, b)
        if b != p:
            b, c, s = c, b, -s
        return (s, 'XB'), (k, a, c), None
    if i == h:
        if b != p:
            b, c, s = c, b, -s
        return (s, 'XC'), (j, k, c), (k, j, c)
    if j != h:
        j, k, s = k, j, -s
    if b != p:
        b, c, s = c, b, -s
    return (s, 'XD'), (i, k, c), None


def gather(idx, R, o, v, hole, part):
    """Residual values at the slice positions from the blocks RA..RD."""
    out = np.zeros(len(idx))
    for q, (i, j, k, a, b, c) in enumerate(idx):
        (s, blk), key, _ = _locate(i, j, k, a, b, c, hole, part)
        out[q] = s * R['R' + blk[1]][key]
    return out


def residual(blk, t2, t3_idx, t3_vals, hole, part, linearize=False):
    """T3' contributions (R1, R2) and R3' at the slice positions.

    blk: the blocks of H-hat = exp(-T1) H-bar exp(T1) (spinadapted.Blocks:
    Fock matrix and cached (pq|rs) blocks); t2 spin-adapted doubles;
    (t3_idx, t3_vals) the slice.  linearize=True drops T2^M T2^M and
    T2^M T3' from R3'.
    """
    o, v = blk.o, t2.shape[2]
    X = blocks_from_slice(t3_idx, t3_vals, o, v, hole, part)
    ops = Operands(blk, hole, part, X)
    acc = {'r1': np.zeros((o, v)), 'r2': np.zeros((o, o, v, v)),
           'RA': np.zeros((o, v, v)), 'RB': np.zeros((o, v, v)),
           'RC': np.zeros((o, o, v)), 'RD': np.zeros((o, o, v))}
    s1 = {'i': ALPHA, 'a': ALPHA}
    s2 = {'i': ALPHA, 'j': BETA, 'a': ALPHA, 'b': BETA}
    s3 = {'i': ALPHA, 'j': BETA, 'k': BETA, 'a': ALPHA, 'b': BETA, 'c': BETA}
    lab3 = ('i', 'j', 'k', 'a', 'b', 'c')
    blocks3 = [('RA', lab3, s3, {'i': 'h', 'j': 'h', 'a': 'p'}),
               ('RB', lab3, s3, {'i': 'h', 'j': 'h', 'b': 'p'}),
               ('RC', lab3, s3, {'i': 'h', 'a': 'p', 'b': 'p'}),
               ('RD', lab3, s3, {'j': 'h', 'a': 'p', 'b': 'p'})]
    evaluate(R1_T3, [('r1', ('i', 'a'), s1, {})], ops, t2, acc)
    evaluate(R2_T3, [('r2', ('i', 'j', 'a', 'b'), s2, {})], ops, t2, acc)
    outs = _block_views(acc)
    evaluate(TERMS['H_T2'], blocks3, ops, t2, outs)
    evaluate(TERMS['H_T2_T2'], blocks3, ops, t2, outs)
    evaluate(TERMS['H_T3'], blocks3, ops, t2, outs)
    if linearize:
        _, M2, _ = amp.t2_class_masks(o, v, hole, part)
        tm = np.where(M2, t2, 0.0)
        evaluate(TERMS['H_T2_T2'], blocks3, ops, tm, outs, scale=-1.0)
        evaluate(TERMS['H_T2_T3'], blocks3, ops, t2 - tm, outs)
    else:
        evaluate(TERMS['H_T2_T3'], blocks3, ops, t2, outs)
    return acc['r1'], acc['r2'], gather(t3_idx, acc, o, v, hole, part)


class _BlockView:
    """Writes to R3'[i,j,k,a,b,c] at the fixed positions of one block land in
    that block's array (indexed by its free labels)."""

    def __init__(self, arr, free_pos):
        self.arr, self.free_pos = arr, free_pos

    def __getitem__(self, sel):
        return self.arr[tuple(sel[q] for q in self.free_pos)]

    def __setitem__(self, sel, val):
        self.arr[tuple(sel[q] for q in self.free_pos)] = val


def _block_views(acc):
    # free positions of each block among (i, j, k, a, b, c)
    return {'r1': acc['r1'], 'r2': acc['r2'],
            'RA': _BlockView(acc['RA'], (2, 4, 5)), 'RB': _BlockView(acc['RB'], (2, 3, 5)),
            'RC': _BlockView(acc['RC'], (1, 2, 5)), 'RD': _BlockView(acc['RD'], (0, 2, 5))}
