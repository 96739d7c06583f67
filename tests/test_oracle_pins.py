"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test below checks the oracle against something other than itself:
brute-force determinant algebra, closed forms, spectra, or structural
properties the paper states (Secs. II.A-II.D, S1).
"""
import itertools
import math
import os

import numpy as np
import pytest

from synth import make_system, random_amplitudes
from oracle import amplitudes as amp
from oracle import ascc
from oracle import bruteforce as bf
from oracle import hamiltonian as ham
from oracle import spinadapted as sa
from oracle import spinorb as so
from oracle import solver

GOLDEN = os.path.join(os.path.dirname(__file__), 'golden', 'paper_constants.txt')


def golden():
    out = {}
    for line in open(GOLDEN):
        if line.startswith('#') or not line.strip():
            continue
        name, val = line.split()[:2]
        out[name] = val
    return out


def system(o, v, seed=3, sigma=None):
    s = make_system(o, v, seed=seed, sigma=sigma)
    h, e_hf = ham.bare_hamiltonian(s.eps, s.B, o)
    return s, h, e_hf


# ------------------------------------------------------------ paper constants
def test_initial_guess_matches_paper_constants():
    g = golden()
    t1, t2, _ = amp.initial_guess(3, 5, 2, 1)
    assert t1[2, 1] == pytest.approx(float(g['beta']) * float(g['s_coefficient']), abs=1e-15)
    assert t2[2, 2, 1, 1] == pytest.approx(float(g['gamma']), abs=1e-15)
    assert np.count_nonzero(t1) == 1 and np.count_nonzero(t2) == 1
    b = 1.25
    t1, t2, _ = amp.initial_guess(3, 5, 2, 1, beta=b)
    assert t2[2, 2, 1, 1] == pytest.approx(float(g['gamma_of_beta_1.25']), abs=1e-15)
    lo, hi = amp.beta_from_alpha(float(g['aufbau_weight_beta_0.8']))
    assert lo == pytest.approx(0.8)


def test_spin_relations_signs():
    g = golden()
    assert g['s1_signs'] == '+1,-1' and g['s2_signs'] == '+1,-1,+1'
    rng = np.random.default_rng(0)
    o, v = 3, 3
    t3 = rng.standard_normal((o, o, o, v, v, v))
    t3 = t3 - t3.transpose(0, 2, 1, 3, 4, 5)
    t3 = t3 - t3.transpose(0, 1, 2, 3, 5, 4)
    ss = amp.t3_same_spin(t3)
    i, j, k, a, b, c = 0, 1, 2, 0, 1, 2
    want = t3[k, i, j, c, a, b] - t3[k, i, j, b, a, c] + t3[k, i, j, a, b, c]
    assert ss[i, j, k, a, b, c] == pytest.approx(want)
    # the same-spin triple built from a singlet is fully antisymmetric
    assert np.allclose(ss, -ss.transpose(1, 0, 2, 3, 4, 5))
    assert np.allclose(ss, -ss.transpose(0, 1, 2, 4, 3, 5))


def _det_apply(ops, det):
    """Applies a string of creation (True, q) / annihilation (False, q)
    operators, rightmost first, to the determinant bit mask det (spin orbital
    q = 2 p + spin, alpha = 0); returns (sign, det), sign 0 if it vanishes."""
    sign = 1
    for dag, q in reversed(ops):
        bit = 1 << q
        if dag == ((det & bit) != 0):
            return 0, 0
        if bin(det & (bit - 1)).count("1") & 1:
            sign = -sign
        det ^= bit
    return sign, det


def _singlet_amplitudes(o, v, rank, seed):
    """T|phi0> for T = sum s[i..,a..] E_ai E_bj (E_ck), E_ai = sum_spin
    a+_{a spin} a_{i spin} the spin-free excitation generators: T|phi0> is a
    singlet whatever s is.  Returns a function giving the coefficient of the
    determinant that an operator string makes from phi0, in the phase of
    that string."""
    import itertools
    so = lambda p, sp: 2 * p + sp
    phi0 = sum(1 << so(i, sp) for i in range(o) for sp in (0, 1))
    s = np.random.default_rng(seed).standard_normal((o,) * rank + (v,) * rank)
    wf = {}
    for idx in itertools.product(*([range(o)] * rank + [range(v)] * rank)):
        dets = {phi0: 1.0}
        for a, i in zip(idx[rank:], idx[:rank]):
            new = {}
            for d, c in dets.items():
                for sp in (0, 1):
                    sg, d2 = _det_apply([(True, so(o + a, sp)), (False, so(i, sp))], d)
                    if sg:
                        new[d2] = new.get(d2, 0.0) + sg * c
            dets = new
        for d, c in dets.items():
            wf[d] = wf.get(d, 0.0) + s[idx] * c

    def coef(occ, vir):
        # occ, vir: (spatial index, spin) in the order of
        # a+_vir[0] a+_vir[1] ... a_occ[-1] ... a_occ[0]
        ops = [(True, so(o + a, sp)) for a, sp in vir] + [(False, so(i, sp)) for i, sp in occ[::-1]]
        sg, d = _det_apply(ops, phi0)
        return sg * wf.get(d, 0.0) if sg else 0.0
    return coef


def test_same_spin_relations_hold_for_a_spin_free_singlet():
    """Eqs. S1 and S2 against determinant algebra: the same-spin doubles and
    triples of a singlet built from spin-free generators equal the relations
    applied to its alpha-beta / alpha-beta-beta amplitudes (amplitude = the
    coefficient of a+_a a+_b (a+_c) ... a_j a_i phi0, as T is written).  A sign
    or index slip in either relation fails this (checked below by planting
    one)."""
    import itertools
    o, v = 3, 4
    coef = _singlet_amplitudes(o, v, 2, seed=11)
    t2 = np.zeros((o, o, v, v))
    for i, j, a, b in itertools.product(range(o), range(o), range(v), range(v)):
        t2[i, j, a, b] = coef([(i, 0), (j, 1)], [(a, 0), (b, 1)])
    assert np.abs(t2 - t2.transpose(1, 0, 3, 2)).max() < 1e-14   # singlet pair symmetry
    ss2 = amp.t2_same_spin(t2)
    n = 0
    for i, j, a, b in itertools.product(range(o), range(o), range(v), range(v)):
        if i < j and a < b:
            assert ss2[i, j, a, b] == pytest.approx(coef([(i, 0), (j, 0)], [(a, 0), (b, 0)]),
                                                    abs=1e-13)
            n += 1
    assert n == 18

    o, v = 4, 4
    coef = _singlet_amplitudes(o, v, 3, seed=12)
    t3 = np.zeros((o, o, o, v, v, v))
    for i, j, k, a, b, c in itertools.product(*([range(o)] * 3 + [range(v)] * 3)):
        t3[i, j, k, a, b, c] = coef([(i, 0), (j, 1), (k, 1)], [(a, 0), (b, 1), (c, 1)])
    want = {}
    for i, j, k, a, b, c in itertools.product(*([range(o)] * 3 + [range(v)] * 3)):
        if i < j < k and a < b < c:
            want[i, j, k, a, b, c] = coef([(i, 0), (j, 0), (k, 0)], [(a, 0), (b, 0), (c, 0)])
    assert len(want) == 16 and max(abs(x) for x in want.values()) > 0.1
    ss3 = amp.t3_same_spin(t3)
    for key, w in want.items():
        assert ss3[key] == pytest.approx(w, abs=1e-12)
    # a planted sign slip in the middle term fails the comparison
    s_ = t3.transpose(1, 2, 0, 3, 4, 5)
    wrong = s_.transpose(0, 1, 2, 4, 5, 3) + s_.transpose(0, 1, 2, 4, 3, 5) + s_
    assert max(abs(wrong[key] - w) for key, w in want.items()) > 1e-3


# ------------------------------------------------------------ H-bar closed forms
def test_reference_energy_of_hbar_closed_form():
    """<phi0|H-bar|phi0> = E_HF + 1/2 (ph|ph) (Brillouin: f_hp = 0)."""
    o, v = 4, 7
    s, h, e_hf = system(o, v)
    hole, part = 2, 3
    hb, Bb = ham.similarity_transform(h, s.B, o, hole, part)
    blk = sa.dressed_blocks(hb, Bb, o, np.zeros((o, v)))
    p = o + part
    php = float(np.sum(s.B[:, p, hole] * s.B[:, p, hole]))
    assert blk.reference_energy() == pytest.approx(e_hf + 0.5 * php, abs=1e-12)
    # and x = 0 gives E_HF
    blk0 = sa.dressed_blocks(h, s.B, o, np.zeros((o, v)))
    assert blk0.reference_energy() == pytest.approx(e_hf, abs=1e-12)


def test_hbar_changes_only_creation_h_or_annihilation_p():
    o, v = 3, 5
    s, h, _ = system(o, v)
    hole, part = 1, 2
    hb, Bb = ham.similarity_transform(h, s.B, o, hole, part)
    p = o + part
    dh = np.abs(hb - h) > 1e-14
    rows, cols = np.nonzero(dh)
    assert np.all((rows == hole) | (cols == p))
    g = ham.eri_from_df(s.B); gb = ham.eri_from_df(Bb)
    d = np.abs(gb - g) > 1e-14
    P, Q, R, S = np.nonzero(d)
    assert np.all((P == hole) | (R == hole) | (Q == p) | (S == p))
    # the excitation block (ai|bj) is untouched
    ov = (slice(o, None), slice(0, o))
    assert np.allclose(gb[ov[0], ov[1], ov[0], ov[1]], g[ov[0], ov[1], ov[0], ov[1]], atol=1e-15)


def test_similarity_transform_preserves_fci_spectrum():
    """exp(S^+) H exp(-S^+) has the spectrum of H (Sec. II.A)."""
    o, v = 2, 4
    s, h, _ = system(o, v)
    sp = bf.DetSpace(o, v)
    g = ham.eri_from_df(s.B)
    hb, Bb = ham.similarity_transform(h, s.B, o, 1, 2)
    w0 = np.sort(np.linalg.eigvals(sp.hamiltonian_matrix(h, g)).real)
    w1 = np.sort(np.linalg.eigvals(sp.hamiltonian_matrix(hb, ham.eri_from_df(Bb))).real)
    assert np.allclose(w0, w1, atol=1e-10)


def test_reference_construction_beta_one_gives_S_phi0():
    """exp(-S^+) exp(T^P(0)) phi0 = S phi0 for beta = 1 (Eqs. 1csf, TP-guess)."""
    o, v = 2, 3
    sp = bf.DetSpace(o, v)
    hole, part = 1, 0
    t1, t2, _ = amp.initial_guess(o, v, hole, part)
    T = sp.string_matrix(sp.cluster_strings(t1, t2))
    ref = np.zeros(sp.dim); ref[sp.ref] = 1.0
    r = 1 / math.sqrt(2)
    h_, p_ = hole, o + part
    S = sp.string_matrix([(r, [(sp.spin_orb(p_, s), True), (sp.spin_orb(h_, s), False)]) for s in (0, 1)])
    Sd = S.T.tocsr()
    psi = sp.exp_apply(T, ref, +1.0)
    psi = sp.exp_apply(Sd, psi, -1.0)
    assert np.allclose(psi, S @ ref, atol=1e-14)
    # beta != 1 with gamma = -beta^2/2: ((1-beta)/beta) phi0 + S phi0 up to normalisation
    beta = 0.8
    t1, t2, _ = amp.initial_guess(o, v, hole, part, beta=beta)
    T = sp.string_matrix(sp.cluster_strings(t1, t2))
    psi = sp.exp_apply(Sd, sp.exp_apply(T, ref, +1.0), -1.0)
    want = (1 - beta) / beta * ref + S @ ref
    k = np.argmax(np.abs(want))
    assert np.allclose(psi / psi[k] * want[k], want, atol=1e-14)


# ------------------------------------------------------------ residual levels
CASES = [(2, 4, None), (2, 4, (1, 0)), (3, 4, (2, 0)), (3, 4, (0, 3))]


@pytest.mark.parametrize("o,v,exc", CASES)
@pytest.mark.parametrize("linearize", [False, True])
@pytest.mark.parametrize("triples", [False, True])
def test_bruteforce_spinorbital_spinadapted_agree(o, v, exc, linearize, triples):
    """O-BF (definition) = O-SO (spin orbital) = O-SA (spin adapted), Eqs. energy/amp, S1-S2."""
    if exc is None and triples:
        pytest.skip("the ground state has no T3'")
    s, h, _ = system(o, v)
    hole, part = exc if exc else (None, None)
    lh, lp = exc if exc else (o - 1, 0)
    hb, Bb = ham.similarity_transform(h, s.B, o, hole, part)
    g = ham.eri_from_df(Bb)
    idx = amp.t3p_index(o, v, hole, part) if triples else np.zeros((0, 6), np.int64)
    t1, t2, t3 = random_amplitudes(o, v, seed=11, scale=0.1, n_t3=len(idx))
    sp = bf.DetSpace(o, v)
    Eb, R1b, R2b, R3b = bf.projected_equations(sp, hb, g, t1, t2, idx if triples else None, t3,
                                               linearize=linearize, hole=lh, particle=lp)
    Es, R1s, R2s, R3s = so.residual(hb, g, t1, t2, amp.t3_dense(idx, t3, o, v) if triples else None,
                                    linearize=linearize, hole=lh, particle=lp)
    Ea, R1a, R2a, R3a = sa.residual(hb, Bb, o, t1, t2, linearize=linearize, hole=lh, particle=lp,
                                    t3_idx=idx if triples else None, t3_vals=t3)
    tol = 1e-12
    assert abs(Eb - Es) < tol and abs(Ea - Es) < tol
    assert np.abs(R1b - R1s).max() < tol and np.abs(R1a - R1s).max() < tol
    assert np.abs(R2b - R2s).max() < tol and np.abs(R2a - R2s).max() < tol
    if triples:
        assert np.abs(R3b - amp.t3_gather(R3s, idx)).max() < tol
        assert np.abs(R3a - R3b).max() < tol


@pytest.mark.parametrize("o,v,hole,part", [(3, 6, 2, 0), (4, 7, 1, 4), (4, 8, 0, 7)])
@pytest.mark.parametrize("linearize", [False, True])
def test_slice_oracle_matches_spinorbital(o, v, hole, part, linearize):
    """O-SL (the T3' terms evaluated on the four slice blocks, t3slice) equals
    the dense spin-orbital triples of O-SO at sizes beyond brute force."""
    from oracle import t3slice
    s, h, _ = system(o, v, seed=6, sigma=0.15)
    hb, Bb = ham.similarity_transform(h, s.B, o, hole, part)
    idx = amp.t3p_index(o, v, hole, part)
    t1, t2, t3 = random_amplitudes(o, v, seed=12, scale=0.1, n_t3=len(idx))
    blk = sa.dressed_blocks(hb, Bb, o, t1)
    r1, r2, r3 = t3slice.residual(blk, t2, idx, t3, hole, part, linearize=linearize)
    _, r1s, r2s, R3s = so.residual(hb, ham.eri_from_df(Bb), t1, t2, amp.t3_dense(idx, t3, o, v),
                                   linearize=linearize, hole=hole, particle=part,
                                   triples_only=True)
    tol = 1e-12 * max(1.0, np.abs(R3s).max())
    assert np.abs(r1 - r1s).max() < tol
    assert np.abs(r2 - r2s).max() < tol
    assert np.abs(r3 - amp.t3_gather(R3s, idx)).max() < tol
    # the blocks partition the slice: unpacking and gathering is the identity
    X = t3slice.blocks_from_slice(idx, t3, o, v, hole, part)
    R = {'R' + k[1]: X[k] for k in X}
    assert np.array_equal(t3slice.gather(idx, R, o, v, hole, part), t3)


def test_linearisation_changes_the_residual():
    """PLASCC differs from ASCC exactly by the T2^M T2^M terms (Sec. II.C)."""
    o, v = 3, 5
    s, h, _ = system(o, v)
    hb, Bb = ham.similarity_transform(h, s.B, o, 2, 1)
    t1, t2, _ = random_amplitudes(o, v, seed=2, scale=0.1)
    _, _, R2a, _ = sa.residual(hb, Bb, o, t1, t2)
    _, _, R2p, _ = sa.residual(hb, Bb, o, t1, t2, linearize=True, hole=2, particle=1)
    assert np.abs(R2a - R2p).max() > 1e-4
    # with no mixed doubles, nothing is removed
    _, M2, _ = amp.t2_class_masks(o, v, 2, 1)
    t2n = np.where(M2, 0.0, t2)
    _, _, a, _ = sa.residual(hb, Bb, o, t1, t2n)
    _, _, b, _ = sa.residual(hb, Bb, o, t1, t2n, linearize=True, hole=2, particle=1)
    assert np.abs(a - b).max() < 1e-15


# ------------------------------------------------------------ closed forms
def test_first_iteration_energy_is_mp2():
    """From T = 0 the first Jacobi step gives E_HF + E_MP2 (closed form)."""
    o, v = 4, 9
    s, h, e_hf = system(o, v, seed=5)
    eo, ev = s.eps[:o], s.eps[o:]
    ovov = np.einsum('Pia,Pjb->iajb', s.B[:, :o, o:], s.B[:, :o, o:])
    D = eo[:, None, None, None] - ev[None, :, None, None] + eo[None, None, :, None] - ev[None, None, None, :]
    e_mp2 = float(np.sum(ovov * (2 * ovov - ovov.transpose(0, 3, 2, 1)) / D))
    res = ascc.solve_state(s.eps, s.B, o, linearize=False, max_iter=1)
    assert res.history[0][1] == pytest.approx(e_hf, abs=1e-12)
    assert res.history[1][1] == pytest.approx(e_hf + e_mp2, abs=1e-12)


def test_t3p_slice_size_closed_form():
    """|T3'| = (o-1)[C(v,2) + (v-1)^2] + C(o-1,2)(v-1) + (o-1)^2 (v-1)  (Sec. II.B.1)."""
    for o, v in [(2, 4), (3, 5), (5, 7), (6, 3)]:
        n = len(amp.t3p_index(o, v, o - 1, 0))
        want = (o - 1) * (v * (v - 1) // 2 + (v - 1) ** 2) + (o - 1) * (o - 2) // 2 * (v - 1) + (o - 1) ** 2 * (v - 1)
        assert n == want
    # every listed element has >= 3 primary spin-orbital indices and j<k, b<c
    idx = amp.t3p_index(5, 6, 3, 2)
    i, j, k, a, b, c = idx.T
    cnt = (i == 3).astype(int) + ((j == 3) | (k == 3)) + (a == 2) + ((b == 2) | (c == 2))
    assert np.all(cnt >= 3) and np.all(j < k) and np.all(b < c)
    order = np.lexsort(idx.T[::-1])
    assert np.all(order == np.arange(len(idx)))


# ------------------------------------------------------------ FCI limits
def test_two_electron_ccsd_is_fci():
    """o = 1: CCSD is exact for two electrons (Sec. II.A FCI limit)."""
    o, v = 1, 5
    s, h, _ = system(o, v, seed=7, sigma=0.05)
    res = ascc.solve_state(s.eps, s.B, o, linearize=False, r_tol=1e-11, e_tol=1e-13)
    assert res.converged
    w, s2 = bf.fci_energies(bf.DetSpace(o, v), h, ham.eri_from_df(s.B))
    singlets = np.sort(w.real[np.abs(s2) < 1e-8])
    assert res.energy == pytest.approx(singlets[0], abs=1e-10)


def test_two_electron_ascc_hits_excited_fci_root():
    """o = 1: unlinearised ASCC (T1+T2, T3' empty) converges to an excited FCI singlet."""
    o, v = 1, 5
    s, h, _ = system(o, v, seed=7, sigma=0.05)
    assert len(amp.t3p_index(o, v, 0, 0)) == 0
    res = ascc.solve_state(s.eps, s.B, o, 0, 0, linearize=False, triples=True, r_tol=1e-11, e_tol=1e-13)
    assert res.converged
    w, s2 = bf.fci_energies(bf.DetSpace(o, v), h, ham.eri_from_df(s.B))
    singlets = np.sort(w.real[np.abs(s2) < 1e-8])
    d = np.abs(singlets - res.energy)
    assert d.min() < 1e-10 and np.argmin(d) > 0


# ------------------------------------------------------------ size consistency
def _fragment_pair(oA, vA, oB, vB, seed):
    a = make_system(oA, vA, seed=seed)
    b = make_system(oB, vB, seed=seed + 1)
    o, v = oA + oB, vA + vB
    n = o + v
    # orbital order: occ(A) occ(B) vir(A) vir(B)
    mapA = list(range(oA)) + list(range(o, o + vA))
    mapB = list(range(oA, o)) + list(range(o + vA, n))
    eps = np.zeros(n); eps[mapA] = a.eps; eps[mapB] = b.eps
    B = np.zeros((a.naux + b.naux, n, n))
    B[np.ix_(range(a.naux), mapA, mapA)] = a.B
    B[np.ix_(range(a.naux, a.naux + b.naux), mapB, mapB)] = b.B
    return a, b, eps, B, o


@pytest.mark.parametrize("linearize", [False, True])
def test_size_consistency_and_intensivity(linearize):
    """Non-interacting fragments: E(A+B) = E(A) + E(B), omega(A+B) = omega(A) (Secs. II.A, II.C)."""
    oA, vA, oB, vB = 2, 5, 2, 4
    a, b, eps, B, o = _fragment_pair(oA, vA, oB, vB, seed=21)
    kw = dict(r_tol=1e-10, e_tol=1e-12)
    hA, pA = 1, 0            # excitation on fragment A (global indices coincide for A)
    gsA = ascc.solve_state(a.eps, a.B, oA, linearize=linearize, pl_hole=hA, pl_particle=pA, **kw)
    gsB = ascc.solve_state(b.eps, b.B, oB, linearize=False, **kw)   # fragment B holds no primary orbital
    exA = ascc.solve_state(a.eps, a.B, oA, hA, pA, linearize=linearize, **kw)
    gsAB = ascc.solve_state(eps, B, o, linearize=linearize, pl_hole=hA, pl_particle=pA, **kw)
    exAB = ascc.solve_state(eps, B, o, hA, pA, linearize=linearize, **kw)
    for r in (gsA, gsB, exA, gsAB, exAB):
        assert r.converged
    assert gsAB.energy == pytest.approx(gsA.energy + gsB.energy, abs=1e-9)
    assert (exAB.energy - gsAB.energy) == pytest.approx(exA.energy - gsA.energy, abs=1e-9)


# ------------------------------------------------------------ orbital invariance
def test_invariance_to_nonprimary_occupied_rotation():
    """Rotating non-primary occupied orbitals among themselves leaves E unchanged (Sec. II.B)."""
    o, v = 4, 6
    s, h, _ = system(o, v, seed=7)
    hole, part = 3, 0
    kw = dict(r_tol=1e-10, e_tol=1e-12)
    ref = ascc.solve_state(s.eps, s.B, o, hole, part, linearize=True, **kw)
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    R = np.eye(o + v); R[:3, :3] = Q          # rotate occupied 0..2 (hole = 3 untouched)
    B2 = np.einsum('pa,Pab,bq->Ppq', R.T, s.B, R)
    h2 = R.T @ h @ R
    hb, Bb = ham.similarity_transform(h2, B2, o, hole, part)
    idx = np.zeros((0, 6), np.int64)
    t1, t2, t3 = amp.initial_guess(o, v, hole, part)

    def fn(a, b, c):
        E, R1, R2, _ = sa.residual(hb, Bb, o, a, b, linearize=True, hole=hole, particle=part)
        return E, R1, R2, np.zeros(0)
    eps_rot = np.diag(R.T @ np.diag(s.eps) @ R)     # Jacobi denominators from the rotated Fock diagonal
    rot = solver.solve(fn, eps_rot, o, t1, t2, t3, **kw)
    assert ref.converged and rot.converged
    assert rot.energy == pytest.approx(ref.energy, abs=1e-9)


def test_second_ansatz_reference_has_the_same_aufbau_weight():
    """Both ansatz choices of Sec. II.D build alpha phi0 + S phi0 (up to normalisation)."""
    o, v = 2, 3
    sp = bf.DetSpace(o, v)
    hole, part = 1, 0
    alpha = 0.15
    r = 1 / math.sqrt(2)
    h_, p_ = hole, o + part
    S = sp.string_matrix([(r, [(sp.spin_orb(p_, s), True), (sp.spin_orb(h_, s), False)]) for s in (0, 1)])
    Sd = S.T.tocsr()
    ref = np.zeros(sp.dim); ref[sp.ref] = 1.0
    want = alpha * ref + S @ ref
    for ans in (0, 1):
        beta, sign = ascc.ansatz_beta(alpha, ans)
        t1, t2, _ = amp.initial_guess(o, v, hole, part, beta=beta, xsign=sign)
        T = sp.string_matrix(sp.cluster_strings(t1, t2))
        psi = sp.exp_apply(sign * Sd, sp.exp_apply(T, ref, +1.0), -1.0)
        k = np.argmax(np.abs(want))
        assert np.allclose(psi / psi[k] * want[k], want, atol=1e-14)
