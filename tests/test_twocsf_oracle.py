"""The two-CSF ASCC oracle (Sec. II.B.2) against what fixes it independently:
determinant algebra (the zeroth-order guess), FCI (every orbital primary),
the one-CSF oracle (b = 0 with one primary pair), the determinants the
section prints as first-order T4' / T5' members, and spin symmetry."""
import numpy as np
import pytest

import synth
from oracle import ascc
from oracle import twocsf
from oracle.bruteforce import DetSpace, apply_ops


def _state(seed=3, root=2, excited=True):
    s = synth.make_system(3, 3, seed=seed)
    h1, p1, h2, p2, a, b, w = twocsf.cis_two_csf(s.eps, s.B, 3, root)
    st = twocsf.TwoCSF(s.eps, s.B, 3, h1, p1, h2, p2, a, b, excited=excited)
    return s, st, (h1, p1, h2, p2, a, b, w)


def test_guess_makes_the_two_csf_reference():
    """exp(-S+) exp(T^{P(0)}) phi0 is the reference of Eq. 2csf, and
    T^{P(0)} holds all-primary singles to quadruples only."""
    _, st, (h1, p1, h2, p2, a, b, w) = _state()
    assert len({h1, h2}) == 2 and len({p1, p2}) == 2 and min(w[:2]) > 0.3
    assert 2 * a * a + 2 * b * b == pytest.approx(1.0)
    t0 = st.guess()
    psi = st.wavefunction(t0)
    assert np.abs(psi - st.reference_state()).max() < 1e-14
    # Eq. 2csf written out: coefficient a on both spin forms of h1 -> p1, b
    # on those of h2 -> p2, nothing else
    sp_, o = st.space, st.o
    want = np.zeros(sp_.dim)
    for c, (h, p) in ((a, (h1, p1)), (b, (h2, p2))):
        for sg in (0, 1):
            s, d = apply_ops(sp_.dets[sp_.ref], [(sp_.spin_orb(o + p, sg), True),
                                                 (sp_.spin_orb(h, sg), False)])
            want[sp_.index[d]] += s * c
    assert np.abs(psi - want).max() < 1e-14
    nz = np.nonzero(np.abs(t0) > 1e-15)[0]
    assert {len(st.exc[k][0]) for k in nz} == {1, 2, 3, 4}
    prim_o = {sp_.spin_orb(i, sg) for i in (h1, h2) for sg in (0, 1)}
    prim_v = {sp_.spin_orb(o + p, sg) for p in (p1, p2) for sg in (0, 1)}
    for k in nz:
        I, A = st.exc[k]
        assert set(I) <= prim_o and set(A) <= prim_v


@pytest.mark.parametrize("linearize", [False, True])
def test_every_orbital_primary_gives_fci(linearize):
    """o = v = 2 with all four orbitals primary: T holds every excitation, so
    the excited and ground solutions are eigenvalues of H; every excitation
    is then all-primary (T^P), so partial linearisation changes nothing."""
    s = synth.make_system(2, 2, seed=2)
    h1, p1, h2, p2, a, b, _ = twocsf.cis_two_csf(s.eps, s.B, 2, 0)
    st = twocsf.TwoCSF(s.eps, s.B, 2, h1, p1, h2, p2, a, b, prim_occ=[0, 1], prim_vir=[0, 1],
                       linearize=linearize)
    assert not st.scaled.any()
    assert len(st.exc) == st.space.dim - 1
    E, _, _ = st.solve()
    w = np.linalg.eigvals(st.H).real
    assert np.min(np.abs(w - E)) < 1e-10
    assert E > w.min() + 1e-3                       # an excited root
    g = twocsf.TwoCSF(s.eps, s.B, 2, h1, p1, h2, p2, a, b, excited=False,
                      prim_occ=[0, 1], prim_vir=[0, 1], linearize=linearize)
    Eg, _, _ = g.solve()
    assert Eg == pytest.approx(w.min(), abs=1e-10)


@pytest.mark.parametrize("linearize", [False, True])
def test_one_csf_limit_matches_the_one_csf_oracle(linearize):
    """b = 0 with the primary pair (h1, p1) alone: T4' and T5' are empty and
    the state is the one-CSF ASCC + T3' state (Sec. II.B.1), or its PLASCC
    form (Sec. II.C), which the spin-adapted oracle solves with its own
    amplitudes and iteration."""
    o, hole, part = 3, 2, 0
    s = synth.make_system(o, 3, seed=1)
    st = twocsf.TwoCSF(s.eps, s.B, o, hole, part, hole, part, 1 / np.sqrt(2), 0.0,
                       prim_occ=[hole], prim_vir=[part], linearize=linearize)
    assert max(len(I) for I, _ in st.exc) == 3
    E, _, _ = st.solve()
    ref = ascc.solve_state(s.eps, s.B, o, hole, part, linearize=linearize, triples=True,
                           r_tol=1e-11, e_tol=1e-13, max_iter=400)
    assert ref.converged
    assert E == pytest.approx(ref.energy, abs=1e-9)


def test_example_determinants_are_t4_and_t5_members():
    """The first-order quadruples and quintuples the section prints (five and
    seven primary indices; the spins of the non-primary indices chosen to
    conserve S_z) are in the excited-state space; one primary fewer drops
    them; the ground state has the quadruples but no quintuples."""
    o, v = 4, 5
    sp_ = DetSpace(o, v)
    h1, h2, k, l = 0, 1, 2, 3             # occupied: primaries h1, h2
    p1, p2, c, d = 0, 1, 2, 3             # virtual: primaries p1, p2
    occ = lambda i, sg: sp_.spin_orb(i, sg)
    vir = lambda a, sg: sp_.spin_orb(o + a, sg)
    examples = [
        # h1 h1b h2 l -> p1 p1b c d
        ((occ(h1, 0), occ(h1, 1), occ(h2, 0), occ(l, 0)), (vir(p1, 0), vir(p1, 1), vir(c, 0), vir(d, 0)), 5),
        # h1 h1b k l -> p1 p1b p2 d
        ((occ(h1, 0), occ(h1, 1), occ(k, 0), occ(l, 1)), (vir(p1, 0), vir(p1, 1), vir(p2, 0), vir(d, 1)), 5),
        # h1 h1b h2 h2b m -> p1 p1b p2 d e
        ((occ(h1, 0), occ(h1, 1), occ(h2, 0), occ(h2, 1), occ(k, 0)),
         (vir(p1, 0), vir(p1, 1), vir(p2, 0), vir(c, 0), vir(d, 1)), 7),
        # h1 h1b h2 l m -> p1 p1b p2 p2b e
        ((occ(h1, 0), occ(h1, 1), occ(h2, 0), occ(k, 0), occ(l, 1)),
         (vir(p1, 0), vir(p1, 1), vir(p2, 0), vir(p2, 1), vir(c, 0)), 7),
    ]
    excited = set(twocsf.excitations(sp_, [h1, h2], [p1, p2], twocsf.EXCITED_RULE))
    ground = set(twocsf.excitations(sp_, [h1, h2], [p1, p2], twocsf.GROUND_RULE))
    prim = {occ(i, sg) for i in (h1, h2) for sg in (0, 1)} | {vir(a, sg) for a in (p1, p2) for sg in (0, 1)}
    for I, A, n in examples:
        key = (tuple(sorted(I)), tuple(sorted(A)))
        assert sum(q in prim for q in I + A) == n
        assert key in excited
        assert (key in ground) == (len(I) == 4)
        # replace the primary p1 (alpha) by the non-primary virtual of the same spin
        free = [vir(x, 0) for x in range(v) if x not in (p1, p2) and vir(x, 0) not in A]
        A2 = tuple(sorted([q for q in A if q != vir(p1, 0)] + [free[0]]))
        assert (tuple(sorted(I)), A2) not in excited
    assert not any(len(I) == 5 for I, _ in ground)


def test_two_csf_state_converges_to_a_singlet_with_t5():
    """A genuine two-CSF state (CSF weights 0.86 and 0.48, four distinct
    primary orbitals) converges; its wave function is a singlet, and its
    T4' and T5' amplitudes are nonzero."""
    _, st, _ = _state()
    E, t, its = st.solve()
    _, R = st.equations(t)
    assert np.abs(R).max() < 1e-11 and its < 20
    psi = st.wavefunction(t)
    S2 = st.space.s2_matrix()
    assert abs(psi @ S2 @ psi) / (psi @ psi) < 1e-10
    rank = np.array([len(I) for I, _ in st.exc])
    assert np.abs(t[rank == 4]).max() > 1e-6 and np.abs(t[rank == 5]).max() > 1e-8
    # the ground state with the same labels lies below
    _, g, _ = _state(excited=False)
    Eg, _, _ = g.solve()
    assert 0.05 < E - Eg < 5.0


def test_linearised_jacobian_matches_central_differences():
    """Newton's Jacobian of the PLASCC equations (the lambda factor of a scaled
    amplitude's column included) against central differences of the
    residual, at a perturbed two-CSF guess."""
    s = synth.make_system(3, 3, seed=3)
    h1, p1, h2, p2, a, b, _ = twocsf.cis_two_csf(s.eps, s.B, 3, 2)
    st = twocsf.TwoCSF(s.eps, s.B, 3, h1, p1, h2, p2, a, b, linearize=True)
    x = st.guess() + 0.01 * np.random.default_rng(0).standard_normal(len(st.exc))
    J = st.jacobian(x)
    cols = [0, int(np.nonzero(st.scaled)[0][5]), int(np.nonzero(~st.scaled)[0][-1])]
    for k in cols:
        e = np.zeros(len(x))
        e[k] = 1e-6
        fd = (st.equations(x + e)[1] - st.equations(x - e)[1]) / 2e-6
        assert np.abs(J[:, k] - fd).max() < 1e-7 * max(1.0, np.abs(fd).max())


def test_cis_matrix_is_h_on_the_singlet_singles():
    """The CIS matrix that picks the reference equals <CSF_ia| H - E_HF |CSF_jb>
    for the singlet CSFs (phi_i^a + phi_ib^ab) / sqrt(2), built in the
    determinant space from H itself."""
    o, v = 3, 3
    s = synth.make_system(o, v, seed=4)
    st = twocsf.TwoCSF(s.eps, s.B, o, 0, 0, 0, 0, 0.0, 0.0, excited=False)
    sp_ = st.space
    C = np.zeros((sp_.dim, o * v))
    for i in range(o):
        for a in range(v):
            for sg in (0, 1):
                sgn, d = apply_ops(sp_.dets[sp_.ref], [(sp_.spin_orb(o + a, sg), True),
                                                       (sp_.spin_orb(i, sg), False)])
                C[sp_.index[d], i * v + a] += sgn / np.sqrt(2.0)
    e_hf = st.H[sp_.ref, sp_.ref]
    want = C.T @ st.H @ C - e_hf * np.eye(o * v)
    assert np.abs(twocsf.cis_singlet_matrix(s.eps, s.B, o) - want).max() < 1e-12
