"""Pins for the (0h,2p) oracle (oracle/fs0h2p.py).

  * Normal products: the reordering drops exactly the contraction of a valence line
    (hand-checked strings).
  * Two electrons on an empty reference (o = 0, T = 0) with a non-diagonal Fock matrix
    (so the (0h,1p) amplitudes are nonzero and {S1 S1} takes part): the Bloch equation
    is exact there, so every H_eff eigenvalue is a two-electron full-CI eigenvalue.
  * With occupied spinors (T, s_x^a and s_xj^ab all nonzero), against a second,
    independent construction of the same sector: every active spinor becomes a
    non-interacting occupied "ghost" whose CCSD amplitudes (oracle.ccsd) carry the
    valence amplitudes; the (0h,2p) equation is the ghost-ghost doubles residual minus
    the H_eff terms of Omega H_eff, sum_z s_zy^ab H1_zx + sum_w s_xw^ab H1_wy
    + 1/2 sum_zw tau_zw^ab H2_zw,xy.  The two routes share no code and must give the
    same H_eff eigenvalues."""
import numpy as np
import pytest

import brute_force as bf
from oracle import ccsd, fs0h1p, fs0h2p, integrals
from paper_2004_03682_gb300 import synthetic as syn


def test_normal_product_drops_valence_contractions():
    o = 1
    x, i = 3, 0  # a virtual and an occupied spinor
    ops, sg = fs0h2p.normal_product([(x, False), (x, True)], o)  # {x x+} = -x+ x
    assert ops == [(x, True), (x, False)] and sg == -1
    ops, sg = fs0h2p.normal_product([(i, True), (i, False)], o)  # {i+ i} = -i i+
    assert ops == [(i, False), (i, True)] and sg == -1
    ref = 0b1
    # plain x x+ |0> = |0>; the normal product has no contraction: 0
    d, s = fs0h2p.apply_ops([(x, False), (x, True)], ref)
    assert d == ref and s == 1
    d, s = fs0h2p.apply_ops(ops, ref)
    assert d is None
    # an already normal-ordered string is unchanged
    A = [(4, True), (5, True), (0, False), (3, False)]
    assert fs0h2p.normal_product(A, o) == (A, 1)


def _empty_reference(seed, nv, G, general):
    """v virtual spinors and no occupied ones: the virtual block of a two-occupied problem
    (one occupied spinor would leave <ab||ij> = 0 and no MP2 scale)."""
    prob = syn.make_problem(seed, 2, nv, G)
    V, f = integrals.integrals(prob), integrals.fock(prob)
    V, f = V[2:, 2:, 2:, 2:], f[2:, 2:].copy()
    if general:
        rng = np.random.default_rng(seed)
        gv = prob.irrep_of[2:]
        X = 0.05 * (rng.standard_normal((nv, nv)) + 1j * rng.standard_normal((nv, nv)))
        X = X * (gv[:, None] == gv[None, :])
        f = f + X + X.conj().T
    return V, f


@pytest.mark.parametrize("seed,nv,G,nact,general", [(901, 5, 1, 2, True), (902, 6, 1, 3, True),
                                                    (903, 6, 2, 3, True), (904, 5, 1, 3, False)])
def test_two_electrons_on_empty_reference_equal_full_ci(seed, nv, G, nact, general):
    V, f = _empty_reference(seed, nv, G, general)
    act = np.arange(nact)  # the lowest virtual spinors of the stored order
    t1, t2 = np.zeros((0, nv), complex), np.zeros((0, 0, nv, nv), complex)
    H1, w1, s1, s2, _, conv = fs0h1p.solve(V, f, 0, t1, t2, act, tol=1e-12, max_iter=500)
    assert conv
    if general:
        assert np.max(np.abs(s1)) > 1e-4  # the (0h,1p) amplitudes take part
    Heff, w, s, pairs, qp, nit, conv = fs0h2p.solve(V, f, 0, t1, t2, 0.0, act, s1, s2, tol=1e-12, max_iter=500)
    assert conv
    fci = bf.sector_spectrum(f, V, 0, 2)
    for e in w:
        assert abs(e.imag) < 1e-9
        assert np.min(np.abs(fci - e.real)) < 1e-9, (e, fci)


@pytest.mark.parametrize("seed,no,nv,G,nact", [(911, 2, 5, 1, 2), (916, 2, 6, 2, 3), (918, 3, 6, 2, 2),
                                               (921, 2, 6, 4, 3)])
def test_occupied_reference_equals_ghost_construction(seed, no, nv, G, nact):
    prob = syn.make_problem(seed, no, nv, G)
    V, f = integrals.integrals(prob), integrals.fock(prob)
    b = ccsd.Blocks(V, f, no)
    t1, t2, E, _, conv, _ = ccsd.solve(b, tol=1e-12, max_iter=600)
    assert conv
    act = np.argsort(prob.eps_virt)[:nact]
    H1, w1, s1, s2, _, conv = fs0h1p.solve(V, f, no, t1, t2, act, tol=1e-12, max_iter=600)
    assert conv
    assert np.max(np.abs(s2)) > 1e-5
    Heff, w, s, pairs, qp, nit, conv = fs0h2p.solve(V, f, no, t1, t2, E, act, s1, s2, tol=1e-11, max_iter=600)
    assert conv
    Hg, wg, conv_g = fs0h2p.solve_ghost(V, f, no, t1, t2, act, s1, s2)
    assert conv_g
    np.testing.assert_allclose(np.sort_complex(w), np.sort_complex(wg), atol=1e-9, rtol=0)


def test_sign_slip_in_normal_product_is_caught(monkeypatch):
    """Control: dropping the permutation sign of the normal product flips 1/2 {S1 S1}.
    With an empty reference that term only feeds two-particle components, which S2
    absorbs (the eigenvalues cannot see it); with occupied spinors the products with
    s_xj^ab reach three-particle-one-hole components, and the eigenvalues move away from
    the ghost construction's."""
    prob = syn.make_problem(911, 2, 5, 1)
    V, f = integrals.integrals(prob), integrals.fock(prob)
    b = ccsd.Blocks(V, f, 2)
    t1, t2, E, _, conv, _ = ccsd.solve(b, tol=1e-12, max_iter=600)
    act = np.argsort(prob.eps_virt)[:2]
    H1, w1, s1, s2, _, conv = fs0h1p.solve(V, f, 2, t1, t2, act, tol=1e-12, max_iter=600)
    Hg, wg, conv_g = fs0h2p.solve_ghost(V, f, 2, t1, t2, act, s1, s2)
    right = fs0h2p.normal_product
    monkeypatch.setattr(fs0h2p, "normal_product", lambda ops, o: (right(ops, o)[0], 1))
    Heff, w, s, pairs, qp, nit, conv = fs0h2p.solve(V, f, 2, t1, t2, E, act, s1, s2, tol=1e-11, max_iter=600)
    assert np.max(np.abs(np.sort_complex(w) - np.sort_complex(wg))) > 1e-6
