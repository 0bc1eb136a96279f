"""Pins for the (0h,1p) FS-CCSD oracle against things other than itself."""
import itertools

import numpy as np
import pytest

import brute_force as bf
from oracle import ccsd, fs0h1p, integrals
from paper_2004_03682_gb300 import synthetic as syn


def _converged(seed, no, nv, G=1):
    prob = syn.make_problem(seed, no, nv, G)
    if no == 1:
        # a one-electron vacuum has no doubles, so the MP2-based scale is undefined:
        # use a fixed small scale instead
        V = 0.02 * integrals.unscaled_integrals(prob)
    else:
        V = integrals.integrals(prob)
    f = integrals.fock(prob)
    b = ccsd.Blocks(V, f, no)
    t1, t2, E, _, conv, _ = ccsd.solve(b, tol=1e-12, max_iter=400)
    assert conv
    return prob, V, f, t1, t2


@pytest.mark.parametrize("no,nv", [(2, 4), (1, 5)])
def test_hbar_on_attached_vectors_equals_brute_force(rng, no, nv):
    prob, V, f, t1, t2 = _converged(41 + no, no, nv)
    M, labels = bf.ea_eom_matrix(f, V, no, t1, t2)
    Va, fa = fs0h1p.augment(V, f, no, 2)
    b_aug = ccsd.Blocks(Va, fa, no + 2)
    r1 = rng.standard_normal((2, nv)) + 1j * rng.standard_normal((2, nv))
    x = rng.standard_normal((2, no, nv, nv)) + 1j * rng.standard_normal((2, no, nv, nv))
    r2 = x - x.transpose(0, 1, 3, 2)
    s1, s2 = fs0h1p.hbar_ea(b_aug, t1, t2, no, r1, r2)
    for k in range(2):
        vec = np.array([r1[k, l[1]] if l[0] == "p" else r2[k, l[1], l[2], l[3]] for l in labels])
        out = M @ vec
        got = np.array([s1[k, l[1]] if l[0] == "p" else s2[k, l[1], l[2], l[3]] for l in labels])
        np.testing.assert_allclose(got, out, atol=1e-13 * np.max(np.abs(out)), rtol=0)


def test_heff_eigenvalues_in_attached_spectrum_and_one_electron_fci():
    # one-electron vacuum: CCSD is exact and {1p, 2p1h} spans every two-electron state
    prob, V, f, t1, t2 = _converged(53, 1, 6)
    assert np.max(np.abs(t1)) < 1e-15 and np.max(np.abs(t2)) < 1e-15
    act = syn.active_virtuals(prob, 2)
    Heff, w, _, _, nit, conv = fs0h1p.solve(V, f, 1, t1, t2, act, tol=1e-12)
    assert conv
    spec2 = bf.sector_spectrum(f, V, 1, 2)       # E(2e) - E_ref(1e), E_CC(1e) = 0
    for e in w:
        assert np.min(np.abs(spec2 - e)) < 1e-10
    M, _ = bf.ea_eom_matrix(f, V, 1, t1, t2)
    ev = np.linalg.eigvals(M)
    for e in w:
        assert np.min(np.abs(ev - e)) < 1e-10


def test_heff_eigenvalues_in_ea_eom_spectrum_two_electrons():
    prob, V, f, t1, t2 = _converged(59, 2, 5)
    act = syn.active_virtuals(prob, 2)
    Heff, w, _, _, nit, conv = fs0h1p.solve(V, f, 2, t1, t2, act, tol=1e-12)
    assert conv
    M, _ = bf.ea_eom_matrix(f, V, 2, t1, t2)
    ev = np.linalg.eigvals(M)
    for e in w:
        assert np.min(np.abs(ev - e)) < 1e-9


def test_heff_block_diagonal_by_irrep():
    prob = syn.make_problem(306, 6, 20, G=4)
    V = integrals.integrals(prob)
    f = integrals.fock(prob)
    t1, t2, E, _, conv, _ = ccsd.solve(ccsd.Blocks(V, f, 6), tol=1e-11)
    assert conv
    act = syn.active_virtuals(prob, 4)
    Heff, w, s1, s2, nit, conv = fs0h1p.solve(V, f, 6, t1, t2, act, tol=1e-11)
    assert conv
    g = prob.irrep_of[6:][act]
    for y, x in itertools.product(range(4), range(4)):
        if g[y] != g[x]:
            assert Heff[y, x] == 0
