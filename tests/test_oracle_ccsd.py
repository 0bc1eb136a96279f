"""Pins for the CCSD oracle against things other than itself.

* brute-force second quantisation (e^-T H e^T on determinants) for the residual
  and the energy at random amplitudes, with a general Hermitian Fock matrix;
* full CI for two electrons (CCSD is exact there);
* the closed-form MP2 energy and the first Jacobi step from T = 0;
* antisymmetry, real-integral and gauge invariants, symmetry-blocked == C1.
"""
import numpy as np
import pytest

import brute_force as bf
from oracle import ccsd, integrals
from paper_2004_03682_gb300 import synthetic as syn


def _random_amplitudes(rng, no, nv, scale=0.1):
    t1 = scale * (rng.standard_normal((no, nv)) + 1j * rng.standard_normal((no, nv)))
    x = scale * (rng.standard_normal((no, no, nv, nv)) + 1j * rng.standard_normal((no, no, nv, nv)))
    t2 = x - x.swapaxes(0, 1) - x.swapaxes(2, 3) + x.swapaxes(0, 1).swapaxes(2, 3)
    return t1, t2


def _random_hermitian(rng, n, scale):
    x = scale * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    return x + x.conj().T


def _problem(seed, no, nv, G=1):
    prob = syn.make_problem(seed, no, nv, G)
    V = integrals.integrals(prob)
    return prob, V


@pytest.mark.parametrize("no,nv,G", [(3, 4, 1), (2, 5, 1), (3, 4, 2)])
def test_residual_and_energy_match_brute_force(rng, no, nv, G):
    prob, V = _problem(7 + no + nv, no, nv, G)
    # general Hermitian Fock matrix: pins the f_ov, off-diagonal f_oo/f_vv terms
    f = np.diag(prob.eps).astype(complex) + _random_hermitian(rng, prob.n, 0.05)
    b = ccsd.Blocks(V, f, no)
    t1, t2 = _random_amplitudes(rng, no, nv)
    E_bf, R1_bf, R2_bf = bf.ccsd_projections(f, V, no, t1, t2)
    R1, R2 = ccsd.residual(t1, t2, b)
    E = ccsd.energy(t1, t2, b)
    assert abs(E - E_bf) < 1e-12
    np.testing.assert_allclose(R1, R1_bf, atol=1e-12, rtol=0)
    np.testing.assert_allclose(R2, R2_bf, atol=1e-12, rtol=0)


def test_two_electron_ccsd_equals_fci():
    prob, V = _problem(31, 2, 6)
    f = integrals.fock(prob)
    b = ccsd.Blocks(V, f, 2)
    t1, t2, E, nit, conv, _ = ccsd.solve(b, tol=1e-12, max_iter=200)
    assert conv
    E_fci, _ = bf.fci_correlation(f, V, 2)
    assert abs(E.real - E_fci) < 1e-11
    assert abs(E.imag) < 1e-12


def test_first_iteration_is_mp2_closed_form():
    prob, V = _problem(5, 4, 12)
    b = ccsd.Blocks(V, integrals.fock(prob), 4)
    _, _, _, _, _, recs = ccsd.solve(b, tol=1e-9, max_iter=1)
    e_mp2 = ccsd.mp2_energy(b)
    assert e_mp2 < 0
    assert abs(recs[0].energy.real - e_mp2) < 1e-14 * max(1.0, abs(e_mp2))
    assert abs(recs[0].energy.imag) < 1e-15
    # one Jacobi step from T = 0 gives t1 = 0 (f_ov = 0) and t2 = MP2
    z1 = np.zeros((4, 12), complex)
    z2 = np.zeros((4, 4, 12, 12), complex)
    r1, r2 = ccsd.rhs(z1, z2, b)
    D1, D2 = ccsd.denominators(b)
    assert np.max(np.abs(r1)) == 0.0
    np.testing.assert_allclose(r2 / D2, ccsd.mp2_guess(b)[1], atol=0, rtol=1e-15)


def test_max_mp2_amplitude_scaled_to_0p05():
    prob, V = _problem(9, 4, 12, G=2)
    b = ccsd.Blocks(V, integrals.fock(prob), 4)
    assert abs(np.max(np.abs(ccsd.mp2_guess(b)[1])) - 0.05) < 1e-15


@pytest.fixture(scope="module")
def small_solution():
    prob, V = _problem(11, 4, 14)
    b = ccsd.Blocks(V, integrals.fock(prob), 4)
    out = ccsd.solve(b, tol=1e-11, max_iter=200)
    return prob, V, b, out


def test_converged_amplitudes_antisymmetric(small_solution):
    _, _, b, (t1, t2, E, nit, conv, _) = small_solution
    assert conv
    np.testing.assert_allclose(t2, -t2.swapaxes(0, 1), atol=1e-15)
    np.testing.assert_allclose(t2, -t2.swapaxes(2, 3), atol=1e-15)
    r1, r2 = ccsd.residual(t1, t2, b)
    assert np.max(np.abs(r2)) < 1e-9 and np.max(np.abs(r1)) < 1e-9


def test_diis_subspace_does_not_change_the_fixed_point(small_solution):
    """Plain Jacobi diverges on these Hamiltonians; DIIS(4) and DIIS(6) must agree."""
    _, _, b, (_, _, E, _, _, _) = small_solution
    _, _, E4, _, conv, _ = ccsd.solve(b, tol=1e-11, max_iter=400, diis_dim=4)
    assert conv
    assert abs(E - E4) < 1e-10


def test_diis_solve_matches_lstsq(rng):
    errs = [rng.standard_normal(50) + 1j * rng.standard_normal(50) for _ in range(6)]
    d = ccsd.DIIS(6)
    for e in errs:
        d.push(np.zeros(50, complex), e)
    c = d.coefficients()
    m = len(errs)
    B = np.array([[np.real(np.vdot(a, b_)) for b_ in errs] for a in errs])
    A = np.block([[B, -np.ones((m, 1))], [-np.ones((1, m)), np.zeros((1, 1))]])
    y = np.zeros(m + 1)
    y[m] = -1
    ref = np.linalg.lstsq(A, y, rcond=None)[0][:m]
    np.testing.assert_allclose(c, ref, rtol=1e-10, atol=1e-12)
    assert abs(c.sum() - 1) < 1e-13


def test_real_integrals_give_real_energy():
    prob = syn.make_problem(13, 4, 12)
    V = integrals.integrals(prob).real.astype(complex)
    b = ccsd.Blocks(V, integrals.fock(prob), 4)
    t1, t2, E, _, conv, _ = ccsd.solve(b, tol=1e-11)
    assert conv
    assert abs(E.imag) < 1e-12
    assert np.max(np.abs(t2.imag)) < 1e-14


def test_gauge_rotated_real_instance():
    """V'_pqrs = e^{i(th_p+th_q-th_r-th_s)} V_pqrs with real V: same E, Im E ~ 0."""
    prob = syn.make_problem(17, 4, 12)
    V = integrals.integrals(prob).real.astype(complex)
    b = ccsd.Blocks(V, integrals.fock(prob), 4)
    E_real = ccsd.solve(b, tol=1e-11)[2]
    th = np.random.default_rng(3).uniform(0, 2 * np.pi, prob.n)
    ph = np.exp(1j * th)
    Vg = V * (ph[:, None, None, None] * ph[None, :, None, None]
              * ph.conj()[None, None, :, None] * ph.conj()[None, None, None, :])
    bg = ccsd.Blocks(Vg, integrals.fock(prob), 4)
    E_g = ccsd.solve(bg, tol=1e-11)[2]
    assert abs(E_g - E_real) < 1e-12
    assert abs(E_g.imag) < 1e-12


@pytest.mark.parametrize("seed,no,nv,G", [(19, 4, 12, 4), (1604, 8, 32, 16)])
def test_symmetry_blocked_equals_c1_and_forbidden_stay_zero(seed, no, nv, G):
    """A Z_G problem solved densely (Z16: most irreps hold no occupied spinor): amplitudes
    of forbidden blocks stay exactly 0, and the result equals the same Hamiltonian with
    the labels ignored (C1)."""
    prob = syn.make_problem(seed, no, nv, G=G)
    V = integrals.integrals(prob)
    f = integrals.fock(prob)
    b = ccsd.Blocks(V, f, no)
    t1, t2, E, _, conv, _ = ccsd.solve(b, tol=1e-11)
    assert conv
    g = prob.irrep_of
    go, gv = g[:no], g[no:]
    forb1 = (gv[None, :] - go[:, None]) % G != 0
    forb2 = (gv[None, None, :, None] + gv[None, None, None, :]
             - go[:, None, None, None] - go[None, :, None, None]) % G != 0
    assert np.any(forb2)
    assert np.all(t1[forb1] == 0) and np.all(t2[forb2] == 0)
    # spinor order permuted (labels ignored): the same physics in C1 ordering
    perm_o = np.random.default_rng(1).permutation(no)
    perm_v = np.random.default_rng(2).permutation(nv)
    perm = np.concatenate([perm_o, no + perm_v])
    Vp = V[np.ix_(perm, perm, perm, perm)]
    fp = f[np.ix_(perm, perm)]
    Ep = ccsd.solve(ccsd.Blocks(Vp, fp, no), tol=1e-11)[2]
    assert abs(Ep - E) < 1e-12
