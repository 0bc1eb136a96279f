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


def _attached_block(H, no, nv, labels):
    """The matrix of H.sigma on the brute-force basis {a+|0>, a+ b+ j|0> (a<b)}, column by column."""
    n = len(labels)
    M = np.zeros((n, n), dtype=np.complex128)
    for c, l in enumerate(labels):
        r1 = np.zeros((1, nv), dtype=np.complex128)
        r2 = np.zeros((1, no, nv, nv), dtype=np.complex128)
        if l[0] == "p":
            r1[0, l[1]] = 1.0
        else:
            r2[0, l[1], l[2], l[3]], r2[0, l[1], l[3], l[2]] = 1.0, -1.0
        s1, s2 = H.sigma(r1, r2)
        M[:, c] = [s1[0, q[1]] if q[0] == "p" else s2[0, q[1], q[2], q[3]] for q in labels]
    return M


def _general_fock(f, seed):
    """f plus a small Hermitian perturbation with occupied-virtual and off-diagonal parts."""
    rng = np.random.default_rng(seed)
    n = f.shape[0]
    X = 0.01 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    return f + X + X.conj().T


@pytest.mark.parametrize("seed,no,nv,G,general_f", [(43, 2, 4, 1, False), (42, 1, 5, 1, False), (61, 2, 6, 4, False),
                                                    (43, 2, 4, 1, True)])
def test_sigma_equations_equal_brute_force_attached_block(seed, no, nv, G, general_f):
    """Every element of the electron-attached block of Hbar - E_CC: the sigma equations
    (each block: 1p<-1p, 1p<-2p1h, 2p1h<-1p, 2p1h<-2p1h) against explicit second
    quantisation in the (o+1)-electron determinant space, with converged T.  The Z4
    case has forbidden blocks; the general-Fock case exercises the f_ov, off-diagonal
    f_oo and f_vv terms."""
    prob = syn.make_problem(seed, no, nv, G)
    V = 0.02 * integrals.unscaled_integrals(prob) if no == 1 else integrals.integrals(prob)
    f = integrals.fock(prob)
    if general_f:
        f = _general_fock(f, 5)
    b = ccsd.Blocks(V, f, no)
    t1, t2, E, _, conv, _ = ccsd.solve(b, tol=1e-12, max_iter=600)
    assert conv
    if no > 1:
        assert np.max(np.abs(t1)) > 1e-6  # the T1 terms of every element take part
    M, labels = bf.ea_eom_matrix(f, V, no, t1, t2)
    got = _attached_block(fs0h1p.HbarEA(b, t1, t2), no, nv, labels)
    # converged to 1e-12: the brute-force block also holds r_a R1_j^b with the singles
    # residual R1 ~ 1e-12, well inside the tolerance
    np.testing.assert_allclose(got, M, atol=1e-12 * np.max(np.abs(M)), rtol=0)


def test_sigma_equations_on_random_attached_vectors(rng):
    """The batched sigma on random (antisymmetrised) vectors equals the brute-force block
    times those vectors."""
    prob, V, f, t1, t2 = _converged(43, 2, 4)
    nv = 4
    M, labels = bf.ea_eom_matrix(f, V, 2, t1, t2)
    H = fs0h1p.HbarEA(ccsd.Blocks(V, f, 2), t1, t2)
    r1 = rng.standard_normal((2, nv)) + 1j * rng.standard_normal((2, nv))
    x = rng.standard_normal((2, 2, nv, nv)) + 1j * rng.standard_normal((2, 2, nv, nv))
    r2 = x - x.transpose(0, 1, 3, 2)
    s1, s2 = H.sigma(r1, r2)
    for k in range(2):
        vec = np.array([r1[k, l[1]] if l[0] == "p" else r2[k, l[1], l[2], l[3]] for l in labels])
        out = M @ vec
        got = np.array([s1[k, l[1]] if l[0] == "p" else s2[k, l[1], l[2], l[3]] for l in labels])
        np.testing.assert_allclose(got, out, atol=1e-12 * np.max(np.abs(out)), rtol=0)
        # sigma keeps the antisymmetry of the 2p1h part
        np.testing.assert_allclose(s2[k], -s2[k].transpose(0, 2, 1), atol=1e-14 * np.max(np.abs(s2)))


def test_sigma_detects_a_planted_sign_error():
    """Control: the pin above is sharp enough to see a plausible slip (the sign of the
    three-body term flipped) in the oracle's arithmetic."""
    prob, V, f, t1, t2 = _converged(43, 2, 4)
    M, labels = bf.ea_eom_matrix(f, V, 2, t1, t2)
    H = fs0h1p.HbarEA(ccsd.Blocks(V, f, 2), t1, t2)
    H.t2 = -H.t2  # only the three-body term reads t2 directly
    got = _attached_block(H, 2, 4, labels)
    assert np.max(np.abs(got - M)) > 1e-6 * np.max(np.abs(M))


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
    # the Bloch iteration's own stopping point: DIIS(6) reaches max |ds| ~ 2e-11 and
    # wanders there (rounding amplified by a near-singular DIIS matrix), so the solve
    # stops at 1e-11; the eigenvalues then sit within 1e-12 of the brute-force spectrum
    Heff, w, _, _, nit, conv = fs0h1p.solve(V, f, 2, t1, t2, act, tol=1e-11, max_iter=300)
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
