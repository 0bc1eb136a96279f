"""Pins for the seeded generator and the oracle's integral recipe."""
import numpy as np

from oracle import integrals
from paper_2004_03682_gb300 import synthetic as syn


def test_philox_known_answers():
    """Philox4x32-10 known-answer vectors published with the Random123 library."""
    cases = [
        ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 4, (0xFFFFFFFF, 0xFFFFFFFF),
         (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for ctr, key, want in cases:
        got = syn.philox4x32_10(*ctr, *key)
        assert tuple(int(x) for x in got) == want


def test_gaussian_field_moments():
    z = syn.gaussian_field(np.arange(200_000), seed=99)
    assert abs(z.real.mean()) < 0.01 and abs(z.imag.mean()) < 0.01
    assert abs(z.real.var() - 1) < 0.02 and abs(z.imag.var() - 1) < 0.02
    assert abs(np.mean(z.real * z.imag)) < 0.01


def test_irrep_counts_sum_and_dirichlet():
    rng = np.random.default_rng(0)
    for G in (1, 4, 8, 16):
        c = syn.irrep_counts(200, G, rng)
        assert c.sum() == 200 and len(c) == G and np.all(c >= 0)


def test_recipe_symmetries_and_blocks():
    prob = syn.make_problem(3, 3, 7, G=4)
    V = integrals.integrals(prob)
    # exact up to the rounding of the four-term sums
    np.testing.assert_allclose(V, -V.transpose(1, 0, 2, 3), atol=1e-15, rtol=0)
    np.testing.assert_allclose(V, -V.transpose(0, 1, 3, 2), atol=1e-15, rtol=0)
    np.testing.assert_allclose(V, V.transpose(2, 3, 0, 1).conj(), atol=1e-17, rtol=0)
    mask = integrals.allowed_mask(prob.irrep_of, prob.G)
    assert np.all(V[~mask] == 0)
    assert np.count_nonzero(V[mask]) > 0.5 * mask.sum()


def test_elementwise_recipe_matches_dense():
    """Any single V_pqrs follows from 8 evaluations of A (index-addressable)."""
    prob = syn.make_problem(8, 3, 5, G=2)
    V = integrals.unscaled_integrals(prob)
    n, g = prob.n, prob.irrep_of
    rng = np.random.default_rng(4)
    for _ in range(20):
        p, q, r, s = rng.integers(0, n, 4)
        A = lambda a, b, c, d: syn.gaussian_tensor(prob.seed, n, [a], [b], [c], [d])[0, 0, 0, 0]
        x = A(p, q, r, s) - A(q, p, r, s) - A(p, q, s, r) + A(q, p, s, r)
        y = A(r, s, p, q) - A(s, r, p, q) - A(r, s, q, p) + A(s, r, q, p)
        v = 0.5 * (x + np.conj(y)) if (g[p] + g[q] - g[r] - g[s]) % prob.G == 0 else 0
        assert abs(V[p, q, r, s] - v) < 1e-14


def test_real_recipe_is_real_antisymmetric_symmetric_and_scaled():
    import numpy as np
    from oracle import integrals
    from paper_2004_03682_gb300 import synthetic as syn
    prob = syn.make_problem(31, 3, 7, 2)
    V = integrals.real_integrals(prob)
    assert np.max(np.abs(V.imag)) == 0.0
    tol = 1e-14 * np.max(np.abs(V))
    np.testing.assert_allclose(V, -V.transpose(1, 0, 2, 3), atol=tol, rtol=0)
    np.testing.assert_allclose(V, -V.transpose(0, 1, 3, 2), atol=tol, rtol=0)
    np.testing.assert_allclose(V, V.transpose(2, 3, 0, 1), atol=tol, rtol=0)
    o = prob.n_occ
    t = V[o:, o:, :o, :o].transpose(2, 3, 0, 1) / integrals.denominators2(prob.eps_occ, prob.eps_virt)
    assert abs(np.max(np.abs(t)) - 0.05) < 1e-15
    # the real part of the complex recipe, up to the scale
    Vc = integrals.unscaled_integrals(prob)
    ratio = V[np.abs(Vc.real) > 1e-3] / Vc.real[np.abs(Vc.real) > 1e-3]
    assert np.max(np.abs(ratio - ratio.flat[0])) < 1e-12


def test_real_ccsd_solution_is_real():
    import numpy as np
    from oracle import ccsd, integrals
    from paper_2004_03682_gb300 import synthetic as syn
    prob = syn.make_problem(33, 4, 12, 2)
    b = ccsd.Blocks(integrals.real_integrals(prob), integrals.fock(prob), 4)
    t1, t2, E, nit, conv, _ = ccsd.solve(b, tol=1e-11, max_iter=400)
    assert conv
    assert abs(E.imag) < 1e-14 and np.max(np.abs(t2.imag)) < 1e-14 and np.max(np.abs(t1.imag)) < 1e-14
