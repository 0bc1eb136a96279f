"""Pins for the (T) oracle (oracle/triples.py) against explicit second quantisation."""
import numpy as np
import pytest

import brute_force as bf
from oracle import ccsd, integrals, triples
from paper_2004_03682_gb300 import synthetic as syn


def _random_t(rng, no, nv, prob, scale=0.05):
    t1 = 0.01 * (rng.standard_normal((no, nv)) + 1j * rng.standard_normal((no, nv)))
    x = rng.standard_normal((no, no, nv, nv)) + 1j * rng.standard_normal((no, no, nv, nv))
    t2 = scale * (x - x.transpose(1, 0, 2, 3) - x.transpose(0, 1, 3, 2) + x.transpose(1, 0, 3, 2))
    irr = prob.irrep_of
    go, gv = irr[:no], irr[no:]
    t1 = t1 * (go[:, None] == gv[None, :])
    t2 = t2 * ((go[:, None, None, None] + go[None, :, None, None] - gv[None, None, :, None]
                - gv[None, None, None, :]) % prob.G == 0)
    return t1, t2


@pytest.mark.parametrize("no,nv,G", [(3, 4, 1), (3, 5, 1), (4, 4, 2)])
def test_triples_energy_equals_brute_force(no, nv, G):
    """Random t1, t2 (the formula holds for any amplitudes): every sign and factor of the
    connected and disconnected triples, through the energy sum."""
    rng = np.random.default_rng(no * 10 + nv + G)
    prob = syn.make_problem(700 + no + nv + G, no, nv, G)
    V, f = integrals.integrals(prob), integrals.fock(prob)
    t1, t2 = _random_t(rng, no, nv, prob)
    E = triples.energy(t1, t2, ccsd.Blocks(V, f, no))
    Ebf = bf.triples_energy(f, V, no, t1, t2)
    assert abs(Ebf) > 1e-8
    assert abs(E - Ebf) < 1e-12 * max(1.0, abs(Ebf))


def test_triples_vanish_for_two_electrons():
    prob = syn.make_problem(71, 2, 6, 1)
    V, f = integrals.integrals(prob), integrals.fock(prob)
    b = ccsd.Blocks(V, f, 2)
    t1, t2, E, _, conv, _ = ccsd.solve(b, tol=1e-11)
    assert abs(triples.energy(t1, t2, b)) < 1e-15  # every term has a repeated occupied index


def test_triples_are_antisymmetric():
    rng = np.random.default_rng(3)
    prob = syn.make_problem(77, 4, 6, 1)
    V, f = integrals.integrals(prob), integrals.fock(prob)
    t1, t2 = _random_t(rng, 4, 6, prob)
    c, d = triples.triples(t1, t2, ccsd.Blocks(V, f, 4))
    for x in (c, d):
        np.testing.assert_allclose(x, -x.transpose(1, 0, 2, 3, 4, 5), atol=1e-15)
        np.testing.assert_allclose(x, -x.transpose(0, 2, 1, 3, 4, 5), atol=1e-15)
        np.testing.assert_allclose(x, -x.transpose(0, 1, 2, 4, 3, 5), atol=1e-15)
        np.testing.assert_allclose(x, -x.transpose(0, 1, 2, 3, 5, 4), atol=1e-15)


def test_sign_slip_is_caught():
    """Control: flipping the sign of the disconnected term moves the energy."""
    rng = np.random.default_rng(5)
    prob = syn.make_problem(703, 3, 5, 1)
    V, f = integrals.integrals(prob), integrals.fock(prob)
    t1, t2 = _random_t(rng, 3, 5, prob)
    b = ccsd.Blocks(V, f, 3)
    c, d = triples.triples(t1, t2, b)
    D = triples.denominators3(b)
    E_wrong = complex(np.sum(np.conj(c - d) * c / D) / 36.0)
    Ebf = bf.triples_energy(f, V, 3, t1, t2)
    assert abs(E_wrong - Ebf) > 1e-6 * abs(Ebf)


@pytest.mark.parametrize("no,nv,G", [(4, 6, 1), (5, 8, 2)])
def test_per_triple_energies_sum_to_the_energy(no, nv, G):
    """The split over occupied triples is exact, and only i<j<k carry energy."""
    rng = np.random.default_rng(no + nv + G)
    prob = syn.make_problem(720 + no + nv + G, no, nv, G)
    V, f = integrals.integrals(prob), integrals.fock(prob)
    b = ccsd.Blocks(V, f, no)
    t1, t2 = _random_t(rng, no, nv, prob)
    e = triples.per_triple(t1, t2, b)
    E = triples.energy(t1, t2, b)
    assert abs(np.sum(e) - E) < 1e-14 * max(1.0, abs(E))
    for i in range(no):
        for j in range(no):
            for k in range(no):
                if not (i < j < k):
                    assert e[i, j, k] == 0
    assert np.count_nonzero(e) > 0


@pytest.mark.parametrize("no,nv,G", [(4, 7, 1), (5, 9, 2), (6, 10, 4)])
def test_sampled_triple_energy_matches_dense(no, nv, G):
    """One triple from generated integral slices equals the dense per-triple energy, for
    every i<j<k (the slice generator is itself pinned to the dense integrals)."""
    from oracle import sampled
    rng = np.random.default_rng(10 * no + nv + G)
    prob = syn.make_problem(730 + no + nv + G, no, nv, G)
    V, f = integrals.integrals(prob), integrals.fock(prob)
    b = ccsd.Blocks(V, f, no)
    t1, t2 = _random_t(rng, no, nv, prob)
    e = triples.per_triple(t1, t2, b)
    ints = sampled.Integrals(prob)
    for i in range(no):
        for j in range(i + 1, no):
            for k in range(j + 1, no):
                ek = triples.triple_energy(prob, ints, t1, t2, i, j, k)
                assert abs(ek - e[i, j, k]) < 1e-14 + 1e-12 * abs(e[i, j, k])
