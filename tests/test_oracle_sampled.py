"""Pins for oracle/sampled.py: the integral slices and the per-element right-hand
sides agree with the dense oracle (oracle.integrals, oracle.ccsd) everywhere on
small problems, away from the MP2 guess (t1 != 0)."""
import itertools

import numpy as np
import pytest

from oracle import ccsd, integrals, sampled
from paper_2004_03682_gb300 import synthetic as syn


@pytest.mark.parametrize("no,nv,G", [(3, 7, 1), (4, 10, 2), (4, 11, 3)])
def test_vblock_matches_dense_integrals(no, nv, G):
    prob = syn.make_problem(900 + no + nv + G, no, nv, G)
    V = integrals.unscaled_integrals(prob)
    rng = np.random.default_rng(1)
    for _ in range(4):
        idx = [rng.choice(prob.n, size=rng.integers(1, 5), replace=False) for _ in range(4)]
        np.testing.assert_allclose(sampled.vblock(prob, *idx), V[np.ix_(*idx)], atol=1e-14, rtol=0)
    I = sampled.Integrals(prob)
    assert abs(I.s - integrals.mp2_scale(V, prob) * prob.scale_mult) < 1e-15 * I.s


@pytest.mark.parametrize("no,nv,G", [(3, 8, 1), (4, 10, 2), (5, 12, 4)])
def test_rhs_elements_match_dense_rhs(no, nv, G):
    prob = syn.make_problem(950 + no + nv + G, no, nv, G)
    b = ccsd.Blocks(integrals.integrals(prob), integrals.fock(prob), no)
    t1, t2 = syn.trial_amplitudes(prob, 3)
    r1, r2 = ccsd.rhs(t1, t2, b)
    irr = prob.irrep_of
    s2 = [(i, j, a, b_) for i, j, a, b_ in itertools.product(range(no), range(no), range(nv), range(nv))
          if (irr[i] + irr[j] - irr[no + a] - irr[no + b_]) % G == 0]
    rng = np.random.default_rng(2)
    s2 = [s2[k] for k in rng.choice(len(s2), size=min(40, len(s2)), replace=False)]
    s1 = [(i, a) for i in range(no) for a in range(nv) if irr[i] == irr[no + a]][:12]
    g2, g1 = sampled.rhs_elements(prob, t1, t2, s2, s1)
    scale = max(np.max(np.abs(r2)), 1e-3)
    np.testing.assert_allclose(g2, [r2[s] for s in s2], atol=1e-13 * scale, rtol=0)
    np.testing.assert_allclose(g1, [r1[s] for s in s1], atol=1e-13 * scale, rtol=0)
    assert np.max(np.abs(t1)) > 0  # the t1 terms are exercised
