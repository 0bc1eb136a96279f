"""GPU parity for the (0h,1p) sector: H_eff and its eigenvalues against the oracle."""
import dataclasses

import numpy as np
import pytest

import brute_force as bf
from oracle import ccsd, fs0h1p, integrals
from paper_2004_03682_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def expgb():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    from paper_2004_03682_gb300 import build, expgb as e
    build.build()
    e.lib()
    return e


def _oracle(prob, act, tol=1e-10):
    V = integrals.integrals(prob)
    f = integrals.fock(prob)
    t1, t2, E, _, conv, _ = ccsd.solve(ccsd.Blocks(V, f, prob.n_occ), tol=1e-11, max_iter=400)
    assert conv
    H, w, _, _, nit, conv = fs0h1p.solve(V, f, prob.n_occ, t1, t2, act, tol=tol, max_iter=300)
    assert conv
    return E, H, w, (V, f, t1, t2)


@pytest.mark.parametrize("seed,no,nv,G,na", [(306, 6, 20, 4, 4), (59, 2, 5, 1, 2)])
def test_fs_0h1p_matches_oracle(expgb, seed, no, nv, G, na):
    prob = syn.make_problem(seed, no, nv, G)
    act = syn.active_virtuals(prob, na)
    E, H, w, _ = _oracle(prob, act)
    ctx = expgb.from_problems([prob], conv_tol=1e-11, max_iter=400, active=act)
    ctx.init_integrals([prob.seed])
    _, conv, _ = ctx.iterate(400)
    assert conv
    assert abs(ctx.energy(0) - E) < 1e-10      # ghosts leave the (0h,0p) solution untouched
    Hg, wg, nit, st = ctx.fs_sector_0h1p(0)
    assert st == 0
    np.testing.assert_allclose(Hg, H, atol=1e-9, rtol=0)
    np.testing.assert_allclose(wg, w, atol=1e-9, rtol=0)


def test_fs_eigenvalues_in_brute_force_attached_spectrum(expgb):
    prob = syn.make_problem(61, 2, 5, 1)
    act = syn.active_virtuals(prob, 2)
    E, H, w, (V, f, t1, t2) = _oracle(prob, act, tol=1e-12)
    ctx = expgb.from_problems([prob], conv_tol=1e-12, max_iter=400, active=act)
    ctx.init_integrals([prob.seed])
    ctx.iterate(400)
    _, wg, _, st = ctx.fs_sector_0h1p(0)
    assert st == 0
    M, _ = bf.ea_eom_matrix(f, V, 2, t1, t2)
    ev = np.linalg.eigvals(M)
    for e in wg:
        assert np.min(np.abs(ev - e)) < 1e-9


def test_fs_batched_instances(expgb):
    base = [syn.make_problem(seed, 6, 20, 4) for seed in (306, 329)]
    probs = [dataclasses.replace(p, irrep_occ=base[0].irrep_occ, irrep_virt=base[0].irrep_virt) for p in base]
    act = syn.active_virtuals(probs[0], 4)
    ctx = expgb.from_problems(probs, conv_tol=1e-11, max_iter=400, active=act)
    ctx.init_integrals([p.seed for p in probs])
    _, conv, _ = ctx.iterate(400)
    assert conv
    for k, p in enumerate(probs):
        _, _, w, _ = _oracle(p, act)
        _, wg, _, st = ctx.fs_sector_0h1p(k)
        np.testing.assert_allclose(wg, w, atol=1e-9, rtol=0)


def test_fs_before_convergence_is_a_state_error(expgb):
    prob = syn.make_problem(306, 6, 20, 4)
    ctx = expgb.from_problems([prob], conv_tol=1e-11, max_iter=400, active=syn.active_virtuals(prob, 4))
    ctx.init_integrals([prob.seed])
    ctx.iterate(2)
    with pytest.raises(expgb.ExpError) as e:
        ctx.fs_sector_0h1p(0)
    assert e.value.status == 7
