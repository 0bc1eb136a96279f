"""GPU parity for the (0h,2p) Fock-space sector (exp_fs_sector_0h2p) against
oracle/fs0h2p.py.

  * Tiny problems against the determinant-basis Bloch equation (oracle.fs0h2p.solve):
    the H_eff eigenvalues within 1e-9 and |H_eff| element by element within 1e-9 (the
    pair-basis signs of the two constructions may differ).
  * Larger problems (o=6 v=20 Z4 and o=6 v=18 Z2) against the ghost-spinor construction
    (oracle.fs0h2p.solve_ghost, itself pinned to the determinant basis): FP64 within
    1e-9, the emulated path within 1e-7.
  * Fewer than two active spinors: ESTATE."""
import numpy as np
import pytest

from oracle import ccsd, fs0h1p, fs0h2p, integrals
from paper_2004_03682_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def expgb():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2004_03682_gb300 import build, expgb as e
    build.build()
    e.lib()
    return e


def _oracle_sectors(prob, act):
    V, f = integrals.integrals(prob), integrals.fock(prob)
    no = prob.n_occ
    t1, t2, E, _, conv, _ = ccsd.solve(ccsd.Blocks(V, f, no), tol=1e-12, max_iter=800)
    assert conv
    H1, w1, s1, s2, _, conv = fs0h1p.solve(V, f, no, t1, t2, act, tol=1e-12, max_iter=800)
    assert conv
    return V, f, t1, t2, E, s1, s2


def _gpu_sector(expgb, prob, act, precision=0):
    ctx = expgb.from_problems([prob], conv_tol=1e-11, max_iter=800, active=act, precision=precision,
                              n_slices=6, emu_min_macs=1e3)
    ctx.init_integrals([prob.seed])
    _, conv, _ = ctx.iterate(800)
    assert conv
    _, _, _, st1 = ctx.fs_sector_0h1p(0)
    assert st1 == 0
    H, w, nit, st = ctx.fs_sector_0h2p(0)
    ctx.close()
    assert st == 0, (st, nit)
    return H, w


@pytest.mark.parametrize("seed,no,nv,G,nact", [(911, 2, 5, 1, 2), (916, 2, 6, 2, 3), (918, 3, 6, 2, 2),
                                               (921, 2, 6, 4, 3)])
def test_0h2p_matches_determinant_oracle(expgb, seed, no, nv, G, nact):
    prob = syn.make_problem(seed, no, nv, G)
    act = np.argsort(prob.eps_virt)[:nact]
    V, f, t1, t2, E, s1, s2 = _oracle_sectors(prob, act)
    Ho, wo, s, pairs, qp, nit, conv = fs0h2p.solve(V, f, no, t1, t2, E, act, s1, s2, tol=1e-11, max_iter=800)
    assert conv
    Hg, wg = _gpu_sector(expgb, prob, act)
    np.testing.assert_allclose(wg, wo, atol=1e-9, rtol=0)
    np.testing.assert_allclose(np.abs(Hg), np.abs(Ho), atol=1e-9, rtol=0)


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-7)])
@pytest.mark.parametrize("seed,no,nv,G,nact", [(933, 6, 20, 4, 3), (934, 6, 18, 2, 4)])
def test_0h2p_matches_ghost_oracle(expgb, seed, no, nv, G, nact, precision, tol):
    prob = syn.make_problem(seed, no, nv, G)
    act = np.argsort(prob.eps_virt)[:nact]
    V, f, t1, t2, E, s1, s2 = _oracle_sectors(prob, act)
    Ho, wo, conv = fs0h2p.solve_ghost(V, f, no, t1, t2, act, s1, s2, tol=1e-11, max_iter=800)
    assert conv
    Hg, wg = _gpu_sector(expgb, prob, act, precision)
    np.testing.assert_allclose(wg, wo, atol=tol, rtol=0)


def test_0h2p_needs_two_active_spinors(expgb):
    prob = syn.make_problem(941, 4, 12, 2)
    act = np.argsort(prob.eps_virt)[:1]
    ctx = expgb.from_problems([prob], conv_tol=1e-10, max_iter=400, active=act)
    ctx.init_integrals([prob.seed])
    ctx.iterate(400)
    with pytest.raises(expgb.ExpError) as ei:
        ctx.fs_sector_0h2p(0)
    assert ei.value.status == expgb.EXP_ESTATE
    ctx.close()
