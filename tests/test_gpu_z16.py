"""GPU parity on Z16 problems, the symmetry group of the (0h,1p) production shape
(o=80 v=480 Z16, whose dense amplitudes are too large for a host-side oracle): the same
kernels on a small Z16 problem (o=8 v=32, most irreps holding zero, one or two occupied
spinors), element by element against the oracle.

  * (0h,0p): the first two Jacobi iterates, every amplitude, full pairs and packed pairs
    (FP64, 1e-12 of max|t2|); the emulated path (six slices, every product on the tensor
    cores) to convergence, energy within 1e-9 Eh of the oracle's fixed point.
  * (0h,1p): H_eff element by element and its eigenvalues within 1e-9 (four active
    spinors, in distinct and in shared irreps).
  * (0h,2p): pair eigenvalues against the ghost-spinor oracle, FP64 1e-9 and emulated 1e-7."""
import numpy as np
import pytest

from oracle import ccsd, fs0h1p, fs0h2p, integrals
from paper_2004_03682_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

NO, NV, G = 8, 32, 16


@pytest.fixture(scope="module")
def expgb():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2004_03682_gb300 import build, expgb as e
    build.build()
    e.lib()
    return e


def _blocks(prob):
    V, f = integrals.integrals(prob), integrals.fock(prob)
    return V, f, ccsd.Blocks(V, f, prob.n_occ)


@pytest.mark.parametrize("packed", [False, True])
@pytest.mark.parametrize("seed", [1602, 1608])
def test_z16_first_iterations_elementwise(expgb, seed, packed):
    prob = syn.make_problem(seed, NO, NV, G)
    assert np.count_nonzero(prob.irrep_occ == 0) >= 6     # empty occupied irreps
    _, _, b = _blocks(prob)
    ctx = expgb.from_problems([prob], diis_dim=0, packed=packed)
    ctx.init_integrals([prob.seed])
    t1, t2 = ccsd.mp2_guess(b)
    D1, D2 = ccsd.denominators(b)
    for _ in range(2):
        ctx.iterate(1)
        r1, r2 = ccsd.rhs(t1, t2, b)
        t1, t2 = r1 / D1, r2 / D2
        g1, g2 = ctx.get_amplitudes(0)
        scale = max(np.max(np.abs(t2)), 1e-3)
        np.testing.assert_allclose(g1.cpu().numpy(), t1, atol=1e-12 * scale, rtol=0)
        np.testing.assert_allclose(g2.cpu().numpy(), t2, atol=1e-12 * scale, rtol=0)
        assert abs(ctx.energy(0) - ccsd.energy(t1, t2, b)) < 1e-11
    ctx.close()


def test_z16_emulated_converged_energy(expgb):
    prob = syn.make_problem(1604, NO, NV, G)
    _, _, b = _blocks(prob)
    E = ccsd.solve(b, tol=1e-12, max_iter=400)[2]
    ctx = expgb.from_problems([prob], conv_tol=1e-11, max_iter=400, precision=expgb.EXP_EMU_BF16,
                              n_slices=6, emu_min_macs=1e3, packed=True)
    ctx.init_integrals([prob.seed])
    _, conv, _ = ctx.iterate(400)
    assert conv
    assert abs(ctx.energy(0) - E) < 1e-9
    ctx.close()


@pytest.mark.parametrize("seed", [1601, 1604])
def test_z16_0h1p_matches_oracle(expgb, seed):
    prob = syn.make_problem(seed, NO, NV, G)
    act = syn.active_virtuals(prob, 4)
    V, f, b = _blocks(prob)
    t1, t2, E, _, conv, _ = ccsd.solve(b, tol=1e-12, max_iter=400)
    assert conv
    H, w, _, _, _, conv = fs0h1p.solve(V, f, NO, t1, t2, act, tol=1e-11, max_iter=400)
    assert conv
    ctx = expgb.from_problems([prob], conv_tol=1e-11, max_iter=400, active=act)
    ctx.init_integrals([prob.seed])
    _, conv, _ = ctx.iterate(400)
    assert conv
    assert abs(ctx.energy(0) - E) < 1e-10
    Hg, wg, _, st = ctx.fs_sector_0h1p(0)
    ctx.close()
    assert st == 0
    np.testing.assert_allclose(Hg, H, atol=1e-9, rtol=0)
    np.testing.assert_allclose(wg, w, atol=1e-9, rtol=0)


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-7)])
def test_z16_0h2p_matches_ghost_oracle(expgb, precision, tol):
    prob = syn.make_problem(1604, NO, NV, G)
    act = np.argsort(prob.eps_virt)[:3]
    V, f, b = _blocks(prob)
    t1, t2, _, _, conv, _ = ccsd.solve(b, tol=1e-12, max_iter=800)
    assert conv
    _, _, s1, s2, _, conv = fs0h1p.solve(V, f, NO, t1, t2, act, tol=1e-12, max_iter=800)
    assert conv
    _, wo, conv = fs0h2p.solve_ghost(V, f, NO, t1, t2, act, s1, s2, tol=1e-11, max_iter=800)
    assert conv
    ctx = expgb.from_problems([prob], conv_tol=1e-11, max_iter=800, active=act, precision=precision,
                              n_slices=6, emu_min_macs=1e3)
    ctx.init_integrals([prob.seed])
    _, conv, _ = ctx.iterate(800)
    assert conv
    assert ctx.fs_sector_0h1p(0)[3] == 0
    _, wg, nit, st = ctx.fs_sector_0h2p(0)
    ctx.close()
    assert st == 0, (st, nit)
    np.testing.assert_allclose(wg, wo, atol=tol, rtol=0)
