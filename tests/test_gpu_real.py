"""GPU parity for the real-arithmetic path (exp_config.real_arith; the paper's real double
groups, Sec. II.C): the real part of the integral recipe, real emulated products (A' = Re A,
one B row per output column), complex storage with zero imaginary parts.  Against the
oracle on the real recipe (oracle.integrals.real_integrals):

  * the MP2 guess element by element (the generator and the scale);
  * the first two iterates element by element, FP64 (1e-12) and with every product above
    1e3 complex MACs emulated in real arithmetic (5 slices, 1e-9);
  * converged energies (FP64 1e-10 Eh, emulated 1e-8 Eh) with imaginary parts exactly 0."""
import numpy as np
import pytest

from oracle import ccsd, integrals
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


def _oracle(prob):
    return ccsd.Blocks(integrals.real_integrals(prob), integrals.fock(prob), prob.n_occ)


@pytest.mark.parametrize("no,nv,G", [(4, 12, 2), (6, 20, 4), (10, 40, 1)])
def test_real_mp2_guess_matches_oracle(expgb, no, nv, G):
    prob = syn.make_problem(500 + no + nv + G, no, nv, G)
    b = _oracle(prob)
    ctx = expgb.from_problems([prob], real_arith=True)
    ctx.init_integrals([prob.seed])
    ctx.iterate(0)
    t1, t2 = ctx.get_amplitudes(0)
    r1, r2 = ccsd.mp2_guess(b)
    np.testing.assert_allclose(t2.cpu().numpy(), r2, atol=1e-14, rtol=0)
    assert np.max(np.abs(t2.cpu().numpy().imag)) == 0.0
    ctx.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
@pytest.mark.parametrize("no,nv,G", [(4, 12, 2), (6, 20, 4), (10, 40, 1)])
def test_real_first_iterations_elementwise(expgb, no, nv, G, precision, tol):
    prob = syn.make_problem(600 + no + nv + G, no, nv, G)
    b = _oracle(prob)
    ctx = expgb.from_problems([prob], diis_dim=0, real_arith=True, precision=precision, n_slices=5,
                              emu_min_macs=1e3)
    ctx.init_integrals([prob.seed])
    t1, t2 = ccsd.mp2_guess(b)
    D1, D2 = ccsd.denominators(b)
    for it in range(2):
        ctx.iterate(1)
        r1, r2 = ccsd.rhs(t1, t2, b)
        t1, t2 = r1 / D1, r2 / D2
        g1, g2 = (x.cpu().numpy() for x in ctx.get_amplitudes(0))
        scale = max(np.max(np.abs(t2)), 1e-3)
        np.testing.assert_allclose(g1, t1, atol=tol * scale, rtol=0)
        np.testing.assert_allclose(g2, t2, atol=tol * scale, rtol=0)
        assert np.max(np.abs(g2.imag)) == 0.0 and np.max(np.abs(g1.imag)) == 0.0
    ctx.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-8)])
def test_real_converged_energy(expgb, precision, tol):
    prob = syn.make_problem(33, 4, 12, 2)
    E = ccsd.solve(_oracle(prob), tol=1e-12, max_iter=600)[2]
    assert abs(E.imag) < 1e-14
    ctx = expgb.from_problems([prob], conv_tol=1e-11, max_iter=600, real_arith=True, precision=precision,
                              n_slices=5, emu_min_macs=1e3)
    ctx.init_integrals([prob.seed])
    _, conv, _ = ctx.iterate(600)
    assert conv
    e = ctx.energy(0)
    assert e.imag == 0.0
    assert abs(e - E) < tol
    ctx.close()
