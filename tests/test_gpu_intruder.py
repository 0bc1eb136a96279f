"""GPU parity for the intruder-state denominator shift (exp_config.denom_shift, both
sectors) and the zero-shift extrapolation, against oracle/intruder.py:

  * (0h,0p): the shifted CCSD energy (guess V/D~, t = RHS/D~) within 1e-10 Eh;
  * (0h,1p): H_eff eigenvalues of the shifted Bloch equation within 1e-9, on a
    well-conditioned Z4 case and on an intruder case whose unshifted iteration runs away;
  * the Pade-extrapolated energy of GPU solves at three shifts lands much closer to the
    unshifted GPU energy than the smallest shift, and exp_pade_zero of those values
    equals the oracle's fit of them."""
import numpy as np
import pytest

from oracle import ccsd, integrals, intruder
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


def _gpu_energy(expgb, prob, s, n, tol=1e-11):
    ctx = expgb.from_problems([prob], conv_tol=tol, max_iter=600, denom_shift=s, denom_shift_n=n)
    ctx.init_integrals([prob.seed])
    _, conv, _ = ctx.iterate(600)
    assert conv
    e = ctx.energy(0)
    ctx.close()
    return e


@pytest.mark.parametrize("seed,no,nv,G", [(11, 4, 14, 1), (306, 6, 20, 4)])
def test_shifted_ccsd_energy_matches_oracle(expgb, seed, no, nv, G):
    prob = syn.make_problem(seed, no, nv, G)
    b = ccsd.Blocks(integrals.integrals(prob), integrals.fock(prob), no)
    E = intruder.ccsd_shifted(b, 0.3, 2, tol=1e-12)[2]
    assert abs(_gpu_energy(expgb, prob, 0.3, 2) - E) < 1e-10


def test_extrapolated_gpu_energy_approaches_unshifted(expgb):
    prob = syn.make_problem(11, 4, 14, 1)
    E0 = _gpu_energy(expgb, prob, 0.0, 1)
    xs = [0.1, 0.2, 0.3]
    Es = [_gpu_energy(expgb, prob, x, 2) for x in xs]
    ys = [x ** 3 for x in xs]
    ext = expgb.pade_zero(ys, Es, 1, 1)
    # the fit's rows are Vandermonde-like in s^3 (1e-3 .. 3e-2): two solvers agree to about
    # cond x 1e-16
    assert abs(ext - intruder.pade_zero(ys, Es, 1, 1)) < 1e-10 * abs(ext)
    assert abs(ext - E0) < abs(Es[0] - E0) / 10


def _fs_case(expgb, prob, act, s, n):
    V, f = integrals.integrals(prob), integrals.fock(prob)
    b = ccsd.Blocks(V, f, prob.n_occ)
    t1, t2, E, _, conv = intruder.ccsd_shifted(b, s, n, tol=1e-11)
    assert conv
    H, w, _, _, nit, conv = intruder.fs_shifted(V, f, prob.n_occ, t1, t2, act, s, n, tol=1e-10, max_iter=300)
    assert conv
    ctx = expgb.from_problems([prob], conv_tol=1e-11, max_iter=400, active=act, denom_shift=s, denom_shift_n=n)
    ctx.init_integrals([prob.seed])
    _, conv, _ = ctx.iterate(400)
    assert conv
    assert abs(ctx.energy(0) - E) < 1e-10
    Hg, wg, nit_g, st = ctx.fs_sector_0h1p(0)
    ctx.close()
    assert st == 0
    np.testing.assert_allclose(Hg, H, atol=1e-9, rtol=0)
    np.testing.assert_allclose(wg, w, atol=1e-9, rtol=0)


def test_shifted_fs_sector_matches_oracle(expgb):
    prob = syn.make_problem(306, 6, 20, 4)
    _fs_case(expgb, prob, syn.active_virtuals(prob, 4), 0.3, 2)


def test_shifted_fs_sector_on_an_intruder_case(expgb):
    """The active spinor is the 13th lowest of 20 virtuals: 68 positive D_xj^ab."""
    prob = syn.make_problem(306, 6, 20, 4)
    x = int(np.argsort(prob.eps_virt)[12])
    _fs_case(expgb, prob, np.array([x]), 2.0, 1)
