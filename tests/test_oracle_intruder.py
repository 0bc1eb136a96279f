"""Pins for the intruder-state shift and Pade extrapolation oracle (oracle/intruder.py)
against things other than itself: the unshifted method at s = 0, exact rational
functions, and the zero-shift limit of the shifted solutions on well-conditioned cases."""
import numpy as np
import pytest

from oracle import ccsd, fs0h1p, integrals, intruder
from paper_2004_03682_gb300 import synthetic as syn


def test_dynamic_shift_limits():
    D = np.array([-3.0, -1.0, -0.05, 0.0, 0.02, 0.4])
    assert np.array_equal(intruder.dynamic_shift(D, 0.0, 2), D)
    s = 0.5
    Ds = intruder.dynamic_shift(D, s, 2)
    # near-zero denominators move by about -s, large ones by s (s/|D|)^2 at most
    assert abs((Ds[3] - D[3]) + s) < 1e-15
    assert np.all(Ds < D)
    assert abs(Ds[0] - D[0]) < s * (s / 3.0) ** 2 + 1e-15
    # a denominator of the unshifted sign moves away from zero
    assert np.all(Ds[:3] < D[:3])


@pytest.mark.parametrize("L,M", [(1, 1), (2, 1), (1, 2), (3, 0)])
def test_pade_reproduces_rational_function_of_its_degree(L, M):
    rng = np.random.default_rng(L * 10 + M)
    a = rng.standard_normal(L + 1) + 1j * rng.standard_normal(L + 1)
    b = 0.3 * (rng.standard_normal(M) + 1j * rng.standard_normal(M))

    def f(x):
        return sum(a[j] * x ** j for j in range(L + 1)) / (1 + sum(b[j - 1] * x ** j for j in range(1, M + 1)))
    x = np.linspace(0.1, 0.6, L + M + 1)
    assert abs(intruder.pade_zero(x, f(x), L, M) - a[0]) < 1e-10 * abs(a[0])
    # more points than unknowns: least squares, still exact
    x2 = np.linspace(0.1, 0.7, L + M + 4)
    assert abs(intruder.pade_zero(x2, f(x2), L, M) - a[0]) < 1e-9 * abs(a[0])


def test_zero_shift_is_the_unshifted_ccsd():
    prob = syn.make_problem(11, 4, 14, 1)
    b = ccsd.Blocks(integrals.integrals(prob), integrals.fock(prob), 4)
    E0 = ccsd.solve(b, tol=1e-11, max_iter=600)[2]
    Es = intruder.ccsd_shifted(b, 0.0, 2, tol=1e-11)[2]
    assert abs(E0 - Es) < 1e-12


def _shift_series(n=2):
    xs = [0.1, 0.2, 0.3, 0.4]
    return xs, [x ** (n + 1) for x in xs]


def test_ccsd_energy_extrapolates_to_the_unshifted_one():
    """Well-conditioned (0h,0p) case (o=4 v=14): the shifted energies approach E(0) only
    as s^3 (n = 2); their Pade extrapolation in s^(n+1) lands far closer to the
    unshifted energy than the smallest shift does."""
    prob = syn.make_problem(11, 4, 14, 1)
    b = ccsd.Blocks(integrals.integrals(prob), integrals.fock(prob), 4)
    E0 = ccsd.solve(b, tol=1e-12, max_iter=600)[2]
    xs, ys = _shift_series()
    Es = [intruder.ccsd_shifted(b, x, 2, tol=1e-12)[2] for x in xs]
    err_shift = abs(Es[0] - E0)
    assert err_shift > 1e-6  # the shift does change the solution
    err_pade = abs(intruder.pade_zero(ys[:3], Es[:3], 1, 1) - E0)  # square [1/1] fit
    assert err_pade < err_shift / 10


def test_heff_eigenvalues_extrapolate_to_the_unshifted_ones():
    """(0h,1p) sector on a Z4 case (o=6 v=20, four active): the Pade-extrapolated H_eff
    eigenvalues approach the unshifted ones several times more closely than the
    smallest shift."""
    prob = syn.make_problem(306, 6, 20, 4)
    V, f = integrals.integrals(prob), integrals.fock(prob)
    t1, t2, E, _, conv, _ = ccsd.solve(ccsd.Blocks(V, f, 6), tol=1e-11)
    assert conv
    act = syn.active_virtuals(prob, 4)
    w0 = fs0h1p.solve(V, f, 6, t1, t2, act, tol=1e-11)[1]
    xs, ys = _shift_series()
    ws = np.array([intruder.fs_shifted(V, f, 6, t1, t2, act, x, 2, tol=1e-11)[1] for x in xs])
    err_shift = np.max(np.abs(ws[0] - w0))
    assert err_shift > 1e-6
    ext = np.array([intruder.pade_zero(ys[:3], ws[:3, k], 1, 1) for k in range(len(w0))])
    assert np.max(np.abs(ext - w0)) < err_shift / 5


def test_shift_stabilises_an_intruder_case():
    """A (0h,1p) case with intruders: a high-lying active spinor x (the 13th lowest of 20
    virtuals) makes 68 of the D_xj^ab positive.  The unshifted Bloch iteration runs away
    (overflow); with the shift s = 2 (n = 1) it converges to a finite H_eff."""
    prob = syn.make_problem(306, 6, 20, 4)
    V, f = integrals.integrals(prob), integrals.fock(prob)
    t1, t2, E, _, conv, _ = ccsd.solve(ccsd.Blocks(V, f, 6), tol=1e-11)
    eo, ev = prob.eps_occ, prob.eps_virt
    x = int(np.argsort(ev)[12])
    D2 = ev[x] + eo[:, None, None] - ev[None, :, None] - ev[None, None, :]
    assert np.sum(D2 > 0) > 20  # positive denominators: intruders
    with np.errstate(all="ignore"):
        try:
            conv0 = fs0h1p.solve(V, f, 6, t1, t2, [x], tol=1e-9, max_iter=150)[-1]
        except np.linalg.LinAlgError:  # H_eff turned NaN / Inf
            conv0 = False
    H, w, _, _, nit, conv1 = intruder.fs_shifted(V, f, 6, t1, t2, [x], 2.0, 1, tol=1e-9, max_iter=150)
    assert not conv0
    assert conv1 and np.all(np.isfinite(w))
