"""Oracle: intruder-state denominator shifts and Pade extrapolation to zero shift.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Intruder states show up as small or positive energy denominators D in Eq.
(amplitudes) (Sec. II.A, the paragraph after Eq. (sectors)); the method shifts the
ill-defined denominators so that the amplitude equations have stable solutions, and
the results can then be extrapolated to the zero-shift limit with Pade approximants
(Sec. III.A, the feature list: "dynamic" denominator shifts).  The paper gives no
formula; the reading taken here:

  * dynamic shift: every denominator D is replaced by
        D~ = D - s (s / (s + |D|))^n,          s >= 0, n >= 1,
    so a denominator near zero (or positive) moves by about -s while one with
    |D| >> s moves by s (s/|D|)^n only; s = 0 is the unshifted method;
  * the shifted equations keep their form with D~ in place of D: (0h,0p)
    D~ t = RHS(t), and in the (0h,1p) Bloch form rho + (D - D~) s = 0 with
    rho = Q Hbar (P+S) - S H_eff, iterated as s <- s + (rho + (D - D~) s) / D~;
  * extrapolation: values E(x_k) computed at shift scales x_k (the shift x_k s0),
    k = 1..m, are fitted by the Pade form E(x) = (a0 + a1 x + ... + aL x^L) /
    (1 + b1 x + ... + bM x^M) through the linear system
        a0 + a1 x_k + ... + aL x_k^L - E_k (b1 x_k + ... + bM x_k^M) = E_k
    (square when L + M + 1 = m, least squares otherwise); the zero-shift value is a0.

Parity: pinned by tests/test_oracle_intruder.py (s = 0 is the unshifted method; the
Pade fit reproduces a rational function of its own degree exactly and a0 equals its
value at 0; on a well-conditioned case the extrapolated energy approaches the
unshifted one much more closely than any shifted energy).
"""
from __future__ import annotations

import numpy as np

from oracle import ccsd, fs0h1p


def dynamic_shift(D, s: float, n: int = 1):
    """D~ = D - s (s / (s + |D|))^n (elementwise; s = 0 leaves D unchanged)."""
    D = np.asarray(D, dtype=np.float64)
    if s <= 0.0:
        return D.copy()
    return D - s * (s / (s + np.abs(D))) ** n


def ccsd_shifted(b: ccsd.Blocks, s: float, n: int = 1, tol: float = 1e-10, max_iter: int = 600):
    """(0h,0p) CCSD with shifted denominators: MP2-like guess V/D~, then t = RHS(t)/D~
    with DIIS, as oracle.ccsd.solve.  Returns (t1, t2, E, n_iter, converged)."""
    D1, D2 = ccsd.denominators(b)
    D1s, D2s = dynamic_shift(D1, s, n), dynamic_shift(D2, s, n)
    t1 = np.zeros_like(D1, dtype=np.complex128)
    t2 = b.v("vvoo").transpose(2, 3, 0, 1) / D2s
    t1, t2, E, nit, conv, _ = ccsd.solve(b, tol=tol, max_iter=max_iter, t_init=(t1, t2), D=(D1s, D2s))
    return t1, t2, E, nit, conv


def fs_shifted(V, f, o, t1, t2, act, s: float, n: int = 1, tol: float = 1e-10, max_iter: int = 300):
    """(0h,1p) FS-CCSD (oracle.fs0h1p) with shifted Bloch denominators."""
    return fs0h1p.solve(V, f, o, t1, t2, act, tol=tol, max_iter=max_iter, shift=(s, n))


def pade_zero(x, values, L: int, M: int) -> complex:
    """The zero-shift value a0 of the [L/M] Pade fit of values E_k at scales x_k."""
    x = np.asarray(x, dtype=np.float64)
    E = np.asarray(values, dtype=np.complex128)
    m = len(x)
    if L + M + 1 > m:
        raise ValueError("need at least L + M + 1 points")
    A = np.zeros((m, L + 1 + M), dtype=np.complex128)
    for k in range(m):
        for j in range(L + 1):
            A[k, j] = x[k] ** j
        for j in range(1, M + 1):
            A[k, L + j] = -E[k] * x[k] ** j
    coef = np.linalg.lstsq(A, E, rcond=None)[0]
    return complex(coef[0])
