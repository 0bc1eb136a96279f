"""Oracle: Fock-space CCSD for the (0h,1p) sector, complex128, dense.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

After the (0h,0p) amplitudes T are converged, the (0h,1p) cluster operator S
(s_x^a for inactive virtual a, s_xj^ab) of an active particle x solves the
Bloch equation of Eq. (amplitudes) restricted to that sector (Eq. (sectors):
sectors solved one after another, T fixed):

    Q Hbar (P + S) P = S H_eff,      H_eff = P Hbar (P + S) P,

Hbar = e^-T (H - E_ref) e^T - E_CC on the electron-attached space
{a+|0>, a+ b+ j|0>}; the eigenvalues of H_eff are the attachment energies of the
states with active character.  The iteration takes the method's fixed-point form
s <- s + D^-1 (Q Hbar (P+S) - S H_eff), with D_x^a = e_x - e_a and
D_xj^ab = e_x + e_j - e_a - e_b.

Hbar acting on an electron-attached vector r is evaluated as the CCSD residual
(oracle/ccsd.residual, itself pinned by brute force) of an augmented system in
which one extra occupied spinor g (orbital energy 0, every integral with g
zero) carries r as its amplitudes: t_g^a = r_a, t_gj^ab = r_j^ab.  The residual
is linear in those amplitudes and its g-projections are exactly
(Hbar_N - E_CC) r; one ghost per active spinor gives all H_eff columns at once.
Parity: pinned by tests/test_oracle_fs.py against the electron-attached block of
an explicit second-quantised Hbar, full CI for one-electron vacua, and the
containment of the H_eff eigenvalues in that block's spectrum.
"""
from __future__ import annotations

import numpy as np

from oracle import ccsd


def augment(V, f, o, n_ghost):
    """Insert n_ghost non-interacting occupied spinors after the real occupied ones."""
    n = V.shape[0]
    keep = np.r_[0:o, o + n_ghost:n + n_ghost]
    Va = np.zeros((n + n_ghost,) * 4, dtype=np.complex128)
    Va[np.ix_(keep, keep, keep, keep)] = V
    fa = np.zeros((n + n_ghost,) * 2, dtype=np.complex128)
    fa[np.ix_(keep, keep)] = f
    return Va, fa


def hbar_ea(b_aug: ccsd.Blocks, t1, t2, o, r1, r2):
    """(Hbar_N - E_CC) applied to electron-attached vectors r1[k, a], r2[k, j, a, b]
    (k = ghost slot).  t1, t2: converged (0h,0p) amplitudes of the real system."""
    ng, nv = r1.shape
    oa = o + ng
    T1 = np.zeros((oa, nv), dtype=np.complex128)
    T2 = np.zeros((oa, oa, nv, nv), dtype=np.complex128)
    T1[:o] = t1
    T2[:o, :o] = t2
    for k in range(ng):
        T1[o + k] = r1[k]
        T2[o + k, :o] = r2[k]
        T2[:o, o + k] = -r2[k]
    R1, R2 = ccsd.residual(T1, T2, b_aug)
    s1 = np.stack([R1[o + k] for k in range(ng)])
    s2 = np.stack([R2[o + k, :o] for k in range(ng)])
    return s1, s2


def solve(V, f, o, t1, t2, act, tol=1e-10, max_iter=300, diis_dim=6):
    """(0h,1p) FS-CCSD.  act: virtual (local) indices of the active spinors.
    Each iteration: Jacobi step s_new = s + rho/D, error s_new - s, residual
    max |s_new - s|; DIIS(diis_dim) over (s_new, error) as in oracle/ccsd (the
    paper is silent on acceleration; plain Jacobi diverges on these Hamiltonians).
    Returns (Heff, eigenvalues sorted by real part, s1, s2, n_iter, converged)."""
    nv = t1.shape[1]
    na = len(act)
    act = np.asarray(act)
    Va, fa = augment(V, f, o, na)
    b_aug = ccsd.Blocks(Va, fa, o + na)
    eps = np.real(np.diag(f))
    eo, ev = eps[:o], eps[o:]
    ex = ev[act]
    inactive = np.ones(nv, bool)
    inactive[act] = False
    D1 = ex[:, None] - ev[None, :]
    D1[:, act] = 1.0  # P-space entries are not updated
    D2 = (ex[:, None, None, None] + eo[None, :, None, None]
          - ev[None, None, :, None] - ev[None, None, None, :])
    s1 = np.zeros((na, nv), dtype=np.complex128)
    s2 = np.zeros((na, o, nv, nv), dtype=np.complex128)
    Heff = None
    diis = ccsd.DIIS(diis_dim) if diis_dim > 0 else None
    n1 = s1.size
    for it in range(1, max_iter + 1):
        r1 = s1.copy()
        r1[np.arange(na), act] = 1.0           # P + S
        sig1, sig2 = hbar_ea(b_aug, t1, t2, o, r1, s2)
        Heff = sig1[:, act].T                  # Heff[y, x] = (Hbar (P+S))_x at active y
        rho1 = sig1 - np.einsum("ya,yx->xa", s1, Heff)
        rho2 = sig2 - np.einsum("yjab,yx->xjab", s2, Heff)
        rho1[:, ~inactive] = 0.0
        d1, d2 = rho1 / D1, rho2 / D2
        d1[:, ~inactive] = 0.0
        res = max(np.max(np.abs(d1)), np.max(np.abs(d2)))
        new = np.concatenate([(s1 + d1).ravel(), (s2 + d2).ravel()])
        if res < tol:
            s1, s2 = new[:n1].reshape(s1.shape), new[n1:].reshape(s2.shape)
            w = np.linalg.eigvals(Heff)
            return Heff, w[np.lexsort((w.imag, w.real))], s1, s2, it, True
        if diis is not None:
            diis.push(new, np.concatenate([d1.ravel(), d2.ravel()]))
            new = diis.extrapolate()
        s1, s2 = new[:n1].reshape(s1.shape), new[n1:].reshape(s2.shape)
    w = np.linalg.eigvals(Heff)
    return Heff, w[np.lexsort((w.imag, w.real))], s1, s2, max_iter, False
