"""Oracle: Fock-space CCSD for the (0h,1p) sector, complex128, dense.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

After the (0h,0p) amplitudes T are converged, the (0h,1p) cluster operator S
(s_x^a for inactive virtual a, s_xj^ab) of an active particle x solves the
Bloch equation of Eq. (amplitudes) restricted to that sector (Eq. (sectors):
sectors solved one after another, T fixed):

    Q Hbar (P + S) P = S H_eff,      H_eff = P Hbar (P + S) P,

Hbar = e^-T H_N e^T - E_CC on the electron-attached space {a+|0>, a+ b+ j|0>};
the eigenvalues of H_eff are the attachment energies of the states with active
character.  The iteration takes the method's fixed-point form
s <- s + D^-1 (Q Hbar (P+S) - S H_eff), with D_x^a = e_x - e_a and
D_xj^ab = e_x + e_j - e_a - e_b.

Hbar acting on an electron-attached vector r = sum_a r_a a+ + 1/2 sum_jab r_j^ab a+ b+ j
is written out term by term as the EA-EOM-CCSD sigma equations (Nooijen and
Bartlett, J. Chem. Phys. 102, 3629 (1995)); FS-CCSD in the (0h,1p) sector and
EA-EOM-CCSD share that operator.  The one- and two-body elements of Hbar it needs
(F_ae, F_me, F_mi, W_amef, W_mbej, W_abef, W_abej), with every T1 and T2
contribution, plus the one three-body piece (<mn||ef> t_mj^ab contracted with
r_n^ef):

    sigma_a     = F_ae r_e + F_me r_m^ae + 1/2 W_amef r_m^ef
    sigma_j^ab  = W_abej r_e + P(ab) F_be r_j^ae - F_mj r_m^ab + P(ab) W_mbej r_m^ae
                  + 1/2 W_abef r_j^ef - 1/2 t_mj^ab <mn||ef> r_n^ef

(sums over repeated indices, P(ab) X = X - X(a<->b)).  Parity: pinned by
tests/test_oracle_fs.py against the electron-attached block of an explicit
second-quantised Hbar (brute force on a determinant basis, C1 and Z4 cases), full
CI for one-electron vacua, and the containment of the H_eff eigenvalues in that
block's spectrum.
"""
from __future__ import annotations

import numpy as np

from oracle import ccsd


def es(spec, *ops):
    return np.einsum(spec, *ops, optimize=True)


class HbarEA:
    """The elements of Hbar that act on the electron-attached space, at amplitudes t1, t2."""

    def __init__(self, b: ccsd.Blocks, t1, t2):
        v = b.v
        fov, foo, fvv = b.fb("ov"), b.fb("oo"), b.fb("vv")
        tau = ccsd.tau(t1, t2)
        self.t2 = t2
        self.oovv = v("oovv")
        # one-body elements
        self.Fme = fov + es("nf,mnef->me", t1, v("oovv"))
        self.Fmi = (foo + es("ie,me->mi", t1, self.Fme) + es("ne,mnie->mi", t1, v("ooov"))
                    + 0.5 * es("inef,mnef->mi", t2, v("oovv")))
        self.Fae = (fvv - es("ma,me->ae", t1, self.Fme) + es("mf,amef->ae", t1, v("vovv"))
                    - 0.5 * es("mnaf,mnef->ae", t2, v("oovv")))
        # two-body elements
        self.Wamef = v("vovv") - es("na,nmef->amef", t1, v("oovv"))
        self.Wmbej = (v("ovvo") + es("jf,mbef->mbej", t1, v("ovvv")) - es("nb,mnej->mbej", t1, v("oovo"))
                      - es("jnfb,mnef->mbej", t2 + es("jf,nb->jnfb", t1, t1), v("oovv")))
        P01 = lambda x: x - x.swapaxes(0, 1)
        self.Wabef = (v("vvvv") - P01(es("mb,amef->abef", t1, v("vovv")))
                      + 0.5 * es("mnab,mnef->abef", tau, v("oovv")))
        # W_abej = <ab||ej> - F_me t_mj^ab + t_j^f W_abef + 1/2 <mn||ej> tau_mn^ab
        #          - P(ab) <mb||ef> t_mj^af - P(ab) t_m^a (<mb||ej> - t_nj^bf <mn||ef>)
        x = es("mbef,mjaf->abej", v("ovvv"), t2)
        y = es("ma,mbej->abej", t1, v("ovvo") - es("njbf,mnef->mbej", t2, v("oovv")))
        self.Wabej = (v("vvvo") - es("me,mjab->abej", self.Fme, t2) + es("jf,abef->abej", t1, self.Wabef)
                      + 0.5 * es("mnej,mnab->abej", v("oovo"), tau)
                      - P01(x) - P01(y))

    def sigma(self, r1, r2):
        """(Hbar_N - E_CC) on vectors r1[k, a], r2[k, j, a, b] (r2 antisymmetric in a, b)."""
        s1 = (es("ae,ke->ka", self.Fae, r1) + es("me,kmae->ka", self.Fme, r2)
              + 0.5 * es("amef,kmef->ka", self.Wamef, r2))
        x = es("be,kjae->kjab", self.Fae, r2) + es("mbej,kmae->kjab", self.Wmbej, r2)
        chi = es("mnef,knef->km", self.oovv, r2)
        s2 = (es("abej,ke->kjab", self.Wabej, r1) + (x - x.swapaxes(2, 3))
              - es("mj,kmab->kjab", self.Fmi, r2)
              + 0.5 * es("abef,kjef->kjab", self.Wabef, r2)
              - 0.5 * es("km,mjab->kjab", chi, self.t2))
        return s1, s2


def solve(V, f, o, t1, t2, act, tol=1e-10, max_iter=300, diis_dim=6, shift=None):
    """(0h,1p) FS-CCSD.  act: virtual (local) indices of the active spinors.
    Each iteration: Jacobi step s_new = s + rho/D, error s_new - s, residual
    max |s_new - s|; DIIS(diis_dim) over (s_new, error) as in oracle/ccsd (the
    paper is silent on acceleration; plain Jacobi diverges on these Hamiltonians).
    shift = (s, n): the intruder-state shifted equations of oracle/intruder.py,
    rho + (D - D~) s = 0 stepped with 1/D~ (D~ = D - s (s/(s+|D|))^n); None = unshifted.
    Returns (Heff, eigenvalues sorted by real part, s1, s2, n_iter, converged)."""
    nv = t1.shape[1]
    na = len(act)
    act = np.asarray(act)
    b = ccsd.Blocks(V, f, o)
    H = HbarEA(b, t1, t2)
    eps = np.real(np.diag(f))
    eo, ev = eps[:o], eps[o:]
    ex = ev[act]
    inactive = np.ones(nv, bool)
    inactive[act] = False
    D1 = ex[:, None] - ev[None, :]
    D1[:, act] = 1.0  # P-space entries are not updated
    D2 = (ex[:, None, None, None] + eo[None, :, None, None]
          - ev[None, None, :, None] - ev[None, None, None, :])
    if shift is not None and shift[0] > 0.0:
        sh, nn = float(shift[0]), int(shift[1])
        D1s = D1 - sh * (sh / (sh + np.abs(D1))) ** nn
        D2s = D2 - sh * (sh / (sh + np.abs(D2))) ** nn
    else:
        D1s, D2s = D1, D2
    s1 = np.zeros((na, nv), dtype=np.complex128)
    s2 = np.zeros((na, o, nv, nv), dtype=np.complex128)
    Heff = None
    diis = ccsd.DIIS(diis_dim) if diis_dim > 0 else None
    n1 = s1.size
    for it in range(1, max_iter + 1):
        r1 = s1.copy()
        r1[np.arange(na), act] = 1.0           # P + S
        sig1, sig2 = H.sigma(r1, s2)
        Heff = sig1[:, act].T                  # Heff[y, x] = (Hbar (P+S))_x at active y
        rho1 = sig1 - np.einsum("ya,yx->xa", s1, Heff)
        rho2 = sig2 - np.einsum("yjab,yx->xjab", s2, Heff)
        rho1 = rho1 + (D1 - D1s) * s1  # the shifted equations (zero when unshifted)
        rho2 = rho2 + (D2 - D2s) * s2
        rho1[:, ~inactive] = 0.0
        d1, d2 = rho1 / D1s, rho2 / D2s
        d1[:, ~inactive] = 0.0
        res = max(np.max(np.abs(d1), initial=0.0), np.max(np.abs(d2), initial=0.0))
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
