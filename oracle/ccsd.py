"""Oracle: spin-orbital CCSD for the (0h,0p) sector, complex128, dense.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The amplitude equations of Eq. (amplitudes) restricted to the vacuum sector,
t = D^-1 (V Omega)_conn, truncated to singles and doubles, in the intermediate
form of Stanton, Gauss, Watts and Bartlett (J. Chem. Phys. 94, 4334 (1991)).
Every integral is written <created created || annihilated annihilated>, so the
complex case differs from the real one only in its drivers: <ab||ij> (not
<ij||ab>) in the T2 equation and f_ai in the T1 equation.  D are the negated
differences of H0 eigenvalues (the paragraph after Eq. (amplitudes)):
D_i^a = e_i - e_a,  D_ij^ab = e_i + e_j - e_a - e_b.

Arrays: t1[i, a], t2[i, j, a, b], V[p, q, r, s] over all spinors (occupied
first), f the Fock matrix.  Parity: pinned by tests/test_oracle_ccsd.py against
an explicit second-quantised e^-T H e^T (brute force on a determinant basis),
against full CI for two electrons (CCSD is exact there), the closed-form MP2
energy, antisymmetry, real/gauge invariants and symmetry-blocked == C1.

Iteration (the method's fixed-point form, the paper is silent on acceleration):
MP2 guess (t1 = 0, t2 = <ab||ij>/D), then repeated Jacobi updates
t_new = RHS(t)/D with DIIS(6) extrapolation; the residual is max |t_new - t|.
"""
from __future__ import annotations

import dataclasses
import numpy as np

def es(spec, *ops):
    """einsum with a BLAS-backed contraction path (a library contraction primitive)."""
    return np.einsum(spec, *ops, optimize=True)


def _P01(x):
    """P(pq) X = X - X(p<->q) on the first two indices."""
    return x - x.swapaxes(0, 1)


def _P23(x):
    """P(pq) X on the last two indices."""
    return x - x.swapaxes(2, 3)


@dataclasses.dataclass
class Blocks:
    """Views of V and f split into occupied (o) / virtual (v) slices."""
    V: np.ndarray
    f: np.ndarray
    o: int

    def __post_init__(self):
        o = self.o
        self.O = slice(0, o)
        self.Vs = slice(o, self.V.shape[0])

    def v(self, spec: str) -> np.ndarray:
        sl = [self.O if c == "o" else self.Vs for c in spec]
        return self.V[tuple(sl)]

    def fb(self, spec: str) -> np.ndarray:
        sl = [self.O if c == "o" else self.Vs for c in spec]
        return self.f[tuple(sl)]

    @property
    def eps_o(self):
        return np.real(np.diag(self.f))[: self.o]

    @property
    def eps_v(self):
        return np.real(np.diag(self.f))[self.o:]


def denominators(b: Blocks):
    eo, ev = b.eps_o, b.eps_v
    D1 = eo[:, None] - ev[None, :]
    D2 = (eo[:, None, None, None] + eo[None, :, None, None]
          - ev[None, None, :, None] - ev[None, None, None, :])
    return D1, D2


def tau_tilde(t1, t2):
    return t2 + 0.5 * (es("ia,jb->ijab", t1, t1) - es("ib,ja->ijab", t1, t1))


def tau(t1, t2):
    return t2 + es("ia,jb->ijab", t1, t1) - es("ib,ja->ijab", t1, t1)


def intermediates(t1, t2, b: Blocks):
    """F_ae, F_mi, F_me, W_mnij, W_abef, W_mbej (Stanton-Gauss Eqs. 3-8)."""
    tt = tau_tilde(t1, t2)
    ta = tau(t1, t2)
    fov, foo, fvv = b.fb("ov"), b.fb("oo"), b.fb("vv")
    no, nv = t1.shape
    Fae = (fvv * (1 - np.eye(nv)) - 0.5 * es("me,ma->ae", fov, t1)
           + es("mf,mafe->ae", t1, b.v("ovvv"))
           - 0.5 * es("mnaf,mnef->ae", tt, b.v("oovv")))
    Fmi = (foo * (1 - np.eye(no)) + 0.5 * es("ie,me->mi", t1, fov)
           + es("ne,mnie->mi", t1, b.v("ooov"))
           + 0.5 * es("inef,mnef->mi", tt, b.v("oovv")))
    Fme = fov + es("nf,mnef->me", t1, b.v("oovv"))
    Wmnij = (b.v("oooo")
             + (lambda x: x - x.swapaxes(2, 3))(es("je,mnie->mnij", t1, b.v("ooov")))
             + 0.25 * es("ijef,mnef->mnij", ta, b.v("oovv")))
    Wabef = (b.v("vvvv")
             - _P01(es("mb,amef->abef", t1, b.v("vovv")))
             + 0.25 * es("mnab,mnef->abef", ta, b.v("oovv")))
    zeta = 0.5 * t2 + es("jf,nb->jnfb", t1, t1)
    Wmbej = (b.v("ovvo")
             + es("jf,mbef->mbej", t1, b.v("ovvv"))
             - es("nb,mnej->mbej", t1, b.v("oovo"))
             - es("jnfb,mnef->mbej", zeta, b.v("oovv")))
    return Fae, Fmi, Fme, Wmnij, Wabef, Wmbej


def rhs(t1, t2, b: Blocks):
    """Right-hand sides of D t1 = R1 and D t2 = R2 (Stanton-Gauss Eqs. 1-2)."""
    Fae, Fmi, Fme, Wmnij, Wabef, Wmbej = intermediates(t1, t2, b)
    ta = tau(t1, t2)
    r1 = (b.fb("vo").T
          + es("ie,ae->ia", t1, Fae)
          - es("ma,mi->ia", t1, Fmi)
          + es("imae,me->ia", t2, Fme)
          - es("nf,naif->ia", t1, b.v("ovov"))
          - 0.5 * es("imef,maef->ia", t2, b.v("ovvv"))
          - 0.5 * es("mnae,nmei->ia", t2, b.v("oovo")))
    Fbe = Fae - 0.5 * es("mb,me->be", t1, Fme)
    Fmj = Fmi + 0.5 * es("je,me->mj", t1, Fme)
    ring = (es("imae,mbej->ijab", t2, Wmbej)
            - es("ie,ma,mbej->ijab", t1, t1, b.v("ovvo")))
    r2 = (b.v("vvoo").transpose(2, 3, 0, 1)
          + _P23(es("ijae,be->ijab", t2, Fbe))
          - _P01(es("imab,mj->ijab", t2, Fmj))
          + 0.5 * es("mnab,mnij->ijab", ta, Wmnij)
          + 0.5 * es("ijef,abef->ijab", ta, Wabef)
          + _P01(_P23(ring))
          + _P01(es("ie,abej->ijab", t1, b.v("vvvo")))
          - _P23(es("ma,mbij->ijab", t1, b.v("ovoo"))))
    return r1, r2


def residual(t1, t2, b: Blocks):
    """<mu| e^-T H_N e^T |0> for singles and doubles: RHS - D t."""
    D1, D2 = denominators(b)
    r1, r2 = rhs(t1, t2, b)
    return r1 - D1 * t1, r2 - D2 * t2


def energy(t1, t2, b: Blocks) -> complex:
    """E = sum f_ia t_i^a + 1/4 sum <ij||ab> t_ij^ab + 1/2 sum <ij||ab> t_i^a t_j^b."""
    Vo = b.v("oovv")
    return complex(es("ia,ia->", b.fb("ov"), t1)
                   + 0.25 * es("ijab,ijab->", Vo, t2)
                   + 0.5 * es("ijab,ia,jb->", Vo, t1, t1))


def mp2_guess(b: Blocks):
    """t1 = 0, t2 = <ab||ij> / D_ij^ab (first-order amplitudes)."""
    D1, D2 = denominators(b)
    t2 = b.v("vvoo").transpose(2, 3, 0, 1) / D2
    return np.zeros_like(D1, dtype=np.complex128), t2


def mp2_energy(b: Blocks) -> float:
    """Closed form E_MP2 = 1/4 sum |<ab||ij>|^2 / D_ij^ab."""
    _, D2 = denominators(b)
    return float(0.25 * np.sum(np.abs(b.v("vvoo").transpose(2, 3, 0, 1)) ** 2 / D2))


class DIIS:
    """Pulay DIIS over the last `dim` (t_new, e) pairs.

    B_kl = Re <e_k, e_l> (all stored amplitude elements), the constrained
    system [B -1; -1 0][c; lam] = [0; -1]; extrapolation starts with 2 vectors.
    A near-singular B (smallest |pivot| < 1e-14 max diag) drops the oldest pair.
    """

    def __init__(self, dim: int = 6):
        self.dim = dim
        self.vecs: list[np.ndarray] = []
        self.errs: list[np.ndarray] = []

    def push(self, vec, err):
        self.vecs.append(vec.copy())
        self.errs.append(err.copy())
        if len(self.vecs) > self.dim:
            self.vecs.pop(0)
            self.errs.pop(0)

    def coefficients(self):
        while len(self.vecs) >= 2:
            m = len(self.vecs)
            B = np.empty((m + 1, m + 1))
            for k in range(m):
                for l in range(m):
                    B[k, l] = np.real(np.vdot(self.errs[k], self.errs[l]))
            B[m, :m] = B[:m, m] = -1.0
            B[m, m] = 0.0
            rhs_ = np.zeros(m + 1)
            rhs_[m] = -1.0
            c = gauss_solve(B, rhs_, 1e-14 * np.max(np.diag(B)[:m]))
            if c is not None:
                return c[:m]
            self.vecs.pop(0)
            self.errs.pop(0)
        return None

    def extrapolate(self):
        c = self.coefficients()
        if c is None:
            return self.vecs[-1].copy()
        return sum(ck * v for ck, v in zip(c, self.vecs))


def gauss_solve(A, y, tiny):
    """Gaussian elimination with partial pivoting; None if a pivot is below `tiny`."""
    A = np.array(A, dtype=np.float64)
    y = np.array(y, dtype=np.float64)
    n = len(y)
    for k in range(n):
        p = k + int(np.argmax(np.abs(A[k:, k])))
        if abs(A[p, k]) < tiny:
            return None
        if p != k:
            A[[k, p]] = A[[p, k]]
            y[[k, p]] = y[[p, k]]
        for r in range(k + 1, n):
            m = A[r, k] / A[k, k]
            A[r, k:] -= m * A[k, k:]
            y[r] -= m * y[k]
    x = np.zeros(n)
    for k in range(n - 1, -1, -1):
        x[k] = (y[k] - A[k, k + 1:] @ x[k + 1:]) / A[k, k]
    return x


def pack(t1, t2):
    return np.concatenate([t1.ravel(), t2.ravel()])


def unpack(vec, no, nv):
    n1 = no * nv
    return vec[:n1].reshape(no, nv), vec[n1:].reshape(no, no, nv, nv)


@dataclasses.dataclass
class IterRecord:
    it: int
    energy: complex
    max_dt: float
    diis_n: int


def solve(b: Blocks, tol: float = 1e-9, max_iter: int = 200, diis_dim: int = 6,
          t_init=None, history: bool = False, D=None):
    """CCSD fixed point from the MP2 (or a given) guess with DIIS.

    Iteration 0 reports E(t_guess) (= E_MP2 for the MP2 guess).  Each iteration
    k >= 1 computes t_new = RHS(t)/D, residual max|t_new - t| and E(t_new);
    it stops when the residual is below `tol`, else extrapolates with DIIS.
    D: (D1, D2) in place of the denominators of b (the shifted equations of
    oracle/intruder.py); None = the plain ones.
    Returns (t1, t2, E, n_iter, converged, records).
    """
    D1, D2 = denominators(b) if D is None else D
    no, nv = D1.shape
    t1, t2 = mp2_guess(b) if t_init is None else (t_init[0].copy(), t_init[1].copy())
    recs = [IterRecord(0, energy(t1, t2, b), float("nan"), 0)]
    diis = DIIS(diis_dim) if diis_dim > 0 else None
    t = pack(t1, t2)
    E = recs[0].energy
    for it in range(1, max_iter + 1):
        r1, r2 = rhs(*unpack(t, no, nv), b)
        tn = pack(r1 / D1, r2 / D2)
        err = tn - t
        res = float(np.max(np.abs(err)))
        E = energy(*unpack(tn, no, nv), b)
        if res < tol:
            recs.append(IterRecord(it, E, res, 0))
            t = tn
            return (*unpack(t, no, nv), E, it, True, recs)
        if diis is not None:
            diis.push(tn, err)
            t = diis.extrapolate()
            recs.append(IterRecord(it, E, res, len(diis.vecs)))
        else:
            t = tn
            recs.append(IterRecord(it, E, res, 0))
    return (*unpack(t, no, nv), E, max_iter, False, recs)
