"""Oracle: Fock-space CCSD for the (0h,2p) sector, complex128, on a determinant basis.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sectors are solved one after another (Eq. (sectors)).  With the (0h,0p) amplitudes T
(oracle.ccsd) and the (0h,1p) amplitudes S1 = {s_x^a, s_xj^ab} (oracle.fs0h1p) fixed,
the (0h,2p) cluster operator

    S2 = sum over x<y active, a<b not both active of s_xy^ab {a+ b+ y x}

solves the Bloch equation of Eq. (amplitudes) in that sector, projected on the
two-particle determinants |ab> = a+ b+ |0>:

    <ab| Hbar Omega |xy>  =  sum over z<w of <ab| Omega |zw> H_eff(zw, xy),
    H_eff(zw, xy) = <zw| Hbar Omega |xy>,           Omega = {exp(S1 + S2)},

with Hbar = e^-T (H - E_0) e^T, E_0 = <0|H|0> + E_CC, and |xy> = x+ y+ |0> for active
x < y.  The eigenvalues of H_eff are the double-attachment energies (relative to the
CCSD ground state) of the states with active character.  The iteration takes the
method's fixed-point form s <- s + rho / D, D_xy^ab = e_x + e_y - e_a - e_b, with DIIS.

Everything is evaluated literally, for tiny problems only: operators are matrices on
the determinants of N + 2 electrons (occupation bit strings with the Jordan-Wigner
sign); H is built from the core Hamiltonian and V term by term; e^T is a finite power
series (T is nilpotent); the normal-ordered exponential acting on |xy> is built from
the normal products of the S operator strings: a product of strings is reordered into
quasi-particle normal order relative to |0> with the sign of the permutation and no
contractions.  On a state with two valence particles only products of at most two
(0h,1p) factors survive, and S2 enters only through S2 |xy>, so

    Omega |xy> = e^T ( |xy> + S1 |xy> + 1/2 {S1 S1} |xy> + sum_{a<b} s_xy^ab |ab> ).

Parity: pinned by tests/test_oracle_fs2.py:
  * two electrons on an empty reference (o = 0: T = 0): the H_eff eigenvalues are
    eigenvalues of the two-electron full CI (the Bloch equation is exact there);
  * the normal product differs from the plain operator product exactly where a
    valence line would be contracted (a hand-checked case);
  * with occupied spinors, the same sector built a second way (ghost occupied spinors
    carrying the valence amplitudes through the CCSD residual of oracle.ccsd): the
    oracle's converged S2 zeroes that construction's residual and the H_eff
    eigenvalues agree;
  * a planted sign slip in the normal product is caught by the comparison with the
    ghost construction (with occupied spinors; on an empty reference that term feeds only
    two-particle components, which S2 absorbs).
"""
from __future__ import annotations

import itertools

import numpy as np

from oracle import ccsd


# ---------------------------------------------------------------------------
# Second quantisation on occupation bit strings
def _ann(p, det):
    if not (det >> p) & 1:
        return None, 0
    return det ^ (1 << p), (-1 if bin(det & ((1 << p) - 1)).count("1") % 2 else 1)


def _cre(p, det):
    if (det >> p) & 1:
        return None, 0
    return det | (1 << p), (-1 if bin(det & ((1 << p) - 1)).count("1") % 2 else 1)


def apply_ops(ops, det):
    """Apply the operator product ops = [(p, dagger), ...] (rightmost acts first)."""
    sign = 1
    for p, dag in reversed(ops):
        det, s = (_cre if dag else _ann)(p, det)
        if det is None:
            return None, 0
        sign *= s
    return det, sign


def quasi_creator(op, o):
    """Relative to the reference with spinors 0..o-1 occupied: a+ of a virtual and a of an
    occupied spinor create quasi-particles."""
    p, dag = op
    return dag if p >= o else not dag


def normal_product(ops, o):
    """{ops}: the string reordered with every quasi-creator left of every quasi-annihilator
    (relative orders kept), times the sign of that permutation; no contraction terms."""
    cre = [x for x in ops if quasi_creator(x, o)]
    ann = [x for x in ops if not quasi_creator(x, o)]
    # each (annihilator, later creator) pair is one transposition
    inv, seen_ann = 0, 0
    for x in ops:
        if quasi_creator(x, o):
            inv += seen_ann
        else:
            seen_ann += 1
    return cre + ann, (-1 if inv % 2 else 1)


class Basis:
    """All determinants of nel electrons in n spinors."""

    def __init__(self, n, nel):
        self.dets = [sum(1 << k for k in c) for c in itertools.combinations(range(n), nel)]
        self.index = {d: k for k, d in enumerate(self.dets)}

    def __len__(self):
        return len(self.dets)

    def vector(self, det, coef=1.0):
        v = np.zeros(len(self), dtype=np.complex128)
        if det is not None:
            v[self.index[det]] = coef
        return v

    def matrix(self, terms):
        """sum_k c_k (operator string k) as a matrix on this basis."""
        M = np.zeros((len(self), len(self)), dtype=np.complex128)
        for coef, ops in terms:
            if coef == 0:
                continue
            for col, d in enumerate(self.dets):
                nd, s = apply_ops(ops, d)
                if nd is not None:
                    M[self.index[nd], col] += s * coef
        return M

    def apply(self, terms, vec):
        """sum_k c_k (operator string k) applied to a vector of this basis."""
        out = np.zeros(len(self), dtype=np.complex128)
        for col in np.nonzero(vec)[0]:
            d = self.dets[col]
            for coef, ops in terms:
                nd, s = apply_ops(ops, d)
                if nd is not None:
                    out[self.index[nd]] += s * coef * vec[col]
        return out


# ---------------------------------------------------------------------------
# Operators of the method
def hamiltonian_terms(f, V, o):
    """H = sum h_pq p+ q + 1/4 sum V_pqrs p+ q+ s r, with h = f - sum_i <pi||qi> the core
    Hamiltonian whose reference Fock matrix is f (Eq. (ham))."""
    n = f.shape[0]
    h = f - np.einsum("piqi->pq", V[:, :o, :, :o])
    terms = [(h[p, q], [(p, True), (q, False)]) for p in range(n) for q in range(n) if h[p, q] != 0]
    for p, q, r, s in np.argwhere(V != 0):
        terms.append((0.25 * V[p, q, r, s], [(p, True), (q, True), (s, False), (r, False)]))
    return terms, h


def reference_energy(h, V, o):
    return complex(np.trace(h[:o, :o]) + 0.5 * np.einsum("ijij->", V[:o, :o, :o, :o]))


def cluster_terms(t1, t2, o):
    """T = sum t_i^a a+ i + 1/4 sum t_ij^ab a+ b+ j i."""
    nv = t1.shape[1]
    out = [(t1[i, a], [(o + a, True), (i, False)]) for i in range(o) for a in range(nv) if t1[i, a] != 0]
    for i, j, a, b in itertools.product(range(o), range(o), range(nv), range(nv)):
        if t2[i, j, a, b] != 0:
            out.append((0.25 * t2[i, j, a, b], [(o + a, True), (o + b, True), (j, False), (i, False)]))
    return out


def sector1_terms(s1, s2, act, o):
    """S1 = sum_x [ sum_a s_x^a {a+ x} + 1/2 sum_jab s_xj^ab {a+ b+ j x} ] in the
    conventions of oracle.fs0h1p (s1[x, a], s2[x, j, a, b], x the active slot)."""
    na, nv = s1.shape
    out = []
    for x in range(na):
        X = (o + int(act[x]), False)
        out += [(s1[x, a], [(o + a, True), X]) for a in range(nv) if s1[x, a] != 0]
        for j, a, b in itertools.product(range(o), range(nv), range(nv)):
            if s2[x, j, a, b] != 0:
                out.append((0.5 * s2[x, j, a, b], [(o + a, True), (o + b, True), (j, False), X]))
    return out


def expm_nilpotent(A):
    out = np.eye(A.shape[0], dtype=np.complex128)
    term = out.copy()
    for k in range(1, A.shape[0] + 1):
        term = term @ A / k
        if not np.any(term):
            break
        out = out + term
    return out


def solve(V, f, o, t1, t2, e_cc, act, s1, s2, tol=1e-10, max_iter=300, diis_dim=6):
    """(0h,2p) FS-CCSD for active virtual spinors `act` (local indices), from converged
    T = (t1, t2) with correlation energy e_cc and (0h,1p) amplitudes (s1, s2) of
    oracle.fs0h1p.  Returns (H_eff over the active pairs x<y (row = (z, w), column =
    (x, y), pairs in the order of `pairs`), eigenvalues sorted by real then imaginary
    part, s (pairs x Q pairs), pairs, Q pairs, n_iter, converged)."""
    n = f.shape[0]
    nv = n - o
    act = np.asarray(act)
    na = len(act)
    basis = Basis(n, o + 2)
    hterms, h = hamiltonian_terms(f, V, o)
    E0 = reference_energy(h, V, o) + e_cc
    Hm = basis.matrix(hterms) - E0 * np.eye(len(basis))
    Tm = basis.matrix(cluster_terms(t1, t2, o))
    M = expm_nilpotent(-Tm) @ Hm @ expm_nilpotent(Tm)  # Hbar on N + 2 electrons
    S1 = sector1_terms(s1, s2, act, o)
    ref = (1 << o) - 1
    pairs = [(x, y) for x in range(na) for y in range(x + 1, na)]
    actset = set(int(a) for a in act)
    qpairs = [(a, b) for a in range(nv) for b in range(a + 1, nv) if not (a in actset and b in actset)]

    def det_of(p, q):  # p+ q+ |0> as (vector index, sign)
        d, sg = apply_ops([(o + p, True), (o + q, True)], ref)
        return basis.index[d], sg

    # the S2-free part of Omega |xy> before e^T: |xy> + S1 |xy> + 1/2 {S1 S1} |xy>
    F = []
    for x, y in pairs:
        k, sg = det_of(int(act[x]), int(act[y]))
        v = basis.vector(basis.dets[k], sg)
        d0 = basis.dets[k]
        v = v + basis.apply(S1, v)
        for (ca, A), (cb, B) in itertools.product(S1, S1):
            ops, sn = normal_product(A + B, o)
            nd, s = apply_ops(ops, d0)
            if nd is not None:
                v[basis.index[nd]] += 0.5 * ca * cb * sn * s * sg
        F.append(v)
    F = np.array(F)                                      # [pair, det]
    qdet = np.array([det_of(a, b) for a, b in qpairs], dtype=np.int64).reshape(-1, 2)
    pdet = np.array([det_of(int(act[z]), int(act[w])) for z, w in pairs], dtype=np.int64).reshape(-1, 2)
    eps = np.real(np.diag(f))
    ev = eps[o:]
    D = np.array([[ev[act[x]] + ev[act[y]] - ev[a] - ev[b] for a, b in qpairs] for x, y in pairs])
    s = np.zeros((len(pairs), len(qpairs)), dtype=np.complex128)
    diis = ccsd.DIIS(diis_dim) if diis_dim > 0 else None
    Heff = None

    def project(vecs, dets):  # <p+ q+ 0| v for the listed determinants
        return vecs[:, dets[:, 0]] * dets[:, 1][None, :]

    for it in range(1, max_iter + 1):
        Om = F.copy()
        if len(qpairs):
            Om[:, qdet[:, 0]] += s * qdet[:, 1][None, :]
        HO = Om @ M.T                                    # rows: Hbar Omega |xy>
        Heff = project(HO, pdet).T                       # Heff[zw, xy]
        rho = project(HO, qdet) - (project(Om, qdet).T @ Heff).T if len(qpairs) else np.zeros_like(s)
        d = rho / D if len(qpairs) else rho
        res = np.max(np.abs(d), initial=0.0)
        new = s + d
        if res < tol:
            w = np.linalg.eigvals(Heff)
            return Heff, w[np.lexsort((w.imag, w.real))], new, pairs, qpairs, it, True
        if diis is not None and new.size:
            diis.push(new.ravel(), d.ravel())
            new = diis.extrapolate().reshape(s.shape)
        s = new
    w = np.linalg.eigvals(Heff)
    return Heff, w[np.lexsort((w.imag, w.real))], s, pairs, qpairs, max_iter, False


def solve_ghost(V, f, o, t1, t2, act, s1, s2, tol=1e-11, max_iter=500):
    """The same sector built a second way, for sizes the determinant basis cannot hold:
    every active spinor x becomes a non-interacting occupied "ghost" g_x (no integrals,
    zero orbital energy) whose CCSD amplitudes carry the valence amplitudes (t_{g_x}^a =
    s_x^a with t_{g_x}^x = 1, t_{g_x j}^{ab} = s_xj^ab, t_{g_x g_y}^{ab} = s_xy^ab), so the
    connected part of Hbar Omega |xy> is the CCSD doubles residual of oracle.ccsd at
    (g_x, g_y).  The disconnected products of the Bloch equation cancel against the
    (0h,1p) equations, leaving
        rho_xy^ab = R_{g_x g_y}^{ab} - sum_z s_zy^ab H1_zx - sum_w s_xw^ab H1_wy
                    - 1/2 sum_zw tau_zw^ab H2_zw,xy,
    H1 the (0h,1p) H_eff (the singles residual at the active columns), H2_zw,xy the
    doubles residual at (a, b) = (z, w) and tau_zw^ab = s_zw^ab + c_z^a c_w^b - c_z^b c_w^a.
    H_eff = H1 (x) 1 + 1 (x) H1 + H2 on the pairs x < y.  Returns (H_eff, sorted
    eigenvalues, converged)."""
    n = f.shape[0]
    nv = n - o
    na = len(act)
    no = o + na
    idx = np.r_[np.arange(o), no + np.arange(nv)]  # real spinors in the extended order
    Ve = np.zeros((no + nv,) * 4, complex)
    Ve[np.ix_(idx, idx, idx, idx)] = V
    fe = np.zeros((no + nv, no + nv), complex)
    fe[np.ix_(idx, idx)] = f
    b = ccsd.Blocks(Ve, fe, no)
    t1e = np.zeros((no, nv), complex)
    t1e[:o] = t1
    t1e[o:] = s1
    t1e[o + np.arange(na), act] = 1.0  # P
    t2e = np.zeros((no, no, nv, nv), complex)
    t2e[:o, :o] = t2
    t2e[o:, :o] = s2
    t2e[:o, o:] = -s2.transpose(1, 0, 2, 3)
    actset = set(int(a) for a in act)
    # the unknowns: x<y, a<b, not both a and b active; each step is taken on these and
    # written into the four antisymmetric copies (a step on all copies separately lets
    # rounding grow a symmetric part that the equations do not damp)
    up = np.zeros((na, na, nv, nv), bool)
    for x, y in itertools.combinations(range(na), 2):
        for a, bq in itertools.combinations(range(nv), 2):
            up[x, y, a, bq] = not (a in actset and bq in actset)

    def anti(u):
        full = np.zeros((na, na, nv, nv), complex)
        full[up] = u
        return full - full.transpose(1, 0, 2, 3) - full.transpose(0, 1, 3, 2) + full.transpose(1, 0, 3, 2)

    eps = np.real(np.diag(f))
    ex, ev = eps[o + act], eps[o:]
    D = ex[:, None, None, None] + ex[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    sg = np.zeros((na, na, nv, nv), complex)
    diis = ccsd.DIIS(6)
    for it in range(max_iter):
        t2e[o:, o:] = sg
        r1, r2 = ccsd.residual(t1e, t2e, b)
        H1 = r1[o:, act].T                                   # H1[z, x]
        c = t1e[o:]
        tau = sg + np.einsum("za,wb->zwab", c, c) - np.einsum("zb,wa->zwab", c, c)
        H2 = r2[o:, o:][:, :, act][:, :, :, act].transpose(2, 3, 0, 1)  # H2[z, w, x, y]
        rho = (r2[o:, o:] - np.einsum("zyab,zx->xyab", sg, H1) - np.einsum("xwab,wy->xyab", sg, H1)
               - 0.5 * np.einsum("zwab,zwxy->xyab", tau, H2))
        d = rho[up] / D[up]
        res = np.max(np.abs(d), initial=0.0)
        new = sg[up] + d
        if res < tol:
            sg = anti(new)
            break
        diis.push(new, d)
        sg = anti(diis.extrapolate())
    pairs = [(x, y) for x in range(na) for y in range(x + 1, na)]
    I = np.eye(na)
    Hp = np.array([[H1[z, x] * I[w, y] + I[z, x] * H1[w, y] - H1[w, x] * I[z, y] - I[w, x] * H1[z, y] + H2[z, w, x, y]
                    for x, y in pairs] for z, w in pairs])
    w = np.linalg.eigvals(Hp)
    return Hp, w[np.lexsort((w.imag, w.real))], res < tol
