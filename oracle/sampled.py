"""Oracle: selected elements of the CCSD right-hand sides where the dense integrals
do not fit (the o=40, v=200 workload needs ~53 GB), for full-size parity checks.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The recipe of ``oracle.integrals`` and the Stanton-Gauss equations of
``oracle.ccsd`` (Eq. (amplitudes) truncated to singles and doubles), evaluated
only on the rows and columns that the requested output elements use:

  * ``vblock(prob, P, Q, R, S)``: the unscaled <pq||rs> on the outer product of four
    global index lists -- antisymmetrise the seeded field, Hermitise, keep the
    symmetry-allowed irrep tuples (only those are generated);
  * ``mp2_scale``: 0.05 / max |<ab||ij> / D_ij^ab| from the (vv|oo) block;
  * ``rhs_elements``: R2_ij^ab and R1_i^a (the right-hand sides of D t = R) at
    listed index tuples, with every intermediate (F_ae, F_mi, F_me, W_mnij,
    W_abef, W_mbej) formed only for the rows / columns those elements read.

f is diagonal (f_ov = 0), as in the synthetic Hamiltonian.  Parity:
tests/test_oracle_sampled.py checks vblock against ``oracle.integrals`` and
rhs_elements against ``oracle.ccsd.rhs`` element by element on small problems.
"""
from __future__ import annotations

import numpy as np

from paper_2004_03682_gb300.synthetic import Problem, gaussian_tensor


def es(spec, *ops):
    return np.einsum(spec, *ops, optimize=True)


def _anti(prob: Problem, P, Q, R, S) -> np.ndarray:
    """A - A(qp rs) - A(pq sr) + A(qp sr) on the outer product P x Q x R x S."""
    def A(a, b, c, d):
        return gaussian_tensor(prob.seed, prob.n, a, b, c, d)
    return (A(P, Q, R, S) - A(Q, P, R, S).transpose(1, 0, 2, 3)
            - A(P, Q, S, R).transpose(0, 1, 3, 2) + A(Q, P, S, R).transpose(1, 0, 3, 2))


def vblock(prob: Problem, P, Q, R, S) -> np.ndarray:
    """Unscaled <pq||rs> for p in P, q in Q, r in R, s in S (global indices)."""
    P, Q, R, S = (np.atleast_1d(np.asarray(x, dtype=np.int64)) for x in (P, Q, R, S))
    irr, G = prob.irrep_of, prob.G
    out = np.zeros((len(P), len(Q), len(R), len(S)), dtype=np.complex128)

    def groups(X):
        return [np.nonzero(irr[X] == g)[0] for g in range(G)]

    gP, gQ, gR, gS = groups(P), groups(Q), groups(R), groups(S)
    for a in range(G):
        for b in range(G):
            for c in range(G):
                d = (a + b - c) % G  # allowed: G_p + G_q - G_r - G_s = 0 mod G
                ip, iq, ir, js = gP[a], gQ[b], gR[c], gS[d]
                if not (len(ip) and len(iq) and len(ir) and len(js)):
                    continue
                p, q, r, s = P[ip], Q[iq], R[ir], S[js]
                h = 0.5 * (_anti(prob, p, q, r, s) + _anti(prob, r, s, p, q).transpose(2, 3, 0, 1).conj())
                out[np.ix_(ip, iq, ir, js)] = h
    return out


def mp2_scale(prob: Problem, Vvvoo: np.ndarray) -> float:
    """s such that max |s <ab||ij> / D_ij^ab| = 0.05 (times the problem's scale_mult)."""
    eo, ev = prob.eps_occ, prob.eps_virt
    D = (eo[None, None, :, None] + eo[None, None, None, :] - ev[:, None, None, None] - ev[None, :, None, None])
    return 0.05 / np.max(np.abs(Vvvoo / D)) * prob.scale_mult


class Integrals:
    """Scaled integral slices of one problem, generated on demand and cached."""

    def __init__(self, prob: Problem):
        self.prob = prob
        o, n = prob.n_occ, prob.n
        self.occ = np.arange(o)
        self.vir = np.arange(o, n)
        Vvvoo = vblock(prob, self.vir, self.vir, self.occ, self.occ)
        self.s = mp2_scale(prob, Vvvoo)
        self.vvoo = self.s * Vvvoo
        # <ij||ab> = conj <ab||ij> (the recipe is exactly Hermitian)
        self.oovv = self.vvoo.transpose(2, 3, 0, 1).conj()
        self._cache = {}

    def get(self, key, P, Q, R, S):
        if key not in self._cache:
            self._cache[key] = self.s * vblock(self.prob, P, Q, R, S)
        return self._cache[key]

    # <m x||e f> for one virtual x: (o, v, v)
    def ovvv(self, x):
        return self.get(("ovvv", x), self.occ, self.vir[x], self.vir, self.vir)[:, 0]

    # <m n||y e> for one occupied y: (o, o, v)
    def ooov(self, y):
        return self.get(("ooov", y), self.occ, self.occ, y, self.vir)[:, :, 0, :]

    # <m n||e y>: (o, o, v)
    def oovo(self, y):
        return self.get(("oovo", y), self.occ, self.occ, self.vir, y)[:, :, :, 0]

    # <m x||e y>: (o, v)
    def ovvo(self, x, y):
        return self.get(("ovvo", x, y), self.occ, self.vir[x], self.vir, y)[:, 0, :, 0]

    # <n x||y f>: (o, v)
    def ovov(self, x, y):
        return self.get(("ovov", x, y), self.occ, self.vir[x], y, self.vir)[:, 0, 0, :]

    # <a b||e f>: (v, v)
    def vvvv(self, a, b):
        return self.get(("vvvv", a, b), self.vir[a], self.vir[b], self.vir, self.vir)[0, 0]

    # <a b||e j>: (v,)
    def vvvo(self, a, b, j):
        return self.get(("vvvo", a, b, j), self.vir[a], self.vir[b], self.vir, j)[0, 0, :, 0]

    # <m b||i j>: (o,)
    def ovoo(self, b, i, j):
        return self.get(("ovoo", b, i, j), self.occ, self.vir[b], i, j)[:, 0, 0, 0]

    # <m n||i j>: (o, o)
    def oooo(self, i, j):
        return self.get(("oooo", i, j), self.occ, self.occ, i, j)[:, :, 0, 0]


def rhs_elements(prob: Problem, t1: np.ndarray, t2: np.ndarray, samples2, samples1, ints: Integrals = None):
    """R2[i, j, a, b] for (i, j, a, b) in samples2 and R1[i, a] for (i, a) in samples1
    (virtual indices local, 0..v-1), at amplitudes t1[i, a], t2[i, j, a, b]."""
    I = ints or Integrals(prob)
    Voovv = I.oovv
    tau = t2 + es("ia,jb->ijab", t1, t1) - es("ib,ja->ijab", t1, t1)
    tt = t2 + 0.5 * (es("ia,jb->ijab", t1, t1) - es("ib,ja->ijab", t1, t1))
    Fme = es("nf,mnef->me", t1, Voovv)

    fae, fbe, fmi, fmj, wmbej = {}, {}, {}, {}, {}

    def Fae(x):  # row x of F_ae
        if x not in fae:
            fae[x] = es("mf,mfe->e", t1, I.ovvv(x)) - 0.5 * es("mnf,mnef->e", tt[:, :, x, :], Voovv)
        return fae[x]

    def Fbe(x):
        if x not in fbe:
            fbe[x] = Fae(x) - 0.5 * es("m,me->e", t1[:, x], Fme)
        return fbe[x]

    def Fmi(y):  # column y of F_mi
        if y not in fmi:
            fmi[y] = es("ne,mne->m", t1, I.ooov(y)) + 0.5 * es("nef,mnef->m", tt[y], Voovv)
        return fmi[y]

    def Fmj(y):
        if y not in fmj:
            fmj[y] = Fmi(y) + 0.5 * es("e,me->m", t1[y], Fme)
        return fmj[y]

    def Wmbej(x, y):  # W[m, x, e, y] over (m, e)
        if (x, y) not in wmbej:
            zeta = 0.5 * t2[y, :, :, x] + es("f,n->nf", t1[y], t1[:, x])  # zeta_yn^fx over (n, f)
            wmbej[(x, y)] = (I.ovvo(x, y) + es("f,mef->me", t1[y], I.ovvv(x))
                             - es("n,mne->me", t1[:, x], I.oovo(y))
                             - es("nf,mnef->me", zeta, Voovv))
        return wmbej[(x, y)]

    def ring(i, j, a, b):
        return (es("me,me->", t2[i, :, a, :], Wmbej(b, j))
                - es("e,m,me->", t1[i], t1[:, a], I.ovvo(b, j)))

    out2 = []
    for (i, j, a, b) in samples2:
        Wmn = (I.oooo(i, j) + es("e,mne->mn", t1[j], I.ooov(i)) - es("e,mne->mn", t1[i], I.ooov(j))
               + 0.25 * es("ef,mnef->mn", tau[i, j], Voovv))
        Wab = (I.vvvv(a, b) - (es("m,mef->ef", t1[:, b], -I.ovvv(a)) - es("m,mef->ef", t1[:, a], -I.ovvv(b)))
               + 0.25 * es("mn,mnef->ef", tau[:, :, a, b], Voovv))
        r = (I.vvoo[a, b, i, j]
             + (t2[i, j, a, :] @ Fbe(b) - t2[i, j, b, :] @ Fbe(a))
             - (t2[i, :, a, b] @ Fmj(j) - t2[j, :, a, b] @ Fmj(i))
             + 0.5 * es("mn,mn->", tau[:, :, a, b], Wmn)
             + 0.5 * es("ef,ef->", tau[i, j], Wab)
             + ring(i, j, a, b) - ring(i, j, b, a) - ring(j, i, a, b) + ring(j, i, b, a)
             + (t1[i] @ I.vvvo(a, b, j) - t1[j] @ I.vvvo(a, b, i))
             - (t1[:, a] @ I.ovoo(b, i, j) - t1[:, b] @ I.ovoo(a, i, j)))
        out2.append(complex(r))
    out1 = []
    for (i, a) in samples1:
        r = (t1[i] @ Fae(a) - t1[:, a] @ Fmi(i) + es("me,me->", t2[i, :, a, :], Fme)
             - es("nf,nf->", t1, I.ovov(a, i))
             - 0.5 * es("mef,mef->", t2[i], I.ovvv(a))
             - 0.5 * es("mne,nme->", t2[:, :, a, :], I.oovo(i)))
        out1.append(complex(r))
    return np.array(out2), np.array(out1)
