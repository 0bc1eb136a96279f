"""Oracle: the perturbative triples correction (T) to CCSD, complex128, dense.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper lists CCSD(T) among its models (Sec. III.A, the model list).  For a
Hartree-Fock reference (f diagonal, f_ov = 0) the triples enter through two projections
of the Hamiltonian on the triple excitations |ijk->abc> = a+ b+ c+ k j i |0>:

  connected     c_ijk^abc = <ijk->abc| H_N T2 |0>
                          = P(i/jk) P(a/bc) [ sum_e <bc||ei> t_jk^ae - sum_m <ma||jk> t_im^bc ]
  disconnected  d_ijk^abc = <ijk->abc| V_N T1 |0> = P(i/jk) P(a/bc) t_i^a <bc||jk>

with P(i/jk) f = f - f(i<->j) - f(i<->k) (and P(a/bc) likewise), the integrals in the
<created created||annihilated annihilated> convention.  The triples amplitudes of second
order are t3 = c / D, D_ijk^abc = e_i + e_j + e_k - e_a - e_b - e_c, and (T) takes T1^+ and
T2^+ for the left state:

  E(T) = E[4]_T + E[5]_ST = sum over i<j<k, a<b<c of conj(c + d) c / D.

The energy splits over the occupied triples: e_ijk = sum over a<b<c of conj(c + d) c / D
for one i<j<k, and E(T) = sum over i<j<k of e_ijk.  ``per_triple`` gives every e_ijk from
the dense arrays; ``triple_energy`` gives one e_ijk from integral slices generated on
demand (oracle.sampled), for workloads whose dense integrals do not fit in memory.

Parity: pinned by tests/test_oracle_triples.py against explicit second quantisation
(the projections <mu3|H T2|0> and <mu3|H T1|0> on a determinant basis, then the same
sum), against zero for two electrons (no triples), and against the permutation
symmetry of c and d; per_triple against energy (the split is exact), triple_energy
against per_triple element by element.
"""
from __future__ import annotations

import numpy as np

from oracle import ccsd


def es(spec, *ops):
    return np.einsum(spec, *ops, optimize=True)


def _P3(x, axes):
    """P(p/qr) on three axes of x: x - x(p<->q) - x(p<->r)."""
    p, q, r = axes
    return x - x.swapaxes(p, q) - x.swapaxes(p, r)


def triples(t1, t2, b: ccsd.Blocks):
    """(c, d) as dense arrays [i, j, k, a, b, c]."""
    X = es("jkae,bcei->ijkabc", t2, b.v("vvvo")) - es("imbc,majk->ijkabc", t2, b.v("ovoo"))
    c = _P3(_P3(X, (0, 1, 2)), (3, 4, 5))
    Y = es("ia,bcjk->ijkabc", t1, b.v("vvoo"))
    d = _P3(_P3(Y, (0, 1, 2)), (3, 4, 5))
    return c, d


def denominators3(b: ccsd.Blocks):
    eo, ev = b.eps_o, b.eps_v
    return (eo[:, None, None, None, None, None] + eo[None, :, None, None, None, None]
            + eo[None, None, :, None, None, None] - ev[None, None, None, :, None, None]
            - ev[None, None, None, None, :, None] - ev[None, None, None, None, None, :])


def energy(t1, t2, b: ccsd.Blocks) -> complex:
    """E(T) = sum over i<j<k, a<b<c of conj(c + d) c / D (= 1/36 of the unrestricted sum)."""
    c, d = triples(t1, t2, b)
    D = denominators3(b)
    return complex(np.sum(np.conj(c + d) * c / D) / 36.0)


def per_triple(t1, t2, b: ccsd.Blocks) -> np.ndarray:
    """e[i, j, k] = sum over a<b<c of conj(c + d) c / D for i<j<k, zero elsewhere."""
    c, d = triples(t1, t2, b)
    D = denominators3(b)
    full = np.sum(np.conj(c + d) * c / D, axis=(3, 4, 5)) / 6.0  # the abc sum is 6 x the a<b<c sum
    o = full.shape[0]
    i, j, k = np.meshgrid(np.arange(o), np.arange(o), np.arange(o), indexing="ij")
    return np.where((i < j) & (j < k), full, 0.0)


def triple_energy(prob, ints, t1, t2, i: int, j: int, k: int) -> complex:
    """e_ijk for one occupied triple i<j<k (local indices), from the definitions above with
    the integral slices it reads generated by ``ints`` (an oracle.sampled.Integrals of prob):
    <bc||ep> for p in (i, j, k), <ma||qr> for the three pairs (q, r), <bc||yz> and the
    orbital energies.  t1[i, a], t2[i, j, a, b] dense (virtual indices local)."""
    occ, vir = ints.occ, ints.vir

    def Vvvvo(p):  # <b c || e p>: (v, v, v)
        return ints.get(("t3_vvvo", p), vir, vir, vir, np.array([p]))[:, :, :, 0]

    def Vovoo(q, r):  # <m a || q r>: (o, v)
        return ints.get(("t3_ovoo", q, r), occ, vir, np.array([q]), np.array([r]))[:, :, 0, 0]

    def Xc(p, q, r):  # sum_e t_qr^ae <bc||ep> - sum_m t_pm^bc <ma||qr>, as [a, b, c]
        return es("ae,bce->abc", t2[q, r], Vvvvo(p)) - es("mbc,ma->abc", t2[p], Vovoo(q, r))

    def Pabc(y):  # P(a/bc) on axes (a, b, c)
        return y - y.transpose(1, 0, 2) - y.transpose(2, 1, 0)

    c = Pabc(Xc(i, j, k) - Xc(j, i, k) - Xc(k, j, i))
    vvoo = ints.vvoo  # <b c || y z>, [b, c, y, z]

    def Yd(x, y, z):  # t_x^a <bc||yz>, as [a, b, c]
        return es("a,bc->abc", t1[x], vvoo[:, :, y, z])

    d = Pabc(Yd(i, j, k) - Yd(j, i, k) - Yd(k, j, i))
    eo, ev = prob.eps_occ, prob.eps_virt
    D = eo[i] + eo[j] + eo[k] - ev[:, None, None] - ev[None, :, None] - ev[None, None, :]
    return complex(np.sum(np.conj(c + d) * c / D) / 6.0)
