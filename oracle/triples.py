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

Parity: pinned by tests/test_oracle_triples.py against explicit second quantisation
(the projections <mu3|H T2|0> and <mu3|H T1|0> on a determinant basis, then the same
sum), against zero for two electrons (no triples), and against the permutation
symmetry of c and d.
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
