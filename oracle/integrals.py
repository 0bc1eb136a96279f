"""Oracle: the synthetic relativistic Hamiltonian, dense.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The Hamiltonian has the second-quantised form of Eq. (ham): one-body part with
Fock matrix f = diag(eps) (Hartree-Fock spinors, so f is diagonal and f_ov = 0)
and antisymmetrised two-electron integrals V_pqrs = <pq||rs>, the coefficient
of (1/4) {p+ q+ s r}.  The synthetic recipe for V is:

    V  = A - A(qp rs) - A(pq sr) + A(qp sr)          (antisymmetrise)
    V <- (V_pqrs + conj V_rspq) / 2                  (Hermitise)
    V_pqrs = 0 unless  G_p + G_q - G_r - G_s = 0 mod G   (Abelian double group:
                                                     bra labels enter conjugated)
    V <- s V,  s = 0.05 / max_ijab |V_abij / D_ij^ab| (then x scale_mult)

with A the seeded complex Gaussian field and D_ij^ab = e_i + e_j - e_a - e_b.
Parity: pinned by tests/test_oracle_integrals.py (antisymmetry, Hermiticity,
forbidden blocks exactly zero, max |t_MP2| = 0.05).
"""
from __future__ import annotations

import numpy as np

from paper_2004_03682_gb300.synthetic import Problem, gaussian_tensor


def allowed_mask(irr: np.ndarray, G: int) -> np.ndarray:
    """Boolean n^4 mask of the symmetry-allowed integrals."""
    g = irr.astype(np.int64)
    s = (g[:, None, None, None] + g[None, :, None, None]
         - g[None, None, :, None] - g[None, None, None, :])
    return (s % G) == 0


def unscaled_integrals(prob: Problem) -> np.ndarray:
    """Antisymmetrised, Hermitised, symmetry-masked V before the MP2 scaling."""
    n = prob.n
    idx = np.arange(n)
    A = gaussian_tensor(prob.seed, n, idx, idx, idx, idx)
    V = A - A.transpose(1, 0, 2, 3) - A.transpose(0, 1, 3, 2) + A.transpose(1, 0, 3, 2)
    V = 0.5 * (V + V.transpose(2, 3, 0, 1).conj())
    V[~allowed_mask(prob.irrep_of, prob.G)] = 0.0
    return V


def denominators2(eps_o: np.ndarray, eps_v: np.ndarray) -> np.ndarray:
    """D_ij^ab = e_i + e_j - e_a - e_b, shape (o, o, v, v)."""
    return (eps_o[:, None, None, None] + eps_o[None, :, None, None]
            - eps_v[None, None, :, None] - eps_v[None, None, None, :])


def mp2_scale(V: np.ndarray, prob: Problem) -> float:
    """s such that max |s V_abij / D_ij^ab| = 0.05."""
    o = prob.n_occ
    Vabij = V[o:, o:, :o, :o].transpose(2, 3, 0, 1)
    m = np.max(np.abs(Vabij / denominators2(prob.eps_occ, prob.eps_virt)))
    return 0.05 / m


def integrals(prob: Problem) -> np.ndarray:
    """Dense scaled V (n, n, n, n) for a synthetic problem."""
    V = unscaled_integrals(prob)
    return V * (mp2_scale(V, prob) * prob.scale_mult)


def real_integrals(prob: Problem) -> np.ndarray:
    """The real-arithmetic variant of the recipe (Sec. II.C, Table `tab:time`: point groups
    whose spinor integrals are real): the real part of the antisymmetrised, Hermitised,
    symmetry-masked V -- the recipe applied to Re A, as every step is real-linear -- then
    scaled so that max |t_MP2| = 0.05 (times scale_mult).  Real, antisymmetric in each
    pair and symmetric under (pq) <-> (rs); stored complex with zero imaginary part."""
    V = unscaled_integrals(prob).real.astype(np.complex128)
    return V * (mp2_scale(V, prob) * prob.scale_mult)


def fock(prob: Problem) -> np.ndarray:
    return np.diag(prob.eps).astype(np.complex128)
