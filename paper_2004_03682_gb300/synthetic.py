"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds only random draws: orbital energies, the irrep partition of
the spinors and the counter-based Gaussian field A_pqrs.  It performs none of
the coupled-cluster arithmetic, and none of the integral recipe (antisymmetrise,
Hermitise, scale), which each side implements on its own.

Counter-based generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11), written here from its published
definition.  A_pqrs = z_re + i z_im where (z_re, z_im) is the Box-Muller pair
of two 53-bit uniforms taken from one Philox block:

    counter = (lo32(idx), hi32(idx), 0, 0),   key = (lo32(seed), hi32(seed))
    idx     = ((p*n + q)*n + r)*n + s          (global spinor indices)
    u1 = ((x1<<32 | x0) >> 11 + 0.5) * 2^-53,  u2 likewise from (x3, x2)
    z  = sqrt(-2 ln u1) * (cos 2 pi u2, sin 2 pi u2)

Spinors are numbered occupied first (0..o-1) then virtual (o..o+v-1); inside
each space they are ordered by irrep, then by orbital energy.
"""
from __future__ import annotations

import dataclasses
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Philox4x32 with 10 rounds on uint64-held 32-bit lanes (arrays or scalars)."""
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK
    k0 &= 0xFFFFFFFF
    k1 &= 0xFFFFFFFF
    for r in range(10):
        if r:
            k0 = (k0 + _W0) & 0xFFFFFFFF
            k1 = (k1 + _W1) & 0xFFFFFFFF
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1,
                          hi0 ^ c3 ^ np.uint64(k1), lo0)
    return c0, c1, c2, c3


def gaussian_field(idx, seed: int) -> np.ndarray:
    """Complex standard-normal draws A[idx] (re and im each N(0,1))."""
    idx = np.asarray(idx, dtype=np.uint64)
    x0, x1, x2, x3 = philox4x32_10(idx & _MASK, idx >> _S32, 0, 0,
                                   seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    a = ((x1 << _S32) | x0) >> np.uint64(11)
    b = ((x3 << _S32) | x2) >> np.uint64(11)
    u1 = (a.astype(np.float64) + 0.5) * 2.0 ** -53
    u2 = (b.astype(np.float64) + 0.5) * 2.0 ** -53
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    return rad * np.cos(ang) + 1j * (rad * np.sin(ang))


def gaussian_tensor(seed: int, n: int, p, q, r, s) -> np.ndarray:
    """A[p, q, r, s] on the outer product of four global index arrays."""
    p = np.asarray(p, dtype=np.uint64).reshape(-1, 1, 1, 1)
    q = np.asarray(q, dtype=np.uint64).reshape(1, -1, 1, 1)
    r = np.asarray(r, dtype=np.uint64).reshape(1, 1, -1, 1)
    s = np.asarray(s, dtype=np.uint64).reshape(1, 1, 1, -1)
    nn = np.uint64(n)
    idx = ((p * nn + q) * nn + r) * nn + s
    return gaussian_field(idx, seed)


def _stream(seed: int, tag: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed & (2**64 - 1), tag]))


def irrep_counts(n: int, G: int, rng: np.random.Generator) -> np.ndarray:
    """Dirichlet(1,...,1) weights, counts by largest remainder (ties -> lower irrep)."""
    if G == 1:
        return np.array([n], dtype=np.int64)
    e = rng.exponential(1.0, size=G)
    w = e / e.sum()
    exact = w * n
    base = np.floor(exact).astype(np.int64)
    rem = exact - base
    order = sorted(range(G), key=lambda k: (-rem[k], k))
    for k in order[: n - int(base.sum())]:
        base[k] += 1
    return base


@dataclasses.dataclass
class Problem:
    """One synthetic Hamiltonian's seeded draws (no integrals)."""
    seed: int
    n_occ: int
    n_virt: int
    G: int
    irrep_occ: np.ndarray     # counts per irrep, occupied
    irrep_virt: np.ndarray    # counts per irrep, virtual
    eps_occ: np.ndarray       # ordered by irrep, then energy
    eps_virt: np.ndarray
    scale_mult: float = 1.0   # extra factor applied after the max|t_MP2| = 0.05 scaling

    @property
    def n(self) -> int:
        return self.n_occ + self.n_virt

    @property
    def irrep_of(self) -> np.ndarray:
        """Irrep label of every global spinor index."""
        occ = np.repeat(np.arange(self.G), self.irrep_occ)
        vir = np.repeat(np.arange(self.G), self.irrep_virt)
        return np.concatenate([occ, vir]).astype(np.int64)

    @property
    def eps(self) -> np.ndarray:
        return np.concatenate([self.eps_occ, self.eps_virt])


def _energies(counts, lo, hi, rng):
    out = []
    for c in counts:
        out.append(np.sort(rng.uniform(lo, hi, size=int(c))))
    return np.concatenate(out) if out else np.zeros(0)


def make_problem(seed: int, n_occ: int, n_virt: int, G: int = 1,
                 occ_range=(-2.0, -0.5), virt_range=(0.2, 5.0),
                 scale_mult: float = 1.0) -> Problem:
    """Seeded orbital energies and irrep partition (Dirichlet(1) over irreps)."""
    rng_irr = _stream(seed, 2)
    io = irrep_counts(n_occ, G, rng_irr)
    iv = irrep_counts(n_virt, G, rng_irr)
    rng_eps = _stream(seed, 1)
    eo = _energies(io, occ_range[0], occ_range[1], rng_eps)
    ev = _energies(iv, virt_range[0], virt_range[1], rng_eps)
    return Problem(seed, n_occ, n_virt, G, io, iv, eo, ev, float(scale_mult))


def family_member(k: int, n_occ: int = 10, n_virt: int = 40) -> Problem:
    """Member k of the learned-guess family: scale x U[0.5,1.5], virtual floor g ~ U[0.1,0.6]."""
    rng = _stream(4000 + k, 3)
    mult = float(rng.uniform(0.5, 1.5))
    gap = float(rng.uniform(0.1, 0.6))
    return make_problem(4000 + k, n_occ, n_virt, 1, virt_range=(gap, 5.0),
                        scale_mult=mult)


def active_virtuals(prob: Problem, n_act: int) -> np.ndarray:
    """Indices (within the virtual space) of the n_act lowest-energy virtual spinors."""
    order = np.lexsort((np.arange(prob.n_virt), prob.eps_virt))
    return np.sort(order[:n_act])


# Workloads named by their sizes.
CCSD_C1_O10_V40 = dict(n_occ=10, n_virt=40, G=1, seed=1001)
CCSD_Z8_O40_V200 = dict(n_occ=40, n_virt=200, G=8, seed=2001)
CCSD_Z8_O60_V400 = dict(n_occ=60, n_virt=400, G=8, seed=3001)
FS_Z16_O80_V480 = dict(n_occ=80, n_virt=480, G=16, seed=5001)


def trial_amplitudes(prob: Problem, seed: int, t1_max: float = 0.01, t2_max: float = 0.05):
    """Seeded amplitudes with the structure of CCSD ones, for residual checks away from
    the MP2 guess: t1[i, a] nonzero only for equal irreps, t2[i, j, a, b] antisymmetric
    in (i, j) and in (a, b) and nonzero only when the irreps of i + j and a + b agree
    (mod G); complex Gaussian entries scaled to the given maxima."""
    rng = _stream(seed, 7)
    o, v = prob.n_occ, prob.n_virt
    irr = prob.irrep_of
    go, gv = irr[:o], irr[o:]
    t1 = rng.standard_normal((o, v)) + 1j * rng.standard_normal((o, v))
    t1 *= (go[:, None] == gv[None, :])
    m1 = np.max(np.abs(t1))
    t1 *= (t1_max / m1) if m1 > 0 else 0.0
    x = rng.standard_normal((o, o, v, v)) + 1j * rng.standard_normal((o, o, v, v))
    t2 = x - x.transpose(1, 0, 2, 3) - x.transpose(0, 1, 3, 2) + x.transpose(1, 0, 3, 2)
    del x
    allowed = ((go[:, None, None, None] + go[None, :, None, None]
                - gv[None, None, :, None] - gv[None, None, None, :]) % prob.G) == 0
    t2 *= allowed
    m2 = np.max(np.abs(t2))
    t2 *= (t2_max / m2) if m2 > 0 else 0.0
    return t1, t2
