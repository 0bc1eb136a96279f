"""Brute-force second quantisation on a determinant basis (test helper).

Independent of the oracle's diagram algebra: operators act on occupation
bit-strings with the Jordan-Wigner sign, H is built from Eq. (ham) term by term,
and e^T is a finite power series (T is nilpotent).  Used to pin the oracle's
CCSD residual and energy, and the full-CI limits (two electrons for CCSD,
the electron-attached sector for FS-CCSD(0h1p)).
"""
from __future__ import annotations

import itertools
import numpy as np


def _apply_ann(p, det):
    if not (det >> p) & 1:
        return None, 0
    sign = -1 if bin(det & ((1 << p) - 1)).count("1") % 2 else 1
    return det ^ (1 << p), sign


def _apply_cre(p, det):
    if (det >> p) & 1:
        return None, 0
    sign = -1 if bin(det & ((1 << p) - 1)).count("1") % 2 else 1
    return det | (1 << p), sign


def apply_string(ops, det):
    """Apply a product of operators (rightmost first). ops: list of (p, dagger)."""
    sign = 1
    for p, dag in reversed(ops):
        det, s = (_apply_cre if dag else _apply_ann)(p, det)
        if det is None:
            return None, 0
        sign *= s
    return det, sign


class Space:
    """All determinants with `nel` electrons in `n` spinors."""

    def __init__(self, n: int, nel: int):
        self.n, self.nel = n, nel
        self.dets = [sum(1 << k for k in c) for c in itertools.combinations(range(n), nel)]
        self.index = {d: k for k, d in enumerate(self.dets)}

    def __len__(self):
        return len(self.dets)

    def operator(self, terms, target=None):
        """Matrix of sum_k c_k * (operator string k) from this space to `target`."""
        target = target or self
        M = np.zeros((len(target), len(self)), dtype=np.complex128)
        for coef, ops in terms:
            if coef == 0:
                continue
            for col, d in enumerate(self.dets):
                nd, s = apply_string(ops, d)
                if nd is not None and nd in target.index:
                    M[target.index[nd], col] += coef * s
        return M

    def vector(self, ops, det):
        v = np.zeros(len(self), dtype=np.complex128)
        nd, s = apply_string(ops, det)
        if nd is not None:
            v[self.index[nd]] = s
        return v


def hamiltonian_terms(h, V, thresh=0.0):
    """Eq. (ham): sum h_pq p+ q + 1/4 sum V_pqrs p+ q+ s r (not normal ordered)."""
    n = h.shape[0]
    terms = []
    for p in range(n):
        for q in range(n):
            if abs(h[p, q]) > thresh:
                terms.append((h[p, q], [(p, 1), (q, 0)]))
    for p, q, r, s in itertools.product(range(n), repeat=4):
        if abs(V[p, q, r, s]) > thresh:
            terms.append((0.25 * V[p, q, r, s], [(p, 1), (q, 1), (s, 0), (r, 0)]))
    return terms


def core_hamiltonian(f, V, o):
    """h_pq = f_pq - sum_k <pk||qk> (k occupied), and E_ref = sum_i h_ii + 1/2 sum_ij <ij||ij>."""
    h = f - np.einsum("pkqk->pq", V[:, :o, :, :o])
    eref = np.trace(h[:o, :o]) + 0.5 * np.einsum("ijij->", V[:o, :o, :o, :o])
    return h, complex(eref)


def cluster_terms(t1, t2, o):
    """T = sum t_i^a a+ i + 1/4 sum t_ij^ab a+ b+ j i (global indices: virt a -> o + a)."""
    no, nv = t1.shape
    terms = []
    for i in range(no):
        for a in range(nv):
            terms.append((t1[i, a], [(o + a, 1), (i, 0)]))
    for i, j, a, b in itertools.product(range(no), range(no), range(nv), range(nv)):
        terms.append((0.25 * t2[i, j, a, b], [(o + a, 1), (o + b, 1), (j, 0), (i, 0)]))
    return terms


def expm_nilpotent(T):
    out = np.eye(T.shape[0], dtype=np.complex128)
    term = out.copy()
    for k in range(1, T.shape[0] + 1):
        term = term @ T / k
        if not np.any(term):
            break
        out = out + term
    return out


def ccsd_projections(f, V, o, t1, t2):
    """Brute-force E = <0|e^-T H_N e^T|0> and residuals <mu|e^-T H_N e^T|0>."""
    n = f.shape[0]
    sp = Space(n, o)
    h, eref = core_hamiltonian(f, V, o)
    H = sp.operator(hamiltonian_terms(h, V)) - eref * np.eye(len(sp))
    T = sp.operator(cluster_terms(t1, t2, o))
    Hbar = expm_nilpotent(-T) @ H @ expm_nilpotent(T)
    ref = (1 << o) - 1
    phi0 = sp.vector([], ref)
    hp = Hbar @ phi0
    E = np.vdot(phi0, hp)
    no, nv = t1.shape
    R1 = np.zeros((no, nv), dtype=np.complex128)
    R2 = np.zeros((no, no, nv, nv), dtype=np.complex128)
    for i in range(no):
        for a in range(nv):
            R1[i, a] = np.vdot(sp.vector([(o + a, 1), (i, 0)], ref), hp)
    for i, j, a, b in itertools.product(range(no), range(no), range(nv), range(nv)):
        if i != j and a != b:
            R2[i, j, a, b] = np.vdot(sp.vector([(o + a, 1), (o + b, 1), (j, 0), (i, 0)], ref), hp)
    return E, R1, R2


def fci_correlation(f, V, o):
    """Lowest eigenvalue of H in the o-electron space, minus E_ref."""
    n = f.shape[0]
    sp = Space(n, o)
    h, eref = core_hamiltonian(f, V, o)
    H = sp.operator(hamiltonian_terms(h, V))
    w = np.linalg.eigvalsh(H)
    return float(w[0] - eref.real), eref


def sector_spectrum(f, V, o, nel):
    """All eigenvalues of H (minus E_ref of the o-electron vacuum) with `nel` electrons."""
    n = f.shape[0]
    sp = Space(n, nel)
    h, eref = core_hamiltonian(f, V, o)
    H = sp.operator(hamiltonian_terms(h, V))
    return np.linalg.eigvalsh(H) - eref.real


def ea_eom_matrix(f, V, o, t1, t2):
    """Electron-attached block of Hbar_N - E_CC on {a+|0>, a+ b+ j|0> (a<b)} by explicit
    second quantisation in the (o+1)-electron space.  Returns (M, labels)."""
    n = f.shape[0]
    nv = n - o
    h, eref = core_hamiltonian(f, V, o)
    sp0 = Space(n, o)
    sp1 = Space(n, o + 1)
    H0 = sp0.operator(hamiltonian_terms(h, V)) - eref * np.eye(len(sp0))
    T0 = sp0.operator(cluster_terms(t1, t2, o))
    Hbar0 = expm_nilpotent(-T0) @ H0 @ expm_nilpotent(T0)
    ref = (1 << o) - 1
    phi0 = sp0.vector([], ref)
    ecc = np.vdot(phi0, Hbar0 @ phi0)
    H1 = sp1.operator(hamiltonian_terms(h, V)) - eref * np.eye(len(sp1))
    T1 = sp1.operator(cluster_terms(t1, t2, o))
    Hbar1 = expm_nilpotent(-T1) @ H1 @ expm_nilpotent(T1)
    basis, labels = [], []
    for a in range(nv):
        basis.append(sp1.vector([(o + a, 1)], ref))
        labels.append(("p", a))
    for j in range(o):
        for a in range(nv):
            for b in range(a + 1, nv):
                basis.append(sp1.vector([(o + a, 1), (o + b, 1), (j, 0)], ref))
                labels.append(("pph", j, a, b))
    B = np.stack(basis, axis=1)
    M = B.conj().T @ Hbar1 @ B - ecc * np.eye(B.shape[1])
    return M, labels


def triples_energy(f, V, o, t1, t2):
    """(T) by explicit second quantisation: c_mu = <mu|H T2|0>, d_mu = <mu|H T1|0> on the
    triple excitations mu = a+ b+ c+ k j i |0> (i<j<k, a<b<c), E = sum conj(c + d) c / D_mu.
    H is the full Hamiltonian of Eq. (ham); for mu != 0 it projects like H_N.  f must be
    diagonal (a Hartree-Fock reference)."""
    n = f.shape[0]
    no, nv = t1.shape
    sp = Space(n, o)
    h, eref = core_hamiltonian(f, V, o)
    H = sp.operator(hamiltonian_terms(h, V))
    ref = (1 << o) - 1
    phi0 = sp.vector([], ref)
    T2 = sp.operator(cluster_terms(np.zeros_like(t1), t2, o))
    T1 = sp.operator(cluster_terms(t1, np.zeros_like(t2), o))
    cv = H @ (T2 @ phi0)
    dv = H @ (T1 @ phi0)
    eps = np.real(np.diag(f))
    E = 0.0 + 0.0j
    for i, j, k in itertools.combinations(range(no), 3):
        for a, b, c in itertools.combinations(range(nv), 3):
            mu = sp.vector([(o + a, 1), (o + b, 1), (o + c, 1), (k, 0), (j, 0), (i, 0)], ref)
            cm, dm = np.vdot(mu, cv), np.vdot(mu, dv)
            D = eps[i] + eps[j] + eps[k] - eps[o + a] - eps[o + b] - eps[o + c]
            E += np.conj(cm + dm) * cm / D
    return complex(E)
