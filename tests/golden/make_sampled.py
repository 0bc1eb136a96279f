"""Write sampled right-hand-side values of full-size workloads (calls only oracle/ and
the seeded input module).

    python tests/golden/make_sampled.py [c3] [t3]

For the precision workload o=60, v=400, Z8 (seed 3001): R2_ij^ab and R1_i^a of the CCSD
equations (oracle/sampled.py, the right-hand sides of D t = R) at seeded trial
amplitudes (synthetic.trial_amplitudes, seed 17: t1 != 0, so every term contributes),
on sampled elements spread over all irreps: one virtual spinor per irrep and nine
occupied spinors for R2 (every symmetry-allowed i<j, a<b), two virtuals per irrep and
all occupied spinors for R1.  The dense oracle cannot hold these integrals (0.7 TB), so
the oracle evaluates each requested element from integral slices generated on demand.

For o=40, v=200, Z8 (seed 2001): the (T) energies e_ijk of sampled occupied triples at
seeded trial amplitudes (seed 23), from oracle/triples.py triple_energy.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import sampled  # noqa: E402
from paper_2004_03682_gb300 import synthetic as syn  # noqa: E402

C3 = dict(name="rhs_z8_o60_v400", seed=3001, n_occ=60, n_virt=400, G=8, trial_seed=17)
T3_C2 = dict(name="t3_z8_o40_v200", seed=2001, n_occ=40, n_virt=200, G=8, trial_seed=23)


def choose_samples(prob, n_occ_r2=9):
    """Deterministic sample lists: R2 over one virtual per irrep (the lowest index of
    each nonempty irrep) and n_occ_r2 occupied spinors spread over the occupied irreps;
    R1 over two virtuals per irrep and every occupied spinor of the same irrep."""
    o, v, G = prob.n_occ, prob.n_virt, prob.G
    irr = prob.irrep_of
    go, gv = irr[:o], irr[o:]
    vir1 = [int(np.nonzero(gv == g)[0][0]) for g in range(G) if np.any(gv == g)]
    vir2 = []
    for g in range(G):
        idx = np.nonzero(gv == g)[0]
        vir2 += [int(x) for x in idx[:1]] + ([int(idx[-1])] if len(idx) > 1 else [])
    # occupied: round-robin over irreps, lowest index first
    by = [list(np.nonzero(go == g)[0]) for g in range(G)]
    occ = []
    while len(occ) < n_occ_r2 and any(by):
        for g in range(G):
            if by[g] and len(occ) < n_occ_r2:
                occ.append(int(by[g].pop(0)))
    occ.sort()
    s2 = []
    for ii, i in enumerate(occ):
        for j in occ[ii + 1:]:
            for aa, a in enumerate(vir1):
                for b in vir1[aa + 1:]:
                    if (go[i] + go[j] - gv[a] - gv[b]) % G == 0:
                        s2.append((i, j, a, b))
    s1 = [(int(i), a) for a in vir2 for i in range(o) if go[i] == gv[a]]
    return s2, s1


def sampled_rhs(spec):
    prob = syn.make_problem(spec["seed"], spec["n_occ"], spec["n_virt"], spec["G"])
    t0 = time.perf_counter()
    t1, t2 = syn.trial_amplitudes(prob, spec["trial_seed"])
    I = sampled.Integrals(prob)
    s2, s1 = choose_samples(prob)
    r2, r1 = sampled.rhs_elements(prob, t1, t2, s2, s1, I)
    out = dict(spec, mp2_scale=I.s, samples2=s2, samples1=s1,
               r2=[[z.real, z.imag] for z in r2], r1=[[z.real, z.imag] for z in r1],
               seconds=time.perf_counter() - t0,
               source="oracle/sampled.py rhs_elements at synthetic.trial_amplitudes(prob, trial_seed)")
    path = os.path.join(HERE, spec["name"] + ".json")
    json.dump(out, open(path, "w"))
    print(path, len(s2), len(s1), out["seconds"])


def choose_triples(prob):
    """Deterministic occupied triples i<j<k: the lowest spinor of each nonempty occupied
    irrep, taken three at a time cyclically (mixed irreps), plus the three lowest spinors
    of the largest irrep (one irrep) and the three highest occupied spinors."""
    o, G = prob.n_occ, prob.G
    go = prob.irrep_of[:o]
    low = [int(np.nonzero(go == g)[0][0]) for g in range(G) if np.any(go == g)]
    tri = set()
    for n in range(len(low)):
        t = sorted({low[n], low[(n + 1) % len(low)], low[(n + 2) % len(low)]})
        if len(t) == 3:
            tri.add(tuple(t))
    big = int(np.argmax(np.bincount(go, minlength=G)))
    idx = [int(x) for x in np.nonzero(go == big)[0][:3]]
    if len(idx) == 3:
        tri.add(tuple(idx))
    tri.add((o - 3, o - 2, o - 1))
    return sorted(tri)


def sampled_t3(spec):
    """(T) energies e_ijk of sampled occupied triples at seeded trial amplitudes
    (oracle/triples.py triple_energy, integral slices from oracle/sampled.py)."""
    from oracle import triples
    prob = syn.make_problem(spec["seed"], spec["n_occ"], spec["n_virt"], spec["G"])
    t0 = time.perf_counter()
    t1, t2 = syn.trial_amplitudes(prob, spec["trial_seed"])
    I = sampled.Integrals(prob)
    tris = choose_triples(prob)
    e3 = [triples.triple_energy(prob, I, t1, t2, i, j, k) for i, j, k in tris]
    out = dict(spec, mp2_scale=I.s, triples=tris, e3=[[z.real, z.imag] for z in e3],
               seconds=time.perf_counter() - t0,
               source="oracle/triples.py triple_energy at synthetic.trial_amplitudes(prob, trial_seed)")
    path = os.path.join(HERE, spec["name"] + ".json")
    json.dump(out, open(path, "w"))
    print(path, len(tris), out["seconds"])


if __name__ == "__main__":
    which = sys.argv[1:] or ["c3"]
    if "c3" in which:
        sampled_rhs(C3)
    if "t3" in which:
        sampled_t3(T3_C2)
