"""Write sampled right-hand-side values of full-size workloads (calls only oracle/ and
the seeded input module).

    python tests/golden/make_sampled.py [c3]

For the precision workload o=60, v=400, Z8 (seed 3001): R2_ij^ab and R1_i^a of the CCSD
equations (oracle/sampled.py, the right-hand sides of D t = R) at seeded trial
amplitudes (synthetic.trial_amplitudes, seed 17: t1 != 0, so every term contributes),
on sampled elements spread over all irreps: one virtual spinor per irrep and nine
occupied spinors for R2 (every symmetry-allowed i<j, a<b), two virtuals per irrep and
all occupied spinors for R1.  The dense oracle cannot hold these integrals (0.7 TB), so
the oracle evaluates each requested element from integral slices generated on demand.
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


if __name__ == "__main__":
    which = sys.argv[1:] or ["c3"]
    if "c3" in which:
        sampled_rhs(C3)
