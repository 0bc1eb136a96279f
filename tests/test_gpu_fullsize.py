"""GPU parity at the full bench size, in the configuration bench.py times: o=40,
v=200, Z8 (seed 2001), emulated contractions with 5 BF16 slices, pair-packed tau
products, level shift 8.  The dense oracle cannot hold these integrals (~53 GB), so
the check runs on sampled output elements that oracle/sampled.py computes one by
one: the right-hand sides R1, R2 of one iteration started from seeded amplitudes
with t1 != 0 (every term of the equations contributes)."""
import numpy as np
import pytest

from oracle import sampled
from paper_2004_03682_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

SEED, NO, NV, G, SHIFT = 2001, 40, 200, 8, 8.0


@pytest.fixture(scope="module")
def expgb():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2004_03682_gb300 import build, expgb as e
    build.build()
    e.lib()
    return e


def _samples(prob, rng, n2=16, n1=12):
    irr, no, nv = prob.irrep_of, prob.n_occ, prob.n_virt
    occ = rng.choice(no, size=8, replace=False)
    vir = rng.choice(nv, size=10, replace=False)
    s2 = []
    while len(s2) < n2:
        i, j = rng.choice(occ, 2, replace=False)
        a = rng.choice(vir)
        cand = [b for b in range(nv) if b != a and (irr[i] + irr[j] - irr[no + a] - irr[no + b]) % prob.G == 0]
        if cand:
            s2.append((int(i), int(j), int(a), int(rng.choice(cand))))
    s1 = []
    for i in occ:
        cand = [a for a in range(nv) if irr[i] == irr[no + a]]
        if cand:
            s1.append((int(i), int(rng.choice(cand))))
    return s2, s1[:n1]


def test_fullsize_rhs_samples_match_oracle(expgb):
    import torch
    prob = syn.make_problem(SEED, NO, NV, G)
    t1, t2 = syn.trial_amplitudes(prob, 17)
    ctx = expgb.from_problems([prob], precision=expgb.EXP_EMU_BF16, n_slices=5, diis_dim=0, conv_tol=1e-30,
                              max_iter=5, level_shift=SHIFT)
    scale = ctx.init_integrals([prob.seed])[0]
    ctx.set_amplitudes(0, torch.from_numpy(t1), torch.from_numpy(t2))
    ctx.iterate(1)
    n1, n2 = (x.cpu().numpy() for x in ctx.get_amplitudes(0))
    ctx.close()

    rng = np.random.default_rng(5)
    s2, s1 = _samples(prob, rng)
    eo, ev = prob.eps_occ, prob.eps_virt
    # the update is t_new = (R - sigma t) / (D - sigma): recover R from the GPU iterate
    g2 = np.array([n2[s] * (eo[s[0]] + eo[s[1]] - ev[s[2]] - ev[s[3]] - SHIFT) + SHIFT * t2[s] for s in s2])
    g1 = np.array([n1[s] * (eo[s[0]] - ev[s[1]] - SHIFT) + SHIFT * t1[s] for s in s1])

    I = sampled.Integrals(prob)
    assert abs(I.s - scale) <= 1e-13 * scale  # the generator's MP2 scale, computed independently
    r2, r1 = sampled.rhs_elements(prob, t1, t2, s2, s1, I)
    # 5 slices of 7 bits: each emulated product carries a relative error of about
    # 2^-32 of its operands' row / column maxima; 1e-8 of the largest sampled R
    # leaves two orders of magnitude over what the tests at small sizes observe
    tol = 1e-8 * max(np.max(np.abs(r2)), np.max(np.abs(r1)))
    np.testing.assert_allclose(g2, r2, atol=tol, rtol=0)
    np.testing.assert_allclose(g1, r1, atol=tol, rtol=0)
    assert np.max(np.abs(r2)) > 0 and np.max(np.abs(r1)) > 0
