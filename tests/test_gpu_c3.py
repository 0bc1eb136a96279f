"""GPU parity at the precision workload the bench times: o=60, v=400, Z8 (seed 3001),
pair-packed products.  The dense oracle cannot hold these integrals (0.7 TB), so the
expected values are the right-hand sides R1, R2 of one iteration at seeded trial
amplitudes (t1 != 0: every term contributes) on 128 R2 and 120 R1 elements spread over
all irreps, written by tests/golden/make_sampled.py from oracle/sampled.py.

Both GPU paths run one iteration from those amplitudes (plain update t_new = R/D, so
R = D t_new):
  * FP64: within 1e-11 of the element's scale;
  * emulated, six BF16 slices (the bench's count): within 1e-8 of the element's scale.
An element's scale is its own |R| plus the largest sampled |R| of its pair-irrep block
(R2) or irrep (R1): the emulation's error follows the row and column magnitudes of the
products, not the element's own size, which can be small through cancellation."""
import json
import os

import numpy as np
import pytest

from paper_2004_03682_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "rhs_z8_o60_v400.json")


@pytest.fixture(scope="module")
def expgb():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2004_03682_gb300 import build, expgb as e
    build.build()
    e.lib()
    return e


@pytest.fixture(scope="module")
def case():
    g = json.load(open(GOLDEN))
    prob = syn.make_problem(g["seed"], g["n_occ"], g["n_virt"], g["G"])
    t1, t2 = syn.trial_amplitudes(prob, g["trial_seed"])
    s2 = [tuple(x) for x in g["samples2"]]
    s1 = [tuple(x) for x in g["samples1"]]
    r2 = np.array([complex(*z) for z in g["r2"]])
    r1 = np.array([complex(*z) for z in g["r1"]])
    irr = prob.irrep_of
    o, G = prob.n_occ, prob.G
    # per-element scale: own |R| + the largest sampled |R| of its pair irrep / irrep
    k2 = np.array([(irr[i] + irr[j]) % G for i, j, a, b in s2])
    k1 = np.array([irr[i] for i, a in s1])
    m2 = np.array([np.max(np.abs(r2[k2 == k])) for k in k2])
    m1 = np.array([np.max(np.abs(r1[k1 == k])) for k in k1])
    return dict(g=g, prob=prob, t1=t1, t2=t2, s2=s2, s1=s1, r2=r2, r1=r1,
                scale2=np.abs(r2) + m2, scale1=np.abs(r1) + m1)


def _one_iteration(expgb, case, precision, slices):
    import torch
    prob = case["prob"]
    ctx = expgb.from_problems([prob], precision=precision, n_slices=slices, diis_dim=0, conv_tol=1e-30,
                              max_iter=3)
    scale = ctx.init_integrals([prob.seed])[0]
    ctx.set_amplitudes(0, torch.from_numpy(case["t1"]), torch.from_numpy(case["t2"]))
    ctx.iterate(1)
    n1, n2 = ctx.get_amplitudes(0)
    ctx.close()
    i2 = torch.tensor(np.array(case["s2"]).T, device=n2.device)
    i1 = torch.tensor(np.array(case["s1"]).T, device=n1.device)
    g2 = n2[i2[0], i2[1], i2[2], i2[3]].cpu().numpy()
    g1 = n1[i1[0], i1[1]].cpu().numpy()
    del n1, n2
    torch.cuda.empty_cache()
    eo, ev = prob.eps_occ, prob.eps_virt
    d2 = np.array([eo[i] + eo[j] - ev[a] - ev[b] for i, j, a, b in case["s2"]])
    d1 = np.array([eo[i] - ev[a] for i, a in case["s1"]])
    return scale, g2 * d2, g1 * d1


def test_sample_spread(case):
    """The samples cover every pair irrep of R2 and every occupied irrep of R1."""
    prob = case["prob"]
    irr, G, o = prob.irrep_of, prob.G, prob.n_occ
    pairs = {(irr[i] + irr[j]) % G for i, j, a, b in case["s2"]}
    assert len(case["s2"]) >= 100 and len(case["s1"]) >= 100
    allowed = {(irr[i] + irr[j]) % G for i in range(o) for j in range(o) if i != j}
    assert pairs == allowed
    assert {irr[i] for i, a in case["s1"]} == {irr[i] for i in range(o)}


@pytest.mark.parametrize("path", ["fp64", "emu6"])
def test_c3_rhs_samples_match_oracle(expgb, case, path):
    prec, S, rel = (expgb.EXP_FP64, 5, 1e-11) if path == "fp64" else (expgb.EXP_EMU_BF16, 6, 1e-8)
    scale, g2, g1 = _one_iteration(expgb, case, prec, S)
    assert abs(scale - case["g"]["mp2_scale"]) <= 1e-13 * scale
    e2 = np.abs(g2 - case["r2"]) / case["scale2"]
    e1 = np.abs(g1 - case["r1"]) / case["scale1"]
    print(f"{path}: max rel error R2 {e2.max():.3e} R1 {e1.max():.3e}")
    assert e2.max() < rel, (e2.max(), int(np.argmax(e2)))
    assert e1.max() < rel, (e1.max(), int(np.argmax(e1)))
