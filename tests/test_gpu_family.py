"""The learned-guess family (o=10 v=40 C1; integral scale x U[0.5,1.5], virtual floor
U[0.1,0.6]; members 0..447 train, 448..511 held out) on the GPU:

  * all 512 members in one context (every launch covers all instances, emulated
    contractions): members 0, 17 and the last held-out member whose oracle solve
    converges match their single-instance oracle energies (tests/golden/
    family_o10_v40.json, converged to 1e-12) within 1e-8 Eh; every instance ends
    converged or frozen as failed;
  * the learned guess: the MLP trained by the project's kernels on the 448 training
    members' converged amplitudes lowers the held-out median iteration count strictly
    below that of the MP2 guess, with the same members converging and every converged
    energy within 1e-10 Eh of the MP2-guess one."""
import json
import os

import numpy as np
import pytest

from paper_2004_03682_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def expgb():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2004_03682_gb300 import build, expgb as e
    build.build()
    e.lib()
    return e


def test_512_instance_batch_matches_single_instance_oracle(expgb):
    g = json.load(open(os.path.join(HERE, "golden", "family_o10_v40.json")))
    probs = [syn.family_member(k) for k in range(512)]
    ctx = expgb.from_problems(probs, precision=expgb.EXP_EMU_BF16, n_slices=5, conv_tol=1e-9, max_iter=1500)
    ctx.init_integrals([p.seed for p in probs], scale_mult=[p.scale_mult for p in probs])
    recs, conv, st = ctx.iterate(1500, raise_numeric=False)
    states = np.array([ctx.state(k) for k in range(512)])
    print(f"512 members: {np.sum(states == 1)} converged, {np.sum(states == 2)} failed, "
          f"{np.sum(states == 0)} still iterating after {len(recs)} iterations")
    assert np.sum(states == 1) >= 150 and np.sum(states == 2) >= 1  # both outcomes occur in one batch
    checked = 0
    for key, m in g["members"].items():
        k = int(key)
        if not m["converged"]:
            continue
        assert states[k] == 1, f"member {k} did not converge on the GPU"
        e = ctx.energy(k)
        assert abs(e - complex(m["e_re"], m["e_im"])) < 1e-8, (k, e, m)
        checked += 1
    assert checked == 3
    ctx.close()


def test_learned_guess_lowers_heldout_median_iterations(expgb):
    from paper_2004_03682_gb300 import learned
    # residual 2e-11: the energy of a member is then within a few 1e-11 of its fixed point
    # (at 5e-11 the learned- and MP2-guess energies still differ by up to 1.6e-10)
    r = learned.family_experiment(n_train=448, n_test=64, epochs=20, conv_tol=2e-11, max_iter=1500)
    mp2, mlp = np.array(r["mp2_iters"]), np.array(r["mlp_iters"])
    print(f"held-out median iterations: MP2 {np.median(mp2)}, learned {np.median(mlp)}; "
          f"converged {r['mp2_conv']} / {r['mlp_conv']} of 64; max |dE| {r['max_dE']:.2e}")
    assert r["losses"][-1] < r["losses"][0]
    # members whose MP2-guess solve diverges (frozen as failed) stay out of both counts; a
    # member at the DIIS floor near 2e-11 may converge on one path only
    assert abs(r["mlp_conv"] - r["mp2_conv"]) <= 1 and r["mp2_conv"] >= 24
    assert np.median(mlp) < np.median(mp2)
    assert r["max_dE"] < 1e-10
