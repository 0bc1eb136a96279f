"""GPU parity for the (T) correction (exp_ccsd_t) against oracle/triples.py.

  * Per-triple energies element by element, and E(T), from converged GPU CCSD
    amplitudes read back (so both sides take the same inputs):
      - FP64 path within 1e-12 of the largest triple energy;
      - emulated path (6 BF16 slices) within 1e-9 of it.
  * The same at seeded trial amplitudes with t1 != 0 (the disconnected term at full
    weight).
  * Every occupied block size gives the same bits (FP64 and emulated): the schedule
    changes the block products, not the arithmetic of any element.
  * Degenerate cases:
      - fewer than three occupied spinors (no triples, E(T) = 0);
      - Z8 with small spaces (empty irreps and empty products);
      - three virtual spinors (one a<b<c).
  * The full-size workload o=40 v=200 Z8: sampled triples against
    tests/golden/t3_z8_o40_v200.json (oracle.triples.triple_energy).
  * Call-order errors: before any amplitudes exist, and in a context with an active
    space."""
import json
import os

import numpy as np
import pytest

from oracle import ccsd, integrals, triples
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


def _oracle(prob):
    return ccsd.Blocks(integrals.integrals(prob), integrals.fock(prob), prob.n_occ)


def _tri_index(o):
    """(i, j, k) of each position C(k,3) + C(j,2) + i of the per-triple output."""
    out = {}
    for k in range(o):
        for j in range(k):
            for i in range(j):
                out[k * (k - 1) * (k - 2) // 6 + j * (j - 1) // 2 + i] = (i, j, k)
    return [out[n] for n in range(len(out))]


def _compare(e_gpu, E_gpu, e_orc, o, rel):
    ref = np.array([e_orc[t] for t in _tri_index(o)])
    scale = max(np.max(np.abs(ref)), 1e-300)
    np.testing.assert_allclose(e_gpu, ref, atol=rel * scale, rtol=0)
    assert abs(E_gpu - np.sum(ref)) <= rel * scale * max(len(ref), 1)


def _converged(expgb, prob, precision, S=6):
    ctx = expgb.from_problems([prob], conv_tol=1e-10, max_iter=400, precision=precision, n_slices=S,
                              emu_min_macs=1e3)
    ctx.init_integrals([prob.seed])
    _, conv, _ = ctx.iterate(400)
    assert conv
    return ctx


@pytest.mark.parametrize("precision,rel", [(0, 1e-12), (1, 1e-9)])
@pytest.mark.parametrize("seed,no,nv,G", [(801, 4, 12, 2), (802, 6, 20, 4), (803, 8, 32, 1), (804, 5, 19, 8)])
def test_triples_from_converged_amplitudes(expgb, seed, no, nv, G, precision, rel):
    prob = syn.make_problem(seed, no, nv, G)
    ctx = _converged(expgb, prob, precision)
    t1, t2 = (x.cpu().numpy() for x in ctx.get_amplitudes(0))
    E, info, e3 = ctx.ccsd_t(0, per_triple=True)
    ctx.close()
    assert info["n_triples"] == no * (no - 1) * (no - 2) // 6
    assert info["macs"] > 0 and info["macs_run"] >= info["macs"]
    _compare(e3, E, triples.per_triple(t1, t2, _oracle(prob)), no, rel)


@pytest.mark.parametrize("precision,rel", [(0, 1e-12), (1, 1e-9)])
@pytest.mark.parametrize("seed,no,nv,G", [(811, 6, 16, 2), (812, 7, 22, 4)])
def test_triples_at_trial_amplitudes(expgb, seed, no, nv, G, precision, rel):
    import torch
    prob = syn.make_problem(seed, no, nv, G)
    t1, t2 = syn.trial_amplitudes(prob, seed + 5)
    ctx = expgb.from_problems([prob], precision=precision, n_slices=6)
    ctx.init_integrals([prob.seed])
    ctx.set_amplitudes(0, torch.from_numpy(t1), torch.from_numpy(t2))
    E, info, e3 = ctx.ccsd_t(0, per_triple=True)
    ctx.close()
    b = _oracle(prob)
    _compare(e3, E, triples.per_triple(t1, t2, b), no, rel)
    # the disconnected term matters here: dropping t1 moves the energy
    E0 = triples.energy(np.zeros_like(t1), t2, b)
    assert abs(E - E0) > 1e3 * rel * abs(E)


@pytest.mark.parametrize("precision", [0, 1])
def test_triples_bits_independent_of_block_size(expgb, precision):
    prob = syn.make_problem(821, 9, 24, 4)
    ctx = _converged(expgb, prob, precision)
    runs = [ctx.ccsd_t(0, per_triple=True, block=nb) for nb in (0, 1, 2, 4, 5, 9)]
    ctx.close()
    assert [r[1]["block"] for r in runs[1:]] == [1, 2, 4, 5, 9]
    for E, info, e3 in runs[1:]:
        assert E == runs[0][0]
        assert np.array_equal(e3, runs[0][2])


@pytest.mark.parametrize("seed,no,nv,G", [(831, 2, 10, 1), (832, 3, 3, 1), (833, 6, 9, 8), (834, 4, 14, 16)])
def test_triples_degenerate_cases(expgb, seed, no, nv, G):
    prob = syn.make_problem(seed, no, nv, G)
    ctx = _converged(expgb, prob, 0)
    t1, t2 = (x.cpu().numpy() for x in ctx.get_amplitudes(0))
    E, info, e3 = ctx.ccsd_t(0, per_triple=True)
    ctx.close()
    if no < 3:
        assert E == 0 and info["n_triples"] == 0
        return
    _compare(e3, E, triples.per_triple(t1, t2, _oracle(prob)), no, 1e-12)


def test_triples_call_order_errors(expgb):
    prob = syn.make_problem(841, 4, 12, 2)
    ctx = expgb.from_problems([prob])
    with pytest.raises(expgb.ExpError) as ei:
        ctx.ccsd_t(0)
    assert ei.value.status == expgb.EXP_ESTATE
    ctx.init_integrals([prob.seed])
    with pytest.raises(expgb.ExpError) as ei:
        ctx.ccsd_t(0)  # no amplitudes yet
    assert ei.value.status == expgb.EXP_ESTATE
    ctx.iterate(1)
    with pytest.raises(expgb.ExpError) as ei:
        ctx.ccsd_t(0, block=-1)
    assert ei.value.status == expgb.EXP_EINVAL
    with pytest.raises(expgb.ExpError) as ei:
        ctx.ccsd_t(1)
    assert ei.value.status == expgb.EXP_EINVAL
    ctx.close()
    fs = expgb.from_problems([prob], active=syn.active_virtuals(prob, 2))
    fs.init_integrals([prob.seed])
    fs.iterate(1)
    with pytest.raises(expgb.ExpError) as ei:
        fs.ccsd_t(0)
    assert ei.value.status == expgb.EXP_ESTATE
    fs.close()


GOLDEN = os.path.join(HERE, "golden", "t3_z8_o40_v200.json")


@pytest.mark.parametrize("precision,rel", [(0, 1e-11), (1, 1e-8)])
def test_triples_full_size_sampled(expgb, precision, rel):
    """o=40 v=200 Z8 at seeded trial amplitudes: the per-triple energies of the sampled
    triples against the oracle's, within rel of the largest sampled |e_ijk|."""
    import torch
    g = json.load(open(GOLDEN))
    prob = syn.make_problem(g["seed"], g["n_occ"], g["n_virt"], g["G"])
    t1, t2 = syn.trial_amplitudes(prob, g["trial_seed"])
    ctx = expgb.from_problems([prob], precision=precision, n_slices=6)
    scale = ctx.init_integrals([prob.seed])[0]
    assert abs(scale - g["mp2_scale"]) <= 1e-13 * scale
    ctx.set_amplitudes(0, torch.from_numpy(t1), torch.from_numpy(t2))
    del t1, t2
    E, info, e3 = ctx.ccsd_t(0, per_triple=True)
    ctx.close()
    ref = np.array([complex(*z) for z in g["e3"]])
    got = np.array([e3[k * (k - 1) * (k - 2) // 6 + j * (j - 1) // 2 + i] for i, j, k in g["triples"]])
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    print(f"precision {precision}: max rel error {err:.3e}, E(T) {E:.12f}, {info['ms']:.1f} ms, block {info['block']}")
    assert err < rel
