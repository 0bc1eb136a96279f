"""GPU: the learned-guess kernels against the FP64 MLP oracle, and the guess in use."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2004_03682_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def expgb():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    from paper_2004_03682_gb300 import build, expgb as e
    build.build()
    e.lib()
    return e


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    p = omlp.init_params(seed)
    k = omlp.NO * omlp.W + omlp.NO
    p[-k:] = 0.1 * rng.standard_normal(k)
    x = rng.uniform(0, 1, (n, omlp.NF)).astype(np.float32)
    tmp2 = (0.05 * (rng.standard_normal(n) + 1j * rng.standard_normal(n))).astype(np.complex64)
    target = (tmp2 * (0.8 + 0.1j) + 0.002 * rng.standard_normal(n)).astype(np.complex64)
    return p.astype(np.float32), x, tmp2.astype(np.complex128), target.astype(np.complex128)


@pytest.mark.parametrize("n", [40, 200, 1000])
def test_gradient_fp32_matches_oracle(expgb, n):
    p, x, tmp2, target = _batch(n, n)
    m = expgb.Mlp(seed=1, bf16=False)
    m.params(set=p)
    L, g = m.loss_grad(x, tmp2, target)
    Lr, gr = omlp.loss_grad(p.astype(np.float64), x.astype(np.float64), tmp2, target)
    assert abs(L - Lr) < 1e-5 * max(1, abs(Lr))
    np.testing.assert_allclose(g, gr, atol=2e-5 * np.max(np.abs(gr)), rtol=0)


def test_gradient_bf16_close_to_oracle(expgb):
    p, x, tmp2, target = _batch(500, 7)
    m = expgb.Mlp(seed=1, bf16=True)
    m.params(set=p)
    L, g = m.loss_grad(x, tmp2, target)
    Lr, gr = omlp.loss_grad(p.astype(np.float64), x.astype(np.float64), tmp2, target)
    assert abs(L - Lr) < 3e-2 * abs(Lr)
    assert np.linalg.norm(g - gr) < 3e-2 * np.linalg.norm(gr)


def _round_bf16(a):
    """Round to the nearest BF16 value (ties to even), as __float2bfloat16_rn does."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_loss_matches_rounded_oracle(expgb):
    """bf16 mode: the loss through the tensor-core layer products equals the FP64 oracle
    forward with the weights and hidden activations rounded to BF16 where the kernels round
    them, up to FP32 accumulation order and the occasional activation that rounds to the
    other BF16 neighbour (relative 2e-3; a wrong fragment layout is off by order one)."""
    p, x, tmp2, target = _batch(500, 11)
    m = expgb.Mlp(seed=1, bf16=True)
    m.params(set=p)
    L, _ = m.loss_grad(x, tmp2, target)
    W1, b1, W2, b2, W3, b3 = omlp.unflatten(p)
    h1 = _round_bf16(np.maximum(x.astype(np.float64) @ _round_bf16(W1).T + b1, 0.0))
    h2 = _round_bf16(np.maximum(h1 @ _round_bf16(W2).T + b2, 0.0))
    y = h2 @ _round_bf16(W3).T + b3
    pred = (1.0 + y[:, 0] + 1j * y[:, 1]) * tmp2
    Lr = float(np.mean(np.abs(pred - target) ** 2) / 0.05 ** 2)
    assert abs(L - Lr) < 2e-3 * abs(Lr), (L, Lr)


def test_untrained_model_is_the_mp2_guess(expgb):
    prob = syn.make_problem(77, 4, 12, G=2)
    a = expgb.from_problems([prob])
    a.init_integrals([prob.seed])
    a.iterate(0)
    b = expgb.from_problems([prob])
    b.init_integrals([prob.seed])
    m = expgb.Mlp(seed=5)
    m.apply(b)
    ta, tb = a.get_amplitudes(0), b.get_amplitudes(0)
    assert np.array_equal(ta[1].cpu().numpy(), tb[1].cpu().numpy())
    assert abs(a.energy(0) - b.energy(0)) < 1e-15


def test_training_reduces_loss_and_keeps_the_fixed_point(expgb):
    """A small family: the trained guess converges to the same energies as MP2."""
    from paper_2004_03682_gb300 import learned
    r = learned.family_experiment(n_train=24, n_test=8, epochs=8, batch=16384, n_occ=6, n_virt=24,
                                  max_iter=400)
    assert r["train_converged"] >= 12
    assert r["losses"][-1] < r["losses"][0]
    assert r["mlp_conv"] == r["mp2_conv"]
    assert r["max_dE"] is not None and r["max_dE"] < 1e-8
