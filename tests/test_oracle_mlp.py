"""Pin the MLP oracle's backward pass against central finite differences."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = mlp.init_params(1)
    p[-(mlp.NO * mlp.W + mlp.NO):] = 0.1 * rng.standard_normal(mlp.NO * mlp.W + mlp.NO)  # live output layer
    n = 40
    x = rng.uniform(0, 1, (n, mlp.NF))
    tmp2 = 0.05 * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
    target = tmp2 * (0.8 + 0.1j) + 0.002 * rng.standard_normal(n)
    L, g = mlp.loss_grad(p, x, tmp2, target)
    assert abs(L - mlp.loss(p, x, tmp2, target)) < 1e-14 * max(1, L)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    for k in idx:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (mlp.loss(pp, x, tmp2, target) - mlp.loss(pm, x, tmp2, target)) / (2 * h)
        assert abs(fd - g[k]) < 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])


def test_untrained_model_is_the_mp2_guess():
    p = mlp.init_params(3)
    x = np.random.default_rng(1).uniform(0, 1, (10, mlp.NF))
    y, _ = mlp.forward(p, x)
    assert np.all(y == 0)
