"""GPU: the contraction kernels in isolation (exp_zgemm), against numpy FP64.

The split-precision emulation is pinned bit-exactly on integer-valued inputs
(every slice product and every chunk sum is then an exact integer, so any error
in the descriptors, slicing, stacking or recombination shows up), and against
its error bound on random inputs for each slice count."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    from paper_2004_03682_gb300 import build, expgb
    build.build()
    expgb.lib()
    return torch, expgb


def _c(rng, shape, scale=1.0, integer=False):
    if integer:
        return (rng.integers(-8, 9, shape) + 1j * rng.integers(-8, 9, shape)).astype(np.complex128)
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


SHAPES = [(1, 1, 1), (7, 3, 5), (128, 24, 32), (200, 37, 333), (257, 49, 1200), (64, 300, 17), (130, 25, 2049)]


@pytest.mark.parametrize("M,N,K", SHAPES + [(14, 14, 250000), (81, 14, 46000)])
def test_fp64_kernel_matches_numpy(env, M, N, K):
    torch, expgb = env
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A, B, C0 = _c(rng, (M, K)), _c(rng, (K, N)), _c(rng, (M, N))
    dA, dB = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
    dC = torch.tensor(C0, device="cuda")
    out = expgb.zgemm(dA, dB, dC, alpha=0.5 - 0.25j, beta=True).cpu().numpy()
    ref = (0.5 - 0.25j) * (A @ B) + C0
    tol = 1e-14 * np.sqrt(K) * 4
    np.testing.assert_allclose(out, ref, atol=tol * max(1, np.abs(ref).max()), rtol=0)


@pytest.mark.parametrize("S", [3, 4, 5, 6])
@pytest.mark.parametrize("M,N,K", SHAPES + [(14, 14, 40000), (81, 14, 30000)])
def test_emulated_exact_on_integer_inputs(env, S, M, N, K):
    """(the two long-K shapes run split over K: exact integer partials, added exactly)"""
    torch, expgb = env
    rng = np.random.default_rng(S * 100 + M + N + K)
    A, B = _c(rng, (M, K), integer=True), _c(rng, (K, N), integer=True)
    dA, dB = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
    out = expgb.zgemm(dA, dB, precision=expgb.EXP_EMU_BF16, n_slices=S).cpu().numpy()
    np.testing.assert_array_equal(out, A @ B)


@pytest.mark.parametrize("S", [5, 6])
def test_emulated_long_k_equal_magnitudes_exact(env, S):
    """Every element at its row's / column's maximum makes every leading slice
    digit as large as it gets: the exact integer accumulator then grows fastest.
    K' = 2K = 100000 real terms is past what one int64 accumulator holds with six
    slices, so this pins the forced K splits and the 128-bit sum of the partials."""
    torch, expgb = env
    M, N, K = 8, 8, 50000
    A = np.full((M, K), 8 + 8j)
    B = np.full((K, N), 8 - 8j)
    dA, dB = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
    out = expgb.zgemm(dA, dB, precision=expgb.EXP_EMU_BF16, n_slices=S).cpu().numpy()
    np.testing.assert_array_equal(out, A @ B)


@pytest.mark.parametrize("S", [3, 4, 5, 6])
def test_emulated_error_bound_random(env, S):
    torch, expgb = env
    rng = np.random.default_rng(S)
    M, N, K = 300, 90, 3000
    A = _c(rng, (M, K)) * np.exp(rng.uniform(-3, 3, (M, 1)))   # uneven row scales
    B = _c(rng, (K, N)) * np.exp(rng.uniform(-3, 3, (1, N)))
    dA, dB = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
    out = expgb.zgemm(dA, dB, precision=expgb.EXP_EMU_BF16, n_slices=S).cpu().numpy()
    ref = A @ B
    rmax = np.max(np.maximum(np.abs(A.real), np.abs(A.imag)), axis=1)[:, None]
    cmax = np.max(np.maximum(np.abs(B.real), np.abs(B.imag)), axis=0)[None, :]
    bound = 2.0 * K * rmax * cmax * 2.0 ** (-(7 * S - 3))
    err = np.abs(out - ref)
    assert np.all(err <= bound), float(np.max(err / bound))
    if S <= 4:
        # the slicing really ran: truncation error far above FP64 rounding
        assert np.max(err / (K * rmax * cmax)) > 2.0 ** (-(7 * S + 12))


def test_emulated_alpha_beta_and_zero_rows(env):
    torch, expgb = env
    rng = np.random.default_rng(9)
    A, B, C0 = _c(rng, (150, 64), integer=True), _c(rng, (64, 30), integer=True), _c(rng, (150, 30))
    A[5] = 0
    dA, dB, dC = (torch.tensor(x, device="cuda") for x in (A, B, C0))
    out = expgb.zgemm(dA, dB, dC, alpha=2 - 1j, beta=True, precision=expgb.EXP_EMU_BF16, n_slices=4).cpu().numpy()
    np.testing.assert_allclose(out, (2 - 1j) * (A @ B) + C0, atol=1e-12, rtol=0)
