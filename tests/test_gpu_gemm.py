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


DS_SHAPES = [(1, 1, 1), (7, 3, 5), (128, 16, 16), (300, 37, 9), (129, 81, 14), (1000, 5, 1)]


@pytest.mark.parametrize("M,N,K", DS_SHAPES)
@pytest.mark.parametrize("alpha,beta", [(1.0, False), (-0.5, True), (0.3 + 0.2j, True)])
def test_double_single_within_bound(env, M, N, K, alpha, beta):
    """The double-single product (FP32 h + l per operand, error-free products and sums,
    one rounding to FP64) against numpy: each element within 2^-44 of sum_k |a||b|
    (48-bit operands, K <= 16 terms), on rows and columns spanning 2^-60 .. 2^20,
    exact zeros, and a ragged last row / column tile."""
    torch, expgb = env
    rng = np.random.default_rng(M + 3 * N + 7 * K)
    A = _c(rng, (M, K)) * np.exp2(rng.integers(-60, 20, (M, 1)))
    B = _c(rng, (K, N)) * np.exp2(rng.integers(-10, 10, (1, N)))
    A[0, 0] = 0.0
    C0 = _c(rng, (M, N))
    dA, dB, dC = (torch.tensor(x, device="cuda") for x in (A, B, C0))
    out = expgb.zgemm(dA, dB, dC, alpha=alpha, beta=beta, precision=expgb.EXP_EMU_DS).cpu().numpy()
    ref = alpha * (A @ B) + (C0 if beta else 0)
    bound = 2.0 ** -44 * abs(alpha) * 2 * (np.abs(A) @ np.abs(B)) + (1e-15 * np.abs(C0) if beta else 0) + 1e-300
    assert np.all(np.abs(out - ref) <= bound)


def test_double_single_exact_on_integer_inputs(env):
    """Integer inputs below 2^11: every product and partial sum is exact in h + l,
    so the result is bit-exact."""
    torch, expgb = env
    rng = np.random.default_rng(9)
    A = (rng.integers(-1000, 1001, (333, 16)) + 1j * rng.integers(-1000, 1001, (333, 16))).astype(np.complex128)
    B = (rng.integers(-1000, 1001, (16, 45)) + 1j * rng.integers(-1000, 1001, (16, 45))).astype(np.complex128)
    dA, dB = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
    out = expgb.zgemm(dA, dB, precision=expgb.EXP_EMU_DS).cpu().numpy()
    np.testing.assert_array_equal(out, A @ B)


def test_double_single_refuses_long_k(env):
    torch, expgb = env
    dA = torch.zeros((4, 17), dtype=torch.complex128, device="cuda")
    dB = torch.zeros((17, 4), dtype=torch.complex128, device="cuda")
    with pytest.raises(expgb.ExpError):
        expgb.zgemm(dA, dB, precision=expgb.EXP_EMU_DS)
