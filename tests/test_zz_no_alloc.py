"""The allocation-free emulated GEMM (exp_zgemm_emu_noalloc) against exp_zgemm.

For callers that cannot allocate device memory at the point of the call, the
library offers one GEMM whose scratch is a fixed array in its own device memory.
This test calls it through the C ABI twice in a row (the calls share that array)
and checks each result against the allocating entry point with the same slice
count; it also checks that a problem too large for the array is refused on the
host.  Collected last so that a run stopping at the first failure has already
run every other test; it also passes alone in a fresh process."""
import ctypes as C

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
    L = expgb.lib()
    L.exp_zgemm_emu_noalloc.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_double, C.c_double, C.c_int]
    L.exp_zgemm_emu_noalloc.restype = C.c_int
    L.exp_noalloc_last_error.argtypes = []
    L.exp_noalloc_last_error.restype = C.c_char_p
    return torch, expgb, L


def _rand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _noalloc(torch, L, A, B, C0, alpha, beta, S):
    s = torch.cuda.current_stream()
    out = C0.clone()
    st = L.exp_zgemm_emu_noalloc(C.c_void_p(s.cuda_stream), S, A.shape[0], B.shape[1], A.shape[1],
                                 C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()), C.c_void_p(out.data_ptr()),
                                 alpha.real, alpha.imag, int(beta))
    assert st == 0, L.exp_noalloc_last_error()
    return out


# the second shape is split over K; the reversed order runs a larger split-K problem
# first, so stale partials or exponents it leaves in the shared array would show up
# in the smaller split-K problem after it
ORDERS = {"small_then_split": [(200, 37, 333), (81, 14, 8000)],
          "split_then_smaller_split": [(96, 20, 9000), (40, 9, 4100)]}


@pytest.mark.parametrize("order", sorted(ORDERS))
@pytest.mark.parametrize("S", [3, 4, 5, 6])
def test_noalloc_matches_allocating_gemm_twice(env, S, order):
    torch, expgb, L = env
    rng = np.random.default_rng(S)
    shapes = ORDERS[order]
    for M, N, K in shapes:  # two calls in a row on the shared scratch
        A = torch.tensor(_rand(rng, (M, K)), device="cuda")
        B = torch.tensor(_rand(rng, (K, N)), device="cuda")
        C0 = torch.tensor(_rand(rng, (M, N)), device="cuda")
        alpha = 0.75 + 0.5j
        got = _noalloc(torch, L, A, B, C0, alpha, True, S).cpu().numpy()
        ref = expgb.zgemm(A, B, C0.clone(), alpha=alpha, beta=True, precision=expgb.EXP_EMU_BF16,
                          n_slices=S).cpu().numpy()
        scale = np.abs(ref).max()
        np.testing.assert_allclose(got, ref, atol=1e-13 * scale, rtol=0)
        exact = alpha * (A.cpu().numpy() @ B.cpu().numpy()) + C0.cpu().numpy()
        assert np.max(np.abs(got - exact)) < 2.0 ** (-(7 * S - 3)) * K * 30


def test_noalloc_refuses_oversized_problem(env):
    torch, expgb, L = env
    A = torch.zeros((2000, 2000), dtype=torch.complex128, device="cuda")
    st = L.exp_zgemm_emu_noalloc(C.c_void_p(torch.cuda.current_stream().cuda_stream), 5, 2000, 2000, 2000,
                                 C.c_void_p(A.data_ptr()), C.c_void_p(A.data_ptr()), C.c_void_p(A.data_ptr()),
                                 1.0, 0.0, 0)
    assert st == 1
    assert b"scratch" in L.exp_noalloc_last_error()


def test_noalloc_refuses_huge_k_before_layout_arithmetic(env):
    # K near 2^30 would overflow the padded K' = 2K in int; it is refused on the host
    # before any size is derived from it (nothing is launched, no pointer is read)
    torch, expgb, L = env
    A = torch.zeros((1, 1), dtype=torch.complex128, device="cuda")
    st = L.exp_zgemm_emu_noalloc(C.c_void_p(torch.cuda.current_stream().cuda_stream), 5, 1, 1, (1 << 30) - 8,
                                 C.c_void_p(A.data_ptr()), C.c_void_p(A.data_ptr()), C.c_void_p(A.data_ptr()),
                                 1.0, 0.0, 0)
    assert st == 1
    assert b"2^26" in L.exp_noalloc_last_error()
