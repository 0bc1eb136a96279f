"""The status codes of the failure paths, each made on the host or by a bounded
device wait that a test lets run out (no GPU fault, trap or hang):

  * EXP_ENOMEM: an allocator that returns NULL on its n-th call, at context creation
    and inside the first iteration; every buffer the library obtained is returned to
    the allocator (on the failed call, or by exp_destroy).
  * EXP_ENOTCONV: max_iter reached without convergence.
  * EXP_ETIMEOUT: the emulated GEMM's waits limited to 5 ms while CTA 0 leaves one
    k-block's slice copies unissued, so its MMA issuer's wait runs out; the kernel sets
    the error flag, waits for its own copies in flight, frees its tensor memory and
    returns.  The next product on the same device is correct."""
import numpy as np
import pytest

from paper_2004_03682_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def expgb():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2004_03682_gb300 import build, expgb as e
    build.build()
    e.lib()
    return e


def _failing(expgb, fail_at):
    """Allocator factory: the TorchAllocator, with allocation number fail_at returning NULL."""
    class Failing(expgb.TorchAllocator):
        def __init__(self, device, stream):
            super().__init__(device, stream)
            self.calls = 0
            inner = self._a

            def _alloc(nbytes, user):
                k = self.calls
                self.calls += 1
                return None if k == fail_at else inner(nbytes, user)

            self._a = expgb.ALLOC_FN(_alloc)
            self.struct = expgb.Allocator(self._a, self._f, None)
    return Failing


def test_enomem_at_creation_releases_everything(expgb):
    prob = syn.make_problem(11, 4, 14, 2)
    for fail_at in (0, 3, 9):
        made = []

        def factory(device, stream):
            a = _failing(expgb, fail_at)(device, stream)
            made.append(a)
            return a
        with pytest.raises(expgb.ExpError) as ei:
            expgb.from_problems([prob], allocator=factory)
        assert ei.value.status == 2, str(ei.value)
        assert made[0].calls == fail_at + 1
        assert made[0].live == {}, f"{len(made[0].live)} buffers left after a failed create"


def test_enomem_in_first_iteration_then_destroy_releases_everything(expgb):
    prob = syn.make_problem(12, 4, 14, 2)
    # count the allocator calls of create + integrals, then fail a few calls into the iteration
    probe = []

    def counting(device, stream):
        probe.append(_failing(expgb, -1)(device, stream))
        return probe[-1]
    ctx = expgb.from_problems([prob], allocator=counting)
    ctx.init_integrals([prob.seed])
    n0 = probe[0].calls
    ctx.close()
    assert probe[0].live == {}
    made = []

    def factory(device, stream):
        a = _failing(expgb, n0 + 4)(device, stream)
        made.append(a)
        return a
    ctx = expgb.from_problems([prob], allocator=factory)
    ctx.init_integrals([prob.seed])
    with pytest.raises(expgb.ExpError) as ei:
        ctx.iterate(3)
    assert ei.value.status == 2, str(ei.value)
    assert len(made[0].live) > 0
    ctx.close()
    assert made[0].live == {}


def test_enotconv_after_max_iter(expgb):
    prob = syn.make_problem(13, 4, 14, 2)
    ctx = expgb.from_problems([prob], conv_tol=1e-30, max_iter=2)
    ctx.init_integrals([prob.seed])
    recs, conv, st = ctx.iterate(5)
    assert st == 4 and not conv and len(recs) == 2
    recs, conv, st = ctx.iterate(1)  # nothing more runs
    assert st == 4 and recs == []
    ctx.close()


def test_etimeout_from_a_wait_that_runs_out_then_recovery(expgb):
    import torch
    L = expgb.lib()
    rng = np.random.default_rng(3)
    M, N, K = 300, 40, 200  # several k-blocks per work item
    A = torch.tensor(rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K)), device="cuda")
    B = torch.tensor(rng.standard_normal((K, N)) + 1j * rng.standard_normal((K, N)), device="cuda")
    assert L.exp_test_emu_wait(1, 5.0) == 0
    try:
        with pytest.raises(expgb.ExpError) as ei:
            expgb.zgemm(A, B, precision=expgb.EXP_EMU_BF16, n_slices=5)
        assert ei.value.status == 6, str(ei.value)
    finally:
        assert L.exp_test_emu_wait(-1, 2000.0) == 0
    assert L.exp_test_emu_wait(-2, 1.0) == 1 and L.exp_test_emu_wait(0, 0.0) == 1
    got = expgb.zgemm(A, B, precision=expgb.EXP_EMU_BF16, n_slices=5).cpu().numpy()
    ref = A.cpu().numpy() @ B.cpu().numpy()
    assert np.max(np.abs(got - ref)) < 1e-9 * np.max(np.abs(ref))
