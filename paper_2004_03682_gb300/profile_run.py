"""Profiling entry point: one workload, a few warm iterations, then the part to be
captured inside an NVTX range, so that a profiler can select it with
``--nvtx --nvtx-include "<range>/"``.

    python -m paper_2004_03682_gb300.profile_run --occ 40 --virt 200 --irreps 8            # range "iter3"
    python -m paper_2004_03682_gb300.profile_run --occ 40 --virt 200 --irreps 8 --top      # range "top"
    python -m paper_2004_03682_gb300.profile_run --occ 24 --virt 120 --irreps 8 --top --site R2b
    python -m paper_2004_03682_gb300.profile_run --occ 60 --virt 400 --irreps 8 --seed 3001 --slices 6 --shift 32

    python -m paper_2004_03682_gb300.profile_run --zgemm 2048 2048 2048 --slices 6        # range "zgemm"
    python -m paper_2004_03682_gb300.profile_run --family 512                               # range "iter3"
    python -m paper_2004_03682_gb300.profile_run --t3 --slices 6                            # range "t3"
    python -m paper_2004_03682_gb300.profile_run --occ 24 --virt 120 --t3 --t3-block 4      # range "t3"

Without --top the range holds one whole CCSD iteration (the CUDA graph the bench
replays); with --top it holds the contraction with the most complex multiply-adds per
iteration, or the one at call site --site (``Context.profile_top``): one full product
(slicing passes and GEMM) and one more launch of its GEMM kernel.  With --zgemm M N K
the range holds one emulated complex GEMM of that shape through exp_zgemm (seeded
operands, a few hundred MB: a bounded case for full profiler captures of the tensor-core
kernel).  With --family N the workload is the first N members of the learned-guess
family (o=10 v=40 C1, all in one context; --occ/--virt/--irreps ignored).  Prints the
iteration times (or the top contraction's site, time and work, or the GEMM time) as one
line.  With --t3 the range holds one (T) evaluation (exp_ccsd_t, block size --t3-block,
0 = automatic) from the amplitudes of two CCSD iterations, after one untimed evaluation.
"""
from __future__ import annotations

import argparse

from . import expgb
from . import synthetic as syn


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--occ", type=int, default=40)
    ap.add_argument("--virt", type=int, default=200)
    ap.add_argument("--irreps", type=int, default=8)
    ap.add_argument("--seed", type=int, default=2001)
    ap.add_argument("--slices", type=int, default=5)
    ap.add_argument("--shift", type=float, default=8.0, help="level shift (32 for o=60 v=400)")
    ap.add_argument("--fp64", action="store_true", help="plain FP64 contractions instead of the emulation")
    ap.add_argument("--top", action="store_true", help="capture the top contraction instead of an iteration")
    ap.add_argument("--site", default=None, help="with --top: this call site instead of the largest")
    ap.add_argument("--zgemm", type=int, nargs=3, default=None, metavar=("M", "N", "K"),
                    help="one emulated complex GEMM of this shape instead of a CCSD workload")
    ap.add_argument("--family", type=int, default=0, help="the first N learned-guess family members, batched")
    ap.add_argument("--slices-major", type=int, default=0, help="slices of the ladder and ring products")
    ap.add_argument("--t3", action="store_true", help="capture one (T) evaluation")
    ap.add_argument("--t3-block", type=int, default=0, help="with --t3: occupied block size (0 = automatic)")
    a = ap.parse_args()
    if a.zgemm:
        return zgemm_case(*a.zgemm, a.slices)
    probs = ([syn.family_member(k) for k in range(a.family)] if a.family else
             [syn.make_problem(a.seed, a.occ, a.virt, a.irreps)])
    prec = expgb.EXP_FP64 if a.fp64 else expgb.EXP_EMU_BF16
    ctx = expgb.from_problems(probs, conv_tol=1e-30, max_iter=50, precision=prec, n_slices=a.slices,
                              level_shift=0.0 if a.family else a.shift, n_slices_major=a.slices_major)
    ctx.init_integrals([p.seed for p in probs], scale_mult=[p.scale_mult for p in probs])
    recs, _, _ = ctx.iterate(2, raise_numeric=False)
    torch.cuda.synchronize()
    if a.t3:
        ctx.ccsd_t(0, block=a.t3_block)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("t3")
        E, info, _ = ctx.ccsd_t(0, block=a.t3_block)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(f"t3 {info['ms']:.3f} ms (products {info['ms_products']:.3f}, energies {info['ms_energy']:.3f}), "
              f"block {info['block']}, E(T) {E}")
    elif a.top:
        torch.cuda.nvtx.range_push("top")
        site, ms, macs = ctx.profile_top(reps=1, site=a.site)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(f"top {site} {ms:.4f} ms {macs:.4e} complex MACs")
    else:
        torch.cuda.nvtx.range_push("iter3")
        recs3, _, _ = ctx.iterate(1, raise_numeric=False)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print("iteration ms", [round(r["ms"], 3) for r in recs + recs3])
    ctx.close()


def zgemm_case(M, N, K, slices):
    import numpy as np
    import torch
    rng = np.random.default_rng(7)
    A = torch.tensor(rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K)), device="cuda")
    B = torch.tensor(rng.standard_normal((K, N)) + 1j * rng.standard_normal((K, N)), device="cuda")
    for _ in range(2):
        expgb.zgemm(A, B, precision=expgb.EXP_EMU_BF16, n_slices=slices)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("zgemm")
    e0.record()
    expgb.zgemm(A, B, precision=expgb.EXP_EMU_BF16, n_slices=slices)
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(f"zgemm {M}x{N}x{K} slices {slices}: {e0.elapsed_time(e1):.3f} ms (slicing, GEMM, allocation)")


if __name__ == "__main__":
    main()
