"""Emulated vs plain FP64 GPU path at fixed iteration count, over the BF16 slice
count: both paths start from the same MP2 guess and run the same number of
iterations (level shift, DIIS(6)); the difference of the energies and the largest
difference of the T2 amplitudes measure how far the emulation moves the
iteration.  T2 stays on the device (at o=60 v=400 one dense copy is 9 GB).

    python -m paper_2004_03682_gb300.precision_sweep --occ 60 --virt 400 --irreps 8 --iters 10 --slices 3 4 5 6
"""
from __future__ import annotations

import argparse
import json
import time

from . import expgb
from . import synthetic as syn


def run(prob, precision, n_slices, iters, shift):
    import torch
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    torch.cuda.reset_peak_memory_stats()
    t0 = time.perf_counter()
    ctx = expgb.from_problems([prob], precision=precision, n_slices=n_slices, conv_tol=1e-30, max_iter=iters + 1,
                              level_shift=shift)
    ctx.init_integrals([prob.seed])
    recs, _, st = ctx.iterate(iters, raise_notconv=False, raise_numeric=False)
    e = ctx.energy(0)
    _, t2 = ctx.get_amplitudes(0)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = [r["ms"] for r in recs]
    ctx.close()
    steady = ms[1:] if len(ms) > 1 else ms
    return e, t2, dict(iterations=len(recs), wall_s=wall, iteration_ms=sum(steady) / max(len(steady), 1),
                       energy=[e.real, e.imag], status=st, peak_device_gb=torch.cuda.max_memory_allocated() / 1e9)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--occ", type=int, default=60)
    ap.add_argument("--virt", type=int, default=400)
    ap.add_argument("--irreps", type=int, default=8)
    ap.add_argument("--seed", type=int, default=3001)
    ap.add_argument("--shift", type=float, default=8.0)
    ap.add_argument("--iters", type=int, default=10)
    ap.add_argument("--slices", type=int, nargs="+", default=[3, 4, 5, 6])
    a = ap.parse_args()
    prob = syn.make_problem(a.seed, a.occ, a.virt, a.irreps)
    e64, t64, r64 = run(prob, expgb.EXP_FP64, 5, a.iters, a.shift)
    out = dict(workload=f"o{a.occ}_v{a.virt}_z{a.irreps}", seed=a.seed, level_shift=a.shift, iterations=a.iters,
               fp64=r64, emulated={})
    for S in a.slices:
        e, t2, r = run(prob, expgb.EXP_EMU_BF16, S, a.iters, a.shift)
        r["abs_dE"] = abs(e - e64)
        r["max_abs_dT2"] = float((t2 - t64).abs().max().item())
        r["max_abs_T2"] = float(t64.abs().max().item())
        del t2
        out["emulated"][str(S)] = r
        print(json.dumps({"slices": S, **r}), flush=True)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
