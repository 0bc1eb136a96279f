"""Solve one synthetic CCSD workload to convergence on the plain FP64 path and on
the BF16-sliced emulated path; report iterations, time to converged energy and
the energy difference.  Every step runs through the C ABI (expgb).

    python -m paper_2004_03682_gb300.converge [--occ 40 --virt 200 --irreps 8 --shift 8]
"""
from __future__ import annotations

import argparse
import json
import time

from . import expgb
from . import synthetic as syn


def solve(prob, precision, shift, tol=1e-9, max_iter=1000, n_slices=5):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = expgb.from_problems([prob], precision=precision, n_slices=n_slices, conv_tol=tol, max_iter=max_iter,
                              level_shift=shift)
    ctx.init_integrals([prob.seed])
    recs, conv, st = ctx.iterate(max_iter, raise_numeric=False)
    e = ctx.energy(0)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = sum(r["ms"] for r in recs)
    ctx.close()
    return dict(converged=conv, iterations=len(recs), energy=[e.real, e.imag], wall_s=wall,
                iteration_ms_mean=ms / max(len(recs), 1), status=st)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--occ", type=int, default=40)
    ap.add_argument("--virt", type=int, default=200)
    ap.add_argument("--irreps", type=int, default=8)
    ap.add_argument("--seed", type=int, default=2001)
    ap.add_argument("--shift", type=float, default=8.0)
    ap.add_argument("--tol", type=float, default=1e-9)
    ap.add_argument("--max-iter", type=int, default=1000)
    ap.add_argument("--slices", type=int, default=5)
    a = ap.parse_args()
    prob = syn.make_problem(a.seed, a.occ, a.virt, a.irreps)
    emu = solve(prob, expgb.EXP_EMU_BF16, a.shift, a.tol, a.max_iter, a.slices)
    f64 = solve(prob, expgb.EXP_FP64, a.shift, a.tol, a.max_iter)
    de = abs(complex(*emu["energy"]) - complex(*f64["energy"]))
    print(json.dumps(dict(workload=f"o{a.occ}_v{a.virt}_z{a.irreps}", seed=a.seed, level_shift=a.shift, tol=a.tol,
                          emulated=emu, fp64=f64, abs_dE_emulated_vs_fp64=de,
                          speedup_time_to_converged=f64["wall_s"] / emu["wall_s"])))


if __name__ == "__main__":
    main()
