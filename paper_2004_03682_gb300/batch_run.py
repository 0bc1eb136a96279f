"""Many small instances in one context: the learned-guess family (o=10 v=40 C1,
integral scale x U[0.5,1.5], virtual floor U[0.1,0.6]) solved together, every
launch covering all instances.  Measures steady-state iteration time (CUDA-graph
replays, no instance converging) for n_inst instances and for one, so the batched
throughput in instance-iterations/s can be set against the single-instance rate.

    python -m paper_2004_03682_gb300.batch_run --n-inst 512 --iters 12

Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import expgb
from . import synthetic as syn


def steady_ms(n_inst, iters, precision, n_occ, n_virt):
    import torch
    probs = [syn.family_member(k, n_occ, n_virt) for k in range(n_inst)]
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    t0 = time.perf_counter()
    ctx = expgb.from_problems(probs, precision=precision, conv_tol=1e-30, max_iter=iters + 1)
    ctx.init_integrals([p.seed for p in probs], scale_mult=[p.scale_mult for p in probs])
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    recs, _, _ = ctx.iterate(iters, raise_numeric=False)
    ms = [r["ms"] for r in recs]
    e0 = ctx.energy(0)
    ctx.close()
    steady = ms[2:] if len(ms) > 3 else ms[1:]
    return dict(n_inst=n_inst, setup_s=setup_s, first_ms=ms[0], ms_per_iteration=float(np.median(steady)),
                instance_iterations_per_s=n_inst * 1e3 / float(np.median(steady)),
                energy0=[e0.real, e0.imag], peak_device_gb=torch.cuda.max_memory_allocated() / 1e9)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-inst", type=int, default=512)
    ap.add_argument("--iters", type=int, default=12)
    ap.add_argument("--occ", type=int, default=10)
    ap.add_argument("--virt", type=int, default=40)
    ap.add_argument("--fp64", action="store_true")
    a = ap.parse_args()
    prec = expgb.EXP_FP64 if a.fp64 else expgb.EXP_EMU_BF16
    one = steady_ms(1, a.iters, prec, a.occ, a.virt)
    many = steady_ms(a.n_inst, a.iters, prec, a.occ, a.virt)
    out = dict(workload=f"family_o{a.occ}_v{a.virt}_c1", precision="fp64" if a.fp64 else "emu", single=one,
               batched=many, batching_gain=many["instance_iterations_per_s"] / one["instance_iterations_per_s"])
    print(json.dumps(out))


if __name__ == "__main__":
    main()
