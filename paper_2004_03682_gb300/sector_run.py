"""The (0h,1p) sector end to end on one large instance: a learned T2 guess (an MLP
trained on converged amplitudes of a small o=10 v=40 family), the (0h,0p) CCSD
iteration on emulated contractions with pair-packed tau products, then the (0h,1p)
Bloch iteration and the eigenvalues of H_eff.  Every step runs through the C ABI.

    python -m paper_2004_03682_gb300.sector_run --occ 80 --virt 480 --irreps 16 --active 16 --tol 1e-3
    python -m paper_2004_03682_gb300.sector_run --occ 24 --virt 120 --irreps 8 --active 8 --tol 1e-6 --shift 8 --sector2

Prints one JSON line: times per (0h,0p) and per (0h,1p) iteration, iteration
counts, the H_eff eigenvalues and the peak device memory; with --sector2 also the
(0h,2p) sector's iterations, time and eigenvalues.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import expgb
from . import synthetic as syn


def train_guess(n_train, epochs, device=0):
    probs = [syn.family_member(k) for k in range(n_train)]
    ctx = expgb.from_problems(probs, precision=expgb.EXP_EMU_BF16, conv_tol=1e-9, max_iter=600, device=device)
    ctx.init_integrals([p.seed for p in probs], scale_mult=[p.scale_mult for p in probs])
    ctx.iterate(600, raise_numeric=False)
    model = expgb.Mlp(seed=0, bf16=True, device=device)
    model.add_training_data(ctx)
    ctx.close()
    losses = model.train(epochs, batch=65536, lr=2e-3, seed=0)
    return model, losses


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--occ", type=int, default=80)
    ap.add_argument("--virt", type=int, default=480)
    ap.add_argument("--irreps", type=int, default=16)
    ap.add_argument("--active", type=int, default=16)
    ap.add_argument("--seed", type=int, default=5001)
    ap.add_argument("--shift", type=float, default=32.0)
    ap.add_argument("--tol", type=float, default=1e-3)
    ap.add_argument("--max-iter", type=int, default=200)
    ap.add_argument("--train", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--sector2", action="store_true", help="then the (0h,2p) sector")
    a = ap.parse_args()

    model, losses = (None, []) if a.train <= 0 else train_guess(a.train, a.epochs)
    prob = syn.make_problem(a.seed, a.occ, a.virt, a.irreps)
    act = syn.active_virtuals(prob, a.active)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    torch.cuda.reset_peak_memory_stats()
    t0 = time.perf_counter()
    ctx = expgb.from_problems([prob], precision=expgb.EXP_EMU_BF16, n_slices=5, conv_tol=a.tol,
                              max_iter=a.max_iter, level_shift=a.shift, active=act)
    ctx.init_integrals([prob.seed])
    if model is not None:
        model.apply(ctx)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    recs, conv, st = ctx.iterate(a.max_iter, raise_numeric=False)
    ms = [r["ms"] for r in recs]
    e0 = ctx.energy(0)
    out = dict(workload=f"o{a.occ}_v{a.virt}_z{a.irreps}_act{a.active}", seed=a.seed, level_shift=a.shift,
               tol=a.tol, learned_guess=model is not None, mlp_final_loss=float(losses[-1]) if len(losses) else None,
               setup_s=setup_s, ccsd_iterations=len(recs), ccsd_converged=bool(conv), ccsd_status=st,
               ccsd_first_ms=ms[0] if ms else None,
               ccsd_ms_per_iteration=float(np.mean(ms[1:])) if len(ms) > 1 else None,
               energy=[e0.real, e0.imag])
    if conv:
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        H, eig, n_fs, st_fs = ctx.fs_sector_0h1p(0)
        torch.cuda.synchronize()
        fs_s = time.perf_counter() - t1
        out.update(fs_iterations=n_fs, fs_status=st_fs, fs_s=fs_s, fs_ms_per_iteration=1e3 * fs_s / max(n_fs, 1),
                   eigenvalues=[[float(z.real), float(z.imag)] for z in eig])
        if a.sector2 and st_fs == 0:
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            H2, eig2, n2, st2 = ctx.fs_sector_0h2p(0)
            torch.cuda.synchronize()
            s2 = time.perf_counter() - t2
            out.update(fs2_iterations=n2, fs2_status=st2, fs2_s=s2, fs2_ms_per_iteration=1e3 * s2 / max(n2, 1),
                       eigenvalues2=[[float(z.real), float(z.imag)] for z in eig2])
    out["peak_device_gb"] = torch.cuda.max_memory_allocated() / 1e9
    ctx.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
