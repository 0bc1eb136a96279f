"""Learned initial guess on a family of Hamiltonians: train on converged solves,
evaluate iteration counts and converged energies on held-out members against the
MP2 guess.  Every step runs through the C ABI (expgb); nothing here computes."""
from __future__ import annotations

import time

import numpy as np

from . import expgb
from . import synthetic as syn


def _solve(probs, guess_model=None, max_iter=600, conv_tol=1e-9, precision=expgb.EXP_EMU_BF16, device=0):
    import torch
    ctx = expgb.from_problems(probs, conv_tol=conv_tol, max_iter=max_iter, precision=precision, device=device)
    ctx.init_integrals([p.seed for p in probs], scale_mult=[p.scale_mult for p in probs])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if guess_model is not None:
        guess_model.apply(ctx)
    recs, conv, _ = ctx.iterate(max_iter, raise_numeric=False)  # diverging members drop out
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    n = len(probs)
    conv_at = []  # iteration at which the k-th instance converged (distribution)
    prev = 0
    for it, r in enumerate(recs, 1):
        conv_at += [it] * (r["n_converged"] - prev)
        prev = r["n_converged"]
    states = np.array([ctx.state(k) for k in range(n)])
    energies = np.array([ctx.energy(k) if states[k] == 1 else complex(np.nan, np.nan) for k in range(n)])
    return ctx, dict(conv_at=conv_at, n_conv=prev, n_iter=len(recs), wall_s=wall, energies=energies)


def family_experiment(n_train=448, n_test=64, epochs=20, batch=65536, lr=2e-3, max_iter=600, conv_tol=1e-9,
                      n_occ=10, n_virt=40, seed=0, device=0):
    probs = [syn.family_member(k, n_occ, n_virt) for k in range(n_train + n_test)]
    train, test = probs[:n_train], probs[n_train:]
    ctx, tr = _solve(train, max_iter=max_iter, conv_tol=conv_tol, device=device)
    model = expgb.Mlp(seed=seed, bf16=True, device=device)
    model.add_training_data(ctx)
    ctx.close()
    t0 = time.perf_counter()
    losses = model.train(epochs, batch=batch, lr=lr, seed=seed)
    train_s = time.perf_counter() - t0
    c_mp2, mp2 = _solve(test, None, max_iter, conv_tol, device=device)
    c_mp2.close()
    c_mlp, mlp = _solve(test, model, max_iter, conv_tol, device=device)
    c_mlp.close()
    c_f64, f64 = _solve(test, None, max_iter, conv_tol, precision=expgb.EXP_FP64, device=device)
    c_f64.close()
    both = np.isfinite(mp2["energies"]) & np.isfinite(mlp["energies"])
    de = np.abs(mp2["energies"] - mlp["energies"])[both]
    return dict(train_converged=tr["n_conv"], losses=losses.tolist(), train_s=train_s,
                mp2_iters=mp2["conv_at"], mlp_iters=mlp["conv_at"], mp2_conv=mp2["n_conv"], mlp_conv=mlp["n_conv"],
                mp2_wall_s=mp2["wall_s"], mlp_wall_s=mlp["wall_s"], max_dE=float(de.max()) if de.size else None,
                fp64_mp2_iters=f64["conv_at"], fp64_mp2_conv=f64["n_conv"], fp64_mp2_wall_s=f64["wall_s"],
                max_dE_fp64=float(np.nanmax(np.abs(f64["energies"] - mlp["energies"]))),
                model=model)


def summary(r):
    """Condensed report: iterations and time to converged energy on the held-out set."""
    def st(x):
        return dict(n=len(x), mean=float(np.mean(x)) if x else None, median=float(np.median(x)) if x else None,
                    max=int(max(x)) if x else None)
    return dict(train_converged=r["train_converged"], loss_first=r["losses"][0], loss_last=r["losses"][-1],
                train_s=r["train_s"], mp2_guess=st(r["mp2_iters"]), learned_guess=st(r["mlp_iters"]),
                fp64_mp2_guess=st(r["fp64_mp2_iters"]),
                time_to_converged_s=dict(fp64_mp2=r["fp64_mp2_wall_s"], emulated_mp2=r["mp2_wall_s"],
                                         emulated_learned=r["mlp_wall_s"]),
                max_dE_learned_vs_mp2=r["max_dE"], max_dE_learned_vs_fp64=r["max_dE_fp64"])


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="learned T2 guess on the o=10 v=40 Hamiltonian family")
    ap.add_argument("--train", type=int, default=448)
    ap.add_argument("--test", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=20)
    args = ap.parse_args()
    r = family_experiment(n_train=args.train, n_test=args.test, epochs=args.epochs)
    print(json.dumps(summary(r)))
