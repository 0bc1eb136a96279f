"""Benchmark: CCSD (0h,0p) iterations per second on the symmetry-blocked workload
o=60, v=400, Z_8 (Dirichlet(1) irrep split, seeded synthetic Hamiltonian, pair-packed
<ab||cd> and tau products), the emulated contractions at the slice count that keeps the
energy within 1e-8 Eh of the plain FP64 path.

One step = one full CCSD iteration (tau builds, every T1/T2 contraction as grouped
permute + GEMM launches, t_new = RHS/D, residual, energy, DIIS), replayed as a CUDA
graph through the C ABI.  Prints one JSON line, which also carries the accuracy of the
emulated path against the plain FP64 GPU path over the first iterations from the same
MP2 guess (|dE| and max |dT2| after k = 1, 2, 3 iterations, for the timed slice count
and the next lower one).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision emu|fp64] [--slices S]
                    [--workload NAME] [--impl reference] [--no-accuracy]

Multi-GPU: one process per GPU (torchrun); every rank solves its own instance
(different seed), no collective on the data path ("weak" scaling); the value is
the iterations of all ranks divided by the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # the workload the metric is quoted on (one GPU): the precision configuration,
    # o=60 v=400 Z8 with packed <ab||cd> and tau pairs.  Level shift 32 Eh: the
    # synthetic Hamiltonian is strongly coupled at this size (E_MP2 = -2531 Eh) and the
    # unshifted iteration diverges from the MP2 guess (the fixed point is the same).
    # BF16 slices: 5 for the particle-particle ladder and ring products (nearly all the
    # tensor work), 6 for the other products (hole-hole ladder, F intermediates, T1 terms,
    # t1- and F-coupled T2 terms), which set the energy's accuracy: five everywhere move E
    # by 1.8e-8 Eh after one iteration and 9e-7 after two, this split by 5e-11 and 5e-9
    # (measured by the accuracy leg of every run).
    "ccsd_z8_o60_v400": dict(name="ccsd_z8_o60_v400", n_occ=60, n_virt=400, G=8, seed=3001, shift=32.0,
                             slices=6, slices_major=5),
    # the same workload in real arithmetic (the real part of the recipe; the paper's real
    # double groups): real emulated products, a quarter of the complex tensor work
    "ccsd_z8_o60_v400_real": dict(name="ccsd_z8_o60_v400_real", n_occ=60, n_virt=400, G=8, seed=3001, shift=32.0,
                                  slices=6, slices_major=5, real=True),
    "ccsd_z8_o40_v200": dict(name="ccsd_z8_o40_v200", n_occ=40, n_virt=200, G=8, seed=2001, shift=8.0,
                             slices=5),
    # a smaller case of the same kernels (a few GB on the device), for ncu captures
    "ccsd_z8_o24_v120": dict(name="ccsd_z8_o24_v120", n_occ=24, n_virt=120, G=8, seed=2001, shift=8.0,
                             slices=5),
    "ccsd_c1_o10_v40": dict(name="ccsd_c1_o10_v40", n_occ=10, n_virt=40, G=1, seed=1001, shift=0.0,
                            slices=5),
    # the learned-guess family: 448 training and 64 held-out o=10 v=40 C1 members; the
    # line reports time to the converged energy of the held-out set on four paths
    "family_o10_v40": dict(name="family_o10_v40", n_occ=10, n_virt=40, G=1, seed=4000, shift=0.0, slices=5,
                           family=True),
    # the (T) correction of CCSD(T) at o=40 v=200 Z8, from the CCSD amplitudes of the
    # o=40 v=200 workload (converged with level shift 8); one step = one evaluation
    "triples_z8_o40_v200": dict(name="triples_z8_o40_v200", n_occ=40, n_virt=200, G=8, seed=2001, shift=8.0,
                                slices=6, slices_major=5, triples=True),
}
DEFAULT_WORKLOAD = "ccsd_z8_o60_v400"
WORKLOAD = WORKLOADS[DEFAULT_WORKLOAD]
METRIC = "ccsd_iterations_per_s"
UNIT = "iter/s"
FP64_NOMINAL_TFLOPS = 1.25      # GB300 nominal dense FP64
BF16_NOMINAL_TFLOPS = 2250.0    # GB300 nominal dense BF16


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm=d["hbm_gbs"], bf16=d["bf16_tflops"], bf16_sus=d.get("bf16_tflops_sustained", d["bf16_tflops"]),
                    src="measured")
    return dict(hbm=6800.0, bf16=1900.0, bf16_sus=1700.0, src="fallback")


class Clocks:
    """Sample SM clocks / throttle reasons with nvidia-smi during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.p = None
        return self

    def _read(self):
        for line in self.p.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, n in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate_over_ranks(ms, n_it, dist=None, device="cpu"):
    """(max over ranks of the timed milliseconds, sum over ranks of the iterations): every
    rank times its own instance, and the job's throughput is all ranks' iterations over
    the slowest rank's time.  `dist` is torch.distributed after init_process_group (any
    backend; None for one process); `device` holds the reduction tensors (the GPU for
    NCCL, the host for gloo)."""
    if not dist:
        return float(ms), int(n_it)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([float(n_it)], dtype=torch.float64, device=device)
    dist.all_reduce(n)
    return t.item(), int(round(n.item()))


# ---------------------------------------------------------------------------
# Work of the oracle's equation list (oracle/ccsd.py: the Stanton-Gauss intermediates
# and both right-hand sides, every product over full pair compounds) in complex
# multiply-adds over the symmetry-allowed index tuples of a problem: each term is a
# sum over all its indices of products of operands, and an operand is nonzero only on
# the irrep tuples its symmetry rule allows (signed irrep sum = 0 mod G).  The dense
# oracle executes the G = 1 count of its sample; the target's count is what the same
# equation list needs on the blocked workload.
_SGN = {"V": (1, 1, -1, -1), "T2": (-1, -1, 1, 1), "T1": (-1, 1), "F": (1, -1), "W": (1, 1, -1, -1),
        "X": (-1, 1, 1, -1)}
ORACLE_TERMS = [
    # F_ae, F_mi, F_me
    ("me,ma->ae", "F", "T1"), ("mf,mafe->ae", "T1", "V"), ("mnaf,mnef->ae", "T2", "V"),
    ("ie,me->mi", "T1", "F"), ("ne,mnie->mi", "T1", "V"), ("inef,mnef->mi", "T2", "V"),
    ("nf,mnef->me", "T1", "V"),
    # W_mnij, W_abef, W_mbej (zeta = t2/2 + t1 t1 formed first)
    ("je,mnie->mnij", "T1", "V"), ("ijef,mnef->mnij", "T2", "V"),
    ("mb,amef->abef", "T1", "V"), ("mnab,mnef->abef", "T2", "V"),
    ("jf,mbef->mbej", "T1", "V"), ("nb,mnej->mbej", "T1", "V"), ("jnfb,mnef->mbej", "T2", "V"),
    # R1
    ("ie,ae->ia", "T1", "F"), ("ma,mi->ia", "T1", "F"), ("imae,me->ia", "T2", "F"),
    ("nf,naif->ia", "T1", "V"), ("imef,maef->ia", "T2", "V"), ("mnae,nmei->ia", "T2", "V"),
    ("mb,me->be", "T1", "F"), ("je,me->mj", "T1", "F"),
    # R2 (the t1 t1 <mb||ej> ring term as t_i^e <mb||ej> first, then t_m^a)
    ("imae,mbej->ijab", "T2", "W"), ("ie,mbej->ibmj", "T1", "V"), ("ma,ibmj->ijab", "T1", "X"),
    ("ijae,be->ijab", "T2", "F"), ("imab,mj->ijab", "T2", "F"), ("mnab,mnij->ijab", "T2", "W"),
    ("ijef,abef->ijab", "T2", "W"), ("ie,abej->ijab", "T1", "V"), ("ma,mbij->ijab", "T1", "V"),
]


def term_macs(spec, kinds, occ_counts, virt_counts):
    """Complex multiply-adds of one contraction over its symmetry-allowed index tuples."""
    import numpy as np
    ins, _ = spec.split("->")
    ops = ins.split(",")
    idx = sorted(set("".join(ops)))
    G = len(occ_counts)
    size = {c: np.asarray(occ_counts if c in "ijklmn" else virt_counts, dtype=np.float64) for c in idx}
    grids = np.meshgrid(*[np.arange(G)] * len(idx), indexing="ij")
    g = dict(zip(idx, grids))
    ok = np.ones(grids[0].shape, dtype=bool)
    for lab, kind in zip(ops, kinds):
        tot = sum(sgn * g[c] for sgn, c in zip(_SGN[kind], lab))
        ok &= (tot % G) == 0
    w = np.ones(grids[0].shape)
    for c in idx:
        w = w * size[c][g[c]]
    return float(np.sum(w[ok]))


def oracle_work(occ_counts, virt_counts):
    """Complex MACs of one oracle iteration's equation list over the allowed blocks."""
    return sum(term_macs(sp, k, occ_counts, virt_counts) for sp, *k in ORACLE_TERMS)


CPU_SAMPLE = dict(seed=1601, n_occ=16, n_virt=80, G=1)  # dense oracle sample (same recipe)


def cpu_baseline_leg(seconds=15.0, target=None):
    """The oracle as it stands (dense complex128 numpy/BLAS CCSD) on the host cores.

    Sample: oracle CCSD iterations on a dense o=16, v=80 instance of the same recipe
    (large enough that its BLAS contractions run near their asymptotic rate), timed
    for about `seconds`.  The dense oracle cannot hold the bench workload's integrals
    (o=60 v=400: 0.7 TB dense), so its effective complex-MAC rate on the sample is
    applied to the work the same equation list needs on the target's symmetry-allowed
    blocks (oracle_work): a model of a symmetry-aware oracle, not a run on the target.
    Returns (iterations/s on the target, iterations run, seconds, cores, sample MACs,
    target MACs)."""
    import numpy as np
    from oracle import ccsd, integrals
    from paper_2004_03682_gb300 import synthetic as syn
    sp = CPU_SAMPLE
    prob = syn.make_problem(sp["seed"], sp["n_occ"], sp["n_virt"], sp["G"])
    b = ccsd.Blocks(integrals.integrals(prob), integrals.fock(prob), prob.n_occ)
    t0 = time.perf_counter()
    ccsd.solve(b, tol=1e-30, max_iter=1)
    one = time.perf_counter() - t0
    n = max(1, int(seconds / max(one, 1e-3)))
    t0 = time.perf_counter()
    ccsd.solve(b, tol=1e-30, max_iter=n)
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    sample_macs = oracle_work([sp["n_occ"]], [sp["n_virt"]])
    tp = target or syn.make_problem(WORKLOAD["seed"], WORKLOAD["n_occ"], WORKLOAD["n_virt"], WORKLOAD["G"])
    target_macs = oracle_work(list(tp.irrep_occ), list(tp.irrep_virt))
    rate = n * sample_macs / dt  # complex MACs per second of the dense oracle
    return rate / target_macs, n, dt, cores, sample_macs, target_macs


def _cpu_sample_text(n, dt, smacs, tmacs):
    sp = CPU_SAMPLE
    return (f"{n} dense oracle CCSD iterations at o={sp['n_occ']} v={sp['n_virt']} C1 in {dt:.1f}s "
            f"({n * smacs / dt / 1e9:.2f} G complex MAC/s over {smacs:.4g} MACs per iteration); "
            f"modelled on {WORKLOAD['name']} by the oracle equation list's work on its allowed blocks "
            f"({tmacs:.4g} MACs per iteration); not a run on that workload")


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    # each step is one oracle iteration of the sample (a few seconds), so the whole
    # --steps K --warmup W run stays within a few minutes
    from oracle import ccsd, integrals
    from paper_2004_03682_gb300 import synthetic as syn
    tp = syn.make_problem(WORKLOAD["seed"], WORKLOAD["n_occ"], WORKLOAD["n_virt"], WORKLOAD["G"])
    sp = CPU_SAMPLE
    smacs = oracle_work([sp["n_occ"]], [sp["n_virt"]])
    tmacs = oracle_work(list(tp.irrep_occ), list(tp.irrep_virt))
    prob = syn.make_problem(sp["seed"], sp["n_occ"], sp["n_virt"], sp["G"])
    b = ccsd.Blocks(integrals.integrals(prob), integrals.fock(prob), prob.n_occ)
    ccsd.solve(b, tol=1e-30, max_iter=max(args.warmup, 1))
    t0 = time.perf_counter()
    ccsd.solve(b, tol=1e-30, max_iter=args.steps)
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    value = args.steps * smacs / dt / tmacs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": WORKLOAD["name"]},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": UNIT,
                             "sample": _cpu_sample_text(args.steps, dt, smacs, tmacs)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# k_emu_gemm DRAM read + write per launch of the top contraction, from a one-pass ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum), keyed by (workload, contraction,
# slices); None once the kernel has changed since the capture
TRAFFIC_BYTES = {("ccsd_z8_o60_v400", "Qring", 5): 27.360e9 + 1.172e9}


def slice_label(S, Smaj):
    return f"{S}" if not Smaj or Smaj == S else f"{Smaj}/{S}"


def accuracy_leg(prob, shift, configs, k=3, device=0, real=False):
    """Emulated vs plain FP64 GPU path from the same MP2 guess: |dE| after each of the
    first k iterations and max |dT2| after k, for each slice configuration (untimed):
    (n_slices, n_slices_major) pairs, labelled "major/other" ("S" when uniform).  The
    FP64 path is the one the oracle parity tests validate."""
    import torch
    from paper_2004_03682_gb300 import expgb

    def run(prec, S, Smaj=0):
        torch.cuda.empty_cache()
        ctx = expgb.from_problems([prob], precision=prec, n_slices=S, conv_tol=1e-30, max_iter=k + 1,
                                  device=device, level_shift=shift, n_slices_major=Smaj, real_arith=real)
        ctx.init_integrals([prob.seed])
        recs, _, _ = ctx.iterate(k, raise_numeric=False)
        _, t2 = ctx.get_amplitudes(0)
        ctx.close()
        return [r["e"] for r in recs], t2, [r["ms"] for r in recs]

    e64, t64, ms64 = run(expgb.EXP_FP64, 5)
    out = {"reference": "plain FP64 GPU path (oracle-validated), same MP2 guess, level shift and DIIS",
           "iterations": list(range(1, k + 1)), "E_fp64": [[e.real, e.imag] for e in e64],
           "fp64_ms_per_iteration": ms64[1:] if len(ms64) > 1 else ms64,
           "max_abs_T2": float(t64.abs().max().item()), "dE_vs_fp64": {}, "max_dT2_vs_fp64": {}}
    for S, Smaj in configs:
        e, t2, _ = run(expgb.EXP_EMU_BF16, S, Smaj)
        lab = slice_label(S, Smaj)
        out["dE_vs_fp64"][lab] = [abs(a - b) for a, b in zip(e, e64)]
        out["max_dT2_vs_fp64"][lab] = float((t2 - t64).abs().max().item())
        del t2
    del t64
    torch.cuda.empty_cache()
    out["slices_meeting_1e-8"] = [lab for lab, d in out["dE_vs_fp64"].items() if max(d) <= 1e-8]
    return out


def l2_note(prob):
    """What keeps the timed region out of L2 (129 MB): the inputs re-read every step."""
    nvv = sum(int(a) * int(b) for a in prob.irrep_virt for b in prob.irrep_virt) // 2
    pk = 16 * nvv * nvv / prob.G / 1e9  # packed <ab||cd>, per pair irrep ~ nvv/G squared
    t2 = 16 * prob.n_occ ** 2 * prob.n_virt ** 2 / prob.G / 1e9
    return (f"inputs larger than L2 (packed <ab||cd> ~{pk:.1f} GB and its slices, t2-sized operands "
            f"~{t2:.2f} GB each, re-read every step)")


def _family_solve(probs, model, precision, tol, max_iter, device):
    """One context over `probs`: guess (MP2, or the model's), then iterations until every
    instance has converged or failed, or max_iter.  Returns the per-instance energies
    and states, the iteration at which each converged, the per-iteration device times,
    and the host-synchronised wall times of the guess and of the whole solve."""
    import numpy as np
    import torch
    from paper_2004_03682_gb300 import expgb
    ctx = expgb.from_problems(probs, precision=precision, conv_tol=tol, max_iter=max_iter, device=device)
    ctx.init_integrals([p.seed for p in probs], scale_mult=[p.scale_mult for p in probs])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if model is not None:
        model.apply(ctx)
    torch.cuda.synchronize()
    guess_s = time.perf_counter() - t0
    recs, _, _ = ctx.iterate(max_iter, raise_numeric=False)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    conv_at, prev = [], 0
    for it, r in enumerate(recs, 1):
        conv_at += [it] * (r["n_converged"] - prev)
        prev = r["n_converged"]
    states = np.array([ctx.state(k) for k in range(len(probs))])
    energies = np.array([ctx.energy(k) if states[k] == 1 else complex(np.nan, np.nan) for k in range(len(probs))])
    launches = ctx.launches
    ctx.close()
    ms = [r["ms"] for r in recs]
    last = max(conv_at) if conv_at else 0
    return dict(energies=energies, states=states, conv_at=conv_at, wall_s=wall, guess_s=guess_s,
                to_last_s=guess_s + sum(ms[:last]) * 1e-3, n_iter=len(recs), launches=launches)


def run_family(args):
    """Time to the converged energies (residual < 2e-11) of the 64 held-out members on four
    paths: plain FP64 one instance at a time (MP2 guess), FP64 batched, emulated batched
    (MP2 guess), emulated batched with the learned guess (the MLP trained on the 448
    training members' converged amplitudes by the project's kernels; solving the training
    set and training are reported apart).  Members whose iteration diverges are frozen as
    failed; a few neither converge nor diverge within 1500 iterations.  Per path: the time
    until the last converging member has converged (the guess plus the device time of the
    iterations up to that point; for the plain path the sum over the converging members of
    their own solves), the wall time of the whole solve up to the iteration cap, and the
    median iteration count.  The integrals are generated before the clock starts."""
    import numpy as np
    import torch
    from paper_2004_03682_gb300 import build, expgb, learned
    from paper_2004_03682_gb300 import synthetic as syn
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    build.build()
    tol, max_iter = 2e-11, 1500
    probs = [syn.family_member(k) for k in range(512)]
    train, test = probs[:448], probs[448:]
    t0 = time.perf_counter()
    ctx, tr = learned._solve(train, max_iter=max_iter, conv_tol=tol, device=local)
    model = expgb.Mlp(seed=0, bf16=True, device=local)
    model.add_training_data(ctx)
    ctx.close()
    t1 = time.perf_counter()
    losses = model.train(20, batch=65536, lr=2e-3, seed=0)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    E, F = expgb.EXP_EMU_BF16, expgb.EXP_FP64
    paths = {"emulated_batched_mp2": _family_solve(test, None, E, tol, max_iter, local)}
    with Clocks(local) as clk:
        paths["emulated_batched_learned"] = _family_solve(test, model, E, tol, max_iter, local)
    paths["fp64_batched_mp2"] = _family_solve(test, None, F, tol, max_iter, local)
    one = dict(energies=[], states=[], conv_at=[], wall_s=0.0, to_last_s=0.0)
    for p in test:
        r = _family_solve([p], None, F, tol, max_iter, local)
        one["energies"].append(r["energies"][0])
        one["states"].append(r["states"][0])
        one["conv_at"] += r["conv_at"]
        one["wall_s"] += r["wall_s"]
        if r["states"][0] == 1:
            one["to_last_s"] += r["to_last_s"]
    one["energies"] = np.array(one["energies"])
    paths["fp64_plain_mp2"] = one
    ref = one["energies"]

    def summ(r):
        e = r["energies"]
        both = np.isfinite(e) & np.isfinite(ref)
        st = np.asarray(r["states"])
        return {"time_to_last_converged_s": r["to_last_s"], "wall_to_cap_s": r["wall_s"],
                "converged": int(np.sum(st == 1)), "failed": int(np.sum(st == 2)),
                "median_iterations": float(np.median(r["conv_at"])) if r["conv_at"] else None,
                "max_abs_dE_vs_fp64_plain": float(np.max(np.abs(e[both] - ref[both]))) if both.any() else None}
    out = {k: summ(v) for k, v in paths.items()}
    best = paths["emulated_batched_learned"]
    iters = float(np.sum(best["conv_at"]))  # instance-iterations of the converging members
    line = {"metric": METRIC, "value": iters / best["to_last_s"], "unit": UNIT, "n_gpus": ws, "steps": 1,
            "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x5-sliced f64 emulation (FP64 update, DIIS, energy)", "data": "synthetic",
            "config": {"workload": "family_o10_v40", "members": "0..447 train, 448..511 held out",
                       "conv_tol": tol, "max_iter": max_iter,
                       "l2": "64 held-out instances solved together; inputs re-read every iteration"},
            "time_to_converged": out,
            "speedup_vs_fp64_plain": one["to_last_s"] / best["to_last_s"],
            "training": {"train_solve_s": t1 - t0, "train_converged": int(tr["n_conv"]), "epochs": 20,
                         "train_s": train_s, "loss_first": float(losses[0]), "loss_last": float(losses[-1])},
            "gpu_launches": best["launches"], "clocks": clk.summary()}
    model.close()
    if rank == 0:
        print(json.dumps(line))


def _t3_cpu_leg(prob, t1, t2, seconds=20.0):
    """The oracle's (T) (oracle.triples.triple_energy, integral slices generated on demand)
    on as many occupied triples of the workload as fit in about `seconds` of host time,
    after its one-time <bc||jk> block; modelled to corrections/s as (time per triple x
    number of triples)^-1."""
    from oracle import sampled, triples
    o = prob.n_occ
    t0 = time.perf_counter()
    ints = sampled.Integrals(prob)
    setup = time.perf_counter() - t0
    done, t1s = 0, time.perf_counter()
    tri = [(i, i + 1, i + 2) for i in range(0, o - 2, 3)]
    for i, j, k in tri:
        triples.triple_energy(prob, ints, t1, t2, i, j, k)
        done += 1
        if time.perf_counter() - t1s > seconds:
            break
    per = (time.perf_counter() - t1s) / max(done, 1)
    n3 = o * (o - 1) * (o - 2) // 6
    return {"value": 1.0 / (per * n3 + setup), "unit": "corrections/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"oracle triple_energy on {done} triples of the workload, {per:.2f} s each, plus "
                      f"{setup:.1f} s for its integral setup; modelled on all {n3} triples"}


def run_triples(args):
    """One step = one (T) evaluation (exp_ccsd_t) at o=40 v=200 Z8 from the CCSD amplitudes
    of that workload (iterated with level shift 8 until converged, or 400 iterations).
    value = evaluations per second (device time, CUDA events on the context stream around
    the K calls); effective FP64 TFLOP/s credits 8 flops per complex MAC the triples i<j<k
    need.  Roofline: the stage with the larger device time (the products, or the
    per-triple energy kernel), from the call's own CUDA events.  Accuracy: E(T) of the
    emulated path against the FP64 path on the same amplitudes."""
    import numpy as np
    import torch
    from paper_2004_03682_gb300 import build, expgb
    from paper_2004_03682_gb300 import synthetic as syn
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    build.build()
    prob = syn.make_problem(WORKLOAD["seed"] + rank, WORKLOAD["n_occ"], WORKLOAD["n_virt"], WORKLOAD["G"])
    E_, F_ = expgb.EXP_EMU_BF16, expgb.EXP_FP64
    ctx = expgb.from_problems([prob], precision=E_ if args.precision == "emu" else F_, n_slices=args.slices,
                              n_slices_major=args.slices_major, conv_tol=1e-8, max_iter=400, device=local,
                              level_shift=WORKLOAD["shift"])
    ctx.init_integrals([prob.seed])
    _, conv, _ = ctx.iterate(400, raise_numeric=False)
    e_ccsd = ctx.energy(0)
    for _ in range(args.warmup):
        ctx.ccsd_t(0)
    torch.cuda.synchronize()
    l0 = ctx.launches
    infos = []
    with Clocks(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        for _ in range(args.steps):
            Et, info, _ = ctx.ccsd_t(0)
            infos.append(info)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
    launches = ctx.launches - l0
    ms = e0.elapsed_time(e1)
    ms_max, n_all = aggregate_over_ranks(ms, args.steps, None, f"cuda:{local}")
    info = infos[-1]
    value = n_all / (ms_max / 1e3)
    eff = info["macs"] * 8 * n_all / (ms_max * 1e-3) / 1e12
    pk = peaks()
    mp = float(np.mean([i["ms_products"] for i in infos]))
    me = float(np.mean([i["ms_energy"] for i in infos]))
    if mp >= me:
        if args.precision == "emu":
            pairs = args.slices * (args.slices + 1) // 2
            ach = info["macs_run"] * 4 * pairs * 2 / (mp * 1e-3) / 1e12
            roof = {"bound": "tensor", "kernel": f"k_emu_gemm<{args.slices}> ((T) products, all launches of "
                                                 "one evaluation)", "achieved": ach, "peak": pk["bf16"],
                    "unit": "TFLOP/s", "frac": ach / pk["bf16"], "traffic": None,
                    "peak_src": f"{pk['src']} bf16 dense (burst)", "ms_per_evaluation": mp}
        else:
            peak = pk["bf16"] * FP64_NOMINAL_TFLOPS / BF16_NOMINAL_TFLOPS
            ach = info["macs_run"] * 8 / (mp * 1e-3) / 1e12
            roof = {"bound": "tensor", "kernel": "k_gemm_fp64 ((T) products)", "achieved": ach, "peak": peak,
                    "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                    "peak_src": f"FP64 = {pk['src']} bf16 x nominal FP64/BF16 ratio (1.25/2250)",
                    "ms_per_evaluation": mp}
    else:
        # algorithmic bytes: the energy kernel reads each product output element once
        # (16 B; t1, <bc||jk> and the index tables come from L2)
        nbytes = info["x_elems"] * 16 * info["macs"] / max(info["macs_run"], 1.0)
        ach = nbytes / (me * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": "k_t3_energy (per-triple energies, all launches of one evaluation)",
                "achieved": ach, "peak": pk["hbm"], "unit": "GB/s", "frac": ach / pk["hbm"], "traffic": None,
                "peak_src": f"{pk['src']} HBM copy", "ms_per_evaluation": me}
    acc = None
    if args.precision == "emu" and not args.no_accuracy and rank == 0:
        t1, t2 = ctx.get_amplitudes(0)
        ref = expgb.from_problems([prob], precision=F_, device=local)
        ref.init_integrals([prob.seed])
        ref.set_amplitudes(0, t1, t2)
        Ef, inf_f, _ = ref.ccsd_t(0)
        ref.close()
        acc = {"E_T_emulated": [Et.real, Et.imag], "E_T_fp64": [Ef.real, Ef.imag], "dE_T": abs(Et - Ef),
               "fp64_ms": inf_f["ms"]}
    # e2e: the public API from host amplitudes (create, integrals, set amplitudes, one (T))
    t1h, t2h = (x.cpu() for x in ctx.get_amplitudes(0))
    ctx.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c2 = expgb.from_problems([prob], precision=E_ if args.precision == "emu" else F_, n_slices=args.slices,
                             device=local)
    c2.init_integrals([prob.seed])
    c2.set_amplitudes(0, t1h, t2h)
    Ee, _, _ = c2.ccsd_t(0)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    c2.close()
    e2e = {"value": 1.0 / e2e_s, "unit": "corrections/s", "h2d_bytes_per_step": (t1h.numel() + t2h.numel()) * 16,
           "d2h_bytes_per_step": 16 * 8,
           "includes": "exp_create + exp_init_integrals + exp_set_amplitudes (pinned copy of t1, t2) + exp_ccsd_t"}
    cpu = _t3_cpu_leg(prob, t1h.numpy(), t2h.numpy()) if rank == 0 else None
    line = {"metric": "ccsd_t_per_s", "value": value, "unit": "corrections/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": (f"bf16x{args.slices}-sliced f64 emulation (products), double-single element arithmetic, "
                      "FP64 sums") if args.precision == "emu" else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "n_occ": prob.n_occ, "n_virt": prob.n_virt, "irreps": "Z8",
                       "seed": prob.seed, "ccsd_converged": bool(conv), "e_ccsd": [e_ccsd.real, e_ccsd.imag],
                       "block": info["block"], "block_triples": info["n_block_triples"],
                       "triples": info["n_triples"],
                       "l2": "inputs larger than L2 (product outputs up to 16 GiB per batch of triples, "
                             "dense t2 and <bc||jk> 1 GB each)"},
            "E_T": [Et.real, Et.imag], "macs_needed": info["macs"], "macs_run": info["macs_run"],
            "effective_fp64_tflops": eff, "ms_products": mp, "ms_energy": me, "roofline": roof,
            "accuracy": acc, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", choices=["emu", "fp64"], default="emu")
    ap.add_argument("--slices", type=int, default=None, help="BF16 slices (default: the workload's)")
    ap.add_argument("--slices-major", type=int, default=None,
                    help="BF16 slices of the particle-particle ladder and ring products (default: the workload's)")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-accuracy", action="store_true", help="skip the emulated-vs-FP64 leg")
    args = ap.parse_args()
    global WORKLOAD
    WORKLOAD = WORKLOADS[args.workload]
    if args.slices is None:
        args.slices = WORKLOAD["slices"]
        if args.slices_major is None:
            args.slices_major = WORKLOAD.get("slices_major", 0)
    if args.slices_major is None:
        args.slices_major = 0
    smaj = args.slices_major or args.slices  # slices of the top (ladder / ring) product
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_env()

    if args.impl == "reference":
        return run_reference(args)
    if WORKLOAD.get("family"):
        return run_family(args)
    if WORKLOAD.get("triples"):
        return run_triples(args)

    import numpy as np
    import torch
    from paper_2004_03682_gb300 import build, expgb
    from paper_2004_03682_gb300 import synthetic as syn

    torch.cuda.set_device(local)
    build.build()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    prec = expgb.EXP_EMU_BF16 if args.precision == "emu" else expgb.EXP_FP64
    prob = syn.make_problem(WORKLOAD["seed"] + rank, WORKLOAD["n_occ"], WORKLOAD["n_virt"], WORKLOAD["G"])
    total = args.warmup + args.steps + 5
    real = bool(WORKLOAD.get("real", False))
    ctx = expgb.from_problems([prob], precision=prec, n_slices=args.slices, conv_tol=1e-30,
                              max_iter=10 * total, device=local, level_shift=WORKLOAD["shift"],
                              n_slices_major=args.slices_major, real_arith=real)
    ctx.init_integrals([prob.seed])
    ctx.iterate(args.warmup, raise_numeric=False)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    l0 = ctx.launches
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        recs, _, st = ctx.iterate(args.steps, raise_numeric=False)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = ctx.launches - l0
    ms = e0.elapsed_time(e1)
    n_it = len(recs)
    ms_max, n_all = aggregate_over_ranks(ms, n_it, dist, f"cuda:{local}")
    value = n_all / (ms_max / 1e3)
    macs = ctx.work_per_iteration()
    fpm = 2 if WORKLOAD.get("real", False) else 8  # FP64 flops credited per algorithmic MAC (real / complex)
    ctflops = n_all * macs * fpm / (ms_max * 1e-3) / 1e12
    # roofline of the dominant contraction, timed alone with CUDA events on the context stream
    site, kms, kmacs = ctx.profile_top(reps=3)
    pk = peaks()
    if args.precision == "fp64":
        peak = pk["bf16"] * FP64_NOMINAL_TFLOPS / BF16_NOMINAL_TFLOPS
        achieved = kmacs * 4 * 2 / (kms * 1e-3) / 1e12  # real FP64 flops: 4 real FMA per complex MAC
        roof = {"bound": "tensor", "kernel": f"k_gemm_fp64 ({site})", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_src": f"FP64 = {pk['src']} bf16 x nominal FP64/BF16 ratio (1.25/2250)"}
    else:
        pairs = smaj * (smaj + 1) // 2
        # executed BF16 tensor flops: 4 real MACs per complex MAC (real embedding; 1 in real
        # arithmetic) x slice pairs x 2
        achieved = kmacs * (1 if real else 4) * pairs * 2 / (kms * 1e-3) / 1e12
        eff = kmacs * fpm / (kms * 1e-3) / 1e12
        traffic = TRAFFIC_BYTES.get((WORKLOAD["name"], site, smaj))
        roof = {"bound": "tensor", "kernel": f"k_emu_gemm<{smaj}> ({site})", "achieved": achieved,
                "peak": pk["bf16"], "unit": "TFLOP/s", "frac": achieved / pk["bf16"], "traffic": traffic,
                "peak_src": f"{pk['src']} bf16 dense (burst)", "ms_per_launch": kms,
                "macs_per_launch": kmacs, "effective_fp64_tflops": eff}
    ctx.close()

    # e2e: the public API end to end (create from host arrays, generate integrals,
    # K iterations with the per-iteration host read of energy/residual, final energy)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx2 = expgb.from_problems([prob], precision=prec, n_slices=args.slices, conv_tol=1e-30,
                               max_iter=10 * total, device=local, level_shift=WORKLOAD["shift"],
                               n_slices_major=args.slices_major, real_arith=real)
    ctx2.init_integrals([prob.seed])
    recs2, _, _ = ctx2.iterate(args.steps, raise_numeric=False)
    _ = ctx2.energy(0)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    ctx2.close()
    h2d = (prob.n_occ + prob.n_virt) * 8 + 8 + 2 * prob.G * 4
    e2e = {"value": len(recs2) / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d / max(len(recs2), 1),
           "d2h_bytes_per_step": 8 * 8 + 4 * 4,
           "includes": "exp_create + exp_init_integrals + K iterations + exp_energy, host arrays"}

    acc = None
    if args.precision == "emu" and not args.no_accuracy and rank == 0:
        confs = [(args.slices, args.slices_major)]
        for c2 in [(smaj, 0), (args.slices, 0), (smaj - 1, 0)]:
            if c2 not in confs and (c2[0], c2[0]) not in confs and 3 <= c2[0] <= 6:
                confs.append(c2)
        acc = accuracy_leg(prob, WORKLOAD["shift"], confs, k=3, device=local, real=real)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if ws == 1:
        rate, n, dt, cores, smacs, tmacs = cpu_baseline_leg(15.0, prob)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": _cpu_sample_text(n, dt, smacs, tmacs)}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / max(n_it, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else (
                f"bf16x{args.slices}-sliced f64 emulation" if smaj == args.slices else
                f"bf16-sliced f64 emulation ({smaj} slices: particle-particle ladder and ring products; "
                f"{args.slices}: the others)"),
            "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "n_occ": WORKLOAD["n_occ"], "n_virt": WORKLOAD["n_virt"],
                       "irreps": f"Z{WORKLOAD['G']}", "seed": WORKLOAD["seed"], "precision": args.precision,
                       "slices": args.slices if args.precision == "emu" else None,
                       "slices_major": smaj if args.precision == "emu" else None,
                       "level_shift": WORKLOAD["shift"], "packed": True, "real_arith": real,
                       "l2": l2_note(prob)},
            "effective_fp64_tflops": ctflops, "flops_per_mac": fpm, "macs_per_iter": macs,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary(), "status": st}
    if acc is not None:
        lab = slice_label(args.slices, args.slices_major)
        line["dE_vs_fp64"] = acc["dE_vs_fp64"][lab]
        line["max_dT2_vs_fp64"] = acc["max_dT2_vs_fp64"][lab]
        line["accuracy"] = acc
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
