"""Benchmark: CCSD (0h,0p) iterations per second on the symmetry-blocked workload
o=40, v=200, Z_8 (Dirichlet(1) irrep split, seeded synthetic Hamiltonian).

One step = one full CCSD iteration (tau builds, every T1/T2 contraction as grouped
permute + GEMM launches, t_new = RHS/D, residual, energy, DIIS), replayed as a CUDA
graph through the C ABI.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision emu|fp64] [--impl reference]

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
    # the workload the metric is quoted on (one GPU)
    # (level shift 8 Eh: the synthetic Hamiltonian is strongly coupled at this size and the
    # unshifted iteration diverges from the MP2 guess; the fixed point is the same)
    "ccsd_z8_o40_v200": dict(name="ccsd_z8_o40_v200", n_occ=40, n_virt=200, G=8, seed=2001, shift=8.0),
    # a smaller case of the same kernels (a few GB on the device), for ncu captures
    "ccsd_z8_o24_v120": dict(name="ccsd_z8_o24_v120", n_occ=24, n_virt=120, G=8, seed=2001, shift=8.0),
    "ccsd_c1_o10_v40": dict(name="ccsd_c1_o10_v40", n_occ=10, n_virt=40, G=1, seed=1001, shift=0.0),
}
WORKLOAD = WORKLOADS["ccsd_z8_o40_v200"]
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


def cpu_baseline_leg(seconds=15.0):
    """The oracle as it stands (dense complex128 numpy/BLAS CCSD) on the host cores.

    Sample: oracle CCSD iterations on the C1 instance (o=10, v=40), timed for about
    `seconds`; converted to the bench workload's unit by dividing its effective
    complex-MAC rate by the blocked work of one o=40, v=200, Z_8 iteration (the
    dense oracle cannot hold that workload's integrals: ~53 GB)."""
    from oracle import ccsd, integrals
    from paper_2004_03682_gb300 import synthetic as syn
    prob = syn.make_problem(1001, 10, 40, 1)
    b = ccsd.Blocks(integrals.integrals(prob), integrals.fock(prob), 10)
    t0 = time.perf_counter()
    ccsd.solve(b, tol=1e-30, max_iter=2)
    one = (time.perf_counter() - t0) / 2
    n = max(2, int(seconds / one))
    t0 = time.perf_counter()
    ccsd.solve(b, tol=1e-30, max_iter=n)
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return n / dt, n, dt, cores


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    gpu_macs = ORACLE_MACS[WORKLOAD["name"]]
    if gpu_macs is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no oracle work count for {WORKLOAD['name']}"}))
        return
    rate, n, dt, cores = cpu_baseline_leg(max(5.0, 2.0 * args.steps))
    # effective complex MAC rate of the oracle on the sample, in the workload's unit
    c1_macs = C1_MACS
    value = rate * c1_macs / gpu_macs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": WORKLOAD["name"]},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": UNIT,
                             "sample": f"{n} oracle CCSD iterations at o=10 v=40 C1 in {dt:.1f}s, scaled by "
                                       f"complex-MAC work ({c1_macs:.3g} -> {gpu_macs:.3g} per iteration)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# Complex MACs of one CCSD iteration as the oracle evaluates it: every product of its
# equation list (R1's <ma||ef> t_im^ef term included) over full pair compounds (it
# sums over every c, d, e, f, m, n), counted by the blocked planner on o=10 v=40 C1
# (the oracle sample) and the bench workloads.  The oracle baseline is converted
# between them; the GPU arm's own count is that of its packed products.
C1_MACS = 5.264e8
ORACLE_MACS = {"ccsd_z8_o40_v200": 8.948e10, "ccsd_z8_o24_v120": None, "ccsd_c1_o10_v40": C1_MACS}
# k_emu_gemm<5> DRAM read + write per launch of the top contraction, from ncu
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by (workload, contraction)
TRAFFIC_BYTES = {("ccsd_z8_o40_v200", "Qring"): 0.938e9 + 0.127e9}  # one-pass capture of the full-size launch


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", choices=["emu", "fp64"], default="emu")
    ap.add_argument("--slices", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="ccsd_z8_o40_v200")
    args = ap.parse_args()
    global WORKLOAD
    WORKLOAD = WORKLOADS[args.workload]
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_env()

    if args.impl == "reference":
        return run_reference(args)

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
    ctx = expgb.from_problems([prob], precision=prec, n_slices=args.slices, conv_tol=1e-30,
                              max_iter=10 * total, device=local, level_shift=WORKLOAD["shift"])
    ctx.init_integrals([prob.seed])
    ctx.iterate(args.warmup)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    l0 = ctx.launches
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        recs, _, st = ctx.iterate(args.steps)
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
    ctflops = n_all * macs * 8 / (ms_max * 1e-3) / 1e12  # complex flops credited (8 per complex MAC)
    # roofline of the dominant contraction, timed alone with CUDA events
    site, kms, kmacs = ctx.profile_top(reps=3)
    pk = peaks()
    if args.precision == "fp64":
        peak = pk["bf16"] * FP64_NOMINAL_TFLOPS / BF16_NOMINAL_TFLOPS
        achieved = kmacs * 4 * 2 / (kms * 1e-3) / 1e12  # real FP64 flops: 4 real FMA per complex MAC
        roof = {"bound": "tensor", "kernel": f"k_gemm_fp64 ({site})", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_src": f"FP64 = {pk['src']} bf16 x nominal FP64/BF16 ratio (1.25/2250)"}
    else:
        pairs = args.slices * (args.slices + 1) // 2
        # executed BF16 tensor flops: 4 real MACs per complex MAC (real embedding) x slice pairs x 2
        achieved = kmacs * 4 * pairs * 2 / (kms * 1e-3) / 1e12
        eff = kmacs * 8 / (kms * 1e-3) / 1e12
        traffic = TRAFFIC_BYTES.get((WORKLOAD["name"], site)) if args.slices == 5 else None
        roof = {"bound": "tensor", "kernel": f"k_emu_gemm<{args.slices}> ({site})", "achieved": achieved,
                "peak": pk["bf16"], "unit": "TFLOP/s", "frac": achieved / pk["bf16"], "traffic": traffic,
                "peak_src": f"{pk['src']} bf16 dense (burst)",
                "effective_complex_fp64_tflops": eff}
    e_final = ctx.energy(0)
    ctx.close()

    # e2e: the public API end to end (create from host arrays, generate integrals,
    # K iterations with the per-iteration host read of energy/residual, final energy)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx2 = expgb.from_problems([prob], precision=prec, n_slices=args.slices, conv_tol=1e-30,
                               max_iter=10 * total, device=local, level_shift=WORKLOAD["shift"])
    ctx2.init_integrals([prob.seed])
    recs2, _, _ = ctx2.iterate(args.steps)
    _ = ctx2.energy(0)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    ctx2.close()
    h2d = (prob.n_occ + prob.n_virt) * 8 + 8 + 2 * prob.G * 4
    e2e = {"value": len(recs2) / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d / max(len(recs2), 1),
           "d2h_bytes_per_step": 8 * 8 + 4 * 4,
           "includes": "exp_create + exp_init_integrals + K iterations + exp_energy, host arrays"}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if ws == 1:
        c1_macs = C1_MACS
        omacs = ORACLE_MACS.get(WORKLOAD["name"]) or macs
        rate, n, dt, cores = cpu_baseline_leg(15.0)
        v = rate * c1_macs / omacs
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n} oracle CCSD iterations at o=10 v=40 C1 in {dt:.1f}s "
                         f"({rate:.2f} iter/s), scaled by the oracle's complex-MAC work per iteration "
                         f"(full pairs: {c1_macs:.4g} -> {omacs:.4g})"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / max(n_it, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else f"bf16x{args.slices}-sliced f64 emulation",
            "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "n_occ": WORKLOAD["n_occ"], "n_virt": WORKLOAD["n_virt"],
                       "irreps": f"Z{WORKLOAD['G']}", "seed": WORKLOAD["seed"], "precision": args.precision,
                       "level_shift": WORKLOAD["shift"],
                       "packed": True,
                       "l2": "inputs larger than L2 (packed <ab||cd> 0.8 GB and its slices 1 GB, "
                             "t2-sized operands 128 MB each, re-read every step)"},
            "complex_tflops": ctflops, "complex_macs_per_iter": macs,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary(), "status": st}
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
