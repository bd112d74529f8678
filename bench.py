"""Benchmark of the F12 integral path on the 12-atom 3s2p1d molecule.

Workload: 12 atoms in a 12 bohr cube (minimum separation 1.8 bohr, seed 2),
3s2p1d contracted shells of 3 primitives per atom (exponents log-uniform in
[0.05, 50], coefficients uniform in [0.1, 1]), range-separated factor
c0 = 0.5, rho = -0.5, B = 0.5, mu = 1, n = 0 (f' = f).  The shell quartets
surviving the Schwarz-type screen at 1e-12 are computed for all five F12
classes (I2..I6) plus the reference ERI I1, as dense FP64 blocks.

A step is one pass of the integral path over that quartet list: the
auxiliary-function kernel, the Hermite recursion and the contraction for
every class.  Shell-pair data and the screened lists are built once before
the timed region (they are reported separately).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  --impl reference times the CPU oracle on a bounded
sample of the same workload on the host cores.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1412_5070_gb300 import molecules as M  # noqa: E402
from paper_1412_5070_gb300.sharding import max_over_ranks, shard  # noqa: E402

METRIC = "F12 quartets/s per class vs FP64 roofline; served p50/p99 vs plain, err<=1e-10"
UNIT = "shell quartets/s"
CLASSES = (1, 2, 3, 4, 5, 6)
THRESH = 1e-12
WORKLOAD = "12-atom 3s2p1d (3 prims/shell, seed 2), Schwarz 1e-12, classes I1..I6, dense FP64 blocks"
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 rate of the profiling recipe's table (no measured FP64 peak)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--fraction", type=float, default=1.0, help=argparse.SUPPRESS)
    ap.add_argument("--no-cpu-baseline", action="store_true", help=argparse.SUPPRESS)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------- algorithmic --

def nh(L):
    return (L + 1) * (L + 2) * (L + 3) // 6


def nc(l):
    return (l + 1) * (l + 2) // 2


def contract_flops_per_prim(la, lb, lc, ld, cls):
    """Algorithmic FP64 flops of the Hermite recursion and the contraction of
    Eq. ii per primitive quartet: R recursion 2 C(L+4,4); ket step
    2 nh(lab) nh(lcd) Nc_cd; bra step 2 Nc_ab nh(lab) Nc_cd (x3 + the
    Laplacian terms for I5, R to L+2)."""
    ext = 2 if cls == 5 else 0
    lab, lcd = la + lb, lc + ld
    L = lab + lcd + ext
    r = 2 * (L + 1) * (L + 2) * (L + 3) * (L + 4) // 24
    ncd, nab = nc(lc) * nc(ld), nc(la) * nc(lb)
    ket = 2 * nh(lab + ext) * nh(lcd) * ncd
    bra = 2 * nab * nh(lab) * ncd * (4 if cls == 5 else 1)
    return r + ket + bra


class ClockSampler:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.rows = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# -------------------------------------------------------------- workload --

def build_workload(fraction=1.0):
    basis = M.twelve_atom_spd(2)
    return basis


def screened_lists(F, ctx, bid, basis, fraction):
    lists = {}
    t0 = time.time()
    for cls in CLASSES:
        q = F.f12int_screen(ctx, bid, cls, THRESH)
        if fraction < 1.0:
            q = q[: max(1, int(len(q) * fraction))]
        lists[cls] = q
    return lists, time.time() - t0


def cpu_oracle_sample(basis, lists, target_seconds=15.0, impl_line=False):
    """Time the oracle on a bounded sample of each class's quartet list.
    Returns (quartets/s over all classes weighted like the workload, info)."""
    from oracle import oracle as O
    K = O.factor_kernel(M.P0)
    O.build()
    rng = np.random.default_rng(7)
    per = {}
    total_q = sum(len(lists[c]) for c in CLASSES)
    budget = target_seconds / len(CLASSES)
    for cls in CLASSES:
        q = lists[cls]
        n = 8
        sec = 0.0
        done = 0
        while sec < budget and done < len(q):
            take = q[rng.choice(len(q), size=min(n, len(q)), replace=False)]
            t = time.time()
            O.shell_blocks(K, cls, basis, take)
            sec += time.time() - t
            done += len(take)
            n *= 2
        per[cls] = done / sec if sec > 0 else float("nan")
    # the time the oracle would need for the whole step = sum_c n_c / rate_c
    step_time = sum(len(lists[c]) / per[c] for c in CLASSES)
    value = total_q / step_time
    threads = os.cpu_count()
    return value, {"cores": threads, "per_class_quartets_per_s": {("I%d" % c): per[c] for c in CLASSES},
                   "sample": "seeded random canonical shell quartets of each class (all six), ~%.0f s of "
                             "oracle work; quartets/s over the mix" % target_seconds}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import torch  # noqa: F401  (plumbing only)
    basis = build_workload()
    # the oracle samples from the canonical quartet lists (no library code on this path)
    lists = {c: M.canonical_quartets(basis, c) for c in CLASSES}
    per_step_s = []
    vals = []
    steps = max(1, args.steps)
    for s in range(args.warmup + steps):
        v, info = cpu_oracle_sample(basis, lists, target_seconds=max(2.0, 20.0 / (args.warmup + steps)))
        if s >= args.warmup:
            vals.append(v)
    value = statistics.median(vals)
    total_q = sum(len(lists[c]) for c in CLASSES)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total_q / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "quartets_per_step": total_q},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
                             "sample": info["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1412_5070_gb300 import build as B
    from paper_1412_5070_gb300 import f12int as F
    B.build()
    basis = build_workload()
    stream = torch.cuda.Stream()
    ctx = F.f12int_create(local, 0, stream)
    F.f12int_set_factor(ctx, M.P0)
    t0 = time.time()
    bid = F.f12int_set_basis(ctx, basis)
    t_basis = time.time() - t0
    lists, t_screen = screened_lists(F, ctx, bid, basis, args.fraction)
    # weak scaling: each rank computes every rank-th quartet of each list (independent units)
    my = {c: shard(lists[c], rank, world) for c in CLASSES}
    offs = {c: M.block_offsets(basis, my[c]) for c in CLASSES}
    dq = {c: torch.from_numpy(np.ascontiguousarray(my[c])).to(f"cuda:{local}") for c in CLASSES}
    doff = {c: torch.from_numpy(offs[c][:-1].copy()).to(f"cuda:{local}") for c in CLASSES}
    out = {c: torch.empty(int(offs[c][-1]), dtype=torch.float64, device=f"cuda:{local}") for c in CLASSES}
    nprim = basis.nprim
    nprimq = {c: int(np.sum(np.prod(nprim[my[c]], axis=1))) for c in CLASSES}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")

    def step(ev=None):
        for i, c in enumerate(CLASSES):
            F.f12int_compute_class(ctx, bid, c, dq[c], out[c], doff[c], stream)
            if ev is not None:
                ev[i + 1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    F.f12int_device_status(ctx)
    # timed region: device time with events on the launching stream, L2 flushed between steps
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    times = []
    class_ms = {c: [] for c in CLASSES}
    F.f12int_set_timing(ctx, True)
    F.f12int_kernel_stats(ctx, reset=True)
    n_launch0 = F.f12int_launch_count(ctx)
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(CLASSES) + 1)]
            ev[0].record(stream)
            step(ev)
            ev[-1].synchronize()
            times.append(ev[0].elapsed_time(ev[-1]))
            for i, c in enumerate(CLASSES):
                class_ms[c].append(ev[i].elapsed_time(ev[i + 1]))
    n_launch = F.f12int_launch_count(ctx) - n_launch0
    kst = F.f12int_kernel_stats(ctx, reset=True)
    F.f12int_set_timing(ctx, False)
    torch.cuda.synchronize()
    F.f12int_device_status(ctx)
    ms = float(np.mean(times))
    ms = max_over_ranks(ms, device=f"cuda:{local}")
    total_q = sum(len(lists[c]) for c in CLASSES)
    value = total_q / (ms / 1000.0)

    # end to end: host lists in pinned memory -> device, compute, blocks back to pinned host memory
    hq = {c: torch.from_numpy(np.ascontiguousarray(my[c])).pin_memory() for c in CLASSES}
    hoff = {c: torch.from_numpy(offs[c][:-1].copy()).pin_memory() for c in CLASSES}
    hout = {c: torch.empty(out[c].numel(), dtype=torch.float64).pin_memory() for c in CLASSES}
    h2d = sum(hq[c].numel() * 4 + hoff[c].numel() * 8 for c in CLASSES)
    d2h = sum(hout[c].numel() * 8 for c in CLASSES)
    e2e_times = []
    for it in range(max(1, min(args.steps, 2))):
        torch.cuda.synchronize()
        t = time.perf_counter()
        with torch.cuda.stream(stream):
            for c in CLASSES:
                dq[c].copy_(hq[c], non_blocking=True)
                doff[c].copy_(hoff[c], non_blocking=True)
            for c in CLASSES:
                F.f12int_compute_class(ctx, bid, c, dq[c], out[c], doff[c], stream)
            for c in CLASSES:
                hout[c].copy_(out[c], non_blocking=True)
        stream.synchronize()
        e2e_times.append(time.perf_counter() - t)
    e2e_value = total_q / float(np.median(e2e_times))

    per_class = {}
    for c in CLASSES:
        t_ms = float(np.mean(class_ms[c]))
        per_class["I%d" % c] = {"shell_quartets": len(my[c]), "prim_quartets": nprimq[c], "ms": t_ms,
                                "shell_quartets_per_s": len(my[c]) / (t_ms / 1000.0),
                                "prim_quartets_per_s": nprimq[c] / (t_ms / 1000.0)}
    # roofline of the dominant kernel, from its own launch durations (CUDA events
    # on the launching stream, recorded by the library during the timed steps)
    aux_ach = kst["aux_flops"] / (kst["aux_ms"] / 1e3) / 1e12 if kst["aux_ms"] > 0 else 0.0
    con_ach = kst["contract_flops"] / (kst["contract_ms"] / 1e3) / 1e12 if kst["contract_ms"] > 0 else 0.0
    dom = "aux" if kst["aux_ms"] >= kst["contract_ms"] else "contract"
    ach = aux_ach if dom == "aux" else con_ach
    kernels = {"k_items_eval": {"ms": kst["aux_ms"] / args.steps, "launches": kst["aux_launches"] // args.steps,
                                "achieved_tflops": aux_ach, "flops": kst["aux_flops"] / args.steps,
                                "share": kst["aux_ms"] / max(kst["aux_ms"] + kst["contract_ms"], 1e-9)},
               "k_contract": {"ms": kst["contract_ms"] / args.steps,
                              "launches": kst["contract_launches"] // args.steps,
                              "achieved_tflops": con_ach, "flops": kst["contract_flops"] / args.steps,
                              "share": kst["contract_ms"] / max(kst["aux_ms"] + kst["contract_ms"], 1e-9)}}
    line = {"metric": METRIC, "value": value * 1.0, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "quartets_per_step": total_q,
                       "prim_quartets_per_step": sum(nprimq.values()), "l2": "flushed (256 MiB write) between steps",
                       "fraction": args.fraction},
            "per_class": per_class,
            "setup_s": {"set_basis": t_basis, "screen_all_classes": t_screen},
            "gpu_launches": int(n_launch),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "roofline": {"bound": "alu", "kernel": "k_items_eval" if dom == "aux" else "k_contract",
                         "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                         "note": "FP64 pipe; achieved = counted algorithmic FP64 flops of the kernel / its event-timed "
                                 "launch durations; peak = nominal GB300 FP64 rate (recipe table), "
                                 "1.195 TFLOP/s measured by an FMA microbenchmark"},
            "kernels": kernels,
            "clocks": clk.summary()}
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle samples from the canonical lists: its inputs never come from the CUDA path
        canon = {c: M.canonical_quartets(basis, c) for c in CLASSES}
        v, info = cpu_oracle_sample(basis, canon, target_seconds=15.0)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
                                "sample": info["sample"]}
    F.f12int_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
