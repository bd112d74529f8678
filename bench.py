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

Two further workloads, each printing its own JSON line:
  --workload batch64  64 molecules (2-30 atoms, 4s3p2d1f, 1-6 primitives,
                      exponents in [0.03, 200]); per molecule a block of 64 x 64
                      significant shell pairs, all six classes: the batched
                      request path (f12int_submit) against one plain
                      f12int_compute_class launch per class and molecule.
  --workload mixed    40 atoms, 5s4p3d2f, 1-8 primitives, exponents [0.02, 500]:
                      per class a bound-stratified sample of shell quartets (half
                      with Schwarz bound product >= 1e-4, half below), FP64 against
                      the mixed path (FP32 recursion and contraction below 1e-4):
                      time and the mixed path's max abs/rel difference.
  --workload perl     the 12-atom workload split by class and (la, lb, lc, ld): shell and
                      primitive quartets/s of every combination, with the FP64 rate of each
                      kernel from the library's event timing and work counters.
  --workload factors  the 12-atom workload (a seeded sample of 200k screened shell quartets
                      per class, I2..I6) for five forms of the correlation factor: Eq. rs12
                      with B = +0.5, with B = -0.5 (a decaying long range, second
                      evaluation launch) and with rho = -1 (singular families, evaluated
                      in groups), the Ten-no factor exp(-1.2 r) and a six-Gaussian
                      geminal (both as term lists): shell quartets/s per class and launches.
  --workload slice    the first --fraction of the 12-atom lists of one class (--cls N) or of
                      all six: one untimed pass, then one pass inside an NVTX range named
                      "profiled" (a profiler can restrict its capture to it with --nvtx
                      --nvtx-include "profiled/"), with the library's per-kernel event
                      timing and work counters: the case every ncu summary names.
  --workload peak     the device's measured FP64 FMA, FP64 matrix (mma.sync) and FP32 FMA
                      peaks (f12int_measure_peak), each twice.
  --workload serve    Poisson request streams at 10..2000 requests/s over 24
                      molecules of 2-60 atoms (one minute of arrivals per rate,
                      at most 2000 requests); half the requests ask for one
                      class, half for I2..I6, each over U{8..64} x U{8..64}
                      significant shell pairs: p50/p99 latency (submit to done)
                      and throughput of the request path against serial plain
                      launches in arrival order (capped at 45 s per rate).

The default line also carries reduced forms of the last two: "batched" (the
first 16 molecules of batch64) and "served" (6 molecules, 2 rates, 300
requests each); --no-legs leaves them out.
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
# DRAM bytes (read + written) of k_items_eval per primitive quartet, per class,
# from one ncu capture of its launches on the 1% slices of the 12-atom lists:
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum
#       --clock-control none --nvtx --nvtx-include "profiled/" -k regex:k_items_eval
#       python bench.py --workload slice --fraction 0.01
# The roofline's traffic is these times the step's primitive quartets per
# class, over the step's launches of the kernel (valid while the kernel is the
# one captured).
AUX_DRAM_BYTES_PER_PRIM_QUARTET = {1: 53.8, 2: 1003.1, 3: 1006.5, 4: 2643.1, 5: 1785.0, 6: 3054.0}
UNIT = "shell quartets/s"
CLASSES = (1, 2, 3, 4, 5, 6)
THRESH = 1e-12
WORKLOAD = "12-atom 3s2p1d (3 prims/shell, seed 2), Schwarz 1e-12, classes I1..I6, dense FP64 blocks"
SLICE_FACTORS = {"P0": M.P0, "Bneg": dict(M.P0, B=-0.5)}
KST_KEYS = ("aux_ms", "aux_launches", "contract_ms", "contract_launches", "aux_flops", "contract_flops")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--workload", default="spd12",
                    choices=("spd12", "batch64", "serve", "mixed", "perl", "factors", "slice", "peak"))
    ap.add_argument("--fraction", type=float, default=1.0,
                    help="spd12/slice: the first fraction of each screened list")
    ap.add_argument("--cls", type=int, default=0, help="slice: one class (0: all six)")
    ap.add_argument("--factor", default="P0", choices=tuple(SLICE_FACTORS),
                    help="slice: correlation factor (P0: Eq. rs12 with B = +0.5; Bneg: B = -0.5, whose "
                         "families with b < 0 go through the quadrature launch)")
    ap.add_argument("--no-cpu-baseline", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--no-legs", action="store_true",
                    help="default workload: skip the reduced batched and served measurements")
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


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip() + " (%s)" % os.uname().machine
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return os.uname().machine


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
    return value, {"cores": threads, "cpu_model": cpu_model(),
                   "per_class_quartets_per_s": {("I%d" % c): per[c] for c in CLASSES},
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
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": info["cores"], "cpu_model": info["cpu_model"], "kind": "oracle",
                             "sample": info["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def aux_traffic_per_launch(nprimq, launches):
    """DRAM bytes per launch of k_items_eval for a step over nprimq[c]
    primitive quartets of class c in `launches` launches (the captured bytes
    per primitive quartet, scaled)."""
    if launches <= 0:
        return None
    return sum(AUX_DRAM_BYTES_PER_PRIM_QUARTET[c] * n for c, n in nprimq.items()) / launches


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
    # per class: the library's kernel stats (event-timed launches, work counters),
    # read after each class (a host synchronisation between classes)
    cls_kst = {c: {k: 0.0 for k in KST_KEYS + ("plan_ms",)} for c in CLASSES}
    F.f12int_host_stats(ctx, reset=True)

    def step_with_stats(ev):
        for i, c in enumerate(CLASSES):
            F.f12int_compute_class(ctx, bid, c, dq[c], out[c], doff[c], stream)
            ev[i + 1].record(stream)
            st = F.f12int_kernel_stats(ctx, reset=True)
            for k in KST_KEYS:
                cls_kst[c][k] += st[k]
            cls_kst[c]["plan_ms"] += F.f12int_host_stats(ctx, reset=True)["plan_ms"]

    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(CLASSES) + 1)]
            ev[0].record(stream)
            step_with_stats(ev)
            ev[-1].synchronize()
            times.append(ev[0].elapsed_time(ev[-1]))
            for i, c in enumerate(CLASSES):
                class_ms[c].append(ev[i].elapsed_time(ev[i + 1]))
    n_launch = F.f12int_launch_count(ctx) - n_launch0
    kst = {k: sum(cls_kst[c][k] for c in CLASSES) for k in KST_KEYS}
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

    # measured arithmetic peaks of this device (the roofline denominators)
    peaks = {k: F.f12int_measure_peak(local, k) for k in ("fp64_fma", "fp64_mma_m8n8k4", "fp32_fma")}
    peak64 = peaks["fp64_fma"]
    per_class = {}
    for c in CLASSES:
        t_ms = float(np.mean(class_ms[c]))
        ks = cls_kst[c]
        a_t = ks["aux_flops"] / (ks["aux_ms"] / 1e3) / 1e12 if ks["aux_ms"] > 0 else 0.0
        c_t = ks["contract_flops"] / (ks["contract_ms"] / 1e3) / 1e12 if ks["contract_ms"] > 0 else 0.0
        per_class["I%d" % c] = {"shell_quartets": len(my[c]), "prim_quartets": nprimq[c], "ms": t_ms,
                                "shell_quartets_per_s": len(my[c]) / (t_ms / 1000.0),
                                "prim_quartets_per_s": nprimq[c] / (t_ms / 1000.0),
                                "aux": {"ms": ks["aux_ms"] / args.steps, "tflops": a_t, "frac": a_t / peak64},
                                "contract": {"ms": ks["contract_ms"] / args.steps, "tflops": c_t,
                                             "frac": c_t / peak64},
                                "host_plan_ms": ks["plan_ms"] / args.steps}
    # roofline of the dominant kernel, from its own launch durations (CUDA events
    # on the launching stream, recorded by the library during the timed steps)
    aux_ach = kst["aux_flops"] / (kst["aux_ms"] / 1e3) / 1e12 if kst["aux_ms"] > 0 else 0.0
    con_ach = kst["contract_flops"] / (kst["contract_ms"] / 1e3) / 1e12 if kst["contract_ms"] > 0 else 0.0
    dom = "aux" if kst["aux_ms"] >= kst["contract_ms"] else "contract"
    ach = aux_ach if dom == "aux" else con_ach
    traffic = aux_traffic_per_launch(nprimq, kst["aux_launches"] / args.steps) if dom == "aux" else None
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
                         "achieved": ach, "peak": peak64, "unit": "TFLOP/s",
                         "frac": ach / peak64, "traffic": traffic,
                         "traffic_note": "DRAM bytes per launch, scaled from an ncu capture of the 1% slices "
                                         "(bytes per primitive quartet and class); mostly local memory of "
                                         "the series (window and coefficient vector per thread)",
                         "note": "FP64 pipe; achieved = counted FP64 flops of the kernel (series and quadrature "
                                 "multiply-adds for k_items_eval, the algorithmic count for k_contract) / its "
                                 "event-timed launch durations; peak = FP64 FMA rate measured in this run "
                                 "(f12int_measure_peak), of measured"},
            "peaks_tflops": peaks,
            "kernels": kernels,
            "streams": {"output_bytes_per_step": int(d2h), "output_gbs": d2h / (ms / 1e3) / 1e9,
                        "note": "dense FP64 blocks the contraction writes per step, over the device step time"},
            "clocks": clk.summary()}
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle samples from the canonical lists: its inputs never come from the CUDA path
        canon = {c: M.canonical_quartets(basis, c) for c in CLASSES}
        v, info = cpu_oracle_sample(basis, canon, target_seconds=15.0)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": info["cores"], "cpu_model": info["cpu_model"],
                                "kind": "oracle", "sample": info["sample"]}
    F.f12int_destroy(ctx)
    del out, dq, doff, flush
    torch.cuda.empty_cache()
    # the batched and served forms on reduced workloads (rank 0 at N = 1 only)
    if rank == 0 and world == 1 and not args.no_legs:
        b = batching_measure(16, 1, 1)
        line["batched"] = {"workload": b["workload"] + " (the first 16 of the 64-molecule batching workload)",
                           "shell_quartets_per_pass": b["shell_quartets_per_pass"],
                           "batched": b["batched"], "plain": b["plain"], "speedup": b["speedup"],
                           "schedule": b["schedule"]}
        r = serving_measure(6, rates=(20, 200), nreq=lambda lam: 300, plain_cap_s=20.0, verbose=False)
        line["served"] = {"workload": r["workload"] + " (6 of the 24 molecules of the serving workload, "
                                                      "2 rates, 300 requests each)",
                          "rates": [{"rate_per_s": x["rate_per_s"], "requests": x["requests"],
                                     "requests_path": x["requests_path"], "plain_serial": x["plain_serial"]}
                                    for x in r["rates"]]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _sizes(basis, quartets):
    nc = (basis.l + 1) * (basis.l + 2) // 2
    q = np.asarray(quartets)
    return nc[q[:, 0]] * nc[q[:, 1]] * nc[q[:, 2]] * nc[q[:, 3]]


def _request_layout(basis, quartets, classes):
    sz = _sizes(basis, quartets).astype(np.int64)
    per = int(sz.sum())
    first = np.concatenate([[0], np.cumsum(sz)[:-1]]).astype(np.int64)
    return np.stack([first + k * per for k in range(len(classes))]), per * len(classes)


def batching_measure(nmol=64, steps=1, warmup=1):
    """Batched requests (f12int_submit, graph replays) against one plain
    f12int_compute_class per class and molecule, over nmol uneven molecules
    (all six classes): seconds per pass and quartets/s of each path."""
    import torch
    from paper_1412_5070_gb300 import build as B
    from paper_1412_5070_gb300 import f12int as F
    B.build()
    work = M.batching_workload(nmol)
    stream = torch.cuda.Stream()
    ctx = F.f12int_create(0, 0, stream)
    try:
        return _batching_measure(F, torch, ctx, stream, work, steps, warmup)
    finally:
        F.f12int_destroy(ctx)   # waits for the engine's work in flight, also on an error


def _batching_measure(F, torch, ctx, stream, work, steps, warmup):
    nmol = len(work)
    F.f12int_set_factor(ctx, M.P0)
    F.f12int_batch_limits(ctx, 1 << 19, 1 << 26)
    t0 = time.time()
    bids = [F.f12int_set_basis(ctx, b) for b, _ in work]
    t_basis = time.time() - t0
    lay = [_request_layout(b, q, CLASSES) for b, q in work]
    outs = [torch.empty(tot, dtype=torch.float64, device="cuda") for _, tot in lay]
    nq = sum(len(q) * len(CLASSES) for _, q in work)
    npq = sum(int(np.sum(np.prod(b.nprim[q], axis=1))) * len(CLASSES) for b, q in work)

    def batched():
        ts = [F.f12int_submit(ctx, bids[i], work[i][1], CLASSES, outs[i], lay[i][0]) for i in range(len(work))]
        left = ts
        while left:
            left = [t for t in left if not F.f12int_poll(ctx, t, 200)]

    dq = [torch.from_numpy(np.ascontiguousarray(q)).cuda() for _, q in work]
    doff = [[torch.from_numpy(lay[i][0][k].copy()).cuda() for k in range(len(CLASSES))] for i in range(len(work))]

    def plain():
        for i in range(len(work)):
            for k, c in enumerate(CLASSES):
                F.f12int_compute_class(ctx, bids[i], c, dq[i], outs[i], doff[i][k], stream)
        stream.synchronize()

    t0 = time.time()
    batched()   # first pass: primitive bounds of every (molecule, class), buffers, graph capture
    t_first = time.time() - t0
    # per-class schedules measured on the first molecule's block
    t0 = time.time()
    tuned = F.f12int_batch_autotune(ctx, bids[0], work[0][1], CLASSES)
    t_tune = time.time() - t0
    for _ in range(max(0, warmup - 1)):
        batched()
        plain()
    res = {}
    for name, fn in (("batched", batched), ("plain", plain)):
        ts = []
        for _ in range(max(1, steps)):
            torch.cuda.synchronize()
            l0 = F.f12int_launch_count(ctx)
            b0 = F.f12int_batch_stats(ctx)["batches"]
            t = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t)
            launches = F.f12int_launch_count(ctx) - l0
            batches = F.f12int_batch_stats(ctx)["batches"] - b0
        sec = float(np.median(ts))
        res[name] = {"s_per_pass": sec, "shell_quartets_per_s": nq / sec, "prim_quartets_per_s": npq / sec,
                     "graph_replays": batches if name == "batched" else 0,
                     "plain_launches": launches if name == "plain" else 0}
    F.f12int_device_status(ctx)
    return {"workload": "%d molecules (seeds 1000-%d, 2-30 atoms, 4s3p2d1f, 1-6 primitives, exponents "
                        "[0.03, 200]); 64 x 64 significant shell pairs each; I1..I6" % (nmol, 999 + nmol),
            "shell_quartets_per_pass": nq, "prim_quartets_per_pass": npq,
            "batched": res["batched"], "plain": res["plain"],
            "speedup": res["plain"]["s_per_pass"] / res["batched"]["s_per_pass"],
            "setup_s": {"set_basis": t_basis, "first_pass_with_bounds": t_first, "autotune": t_tune},
            "schedule": {"I%d" % c: {"task_flops": v[0], "aux_grid_divisor": v[1]} for c, v in tuned.items()},
            "timing": "wall clock from first submit to last completion (host list building included)"}


def run_batching(args):
    """64 uneven molecules, all six classes: batched requests vs plain launches."""
    r = batching_measure(64, args.steps, args.warmup)
    line = {"metric": "F12 quartets/s over an uneven 64-molecule batch, graph-replayed requests vs plain launches",
            "value": r["batched"]["shell_quartets_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": r["workload"], "shell_quartets_per_pass": r["shell_quartets_per_pass"],
                       "prim_quartets_per_pass": r["prim_quartets_per_pass"],
                       "batch_limits": {"quartets_per_class": 1 << 19, "items_per_class": 1 << 26}},
            **{k: r[k] for k in ("batched", "plain", "speedup", "setup_s", "schedule", "timing")}}
    print(json.dumps(line), flush=True)


def serving_measure(pool_n=12, rates=(10, 20, 50, 100, 200, 500, 1000, 2000), nreq=None, plain_cap_s=90.0,
                    verbose=True):
    """Poisson request streams over a pool of seeded molecules: p50/p99
    latency (arrival to completion seen by poll) and shell quartets/s of the
    request path (f12int_submit / f12int_poll, continuous batching), against
    the same requests run one after another with plain f12int_compute_class
    calls (capped at plain_cap_s per rate).  nreq(rate) gives the requests per
    rate (default: one minute of arrivals, at most 2000)."""
    import torch
    from paper_1412_5070_gb300 import build as B
    from paper_1412_5070_gb300 import f12int as F
    B.build()
    if nreq is None:
        nreq = lambda lam: int(min(2000, 60 * lam))
    pool = M.serving_pool(pool_n)
    stream = torch.cuda.Stream()
    ctx = F.f12int_create(0, 0, stream)
    try:
        return _serving_measure(F, torch, ctx, stream, pool, pool_n, rates, nreq, plain_cap_s, verbose)
    finally:
        F.f12int_destroy(ctx)   # waits for the engine's work in flight, also on an error


def _serving_measure(F, torch, ctx, stream, pool, pool_n, rates, nreq, plain_cap_s, verbose):
    F.f12int_set_factor(ctx, M.P0)
    F.f12int_batch_limits(ctx, 1 << 18, 1 << 25)
    bids = [F.f12int_set_basis(ctx, b) for b in pool]
    # one-time bounds of every (molecule, class) before any timing
    t0 = time.time()
    warm = []
    for i, b in enumerate(pool):
        q = M.pair_block(b, 2, 2, 7)
        off, tot = _request_layout(b, q, (2, 3, 4, 5, 6))
        o = torch.empty(tot, dtype=torch.float64, device="cuda")
        warm.append((o, F.f12int_submit(ctx, bids[i], q, (2, 3, 4, 5, 6), o, off)))
    for _, t in warm:
        while not F.f12int_poll(ctx, t, 1000):
            pass
    t_bounds = time.time() - t0
    # per-class schedules measured on one request-sized block (40 x 40 pairs of a mid-size molecule)
    mid = int(np.argsort([b.nshell for b in pool])[len(pool) // 2])
    tuned = F.f12int_batch_autotune(ctx, bids[mid], M.pair_block(pool[mid], 40, 40, 3), (2, 3, 4, 5, 6))
    t_setup = time.time() - t0
    if verbose:
        print("serving: setup %.1f s (bounds %.1f s)" % (t_setup, t_bounds), file=sys.stderr, flush=True)
    rows = []
    for lam in rates:
        reqs = M.serving_requests(nreq(lam), float(lam), pool, seed=5 + lam)
        prep = []
        for (ta, m, classes, q) in reqs:
            off, tot = _request_layout(pool[m], q, classes)
            o = torch.empty(tot, dtype=torch.float64, device="cuda")
            prep.append((ta, m, classes, q, off, o))
        nq = sum(len(r[3]) * len(r[2]) for r in prep)
        torch.cuda.synchronize()
        # request path: submit at the arrival times, a poller records completions
        done = {}
        tickets = {}
        lock = threading.Lock()
        stop = [False]

        def poller():
            while True:
                with lock:
                    items = list(tickets.items())
                for k, t in items:
                    if F.f12int_poll(ctx, t, 0):
                        done[k] = time.perf_counter()
                        with lock:
                            del tickets[k]
                if stop[0] and not tickets:
                    return
                time.sleep(50e-6)

        th = threading.Thread(target=poller)
        start = time.perf_counter()
        th.start()
        sub = {}
        for k, (ta, m, classes, q, off, o) in enumerate(prep):
            wait_s = start + ta - time.perf_counter()
            if wait_s > 0:
                time.sleep(wait_s)
            sub[k] = start + ta
            t = F.f12int_submit(ctx, bids[m], q, classes, o, off)
            with lock:
                tickets[k] = t
        stop[0] = True
        th.join()
        lat = np.array([done[k] - sub[k] for k in range(len(prep))]) * 1e3
        span = max(done.values()) - start
        eng = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
               "shell_quartets_per_s": nq / span, "requests_per_s": len(prep) / span}
        if verbose:
            print("serving: rate %d/s, %d requests: requests path p50 %.1f ms p99 %.1f ms" % (
                lam, len(prep), eng["p50_ms"], eng["p99_ms"]), file=sys.stderr, flush=True)
        # serial plain launches in arrival order (capped)
        lat2 = []
        nq2 = 0
        start = time.perf_counter()
        for (ta, m, classes, q, off, o) in prep:
            if time.perf_counter() - start > plain_cap_s:
                break
            wait_s = start + ta - time.perf_counter()
            if wait_s > 0:
                time.sleep(wait_s)
            dq = torch.from_numpy(np.ascontiguousarray(q)).cuda()
            for k, c in enumerate(classes):
                F.f12int_compute_class(ctx, bids[m], c, dq, o, torch.from_numpy(off[k].copy()).cuda(), stream)
            stream.synchronize()
            lat2.append(time.perf_counter() - (start + ta))
            nq2 += len(q) * len(classes)
        span2 = time.perf_counter() - start
        lat2 = np.array(lat2) * 1e3
        plain = {"p50_ms": float(np.percentile(lat2, 50)), "p99_ms": float(np.percentile(lat2, 99)),
                 "shell_quartets_per_s": nq2 / span2, "requests_completed": len(lat2),
                 "truncated": len(lat2) < len(prep)}
        if verbose:
            print("serving: rate %d/s: plain p50 %.1f ms p99 %.1f ms (%d of %d)" % (
                lam, plain["p50_ms"], plain["p99_ms"], len(lat2), len(prep)), file=sys.stderr, flush=True)
        rows.append({"rate_per_s": lam, "requests": len(prep), "shell_quartets": nq, "requests_path": eng,
                     "plain_serial": plain})
        del prep
    F.f12int_device_status(ctx)
    return {"workload": "%d molecules (seeds 500-%d, 2-60 atoms, 4s3p2d1f, 1-6 primitives); Poisson arrivals; "
                        "half one class of I2..I6, half all five; U{8..64} x U{8..64} significant shell pairs "
                        "per request" % (pool_n, 499 + pool_n),
            "batch_limits": {"quartets_per_class": 1 << 18, "items_per_class": 1 << 25},
            "rates": rows, "setup_s": t_setup, "bounds_s": t_bounds,
            "schedule": {"I%d" % c: {"task_flops": v[0], "aux_grid_divisor": v[1]} for c, v in tuned.items()}}


def run_serving(args):
    """Poisson request streams: latency and throughput, requests vs serial plain launches."""
    r = serving_measure(24, plain_cap_s=45.0)
    best = max(x["requests_path"]["shell_quartets_per_s"] for x in r["rates"])
    line = {"metric": "served p50/p99 latency (submit to done) and quartets/s, requests vs serial plain launches",
            "value": best, "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": "f64",
            "data": "synthetic", "config": {"workload": r["workload"], "batch_limits": r["batch_limits"]},
            **{k: r[k] for k in ("rates", "setup_s", "bounds_s", "schedule")}}
    print(json.dumps(line), flush=True)


def run_mixed(args):
    """FP64 vs mixed precision on a bound-stratified sample of a large f-shell molecule."""
    import torch
    from paper_1412_5070_gb300 import build as B
    from paper_1412_5070_gb300 import f12int as F
    B.build()
    basis = M.c4_molecule(40)
    stream = torch.cuda.Stream()
    ctx = F.f12int_create(0, 0, stream)
    F.f12int_set_factor(ctx, M.P0)
    bid = F.f12int_set_basis(ctx, basis)
    split = 1e-4   # sample split; errors are reported per decade of the estimate
    per_class = {}
    total = {"fp64_s": 0.0, "mixed_s": 0.0, "quartets": 0}
    nper = 1_000_000 // len(CLASSES)
    for c in CLASSES:
        pb = F.f12int_pair_bounds(ctx, bid, c, basis.nshell)
        # candidates from the pair bounds, kept by the library's screening estimate
        cand = M.bound_stratified_quartets(pb, 4 * nper, split, 1e-16, 400 + c, canonical_braket=(c != 5))
        est_c = F.f12int_quartet_estimates(ctx, bid, c, cand)
        hi = cand[est_c >= split][: nper // 2]
        lo = cand[(est_c < split) & (est_c >= 1e-12)][: nper - len(hi)]
        q = np.ascontiguousarray(np.concatenate([hi, lo]))
        est = F.f12int_quartet_estimates(ctx, bid, c, q)
        off = M.block_offsets(basis, q)
        dq = torch.from_numpy(q).cuda()
        doff = torch.from_numpy(off[:-1].copy()).cuda()
        o64 = torch.empty(int(off[-1]), dtype=torch.float64, device="cuda")
        o32 = torch.empty(int(off[-1]), dtype=torch.float64, device="cuda")
        F.f12int_compute_class(ctx, bid, c, dq, o64, doff, stream)   # warm-up
        F.f12int_compute_class_mixed(ctx, bid, c, dq, o32, doff, split, stream)
        stream.synchronize()
        ts, kst = {}, {}
        for name in ("fp64", "mixed"):
            F.f12int_set_timing(ctx, True)
            F.f12int_kernel_stats(ctx, reset=True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if name == "fp64":
                F.f12int_compute_class(ctx, bid, c, dq, o64, doff, stream)
            else:
                F.f12int_compute_class_mixed(ctx, bid, c, dq, o32, doff, split, stream)
            e1.record(stream)
            e1.synchronize()
            ts[name] = e0.elapsed_time(e1) / 1e3
            st = F.f12int_kernel_stats(ctx, reset=True)
            F.f12int_set_timing(ctx, False)
            kst[name] = {"aux_ms": st["aux_ms"], "contract_ms": st["contract_ms"]}
        a = o64.cpu().numpy()
        b = o32.cpu().numpy()
        d = np.abs(a - b)
        big = np.abs(a) > 1e-12
        # largest difference per decade of the quartets' bound product (FP32 side)
        prod = est
        qmax = np.maximum.reduceat(d, off[:-1]) if len(d) else np.zeros(0)
        by_decade = {}
        for k in range(4, 13):
            sel = (prod < 10.0 ** -k * 10) & (prod >= 10.0 ** -k)
            if sel.any():
                by_decade["[1e-%d,1e-%d)" % (k, k - 1)] = float(qmax[sel].max())
        nprim = int(np.sum(np.prod(basis.nprim[q], axis=1)))
        per_class["I%d" % c] = {"shell_quartets": len(q), "prim_quartets": nprim,
                                "fp32_quartets": int(np.sum(est < split)),
                                "fp64_s": ts["fp64"], "mixed_s": ts["mixed"], "speedup": ts["fp64"] / ts["mixed"],
                                "kernels_ms": kst,
                                "max_abs_diff": float(d.max()),
                                "max_rel_diff_where_abs_gt_1e-12": float((d[big] / np.abs(a[big])).max()) if big.any() else 0.0,
                                "max_abs_diff_by_bound_decade": by_decade}
        total["fp64_s"] += ts["fp64"]
        total["mixed_s"] += ts["mixed"]
        total["quartets"] += len(q)
        print("mixed: I%d %s" % (c, json.dumps(per_class["I%d" % c])), file=sys.stderr, flush=True)
        del o64, o32
    F.f12int_device_status(ctx)
    line = {"metric": "F12 quartets/s, mixed precision (FP32 recursion/contraction below Schwarz 1e-4) vs FP64",
            "value": total["quartets"] / total["mixed_s"], "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
            "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": "40 atoms (seed 40, 20 bohr cube), 5s4p3d2f, 1-8 primitives, exponents "
                                   "[0.02, 500]; per class up to %d shell quartets, half with screening estimate >= 1e-4, "
                                   "half in [1e-12, 1e-4)" % nper, "fp32_below": split},
            "fp64_value": total["quartets"] / total["fp64_s"], "per_class": per_class,
            "error_reference": "the FP64 path of the same library (itself checked against the oracle)"}
    F.f12int_destroy(ctx)
    print(json.dumps(line), flush=True)


def run_per_l(args):
    """Per class and (la, lb, lc, ld): rates and kernel FP64 rates on the 12-atom workload."""
    import torch
    from paper_1412_5070_gb300 import build as B
    from paper_1412_5070_gb300 import f12int as F
    B.build()
    basis = build_workload()
    stream = torch.cuda.Stream()
    ctx = F.f12int_create(0, 0, stream)
    F.f12int_set_factor(ctx, M.P0)
    bid = F.f12int_set_basis(ctx, basis)
    lists, _ = screened_lists(F, ctx, bid, basis, 1.0)
    rows = []
    for c in CLASSES:
        q = lists[c]
        key = basis.l[q] @ np.array([1000, 100, 10, 1])
        for k in np.unique(key):
            sub = np.ascontiguousarray(q[key == k])
            off = M.block_offsets(basis, sub)
            dq = torch.from_numpy(sub).cuda()
            doff = torch.from_numpy(off[:-1].copy()).cuda()
            out = torch.empty(int(off[-1]), dtype=torch.float64, device="cuda")
            F.f12int_compute_class(ctx, bid, c, dq, out, doff, stream)   # warm-up
            stream.synchronize()
            F.f12int_set_timing(ctx, True)
            F.f12int_kernel_stats(ctx, reset=True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            F.f12int_compute_class(ctx, bid, c, dq, out, doff, stream)
            e1.record(stream)
            e1.synchronize()
            st = F.f12int_kernel_stats(ctx, reset=True)
            F.f12int_set_timing(ctx, False)
            ms = e0.elapsed_time(e1)
            npq = int(np.sum(np.prod(basis.nprim[sub], axis=1)))
            rows.append({"class": "I%d" % c, "l": [int(x) for x in basis.l[sub[0]]], "shell_quartets": len(sub),
                         "prim_quartets": npq, "ms": ms, "shell_quartets_per_s": len(sub) / (ms / 1e3),
                         "prim_quartets_per_s": npq / (ms / 1e3),
                         "aux_tflops": st["aux_flops"] / (st["aux_ms"] / 1e3) / 1e12 if st["aux_ms"] else 0.0,
                         "contract_tflops": st["contract_flops"] / (st["contract_ms"] / 1e3) / 1e12
                         if st["contract_ms"] else 0.0,
                         "aux_share": st["aux_ms"] / max(st["aux_ms"] + st["contract_ms"], 1e-9)})
            del out
        print("perl: I%d done" % c, file=sys.stderr, flush=True)
    F.f12int_device_status(ctx)
    line = {"metric": "F12 quartets/s per class and (la,lb,lc,ld), with kernel FP64 rates", "unit": UNIT,
            "n_gpus": 1, "dtype": "f64", "data": "synthetic", "config": {"workload": WORKLOAD},
            "fp64_peak_tflops": F.f12int_measure_peak(0, "fp64_fma"), "rows": rows}
    F.f12int_destroy(ctx)
    print(json.dumps(line), flush=True)


FACTOR_FORMS = {
    "rs12 B=+0.5": ("rs12", M.P0),
    "rs12 B=-0.5": ("rs12", dict(M.P0, B=-0.5)),
    "rs12 rho=-1 (singular)": ("rs12", dict(M.P0, rho=-1.0)),
    "Ten-no exp(-1.2 r)": ("terms", [(1.0, 0, -1.2, 0)]),
    "6 Gaussians": ("terms", [(0.5 / (i + 1), 0, 0, 0.2 * 2.5 ** i) for i in range(6)]),
}


def run_factors(args):
    """Shell quartets/s per class for several forms of the correlation factor."""
    import torch
    from paper_1412_5070_gb300 import build as B
    from paper_1412_5070_gb300 import f12int as F
    B.build()
    basis = build_workload()
    stream = torch.cuda.Stream()
    ctx = F.f12int_create(0, 0, stream)
    bid = F.f12int_set_basis(ctx, basis)
    rng = np.random.default_rng(11)
    per = 200_000
    steps = max(1, args.steps)
    results = {}
    for name, (kind, f) in FACTOR_FORMS.items():
        if kind == "rs12":
            F.f12int_set_factor(ctx, f)
        else:
            F.f12int_set_factor_terms(ctx, f)
        row = {}
        for c in (2, 3, 4, 5, 6):
            q = F.f12int_screen(ctx, bid, c, THRESH)
            q = np.ascontiguousarray(q[np.sort(rng.choice(len(q), size=min(per, len(q)), replace=False))])
            off = M.block_offsets(basis, q)
            dq = torch.from_numpy(q).cuda()
            doff = torch.from_numpy(off[:-1].copy()).cuda()
            out = torch.empty(int(off[-1]), dtype=torch.float64, device="cuda")
            F.f12int_compute_class(ctx, bid, c, dq, out, doff, stream)   # warm-up
            stream.synchronize()
            n0 = F.f12int_launch_count(ctx)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                F.f12int_compute_class(ctx, bid, c, dq, out, doff, stream)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / steps
            row["I%d" % c] = {"shell_quartets": len(q), "ms": ms, "shell_quartets_per_s": len(q) / (ms / 1e3),
                              "launches": (F.f12int_launch_count(ctx) - n0) // steps}
            del out
        F.f12int_device_status(ctx)
        results[name] = row
        print("factors: %s done" % name, file=sys.stderr, flush=True)
    F.f12int_destroy(ctx)
    line = {"metric": "F12 shell quartets/s per class for several correlation-factor forms", "unit": UNIT,
            "n_gpus": 1, "steps": steps, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "12-atom 3s2p1d (seed 2), Schwarz 1e-12 per factor, seeded sample of "
                                   "%d quartets per class" % per,
                       "factors": {k: v[1] for k, v in FACTOR_FORMS.items()}},
            "results": results}
    print(json.dumps(line), flush=True)


def run_slice(args):
    """One class (or all) on a slice of the 12-atom lists, for profilers."""
    import torch
    from paper_1412_5070_gb300 import build as B
    from paper_1412_5070_gb300 import f12int as F
    B.build()
    basis = build_workload()
    stream = torch.cuda.Stream()
    ctx = F.f12int_create(0, 0, stream)
    F.f12int_set_factor(ctx, SLICE_FACTORS[args.factor])
    bid = F.f12int_set_basis(ctx, basis)
    classes = CLASSES if args.cls == 0 else (args.cls,)
    lists, _ = screened_lists(F, ctx, bid, basis, args.fraction)
    rows = {}
    for c in classes:
        q = np.ascontiguousarray(lists[c])
        off = M.block_offsets(basis, q)
        dq = torch.from_numpy(q).cuda()
        doff = torch.from_numpy(off[:-1].copy()).cuda()
        out = torch.empty(int(off[-1]), dtype=torch.float64, device="cuda")
        F.f12int_compute_class(ctx, bid, c, dq, out, doff, stream)   # warm-up (and primitive bounds)
        stream.synchronize()
        F.f12int_set_timing(ctx, True)
        F.f12int_kernel_stats(ctx, reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("profiled")
        e0.record(stream)
        F.f12int_compute_class(ctx, bid, c, dq, out, doff, stream)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        e1.synchronize()
        st = F.f12int_kernel_stats(ctx, reset=True)
        F.f12int_set_timing(ctx, False)
        npq = int(np.sum(np.prod(basis.nprim[q], axis=1)))
        rows["I%d" % c] = {"shell_quartets": len(q), "prim_quartets": npq, "ms": e0.elapsed_time(e1),
                           "aux_ms": st["aux_ms"], "aux_launches": st["aux_launches"],
                           "contract_ms": st["contract_ms"], "contract_launches": st["contract_launches"],
                           "aux_counted_tflops": st["aux_flops"] / (st["aux_ms"] / 1e3) / 1e12 if st["aux_ms"] else 0,
                           "contract_tflops": st["contract_flops"] / (st["contract_ms"] / 1e3) / 1e12
                           if st["contract_ms"] else 0}
        del out
    F.f12int_device_status(ctx)
    F.f12int_destroy(ctx)
    print(json.dumps({"workload": "slice", "fraction": args.fraction, "factor": args.factor, "classes": rows}),
          flush=True)


def run_peak(args):
    from paper_1412_5070_gb300 import build as B
    from paper_1412_5070_gb300 import f12int as F
    B.build()
    res = {k: [F.f12int_measure_peak(0, k) for _ in range(2)] for k in F.PEAK_KINDS}
    print(json.dumps({"workload": "peak", "unit": "TFLOP/s", "peaks": res}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batching(args)
    elif args.workload == "serve":
        run_serving(args)
    elif args.workload == "mixed":
        run_mixed(args)
    elif args.workload == "perl":
        run_per_l(args)
    elif args.workload == "factors":
        run_factors(args)
    elif args.workload == "slice":
        run_slice(args)
    elif args.workload == "peak":
        run_peak(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
