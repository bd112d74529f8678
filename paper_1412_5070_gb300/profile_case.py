"""Run one integral class on a slice of the 12-atom 3s2p1d workload.

  python -m paper_1412_5070_gb300.profile_case --cls 3 --fraction 0.003

Builds the library if needed, screens the class at 1e-12, computes the
first `fraction` of the surviving quartets once untimed, then once more
inside an NVTX range named "profiled" (so a profiler can restrict its
capture to that pass with --nvtx --nvtx-include "profiled/"), and prints
the event-timed milliseconds of the second pass.
"""
from __future__ import annotations

import argparse

import numpy as np
import torch

from . import build as B
from . import f12int as F
from . import molecules as M


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cls", type=int, default=3)
    ap.add_argument("--fraction", type=float, default=0.003)
    args = ap.parse_args()
    B.build()
    basis = M.twelve_atom_spd(2)
    ctx = F.f12int_create(0, 0, None)
    try:
        F.f12int_set_factor(ctx, M.P0)
        bid = F.f12int_set_basis(ctx, basis)
        q = F.f12int_screen(ctx, bid, args.cls, 1e-12)
        q = np.ascontiguousarray(q[: max(1, int(len(q) * args.fraction))])
        off = M.block_offsets(basis, q)
        dq = torch.from_numpy(q).cuda()
        doff = torch.from_numpy(off[:-1].copy()).cuda()
        out = torch.empty(int(off[-1]), dtype=torch.float64, device="cuda")
        F.f12int_compute_class(ctx, bid, args.cls, dq, out, doff)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("profiled")
        e0.record()
        F.f12int_compute_class(ctx, bid, args.cls, dq, out, doff)
        e1.record()
        torch.cuda.nvtx.range_pop()
        e1.synchronize()
        F.f12int_device_status(ctx)
        print("class I%d: %d shell quartets, %.2f ms" % (args.cls, len(q), e0.elapsed_time(e1)))
    finally:
        F.f12int_destroy(ctx)


if __name__ == "__main__":
    main()
