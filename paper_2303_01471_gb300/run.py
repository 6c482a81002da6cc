"""Command-line runner: one seeded instance through the C ABI.

  python -m paper_2303_01471_gb300.run --shape 256 256 256 --family wells --K 32 \
      --T 0.02 --dt 1e-3 [--repeat 2] [--batch B] [--tc PRODUCTS]

Prints the observables and the device time of the evolve call as JSON.  Used
for profiling single configurations (e.g. under ncu) and as a usage example.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    import numpy as np
    import torch
    import workloads
    from paper_2303_01471_gb300 import qhd

    ap = argparse.ArgumentParser()
    ap.add_argument("--shape", type=int, nargs="+", default=[128, 128])
    ap.add_argument("--family", choices=["wells", "rastrigin"], default="wells")
    ap.add_argument("--K", type=int, default=8)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--T", type=float, default=10.0)
    ap.add_argument("--dt", type=float, default=0.01)
    ap.add_argument("--batch", type=int, default=1)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--tc", type=int, default=0, choices=[0, 3, 5, 10],
                    help="tensor-core DFT transform with this many products (0: FFT passes)")
    a = ap.parse_args(argv)
    kw = {"K": a.K} if a.family == "wells" else {}
    insts = [workloads.make(a.family, a.seed + b, a.shape, **kw) for b in range(a.batch)]
    f = np.stack([i.f for i in insts])
    sim = qhd.QHD(a.shape, batch=a.batch)
    sim.set_potential(f)
    sim.set_schedule(qhd.Schedule())
    if a.tc:
        sim.set_transform(qhd.TRANSFORM_TC_DFT, a.tc)
    times = []
    for _ in range(a.repeat):
        sim.reset_state()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sim.evolve(a.T, a.dt)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    obs = sim.observables(0.1)
    steps = int(round(a.T / a.dt))
    g = int(np.prod(a.shape))
    print(json.dumps({"shape": a.shape, "batch": a.batch, "steps": steps, "evolve_ms": times,
                      "pt_steps_per_s": g * a.batch * steps / (min(times) / 1e3),
                      "obs": [o.__dict__ for o in obs]}))
    sim.close()


if __name__ == "__main__":
    main()
