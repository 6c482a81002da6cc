"""Write the FP64 oracle's full-length results for the two instances of the scale
workload (10^4 Strang steps, T = 10, dt = 1e-3, the paper's schedule):

  * 2-D 1024x1024 Rastrigin type, seed 0,
  * 3-D 256^3 Gaussian wells (K = 32), seed 1.

This calls only the oracle and the seeded input generator.  For each instance it
stores, in tests/golden/fullsize_<name>.npz: the observables (norm, E[f], P_succ,
x*), the probability mass p = |psi|^2 on the smallest set of mesh points that
holds all but MASS_LEFT of it, at most keep_max points per case (flat indices and
FP64 values, largest first), the mass outside that set, and the mass outside the
top 2^k points for k = 10..24.  A test then bounds the total-variation distance of
any other p from above without the full array:
  TV <= 1/2 [ sum_{i in S} |p_i - q_i| + (mass of p outside S) + (mass of q outside S) ].

The key of each file is a hash of the instance parameters and the step setup, so
a changed workload is never compared with a stale reference.

  python tests/golden/make_fullsize_reference.py [name ...]    (hours for 256^3 on 8 cores)
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402

T_END, DT = 10.0, 1e-3
NSTEPS = 10000
MASS_LEFT = 1e-7
# at most this many points per file (the rest is stored as one mass): the 2-D state
# is concentrated, the 3-D one is spread over a ball of ~10^5 points and a long tail
CASES = {
    "1024sq_rastrigin": dict(family="rastrigin", seed=0, shape=(1024, 1024), kw={}, keep_max=32768),
    "256cube_wells": dict(family="wells", seed=1, shape=(256, 256, 256), kw={"K": 32}, keep_max=262144),
}


def case_key(name: str) -> str:
    c = CASES[name]
    text = json.dumps({"family": c["family"], "seed": c["seed"], "shape": list(c["shape"]), "kw": c["kw"],
                       "T": T_END, "dt": DT, "nsteps": NSTEPS, "schedule": "nesterov c_phi=2 eps=1e-3 c_chi=2",
                       "psi0": "uniform", "split": "strang"}, sort_keys=True)
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def path_of(name: str) -> str:
    return os.path.join(HERE, f"fullsize_{name}.npz")


def make(name: str) -> str:
    c = CASES[name]
    inst = workloads.make(c["family"], c["seed"], c["shape"], **c["kw"])
    psi = oracle.uniform_state(inst.shape)
    t0 = time.time()
    chunk = 500
    for j0 in range(0, NSTEPS, chunk):
        psi = oracle.evolve(inst.f, psi, j0 * DT, DT, chunk, oracle.Schedule())
        print(f"{name}: {j0 + chunk}/{NSTEPS} steps, {time.time() - t0:.0f} s", flush=True)
    ob = oracle.observables(inst.f, psi, 0.1)
    p = ob.prob.ravel()
    order = np.argsort(p)[::-1]
    cum = np.cumsum(p[order])
    keep = min(int(np.searchsorted(cum, cum[-1] - MASS_LEFT)) + 1, c["keep_max"])
    idx = order[:keep].astype(np.int64 if p.size >= 2 ** 31 else np.int32)
    # mass outside the top 2^k points, for k = 10 .. 24 (how spread the state is)
    profile = np.array([[2 ** k, float(cum[-1] - cum[min(2 ** k, p.size) - 1])] for k in range(10, 25)
                        if 2 ** k <= p.size])
    out = path_of(name)
    np.savez_compressed(out, key=case_key(name), norm=ob.norm, e_f=ob.e_f, p_succ=ob.p_succ,
                        x_star=np.asarray(ob.x_star, dtype=np.float64), idx=idx, p=p[idx],
                        mass_outside=float(p.sum() - p[idx].sum()), f_ptp=float(np.ptp(inst.f)),
                        mass_profile=profile, seconds=time.time() - t0, threads=oracle.max_threads())
    return out


if __name__ == "__main__":
    for nm in sys.argv[1:] or list(CASES):
        print(make(nm))
