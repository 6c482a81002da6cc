#!/usr/bin/env python3
"""Benchmark of the QHD split-operator path on GB300.

Workload (one bench step = one complete simulation of each instance, every
row of the hot path: set f, schedule tables, uniform psi0, 10^4 Strang steps,
observables):
  * 2-D 1024x1024 mesh on [0,1]^2, shifted Rastrigin f (A=10, B=1, omega=5),
  * 3-D 256^3 mesh on [0,1]^3, Gaussian-well f (K=32),
both complex64, T = 10, dt = 1e-3, e^phi = 2/(1e-3 + t^3), e^chi = 2 t^3.

Metric: grid-point Strang steps per second (sum over instances of
G * steps / wall time of the device work), plus instances/s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own replica of the workload with
its own seeds ("replicas only": the instances are independent, no data-path
collective); rank 0 prints the single JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

T_END, DT = 10.0, 1e-3
NSTEPS = int(round(T_END / DT))
METRIC = "grid-point Strang steps/s"
WORKLOAD = ("QHD at scale, complex64, T=10, dt=1e-3 (10^4 Strang steps each): "
            "2-D 1024^2 shifted Rastrigin (A=10,B=1,omega=5) + 3-D 256^3 Gaussian wells (K=32), "
            "paper schedule e^phi=2/(1e-3+t^3), e^chi=2t^3, uniform psi0")
# algorithmic bytes per grid point per launch of each pass (psi read+write,
# plus the 32-bit fixed-point potential in the pass that applies it)
BYTES_PER_POINT = {"row": 20, "axis1_fwd": 16, "axis0": 16, "axis1_inv": 16, "plane": 20}
# DRAM bytes (read + write) of one launch from an ncu capture (not measured by
# this run), with the SHA-256 (first 16 hex digits) of the kernel sources it was
# taken on; bench lines carry the figure only while those sources are unchanged.
TRAFFIC_PER_LAUNCH = {("plane", "256x256x256"): {"bytes": 201427968 + 77629696, "sources_sha16": "d0e447d7b574d27d",
                                                  "captured": "ncu --metrics dram__bytes_read.sum,"
                                                              "dram__bytes_write.sum, one launch, 256^3 wells"}}
TRAFFIC_SOURCES = ["paper_2303_01471_gb300/csrc/qhd_plane.cu", "paper_2303_01471_gb300/csrc/qhd_plane.cuh",
                   "paper_2303_01471_gb300/csrc/qhd_device.cuh"]


def sources_sha16(paths=TRAFFIC_SOURCES) -> str:
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_entry(kernel: str, instance: str):
    """(bytes, note) of the recorded capture, or (None, why) when there is none or
    the kernel sources changed since it was taken."""
    e = TRAFFIC_PER_LAUNCH.get((kernel, instance))
    if e is None:
        return None, "no ncu capture recorded for this kernel"
    if e["sources_sha16"] != sources_sha16():
        return None, "kernel sources changed since the recorded ncu capture"
    return e["bytes"], f"from an earlier ncu capture ({e['captured']}), not measured in this run"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def cases_for_rank(rank: int):
    return [("rastrigin", 1000 * rank + 0, (1024, 1024), {}),
            ("wells", 1000 * rank + 1, (256, 256, 256), {"K": 32})]


def make_instances(rank: int):
    out = []
    for fam, seed, shape, kw in cases_for_rank(rank):
        out.append(workloads.make(fam, seed, shape, **kw))
    return out


# ------------------------------------------------------------- clocks sampler
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def device_record(dev):
    """SM count, L2 size and the measured arithmetic rates of the device the bench ran on."""
    import torch
    from paper_2303_01471_gb300 import probe
    p = torch.cuda.get_device_properties(dev)
    rates = probe.alu_rates()
    return {"name": p.name, "sms": p.multi_processor_count,
            "l2_bytes": getattr(p, "L2_cache_size", None),
            "measured": {"fp32_fma_per_s": rates[0], "int64_mad_per_s": rates[1],
                         "fp64_fma_per_s": rates[2], "sfu_sin_per_s": rates[3]}}


# ------------------------------------------------------------ multi-rank logic
def max_over_ranks(value: float, dist, device=None) -> float:
    """Maximum of a per-rank timing over all ranks (every rank gets the result)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput of weak-scaled replicas: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / seconds_max


# --------------------------------------------------------------- CPU oracle leg
def oracle_sample(insts, budget_s: float = 15.0, max_steps=(400, 40)):
    """Time the FP64 oracle on a bounded number of Strang steps of each instance
    (the same workload, truncated); returns (grid-point steps/s, cores, text)."""
    import oracle
    cores = oracle.max_threads()
    tot_pts, tot_t, parts = 0.0, 0.0, []
    per = budget_s / len(insts)
    for inst, cap in zip(insts, max_steps):
        psi = oracle.uniform_state(inst.shape)
        steps, t_used = 0, 0.0
        chunk = 1
        while steps < cap and t_used < per:
            t0 = time.perf_counter()
            psi = oracle.evolve(inst.f, psi, steps * DT, DT, chunk, oracle.Schedule())
            t_used += time.perf_counter() - t0
            steps += chunk
        g = int(np.prod(inst.shape))
        tot_pts += g * steps
        tot_t += t_used
        parts.append(f"{'x'.join(map(str, inst.shape))} {inst.family}: {steps} steps in {t_used:.1f}s")
    return tot_pts / tot_t, cores, "; ".join(parts)


# -------------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank, dist):
    import torch
    from paper_2303_01471_gb300 import qhd

    t_end = args.profile_T if args.profile_T is not None else T_END
    nsteps = int(round(t_end / DT))
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    qhd.load()
    insts = make_instances(rank)
    sims, f_dev = [], []
    for inst in insts:
        sim = qhd.QHD(inst.shape, batch=1, device=dev)
        sim.set_schedule(qhd.Schedule())
        sims.append(sim)
        f_dev.append(torch.from_numpy(inst.f).to(dev))
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > L2 (126 MB)
    prob = [torch.empty(int(np.prod(i.shape)), dtype=torch.float32, device=dev) for i in insts]
    prob_host = [torch.empty(int(np.prod(i.shape)), dtype=torch.float32).pin_memory() for i in insts]
    pts_per_step = sum(int(np.prod(i.shape)) * nsteps for i in insts)

    def one_step(device_inputs=True):
        obs = []
        for k, sim in enumerate(sims):
            if device_inputs:
                sim.set_potential(f_dev[k])
            else:
                sim.set_potential(insts[k].f)        # host FP64 -> device inside the call
            sim.reset_state()
            sim.evolve(t_end, DT)
            obs.append(sim.observables(0.1, prob=prob[k])[0])
            if not device_inputs:
                prob_host[k].copy_(prob[k], non_blocking=False)
        return obs

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    # ---------------- timed region: device-resident inputs, no per-launch events
    launches0 = sum(s.launch_count() for s in sims)
    step_ms = []
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with Clocks(local_rank) as clk:
        for _ in range(args.steps):
            flush.random_(0, 255)             # evict psi/f of the previous step from L2
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            obs = one_step()
            e1.record()
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
    barrier()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches = sum(s.launch_count() for s in sims) - launches0
    total_ms = max_over_ranks(float(sum(step_ms)), dist, dev)
    # ---------------- one instrumented step after the timed region: CUDA events
    # around every 16th launch of each kernel class give the per-kernel durations
    for sim in sims:
        sim.timing_read(reset=True)
        sim.timing_enable(16)
    flush.random_(0, 255)
    one_step()
    torch.cuda.synchronize()
    timing = [s.timing_read(reset=True) for s in sims]
    for sim in sims:
        sim.timing_enable(0)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(pts_per_step, world, ms_per_step / 1e3)

    # ---------------- e2e: host inputs and host result through the C ABI
    e2e_ms = []
    for _ in range(args.steps):
        flush.random_(0, 255)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        one_step(device_inputs=False)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_step = max_over_ranks(statistics.mean(e2e_ms), dist, dev)
    h2d = sum(8 * int(np.prod(i.shape)) for i in insts)
    d2h = sum(4 * int(np.prod(i.shape)) + 64 for i in insts)

    # ---------------- roofline of the dominant kernel class
    peak, peak_src = peaks()
    kernels = []
    for inst, tm in zip(insts, timing):
        g = int(np.prod(inst.shape))
        for cls, (ms, cnt) in tm.items():
            if cnt == 0:
                continue
            avg_ms = ms / cnt
            bpp = BYTES_PER_POINT.get(cls)
            row = {"instance": "x".join(map(str, inst.shape)), "kernel": cls, "timed_launches": cnt,
                   "avg_us": round(avg_ms * 1e3, 3), "share_est": None}
            if bpp is not None:
                row["bytes_per_launch"] = bpp * g
                row["gbs"] = round(bpp * g / (avg_ms * 1e-3) / 1e9, 1)
            kernels.append(row)
    # share of device time per class, scaling sampled launches to all steps
    est = []
    for row in kernels:
        n_launch = nsteps + (1 if row["kernel"] in ("row", "plane") else 0) if row["kernel"] != "prep" else None
        if n_launch is None:
            n_launch = row["timed_launches"]
        est.append(row["avg_us"] * 1e-3 * n_launch)
    tot = sum(est)
    for row, e in zip(kernels, est):
        row["share_est"] = round(e / tot, 4) if tot > 0 else None
    dom = max((r for r in kernels if "gbs" in r), key=lambda r: r["share_est"] or 0)
    traffic, traffic_note = traffic_entry(dom["kernel"], dom["instance"])
    roofline = {"bound": "hbm", "kernel": f"{dom['kernel']} pass, {dom['instance']}",
                "achieved": dom["gbs"], "peak": peak, "unit": "GB/s",
                "frac": round(dom["gbs"] / peak, 4), "peak_source": peak_src,
                "traffic": traffic,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch; " + traffic_note,
                "algorithmic_bytes_per_launch": dom["bytes_per_launch"],
                "timing": "CUDA events around every 16th launch of each class, in one step run after the timed region"}

    result = {
        "metric": METRIC, "value": value, "unit": "grid-point Strang steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded Rastrigin / Gaussian wells)",
        "instances_per_s": len(insts) * world / (ms_per_step / 1e3),
        "config": {"workload": WORKLOAD, "instances_per_rank": len(insts),
                   "grid_points_x_steps_per_step": pts_per_step, "parallelism": f"replicas x{world}",
                   "l2": "psi+f of the 256^3 instance exceed L2; a 512 MiB write flushes L2 between timed steps"},
        "e2e": {"value": whole_job_rate(pts_per_step, world, e2e_step / 1e3), "unit": "grid-point Strang steps/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_step},
        "gpu_launches": launches,
        "roofline": roofline,
        "kernels": kernels,
        "clocks": clk.summary(),
        "device": device_record(dev),
        "wall_s_timed_region": wall,
        "observables": [{"instance": "x".join(map(str, i.shape)), "norm": o.norm, "e_f": o.e_f,
                         "p_succ": o.p_succ} for i, o in zip(insts, obs)],
    }
    if args.profile_T is not None:
        result["profiling_run"] = f"evolutions shortened to T={t_end}: not a bench value"
    for sim in sims:
        sim.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample = oracle_sample(insts, budget_s=args.cpu_budget)
        result["cpu_baseline"] = {"value": v, "unit": "grid-point Strang steps/s", "cores": cores,
                                  "kind": "oracle", "sample": sample}
    if world == 1 and not args.no_configs and args.profile_T is None:
        # the other configurations, each device-timed with its own parity and roofline
        result["configs"] = {"c1": c1_plain(args, dev, rank), "c3": c3_ragged(args, dev, rank)}
    return result


# ------------------------------------------------------------ Sim-QHD (box mesh)
SIMQHD_WORKLOAD = ("Sim-QHD on 5-d box QPs: 256 seeded instances of 1/2 x^T Q x + b^T x on [0,1]^5 "
                   "(Q symmetric, entries U[-1,1]; b U[-1,1]), finite-difference mesh r=8 (9^5 points), relaxed "
                   "kinetic operator A' of the Hamming encoding, binomial (discrete Gaussian) psi0, "
                   "e^phi=2/(1e-3+t^3), e^chi=2 sigma t^3 with sigma ~ U(0.5,2), T=10, dt=0.01 (1000 Strang steps), "
                   "complex64")


def run_simqhd(args, rank, world, local_rank, dist):
    """One bench step: set F from (Q, b) on the device, binomial psi0, 1000
    Strang steps and the observables of every instance, all in one batched
    context.  Roofline: the dominant pass against the measured rate of 64-bit
    integer multiply-adds (the fixed-point line products)."""
    import torch
    from paper_2303_01471_gb300 import lattice, qhd

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    d, r, B = 5, 8, args.simqhd_count
    T = args.profile_T if args.profile_T is not None else 10.0
    dt = 0.01
    nsteps = int(round(T / dt))
    qps = [workloads.box_qp(100000 * rank + i, d) for i in range(B)]
    Q = np.stack([q for q, _ in qps])
    bvec = np.stack([b for _, b in qps])
    sig = np.random.default_rng(7 + rank).uniform(0.5, 2.0, B)
    lat = lattice.Lattice(d, r, lattice.RELAXED, batch=B, device=dev)
    lat.set_schedule([qhd.Schedule(c_chi=2.0 * s) for s in sig])
    G = lat.grid_points
    pts_per_step = G * B * nsteps
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def one_step():
        lat.set_qp(Q, bvec)
        lat.reset_state(lattice.INIT_GROUND)
        lat.evolve(T, dt)
        return lat.observables(0.1, 0.01)

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    launches0 = lat.launch_count()
    step_ms = []
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with Clocks(local_rank) as clk:
        for _ in range(args.steps):
            flush.random_(0, 255)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            obs = one_step()
            e1.record()
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
    barrier()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches = lat.launch_count() - launches0
    # per-pass durations from one instrumented step after the timed region
    lat.timing_read(reset=True)
    lat.timing_enable(8)
    flush.random_(0, 255)
    one_step()
    torch.cuda.synchronize()
    tm = lat.timing_read(reset=True)
    lat.timing_enable(0)
    ms_per_step = max_over_ranks(float(sum(step_ms)), dist, dev) / args.steps
    value = whole_job_rate(pts_per_step, world, ms_per_step / 1e3)

    # end to end through the public API: Q, b from the host, observables back
    e2e_ms = []
    for _ in range(args.steps):
        flush.random_(0, 255)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        one_step()
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_step = max_over_ranks(statistics.mean(e2e_ms), dist, dev)

    # roofline: the passes are bound by 32x32->64-bit integer multiply-adds.
    # Algorithmic work per point and axis: the reversal-symmetric blocks of the
    # n x n propagator, M^2 + H^2 complex terms per line (M = n - n//2, H = n//2)
    # of three integer MADs each (Gauss's three-product complex multiply).
    n = r + 1
    hh, mm = n // 2, n - n // 2
    mads_pp_axis = 3.0 * (mm * mm + hh * hh) / n
    from paper_2303_01471_gb300 import probe
    ffma_rate, imad_rate, _, _ = probe.alu_rates()
    axes = {"pass0": 3, "pass1": 2}
    kernels, best = [], None
    for cls in ("pass0", "pass1"):
        ms, cnt = tm[cls]
        if cnt == 0:
            continue
        avg_s = ms / cnt / 1e3
        mads = mads_pp_axis * axes[cls] * G * B
        row = {"kernel": cls, "axes": axes[cls], "timed_launches": cnt, "avg_us": round(avg_s * 1e6, 3),
               "tmads": round(mads / avg_s / 1e12, 3),
               "gbs": round((20 if cls == "pass0" else 16) * G * B / avg_s / 1e9, 1),
               "share_est": round(avg_s * nsteps / (ms_per_step / 1e3), 4)}
        kernels.append(row)
        if best is None or row["share_est"] > best["share_est"]:
            best = row
    clk_sum = clk.summary()
    roofline = {"bound": "alu", "kernel": f"{best['kernel']} (U along {best['axes']} axes)",
                "achieved": best["tmads"], "peak": round(imad_rate / 1e12, 3), "unit": "T int64-MAD/s",
                "frac": round(best["tmads"] * 1e12 / imad_rate, 4),
                "peak_source": "measured: qhd_probe_alu_rates (32x32->64-bit multiply-add loop on every SM)",
                "traffic": None, "algorithmic_mads_per_point_per_axis": round(mads_pp_axis, 3),
                "fp32_fma_rate_measured_tfma": round(ffma_rate / 1e12, 2)}
    result = {
        "metric": METRIC, "value": value, "unit": "grid-point Strang steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded box QPs)",
        "instances_per_s": B * world / (ms_per_step / 1e3),
        "config": {"workload": SIMQHD_WORKLOAD, "instances_per_rank": B, "parallelism": f"replicas x{world}",
                   "l2": "psi + fixed-point F of 256 instances (181 MB) exceed L2; a 512 MiB write flushes L2 between timed steps"},
        "e2e": {"value": whole_job_rate(pts_per_step, world, e2e_step / 1e3), "unit": "grid-point Strang steps/s",
                "h2d_bytes_per_step": int(Q.nbytes + bvec.nbytes), "d2h_bytes_per_step": 64 * B,
                "ms_per_step": e2e_step},
        "gpu_launches": launches, "roofline": roofline, "kernels": kernels, "clocks": clk_sum,
        "device": device_record(dev),
        "wall_s_timed_region": wall,
        "observables_first": {"norm": obs[0].norm, "e_f": obs[0].e_f, "p_succ": obs[0].p_succ,
                              "p_gap": obs[0].p_gap},
    }
    if args.profile_T is not None:
        result["profiling_run"] = f"evolutions shortened to T={T}: not a bench value"
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        from oracle import lattice as OL
        F = OL.qp_potential(Q[0], bvec[0], r)
        psi = OL.initial_state(d, r, OL.LATTICE_RELAXED, OL.INIT_KINETIC_GROUND)
        steps_done, t_used = 0, 0.0
        while steps_done < nsteps and t_used < args.cpu_budget:
            k = min(50, nsteps - steps_done)
            t0 = time.perf_counter()
            psi = OL.evolve(F, psi, r, OL.LATTICE_RELAXED, steps_done * dt, dt, k,
                            oracle.Schedule(c_chi=2.0 * sig[0]))
            t_used += time.perf_counter() - t0
            steps_done += k
        result["cpu_baseline"] = {"value": G * steps_done / t_used, "unit": "grid-point Strang steps/s",
                                  "cores": 1, "kind": "oracle",
                                  "sample": f"instance 0, {steps_done} of {nsteps} steps in {t_used:.1f}s (numpy FP64)"}
        if steps_done == nsteps:
            o = OL.observables(F, psi, r)
            prob = torch.empty((B, *lat.shape), dtype=torch.float32, device=dev)
            lat.observables(prob=prob)
            result["parity_instance0"] = {"tv": float(0.5 * np.abs(prob[0].double().cpu().numpy() - o.prob).sum()),
                                          "ef_rel": abs(obs[0].e_f - o.e_f) / max(abs(o.e_f), 1e-3 * np.ptp(F)),
                                          "norm_drift": obs[0].norm - 1.0}
    lat.close()
    return result


# ------------------------------------------------------------- ragged batch
FLOP_PER_POINT_STEP_2D = {n: 2 * 2 * 5 * int(np.log2(n)) + 12 for n in (64, 128, 256)}  # FFTs + phases


def timed_ms(fn, stream, reps):
    """Device time (ms) of fn() on `stream`, CUDA events, one value per repetition."""
    import torch
    out = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def fp32_peak_flops():
    """Measured FP32 FMA rate of this GPU (the probe library), as flop/s."""
    from paper_2303_01471_gb300 import probe
    return 2.0 * probe.alu_rates()[0]


def c1_plain(args, dev, rank):
    """C1: one 128^2 Gaussian-well instance (K=8) at a time, T=10, dt=0.01 (1000
    Strang steps), seeds 0..9: the whole run is one launch of one cluster (8 CTAs:
    a lone instance takes the wide split).
    Device-timed per seed (set f on the device, reset, evolve, observables),
    median reported, parity of each seed against the FP64 oracle."""
    import torch
    import oracle
    from paper_2303_01471_gb300 import qhd
    seeds = list(range(10))
    n, T, dt = 128, 10.0, 0.01
    nsteps = int(round(T / dt))
    insts = [workloads.gaussian_wells(1000 * rank + s, (n, n), K=8) for s in seeds]
    sim = qhd.QHD((n, n), device=dev)
    sim.set_schedule(qhd.Schedule())
    fdev = [torch.from_numpy(i.f).to(dev) for i in insts]
    prob = torch.empty(n * n, dtype=torch.float32, device=dev)
    ms, parity = [], []
    with Clocks(dev.index or 0) as clk:
        for k, inst in enumerate(insts):
            def run():
                sim.set_potential(fdev[k])
                sim.reset_state()
                sim.evolve(T, dt)
            run()  # warm-up
            ms.append(statistics.median(timed_ms(run, sim.stream, 5)))
            obs = sim.observables(0.1, prob=prob)[0]
            po = oracle.evolve(inst.f, oracle.uniform_state((n, n)), 0.0, dt, nsteps, oracle.Schedule())
            ob = oracle.observables(inst.f, po)
            p = prob.double().cpu().numpy().reshape(n, n)
            parity.append({"seed": 1000 * rank + seeds[k], "tv": float(0.5 * np.abs(p - ob.prob).sum()),
                           "ef_rel": abs(obs.e_f - ob.e_f) / max(abs(ob.e_f), 1e-3 * np.ptp(inst.f)),
                           "norm_drift": obs.norm - 1.0})
    sms_used = sim.cluster_ctas()
    sim.close()
    med = statistics.median(ms)
    pts = n * n * nsteps
    flops = pts * FLOP_PER_POINT_STEP_2D[n]
    peak_sms = fp32_peak_flops() * sms_used / torch.cuda.get_device_properties(dev).multi_processor_count
    return {"workload": "128^2 Gaussian wells (K=8), T=10, dt=0.01 (1000 Strang steps), one instance per run, "
                        "seeds 0..9 (median)",
            "metric": "grid-point Strang steps/s", "value": pts / (med / 1e3), "ms_per_run_median": med,
            "ms_per_run": ms, "parity": parity,
            "parity_max": {"tv": max(r["tv"] for r in parity), "ef_rel": max(r["ef_rel"] for r in parity),
                           "norm_drift": max(abs(r["norm_drift"]) for r in parity)},
            "roofline": {"bound": "fp32", "achieved": flops / (med / 1e3) / 1e12,
                         "peak": peak_sms / 1e12, "unit": "TFLOP/s", "frac": flops / (med / 1e3) / peak_sms,
                         "peak_source": f"measured FP32 FMA rate x 2, scaled to the {sms_used} SMs one cluster occupies",
                         "algorithmic_flop_per_point_step": FLOP_PER_POINT_STEP_2D[n]},
            "timing": "CUDA events on the context's stream, median of 5 runs per seed after a warm-up",
            "clocks": clk.summary()}


RAGGED_WORKLOAD = ("Batched QHD: 4096 instances, 2048 x 128^2 + 2048 x 256^2 on [0,1]^2, families alternating "
                   "Gaussian wells (K=8) / Rastrigin type, per-instance sigma ~ U(0.5,2) (e^chi = 2 sigma t^3), "
                   "T=10, dt=0.01 (1000 Strang steps), complex64; one persistent launch (CUDA graph) over both "
                   "size classes, launch configuration from the autotuner")


def c3_ragged(args, dev, rank):
    """C3: every instance of both size classes in one persistent launch per chunk
    (qhd_group_*, replayed as a CUDA graph), configuration picked by the autotuner.
    Baseline: one context per instance, each run a launch sequence of its own,
    device-timed on a sample of each size."""
    import torch
    import oracle
    from paper_2303_01471_gb300 import autotune, qhd
    count = args.ragged_count
    spec = workloads.ragged_batch_spec(count, seed0=100000 * rank)
    classes = {}
    for fam, seed, shape in spec:
        classes.setdefault(shape, []).append((fam, seed))
    T, dt = 10.0, 0.01
    nsteps = int(round(T / dt))
    sims, fdev, sigmas = [], [], []
    for shape, sp in classes.items():
        f, sig = workloads.batch_on_device(sp, shape, dev)
        sim = qhd.QHD(shape, batch=len(sp), device=dev)
        sim.set_schedule([qhd.Schedule(c_chi=2.0 * g) for g in sig])
        sim.set_potential(f)
        sims.append(sim)
        fdev.append(f)
        sigmas.append(sig)
    tune = autotune.tune_group(sims, T=0.2, dt=dt)
    grp = qhd.Group(sims, tune["config"])
    stream = sims[0].stream

    def one_step():
        for sim in sims:
            sim.reset_state()
        grp.evolve(T, dt)

    one_step()
    torch.cuda.synchronize()
    launches0 = grp.info()["launches"]
    with Clocks(dev.index or 0) as clk:
        ms = timed_ms(one_step, stream, max(2, args.steps))
    status = grp.status()
    info = grp.info()
    step_s = statistics.mean(ms) / 1e3
    obs = [sim.observables(0.1) for sim in sims]
    # baseline: one context per instance (prep + whole-run launch per instance)
    per_inst = {}
    for (shape, sp), sig in zip(classes.items(), sigmas):
        nsamp = min(args.ragged_sample, len(sp))
        f1, _ = workloads.batch_on_device(sp[:nsamp], shape, dev)
        one = qhd.QHD(shape, device=dev)
        ts = []
        for i in range(nsamp):
            one.set_schedule(qhd.Schedule(c_chi=2.0 * sig[i]))
            one.set_potential(f1[i])

            def run():
                one.reset_state()
                one.evolve(T, dt)
            run()
            ts.append(statistics.median(timed_ms(run, one.stream, 3)))
        one.close()
        per_inst[shape] = statistics.mean(ts) / 1e3
    single_s = sum(per_inst[sh] * len(sp) for sh, sp in classes.items())
    # parity on two instances of each size against the FP64 oracle
    parity = []
    for ci, ((shape, sp), sig) in enumerate(zip(classes.items(), sigmas)):
        prob = torch.empty(len(sp) * shape[0] * shape[1], dtype=torch.float32, device=dev)
        sims[ci].observables(0.1, prob=prob)
        for i in (0, len(sp) - 1):
            fam, seed = sp[i]
            inst = workloads.make(fam, seed, shape)
            po = oracle.evolve(inst.f, oracle.uniform_state(shape), 0.0, dt, nsteps,
                               oracle.Schedule(c_chi=2.0 * sig[i]))
            ob = oracle.observables(inst.f, po)
            p = prob[i * shape[0] * shape[1]:(i + 1) * shape[0] * shape[1]].double().cpu().numpy().reshape(shape)
            o = obs[ci][i]
            parity.append({"shape": "x".join(map(str, shape)), "seed": seed,
                           "tv": float(0.5 * np.abs(p - ob.prob).sum()),
                           "ef_rel": abs(o.e_f - ob.e_f) / max(abs(ob.e_f), 1e-3 * np.ptp(inst.f)),
                           "norm_drift": o.norm - 1.0})
    grp.close()
    for sim in sims:
        sim.close()
    pts = sum(sh[0] * sh[1] * len(sp) for sh, sp in classes.items()) * nsteps
    flops = sum(sh[0] * sh[1] * len(sp) * FLOP_PER_POINT_STEP_2D[sh[0]] for sh, sp in classes.items()) * nsteps
    peak = fp32_peak_flops()
    cfg = tune["config"].as_dict()
    return {"workload": RAGGED_WORKLOAD, "metric": "instances/s", "value": count / step_s,
            "ms_per_step": step_s * 1e3, "ms_per_step_runs": ms,
            "grid_point_steps_per_s": pts / step_s,
            "one_context_per_instance": {"instances_per_s": count / single_s, "sample_per_size": args.ragged_sample,
                                         "ms_per_instance": {"x".join(map(str, k)): v * 1e3
                                                             for k, v in per_inst.items()}},
            "speedup_vs_one_launch_sequence_per_instance": single_s / step_s,
            "launch": {"kernel_launches_per_step": info["launches"] - launches0, "graph_captures": info["captures"],
                       "persistent_clusters": info["clusters"], "ctas_per_cluster": 8,
                       "config": cfg, "autotuner": {"cached": tune["cached"], "candidates_ms": tune["ms"]},
                       "status": qhd.STATUS.get(status, status)},
            "roofline": {"bound": "fp32", "achieved": flops / step_s / 1e12, "peak": peak / 1e12,
                         "unit": "TFLOP/s", "frac": flops / step_s / peak,
                         "peak_source": "measured FP32 FMA rate x 2 (whole GPU)",
                         "algorithmic_flop_per_point_step": {str(k): v for k, v in FLOP_PER_POINT_STEP_2D.items()}},
            "timing": "CUDA events on the group's stream around reset + group evolve (device time)",
            "parity": parity, "clocks": clk.summary()}


def run_ragged(args, rank, world, local_rank, dist):
    """--workload ragged: C3 as its own bench line."""
    import torch
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    r = c3_ragged(args, dev, rank)
    step_s = max_over_ranks(r["ms_per_step"] / 1e3, dist, dev)
    return {"metric": "instances/s", "value": whole_job_rate(args.ragged_count, world, step_s),
            "unit": "instances/s", "n_gpus": world, "steps": max(2, args.steps), "warmup": 1,
            "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (seeded Rastrigin / Gaussian wells)",
            "config": {"workload": RAGGED_WORKLOAD, "instances_per_rank": args.ragged_count},
            "gpu_launches": r["launch"]["kernel_launches_per_step"], "roofline": r["roofline"],
            "clocks": r["clocks"], "details": r}


# ------------------------------------------------------ tensor-core DFT form
TC_WORKLOAD = ("Split-precision tensor-core DFT: 256 instances of a 2-D 512^2 mesh on [0,1]^2, Gaussian wells "
               "(K=16), T=10, dt=0.01 (1000 Strang steps), paper schedule, complex64 state; per-axis DFTs as "
               "FP16 split-operand GEMMs with FP32 accumulation (3/5 products: block-scaled hi/lo integer slices; "
               "10 products: fixed-point slices)")


def run_tcdft(args, rank, world, local_rank, dist):
    """The batch once with the tensor-core transform (3, 5 or 10 split products) and once
    with the shared-memory FFT passes, on the same device-resident inputs; accuracy
    of both against the FP64 oracle on a sample of the instances."""
    import torch
    import oracle
    from paper_2303_01471_gb300 import qhd

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    qhd.load()
    count, n = args.tc_count, 512
    T, dt = 10.0, 0.01
    nsteps = int(round(T / dt))
    spec = [("wells", 10000 * rank + i) for i in range(count)]
    f_dev, _ = workloads.batch_on_device(spec, (n, n), dev, K=16)
    f_host = f_dev.cpu().numpy()
    pts = count * n * n * nsteps

    def make_sim(transform):
        sim = qhd.QHD((n, n), batch=count, device=dev)
        sim.set_schedule(qhd.Schedule())
        if transform:
            sim.set_transform(qhd.TRANSFORM_TC_DFT, args.tc_products)
        return sim

    prob = torch.empty(count * n * n, dtype=torch.float32, device=dev)
    prob_host = torch.empty(count * n * n, dtype=torch.float32).pin_memory()

    def one_step(sim, device_inputs=True):
        sim.set_potential(f_dev if device_inputs else f_host)
        sim.reset_state()
        sim.evolve(T, dt)
        obs = sim.observables(0.1, prob=prob)
        if not device_inputs:
            prob_host.copy_(prob)
        return obs

    def timed(sim, k, timing=False):
        for _ in range(args.warmup):
            one_step(sim)
        torch.cuda.synchronize()
        l0, g0 = sim.launch_count(), sim.library_call_count()
        ms = []
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        for _ in range(k):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            obs = one_step(sim)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        if dist is not None:
            dist.barrier()
        launches, calls = sim.launch_count() - l0, sim.library_call_count() - g0
        tm = None
        if timing:
            # per-kernel durations from one instrumented step after the timed region
            sim.timing_read(reset=True)
            sim.timing_enable(25)
            one_step(sim)
            torch.cuda.synchronize()
            tm = sim.timing_read(reset=True)
            sim.timing_enable(0)
        return max_over_ranks(sum(ms), dist, dev) / k, launches, calls, tm, obs

    results = {}
    # ---------------- tensor-core transform
    sim = make_sim(True)
    with Clocks(local_rank) as clk:
        ms_tc, launches, gemms, tm, obs_tc = timed(sim, args.steps, timing=True)
    psi_tc = sim.psi[: args.tc_accuracy_sample].cpu().numpy()
    e2e_ms = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        one_step(sim, device_inputs=False)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_step = max_over_ranks(statistics.mean(e2e_ms), dist, dev)
    sim.close()
    # ---------------- FFT passes on the same batch
    sim = make_sim(False)
    ms_fft, _, _, _, obs_fft = timed(sim, args.steps)
    psi_fft = sim.psi[: args.tc_accuracy_sample].cpu().numpy()
    sim.close()

    # ---------------- roofline: the GEMMs against the dense FP16 tensor peak
    m, kp = 2 * n, args.tc_products * 2 * n
    flop_per_gemm = 2.0 * count * n * m * kp
    gemm_ms, gemm_cnt = tm["tc_gemm"]
    split_ms, split_cnt = tm["tc_split"]
    achieved = flop_per_gemm / (gemm_ms / gemm_cnt * 1e-3) / 1e12
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        tpeak, tsrc = float(pk.get("bf16_tflops_sustained", pk["bf16_tflops"])), \
            "measured (cuBLAS bf16 GEMM, sustained; the fp16 dense rate equals bf16)"
    except Exception:
        tpeak, tsrc = 1700.0, "fallback"
    # per point: read the FP32 product (8 B), write the FP16 operand segments
    # (2 x 2 B each; the block-scaled form adds one exponent byte per 16 values),
    # the fixed-point form also reads the product once for its max
    segs = 4 if args.tc_products == 10 else 2
    split_bytes = count * n * n * (8 + 4 * segs + (8 if args.tc_products == 10 else 2 / 16))
    roofline = {"bound": "tensor", "kernel": "tcgen05 FP16 GEMM of one axis transform (qhd_umma_gemm.cu)",
                "achieved": round(achieved, 1), "peak": tpeak, "unit": "TFLOP/s",
                "frac": round(achieved / tpeak, 4), "peak_source": tsrc, "traffic": None,
                "algorithmic_flop_per_launch": flop_per_gemm,
                "flop_per_point_step": 4 * 8 * args.tc_products * n}

    # ---------------- accuracy on a sample against the FP64 oracle
    acc, cpu_t, cpu_pts = [], 0.0, 0
    if not args.no_cpu_baseline:
        oracle.set_threads(oracle.max_threads())
        for i in range(args.tc_accuracy_sample):
            f = f_host[i]
            t0 = time.perf_counter()
            po = oracle.evolve(f, oracle.uniform_state((n, n)), 0.0, dt, nsteps, oracle.Schedule())
            cpu_t += time.perf_counter() - t0
            cpu_pts += n * n * nsteps
            ob = oracle.observables(f, po)
            row = {"instance": i}
            for name, psi, obs in (("tc", psi_tc[i], obs_tc[i]), ("fft", psi_fft[i], obs_fft[i])):
                p = np.abs(psi.astype(np.complex128)) ** 2
                row[name] = {"tv": float(0.5 * np.abs(p - ob.prob).sum()),
                             "ef_rel": abs(obs.e_f - ob.e_f) / max(abs(ob.e_f), 1e-3 * np.ptp(f)),
                             "norm_drift": obs.norm - 1.0}
            acc.append(row)
    res = {
        "metric": METRIC, "value": whole_job_rate(pts, world, ms_tc / 1e3), "unit": "grid-point Strang steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_tc,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16 split / f32 accumulate",
        "data": "synthetic (seeded Gaussian wells)",
        "instances_per_s": count * world / (ms_tc / 1e3),
        "config": {"workload": TC_WORKLOAD, "instances_per_rank": count, "products": args.tc_products,
                   "l2": "psi (512 MiB) and the split operands exceed L2; no flush needed"},
        "fft_path": {"value": whole_job_rate(pts, world, ms_fft / 1e3), "ms_per_step": ms_fft,
                     "instances_per_s": count * world / (ms_fft / 1e3)},
        "tc_over_fft_time": ms_tc / ms_fft,
        "e2e": {"value": whole_job_rate(pts, world, e2e_step / 1e3), "unit": "grid-point Strang steps/s",
                "h2d_bytes_per_step": 8 * count * n * n, "d2h_bytes_per_step": 4 * count * n * n + 64 * count,
                "ms_per_step": e2e_step},
        "gpu_launches": launches, "library_gemm_calls": gemms,
        "roofline": roofline,
        "kernels": {"tc_gemm_avg_us": round(gemm_ms / gemm_cnt * 1e3, 2),
                    "tc_split_avg_us": round(split_ms / split_cnt * 1e3, 2),
                    "tc_split_gbs": round(split_bytes / (split_ms / split_cnt * 1e-3) / 1e9, 1),
                    "gemm_share_est": round(gemm_ms / (gemm_ms + split_ms), 4)},
        "clocks": clk.summary(), "accuracy_vs_oracle": acc,
    }
    if acc and rank == 0 and world == 1:
        res["cpu_baseline"] = {"value": cpu_pts / cpu_t, "unit": "grid-point Strang steps/s",
                               "cores": oracle.max_threads(), "kind": "oracle",
                               "sample": f"{args.tc_accuracy_sample} instances x 1000 steps, 512^2, "
                                         f"{cpu_t:.1f}s"}
    return res


# ------------------------------------------------------------ FNO surrogate
FNO_WORKLOAD = ("Learned surrogate: FNO (4 spectral layers, width 32, 16 modes per axis, projection 128) on a "
                "128^2 mesh, f = Gaussian wells (K=8) / Rastrigin type 50/50 with sigma ~ U(0.5,2); targets "
                "|psi(T)|^2 from the solver (T=10, dt=0.01); BF16 activations, FP32 accumulate; trained on "
                "solver-generated instances, evaluated on held-out seeds >= 10^6; fallback to the solver above "
                "TV 1e-2")


def run_fno(args, rank, world, local_rank, dist):
    """Generate the data with the solver, train the surrogate with its own kernels,
    then time inference and the solver on the held-out set and report the TV
    distribution and the fallback rate."""
    import torch
    from paper_2303_01471_gb300 import fno, qhd, surrogate

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    qhd.load()
    n, ntr, nte = 128, args.fno_train, args.fno_test
    T, dt = 10.0, 0.01

    def spec(seed0, count):
        return [("wells" if i % 2 == 0 else "rastrigin", seed0 + i) for i in range(count)]

    t0 = time.perf_counter()
    f_tr, s_tr = workloads.batch_fast_on_device(spec(10_000_000 * rank, ntr), (n, n), dev, K=8)
    f_te, s_te = workloads.batch_fast_on_device(spec(1_000_000 + 10_000_000 * rank, nte), (n, n), dev, K=8)
    sig_tr = torch.tensor(s_tr, dtype=torch.float32, device=dev)
    sig_te = torch.tensor(s_te, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    t_inputs = time.perf_counter() - t0
    t0 = time.perf_counter()
    p_tr = surrogate.solver_distributions(f_tr, s_tr, T, dt)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0

    cfg = fno.FNOConfig()
    net = fno.FNO(cfg, batch_max=max(args.fno_batch, args.fno_infer_batch), train=True, seed=args.fno_seed)
    k0 = min(512, nte)
    tv_untrained = surrogate.tv_distance(surrogate.predict(net, f_te[:k0], sig_te[:k0], args.fno_infer_batch),
                                         surrogate.solver_distributions(f_te[:k0], s_te[:k0], T, dt))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist, nsteps = surrogate.train(net, f_tr, sig_tr, p_tr, epochs=args.fno_epochs, batch=args.fno_batch,
                                   lr=args.fno_lr, seed=args.fno_seed, time_budget_s=args.fno_train_budget)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del p_tr

    # held-out evaluation: the surrogate's distributions (timed) and the solver's (timed)
    for _ in range(args.warmup):
        surrogate.predict(net, f_te[:args.fno_infer_batch], sig_te[:args.fno_infer_batch], args.fno_infer_batch)
    torch.cuda.synchronize()
    l0 = net.launch_count()
    with Clocks(local_rank) as clk:
        t_inf = []
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            pred = surrogate.predict(net, f_te, sig_te, args.fno_infer_batch)
            e1.record()
            torch.cuda.synchronize()
            t_inf.append(e0.elapsed_time(e1) / 1e3)
    launches = net.launch_count() - l0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    p_te = surrogate.solver_distributions(f_te, s_te, T, dt)
    e1.record()
    torch.cuda.synchronize()
    t_solver = e0.elapsed_time(e1) / 1e3
    tv = surrogate.tv_distance(pred, p_te).cpu().numpy()
    tv_u = surrogate.tv_distance(torch.full_like(p_te[:k0], 1.0 / (n * n)), p_te[:k0]).cpu().numpy()
    net.close()
    inf_s = max_over_ranks(statistics.mean(t_inf), dist, dev)
    inf_rate = nte / inf_s
    solver_rate = nte / t_solver
    fallback = float((tv > 1e-2).mean())
    eff = 1.0 / (1.0 / inf_rate + fallback / solver_rate)
    q = lambda a, x: float(np.quantile(a, x))
    # forward flop per instance: axis-1 stage, axis-0 stages and mode mixing, inverse
    # axis-1 stage with the pointwise part (per layer), projection and lift
    C, M, H, L = cfg.width, cfg.modes, cfg.hidden, cfg.layers
    g = n * n
    mac = L * (g * C * M * 2 + M * (2 * M * C * n * 4 * 2 + 2 * M * C * C * 4) + g * C * (2 * (M - 1) + C)) \
        + g * (H * C + H + 4 * C)
    flop = 2.0 * mac
    # forward bytes per instance, what the kernel sequence must move (BF16 activations
    # of C channels = 2C bytes per point; spectra FP32 complex): lift reads f (8) and
    # writes the features (16) and v0; per layer the axis-1 stage reads v and writes
    # its M-mode spectrum, the axis-0 stage reads it and writes the mixed spectrum
    # and the retained modes, the layer output reads the spectrum and v and writes
    # v (and the pre-activation a, except after the last layer); the projection
    # reads v and writes z, the softmax reads z and writes p
    act, spec = 2 * C, 8 * M * C / n
    vhat = 8 * 2 * M * M * C / g
    per_layer = act + spec + spec + vhat + spec + spec + act + act + act
    bytes_pt = (8 + 16 + act) + L * per_layer - act + (act + 4) + 8
    bytes_inst = bytes_pt * g
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            hpeak, hsrc = float(json.load(fh)["hbm_gbs"]), "measured (STREAM-style copy)"
    except Exception:
        hpeak, hsrc = 6800.0, "fallback"
    achieved = bytes_inst * nte / inf_s / 1e9
    fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    return {
        "metric": "instances/s", "value": inf_rate * world, "unit": "instances/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": inf_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16 activations / f32 accumulate",
        "data": "synthetic (seeded Gaussian wells / Rastrigin; targets from the solver)",
        "config": {"workload": FNO_WORKLOAD, "train_instances": ntr, "heldout_instances": nte,
                   "epochs_run": len(hist), "optimizer_steps": nsteps, "batch": args.fno_batch,
                   "lr": args.fno_lr, "infer_batch": args.fno_infer_batch},
        "solver_instances_per_s": solver_rate * world,
        "surrogate_over_solver_speed": inf_rate / solver_rate,
        "tv_heldout": {"mean": float(tv.mean()), "median": q(tv, 0.5), "p10": q(tv, 0.1), "p90": q(tv, 0.9),
                       "min": float(tv.min()), "max": float(tv.max())},
        "fallback_rate_tv_1e-2": fallback,
        "effective_instances_per_s_with_fallback": eff * world,
        "tv_untrained_mean": float(tv_untrained.mean().item()), "tv_uniform_mean": float(tv_u.mean()),
        "train": {"loss_first_epoch": hist[0] if hist else None, "loss_last_epoch": hist[-1] if hist else None,
                  "seconds": t_train, "instances_per_s": nsteps * args.fno_batch / t_train},
        "data_generation_s": {"inputs": t_inputs, "solver_targets": t_data},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": "FNO forward (all kernels; dense parts on BF16 MMA)",
                     "achieved": round(achieved, 1), "peak": hpeak, "unit": "GB/s",
                     "frac": round(achieved / hpeak, 4), "peak_source": hsrc, "traffic": None,
                     "algorithmic_bytes_per_instance": bytes_inst, "flop_per_instance": flop,
                     "flop_rate_tflops": round(flop * nte / inf_s / 1e12, 2),
                     "fp32_simt_peak_tflops": round(fp32_peak, 1)},
        "clocks": clk.summary(),
    }


# -------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The paper ships no code; the reference arm is the FP64 oracle on the host
    cores, each step a bounded sample of the same workload."""
    if rank != 0:
        return None
    insts = make_instances(0)
    per_step = max(2.0, args.cpu_budget / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_sample(insts, budget_s=per_step, max_steps=(2, 1))
    vals, samples = [], []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, cores, sample = oracle_sample(insts, budget_s=per_step, max_steps=(400, 40))
        vals.append(v)
        samples.append(sample)
    wall = time.perf_counter() - t0
    v = statistics.mean(vals)
    pts_per_step = sum(int(np.prod(i.shape)) * NSTEPS for i in insts)
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "grid-point Strang steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": pts_per_step / v * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Rastrigin / Gaussian wells)",
            "config": {"workload": WORKLOAD, "instances_per_rank": len(insts),
                       "note": "FP64 CPU oracle timed on a bounded prefix of the 10^4 steps"},
            "cpu_baseline": {"value": v, "unit": "grid-point Strang steps/s", "cores": cores,
                             "kind": "oracle", "sample": samples[-1]},
            "e2e": {"value": v, "unit": "grid-point Strang steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s_timed_region": wall}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="default workload only: skip the 128^2 and ragged-batch configurations")
    ap.add_argument("--workload", choices=["scale", "ragged", "tcdft", "fno", "simqhd"], default="scale")
    ap.add_argument("--simqhd-count", type=int, default=256)
    ap.add_argument("--fno-train", type=int, default=50000)
    ap.add_argument("--fno-test", type=int, default=10000)
    ap.add_argument("--fno-epochs", type=int, default=10)
    ap.add_argument("--fno-batch", type=int, default=64)
    ap.add_argument("--fno-infer-batch", type=int, default=512)
    ap.add_argument("--fno-lr", type=float, default=1e-3)
    ap.add_argument("--fno-seed", type=int, default=0)
    ap.add_argument("--fno-train-budget", type=float, default=600.0)
    ap.add_argument("--tc-count", type=int, default=256)
    ap.add_argument("--tc-products", type=int, choices=[3, 5, 10], default=3)
    ap.add_argument("--tc-accuracy-sample", type=int, default=2)
    ap.add_argument("--ragged-count", type=int, default=4096)
    ap.add_argument("--ragged-sample", type=int, default=8)
    ap.add_argument("--profile-T", type=float, default=None,
                    help="shorten each evolution to this simulated time (profiling runs only; "
                         "the printed line is then not a bench value)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if (args.impl == "ours" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local_rank)
        tdist.init_process_group(backend)
        dist = tdist
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    elif args.workload == "ragged":
        res = run_ragged(args, rank, world, local_rank, dist)
    elif args.workload == "tcdft":
        res = run_tcdft(args, rank, world, local_rank, dist)
    elif args.workload == "fno":
        res = run_fno(args, rank, world, local_rank, dist)
    elif args.workload == "simqhd":
        res = run_simqhd(args, rank, world, local_rank, dist)
    else:
        res = run_ours(args, rank, world, local_rank, dist)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
