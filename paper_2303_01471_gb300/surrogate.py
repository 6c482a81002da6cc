"""Training and evaluation driver of the FNO surrogate (argument marshalling
and loops only: the solver, the network's forward/backward and Adam run in
libqhd.so's kernels).

The solver produces the training targets: |psi(T)|^2 of each instance under
the paper's schedule with its own potential weight sigma (e^chi = 2 sigma t^3),
computed by batched contexts of the split-operator path.  The surrogate then
predicts that distribution directly from f and sigma; the solver is the measure
of its error (TV against the solver's |psi(T)|^2) and the fallback for
instances above the accepted TV.
"""
from __future__ import annotations

import math
import time
from typing import List, Optional

from . import qhd
from .fno import FNO


def solver_distributions(f, sigmas: List[float], T: float = 10.0, dt: float = 0.01, chunk: int = 4096,
                         stream=None):
    """|psi(T)|^2 of every instance (FP32, same shape as f) from the split-operator
    solver, in batched contexts of at most `chunk` instances."""
    import torch
    B, shape = f.shape[0], tuple(f.shape[1:])
    out = torch.empty((B,) + shape, dtype=torch.float32, device=f.device)
    sim = None
    for i0 in range(0, B, chunk):
        i1 = min(B, i0 + chunk)
        if sim is None or sim.batch != i1 - i0:
            if sim is not None:
                sim.close()
            sim = qhd.QHD(shape, batch=i1 - i0, device=f.device, stream=stream)
        sim.set_potential(f[i0:i1].contiguous())
        sim.set_schedule([qhd.Schedule(c_chi=2.0 * s) for s in sigmas[i0:i1]])
        sim.reset_state()
        sim.evolve(T, dt)
        sim.observables(0.1, prob=out[i0:i1])
    if sim is not None:
        sim.close()
    return out


def tv_distance(p, q):
    """1/2 sum |p - q| per instance (FP64 accumulation), a torch vector."""
    return 0.5 * (p.double() - q.double()).abs().flatten(1).sum(1)


def train(net: FNO, f, sigma, p_true, epochs: int, batch: int, lr: float = 1e-3, lr_final: Optional[float] = None,
          seed: int = 0, log=None, time_budget_s: Optional[float] = None):
    """Adam over shuffled mini-batches with a cosine decay from lr to lr_final.
    Returns the last-batch loss of every epoch and the optimiser steps taken."""
    import torch
    B = f.shape[0]
    nb = B // batch
    total = max(1, epochs * nb)
    lr_final = lr * 0.05 if lr_final is None else lr_final
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    hist, step = [], 0
    t0 = time.perf_counter()
    for ep in range(epochs):
        perm = torch.randperm(B, generator=g).to(f.device)
        for k in range(nb):
            idx = perm[k * batch:(k + 1) * batch]
            fb, sb, pb = f[idx].contiguous(), sigma[idx].contiguous(), p_true[idx].contiguous()
            want = k == nb - 1
            loss = net.loss_grad(fb, sb, pb, want_loss=want)
            a = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * step / total))
            net.adam(lr=a)
            step += 1
            if want:
                hist.append(loss)
        if log:
            log(f"epoch {ep}: last-batch loss {hist[-1]:.4f}, {time.perf_counter() - t0:.1f}s")
        if time_budget_s is not None and time.perf_counter() - t0 > time_budget_s:
            break
    return hist, step


def predict(net: FNO, f, sigma, batch: int):
    import torch
    out = torch.empty(f.shape, dtype=torch.float32, device=f.device)
    for i0 in range(0, f.shape[0], batch):
        i1 = min(f.shape[0], i0 + batch)
        net.forward(f[i0:i1].contiguous(), sigma[i0:i1].contiguous(), out=out[i0:i1])
    return out
