"""Seeded synthetic QHD instances -- input data shared by the oracle and the GPU path.

This module holds no arithmetic of the simulation method: it only draws the
random problem parameters and samples the objective f on the mesh
x_j = lo + j (hi - lo) / N (the regular periodic mesh of the paper's
"Spatial discretization" paragraph).  Both the CPU oracle and the CUDA path
receive the same FP64 array f.

The paper's 22 two-dimensional test functions (Sec. "Test problems") are not
reproduced; two synthetic families of the same shape stand in for them:

* Gaussian wells: f(x) = 0.5 |x - 0.5|^2 - sum_k D_k exp(-|x - c_k|^2 / (2 w_k^2)),
  c_k ~ U[0,1]^d, w_k ~ U(0.05, 0.2), D_k ~ U(0.5, 2).
* Rastrigin type: f(x) = sum_i [A (x_i - s_i)^2 - B cos(2 pi omega (x_i - s_i))],
  s ~ U[0.2, 0.8]^d, A=10, B=1, omega=5.

Random draws use numpy.random.default_rng(seed) (PCG64) in a fixed order:
wells -> centres (K, d), widths (K), depths (K), then sigma; Rastrigin ->
s (d), then sigma.  sigma ~ U(0.5, 2) scales the potential weight of the
schedule for batched instances; it is 1 where a workload says so.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Sequence, Tuple

import numpy as np


@dataclass
class Instance:
    family: str
    seed: int
    shape: Tuple[int, ...]
    lo: float
    hi: float
    f: np.ndarray          # FP64, row-major, last axis fastest
    sigma: float           # potential-weight scale of the schedule
    params: dict


def mesh_axes(shape: Sequence[int], lo: float = 0.0, hi: float = 1.0):
    """Coordinates of the periodic mesh along each axis: lo + j (hi-lo)/N."""
    return [lo + np.arange(n, dtype=np.float64) * ((hi - lo) / n) for n in shape]


def _sq_dist_chunks(shape, lo, hi, center):
    axes = mesh_axes(shape, lo, hi)
    d2 = np.zeros(shape, dtype=np.float64)
    for ax, (xs, c) in enumerate(zip(axes, center)):
        sh = [1] * len(shape)
        sh[ax] = len(xs)
        d2 = d2 + ((xs - c) ** 2).reshape(sh)
    return d2


def gaussian_wells(seed: int, shape: Sequence[int], K: int = 8, lo: float = 0.0,
                   hi: float = 1.0, draw_sigma: bool = False) -> Instance:
    shape = tuple(int(n) for n in shape)
    d = len(shape)
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, 1.0, size=(K, d))
    widths = rng.uniform(0.05, 0.2, size=K)
    depths = rng.uniform(0.5, 2.0, size=K)
    sigma = float(rng.uniform(0.5, 2.0)) if draw_sigma else 1.0
    f = 0.5 * _sq_dist_chunks(shape, lo, hi, [0.5] * d)
    for k in range(K):
        d2 = _sq_dist_chunks(shape, lo, hi, centres[k])
        f -= depths[k] * np.exp(-d2 / (2.0 * widths[k] ** 2))
    return Instance("wells", seed, shape, lo, hi, np.ascontiguousarray(f), sigma,
                    {"K": K, "centres": centres, "widths": widths, "depths": depths})


def rastrigin(seed: int, shape: Sequence[int], A: float = 10.0, B: float = 1.0,
              omega: float = 5.0, lo: float = 0.0, hi: float = 1.0,
              draw_sigma: bool = False) -> Instance:
    shape = tuple(int(n) for n in shape)
    d = len(shape)
    rng = np.random.default_rng(seed)
    s = rng.uniform(0.2, 0.8, size=d)
    sigma = float(rng.uniform(0.5, 2.0)) if draw_sigma else 1.0
    axes = mesh_axes(shape, lo, hi)
    f = np.zeros(shape, dtype=np.float64)
    for ax, xs in enumerate(axes):
        u = xs - s[ax]
        term = A * u * u - B * np.cos(2.0 * np.pi * omega * u)
        sh = [1] * d
        sh[ax] = len(xs)
        f = f + term.reshape(sh)
    return Instance("rastrigin", seed, shape, lo, hi, np.ascontiguousarray(f), sigma,
                    {"A": A, "B": B, "omega": omega, "s": s})


def ragged_batch_spec(count: int = 4096, seed0: int = 0):
    """Instance list of the ragged batch: half 128^2, half 256^2, families
    alternating wells (K=8) / Rastrigin, sigma ~ U(0.5, 2), seeds seed0.."""
    spec = []
    for i in range(count):
        n = 128 if i < count // 2 else 256
        fam = "wells" if i % 2 == 0 else "rastrigin"
        spec.append((fam, seed0 + i, (n, n)))
    return spec


def batch_on_device(spec, shape, device, K: int = 8, lo: float = 0.0, hi: float = 1.0):
    """FP64 objective values of many same-shape instances, evaluated on a torch
    device with the same seeded draws and formulas as gaussian_wells / rastrigin.
    spec: list of (family, seed).  Returns (f of shape (B, *shape), sigmas)."""
    import torch
    shape = tuple(int(n) for n in shape)
    d = len(shape)
    axes = [torch.as_tensor(a, dtype=torch.float64, device=device) for a in mesh_axes(shape, lo, hi)]
    grids = torch.meshgrid(*axes, indexing="ij")
    out = torch.empty((len(spec),) + shape, dtype=torch.float64, device=device)
    sig = []
    for i, (fam, seed) in enumerate(spec):
        rng = np.random.default_rng(seed)
        if fam == "wells":
            centres = rng.uniform(0.0, 1.0, size=(K, d))
            widths = rng.uniform(0.05, 0.2, size=K)
            depths = rng.uniform(0.5, 2.0, size=K)
            sig.append(float(rng.uniform(0.5, 2.0)))
            f = 0.5 * sum((g - 0.5) ** 2 for g in grids)
            for k in range(K):
                d2 = sum((g - centres[k, ax]) ** 2 for ax, g in enumerate(grids))
                f = f - depths[k] * torch.exp(-d2 / (2.0 * widths[k] ** 2))
        else:
            s = rng.uniform(0.2, 0.8, size=d)
            sig.append(float(rng.uniform(0.5, 2.0)))
            f = 0.0
            for ax, g in enumerate(grids):
                u = g - s[ax]
                f = f + (10.0 * u * u - 1.0 * torch.cos(2.0 * np.pi * 5.0 * u))
        out[i] = f
    return out, sig


def batch_fast_on_device(spec, shape, device, K: int = 8, lo: float = 0.0, hi: float = 1.0, chunk: int = 512):
    """Same draws and formulas as batch_on_device (sigma drawn for every instance),
    evaluated for many instances at once: parameters are drawn per seed on the
    host, then each chunk of instances is evaluated with one batched expression.
    spec: list of (family, seed).  Returns (f (B, *shape) float64, sigmas list)."""
    import torch
    shape = tuple(int(n) for n in shape)
    d = len(shape)
    B = len(spec)
    cen = np.zeros((B, K, d))
    wid = np.ones((B, K))
    dep = np.zeros((B, K))
    sft = np.zeros((B, d))
    sig = np.zeros(B)
    is_w = np.zeros(B, dtype=bool)
    for i, (fam, seed) in enumerate(spec):
        rng = np.random.default_rng(seed)
        if fam == "wells":
            is_w[i] = True
            cen[i] = rng.uniform(0.0, 1.0, size=(K, d))
            wid[i] = rng.uniform(0.05, 0.2, size=K)
            dep[i] = rng.uniform(0.5, 2.0, size=K)
        else:
            sft[i] = rng.uniform(0.2, 0.8, size=d)
        sig[i] = rng.uniform(0.5, 2.0)
    axes = [torch.as_tensor(a, dtype=torch.float64, device=device) for a in mesh_axes(shape, lo, hi)]
    grids = torch.meshgrid(*axes, indexing="ij")
    out = torch.empty((B,) + shape, dtype=torch.float64, device=device)
    tc = torch.as_tensor(cen, device=device)
    tw = torch.as_tensor(wid, device=device)
    td = torch.as_tensor(dep, device=device)
    ts = torch.as_tensor(sft, device=device)
    view = (-1,) + (1,) * d
    quad = 0.5 * sum((g - 0.5) ** 2 for g in grids)
    for i0 in range(0, B, chunk):
        i1 = min(B, i0 + chunk)
        fw = quad.unsqueeze(0).expand((i1 - i0,) + shape).clone()
        for k in range(K):
            d2 = sum((g.unsqueeze(0) - tc[i0:i1, k, ax].reshape(view)) ** 2 for ax, g in enumerate(grids))
            fw = fw - td[i0:i1, k].reshape(view) * torch.exp(-d2 / (2.0 * tw[i0:i1, k].reshape(view) ** 2))
        fr = 0.0
        for ax, g in enumerate(grids):
            u = g.unsqueeze(0) - ts[i0:i1, ax].reshape(view)
            fr = fr + (10.0 * u * u - 1.0 * torch.cos(2.0 * np.pi * 5.0 * u))
        mask = torch.as_tensor(is_w[i0:i1], device=device).reshape(view)
        out[i0:i1] = torch.where(mask, fw, fr)
    return out, [float(x) for x in sig]


def make(family: str, seed: int, shape, **kw) -> Instance:
    if family == "wells":
        return gaussian_wells(seed, shape, **kw)
    if family == "rastrigin":
        return rastrigin(seed, shape, **kw)
    raise ValueError(f"unknown family {family!r}")


def box_qp(seed: int, d: int = 5):
    """A seeded synthetic box-constrained QP, minimise 1/2 x^T Q x + b^T x over
    [0,1]^d, standing in for the paper's QP benchmark instances (which are not
    in this repository): Q symmetric with upper-triangle entries ~ U[-1, 1]
    (indefinite in general, so the problem is non-convex), b ~ U[-1, 1]^d.
    Draw order: the upper triangle of Q row by row, then b.  Returns (Q, b)."""
    rng = np.random.default_rng(seed)
    Q = np.zeros((d, d))
    iu = np.triu_indices(d)
    Q[iu] = rng.uniform(-1.0, 1.0, len(iu[0]))
    Q = Q + np.triu(Q, 1).T
    b = rng.uniform(-1.0, 1.0, d)
    return Q, b
