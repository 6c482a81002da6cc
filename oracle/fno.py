"""FP64 CPU reference of the FNO surrogate network -- TEST INFRASTRUCTURE.

Only ``tests/`` and the CPU legs of ``bench.py`` may import this module.  It
shares no code with the CUDA kernels: the network is written here from its
definition with explicit DFT matrices and numpy contractions, slow and
obviously correct, and serves as the reference for the GPU forward pass and (by
central finite differences) of the GPU gradients.

Network (per instance; the paper has no surrogate, this is the definition the
library documents for it):
  q        = ((f - mean f) / std f, sigma, x0, x1)              population std, mesh coords j/n
  v0       = Wl q + bl
  a_l      = SC_l(v_l) + W_l v_l + b_l,  v_{l+1} = gelu(a_l)     (no gelu after the last layer)
  SC(v)(x) = n^-2 sum_{kx in Kx, ky < M} c_ky Re( R(kx,ky)^T V(kx,ky) e^{+2 pi i (kx x0 + ky x1)/n} )
             V(kx,ky) = sum_x v(x) e^{-2 pi i (kx x0 + ky x1)/n},  Kx = {0..M-1} U {n-M..n-1},
             c_0 = 1, c_ky = 2 (the real-input half spectrum), R(kx,ky)[i][o] complex
  z        = Wp2 gelu(Wp1 v_L + bp1) + bp2,   p = softmax over the mesh of z
  loss     = mean over the batch of KL(p_true || p)
gelu(a) = a/2 (1 + erf(a / sqrt 2)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

try:
    from scipy.special import erf as _erf
except Exception:  # pragma: no cover - scipy is present on both machines
    _erf = np.vectorize(math.erf)


@dataclass(frozen=True)
class Shape:
    n: int
    width: int
    modes: int
    layers: int
    hidden: int


def unpack(params: np.ndarray, s: Shape) -> dict:
    """Split the flat parameter vector into named FP64 arrays.  Layout: lift W[C][4],
    b[C]; per layer R[2M][M][C][C] complex as (re, im) pairs, W[C][C], b[C]; then
    Wp1[H][C], bp1[H], Wp2[H], bp2; every block starts at an even offset."""
    p = np.asarray(params, dtype=np.float64)
    C, M, H = s.width, s.modes, s.hidden
    out, off = {}, 0

    def take(k):
        nonlocal off
        blk = p[off:off + k]
        off += k + (k & 1)
        return blk

    out["lift_w"] = take(4 * C).reshape(C, 4)
    out["lift_b"] = take(C)
    for l in range(s.layers):
        r = take(2 * M * M * C * C * 2).reshape(2 * M, M, C, C, 2)
        out[f"R{l}"] = r[..., 0] + 1j * r[..., 1]
        out[f"W{l}"] = take(C * C).reshape(C, C)
        out[f"b{l}"] = take(C)
    out["p1_w"] = take(H * C).reshape(H, C)
    out["p1_b"] = take(H)
    out["p2_w"] = take(H)
    out["p2_b"] = take(1)[0]
    assert off == len(p), (off, len(p))
    return out


def gelu(a):
    return 0.5 * a * (1.0 + _erf(a / math.sqrt(2.0)))


def features(f: np.ndarray, sigma: np.ndarray) -> np.ndarray:
    """(B, n, n) FP64 objective values and (B,) sigma -> (B, n, n, 4)."""
    B, n, _ = f.shape
    mean = f.mean(axis=(1, 2), keepdims=True)
    std = np.sqrt((f * f).mean(axis=(1, 2), keepdims=True) - mean ** 2)
    q = np.empty((B, n, n, 4))
    q[..., 0] = (f - mean) / std
    q[..., 1] = np.asarray(sigma, dtype=np.float64)[:, None, None]
    grid = np.arange(n) / n
    q[..., 2] = grid[None, :, None]
    q[..., 3] = grid[None, None, :]
    return q


def retained_kx(n: int, M: int) -> np.ndarray:
    return np.concatenate([np.arange(M), np.arange(n - M, n)])


def spectral_conv(v: np.ndarray, R: np.ndarray, M: int) -> np.ndarray:
    """v (B, n, n, C) real, R (2M, M, C, C) complex -> (B, n, n, C) real, by the
    definition with explicit DFT matrices."""
    n = v.shape[1]
    kx = retained_kx(n, M)
    ky = np.arange(M)
    x = np.arange(n)
    Ex = np.exp(-2j * np.pi * np.outer(kx, x) / n)   # (2M, n)
    Ey = np.exp(-2j * np.pi * np.outer(ky, x) / n)   # (M, n)
    V = np.einsum("qx,ky,bxyc->bqkc", Ex, Ey, v)     # (B, 2M, M, C)
    W = np.einsum("qkio,bqki->bqko", R, V)
    c = np.where(ky == 0, 1.0, 2.0)
    U = np.einsum("qx,ky,bqko->bxyo", np.conj(Ex), np.conj(Ey), W * c[None, None, :, None])
    return U.real / (n * n)


def forward(params: np.ndarray, s: Shape, f: np.ndarray, sigma: np.ndarray):
    """Returns (p, z) for f (B, n, n) FP64 and sigma (B,)."""
    w = unpack(params, s)
    q = features(f, sigma)
    v = q @ w["lift_w"].T + w["lift_b"]
    for l in range(s.layers):
        a = spectral_conv(v, w[f"R{l}"], s.modes) + v @ w[f"W{l}"].T + w[f"b{l}"]
        v = gelu(a) if l + 1 < s.layers else a
    h = gelu(v @ w["p1_w"].T + w["p1_b"])
    z = h @ w["p2_w"] + w["p2_b"]                   # (B, n, n)
    zz = z.reshape(z.shape[0], -1)
    zz = zz - zz.max(axis=1, keepdims=True)
    e = np.exp(zz)
    p = (e / e.sum(axis=1, keepdims=True)).reshape(z.shape)
    return p, z


def kl_loss(p_true: np.ndarray, p: np.ndarray) -> float:
    """Mean over instances of sum p_true (log p_true - log p) (0 log 0 = 0)."""
    pt = p_true.reshape(p_true.shape[0], -1)
    pp = p.reshape(p.shape[0], -1)
    m = pt > 0
    terms = np.zeros_like(pt)
    terms[m] = pt[m] * (np.log(pt[m]) - np.log(pp[m]))
    return float(terms.sum(axis=1).mean())


def loss(params, s: Shape, f, sigma, p_true) -> float:
    p, _ = forward(params, s, f, sigma)
    return kl_loss(p_true, p)


def fd_gradient(params, s: Shape, f, sigma, p_true, idx, h=1e-6):
    """Central finite differences of the loss at the parameter indices idx."""
    base = np.asarray(params, dtype=np.float64).copy()
    g = np.empty(len(idx))
    for k, i in enumerate(idx):
        old = base[i]
        base[i] = old + h
        lp = loss(base, s, f, sigma, p_true)
        base[i] = old - h
        lm = loss(base, s, f, sigma, p_true)
        base[i] = old
        g[k] = (lp - lm) / (2 * h)
    return g
