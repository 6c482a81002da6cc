"""Thin Python binding of the FNO surrogate entry points of include/qhd.h.

Argument marshalling only: forward, loss/gradient and Adam run in the CUDA
kernels of libqhd.so; PyTorch provides the device memory (parameters,
gradients, workspace) and the stream.  No CPU fallback.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import qhd as _qhd


class _Cfg(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("width", ctypes.c_int32), ("modes", ctypes.c_int32),
                ("layers", ctypes.c_int32), ("hidden", ctypes.c_int32), ("act_bf16", ctypes.c_int32)]


@dataclass(frozen=True)
class FNOConfig:
    n: int = 128
    width: int = 32
    modes: int = 16
    layers: int = 4
    hidden: int = 128
    act_bf16: bool = True

    def c(self) -> _Cfg:
        return _Cfg(self.n, self.width, self.modes, self.layers, self.hidden, 1 if self.act_bf16 else 0)


_bound = False


def _lib():
    global _bound
    lib = _qhd.load()
    if not _bound:
        vp = ctypes.c_void_p
        cp = ctypes.POINTER(_Cfg)
        st = ctypes.c_int
        lib.qhd_fno_param_count.argtypes = [cp]
        lib.qhd_fno_param_count.restype = ctypes.c_int64
        lib.qhd_fno_workspace_bytes.argtypes = [cp, ctypes.c_int64, ctypes.c_int]
        lib.qhd_fno_workspace_bytes.restype = ctypes.c_size_t
        lib.qhd_fno_create.argtypes = [ctypes.POINTER(vp), cp, ctypes.c_int64, ctypes.c_int, vp, vp,
                                       ctypes.c_size_t, vp]
        lib.qhd_fno_create.restype = st
        lib.qhd_fno_forward.argtypes = [vp, vp, vp, ctypes.c_int64, vp]
        lib.qhd_fno_forward.restype = st
        lib.qhd_fno_loss_grad.argtypes = [vp, vp, vp, vp, ctypes.c_int64, vp, ctypes.POINTER(ctypes.c_double)]
        lib.qhd_fno_loss_grad.restype = st
        lib.qhd_fno_adam_step.argtypes = [vp, vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                          ctypes.c_int64]
        lib.qhd_fno_adam_step.restype = st
        lib.qhd_fno_launch_count.argtypes = [vp]
        lib.qhd_fno_launch_count.restype = ctypes.c_int64
        lib.qhd_fno_last_error.argtypes = [vp]
        lib.qhd_fno_last_error.restype = ctypes.c_char_p
        lib.qhd_fno_destroy.argtypes = [vp]
        lib.qhd_fno_destroy.restype = st
        _bound = True
    return lib


def param_count(cfg: FNOConfig) -> int:
    c = cfg.c()
    return int(_lib().qhd_fno_param_count(ctypes.byref(c)))


def param_layout(cfg: FNOConfig) -> dict:
    """Offsets (in FP32 values) and sizes of every parameter block, as documented
    in include/qhd.h (each block starts at an even offset)."""
    C, M, H = cfg.width, cfg.modes, cfg.hidden
    off, out = 0, {}

    def take(name, k):
        nonlocal off
        out[name] = (off, k)
        off += (k + 1) & ~1

    take("lift_w", 4 * C)
    take("lift_b", C)
    for l in range(cfg.layers):
        take(f"R{l}", 2 * M * M * C * C * 2)
        take(f"W{l}", C * C)
        take(f"b{l}", C)
    take("p1_w", H * C)
    take("p1_b", H)
    take("p2_w", H)
    take("p2_b", 1)
    out["_total"] = (off, 0)
    return out


def init_params(cfg: FNOConfig, seed: int) -> np.ndarray:
    """Seeded initial weights (FP32): uniform(+-1/sqrt(fan_in)) for the dense
    layers, (re, im) ~ U(0, 1) / width^2 for the spectral weights, zero biases."""
    rng = np.random.default_rng(seed)
    lay = param_layout(cfg)
    w = np.zeros(lay["_total"][0], dtype=np.float32)
    C, H = cfg.width, cfg.hidden

    def put(name, vals):
        o, k = lay[name]
        w[o:o + k] = vals.astype(np.float32).ravel()

    put("lift_w", rng.uniform(-0.5, 0.5, 4 * C))
    for l in range(cfg.layers):
        put(f"R{l}", rng.uniform(0.0, 1.0, lay[f"R{l}"][1]) / (C * C))
        put(f"W{l}", rng.uniform(-1, 1, C * C) / np.sqrt(C))
    put("p1_w", rng.uniform(-1, 1, H * C) / np.sqrt(C))
    put("p2_w", rng.uniform(-1, 1, H) / np.sqrt(H))
    return w


class FNO:
    """An FNO surrogate bound to device parameters (a torch float32 tensor)."""

    def __init__(self, cfg: FNOConfig, batch_max: int, train: bool = False, params=None, seed: int = 0,
                 device=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the FNO surrogate needs a CUDA device; there is no CPU fallback")
        self.lib = _lib()
        self.cfg = cfg
        self.batch_max = int(batch_max)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        c = cfg.c()
        npar = int(self.lib.qhd_fno_param_count(ctypes.byref(c)))
        ws = int(self.lib.qhd_fno_workspace_bytes(ctypes.byref(c), self.batch_max, 1 if train else 0))
        if npar == 0 or ws == 0:
            raise _qhd.QHDError(1, f"unsupported FNO configuration {cfg} x {batch_max}")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            if params is None:
                params = torch.from_numpy(init_params(cfg, seed))
            self.params = params.to(self.device, torch.float32).contiguous().clone()
            if self.params.numel() != npar:
                raise ValueError(f"parameter vector has {self.params.numel()} values, expected {npar}")
            self.grad = torch.zeros(npar, dtype=torch.float32, device=self.device) if train else None
            self._work = torch.empty(ws + 256, dtype=torch.uint8, device=self.device)
        addr = self._work.data_ptr()
        ptr = addr + (-addr) % 256
        h = ctypes.c_void_p()
        st = self.lib.qhd_fno_create(ctypes.byref(h), ctypes.byref(c), self.batch_max, 1 if train else 0,
                                     ctypes.c_void_p(self.params.data_ptr()), ctypes.c_void_p(ptr),
                                     ctypes.c_size_t(ws), ctypes.c_void_p(self.stream.cuda_stream))
        if st != 0:
            raise _qhd.QHDError(st, "qhd_fno_create failed")
        self.h = h
        self.step = 0

    def _check(self, st, what):
        if st != 0:
            msg = self.lib.qhd_fno_last_error(self.h)
            raise _qhd.QHDError(st, f"{what}: {msg.decode() if msg else ''}")

    @staticmethod
    def _need(t, dtype, shape, what):
        """The kernels read raw device pointers: insist on the exact dtype, shape and layout."""
        if not (t.is_cuda and t.dtype == dtype and tuple(t.shape) == tuple(shape) and t.is_contiguous()):
            raise ValueError(f"{what}: need a contiguous CUDA {dtype} tensor of shape {tuple(shape)}, "
                             f"got {t.dtype} {tuple(t.shape)} on {t.device}")

    def forward(self, f, sigma, out=None):
        """f: torch float64 CUDA (B, n, n); sigma: torch float32 CUDA (B,).  Returns p (B, n, n)."""
        import torch
        B, n = f.shape[0], self.cfg.n
        self._need(f, torch.float64, (B, n, n), "f")
        self._need(sigma, torch.float32, (B,), "sigma")
        if out is None:
            out = torch.empty((B, n, n), dtype=torch.float32, device=self.device)
        self._need(out, torch.float32, (B, n, n), "out")
        self._check(self.lib.qhd_fno_forward(self.h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(sigma.data_ptr()),
                                             B, ctypes.c_void_p(out.data_ptr())), "qhd_fno_forward")
        return out

    def loss_grad(self, f, sigma, p_true, want_loss=True):
        """Overwrites self.grad with dL/dparams; returns the mean KL loss (synchronises) or None."""
        import torch
        B, n = f.shape[0], self.cfg.n
        self._need(f, torch.float64, (B, n, n), "f")
        self._need(sigma, torch.float32, (B,), "sigma")
        self._need(p_true, torch.float32, (B, n, n), "p_true")
        if self.grad is None:
            raise _qhd.QHDError(3, "qhd_fno_loss_grad: created without training buffers")
        loss = ctypes.c_double()
        self._check(self.lib.qhd_fno_loss_grad(self.h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(sigma.data_ptr()),
                                               ctypes.c_void_p(p_true.data_ptr()), f.shape[0],
                                               ctypes.c_void_p(self.grad.data_ptr()),
                                               ctypes.byref(loss) if want_loss else None), "qhd_fno_loss_grad")
        return loss.value if want_loss else None

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step += 1
        self._check(self.lib.qhd_fno_adam_step(self.h, ctypes.c_void_p(self.grad.data_ptr()), lr, beta1, beta2, eps,
                                               self.step), "qhd_fno_adam_step")

    def launch_count(self) -> int:
        return int(self.lib.qhd_fno_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.qhd_fno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
