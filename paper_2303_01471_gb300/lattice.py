"""Binding of the box-mesh QHD entry points (qhd_lattice_* in include/qhd.h).

Argument marshalling only: evolution, potential assembly and observables run
in libqhd.so's kernels.  PyTorch provides psi, the workspace and the stream.
There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import qhd

CHAIN = 0
RELAXED = 1
INIT_UNIFORM = 0
INIT_GROUND = 1
KCLASS = ["prep", "pass0", "pass1"]


class _LatObs(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("norm", ctypes.c_double), ("e_f", ctypes.c_double),
                ("p_succ", ctypes.c_double), ("p_gap", ctypes.c_double), ("f_min", ctypes.c_double),
                ("argmin", ctypes.c_int64), ("steps_done", ctypes.c_int64)]


@dataclass
class LatticeObservables:
    t: float
    norm: float
    e_f: float
    p_succ: float
    p_gap: float
    f_min: float
    argmin: int
    steps_done: int
    marginals: Optional[np.ndarray] = None


_ready = False


def _lib():
    global _ready
    lib = qhd.load()
    if _ready:
        return lib
    vp, st = ctypes.c_void_p, ctypes.c_int
    dp = ctypes.POINTER(ctypes.c_double)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.qhd_lattice_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64]
    lib.qhd_lattice_workspace_bytes.restype = ctypes.c_size_t
    lib.qhd_lattice_init.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                     vp, vp, ctypes.c_size_t, vp]
    lib.qhd_lattice_init.restype = st
    lib.qhd_lattice_set_potential.argtypes = [vp, vp]
    lib.qhd_lattice_set_potential.restype = st
    lib.qhd_lattice_set_qp.argtypes = [vp, dp, dp]
    lib.qhd_lattice_set_qp.restype = st
    lib.qhd_lattice_set_schedule.argtypes = [vp, ctypes.POINTER(qhd._Schedule)]
    lib.qhd_lattice_set_schedule.restype = st
    lib.qhd_lattice_reset_state.argtypes = [vp, ctypes.c_int]
    lib.qhd_lattice_reset_state.restype = st
    lib.qhd_lattice_get_state.argtypes = [vp, vp]
    lib.qhd_lattice_get_state.restype = st
    lib.qhd_lattice_set_state.argtypes = [vp, vp]
    lib.qhd_lattice_set_state.restype = st
    lib.qhd_lattice_evolve.argtypes = [vp, ctypes.c_double, ctypes.c_double]
    lib.qhd_lattice_evolve.restype = st
    lib.qhd_lattice_evolve_trajectory.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                                  ctypes.c_double, ctypes.c_double, vp]
    lib.qhd_lattice_evolve_trajectory.restype = st
    lib.qhd_lattice_observables.argtypes = [vp, ctypes.POINTER(_LatObs), vp, dp, ctypes.c_double, ctypes.c_double]
    lib.qhd_lattice_observables.restype = st
    lib.qhd_lattice_timing_enable.argtypes = [vp, ctypes.c_int]
    lib.qhd_lattice_timing_enable.restype = st
    lib.qhd_lattice_timing_read.argtypes = [vp, dp, i64p, ctypes.c_int]
    lib.qhd_lattice_timing_read.restype = st
    lib.qhd_lattice_launch_count.argtypes = [vp]
    lib.qhd_lattice_launch_count.restype = ctypes.c_int64
    lib.qhd_lattice_last_error.argtypes = [vp]
    lib.qhd_lattice_last_error.restype = ctypes.c_char_p
    lib.qhd_lattice_destroy.argtypes = [vp]
    lib.qhd_lattice_destroy.restype = st
    _ready = True
    return lib


def workspace_bytes(ndim: int, r: int, batch: int = 1) -> int:
    return int(_lib().qhd_lattice_workspace_bytes(int(ndim), int(r), int(batch)))


class Lattice:
    """`batch` instances of QHD on the mesh {0, 1/r, ..., 1}^ndim with the chain
    (CHAIN) or relaxed (RELAXED) kinetic operator.  The working state `psi_fx`
    (torch int32, shape (batch, r+1, ..., r+1, 2): re, im in units of 2^-29) is
    owned here and borrowed by the library; state() / set_state() convert."""

    def __init__(self, ndim: int, r: int, kind: int = RELAXED, batch: int = 1, device=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Lattice needs a CUDA device; there is no CPU fallback")
        self.lib = _lib()
        self.ndim, self.r, self.kind, self.batch = int(ndim), int(r), int(kind), int(batch)
        self.n = self.r + 1
        self.shape = (self.n,) * self.ndim
        ws = workspace_bytes(self.ndim, self.r, self.batch)
        if ws == 0:
            raise qhd.QHDError(1, f"unsupported lattice d={ndim} r={r} batch={batch}")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.psi_fx = torch.zeros((self.batch, *self.shape, 2), dtype=torch.int32, device=self.device)
            self._work_raw = torch.empty(ws + 256, dtype=torch.uint8, device=self.device)
        addr = self._work_raw.data_ptr()
        self.work_ptr = addr + (-addr) % 256
        h = ctypes.c_void_p()
        st = self.lib.qhd_lattice_init(ctypes.byref(h), self.ndim, self.r, self.kind, self.batch,
                                       ctypes.c_void_p(self.psi_fx.data_ptr()), ctypes.c_void_p(self.work_ptr),
                                       ctypes.c_size_t(ws), ctypes.c_void_p(self.stream.cuda_stream))
        if st != qhd.QHD_OK:
            raise qhd.QHDError(st, "qhd_lattice_init failed")
        self.h = h

    def _check(self, st: int, what: str):
        if st != qhd.QHD_OK:
            msg = self.lib.qhd_lattice_last_error(self.h)
            raise qhd.QHDError(st, f"{what}: {msg.decode() if msg else ''}")

    @property
    def grid_points(self) -> int:
        return self.n ** self.ndim

    def set_potential(self, f) -> None:
        """f: torch float64 CUDA tensor with batch * (r+1)^ndim values."""
        import torch
        ff = f.contiguous()
        if not ff.is_cuda or ff.dtype != torch.float64 or ff.numel() != self.batch * self.grid_points:
            raise ValueError("f must be a float64 CUDA tensor with batch*G values")
        self._check(self.lib.qhd_lattice_set_potential(self.h, ctypes.c_void_p(ff.data_ptr())),
                    "qhd_lattice_set_potential")

    def set_qp(self, Q, b) -> None:
        """F(x) = 1/2 x^T Q x + b^T x on the mesh; Q (batch, d, d), b (batch, d)."""
        Qa = np.ascontiguousarray(np.asarray(Q, dtype=np.float64).reshape(self.batch, self.ndim, self.ndim))
        ba = np.ascontiguousarray(np.asarray(b, dtype=np.float64).reshape(self.batch, self.ndim))
        dp = ctypes.POINTER(ctypes.c_double)
        self._check(self.lib.qhd_lattice_set_qp(self.h, Qa.ctypes.data_as(dp), ba.ctypes.data_as(dp)),
                    "qhd_lattice_set_qp")

    def set_schedule(self, sched) -> None:
        arr, keep = qhd.schedule_array(sched, self.batch)
        self._check(self.lib.qhd_lattice_set_schedule(self.h, arr), "qhd_lattice_set_schedule")

    def reset_state(self, init: int = INIT_GROUND) -> None:
        self._check(self.lib.qhd_lattice_reset_state(self.h, int(init)), "qhd_lattice_reset_state")

    def state(self):
        """The state as a new complex64 tensor (batch, r+1, ..., r+1)."""
        import torch
        out = torch.empty((self.batch, *self.shape), dtype=torch.complex64, device=self.device)
        self._check(self.lib.qhd_lattice_get_state(self.h, ctypes.c_void_p(out.data_ptr())), "qhd_lattice_get_state")
        return out

    def set_state(self, psi) -> None:
        """Load a complex64 CUDA tensor with batch * (r+1)^ndim values."""
        import torch
        z = psi.to(torch.complex64).contiguous()
        if not z.is_cuda or z.numel() != self.batch * self.grid_points:
            raise ValueError("psi must be a CUDA tensor with batch*G values")
        self._check(self.lib.qhd_lattice_set_state(self.h, ctypes.c_void_p(z.data_ptr())), "qhd_lattice_set_state")

    def evolve(self, T: float, dt: float) -> None:
        self._check(self.lib.qhd_lattice_evolve(self.h, float(T), float(dt)), "qhd_lattice_evolve")

    def evolve_trajectory(self, T: float, dt: float, every: int, radius: float = 0.1, gap: float = 0.01):
        """Evolve like evolve() and return a (T/dt/every, batch, 4) float64 CUDA tensor of
        (norm, E[F], p_succ, p_gap) after every `every` steps."""
        import torch
        n = int(round(T / dt))
        out = torch.empty((max(1, n // max(1, int(every))), self.batch, 4), dtype=torch.float64, device=self.device)
        self._check(self.lib.qhd_lattice_evolve_trajectory(self.h, float(T), float(dt), int(every), float(radius),
                                                           float(gap), ctypes.c_void_p(out.data_ptr())),
                    "qhd_lattice_evolve_trajectory")
        return out

    def observables(self, radius: float = 0.1, gap: float = 0.01, prob=None, marginals: bool = False):
        import torch
        out = (_LatObs * self.batch)()
        if prob is not None:
            qhd.need_tensor(prob, torch.float32, self.batch * self.grid_points, "prob")
        marg = np.zeros((self.batch, self.ndim, self.n)) if marginals else None
        mp = marg.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if marginals else None
        pp = ctypes.c_void_p(prob.data_ptr()) if prob is not None else None
        self._check(self.lib.qhd_lattice_observables(self.h, out, pp, mp, float(radius), float(gap)),
                    "qhd_lattice_observables")
        return [LatticeObservables(o.t, o.norm, o.e_f, o.p_succ, o.p_gap, o.f_min, o.argmin, o.steps_done,
                                   marg[i] if marginals else None) for i, o in enumerate(out)]

    def timing_enable(self, every: int) -> None:
        self._check(self.lib.qhd_lattice_timing_enable(self.h, int(every)), "qhd_lattice_timing_enable")

    def timing_read(self, reset: bool = True):
        ms = (ctypes.c_double * 3)()
        cnt = (ctypes.c_int64 * 3)()
        self._check(self.lib.qhd_lattice_timing_read(self.h, ms, cnt, int(reset)), "qhd_lattice_timing_read")
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KCLASS)}

    def launch_count(self) -> int:
        return int(self.lib.qhd_lattice_launch_count(self.h))

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.qhd_lattice_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
