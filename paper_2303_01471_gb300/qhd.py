"""Thin Python binding of the C ABI in include/qhd.h.

Argument marshalling only: every step of the simulation runs in the CUDA
kernels of libqhd.so.  PyTorch provides the device memory (psi and the
workspace) and the stream.  There is no CPU fallback: if the library or a
CUDA device is missing, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build

QHD_OK = 0
QHD_ERR_INVALID_ARG = 1
QHD_ERR_UNSUPPORTED = 2
QHD_ERR_STATE = 3
QHD_ERR_CUDA = 4
QHD_ERR_TIMEOUT = 5
QHD_ERR_WORKSPACE = 6
STATUS = {0: "QHD_OK", 1: "QHD_ERR_INVALID_ARG", 2: "QHD_ERR_UNSUPPORTED", 3: "QHD_ERR_STATE",
          4: "QHD_ERR_CUDA", 5: "QHD_ERR_TIMEOUT", 6: "QHD_ERR_WORKSPACE"}
SCHED_NESTEROV = 0
SCHED_TABLE = 1
SCHED_POWER = 2

# Every entry point declared in include/qhd.h.
EXPORTS = ["qhd_workspace_bytes", "qhd_init_grid", "qhd_set_potential", "qhd_set_potential_device",
           "qhd_set_schedule", "qhd_reset_state", "qhd_set_time", "qhd_get_time", "qhd_evolve",
           "qhd_observables", "qhd_launch_count", "qhd_timing_enable", "qhd_timing_read",
           "qhd_destroy", "qhd_status_string", "qhd_last_error", "qhd_observables_static",
           "qhd_set_splitting", "qhd_evolve_trajectory", "qhd_tc_workspace_bytes", "qhd_set_transform",
           "qhd_library_call_count", "qhd_cluster_ctas", "qhd_set_kinetic", "qhd_spectrum_workspace_bytes",
           "qhd_apply_hamiltonian", "qhd_lowest_eigenpairs", "qhd_fno_param_count", "qhd_fno_workspace_bytes", "qhd_fno_create",
           "qhd_fno_forward", "qhd_fno_loss_grad", "qhd_fno_adam_step", "qhd_fno_launch_count",
           "qhd_fno_last_error", "qhd_fno_destroy", "qhd_lattice_workspace_bytes", "qhd_lattice_init",
           "qhd_lattice_set_potential", "qhd_lattice_set_qp", "qhd_lattice_set_schedule",
           "qhd_lattice_reset_state", "qhd_lattice_get_state", "qhd_lattice_set_state", "qhd_lattice_evolve",
           "qhd_lattice_evolve_trajectory", "qhd_lattice_observables",
           "qhd_lattice_timing_enable", "qhd_lattice_timing_read", "qhd_lattice_launch_count",
           "qhd_lattice_last_error", "qhd_lattice_destroy", "qhd_inject_failure",
           "qhd_group_workspace_bytes", "qhd_group_create", "qhd_group_evolve", "qhd_group_status",
           "qhd_group_inject_wait_timeout", "qhd_group_info", "qhd_group_last_error", "qhd_group_destroy",
           "qhd_tc_gemm_f16", "qhd_tc_gemm_last_error"]
SPLIT_STRANG = 0
SPLIT_LIE_TROTTER = 1
KINETIC_SPECTRAL = 0
KINETIC_FD2 = 1
KCLASS = ["prep", "row", "axis1_fwd", "axis0", "axis1_inv", "oned", "plane", "whole", "tc_split", "tc_gemm"]
TRANSFORM_FFT = 0
TRANSFORM_TC_DFT = 1


class QHDError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Schedule(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("c_phi", ctypes.c_double), ("eps", ctypes.c_double),
                ("c_chi", ctypes.c_double), ("t", ctypes.POINTER(ctypes.c_double)),
                ("phi", ctypes.POINTER(ctypes.c_double)), ("chi", ctypes.POINTER(ctypes.c_double)),
                ("n_samples", ctypes.c_int64), ("power", ctypes.c_double)]


class GroupConfig(ctypes.Structure):
    """Launch choices of a batched group (qhd_group_config): CTAs per instance for
    mesh edge 64 / 128 / 256 (0 = default 2 / 4 / 8), resident CTAs per SM the
    kernel is compiled for (1 or 2, 0 = 2), persistent clusters (0 = all that fit)."""
    _fields_ = [("sub_cluster", ctypes.c_int32 * 3), ("min_blocks", ctypes.c_int32), ("clusters", ctypes.c_int32)]

    @classmethod
    def make(cls, sub=(0, 0, 0), min_blocks=0, clusters=0):
        c = cls()
        for i, v in enumerate(sub):
            c.sub_cluster[i] = int(v)
        c.min_blocks = int(min_blocks)
        c.clusters = int(clusters)
        return c

    def as_dict(self):
        return {"sub": list(self.sub_cluster), "min_blocks": self.min_blocks, "clusters": self.clusters}


class _Obs(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("norm", ctypes.c_double), ("e_f", ctypes.c_double),
                ("p_succ", ctypes.c_double), ("x_star", ctypes.c_double * 3),
                ("steps_done", ctypes.c_int64)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libqhd.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libqhd.so not built ({_build.LIB}); run paper_2303_01471_gb300.build")
    lib = ctypes.CDLL(_build.LIB)
    i64p = ctypes.POINTER(ctypes.c_int64)
    dp = ctypes.POINTER(ctypes.c_double)
    vp = ctypes.c_void_p
    st = ctypes.c_int
    lib.qhd_workspace_bytes.argtypes = [ctypes.c_int, i64p, ctypes.c_int64]
    lib.qhd_workspace_bytes.restype = ctypes.c_size_t
    lib.qhd_init_grid.argtypes = [ctypes.POINTER(vp), ctypes.c_int, i64p, dp, dp, ctypes.c_int64,
                                  vp, vp, ctypes.c_size_t, vp]
    lib.qhd_init_grid.restype = st
    lib.qhd_set_potential.argtypes = [vp, dp]
    lib.qhd_set_potential.restype = st
    lib.qhd_set_potential_device.argtypes = [vp, vp]
    lib.qhd_set_potential_device.restype = st
    lib.qhd_set_schedule.argtypes = [vp, ctypes.POINTER(_Schedule)]
    lib.qhd_set_schedule.restype = st
    lib.qhd_reset_state.argtypes = [vp]
    lib.qhd_reset_state.restype = st
    lib.qhd_set_time.argtypes = [vp, ctypes.c_double]
    lib.qhd_set_time.restype = st
    lib.qhd_get_time.argtypes = [vp, dp, i64p]
    lib.qhd_get_time.restype = st
    lib.qhd_evolve.argtypes = [vp, ctypes.c_double, ctypes.c_double]
    lib.qhd_evolve.restype = st
    lib.qhd_observables.argtypes = [vp, ctypes.POINTER(_Obs), vp, ctypes.c_double]
    lib.qhd_observables.restype = st
    lib.qhd_launch_count.argtypes = [vp]
    lib.qhd_launch_count.restype = ctypes.c_int64
    lib.qhd_timing_enable.argtypes = [vp, ctypes.c_int]
    lib.qhd_timing_enable.restype = st
    lib.qhd_timing_read.argtypes = [vp, dp, i64p, ctypes.c_int]
    lib.qhd_timing_read.restype = st
    lib.qhd_observables_static.argtypes = [ctypes.c_int, i64p, dp, dp, ctypes.c_int64, vp, vp, dp,
                                           ctypes.c_double, vp, vp, vp]
    lib.qhd_observables_static.restype = st
    lib.qhd_evolve_trajectory.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                          ctypes.c_double, vp]
    lib.qhd_evolve_trajectory.restype = st
    lib.qhd_set_splitting.argtypes = [vp, ctypes.c_int]
    lib.qhd_set_splitting.restype = st
    lib.qhd_set_kinetic.argtypes = [vp, ctypes.c_int]
    lib.qhd_set_kinetic.restype = st
    lib.qhd_spectrum_workspace_bytes.argtypes = [vp, ctypes.c_int]
    lib.qhd_spectrum_workspace_bytes.restype = ctypes.c_size_t
    lib.qhd_apply_hamiltonian.argtypes = [vp, ctypes.c_int64, ctypes.c_double, vp, vp]
    lib.qhd_apply_hamiltonian.restype = st
    lib.qhd_lowest_eigenpairs.argtypes = [vp, ctypes.c_int64, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_uint64, vp, ctypes.c_size_t, dp, dp, dp, vp]
    lib.qhd_lowest_eigenpairs.restype = st
    lib.qhd_tc_workspace_bytes.argtypes = [ctypes.c_int, i64p, ctypes.c_int64, ctypes.c_int]
    lib.qhd_tc_workspace_bytes.restype = ctypes.c_size_t
    lib.qhd_set_transform.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_size_t]
    lib.qhd_set_transform.restype = st
    lib.qhd_library_call_count.argtypes = [vp]
    lib.qhd_library_call_count.restype = ctypes.c_int64
    lib.qhd_cluster_ctas.argtypes = [vp]
    lib.qhd_cluster_ctas.restype = ctypes.c_int
    lib.qhd_group_workspace_bytes.argtypes = [ctypes.c_int]
    lib.qhd_group_workspace_bytes.restype = ctypes.c_size_t
    lib.qhd_group_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int,
                                     ctypes.POINTER(GroupConfig), vp, ctypes.c_size_t]
    lib.qhd_group_create.restype = st
    lib.qhd_group_evolve.argtypes = [vp, ctypes.c_double, ctypes.c_double]
    lib.qhd_group_evolve.restype = st
    lib.qhd_group_status.argtypes = [vp]
    lib.qhd_group_status.restype = st
    lib.qhd_group_inject_wait_timeout.argtypes = [vp, ctypes.c_int]
    lib.qhd_group_inject_wait_timeout.restype = st
    lib.qhd_group_info.argtypes = [vp, i64p]
    lib.qhd_group_info.restype = st
    lib.qhd_group_last_error.argtypes = [vp]
    lib.qhd_group_last_error.restype = ctypes.c_char_p
    lib.qhd_group_destroy.argtypes = [vp]
    lib.qhd_group_destroy.restype = st
    lib.qhd_tc_gemm_f16.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.c_int, ctypes.c_float, ctypes.c_float, vp, vp]
    lib.qhd_tc_gemm_f16.restype = st
    lib.qhd_tc_gemm_last_error.argtypes = []
    lib.qhd_tc_gemm_last_error.restype = ctypes.c_char_p
    lib.qhd_inject_failure.argtypes = [vp, ctypes.c_int, ctypes.c_int64]
    lib.qhd_inject_failure.restype = st
    lib.qhd_destroy.argtypes = [vp]
    lib.qhd_destroy.restype = st
    lib.qhd_status_string.argtypes = [st]
    lib.qhd_status_string.restype = ctypes.c_char_p
    lib.qhd_last_error.argtypes = [vp]
    lib.qhd_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


@dataclass
class Schedule:
    """Damping schedule of one instance (see QHD_SCHED_* in include/qhd.h)."""
    kind: int = SCHED_NESTEROV
    c_phi: float = 2.0
    eps: float = 1e-3
    c_chi: float = 2.0
    ts: Optional[np.ndarray] = None
    phis: Optional[np.ndarray] = None
    chis: Optional[np.ndarray] = None
    power: float = 2.0   # SCHED_POWER only


@dataclass
class Observables:
    t: float
    norm: float
    e_f: float
    p_succ: float
    x_star: tuple
    steps_done: int


def schedule_array(sched, batch: int):
    """A ctypes array of `batch` qhd_schedule records from one Schedule (shared)
    or a list of them, plus the numpy arrays its table pointers refer to (keep
    them alive for the call)."""
    scheds: List[Schedule] = list(sched) if isinstance(sched, (list, tuple)) else [sched] * batch
    if len(scheds) != batch:
        raise ValueError("one schedule per instance")
    arr = (_Schedule * batch)()
    keep = []
    for i, s in enumerate(scheds):
        arr[i].kind = s.kind
        arr[i].c_phi = s.c_phi
        arr[i].eps = s.eps
        arr[i].c_chi = s.c_chi
        arr[i].power = s.power
        if s.kind == SCHED_TABLE:
            t = np.ascontiguousarray(s.ts, dtype=np.float64)
            p = np.ascontiguousarray(s.phis, dtype=np.float64)
            c = np.ascontiguousarray(s.chis, dtype=np.float64)
            keep += [t, p, c]
            dp = ctypes.POINTER(ctypes.c_double)
            arr[i].t = t.ctypes.data_as(dp)
            arr[i].phi = p.ctypes.data_as(dp)
            arr[i].chi = c.ctypes.data_as(dp)
            arr[i].n_samples = len(t)
    return arr, keep


def need_tensor(t, dtype, numel: int, what: str) -> None:
    """The library reads raw device pointers: insist on a contiguous CUDA tensor of
    the exact dtype and number of values."""
    if not (t.is_cuda and t.dtype == dtype and t.numel() == numel and t.is_contiguous()):
        raise ValueError(f"{what}: need a contiguous CUDA {dtype} tensor with {numel} values, "
                         f"got {t.dtype} with {t.numel()} on {t.device}")


def workspace_bytes(shape: Sequence[int], batch: int = 1) -> int:
    lib = load()
    n = (ctypes.c_int64 * len(shape))(*shape)
    return int(lib.qhd_workspace_bytes(len(shape), n, int(batch)))


class QHD:
    """One simulation context: a mesh, `batch` instances, psi and workspace on the GPU.

    psi is a torch complex64 tensor of shape (batch, *shape) owned by this
    object (the library only borrows it); the workspace is a uint8 tensor.
    All calls run on `stream` (default: torch's current stream at creation).
    """

    def __init__(self, shape: Sequence[int], lo=0.0, hi=1.0, batch: int = 1, device=None,
                 stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("QHD needs a CUDA device; there is no CPU fallback")
        self.lib = load()
        self.shape = tuple(int(n) for n in shape)
        self.ndim = len(self.shape)
        self.batch = int(batch)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.lo = np.broadcast_to(np.asarray(lo, dtype=np.float64), (self.ndim,)).copy()
        self.hi = np.broadcast_to(np.asarray(hi, dtype=np.float64), (self.ndim,)).copy()
        n = (ctypes.c_int64 * self.ndim)(*self.shape)
        ws = int(self.lib.qhd_workspace_bytes(self.ndim, n, self.batch))
        if ws == 0:
            raise QHDError(1, f"unsupported grid {self.shape} x batch {self.batch}")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.psi = torch.zeros((self.batch, *self.shape), dtype=torch.complex64, device=self.device)
            self._work_raw = torch.empty(ws + 256, dtype=torch.uint8, device=self.device)
        addr = self._work_raw.data_ptr()
        off = (-addr) % 256
        self.work_ptr = addr + off
        self.work_bytes = ws
        ctx = ctypes.c_void_p()
        lo_c = (ctypes.c_double * self.ndim)(*self.lo)
        hi_c = (ctypes.c_double * self.ndim)(*self.hi)
        st = self.lib.qhd_init_grid(ctypes.byref(ctx), self.ndim, n, lo_c, hi_c, self.batch,
                                    ctypes.c_void_p(self.psi.data_ptr()), ctypes.c_void_p(self.work_ptr),
                                    ctypes.c_size_t(ws), ctypes.c_void_p(self.stream.cuda_stream))
        if st != QHD_OK:
            raise QHDError(st, "qhd_init_grid failed")
        self.ctx = ctx

    # -- helpers
    def _check(self, st: int, what: str):
        if st != QHD_OK:
            msg = self.lib.qhd_last_error(self.ctx)
            raise QHDError(st, f"{what}: {msg.decode() if msg else ''}")

    @property
    def grid_points(self) -> int:
        return int(np.prod(self.shape))

    # -- API
    def set_potential(self, f) -> None:
        """f: numpy FP64 host array (batch, *shape) or (*shape) for batch 1, or a
        torch float64 CUDA tensor of the same size (device path)."""
        import torch
        if isinstance(f, torch.Tensor) and f.is_cuda:
            ff = f.contiguous()
            if ff.dtype != torch.float64 or ff.numel() != self.batch * self.grid_points:
                raise ValueError("device f must be float64 with batch*G values")
            self._check(self.lib.qhd_set_potential_device(self.ctx, ctypes.c_void_p(ff.data_ptr())),
                        "qhd_set_potential_device")
            return
        arr = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
        if arr.size != self.batch * self.grid_points:
            raise ValueError(f"f has {arr.size} values, expected {self.batch * self.grid_points}")
        self._check(self.lib.qhd_set_potential(self.ctx, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                    "qhd_set_potential")

    def set_schedule(self, sched) -> None:
        arr, keep = schedule_array(sched, self.batch)
        self._check(self.lib.qhd_set_schedule(self.ctx, arr), "qhd_set_schedule")

    def reset_state(self) -> None:
        self._check(self.lib.qhd_reset_state(self.ctx), "qhd_reset_state")

    def set_splitting(self, kind: int) -> None:
        """SPLIT_STRANG (default) or SPLIT_LIE_TROTTER (Eq. (prod_qhd) as printed)."""
        self._check(self.lib.qhd_set_splitting(self.ctx, int(kind)), "qhd_set_splitting")

    def set_transform(self, kind: int, products: int = 3) -> None:
        """TRANSFORM_FFT (default) or TRANSFORM_TC_DFT (dense DFT GEMMs on the tensor
        cores on FP16 operands: `products` = 3 or 5 block-scaled hi/lo slice
        products, or 10 fixed-point slice products); the tensor-core workspace is allocated
        here and kept with this object."""
        import torch
        if kind == TRANSFORM_FFT:
            self._check(self.lib.qhd_set_transform(self.ctx, 0, 0, None, 0), "qhd_set_transform")
            self._tc_raw = None
            return
        n = (ctypes.c_int64 * self.ndim)(*self.shape)
        ws = int(self.lib.qhd_tc_workspace_bytes(self.ndim, n, self.batch, int(products)))
        if ws == 0:
            raise QHDError(2, f"tensor-core transform unsupported for {self.shape} x {self.batch}, "
                              f"products={products}")
        with torch.cuda.device(self.device):
            raw = torch.empty(ws + 256, dtype=torch.uint8, device=self.device)
        addr = raw.data_ptr()
        ptr = addr + (-addr) % 256
        self._check(self.lib.qhd_set_transform(self.ctx, int(kind), int(products), ctypes.c_void_p(ptr),
                                               ctypes.c_size_t(ws)), "qhd_set_transform")
        self._tc_raw = raw

    def library_call_count(self) -> int:
        return int(self.lib.qhd_library_call_count(self.ctx))

    def cluster_ctas(self) -> int:
        """CTAs per instance (2-D) or per plane (3-D) of the cluster engine, 0 if unused."""
        return int(self.lib.qhd_cluster_ctas(self.ctx))

    def set_kinetic(self, kind: int) -> None:
        """KINETIC_SPECTRAL (default) or KINETIC_FD2 (central second difference of
        Eq. (discretize-pde) on the periodic mesh)."""
        self._check(self.lib.qhd_set_kinetic(self.ctx, int(kind)), "qhd_set_kinetic")

    def apply_hamiltonian(self, x, t: float, inst: int = 0):
        """H(t) x for instance `inst` (x: complex64 CUDA tensor with the mesh's G values)."""
        import torch
        x = x.contiguous()
        need_tensor(x, torch.complex64, self.grid_points, "x")
        out = torch.empty_like(x)
        self._check(self.lib.qhd_apply_hamiltonian(self.ctx, int(inst), float(t), ctypes.c_void_p(x.data_ptr()),
                                                   ctypes.c_void_p(out.data_ptr())), "qhd_apply_hamiltonian")
        return out

    def lowest_eigenpairs(self, t: float, k: int, m: int = 400, inst: int = 0, seed: int = 1, vectors: bool = False):
        """The k lowest eigenvalues of H(t) (Lanczos, m steps) with residuals and the
        probability spectrum |<n|psi>|^2 of the current state; returns numpy arrays
        (eigvals, residuals, overlaps) and, with vectors=True, a (k, *shape) tensor."""
        import torch
        ws = int(self.lib.qhd_spectrum_workspace_bytes(self.ctx, int(m)))
        if ws == 0:
            raise QHDError(1, f"bad Lanczos size m={m}")
        work = torch.empty(ws + 256, dtype=torch.uint8, device=self.device)
        ptr = work.data_ptr() + (-work.data_ptr()) % 256
        ev = np.zeros(k)
        rs = np.zeros(k)
        ov = np.zeros(k)
        vecs = torch.empty((k, *self.shape), dtype=torch.complex64, device=self.device) if vectors else None
        dp = ctypes.POINTER(ctypes.c_double)
        self._check(self.lib.qhd_lowest_eigenpairs(
            self.ctx, int(inst), float(t), int(m), int(k), int(seed), ctypes.c_void_p(ptr), ctypes.c_size_t(ws),
            ev.ctypes.data_as(dp), rs.ctypes.data_as(dp), ov.ctypes.data_as(dp),
            ctypes.c_void_p(vecs.data_ptr()) if vectors else None), "qhd_lowest_eigenpairs")
        return (ev, rs, ov, vecs) if vectors else (ev, rs, ov)

    def set_time(self, t: float) -> None:
        self._check(self.lib.qhd_set_time(self.ctx, float(t)), "qhd_set_time")

    def time(self):
        t = ctypes.c_double()
        s = ctypes.c_int64()
        self._check(self.lib.qhd_get_time(self.ctx, ctypes.byref(t), ctypes.byref(s)), "qhd_get_time")
        return t.value, s.value

    def evolve(self, T: float, dt: float) -> None:
        self._check(self.lib.qhd_evolve(self.ctx, float(T), float(dt)), "qhd_evolve")

    def evolve_trajectory(self, T: float, dt: float, every: int, radius: float = 0.1):
        """Evolve and record (norm, E[f], P_succ) every `every` steps; returns a torch
        float64 CUDA tensor of shape (n/every, batch, 3)."""
        import torch
        n = int(round(T / dt))
        if every < 1 or n % every:
            raise ValueError("every must divide the number of steps")
        traj = torch.empty((n // every, self.batch, 3), dtype=torch.float64, device=self.device)
        self._check(self.lib.qhd_evolve_trajectory(self.ctx, float(T), float(dt), int(every), float(radius),
                                                   ctypes.c_void_p(traj.data_ptr())), "qhd_evolve_trajectory")
        return traj

    def observables(self, radius: float = 0.1, prob=None) -> List[Observables]:
        """prob: optional torch float32 CUDA tensor with batch*G values receiving |psi|^2."""
        import torch
        out = (_Obs * self.batch)()
        if prob is not None:
            need_tensor(prob, torch.float32, self.batch * self.grid_points, "prob")
        pp = ctypes.c_void_p(prob.data_ptr()) if prob is not None else ctypes.c_void_p()
        self._check(self.lib.qhd_observables(self.ctx, out, pp, float(radius)), "qhd_observables")
        return [Observables(o.t, o.norm, o.e_f, o.p_succ, tuple(o.x_star), o.steps_done) for o in out]

    def launch_count(self) -> int:
        return int(self.lib.qhd_launch_count(self.ctx))

    def timing_enable(self, every: int) -> None:
        self._check(self.lib.qhd_timing_enable(self.ctx, int(every)), "qhd_timing_enable")

    def timing_read(self, reset: bool = True) -> dict:
        """{class: (device ms summed, timed launches)} for the sampled launches."""
        n = len(KCLASS)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        self._check(self.lib.qhd_timing_read(self.ctx, ms, cnt, 1 if reset else 0), "qhd_timing_read")
        return {KCLASS[k]: (ms[k], cnt[k]) for k in range(n)}

    def close(self) -> None:
        if getattr(self, "ctx", None):
            self.lib.qhd_destroy(self.ctx)
            self.ctx = None
        self._tc_raw = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """One persistent launch over every instance of several 2-D contexts
    (qhd_group_*): `sims` are QHD objects on one stream, each 2-D with a square
    mesh of edge 64, 128 or 256 and a potential and schedule loaded.  evolve(T, dt)
    advances all of them; the launch is a CUDA graph replayed while T, dt and the
    contexts' clocks repeat."""

    def __init__(self, sims, config: "GroupConfig" = None):
        import torch
        self.lib = load()
        self.sims = list(sims)
        n = len(self.sims)
        ws = int(self.lib.qhd_group_workspace_bytes(n))
        if ws == 0:
            raise QHDError(1, f"a group holds 1..8 contexts, got {n}")
        dev = self.sims[0].device
        self._work_raw = torch.empty(ws + 256, dtype=torch.uint8, device=dev)
        addr = self._work_raw.data_ptr()
        ptr = addr + (-addr) % 256
        arr = (ctypes.c_void_p * n)(*[s.ctx.value for s in self.sims])
        self.config = config if config is not None else GroupConfig.make()
        g = ctypes.c_void_p()
        st = self.lib.qhd_group_create(ctypes.byref(g), arr, n, ctypes.byref(self.config), ctypes.c_void_p(ptr),
                                       ctypes.c_size_t(ws))
        if st != QHD_OK:
            raise QHDError(st, "qhd_group_create failed")
        self.g = g

    def _check(self, st, what):
        if st != QHD_OK:
            msg = self.lib.qhd_group_last_error(self.g)
            raise QHDError(st, f"{what}: {msg.decode() if msg else ''}")

    def evolve(self, T: float, dt: float) -> None:
        self._check(self.lib.qhd_group_evolve(self.g, float(T), float(dt)), "qhd_group_evolve")

    def status(self) -> int:
        """Synchronise; QHD_OK, or QHD_ERR_TIMEOUT when a bounded wait gave up (raises nothing)."""
        return int(self.lib.qhd_group_status(self.g))

    def inject_wait_timeout(self, on: bool = True) -> None:
        self._check(self.lib.qhd_group_inject_wait_timeout(self.g, 1 if on else 0), "inject")

    def info(self) -> dict:
        out = (ctypes.c_int64 * 8)()
        self._check(self.lib.qhd_group_info(self.g, out), "qhd_group_info")
        return {"clusters": out[0], "min_blocks": out[1], "smem_per_cta": out[2], "launches": out[3],
                "captures": out[4], "sub": {64: out[5], 128: out[6], 256: out[7]}}

    def close(self) -> None:
        if getattr(self, "g", None):
            self.lib.qhd_group_destroy(self.g)
            self.g = None
        self._work_raw = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tc_gemm_f16(A, B, C=None, every_mma=True, alpha=1.0, beta=0.0, err=None):
    """C = alpha * A . B^T + beta * C on the tensor cores (qhd_tc_gemm_f16).  A
    (rows, k) and B (n, k) float16 CUDA tensors, C float32 (rows, n); every_mma:
    False (one accumulation), True (per-MMA partials) or "float" (per-MMA
    partials with the expected-truncation correction).  Returns (C, err) with err
    a 2-word int32 tensor (err[0] = 1: a bounded wait gave up)."""
    import torch
    lib = load()
    rows, k = A.shape
    n = B.shape[0]
    need_tensor(A, torch.float16, rows * k, "A")
    need_tensor(B, torch.float16, n * k, "B")
    if C is None:
        C = torch.zeros((rows, n), dtype=torch.float32, device=A.device)
    need_tensor(C, torch.float32, rows * n, "C")
    if err is None:
        err = torch.zeros(2, dtype=torch.int32, device=A.device)
    stream = torch.cuda.current_stream(A.device).cuda_stream
    st = lib.qhd_tc_gemm_f16(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                             ctypes.c_void_p(C.data_ptr()), n, rows, n, k,
                             2 if every_mma == "float" else (1 if every_mma else 0),
                             float(alpha), float(beta), ctypes.c_void_p(err.data_ptr()), ctypes.c_void_p(stream))
    if st != QHD_OK:
        raise QHDError(st, "qhd_tc_gemm_f16: " + lib.qhd_tc_gemm_last_error().decode())
    return C, err
