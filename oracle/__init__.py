"""FP64 CPU oracle for the QHD split-operator simulation -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library
(``paper_2303_01471_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``qhd_oracle.c`` (plain C, FP64, its own recursive
radix-2 FFT).  This module compiles it with gcc and exposes it through ctypes
with numpy arrays.  Every function follows the paper (arXiv 2303.01471):

* ``evolve``      -- Strang form of the pseudo-spectral product formula,
                     Eqs. (prod_qhd), (prod_qhd_fft), Algorithm 1, with the
                     coefficients at step midpoints.
* ``evolve_trotter`` -- the first-order formula exactly as printed in
                     Eq. (prod_qhd) (coefficients at t_j = j s).
* ``observables`` -- |psi|^2, E[f] (Eq. (expect_O)) and the success
                     probability of Fig. 2 (mass within 0.1 of x*).
* ``fft``         -- the oracle's own multi-dimensional DFT.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libqhd_oracle.so")
_SRC = os.path.join(_HERE, "qhd_oracle.c")

SCHED_NESTEROV = 0
SCHED_TABLE = 1
SCHED_POWER = 2


def build_oracle(force: bool = False) -> str:
    """Compile the C oracle into oracle/_lib (gcc, FP64, no FMA contraction)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
            _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        build_oracle()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_evolve.argtypes = [ctypes.c_int, ip, dp, dp, dp, dp,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                      ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, dp, dp, dp, ctypes.c_int64,
                                      ctypes.c_double, ctypes.c_int]
        lib.oracle_evolve.restype = ctypes.c_int
        lib.oracle_evolve_trotter.argtypes = [ctypes.c_int, ip, dp, dp, dp, dp,
                                              ctypes.c_double, ctypes.c_double,
                                              ctypes.c_int64, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_int]
        lib.oracle_evolve_trotter.restype = ctypes.c_int
        lib.oracle_observables.argtypes = [ctypes.c_int, ip, dp, dp, dp, dp,
                                           ctypes.c_double, dp, dp]
        lib.oracle_observables.restype = ctypes.c_int
        lib.oracle_fft.argtypes = [ctypes.c_int, ip, dp, ctypes.c_int]
        lib.oracle_fft.restype = None
        lib.oracle_schedule.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, dp, dp, dp, ctypes.c_int64,
                                        ctypes.c_double, ctypes.c_double, dp, dp]
        lib.oracle_schedule.restype = None
        lib.oracle_apply_h.argtypes = [ctypes.c_int, ip, dp, dp, dp, dp, dp, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int]
        lib.oracle_apply_h.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_threads.restype = None
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


@dataclass
class Schedule:
    """Damping schedule: a(t)=e^{phi_t} weights the kinetic term, b(t)=e^{chi_t}
    the potential (Eq. (qhd_operator)).

    kind=SCHED_NESTEROV: a = c_phi/(eps+t^3), b = c_chi t^3 (Eq. (nonconvex_QHD_h)
    has c_phi=2, eps=s=1e-3, c_chi=2).  kind=SCHED_TABLE: phi(t), chi(t) are
    piecewise linear through the samples (ts increasing), constant beyond.
    kind=SCHED_POWER: a = c_phi/(eps+|t|^{p+1}), b = c_chi |t|^{2p-1}, p = power:
    the three-parameter form (Eq. (qhd_operator_convex)) with the ideal scaling
    condition (Eq. (ideal_scaling)) met with equality, alpha = log p - log t,
    beta = p log t + log C, gamma = p log t (c_phi = p, c_chi = p C, eps = 0).
    """
    kind: int = SCHED_NESTEROV
    c_phi: float = 2.0
    eps: float = 1e-3
    c_chi: float = 2.0
    ts: Optional[np.ndarray] = None
    phis: Optional[np.ndarray] = None
    chis: Optional[np.ndarray] = None
    power: float = 2.0

    def arrays(self):
        if self.kind == SCHED_TABLE:
            ts = np.ascontiguousarray(self.ts, dtype=np.float64)
            ph = np.ascontiguousarray(self.phis, dtype=np.float64)
            ch = np.ascontiguousarray(self.chis, dtype=np.float64)
            return ts, ph, ch, len(ts)
        return None, None, None, 0


def schedule_ab(sched: Schedule, t: float):
    """(a, b) = (e^{phi_t}, e^{chi_t}) as the oracle evaluates them."""
    lib = _load()
    ts, ph, ch, ns = sched.arrays()
    a = ctypes.c_double()
    b = ctypes.c_double()
    lib.oracle_schedule(sched.kind, sched.c_phi, sched.eps, sched.c_chi,
                        _dp(ts), _dp(ph), _dp(ch), ns, float(sched.power), float(t),
                        ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def _grid_args(shape, lo, hi):
    ndim = len(shape)
    n = np.ascontiguousarray(shape, dtype=np.int64)
    lo = np.ascontiguousarray(np.broadcast_to(np.asarray(lo, dtype=np.float64), (ndim,)))
    hi = np.ascontiguousarray(np.broadcast_to(np.asarray(hi, dtype=np.float64), (ndim,)))
    return ndim, n, lo, hi


def uniform_state(shape) -> np.ndarray:
    """psi0 = G^{-1/2}: the uniform superposition over the mesh."""
    g = int(np.prod(shape))
    return np.full(shape, 1.0 / np.sqrt(g), dtype=np.complex128)


KINETIC_SPECTRAL = 0
KINETIC_FD2 = 1


def evolve(f: np.ndarray, psi: np.ndarray, t0: float, dt: float, nsteps: int,
           sched: Schedule = Schedule(), lo=0.0, hi=1.0, kinetic: int = KINETIC_SPECTRAL) -> np.ndarray:
    """Return psi after nsteps Strang steps (complex128, shape of f).  kinetic:
    KINETIC_SPECTRAL (-Lap exact on the mesh's Fourier modes) or KINETIC_FD2 (the
    central second difference of Eq. (discretize-pde) on the periodic mesh)."""
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    ndim, n, lo_, hi_ = _grid_args(f.shape, lo, hi)
    ts, ph, ch, ns = sched.arrays()
    rc = lib.oracle_evolve(ndim, _ip(n), _dp(lo_), _dp(hi_), _dp(f),
                           _dp(out.view(np.float64)), float(t0), float(dt), int(nsteps),
                           sched.kind, sched.c_phi, sched.eps, sched.c_chi,
                           _dp(ts), _dp(ph), _dp(ch), ns, float(sched.power), int(kinetic))
    if rc != 0:
        raise ValueError("oracle_evolve rejected its arguments")
    return out


def evolve_trotter(f, psi, t0, dt, nsteps, c_phi=2.0, eps=1e-3, c_chi=2.0,
                   lo=0.0, hi=1.0, kinetic: int = KINETIC_SPECTRAL) -> np.ndarray:
    """First-order product formula of Eq. (prod_qhd), left-end-point coefficients."""
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    ndim, n, lo_, hi_ = _grid_args(f.shape, lo, hi)
    rc = lib.oracle_evolve_trotter(ndim, _ip(n), _dp(lo_), _dp(hi_), _dp(f),
                                   _dp(out.view(np.float64)), float(t0), float(dt),
                                   int(nsteps), c_phi, eps, c_chi, int(kinetic))
    if rc != 0:
        raise ValueError("oracle_evolve_trotter rejected its arguments")
    return out


@dataclass
class Obs:
    norm: float
    e_f: float
    p_succ: float
    x_star: np.ndarray = field(default_factory=lambda: np.zeros(3))
    prob: Optional[np.ndarray] = None


def observables(f: np.ndarray, psi: np.ndarray, radius: float = 0.1, lo=0.0, hi=1.0,
                want_prob: bool = True) -> Obs:
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    ndim, n, lo_, hi_ = _grid_args(f.shape, lo, hi)
    out = np.zeros(6, dtype=np.float64)
    prob = np.empty(f.shape, dtype=np.float64) if want_prob else None
    rc = lib.oracle_observables(ndim, _ip(n), _dp(lo_), _dp(hi_), _dp(f),
                                _dp(psi.view(np.float64)), float(radius), _dp(out),
                                _dp(prob))
    if rc != 0:
        raise ValueError("oracle_observables rejected its arguments")
    return Obs(norm=out[0], e_f=out[1], p_succ=out[2], x_star=out[3:6].copy(), prob=prob)


def fft(data: np.ndarray, sign: int = -1) -> np.ndarray:
    """The oracle's own DFT over all axes: sign=-1 forward (unnormalised),
    sign=+1 inverse with the 1/G factor."""
    lib = _load()
    out = np.ascontiguousarray(data, dtype=np.complex128).copy()
    n = np.ascontiguousarray(out.shape, dtype=np.int64)
    lib.oracle_fft(out.ndim, _ip(n), _dp(out.view(np.float64)), int(sign))
    return out


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def apply_h(f: np.ndarray, psi: np.ndarray, a: float, b: float, lo=0.0, hi=1.0,
            kinetic: int = KINETIC_SPECTRAL) -> np.ndarray:
    """H psi with H = a (-Lap/2) + b f (Eq. (qhd_operator)) on the mesh, with the
    spectral or the finite-difference kinetic operator."""
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    x = np.ascontiguousarray(psi, dtype=np.complex128).reshape(f.shape)
    out = np.empty_like(x)
    ndim, n, lo_, hi_ = _grid_args(f.shape, lo, hi)
    rc = lib.oracle_apply_h(ndim, _ip(n), _dp(lo_), _dp(hi_), _dp(f), _dp(x.view(np.float64)),
                            _dp(out.view(np.float64)), float(a), float(b), int(kinetic))
    if rc != 0:
        raise ValueError("oracle_apply_h rejected its arguments")
    return out


def lowest_eigs(f: np.ndarray, a: float, b: float, k: int, lo=0.0, hi=1.0,
                kinetic: int = KINETIC_SPECTRAL, return_vectors: bool = False):
    """The k lowest eigenvalues (ascending) of H = a (-Lap/2) + b f, a real symmetric
    operator on the mesh: scipy's Lanczos (ARPACK eigsh) on the oracle's apply_h."""
    import scipy.sparse.linalg as sla
    shape = f.shape
    G = int(np.prod(shape))

    def mv(x):
        return apply_h(f, x.reshape(shape).astype(np.complex128), a, b, lo, hi, kinetic).real.ravel()

    op = sla.LinearOperator((G, G), matvec=mv, dtype=np.float64)
    v0 = np.random.default_rng(0).standard_normal(G)     # fixed start: reproducible runs
    vals, vecs = sla.eigsh(op, k=k, which="SA", tol=1e-12, ncv=max(2 * k + 1, 40), v0=v0)
    order = np.argsort(vals)
    if return_vectors:
        return vals[order], vecs[:, order]
    return vals[order]
