"""FP64 CPU oracle of QHD on the finite-difference box mesh -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this module.  The product library never imports it and shares no
code with it.

The discretisation is the one of the paper's section on finite-difference
discretisation of PDEs and on the relaxed implementation for quadratic
programming: r cells per edge of the unit box, mesh points x_j = j / r
(j = 0..r, so n = r + 1 points per axis), and the semi-discrete equation

    i d/dt phi = [ e^{phi_t} sum_k K_k + e^{chi_t} F ] phi,     K = -(r^2 / 2) A,

with A either the adjacency matrix of the chain graph (Eq. (discretize-pde)
and the remark after it: the central second difference with the vanishing
boundary condition, its -2I diagonal dropped as a global phase) or the relaxed
matrix A' of Eq. (relaxed_adjacency), and F the potential sampled on the mesh
(Eq. (finite-quadratic-obj) for a quadratic objective).  Readings where the
text is garbled:

* A' has the entries sqrt((j + 1)(r - j) / r), j = 0..r-1: the Hamming-weight
  block of S_x / sqrt(r) on r qubits, which is what the Hamming-encoding table
  maps -A'/2 to (the printed (r + 1) would belong to r + 1 qubits).
* The r^2 = 1/h^2 of Eq. (discretize-pde) stays in the kinetic term (the
  Ising-machine dictionary, A(t)/h = lambda r^{3/2} e^{phi_t}, carries it).
* The initial "discrete Gaussian" state has the amplitudes
  sqrt(binom(r, j) / 2^r) per axis (normalised; the image of |+>^r).

Time stepping is the Strang form of the product formula used on the Fourier
mesh (Eq. (prod_qhd) with a, b at the step midpoints, half potential phases
not merged).  The kinetic factor separates over the axes because the axis
terms commute, so it is applied as the per-axis matrix exponential
expm(i dt a (r^2 / 2) A) (scipy's Pade scaling-and-squaring).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np
import scipy.linalg

from . import Schedule, schedule_ab

LATTICE_CHAIN = 0
LATTICE_RELAXED = 1

INIT_UNIFORM = 0
INIT_KINETIC_GROUND = 1


def mesh(r: int) -> np.ndarray:
    """Mesh coordinates j / r, j = 0..r, of one axis."""
    return np.arange(r + 1, dtype=np.float64) / r


def adjacency(r: int, kind: int) -> np.ndarray:
    """The per-axis (r+1) x (r+1) off-diagonal operator: the chain adjacency
    (remark after Eq. (discretize-pde)) or the relaxed A' (Eq. (relaxed_adjacency),
    read as sqrt((j+1)(r-j)/r))."""
    n = r + 1
    A = np.zeros((n, n))
    for j in range(r):
        w = 1.0 if kind == LATTICE_CHAIN else np.sqrt((j + 1) * (r - j) / r)
        A[j, j + 1] = w
        A[j + 1, j] = w
    return A


def kinetic_matrix(r: int, kind: int) -> np.ndarray:
    """K = -(r^2 / 2) A: the per-axis kinetic operator at e^{phi} = 1."""
    return -0.5 * r * r * adjacency(r, kind)


def axis_propagator(r: int, kind: int, theta: float) -> np.ndarray:
    """exp(-i theta K) for one axis (theta = dt * e^{phi})."""
    return scipy.linalg.expm(-1j * theta * kinetic_matrix(r, kind))


def qp_potential(Q: np.ndarray, b: np.ndarray, r: int) -> np.ndarray:
    """F(x) = 1/2 x^T Q x + b^T x on the mesh {0, 1/r, ..., 1}^d
    (Eq. (finite-quadratic-obj)); row-major, last axis fastest."""
    d = len(b)
    axes = np.meshgrid(*([mesh(r)] * d), indexing="ij")
    X = np.stack([a.ravel() for a in axes], axis=1)          # (G, d)
    f = 0.5 * np.einsum("gi,ij,gj->g", X, np.asarray(Q, dtype=np.float64), X) + X @ np.asarray(b, np.float64)
    return f.reshape((r + 1,) * d)


def axis_ground(r: int, kind: int) -> np.ndarray:
    """Ground state of -A (top eigenvector of A) in closed form: the binomial
    amplitudes sqrt(binom(r, j) / 2^r) for A' (the Hamming-encoding table's
    initial state), the sine sqrt(2/(r+2)) sin(pi (j+1) / (r+2)) for the chain."""
    j = np.arange(r + 1)
    if kind == LATTICE_RELAXED:
        from math import comb
        return np.sqrt(np.array([comb(r, int(k)) for k in j], dtype=np.float64) / 2.0 ** r)
    return np.sqrt(2.0 / (r + 2)) * np.sin(np.pi * (j + 1) / (r + 2))


def initial_state(d: int, r: int, kind: int, init: int) -> np.ndarray:
    n = r + 1
    if init == INIT_UNIFORM:
        return np.full((n,) * d, n ** (-d / 2), dtype=np.complex128)
    v = axis_ground(r, kind)
    psi = np.ones((), dtype=np.float64)
    for _ in range(d):
        psi = np.multiply.outer(psi, v)
    return psi.astype(np.complex128)


def apply_axis(U: np.ndarray, psi: np.ndarray, k: int) -> np.ndarray:
    """(U acting on axis k) psi."""
    return np.moveaxis(np.tensordot(U, psi, axes=([1], [k])), 0, k)


def potential_phase(f: np.ndarray, theta: float) -> np.ndarray:
    """exp(-i theta f), the angle reduced modulo 2 pi in FP64 first."""
    return np.exp(-1j * np.mod(theta * f, 2.0 * np.pi))


def evolve(f: np.ndarray, psi: np.ndarray, r: int, kind: int, t0: float, dt: float, nsteps: int,
           sched: Schedule = Schedule()) -> np.ndarray:
    """nsteps Strang steps P(dt b/2) [prod_k exp(-i dt a K_k)] P(dt b/2), with
    a = e^{phi}, b = e^{chi} at the step midpoints.  dt < 0 runs backwards."""
    f = np.asarray(f, dtype=np.float64)
    psi = np.array(psi, dtype=np.complex128)
    d = f.ndim
    for j in range(nsteps):
        a, b = schedule_ab(sched, t0 + (j + 0.5) * dt)
        P = potential_phase(f, 0.5 * dt * b)
        U = axis_propagator(r, kind, dt * a)
        psi *= P
        for k in range(d):
            psi = apply_axis(U, psi, k)
        psi *= P
    return psi


@dataclass
class LatticeObs:
    norm: float
    e_f: float
    p_succ: float
    p_gap: float
    argmin: int
    f_min: float
    marginals: np.ndarray          # (d, r+1)
    prob: Optional[np.ndarray] = None


def observables(f: np.ndarray, psi: np.ndarray, r: int, radius: float = 0.1, gap: float = 0.01) -> LatticeObs:
    """p = |phi|^2, norm, E[f], the mass within `radius` (Euclidean) of the mesh
    argmin x* (lowest flat index on ties), the mass on points with
    f - min f <= gap, and the marginal of every axis (the measurement
    elements E^{(k)}_j of Eq. (Ekj))."""
    f = np.asarray(f, dtype=np.float64)
    p = np.abs(psi) ** 2
    d = f.ndim
    am = int(np.argmin(f.ravel()))
    xs = np.array(np.unravel_index(am, f.shape), dtype=np.float64) / r
    axes = np.meshgrid(*([mesh(r)] * d), indexing="ij")
    r2 = sum((ax - xs[k]) ** 2 for k, ax in enumerate(axes))
    fmin = float(f.ravel()[am])
    marg = np.stack([p.sum(axis=tuple(i for i in range(d) if i != k)) for k in range(d)])
    return LatticeObs(norm=float(p.sum()), e_f=float((p * f).sum()), p_succ=float(p[r2 < radius ** 2].sum()),
                      p_gap=float(p[f - fmin <= gap].sum()), argmin=am, f_min=fmin, marginals=marg, prob=p)


def hamiltonian_dense(f: np.ndarray, r: int, kind: int, a: float, b: float) -> np.ndarray:
    """The full (r+1)^d x (r+1)^d matrix a sum_k I..K..I + b diag(F) (small cases)."""
    f = np.asarray(f, dtype=np.float64)
    d = f.ndim
    n = r + 1
    K = kinetic_matrix(r, kind)
    H = np.diag(b * f.ravel()).astype(np.complex128)
    for k in range(d):
        H += a * np.kron(np.kron(np.eye(n ** k), K), np.eye(n ** (d - 1 - k)))
    return H
