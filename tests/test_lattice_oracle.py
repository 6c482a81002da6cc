"""Pins of the FP64 oracle of QHD on the finite-difference box mesh
(oracle/lattice.py): the relaxed operator against the Ising-machine
construction it encodes, the closed-form spectra and ground states of both
per-axis operators, the mesh potential against the Ising-format problem
Hamiltonian, and the time stepping against dense exponentials, exact free
evolution, separability, time reversal and mirror symmetry."""
from itertools import product

import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import lattice as L

SX = np.array([[0.0, 1.0], [1.0, 0.0]])
SZ = np.array([[1.0, 0.0], [0.0, -1.0]])


def site_op(op, j, nq):
    """op on qubit j of nq (qubit 0 is the most significant factor)."""
    return np.kron(np.kron(np.eye(2 ** j), op), np.eye(2 ** (nq - 1 - j)))


def s_x(nq):
    return sum(site_op(SX, j, nq) for j in range(nq))


def dicke_basis(r):
    """Columns: the normalised Hamming-weight states |D_w>, w = 0..r."""
    W = np.zeros((2 ** r, r + 1))
    for s in range(2 ** r):
        W[s, bin(s).count("1")] = 1.0
    return W / np.sqrt(W.sum(axis=0))


def random_qp(rng, d):
    Q = rng.uniform(-1, 1, (d, d))
    Q = 0.5 * (Q + Q.T)
    return Q, rng.uniform(-1, 1, d)


@pytest.mark.parametrize("r", [1, 2, 3, 4, 5])
def test_relaxed_operator_is_sx_on_hamming_weight_states(r):
    """The relaxed kinetic operator is S_x / sqrt(r) restricted to the span of
    the Hamming-weight states of r qubits, and that span is invariant
    (Hamming-encoding table: -A'/2 <-> -S_x / (2 sqrt(r)))."""
    W = dicke_basis(r)
    S = s_x(r)
    A = L.adjacency(r, L.LATTICE_RELAXED)
    assert np.abs(W.T @ S @ W / np.sqrt(r) - A).max() < 1e-13
    assert np.abs(S @ W - W @ (W.T @ S @ W)).max() < 1e-13
    # the end couplings are 1, the middle ones larger than the chain's
    assert A[0, 1] == pytest.approx(1.0) and A[r - 1, r] == pytest.approx(1.0)
    if r >= 3:
        assert A[1, 2] > 1.0


@pytest.mark.parametrize("r", [1, 2, 5, 8, 16])
def test_operator_spectra_closed_forms(r):
    """A' is 2 J_x / sqrt(r) of a spin r/2: eigenvalues (r - 2k) / sqrt(r);
    the chain adjacency of r+1 nodes: 2 cos(pi k / (r + 2)), k = 1..r+1."""
    ev = np.sort(np.linalg.eigvalsh(L.adjacency(r, L.LATTICE_RELAXED)))
    want = np.sort((r - 2.0 * np.arange(r + 1)) / np.sqrt(r))
    assert np.abs(ev - want).max() < 1e-12
    ev = np.sort(np.linalg.eigvalsh(L.adjacency(r, L.LATTICE_CHAIN)))
    want = np.sort(2 * np.cos(np.pi * np.arange(1, r + 2) / (r + 2)))
    assert np.abs(ev - want).max() < 1e-12


@pytest.mark.parametrize("kind", [L.LATTICE_CHAIN, L.LATTICE_RELAXED])
@pytest.mark.parametrize("r", [1, 3, 8])
def test_ground_states_are_top_eigenvectors(kind, r):
    A = L.adjacency(r, kind)
    v = L.axis_ground(r, kind)
    lam = np.linalg.eigvalsh(A).max()
    assert abs(v @ v - 1) < 1e-14
    assert np.abs(A @ v - lam * v).max() < 1e-13
    if kind == L.LATTICE_RELAXED:
        plus = np.full(2 ** r, 2.0 ** (-r / 2))          # |+>^r
        assert np.abs(dicke_basis(r).T @ plus - v).max() < 1e-14


@pytest.mark.parametrize("d,r", [(2, 2), (2, 3), (3, 2)])
def test_mesh_potential_equals_ising_format(d, r):
    """F on the mesh at x_p = |b_p| / r equals the Ising-format problem
    Hamiltonian of Eq. (ising-format-qp) on every bit string b (h_j, J_jk, g as
    printed there), i.e. Eq. (finite-quadratic-obj) evaluated on the mesh."""
    rng = np.random.default_rng(10 * d + r)
    Q, b = random_qp(rng, d)
    F = L.qp_potential(Q, b, r)
    n = d * r
    blk = np.repeat(np.arange(d), r)
    h = -(Q.sum(axis=1)[blk] + 2 * b[blk]) / (4 * r)
    g = (1 + 1 / r) * np.trace(Q) / 8 + sum(Q[p, q] for p in range(d) for q in range(p)) / 4 + b.sum() / 2
    for bits in product((0, 1), repeat=n):
        z = 1 - 2 * np.array(bits)
        hp = h @ z + g
        for j in range(n):
            for k in range(j):
                hp += Q[blk[j], blk[k]] / (4 * r * r) * z[j] * z[k]
        w = tuple(np.add.reduceat(np.array(bits), np.arange(0, n, r)))
        assert hp == pytest.approx(F[w], abs=1e-13)


def test_relaxed_hamiltonian_is_the_ising_machine_restricted():
    """With A(t) = r^{3/2} e^{phi}, B(t) = 2 e^{chi} (the dictionary's time
    functions, lambda = 1), -A/2 S_x + B/2 H_P leaves the product of
    Hamming-weight spans invariant and equals the relaxed QHD Hamiltonian there."""
    d, r = 2, 3
    rng = np.random.default_rng(3)
    Q, b = random_qp(rng, d)
    F = L.qp_potential(Q, b, r)
    n = d * r
    blk = np.repeat(np.arange(d), r)
    HP = np.zeros((2 ** n, 2 ** n))
    for j in range(n):
        HP += -(Q[blk[j]].sum() + 2 * b[blk[j]]) / (4 * r) * site_op(SZ, j, n)
        for k in range(j):
            HP += Q[blk[j], blk[k]] / (4 * r * r) * site_op(SZ, j, n) @ site_op(SZ, k, n)
    HP += ((1 + 1 / r) * np.trace(Q) / 8 + Q[1, 0] / 4 + b.sum() / 2) * np.eye(2 ** n)
    a, bb = 0.7, 1.9
    Hsim = -(r ** 1.5 * a) / 2 * s_x(n) + (2 * bb) / 2 * HP
    Wd = np.kron(dicke_basis(r), dicke_basis(r))
    Hlat = L.hamiltonian_dense(F, r, L.LATTICE_RELAXED, a, bb)
    assert np.abs(Wd.T @ Hsim @ Wd - Hlat).max() < 1e-12
    assert np.abs(Hsim @ Wd - Wd @ Hlat).max() < 1e-12


def const_schedule(a, b):
    return oracle.Schedule(kind=oracle.SCHED_TABLE, ts=np.array([0.0, 1.0]),
                           phis=np.array([np.log(a)] * 2), chis=np.array([np.log(b)] * 2))


@pytest.mark.parametrize("kind", [L.LATTICE_CHAIN, L.LATTICE_RELAXED])
def test_strang_orders_against_dense_exponential(kind):
    """Constant coefficients: one step is exp(-i dt H) up to O(dt^3), a fixed
    time T up to O(dt^2)."""
    d, r = 2, 3
    rng = np.random.default_rng(4)
    Q, b = random_qp(rng, d)
    F = 3 * L.qp_potential(Q, b, r)
    a, bb = 0.05, 1.0
    sch = const_schedule(a, bb)
    H = L.hamiltonian_dense(F, r, kind, a, bb)
    psi0 = (rng.standard_normal(F.shape) + 1j * rng.standard_normal(F.shape))
    psi0 /= np.linalg.norm(psi0)

    def err(dt, n):
        got = L.evolve(F, psi0, r, kind, 0.0, dt, n, sch).ravel()
        return np.linalg.norm(got - scipy.linalg.expm(-1j * dt * n * H) @ psi0.ravel())

    local = [err(dt, 1) for dt in (0.08, 0.04, 0.02)]
    assert 7.0 < local[0] / local[1] < 9.0 and 7.0 < local[1] / local[2] < 9.0, local
    glob = [err(0.8 / n, n) for n in (10, 20, 40)]
    assert 3.6 < glob[0] / glob[1] < 4.4 and 3.6 < glob[1] / glob[2] < 4.4, glob


@pytest.mark.parametrize("kind", [L.LATTICE_CHAIN, L.LATTICE_RELAXED])
def test_free_ground_state_only_turns_its_phase(kind):
    """f = 0: the kinetic ground state is an eigenvector of every factor, so
    psi(T) = exp(+i (r^2/2) d lambda_top sum_j dt a_j) psi0 exactly."""
    d, r = 3, 4
    lam = np.linalg.eigvalsh(L.adjacency(r, kind)).max()
    psi0 = L.initial_state(d, r, kind, L.INIT_KINETIC_GROUND)
    sch = oracle.Schedule()
    t0, dt, n = 1.0, 0.01, 150
    got = L.evolve(np.zeros(psi0.shape), psi0, r, kind, t0, dt, n, sch)
    phase = sum(dt * oracle.schedule_ab(sch, t0 + (j + 0.5) * dt)[0] for j in range(n)) * 0.5 * r * r * d * lam
    assert np.abs(got - np.exp(1j * phase) * psi0).max() < 1e-11


def test_separable_problem_factorises_over_axes():
    """Diagonal Q: F = sum_k F_k(x_k), so a product state stays the product of
    the one-dimensional evolutions (fixes the axis each factor acts on)."""
    d, r = 3, 4
    rng = np.random.default_rng(5)
    q = rng.uniform(-1, 1, d)
    b = rng.uniform(-1, 1, d)
    F = L.qp_potential(np.diag(q), b, r)
    vs = [rng.standard_normal(r + 1) + 1j * rng.standard_normal(r + 1) for _ in range(d)]
    vs = [v / np.linalg.norm(v) for v in vs]
    psi0 = np.einsum("i,j,k->ijk", *vs)
    sch = oracle.Schedule()
    got = L.evolve(F, psi0, r, L.LATTICE_RELAXED, 0.0, 0.01, 120, sch)
    parts = [L.evolve(L.qp_potential(np.array([[q[k]]]), b[k:k + 1], r), vs[k], r, L.LATTICE_RELAXED,
                      0.0, 0.01, 120, sch) for k in range(d)]
    assert np.abs(got - np.einsum("i,j,k->ijk", *parts)).max() < 1e-12


def test_norm_time_reversal_and_mirror_symmetry():
    d, r = 3, 4
    rng = np.random.default_rng(6)
    Q, _ = random_qp(rng, d)
    b = -0.5 * Q.sum(axis=1)          # f(x) = 1/2 (x - 1/2)^T Q (x - 1/2) + const: even under x -> 1 - x
    F = L.qp_potential(Q, b, r)
    sch = oracle.Schedule()
    for kind in (L.LATTICE_CHAIN, L.LATTICE_RELAXED):
        psi0 = L.initial_state(d, r, kind, L.INIT_KINETIC_GROUND)
        psi = L.evolve(F, psi0, r, kind, 0.0, 0.01, 400, sch)
        p = np.abs(psi) ** 2
        assert abs(p.sum() - 1) < 1e-12
        assert np.abs(p - p[::-1, ::-1, ::-1]).max() < 1e-13
        back = L.evolve(F, psi, r, kind, 4.0, -0.01, 400, sch)
        assert np.abs(back - psi0).max() < 1e-11


def test_observables_definitions():
    r = 4
    f = np.zeros((r + 1, r + 1))
    f[1, 2] = -1.0
    f[3, 0] = -1.0                    # tie: the lower flat index (1, 2) is x*
    f[1, 3] = -0.995
    p = np.zeros_like(f)
    p[1, 2], p[1, 3], p[0, 0], p[3, 0] = 0.4, 0.3, 0.2, 0.1
    o = L.observables(f, np.sqrt(p), r, radius=0.3, gap=0.01)
    assert o.argmin == 1 * (r + 1) + 2 and o.f_min == -1.0
    assert o.p_succ == pytest.approx(0.7)          # (1,3) is 0.25 away, (3,0) is not within 0.3
    assert o.p_gap == pytest.approx(0.8)           # -1, -1 and -0.995
    assert o.e_f == pytest.approx(-0.4 - 0.1 - 0.3 * 0.995)
    assert np.allclose(o.marginals[0], [0.2, 0.7, 0, 0.1, 0]) and np.allclose(o.marginals[1], [0.3, 0, 0.4, 0.3, 0])
    assert o.norm == pytest.approx(1.0)


def test_chain_drops_only_a_global_phase_of_the_printed_laplacian():
    """Eq. (discretize-pde) prints L = r^2 tridiag(1, -2, 1); the chain operator
    drops the -2 diagonal.  A Strang run with the printed operator (dense
    exponentials of the Kronecker sum) equals the oracle's run times the global
    phase exp(-i r^2 d sum_j dt a_j)."""
    d, r = 2, 3
    n = r + 1
    rng = np.random.default_rng(8)
    Q, b = random_qp(rng, d)
    F = L.qp_potential(Q, b, r)
    Lp = r * r * (np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1))
    Kp = np.kron(-0.5 * Lp, np.eye(n)) + np.kron(np.eye(n), -0.5 * Lp)
    sch = oracle.Schedule()
    t0, dt, steps = 0.5, 0.01, 60
    psi0 = L.initial_state(d, r, L.LATTICE_CHAIN, L.INIT_UNIFORM)
    psi = psi0.ravel().astype(complex)
    acc = 0.0
    for j in range(steps):
        a, bb = oracle.schedule_ab(sch, t0 + (j + 0.5) * dt)
        P = np.exp(-0.5j * dt * bb * F.ravel())
        psi = P * (scipy.linalg.expm(-1j * dt * a * Kp) @ (P * psi))
        acc += dt * a
    got = L.evolve(F, psi0, r, L.LATTICE_CHAIN, t0, dt, steps, sch).ravel()
    assert np.abs(psi - np.exp(-1j * r * r * d * acc) * got).max() < 1e-10


def test_ising_machine_evolution_reproduces_relaxed_qhd():
    """The relaxed QHD dynamics through the Hamming encoding, end to end: Strang
    steps of -A(t)/2 S_x + B(t)/2 H_P on d r qubits from |+>^{dr}, with the
    dictionary's A = r^{3/2} e^{phi}, B = 2 e^{chi} (lambda = 1), give
    Hamming-weight probabilities equal to the oracle's box-mesh p from the
    binomial state, step for step (each factor preserves the encoding span and
    restricts to the box-mesh factor)."""
    d, r = 2, 3
    rng = np.random.default_rng(9)
    Q, b = random_qp(rng, d)
    F = L.qp_potential(Q, b, r)
    nq = d * r
    blk = np.repeat(np.arange(d), r)
    HP = np.zeros((2 ** nq, 2 ** nq))
    for j in range(nq):
        HP += -(Q[blk[j]].sum() + 2 * b[blk[j]]) / (4 * r) * site_op(SZ, j, nq)
        for k in range(j):
            HP += Q[blk[j], blk[k]] / (4 * r * r) * site_op(SZ, j, nq) @ site_op(SZ, k, nq)
    HP += ((1 + 1 / r) * np.trace(Q) / 8 + Q[1, 0] / 4 + b.sum() / 2) * np.eye(2 ** nq)
    SXn = s_x(nq)
    sch = oracle.Schedule()
    t0, dt, steps = 0.2, 0.02, 40
    q = np.full(2 ** nq, 2.0 ** (-nq / 2), dtype=complex)
    lat = L.initial_state(d, r, L.LATTICE_RELAXED, L.INIT_KINETIC_GROUND)
    weights = np.array([[bin(s >> r).count("1"), bin(s & (2 ** r - 1)).count("1")] for s in range(2 ** nq)])
    for j in range(steps):
        a, bb = oracle.schedule_ab(sch, t0 + (j + 0.5) * dt)
        A, B = r ** 1.5 * a, 2 * bb
        half = scipy.linalg.expm(-0.5j * dt * (B / 2) * HP)
        q = half @ (scipy.linalg.expm(-1j * dt * (-(A / 2) * SXn)) @ (half @ q))
        lat = L.evolve(F, lat, r, L.LATTICE_RELAXED, t0 + j * dt, dt, 1, sch)
        pw = np.zeros((r + 1, r + 1))
        np.add.at(pw, (weights[:, 0], weights[:, 1]), np.abs(q) ** 2)
        assert np.abs(pw - np.abs(lat) ** 2).max() < 1e-12, j
