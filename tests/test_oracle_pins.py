"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: each checks it against a brute
force, a closed form, a textbook construction or an exact invariant, so that a
dropped term, a wrong sign or index, or a transposed operand fails one of them.
Paper: arXiv 2303.01471 (QHD).
"""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import Schedule, SCHED_TABLE
import workloads


def const_schedule(a, b):
    """Time-independent a=e^phi, b=e^chi as a flat table."""
    return Schedule(kind=SCHED_TABLE, ts=np.array([-1e9, 1e9]),
                    phis=np.array([math.log(a)] * 2), chis=np.array([math.log(b)] * 2))


def brute_dft(x, sign=-1):
    """Direct O(N^2)-per-axis DFT from the definition sum_j x_j e^{sign 2 pi i jk/N}."""
    out = np.asarray(x, dtype=np.complex128)
    for ax, n in enumerate(out.shape):
        j = np.arange(n)
        mat = np.exp(sign * 2j * np.pi * np.outer(j, j) / n)
        out = np.moveaxis(np.tensordot(mat, np.moveaxis(out, ax, 0), axes=(1, 0)), 0, ax)
    return out


# ------------------------------------------------------------------ P1: FFT

@pytest.mark.parametrize("shape", [(1,), (2,), (4,), (8,), (16,), (32,), (4, 8), (16, 2),
                                   (8, 4, 2), (4, 4, 4), (2, 16, 8)])
def test_fft_matches_brute_force_dft(shape):
    rng = np.random.default_rng(1)
    x = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    got = oracle.fft(x, -1)
    ref = brute_dft(x, -1)
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
    inv = oracle.fft(x, +1)
    ref_inv = brute_dft(x, +1) / x.size
    assert np.max(np.abs(inv - ref_inv)) <= 1e-13 * max(1.0, np.max(np.abs(ref_inv)))


@pytest.mark.parametrize("shape", [(64, 32), (16, 8, 32), (1024,)])
def test_fft_round_trip_parseval_and_library(shape):
    rng = np.random.default_rng(2)
    x = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    X = oracle.fft(x, -1)
    assert np.allclose(X, np.fft.fftn(x), rtol=0, atol=1e-11 * np.abs(X).max())
    back = oracle.fft(X, +1)
    assert np.max(np.abs(back - x)) <= 1e-13 * np.abs(x).max() * 10
    # Parseval: sum |x|^2 = sum |X|^2 / G
    assert abs(np.sum(np.abs(x) ** 2) - np.sum(np.abs(X) ** 2) / x.size) <= 1e-12 * np.sum(np.abs(x) ** 2)


# ------------------------------------------------------- schedule (paper)

def test_default_schedule_is_the_papers():
    """Eq. (nonconvex_QHD_h): e^{phi_t} = 2/(s+t^3), e^{chi_t} = 2 t^3, s = 0.001
    (values from the paper fixture in tests/golden)."""
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "paper_qhd_simulation.json")))
    s_paper = gold["s"]
    s = Schedule()
    assert s.eps == s_paper and s.c_phi == 2.0 and s.c_chi == 2.0
    for t in (0.0, 0.5, 1.0, 3.7, gold["T"]):
        a, b = oracle.schedule_ab(s, t)
        assert a == pytest.approx(2.0 / (s_paper + t ** 3), rel=1e-15)
        assert b == pytest.approx(2.0 * t ** 3, rel=1e-15, abs=0)


def test_table_schedule_is_piecewise_linear_in_phi_chi():
    ts = np.array([0.0, 1.0, 3.0])
    ph = np.array([0.0, 1.0, -1.0])
    ch = np.array([2.0, 0.0, 0.0])
    s = Schedule(kind=SCHED_TABLE, ts=ts, phis=ph, chis=ch)
    for t, phi, chi in [(-1, 0, 2), (0.25, 0.25, 1.5), (2.0, 0.0, 0.0), (5.0, -1.0, 0.0)]:
        a, b = oracle.schedule_ab(s, t)
        assert a == pytest.approx(math.exp(phi), rel=1e-15)
        assert b == pytest.approx(math.exp(chi), rel=1e-15)


# --------------------------------------------- P2: free particle closed form

def free_gaussian_density(xs_axes, x0, k0, sig0, A):
    """|psi|^2 of exp(-(x-x0)^2/(4 sig0^2) + i k0 x) after i d_t psi = -(a/2) Lap psi
    with int a dt = A: centre x0 + k0 A, variance sig0^2 (1 + (A/(2 sig0^2))^2)."""
    dens = 1.0
    for ax, xs in enumerate(xs_axes):
        var = sig0[ax] ** 2 * (1.0 + (A / (2.0 * sig0[ax] ** 2)) ** 2)
        c = x0[ax] + k0[ax] * A
        sh = [1] * len(xs_axes)
        sh[ax] = len(xs)
        dens = dens * np.exp(-((xs - c) ** 2) / (2.0 * var)).reshape(sh)
    return dens


@pytest.mark.parametrize("shape,lo,hi", [((256,), -10.0, 10.0),
                                         ((128, 64), (-10.0, -8.0), (10.0, 8.0))])
def test_free_particle_matches_closed_form(shape, lo, hi):
    d = len(shape)
    lo_ = np.broadcast_to(np.asarray(lo, float), (d,))
    hi_ = np.broadcast_to(np.asarray(hi, float), (d,))
    axes = [lo_[i] + np.arange(shape[i]) * (hi_[i] - lo_[i]) / shape[i] for i in range(d)]
    x0 = [-1.0, 0.5][:d]
    k0 = [2.0, -1.5][:d]
    sig0 = [0.5, 0.6][:d]
    psi = 1.0
    for ax, xs in enumerate(axes):
        sh = [1] * d
        sh[ax] = len(xs)
        psi = psi * np.exp(-((xs - x0[ax]) ** 2) / (4 * sig0[ax] ** 2) + 1j * k0[ax] * xs).reshape(sh)
    psi = psi / np.sqrt(np.sum(np.abs(psi) ** 2))
    sched = Schedule()
    t0, dt, n = 1.0, 0.01, 100
    out = oracle.evolve(np.zeros(shape), psi, t0, dt, n, sched, lo=lo_, hi=hi_)
    # the method applies exp(-i sum_j dt a(t_{j+1/2}) |k|^2/2): A is that sum
    A = sum(dt * 2.0 / (1e-3 + (t0 + (j + 0.5) * dt) ** 3) for j in range(n))
    ref = free_gaussian_density(axes, x0, k0, sig0, A)
    ref = ref / ref.sum()
    p = np.abs(out) ** 2
    assert np.max(np.abs(p - ref)) <= 1e-10 * ref.max()
    # a wrong kinetic sign would move the packet to x0 - k0 A
    centre = [np.sum(p * axes[ax].reshape([-1 if i == ax else 1 for i in range(d)])) for ax in range(d)]
    for ax in range(d):
        assert centre[ax] == pytest.approx(x0[ax] + k0[ax] * A, abs=1e-8)


# -------------------------------------------------- P3: static oscillator

def ho_setup(n=128, L=16.0, omega=1.1, a=1.3, b=0.7, shift=0.0):
    xs = -L / 2 + np.arange(n) * L / n
    f = 0.5 * omega ** 2 * xs ** 2
    alpha = omega * math.sqrt(b / a)   # ground state exp(-alpha x^2 / 2)
    psi = np.exp(-alpha * (xs - shift) ** 2 / 2).astype(np.complex128)
    psi /= np.linalg.norm(psi)
    return xs, f, psi, alpha


def test_oscillator_ground_state_is_stationary_and_virial():
    """Lemma (expect_potential): for an oscillator eigenstate <K> = <V>; the
    scaled Hamiltonian a(-Lap/2) + b w^2 x^2/2 has ground state exp(-w sqrt(b/a) x^2/2)."""
    a, b, omega = 1.3, 0.7, 1.1
    errs = []
    for dt in (0.02, 0.01):
        xs, f, psi, alpha = ho_setup(a=a, b=b, omega=omega)
        out = oracle.evolve(f, psi, 0.0, dt, int(round(2.0 / dt)), const_schedule(a, b),
                            lo=-8.0, hi=8.0)
        errs.append(np.max(np.abs(np.abs(out) ** 2 - np.abs(psi) ** 2)))
    assert errs[0] < 1e-4
    assert 3.6 < errs[0] / errs[1] < 4.4
    # virial on the evolved state
    k = 2 * np.pi * np.fft.fftfreq(len(xs), d=16.0 / len(xs))
    ph = np.fft.fft(out)
    kin = a * np.sum(np.abs(ph) ** 2 * k ** 2 / 2) / len(xs)
    pot = b * np.sum(np.abs(out) ** 2 * f)
    assert kin == pytest.approx(pot, rel=1e-4)
    assert kin + pot == pytest.approx(omega * math.sqrt(a * b) / 2, rel=1e-4)


def test_oscillator_coherent_state_oscillates_at_omega_sqrt_ab():
    a, b, omega, shift = 1.3, 0.7, 1.1, 1.0
    big_omega = omega * math.sqrt(a * b)
    T = 2.0
    errs = []
    for dt in (0.02, 0.01):
        xs, f, psi, alpha = ho_setup(a=a, b=b, omega=omega, shift=shift)
        out = oracle.evolve(f, psi, 0.0, dt, int(round(T / dt)), const_schedule(a, b),
                            lo=-8.0, hi=8.0)
        xc = shift * math.cos(big_omega * T)
        ref = np.exp(-alpha * (xs - xc) ** 2)
        ref /= ref.sum()
        errs.append(np.max(np.abs(np.abs(out) ** 2 - ref)))
    assert errs[0] < 1e-3
    assert 3.6 < errs[0] / errs[1] < 4.4


# ------------------------------------ P4 / P7: time-dependent Gaussian (Riccati)

def riccati_variance(t0, t1, y0, omega, sched, nsub=200000, paper_form=False):
    """Integrate y' = i a(t) - i b(t) w^2 y^2 (ansatz exp(-x^2/(2y)) in
    H = a(-d^2/2) + b w^2 x^2/2) by RK4; variance of |psi|^2 is 1/(2 Re(1/y)).
    paper_form=True integrates the coefficients as printed in Eq. (ode-a),
    y' = -i (t^3 y^2 - t^{-3}), for the same Hamiltonian Eq. (quadratic_model_qhd)."""
    def rhs(t, y):
        if paper_form:
            return -1j * (t ** 3 * y * y - t ** -3)
        a, b = oracle.schedule_ab(sched, t)
        return 1j * a - 1j * b * omega ** 2 * y * y
    h = (t1 - t0) / nsub
    y = complex(y0)
    t = t0
    for _ in range(nsub):
        k1 = rhs(t, y)
        k2 = rhs(t + h / 2, y + h / 2 * k1)
        k3 = rhs(t + h / 2, y + h / 2 * k2)
        k4 = rhs(t + h, y + h * k3)
        y += h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        t += h
    return 1.0 / (2.0 * (1.0 / y).real)


@pytest.mark.slow
def test_time_dependent_gaussian_matches_riccati():
    """Prop. (quadratic_rate): f = x^2/2 with a = 2/t^3, b = 2 t^3 keeps a Gaussian;
    its variance follows the Riccati equation, which we derive for the paper's H."""
    omega = 1.0
    sched = Schedule(c_phi=2.0, eps=0.0, c_chi=2.0)
    t0, t1 = 1.0, 2.0
    n, L = 256, 12.0
    xs = -L / 2 + np.arange(n) * L / n
    f = 0.5 * omega ** 2 * xs ** 2
    y0 = 2.0  # Eq. (ode-c): y(0)=2, i.e. variance 1
    psi = np.exp(-xs ** 2 / (2 * y0)).astype(np.complex128)
    psi /= np.linalg.norm(psi)
    var_ode = riccati_variance(t0, t1, y0, omega, sched, nsub=20000)
    vs = []
    for dt in (0.004, 0.002):
        out = oracle.evolve(f, psi, t0, dt, int(round((t1 - t0) / dt)), sched, lo=-L / 2, hi=L / 2)
        p = np.abs(out) ** 2
        vs.append(np.sum(p * xs ** 2) / np.sum(p))
    e0, e1 = abs(vs[0] - var_ode), abs(vs[1] - var_ode)
    assert e1 < 2e-5 * var_ode
    assert 3.0 < e0 / e1 < 5.0
    # the coefficients printed in Eq. (ode-a) miss a factor 2 for this H
    var_paper = riccati_variance(t0, t1, y0, omega, sched, nsub=20000, paper_form=True)
    assert abs(var_paper - var_ode) > 100 * e1


# ------------------------------------------------------- P5 norm, P6 order

def test_norm_conserved_over_many_steps():
    inst = workloads.gaussian_wells(3, (32, 32), K=8)
    psi = oracle.uniform_state(inst.f.shape)
    out = oracle.evolve(inst.f, psi, 0.0, 1e-3, 10000, Schedule())
    assert abs(np.sum(np.abs(out) ** 2) - 1.0) <= 1e-12


def smooth_periodic_f(shape):
    """Band-limited periodic objective: the split error is then in its asymptotic regime."""
    X, Y = np.meshgrid(*workloads.mesh_axes(shape), indexing="ij")
    return -np.cos(2 * np.pi * X) - 0.5 * np.cos(2 * np.pi * Y) + 0.3 * np.sin(2 * np.pi * (X + Y))


def test_second_order_convergence_in_dt():
    """Strang with midpoint coefficients is second order even for the time-dependent
    schedule (a left-end-point sample would make it first order)."""
    f = smooth_periodic_f((32, 32))
    psi = oracle.uniform_state(f.shape)
    t0, T = 1.0, 0.4
    ref = oracle.evolve(f, psi, t0, T / 2560, 2560, Schedule())
    errs = [np.linalg.norm(oracle.evolve(f, psi, t0, T / n, n, Schedule()) - ref)
            for n in (20, 40, 80)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.8 < r1 < 4.2 and 3.8 < r2 < 4.2, (errs, r1, r2)


def test_lie_trotter_is_first_order():
    """Eq. (prod_qhd) as printed is a first-order formula: halving dt halves the error."""
    f = smooth_periodic_f((32, 32))
    psi = oracle.uniform_state(f.shape)
    t0, T = 1.0, 0.4
    ref = oracle.evolve(f, psi, t0, T / 2560, 2560, Schedule())
    errs = [np.linalg.norm(oracle.evolve_trotter(f, psi, t0, T / n, n) - ref)
            for n in (20, 40, 80)]
    assert 1.9 < errs[0] / errs[1] < 2.1 and 1.9 < errs[1] / errs[2] < 2.1, errs


def commuting_closed_form(psi0, c, A, B, lo, hi):
    """Exact map of i dpsi/dt = [a(t)(-Lap/2) + b(t) c] psi for a constant objective
    f = c, whose two terms commute: psi(T) = e^{-i c B} F^-1[e^{-i A |k|^2/2} F psi0]
    with A = int a, B = int b (numpy's FFT, k = 2 pi m / L)."""
    psi_k = np.fft.fftn(psi0)
    k2 = 0.0
    for ax, n in enumerate(psi0.shape):
        k = 2.0 * np.pi * np.fft.fftfreq(n, d=(hi - lo) / n)
        sh = [1] * psi0.ndim
        sh[ax] = n
        k2 = k2 + (k ** 2).reshape(sh)
    return np.exp(-1j * c * B) * np.fft.ifftn(np.exp(-1j * A * k2 / 2.0) * psi_k)


@pytest.mark.parametrize("shape", [(64,), (32, 16)])
def test_lie_trotter_samples_the_left_end_point(shape):
    """Eq. (prod_qhd) takes a_j = e^{phi(js)}, b_j = e^{chi(js)} at the left end of
    each step.  With a constant objective the potential and kinetic factors commute,
    so the product formula is exact for whatever times it samples: the result must
    be the closed form with A = sum_j dt a(t0 + j dt), B = sum_j dt b(t0 + j dt).
    The midpoint or right-end sums give states far from it, so a misread sampling
    time fails here (the order test alone cannot tell them apart)."""
    rng = np.random.default_rng(3)
    lo, hi = -4.0, 4.0
    psi0 = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    psi0 /= np.linalg.norm(psi0)
    c = 0.7
    f = np.full(shape, c)
    t0, dt, n = 0.6, 0.05, 24
    sched = Schedule()
    def sums(offset):
        ab = [oracle.schedule_ab(sched, t0 + (j + offset) * dt) for j in range(n)]
        return dt * sum(a for a, _ in ab), dt * sum(b for _, b in ab)
    got = oracle.evolve_trotter(f, psi0, t0, dt, n, lo=lo, hi=hi)
    left = commuting_closed_form(psi0, c, *sums(0.0), lo, hi)
    assert np.max(np.abs(got - left)) <= 1e-10
    for offset in (0.5, 1.0):
        other = commuting_closed_form(psi0, c, *sums(offset), lo, hi)
        assert np.max(np.abs(got - other)) > 1e-2
    # Strang (Eq. (prod_qhd) in symmetric form, midpoint coefficients) is exact
    # here too, with the midpoint sums
    strang = oracle.evolve(f, psi0, t0, dt, n, sched, lo=lo, hi=hi)
    mid = commuting_closed_form(psi0, c, *sums(0.5), lo, hi)
    assert np.max(np.abs(strang - mid)) <= 1e-10


# ----------------------------------------------- P8 reversal, P9 dilation

def test_time_reversal_returns_initial_state():
    inst = workloads.gaussian_wells(5, (16, 16), K=8)
    rng = np.random.default_rng(0)
    psi = rng.normal(size=(16, 16)) + 1j * rng.normal(size=(16, 16))
    psi /= np.linalg.norm(psi)
    # start at t=1 so the per-step kinetic phases stay O(10) rad: the backward
    # midpoints 2 - (j+1/2) dt differ from the forward ones in the last bit,
    # which a phase of 1e4 rad (t near 0) would amplify to ~1e-12.
    fwd = oracle.evolve(inst.f, psi, 1.0, 0.01, 100, Schedule())
    back = oracle.evolve(inst.f, fwd, 2.0, -0.01, 100, Schedule())
    assert np.max(np.abs(back - psi)) <= 1e-12
    assert np.max(np.abs(fwd - psi)) > 1e-2


def test_time_dilation_invariance():
    """Prop. (time_dilation): tau(t)=2t gives e^{phi~}=2 e^{phi(2t)}, e^{chi~}=2 e^{chi(2t)};
    for the Nesterov family that is c_phi/4, eps/8, 16 c_chi.  Midpoints map onto
    midpoints, so the discrete trajectories coincide."""
    inst = workloads.gaussian_wells(6, (32, 32), K=8)
    psi = oracle.uniform_state(inst.f.shape)
    s = Schedule(c_phi=2.0, eps=1e-3, c_chi=2.0)
    sd = Schedule(c_phi=0.5, eps=1e-3 / 8, c_chi=32.0)
    a = oracle.evolve(inst.f, psi, 0.2, 0.01, 200, s)
    b = oracle.evolve(inst.f, psi, 0.1, 0.005, 200, sd)
    assert np.max(np.abs(a - b)) <= 1e-11


# ------------------------------------- P9b ideal-scaling power family

def test_power_family_meets_ideal_scaling_with_equality():
    """Eq. (qhd_operator_convex) / Eq. (ideal_scaling): the power kind with eps = 0,
    c_phi = p, c_chi = p C comes from alpha, beta = gamma + log C, gamma with
    gamma' = e^alpha and beta' = e^alpha.  Recover gamma = (log b - log a - log C)/3 and
    alpha = log a + gamma from the oracle's (a, b) and check gamma' = e^alpha."""
    for p, C in [(2.0, 1.0), (1.5, 0.7), (3.0, 2.0)]:
        s = Schedule(kind=oracle.SCHED_POWER, c_phi=p, eps=0.0, c_chi=p * C, power=p)

        def alpha_gamma(t):
            a, b = oracle.schedule_ab(s, t)
            g = (math.log(b) - math.log(a) - math.log(C)) / 3.0
            return math.log(a) + g, g

        for t in [0.3, 1.0, 2.7]:
            h = 1e-5
            dg = (alpha_gamma(t + h)[1] - alpha_gamma(t - h)[1]) / (2 * h)
            assert dg == pytest.approx(math.exp(alpha_gamma(t)[0]), rel=1e-8), (p, t)


def test_power_family_p2_is_the_paper_schedule():
    """p = 2 gives e^phi = c_phi/(eps + t^3), e^chi = c_chi t^3 (Eq. (nonconvex_QHD_h))."""
    inst = workloads.gaussian_wells(4, (32, 32), K=8)
    psi = oracle.uniform_state(inst.f.shape)
    a = oracle.evolve(inst.f, psi, 0.0, 0.01, 200, Schedule())
    b = oracle.evolve(inst.f, psi, 0.0, 0.01, 200, Schedule(kind=oracle.SCHED_POWER, power=2.0))
    assert np.max(np.abs(a - b)) <= 1e-12


def test_power_family_time_dilation():
    """Prop. (time_dilation) with tau = k t maps the power family onto itself:
    (c_phi, eps, c_chi) -> (c_phi k^-p, eps k^-(p+1), c_chi k^2p); midpoints map onto
    midpoints, so the discrete trajectories at dt and dt/k coincide."""
    inst = workloads.gaussian_wells(7, (32, 32), K=8)
    psi = oracle.uniform_state(inst.f.shape)
    p, k = 1.5, 2.0
    s = Schedule(kind=oracle.SCHED_POWER, c_phi=1.5, eps=1e-3, c_chi=3.0, power=p)
    sd = Schedule(kind=oracle.SCHED_POWER, c_phi=1.5 * k ** -p, eps=1e-3 * k ** -(p + 1),
                  c_chi=3.0 * k ** (2 * p), power=p)
    a = oracle.evolve(inst.f, psi, 0.2, 0.01, 200, s)
    b = oracle.evolve(inst.f, psi, 0.2 / k, 0.01 / k, 200, sd)
    assert np.max(np.abs(a - b)) <= 1e-11
    assert np.max(np.abs(np.abs(a) ** 2 - np.abs(psi) ** 2)) > 1e-4   # it did evolve


# ------------------------------------------------------- P10 mirror symmetry

def test_mirror_symmetry():
    shape = (32, 16)
    axes = workloads.mesh_axes(shape)
    X, Y = np.meshgrid(*axes, indexing="ij")
    f = 0.5 * ((X - 0.5) ** 2 + (Y - 0.5) ** 2) - 1.2 * np.exp(-((X - 0.5) ** 2) / 0.02) \
        - 0.7 * np.exp(-((Y - 0.5) ** 2) / 0.01)
    psi = oracle.uniform_state(shape)
    out = oracle.evolve(f, psi, 0.0, 0.01, 300, Schedule())
    p = np.abs(out) ** 2
    mirrored = p[(-np.arange(32)) % 32][:, (-np.arange(16)) % 16]
    assert np.max(np.abs(p - mirrored)) <= 1e-13
    assert np.max(np.abs(p - p.mean())) > 1e-4   # it did evolve


# ------------------------------------- P11 dense exponential (textbook D2)

def trefethen_d2(n):
    """Second-derivative matrix of the periodic band-limited interpolant on
    [0, 2 pi), n even (Trefethen, Spectral Methods in MATLAB, ch. 3)."""
    h = 2 * np.pi / n
    d2 = np.empty((n, n))
    for j in range(n):
        for l in range(n):
            if j == l:
                d2[j, l] = -np.pi ** 2 / (3 * h ** 2) - 1.0 / 6.0
            else:
                d2[j, l] = -((-1.0) ** (j - l)) / (2 * np.sin((j - l) * h / 2) ** 2)
    return d2


def dense_kinetic(shape, lengths):
    mats = [-0.5 * (2 * np.pi / L) ** 2 * trefethen_d2(n) for n, L in zip(shape, lengths)]
    K = np.zeros((int(np.prod(shape)),) * 2)
    for ax in range(len(shape)):
        term = np.ones((1, 1))
        for j in range(len(shape)):
            term = np.kron(term, mats[j] if j == ax else np.eye(shape[j]))
        K += term
    return K


@pytest.mark.parametrize("shape,lengths", [((8,), (1.0,)), ((4, 4), (1.0, 2.0))])
def test_one_strang_step_equals_dense_exponentials(shape, lengths):
    rng = np.random.default_rng(7)
    f = rng.uniform(-1, 1, size=shape)
    psi = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    psi /= np.linalg.norm(psi)
    K = dense_kinetic(shape, lengths)
    V = np.diag(f.ravel())
    sched = Schedule()
    t0, dt = 0.7, 0.013
    a, b = oracle.schedule_ab(sched, t0 + dt / 2)
    U = scipy.linalg.expm(-0.5j * dt * b * V) @ scipy.linalg.expm(-1j * dt * a * K) \
        @ scipy.linalg.expm(-0.5j * dt * b * V)
    ref = (U @ psi.ravel()).reshape(shape)
    out = oracle.evolve(f, psi, t0, dt, 1, sched, lo=0.0, hi=np.asarray(lengths))
    assert np.max(np.abs(out - ref)) <= 1e-12


def fd_laplacian(n, L):
    """Central second difference of Eq. (discretize-pde), (psi_{j+1} - 2 psi_j +
    psi_{j-1}) / h^2 with h = L / n, with the periodic wrap of the mesh."""
    h = L / n
    D = -2.0 * np.eye(n)
    for j in range(n):
        D[j, (j + 1) % n] += 1.0
        D[j, (j - 1) % n] += 1.0
    return D / h ** 2


@pytest.mark.parametrize("shape,lengths", [((8,), (1.0,)), ((4, 8), (1.0, 2.0)), ((4, 2, 4), (1.0, 1.0, 0.5))])
def test_fd_kinetic_step_equals_dense_exponentials(shape, lengths):
    """The finite-difference kinetic operator: one Strang step equals
    e^{-i dt b F/2} e^{-i dt a (-D/2)} e^{-i dt b F/2} with D the Kronecker sum of the
    per-axis central-difference matrices, written out from Eq. (discretize-pde)."""
    rng = np.random.default_rng(8)
    f = rng.uniform(-1, 1, size=shape)
    psi = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    psi /= np.linalg.norm(psi)
    G = int(np.prod(shape))
    D = np.zeros((G, G))
    for ax in range(len(shape)):
        term = np.ones((1, 1))
        for j in range(len(shape)):
            term = np.kron(term, fd_laplacian(shape[j], lengths[j]) if j == ax else np.eye(shape[j]))
        D += term
    sched = Schedule()
    t0, dt = 0.4, 0.011
    a, b = oracle.schedule_ab(sched, t0 + dt / 2)
    F = np.diag(f.ravel())
    U = scipy.linalg.expm(-0.5j * dt * b * F) @ scipy.linalg.expm(-1j * dt * a * (-0.5 * D)) \
        @ scipy.linalg.expm(-0.5j * dt * b * F)
    ref = (U @ psi.ravel()).reshape(shape)
    out = oracle.evolve(f, psi, t0, dt, 1, sched, lo=0.0, hi=np.asarray(lengths), kinetic=oracle.KINETIC_FD2)
    assert np.max(np.abs(out - ref)) <= 1e-12
    # and the spectral operator is a different one on the same mesh
    spec = oracle.evolve(f, psi, t0, dt, 1, sched, lo=0.0, hi=np.asarray(lengths))
    assert np.max(np.abs(spec - out)) > 1e-6


def test_fd_kinetic_converges_to_spectral_at_second_order():
    """For a smooth state the central difference differs from the exact second
    derivative by O(h^2): halving h divides the FD-vs-spectral difference by ~4
    (a smooth periodic potential, kinetic-dominated weights)."""
    def diff(n):
        x = np.arange(n) / n
        X, Y = np.meshgrid(x, x, indexing="ij")
        f = np.cos(2 * np.pi * X) * np.cos(2 * np.pi * Y)
        psi = np.exp(2j * np.pi * X) * np.exp(np.cos(2 * np.pi * Y)) + 0j
        psi /= np.linalg.norm(psi)
        sched = const_schedule(1.0, 1e-2)
        a = oracle.evolve(f, psi, 0.0, 0.01, 20, sched)
        b = oracle.evolve(f, psi, 0.0, 0.01, 20, sched, kinetic=oracle.KINETIC_FD2)
        return np.max(np.abs(a - b)) * n   # per-point amplitude scale ~ 1/n
    r = diff(64) / diff(128)
    assert 3.5 < r < 4.5, r


def test_strang_local_error_is_third_order():
    shape, lengths = (8,), (1.0,)
    rng = np.random.default_rng(8)
    f = rng.uniform(-1, 1, size=shape) * 40
    psi = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    psi /= np.linalg.norm(psi)
    a, b = 0.01, 1.0
    H = a * dense_kinetic(shape, lengths) + b * np.diag(f)
    errs = []
    for dt in (0.02, 0.01, 0.005):
        ex = scipy.linalg.expm(-1j * dt * H) @ psi
        out = oracle.evolve(f, psi, 0.0, dt, 1, const_schedule(a, b))
        errs.append(np.linalg.norm(out - ex))
    for e0, e1 in zip(errs, errs[1:]):
        assert 7.0 < e0 / e1 < 9.0, errs


# ------------------------------------------------------------- observables

def test_observables_brute_force():
    shape = (32, 16)
    inst = workloads.gaussian_wells(9, shape, K=8)
    rng = np.random.default_rng(3)
    psi = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    psi /= np.linalg.norm(psi)
    ob = oracle.observables(inst.f, psi, radius=0.1)
    p = np.abs(psi) ** 2
    assert ob.norm == pytest.approx(1.0, abs=1e-14)
    assert ob.e_f == pytest.approx(float(np.sum(p * inst.f)), rel=1e-13)
    i, j = np.unravel_index(np.argmin(inst.f), shape)
    xs = (i / 32, j / 16)
    assert tuple(ob.x_star[:2]) == pytest.approx(xs)
    tot = 0.0
    for a in range(32):
        for b in range(16):
            if math.hypot(a / 32 - xs[0], b / 16 - xs[1]) < 0.1:
                tot += p[a, b]
    assert ob.p_succ == pytest.approx(tot, rel=1e-13)
    uni = oracle.observables(inst.f, oracle.uniform_state(shape))
    assert uni.e_f == pytest.approx(inst.f.mean(), rel=1e-13)


def test_observables_argmin_tie_takes_lowest_index():
    f = np.ones((4, 4))
    f[1, 2] = 0.0
    f[3, 0] = 0.0
    ob = oracle.observables(f, oracle.uniform_state((4, 4)), lo=0.0, hi=1.0)
    assert tuple(ob.x_star[:2]) == (0.25, 0.5)


# ------------------------------------- P13 the Hamiltonian and its spectrum

@pytest.mark.parametrize("kinetic", [0, 1])
@pytest.mark.parametrize("shape,lengths", [((8,), (1.0,)), ((4, 8), (1.0, 2.0)), ((4, 2, 4), (1.0, 1.0, 0.5))])
def test_apply_h_equals_dense_matrix(shape, lengths, kinetic):
    """H = a (-Lap/2) + b f (Eq. (qhd_operator)) against dense matrices written out
    independently: Trefethen's spectral second derivative, or the central
    difference of Eq. (discretize-pde)."""
    rng = np.random.default_rng(9)
    f = rng.uniform(-1, 1, size=shape)
    psi = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    a, b = 0.7, 1.9
    if kinetic == 0:
        K = dense_kinetic(shape, lengths)
    else:
        G = int(np.prod(shape))
        D = np.zeros((G, G))
        for ax in range(len(shape)):
            term = np.ones((1, 1))
            for j in range(len(shape)):
                term = np.kron(term, fd_laplacian(shape[j], lengths[j]) if j == ax else np.eye(shape[j]))
            D += term
        K = -0.5 * D
    H = a * K + b * np.diag(f.ravel())
    got = oracle.apply_h(f, psi, a, b, lo=0.0, hi=np.asarray(lengths), kinetic=kinetic)
    assert np.max(np.abs(got.ravel() - H @ psi.ravel())) <= 1e-11 * np.abs(H).max() * np.abs(psi).max() * 10


def test_free_particle_spectrum_closed_form():
    """f = 0: the eigenvalues are a |k|^2 / 2, k = 2 pi m / L, with their multiplicities.
    k = 11 ends on a whole level (the fourfold 32.08): a cut inside a degenerate
    level leaves Lanczos free to return a copy of the next level instead."""
    shape, L, a = (16, 8), (1.0, 2.0), 1.3
    got = oracle.lowest_eigs(np.zeros(shape), a, 1.0, 11, hi=np.asarray(L))
    ms = [(m0, m1) for m0 in range(-8, 8) for m1 in range(-4, 4)]
    want = sorted(a / 2 * ((2 * np.pi * m0 / L[0]) ** 2 + (2 * np.pi * m1 / L[1]) ** 2) for m0, m1 in ms)[:11]
    assert np.allclose(got, want, rtol=1e-9, atol=1e-9)


def test_harmonic_oscillator_spectrum():
    """H = a (-1/2 d^2/dx^2) + b omega^2 x^2 / 2 has E_n = sqrt(a b) omega (n + 1/2)
    (the oscillator of Lemma (expect_potential)); a wide, fine periodic box resolves
    the low levels to spectral accuracy."""
    n, L = 128, 24.0
    x = -L / 2 + np.arange(n) * L / n
    a, b, om = 0.8, 1.7, 1.1
    got = oracle.lowest_eigs(0.5 * om ** 2 * x ** 2, a, b, 5, lo=-L / 2, hi=L / 2)
    want = np.sqrt(a * b) * om * (np.arange(5) + 0.5)
    assert np.allclose(got, want, rtol=1e-9)


def test_paper_levy_semiclassical_energy_ratio():
    """The paper's worked example: the Levy function's Hessian at (1, 1) gives
    omega_1 ~ 1.4979, omega_2 ~ 0.3536 and the semi-classical ratio E1/E0 ~ 1.3819
    (fixture).  The printed omegas follow from the printed Hessian eigenvalues, and
    the oracle's lowest levels of H for the quadratic model reproduce the ratio."""
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_levy_energy_ratio.json")))
    lam1 = (np.pi ** 2 + 1 + 10 * np.sin(1.0) ** 2) / 8
    om1, om2 = np.sqrt(lam1), np.sqrt(gold["hessian_eigenvalue_2"])
    tol = 0.5 * 10.0 ** -gold["printed_digits"]
    assert abs(om1 - gold["omega_1"]) <= tol and abs(om2 - gold["omega_2"]) <= tol
    n, L = 64, 24.0
    x = -L / 2 + np.arange(n) * L / n
    X1, X2 = np.meshgrid(x, x, indexing="ij")
    f = 0.5 * om1 ** 2 * X1 ** 2 + 0.5 * om2 ** 2 * X2 ** 2
    E = oracle.lowest_eigs(f, 1.0, 1.0, 2, lo=-L / 2, hi=L / 2)
    assert abs(E[1] / E[0] - gold["semiclassical_ratio"]) <= tol
    assert E[1] / E[0] == pytest.approx((om1 + 3 * om2) / (om1 + om2), rel=1e-8)
