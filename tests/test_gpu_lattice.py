"""The box-mesh QHD kernels (qhd_lattice_*) against the FP64 oracle of
oracle/lattice.py: the Sim-QHD configuration (5-d box QPs, r = 8, relaxed
operator, Hamming-encoding initial state, T = 10, dt = 0.01) element by
element, the chain operator, every line length class (odd and even n, one
and several passes per step, ragged tiles), per-instance schedules, several
chunks, time reversal, the closed-form initial states and the error paths."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
import workloads
from oracle import lattice as OL
from paper_2303_01471_gb300 import lattice, qhd

TV_MAX, EF_MAX, NORM_MAX = 1e-4, 1e-5, 1e-6


def oracle_run(F, r, kind, init, T, dt, sched):
    psi0 = OL.initial_state(F.ndim, r, kind, init)
    return OL.evolve(F, psi0, r, kind, 0.0, dt, int(round(T / dt)), sched)


def compare(lat, Fs, psis_ref, r, radius=0.1, gap=0.01, steps=1000):
    prob = torch.empty((lat.batch, *lat.shape), dtype=torch.float32, device="cuda")
    obs = lat.observables(radius, gap, prob=prob, marginals=True)
    p_gpu = prob.double().cpu().numpy()
    for i, (F, psi) in enumerate(zip(Fs, psis_ref)):
        o = OL.observables(F, psi, r, radius, gap)
        tv = 0.5 * np.abs(p_gpu[i] - o.prob).sum()
        den = max(abs(o.e_f), 1e-3 * (F.max() - F.min()))
        assert tv <= TV_MAX, (i, tv)
        assert abs(obs[i].e_f - o.e_f) <= EF_MAX * den, (i, obs[i].e_f, o.e_f)
        assert abs(obs[i].norm - 1.0) <= NORM_MAX, (i, obs[i].norm)
        assert abs(obs[i].p_succ - o.p_succ) <= TV_MAX and abs(obs[i].p_gap - o.p_gap) <= TV_MAX
        assert obs[i].argmin == o.argmin and obs[i].f_min == pytest.approx(o.f_min, abs=1e-12)
        assert np.abs(obs[i].marginals - o.marginals).max() <= TV_MAX
        # the observables of the GPU's own p agree with its FP64 reductions
        assert abs(p_gpu[i].sum() - obs[i].norm) <= 1e-5
    return obs


def test_sim_qhd_5d_box_qp_relaxed():
    """Sim-QHD: two 5-d box QPs on 9^5 mesh points, relaxed operator, discrete
    Gaussian start, Nesterov schedule with sigma per instance (shared kinetic
    factor), 1000 steps; the mesh F is formed on the device from (Q, b)."""
    d, r, T, dt = 5, 8, 10.0, 0.01
    qps = [workloads.box_qp(s, d) for s in (11, 12)]
    sig = [1.0, 1.7]
    lat = lattice.Lattice(d, r, lattice.RELAXED, batch=2)
    lat.set_qp(np.stack([q for q, _ in qps]), np.stack([b for _, b in qps]))
    lat.set_schedule([qhd.Schedule(c_chi=2 * s) for s in sig])
    lat.reset_state(lattice.INIT_GROUND)
    lat.evolve(T, dt)
    Fs = [OL.qp_potential(Q, b, r) for Q, b in qps]
    refs = [oracle_run(F, r, OL.LATTICE_RELAXED, OL.INIT_KINETIC_GROUND, T, dt, oracle.Schedule(c_chi=2 * s))
            for F, s in zip(Fs, sig)]
    obs = compare(lat, Fs, refs, r)
    assert obs[0].steps_done == 1000 and obs[0].t == pytest.approx(10.0)
    lat.close()


def test_chain_3d_r16_uniform_per_instance_kinetic():
    """Chain operator, n = 17 (two passes: the last two axes, then axis 0),
    three instances with different e^{phi} (one propagator each), one of them
    on the power-law schedule."""
    d, r, T, dt = 3, 16, 5.0, 0.01
    qps = [workloads.box_qp(s, d) for s in (21, 22, 23)]
    scheds = [qhd.Schedule(c_phi=2.0), qhd.Schedule(c_phi=1.0, c_chi=3.0),
              qhd.Schedule(kind=qhd.SCHED_POWER, c_phi=3.0, eps=1e-3, c_chi=3.0, power=3.0)]
    oscheds = [oracle.Schedule(c_phi=2.0), oracle.Schedule(c_phi=1.0, c_chi=3.0),
               oracle.Schedule(kind=oracle.SCHED_POWER, c_phi=3.0, eps=1e-3, c_chi=3.0, power=3.0)]
    lat = lattice.Lattice(d, r, lattice.CHAIN, batch=3)
    lat.set_qp(np.stack([q for q, _ in qps]), np.stack([b for _, b in qps]))
    lat.set_schedule(scheds)
    lat.reset_state(lattice.INIT_UNIFORM)
    lat.evolve(T, dt)
    Fs = [OL.qp_potential(Q, b, r) for Q, b in qps]
    refs = [oracle_run(F, r, OL.LATTICE_CHAIN, OL.INIT_UNIFORM, T, dt, s) for F, s in zip(Fs, oscheds)]
    compare(lat, Fs, refs, r, radius=0.15, steps=500)
    lat.close()


@pytest.mark.parametrize("d,r,kind", [(4, 7, lattice.RELAXED),    # n = 8: padded lines, two passes
                                      (6, 2, lattice.CHAIN),      # 3^6 in one pass (both phases)
                                      (1, 1, lattice.RELAXED),    # n = 2, one axis
                                      (2, 5, lattice.CHAIN),      # n = 6 even, one pass
                                      (3, 11, lattice.RELAXED)])  # n = 12: 144-point group + strided axis
def test_shapes_against_oracle(d, r, kind):
    T, dt = 3.0, 0.01
    B = 2
    rng = np.random.default_rng(100 * d + r)
    Fs = [3.0 * rng.standard_normal((r + 1,) * d) for _ in range(B)]   # an arbitrary potential on the mesh
    lat = lattice.Lattice(d, r, kind, batch=B)
    lat.set_potential(torch.from_numpy(np.stack(Fs)).cuda())
    lat.set_schedule(qhd.Schedule())
    lat.reset_state(lattice.INIT_GROUND)
    lat.evolve(T, dt)
    okind = OL.LATTICE_CHAIN if kind == lattice.CHAIN else OL.LATTICE_RELAXED
    refs = [oracle_run(F, r, okind, OL.INIT_KINETIC_GROUND, T, dt, oracle.Schedule()) for F in Fs]
    compare(lat, Fs, refs, r, radius=0.3, gap=0.5, steps=300)
    lat.close()


def test_several_chunks_and_split_evolve_calls():
    """2500 steps in one call (three chunks of propagators) equal the oracle;
    two calls of 1250 steps each are two Strang runs joined at t = 12.5."""
    d, r = 2, 8
    Q, b = workloads.box_qp(31, d)
    F = OL.qp_potential(Q, b, r)
    lat = lattice.Lattice(d, r, lattice.RELAXED)
    lat.set_qp(Q[None], b[None])
    lat.set_schedule(qhd.Schedule())
    lat.reset_state(lattice.INIT_GROUND)
    lat.evolve(25.0, 0.01)
    ref = oracle_run(F, r, OL.LATTICE_RELAXED, OL.INIT_KINETIC_GROUND, 25.0, 0.01, oracle.Schedule())
    compare(lat, [F], [ref], r, steps=2500)
    lat.reset_state(lattice.INIT_GROUND)
    lat.evolve(12.5, 0.01)
    lat.evolve(12.5, 0.01)
    mid = oracle_run(F, r, OL.LATTICE_RELAXED, OL.INIT_KINETIC_GROUND, 12.5, 0.01, oracle.Schedule())
    ref2 = OL.evolve(F, mid, r, OL.LATTICE_RELAXED, 12.5, 0.01, 1250, oracle.Schedule())
    compare(lat, [F], [ref2], r, steps=2500)
    lat.close()


def test_initial_states_state_io_and_time_reversal():
    d, r = 3, 8
    for kind, okind in ((lattice.RELAXED, OL.LATTICE_RELAXED), (lattice.CHAIN, OL.LATTICE_CHAIN)):
        lat = lattice.Lattice(d, r, kind)
        lat.reset_state(lattice.INIT_GROUND)
        want = OL.initial_state(d, r, okind, OL.INIT_KINETIC_GROUND)
        assert np.abs(lat.psi_fx[0].double().cpu().numpy()[..., 0] / 2 ** 29 - want.real).max() <= 2 ** -30
        assert int(lat.psi_fx[..., 1].abs().max()) == 0
        assert np.abs(lat.state()[0].cpu().numpy() - want).max() <= 1e-7
        lat.reset_state(lattice.INIT_UNIFORM)
        assert np.abs(lat.state()[0].cpu().numpy() - 9 ** -1.5).max() <= 1e-8
        Q, b = workloads.box_qp(41, d)
        lat.set_qp(Q[None], b[None])
        lat.set_schedule(qhd.Schedule())
        # a state of the caller's own, loaded through set_state, evolved, and back
        rng = np.random.default_rng(3)
        z = rng.standard_normal((1,) + (r + 1,) * d) + 1j * rng.standard_normal((1,) + (r + 1,) * d)
        z /= np.linalg.norm(z)
        lat.set_state(torch.from_numpy(z.astype(np.complex64)).cuda())
        psi0 = lat.state()[0].cpu().numpy().astype(np.complex128)
        lat.evolve(5.0, 0.01)
        ref = OL.evolve(OL.qp_potential(Q, b, r), z[0], r, okind, 0.0, 0.01, 500, oracle.Schedule())
        got = lat.state()[0].cpu().numpy()
        assert 0.5 * np.abs(np.abs(got) ** 2 - np.abs(ref) ** 2).sum() <= TV_MAX
        lat.evolve(-5.0, -0.01)
        # back to psi0 up to a global phase (each step adds a pseudo-random one)
        back = lat.state()[0].cpu().numpy().astype(np.complex128)
        assert abs(abs(np.vdot(psi0, back)) - 1.0) <= 1e-6
        assert np.abs(np.abs(back) ** 2 - np.abs(psi0) ** 2).max() <= 1e-7
        bad = torch.zeros((1,) + (r + 1,) * d, dtype=torch.complex64, device="cuda")
        bad[0, 1, 2, 3] = 3.0                   # not representable
        with pytest.raises(qhd.QHDError):
            lat.set_state(bad)
        big = torch.full((1,) + (r + 1,) * d, 0.5, dtype=torch.complex64, device="cuda")   # norm^2 = 182
        with pytest.raises(qhd.QHDError):
            lat.set_state(big)
        assert int(lat.psi_fx.abs().max()) == 0
        lat.close()


def test_full_size_sampled_instances():
    """The benchmark's launch configuration and instances (bench.py --workload
    simqhd, rank 0: 256 instances of the 5-d, r = 8 Sim-QHD problem, seeds
    0..255, sigma ~ U(0.5, 2) from seed 7): two sampled instances against the oracle."""
    d, r, B, T, dt = 5, 8, 256, 10.0, 0.01
    qps = [workloads.box_qp(i, d) for i in range(B)]
    sig = np.random.default_rng(7).uniform(0.5, 2.0, B)
    lat = lattice.Lattice(d, r, lattice.RELAXED, batch=B)
    lat.set_qp(np.stack([q for q, _ in qps]), np.stack([b for _, b in qps]))
    lat.set_schedule([qhd.Schedule(c_chi=2 * s) for s in sig])
    lat.reset_state(lattice.INIT_GROUND)
    lat.evolve(T, dt)
    prob = torch.empty((B, *lat.shape), dtype=torch.float32, device="cuda")
    obs = lat.observables(prob=prob)
    for i in (0, B - 1):
        F = OL.qp_potential(*qps[i], r)
        ref = oracle_run(F, r, OL.LATTICE_RELAXED, OL.INIT_KINETIC_GROUND, T, dt, oracle.Schedule(c_chi=2 * sig[i]))
        o = OL.observables(F, ref, r)
        assert 0.5 * np.abs(prob[i].double().cpu().numpy() - o.prob).sum() <= TV_MAX
        assert abs(obs[i].e_f - o.e_f) <= EF_MAX * max(abs(o.e_f), 1e-3 * (F.max() - F.min()))
    assert max(abs(o.norm - 1) for o in obs) <= NORM_MAX
    lat.close()


def test_error_paths():
    lat = lattice.Lattice(2, 4, lattice.RELAXED)
    with pytest.raises(qhd.QHDError) as e:
        lat.evolve(1.0, 0.1)                # no potential / schedule yet
    assert e.value.status == 3
    with pytest.raises(qhd.QHDError):
        lat.reset_state(7)
    lat.set_potential(torch.zeros(25, dtype=torch.float64, device="cuda"))
    lat.set_schedule(qhd.Schedule())
    for T, dt in [(1.0, 0.3), (1.0, 0.0), (-1.0, 0.1)]:
        with pytest.raises(qhd.QHDError) as e:
            lat.evolve(T, dt)
        assert e.value.status == 1
    bad = torch.zeros(25, dtype=torch.float64, device="cuda")
    bad[3] = float("nan")
    with pytest.raises(qhd.QHDError):
        lat.set_potential(bad)
    with pytest.raises(qhd.QHDError) as e:     # the rejected potential discarded the loaded one
        lat.evolve(1.0, 0.1)
    assert e.value.status == 3
    lat.close()


def test_trajectory_records_equal_separate_runs_and_the_oracle():
    """E[F](t), P_succ(t), p_gap(t) and the norm every 50 steps in one call: the
    points equal the oracle's observables at those times, and the state at the
    end equals a plain evolve of the same length."""
    d, r = 3, 8
    Q, b = workloads.box_qp(51, d)
    F = OL.qp_potential(Q, b, r)
    lat = lattice.Lattice(d, r, lattice.RELAXED)
    lat.set_qp(Q[None], b[None])
    lat.set_schedule(qhd.Schedule())
    lat.reset_state(lattice.INIT_GROUND)
    traj = lat.evolve_trajectory(3.0, 0.01, 50, radius=0.2, gap=0.05).cpu().numpy()
    end = lat.state()[0].cpu().numpy()
    assert traj.shape == (6, 1, 4)
    psi = OL.initial_state(d, r, OL.LATTICE_RELAXED, OL.INIT_KINETIC_GROUND)
    for k in range(6):
        psi = OL.evolve(F, psi, r, OL.LATTICE_RELAXED, 0.5 * k, 0.01, 50, oracle.Schedule())
        o = OL.observables(F, psi, r, 0.2, 0.05)
        assert abs(traj[k, 0, 0] - 1.0) <= NORM_MAX
        assert abs(traj[k, 0, 1] - o.e_f) <= EF_MAX * max(abs(o.e_f), 1e-3 * np.ptp(F)), k
        assert abs(traj[k, 0, 2] - o.p_succ) <= TV_MAX and abs(traj[k, 0, 3] - o.p_gap) <= TV_MAX, k
    lat.reset_state(lattice.INIT_GROUND)
    lat.evolve(3.0, 0.01)
    plain = lat.state()[0].cpu().numpy().astype(np.complex128)
    # equal up to the pseudo-random global phase of the segment boundaries
    assert abs(abs(np.vdot(plain, end.astype(np.complex128))) - 1.0) <= 1e-6
    assert np.abs(np.abs(plain) ** 2 - np.abs(end) ** 2).max() <= 1e-7
    with pytest.raises(qhd.QHDError):
        lat.evolve_trajectory(1.0, 0.01, 30)          # 30 does not divide 100
    lat.close()
