"""Parity at the full sizes of the scale workload, in the launch configuration the
benchmark times: a 2-D 1024x1024 Rastrigin-type instance and a 3-D 256^3 Gaussian-well
instance (K = 32), T = 10, dt = 1e-3, the paper's schedule.

The oracle cannot run 10^4 steps of these grids in test time, so parity is checked
(a) element by element against the oracle over the first steps of the same run
(same kernels, same grid), (b) at full length against the oracle's stored results
(tests/golden/make_fullsize_reference.py: observables and the probability mass on
the points that hold all but ~1e-7 of it, which bounds the TV distance from above),
and (c) by invariants over the full 10^4 steps: the norm, and time reversal (10^4
steps forward then back returns psi0 up to a global phase).
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
import workloads
from paper_2303_01471_gb300 import qhd

TV_TOL = 1e-4
EF_TOL = 1e-5
NORM_TOL = 1e-6
# FP32 rounding of the state is a random walk of the norm once the systematic part
# is removed (the compensated product's order, qhd_device.cuh), and the zero-mode
# split (qhd_device.cuh) keeps the near-uniform early state's dominant Fourier value
# out of the butterflies, which removes most of the walk on fine meshes.  Measured
# spread (std) over 10^4 steps of dt = 1e-3: 1024^2 Rastrigin 0.9e-6 (12 seeds),
# 256^3 wells 0.35e-6 (3 seeds), 128^2 wells 1.8e-6 (64 seeds; a coarse mesh
# concentrates the late state on fewer points), each mean within 1.5 standard
# errors of 0 (test_norm_drift_is_unbiased_over_seeds).
NORM_WALK_10K = {"1024sq_rastrigin": 0.9e-6, "256cube_wells": 0.35e-6, "128sq": 1.8e-6}
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

CASES = {
    "1024sq_rastrigin": (lambda: workloads.rastrigin(0, (1024, 1024)), 20),
    "256cube_wells": (lambda: workloads.gaussian_wells(1, (256, 256, 256), K=32), 4),
}
_INST = {}


def inst(name):
    if name not in _INST:
        _INST[name] = CASES[name][0]()
    return _INST[name]


def align(psi_g, psi_o):
    ov = np.vdot(psi_g.ravel(), psi_o.ravel())
    return psi_g * (ov / abs(ov))


@pytest.mark.parametrize("name", list(CASES))
def test_fullsize_first_steps_match_oracle(name):
    ins = inst(name)
    nsteps = CASES[name][1]
    dt = 1e-3
    sim = qhd.QHD(ins.shape)
    sim.set_potential(torch.from_numpy(ins.f).cuda())
    sim.set_schedule(qhd.Schedule())
    sim.reset_state()
    sim.evolve(nsteps * dt, dt)
    obs = sim.observables(0.1)[0]
    psi_g = sim.psi.cpu().numpy()[0].astype(np.complex128)
    sim.close()
    psi_o = oracle.evolve(ins.f, oracle.uniform_state(ins.shape), 0.0, dt, nsteps, oracle.Schedule())
    ob = oracle.observables(ins.f, psi_o)
    p_g = np.abs(psi_g) ** 2
    tv = 0.5 * np.abs(p_g - ob.prob).sum()
    assert tv <= TV_TOL, tv
    assert abs(obs.e_f - ob.e_f) / max(abs(ob.e_f), 1e-3 * np.ptp(ins.f)) <= EF_TOL
    assert abs(obs.norm - 1.0) <= NORM_TOL
    assert abs(obs.p_succ - ob.p_succ) <= 2 * TV_TOL
    assert tuple(obs.x_star[: ins.f.ndim]) == tuple(ob.x_star[: ins.f.ndim])
    err = np.max(np.abs(align(psi_g, psi_o) - psi_o))
    assert err <= 2e-5 * np.abs(psi_o).max() * np.sqrt(nsteps + 1), err


_FULL = {}


def full_run(name):
    """10^4 steps forward (observables at T), then 10^4 steps back."""
    if name not in _FULL:
        ins = inst(name)
        sim = qhd.QHD(ins.shape)
        sim.set_potential(torch.from_numpy(ins.f).cuda())
        sim.set_schedule(qhd.Schedule())
        sim.reset_state()
        psi0 = sim.psi.clone()
        sim.evolve(10.0, 1e-3)
        obs = sim.observables(0.1)[0]
        p_T = (sim.psi.abs().double() ** 2).cpu().numpy().ravel()
        sim.evolve(-10.0, -1e-3)
        back = sim.observables(0.1)[0]
        p0 = (psi0.abs().double() ** 2).cpu().numpy()
        pb = (sim.psi.abs().double() ** 2).cpu().numpy()
        t, steps = sim.time()
        sim.close()
        _FULL[name] = (obs, back, 0.5 * np.abs(pb - p0).sum(), t, steps, p_T)
    return _FULL[name]


def golden(name):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_ref", os.path.join(GOLDEN, "make_fullsize_reference.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    path = mod.path_of(name)
    assert os.path.exists(path), f"missing {path}: run tests/golden/make_fullsize_reference.py {name}"
    ref = np.load(path)
    assert str(ref["key"]) == mod.case_key(name), "stale reference: the workload changed"
    return ref


@pytest.mark.parametrize("name", list(CASES))
def test_fullsize_10k_steps_match_oracle_reference(name):
    """The benchmark's instances after the full 10^4 steps against the FP64 oracle's
    stored results: TV (bounded from above through the stored mass), raw E[f],
    P_succ and x*."""
    ref = golden(name)
    obs, back, tv_back, t, steps, p_g = full_run(name)
    idx, p_o = ref["idx"], ref["p"]
    inside = p_g[idx]
    m_out_o, m_out_g = float(ref["mass_outside"]), p_g.sum() - inside.sum()
    l1_in = np.abs(inside - p_o).sum()
    # TV from above (S = the stored points, the rest as one unknown block) and from
    # below (the TV of the two distributions coarsened to S and its complement)
    tv_upper = 0.5 * (l1_in + m_out_g + m_out_o)
    tv_lower = 0.5 * (l1_in + abs(m_out_g - m_out_o))
    print(f"{name}: TV in [{tv_lower:.2e}, {tv_upper:.2e}], stored points {len(idx)}, mass outside {m_out_o:.2e}")
    if m_out_o <= 0.1 * TV_TOL:
        assert tv_upper <= TV_TOL, tv_upper
    else:
        # 256^3: the final state is spread (the stored 32768 points hold 99.7% of the
        # mass), so the stored subset certifies only the lower bound and the
        # agreement on the points it holds
        assert tv_lower <= 0.5 * TV_TOL, tv_lower
        assert l1_in <= TV_TOL * (1.0 - m_out_o), l1_in
    scale = max(abs(float(ref["e_f"])), 1e-3 * float(ref["f_ptp"]))
    assert abs(obs.e_f - float(ref["e_f"])) / scale <= EF_TOL, (obs.e_f, float(ref["e_f"]))
    assert abs(obs.p_succ - float(ref["p_succ"])) <= 2 * TV_TOL
    assert tuple(obs.x_star[: len(inst(name).shape)]) == tuple(ref["x_star"][: len(inst(name).shape)])


@pytest.mark.parametrize("name", list(CASES))
def test_fullsize_10k_steps_norm(name):
    """The benchmark's instances meet the stated norm bound (1e-6) after their 10^4
    steps; after the 10^4 steps back (twice the rounding) the norm is within 3
    standard deviations of the measured walk, scaled by sqrt(2)."""
    obs, back, tv_back, t, steps, _ = full_run(name)
    print(f"{name}: norm - 1 after 10^4 steps {obs.norm - 1:+.2e}, after the steps back {back.norm - 1:+.2e}")
    assert steps == 20000 and abs(t) < 1e-9
    assert abs(obs.norm - 1.0) <= NORM_TOL, obs.norm
    assert abs(back.norm - 1.0) <= max(NORM_TOL, 3 * NORM_WALK_10K[name] * np.sqrt(2)), back.norm


def test_norm_drift_is_unbiased_over_seeds():
    """Over many instances the 10^4-step norm drift has no systematic part: its mean
    is within 3 standard errors of 0 (before the fix of the compensated product's
    order every one of 32 instances drifted up, mean +1.1e-5, std 3.5e-6)."""
    seeds = list(range(32))
    fs = np.stack([workloads.gaussian_wells(s, (128, 128), K=8).f for s in seeds])
    sim = qhd.QHD((128, 128), batch=len(seeds))
    sim.set_potential(fs)
    sim.set_schedule(qhd.Schedule())
    sim.reset_state()
    sim.evolve(10.0, 1e-3)
    d = np.array([o.norm - 1.0 for o in sim.observables(0.1)])
    sim.close()
    se = d.std() / np.sqrt(len(d))
    assert abs(d.mean()) <= 3 * se + 1e-7, (d.mean(), se)
    assert np.abs(d).max() <= 4 * NORM_WALK_10K["128sq"], np.abs(d).max()
    assert 0.25 * len(d) <= (d > 0).sum() <= 0.75 * len(d), (d > 0).sum()


@pytest.mark.parametrize("name", list(CASES))
def test_fullsize_time_reversal(name):
    obs, back, tv_back, t, steps, _ = full_run(name)
    # the forward run moved far away from the uniform state ...
    assert obs.p_succ > 0.5
    # ... and the exact inverse map brings |psi|^2 back to uniform
    assert tv_back <= TV_TOL, tv_back


def test_paper_resolution_256sq_lie_trotter_and_strang():
    """The paper's second simulation setting: a 256^2 mesh, dt = 1e-3, T = 10
    (10^4 steps), run with the first-order formula exactly as printed
    (Eq. (prod_qhd), left-end-point coefficients) and with the Strang form.  Each
    matches its oracle; the two differ from each other by the splitting error,
    which the GPU path resolves (it is well above the GPU-oracle difference)."""
    ins = workloads.gaussian_wells(2, (256, 256), K=8)
    psi0 = oracle.uniform_state(ins.shape)
    oracle.set_threads(oracle.max_threads())
    res = {}
    for name, split in [("trotter", qhd.SPLIT_LIE_TROTTER), ("strang", qhd.SPLIT_STRANG)]:
        sim = qhd.QHD(ins.shape)
        sim.set_potential(ins.f)
        sim.set_schedule(qhd.Schedule())
        sim.set_splitting(split)
        sim.reset_state()
        sim.evolve(10.0, 1e-3)
        obs = sim.observables(0.1)[0]
        p_g = (sim.psi.abs().double() ** 2).cpu().numpy()[0]
        sim.close()
        if name == "trotter":
            psi_o = oracle.evolve_trotter(ins.f, psi0, 0.0, 1e-3, 10000)
        else:
            psi_o = oracle.evolve(ins.f, psi0, 0.0, 1e-3, 10000, oracle.Schedule())
        ob = oracle.observables(ins.f, psi_o)
        tv = 0.5 * np.abs(p_g - ob.prob).sum()
        scale = max(abs(ob.e_f), 1e-3 * np.ptp(ins.f))
        ef_raw = abs(obs.e_f - ob.e_f) / scale
        assert tv <= TV_TOL, (name, tv)
        assert ef_raw <= EF_TOL, (name, ef_raw)
        assert abs(obs.norm - 1.0) <= 3 * NORM_WALK_10K["128sq"], (name, obs.norm)
        res[name] = (p_g, ob.prob, tv)
    between = 0.5 * np.abs(res["trotter"][1] - res["strang"][1]).sum()
    assert between > 5 * max(res["trotter"][2], res["strang"][2]), (between, res["trotter"][2], res["strang"][2])
