"""Parity of the tensor-core DFT transform (dense DFT GEMMs on FP16 operands,
FP32 accumulation, the project's tcgen05 kernel) with the FP64 oracle, through
the C ABI.  No library GEMM is called (library_call_count stays 0).

The fixed-point form (10 products) is held to the tolerances of the FFT path:
TV(|psi|^2) <= 1e-4, relative E[f] error <= 1e-5, and the norm within the FP32
floor.  Its integer slices have level sums FP32 holds exactly, so the
truncation of the tensor cores' own accumulation never enters.

The block-scaled FP16 hi/lo forms (3 products: the configured "hi-lo" form;
5 products: the DFT matrix to 32 bits) are exact per MMA as well; the tests
state what they reach over 1000 steps.  The DFT matrix has only n distinct
entries, so a fixed rounding of it is the same structured perturbation in every
transform of every step and its effect on the norm adds up coherently instead
of as a random walk: with 21-bit entries rounded once the norm fell by
1.4-2.6e-4 over 1000 steps, E[f] moved with it, TV reached 1.0-1.3e-4 (a CPU
emulation of the step split this into 2.4e-4 from the 21-bit matrix, 5e-7 from
a 32-bit one, 3.6e-5 from the FP32 accumulation of the per-MMA partials).  The
last slice is therefore re-rounded every step as floor(r + u) with a fresh
offset u: exact on average over steps, so its errors add as a random walk; the
3-product form then reaches TV 1.1-2.6e-5 and E[f] 0.4-1.05e-5.  The 5-product
form keeps a steady loss of ~1e-4 that the matrix's last slice does not
explain.  The 512^2 case is the batch shape of the tensor-core workload
(Gaussian wells K = 16, T = 10, dt = 0.01) on 8 of its instances.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
import workloads
from paper_2303_01471_gb300 import qhd

TV_TOL = 1e-4
EF_TOL = 1e-5
# Norm walk of the tensor-core forms over 1000 steps: the operands are re-split
# (rounded to FP16 slices or to 2^-28 of the instance maximum) four times a step,
# so it is wider than the FFT path's (measured up to 3.7e-6, fixed form).
TC_NORM_1K = 4e-6


def run_tc(fb, scheds, T, dt, products, split=qhd.SPLIT_STRANG, t0=None, pieces=1, transform=None):
    batch, shape = fb.shape[0], fb.shape[1:]
    sim = qhd.QHD(shape, batch=batch)
    sim.set_potential(fb)
    sim.set_schedule(scheds)
    sim.set_splitting(split)
    if transform is None or transform == qhd.TRANSFORM_TC_DFT:
        sim.set_transform(qhd.TRANSFORM_TC_DFT, products)
    sim.reset_state()
    if t0 is not None:
        sim.set_time(t0)
    for _ in range(pieces):
        sim.evolve(T / pieces, dt)
    obs = sim.observables(0.1)
    psi = sim.psi.cpu().numpy().astype(np.complex128)
    gemms, launches = sim.library_call_count(), sim.launch_count()
    sim.close()
    return psi, obs, gemms, launches


def errors(psi_g, obs_g, f, psi_o):
    psi_g = psi_g.reshape(psi_o.shape)
    ob = oracle.observables(f, psi_o, 0.1)
    tv = 0.5 * np.abs(np.abs(psi_g) ** 2 - ob.prob).sum()
    ef = abs(obs_g.e_f - ob.e_f) / max(abs(ob.e_f), 1e-3 * np.ptp(f))
    ov = np.vdot(psi_g.ravel(), psi_o.ravel())
    el = np.max(np.abs(psi_g * (ov / abs(ov)) - psi_o)) / np.abs(psi_o).max()
    return tv, ef, el, ob


def check(psi_g, obs_g, f, psi_o, steps, elementwise=True):
    tv, ef, el, ob = errors(psi_g, obs_g, f, psi_o)
    assert tv <= TV_TOL, f"TV {tv:.3e}"
    assert ef <= EF_TOL, f"E[f] rel err {ef:.3e}"
    assert abs(obs_g.norm - 1.0) <= TC_NORM_1K * max(1.0, math.sqrt(steps / 1000)), \
        f"norm drift {obs_g.norm - 1:.3e}"
    assert abs(obs_g.p_succ - ob.p_succ) <= 2 * TV_TOL
    assert tuple(obs_g.x_star[: f.ndim]) == tuple(ob.x_star[: f.ndim])
    if elementwise:
        assert el <= 2e-5 * math.sqrt(steps + 1), f"max |dpsi| {el:.3e}"
    return tv, ef


def short_batch(n):
    insts = [workloads.make(fam, s, (n, n), draw_sigma=True)
             for fam, s in [("wells", 21), ("rastrigin", 22), ("wells", 23)]]
    fb = np.stack([i.f for i in insts])
    scheds = [qhd.Schedule(c_chi=2.0 * i.sigma) for i in insts]
    return insts, fb, scheds


@pytest.mark.parametrize("n", [64, 128, 256, 512])
def test_tc_fixed_short_runs_own_schedules(n):
    """Three instances with their own f and potential scale sigma (shared kinetic table)."""
    insts, fb, scheds = short_batch(n)
    dt, steps = 0.01, 100
    psi, obs, gemms, launches = run_tc(fb, scheds, steps * dt, dt, 10)
    assert gemms == 0
    for b, inst in enumerate(insts):
        psi_o = oracle.evolve(inst.f, oracle.uniform_state((n, n)), 0.0, dt, steps,
                              oracle.Schedule(c_chi=2.0 * inst.sigma))
        check(psi[b], obs[b], inst.f, psi_o, steps)


# What the block-scaled forms reach (measured on GB300, see the module docstring):
# over 100 steps TV <= 1e-4 and |norm - 1| <= 9e-6, E[f] <= 1.2e-5.  Over 1000
# steps the 3-product form, whose last DFT-matrix slice is re-rounded with a fresh
# offset every step, reaches TV 1.1-2.6e-5, E[f] 0.4-1.05e-5 and a norm drift of
# either sign up to 1e-5 (128^2 and 512^2, two instances each; 1.1-1.3e-4, 1.4-2.6e-4
# and a steady loss of 1.4-2.6e-4 with the fixed rounding); the 5-product form
# keeps a steady loss of at most 1.4e-4.
BS_100 = {"tv": 1e-4, "ef": 2e-5, "norm": 1.5e-5}
# Pointwise error per sqrt(step) over 100 steps, relative to the largest amplitude.
# The 3-product form's re-rounded slice is a fresh perturbation every step; at
# n = 1024 (K = 2048) its pointwise effect after 100 steps measured 3.3e-4 (2e-4
# with the fixed rounding, whose coherent part instead grows to TV 1e-4 by 1000
# steps), while TV, E[f] and the norm stay within the bounds above.
BS_EL = {3: 4e-5, 5: 2e-5}
BS_1K = {3: {"tv": 5e-5, "ef": 3e-5, "norm": 3e-5}, 5: {"tv": 1e-4, "ef": 2e-4, "loss": 2e-4}}


@pytest.mark.parametrize("products", [3, 5])
@pytest.mark.parametrize("n", [64, 128, 256, 1024])
def test_tc_block_scaled_forms_100_steps(n, products):
    """The block-scaled hi/lo forms over 100 steps against the oracle, element by
    element (1024^2 is beyond the fixed form's range)."""
    insts, fb, scheds = short_batch(n)
    dt, steps = 0.01, 100
    psi, obs, gemms, _ = run_tc(fb, scheds, steps * dt, dt, products)
    assert gemms == 0
    for b, inst in enumerate(insts):
        psi_o = oracle.evolve(inst.f, oracle.uniform_state((n, n)), 0.0, dt, steps,
                              oracle.Schedule(c_chi=2.0 * inst.sigma))
        tv, ef, el, ob = errors(psi[b], obs[b], inst.f, psi_o)
        assert tv <= BS_100["tv"] and ef <= BS_100["ef"], (tv, ef)
        assert abs(obs[b].norm - 1.0) <= BS_100["norm"], obs[b].norm - 1.0
        assert el <= BS_EL[products] * math.sqrt(steps + 1), el
        assert tuple(obs[b].x_star[:2]) == tuple(ob.x_star[:2])


def block_scaled_1k(products, psi, obs, insts, psi_o):
    lim = BS_1K[products]
    for b, inst in enumerate(insts):
        tv, ef, _, ob = errors(psi[b], obs[b], inst.f, psi_o[b])
        drift = obs[b].norm - 1.0
        print(f"{products} products, instance {b}: TV {tv:.2e} E[f] {ef:.2e} norm - 1 {drift:+.2e}")
        if "loss" in lim:
            # the steady loss of the 5-product form: always a loss, bounded
            assert -lim["loss"] <= drift < 0.0, drift
        else:
            assert abs(drift) <= lim["norm"], drift
        assert tv <= lim["tv"] and ef <= lim["ef"], (tv, ef)
        assert tuple(obs[b].x_star[:2]) == tuple(ob.x_star[:2])


@pytest.mark.parametrize("products", [3, 5])
def test_tc_block_scaled_forms_128sq_1000_steps(products):
    insts = [workloads.gaussian_wells(s, (128, 128), K=8) for s in (0, 1)]
    psi_o = [oracle.evolve(i.f, oracle.uniform_state(i.shape), 0.0, 0.01, 1000, oracle.Schedule()) for i in insts]
    psi, obs, gemms, _ = run_tc(np.stack([i.f for i in insts]), qhd.Schedule(), 10.0, 0.01, products)
    assert gemms == 0
    block_scaled_1k(products, psi, obs, insts, psi_o)


def test_tc_own_kinetic_tables_and_chunks():
    """Per-instance kinetic weights (one kinetic table per instance) over several
    chunks of steps, evolved in two calls."""
    n = 64
    insts = [workloads.gaussian_wells(s, (n, n), K=8) for s in (31, 32)]
    fb = np.stack([i.f for i in insts])
    scheds = [qhd.Schedule(c_phi=1.5), qhd.Schedule(c_phi=2.5)]
    dt, steps = 0.01, 600
    psi, obs, gemms, _ = run_tc(fb, scheds, steps * dt, dt, 10, pieces=2)
    assert gemms == 0
    for b, inst in enumerate(insts):
        psi_o = oracle.evolve(inst.f, oracle.uniform_state((n, n)), 0.0, dt, steps,
                              oracle.Schedule(c_phi=scheds[b].c_phi))
        check(psi[b], obs[b], inst.f, psi_o, steps, elementwise=False)


def test_tc_lie_trotter_matches_oracle():
    n = 128
    inst = workloads.gaussian_wells(12, (n, n), K=4)
    psi, obs, _, _ = run_tc(inst.f[None], qhd.Schedule(), 0.5, 0.01, 10, split=qhd.SPLIT_LIE_TROTTER, t0=0.5)
    psi_o = oracle.evolve_trotter(inst.f, oracle.uniform_state((n, n)), 0.5, 0.01, 50)
    check(psi[0], obs[0], inst.f, psi_o, 50)


def test_tc_fixed_128sq_wells_1000_steps():
    """128^2 wells (K = 8), T = 10, dt = 0.01 against the oracle."""
    inst = workloads.gaussian_wells(0, (128, 128), K=8)
    psi_o = oracle.evolve(inst.f, oracle.uniform_state(inst.shape), 0.0, 0.01, 1000, oracle.Schedule())
    psi, obs, _, _ = run_tc(inst.f[None], qhd.Schedule(), 10.0, 0.01, 10)
    check(psi[0], obs[0], inst.f, psi_o, 1000, elementwise=False)


_C4 = {}


def c4_batch():
    if not _C4:
        insts = [workloads.gaussian_wells(s, (512, 512), K=16) for s in range(8)]
        oracle.set_threads(oracle.max_threads())
        psi_o = [oracle.evolve(i.f, oracle.uniform_state(i.shape), 0.0, 0.01, 1000, oracle.Schedule())
                 for i in insts]
        _C4["insts"], _C4["psi_o"] = insts, psi_o
    return _C4["insts"], _C4["psi_o"]


def test_tc_fixed_512sq_wells_batch_vs_oracle():
    """8 instances of the tensor-core batch shape: 512^2, Gaussian wells K = 16,
    T = 10, dt = 0.01 (1000 Strang steps)."""
    insts, psi_o = c4_batch()
    fb = np.stack([i.f for i in insts])
    psi, obs, gemms, _ = run_tc(fb, qhd.Schedule(), 10.0, 0.01, 10)
    assert gemms == 0
    for b, inst in enumerate(insts):
        check(psi[b], obs[b], inst.f, psi_o[b], 1000, elementwise=False)


@pytest.mark.parametrize("products", [3, 5])
def test_tc_block_scaled_512sq_wells_batch_vs_oracle(products):
    """The block-scaled forms (3 products: the configured FP16 hi-lo form) on the
    batch shape, 1000 steps, against the oracle: the accuracy they reach."""
    insts, psi_o = c4_batch()
    fb = np.stack([i.f for i in insts])
    psi, obs, gemms, _ = run_tc(fb, qhd.Schedule(), 10.0, 0.01, products)
    assert gemms == 0
    block_scaled_1k(products, psi, obs, insts, psi_o)


def test_tc_switch_back_to_fft():
    n = 64
    inst = workloads.rastrigin(5, (n, n))
    sim = qhd.QHD((n, n))
    sim.set_potential(inst.f)
    sim.set_schedule(qhd.Schedule())
    sim.set_transform(qhd.TRANSFORM_TC_DFT, 3)
    sim.set_transform(qhd.TRANSFORM_FFT)
    sim.reset_state()
    sim.evolve(0.5, 0.01)
    assert sim.library_call_count() == 0
    obs = sim.observables(0.1)
    psi = sim.psi.cpu().numpy().astype(np.complex128)
    sim.close()
    psi_o = oracle.evolve(inst.f, oracle.uniform_state((n, n)), 0.0, 0.01, 50, oracle.Schedule())
    check(psi[0], obs[0], inst.f, psi_o, 50)


def test_tc_error_paths():
    import ctypes
    lib = qhd.load()

    def ws(shape, batch=1, products=3):
        n = (ctypes.c_int64 * len(shape))(*shape)
        return int(lib.qhd_tc_workspace_bytes(len(shape), n, batch, products))

    assert ws((512, 512)) > 0 and ws((64, 64), products=3) > 0 and ws((512, 512), products=10) > 0
    assert ws((1024, 1024), products=3) > 0 and ws((1024, 1024), products=10) == 0
    for shape in [(32, 32), (64, 128), (2048, 2048), (64, 64, 64), (64,)]:
        assert ws(shape) == 0, shape
    assert ws((64, 64), products=4) == 0 and ws((64, 64), products=5) > 0
    for shape in [(32, 32), (64, 128), (8, 64, 64)]:
        sim = qhd.QHD(shape)
        with pytest.raises(qhd.QHDError) as e:
            sim.set_transform(qhd.TRANSFORM_TC_DFT, 3)
        assert e.value.status == 2
        # the library itself rejects the shape before it looks at the workspace
        st = lib.qhd_set_transform(sim.ctx, 1, 3, ctypes.c_void_p(sim.work_ptr), 1 << 30)
        assert st == 2, shape
        sim.close()
    sim = qhd.QHD((64, 64))
    for kind, products in [(7, 3), (qhd.TRANSFORM_TC_DFT, 4), (qhd.TRANSFORM_TC_DFT, 6), (qhd.TRANSFORM_TC_DFT, 7)]:
        st = lib.qhd_set_transform(sim.ctx, kind, products, ctypes.c_void_p(sim.work_ptr), 1 << 30)
        assert st == 1, (kind, products)
    need = ws((64, 64))
    buf = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    base = buf.data_ptr() + (-buf.data_ptr()) % 256
    assert lib.qhd_set_transform(sim.ctx, 1, 3, ctypes.c_void_p(base), need - 1) == 6
    assert lib.qhd_set_transform(sim.ctx, 1, 3, ctypes.c_void_p(base + 16), need) == 6
    assert lib.qhd_set_transform(sim.ctx, 1, 3, None, need) == 6
    assert lib.qhd_set_transform(sim.ctx, 1, 3, ctypes.c_void_p(base), need) == 0
    assert lib.qhd_set_transform(sim.ctx, 0, 0, None, 0) == 0
    sim.close()


def test_tc_fixed_with_fd_kinetic_operator():
    """The tensor-core form with the central-difference kinetic operator."""
    n = 128
    inst = workloads.gaussian_wells(15, (n, n), K=8)
    sim = qhd.QHD((n, n))
    sim.set_potential(inst.f)
    sim.set_schedule(qhd.Schedule())
    sim.set_kinetic(qhd.KINETIC_FD2)
    sim.set_transform(qhd.TRANSFORM_TC_DFT, 10)
    sim.reset_state()
    sim.evolve(1.0, 0.01)
    obs = sim.observables(0.1)
    psi = sim.psi.cpu().numpy().astype(np.complex128)
    sim.close()
    psi_o = oracle.evolve(inst.f, oracle.uniform_state((n, n)), 0.0, 0.01, 100, oracle.Schedule(),
                          kinetic=oracle.KINETIC_FD2)
    check(psi[0], obs[0], inst.f, psi_o, 100)
