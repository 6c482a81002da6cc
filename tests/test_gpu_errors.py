"""The error contract of the C ABI on a live context: a CUDA failure or a device
time-out makes the context sticky-failed until qhd_destroy, while argument and
workspace errors leave it usable.  Failures are injected on the host
(qhd_inject_failure skips the CUDA call and reports the error), so no GPU
fault is ever raised."""
import ctypes

import numpy as np
import pytest
import torch

import workloads
from paper_2303_01471_gb300 import qhd

pytestmark = pytest.mark.gpu

OK, INVALID, STATE, CUDA, TIMEOUT, WORKSPACE = 0, 1, 3, 4, 5, 6


def fresh(shape=(64, 64)):
    inst = workloads.gaussian_wells(0, shape, K=8)
    sim = qhd.QHD(shape)
    sim.set_potential(inst.f)
    sim.set_schedule(qhd.Schedule())
    sim.reset_state()
    return sim, inst


def calls_after_failure(sim, inst):
    """Status of every kind of entry point on a (possibly failed) context."""
    lib, ctx = sim.lib, sim.ctx
    out = (qhd._Obs * 1)()
    f = np.ascontiguousarray(inst.f)
    return {
        "evolve": lib.qhd_evolve(ctx, 0.1, 0.01),
        "observables": lib.qhd_observables(ctx, out, None, 0.1),
        "reset_state": lib.qhd_reset_state(ctx),
        "set_potential": lib.qhd_set_potential(ctx, f.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
        "set_time": lib.qhd_set_time(ctx, 0.0),
        "set_splitting": lib.qhd_set_splitting(ctx, 0),
    }


@pytest.mark.parametrize("kind", [CUDA, TIMEOUT])
@pytest.mark.parametrize("after", [1, 2])
def test_injected_failure_inside_evolve_is_sticky_until_destroy(kind, after):
    sim, inst = fresh()
    lib, ctx = sim.lib, sim.ctx
    assert lib.qhd_inject_failure(ctx, kind, after) == OK
    n0 = sim.launch_count()
    assert lib.qhd_evolve(ctx, 0.1, 0.01) == kind        # 10 steps: prep + one whole-run launch
    assert sim.launch_count() - n0 == after - 1           # the launches before the injected one ran
    assert b"injected" in lib.qhd_last_error(ctx)
    st = calls_after_failure(sim, inst)
    assert all(v == kind for v in st.values()), st
    assert lib.qhd_inject_failure(ctx, OK, 0) == kind    # even cancelling returns the sticky status
    torch.cuda.synchronize()                             # the enqueued work completed normally
    assert lib.qhd_destroy(ctx) == OK
    sim.ctx = None


def test_injected_failure_in_a_copy_of_set_potential():
    sim, inst = fresh()
    lib, ctx = sim.lib, sim.ctx
    assert lib.qhd_inject_failure(ctx, CUDA, 1) == OK
    f = np.ascontiguousarray(inst.f)
    assert lib.qhd_set_potential(ctx, f.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == CUDA
    assert lib.qhd_evolve(ctx, 0.1, 0.01) == CUDA
    assert lib.qhd_destroy(ctx) == OK
    sim.ctx = None


def test_cancelled_injection_and_argument_errors_leave_the_context_usable():
    sim, inst = fresh()
    lib, ctx = sim.lib, sim.ctx
    assert lib.qhd_inject_failure(ctx, CUDA, 2) == OK
    assert lib.qhd_inject_failure(ctx, OK, 0) == OK
    assert lib.qhd_inject_failure(ctx, 7, 1) == INVALID
    assert lib.qhd_inject_failure(ctx, CUDA, 0) == INVALID
    assert lib.qhd_evolve(ctx, 0.1, 0.03) == INVALID       # T/dt not an integer
    assert lib.qhd_observables(ctx, (qhd._Obs * 1)(), None, -1.0) == INVALID
    assert lib.qhd_set_splitting(ctx, 9) == INVALID
    sim.evolve(0.1, 0.01)
    o = sim.observables(0.1)[0]
    assert abs(o.norm - 1.0) < 1e-6 and o.steps_done == 10
    sim.close()


def test_transform_workspace_errors_are_not_sticky():
    shape = (64, 64)
    sim, inst = fresh(shape)
    lib, ctx = sim.lib, sim.ctx
    n = (ctypes.c_int64 * 2)(*shape)
    need = int(lib.qhd_tc_workspace_bytes(2, n, 1, 10))
    assert need > 0
    buf = torch.empty(need + 512, dtype=torch.uint8, device=sim.device)
    base = buf.data_ptr() + (-buf.data_ptr()) % 256
    assert lib.qhd_set_transform(ctx, qhd.TRANSFORM_TC_DFT, 10, None, need) == WORKSPACE
    assert lib.qhd_set_transform(ctx, qhd.TRANSFORM_TC_DFT, 10, ctypes.c_void_p(base + 16), need) == WORKSPACE
    assert lib.qhd_set_transform(ctx, qhd.TRANSFORM_TC_DFT, 10, ctypes.c_void_p(base), need - 1) == WORKSPACE
    assert lib.qhd_set_transform(ctx, qhd.TRANSFORM_TC_DFT, 4, ctypes.c_void_p(base), need) == INVALID
    assert lib.qhd_set_transform(ctx, 5, 10, ctypes.c_void_p(base), need) == INVALID
    sim.evolve(0.1, 0.01)                                  # still the FFT path, still healthy
    assert abs(sim.observables(0.1)[0].norm - 1.0) < 1e-6
    sim.close()
