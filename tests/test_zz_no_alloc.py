"""qhd_observables_static: the observables entry point for callers that cannot
allocate device memory (e.g. their device memory is wholly owned by another
allocator, or they must not pay cudaMalloc's cost or its device
synchronisation).  Its scratch is a fixed array inside the library.

It is checked against the context-based qhd_observables on the same state, on
two calls in a row (the second call reuses the array the first one left
behind).  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads
from paper_2303_01471_gb300 import qhd

REL_TOL = 1e-12   # same kernels, same block counts: identical up to FP64 rounding order


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_static_scratch_observables_match_context_path():
    lib = qhd.load()
    shape, batch = (64, 128), 3
    insts = [workloads.make(fam, s, shape) for fam, s in [("wells", 21), ("rastrigin", 22), ("wells", 23)]]
    fb = np.stack([i.f for i in insts])
    sim = qhd.QHD(shape, batch=batch)
    sim.set_potential(fb)
    sim.set_schedule(qhd.Schedule())
    sim.reset_state()
    sim.evolve(2.0, 0.01)
    g = int(np.prod(shape))
    prob_ctx = torch.empty(batch * g, dtype=torch.float32, device="cuda")
    ref = sim.observables(0.1, prob=prob_ctx)

    f_dev = torch.from_numpy(fb).cuda()
    n = (ctypes.c_int64 * 2)(*shape)
    lo = (ctypes.c_double * 2)(0.0, 0.0)
    hi = (ctypes.c_double * 2)(1.0, 1.0)
    xs = np.array([o.x_star for o in ref], dtype=np.float64).ravel()
    stream = torch.cuda.current_stream()
    for call in range(2):
        out = torch.full((batch * 3,), float("nan"), dtype=torch.float64, device="cuda")
        prob = torch.full((batch * g,), -1.0, dtype=torch.float32, device="cuda")
        st = lib.qhd_observables_static(2, n, lo, hi, batch, _dptr(sim.psi), _dptr(f_dev),
                                        xs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0.1,
                                        _dptr(out), _dptr(prob), ctypes.c_void_p(stream.cuda_stream))
        assert st == qhd.QHD_OK, f"call {call}: status {st}"
        stream.synchronize()
        got = out.cpu().numpy().reshape(batch, 3)
        for b, o in enumerate(ref):
            assert got[b, 0] == pytest.approx(o.norm, rel=REL_TOL), (call, b)
            assert got[b, 1] == pytest.approx(o.e_f, rel=REL_TOL), (call, b)
            assert got[b, 2] == pytest.approx(o.p_succ, rel=REL_TOL, abs=1e-300), (call, b)
        assert torch.equal(prob, prob_ctx), call
    sim.close()


def test_static_scratch_rejects_sizes_beyond_its_limit():
    lib = qhd.load()
    n = (ctypes.c_int64 * 2)(8, 8)
    lo = (ctypes.c_double * 2)(0.0, 0.0)
    hi = (ctypes.c_double * 2)(1.0, 1.0)
    xs = np.zeros(3 * 33)
    fake = ctypes.c_void_p(0x10000000)  # never dereferenced: the size check fails first
    st = lib.qhd_observables_static(2, n, lo, hi, 33, fake, fake,
                                    xs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0.1,
                                    fake, None, None)
    assert st == 1
    n2 = (ctypes.c_int64 * 2)(2048, 8)
    st = lib.qhd_observables_static(2, n2, lo, hi, 1, fake, fake,
                                    xs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0.1,
                                    fake, None, None)
    assert st == 1
