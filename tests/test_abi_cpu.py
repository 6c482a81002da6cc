"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/qhd.h declares, sizes workspaces and rejects bad
arguments before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2303_01471_gb300 import qhd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points(header=None):
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h") and (header is None and fn != "qhd_probe.h" or fn == header):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(qhd_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    return qhd.load()


def test_library_exports_every_declared_symbol(lib):
    names = declared_entry_points()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(qhd.EXPORTS)


def test_workspace_bytes_valid_and_invalid(lib):
    assert qhd.workspace_bytes((128, 128)) > 128 * 128 * 12
    assert qhd.workspace_bytes((1024, 1024)) > 1024 * 1024 * 12
    assert qhd.workspace_bytes((256, 256, 256)) > 256 ** 3 * 12
    assert qhd.workspace_bytes((64,), batch=16) > 16 * 64 * 12
    for bad in [(3, 4), (2048,), (1,), (4, 4, 4, 4), ()]:
        n = (ctypes.c_int64 * max(1, len(bad)))(*bad)
        assert lib.qhd_workspace_bytes(len(bad), n, 1) == 0, bad
    n = (ctypes.c_int64 * 2)(8, 8)
    assert lib.qhd_workspace_bytes(2, n, 0) == 0
    assert lib.qhd_workspace_bytes(2, n, 65535) > 0 and lib.qhd_workspace_bytes(2, n, 65536) == 0


def test_init_rejects_bad_arguments_without_a_device(lib):
    ctx = ctypes.c_void_p()
    n = (ctypes.c_int64 * 2)(8, 8)
    lo = (ctypes.c_double * 2)(0.0, 0.0)
    hi = (ctypes.c_double * 2)(1.0, 1.0)
    bad_hi = (ctypes.c_double * 2)(1.0, 0.0)
    ws = lib.qhd_workspace_bytes(2, n, 1)
    fake = ctypes.c_void_p(0x10000000)  # never dereferenced: checks fail first
    assert lib.qhd_init_grid(None, 2, n, lo, hi, 1, fake, fake, ws, None) == 1
    assert lib.qhd_init_grid(ctypes.byref(ctx), 2, n, lo, bad_hi, 1, fake, fake, ws, None) == 1
    assert lib.qhd_init_grid(ctypes.byref(ctx), 2, n, lo, hi, 1, None, fake, ws, None) == 1
    # psi 8-byte but not 16-byte aligned: the passes copy it 16 bytes at a time
    assert lib.qhd_init_grid(ctypes.byref(ctx), 2, n, lo, hi, 1, ctypes.c_void_p(0x10000008), fake, ws, None) == 1
    assert lib.qhd_init_grid(ctypes.byref(ctx), 2, n, lo, hi, 1, fake, None, ws, None) == 6
    assert lib.qhd_init_grid(ctypes.byref(ctx), 2, n, lo, hi, 1, fake, fake, ws - 1, None) == 6
    assert lib.qhd_init_grid(ctypes.byref(ctx), 2, n, lo, hi, 1, fake,
                             ctypes.c_void_p(0x10000010), ws, None) == 6
    assert not ctx.value


def test_null_context_and_status_strings(lib):
    assert lib.qhd_evolve(None, 1.0, 0.1) == 1
    assert lib.qhd_reset_state(None) == 1
    assert lib.qhd_destroy(None) == 0
    assert lib.qhd_last_error(None) == b""
    assert lib.qhd_launch_count(None) == 0
    for s in range(7):
        assert lib.qhd_status_string(s)


def test_lattice_sizes_and_argument_checks_without_a_device(lib):
    from paper_2303_01471_gb300 import lattice
    lib = lattice._lib()
    ws = lib.qhd_lattice_workspace_bytes(5, 8, 4)
    assert ws > 4 * 9 ** 5 * 12
    for bad in [(0, 8, 1), (7, 8, 1), (2, 0, 1), (2, 17, 1), (2, 8, 0), (6, 16, 1 << 10), (1, 1, 65536)]:
        assert lib.qhd_lattice_workspace_bytes(*bad) == 0, bad
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(0x10000000)  # never dereferenced: checks fail first
    assert lib.qhd_lattice_init(None, 2, 8, 1, 1, fake, fake, ws, None) == 1
    assert lib.qhd_lattice_init(ctypes.byref(h), 2, 8, 2, 1, fake, fake, ws, None) == 1       # kind
    assert lib.qhd_lattice_init(ctypes.byref(h), 2, 8, 1, 1, None, fake, ws, None) == 1
    assert lib.qhd_lattice_init(ctypes.byref(h), 2, 8, 1, 1, ctypes.c_void_p(0x10000004), fake, ws, None) == 1
    small = lib.qhd_lattice_workspace_bytes(2, 8, 1)
    assert lib.qhd_lattice_init(ctypes.byref(h), 2, 8, 1, 1, fake, None, small, None) == 6
    assert lib.qhd_lattice_init(ctypes.byref(h), 2, 8, 1, 1, fake, fake, small - 1, None) == 6
    assert lib.qhd_lattice_init(ctypes.byref(h), 2, 8, 1, 1, fake, ctypes.c_void_p(0x10000010), small, None) == 6
    assert not h.value
    assert lib.qhd_lattice_evolve(None, 1.0, 0.1) == 1
    assert lib.qhd_lattice_reset_state(None, 0) == 1
    assert lib.qhd_lattice_destroy(None) == 0
    assert lib.qhd_lattice_last_error(None) == b""
    assert lib.qhd_lattice_launch_count(None) == 0


def test_probe_library_is_separate_and_rejects_null_output_without_a_device(lib):
    from paper_2303_01471_gb300 import probe
    plib = probe.load()
    for n in declared_entry_points("qhd_probe.h"):
        assert hasattr(plib, n), n
        assert not hasattr(lib, n), n      # not part of the simulator's ABI
    assert plib.qhd_probe_alu_rates(None) == 1


def test_bindings_reject_tensors_they_cannot_pass_as_raw_pointers():
    import torch
    from paper_2303_01471_gb300 import fno
    with pytest.raises(ValueError):
        qhd.need_tensor(torch.zeros(4, dtype=torch.float32), torch.float32, 4, "prob")      # host tensor
    with pytest.raises(ValueError):
        fno.FNO._need(torch.zeros((2, 8, 8), dtype=torch.float32), torch.float64, (2, 8, 8), "f")
