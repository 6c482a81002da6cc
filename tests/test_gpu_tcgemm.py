"""The tcgen05 GEMM of the tensor-core transform (qhd_tc_gemm_f16) against exact
and FP64 references: exact integer products (both accumulation modes), FP16
products against an FP64 sum of the same FP16 operands, the accumulation bias
of the hardware's long sums versus per-MMA partials added with round-to-nearest,
alpha / beta, and the argument checks."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_01471_gb300 import qhd


def ref64(A, B):
    return A.double().cpu().numpy() @ B.double().cpu().numpy().T


# one accumulation with 256 columns (or a multiple) runs the 256-wide tile, everything else the 128-wide one
@pytest.mark.parametrize("shape", [(128, 128, 64), (256, 256, 128), (384, 512, 1024), (192, 128, 128), (1, 128, 64),
                                   (200, 768, 192)])
@pytest.mark.parametrize("every", [True, False])
def test_exact_integer_products(shape, every):
    rows, n, k = shape
    g = torch.Generator(device="cuda").manual_seed(rows + n + k)
    A = torch.randint(-8, 9, (rows, k), device="cuda", generator=g).half()
    B = torch.randint(-8, 9, (n, k), device="cuda", generator=g).half()
    C, err = qhd.tc_gemm_f16(A, B, every_mma=every)
    torch.cuda.synchronize()
    assert int(err[0]) == 0
    ref = ref64(A, B)                       # |sums| <= 64 k < 2^24: exact in FP32 either way
    assert np.array_equal(C.double().cpu().numpy(), ref)


def test_full_range_integer_partials_are_exact():
    """Operands over the whole integer range of the block-scaled slices
    ([-1024, 1024]): each 16-term MMA sum (up to 2^24) comes back exactly, and
    the per-MMA partials are added in order with round-to-nearest FP32."""
    rows, n, k = 256, 256, 256
    g = torch.Generator(device="cuda").manual_seed(7)
    A = torch.randint(-1024, 1025, (rows, k), device="cuda", generator=g)
    B = torch.randint(-1024, 1025, (n, k), device="cuda", generator=g)
    A[:4] = 1024                            # rows and columns that reach the 2^24 bound
    B[:4] = 1024
    A[4:8] = -1024
    C, err = qhd.tc_gemm_f16(A.half(), B.half(), every_mma=True)
    torch.cuda.synchronize()
    assert int(err[0]) == 0
    a, b = A.cpu().numpy().astype(np.int64), B.cpu().numpy().astype(np.int64)
    acc = np.zeros((rows, n), dtype=np.float32)
    for j in range(0, k, 16):
        part = a[:, j:j + 16] @ b[:, j:j + 16].T
        assert np.abs(part).max() <= 2 ** 24
        acc = (acc + part.astype(np.float32)).astype(np.float32)
    assert np.array_equal(C.cpu().numpy(), acc)


def test_fp16_products_and_accumulation_bias():
    """Random FP16 operands: per-MMA partials added with round-to-nearest agree with
    the FP64 sum to FP32 rounding and carry no bias; the one long tensor-memory
    accumulation is biased towards zero (recorded, not required)."""
    rows, n, k = 1024, 512, 2048
    g = torch.Generator(device="cuda").manual_seed(7)
    A = (torch.rand((rows, k), device="cuda", generator=g) * 2 - 1).half()
    B = (torch.rand((n, k), device="cuda", generator=g) * 2 - 1).half()
    ref = ref64(A, B)
    res = {}
    for every in (True, False, "float"):
        C, err = qhd.tc_gemm_f16(A, B, every_mma=every)
        torch.cuda.synchronize()
        assert int(err[0]) == 0
        d = C.double().cpu().numpy() - ref
        scale = np.abs(ref).mean()
        res[every] = (np.abs(d).max() / scale, float(np.mean(d * np.sign(ref)) / scale))
    err_rn, bias_rn = res[True]
    err_hw, bias_hw = res[False]
    err_fl, bias_fl = res["float"]
    print(f"per-MMA partials: max rel err {err_rn:.2e}, bias {bias_rn:+.2e}; with the truncation correction: "
          f"{err_fl:.2e}, {bias_fl:+.2e}; one accumulation: max rel err {err_hw:.2e}, bias {bias_hw:+.2e}")
    assert err_rn <= 1e-5 and err_fl <= 1e-5, res
    # the hardware's long accumulation drifts towards zero by ~1e-9 K; per-MMA partials
    # leave only each MMA's truncation of its exact 16-term sum (measured -3.9e-8),
    # which the expected-truncation correction of the floating mode removes
    assert bias_hw < -5e-7, res
    assert abs(bias_rn) <= 1e-7 and abs(bias_rn) <= abs(bias_hw) / 20, res
    assert abs(bias_fl) <= abs(bias_rn) / 4, res


@pytest.mark.parametrize("every", [True, False])   # per-MMA groups: 128-wide tiles; one accumulation: 256-wide
def test_alpha_beta(every):
    rows, n, k = 256, 256, 256
    g = torch.Generator(device="cuda").manual_seed(3)
    A = torch.randint(-4, 5, (rows, k), device="cuda", generator=g).half()
    B = torch.randint(-4, 5, (n, k), device="cuda", generator=g).half()
    C0 = torch.randint(-100, 101, (rows, n), device="cuda", generator=g).float()
    C, err = qhd.tc_gemm_f16(A, B, C=C0.clone(), every_mma=every, alpha=0.5, beta=2.0)
    torch.cuda.synchronize()
    assert int(err[0]) == 0
    assert np.array_equal(C.double().cpu().numpy(), 0.5 * ref64(A, B) + 2.0 * C0.double().cpu().numpy())


def test_argument_checks():
    lib = qhd.load()
    A = torch.zeros((128, 64), dtype=torch.float16, device="cuda")
    B = torch.zeros((256, 64), dtype=torch.float16, device="cuda")
    C = torch.zeros((128, 256), dtype=torch.float32, device="cuda")
    e = torch.zeros(2, dtype=torch.int32, device="cuda")
    p = lambda t: t.data_ptr()
    ok = lib.qhd_tc_gemm_f16(p(A), p(B), p(C), 256, 128, 256, 64, 1, 1.0, 0.0, p(e), None)
    assert ok == qhd.QHD_OK
    bad = [(p(A), p(B), p(C), 256, 0, 256, 64, 1),       # no rows
           (p(A), p(B), p(C), 256, 128, 200, 64, 1),     # n_cols not a multiple of 128
           (p(A), p(B), p(C), 256, 128, 256, 48, 1),     # k not a multiple of 64
           (p(A), p(B), p(C), 100, 128, 256, 64, 1),     # ldc < n_cols
           (p(A), p(B), p(C), 256, 128, 256, 64, 3),     # mode
           (None, p(B), p(C), 256, 128, 256, 64, 1),
           (p(A) + 2, p(B), p(C), 256, 128, 256, 64, 1)]  # misaligned
    for args in bad:
        assert lib.qhd_tc_gemm_f16(*args, 1.0, 0.0, p(e), None) == qhd.QHD_ERR_INVALID_ARG, args
    torch.cuda.synchronize()
