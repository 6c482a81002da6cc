"""The FNO surrogate's CUDA kernels against the FP64 CPU reference (forward
values, and gradients against central finite differences of the reference
loss), its training, and what the trained network gains over an untrained one
on solver-generated data."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads
from oracle import fno as ref
from paper_2303_01471_gb300 import fno, surrogate

CFG = fno.FNOConfig(n=16, width=4, modes=3, layers=2, hidden=8, act_bf16=False)
SHAPE = ref.Shape(CFG.n, CFG.width, CFG.modes, CFG.layers, CFG.hidden)


def tiny_batch(seed, B=3, n=16):
    rng = np.random.default_rng(seed)
    x = np.arange(n) / n
    f = np.empty((B, n, n))
    for b in range(B):
        a, c = rng.uniform(0.5, 2, 2)
        f[b] = np.sin(2 * np.pi * (a * x[:, None] + rng.uniform())) + c * np.cos(2 * np.pi * x[None, :]) \
            + 0.3 * rng.standard_normal((n, n))
    sigma = rng.uniform(0.5, 2.0, B)
    z = rng.standard_normal((B, n, n))
    pt = np.exp(2 * z)
    pt /= pt.sum(axis=(1, 2), keepdims=True)
    return f, sigma, pt


def perturbed_params(cfg, seed):
    rng = np.random.default_rng(seed + 100)
    p = fno.init_params(cfg, seed).astype(np.float64)
    p += 0.05 * rng.standard_normal(p.shape)   # non-zero biases and asymmetric weights
    return p.astype(np.float32)


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def lay_name(lay, i):
    for name, (o, k) in lay.items():
        if o <= i < o + k:
            return name
    return "?"


def test_forward_matches_reference():
    f, sigma, _ = tiny_batch(0)
    params = perturbed_params(CFG, 1)
    net = fno.FNO(CFG, batch_max=4, params=torch.from_numpy(params))
    p = net.forward(dev(f, torch.float64), dev(sigma, torch.float32)).cpu().numpy()
    net.close()
    p_ref, _ = ref.forward(params.astype(np.float64), SHAPE, f, sigma)
    assert np.abs(p - p_ref).max() <= 2e-5 * p_ref.max(), np.abs(p - p_ref).max() / p_ref.max()
    assert np.allclose(p.sum(axis=(1, 2)), 1.0, atol=1e-5)


def test_gradients_match_finite_differences():
    f, sigma, pt = tiny_batch(1)
    params = perturbed_params(CFG, 2)
    net = fno.FNO(CFG, batch_max=4, train=True, params=torch.from_numpy(params))
    loss = net.loss_grad(dev(f, torch.float64), dev(sigma, torch.float32), dev(pt, torch.float32))
    g = net.grad.cpu().numpy().astype(np.float64)
    net.close()
    p64 = params.astype(np.float64)
    assert loss == pytest.approx(ref.loss(p64, SHAPE, f, sigma, pt), rel=1e-5)
    lay = fno.param_layout(CFG)
    rng = np.random.default_rng(5)
    idx = []
    for name, (o, k) in lay.items():
        if name == "_total":
            continue
        idx += list(o + rng.choice(k, size=min(k, 6), replace=False))
    g_fd = ref.fd_gradient(p64, SHAPE, f, sigma, pt, idx, h=1e-5)
    scale = np.abs(g_fd).max()
    err = np.abs(g[idx] - g_fd)
    assert (err <= 2e-3 * np.abs(g_fd) + 2e-4 * scale).all(), \
        [(lay_name(lay, i), g[i], gf) for i, gf, e in zip(idx, g_fd, err) if e > 2e-3 * abs(gf) + 2e-4 * scale]


def test_bf16_activations_stay_close():
    f, sigma, _ = tiny_batch(2)
    cfg16 = fno.FNOConfig(**{**CFG.__dict__, "act_bf16": True})
    params = perturbed_params(CFG, 3)
    net = fno.FNO(cfg16, batch_max=4, params=torch.from_numpy(params))
    p = net.forward(dev(f, torch.float64), dev(sigma, torch.float32)).cpu().numpy()
    net.close()
    p_ref, _ = ref.forward(params.astype(np.float64), SHAPE, f, sigma)
    tv = 0.5 * np.abs(p - p_ref).sum(axis=(1, 2))
    assert (tv <= 5e-3).all(), tv


def test_tensor_core_forward_matches_reference():
    """Width 32 with BF16 activations runs the layer outputs and the projection on
    the tensor cores (BF16 MMA, FP32 accumulation); against the FP64 reference and
    against the FP32-activation (SIMT) path on the same parameters."""
    n = 64
    cfg = fno.FNOConfig(n=n, width=32, modes=16, layers=4, hidden=128, act_bf16=True)
    shape = ref.Shape(n, 32, 16, 4, 128)
    f, sigma, _ = tiny_batch(5, B=3, n=n)
    params = perturbed_params(cfg, 6)
    p_ref, _ = ref.forward(params.astype(np.float64), shape, f, sigma)
    out = {}
    for bf16 in (True, False):
        net = fno.FNO(fno.FNOConfig(**{**cfg.__dict__, "act_bf16": bf16}), batch_max=4,
                      params=torch.from_numpy(params))
        out[bf16] = net.forward(dev(f, torch.float64), dev(sigma, torch.float32)).cpu().numpy()
        net.close()
    tv_tc = 0.5 * np.abs(out[True] - p_ref).sum(axis=(1, 2))
    tv_32 = 0.5 * np.abs(out[False] - p_ref).sum(axis=(1, 2))
    print(f"TV vs FP64 reference: tensor-core BF16 {tv_tc}, FP32 SIMT {tv_32}")
    assert (tv_32 <= 1e-5).all(), tv_32
    assert (tv_tc <= 1e-2).all(), tv_tc
    assert np.allclose(out[True].sum(axis=(1, 2)), 1.0, atol=1e-5)


def test_tensor_core_gradients_match_the_fp32_path():
    """The BF16 training path (tensor-core forward, layer-input and projection
    backward, axis-1 DFT stages) against the FP32-activation SIMT path on the same
    parameters and data: every parameter block's gradient agrees to BF16 accuracy."""
    n = 32
    cfg = fno.FNOConfig(n=n, width=32, modes=16, layers=2, hidden=128, act_bf16=True)
    f, sigma, pt = tiny_batch(7, B=3, n=n)
    params = perturbed_params(cfg, 8)
    grads = {}
    for bf16 in (True, False):
        net = fno.FNO(fno.FNOConfig(**{**cfg.__dict__, "act_bf16": bf16}), batch_max=4, train=True,
                      params=torch.from_numpy(params))
        net.loss_grad(dev(f, torch.float64), dev(sigma, torch.float32), dev(pt, torch.float32))
        grads[bf16] = net.grad.cpu().numpy().astype(np.float64)
        net.close()
    worst = {}
    total = np.linalg.norm(grads[False])
    for name, (o, k) in fno.param_layout(cfg).items():
        if k == 0:
            continue
        g16, g32 = grads[True][o:o + k], grads[False][o:o + k]
        if name == "p2_b":
            # the output bias shifts every logit alike and the softmax ignores such a
            # shift: its exact gradient is zero, both paths leave only rounding
            assert np.abs(g16).max() <= 1e-4 * total and np.abs(g32).max() <= 1e-4 * total, (g16, g32)
            continue
        worst[name] = np.linalg.norm(g16 - g32) / max(np.linalg.norm(g32), 1e-30)
    print("relative gradient difference, BF16 tensor-core vs FP32:", {k: f"{v:.1e}" for k, v in worst.items()})
    assert max(worst.values()) <= 5e-2, worst


def test_adam_steps_reduce_the_loss():
    f, sigma, pt = tiny_batch(3, B=4)
    net = fno.FNO(CFG, batch_max=4, train=True, seed=4)
    args = (dev(f, torch.float64), dev(sigma, torch.float32), dev(pt, torch.float32))
    first = net.loss_grad(*args)
    for _ in range(60):
        net.loss_grad(*args, want_loss=False)
        net.adam(lr=1e-2)
    last = net.loss_grad(*args)
    net.close()
    assert last < 0.7 * first, (first, last)


def test_error_paths():
    import ctypes
    lib = fno._lib()
    net = fno.FNO(CFG, batch_max=2, train=False, seed=0)
    f = torch.zeros((3, 16, 16), dtype=torch.float64, device="cuda")
    s = torch.ones(3, dtype=torch.float32, device="cuda")
    with pytest.raises(Exception):
        net.forward(f, s)          # batch above batch_max
    st = lib.qhd_fno_loss_grad(net.h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(s.data_ptr()),
                               ctypes.c_void_p(f.data_ptr()), 2, ctypes.c_void_p(f.data_ptr()), None)
    assert st == 3                 # no training buffers
    net.close()


def test_surrogate_with_fallback_against_the_solver_alone():
    """What the trained surrogate gains over the method without it.  Solver-generated
    data (64^2, wells / Rastrigin, sigma ~ U(0.5, 2), T = 10, dt = 0.01), a short
    training, then on held-out instances: the surrogate's TV against the solver,
    the fallback set (TV > 1e-2: the solver reruns those instances) and the
    device time of (a) the solver alone and (b) surrogate inference plus the
    solver on the fallback set.  The gain is (a)/(b); with the fallback rate the
    measured TV distribution gives, the pipeline is slower than the solver alone
    (gain < 1).  Training must still cut the held-out TV well below the untrained
    network's and the uniform guess's."""
    n, ntr, nte = 64, 4096, 256
    spec = [("wells" if i % 2 == 0 else "rastrigin", 700000 + i) for i in range(ntr + nte)]
    f, sig = workloads.batch_fast_on_device(spec, (n, n), "cuda", K=8)
    sigma = torch.tensor(sig, dtype=torch.float32, device="cuda")
    p = surrogate.solver_distributions(f, sig, 10.0, 0.01)
    cfg = fno.FNOConfig(n=n, width=16, modes=8, layers=4, hidden=64, act_bf16=True)
    net = fno.FNO(cfg, batch_max=64, train=True, seed=7)
    te = slice(ntr, ntr + nte)
    tv0 = surrogate.tv_distance(surrogate.predict(net, f[te], sigma[te], 64), p[te]).mean().item()
    surrogate.train(net, f[:ntr], sigma[:ntr], p[:ntr], epochs=15, batch=32, lr=2e-3)

    def device_ms(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    fte, ste, sig_te = f[te].contiguous(), sigma[te].contiguous(), sig[ntr:ntr + nte]
    ms_solver, _ = device_ms(lambda: surrogate.solver_distributions(fte, sig_te, 10.0, 0.01))
    ms_net, pred = device_ms(lambda: surrogate.predict(net, fte, ste, 64))
    tv = surrogate.tv_distance(pred, p[te])
    fallback = (tv > 1e-2).nonzero().flatten()
    rate = fallback.numel() / nte
    if fallback.numel():
        idx = fallback.tolist()
        ffb = fte[fallback].contiguous()
        ms_fb, _ = device_ms(lambda: surrogate.solver_distributions(ffb, [sig_te[i] for i in idx], 10.0, 0.01))
    else:
        ms_fb = 0.0
    gain = ms_solver / (ms_net + ms_fb)
    uniform = torch.full_like(p[te], 1.0 / (n * n))
    tv_u = surrogate.tv_distance(uniform, p[te]).mean().item()
    net.close()
    print(f"surrogate TV mean {tv.mean().item():.3f} median {tv.median().item():.3f} (untrained {tv0:.3f}, uniform "
          f"{tv_u:.3f}); fallback rate {rate:.2f}; solver {ms_solver:.1f} ms, surrogate {ms_net:.1f} ms + fallback "
          f"{ms_fb:.1f} ms: gain {gain:.2f}")
    assert tv.mean().item() < 0.6 * tv0 and tv.mean().item() < 0.6 * tv_u
    if rate > 0.5:
        assert gain < 1.0, gain      # the surrogate does not pay for itself at this fallback rate
    assert ms_net < ms_solver        # inference alone is faster than the solver
