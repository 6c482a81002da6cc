"""Pins of the FP64 CPU reference of the FNO surrogate (oracle/fno.py): its
spectral convolution against numpy's real FFT routines and against exact
reconstruction, its loss at the optimum, and the parameter-count contract of
the library."""
import numpy as np
import pytest

from oracle import fno as ref


def test_spectral_conv_matches_masked_real_fft():
    """SC = irfft2( R^T . (rfft2 v restricted to the retained modes) ), per channel
    pair, with numpy's own transforms as an independent route."""
    rng = np.random.default_rng(0)
    B, n, C, M = 2, 16, 3, 4
    v = rng.standard_normal((B, n, n, C))
    R = rng.standard_normal((2 * M, M, C, C)) + 1j * rng.standard_normal((2 * M, M, C, C))
    got = ref.spectral_conv(v, R, M)
    Vf = np.fft.rfft2(v, axes=(1, 2))                 # (B, n, n/2+1, C)
    kx = ref.retained_kx(n, M)
    Wf = np.zeros_like(Vf)
    for q, k in enumerate(kx):
        for ky in range(M):
            Wf[:, k, ky, :] = Vf[:, k, ky, :] @ R[q, ky]
    want = np.fft.irfft2(Wf, s=(n, n), axes=(1, 2))
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_identity_weights_reproduce_band_limited_fields():
    """With R = identity on every retained mode, SC reproduces any real field whose
    spectrum lies inside the retained modes (fixes the signs, the 1/n^2 and the
    factor 2 of the half spectrum).  kx = n - M is left out: its partner +M is not
    retained, so a real field cannot carry it in the ky = 0 column."""
    rng = np.random.default_rng(1)
    n, C, M = 16, 2, 5
    spec = np.zeros((1, n, n // 2 + 1, C), dtype=complex)
    for k in ref.retained_kx(n, M)[:M].tolist() + ref.retained_kx(n, M)[M + 1:].tolist():
        for ky in range(M):
            spec[0, k, ky] = rng.standard_normal(C) + 1j * rng.standard_normal(C)
    v = np.fft.irfft2(spec, s=(n, n), axes=(1, 2))
    R = np.zeros((2 * M, M, C, C), dtype=complex)
    R[:, :, np.arange(C), np.arange(C)] = 1.0
    u = ref.spectral_conv(v, R, M)
    assert np.abs(u - v).max() <= 1e-12 * np.abs(v).max()
    # a field outside the retained modes is removed entirely
    w = np.cos(2 * np.pi * (n // 2 - 1) * np.arange(n) / n)[None, None, :, None] * np.ones((1, n, 1, C))
    assert np.abs(ref.spectral_conv(w, R, M)).max() <= 1e-12


def test_features_and_loss_definitions():
    rng = np.random.default_rng(2)
    f = rng.standard_normal((2, 8, 8)) * 3 + 1
    q = ref.features(f, np.array([0.5, 2.0]))
    assert np.allclose(q[..., 0].mean(axis=(1, 2)), 0, atol=1e-12)
    assert np.allclose(q[..., 0].std(axis=(1, 2)), 1, atol=1e-12)
    assert q[1, 3, 5, 1] == 2.0 and q[0, 3, 5, 2] == 3 / 8 and q[0, 3, 5, 3] == 5 / 8
    p = rng.uniform(0.1, 1, (2, 8, 8))
    p /= p.sum(axis=(1, 2), keepdims=True)
    assert ref.kl_loss(p, p) == pytest.approx(0.0, abs=1e-15)
    p2 = np.roll(p, 1, axis=1)
    assert ref.kl_loss(p, p2) > 0


def test_reference_forward_is_a_distribution_and_fd_is_consistent():
    s = ref.Shape(n=8, width=2, modes=2, layers=2, hidden=4)
    rng = np.random.default_rng(3)
    npar = 0
    for k in [4 * 2, 2] + [2 * 2 * 2 * 2 * 2 * 2, 4, 2] * 2 + [8, 4, 4, 1]:
        npar += k + (k & 1)
    params = rng.standard_normal(npar) * 0.3
    f = rng.standard_normal((2, 8, 8))
    sig = np.array([1.0, 1.5])
    p, _ = ref.forward(params, s, f, sig)
    assert np.allclose(p.sum(axis=(1, 2)), 1.0, atol=1e-14) and (p > 0).all()
    pt = np.roll(p, 2, axis=2)
    # central differences at two step sizes agree (the loss is smooth)
    g1 = ref.fd_gradient(params, s, f, sig, pt, [0, 20, npar - 2], h=1e-5)
    g2 = ref.fd_gradient(params, s, f, sig, pt, [0, 20, npar - 2], h=1e-6)
    assert np.allclose(g1, g2, rtol=1e-5, atol=1e-9)


def test_library_param_count_matches_documented_layout():
    from paper_2303_01471_gb300 import fno
    for cfg in [fno.FNOConfig(), fno.FNOConfig(n=16, width=4, modes=3, layers=2, hidden=8, act_bf16=False)]:
        lay = fno.param_layout(cfg)
        assert fno.param_count(cfg) == lay["_total"][0]
        params = np.zeros(lay["_total"][0])
        w = ref.unpack(params, ref.Shape(cfg.n, cfg.width, cfg.modes, cfg.layers, cfg.hidden))
        assert w[f"R{cfg.layers - 1}"].shape == (2 * cfg.modes, cfg.modes, cfg.width, cfg.width)
    bad = [fno.FNOConfig(n=12), fno.FNOConfig(width=3), fno.FNOConfig(width=64), fno.FNOConfig(modes=65),
           fno.FNOConfig(n=16, modes=9), fno.FNOConfig(hidden=7), fno.FNOConfig(layers=0)]
    for cfg in bad:
        assert fno.param_count(cfg) == 0, cfg
