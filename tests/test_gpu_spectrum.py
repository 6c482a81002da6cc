"""The QHD Hamiltonian on the GPU and its lowest eigenpairs (Lanczos with full
reorthogonalisation) against the FP64 oracle's operator and ARPACK eigenvalues,
the harmonic-oscillator closed form, the paper's Levy semi-classical ratio, and
the probability spectrum of an evolved state."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
import workloads
from paper_2303_01471_gb300 import qhd


def make_sim(f, lo=0.0, hi=1.0, sched=None, kinetic=None):
    sim = qhd.QHD(f.shape, lo=lo, hi=hi)
    sim.set_potential(f)
    sim.set_schedule(sched or qhd.Schedule())
    if kinetic is not None:
        sim.set_kinetic(kinetic)
    sim.reset_state()
    return sim


@pytest.mark.parametrize("kinetic", [qhd.KINETIC_SPECTRAL, qhd.KINETIC_FD2])
@pytest.mark.parametrize("shape", [(64,), (32, 64), (8, 16, 32)], ids=lambda s: "x".join(map(str, s)))
def test_apply_hamiltonian_matches_oracle(shape, kinetic):
    inst = workloads.gaussian_wells(21, shape, K=4)
    sim = make_sim(inst.f, hi=2.0, kinetic=kinetic)
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
    t = 0.7
    got = sim.apply_hamiltonian(torch.from_numpy(x).cuda(), t).cpu().numpy()
    sim.close()
    a, b = oracle.schedule_ab(oracle.Schedule(), t)
    want = oracle.apply_h(inst.f, x.astype(np.complex128), a, b, hi=2.0, kinetic=kinetic)
    assert np.max(np.abs(got - want)) <= 2e-5 * np.abs(want).max()


def test_lowest_eigenvalues_match_arpack():
    inst = workloads.gaussian_wells(22, (64, 64), K=8)
    t = 2.0
    sim = make_sim(inst.f)
    ev, rs, ov = sim.lowest_eigenpairs(t, k=4, m=400)
    sim.close()
    a, b = oracle.schedule_ab(oracle.Schedule(), t)
    want = oracle.lowest_eigs(inst.f, a, b, 4)
    scale = np.abs(want).max()
    assert np.allclose(ev, want, rtol=0, atol=2e-5 * scale), (ev, want)
    assert (rs <= 1e-3 * scale).all(), rs


def test_harmonic_oscillator_levels():
    n, L = 128, 24.0
    x = -L / 2 + np.arange(n) * L / n
    om = 1.1
    f = 0.5 * om ** 2 * x ** 2
    a, b = 0.8, 1.7
    sched = qhd.Schedule(kind=qhd.SCHED_TABLE, ts=np.array([-1e9, 1e9]), phis=np.log([a, a]), chis=np.log([b, b]))
    sim = make_sim(f, lo=-L / 2, hi=L / 2, sched=sched)
    ev, rs, _ = sim.lowest_eigenpairs(0.0, k=4, m=100)
    sim.close()
    want = np.sqrt(a * b) * om * (np.arange(4) + 0.5)
    assert np.allclose(ev, want, rtol=2e-5), (ev, want)


def test_paper_levy_semiclassical_ratio_on_gpu():
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_levy_energy_ratio.json")))
    om1 = np.sqrt((np.pi ** 2 + 1 + 10 * np.sin(1.0) ** 2) / 8)
    om2 = np.sqrt(gold["hessian_eigenvalue_2"])
    n, L = 64, 24.0
    x = -L / 2 + np.arange(n) * L / n
    X1, X2 = np.meshgrid(x, x, indexing="ij")
    f = 0.5 * om1 ** 2 * X1 ** 2 + 0.5 * om2 ** 2 * X2 ** 2
    sched = qhd.Schedule(kind=qhd.SCHED_TABLE, ts=np.array([-1e9, 1e9]), phis=np.zeros(2), chis=np.zeros(2))
    sim = make_sim(f, lo=-L / 2, hi=L / 2, sched=sched)
    ev, rs, _ = sim.lowest_eigenpairs(0.0, k=2, m=400)
    sim.close()
    assert abs(ev[1] / ev[0] - gold["semiclassical_ratio"]) <= 0.5 * 10.0 ** -gold["printed_digits"] + 1e-5


def test_probability_spectrum_of_an_evolved_state():
    """After QHD evolution the state sits mostly in the lowest levels of H(T);
    the overlaps are a sub-distribution (sum <= 1) and match the oracle's
    eigenvectors' overlaps with the oracle's state."""
    inst = workloads.gaussian_wells(23, (64, 64), K=8)
    sim = make_sim(inst.f)
    sim.evolve(5.0, 0.01)
    ev, rs, ov, vecs = sim.lowest_eigenpairs(5.0, k=3, m=400, vectors=True)
    sim.close()
    assert 0.0 <= ov.sum() <= 1.0 + 1e-5
    psi_o = oracle.evolve(inst.f, oracle.uniform_state(inst.shape), 0.0, 0.01, 500, oracle.Schedule())
    a, b = oracle.schedule_ab(oracle.Schedule(), 5.0)
    vals, V = oracle.lowest_eigs(inst.f, a, b, 3, return_vectors=True)
    gap = np.diff(vals).min()
    if gap > 1e-3 * np.abs(vals).max():   # well-separated levels: overlaps are unique
        ov_o = np.abs(V.T @ psi_o.ravel()) ** 2
        assert np.allclose(ov, ov_o, atol=1e-3), (ov, ov_o)
    assert np.allclose(ev, vals, rtol=0, atol=1e-4 * np.abs(vals).max())


def test_energy_ratio_approaches_the_semiclassical_limit():
    """Eq. (semiclassical_ratio) on a synthetic wells instance: along a QHD run
    the energy ratio, measured from the bottom of the well, approaches
    (omega_1 + 3 omega_2) / (omega_1 + omega_2) from the Hessian of f at its
    minimiser (measured: 0.1-0.6% at T = 10 on three seeds)."""
    from paper_2303_01471_gb300 import spectrum
    out = spectrum.energy_ratio_trajectory((128, 128), 2, [2.0, 7.5], m=400, k=2)
    r = out["trajectory"][-1]["E1_over_E0"]
    assert abs(r / out["semiclassical_ratio"] - 1) < 0.01, (r, out["semiclassical_ratio"])
    # the approach is from far away: early in the run the ratio is elsewhere
    assert abs(out["trajectory"][0]["E1_over_E0"] / out["semiclassical_ratio"] - 1) > 0.05
