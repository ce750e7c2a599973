"""The spectral heat current on the GPU (nep_md_set_shc / nep_md_get_shc /
nep_shc_spectrum) against the oracle: the same HNEMD trajectory of the
461-atom replica, its sampled per-atom virials and velocities correlated by
the oracle (orc_shc, pinned in test_oracle_shc.py).

Tolerance: K[tau] is an average of J-like sums W_i . v_i; the heat current
itself matches the oracle within TOL_W times 1.5 sum |v| (test_gpu_md.py),
so K gets the same bound."""
import numpy as np
import pytest

from gpu_util import f32_exact, soa
from paper_2107_08119_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL_W = 1e-4
FE = [2e-3, -1e-3, 5e-4]


@pytest.fixture(scope="module")
def N():
    from paper_2107_08119_gb300 import build
    build.build()
    from paper_2107_08119_gb300 import nep
    return nep


def _run(N, steps, n_lags, every, split=None):
    import torch
    pos, vel, box, z = inputs.config3(cells=(4, 4, 4))
    model = N.NEP(z)
    md = N.MD(model, len(pos), box, inputs.MASS_SI)
    md.set_hnemd(FE)
    md.set_shc(n_lags, every)
    p, v = soa(pos), soa(vel)
    heat = torch.zeros(steps, 3, dtype=torch.float64, device="cuda")
    for a, b in (split or [(0, steps)]):
        md.step(p, v, b - a, 1.0, None, heat[a:b])
    K, ns = md.shc()
    md.sync_status()
    out = (K.cpu().numpy(), ns, heat.cpu().numpy())
    md.close()
    model.close()
    return out


@pytest.mark.parametrize("every,n_lags", [(1, 8), (3, 5)])
def test_shc_matches_oracle(N, orc, every, n_lags):
    steps = 30
    K, ns, J = _run(N, steps, n_lags, every)
    pos, vel, box, z = inputs.config3(cells=(4, 4, 4))
    _, vo, _, J_o, W_h, v_h = orc.md_record(orc.NepHyper(), f32_exact(z), pos, vel, box, inputs.MASS_SI, 1.0,
                                           steps, fe=FE)
    sel = np.arange(0, steps, every)
    assert ns == len(sel)
    Ko = orc.shc(W_h[sel], v_h[sel], n_lags) / (len(sel) - np.arange(n_lags))[:, None]
    vmax = np.abs(vo).sum() * 1.5
    assert np.abs(K - Ko).max() <= TOL_W * vmax, (np.abs(K - Ko).max(), TOL_W * vmax)
    # lag 0 is the mean heat current of the sampled steps (the same FP32 terms)
    assert np.allclose(K[0], J[sel].mean(axis=0), rtol=1e-9, atol=1e-12 * vmax)


def test_shc_split_calls_and_fewer_samples_than_lags(N):
    K1, n1, _ = _run(N, 12, 20, 2)
    K2, n2, _ = _run(N, 12, 20, 2, split=[(0, 5), (5, 12)])
    assert n1 == n2 == 6
    assert np.array_equal(K1, K2)
    assert np.all(K1[6:] == 0.0) and np.any(K1[5] != 0.0)


def test_spectrum_matches_oracle(N, orc):
    import torch
    rng = np.random.default_rng(11)
    K = rng.normal(size=(40, 3))
    om = np.linspace(0.0, 0.3, 17)
    for window in (False, True):
        out = N.shc_spectrum(torch.tensor(K, device="cuda"), 2.0, torch.tensor(om, device="cuda"), 0.5,
                             window).cpu().numpy()
        want = orc.shc_spectrum(K, 2.0, om, 0.5, window)
        assert np.allclose(out, want, rtol=1e-12, atol=1e-12)


def test_shc_errors(N):
    pos, vel, box, z = inputs.config3(cells=(4, 4, 4))
    model = N.NEP(z)
    md = N.MD(model, len(pos), box, inputs.MASS_SI)
    with pytest.raises(N.NepError):
        md.shc()                      # not switched on
    for bad in ((-1, 1), (4, 0)):
        with pytest.raises(N.NepError) as e:
            md.set_shc(*bad)
        assert e.value.code == -1
    md.set_shc(4, 1)
    md.set_shc(0)                     # off again
    with pytest.raises(N.NepError):
        md.shc()
    md.close()
    model.close()


def test_quantum_correction_matches_oracle(N):
    """nep_shc_quantum (h / sinh h)^2 against the oracle's x^2 e^x / (e^x - 1)^2
    (pinned in test_oracle_shc.py) over x from 0 through the small-h branch
    to underflow, negative frequencies included; and kappa_spectrum's quantum
    option is the classical spectrum times that factor at hbar / (k_B T)."""
    import torch

    from oracle import oracle as orc
    rng = np.random.default_rng(9)
    x = np.concatenate([[0.0, 1e-9, 1e-5, 1.99e-4, 2.01e-4], np.linspace(0.01, 80.0, 300), [700.0, 1500.0, 4000.0]])
    omega = np.concatenate([x, -x[1:20]]) / 0.37
    spec = rng.normal(size=(len(omega), 3))
    want = orc.shc_quantum(spec, omega, 0.37)
    got = N.shc_quantum(torch.tensor(spec, device="cuda"), torch.tensor(omega, device="cuda"), 0.37).cpu().numpy()
    assert np.allclose(got, want, rtol=1e-13, atol=1e-300)
    assert np.array_equal(got[0], spec[0])
    with pytest.raises(N.NepError):
        N.shc_quantum(torch.tensor(spec, device="cuda"), torch.tensor(omega, device="cuda"), float("nan"))
    # through kappa_spectrum at 300 K: 0.5-40 THz, window on
    K = torch.tensor(np.exp(-np.arange(200) / 30.0)[:, None] * [1.0, 0.5, 0.2], device="cuda")
    nu = torch.linspace(0.0, 40.0, 81, dtype=torch.float64, device="cuda")
    cl = N.kappa_spectrum(K, 2.0, nu, 300.0, 2e4, 1e-4).cpu().numpy()
    qc = N.kappa_spectrum(K, 2.0, nu, 300.0, 2e4, 1e-4, quantum=True).cpu().numpy()
    # the units nep_kappa_spectrum applies: omega = 2 pi nu in rad/fs for nu in
    # THz; W / (m K) per eV / (A fs K); per THz of nu (1e-3 ps per fs)
    hbar_ev_fs, kb_ev = 0.6582119569, 8.617333262e-5
    w = 2 * np.pi * nu.cpu().numpy() * 1e-3
    scale = 2.0 / (300.0 * 2e4 * 1e-4) * 1.602176634e6 * 1e-3
    assert np.allclose(cl, orc.shc_spectrum(K.cpu().numpy(), 2.0, w, scale, window=True), rtol=1e-12, atol=0)
    xq = hbar_ev_fs / (kb_ev * 300.0)
    assert np.allclose(qc, orc.shc_quantum(cl, w, xq), rtol=1e-12, atol=0)
    assert (np.abs(qc[1:]) < np.abs(cl[1:])).all()  # the factor is below 1 for w > 0


@pytest.mark.parametrize("n", [1, 7, 256, 1000, 4099])
def test_running_hnemd_estimate_matches_oracle(N, n):
    """nep_hnemd_kappa (segment sums, then their prefix) against the oracle's
    sums in step order (pinned in test_oracle_shc.py), ragged lengths
    included; and the W/(m K) conversion of hnemd_kappa."""
    import torch

    from oracle import oracle as orc
    J = np.random.default_rng(n).normal(1.0, 3.0, size=(n, 3))
    got = N.hnemd_kappa(torch.tensor(J, device="cuda"), 0, 0, 0, scale=0.37).cpu().numpy()
    assert np.allclose(got, orc.hnemd_kappa(J, 0.37), rtol=1e-12, atol=1e-15)
    k = N.hnemd_kappa(torch.tensor(J, device="cuda"), 300.0, 2.0e4, 1e-4).cpu().numpy()
    assert np.allclose(k, orc.hnemd_kappa(J, 1.602176634e6 / (300.0 * 2.0e4 * 1e-4)), rtol=1e-12)
    with pytest.raises(N.NepError):
        N.hnemd_kappa(torch.zeros(0, 3, dtype=torch.float64, device="cuda"), 300.0, 1.0, 1.0)
