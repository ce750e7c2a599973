"""Parity of the CUDA SNES path with the FP64 oracle: training-set
descriptors, per-member losses (Eqs. 29-34), the ranking, one SNES update
(Eqs. 35-39) and the Philox4x32-10 draws."""
import numpy as np
import pytest

from gpu_util import f32_exact
from paper_2107_08119_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL_U, TOL_F, TOL_W = 1e-6, 1e-4, 1e-4
# |dL_e| <= max per-atom energy error; |dL_f| <= RMS force error <= TOL_F;
# |dL_v| <= RMS per-atom virial error <= TOL_W (triangle inequality of the RMS)
LOSS_BOUND = {1: TOL_U, 2: TOL_F, 3: TOL_W}


@pytest.fixture(scope="module")
def N():
    from paper_2107_08119_gb300 import build
    build.build()
    from paper_2107_08119_gb300 import nep
    return nep


def labels(orc, teacher, structures):
    h = orc.NepHyper()
    E, F, W = [], [], []
    for s in structures:
        U, Fs, Ws = orc.efv(h, teacher, s["pos"], s["box"])
        Wt = Ws.sum(axis=0)
        E.append(U.sum())
        F.append(Fs)
        W.append([Wt[0, 0], Wt[1, 1], Wt[2, 2], Wt[0, 1], Wt[1, 2], Wt[2, 0]])
    return np.array(E), np.concatenate(F), np.array(W)


@pytest.fixture(scope="module")
def small_set(orc):
    structures = inputs.training_structures(12, seed_stream=21)
    rng = np.random.default_rng(99)
    teacher = f32_exact(inputs.random_z(1021, rng))
    E, F, W = labels(orc, teacher, structures)
    pop = f32_exact(rng.normal(0.0, 0.1, size=(8, 1021)))
    return structures, teacher, E, F, W, pop


def _check_losses(orc, gpu, structures, pop, E, F, W):
    h = orc.NepHyper()
    want = np.array([orc.loss(h, z, structures, E, F, W) for z in pop])
    for col, b in LOSS_BOUND.items():
        assert np.abs(gpu[:, col] - want[:, col]).max() <= b, (col, np.abs(gpu[:, col] - want[:, col]).max())
    assert np.allclose(gpu[:, 4:6], want[:, 4:6], rtol=1e-6)
    assert np.abs(gpu[:, 0] - want[:, 0]).max() <= sum(LOSS_BOUND.values()) + 1e-6
    return want


def test_dataset_descriptors(N, orc, small_set):
    import torch
    structures, teacher, E, F, W, pop = small_set
    model = N.NEP(teacher.astype(np.float32))
    ds = N.Dataset(model, structures, E, F, W)
    q = ds.descriptors().cpu().numpy()
    want = np.concatenate([orc.descriptors(orc.NepHyper(), s["pos"], s["box"]) for s in structures])
    assert np.abs(q - want).max() < 2e-5, np.abs(q - want).max()
    info = ds.info()
    assert info["atoms"] == sum(len(s["pos"]) for s in structures)
    ds.close()
    model.close()


def test_population_losses_fp32(N, orc, small_set):
    import torch
    structures, teacher, E, F, W, pop = small_set
    model = N.NEP(teacher.astype(np.float32))
    ds = N.Dataset(model, structures, E, F, W)
    zp = torch.tensor(pop, dtype=torch.float32, device="cuda")
    gpu = ds.evaluate(zp, N.PREC_FP32).cpu().numpy()
    want = _check_losses(orc, gpu, structures, pop, E, F, W)
    assert list(np.argsort(gpu[:, 0], kind="stable")) == list(np.argsort(want[:, 0], kind="stable"))
    # at the teacher the data terms vanish (to the force path's FP32 error)
    t = ds.evaluate(torch.tensor(teacher[None, :], dtype=torch.float32, device="cuda")).cpu().numpy()[0]
    assert t[1] <= TOL_U and t[2] <= TOL_F and t[3] <= TOL_W
    assert t[0] == pytest.approx(0.05 * t[4] + 0.05 * t[5], abs=3e-4)
    # bitwise reproducible
    again = ds.evaluate(zp, N.PREC_FP32).cpu().numpy()
    assert np.array_equal(gpu, again)
    ds.close()
    model.close()


def test_snes_update_matches_oracle(N, orc, small_set):
    """Same draws r_k (passed in), same losses ranking => same m, s."""
    import torch
    structures, teacher, E, F, W, pop = small_set
    model = N.NEP(teacher.astype(np.float32))
    ds = N.Dataset(model, structures, E, F, W)
    rng = np.random.default_rng(3)
    m0 = f32_exact(rng.uniform(-0.5, 0.5, 1021))
    s0 = np.full(1021, 0.1)
    r = f32_exact(rng.normal(size=(8, 1021)))
    snes = N.SNES(model, 8, m0, s0, seed=7)
    loss = torch.empty(8, N.LOSS_COLS, dtype=torch.float64, device="cuda")
    snes.step(ds, N.PREC_FP32, r=torch.tensor(r, dtype=torch.float32, device="cuda"), loss=loss)
    m1, s1, r_used, order = snes.state()
    zk = f32_exact(m0[None, :] + np.float32(0.1) * r.astype(np.float32))   # the GPU's FP32 population
    want_loss = _check_losses(orc, loss.cpu().numpy(), structures, zk, E, F, W)
    mo, so, oo = orc.snes_update(want_loss[:, 0], r, m0, s0)
    assert list(order.cpu().numpy()) == list(oo)
    assert np.allclose(m1.cpu().numpy(), mo, rtol=0, atol=2e-6)
    assert np.allclose(s1.cpu().numpy(), so, rtol=2e-6, atol=0)
    snes.close()
    ds.close()
    model.close()


def test_philox_draws_match_oracle(N, orc, small_set):
    import torch
    structures, teacher, E, F, W, pop = small_set
    model = N.NEP(teacher.astype(np.float32))
    ds = N.Dataset(model, structures, E, F, W)
    snes = N.SNES(model, 6, np.zeros(1021), np.full(1021, 0.1), seed=2107081194)
    for gen in range(2):
        snes.step(ds, N.PREC_FP32)
        _, _, r, _ = snes.state()
        want = orc.gaussian(2107081194, gen, 6 * 1021).reshape(6, 1021)
        assert np.allclose(r.cpu().numpy(), want, rtol=2e-5, atol=2e-5)
    snes.close()
    ds.close()
    model.close()


def test_bf16_generation_draws_while_packing(N, orc, small_set):
    """In BF16 mode a generation draws r, forms z = m + s r and packs the
    tensor-core records in one kernel: the draws are the FP32 generation's
    bits (the same Philox stream), and with m = 0 (z = s r exactly) the
    generation's losses are the bits of snes_evaluate_population on that z."""
    import torch
    structures, teacher, E, F, W, pop = small_set
    model = N.NEP(teacher.astype(np.float32))
    ds = N.Dataset(model, structures, E, F, W)
    s0 = np.full(1021, 0.1)
    a = N.SNES(model, 6, np.zeros(1021), s0, seed=2107081194)
    b = N.SNES(model, 6, np.zeros(1021), s0, seed=2107081194)
    la = torch.empty(6, N.LOSS_COLS, dtype=torch.float64, device="cuda")
    lb = torch.empty(6, N.LOSS_COLS, dtype=torch.float64, device="cuda")
    a.step(ds, N.PREC_FP32, loss=la)
    b.step(ds, N.PREC_BF16, loss=lb)
    ra = a.state()[2]
    rb = b.state()[2]
    assert torch.equal(ra, rb)
    z = (torch.tensor(s0, dtype=torch.float32, device="cuda")[None, :] * rb).contiguous()
    want = ds.evaluate(z, N.PREC_BF16)
    torch.cuda.synchronize()
    assert torch.equal(lb, want)
    assert torch.equal(la[:, 4:6], lb[:, 4:6])   # L_1, L_2: functions of z alone
    # the next generation's draws too (they do not depend on m and s)
    a.step(ds, N.PREC_FP32)
    b.step(ds, N.PREC_BF16)
    assert torch.equal(a.state()[2], b.state()[2])
    assert np.allclose(b.state()[2].cpu().numpy(), orc.gaussian(2107081194, 1, 6 * 1021).reshape(6, 1021),
                       rtol=2e-5, atol=2e-5)
    a.close()
    b.close()
    ds.close()
    model.close()


def test_config4_training_set_full_size(N, orc):
    """All 200 structures (uneven 32-256 atoms); four members, oracle losses."""
    import torch
    structures, teacher, pop = inputs.config4()
    teacher = f32_exact(teacher)
    E, F, W = labels(orc, teacher, structures)
    model = N.NEP(teacher.astype(np.float32))
    ds = N.Dataset(model, structures, E, F, W)
    sel = f32_exact(pop[[0, 17, 33, 49]])
    gpu = ds.evaluate(torch.tensor(sel, dtype=torch.float32, device="cuda"), N.PREC_FP32).cpu().numpy()
    _check_losses(orc, gpu, structures, sel, E, F, W)
    ds.close()
    model.close()
