"""Multicomponent weighting on the GPU (nep_set_species,
nep_dataset_create_species) against the oracle's (orc_*_z, pinned in
test_oracle_species.py): forces and virials, an MD trajectory, the SNES
losses and the force-loss gradient of a two-species set.

Species numbers of 0.8 and 1.3 keep the descriptors in the range of the
single-species tests, so the tolerances are theirs (the weight
sqrt(Z_i Z_j) is one correctly rounded FP32 square root of an exact product,
about 6e-8 relative)."""
import numpy as np
import pytest

from gpu_util import aos, f32_exact, soa, virial_aos
from paper_2107_08119_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL_U, TOL_F, TOL_W = 1e-6, 1e-4, 1e-4
ZA, ZB = 0.8, 1.3


@pytest.fixture(scope="module")
def N():
    from paper_2107_08119_gb300 import build
    build.build()
    from paper_2107_08119_gb300 import nep
    return nep


def _species(n, seed):
    return np.where(np.random.default_rng(seed).random(n) < 0.4, ZA, ZB)


def test_forces_and_virials_match_oracle(N, orc):
    pos, box, z = inputs.config1()
    Z = _species(len(pos), 1)
    model = N.NEP(z)
    model.set_species(Z)
    out = model.compute(soa(pos), box)
    U, F, W = orc.efv(orc.NepHyper(), f32_exact(z), pos, box, Z=Z)
    assert np.abs(out["e_atom"].cpu().numpy() - U).max() <= TOL_U
    assert np.abs(aos(out["force"]) - F).max() <= TOL_F
    assert np.abs(virial_aos(out["virial_atom"]) - W).max() <= TOL_W
    # the species matter, and one species of Z = 1 is the unweighted model bit for bit
    U1 = orc.efv(orc.NepHyper(), f32_exact(z), pos, box)[0]
    assert np.abs(U1 - U).max() > 1e-3
    model.set_species(np.ones(len(pos)))
    a = model.compute(soa(pos), box)
    model.set_species(None)
    b = model.compute(soa(pos), box)
    for k in ("e_atom", "force", "virial_atom"):
        assert np.array_equal(a[k].cpu().numpy(), b[k].cpu().numpy()), k
    model.close()


def test_md_trajectory_matches_oracle(N, orc):
    import torch
    pos, vel, box, z = inputs.config3(cells=(4, 4, 4))
    n = len(pos)
    Z = _species(n, 2)
    steps = 30
    model = N.NEP(z)
    model.set_species(Z)
    md = N.MD(model, n, box, inputs.MASS_SI)
    p, v = soa(pos), soa(vel)
    thermo = torch.zeros(steps, N.THERMO_COLS, dtype=torch.float64, device="cuda")
    heat = torch.zeros(steps, 3, dtype=torch.float64, device="cuda")
    md.step(p, v, steps, 1.0, thermo, heat)
    md.sync_status()
    po, vo, th_o, J_o, _, _ = orc.md_record(orc.NepHyper(), f32_exact(z), pos, vel, box, inputs.MASS_SI, 1.0, steps,
                                            Z=Z)
    th = thermo.cpu().numpy()
    assert np.abs(th[:, 0] - th_o[:, 0]).max() <= TOL_U * n
    assert np.abs(th[:, 1] - th_o[:, 1]).max() <= 1e-6 * n
    vmax = np.abs(vo).sum() * 1.5
    assert np.abs(heat.cpu().numpy() - J_o).max() <= TOL_W * vmax
    L = np.diag(box)
    dx = aos(p) - po
    dx -= L * np.round(dx / L)
    assert np.abs(dx).max() < 1e-6
    assert np.abs(aos(v) - vo).max() < 1e-7
    md.close()
    model.close()


def _labels(orc, teacher, structures, Z):
    h = orc.NepHyper()
    E, F, W = [], [], []
    off = 0
    for s in structures:
        na = len(s["pos"])
        U, Fs, Ws = orc.efv(h, teacher, s["pos"], s["box"], Z=Z[off:off + na])
        Wt = Ws.sum(axis=0)
        E.append(U.sum())
        F.append(Fs)
        W.append([Wt[0, 0], Wt[1, 1], Wt[2, 2], Wt[0, 1], Wt[1, 2], Wt[2, 0]])
        off += na
    return np.array(E), np.concatenate(F), np.array(W)


def test_training_set_losses_and_gradient_match_oracle(N, orc):
    import torch
    structures = inputs.training_structures(8, seed_stream=41)
    ntot = sum(len(s["pos"]) for s in structures)
    Z = _species(ntot, 3)
    rng = np.random.default_rng(41)
    teacher = f32_exact(inputs.random_z(1021, rng))
    pop = f32_exact(rng.normal(0.0, 0.1, size=(6, 1021)))
    E, F, W = _labels(orc, teacher, structures, Z)
    model = N.NEP(teacher.astype(np.float32))
    ds = N.Dataset(model, structures, E, F, W, species=Z)
    q = ds.descriptors().cpu().numpy()
    qo, off = [], 0
    for s in structures:
        na = len(s["pos"])
        qo.append(orc.descriptors(orc.NepHyper(), s["pos"], s["box"], Z=Z[off:off + na]))
        off += na
    qo = np.concatenate(qo)
    assert np.abs(q - qo).max() < 2e-5
    gpu = ds.evaluate(torch.tensor(pop, dtype=torch.float32, device="cuda"), N.PREC_FP32).cpu().numpy()
    want = np.array([orc.loss(orc.NepHyper(), zk, structures, E, F, W, Z=Z) for zk in pop])
    assert np.abs(gpu[:, 1] - want[:, 1]).max() <= TOL_U
    assert np.abs(gpu[:, 2] - want[:, 2]).max() <= TOL_F
    assert np.abs(gpu[:, 3] - want[:, 3]).max() <= TOL_W
    # force-loss gradient of one member
    g_o, lf_o = orc.force_loss_grad(orc.NepHyper(), pop[2], structures, F, Z=Z)
    lf = ds.force_loss(torch.tensor(pop[2], dtype=torch.float32, device="cuda")).item()
    g = ds.force_loss_backward().cpu().numpy()
    assert abs(lf - lf_o) <= TOL_F
    assert np.abs(g - g_o).max() <= 4.0 * (TOL_F / lf_o + 1e-5) * np.abs(g_o).max()
    model.sync_status()
    ds.close()
    model.close()


def test_species_errors(N):
    pos, box, z = inputs.config1()
    model = N.NEP(z)
    with pytest.raises(N.NepError) as e:
        model.set_species([1.0, -1.0])
    assert e.value.code == -1
    model.set_species(np.ones(10))
    with pytest.raises(N.NepError) as e:
        model.compute(soa(pos), box)      # species set for another atom count
    assert e.value.code == -1
    model.set_species(np.ones(len(pos)))
    with pytest.raises(N.NepError) as e:
        model.compute(soa(pos), box, plain=True)
    assert e.value.code == -8            # NEP_ERR_UNSUPPORTED
    model.close()
