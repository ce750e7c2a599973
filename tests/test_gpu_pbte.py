"""The split-hyperparameter model of the paper's PbTe potential (Table I:
radial cutoff 8 A with Chebyshev orders 0..12, angular cutoff 4 A with
radial orders 0..6 and l = 1..4, 41 descriptors, 40 neurons) on a
two-species rocksalt box weighted by sqrt(Z_i Z_j) (Sec. II.A), against the
FP64 oracle at the force path's bars: 1e-6 eV per site energy, 1e-4 eV/A per
force component, 1e-4 eV per virial component; and an MD trajectory."""
import numpy as np
import pytest

from gpu_util import aos, f32_exact, soa, virial_aos
from paper_2107_08119_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL_U, TOL_F, TOL_W = 1e-6, 1e-4, 1e-4


@pytest.fixture(scope="module")
def N():
    from paper_2107_08119_gb300 import build
    build.build()
    from paper_2107_08119_gb300 import nep
    return nep


def _hyper(N, max_neighbors=128):
    return N.Hyper(max_neighbors=max_neighbors, **inputs.PBTE_HYPER)


def _orc_hyper(orc):
    return orc.NepHyper(**inputs.PBTE_HYPER)


@pytest.mark.parametrize("cells,species", [((4, 4, 4), True), ((5, 4, 6), True), ((4, 4, 4), False)])
def test_split_model_matches_oracle(N, orc, cells, species):
    pos, vel, box, z, Z = inputs.config_pbte(cells)
    assert len(z) == 1721  # N_par of the PbTe model, Table I
    model = N.NEP(z, _hyper(N))
    if species:
        model.set_species(Z)
    out = model.compute(soa(pos), box)
    U, F, W = orc.efv(_orc_hyper(orc), f32_exact(z), pos, box, Z=Z if species else None)
    dU = np.abs(out["e_atom"].cpu().numpy() - U).max()
    dF = np.abs(aos(out["force"]) - F).max()
    dW = np.abs(virial_aos(out["virial_atom"]) - W).max()
    print(f"PbTe-like {cells}, species {species}: |dU| {dU:.2e}, |dF| {dF:.2e}, |dW| {dW:.2e}")
    assert dU <= TOL_U and dF <= TOL_F and dW <= TOL_W, (dU, dF, dW)
    assert abs(out["e_total"].item() - U.sum()) <= TOL_U * len(pos)
    model.close()


def test_split_model_md_trajectory(N, orc):
    """20 velocity-Verlet steps of 1 fs (one mass for both species) against
    the oracle integrator: site energies per step within n x 1e-6 eV, final
    positions within 1e-6 A."""
    import torch
    pos, vel, box, z, Z = inputs.config_pbte((4, 4, 4))
    n, steps = len(pos), 20
    model = N.NEP(z, _hyper(N, max_neighbors=160))
    model.set_species(Z)
    md = N.MD(model, n, box, inputs.MASS_PBTE)
    p, v = soa(pos), soa(vel)
    thermo = torch.zeros(steps, N.THERMO_COLS, dtype=torch.float64, device="cuda")
    md.step(p, v, steps, 1.0, thermo)
    md.sync_status()
    po, vo, th_o, _, _, _ = orc.md_record(_orc_hyper(orc), f32_exact(z), pos, vel, box, inputs.MASS_PBTE, 1.0,
                                          steps, Z=Z)
    assert np.abs(thermo.cpu().numpy()[:, 0] - th_o[:, 0]).max() <= TOL_U * n
    L = np.diag(box)
    dx = aos(p) - po
    dx -= L * np.round(dx / L)
    assert np.abs(dx).max() < 1e-6
    assert np.abs(aos(v) - vo).max() < 1e-7
    md.close()
    model.close()


def test_split_model_paths_without_kernels(N):
    """The training set, the plain comparator and the allocation-free call
    have kernels for the 32-descriptor model only: NEP_ERR_UNSUPPORTED."""
    pos, vel, box, z, Z = inputs.config_pbte((4, 4, 4))
    model = N.NEP(z, _hyper(N))
    with pytest.raises(N.NepError) as e:
        model.compute(soa(pos), box, plain=True)
    assert e.value.code == -8
    s = {"pos": pos[:64], "box": box}
    with pytest.raises(N.NepError) as e:
        N.Dataset(model, [s], np.zeros(1), np.zeros((64, 3)), np.zeros((1, 6)))
    assert e.value.code == -8
    model.compute(soa(pos), box)  # the handle still works
    model.close()
