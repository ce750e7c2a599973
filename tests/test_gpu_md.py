"""Parity of the CUDA MD step (velocity Verlet, skin-triggered rebuilds,
heat current) with the FP64 oracle's integrator from the same state."""
import numpy as np
import pytest

from gpu_util import aos, f32_exact, soa
from paper_2107_08119_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL_U, TOL_W = 1e-6, 1e-4


@pytest.fixture(scope="module")
def N():
    from paper_2107_08119_gb300 import build
    build.build()
    from paper_2107_08119_gb300 import nep
    return nep


def test_md_trajectory_thermo_and_heat_current(N, orc):
    """461-atom replica of the heat-transport workload, 40 steps of 1 fs:
    E_pot per step within n x 1e-6 eV, J per step within the bound implied
    by the virial tolerance, final positions close."""
    import torch
    pos, vel, box, z = inputs.config3(cells=(4, 4, 4))
    n, steps = len(pos), 40
    model = N.NEP(z)
    md = N.MD(model, n, box, inputs.MASS_SI)
    p, v = soa(pos), soa(vel)
    thermo = torch.zeros(steps, N.THERMO_COLS, dtype=torch.float64, device="cuda")
    heat = torch.zeros(steps, 3, dtype=torch.float64, device="cuda")
    md.step(p, v, steps, 1.0, thermo, heat)
    md.sync_status()
    po, vo, th_o, J_o = orc.md(orc.NepHyper(), f32_exact(z), pos, vel, box, inputs.MASS_SI, 1.0, steps)
    th = thermo.cpu().numpy()
    J = heat.cpu().numpy()
    assert np.abs(th[:, 0] - th_o[:, 0]).max() <= TOL_U * n
    assert np.abs(th[:, 1] - th_o[:, 1]).max() <= 1e-6 * n
    vmax = np.abs(vo).sum() * 1.5
    assert np.abs(J - J_o).max() <= TOL_W * vmax, np.abs(J - J_o).max()
    L = np.diag(box)
    dx = aos(p) - po
    dx -= L * np.round(dx / L)            # the GPU wraps positions at rebuilds
    assert np.abs(dx).max() < 1e-6
    assert np.abs(aos(v) - vo).max() < 1e-7
    md.close()
    model.close()


def test_md_rebuilds_and_energy_conservation(N):
    """The random-weight potential heats quickly, so the list is rebuilt on
    displacement; total energy stays conserved to second order in dt."""
    import torch
    pos, vel, box, z = inputs.config3(cells=(4, 4, 4))
    n = len(pos)
    res = {}
    for dt, steps in ((1.0, 200), (0.5, 400)):
        model = N.NEP(z)
        md = N.MD(model, n, box, inputs.MASS_SI)
        p, v = soa(pos), soa(vel)
        thermo = torch.zeros(steps, N.THERMO_COLS, dtype=torch.float64, device="cuda")
        md.step(p, v, steps, dt, thermo)
        md.sync_status()
        e = thermo[:, 0] + thermo[:, 1]
        res[dt] = (float((e - e[0]).abs().max()), md.rebuild_count())
        md.close()
        model.close()
    assert res[1.0][1] >= 3, res      # rebuilt on displacement
    ratio = res[1.0][0] / res[0.5][0]
    assert 2.5 < ratio < 6.0, res


def test_md_split_calls_equal_one_call(N):
    """k + k steps in two calls give bitwise the same state as 2k in one."""
    import torch
    pos, vel, box, z = inputs.config3(cells=(4, 4, 4))
    n = len(pos)
    model = N.NEP(z)
    outs = []
    for split in (False, True):
        md = N.MD(model, n, box, inputs.MASS_SI)
        p, v = soa(pos), soa(vel)
        if split:
            md.step(p, v, 25, 1.0)
            md.step(p, v, 25, 1.0)
        else:
            md.step(p, v, 50, 1.0)
        md.sync_status()
        outs.append((p.clone(), v.clone()))
        md.close()
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    model.close()


def _md_ext_compare(N, orc, steps, t0, tau, fe):
    import torch
    pos, vel, box, z = inputs.config3(cells=(4, 4, 4))
    n = len(pos)
    model = N.NEP(z)
    md = N.MD(model, n, box, inputs.MASS_SI)
    md.set_thermostat(t0, tau)
    md.set_hnemd(fe)
    p, v = soa(pos), soa(vel)
    thermo = torch.zeros(steps, N.THERMO_COLS, dtype=torch.float64, device="cuda")
    heat = torch.zeros(steps, 3, dtype=torch.float64, device="cuda")
    md.step(p, v, steps, 1.0, thermo, heat)
    md.sync_status()
    po, vo, th_o, J_o = orc.md_ext(orc.NepHyper(), f32_exact(z), pos, vel, box, inputs.MASS_SI, 1.0, steps,
                                   t0=t0, tau=tau, fe=fe)
    th = thermo.cpu().numpy()
    J = heat.cpu().numpy()
    assert np.abs(th[:, 0] - th_o[:, 0]).max() <= TOL_U * n
    assert np.abs(th[:, 1] - th_o[:, 1]).max() <= 1e-6 * n
    vmax = np.abs(vo).sum() * 1.5
    assert np.abs(J - J_o).max() <= TOL_W * vmax, np.abs(J - J_o).max()
    L = np.diag(box)
    dx = aos(p) - po
    dx -= L * np.round(dx / L)
    assert np.abs(dx).max() < 1e-6
    assert np.abs(aos(v) - vo).max() < 1e-7
    md.close()
    model.close()
    return th, J, aos(v)


def test_md_berendsen_thermostat_matches_oracle(N, orc):
    """Berendsen rescaling towards 900 K (tau = 20 fs), 40 steps from the
    461-atom replica: thermo, J and the final state follow the oracle."""
    _md_ext_compare(N, orc, 40, 900.0, 20.0, None)


def test_md_hnemd_matches_oracle_and_keeps_momentum(N, orc):
    """HNEMD driving F_e = (2e-3, -1e-3, 5e-4) /A with the thermostat on:
    the state follows the oracle's integrator and the total momentum stays
    zero (the mean driving force is removed)."""
    th, J, v = _md_ext_compare(N, orc, 40, 300.0, 50.0, [2e-3, -1e-3, 5e-4])
    # FP32 forces sum to zero only to rounding (|sum v| ~ 1e-9 A/fs here); an
    # unremoved mean driving force would add ~1e-4 A/fs per step
    assert np.abs(v.sum(axis=0)).max() < 1e-6


def test_md_thermostat_and_drive_errors(N):
    pos, box, z = inputs.config1()
    model = N.NEP(np.asarray(z, np.float32))
    md = N.MD(model, len(pos), box, inputs.MASS_SI)
    with pytest.raises(N.NepError):
        md.set_thermostat(-1.0, 10.0)
    md.set_thermostat(300.0, 0.0)     # off
    md.set_hnemd(None)                # off
    md.set_hnemd([0.0, 0.0, 0.0])     # off
    md.close()
    model.close()


@pytest.mark.parametrize("variant", ["nve", "nvt_hnemd"])
def test_step_graph_equals_eager_steps(N, variant):
    """Without phase timing a step replays the captured step graph (the list
    rebuild behind a conditional node); with it the kernels are launched one by
    one.  Both give bitwise the same trajectory, thermo rows and heat current,
    through list rebuilds."""
    import torch
    pos, vel, box, z = inputs.config3(cells=(4, 4, 4))
    n = len(pos)
    model = N.NEP(z)
    outs = []
    for eager in (False, True):
        md = N.MD(model, n, box, inputs.MASS_SI)
        if variant == "nvt_hnemd":
            md.set_thermostat(600.0, 30.0)
            md.set_hnemd([1e-3, 0.0, -5e-4])
        p, v = soa(pos), soa(vel)
        thermo = torch.zeros(60, N.THERMO_COLS, dtype=torch.float64, device="cuda")
        heat = torch.zeros(60, 3, dtype=torch.float64, device="cuda")
        model.profile(eager)
        md.step(p, v, 40, 1.0, thermo, heat)
        md.step(p, v, 20, 1.0, thermo[40:], heat[40:])   # another key: a recapture
        model.profile(False)
        model.profile_read()
        md.sync_status()
        outs.append((p.clone(), v.clone(), thermo.clone(), heat.clone(), md.rebuild_count()))
        md.close()
    for a, b in zip(outs[0][:4], outs[1][:4]):
        assert torch.equal(a, b)
    assert outs[0][4] == outs[1][4] and outs[0][4] >= 1
    model.close()
