"""Pins of the oracle's thermostatted / HNEMD integrator (orc_md_ext).

- With both extensions off it is the NVE integrator step for step.
- Berendsen with tau = dt sets the temperature to T0 after every step.
- HNEMD: the external forces F_i = F_e . W_i (mean removed) conserve the total
  momentum, and the total energy changes by the work they do,
  dH/dt = sum_i v_i . F_i^ext = F_e . J with J = sum_i W_i v_i (Eq. 7), so the
  gap between the energy change and the integrated F_e . J shrinks as dt^2.
  A transposed W_i (F = W_i F_e) would leave a gap that does not vanish."""
import numpy as np
import pytest

from paper_2107_08119_gb300 import inputs


@pytest.fixture(scope="module")
def state(orc):
    h = orc.NepHyper()
    pos, box, teacher, student = inputs.config5(orc.n_par(h))
    rng = np.random.default_rng(7)
    vel = inputs.maxwell_boltzmann(len(pos), 300.0, inputs.MASS_SI, rng)
    z = np.asarray(teacher, np.float32).astype(np.float64)
    return h, z, pos, vel, box


def test_extensions_off_is_nve(orc, state):
    h, z, pos, vel, box = state
    a = orc.md(h, z, pos, vel, box, inputs.MASS_SI, 1.0, 15)
    b = orc.md_ext(h, z, pos, vel, box, inputs.MASS_SI, 1.0, 15)
    c = orc.md_ext(h, z, pos, vel, box, inputs.MASS_SI, 1.0, 15, fe=[0.0, 0.0, 0.0])
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    for x, y in zip(a, c):
        assert np.array_equal(x, y)


def test_berendsen_with_tau_dt_holds_the_target(orc, state):
    h, z, pos, vel, box = state
    n = len(pos)
    for t0 in (150.0, 900.0):
        _, v, th, _ = orc.md_ext(h, z, pos, vel, box, inputs.MASS_SI, 1.0, 12, t0=t0, tau=1.0)
        target = 0.5 * (3 * n - 3) * inputs.KB_EV * t0
        assert np.allclose(th[:, 1], target, rtol=1e-12, atol=0)
        ek = 0.5 * inputs.MASS_SI * inputs.AMU_A2_FS2_EV * (v ** 2).sum()
        assert ek == pytest.approx(target, rel=1e-12)


def test_berendsen_relaxes_towards_the_target(orc, state):
    h, z, pos, vel, box = state
    n = len(pos)
    _, _, th, _ = orc.md_ext(h, z, pos, vel, box, inputs.MASS_SI, 1.0, 60, t0=1200.0, tau=10.0)
    T = 2 * th[:, 1] / ((3 * n - 3) * inputs.KB_EV)
    assert T[-1] > 900.0 and T[0] < T[-1]


def _energy_gap(orc, state, dt, steps, fe):
    h, z, pos, vel, box = state
    U0, F0, W0 = orc.efv(h, z, pos, box)
    J0 = np.einsum("iab,ib->a", W0, vel)
    E0 = U0.sum() + 0.5 * inputs.MASS_SI * inputs.AMU_A2_FS2_EV * (vel ** 2).sum()
    _, v, th, J = orc.md_ext(h, z, pos, vel, box, inputs.MASS_SI, dt, steps, fe=fe)
    Js = np.vstack([J0, J]) @ np.asarray(fe)
    work = np.cumsum(0.5 * dt * (Js[:-1] + Js[1:]))
    gap = np.abs(th[:, 0] + th[:, 1] - E0 - work).max()
    return gap, np.abs(work).max(), v


def test_hnemd_momentum_and_energy_balance(orc, state):
    fe = [5e-3, -2e-3, 1e-3]
    g1, w1, v1 = _energy_gap(orc, state, 0.5, 400, fe)
    g2, w2, v2 = _energy_gap(orc, state, 0.25, 800, fe)
    # total momentum stays zero (the mean external force is removed)
    assert np.abs(v1.sum(axis=0)).max() < 1e-12 and np.abs(v2.sum(axis=0)).max() < 1e-12
    # the work is not negligible, and the energy gap converges as dt^2
    assert w2 > 20 * g2
    assert 3.0 < g1 / g2 < 5.5, (g1, g2)
