"""The plain FP32 comparator (nep_compute_efv_plain: literal O(M^2) angular
sum of Eq. 13, Eqs. 24-25, unfused passes, no compensated sums) against the
FP64 oracle.

Tolerance: plain FP32 sums of up to ~M^2 = 256 angular terms (q_nl up to
~50) and of 32-term network dot products carry ~1e-6 relative rounding, i.e.
~1e-5 eV in a site energy of ~3 eV and ~1e-5 eV/A in forces; the test allows
1e-4 eV per site and 1e-3 eV/A (eV for per-atom virials), an order above
that.  The optimised path meets 1e-6 / 1e-4 / 1e-4 (test_gpu_force.py)."""
import numpy as np
import pytest

from gpu_util import aos, f32_exact, soa, virial_aos
from paper_2107_08119_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL_U, TOL_F, TOL_W = 1e-4, 1e-3, 1e-3


@pytest.fixture(scope="module")
def N():
    from paper_2107_08119_gb300 import build
    build.build()
    from paper_2107_08119_gb300 import nep
    return nep


def _check(N, orc, pos, box, z):
    model = N.NEP(z)
    out = model.compute(soa(pos), box, plain=True)
    U, F, W = orc.efv(orc.NepHyper(), f32_exact(z), pos, box)
    dU = np.abs(out["e_atom"].cpu().numpy() - U).max()
    dF = np.abs(aos(out["force"]) - F).max()
    dW = np.abs(virial_aos(out["virial_atom"]) - W).max()
    assert dU <= TOL_U and dF <= TOL_F and dW <= TOL_W, (dU, dF, dW)
    model.close()
    return dU, dF, dW


def test_plain_config1(N, orc):
    pos, box, z = inputs.config1()
    _check(N, orc, pos, box, z)


def test_plain_ragged_and_small_cells(N, orc):
    pos, vel, box, z = inputs.config3(cells=(4, 4, 4))
    _check(N, orc, pos, box, z)
    z = inputs.random_z(1021, np.random.default_rng(3))
    for s in inputs.training_structures(3, seed_stream=9):
        _check(N, orc, s["pos"], s["box"], z)


def test_plain_and_optimised_agree_at_full_size(N):
    """125,000 atoms: the two GPU forms agree within the plain form's bound."""
    pos, vel, box, z = inputs.config2()
    model = N.NEP(np.asarray(z, np.float32))
    p = soa(pos)
    a = model.compute(p, box)
    b = model.compute(p, box, plain=True)
    assert (a["e_atom"] - b["e_atom"]).abs().max().item() <= TOL_U
    assert (a["force"] - b["force"]).abs().max().item() <= TOL_F
    assert (a["virial_atom"] - b["virial_atom"]).abs().max().item() <= TOL_W
    model.close()


def test_plain_form_md_trajectory(N, orc):
    """MD with the plain FP32 force pass (nep_md_set_force_form): the 461-atom
    replica of the heat-transport workload for 40 steps of 1 fs against the
    oracle integrator from the same state.  Forces within the plain form's
    1e-3 eV/A bound move an atom of 28 amu by at most
    dF t^2 / (2 m) ~ 1e-3 x 40^2 / (2 x 28 x 103.64) ~ 3e-4 A in 40 fs; the
    test allows 1e-3 A and 1e-4 A/fs, and site energies within n x 1e-4 eV.
    Switching back to the optimised form restores its own bars."""
    import torch
    pos, vel, box, z = inputs.config3(cells=(4, 4, 4))
    n, steps = len(pos), 40
    model = N.NEP(z)
    md = N.MD(model, n, box, inputs.MASS_SI)
    md.set_force_form(True)
    p, v = soa(pos), soa(vel)
    thermo = torch.zeros(steps, N.THERMO_COLS, dtype=torch.float64, device="cuda")
    md.step(p, v, steps, 1.0, thermo)
    md.sync_status()
    po, vo, th_o, _ = orc.md(orc.NepHyper(), f32_exact(z), pos, vel, box, inputs.MASS_SI, 1.0, steps)
    assert np.abs(thermo.cpu().numpy()[:, 0] - th_o[:, 0]).max() <= TOL_U * n
    L = np.diag(box)
    dx = aos(p) - po
    dx -= L * np.round(dx / L)
    assert np.abs(dx).max() < 1e-3
    assert np.abs(aos(v) - vo).max() < 1e-4
    # back to the optimised form: one more step from the oracle's state agrees
    # with the oracle's next step at the optimised path's bars
    md.set_force_form(False)
    p2, v2 = soa(po), soa(vo)
    md.step(p2, v2, 1, 1.0)
    md.sync_status()
    po2, vo2, _, _ = orc.md(orc.NepHyper(), f32_exact(z), po, vo, box, inputs.MASS_SI, 1.0, 1)
    dx = aos(p2) - po2
    dx -= L * np.round(dx / L)
    assert np.abs(dx).max() < 1e-8 and np.abs(aos(v2) - vo2).max() < 1e-9
    md.close()
    model.close()
