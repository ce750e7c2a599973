"""Parity of the CUDA force-loss adjoint (nep_force_loss / _backward) with the
FP64 oracle gradient (itself pinned by central differences), central
differences of the CUDA loss, the SNES path's L_f, and the torch autograd
wrapper.

Error budget: the CUDA forces are within TOL_F = 1e-4 eV/A of the oracle's
per component, so L_f is within TOL_F (triangle inequality of the RMS) and the
adjoint's seed delta = e / (3N L_f) is within ~TOL_F / L_f relative; the
recomputed descriptor derivatives and the network terms are FP32 (~1e-6
relative).  The gradient test therefore allows 4 (TOL_F / L_f + 1e-5) of the
largest gradient component on every component."""
import numpy as np
import pytest

from gpu_util import f32_exact
from paper_2107_08119_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL_F = 1e-4


@pytest.fixture(scope="module")
def N():
    from paper_2107_08119_gb300 import build
    build.build()
    from paper_2107_08119_gb300 import nep
    return nep


def _hyper(orc, N, n_neu):
    return orc.NepHyper(n_neu=n_neu), N.Hyper(n_neu=n_neu)


def _grad_bound(lf, g):
    return 4.0 * (TOL_F / lf + 1e-5) * np.abs(g).max()


def _dataset(N, model, structures, f_tar):
    e = np.zeros(len(structures))
    w = np.zeros((len(structures), 6))
    return N.Dataset(model, structures, e, f_tar, w)


def _check_against_oracle(orc, N, n_neu, structures, teacher, student):
    import torch
    ho, hg = _hyper(orc, N, n_neu)
    Ft = np.concatenate([orc.efv(ho, teacher, s["pos"], s["box"])[1] for s in structures])
    g_orc, lf_orc = orc.force_loss_grad(ho, student, structures, Ft)
    model = N.NEP(student.astype(np.float32), hg)
    ds = _dataset(N, model, structures, Ft)
    z = torch.tensor(student, dtype=torch.float32, device="cuda")
    lf = ds.force_loss(z).item()
    g = ds.force_loss_backward().cpu().numpy()
    model.sync_status()
    assert abs(lf - lf_orc) <= TOL_F, (lf, lf_orc)
    err = np.abs(g - g_orc).max()
    assert err <= _grad_bound(lf_orc, g_orc), (err, np.abs(g_orc).max(), lf_orc)
    assert g[-1] == 0.0
    ds.close()
    model.close()
    return g, g_orc, lf


def test_gradient_matches_oracle_on_check_structure(N, orc):
    """64-atom check structure (2^3 diamond cells, sigma 0.15 A), 32-30-1."""
    pos, box, teacher, student = inputs.config5(1021)
    _check_against_oracle(orc, N, 30, [{"pos": pos, "box": box}], f32_exact(teacher), f32_exact(student))


@pytest.mark.parametrize("n_neu", [1, 7, 64])
def test_gradient_other_widths(N, orc, n_neu):
    """Other hidden widths exercise the reduction layout (odd row strides,
    the largest shared-memory footprint at 64 neurons)."""
    n_par = 34 * n_neu + 1
    pos, box, _, _ = inputs.config5(1021)
    rng = np.random.default_rng(500 + n_neu)
    teacher = f32_exact(inputs.random_z(n_par, rng))
    student = f32_exact(inputs.random_z(n_par, rng))
    _check_against_oracle(orc, N, n_neu, [{"pos": pos, "box": box}], teacher, student)


def test_gradient_on_mixed_training_structures(N, orc):
    """Ten structures of uneven size and box (ragged per-block atom ranges,
    blocks spanning structure boundaries)."""
    structures = inputs.training_structures(10, seed_stream=31)
    rng = np.random.default_rng(31)
    teacher = f32_exact(inputs.random_z(1021, rng))
    student = f32_exact(inputs.random_z(1021, rng))
    _check_against_oracle(orc, N, 30, structures, teacher, student)


def test_central_differences_of_cuda_loss(N, orc):
    """dL_f/dz against central differences (h = 1e-4) of the CUDA loss itself
    on the largest gradient components.  The step is the FP32 difference
    actually applied; the FP32 loss is smooth to ~1e-6 relative, so the
    difference quotient carries ~1e-6 L_f / h of noise."""
    import torch
    pos, box, teacher, student = inputs.config5(1021)
    s = [{"pos": pos, "box": box}]
    ho, hg = _hyper(orc, N, 30)
    Ft = orc.efv(ho, f32_exact(teacher), pos, box)[1]
    model = N.NEP(np.asarray(student, np.float32), hg)
    ds = _dataset(N, model, s, Ft)
    z0 = torch.tensor(np.asarray(student, np.float32), device="cuda")
    lf = ds.force_loss(z0).item()
    g = ds.force_loss_backward().cpu().numpy()
    top = np.argsort(-np.abs(g))[:12]
    for k in top:
        zp, zm = z0.clone(), z0.clone()
        zp[k] += 1e-4
        zm[k] -= 1e-4
        hk = float(zp[k].item()) - float(zm[k].item())
        fd = (ds.force_loss(zp).item() - ds.force_loss(zm).item()) / hk
        assert fd == pytest.approx(g[k], rel=5e-3, abs=2e-6 * lf / hk), (k, fd, g[k])
    ds.close()
    model.close()


def test_loss_matches_snes_evaluation_and_is_deterministic(N, orc):
    """On the 200-structure training workload: L_f of the adjoint's forward
    (forces from partial forces) equals the SNES evaluation's L_f column
    (forces from precomputed Jacobians) to FP32 rounding, and two runs give
    bitwise-identical gradients."""
    import torch
    structures, teacher, pop = inputs.config4()
    model = N.NEP(np.asarray(teacher, np.float32))
    F = []
    for st in structures:
        out = model.compute(torch.tensor(st["pos"].T.copy(), dtype=torch.float64, device="cuda"), st["box"])
        F.append(out["force"].cpu().numpy().T)
    ds = _dataset(N, model, structures, np.concatenate(F))
    z = torch.tensor(np.asarray(pop[3], np.float32), device="cuda")
    lf = ds.force_loss(z).item()
    g1 = ds.force_loss_backward().clone()
    lf2 = ds.force_loss(z).item()
    g2 = ds.force_loss_backward()
    assert lf == lf2
    assert torch.equal(g1, g2)
    assert torch.isfinite(g1).all()
    loss = ds.evaluate(z[None].contiguous(), N.PREC_FP32).cpu().numpy()
    assert lf == pytest.approx(loss[0, 2], rel=1e-5)
    model.sync_status()
    ds.close()
    model.close()


def test_autograd_function(N, orc):
    """torch.autograd through ForceLoss: the gradient equals the adjoint's,
    and an upstream factor scales it (seed)."""
    import torch
    pos, box, teacher, student = inputs.config5(1021)
    s = [{"pos": pos, "box": box}]
    Ft = orc.efv(orc.NepHyper(), f32_exact(teacher), pos, box)[1]
    model = N.NEP(np.asarray(student, np.float32))
    ds = _dataset(N, model, s, Ft)
    z = torch.tensor(np.asarray(student, np.float32), device="cuda", requires_grad=True)
    L = N.force_loss(z, ds)
    L.backward()
    g_ref = ds.force_loss_backward()
    assert torch.equal(z.grad, g_ref.to(torch.float32))
    z.grad = None
    (3.0 * N.force_loss(z, ds)).backward()
    assert torch.allclose(z.grad.double(), 3.0 * g_ref, rtol=1e-6, atol=0)
    ds.close()
    model.close()


def test_backward_requires_forward(N, orc):
    pos, box, teacher, student = inputs.config5(1021)
    model = N.NEP(np.asarray(student, np.float32))
    ds = _dataset(N, model, [{"pos": pos, "box": box}], np.zeros((len(pos), 3)))
    with pytest.raises(N.NepError) as e:
        ds.force_loss_backward()
    assert e.value.code == -1  # NEP_ERR_ARG
    ds.close()
    model.close()
