"""The BF16 tensor-core (tcgen05) population path: one tile against a plain
PyTorch FP32 GEMM of the same BF16 operands, then the population losses of
NEP_PREC_BF16 against the FP32 path (within 1e-3 relative, same ranking)."""
import numpy as np
import pytest

from gpu_util import f32_exact
from paper_2107_08119_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    from paper_2107_08119_gb300 import build
    build.build()
    from paper_2107_08119_gb300 import nep
    return nep


def test_tcgen05_tile_matches_plain_gemm(N):
    import torch
    g = torch.Generator(device="cuda").manual_seed(5)
    for n in (240, 64, 32, 16, 256):
        A = torch.randn(128, 32, generator=g, device="cuda").to(torch.bfloat16)
        B = torch.randn(n, 32, generator=g, device="cuda").to(torch.bfloat16)
        D, err = N.tc_selftest(A, B)
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        ref = A.float() @ B.float().T          # products of BF16 values are exact in FP32
        assert (D - ref).abs().max().item() <= 1e-5 * max(1.0, ref.abs().max().item()), n


def _labels_gpu(N, model, structures):
    import torch
    E, F, W = [], [], []
    for s in structures:
        out = model.compute(torch.tensor(s["pos"].T.copy(), dtype=torch.float64, device="cuda"), s["box"])
        wt = out["virial_total"].cpu().numpy().reshape(3, 3)
        E.append(out["e_total"].item())
        F.append(out["force"].cpu().numpy().T)
        W.append([wt[0, 0], wt[1, 1], wt[2, 2], wt[0, 1], wt[1, 2], wt[2, 0]])
    return np.array(E), np.concatenate(F), np.array(W)


def test_bf16_population_losses_track_fp32(N):
    """All 50 members on the 200-structure training workload: BF16 GEMMs with
    FP32 accumulation give losses within 1e-3 relative of the FP32 path and the
    same fitness ranking."""
    import torch
    structures, teacher, pop = inputs.config4()
    model = N.NEP(np.asarray(teacher, np.float32))
    E, F, W = _labels_gpu(N, model, structures)
    ds = N.Dataset(model, structures, E, F, W)
    zp = torch.tensor(f32_exact(pop), dtype=torch.float32, device="cuda")
    l32 = ds.evaluate(zp, N.PREC_FP32).cpu().numpy()
    l16 = ds.evaluate(zp, N.PREC_BF16).cpu().numpy()
    model.sync_status()
    rel = np.abs(l16 - l32) / np.abs(l32)
    assert rel[:, 0].max() <= 1e-3, rel[:, 0].max()
    assert list(np.argsort(l16[:, 0], kind="stable")) == list(np.argsort(l32[:, 0], kind="stable"))
    # deterministic
    assert np.array_equal(l16, ds.evaluate(zp, N.PREC_BF16).cpu().numpy())
    ds.close()
    model.close()
