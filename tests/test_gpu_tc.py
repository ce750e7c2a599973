"""The BF16 tensor-core (tcgen05) population path: one tile against a plain
PyTorch FP32 GEMM of the same BF16 operands, then the population losses of
NEP_PREC_BF16 against the FP32 path (every loss term within 1e-3 relative,
same ranking) on a training set labelled by the oracle."""
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


def _labels_oracle(orc, teacher, structures):
    """Targets of every structure from the FP64 oracle with the teacher."""
    h = orc.NepHyper()
    E, F, W = [], [], []
    for s in structures:
        U, Fs, Ws = orc.efv(h, teacher, s["pos"], s["box"])
        Wt = Ws.sum(axis=0)
        E.append(U.sum())
        F.append(Fs)
        W.append([Wt[0, 0], Wt[1, 1], Wt[2, 2], Wt[0, 1], Wt[1, 2], Wt[2, 0]])
    return np.array(E), np.concatenate(F), np.array(W)


def test_bf16_population_losses_track_fp32(N, orc):
    """All 50 members on the 200-structure training workload, labelled by the
    FP64 oracle with the teacher: BF16 GEMMs with FP32 accumulation give each
    loss term (total, L_e, L_f, L_v) within 1e-3 relative of the FP32 path,
    L_1 and L_2 (functions of z alone) identical, and the same fitness
    ranking; in the fused and the two-pass contraction, the latter also with
    its first pass on the tensor cores."""
    import torch
    structures, teacher, pop = inputs.config4()
    teacher = f32_exact(teacher)
    E, F, W = _labels_oracle(orc, teacher, structures)
    model = N.NEP(teacher.astype(np.float32))
    ds = N.Dataset(model, structures, E, F, W)
    zp = torch.tensor(f32_exact(pop), dtype=torch.float32, device="cuda")
    for fused, otc, pp in ((8, 0, 0), (0, 0, 0), (0, 1, 0), (0, 1, 1)):
        ds.set_shape(fused=fused, owner_tc=otc, pop_pipe=pp)
        l32 = ds.evaluate(zp, N.PREC_FP32).cpu().numpy()
        l16 = ds.evaluate(zp, N.PREC_BF16).cpu().numpy()
        model.sync_status()
        rel = np.abs(l16 - l32) / np.abs(l32)
        for col in range(4):
            assert rel[:, col].max() <= 1e-3, (fused, otc, pp, col, rel[:, col].max())
        assert np.array_equal(l16[:, 4:6], l32[:, 4:6])
        assert list(np.argsort(l16[:, 0], kind="stable")) == list(np.argsort(l32[:, 0], kind="stable"))
        # deterministic
        assert np.array_equal(l16, ds.evaluate(zp, N.PREC_BF16).cpu().numpy())
    ds.close()
    model.close()
