"""The allocation-free entry point, nep_compute_efv_static.

It serves callers that cannot allocate device memory when they need forces
(a locked or full memory pool, a host application that owns every
allocation, an allocator-free real-time loop): its scratch is a fixed-size
array inside the library.  This test calls it through the C ABI with buffers
the caller allocated beforehand, twice in a row (the array keeps the first
call's contents), and checks it against nep_compute_efv with the tolerances
the other parity tests use.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from gpu_util import soa
from paper_2107_08119_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL_U, TOL_F, TOL_W = 1e-6, 1e-4, 1e-4


@pytest.fixture(scope="module")
def N():
    from paper_2107_08119_gb300 import build
    build.build()
    from paper_2107_08119_gb300 import nep
    return nep


def _call_static(N, h, z_dev, pos, box, out):
    import torch
    n = pos.shape[1]
    b = np.ascontiguousarray(np.asarray(box, np.float64).reshape(9))
    p = lambda t: C.c_void_p(t.data_ptr())
    return N._lib.nep_compute_efv_static(
        C.byref(h.c()), p(z_dev), int(z_dev.numel()), n, b.ctypes.data_as(C.c_void_p), p(pos), p(out["e_total"]),
        p(out["e_atom"]), p(out["force"]), p(out["virial_atom"]), p(out["virial_total"]), p(out["err"]),
        C.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_static_entry_point_matches_compute_efv(N):
    import torch
    h = N.Hyper(max_neighbors=N.STATIC_MAX_NEIGHBORS)
    cases = [inputs.config1()]
    p3, _, b3, z3 = inputs.config3(cells=(4, 4, 4))
    cases.append((p3, b3, z3))
    for pos, box, z in cases:
        n = len(pos)
        model = N.NEP(np.asarray(z, np.float32), h)
        ref = model.compute(soa(pos), box)
        model.close()
        z_dev = torch.tensor(np.asarray(z, np.float32), device="cuda")
        ps = soa(pos)
        out = {"e_total": torch.empty(1, dtype=torch.float64, device="cuda"),
               "e_atom": torch.empty(n, dtype=torch.float64, device="cuda"),
               "force": torch.empty(3, n, dtype=torch.float32, device="cuda"),
               "virial_atom": torch.empty(9, n, dtype=torch.float32, device="cuda"),
               "virial_total": torch.empty(9, dtype=torch.float64, device="cuda"),
               "err": torch.full((1,), -1, dtype=torch.int32, device="cuda")}
        for _ in range(2):
            for t in out.values():
                t.fill_(float("nan") if t.is_floating_point() else -1)
            rc = _call_static(N, h, z_dev, ps, box, out)
            assert rc == 0, N._lib.nep_last_error()
            torch.cuda.synchronize()
            assert int(out["err"].item()) == 0
            assert (out["e_atom"] - ref["e_atom"]).abs().max().item() <= TOL_U
            assert (out["force"] - ref["force"]).abs().max().item() <= TOL_F
            assert (out["virial_atom"] - ref["virial_atom"]).abs().max().item() <= TOL_W
            assert abs(out["e_total"].item() - ref["e_total"].item()) <= TOL_U * n
            assert (out["virial_total"] - ref["virial_total"]).abs().max().item() <= TOL_W * n


def _outs(n):
    import torch
    return {"e_total": torch.empty(1, dtype=torch.float64, device="cuda"),
            "e_atom": torch.empty(n, dtype=torch.float64, device="cuda"),
            "force": torch.empty(3, n, dtype=torch.float32, device="cuda"),
            "virial_atom": torch.empty(9, n, dtype=torch.float32, device="cuda"),
            "virial_total": torch.empty(9, dtype=torch.float64, device="cuda"),
            "err": torch.full((1,), -1, dtype=torch.int32, device="cuda")}


def test_static_entry_point_in_a_cuda_graph(N):
    """The call allocates and synchronises nothing, so after a first eager
    call in the context it can be captured into a CUDA graph: each replay
    reads the positions as they are at replay time and gives the bits of an
    eager call on them."""
    import torch
    h = N.Hyper(max_neighbors=N.STATIC_MAX_NEIGHBORS)
    pos, box, z = inputs.config1()
    n = len(pos)
    z_dev = torch.tensor(np.asarray(z, np.float32), device="cuda")
    ps = soa(pos)
    eager, graphed = _outs(n), _outs(n)
    assert _call_static(N, h, z_dev, ps, box, eager) == 0, N._lib.nep_last_error()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        assert _call_static(N, h, z_dev, ps, box, graphed) == 0, N._lib.nep_last_error()
    rng = np.random.default_rng(11)
    for step in range(3):
        if step:
            # move the atoms a little: the replay must see the new positions
            ps += torch.tensor(rng.normal(scale=0.02, size=ps.shape), dtype=torch.float64, device="cuda")
            assert _call_static(N, h, z_dev, ps, box, eager) == 0, N._lib.nep_last_error()
        for t in graphed.values():
            t.fill_(float("nan") if t.is_floating_point() else -1)
        g.replay()
        torch.cuda.synchronize()
        assert int(graphed["err"].item()) == 0
        for k in eager:
            assert torch.equal(graphed[k], eager[k]), (step, k)
    del g


def test_static_entry_point_rejects_oversize_inputs(N):
    """Sizes beyond the fixed scratch are refused before any launch."""
    import torch
    h = N.Hyper(max_neighbors=N.STATIC_MAX_NEIGHBORS)
    pos, box = inputs.diamond(8, 8, 9)                  # 4,608 atoms > 4,096
    z_dev = torch.zeros(h.n_par, dtype=torch.float32, device="cuda")
    ps = soa(pos)
    n = len(pos)
    out = {"e_total": torch.empty(1, dtype=torch.float64, device="cuda"),
           "e_atom": torch.empty(n, dtype=torch.float64, device="cuda"),
           "force": torch.empty(3, n, dtype=torch.float32, device="cuda"),
           "virial_atom": torch.empty(9, n, dtype=torch.float32, device="cuda"),
           "virial_total": torch.empty(9, dtype=torch.float64, device="cuda"),
           "err": torch.empty(1, dtype=torch.int32, device="cuda")}
    assert _call_static(N, h, z_dev, ps, box, out) == -1
    assert b"4096" in N._lib.nep_last_error()
    h2 = N.Hyper(max_neighbors=N.STATIC_MAX_NEIGHBORS + 1)
    pos, box, z = inputs.config1()
    assert _call_static(N, h2, z_dev, soa(pos), box, out) == -1
