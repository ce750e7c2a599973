"""The graph-replayed SNES loop (snes_run) and the evaluation's launch shapes.

snes_run replays one captured generation; its generation counter lives on the
device, so n generations of snes_run must equal n calls of snes_step bit for
bit (draws, losses, m, s).  Within each contraction form no launch shape may
change a result bit: in the two-pass form every value keeps its single writer
and its summation order; in the fused form the force sums are exact integer
sums and every other sum runs over the atoms in an order independent of the
members per block.  So the losses of every shape of one form must be
identical, and the two forms agree to the rounding of the two-pass form's
FP32 force sums.  In BF16 precision the two-pass form with its first pass on
the tensor cores (owner_tc) is a third form: FP16 Jacobian rows, the same
losses to ~1e-4 relative."""
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


def _gpu_labels(N, model, structures):
    """Targets from the GPU force path of the model itself (values do not
    matter here, only that every run sees the same ones)."""
    import torch
    E, F, W = [], [], []
    for st in structures:
        out = model.compute(torch.tensor(st["pos"].T.copy(), dtype=torch.float64, device="cuda"), st["box"])
        E.append(out["e_atom"].double().sum().item() + 0.01 * len(st["pos"]))
        F.append(out["force"].cpu().numpy().T + 0.02)
        W.append(np.full(6, 0.1))
    return np.array(E), np.concatenate(F), np.array(W)


@pytest.fixture(scope="module")
def full_set(N):
    structures, teacher, pop = inputs.config4()
    rng = np.random.default_rng(5)
    model = N.NEP(f32_exact(inputs.random_z(1021, rng)).astype(np.float32))
    E, F, W = _gpu_labels(N, model, structures)
    ds = N.Dataset(model, structures, E, F, W)
    yield model, ds, f32_exact(pop)
    ds.close()
    model.close()


def _two_pass_shapes(precision, N):
    out = []
    for w in (1, 2, 4):
        for ow in (4, 8):
            for dc in (0, 1):
                for mt in ((128, 256) if precision == N.PREC_FP32 else (256,)):
                    for ru in (1, 4, 8, 12, 16):
                        for pp in ((0, 1) if precision == N.PREC_BF16 else (0,)):
                            out.append(dict(waves=w, owner_warps=ow, discard=dc, mlp_threads=mt, recv_unroll=ru,
                                            fused=0, owner_tc=0, pop_pipe=pp))
    return out


def _tc_shapes():
    """Two-pass shapes with the first pass on the tensor cores (BF16)."""
    return [dict(waves=w, owner_warps=4, discard=dc, mlp_threads=256, recv_unroll=ru, fused=0, owner_tc=1, pop_pipe=pp)
            for w in (1, 2, 4) for dc in (0, 1) for ru in (1, 4, 8, 12, 16) for pp in (0, 1)]


def _fused_shapes(precision, N):
    return [dict(waves=1, owner_warps=4, discard=0, mlp_threads=mt, recv_unroll=4, fused=gm, owner_tc=0, pop_pipe=pp)
            for gm in (4, 8, 16) for mt in ((128, 256) if precision == N.PREC_FP32 else (256,))
            for pp in ((0, 1) if precision == N.PREC_BF16 else (0,))]


def _all_shapes(precision, N):
    return (_fused_shapes(precision, N) + _two_pass_shapes(precision, N) +
            (_tc_shapes() if precision == N.PREC_BF16 else []))


def _form(shape):
    return "fused" if shape["fused"] else ("two-pass-tc" if shape["owner_tc"] else "two-pass")


@pytest.mark.parametrize("prec", [0, 1])
def test_every_shape_gives_identical_losses(N, full_set, prec):
    import torch
    model, ds, pop = full_set
    zp = torch.tensor(pop, dtype=torch.float32, device="cuda")
    refs = {}
    extra = [dict(waves=16, owner_warps=8, discard=1, mlp_threads=128, recv_unroll=8, fused=0, owner_tc=0,
                  pop_pipe=0)]
    forms = [("fused", _fused_shapes(prec, N))]
    if prec == N.PREC_FP32:
        # owner_tc does not apply in FP32: the same form, the same bits
        forms.append(("two-pass", _two_pass_shapes(prec, N) + extra +
                      [dict(sh, mlp_threads=256) for sh in _tc_shapes()] +
                      [dict(extra[0], pop_pipe=1)]))
    else:
        forms.append(("two-pass", _two_pass_shapes(prec, N) + extra))
        forms.append(("two-pass-tc", _tc_shapes() + [dict(extra[0], owner_tc=1)]))
    for form, shapes in forms:
        ds.set_shape(**shapes[0])
        ref = refs[form] = ds.evaluate(zp, prec).cpu().numpy()
        assert np.isfinite(ref).all()
        for sh in shapes:
            ds.set_shape(**sh)
            assert ds.shape() == sh
            for _ in range(3):  # repeated: a race would show as a changed bit
                got = ds.evaluate(zp, prec).cpu().numpy()
                assert np.array_equal(got, ref), sh
    # the two forms: the same losses up to the two-pass form's force sums
    # (FP32; in BF16 mode its partial forces pass through FP16, ~1e-6 relative
    # in each loss term after the average over all force components)
    rtol = 1e-6 if prec == N.PREC_FP32 else 2e-5
    assert np.allclose(refs["fused"], refs["two-pass"], rtol=rtol, atol=0.0), \
        np.abs(refs["fused"] / refs["two-pass"] - 1).max()
    if "two-pass-tc" in refs:
        # FP16 Jacobian rows (11-bit significands) instead of FP32 ones
        rel = np.abs(refs["two-pass-tc"] / refs["two-pass"] - 1)
        print(f"owner pass on the tensor cores: loss terms within {rel.max(axis=0)} relative")
        assert rel.max() <= 2e-4, rel.max(axis=0)
    ds.set_shape()
    model.sync_status()


def test_autotuner_picks_a_candidate(N, full_set):
    import torch
    model, ds, pop = full_set
    zp = torch.tensor(pop, dtype=torch.float32, device="cuda")
    refs = {}
    for sh in (dict(fused=8), dict(fused=0), dict(fused=0, owner_tc=1)):
        ds.set_shape(**sh)
        refs[_form(ds.shape())] = ds.evaluate(zp, N.PREC_BF16).cpu().numpy()
    shape, ms = ds.tune(50, N.PREC_BF16, reps=2)
    assert shape in _all_shapes(N.PREC_BF16, N)
    assert ds.shape() == shape
    assert 0.0 < ms < 100.0
    assert np.array_equal(ds.evaluate(zp, N.PREC_BF16).cpu().numpy(), refs[_form(shape)])
    ds.set_shape()


def test_shape_validation(N, full_set):
    model, ds, pop = full_set
    assert ds.default_shape() == dict(waves=1, owner_warps=4, discard=0, mlp_threads=256, recv_unroll=4, fused=8,
                                      owner_tc=0, pop_pipe=0)
    for bad in (dict(waves=0), dict(waves=17), dict(owner_warps=6), dict(discard=2), dict(mlp_threads=64),
                dict(recv_unroll=0), dict(recv_unroll=2), dict(recv_unroll=6), dict(fused=2), dict(fused=32), dict(fused=-4),
                dict(owner_tc=2), dict(owner_tc=-1), dict(pop_pipe=2), dict(pop_pipe=-1)):
        with pytest.raises(N.NepError) as e:
            ds.set_shape(**bad)
        assert e.value.code == -1  # NEP_ERR_ARG
    assert ds.shape() == ds.default_shape()


@pytest.mark.parametrize("shape", [dict(), dict(fused=0, waves=1), dict(fused=0, waves=4, discard=1),
                                   dict(fused=0, owner_tc=1), dict(fused=0, waves=4, owner_tc=1),
                                   dict(fused=0, owner_tc=1, recv_unroll=1, pop_pipe=1)])
def test_run_equals_steps(N, full_set, shape):
    """Generations from the replayed graph equal eager snes_step calls bit
    for bit, the loss history included, and the two interleave (the fused
    contraction, and the two-pass form with one and with four ranges)."""
    import torch
    model, ds, pop = full_set
    ds.set_shape(**shape)
    m0 = f32_exact(np.random.default_rng(8).uniform(-0.5, 0.5, 1021))
    a = N.SNES(model, 50, m0, np.full(1021, 0.1), seed=77)
    b = N.SNES(model, 50, m0, np.full(1021, 0.1), seed=77)
    steps = []
    for _ in range(3):
        loss = torch.empty(50, N.LOSS_COLS, dtype=torch.float64, device="cuda")
        a.step(ds, N.PREC_BF16, loss=loss)
        steps.append(loss)
    hist = b.run(ds, 3, N.PREC_BF16, history=True)
    assert torch.equal(hist, torch.stack(steps))
    for x, y in zip(a.state(), b.state()):
        assert torch.equal(x, y)
    # interleave: graph, eager, graph (precision switch recaptures)
    a.run(ds, 2, N.PREC_FP32)
    b.step(ds, N.PREC_FP32)
    b.step(ds, N.PREC_FP32)
    h2 = a.run(ds, 1, N.PREC_BF16, history=True)
    loss = torch.empty(50, N.LOSS_COLS, dtype=torch.float64, device="cuda")
    b.step(ds, N.PREC_BF16, loss=loss)
    assert torch.equal(h2[0], loss)
    for x, y in zip(a.state(), b.state()):
        assert torch.equal(x, y)
    assert a.run(ds, 0) is None
    a.close()
    b.close()
    ds.set_shape()
    model.sync_status()


def test_fused_shape_follows_the_largest_structure(N):
    """The fused contraction keeps a structure's force sums in shared memory
    (atoms x members x 48 bytes, at most 220 KB): with a 600-atom structure in
    the set, 8 or 16 members per block do not fit, the default becomes 4
    members per block, the larger shapes are rejected, and the fused and
    two-pass forms agree."""
    import torch
    rng = np.random.default_rng(11)
    pos, box = inputs.diamond(5, 5, 3)
    big = {"pos": inputs.displace(pos, 0.1, rng), "box": box}
    structures = inputs.training_structures(6, seed_stream=13) + [big]
    assert len(big["pos"]) == 600
    model = N.NEP(f32_exact(inputs.random_z(1021, rng)).astype(np.float32))
    E, F, W = _gpu_labels(N, model, structures)
    ds = N.Dataset(model, structures, E, F, W)
    assert ds.counts()["largest_structure"] == 600
    assert ds.shape()["fused"] == 4
    for bad in (8, 16):
        with pytest.raises(N.NepError) as e:
            ds.set_shape(fused=bad)
        assert e.value.code == -1
    zp = torch.tensor(f32_exact(rng.normal(0.0, 0.1, size=(12, 1021))), dtype=torch.float32, device="cuda")
    for prec in (N.PREC_FP32, N.PREC_BF16):
        ds.set_shape(fused=4)
        a = ds.evaluate(zp, prec).cpu().numpy()
        ds.set_shape(fused=0)
        b = ds.evaluate(zp, prec).cpu().numpy()
        assert np.isfinite(a).all()
        assert np.allclose(a, b, rtol=1e-6 if prec == N.PREC_FP32 else 2e-5, atol=0.0), np.abs(a / b - 1).max()
    model.sync_status()
    ds.close()
    model.close()


@pytest.mark.parametrize("n_pop", [1, 5, 64])
def test_population_sizes_at_the_edges(N, full_set, n_pop):
    """One member, a ragged last member group (5 = 4 + 1) and the largest
    population (64, a full last group and the widest owner-pass MMA): in BF16
    the pipelined and the one-CTA-per-tile network give the same bits, with
    the tensor-core owner pass and the bulk receiver too; FP32 and BF16 agree
    to 1e-3 on every loss term and rank the members alike."""
    import torch
    model, ds, pop = full_set
    z = np.random.default_rng(31 + n_pop).normal(0.0, 0.1, size=(n_pop, 1021))
    zp = torch.tensor(f32_exact(z), dtype=torch.float32, device="cuda")
    got = {}
    for pp in (0, 1):
        for otc, ru in ((0, 4), (1, 1)):
            ds.set_shape(fused=0, owner_tc=otc, recv_unroll=ru, pop_pipe=pp)
            got[(pp, otc)] = ds.evaluate(zp, N.PREC_BF16).cpu().numpy()
    for otc in (0, 1):
        assert np.array_equal(got[(0, otc)], got[(1, otc)]), otc
    ds.set_shape(fused=0)
    l32 = ds.evaluate(zp, N.PREC_FP32).cpu().numpy()
    for otc in (0, 1):
        l16 = got[(1, otc)]
        assert np.isfinite(l16).all()
        rel = np.abs(l16[:, :4] - l32[:, :4]) / np.abs(l32[:, :4])
        assert rel.max() <= 1e-3, (otc, rel.max(axis=0))
        assert list(np.argsort(l16[:, 0], kind="stable")) == list(np.argsort(l32[:, 0], kind="stable"))
    ds.set_shape()
    model.sync_status()
