"""Pins of the oracle's forces (Eqs. 4-5, 23-25), per-atom virial (Eq. 6) and
heat current (Eq. 7) to finite differences of the energy, conservation laws,
invariances and extensivity."""
import numpy as np
import pytest

from geometry import cluster, rotation
from paper_2107_08119_gb300 import inputs

H = dict(n_max_R=7, n_max_A=5, l_max=4, n_neu=30, rc_R=5.0, rc_A=4.0)


@pytest.fixture(scope="module")
def model(orc):
    h = orc.NepHyper(**H)
    z = inputs.random_z(orc.n_par(h), np.random.default_rng(42))
    return h, z


def _periodic(cells=(2, 2, 2), sigma=0.15, seed=5, a=5.43):
    pos, box = inputs.diamond(*cells, a)
    return inputs.displace(pos, sigma, np.random.default_rng(seed)), box


def test_force_is_minus_energy_gradient(orc, model):
    """F_i = -dE/dr_i by central differences (h = 1e-5 A) in a small periodic
    cell with several image layers and in a cluster."""
    h, z = model
    for pos, box in (_periodic((1, 2, 2)), cluster(9, seed=4)):
        U, F, W = orc.efv(h, z, pos, box)
        for i in range(0, len(pos), max(1, len(pos) // 6)):
            for a in range(3):
                d = 1e-5
                p = pos.copy()
                p[i, a] += d
                ep = orc.efv(h, z, p, box)[0].sum()
                p[i, a] -= 2 * d
                em = orc.efv(h, z, p, box)[0].sum()
                assert F[i, a] == pytest.approx(-(ep - em) / (2 * d), abs=2e-8)


def test_net_force_zero_and_zero_weights(orc, model):
    h, z = model
    pos, box = _periodic((2, 2, 2))
    U, F, W = orc.efv(h, z, pos, box)
    assert np.abs(F.sum(axis=0)).max() < 1e-12
    z0 = z.copy()
    nd = orc.n_des(h)
    z0[: h.n_neu * nd] = 0.0           # w1 = 0: the energy no longer depends on positions
    U0, F0, W0 = orc.efv(h, z0, pos, box)
    assert np.abs(F0).max() == 0.0 and np.abs(W0).max() == 0.0
    assert np.allclose(U0, U0[0])


def test_total_virial_is_strain_derivative(orc, model):
    """sum_i W_i = -dE/d(epsilon) for a homogeneous deformation of box and
    positions, and the total is symmetric (Sec. II.B)."""
    h, z = model
    for pos, box in (_periodic((1, 2, 2)), _periodic((2, 2, 2), seed=9)):
        U, F, W = orc.efv(h, z, pos, box)
        Wt = W.sum(axis=0)
        assert np.abs(Wt - Wt.T).max() < 1e-10
        d = 1e-6
        for a in range(3):
            for b in range(3):
                e = np.zeros((3, 3))
                e[a, b] = d
                Dp, Dm = np.eye(3) + e, np.eye(3) - e
                ep = orc.efv(h, z, pos @ Dp.T, box @ Dp.T)[0].sum()
                em = orc.efv(h, z, pos @ Dm.T, box @ Dm.T)[0].sum()
                assert Wt[b, a] == pytest.approx(-(ep - em) / (2 * d), abs=1e-7)


def test_per_atom_virial_by_finite_differences(orc, model):
    """W_i^{ab} = sum_k r_ik^a dU_k/dr_i^b with the site energies U_k
    differentiated numerically; checks every component of the non-symmetric
    per-atom tensor (Eq. 6), in a cluster and in a periodic box > 2 r_c."""
    h, z = model
    for pos, box, atoms in ((*cluster(10, seed=8), range(10)), (*_periodic((3, 3, 3), seed=12), (0, 77, 150))):
        U, F, W = orc.efv(h, z, pos, box)
        L = np.diag(box)
        for i in atoms:
            rik = pos - pos[i]
            rik -= L * np.round(rik / L)
            dU = np.zeros((len(pos), 3))
            for b in range(3):
                d = 1e-5
                p = pos.copy()
                p[i, b] += d
                up = orc.efv(h, z, p, box)[0]
                p[i, b] -= 2 * d
                um = orc.efv(h, z, p, box)[0]
                dU[:, b] = (up - um) / (2 * d)
            want = np.einsum("ka,kb->ab", rik, dU)
            assert np.allclose(W[i], want, atol=1e-8)


def test_heat_current_energy_moment_identity(orc, model):
    """In an isolated cluster the heat current of Eq. 7 equals
    sum_k r_k dU_k/dt + sum_k r_k (F_k . v_k), the time derivative of the
    potential energy moment plus the work term (dU_k/dt by differences)."""
    h, z = model
    pos, box = cluster(11, seed=21)
    v = np.random.default_rng(3).normal(0, 0.01, pos.shape)
    U, F, W = orc.efv(h, z, pos, box)
    J = orc.heat_current(W, v)
    assert np.allclose(J, np.einsum("iab,ib->a", W, v), atol=1e-14)
    d = 1e-4
    dUdt = (orc.efv(h, z, pos + d * v, box)[0] - orc.efv(h, z, pos - d * v, box)[0]) / (2 * d)
    want = (pos * dUdt[:, None]).sum(axis=0) + (pos * np.sum(F * v, axis=1)[:, None]).sum(axis=0)
    assert np.allclose(J, want, atol=1e-9)


def test_rotation_covariance(orc, model):
    h, z = model
    pos, box = cluster(12, seed=6)
    U, F, W = orc.efv(h, z, pos, box)
    R = rotation([1, 2, -1], 0.7)
    c = pos.mean(axis=0)
    U2, F2, W2 = orc.efv(h, z, (pos - c) @ R.T + c, box)
    assert np.allclose(U2, U, atol=1e-12)
    assert np.allclose(F2, F @ R.T, atol=1e-12)
    assert np.allclose(W2, np.einsum("ab,ibc,dc->iad", R, W, R), atol=1e-12)


def test_extensivity_and_brute_force(orc, model):
    """E of a 2x2x2 replica is 8 E; per-atom U, F, W replicate; cell-list and
    brute-force neighbour search give the same results."""
    h, z = model
    pos, box = _periodic((2, 2, 2), seed=31)
    U, F, W = orc.efv(h, z, pos, box)
    Ub, Fb, Wb = orc.efv(h, z, pos, box, brute=True)
    assert np.allclose(U, Ub, atol=1e-13) and np.allclose(F, Fb, atol=1e-13) and np.allclose(W, Wb, atol=1e-13)
    reps = [pos + box[0] * a + box[1] * b + box[2] * c for a in range(2) for b in range(2) for c in range(2)]
    big = np.concatenate(reps)
    U8, F8, W8 = orc.efv(h, z, big, box * 2)
    assert U8.sum() == pytest.approx(8 * U.sum(), rel=1e-13)
    n = len(pos)
    for k in range(8):
        assert np.allclose(U8[k * n:(k + 1) * n], U, atol=1e-12)
        assert np.allclose(F8[k * n:(k + 1) * n], F, atol=1e-12)
        assert np.allclose(W8[k * n:(k + 1) * n], W, atol=1e-12)


def test_sampled_evaluation_equals_full(orc, model):
    """The per-atom sampler used for full-size parity gives the full result."""
    h, z = model
    for pos, box in (_periodic((3, 3, 3), seed=41), _periodic((1, 2, 2), seed=42)):
        U, F, W = orc.efv(h, z, pos, box)
        idx = np.array([0, 5, len(pos) // 2, len(pos) - 1])
        Us, Fs, Ws = orc.efv_sample(h, z, pos, box, idx)
        assert np.allclose(Us, U[idx], atol=1e-13)
        assert np.allclose(Fs, F[idx], atol=1e-12)
        assert np.allclose(Ws, W[idx], atol=1e-12)
