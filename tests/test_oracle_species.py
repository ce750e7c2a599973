"""Pins of the oracle's multicomponent weighting (Sec. II.A, "Multicomponent
systems"): the cutoff function of a pair becomes f_c(r_ij) sqrt(Z_i Z_j).

- one species of atomic number c scales every radial descriptor by c and
  every angular one by c^2 (g_n is linear in f_c);
- a dimer of Z_a and Z_b has q_n = sqrt(Z_a Z_b) g_n(r) and
  q_nl = Z_a Z_b g_n(r)^2 on both atoms (P_l(1) = 1);
- the central atom's own species matters: the same environment with the
  centre's Z four times larger doubles the radial and quadruples the
  angular descriptors (the point of the sqrt(Z_i) factor);
- forces stay minus the energy gradient and relabelling atoms together with
  their species permutes every output."""
import numpy as np
import pytest

from geometry import cluster
from paper_2107_08119_gb300 import inputs

H = dict(n_max_R=7, n_max_A=5, l_max=4, n_neu=30, rc_R=5.0, rc_A=4.0)
NR = 8


@pytest.fixture(scope="module")
def model(orc):
    h = orc.NepHyper(**H)
    z = inputs.random_z(orc.n_par(h), np.random.default_rng(17))
    return h, z


def _periodic(cells=(1, 2, 2), sigma=0.15, seed=8):
    pos, box = inputs.diamond(*cells, 5.43)
    return inputs.displace(pos, sigma, np.random.default_rng(seed)), box


def test_uniform_species_scales_radial_by_c_and_angular_by_c2(orc, model):
    h, _ = model
    pos, box = _periodic()
    q1 = orc.descriptors(h, pos, box)
    q4 = orc.descriptors(h, pos, box, Z=np.full(len(pos), 4.0))
    assert np.allclose(q4[:, :NR], 4.0 * q1[:, :NR], rtol=1e-13, atol=1e-15)
    assert np.allclose(q4[:, NR:], 16.0 * q1[:, NR:], rtol=1e-13, atol=1e-15)


def test_dimer_closed_form(orc, model):
    h, _ = model
    r = 2.7
    pos = np.array([[10.0, 10.0, 10.0], [10.0 + r, 10.0, 10.0]])
    box = np.eye(3) * 30.0
    za, zb = 14.0, 32.0
    q = orc.descriptors(h, pos, box, Z=[za, zb])
    gR, _ = orc.radial(r, 5.0, 7)
    gA, _ = orc.radial(r, 4.0, 5)
    w = np.sqrt(za * zb)
    for i in range(2):
        assert np.allclose(q[i, :NR], w * gR, rtol=1e-13)
        want = np.repeat((w * gA) ** 2, 4)  # n outer, l inner; P_l(1) = 1
        assert np.allclose(q[i, NR:], want, rtol=1e-12)


def test_central_species_is_distinguished(orc, model):
    h, _ = model
    pos, box = cluster(7, seed=3)
    Z = np.array([1.0, 2.0, 3.0, 1.0, 2.0, 3.0, 1.0])
    q = orc.descriptors(h, pos, box, Z=Z)
    Z4 = Z.copy()
    Z4[0] *= 4.0
    q4 = orc.descriptors(h, pos, box, Z=Z4)
    assert np.allclose(q4[0, :NR], 2.0 * q[0, :NR], rtol=1e-13, atol=1e-15)
    assert np.allclose(q4[0, NR:], 4.0 * q[0, NR:], rtol=1e-13, atol=1e-15)


def test_forces_are_minus_energy_gradient_with_two_species(orc, model):
    h, z = model
    pos, box = _periodic()
    Z = np.where(np.arange(len(pos)) % 3 == 0, 52.0, 82.0) / 60.0
    U, F, W = orc.efv(h, z, pos, box, Z=Z)
    for i in range(0, len(pos), 5):
        for a in range(3):
            d = 1e-5
            p = pos.copy()
            p[i, a] += d
            ep = orc.efv(h, z, p, box, Z=Z)[0].sum()
            p[i, a] -= 2 * d
            em = orc.efv(h, z, p, box, Z=Z)[0].sum()
            assert F[i, a] == pytest.approx(-(ep - em) / (2 * d), abs=3e-8)
    assert np.abs(F.sum(axis=0)).max() < 1e-10


def test_relabelling_atoms_with_their_species_permutes_outputs(orc, model):
    h, z = model
    pos, box = _periodic()
    rng = np.random.default_rng(4)
    Z = rng.choice([0.5, 1.0, 1.5], size=len(pos))
    perm = rng.permutation(len(pos))
    U, F, W = orc.efv(h, z, pos, box, Z=Z)
    Up, Fp, Wp = orc.efv(h, z, pos[perm], box, Z=Z[perm])
    assert np.allclose(Up, U[perm], rtol=1e-12, atol=1e-13)
    assert np.allclose(Fp, F[perm], rtol=1e-11, atol=1e-12)
    assert np.allclose(Wp, W[perm], rtol=1e-11, atol=1e-12)
    # and the species are not ignored
    U1 = orc.efv(h, z, pos, box)[0]
    assert np.abs(U1 - U).max() > 1e-3
