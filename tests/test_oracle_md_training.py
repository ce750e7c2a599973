"""Pins of the oracle's integrator, loss (Eqs. 29-34), force-loss gradient,
SNES update (Eqs. 35-39) and Philox generator."""
import os

import numpy as np
import pytest

from paper_2107_08119_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
H = dict(n_max_R=7, n_max_A=5, l_max=4, n_neu=30, rc_R=5.0, rc_A=4.0)


@pytest.fixture(scope="module")
def model(orc):
    h = orc.NepHyper(**H)
    z = inputs.random_z(orc.n_par(h), np.random.default_rng(42))
    return h, z


def _state(seed=1, cells=(2, 2, 2)):
    rng = np.random.default_rng(seed)
    pos, box = inputs.diamond(*cells)
    pos = inputs.displace(pos, 0.1, rng)
    vel = inputs.maxwell_boltzmann(len(pos), 300.0, inputs.MASS_SI, rng)
    return pos, vel, box


def test_md_energy_and_momentum_conservation(orc, model):
    h, z = model
    pos, vel, box = _state()
    p2, v2, thermo, J = orc.md(h, z, pos, vel, box, inputs.MASS_SI, 1.0, 200)
    etot = thermo.sum(axis=1)
    # the random-weight potential heats the lattice to thousands of K within
    # 0.2 ps, so the bound is loose; the dt^2 scaling below is the sharp check
    assert np.abs(etot - etot[0]).max() < 1e-3 * len(pos)
    assert np.abs((v2 - vel).sum(axis=0)).max() < 1e-12   # equal masses: sum v conserved
    # halving dt reduces the energy fluctuation about fourfold (second-order scheme)
    _, _, th_half, _ = orc.md(h, z, pos, vel, box, inputs.MASS_SI, 0.5, 400)
    fl1 = np.abs(etot - etot[0]).max()
    fl2 = np.abs(th_half.sum(axis=1) - th_half.sum(axis=1)[0]).max()
    assert 2.5 < fl1 / fl2 < 6.0


def test_md_time_reversibility(orc, model):
    h, z = model
    pos, vel, box = _state(seed=2)
    p1, v1, _, _ = orc.md(h, z, pos, vel, box, inputs.MASS_SI, 1.0, 50)
    p0, v0, _, _ = orc.md(h, z, p1, -v1, box, inputs.MASS_SI, 1.0, 50)
    assert np.abs(p0 - pos).max() < 1e-9
    assert np.abs(v0 + vel).max() < 1e-12


def test_md_heat_current_matches_state(orc, model):
    """The integrator's per-step J is Eq. 7 applied to the state it reaches."""
    h, z = model
    pos, vel, box = _state(seed=3)
    p1, v1, _, J = orc.md(h, z, pos, vel, box, inputs.MASS_SI, 1.0, 3)
    U, F, W = orc.efv(h, z, p1, box)
    assert np.allclose(J[-1], orc.heat_current(W, v1), atol=1e-14)


def _toy(orc, h, teacher, n=2):
    structs = inputs.training_structures(n, seed_stream=77)
    E, Fs, Ws = [], [], []
    for s in structs:
        U, F, W = orc.efv(h, teacher, s["pos"], s["box"])
        Wt = W.sum(axis=0)
        E.append(U.sum())
        Fs.append(F)
        Ws.append([Wt[0, 0], Wt[1, 1], Wt[2, 2], Wt[0, 1], Wt[1, 2], Wt[2, 0]])
    return structs, np.array(E), np.concatenate(Fs), np.array(Ws)


def test_loss_teacher_and_hand_computed(orc, model):
    """Teacher labels give L = l1 L1 + l2 L2 exactly; shifted labels give the
    hand-computed RMSEs of Eqs. 30-34."""
    h, z = model
    structs, E, F, W = _toy(orc, h, z)
    out = orc.loss(h, z, structs, E, F, W)
    assert out[1] == pytest.approx(0, abs=1e-12) and out[2] == pytest.approx(0, abs=1e-12)
    assert out[3] == pytest.approx(0, abs=1e-12)
    assert out[4] == pytest.approx(np.mean(np.abs(z)), rel=1e-14)
    assert out[5] == pytest.approx(np.sqrt(np.mean(z * z)), rel=1e-14)
    assert out[0] == pytest.approx(0.05 * out[4] + 0.05 * out[5], rel=1e-12)
    n_at = np.array([len(s["pos"]) for s in structs])
    de = np.array([0.3, -0.1])            # eV per atom
    dv = np.array([[0.1, 0, 0, 0, 0, 0.2], [0, 0, 0.4, 0, 0, 0]])  # eV per atom
    df = 0.05
    out = orc.loss(h, z, structs, E + de * n_at, F + df, W + dv * n_at[:, None], lambdas=(1, 2, 3, 0, 0))
    Le = np.sqrt(np.mean(de ** 2))
    Lf = df
    Lv = np.sqrt(np.sum(dv ** 2) / 12)
    assert out[1] == pytest.approx(Le, rel=1e-10)
    assert out[2] == pytest.approx(Lf, rel=1e-10)
    assert out[3] == pytest.approx(Lv, rel=1e-10)
    assert out[0] == pytest.approx(Le + 2 * Lf + 3 * Lv, rel=1e-10)


def test_force_loss_gradient_by_finite_differences(orc):
    """Analytic dL_f/dz against central differences (h = 1e-4) on the 64-atom
    check structure, every parameter group (w1, b1, w2, b2)."""
    h = orc.NepHyper(**H)
    pos, box, teacher, student = inputs.config5(orc.n_par(h))
    s = [{"pos": pos, "box": box}]
    _, Ft, _ = orc.efv(h, teacher, pos, box)
    grad, lf = orc.force_loss_grad(h, student, s, Ft)
    _, F, _ = orc.efv(h, student, pos, box)
    assert lf == pytest.approx(np.sqrt(np.mean((F - Ft) ** 2)), rel=1e-13)
    nd, nh = orc.n_des(h), h.n_neu
    idx = list(range(0, nh * nd, 37)) + list(range(nh * nd, nh * nd + 2 * nh, 3)) + [orc.n_par(h) - 1]
    for k in idx:
        d = 1e-4
        zp = student.copy()
        zp[k] += d
        zm = student.copy()
        zm[k] -= d
        lp = np.sqrt(np.mean((orc.efv(h, zp, pos, box)[1] - Ft) ** 2))
        lm = np.sqrt(np.mean((orc.efv(h, zm, pos, box)[1] - Ft) ** 2))
        fd = (lp - lm) / (2 * d)
        assert grad[k] == pytest.approx(fd, rel=1e-6, abs=1e-10), k
    assert grad[-1] == 0.0


def test_snes_utilities(orc):
    for lam in (2, 5, 10, 50):
        u = orc.snes_utilities(lam)
        assert abs(u.sum()) < 1e-14
        assert np.all(np.diff(u) <= 1e-15)
        assert u[-1] == pytest.approx(-1.0 / lam)
    assert np.allclose(orc.snes_utilities(2), [0.5, -0.5])
    assert orc.snes_eta_s(1021) == pytest.approx((3 + np.log(1021)) / (5 * np.sqrt(1021)), rel=1e-15)


def test_snes_update_closed_form_and_ties(orc):
    """Two members: grad_m = (r_best - r_worst)/2, grad_s = ((r_b^2 - 1) - (r_w^2 - 1))/2,
    m += s grad_m (old s), s *= exp(eta_s/2 grad_s).  Ties keep index order."""
    rng = np.random.default_rng(0)
    r = rng.normal(size=(2, 7))
    m = rng.normal(size=7)
    s = np.full(7, 0.1)
    m2, s2, order = orc.snes_update([3.0, 1.0], r, m, s, 1.0, 0.2)
    gm = 0.5 * (r[1] - r[0])
    gs = 0.5 * ((r[1] ** 2 - 1) - (r[0] ** 2 - 1))
    assert list(order) == [1, 0]
    assert np.allclose(m2, m + s * gm, atol=1e-15)
    assert np.allclose(s2, s * np.exp(0.1 * gs), atol=1e-15)
    _, _, order = orc.snes_update([1.0, 2.0, 1.0, 0.5], rng.normal(size=(4, 3)), np.zeros(3), np.ones(3))
    assert list(order) == [3, 0, 2, 1]


def test_snes_minimises_sphere(orc):
    """SNES with the paper's learning rates drives the sphere function down."""
    npar, npop = 20, 16
    rng = np.random.default_rng(5)
    m = rng.uniform(-0.5, 0.5, npar) + 2.0
    s = np.full(npar, 0.1)
    f0 = np.sum(m * m)
    for g in range(300):
        r = rng.normal(size=(npop, npar))
        zk = m + s * r
        m, s, _ = orc.snes_update(np.sum(zk * zk, axis=1), r, m, s)
    assert np.sum(m * m) < 1e-3 * f0


def test_philox_known_answers_and_normals(orc):
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        assert list(orc.philox4x32_10(w[0:4], w[4:6])) == w[6:10]
    g = orc.gaussian(2107081194, 3, 200000)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1) < 0.01
    assert abs(np.mean(g ** 4) - 3) < 0.05
    assert not np.array_equal(g[:100], orc.gaussian(2107081194, 4, 100))
