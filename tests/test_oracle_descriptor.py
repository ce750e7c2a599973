"""Pins of the oracle's descriptor (Eqs. 12-13) to closed forms, an
independent spherical-harmonic formulation (Eqs. 17-18) and invariances."""
import numpy as np
import pytest
from scipy.special import eval_legendre, sph_harm_y

from geometry import cheb_g, cluster, rotation

H_CFG = dict(n_max_R=7, n_max_A=5, l_max=4, n_neu=30, rc_R=5.0, rc_A=4.0)


def _h(orc, **kw):
    d = dict(H_CFG)
    d.update(kw)
    return orc.NepHyper(**d)


def _idx_nl(h, n, l):
    return (h.n_max_R + 1) + n * h.l_max + (l - 1)


def test_dimer_closed_form(orc):
    """Two atoms at distance r: q_n = g_n(r) and q_nl = g_n(r)^2 (only the k = j
    term, P_l(1) = 1)."""
    h = _h(orc)
    for r in (1.9, 2.35, 3.1, 3.99, 4.5):
        pos = np.array([[20.0, 20.0, 20.0], [20.0 + r * 0.6, 20.0 + r * 0.8, 20.0]])
        q = orc.descriptors(h, pos, np.eye(3) * 40.0)
        for i in range(2):
            for n in range(h.n_max_R + 1):
                assert q[i, n] == pytest.approx(cheb_g(r, 5.0, n), abs=1e-13)
            for n in range(h.n_max_A + 1):
                for l in range(1, h.l_max + 1):
                    assert q[i, _idx_nl(h, n, l)] == pytest.approx(cheb_g(r, 4.0, n) ** 2, abs=1e-13)


def test_trimer_closed_form(orc):
    """Centre atom with two neighbours at (r1, r2, theta):
    q_nl = g(r1)^2 + g(r2)^2 + 2 g(r1) g(r2) P_l(cos theta)."""
    h = _h(orc)
    r1, r2, th = 2.3, 3.2, 1.9
    c = np.array([20.0, 20.0, 20.0])
    # the two outer atoms are 4.9 A apart, beyond r_c^A = 4 but inside r_c^R = 5
    pos = np.array([c, c + r1 * np.array([1, 0, 0]), c + r2 * np.array([np.cos(th), np.sin(th), 0])])
    q = orc.descriptors(h, pos, np.eye(3) * 40.0)
    d12 = np.linalg.norm(pos[1] - pos[2])
    for n in range(h.n_max_A + 1):
        g1, g2 = cheb_g(r1, 4.0, n), cheb_g(r2, 4.0, n)
        for l in range(1, h.l_max + 1):
            want = g1 * g1 + g2 * g2 + 2 * g1 * g2 * eval_legendre(l, np.cos(th))
            assert q[0, _idx_nl(h, n, l)] == pytest.approx(want, abs=1e-13)
    for n in range(h.n_max_R + 1):
        assert q[0, n] == pytest.approx(cheb_g(r1, 5.0, n) + cheb_g(r2, 5.0, n), abs=1e-13)
        assert q[1, n] == pytest.approx(cheb_g(r1, 5.0, n) + cheb_g(d12, 5.0, n), abs=1e-13)


def test_addition_theorem_form(orc):
    """The literal pair sum equals 4 pi/(2l+1) sum_m |sum_j g_n Y_lm|^2 computed with
    scipy's complex spherical harmonics (Eqs. 17-18 with n = n'), on a periodic
    solid where every atom has many neighbours."""
    from paper_2107_08119_gb300 import inputs
    h = _h(orc)
    pos, box = inputs.diamond(3, 3, 3)
    pos = inputs.displace(pos, 0.2, np.random.default_rng(7))
    q = orc.descriptors(h, pos, box)
    cnt, js, rs = orc.neighbors(pos, box, 4.0, method=0, cap=128)
    for i in (0, 17, 101):
        rij = rs[i, :cnt[i]]
        r = np.linalg.norm(rij, axis=1)
        theta = np.arccos(rij[:, 2] / r)
        phi = np.arctan2(rij[:, 1], rij[:, 0])
        for n in range(h.n_max_A + 1):
            g = np.array([cheb_g(x, 4.0, n) for x in r])
            for l in range(1, h.l_max + 1):
                c = [np.sum(g * np.conj(sph_harm_y(l, m, theta, phi))) for m in range(-l, l + 1)]
                want = 4 * np.pi / (2 * l + 1) * np.sum(np.abs(c) ** 2)
                assert q[i, _idx_nl(h, n, l)] == pytest.approx(want, rel=1e-11, abs=1e-13)


def test_invariances(orc):
    """Translation, rotation, inversion and permutation of a cluster leave every
    atom's descriptor unchanged; shifting an atom by a lattice vector of a
    periodic cell does too."""
    h = _h(orc)
    pos, box = cluster(12, seed=3)
    q0 = orc.descriptors(h, pos, box)
    ctr = pos.mean(axis=0)
    R = rotation([0.3, -0.5, 0.8], 1.1)
    for p in (pos + np.array([1.3, -0.7, 2.1]),
              (pos - ctr) @ R.T + ctr,
              -(pos - ctr) + ctr):
        assert np.allclose(orc.descriptors(h, p, box), q0, atol=1e-12)
    perm = np.random.default_rng(1).permutation(len(pos))
    assert np.allclose(orc.descriptors(h, pos[perm], box), q0[perm], atol=1e-12)

    from paper_2107_08119_gb300 import inputs
    pos, box = inputs.diamond(2, 2, 3, 5.5)
    pos = inputs.displace(pos, 0.2, np.random.default_rng(2))
    q0 = orc.descriptors(h, pos, box)
    p = pos.copy()
    p[5] += box[0] - 2 * box[2]
    p[9] -= box[1]
    assert np.allclose(orc.descriptors(h, p, box), q0, atol=1e-12)


def test_neighbor_search_brute_vs_cells(orc):
    """Cell-list neighbours equal brute-force image enumeration (as sets of
    (j, r_ij)), on boxes from one image layer up to many cells."""
    from paper_2107_08119_gb300 import inputs
    rng = np.random.default_rng(11)
    for cells, rc in (((1, 1, 1), 5.0), ((2, 2, 2), 5.0), ((4, 4, 4), 6.0), ((3, 4, 5), 6.0), ((2, 3, 4), 4.0)):
        pos, box = inputs.diamond(*cells)
        pos = inputs.displace(pos, 0.25, rng)
        cb, jb, rb = orc.neighbors(pos, box, rc, method=0, cap=1024)
        cc, jc, rcl = orc.neighbors(pos, box, rc, method=1, cap=1024)
        assert np.array_equal(cb, cc)
        for i in range(len(pos)):
            A = sorted((int(j), *np.round(r, 9)) for j, r in zip(jb[i, :cb[i]], rb[i, :cb[i]]))
            B = sorted((int(j), *np.round(r, 9)) for j, r in zip(jc[i, :cc[i]], rcl[i, :cc[i]]))
            assert A == B
        # every pair has its reverse with the opposite vector
        for i in range(len(pos)):
            for j, r in zip(jb[i, :cb[i]], rb[i, :cb[i]]):
                back = rb[j, :cb[j]][jb[j, :cb[j]] == i]
                assert np.any(np.all(np.abs(back + r) < 1e-9, axis=1))


def test_network_closed_form_on_dimer(orc):
    """Site energy of Eqs. 21-22 written out by hand for a dimer, with the
    parameter layout z = [w1 (n_neu x N_des row-major), b1, w2, b2] and the
    minus signs on both biases."""
    h = orc.NepHyper(n_max_R=2, n_max_A=1, l_max=2, n_neu=2, rc_R=5.0, rc_A=4.0)
    nd = orc.n_des(h)                      # 3 + 2*2 = 7
    rng = np.random.default_rng(4)
    w1 = rng.uniform(-1, 1, (2, nd))
    b1 = np.array([0.3, -0.2])
    w2 = np.array([0.7, -1.1])
    b2 = 0.45
    z = np.concatenate([w1.ravel(), b1, w2, [b2]])
    r = 3.1
    pos = np.array([[20.0, 20.0, 20.0], [20.0, 20.0 + r, 20.0]])
    U, F, W = orc.efv(h, z, pos, np.eye(3) * 40.0)
    gR = [cheb_g(r, 5.0, n) for n in range(3)]
    gA = [cheb_g(r, 4.0, n) for n in range(2)]
    q = np.array(gR + [gA[0] ** 2, gA[0] ** 2, gA[1] ** 2, gA[1] ** 2])
    want = w2 @ np.tanh(w1 @ q - b1) - b2
    assert U[0] == pytest.approx(want, abs=1e-14) and U[1] == pytest.approx(want, abs=1e-14)
    # F on atom 1 along the bond is -dE/dr, both atoms contribute equally
    d = 1e-6
    def e(rr):
        gr = [cheb_g(rr, 5.0, n) for n in range(3)]
        ga = [cheb_g(rr, 4.0, n) for n in range(2)]
        qq = np.array(gr + [ga[0] ** 2, ga[0] ** 2, ga[1] ** 2, ga[1] ** 2])
        return 2 * (w2 @ np.tanh(w1 @ qq - b1) - b2)
    assert F[1, 1] == pytest.approx(-(e(r + d) - e(r - d)) / (2 * d), abs=1e-8)
