"""Pins of the oracle's special functions and sizes to closed forms, library
routines and the paper's printed numbers (Eqs. 14-16, 26, A1-A3; Table I)."""
import json
import os

import numpy as np
import pytest
from scipy.special import eval_chebyt, eval_chebyu, eval_legendre

from geometry import cheb_g

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_sizes_match_paper_table1(orc):
    """N_des (Eq. 16) and N_par (Eq. 26) reproduce the paper's 80/65/41 and 4101/2681/1721."""
    data = json.load(open(os.path.join(GOLDEN, "table1_sizes.json")))
    for m in data["models"]:
        h = orc.NepHyper(m["n_max_R"], m["n_max_A"], m["l_max"], m["n_neu"], 5.0, 5.0)
        assert orc.n_des(h) == m["N_des"], m["name"]
        assert orc.n_par(h) == m["N_par"], m["name"]
    assert orc.n_des(orc.NepHyper()) == 32 and orc.n_par(orc.NepHyper()) == 1021


def test_chebyshev_trig_identities(orc):
    """T_n(cos t) = cos(n t) and U_{n-1}(cos t) = sin(n t)/sin t (App. A recurrences)."""
    for t in np.linspace(0.05, 3.09, 23):
        T, U = orc.chebyshev(np.cos(t), 16)
        for n in range(17):
            assert T[n] == pytest.approx(np.cos(n * t), abs=1e-12)
            if n >= 1:
                assert U[n - 1] == pytest.approx(np.sin(n * t) / np.sin(t), abs=1e-10)
    T, U = orc.chebyshev(0.37, 12)
    assert np.allclose(T, [eval_chebyt(n, 0.37) for n in range(13)], atol=1e-13)
    assert np.allclose(U, [eval_chebyu(n, 0.37) for n in range(13)], atol=1e-13)


def test_legendre_closed_forms(orc):
    closed = {1: lambda t: t, 2: lambda t: 0.5 * (3 * t * t - 1), 3: lambda t: 0.5 * (5 * t ** 3 - 3 * t),
              4: lambda t: (35 * t ** 4 - 30 * t * t + 3) / 8}
    for t in np.linspace(-1, 1, 41):
        for l, f in closed.items():
            p, d = orc.legendre(l, t)
            assert p == pytest.approx(f(t), abs=1e-14)
            h = 1e-6
            assert d == pytest.approx((f(t + h) - f(t - h)) / (2 * h), abs=1e-7)
        for l in range(0, 9):
            assert orc.legendre(l, t)[0] == pytest.approx(eval_legendre(l, t), abs=1e-13)
    for l in range(1, 9):
        assert orc.legendre(l, 1.0)[0] == pytest.approx(1.0, abs=1e-15)


def test_cutoff_function(orc):
    rc = 4.0
    assert orc.cutoff(0.0, rc)[0] == pytest.approx(1.0)
    assert orc.cutoff(rc, rc)[0] == pytest.approx(0.0, abs=1e-16)
    assert orc.cutoff(rc, rc)[1] == pytest.approx(0.0, abs=1e-15)
    assert orc.cutoff(rc + 1e-9, rc) == (0.0, 0.0)
    for r in np.linspace(0.3, 3.9, 13):
        h = 1e-6
        fd = (orc.cutoff(r + h, rc)[0] - orc.cutoff(r - h, rc)[0]) / (2 * h)
        assert orc.cutoff(r, rc)[1] == pytest.approx(fd, abs=1e-8)


def test_radial_functions(orc):
    """g_n of Eq. 14: g_0 = f_c, 0 <= g_n <= 1, g_n(r_c) = 0, derivative by FD,
    values equal to scipy's T_n with the cosine cutoff."""
    for rc in (4.0, 5.0):
        nmax = 9
        for r in np.linspace(0.5, rc, 37):
            g, dg = orc.radial(r, rc, nmax)
            assert g[0] == pytest.approx(orc.cutoff(r, rc)[0], abs=1e-15)
            assert np.all(g >= -1e-15) and np.all(g <= 1 + 1e-15)
            for n in range(nmax + 1):
                assert g[n] == pytest.approx(cheb_g(r, rc, n), abs=1e-13)
            if r < rc - 1e-3:
                h = 1e-6
                gp, _ = orc.radial(r + h, rc, nmax)
                gm, _ = orc.radial(r - h, rc, nmax)
                assert np.allclose(dg, (gp - gm) / (2 * h), atol=1e-7)
        g, dg = orc.radial(rc, rc, nmax)
        assert np.allclose(g, 0, atol=1e-15) and np.allclose(dg, 0, atol=1e-13)
