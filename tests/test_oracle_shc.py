"""Pins of the oracle's spectral heat current (Sec. II.B): the
virial-velocity correlation K(t) = sum_i <W_i(0) . v_i(t)> over time origins,
and its cosine transform.

- K at lag 0 is the heat current of Eq. 7 summed over the samples (the
  integrator's own J, computed by a different routine);
- constant histories give (S - tau) sum_i W_i . v_i at every lag (the count
  of origins per lag);
- a virial present only at sample s0 and a velocity only at s1 give a single
  non-zero lag, s1 - s0, with the value of their contraction (the direction
  of the lag and the index order of W . v);
- the transform of an exponential is the Lorentzian 2 tau / (1 + w^2 tau^2)
  up to the trapezoid error, and on the grid w_k = pi k / T it is dt times
  scipy's DCT-I (with and without the Hann window)."""
import numpy as np
import pytest

from paper_2107_08119_gb300 import inputs


def test_lag_zero_is_the_summed_heat_current(orc):
    pos, vel, box, z = inputs.config3(cells=(2, 2, 2))
    h = orc.NepHyper()
    _, _, _, J, W, v = orc.md_record(h, z, pos, vel, box, inputs.MASS_SI, 1.0, 12, fe=[1e-3, 0.0, 0.0])
    K = orc.shc(W, v, 5)
    assert np.allclose(K[0], J.sum(axis=0), rtol=1e-12, atol=1e-12 * np.abs(J).sum())
    # and J itself is W_i . v_i with W^{ab} v^b (the first index of W is free)
    Jd = np.einsum("siab,sib->sa", W, v)
    assert np.allclose(Jd, J, rtol=1e-12, atol=1e-14)


def test_constant_histories_count_the_origins():
    from oracle import oracle as orc
    rng = np.random.default_rng(2)
    n, S, L = 7, 9, 5
    W1 = rng.normal(size=(n, 3, 3))
    v1 = rng.normal(size=(n, 3))
    W = np.broadcast_to(W1, (S, n, 3, 3)).copy()
    v = np.broadcast_to(v1, (S, n, 3)).copy()
    K = orc.shc(W, v, L)
    one = np.einsum("iab,ib->a", W1, v1)
    for t in range(L):
        assert np.allclose(K[t], (S - t) * one, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("s0,s1", [(1, 4), (0, 0), (2, 6), (5, 3)])
def test_single_spikes_fix_the_lag_direction(s0, s1):
    from oracle import oracle as orc
    rng = np.random.default_rng(3 + s0 + 7 * s1)
    n, S, L = 4, 8, 6
    W = np.zeros((S, n, 3, 3))
    v = np.zeros((S, n, 3))
    A = rng.normal(size=(n, 3, 3))
    B = rng.normal(size=(n, 3))
    W[s0] = A
    v[s1] = B
    K = orc.shc(W, v, L)
    want = np.zeros((L, 3))
    if 0 <= s1 - s0 < L:
        want[s1 - s0] = np.einsum("iab,ib->a", A, B)
    assert np.allclose(K, want, rtol=1e-13, atol=1e-13)
    # a transposed W (contracting its first index) gives a different value
    if 0 <= s1 - s0 < L:
        assert not np.allclose(np.einsum("iba,ib->a", A, B), want[s1 - s0])


def test_transform_of_an_exponential_is_a_lorentzian():
    """K(t) = exp(-t / tau): the trapezoid sum is a geometric series,
    2 dt (Re 1 / (1 - q) - 1/2) with q = exp((-1/tau + i w) dt) (the tail
    beyond T is below e^-40), and tends to 2 tau / (1 + w^2 tau^2) as dt -> 0."""
    from oracle import oracle as orc
    tau, dt = 50.0, 1.0
    t = np.arange(0, 2001) * dt
    K = np.repeat(np.exp(-t / tau)[:, None], 3, axis=1)
    w = np.linspace(0.0, 0.2, 41)
    out = orc.shc_spectrum(K, dt, w)
    q = np.exp((-1.0 / tau + 1j * w) * dt)
    exact = 2.0 * dt * (np.real(1.0 / (1.0 - q)) - 0.5)
    assert np.allclose(out[:, 0], exact, rtol=1e-10, atol=1e-12)
    small = w <= 0.02
    lorentz = 2.0 * tau / (1.0 + (w * tau) ** 2)
    assert np.allclose(out[small, 0], lorentz[small], rtol=1e-3)
    assert np.allclose(out[:, 1], out[:, 0]) and np.allclose(out[:, 2], out[:, 0])


@pytest.mark.parametrize("window", [False, True])
def test_transform_on_the_dct_grid_is_scipy_dct1(window):
    from scipy.fft import dct

    from oracle import oracle as orc
    rng = np.random.default_rng(5)
    M, dt = 33, 2.5
    K = rng.normal(size=(M, 3))
    w = np.pi * np.arange(M) / ((M - 1) * dt)
    out = orc.shc_spectrum(K, dt, w, scale=0.7, window=window)
    Kw = K.copy()
    if window:
        Kw *= (0.5 * (1.0 + np.cos(np.pi * np.arange(M) / (M - 1))))[:, None]
    want = 0.7 * dt * dct(Kw, type=1, axis=0)
    assert np.allclose(out, want, rtol=1e-12, atol=1e-12)


def test_quantum_factor_is_the_oscillator_heat_capacity():
    """The quantum correction factor at x = hbar w / (k_B T) is the heat
    capacity of one quantum harmonic oscillator in units of k_B: the T
    derivative of its mean thermal energy hbar w / (e^{hbar w / k_B T} - 1).
    Checked by a central difference in the reduced temperature theta = 1/x
    (energy in units of hbar w), and by the two limits: 1 - x^2/12 + x^4/240
    at high temperature, x^2 e^{-x} at low temperature."""
    from oracle import oracle as orc
    xs = np.array([1e-3, 0.05, 0.3, 1.0, 2.5, 7.0, 15.0])
    spec = np.ones((len(xs), 3))
    f = orc.shc_quantum(spec, xs, 1.0)[:, 0]

    def energy(theta):
        return 1.0 / np.expm1(1.0 / theta)

    for x, fx in zip(xs, f):
        th, h = 1.0 / x, 1e-5 / x
        c = (energy(th + h) - energy(th - h)) / (2 * h)
        assert fx == pytest.approx(c, rel=1e-7)
    small = np.array([1e-4, 1e-3, 1e-2])
    fs = orc.shc_quantum(np.ones((3, 3)), small, 1.0)[:, 0]
    assert np.allclose(fs, 1 - small**2 / 12 + small**4 / 240, rtol=1e-14, atol=0)
    big = np.array([40.0, 60.0, 800.0])
    fb = orc.shc_quantum(np.ones((3, 3)), big, 1.0)[:, 0]
    assert np.allclose(fb, big**2 * np.exp(-big), rtol=1e-12)
    # x = 0 (w = 0) is the classical limit, and the factor is even in w
    assert np.array_equal(orc.shc_quantum(np.ones((1, 3)), [0.0], 3.0), np.ones((1, 3)))
    assert np.array_equal(orc.shc_quantum(spec, -xs, 1.0), orc.shc_quantum(spec, xs, 1.0))


def test_quantum_corrected_flat_spectrum_integrates_to_pi2_over_3():
    """A flat classical spectrum kappa(w) = 1 corrected and integrated over
    x = hbar w / k_B T gives int_0^inf x^2 e^x / (e^x - 1)^2 dx = pi^2 / 3;
    the per-row scaling leaves the three components and their ratios alone."""
    from scipy.integrate import simpson

    from oracle import oracle as orc
    x = np.linspace(0.0, 60.0, 60001)
    spec = np.tile([1.0, 2.0, -0.5], (len(x), 1))
    f = orc.shc_quantum(spec, x, 1.0)
    assert simpson(f[:, 0], x=x) == pytest.approx(np.pi**2 / 3, rel=1e-9)
    assert np.allclose(f[:, 1], 2.0 * f[:, 0]) and np.allclose(f[:, 2], -0.5 * f[:, 0])
    # omega in other units: x_per_omega scales the argument
    g = orc.shc_quantum(spec[:5], x[:5] * 4.0, 0.25)
    assert np.allclose(g, f[:5], rtol=1e-15)


def test_running_hnemd_estimate_closed_forms():
    """The running estimate scale * mean(J[0..t]): a constant current gives the
    constant; J_t = t gives t / 2; an alternating +-1 gives 1/(t+1) after even
    steps and 0 after odd ones; the three components are independent."""
    from oracle import oracle as orc
    n = 101
    t = np.arange(n, dtype=float)
    J = np.stack([np.full(n, 2.5), t, (-1.0) ** t], axis=1)
    k = orc.hnemd_kappa(J, 0.4)
    assert np.allclose(k[:, 0], 0.4 * 2.5, rtol=1e-15)
    assert np.allclose(k[:, 1], 0.4 * t / 2, rtol=1e-15, atol=0)
    want = np.where(t % 2 == 0, 1.0 / (t + 1), 0.0) * 0.4
    assert np.allclose(k[:, 2], want, rtol=1e-14, atol=1e-16)
