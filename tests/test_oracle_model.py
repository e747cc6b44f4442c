"""Pins for the oracle's SCH discretisation (oracle/model.py).

Each test checks the oracle against something the paper and the mathematics
fix, not against a retyped copy of its own formulas:
* cyclic tridiagonal solves against a dense LAPACK solve;
* the P1 mass / stiffness symbols and the Helmholtz relation (Eq. sde1) on
  discrete Fourier modes, where they are exact, and their continuum limit;
* the closed-form element assembly against 3-point Gauss quadrature of the
  weak form of Eq. fde1, and the fixed point of the step against that residual;
* the linearised viscous decay of Fourier modes (closed-form amplification);
* exact conservation of H = 1/2 (m, u) by the midpoint rule at mu = 0 with no
  noise, and refinement behaviour of (m, 1);
* a travelling CH peakon keeping its speed c;
* the mode-expansion SALT noise on its Fourier content: each slot's unit increment
  excites exactly its wavenumber, sin slots in the imaginary and cos slots in the
  real part of the FFT, with amplitude a_j n / 2.
"""
import math

import numpy as np
import pytest

from oracle.model import Model


def make(n=64, L=40.0, alpha=1.0, mu=0.02, dt=0.025, K=4, tol=1e-13):
    return Model(L=L, n=n, alpha=alpha, mu=mu, dt=dt, amps=np.full(K // 2, 0.05), tol=tol)


def test_cyclic_solve_matches_dense():
    r = np.random.default_rng(0)
    for n in (3, 4, 7, 32):
        a, c = r.normal(size=n), r.normal(size=n)
        b = np.abs(a) + np.abs(c) + 1.0 + r.random(n)
        d = r.normal(size=n)
        x = Model.solve((a, b, c), d)
        ref = np.linalg.solve(Model.dense((a, b, c)), d)
        assert np.allclose(x, ref, rtol=1e-13, atol=1e-13)


def _fourier(n, j):
    i = np.arange(n)
    return np.cos(2 * math.pi * j * i / n), 2 * math.pi * j / n


@pytest.mark.parametrize("j", [0, 1, 5, 17])
def test_mass_stiffness_symbols(j):
    m = make(n=64)
    v, th = _fourier(m.n, j)
    Mv = Model.apply(m.mass(), v)
    Kv = Model.apply(m.stiffness(), v)
    assert np.allclose(Mv, m.h / 6 * (4 + 2 * math.cos(th)) * v, atol=1e-14)
    assert np.allclose(Kv, (2 - 2 * math.cos(th)) / m.h * v, atol=1e-12)


@pytest.mark.parametrize("j", [1, 3, 11])
def test_helmholtz_on_fourier_modes(j):
    m = make(n=128, alpha=1.3)
    v, th = _fourier(m.n, j)
    Mh = m.h / 6 * (4 + 2 * math.cos(th))
    Kh = (2 - 2 * math.cos(th)) / m.h
    ratio = (Mh + m.alpha ** 2 * Kh) / Mh
    assert np.allclose(m.m_from_u(v), ratio * v, rtol=0, atol=1e-13 * ratio)
    assert np.allclose(m.u_from_m(v), v / ratio, rtol=0, atol=1e-14)


def _matern(n=128, kappa=0.7, eta=1.3, k=3, L=40.0):
    return Model(L=L, n=n, alpha=1.0, mu=0.02, dt=0.025, amps=np.full(2, 0.05), noise_model="matern",
                 kappa=kappa, eta=eta, matern_k=k)


@pytest.mark.parametrize("j", [0, 1, 4, 13])
@pytest.mark.parametrize("k", [1, 3])
def test_matern_noise_on_fourier_modes(j, k):
    # cell values cos / sin(theta (c + 1/2)), theta = 2 pi j / n: the load is
    # eta sqrt(h) cos(theta/2) times the nodal mode, and each solve divides by
    # the symbol of M + kappa^-2 K, each later load multiplies by that of M
    m = _matern(k=k)
    th = 2 * math.pi * j / m.n
    c = np.arange(m.n) + 0.5
    i = np.arange(m.n)
    Mh = m.h / 6 * (4 + 2 * math.cos(th))
    Gh = Mh + m.kappa ** -2 * (2 - 2 * math.cos(th)) / m.h
    amp = m.eta * math.sqrt(m.h) * math.cos(th / 2) * Mh ** (k - 1) / Gh ** k
    for f in (np.cos, np.sin):
        assert np.allclose(m.noise(f(th * c)), amp * f(th * i), rtol=0, atol=1e-12 * max(amp, 1e-3))


def test_matern_noise_constant_field_and_drift():
    # w = 1 on every cell: every load and solve keeps the constant, U = eta / sqrt(h);
    # the drift enters as dW + lambda dt
    m = _matern()
    assert np.allclose(m.noise(np.ones(m.n)), m.eta / math.sqrt(m.h), rtol=1e-13)
    r = np.random.default_rng(3)
    dW, lam = r.normal(size=m.n), r.normal(size=m.n)
    assert np.allclose(m.noise(dW, lam), m.noise(dW + m.dt * lam), rtol=1e-13, atol=1e-15)
    assert m.Q == m.n


def test_matern_noise_continuum_limit():
    # a smooth cell field f(x) = cos(2 pi j x / L): the load is (h^-1/2 f, phi_i), so
    # dU -> eta h^-1/2 (1 + (2 pi j / (L kappa))^2)^-k f at the nodes, with an O(h^2) error
    j, errs = 3, []
    for n in (64, 128, 256):
        m = _matern(n=n)
        x = (np.arange(n) + 0.5) * m.h
        ref = m.eta / math.sqrt(m.h) * (1 + (2 * math.pi * j / (m.L * m.kappa)) ** 2) ** -m.matern_k
        dU = m.noise(np.cos(2 * math.pi * j * x / m.L))
        errs.append(np.max(np.abs(dU - ref * np.cos(2 * math.pi * j * m.x / m.L))) / ref)
    assert errs[0] < 0.05
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_helmholtz_continuum_limit():
    # m/u -> 1 + alpha^2 k^2 with O(h^2) error for the fixed physical wavenumber k
    errs = []
    for n in (64, 128, 256):
        m = make(n=n)
        v, _ = _fourier(n, 3 * n // 64)
        v, _ = _fourier(n, 3)
        k = 2 * math.pi * 3 / m.L
        ratio = m.m_from_u(v)[0] / v[0]
        errs.append(abs(ratio - (1 + k * k)))
    assert errs[1] < errs[0] / 3.5 and errs[2] < errs[1] / 3.5


def test_assembly_matches_gauss_quadrature():
    r = np.random.default_rng(1)
    m = make(n=16)
    m0, m1, dU = r.normal(size=(3, m.n))
    u0, u1 = m.u_from_m(m0), m.u_from_m(m1)
    R = m.residual(m1, m0, u1, u0, dU)
    Rq = m.residual_quadrature(m1, m0, dU)
    assert np.allclose(R, Rq, rtol=0, atol=1e-13 * np.max(np.abs(Rq)))


@pytest.mark.parametrize("scheme", ["li", "ea"])
def test_step_solves_fde1(scheme):
    r = np.random.default_rng(2)
    m = make(n=32)
    m.scheme = scheme
    x = m.x
    u0 = 0.2 / np.cosh(x - 27) + 0.5 / np.cosh(x - 13)
    m0 = m.m_from_u(u0)
    dU = m.noise(r.normal(scale=math.sqrt(m.dt), size=m.K), r.normal(size=m.K))
    m1, u1, it, ok = m.step(m0, u0, dU)
    assert ok and 2 <= it < 30
    Rq = m.residual_quadrature(m1, m0, dU)
    scale = np.max(np.abs(m.residual_quadrature(m0 + 0.0, m0, 0 * dU))) + np.max(np.abs(Model.apply(m.mass(), m1 - m0)))
    assert np.max(np.abs(Rq)) <= 1e-12 * scale


@pytest.mark.parametrize("j", [1, 4, 9])
def test_linear_viscous_decay(j):
    m = make(n=128, mu=0.05)
    v, th = _fourier(m.n, j)
    eps = 1e-8
    m0 = eps * v
    m1, _, _, ok = m.step(m0, m.u_from_m(m0), np.zeros(m.n))
    Mh = m.h / 6 * (4 + 2 * math.cos(th))
    Kh = (2 - 2 * math.cos(th)) / m.h
    g = (Mh - 0.5 * m.mu * m.dt * Kh) / (Mh + 0.5 * m.mu * m.dt * Kh)
    assert ok
    assert np.max(np.abs(m1 - g * m0)) <= 1e-7 * eps


def test_viscous_decay_continuum_limit():
    # the per-step amplification tends to exp(-mu k^2 dt) as h -> 0 (O(h^2) in space)
    j, mu, dt, L = 3, 0.05, 0.025, 40.0
    k = 2 * math.pi * j / L
    errs = []
    for n in (64, 256):
        th = 2 * math.pi * j / n
        h = L / n
        Mh = h / 6 * (4 + 2 * math.cos(th))
        Kh = (2 - 2 * math.cos(th)) / h
        g = (Mh - 0.5 * mu * dt * Kh) / (Mh + 0.5 * mu * dt * Kh)
        m = make(n=n, mu=mu)
        v, _ = _fourier(n, j)
        m1, _, _, _ = m.step(1e-8 * v, m.u_from_m(1e-8 * v), np.zeros(n))
        assert abs(m1[0] / (1e-8 * v[0]) - g) < 1e-9
        errs.append(abs(g - math.exp(-mu * k * k * dt)))
    assert errs[1] < errs[0] / 10


def test_energy_conserved_inviscid_noiseless():
    m = make(n=128, mu=0.0)
    x = m.x
    u0 = 0.2 / np.cosh(x - 27) + 0.5 / np.cosh(x - 13)
    m0 = m.m_from_u(u0)
    E0 = m.energy(m0)
    mm, uu = m0, u0
    for _ in range(20):
        mm, uu, _, ok = m.step(mm, uu, np.zeros(m.n))
        assert ok
    assert abs(m.energy(mm) - E0) <= 1e-11 * E0
    # with viscosity the energy decays
    mv = make(n=128, mu=0.05)
    m2, _, _, _ = mv.window(m0, np.zeros((20, mv.K)))
    assert mv.energy(m2) < E0


def test_momentum_integral_drift_shrinks_with_refinement():
    drifts = []
    for n in (64, 256):
        m = make(n=n, mu=0.0)
        x = m.x
        u0 = 0.2 / np.cosh(x - 27) + 0.5 / np.cosh(x - 13)
        m0 = m.m_from_u(u0)
        m1, _, _, _ = m.window(m0, np.zeros((40, m.K)))
        drifts.append(abs(m.mass_integral(m1) - m.mass_integral(m0)))
    assert drifts[1] < drifts[0] / 4 or drifts[1] < 1e-13


@pytest.mark.slow
def test_peakon_speed():
    L, alpha, c = 40.0, 1.0, 0.5
    n = 1024
    m = make(n=n, L=L, alpha=alpha, mu=0.0)
    x = m.x
    x0 = 10.0
    d = np.mod(x - x0, L)
    u0 = c * np.cosh((d - L / 2) / alpha) / np.cosh(L / (2 * alpha))
    mm = m.m_from_u(u0)
    uu = u0
    T = 10.0
    nsteps = int(round(T / m.dt))
    for _ in range(nsteps):
        mm, uu, _, ok = m.step(mm, uu, np.zeros(n))
        assert ok
    # crest: the peak of u, refined by the intersection of the two straight flanks
    i = int(np.argmax(uu))
    sl = (uu[i - 1] - uu[i - 3]) / (2 * m.h)
    sr = (uu[i + 3] - uu[i + 1]) / (2 * m.h)
    xl, xr = x[i - 2], x[i + 2]
    ul, ur = uu[i - 2], uu[i + 2]
    xc = (ur - ul + sl * xl - sr * xr) / (sl - sr)
    speed = (xc - x0) / T
    assert abs(speed - c) < 0.02 * c


def test_both_picard_schemes_reach_the_same_step():
    r = np.random.default_rng(9)
    li = make(n=128)
    ea = make(n=128)
    ea.scheme = "ea"
    x = li.x
    u0 = 0.2 / np.cosh(x - 27) + 0.5 / np.cosh(x - 13)
    m0 = li.m_from_u(u0)
    dW = r.normal(scale=math.sqrt(li.dt), size=(5, li.K))
    a = li.window(m0, dW)
    b = ea.window(m0, dW)
    assert a[3] and b[3]
    assert np.max(np.abs(a[0] - b[0])) <= 1e-12 * np.max(np.abs(a[0]))
    # explicit advection contracts more slowly
    assert b[2].sum() >= a[2].sum()


@pytest.mark.parametrize("j", [1, 5])
def test_exp1_field_on_constant_and_fourier_loads(j):
    # |W| = c on every cell: each (I - d_xx) solve keeps the constant, u = a^2 c + b^2.
    # |W| = c + d cos(theta (cell + 1/2)) (c > d): the cosine part follows the symbols
    # of M + K and M, as in the Matern map with kappa = 1
    m = make(n=128)
    a, b, c, d = 1.3, -0.7, 0.4, 0.25
    assert np.allclose(m.exp1_field(np.full(m.n, -c), a, b), a * a * c + b * b, rtol=1e-13)
    th = 2 * math.pi * j / m.n
    cells = c + d * np.cos(th * (np.arange(m.n) + 0.5))
    Mh = m.h / 6 * (4 + 2 * math.cos(th))
    Sh = Mh + (2 - 2 * math.cos(th)) / m.h
    amp = d * m.h * math.cos(th / 2) * Mh ** 2 / Sh ** 3
    ref = a * a * (c + amp * np.cos(th * np.arange(m.n))) + b * b
    assert np.allclose(m.exp1_field(cells, a, b), ref, rtol=0, atol=1e-13)


def test_exp1_prior_is_positive_and_reproducible():
    # the solves of (I - d_xx) keep a nonnegative load nonnegative (an M-matrix inverse
    # applied to nonnegative data), so u >= b^2 >= 0 for every member
    m = make(n=128)
    mm, u = m.prior_exp1(7, 6)
    assert np.all(u >= 0.0)
    mm2, u2 = m.prior_exp1(7, 3, particle0=3)
    assert np.array_equal(u[3:], u2)
    assert np.allclose(np.stack([m.u_from_m(x) for x in mm]), u, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("n", [32, 64])
def test_prior_sample_fourier_symbol(n):
    # the prior (reading c-13 of Eq. init_solve): u_p = u_truth + s (a_p S^3 W_p + b_p) with W_p
    # the DG0 field of cell values sqrt(h) z_c.  Its load h/2 (W_{i-1} + W_i) multiplies the
    # half-cell-shifted cell DFT by h cos(theta/2); each of the three P1 solves of
    # (U, v) + (U', v') divides by the symbol G = M + K, and the two mass products between
    # them multiply by M.  So the DFT of S^3 W is h cos(theta/2) M^2 / G^3 times that of W,
    # checked here through np.fft on the oracle's output and its keyed draws
    from oracle import rng
    m = make(n=n)
    u_truth = np.cos(2 * math.pi * m.x / m.L) + 0.3 * np.sin(6 * math.pi * m.x / m.L)
    seed, N, scale = 5, 3, 0.05
    mm, u = m.prior_sample(u_truth, seed, N, scale)
    z = rng.normals(seed, rng.TAG_INIT, m.n + 2, np.uint64(0), np.arange(N, dtype=np.uint64), np.uint64(0))
    th = 2 * math.pi * np.arange(n) / n
    Mh = m.h / 6 * (4 + 2 * np.cos(th))
    Gh = Mh + (2 - 2 * np.cos(th)) / m.h
    sym = m.h * np.cos(th / 2) * Mh ** 2 / Gh ** 3
    for p in range(N):
        a, b = z[p, n], z[p, n + 1]
        S3W = (u[p] - u_truth - scale * b) / (scale * a)
        W_hat = np.exp(-0.5j * th) * np.fft.fft(math.sqrt(m.h) * z[p, :n])
        U_hat = np.fft.fft(S3W)
        assert np.allclose(U_hat, sym * W_hat, rtol=0, atol=1e-11 * np.max(np.abs(U_hat)))
        # the momenta are the velocities' through the Helmholtz relation (pinned above)
        assert np.allclose(mm[p], m.m_from_u(u[p]), rtol=1e-13, atol=1e-13)
    # scale 0 gives the truth itself
    _, u0 = m.prior_sample(u_truth, seed, N, 0.0)
    assert np.array_equal(u0, np.tile(u_truth, (N, 1)))


@pytest.mark.parametrize("n,amps", [(64, [0.05, 0.05]), (256, [0.05 / j for j in range(1, 9)])])
def test_mode_noise_fourier_content(n, amps):
    """The mode-expansion noise (Sec. 2; SALT mode functions read as K/2 wavenumbers x
    {sin, cos}): for the unit increment of slot k, the nodal field noise(e_k) has, under the
    FFT (x_m -> sum_m x_m exp(-2 pi i q m / n)), energy only at wavenumbers q = j and n - j,
    with j = k // 2 + 1.  A sin slot (even k) gives X_j = -i a_j n / 2 (purely imaginary), a
    cos slot (odd k) X_j = a_j n / 2 (purely real).  A swapped sin/cos slot, a wrong
    wavenumber factor or a wrong amplitude fails; the drift enters as dW + lambda dt."""
    m = Model(L=40.0, n=n, alpha=1.0, mu=0.02, dt=0.025, amps=np.array(amps))
    K = 2 * len(amps)
    for k in range(K):
        e = np.zeros(K)
        e[k] = 1.0
        X = np.fft.fft(m.noise(e))
        j = k // 2 + 1
        a = amps[j - 1]
        expect = np.zeros(n, dtype=complex)
        if k % 2 == 0:
            expect[j], expect[n - j] = -0.5j * a * n, 0.5j * a * n
        else:
            expect[j], expect[n - j] = 0.5 * a * n, 0.5 * a * n
        assert np.max(np.abs(X - expect)) <= 1e-12 * n
    rng = np.random.default_rng(5)
    dW, lam = rng.normal(size=K), rng.normal(size=K)
    assert np.allclose(m.noise(dW, lam), m.noise(dW + m.dt * lam), rtol=0, atol=1e-15)
    # the noise of a general increment is the sum of its slots' fields (linearity)
    assert np.allclose(m.noise(dW), sum(dW[k] * m.noise(np.eye(K)[k]) for k in range(K)), rtol=0, atol=1e-14)
