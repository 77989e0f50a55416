"""Observed orders of the oracle against the paper's predictions: dissipative
2m-1 (lambda<1) and 2m (lambda=1), conservative 2m and 2m+2 (Sec. 3.4, 4.4,
5.1, 5.3; Thm. thm:diss1d, cconthm).  Single Fourier modes and short runs
are superconvergent for the conservative scheme, so the lambda < 1
conservative rate of 2m is checked on the long E1 run of Sec. 5.1."""
import math

import numpy as np
import pytest

from paper_1802_05246_b300 import inputs as I


def _slope(Ns, errs):
    x = np.log(1.0 / np.asarray(Ns, float))
    y = np.log(np.asarray(errs))
    return np.polyfit(x, y, 1)[0]


def _gauss1d(orc, m, N, lam, variant, w=0.12, T=0.5):
    h = 1.0 / N
    nsteps = int(math.ceil(T / (lam * h)))
    dt = T / nsteps
    P = orc.Problem(1, m, N, 1.0, h, dt, variant, orc.PERIODIC)
    u0 = I.gaussian_data(1, m, N, h, I.PERIODIC, 0, [[0.5]], [w], [1.0])
    if variant == orc.CONSERVATIVE:
        u, _ = P.run(u0, nsteps=nsteps, dual_u=P.cons_start(u0))
    else:
        u, _ = P.run(u0, np.zeros((N, m)), nsteps=nsteps)
    t = nsteps * dt

    def g(s):
        return I.gaussian_1d(s.reshape(-1), 0, 1.0, 0.5, w, 1.0, I.PERIODIC)[:, 0].reshape(s.shape)

    return P.l2_error(0, u, 2 * m + 4, lambda X: 0.5 * (g(X[..., 0] - t) + g(X[..., 0] + t)))


@pytest.mark.parametrize("m", [1, 2, 3])
@pytest.mark.parametrize("lam", [0.8, 1.0])
def test_1d_dissipative_order(orc, m, lam):
    Ns = [16, 24, 32, 48]
    errs = [_gauss1d(orc, m, N, lam, orc.DISSIPATIVE) for N in Ns]
    p = 2 * m - 1 if lam < 1 else 2 * m
    assert abs(_slope(Ns, errs) - p) <= 0.35, (errs, _slope(Ns, errs))


@pytest.mark.parametrize("m", [1, 2, 3])
def test_1d_conservative_order_lambda1(orc, m):
    Ns = [16, 24, 32, 48]
    errs = [_gauss1d(orc, m, N, 1.0, orc.CONSERVATIVE) for N in Ns]
    assert abs(_slope(Ns, errs) - (2 * m + 2)) <= 0.35


@pytest.mark.parametrize("m", [1, 2, 3])
def test_1d_conservative_order_lambda08_at_least(orc, m):
    Ns = [16, 24, 32, 48]
    errs = [_gauss1d(orc, m, N, 0.8, orc.CONSERVATIVE) for N in Ns]
    assert _slope(Ns, errs) >= 2 * m - 0.3


def test_e1_gaussian_box_conservative(orc):
    """Sec. 5.1 experiment E1 (m=1): u0 = exp(-20 x^2) on [-3/2,3/2] (shifted to
    [0,3]), Dirichlet, run to t ~ 12.25; order 2m at lambda = 0.8 and 2m+2 at 1."""
    w, L = 1 / math.sqrt(20.0), 3.0

    def g(s):
        return I.gaussian_1d(s.reshape(-1), 0, 1.0, 1.5, w, L, I.DIRICHLET)[:, 0].reshape(s.shape)

    for lam, p in ((0.8, 2), (1.0, 4)):
        errs = []
        Ns = [40, 48, 58, 70]
        for N in Ns:
            h = L / N
            nsteps = int(round(12.25 / (lam * h)))
            P = orc.Problem(1, 1, N, 1.0, h, lam * h, orc.CONSERVATIVE, orc.DIRICHLET)
            u0 = I.gaussian_data(1, 1, N, h, I.DIRICHLET, 0, [[1.5]], [w], [1.0])
            u, _ = P.run(u0, nsteps=nsteps, dual_u=P.cons_start(u0))
            t = nsteps * lam * h
            errs.append(P.l2_error(0, u, 6, lambda X: 0.5 * (g(X[..., 0] - t) + g(X[..., 0] + t))))
        assert abs(_slope(Ns, errs) - p) <= 0.35, (lam, errs)


def _plane2d(orc, m, N, lam, variant, T=0.25):
    kap = m + 1
    h = 1.0 / N
    nsteps = int(math.ceil(T / (lam * h)))
    dt = T / nsteps
    P = orc.Problem(2, m, N, 1.0, h, dt, variant, orc.PERIODIC)
    a = 2 * np.pi * kap
    om = a * math.sqrt(2.0)
    u0 = I.sine_data(2, m, N, h, I.PERIODIC, 0, [a, a])
    t = nsteps * dt
    if variant == orc.CONSERVATIVE:
        q = I.sine_data(2, m, N, h, I.PERIODIC, 1, [a, a], phase=om * dt / 2)
        u, _ = P.run(u0, nsteps=nsteps, dual_u=q)
    else:
        v0 = I.sine_data(2, m - 1, N, h, I.PERIODIC, 0, [a, a], phase=np.pi / 2, amp=om)
        u, _ = P.run(u0, v0, nsteps=nsteps)
    return P.l2_error(0, u, 2 * m + 4, lambda X: np.sin(a * (X[..., 0] + X[..., 1]) + om * t))


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("lam", [0.8, 1.0])
@pytest.mark.parametrize("m", [1, 2])
def test_2d_plane_wave_order(orc, variant, lam, m):
    """Sec. 5.3 (E3): plane wave sin(2 pi kappa (x + y + sqrt2 t)), kappa = m+1."""
    Ns = [8, 12, 16, 24]
    errs = [_plane2d(orc, m, N, lam, variant) for N in Ns]
    if variant == orc.CONSERVATIVE:
        p = 2 * m + 2 if lam == 1.0 else 2 * m
    else:
        p = 2 * m if lam == 1.0 else 2 * m - 1
    assert _slope(Ns, errs) >= p - 0.35, (errs, _slope(Ns, errs))


@pytest.mark.parametrize("m", [1, 2, 3])
@pytest.mark.parametrize("lam", [0.5, 0.7])
def test_conservative_truncation_constant(orc, m, lam):
    """Sec. 4.4 (Eq. Ctrunc): the one-step error of the conservative update
    from exact data (primal level at 0, dual level at dt/2, target at dt) is
    2^-(2m+1) h^(2m+2) (lam^2 - 1)^(m+1) u^(2m+2) / (2m+2)! to leading order:
    the cosine propagator acts on a polynomial by d'Alembert's formula,
    2 C f(0) = f(c dt/2) + f(-c dt/2), and the interpolation error is
    -(x^2 - h^2/4)^(m+1) u^(2m+2) / (2m+2)! (Eq. Imtrunc).  This is Eq. Ctrunc
    with (c dt)^2 in place of (c dt / 2)^2; the lam- and m-dependence are the
    paper's.  u = sin x cos t, h = 2 pi / N: the ratio of the error to this
    constant tends to 1 at the rate h^2."""
    ratios = []
    for N in (16, 32):
        h = 2 * np.pi / N
        dt = lam * h
        P = orc.Problem(1, m, N, 1.0, h, dt, orc.CONSERVATIVE, orc.PERIODIC)
        p0 = I.sine_data(1, m, N, h, 0, 0, [1.0])
        q = math.cos(dt / 2) * I.sine_data(1, m, N, h, 0, 1, [1.0])
        new = P.half_step(0, q, dst_u=p0)
        ex = math.cos(dt) * I.sine_data(1, m, N, h, 0, 0, [1.0])
        err = ex[:, 0] - new[:, 0]
        lead = 2.0 ** (-(2 * m + 1)) * h ** (2 * m + 2) * (lam**2 - 1) ** (m + 1) / math.factorial(2 * m + 2)
        pred = lead * (-1) ** (m + 1) * np.sin(np.arange(N) * h)  # u^(2m+2) of sin x
        i = int(np.argmax(np.abs(pred)))
        ratios.append(err[i] / pred[i])
    assert abs(ratios[1] - 1) <= 0.02, ratios
    assert abs(ratios[1] - 1) < abs(ratios[0] - 1), ratios


@pytest.mark.parametrize("m", [1, 2, 3])
@pytest.mark.parametrize("lam", [0.5, 0.7, 0.9])
def test_dissipative_truncation_constant_nu(orc, m, lam):
    """Sec. 3.2 (Eq. vtrunc): with u = 0 and v = sin x at t = 0 only the
    velocity term of the half-step's velocity error survives,
    lam h/2 * nu h^(2m-1) v^(2m) with nu = 2^-(2m-1) / (2m)! (lam^2-1)^m / lam;
    the ratio of the oracle's error at the dual nodes to it tends to 1."""
    ratios = []
    for N in (16, 32):
        h = 2 * np.pi / N
        dt = lam * h
        P = orc.Problem(1, m, N, 1.0, h, dt, orc.DISSIPATIVE, orc.PERIODIC)
        v0 = I.sine_data(1, m - 1, N, h, 0, 0, [1.0])
        _, dv = P.half_step(1, np.zeros((N, m + 1)), v0)
        xd = (np.arange(N) + 0.5) * h
        err = math.cos(dt / 2) * np.sin(xd) - dv[:, 0]
        nu = 2.0 ** (-(2 * m - 1)) / math.factorial(2 * m) * (lam**2 - 1) ** m / lam
        pred = lam * h / 2 * nu * h ** (2 * m - 1) * (-1) ** m * np.sin(xd)
        i = int(np.argmax(np.abs(pred)))
        ratios.append(err[i] / pred[i])
    assert abs(ratios[1] - 1) <= 0.005, ratios
    assert abs(ratios[1] - 1) < abs(ratios[0] - 1), ratios
