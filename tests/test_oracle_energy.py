"""Pins of the oracle's energies: quadrature against closed forms, the 1-D
dissipative energy decay (Sec. 3.2, Eqs. stable1, Energyeq), and the
conservative invariant (Sec. 4.2, Eq. Vconst; Sec. 5.2)."""
import math

import numpy as np
import pytest
from numpy.polynomial import Polynomial

from paper_1802_05246_b300 import inputs as I
from tests.gpu_util import hermite_cond


def _sin_state(d, m, N, a, grid=0, bc=I.PERIODIC):
    h = 1.0 / N
    return I.sine_data(d, m, N, h, bc, grid, [a] * d if d == 1 else [a] + [0.0] * (d - 1))


def test_plain_energy_quadrature_1d(orc):
    N, m, c = 32, 3, 1.7
    h = 1.0 / N
    P = orc.Problem(1, m, N, c, h, 0.5 * h / c, orc.DISSIPATIVE, orc.PERIODIC)
    a = 2 * np.pi
    u = I.sine_data(1, m, N, h, I.PERIODIC, 0, [a])
    v = I.sine_data(1, m - 1, N, h, I.PERIODIC, 0, [a], phase=np.pi / 2, amp=3.0)
    e_u = P.diss_energy(0, u, np.zeros((N, m)))[0]
    e_v = P.diss_energy(0, np.zeros((N, m + 1)), v)[0]
    np.testing.assert_allclose(e_u, c * c * a * a / 2, rtol=1e-8)
    np.testing.assert_allclose(e_v, 9.0 / 2, rtol=1e-8)


def test_plain_energy_quadrature_2d(orc):
    N, m = 16, 2
    h = 1.0 / N
    P = orc.Problem(2, m, N, 1.0, 0.5 * h, 0.5 * h, orc.DISSIPATIVE, orc.PERIODIC)
    P = orc.Problem(2, m, N, 1.0, h, 0.5 * h, orc.DISSIPATIVE, orc.PERIODIC)
    a = 2 * np.pi
    # sin(ax) sin(ay) = (cos(a(x-y)) - cos(a(x+y)))/2
    u = 0.5 * (I.sine_data(2, m, N, h, 0, 0, [a, -a], phase=np.pi / 2)
               - I.sine_data(2, m, N, h, 0, 0, [a, a], phase=np.pi / 2))
    e = P.diss_energy(0, u, np.zeros((N * N, m * m)))[0]
    np.testing.assert_allclose(e, 2 * np.pi ** 2, rtol=1e-6)
    f = P.__class__(2, m, N, 1.0, h, 0.5 * h, orc.CONSERVATIVE, orc.PERIODIC).cons_forms(0, u, u)
    np.testing.assert_allclose(f[1], 2 * np.pi ** 2, rtol=1e-6)
    np.testing.assert_allclose(f[0], a ** (4 * (m + 1)) / 4, rtol=2e-2)


@pytest.mark.parametrize("m", [1, 2, 3])
def test_seminorm_energy_quadrature_1d(orc, m):
    """c^2 |d_x I_m u|_m^2 -> c^2 int (u^(m+1))^2 as h -> 0 for u = sin(2 pi x)."""
    N = 256
    h = 1.0 / N
    P = orc.Problem(1, m, N, 1.0, h, 0.5 * h, orc.DISSIPATIVE, orc.PERIODIC)
    a = 2 * np.pi
    u = I.sine_data(1, m, N, h, 0, 0, [a])
    e = P.diss_energy(0, u, np.zeros((N, m)))[1]
    np.testing.assert_allclose(e, a ** (2 * m + 2) / 2, rtol=1e-3)


def test_boundary_half_cells(orc):
    """Dual-grid levels of non-periodic problems: boundary cells count half."""
    N, m = 40, 2
    h = 1.0 / N
    for bc, fn in ((I.DIRICHLET, 0.0), (I.NEUMANN, np.pi / 2)):
        P = orc.Problem(1, m, N, 1.0, h, 0.5 * h, orc.DISSIPATIVE, bc)
        u = I.sine_data(1, m, N, h, bc, 1, [np.pi], phase=fn)
        e = P.diss_energy(1, u, np.zeros((N, m)))[0]
        np.testing.assert_allclose(e, np.pi ** 2 / 2, rtol=1e-7)


@pytest.mark.parametrize("m", [1, 2, 3, 4])
@pytest.mark.parametrize("lam", [0.5, 0.9, 1.0])
def test_1d_dissipative_energy_nonincreasing(orc, m, lam):
    """Eq. (stable1)/(Energyeq): c^2|d_x I_m u|_m^2 + |I_{m-1} v|_m^2 does not grow
    over any half-step, and decays for rough data (random U(0,1) coefficients)."""
    N = 12
    h = 1.0 / N
    P = orc.Problem(1, m, N, 1.3, h, lam * h / 1.3, orc.DISSIPATIVE, orc.PERIODIC)
    rng = np.random.default_rng(m * 10 + int(lam * 10))
    u = rng.uniform(0, 1, (N, m + 1))
    v = rng.uniform(0, 1, (N, m))
    E = [P.diss_energy(0, u, v)[1]]
    for _ in range(15):
        du, dv = P.half_step(1, u, v)
        E.append(P.diss_energy(1, du, dv)[1])
        u, v = P.half_step(0, du, dv)
        E.append(P.diss_energy(0, u, v)[1])
    E = np.array(E)
    assert np.all(E[1:] <= E[:-1] * (1 + 1e-12)), np.diff(E) / E[:-1]
    assert E[-1] < E[0] * 0.999


@pytest.mark.parametrize("d,m,lam", [(1, 1, 0.8), (1, 3, 1.0), (1, 5, 0.6), (2, 1, 1.0), (2, 2, 0.8), (3, 1, 0.9)])
def test_conservative_invariant(orc, d, m, lam):
    """G^n = |p^{n+1/2}|^2 - <p^{n+1}, p^n> in |.|_{m+1,..,m+1} is constant; for
    random U(0,1) coefficients as in Sec. 5.2."""
    N = 6 if d > 1 else 10
    h = 1.0 / N
    P = orc.Problem(d, m, N, 1.0, h, lam * h, orc.CONSERVATIVE, orc.PERIODIC)
    rng = np.random.default_rng(d * 100 + m)
    p = rng.uniform(0, 1, (N ** d, P.Nu))
    q = rng.uniform(0, 1, (N ** d, P.Nu))
    G0 = P.cons_G(p, q)
    for _ in range(6 if d > 1 else 20):
        p, q = P.run(p, nsteps=1, dual_u=q)
        G = P.cons_G(p, q)
        assert abs(G - G0) <= 1e-11 * abs(G0), (G, G0)


def _piecewise(orc, data, m, h, centre_offset):
    """Cell polynomials (in xi) of grid data; cell i is centred at (i + off) h
    with corners data[i - 1 + (off>0)] ... returns callable giving (coef, centre)."""
    N = data.shape[0]

    def cell(x):
        if centre_offset == 0.0:  # dual data, cells centred at primal nodes
            i = int(math.floor(x / h + 0.5))
            left, right = data[(i - 1) % N], data[i % N]
            return orc.interp1d(m, left, right), i * h
        j = int(math.floor(x / h))
        left, right = data[j % N], data[(j + 1) % N]
        return orc.interp1d(m, left, right), (j + 0.5) * h

    return cell


@pytest.mark.parametrize("m", [1, 2, 3])
def test_conserved_variables_identity(orc, m):
    """Sec. 5.2 measures |P+|^2 + |P-|^2 with P(+-) = p - S(+-) p (Eq. Vdef) at
    dt = h/2 by splitting cells into quarters; it equals 2G."""
    N = 8
    h = 1.0 / N
    P = orc.Problem(1, m, N, 1.0, h, 0.5 * h, orc.CONSERVATIVE, orc.PERIODIC)
    rng = np.random.default_rng(200 + m)
    p = rng.uniform(0, 1, (N, m + 1))
    q = rng.uniform(0, 1, (N, m + 1))
    A = _piecewise(orc, q, m, h, 0.0)  # p^{n+1/2}, dual data
    B = _piecewise(orc, p, m, h, 0.5)  # p^n, primal data
    k = m + 1
    total = 0.0
    for sgn in (+1, -1):
        for s in range(4 * N):
            a0 = s * h / 4
            xm = a0 + h / 8
            ca, xa = A(xm)
            cb, xb = B(xm + sgn * h / 4)
            pa = Polynomial(ca).deriv(k)(Polynomial([(a0 - xa) / h, 1 / h])) * h ** (-k)
            pb = Polynomial(cb).deriv(k)(Polynomial([(a0 + sgn * h / 4 - xb) / h, 1 / h])) * h ** (-k)
            integ = ((pa - pb) ** 2).integ()
            total += integ(h / 4) - integ(0.0)
    G = P.cons_G(p, q)
    np.testing.assert_allclose(total, 2 * G, rtol=1e-10)


# ----------------------------------------------- d > 1: Eq. (stable2)
def _stable2_exact(d, m, wu, wv, c):
    """Limit of the Sec. 3.3 functional c^2 sum_i |d_i I^(i) u|^2_{m..m} +
    |I_{m-1} v|^2_{m..m} for u = prod sin(wu_i x_i), v = prod sin(wv_i x_i) on
    the unit cube: c^2 sum_i int (d_i^{m+1} prod_{j!=i} d_j^m u)^2 +
    int (prod_j d_j^m v)^2, every square of a product of sines or cosines
    integrating to 2^-d."""
    e = 0.0
    for i in range(d):
        t = c * c
        for j in range(d):
            t *= wu[j] ** (2 * (m + 1) if j == i else 2 * m)
        e += t
    t = 1.0
    for j in range(d):
        t *= wv[j] ** (2 * m)
    return (e + t) / 2**d


@pytest.mark.parametrize("d,m,N1,N2", [(2, 1, 16, 32), (2, 2, 16, 32), (2, 3, 16, 32), (3, 1, 8, 16), (3, 2, 8, 16),
                                       (3, 3, 6, 8)])
def test_stable2_functional_converges_to_its_closed_form(orc, d, m, N1, N2):
    """The d > 1 invariant of or_diss_energy (out[1], Eq. stable2) tends to
    its closed form as h -> 0, at the observed order 2m (the derivatives of
    order m of the degree-(2m-1) interpolants converge at h^m, squared).  The
    wave numbers differ per axis, so a derivative order given to the wrong
    axis, a wrong power of h or a dropped term changes the limit itself."""
    c = 1.3
    wu = [2 * np.pi, 4 * np.pi, 2 * np.pi][:d]
    wv = [4 * np.pi, 2 * np.pi, 6 * np.pi][:d]
    exact = _stable2_exact(d, m, wu, wv, c)
    errs = []
    for N in (N1, N2):
        h = 1.0 / N
        P = orc.Problem(d, m, N, c, h, 0.5 * h / c, orc.DISSIPATIVE, orc.PERIODIC)
        u = I.tensor_data([I.sine_data(1, m, N, h, 0, 0, [wu[i]]) for i in range(d)])
        v = I.tensor_data([I.sine_data(1, m - 1, N, h, 0, 0, [wv[i]]) for i in range(d)])
        errs.append(abs(P.diss_energy(0, u, v)[1] - exact) / exact)
    order = np.log(errs[0] / errs[1]) / np.log(N2 / N1)
    assert order >= 2 * m - 0.5, (errs, order)
    assert errs[1] < (0.06 if m == 1 else 2e-3), errs


# ------------------------------------------- long runs (Sec. 5.2, E2)
@pytest.mark.parametrize("m", [1, 3, 5])
@pytest.mark.parametrize("data", ["random", "sine"])
def test_conservative_invariant_long_run(orc, m, data):
    """Sec. 5.2: the conservative method conserves its energy to round-off over
    long runs.  1-D periodic on [0, 2 pi), h = 2 pi / 30, dt = h/2, 10^4 full
    steps, G checked every 10^3 steps.
    Random U(0,1) coefficients: |G^n - G^0| <= sqrt(n) 1e-12 |G^0|.
    sin x cos t: the seminorm of smooth data is carried by its top
    coefficients, whose rounding in the oracle's LU solve (forward error
    ~ eps * cond of the Eq. Hermcon system) accumulates step after step, so the
    bound is linear: |G^n - G^0| <= n 8 eps cond |p|^2_{m+1}; for m = 5 the
    state itself stays within 1e-9 of the exact solution."""
    N = 30
    h = 2 * np.pi / N
    dt = h / 2
    P = orc.Problem(1, m, N, 1.0, h, dt, orc.CONSERVATIVE, orc.PERIODIC)
    if data == "random":
        rng = np.random.default_rng(m)
        p, q = rng.uniform(0, 1, (N, m + 1)), rng.uniform(0, 1, (N, m + 1))
    else:
        p = I.sine_data(1, m, N, h, 0, 0, [1.0])
        q = np.cos(dt / 2) * I.sine_data(1, m, N, h, 0, 1, [1.0])
    G0 = P.cons_G(p, q)
    scale = P.cons_forms(0, p, p)[0]
    n = 0
    for _ in range(10):
        p, q = P.run(p, nsteps=1000, dual_u=q)
        n += 1000
        dG = abs(P.cons_G(p, q) - G0)
        if data == "random":
            assert dG <= np.sqrt(n) * 1e-12 * abs(G0), (n, dG / abs(G0))
        else:
            assert dG <= n * 8 * np.finfo(float).eps * hermite_cond(m) * scale, (n, dG)
    if data == "sine" and m == 5:
        pe = np.cos(n * dt) * I.sine_data(1, m, N, h, 0, 0, [1.0])
        assert np.linalg.norm(p - pe) <= 1e-9 * np.linalg.norm(pe)
