"""Pins of the oracle's time evolution: exact evolution of polynomial data
(Sec. 3.1.2, 3.3, 4.1), the exact lambda = 1 d'Alembert identity of the
conservative scheme, the d-dimensional conservative formula of Sec. 4.3 and
the reflection symmetry of a half-step."""
import math

import numpy as np
import pytest
from numpy.polynomial import Polynomial

from tests import polyref


def _problem(orc, d, m, variant, lam=0.7, h=0.3, c=1.3):
    return orc.Problem(d, m, 4, c, h, lam * h / c, variant, orc.PERIODIC)


@pytest.mark.parametrize("m", range(1, 7))
def test_1d_dissipative_exact_dalembert(orc, m):
    """Degree-(2m+1) u and degree-(2m-1) v are evolved exactly (Sec. 3.1.2);
    reference: d'Alembert's formula on numpy polynomials."""
    rng = np.random.default_rng(m)
    P = _problem(orc, 1, m, orc.DISSIPATIVE)
    U = Polynomial(rng.standard_normal(2 * m + 2))
    V = Polynomial(rng.standard_normal(2 * m))
    ct = P.c * P.dt / 2
    W = V.integ()
    xp, xm = Polynomial([ct, 1]), Polynomial([-ct, 1])
    u = (U(xp) + U(xm)) / 2 + (W(xp) - W(xm)) / (2 * P.c)
    v = P.c * (U.deriv()(xp) - U.deriv()(xm)) / 2 + (V(xp) + V(xm)) / 2
    cu = polyref.corner_data(U.coef, 1, P.h, m)
    cv = polyref.corner_data(V.coef, 1, P.h, m - 1)
    nu, nv = P.diss_cell(cu, cv)
    wu = polyref.scaled_derivs(u.coef, [0.0], P.h, m)
    wv = polyref.scaled_derivs(v.coef, [0.0], P.h, m - 1)
    np.testing.assert_allclose(nu, wu, rtol=0, atol=1e-12 * np.abs(wu).max())
    np.testing.assert_allclose(nv, wv, rtol=0, atol=1e-12 * np.abs(wv).max())


@pytest.mark.parametrize("d,m", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2)])
def test_full_dissipative_exact_for_low_degree(orc, d, m):
    """The d > 1 'full' method evolves data exactly when all its interpolants
    are exact, i.e. u and v of degree <= 2m-1 per axis."""
    rng = np.random.default_rng(10 * d + m)
    P = _problem(orc, d, m, orc.DISSIPATIVE)
    U = polyref.random_poly(rng, [2 * m - 1] * d)
    V = polyref.random_poly(rng, [2 * m - 1] * d)
    u, v = polyref.wave_taylor(U, V, P.dt / 2, P.c)
    nu, nv = P.diss_cell(polyref.corner_data(U, d, P.h, m), polyref.corner_data(V, d, P.h, m - 1))
    wu = polyref.scaled_derivs(u, [0.0] * d, P.h, m)
    wv = polyref.scaled_derivs(v, [0.0] * d, P.h, m - 1)
    np.testing.assert_allclose(nu, wu, atol=1e-12 * np.abs(wu).max())
    np.testing.assert_allclose(nv, wv, atol=1e-12 * np.abs(wv).max())


@pytest.mark.parametrize("d,m", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2)])
def test_simple_dissipative_exact(orc, d, m):
    """The plain tensor-product extension evolves u of degree 2m+1 and v of
    degree 2m-1 per axis exactly."""
    rng = np.random.default_rng(20 * d + m)
    P = _problem(orc, d, m, orc.DISSIPATIVE_SIMPLE)
    U = polyref.random_poly(rng, [2 * m + 1] * d)
    V = polyref.random_poly(rng, [2 * m - 1] * d)
    u, v = polyref.wave_taylor(U, V, P.dt / 2, P.c)
    nu, nv = P.diss_cell(polyref.corner_data(U, d, P.h, m), polyref.corner_data(V, d, P.h, m - 1))
    wu = polyref.scaled_derivs(u, [0.0] * d, P.h, m)
    wv = polyref.scaled_derivs(v, [0.0] * d, P.h, m - 1)
    np.testing.assert_allclose(nu, wu, atol=1e-12 * np.abs(wu).max())
    np.testing.assert_allclose(nv, wv, atol=1e-12 * np.abs(wv).max())


def test_full_differs_from_simple_for_high_degree(orc):
    """The special interpolants change the first step for degree-(2m+1) data
    (the full method does not evolve such data exactly)."""
    rng = np.random.default_rng(3)
    d, m = 2, 2
    Pf = _problem(orc, d, m, orc.DISSIPATIVE)
    Ps = _problem(orc, d, m, orc.DISSIPATIVE_SIMPLE)
    U = polyref.random_poly(rng, [2 * m + 1] * d)
    cu = polyref.corner_data(U, d, Pf.h, m)
    cv = np.zeros((4, m * m))
    assert np.abs(Pf.diss_cell(cu, cv)[1] - Ps.diss_cell(cu, cv)[1]).max() > 1e-6


@pytest.mark.parametrize("d,m", [(1, 0), (1, 1), (1, 3), (1, 5), (2, 1), (2, 3), (3, 1), (3, 2)])
def test_conservative_exact_for_polynomials(orc, d, m):
    """Eq. (update)/(convUpdate): old = exact data at -dt/2 gives exact data at +dt/2."""
    rng = np.random.default_rng(30 * d + m)
    P = _problem(orc, d, m, orc.CONSERVATIVE)
    U = polyref.random_poly(rng, [2 * m + 1] * d)
    V = polyref.random_poly(rng, [2 * m + 1] * d)
    up, _ = polyref.wave_taylor(U, V, P.dt / 2, P.c)
    um, _ = polyref.wave_taylor(U, V, -P.dt / 2, P.c)
    cu = polyref.corner_data(U, d, P.h, m)
    old = polyref.scaled_derivs(um, [0.0] * d, P.h, m)
    out = P.cons_cell(cu, old)
    want = polyref.scaled_derivs(up, [0.0] * d, P.h, m)
    np.testing.assert_allclose(out, want, atol=1e-11 * np.abs(want).max())


@pytest.mark.parametrize("d,m", [(1, 1), (1, 3), (2, 2), (3, 1)])
def test_conservative_startup_exact(orc, d, m):
    rng = np.random.default_rng(40 * d + m)
    P = _problem(orc, d, m, orc.CONSERVATIVE)
    U = polyref.random_poly(rng, [2 * m + 1] * d)
    V = polyref.random_poly(rng, [2 * m - 1] * d)
    up, _ = polyref.wave_taylor(U, V, P.dt / 2, P.c)
    out = P.cons_start_cell(polyref.corner_data(U, d, P.h, m), polyref.corner_data(V, d, P.h, m - 1))
    want = polyref.scaled_derivs(up, [0.0] * d, P.h, m)
    np.testing.assert_allclose(out, want, atol=1e-11 * np.abs(want).max())


@pytest.mark.parametrize("m", range(0, 6))
def test_conservative_lambda1_is_dalembert(orc, m):
    """At c dt = h the cosine series of Eq. (update) samples the interpolant at
    the two corners, where it equals the data: new = left + right - old."""
    rng = np.random.default_rng(50 + m)
    h = 0.37
    P = orc.Problem(1, m, 4, 1.0, h, h, orc.CONSERVATIVE, orc.PERIODIC)
    cu = rng.standard_normal((2, m + 1))
    old = rng.standard_normal(m + 1)
    out = P.cons_cell(cu, old)
    np.testing.assert_allclose(out, cu[0] + cu[1] - old, atol=2e-12 * (1 + np.abs(cu).max()))


def _pascal_update(a, m, lam, scale_2r):
    """Sec. 4.3 printed 2-D update applied to interpolant coefficients a[k,l]
    (k,l <= 2m+1): 2/(k! l!) sum_r sum_{ix+iy=r} (k+2ix)!(l+2iy)! P_{ix,iy} a,
    P_{ij} = binom(i+j,i)/(2i+2j)! lam^{2i+2j} (times 2^{-2r} if scale_2r)."""
    out = np.zeros((m + 1, m + 1))
    for k in range(m + 1):
        for l in range(m + 1):
            acc = 0.0
            for ix in range(0, m + 2):
                for iy in range(0, m + 2):
                    if k + 2 * ix > 2 * m + 1 or l + 2 * iy > 2 * m + 1:
                        continue
                    r = ix + iy
                    Pij = math.comb(r, ix) / math.factorial(2 * r) * lam ** (2 * r)
                    if scale_2r:
                        Pij *= 2.0 ** (-2 * r)
                    acc += math.factorial(k + 2 * ix) * math.factorial(l + 2 * iy) * Pij * a[k + 2 * ix, l + 2 * iy]
            out[k, l] = 2.0 / (math.factorial(k) * math.factorial(l)) * acc
    return out


@pytest.mark.parametrize("m", [1, 2, 3])
def test_conservative_2d_pascal_form(orc, m):
    """Reading of Sec. 4.3: the Pascal-matrix update with the factor 2^{-2r}
    (the Taylor weight (c dt/2h)^{2r} of Eq. update / convUpdate) equals the
    oracle's update; the form as printed does not reduce to Eq. (convUpdate)."""
    rng = np.random.default_rng(60 + m)
    h, lam = 0.25, 0.9
    P2 = orc.Problem(2, m, 4, 1.0, h, lam * h, orc.CONSERVATIVE, orc.PERIODIC)
    cu = rng.standard_normal((4, (m + 1) ** 2))
    old = np.zeros((m + 1) ** 2)
    a = orc.interp((m, m), cu)
    got = P2.cons_cell(cu, old).reshape(m + 1, m + 1)
    np.testing.assert_allclose(got, _pascal_update(a, m, lam, True), atol=1e-12 * np.abs(got).max())
    # y-independent data: 2-D update = 1-D update (Eq. convUpdate) in the l=0 row
    cu1 = rng.standard_normal((2, m + 1))
    cu2 = np.zeros((4, m + 1, m + 1))
    for s in range(4):
        cu2[s, :, 0] = cu1[s >> 1]
    P1 = orc.Problem(1, m, 4, 1.0, h, lam * h, orc.CONSERVATIVE, orc.PERIODIC)
    one = P1.cons_cell(cu1, np.zeros(m + 1))
    two = P2.cons_cell(cu2.reshape(4, -1), old).reshape(m + 1, m + 1)
    np.testing.assert_allclose(two[:, 0], one, atol=1e-13 * np.abs(one).max())
    assert np.abs(two[:, 1:]).max() == 0.0
    a2 = orc.interp((m, m), cu2.reshape(4, -1))
    printed = _pascal_update(a2, m, lam, False)
    assert np.abs(printed[:, 0] - one).max() > 1e-3 * np.abs(one).max()


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("d", [1, 2])
def test_reflection_symmetry(orc, variant, d):
    """Mirroring the data (x -> -x per axis, odd coefficients change sign)
    mirrors the result of a full step (Sec. 2.2, reflection of the cell)."""
    m, N, h = 2, 6, 1.0 / 6
    P = orc.Problem(d, m, N, 1.0, h, 0.8 * h, variant, orc.PERIODIC)
    rng = np.random.default_rng(70 + d + 3 * variant)
    n = N ** d
    u = rng.standard_normal((n, P.Nu))
    v = rng.standard_normal((n, P.Nv))

    def mirror(a, q, grid):
        a = a.reshape([N] * d + [q + 1] * d)
        for ax in range(d):
            if grid == 0:
                a = np.roll(np.flip(a, ax), 1, ax)
            else:
                a = np.flip(a, ax)
            sgn = (-1.0) ** np.arange(q + 1)
            shp = [1] * (2 * d)
            shp[d + ax] = q + 1
            a = a * sgn.reshape(shp)
        return a.reshape(n, -1)

    if variant == orc.CONSERVATIVE:
        q0 = rng.standard_normal((n, P.Nu))
        a1, b1 = P.run(u, nsteps=1, dual_u=q0)
        a2, b2 = P.run(mirror(u, m, 0), nsteps=1, dual_u=mirror(q0, m, 1))
        np.testing.assert_allclose(a2, mirror(a1, m, 0), atol=1e-12)
        np.testing.assert_allclose(b2, mirror(b1, m, 1), atol=1e-12)
    else:
        a1, b1 = P.run(u, v, nsteps=1)
        a2, b2 = P.run(mirror(u, m, 0), mirror(v, m - 1, 0), nsteps=1)
        np.testing.assert_allclose(a2, mirror(a1, m, 0), atol=1e-12)
        np.testing.assert_allclose(b2, mirror(b1, m - 1, 0), atol=1e-12)
