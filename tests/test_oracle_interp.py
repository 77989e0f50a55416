"""Pins of the oracle's Hermite interpolation (Sec. 2.2, Eqs. Hermn, Hermcon,
Hermn2, Hermcon2; properties Eq. orthlem, Pyth, Imtrunc)."""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import polynomial as npoly

from tests import polyref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hermite_basis_s.txt")


def _s_to_xi(coef_s):
    """Coefficients in s = xi + 1/2 -> coefficients in xi."""
    return polyref.shift_scale(np.asarray(coef_s, float), [0.5], 1.0)


def test_textbook_basis_golden(orc):
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 10
    for r in rows:
        m, corner, l = int(r[0]), int(r[1]), int(r[2])
        coef_s = np.array([float(x) for x in r[3:]])
        left = np.zeros(m + 1)
        right = np.zeros(m + 1)
        # the scaled datum f^(l)/l! = 1 corresponds to f^(l) = l!
        (left if corner == 0 else right)[l] = 1.0
        a = orc.interp1d(m, left, right)
        want = math.factorial(l) * _s_to_xi(coef_s)
        want = np.pad(want, (0, 2 * m + 2 - want.size))
        np.testing.assert_allclose(a, want, atol=1e-14)


@pytest.mark.parametrize("q", range(0, 7))
def test_reproduces_polynomials(orc, q):
    rng = np.random.default_rng(100 + q)
    for _ in range(5):
        C = rng.standard_normal(2 * q + 2)
        left = polyref.scaled_derivs(C, [-0.5], 1.0, q)
        right = polyref.scaled_derivs(C, [0.5], 1.0, q)
        a = orc.interp1d(q, left, right)
        np.testing.assert_allclose(a, C, atol=1e-12 * np.abs(C).max())


@pytest.mark.parametrize("q", range(0, 7))
def test_leading_error_exact_for_monomial(orc, q):
    """Eq. (Imtrunc) is exact for x^{2q+2}: I f - f = -(x^2 - h^2/4)^{q+1}."""
    n = 2 * q + 2
    C = np.zeros(n + 1)
    C[n] = 1.0
    left = polyref.scaled_derivs(C, [-0.5], 1.0, q)
    right = polyref.scaled_derivs(C, [0.5], 1.0, q)
    a = orc.interp1d(q, left, right)
    diff = np.pad(a, (0, 1)) - C
    want = -npoly.polypow([-0.25, 0.0, 1.0], q + 1)
    np.testing.assert_allclose(diff, want, atol=1e-12)


@pytest.mark.parametrize("q", range(0, 7))
def test_matches_numpy_solve(orc, q):
    n = 2 * q + 2
    A = np.zeros((n, n))
    for s, xi in enumerate((-0.5, 0.5)):
        for l in range(q + 1):
            for j in range(l, n):
                A[s * (q + 1) + l, j] = math.comb(j, l) * xi ** (j - l)
    rng = np.random.default_rng(7 + q)
    b = rng.standard_normal(n)
    a = orc.interp1d(q, b[: q + 1], b[q + 1 :])
    np.testing.assert_allclose(a, np.linalg.solve(A, b), rtol=1e-11, atol=1e-12)


def _seminorm_ip(f, g, k):
    """int_{-1/2}^{1/2} f^(k) g^(k) dxi for coefficient vectors f, g."""
    fk = npoly.polyder(f, k) if len(f) > k else np.zeros(1)
    gk = npoly.polyder(g, k) if len(g) > k else np.zeros(1)
    p = npoly.polyint(npoly.polymul(fk, gk))
    return npoly.polyval(0.5, p) - npoly.polyval(-0.5, p)


@pytest.mark.parametrize("q", range(0, 6))
def test_orthogonality_and_pythagoras(orc, q):
    """Eq. (orthlem) and (Pyth) on a cell for rough (high-degree) functions."""
    rng = np.random.default_rng(11 + q)
    for _ in range(4):
        u = rng.standard_normal(2 * q + 7)
        v = rng.standard_normal(2 * q + 7)
        Iu = orc.interp1d(q, polyref.scaled_derivs(u, [-0.5], 1, q), polyref.scaled_derivs(u, [0.5], 1, q))
        Iv = orc.interp1d(q, polyref.scaled_derivs(v, [-0.5], 1, q), polyref.scaled_derivs(v, [0.5], 1, q))
        e = npoly.polysub(v, Iv)
        ortho = _seminorm_ip(Iu, e, q + 1)
        scale = math.sqrt(_seminorm_ip(Iu, Iu, q + 1) * _seminorm_ip(e, e, q + 1)) + 1e-300
        assert abs(ortho) <= 1e-11 * scale
        lhs = _seminorm_ip(v, v, q + 1)
        rhs = _seminorm_ip(Iv, Iv, q + 1) + _seminorm_ip(e, e, q + 1)
        assert abs(lhs - rhs) <= 1e-11 * lhs


@pytest.mark.parametrize("d,qs", [(2, (2, 2)), (2, (3, 1)), (3, (1, 2, 1)), (3, (2, 2, 2))])
def test_tensor_interpolation_reproduces(orc, d, qs):
    """Eq. (Hermn2)/(Hermcon2), including mixed degrees m_x != m_y."""
    rng = np.random.default_rng(5)
    C = rng.standard_normal([2 * q + 2 for q in qs])
    corners = []
    for p in polyref.corner_points(d, 1.0):
        S = polyref.shift_scale(C, p, 1.0)
        corners.append(S[tuple(slice(0, q + 1) for q in qs)].reshape(-1))
    a = orc.interp(qs, np.stack(corners))
    np.testing.assert_allclose(a, C, atol=1e-11 * np.abs(C).max())


def test_multi_d_leading_error(orc):
    """Eq. (Imtrunc) in 2-D for f = x^{2m+2} + y^{2m+2}: exact with both terms."""
    m = 2
    n = 2 * m + 2
    C = np.zeros((n + 1, n + 1))
    C[n, 0] = 1.0
    C[0, n] = 1.0
    corners = []
    for p in polyref.corner_points(2, 1.0):
        S = polyref.shift_scale(C, p, 1.0)
        corners.append(S[: m + 1, : m + 1].reshape(-1))
    a = orc.interp((m, m), np.stack(corners))
    diff = np.pad(a, ((0, 1), (0, 1))) - C
    e1 = -npoly.polypow([-0.25, 0.0, 1.0], m + 1)
    want = np.zeros_like(diff)
    want[:, 0] += e1
    want[0, :] += e1
    np.testing.assert_allclose(diff, want, atol=1e-11)
