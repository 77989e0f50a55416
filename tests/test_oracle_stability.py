"""Fourier-symbol stability of the oracle's full step (periodic grids).

The one-step map is translation invariant, so its spectrum is the union over
wavenumbers theta of the eigenvalues of the symbol G(theta), built here from
the oracle's responses to unit data at one node.  Stability at c dt = h for
every m is claimed for both methods (Sec. 1, 3.3, 6); it is proved in 1-D.
The constant and linear-in-time modes make theta = 0 defective, so eigenvalue
moduli are compared with a sqrt(eps)-level tolerance there.
"""
import itertools

import numpy as np
import pytest


def _symbol(orc, d, m, lam, variant, N=5):
    h = 1.0 / N
    P = orc.Problem(d, m, N, 1.0, h, lam * h, variant, orc.PERIODIC)
    n = N ** d
    cons = variant == orc.CONSERVATIVE
    nc = 2 * P.Nu if cons else P.Nu + P.Nv
    R = np.zeros((nc, n, nc))
    for j in range(nc):
        if cons:
            p = np.zeros((n, P.Nu))
            q = np.zeros((n, P.Nu))
            (p if j < P.Nu else q)[0, j % P.Nu] = 1.0
            a, b = P.run(p, nsteps=1, dual_u=q)
        else:
            u = np.zeros((n, P.Nu))
            v = np.zeros((n, P.Nv))
            if j < P.Nu:
                u[0, j] = 1.0
            else:
                v[0, j - P.Nu] = 1.0
            a, b = P.run(u, v, nsteps=1)
        R[j] = np.concatenate([a, b], 1)
    idx = np.array(np.unravel_index(np.arange(n), [N] * d)).T
    off = np.where(idx > N // 2, idx - N, idx)

    def G(theta):
        return np.einsum("jnk,n->kj", R, np.exp(1j * off @ np.asarray(theta)))

    return G


def _moduli(G, d, nth, skip_zero=True):
    th = np.linspace(-np.pi, np.pi, nth)
    out = []
    for t in itertools.product(th, repeat=d):
        if skip_zero and max(abs(x) for x in t) < 1e-12:
            continue
        out.append(np.abs(np.linalg.eigvals(G(list(t)))))
    return np.concatenate(out)


@pytest.mark.parametrize("m", range(1, 7))
@pytest.mark.parametrize("lam", [0.5, 1.0])
def test_1d_dissipative_stable_every_m(orc, m, lam):
    mod = _moduli(_symbol(orc, 1, m, lam, orc.DISSIPATIVE), 1, 181)
    assert mod.max() <= 1 + 1e-9


@pytest.mark.parametrize("m", range(0, 6))
@pytest.mark.parametrize("lam", [0.6, 1.0])
def test_1d_conservative_on_unit_circle(orc, m, lam):
    mod = _moduli(_symbol(orc, 1, m, lam, orc.CONSERVATIVE), 1, 91)
    assert np.abs(mod - 1).max() <= 1e-6


@pytest.mark.parametrize("m,lam", [(1, 1.0), (2, 1.0), (3, 1.0), (4, 0.9)])
def test_2d_full_dissipative_stable(orc, m, lam):
    """Sec. 3.3 full variant: no growing mode at CFL 1 for m <= 3 (and m = 4 at 0.9)."""
    mod = _moduli(_symbol(orc, 2, m, lam, orc.DISSIPATIVE), 2, 37)
    assert mod.max() <= 1 + 1e-9


@pytest.mark.parametrize("m", [1, 2])
def test_2d_conservative_on_unit_circle(orc, m):
    mod = _moduli(_symbol(orc, 2, m, 1.0, orc.CONSERVATIVE), 2, 25)
    assert np.abs(mod - 1).max() <= 1e-6


def test_2d_full_dissipative_weak_growth_m5_finding(orc):
    """Recorded finding: with the first step exactly as printed in Sec. 3.3, the
    2-D full variant has a weakly growing high-frequency mode for m = 5 at
    c dt = h (about 1.6e-2 per step), below what the paper's smooth-data runs
    could reveal.  The paper gives no proof for d > 1."""
    mod = _moduli(_symbol(orc, 2, 5, 1.0, orc.DISSIPATIVE), 2, 41)
    assert 1e-3 < mod.max() - 1 < 1e-1
