"""Long runs on the GPU (Sec. 5.2, experiment E2): the conservative method's
energy over the paper's 10^6 steps, and the 1-D dissipative energy of
Eq. (stable1), which never grows.

Setup of Sec. 5.2: 1-D periodic on [0, 2 pi), h = 2 pi / 30, dt = h / 2,
m = 1, 3, 5, for the exact solution sin x cos t and for random U(0, 1)
coefficients on both levels.  The paper reports that the change of the
energy grows with t under round-off, faster for random than for smooth data,
without printing values; the bounds below read "conserved to round-off" as:

* smooth data, m = 1, 3: |G^n - G^0| <= 1e-11 |G^0| at every checkpoint;
* smooth data, m = 5: the linear bound of the oracle's long runs,
  |G^n - G^0| <= n 8 eps cond(m) |p|^2_{m+1} (the top scaled coefficients
  carry the seminorm and their rounding accumulates step after step; the
  seminorm of the initial level is the oracle's);
* random data: |G^n - G^0| <= 1e-6 |G^0| (FP64) and 1e-5 |G^0| (split) after
  10^6 steps -- round-off growth, many orders below the change any
  non-conservative operator would show (the dissipative method loses a
  visible share of its energy within a few steps on such data).
"""
import numpy as np
import pytest

from paper_1802_05246_b300 import inputs as I
from tests.gpu_util import hermite_cond, lib_built, need_gpu

pytestmark = pytest.mark.gpu

N_CELLS = 30
H = 2 * np.pi / N_CELLS
DT = H / 2


@pytest.fixture(scope="module")
def hb():
    need_gpu()
    return lib_built()


def _drift(hb, m, precision, p, q, nsteps=10**6, every=10**5):
    """Relative change (G^n - G^0) / G^0 of the conservative invariant at
    every checkpoint, and G^0."""
    g = hb.Hermite(1, m, N_CELLS, 1.0, H, DT, hb.CONSERVATIVE, hb.PERIODIC, precision=precision)
    g.set_state2(p, q)
    G0 = g.energy()[1]
    assert np.isfinite(G0) and G0 != 0.0
    rel, n = [], 0
    while n < nsteps:
        g.step(every)
        n += every
        rel.append((g.energy()[1] - G0) / G0)
    assert g.half_steps == 2 * nsteps
    g.close()
    return np.array(rel), G0


@pytest.mark.parametrize("m", [1, 3, 5])
def test_conservative_energy_smooth_data_10_6_steps(hb, orc, m):
    p = I.sine_data(1, m, N_CELLS, H, 0, 0, [1.0])
    q = np.cos(DT / 2) * I.sine_data(1, m, N_CELLS, H, 0, 1, [1.0])
    every = 10**5
    rel, G0 = _drift(hb, m, hb.FP64, p, q, every=every)
    n = every * np.arange(1, len(rel) + 1)
    if m < 5:
        assert np.all(np.abs(rel) <= 1e-11), rel
    else:
        P = orc.Problem(1, m, N_CELLS, 1.0, H, DT, orc.CONSERVATIVE, orc.PERIODIC)
        seminorm = P.cons_forms(0, p, p)[0]
        bound = n * 8 * np.finfo(float).eps * hermite_cond(m) * seminorm
        assert np.all(np.abs(rel * G0) <= bound), (rel, seminorm)


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-6), ("split", 1e-5)])
@pytest.mark.parametrize("m", [1, 3, 5])
def test_conservative_energy_random_data_10_6_steps(hb, m, precision, bound):
    rng = np.random.default_rng(100 + m)
    p, q = rng.uniform(0, 1, (N_CELLS, m + 1)), rng.uniform(0, 1, (N_CELLS, m + 1))
    rel, _ = _drift(hb, m, hb.FP64 if precision == "fp64" else hb.SPLIT32, p, q)
    assert np.all(np.abs(rel) <= bound), rel


@pytest.mark.parametrize("m", [1, 3, 5])
def test_dissipative_energy_never_grows_over_long_runs(hb, m):
    """Eq. (stable1)/(Energyeq): in 1-D the dissipative method's energy
    c^2|d_x I_m u|_m^2 + |I_{m-1} v|_m^2 does not grow.  10^5 steps of random
    data, c dt/h = 0.9, checked every 10^3 steps: no checkpoint exceeds the one
    before by more than round-off (1e-13 of it, plus 1e-14 of the initial
    energy once everything but the smoothest modes has decayed)."""
    g = hb.Hermite(1, m, N_CELLS, 1.0, H, 0.9 * H, hb.DISSIPATIVE, hb.PERIODIC)
    rng = np.random.default_rng(7 + m)
    g.set_state(rng.uniform(0, 1, (N_CELLS, m + 1)), rng.uniform(0, 1, (N_CELLS, m)))
    first = prev = g.energy()[1]
    for _ in range(100):
        g.step(1000)
        e = g.energy()[1]
        assert np.isfinite(e)
        assert e <= prev * (1 + 1e-13) + 1e-14 * first, (m, e, prev)
        prev = e
    assert prev < first
    g.close()
