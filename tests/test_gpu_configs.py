"""Whole runs of the benchmark workloads' step counts.

* 3-D, m = 3, c dt/h = 0.9, the eight seeded Gaussian pulses, 200 full steps:
  the oracle cannot run 128^3 for 200 steps, so the full step count runs on
  8^3 cells, GPU against the oracle element by element (FP64: rel. L2 <= 1e-11;
  split: 1e-9, its drift over 400 half-steps), both the full dissipative and
  the conservative method.
* 2-D, m = 4, 256^2 cells, c dt/h = 1, u0 = sin 2 pi x sin 2 pi y, 512 steps
  to T = 2 with the energy every 8 steps, at full size: against the exact
  solution cos(2 sqrt2 pi t) u0 (FP64 error, split within 1.2x of it or below
  1e-9), the conservative potential energy following cos^2(omega t), the
  dissipative plain energy never above its start.
"""
import math

import numpy as np
import pytest

from paper_1802_05246_b300 import inputs as I
from tests.gpu_util import lib_built, need_gpu, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    need_gpu()
    return lib_built()


@pytest.mark.parametrize("variant", [0, 1])
def test_3d_pulses_200_steps_match_the_oracle(hb, orc, variant):
    d, m, N, steps = 3, 3, 8, 200
    h = 1.0 / N
    cen, wid, amp = I.pulses_3d_config(0)
    u0 = I.gaussian_data(d, m, N, h, 0, 0, cen, wid, amp)
    v0 = np.zeros((N ** 3, m ** 3))
    P = orc.Problem(d, m, N, 1.0, h, 0.9 * h, variant, 0)
    if variant == orc.CONSERVATIVE:
        want, _ = P.run(u0, nsteps=steps, dual_u=P.cons_start(u0, None))
    else:
        wu, wv = P.run(u0, v0, nsteps=steps)
        want = np.concatenate([wu, wv], 1)
    for precision, tol in ((hb.FP64, 1e-11), (hb.SPLIT32, 1e-9)):
        g = hb.Hermite(d, m, N, 1.0, h, 0.9 * h, variant, 0, precision=precision)
        g.set_state(u0, v0)
        g.step(steps)
        u, v = g.get_state()
        got = u if variant == orc.CONSERVATIVE else np.concatenate([u, v], 1)
        assert rel_l2(got, want) <= tol, (precision, rel_l2(got, want))
        assert abs(g.time - steps * 0.9 * h) < 1e-12
        g.close()


def _standing_wave(N, m):
    h = 1.0 / N
    a = 2 * np.pi
    return 0.5 * (I.sine_data(2, m, N, h, 0, 0, [a, -a], phase=np.pi / 2)
                  - I.sine_data(2, m, N, h, 0, 0, [a, a], phase=np.pi / 2))


@pytest.mark.parametrize("variant", [0, 1])
def test_2d_standing_wave_512_steps_with_energy_history(hb, variant):
    d, m, N, steps = 2, 4, 256, 512
    h = 1.0 / N
    u0 = _standing_wave(N, m)
    exact = math.cos(2 * math.sqrt(2) * math.pi * steps * h) * u0
    errs, hist = {}, {}
    for precision in (hb.FP64, hb.SPLIT32):
        g = hb.Hermite(d, m, N, 1.0, h, h, variant, 0, precision=precision)
        g.set_state(u0, np.zeros((N * N, m * m)))
        e = [g.energy()]
        for _ in range(steps // 8):
            g.step(8)
            e.append(g.energy())
        u, _ = g.get_state()
        errs[precision] = rel_l2(u, exact)
        hist[precision] = np.array(e)
        assert abs(g.time - 2.0) < 1e-12
        g.close()
    e64, esp = errs[hb.FP64], errs[hb.SPLIT32]
    assert e64 < 1e-8, e64
    assert esp <= 1.2 * e64 or esp < 1e-9, (esp, e64)
    t = 8 * h * np.arange(steps // 8 + 1)
    for precision, e in hist.items():
        if variant == 1:
            # c^2 int |grad p|^2 of the primal level follows cos^2(omega t) of
            # the exact solution.  (The invariant G weights the highest scaled
            # coefficients by h^-2(m+1)d; on smooth data at this resolution it
            # is made of their rounding noise, so it is checked on random data
            # in the parity tests instead.)
            E = e[:, 0]
            want = E[0] * np.cos(2 * math.sqrt(2) * math.pi * t) ** 2
            assert np.max(np.abs(E - want)) <= 1e-8 * E[0], (precision, np.max(np.abs(E - want)) / E[0])
        else:
            E = e[:, 0]  # plain energy of the dissipative method: never above its start
            assert np.all(E <= E[0] * (1 + 1e-12)), (precision, E[:4])
