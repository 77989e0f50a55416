"""The tensor-core split-precision half-step (hermite_set_split_engine 1)
against the oracle and against the CUDA-core split kernel, on random states
(rough data exercise every digit), with ragged last tiles (node counts not a
multiple of 128), all variants and boundary conditions it covers, and on the
3-D pulse workload's data against the exact solution."""
import numpy as np
import pytest

from tests.gpu_util import lib_built, need_gpu, rel_l2

pytestmark = pytest.mark.gpu
TOL_SPLIT = 1e-10  # relative L2 after the run, as for the CUDA-core split kernel

CASES = [
    # d, m, N, c dt/h, variant, bc, full steps
    (3, 3, 5, 0.9, 0, 0, 2), (3, 3, 5, 0.9, 1, 0, 2), (3, 3, 4, 0.9, 2, 0, 2), (3, 3, 4, 1.0, 0, 1, 2),
    (3, 3, 3, 0.9, 1, 2, 2), (3, 2, 6, 0.9, 0, 2, 3), (3, 2, 4, 0.9, 1, 1, 2), (3, 1, 7, 0.9, 0, 0, 3),
    (2, 4, 10, 1.0, 0, 0, 4), (2, 4, 9, 0.9, 1, 1, 4), (2, 3, 13, 0.9, 2, 2, 4),
    (2, 2, 11, 0.8, 1, 0, 4), (2, 1, 6, 0.9, 0, 2, 3),
]


@pytest.fixture(scope="module")
def hb():
    need_gpu()
    return lib_built()


def _state(P, seed):
    rng = np.random.default_rng(seed)
    n0 = P.nnodes(0)
    return rng.standard_normal((n0, P.Nu)), rng.standard_normal((n0, P.Nv))


@pytest.mark.parametrize("d,m,N,lam,variant,bc,nsteps", CASES)
def test_tc_engine_matches_oracle(hb, orc, d, m, N, lam, variant, bc, nsteps):
    h = 1.0 / N
    g = hb.Hermite(d, m, N, 1.0, h, lam * h, variant, bc, precision=hb.SPLIT32)
    g.set_split_engine(1)
    P = orc.Problem(d, m, N, 1.0, h, lam * h, variant, bc)
    u0, v0 = _state(P, 10 * d + m)
    g.set_state(u0, v0)
    g.step(nsteps)
    gu, gv = g.get_state()
    if variant == orc.CONSERVATIVE:
        ou, oq = P.run(u0, nsteps=nsteps, dual_u=P.cons_start(u0, v0))
        assert rel_l2(gu, ou) <= TOL_SPLIT
        assert rel_l2(g.get_grid(1)[0], oq) <= TOL_SPLIT
    else:
        ou, ov = P.run(u0, v0, nsteps=nsteps)
        assert rel_l2(np.concatenate([gu, gv], 1), np.concatenate([ou, ov], 1)) <= TOL_SPLIT
    g.close()


@pytest.mark.parametrize("d,m,N,lam,variant,bc,nsteps", CASES[:8])
def test_tc_engine_matches_cuda_core_split(hb, orc, d, m, N, lam, variant, bc, nsteps):
    h = 1.0 / N
    P = orc.Problem(d, m, N, 1.0, h, lam * h, variant, bc)
    u0, v0 = _state(P, 3)
    out = []
    for engine in (0, 1):
        g = hb.Hermite(d, m, N, 1.0, h, lam * h, variant, bc, precision=hb.SPLIT32)
        g.set_split_engine(engine)
        assert g.split_engine == engine
        g.set_state(u0, v0)
        g.step(nsteps)
        out.append(np.concatenate([x for x in (g.get_grid(0)[0], g.get_grid(1)[0]) if x is not None], 0))
        g.close()
    # both carry ~48 bits: per element (CUDA cores) or per node, class and
    # operator row (tensor-core digits), so rough data differ at the oracle tolerance
    assert rel_l2(out[1], out[0]) <= TOL_SPLIT


def test_tc_engine_availability(hb):
    g = hb.Hermite(1, 3, 16, 1.0, 1 / 16, 0.9 / 16, 0, 0, precision=hb.SPLIT32)
    assert g.split_engine == 0
    with pytest.raises(hb.HermiteError) as e:
        g.set_split_engine(1)
    assert e.value.code == -7
    g.close()
    g = hb.Hermite(2, 6, 4, 1.0, 0.25, 0.2, 0, 0, precision=hb.SPLIT32)  # classes of 25 coefficients
    assert g.split_engine == 0
    g.close()
    g = hb.Hermite(3, 3, 4, 1.0, 0.25, 0.2, 0, 0)
    assert g.split_engine == -1
    with pytest.raises(hb.HermiteError) as e:
        g.set_split_engine(0)
    assert e.value.code == -6
    g.close()


def test_tc_engine_accuracy_bar_3d_pulses(hb):
    """The 3-D pulse workload (m = 3, c dt/h = 0.9, eight seeded pulses) over
    200 steps at 32^3: the tensor-core engine's error against the exact
    solution is within 1.2x of the FP64 error, and the two arithmetics agree
    far below the discretisation error."""
    from tests.test_gpu_accuracy import pulse_errors

    e64 = pulse_errors(hb, 32, hb.FP64)
    etc = pulse_errors(hb, 32, hb.SPLIT32, engine=1)
    assert e64 >= 1e-9 and etc <= 1.2 * e64
    assert abs(etc - e64) <= 1e-3 * e64


@pytest.mark.parametrize("variant", [0, 1])
def test_tc_engine_full_size_3d_sampled(hb, orc, variant):
    """The 3-D workload at its full size (m = 3, 128^3, c dt/h = 0.9, eight
    seeded pulses) on the tensor-core engine, launched as the benchmark's
    split_tc arm launches it: two half-steps, 600 sampled targets of each
    recomputed by the oracle from the GPU's input level."""
    d, m, N = 3, 3, 128
    h = 1.0 / N
    g = hb.Hermite(d, m, N, 1.0, h, 0.9 * h, variant, 0, precision=hb.SPLIT32)
    g.set_split_engine(1)
    P = orc.Problem(d, m, N, 1.0, h, 0.9 * h, variant, 0)
    from paper_1802_05246_b300 import inputs as I

    cen, wid, amp = I.pulses_3d_config(0)
    u0 = I.gaussian_data(d, m, N, h, 0, 0, cen, wid, amp)
    v0 = np.zeros((N ** 3, m ** 3))
    g.set_state(u0, v0)
    rng = np.random.default_rng(12)
    t = np.concatenate([rng.integers(0, N ** 3, 600), [0, N ** 3 - 1, N - 1, N * N - 1]])
    if variant == orc.CONSERVATIVE:
        q0, _ = g.get_grid(1)
        g.advance_half(1)
        p1, _ = g.get_grid(0)
        assert rel_l2(p1[t], P.half_step_sample(0, q0, None, t, old_u=u0[t])) <= TOL_SPLIT
        g.advance_half(1)
        q1, _ = g.get_grid(1)
        assert rel_l2(q1[t], P.half_step_sample(1, p1, None, t, old_u=q0[t])) <= TOL_SPLIT
    else:
        g.advance_half(1)
        du, dv = g.get_grid(1)
        wu, wv = P.half_step_sample(1, u0, v0, t)
        assert rel_l2(np.concatenate([du[t], dv[t]], 1), np.concatenate([wu, wv], 1)) <= TOL_SPLIT
        g.advance_half(1)
        pu, pv = g.get_grid(0)
        wu, wv = P.half_step_sample(0, du, dv, t)
        assert rel_l2(np.concatenate([pu[t], pv[t]], 1), np.concatenate([wu, wv], 1)) <= TOL_SPLIT
    g.close()


@pytest.mark.parametrize("d,m,N,c,variant,bc", [(3, 3, 5, 2.3, 0, 0), (2, 4, 7, 0.37, 0, 1), (3, 2, 5, 5.0, 1, 2)])
def test_tc_engine_wave_speed(hb, orc, d, m, N, c, variant, bc):
    """Wave speeds c != 1 change the velocity scaling h/c that balances the
    u and v digits (2^vexp): parity with the oracle as for c = 1."""
    h = 1.0 / N
    dt = 0.9 * h / c
    g = hb.Hermite(d, m, N, c, h, dt, variant, bc, precision=hb.SPLIT32)
    g.set_split_engine(1)
    P = orc.Problem(d, m, N, c, h, dt, variant, bc)
    u0, v0 = _state(P, 99)
    v0 = v0 * c / h  # velocity data of the size a wave of speed c carries
    g.set_state(u0, v0)
    g.step(2)
    gu, gv = g.get_state()
    if variant == orc.CONSERVATIVE:
        ou, _ = P.run(u0, nsteps=2, dual_u=P.cons_start(u0, v0))
        assert rel_l2(gu, ou) <= TOL_SPLIT
    else:
        ou, ov = P.run(u0, v0, nsteps=2)
        assert rel_l2(np.concatenate([gu, gv * h / c], 1), np.concatenate([ou, ov * h / c], 1)) <= TOL_SPLIT
    g.close()
