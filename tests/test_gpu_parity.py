"""GPU (C-ABI) vs oracle parity: element by element on seeded inputs.

Tolerance: relative L2 <= 1e-11 over all stored scaled coefficients after the
whole run (the FP64 target); operator entries to max(1e-13, eps*cond) of the
largest entry, cond being that of the oracle's Hermite interpolation system.
"""
import math

import numpy as np
import pytest

from paper_1802_05246_b300 import inputs as I
from tests.gpu_util import lib_built, need_gpu, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-11


@pytest.fixture(scope="module")
def hb():
    need_gpu()
    return lib_built()


def _rand_state(rng, n, Nu, Nv):
    return rng.standard_normal((n, Nu)), rng.standard_normal((n, Nv))


def _oracle_tol(m):
    """Forward-error scale of the oracle's LU solve of the (2m+2)^2 confluent
    Vandermonde system of Eq. (Hermcon): eps * cond, at least 1e-13."""
    n = 2 * m + 2
    A = np.zeros((n, n))
    for s, xi in enumerate((-0.5, 0.5)):
        for l in range(m + 1):
            for j in range(l, n):
                A[s * (m + 1) + l, j] = math.comb(j, l) * xi ** (j - l)
    return max(1e-13, 1e-16 * np.linalg.cond(A))


def _make(hb, orc, d, m, N, lam, variant, bc, c=1.0):
    h = 1.0 / N
    dt = lam * h / c
    return hb.Hermite(d, m, N, c, h, dt, variant, bc), orc.Problem(d, m, N, c, h, dt, variant, bc)


# ---------------------------------------------------------------- operator
@pytest.mark.parametrize("d,m,variant", [(1, 1, 0), (1, 3, 0), (1, 6, 0), (1, 3, 1), (1, 0, 1), (2, 2, 0),
                                         (2, 4, 0), (2, 3, 2), (2, 4, 1), (3, 1, 0), (3, 3, 0), (3, 3, 1),
                                         (3, 2, 2)])
def test_operator_matches_oracle_cell(hb, orc, d, m, variant):
    """Every column of the device-built operator (closed-form Taylor series) equals
    the oracle's single-cell half-step (LU interpolation + recursion) on unit data
    at the reference corner."""
    g, P = _make(hb, orc, d, m, 4, 0.83, variant, 0, c=1.7)
    M = g.operator(0)
    nc = 1 << d
    if variant == orc.CONSERVATIVE:
        for b in range(P.Nu):
            cu = np.zeros((nc, P.Nu))
            cu[0, b] = 1.0
            col = P.cons_cell(cu, np.zeros(P.Nu))
            np.testing.assert_allclose(M[:, b], col, rtol=0, atol=_oracle_tol(m) * np.abs(M).max())
        return
    for b in range(P.Nu + P.Nv):
        cu = np.zeros((nc, P.Nu))
        cv = np.zeros((nc, P.Nv))
        if b < P.Nu:
            cu[0, b] = 1.0
        else:
            cv[0, b - P.Nu] = 1.0
        nu, nv = P.diss_cell(cu, cv)
        col = np.concatenate([nu, nv])
        np.testing.assert_allclose(M[:, b], col, rtol=0, atol=_oracle_tol(m) * np.abs(M).max())


@pytest.mark.parametrize("d,m,variant", [(2, 3, 0), (3, 2, 0), (3, 2, 1)])
def test_corner_reflection_symmetry(hb, orc, d, m, variant):
    """The kernel uses M_s[a][b] = sign_s(a) sign_s(b) M_0[a][b]; check it against
    the oracle's response to unit data at every corner s."""
    g, P = _make(hb, orc, d, m, 4, 0.9, variant, 0)
    M = g.operator(0)
    nc = 1 << d

    def par(k, q):
        idx = np.unravel_index(k, [q + 1] * d)
        return [i & 1 for i in idx]

    ins = [par(k, m) for k in range(P.Nu)] + ([par(k, m - 1) for k in range(P.Nv)] if variant != 1 else [])
    outs = ins
    for corner in range(1, nc):
        bits = [(corner >> (d - 1 - i)) & 1 for i in range(d)]
        for b in range(len(ins)):
            cu = np.zeros((nc, P.Nu))
            if variant == orc.CONSERVATIVE:
                cu[corner, b] = 1.0
                col = P.cons_cell(cu, np.zeros(P.Nu))
            else:
                cv = np.zeros((nc, P.Nv))
                if b < P.Nu:
                    cu[corner, b] = 1.0
                else:
                    cv[corner, b - P.Nu] = 1.0
                nu, nv = P.diss_cell(cu, cv)
                col = np.concatenate([nu, nv])
            sb = (-1) ** sum(bi * pi for bi, pi in zip(bits, ins[b]))
            sa = np.array([(-1) ** sum(bi * pi for bi, pi in zip(bits, o)) for o in outs])
            np.testing.assert_allclose(col, sa * sb * M[:, b], rtol=0, atol=1e-13 * np.abs(M).max())


# ------------------------------------------------------------ full runs
def _run_both(hb, orc, d, m, N, lam, variant, bc, nsteps, seed=0, c=1.0):
    g, P = _make(hb, orc, d, m, N, lam, variant, bc, c=c)
    rng = np.random.default_rng(seed)
    n0 = P.nnodes(0)
    u0, v0 = _rand_state(rng, n0, P.Nu, P.Nv)
    if variant == orc.CONSERVATIVE:
        g.set_state(u0, v0)
        q0 = P.cons_start(u0, v0 if m >= 1 else None)
        gq = g.get_grid(1)[0]
        assert rel_l2(gq, q0) <= TOL
        g.step(nsteps)
        gu, _ = g.get_state()
        gq = g.get_grid(1)[0]
        ou, oq = P.run(u0, nsteps=nsteps, dual_u=q0)
        return rel_l2(gu, ou), rel_l2(gq, oq)
    g.set_state(u0, v0)
    g.step(nsteps)
    gu, gv = g.get_state()
    ou, ov = P.run(u0, v0, nsteps=nsteps)
    return rel_l2(np.concatenate([gu.ravel(), gv.ravel()]), np.concatenate([ou.ravel(), ov.ravel()])), 0.0


@pytest.mark.parametrize("variant", [0, 1])
def test_config_1d_standing_wave(hb, orc, variant):
    """1-D periodic [0,1], c=1, m=3, N=64, c dt/h = 0.9 read as 72 steps to T=1
    (lambda_eff = 0.8889), u0 = sin(2 pi x), v0 = 0; GPU = oracle to 1e-11 and
    both close to cos(2 pi t) sin(2 pi x)."""
    N, m, T = 64, 3, 1.0
    h = 1.0 / N
    nsteps = math.ceil(T / (0.9 * h))
    dt = T / nsteps
    g = hb.Hermite(1, m, N, 1.0, h, dt, variant, 0)
    P = orc.Problem(1, m, N, 1.0, h, dt, variant, 0)
    a = 2 * np.pi
    u0 = I.sine_data(1, m, N, h, 0, 0, [a])
    v0 = np.zeros((N, m))
    g.set_state(u0, v0)
    g.step(nsteps)
    gu, _ = g.get_state()
    if variant == orc.CONSERVATIVE:
        ou, _ = P.run(u0, nsteps=nsteps, dual_u=P.cons_start(u0, v0))
    else:
        ou, _ = P.run(u0, v0, nsteps=nsteps)
    assert rel_l2(gu, ou) <= TOL
    exact = np.cos(a * T) * I.sine_data(1, m, N, h, 0, 0, [a])
    assert rel_l2(gu, exact) < 1e-5
    assert abs(g.time - T) < 1e-12


@pytest.mark.parametrize("d,m,N,lam,variant,nsteps", [
    (1, 1, 17, 1.0, 0, 20), (1, 5, 9, 0.7, 0, 15), (1, 4, 11, 0.6, 1, 15), (1, 0, 10, 1.0, 1, 12),
    (2, 4, 12, 1.0, 0, 6), (2, 4, 12, 1.0, 1, 6), (2, 2, 9, 0.9, 2, 6), (2, 6, 5, 0.8, 0, 3),
    (3, 3, 6, 0.9, 0, 2), (3, 3, 6, 0.9, 1, 2), (3, 1, 7, 1.0, 0, 4), (3, 2, 5, 0.7, 2, 2),
])
def test_random_state_periodic(hb, orc, d, m, N, lam, variant, nsteps):
    e1, e2 = _run_both(hb, orc, d, m, N, lam, variant, 0, nsteps, seed=d * 100 + m)
    assert e1 <= TOL and e2 <= TOL, (e1, e2)


@pytest.mark.parametrize("bc", [1, 2])
@pytest.mark.parametrize("d,m,N,variant", [(1, 3, 13, 0), (1, 2, 13, 1), (2, 2, 7, 0), (2, 3, 6, 1),
                                           (3, 1, 5, 0), (3, 2, 4, 1), (2, 2, 6, 2)])
def test_random_state_boundaries(hb, orc, bc, d, m, N, variant):
    e1, e2 = _run_both(hb, orc, d, m, N, 0.85, variant, bc, 3, seed=7 + bc)
    assert e1 <= TOL and e2 <= TOL, (e1, e2)


@pytest.mark.parametrize("N", [1, 2, 3])
@pytest.mark.parametrize("variant", [0, 1])
def test_tiny_periodic_grids(hb, orc, N, variant):
    """Self- and double-neighbour wrap on one- and two-cell periodic grids."""
    e1, e2 = _run_both(hb, orc, 2, 2, N, 1.0, variant, 0, 3, seed=N)
    assert e1 <= TOL and e2 <= TOL


def test_dirichlet_standing_wave_even_coefficients(hb, orc):
    """Dirichlet sin(2 pi x) cos(2 pi t): boundary nodes keep their even
    coefficients at exactly zero (odd ghost extension, Sec. 3.1.3)."""
    N, m = 20, 3
    h = 1.0 / N
    g = hb.Hermite(1, m, N, 1.0, h, 0.9 * h, 0, 1)
    g.set_state(I.sine_data(1, m, N, h, 1, 0, [2 * np.pi]), np.zeros((N + 1, m)))
    g.step(11)
    u, v = g.get_state()
    assert np.all(u[[0, -1]][:, 0::2] == 0.0)
    assert np.all(v[[0, -1]][:, 0::2] == 0.0)


# -------------------------------------------------------------- energies
@pytest.mark.parametrize("d,m,N,variant,bc", [(1, 3, 16, 0, 0), (2, 2, 8, 0, 0), (2, 3, 6, 2, 0),
                                              (3, 1, 5, 0, 0), (1, 2, 9, 0, 1), (2, 2, 5, 0, 2),
                                              (3, 2, 4, 0, 0), (3, 3, 3, 0, 0), (3, 3, 3, 2, 1), (3, 2, 3, 0, 2),
                                              (2, 4, 5, 0, 1), (1, 4, 11, 2, 2), (2, 5, 4, 0, 0),
                                              (2, 6, 3, 2, 1), (1, 8, 7, 0, 0)])
def test_dissipative_energy_parity(hb, orc, d, m, N, variant, bc):
    g, P = _make(hb, orc, d, m, N, 0.9, variant, bc)
    rng = np.random.default_rng(3)
    u, v = _rand_state(rng, P.nnodes(0), P.Nu, P.Nv)
    g.set_state(u, v)
    for k in range(3):
        e = g.energy()
        grid = k % 2
        gu, gv = g.get_grid(grid)
        oe = P.diss_energy(grid, gu, gv)
        np.testing.assert_allclose(e[:2], oe, rtol=max(1e-12, 10 * _oracle_tol(m)))
        g.advance_half(1)


def test_dissipative_energy_parity_many_tiles(hb, orc):
    """A grid with more 32-cell tiles than the energy kernel's persistent
    blocks (2-D, m = 2, 200^2 cells, Dirichlet): every block loops over several
    tiles.  FP64 and split energies of both grids against the oracle."""
    d, m, N = 2, 2, 200
    rng = np.random.default_rng(11)
    for precision, rtol in ((hb.FP64, 1e-12), (hb.SPLIT32, 1e-10)):
        h = 1.0 / N
        g = hb.Hermite(d, m, N, 1.0, h, 0.9 * h, 0, 1, precision=precision)
        P = orc.Problem(d, m, N, 1.0, h, 0.9 * h, 0, 1)
        u, v = _rand_state(rng, P.nnodes(0), P.Nu, P.Nv)
        g.set_state(u, v)
        for grid in (0, 1):
            e = g.energy()
            gu, gv = g.get_grid(grid)
            oe = P.diss_energy(grid, gu, gv)
            np.testing.assert_allclose(e[:2], oe, rtol=rtol)
            g.advance_half(1)
        g.close()


@pytest.mark.parametrize("d,m,N,bc", [(1, 2, 12, 0), (2, 2, 6, 0), (3, 1, 5, 0), (1, 3, 9, 1), (2, 1, 5, 2),
                                      (2, 4, 5, 0), (2, 6, 4, 1), (3, 3, 3, 0), (3, 2, 4, 2), (1, 8, 9, 0),
                                      (1, 0, 7, 0)])
def test_conservative_energy_parity_and_conservation(hb, orc, d, m, N, bc):
    g, P = _make(hb, orc, d, m, N, 0.95, 1, bc)
    rng = np.random.default_rng(4)
    p = rng.uniform(0, 1, (P.nnodes(0), P.Nu))
    q = rng.uniform(0, 1, (P.nnodes(1), P.Nu))
    g.set_state2(p, q)
    G0 = None
    for k in range(4):
        e = g.energy()
        gp, _ = g.get_grid(0)
        gq, _ = g.get_grid(1)
        if k % 2 == 0:
            oG = P.cons_G(gp, gq)
        else:  # newest level is the primal one: roles of the grids swap
            p_next = P.half_step(1, gp, dst_u=gq)
            oG = P.cons_forms(0, gp, gp)[0] - P.cons_forms(1, p_next, gq)[0]
        tol = 10 * _oracle_tol(m)
        np.testing.assert_allclose(e[1], oG, rtol=max(1e-11, tol))
        np.testing.assert_allclose(e[0], P.cons_forms(0, gp, gp)[1], rtol=max(1e-12, tol))
        if bc == 0:
            G0 = e[1] if G0 is None else G0
            assert abs(e[1] - G0) <= max(1e-11, tol) * abs(G0)
        g.advance_half(1)


# -------------------------------------------------- full-size sampled parity
@pytest.mark.parametrize("variant", [0, 1])
def test_full_size_3d_sampled(hb, orc, variant):
    """3-D periodic m=3, 128^3, c dt/h = 0.9, eight seeded Gaussian pulses: two
    half-steps in the benchmark's launch configuration; 600 sampled targets of
    each half-step recomputed by the oracle from the GPU's input level."""
    d, m, N = 3, 3, 128
    h = 1.0 / N
    g = hb.Hermite(d, m, N, 1.0, h, 0.9 * h, variant, 0)
    P = orc.Problem(d, m, N, 1.0, h, 0.9 * h, variant, 0)
    cen, wid, amp = I.pulses_3d_config(0)
    u0 = I.gaussian_data(d, m, N, h, 0, 0, cen, wid, amp)
    v0 = np.zeros((N ** 3, m ** 3))
    g.set_state(u0, v0)
    rng = np.random.default_rng(11)
    t = np.concatenate([rng.integers(0, N ** 3, 600), [0, N ** 3 - 1, N - 1, N * N - 1]])
    if variant == orc.CONSERVATIVE:
        q0, _ = g.get_grid(1)
        g.advance_half(1)  # primal update from the dual level
        p1, _ = g.get_grid(0)
        want = P.half_step_sample(0, q0, None, t, old_u=u0[t])
        assert rel_l2(p1[t], want) <= TOL
        g.advance_half(1)
        q1, _ = g.get_grid(1)
        want = P.half_step_sample(1, p1, None, t, old_u=q0[t])
        assert rel_l2(q1[t], want) <= TOL
        return
    g.advance_half(1)
    du, dv = g.get_grid(1)
    wu, wv = P.half_step_sample(1, u0, v0, t)
    assert rel_l2(np.concatenate([du[t], dv[t]], 1), np.concatenate([wu, wv], 1)) <= TOL
    g.advance_half(1)
    pu, pv = g.get_grid(0)
    wu, wv = P.half_step_sample(0, du, dv, t)
    assert rel_l2(np.concatenate([pu[t], pv[t]], 1), np.concatenate([wu, wv], 1)) <= TOL


def _boundary_targets(rng, n, count):
    """Random node indices of an n^3 grid plus every corner and some face and
    edge nodes (where the ghost polynomials enter)."""
    idx = [rng.integers(0, n ** 3, count)]
    ends = [0, n - 1]
    idx.append(np.array([(i * n + j) * n + k for i in ends for j in ends for k in ends]))
    f = rng.integers(0, n, (3, 40))
    for ax in range(3):
        c = f.copy()
        c[ax] = rng.choice(ends, 40)
        idx.append((c[0] * n + c[1]) * n + c[2])
    return np.concatenate(idx)


_BC_DATA = {}


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("bc", [1, 2])
@pytest.mark.parametrize("variant", [0, 1, 2])
def test_full_size_3d_boundaries_sampled(hb, orc, variant, bc, precision):
    """3-D m=3, 96^3 cells (97^3 primal nodes) with Dirichlet or Neumann
    boundaries, every variant, FP64 (0), split on the CUDA cores (1) and split
    on the tensor cores (2): two half-steps from seeded odd or even
    Gaussian-pulse data, sampled targets (all corners, faces, edges)
    recomputed by the oracle from the GPU's input level."""
    d, m, N = 3, 3, 96
    h = 1.0 / N
    g = hb.Hermite(d, m, N, 1.0, h, 0.9 * h, variant, bc, precision=min(precision, 1))
    if precision > 0:
        g.set_split_engine(precision - 1)
    P = orc.Problem(d, m, N, 1.0, h, 0.9 * h, variant, bc)
    if (N, bc) not in _BC_DATA:
        cen, wid, amp = I.pulses_3d_config(1)
        _BC_DATA[(N, bc)] = I.gaussian_data(d, m, N, h, bc, 0, cen, wid, amp)
    u0 = _BC_DATA[(N, bc)]
    n0 = g.nodes(0)
    v0 = np.zeros((n0, m ** 3))
    g.set_state(u0, v0)
    rng = np.random.default_rng(21 + bc)
    tol = TOL if precision == 0 else 1e-9
    assert n0 == (N + 1) ** 3 and g.nodes(1) == N ** 3  # primal N+1, dual N nodes per axis
    t1 = _boundary_targets(rng, N, 300)
    t0 = _boundary_targets(rng, N + 1, 300)
    if variant == orc.CONSERVATIVE:
        q0, _ = g.get_grid(1)
        g.advance_half(1)
        p1, _ = g.get_grid(0)
        assert rel_l2(p1[t0], P.half_step_sample(0, q0, None, t0, old_u=u0[t0])) <= tol
        g.advance_half(1)
        q1, _ = g.get_grid(1)
        assert rel_l2(q1[t1], P.half_step_sample(1, p1, None, t1, old_u=q0[t1])) <= tol
        return
    g.advance_half(1)
    du, dv = g.get_grid(1)
    wu, wv = P.half_step_sample(1, u0, v0, t1)
    assert rel_l2(np.concatenate([du[t1], dv[t1]], 1), np.concatenate([wu, wv], 1)) <= tol
    g.advance_half(1)
    pu, pv = g.get_grid(0)
    wu, wv = P.half_step_sample(0, du, dv, t0)
    assert rel_l2(np.concatenate([pu[t0], pv[t0]], 1), np.concatenate([wu, wv], 1)) <= tol


@pytest.mark.parametrize("variant", [0, 1])
def test_full_size_2d_sampled(hb, orc, variant):
    """2-D periodic m=4, 256^2, lambda = 1, u0 = sin 2pi x sin 2pi y: 8 steps on
    the GPU, then one more half-step sampled against the oracle."""
    d, m, N = 2, 4, 256
    h = 1.0 / N
    g = hb.Hermite(d, m, N, 1.0, h, h, variant, 0)
    P = orc.Problem(d, m, N, 1.0, h, h, variant, 0)
    a = 2 * np.pi
    u0 = 0.5 * (I.sine_data(2, m, N, h, 0, 0, [a, -a], phase=np.pi / 2)
                - I.sine_data(2, m, N, h, 0, 0, [a, a], phase=np.pi / 2))
    g.set_state(u0, np.zeros((N * N, m * m)))
    g.step(8)
    rng = np.random.default_rng(5)
    t = rng.integers(0, N * N, 800)
    if variant == orc.CONSERVATIVE:
        pu, _ = g.get_grid(0)
        qu, _ = g.get_grid(1)
        g.advance_half(1)
        nu, _ = g.get_grid(0)
        assert rel_l2(nu[t], P.half_step_sample(0, qu, None, t, old_u=pu[t])) <= TOL
    else:
        pu, pv = g.get_grid(0)
        g.advance_half(1)
        du, dv = g.get_grid(1)
        wu, wv = P.half_step_sample(1, pu, pv, t)
        assert rel_l2(np.concatenate([du[t], dv[t]], 1), np.concatenate([wu, wv], 1)) <= TOL
    # and the solution itself is right: cos(2 sqrt2 pi t) u0 after 8 steps
    g2 = hb.Hermite(d, m, N, 1.0, h, h, variant, 0)
    g2.set_state(u0, np.zeros((N * N, m * m)))
    g2.step(8)
    u, _ = g2.get_state()
    assert rel_l2(u, np.cos(2 * math.sqrt(2) * np.pi * 8 * h) * u0) < 1e-8


# ------------------------------------------------ checkpoint / edge cases
def test_checkpoint_resume_bit_identical(hb, orc):
    g, P = _make(hb, orc, 2, 3, 10, 0.9, 0, 0)
    rng = np.random.default_rng(9)
    u, v = _rand_state(rng, P.nnodes(0), P.Nu, P.Nv)
    g.set_state(u, v)
    g.step(6)
    a_u, a_v = g.get_state()
    g2, _ = _make(hb, orc, 2, 3, 10, 0.9, 0, 0)
    g2.set_state(u, v)
    g2.step(3)
    cu, cv = g2.get_state()
    g3, _ = _make(hb, orc, 2, 3, 10, 0.9, 0, 0)
    g3.set_state(cu, cv)
    g3.step(3)
    b_u, b_v = g3.get_state()
    assert np.array_equal(a_u, b_u) and np.array_equal(a_v, b_v)


def test_conservative_checkpoint_resume(hb, orc):
    g, P = _make(hb, orc, 1, 3, 16, 0.9, 1, 0)
    rng = np.random.default_rng(10)
    u = rng.standard_normal((16, 4))
    g.set_state(u, None)
    g.step(8)
    a, _ = g.get_grid(0)
    g2, _ = _make(hb, orc, 1, 3, 16, 0.9, 1, 0)
    g2.set_state(u, None)
    g2.step(4)
    p, _ = g2.get_grid(0)
    q, _ = g2.get_grid(1)
    g3, _ = _make(hb, orc, 1, 3, 16, 0.9, 1, 0)
    g3.set_state2(p, q)
    g3.step(4)
    b, _ = g3.get_grid(0)
    assert np.array_equal(a, b)


def test_deterministic(hb, orc):
    out = []
    for _ in range(2):
        g, P = _make(hb, orc, 3, 2, 6, 0.9, 0, 0)
        rng = np.random.default_rng(1)
        g.set_state(*_rand_state(rng, P.nnodes(0), P.Nu, P.Nv))
        g.step(2)
        out.append((g.get_state(), g.energy()))
    assert np.array_equal(out[0][0][0], out[1][0][0]) and np.array_equal(out[0][1], out[1][1])


def test_device_pointer_state_matches_host(hb, orc):
    import torch

    g, P = _make(hb, orc, 2, 2, 8, 0.9, 0, 0)
    rng = np.random.default_rng(2)
    u, v = _rand_state(rng, P.nnodes(0), P.Nu, P.Nv)
    g.set_state(u, v)
    g.step(2)
    a = g.get_state()
    g2, _ = _make(hb, orc, 2, 2, 8, 0.9, 0, 0)
    s = torch.cuda.Stream()
    g2.set_stream(s)
    tu, tv = torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()
    torch.cuda.synchronize()
    g2.set_state_device(tu, tv)
    g2.step(2)
    ou = torch.empty_like(tu)
    ov = torch.empty_like(tv)
    g2.get_grid_device(0, ou, ov)
    assert np.array_equal(ou.cpu().numpy(), a[0]) and np.array_equal(ov.cpu().numpy(), a[1])


def test_error_statuses(hb, orc):
    g, P = _make(hb, orc, 1, 2, 8, 0.9, 0, 0)
    g.set_state(np.zeros((8, 3)), np.zeros((8, 2)))
    g.advance_half(1)
    with pytest.raises(hb.HermiteError) as e:
        g.get_state()
    assert e.value.code == -6
    with pytest.raises(hb.HermiteError) as e:
        g.set_state2(np.zeros((8, 3)), np.zeros((8, 3)))
    assert e.value.code == -6
    u = np.zeros((8, 3))
    u[3, 1] = np.nan
    g.set_state(u, np.zeros((8, 2)))
    with pytest.raises(hb.HermiteError) as e:
        g.energy()
    assert e.value.code == -4
    with pytest.raises(hb.HermiteError) as e:
        g.step(-1)
    assert e.value.code == -1


def test_time_of_the_primal_level(hb, orc):
    """hermite_time: dissipative half * dt/2; conservative ((half + 1) / 2) * dt
    (the first half-step moves the primal level from 0 to dt)."""
    N, dt = 8, 0.1
    for variant, want in ((0, [0, 0.05, 0.1, 0.15, 0.2]), (1, [0, 0.1, 0.1, 0.2, 0.2])):
        g = hb.Hermite(1, 2, N, 1.0, 1.0 / N * 2, dt, variant, 0)
        g.set_state(np.zeros((N, 3)), np.zeros((N, 2)) if variant == 0 else None)
        got = []
        for k in range(5):
            got.append(g.time)
            g.advance_half(1)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)
        g.close()
