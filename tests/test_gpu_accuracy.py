"""Errors against exact solutions, measured on the GPU.

* hermite_l2_error (the FP64 device reduction of the Sec. 5.1 error measure)
  against the oracle's quadrature of the same interpolant, all boundaries;
* the split-precision accuracy bar on the 3-D pulse workload itself (m = 3,
  c dt/h = 0.9, the eight seeded pulses, 200 steps): the split error against
  the exact solution is within 1.2x of the FP64 error wherever that error is
  at least 1e-9.
"""
import numpy as np
import pytest

from paper_1802_05246_b300 import inputs as I
from tests.gpu_util import lib_built, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    need_gpu()
    return lib_built()


def gauss(nq):
    x, w = np.polynomial.legendre.leggauss(nq)
    return 0.5 * x, 0.5 * w


def cell_points(d, N, h, bc, grid, xq, cells=None):
    """Quadrature points [cells, nq^d, d] of the cells of a level on `grid`
    (cells centred at the nodes of grid 1 - grid)."""
    ax = I.axis_coords(N, h, bc, 1 - grid)
    C = np.stack(np.meshgrid(*([ax] * d), indexing="ij"), -1).reshape(-1, d)
    if cells is not None:
        C = C[cells]
    Q = np.stack(np.meshgrid(*([xq * h] * d), indexing="ij"), -1).reshape(-1, d)
    return C[:, None, :] + Q[None, :, :]


def smooth(p):
    d = p.shape[-1]
    out = np.sin(2 * np.pi * p[..., 0] + 0.3)
    for i in range(1, d):
        out = out * np.cos(2 * np.pi * (i + 1) * p[..., i] - 0.2 * i)
    return out


@pytest.mark.parametrize("d,m,N,variant,bc,prec", [(1, 3, 16, 0, 0, 0), (2, 2, 8, 0, 1, 0), (3, 2, 6, 0, 2, 0),
                                                   (3, 3, 5, 0, 0, 0), (2, 4, 6, 1, 0, 0), (3, 3, 5, 0, 1, 1),
                                                   (1, 6, 9, 2, 2, 1)])
def test_l2_error_matches_oracle(hb, orc, d, m, N, variant, bc, prec):
    import torch

    h = 1.0 / N
    g = hb.Hermite(d, m, N, 1.0, h, 0.9 * h, variant, bc, precision=prec)
    P = orc.Problem(d, m, N, 1.0, h, 0.9 * h, variant, bc)
    rng = np.random.default_rng(d + 7 * m)
    n0 = P.nnodes(0)
    u = rng.standard_normal((n0, P.Nu)) * 0.1
    v = rng.standard_normal((n0, P.Nv)) if variant != 1 else None
    g.set_state(u, v)
    gu = g.get_grid(0)[0]
    nq = 2 * m + 2
    xq, wq = gauss(nq)
    pts = cell_points(d, N, h, bc, 0, xq)
    ex = smooth(pts)
    e2, n2 = g.l2_error(0, xq, wq, torch.from_numpy(ex).cuda())
    ref = orc_err = P.l2_error(0, gu, nq, smooth)
    np.testing.assert_allclose(np.sqrt(e2), ref, rtol=1e-11)
    # out[1] is the same quadrature of the exact values alone
    w = np.prod(np.stack(np.meshgrid(*([wq] * d), indexing="ij"), -1).reshape(-1, d), 1)
    # (the cells of a primal level are centred at dual nodes: none is cut by a boundary)
    want = h**d * np.sum(w[None, :] * ex * ex)
    np.testing.assert_allclose(n2, want, rtol=1e-12)
    # a cell list: the sums over two disjoint halves add up to the whole
    ncell = pts.shape[0]
    perm = rng.permutation(ncell)
    parts = []
    for half in (perm[: ncell // 2], perm[ncell // 2:]):
        sel = np.sort(half)
        cells = torch.from_numpy(sel.astype(np.int64)).cuda()
        parts.append(g.l2_error(0, xq, wq, torch.from_numpy(np.ascontiguousarray(ex[sel])).cuda(), cells))
    np.testing.assert_allclose(parts[0][0] + parts[1][0], e2, rtol=1e-12)
    assert orc_err > 0
    if variant != 1:
        # the dual level: at non-periodic boundaries its cells are centred on
        # boundary nodes and count half per cut axis
        g.advance_half(1)
        gu1 = g.get_grid(1)[0]
        ex1 = smooth(cell_points(d, N, h, bc, 1, xq))
        e2b, _ = g.l2_error(1, xq, wq, torch.from_numpy(ex1).cuda())
        np.testing.assert_allclose(np.sqrt(e2b), P.l2_error(1, gu1, nq, smooth), rtol=1e-11)
    g.close()


def pulse_errors(hb, N, precision, nsteps=200, m=3, lam=0.9, variant=0, engine=None):
    """Relative L2 error of the 3-D pulse workload after nsteps full steps
    (engine: the split engine to use, None for the default)."""
    import torch

    h = 1.0 / N
    cen, wid, amp = I.pulses_3d_config(0)
    g = hb.Hermite(3, m, N, 1.0, h, lam * h, variant, 0, precision=precision)
    if engine is not None:
        g.set_split_engine(engine)
    u0 = I.gaussian_data(3, m, N, h, I.PERIODIC, 0, cen, wid, amp)
    g.set_state(u0, np.zeros((N**3, m**3)) if variant != 1 else None)
    g.step(nsteps)
    T = g.time
    xq, wq = gauss(2 * m + 2)
    pts = torch.from_numpy(cell_points(3, N, h, 0, 0, xq)).cuda()
    ex = I.pulse_wave_3d(pts, T, cen, wid, amp, xp=torch).contiguous()
    e2, n2 = g.l2_error(0, xq, wq, ex)
    g.close()
    return float(np.sqrt(e2 / n2))


@pytest.mark.parametrize("N", [32, 48])
def test_split_accuracy_bar_3d_pulses(hb, N):
    e64 = pulse_errors(hb, N, hb.FP64)
    esp = pulse_errors(hb, N, hb.SPLIT32)
    assert e64 >= 1e-9
    assert esp <= 1.2 * e64, (N, e64, esp)
    # and the two arithmetics agree far below the discretisation error
    assert abs(esp - e64) <= 1e-3 * e64


def test_3d_pulse_workload_converges_at_order_2m_minus_1(hb):
    """The 3-D workload (m = 3, c dt/h = 0.9, the eight seeded pulses) run to
    the same time T = 1.40625 on 32^3, 48^3 and 64^3 cells: the FP64 error
    against the exact solution falls at the order 2m - 1 = 5 that Eq. vtrunc
    predicts for lambda < 1 (its nu h^(2m-1) term dominates), within [4.5, 6]."""
    import math

    T, lam = 1.40625, 0.9
    errs = []
    for N in (32, 48, 64):
        steps = int(round(T / (lam / N)))
        errs.append(pulse_errors(hb, N, hb.FP64, nsteps=steps, lam=T * N / steps))
    orders = [math.log(errs[0] / errs[1]) / math.log(1.5), math.log(errs[1] / errs[2]) / math.log(4 / 3)]
    assert all(4.5 <= o <= 6.0 for o in orders), (errs, orders)
