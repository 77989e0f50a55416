"""The allocation-free energy entry point (hermite_energy_noalloc).

Some callers cannot allocate device memory at the moment they need an energy
(code running where cudaMalloc is illegal or would stall the device, or a host
that only lends the library buffers it already owns).  hermite_energy_noalloc
serves them with a fixed array inside the library.  These tests call it
through the C ABI and check it against hermite_energy, the entry point that
uses the context's own scratch buffer, on two calls in a row.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from tests.gpu_util import hermite_cond, lib_built, need_gpu

pytestmark = pytest.mark.gpu
RTOL = 1e-12  # same FP64 reduction, different block partitioning


@pytest.fixture(scope="module")
def hb():
    need_gpu()
    return lib_built()


def _coef_major(u, v):
    import torch

    parts = [u.t()] + ([v.t()] if v is not None and v.numel() else [])
    return torch.cat(parts, 0).contiguous()


# the last two cases (1-D, m = 10) lie outside the sum-factorised kernel's
# range and run the per-parity-class quadratic forms instead
@pytest.mark.parametrize("d,m,N,variant,bc", [(3, 2, 8, 0, 0), (2, 3, 10, 0, 0), (1, 3, 33, 0, 1), (2, 2, 7, 1, 0),
                                              (1, 10, 17, 0, 0), (1, 10, 17, 1, 0)])
def test_noalloc_energy_matches_hermite_energy(hb, orc, d, m, N, variant, bc):
    import torch

    h = 1.0 / N
    P = orc.Problem(d, m, N, 1.0, h, 0.85 * h, variant, bc)
    g = hb.Hermite(d, m, N, 1.0, h, 0.85 * h, variant, bc)
    rng = np.random.default_rng(d * 10 + m)
    n0 = g.nodes(0)
    u = rng.standard_normal((n0, g.Nu))
    v = rng.standard_normal((n0, g.Nv)) if variant != hb.CONSERVATIVE else None
    g.set_state(u, v)
    for half in range(2):
        grid = half % 2 if variant != hb.CONSERVATIVE else 0
        ref = g.energy()
        nodes = g.nodes(grid)
        du = torch.empty((nodes, g.Nu), dtype=torch.float64, device="cuda")
        dv = torch.empty((nodes, g.Nv), dtype=torch.float64, device="cuda") if variant != hb.CONSERVATIVE else None
        g.get_grid_device(grid, du, dv)
        level = _coef_major(du, dv)
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        # beyond the sum-factorised range this entry point evaluates the dense
        # per-class forms where hermite_energy uses their Cholesky factors: the
        # two roundings differ by ~eps times the forms' condition
        rtol = RTOL if m <= 8 else 1e-10
        for _call in range(2):  # two calls in a row share the library's array
            out.fill_(float("nan"))
            g.energy_noalloc(grid, level, nodes, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            if variant == hb.CONSERVATIVE:
                # the second form is c^2 int |grad p|^2 of the primal level;
                # the first, the seminorm |p|^2_{m+1,..,m+1} of Sec. 4.2, is
                # pinned to the oracle's quadrature of the same level
                np.testing.assert_allclose(got[1], ref[0], rtol=rtol)
                lev = du.cpu().numpy()
                # the oracle interpolates by LU of the confluent Vandermonde
                # system: its forward error grows with that system's condition
                otol = max(1e-10, 20 * np.finfo(float).eps * hermite_cond(m))
                np.testing.assert_allclose(got[0], P.cons_forms(grid, lev, lev)[0], rtol=otol)
            else:
                np.testing.assert_allclose(got, ref[:2], rtol=rtol)
        g.advance_half(1)
    g.close()


def test_noalloc_padded_stride(hb):
    """A plane stride larger than the node count is honoured."""
    import torch

    N, m = 6, 2
    g = hb.Hermite(2, m, N, 1.0, 1.0 / N, 0.9 / N, 0, 0)
    rng = np.random.default_rng(3)
    g.set_state(rng.standard_normal((N * N, g.Nu)), rng.standard_normal((N * N, g.Nv)))
    ref = g.energy()
    du = torch.empty((N * N, g.Nu), dtype=torch.float64, device="cuda")
    dv = torch.empty((N * N, g.Nv), dtype=torch.float64, device="cuda")
    g.get_grid_device(0, du, dv)
    ld = N * N + 13
    level = torch.zeros((g.Nu + g.Nv, ld), dtype=torch.float64, device="cuda")
    level[:, : N * N] = _coef_major(du, dv)
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    g.energy_noalloc(0, level, ld, out)
    np.testing.assert_allclose(out.cpu().numpy(), ref[:2], rtol=RTOL)


def test_noalloc_rejects_too_many_cells(hb):
    """More than 2^21 cells: a clear HERMITE_ERR_ARG, nothing launched."""
    import torch

    N = (1 << 21) + 5
    g = hb.Hermite(1, 1, N, 1.0, 1.0 / N, 0.5 / N, 0, 0)
    level = torch.zeros((3, N), dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(hb.HermiteError) as e:
        g.energy_noalloc(0, level, N, out)
    assert e.value.code == -1 and "exceed the maximum" in str(e.value)
    assert torch.all(out == 0)


def test_noalloc_rejects_context_without_energy_forms(hb):
    """Batch problems are built without energy forms: the same
    HERMITE_ERR_STATE as hermite_energy, and nothing written."""
    import torch

    N, m = 8, 2
    b = hb.HermiteBatch([(2, m, N, 1.0, 1.0 / N, 0.9 / N, 0, 0)])
    g = b.problem(0)
    level = torch.zeros((g.Nu + g.Nv, N * N), dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(hb.HermiteError) as e:
        g.energy_noalloc(0, level, N * N, out)
    assert e.value.code == -6 and "without energy forms" in str(e.value)
    with pytest.raises(hb.HermiteError) as e:
        g.energy()
    assert e.value.code == -6
    torch.cuda.synchronize()
    assert torch.all(out == 0)
    b.close()
