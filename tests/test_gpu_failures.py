"""Failure detection without a GPU fault: injected allocation failures on the
host side, a bounded device wait that runs out, and canaries around the
output buffers of the ABI calls (nothing is written past the documented
extent)."""
import numpy as np
import pytest

from tests.gpu_util import lib_built, need_gpu, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    need_gpu()
    return lib_built()


@pytest.fixture
def no_fail(hb):
    yield
    assert hb.lib().hermite_debug_fail_alloc(0) == 0


def _problem(m=3):
    N = 6
    return (3, m, N, 1.0, 1.0 / N, 0.9 / N, 0, 0)


@pytest.mark.parametrize("precision", [0, 1])
def test_every_allocation_failure_of_create_is_reported_and_cleaned_up(hb, no_fail, precision):
    """Fail the k-th device allocation of a context build for every k: the
    call returns HERMITE_ERR_ALLOC (nothing half-built survives), and once the
    hook is off the same process builds and steps a context normally."""
    L = hb.lib()
    seen_success = False
    for k in range(1, 80):
        assert L.hermite_debug_fail_alloc(k) == 0
        try:
            g = hb.Hermite(*_problem(), precision=precision)
        except hb.HermiteError as e:
            assert e.code == -2, (k, e)
            continue
        # fewer than k allocations: the build succeeded before the hook fired
        g.close()
        seen_success = True
        break
    assert seen_success
    assert L.hermite_debug_fail_alloc(0) == 0
    g = hb.Hermite(*_problem(), precision=precision)
    rng = np.random.default_rng(0)
    u = rng.standard_normal((g.nodes(0), g.Nu))
    v = rng.standard_normal((g.nodes(0), g.Nv))
    g.set_state(u, v)
    g.step(1)
    ref = hb.Hermite(*_problem(), precision=precision)
    ref.set_state(u, v)
    ref.step(1)
    assert rel_l2(g.get_state()[0], ref.get_state()[0]) == 0.0


def test_allocation_failures_in_batches(hb, no_fail):
    import torch

    L = hb.lib()
    probs = [_problem(m) for m in (1, 2, 3)]
    failures = 0
    for k in range(1, 200):
        assert L.hermite_debug_fail_alloc(k) == 0
        try:
            b = hb.HermiteBatch(probs)
        except hb.HermiteError as e:
            assert e.code in (-2, -3), (k, e)
            failures += 1
            continue
        b.close()
        break
    assert failures > 3
    assert L.hermite_debug_fail_alloc(0) == 0
    b = hb.HermiteBatch(probs)
    b.set_stream(torch.cuda.Stream())
    n = sum(g.nodes(0) * g.Nu for g in b.problems)
    U = torch.zeros(n, dtype=torch.float64, device="cuda")
    # the batched state transfer allocates its descriptor table on first use
    assert L.hermite_debug_fail_alloc(1) == 0
    with pytest.raises(hb.HermiteError) as e:
        b.get_states_device(0, U)
    assert e.value.code == -2
    assert L.hermite_debug_fail_alloc(0) == 0
    b.get_states_device(0, U)  # works now
    b.close()


def test_bounded_device_wait_reports_timeout_and_context_survives(hb):
    import torch

    L = hb.lib()
    s = torch.cuda.current_stream().cuda_stream
    assert L.hnn_conv_status() == 0
    assert L.hnn_wait_selftest(s) == 0
    assert L.hnn_conv_status() == -5  # the wait gave up and said so
    assert L.hnn_conv_status() == 0   # and the flag was cleared
    # the context is still usable: a tensor-core convolution runs and is right
    x = torch.ones((1, 2, 128, 64), dtype=torch.bfloat16, device="cuda")
    w = torch.full((64, 9, 64), 0.125, dtype=torch.bfloat16, device="cuda")
    y = torch.empty((1, 2, 128, 64), dtype=torch.float32, device="cuda")
    assert L.hnn_conv3x3_fwd(x.data_ptr(), w.data_ptr(), None, None, 1, 2, 128, 64, 64, 1, 0, None, y.data_ptr(),
                             s) == 0
    torch.cuda.synchronize()
    assert torch.all(y == 9 * 64 * 0.125).item()
    assert L.hnn_conv_status() == 0


CANARY = 1.2345e300


def _canaried(torch, n, dtype=None, fill=CANARY):
    import torch as T

    dtype = dtype or T.float64
    buf = T.full((n + 97,), fill, dtype=dtype, device="cuda")
    return buf


def test_outputs_stay_inside_their_extent(hb):
    import torch

    L = hb.lib()
    s = torch.cuda.current_stream().cuda_stream
    # single-problem device download
    g = hb.Hermite(2, 3, 5, 1.0, 0.2, 0.18, 0, 1)  # Dirichlet: 36 primal, 25 dual nodes
    rng = np.random.default_rng(1)
    g.set_state(rng.standard_normal((g.nodes(0), g.Nu)), rng.standard_normal((g.nodes(0), g.Nv)))
    for grid in (0, 1):
        nu, nv = g.nodes(grid) * g.Nu, g.nodes(grid) * g.Nv
        U, V = _canaried(torch, nu), _canaried(torch, nv)
        g.get_grid_device(grid, U, V)
        torch.cuda.synchronize()
        assert torch.all(U[nu:] == CANARY).item() and torch.all(V[nv:] == CANARY).item()
        assert not torch.any(U[:nu] == CANARY).item()
    # batched download
    b = hb.HermiteBatch([(2, m, 4 + m, 1.0, 0.2, 0.15, 0, 0) for m in (2, 3, 4)])
    nu = sum(p.nodes(0) * p.Nu for p in b.problems)
    nv = sum(p.nodes(0) * p.Nv for p in b.problems)
    U, V = _canaried(torch, nu), _canaried(torch, nv)
    b.get_states_device(0, U, V)
    torch.cuda.synchronize()
    assert torch.all(U[nu:] == CANARY).item() and torch.all(V[nv:] == CANARY).item()
    b.close()
    # network kernels: forward outputs (both engines), pack, unpack
    B, H = 1, 3
    for cin, cout in ((64, 64), (32, 64), (64, 32)):
        x = torch.randn((B * H * 128 * cin,), device="cuda").to(torch.bfloat16)
        w = (torch.randn((cout * 9 * cin,), device="cuda") * 0.1).to(torch.bfloat16)
        n = B * H * 128 * cout
        y32 = _canaried(torch, n, torch.float32, 7.0e30)
        y16 = torch.full((n + 97,), 3.0, dtype=torch.bfloat16, device="cuda")
        assert L.hnn_conv3x3_fwd(x.data_ptr(), w.data_ptr(), None, None, B, H, 128, cin, cout, 2, 0, y16.data_ptr(),
                                 y32.data_ptr(), s) == 0
        torch.cuda.synchronize()
        assert torch.all(y32[n:] == 7.0e30).item() and torch.all(y16[n:] == 3.0).item()
    n, Nu, Nv, C = 300, 16, 9, 32
    u = torch.randn((n, Nu), dtype=torch.float64, device="cuda")
    v = torch.randn((n, Nv), dtype=torch.float64, device="cuda")
    one = torch.ones(25, dtype=torch.float64, device="cuda")
    xp = torch.full((n * C + 97,), 3.0, dtype=torch.bfloat16, device="cuda")
    assert L.hnn_pack_state(u.data_ptr(), v.data_ptr(), n, Nu, Nv, 0.5, one.data_ptr(), one.data_ptr(), C,
                            xp.data_ptr(), s) == 0
    yv = torch.randn((n * C,), dtype=torch.float32, device="cuda")
    uo, vo = _canaried(torch, n * Nu), _canaried(torch, n * Nv)
    assert L.hnn_unpack_state(u.data_ptr(), v.data_ptr(), yv.data_ptr(), n, Nu, Nv, 0.5, one.data_ptr(), C,
                              uo.data_ptr(), vo.data_ptr(), s) == 0
    torch.cuda.synchronize()
    assert torch.all(xp[n * C:] == 3.0).item()
    assert torch.all(uo[n * Nu:] == CANARY).item() and torch.all(vo[n * Nv:] == CANARY).item()
