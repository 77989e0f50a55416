"""Network kernels of the learned super-stepper (include/hermite_nn.h) against
the FP64 reference oracle/conv_ref.py, evaluated on the same BF16-rounded
inputs: forward, input gradient (flipped weights + ReLU mask), weight and bias
gradients, loss, Adam, the state conversions, and a whole-network gradient
with the kernels' BF16 rounding points emulated in the reference.

Tolerances: the products of BF16 numbers are exact in FP32, so only the FP32
accumulation differs from the FP64 reference; recursive FP32 summation of n
terms is off by at most about n * 2^-24 times the sum of |terms| (S).  The
bound used is 1e-4 * S (n <= 576 per output for the forward kernels, partial
sums over 128-node rows for the weight gradient)."""
import numpy as np
import pytest

from oracle import conv_ref as cr
from tests.gpu_util import lib_built, need_gpu

pytestmark = pytest.mark.gpu

W = 128


@pytest.fixture(scope="module")
def hb():
    need_gpu()
    return lib_built()


def _bf(a):
    """Host float array -> (BF16 device tensor, FP64 host copy of the rounded values)."""
    import torch

    t = torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.cuda(), t.float().numpy().astype(np.float64)


def _f32(a):
    import torch

    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _rng(seed):
    return np.random.default_rng(seed)


def _stream():
    import torch

    return torch.cuda.current_stream().cuda_stream


def _host(t):
    import torch

    torch.cuda.synchronize()
    return t.float().cpu().numpy().astype(np.float64)


def _conv_abs(x, w, b, dil):
    return cr.conv3x3(np.abs(x), np.abs(w), None if b is None else np.abs(b), dil)


@pytest.fixture
def engine(hb, request):
    """Selects the convolution engine for one test (0: tcgen05 where supported,
    1: mma.sync) and checks afterwards that no tensor-core wait ran out."""
    L = hb.lib()
    assert L.hnn_set_conv_engine(request.param) == 0
    yield request.param
    assert L.hnn_set_conv_engine(0) == 0
    assert L.hnn_conv_status() == 0


@pytest.mark.parametrize("N", [64, 32])
def test_tensor_core_selftest_gemm(hb, N):
    """One 128 x N x 64 tile through tcgen05 (shared-memory descriptors,
    instruction descriptor, tensor-memory accumulator and load) against FP64."""
    import torch

    rng = _rng(40 + N)
    A, Ah = _bf(rng.standard_normal((128, 64)))
    B, Bh = _bf(rng.standard_normal((N, 64)))
    D = torch.full((128, N), float("nan"), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert hb.lib().hnn_tc_gemm_selftest(A.data_ptr(), B.data_ptr(), D.data_ptr(), N, st.data_ptr(), _stream()) == 0
    got = _host(D)
    assert int(st.item()) == 0
    ref = Ah @ Bh.T
    S = np.abs(Ah) @ np.abs(Bh).T
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - ref) / S) <= 1e-4


@pytest.mark.parametrize("engine", [0, 1], indirect=True)
@pytest.mark.parametrize("cin,cout", [(32, 64), (64, 64), (64, 32), (32, 32)])
@pytest.mark.parametrize("dil", [1, 3, 8, 12])
@pytest.mark.parametrize("relu", [0, 1])
def test_conv_forward(hb, engine, cin, cout, dil, relu):
    import torch

    B, H = 2, 5  # H < 2*dil: the row offsets wrap around more than once
    rng = _rng(100 + cin + cout + dil)
    x, xh = _bf(rng.standard_normal((B, H, W, cin)))
    w, wh = _bf(rng.standard_normal((cout, 9, cin)) * 0.1)
    bh = rng.standard_normal(cout).astype(np.float32).astype(np.float64)
    b = _f32(bh)
    y32 = torch.empty((B, H, W, cout), dtype=torch.float32, device="cuda")
    y16 = torch.empty((B, H, W, cout), dtype=torch.bfloat16, device="cuda")
    rc = hb.lib().hnn_conv3x3_fwd(x.data_ptr(), w.data_ptr(), b.data_ptr(), None, B, H, W, cin, cout, dil, relu,
                                  y16.data_ptr(), y32.data_ptr(), _stream())
    assert rc == 0
    ref = cr.conv3x3(xh, wh, bh, dil)
    if relu:
        ref = np.maximum(ref, 0)
    S = _conv_abs(xh, wh, bh, dil)
    got = _host(y32)
    assert np.max(np.abs(got - ref) / S) <= 1e-4
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
    g16 = _host(y16)
    assert np.all(np.abs(g16 - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-4 * S)


@pytest.mark.parametrize("engine", [0, 1], indirect=True)
@pytest.mark.parametrize("cin,cout", [(32, 64), (64, 64), (64, 32)])
@pytest.mark.parametrize("dil", [1, 2, 4, 8])
def test_input_gradient_via_flipped_weights_and_mask(hb, engine, cin, cout, dil):
    import torch

    B, H = 2, 6
    rng = _rng(200 + cin + cout + dil)
    dy, dyh = _bf(rng.standard_normal((B, H, W, cout)))
    w, wh = _bf(rng.standard_normal((cout, 9, cin)) * 0.1)
    a, ah = _bf(np.maximum(rng.standard_normal((B, H, W, cin)), 0))  # a ReLU output: about half zeros
    wt = torch.empty(cin * 9 * cout, dtype=torch.bfloat16, device="cuda")
    dx32 = torch.empty((B, H, W, cin), dtype=torch.float32, device="cuda")
    dx16 = torch.empty((B, H, W, cin), dtype=torch.bfloat16, device="cuda")
    L = hb.lib()
    assert L.hnn_flip_weights(w.data_ptr(), cout, cin, wt.data_ptr(), _stream()) == 0
    assert L.hnn_conv3x3_fwd(dy.data_ptr(), wt.data_ptr(), None, a.data_ptr(), B, H, W, cout, cin, dil, 0,
                             dx16.data_ptr(), dx32.data_ptr(), _stream()) == 0
    dx, _, _ = cr.conv3x3_backward(np.zeros((B, H, W, cin)), wh, dyh, dil)
    ref = dx * (ah > 0)
    wt_h = _host(wt).reshape(cin, 9, cout)
    assert np.array_equal(wt_h, np.transpose(wh[:, ::-1, :], (2, 1, 0)))
    S = np.abs(cr.conv3x3_backward(np.zeros((B, H, W, cin)), np.abs(wh), np.abs(dyh), dil)[0])
    got = _host(dx32)
    assert np.all(got[ah <= 0] == 0)
    assert np.max(np.abs(got - ref) / (S + 1e-30)) <= 1e-4
    g16 = _host(dx16)
    assert np.all(np.abs(g16 - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-4 * S)


@pytest.mark.parametrize("cin,cout", [(32, 64), (64, 64), (64, 32)])
@pytest.mark.parametrize("dil", [1, 4, 8])
def test_weight_and_bias_gradients_accumulate(hb, cin, cout, dil):
    B, H = 2, 5
    rng = _rng(300 + cin + cout + dil)
    x, xh = _bf(rng.standard_normal((B, H, W, cin)))
    dy, dyh = _bf(rng.standard_normal((B, H, W, cout)))
    dw0 = rng.standard_normal((cout, 9, cin)).astype(np.float32)
    db0 = rng.standard_normal(cout).astype(np.float32)
    dw, db = _f32(dw0), _f32(db0)
    L = hb.lib()
    assert L.hnn_conv3x3_wgrad(x.data_ptr(), dy.data_ptr(), B, H, W, cin, cout, dil, dw.data_ptr(), _stream()) == 0
    assert L.hnn_bias_grad(dy.data_ptr(), B * H * W, cout, db.data_ptr(), _stream()) == 0
    _, gw, gb = cr.conv3x3_backward(xh, np.zeros((cout, 9, cin)), dyh, dil)
    _, Sw, Sb = cr.conv3x3_backward(np.abs(xh), np.zeros((cout, 9, cin)), np.abs(dyh), dil)
    got_w, got_b = _host(dw), _host(db)
    assert np.max(np.abs(got_w - (dw0 + gw)) / (Sw + np.abs(dw0))) <= 1e-4
    assert np.max(np.abs(got_b - (db0 + gb)) / (Sb + np.abs(db0))) <= 1e-4


@pytest.mark.parametrize("engine", [0, 1], indirect=True)
def test_full_size_forward_and_weight_gradient_sampled(hb, engine):
    """The launch configuration of training and inference (32 images of
    128 x 128, 64 -> 64 channels, dilation 8): sampled outputs and weight
    gradient entries computed one by one in FP64."""
    import torch

    B, H, cin, cout, dil = 32, 128, 64, 64, 8
    g = torch.Generator().manual_seed(7)
    x = torch.randn((B, H, W, cin), generator=g).to(torch.bfloat16)
    dy = torch.randn((B, H, W, cout), generator=g).to(torch.bfloat16)
    w = (torch.randn((cout, 9, cin), generator=g) * 0.05).to(torch.bfloat16)
    xd, dyd, wd = x.cuda(), dy.cuda(), w.cuda()
    y = torch.empty((B, H, W, cout), dtype=torch.float32, device="cuda")
    dw = torch.zeros((cout, 9, cin), dtype=torch.float32, device="cuda")
    L = hb.lib()
    assert L.hnn_conv3x3_fwd(xd.data_ptr(), wd.data_ptr(), None, None, B, H, W, cin, cout, dil, 0, None,
                             y.data_ptr(), _stream()) == 0
    assert L.hnn_conv3x3_wgrad(xd.data_ptr(), dyd.data_ptr(), B, H, W, cin, cout, dil, dw.data_ptr(), _stream()) == 0
    yh, dwh = _host(y), _host(dw)
    xh = x.float().numpy().astype(np.float64)
    dyh = dy.float().numpy().astype(np.float64)
    wh = w.float().numpy().astype(np.float64)
    rng = _rng(8)
    for _ in range(200):
        b, i, j, co = (int(rng.integers(0, n)) for n in (B, H, W, cout))
        s = S = 0.0
        for tap in range(9):
            ky, kx = divmod(tap, 3)
            xv = xh[b, (i + (ky - 1) * dil) % H, (j + (kx - 1) * dil) % W]
            s += float(xv @ wh[co, tap])
            S += float(np.abs(xv) @ np.abs(wh[co, tap]))
        assert abs(yh[b, i, j, co] - s) <= 1e-4 * S
    for _ in range(24):
        co, tap, ci = int(rng.integers(0, cout)), int(rng.integers(0, 9)), int(rng.integers(0, cin))
        xs = cr.shifted(xh[..., ci:ci + 1], tap, dil)[..., 0]
        s = float(np.sum(dyh[..., co] * xs))
        S = float(np.sum(np.abs(dyh[..., co] * xs)))
        assert abs(dwh[co, tap, ci] - s) <= 1e-4 * S


def test_mse_and_adam(hb):
    import torch

    rng = _rng(9)
    npix, C = 1000, 32
    y = rng.standard_normal((npix, C)).astype(np.float32)
    t = rng.standard_normal((npix, C)).astype(np.float32)
    wch = np.abs(rng.standard_normal(C)).astype(np.float32)
    wch[25:] = 0
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    dy = torch.empty((npix, C), dtype=torch.bfloat16, device="cuda")
    L = hb.lib()
    assert L.hnn_mse(_f32(y).data_ptr(), _f32(t).data_ptr(), _f32(wch).data_ptr(), npix, C, 0.001, loss.data_ptr(),
                     dy.data_ptr(), _stream()) == 0
    ref_loss, ref_dy = cr.weighted_mse(y, t, wch, 0.001)
    assert abs(loss.item() - ref_loss) <= 1e-6 * ref_loss
    got = _host(dy)
    assert np.all(np.abs(got - ref_dy) <= 2.0 ** -8 * np.abs(ref_dy) + 1e-12)
    assert np.all(got[:, 25:] == 0)

    n = 5000
    p0, g0, m0 = (rng.standard_normal(n).astype(np.float32) for _ in range(3))
    v0 = np.abs(rng.standard_normal(n)).astype(np.float32)
    p, g, m, v = _f32(p0), _f32(g0), _f32(m0), _f32(v0)
    p16 = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    assert L.hnn_adam(p.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), n, 1e-3, 0.9, 0.999, 1e-8, 3,
                      p16.data_ptr(), _stream()) == 0
    # the kernel works with the FP32 values of the hyper-parameters (1 - beta2
    # is then 0.00099998713, not 0.001): the reference takes the same values
    f = lambda a: float(np.float32(a))
    rp, rm, rv = cr.adam_step(p0.astype(np.float64), g0.astype(np.float64), m0.astype(np.float64),
                              v0.astype(np.float64), f(1e-3), f(0.9), f(0.999), f(1e-8), 3)
    assert np.allclose(_host(p), rp, rtol=1e-6, atol=1e-7)
    assert np.allclose(_host(m), rm, rtol=1e-6, atol=1e-7)
    assert np.allclose(_host(v), rv, rtol=1e-6, atol=1e-7)
    assert np.all(_host(g) == 0)
    assert np.array_equal(_host(p16), torch.as_tensor(_host(p).astype(np.float32)).to(torch.bfloat16).float().numpy())


def test_state_conversions(hb):
    import torch

    rng = _rng(10)
    n, Nu, Nv, C, vs = 777, 16, 9, 32, 0.01
    u = rng.standard_normal((n, Nu))
    v = rng.standard_normal((n, Nv)) * 50
    ud, vd = torch.as_tensor(u).cuda(), torch.as_tensor(v).cuda()
    s_ref = np.concatenate([u, vs * v], 1)
    L = hb.lib()
    out = torch.zeros((n, Nu + Nv), dtype=torch.float32, device="cuda")
    assert L.hnn_state_to_f32(ud.data_ptr(), vd.data_ptr(), n, Nu, Nv, vs, out.data_ptr(), Nu + Nv, _stream()) == 0
    assert np.array_equal(_host(out), s_ref.astype(np.float32).astype(np.float64))
    shift, scale = rng.standard_normal(25), np.abs(rng.standard_normal(25)) + 0.5
    x = torch.empty((n, C), dtype=torch.bfloat16, device="cuda")
    assert L.hnn_pack_state(ud.data_ptr(), vd.data_ptr(), n, Nu, Nv, vs, torch.as_tensor(shift).cuda().data_ptr(),
                            torch.as_tensor(scale).cuda().data_ptr(), C, x.data_ptr(), _stream()) == 0
    f = np.float32
    sf = np.concatenate([u.astype(f), v.astype(f) * f(vs)], 1)
    xr = (sf - shift.astype(f)) * (1.0 / scale).astype(f)  # the kernel's FP32 arithmetic
    got = _host(x)
    assert np.array_equal(got[:, :25], torch.as_tensor(xr).to(torch.bfloat16).float().numpy())
    assert np.allclose(got[:, :25], (s_ref - shift) / scale, rtol=2.0 ** -8, atol=1e-6)
    assert np.all(got[:, 25:] == 0)
    y = rng.standard_normal((n, C)).astype(np.float32)
    ds = np.abs(rng.standard_normal(25)) + 0.1
    uo = torch.empty_like(ud)
    vo = torch.empty_like(vd)
    assert L.hnn_unpack_state(ud.data_ptr(), vd.data_ptr(), _f32(y).data_ptr(), n, Nu, Nv, vs,
                              torch.as_tensor(ds).cuda().data_ptr(), C, uo.data_ptr(), vo.data_ptr(), _stream()) == 0
    torch.cuda.synchronize()
    d = (ds.astype(np.float32) * y[:, :25]).astype(np.float64)  # the FP32 change
    assert np.allclose(uo.cpu().numpy(), u + d[:, :16], rtol=1e-15, atol=1e-15)
    assert np.allclose(vo.cpu().numpy(), v + d[:, 16:25] / vs, rtol=1e-14, atol=1e-14)
    assert np.allclose(uo.cpu().numpy(), u + ds[:16] * y[:, :16], rtol=1e-6, atol=1e-7)
    out2 = torch.zeros(2, dtype=torch.float64, device="cuda")
    assert L.hnn_sqdiff(uo.data_ptr(), vo.data_ptr(), ud.data_ptr(), vd.data_ptr(), n, Nu, Nv, vs, out2.data_ptr(),
                        _stream()) == 0
    d = np.concatenate([uo.cpu().numpy() - u, vs * (vo.cpu().numpy() - v)], 1)
    o = out2.cpu().numpy()
    assert o[0] == pytest.approx(np.sum(d * d), rel=1e-12)
    assert o[1] == pytest.approx(np.sum(s_ref * s_ref), rel=1e-12)


def test_make_pairs_and_moments(hb):
    import torch

    rng = _rng(11)
    ntr, nlev, n, C0, C = 3, 4, 500, 25, 32
    lev = rng.standard_normal((ntr, nlev, n, C0)).astype(np.float32)
    levd = _f32(lev)
    pairs = [(0, 1), (2, 2), (1, 0)]
    src = torch.as_tensor([(t * nlev + k) * n * C0 for t, k in pairs], dtype=torch.int64).cuda()
    dst = src + n * C0
    shift, scale, dscale = rng.standard_normal(C0), np.abs(rng.standard_normal(C0)) + 0.5, np.abs(
        rng.standard_normal(C0)) + 0.5
    x = torch.empty((3, n, C), dtype=torch.bfloat16, device="cuda")
    t = torch.empty((3, n, C), dtype=torch.float32, device="cuda")
    L = hb.lib()
    dev = lambda a: torch.as_tensor(a).cuda()
    sh, sc, ds = dev(shift), dev(scale), dev(dscale)
    assert L.hnn_make_pairs(levd.data_ptr(), src.data_ptr(), dst.data_ptr(), 3, n, C0, sh.data_ptr(), sc.data_ptr(),
                            ds.data_ptr(), C, x.data_ptr(), t.data_ptr(), _stream()) == 0
    xh, th = _host(x), _host(t)
    for s, (tr, k) in enumerate(pairs):
        a = lev[tr, k].astype(np.float64)
        b = lev[tr, k + 1].astype(np.float64)
        f = np.float32
        xr = (a.astype(f) - shift.astype(f)) * (1.0 / scale).astype(f)
        assert np.array_equal(xh[s, :, :C0], torch.as_tensor(xr).to(torch.bfloat16).float().numpy())
        assert np.allclose(th[s, :, :C0], (b - a) / dscale, rtol=1e-6, atol=1e-6)
        assert np.all(xh[s, :, C0:] == 0) and np.all(th[s, :, C0:] == 0)
    mom = torch.zeros(2 * C0, dtype=torch.float64, device="cuda")
    assert L.hnn_moments(levd[0, 1].data_ptr(), levd[0, 0].data_ptr(), n, C0, mom.data_ptr(), _stream()) == 0
    d = lev[0, 1].astype(np.float64) - lev[0, 0]
    mh = mom.cpu().numpy()
    assert np.allclose(mh[:C0], d.sum(0), rtol=1e-10, atol=1e-10)
    assert np.allclose(mh[C0:], (d * d).sum(0), rtol=1e-10)


@pytest.mark.parametrize("act", ["relu", "none"])
def test_network_gradient_against_fp64_reference(hb, act):
    """Whole network on a tiny batch (1 x 4 x 128): gradients of the kernels
    against the FP64 reference with the kernels' BF16 rounding points
    emulated (activations, loss gradient, input gradients)."""
    import torch

    from paper_1802_05246_b300.learned import CPAD, ConvNet

    B, H = 1, 4
    relu = act == "relu"
    net = ConvNet(cin=25, cout=25, seed=3, act=act)
    rng = _rng(12)
    flat = net.get_params()
    # a nonzero last layer so that every layer receives a gradient
    wo, bo, ci, co = net.layout[-1]
    flat[wo:wo + co * 9 * ci] = (rng.standard_normal((co, 9, ci)) * 0.05).astype(np.float32).reshape(-1)
    lastw = flat[wo:wo + co * 9 * ci].reshape(co, 9, ci)
    lastw[25:] = 0
    for (wo_, bo_, ci_, co_) in net.layout:
        flat[bo_:bo_ + co_] = (rng.standard_normal(co_) * 0.1).astype(np.float32)
    flat[bo:bo + co][25:] = 0
    net.set_params(flat)
    xin = rng.standard_normal((B, H, W, CPAD))
    xin[..., 25:] = 0
    x, xh = _bf(xin)
    tgt = rng.standard_normal((B, H, W, CPAD)).astype(np.float32)
    tgt[..., 25:] = 0
    wch = np.ones(CPAD, dtype=np.float32)
    wch[25:] = 0
    out = net.forward(x, B, H)
    bufs = net.buffers(B, H)
    scale = 1.0 / (B * H * W * 25)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    L = hb.lib()
    assert L.hnn_mse(out.data_ptr(), _f32(tgt).data_ptr(), _f32(wch).data_ptr(), B * H * W, CPAD, scale,
                     loss.data_ptr(), bufs["dyout"].data_ptr(), _stream()) == 0
    net.backward(x, B, bufs["dyout"], H)
    torch.cuda.synchronize()
    G = net.G.cpu().numpy().astype(np.float64)

    def r16(a):
        return torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)

    params = [(r16(w), b.astype(np.float64)) for (w, b) in net.layer_params()]
    # forward with BF16 activations, as the kernels store them
    acts, a = [], xh
    for li, ((w, b), d) in enumerate(zip(params, net.dils)):
        z = cr.conv3x3(a, w, b, d)
        a = r16(np.maximum(z, 0) if relu else z) if li + 1 < len(params) else z
        acts.append(a)
    lref, dy = cr.weighted_mse(acts[-1], tgt, wch, scale)
    assert abs(loss.item() - lref) <= 1e-3 * lref
    dy = r16(dy)
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        inp = xh if li == 0 else acts[li - 1]
        dx, dw, db = cr.conv3x3_backward(inp, params[li][0], dy, net.dils[li])
        grads[li] = (dw, db)
        if li > 0:
            dy = r16(dx * (acts[li - 1] > 0) if relu else dx)
    # and the pure FP64 network (no rounding) for scale
    acts64 = cr.net_forward(xh, params, net.dils, relu)
    _, dy64 = cr.weighted_mse(acts64[-1], tgt, wch, scale)
    grads64 = cr.net_backward(xh, params, net.dils, acts64, dy64, relu)
    for li, (wo, bo, ci, co) in enumerate(net.layout):
        gw = G[wo:wo + co * 9 * ci].reshape(co, 9, ci)
        gb = G[bo:bo + co]
        assert np.linalg.norm(gw - grads[li][0]) <= 1e-2 * np.linalg.norm(grads[li][0]), li
        assert np.linalg.norm(gb - grads[li][1]) <= 1e-2 * np.linalg.norm(grads[li][1]) + 1e-12, li
        assert np.linalg.norm(gw - grads64[li][0]) <= 5e-2 * np.linalg.norm(grads64[li][0]), li


def test_argument_errors(hb):
    L = hb.lib()
    s = _stream()
    assert L.hnn_conv3x3_fwd(1, 1, None, None, 1, 1, 64, 32, 64, 1, 0, 1, None, s) == -1  # W != 128
    assert L.hnn_conv3x3_fwd(1, 1, None, None, 1, 1, 128, 48, 64, 1, 0, 1, None, s) == -1  # channels
    assert L.hnn_conv3x3_fwd(1, 1, None, None, 1, 1, 128, 32, 64, 0, 0, 1, None, s) == -1  # dilation
    assert L.hnn_conv3x3_fwd(1, 1, None, None, 1, 1, 128, 32, 64, 1, 0, None, None, s) == -1  # no output
    assert L.hnn_conv3x3_fwd(None, None, None, None, 0, 5, 128, 32, 64, 1, 0, None, None, s) == 0  # empty batch
    assert L.hnn_conv3x3_wgrad(1, 1, 1, 1, 128, 32, 32, 1, 1, s) == -1  # unsupported pair
    assert L.hnn_adam(1, 1, 1, 1, 10, 0.1, 0.9, 0.999, 1e-8, 0, None, s) == -1  # t = 0
