"""Learned super-stepper for 2-D periodic dissipative Hermite problems.

A five-layer dilated 3x3 convolution network maps the primal nodal data of an
m = 3, 128 x 128 periodic dissipative problem at time t to the data at
t + K dt (K = 16 full steps by default).  The library's CUDA kernels
(include/hermite_nn.h) run the forward pass, the backward pass and the Adam
update: BF16 activations and weights, FP32 accumulation on the tensor cores.

* Input: the 16 u and 9 v coefficients per node in "metric space" (v scaled
  by h/c), standardised per channel and zero-padded to 32 channels.
* Output: the standardised change over K steps, added to the FP64 input
  (residual form x + s * f(x)).
* Receptive field: the dependence cone of K full Hermite steps reaches K
  cells (each half-step couples a node to the 2^d corners of its cell), so
  the dilations (1, 2, 4, 8, 1) give a radius of 16 nodes.
* Data: trajectories of the batched Hermite solver from seeded Gaussian-pulse
  initial data, states stored every K steps.
* Check: the commutation residual r = |H(N(x)) - N(H(x))| / |N(x)| with one
  true Hermite step H, calibrated against the true K-step error on held-out
  data; a prediction whose estimated error exceeds the bar is replaced by K
  plain Hermite steps.

PyTorch only provides device memory and the stream; every arithmetic step runs
in the library's kernels.
"""
from __future__ import annotations

import argparse
import math
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import DISSIPATIVE, FP64, PERIODIC, PRIMAL, HermiteBatch, HermiteError, inputs, lib

WIDTH = 128  # image width handled by the convolution kernels
CPAD = 32  # network input and output channels (state channels, zero padded)


def _p(t):
    return None if t is None else t.data_ptr()


def _check(rc, what):
    if rc != 0:
        raise HermiteError(rc, what)


def _stream():
    import torch

    return torch.cuda.current_stream().cuda_stream


class ConvNet:
    """Dilated 3x3 convolution network, NHWC, BF16 storage, FP32 accumulation.

    Layers l = 0..L-1 map chans[l] -> chans[l+1] channels with dilation
    dilations[l]; act = "relu" puts a ReLU after every layer but the last,
    act = "none" makes the network a composition of linear convolutions.
    Parameters live in one flat FP32 buffer (weights [co][9][ci] then bias
    [co] per layer) with a BF16 copy that the forward kernels read."""

    def __init__(self, cin=25, cout=25, width=64, dilations=(1, 2, 4, 8, 1), seed=0, act="relu"):
        import torch

        if not (1 <= cin <= CPAD and 1 <= cout <= CPAD):
            raise ValueError("cin and cout must be in 1..32")
        if act not in ("relu", "none"):
            raise ValueError("act must be 'relu' or 'none'")
        self.act = act
        self.relu = 1 if act == "relu" else 0
        self.dils = tuple(int(d) for d in dilations)
        nl = len(self.dils)
        self.chans = [CPAD] + [int(width)] * (nl - 1) + [CPAD]
        self.cin, self.cout = int(cin), int(cout)
        self.layout = []
        n = 0
        for layer in range(nl):
            ci, co = self.chans[layer], self.chans[layer + 1]
            wo = n
            n += -(-co * 9 * ci // 64) * 64
            bo = n
            n += -(-co // 64) * 64
            self.layout.append((wo, bo, ci, co))
        self.nparam = n
        f32 = dict(dtype=torch.float32, device="cuda")
        self.P = torch.zeros(n, **f32)
        self.G = torch.zeros(n, **f32)
        self.M = torch.zeros(n, **f32)
        self.V = torch.zeros(n, **f32)
        self.P16 = torch.zeros(n, dtype=torch.bfloat16, device="cuda")
        self.wt = [torch.empty(co * 9 * ci, dtype=torch.bfloat16, device="cuda") for (_, _, ci, co) in self.layout]
        self.t = 0
        self._bufs = {}
        self.set_params(self.initial_params(seed))

    # -- parameters ---------------------------------------------------------
    def initial_params(self, seed):
        """Normal weights with variance 2/fan_in (ReLU) or 1/fan_in (linear)
        for layers 0..L-2, zero last layer (the residual form starts as the
        identity map), zero biases, zero padded channels."""
        rng = np.random.default_rng(seed)
        flat = np.zeros(self.nparam, dtype=np.float32)
        for layer, (wo, bo, ci, co) in enumerate(self.layout):
            fan = 9 * (self.cin if layer == 0 else ci)
            if layer + 1 < len(self.layout):
                w = rng.standard_normal((co, 9, ci)) * math.sqrt((2.0 if self.relu else 1.0) / fan)
                if layer == 0:
                    w[:, :, self.cin:] = 0.0
            else:
                w = np.zeros((co, 9, ci))
            flat[wo:wo + co * 9 * ci] = w.reshape(-1)
        return flat

    def set_params(self, flat):
        """Load FP32 parameters (host array) and derive the BF16 copy with a
        zero-rate Adam call (moments and step count reset)."""
        import torch

        flat = np.ascontiguousarray(flat, dtype=np.float32)
        if flat.size != self.nparam:
            raise ValueError("parameter count mismatch")
        self.P.copy_(torch.from_numpy(flat))
        self.M.zero_()
        self.V.zero_()
        self.G.zero_()
        _check(lib().hnn_adam(_p(self.P), _p(self.G), _p(self.M), _p(self.V), self.nparam, 0.0, 0.9, 0.999, 1e-8, 1,
                              _p(self.P16), _stream()), "adam (copy)")
        self.t = 0

    def get_params(self):
        return self.P.detach().cpu().numpy().copy()

    def layer_params(self, flat=None):
        """[(w [co,9,ci], b [co])] views of a flat host parameter array."""
        flat = self.get_params() if flat is None else flat
        return [(flat[wo:wo + co * 9 * ci].reshape(co, 9, ci), flat[bo:bo + co]) for (wo, bo, ci, co) in self.layout]

    # -- buffers ------------------------------------------------------------
    def buffers(self, B, H=WIDTH):
        import torch

        key = (B, H)
        if key not in self._bufs:
            self._bufs.clear()
            bf = dict(dtype=torch.bfloat16, device="cuda")
            shape = (B, H, WIDTH)
            self._bufs[key] = {
                "act": [torch.empty(shape + (co,), **bf) for (_, _, _, co) in self.layout[:-1]],
                "out": torch.empty(shape + (CPAD,), dtype=torch.float32, device="cuda"),
                "dy": [torch.empty(shape + (max(self.chans),), **bf) for _ in range(2)],
                "dyout": torch.empty(shape + (CPAD,), **bf),
            }
        return self._bufs[key]

    # -- passes ---------------------------------------------------------------
    def forward(self, x, B, H=WIDTH):
        """x: BF16 [B,H,128,32] device tensor -> FP32 [B,H,128,32] (internal buffer)."""
        L = lib()
        s = _stream()
        bufs = self.buffers(B, H)
        a = x
        p16, p32 = self.P16.data_ptr(), self.P.data_ptr()
        for layer, ((wo, bo, ci, co), d) in enumerate(zip(self.layout, self.dils)):
            last = layer + 1 == len(self.layout)
            y16 = None if last else bufs["act"][layer]
            y32 = bufs["out"] if last else None
            _check(L.hnn_conv3x3_fwd(_p(a), p16 + 2 * wo, p32 + 4 * bo, None, B, H, WIDTH, ci, co, d,
                                     0 if last else self.relu, _p(y16), _p(y32), s), "conv forward")
            a = y16
        return bufs["out"]

    def backward(self, x, B, dy_out, H=WIDTH):
        """Accumulate parameter gradients of sum(dy_out * forward(x)) into G
        (forward(x) must be the last forward pass; dy_out BF16 [B,H,128,32])."""
        L = lib()
        s = _stream()
        bufs = self.buffers(B, H)
        acts = bufs["act"]
        p16, g = self.P16.data_ptr(), self.G.data_ptr()
        dy = dy_out
        for layer in range(len(self.layout) - 1, -1, -1):
            wo, bo, ci, co = self.layout[layer]
            d = self.dils[layer]
            inp = x if layer == 0 else acts[layer - 1]
            _check(L.hnn_conv3x3_wgrad(_p(inp), _p(dy), B, H, WIDTH, ci, co, d, g + 4 * wo, s), "weight gradient")
            _check(L.hnn_bias_grad(_p(dy), B * H * WIDTH, co, g + 4 * bo, s), "bias gradient")
            if layer > 0:
                _check(L.hnn_flip_weights(p16 + 2 * wo, co, ci, _p(self.wt[layer]), s), "flip")
                nxt = bufs["dy"][layer % 2]
                mask = acts[layer - 1] if self.relu else None
                _check(L.hnn_conv3x3_fwd(_p(dy), _p(self.wt[layer]), None, _p(mask), B, H, WIDTH, co, ci, d, 0,
                                         _p(nxt), None, s), "input gradient")
                dy = nxt

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.t += 1
        _check(lib().hnn_adam(_p(self.P), _p(self.G), _p(self.M), _p(self.V), self.nparam, float(lr), beta1, beta2,
                              eps, self.t, _p(self.P16), _stream()), "adam")

    def flops_per_node(self):
        """Multiply-adds x 2 of one forward pass per output node (padded channels included)."""
        return sum(2 * 9 * ci * co for (_, _, ci, co) in self.layout)


class SuperStepper:
    """K-step learned update of m-th order, N x N periodic dissipative problems
    (N = 128), with the Hermite solver as data generator, checker and fallback."""

    def __init__(self, K=16, m=3, N=WIDTH, lam=0.9, c=1.0, net=None, seed=0):
        import torch

        if N != WIDTH:
            raise ValueError(f"the network kernels handle {WIDTH} x {WIDTH} grids")
        self.K, self.m, self.N, self.c = int(K), int(m), int(N), float(c)
        self.h = 1.0 / N
        self.dt = lam * self.h / c
        self.problem = (2, self.m, self.N, self.c, self.h, self.dt, DISSIPATIVE, PERIODIC)
        self.Nu, self.Nv = (m + 1) ** 2, m * m
        self.C0 = self.Nu + self.Nv
        if self.C0 > CPAD:
            raise ValueError("m too large for 32 channels")
        self.vscale = self.h / self.c
        self.n = N * N
        self.net = net if net is not None else ConvNet(cin=self.C0, cout=self.C0, seed=seed)
        f64 = dict(dtype=torch.float64, device="cuda")
        self.shift = torch.zeros(self.C0, **f64)
        self.scale = torch.ones(self.C0, **f64)
        self.dscale = torch.ones(self.C0, **f64)
        self.wch = torch.zeros(CPAD, dtype=torch.float32, device="cuda")
        self.kappa = None
        self._fb = None

    # -- data -----------------------------------------------------------------
    def initial_u(self, traj):
        c, w, a = inputs.superstep_pulses(int(traj))
        return inputs.gaussian_data_2d(self.m, self.N, self.h, PERIODIC, PRIMAL, c, w, a)

    def _batch(self, B, precision=FP64):
        import torch

        b = HermiteBatch([self.problem] * B, precision=precision)
        b.set_stream(torch.cuda.current_stream())
        return b

    def load_initial(self, batch, trajs, U, V, pool=None):
        """Initial data of the given trajectories into the batch (one upload,
        one batched set; slots beyond len(trajs) repeat the first)."""
        import torch

        B = len(batch.problems)
        ids = [trajs[p] if p < len(trajs) else trajs[0] for p in range(B)]
        ics = list(pool.map(self.initial_u, ids)) if pool is not None else [self.initial_u(t) for t in ids]
        host = torch.from_numpy(np.stack(ics)).pin_memory()
        U.copy_(host, non_blocking=True)
        V.zero_()
        batch.set_states_device(U, V)

    def generate(self, trajs, nlev=5, chunk=256, precision=FP64, threads=4, log=None):
        """Trajectories (list of seeds) -> FP32 metric-space levels
        [nlev, len(trajs), N*N, C0]: level k of trajectory t at time k K dt."""
        import torch

        trajs = list(trajs)
        nt = len(trajs)
        levels = torch.empty((nlev, nt, self.n, self.C0), dtype=torch.float32, device="cuda")
        chunk = min(chunk, nt)
        batch = self._batch(chunk, precision)
        U, V = self._alloc_states(chunk)
        L, s = lib(), _stream()
        t0 = time.time()
        with ThreadPoolExecutor(threads) as pool:
            for c0 in range(0, nt, chunk):
                ids = trajs[c0:c0 + chunk]
                self.load_initial(batch, ids, U, V, pool)
                for k in range(nlev):
                    if k:
                        batch.step(self.K)
                    self.gather(batch, U, V)
                    _check(L.hnn_state_to_f32(_p(U), _p(V), len(ids) * self.n, self.Nu, self.Nv, self.vscale,
                                              _p(levels[k, c0]), self.C0, s), "state to f32")
                if log:
                    torch.cuda.synchronize()
                    log(f"generated {c0 + len(ids)}/{nt} trajectories ({time.time() - t0:.1f} s)")
        torch.cuda.synchronize()
        batch.close()
        return levels

    def fit_stats(self, levels, ntraj=256):
        """Per-channel mean and standard deviation of the levels (input
        standardisation) and of the K-step changes (output scaling); loss
        weights proportional to the squared change scale, so that the loss
        measures the metric-space error."""
        import torch

        L, s = lib(), _stream()
        nlev = levels.shape[0]
        nt = min(ntraj, levels.shape[1])
        mom = torch.zeros(2 * self.C0, dtype=torch.float64, device="cuda")
        dmom = torch.zeros(2 * self.C0, dtype=torch.float64, device="cuda")
        for k in range(nlev):
            _check(L.hnn_moments(_p(levels[k]), None, nt * self.n, self.C0, _p(mom), s), "moments")
            if k + 1 < nlev:
                _check(L.hnn_moments(_p(levels[k + 1]), _p(levels[k]), nt * self.n, self.C0, _p(dmom), s), "moments")
        m = mom.cpu().numpy()
        dm = dmom.cpu().numpy()
        cnt = nt * nlev * self.n
        dcnt = nt * (nlev - 1) * self.n
        mean = m[:self.C0] / cnt
        std = np.sqrt(np.maximum(m[self.C0:] / cnt - mean ** 2, 1e-300))
        dstd = np.sqrt(np.maximum(dm[self.C0:] / dcnt, 1e-300))
        self.set_stats(mean, std, dstd)

    def set_stats(self, shift, scale, dscale):
        import torch

        self.shift.copy_(torch.as_tensor(np.asarray(shift, dtype=np.float64)))
        self.scale.copy_(torch.as_tensor(np.asarray(scale, dtype=np.float64)))
        self.dscale.copy_(torch.as_tensor(np.asarray(dscale, dtype=np.float64)))
        d2 = np.asarray(dscale, dtype=np.float64) ** 2
        w = np.zeros(CPAD, dtype=np.float32)
        w[:self.C0] = d2 / d2.mean()
        self.wch.copy_(torch.as_tensor(w))

    # -- training ---------------------------------------------------------------
    def train(self, levels, iters, batch=32, lr=1e-3, lr_min=1e-5, seed=0, log_every=500, log=None):
        """Adam on the channel-weighted squared error of the standardised
        K-step change; pairs (level k, level k+1) drawn uniformly.  Returns
        the list of (iteration, mean loss since the previous report)."""
        import torch

        L, s = lib(), _stream()
        nlev, nt = levels.shape[0], levels.shape[1]
        rng = np.random.default_rng(seed)
        stride = self.n * self.C0
        tr = rng.integers(0, nt, size=(iters, batch))
        kk = rng.integers(0, nlev - 1, size=(iters, batch))
        src_all = torch.as_tensor((kk * nt + tr) * stride, dtype=torch.int64).cuda()
        dst_all = src_all + nt * stride
        x = torch.empty((batch, self.N, WIDTH, CPAD), dtype=torch.bfloat16, device="cuda")
        tgt = torch.empty((batch, self.N, WIDTH, CPAD), dtype=torch.float32, device="cuda")
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        bufs = self.net.buffers(batch, self.N)
        scale = 1.0 / (batch * self.n * self.C0)
        hist, last, t0 = [], 0.0, time.time()
        for it in range(iters):
            _check(L.hnn_make_pairs(_p(levels), _p(src_all[it]), _p(dst_all[it]), batch, self.n, self.C0,
                                    _p(self.shift), _p(self.scale), _p(self.dscale), CPAD, _p(x), _p(tgt), s), "pairs")
            out = self.net.forward(x, batch, self.N)
            _check(L.hnn_mse(_p(out), _p(tgt), _p(self.wch), batch * self.n, CPAD, scale, _p(loss),
                             _p(bufs["dyout"]), s), "loss")
            self.net.backward(x, batch, bufs["dyout"], self.N)
            frac = it / max(1, iters - 1)
            self.net.adam(lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * frac)))
            if (it + 1) % log_every == 0 or it + 1 == iters:
                tot = float(loss.item())
                n_since = log_every if (it + 1) % log_every == 0 else (it + 1) % log_every
                hist.append((it + 1, (tot - last) / n_since))
                last = tot
                if log:
                    log(f"iter {it + 1}: loss {hist[-1][1]:.4e} ({time.time() - t0:.1f} s)")
        return hist

    # -- inference ----------------------------------------------------------------
    def _alloc_states(self, B):
        import torch

        f64 = dict(dtype=torch.float64, device="cuda")
        return torch.empty((B, self.n, self.Nu), **f64), torch.empty((B, self.n, self.Nv), **f64)

    def gather(self, batch, U, V):
        """Primal states of every problem of the batch into U [B][n][Nu], V [B][n][Nv]."""
        batch.get_states_device(PRIMAL, U, V)

    def scatter(self, batch, U, V):
        batch.set_states_device(U, V)

    def predict(self, U, V, outU, outV):
        """outU/outV = network K-step prediction from the states U/V (FP64,
        device, [B][n][.]); one packing launch, the network, one unpacking launch."""
        import torch

        L, s = lib(), _stream()
        B = U.shape[0]
        if getattr(self, "_x", None) is None or self._x.shape[0] != B:
            self._x = torch.empty((B, self.N, WIDTH, CPAD), dtype=torch.bfloat16, device="cuda")
        _check(L.hnn_pack_state(_p(U), _p(V), B * self.n, self.Nu, self.Nv, self.vscale, _p(self.shift),
                                _p(self.scale), CPAD, _p(self._x), s), "pack")
        y = self.net.forward(self._x, B, self.N)
        _check(L.hnn_unpack_state(_p(U), _p(V), _p(y), B * self.n, self.Nu, self.Nv, self.vscale, _p(self.dscale),
                                  CPAD, _p(outU), _p(outV), s), "unpack")

    def _sqdiff(self, AU, AV, BU, BV):
        import torch

        out = torch.zeros((AU.shape[0], 2), dtype=torch.float64, device="cuda")
        _check(lib().hnn_sqdiff_batch(_p(AU), _p(AV), _p(BU), _p(BV), AU.shape[0], self.n, self.Nu, self.Nv,
                                      self.vscale, _p(out), _stream()), "sqdiff")
        return out

    def rel_errors(self, AU, AV, BU, BV):
        """Per-sample metric-space |A - B| / |B| (FP64 device reductions)."""
        o = self._sqdiff(AU, AV, BU, BV).cpu().numpy()
        return np.sqrt(o[:, 0] / np.maximum(o[:, 1], 1e-300))

    def residuals(self, batch, X, A, work):
        """Commutation residual |H(N(x)) - N(H(x))| / |N(x)| for every problem
        of batch (whose state is x = X on entry and H(N(x)) on exit)."""
        HXu, HXv, NHu, NHv = work
        batch.step(1)
        self.gather(batch, HXu, HXv)
        self.predict(HXu, HXv, NHu, NHv)
        self.scatter(batch, *A)
        batch.step(1)
        self.gather(batch, HXu, HXv)  # now H(N(x))
        d = self._sqdiff(HXu, HXv, NHu, NHv)
        na = self._sqdiff(A[0], A[1], A[0], A[1])
        o, a = d.cpu().numpy(), na.cpu().numpy()
        return np.sqrt(o[:, 0] / np.maximum(a[:, 1], 1e-300))

    def advance(self, batch, bar=1e-3, check=True, fallback=True):
        """Advance every problem of batch (all at the same time level) by
        K dt: the network's prediction where the calibrated residual estimate
        is within bar, else K plain Hermite steps.  Returns (accepted mask,
        estimated errors).  The contexts' clocks restart at 0."""
        import torch

        B = len(batch.problems)
        X = self._alloc_states(B)
        A = self._alloc_states(B)
        self.gather(batch, *X)
        self.predict(X[0], X[1], A[0], A[1])
        if not check:
            self.scatter(batch, *A)
            return np.ones(B, dtype=bool), np.zeros(B)
        if self.kappa is None:
            raise RuntimeError("calibrate() first")
        work = self._alloc_states(B) + self._alloc_states(B)
        r = self.residuals(batch, X, A, work)
        est = self.kappa * r
        acc = est <= bar
        rej = np.flatnonzero(~acc)
        if len(rej) and fallback:
            L, s = lib(), _stream()
            fb = self.fallback_batch(len(rej), batch.precision)
            idx = torch.as_tensor(rej, dtype=torch.int64).cuda()
            Fu, Fv = work[0][:len(rej)], work[1][:len(rej)]
            bu, bv = self.n * self.Nu, self.n * self.Nv
            _check(L.hnn_copy_blocks(_p(X[0]), _p(idx), _p(Fu), None, len(rej), bu, s), "copy")
            _check(L.hnn_copy_blocks(_p(X[1]), _p(idx), _p(Fv), None, len(rej), bv, s), "copy")
            fb.set_states_device(Fu, Fv)
            fb.step(self.K)
            fb.get_states_device(PRIMAL, Fu, Fv)
            _check(L.hnn_copy_blocks(_p(Fu), None, _p(A[0]), _p(idx), len(rej), bu, s), "copy")
            _check(L.hnn_copy_blocks(_p(Fv), None, _p(A[1]), _p(idx), len(rej), bv, s), "copy")
        self.scatter(batch, *A)
        return acc, est

    def fallback_batch(self, n, precision=FP64):
        """A batch of n problems for the rejected predictions, in the
        arithmetic of the caller's batch (kept for the next call)."""
        if self._fb is None or len(self._fb.problems) != n or self._fb.precision != precision:
            if self._fb is not None:
                self._fb.close()
            self._fb = self._batch(n, precision)
        return self._fb

    def evaluate(self, trajs, chunk=256):
        """True K-step error and residual of the network on fresh initial
        data: returns (true rel. errors, residuals) per trajectory."""
        trajs = list(trajs)
        errs, ress = [], []
        B = min(chunk, len(trajs))
        batch = self._batch(B)
        X, A, T = self._alloc_states(B), self._alloc_states(B), self._alloc_states(B)
        work = self._alloc_states(B) + self._alloc_states(B)
        with ThreadPoolExecutor(4) as pool:
            for c0 in range(0, len(trajs), B):
                ids = trajs[c0:c0 + B]
                self.load_initial(batch, ids, X[0], X[1], pool)
                self.predict(X[0], X[1], A[0], A[1])
                batch.step(self.K)
                self.gather(batch, *T)
                e = self.rel_errors(A[0], A[1], T[0], T[1])
                self.scatter(batch, *X)
                r = self.residuals(batch, X, A, work)
                errs.append(e[:len(ids)])
                ress.append(r[:len(ids)])
        batch.close()
        return np.concatenate(errs), np.concatenate(ress)

    def calibrate(self, trajs, quantile=1.0):
        """kappa = the given quantile (default: the maximum) of true error /
        residual over held-out trajectories."""
        e, r = self.evaluate(trajs)
        self.kappa = float(np.quantile(e / np.maximum(r, 1e-300), quantile))
        return e, r

    # -- persistence ------------------------------------------------------------------
    def save(self, path):
        np.savez(path, params=self.net.get_params(), shift=self.shift.cpu().numpy(), scale=self.scale.cpu().numpy(),
                 dscale=self.dscale.cpu().numpy(), kappa=np.array(np.nan if self.kappa is None else self.kappa),
                 meta=np.array([self.K, self.m, self.N, self.dt / self.h * self.c, self.c]),
                 dils=np.array(self.net.dils), act=np.array(self.net.act))

    @classmethod
    def load(cls, path):
        z = np.load(path)
        K, m, N, lam, c = z["meta"]
        act = str(z["act"]) if "act" in z.files else "relu"
        net = ConvNet(cin=int((m + 1) ** 2 + m * m), cout=int((m + 1) ** 2 + m * m),
                      dilations=tuple(int(d) for d in z["dils"]), act=act)
        st = cls(K=int(K), m=int(m), N=int(N), lam=float(lam), c=float(c), net=net)
        net.set_params(z["params"])
        st.set_stats(z["shift"], z["scale"], z["dscale"])
        k = float(z["kappa"])
        st.kappa = None if math.isnan(k) else k
        return st


def recalibrate(path, quantile, ncal, log=print):
    """Re-calibrate a trained super-stepper: kappa = the given quantile of
    true error / residual over ncal held-out trajectories (seeds 10^6 ..),
    checked on ncal further held-out trajectories (seeds 2 * 10^6 ..) at the
    bars 1e-3 .. 1e-1; the new kappa is written back to `path`.  Returns the
    verification table."""
    st = SuperStepper.load(path)
    e, r = st.calibrate(range(10 ** 6, 10 ** 6 + ncal), quantile=quantile)
    log(f"calibration set ({ncal}): error/residual median {np.median(e / r):.3f}, "
        f"{quantile:.3f} quantile {st.kappa:.3f}, max {np.max(e / r):.3f}")
    e2, r2 = st.evaluate(range(2 * 10 ** 6, 2 * 10 ** 6 + ncal))
    est = st.kappa * r2
    table = {}
    for bar in (1e-3, 3e-3, 1e-2, 3e-2, 1e-1):
        acc = est <= bar
        table[bar] = {"accepted": float(acc.mean()), "true_error_within": float(np.mean(e2 <= bar)),
                      "false_accepts": int(np.sum(acc & (e2 > bar)))}
        log(f"  verification bar {bar:.0e}: {table[bar]}")
    st.save(path)
    return table


def main(argv=None):
    ap = argparse.ArgumentParser(description="Train the learned super-stepper on solver trajectories")
    ap.add_argument("--recalibrate", default=None, help="only re-calibrate kappa of these trained weights")
    ap.add_argument("--quantile", type=float, default=0.99, help="kappa quantile of true error / residual")
    ap.add_argument("--ntraj", type=int, default=10000)
    ap.add_argument("--nlev", type=int, default=5)
    ap.add_argument("--iters", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--act", default="relu", help="comma-separated activations to train, each on the same data")
    ap.add_argument("--calib", type=int, default=256, help="held-out trajectories for the residual calibration")
    ap.add_argument("--out", default=None, help="output path; with several activations, {act} is replaced")
    a = ap.parse_args(argv)
    import torch

    if a.recalibrate:
        recalibrate(a.recalibrate, a.quantile, a.calib)
        return
    if not a.out:
        ap.error("--out is required for training")

    log = lambda s: print(s, flush=True)
    gen = SuperStepper()
    t0 = time.time()
    levels = gen.generate(range(a.ntraj), nlev=a.nlev, log=log)
    log(f"data: {a.ntraj} trajectories x {a.nlev} levels in {time.time() - t0:.1f} s")
    gen.fit_stats(levels)
    for act in a.act.split(","):
        st = SuperStepper(net=ConvNet(act=act))
        st.set_stats(gen.shift.cpu().numpy(), gen.scale.cpu().numpy(), gen.dscale.cpu().numpy())
        torch.cuda.synchronize()
        t0 = time.time()
        st.train(levels, a.iters, batch=a.batch, lr=a.lr, log_every=max(1, a.iters // 40), log=log)
        torch.cuda.synchronize()
        log(f"[{act}] training: {a.iters} iterations in {time.time() - t0:.1f} s")
        e, r = st.calibrate(range(10 ** 6, 10 ** 6 + a.calib), quantile=a.quantile)
        log(f"[{act}] calibration set: true error median {np.median(e):.3e}, max {e.max():.3e}; "
            f"error/residual median {np.median(e / r):.3f}, kappa ({a.quantile} quantile) {st.kappa:.3f}")
        out = a.out.replace("{act}", act)
        st.save(out)
        log(f"[{act}] saved {out}")
        e2, r2 = st.evaluate(range(2 * 10 ** 6, 2 * 10 ** 6 + a.calib))
        est = st.kappa * r2
        log(f"[{act}] test set: true error quantiles (10, 50, 90, 100 %) {np.quantile(e2, [0.1, 0.5, 0.9, 1.0])}")
        for bar in (1e-3, 3e-3, 1e-2, 3e-2, 1e-1):
            acc = est <= bar
            log(f"  bar {bar:.0e}: accepted {acc.mean():.3f}, true error <= bar {np.mean(e2 <= bar):.3f}, "
                f"accepted with true error > bar {np.sum(acc & (e2 > bar))}")


if __name__ == "__main__":
    main()
