"""Hermite-method ORACLE (test infrastructure only).

A plain FP64 CPU implementation of the dissipative and conservative Hermite
half-steps, written from the paper (Appelo, Hagstrom, Vargas, "Hermite Methods
for the Scalar Wave Equation"): Sec. 2.2 interpolation by the confluent
Vandermonde system of Eq. (Hermcon), Sec. 3.1/3.3 Taylor recursions, Sec. 4
conservative update, Sec. 3.1.3 ghost polynomials, Sec. 3.2/3.3/4.2 energies.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and never imports it.

Arrays follow the host layout ``[node][coef]`` (nodes in C order, axis 0
slowest; coefficient multi-index in C order), with the paper's scaled
derivatives h^|k|/k! d^k u and h^|k|/k! d^k v.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hermite_oracle.c")
_HDR = os.path.join(_HERE, "hermite_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

DISSIPATIVE, CONSERVATIVE, DISSIPATIVE_SIMPLE = 0, 1, 2
PERIODIC, DIRICHLET, NEUMANN = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no FMA contraction)."""
    stale = not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(_HDR)
    )
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fPIC",
             "-shared", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int), ("m", ctypes.c_int), ("variant", ctypes.c_int), ("bc", ctypes.c_int),
        ("N", ctypes.c_int64), ("c", ctypes.c_double), ("h", ctypes.c_double), ("dt", ctypes.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_Problem)
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        ip = ctypes.POINTER(ctypes.c_int)
        sig = {
            "or_npts": (ctypes.c_int64, [P, ctypes.c_int]),
            "or_nnodes": (ctypes.c_int64, [P, ctypes.c_int]),
            "or_interp1d": (ctypes.c_int, [ctypes.c_int, dp, dp, dp]),
            "or_interp": (ctypes.c_int, [ctypes.c_int, ip, dp, dp]),
            "or_diss_cell": (ctypes.c_int, [P, dp, dp, dp, dp]),
            "or_cons_cell": (ctypes.c_int, [P, dp, dp, dp]),
            "or_cons_start_cell": (ctypes.c_int, [P, dp, dp, dp]),
            "or_half_step": (ctypes.c_int, [P, ctypes.c_int, dp, dp, dp, dp]),
            "or_half_step_sample": (ctypes.c_int, [P, ctypes.c_int, dp, dp, i64p, ctypes.c_int64, dp, dp, dp]),
            "or_cons_start": (ctypes.c_int, [P, dp, dp, dp]),
            "or_diss_energy": (ctypes.c_int, [P, ctypes.c_int, dp, dp, dp]),
            "or_cons_forms": (ctypes.c_int, [P, ctypes.c_int, dp, dp, dp]),
            "or_gauss_points": (ctypes.c_int, [ctypes.c_int, dp, dp]),
            "or_l2_error": (ctypes.c_int, [P, ctypes.c_int, dp, ctypes.c_int, dp, dp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def interp1d(q, left, right):
    a = np.zeros(2 * q + 2)
    _check(lib().or_interp1d(q, _p(_f64(left)), _p(_f64(right)), _p(a)), "interp1d")
    return a


def interp(q, corner):
    """Tensor interpolation on one cell. q: per-axis data degrees; corner [2^d][prod(q+1)]."""
    q = list(q)
    d = len(q)
    out = np.zeros(int(np.prod([2 * x + 2 for x in q])))
    qa = (ctypes.c_int * d)(*q)
    c = _f64(corner)
    _check(lib().or_interp(d, qa, _p(c), _p(out)), "interp")
    return out.reshape([2 * x + 2 for x in q])


class Problem:
    """One wave problem: dimension d, order m, N cells per axis, speed c,
    spacing h, time step dt, variant and boundary condition."""

    def __init__(self, d, m, N, c, h, dt, variant=DISSIPATIVE, bc=PERIODIC):
        self.d, self.m, self.N = int(d), int(m), int(N)
        self.c, self.h, self.dt = float(c), float(h), float(dt)
        self.variant, self.bc = int(variant), int(bc)
        self._s = _Problem(self.d, self.m, self.variant, self.bc, self.N, self.c, self.h, self.dt)
        self.Nu = (self.m + 1) ** self.d
        self.Nv = self.m ** self.d

    @property
    def ptr(self):
        return ctypes.byref(self._s)

    def npts(self, g):
        return int(lib().or_npts(self.ptr, g))

    def nnodes(self, g):
        return int(lib().or_nnodes(self.ptr, g))

    # single cells -------------------------------------------------------
    def diss_cell(self, cu, cv):
        nu, nv = np.zeros(self.Nu), np.zeros(self.Nv)
        _check(lib().or_diss_cell(self.ptr, _p(_f64(cu)), _p(_f64(cv)), _p(nu), _p(nv)), "diss_cell")
        return nu, nv

    def cons_cell(self, cu, old):
        out = np.zeros(self.Nu)
        _check(lib().or_cons_cell(self.ptr, _p(_f64(cu)), _p(_f64(old)), _p(out)), "cons_cell")
        return out

    def cons_start_cell(self, cu, cv=None):
        out = np.zeros(self.Nu)
        cvp = _f64(cv) if cv is not None else None
        _check(lib().or_cons_start_cell(self.ptr, _p(_f64(cu)), _p(cvp), _p(out)), "cons_start_cell")
        return out

    # grids --------------------------------------------------------------
    def half_step(self, dst, src_u, src_v=None, dst_u=None, dst_v=None):
        """Dissipative: returns (u, v) on grid dst.  Conservative: dst_u holds the
        earlier level on grid dst; returns the updated copy."""
        nd = self.nnodes(dst)
        su = _f64(src_u)
        if self.variant == CONSERVATIVE:
            out = _f64(dst_u).copy()
            _check(lib().or_half_step(self.ptr, dst, _p(su), None, _p(out), None), "half_step")
            return out
        sv = _f64(src_v)
        ou, ov = np.zeros((nd, self.Nu)), np.zeros((nd, self.Nv))
        _check(lib().or_half_step(self.ptr, dst, _p(su), _p(sv), _p(ou), _p(ov)), "half_step")
        return ou, ov

    def half_step_sample(self, dst, src_u, src_v, targets, old_u=None):
        t = np.ascontiguousarray(targets, dtype=np.int64)
        nt = t.size
        ou, ov = np.zeros((nt, self.Nu)), np.zeros((nt, max(self.Nv, 1)))
        sv = _f64(src_v) if src_v is not None else None
        old = _f64(old_u) if old_u is not None else None
        _check(
            lib().or_half_step_sample(
                self.ptr, dst, _p(_f64(src_u)), _p(sv), t.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                nt, _p(old), _p(ou), _p(ov),
            ),
            "half_step_sample",
        )
        if self.variant == CONSERVATIVE:
            return ou
        return ou, ov[:, : self.Nv]

    def cons_start(self, u0, v0=None):
        out = np.zeros((self.nnodes(1), self.Nu))
        v = _f64(v0) if v0 is not None else None
        _check(lib().or_cons_start(self.ptr, _p(_f64(u0)), _p(v), _p(out)), "cons_start")
        return out

    def run(self, u, v=None, nsteps=1, dual_u=None):
        """Full steps (two half-steps each).  Dissipative: primal -> dual -> primal.
        Conservative: state is (primal level t, dual level t+dt/2); each full step
        updates the primal then the dual grid.  Returns the new state."""
        if self.variant == CONSERVATIVE:
            p, q = _f64(u).copy(), _f64(dual_u).copy()
            for _ in range(nsteps):
                p = self.half_step(0, q, dst_u=p)
                q = self.half_step(1, p, dst_u=q)
            return p, q
        pu, pv = _f64(u), _f64(v)
        for _ in range(nsteps):
            du, dv = self.half_step(1, pu, pv)
            pu, pv = self.half_step(0, du, dv)
        return pu, pv

    # diagnostics ---------------------------------------------------------
    def diss_energy(self, g, u, v):
        out = np.zeros(2)
        _check(lib().or_diss_energy(self.ptr, g, _p(_f64(u)), _p(_f64(v)), _p(out)), "diss_energy")
        return out

    def cons_forms(self, g, ua, ub):
        out = np.zeros(2)
        _check(lib().or_cons_forms(self.ptr, g, _p(_f64(ua)), _p(_f64(ub)), _p(out)), "cons_forms")
        return out

    def cons_G(self, p_int, q_half):
        """Conserved quantity of the conservative scheme with primal level p^n and
        dual level p^{n+1/2}: G = |p^{n+1/2}|^2 - <p^{n+1}, p^n> (seminorm
        |.|_{m+1,..,m+1}), the tentative p^{n+1} computed here."""
        p_next = self.half_step(0, q_half, dst_u=p_int)
        a = self.cons_forms(1, q_half, q_half)[0]
        b = self.cons_forms(0, p_next, p_int)[0]
        return a - b

    def gauss(self, n):
        x, w = np.zeros(n), np.zeros(n)
        _check(lib().or_gauss_points(n, _p(x), _p(w)), "gauss")
        return x, w

    def l2_error(self, g, u, nq, exact_fn):
        """L2 error of the I_m interpolant of grid-g data vs exact_fn(points[..., d])."""
        x, _ = self.gauss(nq)
        nt = self.npts(1 - g)
        centres = (np.arange(nt) + (0.0 if g == 1 else 0.5)) * self.h
        grids = np.meshgrid(*([centres] * self.d), indexing="ij")
        cc = np.stack([gg.reshape(-1) for gg in grids], -1)  # [cells, d]
        qg = np.meshgrid(*([x * self.h] * self.d), indexing="ij")
        qq = np.stack([gg.reshape(-1) for gg in qg], -1)  # [nq^d, d]
        pts = cc[:, None, :] + qq[None, :, :]
        ex = _f64(exact_fn(pts))
        err2 = ctypes.c_double(0.0)
        _check(lib().or_l2_error(self.ptr, g, _p(_f64(u)), nq, _p(ex), ctypes.byref(err2)), "l2_error")
        return float(np.sqrt(err2.value))
