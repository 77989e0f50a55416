"""Python binding of the B300 Hermite wave-equation library (libhermite_b300.so).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  The names mirror the C ABI in ``include/hermite.h``.  Importing
this package does not need a GPU; creating a context does.  If the shared
library is missing the import of :func:`lib` raises -- there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhermite_b300.so")

DISSIPATIVE, CONSERVATIVE, DISSIPATIVE_SIMPLE = 0, 1, 2
PERIODIC, DIRICHLET, NEUMANN = 0, 1, 2
PRIMAL, DUAL = 0, 1
FP64, SPLIT32 = 0, 1

ERRORS = {
    -1: "HERMITE_ERR_ARG", -2: "HERMITE_ERR_ALLOC", -3: "HERMITE_ERR_CUDA", -4: "HERMITE_ERR_NONFINITE",
    -5: "HERMITE_ERR_TIMEOUT", -6: "HERMITE_ERR_STATE", -7: "HERMITE_ERR_UNSUPPORTED",
}

# every symbol declared in include/hermite.h
EXPORTS = [
    "hermite_create", "hermite_destroy", "hermite_set_stream", "hermite_set_state", "hermite_set_state_device",
    "hermite_set_state2", "hermite_step", "hermite_advance_half", "hermite_half_steps", "hermite_time",
    "hermite_get_state", "hermite_get_grid", "hermite_set_grid", "hermite_get_grid_device", "hermite_energy",
    "hermite_nodes", "hermite_ncoef", "hermite_operator", "hermite_last_error", "hermite_energy_noalloc", "hermite_peak_probe",
    "hermite_l2_error", "hermite_tc_selftest", "hermite_set_split_engine", "hermite_get_split_engine",
    "hermite_create_ex", "hermite_batch_create", "hermite_batch_destroy", "hermite_batch_problem",
    "hermite_batch_set_stream", "hermite_batch_step", "hermite_batch_dof_per_step", "hermite_batch_autotune",
    "hermite_batch_config", "hermite_batch_last_error", "hermite_batch_get_states_device",
    "hermite_batch_set_states_device",
    # include/hermite_nn.h
    "hnn_conv3x3_fwd", "hnn_flip_weights", "hnn_conv3x3_wgrad", "hnn_bias_grad", "hnn_mse", "hnn_adam",
    "hnn_state_to_f32", "hnn_pack_state", "hnn_unpack_state", "hnn_make_pairs", "hnn_moments", "hnn_sqdiff",
    "hnn_set_conv_engine", "hnn_conv_status", "hnn_tc_gemm_selftest", "hnn_sqdiff_batch", "hnn_copy_blocks",
    "hnn_wait_selftest", "hermite_debug_fail_alloc",
]


class HermiteError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} not found: build it with `python -m paper_1802_05246_b300.build`")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, i64, c_int, c_dbl = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_int, ctypes.c_double
    ip = ctypes.POINTER(ctypes.c_int)
    sig = {
        "hermite_create": (c_int, [c_int, c_int, i64, c_dbl, c_dbl, c_dbl, c_int, c_int, ctypes.POINTER(vp)]),
        "hermite_destroy": (None, [vp]),
        "hermite_set_stream": (c_int, [vp, vp]),
        "hermite_set_state": (c_int, [vp, vp, vp]),
        "hermite_set_state_device": (c_int, [vp, vp, vp]),
        "hermite_set_state2": (c_int, [vp, vp, vp]),
        "hermite_step": (c_int, [vp, i64]),
        "hermite_advance_half": (c_int, [vp, i64]),
        "hermite_half_steps": (i64, [vp]),
        "hermite_time": (c_dbl, [vp]),
        "hermite_get_state": (c_int, [vp, vp, vp]),
        "hermite_get_grid": (c_int, [vp, c_int, vp, vp]),
        "hermite_set_grid": (c_int, [vp, c_int, vp, vp]),
        "hermite_get_grid_device": (c_int, [vp, c_int, vp, vp]),
        "hermite_energy": (c_int, [vp, dp]),
        "hermite_nodes": (i64, [vp, c_int]),
        "hermite_ncoef": (c_int, [vp, ip, ip]),
        "hermite_operator": (c_int, [vp, c_int, vp, ip, ip]),
        "hermite_last_error": (ctypes.c_char_p, [vp]),
        "hermite_energy_noalloc": (c_int, [vp, c_int, vp, i64, vp]),
        "hermite_peak_probe": (c_int, [c_int, ctypes.POINTER(c_dbl)]),
        "hermite_l2_error": (c_int, [vp, c_int, i64, vp, c_int, dp, dp, vp, dp]),
        "hermite_tc_selftest": (c_int, [c_int, c_int, vp, vp, vp, vp]),
        "hermite_set_split_engine": (c_int, [vp, c_int]),
        "hermite_get_split_engine": (c_int, [vp]),
        "hermite_create_ex": (c_int, [c_int, c_int, i64, c_dbl, c_dbl, c_dbl, c_int, c_int, c_int, ctypes.POINTER(vp)]),
        "hermite_batch_create": (c_int, [c_int, vp, vp, vp, vp, vp, vp, vp, vp, c_int, ctypes.POINTER(vp)]),
        "hermite_batch_destroy": (None, [vp]),
        "hermite_batch_problem": (vp, [vp, c_int]),
        "hermite_batch_set_stream": (c_int, [vp, vp]),
        "hermite_batch_step": (c_int, [vp, i64]),
        "hermite_batch_dof_per_step": (i64, [vp]),
        "hermite_batch_autotune": (c_int, [vp, ip, ip, dp]),
        "hermite_batch_config": (c_int, [vp, c_int, c_int]),
        "hermite_batch_last_error": (ctypes.c_char_p, [vp]),
        "hermite_batch_get_states_device": (c_int, [vp, c_int, vp, vp]),
        "hermite_batch_set_states_device": (c_int, [vp, vp, vp]),
        "hnn_conv3x3_fwd": (c_int, [vp, vp, vp, vp, c_int, c_int, c_int, c_int, c_int, c_int, c_int, vp, vp, vp]),
        "hnn_flip_weights": (c_int, [vp, c_int, c_int, vp, vp]),
        "hnn_conv3x3_wgrad": (c_int, [vp, vp, c_int, c_int, c_int, c_int, c_int, c_int, vp, vp]),
        "hnn_bias_grad": (c_int, [vp, i64, c_int, vp, vp]),
        "hnn_mse": (c_int, [vp, vp, vp, i64, c_int, ctypes.c_float, vp, vp, vp]),
        "hnn_adam": (c_int, [vp, vp, vp, vp, i64, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                             c_int, vp, vp]),
        "hnn_state_to_f32": (c_int, [vp, vp, i64, c_int, c_int, c_dbl, vp, c_int, vp]),
        "hnn_pack_state": (c_int, [vp, vp, i64, c_int, c_int, c_dbl, vp, vp, c_int, vp, vp]),
        "hnn_unpack_state": (c_int, [vp, vp, vp, i64, c_int, c_int, c_dbl, vp, c_int, vp, vp, vp]),
        "hnn_make_pairs": (c_int, [vp, vp, vp, c_int, i64, c_int, vp, vp, vp, c_int, vp, vp, vp]),
        "hnn_moments": (c_int, [vp, vp, i64, c_int, vp, vp]),
        "hnn_sqdiff": (c_int, [vp, vp, vp, vp, i64, c_int, c_int, c_dbl, vp, vp]),
        "hnn_set_conv_engine": (c_int, [c_int]),
        "hnn_conv_status": (c_int, []),
        "hnn_tc_gemm_selftest": (c_int, [vp, vp, vp, c_int, vp, vp]),
        "hnn_sqdiff_batch": (c_int, [vp, vp, vp, vp, c_int, i64, c_int, c_int, c_dbl, vp, vp]),
        "hnn_copy_blocks": (c_int, [vp, vp, vp, vp, c_int, i64, vp]),
        "hnn_wait_selftest": (c_int, [vp]),
        "hermite_debug_fail_alloc": (c_int, [c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(a):
    """Data pointer of a C-contiguous float64 numpy array or torch tensor (or None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("expected a C-contiguous float64 array")
        return a.ctypes.data
    # torch tensor (host or device)
    if str(a.dtype) != "torch.float64" or not a.is_contiguous():
        raise ValueError("expected a contiguous float64 tensor")
    return a.data_ptr()


class Hermite:
    """One problem on the current CUDA device (see ``hermite_create``)."""

    def __init__(self, d, m, N, c, h, dt, variant=DISSIPATIVE, bc=PERIODIC, precision=FP64):
        L = lib()
        h_ = ctypes.c_void_p()
        rc = L.hermite_create_ex(int(d), int(m), int(N), float(c), float(h), float(dt), int(variant), int(bc),
                                 int(precision), ctypes.byref(h_))
        if rc != 0:
            raise HermiteError(rc, L.hermite_last_error(None).decode())
        self._h = h_
        self.d, self.m, self.N, self.c, self.h, self.dt = int(d), int(m), int(N), float(c), float(h), float(dt)
        self.variant, self.bc, self.precision = int(variant), int(bc), int(precision)
        nu, nv = ctypes.c_int(), ctypes.c_int()
        L.hermite_ncoef(self._h, ctypes.byref(nu), ctypes.byref(nv))
        self.Nu, self.Nv = nu.value, nv.value

    def _check(self, rc):
        if rc != 0:
            raise HermiteError(rc, lib().hermite_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            if getattr(self, "_owned", True):
                lib().hermite_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def nodes(self, grid):
        return int(lib().hermite_nodes(self._h, grid))

    @property
    def half_steps(self):
        return int(lib().hermite_half_steps(self._h))

    @property
    def time(self):
        return float(lib().hermite_time(self._h))

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
        raw = getattr(stream, "cuda_stream", stream)
        self._check(lib().hermite_set_stream(self._h, raw))

    def set_state(self, u, v=None):
        self._check(lib().hermite_set_state(self._h, _ptr(u), _ptr(v)))

    def set_state_device(self, u, v=None):
        self._check(lib().hermite_set_state_device(self._h, _ptr(u), _ptr(v)))

    def set_state2(self, u_primal, u_dual):
        self._check(lib().hermite_set_state2(self._h, _ptr(u_primal), _ptr(u_dual)))

    def step(self, n=1):
        self._check(lib().hermite_step(self._h, int(n)))

    def advance_half(self, n=1):
        self._check(lib().hermite_advance_half(self._h, int(n)))

    def _alloc(self, grid):
        n = self.nodes(grid)
        return np.empty((n, self.Nu)), (np.empty((n, self.Nv)) if self.variant != CONSERVATIVE else None)

    def get_state(self, out_u=None, out_v=None):
        u, v = (out_u, out_v) if out_u is not None else self._alloc(PRIMAL)
        self._check(lib().hermite_get_state(self._h, _ptr(u), _ptr(v)))
        return u, v

    def get_grid(self, grid):
        u, v = self._alloc(grid)
        self._check(lib().hermite_get_grid(self._h, grid, _ptr(u), _ptr(v)))
        return u, v

    def get_grid_device(self, grid, u, v=None):
        self._check(lib().hermite_get_grid_device(self._h, grid, _ptr(u), _ptr(v)))

    def set_grid(self, grid, u, v=None):
        self._check(lib().hermite_set_grid(self._h, grid, _ptr(u), _ptr(v)))

    def energy(self):
        out = (ctypes.c_double * 3)()
        self._check(lib().hermite_energy(self._h, out))
        return np.array(out[:])

    def energy_noalloc(self, grid, level, ld, out):
        """Allocation-free energy of a device level (see hermite_energy_noalloc);
        level: coefficient-major float64 device tensor, out: 2-element device tensor."""
        self._check(lib().hermite_energy_noalloc(self._h, int(grid), _ptr(level), int(ld), _ptr(out)))

    @property
    def split_engine(self):
        """Half-step engine of a split context: 0 CUDA cores, 1 tensor cores (-1: FP64)."""
        return int(lib().hermite_get_split_engine(self._h))

    def set_split_engine(self, engine):
        self._check(lib().hermite_set_split_engine(self._h, int(engine)))

    def l2_error(self, grid, xq, wq, exact, cells=None):
        """(sum of (I_m u - exact)^2, sum of exact^2) over cells by quadrature
        (see hermite_l2_error).  xq, wq: 1-D points on [-1/2, 1/2] and weights
        summing to 1; exact: float64 device tensor [ncells, nq^d]; cells: int64
        device tensor of cell indices, or None for every cell."""
        xq = np.ascontiguousarray(xq, dtype=np.float64)
        wq = np.ascontiguousarray(wq, dtype=np.float64)
        out = (ctypes.c_double * 2)()
        ncells = int(exact.shape[0])
        if str(exact.dtype) != "torch.float64" or int(exact.numel()) != ncells * int(xq.size) ** self.d:
            raise ValueError("exact: float64 device tensor [ncells, nq^d]")
        if cells is not None:
            if str(cells.dtype) != "torch.int64" or not cells.is_contiguous() or int(cells.numel()) != ncells:
                raise ValueError("cells: a contiguous int64 device tensor with one entry per row of exact")
        cptr = None if cells is None else cells.data_ptr()
        self._check(lib().hermite_l2_error(self._h, int(grid), ncells, cptr, int(xq.size),
                                           xq.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           wq.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(exact), out))
        return out[0], out[1]

    def operator(self, which=0):
        r, c = ctypes.c_int(), ctypes.c_int()
        self._check(lib().hermite_operator(self._h, which, None, ctypes.byref(r), ctypes.byref(c)))
        M = np.empty((r.value, c.value))
        self._check(lib().hermite_operator(self._h, which, _ptr(M), ctypes.byref(r), ctypes.byref(c)))
        return M


def _borrow(handle, d, m, N, c, h, dt, variant, bc, precision):
    """A non-owning Hermite view of a context that belongs to a batch."""
    g = Hermite.__new__(Hermite)
    g._h = ctypes.c_void_p(handle)
    g._owned = False
    g.d, g.m, g.N, g.c, g.h, g.dt = int(d), int(m), int(N), float(c), float(h), float(dt)
    g.variant, g.bc, g.precision = int(variant), int(bc), int(precision)
    nu, nv = ctypes.c_int(), ctypes.c_int()
    lib().hermite_ncoef(g._h, ctypes.byref(nu), ctypes.byref(nv))
    g.Nu, g.Nv = nu.value, nv.value
    return g


def peak_probe(kind):
    """Measured FMA throughput (flop/s, an FMA = 2) of the current device:
    kind 0 FP64, 1 FP32, 2 FP32 packed pairs (see hermite_peak_probe)."""
    out = ctypes.c_double()
    rc = lib().hermite_peak_probe(int(kind), ctypes.byref(out))
    if rc != 0:
        raise HermiteError(rc, "hermite_peak_probe failed")
    return out.value


class HermiteBatch:
    """Ragged batch of problems advanced together (see hermite_batch_create).

    problems: sequence of (d, m, N, c, h, dt, variant, bc) tuples, one d for all."""

    def __init__(self, problems, precision=FP64):
        L = lib()
        probs = [tuple(p) for p in problems]
        n = len(probs)
        cols = list(zip(*probs))
        arr = lambda typ, xs: (typ * n)(*xs)
        self._b = ctypes.c_void_p()
        rc = L.hermite_batch_create(n, arr(ctypes.c_int, cols[0]), arr(ctypes.c_int, cols[1]),
                                    arr(ctypes.c_int64, cols[2]), arr(ctypes.c_double, cols[3]),
                                    arr(ctypes.c_double, cols[4]), arr(ctypes.c_double, cols[5]),
                                    arr(ctypes.c_int, cols[6]), arr(ctypes.c_int, cols[7]), int(precision),
                                    ctypes.byref(self._b))
        if rc != 0:
            raise HermiteError(rc, L.hermite_batch_last_error(None).decode())
        self.precision = int(precision)
        self.problems = [_borrow(L.hermite_batch_problem(self._b, i), *probs[i], precision) for i in range(n)]

    def _check(self, rc):
        if rc != 0:
            raise HermiteError(rc, lib().hermite_batch_last_error(self._b).decode())

    def problem(self, p):
        return self.problems[p]

    def set_stream(self, stream):
        raw = getattr(stream, "cuda_stream", stream)
        self._check(lib().hermite_batch_set_stream(self._b, raw))

    def step(self, n=1):
        self._check(lib().hermite_batch_step(self._b, int(n)))

    @property
    def dof_per_step(self):
        return int(lib().hermite_batch_dof_per_step(self._b))

    def autotune(self):
        a, b, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        self._check(lib().hermite_batch_autotune(self._b, ctypes.byref(a), ctypes.byref(b), ctypes.byref(ms)))
        return a.value, b.value, ms.value

    def config(self, item_nodes, blocks_per_sm):
        self._check(lib().hermite_batch_config(self._b, int(item_nodes), int(blocks_per_sm)))

    def get_states_device(self, grid, u, v=None):
        """All problems' levels on `grid` into device buffers, back to back."""
        self._check(lib().hermite_batch_get_states_device(self._b, int(grid), _ptr(u), _ptr(v)))

    def set_states_device(self, u, v=None):
        """All (dissipative) problems' states from device buffers, back to back."""
        self._check(lib().hermite_batch_set_states_device(self._b, _ptr(u), _ptr(v)))

    def close(self):
        if getattr(self, "_b", None):
            lib().hermite_batch_destroy(self._b)
            self._b = None
            self.problems = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
