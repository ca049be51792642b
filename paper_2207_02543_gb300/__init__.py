"""GB300-native POD-2G-preconditioned conjugate gradients (arXiv 2207.02543, Algorithm 3).

Thin Python binding of the C ABI declared in include/pod2g.h: argument marshalling
only. Every step of the solve runs in the CUDA library libpod2g.so built in this
directory (see build.py); there is no CPU fallback, and importing the binding
without the built library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpod2g.so")

OK, NOT_CONVERGED, BREAKDOWN, NOT_SPD, INVALID_ARG, ADMISSION, OOM, CUDA_ERROR, TIMEOUT, NONFINITE, PENDING = range(11)
FP64, MIXED_FP32PHI, MIXED_BF16PHI = 0, 1, 2
PCG, STATIONARY = 0, 1  # solution methods: Algorithm 3, or the two-grid cycle of Algorithm 2 iterated
SMOOTHER_JACOBI, SMOOTHER_SGS = 0, 1  # relaxation: damped Jacobi, or multicolour symmetric Gauss-Seidel

EXPORTS = [
    "pod2g_default_opts", "pod2g_create", "pod2g_set_values", "pod2g_set_values_batch_dev", "pod2g_solve",
    "pod2g_solve_batch", "pod2g_solve_batch_dev", "pod2g_serve_start", "pod2g_submit", "pod2g_poll",
    "pod2g_serve_stop", "pod2g_info", "pod2g_launch_count", "pod2g_kernel_timing", "pod2g_kernel_times",
    "pod2g_destroy", "pod2g_strerror", "pod2g_solve_noalloc", "pod2g_device_bytes", "pod2g_create_elements",
    "pod2g_set_coeffs", "pod2g_set_coeffs_batch_dev", "pod2g_get_tuning", "pod2g_set_tuning", "pod2g_autotune",
    "pod2g_rom_solution_dev", "pod2g_set_field", "pod2g_set_theta", "pod2g_set_theta_batch", "pod2g_submit_theta",
    "pod2g_coarse_factor", "pod2g_surrogate_create", "pod2g_surrogate_predict_dev", "pod2g_surrogate_destroy",
]
COARSE_DF, COARSE_TENSOR = 0, 1  # K_c contraction of the mixed paths: double-float CUDA cores, or tensor cores
NOALLOC_MAX_N, NOALLOC_MAX_K = 16384, 32
TOO_LARGE = 11
KERNEL_NAMES = ["k_p", "k_spmv", "k_upd", "k_smooth1", "k_restrict", "k_coarse", "k_prol", "k_post"]


class Pattern(C.Structure):
    _fields_ = [("n_brows", C.c_int32), ("bs", C.c_int32), ("row_ptr", C.POINTER(C.c_int32)),
                ("col_idx", C.POINTER(C.c_int32))]


class Elements(C.Structure):
    _fields_ = [("n_elems", C.c_int32), ("npe", C.c_int32), ("conn", C.POINTER(C.c_int32)),
                ("k_ref", C.POINTER(C.c_double)), ("fixed", C.POINTER(C.c_uint8))]


class Tuning(C.Structure):
    _fields_ = [("grid_rows", C.c_int32), ("grid_restrict", C.c_int32), ("grid_prol", C.c_int32),
                ("grid_vec", C.c_int32), ("grid_spmv", C.c_int32), ("rows_kernel", C.c_int32),
                ("restrict_rows", C.c_int32), ("grid_persist", C.c_int32)]


class Opts(C.Structure):
    _fields_ = [("omega", C.c_double), ("pre", C.c_int), ("post", C.c_int), ("precision", C.c_int),
                ("beta_pr", C.c_int), ("max_batch", C.c_int), ("hbm_budget", C.c_size_t),
                ("spin_limit", C.c_int64), ("chunk", C.c_int), ("stream", C.c_void_p), ("method", C.c_int),
                ("smoother", C.c_int), ("coarse", C.c_int)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libpod2g.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} is missing: build it with `python -m paper_2207_02543_gb300.build` "
                      "(the solver has no CPU fallback)")
    lib = C.CDLL(path)
    P, I, D = C.c_void_p, C.c_int, C.c_double
    IP, DP = C.POINTER(C.c_int), C.POINTER(C.c_double)
    lib.pod2g_default_opts.argtypes = [C.POINTER(Opts)]
    lib.pod2g_default_opts.restype = None
    lib.pod2g_create.argtypes = [C.POINTER(Pattern), DP, I, C.POINTER(Opts), C.POINTER(P)]
    lib.pod2g_create_elements.argtypes = [C.POINTER(Pattern), C.POINTER(Elements), DP, I, C.POINTER(Opts),
                                          C.POINTER(P)]
    lib.pod2g_set_coeffs.argtypes = [P, I, P, I]
    lib.pod2g_get_tuning.argtypes = [P, C.POINTER(Tuning)]
    lib.pod2g_rom_solution_dev.argtypes = [P, I, IP, P, P]
    lib.pod2g_set_field.argtypes = [P, DP, I, D, D, I]
    lib.pod2g_set_theta.argtypes = [P, I, DP]
    lib.pod2g_set_theta_batch.argtypes = [P, I, IP, DP, IP]
    lib.pod2g_submit_theta.argtypes = [P, DP, DP, DP, D, I, C.POINTER(C.c_uint64)]
    lib.pod2g_set_tuning.argtypes = [P, C.POINTER(Tuning)]
    lib.pod2g_autotune.argtypes = [P, I, IP, P, I, C.POINTER(Tuning)]
    lib.pod2g_set_coeffs_batch_dev.argtypes = [P, I, IP, P, IP]
    lib.pod2g_set_values.argtypes = [P, I, P, I]
    lib.pod2g_set_values_batch_dev.argtypes = [P, I, IP, P, IP]
    lib.pod2g_solve.argtypes = [P, I, DP, DP, D, I, DP, IP, DP]
    lib.pod2g_solve_batch.argtypes = [P, I, IP, C.POINTER(DP), C.POINTER(DP), D, I, C.POINTER(DP), IP, DP, IP]
    lib.pod2g_solve_batch_dev.argtypes = [P, I, IP, P, P, D, I, P, IP, DP, IP]
    lib.pod2g_serve_start.argtypes = [P, I]
    lib.pod2g_submit.argtypes = [P, DP, DP, DP, D, I, C.POINTER(C.c_uint64)]
    lib.pod2g_poll.argtypes = [P, C.c_uint64, DP, IP, DP, IP, DP]
    lib.pod2g_serve_stop.argtypes = [P]
    lib.pod2g_info.argtypes = [P, IP, IP, IP, IP]
    lib.pod2g_launch_count.argtypes = [P]
    lib.pod2g_launch_count.restype = C.c_int64
    lib.pod2g_device_bytes.argtypes = [P]
    lib.pod2g_device_bytes.restype = C.c_int64
    lib.pod2g_kernel_timing.argtypes = [P, I]
    lib.pod2g_kernel_times.argtypes = [P, DP, C.POINTER(C.c_int64)]
    lib.pod2g_kernel_timing.restype = C.c_int
    lib.pod2g_kernel_times.restype = C.c_int
    lib.pod2g_solve_noalloc.argtypes = [C.c_int32, C.c_int32, C.c_int32, P, P, P, P, I, C.POINTER(Opts), P, P, D, I,
                                        P, IP, DP, IP, P]
    lib.pod2g_solve_noalloc.restype = C.c_int
    lib.pod2g_surrogate_create.argtypes = [C.c_int64, I, I, I, DP, DP, DP, DP, DP, DP, DP, DP, DP, P,
                                           C.POINTER(C.c_void_p)]
    lib.pod2g_surrogate_create.restype = C.c_int
    lib.pod2g_surrogate_predict_dev.argtypes = [P, I, DP, DP, P]
    lib.pod2g_surrogate_predict_dev.restype = C.c_int
    lib.pod2g_surrogate_destroy.argtypes = [P]
    lib.pod2g_surrogate_destroy.restype = None
    lib.pod2g_coarse_factor.argtypes = [P, I, DP]
    lib.pod2g_coarse_factor.restype = C.c_int
    lib.pod2g_destroy.argtypes = [P]
    lib.pod2g_destroy.restype = None
    lib.pod2g_strerror.argtypes = [I]
    lib.pod2g_strerror.restype = C.c_char_p
    for name in ("pod2g_set_field", "pod2g_set_theta", "pod2g_set_theta_batch", "pod2g_submit_theta",
                 "pod2g_rom_solution_dev", "pod2g_get_tuning", "pod2g_set_tuning", "pod2g_autotune", "pod2g_create", "pod2g_create_elements", "pod2g_set_coeffs", "pod2g_set_coeffs_batch_dev",
                 "pod2g_set_values", "pod2g_set_values_batch_dev", "pod2g_solve",
                 "pod2g_solve_batch", "pod2g_solve_batch_dev", "pod2g_serve_start", "pod2g_submit", "pod2g_poll",
                 "pod2g_serve_stop", "pod2g_info"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def strerror(status: int) -> str:
    return load_library().pod2g_strerror(int(status)).decode()


class Pod2gError(RuntimeError):
    def __init__(self, status, where=""):
        super().__init__(f"{where}: {strerror(status)} (status {status})")
        self.status = status


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _is_cuda(t) -> bool:
    return hasattr(t, "is_cuda") and t.is_cuda


class Solver:
    """One context: a shared block-CSR pattern, a POD basis Phi (n x k) and `max_batch` instance slots."""

    def __init__(self, row_ptr, col_idx, bs, phi, *, precision=MIXED_FP32PHI, omega=2.0 / 3.0, pre=1, post=1,
                 beta_pr=False, max_batch=1, hbm_budget=0, chunk=8, spin_limit=0, stream=None, method=0,
                 elements=None, smoother=0, coarse=None):
        """elements: None (instances are given as assembled block values), or a dict with
        conn [n_el, npe] int, k_ref [(npe*bs)^2] float64 and optional fixed [n_brows] bool:
        the element-factored operator, instances given as element coefficients."""
        lib = load_library()
        self._lib = lib
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        self.col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        phi = np.asarray(phi, dtype=np.float64)
        if phi.ndim == 1:
            phi = phi[:, None]
        self.n = (len(self.row_ptr) - 1) * bs
        k = phi.shape[1] if phi.size else 0
        phi_cm = np.asfortranarray(phi) if k else np.zeros(1)
        pat = Pattern(len(self.row_ptr) - 1, bs, self.row_ptr.ctypes.data_as(C.POINTER(C.c_int32)),
                      self.col_idx.ctypes.data_as(C.POINTER(C.c_int32)))
        o = Opts()
        lib.pod2g_default_opts(C.byref(o))
        o.omega, o.pre, o.post, o.precision = omega, pre, post, precision
        o.beta_pr, o.max_batch, o.hbm_budget, o.chunk = int(beta_pr), max_batch, hbm_budget, chunk
        o.spin_limit = spin_limit
        o.stream = C.c_void_p(stream) if stream else None
        o.method = method
        o.smoother = smoother
        if coarse is not None:
            o.coarse = coarse
        h = C.c_void_p()
        if elements is None:
            st = lib.pod2g_create(C.byref(pat), phi_cm.ctypes.data_as(C.POINTER(C.c_double)), k, C.byref(o),
                                  C.byref(h))
            self.inst_len = int(self.row_ptr[-1]) * bs * bs
        else:
            conn = np.ascontiguousarray(elements["conn"], dtype=np.int32)
            kref = np.ascontiguousarray(elements["k_ref"], dtype=np.float64)
            fixed = elements.get("fixed")
            fixed = None if fixed is None else np.ascontiguousarray(fixed, dtype=np.uint8)
            el = Elements(conn.shape[0], conn.shape[1], conn.ctypes.data_as(C.POINTER(C.c_int32)),
                          kref.ctypes.data_as(C.POINTER(C.c_double)),
                          fixed.ctypes.data_as(C.POINTER(C.c_uint8)) if fixed is not None else None)
            st = lib.pod2g_create_elements(C.byref(pat), C.byref(el), phi_cm.ctypes.data_as(C.POINTER(C.c_double)),
                                           k, C.byref(o), C.byref(h))
            self.inst_len = conn.shape[0]
        self.elements = elements is not None
        if st != OK:
            raise Pod2gError(st, "pod2g_create_elements" if elements is not None else "pod2g_create")
        self.h = h
        self.k, self.bs, self.max_batch, self.precision = k, bs, max_batch, precision
        self.nnzb = int(self.row_ptr[-1])

    def coarse_factor(self, slot):
        """The slot's k x k lower Cholesky factor L of K_c = Phi^T K Phi (K_c = L L^T)."""
        L = np.zeros((self.k, self.k))
        st = self._lib.pod2g_coarse_factor(self.h, slot, L.ctypes.data_as(C.POINTER(C.c_double)))
        if st != OK:
            raise Pod2gError(st, "pod2g_coarse_factor")
        return L

    def close(self):
        if getattr(self, "h", None):
            self._lib.pod2g_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch_count(self) -> int:
        return int(self._lib.pod2g_launch_count(self.h))

    def device_bytes(self) -> int:
        return int(self._lib.pod2g_device_bytes(self.h))

    def kernel_timing(self, on: bool = True) -> int:
        return self._lib.pod2g_kernel_timing(self.h, int(on))

    def kernel_times(self):
        """{kernel name: (total ms, timed launches)} of the batched iteration kernels."""
        ms = np.zeros(8)
        cnt = np.zeros(8, dtype=np.int64)
        self._lib.pod2g_kernel_times(self.h, _dptr(ms), cnt.ctypes.data_as(C.POINTER(C.c_int64)))
        return {name: (float(ms[j]), int(cnt[j])) for j, name in enumerate(KERNEL_NAMES)}

    # -------------------------------------------------------------- set-up
    def set_values(self, slot: int, values) -> int:
        """values: numpy float64 (host) or a CUDA float64 tensor, nnzb*bs*bs entries."""
        if _is_cuda(values):
            if values.numel() != self.inst_len:
                return INVALID_ARG
            st = self._lib.pod2g_set_values(self.h, slot, C.c_void_p(values.data_ptr()), 1)
        else:
            v = _f64(values).reshape(-1)
            if v.size != self.inst_len:
                return INVALID_ARG
            st = self._lib.pod2g_set_values(self.h, slot, v.ctypes.data_as(C.c_void_p), 0)
        return st

    def rom_solution_dev(self, slots, b_dev, x_dev) -> int:
        """POD reduced-order solution Phi K_c^-1 Phi^T b for set-up slots (CUDA float64
        tensors [len(slots), n]); use it as x0."""
        slots = np.ascontiguousarray(slots, dtype=np.int32)
        if b_dev.numel() != len(slots) * self.n or x_dev.numel() != len(slots) * self.n:
            return INVALID_ARG
        return self._lib.pod2g_rom_solution_dev(self.h, len(slots), slots.ctypes.data_as(C.POINTER(C.c_int)),
                                                C.c_void_p(b_dev.data_ptr()), C.c_void_p(x_dev.data_ptr()))

    # -------------------------------------------------------------- launch shapes
    def get_tuning(self):
        t = Tuning()
        st = self._lib.pod2g_get_tuning(self.h, C.byref(t))
        if st != OK:
            raise Pod2gError(st, "pod2g_get_tuning")
        return {f: getattr(t, f) for f, _ in Tuning._fields_}

    def set_tuning(self, **shape) -> int:
        cur = self.get_tuning()
        cur.update(shape)
        return self._lib.pod2g_set_tuning(self.h, C.byref(Tuning(**cur)))

    def autotune(self, slots, b_dev, iters=16):
        """Time candidate launch shapes on the given set-up slots (b_dev: CUDA float64 tensor
        [len(slots), n]) and keep the fastest per kernel group. Returns (status, shape)."""
        slots = np.ascontiguousarray(slots, dtype=np.int32)
        if b_dev.numel() != len(slots) * self.n:
            return INVALID_ARG, None
        t = Tuning()
        st = self._lib.pod2g_autotune(self.h, len(slots), slots.ctypes.data_as(C.POINTER(C.c_int)),
                                      C.c_void_p(b_dev.data_ptr()), iters, C.byref(t))
        return st, ({f: getattr(t, f) for f, _ in Tuning._fields_} if st == OK else None)

    def set_coeffs(self, slot: int, coeffs) -> int:
        """Element contexts: coeffs, numpy float64 (host) or a CUDA float64 tensor, n_elems entries."""
        if _is_cuda(coeffs):
            if coeffs.numel() != self.inst_len:
                return INVALID_ARG
            return self._lib.pod2g_set_coeffs(self.h, slot, C.c_void_p(coeffs.data_ptr()), 1)
        v = _f64(coeffs).reshape(-1)
        if v.size != self.inst_len:
            return INVALID_ARG
        return self._lib.pod2g_set_coeffs(self.h, slot, v.ctypes.data_as(C.c_void_p), 0)

    def set_field(self, modes, mu=0.0, sigma=1.0, lognormal=True) -> int:
        """Element contexts: c_e(theta) = exp(mu + sigma * modes[e] . theta) (or without exp).
        modes: [n_elems, m] float64 (host)."""
        modes = np.ascontiguousarray(modes, dtype=np.float64)
        if modes.ndim != 2 or modes.shape[0] != self.inst_len:
            return INVALID_ARG
        self.field_m = modes.shape[1]
        return self._lib.pod2g_set_field(self.h, _dptr(modes), modes.shape[1], mu, sigma, int(lognormal))

    def set_theta(self, slot: int, theta) -> int:
        t = _f64(theta).reshape(-1)
        if t.size != getattr(self, "field_m", -1):
            return INVALID_ARG
        return self._lib.pod2g_set_theta(self.h, slot, _dptr(t))

    def set_theta_batch(self, slots, thetas):
        slots = np.ascontiguousarray(slots, dtype=np.int32)
        t = _f64(thetas).reshape(-1)
        status = np.zeros(len(slots), dtype=np.int32)
        if t.size != len(slots) * getattr(self, "field_m", -1):
            return INVALID_ARG, status
        st = self._lib.pod2g_set_theta_batch(self.h, len(slots), slots.ctypes.data_as(C.POINTER(C.c_int)), _dptr(t),
                                             status.ctypes.data_as(C.POINTER(C.c_int)))
        return st, status

    def submit_theta(self, theta, b, x0=None, tol=1e-8, maxit=1000):
        t = _f64(theta).reshape(-1)
        b = _f64(b)
        if t.size != getattr(self, "field_m", -1) or b.size != self.n or (x0 is not None and np.size(x0) != self.n):
            return INVALID_ARG, 0
        x0a = _f64(x0) if x0 is not None else None
        tk = C.c_uint64(0)
        st = self._lib.pod2g_submit_theta(self.h, _dptr(t), _dptr(b), _dptr(x0a) if x0a is not None else None, tol,
                                          maxit, C.byref(tk))
        return st, tk.value

    def set_coeffs_batch_dev(self, slots, coeffs_dev):
        """coeffs_dev: CUDA float64 tensor [len(slots), n_elems]."""
        slots = np.ascontiguousarray(slots, dtype=np.int32)
        status = np.zeros(len(slots), dtype=np.int32)
        if coeffs_dev.numel() != len(slots) * self.inst_len:
            return INVALID_ARG, status
        st = self._lib.pod2g_set_coeffs_batch_dev(self.h, len(slots), slots.ctypes.data_as(C.POINTER(C.c_int)),
                                                  C.c_void_p(coeffs_dev.data_ptr()),
                                                  status.ctypes.data_as(C.POINTER(C.c_int)))
        return st, status

    def set_values_batch_dev(self, slots, values_dev):
        slots = np.ascontiguousarray(slots, dtype=np.int32)
        status = np.zeros(len(slots), dtype=np.int32)
        if values_dev.numel() != len(slots) * self.inst_len:
            return INVALID_ARG, status
        st = self._lib.pod2g_set_values_batch_dev(self.h, len(slots), slots.ctypes.data_as(C.POINTER(C.c_int)),
                                                  C.c_void_p(values_dev.data_ptr()),
                                                  status.ctypes.data_as(C.POINTER(C.c_int)))
        return st, status

    # -------------------------------------------------------------- solves
    def solve(self, slot, b, x0=None, tol=1e-8, maxit=1000):
        """Single instance, host arrays. Returns (x, iters, relres, status)."""
        b = _f64(b)
        x = np.empty(self.n)
        x0a = _f64(x0) if x0 is not None else None
        it = C.c_int(0)
        rr = C.c_double(0)
        st = self._lib.pod2g_solve(self.h, slot, _dptr(b), _dptr(x0a) if x0a is not None else None, tol, maxit,
                                   _dptr(x), C.byref(it), C.byref(rr))
        return x, it.value, rr.value, st

    def solve_batch(self, slots, B, X0=None, tol=1e-8, maxit=1000):
        """Host arrays B[i], X0[i]. Returns (X, iters, relres, status, rc)."""
        slots = np.ascontiguousarray(slots, dtype=np.int32)
        m = len(slots)
        Bs = [_f64(B[i]) for i in range(m)]
        Xs = [np.empty(self.n) for _ in range(m)]
        X0s = [(_f64(X0[i]) if X0 is not None and X0[i] is not None else None) for i in range(m)]
        DP = C.POINTER(C.c_double)
        barr = (DP * m)(*[_dptr(a) for a in Bs])
        xarr = (DP * m)(*[_dptr(a) for a in Xs])
        x0arr = (DP * m)(*[(_dptr(a) if a is not None else DP()) for a in X0s]) if X0 is not None else None
        iters = np.zeros(m, dtype=np.int32)
        rel = np.zeros(m)
        status = np.zeros(m, dtype=np.int32)
        rc = self._lib.pod2g_solve_batch(self.h, m, slots.ctypes.data_as(C.POINTER(C.c_int)), barr, x0arr, tol, maxit,
                                         xarr, iters.ctypes.data_as(C.POINTER(C.c_int)), _dptr(rel),
                                         status.ctypes.data_as(C.POINTER(C.c_int)))
        return np.stack(Xs), iters, rel, status, rc

    def solve_batch_dev(self, slots, b_dev, x_dev, x0_dev=None, tol=1e-8, maxit=1000):
        """Device tensors b_dev, x_dev (and x0_dev): [len(slots), n] float64 on the context's GPU."""
        slots = np.ascontiguousarray(slots, dtype=np.int32)
        m = len(slots)
        iters = np.zeros(m, dtype=np.int32)
        rel = np.zeros(m)
        status = np.zeros(m, dtype=np.int32)
        if b_dev.numel() != m * self.n or x_dev.numel() != m * self.n or \
                (x0_dev is not None and x0_dev.numel() != m * self.n):
            return iters, rel, status, INVALID_ARG
        rc = self._lib.pod2g_solve_batch_dev(self.h, m, slots.ctypes.data_as(C.POINTER(C.c_int)),
                                             C.c_void_p(b_dev.data_ptr()),
                                             C.c_void_p(x0_dev.data_ptr()) if x0_dev is not None else None, tol, maxit,
                                             C.c_void_p(x_dev.data_ptr()), iters.ctypes.data_as(C.POINTER(C.c_int)),
                                             _dptr(rel), status.ctypes.data_as(C.POINTER(C.c_int)))
        return iters, rel, status, rc

    # -------------------------------------------------------------- serving
    def serve_start(self, max_queue=1024):
        st = self._lib.pod2g_serve_start(self.h, max_queue)
        if st != OK:
            raise Pod2gError(st, "pod2g_serve_start")

    def submit(self, values, b, x0=None, tol=1e-8, maxit=1000):
        """values: the instance's block values, or its element coefficients for an element context."""
        v = _f64(values).reshape(-1)
        b = _f64(b)
        if v.size != self.inst_len or b.size != self.n or (x0 is not None and np.size(x0) != self.n):
            return INVALID_ARG, 0
        x0a = _f64(x0) if x0 is not None else None
        t = C.c_uint64(0)
        st = self._lib.pod2g_submit(self.h, _dptr(v), _dptr(b), _dptr(x0a) if x0a is not None else None, tol, maxit,
                                    C.byref(t))
        return st, t.value

    def poll(self, ticket):
        x = np.empty(self.n)
        it = C.c_int(0)
        rr = C.c_double(0)
        s = C.c_int(0)
        lat = C.c_double(0)
        st = self._lib.pod2g_poll(self.h, ticket, _dptr(x), C.byref(it), C.byref(rr), C.byref(s), C.byref(lat))
        if st != OK:
            return st, None
        return OK, dict(x=x, iters=it.value, relres=rr.value, status=s.value, latency_s=lat.value)

    def serve_stop(self):
        return self._lib.pod2g_serve_stop(self.h)


def solve_noalloc(row_ptr_dev, col_idx_dev, bs, values_dev, phi_dev, k, b_dev, x_dev, x0_dev=None, tol=1e-8,
                  maxit=1000, omega=2.0 / 3.0, pre=1, post=1, beta_pr=False, stream=None):
    """pod2g_solve_noalloc: FP64 solve with no device allocation. All arrays are CUDA tensors
    (row_ptr/col_idx int32, values/phi/b/x0/x float64; phi column-major [k][n] flattened).
    Returns (rc, iters, relres, status)."""
    lib = load_library()
    o = Opts()
    lib.pod2g_default_opts(C.byref(o))
    o.omega, o.pre, o.post, o.beta_pr, o.precision = omega, pre, post, int(beta_pr), FP64
    it = C.c_int(0)
    rr = C.c_double(0.0)
    st = C.c_int(0)
    ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    nb = row_ptr_dev.numel() - 1
    rc = lib.pod2g_solve_noalloc(nb, bs, col_idx_dev.numel(), ptr(row_ptr_dev), ptr(col_idx_dev), ptr(values_dev),
                                 ptr(phi_dev), k, C.byref(o), ptr(b_dev), ptr(x0_dev), tol, maxit, ptr(x_dev),
                                 C.byref(it), C.byref(rr), C.byref(st), C.c_void_p(stream) if stream else None)
    return rc, it.value, rr.value, st.value


class ServingMix:
    """Requests for several registered problems, served concurrently.

    Each problem gets its own context (its pattern, POD basis and instance slots) whose
    serving worker batches that problem's requests continuously; the contexts run on
    their own streams, so the problems' work overlaps on the device. Problems are
    admitted under one HBM budget: registering a problem whose context would exceed
    the remaining budget fails with ADMISSION. Requests beyond a problem's queue
    limit are refused with ADMISSION by pod2g_submit."""

    def __init__(self, hbm_budget: int, max_queue: int = 1024):
        self.budget = int(hbm_budget)
        self.max_queue = max_queue
        self.solvers = {}

    def used_bytes(self) -> int:
        return sum(s.device_bytes() for s in self.solvers.values())

    def register(self, name, row_ptr, col_idx, bs, phi, **kw) -> int:
        remaining = self.budget - self.used_bytes()
        if remaining <= 0:
            return ADMISSION
        try:
            s = Solver(row_ptr, col_idx, bs, phi, hbm_budget=remaining, **kw)
        except Pod2gError as e:
            return e.status
        s.serve_start(self.max_queue)
        self.solvers[name] = s
        return OK

    def submit(self, name, values, b, x0=None, tol=1e-8, maxit=1000):
        st, t = self.solvers[name].submit(values, b, x0=x0, tol=tol, maxit=maxit)
        return st, (name, t)

    def poll(self, handle):
        name, t = handle
        return self.solvers[name].poll(t)

    def close(self):
        for s in self.solvers.values():
            s.serve_stop()
            s.close()
        self.solvers = {}


class Surrogate:
    """Surrogate initial guess on the device (Section 3.2): u = s * Psi (z_mean + z_std * FFNN(theta)).

    weights: an object with psi [n, ks], w1 [H, m], b1 [H], w2 [H, H], b2 [H], w3 [ks, H], b3 [ks],
    z_mean [ks], z_std [ks] (float64 arrays)."""

    def __init__(self, weights, stream=None):
        lib = load_library()
        self._lib = lib
        psi = np.asfortranarray(np.asarray(weights.psi, dtype=np.float64))
        self.n, self.ks = psi.shape
        w1 = np.ascontiguousarray(weights.w1, dtype=np.float64)
        self.H, self.m = w1.shape
        arrs = [psi, w1] + [np.ascontiguousarray(getattr(weights, k), dtype=np.float64)
                            for k in ("b1", "w2", "b2", "w3", "b3", "z_mean", "z_std")]
        self._keep = arrs
        h = C.c_void_p()
        st = lib.pod2g_surrogate_create(self.n, self.m, self.ks, self.H, *[_dptr(a) for a in arrs],
                                        C.c_void_p(stream) if stream else None, C.byref(h))
        if st != OK:
            raise Pod2gError(st, "pod2g_surrogate_create")
        self.h = h

    def predict_dev(self, theta, scale, x_dev) -> int:
        """x_dev[q] = prediction for theta[q] (host [nq, m]) and load factor scale[q] (host [nq])."""
        theta = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1, self.m)
        scale = None if scale is None else np.ascontiguousarray(scale, dtype=np.float64)
        return self._lib.pod2g_surrogate_predict_dev(self.h, theta.shape[0], _dptr(theta),
                                                     _dptr(scale) if scale is not None else None,
                                                     C.c_void_p(x_dev.data_ptr()))

    def close(self):
        if getattr(self, "h", None):
            self._lib.pod2g_surrogate_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass
