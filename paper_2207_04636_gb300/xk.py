"""Python binding of libxk (ctypes): argument marshalling only.

Every step of the exchange build runs in the CUDA kernels of libxk.so; this
module checks shapes and dtypes, passes pointers and turns return codes into
exceptions.  The library must have been built (paper_2207_04636_gb300.build);
importing this module without it raises at once rather than falling back to
anything else.
"""
import ctypes
import os

import numpy as np

from . import build as _build

XK_OK, XK_PENDING = 0, 1
XK_EINVAL, XK_ENOMEM, XK_ETIMEDOUT, XK_ECUDA, XK_EBUSY = -1, -2, -3, -4, -5
XK_FP64, XK_TF32, XK_F16X3 = 0, 1, 2
MODES = {"fp64": XK_FP64, "f16x3": XK_F16X3}
STEPS = ("orbitals", "pair", "m2", "m1", "line1", "line2", "line3", "assemble")
_NAMES = {XK_EINVAL: "XK_EINVAL", XK_ENOMEM: "XK_ENOMEM", XK_ETIMEDOUT: "XK_ETIMEDOUT",
          XK_ECUDA: "XK_ECUDA", XK_EBUSY: "XK_EBUSY"}


class XKError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """The loaded libxk.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise ImportError(f"libxk.so is missing ({_build.LIB}); build it with "
                              "paper_2207_04636_gb300.build.build_library()")
        L = ctypes.CDLL(_build.LIB)
        c_d, c_i64, c_i32, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
        L.xk_footprint.argtypes = [c_i64, c_i32, c_i32, c_i32, c_int, ctypes.POINTER(ctypes.c_size_t)]
        L.xk_setup.argtypes = [c_i64, c_i32, c_i32, c_i32, c_d, c_d, c_d, c_d, ctypes.c_double,
                               c_int, ctypes.POINTER(ctypes.c_void_p)]
        L.xk_setup_isdf.argtypes = [c_i64, c_i32, c_i32, c_i32, c_d, c_d, c_i32, ctypes.c_double,
                                    c_int, ctypes.POINTER(ctypes.c_void_p)]
        L.xk_setup_queued.argtypes = [c_i64, c_i32, c_i32, c_i32, c_d, c_d, c_d, c_d,
                                      ctypes.c_double, c_int, ctypes.c_double, c_d]
        L.xk_admit_reserve.argtypes = [ctypes.c_uint64, ctypes.c_double,
                                       ctypes.POINTER(ctypes.c_uint64)]
        L.xk_admit_release.argtypes = [ctypes.c_uint64]
        L.xk_autotune_info.argtypes = [c_d, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]
        L.xk_admit_state.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32)]
        L.xk_setup_shard.argtypes = [c_i64, c_i32, c_i32, c_i32, c_i32, c_i32, c_d, c_d, c_d, c_d,
                                     ctypes.c_double, c_int, ctypes.POINTER(ctypes.c_void_p)]
        L.xk_tables.argtypes = [c_d, c_d, c_d, c_i32, c_d, c_d]
        L.xk_isdf_points.argtypes = [c_i32, c_i32, c_d, c_i32, ctypes.c_double, c_d, c_d]
        L.xk_build.argtypes = [c_d, c_d, c_d, c_d]
        L.xk_build_device.argtypes = [c_d, c_d, c_d, c_d, c_d]
        L.xk_energy.argtypes = [c_d, c_d, c_d]
        L.xk_build_full.argtypes = [c_d, c_d, c_d]
        L.xk_coulomb.argtypes = [c_d, c_i32, ctypes.c_double, c_d, c_d, c_d]
        L.xk_energy_device.argtypes = [c_d, c_d, c_d, c_d]
        L.xk_ace.argtypes = [c_d, c_d, c_d, c_d, ctypes.POINTER(c_int)]
        L.xk_submit.argtypes = [c_d, c_d, ctypes.c_double, ctypes.POINTER(ctypes.c_uint64)]
        L.xk_poll.argtypes = [ctypes.c_uint64, c_d, c_d, c_d]
        L.xk_release.argtypes = [c_d]
        L.xk_timing_enable.argtypes = [c_d, c_int]
        L.xk_timing_read.argtypes = [c_d, c_int, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_uint64)]
        L.xk_exchange_energy_noalloc.argtypes = [c_d, c_d, c_i64, c_d, c_d]
        L.xk_batch_create.argtypes = [c_d, c_int, ctypes.POINTER(ctypes.c_void_p)]
        L.xk_batch_build.argtypes = [c_d, c_d, c_d, c_d]
        L.xk_batch_release.argtypes = [c_d]
        L.xk_set_wait_limit.argtypes = [c_d, c_i64]
        L.xk_error_estimate.argtypes = [c_d, c_d]
        L.xk_last_error.restype = ctypes.c_char_p
        L.xk_kernel_launches.restype = ctypes.c_uint64
        for f in ("xk_footprint", "xk_setup", "xk_setup_shard", "xk_setup_isdf", "xk_tables", "xk_isdf_points",
                  "xk_build",
                  "xk_build_device", "xk_build_full",
                  "xk_coulomb",
                  "xk_energy",
                  "xk_energy_device", "xk_ace",
                  "xk_submit", "xk_poll", "xk_release", "xk_timing_enable", "xk_timing_read",
                  "xk_exchange_energy_noalloc", "xk_batch_create", "xk_batch_build",
                  "xk_batch_release", "xk_set_wait_limit", "xk_error_estimate"):
            getattr(L, f).restype = c_int
        _lib = L
    return _lib


def last_error() -> str:
    return lib().xk_last_error().decode()


def kernel_launches() -> int:
    return int(lib().xk_kernel_launches())


def _check(rc):
    if rc < 0:
        raise XKError(rc, last_error())
    return rc


def _f64(a, shape, name):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != shape:
        raise ValueError(f"{name}: expected shape {shape}, got {a.shape}")
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def footprint(Ng, N, n, Naux, mode="fp64") -> int:
    out = ctypes.c_size_t()
    _check(lib().xk_footprint(Ng, N, n, Naux, MODES[mode], ctypes.byref(out)))
    return int(out.value)


def admit_reserve(nbytes, timeout_ms=-1.0):
    """Reserve nbytes against the admission budget (xk_admit_reserve); returns
    the token.  timeout_ms < 0: now or XKError(XK_ENOMEM); else wait in the
    admission queue (XKError(XK_ETIMEDOUT) when not admitted in time)."""
    tok = ctypes.c_uint64()
    _check(lib().xk_admit_reserve(int(nbytes), float(timeout_ms), ctypes.byref(tok)))
    return tok.value


def admit_release(token):
    """Return a reservation's bytes and wake the admission queue (xk_admit_release)."""
    _check(lib().xk_admit_release(int(token)))


def admit_state():
    """(bytes admitted, requests waiting) of the admission queue (xk_admit_state)."""
    b = ctypes.c_uint64()
    w = ctypes.c_uint32()
    _check(lib().xk_admit_state(ctypes.byref(b), ctypes.byref(w)))
    return b.value, w.value


class Handle:
    """Per-geometry device tables plus build scratch (xk_setup / xk_release)."""

    def __init__(self, phi, idx, V, W, dV, n, mode="fp64", queue_timeout_ms=None):
        """queue_timeout_ms: None admits now or raises (xk_setup); a number waits
        in the admission queue up to that many milliseconds (xk_setup_queued)."""
        phi = np.asarray(phi)
        Ng, N = phi.shape
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        Naux = idx.shape[0]
        self.Ng, self.N, self.n, self.Naux, self.mode = Ng, N, int(n), Naux, mode
        phi = _f64(phi, (Ng, N), "phi")
        V = _f64(V, (Naux, Ng), "V")
        W = _f64(W, (Naux, Naux), "W")
        h = ctypes.c_void_p()
        if queue_timeout_ms is None:
            _check(lib().xk_setup(Ng, N, self.n, Naux, _ptr(phi), _ptr(idx), _ptr(V), _ptr(W),
                                  float(dV), MODES[mode], ctypes.byref(h)))
        else:
            _check(lib().xk_setup_queued(Ng, N, self.n, Naux, _ptr(phi), _ptr(idx), _ptr(V),
                                         _ptr(W), float(dV), MODES[mode], float(queue_timeout_ms),
                                         ctypes.byref(h)))
        self._h = h

    @classmethod
    def shard(cls, phi, idx, V_rows, W_rows, g0, g1, dV, n, mode="fp64"):
        """Handle of the g-slice [g0, g1) (xk_setup_shard): V_rows and W_rows are
        the slice's rows of V (N_g columns) and W (all N_aux columns); its builds
        return the slice's share of K and E_x."""
        self = cls.__new__(cls)
        phi = np.asarray(phi)
        Ng, N = phi.shape
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        Naux = idx.shape[0]
        self.Ng, self.N, self.n, self.Naux, self.mode = Ng, N, int(n), Naux, mode
        phi = _f64(phi, (Ng, N), "phi")
        V_rows = _f64(V_rows, (g1 - g0, Ng), "V_rows")
        W_rows = _f64(W_rows, (g1 - g0, Naux), "W_rows")
        h = ctypes.c_void_p()
        _check(lib().xk_setup_shard(Ng, N, self.n, Naux, int(g0), int(g1), _ptr(phi), _ptr(idx),
                                    _ptr(V_rows), _ptr(W_rows), float(dV), MODES[mode],
                                    ctypes.byref(h)))
        self._h = h
        return self

    @classmethod
    def isdf(cls, phi, idx, grid, L, n, mode="fp64"):
        """Handle whose chi, V and W are formed on the device from the basis and
        the interpolation points of a cubic grid^3 cell of side L (xk_setup_isdf)."""
        self = cls.__new__(cls)
        phi = np.asarray(phi)
        Ng, N = phi.shape
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        self.Ng, self.N, self.n, self.Naux, self.mode = Ng, N, int(n), idx.shape[0], mode
        phi = _f64(phi, (Ng, N), "phi")
        h = ctypes.c_void_p()
        _check(lib().xk_setup_isdf(Ng, N, self.n, self.Naux, _ptr(phi), _ptr(idx), int(grid),
                                   float(L), MODES[mode], ctypes.byref(h)))
        self._h = h
        return self

    def tables(self, rows=()):
        """(W, V[rows], ridge) of an XK_FP64 handle (xk_tables)."""
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        W = np.empty((self.Naux, self.Naux))
        Vr = np.empty((max(rows.size, 1), self.Ng))
        rg = np.empty(1)
        _check(lib().xk_tables(self._h, _ptr(W), _ptr(rows) if rows.size else None, rows.size,
                               _ptr(Vr) if rows.size else None, _ptr(rg)))
        return W, Vr[:rows.size], float(rg[0])

    def build(self, C):
        """Blocking build from host C (N x n): returns (K_{mu i}, E_x)."""
        C = _f64(C, (self.N, self.n), "C")
        K = np.empty((self.N, self.n))
        Ex = np.empty(1)
        _check(lib().xk_build(self._h, _ptr(C), _ptr(K), _ptr(Ex)))
        return K, float(Ex[0])

    def build_device(self, C_dev, K_dev, Ex_dev, stream=0):
        """Enqueue a build on device buffers (integers: device addresses,
        e.g. torch tensor .data_ptr()) on the given cudaStream_t handle."""
        _check(lib().xk_build_device(self._h, ctypes.c_void_p(C_dev), ctypes.c_void_p(K_dev),
                                     ctypes.c_void_p(Ex_dev), ctypes.c_void_p(stream)))

    def build_full(self, C):
        """Full K_{mu nu} (N x N) from host C (xk_build_full)."""
        C = _f64(C, (self.N, self.n), "C")
        K = np.empty((self.N, self.N))
        _check(lib().xk_build_full(self._h, _ptr(C), _ptr(K)))
        return K

    def coulomb(self, C, grid, L):
        """(J (N x N), E_J) on a cubic grid of side L with grid^3 = N_g (xk_coulomb)."""
        C = _f64(C, (self.N, self.n), "C")
        J = np.empty((self.N, self.N))
        EJ = np.empty(1)
        _check(lib().xk_coulomb(self._h, int(grid), float(L), _ptr(C), _ptr(J), _ptr(EJ)))
        return J, float(EJ[0])

    def energy(self, C):
        """E_x alone from host C (N x n), without K (xk_energy)."""
        C = _f64(C, (self.N, self.n), "C")
        Ex = np.empty(1)
        _check(lib().xk_energy(self._h, _ptr(C), _ptr(Ex)))
        return float(Ex[0])

    def energy_device(self, C_dev, Ex_dev, stream=0):
        """Enqueue xk_energy on device buffers (integers: device addresses)."""
        _check(lib().xk_energy_device(self._h, ctypes.c_void_p(C_dev), ctypes.c_void_p(Ex_dev),
                                      ctypes.c_void_p(stream)))

    def ace(self):
        """(K_ij, xi, sign, branch) of the last build: branch 'cholesky' or 'eigen'."""
        Kij = np.empty((self.n, self.n))
        xi = np.empty((self.N, self.n))
        sg = np.empty(self.n)
        br = ctypes.c_int()
        _check(lib().xk_ace(self._h, _ptr(Kij), _ptr(xi), _ptr(sg), ctypes.byref(br)))
        return Kij, xi, sg, ("cholesky" if br.value == 0 else "eigen")

    def submit(self, C, deadline_ms=0.0) -> int:
        C = _f64(C, (self.N, self.n), "C")
        t = ctypes.c_uint64()
        _check(lib().xk_submit(self._h, _ptr(C), float(deadline_ms), ctypes.byref(t)))
        return int(t.value)

    def error_estimate(self) -> float:
        """|E_x - E_K| of the last build (E_K = -sum K o C of the returned K)."""
        est = np.empty(1)
        _check(lib().xk_error_estimate(self._h, _ptr(est)))
        return float(est[0])

    def autotune_info(self):
        """The set-up autotuner's choices (xk_autotune_info): {"back_tiles": 128 |
        256 | 0, "m2_split": int, "ms_128": t, "ms_256": t, "ms_tuned_pair": t}."""
        info = (ctypes.c_int32 * 2)()
        ms = (ctypes.c_double * 3)()
        _check(lib().xk_autotune_info(self._h, info, ms))
        return {"back_tiles": info[0], "m2_split": info[1], "ms_128": ms[0], "ms_256": ms[1],
                "ms_tuned_pair": ms[2]}

    def set_wait_limit(self, cycles: int):
        """Bound (SM cycles) on the pipeline waits of this handle's kernels; 0 = default."""
        _check(lib().xk_set_wait_limit(self._h, int(cycles)))

    def timing(self, enable=True):
        """Turn per-step CUDA-event timing on (clearing it) or off."""
        _check(lib().xk_timing_enable(self._h, 1 if enable else 0))

    def step_times(self):
        """{step name: (total device ms, builds)} since timing was enabled."""
        out = {}
        for i, name in enumerate(STEPS):
            ms = ctypes.c_double()
            nb = ctypes.c_uint64()
            _check(lib().xk_timing_read(self._h, i, ctypes.byref(ms), ctypes.byref(nb)))
            out[name] = (ms.value, int(nb.value))
        return out

    def release(self):
        if getattr(self, "_h", None):
            lib().xk_release(self._h)
            self._h = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class Batch:
    """One build of each of several XK_F16X3 handles per call, captured into
    a CUDA graph (xk_batch_create / xk_batch_build / xk_batch_release).  The
    handles must outlive the batch."""

    def __init__(self, handles):
        self.handles = list(handles)
        arr = (ctypes.c_void_p * len(self.handles))(*[h._h for h in self.handles])
        b = ctypes.c_void_p()
        _check(lib().xk_batch_create(arr, len(self.handles), ctypes.byref(b)))
        self._b = b

    def build(self, Cs):
        """Cs: one host C (N_i x n_i) per handle; returns ([K_i], [E_i])."""
        Cs = [_f64(C, (h.N, h.n), "C") for C, h in zip(Cs, self.handles)]
        Ks = [np.empty((h.N, h.n)) for h in self.handles]
        Ex = np.empty(len(self.handles))
        cp = (ctypes.c_void_p * len(Cs))(*[C.ctypes.data for C in Cs])
        kp = (ctypes.c_void_p * len(Ks))(*[K.ctypes.data for K in Ks])
        _check(lib().xk_batch_build(self._b, cp, kp, _ptr(Ex)))
        return Ks, [float(e) for e in Ex]

    def release(self):
        if getattr(self, "_b", None):
            lib().xk_batch_release(self._b)
            self._b = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def isdf_points(rows, want, tol_rel=1e-14):
    """Pivots (indices into rows, selection order) of the greedy pivoted
    Cholesky of the pair Gram of the candidate rows (xk_isdf_points)."""
    rows = np.ascontiguousarray(rows, dtype=np.float64)
    m, N = rows.shape
    piv = np.empty(max(int(want), 1), dtype=np.int32)
    cnt = np.empty(1, dtype=np.int32)
    _check(lib().xk_isdf_points(m, N, _ptr(rows), int(want), float(tol_rel), _ptr(piv), _ptr(cnt)))
    return piv[:int(cnt[0])].astype(np.int64)


def exchange_energy_noalloc(K_dev, C_dev, count, Ex_dev, stream=0):
    """E_x = -sum K*C over `count` device doubles into the device double at
    Ex_dev, without any allocation (integers: device addresses)."""
    _check(lib().xk_exchange_energy_noalloc(ctypes.c_void_p(K_dev), ctypes.c_void_p(C_dev),
                                            int(count), ctypes.c_void_p(Ex_dev),
                                            ctypes.c_void_p(stream)))


def poll(ticket, N, n):
    """(status, K, E_x, err_est); status XK_PENDING while running."""
    K = np.empty((N, n))
    Ex = np.empty(1)
    eb = np.empty(1)
    rc = lib().xk_poll(ctypes.c_uint64(ticket), _ptr(K), _ptr(Ex), _ptr(eb))
    if rc == XK_PENDING:
        return rc, None, None, None
    _check(rc)
    return rc, K, float(Ex[0]), float(eb[0])
