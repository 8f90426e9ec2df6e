"""ctypes binding of libmoma (include/moma.h): the same entry points, with
argument marshalling only.  Every computation runs in the CUDA library;
there is no Python or CPU fallback -- a missing library raises.

Buffers may be numpy arrays (host memory) or torch tensors (host or CUDA
memory); they must be C-contiguous complex128 or complex64 arrays in the
layouts of moma.h.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmoma.so")

MOMA_OK = 0
STATUS = {
    0: "MOMA_OK", 1: "MOMA_ERR_ARG", 2: "MOMA_ERR_STATE", 3: "MOMA_ERR_OOM", 4: "MOMA_ERR_CUDA",
    5: "MOMA_ERR_NOT_PD", 6: "MOMA_ERR_NOT_CONVERGED", 7: "MOMA_ERR_BREAKDOWN", 8: "MOMA_ERR_NONFINITE",
    9: "MOMA_ERR_TIMEOUT",
}
MOMA_C128, MOMA_C64 = 0, 1
MOMA_PREC_FP64, MOMA_PREC_MIXED = 0, 1
MOMA_OP_Z, MOMA_OP_ZH, MOMA_OP_NORMAL = 0, 1, 2
KERNEL_IDS = {"bin_c64": 0, "bin_c128": 1, "precond": 2, "fft_c64": 3, "block_fft": 4, "fft_c128": 5,
              "gram": 6, "box_sums": 7, "cholesky": 8, "tri_inverse": 9, "krylov": 10, "misc": 11,
              "bin_tc": 12, "precond_tc": 13}

# Every symbol include/moma.h declares, for the export check.
EXPORTS = [
    "moma_create_array", "moma_set_blocks", "moma_matvec", "moma_apply_precond", "moma_get_bin",
    "moma_get_precond_block", "moma_solve", "moma_active_impedance", "moma_profile", "moma_kernel_stats",
    "moma_launch_count", "moma_device_bytes", "moma_destroy", "moma_last_error", "moma_matvec_noalloc",
    "moma_set_stream", "moma_release_setup", "moma_estimate_bytes", "moma_tuning_report", "moma_array_stream",
    "moma_set_blocks_batch", "moma_solve_batch", "moma_port_impedance",
    "moma_column_coupling", "moma_s_to_z", "moma_s_ideal", "moma_xi_z", "moma_xi_s", "moma_set_margin",
    "moma_server_create", "moma_server_submit", "moma_server_wait", "moma_server_get_stats", "moma_server_destroy",
    "moma_time_operator",
]


class MomaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


MOMA_FLAG_NO_GRAPHS, MOMA_FLAG_NO_AUTOTUNE, MOMA_FLAG_NO_TENSOR, MOMA_FLAG_TENSOR_ALWAYS = 1, 2, 4, 8
MOMA_FLAG_FP64_RESIDUAL, MOMA_FLAG_AXIS_FFT, MOMA_FLAG_PRECOND_PER_ELEMENT, MOMA_FLAG_SPLIT_ARNOLDI = 16, 32, 64, 128


class moma_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("mx", ctypes.c_int), ("my", ctypes.c_int), ("restart", ctypes.c_int),
                ("flags", ctypes.c_int)]


MOMA_SOLVER_GMRES, MOMA_SOLVER_PCG = 0, 1
MOMA_TIME_Z, MOMA_TIME_BIN, MOMA_TIME_PRECOND, MOMA_TIME_NORMAL = 0, 1, 2, 3


class moma_solve_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("warm_start", ctypes.c_int), ("solver", ctypes.c_int), ("max_inner", ctypes.c_int)]


class moma_solve_info(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int), ("converged", ctypes.c_int),
                ("max_rel_residual", ctypes.c_double), ("first_inner_reduction", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class moma_server_opts(ctypes.Structure):
    _fields_ = [("max_device_bytes", ctypes.c_size_t), ("slots", ctypes.c_int), ("precision", ctypes.c_int),
                ("restart", ctypes.c_int)]


class moma_request(ctypes.Structure):
    _fields_ = [("key", ctypes.c_ulonglong), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("b", ctypes.c_int),
                ("blocks", ctypes.c_void_p), ("blocks_dtype", ctypes.c_int), ("nrhs", ctypes.c_int),
                ("V", ctypes.c_void_p), ("I", ctypes.c_void_p), ("Za", ctypes.c_void_p), ("Gamma", ctypes.c_void_p),
                ("port_basis", ctypes.c_int), ("z0", ctypes.c_double), ("tol", ctypes.c_double)]


class moma_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("resident_hit", ctypes.c_int), ("queue_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double), ("total_ms", ctypes.c_double), ("info", moma_solve_info),
                ("message", ctypes.c_char * 256)]

    def as_dict(self):
        return {"status": self.status, "resident_hit": self.resident_hit, "queue_ms": self.queue_ms,
                "run_ms": self.run_ms, "total_ms": self.total_ms, "info": self.info.as_dict(),
                "message": self.message.decode(errors="replace")}


class moma_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_ulonglong), ("completed", ctypes.c_ulonglong), ("hits", ctypes.c_ulonglong),
                ("misses", ctypes.c_ulonglong), ("evictions", ctypes.c_ulonglong), ("resident_arrays", ctypes.c_int),
                ("queued", ctypes.c_int), ("resident_bytes", ctypes.c_size_t), ("budget_bytes", ctypes.c_size_t)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib():
    """Load libmoma.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2608_17844_b300.build`")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.moma_create_array.argtypes = [i, i, i, ctypes.POINTER(moma_options), vp, ctypes.POINTER(vp)]
    L.moma_set_blocks.argtypes = [vp, vp, i]
    L.moma_matvec.argtypes = [vp, i, i, vp, vp, i]
    L.moma_apply_precond.argtypes = [vp, i, vp, vp, i]
    L.moma_matvec_noalloc.argtypes = [vp, i, i, vp, vp, i]
    L.moma_set_stream.argtypes = [vp, vp]
    L.moma_port_impedance.argtypes = [vp, i, i, ctypes.POINTER(moma_solve_opts), vp, vp]
    d = ctypes.c_double
    L.moma_column_coupling.argtypes = [vp, i, i, i, d, ctypes.POINTER(moma_solve_opts), vp, vp]
    L.moma_s_to_z.argtypes = [vp, i, d, vp, vp]
    L.moma_set_margin.argtypes = [vp, i, vp, vp, i]
    L.moma_s_ideal.argtypes = [i, i, d, d, d, d, d, vp, vp]
    L.moma_xi_z.argtypes = [vp, i, i, ctypes.POINTER(ctypes.c_double)]
    L.moma_xi_s.argtypes = [i, i, d, d, d, d, d, d, ctypes.POINTER(ctypes.c_double)]
    L.moma_tuning_report.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    L.moma_array_stream.argtypes = [vp]
    L.moma_array_stream.restype = vp
    L.moma_set_blocks_batch.argtypes = [i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i), i, i,
                                        ctypes.POINTER(i)]
    L.moma_solve_batch.argtypes = [i, ctypes.POINTER(vp), ctypes.POINTER(i), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                   ctypes.POINTER(moma_solve_opts), ctypes.POINTER(moma_solve_info), i,
                                   ctypes.POINTER(i)]
    L.moma_release_setup.argtypes = [vp]
    L.moma_time_operator.argtypes = [vp, i, i, i, ctypes.POINTER(ctypes.c_double)]
    L.moma_estimate_bytes.argtypes = [i, i, i, ctypes.POINTER(moma_options), i, i]
    L.moma_estimate_bytes.restype = ctypes.c_size_t
    L.moma_server_create.argtypes = [ctypes.POINTER(moma_server_opts), ctypes.POINTER(vp)]
    L.moma_server_submit.argtypes = [vp, ctypes.POINTER(moma_request), ctypes.POINTER(ctypes.c_ulonglong)]
    L.moma_server_wait.argtypes = [vp, ctypes.c_ulonglong, d, ctypes.POINTER(moma_result)]
    L.moma_server_get_stats.argtypes = [vp, ctypes.POINTER(moma_server_stats)]
    L.moma_server_destroy.argtypes = [vp]
    L.moma_server_destroy.restype = None
    L.moma_get_bin.argtypes = [vp, i, i, i, vp]
    L.moma_get_precond_block.argtypes = [vp, i, i, vp]
    L.moma_solve.argtypes = [vp, i, vp, vp, ctypes.POINTER(moma_solve_opts), ctypes.POINTER(moma_solve_info),
                             ctypes.POINTER(d)]
    L.moma_active_impedance.argtypes = [vp, i, vp, vp, i, d, vp, vp]
    L.moma_profile.argtypes = [vp, i]
    L.moma_kernel_stats.argtypes = [vp, i, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(d)]
    L.moma_launch_count.argtypes = [vp]
    L.moma_launch_count.restype = ctypes.c_longlong
    L.moma_device_bytes.argtypes = [vp]
    L.moma_device_bytes.restype = ctypes.c_size_t
    L.moma_destroy.argtypes = [vp]
    L.moma_destroy.restype = None
    L.moma_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("moma_launch_count", "moma_device_bytes", "moma_destroy", "moma_last_error",
                        "moma_estimate_bytes", "moma_server_destroy", "moma_array_stream"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(st):
    if st != MOMA_OK:
        raise MomaError(st, lib().moma_last_error().decode())


def _ptr_dtype(a):
    """(pointer, moma_dtype) of a C-contiguous complex numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if a.dtype == np.complex128:
            return a.ctypes.data, MOMA_C128
        if a.dtype == np.complex64:
            return a.ctypes.data, MOMA_C64
        raise TypeError(f"unsupported dtype {a.dtype}")
    import torch
    if isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if a.dtype == torch.complex128:
            return a.data_ptr(), MOMA_C128
        if a.dtype == torch.complex64:
            return a.data_ptr(), MOMA_C64
        raise TypeError(f"unsupported dtype {a.dtype}")
    raise TypeError(type(a))


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


def moma_create_array(nx, ny, b, precision=MOMA_PREC_MIXED, mx=0, my=0, restart=0, stream=None, flags=0):
    h = ctypes.c_void_p()
    opt = moma_options(precision, mx, my, restart, flags)
    _check(lib().moma_create_array(nx, ny, b, ctypes.byref(opt), _stream_handle(stream), ctypes.byref(h)))
    return h


def moma_set_blocks(h, blocks):
    p, dt = _ptr_dtype(blocks)
    _check(lib().moma_set_blocks(h, p, dt))


def moma_matvec(h, op, x, y):
    px, dt = _ptr_dtype(x)
    py, dty = _ptr_dtype(y)
    if dt != dty:
        raise TypeError("x and y must have the same dtype")
    _check(lib().moma_matvec(h, op, x.shape[0], px, py, dt))


def moma_matvec_noalloc(h, op, x, y):
    """Z or Z^H product without any device allocation (device tensors only)."""
    px, dt = _ptr_dtype(x)
    py, dty = _ptr_dtype(y)
    if dt != dty:
        raise TypeError("x and y must have the same dtype")
    _check(lib().moma_matvec_noalloc(h, op, x.shape[0], px, py, dt))


def moma_apply_precond(h, x, y):
    px, dt = _ptr_dtype(x)
    py, _ = _ptr_dtype(y)
    _check(lib().moma_apply_precond(h, x.shape[0], px, py, dt))


def moma_get_bin(h, kx, ky, out):
    p, dt = _ptr_dtype(out)
    _check(lib().moma_get_bin(h, kx, ky, dt, p))


def moma_get_precond_block(h, ex, ey, out):
    p, _ = _ptr_dtype(out)
    _check(lib().moma_get_precond_block(h, ex, ey, p))


def moma_solve(h, V, I, tol=0.0, inner_tol=0.0, max_outer=0, warm_start=False, rel_residual=None, solver=0,
               max_inner=0):
    """Returns the moma_solve_info as a dict; raises MomaError on failure
    (the exception carries .info for MOMA_ERR_NOT_CONVERGED)."""
    pv, dv = _ptr_dtype(V)
    pi, di = _ptr_dtype(I)
    if dv != MOMA_C128 or di != MOMA_C128:
        raise TypeError("V and I are complex128")
    opts = moma_solve_opts(tol, inner_tol, max_outer, 1 if warm_start else 0, solver, max_inner)
    info = moma_solve_info()
    rr = None
    if rel_residual is not None:
        rr = rel_residual.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = lib().moma_solve(h, V.shape[0], pv, pi, ctypes.byref(opts), ctypes.byref(info), rr)
    if st != MOMA_OK:
        e = MomaError(st, lib().moma_last_error().decode())
        e.info = info.as_dict()
        raise e
    return info.as_dict()


def moma_active_impedance(h, I, V, Za, Gamma=None, port_basis=0, z0=50.0):
    pi, _ = _ptr_dtype(I)
    pv, _ = _ptr_dtype(V)
    pz, _ = _ptr_dtype(Za)
    pg = _ptr_dtype(Gamma)[0] if Gamma is not None else None
    _check(lib().moma_active_impedance(h, I.shape[0], pi, pv, port_basis, z0, pz, pg))


def moma_profile(h, enable):
    _check(lib().moma_profile(h, 1 if enable else 0))


def moma_kernel_stats(h, kernel):
    n = ctypes.c_longlong()
    ms = ctypes.c_double()
    kid = KERNEL_IDS[kernel] if isinstance(kernel, str) else kernel
    _check(lib().moma_kernel_stats(h, kid, ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def moma_launch_count(h):
    return lib().moma_launch_count(h)


def moma_device_bytes(h):
    return lib().moma_device_bytes(h)


def moma_destroy(h):
    if h:
        lib().moma_destroy(h)


def moma_last_error():
    return lib().moma_last_error().decode()


def moma_set_stream(h, stream):
    _check(lib().moma_set_stream(h, _stream_handle(stream)))


def moma_time_operator(h, what, nrhs, reps=20):
    """Microseconds per back-to-back application of a c64 operator (MOMA_TIME_*)."""
    us = ctypes.c_double()
    _check(lib().moma_time_operator(h, what, nrhs, reps, ctypes.byref(us)))
    return us.value


def moma_release_setup(h):
    _check(lib().moma_release_setup(h))


def moma_estimate_bytes(nx, ny, b, nrhs, precision=MOMA_PREC_MIXED, with_setup=True):
    opt = moma_options(precision, 0, 0, 0, 0)
    return lib().moma_estimate_bytes(nx, ny, b, ctypes.byref(opt), nrhs, 1 if with_setup else 0)


def moma_server_create(slots=4, max_device_bytes=0, precision=MOMA_PREC_MIXED, restart=0):
    s = ctypes.c_void_p()
    o = moma_server_opts(max_device_bytes, slots, precision, restart)
    _check(lib().moma_server_create(ctypes.byref(o), ctypes.byref(s)))
    return s


def moma_server_submit(s, key, blocks, V, I, Za=None, Gamma=None, port_basis=0, z0=50.0, tol=0.0):
    """Queue a solve; the arrays must stay alive until moma_server_wait returns."""
    pb, dtb = _ptr_dtype(blocks)
    pv, _ = _ptr_dtype(V)
    pi, _ = _ptr_dtype(I)
    ny, nx, b = V.shape[1], V.shape[2], V.shape[3]
    r = moma_request(key, nx, ny, b, pb, dtb, V.shape[0], pv, pi,
                     _ptr_dtype(Za)[0] if Za is not None else None,
                     _ptr_dtype(Gamma)[0] if Gamma is not None else None, port_basis, z0, tol)
    t = ctypes.c_ulonglong()
    _check(lib().moma_server_submit(s, ctypes.byref(r), ctypes.byref(t)))
    return t.value


def moma_server_wait(s, ticket, timeout_s=-1.0):
    out = moma_result()
    _check(lib().moma_server_wait(s, ticket, timeout_s, ctypes.byref(out)))
    return out.as_dict()


def moma_server_get_stats(s):
    out = moma_server_stats()
    _check(lib().moma_server_get_stats(s, ctypes.byref(out)))
    return out.as_dict()


def moma_server_destroy(s):
    if s:
        lib().moma_server_destroy(s)


def moma_tuning_report(h):
    buf = ctypes.create_string_buffer(8192)
    _check(lib().moma_tuning_report(h, buf, len(buf)))
    return buf.value.decode()


def moma_array_stream(h):
    return lib().moma_array_stream(h)


def moma_set_blocks_batch(handles, blocks, release_setup=False, workers=0):
    """Build many arrays concurrently; returns the per-array statuses."""
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.value for h in handles])
    pd = [_ptr_dtype(b) for b in blocks]
    bp = (ctypes.c_void_p * n)(*[p for p, _ in pd])
    dt = (ctypes.c_int * n)(*[d for _, d in pd])
    st = (ctypes.c_int * n)()
    s = lib().moma_set_blocks_batch(n, hs, bp, dt, 1 if release_setup else 0, workers, st)
    if s != MOMA_OK:
        raise MomaError(s, f"batch set_blocks: statuses {list(st)}")
    return list(st)


def moma_solve_batch(handles, Vs, Is, tol=0.0, workers=0, solver=0):
    """Solve many independent problems concurrently; returns the infos."""
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.value for h in handles])
    nr = (ctypes.c_int * n)(*[v.shape[0] for v in Vs])
    vp = (ctypes.c_void_p * n)(*[_ptr_dtype(v)[0] for v in Vs])
    ip = (ctypes.c_void_p * n)(*[_ptr_dtype(x)[0] for x in Is])
    infos = (moma_solve_info * n)()
    st = (ctypes.c_int * n)()
    opts = moma_solve_opts(tol, 0.0, 0, 0, solver, 0)
    s = lib().moma_solve_batch(n, hs, nr, vp, ip, ctypes.byref(opts), infos, workers, st)
    if s != MOMA_OK:
        raise MomaError(s, f"batch solve: statuses {list(st)}")
    return [x.as_dict() for x in infos]


def moma_port_impedance(h, Zp=None, Yp=None, port_basis=0, chunk=0, solver=0, tol=0.0):
    """Passive port impedance matrix (and/or port admittance) [Nel][Nel]."""
    opts = moma_solve_opts(tol, 0.0, 0, 0, solver, 0)
    pz = _ptr_dtype(Zp)[0] if Zp is not None else None
    py = _ptr_dtype(Yp)[0] if Yp is not None else None
    _check(lib().moma_port_impedance(h, port_basis, chunk, ctypes.byref(opts), pz, py))


def moma_column_coupling(h, nq, nmax, C, gamma=None, port_basis=0, z0=50.0, solver=0, tol=0.0):
    """Column coupling C_n, n = -nmax..nmax, from an nq-sample phase sweep."""
    opts = moma_solve_opts(tol, 0.0, 0, 0, solver, 0)
    pg = _ptr_dtype(gamma)[0] if gamma is not None else None
    _check(lib().moma_column_coupling(h, port_basis, nq, nmax, z0, ctypes.byref(opts), _ptr_dtype(C)[0], pg))


def moma_s_to_z(S, Zp, z0=50.0, stream=None):
    _check(lib().moma_s_to_z(_ptr_dtype(S)[0], S.shape[0], z0, _ptr_dtype(Zp)[0], _stream_handle(stream)))


def moma_s_ideal(nx, ny, s_cc, s1, kd, S, stream=None):
    _check(lib().moma_s_ideal(nx, ny, s_cc.real, s_cc.imag, s1.real, s1.imag, kd, _ptr_dtype(S)[0],
                              _stream_handle(stream)))


def moma_xi_z(Zp, nx, ny):
    """(xi_Z predictor (Eq. 25), xi_Z max (Eq. 24), border bound (Eq. 23))."""
    out = (ctypes.c_double * 3)()
    _check(lib().moma_xi_z(_ptr_dtype(Zp)[0], nx, ny, out))
    return tuple(out)


def moma_xi_s(nx, ny, s_cc, s1, kd, z0=50.0):
    out = ctypes.c_double()
    _check(lib().moma_xi_s(nx, ny, s_cc.real, s_cc.imag, s1.real, s1.imag, kd, z0, ctypes.byref(out)))
    return out.value


def moma_set_margin(h, ZB, ZC):
    """Margin blocks Z_B [nm][N], Z_C [nm][nm] (same dtype); ZB=None removes the margin."""
    if ZB is None:
        _check(lib().moma_set_margin(h, 0, None, None, MOMA_C128))
        return
    pb, db = _ptr_dtype(ZB)
    pc, dc = _ptr_dtype(ZC)
    if db != dc:
        raise TypeError("ZB and ZC must have the same dtype")
    _check(lib().moma_set_margin(h, ZB.shape[0], pb, pc, db))
