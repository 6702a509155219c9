"""Python binding of the GB300 initial-guess / SEM / Jacobi-PCG library.

Thin ctypes layer over the C ABI in ``include/sg.h``: it marshals PyTorch
tensors (device memory) and the current CUDA stream into the library calls.
Every step of the computation runs in the library's CUDA kernels; there is no
CPU or PyTorch fallback, and loading fails loudly if ``libsg.so`` is missing.

Method: Austin, Chalmers & Warburton, "Initial Guesses for Sequences of Linear
Systems in a GPU-Accelerated Incompressible Flow Solver" (arXiv:2009.10863).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsg.so")

F64, F32 = 0, 1
ZERO, LAST, EXTRAP, PROJ_QR, PROJ_CLASSIC, SPEXTRAP, PROJ_ENERGY = 0, 1, 2, 3, 4, 5, 6
STOP_REL_B, STOP_INITRESID, STOP_RHS = 0, 1, 2
OK, NOT_CONVERGED = 0, 1
ERR_INVALID, ERR_CUDA, ERR_BREAKDOWN, ERR_TIMEOUT, ERR_STATE = -1, -2, -3, -4, -5
BATCH_MAX = 4
MAX_HISTORY, MAX_DEGREE = 16, 8
NOALLOC_MAX_NODES, NOALLOC_SCRATCH_BYTES = 131072, 6815744
PROF_SEM, PROF_PCG_APPLY, PROF_PCG_UPDATE, PROF_EXTRAP = 0, 1, 2, 3
PROF_PROJ_DOTS, PROF_PROJ_LINCOMB, PROF_PROJ_UPDATE = 4, 5, 6

METHOD_NAMES = {"zero": ZERO, "last": LAST, "extrap": EXTRAP, "qr": PROJ_QR,
                "classic": PROJ_CLASSIC, "spextrap": SPEXTRAP, "energy": PROJ_ENERGY}

# (name, restype, argtypes) of every exported entry point
_VP, _I, _D, _I64, _SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_size_t
SIGNATURES = [
    ("sg_version", _I, []),
    ("sg_last_error", ctypes.c_char_p, []),
    ("sg_op_create", _I, [ctypes.POINTER(_VP), _I, _I, _I, _I, _D, _I]),
    ("sg_op_destroy", _I, [_VP]),
    ("sg_op_size", _I64, [_VP]),
    ("sg_op_gll", _I, [_VP, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    ("sg_op_set_layers", _I, [_VP, _I]),
    ("sg_sem_apply", _I, [_VP, _VP, _VP, _VP]),
    ("sg_op_diagonal", _I, [_VP, _VP, _VP]),
    ("sg_pcg_workspace_bytes", _SZ, [_VP]),
    ("sg_residual_norm", _I, [_VP, _VP, _VP, _VP, ctypes.POINTER(_D), _VP]),
    ("sg_pcg_solve", _I, [_VP, _VP, _VP, _D, _I, _I, _VP, ctypes.POINTER(_I), ctypes.POINTER(_D), _VP]),
    ("sg_pcg_solve_async", _I, [_VP, _VP, _VP, _D, _I, _I, _VP, _VP]),
    ("sg_pcg_result", _I, [_VP, _VP, ctypes.POINTER(_I), _VP]),
    ("sg_guess_workspace_bytes", _SZ, [_I64, _I, _I, _I]),
    ("sg_guess_create", _I, [ctypes.POINTER(_VP), _I64, _I, _I, _I, _D, _VP, _VP, _I]),
    ("sg_guess_destroy", _I, [_VP]),
    ("sg_guess_form", _I, [_VP, _VP, _VP, _VP]),
    ("sg_guess_next_slot", _VP, [_VP]),
    ("sg_guess_update", _I, [_VP, _VP, _VP, _VP]),
    ("sg_guess_info", _I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_D), _VP]),
    ("sg_guess_image_bytes", _SZ, [_VP]),
    ("sg_guess_export", _I, [_VP, _VP, _VP]),
    ("sg_guess_import", _I, [_VP, _VP, _SZ, _VP]),
    ("sg_profile_enable", _I, [_I]),
    ("sg_profile_read", _I, [_I, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong)]),
    ("sg_profile_reset", _I, []),
    ("sg_launch_count", ctypes.c_longlong, []),
    ("sg_convert", _I, [_VP, _I, _VP, _I, _I64, _VP]),
    ("sg_ir_workspace_bytes", _SZ, [_VP, _VP]),
    ("sg_ir_solve", _I, [_VP, _VP, _VP, _VP, _D, _D, _I, _I, _VP, ctypes.POINTER(_I), ctypes.POINTER(_I),
                         ctypes.POINTER(_D), _VP]),
    ("sg_ir_solve_ru", _I, [_VP, _VP, _VP, _VP, _D, _D, _I, _I, _VP, ctypes.POINTER(_I), ctypes.POINTER(_I),
                            ctypes.POINTER(_D), _VP]),
    ("sg_batch_workspace_bytes", _SZ, [_I, ctypes.POINTER(_VP), ctypes.POINTER(_VP)]),
    ("sg_batch_create", _I, [ctypes.POINTER(_VP), _I, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _VP]),
    ("sg_batch_destroy", _I, [_VP]),
    ("sg_batch_tune", _I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_D), _VP]),
    ("sg_batch_ir_solve", _I, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _D, _D, _I, _I,
                               ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_D), _VP]),
    ("sg_seq_workspace_bytes", _SZ, [_VP]),
    ("sg_mass_rhs", _I, [_VP, _D, _VP, _VP, _VP, _VP]),
    ("sg_adjoint_rhs", _I, [_VP, _D, _VP, _VP, _D, _VP, _VP, _VP]),
    ("sg_adjoint_accum", _I, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    ("sg_sqdiff_accum", _I, [_VP, _VP, _VP, _VP, _VP, _VP]),
    ("sg_selftest_barrier", _I, [_I, ctypes.c_longlong, _VP, _VP]),
    ("sg_pcg_solve_noalloc", _I, [_VP, _VP, _VP, _D, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_D), _VP]),
]

_lib = None


class SGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("sg error %d: %s" % (code, msg))
        self.code = code


def lib():
    """Load libsg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsg.so not found at %s: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        _lib = L
    return _lib


def _check(rc, allow=(OK,)):
    if rc in allow:
        return rc
    raise SGError(rc, lib().sg_last_error().decode())


def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _dtype_code(dtype):
    torch = _torch()
    if dtype in (torch.float64, "f64", F64):
        return F64
    if dtype in (torch.float32, "f32", F32):
        return F32
    raise ValueError("dtype must be float64 or float32")


def _torch_dtype(code):
    torch = _torch()
    return torch.float64 if code == F64 else torch.float32


class Op:
    """Matrix-free GLL SEM operator A = K + lam M on the unit box (Sec. 5.1)."""

    def __init__(self, ex, ey, ez, p, lam=0.0, dtype="f64"):
        self.code = _dtype_code(dtype)
        self.dtype = _torch_dtype(self.code)
        h = ctypes.c_void_p()
        _check(lib().sg_op_create(ctypes.byref(h), int(ex), int(ey), int(ez), int(p), float(lam), self.code))
        self.h = h
        self.ex, self.ey, self.ez, self.p, self.lam = int(ex), int(ey), int(ez), int(p), float(lam)
        self.nx, self.ny, self.nz = p * ex + 1, p * ey + 1, p * ez + 1
        self.n = int(lib().sg_op_size(self.h))
        self._pcg_ws = None

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.sg_op_destroy(self.h)
            self.h = None

    def set_layers(self, zl):
        """Element layers per CTA of the operator kernel (0 = automatic)."""
        _check(lib().sg_op_set_layers(self.h, int(zl)))

    def gll(self):
        x = (ctypes.c_double * (self.p + 1))()
        w = (ctypes.c_double * (self.p + 1))()
        _check(lib().sg_op_gll(self.h, x, w))
        return np.array(x[:]), np.array(w[:])

    def coords_1d(self):
        """Global node coordinates per axis (GLL nodes mapped to each element)."""
        xi, _ = self.gll()
        out = []
        for ne in (self.ex, self.ey, self.ez):
            h = 1.0 / ne
            c = np.empty(self.p * ne + 1)
            for e in range(ne):
                c[e * self.p:(e + 1) * self.p + 1] = e * h + 0.5 * (xi + 1.0) * h
            out.append(c)
        return out

    def empty(self):
        torch = _torch()
        return torch.empty(self.n, dtype=self.dtype, device="cuda")

    def zeros(self):
        torch = _torch()
        return torch.zeros(self.n, dtype=self.dtype, device="cuda")

    def _vec(self, t, name):
        if t.dtype != self.dtype or not t.is_cuda or not t.is_contiguous() or t.numel() != self.n:
            raise ValueError("%s must be a contiguous CUDA %s tensor of %d elements" % (name, self.dtype, self.n))
        return t

    def apply(self, x, out=None):
        """out = A x."""
        self._vec(x, "x")
        out = self.empty() if out is None else self._vec(out, "out")
        _check(lib().sg_sem_apply(self.h, _ptr(x), _ptr(out), _stream()))
        return out

    def diagonal(self):
        out = self.empty()
        _check(lib().sg_op_diagonal(self.h, _ptr(out), _stream()))
        return out

    def pcg_workspace(self):
        if self._pcg_ws is None:
            torch = _torch()
            nb = int(lib().sg_pcg_workspace_bytes(self.h))
            self._pcg_ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        return self._pcg_ws

    def pcg(self, b, x, tol, maxit=10000, criterion=STOP_REL_B, raise_on_maxit=False, true_residual=True):
        """Solve A x = b in place (x: initial guess in, solution out).
        Returns (iterations, true relative residual or None)."""
        self._vec(b, "b")
        self._vec(x, "x")
        ws = self.pcg_workspace()
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        allow = (OK,) if raise_on_maxit else (OK, NOT_CONVERGED)
        _check(lib().sg_pcg_solve(self.h, _ptr(b), _ptr(x), float(tol), int(maxit), int(criterion),
                                  _ptr(ws), ctypes.byref(it), ctypes.byref(rr) if true_residual else None,
                                  _stream()), allow)
        return it.value, (rr.value if true_residual else None)

    def pcg_async(self, b, x, tol, maxit=10000, criterion=STOP_REL_B):
        """Enqueue the solve of A x = b on the current stream without waiting;
        read the outcome with ``pcg_result`` before the next solve."""
        self._vec(b, "b")
        self._vec(x, "x")
        _check(lib().sg_pcg_solve_async(self.h, _ptr(b), _ptr(x), float(tol), int(maxit), int(criterion),
                                        _ptr(self.pcg_workspace()), _stream()))

    def pcg_result(self, raise_on_maxit=False):
        """Iteration count of the last solve (waits for it)."""
        it = ctypes.c_int(0)
        allow = (OK,) if raise_on_maxit else (OK, NOT_CONVERGED)
        _check(lib().sg_pcg_result(self.h, _ptr(self.pcg_workspace()), ctypes.byref(it), _stream()), allow)
        return it.value

    def residual_norm(self, b, x):
        """||b - A x|| / ||b|| (synchronises)."""
        self._vec(b, "b")
        self._vec(x, "x")
        rr = ctypes.c_double(0.0)
        _check(lib().sg_residual_norm(self.h, _ptr(b), _ptr(x), _ptr(self.pcg_workspace()), ctypes.byref(rr),
                                      _stream()))
        return rr.value


class Guess:
    """Initial-guess history: ZERO, LAST, EXTRAP(m, s), SPEXTRAP(m, s),
    QR(s) (Algorithm 2), CLASSIC(s) (Algorithm 1) or ENERGY(s) (the QR(s)
    window in the energy inner product)."""

    def __init__(self, n, s, method, m=-1, eps_rel=1e-10, op=None, dtype="f64"):
        torch = _torch()
        if isinstance(method, str):
            method = METHOD_NAMES[method]
        self.code = _dtype_code(dtype)
        self.dtype = _torch_dtype(self.code)
        self.n, self.s, self.method = int(n), int(s), int(method)
        nb = int(lib().sg_guess_workspace_bytes(self.n, self.s, self.method, self.code))
        if nb == 0:
            raise ValueError("invalid guess parameters")
        self.ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        self.op = op
        h = ctypes.c_void_p()
        torch.cuda.synchronize()
        _check(lib().sg_guess_create(ctypes.byref(h), self.n, self.s, self.method, int(m), float(eps_rel),
                                     op.h if op is not None else None, _ptr(self.ws), self.code))
        torch.cuda.synchronize()
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.sg_guess_destroy(self.h)
            self.h = None

    def form(self, b, x0):
        """Write the initial guess for right-hand side b into x0 (in place)."""
        _check(lib().sg_guess_form(self.h, _ptr(b) if b is not None else None, _ptr(x0), _stream()))
        return x0

    def next_slot(self):
        """Ring slot of the next solution as a tensor view (EXTRAP family), else None."""
        p = lib().sg_guess_next_slot(self.h)
        if not p:
            return None
        base = self.ws.data_ptr()
        es = 8 if self.code == F64 else 4
        off = p - base
        return self.ws[off:off + es * self.n].view(self.dtype)

    def update(self, x, b=None):
        _check(lib().sg_guess_update(self.h, _ptr(x), _ptr(b) if b is not None else None, _stream()))

    def export(self):
        """Host image of the history (numpy uint8 array) -- synchronises."""
        img = np.empty(int(lib().sg_guess_image_bytes(self.h)), dtype=np.uint8)
        _check(lib().sg_guess_export(self.h, img.ctypes.data_as(ctypes.c_void_p), _stream()))
        return img

    def restore(self, image):
        """Load a history exported by a handle with the same parameters."""
        img = np.ascontiguousarray(image, dtype=np.uint8).reshape(-1)
        _check(lib().sg_guess_import(self.h, img.ctypes.data_as(ctypes.c_void_p), img.size, _stream()))

    def info(self):
        """(d, R or beta as an s x s / s array) -- synchronises."""
        d = ctypes.c_int(0)
        buf = (ctypes.c_double * (self.s * self.s))()
        _check(lib().sg_guess_info(self.h, ctypes.byref(d), buf, _stream()))
        arr = np.array(buf[:])
        if self.method in (PROJ_QR, PROJ_CLASSIC, PROJ_ENERGY):
            return d.value, arr.reshape(self.s, self.s)
        return d.value, arr[:self.s]


def convert(src, dst):
    """dst = src converted between float64 and float32 (device tensors, same size)."""
    if src.numel() != dst.numel():
        raise ValueError("size mismatch")
    _check(lib().sg_convert(_ptr(src), _dtype_code(src.dtype), _ptr(dst), _dtype_code(dst.dtype),
                            src.numel(), _stream()))
    return dst


class MixedSolver:
    """FP32 operator + FP32 Jacobi-PCG inside FP64 iterative refinement."""

    def __init__(self, ex, ey, ez, p, lam=0.0):
        torch = _torch()
        self.op64 = Op(ex, ey, ez, p, lam, "f64")
        self.op32 = Op(ex, ey, ez, p, lam, "f32")
        self.n = self.op64.n
        nb = int(lib().sg_ir_workspace_bytes(self.op64.h, self.op32.h))
        self.ws = torch.empty(nb, dtype=torch.uint8, device="cuda")

    def solve(self, b, x, tol, inner_tol=None, max_outer=30, maxit_inner=10000, method="restart"):
        """Solve in place; returns (outer steps or FP64 updates, total inner FP32
        iterations, FP64 relres).  method "restart": refinement with an FP32 PCG
        solve from zero per outer step to inner_tol (default 1e-4; sg_ir_solve);
        "replace": one FP32 PCG with its residual replaced by the FP64 one each
        time it has dropped by inner_tol (default 0.1; sg_ir_solve_ru)."""
        if inner_tol is None:
            inner_tol = 1e-4 if method == "restart" else 0.1
        self.op64._vec(b, "b")
        self.op64._vec(x, "x")
        oi, ii, rr = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
        if method == "restart":
            fn = lib().sg_ir_solve
        elif method == "replace":
            fn = lib().sg_ir_solve_ru
        else:
            raise ValueError("method must be 'restart' or 'replace'")
        _check(fn(self.op64.h, self.op32.h, _ptr(b), _ptr(x), float(tol), float(inner_tol), int(max_outer),
                  int(maxit_inner), _ptr(self.ws), ctypes.byref(oi), ctypes.byref(ii), ctypes.byref(rr),
                  _stream()), (OK, NOT_CONVERGED))
        return oi.value, ii.value, rr.value


class BatchSolver:
    """Up to BATCH_MAX systems (p = 7, own mesh and lambda each) solved together:
    one persistent launch per FP32 CG iteration inside FP64 refinement."""

    def __init__(self, meshes):
        """meshes: list of (ex, ey, ez, lam)."""
        torch = _torch()
        self.ops64 = [Op(ex, ey, ez, 7, lam, "f64") for ex, ey, ez, lam in meshes]
        self.ops32 = [Op(ex, ey, ez, 7, lam, "f32") for ex, ey, ez, lam in meshes]
        k = len(meshes)
        self.k = k
        a64 = (ctypes.c_void_p * k)(*[o.h.value for o in self.ops64])
        a32 = (ctypes.c_void_p * k)(*[o.h.value for o in self.ops32])
        nb = int(lib().sg_batch_workspace_bytes(k, a64, a32))
        if nb == 0:
            raise ValueError("invalid batch")
        self.ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        h = ctypes.c_void_p()
        _check(lib().sg_batch_create(ctypes.byref(h), k, a64, a32, _ptr(self.ws)))
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.sg_batch_destroy(self.h)
            self.h = None

    def tune(self):
        zl, bps, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
        _check(lib().sg_batch_tune(self.h, ctypes.byref(zl), ctypes.byref(bps), ctypes.byref(ms), _stream()))
        return zl.value, bps.value, ms.value

    def solve(self, bs, xs, tol, inner_tol=1e-4, max_outer=30, maxit_inner=10000):
        """Solve every system in place.  Returns (outer, inner, relres) lists."""
        k = self.k
        for o, b, x in zip(self.ops64, bs, xs):
            o._vec(b, "b")
            o._vec(x, "x")
        bp = (ctypes.c_void_p * k)(*[b.data_ptr() for b in bs])
        xp = (ctypes.c_void_p * k)(*[x.data_ptr() for x in xs])
        oi, ii, rr = (ctypes.c_int * k)(), (ctypes.c_int * k)(), (ctypes.c_double * k)()
        _check(lib().sg_batch_ir_solve(self.h, bp, xp, float(tol), float(inner_tol), int(max_outer),
                                       int(maxit_inner), oi, ii, rr, _stream()), (OK, NOT_CONVERGED))
        return list(oi), list(ii), list(rr)


def profile_enable(on=True):
    _check(lib().sg_profile_enable(1 if on else 0))


def profile_reset():
    _check(lib().sg_profile_reset())


def profile_read(kernel_id):
    ms = ctypes.c_double(0.0)
    cnt = ctypes.c_longlong(0)
    _check(lib().sg_profile_read(int(kernel_id), ctypes.byref(ms), ctypes.byref(cnt)))
    return ms.value, cnt.value


def launch_count():
    """Kernels launched by the library so far in this process."""
    return int(lib().sg_launch_count())
