"""Thin ctypes binding of libiga (include/iga.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Functions keep the C names; ``Discretization`` bundles a handle with
its host-side arrays and takes torch CUDA tensors for device buffers.  There is
no fallback: if libiga.so is missing, ``lib()`` raises.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libiga.so")

IGA_OK, IGA_EINVAL, IGA_ENOMEM, IGA_ECUDA, IGA_ENOCONV, IGA_EDIVERGED, IGA_ETIMEOUT, IGA_ENAN = range(8)
STATUS_NAMES = ["IGA_OK", "IGA_EINVAL", "IGA_ENOMEM", "IGA_ECUDA", "IGA_ENOCONV", "IGA_EDIVERGED", "IGA_ETIMEOUT", "IGA_ENAN"]
IGA_FP64, IGA_JAC_TF32, IGA_JAC_BF16, IGA_JAC_FP32, IGA_JAC_NONE, IGA_JAC_FD = 0, 1, 2, 3, 4, 5

# every symbol include/iga.h declares
EXPORTS = ["iga_create", "iga_set_boundary_value", "iga_set_lambda", "iga_get_pattern", "iga_form_residual",
           "iga_form_jacobian", "iga_newton_defaults", "iga_solve_newton", "iga_solve_newton_host", "iga_destroy",
           "iga_last_error", "iga_profile_enable", "iga_profile_read", "iga_form_residual_noalloc",
           "iga_batch_create", "iga_batch_offsets", "iga_batch_set_launch", "iga_batch_solve", "iga_batch_destroy",
           "iga_batch_last_error", "iga_nn_create", "iga_nn_num_params", "iga_nn_get_params", "iga_nn_set_params",
           "iga_nn_forward", "iga_nn_loss_grad", "iga_nn_adam_step", "iga_nn_destroy", "iga_nn_last_error",
           "iga_nn_set_h1_weight", "iga_apply_jacobian", "iga_apply_jacobian_mf", "iga_form_jacobian_diagonal",
           "iga_form_residual_ts", "iga_form_jacobian_ts", "iga_ts_alpha_step", "iga_measure_peaks",
           "iga_set_wait_limit", "iga_inject_stall", "iga_batch_set_tiles", "iga_exp_eval",
           "iga_set_gmres_fused", "iga_set_jacobian_plan"]

KERNEL_CLASSES = ["geometry", "residual_element", "residual_gather", "q00", "jac_stage1", "jac_stage2", "jac_final",
                  "spmv", "gs_orth", "gmres_scalar", "vector", "combine", "pattern", "elem_tc", "elem_gather",
                  "residual_spmv"]


class IgaDesc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("degree", ctypes.c_int * 3),
        ("nel", ctypes.c_int * 3),
        ("continuity", ctypes.c_int * 3),
        ("knots", ctypes.c_void_p * 3),
        ("nknots", ctypes.c_int * 3),
        ("quad", ctypes.c_int * 3),
        ("ctrl", ctypes.c_void_p),
        ("weights", ctypes.c_void_p),
        ("periodic", ctypes.c_int * 3),
    ]


class IgaBratu(ctypes.Structure):
    _fields_ = [("lam", ctypes.c_double), ("log_kappa", ctypes.c_void_p)]


class IgaNewtonOpts(ctypes.Structure):
    _fields_ = [
        ("atol", ctypes.c_double),
        ("max_newton", ctypes.c_int),
        ("gmres_restart", ctypes.c_int),
        ("max_krylov", ctypes.c_int),
        ("krylov_rtol", ctypes.c_double),
        ("jac", ctypes.c_int),
        ("reuse_stiffness", ctypes.c_int),
        ("ksp", ctypes.c_int),
        ("gmres_cgs_refine", ctypes.c_int),
    ]


IGA_KSP_GMRES, IGA_KSP_CG = 0, 1
IGA_CGS_REFINE_NEVER, IGA_CGS_REFINE_IFNEEDED, IGA_CGS_REFINE_ALWAYS = 0, 1, 2


class IgaNewtonReport(ctypes.Structure):
    _fields_ = [
        ("newton_its", ctypes.c_int),
        ("krylov_its", ctypes.c_int),
        ("fnorm0", ctypes.c_double),
        ("fnorm", ctypes.c_double),
        ("fnorm_hist", ctypes.c_double * 64),
        ("status", ctypes.c_int),
    ]


class IgaTsOpts(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("rho_inf", ctypes.c_double)]


class IgaPeaks(ctypes.Structure):
    _fields_ = [("fp64_tflops", ctypes.c_double), ("fp32_tflops", ctypes.c_double), ("copy_gbs", ctypes.c_double),
                ("sms", ctypes.c_int)]


class IgaProfile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 16), ("timed", ctypes.c_longlong * 16), ("launches", ctypes.c_longlong * 16)]


_lib = None


def lib():
    """Load libiga.so (build it first with paper_1305_4452_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libiga.so is not built (%s); run paper_1305_4452_gb300.build.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
        L.iga_create.argtypes = [ctypes.POINTER(IgaDesc), ctypes.POINTER(IgaBratu), vp, ctypes.POINTER(vp)]
        L.iga_create.restype = ctypes.c_int
        L.iga_set_boundary_value.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double]
        L.iga_set_lambda.argtypes = [vp, ctypes.c_double]
        L.iga_get_pattern.argtypes = [vp, i64p, i64p, ctypes.POINTER(vp), ctypes.POINTER(vp)]
        L.iga_form_residual.argtypes = [vp, vp, vp]
        L.iga_form_jacobian.argtypes = [vp, vp, vp, ctypes.c_int]
        L.iga_apply_jacobian.argtypes = [vp, vp, ctypes.c_int, vp, vp]
        L.iga_apply_jacobian_mf.argtypes = [vp, vp, vp, vp]
        L.iga_form_jacobian_diagonal.argtypes = [vp, vp, vp]
        L.iga_form_residual_noalloc.argtypes = [vp, vp, vp]
        L.iga_newton_defaults.argtypes = [ctypes.POINTER(IgaNewtonOpts)]
        L.iga_newton_defaults.restype = None
        L.iga_solve_newton.argtypes = [vp, vp, ctypes.POINTER(IgaNewtonOpts), ctypes.POINTER(IgaNewtonReport)]
        L.iga_solve_newton_host.argtypes = [vp, vp, ctypes.POINTER(IgaNewtonOpts), ctypes.POINTER(IgaNewtonReport)]
        L.iga_form_residual_ts.argtypes = [vp, vp, vp, vp]
        L.iga_form_jacobian_ts.argtypes = [vp, ctypes.c_double, vp, vp, ctypes.c_int]
        L.iga_ts_alpha_step.argtypes = [vp, ctypes.POINTER(IgaTsOpts), vp, vp, ctypes.POINTER(IgaNewtonOpts),
                                        ctypes.POINTER(IgaNewtonReport)]
        L.iga_destroy.argtypes = [vp]
        L.iga_destroy.restype = None
        L.iga_last_error.argtypes = [vp]
        L.iga_last_error.restype = ctypes.c_char_p
        L.iga_profile_enable.argtypes = [vp, ctypes.c_uint]
        L.iga_profile_read.argtypes = [vp, ctypes.POINTER(IgaProfile)]
        L.iga_measure_peaks.argtypes = [vp, ctypes.POINTER(IgaPeaks)]
        L.iga_set_wait_limit.argtypes = [vp, ctypes.c_double]
        L.iga_inject_stall.argtypes = [vp]
        L.iga_set_gmres_fused.argtypes = [vp, ctypes.c_int]
        L.iga_set_jacobian_plan.argtypes = [vp, ctypes.c_int]
        L.iga_exp_eval.argtypes = [vp, vp, vp, ctypes.c_int64]
        _lib = L
    return _lib


class IgaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 8 else status, msg))
        self.status = status


def _check(rc, handle=None):
    if rc != IGA_OK:
        raise IgaError(rc, lib().iga_last_error(handle).decode())
    return rc


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def newton_defaults():
    o = IgaNewtonOpts()
    lib().iga_newton_defaults(ctypes.byref(o))
    return o


def exp_eval(x, y=None, stream=None):
    """y = e^x (device FP64 tensors) with the library's Gauss-point exponential."""
    import torch
    if y is None:
        y = torch.empty_like(x)
    assert x.is_cuda and x.dtype == torch.float64 and x.is_contiguous() and y.shape == x.shape
    _check(lib().iga_exp_eval(ctypes.c_void_p(_stream_ptr(stream)), ctypes.c_void_p(x.data_ptr()),
                              ctypes.c_void_p(y.data_ptr()), x.numel()))
    return y


def measure_peaks(stream=None):
    """iga_measure_peaks on the current device: FP64 and FP32 FMA rates (TFLOP/s) and
    the device-to-device copy bandwidth (GB/s)."""
    p = IgaPeaks()
    _check(lib().iga_measure_peaks(ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(p)))
    return {"fp64_tflops": p.fp64_tflops, "fp32_tflops": p.fp32_tflops, "copy_gbs": p.copy_gbs, "sms": p.sms}


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(stream)


class Discretization:
    """An iga_t handle: a scalar Bratu problem on a tensor-product NURBS space.

    knots: per-direction knot vectors (None: uniform from nel/continuity);
    ctrl (N, dim) / weights (N,) / log_kappa (N,) host arrays or None;
    periodic: {axis: k}, C^k periodic directions (Sec. 2.4; open knots unclamped by
    the library, N counting the wrapped functions).
    """

    def __init__(self, dim, degree, nel=None, continuity=None, knots=None, ctrl=None, weights=None, lam=1.0,
                 log_kappa=None, dirichlet=None, stream=None, periodic=None):
        d = IgaDesc()
        d.dim = dim
        self._keep = []
        for ax, k in (periodic or {}).items():
            d.periodic[ax] = int(k) + 1
        for ax in range(dim):
            d.degree[ax] = degree if np.isscalar(degree) else degree[ax]
            d.continuity[ax] = -1 if continuity is None else (continuity if np.isscalar(continuity) else continuity[ax])
            if knots is not None and knots[ax] is not None:
                k = _f64(knots[ax])
                self._keep.append(k)
                d.knots[ax] = k.ctypes.data
                d.nknots[ax] = len(k)
            else:
                d.nel[ax] = nel if np.isscalar(nel) else nel[ax]
        ctrl, weights, log_kappa = _f64(ctrl), _f64(weights), _f64(log_kappa)
        self._keep += [a for a in (ctrl, weights, log_kappa) if a is not None]
        d.ctrl = None if ctrl is None else ctrl.ctypes.data
        d.weights = None if weights is None else weights.ctypes.data
        b = IgaBratu(float(lam), None if log_kappa is None else log_kappa.ctypes.data)
        h = ctypes.c_void_p()
        self.stream = _stream_ptr(stream)
        _check(lib().iga_create(ctypes.byref(d), ctypes.byref(b), ctypes.c_void_p(self.stream), ctypes.byref(h)))
        self.h = h
        self.dim = dim
        for (ax, side), v in (dirichlet or {}).items():
            _check(lib().iga_set_boundary_value(self.h, ax, side, float(v)), self.h)
        n = ctypes.c_int64()
        nnz = ctypes.c_int64()
        rp = ctypes.c_void_p()
        ci = ctypes.c_void_p()
        _check(lib().iga_get_pattern(self.h, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(rp), ctypes.byref(ci)), self.h)
        self.N, self.nnz = n.value, nnz.value
        self.rowptr_ptr, self.colidx_ptr = rp.value, ci.value

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().iga_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def profile_enable(self, classes=()):
        """Time the named kernel classes (see KERNEL_CLASSES) with CUDA events."""
        mask = 0
        for c in classes:
            mask |= 1 << KERNEL_CLASSES.index(c)
        _check(lib().iga_profile_enable(self.h, mask), self.h)

    def profile_read(self):
        """{class: (ms, timed launches, all launches)} since the last read."""
        p = IgaProfile()
        _check(lib().iga_profile_read(self.h, ctypes.byref(p)), self.h)
        return {c: (p.ms[i], p.timed[i], p.launches[i]) for i, c in enumerate(KERNEL_CLASSES)}

    def set_lambda(self, lam):
        _check(lib().iga_set_lambda(self.h, float(lam)), self.h)

    def set_gmres_fused(self, fused):
        _check(lib().iga_set_gmres_fused(self.h, int(fused)), self.h)

    def set_jacobian_plan(self, general):
        _check(lib().iga_set_jacobian_plan(self.h, int(general)), self.h)

    def pattern(self):
        """Copy the device CSR pattern into torch tensors (rowptr int64, colidx int32)."""
        import torch
        rp = torch.empty(self.N + 1, dtype=torch.int64, device="cuda")
        ci = torch.empty(self.nnz, dtype=torch.int32, device="cuda")
        rp.copy_(_wrap_device(self.rowptr_ptr, self.N + 1, torch.int64))
        ci.copy_(_wrap_device(self.colidx_ptr, self.nnz, torch.int32))
        return rp, ci

    def form_residual(self, U, F=None):
        import torch
        if F is None:
            F = torch.empty_like(U)
        _check(lib().iga_form_residual(self.h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(F.data_ptr())), self.h)
        return F

    def form_jacobian(self, U, prec=IGA_FP64, vals=None):
        import torch
        if vals is None:
            vals = torch.empty(self.nnz, dtype=torch.float64 if prec in (IGA_FP64, IGA_JAC_FD) else torch.float32,
                               device=U.device)
        _check(lib().iga_form_jacobian(self.h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(vals.data_ptr()), int(prec)), self.h)
        return vals

    def apply_jacobian(self, vals, x, y=None, prec=None):
        """y = J x for CSR values `vals` on the library's pattern (FP64 or FP32 values)."""
        import torch
        if prec is None:
            prec = IGA_FP64 if vals.dtype == torch.float64 else IGA_JAC_FP32
        if y is None:
            y = torch.empty_like(x)
        _check(lib().iga_apply_jacobian(self.h, ctypes.c_void_p(vals.data_ptr()), int(prec), ctypes.c_void_p(x.data_ptr()),
                                        ctypes.c_void_p(y.data_ptr())), self.h)
        return y

    def apply_jacobian_mf(self, U, x, y=None):
        """y = J(U) x without assembling J (matrix-free)."""
        import torch
        if y is None:
            y = torch.empty_like(x)
        _check(lib().iga_apply_jacobian_mf(self.h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                           ctypes.c_void_p(y.data_ptr())), self.h)
        return y

    def jacobian_diagonal(self, U, d=None):
        """diag(J(U)) without assembling J (1 on Dirichlet rows)."""
        import torch
        if d is None:
            d = torch.empty_like(U)
        _check(lib().iga_form_jacobian_diagonal(self.h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(d.data_ptr())), self.h)
        return d

    def solve_newton(self, U, opts=None, check=True):
        o = opts if opts is not None else newton_defaults()
        r = IgaNewtonReport()
        rc = lib().iga_solve_newton(self.h, ctypes.c_void_p(U.data_ptr()), ctypes.byref(o), ctypes.byref(r))
        if check and rc not in (IGA_OK,):
            raise IgaError(rc, lib().iga_last_error(self.h).decode())
        return r

    def form_residual_ts(self, V, U, F=None):
        """R(V, U) of the time-dependent problem, V the rates U-dot (Sec. 4.2)."""
        import torch
        if F is None:
            F = torch.empty_like(U)
        _check(lib().iga_form_residual_ts(self.h, ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(U.data_ptr()),
                                          ctypes.c_void_p(F.data_ptr())), self.h)
        return F

    def form_jacobian_ts(self, shift, U, prec=IGA_FP64, vals=None):
        """dR/dU + shift dR/dU-dot at U (FP64 or FP32 values on the pattern)."""
        import torch
        if vals is None:
            vals = torch.empty(self.nnz, dtype=torch.float64 if prec == IGA_FP64 else torch.float32, device=U.device)
        _check(lib().iga_form_jacobian_ts(self.h, float(shift), ctypes.c_void_p(U.data_ptr()),
                                          ctypes.c_void_p(vals.data_ptr()), int(prec)), self.h)
        return vals

    def ts_alpha_step(self, U, V, dt, rho_inf=0.5, opts=None, check=True):
        """One generalized-alpha step (Sec. 4.2): U = U_n, V = U-dot_n in, U_{n+1} and
        U-dot_{n+1} out (in place)."""
        o = opts if opts is not None else newton_defaults()
        t = IgaTsOpts(float(dt), float(rho_inf))
        r = IgaNewtonReport()
        rc = lib().iga_ts_alpha_step(self.h, ctypes.byref(t), ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(V.data_ptr()),
                                     ctypes.byref(o), ctypes.byref(r))
        if check and rc != IGA_OK:
            raise IgaError(rc, lib().iga_last_error(self.h).decode())
        return r

    def solve_newton_host(self, U_host, opts=None, check=True):
        """U_host: numpy float64 array (ideally in pinned memory), updated in place."""
        o = opts if opts is not None else newton_defaults()
        r = IgaNewtonReport()
        rc = lib().iga_solve_newton_host(self.h, ctypes.c_void_p(U_host.ctypes.data if isinstance(U_host, np.ndarray) else U_host.data_ptr()),
                                         ctypes.byref(o), ctypes.byref(r))
        if check and rc != IGA_OK:
            raise IgaError(rc, lib().iga_last_error(self.h).decode())
        return r


def _wrap_device(ptr, n, dtype):
    """A torch view of library-owned device memory (no copy)."""
    import torch

    class _Arr:
        pass

    a = _Arr()
    typestr = {torch.int64: "<i8", torch.int32: "<i4", torch.float64: "<f8", torch.float32: "<f4"}[dtype]
    a.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 2}
    return torch.as_tensor(a, device="cuda")


# ------------------------------------------------------------------ batched ---
class IgaBatchReport(ctypes.Structure):
    _fields_ = [("solved", ctypes.c_int), ("newton_its", ctypes.c_void_p), ("krylov_its", ctypes.c_void_p),
                ("fnorm", ctypes.c_void_p), ("status", ctypes.c_void_p), ("solve_us", ctypes.c_void_p)]


def _batch_lib():
    L = lib()
    if not getattr(L, "_batch_ready", False):
        vp = ctypes.c_void_p
        L.iga_batch_create.argtypes = [ctypes.c_int, vp, vp, vp, ctypes.POINTER(vp)]
        L.iga_batch_offsets.argtypes = [vp, vp]
        L.iga_batch_set_launch.argtypes = [vp, ctypes.c_int, ctypes.c_int]
        L.iga_batch_set_tiles.argtypes = [vp, ctypes.c_int, ctypes.c_int]
        L.iga_batch_solve.argtypes = [vp, vp, ctypes.POINTER(IgaNewtonOpts), ctypes.POINTER(IgaBatchReport)]
        L.iga_batch_destroy.argtypes = [vp]
        L.iga_batch_destroy.restype = None
        L.iga_batch_last_error.argtypes = [vp]
        L.iga_batch_last_error.restype = ctypes.c_char_p
        L._batch_ready = True
    return L


class Batch:
    """iga_batch_t: many independent 2D problems solved in one persistent launch.

    instances: list of dicts {"nel": int or (n0, n1), "p": int, "lam": float,
    optional "knots": [U0, U1], "log_kappa": array}.
    """

    def __init__(self, instances):
        L = _batch_lib()
        n = len(instances)
        descs = (IgaDesc * n)()
        params = (IgaBratu * n)()
        self._keep = []
        for i, ins in enumerate(instances):
            d = descs[i]
            d.dim = 2
            nel = ins.get("nel")
            for ax in range(2):
                d.degree[ax] = int(ins["p"])
                d.continuity[ax] = -1
                if ins.get("knots") is not None:
                    k = _f64(ins["knots"][ax])
                    self._keep.append(k)
                    d.knots[ax] = k.ctypes.data
                    d.nknots[ax] = len(k)
                else:
                    d.nel[ax] = int(nel if np.isscalar(nel) else nel[ax])
            lk = ins.get("log_kappa")
            if lk is not None:
                lk = _f64(lk)
                self._keep.append(lk)
            params[i].lam = float(ins["lam"])
            params[i].log_kappa = None if lk is None else lk.ctypes.data
        h = ctypes.c_void_p()
        rc = L.iga_batch_create(n, ctypes.addressof(descs), ctypes.addressof(params), None, ctypes.byref(h))
        if rc != IGA_OK:
            raise IgaError(rc, L.iga_batch_last_error(None).decode())
        self.h = h
        self.count = n
        self.dot_chunks, self.jac_lines = 1, 4  # the library's defaults
        off = np.zeros(n + 1, dtype=np.int64)
        L.iga_batch_offsets(self.h, off.ctypes.data)
        self.offsets = off
        self.total = int(off[-1])

    def set_launch(self, ctas_per_sm, threads=512):
        """Launch shape of the persistent kernel: CTAs per SM and threads per CTA
        (256 or 512)."""
        L = _batch_lib()
        rc = L.iga_batch_set_launch(self.h, int(ctas_per_sm), int(threads))
        if rc != IGA_OK:
            raise IgaError(rc, L.iga_batch_last_error(self.h).decode())

    def set_tiles(self, dot_chunks, jac_lines=None):
        """Work unit of the Gram-Schmidt dots: row chunks per dot (0: enough to keep every
        warp busy; 1..16); element tile of the Jacobian's first stage: Gauss lines per
        shared-memory tile (1, 2, 4, 8; None keeps the current value)."""
        L = _batch_lib()
        if jac_lines is None:
            jac_lines = self.jac_lines
        rc = L.iga_batch_set_tiles(self.h, int(dot_chunks), int(jac_lines))
        if rc != IGA_OK:
            raise IgaError(rc, L.iga_batch_last_error(self.h).decode())
        self.dot_chunks, self.jac_lines = int(dot_chunks), int(jac_lines)

    def solve(self, U, opts=None, check=True):
        """U: torch CUDA float64 tensor of length self.total (in/out).  Returns a dict
        of per-instance arrays (newton_its, krylov_its, fnorm, status, solve_us: device time
        of each instance's solve) and 'solved'."""
        L = _batch_lib()
        o = opts if opts is not None else newton_defaults()
        nit = np.zeros(self.count, dtype=np.int32)
        kit = np.zeros(self.count, dtype=np.int32)
        fn = np.zeros(self.count)
        st = np.zeros(self.count, dtype=np.int32)
        us = np.zeros(self.count)
        r = IgaBatchReport(0, nit.ctypes.data, kit.ctypes.data, fn.ctypes.data, st.ctypes.data, us.ctypes.data)
        rc = L.iga_batch_solve(self.h, ctypes.c_void_p(U.data_ptr()), ctypes.byref(o), ctypes.byref(r))
        if check and rc != IGA_OK:
            raise IgaError(rc, L.iga_batch_last_error(self.h).decode())
        return {"solved": r.solved, "newton_its": nit, "krylov_its": kit, "fnorm": fn, "status": st, "solve_us": us,
                "rc": rc}

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _batch_lib().iga_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
