"""ctypes front end of the C oracle (``iga_oracle.c``) plus the oracle's own Newton.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every function follows a
passage of the PetIGA paper, cited where it is defined in ``iga_oracle.c``:

* ``open_uniform_knots``      -- open knot vector with interior knots repeated
  p-k times for continuity C^k (Sec. 2.1, 2.4; PetIGA's default space is the
  uniform, maximally smooth one, Sec. 3.2).
* ``Problem``                 -- the discretisation (Sec. 2.2-2.3) and the Bratu
  parameters (Sec. 3.1).
* ``residual``/``jacobian``   -- Algorithm 3 (Sec. 2.7) with Eq. (residual) and
  Eq. (jacobian).
* ``pattern``                 -- Algorithm 2 (Sec. 2.5).
* ``newton``                  -- Newton's method on R(U) = 0 (Sec. 3.1), each
  linear system solved exactly by a sparse LU (a library primitive).
* ``mass``/``residual_ts``/``jacobian_ts`` -- the semi-discrete time-dependent
  residual R(U-dot, U) of Sec. 4.2 for the transient Bratu problem, and its
  derivative dR/dU + shift dR/dU-dot.
* ``unclamp_knots``           -- Sec. 2.4 Eqs. (unclamp-left)-(unclamp-right): the
  knot vector of a periodic direction with continuity C^k across the boundary.
* ``alpha_params``/``alpha_step`` -- one step of the generalized-alpha method for
  first-order systems, Sec. 4.2 Eq. (ga), parameters from rho_infinity.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "iga_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force=False):
    """Compile the C oracle with gcc (plain -O2, no fast-math).  OpenMP serves only the
    colour-loop timing mode; without it (no libgomp) the oracle builds single-threaded."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC]
    if subprocess.call(base + ["-fopenmp", "-lm"], stderr=subprocess.DEVNULL) != 0:
        subprocess.check_call(base + ["-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


class _Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("p", ctypes.c_int * 3),
        ("m", ctypes.c_int * 3),
        ("U", ctypes.c_void_p * 3),
        ("q", ctypes.c_int * 3),
        ("ctrl", ctypes.c_void_p),
        ("weights", ctypes.c_void_p),
        ("lam", ctypes.c_double),
        ("log_kappa", ctypes.c_void_p),
        ("bnd", (ctypes.c_int * 2) * 3),
        ("bval", (ctypes.c_double * 2) * 3),
        ("source", ctypes.c_int),
        ("wrap", ctypes.c_int * 3),
    ]


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.POINTER(_Problem)
        vp, i64 = ctypes.c_void_p, ctypes.c_int64
        L.or_bspline.restype = ctypes.c_double
        L.or_bspline.argtypes = [ctypes.c_int, ctypes.c_int, vp, ctypes.c_double]
        L.or_bspline_der.restype = ctypes.c_double
        L.or_bspline_der.argtypes = [ctypes.c_int, ctypes.c_int, vp, ctypes.c_double]
        L.or_gauss_legendre.argtypes = [ctypes.c_int, vp, vp]
        L.or_spans.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp]
        L.or_stencil.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp]
        L.or_num_dofs.restype = i64
        L.or_num_dofs.argtypes = [P]
        L.or_pattern.restype = i64
        L.or_pattern.argtypes = [P, vp, vp]
        L.or_pattern_dense_from_elements.argtypes = [P, vp]
        L.or_residual.argtypes = [P, vp, vp]
        L.or_jacobian.argtypes = [P, vp, vp, vp, vp]
        L.or_jacobian_fd.argtypes = [P, vp, vp, vp, vp]
        L.or_mass.argtypes = [P, vp, vp, vp]
        L.or_residual_colored.argtypes = [P, vp, vp]
        L.or_jacobian_colored.argtypes = [P, vp, vp, vp, vp]
        L.or_num_threads.restype = ctypes.c_int
        L.or_residual_rows.argtypes = [P, vp, i64, vp, vp]
        L.or_jacobian_rows.argtypes = [P, vp, i64, vp, vp, vp, vp]
        L.or_dense_bruteforce.argtypes = [P, vp, vp, vp, ctypes.c_int]
        L.or_l2_error_sq.restype = ctypes.c_double
        L.or_l2_error_sq.argtypes = [P, vp]
        L.or_map_point.argtypes = [P, vp, vp, vp]
        L.or_is_dirichlet.argtypes = [P, i64]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data if a is not None else None


def open_uniform_knots(nel, p, k=None):
    """Open knot vector on [0, 1] with nel uniform spans, p+1 end knots and every
    interior knot repeated p-k times (continuity C^k; default k = p-1)."""
    if k is None or k < 0:
        k = p - 1
    mult = p - k
    U = [0.0] * (p + 1)
    for e in range(1, nel):
        U += [e / nel] * mult
    U += [1.0] * (p + 1)
    return np.asarray(U, dtype=np.float64)


def num_threads():
    """Threads of the colour-loop timing mode (OpenMP's default: all host cores)."""
    return int(lib().or_num_threads())


def gauss_legendre(q):
    x = np.zeros(q)
    w = np.zeros(q)
    rc = lib().or_gauss_legendre(q, _ptr(x), _ptr(w))
    assert rc == 0
    return x, w


def bspline(i, p, U, xi):
    U = np.ascontiguousarray(U, dtype=np.float64)
    return lib().or_bspline(i, p, _ptr(U), float(xi))


def bspline_der(i, p, U, xi):
    U = np.ascontiguousarray(U, dtype=np.float64)
    return lib().or_bspline_der(i, p, _ptr(U), float(xi))


def unclamp_knots(U, p, k):
    """Sec. 2.4: redefine the k+1 end knots at each side of an open knot vector
    (m = n + p + 1 its last index) so the space is C^k across the boundary:
        xi_{k-i}   = xi_p - xi_{n+1} + xi_{n-i},       0 <= i <= k,
        xi_{m-k+i} = xi_{n+1} - xi_p + xi_{p+i+1},     0 <= i <= k."""
    X = np.array(U, dtype=np.float64)
    m = len(X) - 1
    n = m - p - 1
    assert 0 <= k <= p - 1
    for i in range(k + 1):
        X[k - i] = X[p] - X[n + 1] + X[n - i]
    for i in range(k + 1):
        X[m - k + i] = X[n + 1] - X[p] + X[p + i + 1]
    return X


def stencil(i, p, U):
    U = np.ascontiguousarray(U, dtype=np.float64)
    l = ctypes.c_int()
    r = ctypes.c_int()
    lib().or_stencil(i, p, _ptr(U), ctypes.byref(l), ctypes.byref(r))
    return l.value, r.value


class Problem:
    """A scalar Bratu problem on a tensor-product NURBS space.

    knots: list of per-direction knot vectors; degrees: list of p; quad: list of
    Gauss points per direction (default p+1); ctrl: (N, dim) control points or
    None (identity map); weights: (N,) or None; lam: lambda; log_kappa: (N,) or
    None; dirichlet: dict {(axis, side): value}; periodic: dict {axis: k}, the
    open knot vector of that axis unclamped for C^k periodicity (Sec. 2.4), its
    n - k functions numbered by Eq. (map-wrap).  ctrl, weights and log_kappa hold
    one entry per (wrapped) function.
    """

    def __init__(self, knots, degrees, quad=None, ctrl=None, weights=None, lam=1.0,
                 log_kappa=None, dirichlet=None, source=False, periodic=None):
        dim = len(knots)
        self.dim = dim
        self.periodic = dict(periodic or {})
        self.wrap = [self.periodic[d] + 1 if d in self.periodic else 0 for d in range(dim)]
        self.knots = [np.ascontiguousarray(unclamp_knots(k, p, self.periodic[d]) if d in self.periodic else k,
                                           dtype=np.float64) for d, (k, p) in enumerate(zip(knots, degrees))]
        self.degrees = list(degrees)
        self.quad = list(quad) if quad is not None else [p + 1 for p in degrees]
        self.n = [len(k) - p - 1 - w for k, p, w in zip(self.knots, self.degrees, self.wrap)]
        self.N = int(np.prod(self.n))
        self.ctrl = None if ctrl is None else np.ascontiguousarray(ctrl, dtype=np.float64).reshape(self.N, dim)
        self.weights = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64).reshape(self.N)
        self.lam = float(lam)
        self.log_kappa = None if log_kappa is None else np.ascontiguousarray(log_kappa, dtype=np.float64).reshape(self.N)
        self.dirichlet = dict(dirichlet or {})
        self.source = bool(source)
        self._pat = None

    def _c(self):
        s = _Problem()
        s.dim = self.dim
        for d in range(self.dim):
            s.p[d] = self.degrees[d]
            s.m[d] = len(self.knots[d])
            s.U[d] = self.knots[d].ctypes.data
            s.q[d] = self.quad[d]
        s.ctrl = _ptr(self.ctrl)
        s.weights = _ptr(self.weights)
        s.lam = self.lam
        s.log_kappa = _ptr(self.log_kappa)
        for (ax, side), v in self.dirichlet.items():
            s.bnd[ax][side] = 1
            s.bval[ax][side] = float(v)
        s.source = 1 if self.source else 0
        for d in range(self.dim):
            s.wrap[d] = self.wrap[d]
        return s

    # -- Sec. 2.5 Algorithm 2 -------------------------------------------------
    def pattern(self):
        if self._pat is None:
            c = self._c()
            rowptr = np.zeros(self.N + 1, dtype=np.int64)
            nnz = lib().or_pattern(ctypes.byref(c), _ptr(rowptr), None)
            assert nnz >= 0
            colidx = np.zeros(nnz, dtype=np.int32)
            lib().or_pattern(ctypes.byref(c), _ptr(rowptr), _ptr(colidx))
            self._pat = (rowptr, colidx)
        return self._pat

    def pattern_dense_from_elements(self):
        c = self._c()
        mark = np.zeros((self.N, self.N), dtype=np.uint8)
        rc = lib().or_pattern_dense_from_elements(ctypes.byref(c), _ptr(mark))
        assert rc == 0
        return mark

    def is_dirichlet(self, A):
        c = self._c()
        return bool(lib().or_is_dirichlet(ctypes.byref(c), int(A)))

    # -- Sec. 2.7 Algorithm 3 ----------------------------------------------------
    def residual(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        F = np.zeros(self.N)
        c = self._c()
        rc = lib().or_residual(ctypes.byref(c), _ptr(U), _ptr(F))
        if rc:
            raise RuntimeError("or_residual failed: %d" % rc)
        return F

    def jacobian(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        rowptr, colidx = self.pattern()
        vals = np.zeros(len(colidx))
        c = self._c()
        rc = lib().or_jacobian(ctypes.byref(c), _ptr(U), _ptr(rowptr), _ptr(colidx), _ptr(vals))
        if rc:
            raise RuntimeError("or_jacobian failed: %d" % rc)
        return vals

    # -- timing mode: the same loops colour by colour on all OpenMP threads --------
    def residual_colored(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        F = np.zeros(self.N)
        c = self._c()
        rc = lib().or_residual_colored(ctypes.byref(c), _ptr(U), _ptr(F))
        if rc:
            raise RuntimeError("or_residual_colored failed: %d" % rc)
        return F

    def jacobian_colored(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        rowptr, colidx = self.pattern()
        vals = np.zeros(len(colidx))
        c = self._c()
        rc = lib().or_jacobian_colored(ctypes.byref(c), _ptr(U), _ptr(rowptr), _ptr(colidx), _ptr(vals))
        if rc:
            raise RuntimeError("or_jacobian_colored failed: %d" % rc)
        return vals

    def jacobian_fd(self, U):
        """Sec. 2.8 local numerical differentiation, Eq. (fdjac), on the pattern."""
        U = np.ascontiguousarray(U, dtype=np.float64)
        rowptr, colidx = self.pattern()
        vals = np.zeros(len(colidx))
        c = self._c()
        rc = lib().or_jacobian_fd(ctypes.byref(c), _ptr(U), _ptr(rowptr), _ptr(colidx), _ptr(vals))
        if rc:
            raise RuntimeError("or_jacobian_fd failed: %d" % rc)
        return vals

    def mass(self):
        """Mass matrix (N_A, N_B) on the pattern, no Dirichlet fix (Sec. 4.2)."""
        rowptr, colidx = self.pattern()
        vals = np.zeros(len(colidx))
        c = self._c()
        rc = lib().or_mass(ctypes.byref(c), _ptr(rowptr), _ptr(colidx), _ptr(vals))
        if rc:
            raise RuntimeError("or_mass failed: %d" % rc)
        return vals

    def mass_csr(self):
        import scipy.sparse as sp
        rowptr, colidx = self.pattern()
        return sp.csr_matrix((self.mass(), colidx, rowptr), shape=(self.N, self.N))

    def residual_ts(self, V, U):
        """Sec. 4.2: R_A(U-dot, U) = (N_A, u-dot^h) + [Eq. (residual)]_A on the rows
        without Dirichlet data; Dirichlet rows U_A - g as in ``residual``."""
        F = self.residual(U)
        MV = self.mass_csr() @ np.asarray(V, dtype=np.float64)
        free = ~self.dirichlet_mask()
        F[free] += MV[free]
        return F

    def jacobian_ts(self, shift, U):
        """dR/dU + shift dR/dU-dot on the pattern: Eq. (jacobian) plus shift times the
        mass matrix, with the Dirichlet fix of ``jacobian`` (identity rows, zero columns)."""
        J = self.jacobian(U)
        M = self.mass()
        rowptr, colidx = self.pattern()
        bnd = self.dirichlet_mask()
        rows = np.repeat(np.arange(self.N), np.diff(rowptr))
        keep = ~bnd[rows] & ~bnd[colidx]
        J[keep] += shift * M[keep]
        return J

    def jacobian_csr(self, U):
        import scipy.sparse as sp
        rowptr, colidx = self.pattern()
        return sp.csr_matrix((self.jacobian(U), colidx, rowptr), shape=(self.N, self.N))

    def residual_rows(self, U, rows):
        U = np.ascontiguousarray(U, dtype=np.float64)
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.zeros(len(rows))
        c = self._c()
        rc = lib().or_residual_rows(ctypes.byref(c), _ptr(U), len(rows), _ptr(rows), _ptr(out))
        if rc:
            raise RuntimeError("or_residual_rows failed: %d" % rc)
        return out

    def jacobian_rows(self, U, rows):
        """Values of the selected CSR rows, concatenated in the order of rows."""
        U = np.ascontiguousarray(U, dtype=np.float64)
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        rowptr, colidx = self.pattern()
        total = int(sum(rowptr[r + 1] - rowptr[r] for r in rows))
        out = np.zeros(total)
        c = self._c()
        rc = lib().or_jacobian_rows(ctypes.byref(c), _ptr(U), len(rows), _ptr(rows), _ptr(rowptr),
                                    _ptr(colidx), _ptr(out))
        if rc:
            raise RuntimeError("or_jacobian_rows failed: %d" % rc)
        return out

    def dense_bruteforce(self, U, fix=True):
        U = np.ascontiguousarray(U, dtype=np.float64)
        F = np.zeros(self.N)
        J = np.zeros((self.N, self.N))
        c = self._c()
        rc = lib().or_dense_bruteforce(ctypes.byref(c), _ptr(U), _ptr(F), _ptr(J), 1 if fix else 0)
        if rc:
            raise RuntimeError("or_dense_bruteforce failed: %d" % rc)
        return F, J

    def l2_error(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        c = self._c()
        return float(np.sqrt(lib().or_l2_error_sq(ctypes.byref(c), _ptr(U))))

    def map_point(self, xi):
        xi = np.ascontiguousarray(list(xi) + [0.0] * (3 - len(xi)), dtype=np.float64)
        x = np.zeros(3)
        det = ctypes.c_double()
        c = self._c()
        rc = lib().or_map_point(ctypes.byref(c), _ptr(xi), _ptr(x), ctypes.byref(det))
        assert rc == 0
        return x[: self.dim], det.value

    def dirichlet_mask(self):
        m = np.zeros(self.N, dtype=bool)
        if not self.dirichlet:
            return m
        idx = np.indices(self.n[::-1]).reshape(self.dim, -1)[::-1]  # idx[d] = i_d of natural A
        for (ax, side) in self.dirichlet:
            m |= idx[ax] == (0 if side == 0 else self.n[ax] - 1)
        return m


def newton(prob, U0, atol=1e-10, max_it=50):
    """Newton's method on R(U) = 0 (Sec. 3.1): J(U_k) dU = -R(U_k), U_{k+1} = U_k + dU,
    with each linear system solved exactly by sparse LU.  Returns (U, history)."""
    import scipy.sparse.linalg as spla
    U = np.array(U0, dtype=np.float64)
    hist = []
    for _ in range(max_it + 1):
        F = prob.residual(U)
        nf = float(np.linalg.norm(F))
        hist.append(nf)
        if nf <= atol or not np.isfinite(nf):
            break
        J = prob.jacobian_csr(U)
        U = U + spla.spsolve(J.tocsc(), -F)
    return U, hist


def alpha_params(rho_inf):
    """Sec. 4.2: alpha_m, alpha_f and gamma of the generalized-alpha method from the
    spectral radius rho_infinity of the amplification matrix as dt -> infinity."""
    am = 0.5 * (3.0 - rho_inf) / (1.0 + rho_inf)
    af = 1.0 / (1.0 + rho_inf)
    return am, af, 0.5 + am - af


def alpha_step(prob, U_n, V_n, dt, rho_inf, atol=1e-12, max_it=50):
    """One step of Eq. (ga) (Sec. 4.2) for the transient residual ``residual_ts``:
    given U_n and U-dot_n, find U-dot_{n+1} (and U_{n+1}) with
        R(U-dot_{n+alpha_m}, U_{n+alpha_f}) = 0,
        U-dot_{n+alpha_m} = U-dot_n + alpha_m (U-dot_{n+1} - U-dot_n),
        U_{n+alpha_f}     = U_n + alpha_f (U_{n+1} - U_n),
        U_{n+1}           = U_n + dt (gamma U-dot_{n+1} + (1 - gamma) U-dot_n).
    Newton on the unknown U-dot_{n+1}, starting from the value that makes U_{n+1} = U_n
    (U-dot_{n+1} = (gamma - 1) / gamma U-dot_n); its Jacobian is
    alpha_m dR/dU-dot + alpha_f gamma dt dR/dU at the stage values, each linear
    system solved by sparse LU.  Returns (U_{n+1}, U-dot_{n+1}, history of ||R||)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    am, af, gam = alpha_params(rho_inf)
    U_n = np.asarray(U_n, dtype=np.float64)
    V_n = np.asarray(V_n, dtype=np.float64)
    rowptr, colidx = prob.pattern()
    V1 = (gam - 1.0) / gam * V_n
    hist = []
    for _ in range(max_it + 1):
        U1 = U_n + dt * (gam * V1 + (1.0 - gam) * V_n)
        Vm = V_n + am * (V1 - V_n)
        Uf = U_n + af * (U1 - U_n)
        R = prob.residual_ts(Vm, Uf)
        nr = float(np.linalg.norm(R))
        hist.append(nr)
        if nr <= atol or not np.isfinite(nr):
            break
        # dR/dU-dot_{n+1} = alpha_m dR/dU-dot + alpha_f gamma dt dR/dU; the Dirichlet rows
        # U_A - g depend on U-dot_{n+1} through U_{n+alpha_f} only
        vals = af * gam * dt * prob.jacobian_ts(am / (af * gam * dt), Uf)
        J = sp.csr_matrix((vals, colidx, rowptr), shape=(prob.N, prob.N))
        V1 = V1 + spla.spsolve(J.tocsc(), -R)
    U1 = U_n + dt * (gam * V1 + (1.0 - gam) * V_n)
    return U1, V1, hist
