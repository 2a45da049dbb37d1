"""Seeded synthetic inputs shaped like the paper's workloads.

This module is the only code shared by the CUDA path's tests/benchmarks and the
oracle: it draws random numbers and builds input geometry, and holds none of the
assembly or solver arithmetic.

* ``splitmix64`` / ``uniform``: a counter-based stream (Steele, Lea, Flood,
  "Fast splittable pseudorandom number generators", 2014): state += 0x9E37..,
  then the two xor-shift-multiply rounds; 53 high bits give a double in [0, 1).
* ``interior_field``: U ~ U[lo, hi] on interior control variables, 0 on the
  boundary (open knot vectors interpolate at the ends, so boundary control
  variables are those with an index 0 or n-1 in some direction).
* ``quarter_annulus``: the NURBS quarter annulus extruded in z (inner radius 1,
  outer radius 2, height 1).  Angular direction: the rational quadratic Bezier
  quarter circle (weights 1, sqrt(2)/2, 1); radial and axial directions: linear.
  Every direction is raised to the requested degree by Bezier degree elevation in
  homogeneous coordinates and refined by inserting the interior knots of a
  uniform open knot vector one at a time (Boehm's algorithm), the geometry
  preparation the paper does with igakit (Sec. 2.9).
* ``ring``: a closed annular ring for a periodic angular direction: uniform B-spline
  control points on circles (radius at the radial Greville abscissae, angles
  2 pi j / n for the n wrapped angular functions), weights 1; optionally extruded in
  z.  A smooth closed approximation of the circle, positively oriented.
* ``unclamp_curve``: Sec. 2.4's unclamping of a curve's control points (the task of
  Algorithm 1): the knot vector is unclamped by Eqs. (unclamp-left)-(unclamp-right) and
  the new control points are the unique ones that reproduce the curve on the parametric
  domain -- here found by collocation (a linear solve at n+1 points of the domain), not by
  the printed loop.  With a closed curve of C^k continuity across the seam, the first and
  last k+1 unclamped control points coincide, and the periodic space keeps n-k of them.
* ``full_annulus``: the exact NURBS annulus (inner radius 1, outer 2) as a closed
  curve of four rational quadratic quarter arcs (C^0 at the quarter points, knots of
  multiplicity p there), raised to degree p and refined uniformly per quarter; its
  angular direction is meant to be periodic with C^0 continuity across the seam
  (k = 0, the last control points equal the first and are dropped).
* ``grf_log_kappa``: a Gaussian random field with a separable squared-exponential
  covariance on the control grid's Greville abscissae, sampled by Cholesky.
* ``batch_instances``: the draw of the heterogeneous batched workload.
"""
import math

import numpy as np

_M64 = (1 << 64) - 1


def splitmix64(seed, n):
    """n outputs of splitmix64 started from `seed` (uint64 array)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & _M64) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed, n, lo=0.0, hi=1.0):
    """n doubles uniform in [lo, hi) from the top 53 bits of splitmix64."""
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    return lo + (hi - lo) * u


def boundary_mask(n):
    """Boolean mask over natural order (first index fastest) of control variables
    with index 0 or n_d-1 in some direction."""
    n = list(n)
    idx = np.indices(n[::-1]).reshape(len(n), -1)[::-1]
    m = np.zeros(idx.shape[1], dtype=bool)
    for d, nd in enumerate(n):
        m |= (idx[d] == 0) | (idx[d] == nd - 1)
    return m


def interior_field(n, seed, lo=-0.1, hi=0.1):
    """U ~ U[lo, hi] (splitmix64 seed) on interior control variables, 0 on the boundary."""
    N = int(np.prod(n))
    U = uniform(seed, N, lo, hi)
    U[boundary_mask(n)] = 0.0
    return U


def uniform_open_knots(nel, p, k=None):
    """Open uniform knot vector on [0,1]; interior knots repeated p-k times."""
    if k is None or k < 0:
        k = p - 1
    U = [0.0] * (p + 1)
    for e in range(1, nel):
        U += [e / nel] * (p - k)
    U += [1.0] * (p + 1)
    return np.asarray(U, dtype=np.float64)


def graded_open_knots(nel, p, seed, k=None, extra=(), spread=0.6):
    """Open knot vector on [0,1] with nel spans of seeded, unequal lengths (length of
    span e proportional to 1 + spread * (2 u_e - 1), u_e from splitmix64(seed)); every
    interior knot repeated p-k times, and the interior knots listed in `extra`
    (1..nel-1) repeated once more each (a local drop of continuity)."""
    if k is None or k < 0:
        k = p - 1
    h = 1.0 + spread * (2.0 * uniform(seed, nel) - 1.0)
    x = np.concatenate([[0.0], np.cumsum(h)])
    x /= x[-1]
    U = [0.0] * (p + 1)
    for e in range(1, nel):
        U += [x[e]] * (p - k + (1 if e in extra else 0))
    U += [1.0] * (p + 1)
    return np.asarray(U, dtype=np.float64)


# ---------------------------------------------------------------- geometry ---

def _bezier_elevate(Pw, times):
    """Raise a Bezier curve (homogeneous control points, shape (p+1, c)) by `times`
    degrees: Q_i = (i/(p+1)) P_{i-1} + (1 - i/(p+1)) P_i."""
    for _ in range(times):
        p = Pw.shape[0] - 1
        Q = np.zeros((p + 2, Pw.shape[1]))
        Q[0] = Pw[0]
        Q[p + 1] = Pw[p]
        for i in range(1, p + 1):
            a = i / (p + 1.0)
            Q[i] = a * Pw[i - 1] + (1.0 - a) * Pw[i]
        Pw = Q
    return Pw


def _insert_knot(U, Pw, p, u):
    """Insert knot u once (Boehm): returns the new knot vector and control points."""
    k = int(np.searchsorted(U, u, side="right")) - 1  # U[k] <= u < U[k+1]
    n = Pw.shape[0]
    Q = np.zeros((n + 1, Pw.shape[1]))
    for i in range(n + 1):
        if i <= k - p:
            Q[i] = Pw[i]
        elif i >= k + 1:
            Q[i] = Pw[i - 1]
        else:
            a = (u - U[i]) / (U[i + p] - U[i])
            Q[i] = a * Pw[i] + (1.0 - a) * Pw[i - 1]
    U2 = np.concatenate([U[: k + 1], [u], U[k + 1:]])
    return U2, Q


def _refine_curve(Pw_bezier, degree, nel):
    """Elevate a single-span Bezier curve to `degree` and insert nel-1 uniform knots."""
    p0 = Pw_bezier.shape[0] - 1
    Pw = _bezier_elevate(np.asarray(Pw_bezier, dtype=np.float64), degree - p0)
    U = np.array([0.0] * (degree + 1) + [1.0] * (degree + 1))
    for e in range(1, nel):
        U, Pw = _insert_knot(U, Pw, degree, e / nel)
    return U, Pw


def quarter_annulus(nel, degree=3, r_in=1.0, r_out=2.0, height=1.0):
    """NURBS quarter annulus extruded in z.  Axis 0 = radius, axis 1 = angle,
    axis 2 = height.  Returns (knots[3], ctrl (N,3), weights (N,)) in natural
    order (axis 0 fastest)."""
    if np.isscalar(nel):
        nel = (nel, nel, nel)
    s = math.sqrt(0.5)
    # angular: rational quadratic quarter circle, homogeneous (w x, w y, w)
    arc = np.array([[1.0, 0.0, 1.0], [s * 1.0, s * 1.0, s], [0.0, 1.0, 1.0]])
    Uth, Pth = _refine_curve(arc, degree, nel[1])
    # radial and axial: straight lines (weights 1)
    Ur, Pr = _refine_curve(np.array([[r_in, 1.0], [r_out, 1.0]]), degree, nel[0])
    Uz, Pz = _refine_curve(np.array([[0.0, 1.0], [height, 1.0]]), degree, nel[2])
    r = Pr[:, 0] / Pr[:, 1]
    z = Pz[:, 0] / Pz[:, 1]
    wth = Pth[:, 2]
    cth = Pth[:, :2] / wth[:, None]
    n0, n1, n2 = len(r), len(wth), len(z)
    ctrl = np.zeros((n2, n1, n0, 3))
    ctrl[..., 0] = r[None, None, :] * cth[None, :, 0, None]
    ctrl[..., 1] = r[None, None, :] * cth[None, :, 1, None]
    ctrl[..., 2] = z[:, None, None]
    weights = np.broadcast_to(wth[None, :, None], (n2, n1, n0)).copy()
    return [Ur, Uth, Uz], ctrl.reshape(-1, 3), weights.reshape(-1)


def ring(nel_r, nel_t, p, r_in=1.0, r_out=2.0, nel_z=None, height=1.0):
    """Open knot vectors (radial, angular[, axial]) and control points (N, dim) of a ring
    whose angular direction (axis 1) is meant to be C^(p-1) periodic: nel_t wrapped
    angular functions with control points at angles 2 pi j / nel_t (natural order,
    axis 0 fastest)."""
    kr = uniform_open_knots(nel_r, p)
    kt = uniform_open_knots(nel_t, p)
    r = r_in + (r_out - r_in) * greville(kr, p)
    th = 2.0 * math.pi * np.arange(nel_t) / nel_t
    if nel_z is None:
        X = np.stack([np.outer(np.cos(th), r), np.outer(np.sin(th), r)], axis=-1)  # [j][i][2]
        return [kr, kt], X.reshape(-1, 2)
    kz = uniform_open_knots(nel_z, p)
    z = height * greville(kz, p)
    X = np.zeros((len(z), nel_t, len(r), 3))
    X[..., 0] = np.cos(th)[None, :, None] * r[None, None, :]
    X[..., 1] = np.sin(th)[None, :, None] * r[None, None, :]
    X[..., 2] = z[:, None, None]
    return [kr, kt, kz], X.reshape(-1, 3)


def _unclamp_knots(U, p, k):
    X = np.array(U, dtype=np.float64)
    m = len(X) - 1
    n = m - p - 1
    for i in range(k + 1):
        X[k - i] = X[p] - X[n + 1] + X[n - i]
    for i in range(k + 1):
        X[m - k + i] = X[n + 1] - X[p] + X[p + i + 1]
    return X


def _basis_row(U, p, nfun, xi):
    """Values of the nfun B-splines of knot vector U at xi (Cox-de Boor, degree by degree),
    xi strictly inside the domain [U_p, U_{nfun}]."""
    N = np.zeros(len(U) - 1)
    s = int(np.searchsorted(U, xi, side="right")) - 1
    N[s] = 1.0
    for d in range(1, p + 1):
        M = np.zeros_like(N)
        for i in range(len(U) - d - 1):
            a = (xi - U[i]) / (U[i + d] - U[i]) * N[i] if U[i + d] > U[i] else 0.0
            b = (U[i + d + 1] - xi) / (U[i + d + 1] - U[i + 1]) * N[i + 1] if U[i + d + 1] > U[i + 1] else 0.0
            M[i] = a + b
        N = M
    return N[:nfun]


def unclamp_curve(U, Pw, p, k):
    """Unclamped knot vector and control points (homogeneous, rows of Pw) of the curve
    sum_i N_i(xi; U) Pw_i, for C^k periodicity (Sec. 2.4): same curve on [U_p, U_{n+1}]."""
    U = np.asarray(U, dtype=np.float64)
    Pw = np.asarray(Pw, dtype=np.float64)
    nfun = len(U) - p - 1
    V = _unclamp_knots(U, p, k)
    lo, hi = U[p], U[nfun]
    xs = lo + (hi - lo) * (np.arange(nfun) + 0.5) / nfun  # interior collocation points
    A = np.array([_basis_row(V, p, nfun, x) for x in xs])
    C = np.array([_basis_row(U, p, nfun, x) @ Pw for x in xs])
    return V, np.linalg.solve(A, C)


def full_annulus(nel_r, nel_q, p=2, r_in=1.0, r_out=2.0):
    """Knot vectors (radial, angular; open) and control points (N, 2) with weights (N,)
    of the exact annulus; nel_q elements per quarter of the angular direction.  The
    angular control points are those of the wrapped periodic space (C^0 across the
    seam: the closed curve's last control point, equal to its first, is left out)."""
    s = math.sqrt(0.5)
    quarter = np.array([[1.0, 0.0, 1.0], [s, s, s], [0.0, 1.0, 1.0]])  # homogeneous (w x, w y, w)
    Ut, Pt = None, None
    for j in range(4):
        c, sn = math.cos(j * math.pi / 2), math.sin(j * math.pi / 2)
        R = np.array([[c, -sn, 0.0], [sn, c, 0.0], [0.0, 0.0, 1.0]])
        Uq, Pq = _refine_curve(quarter @ R.T, p, nel_q)  # one quarter, degree p, nel_q elements on [0, 1]
        Uq = (Uq + j) / 4.0
        if Ut is None:
            Ut, Pt = Uq, Pq
        else:  # join at the quarter point: knot of multiplicity p, shared end control point
            Ut = np.concatenate([Ut[:-1], Uq[p + 1:]])
            Pt = np.concatenate([Pt, Pq[1:]])
    Pt = Pt[:-1]  # the last equals the first: the periodic space wraps it
    Ur, Pr = _refine_curve(np.array([[r_in, 1.0], [r_out, 1.0]]), p, nel_r)
    r = Pr[:, 0] / Pr[:, 1]
    wt = Pt[:, 2]
    ct = Pt[:, :2] / wt[:, None]
    ctrl = (r[None, :, None] * ct[:, None, :]).reshape(-1, 2)   # [j][i][2], axis 0 (radius) fastest
    weights = np.broadcast_to(wt[:, None], (len(wt), len(r))).reshape(-1).copy()
    return [Ur, Ut], ctrl, weights


def greville(U, p):
    """Greville abscissae of a knot vector."""
    n = len(U) - p - 1
    return np.array([np.mean(U[i + 1: i + p + 1]) for i in range(n)]) if p > 0 else 0.5 * (U[:-1] + U[1:])[:n]


# ------------------------------------------------------------ random fields --

def grf_log_kappa(n, p, nel, seed, variance=0.5, length=0.2, jitter=1e-8):
    """log kappa on the control grid: a zero-mean Gaussian field with covariance
    variance * exp(-|x - y|^2 / (2 length^2)), separable over directions, sampled
    as L_1 Z L_0^T with L_d the Cholesky factor of the 1D covariance on the
    Greville abscissae.  Z is N(0,1) by Box-Muller on splitmix64 uniforms."""
    g = [greville(uniform_open_knots(nel[d], p), p) for d in range(2)]
    L = []
    for d in range(2):
        C = np.exp(-(g[d][:, None] - g[d][None, :]) ** 2 / (2.0 * length * length))
        L.append(np.linalg.cholesky(C + jitter * np.eye(len(g[d]))))
    N = n[0] * n[1]
    u = uniform(seed, 2 * N)
    u1 = np.maximum(u[:N], 1e-300)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u[N:])
    Z = z.reshape(n[1], n[0])
    field = math.sqrt(variance) * (L[1] @ Z @ L[0].T)
    return field.reshape(-1)


def batch_instances(count, seed=0, nmin=16, nmax=128, degrees=(2, 3), lam=(0.5, 6.0)):
    """Heterogeneous 2D Bratu instances: square meshes n ~ U{nmin..nmax},
    p ~ U{degrees}, lambda ~ U[lam]; instance i draws from splitmix64(seed + i)."""
    out = []
    for i in range(count):
        u = uniform((seed * 1000003 + i) & _M64, 3)
        nel = nmin + int(u[0] * (nmax - nmin + 1))
        p = degrees[int(u[1] * len(degrees))]
        lm = lam[0] + (lam[1] - lam[0]) * u[2]
        out.append({"nel": nel, "p": p, "lam": float(lm)})
    return out
