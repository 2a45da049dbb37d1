"""Pins for the oracle against what the paper and the mathematics fix (CPU only).

Each test names the passage or property it pins.  A plausible mistake in the
oracle -- a dropped rational term, a wrong sign in Eq. (3), a wrong index in the
element-to-global map, a wrong quadrature weight -- fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_1305_4452_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def dirichlet_all(dim, value=0.0):
    return {(a, s): value for a in range(dim) for s in range(2)}


# ---------------------------------------------------------------- Sec. 2.9 GL

@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 7, 10])
def test_gauss_legendre_exactness(q):
    x, w = O.gauss_legendre(q)
    assert abs(w.sum() - 2.0) < 1e-14
    assert np.all(np.diff(x) > 0) and np.allclose(x, -x[::-1], atol=1e-15)
    for k in range(2 * q):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 2e-14, (q, k)
    # degree 2q is not integrated exactly (the rule is not over-claimed)
    assert abs(np.dot(w, x ** (2 * q)) - 2.0 / (2 * q + 1)) > 1e-6


# ---------------------------------------------------------- Sec. 2.1 B-splines

KNOTS = [
    (2, O.open_uniform_knots(5, 2)),
    (3, O.open_uniform_knots(6, 3)),
    (3, np.array([0, 0, 0, 0, 2, 4, 4, 6, 6, 6, 8, 8, 8, 8], float) / 8.0),  # Sec. 2.5 figure
    (4, O.open_uniform_knots(4, 4, 2)),
    (1, O.open_uniform_knots(7, 1)),
]


@pytest.mark.parametrize("p,U", KNOTS)
def test_partition_of_unity_and_derivative_sum(p, U):
    n = len(U) - p - 1
    rng = np.random.default_rng(1)
    for xi in rng.random(25) * 0.999999:
        vals = np.array([O.bspline(i, p, U, xi) for i in range(n)])
        ders = np.array([O.bspline_der(i, p, U, xi) for i in range(n)])
        assert abs(vals.sum() - 1.0) < 1e-15 * 4
        assert np.all(vals >= 0.0)
        # Eq. (3) with the sign that differentiating Eq. (2) gives; a "+" fails here
        assert abs(ders.sum()) < 1e-12 * max(1.0, np.abs(ders).max())
        # support [U_i, U_{i+p+1})
        for i in range(n):
            if not (U[i] <= xi < U[i + p + 1]):
                assert vals[i] == 0.0


@pytest.mark.parametrize("p,U", KNOTS)
def test_derivative_matches_central_difference(p, U):
    n = len(U) - p - 1
    h = 1e-6
    for xi in [0.123, 0.377, 0.61, 0.905]:
        for i in range(n):
            fd = (O.bspline(i, p, U, xi + h) - O.bspline(i, p, U, xi - h)) / (2 * h)
            assert abs(fd - O.bspline_der(i, p, U, xi)) < 1e-6 * (1 + abs(fd))


def test_bernstein_special_case():
    # one span, open knots: the B-splines are the Bernstein polynomials
    U = np.array([0, 0, 0, 1, 1, 1], float)
    for xi in [0.1, 0.5, 0.73]:
        ref = [(1 - xi) ** 2, 2 * xi * (1 - xi), xi ** 2]
        dref = [-2 * (1 - xi), 2 - 4 * xi, 2 * xi]
        for i in range(3):
            assert abs(O.bspline(i, 2, U, xi) - ref[i]) < 1e-15
            assert abs(O.bspline_der(i, 2, U, xi) - dref[i]) < 1e-14


def test_polynomial_reproduction_by_blossom():
    # x^2 = sum_i c_i B_{i,p}(x) with c_i the blossom of x^2 at (U_{i+1},...,U_{i+p});
    # x = sum_i g_i B_{i,p} with g_i the Greville abscissae (linear precision)
    for p, U in [(2, O.open_uniform_knots(5, 2)), (3, O.open_uniform_knots(4, 3, 1)), (4, O.open_uniform_knots(3, 4))]:
        n = len(U) - p - 1
        c = []
        for i in range(n):
            t = U[i + 1: i + p + 1]
            s = sum(t[a] * t[b] for a in range(p) for b in range(a + 1, p))
            c.append(2.0 * s / (p * (p - 1)))
        g = [np.mean(U[i + 1: i + p + 1]) for i in range(n)]
        for xi in [0.05, 0.31, 0.5, 0.88]:
            B = [O.bspline(i, p, U, xi) for i in range(n)]
            assert abs(np.dot(c, B) - xi * xi) < 1e-14
            assert abs(np.dot(g, B) - xi) < 1e-14


# ------------------------------------------------------------- Sec. 2.5 Alg. 2

@pytest.mark.parametrize("p,U", KNOTS)
def test_stencil_matches_support_overlap(p, U):
    n = len(U) - p - 1
    for i in range(n):
        l, r = O.stencil(i, p, U)
        overl = [j for j in range(n) if max(U[i], U[j]) < min(U[i + p + 1], U[j + p + 1])]
        assert (l, r) == (min(overl), max(overl)), (i, l, r, overl)


@pytest.mark.parametrize("dim,p,nel,k", [(2, 2, 4, 1), (2, 3, 3, 1), (3, 2, 2, 1), (2, 1, 5, 0), (2, 3, 3, 2)])
def test_pattern_two_constructions_agree(dim, p, nel, k):
    U = O.open_uniform_knots(nel, p, k)
    P = O.Problem([U] * dim, [p] * dim)
    rowptr, colidx = P.pattern()
    mark = P.pattern_dense_from_elements()
    dense = np.zeros((P.N, P.N), np.uint8)
    rows = np.repeat(np.arange(P.N), np.diff(rowptr))
    dense[rows, colidx] = 1
    assert np.array_equal(dense, mark)
    for A in range(P.N):
        assert np.all(np.diff(colidx[rowptr[A]:rowptr[A + 1]]) > 0)


def test_pattern_counts_of_the_configs():
    # n = nel + p functions per direction at maximal continuity; counted nnz
    U = O.open_uniform_knots(16, 2)
    P = O.Problem([U, U], [2, 2])
    rowptr, colidx = P.pattern()
    assert P.N == 324 and len(colidx) == 7056
    U3 = O.open_uniform_knots(8, 3)
    P3 = O.Problem([U3] * 3, [3] * 3)
    n1 = sum(min(i, 3) + min(10 - i, 3) + 1 for i in range(11))
    assert len(P3.pattern()[1]) == n1 ** 3


# ------------------------------------------------- Sec. 3 / App. B: the residual

def integral_1d(U, p):
    n = len(U) - p - 1
    return np.array([(U[i + p + 1] - U[i]) / (p + 1) for i in range(n)])


@pytest.mark.parametrize("dim,p,nel,lam", [(2, 2, 6, 1.0), (2, 3, 5, 2.5), (3, 2, 3, 2.0)])
def test_residual_at_zero_is_minus_lambda_times_basis_integrals(dim, p, nel, lam):
    U = O.open_uniform_knots(nel, p)
    P = O.Problem([U] * dim, [p] * dim, lam=lam, dirichlet=dirichlet_all(dim))
    F = P.residual(np.zeros(P.N))
    I1 = integral_1d(U, p)
    ref = -lam * I1
    for _ in range(dim - 1):
        ref = np.kron(I1, ref)
    ref[P.dirichlet_mask()] = 0.0
    assert np.abs(F - ref).max() < 1e-15


def read_trace():
    rows = []
    with open(os.path.join(HERE, "golden", "bratu_appB_trace.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                it, v = line.split()
                rows.append(float(v))
    return rows


def test_appendix_b_initial_residual_norm():
    trace = read_trace()
    U = O.open_uniform_knots(128, 2)
    P = O.Problem([U, U], [2, 2], lam=6.80, dirichlet=dirichlet_all(2))
    assert P.N == 130 * 130
    F = P.residual(np.zeros(P.N))
    assert abs(np.linalg.norm(F) - trace[0]) <= 1e-12 * trace[0]


@pytest.mark.slow
def test_appendix_b_newton_trace():
    # exact-solve Newton follows the printed trace to the accuracy of PETSc's CG
    trace = read_trace()
    U = O.open_uniform_knots(128, 2)
    P = O.Problem([U, U], [2, 2], lam=6.80, dirichlet=dirichlet_all(2))
    _, hist = O.newton(P, np.zeros(P.N))
    assert len(hist) == len(trace)
    for k in range(1, 5):
        assert abs(hist[k] - trace[k]) < 1e-5 * trace[k], (k, hist[k], trace[k])
    for k in (5, 6):
        assert abs(hist[k] - trace[k]) < 1e-4 * trace[k]
    assert hist[-1] <= 1e-10


# ----------------------------------------------------- closed-form Jacobian rows

def test_jacobian_at_zero_matches_kronecker_closed_form():
    # uniform quadratic C1: 1D mass row h/120 [1,26,66,26,1], stiffness 1/(6h) [-1,-2,6,-2,-1];
    # at U = 0 on the identity map, J = K x M + M x K - lambda M x M
    nel, lam = 10, 1.7
    h = 1.0 / nel
    m1 = h / 120.0 * np.array([1, 26, 66, 26, 1.0])
    k1 = 1.0 / (6.0 * h) * np.array([-1, -2, 6, -2, -1.0])
    U = O.open_uniform_knots(nel, 2)
    P = O.Problem([U, U], [2, 2], lam=lam)
    J = P.jacobian_csr(np.zeros(P.N)).toarray()
    n = nel + 2
    for i in range(4, n - 4):
        for j in range(4, n - 4):
            A = i + n * j
            for a in range(-2, 3):
                for b in range(-2, 3):
                    B = (i + a) + n * (j + b)
                    ref = k1[a + 2] * m1[b + 2] + m1[a + 2] * k1[b + 2] - lam * m1[a + 2] * m1[b + 2]
                    assert abs(J[A, B] - ref) < 1e-14 * (1 + abs(ref))


def test_stiffness_annihilates_constants_and_mass_total_is_area():
    kn, ctrl, w = W.quarter_annulus(3, 3)
    P0 = O.Problem(kn, [3] * 3, quad=[8] * 3, ctrl=ctrl, weights=w, lam=0.0)
    P1 = O.Problem(kn, [3] * 3, quad=[8] * 3, ctrl=ctrl, weights=w, lam=1.0)
    Z = np.zeros(P0.N)
    K = P0.jacobian_csr(Z)
    M = K - P1.jacobian_csr(Z)
    assert np.abs(K @ np.ones(P0.N)).max() < 1e-14 * abs(K).max()
    assert abs(M.sum() - 3.0 * math.pi / 4.0) < 1e-13
    # the unit cube
    U = O.open_uniform_knots(3, 2)
    Q0 = O.Problem([U] * 3, [2] * 3, lam=0.0)
    Q1 = O.Problem([U] * 3, [2] * 3, lam=1.0)
    Z = np.zeros(Q0.N)
    assert abs((Q0.jacobian_csr(Z) - Q1.jacobian_csr(Z)).sum() - 1.0) < 1e-14


def test_laplacian_of_reproduced_quadratic():
    # u = x^2 + y^2 is reproduced exactly (blossom coefficients); with lambda = 0 an
    # interior row is (grad N_A, grad u) = -(N_A, lap u) = -4 int N_A
    nel, p = 7, 2
    U = O.open_uniform_knots(nel, p)
    n = nel + p
    c = np.array([U[i + 1] * U[i + 2] for i in range(n)])  # blossom of x^2, p = 2
    Uc = (c[None, :] + c[:, None]).reshape(-1)  # natural order: x fastest
    P = O.Problem([U, U], [p, p], lam=0.0)
    F = P.residual(Uc)
    I1 = integral_1d(U, p)
    for i in range(p + 1, n - p - 1):
        for j in range(p + 1, n - p - 1):
            assert abs(F[i + n * j] - (-4.0 * I1[i] * I1[j])) < 1e-14


# ------------------------------------------------- brute force and consistency

def random_nurbs_2d(nel0, nel1, p, seed):
    kn, ctrl, w = W.quarter_annulus((nel0, nel1, 1), p)
    n0, n1 = len(kn[0]) - p - 1, len(kn[1]) - p - 1
    # take the z = 0 layer as a planar rational geometry
    ctrl2 = ctrl.reshape(-1, n1, n0, 3)[0, :, :, :2].reshape(-1, 2)
    w2 = w.reshape(-1, n1, n0)[0].reshape(-1)
    return kn[:2], ctrl2, w2


@pytest.mark.parametrize("case", ["identity2d", "nurbs2d", "identity3d", "kappa2d"])
def test_element_assembly_equals_global_bruteforce(case):
    if case == "identity2d":
        U = O.open_uniform_knots(2, 2)
        P = O.Problem([U, U], [2, 2], lam=1.3, dirichlet=dirichlet_all(2))
    elif case == "nurbs2d":
        kn, c, w = random_nurbs_2d(2, 2, 3, 0)
        P = O.Problem(kn, [3, 3], ctrl=c, weights=w, lam=2.0, dirichlet=dirichlet_all(2))
    elif case == "identity3d":
        U = O.open_uniform_knots(2, 2)
        P = O.Problem([U] * 3, [2] * 3, lam=2.0, dirichlet=dirichlet_all(3))
    else:
        U = O.open_uniform_knots(2, 2)
        lk = W.uniform(9, 16, -0.5, 0.5)
        P = O.Problem([U, U], [2, 2], lam=1.0, log_kappa=lk, dirichlet=dirichlet_all(2))
    Uc = W.uniform(5, P.N, -0.3, 0.3)
    F = P.residual(Uc)
    J = P.jacobian_csr(Uc).toarray()
    Fb, Jb = P.dense_bruteforce(Uc, fix=True)
    assert np.abs(F - Fb).max() < 1e-14 * max(1.0, np.abs(Fb).max())
    assert np.abs(J - Jb).max() < 1e-14 * max(1.0, np.abs(Jb).max())


@pytest.mark.parametrize("case", ["nurbs2d", "kappa2d"])
def test_jacobian_is_derivative_of_residual(case):
    if case == "nurbs2d":
        kn, c, w = random_nurbs_2d(3, 2, 2, 0)
        P = O.Problem(kn, [2, 2], ctrl=c, weights=w, lam=2.0, dirichlet=dirichlet_all(2))
    else:
        U = O.open_uniform_knots(3, 2)
        lk = W.uniform(3, 25, -0.5, 0.5)
        P = O.Problem([U, U], [2, 2], lam=1.0, log_kappa=lk)
    Uc = W.interior_field(P.n, 7, -0.5, 0.5)
    J = P.jacobian_csr(Uc).toarray()
    h = 1e-6
    for B in range(P.N):
        e = np.zeros(P.N)
        e[B] = h
        col = (P.residual(Uc + e) - P.residual(Uc - e)) / (2 * h)
        mask = np.ones(P.N, bool)
        if P.dirichlet:
            # boundary columns are zeroed on purpose (symmetric Dirichlet reading)
            if P.dirichlet_mask()[B]:
                continue
        assert np.abs(col[mask] - J[mask, B]).max() < 1e-7 * max(1.0, np.abs(J).max())


def test_jacobian_symmetric_on_nurbs():
    kn, c, w = random_nurbs_2d(3, 3, 3, 0)
    P = O.Problem(kn, [3, 3], ctrl=c, weights=w, lam=2.0, dirichlet=dirichlet_all(2))
    J = P.jacobian_csr(W.interior_field(P.n, 3)).toarray()
    assert np.abs(J - J.T).max() < 1e-15 * 8 * np.abs(J).max()


def test_greville_geometry_equals_identity_map():
    # linear precision: control points at the Greville abscissae give x = xi, so the
    # general rational/geometry path must reproduce the identity-map assembly
    p, nel = 3, 3
    U = O.open_uniform_knots(nel, p, 1)
    g = np.array([np.mean(U[i + 1:i + p + 1]) for i in range(len(U) - p - 1)])
    n = len(g)
    ctrl = np.stack(np.meshgrid(g, g, indexing="xy"), -1).reshape(-1, 2)
    Pi = O.Problem([U, U], [p, p], lam=1.5, dirichlet=dirichlet_all(2))
    Pg = O.Problem([U, U], [p, p], ctrl=ctrl, weights=np.ones(n * n), lam=1.5, dirichlet=dirichlet_all(2))
    Uc = W.interior_field([n, n], 11)
    assert np.abs(Pi.residual(Uc) - Pg.residual(Uc)).max() < 1e-15
    assert np.abs(Pi.jacobian(Uc) - Pg.jacobian(Uc)).max() < 1e-13


def test_annulus_geometry():
    kn, ctrl, w = W.quarter_annulus(5, 3)
    assert [len(k) - 4 for k in kn] == [8, 8, 8]
    P = O.Problem(kn, [3] * 3, ctrl=ctrl, weights=w)
    rng = np.random.default_rng(3)
    for xi in rng.random((30, 3)):
        x, det = P.map_point(xi)
        assert abs(math.hypot(x[0], x[1]) - (1.0 + xi[0])) < 1e-14
        assert abs(x[2] - xi[2]) < 1e-15
        assert det > 0
    # corners of the angular range
    x, _ = P.map_point([0.0, 0.0, 0.0])
    assert np.allclose(x, [1, 0, 0], atol=1e-15)
    x, _ = P.map_point([1.0, 1.0, 1.0])
    assert np.allclose(x, [0, 2, 1], atol=1e-14)


def test_annulus_parametrisation_is_orthogonal_and_its_weights_depend_on_the_angle():
    """The premise of the diagonal-S stiffness plan (reading 18): on the quarter annulus the
    three parametric directions of the map are mutually perpendicular at every point (radial,
    angular, height), so F^T F is diagonal and so is S = det F F^-1 F^-T; and the rational
    weights depend on the angle's index alone, so grad W is along xi_1 and (S g)_0 = (S g)_2 = 0.
    Checked on the oracle's map by central differences (their error, about 1e-9 of the column
    norms, is the tolerance) and on the control net exactly; a perturbed map fails the first."""
    kn, ctrl, w = W.quarter_annulus(6, 3)
    n = [len(k) - 4 for k in kn]
    Wn = w.reshape(n[2], n[1], n[0])
    assert np.array_equal(Wn, np.broadcast_to(Wn[:1, :, :1], Wn.shape))
    P = O.Problem(kn, [3] * 3, ctrl=ctrl, weights=w)
    rng = np.random.default_rng(7)
    h = 1e-6

    def columns(prob, xi):
        cols = []
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            xp, _ = prob.map_point(np.clip(xi + e, 0.0, 1.0))
            xm, _ = prob.map_point(np.clip(xi - e, 0.0, 1.0))
            cols.append((np.asarray(xp) - np.asarray(xm)) / (2 * h))
        return cols

    for xi in 0.05 + 0.9 * rng.random((12, 3)):
        c = columns(P, xi)
        for a in range(3):
            for b in range(a + 1, 3):
                assert abs(np.dot(c[a], c[b])) <= 1e-8 * np.linalg.norm(c[a]) * np.linalg.norm(c[b]), (xi, a, b)
    # the test can fail: a sheared copy of the same net is not orthogonal
    sheared = ctrl.copy()
    sheared[:, 0] += 0.2 * sheared[:, 2]
    Ps = O.Problem(kn, [3] * 3, ctrl=sheared, weights=w)
    c = columns(Ps, np.array([0.4, 0.3, 0.6]))
    assert abs(np.dot(c[0], c[2])) > 1e-3 * np.linalg.norm(c[0]) * np.linalg.norm(c[2])


def test_dirichlet_rows_and_columns():
    U = O.open_uniform_knots(3, 2)
    P = O.Problem([U, U], [2, 2], lam=1.0, dirichlet={(0, 0): 0.5, (1, 1): -0.25})
    Uc = W.uniform(4, P.N, -1, 1)
    F = P.residual(Uc)
    J = P.jacobian_csr(Uc).toarray()
    n = 5
    for A in range(P.N):
        i, j = A % n, A // n
        on = i == 0 or j == n - 1
        if on:
            g = -0.25 if j == n - 1 else 0.5
            assert F[A] == Uc[A] - g
            assert J[A, A] == 1.0 and np.count_nonzero(J[A]) == 1
            assert np.count_nonzero(J[:, A]) == 1


@pytest.mark.slow
def test_l2_convergence_rate():
    # manufactured u* = sin(pi x) sin(pi y): ||u_h - u*||_L2 = O(h^{p+1})
    for p in (2, 3):
        errs, hs = [], []
        for nel in (8, 16, 32):
            U = O.open_uniform_knots(nel, p)
            P = O.Problem([U, U], [p, p], lam=1.0, dirichlet=dirichlet_all(2), source=True)
            Uh, hist = O.newton(P, np.zeros(P.N))
            assert hist[-1] < 1e-10
            errs.append(P.l2_error(Uh))
            hs.append(1.0 / nel)
        slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
        assert abs(slope - (p + 1)) < 0.2, (p, slope, errs)


def test_lambda_beyond_fold_does_not_converge():
    # no solution exists above lambda_max = 6.80812 (Sec. 3.1)
    U = O.open_uniform_knots(16, 2)
    P = O.Problem([U, U], [2, 2], lam=7.5, dirichlet=dirichlet_all(2))
    _, hist = O.newton(P, np.zeros(P.N), max_it=30)
    assert not (hist[-1] <= 1e-10)


@pytest.mark.parametrize("case", [(2, 2, 8, 1.0, None), (2, 3, 6, 2.5, "kappa"), (3, 2, 3, 1.5, None), (3, 3, 3, 2.0, "annulus")])
def test_fd_jacobian_matches_the_analytic_jacobian(case):
    """Sec. 2.8 Eq. (fdjac): first-order differences with step sqrt(eps) sqrt(1 + ||U_e||)
    differ from the analytic Eq. (jacobian) by O(delta) + O(eps / delta) ~ 1e-8 relative;
    a dropped term, a wrong step or a transposed column fails by orders of magnitude."""
    dim, p, nel, lam, kind = case
    lk = None
    if kind == "annulus":
        kn, ctrl, w = W.quarter_annulus((nel, nel, nel), p)
    else:
        kn, ctrl, w = [O.open_uniform_knots(nel, p)] * dim, None, None
    n = [len(k) - p - 1 for k in kn]
    N = int(np.prod(n))
    if kind == "kappa":
        lk = W.uniform(3, N, -0.5, 0.5)
    bc = {(a, s): 0.0 for a in range(dim) for s in range(2)}
    prob = O.Problem(kn, [p] * dim, ctrl=ctrl, weights=w, lam=lam, log_kappa=lk, dirichlet=bc)
    U = W.uniform(11, N, -0.5, 0.5)
    J = prob.jacobian(U)
    Jfd = prob.jacobian_fd(U)
    err = np.abs(Jfd - J).max() / np.abs(J).max()
    assert err < 1e-6, err
    assert err > 1e-12  # it is an approximation, not the analytic formula again
    # the Dirichlet rows and columns are fixed the same way
    rowptr, colidx = prob.pattern()
    diag_rows = np.flatnonzero(prob.dirichlet_mask())[:5]
    for A in diag_rows:
        row = Jfd[rowptr[A]:rowptr[A + 1]]
        assert np.array_equal(row, (colidx[rowptr[A]:rowptr[A + 1]] == A).astype(float))


def test_fd_jacobian_of_a_linear_problem_is_the_stiffness():
    """lambda = 0: the residual is linear in U, so the difference quotient equals the
    stiffness up to the rounding of the differences (eps / delta ~ 1e-8)."""
    kn = [O.open_uniform_knots(6, 2)] * 2
    prob = O.Problem(kn, [2, 2], lam=0.0)
    U = W.uniform(2, prob.N, -1.0, 1.0)
    J = prob.jacobian(U)
    assert np.abs(prob.jacobian_fd(U) - J).max() <= 1e-6 * np.abs(J).max()


# ------------------------------------------- Sec. 4.2 time-dependent problems

def test_mass_matrix_linear_kronecker_and_volume():
    """(N_A, N_B) for p = 1 on a uniform mesh is the Kronecker product of the
    textbook 1D linear-element mass matrix h/6 tridiag(1, 4, 1) (h/3 at the two
    ends); on the NURBS annulus its entries sum to the volume 3 pi / 4."""
    nel = 5
    h = 1.0 / nel
    kn = O.open_uniform_knots(nel, 1)
    P = O.Problem([kn, kn], [1, 1], lam=0.0)
    M = P.mass_csr().toarray()
    M1 = np.diag(np.full(nel + 1, 4.0 * h / 6.0)) + np.diag(np.full(nel, h / 6.0), 1) + np.diag(np.full(nel, h / 6.0), -1)
    M1[0, 0] = M1[-1, -1] = h / 3.0
    assert np.abs(M - np.kron(M1, M1)).max() < 1e-16
    kn3, ctrl, w = W.quarter_annulus(3, 3)
    A = O.Problem(kn3, [3] * 3, quad=[8] * 3, ctrl=ctrl, weights=w, lam=0.0)
    assert abs(A.mass().sum() - 3.0 * math.pi / 4.0) < 1e-13


def test_alpha_parameters():
    """rho_inf = 1 gives the implicit midpoint rule (alpha_m = alpha_f = gamma = 1/2);
    every rho_inf gives gamma = 1/2 + alpha_m - alpha_f (second order)."""
    assert O.alpha_params(1.0) == (0.5, 0.5, 0.5)
    am, af, g = O.alpha_params(0.0)
    assert (am, af, g) == (1.5, 1.0, 1.0)


def _heat_mode(nel=6, p=2):
    """lambda = 0 (the heat equation M U-dot + K U = 0): lowest generalised
    eigenpair K phi = omega M phi on the free variables (a library eigensolver)."""
    import scipy.linalg as sla
    kn = O.open_uniform_knots(nel, p)
    P = O.Problem([kn, kn], [p, p], lam=0.0, dirichlet=dirichlet_all(2))
    free = ~P.dirichlet_mask()
    K = P.jacobian_csr(np.zeros(P.N)).toarray()[np.ix_(free, free)]
    M = P.mass_csr().toarray()[np.ix_(free, free)]
    om, vec = sla.eigh(K, M)
    phi = np.zeros(P.N)
    phi[free] = vec[:, 0]  # M-normalised
    Mf = np.zeros((P.N, P.N))
    Mf[np.ix_(free, free)] = M
    return P, phi, float(om[0]), Mf


def test_alpha_midpoint_amplification():
    """With rho_inf = 1 the method is the implicit midpoint rule, whose amplification
    of a mode y' = -omega y is (1 - omega dt / 2) / (1 + omega dt / 2) whatever the
    starting rate."""
    P, phi, om, Mf = _heat_mode()
    for dt in (0.01, 0.1, 1.0):
        U1, V1, hist = O.alpha_step(P, phi, 0.3 * phi, dt, 1.0)
        y1 = phi @ Mf @ U1
        assert abs(y1 - (1 - om * dt / 2) / (1 + om * dt / 2)) < 1e-11, dt


@pytest.mark.parametrize("rho", [0.0, 0.5])
def test_alpha_spectral_radius_at_infinite_step(rho):
    """Sec. 4.2: rho_inf is the spectral radius of the amplification matrix as
    dt -> infinity.  The step maps (y_n, ydot_n) of one mode linearly; its 2 x 2 matrix
    is read off two steps and its eigenvalues measured at omega dt ~ 2e9."""
    P, phi, om, Mf = _heat_mode()
    dt = 1e8
    G = np.zeros((2, 2))
    for j, (u0, v0) in enumerate([(phi, 0 * phi), (0 * phi, phi)]):
        U1, V1, _ = O.alpha_step(P, u0, v0, dt, rho)
        G[:, j] = [phi @ Mf @ U1, phi @ Mf @ V1]
    r = np.abs(np.linalg.eigvals(G)).max()
    assert abs(r - rho) < 1e-4, r


def test_alpha_second_order():
    """Second-order accuracy (Sec. 4.2): with the consistent start ydot_0 = -omega y_0
    the error of a mode at T against exp(-omega T) falls 4x per halving of dt."""
    P, phi, om, Mf = _heat_mode()
    T = 0.1
    errs = []
    for nsteps in (4, 8, 16, 32):
        dt = T / nsteps
        U, V = phi.copy(), -om * phi
        for _ in range(nsteps):
            U, V, _ = O.alpha_step(P, U, V, dt, 0.5)
        errs.append(abs(phi @ Mf @ U - math.exp(-om * T)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert all(abs(o - 2.0) < 0.15 for o in orders[1:]), orders


def test_alpha_step_keeps_a_steady_state():
    """A steady Bratu solution (Sec. 3.1) with zero rate is a fixed point of the step."""
    kn = O.open_uniform_knots(8, 2)
    P = O.Problem([kn, kn], [2, 2], lam=1.0, dirichlet=dirichlet_all(2))
    Us, hist = O.newton(P, np.zeros(P.N), atol=1e-13)
    assert hist[-1] <= 1e-13
    U1, V1, h = O.alpha_step(P, Us, np.zeros(P.N), 0.1, 0.5)
    assert np.abs(U1 - Us).max() < 1e-13 and np.abs(V1).max() < 1e-12


def test_transient_jacobian_is_derivative_of_transient_residual():
    """dR/dU + a dR/dU-dot against central differences of R(V + a x, U + x) on a
    NURBS annulus with random U and V (Dirichlet rows and columns removed)."""
    kn, ctrl, w = W.quarter_annulus(2, 2)
    P = O.Problem(kn, [2] * 3, ctrl=ctrl, weights=w, lam=1.5, dirichlet=dirichlet_all(3))
    rng = np.random.default_rng(3)
    free = ~P.dirichlet_mask()
    U = np.where(free, rng.uniform(-0.3, 0.3, P.N), 0.0)
    V = rng.uniform(-1, 1, P.N)
    a = 7.0
    rowptr, colidx = P.pattern()
    J = sp.csr_matrix((P.jacobian_ts(a, U), colidx, rowptr), shape=(P.N, P.N)).toarray()
    eps = 1e-6
    for B in np.flatnonzero(free)[::7]:
        e = np.zeros(P.N)
        e[B] = eps
        col = (P.residual_ts(V + a * e, U + e) - P.residual_ts(V - a * e, U - e)) / (2 * eps)
        assert np.abs(col[free] - J[free, B]).max() < 1e-7 * max(1.0, np.abs(J).max()), B


# ---------------------------------------------------- Sec. 2.4 periodic spaces

def test_unclamped_knots_match_the_papers_figure():
    """Eqs. (unclamp-left)-(unclamp-right) against the three knot vectors printed for
    the C^0, C^1 and C^2 periodic cubic spaces (tests/golden/unclamp_fig.txt)."""
    U = [0, 0, 0, 0, 0.2, 0.4, 0.6, 0.8, 1, 1, 1, 1]
    rows = np.loadtxt(os.path.join(HERE, "golden", "unclamp_fig.txt"))
    for row in rows:
        k = int(row[0])
        assert np.abs(O.unclamp_knots(U, 3, k) - row[1:]).max() < 1e-15, k


PERIODIC = [  # (p, nel, {axis: k}), 2D unless nel has three entries
    (2, (6, 5), {0: 1}),
    (3, (7, 6), {0: 2, 1: 0}),
    (3, (8, 5), {1: 1}),
    (2, (5, 4, 4), {0: 1, 2: 0}),
    (1, (6, 5), {0: 0}),
]


@pytest.mark.parametrize("case", PERIODIC)
def test_periodic_assembly_equals_global_bruteforce(case):
    """Element assembly with wrapped indices (Eq. map-wrap) against the dense brute
    force that evaluates every periodic function as the sum of the unclamped B-splines
    wrapping onto it; the wrapped BasisStencil pattern against element connectivity."""
    p, nel, per = case
    dim = len(nel)
    kn = [O.open_uniform_knots(nel[d], p) for d in range(dim)]
    P = O.Problem(kn, [p] * dim, lam=1.3, periodic=per)
    rng = np.random.default_rng(5)
    U = rng.uniform(-0.3, 0.3, P.N)
    F, J = P.dense_bruteforce(U, fix=False)
    assert np.abs(F - P.residual(U)).max() < 1e-14
    assert np.abs(J - P.jacobian_csr(U).toarray()).max() < 1e-13
    rowptr, colidx = P.pattern()
    mark = P.pattern_dense_from_elements()
    dense = np.zeros_like(mark)
    for A in range(P.N):
        dense[A, colidx[rowptr[A]:rowptr[A + 1]]] = 1
        assert np.all(np.diff(colidx[rowptr[A]:rowptr[A + 1]]) > 0)
    assert np.array_equal(dense, mark)


def test_fully_periodic_space_reproduces_constants_and_is_shift_invariant():
    """With both directions periodic the constant is in the space on every row (K 1 = 0),
    the mass totals the area, and on a uniform mesh M and K commute with the shift of
    the function index by one along x (circulant structure)."""
    p, nel = 3, 7
    kn = O.open_uniform_knots(nel, p)
    P = O.Problem([kn, kn], [p, p], lam=0.0, periodic={0: p - 1, 1: p - 1})
    K = P.jacobian_csr(np.zeros(P.N)).toarray()
    M = P.mass_csr().toarray()
    assert np.abs(K @ np.ones(P.N)).max() < 1e-13
    assert abs(M.sum() - 1.0) < 1e-14
    n0, n1 = P.n
    idx = np.arange(P.N)
    shift = ((idx % n0 + 1) % n0) + n0 * (idx // n0)
    assert np.abs(M[np.ix_(shift, shift)] - M).max() < 1e-15
    assert np.abs(K[np.ix_(shift, shift)] - K).max() < 1e-12


def test_periodic_laplacian_eigenvalue_converges_at_order_2p():
    """The lowest nonzero eigenvalue of -u'' = mu u on the periodic unit square is
    (2 pi)^2; the discrete generalised eigenvalue of (K, M) converges as h^(2p)."""
    import scipy.linalg as sla
    errs = []
    for nel in (6, 12):
        kn = O.open_uniform_knots(nel, 2)
        P = O.Problem([kn, kn], [2, 2], lam=0.0, periodic={0: 1, 1: 1})
        K = P.jacobian_csr(np.zeros(P.N)).toarray()
        M = P.mass_csr().toarray()
        mu = sla.eigh(K, M, eigvals_only=True)
        assert abs(mu[0]) < 1e-9
        errs.append(mu[1] - (2 * math.pi) ** 2)
    assert errs[0] > 0 and errs[1] > 0
    assert abs(math.log2(errs[0] / errs[1]) - 4.0) < 0.3, errs


def test_periodic_direction_with_x_independent_data_matches_natural_boundaries():
    """Bratu periodic in x with Dirichlet faces in y: by the translation symmetry the
    solution does not depend on x; so does the solution with natural (no) conditions on
    the x faces, and the two coefficient profiles along y coincide."""
    p, nel = 2, (6, 10)
    kx, ky = O.open_uniform_knots(nel[0], p), O.open_uniform_knots(nel[1], p)
    bc = {(1, 0): 0.0, (1, 1): 0.0}
    Pp = O.Problem([kx, ky], [p, p], lam=1.5, dirichlet=bc, periodic={0: p - 1})
    Pn = O.Problem([kx, ky], [p, p], lam=1.5, dirichlet=bc)
    Up, hp = O.newton(Pp, np.zeros(Pp.N), atol=1e-12)
    Un, hn = O.newton(Pn, np.zeros(Pn.N), atol=1e-12)
    assert hp[-1] <= 1e-12 and hn[-1] <= 1e-12
    Up = Up.reshape(Pp.n[1], Pp.n[0])
    Un = Un.reshape(Pn.n[1], Pn.n[0])
    assert np.abs(Up - Up[:, :1]).max() < 1e-13
    assert np.abs(Un - Un[:, :1]).max() < 1e-12
    assert np.abs(Up[:, 0] - Un[:, 0]).max() < 1e-12


def test_exact_full_annulus_as_a_periodic_space():
    """The closed annulus of four rational quarter arcs, periodic across the seam with
    C^0 continuity (k = 0): every point lies on the circle of its radius, constants are in
    the space, and the mass totals the area 3 pi (over-integrated rule)."""
    for p, nq in ((2, 4), (3, 3)):
        kn, ctrl, w = W.full_annulus(3, nq, p)
        P = O.Problem(kn, [p, p], ctrl=ctrl, weights=w, lam=0.0, periodic={1: 0}, quad=[p + 3, p + 3])
        rng = np.random.default_rng(p)
        for xi in rng.uniform(0, 1, (20, 2)):
            x, det = P.map_point(xi)
            assert abs(math.hypot(*x) - (1 + xi[0])) < 1e-14 and det > 0
        K = P.jacobian_csr(np.zeros(P.N))
        assert np.abs(K @ np.ones(P.N)).max() < 1e-13
        assert abs(P.mass().sum() - 3 * math.pi) < 1e-9


def test_unclamping_a_curve_keeps_it():
    """Sec. 2.4 (Algorithm 1's task): a quarter arc of degree four, unclamped for C^0-C^3,
    traces the same points on the parametric domain (evaluated with the oracle's
    Cox-de Boor recursion on both knot vectors)."""
    s = math.sqrt(0.5)
    U, Pw = W._refine_curve(np.array([[1.0, 0, 1], [s, s, s], [0, 1, 1.0]]), 4, 3)
    n = len(Pw)
    for k in range(4):
        V, Q = W.unclamp_curve(U, Pw, 4, k)
        assert np.abs(V - O.unclamp_knots(U, 4, k)).max() < 1e-15
        for xi in np.linspace(0.003, 0.997, 40):
            a = sum(O.bspline(i, 4, U, xi) * Pw[i] for i in range(n))
            b = sum(O.bspline(i, 4, V, xi) * Q[i] for i in range(n))
            assert np.abs(a - b).max() < 1e-13, (k, xi)


def test_unclamping_a_closed_curve_gives_periodic_control_points():
    """A closed uniform C^(p-1) curve written on the clamped knot vector (control points by
    least squares on the oracle's basis) unclamps to control points whose last p equal the
    first p: the wrapped periodic space's control points."""
    p, nel = 3, 8
    th = 2 * math.pi * np.arange(nel) / nel
    P = np.stack([np.cos(th), np.sin(th), np.ones(nel)], axis=1)   # periodic control points
    Pext = np.concatenate([P, P[:p]])                               # unclamped numbering
    U = O.open_uniform_knots(nel, p)
    V = O.unclamp_knots(U, p, p - 1)
    n = nel + p
    xs = np.linspace(0.001, 0.999, 4 * n)
    C = np.array([sum(O.bspline(i, p, V, x) * Pext[i] for i in range(n)) for x in xs])
    B = np.array([[O.bspline(i, p, U, x) for i in range(n)] for x in xs])
    Q = np.linalg.lstsq(B, C, rcond=None)[0]                         # the clamped description
    V2, P2 = W.unclamp_curve(U, Q, p, p - 1)
    assert np.abs(V2 - V).max() < 1e-15
    assert np.abs(P2 - Pext).max() < 1e-11
    assert np.abs(P2[-p:] - P2[:p]).max() < 1e-11


# ------------------------------------ row helpers against the whole assembly
# or_residual_rows / or_jacobian_rows compute selected rows from the elements that
# contain each row's function (Sec. 2.7: the support of N_A is p+1 spans per
# direction).  They check the full-size GPU runs, so they are pinned here to the
# whole-mesh element loop (Algorithm 3), row by row, on every face, edge and
# corner and on rows next to repeated or unequal knots.

def _boundary_and_sampled_rows(n, count, seed):
    idx = np.indices(n[::-1]).reshape(len(n), -1)[::-1]
    N = idx.shape[1]
    pick = np.zeros(N, dtype=bool)
    for d, nd in enumerate(n):
        for v in (0, 1, nd - 2, nd - 1):  # faces and the layer next to them
            pick |= idx[d] == v
    sel = np.flatnonzero(pick)
    rng = np.random.default_rng(seed)
    extra = rng.choice(N, size=min(count, N), replace=False)
    return np.unique(np.concatenate([sel, extra]))


ROW_CASES = [
    # (dim, p, knots factory, geometry, kappa, dirichlet)
    (2, 1, lambda: [W.uniform_open_knots(6, 1), W.graded_open_knots(5, 1, 3)], None, False, True),
    (2, 2, lambda: [W.graded_open_knots(6, 2, 1, extra=(2,)), W.graded_open_knots(5, 2, 2)], None, True, True),
    (2, 3, lambda: [W.uniform_open_knots(5, 3, 1), W.graded_open_knots(6, 3, 4, extra=(1, 4))], None, False, False),
    (2, 4, lambda: [W.graded_open_knots(4, 4, 5), W.uniform_open_knots(4, 4, 2)], None, False, True),
    (2, 3, None, "annulus", False, True),
    (3, 2, lambda: [W.graded_open_knots(4, 2, 6, extra=(2,)), W.uniform_open_knots(3, 2), W.graded_open_knots(3, 2, 7)],
     None, False, True),
    (3, 3, None, "annulus", True, True),
    (3, 4, lambda: [W.uniform_open_knots(2, 4, 2)] * 2 + [W.graded_open_knots(3, 4, 8)], None, False, False),
    (3, 1, lambda: [W.graded_open_knots(4, 1, 9), W.uniform_open_knots(3, 1), W.uniform_open_knots(3, 1)], None,
     False, True),
]


@pytest.mark.parametrize("case", ROW_CASES, ids=lambda c: "d%dp%d_%s_kap%d_bc%d" % (c[0], c[1], c[3], c[4], c[5]))
def test_row_helpers_equal_the_whole_mesh_assembly(case):
    dim, p, knots_f, geom, kap, bc = case
    ctrl = w = None
    if geom == "annulus":
        if dim == 3:
            knots, ctrl, w = W.quarter_annulus((3, 4, 2), p)
        else:
            knots, ctrl, w = random_nurbs_2d(4, 3, p, 0)
    else:
        knots = knots_f()
    n = [len(k) - p - 1 for k in knots]
    N = int(np.prod(n))
    lk = W.uniform(17, N, -0.5, 0.5) if kap else None
    prob = O.Problem(knots, [p] * dim, ctrl=ctrl, weights=w, lam=1.9, log_kappa=lk,
                     dirichlet=dirichlet_all(dim, 0.25) if bc else None)
    U = W.uniform(23, N, -0.4, 0.4)
    F = prob.residual(U)
    J = prob.jacobian(U)
    rowptr, _ = prob.pattern()
    rows = _boundary_and_sampled_rows(n, 20, 5)
    Fr = prob.residual_rows(U, rows)
    Jr = prob.jacobian_rows(U, rows)
    Jsel = np.concatenate([J[rowptr[r]:rowptr[r + 1]] for r in rows])
    sf, sj = np.abs(F).max(), np.abs(J).max()
    assert np.abs(Fr - F[rows]).max() <= 1e-14 * sf
    assert np.abs(Jr - Jsel).max() <= 1e-14 * sj
    # every row once, in a shuffled order: the helpers do not depend on the order asked
    perm = np.random.default_rng(1).permutation(N)
    assert np.abs(prob.residual_rows(U, perm) - F[perm]).max() <= 1e-14 * sf


# --------------------------------------------- colour-loop timing mode (OpenMP)

@pytest.mark.parametrize("case", [(2, 2, (9, 7), None), (2, 3, (6, 5), "graded"), (3, 3, (4, 3, 5), "annulus"),
                                  (3, 2, (5, 4, 3), "kappa"), (3, 1, (3, 3, 2), None)])
def test_colored_timing_mode_equals_the_serial_loops(case):
    """The timing mode visits the same elements with the same arithmetic in another
    order: equal to the serial oracle up to the rounding of the additions, and every
    element is visited exactly once (a skipped or doubled colour would show)."""
    dim, p, nel, kind = case
    ctrl = w = lk = None
    if kind == "annulus":
        knots, ctrl, w = W.quarter_annulus(nel, p)
    elif kind == "graded":
        knots = [W.graded_open_knots(nel[d], p, 50 + d, extra=(2,) if d == 0 else ()) for d in range(dim)]
    else:
        knots = [W.uniform_open_knots(nel[d], p) for d in range(dim)]
    n = [len(k) - p - 1 for k in knots]
    N = int(np.prod(n))
    if kind == "kappa":
        lk = W.uniform(3, N, -0.5, 0.5)
    prob = O.Problem(knots, [p] * dim, ctrl=ctrl, weights=w, lam=2.1, log_kappa=lk, dirichlet=dirichlet_all(dim, 0.1))
    U = W.uniform(4, N, -0.3, 0.3)
    F, Fc = prob.residual(U), prob.residual_colored(U)
    J, Jc = prob.jacobian(U), prob.jacobian_colored(U)
    assert np.abs(F - Fc).max() <= 1e-14 * np.abs(F).max()
    assert np.abs(J - Jc).max() <= 1e-14 * np.abs(J).max()
    assert O.num_threads() >= 1
