"""Parity of the CUDA path (through the C ABI) with the oracle.

Bar (from the method's statement of the target): FP64 residual and Jacobian
equal to the oracle within 1e-12 relative max-norm; CSR pattern bit-exact.
"""
import numpy as np
import pytest

import oracle as O
from paper_1305_4452_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1305_4452_gb300 import build
    build.build()
    O.build()


def iga():
    from paper_1305_4452_gb300 import iga as I
    return I


def bc_all(dim, v=0.0):
    return {(a, s): v for a in range(dim) for s in range(2)}


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def graded_knots(dim, p, nel, k=None):
    """Seeded unequal spans per direction; direction 0 also drops the continuity by one
    at its second interior knot (a repeated knot) when that keeps k >= 0."""
    out = []
    for d in range(dim):
        kk = p - 1 if k is None else k
        extra = (2,) if d == 0 and kk >= 1 and nel[d] > 2 else ()
        out.append(W.graded_open_knots(nel[d], p, 31 + d, k=k, extra=extra))
    return out


def perturbed_nurbs(knots, p, seed):
    """A rational map near the identity on the given knots: Greville control points moved by
    a smooth bump of amplitude 0.03 and weights drawn in [0.9, 1.1] (det J stays > 0)."""
    dim = len(knots)
    gr = [W.greville(kn, p) for kn in knots]
    mesh = np.meshgrid(*gr[::-1], indexing="ij")[::-1]  # natural order: axis 0 fastest
    X = np.stack([m.reshape(-1) for m in mesh], axis=1)
    bump = np.prod(np.sin(np.pi * X), axis=1)
    for d in range(dim):
        X[:, d] += 0.03 * bump * (1.0 if d == 0 else -1.0)
    return X, W.uniform(seed, X.shape[0], 0.9, 1.1)


def make_pair(dim, p, nel, lam=1.0, k=None, geom=None, kappa_seed=None, bc=True, dirichlet=None):
    """GPU discretisation and oracle problem on the same inputs.  geom: None (identity map
    on uniform knots), "annulus", "graded" (identity map, unequal spans and a repeated
    knot) or "graded_nurbs" (the same knots under a rational map)."""
    I = iga()
    nel = [nel] * dim if np.isscalar(nel) else list(nel)
    ctrl = weights = knots = None
    if geom in ("graded", "graded_nurbs"):
        knots = graded_knots(dim, p, nel, k)
        if geom == "graded_nurbs":
            ctrl, weights = perturbed_nurbs(knots, p, 41)
    elif geom == "annulus":
        kn, ctrl, weights = W.quarter_annulus(tuple(nel) if dim == 3 else (nel[0], nel[1], 1), p)
        if dim == 2:
            n0, n1 = len(kn[0]) - p - 1, len(kn[1]) - p - 1
            ctrl = ctrl.reshape(-1, n1, n0, 3)[0, :, :, :2].reshape(-1, 2)
            weights = weights.reshape(-1, n1, n0)[0].reshape(-1)
            kn = kn[:2]
        knots = kn
    else:
        knots = [W.uniform_open_knots(nel[d], p, k) for d in range(dim)]
    n = [len(kk) - p - 1 for kk in knots]
    lk = None
    if kappa_seed is not None:
        grf = dim == 2 and geom not in ("graded", "graded_nurbs")  # the field generator assumes uniform knots
        lk = W.grf_log_kappa(n, p, nel, kappa_seed) if grf else W.uniform(kappa_seed, int(np.prod(n)), -0.5, 0.5)
    if dirichlet is None:
        dirichlet = bc_all(dim) if bc else None
    disc = I.Discretization(dim, p, knots=knots, ctrl=ctrl, weights=weights, lam=lam, log_kappa=lk, dirichlet=dirichlet)
    prob = O.Problem(knots, [p] * dim, ctrl=ctrl, weights=weights, lam=lam, log_kappa=lk, dirichlet=dirichlet)
    return disc, prob, n


SMALL = [
    # (dim, p, nel, k, geom, kappa)
    (2, 2, 16, None, None, None),      # the 16x16 quadratic C1 configuration
    (2, 1, (7, 5), None, None, None),
    (2, 3, (6, 9), 1, None, None),     # reduced continuity
    (2, 4, (5, 4), None, None, None),
    (2, 3, (7, 6), None, "annulus", None),
    (2, 2, (9, 7), None, None, 3),     # kappa-weighted
    (3, 2, (7, 5, 3), None, None, None),
    (3, 3, (5, 6, 3), None, "annulus", None),
    (3, 1, (4, 3, 5), None, None, None),
    (3, 4, (3, 2, 3), 2, None, None),
    # unequal spans (Sec. 2.1 allows any non-decreasing knot vector), a repeated interior knot
    (2, 2, (9, 7), None, "graded", None),
    (2, 3, (7, 6), None, "graded", 5),
    (2, 4, (6, 5), None, "graded_nurbs", None),
    (2, 3, (8, 6), 1, "graded", None),
    (3, 2, (6, 5, 4), None, "graded", None),
    (3, 3, (5, 4, 4), None, "graded_nurbs", None),
    (3, 4, (4, 3, 3), None, "graded", None),
    # the sum-factorised geometry at the degrees where its per-block element count changes
    # (p = 1: 16 elements per block, p = 4: one), under a rational map; the diagonal-S plan
    # with a kappa field folded into S (annulus), and the general plan with kappa
    (3, 4, (3, 3, 2), None, "graded_nurbs", None),
    (3, 1, (4, 3, 3), None, "graded_nurbs", None),
    (2, 1, (6, 5), None, "graded_nurbs", None),
    (3, 3, (5, 4, 3), None, "annulus", 7),
    (2, 2, (8, 7), None, "annulus", 9),
    (3, 2, (4, 4, 3), None, "graded_nurbs", 11),
]


@pytest.mark.parametrize("case", SMALL, ids=lambda c: "d%dp%d_%s_%s_%s_%s" % (c[0], c[1], c[2], c[3], c[4], c[5]))
def test_small_full_parity(case):
    dim, p, nel, k, geom, kap = case
    disc, prob, n = make_pair(dim, p, nel, lam=1.7, k=k, geom=geom, kappa_seed=kap)
    U0 = W.interior_field(n, seed=11, lo=-0.3, hi=0.3)
    U = torch.tensor(U0, device="cuda")
    F = disc.form_residual(U).cpu().numpy()
    J = disc.form_jacobian(U).cpu().numpy()
    rp, ci = disc.pattern()
    rpo, cio = prob.pattern()
    assert np.array_equal(rp.cpu().numpy(), rpo)
    assert np.array_equal(ci.cpu().numpy(), cio)
    Fo = prob.residual(U0)
    Jo = prob.jacobian(U0)
    assert rel(F, Fo) <= TOL, rel(F, Fo)
    assert rel(J, Jo) <= TOL, rel(J, Jo)
    disc.close()


def test_no_dirichlet_and_mixed_faces():
    I = iga()
    p, nel = 2, (6, 5)
    knots = [W.uniform_open_knots(e, p) for e in nel]
    n = [len(kk) - p - 1 for kk in knots]
    for bc in (None, {(0, 0): 0.5, (1, 1): -0.25}):
        disc = I.Discretization(2, p, knots=knots, lam=0.9, dirichlet=bc)
        prob = O.Problem(knots, [p, p], lam=0.9, dirichlet=bc)
        U0 = W.uniform(4, int(np.prod(n)), -0.4, 0.4)
        U = torch.tensor(U0, device="cuda")
        assert rel(disc.form_residual(U).cpu().numpy(), prob.residual(U0)) <= TOL
        assert rel(disc.form_jacobian(U).cpu().numpy(), prob.jacobian(U0)) <= TOL
        disc.close()


def test_deterministic_bitwise():
    disc, prob, n = make_pair(3, 3, (5, 4, 3), geom="annulus")
    U = torch.tensor(W.interior_field(n, 5), device="cuda")
    F1, F2 = disc.form_residual(U).clone(), disc.form_residual(U).clone()
    J1, J2 = disc.form_jacobian(U).clone(), disc.form_jacobian(U).clone()
    assert torch.equal(F1, F2) and torch.equal(J1, J2)
    disc.close()


def test_appendix_b_initial_norm_on_gpu():
    I = iga()
    disc = I.Discretization(2, 2, nel=128, lam=6.80, dirichlet=bc_all(2))
    U = torch.zeros(disc.N, dtype=torch.float64, device="cuda")
    F = disc.form_residual(U)
    trace0 = 5.266384548611e-02  # Appendix B, iteration 0
    assert abs(torch.linalg.norm(F).item() - trace0) <= 1e-12 * trace0
    rep = disc.solve_newton(U)
    assert rep.fnorm <= 1e-10 and rep.status == 0
    # loose pin: the paper's run took 7 Newton steps
    assert 5 <= rep.newton_its <= 9
    disc.close()


def test_newton_config1_and_oracle_residual_at_solution():
    disc, prob, n = make_pair(2, 2, 16, lam=1.0)
    U0 = W.interior_field(n, seed=1)
    U = torch.tensor(U0, device="cuda")
    rep = disc.solve_newton(U)
    assert rep.status == 0 and rep.fnorm <= 1e-10
    Fo = prob.residual(U.cpu().numpy())
    assert np.linalg.norm(Fo) <= 1e-10 + 1e-12
    disc.close()


@pytest.mark.parametrize("jac_reuse", [0, 1])
def test_newton_3d_annulus_small(jac_reuse):
    I = iga()
    disc, prob, n = make_pair(3, 3, (8, 8, 6), lam=2.0, geom="annulus")
    U = torch.zeros(disc.N, dtype=torch.float64, device="cuda")
    o = I.newton_defaults()
    o.reuse_stiffness = jac_reuse
    rep = disc.solve_newton(U, o)
    assert rep.status == 0 and rep.fnorm <= 1e-10
    assert np.linalg.norm(prob.residual(U.cpu().numpy())) <= 1.5e-10
    disc.close()


def test_beyond_fold_reports_failure():
    I = iga()
    disc = I.Discretization(2, 2, nel=16, lam=7.5, dirichlet=bc_all(2))
    U = torch.zeros(disc.N, dtype=torch.float64, device="cuda")
    o = I.newton_defaults()
    o.max_newton = 25
    rep = disc.solve_newton(U, o, check=False)
    assert rep.status in (I.IGA_ENOCONV, I.IGA_EDIVERGED)
    assert rep.newton_its <= 25
    disc.close()


def test_nan_input_reports_enan():
    I = iga()
    disc = I.Discretization(2, 2, nel=8, lam=1.0, dirichlet=bc_all(2))
    U = torch.zeros(disc.N, dtype=torch.float64, device="cuda")
    U[disc.N // 2] = float("nan")
    rep = disc.solve_newton(U, check=False)
    assert rep.status == I.IGA_ENAN
    disc.close()


def sample_rows(N, count, seed):
    rows = np.unique(np.concatenate([[0, N - 1, N // 2], (W.uniform(seed, count) * N).astype(np.int64)]))
    return rows


@pytest.mark.slow
def test_full_size_annulus_64_cubed_sampled():
    """3D annulus, 64^3 cubic C2, lambda = 2: pattern bit-exact, sampled rows of F and J."""
    disc, prob, n = make_pair(3, 3, 64, lam=2.0, geom="annulus")
    assert disc.N == 300763 and disc.nnz == 95443993
    U0 = W.interior_field(n, seed=2)
    U = torch.tensor(U0, device="cuda")
    F = disc.form_residual(U).cpu().numpy()
    J = disc.form_jacobian(U)
    rp, ci = disc.pattern()
    rpo, cio = prob.pattern()
    assert np.array_equal(rp.cpu().numpy(), rpo) and np.array_equal(ci.cpu().numpy(), cio)
    rows = sample_rows(disc.N, 12, 77)
    Fo = prob.residual_rows(U0, rows)
    scale = np.abs(F).max()
    assert np.abs(F[rows] - Fo).max() <= TOL * scale
    Jo = prob.jacobian_rows(U0, rows)
    rp_h = rpo
    Jg = np.concatenate([J[rp_h[r]:rp_h[r + 1]].cpu().numpy() for r in rows])
    jscale = torch.abs(J).max().item()
    assert np.abs(Jg - Jo).max() <= TOL * jscale
    del J
    # the benchmark's solve (U = 0, FP64 Jacobian, GMRES + Jacobi): the oracle's residual at
    # the GPU's solution, on the sampled rows plus the rows next to every face
    U.zero_()
    rep = disc.solve_newton(U)
    assert rep.status == 0 and rep.fnorm <= 1e-10
    Us = U.cpu().numpy()
    edge = np.flatnonzero(~W.boundary_mask(n) & (np.indices(n[::-1]).reshape(3, -1)[::-1] == 1).any(axis=0))
    chk = np.unique(np.concatenate([rows, edge[(W.uniform(91, 64) * len(edge)).astype(np.int64)]]))
    Fs = prob.residual_rows(Us, chk)
    assert np.abs(Fs).max() <= 1e-10 * (1 + 1e-12), np.abs(Fs).max()
    disc.close()


@pytest.mark.slow
def test_full_size_cube_128_cubed_sampled():
    """3D unit cube, 128^3 quadratic, lambda = 2 (FP64 Jacobian): sampled rows."""
    disc, prob, n = make_pair(3, 2, 128, lam=2.0)
    assert disc.N == 2197000 and disc.nnz == 267089984
    U0 = W.interior_field(n, seed=3)
    U = torch.tensor(U0, device="cuda")
    F = disc.form_residual(U).cpu().numpy()
    rows = sample_rows(disc.N, 12, 78)
    assert np.abs(F[rows] - prob.residual_rows(U0, rows)).max() <= TOL * np.abs(F).max()
    J = disc.form_jacobian(U)
    rpo, _ = prob.pattern()
    Jg = np.concatenate([J[rpo[r]:rpo[r + 1]].cpu().numpy() for r in rows])
    assert np.abs(Jg - prob.jacobian_rows(U0, rows)).max() <= TOL * torch.abs(J).max().item()
    disc.close()


@pytest.mark.slow
def test_full_size_cube_48_cubed_quartic_sampled():
    """3D unit cube, 48^3 quartic C^3, lambda = 2: pattern counts, sampled rows of F and of
    the FP64 Jacobian at 1e-12, and of the BF16 element-GEMM Jacobian at the BF16 bound."""
    I = iga()
    disc, prob, n = make_pair(3, 4, 48, lam=2.0)
    assert disc.N == 140608 and disc.nnz == 89915392
    U0 = W.interior_field(n, seed=4)
    U = torch.tensor(U0, device="cuda")
    F = disc.form_residual(U).cpu().numpy()
    rows = sample_rows(disc.N, 6, 79)
    assert np.abs(F[rows] - prob.residual_rows(U0, rows)).max() <= TOL * np.abs(F).max()
    rpo, _ = prob.pattern()
    Jo = prob.jacobian_rows(U0, rows)
    J = disc.form_jacobian(U)
    Jg = np.concatenate([J[rpo[r]:rpo[r + 1]].cpu().numpy() for r in rows])
    jscale = torch.abs(J).max().item()
    assert np.abs(Jg - Jo).max() <= TOL * jscale
    del J
    Jb = disc.form_jacobian(U, prec=I.IGA_JAC_BF16)
    Jbg = np.concatenate([Jb[rpo[r]:rpo[r + 1]].double().cpu().numpy() for r in rows])
    assert np.linalg.norm(Jbg - Jo) <= 1.5e-5 * np.linalg.norm(Jo)  # measured 3.6e-6
    disc.close()


@pytest.mark.slow
def test_full_size_cube_128_cubed_bf16_element_gemm_sampled():
    """128^3 quadratic: sampled rows of the BF16 tensor-core Jacobian against the oracle's
    FP64 rows, within the BF16 bound."""
    I = iga()
    disc, prob, n = make_pair(3, 2, 128, lam=2.0)
    U0 = W.interior_field(n, seed=3)
    U = torch.tensor(U0, device="cuda")
    Jb = disc.form_jacobian(U, prec=I.IGA_JAC_BF16)
    rows = sample_rows(disc.N, 12, 80)
    rpo, _ = prob.pattern()
    Jbg = np.concatenate([Jb[rpo[r]:rpo[r + 1]].double().cpu().numpy() for r in rows])
    Jo = prob.jacobian_rows(U0, rows)
    assert np.linalg.norm(Jbg - Jo) <= 2e-5 * np.linalg.norm(Jo)  # measured 6.5e-6
    disc.close()


@pytest.mark.parametrize("jac", ["fp64", "fp32"])
def test_newton_cg_matches_gmres_solution(jac):
    I = iga()
    disc, prob, n = make_pair(3, 3, (8, 8, 6), lam=2.0, geom="annulus")
    o = I.newton_defaults()
    o.jac = I.IGA_FP64 if jac == "fp64" else I.IGA_JAC_FP32
    Ug = torch.zeros(disc.N, dtype=torch.float64, device="cuda")
    disc.solve_newton(Ug, o)
    o.ksp = I.IGA_KSP_CG
    Uc = torch.zeros_like(Ug)
    rep = disc.solve_newton(Uc, o)
    assert rep.status == 0 and rep.fnorm <= 1e-10
    assert torch.abs(Ug - Uc).max().item() <= 1e-8
    assert np.linalg.norm(prob.residual(Uc.cpu().numpy())) <= 1.5e-10
    disc.close()


@pytest.mark.parametrize("nel,restart", [((8, 8, 6), 60), ((24, 24, 20), 12)], ids=["2blocks", "20blocks_restarted"])
@pytest.mark.parametrize("fused", [1, 0], ids=["fused", "passes"])
@pytest.mark.parametrize("refine", ["never", "ifneeded", "always"])
def test_gmres_cgs_refinement_modes_reach_the_oracle_solution(refine, fused, nel, restart):
    """GMRES with classical Gram-Schmidt once (PETSc's default refinement type), where
    needed, or twice; in one cooperative launch per Arnoldi step or by the separate pass
    kernels; a row partition of 2 or 20 blocks with a ragged last block, with and without
    restarts.  Newton reaches ||F|| <= 1e-10, the oracle's residual at the GPU's solution is
    at that level, and the solution agrees with the default solve's (the solutions of
    different Krylov iterations agree to about the tolerance over the Jacobian's smallest
    singular value)."""
    I = iga()
    disc, prob, n = make_pair(3, 3, nel, lam=2.0, geom="annulus")
    Ur = torch.zeros(disc.N, dtype=torch.float64, device="cuda")
    disc.solve_newton(Ur)
    o = I.newton_defaults()
    o.gmres_restart = restart
    o.gmres_cgs_refine = {"never": I.IGA_CGS_REFINE_NEVER, "ifneeded": I.IGA_CGS_REFINE_IFNEEDED,
                          "always": I.IGA_CGS_REFINE_ALWAYS}[refine]
    disc.set_gmres_fused(fused)
    U = torch.zeros_like(Ur)
    rep = disc.solve_newton(U, o)
    assert rep.status == 0 and rep.fnorm <= 1e-10
    assert torch.abs(U - Ur).max().item() <= 1e-8
    assert np.linalg.norm(prob.residual(U.cpu().numpy())) <= 1.5e-10
    disc.close()


@pytest.mark.parametrize("dim,p,nel", [(3, 3, (10, 9, 8)), (3, 2, (9, 8, 7)), (2, 3, (12, 10))])
def test_diagonal_s_plan_equals_the_general_plan(dim, p, nel):
    """The annulus's orthogonal parametrisation (radial and angular directions perpendicular,
    the height separate, weights a function of the angle) selects the diagonal-S plan, which
    drops the off-diagonal S and the zero weight-gradient terms that the geometry cache holds
    at rounding level.  Its FP64 and FP32 Jacobians agree with the general plan's to that
    level (a dropped term that is not zero would show at 1e-3 or more), they differ from them
    in the last bits (so the other plan did run), and the FP64 one equals the oracle's at
    1e-12."""
    I = iga()
    disc, prob, n = make_pair(dim, p, nel, lam=2.0, geom="annulus")
    U0 = W.interior_field(n, seed=5)
    U = torch.tensor(U0, device="cuda")
    Ja = disc.form_jacobian(U)
    Ja32 = disc.form_jacobian(U, prec=I.IGA_JAC_FP32)
    disc.set_jacobian_plan(1)
    Jg = disc.form_jacobian(U)
    Jg32 = disc.form_jacobian(U, prec=I.IGA_JAC_FP32)
    disc.set_jacobian_plan(0)
    scale = torch.abs(Jg).max().item()
    assert torch.abs(Ja - Jg).max().item() <= 5e-13 * scale
    assert not torch.equal(Ja, Jg)
    assert torch.abs(Ja32.double() - Jg32.double()).max().item() <= 1e-6 * scale
    assert rel(Ja.cpu().numpy(), prob.jacobian(U0)) <= TOL
    with pytest.raises(I.IgaError):
        disc.set_jacobian_plan(2)
    disc.close()


def test_gmres_option_rejections():
    I = iga()
    disc, prob, n = make_pair(2, 2, (6, 6), lam=1.0)
    U = torch.zeros(disc.N, dtype=torch.float64, device="cuda")
    for bad in (-1, 3):
        o = I.newton_defaults()
        o.gmres_cgs_refine = bad
        with pytest.raises(I.IgaError) as ei:
            disc.solve_newton(U, o)
        assert ei.value.status == I.IGA_EINVAL
    with pytest.raises(I.IgaError) as ei:
        disc.set_gmres_fused(2)
    assert ei.value.status == I.IGA_EINVAL
    disc.close()


@pytest.mark.parametrize("case", [SMALL[0], SMALL[2], SMALL[4], SMALL[6], SMALL[7], SMALL[9]],
                         ids=lambda c: "d%dp%d_%s_%s" % (c[0], c[1], c[3], c[4]))
def test_apply_jacobian_matches_oracle_csr_product(case):
    """The operator product reads no column indices (they follow from the stencil
    structure); it must equal the CSR product of the oracle's Jacobian up to the
    rounding of a dot product: |y - y_ref| <= 1e-13 (|J| |x|) row by row."""
    import scipy.sparse as sp
    dim, p, nel, k, geom, kap = case
    disc, prob, n = make_pair(dim, p, nel, lam=1.3, k=k, geom=geom, kappa_seed=kap)
    U0 = W.interior_field(n, seed=2, lo=-0.2, hi=0.2)
    rpo, cio = prob.pattern()
    Jo = prob.jacobian(U0)
    A = sp.csr_matrix((Jo, cio, rpo), shape=(disc.N, disc.N))
    absA = sp.csr_matrix((np.abs(Jo), cio, rpo), shape=(disc.N, disc.N))
    x = W.uniform(9, disc.N, -1.0, 1.0)
    xd = torch.tensor(x, device="cuda")
    U = torch.tensor(U0, device="cuda")
    J = disc.form_jacobian(U)
    y = disc.apply_jacobian(J, xd).cpu().numpy()
    assert np.all(np.abs(y - A @ x) <= 1e-13 * (absA @ np.abs(x)) + 1e-300)
    # FP32 values are widened; the product stays FP64
    J32 = disc.form_jacobian(U, prec=iga().IGA_JAC_FP32)
    A32 = sp.csr_matrix((J32.cpu().numpy().astype(np.float64), cio, rpo), shape=(disc.N, disc.N))
    y32 = disc.apply_jacobian(J32, xd).cpu().numpy()
    assert np.all(np.abs(y32 - A32 @ x) <= 1e-13 * (abs(A32) @ np.abs(x)) + 1e-300)
    y2 = disc.apply_jacobian(J, xd).cpu().numpy()
    assert np.array_equal(y, y2)
    disc.close()


@pytest.mark.parametrize("case", [(2, 2, (9, 7), None), (3, 3, (4, 5, 3), "annulus"), (3, 2, (5, 4, 3), None)],
                         ids=["d2p2", "d3p3_annulus", "d3p2"])
def test_newton_split_residual_matches_oracle(case):
    """After the first step the FP64 Newton solver evaluates F as K U plus the
    reaction term (K: stiffness without the Dirichlet fix, assembled once per
    solve).  One step from a rough start with nonzero Dirichlet data: the norm it
    reports must be the oracle's ||F(U_1)|| at U_1 (relative 1e-12)."""
    I = iga()
    dim, p, nel, geom = case
    # two Dirichlet faces, natural conditions elsewhere: lambda small enough for a solution to exist
    disc, prob, n = make_pair(dim, p, nel, lam=0.4, geom=geom, dirichlet={(0, 0): 0.5, (1, 1): -0.25})
    U0 = W.uniform(21, disc.N, -0.3, 0.3)
    U = torch.tensor(U0, device="cuda")
    o = I.newton_defaults()
    o.max_newton = 1
    rep = disc.solve_newton(U, o, check=False)
    assert rep.newton_its == 1
    U1 = U.cpu().numpy()
    f0 = np.linalg.norm(prob.residual(U0))
    f1 = np.linalg.norm(prob.residual(U1))
    assert abs(rep.fnorm0 - f0) <= 1e-12 * f0
    assert abs(rep.fnorm_hist[1] - f1) <= 1e-12 * f1, (rep.fnorm_hist[1], f1)
    # the solve continues to convergence from there
    rep2 = disc.solve_newton(U, I.newton_defaults())
    assert rep2.fnorm <= 1e-10
    assert np.linalg.norm(prob.residual(U.cpu().numpy())) <= 1e-10 * (1 + 1e-12)
    disc.close()


MF_CASES = [(2, 2, (9, 7), None, "graded", None), (3, 3, (5, 4, 4), None, "graded_nurbs", None),
            (2, 2, (9, 7), None, None, None), (2, 3, (7, 6), None, "annulus", None), (2, 2, (9, 7), None, None, 3),
            (3, 3, (5, 4, 3), None, "annulus", None), (3, 2, (5, 4, 3), 0, None, None), (3, 4, (3, 2, 3), 2, None, None)]


@pytest.mark.parametrize("case", MF_CASES, ids=lambda c: "d%dp%d_%s_%s_%s" % (c[0], c[1], c[3], c[4], c[5]))
def test_matrix_free_product_and_diagonal_match_the_assembled_jacobian(case):
    """J(U) x computed on the fly (no assembled matrix) equals the CSR product of the
    oracle's Jacobian up to the rounding of the sums, |dy| <= 1e-12 (|J| |x|) row by
    row; the diagonal equals the oracle's at 1e-12 relative.  Nonzero Dirichlet data
    and nonzero x on Dirichlet variables check the masked columns and identity rows."""
    import scipy.sparse as sp
    dim, p, nel, k, geom, kap = case
    disc, prob, n = make_pair(dim, p, nel, lam=1.3, k=k, geom=geom, kappa_seed=kap,
                              dirichlet={(0, 0): 0.3, (1, 1): -0.2, (0, 1): 0.1})
    U0 = W.uniform(5, disc.N, -0.3, 0.3)
    x = W.uniform(6, disc.N, -1.0, 1.0)
    rpo, cio = prob.pattern()
    Jo = prob.jacobian(U0)
    A = sp.csr_matrix((Jo, cio, rpo), shape=(disc.N, disc.N))
    absA = sp.csr_matrix((np.abs(Jo), cio, rpo), shape=(disc.N, disc.N))
    U, xd = torch.tensor(U0, device="cuda"), torch.tensor(x, device="cuda")
    y = disc.apply_jacobian_mf(U, xd).cpu().numpy()
    assert np.all(np.abs(y - A @ x) <= 1e-12 * (absA @ np.abs(x)) + 1e-300)
    d = disc.jacobian_diagonal(U).cpu().numpy()
    assert rel(d, A.diagonal()) <= TOL
    disc.close()


@pytest.mark.parametrize("ksp", ["gmres", "cg"])
def test_matrix_free_newton_reaches_the_oracle_solution(ksp):
    I = iga()
    disc, prob, n = make_pair(3, 3, (6, 5, 4), lam=2.0, geom="annulus")
    U = torch.zeros(disc.N, dtype=torch.float64, device="cuda")
    o = I.newton_defaults()
    o.jac = I.IGA_JAC_NONE
    o.ksp = I.IGA_KSP_CG if ksp == "cg" else I.IGA_KSP_GMRES
    rep = disc.solve_newton(U, o)
    assert rep.status == 0 and rep.fnorm <= 1e-10
    assert np.linalg.norm(prob.residual(U.cpu().numpy())) <= 1e-10 * (1 + 1e-12)
    U2 = torch.zeros_like(U)
    rep2 = disc.solve_newton(U2, I.newton_defaults())
    assert abs(rep.newton_its - rep2.newton_its) <= 1
    # both iterates meet ||F|| <= 1e-10; they differ by at most ||J^-1|| (||F1|| + ||F2||)
    assert torch.max(torch.abs(U - U2)).item() <= 1e-8
    disc.close()


FD_CASES = [(2, 2, (9, 7), None, None, None), (2, 4, (5, 4), None, None, None), (2, 3, (7, 6), None, "annulus", None),
            (2, 2, (9, 7), None, None, 3), (3, 2, (5, 4, 3), 0, None, None), (3, 3, (5, 4, 3), None, "annulus", None),
            (3, 1, (4, 3, 5), None, None, None)]


@pytest.mark.parametrize("case", FD_CASES, ids=lambda c: "d%dp%d_%s_%s_%s" % (c[0], c[1], c[3], c[4], c[5]))
def test_local_fd_jacobian_matches_the_oracle(case):
    """Sec. 2.8 Eq. (fdjac) on the GPU against the oracle's implementation of the same
    formula: both are FP64 difference quotients with step ~1.5e-8 sqrt(1 + ||U_e||), so
    their rounding differs by ~eps |F_q| / delta ~ 1e-8 |J|; the bar is 1e-7 relative in
    the max norm.  Against the analytic Jacobian the FD error is O(delta) (< 1e-6)."""
    I = iga()
    dim, p, nel, k, geom, kap = case
    disc, prob, n = make_pair(dim, p, nel, lam=1.4, k=k, geom=geom, kappa_seed=kap,
                              dirichlet={(0, 0): 0.2, (1, 1): -0.1, (0, 1): 0.0})
    U0 = W.uniform(8, disc.N, -0.4, 0.4)
    U = torch.tensor(U0, device="cuda")
    J = disc.form_jacobian(U, prec=I.IGA_JAC_FD).cpu().numpy()
    Jfd = prob.jacobian_fd(U0)
    assert rel(J, Jfd) <= 1e-7, rel(J, Jfd)
    assert rel(J, prob.jacobian(U0)) <= 1e-6
    J2 = disc.form_jacobian(U, prec=I.IGA_JAC_FD).cpu().numpy()
    assert np.array_equal(J, J2)
    disc.close()


def test_newton_with_fd_jacobian_reaches_the_oracle_solution():
    I = iga()
    disc, prob, n = make_pair(3, 2, (6, 5, 4), lam=2.0)
    U = torch.zeros(disc.N, dtype=torch.float64, device="cuda")
    o = I.newton_defaults()
    o.jac = I.IGA_JAC_FD
    rep = disc.solve_newton(U, o)
    assert rep.status == 0 and rep.fnorm <= 1e-10
    assert np.linalg.norm(prob.residual(U.cpu().numpy())) <= 1e-10 * (1 + 1e-12)
    disc.close()


# ------------------------------------------- Sec. 4.2 time-dependent problems

TS_CASES = [(2, 3, (7, 6), None, "graded_nurbs", None), (3, 2, (5, 4, 3), None, "graded", None),
            (2, 2, (9, 7), None, None, None), (2, 3, (7, 6), None, "annulus", None), (2, 2, (9, 7), None, None, 3),
            (3, 3, (4, 5, 3), None, "annulus", None), (3, 2, (5, 4, 3), None, None, None), (2, 4, (5, 4), None, None, None)]


@pytest.mark.parametrize("case", TS_CASES, ids=lambda c: "d%dp%d_%s_%s_%s" % (c[0], c[1], c[3], c[4], c[5]))
def test_transient_residual_and_shifted_jacobian_match_the_oracle(case):
    dim, p, nel, k, geom, kap = case
    disc, prob, n = make_pair(dim, p, nel, lam=1.3, k=k, geom=geom, kappa_seed=kap)
    U0 = W.interior_field(n, seed=21, lo=-0.3, hi=0.3)
    V0 = W.uniform(22, disc.N, -1.0, 1.0)
    U = torch.tensor(U0, device="cuda")
    V = torch.tensor(V0, device="cuda")
    F = disc.form_residual_ts(V, U).cpu().numpy()
    Fo = prob.residual_ts(V0, U0)
    assert rel(F, Fo) <= TOL, rel(F, Fo)
    for shift in (0.0, 37.5):
        J = disc.form_jacobian_ts(shift, U).cpu().numpy()
        Jo = prob.jacobian_ts(shift, U0)
        assert rel(J, Jo) <= TOL, (shift, rel(J, Jo))
    J32 = disc.form_jacobian_ts(37.5, U, prec=iga().IGA_JAC_FP32).cpu().numpy().astype(np.float64)
    assert rel(J32, prob.jacobian_ts(37.5, U0)) <= 1e-5
    # the steady residual is unchanged by the transient calls (state restored)
    assert rel(disc.form_residual(U).cpu().numpy(), prob.residual(U0)) <= TOL
    disc.close()


def _stage_residual(prob, Un, Vn, U1, V1, dt, rho):
    am, af, g = O.alpha_params(rho)
    return prob.residual_ts(Vn + am * (V1 - Vn), Un + af * (U1 - Un))


@pytest.mark.parametrize("jac", ["fp64", "fp32_cg", "mf"])
def test_alpha_steps_match_the_oracle(jac):
    """Three generalized-alpha steps of the transient Bratu problem (Sec. 4.2) from a
    random start: U_{n+1}, U-dot_{n+1} against the oracle's steps (which iterate on
    U-dot_{n+1}, not on the stage value), and the oracle's stage residual at the GPU's
    result."""
    I = iga()
    disc, prob, n = make_pair(2, 2, (12, 10), lam=1.5)
    U0 = W.interior_field(n, seed=31, lo=-0.2, hi=0.2)
    V0 = np.zeros(disc.N)
    U = torch.tensor(U0, device="cuda")
    V = torch.tensor(V0, device="cuda")
    o = I.newton_defaults()
    o.atol = 1e-12
    if jac == "fp32_cg":
        o.jac, o.ksp = I.IGA_JAC_FP32, I.IGA_KSP_CG
    elif jac == "mf":
        o.jac = I.IGA_JAC_NONE
    Uo, Vo = U0.copy(), V0.copy()
    dt, rho = 0.02, 0.5
    for step in range(3):
        Un, Vn = Uo, Vo
        rep = disc.ts_alpha_step(U, V, dt, rho, o)
        assert rep.status == 0 and rep.fnorm <= 1e-12
        Uo, Vo, hist = O.alpha_step(prob, Un, Vn, dt, rho, atol=1e-13)
        Ug, Vg = U.cpu().numpy(), V.cpu().numpy()
        assert np.abs(Ug - Uo).max() <= 1e-10 * np.abs(Uo).max(), (step, np.abs(Ug - Uo).max())
        assert np.abs(Vg - Vo).max() <= 1e-8 * np.abs(Vo).max(), (step, np.abs(Vg - Vo).max())
        assert np.linalg.norm(_stage_residual(prob, Un, Vn, Ug, Vg, dt, rho)) <= 2e-12
        Uo, Vo = Ug, Vg  # continue both from the GPU's state
    disc.close()


def test_alpha_step_3d_annulus_and_midpoint():
    I = iga()
    disc, prob, n = make_pair(3, 3, (4, 5, 3), lam=2.0, geom="annulus")
    U0 = W.interior_field(n, seed=41, lo=-0.1, hi=0.1)
    V0 = np.zeros(disc.N)
    for rho in (1.0, 0.0):
        U = torch.tensor(U0, device="cuda")
        V = torch.tensor(V0, device="cuda")
        o = I.newton_defaults()
        o.atol = 1e-12
        rep = disc.ts_alpha_step(U, V, 0.05, rho, o)
        assert rep.status == 0
        Uo, Vo, _ = O.alpha_step(prob, U0, V0, 0.05, rho, atol=1e-13)
        Ug, Vg = U.cpu().numpy(), V.cpu().numpy()
        # what is unique: the stage equations hold at the GPU's result; the iterates of the
        # two solvers (each stopped at ||R|| <= 1e-12) differ by ||J^-1|| ||R||, ||J^-1|| ~ 30 here
        assert np.linalg.norm(_stage_residual(prob, U0, V0, Ug, Vg, 0.05, rho)) <= 2e-12
        assert np.abs(Ug - Uo).max() <= 1e-9 * np.abs(Uo).max()
        assert np.abs(Vg - Vo).max() <= 1e-7 * np.abs(Vo).max()
    disc.close()


def test_alpha_step_rejects_bad_input_and_keeps_state():
    I = iga()
    disc, prob, n = make_pair(2, 2, (6, 5), lam=1.0)
    U = torch.tensor(W.interior_field(n, seed=5, lo=-0.1, hi=0.1), device="cuda")
    V = torch.zeros_like(U)
    U_before = U.clone()
    for dt, rho in ((0.0, 0.5), (0.1, 1.5), (0.1, -0.1), (float("nan"), 0.5)):
        with pytest.raises(I.IgaError) as ei:
            disc.ts_alpha_step(U, V, dt, rho)
        assert ei.value.status == I.IGA_EINVAL
    o = I.newton_defaults()
    o.jac = I.IGA_JAC_BF16
    with pytest.raises(I.IgaError):
        disc.ts_alpha_step(U, V, 0.1, 0.5, o)
    # a Newton failure (one iteration allowed, tight tolerance) leaves U_n and U-dot_n
    o = I.newton_defaults()
    o.max_newton, o.atol = 1, 1e-30
    rep = disc.ts_alpha_step(U, V, 0.1, 0.5, o, check=False)
    assert rep.status != 0
    assert torch.equal(U, U_before) and torch.count_nonzero(V).item() == 0
    disc.close()


# ---------------------------------------------------- Sec. 2.4 periodic spaces

PER_CASES = [
    # (dim, p, nel, interior k, periodic {axis: k}, rational weights, kappa seed)
    (2, 2, (9, 7), None, {0: 1}, False, None),
    (2, 3, (7, 8), None, {0: 2, 1: 0}, False, None),   # no Dirichlet face at all
    (2, 2, (8, 9), None, {1: 1}, True, None),          # rational basis, identity map
    (2, 2, (9, 7), None, {0: 1}, False, 3),            # kappa-weighted
    (2, 3, (4, 5), None, {0: 2}, False, None),         # n - k = 4 < 2p + 1: columns wrap onto themselves
    (2, 1, (6, 5), None, {0: 0}, False, None),
    (2, 3, (6, 5), 1, {0: 1}, False, None),            # C^1 inside, C^1 across the boundary
    (3, 2, (5, 4, 4), None, {0: 1, 2: 0}, False, None),
    (3, 3, (6, 5, 4), None, {1: 2}, True, None),
]


def make_periodic_pair(dim, p, nel, k, per, rational, kappa_seed, lam=1.3):
    I = iga()
    knots = [W.uniform_open_knots(nel[d], p, k) for d in range(dim)]
    bc = {(a, s): 0.0 for a in range(dim) if a not in per for s in range(2)}
    prob = O.Problem(knots, [p] * dim, lam=lam, dirichlet=bc, periodic=per)
    weights = W.uniform(7, prob.N, 0.8, 1.2) if rational else None
    lk = W.uniform(kappa_seed, prob.N, -0.5, 0.5) if kappa_seed is not None else None
    prob = O.Problem(knots, [p] * dim, lam=lam, dirichlet=bc, periodic=per, weights=weights, log_kappa=lk)
    disc = I.Discretization(dim, p, knots=knots, lam=lam, dirichlet=bc, periodic=per, weights=weights, log_kappa=lk)
    return disc, prob


@pytest.mark.parametrize("case", PER_CASES, ids=lambda c: "d%dp%d_%s_k%s_%s_w%d_kap%s" % (
    c[0], c[1], "x".join(map(str, c[2])), c[3], "".join("%d%d" % kv for kv in c[4].items()), c[5], c[6]))
def test_periodic_pattern_residual_jacobian_match_the_oracle(case):
    disc, prob = make_periodic_pair(*case)
    assert disc.N == prob.N
    rng = np.random.default_rng(13)
    U0 = np.where(prob.dirichlet_mask(), 0.0, rng.uniform(-0.3, 0.3, prob.N))
    U = torch.tensor(U0, device="cuda")
    rp, ci = disc.pattern()
    rpo, cio = prob.pattern()
    assert np.array_equal(rp.cpu().numpy(), rpo) and np.array_equal(ci.cpu().numpy(), cio)
    F = disc.form_residual(U).cpu().numpy()
    assert rel(F, prob.residual(U0)) <= TOL, rel(F, prob.residual(U0))
    J = disc.form_jacobian(U)
    Jo = prob.jacobian(U0)
    assert rel(J.cpu().numpy(), Jo) <= TOL, rel(J.cpu().numpy(), Jo)
    J32 = disc.form_jacobian(U, prec=iga().IGA_JAC_FP32).cpu().numpy().astype(np.float64)
    assert rel(J32, Jo) <= 1e-5
    x0 = rng.uniform(-1, 1, prob.N)
    y = disc.apply_jacobian(J, torch.tensor(x0, device="cuda")).cpu().numpy()
    Jc = prob.jacobian_csr(U0)
    yo = Jc @ x0
    assert np.all(np.abs(y - yo) <= 1e-13 * (abs(Jc) @ np.abs(x0)))
    V0 = rng.uniform(-1, 1, prob.N)
    Fts = disc.form_residual_ts(torch.tensor(V0, device="cuda"), U).cpu().numpy()
    assert rel(Fts, prob.residual_ts(V0, U0)) <= TOL
    Jts = disc.form_jacobian_ts(21.0, U).cpu().numpy()
    assert rel(Jts, prob.jacobian_ts(21.0, U0)) <= TOL
    disc.close()


@pytest.mark.parametrize("jac", ["fp64_gmres", "fp32_cg"])
def test_periodic_newton_reaches_the_oracle_solution(jac):
    I = iga()
    disc, prob = make_periodic_pair(2, 2, (12, 10), None, {0: 1}, False, None, lam=1.5)
    U = torch.zeros(disc.N, dtype=torch.float64, device="cuda")
    o = I.newton_defaults()
    if jac == "fp32_cg":
        o.jac, o.ksp = I.IGA_JAC_FP32, I.IGA_KSP_CG
    rep = disc.solve_newton(U, o)
    assert rep.status == 0 and rep.fnorm <= 1e-10
    Ug = U.cpu().numpy()
    assert np.linalg.norm(prob.residual(Ug)) <= 1e-10 * (1 + 1e-12)
    Uo, hist = O.newton(prob, np.zeros(prob.N), atol=1e-12)
    assert np.abs(Ug - Uo).max() <= 1e-8
    disc.close()


def test_periodic_alpha_step_matches_the_oracle():
    I = iga()
    disc, prob = make_periodic_pair(3, 2, (5, 4, 6), None, {0: 1, 1: 1}, False, None, lam=1.0)
    rng = np.random.default_rng(17)
    U0 = np.where(prob.dirichlet_mask(), 0.0, rng.uniform(-0.2, 0.2, prob.N))
    V0 = np.zeros(prob.N)
    U = torch.tensor(U0, device="cuda")
    V = torch.tensor(V0, device="cuda")
    o = I.newton_defaults()
    o.atol = 1e-12
    rep = disc.ts_alpha_step(U, V, 0.03, 0.5, o)
    assert rep.status == 0
    Uo, Vo, _ = O.alpha_step(prob, U0, V0, 0.03, 0.5, atol=1e-13)
    Ug, Vg = U.cpu().numpy(), V.cpu().numpy()
    assert np.linalg.norm(_stage_residual(prob, U0, V0, Ug, Vg, 0.03, 0.5)) <= 2e-12
    assert np.abs(Ug - Uo).max() <= 1e-9 * np.abs(Uo).max()
    assert np.abs(Vg - Vo).max() <= 1e-7 * np.abs(Vo).max()
    disc.close()


def test_periodic_rejections():
    I = iga()
    disc, prob = make_periodic_pair(2, 2, (6, 5), None, {0: 1}, False, None)
    with pytest.raises(I.IgaError):
        I._check(I.lib().iga_set_boundary_value(disc.h, 0, 0, 0.0), disc.h)
    U = torch.zeros(disc.N, dtype=torch.float64, device="cuda")
    with pytest.raises(I.IgaError):
        disc.form_jacobian(U, prec=I.IGA_JAC_BF16)
    with pytest.raises(I.IgaError):
        disc.apply_jacobian_mf(U, U.clone())
    o = I.newton_defaults()
    o.jac = I.IGA_JAC_NONE
    with pytest.raises(I.IgaError):
        disc.solve_newton(U, o)
    disc.close()
    for nel, per in (((6, 5), {0: 2}), ((1, 5), {0: 1})):  # k > p - 1; n - k < k + 1
        with pytest.raises(I.IgaError):
            I.Discretization(2, 2, nel=list(nel), periodic=per)


@pytest.mark.parametrize("case", [(2, 2, 6, 12, None), (2, 3, 5, 10, None), (3, 2, 4, 9, 3)],
                         ids=["d2p2", "d2p3", "d3p2"])
def test_periodic_ring_geometry_matches_the_oracle(case):
    """A mapped periodic space: the ring with a C^(p-1) periodic angular direction, its
    control points given per wrapped function; residual, Jacobian and a Newton solve."""
    I = iga()
    dim, p, nel_r, nel_t, nel_z = case
    knots, ctrl = W.ring(nel_r, nel_t, p, nel_z=nel_z)
    per = {1: p - 1}
    bc = {(a, s): 0.0 for a in range(dim) if a != 1 for s in range(2)}
    prob = O.Problem(knots, [p] * dim, ctrl=ctrl, lam=1.2, dirichlet=bc, periodic=per)
    disc = I.Discretization(dim, p, knots=knots, ctrl=ctrl, lam=1.2, dirichlet=bc, periodic=per)
    assert disc.N == prob.N == ctrl.shape[0]
    rng = np.random.default_rng(23)
    U0 = np.where(prob.dirichlet_mask(), 0.0, rng.uniform(-0.3, 0.3, prob.N))
    U = torch.tensor(U0, device="cuda")
    assert rel(disc.form_residual(U).cpu().numpy(), prob.residual(U0)) <= TOL
    assert rel(disc.form_jacobian(U).cpu().numpy(), prob.jacobian(U0)) <= TOL
    Us = torch.zeros_like(U)
    rep = disc.solve_newton(Us, I.newton_defaults())
    assert rep.status == 0
    assert np.linalg.norm(prob.residual(Us.cpu().numpy())) <= 1e-10 * (1 + 1e-12)
    disc.close()


@pytest.mark.parametrize("p,nel_r,nel_q", [(2, 4, 3), (3, 3, 2)])
def test_periodic_exact_full_annulus_matches_the_oracle(p, nel_r, nel_q):
    """The exact NURBS annulus, periodic across the seam with C^0 continuity; Dirichlet
    on the inner and outer circles: residual, Jacobian and Newton against the oracle."""
    I = iga()
    kn, ctrl, w = W.full_annulus(nel_r, nel_q, p)
    bc = {(0, 0): 0.0, (0, 1): 0.0}
    prob = O.Problem(kn, [p, p], ctrl=ctrl, weights=w, lam=1.0, dirichlet=bc, periodic={1: 0})
    disc = I.Discretization(2, p, knots=kn, ctrl=ctrl, weights=w, lam=1.0, dirichlet=bc, periodic={1: 0})
    assert disc.N == prob.N
    rng = np.random.default_rng(31)
    U0 = np.where(prob.dirichlet_mask(), 0.0, rng.uniform(-0.3, 0.3, prob.N))
    U = torch.tensor(U0, device="cuda")
    assert rel(disc.form_residual(U).cpu().numpy(), prob.residual(U0)) <= TOL
    assert rel(disc.form_jacobian(U).cpu().numpy(), prob.jacobian(U0)) <= TOL
    Us = torch.zeros_like(U)
    rep = disc.solve_newton(Us, I.newton_defaults())
    assert rep.status == 0
    assert np.linalg.norm(prob.residual(Us.cpu().numpy())) <= 1e-10 * (1 + 1e-12)
    disc.close()


@pytest.mark.parametrize("dim,p,nel,k", [(2, 2, (7, 6), None), (2, 3, (6, 5), 1), (3, 2, (5, 4, 3), None), (3, 3, (4, 3, 3), None)])
def test_identity_map_plan_matches_the_general_plan(dim, p, nel, k):
    """Without control points the Jacobian stages use the plan of an identity map with unit
    weights (geometry factors g = 0, S diagonal); the same cube given its Greville points
    as control points (x = xi by linear precision) takes the general plan.  Both equal the
    oracle, and each other to rounding."""
    I = iga()
    knots = [W.uniform_open_knots(nel[d], p, k) for d in range(dim)]
    n = [len(kk) - p - 1 for kk in knots]
    g = [W.greville(knots[d], p) for d in range(dim)]
    mesh = np.meshgrid(*g[::-1], indexing="ij")  # axis 0 fastest in the flattened order
    ctrl = np.stack([m.reshape(-1) for m in mesh[::-1]], axis=1).copy()
    bc = bc_all(dim)
    plain = I.Discretization(dim, p, knots=knots, lam=1.3, dirichlet=bc)
    mapped = I.Discretization(dim, p, knots=knots, ctrl=ctrl, lam=1.3, dirichlet=bc)
    prob = O.Problem(knots, [p] * dim, lam=1.3, dirichlet=bc)
    U0 = W.interior_field(n, 11)
    U = torch.tensor(U0, device="cuda")
    Jp = plain.form_jacobian(U).cpu().numpy()
    Jm = mapped.form_jacobian(U).cpu().numpy()
    Jo = prob.jacobian(U0)
    assert rel(Jp, Jo) <= TOL and rel(Jm, Jo) <= TOL
    assert rel(Jp, Jm) <= 1e-13
    Jp32 = plain.form_jacobian(U, prec=I.IGA_JAC_FP32).cpu().numpy().astype(np.float64)
    Jm32 = mapped.form_jacobian(U, prec=I.IGA_JAC_FP32).cpu().numpy().astype(np.float64)
    assert rel(Jp32, Jo) <= 1e-5 and rel(Jm32, Jo) <= 1e-5
    plain.close()
    mapped.close()
