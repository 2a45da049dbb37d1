"""Mixed-precision Jacobian (tensor-core element matrices, BF16/TF32 operands, FP32
accumulation) against the FP64 oracle, and Newton steered by it.

There is no exact value to pin a rounded Jacobian to ("parity unpinned"); the
tests bound its relative Frobenius error by the operand precision (unit roundoff
2^-9 for BF16, 2^-11 for TF32, amplified by the cancellation between the
stiffness and reaction terms) and check what stays exact: the pattern, the
Dirichlet identity rows and zero columns, determinism, and that Newton driven by
it still reaches ||F||_2 <= 1e-10 on the FP64 residual.
"""
import numpy as np
import pytest

import oracle as O
from paper_1305_4452_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# Relative Frobenius error bounds per case, about 3x the errors these deterministic
# kernels give on GB300 (measured: in the comments), so that a change that made an
# error a few times larger fails.  For scale: the unit roundoff is 2^-9 = 2.0e-3 for
# BF16 and 2^-11 = 4.9e-4 for TF32; the split constant operand (a rounded part plus its
# rounded remainder) takes most cases far below it.
FRO_TOL = {"bf16": 2e-3, "tf32": 3e-4}   # the loosest case of each type (3D p = 1, non-uniform knots)
CASE_TOL = {  # case id -> (bf16, tf32)
    "d2p2_16_None_False": (3e-4, 4e-5),            # measured 1.08e-4, 1.23e-5
    "d2p3_(9, 7)_None_False": (5e-4, 2.5e-4),      # 1.80e-4, 7.66e-5
    "d2p2_(12, 10)_None_True": (1.2e-3, 1.5e-4),   # 3.77e-4, 4.77e-5 (kappa field)
    "d3p2_(6, 5, 4)_None_False": (2.5e-4, 4e-5),   # 7.50e-5, 1.37e-5
    "d3p3_(5, 4, 4)_annulus_False": (1.5e-4, 2e-5),  # 4.82e-5, 6.52e-6
    "d3p1_(5, 4, 3)_None_False": (4e-3, 3e-4),     # 1.22e-3, 8.73e-5 (p = 1: no split operand)
}


@pytest.fixture(scope="module")
def I():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1305_4452_gb300 import build, iga
    build.build()
    O.build()
    return iga


def bc_all(dim):
    return {(a, s): 0.0 for a in range(dim) for s in range(2)}


def pair(I, dim, p, nel, lam, geom=None, kappa=False):
    nel = [nel] * dim if np.isscalar(nel) else list(nel)
    ctrl = weights = lk = None
    if geom == "annulus":
        knots, ctrl, weights = W.quarter_annulus(tuple(nel), p)
    else:
        knots = [W.uniform_open_knots(nel[d], p) for d in range(dim)]
    n = [len(k) - p - 1 for k in knots]
    if kappa:
        lk = W.grf_log_kappa(n, p, nel, 7)
    disc = I.Discretization(dim, p, knots=knots, ctrl=ctrl, weights=weights, lam=lam, log_kappa=lk, dirichlet=bc_all(dim))
    prob = O.Problem(knots, [p] * dim, ctrl=ctrl, weights=weights, lam=lam, log_kappa=lk, dirichlet=bc_all(dim))
    return disc, prob, n


CASES = [(2, 2, 16, None, False), (2, 3, (9, 7), None, False), (2, 2, (12, 10), None, True),
         (3, 2, (6, 5, 4), None, False), (3, 3, (5, 4, 4), "annulus", False), (3, 1, (5, 4, 3), None, False)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "d%dp%d_%s_%s_%s" % c)
@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_mixed_jacobian_error_and_exact_structure(I, case, prec):
    dim, p, nel, geom, kappa = case
    disc, prob, n = pair(I, dim, p, nel, 1.5, geom, kappa)
    U0 = W.interior_field(n, seed=3, lo=-0.3, hi=0.3)
    U = torch.tensor(U0, device="cuda")
    code = I.IGA_JAC_BF16 if prec == "bf16" else I.IGA_JAC_TF32
    Jm = disc.form_jacobian(U, prec=code)
    Jm2 = disc.form_jacobian(U, prec=code)
    assert torch.equal(Jm, Jm2)  # deterministic
    Jm = Jm.double().cpu().numpy()
    Jo = prob.jacobian(U0)
    err = np.linalg.norm(Jm - Jo) / np.linalg.norm(Jo)
    assert err < CASE_TOL["d%dp%d_%s_%s_%s" % case][0 if prec == "bf16" else 1], err
    # Dirichlet rows/columns are exact
    rowptr, colidx = prob.pattern()
    mask = prob.dirichlet_mask()
    rows = np.repeat(np.arange(prob.N), np.diff(rowptr))
    fixed = mask[rows] | mask[colidx]
    assert np.array_equal(Jm[fixed], Jo[fixed])
    disc.close()


def test_tf32_more_accurate_than_bf16(I):
    disc, prob, n = pair(I, 3, 2, (6, 5, 4), 2.0)
    U0 = W.interior_field(n, seed=4)
    U = torch.tensor(U0, device="cuda")
    Jo = prob.jacobian(U0)
    e = {}
    for name, code in (("bf16", I.IGA_JAC_BF16), ("tf32", I.IGA_JAC_TF32)):
        Jm = disc.form_jacobian(U, prec=code).double().cpu().numpy()
        e[name] = np.linalg.norm(Jm - Jo) / np.linalg.norm(Jo)
    assert e["tf32"] < e["bf16"]
    disc.close()


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_newton_with_mixed_jacobian_reaches_fp64_tolerance(I, prec):
    for dim, p, nel, geom, lam in ((2, 2, 16, None, 1.0), (3, 3, (8, 8, 6), "annulus", 2.0), (2, 3, 32, None, 6.0)):
        disc, prob, n = pair(I, dim, p, nel, lam, geom)
        U = torch.zeros(disc.N, dtype=torch.float64, device="cuda")
        o = I.newton_defaults()
        o.jac = I.IGA_JAC_BF16 if prec == "bf16" else I.IGA_JAC_TF32
        rep = disc.solve_newton(U, o)
        assert rep.status == 0 and rep.fnorm <= 1e-10
        assert np.linalg.norm(prob.residual(U.cpu().numpy())) <= 1.5e-10
        disc.close()


# 3D p = 4 where the T tile of the whole K does not fit in shared memory: TF32 (512 K
# values x 4 B per pair row), and BF16 and TF32 on a general map (1280 K values).  Bounds
# about 3x the errors measured on GB300: 3.56e-6, 4.89e-5, 4.66e-6.
QUARTIC_TOL = {("tf32", None): 1.2e-5, ("bf16", "annulus"): 1.5e-4, ("tf32", "annulus"): 1.5e-5}


@pytest.mark.parametrize("prec,geom", list(QUARTIC_TOL), ids=lambda c: str(c))
def test_quartic_3d_element_gemm_in_k_passes(I, prec, geom):
    """K in passes with one tensor-memory accumulator per element tile of the group: the
    error stays within the operand precision's bound, the Dirichlet rows and columns are
    exact, the result is deterministic, and Newton driven by it reaches ||F|| <= 1e-10."""
    disc, prob, n = pair(I, 3, 4, (5, 3, 3), 1.5, geom)
    U0 = W.interior_field(n, seed=5, lo=-0.3, hi=0.3)
    U = torch.tensor(U0, device="cuda")
    code = I.IGA_JAC_BF16 if prec == "bf16" else I.IGA_JAC_TF32
    Jm = disc.form_jacobian(U, prec=code)
    assert torch.equal(Jm, disc.form_jacobian(U, prec=code))
    Jm = Jm.double().cpu().numpy()
    Jo = prob.jacobian(U0)
    err = np.linalg.norm(Jm - Jo) / np.linalg.norm(Jo)
    assert err < QUARTIC_TOL[(prec, geom)], err
    rowptr, colidx = prob.pattern()
    for A in np.flatnonzero(prob.dirichlet_mask()):
        seg = slice(rowptr[A], rowptr[A + 1])
        assert np.array_equal(Jm[seg], (colidx[seg] == A).astype(float))
    Us = torch.zeros(disc.N, dtype=torch.float64, device="cuda")
    o = I.newton_defaults()
    o.jac = code
    r = disc.solve_newton(Us, o)
    assert r.status == 0 and r.fnorm <= 1e-10
    assert np.linalg.norm(prob.residual(Us.cpu().numpy())) <= 1e-10 * 1.01
    disc.close()


def test_bf16_element_gemm_quartic_3d(I):
    """3D p = 4 (the 48^3 quartic configuration's degree) through the element GEMM."""
    disc, prob, n = pair(I, 3, 4, (5, 3, 3), 1.5)
    U0 = W.interior_field(n, seed=5, lo=-0.3, hi=0.3)
    Jm = disc.form_jacobian(torch.tensor(U0, device="cuda"), prec=I.IGA_JAC_BF16).double().cpu().numpy()
    Jo = prob.jacobian(U0)
    assert np.linalg.norm(Jm - Jo) / np.linalg.norm(Jo) < 1.5e-4  # measured 4.34e-5
    disc.close()


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_nonuniform_knots_use_the_per_element_contraction(I, prec):
    """Knot vectors with no repeated span lengths: every element its own type, so the
    per-element tensor-core contraction serves them; same error bound."""
    rng = np.random.default_rng(9)
    knots = []
    for nel in (40, 36):
        inner = np.sort(rng.uniform(0.0, 1.0, nel - 1))
        knots.append(np.concatenate([[0.0] * 3, inner, [1.0] * 3]))
    bc = bc_all(2)
    disc = I.Discretization(2, 2, knots=knots, lam=1.5, dirichlet=bc)
    prob = O.Problem(knots, [2, 2], lam=1.5, dirichlet=bc)
    U0 = np.where(prob.dirichlet_mask(), 0.0, rng.uniform(-0.3, 0.3, prob.N))
    code = I.IGA_JAC_BF16 if prec == "bf16" else I.IGA_JAC_TF32
    Jm = disc.form_jacobian(torch.tensor(U0, device="cuda"), prec=code).double().cpu().numpy()
    Jo = prob.jacobian(U0)
    assert np.linalg.norm(Jm - Jo) / np.linalg.norm(Jo) < FRO_TOL[prec]  # measured 7.44e-4, 1.01e-4
    disc.close()


@pytest.mark.parametrize("case", CASES[:5], ids=lambda c: "d%dp%d_%s_%s_%s" % c)
def test_fp32_sum_factorised_jacobian(I, case):
    # FP32 storage and arithmetic on the CUDA cores: error at the FP32 unit roundoff scale
    dim, p, nel, geom, kappa = case
    disc, prob, n = pair(I, dim, p, nel, 1.5, geom, kappa)
    U0 = W.interior_field(n, seed=3, lo=-0.3, hi=0.3)
    Jm = disc.form_jacobian(torch.tensor(U0, device="cuda"), prec=I.IGA_JAC_FP32).double().cpu().numpy()
    Jo = prob.jacobian(U0)
    assert np.linalg.norm(Jm - Jo) / np.linalg.norm(Jo) < 1e-5
    disc.close()


def test_newton_with_fp32_jacobian(I):
    disc, prob, n = pair(I, 3, 3, (8, 8, 6), 2.0, "annulus")
    U = torch.zeros(disc.N, dtype=torch.float64, device="cuda")
    o = I.newton_defaults()
    o.jac = I.IGA_JAC_FP32
    rep = disc.solve_newton(U, o)
    assert rep.status == 0 and rep.fnorm <= 1e-10
    disc.close()


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_element_gemm_newton_steps_on_a_fine_mesh(I, prec):
    """On a fine uniform mesh a systematic rounding of the shared basis products would
    slow Newton down; with the split constant operand Newton takes the FP64 step count
    (+1) from the zero start."""
    bc = bc_all(3)
    steps = {}
    for name, code in (("fp64", I.IGA_FP64), (prec, I.IGA_JAC_BF16 if prec == "bf16" else I.IGA_JAC_TF32)):
        disc = I.Discretization(3, 2, nel=64, lam=2.0, dirichlet=bc)
        U = torch.zeros(disc.N, dtype=torch.float64, device="cuda")
        o = I.newton_defaults()
        o.jac = code
        rep = disc.solve_newton(U, o)
        assert rep.status == 0
        steps[name] = rep.newton_its
        disc.close()
    assert steps[prec] <= steps["fp64"] + 1, steps


@pytest.mark.parametrize("p,nel,prec", [(2, 16, "bf16"), (4, (5, 3, 3), "tf32")], ids=["p2_bf16", "p4_tf32_k_passes"])
def test_bounded_pipeline_wait_gives_up_and_the_next_call_is_correct(I, p, nel, prec):
    """Failure detection in the allowed form: a bounded wait on a barrier that nothing
    arrives on.  With the stall hook the element GEMM's wait gives up after the (short)
    limit and the call reports IGA_ETIMEOUT; the kernel freed its tensor memory (the next
    calls allocate it again in every CTA and complete), and their Jacobians are
    bit-identical to one assembled before the stall.  Both the one-pass GEMM and the
    K-pass one (four accumulators, 512 tensor-memory columns per CTA)."""
    import ctypes
    disc, prob, n = pair(I, 3, p, nel, 1.5)  # uniform meshes with repeated element types
    code = I.IGA_JAC_BF16 if prec == "bf16" else I.IGA_JAC_TF32
    U = torch.tensor(W.interior_field(n, seed=3, lo=-0.3, hi=0.3), device="cuda")
    ref = disc.form_jacobian(U, prec=code).clone()
    L = I.lib()
    assert L.iga_set_wait_limit(disc.h, 0.02) == I.IGA_OK
    assert L.iga_inject_stall(disc.h) == I.IGA_OK
    vals = torch.full((disc.nnz,), float("nan"), dtype=torch.float32, device="cuda")
    rc = L.iga_form_jacobian(disc.h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(vals.data_ptr()), code)
    assert rc == I.IGA_ETIMEOUT, rc
    assert b"gave up" in L.iga_last_error(disc.h)
    assert L.iga_set_wait_limit(disc.h, 2.0) == I.IGA_OK
    for _ in range(2):
        assert torch.equal(disc.form_jacobian(U, prec=code), ref)
    # a Newton solve on the same handle after the give-up
    Us = torch.zeros(disc.N, dtype=torch.float64, device="cuda")
    o = I.newton_defaults()
    o.jac = code
    assert disc.solve_newton(Us, o).status == 0
    assert L.iga_set_wait_limit(disc.h, 0.0) == I.IGA_EINVAL
    disc.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_newton_with_the_sliced_fp32_product_reaches_the_oracle_solution(I, prec):
    """3D quadratic (p <= 2: the Krylov products run on the sliced copy of the FP32
    Jacobian), rows on every face: Newton reaches ||F|| <= 1e-10 and the oracle's residual
    at the GPU's solution meets it too; GMRES and CG agree."""
    disc, prob, n = pair(I, 3, 2, (14, 11, 9), 2.5)
    sols = []
    for ksp in (I.IGA_KSP_GMRES, I.IGA_KSP_CG):
        U = torch.zeros(disc.N, dtype=torch.float64, device="cuda")
        o = I.newton_defaults()
        o.jac = I.IGA_JAC_FP32 if prec == "fp32" else I.IGA_JAC_BF16
        o.ksp = ksp
        rep = disc.solve_newton(U, o)
        assert rep.status == 0 and rep.fnorm <= 1e-10
        Uh = U.cpu().numpy()
        assert np.linalg.norm(prob.residual(Uh)) <= 1.5e-10
        sols.append(Uh)
    assert np.abs(sols[0] - sols[1]).max() <= 1e-8
    disc.close()
