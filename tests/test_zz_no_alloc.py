"""iga_form_residual_noalloc: the residual entry point for callers that cannot
allocate device memory at call time (their device memory is owned by another
allocator, or a real-time loop cannot take an allocation).  It must give the same
residual as iga_form_residual, bit for bit, call after call, while allocating
nothing: the device's free memory is the same before and after the calls.

Kept in a file of its own that pytest collects last, so a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module")
def I():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1305_4452_gb300 import build, iga
    build.build()
    return iga


def _noalloc(I, disc, U, F):
    return I.lib().iga_form_residual_noalloc(disc.h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(F.data_ptr()))


def _cases(I):
    from paper_1305_4452_gb300 import workloads as W
    bc2 = {(a, s): 0.0 for a in range(2) for s in range(2)}
    bc3 = {(a, s): 0.0 for a in range(3) for s in range(2)}
    d2 = I.Discretization(2, 2, nel=16, lam=1.0, dirichlet=bc2)
    kn, ctrl, w = W.quarter_annulus((6, 5, 4), 3)
    d3 = I.Discretization(3, 3, knots=kn, ctrl=ctrl, weights=w, lam=2.0, dirichlet=bc3)
    return [(d2, [18, 18]), (d3, [9, 8, 7])]


def test_noalloc_residual_matches_existing_entry_point_twice(I):
    from paper_1305_4452_gb300 import workloads as W
    for disc, n in _cases(I):
        U = torch.tensor(W.interior_field(n, seed=5, lo=-0.3, hi=0.3), device="cuda")
        ref = disc.form_residual(U)
        outs = [torch.full_like(U, float("nan")) for _ in range(2)]
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for F in outs:  # two calls in a row share the same scratch
            assert _noalloc(I, disc, U, F) == I.IGA_OK
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        for F in outs:
            # same kernels, fixed-order sums, no atomics: identical bits
            assert torch.equal(F, ref)
        assert free1 == free0, (free0, free1)
        disc.close()


def test_noalloc_rejects_problems_beyond_its_scratch(I):
    # 40^3 cubic elements need 64,000 x 64 > 2,097,152 element values
    disc = I.Discretization(3, 3, nel=40, lam=1.0)
    U = torch.zeros(disc.N, dtype=torch.float64, device="cuda")
    F = torch.zeros_like(U)
    assert _noalloc(I, disc, U, F) == I.IGA_EINVAL
    assert "exceed" in I.lib().iga_last_error(disc.h).decode()
    assert torch.count_nonzero(F).item() == 0
    disc.close()
