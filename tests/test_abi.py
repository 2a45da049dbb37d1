"""The C-ABI library builds, loads and exports every symbol include/iga.h declares;
argument validation that needs no GPU (CPU only)."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1305_4452_gb300 import build, iga
    build.build()
    return iga


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "iga.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(iga_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert names, "no declarations found"
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (iga_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    L = lib.lib()
    for n in names:
        assert hasattr(L, n)
    assert sorted(lib.EXPORTS) == names


def test_build_targets_sm103a_only():
    from paper_1305_4452_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


@pytest.mark.parametrize("kwargs,needle", [
    (dict(dim=2, degree=2, knots=[np.array([0, 0, 0, .5, .4, 1, 1, 1.]), None], nel=4), "non-decreasing"),
    (dict(dim=2, degree=5, nel=4), "degrees"),
    (dict(dim=1, degree=2, nel=4), "dim"),
    (dict(dim=2, degree=2, knots=[np.array([0, 0, .5, 1, 1, 1.]), None], nel=4), "open"),
    (dict(dim=2, degree=2, knots=[np.array([0, 0, 0, 1.]), None], nel=4), "too few"),
    (dict(dim=2, degree=2, nel=4, continuity=2), "continuity"),
    (dict(dim=2, degree=2, nel=2, weights=np.array([1.0] * 15 + [-1.0])), "weight"),
    (dict(dim=2, degree=2, nel=2, ctrl=np.full((16, 2), np.nan)), "finite"),
    (dict(dim=2, degree=2, nel=2, log_kappa=np.full(16, np.inf)), "finite"),
    (dict(dim=2, degree=2, knots=[np.array([0, 0, 0, .5, .5, .5, 1, 1, 1.]), None], nel=4), "multiplicity"),
    (dict(dim=2, degree=2, nel=4, periodic={0: 2}), "periodic"),           # C^k with k > p - 1
    (dict(dim=2, degree=2, nel=[1, 4], periodic={0: 1}), "unclamp"),      # n - k < k + 1
    (dict(dim=2, degree=2, knots=[np.array([0, 0, .2, .5, 1, 1, 1.]), None], nel=4, periodic={0: 1}), "open"),
])
def test_invalid_descriptions_rejected_before_any_device_work(lib, kwargs, needle):
    with pytest.raises(lib.IgaError) as ei:
        lib.Discretization(stream=0, lam=1.0, **kwargs)
    assert ei.value.status == lib.IGA_EINVAL
    assert needle in str(ei.value)


def test_newton_defaults(lib):
    o = lib.newton_defaults()
    assert o.atol == 1e-10 and o.max_newton == 50 and o.gmres_restart > 0 and o.jac == lib.IGA_FP64
    assert o.gmres_cgs_refine == lib.IGA_CGS_REFINE_NEVER


@pytest.mark.parametrize("cin,hidden", [(4, 24), (17, 64), (4, 128), (0, 32)])
def test_nn_shapes_outside_the_compiled_convolutions_rejected(lib, cin, hidden):
    import ctypes
    from paper_1305_4452_gb300 import nn
    L = nn._lib()
    dil = (ctypes.c_int * 3)(1, 2, 1)
    h = ctypes.c_void_p()
    rc = L.iga_nn_create(8, 8, cin, hidden, 3, dil, 4, 0, None, ctypes.byref(h))
    assert rc == lib.IGA_EINVAL and not h.value
    assert b"hidden" in L.iga_nn_last_error(None)


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes structures of the binding have the sizes and field offsets that a C
    compiler gives the header's structures (gcc, host ABI)."""
    import ctypes
    from paper_1305_4452_gb300 import iga
    structs = {
        "iga_desc": (iga.IgaDesc, ["dim", "degree", "nel", "continuity", "knots", "nknots", "quad", "ctrl", "weights",
                                   "periodic"]),
        "iga_bratu": (iga.IgaBratu, [("lam", "lambda"), "log_kappa"]),
        "iga_newton_opts": (iga.IgaNewtonOpts, ["atol", "max_newton", "gmres_restart", "max_krylov", "krylov_rtol", "jac",
                                                "reuse_stiffness", "ksp", "gmres_cgs_refine"]),
        "iga_newton_report": (iga.IgaNewtonReport, ["newton_its", "krylov_its", "fnorm0", "fnorm", "fnorm_hist", "status"]),
        "iga_ts_opts": (iga.IgaTsOpts, ["dt", "rho_inf"]),
        "iga_batch_report": (iga.IgaBatchReport, ["solved", "newton_its", "krylov_its", "fnorm", "status", "solve_us"]),
        "iga_peaks": (iga.IgaPeaks, ["fp64_tflops", "fp32_tflops", "copy_gbs", "sms"]),
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "iga.h"', 'int main(void) {']
    for cname, (_, fields) in structs.items():
        lines.append('  printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f in fields:
            cf = f[1] if isinstance(f, tuple) else f
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, cf, cname, cf))
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines())
    for cname, (cls, fields) in structs.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for f in fields:
            pf, cf = f if isinstance(f, tuple) else (f, f)
            assert int(got["%s.%s" % (cname, cf)]) == getattr(cls, pf).offset, (cname, cf)
