"""The FP64 exponential of the Gauss-point kernels (csrc/iga_exp.h: Tang's table-driven
method, ACM TOMS 1989).

CPU: its constants are the doubles nearest to the values the method defines (64/ln2,
ln2/64 split into two parts, 2^(j/64), 1/k!), recomputed here at 60 digits.
GPU: against the host libm exp and CUDA's exp (through torch) on a million arguments
and the special values; at most 2 units in the last place from the host exp.
"""
import os
import re

import numpy as np
import pytest

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_1305_4452_gb300", "csrc", "iga_exp.h")


def _hex_literals(text):
    return [float.fromhex(h) for h in re.findall(r"0x1\.[0-9a-f]+p[+-]\d+", text)]


def test_table_and_constants_are_the_nearest_doubles():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    src = open(HDR).read()
    tab_src = src[src.index("iga_exp_tab[64]"):src.index("};")]
    tab = _hex_literals(tab_src)
    assert len(tab) == 64
    for j, t in enumerate(tab):
        assert t == float(mp.power(2, mp.mpf(j) / 64)), j
    body = src[src.index("double iga_exp("):]
    consts = dict(re.findall(r"const double (\w+) = (0x1\.[0-9a-f]+p[+-]\d+)", body))
    ln2 = mp.log(2)
    assert float.fromhex(consts["inv_l"]) == float(64 / ln2)
    l1, l2 = float.fromhex(consts["l1"]), float.fromhex(consts["l2"])
    assert l1 == float(ln2 / 64) and l2 == float(ln2 / 64 - mp.mpf(l1))
    assert abs(mp.mpf(l1) + mp.mpf(l2) - ln2 / 64) < mp.mpf(2) ** -110
    # Taylor coefficients 1/5! ... 1/2! in the order of the Horner steps
    coeffs = [float.fromhex(h) for h in re.findall(r"fma\(r, (?:q|0x1\.[0-9a-f]+p[+-]\d+), (0x1\.[0-9a-f]+p[+-]\d+)\)", body)]
    first = float.fromhex(re.search(r"fma\(r, (0x1\.[0-9a-f]+p[+-]\d+),", body).group(1))
    assert first == float(1 / mp.factorial(5))
    assert coeffs == [float(1 / mp.factorial(k)) for k in (4, 3, 2)]
    # the range test: the high word of 700.0
    assert int(re.search(r"< (0x[0-9A-Fa-f]+)u", body).group(1), 16) == (int.from_bytes(__import__("struct").pack(">d", 700.0), "big") >> 32)


def test_truncation_bound_of_the_polynomial():
    # |r| <= ln2/128 after the reduction; the dropped Taylor terms are below r^6/6! e^|r|
    r = np.log(2) / 128
    assert r ** 6 / 720 * np.exp(r) < 4e-17


@pytest.mark.gpu
def test_gpu_exp_within_two_ulp_of_the_host_exp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1305_4452_gb300 import build, iga
    build.build()
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.uniform(-20, 20, 600_000), rng.uniform(-700, 700, 300_000),
                        rng.normal(0, 1e-3, 100_000), [0.0, -0.0, 1e-300, -1e-300, 700.0, -700.0,
                                                       np.nextafter(700.0, 0.0), np.nextafter(-700.0, 0.0)],
                        np.log(2) / 128 * np.arange(-128, 129)])
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    y = iga.exp_eval(xd).cpu().numpy()
    ref = np.exp(x)
    ulp = np.spacing(np.abs(ref))
    err = np.abs(y - ref) / ulp
    assert err.max() <= 2.0, (err.max(), x[np.argmax(err)])
    assert np.all(y[x == 0.0] == 1.0)
    # CUDA's own exp agrees to the same few ulp
    yc = torch.exp(xd).cpu().numpy()
    assert (np.abs(y - yc) / ulp).max() <= 3.0
    # outside |x| <= 700 and non-finite arguments: CUDA's exp
    s = torch.tensor([800.0, -800.0, np.inf, -np.inf, np.nan, 709.5, -745.0], dtype=torch.float64, device="cuda")
    ys = iga.exp_eval(s)
    assert torch.equal(torch.isnan(ys), torch.isnan(torch.exp(s)))
    m = ~torch.isnan(ys)
    assert torch.equal(ys[m], torch.exp(s)[m])
    # argument checks: NULL arrays or a negative count are refused, n = 0 does nothing
    assert iga.lib().iga_exp_eval(None, None, None, 5) == iga.IGA_EINVAL
    assert iga.lib().iga_exp_eval(None, xd.data_ptr(), xd.data_ptr(), -1) == iga.IGA_EINVAL
    assert iga.lib().iga_exp_eval(None, None, None, 0) == 0
