"""Learned Newton initial guess for the kappa-weighted Bratu problem.

Binding of the iga_nn_* entry points (argument marshalling only; every forward,
backward and optimizer step runs in libiga's CUDA kernels) and the driver that
generates training data with the batched solver, trains the network and uses it
to start Newton.

Network input per control point (i, j) of the (nel+p) x (nel+p) grid:
[log kappa_ij, lambda / 4, x_i, y_j] with x, y the Greville abscissae; output:
U_ij, multiplied by the interior mask (zero on the Dirichlet boundary).
"""
import ctypes

import numpy as np

from . import iga as _iga
from . import workloads as W

DILATIONS = (1, 2, 4, 8, 16, 1)
IN_CHANNELS = 4


def _lib():
    L = _iga.lib()
    if not getattr(L, "_nn_ready", False):
        vp = ctypes.c_void_p
        L.iga_nn_create.argtypes = [ctypes.c_int] * 5 + [vp, ctypes.c_int, ctypes.c_uint64, vp, ctypes.POINTER(vp)]
        L.iga_nn_num_params.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
        L.iga_nn_get_params.argtypes = [vp, vp]
        L.iga_nn_set_params.argtypes = [vp, vp]
        L.iga_nn_forward.argtypes = [vp, vp, ctypes.c_int, vp, vp]
        L.iga_nn_loss_grad.argtypes = [vp, vp, vp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_float), vp]
        L.iga_nn_adam_step.argtypes = [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]
        L.iga_nn_set_h1_weight.argtypes = [vp, ctypes.c_float]
        L.iga_nn_destroy.argtypes = [vp]
        L.iga_nn_destroy.restype = None
        L.iga_nn_last_error.argtypes = [vp]
        L.iga_nn_last_error.restype = ctypes.c_char_p
        L._nn_ready = True
    return L


def _chk(rc, h=None):
    if rc != _iga.IGA_OK:
        raise _iga.IgaError(rc, _lib().iga_nn_last_error(h).decode())


def layer_shapes(in_channels, hidden, dilations):
    """[(cin, cout, dilation, w_offset, b_offset)] of the flat parameter vector."""
    out, off = [], 0
    L = len(dilations)
    for l, d in enumerate(dilations):
        cin = in_channels if l == 0 else hidden
        cout = 1 if l == L - 1 else hidden
        woff = off
        off += cout * 9 * cin
        out.append((cin, cout, d, woff, off))
        off += cout
    return out, off


class Net:
    def __init__(self, height, width, hidden=64, dilations=DILATIONS, in_channels=IN_CHANNELS, max_batch=64, seed=0):
        import torch
        L = _lib()
        dil = (ctypes.c_int * len(dilations))(*dilations)
        h = ctypes.c_void_p()
        stream = torch.cuda.current_stream().cuda_stream
        _chk(L.iga_nn_create(height, width, in_channels, hidden, len(dilations), dil, max_batch, seed,
                             ctypes.c_void_p(stream), ctypes.byref(h)))
        self.h = h
        self.H, self.W, self.cin, self.hidden, self.dilations, self.max_batch = height, width, in_channels, hidden, tuple(dilations), max_batch
        n = ctypes.c_int64()
        L.iga_nn_num_params(self.h, ctypes.byref(n))
        self.nparams = n.value

    def get_params(self):
        p = np.zeros(self.nparams, dtype=np.float32)
        _chk(_lib().iga_nn_get_params(self.h, p.ctypes.data), self.h)
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.nparams
        _chk(_lib().iga_nn_set_params(self.h, p.ctypes.data), self.h)

    def forward(self, x, mask=None):
        import torch
        B = x.shape[0]
        y = torch.empty((B, self.H, self.W), dtype=torch.float32, device=x.device)
        _chk(_lib().iga_nn_forward(self.h, ctypes.c_void_p(x.data_ptr()), B,
                                   None if mask is None else ctypes.c_void_p(mask.data_ptr()), ctypes.c_void_p(y.data_ptr())), self.h)
        return y

    def loss_grad(self, x, tgt, mask=None, grads=None):
        loss = ctypes.c_float()
        _chk(_lib().iga_nn_loss_grad(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(tgt.data_ptr()),
                                     None if mask is None else ctypes.c_void_p(mask.data_ptr()), x.shape[0], ctypes.byref(loss),
                                     None if grads is None else ctypes.c_void_p(grads.data_ptr())), self.h)
        return loss.value

    def set_h1_weight(self, beta):
        _chk(_lib().iga_nn_set_h1_weight(self.h, float(beta)), self.h)

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        _chk(_lib().iga_nn_adam_step(self.h, lr, beta1, beta2, eps), self.h)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _lib().iga_nn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ the workload ---

def kappa_instances(seeds, nel=64, p=2, lam_range=(0.5, 4.0)):
    """Instances of the learned-guess workload: lambda ~ U[lam_range] and a log-kappa
    Gaussian random field (variance 0.5, length 0.2) per seed."""
    n = nel + p
    out = []
    for s in seeds:
        lam = float(W.uniform(0x5EED0000 + int(s), 1, *lam_range)[0])
        out.append({"seed": int(s), "nel": nel, "p": p, "lam": lam,
                    "log_kappa": W.grf_log_kappa([n, n], p, [nel, nel], int(s))})
    return out


def features(instances, device="cuda"):
    """NHWC float32 network inputs and the interior mask for a list of instances."""
    import torch
    nel, p = instances[0]["nel"], instances[0]["p"]
    n = nel + p
    g = W.greville(W.uniform_open_knots(nel, p), p)
    X = np.zeros((len(instances), n, n, IN_CHANNELS), dtype=np.float32)
    for b, ins in enumerate(instances):
        X[b, :, :, 0] = ins["log_kappa"].reshape(n, n)
        X[b, :, :, 1] = ins["lam"] / 4.0
        X[b, :, :, 2] = g[None, :]
        X[b, :, :, 3] = g[:, None]
    mask = (~W.boundary_mask([n, n])).astype(np.float32).reshape(n, n)
    return torch.tensor(X, device=device), torch.tensor(mask, device=device)


def solve_batch(instances, U0=None, ksp=_iga.IGA_KSP_CG, chunk=2048):
    """Solve instances with the batched solver (chunks of `chunk`); returns
    (U [len, N] numpy float64, report dict, seconds)."""
    import time
    import torch
    n = instances[0]["nel"] + instances[0]["p"]
    N = n * n
    out = np.zeros((len(instances), N))
    reps = {"newton_its": [], "krylov_its": [], "status": [], "fnorm": []}
    secs = 0.0
    o = _iga.newton_defaults()
    o.ksp = ksp
    for a in range(0, len(instances), chunk):
        part = instances[a:a + chunk]
        b = _iga.Batch(part)
        U = torch.zeros(b.total, dtype=torch.float64, device="cuda")
        if U0 is not None:
            U.copy_(torch.as_tensor(U0[a:a + len(part)].reshape(-1), device="cuda"))
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = b.solve(U, o, check=False)
        secs += time.perf_counter() - t
        out[a:a + len(part)] = U.view(len(part), N).cpu().numpy()
        for k in reps:
            reps[k].append(r[k])
        b.close()
    return out, {k: np.concatenate(v) for k, v in reps.items()}, secs
