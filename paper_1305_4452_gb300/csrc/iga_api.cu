// C ABI of libiga (declared in include/iga.h): creation, residual and Jacobian
// assembly, and the device Newton-Krylov driver (SNESSolve analogue, Sec. 3.2).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "iga_internal.h"

static thread_local std::string g_create_err;

#define CK(call)                                                                 \
  do {                                                                           \
    cudaError_t ce_ = (call);                                                    \
    if (ce_ != cudaSuccess) {                                                    \
      h->err = iga_format("%s: %s", #call, cudaGetErrorString(ce_));             \
      return (ce_ == cudaErrorMemoryAllocation) ? IGA_ENOMEM : IGA_ECUDA;        \
    }                                                                            \
  } while (0)

template <typename T>
static cudaError_t upload(T **dst, const std::vector<T> &src) {
  *dst = nullptr;
  if (src.empty()) return cudaSuccess;
  cudaError_t ce = cudaMalloc((void **)dst, src.size() * sizeof(T));
  if (ce) return ce;
  return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

static void free_dir(DirDev &d) {
  void *ps[] = {d.first, d.tab, d.wq, d.l, d.r, d.pair_off, d.pair_i, d.pair_j, d.pair_x0,
                d.pair_np, d.pair_po, d.pair_T, d.pair_c, d.pair_cs, d.pair_val, d.pair_val_f, d.node_e0, d.node_ne};
  for (void *p : ps)
    if (p) cudaFree(p);
  memset(&d, 0, sizeof d);
}

void iga_release(iga_s *h) {
  periodic_release(h);
  elem_gemm_release(h);
  for (int ax = 0; ax < 3; ax++) free_dir(h->ddev[ax]);
  void *ps[] = {h->rowptr, h->rp_line, h->rp_p0, h->colidx, h->weights, h->geom, h->Fe, h->Q00, h->T1, h->T2, h->Kstiff, h->Kstiff_f, h->Ebuf64, h->ts_buf,
                h->Mred, h->Mred_f, h->J64, h->J32, h->wk, h->V, h->red, h->ctl, h->Uhost_dev,
                h->geom32, h->tab32[0], h->tab32[1], h->tab32[2], h->Ebuf, h->z32, h->gsbar, h->J32s};
  for (void *p : ps)
    if (p) cudaFree(p);
  if (h->ctl_host) cudaFreeHost(h->ctl_host);
  for (ProfRec &r : h->prof.pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : h->prof.pool) cudaEventDestroy(e);
}

static iga_status upload_dir(iga_s *h, int ax) {
  Dir &D = h->dir[ax];
  DirDev &d = h->ddev[ax];
  memset(&d, 0, sizeof d);
  d.p = D.p; d.q = D.q; d.nel = D.nel; d.n = D.n; d.np = D.npairs(); d.X = D.X();
  if (ax >= h->dim) return IGA_OK;
  CK(upload(&d.first, D.first));
  CK(upload(&d.tab, D.tab));
  CK(upload(&d.wq, D.wq));
  CK(upload(&d.l, D.l));
  CK(upload(&d.r, D.r));
  CK(upload(&d.pair_off, D.pair_off));
  CK(upload(&d.pair_i, D.pair_i));
  CK(upload(&d.pair_j, D.pair_j));
  CK(upload(&d.pair_x0, D.pair_x0));
  CK(upload(&d.pair_np, D.pair_np));
  CK(upload(&d.pair_po, D.pair_po));
  CK(upload(&d.pair_T, D.pair_T));
  CK(upload(&d.pair_c, D.pair_c));
  CK(upload(&d.pair_cs, D.pair_cs));
  d.nc = (int)D.pair_c.size();
  if (h->w_folded) {
    // the pair tables times w_ax[i] w_ax[j] (the axis's factor of w_A w_B)
    std::vector<double> pv(D.pair_val);
    const std::vector<double> &w = h->wsep[ax];
    for (size_t k = 0; k < D.pair_i.size(); k++) {
      const double f = w[D.pair_i[k]] * w[D.pair_j[k]];
      double *v = pv.data() + (size_t)D.pair_po[k] * IGA_PVS;
      for (int t = 0; t < D.pair_np[k] * IGA_PVS; t++) v[t] *= f;
    }
    CK(upload(&d.pair_val, pv));
    std::vector<float> pf(pv.begin(), pv.end());
    CK(upload(&d.pair_val_f, pf));
  } else {
    CK(upload(&d.pair_val, D.pair_val));
    std::vector<float> pf(D.pair_val.begin(), D.pair_val.end());
    CK(upload(&d.pair_val_f, pf));
  }
  CK(upload(&d.node_e0, D.node_e0));
  CK(upload(&d.node_ne, D.node_ne));
  return IGA_OK;
}

iga_status iga_create_impl(iga_s *h, const iga_desc *d, const iga_bratu *b) {
  iga_status st = iga_build_dirs(h, d);
  if (st != IGA_OK) return st;
  h->lambda = b ? b->lambda : 0.0;
  if (!isfinite(h->lambda)) {
    h->err = "lambda must be finite";
    return IGA_EINVAL;
  }
  h->gl = geom_layout(h->dim);
  h->has_geom = d->ctrl != nullptr;
  h->has_w = d->weights != nullptr;
  h->has_kappa = b && b->log_kappa;
  const int64_t N = h->N;
  if (h->has_w)
    for (int64_t A = 0; A < N; A++)
      if (!(d->weights[A] > 0.0) || !isfinite(d->weights[A])) {
        h->err = iga_format("weight %lld must be positive and finite", (long long)A);
        return IGA_EINVAL;
      }
  if (h->has_geom)
    for (int64_t k = 0; k < N * h->dim; k++)
      if (!isfinite(d->ctrl[k])) {
        h->err = "control points must be finite";
        return IGA_EINVAL;
      }
  if (h->has_kappa)
    for (int64_t A = 0; A < N; A++)
      if (!isfinite(b->log_kappa[A])) {
        h->err = "log-kappa coefficients must be finite";
        return IGA_EINVAL;
      }
  // weights that factor by axis (the annulus: a function of the angle alone), to within a
  // few units of rounding: w0[i] = w(i, 0, 0), w_a[j] = w(0, .., j, .., 0) / w(0, 0, 0)
  h->w_folded = false;
  if (h->has_w && !h->unclamped) {
    const int n0 = h->dir[0].n, n1 = h->dir[1].n, n2 = h->dim == 3 ? h->dir[2].n : 1;
    const double *w = d->weights;
    for (int a = 0; a < 3; a++) h->wsep[a].assign(a < h->dim ? h->dir[a].n : 1, 1.0);
    for (int i = 0; i < n0; i++) h->wsep[0][i] = w[i];
    for (int j = 0; j < n1; j++) h->wsep[1][j] = w[(int64_t)j * n0] / w[0];
    if (h->dim == 3)
      for (int k = 0; k < n2; k++) h->wsep[2][k] = w[(int64_t)k * n0 * n1] / w[0];
    bool sep = true;
    for (int64_t A = 0; A < N && sep; A++) {
      const int i = (int)(A % n0), j = (int)((A / n0) % n1), k = (int)(A / ((int64_t)n0 * n1));
      const double f = h->wsep[0][i] * h->wsep[1][j] * h->wsep[2][k];
      sep = fabs(f - w[A]) <= 8.0 * 2.220446049250313e-16 * w[A];
    }
    h->w_folded = sep;
  }
  for (int ax = 0; ax < 3; ax++) {
    st = upload_dir(h, ax);
    if (st != IGA_OK) return st;
  }
  // CSR pattern (Sec. 2.5)
  std::vector<int64_t> rowptr;
  iga_rowptr(h, rowptr);
  h->nnz = rowptr[N];
  CK(upload(&h->rowptr, rowptr));
  {
    const Dir &D0 = h->dir[0];
    std::vector<int64_t> line((size_t)(N / D0.n));
    for (size_t L = 0; L < line.size(); L++) line[L] = rowptr[L * D0.n];
    std::vector<int> p0(D0.n);
    int acc = 0;
    for (int i = 0; i < D0.n; i++) {
      p0[i] = acc;
      acc += D0.r[i] - D0.l[i] + 1;
    }
    CK(upload(&h->rp_line, line));
    CK(upload(&h->rp_p0, p0));
  }
  CK(cudaMalloc((void **)&h->colidx, (size_t)h->nnz * sizeof(int32_t)));
  CK(launch_colidx(h));
  // weights, geometry factors
  if (h->has_w) {
    CK(cudaMalloc((void **)&h->weights, N * sizeof(double)));
    CK(cudaMemcpy(h->weights, d->weights, N * sizeof(double), cudaMemcpyHostToDevice));
  }
  int nq = (h->dim == 3) ? h->q * h->q * h->q : h->q * h->q;
  int nen = (h->dim == 3) ? (h->p + 1) * (h->p + 1) * (h->p + 1) : (h->p + 1) * (h->p + 1);
  CK(cudaMalloc((void **)&h->geom, (size_t)h->nelem * h->gl.nf * nq * sizeof(double)));
  double *ctrl_dev = nullptr, *logk_dev = nullptr;
  if (h->has_geom) {
    CK(cudaMalloc((void **)&ctrl_dev, (size_t)N * h->dim * sizeof(double)));
    CK(cudaMemcpy(ctrl_dev, d->ctrl, (size_t)N * h->dim * sizeof(double), cudaMemcpyHostToDevice));
  }
  if (h->has_kappa) {
    CK(cudaMalloc((void **)&logk_dev, N * sizeof(double)));
    CK(cudaMemcpy(logk_dev, b->log_kappa, N * sizeof(double), cudaMemcpyHostToDevice));
  }
  cudaError_t ge = launch_geometry(h, ctrl_dev, logk_dev);
  if (ctrl_dev) cudaFree(ctrl_dev);
  if (logk_dev) cudaFree(logk_dev);
  if (ge == cudaErrorInvalidValue) {
    h->err = "geometry map has a non-positive Jacobian determinant at a Gauss point";
    return IGA_EINVAL;
  }
  CK(ge);
  if (h->has_geom || h->has_w) CK(classify_stiffness_plan(h));
  CK(cudaMalloc((void **)&h->Fe, (size_t)h->nelem * nen * sizeof(double)));
  CK(cudaMalloc((void **)&h->Q00, (size_t)h->nelem * nq * sizeof(double)));
  // stage intermediates (sized for FP64)
  const Dir &D0 = h->dir[0], &D1 = h->dir[1], &D2 = h->dir[2];
  size_t ng1 = jacobian_t1_groups(h->dim), ng2 = jacobian_t2_groups(h->dim);
  h->T1_bytes = (size_t)ng1 * D0.npairs() * D1.X() * (h->dim == 3 ? D2.X() : 1) * sizeof(double);
  CK(cudaMalloc(&h->T1, h->T1_bytes));
  if (h->dim == 3) {
    h->T2_bytes = (size_t)ng2 * D0.npairs() * D1.npairs() * D2.X() * sizeof(double);
    CK(cudaMalloc(&h->T2, h->T2_bytes));
  }
  CK(cudaStreamSynchronize(h->stream));
  return IGA_OK;
}

extern "C" iga_status iga_create(const iga_desc *d, const iga_bratu *b, void *stream, iga_t *out) {
  if (!out) return IGA_EINVAL;
  *out = nullptr;
  if (!d) {
    g_create_err = "desc is NULL";
    return IGA_EINVAL;
  }
  iga_s *h = new iga_s();
  h->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&h->device) != cudaSuccess) h->device = -1;
  const bool periodic = d->periodic[0] || d->periodic[1] || (d->dim == 3 && d->periodic[2]);
  iga_status st = periodic ? iga_periodic_setup(h, d, b) : iga_create_impl(h, d, b);
  if (st != IGA_OK) {
    g_create_err = h->err;
    iga_release(h);
    delete h;
    return st;
  }
  if (!periodic) noalloc_setup(h);
  *out = h;
  return IGA_OK;
}

extern "C" void iga_destroy(iga_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  iga_release(h);
  delete h;
}

extern "C" const char *iga_last_error(iga_t h) {
  if (!h) return g_create_err.c_str();
  return h->err.c_str();
}

extern "C" iga_status iga_set_boundary_value(iga_t h, int axis, int side, double value) {
  if (!h) return IGA_EINVAL;
  if (axis < 0 || axis >= h->dim || side < 0 || side > 1 || !isfinite(value)) {
    h->err = iga_format("bad boundary (axis %d, side %d)", axis, side);
    return IGA_EINVAL;
  }
  if (h->inner && h->per_host[axis].n != h->per_host[axis].nu) {
    h->err = iga_format("axis %d is periodic: it has no Dirichlet faces", axis);
    return IGA_EINVAL;
  }
  h->bnd.flag[axis][side] = 1;
  h->bnd.val[axis][side] = value;
  h->K_valid = false;
  return IGA_OK;
}

extern "C" iga_status iga_set_wait_limit(iga_t h, double seconds) {
  if (!h) return IGA_EINVAL;
  if (!(seconds > 0.0) || seconds > 60.0) {
    h->err = "the wait limit must be in (0, 60] seconds";
    return IGA_EINVAL;
  }
  h->wait_limit_ns = (uint64_t)(seconds * 1e9);
  return IGA_OK;
}

extern "C" iga_status iga_inject_stall(iga_t h) {
  if (!h) return IGA_EINVAL;
  h->stall_next = true;
  return IGA_OK;
}

extern "C" iga_status iga_set_jacobian_plan(iga_t h, int general) {
  if (!h) return IGA_EINVAL;
  if (general != 0 && general != 1) {
    h->err = "general must be 0 or 1";
    return IGA_EINVAL;
  }
  h->plan_general = general == 1;
  h->K_valid = false;  // the kept stiffness was assembled under the other plan
  h->K_valid_f = false;
  return IGA_OK;
}

extern "C" iga_status iga_set_gmres_fused(iga_t h, int fused) {
  if (!h) return IGA_EINVAL;
  if (fused != 0 && fused != 1) {
    h->err = "fused must be 0 or 1";
    return IGA_EINVAL;
  }
  h->gs_unfused = fused == 0;
  return IGA_OK;
}

extern "C" iga_status iga_set_lambda(iga_t h, double lambda) {
  if (!h || !isfinite(lambda)) return IGA_EINVAL;
  h->lambda = lambda;
  return IGA_OK;
}

extern "C" iga_status iga_get_pattern(iga_t h, int64_t *n, int64_t *nnz, const int64_t **rowptr, const int32_t **colidx) {
  if (!h) return IGA_EINVAL;
  if (n) *n = h->N;
  if (nnz) *nnz = h->nnz;
  if (rowptr) *rowptr = h->rowptr;
  if (colidx) *colidx = h->colidx;
  return IGA_OK;
}

extern "C" iga_status iga_form_residual(iga_t h, const double *U, double *F) {
  if (!h) return IGA_EINVAL;
  if (!U || !F || U == F) {
    h->err = "U and F must be distinct non-NULL device pointers";
    return IGA_EINVAL;
  }
  CK(launch_residual(h, U, F));
  return IGA_OK;
}

extern "C" iga_status iga_form_jacobian(iga_t h, const double *U, void *vals, iga_precision prec) {
  if (!h) return IGA_EINVAL;
  if (!U || !vals) {
    h->err = "U and vals must be non-NULL device pointers";
    return IGA_EINVAL;
  }
  if (prec == IGA_FP64) {
    CK(launch_jacobian64(h, U, (double *)vals, 0, nullptr));
  } else if (prec == IGA_JAC_FP32) {
    CK(launch_jacobian32(h, U, (float *)vals, 0, nullptr));
  } else if (prec == IGA_JAC_TF32 || prec == IGA_JAC_BF16 || prec == IGA_JAC_FD) {
    if (h->inner) {
      h->err = "periodic handles assemble the IGA_FP64 and IGA_JAC_FP32 Jacobians only";
      return IGA_EINVAL;
    }
    if (prec == IGA_JAC_FD ? !mixed_supported(h->dim, h->p) : !tc_jacobian_supported(h, prec)) {
      h->err = iga_format("no element-matrix Jacobian of this kind for p = %d in %dD on this mesh", h->p, h->dim);
      return IGA_EINVAL;
    }
    if (prec == IGA_JAC_FD) CK(launch_jacobian_fd(h, U, (double *)vals));
    else {
      CK(launch_jacobian_mixed(h, U, (float *)vals, (int)prec));
      if (elem_gemm_failed(h)) {
        h->err = "a tensor-core pipeline wait gave up; the Jacobian values are invalid";
        return IGA_ETIMEOUT;
      }
    }
  } else {
    h->err = "unknown precision";
    return IGA_EINVAL;
  }
  return IGA_OK;
}

extern "C" iga_status iga_apply_jacobian(iga_t h, const void *vals, iga_precision prec, const double *x, double *y) {
  if (!h) return IGA_EINVAL;
  if (!vals || !x || !y || x == y) {
    h->err = "vals, x and y must be non-NULL device pointers, x != y";
    return IGA_EINVAL;
  }
  if (prec == IGA_FP64 || prec == IGA_JAC_FD) {
    CK(launch_spmv64(h, (const double *)vals, x, y));
  } else if (prec == IGA_JAC_FP32 || prec == IGA_JAC_TF32 || prec == IGA_JAC_BF16) {
    CK(launch_spmv32(h, (const float *)vals, x, y));
  } else {
    h->err = "unknown precision";
    return IGA_EINVAL;
  }
  return IGA_OK;
}

extern "C" iga_status iga_apply_jacobian_mf(iga_t h, const double *U, const double *x, double *y) {
  if (!h) return IGA_EINVAL;
  if (!U || !x || !y || x == y) {
    h->err = "U, x and y must be non-NULL device pointers, x != y";
    return IGA_EINVAL;
  }
  if (h->inner) {
    h->err = "matrix-free products are not available on periodic handles";
    return IGA_EINVAL;
  }
  CK(launch_q00(h, U, 0.0, 1.0));
  h->q00_valid = false;
  CK(launch_jv(h, x, y, nullptr));
  return IGA_OK;
}

extern "C" iga_status iga_form_jacobian_diagonal(iga_t h, const double *U, double *d) {
  if (!h) return IGA_EINVAL;
  if (!U || !d) {
    h->err = "U and d must be non-NULL device pointers";
    return IGA_EINVAL;
  }
  if (h->inner) {
    h->err = "the element-wise diagonal is not available on periodic handles";
    return IGA_EINVAL;
  }
  CK(launch_q00(h, U, 0.0, 1.0));
  h->q00_valid = false;
  CK(launch_jacobian_diagonal(h, d));
  return IGA_OK;
}

extern "C" void iga_newton_defaults(iga_newton_opts *o) {
  if (!o) return;
  o->atol = 1e-10;
  o->max_newton = 50;
  o->gmres_restart = 60;
  o->max_krylov = 4000;
  o->krylov_rtol = 1e-2;
  o->jac = IGA_FP64;
  o->reuse_stiffness = 1;
  o->ksp = IGA_KSP_GMRES;
  o->gmres_cgs_refine = IGA_CGS_REFINE_NEVER;
}

// ---- small vector kernels of the Newton driver ----
__global__ static void k_axpby(const double *__restrict__ x, double a, const double *__restrict__ y, double *__restrict__ out,
                               int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = x[i] + a * y[i];
}
__global__ static void k_neg(const double *__restrict__ x, double *__restrict__ y, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) y[i] = -x[i];
}

static iga_status ensure_workspace(iga_s *h, int m, bool f32, bool mf = false) {
  const int64_t N = h->N;
  if (!h->wk) CK(cudaMalloc((void **)&h->wk, (size_t)(8 * N + 64 + 2 * 1025) * sizeof(double)));
  if (!h->ctl_host) CK(cudaMallocHost((void **)&h->ctl_host, 16 * sizeof(double)));
  if (!h->gsbar) {
    CK(cudaMalloc((void **)&h->gsbar, 2 * sizeof(unsigned)));
    CK(cudaMemsetAsync(h->gsbar, 0, 2 * sizeof(unsigned), h->stream));
  }
  if (h->V_m != m) {
    if (h->V) cudaFree(h->V);
    if (h->red) cudaFree(h->red);
    if (h->ctl) cudaFree(h->ctl);
    h->V = nullptr; h->red = nullptr; h->ctl = nullptr;
    CK(cudaMalloc((void **)&h->V, (size_t)(m + 1) * N * sizeof(double)));
    // Gram-Schmidt partials of two passes in flight: 2 (m + 1) x nb (and >= the 304 of the norms)
    const int nb = gs_partition(N).nb > 304 ? gs_partition(N).nb : 304;
    CK(cudaMalloc((void **)&h->red, (size_t)(2 * m + 4) * nb * sizeof(double)));
    CK(cudaMalloc((void **)&h->ctl, (size_t)((m + 1) * m + 4 * m + 16) * sizeof(double)));
    h->V_m = m;
  }
  if (!f32 && !mf && !h->J64) CK(cudaMalloc((void **)&h->J64, h->nnz * sizeof(double)));
  if (f32 && !h->J32) CK(cudaMalloc((void **)&h->J32, h->nnz * sizeof(float)));
  if (f32 && !h->z32) CK(cudaMalloc((void **)&h->z32, N * sizeof(float)));
  return IGA_OK;
}

static iga_status norm_host(iga_s *h, const double *x, double *out) {
  double *scal = h->wk + 8 * h->N;
  CK(launch_norm2(h, x, scal));
  CK(cudaMemcpyAsync(h->ctl_host + 8, scal, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *out = sqrt(h->ctl_host[8]);
  return IGA_OK;
}

// Assemble the Newton Jacobian at U into h->J64 / h->J32.
static iga_status newton_jacobian(iga_s *h, const double *U, bool f32, bool reuse, int prec) {
  h->J32s_valid = false;  // the sliced copy no longer matches once J32 is rewritten
  if (h->inner) reuse = false;  // periodic: full assembly on the unwrapped space, then the fold
  if (prec == IGA_JAC_FD) {  // local numerical differentiation, assembled in full each step
    CK(launch_jacobian_fd(h, U, h->J64));
    return IGA_OK;
  }
  if (f32 && prec != IGA_JAC_FP32) {  // tensor-core element matrices, assembled in full each step
    CK(launch_jacobian_mixed(h, U, h->J32, prec));
    if (elem_gemm_failed(h)) {
      h->err = "a tensor-core pipeline wait gave up";
      return IGA_ETIMEOUT;
    }
    return IGA_OK;
  }
  if (!reuse) {
    if (f32) CK(launch_jacobian32(h, U, h->J32, 0, nullptr));
    else CK(launch_jacobian64(h, U, h->J64, 0, nullptr));
    return IGA_OK;
  }
  // J(U) = K + reaction(U): the stiffness K does not depend on U or lambda
  if (f32) {
    if (!h->Kstiff_f) CK(cudaMalloc((void **)&h->Kstiff_f, h->nnz * sizeof(float)));
    if (!h->K_valid_f) {
      // the FP64 stiffness of the split residual, rounded once, is a closer FP32 stiffness
      // than an FP32 assembly and costs one pass over the values instead of three stages
      if (h->K_valid) CK(launch_round_f32(h, h->Kstiff, h->Kstiff_f, h->nnz));
      else CK(launch_jacobian32(h, nullptr, h->Kstiff_f, 1, nullptr));
      h->K_valid_f = true;
    }
    CK(launch_jacobian32(h, U, h->J32, 2, h->Kstiff_f));
  } else {
    if (!h->Kstiff) CK(cudaMalloc((void **)&h->Kstiff, h->nnz * sizeof(double)));
    if (!h->K_valid) { CK(launch_jacobian64(h, nullptr, h->Kstiff, 1, nullptr)); h->K_valid = true; }
    CK(launch_jacobian64(h, U, h->J64, 2, h->Kstiff));
  }
  return IGA_OK;
}

extern "C" iga_status iga_solve_newton(iga_t h, double *U, const iga_newton_opts *opts_in, iga_newton_report *rep) {
  if (!h) return IGA_EINVAL;
  iga_newton_opts o;
  iga_newton_defaults(&o);
  if (opts_in) o = *opts_in;
  if ((o.jac == IGA_JAC_FD && !mixed_supported(h->dim, h->p)) ||
      ((o.jac == IGA_JAC_TF32 || o.jac == IGA_JAC_BF16) && !h->inner && !tc_jacobian_supported(h, (int)o.jac))) {
    h->err = "element-matrix Jacobian not supported for this degree";
    return IGA_EINVAL;
  }
  if (h->inner && o.jac != IGA_FP64 && o.jac != IGA_JAC_FP32) {
    h->err = "periodic handles solve with the IGA_FP64 or IGA_JAC_FP32 Jacobian";
    return IGA_EINVAL;
  }
  if (!U || o.gmres_restart < 1 || o.gmres_restart > 1000 || o.max_newton < 0 || !(o.atol >= 0.0) ||
      o.gmres_cgs_refine < IGA_CGS_REFINE_NEVER || o.gmres_cgs_refine > IGA_CGS_REFINE_ALWAYS ||
      (o.jac != IGA_FP64 && o.jac != IGA_JAC_TF32 && o.jac != IGA_JAC_BF16 && o.jac != IGA_JAC_FP32 &&
       o.jac != IGA_JAC_NONE && o.jac != IGA_JAC_FD)) {
    h->err = "bad Newton options or NULL U";
    return IGA_EINVAL;
  }
  iga_newton_report R;
  memset(&R, 0, sizeof R);
  R.status = IGA_ENOCONV;
  const bool mf = o.jac == IGA_JAC_NONE;  // matrix-free
  const bool fd = o.jac == IGA_JAC_FD;    // FP64 values by numerical differentiation
  const bool f32 = !mf && !fd && o.jac != IGA_FP64;
  // the FP64 residual as K U + reaction(U) with the FP64 stiffness K assembled once per
  // solve (also when a reduced-precision Jacobian steers Newton: the residual stays FP64)
  const bool split = !mf && !fd && o.reuse_stiffness != 0 && !h->inner;
  iga_status st = ensure_workspace(h, o.gmres_restart, f32, mf);
  if (st != IGA_OK) return st;
  const int64_t N = h->N;
  double *F = h->wk, *dU = h->wk + N, *Ut = h->wk + 2 * N, *Ft = h->wk + 3 * N;
  int eg = (int)((N + 255) / 256);
  if (eg > 608) eg = 608;
  // stiffness part is rebuilt once per solve (reuse across Newton steps only); the
  // steps of a time integration keep it (K depends on the geometry alone)
  if (!h->ts_on) {
    h->K_valid = false;
    h->K_valid_f = false;
  }
  h->q00_valid = false;
  if (split) {
    // the stiffness first, so that every residual of the solve is K U + reaction(U); the
    // reaction pass leaves Q00 at U for the first Jacobian
    if (!h->Kstiff) CK(cudaMalloc((void **)&h->Kstiff, h->nnz * sizeof(double)));
    if (!h->K_valid) {
      CK(launch_jacobian64(h, nullptr, h->Kstiff, 1, nullptr));
      h->K_valid = true;
    }
    CK(launch_residual_split(h, U, F, h->Kstiff, h->wk + 7 * N));
    h->q00_valid = true;
  } else {
    CK(launch_residual(h, U, F));
  }
  double fn;
  st = norm_host(h, F, &fn);
  if (st != IGA_OK) return st;
  R.fnorm0 = fn;
  R.fnorm_hist[0] = fn;
  int k = 0;
  for (;;) {
    if (!isfinite(fn)) { R.status = IGA_ENAN; break; }
    if (fn <= o.atol) { R.status = IGA_OK; break; }
    if (k >= o.max_newton) { R.status = IGA_ENOCONV; break; }
    if (mf) {
      CK(launch_q00(h, U, 0.0, 1.0));  // the reaction coefficient the matrix-free products use
      h->q00_valid = false;
    } else {
      st = newton_jacobian(h, U, f32, o.reuse_stiffness != 0, (int)o.jac);
      if (st != IGA_OK) return st;
      if (f32) CK(launch_slice32(h));  // the Krylov products run on the sliced copy
    }
    IGA_LAUNCH(h, KC_VEC, (k_neg<<<eg, 256, 0, h->stream>>>(F, Ft, N)));
    // forcing term min(rtol, ||F||) (quadratic Newton), but never below half the
    // Newton tolerance: a linear residual under atol/2 already lets the step meet atol
    double rtol = o.krylov_rtol < fn ? o.krylov_rtol : fn;
    // with a reduced-precision Jacobian (and FP32 operator products) a linear solve
    // tighter than the Jacobian's own error buys nothing: the floor is about 20-50 times
    // the relative Frobenius error of each type (BF16 ~2e-5, TF32 ~5e-6, FP32 ~3e-9)
    const double floor_rtol = !f32 ? 0.0 : (o.jac == IGA_JAC_BF16 ? 1e-4 : (o.jac == IGA_JAC_TF32 ? 1e-6 : 1e-8));
    if (rtol < floor_rtol) rtol = floor_rtol;
    double tol_abs = rtol * fn;
    if (tol_abs < 0.5 * o.atol) tol_abs = 0.5 * o.atol;
    if (tol_abs < 1e-14 * fn) tol_abs = 1e-14 * fn;
    int its = 0;
    cudaError_t ce = cudaSuccess;
    const void *Jv = mf ? nullptr : (f32 ? (const void *)h->J32 : (const void *)h->J64);
    // the FP64 Jacobian carries the exact Dirichlet fix: its product skips the fixed rows
    // and the zero columns
    const int kind = mf ? 2 : (f32 ? 1 : (o.jac == IGA_FP64 ? 3 : 0));
    int grc = (o.ksp == IGA_KSP_CG) ? cg_solve(h, Jv, kind, Ft, dU, tol_abs, o.max_krylov, &its, &ce)
                                    : gmres_solve(h, Jv, kind, Ft, dU, tol_abs, o.gmres_restart, o.max_krylov,
                                                  o.gmres_cgs_refine, &its, &ce);
    if (grc < 0) {
      h->err = iga_format("GMRES: %s", cudaGetErrorString(ce));
      return IGA_ECUDA;
    }
    if (grc == 3) {
      h->err = "GMRES: a grid barrier of the fused orthogonalisation gave up";
      return IGA_ETIMEOUT;
    }
    R.krylov_its += its;
    // backtracking on ||F||: halve the step until the norm decreases
    double alpha = 1.0, ft = 0.0;
    bool ok = false;
    for (int ls = 0; ls <= 10; ls++) {
      IGA_LAUNCH(h, KC_VEC, (k_axpby<<<eg, 256, 0, h->stream>>>(U, alpha, dU, Ut, N)));
      // with the stiffness assembled (FP64), F = K U + reaction(U)
      h->q00_valid = false;
      if (split) CK(launch_residual_split(h, Ut, Ft, h->Kstiff, h->wk + 7 * N));
      else CK(launch_residual(h, Ut, Ft));
      st = norm_host(h, Ft, &ft);
      if (st != IGA_OK) return st;
      if (isfinite(ft) && ft < fn) {
        ok = true;
        h->q00_valid = split;  // the split residual left Q00 at the accepted point
        break;
      }
      alpha *= 0.5;
    }
    k++;
    if (!ok) {
      R.status = isfinite(ft) ? IGA_EDIVERGED : IGA_ENAN;
      if (k < 64) R.fnorm_hist[k] = fn;
      break;
    }
    CK(cudaMemcpyAsync(U, Ut, N * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(F, Ft, N * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    fn = ft;
    if (k < 64) R.fnorm_hist[k] = fn;
  }
  CK(cudaStreamSynchronize(h->stream));
  R.newton_its = k;
  R.fnorm = fn;
  if (rep) *rep = R;
  if (R.status != IGA_OK) h->err = iga_format("Newton stopped after %d steps with ||F|| = %.3e", k, fn);
  return R.status;
}

extern "C" iga_status iga_solve_newton_host(iga_t h, double *U_host, const iga_newton_opts *opts, iga_newton_report *rep) {
  if (!h || !U_host) return IGA_EINVAL;
  if (!h->Uhost_dev) CK(cudaMalloc((void **)&h->Uhost_dev, h->N * sizeof(double)));
  CK(cudaMemcpyAsync(h->Uhost_dev, U_host, h->N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  iga_status st = iga_solve_newton(h, h->Uhost_dev, opts, rep);
  if (st == IGA_EINVAL || st == IGA_ECUDA || st == IGA_ENOMEM) return st;
  CK(cudaMemcpyAsync(U_host, h->Uhost_dev, h->N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return st;
}

// ---- time-dependent problems (Sec. 4.2) ----
extern "C" iga_status iga_form_residual_ts(iga_t h, const double *V, const double *U, double *F) {
  if (!h) return IGA_EINVAL;
  if (!V || !U || !F || F == U || F == V) {
    h->err = "V, U and F must be non-NULL device pointers, F distinct from U and V";
    return IGA_EINVAL;
  }
  h->ts_on = true;
  h->ts_a = 0.0;
  h->ts_C = V;
  cudaError_t ce = launch_residual(h, U, F);
  h->ts_on = false;
  h->ts_C = nullptr;
  CK(ce);
  return IGA_OK;
}

extern "C" iga_status iga_form_jacobian_ts(iga_t h, double shift, const double *U, void *vals, iga_precision prec) {
  if (!h) return IGA_EINVAL;
  if (!U || !vals || !isfinite(shift) || (prec != IGA_FP64 && prec != IGA_JAC_FP32)) {
    h->err = "U and vals must be non-NULL device pointers, shift finite, precision IGA_FP64 or IGA_JAC_FP32";
    return IGA_EINVAL;
  }
  h->ts_on = true;
  h->ts_a = shift;
  h->ts_C = nullptr;
  cudaError_t ce = prec == IGA_FP64 ? launch_jacobian64(h, U, (double *)vals, 0, nullptr)
                                    : launch_jacobian32(h, U, (float *)vals, 0, nullptr);
  h->ts_on = false;
  h->ts_a = 0.0;
  CK(ce);
  return IGA_OK;
}

// C = -a U_n + b U-dot_n and a copy of U_n (the Newton start W = U_n stays in U)
__global__ static void k_alpha_begin(const double *__restrict__ U, const double *__restrict__ V, double a, double b,
                                     double *__restrict__ C, double *__restrict__ Un, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double u = U[i];
    C[i] = -a * u + b * V[i];
    Un[i] = u;
  }
}
// From the stage value W = U_{n+alpha_f} in U: U_{n+1} = U_n + (W - U_n) / alpha_f and
// U-dot_{n+1} = (U_{n+1} - U_n) / (gamma dt) - (1 - gamma) / gamma U-dot_n
__global__ static void k_alpha_end(double *__restrict__ U, double *__restrict__ V, const double *__restrict__ Un,
                                   double inv_af, double inv_gdt, double c_v, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double un = Un[i];
    const double du = (U[i] - un) * inv_af;
    U[i] = un + du;
    V[i] = du * inv_gdt - c_v * V[i];
  }
}

extern "C" iga_status iga_ts_alpha_step(iga_t h, const iga_ts_opts *ts, double *U, double *V, const iga_newton_opts *opts,
                                        iga_newton_report *rep) {
  if (!h) return IGA_EINVAL;
  if (!ts || !U || !V || U == V || !(ts->dt > 0.0) || !isfinite(ts->dt) || !(ts->rho_inf >= 0.0) || !(ts->rho_inf <= 1.0)) {
    h->err = "need distinct device U and V, dt > 0 and 0 <= rho_inf <= 1";
    return IGA_EINVAL;
  }
  iga_newton_opts o;
  iga_newton_defaults(&o);
  if (opts) o = *opts;
  if (o.jac != IGA_FP64 && o.jac != IGA_JAC_FP32 && (o.jac != IGA_JAC_NONE || h->inner)) {
    h->err = "time steps support the IGA_FP64, IGA_JAC_FP32 and (not periodic) IGA_JAC_NONE Jacobians";
    return IGA_EINVAL;
  }
  // Sec. 4.2: parameters from rho_inf; with W = U_{n+alpha_f} the unknown,
  // U-dot_{n+alpha_m} = a (W - U_n) + b U-dot_n, a = alpha_m / (alpha_f gamma dt), b = 1 - alpha_m / gamma
  const double rho = ts->rho_inf, dt = ts->dt;
  const double am = 0.5 * (3.0 - rho) / (1.0 + rho), af = 1.0 / (1.0 + rho), gam = 0.5 + am - af;
  const double a = am / (af * gam * dt), b = 1.0 - am / gam;
  const int64_t N = h->N;
  if (!h->ts_buf) CK(cudaMalloc((void **)&h->ts_buf, 2 * N * sizeof(double)));
  double *C = h->ts_buf, *Un = h->ts_buf + N;
  int eg = (int)((N + 255) / 256);
  if (eg > 608) eg = 608;
  IGA_LAUNCH(h, KC_VEC, (k_alpha_begin<<<eg, 256, 0, h->stream>>>(U, V, a, b, C, Un, N)));
  CK(cudaGetLastError());
  h->ts_on = true;
  h->ts_a = a;
  h->ts_C = C;
  iga_status st = iga_solve_newton(h, U, &o, rep);
  h->ts_on = false;
  h->ts_a = 0.0;
  h->ts_C = nullptr;
  if (st == IGA_OK) {
    IGA_LAUNCH(h, KC_VEC, (k_alpha_end<<<eg, 256, 0, h->stream>>>(U, V, Un, 1.0 / af, 1.0 / (gam * dt), (1.0 - gam) / gam, N)));
  } else {  // leave U_n and U-dot_n as they were
    const std::string msg = h->err;
    CK(cudaMemcpyAsync(U, Un, N * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    h->err = msg;
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  return st;
}

// ---- tracing: launch counters and per-class event timing ----
int prof_begin(iga_s *h, int cls) {
  h->prof.launches[cls]++;
  if (!(h->prof.mask & (1u << cls))) return -1;
  ProfRec r;
  r.cls = cls;
  for (int k = 0; k < 2; k++) {
    cudaEvent_t e;
    if (!h->prof.pool.empty()) {
      e = h->prof.pool.back();
      h->prof.pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
      return -1;
    }
    (k == 0 ? r.a : r.b) = e;
  }
  cudaEventRecord(r.a, h->stream);
  h->prof.pending.push_back(r);
  return (int)h->prof.pending.size() - 1;
}

void prof_end(iga_s *h, int token) {
  if (token < 0) return;
  cudaEventRecord(h->prof.pending[token].b, h->stream);
}

static void prof_drain(iga_s *h) {
  if (h->prof.pending.empty()) return;
  cudaStreamSynchronize(h->stream);
  for (ProfRec &r : h->prof.pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      h->prof.ms[r.cls] += ms;
      h->prof.timed[r.cls]++;
    }
    h->prof.pool.push_back(r.a);
    h->prof.pool.push_back(r.b);
  }
  h->prof.pending.clear();
}

extern "C" iga_status iga_profile_enable(iga_t h, unsigned mask) {
  if (!h) return IGA_EINVAL;
  prof_drain(h);
  h->prof.mask = mask;
  if (h->inner) {  // a periodic handle's element kernels run on its inner handle
    prof_drain(h->inner);
    h->inner->prof.mask = mask;
  }
  return IGA_OK;
}

extern "C" iga_status iga_profile_read(iga_t h, iga_profile *out) {
  if (!h || !out) return IGA_EINVAL;
  memset(out, 0, sizeof *out);
  for (iga_s *x : {h, h->inner}) {
    if (!x) continue;
    prof_drain(x);
    for (int c = 0; c < KC_N; c++) {
      out->ms[c] += x->prof.ms[c];
      out->timed[c] += x->prof.timed[c];
      out->launches[c] += x->prof.launches[c];
      x->prof.ms[c] = 0.0;
      x->prof.timed[c] = 0;
      x->prof.launches[c] = 0;
    }
  }
  return IGA_OK;
}
