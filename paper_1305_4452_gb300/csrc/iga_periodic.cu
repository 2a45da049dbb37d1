// Periodic directions (Sec. 2.4): the unclamped space, the wrapped numbering
// (Eq. map-wrap) and the maps between a periodic handle and its inner handle.
//
// The inner handle is an ordinary discretisation on the unclamped knot vectors
// that keeps every unwrapped function i' in [0, nu) (no wrap, no Dirichlet rows),
// so all element, sum-factorisation and gather kernels run on it unchanged.  The
// periodic handle owns the wrapped system of n = nu - (k+1) functions per periodic
// direction:
//   U_u[I]      = U[wrap(I)]                                   (prolongation)
//   F[A]        = sum over the images I of A of F_u[I]          (residual rows)
//   J[A, B]     = sum over images I of A, J of B of J_u[I, J]   (Jacobian entries)
// i.e. the Galerkin system on the wrapped basis, whose functions are the sums of
// the unclamped B-splines that wrap onto them.  All sums run in a fixed order.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "iga_internal.h"

iga_status iga_create_impl(iga_s *h, const iga_desc *d, const iga_bratu *b);
void iga_release(iga_s *h);

namespace {

__device__ __forceinline__ void idx3(int64_t A, int n0, int n1, int &i0, int &i1, int &i2) {
  i0 = (int)(A % n0);
  int64_t t = A / n0;
  i1 = (int)(t % n1);
  i2 = (int)(t / n1);
}

// U_u[I] = U[wrap(I)]
__global__ void k_prolong(PerArgs P, const double *__restrict__ U, double *__restrict__ Uu, int64_t Nu) {
  const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= Nu) return;
  int a0, a1, a2;
  idx3(I, P.ax[0].nu, P.ax[1].nu, a0, a1, a2);
  const int64_t A = P.ax[0].wrap[a0] + (int64_t)P.ax[0].n * (P.ax[1].wrap[a1] + (int64_t)P.ax[1].n * P.ax[2].wrap[a2]);
  Uu[I] = U[A];
}

// F[A] = sum of F_u over the images of A (axis 2 outermost, each axis ascending);
// Dirichlet rows U_A - g (face order as in the non-periodic gather)
__global__ void k_restrict(PerArgs P, const double *__restrict__ Fu, const double *__restrict__ U, BndArgs bnd,
                           double *__restrict__ F, int64_t N) {
  const int64_t A = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (A >= N) return;
  int i[3];
  idx3(A, P.ax[0].n, P.ax[1].n, i[0], i[1], i[2]);
  bool on = false;
  double g = 0.0;
  for (int ax = 0; ax < 3; ax++) {
    if (bnd.flag[ax][0] && i[ax] == 0) { on = true; g = bnd.val[ax][0]; }
    if (bnd.flag[ax][1] && i[ax] == P.ax[ax].n - 1) { on = true; g = bnd.val[ax][1]; }
  }
  if (on) {
    F[A] = U[A] - g;
    return;
  }
  double acc = 0.0;
  for (int c2 = P.ax[2].img_off[i[2]]; c2 < P.ax[2].img_off[i[2] + 1]; c2++)
    for (int c1 = P.ax[1].img_off[i[1]]; c1 < P.ax[1].img_off[i[1] + 1]; c1++)
      for (int c0 = P.ax[0].img_off[i[0]]; c0 < P.ax[0].img_off[i[0] + 1]; c0++)
        acc += Fu[P.ax[0].img[c0] + (int64_t)P.ax[0].nu * (P.ax[1].img[c1] + (int64_t)P.ax[1].nu * P.ax[2].img[c2])];
  F[A] = acc;
}

// Row A of the wrapped Jacobian: for each column slot (t2, t1, t0) the sum of the
// unwrapped entries (I, J) that wrap onto (A, B); Dirichlet fix as the stage kernels
// apply it (identity row, zero column).
template <typename V>
__global__ void k_fold(PerArgs P, const int64_t *__restrict__ rowptr_u, const V *__restrict__ Ju,
                       const int64_t *__restrict__ rowptr, BndArgs bnd, V *__restrict__ vals, int64_t N) {
  const int64_t A = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (A >= N) return;
  int i[3];
  idx3(A, P.ax[0].n, P.ax[1].n, i[0], i[1], i[2]);
  bool row_on = false;
  for (int ax = 0; ax < 3; ax++)
    row_on |= (bnd.flag[ax][0] && i[ax] == 0) || (bnd.flag[ax][1] && i[ax] == P.ax[ax].n - 1);
  const PerAxis &X0 = P.ax[0], &X1 = P.ax[1], &X2 = P.ax[2];
  int64_t k = rowptr[A];
  for (int t2 = X2.col_off[i[2]]; t2 < X2.col_off[i[2] + 1]; t2++)
    for (int t1 = X1.col_off[i[1]]; t1 < X1.col_off[i[1] + 1]; t1++)
      for (int t0 = X0.col_off[i[0]]; t0 < X0.col_off[i[0] + 1]; t0++, k++) {
        const int c[3] = {X0.col[t0], X1.col[t1], X2.col[t2]};
        if (row_on) {
          vals[k] = (c[0] == i[0] && c[1] == i[1] && c[2] == i[2]) ? (V)1 : (V)0;
          continue;
        }
        bool col_on = false;
        for (int ax = 0; ax < 3; ax++)
          col_on |= (bnd.flag[ax][0] && c[ax] == 0) || (bnd.flag[ax][1] && c[ax] == P.ax[ax].n - 1);
        if (col_on) {
          vals[k] = (V)0;
          continue;
        }
        double s = 0.0;
        for (int q2 = X2.con_off[t2]; q2 < X2.con_off[t2 + 1]; q2++)
          for (int q1 = X1.con_off[t1]; q1 < X1.con_off[t1 + 1]; q1++)
            for (int q0 = X0.con_off[t0]; q0 < X0.con_off[t0 + 1]; q0++) {
              const int r0 = X0.con_row[q0], r1 = X1.con_row[q1], r2 = X2.con_row[q2];
              const int64_t I = r0 + (int64_t)X0.nu * (r1 + (int64_t)X1.nu * r2);
              const int64_t pos = X0.con_pos[q0] + (int64_t)X0.ulen[r0] * (X1.con_pos[q1] + (int64_t)X1.ulen[r1] * X2.con_pos[q2]);
              s += (double)Ju[rowptr_u[I] + pos];
            }
        vals[k] = (V)s;
      }
}

// y = A x on an explicit CSR pattern: 8 lanes per row, fixed-order lane sums
template <typename V>
__global__ void k_spmv_csr(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colidx, const V *__restrict__ vals,
                           const double *__restrict__ x, double *__restrict__ y, int64_t N, const double *__restrict__ done) {
  if (done && done[0] != 0.0) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t row = t >> 3;
  const int lane = (int)(t & 7);
  double acc = 0.0;
  if (row < N)
    for (int64_t k = rowptr[row] + lane; k < rowptr[row + 1]; k += 8) acc = fma((double)vals[k], x[colidx[k]], acc);
  acc += __shfl_xor_sync(0xffffffffu, acc, 4);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  if (row < N && lane == 0) y[row] = acc;
}

// dinv = 1 / diag(A) by a binary search of the (ascending) row for its own column
template <typename V>
__global__ void k_diag_csr(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colidx, const V *__restrict__ vals,
                           double *__restrict__ dinv, int64_t N) {
  const int64_t A = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (A >= N) return;
  int64_t lo = rowptr[A], hi = rowptr[A + 1] - 1;
  double d = 0.0;
  while (lo <= hi) {
    const int64_t mid = (lo + hi) >> 1;
    const int32_t c = colidx[mid];
    if (c == A) {
      d = (double)vals[mid];
      break;
    }
    if (c < A) lo = mid + 1;
    else hi = mid - 1;
  }
  dinv[A] = (d != 0.0) ? 1.0 / d : 1.0;
}

unsigned blocks_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

template <typename T>
cudaError_t upload_vec(iga_s *h, const std::vector<T> &v, const T **out) {
  T *p = nullptr;
  size_t bytes = std::max<size_t>(v.size(), 1) * sizeof(T);
  cudaError_t ce = cudaMalloc((void **)&p, bytes);
  if (ce) return ce;
  h->per_bufs.push_back(p);
  *out = p;
  if (v.empty()) return cudaMemset(p, 0, bytes);
  return cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// Per-axis maps from the inner handle's unwrapped stencils [l, r] (k1 = k+1 functions
// eliminated; 0: not periodic).
void build_axis(PerAxisHost &X, int nu, int k1, const std::vector<int> &l, const std::vector<int> &r) {
  X.nu = nu;
  X.n = nu - k1;
  X.wrap.resize(nu);
  for (int iu = 0; iu < nu; iu++) X.wrap[iu] = k1 ? iu % X.n : iu;  // Eq. (map-wrap) on [0, nu)
  X.img_off.assign(1, 0);
  X.img.clear();
  X.col_off.assign(1, 0);
  X.col.clear();
  X.con_off.assign(1, 0);
  X.con_row.clear();
  X.con_pos.clear();
  X.ulen.resize(nu);
  for (int iu = 0; iu < nu; iu++) X.ulen[iu] = r[iu] - l[iu] + 1;
  for (int i = 0; i < X.n; i++) {
    std::vector<int> im;
    for (int iu = i; iu < nu; iu += X.n) {
      im.push_back(iu);
      if (!k1) break;
    }
    X.img.insert(X.img.end(), im.begin(), im.end());
    X.img_off.push_back((int)X.img.size());
    std::vector<int> cols;
    for (int iu : im)
      for (int ju = l[iu]; ju <= r[iu]; ju++) cols.push_back(X.wrap[ju]);
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
    for (int c : cols) {
      X.col.push_back(c);
      for (int iu : im)
        for (int ju = l[iu]; ju <= r[iu]; ju++)
          if (X.wrap[ju] == c) {
            X.con_row.push_back(iu);
            X.con_pos.push_back(ju - l[iu]);
          }
      X.con_off.push_back((int)X.con_row.size());  // one entry per column slot
    }
    X.col_off.push_back((int)X.col.size());  // one entry per row
  }
}

}  // namespace

// Creation of a periodic handle: knots (Eqs. unclamp-left/right), the inner handle
// on the unclamped space with prolonged geometry, weights and log-kappa, the maps
// and the wrapped CSR pattern (Algorithm 2's stencils with wrapped columns).
iga_status iga_periodic_setup(iga_s *h, const iga_desc *d, const iga_bratu *b) {
  if (d->dim < 2 || d->dim > 3) {
    h->err = iga_format("dim must be 2 or 3 (got %d)", d->dim);
    return IGA_EINVAL;
  }
  const int dim = d->dim, p = d->degree[0];
  std::vector<double> K[3];
  int k1[3] = {0, 0, 0};
  for (int ax = 0; ax < dim; ax++) {
    if (d->degree[ax] != p || p < 1 || p > IGA_MAXP) {
      h->err = iga_format("degrees must be equal in every direction and in 1..%d", IGA_MAXP);
      return IGA_EINVAL;
    }
    iga_status st = iga_open_knots(h, d, ax, K[ax]);
    if (st != IGA_OK) return st;
    k1[ax] = d->periodic[ax];
    if (k1[ax] < 0 || k1[ax] > p) {
      h->err = iga_format("axis %d: periodic must be 0 or k+1 with 0 <= k <= p-1 (got %d)", ax, k1[ax]);
      return IGA_EINVAL;
    }
    if (k1[ax]) {
      st = iga_unclamp(h, ax, p, k1[ax] - 1, K[ax]);
      if (st != IGA_OK) return st;
    }
  }
  int nu[3] = {1, 1, 1}, n[3] = {1, 1, 1};
  int64_t N = 1, Nu = 1;
  for (int ax = 0; ax < dim; ax++) {
    nu[ax] = (int)K[ax].size() - p - 1;
    n[ax] = nu[ax] - k1[ax];
    N *= n[ax];
    Nu *= nu[ax];
  }
  // inputs per wrapped function, prolonged to the unwrapped ones
  auto wrapped = [&](int64_t I) {
    int64_t A = 0, s = 1, t = I;
    for (int ax = 0; ax < dim; ax++) {
      const int iu = (int)(t % nu[ax]);
      t /= nu[ax];
      A += (int64_t)(k1[ax] ? iu % n[ax] : iu) * s;
      s *= n[ax];
    }
    return A;
  };
  std::vector<double> ctrl_u, w_u, lk_u;
  if (d->ctrl) {
    ctrl_u.resize((size_t)Nu * dim);
    for (int64_t I = 0; I < Nu; I++)
      for (int c = 0; c < dim; c++) ctrl_u[(size_t)I * dim + c] = d->ctrl[(size_t)wrapped(I) * dim + c];
  }
  if (d->weights) {
    w_u.resize(Nu);
    for (int64_t I = 0; I < Nu; I++) w_u[I] = d->weights[wrapped(I)];
  }
  if (b && b->log_kappa) {
    lk_u.resize(Nu);
    for (int64_t I = 0; I < Nu; I++) lk_u[I] = b->log_kappa[wrapped(I)];
  }
  iga_desc di;
  memset(&di, 0, sizeof di);
  di.dim = dim;
  for (int ax = 0; ax < dim; ax++) {
    di.degree[ax] = p;
    di.continuity[ax] = -1;
    di.knots[ax] = K[ax].data();
    di.nknots[ax] = (int)K[ax].size();
    di.quad[ax] = d->quad[ax];
  }
  di.ctrl = d->ctrl ? ctrl_u.data() : nullptr;
  di.weights = d->weights ? w_u.data() : nullptr;
  iga_bratu bi;
  bi.lambda = b ? b->lambda : 0.0;
  bi.log_kappa = lk_u.empty() ? nullptr : lk_u.data();
  iga_s *in = new iga_s();
  in->stream = h->stream;
  in->unclamped = true;
  iga_status st = iga_create_impl(in, &di, &bi);
  if (st != IGA_OK) {
    h->err = in->err;
    iga_release(in);
    delete in;
    return st;
  }
  h->inner = in;
  h->dim = dim;
  h->p = p;
  h->q = in->q;
  h->N = N;
  h->nelem = in->nelem;
  h->nqp = in->nqp;
  h->lambda = in->lambda;
  h->gl = in->gl;
  h->has_geom = in->has_geom;
  h->has_w = in->has_w;
  h->has_kappa = in->has_kappa;
  for (int ax = 0; ax < 3; ax++) {
    h->dir[ax].p = in->dir[ax].p;
    h->dir[ax].q = in->dir[ax].q;
    h->dir[ax].nel = in->dir[ax].nel;
    h->dir[ax].n = n[ax];
  }
  // maps per axis (trivial ones for the unused third axis of 2D)
  for (int ax = 0; ax < 3; ax++) {
    if (ax < dim) build_axis(h->per_host[ax], nu[ax], k1[ax], in->dir[ax].l, in->dir[ax].r);
    else build_axis(h->per_host[ax], 1, 0, std::vector<int>(1, 0), std::vector<int>(1, 0));
  }
  // wrapped pattern: row A is the lexicographic product of its per-axis column lists
  const PerAxisHost &X0 = h->per_host[0], &X1 = h->per_host[1], &X2 = h->per_host[2];
  std::vector<int64_t> rowptr((size_t)N + 1);
  int64_t nnz = 0;
  for (int64_t A = 0; A < N; A++) {
    const int i0 = (int)(A % n[0]), i1 = (int)((A / n[0]) % n[1]), i2 = (int)(A / ((int64_t)n[0] * n[1]));
    rowptr[A] = nnz;
    nnz += (int64_t)(X0.col_off[i0 + 1] - X0.col_off[i0]) * (X1.col_off[i1 + 1] - X1.col_off[i1]) *
           (X2.col_off[i2 + 1] - X2.col_off[i2]);
  }
  rowptr[N] = nnz;
  if (nnz > (int64_t)INT32_MAX * 8) {
    h->err = "periodic pattern too large";
    return IGA_EINVAL;
  }
  std::vector<int32_t> colidx((size_t)nnz);
  for (int64_t A = 0; A < N; A++) {
    const int i0 = (int)(A % n[0]), i1 = (int)((A / n[0]) % n[1]), i2 = (int)(A / ((int64_t)n[0] * n[1]));
    int64_t k = rowptr[A];
    for (int t2 = X2.col_off[i2]; t2 < X2.col_off[i2 + 1]; t2++)
      for (int t1 = X1.col_off[i1]; t1 < X1.col_off[i1 + 1]; t1++)
        for (int t0 = X0.col_off[i0]; t0 < X0.col_off[i0 + 1]; t0++)
          colidx[k++] = (int32_t)(X0.col[t0] + (int64_t)n[0] * (X1.col[t1] + (int64_t)n[1] * X2.col[t2]));
  }
  h->nnz = nnz;
#define PCK(call)                                                         \
  do {                                                                    \
    cudaError_t ce_ = (call);                                             \
    if (ce_ != cudaSuccess) {                                             \
      h->err = iga_format("%s: %s", #call, cudaGetErrorString(ce_));      \
      return (ce_ == cudaErrorMemoryAllocation) ? IGA_ENOMEM : IGA_ECUDA; \
    }                                                                     \
  } while (0)
  PCK(cudaMalloc((void **)&h->rowptr, rowptr.size() * sizeof(int64_t)));
  PCK(cudaMemcpy(h->rowptr, rowptr.data(), rowptr.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  PCK(cudaMalloc((void **)&h->colidx, std::max<size_t>(colidx.size(), 1) * sizeof(int32_t)));
  PCK(cudaMemcpy(h->colidx, colidx.data(), colidx.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  for (int ax = 0; ax < 3; ax++) {
    const PerAxisHost &X = h->per_host[ax];
    PerAxis &D = h->per.ax[ax];
    D.n = X.n;
    D.nu = X.nu;
    PCK(upload_vec(h, X.wrap, &D.wrap));
    PCK(upload_vec(h, X.img_off, &D.img_off));
    PCK(upload_vec(h, X.img, &D.img));
    PCK(upload_vec(h, X.col_off, &D.col_off));
    PCK(upload_vec(h, X.col, &D.col));
    PCK(upload_vec(h, X.con_off, &D.con_off));
    PCK(upload_vec(h, X.con_row, &D.con_row));
    PCK(upload_vec(h, X.con_pos, &D.con_pos));
    PCK(upload_vec(h, X.ulen, &D.ulen));
  }
  PCK(cudaMalloc((void **)&h->Uu, (size_t)Nu * sizeof(double)));
  PCK(cudaMalloc((void **)&h->Fu, (size_t)Nu * sizeof(double)));
#undef PCK
  return IGA_OK;
}

void periodic_release(iga_s *h) {
  for (void *p : h->per_bufs) cudaFree(p);
  h->per_bufs.clear();
  void *ps[] = {h->Uu, h->Fu, h->Cu, h->Ju, h->Ju32};
  for (void *p : ps)
    if (p) cudaFree(p);
  h->Uu = h->Fu = h->Cu = h->Ju = nullptr;
  h->Ju32 = nullptr;
  if (h->inner) {
    iga_release(h->inner);
    delete h->inner;
    h->inner = nullptr;
  }
}

// The inner handle's time-dependent state follows the periodic handle's (the rate
// data C prolonged like U).
static cudaError_t sync_ts(iga_s *h) {
  iga_s *in = h->inner;
  in->ts_on = h->ts_on;
  in->ts_a = h->ts_a;
  in->ts_C = nullptr;
  if (h->ts_on && h->ts_C) {
    if (!h->Cu) {
      cudaError_t ce = cudaMalloc((void **)&h->Cu, (size_t)in->N * sizeof(double));
      if (ce) return ce;
    }
    IGA_LAUNCH(h, KC_VEC, (k_prolong<<<blocks_for(in->N, 256), 256, 0, h->stream>>>(h->per, h->ts_C, h->Cu, in->N)));
    in->ts_C = h->Cu;
  }
  return cudaSuccess;
}

static void unsync_ts(iga_s *h) {
  h->inner->ts_on = false;
  h->inner->ts_a = 0.0;
  h->inner->ts_C = nullptr;
}

cudaError_t periodic_residual(iga_s *h, const double *U, double *F) {
  iga_s *in = h->inner;
  in->lambda = h->lambda;
  IGA_LAUNCH(h, KC_VEC, (k_prolong<<<blocks_for(in->N, 256), 256, 0, h->stream>>>(h->per, U, h->Uu, in->N)));
  cudaError_t ce = sync_ts(h);
  if (!ce) ce = launch_residual(in, h->Uu, h->Fu);
  unsync_ts(h);
  if (ce) return ce;
  IGA_LAUNCH(h, KC_RES_GATHER, (k_restrict<<<blocks_for(h->N, 256), 256, 0, h->stream>>>(h->per, h->Fu, U, h->bnd, F, h->N)));
  return cudaGetLastError();
}

template <typename V>
static cudaError_t periodic_jacobian(iga_s *h, const double *U, V *vals, V **Ju) {
  iga_s *in = h->inner;
  in->lambda = h->lambda;
  if (!*Ju) {
    cudaError_t ce = cudaMalloc((void **)Ju, (size_t)in->nnz * sizeof(V));
    if (ce) return ce;
  }
  IGA_LAUNCH(h, KC_VEC, (k_prolong<<<blocks_for(in->N, 256), 256, 0, h->stream>>>(h->per, U, h->Uu, in->N)));
  cudaError_t ce = sync_ts(h);
  in->q00_valid = false;
  if (!ce) {
    if (sizeof(V) == 8) ce = launch_jacobian64(in, h->Uu, (double *)*Ju, 3, nullptr);
    else ce = launch_jacobian32(in, h->Uu, (float *)*Ju, 3, nullptr);
  }
  unsync_ts(h);
  if (ce) return ce;
  IGA_LAUNCH(h, KC_COMBINE, (k_fold<V><<<blocks_for(h->N, 128), 128, 0, h->stream>>>(h->per, in->rowptr, *Ju, h->rowptr, h->bnd,
                                                                                      vals, h->N)));
  return cudaGetLastError();
}

cudaError_t periodic_jacobian64(iga_s *h, const double *U, double *vals) { return periodic_jacobian<double>(h, U, vals, &h->Ju); }
cudaError_t periodic_jacobian32(iga_s *h, const double *U, float *vals) { return periodic_jacobian<float>(h, U, vals, &h->Ju32); }

cudaError_t periodic_spmv(iga_s *h, const void *vals, int is_f32, const double *x, double *y, const double *done) {
  const unsigned g = blocks_for(h->N * 8, 256);
  if (is_f32)
    IGA_LAUNCH(h, KC_SPMV, (k_spmv_csr<float><<<g, 256, 0, h->stream>>>(h->rowptr, h->colidx, (const float *)vals, x, y, h->N, done)));
  else
    IGA_LAUNCH(h, KC_SPMV, (k_spmv_csr<double><<<g, 256, 0, h->stream>>>(h->rowptr, h->colidx, (const double *)vals, x, y, h->N, done)));
  return cudaGetLastError();
}

cudaError_t periodic_diag_inv(iga_s *h, const void *vals, int is_f32, double *dinv) {
  const unsigned g = blocks_for(h->N, 256);
  if (is_f32)
    IGA_LAUNCH(h, KC_VEC, (k_diag_csr<float><<<g, 256, 0, h->stream>>>(h->rowptr, h->colidx, (const float *)vals, dinv, h->N)));
  else
    IGA_LAUNCH(h, KC_VEC, (k_diag_csr<double><<<g, 256, 0, h->stream>>>(h->rowptr, h->colidx, (const double *)vals, dinv, h->N)));
  return cudaGetLastError();
}
