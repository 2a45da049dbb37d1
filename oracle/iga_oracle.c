/*
 * Oracle for the isogeometric Bratu assembly path: a plain, slow, single-threaded
 * FP64 CPU implementation written directly from the PetIGA paper (Dalcin et al.,
 * "PetIGA: A framework for high-performance isogeometric analysis").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
 * Python binding) may link, import or call this file; only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark do.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it computes, and where the paper defines it:
 *   - B-spline values by the Cox-de Boor recursion, Sec. 2.1 Eqs. (1)-(2), with
 *     0/0 taken as 0; first derivatives by Eq. (3), read with a MINUS between the
 *     two terms (the printed "+" contradicts differentiating Eq. (2); the pins
 *     "sum of derivatives = 0" in the tests fail with "+").
 *   - Tensor-product basis M_A = B_i B_j B_k and natural index
 *     A = i + j(n+1) + k(n+1)(m+1), Sec. 2.2 Eq. (5).
 *   - Rational basis N_A = w_A M_A / w and its first parametric derivatives,
 *     Sec. 2.3 Eqs. (6)-(7) and Eq. (drational).
 *   - Geometry map x = sum x_A N_A, its parametric derivatives, the inverse map by
 *     solving delta_ij = x_{i,e} xi_{e,j}, and spatial basis gradients
 *     N_{A,i} = N_{A,a} xi_{a,i}, Appendix A Eqs. (identity), (dspatial).
 *   - Element-by-element Gauss-Legendre assembly of the residual, Sec. 2.7
 *     Algorithm 3, with the Bratu integrand of Sec. 3.1 Eq. (residual); the
 *     Jacobian of Eq. (jacobian), assembled "in a similar fashion" (Sec. 2.7).
 *   - The Jacobian by local numerical differentiation, Sec. 2.8 Eq. (fdjac):
 *     forward differences of the quadrature-point integrand in each element value,
 *     step sqrt(eps) sqrt(1 + ||U_e||_2) (or_jacobian_fd).
 *   - The mass matrix (N_A, N_B) of the time-dependent residual of Sec. 4.2
 *     (the u-dot term of R(w; u-dot, u)), by the same quadrature (or_mass).
 *   - Periodic spaces, Sec. 2.4: the caller passes the knot vector unclamped by
 *     Eqs. (unclamp-left)-(unclamp-right) and wrap[d] = k+1, the number of redundant
 *     functions; every function index i is wrapped by Eq. (map-wrap),
 *     i -> mod(i, n-k), in the assembly, the pattern and the brute-force check.
 *   - The CSR adjacency pattern from BasisStencil, Sec. 2.5 Algorithm 2, in
 *     lexicographic tensor-product order.
 *   - Dirichlet rows set with IGASetBoundaryValue (Sec. 3.2): F_A = U_A - g and an
 *     identity row with a zeroed column (the paper gives only the API; this
 *     reading keeps the Jacobian symmetric).
 *   - The kappa-weighted variant -div(kappa grad u) - lambda e^u (not in the paper)
 *     with kappa = exp(sum logkappa_A N_A).
 *
 * Every function returns 0 on success and a negative code on malformed input.
 *
 * Timing mode (or_residual_colored, or_jacobian_colored): the same element loop and
 * element arithmetic, with the elements visited colour by colour and each colour's
 * elements spread over OpenMP threads (when compiled with OpenMP).  Two elements whose
 * span indices agree modulo p+1 in every direction share no basis function (a function
 * is supported on at most p+1 consecutive non-empty spans, Sec. 2.1), so the threads of
 * one colour write disjoint entries.  Only the order in which element contributions are
 * added changes.  It exists to time the oracle on all host cores; the checks use the
 * serial functions.  The per-point scratch arrays are thread-local for this reason.
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXD 3
#define OR_MAXP 8
#define OR_MAXEN 729 /* (OR_MAXP+1)^3 */
#define OR_TLS _Thread_local

typedef struct {
  int dim;
  int p[3];                /* degree per direction */
  int m[3];                /* number of knots per direction */
  const double *U[3];      /* knot vectors */
  int q[3];                /* Gauss-Legendre points per direction */
  const double *ctrl;      /* N*dim physical control points, or NULL: x = xi */
  const double *weights;   /* N rational weights, or NULL: all 1 */
  double lambda;
  const double *log_kappa; /* N coefficients of log kappa, or NULL: kappa = 1 */
  int bnd[3][2];           /* Dirichlet flag per (axis, side) */
  double bval[3][2];       /* Dirichlet value per (axis, side) */
  int source;              /* 1: add the manufactured source of u* = prod sin(pi x) */
  int wrap[3];             /* periodic direction: k+1 (unclamped knots, C^k across the
                              boundary); 0: not periodic */
} or_problem;

/* ---------------- Sec. 2.1: B-spline basis, Cox-de Boor ---------------- */

/* Eq. (1)-(2): B_{i,p}(xi); 0/0 := 0. */
double or_bspline(int i, int p, const double *U, double xi) {
  if (p == 0) return (U[i] <= xi && xi < U[i + 1]) ? 1.0 : 0.0;
  double left = 0.0, right = 0.0;
  double dl = U[i + p] - U[i];
  double dr = U[i + p + 1] - U[i + 1];
  if (dl != 0.0) left = (xi - U[i]) / dl * or_bspline(i, p - 1, U, xi);
  if (dr != 0.0) right = (U[i + p + 1] - xi) / dr * or_bspline(i + 1, p - 1, U, xi);
  return left + right;
}

/* Eq. (3) with the sign that differentiating Eq. (2) gives:
 * B'_{i,p} = p/(U[i+p]-U[i]) B_{i,p-1} - p/(U[i+p+1]-U[i+1]) B_{i+1,p-1}. */
double or_bspline_der(int i, int p, const double *U, double xi) {
  if (p == 0) return 0.0;
  double left = 0.0, right = 0.0;
  double dl = U[i + p] - U[i];
  double dr = U[i + p + 1] - U[i + 1];
  if (dl != 0.0) left = p / dl * or_bspline(i, p - 1, U, xi);
  if (dr != 0.0) right = p / dr * or_bspline(i + 1, p - 1, U, xi);
  return left - right;
}

/* Legendre polynomial P_q(z) and its derivative by the three-term recurrence
 * (k P_k = (2k-1) z P_{k-1} - (k-1) P_{k-2}). */
static void legendre(int q, double z, double *pq, double *dpq) {
  double pkm1 = 1.0, pk = z;
  for (int k = 2; k <= q; k++) {
    double pn = ((2.0 * k - 1.0) * z * pk - (k - 1.0) * pkm1) / k;
    pkm1 = pk;
    pk = pn;
  }
  *pq = pk;
  *dpq = q * (z * pk - pkm1) / (z * z - 1.0);
}

/* Gauss-Legendre nodes/weights on [-1,1] (Sec. 2.9: "standard tensor product
 * Gauss-Legendre quadrature"): Newton iteration on P_q from the usual cosine
 * guesses; w = 2 / ((1 - z^2) P_q'(z)^2).  Nodes ascending. */
int or_gauss_legendre(int q, double *x, double *w) {
  if (q < 1 || q > 64) return -1;
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < q; i++) {
    double z = cos(pi * (i + 0.75) / (q + 0.5)), pq, dp;
    for (int it = 0; it < 100; it++) {
      legendre(q, z, &pq, &dp);
      double dz = pq / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    legendre(q, z, &pq, &dp);
    x[q - 1 - i] = z;
    w[q - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  return 0;
}

/* Number of basis functions in direction d: m - p - 1 (Sec. 2.1), less the k+1
 * functions a periodic direction eliminates (Sec. 2.4). */
static int nfun(const or_problem *P, int d) { return P->m[d] - P->p[d] - 1 - P->wrap[d]; }

/* Eq. (map-wrap): mod(a, b) = a - b floor(a / b), for any integer a. */
static int map_wrap(int a, int b) {
  int q = a / b;
  if (a % b != 0 && a < 0) q -= 1;
  return a - b * q;
}

int or_num_funcs(const or_problem *P, int d) { return nfun(P, d); }

/* Elements are the non-empty knot spans (Sec. 2.6); span index s has
 * U[s] < U[s+1], p <= s <= n-1 for an open knot vector. */
int or_spans(const double *U, int m, int p, int *spans) {
  int n = m - p - 1, c = 0;
  for (int s = p; s < n; s++)
    if (U[s] < U[s + 1]) {
      if (spans) spans[c] = s;
      c++;
    }
  return c;
}

/* Sec. 2.5 Algorithm 2 (BasisStencil): left-most and right-most basis functions
 * whose support overlaps that of basis i. */
void or_stencil(int i, int p, const double *U, int *l, int *r) {
  int j = i;
  while (U[j] == U[j + 1]) j++;
  *l = j - p;
  j = i + p + 1;
  while (U[j] == U[j - 1]) j--;
  *r = j - 1;
}

static int64_t num_dofs(const or_problem *P) {
  int64_t N = 1;
  for (int d = 0; d < P->dim; d++) N *= nfun(P, d);
  return N;
}

int64_t or_num_dofs(const or_problem *P) { return num_dofs(P); }

static int check(const or_problem *P) {
  if (P->dim < 1 || P->dim > 3) return -1;
  for (int d = 0; d < P->dim; d++) {
    if (P->p[d] < 0 || P->p[d] > OR_MAXP) return -2;
    if (P->m[d] < 2 * P->p[d] + 2) return -3;
    if (P->q[d] < 1 || P->q[d] > 16) return -4;
    for (int k = 0; k + 1 < P->m[d]; k++)
      if (P->U[d][k] > P->U[d][k + 1]) return -5; /* knots must not decrease */
    if (P->wrap[d] < 0 || P->wrap[d] > P->p[d] || nfun(P, d) < 1) return -7;
    if (P->wrap[d] && (P->bnd[d][0] || P->bnd[d][1])) return -8; /* no Dirichlet face on a periodic axis */
  }
  int nen = 1;
  for (int d = 0; d < P->dim; d++) nen *= P->p[d] + 1;
  if (nen > OR_MAXEN) return -6;
  return 0;
}

/* CSR pattern by BasisStencil (Algorithm 2) per direction and the lexicographic
 * tensor product of the ranges (Sec. 2.5).  Rows and columns are in the natural
 * order of Eq. (5).  With colidx == NULL only rowptr is filled; returns nnz. */
/* The 1D column list of function i in direction d: BasisStencil's range, each
 * index wrapped by Eq. (map-wrap) in a periodic direction (Sec. 2.5), sorted and
 * without repeats.  Returns its length. */
static int column_list(const or_problem *P, int d, int i, int *cols) {
  int l, r, c = 0, n = nfun(P, d);
  or_stencil(i, P->p[d], P->U[d], &l, &r);
  for (int j = l; j <= r; j++) {
    int w = P->wrap[d] ? map_wrap(j, n) : j, seen = 0;
    for (int t = 0; t < c; t++) seen |= cols[t] == w;
    if (!seen) cols[c++] = w;
  }
  for (int a = 1; a < c; a++)  /* insertion sort */
    for (int b = a; b > 0 && cols[b - 1] > cols[b]; b--) {
      int t = cols[b];
      cols[b] = cols[b - 1];
      cols[b - 1] = t;
    }
  return c;
}

int64_t or_pattern(const or_problem *P, int64_t *rowptr, int32_t *colidx) {
  if (check(P)) return -1;
  int n[3] = {1, 1, 1};
  for (int d = 0; d < P->dim; d++) n[d] = nfun(P, d);
  int64_t N = num_dofs(P), nnz = 0;
  int cl[3][4 * OR_MAXP + 4], len[3] = {1, 1, 1};
  for (int64_t A = 0; A < N; A++) {
    int idx[3] = {0, 0, 0};
    int64_t t = A;
    for (int d = 0; d < P->dim; d++) { idx[d] = (int)(t % n[d]); t /= n[d]; }
    cl[1][0] = cl[2][0] = 0;
    for (int d = 0; d < P->dim; d++) len[d] = column_list(P, d, idx[d], cl[d]);
    if (rowptr) rowptr[A] = nnz;
    for (int k = 0; k < len[2]; k++)
      for (int j = 0; j < len[1]; j++)
        for (int i = 0; i < len[0]; i++) {
          if (colidx) colidx[nnz] = (int32_t)(cl[0][i] + (int64_t)n[0] * (cl[1][j] + (int64_t)n[1] * cl[2][k]));
          nnz++;
        }
  }
  if (rowptr) rowptr[N] = nnz;
  return nnz;
}

/* Second, independent construction of the pattern: every pair of nodes that
 * share an element (the element connectivity of Sec. 2.6), marked in a dense
 * N x N byte matrix.  Small problems only. */
int or_pattern_dense_from_elements(const or_problem *P, unsigned char *mark) {
  if (check(P)) return -1;
  int n[3] = {1, 1, 1}, ne[3] = {1, 1, 1}, pp[3] = {0, 0, 0};
  int *sp[3] = {NULL, NULL, NULL};
  for (int d = 0; d < P->dim; d++) {
    n[d] = nfun(P, d);
    pp[d] = P->p[d];
    ne[d] = or_spans(P->U[d], P->m[d], P->p[d], NULL);
    sp[d] = (int *)malloc(sizeof(int) * (ne[d] + 1));
    or_spans(P->U[d], P->m[d], P->p[d], sp[d]);
  }
  int64_t N = num_dofs(P);
  memset(mark, 0, (size_t)(N * N));
  int s0[3] = {0, 0, 0};
  for (int e2 = 0; e2 < ne[2]; e2++)
    for (int e1 = 0; e1 < ne[1]; e1++)
      for (int e0 = 0; e0 < ne[0]; e0++) {
        int e[3] = {e0, e1, e2};
        for (int d = 0; d < 3; d++) s0[d] = (d < P->dim) ? sp[d][e[d]] - pp[d] : 0;
        for (int c2 = 0; c2 <= pp[2]; c2++)
          for (int c1 = 0; c1 <= pp[1]; c1++)
            for (int c0 = 0; c0 <= pp[0]; c0++) {
              int64_t A = map_wrap(s0[0] + c0, n[0]) +
                          (int64_t)n[0] * (map_wrap(s0[1] + c1, n[1]) + (int64_t)n[1] * map_wrap(s0[2] + c2, n[2]));
              for (int b2 = 0; b2 <= pp[2]; b2++)
                for (int b1 = 0; b1 <= pp[1]; b1++)
                  for (int b0 = 0; b0 <= pp[0]; b0++) {
                    int64_t B = map_wrap(s0[0] + b0, n[0]) +
                                (int64_t)n[0] * (map_wrap(s0[1] + b1, n[1]) + (int64_t)n[1] * map_wrap(s0[2] + b2, n[2]));
                    mark[A * N + B] = 1;
                  }
            }
      }
  for (int d = 0; d < P->dim; d++) free(sp[d]);
  return 0;
}

/* ------------- Sec. 2.2-2.3 and Appendix A: shape functions at a point -------------
 * Given the element's span indices s[d] and a parametric point xi[d], returns for the
 * nen = prod(p+1) nonzero functions (local index first-direction fastest):
 *   gidx[a]        natural global index (Eq. 5),
 *   N[a]           rational basis (Eq. rational),
 *   dN[a*dim+i]    spatial gradient N_{A,i} (Eq. dspatial),
 * and x[i] (the mapped point) and detJ = det(x_{i,alpha}). */
int or_shape(const or_problem *P, const int *s, const double *xi, int64_t *gidx, double *N,
             double *dN, double *x, double *detJ) {
  int dim = P->dim;
  int n[3] = {1, 1, 1}, pp[3] = {0, 0, 0};
  double b[3][OR_MAXP + 1], db[3][OR_MAXP + 1];
  for (int d = 0; d < 3; d++) {
    if (d < dim) {
      n[d] = nfun(P, d);
      pp[d] = P->p[d];
      for (int a = 0; a <= pp[d]; a++) {
        int i = s[d] - pp[d] + a;
        b[d][a] = or_bspline(i, pp[d], P->U[d], xi[d]);
        db[d][a] = or_bspline_der(i, pp[d], P->U[d], xi[d]);
      }
    } else {
      b[d][0] = 1.0;
      db[d][0] = 0.0;
    }
  }
  int nen = (pp[0] + 1) * (pp[1] + 1) * (pp[2] + 1);
  static OR_TLS double M[OR_MAXEN], dM[OR_MAXEN][3], wA[OR_MAXEN];
  int a = 0;
  for (int c2 = 0; c2 <= pp[2]; c2++)
    for (int c1 = 0; c1 <= pp[1]; c1++)
      for (int c0 = 0; c0 <= pp[0]; c0++, a++) {
        int c[3] = {c0, c1, c2};
        int64_t G = 0, stride = 1;
        for (int d = 0; d < dim; d++) {
          G += (int64_t)map_wrap(s[d] - pp[d] + c[d], n[d]) * stride; /* Eq. (map-wrap) */
          stride *= n[d];
        }
        gidx[a] = G;
        /* Eq. (5): tensor product; derivative in direction alpha hits one factor */
        M[a] = b[0][c0] * b[1][c1] * b[2][c2];
        dM[a][0] = db[0][c0] * b[1][c1] * b[2][c2];
        dM[a][1] = b[0][c0] * db[1][c1] * b[2][c2];
        dM[a][2] = b[0][c0] * b[1][c1] * db[2][c2];
        wA[a] = P->weights ? P->weights[G] : 1.0;
      }
  /* Eqs. (6)-(7): weighting function and its first derivatives */
  double W = 0.0, Wd[3] = {0.0, 0.0, 0.0};
  for (a = 0; a < nen; a++) {
    W += wA[a] * M[a];
    for (int al = 0; al < dim; al++) Wd[al] += wA[a] * dM[a][al];
  }
  /* Eq. (rational) and Eq. (drational): N_{A,alpha} = (w_A M_{A,alpha} - N_A w_{,alpha}) / w */
  static OR_TLS double dNp[OR_MAXEN][3];
  for (a = 0; a < nen; a++) {
    N[a] = wA[a] * M[a] / W;
    for (int al = 0; al < dim; al++) dNp[a][al] = (wA[a] * dM[a][al] - N[a] * Wd[al]) / W;
  }
  /* Appendix A: x = sum x_A N_A, x_{i,alpha} = sum x_A N_{A,alpha}; without control
   * points the map is the identity x = xi. */
  double F[3][3];
  for (int i = 0; i < dim; i++) {
    if (P->ctrl) {
      x[i] = 0.0;
      for (int al = 0; al < dim; al++) F[i][al] = 0.0;
      for (a = 0; a < nen; a++) {
        double xa = P->ctrl[gidx[a] * dim + i];
        x[i] += xa * N[a];
        for (int al = 0; al < dim; al++) F[i][al] += xa * dNp[a][al];
      }
    } else {
      x[i] = xi[i];
      for (int al = 0; al < dim; al++) F[i][al] = (i == al) ? 1.0 : 0.0;
    }
  }
  /* Eq. (identity): delta_ij = x_{i,e} xi_{e,j}; solve for xi_{e,j} by Gauss-Jordan
   * elimination with partial pivoting; det from the pivots. */
  double Aug[3][6];
  for (int i = 0; i < dim; i++)
    for (int j = 0; j < 2 * dim; j++) Aug[i][j] = (j < dim) ? F[i][j] : ((j - dim == i) ? 1.0 : 0.0);
  double det = 1.0;
  for (int c = 0; c < dim; c++) {
    int piv = c;
    for (int r = c + 1; r < dim; r++)
      if (fabs(Aug[r][c]) > fabs(Aug[piv][c])) piv = r;
    if (Aug[piv][c] == 0.0) return -10;
    if (piv != c) {
      for (int j = 0; j < 2 * dim; j++) {
        double t = Aug[c][j];
        Aug[c][j] = Aug[piv][j];
        Aug[piv][j] = t;
      }
      det = -det;
    }
    double pv = Aug[c][c];
    det *= pv;
    for (int j = 0; j < 2 * dim; j++) Aug[c][j] /= pv;
    for (int r = 0; r < dim; r++)
      if (r != c) {
        double f = Aug[r][c];
        for (int j = 0; j < 2 * dim; j++) Aug[r][j] -= f * Aug[c][j];
      }
  }
  /* Aug[e][dim + j] = xi_{e,j}; Eq. (dspatial): N_{A,i} = N_{A,e} xi_{e,i} */
  for (a = 0; a < nen; a++)
    for (int i = 0; i < dim; i++) {
      double g = 0.0;
      for (int e = 0; e < dim; e++) g += dNp[a][e] * Aug[e][dim + i];
      dN[a * dim + i] = g;
    }
  *detJ = det;
  return nen;
}

/* Manufactured solution u* = prod sin(pi x_i) and its source
 * f = dim pi^2 u* - lambda exp(u*), so that -lap u* - lambda e^{u*} = f. */
static double manufactured_u(int dim, const double *x) {
  const double pi = 3.14159265358979323846;
  double u = 1.0;
  for (int i = 0; i < dim; i++) u *= sin(pi * x[i]);
  return u;
}

double or_manufactured_u(int dim, const double *x) { return manufactured_u(dim, x); }

static double manufactured_f(int dim, double lambda, const double *x) {
  const double pi = 3.14159265358979323846;
  double u = manufactured_u(dim, x);
  return dim * pi * pi * u - lambda * exp(u);
}

/* Per-element, per-quadrature-point loop of Algorithm 3 (Sec. 2.7), calling back
 * into a consumer with the point data.  Each element's local residual and
 * matrix are formed by the plain loops over test index a and trial index b. */
typedef struct {
  const or_problem *P;
  int ne[3];
  int *sp[3];
  double gx[3][16], gw[3][16];
} or_mesh;

static int mesh_init(const or_problem *P, or_mesh *M) {
  int rc = check(P);
  if (rc) return rc;
  M->P = P;
  for (int d = 0; d < 3; d++) {
    M->sp[d] = NULL;
    M->ne[d] = 1;
  }
  for (int d = 0; d < P->dim; d++) {
    M->ne[d] = or_spans(P->U[d], P->m[d], P->p[d], NULL);
    M->sp[d] = (int *)malloc(sizeof(int) * (M->ne[d] + 1));
    or_spans(P->U[d], P->m[d], P->p[d], M->sp[d]);
    or_gauss_legendre(P->q[d], M->gx[d], M->gw[d]);
  }
  return 0;
}

static void mesh_free(or_mesh *M) {
  for (int d = 0; d < 3; d++) free(M->sp[d]);
}

/* Element integrals of one element: Fe[a] and (optionally) Ke[a*nen+b].
 * Sec. 2.7 Algorithm 3 steps: gather U_e, loop over quadrature points, ShapeFuns,
 * Integrand of Eq. (residual) / Eq. (jacobian), accumulate J_q w_q F_q.
 * fd != 0: Ke by the local numerical differentiation of Sec. 2.8, Eq. (fdjac):
 * at every quadrature point, column b of dF_q/dU_e is (F_q(U_e + delta e_b) - F_q(U_e))
 * / delta with delta = sqrt(eps) * sqrt(1 + ||U_e||_2), F_q recomputed from the
 * perturbed element values. */
static int element_integrals_mode(const or_mesh *Msh, const int *e, const double *Uc, int64_t *gidx,
                                  double *Fe, double *Ke, int fd);
static int element_integrals(const or_mesh *Msh, const int *e, const double *Uc, int64_t *gidx,
                             double *Fe, double *Ke) {
  return element_integrals_mode(Msh, e, Uc, gidx, Fe, Ke, 0);
}

/* F_q[a] (a < nen) at one quadrature point from element values Ue (the integrand of
 * Eq. (residual) times J_q w_q, without the U-independent source term) */
static void point_integrand(int dim, int nen, const double *N, const double *dN, const double *Ue, double kappa,
                            double lambda, double jw, double *Fq) {
  double u = 0.0, gu[3] = {0, 0, 0};
  for (int a = 0; a < nen; a++) {
    u += Ue[a] * N[a];
    for (int i = 0; i < dim; i++) gu[i] += Ue[a] * dN[a * dim + i];
  }
  double re = lambda * exp(u);
  for (int a = 0; a < nen; a++) {
    double gg = 0.0;
    for (int i = 0; i < dim; i++) gg += dN[a * dim + i] * gu[i];
    Fq[a] = jw * (kappa * gg - re * N[a]);
  }
}

static int element_integrals_mode(const or_mesh *Msh, const int *e, const double *Uc, int64_t *gidx,
                                  double *Fe, double *Ke, int fd) {
  const or_problem *P = Msh->P;
  int dim = P->dim;
  int s[3] = {0, 0, 0}, q[3] = {1, 1, 1};
  for (int d = 0; d < dim; d++) {
    s[d] = Msh->sp[d][e[d]];
    q[d] = P->q[d];
  }
  int nen = 1;
  for (int d = 0; d < dim; d++) nen *= P->p[d] + 1;
  for (int a = 0; a < nen; a++) Fe[a] = 0.0;
  if (Ke)
    for (int a = 0; a < nen * nen; a++) Ke[a] = 0.0;
  static OR_TLS double N[OR_MAXEN], dN[OR_MAXEN * 3];
  for (int g2 = 0; g2 < q[2]; g2++)
    for (int g1 = 0; g1 < q[1]; g1++)
      for (int g0 = 0; g0 < q[0]; g0++) {
        int g[3] = {g0, g1, g2};
        double xi[3] = {0, 0, 0}, wq = 1.0;
        for (int d = 0; d < dim; d++) {
          double lo = P->U[d][s[d]], hi = P->U[d][s[d] + 1];
          xi[d] = 0.5 * (lo + hi) + 0.5 * (hi - lo) * Msh->gx[d][g[d]];
          wq *= Msh->gw[d][g[d]] * 0.5 * (hi - lo);
        }
        double x[3], detJ;
        int rc = or_shape(P, s, xi, gidx, N, dN, x, &detJ);
        if (rc < 0) return rc;
        double jw = detJ * wq; /* J_q w_q of Algorithm 3 */
        /* Eqs. (wuh0)-(wuh1): u^h and grad u^h at the point */
        double u = 0.0, gu[3] = {0, 0, 0}, lk = 0.0;
        for (int a = 0; a < nen; a++) {
          double Ua = Uc[gidx[a]];
          u += Ua * N[a];
          for (int i = 0; i < dim; i++) gu[i] += Ua * dN[a * dim + i];
          if (P->log_kappa) lk += P->log_kappa[gidx[a]] * N[a];
        }
        double kappa = P->log_kappa ? exp(lk) : 1.0;
        double re = P->lambda * exp(u);
        double f = P->source ? manufactured_f(dim, P->lambda, x) : 0.0;
        for (int a = 0; a < nen; a++) {
          double gg = 0.0;
          for (int i = 0; i < dim; i++) gg += dN[a * dim + i] * gu[i];
          /* Eq. (residual): (grad N_A, kappa grad u) - (N_A, lambda e^u) [- (N_A, f)] */
          Fe[a] += jw * (kappa * gg - re * N[a] - f * N[a]);
          if (Ke && !fd)
            for (int b = 0; b < nen; b++) {
              double gab = 0.0;
              for (int i = 0; i < dim; i++) gab += dN[a * dim + i] * dN[b * dim + i];
              /* Eq. (jacobian): (grad N_A, kappa grad N_B) - (N_A, lambda e^u N_B) */
              Ke[a * nen + b] += jw * (kappa * gab - re * N[a] * N[b]);
            }
        }
        if (Ke && fd) {
          /* Eq. (fdjac), column by column */
          double Ue[OR_MAXEN], Up[OR_MAXEN], F0[OR_MAXEN], F1[OR_MAXEN], nrm = 0.0;
          for (int a = 0; a < nen; a++) {
            Ue[a] = Uc[gidx[a]];
            nrm += Ue[a] * Ue[a];
          }
          const double delta = sqrt(DBL_EPSILON) * sqrt(1.0 + sqrt(nrm));
          point_integrand(dim, nen, N, dN, Ue, kappa, P->lambda, jw, F0);
          for (int b = 0; b < nen; b++) {
            for (int a = 0; a < nen; a++) Up[a] = Ue[a];
            Up[b] += delta;
            point_integrand(dim, nen, N, dN, Up, kappa, P->lambda, jw, F1);
            for (int a = 0; a < nen; a++) Ke[a * nen + b] += (F1[a] - F0[a]) / delta;
          }
        }
      }
  return nen;
}

/* Dirichlet data: returns 1 and the value g if dof (natural index A) lies on a
 * face with a boundary value; faces are visited axis 0 side 0, axis 0 side 1,
 * axis 1 side 0, ..., and a later face overrides an earlier one. */
static int dirichlet(const or_problem *P, int64_t A, double *g) {
  int hit = 0;
  int64_t t = A;
  for (int d = 0; d < P->dim; d++) {
    int n = nfun(P, d);
    int i = (int)(t % n);
    t /= n;
    if (P->bnd[d][0] && i == 0) { hit = 1; *g = P->bval[d][0]; }
    if (P->bnd[d][1] && i == n - 1) { hit = 1; *g = P->bval[d][1]; }
  }
  return hit;
}

int or_is_dirichlet(const or_problem *P, int64_t A) {
  double g;
  return dirichlet(P, A, &g);
}

/* Full residual F (length N), Algorithm 3 with Dirichlet rows F_A = U_A - g. */
int or_residual(const or_problem *P, const double *Uc, double *F) {
  or_mesh Msh;
  int rc = mesh_init(P, &Msh);
  if (rc) return rc;
  int64_t N = num_dofs(P);
  for (int64_t A = 0; A < N; A++) F[A] = 0.0;
  static int64_t gidx[OR_MAXEN];
  static double Fe[OR_MAXEN];
  for (int e2 = 0; e2 < Msh.ne[2]; e2++)
    for (int e1 = 0; e1 < Msh.ne[1]; e1++)
      for (int e0 = 0; e0 < Msh.ne[0]; e0++) {
        int e[3] = {e0, e1, e2};
        int nen = element_integrals(&Msh, e, Uc, gidx, Fe, NULL);
        if (nen < 0) { mesh_free(&Msh); return nen; }
        for (int a = 0; a < nen; a++) F[gidx[a]] += Fe[a]; /* F_e -> F */
      }
  for (int64_t A = 0; A < N; A++) {
    double g;
    if (dirichlet(P, A, &g)) F[A] = Uc[A] - g;
  }
  mesh_free(&Msh);
  return 0;
}

static int64_t find_col(const int64_t *rowptr, const int32_t *colidx, int64_t A, int64_t B) {
  int64_t lo = rowptr[A], hi = rowptr[A + 1] - 1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) / 2;
    if (colidx[mid] == B) return mid;
    if (colidx[mid] < B) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

static void dirichlet_fix_row(const or_problem *P, int64_t A, const int64_t *rowptr,
                              const int32_t *colidx, double *vals_row) {
  double g;
  int rowfix = dirichlet(P, A, &g);
  for (int64_t k = rowptr[A]; k < rowptr[A + 1]; k++) {
    int64_t B = colidx[k];
    if (rowfix) vals_row[k - rowptr[A]] = (A == B) ? 1.0 : 0.0;
    else if (dirichlet(P, B, &g)) vals_row[k - rowptr[A]] = 0.0;
  }
}

/* Full Jacobian into CSR values on the given pattern; an element entry that
 * falls outside the pattern is an error (-20). */
int or_jacobian(const or_problem *P, const double *Uc, const int64_t *rowptr,
                const int32_t *colidx, double *vals) {
  or_mesh Msh;
  int rc = mesh_init(P, &Msh);
  if (rc) return rc;
  int64_t N = num_dofs(P);
  for (int64_t k = 0; k < rowptr[N]; k++) vals[k] = 0.0;
  static int64_t gidx[OR_MAXEN];
  static double Fe[OR_MAXEN];
  double *Ke = (double *)malloc(sizeof(double) * OR_MAXEN * OR_MAXEN);
  for (int e2 = 0; e2 < Msh.ne[2]; e2++)
    for (int e1 = 0; e1 < Msh.ne[1]; e1++)
      for (int e0 = 0; e0 < Msh.ne[0]; e0++) {
        int e[3] = {e0, e1, e2};
        int nen = element_integrals(&Msh, e, Uc, gidx, Fe, Ke);
        if (nen < 0) { free(Ke); mesh_free(&Msh); return nen; }
        for (int a = 0; a < nen; a++)
          for (int b = 0; b < nen; b++) {
            int64_t k = find_col(rowptr, colidx, gidx[a], gidx[b]);
            if (k < 0) { free(Ke); mesh_free(&Msh); return -20; }
            vals[k] += Ke[a * nen + b];
          }
      }
  for (int64_t A = 0; A < N; A++) dirichlet_fix_row(P, A, rowptr, colidx, vals + rowptr[A]);
  free(Ke);
  mesh_free(&Msh);
  return 0;
}

/* Jacobian by local numerical differentiation (Sec. 2.8, Eq. fdjac) into CSR values
 * on the given pattern, Dirichlet rows and columns as in or_jacobian. */
int or_jacobian_fd(const or_problem *P, const double *Uc, const int64_t *rowptr,
                   const int32_t *colidx, double *vals) {
  or_mesh Msh;
  int rc = mesh_init(P, &Msh);
  if (rc) return rc;
  int64_t N = num_dofs(P);
  for (int64_t k = 0; k < rowptr[N]; k++) vals[k] = 0.0;
  static int64_t gidx[OR_MAXEN];
  static double Fe[OR_MAXEN];
  double *Ke = (double *)malloc(sizeof(double) * OR_MAXEN * OR_MAXEN);
  for (int e2 = 0; e2 < Msh.ne[2]; e2++)
    for (int e1 = 0; e1 < Msh.ne[1]; e1++)
      for (int e0 = 0; e0 < Msh.ne[0]; e0++) {
        int e[3] = {e0, e1, e2};
        int nen = element_integrals_mode(&Msh, e, Uc, gidx, Fe, Ke, 1);
        if (nen < 0) { free(Ke); mesh_free(&Msh); return nen; }
        for (int a = 0; a < nen; a++)
          for (int b = 0; b < nen; b++) {
            int64_t k = find_col(rowptr, colidx, gidx[a], gidx[b]);
            if (k < 0) { free(Ke); mesh_free(&Msh); return -20; }
            vals[k] += Ke[a * nen + b];
          }
      }
  for (int64_t A = 0; A < N; A++) dirichlet_fix_row(P, A, rowptr, colidx, vals + rowptr[A]);
  free(Ke);
  mesh_free(&Msh);
  return 0;
}

/* Number of OpenMP threads the colour-loop timing mode uses (1 without OpenMP). */
int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Element count of colour c (span indices c, c + stride, ...) along one direction. */
static int colour_count(int ne, int c, int stride) { return (c < ne) ? (ne - 1 - c) / stride + 1 : 0; }

/* or_residual with the colour-by-colour element loop of the timing mode (see the file
 * header); the same element integrals, Dirichlet rows and result up to the order of the
 * additions.  Not for periodic directions (-30). */
int or_residual_colored(const or_problem *P, const double *Uc, double *F) {
  if (P->wrap[0] || P->wrap[1] || P->wrap[2]) return -30;
  or_mesh Msh;
  int rc = mesh_init(P, &Msh);
  if (rc) return rc;
  int64_t N = num_dofs(P);
  for (int64_t A = 0; A < N; A++) F[A] = 0.0;
  int st[3] = {1, 1, 1};
  for (int d = 0; d < P->dim; d++) st[d] = P->p[d] + 1;
  int bad = 0;
  for (int c2 = 0; c2 < st[2]; c2++)
    for (int c1 = 0; c1 < st[1]; c1++)
      for (int c0 = 0; c0 < st[0]; c0++) {
        const int k0 = colour_count(Msh.ne[0], c0, st[0]), k1 = colour_count(Msh.ne[1], c1, st[1]);
        const int64_t total = (int64_t)k0 * k1 * colour_count(Msh.ne[2], c2, st[2]);
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t t = 0; t < total; t++) {
          int64_t gidx[OR_MAXEN];
          double Fe[OR_MAXEN];
          int e[3] = {c0 + (int)(t % k0) * st[0], c1 + (int)((t / k0) % k1) * st[1], c2 + (int)(t / ((int64_t)k0 * k1)) * st[2]};
          int nen = element_integrals(&Msh, e, Uc, gidx, Fe, NULL);
          if (nen < 0) {
#pragma omp atomic write
            bad = nen;
            continue;
          }
          for (int a = 0; a < nen; a++) F[gidx[a]] += Fe[a];
        }
      }
  if (bad) { mesh_free(&Msh); return bad; }
  for (int64_t A = 0; A < N; A++) {
    double g;
    if (dirichlet(P, A, &g)) F[A] = Uc[A] - g;
  }
  mesh_free(&Msh);
  return 0;
}

/* or_jacobian with the colour-by-colour element loop of the timing mode. */
int or_jacobian_colored(const or_problem *P, const double *Uc, const int64_t *rowptr, const int32_t *colidx,
                        double *vals) {
  if (P->wrap[0] || P->wrap[1] || P->wrap[2]) return -30;
  or_mesh Msh;
  int rc = mesh_init(P, &Msh);
  if (rc) return rc;
  int64_t N = num_dofs(P);
  for (int64_t k = 0; k < rowptr[N]; k++) vals[k] = 0.0;
  int st[3] = {1, 1, 1};
  for (int d = 0; d < P->dim; d++) st[d] = P->p[d] + 1;
  int bad = 0;
#pragma omp parallel
  {
    int64_t gidx[OR_MAXEN];
    double Fe[OR_MAXEN];
    double *Ke = (double *)malloc(sizeof(double) * OR_MAXEN * OR_MAXEN);
    for (int c2 = 0; c2 < st[2]; c2++)
      for (int c1 = 0; c1 < st[1]; c1++)
        for (int c0 = 0; c0 < st[0]; c0++) {
          const int k0 = colour_count(Msh.ne[0], c0, st[0]), k1 = colour_count(Msh.ne[1], c1, st[1]);
          const int64_t total = (int64_t)k0 * k1 * colour_count(Msh.ne[2], c2, st[2]);
#pragma omp for schedule(dynamic, 1)
          for (int64_t t = 0; t < total; t++) {
            int e[3] = {c0 + (int)(t % k0) * st[0], c1 + (int)((t / k0) % k1) * st[1], c2 + (int)(t / ((int64_t)k0 * k1)) * st[2]};
            int nen = Ke ? element_integrals(&Msh, e, Uc, gidx, Fe, Ke) : -2;
            if (nen < 0) {
#pragma omp atomic write
              bad = nen;
              continue;
            }
            for (int a = 0; a < nen; a++)
              for (int b = 0; b < nen; b++) {
                int64_t k = find_col(rowptr, colidx, gidx[a], gidx[b]);
                if (k < 0) {
#pragma omp atomic write
                  bad = -20;
                  continue;
                }
                vals[k] += Ke[a * nen + b];
              }
          }
        }
    free(Ke);
  }
  if (bad) { mesh_free(&Msh); return bad; }
  for (int64_t A = 0; A < N; A++) dirichlet_fix_row(P, A, rowptr, colidx, vals + rowptr[A]);
  mesh_free(&Msh);
  return 0;
}

/* Mass matrix M_AB = sum_e sum_q J_q w_q N_A N_B (Sec. 4.2: the derivative of the
 * residual's u-dot term (N_A, u-dot^h) in U-dot_B) into CSR values on the given
 * pattern, with no Dirichlet fix; same element loop and quadrature as or_jacobian. */
int or_mass(const or_problem *P, const int64_t *rowptr, const int32_t *colidx, double *vals) {
  or_mesh Msh;
  int rc = mesh_init(P, &Msh);
  if (rc) return rc;
  const int dim = P->dim;
  int64_t N = num_dofs(P);
  for (int64_t k = 0; k < rowptr[N]; k++) vals[k] = 0.0;
  static int64_t gidx[OR_MAXEN];
  static double Nq[OR_MAXEN], dN[OR_MAXEN * 3];
  int nen = 1;
  for (int d = 0; d < dim; d++) nen *= P->p[d] + 1;
  for (int e2 = 0; e2 < Msh.ne[2]; e2++)
    for (int e1 = 0; e1 < Msh.ne[1]; e1++)
      for (int e0 = 0; e0 < Msh.ne[0]; e0++) {
        int e[3] = {e0, e1, e2}, s[3] = {0, 0, 0}, q[3] = {1, 1, 1};
        for (int d = 0; d < dim; d++) {
          s[d] = Msh.sp[d][e[d]];
          q[d] = P->q[d];
        }
        for (int g2 = 0; g2 < q[2]; g2++)
          for (int g1 = 0; g1 < q[1]; g1++)
            for (int g0 = 0; g0 < q[0]; g0++) {
              int g[3] = {g0, g1, g2};
              double xi[3] = {0, 0, 0}, wq = 1.0;
              for (int d = 0; d < dim; d++) {
                double lo = P->U[d][s[d]], hi = P->U[d][s[d] + 1];
                xi[d] = 0.5 * (lo + hi) + 0.5 * (hi - lo) * Msh.gx[d][g[d]];
                wq *= Msh.gw[d][g[d]] * 0.5 * (hi - lo);
              }
              double x[3], detJ;
              rc = or_shape(P, s, xi, gidx, Nq, dN, x, &detJ);
              if (rc < 0) { mesh_free(&Msh); return rc; }
              for (int a = 0; a < nen; a++)
                for (int b = 0; b < nen; b++) {
                  int64_t k = find_col(rowptr, colidx, gidx[a], gidx[b]);
                  if (k < 0) { mesh_free(&Msh); return -20; }
                  vals[k] += detJ * wq * Nq[a] * Nq[b];
                }
            }
      }
  mesh_free(&Msh);
  return 0;
}

/* Elements whose support contains natural node A: span s with s-p <= i <= s
 * (non-periodic directions only). */
static int elements_of_node(const or_mesh *Msh, int64_t A, int lo[3], int hi[3]) {
  const or_problem *P = Msh->P;
  int64_t t = A;
  for (int d = 0; d < 3; d++) { lo[d] = 0; hi[d] = 0; }
  for (int d = 0; d < P->dim; d++) {
    int n = nfun(P, d);
    int i = (int)(t % n);
    t /= n;
    lo[d] = Msh->ne[d];
    hi[d] = -1;
    for (int e = 0; e < Msh->ne[d]; e++) {
      int s = Msh->sp[d][e];
      if (s - P->p[d] <= i && i <= s) {
        if (e < lo[d]) lo[d] = e;
        if (e > hi[d]) hi[d] = e;
      }
    }
    if (hi[d] < lo[d]) return 0;
  }
  return 1;
}

/* Residual entries of selected rows only (same definition as or_residual). */
int or_residual_rows(const or_problem *P, const double *Uc, int64_t nr, const int64_t *rows,
                     double *out) {
  if (P->wrap[0] || P->wrap[1] || P->wrap[2]) return -30;
  or_mesh Msh;
  int rc = mesh_init(P, &Msh);
  if (rc) return rc;
  static int64_t gidx[OR_MAXEN];
  static double Fe[OR_MAXEN];
  for (int64_t r = 0; r < nr; r++) {
    int64_t A = rows[r];
    double acc = 0.0;
    int lo[3], hi[3];
    if (elements_of_node(&Msh, A, lo, hi))
      for (int e2 = lo[2]; e2 <= hi[2]; e2++)
        for (int e1 = lo[1]; e1 <= hi[1]; e1++)
          for (int e0 = lo[0]; e0 <= hi[0]; e0++) {
            int e[3] = {e0, e1, e2};
            int nen = element_integrals(&Msh, e, Uc, gidx, Fe, NULL);
            if (nen < 0) { mesh_free(&Msh); return nen; }
            for (int a = 0; a < nen; a++)
              if (gidx[a] == A) acc += Fe[a];
          }
    double g;
    if (dirichlet(P, A, &g)) acc = Uc[A] - g;
    out[r] = acc;
  }
  mesh_free(&Msh);
  return 0;
}

/* Jacobian values of selected rows (concatenated in the order of `rows`, each
 * row laid out as its pattern row rowptr[A]..rowptr[A+1]). */
int or_jacobian_rows(const or_problem *P, const double *Uc, int64_t nr, const int64_t *rows,
                     const int64_t *rowptr, const int32_t *colidx, double *out) {
  if (P->wrap[0] || P->wrap[1] || P->wrap[2]) return -30;
  or_mesh Msh;
  int rc = mesh_init(P, &Msh);
  if (rc) return rc;
  static int64_t gidx[OR_MAXEN];
  static double Fe[OR_MAXEN];
  double *Ke = (double *)malloc(sizeof(double) * OR_MAXEN * OR_MAXEN);
  int64_t off = 0;
  for (int64_t r = 0; r < nr; r++) {
    int64_t A = rows[r];
    int64_t len = rowptr[A + 1] - rowptr[A];
    double *row = out + off;
    for (int64_t k = 0; k < len; k++) row[k] = 0.0;
    int lo[3], hi[3];
    if (elements_of_node(&Msh, A, lo, hi))
      for (int e2 = lo[2]; e2 <= hi[2]; e2++)
        for (int e1 = lo[1]; e1 <= hi[1]; e1++)
          for (int e0 = lo[0]; e0 <= hi[0]; e0++) {
            int e[3] = {e0, e1, e2};
            int nen = element_integrals(&Msh, e, Uc, gidx, Fe, Ke);
            if (nen < 0) { free(Ke); mesh_free(&Msh); return nen; }
            for (int a = 0; a < nen; a++) {
              if (gidx[a] != A) continue;
              for (int b = 0; b < nen; b++) {
                int64_t k = find_col(rowptr, colidx, A, gidx[b]);
                if (k < 0) { free(Ke); mesh_free(&Msh); return -20; }
                row[k - rowptr[A]] += Ke[a * nen + b];
              }
            }
          }
    dirichlet_fix_row(P, A, rowptr, colidx, row);
    off += len;
  }
  free(Ke);
  mesh_free(&Msh);
  return 0;
}

/* Brute force on small meshes: at every quadrature point of every element,
 * evaluate ALL N global basis functions by the recursion (no element-local
 * indexing), form the rational basis and geometry over all control points, and
 * integrate the residual and Jacobian densely (J is N x N, row-major).  The
 * Dirichlet fix is applied when `fix` is nonzero. */
int or_dense_bruteforce(const or_problem *P, const double *Uc, double *F, double *J, int fix) {
  or_mesh Msh;
  int rc = mesh_init(P, &Msh);
  if (rc) return rc;
  int dim = P->dim;
  int n[3] = {1, 1, 1};
  for (int d = 0; d < dim; d++) n[d] = nfun(P, d);
  int64_t N = num_dofs(P);
  double *M = (double *)malloc(sizeof(double) * N);
  double *dM = (double *)malloc(sizeof(double) * N * 3);
  double *Nr = (double *)malloc(sizeof(double) * N);
  double *dNp = (double *)malloc(sizeof(double) * N * 3);
  double *dNx = (double *)malloc(sizeof(double) * N * 3);
  double *b[3], *db[3];
  for (int d = 0; d < 3; d++) {
    b[d] = (double *)malloc(sizeof(double) * (n[d] + 1));
    db[d] = (double *)malloc(sizeof(double) * (n[d] + 1));
  }
  for (int64_t A = 0; A < N; A++) F[A] = 0.0;
  for (int64_t k = 0; k < N * N; k++) J[k] = 0.0;
  for (int e2 = 0; e2 < Msh.ne[2]; e2++)
    for (int e1 = 0; e1 < Msh.ne[1]; e1++)
      for (int e0 = 0; e0 < Msh.ne[0]; e0++) {
        int e[3] = {e0, e1, e2}, s[3] = {0, 0, 0}, q[3] = {1, 1, 1};
        for (int d = 0; d < dim; d++) { s[d] = Msh.sp[d][e[d]]; q[d] = P->q[d]; }
        for (int g2 = 0; g2 < q[2]; g2++)
          for (int g1 = 0; g1 < q[1]; g1++)
            for (int g0 = 0; g0 < q[0]; g0++) {
              int g[3] = {g0, g1, g2};
              double xi[3] = {0, 0, 0}, wq = 1.0;
              for (int d = 0; d < dim; d++) {
                double lo = P->U[d][s[d]], hi = P->U[d][s[d] + 1];
                xi[d] = 0.5 * (lo + hi) + 0.5 * (hi - lo) * Msh.gx[d][g[d]];
                wq *= Msh.gw[d][g[d]] * 0.5 * (hi - lo);
              }
              for (int d = 0; d < 3; d++)
                for (int i = 0; i < n[d]; i++) {
                  if (d < dim) {
                    /* a periodic function is the sum of the unclamped B-splines whose
                       index wraps onto it (Eq. map-wrap) */
                    b[d][i] = db[d][i] = 0.0;
                    for (int iu = i; iu < P->m[d] - P->p[d] - 1; iu += n[d]) {
                      b[d][i] += or_bspline(iu, P->p[d], P->U[d], xi[d]);
                      db[d][i] += or_bspline_der(iu, P->p[d], P->U[d], xi[d]);
                      if (!P->wrap[d]) break;
                    }
                  } else {
                    b[d][i] = 1.0;
                    db[d][i] = 0.0;
                  }
                }
              double W = 0.0, Wd[3] = {0, 0, 0};
              for (int64_t A = 0; A < N; A++) {
                int64_t t = A;
                int ix[3] = {0, 0, 0};
                for (int d = 0; d < dim; d++) { ix[d] = (int)(t % n[d]); t /= n[d]; }
                M[A] = b[0][ix[0]] * b[1][ix[1]] * b[2][ix[2]];
                dM[A * 3 + 0] = db[0][ix[0]] * b[1][ix[1]] * b[2][ix[2]];
                dM[A * 3 + 1] = b[0][ix[0]] * db[1][ix[1]] * b[2][ix[2]];
                dM[A * 3 + 2] = b[0][ix[0]] * b[1][ix[1]] * db[2][ix[2]];
                double w = P->weights ? P->weights[A] : 1.0;
                W += w * M[A];
                for (int al = 0; al < dim; al++) Wd[al] += w * dM[A * 3 + al];
              }
              for (int64_t A = 0; A < N; A++) {
                double w = P->weights ? P->weights[A] : 1.0;
                Nr[A] = w * M[A] / W;
                for (int al = 0; al < dim; al++) dNp[A * 3 + al] = (w * dM[A * 3 + al] - Nr[A] * Wd[al]) / W;
              }
              double Fm[3][3], x[3];
              for (int i = 0; i < dim; i++) {
                if (P->ctrl) {
                  x[i] = 0.0;
                  for (int al = 0; al < dim; al++) Fm[i][al] = 0.0;
                  for (int64_t A = 0; A < N; A++) {
                    x[i] += P->ctrl[A * dim + i] * Nr[A];
                    for (int al = 0; al < dim; al++) Fm[i][al] += P->ctrl[A * dim + i] * dNp[A * 3 + al];
                  }
                } else {
                  x[i] = xi[i];
                  for (int al = 0; al < dim; al++) Fm[i][al] = (i == al) ? 1.0 : 0.0;
                }
              }
              /* inverse and determinant by cofactors (a second, independent route) */
              double inv[3][3], det;
              if (dim == 1) {
                det = Fm[0][0];
                inv[0][0] = 1.0 / det;
              } else if (dim == 2) {
                det = Fm[0][0] * Fm[1][1] - Fm[0][1] * Fm[1][0];
                inv[0][0] = Fm[1][1] / det;
                inv[0][1] = -Fm[0][1] / det;
                inv[1][0] = -Fm[1][0] / det;
                inv[1][1] = Fm[0][0] / det;
              } else {
                double c00 = Fm[1][1] * Fm[2][2] - Fm[1][2] * Fm[2][1];
                double c01 = Fm[1][2] * Fm[2][0] - Fm[1][0] * Fm[2][2];
                double c02 = Fm[1][0] * Fm[2][1] - Fm[1][1] * Fm[2][0];
                det = Fm[0][0] * c00 + Fm[0][1] * c01 + Fm[0][2] * c02;
                inv[0][0] = c00 / det;
                inv[1][0] = c01 / det;
                inv[2][0] = c02 / det;
                inv[0][1] = (Fm[0][2] * Fm[2][1] - Fm[0][1] * Fm[2][2]) / det;
                inv[1][1] = (Fm[0][0] * Fm[2][2] - Fm[0][2] * Fm[2][0]) / det;
                inv[2][1] = (Fm[0][1] * Fm[2][0] - Fm[0][0] * Fm[2][1]) / det;
                inv[0][2] = (Fm[0][1] * Fm[1][2] - Fm[0][2] * Fm[1][1]) / det;
                inv[1][2] = (Fm[0][2] * Fm[1][0] - Fm[0][0] * Fm[1][2]) / det;
                inv[2][2] = (Fm[0][0] * Fm[1][1] - Fm[0][1] * Fm[1][0]) / det;
              }
              /* inv[alpha][i] = xi_{alpha,i} */
              double u = 0.0, gu[3] = {0, 0, 0}, lk = 0.0;
              for (int64_t A = 0; A < N; A++) {
                for (int i = 0; i < dim; i++) {
                  double gi = 0.0;
                  for (int al = 0; al < dim; al++) gi += dNp[A * 3 + al] * inv[al][i];
                  dNx[A * 3 + i] = gi;
                }
                u += Uc[A] * Nr[A];
                for (int i = 0; i < dim; i++) gu[i] += Uc[A] * dNx[A * 3 + i];
                if (P->log_kappa) lk += P->log_kappa[A] * Nr[A];
              }
              double kappa = P->log_kappa ? exp(lk) : 1.0;
              double jw = det * wq, re = P->lambda * exp(u);
              double f = P->source ? manufactured_f(dim, P->lambda, x) : 0.0;
              for (int64_t A = 0; A < N; A++) {
                if (Nr[A] == 0.0 && dNx[A * 3] == 0.0 && (dim < 2 || dNx[A * 3 + 1] == 0.0) &&
                    (dim < 3 || dNx[A * 3 + 2] == 0.0))
                  continue;
                double gg = 0.0;
                for (int i = 0; i < dim; i++) gg += dNx[A * 3 + i] * gu[i];
                F[A] += jw * (kappa * gg - re * Nr[A] - f * Nr[A]);
                for (int64_t B = 0; B < N; B++) {
                  double gab = 0.0;
                  for (int i = 0; i < dim; i++) gab += dNx[A * 3 + i] * dNx[B * 3 + i];
                  J[A * N + B] += jw * (kappa * gab - re * Nr[A] * Nr[B]);
                }
              }
            }
      }
  if (fix)
    for (int64_t A = 0; A < N; A++) {
      double g;
      if (dirichlet(P, A, &g)) {
        F[A] = Uc[A] - g;
        for (int64_t B = 0; B < N; B++) {
          J[A * N + B] = (A == B) ? 1.0 : 0.0;
          if (B != A) J[B * N + A] = 0.0;
        }
      }
    }
  free(M); free(dM); free(Nr); free(dNp); free(dNx);
  for (int d = 0; d < 3; d++) { free(b[d]); free(db[d]); }
  mesh_free(&Msh);
  return 0;
}

/* Squared L2 error of u^h against the manufactured u* over the mapped domain,
 * by the same Gauss rule. */
double or_l2_error_sq(const or_problem *P, const double *Uc) {
  or_mesh Msh;
  if (mesh_init(P, &Msh)) return -1.0;
  int dim = P->dim;
  static int64_t gidx[OR_MAXEN];
  static double N[OR_MAXEN], dN[OR_MAXEN * 3];
  double err = 0.0;
  for (int e2 = 0; e2 < Msh.ne[2]; e2++)
    for (int e1 = 0; e1 < Msh.ne[1]; e1++)
      for (int e0 = 0; e0 < Msh.ne[0]; e0++) {
        int e[3] = {e0, e1, e2}, s[3] = {0, 0, 0}, q[3] = {1, 1, 1};
        for (int d = 0; d < dim; d++) { s[d] = Msh.sp[d][e[d]]; q[d] = P->q[d]; }
        for (int g2 = 0; g2 < q[2]; g2++)
          for (int g1 = 0; g1 < q[1]; g1++)
            for (int g0 = 0; g0 < q[0]; g0++) {
              int g[3] = {g0, g1, g2};
              double xi[3] = {0, 0, 0}, wq = 1.0;
              for (int d = 0; d < dim; d++) {
                double lo = P->U[d][s[d]], hi = P->U[d][s[d] + 1];
                xi[d] = 0.5 * (lo + hi) + 0.5 * (hi - lo) * Msh.gx[d][g[d]];
                wq *= Msh.gw[d][g[d]] * 0.5 * (hi - lo);
              }
              double x[3], detJ;
              int nen = or_shape(P, s, xi, gidx, N, dN, x, &detJ);
              double u = 0.0;
              for (int a = 0; a < nen; a++) u += Uc[gidx[a]] * N[a];
              double d = u - manufactured_u(dim, x);
              err += detJ * wq * d * d;
            }
      }
  mesh_free(&Msh);
  return err;
}

/* Map a parametric point (any point of the closed domain) to physical space with
 * the rational geometry; at the right end of a direction the last non-empty span
 * is used (the half-open convention of Eq. (1) would give zero there). */
int or_map_point(const or_problem *P, const double *xi, double *x, double *detJ) {
  int s[3] = {0, 0, 0};
  for (int d = 0; d < P->dim; d++) {
    int n = nfun(P, d);
    int sd = -1;
    for (int k = P->p[d]; k < n; k++)
      if (P->U[d][k] <= xi[d] && xi[d] < P->U[d][k + 1]) sd = k;
    if (sd < 0) {
      for (int k = n - 1; k >= P->p[d]; k--)
        if (P->U[d][k] < P->U[d][k + 1]) { sd = k; break; }
    }
    s[d] = sd;
  }
  /* evaluate strictly inside the chosen span when at its right end */
  double xx[3];
  for (int d = 0; d < 3; d++) xx[d] = (d < P->dim) ? xi[d] : 0.0;
  for (int d = 0; d < P->dim; d++)
    if (xx[d] >= P->U[d][s[d] + 1]) xx[d] = nextafter(P->U[d][s[d] + 1], -1e300);
  static int64_t gidx[OR_MAXEN];
  static double N[OR_MAXEN], dN[OR_MAXEN * 3];
  return or_shape(P, s, xx, gidx, N, dN, x, detJ) < 0 ? -1 : 0;
}
