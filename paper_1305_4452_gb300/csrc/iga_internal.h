// Internal state and kernel interfaces of libiga (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/iga.h"

#define IGA_MAXP 4                 // largest supported degree
#define IGA_MAXN (IGA_MAXP + 1)    // largest number of nonzero 1D functions per element
#define IGA_MAXQ (IGA_MAXP + 1)    // largest Gauss rule (q = p + 1)
#define IGA_PVS 5                  // values per Gauss point in the 1D pair tables

// Number of per-quadrature-point geometry fields (see GeomField) for each dimension.
#define IGA_NGF2 11
#define IGA_NGF3 16

// Geometry factor record, one set per quadrature point, element-major layout
// G[e][field][qp].  With W = sum w_A M_A, g = grad_xi W / W, C = Xi Xi^T
// (Xi = inverse of dx/dxi), jw = det(dx/dxi) * (Gauss weight) * prod(span/2):
//   invW            1 / W
//   g[a]            grad_xi W / W
//   S[ab]           kappa * jw * C / W^2   (symmetric; 2D: 00,11,01; 3D: 00,11,22,01,02,12)
//   jwW             jw / W
//   nSg[a]          -(S g)_a
//   gSg             g^T S g
//   jwW2            jw / W^2
// These turn the rational-basis integrands into polynomial-basis contractions:
//   F_A = w_A sum_q [ grad M_A . v + M_A s ],  v = S (grad ũ - ũ g),  s = -g.v - jwW lambda e^u
//   J_AB = w_A w_B sum_q sum_{mu,nu} Q_{mu nu} D_mu M_A D_nu M_B, with
//   Q_00 = gSg - jwW2 lambda e^u, Q_0a = nSg_a, Q_ab = S_ab
// where ũ = sum (w_A U_A) M_A and u = ũ / W.
struct GeomLayout {
  int nf;      // number of fields
  int invW, g, S, jwW, Sg, gSg, jwW2;  // field offsets
};

GeomLayout geom_layout(int dim);
struct iga_s;
cudaError_t classify_stiffness_plan(iga_s *h);

// FP32 copy of the geometry factors for the reduced-precision Jacobians (iga_s::geom32,
// [e][slot][qp]): invW, gSg, jwW2, S (ns), nSg (dim)
template <int DIM> struct G32 {
  static constexpr int NS = DIM * (DIM + 1) / 2;
  static constexpr int INVW = 0, GSG = 1, JWW2 = 2, S = 3, NSG = 3 + NS, NF = 3 + NS + DIM;
};

struct Dir {
  int p = 0, q = 0, nel = 0, n = 0;
  std::vector<double> knots;
  std::vector<int> first;      // [nel] first nonzero function of each element (span - p)
  std::vector<double> tab;     // [nel][q][p+1][2]: B, dB/dxi at the Gauss points
  std::vector<double> wq;      // [nel][q]: Gauss weight * span/2
  std::vector<int> l, r;       // [n] BasisStencil range
  std::vector<int> pair_off;   // [n+1] first pair of each function
  std::vector<int> pair_j;     // [P] second function of each pair
  std::vector<int> pair_i;     // [P] first function of each pair
  std::vector<int> pair_x0;    // [P] first Gauss point (global index) of the overlap
  std::vector<int> pair_np;    // [P] number of Gauss points in the overlap
  std::vector<int> pair_po;    // [P] offset into pair_val (in points)
  std::vector<double> pair_val;// [sum np][5]: B_i B_j, B'_i B_j, B_i B'_j, B'_i B'_j, B'_i B_j + B_i B'_j
  std::vector<int> pair_T;     // [P] index of the transposed pair (j, i)
  std::vector<int> pair_c;     // canonical pairs (pair index <= that of its transpose), ascending
  std::vector<int> pair_cs;    // the same, longest overlap first
  std::vector<int> node_e0;    // [n] first element containing the function
  std::vector<int> node_ne;    // [n] number of elements containing it
  int npairs() const { return (int)pair_j.size(); }
  int X() const { return nel * q; }
};

// Device copies of the per-direction data.
struct DirDev {
  int p, q, nel, n, np, X;
  int *first;
  double *tab;
  double *wq;
  int *l, *r;
  int *pair_off, *pair_i, *pair_j, *pair_x0, *pair_np, *pair_po, *pair_T;
  int nc, *pair_c, *pair_cs;
  double *pair_val;
  float *pair_val_f;  // FP32 copy for the mixed-precision stages
  int *node_e0, *node_ne;
};

struct DirArgs {  // passed by value to kernels
  int p, q, nel, n, np, X;
  const int *first;
  const double *tab;
  const double *wq;
  const int *l, *r;
  const int *pair_off, *pair_i, *pair_j, *pair_x0, *pair_np, *pair_po, *pair_T;
  int nc;
  const int *pair_c, *pair_cs;
  const double *pair_val;
  const float *pair_val_f;
  const int *node_e0, *node_ne;
};

struct BndArgs {
  int flag[3][2];
  double val[3][2];
};

// Periodic directions (Sec. 2.4).  A periodic handle assembles on the unclamped
// space of its inner handle (every unwrapped function kept, no index wrap, no
// Dirichlet rows) and maps between the two numberings: U is prolonged to the
// unwrapped functions, residual rows and Jacobian entries of the unwrapped
// functions whose indices wrap (Eq. map-wrap) onto the same function are summed.
// Per direction, for the outer (wrapped) functions i in [0, n) and the inner
// (unwrapped) functions i' in [0, nu):
struct PerAxisHost {
  int n = 1, nu = 1;
  std::vector<int> wrap;              // [nu] outer index of i'
  std::vector<int> img_off, img;      // images of i: img[img_off[i] .. img_off[i+1])
  std::vector<int> col_off, col;      // sorted wrapped columns of row i: col[col_off[i] .. col_off[i+1])
  std::vector<int> con_off, con_row, con_pos;  // per column slot: unwrapped (i', position in row i') pairs
  std::vector<int> ulen;              // [nu] length of the unwrapped row i'
};
struct PerAxis {  // device copy, passed by value
  int n, nu;
  const int *wrap, *img_off, *img, *col_off, *col, *con_off, *con_row, *con_pos, *ulen;
};
struct PerArgs {
  PerAxis ax[3];
};

// Kernel classes for launch counting and event timing (iga_profile_*).
enum KClass {
  KC_GEOM = 0, KC_RES_ELEM, KC_RES_GATHER, KC_Q00, KC_STAGE1, KC_STAGE2, KC_FINAL, KC_SPMV, KC_ORTH,
  KC_GMRES_SCALAR, KC_VEC, KC_COMBINE, KC_PATTERN, KC_ELEM_TC, KC_ELEM_GATHER, KC_RES_SPMV, KC_N
};

struct ProfRec {
  int cls;
  cudaEvent_t a, b;
};

struct Prof {
  unsigned mask = 0;             // classes timed with events
  long long launches[KC_N] = {}; // every launch is counted
  double ms[KC_N] = {};
  long long timed[KC_N] = {};
  std::vector<ProfRec> pending;
  std::vector<cudaEvent_t> pool;
};

struct iga_s;
struct ElemGemmPlan;
int prof_begin(iga_s *h, int cls);
void prof_end(iga_s *h, int token);
#define IGA_LAUNCH(h, cls, ...)          \
  do {                                   \
    int tok_ = prof_begin((h), (cls));   \
    __VA_ARGS__;                         \
    prof_end((h), tok_);                 \
  } while (0)

struct iga_s {
  Prof prof;
  int dim = 0, p = 0, q = 0;
  int64_t N = 0, nnz = 0, nelem = 0, nqp = 0;
  Dir dir[3];
  DirDev ddev[3];
  cudaStream_t stream = nullptr;
  int device = -1;             // CUDA device current at iga_create
  double *noalloc_scratch = nullptr;  // device address of the allocation-free residual's array
  double lambda = 0.0;
  bool has_geom = false, has_w = false, has_kappa = false;
  // stiffness plan of a mapped or rational geometry (classify_stiffness_plan): S diagonal at
  // every Gauss point (an orthogonal parametrisation, such as the annulus), and which
  // weight-gradient terms (S g)_a are nonzero (bit a)
  bool plan_diag_s = false;
  bool plan_general = false;   // iga_set_jacobian_plan(h, 1): every term, whatever the classification
  int plan_gmask = 7;
  // rational weights that factor by axis, w_A = w0[i0] w1[i1] w2[i2]: the products w_A w_B of
  // the Jacobian are folded into the device pair tables (w_d[i] w_d[j] per pair) and the
  // final stage multiplies by nothing
  bool w_folded = false;
  std::vector<double> wsep[3];
  BndArgs bnd{};
  GeomLayout gl{};
  std::string err;

  // device buffers owned by the library
  int64_t *rowptr = nullptr;
  // rowptr of a tensor-product pattern: row (i0, line) starts at
  // rp_line[line] + (stencil width of the line) * rp_p0[i0], line = i1 + n1 i2 (2D: i1)
  int64_t *rp_line = nullptr;
  int *rp_p0 = nullptr;
  int32_t *colidx = nullptr;
  double *weights = nullptr;   // [N] or null
  double *geom = nullptr;      // [nelem][nf][nq]
  double *Fe = nullptr;        // [nelem][nen] element residuals
  double *Q00 = nullptr;       // [nelem][nq]
  void *T1 = nullptr;          // stage-1 intermediate
  void *T2 = nullptr;          // stage-2 intermediate (3D)
  size_t T1_bytes = 0, T2_bytes = 0;
  double *Kstiff = nullptr;    // U-independent part of J (Newton reuse), nnz doubles
  float *Kstiff_f = nullptr;   // FP32 copy for mixed Newton
  double *Mred = nullptr;      // reaction-only contraction on the CSR layout
  float *Mred_f = nullptr;
  bool K_valid = false, K_valid_f = false;  // Kstiff / Kstiff_f hold the current stiffness
  bool q00_valid = false;      // Q00 holds the reaction part of Q00 at the current Newton iterate
  // time-dependent residual (Sec. 4.2): while ts_on, every residual adds (N_A, v^h) with
  // v = ts_a U + ts_C per control variable, and every Jacobian adds ts_a times the mass matrix
  bool ts_on = false;
  double ts_a = 0.0;
  const double *ts_C = nullptr;
  double *ts_buf = nullptr;    // generalized-alpha workspace: C and U_n (2 N doubles)
  // periodic handles (Sec. 2.4): the unwrapped discretisation and the maps to it
  bool unclamped = false;      // inner handle: knots need not be open; stencils from elements
  iga_s *inner = nullptr;      // set on a periodic handle
  PerAxisHost per_host[3];
  PerArgs per{};
  std::vector<void *> per_bufs;  // device copies of the per-axis tables
  double *Uu = nullptr, *Fu = nullptr, *Cu = nullptr, *Ju = nullptr;  // unwrapped U, F, rate data, Jacobian
  float *Ju32 = nullptr;
  double *Uhost_dev = nullptr; // device copy of U for the host-buffer solve
  // mixed-precision Jacobian (tensor cores)
  float *geom32 = nullptr;     // [nelem][slots][nq] FP32 geometry factors
  float *tab32[3] = {nullptr, nullptr, nullptr};  // FP32 basis tables
  float *Ebuf = nullptr;       // [nelem][nen][nen] element matrices
  double *Ebuf64 = nullptr;    // [nelem][nen][nen] FP64 element matrices (local numerical differentiation)
  float *z32 = nullptr;        // FP32 copy of the Krylov vector for the FP32 SpMV
  ElemGemmPlan *egemm = nullptr;  // element matrices as one GEMM across elements (iga_elem_gemm.cu)
  uint64_t wait_limit_ns = 2000000000ull;  // bound of each pipeline wait of the tensor-core kernels
  bool gs_unfused = false;     // GMRES orthogonalisation by the separate pass kernels only
  bool stall_next = false;     // failure-detection test: the next element GEMM waits on a barrier nothing completes
  // Newton / Krylov workspace
  double *J64 = nullptr;
  float *J32 = nullptr;
  float *J32s = nullptr;       // sliced copy of J32 for the FP32 operator products (launch_slice32)
  bool J32s_valid = false;     // J32s holds the values now in J32
  double *wk = nullptr;        // vectors: F, dU, Utrial, Ftrial, diag, z, w, ...
  double *V = nullptr;         // GMRES basis (m+1) x N
  int V_m = 0;
  double *red = nullptr;       // reduction partials
  double *ctl = nullptr;       // GMRES scalar control block (device)
  double *ctl_host = nullptr;  // pinned mirror
  unsigned *gsbar = nullptr;   // grid barrier of the fused orthogonalisation (count, generation)
  int nblk_red = 0;
};

// ---- host set-up (iga_host.cpp) ----
iga_status iga_build_dirs(iga_s *h, const iga_desc *d);
// The open knot vector of direction ax as iga_create builds it (explicit or uniform)
iga_status iga_open_knots(iga_s *h, const iga_desc *d, int ax, std::vector<double> &U);
// Eqs. (unclamp-left)-(unclamp-right): unclamp an open knot vector for C^k periodicity
iga_status iga_unclamp(iga_s *h, int ax, int p, int k, std::vector<double> &U);
void iga_rowptr(const iga_s *h, std::vector<int64_t> &rowptr);

// ---- element kernels (iga_element.cu) ----
DirArgs dir_args(const DirDev &d);
cudaError_t launch_geometry(iga_s *h, const double *ctrl_dev, const double *logk_dev);
cudaError_t launch_colidx(iga_s *h);
cudaError_t launch_residual(iga_s *h, const double *U, double *F);
// The residual kernels with the element-vector buffer Fe supplied by the caller
// (launch_residual passes the handle's own; non-periodic handles only)
cudaError_t launch_residual_into(iga_s *h, const double *U, double *F, double *Fe);
// ---- allocation-free residual (iga_noalloc.cu) ----
// Looks up, on the current device, the address of the fixed scratch array of
// iga_form_residual_noalloc and keeps it in h->noalloc_scratch (left null on failure)
void noalloc_setup(iga_s *h);
// Q00 = cs * g^T S g - cr * jw/W^2 * lambda * exp(u) at every Gauss point (U may be null when cr == 0)
cudaError_t launch_q00(iga_s *h, const double *U, double cs, double cr);
// the same Q00 computed in FP32 arithmetic (stored as double), for the FP32 Jacobian
cudaError_t launch_q00_f32(iga_s *h, const double *U, double cs, double cr);
// Matrix-free Jacobian: y = J(U) x and diag(J(U)), with h->Q00 holding the reaction
// part of Q00 at U (launch_q00(h, U, 0, 1)); done may be null
cudaError_t launch_jv(iga_s *h, const double *x, double *y, const double *done);
cudaError_t launch_jacobian_diagonal(iga_s *h, double *diag);
// F(U) = K U + reaction(U) with Dirichlet rows, K the assembled stiffness without
// the Dirichlet fix (Jacobian mode 1); KU: scratch of N doubles.  Also leaves the
// reaction part of Q00 at U in h->Q00 (see iga_s::q00_valid).
cudaError_t launch_residual_split(iga_s *h, const double *U, double *F, const double *K, double *KU);

// ---- periodic handles (iga_periodic.cu) ----
iga_status iga_periodic_setup(iga_s *h, const iga_desc *d, const iga_bratu *b);
cudaError_t periodic_residual(iga_s *h, const double *U, double *F);
cudaError_t periodic_jacobian64(iga_s *h, const double *U, double *vals);
cudaError_t periodic_jacobian32(iga_s *h, const double *U, float *vals);
// y = J x on the wrapped CSR pattern (FP64 or FP32 values, FP64 x, y and sums); done may be null
cudaError_t periodic_spmv(iga_s *h, const void *vals, int is_f32, const double *x, double *y, const double *done);
cudaError_t periodic_diag_inv(iga_s *h, const void *vals, int is_f32, double *dinv);
void periodic_release(iga_s *h);
// Creation and release of an ordinary (non-periodic or inner) handle (iga_api.cu)
iga_status iga_create_impl(iga_s *h, const iga_desc *d, const iga_bratu *b);
void iga_release(iga_s *h);

// ---- Jacobian stages (iga_jacobian.cu) ----
// mode 0: full Jacobian; 1: stiffness only (U-independent), without the Dirichlet
// fix; 2: vals = base + reaction(U) with the Dirichlet fix (base from mode 1);
// 3: full Jacobian without the Dirichlet fix
cudaError_t launch_jacobian64(iga_s *h, const double *U, double *vals, int mode, const double *base);
cudaError_t launch_jacobian32(iga_s *h, const double *U, float *vals, int mode, const float *base);
// y = x rounded to FP32 (nnz-sized value arrays)
cudaError_t launch_round_f32(iga_s *h, const double *x, float *y, int64_t n);
size_t jacobian_t1_groups(int dim);
// ---- mixed-precision Jacobian (iga_mixed.cu) ----
bool mixed_supported(int dim, int p);
cudaError_t launch_jacobian_mixed(iga_s *h, const double *U, float *vals, int prec);
// Element matrices as one tcgen05 GEMM across elements of equal 1D tables (iga_elem_gemm.cu):
// available when the knot vectors repeat their spans (uniform meshes); frees in elem_gemm_release
bool elem_gemm_supported(iga_s *h, int prec);
cudaError_t launch_jacobian_elem_gemm(iga_s *h, const double *U, float *vals, int prec);
bool elem_gemm_failed(iga_s *h);
void elem_gemm_release(iga_s *h);
// Degrees and dimensions with a tensor-core Jacobian on this handle
bool tc_jacobian_supported(iga_s *h, int prec);
// Jacobian by local numerical differentiation (Sec. 2.8 Eq. fdjac), FP64 values
cudaError_t launch_jacobian_fd(iga_s *h, const double *U, double *vals);
size_t jacobian_t2_groups(int dim);

// ---- Krylov (iga_krylov.cu) ----
// Row partition of the Gram-Schmidt passes: nb blocks of per rows (the last may be shorter)
struct GsPartition {
  int nb, per;
};
GsPartition gs_partition(int64_t N);
cudaError_t launch_spmv64(iga_s *h, const double *vals, const double *x, double *y);
// the same product, counted and timed as the split residual's stiffness product
cudaError_t launch_spmv64_residual(iga_s *h, const double *vals, const double *x, double *y);
// y = J x for a Dirichlet-fixed Jacobian (rows e_A, zero columns skipped)
cudaError_t launch_spmv64_fixed(iga_s *h, const double *vals, const double *x, double *y);
cudaError_t launch_spmv32(iga_s *h, const float *vals, const double *x, double *y);
// sliced copy of h->J32 (rows in slices of 32, slot-major) for the FP32 Krylov products
cudaError_t launch_slice32(iga_s *h);
cudaError_t launch_diag_inv(iga_s *h, const void *vals, int is_f32, double *dinv);
cudaError_t launch_norm2(iga_s *h, const double *x, double *out_dev);
cudaError_t launch_nan_check(iga_s *h, const double *x, double *out_dev);
int cg_solve(iga_s *h, const void *vals, int is_f32, const double *b, double *x, double tol_abs, int maxit, int *its,
             cudaError_t *cerr);
int gmres_solve(iga_s *h, const void *vals, int is_f32, const double *b, double *x, double rtol_abs,
                int m, int maxit, int refine, int *its, cudaError_t *cerr);

std::string iga_format(const char *fmt, ...);
