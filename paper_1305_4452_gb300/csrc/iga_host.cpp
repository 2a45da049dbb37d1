// Host set-up of libiga: knot vectors, Gauss-Legendre rules, 1D basis tables,
// BasisStencil ranges, 1D pair tables and the CSR row pointers.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>

#include "iga_internal.h"

std::string iga_format(const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return std::string(buf);
}

GeomLayout geom_layout(int dim) {
  GeomLayout g;
  int ns = dim * (dim + 1) / 2;
  g.invW = 0;
  g.g = 1;
  g.S = g.g + dim;
  g.jwW = g.S + ns;
  g.Sg = g.jwW + 1;
  g.gSg = g.Sg + dim;
  g.jwW2 = g.gSg + 1;
  g.nf = g.jwW2 + 1;
  return g;
}

// Gauss-Legendre rule on [-1,1] (the tensor Gauss-Legendre quadrature of Sec. 2.9):
// roots of P_q by Newton's method, P_q and P_q' from the Bonnet recurrence.
static void gauss_rule(int q, double *x, double *w) {
  for (int k = 0; k < q; k++) {
    double t = cos(M_PI * (4.0 * k + 3.0) / (4.0 * q + 2.0));  // k-th root from the right
    double p1 = 0.0, dp = 1.0;
    for (int it = 0; it < 64; it++) {
      double pm = 1.0, pc = t;
      for (int j = 1; j < q; j++) {
        double pn = ((2 * j + 1) * t * pc - j * pm) / (j + 1);
        pm = pc;
        pc = pn;
      }
      if (q == 0) pc = 1.0;
      p1 = pc;
      dp = q * (t * pc - pm) / (t * t - 1.0);
      double step = p1 / dp;
      t -= step;
      if (fabs(step) <= 1e-17) break;
    }
    double pm = 1.0, pc = t;
    for (int j = 1; j < q; j++) {
      double pn = ((2 * j + 1) * t * pc - j * pm) / (j + 1);
      pm = pc;
      pc = pn;
    }
    dp = q * (t * pc - pm) / (t * t - 1.0);
    x[q - 1 - k] = t;
    w[q - 1 - k] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

// Values and xi-derivatives of the p+1 B-splines that are nonzero on span s
// (functions s-p .. s), by Eq. (2) evaluated over the nonzero functions only --
// the triangular scheme of Piegl and Tiller, referred to in Sec. 2.1 -- and the
// first-derivative identity obtained by differentiating Eq. (2).
static void span_basis(const std::vector<double> &U, int p, int s, double xi, double *B, double *dB) {
  double tri[IGA_MAXN][IGA_MAXN];  // tri[k][a]: degree-k function s-k+a
  tri[0][0] = 1.0;
  for (int k = 1; k <= p; k++) {
    for (int a = 0; a <= k; a++) {
      int i = s - k + a;
      double v = 0.0;
      if (a >= 1) {
        double den = U[i + k] - U[i];
        if (den != 0.0) v += (xi - U[i]) / den * tri[k - 1][a - 1];
      }
      if (a <= k - 1) {
        double den = U[i + k + 1] - U[i + 1];
        if (den != 0.0) v += (U[i + k + 1] - xi) / den * tri[k - 1][a];
      }
      tri[k][a] = v;
    }
  }
  for (int a = 0; a <= p; a++) {
    B[a] = tri[p][a];
    if (p == 0) {
      dB[a] = 0.0;
      continue;
    }
    int i = s - p + a;
    double t = 0.0;
    if (a >= 1) {
      double den = U[i + p] - U[i];
      if (den != 0.0) t += tri[p - 1][a - 1] / den;
    }
    if (a <= p - 1) {
      double den = U[i + p + 1] - U[i + 1];
      if (den != 0.0) t -= tri[p - 1][a] / den;
    }
    dB[a] = p * t;
  }
}

// BasisStencil (Sec. 2.5, Algorithm 2): indices of the left-most and right-most
// basis functions whose support overlaps that of function i.
static void basis_stencil(const std::vector<double> &U, int p, int i, int *l, int *r) {
  int j = i;
  while (U[j] == U[j + 1]) j++;
  *l = j - p;
  j = i + p + 1;
  while (U[j] == U[j - 1]) j--;
  *r = j - 1;
}

// The knot vector of direction ax: explicit, or uniform open on [0, 1] with nel
// elements and interior knots repeated p-k times (continuity C^k).
iga_status iga_open_knots(iga_s *h, const iga_desc *d, int ax, std::vector<double> &U) {
  const int p = d->degree[ax];
  if (d->knots[ax]) {
    int m = d->nknots[ax];
    if (m < 2 * p + 2) {
      h->err = iga_format("axis %d: %d knots is too few for degree %d", ax, m, p);
      return IGA_EINVAL;
    }
    U.assign(d->knots[ax], d->knots[ax] + m);
  } else {
    int nel = d->nel[ax], k = d->continuity[ax];
    if (k < 0) k = p - 1;
    if (nel < 1 || nel > (1 << 20) || k > p - 1) {
      h->err = iga_format("axis %d: bad nel=%d or continuity=%d", ax, nel, k);
      return IGA_EINVAL;
    }
    U.assign(p + 1, 0.0);
    for (int e = 1; e < nel; e++)
      for (int r = 0; r < p - k; r++) U.push_back((double)e / (double)nel);
    for (int r = 0; r <= p; r++) U.push_back(1.0);
  }
  return IGA_OK;
}

// Sec. 2.4, Eqs. (unclamp-left)-(unclamp-right): with m the last knot index and
// n = m - p - 1, the k+1 knots at each end are redefined from the other end,
//   U[k-i] = U[p] - U[n+1] + U[n-i],  U[m-k+i] = U[n+1] - U[p] + U[p+i+1],  0 <= i <= k.
// The two sides read only knots neither side writes when n - k >= k + 1.
iga_status iga_unclamp(iga_s *h, int ax, int p, int k, std::vector<double> &U) {
  const int m = (int)U.size() - 1, n = m - p - 1;
  if (k < 0 || k > p - 1 || n - k < k + 1) {
    h->err = iga_format("axis %d: cannot unclamp for C^%d periodicity (degree %d, %d functions)", ax, k, p, n + 1);
    return IGA_EINVAL;
  }
  for (int k2 = 1; k2 <= p; k2++)
    if (U[k2] != U[0] || U[m - k2] != U[m]) {
      h->err = iga_format("axis %d: a periodic direction starts from an open knot vector", ax);
      return IGA_EINVAL;
    }
  const double lo = U[p], hi = U[n + 1];
  for (int i = 0; i <= k; i++) U[k - i] = lo - hi + U[n - i];
  for (int i = 0; i <= k; i++) U[m - k + i] = hi - lo + U[p + i + 1];
  return IGA_OK;
}

static iga_status build_dir(iga_s *h, const iga_desc *d, int ax, Dir &D) {
  int p = d->degree[ax];
  D.p = p;
  D.q = p + 1;
  iga_status kst = iga_open_knots(h, d, ax, D.knots);
  if (kst != IGA_OK) return kst;
  const std::vector<double> &U = D.knots;
  int m = (int)U.size();
  for (int k = 0; k + 1 < m; k++)
    if (!(U[k] <= U[k + 1]) || !std::isfinite(U[k + 1])) {
      h->err = iga_format("axis %d: knots must be finite and non-decreasing", ax);
      return IGA_EINVAL;
    }
  for (int k = 1; k <= p && !h->unclamped; k++)
    if (U[k] != U[0] || U[m - 1 - k] != U[m - 1]) {
      h->err = iga_format("axis %d: knot vector must be open (p+1 repeated end knots)", ax);
      return IGA_EINVAL;
    }
  D.n = m - p - 1;
  // interior multiplicity <= p keeps every basis C^0 or smoother
  for (int k = p + 1; k < D.n; k++) {
    int mult = 1;
    while (k + mult < m - p - 1 && U[k + mult] == U[k]) mult++;
    if (mult > p) {
      h->err = iga_format("axis %d: interior knot multiplicity %d exceeds degree", ax, mult);
      return IGA_EINVAL;
    }
  }
  // elements = non-empty spans
  std::vector<int> spans;
  for (int s = p; s < D.n; s++)
    if (U[s] < U[s + 1]) spans.push_back(s);
  D.nel = (int)spans.size();
  if (D.nel < 1) {
    h->err = iga_format("axis %d: no non-empty knot span", ax);
    return IGA_EINVAL;
  }
  int q = D.q, n1 = p + 1;
  double gx[IGA_MAXQ], gw[IGA_MAXQ];
  gauss_rule(q, gx, gw);
  D.first.resize(D.nel);
  D.tab.assign((size_t)D.nel * q * n1 * 2, 0.0);
  D.wq.assign((size_t)D.nel * q, 0.0);
  for (int e = 0; e < D.nel; e++) {
    int s = spans[e];
    D.first[e] = s - p;
    double lo = U[s], hi = U[s + 1], half = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
    for (int g = 0; g < q; g++) {
      double B[IGA_MAXN], dB[IGA_MAXN];
      span_basis(U, p, s, mid + half * gx[g], B, dB);
      for (int a = 0; a < n1; a++) {
        D.tab[(((size_t)e * q + g) * n1 + a) * 2 + 0] = B[a];
        D.tab[(((size_t)e * q + g) * n1 + a) * 2 + 1] = dB[a];
      }
      D.wq[(size_t)e * q + g] = gw[g] * half;
    }
  }
  // elements containing each function (a contiguous range)
  D.node_e0.assign(D.n, -1);
  D.node_ne.assign(D.n, 0);
  for (int e = 0; e < D.nel; e++)
    for (int a = 0; a < n1; a++) {
      int i = D.first[e] + a;
      if (D.node_e0[i] < 0) D.node_e0[i] = e;
      D.node_ne[i]++;
    }
  for (int i = 0; i < D.n; i++)
    if (D.node_ne[i] == 0) {
      h->err = iga_format("axis %d: function %d has no element", ax, i);
      return IGA_EINVAL;
    }
  // BasisStencil ranges and the 1D pair tables
  D.l.resize(D.n);
  D.r.resize(D.n);
  D.pair_off.assign(D.n + 1, 0);
  D.pair_i.clear();
  D.pair_j.clear();
  D.pair_x0.clear();
  D.pair_np.clear();
  D.pair_po.clear();
  D.pair_val.clear();
  for (int i = 0; i < D.n; i++) {
    if (h->unclamped) {
      // the unwrapped space of a periodic direction: supports reach past the domain,
      // so the range is that of the functions sharing one of i's elements (equal to
      // BasisStencil's on an open knot vector)
      const int ea = D.node_e0[i], eb = D.node_e0[i] + D.node_ne[i] - 1;
      D.l[i] = D.first[ea];
      D.r[i] = D.first[eb] + p;
    } else {
      basis_stencil(U, p, i, &D.l[i], &D.r[i]);
    }
    D.pair_off[i] = (int)D.pair_j.size();
    for (int j = D.l[i]; j <= D.r[i]; j++) {
      int e0 = std::max(D.node_e0[i], D.node_e0[j]);
      int e1 = std::min(D.node_e0[i] + D.node_ne[i], D.node_e0[j] + D.node_ne[j]);
      if (e1 <= e0) {
        h->err = iga_format("axis %d: stencil pair (%d,%d) has no common element", ax, i, j);
        return IGA_EINVAL;
      }
      D.pair_i.push_back(i);
      D.pair_j.push_back(j);
      D.pair_x0.push_back(e0 * q);
      D.pair_np.push_back((e1 - e0) * q);
      D.pair_po.push_back((int)(D.pair_val.size() / IGA_PVS));
      for (int e = e0; e < e1; e++)
        for (int g = 0; g < q; g++) {
          const double *ti = &D.tab[(((size_t)e * q + g) * n1 + (i - D.first[e])) * 2];
          const double *tj = &D.tab[(((size_t)e * q + g) * n1 + (j - D.first[e])) * 2];
          D.pair_val.push_back(ti[0] * tj[0]);
          D.pair_val.push_back(ti[1] * tj[0]);
          D.pair_val.push_back(ti[0] * tj[1]);
          D.pair_val.push_back(ti[1] * tj[1]);
          D.pair_val.push_back(ti[1] * tj[0] + ti[0] * tj[1]);
        }
    }
  }
  D.pair_off[D.n] = (int)D.pair_j.size();
  // index of the transposed pair (j, i); the stencil relation is symmetric
  D.pair_T.resize(D.pair_j.size());
  for (size_t k = 0; k < D.pair_j.size(); k++) {
    int i = D.pair_i[k], j = D.pair_j[k];
    if (i < D.l[j] || i > D.r[j]) {
      h->err = iga_format("axis %d: stencil of %d does not contain %d", ax, j, i);
      return IGA_EINVAL;
    }
    D.pair_T[k] = D.pair_off[j] + (i - D.l[j]);
  }
  // canonical pairs in pair order, and ordered by overlap length (longest first) so
  // that the threads of a warp in the pair loops of the Jacobian run the same number
  // of Gauss points
  D.pair_c.clear();
  for (size_t k = 0; k < D.pair_j.size(); k++)
    if ((int)k <= D.pair_T[k]) D.pair_c.push_back((int)k);
  D.pair_cs = D.pair_c;
  std::stable_sort(D.pair_cs.begin(), D.pair_cs.end(), [&](int a, int b) { return D.pair_np[a] > D.pair_np[b]; });
  return IGA_OK;
}

iga_status iga_build_dirs(iga_s *h, const iga_desc *d) {
  if (d->dim < 2 || d->dim > 3) {
    h->err = iga_format("dim must be 2 or 3 (got %d)", d->dim);
    return IGA_EINVAL;
  }
  int p = d->degree[0];
  for (int ax = 0; ax < d->dim; ax++) {
    if (d->degree[ax] != p || p < 1 || p > IGA_MAXP) {
      h->err = iga_format("degrees must be equal in every direction and in 1..%d", IGA_MAXP);
      return IGA_EINVAL;
    }
    if (d->quad[ax] != 0 && d->quad[ax] != p + 1) {
      h->err = iga_format("only the (p+1)-point Gauss rule is supported (axis %d asked %d)", ax, d->quad[ax]);
      return IGA_EINVAL;
    }
  }
  h->dim = d->dim;
  h->p = p;
  h->q = p + 1;
  h->N = 1;
  h->nelem = 1;
  for (int ax = 0; ax < 3; ax++) {
    if (ax < d->dim) {
      iga_status st = build_dir(h, d, ax, h->dir[ax]);
      if (st != IGA_OK) return st;
    } else {
      Dir &D = h->dir[ax];  // a trivial direction so 2D code can index 3 directions
      D = Dir();
      D.n = 1;
      D.nel = 1;
      D.q = 1;
    }
    h->N *= h->dir[ax].n;
    h->nelem *= h->dir[ax].nel;
  }
  if (h->N > (int64_t)(INT32_MAX / 8)) {  // int32 columns and thread indices (8 lanes per row)
    h->err = "more than 2^28 control variables";
    return IGA_EINVAL;
  }
  int nq = 1;
  for (int ax = 0; ax < d->dim; ax++) nq *= h->q;
  h->nqp = h->nelem * nq;
  return IGA_OK;
}

// Row pointers of the CSR pattern: row A = (i0,i1,i2) holds the lexicographic
// product of the BasisStencil ranges (Sec. 2.5), so its length is the product
// of the 1D range lengths.
void iga_rowptr(const iga_s *h, std::vector<int64_t> &rowptr) {
  const Dir &D0 = h->dir[0], &D1 = h->dir[1], &D2 = h->dir[2];
  rowptr.resize(h->N + 1);
  int64_t acc = 0, A = 0;
  for (int i2 = 0; i2 < D2.n; i2++) {
    int64_t w2 = (h->dim == 3) ? (D2.r[i2] - D2.l[i2] + 1) : 1;
    for (int i1 = 0; i1 < D1.n; i1++) {
      int64_t w1 = D1.r[i1] - D1.l[i1] + 1;
      for (int i0 = 0; i0 < D0.n; i0++) {
        rowptr[A++] = acc;
        acc += w2 * w1 * (D0.r[i0] - D0.l[i0] + 1);
      }
    }
  }
  rowptr[A] = acc;
}
