/*
 * Plain FP64 CPU oracle of the ILUT-smoothed p-multigrid method for Galerkin
 * IgA discretisations of Poisson's equation (Tielen, Moeller, Goeddeke, Vuik,
 * "A p-multigrid method enhanced with an ILUT smoother ...", arXiv 1901.01685).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the
 * library in paper_1901_01685_gb300/.  Only tests/, __graft_entry__.smoke()
 * and the cpu_baseline / reference legs of bench.py may load it.  It shares no
 * code, header, table or helper with the library, and never calls it.
 *
 * Style: every routine follows the paper's definitions literally, single
 * threaded, in FP64, with no blocking, fusion or reordering beyond what the
 * definitions state.  Citations name the paper's section / equation / table.
 *
 * Readings of passages the paper leaves open:
 *   R1  Open uniform knots with span h = 2^-k, p+1 repeated end knots (Sec. 2).
 *   R2  DOF numbering: lexicographic, first parametric direction fastest,
 *       0-based (the index formula printed in Sec. 2 is garbled).
 *   R3  Quadrature: q+1 Gauss points per direction per element for operators
 *       of degree q; max(q, q')+1 for the mixed transfer matrix P_{q'}^{q}.
 *   R4  Quarter annulus map F(xi, eta) = ((1+xi) cos(pi eta/2),
 *       (1+xi) sin(pi eta/2)): xi radial, eta angular.
 *   R5  Dirichlet data: the exact solution sin(pi x) sin(pi y) is non-zero only
 *       on the annulus arcs; there the boundary coefficients are the 1-D L2
 *       projection (parametric measure, end values = exact corner values = 0).
 *       Everywhere else the data vanish and boundary coefficients are 0.
 *       Boundary DOFs are eliminated, f_I <- f_I - A_IB u_B (Sec. 5 setup).
 *   R6  Row-sum lumping uses the full row (boundary columns included),
 *       M^L_ii = sum_j M_ij, then is restricted to interior DOFs (Sec. 3).
 *   R7  ILUT relative drop tolerance tau_i = tau * (sum_j |a_ij|) / nnz(a_i)
 *       over the original row, applied to the multipliers and to the final row.
 *   R8  ILUT row budget M = ceil(m * nnz(A) / N), kept separately in the strict
 *       lower (L) and strict upper (U) parts; the diagonal is always kept.
 *   R9  ILUT selection of the M largest magnitudes: let t be the M-th largest
 *       magnitude; entries above t(1+1e-12) are kept, the remaining places go
 *       to the entries inside [t(1-1e-12), t(1+1e-12)] in ascending column
 *       order.  Exact zeros are never stored.
 *   R10 ILUT in natural (lexicographic) order, no fill-reducing permutation.
 *   R11 Indirect projection p -> p-1 -> ... -> 1 is the default; direct p -> 1
 *       is the alternative (Sec. 3, App. A).  ILUT smoothing on every level
 *       q >= 2.
 *   R12 Coarse solve at p = 1: `coarse_cycles` (default 2, Sec. 3) h-multigrid
 *       V-cycles from a zero guess; levels h, 2h, ... down to h = 2^-3 where a
 *       direct solve is done (Fig. 1); one forward lexicographic Gauss-Seidel
 *       pre-sweep and one backward post-sweep; canonical (bi/tri)linear
 *       interpolation P_c; restriction P_c^T; rediscretised operators.
 *   R13 Residual norm: Euclidean norm of the interior residual, relres =
 *       ||r_k|| / ||r_0||, checked after each V-cycle; divergence if > 1e10.
 *   R14 Benchmark 2 (Sec. 2 gives the strong form): a_ij = int (D grad phi_j)
 *       . grad phi_i + (v . grad phi_j) phi_i + R phi_j phi_i, phi_i the test
 *       function (row); the P1 levels rediscretise the same equation.
 *
 * Parity status: every routine has a pin in tests/ except that the V-cycle as
 * a whole is pinned only softly (iteration counts of Table 4 within +-2,
 * spectral radii of Table 2a in magnitude) plus exact invariants (fixed point,
 * linearity, exact-LU smoother converges in one cycle).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

enum { OR_ANNULUS = 0, OR_SQUARE = 1, OR_CUBE = 2, OR_CDR_SQUARE = 3 };

/* Benchmark 2 (Sec. 2): -div(D grad u) + v . grad u + R u = f on the unit
 * square with these coefficients; the other benchmarks have D = I, v = 0, R = 0. */
static const double CDR_D[2][2] = {{1.2, -0.7}, {-0.4, 0.9}};
static const double CDR_V[2] = {0.4, -0.2};
static const double CDR_R = 0.3;
enum { OR_U_SINPROD = 0, OR_U_PAPER_B1 = 1 };
enum { OR_INDIRECT = 0, OR_DIRECT = 1 };
enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_OOM = 2, OR_ERR_ZERO_PIVOT = 3,
       OR_ERR_DIVERGED = 4, OR_ERR_MAXITER = 5 };

/* ------------------------------------------------------------------------- */
/* B-spline basis, Sec. 2 (Cox-de Boor recursion, open uniform knot vector)   */
/* ------------------------------------------------------------------------- */

/* knot idx (0-based) of the open uniform vector of degree p over ne elements:
 * p+1 zeros, interior knots e/ne, p+1 ones (reading R1). */
static double knot(int p, int ne, int idx) {
  if (idx <= p) return 0.0;
  if (idx >= ne + p) return 1.0;
  return (double)(idx - p) / (double)ne;
}

/* N_{i,deg}(x) on the degree-p knot vector, by the Cox-de Boor recursion with
 * 0/0 := 0.  The last non-empty span is closed at x = 1. */
static double bspl(int p, int ne, int i, int deg, double x) {
  if (deg == 0) {
    double a = knot(p, ne, i), b = knot(p, ne, i + 1);
    if (a < b && ((x >= a && x < b) || (x == 1.0 && b == 1.0))) return 1.0;
    return 0.0;
  }
  double a = knot(p, ne, i), b = knot(p, ne, i + deg);
  double c = knot(p, ne, i + 1), d = knot(p, ne, i + deg + 1);
  double s = 0.0;
  if (b > a) s += (x - a) / (b - a) * bspl(p, ne, i, deg - 1, x);
  if (d > c) s += (d - x) / (d - c) * bspl(p, ne, i + 1, deg - 1, x);
  return s;
}

/* d/dx N_{i,deg}(x): deg/(t_{i+deg}-t_i) N_{i,deg-1} - deg/(t_{i+deg+1}-t_{i+1}) N_{i+1,deg-1}. */
static double bspl_d(int p, int ne, int i, int deg, double x) {
  if (deg == 0) return 0.0;
  double a = knot(p, ne, i), b = knot(p, ne, i + deg);
  double c = knot(p, ne, i + 1), d = knot(p, ne, i + deg + 1);
  double s = 0.0;
  if (b > a) s += deg / (b - a) * bspl(p, ne, i, deg - 1, x);
  if (d > c) s -= deg / (d - c) * bspl(p, ne, i + 1, deg - 1, x);
  return s;
}

double or_bspline(int p, int ne, int i, double x, int deriv) {
  if (p < 0 || ne < 1 || i < 0 || i >= ne + p) return NAN;
  return deriv ? bspl_d(p, ne, i, p, x) : bspl(p, ne, i, p, x);
}

/* ------------------------------------------------------------------------- */
/* Gauss-Legendre rule on [0,1] (Newton iteration on the Legendre polynomial) */
/* ------------------------------------------------------------------------- */
void or_gauss(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(OR_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1; p1 = p2;
      }
      if (n == 1) { p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1; p1 = p2;
      }
      if (n == 1) p0 = 1.0;
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    /* z_i decreases with i: store ascending on [0,1] */
    x[n - 1 - i] = 0.5 * (1.0 + z);
    w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* ------------------------------------------------------------------------- */
/* Geometry map F (Sec. 2; benchmark 1 = quarter annulus, benchmark 4 = cube) */
/* ------------------------------------------------------------------------- */
static void geo(int dom, int d, const double* xi, double* X, double J[3][3], double* det) {
  memset(J, 0, 9 * sizeof(double));
  if (dom == OR_ANNULUS) {
    double r = 1.0 + xi[0], th = 0.5 * OR_PI * xi[1];
    X[0] = r * cos(th); X[1] = r * sin(th);
    J[0][0] = cos(th); J[0][1] = -r * 0.5 * OR_PI * sin(th);
    J[1][0] = sin(th); J[1][1] = r * 0.5 * OR_PI * cos(th);
    *det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  } else {
    for (int a = 0; a < d; ++a) { X[a] = xi[a]; J[a][a] = 1.0; }
    *det = 1.0;
  }
}

/* exact solution u and source f = -Lap(u) (Sec. 2 benchmarks; reading R5). */
static double u_exact(int dom, int ex, int d, const double* X) {
  if (ex == OR_U_PAPER_B1 && dom == OR_ANNULUS) {
    double x = X[0], y = X[1], s = x * x + y * y;
    return -(s - 1.0) * (s - 4.0) * x * y * y;
  }
  double u = 1.0;
  for (int a = 0; a < d; ++a) u *= sin(OR_PI * X[a]);
  return u;
}
static double f_source(int dom, int ex, int d, const double* X) {
  if (ex == OR_U_PAPER_B1 && dom == OR_ANNULUS) {
    double x = X[0], y = X[1];
    return 2.0 * x * (x * x * x * x + 22.0 * x * x * y * y - 5.0 * x * x + 21.0 * y * y * y * y - 45.0 * y * y + 4.0);
  }
  if (dom == OR_CDR_SQUARE) {
    /* f = -sum_ab D_ab d_a d_b u + v . grad u + R u for u = sin(pi x) sin(pi y) */
    double sx = sin(OR_PI * X[0]), sy = sin(OR_PI * X[1]), cx = cos(OR_PI * X[0]), cy = cos(OR_PI * X[1]);
    double uxx = -OR_PI * OR_PI * sx * sy, uyy = uxx, uxy = OR_PI * OR_PI * cx * cy;
    double ux = OR_PI * cx * sy, uy = OR_PI * sx * cy;
    return -(CDR_D[0][0] * uxx + CDR_D[0][1] * uxy + CDR_D[1][0] * uxy + CDR_D[1][1] * uyy) +
           CDR_V[0] * ux + CDR_V[1] * uy + CDR_R * sx * sy;
  }
  double u = 1.0;
  for (int a = 0; a < d; ++a) u *= sin(OR_PI * X[a]);
  return d * OR_PI * OR_PI * u;
}
double or_u_exact(int dom, int ex, double x, double y, double z) {
  double X[3] = {x, y, z}; return u_exact(dom, ex, dom == OR_CUBE ? 3 : 2, X);
}
double or_f_source(int dom, int ex, double x, double y, double z) {
  double X[3] = {x, y, z}; return f_source(dom, ex, dom == OR_CUBE ? 3 : 2, X);
}

/* ------------------------------------------------------------------------- */
/* Sparse storage (CSR) and small helpers                                     */
/* ------------------------------------------------------------------------- */
typedef struct { int nr, nc, nnz; int* rp; int* ci; double* v; } csr;

static void csr_free(csr* a) { free(a->rp); free(a->ci); free(a->v); memset(a, 0, sizeof(*a)); }

static void spmv(const csr* a, const double* x, double* y) {
  for (int i = 0; i < a->nr; ++i) {
    double s = 0.0;
    for (int t = a->rp[i]; t < a->rp[i + 1]; ++t) s += a->v[t] * x[a->ci[t]];
    y[i] = s;
  }
}

static int csr_transpose(const csr* a, csr* t) {
  t->nr = a->nc; t->nc = a->nr; t->nnz = a->nnz;
  t->rp = calloc((size_t)t->nr + 1, sizeof(int));
  t->ci = malloc(sizeof(int) * (size_t)(a->nnz ? a->nnz : 1));
  t->v = malloc(sizeof(double) * (size_t)(a->nnz ? a->nnz : 1));
  if (!t->rp || !t->ci || !t->v) return OR_ERR_OOM;
  for (int k = 0; k < a->nnz; ++k) t->rp[a->ci[k] + 1]++;
  for (int i = 0; i < t->nr; ++i) t->rp[i + 1] += t->rp[i];
  int* pos = malloc(sizeof(int) * (size_t)(t->nr + 1));
  if (!pos) return OR_ERR_OOM;
  memcpy(pos, t->rp, sizeof(int) * (size_t)(t->nr + 1));
  for (int i = 0; i < a->nr; ++i)
    for (int k = a->rp[i]; k < a->rp[i + 1]; ++k) {
      int j = a->ci[k];
      t->ci[pos[j]] = i; t->v[pos[j]] = a->v[k]; pos[j]++;
    }
  free(pos);
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Element-wise Galerkin assembly with Gauss quadrature (Sec. 2, Sec. 3       */
/* "Computational costs", Eq. PM).  Dense slot storage per full-space row.    */
/* ------------------------------------------------------------------------- */
enum { K_STIFF = 0, K_MASS = 1 };

typedef struct {
  int d, ne, q, r;          /* test degree q, trial degree r */
  int nq, nr;               /* functions per direction */
  int w;                    /* slots per direction: q + r + 1 */
  long long rows, slots;    /* nq^d rows, w^d slots */
  double* S;                /* rows x slots */
  double* load;             /* nq^d load vector (test space), may be NULL */
} slotmat;

static long long ipow(long long b, int e) { long long r = 1; while (e-- > 0) r *= b; return r; }

/* one-dimensional tables for degree deg on ne elements, ng Gauss points:
 * val[(e*ng+g)*(deg+1)+a] = N_{e+a,deg}(xi_{e,g}), der likewise. */
static void tab1d(int deg, int ne, int ng, const double* gx, double* val, double* der) {
  for (int e = 0; e < ne; ++e)
    for (int g = 0; g < ng; ++g) {
      double x = ((double)e + gx[g]) / ne;
      for (int a = 0; a <= deg; ++a) {
        val[((size_t)e * ng + g) * (deg + 1) + a] = bspl(deg, ne, e + a, deg, x);
        der[((size_t)e * ng + g) * (deg + 1) + a] = bspl_d(deg, ne, e + a, deg, x);
      }
    }
}

static int assemble(int dom, int d, int ne, int q, int r, int kind, int with_load, int ex, slotmat* out) {
  memset(out, 0, sizeof(*out));
  out->d = d; out->ne = ne; out->q = q; out->r = r;
  out->nq = ne + q; out->nr = ne + r; out->w = q + r + 1;
  out->rows = ipow(out->nq, d); out->slots = ipow(out->w, d);
  out->S = calloc((size_t)(out->rows * out->slots), sizeof(double));
  if (!out->S) return OR_ERR_OOM;
  if (with_load) { out->load = calloc((size_t)out->rows, sizeof(double)); if (!out->load) return OR_ERR_OOM; }
  int ng = (q > r ? q : r) + 1;                          /* reading R3 */
  double gx[16], gw[16];
  or_gauss(ng, gx, gw);
  double* vq = malloc(sizeof(double) * (size_t)ne * ng * (q + 1));
  double* dq = malloc(sizeof(double) * (size_t)ne * ng * (q + 1));
  double* vr = malloc(sizeof(double) * (size_t)ne * ng * (r + 1));
  double* dr = malloc(sizeof(double) * (size_t)ne * ng * (r + 1));
  if (!vq || !dq || !vr || !dr) return OR_ERR_OOM;
  tab1d(q, ne, ng, gx, vq, dq);
  tab1d(r, ne, ng, gx, vr, dr);
  int nloc_q = (int)ipow(q + 1, d), nloc_r = (int)ipow(r + 1, d);
  double *phq = malloc(sizeof(double) * nloc_q), *ghq = malloc(sizeof(double) * nloc_q * 3);
  double *phr = malloc(sizeof(double) * nloc_r), *ghr = malloc(sizeof(double) * nloc_r * 3);
  long long nel = ipow(ne, d), ngp = ipow(ng, d);
  /* slot(offset) = sum_c (aj_c - ai_c + q) w^c = slot_j[lj] - slot_i[li] + slot_q */
  long long* slot_i = malloc(sizeof(long long) * nloc_q);
  long long* slot_j = malloc(sizeof(long long) * nloc_r);
  long long slot_q = 0;
  for (int c = d - 1; c >= 0; --c) slot_q = slot_q * out->w + q;
  for (int li = 0; li < nloc_q; ++li) {
    long long s = 0; int t = li, a[3] = {0, 0, 0};
    for (int c = 0; c < d; ++c) { a[c] = t % (q + 1); t /= (q + 1); }
    for (int c = d - 1; c >= 0; --c) s = s * out->w + a[c];
    slot_i[li] = s;
  }
  for (int lj = 0; lj < nloc_r; ++lj) {
    long long s = 0; int t = lj, a[3] = {0, 0, 0};
    for (int c = 0; c < d; ++c) { a[c] = t % (r + 1); t /= (r + 1); }
    for (int c = d - 1; c >= 0; --c) s = s * out->w + a[c];
    slot_j[lj] = s;
  }
  for (long long el = 0; el < nel; ++el) {
    int e[3] = {0, 0, 0};
    { long long t = el; for (int a = 0; a < d; ++a) { e[a] = (int)(t % ne); t /= ne; } }
    for (long long gp = 0; gp < ngp; ++gp) {
      int g[3] = {0, 0, 0};
      { long long t = gp; for (int a = 0; a < d; ++a) { g[a] = (int)(t % ng); t /= ng; } }
      double xi[3] = {0, 0, 0}, wt = 1.0;
      for (int a = 0; a < d; ++a) { xi[a] = ((double)e[a] + gx[g[a]]) / ne; wt *= gw[g[a]] / ne; }
      double X[3] = {0, 0, 0}, J[3][3], det;
      geo(dom, d, xi, X, J, &det);
      /* Ji = J^{-1}; physical gradients use its transpose */
      double Ji[3][3] = {{0}};
      if (d == 2) {
        Ji[0][0] = J[1][1] / det; Ji[0][1] = -J[0][1] / det;
        Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
      } else {
        for (int a = 0; a < 3; ++a) Ji[a][a] = 1.0 / J[a][a];  /* the cube map is the identity */
      }
      double dv = wt * fabs(det);
      /* values and physical gradients of the active test (q) and trial (r) functions */
      for (int side = 0; side < 2; ++side) {
        int deg = side ? r : q, nloc = side ? nloc_r : nloc_q;
        const double* tv = side ? vr : vq; const double* td = side ? dr : dq;
        double* ph = side ? phr : phq; double* gh = side ? ghr : ghq;
        for (int l = 0; l < nloc; ++l) {
          int a[3] = {0, 0, 0};
          { int t = l; for (int c = 0; c < d; ++c) { a[c] = t % (deg + 1); t /= (deg + 1); } }
          double val = 1.0, gref[3] = {1.0, 1.0, 1.0};
          for (int c = 0; c < d; ++c) {
            size_t o = ((size_t)e[c] * ng + g[c]) * (deg + 1) + a[c];
            val *= tv[o];
            for (int c2 = 0; c2 < d; ++c2) gref[c2] *= (c2 == c) ? td[o] : tv[o];
          }
          ph[l] = val;
          /* physical gradient = J^{-T} (reference gradient) */
          for (int c = 0; c < d; ++c) {
            double s = 0.0;
            for (int c2 = 0; c2 < d; ++c2) s += Ji[c2][c] * gref[c2];
            gh[l * 3 + c] = s;
          }
        }
      }
      double fval = with_load ? f_source(dom, ex, d, X) : 0.0;
      for (int li = 0; li < nloc_q; ++li) {
        int ai[3] = {0, 0, 0};
        { int t = li; for (int c = 0; c < d; ++c) { ai[c] = t % (q + 1); t /= (q + 1); } }
        long long row = 0;
        for (int c = d - 1; c >= 0; --c) row = row * out->nq + (e[c] + ai[c]);
        if (with_load) out->load[row] += dv * fval * phq[li];
        for (int lj = 0; lj < nloc_r; ++lj) {
          /* slot of the offset (trial index - test index + q) per direction */
          long long slot = slot_j[lj] - slot_i[li] + slot_q;
          double integrand;
          if (kind == K_STIFF && dom == OR_CDR_SQUARE) {
            /* (D grad phi_j) . grad phi_i + (v . grad phi_j) phi_i + R phi_j phi_i, i test, j trial */
            integrand = CDR_R * phq[li] * phr[lj];
            for (int a = 0; a < 2; ++a) {
              integrand += CDR_V[a] * ghr[lj * 3 + a] * phq[li];
              for (int b = 0; b < 2; ++b) integrand += CDR_D[a][b] * ghr[lj * 3 + b] * ghq[li * 3 + a];
            }
          } else if (kind == K_STIFF) {
            integrand = 0.0;
            for (int c = 0; c < d; ++c) integrand += ghq[li * 3 + c] * ghr[lj * 3 + c];
          } else {
            integrand = phq[li] * phr[lj];
          }
          out->S[row * out->slots + slot] += dv * integrand;
        }
      }
    }
  }
  free(vq); free(dq); free(vr); free(dr); free(phq); free(ghq); free(phr); free(ghr);
  free(slot_i); free(slot_j);
  return OR_OK;
}

static void slot_free(slotmat* s) { free(s->S); free(s->load); memset(s, 0, sizeof(*s)); }

/* decode multi-index of full-space function index */
static void unflat(long long idx, int n, int d, int* m) {
  for (int a = 0; a < d; ++a) { m[a] = (int)(idx % n); idx /= n; }
}

/* interior index of a full-space multi-index, or -1 if on the boundary */
static long long interior_index(const int* m, int n, int d) {
  long long idx = 0;
  for (int a = d - 1; a >= 0; --a) {
    if (m[a] < 1 || m[a] > n - 2) return -1;
    idx = idx * (n - 2) + (m[a] - 1);
  }
  return idx;
}

/* CSR over rows/cols selected by `interior_only` (both sides) from slot storage. */
static int slots_to_csr(const slotmat* s, int interior_only, csr* out) {
  int d = s->d;
  long long nrow = interior_only ? ipow(s->nq - 2, d) : s->rows;
  long long ncol = interior_only ? ipow(s->nr - 2, d) : ipow(s->nr, d);
  out->nr = (int)nrow; out->nc = (int)ncol;
  out->rp = calloc((size_t)nrow + 1, sizeof(int));
  size_t cap = (size_t)nrow * (size_t)s->slots + 1;
  out->ci = malloc(sizeof(int) * cap);
  out->v = malloc(sizeof(double) * cap);
  if (!out->rp || !out->ci || !out->v) return OR_ERR_OOM;
  long long k = 0, ir = 0;
  for (long long row = 0; row < s->rows; ++row) {
    int mi[3] = {0, 0, 0};
    unflat(row, s->nq, d, mi);
    if (interior_only && interior_index(mi, s->nq, d) < 0) continue;
    for (long long slot = 0; slot < s->slots; ++slot) {
      int off[3] = {0, 0, 0};
      unflat(slot, s->w, d, off);
      int mj[3] = {0, 0, 0}, ok = 1;
      for (int a = 0; a < d; ++a) {
        mj[a] = mi[a] + off[a] - s->q;
        if (mj[a] < 0 || mj[a] >= s->nr) ok = 0;
      }
      if (!ok) continue;
      long long col;
      if (interior_only) { col = interior_index(mj, s->nr, d); if (col < 0) continue; }
      else { col = 0; for (int a = d - 1; a >= 0; --a) col = col * s->nr + mj[a]; }
      out->ci[k] = (int)col; out->v[k] = s->S[row * s->slots + slot]; ++k;
    }
    out->rp[++ir] = (int)k;
  }
  out->nnz = (int)k;
  return OR_OK;
}

/* row sums of the full slot matrix, restricted to interior rows (reading R6) */
static double* lumped_interior(const slotmat* s) {
  long long n = ipow(s->nq - 2, s->d);
  double* ml = malloc(sizeof(double) * (size_t)n);
  if (!ml) return NULL;
  for (long long row = 0; row < s->rows; ++row) {
    int mi[3] = {0, 0, 0};
    unflat(row, s->nq, s->d, mi);
    long long ii = interior_index(mi, s->nq, s->d);
    if (ii < 0) continue;
    double acc = 0.0;
    for (long long slot = 0; slot < s->slots; ++slot) acc += s->S[row * s->slots + slot];
    ml[ii] = acc;
  }
  return ml;
}

/* ------------------------------------------------------------------------- */
/* Dense LU with partial pivoting (coarsest h-level and the 1-D projection)   */
/* ------------------------------------------------------------------------- */
static int dense_lu(int n, double* a, int* piv) {
  for (int k = 0; k < n; ++k) {
    int pr = k; double mx = fabs(a[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) if (fabs(a[(size_t)i * n + k]) > mx) { mx = fabs(a[(size_t)i * n + k]); pr = i; }
    if (mx == 0.0) return OR_ERR_ZERO_PIVOT;
    piv[k] = pr;
    if (pr != k) for (int j = 0; j < n; ++j) { double t = a[(size_t)k * n + j]; a[(size_t)k * n + j] = a[(size_t)pr * n + j]; a[(size_t)pr * n + j] = t; }
    for (int i = k + 1; i < n; ++i) {
      double l = a[(size_t)i * n + k] / a[(size_t)k * n + k];
      a[(size_t)i * n + k] = l;
      for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
    }
  }
  return OR_OK;
}
static void dense_lu_solve(int n, const double* a, const int* piv, double* b) {
  for (int k = 0; k < n; ++k) if (piv[k] != k) { double t = b[k]; b[k] = b[piv[k]]; b[piv[k]] = t; }
  for (int i = 0; i < n; ++i) for (int j = 0; j < i; ++j) b[i] -= a[(size_t)i * n + j] * b[j];
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i + 1; j < n; ++j) b[i] -= a[(size_t)i * n + j] * b[j];
    b[i] /= a[(size_t)i * n + i];
  }
}

/* ------------------------------------------------------------------------- */
/* Dirichlet data (reading R5): 1-D L2 projection on the annulus arcs         */
/* ------------------------------------------------------------------------- */
/* Fills uB (full-space coefficient vector, zero in the interior) for 2-D
 * problems.  Only the annulus with the sin-product solution has non-zero data,
 * on the arcs xi = 0 (r = 1) and xi = 1 (r = 2). */
static int boundary_values(int dom, int ex, int d, int ne, int q, double* uB) {
  int n = ne + q;
  memset(uB, 0, sizeof(double) * (size_t)ipow(n, d));
  if (!(dom == OR_ANNULUS && ex == OR_U_SINPROD)) return OR_OK;
  int ng = q + 1;
  double gx[16], gw[16];
  or_gauss(ng, gx, gw);
  int m = n - 2;  /* unknown interior edge coefficients; end values are 0 */
  double* Mm = calloc((size_t)m * m, sizeof(double));
  int* piv = malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
  double* b = calloc((size_t)(m > 0 ? m : 1), sizeof(double));
  if (!Mm || !piv || !b) return OR_ERR_OOM;
  for (int e = 0; e < ne; ++e)
    for (int g = 0; g < ng; ++g) {
      double s = ((double)e + gx[g]) / ne, wt = gw[g] / ne;
      for (int a = 0; a <= q; ++a) {
        int i = e + a;
        if (i < 1 || i > n - 2) continue;
        double vi = bspl(q, ne, i, q, s);
        for (int c = 0; c <= q; ++c) {
          int j = e + c;
          if (j < 1 || j > n - 2) continue;
          Mm[(size_t)(i - 1) * m + (j - 1)] += wt * vi * bspl(q, ne, j, q, s);
        }
      }
    }
  int st = dense_lu(m, Mm, piv);
  if (st) return st;
  for (int side = 0; side < 2; ++side) {
    double xi0 = side ? 1.0 : 0.0;
    memset(b, 0, sizeof(double) * (size_t)m);
    for (int e = 0; e < ne; ++e)
      for (int g = 0; g < ng; ++g) {
        double s = ((double)e + gx[g]) / ne, wt = gw[g] / ne;
        double xi[3] = {xi0, s, 0}, X[3], J[3][3], det;
        geo(dom, d, xi, X, J, &det);
        double gv = u_exact(dom, ex, d, X);
        for (int a = 0; a <= q; ++a) {
          int i = e + a;
          if (i < 1 || i > n - 2) continue;
          b[i - 1] += wt * gv * bspl(q, ne, i, q, s);
        }
      }
    dense_lu_solve(m, Mm, piv, b);
    int ix = side ? n - 1 : 0;
    for (int iy = 1; iy <= n - 2; ++iy) uB[(size_t)ix + (size_t)n * iy] = b[iy - 1];
  }
  free(Mm); free(piv); free(b);
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* ILUT (Sec. 3 "Smoother": dual threshold; readings R7-R10)                 */
/* ------------------------------------------------------------------------- */
typedef struct { int col; double val; } ent;

static int cmp_mag_desc(const void* x, const void* y) {
  const ent* a = x; const ent* b = y;
  double ma = fabs(a->val), mb = fabs(b->val);
  if (ma > mb) return -1;
  if (ma < mb) return 1;
  return (a->col < b->col) ? -1 : (a->col > b->col);
}
static int cmp_col(const void* x, const void* y) {
  const ent* a = x; const ent* b = y;
  return (a->col < b->col) ? -1 : (a->col > b->col);
}

/* keep the M largest magnitudes of c[0..n) by reading R9; result sorted by column */
static int keep_largest(ent* c, int n, int M, ent* tmp) {
  if (n <= M) { qsort(c, (size_t)n, sizeof(ent), cmp_col); return n; }
  qsort(c, (size_t)n, sizeof(ent), cmp_mag_desc);
  double t = fabs(c[M - 1].val);
  double hi = t * (1.0 + 1e-12), lo = t * (1.0 - 1e-12);
  int K = 0;
  while (K < n && fabs(c[K].val) > hi) ++K;
  int nb = 0;
  for (int s = K; s < n; ++s) {
    double m = fabs(c[s].val);
    if (m >= lo && m <= hi) tmp[nb++] = c[s];
  }
  qsort(tmp, (size_t)nb, sizeof(ent), cmp_col);
  int need = M - K;
  for (int s = 0; s < need && s < nb; ++s) c[K + s] = tmp[s];
  int kept = K + (need < nb ? need : nb);
  qsort(c, (size_t)kept, sizeof(ent), cmp_col);
  return kept;
}

int or_ilut_budget(long long nnz, int n, double m) {
  double b = ceil(m * (double)nnz / (double)n);
  if (b > n) b = n;
  if (b < 0) b = 0;
  return (int)b;
}

/* ILUT of square CSR A (sorted columns): L strict lower (unit diagonal implied),
 * U upper including the diagonal (stored first in each row). */
static int ilut(const csr* A, double tau, double fill, csr* L, csr* U) {
  int n = A->nr;
  int M = or_ilut_budget(A->nnz, n, fill);
  double* w = calloc((size_t)n, sizeof(double));
  char* on = calloc((size_t)n, 1);
  int* touched = malloc(sizeof(int) * (size_t)n);
  ent* cand = malloc(sizeof(ent) * (size_t)n);
  ent* tmp = malloc(sizeof(ent) * (size_t)n);
  size_t capL = (size_t)n * (M + 1) + 1, capU = (size_t)n * (M + 2) + 1;
  L->nr = L->nc = U->nr = U->nc = n;
  L->rp = calloc((size_t)n + 1, sizeof(int)); U->rp = calloc((size_t)n + 1, sizeof(int));
  L->ci = malloc(sizeof(int) * capL); L->v = malloc(sizeof(double) * capL);
  U->ci = malloc(sizeof(int) * capU); U->v = malloc(sizeof(double) * capU);
  int* udiag = malloc(sizeof(int) * (size_t)n);   /* position of u_kk in U */
  if (!w || !on || !touched || !cand || !tmp || !L->rp || !U->rp || !L->ci || !L->v || !U->ci || !U->v || !udiag)
    return OR_ERR_OOM;
  long long nl = 0, nu = 0;
  for (int i = 0; i < n; ++i) {
    int nt = 0;
    double rs = 0.0;
    int cnt = A->rp[i + 1] - A->rp[i];
    for (int t = A->rp[i]; t < A->rp[i + 1]; ++t) {
      int j = A->ci[t];
      w[j] = A->v[t]; on[j] = 1; touched[nt++] = j;
      rs += fabs(A->v[t]);
    }
    double taui = cnt > 0 ? tau * rs / cnt : 0.0;     /* reading R7 */
    int lo = cnt > 0 ? A->ci[A->rp[i]] : i;
    /* eliminate columns k < i in ascending order, including fill created on the way */
    for (int k = lo; k < i; ++k) {
      if (!on[k] || w[k] == 0.0) continue;
      double wk = w[k] / U->v[udiag[k]];
      if (fabs(wk) < taui) { w[k] = 0.0; continue; }
      w[k] = wk;
      for (int t = udiag[k] + 1; t < U->rp[k + 1]; ++t) {
        int j = U->ci[t];
        if (!on[j]) { on[j] = 1; w[j] = 0.0; touched[nt++] = j; }
        w[j] -= wk * U->v[t];
      }
    }
    /* dropping: relative tolerance, then the M largest in L and in U (R8, R9) */
    int ncl = 0, ncu = 0;
    double diag = on[i] ? w[i] : 0.0;
    for (int s = 0; s < nt; ++s) {
      int j = touched[s];
      if (j == i) continue;
      double v = w[j];
      if (v == 0.0 || fabs(v) < taui) continue;
      if (j < i) { cand[ncl].col = j; cand[ncl].val = v; ++ncl; }
    }
    int keptL = keep_largest(cand, ncl, M, tmp);
    for (int s = 0; s < keptL; ++s) { L->ci[nl] = cand[s].col; L->v[nl] = cand[s].val; ++nl; }
    L->rp[i + 1] = (int)nl;
    for (int s = 0; s < nt; ++s) {
      int j = touched[s];
      if (j <= i) continue;
      double v = w[j];
      if (v == 0.0 || fabs(v) < taui) continue;
      cand[ncu].col = j; cand[ncu].val = v; ++ncu;
    }
    int keptU = keep_largest(cand, ncu, M, tmp);
    if (diag == 0.0) return OR_ERR_ZERO_PIVOT;
    udiag[i] = (int)nu;
    U->ci[nu] = i; U->v[nu] = diag; ++nu;
    for (int s = 0; s < keptU; ++s) { U->ci[nu] = cand[s].col; U->v[nu] = cand[s].val; ++nu; }
    U->rp[i + 1] = (int)nu;
    for (int s = 0; s < nt; ++s) { w[touched[s]] = 0.0; on[touched[s]] = 0; }
  }
  L->nnz = (int)nl; U->nnz = (int)nu;
  free(w); free(on); free(touched); free(cand); free(tmp); free(udiag);
  return OR_OK;
}

/* forward substitution with unit lower L, backward with U (Eq. inverse) */
static void lsolve(const csr* L, const double* b, double* y) {
  for (int i = 0; i < L->nr; ++i) {
    double s = b[i];
    for (int t = L->rp[i]; t < L->rp[i + 1]; ++t) s -= L->v[t] * y[L->ci[t]];
    y[i] = s;
  }
}
static void usolve(const csr* U, const double* y, double* x) {
  for (int i = U->nr - 1; i >= 0; --i) {
    double s = y[i], dg = 0.0;
    for (int t = U->rp[i]; t < U->rp[i + 1]; ++t) {
      if (U->ci[t] == i) dg = U->v[t];
      else s -= U->v[t] * x[U->ci[t]];
    }
    x[i] = s / dg;
  }
}

/* ------------------------------------------------------------------------- */
/* The hierarchy                                                              */
/* ------------------------------------------------------------------------- */
typedef struct {
  int q, n1d, N;
  csr A, L, U;
  double* ML;          /* lumped mass, interior */
  csr P;               /* P_{coarse}^{q}: N_q x N_coarse (interior, unscaled) */
  csr Pt;              /* its transpose */
  double* MCB; int mcb;   /* consistent transfers: banded Cholesky factor of the interior mass, half bandwidth */
} plevel;

typedef struct {
  int ne, n1d, N;
  csr A;
  csr P, R;            /* canonical prolongation from the next coarser level, R = P^T */
} hlevel;

typedef struct or_hier {
  int dom, d, p, k, proj, ex, nu1, nu2, ccyc;
  double tau, fill;
  int nlev;
  plevel lev[16];
  double* ML1;         /* lumped mass of V_{h,1}, interior */
  int consistent;      /* 1: transfers with the consistent mass matrices (App. B) */
  double* MC1B; int mc1b;   /* banded Cholesky factor of the interior mass of V_{h,1} */
  int nh;
  hlevel hl[16];
  double* LUc; int* piv; int Nc;
  double* f;           /* interior load vector with the Dirichlet lift */
  double* uB;          /* full-space boundary coefficients (degree p) */
} or_hier;

static void lev_free(plevel* l) { csr_free(&l->A); csr_free(&l->L); csr_free(&l->U); csr_free(&l->P); csr_free(&l->Pt); free(l->ML); free(l->MCB); }

void or_free(or_hier* h) {
  if (!h) return;
  for (int l = 0; l < h->nlev; ++l) lev_free(&h->lev[l]);
  for (int j = 0; j < h->nh; ++j) { csr_free(&h->hl[j].A); csr_free(&h->hl[j].P); csr_free(&h->hl[j].R); }
  free(h->ML1); free(h->MC1B); free(h->LUc); free(h->piv); free(h->f); free(h->uB);
  free(h);
}

/* canonical prolongation between P1 interior node sets: fine has nf elements
 * per direction, coarse nf/2 (Sec. 3, "canonical prolongation"). */
static int canon_prolong(int d, int nf, csr* P) {
  int mf = nf - 1, nc = nf / 2, mc = nc - 1;
  long long Nf = ipow(mf, d), Ncc = ipow(mc, d);
  P->nr = (int)Nf; P->nc = (int)Ncc;
  P->rp = calloc((size_t)Nf + 1, sizeof(int));
  P->ci = malloc(sizeof(int) * (size_t)Nf * (size_t)ipow(2, d));
  P->v = malloc(sizeof(double) * (size_t)Nf * (size_t)ipow(2, d));
  if (!P->rp || !P->ci || !P->v) return OR_ERR_OOM;
  long long k = 0;
  for (long long fi = 0; fi < Nf; ++fi) {
    int f[3] = {0, 0, 0};
    unflat(fi, mf, d, f);
    /* per direction: candidate coarse nodes and weights (node numbers 0..nc) */
    int cn[3][2], nn[3]; double cw[3][2];
    for (int a = 0; a < d; ++a) {
      int node = f[a] + 1;
      if (node % 2 == 0) { cn[a][0] = node / 2; cw[a][0] = 1.0; nn[a] = 1; }
      else { cn[a][0] = (node - 1) / 2; cw[a][0] = 0.5; cn[a][1] = (node + 1) / 2; cw[a][1] = 0.5; nn[a] = 2; }
    }
    int tot = 1; for (int a = 0; a < d; ++a) tot *= nn[a];
    /* emit in ascending coarse index order: last direction slowest */
    ent buf[8]; int nb = 0;
    for (int c = 0; c < tot; ++c) {
      int t = c, ok = 1; long long col = 0; double wv = 1.0; int sel[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) { sel[a] = t % nn[a]; t /= nn[a]; }
      for (int a = d - 1; a >= 0; --a) {
        int node = cn[a][sel[a]];
        if (node < 1 || node > nc - 1) { ok = 0; break; }
        col = col * mc + (node - 1);
        wv *= cw[a][sel[a]];
      }
      if (!ok) continue;
      buf[nb].col = (int)col; buf[nb].val = wv; ++nb;
    }
    qsort(buf, (size_t)nb, sizeof(ent), cmp_col);
    for (int s = 0; s < nb; ++s) { P->ci[k] = buf[s].col; P->v[k] = buf[s].val; ++k; }
    P->rp[fi + 1] = (int)k;
  }
  P->nnz = (int)k;
  return OR_OK;
}

/* interior stiffness (and optionally the lifted load) at degree q, ne elements */
static int build_operator(or_hier* h, int ne, int q, csr* A, double** ML, double** fvec, double** uBout) {
  slotmat s;
  int st = assemble(h->dom, h->d, ne, q, q, K_STIFF, fvec != NULL, h->ex, &s);
  if (st) return st;
  st = slots_to_csr(&s, 1, A);
  if (st) return st;
  if (fvec) {
    int n = ne + q, d = h->d;
    long long Nfull = ipow(n, d), Ni = ipow(n - 2, d);
    double* uB = malloc(sizeof(double) * (size_t)Nfull);
    double* f = malloc(sizeof(double) * (size_t)Ni);
    if (!uB || !f) return OR_ERR_OOM;
    st = (d == 2) ? boundary_values(h->dom, h->ex, d, ne, q, uB) : OR_OK;
    if (d == 3) memset(uB, 0, sizeof(double) * (size_t)Nfull);
    if (st) return st;
    /* f_I = load_I - A_IB u_B */
    for (long long row = 0; row < s.rows; ++row) {
      int mi[3] = {0, 0, 0};
      unflat(row, n, d, mi);
      long long ii = interior_index(mi, n, d);
      if (ii < 0) continue;
      double acc = s.load[row];
      for (long long slot = 0; slot < s.slots; ++slot) {
        int off[3] = {0, 0, 0}, mj[3] = {0, 0, 0}, ok = 1;
        unflat(slot, s.w, d, off);
        for (int a = 0; a < d; ++a) { mj[a] = mi[a] + off[a] - q; if (mj[a] < 0 || mj[a] >= n) ok = 0; }
        if (!ok || interior_index(mj, n, d) >= 0) continue;
        long long col = 0; for (int a = d - 1; a >= 0; --a) col = col * n + mj[a];
        acc -= s.S[row * s.slots + slot] * uB[col];
      }
      f[ii] = acc;
    }
    *fvec = f; *uBout = uB;
  }
  slot_free(&s);
  if (ML) {
    slotmat m;
    st = assemble(h->dom, h->d, ne, q, q, K_MASS, 0, h->ex, &m);
    if (st) return st;
    *ML = lumped_interior(&m);
    slot_free(&m);
    if (!*ML) return OR_ERR_OOM;
  }
  return OR_OK;
}

or_hier* or_setup(int dom, int p, int k, double tau, double fill, int proj, int ex,
                  int nu1, int nu2, int ccyc, int* status) {
  *status = OR_ERR_ARG;
  if (dom < 0 || dom > 3 || p < 2 || p > 8 || k < 3 || k > 12 || ccyc < 1 || nu1 < 0 || nu2 < 0) return NULL;
  if (dom == OR_CUBE && k > 6) return NULL;
  or_hier* h = calloc(1, sizeof(or_hier));
  if (!h) { *status = OR_ERR_OOM; return NULL; }
  h->dom = dom; h->d = dom == OR_CUBE ? 3 : 2; h->p = p; h->k = k; h->proj = proj; h->ex = ex;
  h->nu1 = nu1; h->nu2 = nu2; h->ccyc = ccyc; h->tau = tau; h->fill = fill;
  int ne = 1 << k, st;
  h->nlev = (proj == OR_DIRECT) ? 1 : p - 1;
  for (int l = 0; l < h->nlev; ++l) {
    plevel* L = &h->lev[l];
    L->q = p - l; L->n1d = ne + L->q - 2; L->N = (int)ipow(L->n1d, h->d);
    st = build_operator(h, ne, L->q, &L->A, &L->ML, l == 0 ? &h->f : NULL, l == 0 ? &h->uB : NULL);
    if (st) goto fail;
    st = ilut(&L->A, tau, fill, &L->L, &L->U);
    if (st) goto fail;
    int qc = (proj == OR_DIRECT || L->q == 2) ? 1 : L->q - 1;
    slotmat s;
    st = assemble(dom, h->d, ne, L->q, qc, K_MASS, 0, ex, &s);   /* P_{qc}^{q}, Eq. PM */
    if (st) goto fail;
    st = slots_to_csr(&s, 1, &L->P);
    slot_free(&s);
    if (st) goto fail;
    st = csr_transpose(&L->P, &L->Pt);
    if (st) goto fail;
  }
  /* p = 1 hierarchy, reading R12 */
  h->nh = k - 3 + 1;
  for (int j = 0; j < h->nh; ++j) {
    hlevel* H = &h->hl[j];
    H->ne = ne >> j; H->n1d = H->ne - 1; H->N = (int)ipow(H->n1d, h->d);
    st = build_operator(h, H->ne, 1, &H->A, j == 0 ? &h->ML1 : NULL, NULL, NULL);
    if (st) goto fail;
    if (j + 1 < h->nh) {
      st = canon_prolong(h->d, H->ne, &H->P);
      if (st) goto fail;
      st = csr_transpose(&H->P, &H->R);
      if (st) goto fail;
    }
  }
  {
    hlevel* C = &h->hl[h->nh - 1];
    int n = C->N;
    h->Nc = n;
    h->LUc = calloc((size_t)n * n, sizeof(double));
    h->piv = malloc(sizeof(int) * (size_t)n);
    if (!h->LUc || !h->piv) { st = OR_ERR_OOM; goto fail; }
    for (int i = 0; i < n; ++i)
      for (int t = C->A.rp[i]; t < C->A.rp[i + 1]; ++t) h->LUc[(size_t)i * n + C->A.ci[t]] = C->A.v[t];
    st = dense_lu(n, h->LUc, h->piv);
    if (st) goto fail;
  }
  *status = OR_OK;
  return h;
fail:
  *status = st;
  or_free(h);
  return NULL;
}

/* ------------------------------------------------------------------------- */
/* Cycle pieces                                                               */
/* ------------------------------------------------------------------------- */
static double* dalloc(long long n) { return calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

static void residual(const csr* A, const double* f, const double* u, double* r) {
  spmv(A, u, r);
  for (int i = 0; i < A->nr; ++i) r[i] = f[i] - r[i];
}

/* one ILUT smoothing step, Eq. smooth with S = (LU)^{-1} (Eq. inverse) */
static void ilut_smooth(const plevel* L, const double* f, double* u) {
  double* r = dalloc(L->N); double* y = dalloc(L->N); double* e = dalloc(L->N);
  residual(&L->A, f, u, r);
  lsolve(&L->L, r, y);
  usolve(&L->U, y, e);
  for (int i = 0; i < L->N; ++i) u[i] += e[i];
  free(r); free(y); free(e);
}

static void gs_forward(const csr* A, const double* b, double* x) {
  for (int i = 0; i < A->nr; ++i) {
    double s = b[i], dg = 0.0;
    for (int t = A->rp[i]; t < A->rp[i + 1]; ++t) {
      if (A->ci[t] == i) dg = A->v[t]; else s -= A->v[t] * x[A->ci[t]];
    }
    x[i] = s / dg;
  }
}
static void gs_backward(const csr* A, const double* b, double* x) {
  for (int i = A->nr - 1; i >= 0; --i) {
    double s = b[i], dg = 0.0;
    for (int t = A->rp[i]; t < A->rp[i + 1]; ++t) {
      if (A->ci[t] == i) dg = A->v[t]; else s -= A->v[t] * x[A->ci[t]];
    }
    x[i] = s / dg;
  }
}

/* one h-multigrid V-cycle at P1 level j on A_j x = b (Sec. 3, Fig. 1) */
static void hmg_vcycle(const or_hier* h, int j, const double* b, double* x) {
  const hlevel* H = &h->hl[j];
  if (j == h->nh - 1) {
    memcpy(x, b, sizeof(double) * (size_t)H->N);
    dense_lu_solve(h->Nc, h->LUc, h->piv, x);
    return;
  }
  const hlevel* C = &h->hl[j + 1];
  double* r = dalloc(H->N); double* rc = dalloc(C->N); double* ec = dalloc(C->N); double* pe = dalloc(H->N);
  gs_forward(&H->A, b, x);
  residual(&H->A, b, x, r);
  spmv(&H->R, r, rc);
  hmg_vcycle(h, j + 1, rc, ec);
  spmv(&H->P, ec, pe);
  for (int i = 0; i < H->N; ++i) x[i] += pe[i];
  gs_backward(&H->A, b, x);
  free(r); free(rc); free(ec); free(pe);
}

/* coarse grid correction at p = 1: ccyc h-MG V-cycles from zero (Sec. 3) */
static void coarse_solve(const or_hier* h, const double* r1, double* e1) {
  memset(e1, 0, sizeof(double) * (size_t)h->hl[0].N);
  for (int c = 0; c < h->ccyc; ++c) hmg_vcycle(h, 0, r1, e1);
}

static int coarse_N(const or_hier* h, int l) { return (l + 1 < h->nlev) ? h->lev[l + 1].N : h->hl[0].N; }
static const double* coarse_ML(const or_hier* h, int l) { return (l + 1 < h->nlev) ? h->lev[l + 1].ML : h->ML1; }

/* Banded Cholesky M = L L^T of a symmetric positive definite CSR matrix: row i
 * of L holds L_ij, j = i-b..i, at B[i*(b+1) + (i-j)]; *b: half bandwidth. */
static int band_cholesky(const csr* M, int* bout, double** Bout) {
  int n = M->nr, b = 0;
  for (int i = 0; i < n; ++i)
    for (int t = M->rp[i]; t < M->rp[i + 1]; ++t) if (i - M->ci[t] > b) b = i - M->ci[t];
  double* B = calloc((size_t)n * (size_t)(b + 1), sizeof(double));
  if (!B) return OR_ERR_OOM;
  for (int i = 0; i < n; ++i)
    for (int t = M->rp[i]; t < M->rp[i + 1]; ++t) {
      int j = M->ci[t];
      if (j <= i) B[(size_t)i * (b + 1) + (i - j)] = M->v[t];
    }
  for (int i = 0; i < n; ++i) {
    int j0 = i - b > 0 ? i - b : 0;
    for (int j = j0; j <= i; ++j) {
      double s = B[(size_t)i * (b + 1) + (i - j)];
      int k0 = (i - b > j - b ? i - b : j - b); if (k0 < 0) k0 = 0;
      for (int k = k0; k < j; ++k) s -= B[(size_t)i * (b + 1) + (i - k)] * B[(size_t)j * (b + 1) + (j - k)];
      if (j == i) {
        if (!(s > 0.0)) { free(B); return OR_ERR_ZERO_PIVOT; }
        B[(size_t)i * (b + 1)] = sqrt(s);
      } else {
        B[(size_t)i * (b + 1) + (i - j)] = s / B[(size_t)j * (b + 1)];
      }
    }
  }
  *bout = b; *Bout = B;
  return OR_OK;
}
/* y <- M^{-1} y with the factor of band_cholesky: L z = y, then L^T y = z */
static void band_solve(int n, int b, const double* B, double* y) {
  for (int i = 0; i < n; ++i) {
    double s = y[i];
    for (int j = (i - b > 0 ? i - b : 0); j < i; ++j) s -= B[(size_t)i * (b + 1) + (i - j)] * y[j];
    y[i] = s / B[(size_t)i * (b + 1)];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k <= i + b && k < n; ++k) s -= B[(size_t)k * (b + 1) + (k - i)] * y[k];
    y[i] = s / B[(size_t)i * (b + 1)];
  }
}

/* restriction I_q^{qc}: r_c = (M_{qc})^{-1} P_q^{qc} r  (Eq. restriction), with
 * the lumped mass M^L (default) or the consistent mass M (App. B) */
static void restrict_(const or_hier* h, int l, const double* r, double* rc) {
  spmv(&h->lev[l].Pt, r, rc);
  if (h->consistent) {
    if (l + 1 < h->nlev) band_solve(h->lev[l + 1].N, h->lev[l + 1].mcb, h->lev[l + 1].MCB, rc);
    else band_solve(h->hl[0].N, h->mc1b, h->MC1B, rc);
    return;
  }
  const double* ml = coarse_ML(h, l);
  for (int i = 0; i < coarse_N(h, l); ++i) rc[i] /= ml[i];
}
/* prolongation I_{qc}^{q}: u += (M_q)^{-1} P_{qc}^{q} e_c  (Eq. prolongation), lumped or consistent */
static void prolong_add(const or_hier* h, int l, const double* ec, double* u) {
  const plevel* L = &h->lev[l];
  double* t = dalloc(L->N);
  spmv(&L->P, ec, t);
  if (h->consistent) {
    band_solve(L->N, L->mcb, L->MCB, t);
    for (int i = 0; i < L->N; ++i) u[i] += t[i];
  } else {
    for (int i = 0; i < L->N; ++i) u[i] += t[i] / L->ML[i];
  }
  free(t);
}

/* two-grid correction scheme applied recursively = V-cycle (Sec. 3, steps 1-5) */
static void vcycle(const or_hier* h, int l, const double* f, double* u) {
  const plevel* L = &h->lev[l];
  for (int m = 0; m < h->nu1; ++m) ilut_smooth(L, f, u);
  int Nc = coarse_N(h, l);
  double* r = dalloc(L->N); double* rc = dalloc(Nc); double* ec = dalloc(Nc);
  residual(&L->A, f, u, r);
  restrict_(h, l, r, rc);
  if (l + 1 < h->nlev) vcycle(h, l + 1, rc, ec);   /* e_c^0 = 0 */
  else coarse_solve(h, rc, ec);
  prolong_add(h, l, ec, u);
  for (int m = 0; m < h->nu2; ++m) ilut_smooth(L, f, u);
  free(r); free(rc); free(ec);
}

static double norm2(const double* x, int n) { double s = 0.0; for (int i = 0; i < n; ++i) s += x[i] * x[i]; return sqrt(s); }

/* stand-alone solver: V-cycles until ||r_k||/||r_0|| < tol (Sec. 5) */
int or_solve(const or_hier* h, const double* f, const double* u0, double tol, int maxit,
             double* u, double* hist, int* iters) {
  int N = h->lev[0].N;
  double* r = dalloc(N);
  memcpy(u, u0, sizeof(double) * (size_t)N);
  residual(&h->lev[0].A, f, u, r);
  double r0 = norm2(r, N);
  int st = OR_ERR_MAXITER;
  *iters = 0;
  if (r0 == 0.0) { free(r); return OR_OK; }
  for (int it = 0; it < maxit; ++it) {
    vcycle(h, 0, f, u);
    residual(&h->lev[0].A, f, u, r);
    double rel = norm2(r, N) / r0;
    hist[it] = rel;
    *iters = it + 1;
    if (rel < tol) { st = OR_OK; break; }
    if (rel > 1e10 || rel != rel) { st = OR_ERR_DIVERGED; break; }
  }
  free(r);
  return st;
}

/* ------------------------------------------------------------------------- */
/* Accessors used by the tests                                                */
/* ------------------------------------------------------------------------- */
int or_nlev(const or_hier* h) { return h->nlev; }
int or_nh(const or_hier* h) { return h->nh; }
int or_level_N(const or_hier* h, int l) { return l < h->nlev ? h->lev[l].N : -1; }
int or_level_q(const or_hier* h, int l) { return l < h->nlev ? h->lev[l].q : -1; }
int or_hlevel_N(const or_hier* h, int j) { return j < h->nh ? h->hl[j].N : -1; }

static const csr* pick(const or_hier* h, int which, int l) {
  if (which <= 4 && (l < 0 || l >= h->nlev)) return NULL;
  if (which >= 5 && (l < 0 || l >= h->nh)) return NULL;
  switch (which) {
    case 0: return &h->lev[l].A;
    case 1: return &h->lev[l].L;
    case 2: return &h->lev[l].U;
    case 3: return &h->lev[l].P;
    case 4: return &h->lev[l].Pt;
    case 5: return &h->hl[l].A;
    case 6: return l + 1 < h->nh ? &h->hl[l].P : NULL;
    case 7: return l + 1 < h->nh ? &h->hl[l].R : NULL;
  }
  return NULL;
}

/* which: 0 A, 1 L, 2 U, 3 P (prolongation matrix, unscaled), 4 P^T, 5 P1-level A,
 * 6 canonical P, 7 its transpose.  If rp == NULL only the sizes are returned. */
int or_get_csr(const or_hier* h, int which, int l, int* nr, int* nc, int* nnz, int* rp, int* ci, double* v) {
  const csr* a = pick(h, which, l);
  if (!a) return OR_ERR_ARG;
  *nr = a->nr; *nc = a->nc; *nnz = a->nnz;
  if (rp) {
    memcpy(rp, a->rp, sizeof(int) * (size_t)(a->nr + 1));
    memcpy(ci, a->ci, sizeof(int) * (size_t)a->nnz);
    memcpy(v, a->v, sizeof(double) * (size_t)a->nnz);
  }
  return OR_OK;
}
int or_get_ml(const or_hier* h, int l, double* out) {
  if (l >= 0 && l < h->nlev) { memcpy(out, h->lev[l].ML, sizeof(double) * (size_t)h->lev[l].N); return OR_OK; }
  if (l == h->nlev) { memcpy(out, h->ML1, sizeof(double) * (size_t)h->hl[0].N); return OR_OK; }
  return OR_ERR_ARG;
}
/* Switches the hierarchy's transfers to the consistent mass matrices (App. B):
 * assembles the interior mass matrix of every degree level and of V_{h,1}
 * (the quadrature of the lumped ones) and factors each by banded Cholesky. */
int or_use_consistent(or_hier* h) {
  int ne = 1 << h->k, st;
  for (int l = 0; l <= h->nlev; ++l) {
    int q = l < h->nlev ? h->lev[l].q : 1;
    slotmat m;
    csr M;
    st = assemble(h->dom, h->d, ne, q, q, K_MASS, 0, h->ex, &m);
    if (st) return st;
    st = slots_to_csr(&m, 1, &M);
    slot_free(&m);
    if (st) { csr_free(&M); return st; }
    if (l < h->nlev) st = band_cholesky(&M, &h->lev[l].mcb, &h->lev[l].MCB);
    else st = band_cholesky(&M, &h->mc1b, &h->MC1B);
    csr_free(&M);
    if (st) return st;
  }
  h->consistent = 1;
  return OR_OK;
}

int or_get_rhs(const or_hier* h, double* f) { memcpy(f, h->f, sizeof(double) * (size_t)h->lev[0].N); return OR_OK; }

/* step-level entry points (one hot-path row each) */
int or_residual(const or_hier* h, int l, const double* f, const double* u, double* r) {
  if (l < 0 || l >= h->nlev) return OR_ERR_ARG;
  residual(&h->lev[l].A, f, u, r); return OR_OK;
}
int or_smooth(const or_hier* h, int l, const double* f, double* u) {
  if (l < 0 || l >= h->nlev) return OR_ERR_ARG;
  ilut_smooth(&h->lev[l], f, u); return OR_OK;
}
int or_restrict(const or_hier* h, int l, const double* r, double* rc) {
  if (l < 0 || l >= h->nlev) return OR_ERR_ARG;
  restrict_(h, l, r, rc); return OR_OK;
}
int or_prolong_add(const or_hier* h, int l, const double* ec, double* u) {
  if (l < 0 || l >= h->nlev) return OR_ERR_ARG;
  prolong_add(h, l, ec, u); return OR_OK;
}
int or_coarse_solve(const or_hier* h, const double* r1, double* e1) { coarse_solve(h, r1, e1); return OR_OK; }
int or_hmg_vcycle(const or_hier* h, int j, const double* b, double* x) {
  if (j < 0 || j >= h->nh) return OR_ERR_ARG;
  hmg_vcycle(h, j, b, x); return OR_OK;
}
int or_gs(const or_hier* h, int j, int backward, const double* b, double* x) {
  if (j < 0 || j >= h->nh) return OR_ERR_ARG;
  if (backward) gs_backward(&h->hl[j].A, b, x); else gs_forward(&h->hl[j].A, b, x);
  return OR_OK;
}
int or_vcycle(const or_hier* h, int l, const double* f, double* u) {
  if (l < 0 || l >= h->nlev) return OR_ERR_ARG;
  vcycle(h, l, f, u); return OR_OK;
}

/* ILUT of a caller CSR matrix (tests: tau = 0 and unlimited fill = exact LU) */
int or_ilut(int n, const int* rp, const int* ci, const double* v, double tau, double fill,
            int* nl, int* nu, int* lrp, int* lci, double* lv, int* urp, int* uci, double* uv, int cap) {
  csr A = {n, n, rp[n], (int*)rp, (int*)ci, (double*)v};
  csr L, U;
  memset(&L, 0, sizeof L); memset(&U, 0, sizeof U);
  int st = ilut(&A, tau, fill, &L, &U);
  if (st) { csr_free(&L); csr_free(&U); return st; }
  *nl = L.nnz; *nu = U.nnz;
  if (L.nnz > cap || U.nnz > cap) { csr_free(&L); csr_free(&U); return OR_ERR_ARG; }
  memcpy(lrp, L.rp, sizeof(int) * (size_t)(n + 1)); memcpy(lci, L.ci, sizeof(int) * (size_t)L.nnz); memcpy(lv, L.v, sizeof(double) * (size_t)L.nnz);
  memcpy(urp, U.rp, sizeof(int) * (size_t)(n + 1)); memcpy(uci, U.ci, sizeof(int) * (size_t)U.nnz); memcpy(uv, U.v, sizeof(double) * (size_t)U.nnz);
  csr_free(&L); csr_free(&U);
  return OR_OK;
}

/* full-space (no elimination) matrices for the projection pins:
 * kind 0 stiffness, 1 mass; test degree q, trial degree r.  Two calls: sizes, then data. */
int or_full_matrix(int dom, int k, int q, int r, int kind, int* nr, int* nc, int* nnz, int* rp, int* ci, double* v) {
  int d = dom == OR_CUBE ? 3 : 2;
  slotmat s;
  int st = assemble(dom, d, 1 << k, q, r, kind, 0, 0, &s);
  if (st) return st;
  csr a;
  memset(&a, 0, sizeof a);
  st = slots_to_csr(&s, 0, &a);
  slot_free(&s);
  if (st) return st;
  *nr = a.nr; *nc = a.nc; *nnz = a.nnz;
  if (rp) {
    memcpy(rp, a.rp, sizeof(int) * (size_t)(a.nr + 1));
    memcpy(ci, a.ci, sizeof(int) * (size_t)a.nnz);
    memcpy(v, a.v, sizeof(double) * (size_t)a.nnz);
  }
  csr_free(&a);
  return OR_OK;
}

/* full-space load vector (no lift) for pins */
int or_full_load(int dom, int ex, int k, int q, double* out) {
  int d = dom == OR_CUBE ? 3 : 2;
  slotmat s;
  int st = assemble(dom, d, 1 << k, q, q, K_MASS, 1, ex, &s);
  if (st) return st;
  memcpy(out, s.load, sizeof(double) * (size_t)s.rows);
  slot_free(&s);
  return OR_OK;
}

/* L2 error of the discrete solution (interior coefficients u, boundary from the
 * lift) against the exact solution, (p+3)^d Gauss points per element (App. B). */
double or_l2_error(const or_hier* h, const double* u) {
  int d = h->d, p = h->p, ne = 1 << h->k, n = ne + p;
  long long Nfull = ipow(n, d);
  double* c = malloc(sizeof(double) * (size_t)Nfull);
  if (!c) return NAN;
  memcpy(c, h->uB, sizeof(double) * (size_t)Nfull);
  for (long long idx = 0; idx < Nfull; ++idx) {
    int m[3] = {0, 0, 0};
    unflat(idx, n, d, m);
    long long ii = interior_index(m, n, d);
    if (ii >= 0) c[idx] = u[ii];
  }
  int ng = p + 3;
  double gx[16], gw[16];
  or_gauss(ng, gx, gw);
  double err = 0.0;
  long long nel = ipow(ne, d), ngp = ipow(ng, d);
  int nloc = (int)ipow(p + 1, d);
  for (long long el = 0; el < nel; ++el) {
    int e[3] = {0, 0, 0};
    unflat(el, ne, d, e);
    for (long long gp = 0; gp < ngp; ++gp) {
      int g[3] = {0, 0, 0};
      unflat(gp, ng, d, g);
      double xi[3] = {0, 0, 0}, wt = 1.0;
      for (int a = 0; a < d; ++a) { xi[a] = ((double)e[a] + gx[g[a]]) / ne; wt *= gw[g[a]] / ne; }
      double X[3] = {0, 0, 0}, J[3][3], det;
      geo(h->dom, d, xi, X, J, &det);
      double uh = 0.0;
      for (int l = 0; l < nloc; ++l) {
        int a[3] = {0, 0, 0};
        unflat(l, p + 1, d, a);
        double val = 1.0; long long idx = 0;
        for (int c2 = 0; c2 < d; ++c2) val *= bspl(p, ne, e[c2] + a[c2], p, xi[c2]);
        for (int c2 = d - 1; c2 >= 0; --c2) idx = idx * n + (e[c2] + a[c2]);
        uh += c[idx] * val;
      }
      double diff = u_exact(h->dom, h->ex, d, X) - uh;
      err += wt * fabs(det) * diff * diff;
    }
  }
  free(c);
  return sqrt(err);
}
