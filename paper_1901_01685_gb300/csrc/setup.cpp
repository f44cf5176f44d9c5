// Host-side hierarchy construction (library side).  See setup.h.
//
// Compiled with -ffp-contract=off so that host arithmetic is identical on
// x86-64 and aarch64 builds.
#include "setup.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <queue>
#include <stdexcept>
#include <thread>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace pmgl {
namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;
using clk = std::chrono::steady_clock;
double ms_since(clk::time_point t0) {
  return std::chrono::duration<double, std::milli>(clk::now() - t0).count();
}

long long powi(long long b, int e) {
  long long r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// ---------------------------------------------------------------------------
// Univariate B-splines on the open uniform knot vector (Sec. 2): knots
// t_0 = ... = t_q = 0, t_{q+e} = e/ne, t_{ne+q} = ... = t_{ne+2q} = 1.
// ---------------------------------------------------------------------------
struct Knots {
  int q, ne;
  double t(int i) const {
    if (i <= q) return 0.0;
    if (i >= ne + q) return 1.0;
    return double(i - q) / double(ne);
  }
};

// All non-zero degree-`deg` functions of knot vector `K` on span s at x
// (functions s-deg .. s), by the triangular recurrence on left/right knot
// distances.  out has deg+1 entries.
void span_values(const Knots& K, int s, int deg, double x, double* out) {
  double left[16], right[16];
  out[0] = 1.0;
  for (int j = 1; j <= deg; ++j) {
    left[j] = x - K.t(s + 1 - j);
    right[j] = K.t(s + j) - x;
    double carry = 0.0;
    for (int r = 0; r < j; ++r) {
      double den = right[r + 1] + left[j - r];
      double tmp = out[r] / den;
      out[r] = carry + right[r + 1] * tmp;
      carry = left[j - r] * tmp;
    }
    out[j] = carry;
  }
}

// Values and first derivatives of the q+1 functions active on element e at
// parametric coordinate x (inside the element).
void element_basis(const Knots& K, int e, double x, double* val, double* der) {
  const int q = K.q, s = e + q;
  span_values(K, s, q, x, val);
  if (q == 0) { der[0] = 0.0; return; }
  double low[16];
  span_values(K, s, q - 1, x, low);  // functions s-q+1 .. s of degree q-1
  // derivative of function i = s-q+a: q N_{i,q-1}/(t_{i+q}-t_i) - q N_{i+1,q-1}/(t_{i+q+1}-t_{i+1})
  for (int a = 0; a <= q; ++a) {
    int i = s - q + a;
    double nl = (a >= 1) ? low[a - 1] : 0.0;   // N_{i,q-1}
    double nr = (a <= q - 1) ? low[a] : 0.0;   // N_{i+1,q-1}
    double d1 = K.t(i + q) - K.t(i), d2 = K.t(i + q + 1) - K.t(i + 1);
    double v = 0.0;
    if (d1 > 0.0) v += q * nl / d1;
    if (d2 > 0.0) v -= q * nr / d2;
    der[a] = v;
  }
}

// Gauss-Legendre nodes/weights on [0,1] by Newton's method on P_n.
void gauss_rule(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (4.0 * i + 3.0) / (4.0 * n + 2.0));
    double pn = 0.0, dpn = 1.0;
    for (int it = 0; it < 64; ++it) {
      double pm1 = 1.0;
      pn = z;
      for (int j = 1; j < n; ++j) {
        double pnext = (double(2 * j + 1) * z * pn - double(j) * pm1) / double(j + 1);
        pm1 = pn;
        pn = pnext;
      }
      if (n == 1) pm1 = 1.0;
      dpn = double(n) * (pm1 - z * pn) / (1.0 - z * z);
      double step = pn / dpn;
      z -= step;
      if (std::fabs(step) <= 1e-16) break;
    }
    double pm1 = 1.0;
    pn = z;
    for (int j = 1; j < n; ++j) {
      double pnext = (double(2 * j + 1) * z * pn - double(j) * pm1) / double(j + 1);
      pm1 = pn;
      pn = pnext;
    }
    if (n == 1) pm1 = 1.0;
    dpn = double(n) * (pm1 - z * pn) / (1.0 - z * z);
    int o = n - 1 - i;  // ascending order
    x[o] = 0.5 * (z + 1.0);
    w[o] = 1.0 / ((1.0 - z * z) * dpn * dpn);
  }
}

// ---------------------------------------------------------------------------
// Geometry (Sec. 2): quarter annulus 1 <= r <= 2 by the polar map, or the
// identity on the unit square / cube.
// ---------------------------------------------------------------------------
struct GeoPoint {
  double X[3];
  double Jinv[3][3];  // inverse Jacobian
  double absdet;
};

void map_point(int dom, int d, const double* xi, GeoPoint& g) {
  std::memset(&g, 0, sizeof(g));
  if (dom == PMG_QUARTER_ANNULUS) {
    const double r = 1.0 + xi[0], th = 0.5 * kPi * xi[1];
    const double c = std::cos(th), s = std::sin(th);
    g.X[0] = r * c;
    g.X[1] = r * s;
    // J = [[c, -r(pi/2)s], [s, r(pi/2)c]], det = r pi/2
    const double det = r * 0.5 * kPi;
    g.absdet = std::fabs(det);
    g.Jinv[0][0] = (r * 0.5 * kPi * c) / det;
    g.Jinv[0][1] = (r * 0.5 * kPi * s) / det;
    g.Jinv[1][0] = -s / det;
    g.Jinv[1][1] = c / det;
  } else {
    for (int a = 0; a < d; ++a) { g.X[a] = xi[a]; g.Jinv[a][a] = 1.0; }
    g.absdet = 1.0;
  }
}

double exact_u(int dom, int ex, int d, const double* X) {
  if (dom == PMG_QUARTER_ANNULUS && ex == PMG_U_PAPER_B1) {
    const double x = X[0], y = X[1], rr = x * x + y * y;
    return -(rr - 1.0) * (rr - 4.0) * x * y * y;
  }
  double v = 1.0;
  for (int a = 0; a < d; ++a) v *= std::sin(kPi * X[a]);
  return v;
}

// Benchmark 2 (Sec. 2): -div(D grad u) + v . grad u + R u on the unit square.
constexpr double kCdrD[2][2] = {{1.2, -0.7}, {-0.4, 0.9}};
constexpr double kCdrV[2] = {0.4, -0.2};
constexpr double kCdrR = 0.3;

// The PDE applied to the manufactured solutions (-Lap(u) for benchmarks 1 and 4).
double source_f(int dom, int ex, int d, const double* X) {
  if (dom == PMG_QUARTER_ANNULUS && ex == PMG_U_PAPER_B1) {
    const double x = X[0], y = X[1], x2 = x * x, y2 = y * y;
    return 2.0 * x * (x2 * x2 + 22.0 * x2 * y2 - 5.0 * x2 + 21.0 * y2 * y2 - 45.0 * y2 + 4.0);
  }
  if (dom == PMG_CDR_SQUARE) {
    // u = sin(pi x) sin(pi y): u_xx = u_yy = -pi^2 u, u_xy = pi^2 cos cos
    const double sx = std::sin(kPi * X[0]), sy = std::sin(kPi * X[1]);
    const double cx = std::cos(kPi * X[0]), cy = std::cos(kPi * X[1]);
    const double u = sx * sy, pi2 = kPi * kPi;
    return pi2 * (kCdrD[0][0] + kCdrD[1][1]) * u - pi2 * (kCdrD[0][1] + kCdrD[1][0]) * cx * cy +
           kPi * (kCdrV[0] * cx * sy + kCdrV[1] * sx * cy) + kCdrR * u;
  }
  double v = double(d) * kPi * kPi;
  for (int a = 0; a < d; ++a) v *= std::sin(kPi * X[a]);
  return v;
}

// ---------------------------------------------------------------------------
// Element-by-element Galerkin assembly into per-row offset slots.
// Row = full test-space function (degree q), slot = trial offset (degree r)
// relative to the row, per direction in [-q, r].
// ---------------------------------------------------------------------------
struct SlotMatrix {
  int d = 2, ne = 0, q = 0, r = 0, nq = 0, nr = 0, w = 0;
  long long rows = 0, slots = 0;
  std::vector<double> val;
  std::vector<double> load;
};

struct Tables1D {
  // [e][g][a]
  int ng = 0, nb = 0;
  std::vector<double> v, dv;
  void build(int q, int ne, int ng_, const double* gx) {
    ng = ng_;
    nb = q + 1;
    v.assign(size_t(ne) * ng * nb, 0.0);
    dv.assign(size_t(ne) * ng * nb, 0.0);
    Knots K{q, ne};
    for (int e = 0; e < ne; ++e)
      for (int g = 0; g < ng; ++g) {
        double x = (double(e) + gx[g]) / double(ne);
        element_basis(K, e, x, &v[(size_t(e) * ng + g) * nb], &dv[(size_t(e) * ng + g) * nb]);
      }
  }
  const double* val(int e, int g) const { return &v[(size_t(e) * ng + g) * nb]; }
  const double* der(int e, int g) const { return &dv[(size_t(e) * ng + g) * nb]; }
};

enum Form { kStiffness, kMass };

void assemble(int dom, int d, int ne, int q, int r, Form form, bool want_load, int ex, SlotMatrix& S) {
  S.d = d; S.ne = ne; S.q = q; S.r = r; S.nq = ne + q; S.nr = ne + r; S.w = q + r + 1;
  S.rows = powi(S.nq, d);
  S.slots = powi(S.w, d);
  S.val.assign(size_t(S.rows * S.slots), 0.0);
  if (want_load) S.load.assign(size_t(S.rows), 0.0);
  const int ng = std::max(q, r) + 1;
  double gx[16], gw[16];
  gauss_rule(ng, gx, gw);
  Tables1D Tq, Tr;
  Tq.build(q, ne, ng, gx);
  Tr.build(r, ne, ng, gx);
  const int nlq = int(powi(q + 1, d)), nlr = int(powi(r + 1, d));
  const long long ngp = powi(ng, d);
  // local -> (per-direction index) decode tables
  std::vector<int> locq(size_t(nlq) * 3, 0), locr(size_t(nlr) * 3, 0);
  for (int l = 0; l < nlq; ++l) { int t = l; for (int c = 0; c < d; ++c) { locq[l * 3 + c] = t % (q + 1); t /= (q + 1); } }
  for (int l = 0; l < nlr; ++l) { int t = l; for (int c = 0; c < d; ++c) { locr[l * 3 + c] = t % (r + 1); t /= (r + 1); } }
  // slot of (test local a, trial local b) = sum_c (b_c - a_c + q) w^c
  std::vector<long long> slot_ab(size_t(nlq) * nlr);
  for (int a = 0; a < nlq; ++a)
    for (int b = 0; b < nlr; ++b) {
      long long s = 0;
      for (int c = d - 1; c >= 0; --c) s = s * S.w + (locr[b * 3 + c] - locq[a * 3 + c] + q);
      slot_ab[size_t(a) * nlr + b] = s;
    }
  const int slow = d - 1;
  const int T = std::max(q, r) + 1;          // slab thickness (elements) in the slowest direction
  const int nslab = (ne + T - 1) / T;
  const long long per_slab_elems = powi(ne, d - 1);
  for (int color = 0; color < 2; ++color) {
#pragma omp parallel
    {
      std::vector<double> Ke(size_t(nlq) * nlr), Fe(nlq);
      std::vector<double> phq(nlq), phr(nlr), gq(size_t(nlq) * 3), gr(size_t(nlr) * 3);
#pragma omp for schedule(dynamic, 1)
      for (int sl = color; sl < nslab; sl += 2) {
        for (int es = sl * T; es < std::min(ne, (sl + 1) * T); ++es) {
          for (long long eo = 0; eo < per_slab_elems; ++eo) {
            int e[3] = {0, 0, 0};
            long long t = eo;
            for (int c = 0; c < slow; ++c) { e[c] = int(t % ne); t /= ne; }
            e[slow] = es;
            std::fill(Ke.begin(), Ke.end(), 0.0);
            if (want_load) std::fill(Fe.begin(), Fe.end(), 0.0);
            for (long long gp = 0; gp < ngp; ++gp) {
              int g[3] = {0, 0, 0};
              long long tt = gp;
              for (int c = 0; c < d; ++c) { g[c] = int(tt % ng); tt /= ng; }
              double xi[3] = {0, 0, 0}, wt = 1.0;
              for (int c = 0; c < d; ++c) { xi[c] = (double(e[c]) + gx[g[c]]) / double(ne); wt *= gw[g[c]] / double(ne); }
              GeoPoint G;
              map_point(dom, d, xi, G);
              const double dw = wt * G.absdet;
              // tensor-product values and physical gradients
              for (int side = 0; side < 2; ++side) {
                const Tables1D& Tb = side ? Tr : Tq;
                const int nl = side ? nlr : nlq;
                const std::vector<int>& loc = side ? locr : locq;
                double* ph = side ? phr.data() : phq.data();
                double* gg = side ? gr.data() : gq.data();
                for (int l = 0; l < nl; ++l) {
                  double vv = 1.0, gref[3] = {1.0, 1.0, 1.0};
                  for (int c = 0; c < d; ++c) {
                    const double bv = Tb.val(e[c], g[c])[loc[l * 3 + c]];
                    const double bd = Tb.der(e[c], g[c])[loc[l * 3 + c]];
                    vv *= bv;
                    for (int c2 = 0; c2 < d; ++c2) gref[c2] *= (c2 == c) ? bd : bv;
                  }
                  ph[l] = vv;
                  if (form == kStiffness)
                    for (int c = 0; c < d; ++c) {
                      double s = 0.0;
                      for (int c2 = 0; c2 < d; ++c2) s += G.Jinv[c2][c] * gref[c2];
                      gg[l * 3 + c] = s;
                    }
                }
              }
              if (form == kStiffness && dom == PMG_CDR_SQUARE) {
                // test a, trial b: (D grad phi_b) . grad phi_a + (v . grad phi_b) phi_a + R phi_b phi_a
                for (int a = 0; a < nlq; ++a) {
                  const double ga0 = dw * gq[a * 3 + 0], ga1 = dw * gq[a * 3 + 1], pa = dw * phq[a];
                  const double w0 = ga0 * kCdrD[0][0] + ga1 * kCdrD[1][0] + pa * kCdrV[0];
                  const double w1 = ga0 * kCdrD[0][1] + ga1 * kCdrD[1][1] + pa * kCdrV[1];
                  const double wr = pa * kCdrR;
                  double* row = &Ke[size_t(a) * nlr];
                  for (int b = 0; b < nlr; ++b) row[b] += w0 * gr[b * 3 + 0] + w1 * gr[b * 3 + 1] + wr * phr[b];
                }
              } else if (form == kStiffness) {
                for (int a = 0; a < nlq; ++a) {
                  const double g0 = dw * gq[a * 3 + 0], g1 = dw * gq[a * 3 + 1], g2 = dw * gq[a * 3 + 2];
                  double* row = &Ke[size_t(a) * nlr];
                  if (d == 2)
                    for (int b = 0; b < nlr; ++b) row[b] += g0 * gr[b * 3 + 0] + g1 * gr[b * 3 + 1];
                  else
                    for (int b = 0; b < nlr; ++b) row[b] += g0 * gr[b * 3 + 0] + g1 * gr[b * 3 + 1] + g2 * gr[b * 3 + 2];
                }
              } else {
                for (int a = 0; a < nlq; ++a) {
                  const double pa = dw * phq[a];
                  double* row = &Ke[size_t(a) * nlr];
                  for (int b = 0; b < nlr; ++b) row[b] += pa * phr[b];
                }
              }
              if (want_load) {
                const double fv = dw * source_f(dom, ex, d, G.X);
                for (int a = 0; a < nlq; ++a) Fe[a] += fv * phq[a];
              }
            }
            // scatter
            for (int a = 0; a < nlq; ++a) {
              long long row = 0;
              for (int c = d - 1; c >= 0; --c) row = row * S.nq + (e[c] + locq[a * 3 + c]);
              double* dst = &S.val[size_t(row * S.slots)];
              const double* src = &Ke[size_t(a) * nlr];
              const long long* sl_ab = &slot_ab[size_t(a) * nlr];
              for (int b = 0; b < nlr; ++b) dst[sl_ab[b]] += src[b];
              if (want_load) S.load[size_t(row)] += Fe[a];
            }
          }
        }
      }
    }
  }
}

// full-space multi-index helpers
inline void decode(long long idx, int n, int d, int* m) {
  for (int c = 0; c < d; ++c) { m[c] = int(idx % n); idx /= n; }
}
inline long long interior_of(const int* m, int n, int d) {
  long long idx = 0;
  for (int c = d - 1; c >= 0; --c) {
    if (m[c] <= 0 || m[c] >= n - 1) return -1;
    idx = idx * (n - 2) + (m[c] - 1);
  }
  return idx;
}

// Interior rows x interior columns of a slot matrix as CSR (columns ascending).
void interior_csr(const SlotMatrix& S, Csr& out) {
  const int d = S.d;
  const long long nri = powi(S.nq - 2, d), nci = powi(S.nr - 2, d);
  out.nr = int(nri);
  out.nc = int(nci);
  out.rp.assign(size_t(nri) + 1, 0);
  // offsets table per slot
  std::vector<int> off(size_t(S.slots) * 3, 0);
  for (long long s = 0; s < S.slots; ++s) {
    long long t = s;
    for (int c = 0; c < d; ++c) { off[s * 3 + c] = int(t % S.w) - S.q; t /= S.w; }
  }
  // count
  std::vector<long long> rowfull(static_cast<size_t>(nri));
  for (long long ri = 0; ri < nri; ++ri) {
    long long t = ri, row = 0;
    int m[3] = {0, 0, 0};
    for (int c = 0; c < d; ++c) { m[c] = int(t % (S.nq - 2)) + 1; t /= (S.nq - 2); }
    for (int c = d - 1; c >= 0; --c) row = row * S.nq + m[c];
    rowfull[ri] = row;
  }
  auto visit = [&](long long ri, auto&& emit) {
    int m[3] = {0, 0, 0};
    decode(rowfull[ri], S.nq, d, m);
    for (long long s = 0; s < S.slots; ++s) {
      int mj[3] = {0, 0, 0};
      bool inside = true;
      for (int c = 0; c < d && inside; ++c) {
        mj[c] = m[c] + off[s * 3 + c];
        if (mj[c] <= 0 || mj[c] >= S.nr - 1) inside = false;
      }
      if (!inside) continue;
      long long col = 0;
      for (int c = d - 1; c >= 0; --c) col = col * (S.nr - 2) + (mj[c] - 1);
      emit(int(col), S.val[size_t(rowfull[ri] * S.slots + s)]);
    }
  };
  for (long long ri = 0; ri < nri; ++ri) {
    int cnt = 0;
    visit(ri, [&](int, double) { ++cnt; });
    out.rp[ri + 1] = out.rp[ri] + cnt;
  }
  out.ci.resize(size_t(out.rp.back()));
  out.v.resize(size_t(out.rp.back()));
#pragma omp parallel for schedule(static)
  for (long long ri = 0; ri < nri; ++ri) {
    long long k = out.rp[ri];
    visit(ri, [&](int col, double v) { out.ci[k] = col; out.v[k] = v; ++k; });
  }
}

// Banded Cholesky factor of the interior 1D mass matrix of degree q on ne
// elements (q + 1 Gauss points an element, as for the level's operators),
// weighted by (1 + xi) when `weighted`, times `scale`.  The interior mass
// matrix of a level is the Kronecker product of such matrices (the quarter
// annulus' |det J| = (pi/2)(1 + xi) separates, the quadrature is a tensor
// rule), so its inverse is one banded solve per grid line and direction.
// F[i*(q+1)] = 1/L_ii, F[i*(q+1) + k] = L_{i,i-k} (0 where i - k < 0).
std::vector<double> mass_1d_factor(int ne, int q, bool weighted, double scale) {
  const int n = ne + q, ni = n - 2, ng = q + 1, w = q + 1;
  double gx[16], gw[16];
  gauss_rule(ng, gx, gw);
  Tables1D T;
  T.build(q, ne, ng, gx);
  std::vector<double> M(size_t(std::max(ni, 0)) * w, 0.0);   // M[i][k] = m(i, i - k), interior indices
  for (int e = 0; e < ne; ++e)
    for (int g = 0; g < ng; ++g) {
      const double x = (double(e) + gx[g]) / double(ne);
      const double wt = gw[g] / double(ne) * (weighted ? 1.0 + x : 1.0) * scale;
      const double* B = T.val(e, g);
      for (int a = 0; a <= q; ++a)
        for (int b = 0; b <= a; ++b) {
          const int i = e + a - 1, j = e + b - 1;      // interior indices (full index - 1)
          if (i < 0 || j < 0 || i >= ni || j >= ni) continue;
          M[size_t(i) * w + size_t(i - j)] += wt * B[a] * B[b];
        }
    }
  std::vector<double> F(M.size(), 0.0);
  for (int i = 0; i < ni; ++i) {
    for (int k = std::min(q, i); k >= 1; --k) {        // L_{i,j}, j = i - k, in increasing j
      const int j = i - k;
      double s = M[size_t(i) * w + size_t(k)];
      for (int l = std::max(0, i - q); l < j; ++l) s -= F[size_t(i) * w + size_t(i - l)] * F[size_t(j) * w + size_t(j - l)];
      F[size_t(i) * w + size_t(k)] = s * F[size_t(j) * w];   // times 1/L_jj
    }
    double s = M[size_t(i) * w];
    for (int l = std::max(0, i - q); l < i; ++l) s -= F[size_t(i) * w + size_t(i - l)] * F[size_t(i) * w + size_t(i - l)];
    F[size_t(i) * w] = 1.0 / std::sqrt(s);
  }
  return F;
}

// ∫ Phi_i dOmega for the interior functions of degree q (= lumped mass row sums).
std::vector<double> lumped_mass(int dom, int d, int ne, int q) {
  const int n = ne + q, ng = q + 1;
  double gx[16], gw[16];
  gauss_rule(ng, gx, gw);
  Tables1D Tq;
  Tq.build(q, ne, ng, gx);
  std::vector<double> full(size_t(powi(n, d)), 0.0);
  const long long nel = powi(ne, d), ngp = powi(ng, d);
  const int nl = int(powi(q + 1, d));
  for (long long el = 0; el < nel; ++el) {
    int e[3] = {0, 0, 0};
    decode(el, ne, d, e);
    for (long long gp = 0; gp < ngp; ++gp) {
      int g[3] = {0, 0, 0};
      decode(gp, ng, d, g);
      double xi[3] = {0, 0, 0}, wt = 1.0;
      for (int c = 0; c < d; ++c) { xi[c] = (double(e[c]) + gx[g[c]]) / double(ne); wt *= gw[g[c]] / double(ne); }
      GeoPoint G;
      map_point(dom, d, xi, G);
      for (int l = 0; l < nl; ++l) {
        int a[3] = {0, 0, 0};
        decode(l, q + 1, d, a);
        double v = wt * G.absdet;
        long long idx = 0;
        for (int c = 0; c < d; ++c) v *= Tq.val(e[c], g[c])[a[c]];
        for (int c = d - 1; c >= 0; --c) idx = idx * n + (e[c] + a[c]);
        full[size_t(idx)] += v;
      }
    }
  }
  std::vector<double> out(size_t(powi(n - 2, d)));
  for (long long idx = 0; idx < (long long)full.size(); ++idx) {
    int m[3] = {0, 0, 0};
    decode(idx, n, d, m);
    long long ii = interior_of(m, n, d);
    if (ii >= 0) out[size_t(ii)] = full[size_t(idx)];
  }
  return out;
}

// Symmetric positive definite banded solve (Cholesky), half bandwidth bw.
void band_spd_solve(int n, int bw, std::vector<double>& B /* n x (bw+1), B[i][k] = a(i, i-k) */, std::vector<double>& x) {
  auto at = [&](int i, int k) -> double& { return B[size_t(i) * (bw + 1) + k]; };
  for (int i = 0; i < n; ++i) {
    for (int k = std::min(bw, i); k >= 1; --k) {
      int j = i - k;
      double s = at(i, k);
      for (int m = k + 1; m <= std::min(bw, i); ++m) {
        int jj = m - k;  // column i-m relative to row j: j - (i-m) = m - k
        if (jj <= bw) s -= at(i, m) * at(j, jj);
      }
      at(i, k) = s / at(j, 0);
    }
    double s = at(i, 0);
    for (int m = 1; m <= std::min(bw, i); ++m) s -= at(i, m) * at(i, m);
    at(i, 0) = std::sqrt(s);
  }
  for (int i = 0; i < n; ++i) {
    double s = x[i];
    for (int m = 1; m <= std::min(bw, i); ++m) s -= at(i, m) * x[i - m];
    x[i] = s / at(i, 0);
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int m = 1; m <= bw && i + m < n; ++m) s -= at(i + m, m) * x[i + m];
    x[i] = s / at(i, 0);
  }
}

// Dirichlet lift coefficients (full space, degree q).  Non-zero data only on
// the annulus arcs for the sin-product solution: the interior edge
// coefficients are the 1-D L2 projection of the data in the parametric
// measure, the corner values (on the straight edges) are 0.
std::vector<double> dirichlet_lift(int dom, int ex, int d, int ne, int q) {
  const int n = ne + q;
  std::vector<double> uB(size_t(powi(n, d)), 0.0);
  if (!(dom == PMG_QUARTER_ANNULUS && ex == PMG_U_SINPROD)) return uB;
  const int m = n - 2, ng = q + 1;
  double gx[16], gw[16];
  gauss_rule(ng, gx, gw);
  Tables1D T;
  T.build(q, ne, ng, gx);
  std::vector<double> band(size_t(m) * (q + 1), 0.0);
  for (int e = 0; e < ne; ++e)
    for (int g = 0; g < ng; ++g) {
      const double* v = T.val(e, g);
      const double wt = gw[g] / double(ne);
      for (int a = 0; a <= q; ++a)
        for (int b = 0; b <= a; ++b) {
          int i = e + a, j = e + b;  // j <= i
          if (i < 1 || i > n - 2 || j < 1 || j > n - 2) continue;
          band[size_t(i - 1) * (q + 1) + (i - j)] += wt * v[a] * v[b];
        }
    }
  for (int side = 0; side < 2; ++side) {
    std::vector<double> B = band, rhs(size_t(m), 0.0);
    for (int e = 0; e < ne; ++e)
      for (int g = 0; g < ng; ++g) {
        const double s = (double(e) + gx[g]) / double(ne);
        double xi[3] = {double(side), s, 0.0};
        GeoPoint G;
        map_point(dom, d, xi, G);
        const double gval = exact_u(dom, ex, d, G.X) * gw[g] / double(ne);
        const double* v = T.val(e, g);
        for (int a = 0; a <= q; ++a) {
          int i = e + a;
          if (i >= 1 && i <= n - 2) rhs[i - 1] += gval * v[a];
        }
      }
    band_spd_solve(m, q, B, rhs);
    const int ix = side ? n - 1 : 0;
    for (int iy = 1; iy <= n - 2; ++iy) uB[size_t(ix) + size_t(n) * iy] = rhs[iy - 1];
  }
  return uB;
}

// ---------------------------------------------------------------------------
// Dual-threshold ILUT (Sec. 3 "Smoother"): row-wise incomplete elimination;
// multipliers below tau_i are dropped; afterwards entries below tau_i are
// dropped and only the M largest remain in the lower and in the upper part.
// tau_i = tau * mean |a_ij| of the original row; M = ceil(m * nnz(A) / N).
// Selection of the M largest: entries above t(1+1e-12) (t = M-th largest
// magnitude), then ties within [t(1-1e-12), t(1+1e-12)] by ascending column.
// ---------------------------------------------------------------------------
int row_budget(long long nnz, int n, double m) {
  double b = std::ceil(m * double(nnz) / double(n));
  if (b > double(n)) b = double(n);
  if (b < 0.0) b = 0.0;
  return int(b);
}

void select_largest(std::vector<std::pair<int, double>>& c, int M) {
  if (int(c.size()) > M) {
    auto mag_greater = [](const std::pair<int, double>& a, const std::pair<int, double>& b) {
      const double ma = std::fabs(a.second), mb = std::fabs(b.second);
      return ma > mb || (ma == mb && a.first < b.first);
    };
    std::nth_element(c.begin(), c.begin() + (M - 1), c.end(), mag_greater);
    const double t = std::fabs(c[M - 1].second);
    const double hi = t * (1.0 + 1e-12), lo = t * (1.0 - 1e-12);
    std::vector<std::pair<int, double>> keep, tie;
    keep.reserve(M);
    for (const auto& e : c) {
      const double a = std::fabs(e.second);
      if (a > hi) keep.push_back(e);
      else if (a >= lo) tie.push_back(e);
    }
    std::sort(tie.begin(), tie.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
    for (size_t s = 0; s < tie.size() && int(keep.size()) < M; ++s) keep.push_back(tie[s]);
    c.swap(keep);
  }
  std::sort(c.begin(), c.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
}

pmg_status ilut_factor(const Csr& A, double tau, double m, Csr& L, Csr& U, std::vector<double>& udiag, std::string& err) {
  const int n = A.nr;
  const int M = row_budget(A.nnz(), n, m);
  L = Csr{}; U = Csr{};
  L.nr = L.nc = U.nr = U.nc = n;
  L.rp.assign(size_t(n) + 1, 0);
  U.rp.assign(size_t(n) + 1, 0);
  udiag.assign(size_t(n), 0.0);
  std::vector<double> w(size_t(n), 0.0);
  std::vector<int> mark(size_t(n), -1);     // row stamp: mark[j] == i <=> j in the pattern of w
  std::vector<int> pat;
  pat.reserve(4096);
  std::priority_queue<int, std::vector<int>, std::greater<int>> pending;   // lower columns to eliminate
  std::vector<std::pair<int, double>> lowc, upc;
  for (int i = 0; i < n; ++i) {
    pat.clear();
    double asum = 0.0;
    const int beg = A.rp[i], end = A.rp[i + 1];
    for (int t = beg; t < end; ++t) {
      const int j = A.ci[t];
      w[j] = A.v[t];
      mark[j] = i;
      pat.push_back(j);
      asum += std::fabs(A.v[t]);
      if (j < i) pending.push(j);
    }
    const double tol = (end > beg) ? tau * asum / double(end - beg) : 0.0;
    while (!pending.empty()) {
      const int k = pending.top();
      pending.pop();
      if (w[k] == 0.0) continue;
      const double lk = w[k] / udiag[k];
      if (std::fabs(lk) < tol) { w[k] = 0.0; continue; }
      w[k] = lk;
      for (int t = U.rp[k]; t < U.rp[k + 1]; ++t) {
        const int j = U.ci[t];
        if (mark[j] != i) {
          mark[j] = i;
          w[j] = 0.0;
          pat.push_back(j);
          if (j < i) pending.push(j);
        }
        w[j] -= lk * U.v[t];
      }
    }
    lowc.clear();
    upc.clear();
    double dg = 0.0;
    for (int j : pat) {
      const double v = w[j];
      if (j == i) { dg = v; continue; }
      if (v == 0.0 || std::fabs(v) < tol) continue;
      (j < i ? lowc : upc).emplace_back(j, v);
    }
    select_largest(lowc, M);
    select_largest(upc, M);
    if (dg == 0.0) {
      err = "ILUT: zero pivot in row " + std::to_string(i);
      return PMG_ERR_ZERO_PIVOT;
    }
    udiag[i] = dg;
    for (const auto& e : lowc) { L.ci.push_back(e.first); L.v.push_back(e.second); }
    for (const auto& e : upc) { U.ci.push_back(e.first); U.v.push_back(e.second); }
    L.rp[i + 1] = int(L.ci.size());
    U.rp[i + 1] = int(U.ci.size());
    for (int j : pat) w[j] = 0.0;
  }
  return PMG_OK;
}

Csr transpose(const Csr& a) {
  Csr t;
  t.nr = a.nc; t.nc = a.nr;
  t.rp.assign(size_t(t.nr) + 1, 0);
  for (int c : a.ci) t.rp[c + 1]++;
  for (int i = 0; i < t.nr; ++i) t.rp[i + 1] += t.rp[i];
  t.ci.resize(a.ci.size());
  t.v.resize(a.v.size());
  std::vector<int> fill(t.rp.begin(), t.rp.end() - 1);
  for (int i = 0; i < a.nr; ++i)
    for (int k = a.rp[i]; k < a.rp[i + 1]; ++k) {
      const int c = a.ci[k];
      t.ci[fill[c]] = i;
      t.v[fill[c]] = a.v[k];
      fill[c]++;
    }
  return t;
}

Csr scale_rows(const Csr& a, const std::vector<double>& by) {
  Csr s = a;
  for (int i = 0; i < s.nr; ++i)
    for (int k = s.rp[i]; k < s.rp[i + 1]; ++k) s.v[k] = a.v[k] / by[i];
  return s;
}

// Dense inverse by Gauss-Jordan elimination with partial pivoting.
bool dense_inverse(int n, std::vector<double> a, std::vector<double>& inv) {
  inv.assign(size_t(n) * n, 0.0);
  for (int i = 0; i < n; ++i) inv[size_t(i) * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[size_t(r) * n + c]) > std::fabs(a[size_t(piv) * n + c])) piv = r;
    if (a[size_t(piv) * n + c] == 0.0) return false;
    if (piv != c)
      for (int j = 0; j < n; ++j) {
        std::swap(a[size_t(c) * n + j], a[size_t(piv) * n + j]);
        std::swap(inv[size_t(c) * n + j], inv[size_t(piv) * n + j]);
      }
    const double dinv = 1.0 / a[size_t(c) * n + c];
    for (int j = 0; j < n; ++j) { a[size_t(c) * n + j] *= dinv; inv[size_t(c) * n + j] *= dinv; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = a[size_t(r) * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        a[size_t(r) * n + j] -= f * a[size_t(c) * n + j];
        inv[size_t(r) * n + j] -= f * inv[size_t(c) * n + j];
      }
    }
  }
  return true;
}

}  // namespace

Csr mirror(const Csr& a) {
  Csr m;
  m.nr = a.nr;
  m.nc = a.nc;
  m.rp.assign(size_t(a.nr) + 1, 0);
  m.ci.reserve(a.ci.size());
  m.v.reserve(a.v.size());
  for (int r = 0; r < a.nr; ++r) {
    const int i = a.nr - 1 - r;
    for (int t = a.rp[i + 1] - 1; t >= a.rp[i]; --t) {
      m.ci.push_back(a.nc - 1 - a.ci[t]);
      m.v.push_back(a.v[t]);
    }
    m.rp[size_t(r) + 1] = int(m.ci.size());
  }
  return m;
}

std::vector<int> line_split(const Csr& a, int nx) {
  std::vector<int> sp(size_t(a.nr));
  for (int i = 0; i < a.nr; ++i) {
    const int line_start = (i / nx) * nx;
    int t = a.rp[i];
    while (t < a.rp[i + 1] && a.ci[t] < line_start) ++t;
    sp[size_t(i)] = t;
  }
  return sp;
}

Csr strict_part(const Csr& a, bool lower) {
  Csr s;
  s.nr = a.nr;
  s.nc = a.nc;
  s.rp.assign(size_t(a.nr) + 1, 0);
  for (int i = 0; i < a.nr; ++i) {
    for (int t = a.rp[i]; t < a.rp[i + 1]; ++t) {
      const int j = a.ci[t];
      if (lower ? j < i : j > i) { s.ci.push_back(j); s.v.push_back(a.v[t]); }
    }
    s.rp[size_t(i) + 1] = int(s.ci.size());
  }
  return s;
}

LpLayout build_lp(const Csr& M, int nx, const std::vector<double>* dinv, int win, int lpr) {
  LpLayout P;
  P.lpr = lpr;
  P.win = win;
  const int lanes = win * lpr;
  P.n = M.nr;
  P.nx = nx;
  P.nlines = M.nr / nx;
  P.nwin = (nx + win - 1) / win;
  const int n = M.nr;
  P.dscale.assign(size_t(n), 1.0);
  if (dinv) {
    // the mirrored factors are stored in the solve's index space; dinv is given in it too
    for (int i = 0; i < n; ++i) P.dscale[size_t(i)] = (*dinv)[size_t(i)];
  }
  P.push.assign(size_t(n) * 32, 0.0);
  const int nwin_total = P.nlines * P.nwin;
  P.wofs.assign(size_t(nwin_total) + 1, 0);
  P.waitofs.assign(size_t(nwin_total) + 1, 0);
  std::vector<std::vector<int>> far(static_cast<size_t>(lanes));
  std::vector<std::vector<double>> farv(static_cast<size_t>(lanes));
  for (int ln = 0; ln < P.nlines; ++ln) {
    for (int w = 0; w < P.nwin; ++w) {
      const int W = ln * P.nwin + w;
      for (auto& f : far) f.clear();
      for (auto& f : farv) f.clear();
      // per referenced line distance: rows needed
      std::vector<std::pair<int, int>> need;  // (distance, need)
      auto add_need = [&](int dist, int local) {
        for (auto& q : need)
          if (q.first == dist) { q.second = std::max(q.second, local + 1); return; }
        need.emplace_back(dist, local + 1);
      };
      for (int r = 0; r < win; ++r) {
        const int ix = w * win + r;
        if (ix >= nx) break;
        const int i = ln * nx + ix;
        const int line_start = ln * nx;
        int cnt = 0;
        for (int t = M.rp[i]; t < M.rp[i + 1]; ++t) {
          const int j = M.ci[t];
          const int k = i - j;
          if (j >= line_start && k <= 31) {
            P.push[size_t(j) * 32 + (k - 1)] = M.v[t] * P.dscale[size_t(i)];
            ++P.ring_entries;
            continue;
          }
          const int jl = j / nx;
          add_need(ln - jl, j - jl * nx);
          const int lane = lpr * r + (cnt % lpr);
          far[size_t(lane)].push_back(j);
          farv[size_t(lane)].push_back(M.v[t] * P.dscale[size_t(i)]);
          ++cnt;
          ++P.far_entries;
        }
      }
      size_t K = 0;
      for (auto& f : far) K = std::max(K, f.size());
      P.wofs[size_t(W) + 1] = P.wofs[size_t(W)] + int(lanes * K);
      for (size_t k = 0; k < K; ++k)
        for (int l = 0; l < lanes; ++l) {
          const bool has = k < far[size_t(l)].size();
          P.wcol.push_back(has ? far[size_t(l)][k] : -1);
          P.wval.push_back(has ? farv[size_t(l)][k] : 0.0);
        }
      std::sort(need.begin(), need.end());
      for (auto& q : need) { P.wait.push_back(q.first); P.wait.push_back(q.second); }
      P.waitofs[size_t(W) + 1] = int(P.wait.size() / 2);
    }
  }
  if (P.wcol.empty()) { P.wcol.push_back(-1); P.wval.push_back(0.0); }
  if (P.wait.empty()) { P.wait.push_back(0); P.wait.push_back(0); }
  return P;
}

Csr far_part(const Csr& M, int nx, const std::vector<double>& dscale, int ring) {
  Csr F;
  F.nr = F.nc = M.nr;
  F.rp.assign(size_t(M.nr) + 1, 0);
  for (int i = 0; i < M.nr; ++i) {
    const int line_start = (i / nx) * nx;
    for (int t = M.rp[i]; t < M.rp[i + 1]; ++t) {
      const int j = M.ci[t];
      if (j >= line_start && i - j < ring) continue;
      F.ci.push_back(j);
      F.v.push_back(M.v[t] * dscale[size_t(i)]);
    }
    F.rp[size_t(i) + 1] = int(F.ci.size());
  }
  return F;
}

int critical_path(const Csr& T, bool lower) {
  const int n = T.nr;
  std::vector<int> lvl(size_t(n), 0);
  int depth = 0;
  if (lower) {
    for (int i = 0; i < n; ++i) {
      int l = 0;
      for (int k = T.rp[i]; k < T.rp[i + 1]; ++k)
        if (T.ci[k] < i) l = std::max(l, lvl[T.ci[k]] + 1);
      lvl[i] = l;
      depth = std::max(depth, l + 1);
    }
  } else {
    for (int i = n - 1; i >= 0; --i) {
      int l = 0;
      for (int k = T.rp[i]; k < T.rp[i + 1]; ++k)
        if (T.ci[k] > i) l = std::max(l, lvl[T.ci[k]] + 1);
      lvl[i] = l;
      depth = std::max(depth, l + 1);
    }
  }
  return depth;
}

pmg_status build_hierarchy(int dom, int p, int k, const pmg_options& opt, Hierarchy& H, std::string& err) {
  if (dom < 0 || dom > 3) { err = "unknown domain"; return PMG_ERR_ARG; }
  if (p < 2 || p > 8) { err = "p must be in [2, 8]"; return PMG_ERR_ARG; }
  if (k < 3 || k > 12 || (dom == PMG_UNIT_CUBE && k > 6)) { err = "log2_inv_h out of range"; return PMG_ERR_ARG; }
  if (opt.coarse_cycles < 1 || opt.nu_pre < 0 || opt.nu_post < 0 || opt.drop_tol < 0 || opt.fill_factor <= 0 ||
      (opt.projection != PMG_PROJ_INDIRECT && opt.projection != PMG_PROJ_DIRECT) || opt.exact < 0 || opt.exact > 1) {
    err = "invalid options";
    return PMG_ERR_ARG;
  }
  H = Hierarchy{};
  H.dom = dom; H.p = p; H.k = k; H.opt = opt;
  H.d = (dom == PMG_UNIT_CUBE) ? 3 : 2;
  const int d = H.d, ne = 1 << k;
  const int nlev = (opt.projection == PMG_PROJ_DIRECT) ? 1 : p - 1;
  H.lev.resize(size_t(nlev));
  std::vector<std::thread> workers;
  struct JoinAll {   // every exit path waits for the level threads
    std::vector<std::thread>& t;
    ~JoinAll() { for (auto& x : t) if (x.joinable()) x.join(); }
  } join_all{workers};
  std::vector<pmg_status> wst(static_cast<size_t>(nlev), PMG_OK);
  std::vector<std::string> werr(static_cast<size_t>(nlev));
  std::vector<double> wms(static_cast<size_t>(nlev), 0.0);
  try {
    for (int l = 0; l < nlev; ++l) {
      PLevel& L = H.lev[size_t(l)];
      L.q = p - l;
      L.n1d = ne + L.q - 2;
      L.N = int(powi(L.n1d, d));
      auto t0 = clk::now();
      SlotMatrix S;
      assemble(dom, d, ne, L.q, L.q, kStiffness, l == 0, opt.exact, S);
      interior_csr(S, L.A);
      if (l == 0) {
        H.uB = (d == 2) ? dirichlet_lift(dom, opt.exact, d, ne, L.q) : std::vector<double>(size_t(powi(ne + L.q, d)), 0.0);
        const int n = ne + L.q;
        H.f.assign(size_t(L.N), 0.0);
        for (long long row = 0; row < S.rows; ++row) {
          int m[3] = {0, 0, 0};
          decode(row, n, d, m);
          long long ii = interior_of(m, n, d);
          if (ii < 0) continue;
          double acc = S.load[size_t(row)];
          for (long long s = 0; s < S.slots; ++s) {
            long long t = s, col = 0;
            int mj[3] = {0, 0, 0};
            bool ok = true;
            for (int c = 0; c < d; ++c) { mj[c] = m[c] + int(t % S.w) - L.q; t /= S.w; if (mj[c] < 0 || mj[c] >= n) ok = false; }
            if (!ok || interior_of(mj, n, d) >= 0) continue;
            for (int c = d - 1; c >= 0; --c) col = col * n + mj[c];
            const double ub = H.uB[size_t(col)];
            if (ub != 0.0) acc -= S.val[size_t(row * S.slots + s)] * ub;
          }
          H.f[size_t(ii)] = acc;
        }
      }
      L.ML = lumped_mass(dom, d, ne, L.q);
      H.t_assembly += ms_since(t0);
      // The ILUT factor of each level (a sequential row recurrence) and its
      // solve layouts run on a thread of their own while the next level is
      // assembled; every thread writes only its own level.
      workers.emplace_back([&, l] {
        PLevel& Lw = H.lev[size_t(l)];
        const auto tw = clk::now();
        try {
          wst[size_t(l)] = ilut_factor(Lw.A, opt.drop_tol, opt.fill_factor, Lw.L, Lw.U, Lw.udiag, werr[size_t(l)]);
          if (wst[size_t(l)] != PMG_OK) return;
          Lw.depthL = critical_path(Lw.L, true);
          Lw.depthU = critical_path(Lw.U, false);
          Lw.Lsplit = line_split(Lw.L, Lw.n1d);
          Lw.Um = mirror(Lw.U);
          Lw.Umsplit = line_split(Lw.Um, Lw.n1d);
          Lw.Llp = build_lp(Lw.L, Lw.n1d, nullptr, 4, 8);
          std::vector<double> ud(size_t(Lw.N));
          for (int i = 0; i < Lw.N; ++i) ud[size_t(i)] = 1.0 / Lw.udiag[size_t(Lw.N - 1 - i)];
          Lw.Ulp = build_lp(Lw.Um, Lw.n1d, &ud, 4, 8);
        } catch (const std::bad_alloc&) {
          wst[size_t(l)] = PMG_ERR_OOM;
          werr[size_t(l)] = "host allocation failed";
        }
        wms[size_t(l)] = ms_since(tw);
      });
    }
    for (auto& w : workers) w.join();
    workers.clear();
    for (int l = 0; l < nlev; ++l) {
      H.t_ilut = std::max(H.t_ilut, wms[size_t(l)]);     // concurrent: the longest level
      if (wst[size_t(l)] != PMG_OK) {
        err = werr[size_t(l)];
        return wst[size_t(l)];
      }
    }
    auto t0 = clk::now();
    H.ML1 = lumped_mass(dom, d, ne, 1);
    for (int l = 0; l < nlev; ++l) {
      PLevel& L = H.lev[size_t(l)];
      const int qc = (l + 1 < nlev) ? L.q - 1 : 1;
      SlotMatrix S;
      assemble(dom, d, ne, L.q, qc, kMass, false, opt.exact, S);
      interior_csr(S, L.Praw);
      const std::vector<double>& MLc = (l + 1 < nlev) ? H.lev[size_t(l + 1)].ML : H.ML1;
      if (opt.transfer_mass == PMG_MASS_CONSISTENT) {   // M^{-1} applied by line solves after the product
        L.Pro = L.Praw;
        L.Res = transpose(L.Praw);
      } else {
        L.Pro = scale_rows(L.Praw, L.ML);
        L.Res = scale_rows(transpose(L.Praw), MLc);
      }
    }
    if (opt.transfer_mass == PMG_MASS_CONSISTENT) {
      const bool ann = dom == PMG_QUARTER_ANNULUS;
      const double pi = 3.14159265358979323846;
      for (auto& L : H.lev) {
        L.MF0 = mass_1d_factor(ne, L.q, ann, ann ? 0.5 * pi : 1.0);
        L.MF1 = ann ? mass_1d_factor(ne, L.q, false, 1.0) : L.MF0;
      }
      H.M1F0 = mass_1d_factor(ne, 1, ann, ann ? 0.5 * pi : 1.0);
      H.M1F1 = ann ? mass_1d_factor(ne, 1, false, 1.0) : H.M1F0;
    }
    H.t_transfer += ms_since(t0);
    t0 = clk::now();
    const int nh = k - 3 + 1;
    H.hl.resize(size_t(nh));
    for (int j = 0; j < nh; ++j) {
      HLevel& Hl = H.hl[size_t(j)];
      Hl.ne = ne >> j;
      Hl.n1d = Hl.ne - 1;
      Hl.N = int(powi(Hl.n1d, d));
      SlotMatrix S;
      assemble(dom, d, Hl.ne, 1, 1, kStiffness, false, opt.exact, S);
      interior_csr(S, Hl.A);
      Hl.dinv.assign(size_t(Hl.N), 0.0);
      for (int i = 0; i < Hl.N; ++i)
        for (int t = Hl.A.rp[i]; t < Hl.A.rp[i + 1]; ++t)
          if (Hl.A.ci[t] == i) Hl.dinv[size_t(i)] = 1.0 / Hl.A.v[t];
      Hl.depthGS = critical_path(Hl.A, true);
      Hl.Lo = strict_part(Hl.A, true);
      Hl.Up = strict_part(Hl.A, false);
      Hl.UpM = mirror(Hl.Up);
      Hl.Losplit = line_split(Hl.Lo, Hl.n1d);
      Hl.UpMsplit = line_split(Hl.UpM, Hl.n1d);
      Hl.Lolp = build_lp(Hl.Lo, Hl.n1d, &Hl.dinv, 4, 4);
      {
        std::vector<double> dm(size_t(Hl.N));
        for (int i = 0; i < Hl.N; ++i) dm[size_t(i)] = Hl.dinv[size_t(Hl.N - 1 - i)];
        Hl.UpMlp = build_lp(Hl.UpM, Hl.n1d, &dm, 4, 4);
      }
    }
    {
      const HLevel& C = H.hl.back();
      std::vector<double> dense(size_t(C.N) * C.N, 0.0);
      for (int i = 0; i < C.N; ++i)
        for (int t = C.A.rp[i]; t < C.A.rp[i + 1]; ++t) dense[size_t(i) * C.N + C.A.ci[t]] = C.A.v[t];
      if (!dense_inverse(C.N, dense, H.coarse_inv)) { err = "singular coarsest operator"; return PMG_ERR_ZERO_PIVOT; }
    }
    H.t_hmg += ms_since(t0);
  } catch (const std::bad_alloc&) {
    err = "host allocation failed during setup";
    return PMG_ERR_OOM;
  }
  return PMG_OK;
}

double l2_error(const Hierarchy& H, const double* u) {
  const int d = H.d, p = H.p, ne = 1 << H.k, n = ne + p;
  std::vector<double> c = H.uB;
  for (long long idx = 0; idx < (long long)c.size(); ++idx) {
    int m[3] = {0, 0, 0};
    decode(idx, n, d, m);
    long long ii = interior_of(m, n, d);
    if (ii >= 0) c[size_t(idx)] = u[ii];
  }
  const int ng = p + 3;
  double gx[16], gw[16];
  gauss_rule(ng, gx, gw);
  Tables1D T;
  T.build(p, ne, ng, gx);
  const long long nel = powi(ne, d), ngp = powi(ng, d);
  const int nl = int(powi(p + 1, d));
  double err = 0.0;
#pragma omp parallel for reduction(+ : err) schedule(static)
  for (long long el = 0; el < nel; ++el) {
    int e[3] = {0, 0, 0};
    decode(el, ne, d, e);
    for (long long gp = 0; gp < ngp; ++gp) {
      int g[3] = {0, 0, 0};
      decode(gp, ng, d, g);
      double xi[3] = {0, 0, 0}, wt = 1.0;
      for (int cc = 0; cc < d; ++cc) { xi[cc] = (double(e[cc]) + gx[g[cc]]) / double(ne); wt *= gw[g[cc]] / double(ne); }
      GeoPoint G;
      map_point(H.dom, d, xi, G);
      double uh = 0.0;
      for (int l = 0; l < nl; ++l) {
        int a[3] = {0, 0, 0};
        decode(l, p + 1, d, a);
        double v = 1.0;
        long long idx = 0;
        for (int cc = 0; cc < d; ++cc) v *= T.val(e[cc], g[cc])[a[cc]];
        for (int cc = d - 1; cc >= 0; --cc) idx = idx * n + (e[cc] + a[cc]);
        uh += v * c[size_t(idx)];
      }
      const double diff = exact_u(H.dom, H.opt.exact, d, G.X) - uh;
      err += wt * G.absdet * diff * diff;
    }
  }
  return std::sqrt(err);
}

}  // namespace pmgl
