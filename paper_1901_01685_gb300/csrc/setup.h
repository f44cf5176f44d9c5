// Host-side construction of the p-multigrid hierarchy (library side).
//
// Everything here runs once per hierarchy on the host: IgA assembly with Gauss
// quadrature (Sec. 2), the dual-threshold ILUT factors (Sec. 3 "Smoother"), the
// lumped L2-projection transfer operators (Sec. 3 "Prolongation and
// restriction", Eq. PM) and the rediscretised p = 1 h-multigrid levels
// (Sec. 3, Fig. 1).  The V-cycle itself runs on the GPU (pmg.cu).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pmg.h"

namespace pmgl {

struct Csr {
  int nr = 0, nc = 0;
  std::vector<int> rp, ci;
  std::vector<double> v;
  long long nnz() const { return rp.empty() ? 0 : rp.back(); }
};

// Device layout of one strict-lower solve  x_i = (b_i - sum_{j<i} M_ij x_j) d_i
// for the line-pipelined kernel (lines = runs of nx consecutive rows).
//  - "ring" part: entries in the row's own line at distance 1..31; stored by
//    column j as push[j*32 + k-1] = M(j+k, j) d_{j+k} (zero if absent or if
//    j+k lies in another line).
//  - "far" part: all other entries, grouped in windows of `win` rows of one
//    line with `lpr` lanes per row: lane = lpr*r + s (r: row in window), slot k
//    of lane l is entry s + lpr*k of that row, wcol/wval[wofs[w] + win*lpr*k
//    + l] (col -1 = padding); values scaled by d_i, so that
//    x_i = b_i d_i - sum_far wval x_j - (ring part).
//  - wait list of window w: pairs (line distance, rows needed) in
//    wait[waitofs[w] .. waitofs[w+1]).
//  - dscale[i] = d_i (1 when the matrix has a unit diagonal).
struct LpLayout {
  int n = 0, nx = 0, nlines = 0, nwin = 0;    // nwin: windows per line
  int lpr = 1;                                 // lanes per row in the far part
  int win = 8;                                 // rows per far-part window (win * lpr <= 32)
  std::vector<int> wofs, wcol, waitofs, wait;
  std::vector<double> wval, push, dscale;
  long long far_entries = 0, ring_entries = 0;
};
LpLayout build_lp(const Csr& M, int nx, const std::vector<double>* dinv, int window_rows, int lanes_per_row);

// Far part of a strict-lower solve for the batched ring kernel: every entry
// of M except those of the row's own line at distance 1..ring-1 (which the
// ring of LpLayout::push carries), values scaled by dscale[i].
Csr far_part(const Csr& M, int nx, const std::vector<double>& dscale, int ring);

// One ILUT-smoothed level of degree q >= 2.
struct PLevel {
  int q = 0, n1d = 0, N = 0;
  Csr A;                        // interior stiffness
  Csr L;                        // strict lower ILUT factor (unit diagonal implied)
  Csr U;                        // strict upper ILUT factor (diagonal held in udinv)
  std::vector<double> udiag;    // diagonal of U
  std::vector<double> ML;       // lumped mass (interior)
  Csr Pro;                      // (M^L_q)^{-1} P_{qc}^{q}: prolongation, N_q x N_c
  Csr Res;                      // (M^L_qc)^{-1} (P_{qc}^{q})^T: restriction, N_c x N_q
  Csr Praw;                     // P_{qc}^{q} unscaled (exported for checks)
  // consistent transfers: banded Cholesky factors of the 1D interior mass
  // matrices (first direction, weighted by |det J| on the annulus; the
  // others), [i][k], k = 0..q: 1/L_ii, then L_{i,i-k}
  std::vector<double> MF0, MF1;
  int depthL = 0, depthU = 0;   // critical-path length (levels) of the two solves
  // line-pipelined solve layout: lines are runs of n1d consecutive rows
  std::vector<int> Lsplit;      // per row of L: first entry in the row's own line
  Csr Um;                       // U with rows and columns mirrored (i -> N-1-i): lower triangular
  std::vector<int> Umsplit;
  LpLayout Llp, Ulp;            // line-pipelined layouts of L and mirrored U (with 1/u_ii)
};

// One P1 level of the coarse h-multigrid.
struct HLevel {
  int ne = 0, n1d = 0, N = 0;
  Csr A;
  std::vector<double> dinv;
  int depthGS = 0;
  // Gauss-Seidel as triangular solves: strict lower / upper parts of A
  Csr Lo, Up, UpM;              // UpM: Up mirrored (lower triangular)
  std::vector<int> Losplit, UpMsplit;
  LpLayout Lolp, UpMlp;         // line-pipelined layouts of the two sweeps (with 1/a_ii)
};

struct Hierarchy {
  int dom = 0, d = 2, p = 2, k = 3;
  pmg_options opt{};
  std::vector<PLevel> lev;      // lev[0] has degree p
  std::vector<double> ML1;      // lumped mass of V_{h,1}
  std::vector<double> M1F0, M1F1;   // consistent transfers: factors of V_{h,1}'s 1D mass matrices
  std::vector<HLevel> hl;       // hl[0]: P1 at h; last: coarsest (direct solve)
  std::vector<double> coarse_inv;   // dense inverse of the coarsest operator
  std::vector<double> f;        // interior load with Dirichlet lift
  std::vector<double> uB;       // full-space boundary coefficients, degree p
  double t_assembly = 0, t_ilut = 0, t_transfer = 0, t_hmg = 0;
};

// Builds the hierarchy; returns PMG_OK or an error status with `err` set.
pmg_status build_hierarchy(int domain, int p, int log2_inv_h, const pmg_options& opt,
                           Hierarchy& H, std::string& err);

// Mirror of a square matrix: entry (i, j) -> (n-1-i, n-1-j), columns ascending.
Csr mirror(const Csr& a);

// Per row: index of the first entry whose column lies in the row's own line
// (lines = runs of nx consecutive rows; columns ascending within each row).
std::vector<int> line_split(const Csr& a, int nx);

// Strict lower (lower = true) or strict upper part of a square matrix.
Csr strict_part(const Csr& a, bool lower);

// Longest dependency chain of a strict triangular factor (levels of the
// wavefront schedule); `lower` selects the direction.
int critical_path(const Csr& T, bool lower);

// L2 error of the degree-p solution (interior coefficients u) against the
// exact solution, (p+3)^d Gauss points per element.
double l2_error(const Hierarchy& H, const double* u);

}  // namespace pmgl
