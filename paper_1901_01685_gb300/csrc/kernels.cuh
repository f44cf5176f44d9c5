// CUDA kernels of the p-multigrid V-cycle (sm_103a, FP64).
//
// Hot-path steps (arXiv 1901.01685, Sec. 3):
//   residual r = f - A u                      (Eq. smooth / Eq. res)
//   ILUT smoothing e = U^{-1} L^{-1} r, u += e (Eq. inverse)
//   lumped L2-projection transfers             (Eq. prolongation / restriction)
//   p = 1 h-multigrid: lexicographic Gauss-Seidel, canonical interpolation,
//   its transpose as restriction, dense coarsest solve
//   residual norm for the stopping rule        (Sec. 5)
//
// The triangular solves and Gauss-Seidel sweeps are dependency-driven
// ("sync-free"): each row waits only for the rows it reads, through per-row
// ready flags tagged with a launch epoch; every wait is bounded and sets an
// error word on expiry instead of hanging.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace pmgk {

// Spin limit for a single dependency wait, in SM clock cycles (~1 s).
constexpr long long kWaitCycles = 2000000000LL;
constexpr int kNormBlocks = 256;
constexpr int kNormThreads = 256;

struct Csr {
  int nr;
  const int* rp;
  const int* ci;
  const double* v;
};

// ---------------------------------------------------------------------------
// memory-order helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Waits until flags[j] == epoch; returns false if the wait expired or another
// thread already reported an expiry (err != 0).
__device__ __forceinline__ bool wait_ready(const unsigned* flags, int j, unsigned epoch, unsigned* err) {
  if (ld_acquire(flags + j) == epoch) return true;
  const long long t0 = clock64();
  for (unsigned it = 1;; ++it) {
    if (ld_acquire(flags + j) == epoch) return true;
    if ((it & 31u) == 0u) {
      if (ld_relaxed(err) != 0u) return false;
      if (clock64() - t0 > kWaitCycles) {
        atomicOr(err, 1u);
        return false;
      }
    }
  }
}

template <int W>
__device__ __forceinline__ double group_sum(double s) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, W);
  return s;
}

// ---------------------------------------------------------------------------
// CSR SpMV: W lanes per row.
//   MODE 0: y = b - A x     MODE 1: y = A x     MODE 2: y = b + A x
// ---------------------------------------------------------------------------
template <int W, int MODE>
__global__ void __launch_bounds__(256) k_spmv(Csr A, const double* __restrict__ x, const double* __restrict__ b,
                                              double* __restrict__ y) {
  const int lane = threadIdx.x & (W - 1);
  const int group = (blockIdx.x * blockDim.x + threadIdx.x) / W;
  const int ngroups = (gridDim.x * blockDim.x) / W;
  for (int row = group; row < A.nr; row += ngroups) {
    const int beg = A.rp[row], end = A.rp[row + 1];
    double s = 0.0;
    for (int t = beg + lane; t < end; t += W) s += A.v[t] * x[A.ci[t]];
    s = group_sum<W>(s);
    if (lane == 0) {
      if (MODE == 0) y[row] = b[row] - s;
      else if (MODE == 1) y[row] = s;
      else y[row] = b[row] + s;
    }
  }
}

// ---------------------------------------------------------------------------
// Sync-free triangular solves, one warp per row, rows claimed in dependency
// order through an atomic counter (rows are claimed only by running warps, so
// the lowest unfinished claimed row always has its inputs ready).
// ---------------------------------------------------------------------------
// y = L^{-1} b, L strict lower (unit diagonal implied).
__global__ void __launch_bounds__(256) k_lsolve(Csr L, const double* __restrict__ b, double* y, unsigned* flags,
                                                unsigned epoch, unsigned* counter, unsigned* err) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    int row = 0;
    if (lane == 0) row = int(atomicAdd(counter, 1u));
    row = __shfl_sync(0xffffffffu, row, 0);
    if (row >= L.nr) return;
    const int beg = L.rp[row], end = L.rp[row + 1];
    double s = 0.0;
    for (int t = beg + lane; t < end; t += 32) {
      const int j = L.ci[t];
      wait_ready(flags, j, epoch, err);
      s += L.v[t] * __ldcg(y + j);
    }
    s = group_sum<32>(s);
    if (lane == 0) {
      __stcg(y + row, b[row] - s);
      st_release(flags + row, epoch);
    }
  }
}

// e = U^{-1} y (U = diag + strict upper), then u += e.
__global__ void __launch_bounds__(256) k_usolve_update(Csr U, const double* __restrict__ udinv,
                                                       const double* __restrict__ y, double* e, double* u,
                                                       unsigned* flags, unsigned epoch, unsigned* counter,
                                                       unsigned* err) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    int c = 0;
    if (lane == 0) c = int(atomicAdd(counter, 1u));
    c = __shfl_sync(0xffffffffu, c, 0);
    if (c >= U.nr) return;
    const int row = U.nr - 1 - c;
    const int beg = U.rp[row], end = U.rp[row + 1];
    double s = 0.0;
    for (int t = beg + lane; t < end; t += 32) {
      const int j = U.ci[t];
      wait_ready(flags, j, epoch, err);
      s += U.v[t] * __ldcg(e + j);
    }
    s = group_sum<32>(s);
    if (lane == 0) {
      const double ei = (y[row] - s) * udinv[row];
      __stcg(e + row, ei);
      if (u) u[row] += ei;
      st_release(flags + row, epoch);
    }
  }
}

// One lexicographic Gauss-Seidel sweep on A x = b in place (forward when
// BACKWARD == false).  Rows read new values of already-visited neighbours and
// old values of the others; a neighbour visited later waits for this row, so
// its old value is still in place when read.
template <bool BACKWARD>
__global__ void __launch_bounds__(256) k_gauss_seidel(Csr A, const double* __restrict__ dinv,
                                                      const double* __restrict__ b, double* x, unsigned* flags,
                                                      unsigned epoch, unsigned* counter, unsigned* err) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    int c = 0;
    if (lane == 0) c = int(atomicAdd(counter, 1u));
    c = __shfl_sync(0xffffffffu, c, 0);
    if (c >= A.nr) return;
    const int row = BACKWARD ? A.nr - 1 - c : c;
    const int beg = A.rp[row], end = A.rp[row + 1];
    double s = 0.0;
    for (int t = beg + lane; t < end; t += 32) {
      const int j = A.ci[t];
      if (j == row) continue;
      if (BACKWARD ? (j > row) : (j < row)) wait_ready(flags, j, epoch, err);
      s += A.v[t] * __ldcg(x + j);
    }
    s = group_sum<32>(s);
    if (lane == 0) {
      __stcg(x + row, (b[row] - s) * dinv[row]);
      st_release(flags + row, epoch);
    }
  }
}

// ---------------------------------------------------------------------------
// P1 canonical transfers (matrix-free, structured interior grids).  Fine grid
// has nf elements per direction (interior nodes 1..nf-1), coarse nf/2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double hat_w(int off) { return off == 0 ? 1.0 : 0.5; }

// rc = P^T rf: coarse interior node c gathers fine nodes 2c-1, 2c, 2c+1 per direction.
__global__ void k_p1_restrict(int d, int nf, const double* __restrict__ rf, double* __restrict__ rc) {
  const int nc = nf / 2, mc = nc - 1, mf = nf - 1;
  const long long Nc = (d == 2) ? (long long)mc * mc : (long long)mc * mc * mc;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < Nc;
       idx += (long long)gridDim.x * blockDim.x) {
    const int cx = int(idx % mc) + 1, cy = int((idx / mc) % mc) + 1;
    const int cz = (d == 3) ? int(idx / ((long long)mc * mc)) + 1 : 0;
    double s = 0.0;
    for (int dz = (d == 3 ? -1 : 0); dz <= (d == 3 ? 1 : 0); ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int fx = 2 * cx + dx, fy = 2 * cy + dy, fz = 2 * cz + dz;
          long long fi = (long long)(fx - 1) + (long long)mf * (fy - 1);
          if (d == 3) fi += (long long)mf * mf * (fz - 1);
          const double w = hat_w(dx) * hat_w(dy) * (d == 3 ? hat_w(dz) : 1.0);
          s += w * rf[fi];
        }
    rc[idx] = s;
  }
}

// xf += P ec: fine interior node gathers its coarse parents.
__global__ void k_p1_prolong_add(int d, int nf, const double* __restrict__ ec, double* __restrict__ xf) {
  const int nc = nf / 2, mc = nc - 1, mf = nf - 1;
  const long long Nf = (d == 2) ? (long long)mf * mf : (long long)mf * mf * mf;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < Nf;
       idx += (long long)gridDim.x * blockDim.x) {
    int node[3] = {int(idx % mf) + 1, int((idx / mf) % mf) + 1, (d == 3) ? int(idx / ((long long)mf * mf)) + 1 : 0};
    int par[3][2], np[3];
    double pw[3][2];
    for (int a = 0; a < 3; ++a) {
      if (a >= d) { par[a][0] = 0; pw[a][0] = 1.0; np[a] = 1; continue; }
      if ((node[a] & 1) == 0) { par[a][0] = node[a] / 2; pw[a][0] = 1.0; np[a] = 1; }
      else { par[a][0] = (node[a] - 1) / 2; par[a][1] = (node[a] + 1) / 2; pw[a][0] = pw[a][1] = 0.5; np[a] = 2; }
    }
    double s = 0.0;
    for (int iz = 0; iz < np[2]; ++iz)
      for (int iy = 0; iy < np[1]; ++iy)
        for (int ix = 0; ix < np[0]; ++ix) {
          const int px = par[0][ix], py = par[1][iy], pz = par[2][iz];
          if (px < 1 || px > mc || py < 1 || py > mc) continue;
          if (d == 3 && (pz < 1 || pz > mc)) continue;
          long long ci = (long long)(px - 1) + (long long)mc * (py - 1);
          if (d == 3) ci += (long long)mc * mc * (pz - 1);
          s += pw[0][ix] * pw[1][iy] * pw[2][iz] * ec[ci];
        }
    xf[idx] += s;
  }
}

// x = Ainv b for the coarsest level (dense, row-major), one warp per row.
__global__ void k_dense_matvec(int n, const double* __restrict__ Ainv, const double* __restrict__ b,
                               double* __restrict__ x) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int row = warp; row < n; row += nw) {
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s += Ainv[(size_t)row * n + j] * b[j];
    s = group_sum<32>(s);
    if (lane == 0) x[row] = s;
  }
}

// ---------------------------------------------------------------------------
// Deterministic squared norm: fixed partition into kNormBlocks blocks, fixed
// reduction tree, then one block combines the partials in a fixed order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kNormThreads) k_sqnorm_partial(int n, const double* __restrict__ r,
                                                                double* __restrict__ partial) {
  __shared__ double sh[kNormThreads];
  const long long chunk = (n + (long long)gridDim.x - 1) / gridDim.x;
  const long long beg = blockIdx.x * chunk;
  const long long end = beg + chunk < n ? beg + chunk : n;
  double s = 0.0;
  for (long long i = beg + threadIdx.x; i < end; i += blockDim.x) s += r[i] * r[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// MODE 0: *r0 = sqrt(sum); MODE 1: *out = sqrt(sum) / *r0.
template <int MODE>
__global__ void __launch_bounds__(kNormThreads) k_norm_finalize(int nparts, const double* __restrict__ partial,
                                                               double* r0, double* out) {
  __shared__ double sh[kNormThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += partial[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double nrm = sqrt(sh[0]);
    if (MODE == 0) *r0 = nrm;
    else *out = nrm / *r0;
  }
}

}  // namespace pmgk
