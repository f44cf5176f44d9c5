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
//   MODE 3: y = (b - A x) d (elementwise)
// ---------------------------------------------------------------------------
template <int W, int MODE>
__global__ void __launch_bounds__(256) k_spmv(Csr A, const double* __restrict__ x, const double* __restrict__ b,
                                              double* __restrict__ y, const double* __restrict__ d = nullptr) {
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
      else if (MODE == 2) y[row] = b[row] + s;
      else y[row] = (b[row] - s) * d[row];
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

namespace pmgk {

// ---------------------------------------------------------------------------
// Line-pipelined lower-triangular solve
//   x_i = (b_i - sum_{j<i} M_ij x_j) d_i      (i in the solve's index space;
//   i' = MIRROR ? n-1-i : i addresses b, x and u, so that an upper factor
//   stored with mirrored rows and columns is solved by the same kernel).
//
// Unknowns are numbered lexicographically, so rows form "lines" of nx
// consecutive rows.  A row depends on a few earlier rows of its own line and
// on rows of earlier lines up to a bounded forward offset, so line l can run
// a bounded number of rows behind line l-1.  Each CTA claims B consecutive
// lines in order (an atomic counter; lines a CTA waits for belong to running
// CTAs) and gives each line two warps:
//  - the producer computes, 8 rows at a time, c_i = b_i d_i - sum_far d_i M_ij x_j
//    over the "far" entries (earlier lines, and own-line entries 32 or more
//    rows back) from a window-major layout with coalesced loads, after one wait
//    per window on the rows it needs;
//  - the chain warp keeps the 32 rows in flight in its lanes and, row by row,
//    broadcasts the finished x_i and pushes it into the 31 following rows of
//    the line with one FMA per lane (coefficients stored by column).  Only a
//    shuffle and one FMA lie on the per-row critical path.
// Lines of one CTA exchange values and progress through shared memory; other
// lines through global memory and an epoch-tagged per-line progress word.
// Every wait is bounded; on expiry the error word is set and the kernel
// finishes with invalid values instead of hanging.
// ---------------------------------------------------------------------------
constexpr int kLpAhead = 4;        // chain adds c_i this many rows before row i finishes
constexpr int kLpStage = 16;       // rows of push coefficients per cp.async stage (double buffered)
constexpr int kLpLinesPerCta = 2;
constexpr int kLpProducers = 6;    // producer warps per line (windows dealt round-robin)

// "Not yet computed" marker: the all-ones bit pattern, a NaN that floating-point
// arithmetic never produces (generated NaNs carry the canonical payload).  The
// solve's output vector is filled with it (byte 0xFF) before the launch; every
// consumer polls the value itself, so a value and its readiness travel together
// in one aligned 64-bit access and no fences or counters are needed.
constexpr unsigned long long kPending = 0xFFFFFFFFFFFFFFFFull;

// v where c holds, +0.0 elsewhere, by masking the bit pattern (integer ops).
__device__ __forceinline__ double keep_if(bool c, double v) {
  return __longlong_as_double(__double_as_longlong(v) & (c ? -1ll : 0ll));
}
// the bit pattern of v, with a NaN that reads as the pending marker replaced
// by the canonical NaN
__device__ __forceinline__ unsigned long long publish_bits(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return b == kPending ? 0x7FF8000000000000ull : b;
}

struct Lp2 {
  int n, nx, nlines, nwin, lpr, win;
  const int* wofs;
  const int* wcol;
  const double* wval;
  const int* waitofs;
  const int* wait;      // (line distance, rows needed) pairs
  const double* push;   // [n][32]
  const double* dscale; // [n]
};

template <bool MIRROR>
__device__ __forceinline__ int lp_vec(int i, int n) { return MIRROR ? n - 1 - i : i; }

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const double* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
// generic address (global memory, or this CTA's shared memory written by
// another CTA of the cluster)
__device__ __forceinline__ unsigned long long ld_relaxed_generic_u64(const double* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(double* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_f64(double* p, double v) {
  asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Copies the push coefficients of rows [r0, r0 + kLpStage) of the line
// (clamped to the line end) into `dst` (kLpStage x 32 doubles): 16-byte
// chunks, 8 per lane.
__device__ __forceinline__ void lp_stage_push(double* dst, const double* push, int row0, int r0, int nx, int lane) {
#pragma unroll
  for (int t = 0; t < kLpStage * 16 / 32; ++t) {
    const int chunk = t * 32 + lane;       // 16 chunks of 16 bytes per row
    const int r = chunk >> 4, c = (chunk & 15) * 2;
    if (r0 + r < nx) cp_async16(dst + r * 32 + c, push + (size_t)(row0 + r0 + r) * 32 + c);
  }
}

// Bounded poll of a pending value (global memory); producers back off briefly.
__device__ __forceinline__ double lp_get_global(const double* p, unsigned* err) {
  unsigned long long v = ld_relaxed_u64(p);
  if (v != kPending) return __longlong_as_double((long long)v);
  const long long t0 = clock64();
  for (unsigned it = 1;; ++it) {
    __nanosleep(it < 16 ? 32 : 256);
    v = ld_relaxed_u64(p);
    if (v != kPending) return __longlong_as_double((long long)v);
    if ((it & 15u) == 0u && (ld_relaxed(err) != 0u || clock64() - t0 > kWaitCycles)) {
      atomicOr(err, 1u);
      return 0.0;
    }
  }
}
// Same for a value in shared memory.  BACKOFF: sleep between polls, so that
// waiting producer warps leave the shared-memory pipe to the chain warp (whose
// shuffles and shared loads would otherwise queue behind their polls).
template <bool BACKOFF>
__device__ __forceinline__ double lp_get_shared(const volatile double* p, unsigned* err) {
  const volatile unsigned long long* q = reinterpret_cast<const volatile unsigned long long*>(p);
  unsigned long long v = *q;
  if (v != kPending) return __longlong_as_double((long long)v);
  const long long t0 = clock64();
  for (unsigned it = 1;; ++it) {
    if (BACKOFF) __nanosleep(it < 16 ? 32 : 256);
    v = *q;
    if (v != kPending) return __longlong_as_double((long long)v);
    if ((it & 31u) == 0u && (ld_relaxed(err) != 0u || clock64() - t0 > kWaitCycles)) {
      atomicOr(err, 1u);
      return 0.0;
    }
  }
}

template <bool MIRROR, bool UPDATE, int WIN, int LPR>
__global__ void __launch_bounds__(32 * (kLpProducers + 1) * kLpLinesPerCta)
    k_lp2(Lp2 M, const double* __restrict__ b, double* x, double* u, unsigned* counter, unsigned* err) {
  extern __shared__ __align__(16) unsigned char lp_smem[];
  constexpr int B = kLpLinesPerCta, WPL = kLpProducers + 1;
  __shared__ int s_block;
  const int nx = M.nx;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int myline = warp / WPL, role = warp % WPL;   // role kLpProducers = chain
  volatile double* xs_all = reinterpret_cast<double*>(lp_smem);   // [B][nx] finished values
  volatile double* cs_all = xs_all + (size_t)B * nx;              // [B][nx] producer partial sums
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_block = (int)atomicAdd(counter, 1u);
    for (int t = threadIdx.x; t < 2 * B * nx; t += blockDim.x)
      reinterpret_cast<volatile unsigned long long*>(xs_all)[t] = kPending;
    __syncthreads();
    const int base = s_block * B;
    if (base >= M.nlines) return;
    const int cnt = min(B, M.nlines - base);
    if (myline >= cnt) continue;
    const int line = base + myline;
    const int row0 = line * nx;
    volatile double* xs_line = xs_all + (size_t)myline * nx;
    volatile double* cs_line = cs_all + (size_t)myline * nx;
    if (role < kLpProducers) {
      // ------------------------------ producers ------------------------------
      // Windows of WIN rows, LPR lanes per row.  FP64 FMA chains are slow on
      // this part, so rows with many far entries split them over 8 lanes (short
      // per-lane chains, small windows); rows with few far entries use one
      // lane each.
      static_assert(WIN * LPR <= 32, "window does not fit a warp");
      constexpr int LANES = WIN * LPR;
      for (int w = role; w < M.nwin; w += kLpProducers) {
        const int W = line * M.nwin + w;
        const int o = M.wofs[W], K = (M.wofs[W + 1] - o) / LANES;
        const int ix = w * WIN + lane / LPR;
        double a0 = 0.0, a1 = 0.0;
        if (lane < LANES && ix < nx) {
          for (int k0 = 0; k0 < K; k0 += 8) {
            int jj[8];
            double vv[8];
            unsigned long long raw[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
              const bool in = k0 + t < K;
              jj[t] = in ? M.wcol[o + LANES * (k0 + t) + lane] : -1;
              vv[t] = in ? M.wval[o + LANES * (k0 + t) + lane] : 0.0;
            }
#pragma unroll
            for (int t = 0; t < 8; ++t) {
              const int j = jj[t];
              raw[t] = 0ull;
              if (j >= 0) {
                const int lj = j / nx;
                raw[t] = lj >= base ? reinterpret_cast<const volatile unsigned long long*>(xs_all)[(size_t)(lj - base) * nx + (j - lj * nx)]
                                    : ld_relaxed_u64(x + lp_vec<MIRROR>(j, M.n));
              }
            }
#pragma unroll
            for (int t = 0; t < 8; ++t) {
              double xv = __longlong_as_double((long long)raw[t]);
              if (raw[t] == kPending) {
                const int j = jj[t], lj = j / nx;
                xv = lj >= base ? lp_get_shared<true>(xs_all + (size_t)(lj - base) * nx + (j - lj * nx), err)
                                : lp_get_global(x + lp_vec<MIRROR>(j, M.n), err);
              }
              if (t & 1) a1 = fma(vv[t], xv, a1);
              else a0 = fma(vv[t], xv, a0);
            }
          }
        }
        double acc = a0 + a1;
        if (LPR > 1) {
#pragma unroll
          for (int off = 1; off < LPR; off <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        }
        if (lane < LANES && (lane % LPR) == 0 && ix < nx) {
          const int i = row0 + ix;
          cs_line[ix] = b[lp_vec<MIRROR>(i, M.n)] * M.dscale[i] - acc;   // far values carry d_i
        }
      }
      if (UPDATE) {
        // u += x for this line's rows as the chain finishes them
        for (int ix = role * 32 + lane; ix < nx; ix += 32 * kLpProducers)
          u[lp_vec<MIRROR>(row0 + ix, M.n)] += lp_get_shared<true>(xs_line + ix, err);
      }
      continue;
    }
    // -------------------------------- chain --------------------------------
    double* pbuf = const_cast<double*>(cs_all) + (size_t)B * nx + (size_t)myline * 2 * kLpStage * 32;
    lp_stage_push(pbuf, M.push, row0, 0, nx, lane);
    cp_async_commit();
    double acc = 0.0;
    if (lane < kLpAhead && lane < nx) acc = lp_get_shared<false>(cs_line + lane, err);
    for (int ix0 = 0, st = 0; ix0 < nx; ix0 += kLpStage, st ^= 1) {
      if (ix0 + kLpStage < nx) {
        lp_stage_push(pbuf + (st ^ 1) * kLpStage * 32, M.push, row0, ix0 + kLpStage, nx, lane);
        cp_async_commit();
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncwarp();
      const volatile double* pc = pbuf + st * kLpStage * 32;
#pragma unroll
      for (int q = 0; q < kLpStage; ++q) {
        const int ix = ix0 + q;
        if (ix < nx) {
          const int s = ix & 31;
          const double coef = pc[q * 32 + ((lane - s - 1) & 31)];
          const double xi = __shfl_sync(0xffffffffu, acc, s);
          acc = keep_if(lane != s, fma(-coef, xi, acc));
          const int ia = ix + kLpAhead;
          if (ia < nx && lane == (ia & 31)) acc += lp_get_shared<false>(cs_line + ia, err);
          if (lane == 0) {
            // a NaN must never read as the pending marker
            const double xo = (unsigned long long)__double_as_longlong(xi) == kPending
                                  ? __longlong_as_double(0x7FF8000000000000ll) : xi;
            xs_line[ix] = xo;
            st_relaxed_f64(x + lp_vec<MIRROR>(row0 + ix, M.n), xo);
          }
        }
      }
      __syncwarp();
    }
  }
}

}  // namespace pmgk

namespace pmgk {

// ---------------------------------------------------------------------------
// Line-pipelined lower-triangular solve with the chain and its producers on
// different SMs: thread-block clusters of two CTAs per line, one to four
// consecutive lines per cluster.
//
// Same operation and layout as k_lp2 (Lp2).  On GB300 the FP64 unit is
// shared by a whole SM: one warp's FP64 instruction has a 64-cycle latency and
// the SM retires about one warp-wide FP64 instruction every 19 cycles.  While
// producer warps on the chain's SM issue their FP64 FMAs, the chain's FMA waits
// behind them and its per-row time grows about five-fold (measured: ~1000
// instead of ~205 cycles a row).  Here the chain CTA (cluster rank 2k for the
// group's line k) runs only the chain warp; the producer CTA (rank 2k + 1, eight warps on all four
// sub-partitions) computes c_i = b_i d_i - sum_far d_i M_ij x_j and stores it
// straight into the chain CTA's shared memory (distributed shared memory,
// relaxed cluster-scope stores; the value is its own ready flag, as in
// k_lp2).  Rank 0 claims groups of lines in order through an atomic counter
// (lines a cluster waits for belong to running clusters) and hands the group
// number to the other ranks; one cluster barrier per group orders the resets
// of the receiving buffers before the first stores for the new group.
// Finished values go to global memory; producers read every far value from
// there, except the previous line's when it belongs to the same cluster.
// ---------------------------------------------------------------------------
constexpr int kLp4Warps = 8;
constexpr int kLp4Producers = 8;

__device__ __forceinline__ unsigned cluster_ctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// barrier over all threads of the cluster (release / acquire)
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// address of `local` (this CTA's shared memory) in the shared window of cluster rank `rank`
__device__ __forceinline__ unsigned dsmem_addr(const void* local, unsigned rank) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(local);
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster_u64(unsigned addr, unsigned long long v) {
  asm volatile("st.relaxed.cluster.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}
__device__ __forceinline__ void st_cluster_s32(unsigned addr, int v) {
  asm volatile("st.relaxed.cluster.shared::cluster.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_cluster_local_u64(const void* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.cluster.shared::cta.u64 %0, [%1];"
               : "=l"(v) : "r"((unsigned)__cvta_generic_to_shared(p)) : "memory");
  return v;
}
// Warp-uniform waits.  Every lane of the warp runs them together: lanes whose
// value is not needed or already there keep polling alongside the others.  A
// per-lane wait (some lanes in a spin loop, the rest past it) leaves the warp
// split in two thread groups that then issue every later instruction
// separately until the next reconvergence point -- measured on GB300 as a
// four-fold slower chain loop for the rest of the stage.
//
// Chain side: value of the producer sum at p for lanes with `need` (0.0 for
// the others), waiting while any needed one is pending.
__device__ __noinline__ unsigned long long lp4_wait_c_uniform(const double* p, bool need, unsigned long long v,
                                                              unsigned* err) {
  const long long t0 = clock64();
  for (unsigned it = 1;; ++it) {
    if (need && v == kPending) v = ld_cluster_local_u64(p);
    if (!__any_sync(0xffffffffu, need && v == kPending)) return v;
    if ((it & 31u) == 0u) {
      const bool expired = ld_relaxed(err) != 0u || clock64() - t0 > kWaitCycles;
      if (__any_sync(0xffffffffu, expired)) {
        if ((threadIdx.x & 31) == 0) atomicOr(err, 1u);
        return v == kPending ? 0ull : v;
      }
    }
  }
}
__device__ __forceinline__ double lp4_get_c(const double* p, bool need, unsigned* err) {
  unsigned long long v = need ? ld_cluster_local_u64(p) : 0ull;
  if (__any_sync(0xffffffffu, need && v == kPending)) v = lp4_wait_c_uniform(p, need, v, err);
  return __longlong_as_double((long long)v);   // 0 for lanes without need (never loaded)
}
// Producer warp of k_lp4: windows role, role + kLp4Producers, ... of the
// line; c goes to the chain CTA's buffer at cluster address cs_remote; then
// (UPDATE) u += x for the line's rows.  xin (or nullptr): this CTA's copy of
// the previous line, pushed row by row by that line's chain in the same
// cluster; entries in the previous line are read there, all others from x.
template <bool MIRROR, bool UPDATE, int WIN, int LPR>
__device__ __noinline__ void lp4_producer(Lp2 M, const double* __restrict__ b, double* x, double* u,
                                          unsigned cs_remote, const double* xin, int line, int role, int lane,
                                          unsigned* err) {
  static_assert(WIN * LPR <= 32, "window does not fit a warp");
  constexpr int LANES = WIN * LPR;
  const int nx = M.nx, row0 = line * nx, prev0 = row0 - nx;
  for (int w = role; w < M.nwin; w += kLp4Producers) {
    const int W = line * M.nwin + w;
    const int o = M.wofs[W], K = (M.wofs[W + 1] - o) / LANES;
    const int ix = w * WIN + lane / LPR;
    const bool valid = lane < LANES && ix < nx;
    const bool head = valid && (lane % LPR) == 0;
    // b_i d_i before any wait (the far values carry d_i), so that only the
    // reduction follows the last far value
    const double bd = head ? b[lp_vec<MIRROR>(row0 + ix, M.n)] * M.dscale[row0 + ix] : 0.0;
    double a = 0.0;
    // K is the same for every lane of the window: the loop and its waits stay
    // warp-uniform.  Entries are in column order, the order in which earlier
    // lines finish them, so each entry is summed as soon as every lane has it.
    for (int k0 = 0; k0 < K; k0 += 8) {
      int jj[8];
      double vv[8];
      unsigned long long raw[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const bool in = valid && k0 + t < K;
        jj[t] = in ? M.wcol[o + LANES * (k0 + t) + lane] : -1;
        vv[t] = in ? M.wval[o + LANES * (k0 + t) + lane] : 0.0;
      }
      const double* src[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int j = jj[t] < 0 ? 0 : jj[t];
        src[t] = (xin != nullptr && j >= prev0 && j < row0) ? xin + (j - prev0) : x + lp_vec<MIRROR>(j, M.n);
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) raw[t] = jj[t] >= 0 ? ld_relaxed_generic_u64(src[t]) : 0ull;
      // Sum the entries in order as they arrive; while any is pending, re-read
      // every pending entry of the block at once, so that one round trip to L2
      // picks up all the rows the chain has published meanwhile (entry-by-entry
      // polling paid one round trip per entry).  `next` and kn are warp-uniform.
      const int kn = min(8, K - k0);   // padding slots of the window cost nothing
      int next = 0;
      const long long t0 = clock64();
      for (unsigned it = 0;; ++it) {
#pragma unroll
        for (int t = 0; t < 8; ++t)
          if (t == next && t < kn && !__any_sync(0xffffffffu, raw[t] == kPending)) {
            a = fma(vv[t], __longlong_as_double((long long)raw[t]), a);
            ++next;
          }
        if (next >= kn) break;
        if (it >= 16) __nanosleep(32);
#pragma unroll
        for (int t = 0; t < 8; ++t)
          if (t >= next && raw[t] == kPending) raw[t] = ld_relaxed_generic_u64(src[t]);
        if ((it & 15u) == 15u) {
          const bool expired = ld_relaxed(err) != 0u || clock64() - t0 > kWaitCycles;
          if (__any_sync(0xffffffffu, expired)) {
            if (lane == 0) atomicOr(err, 1u);
            break;   // the remaining entries stay unsummed: the result is invalid and flagged
          }
        }
      }
    }
    if (LPR > 1) {
#pragma unroll
      for (int off = 1; off < LPR; off <<= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
    }
    if (head) {
      const int i = row0 + ix;
      const double c = bd - a;
      // a NaN must never read as the pending marker
      const unsigned long long cb = (unsigned long long)__double_as_longlong(c) == kPending
                                        ? 0x7FF8000000000000ull : (unsigned long long)__double_as_longlong(c);
      st_cluster_u64(cs_remote + 8u * unsigned(ix), cb);
    }
  }
  if (UPDATE) {
    // u += x for this line's rows as the chain publishes them
    for (int ix = role * 32 + lane; ix < nx; ix += 32 * kLp4Producers) {
      const int iv = lp_vec<MIRROR>(row0 + ix, M.n);
      u[iv] += lp_get_global(x + iv, err);
    }
  }
}

// Launch: grid = 2 NL x clusters, cluster dimension 2 NL, 32 * kLp4Warps
// threads, dynamic shared memory lp4_smem_doubles(nx) doubles.  A cluster
// takes NL consecutive lines at a time (rank 2k: chain of line k, rank 2k+1:
// its producers); line k's chain also pushes every finished value into the
// shared memory of line k+1's producer CTA, so that the hop from a line to
// the next inside a cluster is a distributed-shared-memory store and a local
// poll instead of a round trip through L2.  The receiving buffer alternates
// between two halves from one group of lines to the next: a chain may still
// be storing its last values when the next line's producer, done with its
// own rows, loops back and resets a buffer (the cluster barrier of the next
// group orders those stores before the reset of the same half).
__host__ __device__ constexpr int lp4_smem_doubles_for(int nx) {
  return ((nx + 1) & ~1) + 3 * kLpStage * 32 > 2 * ((nx + 1) & ~1) ? ((nx + 1) & ~1) + 3 * kLpStage * 32
                                                                   : 2 * ((nx + 1) & ~1);
}
template <bool MIRROR, bool UPDATE, int WIN, int LPR, int G, int A, int NL>
__global__ void __launch_bounds__(32 * kLp4Warps, 1)
    k_lp4(Lp2 M, const double* __restrict__ b, double* x, double* u, unsigned* counter, unsigned* err) {
  static_assert(A + G < 32, "c must enter a lane after the lane was recycled");
  static_assert(kLpStage % G == 0, "groups of G rows must tile a stage");
  static_assert(NL >= 1 && 2 * NL <= 8, "a cluster holds at most 8 CTAs");
  extern __shared__ __align__(16) unsigned char lp4_smem[];
  __shared__ int s_group;
  const int nx = M.nx, nxe = (nx + 1) & ~1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned rank = cluster_ctarank();
  const int k = int(rank >> 1);
  const bool chain_cta = (rank & 1u) == 0u;
  // chain CTA: [nxe] producer sums c_i, then [3][kLpStage][32] push coefficients
  // (16-byte aligned: cp.async destinations); producer CTA: [2][nxe] copy of
  // the previous line (k > 0)
  double* cs = reinterpret_cast<double*>(lp4_smem);
  double* pbuf = cs + nxe;
  const unsigned cs_remote = dsmem_addr(cs, rank & ~1u);                 // producer -> its chain's c buffer
  const unsigned xin_remote = (chain_cta && k + 1 < NL) ? dsmem_addr(cs, unsigned(2 * k + 3)) : 0u;
  cluster_barrier();   // every CTA running before any distributed shared memory access
  for (int grp = 0;; ++grp) {
    __syncthreads();     // this CTA is done with the previous group's buffers
    const int par = grp & 1;
    if (rank == 0 && threadIdx.x == 0) {
      const int g = (int)atomicAdd(counter, 1u);
      for (unsigned r = 0; r < 2u * NL; ++r) st_cluster_s32(dsmem_addr(&s_group, r), g);
    }
    if (chain_cta) {
      for (int t = threadIdx.x; t < nx; t += blockDim.x) reinterpret_cast<unsigned long long*>(cs)[t] = kPending;
    } else if (k > 0) {
      for (int t = threadIdx.x; t < nx; t += blockDim.x) reinterpret_cast<unsigned long long*>(cs + par * nxe)[t] = kPending;
    }
    cluster_barrier();
    const int g = s_group;
    if (g * NL >= M.nlines) return;
    const int line = g * NL + k;
    if (line >= M.nlines) continue;   // the last group may be partial
    if (!chain_cta) {
      lp4_producer<MIRROR, UPDATE, WIN, LPR>(M, b, x, u, cs_remote, k > 0 ? cs + par * nxe : nullptr, line, warp,
                                             lane, err);
      continue;
    }
    if (warp != 0) continue;
    // ----------------------------- chain ------------------------------------
    const int row0 = line * nx;
    const bool push_next = xin_remote != 0u && line + 1 < M.nlines;
    const unsigned xin_next = xin_remote + 8u * unsigned(par * nxe);
    lp_stage_push(pbuf, M.push, row0, 0, nx, lane);
    cp_async_commit();
    lp_stage_push(pbuf + kLpStage * 32, M.push, row0, kLpStage, nx, lane);
    cp_async_commit();
    double acc = lp4_get_c(cs + lane, lane < A + G && lane < nx, err);
    for (int ix0 = 0, st = 0; ix0 < nx; ix0 += kLpStage, st = (st == 2 ? 0 : st + 1)) {
      cp_async_wait<1>();      // stage k complete (k+1 may still be in flight)
      __syncwarp();
      const double* pc = pbuf + st * kLpStage * 32;
      double cf[kLpStage];
#pragma unroll
      for (int q = 0; q < kLpStage; ++q) cf[q] = pc[q * 32 + ((lane - ix0 - q - 1) & 31)];
#pragma unroll
      for (int q = 0; q < kLpStage; ++q) {
        const int ix = ix0 + q;
        if (ix < nx) {
          const int s = ix & 31;
          const double xi = __shfl_sync(0xffffffffu, acc, s);
          acc = keep_if(lane != s, fma(-cf[q], xi, acc));
          if ((q % G) == G - 1) {   // ix0 is a multiple of kLpStage, so this is (ix % G) == G - 1
            // c of rows [ix + 1 + A, ix + 1 + A + G) enters their lanes
            const int ia0 = ix + 1 + A;
            const int d = (lane - ia0) & 31;
            acc += lp4_get_c(cs + ia0 + d, d < G && ia0 + d < nx, err);
          }
          if (lane == 0) {
            // a NaN must never read as the pending marker
            const unsigned long long xo = publish_bits(xi);
            st_relaxed_u64(x + lp_vec<MIRROR>(row0 + ix, M.n), xo);
            if (NL > 1 && push_next) st_cluster_u64(xin_next + 8u * unsigned(ix), xo);
          }
        }
      }
      __syncwarp();
      const int nb = (st == 0 ? 2 : st - 1);
      lp_stage_push(pbuf + nb * kLpStage * 32, M.push, row0, ix0 + 2 * kLpStage, nx, lane);
      cp_async_commit();
    }
    cp_async_wait<0>();
  }
}

}  // namespace pmgk

namespace pmgk {

// ---------------------------------------------------------------------------
// Lexicographic Gauss-Seidel sweep on a 2D P1 level (m x m interior grid,
// 9-point stencil) as a wavefront over grid lines.
//
// The sweep's lower solve x_i = t_i - sum_{W,SW,S,SE} c x (t = (b - U x_old) d,
// c = a d, d = 1/a_ii; mirrored indices for the backward sweep) couples a row
// to its left neighbour and to three rows of the line below.  Lane k of warp w
// owns grid line l = 32 w + k and, at step s, computes column s - 2k: the line
// below's value at column c + 1 is the one lane k - 1 computed at the previous
// step (one shuffle), columns c and c - 1 are the two before it (registers).
// Warp w's lane 0 takes line 32 w - 1 from warp w - 1's lane 31 through
// shared memory (value-as-flag, as in the line-pipelined solves).  Each row
// sees the same values as the sequential sweep; only the order of its four
// products differs.  The result is written over x (the old values were
// consumed by the SpMV that formed t).
//
// The warps sit on different SMs: one thread-block cluster of ceil(nw / wpc)
// CTAs of wpc warps (wpc = ceil(nw / 8)), the boundary line going to the next
// warp's CTA by distributed shared memory.  One warp issues at most one FP64
// instruction per ~64 cycles on GB300 (measured: independent DFMAs of one
// warp retire one per 64 cycles, four warps on one SM one per 19 cycles), so
// a step costs at least its four FMAs, ~256 cycles; warps on one SM would
// also share that SM's FP64 pipe.  Each lane keeps its own line's (t, c) for
// the next kWavePrefetch steps in registers (lanes read different lines, so
// there is no coalescing to gain from staging them).  Per step, the products
// with the two older values of the line below (SW, S) of the next point are
// formed while the current point waits for its left neighbour, so that the
// dependent path of a step is two FMAs (W, then SE).
// Dynamic shared memory: wave_smem_doubles(m) doubles.
// ---------------------------------------------------------------------------
constexpr int kWaveMaxLines = 800;
constexpr int kWaveMaxClusterCtas = 8;
constexpr int kWavePrefetch = 15;

// warps per CTA for a wavefront over m lines
__host__ __device__ inline int wave_wpc(int m) {
  const int nw = (m + 31) / 32;
  return (nw + kWaveMaxClusterCtas - 1) / kWaveMaxClusterCtas;
}
// the incoming boundary line of each local warp, [wpc][m]
__host__ __device__ inline size_t wave_smem_doubles(int m) { return size_t(wave_wpc(m)) * size_t(m); }

// Lane 0's boundary value at column col of its incoming line (raw: the value
// read so far): a bounded warp-uniform poll, called only while the value is
// pending and kept out of line, so that the unrolled step body holds no loop
// (with the loop inlined in every step a step took ~200 cycles longer, even
// in warps that never wait).
__device__ __noinline__ unsigned long long wave_wait_boundary(const double* inb, bool need, int col,
                                                              unsigned long long raw, long long t0, unsigned* err) {
  for (unsigned it = 1; __any_sync(0xffffffffu, need && raw == kPending); ++it) {
    if (need && raw == kPending) raw = ld_cluster_local_u64(inb + col);
    if ((it & 63u) == 0u) {
      const bool expired = ld_relaxed(err) != 0u || clock64() - t0 > kWaitCycles;
      if (__any_sync(0xffffffffu, expired)) {
        if (need && raw == kPending) { atomicOr(err, 1u); raw = 0ull; }
        break;
      }
    }
  }
  return raw;
}

template <bool MIRROR>
__global__ void __launch_bounds__(32 * ((kWaveMaxLines + 31) / 32 + kWaveMaxClusterCtas - 1) / kWaveMaxClusterCtas, 1)
    k_gs_wave(int m, const double* __restrict__ coef, const double* __restrict__ t, double* x, unsigned* err) {
  extern __shared__ __align__(16) unsigned char wave_smem[];
  double* inb_all = reinterpret_cast<double*>(wave_smem);   // [wpc][m] incoming boundary line of each local warp
  const int lane = threadIdx.x & 31, lw = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  const int warp = int(cluster_ctarank()) * wpc + lw;
  const int nw = (m + 31) / 32;
  const int n = m * m;
  for (int i = threadIdx.x; i < wpc * m; i += blockDim.x) reinterpret_cast<unsigned long long*>(inb_all)[i] = kPending;
  cluster_barrier();   // every buffer reset before any warp of the cluster stores into one
  if (warp < nw) {
    const double* inb = inb_all + lw * m;
    const bool has_prev = warp > 0, has_next = warp + 1 < nw;
    const unsigned next_addr = has_next ? dsmem_addr(inb_all + ((warp + 1) % wpc) * m, unsigned((warp + 1) / wpc)) : 0u;
    const int l = 32 * warp + lane;
    const bool line_ok = l < m;
    const int steps = m + 2 * 31;
    const long long t0 = clock64();
    // rolling prefetch of (t_i, c_SW, c_S, c_SE, c_W) for steps s .. s + kWavePrefetch (registers)
    double pt[kWavePrefetch + 1], pc[kWavePrefetch + 1][4];
    auto fetch = [&](int s, double& tv, double (&cv)[4]) {
      const int c = s - 2 * lane;
      if (line_ok && c >= 0 && c < m) {
        const int i = l * m + c;
        tv = __ldg(t + lp_vec<MIRROR>(i, n));
        const double2 a = __ldg(reinterpret_cast<const double2*>(coef) + 2 * (size_t)i);
        const double2 b = __ldg(reinterpret_cast<const double2*>(coef) + 2 * (size_t)i + 1);
        cv[0] = a.x; cv[1] = a.y; cv[2] = b.x; cv[3] = b.y;
      } else {
        tv = 0.0; cv[0] = cv[1] = cv[2] = cv[3] = 0.0;
      }
    };
#pragma unroll
    for (int q = 0; q <= kWavePrefetch; ++q) fetch(q, pt[q], pc[q]);
    // lane 0's boundary value at column col; other lanes pass through
    auto boundary = [&](bool need, int col, unsigned long long raw) -> unsigned long long {
      if (__any_sync(0xffffffffu, need && raw == kPending)) raw = wave_wait_boundary(inb, need, col, raw, t0, err);
      return raw;
    };
    // below(s): the line below at column c + 1 for step s; bm1 = below(s - 1),
    // bm2 = below(s - 2).  Lane 0 of warp w > 0 starts with column 0 of the
    // boundary line as below(-1).
    double bm1 = 0.0, bm2 = 0.0;
    {
      const bool need = lane == 0 && has_prev;
      const unsigned long long v = boundary(need, 0, need ? ld_cluster_local_u64(inb) : 0ull);
      if (need) bm1 = __longlong_as_double((long long)v);
    }
    // lane 0's boundary value for the next step, read one step ahead
    unsigned long long nb = (lane == 0 && has_prev && 1 < m) ? ld_cluster_local_u64(inb + 1) : 0ull;
    double xl = 0.0, got = 0.0;
    double part = fma(-pc[0][1], bm1, fma(-pc[0][0], bm2, pt[0]));   // step 0: t - c_SW below(-2) - c_S below(-1)
    for (int s0 = 0; s0 < steps; s0 += kWavePrefetch + 1) {
#pragma unroll
      for (int q = 0; q <= kWavePrefetch; ++q) {
        const int s = s0 + q;
        if (s < steps) {
          constexpr int R = kWavePrefetch + 1;
          const int qn = (q + 1) % R;   // slot of step s + 1
          const int c = s - 2 * lane;
          double bs = lane == 0 ? 0.0 : got;
          const bool need = lane == 0 && has_prev && s + 1 < m;
          if (__any_sync(0xffffffffu, need)) {
            const unsigned long long v = boundary(need, s + 1, nb);
            if (need) bs = __longlong_as_double((long long)v);
            if (lane == 0 && s + 2 < m) nb = ld_cluster_local_u64(inb + s + 2);
          }
          // dependent path: W (left neighbour, out(s - 1)), then SE (below(s))
          const double o1 = fma(-pc[q][3], xl, part);
          const double pn1 = fma(-pc[qn][0], bm1, pt[qn]);       // next point: t - c_SW below(s - 1)
          double out = fma(-pc[q][2], bs, o1);
          part = fma(-pc[qn][1], bs, pn1);                        //             - c_S below(s)
          const bool active = line_ok && c >= 0 && c < m;
          out = active ? out : 0.0;
          got = __shfl_up_sync(0xffffffffu, out, 1);
          if (active) {
            x[lp_vec<MIRROR>(l * m + c, n)] = out;
            // a NaN must never read as the pending marker
            if (lane == 31 && has_next) st_cluster_u64(next_addr + 8u * unsigned(c), publish_bits(out));
          }
          xl = out;
          bm2 = bm1;
          bm1 = bs;
          fetch(s + R, pt[q], pc[q]);
        }
      }
    }
  }
  cluster_barrier();   // no CTA leaves while a peer may still store into its shared memory
}

}  // namespace pmgk

namespace pmgk {

// ---------------------------------------------------------------------------
// Sliced-ELL SpMV (residual and transfer operators).  Rows in slices of 32,
// one row per lane; each slice holds its widest row's entry count rounded up
// to a multiple of 4, in groups of four entries a row: per group the column
// indices (one int4 a lane, 512 B a warp), the values of entries 0, 1 (one
// double2 a lane) and of entries 2, 3 (one double2 a lane), each block
// lane-major, so every load is a coalesced 16-byte-per-lane access and every
// lane runs its own FMA chain (no reductions).  Padding slots have column -1
// and are skipped.
//   MODE 0: y = b - A x   1: y = A x   2: y = b + A x   3: y = (b - A x) d
// One warp per slice (8 per CTA), at most 32 registers a thread so that 64
// warps fit an SM: the SM's FP64 pipe is near its limit at 2 flop per 12
// bytes, and the resident warps hide the gathers (measured 0.63 of the HBM
// copy rate cold at 81 non-zeros a row, against 0.51 with 48 warps an SM).
// ---------------------------------------------------------------------------
struct Sell {
  int nr, nslices;
  const long long* sofs;   // [nslices + 1] first slot of each slice (multiple of 128)
  const int4* col4;        // [slots / 4]
  const double2* val2;     // [slots / 2]
};

template <int MODE>
__global__ void __launch_bounds__(256, 8) k_sell(Sell S, const double* __restrict__ x, const double* __restrict__ b,
                                              double* __restrict__ y, const double* __restrict__ d) {
  const int lane = threadIdx.x & 31;
  const int slice = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (slice >= S.nslices) return;
  const long long base = __ldg(S.sofs + slice), end = __ldg(S.sofs + slice + 1);
  const int groups = int((end - base) >> 7);            // groups of 4 entries (128 slots)
  const int4* c4 = S.col4 + (base >> 2) + lane;          // 32 int4 a group
  const double2* v2 = S.val2 + (base >> 1) + lane;       // 64 double2 a group: entries 0,1 then 2,3
  double acc = 0.0;
#pragma unroll 2
  for (int g = 0; g < groups; ++g) {
    const int4 c = __ldg(c4 + 32 * g);
    const double2 va = __ldg(v2 + 64 * g);
    const double2 vb = __ldg(v2 + 64 * g + 32);
    const double x0 = c.x >= 0 ? __ldg(x + c.x) : 0.0;
    const double x1 = c.y >= 0 ? __ldg(x + c.y) : 0.0;
    const double x2 = c.z >= 0 ? __ldg(x + c.z) : 0.0;
    const double x3 = c.w >= 0 ? __ldg(x + c.w) : 0.0;
    acc = fma(va.x, x0, acc);
    acc = fma(va.y, x1, acc);
    acc = fma(vb.x, x2, acc);
    acc = fma(vb.y, x3, acc);
  }
  const int row = slice * 32 + lane;
  if (row < S.nr) {
    if (MODE == 0) y[row] = b[row] - acc;
    else if (MODE == 1) y[row] = acc;
    else if (MODE == 2) y[row] = b[row] + acc;
    else y[row] = (b[row] - acc) * d[row];
  }
}

// ---------------------------------------------------------------------------
// Consistent-mass transfers (Sec. 3, App. B): y <- M_1^{-1} y along one grid
// direction, M_1 = L L^T the banded Cholesky factor of a 1D interior mass
// matrix of degree Q (half bandwidth Q), F[i*(Q+1)] = 1/L_ii and
// F[i*(Q+1) + k] = L_{i,i-k} (0 where i < k).  The interior mass matrix of a
// level is the Kronecker product of such matrices, so one pass per direction
// inverts it.  One thread a line of n entries: line t starts at
// (t / inner) * outer + t % inner and steps by stride.  Forward substitution
// writes z back into y, backward substitution writes y, or out = add + y
// when add is given (the prolongation's update).  Loads are issued eight
// entries ahead of the dependent chain; the factor rows are broadcasts.
// ---------------------------------------------------------------------------
template <int Q>
__global__ void __launch_bounds__(64) k_band_lines(int n, int nlines, long long inner, long long outer, long long stride,
                                                   const double* __restrict__ F, double* y,
                                                   const double* add, double* out) {
  constexpr int kB = 8;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nlines) return;
  double* yl = y + (t / inner) * outer + (t % inner);
  double h[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) h[k] = 0.0;
  // L z = y: z_i = (y_i - sum_k L_{i,i-k} z_{i-k}) / L_ii, h[k-1] = z_{i-k}
  for (int i0 = 0; i0 < n; i0 += kB) {
    double v[kB];
#pragma unroll
    for (int j = 0; j < kB; ++j) v[j] = (i0 + j < n) ? yl[(i0 + j) * stride] : 0.0;
#pragma unroll
    for (int j = 0; j < kB; ++j) {
      const int i = i0 + j;
      if (i < n) {
        const double* f = F + (size_t)i * (Q + 1);
        double s = v[j];
#pragma unroll
        for (int k = Q; k >= 1; --k) s = fma(-__ldg(f + k), h[k - 1], s);
        const double z = s * __ldg(f);
#pragma unroll
        for (int k = Q - 1; k >= 1; --k) h[k] = h[k - 1];
        h[0] = z;
        yl[i * stride] = z;
      }
    }
  }
  // L^T x = z: x_i = (z_i - sum_k L_{i+k,i} x_{i+k}) / L_ii, h[k-1] = x_{i+k}
#pragma unroll
  for (int k = 0; k < Q; ++k) h[k] = 0.0;
  const long long ofs = yl - y;
  for (int i0 = n - 1; i0 >= 0; i0 -= kB) {
    double v[kB], a[kB];
#pragma unroll
    for (int j = 0; j < kB; ++j) {
      const int i = i0 - j;
      v[j] = i >= 0 ? yl[i * stride] : 0.0;
      a[j] = (add && i >= 0) ? add[ofs + i * stride] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < kB; ++j) {
      const int i = i0 - j;
      if (i >= 0) {
        double s = v[j];
#pragma unroll
        for (int k = Q; k >= 1; --k)
          if (i + k < n) s = fma(-__ldg(F + (size_t)(i + k) * (Q + 1) + k), h[k - 1], s);
        const double x = s * __ldg(F + (size_t)i * (Q + 1));
#pragma unroll
        for (int k = Q - 1; k >= 1; --k) h[k] = h[k - 1];
        h[0] = x;
        if (add) out[ofs + i * stride] = a[j] + x;
        else yl[i * stride] = x;
      }
    }
  }
}

}  // namespace pmgk
