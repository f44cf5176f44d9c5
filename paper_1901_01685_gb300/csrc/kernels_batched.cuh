// Batched kernels: many right-hand sides of one hierarchy at once.
//
// Vectors are stored [row][R] with the right-hand sides fastest (R = padded
// count, a multiple of 32), so a warp handles one row for 32 right-hand sides
// with one lane per right-hand side: matrix entries are uniform across the
// warp (broadcast loads) and vector accesses are coalesced.  Value type T is
// double (plain FP64) or float (the inner cycle of FP64 defect correction).
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace pmgk {

template <class T>
struct TCsr {
  int nr;
  const int* rp;
  const int* ci;
  const T* v;
};

// "Not yet computed" markers for value-as-flag publication (all-ones NaNs).
template <class T>
struct Pending;
template <>
struct Pending<double> {
  using U = unsigned long long;
  static constexpr U bits = 0xFFFFFFFFFFFFFFFFull;
  __device__ static bool is(double v) { return (U)__double_as_longlong(v) == bits; }
};
template <>
struct Pending<float> {
  using U = unsigned int;
  static constexpr U bits = 0xFFFFFFFFu;
  __device__ static bool is(float v) { return (U)__float_as_uint(v) == bits; }
};

template <class T>
__device__ __forceinline__ T ld_relaxed_t(const T* p);
template <>
__device__ __forceinline__ double ld_relaxed_t<double>(const double* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return __longlong_as_double((long long)v);
}
template <>
__device__ __forceinline__ float ld_relaxed_t<float>(const float* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return __uint_as_float(v);
}

// Bounded poll of a pending value (global or shared memory).
template <class T, bool SHARED>
__device__ __forceinline__ T lpb_wait(const T* p, unsigned* err) {
  const long long t0 = clock64();
  for (unsigned it = 0;; ++it) {
    const T v = SHARED ? *reinterpret_cast<const volatile T*>(p) : ld_relaxed_t<T>(p);
    if (!Pending<T>::is(v)) return v;
    if (!SHARED) __nanosleep(it < 16 ? 32 : 256);
    if ((it & 31u) == 31u && (ld_relaxed(err) != 0u || clock64() - t0 > kWaitCycles)) {
      atomicOr(err, 1u);
      return T(0);
    }
  }
}

// Accumulation type: float only when both operands are float.
template <class A, class B>
struct AccT { using type = double; };
template <>
struct AccT<float, float> { using type = float; };

// Y = B - A X (MODE 0), A X (MODE 1), B + A X (MODE 2); A in TA, X in TX, B and Y in TY.
// One warp per (row, group of 32 right-hand sides).
template <class TA, class TX, class TY, int MODE>
__global__ void __launch_bounds__(256) k_spmm(TCsr<TA> A, int R, const TX* __restrict__ X, const TY* B, TY* Y) {
  const int lane = threadIdx.x & 31;
  const int G = R >> 5;
  const long long nwork = (long long)A.nr * G;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long w = w0; w < nwork; w += nw) {
    const int row = (int)(w / G), g = (int)(w % G);
    const int col = g * 32 + lane;
    using Acc = typename AccT<TA, TX>::type;
    const int beg = A.rp[row], end = A.rp[row + 1];
    Acc a0 = 0, a1 = 0;
    int t = beg;
    for (; t + 1 < end; t += 2) {
      a0 = fma((Acc)A.v[t], (Acc)X[(size_t)A.ci[t] * R + col], a0);
      a1 = fma((Acc)A.v[t + 1], (Acc)X[(size_t)A.ci[t + 1] * R + col], a1);
    }
    if (t < end) a0 = fma((Acc)A.v[t], (Acc)X[(size_t)A.ci[t] * R + col], a0);
    const Acc s = a0 + a1;
    const size_t o = (size_t)row * R + col;
    if (MODE == 0) Y[o] = (TY)((Acc)B[o] - s);
    else if (MODE == 1) Y[o] = (TY)s;
    else Y[o] = (TY)((Acc)B[o] + s);
  }
}

// Line-pipelined lower solve for 32 right-hand sides per warp (lane = RHS):
//   x_i = (b_i - sum_{j<i} M_ij x_j) d_i   (MIRROR: i -> n-1-i addressing).
// Each CTA claims B consecutive lines of one right-hand-side group (work items
// are claimed in order, so every line a CTA waits for belongs to a running
// CTA); warp w solves line base + w row by row.  Values of the CTA's lines live
// in shared memory; earlier lines are read from global memory.  Outputs start
// "pending" (all-ones bytes) and every read of another line polls the value
// itself (bounded), so no flags, counters or fences are needed.  UPDATE also
// adds x into u (the smoothing update).
constexpr int kLpbMaxLines = 4;

template <class T>
struct LpB {
  int n, nx, nlines;
  const int* rp;
  const int* ci;
  const T* v;
  const T* dscale;
};

template <class T>
__device__ __forceinline__ void st_relaxed_t(T* p, T v);
template <>
__device__ __forceinline__ void st_relaxed_t<double>(double* p, double v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"((unsigned long long)__double_as_longlong(v)) : "memory");
}
template <>
__device__ __forceinline__ void st_relaxed_t<float>(float* p, float v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(__float_as_uint(v)) : "memory");
}

template <class T, bool MIRROR, bool UPDATE>
__global__ void __launch_bounds__(32 * kLpbMaxLines) k_lpb(LpB<T> M, int R, const T* __restrict__ b, T* x, T* u,
                                                           unsigned* counter, unsigned* err) {
  extern __shared__ __align__(16) unsigned char lpb_smem[];
  // [lines per CTA][nx][32]: the values of the CTA's rows, row-major from its first row
  volatile T* xs = reinterpret_cast<volatile T*>(lpb_smem);
  __shared__ int s_item;
  const int nx = M.nx, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lines = blockDim.x >> 5;
  const int G = R >> 5;
  const int nblocks = (M.nlines + lines - 1) / lines;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
    for (int t = threadIdx.x; t < lines * nx * 32; t += blockDim.x)
      reinterpret_cast<volatile typename Pending<T>::U*>(lpb_smem)[t] = Pending<T>::bits;
    __syncthreads();
    const int item = s_item;
    if (item >= nblocks * G) return;
    const int blk = item / G, g = item % G;
    const int line = blk * lines + warp;
    if (line >= M.nlines) continue;
    const int base_row = blk * lines * nx;     // first row held in shared memory
    const int row0 = line * nx;
    const int col = g * 32 + lane;
    for (int i = row0; i < row0 + nx; ++i) {
      const int beg = __ldg(M.rp + i), end = __ldg(M.rp + i + 1);
      T a[4] = {T(0), T(0), T(0), T(0)};
      for (int t0 = beg; t0 < end; t0 += 8) {
        T xv[8], cv[8];
        int jj[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int t = t0 + q;
          jj[q] = t < end ? __ldg(M.ci + t) : -1;
          cv[q] = t < end ? __ldg(M.v + t) : T(0);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int j = jj[q];
          T v = T(0);
          if (j >= base_row) {
            // a row of this CTA: written by this lane (own line, never pending) or by another warp
            volatile T* p = xs + (size_t)(j - base_row) * 32 + lane;
            v = *p;
            if (Pending<T>::is(v)) v = lpb_wait<T, true>(const_cast<const T*>(p), err);
          } else if (j >= 0) {
            const T* p = x + (size_t)lp_vec<MIRROR>(j, M.n) * R + col;
            v = ld_relaxed_t<T>(p);
            if (Pending<T>::is(v)) v = lpb_wait<T, false>(p, err);
          }
          xv[q] = v;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q & 3] = fma(cv[q], xv[q], a[q & 3]);
      }
      const size_t o = (size_t)lp_vec<MIRROR>(i, M.n) * R + col;
      T xt = b[o] - ((a[0] + a[1]) + (a[2] + a[3]));
      if (M.dscale) xt *= __ldg(M.dscale + i);
      xs[(size_t)(i - base_row) * 32 + lane] = xt;
      st_relaxed_t<T>(x + o, xt);
      if (UPDATE) u[o] += xt;
    }
  }
}

// P1 canonical transfers, batched ([node][R]).
__global__ void k_p1_restrict_b(int d, int nf, int R, const double* __restrict__ rf, double* __restrict__ rc) {
  const int nc = nf / 2, mc = nc - 1, mf = nf - 1;
  const long long Nc = (d == 2) ? (long long)mc * mc : (long long)mc * mc * mc;
  const long long total = Nc * R;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long idx = t / R;
    const int r = (int)(t % R);
    const int cx = int(idx % mc) + 1, cy = int((idx / mc) % mc) + 1;
    const int cz = (d == 3) ? int(idx / ((long long)mc * mc)) + 1 : 0;
    double s = 0.0;
    for (int dz = (d == 3 ? -1 : 0); dz <= (d == 3 ? 1 : 0); ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          long long fi = (long long)(2 * cx + dx - 1) + (long long)mf * (2 * cy + dy - 1);
          if (d == 3) fi += (long long)mf * mf * (2 * cz + dz - 1);
          s += hat_w(dx) * hat_w(dy) * (d == 3 ? hat_w(dz) : 1.0) * rf[fi * R + r];
        }
    rc[t] = s;
  }
}

__global__ void k_p1_prolong_add_b(int d, int nf, int R, const double* __restrict__ ec, double* __restrict__ xf) {
  const int nc = nf / 2, mc = nc - 1, mf = nf - 1;
  const long long Nf = (d == 2) ? (long long)mf * mf : (long long)mf * mf * mf;
  const long long total = Nf * R;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long idx = t / R;
    const int r = (int)(t % R);
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
          s += pw[0][ix] * pw[1][iy] * pw[2][iz] * ec[ci * R + r];
        }
    xf[t] += s;
  }
}

// X = Ainv B for the coarsest level (dense), one warp per (row, group).
__global__ void k_dense_mm(int n, int R, const double* __restrict__ Ainv, const double* __restrict__ B,
                           double* __restrict__ X) {
  const int lane = threadIdx.x & 31, G = R >> 5;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long w = w0; w < (long long)n * G; w += nw) {
    const int row = (int)(w / G), col = (int)(w % G) * 32 + lane;
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += Ainv[(size_t)row * n + j] * B[(size_t)j * R + col];
    X[(size_t)row * R + col] = s;
  }
}

// Per-right-hand-side squared norms: fixed partition into kNormBlocks row
// chunks; partial[b][r]; then a fixed-order combination per right-hand side.
__global__ void k_sqnorm_partial_b(int n, int R, const double* __restrict__ r, double* __restrict__ partial) {
  const long long chunk = (n + (long long)gridDim.x - 1) / gridDim.x;
  const long long beg = blockIdx.x * chunk, end = min((long long)n, beg + chunk);
  for (int c = threadIdx.x; c < R; c += blockDim.x) {
    double s = 0.0;
    for (long long i = beg; i < end; ++i) {
      const double v = r[i * R + c];
      s += v * v;
    }
    partial[(size_t)blockIdx.x * R + c] = s;
  }
}
// MODE 0: r0[c] = sqrt(sum); MODE 1: out[c] = sqrt(sum) / r0[c] (0 if r0 == 0).
template <int MODE>
__global__ void k_norm_finalize_b(int nparts, int R, const double* __restrict__ partial, double* r0, double* out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < R; c += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += partial[(size_t)b * R + c];
    const double nrm = sqrt(s);
    if (MODE == 0) r0[c] = nrm;
    else out[c] = r0[c] > 0.0 ? nrm / r0[c] : 0.0;
  }
}

// Layout conversions between the caller's [nrhs][n] and the internal [n][R].
__global__ void k_to_rows(int n, int nrhs, int R, const double* __restrict__ src, double* __restrict__ dst) {
  const long long total = (long long)n * R;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long i = t / R;
    const int c = (int)(t % R);
    dst[t] = c < nrhs ? src[(size_t)c * n + i] : 0.0;
  }
}
__global__ void k_from_rows(int n, int nrhs, int R, const double* __restrict__ src, double* __restrict__ dst) {
  const long long total = (long long)n * nrhs;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t / n);
    const long long i = t % n;
    dst[t] = src[i * R + c];
  }
}

// y = (T) x, and u += mask[c] * x (FP64 update of the active right-hand sides).
template <class TI, class TO>
__global__ void k_cast(long long total, const TI* __restrict__ x, TO* __restrict__ y) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x)
    y[t] = (TO)x[t];
}
template <class TI>
__global__ void k_masked_update(long long n, int R, const TI* __restrict__ e, const double* __restrict__ mask,
                                double* __restrict__ u) {
  const long long total = n * R;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x)
    u[t] += mask[t % R] * (double)e[t];
}
template <class T>
__global__ void k_axpy(long long total, const T* __restrict__ x, T* __restrict__ y) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x)
    y[t] += x[t];
}

}  // namespace pmgk
