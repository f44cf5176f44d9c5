// Batched kernels: many right-hand sides of one hierarchy at once.
//
// Vectors are stored [row][R] with the right-hand sides fastest (R = padded
// count, a multiple of 32), so a warp handles one row for 32 right-hand sides
// with one lane per right-hand side: matrix entries are uniform across the
// warp (broadcast loads) and vector accesses are coalesced.  Value type T is
// double (plain FP64) or float (the inner cycle of FP64 defect correction).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
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
  __device__ static double other_nan() { return __longlong_as_double(0x7FF8000000000000ll); }
};
template <>
struct Pending<float> {
  using U = unsigned int;
  static constexpr U bits = 0xFFFFFFFFu;
  __device__ static bool is(float v) { return (U)__float_as_uint(v) == bits; }
  __device__ static float other_nan() { return __uint_as_float(0x7FC00000u); }
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

// Bounded poll of a pending value (global or shared memory).  On expiry the
// error word gets bit `site` (which wait gave up) and the value reads as 0.
enum : unsigned { kSiteGlobal = 1u, kSiteShared = 2u, kSiteSlotFree = 4u, kSiteSlotFilled = 8u };
// err[0] collects the bits of every wait that gave up; the first one to give
// up also records (site, work item, row, warp) in err[1..3].
__device__ __forceinline__ void wait_expired(unsigned* err, unsigned site, int item, int row) {
  if (atomicCAS(err + 1, 0u, site) == 0u) {
    err[2] = (unsigned)item;
    err[3] = ((unsigned)row << 8) | (threadIdx.x >> 5);
  }
  atomicOr(err, site);
}

template <class T, bool SHARED>
__device__ __forceinline__ T lpb_wait(const T* p, unsigned* err, unsigned site = SHARED ? kSiteShared : kSiteGlobal,
                                      int item = -1, int row = -1) {
  const long long t0 = clock64();
  for (unsigned it = 0;; ++it) {
    const T v = SHARED ? *reinterpret_cast<const volatile T*>(p) : ld_relaxed_t<T>(p);
    if (!Pending<T>::is(v)) return v;
    // Global waits back off (32 ns for 16 polls, then 256 ns); longer or
    // exponential back-off measured slower on the pipeline front.
    if (!SHARED) __nanosleep(it < 16 ? 32u : 256u);
    if ((it & 31u) == 31u && (ld_relaxed(err) != 0u || clock64() - t0 > kWaitCycles)) {
      wait_expired(err, site, item, row);
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
        // rows of this CTA (written by this lane or by another warp) from shared
        // memory, earlier rows from global memory: issue all loads, then resolve
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int j = jj[q];
          xv[q] = T(0);
          if (j >= base_row) xv[q] = xs[(size_t)(j - base_row) * 32 + lane];
          else if (j >= 0) xv[q] = ld_relaxed_t<T>(x + (size_t)lp_vec<MIRROR>(j, M.n) * R + col);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (Pending<T>::is(xv[q])) {
            const int j = jj[q];
            xv[q] = j >= base_row ? lpb_wait<T, true>(const_cast<const T*>(xs + (size_t)(j - base_row) * 32 + lane), err)
                                  : lpb_wait<T, false>(x + (size_t)lp_vec<MIRROR>(j, M.n) * R + col, err);
          }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q & 3] = fma(cv[q], xv[q], a[q & 3]);
      }
      const size_t o = (size_t)lp_vec<MIRROR>(i, M.n) * R + col;
      T xt = b[o] - ((a[0] + a[1]) + (a[2] + a[3]));
      if (M.dscale) xt *= __ldg(M.dscale + i);
      if (Pending<T>::is(xt)) xt = Pending<T>::other_nan();   // never publish the marker
      xs[(size_t)(i - base_row) * 32 + lane] = xt;
      st_relaxed_t<T>(x + o, xt);
      if (UPDATE) u[o] += xt;
    }
  }
}

// Line-pipelined lower solve, 32 right-hand sides per item (lane = RHS; or
// one vector when R == 1), with
// the own-line recurrence split off the critical path (ring width W <= 32):
//   x_i = s_i - sum_{k=1..W-1} c_{i-k,k} x_{i-k},
//   s_i = d_i b_i - sum_{far j} d_i M_ij x_j,     c_{j,k} = d_{j+k} M_{j+k,j}
// (the "ring" entries are those of the row's own line at distance 1..W-1; all
// others are "far").  One CTA takes one line of one right-hand-side group:
//  - LpcProducers<T> producer warps compute s_i for rows p, p+P, ... and hand
//    them over, with the row's ring coefficients, through a 32-slot
//    shared-memory ring (slot pending = empty);
//  - one chain warp keeps W running sums per lane in registers (push form:
//    after x_i is known, every later row of the ring receives c_{i,k} x_i), so
//    one row costs one subtraction and one FMA on its critical path.
// Rows of the CTA's own line are read by the producers from shared memory,
// rows of earlier lines from global memory; both start "pending" (all-ones
// bits) and every read of a pending value polls, bounded.  Items are claimed
// in order (line-major), so every item waited for belongs to a running CTA.
// Producer warps per CTA.  The count must divide 32: hand-over slot k then
// always belongs to the same producer, which fills it in row order, so a
// pending (empty) slot unambiguously means that its previous row has been
// taken by the chain.
template <class T>
struct LpcProducers { static constexpr int value = 8; };
static_assert(32 % LpcProducers<float>::value == 0 && 32 % LpcProducers<double>::value == 0,
              "producer count must divide the 32 hand-over slots");

// CT: storage type of the factor coefficients (T, or FP16 / BF16 with T = float:
// stored at 16 bits, widened on load, accumulated in T).
template <class T, class CT = T>
struct LpC {
  int n, nx, nlines;
  int ring;           // ring width: own-line entries at distance 1..ring-1 are pushed
  const int* frp;
  const int* fci;
  const CT* fv;       // far entries, values scaled by d_i
  const CT* push;     // [n][32]: push[j*32 + k-1] = c_{j,k}
  const T* dscale;    // d_i, or null when d = 1
};

__device__ __forceinline__ float coef_ld(const float* p) { return __ldg(p); }
__device__ __forceinline__ double coef_ld(const double* p) { return __ldg(p); }
__device__ __forceinline__ float coef_ld(const __half* p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ float coef_ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }

// The first NC coefficients of a hand-over row in shared memory (16-byte aligned).
template <int NC>
__device__ __forceinline__ void lds_row(const float* p, float (&c)[NC]) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int m = 0; m < (NC + 3) / 4; ++m) {
    const float4 v = q[m];
    if (4 * m < NC) c[4 * m] = v.x;
    if (4 * m + 1 < NC) c[4 * m + 1] = v.y;
    if (4 * m + 2 < NC) c[4 * m + 2] = v.z;
    if (4 * m + 3 < NC) c[4 * m + 3] = v.w;
  }
}
template <int NC>
__device__ __forceinline__ void lds_row(const double* p, double (&c)[NC]) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int m = 0; m < (NC + 1) / 2; ++m) {
    const double2 v = q[m];
    if (2 * m < NC) c[2 * m] = v.x;
    if (2 * m + 1 < NC) c[2 * m + 1] = v.y;
  }
}

// Warp-uniform wait: every lane's value at p (shared memory when SHARED,
// else a relaxed global load) until no lane of the warp has one pending.
// All lanes loop together; a per-lane spin would leave the warp split into
// thread groups that issue every later instruction separately (measured
// several times slower on GB300).
template <class T, bool SHARED>
__device__ __noinline__ T lpc_wait_uniform(const T* p, T v, unsigned* err, unsigned site, int item, int row) {
  const long long t0 = clock64();
  for (unsigned it = 0;; ++it) {
    if (Pending<T>::is(v)) v = SHARED ? *reinterpret_cast<const volatile T*>(p) : ld_relaxed_t<T>(p);
    if (!__any_sync(0xffffffffu, Pending<T>::is(v))) return v;
    if (!SHARED) __nanosleep(it < 16 ? 32u : 256u);
    if ((it & 31u) == 31u) {
      const bool expired = ld_relaxed(err) != 0u || clock64() - t0 > kWaitCycles;
      if (__any_sync(0xffffffffu, expired)) {
        if (Pending<T>::is(v)) {
          wait_expired(err, site, item, row);
          v = T(0);
        }
        return v;
      }
    }
  }
}

// Producer warp pw of k_lpc: rows pw, pw + P, ... of the line; for each,
// s_i = d_i b_i - sum_far d_i M_ij x_j, handed to the chain with the row's
// ring coefficients through hand-over slot (i mod 32).  Called out of line:
// inlined into the kernel, producer code made the compiler emit a slower
// chain loop.
template <class T, bool MIRROR, int RING, class CT>
__device__ __noinline__ void lpc_producer(LpC<T, CT> M, int R, const T* __restrict__ b, T* x, volatile T* xs,
                                          volatile T* sb, T* cb, int row0, int col, int item, int pw, int lane,
                                          unsigned* err) {
  constexpr int NC = RING - 1;
  constexpr int BATCH = sizeof(T) == 4 ? 32 : 16;
  const int nx = M.nx;
  for (int ix = pw; ix < nx; ix += LpcProducers<T>::value) {
    const int i = row0 + ix;
    const size_t o = (size_t)lp_vec<MIRROR>(i, M.n) * R + col;
    const T bi = M.dscale ? b[o] * __ldg(M.dscale + i) : b[o];
    const T cf = lane < NC ? (T)coef_ld(M.push + (size_t)i * 32 + lane) : T(0);
    const int beg = __ldg(M.frp + i), end = __ldg(M.frp + i + 1);
    T a[4] = {T(0), T(0), T(0), T(0)};
    for (int t0 = beg; t0 < end; t0 += BATCH) {
      int jj[BATCH];
      T cv[BATCH], xv[BATCH];
#pragma unroll
      for (int q = 0; q < BATCH; ++q) {
        const int t = t0 + q;
        jj[q] = t < end ? __ldg(M.fci + t) : -1;
        cv[q] = t < end ? (T)coef_ld(M.fv + t) : T(0);
      }
      // Issue every load of the batch first (own line from shared memory,
      // earlier lines with relaxed loads at GPU scope, which read L2: x is
      // written during this kernel), then wait, warp-uniformly, for the
      // pending ones.
      bool pend = false;
#pragma unroll
      for (int q = 0; q < BATCH; ++q) {
        const int j = jj[q];
        xv[q] = T(0);
        if (j >= row0) xv[q] = xs[(size_t)(j - row0) * 32 + lane];
        else if (j >= 0) xv[q] = ld_relaxed_t<T>(x + (size_t)lp_vec<MIRROR>(j, M.n) * R + col);
        pend |= Pending<T>::is(xv[q]);
      }
      if (__any_sync(0xffffffffu, pend)) {
        const long long tw = clock64();
        for (unsigned it = 0;; ++it) {
          pend = false;
#pragma unroll
          for (int q = 0; q < BATCH; ++q)
            if (Pending<T>::is(xv[q])) {
              const int j = jj[q];
              xv[q] = j >= row0 ? xs[(size_t)(j - row0) * 32 + lane]
                                : ld_relaxed_t<T>(x + (size_t)lp_vec<MIRROR>(j, M.n) * R + col);
              pend |= Pending<T>::is(xv[q]);
            }
          if (!__any_sync(0xffffffffu, pend)) break;
          __nanosleep(it < 16 ? 32u : 256u);
          if ((it & 31u) == 31u) {
            const bool expired = ld_relaxed(err) != 0u || clock64() - tw > kWaitCycles;
            if (__any_sync(0xffffffffu, expired)) {
              if (pend) wait_expired(err, kSiteGlobal, item, ix);
#pragma unroll
              for (int q = 0; q < BATCH; ++q)
                if (Pending<T>::is(xv[q])) xv[q] = T(0);
              break;
            }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < BATCH; ++q) a[q & 3] = fma(cv[q], xv[q], a[q & 3]);
    }
    const T s = bi - ((a[0] + a[1]) + (a[2] + a[3]));
    volatile T* slot = sb + (ix & 31) * 32 + lane;
    // wait, warp-uniformly, for the chain to have taken row ix - 32 out of
    // every lane's slot (bounded)
    const long long t0 = clock64();
    for (unsigned it = 0; __any_sync(0xffffffffu, !Pending<T>::is(*slot)); ++it) {
      if ((it & 31u) == 31u) {
        const bool expired = ld_relaxed(err) != 0u || clock64() - t0 > kWaitCycles;
        if (__any_sync(0xffffffffu, expired)) {
          if (lane == 0) wait_expired(err, kSiteSlotFree, item, ix);
          break;
        }
      }
    }
    // The chain's lane L reads the coefficients of all lanes: every
    // coefficient is written before any lane publishes s.
    __syncwarp();
    cb[(ix & 31) * 32 + lane] = cf;
    __syncwarp();
    __threadfence_block();
    *slot = s;
  }
}

template <class T, bool MIRROR, int RING, class CT = T>
__global__ void __launch_bounds__(32 * (1 + LpcProducers<T>::value)) k_lpc(LpC<T, CT> M, int R, const T* __restrict__ b, T* x,
                                                                   unsigned* counter, unsigned* err) {
  static_assert(RING >= 2 && RING <= 32 && (RING & (RING - 1)) == 0, "ring must be a power of two <= 32");
  constexpr int NC = RING - 1;
  extern __shared__ __align__(16) unsigned char lpc_smem[];
  using PU = typename Pending<T>::U;
  volatile T* xs = reinterpret_cast<volatile T*>(lpc_smem);   // [nx][32] values of the line
  volatile T* sb = xs + (size_t)M.nx * 32;                    // [32][32] hand-over ring: s_i
  T* cb = const_cast<T*>(sb) + 32 * 32;                        // [32][32] hand-over ring: c_{i,.}
  __shared__ int s_item;
  const int nx = M.nx, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // R == 1: one plain vector, every lane computes the same values (loads are
  // broadcasts, stores coincide)
  const bool single = R == 1;
  const int G = single ? 1 : R >> 5;
  const int nitems = M.nlines * G;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
    for (int t = threadIdx.x; t < (nx + 32) * 32; t += blockDim.x)
      reinterpret_cast<volatile PU*>(lpc_smem)[t] = Pending<T>::bits;
    __syncthreads();
    const int item = s_item;
    if (item >= nitems) return;
    const int line = item / G, g = item % G;
    const int row0 = line * nx, col = single ? 0 : g * 32 + lane;
    if (warp != 0) {
      lpc_producer<T, MIRROR, RING, CT>(M, R, b, x, xs, sb, cb, row0, col, item, warp - 1, lane, err);
      continue;
    }
    // ------------------------------- chain -------------------------------
    T acc[RING];
#pragma unroll
    for (int k = 0; k < RING; ++k) acc[k] = T(0);
    for (int i0 = 0; i0 < nx; i0 += 32) {
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        const int ix = i0 + k;
        if (ix < nx) {
          volatile T* slot = sb + k * 32 + lane;
          T s = *slot;
          if (__any_sync(0xffffffffu, Pending<T>::is(s)))
            s = lpc_wait_uniform<T, true>(const_cast<const T*>(slot), s, err, kSiteSlotFilled, item, ix);
          __threadfence_block();              // the row's coefficients were written before s
          T c[NC];
          lds_row<NC>(cb + k * 32, c);
          const int a0 = k & (RING - 1);
          T xv = s - acc[a0];
          if (Pending<T>::is(xv)) xv = Pending<T>::other_nan();   // never publish the marker
          acc[a0] = T(0);
#pragma unroll
          for (int m = 1; m < RING; ++m) acc[(k + m) & (RING - 1)] = fma(c[m - 1], xv, acc[(k + m) & (RING - 1)]);
          // the pushes consumed c: release the slot to its producer
          *reinterpret_cast<volatile PU*>(slot) = Pending<T>::bits;
          xs[(size_t)ix * 32 + lane] = xv;
          st_relaxed_t<T>(x + (size_t)lp_vec<MIRROR>(row0 + ix, M.n) * R + col, xv);
        }
      }
    }
  }
}

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
// Continuous-batching slot bookkeeping.  state: 0 free, 1 active, 2 converged,
// 3 diverged; an active slot has mask 1 (its u is updated by the cycle).
__global__ void k_slots_copy_in(int n, int nload, int R, int slot0, const double* __restrict__ src,
                                double* __restrict__ dst) {
  const long long total = (long long)n * nload;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long i = t / nload;
    const int c = (int)(t % nload);
    dst[i * R + slot0 + c] = src[(size_t)c * n + i];
  }
}
__global__ void k_slots_copy_out(int n, int nread, int R, int slot0, const double* __restrict__ src,
                                 double* __restrict__ dst) {
  const long long total = (long long)n * nread;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t / n);
    const long long i = t % n;
    dst[t] = src[i * R + slot0 + c];
  }
}
// r0 of newly loaded slots; a zero initial residual converges at once.
__global__ void k_slots_start(int nparts, int R, int slot0, int nload, const double* __restrict__ partial, double* r0,
                              double* relres, double* mask, int* state, int* iters) {
  for (int c = slot0 + blockIdx.x * blockDim.x + threadIdx.x; c < slot0 + nload; c += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += partial[(size_t)b * R + c];
    const double nrm = sqrt(s);
    r0[c] = nrm;
    iters[c] = 0;
    relres[c] = nrm > 0.0 ? 1.0 : 0.0;
    state[c] = nrm > 0.0 ? 1 : 2;
    mask[c] = nrm > 0.0 ? 1.0 : 0.0;
  }
}
// After a cycle: relative residual of every active slot, then its stopping test (Sec. 5).
__global__ void k_slots_update(int nparts, int R, double tol, const double* __restrict__ partial,
                               const double* __restrict__ r0, double* relres, double* mask, int* state, int* iters) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < R; c += gridDim.x * blockDim.x) {
    if (state[c] != 1) continue;
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += partial[(size_t)b * R + c];
    const double rel = sqrt(s) / r0[c];
    relres[c] = rel;
    iters[c] += 1;
    if (rel < tol) { state[c] = 2; mask[c] = 0.0; }
    else if (!(rel <= 1e10)) { state[c] = 3; mask[c] = 0.0; }
  }
}
__global__ void k_slots_release(int R, int slot0, int n, double* mask, int* state) {
  for (int c = slot0 + blockIdx.x * blockDim.x + threadIdx.x; c < slot0 + n; c += gridDim.x * blockDim.x) {
    state[c] = 0;
    mask[c] = 0.0;
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
__global__ void k_fill(long long total, T v, T* __restrict__ y) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x)
    y[t] = v;
}
template <class T>
__global__ void k_axpy(long long total, const T* __restrict__ x, T* __restrict__ y) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x)
    y[t] += x[t];
}

}  // namespace pmgk
