// C-ABI and V-cycle driver of the GB300 p-multigrid solver (see include/pmg.h).
//
// The host builds the hierarchy once (setup.cpp); pmg_upload packs it into a
// caller-owned device arena; every solve step then runs in the CUDA kernels of
// kernels.cuh on the caller's stream.  The only host<->device traffic per
// V-cycle is the 8-byte relative residual read for the stopping test.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/pmg.h"
#include "kernels.cuh"
#include "kernels_batched.cuh"
#include "kernels_krylov.cuh"
#include "setup.h"

namespace {

thread_local std::string g_last_error;

pmg_status fail(pmg_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

#define PMG_CUDA(call)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return fail(PMG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

constexpr size_t kAlign = 256;
constexpr int kCounterSlots = 256;
constexpr int kHistCap = 1024;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Layout planner: records (offset, host source, bytes) for every array.
struct Packer {
  size_t size = 0;
  struct Item { size_t off; const void* src; size_t bytes; };
  std::vector<Item> items;
  size_t add(const void* src, size_t bytes) {
    size_t off = size;
    items.push_back({off, src, bytes});
    size = align_up(size + std::max<size_t>(bytes, 1));
    return off;
  }
};

struct DevCsrOff { int nr; long long nnz; size_t rp, ci, v; };

// Sliced-ELL copy of a CSR matrix (k_sell): host arrays, kept until upload.
struct SellHost {
  int nr = 0, nslices = 0;
  std::vector<long long> sofs;
  std::vector<int> col;
  std::vector<double> val;
};
SellHost make_sell(const pmgl::Csr& a) {
  SellHost S;
  S.nr = a.nr;
  S.nslices = (a.nr + 31) / 32;
  S.sofs.assign(size_t(S.nslices) + 1, 0);
  for (int s = 0; s < S.nslices; ++s) {
    int w = 0;
    for (int r = s * 32; r < std::min(a.nr, s * 32 + 32); ++r) w = std::max(w, a.rp[r + 1] - a.rp[r]);
    w = (w + 3) / 4 * 4;
    S.sofs[size_t(s) + 1] = S.sofs[size_t(s)] + 32LL * w;
  }
  S.col.assign(size_t(S.sofs.back()), -1);
  S.val.assign(size_t(S.sofs.back()), 0.0);
  for (int s = 0; s < S.nslices; ++s) {
    const long long base = S.sofs[size_t(s)];
    for (int lane = 0; lane < 32; ++lane) {
      const int r = s * 32 + lane;
      if (r >= a.nr) continue;
      for (int k = a.rp[r]; k < a.rp[r + 1]; ++k) {
        const int e = k - a.rp[r], g = e / 4, t = e % 4;
        const long long grp = base + 128LL * g;
        S.col[size_t(grp + 4 * lane + t)] = a.ci[k];
        // values: entries 0, 1 of every lane, then entries 2, 3 of every lane
        S.val[size_t(grp + (t < 2 ? 0 : 64) + 2 * lane + (t & 1))] = a.v[k];
      }
    }
  }
  return S;
}
struct SellOff { int nr, nslices; size_t sofs, col, val; };

DevCsrOff plan_csr(Packer& P, const pmgl::Csr& a) {
  DevCsrOff o;
  o.nr = a.nr;
  o.nnz = a.nnz();
  o.rp = P.add(a.rp.data(), a.rp.size() * sizeof(int));
  o.ci = P.add(a.ci.data(), a.ci.size() * sizeof(int));
  o.v = P.add(a.v.data(), a.v.size() * sizeof(double));
  return o;
}

pmgk::Csr bind(const DevCsrOff& o, char* base) {
  return pmgk::Csr{o.nr, reinterpret_cast<const int*>(base + o.rp), reinterpret_cast<const int*>(base + o.ci),
                   reinterpret_cast<const double*>(base + o.v)};
}

// Arena offsets of one line-pipelined layout.
struct LpOff { int n, nx, nlines, nwin, lpr, win; size_t wofs, wcol, wval, waitofs, wait, push, dscale; };

LpOff plan_lp(Packer& P, const pmgl::LpLayout& L) {
  LpOff o{L.n, L.nx, L.nlines, L.nwin, L.lpr, L.win, 0, 0, 0, 0, 0, 0, 0};
  o.wofs = P.add(L.wofs.data(), L.wofs.size() * sizeof(int));
  o.wcol = P.add(L.wcol.data(), L.wcol.size() * sizeof(int));
  o.wval = P.add(L.wval.data(), L.wval.size() * sizeof(double));
  o.waitofs = P.add(L.waitofs.data(), L.waitofs.size() * sizeof(int));
  o.wait = P.add(L.wait.data(), L.wait.size() * sizeof(int));
  o.push = P.add(L.push.data(), L.push.size() * sizeof(double));
  o.dscale = P.add(L.dscale.data(), L.dscale.size() * sizeof(double));
  return o;
}

pmgk::Lp2 bind_lp(const LpOff& o, char* base) {
  return pmgk::Lp2{o.n, o.nx, o.nlines, o.nwin, o.lpr, o.win,
                   reinterpret_cast<const int*>(base + o.wofs), reinterpret_cast<const int*>(base + o.wcol),
                   reinterpret_cast<const double*>(base + o.wval), reinterpret_cast<const int*>(base + o.waitofs),
                   reinterpret_cast<const int*>(base + o.wait), reinterpret_cast<const double*>(base + o.push),
                   reinterpret_cast<const double*>(base + o.dscale)};
}

constexpr size_t kLpSmemCap = 200 * 1024;

// Consistent-mass transfers: banded Cholesky factors of the 1D interior mass
// matrices of a level (first direction, the others), n interior functions a
// direction, degree q.  f0 == nullptr: lumped transfers.
struct MassF {
  const double* f0 = nullptr;
  const double* f1 = nullptr;
  int n = 0, q = 0;
};
struct DevPLevel {
  int N = 0;
  double avg_nnz = 0;
  long long nnzA = 0, nnzL = 0, nnzU = 0, nnzP = 0;
  pmgk::Csr A{}, L{}, U{}, Pro{}, Res{};
  pmgk::Sell sA{}, sPro{}, sRes{};   // sliced-ELL copies for the residual and the transfers
  const double* udinv = nullptr;
  pmgk::Lp2 Llp{}, Ulp{};         // line-pipelined layouts (U mirrored)
  // batched solves: FP32 copies for the inner cycle, plain CSR layouts
  pmgk::TCsr<float> A32{}, Res32{}, Pro32{};
  pmgk::LpB<double> Lb64{}, Ub64{};
  pmgk::LpB<float> Lb32{}, Ub32{};
  pmgk::LpC<double> Lc64{}, Uc64{};   // ring kernel layouts (U mirrored)
  pmgk::LpC<float> Lc32{}, Uc32{};
  pmgk::LpC<float, __half> Lc16{}, Uc16{};           // FP16 / BF16 factor storage, FP32 arithmetic
  pmgk::LpC<float, __nv_bfloat16> Lcb{}, Ucb{};
  int inflightL = 0, inflightU = 0;    // lines of one group the solve's pipeline keeps busy at once
  MassF mass{};                        // consistent transfers: factors of this level's mass matrix
};
// Kernel variant of each solve: the line-pipelined windowed kernel (single
// vectors), the ring kernel, or the lines-per-CTA kernel (batched).  Defaults
// are the measured best on GB300; pmg_autotune re-measures them.
enum : unsigned char { kVarLp2 = 0, kVarRing = 1, kVarLines = 2, kVarCluster = 3 };
// single-vector sweeps of 2D P1 levels: value 2 selects the wavefront kernel
constexpr unsigned char kVarWave = kVarLines;
// Chain configurations of the clustered kernel k_lp4: producer sums enter the
// chain in groups of G rows, A+1 .. A+G rows ahead; a cluster takes NL
// consecutive lines at a time.
struct Lp4Cfg { int G, A, NL; };
constexpr Lp4Cfg kLp4Cfgs[] = {{1, 1, 1}, {2, 1, 1}, {4, 1, 1}, {8, 1, 1}, {2, 1, 2}, {4, 1, 2}, {2, 1, 4}, {4, 1, 4}};
constexpr int kNumLp4Cfgs = 8;
struct PTune {
  unsigned char sL = kVarCluster, sU = kVarCluster;   // single vector: forward / backward ILUT solve
  unsigned char cL = 7, cU = 7;                       // k_lp4 chain configuration (index into kLp4Cfgs)
  unsigned char bL[2] = {kVarRing, kVarRing};         // batched, [0] FP64, [1] FP32
  unsigned char bU[2] = {kVarRing, kVarRing};
};
struct HTune {
  unsigned char gF = kVarWave, gB = kVarWave;         // single vector: forward / backward sweep
  unsigned char cF = 7, cB = 7;                       // k_lp4 chain configuration of the sweeps
  unsigned char bF = kVarRing, bB = kVarRing;         // batched
};

struct DevHLevel {
  int N = 0, ne = 0;
  long long nnzA = 0;
  pmgk::Csr A{}, Lo{}, Up{};
  const double* dinv = nullptr;
  pmgk::Lp2 Lolp{}, UpMlp{};
  double avg_lo = 0, avg_up = 0;
  pmgk::LpB<double> Lob{}, UpMb{};   // batched Gauss-Seidel layouts
  pmgk::LpC<double> Loc{}, UpMc{};
  int inflightGS = 0;
  const double* wave_f = nullptr;    // wavefront sweep coefficients (2D levels), forward / backward
  const double* wave_b = nullptr;
};

}  // namespace

struct pmg_hierarchy_s {
  pmgl::Hierarchy H;
  std::vector<double> udinv_host[PMG_MAX_LEVELS];
  Packer pack;
  std::vector<DevCsrOff> off_A, off_L, off_U, off_Pro, off_Res, off_HA;
  std::vector<size_t> off_udinv, off_dinv;
  std::vector<DevCsrOff> off_Lo, off_Up;
  std::vector<LpOff> off_Llp, off_Ulp, off_Lolp, off_UpMlp;
  // batched / mixed-precision data (host copies owned here until upload)
  std::vector<std::vector<float>> f32store;
  struct BOff { DevCsrOff Um; size_t A32, Res32, Pro32, L32, Um32, udm64, udm32; };
  std::vector<BOff> boff;
  struct HBOff { DevCsrOff UpM; size_t dinvM; };
  std::vector<HBOff> hboff;
  // ring kernel layouts: far parts (FP64 CSR + FP32 values), FP32 push rings and scales
  std::vector<pmgl::Csr> farstore;
  struct COff { DevCsrOff far; int ring; size_t far32, push32, d32, far16, push16, farb, pushb; };
  std::vector<std::vector<uint16_t>> h16store;     // FP16 / BF16 bit patterns of the factors
  std::vector<COff> coffL, coffU, coffL32, coffU32, coffLo, coffUpM;
  std::vector<std::vector<double>> wavestore;      // wavefront sweep coefficients (host copies until upload)
  std::vector<SellHost> sellstore;                  // sliced-ELL copies of A, P, R per level (host, until upload)
  std::vector<SellOff> soffA, soffPro, soffRes;
  struct WOff { size_t f, b; bool ok; };
  std::vector<WOff> woff;
  size_t off_cinv = 0;
  struct MOff { size_t f0, f1; int n, q; };
  std::vector<MOff> moff;             // consistent transfers: per p-level, then V_{h,1}
  MassF mass1{};                      // factors of V_{h,1}'s mass matrix (consistent transfers)
  bool uploaded = false;
  char* arena = nullptr;
  std::vector<DevPLevel> dl;
  std::vector<DevHLevel> dh;
  std::vector<PTune> ptune;
  std::vector<HTune> htune;
  unsigned tune_epoch = 0;           // bumped when a kernel choice changes (captured graphs go stale)
  const double* cinv = nullptr;
  int sms = 0;
};

struct pmg_workspace_s {
  pmg_hierarchy_s* h = nullptr;
  int max_rhs = 1;
  // per p-level buffers
  std::vector<double*> f, u, r, y, e;
  // P1 levels
  std::vector<double*> hb, hx, hr, hg;
  // batched solves (max_rhs > 1): [row][R] buffers, R = max_rhs rounded up to 32
  int R = 0;
  std::vector<double*> bf, be, br, by, bt;      // per p-level (reused as float for the inner cycle)
  std::vector<double*> bhb, bhx, bhr, bhg, bht; // per P1 level (FP64)
  double *bF = nullptr, *bU = nullptr, *bR = nullptr;
  double *br0 = nullptr, *brel = nullptr, *bmask = nullptr, *bpart = nullptr;
  // continuous batching: per-slot state and iteration count (device), and the
  // pinned host mirror the end of each cycle is copied into
  int *bstate = nullptr, *biters = nullptr;
  struct SlotMirror { double* relres; int* state; int* iters; unsigned* err; };
  SlotMirror hm{nullptr, nullptr, nullptr, nullptr};
  void* hm_block = nullptr;
  std::vector<int> slot_state;      // host view of the slot states after the last wait / load
  cudaEvent_t slot_ev = nullptr;
  bool slot_pending = false;
  // CUDA-graph replay of the slot cycle, per precision
  struct CycleGraph { cudaGraphExec_t exec = nullptr; double tol = 0; unsigned epoch = 0; long long launches = 0; int eager = 0; };
  CycleGraph cyc[4];
  bool graphs = true;
  long long graph_launches = 0;
  double* kv[8] = {nullptr};          // BiCGSTAB vectors (level 0): r, r-hat, p, v, s, t, p-hat, s-hat
  double* kd = nullptr;                // BiCGSTAB scalar results
  unsigned* flags = nullptr;
  unsigned long long* lprog = nullptr;   // per-line progress words of the line-pipelined solves
  unsigned* counters = nullptr;
  unsigned* err = nullptr;
  double* partial = nullptr;
  double* r0 = nullptr;
  double* hist = nullptr;
  double* f_in = nullptr;   // host-path input staging
  double* u_io = nullptr;
  unsigned epoch = 0;
  int next_slot = 0;
  // launch statistics (per-kernel CUDA-event timing when prof is on)
  bool prof = false;
  struct Pending { int cls; cudaEvent_t a, b; double bytes; };
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<Pending> pending;
  double prof_ms[PMG_NKERN] = {0};
  long long prof_n[PMG_NKERN] = {0};
  double prof_bytes[PMG_NKERN] = {0};
  long long launches = 0;
  // first failed stream-ordered runtime call (fill, copy) since the last check;
  // finish_launches reports it by name
  cudaError_t async_err = cudaSuccess;
  const char* async_what = nullptr;
  void note(cudaError_t e, const char* what) {
    if (e != cudaSuccess && async_err == cudaSuccess) { async_err = e; async_what = what; }
  }
  ~pmg_workspace_s() {
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    if (slot_ev) cudaEventDestroy(slot_ev);
    for (auto& g : cyc)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    if (hm_block) cudaFreeHost(hm_block);
  }
};

namespace {

struct WsLayout {
  size_t total = 0;
  std::vector<size_t> f, u, r, y, e, hb, hx, hr, hg;
  size_t flags, lprog, counters, err, partial, r0, hist, f_in, u_io, kv[8], kd;
  int R = 0;
  std::vector<size_t> bf, be, br, by, bt, bhb, bhx, bhr, bhg, bht;
  size_t bF = 0, bU = 0, bR = 0, br0 = 0, brel = 0, bmask = 0, bpart = 0, bstate = 0, biters = 0;
};

WsLayout plan_ws(const pmg_hierarchy_s* h, int max_rhs) {
  WsLayout W;
  size_t s = 0;
  auto take = [&](size_t bytes) { size_t o = s; s = align_up(s + std::max<size_t>(bytes, 1)); return o; };
  const auto& H = h->H;
  int maxN = 0;
  for (const auto& L : H.lev) {
    const size_t b = size_t(L.N) * sizeof(double);
    W.f.push_back(take(b)); W.u.push_back(take(b)); W.r.push_back(take(b));
    W.y.push_back(take(b)); W.e.push_back(take(b));
    maxN = std::max(maxN, L.N);
  }
  for (const auto& Hl : H.hl) {
    const size_t b = size_t(Hl.N) * sizeof(double);
    W.hb.push_back(take(b)); W.hx.push_back(take(b)); W.hr.push_back(take(b)); W.hg.push_back(take(b));
    maxN = std::max(maxN, Hl.N);
  }
  if (max_rhs > 1) {
    W.R = (max_rhs + 31) / 32 * 32;
    for (const auto& L : H.lev) {
      const size_t b = size_t(L.N) * sizeof(double) * W.R;
      W.bf.push_back(take(b)); W.be.push_back(take(b)); W.br.push_back(take(b));
      W.by.push_back(take(b)); W.bt.push_back(take(b));
    }
    for (const auto& Hl : H.hl) {
      const size_t b = size_t(Hl.N) * sizeof(double) * W.R;
      W.bhb.push_back(take(b)); W.bhx.push_back(take(b)); W.bhr.push_back(take(b));
      W.bhg.push_back(take(b)); W.bht.push_back(take(b));
    }
    const size_t b0 = size_t(H.lev[0].N) * sizeof(double) * W.R;
    W.bF = take(b0); W.bU = take(b0); W.bR = take(b0);
    W.br0 = take(W.R * sizeof(double)); W.brel = take(W.R * sizeof(double)); W.bmask = take(W.R * sizeof(double));
    W.bpart = take(size_t(pmgk::kNormBlocks) * W.R * sizeof(double));
    W.bstate = take(W.R * sizeof(int));
    W.biters = take(W.R * sizeof(int));
  }
  for (auto& o : W.kv) o = take(size_t(H.lev[0].N) * sizeof(double));
  W.kd = take(8 * sizeof(double));
  W.flags = take(size_t(maxN) * sizeof(unsigned));
  int maxLines = 1;
  for (const auto& L : H.lev) maxLines = std::max(maxLines, L.N / std::max(1, L.n1d));
  for (const auto& Hl : H.hl) maxLines = std::max(maxLines, Hl.N / std::max(1, Hl.n1d));
  W.lprog = take(size_t(maxLines) * sizeof(unsigned long long));
  W.counters = take(kCounterSlots * sizeof(unsigned));
  W.err = take(4 * sizeof(unsigned));
  W.partial = take(pmgk::kNormBlocks * sizeof(double));
  W.r0 = take(sizeof(double));
  W.hist = take(kHistCap * sizeof(double));
  W.f_in = take(size_t(H.lev[0].N) * sizeof(double));
  W.u_io = take(size_t(H.lev[0].N) * sizeof(double));
  W.total = s;
  return W;
}

// ---------------------------------------------------------------------------
// kernel launch helpers
// ---------------------------------------------------------------------------
int grid_for(long long work, int threads, int cap) {
  long long g = (work + threads - 1) / threads;
  return int(std::max<long long>(1, std::min<long long>(g, cap)));
}

template <int MODE>
void spmv(const pmgk::Csr& A, double avg, const double* x, const double* b, double* y, cudaStream_t s, int sms,
          const double* d = nullptr) {
  const int threads = 256;
  if (avg >= 24) {
    pmgk::k_spmv<32, MODE><<<grid_for((long long)A.nr * 32, threads, sms * 16), threads, 0, s>>>(A, x, b, y, d);
  } else if (avg >= 12) {
    pmgk::k_spmv<16, MODE><<<grid_for((long long)A.nr * 16, threads, sms * 16), threads, 0, s>>>(A, x, b, y, d);
  } else {
    pmgk::k_spmv<8, MODE><<<grid_for((long long)A.nr * 8, threads, sms * 16), threads, 0, s>>>(A, x, b, y, d);
  }
}

// Lines of one right-hand-side group that a line-pipelined solve keeps busy at
// once: with a critical path of `depth` rows over `nlines` lines of nx rows,
// consecutive lines lag by about (depth - nx) / (nlines - 1) rows, so about
// nx / lag lines are between their first and last row at any time (+4 slack).
int lines_in_flight(int depth, int nx, int nlines) {
  if (nlines <= 1) return 1;
  const int lag = std::max(1, (depth - nx) / (nlines - 1));
  return std::min(nlines, nx / lag + 4);
}

// Raises a kernel's dynamic shared-memory limit to kLpSmemCap once per device.
void allow_smem(const void* fn) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (done.insert({fn, dev}).second) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kLpSmemCap));
}

struct Ctx {
  pmg_hierarchy_s* h;
  pmg_ws w;
  cudaStream_t s;
  int fstore = 0;       // FP32 inner cycle: factor storage 0 FP32, 1 FP16, 2 BF16
};

cudaEvent_t pool_event(pmg_ws w) {
  if (w->ev_used == w->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    w->ev_pool.push_back(e);
  }
  return w->ev_pool[w->ev_used++];
}

// Issues one kernel launch (the callable), counting it and, when profiling is
// on, bracketing it with CUDA events on the launch stream.
template <class F>
void launch(Ctx& c, int cls, double bytes, F&& f, int kernels = 1) {
  pmg_ws w = c.w;
  w->launches += kernels;
  if (!w->prof) { f(); return; }
  cudaEvent_t a = pool_event(w), b = pool_event(w);
  if (!a || !b) { f(); return; }
  cudaEventRecord(a, c.s);
  f();
  cudaEventRecord(b, c.s);
  w->pending.push_back({cls, a, b, bytes});
}

// Folds the timings of completed launches into the statistics (stream synced).
void collect_profile(pmg_ws w) {
  for (const auto& p : w->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      w->prof_ms[p.cls] += ms;
      w->prof_n[p.cls] += 1;
      w->prof_bytes[p.cls] += p.bytes;
    }
  }
  w->pending.clear();
  w->ev_used = 0;
}

double csr_bytes(long long nnz, int nr) { return 12.0 * double(nnz) + 4.0 * (nr + 1); }

unsigned* next_counter(Ctx& c) {
  if (c.w->next_slot >= kCounterSlots) {
    c.w->note(cudaMemsetAsync(c.w->counters, 0, kCounterSlots * sizeof(unsigned), c.s), "reset of the launch counters");
    c.w->next_slot = 0;
  }
  return c.w->counters + c.w->next_slot++;
}
unsigned next_epoch(Ctx& c) {
  if (++c.w->epoch == 0u) {  // wrapped: clear the flags and restart at 1
    const auto& H = c.h->H;
    int maxN = 0;
    for (const auto& L : H.lev) maxN = std::max(maxN, L.N);
    for (const auto& Hl : H.hl) maxN = std::max(maxN, Hl.N);
    c.w->note(cudaMemsetAsync(c.w->flags, 0, size_t(maxN) * sizeof(unsigned), c.s), "reset of the ready flags");
    c.w->epoch = 1u;
  }
  return c.w->epoch;
}
int sync_grid(const Ctx& c) { return c.h->sms * 4; }

template <int MODE>
void sell_spmv(const pmgk::Sell& S, const double* x, const double* b, double* y, cudaStream_t s) {
  const int threads = 256;
  const int grid = std::max(1, (S.nslices * 32 + threads - 1) / threads);
  pmgk::k_sell<MODE><<<grid, threads, 0, s>>>(S, x, b, y, nullptr);
}

void residual(Ctx& c, int l, const double* f, const double* u, double* r) {
  const DevPLevel& D = c.h->dl[l];
  launch(c, PMG_K_RESIDUAL, csr_bytes(D.nnzA, D.N) + 24.0 * D.N, [&] { sell_spmv<0>(D.sA, u, f, r, c.s); });
}

// Line-pipelined solve launch (kLpLinesPerCta lines per CTA, two warps per line).
template <bool MIR, bool UPD, int WIN, int LPR>
bool lp_launch_t(Ctx& c, const pmgk::Lp2& M, const double* b, double* x, double* u) {
  const size_t smem = (size_t(2) * pmgk::kLpLinesPerCta * M.nx + size_t(pmgk::kLpLinesPerCta) * 2 * pmgk::kLpStage * 32) *
                      sizeof(double);
  if (smem > kLpSmemCap) return false;
  allow_smem((const void*)pmgk::k_lp2<MIR, UPD, WIN, LPR>);
  const int nblocks = (M.nlines + pmgk::kLpLinesPerCta - 1) / pmgk::kLpLinesPerCta;
  const int grid = std::max(1, std::min(nblocks, c.h->sms));
  unsigned* cnt = next_counter(c);
  // the output starts as "pending" (all-ones bytes); rows publish by overwriting it
  c.w->note(cudaMemsetAsync(x, 0xFF, size_t(M.n) * sizeof(double), c.s), "pending fill of a solve's output");
  pmgk::k_lp2<MIR, UPD, WIN, LPR><<<grid, 32 * (pmgk::kLpProducers + 1) * pmgk::kLpLinesPerCta, smem, c.s>>>(
      M, b, x, u, cnt, c.w->err);
  return true;
}

// Chain/producer split over two-CTA clusters (k_lp4), chain configuration G, A.
template <bool MIR, bool UPD, int WIN, int LPR, int G, int A, int NL>
bool lp4_launch_t(Ctx& c, const pmgk::Lp2& M, const double* b, double* x, double* u) {
  const size_t smem = size_t(pmgk::lp4_smem_doubles_for(M.nx)) * sizeof(double);
  if (smem > kLpSmemCap) return false;
  const void* fn = (const void*)pmgk::k_lp4<MIR, UPD, WIN, LPR, G, A, NL>;
  allow_smem(fn);
  const int clusters = std::max(1, std::min((M.nlines + NL - 1) / NL, c.h->sms / (2 * NL)));
  unsigned* cnt = next_counter(c);
  // the output starts as "pending" (all-ones bytes); rows publish by overwriting it
  c.w->note(cudaMemsetAsync(x, 0xFF, size_t(M.n) * sizeof(double), c.s), "pending fill of a solve's output");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * NL * clusters);
  cfg.blockDim = dim3(32 * pmgk::kLp4Warps);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c.s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2 * NL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  pmgk::Lp2 m = M;
  c.w->note(cudaLaunchKernelEx(&cfg, pmgk::k_lp4<MIR, UPD, WIN, LPR, G, A, NL>, m, b, x, u, cnt, c.w->err),
            "cluster launch of the line-pipelined solve");
  return true;
}
template <bool MIR, bool UPD, int WIN, int LPR>
bool lp4_launch_c(Ctx& c, int cfg, const pmgk::Lp2& M, const double* b, double* x, double* u) {
  switch (cfg) {
    case 0: return lp4_launch_t<MIR, UPD, WIN, LPR, kLp4Cfgs[0].G, kLp4Cfgs[0].A, kLp4Cfgs[0].NL>(c, M, b, x, u);
    case 1: return lp4_launch_t<MIR, UPD, WIN, LPR, kLp4Cfgs[1].G, kLp4Cfgs[1].A, kLp4Cfgs[1].NL>(c, M, b, x, u);
    case 2: return lp4_launch_t<MIR, UPD, WIN, LPR, kLp4Cfgs[2].G, kLp4Cfgs[2].A, kLp4Cfgs[2].NL>(c, M, b, x, u);
    case 3: return lp4_launch_t<MIR, UPD, WIN, LPR, kLp4Cfgs[3].G, kLp4Cfgs[3].A, kLp4Cfgs[3].NL>(c, M, b, x, u);
    case 4: return lp4_launch_t<MIR, UPD, WIN, LPR, kLp4Cfgs[4].G, kLp4Cfgs[4].A, kLp4Cfgs[4].NL>(c, M, b, x, u);
    case 5: return lp4_launch_t<MIR, UPD, WIN, LPR, kLp4Cfgs[5].G, kLp4Cfgs[5].A, kLp4Cfgs[5].NL>(c, M, b, x, u);
    case 6: return lp4_launch_t<MIR, UPD, WIN, LPR, kLp4Cfgs[6].G, kLp4Cfgs[6].A, kLp4Cfgs[6].NL>(c, M, b, x, u);
    case 7: return lp4_launch_t<MIR, UPD, WIN, LPR, kLp4Cfgs[7].G, kLp4Cfgs[7].A, kLp4Cfgs[7].NL>(c, M, b, x, u);
    default: return false;
  }
}
// Layouts the setup builds: ILUT factors (4 rows x 8 lanes; forward, or
// mirrored backward with or without the update), P1 sweeps (4 rows x 4 lanes).
bool lp4_launch(Ctx& c, int cfg, const pmgk::Lp2& M, bool mirror, const double* b, double* x, double* u) {
  if (M.win == 4 && M.lpr == 8) {
    if (!mirror) return u ? false : lp4_launch_c<false, false, 4, 8>(c, cfg, M, b, x, u);
    return u ? lp4_launch_c<true, true, 4, 8>(c, cfg, M, b, x, u) : lp4_launch_c<true, false, 4, 8>(c, cfg, M, b, x, u);
  }
  if (M.win == 4 && M.lpr == 4 && !u)
    return mirror ? lp4_launch_c<true, false, 4, 4>(c, cfg, M, b, x, u) : lp4_launch_c<false, false, 4, 4>(c, cfg, M, b, x, u);
  return false;
}

template <int WIN, int LPR>
bool lp_launch_l(Ctx& c, const pmgk::Lp2& M, bool mirror, const double* b, double* x, double* u) {
  if (mirror) return u ? lp_launch_t<true, true, WIN, LPR>(c, M, b, x, u) : lp_launch_t<true, false, WIN, LPR>(c, M, b, x, u);
  return u ? lp_launch_t<false, true, WIN, LPR>(c, M, b, x, u) : lp_launch_t<false, false, WIN, LPR>(c, M, b, x, u);
}
// Layouts the setup builds: ILUT factors (4 rows x 8 lanes), P1 sweeps (4 rows x 4 lanes).
bool lp_launch(Ctx& c, const pmgk::Lp2& M, bool mirror, const double* b, double* x, double* u) {
  if (M.win == 4 && M.lpr == 8) return lp_launch_l<4, 8>(c, M, mirror, b, x, u);
  if (M.win == 8 && M.lpr == 1) return lp_launch_l<8, 1>(c, M, mirror, b, x, u);
  if (M.win == 4 && M.lpr == 4) return lp_launch_l<4, 4>(c, M, mirror, b, x, u);
  return false;
}

// Ring-kernel batched solve; false when the line does not fit in shared memory.
template <class T, class CT = T>
bool b_lpc(Ctx& c, int cls, const pmgk::LpC<T, CT>& M, long long nnz, bool mirror, const T* b, T* x, int nrhs = 0,
           int inflight = 0) {
  const size_t smem = size_t(M.nx + 64) * 32 * sizeof(T);
  if (smem > kLpSmemCap) return false;
  const int R = nrhs > 0 ? nrhs : c.w->R, threads = 32 * (1 + pmgk::LpcProducers<T>::value);
  const void* fn = nullptr;
  auto pick = [&](auto mir, auto ring) {
    fn = (const void*)pmgk::k_lpc<T, decltype(mir)::value, decltype(ring)::value, CT>;
  };
  using F_ = std::false_type;
  using T_ = std::true_type;
  using R2 = std::integral_constant<int, 2>;
  using R16 = std::integral_constant<int, 16>;
  using R32 = std::integral_constant<int, 32>;
  switch (M.ring) {
    case 2:
      if constexpr (sizeof(CT) == sizeof(T)) { mirror ? pick(T_{}, R2{}) : pick(F_{}, R2{}); break; }
      return false;   // 16-bit storage only for the ILUT factors
    case 16:
      if constexpr (sizeof(CT) == sizeof(T)) { mirror ? pick(T_{}, R16{}) : pick(F_{}, R16{}); break; }
      return false;
    case 32:
      if constexpr (sizeof(T) == 4) { mirror ? pick(T_{}, R32{}) : pick(F_{}, R32{}); break; }
      return false;   // FP64 chains use narrower rings
    default: return false;
  }
  allow_smem(fn);
  int occ = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem) != cudaSuccess || occ < 1) occ = 1;
  // Only about `inflight` lines per group can make progress at once (the
  // pipeline's lag); more CTAs would only poll, taking issue slots and L2
  // bandwidth from the working ones (and from other streams' kernels).
  const int groups = std::max(1, R / 32);
  const int nitems = M.nlines * groups;
  int grid = std::min(nitems, c.h->sms * occ);
  if (inflight > 0) grid = std::min(grid, inflight * groups);
  grid = std::max(1, grid);
  unsigned* cnt = next_counter(c);
  // algorithmic bytes: each factor entry once (column index + value at the
  // storage precision), row pointers, b read and x written
  launch(c, cls, (4.0 + sizeof(CT)) * nnz + 4.0 * (M.n + 1) + 2.0 * M.n * R * sizeof(T), [&] {
    c.w->note(cudaMemsetAsync(x, 0xFF, size_t(M.n) * R * sizeof(T), c.s), "pending fill of a solve's output");
    pmgk::LpC<T, CT> m = M;
    int r = R;
    const T* bb = b;
    void* args[] = {&m, &r, &bb, &x, &cnt, &c.w->err};
    cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, c.s);
  });
  return true;
}

template <class T>
void b_axpy(Ctx& c, int cls, long long n, const T* x, T* y) {
  launch(c, cls, 3.0 * n * sizeof(T), [&] {
    pmgk::k_axpy<T><<<grid_for(n, 256, c.h->sms * 16), 256, 0, c.s>>>(n, x, y);
  });
}

void lsolve(Ctx& c, int l, const double* b, double* y) {
  const DevPLevel& D = c.h->dl[l];
  if (c.h->ptune[l].sL == kVarRing && b_lpc<double>(c, PMG_K_LSOLVE, D.Lc64, D.nnzL, false, b, y, 1, D.inflightL))
    return;
  launch(c, PMG_K_LSOLVE, csr_bytes(D.nnzL, D.N) + 16.0 * D.N, [&] {
    if (c.h->ptune[l].sL == kVarCluster && lp4_launch(c, c.h->ptune[l].cL, D.Llp, false, b, y, nullptr)) return;
    if (lp_launch(c, D.Llp, false, b, y, nullptr)) return;
    const unsigned ep = next_epoch(c);
    unsigned* cnt = next_counter(c);
    pmgk::k_lsolve<<<sync_grid(c), 256, 0, c.s>>>(D.L, b, y, c.w->flags, ep, cnt, c.w->err);
  });
}
void usolve(Ctx& c, int l, const double* y, double* e, double* u) {
  const DevPLevel& D = c.h->dl[l];
  if (c.h->ptune[l].sU == kVarRing && b_lpc<double>(c, PMG_K_USOLVE, D.Uc64, D.nnzU, true, y, e, 1, D.inflightU)) {
    if (u) b_axpy<double>(c, PMG_K_USOLVE, D.N, e, u);
    return;
  }
  launch(c, PMG_K_USOLVE, csr_bytes(D.nnzU, D.N) + (u ? 40.0 : 24.0) * D.N, [&] {
    if (c.h->ptune[l].sU == kVarCluster && lp4_launch(c, c.h->ptune[l].cU, D.Ulp, true, y, e, u)) return;
    if (lp_launch(c, D.Ulp, true, y, e, u)) return;
    const unsigned ep = next_epoch(c);
    unsigned* cnt = next_counter(c);
    pmgk::k_usolve_update<<<sync_grid(c), 256, 0, c.s>>>(D.U, D.udinv, y, e, u, c.w->flags, ep, cnt, c.w->err);
  });
}

// u += U^{-1} L^{-1} r   (one ILUT smoothing step given r = f - A u)
void smooth_from_residual(Ctx& c, int l, const double* r, double* u) {
  lsolve(c, l, r, c.w->y[l]);
  usolve(c, l, c.w->y[l], c.w->e[l], u);
}

// One lexicographic Gauss-Seidel sweep as a triangular solve:
// forward  (D + L) x_new = b - U x_old,  backward  (D + U) x_new = b - L x_old.
// The new values go to a scratch vector first (the solve polls its output for
// readiness, so it cannot overwrite x in place) and are copied back.
bool wave_sweep(Ctx& c, const DevHLevel& D, bool backward, const double* b, double* x);

void gs(Ctx& c, int j, bool backward, const double* b, double* x) {
  const DevHLevel& D = c.h->dh[j];
  double* t = c.w->hr[j];
  double* xn = c.w->hg[j];
  const pmgk::Csr& other = backward ? D.Lo : D.Up;
  unsigned char var = backward ? c.h->htune[j].gB : c.h->htune[j].gF;
  if (var == kVarWave) {
    if (wave_sweep(c, D, backward, b, x)) return;
    var = kVarCluster;   // no wavefront layout (3D levels): the clustered kernel
  }
  // the ring kernel in its one-vector form: the old-value part as an SpMV, the
  // new values by the line-pipelined solve with a 2-wide ring
  const pmgk::LpC<double>& ring = backward ? D.UpMc : D.Loc;
  if (var == kVarRing && size_t(ring.nx + 64) * 32 * sizeof(double) <= kLpSmemCap) {
    launch(c, PMG_K_GS, csr_bytes(D.nnzA / 2, D.N) + 24.0 * D.N,
           [&] { spmv<0>(other, backward ? D.avg_lo : D.avg_up, x, b, t, c.s, c.h->sms); });
    b_lpc<double>(c, PMG_K_GS, ring, D.nnzA / 2, backward, t, xn, 1, D.inflightGS);
    cudaMemcpyAsync(x, xn, size_t(D.N) * sizeof(double), cudaMemcpyDeviceToDevice, c.s);
    return;
  }
  const pmgk::Lp2& lay = backward ? D.UpMlp : D.Lolp;
  const int cfg = backward ? c.h->htune[j].cB : c.h->htune[j].cF;
  const double half = csr_bytes(D.nnzA / 2, D.N);
  launch(c, PMG_K_GS, half + 24.0 * D.N, [&] { spmv<0>(other, backward ? D.avg_lo : D.avg_up, x, b, t, c.s, c.h->sms); });
  bool done = false;
  launch(c, PMG_K_GS, half + 16.0 * D.N, [&] {
    done = (var == kVarCluster && lp4_launch(c, cfg, lay, backward, t, xn, nullptr)) || lp_launch(c, lay, backward, t, xn, nullptr);
  });
  if (done) {
    cudaMemcpyAsync(x, xn, size_t(D.N) * sizeof(double), cudaMemcpyDeviceToDevice, c.s);
    return;
  }
  launch(c, PMG_K_GS, csr_bytes(D.nnzA, D.N) + 16.0 * D.N, [&] {
    const unsigned ep = next_epoch(c);
    unsigned* cnt = next_counter(c);
    if (backward)
      pmgk::k_gauss_seidel<true><<<sync_grid(c), 256, 0, c.s>>>(D.A, D.dinv, b, x, c.w->flags, ep, cnt, c.w->err);
    else
      pmgk::k_gauss_seidel<false><<<sync_grid(c), 256, 0, c.s>>>(D.A, D.dinv, b, x, c.w->flags, ep, cnt, c.w->err);
  });
}

// Wavefront sweep of a 2D P1 level: t = (b - (other part) x_old) d, then the
// lower solve by k_gs_wave written over x.  False when the level has none.
bool wave_sweep(Ctx& c, const DevHLevel& D, bool backward, const double* b, double* x) {
  const double* coef = backward ? D.wave_b : D.wave_f;
  if (!coef) return false;
  const int m = int(std::lround(std::sqrt(double(D.N))));
  if (m * m != D.N || m > pmgk::kWaveMaxLines) return false;
  const int wpc = pmgk::wave_wpc(m), nw = (m + 31) / 32, ncta = (nw + wpc - 1) / wpc;
  const size_t smem = pmgk::wave_smem_doubles(m) * sizeof(double);
  if (smem > kLpSmemCap) return false;
  double* t = c.w->hr[&D - c.h->dh.data()];
  const double nnz_old = 0.5 * double(D.nnzA - D.N);   // strictly lower / upper part (symmetric pattern)
  launch(c, PMG_K_GS, 12.0 * nnz_old + 4.0 * (D.N + 1) + 32.0 * D.N, [&] {
    spmv<3>(backward ? D.Lo : D.Up, backward ? D.avg_lo : D.avg_up, x, b, t, c.s, c.h->sms, D.dinv);
  });
  launch(c, PMG_K_GS, 48.0 * D.N, [&] {
    // one cluster of ncta CTAs (ncta <= 8, the portable cluster size)
    allow_smem(backward ? (const void*)pmgk::k_gs_wave<true> : (const void*)pmgk::k_gs_wave<false>);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(unsigned(ncta));
    cfg.blockDim = dim3(unsigned(32 * wpc));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c.s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(ncta);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (backward) c.w->note(cudaLaunchKernelEx(&cfg, pmgk::k_gs_wave<true>, m, coef, (const double*)t, x, c.w->err), "wavefront sweep launch");
    else c.w->note(cudaLaunchKernelEx(&cfg, pmgk::k_gs_wave<false>, m, coef, (const double*)t, x, c.w->err), "wavefront sweep launch");
  });
  return true;
}

// y <- M^{-1} y for a level's interior mass matrix M (consistent transfers):
// one banded line solve per direction; with add, the last pass writes
// out = add + M^{-1} y instead of y.
void mass_solve(Ctx& c, const MassF& m, double* y, const double* add, double* out) {
  const int d = c.h->H.d;
  long long total = 1;
  for (int k = 0; k < d; ++k) total *= m.n;
  const int nlines = int(total / m.n);
  long long inner = 1;
  for (int dir = 0; dir < d; ++dir) {
    const bool last = dir == d - 1;
    const double* F = dir == 0 ? m.f0 : m.f1;
    const double* a = last ? add : nullptr;
    double* o = last ? out : nullptr;
    launch(c, PMG_K_TRANSFER, 16.0 * double(total) + (a ? 16.0 * double(total) : 0.0), [&] {
      const int grid = (nlines + 63) / 64;
      switch (m.q) {
#define PMG_BAND_CASE(Q) \
  case Q: pmgk::k_band_lines<Q><<<grid, 64, 0, c.s>>>(m.n, nlines, inner, inner * m.n, inner, F, y, a, o); break;
        PMG_BAND_CASE(1) PMG_BAND_CASE(2) PMG_BAND_CASE(3) PMG_BAND_CASE(4)
        PMG_BAND_CASE(5) PMG_BAND_CASE(6) PMG_BAND_CASE(7) PMG_BAND_CASE(8)
#undef PMG_BAND_CASE
        default: c.w->note(cudaErrorInvalidValue, "mass_solve: degree out of range");
      }
    });
    inner *= m.n;
  }
}

// r_c = M_c^{-1} P^T r and u_out = u_in + M_l^{-1} P e_c (Eq. restriction /
// prolongation), M the lumped mass matrices (folded into the operators) or
// the consistent ones (App. B; the operators are then the unscaled P, P^T)
void restrict_to(Ctx& c, int l, const double* r, double* rc) {
  const DevPLevel& D = c.h->dl[l];
  launch(c, PMG_K_TRANSFER, csr_bytes(D.nnzP, D.Res.nr) + 8.0 * (D.N + D.Res.nr),
         [&] { sell_spmv<1>(D.sRes, r, nullptr, rc, c.s); });
  if (D.mass.f0) {
    const bool last = l + 1 == int(c.h->dl.size());
    mass_solve(c, last ? c.h->mass1 : c.h->dl[l + 1].mass, rc, nullptr, nullptr);
  }
}
void prolong_add(Ctx& c, int l, const double* ec, const double* uin, double* uout) {
  const DevPLevel& D = c.h->dl[l];
  if (D.mass.f0) {
    double* t = c.w->y[l];
    launch(c, PMG_K_TRANSFER, csr_bytes(D.nnzP, D.N) + 8.0 * (D.N + D.Res.nr),
           [&] { sell_spmv<1>(D.sPro, ec, nullptr, t, c.s); });
    mass_solve(c, D.mass, t, uin, uout);
    return;
  }
  launch(c, PMG_K_TRANSFER, csr_bytes(D.nnzP, D.N) + 8.0 * (2 * D.N + D.Res.nr),
         [&] { sell_spmv<2>(D.sPro, ec, uin, uout, c.s); });
}

// one h-multigrid V-cycle on P1 level j: A_j x = b (Sec. 3, Fig. 1)
void hmg_vcycle(Ctx& c, int j, const double* b, double* x) {
  const int nh = int(c.h->dh.size());
  const DevHLevel& D = c.h->dh[j];
  if (j == nh - 1) {
    launch(c, PMG_K_COARSE, 8.0 * D.N * D.N + 16.0 * D.N, [&] {
      pmgk::k_dense_matvec<<<grid_for((long long)D.N * 32, 256, c.h->sms * 4), 256, 0, c.s>>>(D.N, c.h->cinv, b, x);
    });
    return;
  }
  const DevHLevel& Cc = c.h->dh[j + 1];
  const int d = c.h->H.d;
  gs(c, j, false, b, x);
  launch(c, PMG_K_P1, csr_bytes(D.nnzA, D.N) + 24.0 * D.N,
         [&] { spmv<0>(D.A, 9, x, b, c.w->hr[j], c.s, c.h->sms); });
  launch(c, PMG_K_P1, 8.0 * (D.N + Cc.N), [&] {
    pmgk::k_p1_restrict<<<grid_for(Cc.N, 256, c.h->sms * 8), 256, 0, c.s>>>(d, D.ne, c.w->hr[j], c.w->hb[j + 1]);
  });
  cudaMemsetAsync(c.w->hx[j + 1], 0, size_t(Cc.N) * sizeof(double), c.s);
  hmg_vcycle(c, j + 1, c.w->hb[j + 1], c.w->hx[j + 1]);
  launch(c, PMG_K_P1, 8.0 * Cc.N + 16.0 * D.N, [&] {
    pmgk::k_p1_prolong_add<<<grid_for(D.N, 256, c.h->sms * 8), 256, 0, c.s>>>(d, D.ne, c.w->hx[j + 1], x);
  });
  gs(c, j, true, b, x);
}

// coarse grid correction at p = 1: coarse_cycles h-MG V-cycles from zero
void coarse_solve(Ctx& c, const double* b1, double* x1) {
  cudaMemsetAsync(x1, 0, size_t(c.h->dh[0].N) * sizeof(double), c.s);
  for (int k = 0; k < c.h->H.opt.coarse_cycles; ++k) hmg_vcycle(c, 0, b1, x1);
}

// V-cycle at p-level l on A_l u = f.  r_in, when not null, holds f - A_l u
// (the last residual of the previous cycle, or f itself for a zero guess).
void vcycle(Ctx& c, int l, const double* f, double* u, const double* r_in) {
  const auto& H = c.h->H;
  const int nlev = int(c.h->dl.size());
  const DevPLevel& D = c.h->dl[l];
  double* r = c.w->r[l];
  for (int m = 0; m < H.opt.nu_pre; ++m) {
    const double* rr = r_in;
    if (!rr) { residual(c, l, f, u, r); rr = r; }
    smooth_from_residual(c, l, rr, u);
    r_in = nullptr;
  }
  residual(c, l, f, u, r);
  if (l + 1 < nlev) {
    const int Nc = c.h->dl[l + 1].N;
    double* fc = c.w->f[l + 1];
    double* uc = c.w->u[l + 1];
    restrict_to(c, l, r, fc);
    cudaMemsetAsync(uc, 0, size_t(Nc) * sizeof(double), c.s);
    // with a zero initial guess the first residual is the right-hand side itself
    vcycle(c, l + 1, fc, uc, fc);
    prolong_add(c, l, uc, u, u);
  } else {
    double* b1 = c.w->hb[0];
    double* x1 = c.w->hx[0];
    restrict_to(c, l, r, b1);
    coarse_solve(c, b1, x1);
    prolong_add(c, l, x1, u, u);
  }
  for (int m = 0; m < H.opt.nu_post; ++m) {
    residual(c, l, f, u, r);
    smooth_from_residual(c, l, r, u);
  }
}

void sqnorm(Ctx& c, int n, const double* r, int mode, double* out) {
  launch(c, PMG_K_NORM, 8.0 * n, [&] {
    pmgk::k_sqnorm_partial<<<pmgk::kNormBlocks, pmgk::kNormThreads, 0, c.s>>>(n, r, c.w->partial);
  });
  launch(c, PMG_K_NORM, 8.0 * pmgk::kNormBlocks, [&] {
    if (mode == 0)
      pmgk::k_norm_finalize<0><<<1, pmgk::kNormThreads, 0, c.s>>>(pmgk::kNormBlocks, c.w->partial, c.w->r0, nullptr);
    else
      pmgk::k_norm_finalize<1><<<1, pmgk::kNormThreads, 0, c.s>>>(pmgk::kNormBlocks, c.w->partial, c.w->r0, out);
  });
}

pmg_status check_ws(pmg_handle h, pmg_ws ws) {
  if (!h || !ws) return fail(PMG_ERR_ARG, "null handle or workspace");
  if (!h->uploaded) return fail(PMG_ERR_STATE, "hierarchy not uploaded");
  if (ws->h != h) return fail(PMG_ERR_ARG, "workspace belongs to another hierarchy");
  return PMG_OK;
}

pmg_status begin_launches(Ctx& c) {
  c.w->next_slot = 0;
  PMG_CUDA(cudaMemsetAsync(c.w->counters, 0, kCounterSlots * sizeof(unsigned), c.s));
  return PMG_OK;
}

pmg_status finish_launches(Ctx& c) {
  if (c.w->async_err != cudaSuccess) {
    const std::string msg = std::string(c.w->async_what) + " failed: " + cudaGetErrorString(c.w->async_err);
    c.w->async_err = cudaSuccess;
    cudaGetLastError();
    return fail(PMG_ERR_CUDA, msg);
  }
  PMG_CUDA(cudaGetLastError());
  unsigned errw[4] = {0, 0, 0, 0};
  PMG_CUDA(cudaMemcpyAsync(errw, c.w->err, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, c.s));
  const unsigned err = errw[0];
  PMG_CUDA(cudaStreamSynchronize(c.s));
  collect_profile(c.w);
  if (err) {
    cudaMemsetAsync(c.w->err, 0, 4 * sizeof(unsigned), c.s);
    char buf[160];
    std::snprintf(buf, sizeof(buf),
                  "a device-side dependency wait expired (wait sites 0x%x; first: site 0x%x, item %u, row %u, warp %u)",
                  err, errw[1], errw[2], errw[3] >> 8, errw[3] & 0xffu);
    return fail(PMG_ERR_TIMEOUT, buf);
  }
  return PMG_OK;
}

// ---------------------------------------------------------------------------
// BiCGSTAB preconditioned by the V-cycle (Sec. 5, "p-Multigrid as a
// preconditioner"; van der Vorst 1992): right preconditioning, one V-cycle
// with zero initial guess per application, two applications per iteration.
// Scalars come back to the host after each reduction.
// ---------------------------------------------------------------------------
pmg_status krylov_dot(Ctx& c, const double* x, const double* y, double* out) {
  const int N = c.h->dl[0].N;
  launch(c, PMG_K_NORM, 16.0 * N, [&] {
    pmgk::k_dot_partial<<<pmgk::kNormBlocks, pmgk::kNormThreads, 0, c.s>>>(N, x, y, c.w->partial);
    pmgk::k_sum_partials<<<1, pmgk::kNormThreads, 0, c.s>>>(pmgk::kNormBlocks, c.w->partial, c.w->kd);
  }, 2);
  PMG_CUDA(cudaMemcpyAsync(out, c.w->kd, sizeof(double), cudaMemcpyDeviceToHost, c.s));
  return finish_launches(c);
}

// x_hat = M^{-1} x: one V-cycle from zero (its first residual is x itself)
void krylov_precond(Ctx& c, const double* x, double* xh) {
  cudaMemsetAsync(xh, 0, size_t(c.h->dl[0].N) * sizeof(double), c.s);
  vcycle(c, 0, x, xh, x);
}

pmg_status bicgstab_impl(pmg_handle h, pmg_ws ws, const double* f, const double* u0, double tol, int max_iter,
                         double* u, int* iters, double* hist, int hist_cap, cudaStream_t s) {
  Ctx c{h, ws, s};
  const DevPLevel& D = h->dl[0];
  const int N = D.N;
  double *r = ws->kv[0], *rh = ws->kv[1], *p = ws->kv[2], *v = ws->kv[3];
  double *sv = ws->kv[4], *t = ws->kv[5], *ph = ws->kv[6], *sh = ws->kv[7];
  const int gb = grid_for(N, 256, h->sms * 8);
  auto sub_scaled = [&](const double* x, double a, const double* y, double* out) {
    launch(c, PMG_K_NORM, 24.0 * N, [&] { pmgk::k_sub_scaled<<<gb, 256, 0, c.s>>>(N, x, a, y, out); });
  };
  auto matvec = [&](const double* x, double* y) {
    launch(c, PMG_K_RESIDUAL, csr_bytes(D.nnzA, D.N) + 16.0 * D.N, [&] { sell_spmv<1>(D.sA, x, nullptr, y, c.s); });
  };
  if (iters) *iters = 0;
  pmg_status st = begin_launches(c);
  if (st != PMG_OK) return st;
  if (u != u0) PMG_CUDA(cudaMemcpyAsync(u, u0, size_t(N) * sizeof(double), cudaMemcpyDeviceToDevice, s));
  residual(c, 0, f, u, r);
  double rr = 0.0;
  if ((st = krylov_dot(c, r, r, &rr)) != PMG_OK) return st;
  const double r0n = std::sqrt(rr);
  if (r0n == 0.0) return PMG_OK;
  PMG_CUDA(cudaMemcpyAsync(rh, r, size_t(N) * sizeof(double), cudaMemcpyDeviceToDevice, s));
  PMG_CUDA(cudaMemsetAsync(p, 0, size_t(N) * sizeof(double), s));
  PMG_CUDA(cudaMemsetAsync(v, 0, size_t(N) * sizeof(double), s));
  double rho_prev = 1.0, alpha = 1.0, omega = 1.0;
  for (int it = 1; it <= max_iter; ++it) {
    if ((st = begin_launches(c)) != PMG_OK) return st;
    double rho = 0.0;
    if ((st = krylov_dot(c, rh, r, &rho)) != PMG_OK) return st;
    if (rho == 0.0) return fail(PMG_ERR_DIVERGED, "BiCGSTAB breakdown (r-hat . r = 0)");
    const double beta = it == 1 ? 0.0 : (rho / rho_prev) * (alpha / omega);
    launch(c, PMG_K_NORM, 32.0 * N, [&] { pmgk::k_bicg_direction<<<gb, 256, 0, c.s>>>(N, beta, omega, r, v, p); });
    krylov_precond(c, p, ph);
    matvec(ph, v);
    double rhv = 0.0;
    if ((st = krylov_dot(c, rh, v, &rhv)) != PMG_OK) return st;
    alpha = rho / rhv;
    sub_scaled(r, alpha, v, sv);
    double ss = 0.0;
    if ((st = krylov_dot(c, sv, sv, &ss)) != PMG_OK) return st;
    const double srel = std::sqrt(ss) / r0n;
    if (srel < tol) {
      launch(c, PMG_K_NORM, 24.0 * N,
             [&] { pmgk::k_bicg_solution<<<gb, 256, 0, c.s>>>(N, alpha, ph, 0.0, nullptr, u); });
      if (hist && it - 1 < hist_cap) hist[it - 1] = srel;
      if (iters) *iters = it;
      PMG_CUDA(cudaStreamSynchronize(s));
      return PMG_OK;
    }
    if ((st = begin_launches(c)) != PMG_OK) return st;
    krylov_precond(c, sv, sh);
    matvec(sh, t);
    double ts = 0.0, tt = 0.0;
    if ((st = krylov_dot(c, t, sv, &ts)) != PMG_OK) return st;
    if ((st = krylov_dot(c, t, t, &tt)) != PMG_OK) return st;
    omega = ts / tt;
    launch(c, PMG_K_NORM, 32.0 * N,
           [&] { pmgk::k_bicg_solution<<<gb, 256, 0, c.s>>>(N, alpha, ph, omega, sh, u); });
    sub_scaled(sv, omega, t, r);
    double r2 = 0.0;
    if ((st = krylov_dot(c, r, r, &r2)) != PMG_OK) return st;
    const double rel = std::sqrt(r2) / r0n;
    if (hist && it - 1 < hist_cap) hist[it - 1] = rel;
    if (iters) *iters = it;
    if (rel < tol) return PMG_OK;
    if (!(rel <= 1e10)) return fail(PMG_ERR_DIVERGED, "relative residual exceeded 1e10");
    rho_prev = rho;
  }
  return fail(PMG_ERR_MAXITER, "maximum number of BiCGSTAB iterations reached");
}

pmg_status solve_impl(pmg_handle h, pmg_ws ws, const double* f, const double* u0, double tol, int max_iter,
                      double* u, int* iters, double* hist, int hist_cap, cudaStream_t s) {
  Ctx c{h, ws, s};
  const int N = h->dl[0].N;
  if (iters) *iters = 0;
  if (u != u0) PMG_CUDA(cudaMemcpyAsync(u, u0, size_t(N) * sizeof(double), cudaMemcpyDeviceToDevice, s));
  double* r = ws->r[0];
  residual(c, 0, f, u, r);
  sqnorm(c, N, r, 0, nullptr);
  double r0 = 0.0;
  PMG_CUDA(cudaMemcpyAsync(&r0, ws->r0, sizeof(double), cudaMemcpyDeviceToHost, s));
  PMG_CUDA(cudaStreamSynchronize(s));
  collect_profile(ws);
  if (r0 == 0.0) return PMG_OK;
  pmg_status st = PMG_ERR_MAXITER;
  for (int it = 0; it < max_iter; ++it) {
    pmg_status b = begin_launches(c);
    if (b != PMG_OK) return b;
    vcycle(c, 0, f, u, r);
    residual(c, 0, f, u, r);
    double* slot = ws->hist + (it % kHistCap);
    sqnorm(c, N, r, 1, slot);
    double rel = 0.0;
    PMG_CUDA(cudaMemcpyAsync(&rel, slot, sizeof(double), cudaMemcpyDeviceToHost, s));
    pmg_status fin = finish_launches(c);
    if (fin != PMG_OK) { if (iters) *iters = it + 1; return fin; }
    if (hist && it < hist_cap) hist[it] = rel;
    if (iters) *iters = it + 1;
    if (rel < tol) { st = PMG_OK; break; }
    if (!(rel <= 1e10)) { st = PMG_ERR_DIVERGED; break; }
  }
  if (st == PMG_ERR_MAXITER) g_last_error = "maximum number of V-cycles reached";
  if (st == PMG_ERR_DIVERGED) g_last_error = "relative residual exceeded 1e10";
  return st;
}

// ---------------------------------------------------------------------------
// Batched solves: many right-hand sides, plain FP64 or an FP32 inner cycle
// inside FP64 defect correction.  Vectors are [row][R] (right-hand sides
// fastest, R a multiple of 32).  One iteration: r = f - A u (FP64), e = one
// V-cycle with zero initial guess applied to r (inner precision T), u += e
// (FP64) for the right-hand sides that have not converged yet.  The coarse
// correction at p = 1 stays FP64 in both forms.
// ---------------------------------------------------------------------------
int grid_rows(long long work_warps, int sms) {
  return grid_for(work_warps * 32, 256, sms * 16);
}

template <class TA, class TX, class TY, int MODE>
void b_spmm(Ctx& c, int cls, const pmgk::TCsr<TA>& A, long long nnz, const TX* X, const TY* B, TY* Y) {
  const int R = c.w->R;
  launch(c, cls, 12.0 * nnz + 4.0 * (A.nr + 1) + (MODE == 1 ? 2.0 : 3.0) * A.nr * R * sizeof(TY), [&] {
    pmgk::k_spmm<TA, TX, TY, MODE><<<grid_rows((long long)A.nr * (R / 32), c.h->sms), 256, 0, c.s>>>(A, R, X, B, Y);
  });
}
pmgk::TCsr<double> as_t(const pmgk::Csr& a) { return pmgk::TCsr<double>{a.nr, a.rp, a.ci, a.v}; }

template <class T>
void b_lp(Ctx& c, int cls, const pmgk::LpB<T>& M, long long nnz, bool mirror, const T* b, T* x, T* u) {
  const int R = c.w->R;
  int lines = pmgk::kLpbMaxLines;
  const size_t per_line = size_t(M.nx) * 32 * sizeof(T);
  while (lines > 1 && lines * per_line > kLpSmemCap) --lines;
  const size_t smem = lines * per_line;
  const int nitems = ((M.nlines + lines - 1) / lines) * (R / 32);
  const int grid = std::max(1, std::min(nitems, 2 * c.h->sms));
  unsigned* cnt = next_counter(c);
  launch(c, cls, 12.0 * nnz + 4.0 * (M.n + 1) + (u ? 4.0 : 2.0) * M.n * R * sizeof(T), [&] {
    c.w->note(cudaMemsetAsync(x, 0xFF, size_t(M.n) * R * sizeof(T), c.s), "pending fill of a solve's output");
    const int th = 32 * lines;
    const int k = (mirror ? 2 : 0) + (u ? 1 : 0);
    if (k == 0) { allow_smem((const void*)pmgk::k_lpb<T, false, false>); pmgk::k_lpb<T, false, false><<<grid, th, smem, c.s>>>(M, R, b, x, u, cnt, c.w->err); }
    if (k == 1) { allow_smem((const void*)pmgk::k_lpb<T, false, true>); pmgk::k_lpb<T, false, true><<<grid, th, smem, c.s>>>(M, R, b, x, u, cnt, c.w->err); }
    if (k == 2) { allow_smem((const void*)pmgk::k_lpb<T, true, false>); pmgk::k_lpb<T, true, false><<<grid, th, smem, c.s>>>(M, R, b, x, u, cnt, c.w->err); }
    if (k == 3) { allow_smem((const void*)pmgk::k_lpb<T, true, true>); pmgk::k_lpb<T, true, true><<<grid, th, smem, c.s>>>(M, R, b, x, u, cnt, c.w->err); }
  });
}

template <class TI, class TO>
void b_cast(Ctx& c, long long n, const TI* x, TO* y) {
  pmgk::k_cast<TI, TO><<<grid_for(n, 256, c.h->sms * 16), 256, 0, c.s>>>(n, x, y);
  ++c.w->launches;
}

// Gauss-Seidel sweep, batched: the old-value part as an SpMM, the new values by the line-pipelined solve.
void b_gs(Ctx& c, int j, bool backward, const double* b, double* x) {
  const DevHLevel& D = c.h->dh[j];
  const int R = c.w->R;
  double* t = c.w->bht[j];
  double* xn = c.w->bhg[j];
  if (backward) b_spmm<double, double, double, 0>(c, PMG_K_GS, as_t(D.Lo), D.nnzA / 2, x, b, t);
  else b_spmm<double, double, double, 0>(c, PMG_K_GS, as_t(D.Up), D.nnzA / 2, x, b, t);
  const unsigned char var = backward ? c.h->htune[j].bB : c.h->htune[j].bF;
  if (var != kVarRing ||
      !b_lpc<double>(c, PMG_K_GS, backward ? D.UpMc : D.Loc, D.nnzA / 2, backward, t, xn, 0, D.inflightGS))
    b_lp<double>(c, PMG_K_GS, backward ? D.UpMb : D.Lob, D.nnzA / 2, backward, t, xn, nullptr);
  cudaMemcpyAsync(x, xn, size_t(D.N) * R * sizeof(double), cudaMemcpyDeviceToDevice, c.s);
}

void b_hmg(Ctx& c, int j, const double* b, double* x) {
  const int nh = int(c.h->dh.size()), R = c.w->R;
  const DevHLevel& D = c.h->dh[j];
  if (j == nh - 1) {
    launch(c, PMG_K_COARSE, 8.0 * D.N * D.N + 16.0 * D.N * R, [&] {
      pmgk::k_dense_mm<<<grid_rows((long long)D.N * (R / 32), c.h->sms), 256, 0, c.s>>>(D.N, R, c.h->cinv, b, x);
    });
    return;
  }
  const DevHLevel& Cc = c.h->dh[j + 1];
  const int d = c.h->H.d;
  b_gs(c, j, false, b, x);
  b_spmm<double, double, double, 0>(c, PMG_K_P1, as_t(D.A), D.nnzA, x, b, c.w->bhr[j]);
  launch(c, PMG_K_P1, 8.0 * (D.N + Cc.N) * R, [&] {
    pmgk::k_p1_restrict_b<<<grid_for((long long)Cc.N * R, 256, c.h->sms * 16), 256, 0, c.s>>>(d, D.ne, R, c.w->bhr[j], c.w->bhb[j + 1]);
  });
  cudaMemsetAsync(c.w->bhx[j + 1], 0, size_t(Cc.N) * R * sizeof(double), c.s);
  b_hmg(c, j + 1, c.w->bhb[j + 1], c.w->bhx[j + 1]);
  launch(c, PMG_K_P1, (8.0 * Cc.N + 16.0 * D.N) * R, [&] {
    pmgk::k_p1_prolong_add_b<<<grid_for((long long)D.N * R, 256, c.h->sms * 16), 256, 0, c.s>>>(d, D.ne, R, c.w->bhx[j + 1], x);
  });
  b_gs(c, j, true, b, x);
}

// Batched triangular solve of level l (forward L, or mirrored U) with kernel variant `var`.
template <class T>
void b_tri(Ctx& c, int l, bool upper, unsigned char var, const T* b, T* x) {
  const DevPLevel& D = c.h->dl[l];
  const int cls = upper ? PMG_K_USOLVE : PMG_K_LSOLVE;
  const long long nnz = upper ? D.nnzU : D.nnzL;
  const int infl = upper ? D.inflightU : D.inflightL;
  if constexpr (sizeof(T) == 4) {
    if (c.fstore == 1 && b_lpc<float, __half>(c, cls, upper ? D.Uc16 : D.Lc16, nnz, upper, b, x, 0, infl)) return;
    if (c.fstore == 2 && b_lpc<float, __nv_bfloat16>(c, cls, upper ? D.Ucb : D.Lcb, nnz, upper, b, x, 0, infl))
      return;
    if (var == kVarRing && b_lpc<float>(c, cls, upper ? D.Uc32 : D.Lc32, nnz, upper, b, x, 0, infl)) return;
    b_lp<float>(c, cls, upper ? D.Ub32 : D.Lb32, nnz, upper, b, x, nullptr);
  } else {
    if (var == kVarRing && b_lpc<double>(c, cls, upper ? D.Uc64 : D.Lc64, nnz, upper, b, x, 0, infl)) return;
    b_lp<double>(c, cls, upper ? D.Ub64 : D.Lb64, nnz, upper, b, x, nullptr);
  }
}

// e = one V-cycle at p-level l applied to the right-hand side f with zero initial guess (precision T).
template <class T>
void b_vcycle0(Ctx& c, int l, const T* f, T* e) {
  const auto& H = c.h->H;
  const DevPLevel& D = c.h->dl[l];
  const int nlev = int(c.h->dl.size()), R = c.w->R;
  const pmgk::TCsr<T> A = [&] {
    if constexpr (sizeof(T) == 4) return D.A32; else return as_t(D.A);
  }();
  const pmgk::TCsr<T> Res = [&] {
    if constexpr (sizeof(T) == 4) return D.Res32; else return as_t(D.Res);
  }();
  const pmgk::TCsr<T> Pro = [&] {
    if constexpr (sizeof(T) == 4) return D.Pro32; else return as_t(D.Pro);
  }();
  T* r = reinterpret_cast<T*>(c.w->br[l]);
  T* y = reinterpret_cast<T*>(c.w->by[l]);
  T* t = reinterpret_cast<T*>(c.w->bt[l]);
  const size_t nR = size_t(D.N) * R;
  cudaMemsetAsync(e, 0, nR * sizeof(T), c.s);
  auto smooth = [&](bool first) {
    const T* rr = f;
    if (!first) { b_spmm<T, T, T, 0>(c, PMG_K_RESIDUAL, A, D.nnzA, e, f, r); rr = r; }
    const auto& tn = c.h->ptune[l];
    const int pi = sizeof(T) == 4 ? 1 : 0;
    b_tri<T>(c, l, false, tn.bL[pi], rr, y);
    b_tri<T>(c, l, true, tn.bU[pi], y, t);
    b_axpy<T>(c, PMG_K_USOLVE, (long long)D.N * R, t, e);
  };
  for (int m = 0; m < H.opt.nu_pre; ++m) smooth(m == 0);
  b_spmm<T, T, T, 0>(c, PMG_K_RESIDUAL, A, D.nnzA, e, f, r);
  if (l + 1 < nlev) {
    T* fc = reinterpret_cast<T*>(c.w->bf[l + 1]);
    T* ec = reinterpret_cast<T*>(c.w->be[l + 1]);
    b_spmm<T, T, T, 1>(c, PMG_K_TRANSFER, Res, D.nnzP, r, nullptr, fc);
    b_vcycle0<T>(c, l + 1, fc, ec);
    b_spmm<T, T, T, 2>(c, PMG_K_TRANSFER, Pro, D.nnzP, ec, e, e);
  } else {
    const int N1 = c.h->dh[0].N;
    double* b1 = c.w->bhb[0];
    double* x1 = c.w->bhx[0];
    if constexpr (sizeof(T) == 4) {
      float* fc = reinterpret_cast<float*>(c.w->bhr[0]);   // restricted residual before widening
      b_spmm<float, float, float, 1>(c, PMG_K_TRANSFER, Res, D.nnzP, r, nullptr, fc);
      b_cast<float, double>(c, (long long)N1 * R, fc, b1);
    } else {
      b_spmm<double, double, double, 1>(c, PMG_K_TRANSFER, Res, D.nnzP, r, nullptr, b1);
    }
    cudaMemsetAsync(x1, 0, size_t(N1) * R * sizeof(double), c.s);
    for (int k = 0; k < H.opt.coarse_cycles; ++k) b_hmg(c, 0, b1, x1);
    if constexpr (sizeof(T) == 4) {
      float* ec = reinterpret_cast<float*>(c.w->bhg[0]);
      b_cast<double, float>(c, (long long)N1 * R, x1, ec);
      b_spmm<float, float, float, 2>(c, PMG_K_TRANSFER, Pro, D.nnzP, ec, e, e);
    } else {
      b_spmm<double, double, double, 2>(c, PMG_K_TRANSFER, Pro, D.nnzP, x1, e, e);
    }
  }
  for (int m = 0; m < H.opt.nu_post; ++m) smooth(false);
}


// ---------------------------------------------------------------------------
// Slots (continuous batching) and the batched solve built on them.  A slot is
// one column of the [row][R] batch with a device-side state (free, active,
// converged, diverged), iteration count and update mask; a cycle updates only
// active slots, and its stopping test runs on the device.  The end of a cycle
// copies the per-slot state into the workspace's pinned mirror.
// ---------------------------------------------------------------------------
pmg_status slots_load_impl(Ctx& c, int slot0, int n, const double* F, const double* U0) {
  pmg_handle h = c.h;
  pmg_ws ws = c.w;
  const int N = h->dl[0].N, R = ws->R;
  const DevPLevel& D = h->dl[0];
  pmgk::k_slots_copy_in<<<grid_for((long long)N * n, 256, h->sms * 16), 256, 0, c.s>>>(N, n, R, slot0, F, ws->bF);
  pmgk::k_slots_copy_in<<<grid_for((long long)N * n, 256, h->sms * 16), 256, 0, c.s>>>(N, n, R, slot0, U0, ws->bU);
  ws->launches += 2;
  b_spmm<double, double, double, 0>(c, PMG_K_RESIDUAL, as_t(D.A), D.nnzA, ws->bU, ws->bF, ws->bR);
  launch(c, PMG_K_NORM, 8.0 * N * R, [&] {
    pmgk::k_sqnorm_partial_b<<<pmgk::kNormBlocks, 128, 0, c.s>>>(N, R, ws->bR, ws->bpart);
    pmgk::k_slots_start<<<1, 128, 0, c.s>>>(pmgk::kNormBlocks, R, slot0, n, ws->bpart, ws->br0, ws->brel,
                                            ws->bmask, ws->bstate, ws->biters);
  }, 2);
  for (int k = slot0; k < slot0 + n; ++k) ws->slot_state[k] = 1;
  PMG_CUDA(cudaGetLastError());
  return PMG_OK;
}

// One cycle's work, stream-ordered (capturable: no host synchronisation).
pmg_status slots_cycle_body(Ctx& c, int precision, double tol) {
  pmg_handle h = c.h;
  pmg_ws ws = c.w;
  const int N = h->dl[0].N, R = ws->R;
  const DevPLevel& D = h->dl[0];
  pmg_status st = begin_launches(c);
  if (st != PMG_OK) return st;
  if (precision != PMG_PREC_FP64) {
    c.fstore = precision == PMG_PREC_MIXED_FP16 ? 1 : precision == PMG_PREC_MIXED_BF16 ? 2 : 0;
    float* r32 = reinterpret_cast<float*>(ws->bf[0]);
    float* e32 = reinterpret_cast<float*>(ws->be[0]);
    b_cast<double, float>(c, (long long)N * R, ws->bR, r32);
    b_vcycle0<float>(c, 0, r32, e32);
    pmgk::k_masked_update<float><<<grid_for((long long)N * R, 256, h->sms * 16), 256, 0, c.s>>>(N, R, e32, ws->bmask,
                                                                                                 ws->bU);
  } else {
    b_vcycle0<double>(c, 0, ws->bR, ws->be[0]);
    pmgk::k_masked_update<double><<<grid_for((long long)N * R, 256, h->sms * 16), 256, 0, c.s>>>(N, R, ws->be[0],
                                                                                                  ws->bmask, ws->bU);
  }
  ++ws->launches;
  b_spmm<double, double, double, 0>(c, PMG_K_RESIDUAL, as_t(D.A), D.nnzA, ws->bU, ws->bF, ws->bR);
  launch(c, PMG_K_NORM, 8.0 * N * R, [&] {
    pmgk::k_sqnorm_partial_b<<<pmgk::kNormBlocks, 128, 0, c.s>>>(N, R, ws->bR, ws->bpart);
    pmgk::k_slots_update<<<(R + 127) / 128, 128, 0, c.s>>>(pmgk::kNormBlocks, R, tol, ws->bpart, ws->br0, ws->brel,
                                                           ws->bmask, ws->bstate, ws->biters);
  }, 2);
  PMG_CUDA(cudaMemcpyAsync(ws->hm.relres, ws->brel, R * sizeof(double), cudaMemcpyDeviceToHost, c.s));
  PMG_CUDA(cudaMemcpyAsync(ws->hm.state, ws->bstate, R * sizeof(int), cudaMemcpyDeviceToHost, c.s));
  PMG_CUDA(cudaMemcpyAsync(ws->hm.iters, ws->biters, R * sizeof(int), cudaMemcpyDeviceToHost, c.s));
  PMG_CUDA(cudaMemcpyAsync(ws->hm.err, ws->err, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, c.s));
  PMG_CUDA(cudaGetLastError());
  return PMG_OK;
}

// Enqueues one cycle.  On a non-default stream without profiling, the cycle
// runs as a CUDA graph: the second call for a (precision, tolerance, kernel
// choice) captures the launch sequence, later calls replay it with one launch
// (the first call runs eagerly, which also sets every kernel's attributes
// outside any capture).
pmg_status slots_cycle_impl(Ctx& c, int precision, double tol) {
  pmg_handle h = c.h;
  pmg_ws ws = c.w;
  auto& g = ws->cyc[precision];
  const bool graphable = ws->graphs && !ws->prof && c.s != nullptr;
  pmg_status st = PMG_OK;
  if (graphable && g.exec && (g.tol != tol || g.epoch != h->tune_epoch)) {
    cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    g.eager = 0;
  }
  if (graphable && !g.exec && g.eager >= 1) {
    const long long l0 = ws->launches;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(c.s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      st = slots_cycle_body(c, precision, tol);
      const cudaError_t e = cudaStreamEndCapture(c.s, &graph);
      if (st == PMG_OK && e == cudaSuccess && graph &&
          cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess) {
        g.tol = tol;
        g.epoch = h->tune_epoch;
        g.launches = ws->launches - l0;
      } else {
        g.exec = nullptr;
        ws->graphs = false;            // capture refused here: stay eager on this workspace
      }
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
    } else {
      ws->graphs = false;
      cudaGetLastError();
    }
    ws->launches = l0;
    st = PMG_OK;
  }
  if (graphable && g.exec) {
    PMG_CUDA(cudaGraphLaunch(g.exec, c.s));
    ws->launches += g.launches;
    ++ws->graph_launches;
  } else {
    if ((st = slots_cycle_body(c, precision, tol)) != PMG_OK) return st;
    ++g.eager;
  }
  PMG_CUDA(cudaEventRecord(ws->slot_ev, c.s));
  ws->slot_pending = true;
  return PMG_OK;
}

pmg_status slots_wait_impl(pmg_ws ws, bool blocking, bool* ready) {
  *ready = false;
  if (!ws->slot_pending) { *ready = true; return PMG_OK; }
  const cudaError_t q = blocking ? cudaEventSynchronize(ws->slot_ev) : cudaEventQuery(ws->slot_ev);
  if (q == cudaErrorNotReady) return PMG_OK;
  if (q != cudaSuccess) return fail(PMG_ERR_CUDA, cudaGetErrorString(q));
  ws->slot_pending = false;
  *ready = true;
  collect_profile(ws);
  for (int k = 0; k < ws->R; ++k) ws->slot_state[k] = ws->hm.state[k];
  if (ws->hm.err[0]) {
    cudaMemset(ws->err, 0, 4 * sizeof(unsigned));
    char buf[160];
    std::snprintf(buf, sizeof(buf),
                  "a device-side dependency wait expired (wait sites 0x%x; first: site 0x%x, item %u, row %u, warp %u)",
                  ws->hm.err[0], ws->hm.err[1], ws->hm.err[2], ws->hm.err[3] >> 8, ws->hm.err[3] & 0xffu);
    ws->hm.err[0] = 0;
    return fail(PMG_ERR_TIMEOUT, buf);
  }
  return PMG_OK;
}

pmg_status slots_read_impl(Ctx& c, int slot0, int n, double* U) {
  const int N = c.h->dl[0].N;
  pmgk::k_slots_copy_out<<<grid_for((long long)N * n, 256, c.h->sms * 16), 256, 0, c.s>>>(N, n, c.w->R, slot0,
                                                                                           c.w->bU, U);
  ++c.w->launches;
  PMG_CUDA(cudaGetLastError());
  return PMG_OK;
}

pmg_status slots_release_impl(Ctx& c, int slot0, int n) {
  pmgk::k_slots_release<<<1, 128, 0, c.s>>>(c.w->R, slot0, n, c.w->bmask, c.w->bstate);
  ++c.w->launches;
  PMG_CUDA(cudaGetLastError());
  for (int k = slot0; k < slot0 + n; ++k) c.w->slot_state[k] = 0;
  return PMG_OK;
}

// pmg_solve_batched: all right-hand sides in slots 0..nrhs-1, cycles until
// none is active.
pmg_status solve_batched_impl(pmg_handle h, pmg_ws ws, int nrhs, const double* F, const double* U0, double tol,
                              int max_iter, int precision, double* Uout, int* iters, double* hist,
                              cudaStream_t s) {
  Ctx c{h, ws, s};
  bool ready = false;
  pmg_status st = slots_wait_impl(ws, true, &ready);
  if (st != PMG_OK) return st;
  if ((st = slots_release_impl(c, 0, ws->max_rhs)) != PMG_OK) return st;
  if ((st = slots_load_impl(c, 0, nrhs, F, U0)) != PMG_OK) return st;
  for (int k = 0; k < nrhs; ++k) iters[k] = 0;
  for (int it = 0; it < max_iter; ++it) {
    if (std::find(ws->slot_state.begin(), ws->slot_state.begin() + nrhs, 1) == ws->slot_state.begin() + nrhs) break;
    if ((st = slots_cycle_impl(c, precision, tol)) != PMG_OK) return st;
    if ((st = slots_wait_impl(ws, true, &ready)) != PMG_OK) return st;
    for (int k = 0; k < nrhs; ++k) {
      if (ws->hm.iters[k] != it + 1) continue;        // not active in this cycle
      iters[k] = it + 1;
      if (hist) hist[(size_t)it * nrhs + k] = ws->hm.relres[k];
    }
  }
  pmg_status result = PMG_OK;
  for (int k = 0; k < nrhs; ++k) {
    if (ws->slot_state[k] == 3) result = PMG_ERR_DIVERGED;
    else if (ws->slot_state[k] == 1 && result == PMG_OK) result = PMG_ERR_MAXITER;
  }
  if (result == PMG_ERR_MAXITER) g_last_error = "maximum number of V-cycles reached";
  if (result == PMG_ERR_DIVERGED) g_last_error = "relative residual exceeded 1e10 for a right-hand side";
  if ((st = slots_read_impl(c, 0, nrhs, Uout)) != PMG_OK) return st;
  if ((st = slots_release_impl(c, 0, ws->max_rhs)) != PMG_OK) return st;
  PMG_CUDA(cudaStreamSynchronize(s));
  return result;
}

pmg_status slots_check(pmg_handle h, pmg_ws ws) {
  pmg_status st = check_ws(h, ws);
  if (st != PMG_OK) return st;
  if (ws->R == 0) return fail(PMG_ERR_ARG, "workspace has no right-hand-side slots (max_rhs < 2)");
  return PMG_OK;
}

}  // namespace

extern "C" {

pmg_status pmg_default_options(pmg_options* opt) {
  if (!opt) return fail(PMG_ERR_ARG, "opt is NULL");
  opt->drop_tol = 1e-12;
  opt->fill_factor = 1.0;
  opt->nu_pre = 1;
  opt->nu_post = 1;
  opt->projection = PMG_PROJ_INDIRECT;
  opt->coarse_cycles = 2;
  opt->exact = PMG_U_SINPROD;
  opt->transfer_mass = PMG_MASS_LUMPED;
  return PMG_OK;
}

pmg_status pmg_setup(int domain, int p, int log2_inv_h, const pmg_options* opt, pmg_handle* out) {
  if (!out) return fail(PMG_ERR_ARG, "out is NULL");
  *out = nullptr;
  pmg_options o;
  if (opt) o = *opt; else pmg_default_options(&o);
  if (o.transfer_mass != PMG_MASS_LUMPED && o.transfer_mass != PMG_MASS_CONSISTENT)
    return fail(PMG_ERR_ARG, "options.transfer_mass must be PMG_MASS_LUMPED or PMG_MASS_CONSISTENT");
  pmg_hierarchy_s* h = nullptr;
  try {
    h = new pmg_hierarchy_s();
  } catch (...) {
    return fail(PMG_ERR_OOM, "host allocation failed");
  }
  std::string err;
  pmg_status st = pmgl::build_hierarchy(domain, p, log2_inv_h, o, h->H, err);
  if (st != PMG_OK) { delete h; return fail(st, err); }
  if (h->H.lev.size() > PMG_MAX_LEVELS || h->H.hl.size() > PMG_MAX_LEVELS) { delete h; return fail(PMG_ERR_ARG, "too many levels"); }
  // device layout
  Packer& P = h->pack;
  for (size_t l = 0; l < h->H.lev.size(); ++l) {
    const auto& L = h->H.lev[l];
    h->off_A.push_back(plan_csr(P, L.A));
    h->off_L.push_back(plan_csr(P, L.L));
    h->off_U.push_back(plan_csr(P, L.U));
    h->off_Pro.push_back(plan_csr(P, L.Pro));
    h->off_Res.push_back(plan_csr(P, L.Res));
    auto plan_sell = [&](const pmgl::Csr& a) {
      h->sellstore.push_back(make_sell(a));
      const SellHost& S = h->sellstore.back();
      return SellOff{S.nr, S.nslices, P.add(S.sofs.data(), S.sofs.size() * sizeof(long long)),
                     P.add(S.col.data(), S.col.size() * sizeof(int)), P.add(S.val.data(), S.val.size() * sizeof(double))};
    };
    h->soffA.push_back(plan_sell(L.A));
    h->soffPro.push_back(plan_sell(L.Pro));
    h->soffRes.push_back(plan_sell(L.Res));
    auto& ud = h->udinv_host[l];
    ud.resize(L.udiag.size());
    for (size_t i = 0; i < ud.size(); ++i) ud[i] = 1.0 / L.udiag[i];
    h->off_udinv.push_back(P.add(ud.data(), ud.size() * sizeof(double)));
    h->off_Llp.push_back(plan_lp(P, L.Llp));
    h->off_Ulp.push_back(plan_lp(P, L.Ulp));
  }
  for (const auto& Hl : h->H.hl) {
    h->off_HA.push_back(plan_csr(P, Hl.A));
    h->off_dinv.push_back(P.add(Hl.dinv.data(), Hl.dinv.size() * sizeof(double)));
    h->off_Lo.push_back(plan_csr(P, Hl.Lo));
    h->off_Up.push_back(plan_csr(P, Hl.Up));
    h->off_Lolp.push_back(plan_lp(P, Hl.Lolp));
    h->off_UpMlp.push_back(plan_lp(P, Hl.UpMlp));
  }
  h->off_cinv = P.add(h->H.coarse_inv.data(), h->H.coarse_inv.size() * sizeof(double));
  if (o.transfer_mass == PMG_MASS_CONSISTENT) {
    const int ne = 1 << log2_inv_h;
    auto plan_mass = [&](const std::vector<double>& f0, const std::vector<double>& f1, int q) {
      return pmg_hierarchy_s::MOff{P.add(f0.data(), f0.size() * sizeof(double)), P.add(f1.data(), f1.size() * sizeof(double)),
                                   ne + q - 2, q};
    };
    for (const auto& L : h->H.lev) h->moff.push_back(plan_mass(L.MF0, L.MF1, L.q));
    h->moff.push_back(plan_mass(h->H.M1F0, h->H.M1F1, 1));
  }
  // FP32 copies (inner cycle of the mixed-precision batched solve) and CSR
  // layouts of the mirrored factors for the batched line-pipelined solve
  auto f32 = [&](const std::vector<double>& v) {
    h->f32store.emplace_back(v.begin(), v.end());
    const auto& w = h->f32store.back();
    return P.add(w.data(), w.size() * sizeof(float));
  };
  h->f32store.reserve(8 * h->H.lev.size() + 8);
  for (size_t l = 0; l < h->H.lev.size(); ++l) {
    const auto& L = h->H.lev[l];
    pmg_hierarchy_s::BOff b;
    b.Um = plan_csr(P, L.Um);
    b.A32 = f32(L.A.v);
    b.Res32 = f32(L.Res.v);
    b.Pro32 = f32(L.Pro.v);
    b.L32 = f32(L.L.v);
    b.Um32 = f32(L.Um.v);
    b.udm64 = P.add(L.Ulp.dscale.data(), L.Ulp.dscale.size() * sizeof(double));
    b.udm32 = f32(L.Ulp.dscale);
    h->boff.push_back(b);
  }
  for (const auto& Hl : h->H.hl) {
    pmg_hierarchy_s::HBOff b;
    b.UpM = plan_csr(P, Hl.UpM);
    b.dinvM = P.add(Hl.UpMlp.dscale.data(), Hl.UpMlp.dscale.size() * sizeof(double));
    h->hboff.push_back(b);
  }
  // Ring widths: FP32 chains push 31 values a row (one FMA each, cheap);
  // FP64 FMAs are slow on this part, so FP64 ILUT chains push 15 and the P1
  // sweeps (own-line entries at distance 1 only) push 1.
  // 16-bit copies (round to nearest even) of the FP32 ring layouts' values
  h->h16store.reserve(8 * h->H.lev.size());
  auto h16 = [&](const std::vector<double>& v, bool bf16) {
    h->h16store.emplace_back(v.size());
    auto& w = h->h16store.back();
    for (size_t i = 0; i < v.size(); ++i) {
      if (bf16) { const __nv_bfloat16 q = __float2bfloat16_rn(float(v[i])); std::memcpy(&w[i], &q, 2); }
      else { const __half q = __float2half_rn(float(v[i])); std::memcpy(&w[i], &q, 2); }
    }
    return P.add(w.data(), w.size() * sizeof(uint16_t));
  };
  h->farstore.reserve(6 * (h->H.lev.size() + h->H.hl.size()));
  h->f32store.reserve(h->f32store.size() + 6 * h->H.lev.size());
  auto plan_ring = [&](const pmgl::Csr& M, const pmgl::LpLayout& lp, int nx, int ring, bool fp32) {
    h->farstore.push_back(pmgl::far_part(M, nx, lp.dscale, ring));
    const auto& F = h->farstore.back();
    pmg_hierarchy_s::COff c{};
    c.far = plan_csr(P, F);
    c.ring = ring;
    if (fp32) {
      c.far32 = f32(F.v); c.push32 = f32(lp.push); c.d32 = f32(lp.dscale);
      c.far16 = h16(F.v, false); c.push16 = h16(lp.push, false);
      c.farb = h16(F.v, true); c.pushb = h16(lp.push, true);
    }
    return c;
  };
  for (const auto& L : h->H.lev) {
    h->coffL.push_back(plan_ring(L.L, L.Llp, L.n1d, 16, false));
    h->coffU.push_back(plan_ring(L.Um, L.Ulp, L.n1d, 16, false));
    h->coffL32.push_back(plan_ring(L.L, L.Llp, L.n1d, 32, true));
    h->coffU32.push_back(plan_ring(L.Um, L.Ulp, L.n1d, 32, true));
  }
  for (const auto& Hl : h->H.hl) {
    h->coffLo.push_back(plan_ring(Hl.Lo, Hl.Lolp, Hl.n1d, 2, false));
    h->coffUpM.push_back(plan_ring(Hl.UpM, Hl.UpMlp, Hl.n1d, 2, false));
  }
  // Wavefront sweeps of the 2D P1 levels: per row the coefficients (SW, S, SE,
  // W) of the sweep's strict lower part, scaled by 1/a_ii, in the sweep's index
  // space (mirrored for the backward sweep); levels with another pattern keep
  // the other kernels.
  h->wavestore.reserve(2 * h->H.hl.size());
  for (const auto& Hl : h->H.hl) {
    pmg_hierarchy_s::WOff w{0, 0, false};
    const int m = Hl.n1d;
    auto build = [&](const pmgl::Csr& T, const std::vector<double>& d, std::vector<double>& c) {
      c.assign(size_t(Hl.N) * 4, 0.0);
      for (int i = 0; i < Hl.N; ++i)
        for (int t = T.rp[i]; t < T.rp[i + 1]; ++t) {
          const int j = T.ci[t];
          const int dl = i / m - j / m, dx = i % m - j % m;
          int slot = -1;
          if (dl == 0 && dx == 1) slot = 3;
          else if (dl == 1 && dx == 1) slot = 0;
          else if (dl == 1 && dx == 0) slot = 1;
          else if (dl == 1 && dx == -1) slot = 2;
          if (slot < 0) return false;
          c[size_t(i) * 4 + size_t(slot)] = T.v[t] * d[size_t(i)];
        }
      return true;
    };
    if (h->H.d == 2 && m >= 2 && m <= pmgk::kWaveMaxLines && size_t(m) * size_t(m) == size_t(Hl.N)) {
      std::vector<double> cf, cb;
      if (build(Hl.Lo, Hl.dinv, cf) && build(Hl.UpM, Hl.UpMlp.dscale, cb)) {
        h->wavestore.push_back(std::move(cf));
        w.f = P.add(h->wavestore.back().data(), h->wavestore.back().size() * sizeof(double));
        h->wavestore.push_back(std::move(cb));
        w.b = P.add(h->wavestore.back().data(), h->wavestore.back().size() * sizeof(double));
        w.ok = true;
      }
    }
    h->woff.push_back(w);
  }
  *out = h;
  return PMG_OK;
}

pmg_status pmg_info(pmg_handle h, pmg_info_t* info) {
  if (!h || !info) return fail(PMG_ERR_ARG, "null argument");
  std::memset(info, 0, sizeof(*info));
  const auto& H = h->H;
  info->dim = H.d;
  info->p = H.p;
  info->log2_inv_h = H.k;
  info->nlevels = int(H.lev.size());
  double bytes = 0, flops = 0;
  const int nu = H.opt.nu_pre + H.opt.nu_post;
  for (size_t l = 0; l < H.lev.size(); ++l) {
    const auto& L = H.lev[l];
    info->degree[l] = L.q;
    info->n[l] = L.N;
    info->nnz_A[l] = L.A.nnz();
    info->nnz_L[l] = L.L.nnz();
    info->nnz_U[l] = L.U.nnz() + L.N;
    info->nnz_P[l] = L.Praw.nnz();
    info->depth_L[l] = L.depthL;
    info->depth_U[l] = L.depthU;
    // residual SpMVs: 1 + nu per cycle (the pre-smoothing one is reused), TRSVs: 2 per smoothing step
    const double nA = double(L.A.nnz()), nL = double(L.L.nnz()), nU = double(L.U.nnz());
    const double nP = double(L.Praw.nnz()), N = L.N;
    const double spmvs = 1 + nu;
    bytes += spmvs * (12 * nA + 4 * (N + 1) + 3 * 8 * N);
    bytes += nu * (12 * (nL + nU) + 8 * (N + 1) + 8 * N /*udinv*/ + 6 * 8 * N);
    bytes += 2 * (12 * nP) + 4 * 2 * (N + 1) + 2 * 3 * 8 * N;
    flops += spmvs * 2 * nA + nu * (2 * (nL + nU) + 2 * N) + 2 * 2 * nP;
  }
  info->nhlevels = int(H.hl.size());
  for (size_t j = 0; j < H.hl.size(); ++j) {
    const auto& Hl = H.hl[j];
    info->n_h[j] = Hl.N;
    info->nnz_h[j] = Hl.A.nnz();
    info->depth_gs[j] = Hl.depthGS;
    const double nA = double(Hl.A.nnz()), N = Hl.N;
    if (j + 1 < H.hl.size()) {
      // two GS sweeps + one residual + transfers per h-cycle
      bytes += H.opt.coarse_cycles * (3 * (12 * nA + 4 * (N + 1) + 3 * 8 * N) + 8 * 8 * N);
      flops += H.opt.coarse_cycles * (3 * 2 * nA + 2 * 9 * N);
    } else {
      bytes += H.opt.coarse_cycles * (8.0 * N * N + 16 * N);
      flops += H.opt.coarse_cycles * 2.0 * N * N;
    }
  }
  info->device_bytes = h->pack.size;
  info->setup_ms_assembly = H.t_assembly;
  info->setup_ms_ilut = H.t_ilut;
  info->setup_ms_transfer = H.t_transfer;
  info->setup_ms_hmg = H.t_hmg;
  info->cycle_bytes = bytes;
  info->cycle_flops = flops;
  for (size_t l = 0; l < H.lev.size(); ++l) {
    const PTune t = l < h->ptune.size() ? h->ptune[l] : PTune{};
    info->tune_p[l] = t.sL | (t.sU << 2) | (t.bL[0] << 4) | (t.bU[0] << 6) | (t.bL[1] << 8) | (t.bU[1] << 10) |
                      (t.cL << 12) | (t.cU << 15);
  }
  for (size_t j = 0; j < H.hl.size(); ++j) {
    const HTune t = j < h->htune.size() ? h->htune[j] : HTune{};
    info->tune_h[j] = t.gF | (t.gB << 2) | (t.bF << 4) | (t.bB << 6) | (t.cF << 8) | (t.cB << 11);
  }
  return PMG_OK;
}

pmg_status pmg_upload(pmg_handle h, void* arena, size_t bytes, void* stream) {
  if (!h || !arena) return fail(PMG_ERR_ARG, "null argument");
  if (bytes < h->pack.size) return fail(PMG_ERR_ARG, "arena too small");
  if (reinterpret_cast<uintptr_t>(arena) % kAlign) return fail(PMG_ERR_ARG, "arena not 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<char> staging(h->pack.size, 0);
  for (const auto& it : h->pack.items)
    if (it.bytes) std::memcpy(staging.data() + it.off, it.src, it.bytes);
  PMG_CUDA(cudaMemcpyAsync(arena, staging.data(), h->pack.size, cudaMemcpyHostToDevice, s));
  PMG_CUDA(cudaStreamSynchronize(s));
  int dev = 0;
  PMG_CUDA(cudaGetDevice(&dev));
  PMG_CUDA(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev));
  char* base = static_cast<char*>(arena);
  h->arena = base;
  h->dl.clear();
  h->dh.clear();
  for (size_t l = 0; l < h->H.lev.size(); ++l) {
    DevPLevel D;
    D.N = h->H.lev[l].N;
    D.A = bind(h->off_A[l], base);
    D.avg_nnz = double(h->off_A[l].nnz) / std::max(1, D.N);
    D.L = bind(h->off_L[l], base);
    D.U = bind(h->off_U[l], base);
    D.Pro = bind(h->off_Pro[l], base);
    D.Res = bind(h->off_Res[l], base);
    auto bind_sell = [&](const SellOff& o) {
      return pmgk::Sell{o.nr, o.nslices, reinterpret_cast<const long long*>(base + o.sofs),
                        reinterpret_cast<const int4*>(base + o.col), reinterpret_cast<const double2*>(base + o.val)};
    };
    D.sA = bind_sell(h->soffA[l]);
    D.sPro = bind_sell(h->soffPro[l]);
    D.sRes = bind_sell(h->soffRes[l]);
    D.udinv = reinterpret_cast<const double*>(base + h->off_udinv[l]);
    D.nnzA = h->off_A[l].nnz;
    D.nnzL = h->off_L[l].nnz;
    D.nnzU = h->off_U[l].nnz;
    D.nnzP = h->off_Pro[l].nnz;
    D.Llp = bind_lp(h->off_Llp[l], base);
    D.Ulp = bind_lp(h->off_Ulp[l], base);
    {
      const auto& b = h->boff[l];
      const int nx = h->H.lev[l].n1d;
      auto fp = [&](size_t off) { return reinterpret_cast<const float*>(base + off); };
      D.A32 = pmgk::TCsr<float>{D.A.nr, D.A.rp, D.A.ci, fp(b.A32)};
      D.Res32 = pmgk::TCsr<float>{D.Res.nr, D.Res.rp, D.Res.ci, fp(b.Res32)};
      D.Pro32 = pmgk::TCsr<float>{D.Pro.nr, D.Pro.rp, D.Pro.ci, fp(b.Pro32)};
      const pmgk::Csr Um = bind(b.Um, base);
      D.Lb64 = pmgk::LpB<double>{D.N, nx, D.N / nx, D.L.rp, D.L.ci, D.L.v, nullptr};
      D.Ub64 = pmgk::LpB<double>{D.N, nx, D.N / nx, Um.rp, Um.ci, Um.v,
                                 reinterpret_cast<const double*>(base + b.udm64)};
      D.Lb32 = pmgk::LpB<float>{D.N, nx, D.N / nx, D.L.rp, D.L.ci, fp(b.L32), nullptr};
      D.Ub32 = pmgk::LpB<float>{D.N, nx, D.N / nx, Um.rp, Um.ci, fp(b.Um32), fp(b.udm32)};
      const auto& cl = h->coffL[l];
      const auto& cu = h->coffU[l];
      const auto& cl32 = h->coffL32[l];
      const auto& cu32 = h->coffU32[l];
      const pmgk::Csr FL = bind(cl.far, base), FU = bind(cu.far, base);
      const pmgk::Csr FL32 = bind(cl32.far, base), FU32 = bind(cu32.far, base);
      D.inflightL = lines_in_flight(h->H.lev[l].depthL, nx, D.N / nx);
      D.inflightU = lines_in_flight(h->H.lev[l].depthU, nx, D.N / nx);
      D.Lc64 = pmgk::LpC<double>{D.N, nx, D.N / nx, cl.ring, FL.rp, FL.ci, FL.v, D.Llp.push, nullptr};
      D.Uc64 = pmgk::LpC<double>{D.N, nx, D.N / nx, cu.ring, FU.rp, FU.ci, FU.v, D.Ulp.push, D.Ulp.dscale};
      D.Lc32 = pmgk::LpC<float>{D.N, nx, D.N / nx, cl32.ring, FL32.rp, FL32.ci, fp(cl32.far32), fp(cl32.push32),
                                nullptr};
      D.Uc32 = pmgk::LpC<float>{D.N, nx, D.N / nx, cu32.ring, FU32.rp, FU32.ci, fp(cu32.far32), fp(cu32.push32),
                                fp(cu32.d32)};
      auto hp = [&](size_t off) { return reinterpret_cast<const __half*>(base + off); };
      auto bp = [&](size_t off) { return reinterpret_cast<const __nv_bfloat16*>(base + off); };
      D.Lc16 = pmgk::LpC<float, __half>{D.N, nx, D.N / nx, cl32.ring, FL32.rp, FL32.ci, hp(cl32.far16),
                                        hp(cl32.push16), nullptr};
      D.Uc16 = pmgk::LpC<float, __half>{D.N, nx, D.N / nx, cu32.ring, FU32.rp, FU32.ci, hp(cu32.far16),
                                        hp(cu32.push16), fp(cu32.d32)};
      D.Lcb = pmgk::LpC<float, __nv_bfloat16>{D.N, nx, D.N / nx, cl32.ring, FL32.rp, FL32.ci, bp(cl32.farb),
                                              bp(cl32.pushb), nullptr};
      D.Ucb = pmgk::LpC<float, __nv_bfloat16>{D.N, nx, D.N / nx, cu32.ring, FU32.rp, FU32.ci, bp(cu32.farb),
                                              bp(cu32.pushb), fp(cu32.d32)};
    }
    h->dl.push_back(D);
  }
  for (size_t j = 0; j < h->H.hl.size(); ++j) {
    DevHLevel D;
    D.N = h->H.hl[j].N;
    D.ne = h->H.hl[j].ne;
    D.A = bind(h->off_HA[j], base);
    D.dinv = reinterpret_cast<const double*>(base + h->off_dinv[j]);
    D.nnzA = h->off_HA[j].nnz;
    D.Lo = bind(h->off_Lo[j], base);
    D.Up = bind(h->off_Up[j], base);
    if (h->woff[j].ok) {
      D.wave_f = reinterpret_cast<const double*>(base + h->woff[j].f);
      D.wave_b = reinterpret_cast<const double*>(base + h->woff[j].b);
    }
    D.Lolp = bind_lp(h->off_Lolp[j], base);
    D.UpMlp = bind_lp(h->off_UpMlp[j], base);
    {
      const int nx = h->H.hl[j].n1d;
      const pmgk::Csr UpM = bind(h->hboff[j].UpM, base);
      D.Lob = pmgk::LpB<double>{D.N, nx, D.N / nx, D.Lo.rp, D.Lo.ci, D.Lo.v, D.dinv};
      D.UpMb = pmgk::LpB<double>{D.N, nx, D.N / nx, UpM.rp, UpM.ci, UpM.v,
                                 reinterpret_cast<const double*>(base + h->hboff[j].dinvM)};
      D.inflightGS = lines_in_flight(h->H.hl[j].depthGS, nx, D.N / nx);
      const pmgk::Csr FLo = bind(h->coffLo[j].far, base), FUp = bind(h->coffUpM[j].far, base);
      D.Loc = pmgk::LpC<double>{D.N, nx, D.N / nx, h->coffLo[j].ring, FLo.rp, FLo.ci, FLo.v, D.Lolp.push,
                                D.Lolp.dscale};
      D.UpMc = pmgk::LpC<double>{D.N, nx, D.N / nx, h->coffUpM[j].ring, FUp.rp, FUp.ci, FUp.v, D.UpMlp.push,
                                 D.UpMlp.dscale};
    }
    D.avg_lo = double(h->off_Lo[j].nnz) / std::max(1, D.N);
    D.avg_up = double(h->off_Up[j].nnz) / std::max(1, D.N);
    h->dh.push_back(D);
  }
  h->cinv = reinterpret_cast<const double*>(base + h->off_cinv);
  if (!h->moff.empty()) {
    auto bind_mass = [&](const pmg_hierarchy_s::MOff& m) {
      return MassF{reinterpret_cast<const double*>(base + m.f0), reinterpret_cast<const double*>(base + m.f1), m.n, m.q};
    };
    for (size_t l = 0; l < h->dl.size(); ++l) h->dl[l].mass = bind_mass(h->moff[l]);
    h->mass1 = bind_mass(h->moff.back());
  }
  h->ptune.assign(h->dl.size(), PTune{});
  h->htune.assign(h->dh.size(), HTune{});
  h->uploaded = true;
  return PMG_OK;
}

pmg_status pmg_rhs(pmg_handle h, double* f_host) {
  if (!h || !f_host) return fail(PMG_ERR_ARG, "null argument");
  std::memcpy(f_host, h->H.f.data(), h->H.f.size() * sizeof(double));
  return PMG_OK;
}

pmg_status pmg_workspace_bytes(pmg_handle h, int max_rhs, size_t* bytes) {
  if (!h || !bytes || max_rhs < 1) return fail(PMG_ERR_ARG, "invalid argument");
  *bytes = plan_ws(h, max_rhs).total;
  return PMG_OK;
}

pmg_status pmg_workspace_create(pmg_handle h, int max_rhs, void* mem, size_t bytes, void* stream, pmg_ws* out) {
  if (!h || !mem || !out || max_rhs < 1) return fail(PMG_ERR_ARG, "invalid argument");
  *out = nullptr;
  if (max_rhs > 1 && h->H.opt.transfer_mass == PMG_MASS_CONSISTENT)
    return fail(PMG_ERR_ARG, "consistent-mass transfers support single-vector solves only (max_rhs must be 1)");
  WsLayout W = plan_ws(h, max_rhs);
  if (bytes < W.total) return fail(PMG_ERR_ARG, "workspace memory too small");
  if (reinterpret_cast<uintptr_t>(mem) % kAlign) return fail(PMG_ERR_ARG, "workspace memory not 256-byte aligned");
  pmg_workspace_s* w = new (std::nothrow) pmg_workspace_s();
  if (!w) return fail(PMG_ERR_OOM, "host allocation failed");
  char* base = static_cast<char*>(mem);
  auto P = [&](size_t off) { return reinterpret_cast<double*>(base + off); };
  w->h = h;
  w->max_rhs = max_rhs;
  for (size_t l = 0; l < W.f.size(); ++l) {
    w->f.push_back(P(W.f[l])); w->u.push_back(P(W.u[l])); w->r.push_back(P(W.r[l]));
    w->y.push_back(P(W.y[l])); w->e.push_back(P(W.e[l]));
  }
  for (size_t j = 0; j < W.hb.size(); ++j) {
    w->hb.push_back(P(W.hb[j])); w->hx.push_back(P(W.hx[j])); w->hr.push_back(P(W.hr[j]));
    w->hg.push_back(P(W.hg[j]));
  }
  w->R = W.R;
  for (size_t l = 0; l < W.bf.size(); ++l) {
    w->bf.push_back(P(W.bf[l])); w->be.push_back(P(W.be[l])); w->br.push_back(P(W.br[l]));
    w->by.push_back(P(W.by[l])); w->bt.push_back(P(W.bt[l]));
  }
  for (size_t j = 0; j < W.bhb.size(); ++j) {
    w->bhb.push_back(P(W.bhb[j])); w->bhx.push_back(P(W.bhx[j])); w->bhr.push_back(P(W.bhr[j]));
    w->bhg.push_back(P(W.bhg[j])); w->bht.push_back(P(W.bht[j]));
  }
  if (W.R) {
    w->bF = P(W.bF); w->bU = P(W.bU); w->bR = P(W.bR);
    w->br0 = P(W.br0); w->brel = P(W.brel); w->bmask = P(W.bmask); w->bpart = P(W.bpart);
    w->bstate = reinterpret_cast<int*>(base + W.bstate);
    w->biters = reinterpret_cast<int*>(base + W.biters);
    // pinned host mirror of the slot state (host memory; the library allocates no device memory)
    const size_t hb = size_t(W.R) * (sizeof(double) + 2 * sizeof(int)) + 4 * sizeof(unsigned);
    if (cudaHostAlloc(&w->hm_block, hb, cudaHostAllocDefault) != cudaSuccess ||
        cudaEventCreateWithFlags(&w->slot_ev, cudaEventDisableTiming) != cudaSuccess) {
      delete w;
      return fail(PMG_ERR_CUDA, "pinned slot mirror / event creation failed");
    }
    char* hbp = static_cast<char*>(w->hm_block);
    w->hm.relres = reinterpret_cast<double*>(hbp);
    w->hm.state = reinterpret_cast<int*>(hbp + size_t(W.R) * sizeof(double));
    w->hm.iters = w->hm.state + W.R;
    w->hm.err = reinterpret_cast<unsigned*>(w->hm.iters + W.R);
    std::memset(w->hm_block, 0, hb);
    w->slot_state.assign(size_t(W.R), 0);
  }
  for (int k = 0; k < 8; ++k) w->kv[k] = P(W.kv[k]);
  w->kd = P(W.kd);
  w->flags = reinterpret_cast<unsigned*>(base + W.flags);
  w->lprog = reinterpret_cast<unsigned long long*>(base + W.lprog);
  w->counters = reinterpret_cast<unsigned*>(base + W.counters);
  w->err = reinterpret_cast<unsigned*>(base + W.err);
  w->partial = P(W.partial);
  w->r0 = P(W.r0);
  w->hist = P(W.hist);
  w->f_in = P(W.f_in);
  w->u_io = P(W.u_io);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(mem, 0, W.total, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { delete w; return fail(PMG_ERR_CUDA, std::string("workspace init: ") + cudaGetErrorString(e)); }
  *out = w;
  return PMG_OK;
}

pmg_status pmg_solve(pmg_handle h, pmg_ws ws, const double* f, const double* u0, double tol, int max_iter,
                     double* u, int* iters, double* hist, int hist_cap, void* stream) {
  pmg_status st = check_ws(h, ws);
  if (st != PMG_OK) return st;
  if (!f || !u0 || !u || max_iter < 1 || !(tol > 0)) return fail(PMG_ERR_ARG, "invalid solve argument");
  return solve_impl(h, ws, f, u0, tol, max_iter, u, iters, hist, hist_cap, static_cast<cudaStream_t>(stream));
}

pmg_status pmg_solve_bicgstab(pmg_handle h, pmg_ws ws, const double* f, const double* u0, double tol,
                              int max_iter, double* u, int* iters, double* hist, int hist_cap, void* stream) {
  pmg_status st = check_ws(h, ws);
  if (st != PMG_OK) return st;
  if (!f || !u0 || !u || max_iter < 1 || !(tol > 0)) return fail(PMG_ERR_ARG, "invalid solve argument");
  return bicgstab_impl(h, ws, f, u0, tol, max_iter, u, iters, hist, hist_cap, static_cast<cudaStream_t>(stream));
}

pmg_status pmg_solve_host(pmg_handle h, pmg_ws ws, const double* f_host, const double* u0_host, double tol,
                          int max_iter, double* u_host, int* iters, double* hist, int hist_cap, void* stream) {
  pmg_status st = check_ws(h, ws);
  if (st != PMG_OK) return st;
  if (!f_host || !u0_host || !u_host || max_iter < 1 || !(tol > 0)) return fail(PMG_ERR_ARG, "invalid solve argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = size_t(h->dl[0].N) * sizeof(double);
  PMG_CUDA(cudaMemcpyAsync(ws->f_in, f_host, bytes, cudaMemcpyHostToDevice, s));
  PMG_CUDA(cudaMemcpyAsync(ws->u_io, u0_host, bytes, cudaMemcpyHostToDevice, s));
  st = solve_impl(h, ws, ws->f_in, ws->u_io, tol, max_iter, ws->u_io, iters, hist, hist_cap, s);
  if (st == PMG_ERR_CUDA || st == PMG_ERR_TIMEOUT) return st;
  std::string keep = g_last_error;
  PMG_CUDA(cudaMemcpyAsync(u_host, ws->u_io, bytes, cudaMemcpyDeviceToHost, s));
  PMG_CUDA(cudaStreamSynchronize(s));
  g_last_error = keep;
  return st;
}

pmg_status pmg_solve_batched(pmg_handle h, pmg_ws ws, int nrhs, const double* F, const double* U0, double tol,
                             int max_iter, int precision, double* U, int* iters, double* hist, void* stream) {
  pmg_status st = check_ws(h, ws);
  if (st != PMG_OK) return st;
  if (nrhs < 1 || nrhs > ws->max_rhs || ws->R == 0 || !F || !U0 || !U || !iters || max_iter < 1 || !(tol > 0) ||
      precision < PMG_PREC_FP64 || precision > PMG_PREC_MIXED_BF16)
    return fail(PMG_ERR_ARG, "invalid batched solve argument (workspace holds " + std::to_string(ws->R ? ws->max_rhs : 0) + " right-hand sides)");
  return solve_batched_impl(h, ws, nrhs, F, U0, tol, max_iter, precision, U, iters, hist,
                            static_cast<cudaStream_t>(stream));
}

pmg_status pmg_slots_load(pmg_handle h, pmg_ws ws, int slot0, int n, const double* F, const double* U0,
                          void* stream) {
  pmg_status st = slots_check(h, ws);
  if (st != PMG_OK) return st;
  if (slot0 < 0 || n < 1 || slot0 + n > ws->max_rhs || !F || !U0) return fail(PMG_ERR_ARG, "invalid slot range");
  if (ws->slot_pending) return fail(PMG_ERR_BUSY, "a cycle is pending: call pmg_slots_wait first");
  for (int k = slot0; k < slot0 + n; ++k)
    if (ws->slot_state[k] == 1) return fail(PMG_ERR_BUSY, "slot " + std::to_string(k) + " is active");
  Ctx c{h, ws, static_cast<cudaStream_t>(stream)};
  return slots_load_impl(c, slot0, n, F, U0);
}

pmg_status pmg_slots_cycle(pmg_handle h, pmg_ws ws, int precision, double rel_tol, void* stream) {
  pmg_status st = slots_check(h, ws);
  if (st != PMG_OK) return st;
  if (!(rel_tol > 0) || precision < PMG_PREC_FP64 || precision > PMG_PREC_MIXED_BF16)
    return fail(PMG_ERR_ARG, "invalid cycle argument");
  if (ws->slot_pending) return fail(PMG_ERR_BUSY, "a cycle is pending: call pmg_slots_wait first");
  if (std::find(ws->slot_state.begin(), ws->slot_state.end(), 1) == ws->slot_state.end()) return PMG_OK;
  Ctx c{h, ws, static_cast<cudaStream_t>(stream)};
  return slots_cycle_impl(c, precision, rel_tol);
}

pmg_status pmg_slots_wait(pmg_handle h, pmg_ws ws, int blocking, int* ready, double* relres, int* state, int* iters) {
  pmg_status st = slots_check(h, ws);
  if (st != PMG_OK) return st;
  if (!ready) return fail(PMG_ERR_ARG, "ready is NULL");
  bool r = false;
  st = slots_wait_impl(ws, blocking != 0, &r);
  *ready = r ? 1 : 0;
  if (st != PMG_OK || !r) return st;
  for (int k = 0; k < ws->max_rhs; ++k) {
    if (relres) relres[k] = ws->hm.relres[k];
    if (state) state[k] = ws->slot_state[k];
    if (iters) iters[k] = ws->hm.iters[k];
  }
  return PMG_OK;
}

pmg_status pmg_slots_read(pmg_handle h, pmg_ws ws, int slot0, int n, double* U, void* stream) {
  pmg_status st = slots_check(h, ws);
  if (st != PMG_OK) return st;
  if (slot0 < 0 || n < 1 || slot0 + n > ws->max_rhs || !U) return fail(PMG_ERR_ARG, "invalid slot range");
  Ctx c{h, ws, static_cast<cudaStream_t>(stream)};
  return slots_read_impl(c, slot0, n, U);
}

pmg_status pmg_slots_release(pmg_handle h, pmg_ws ws, int slot0, int n, void* stream) {
  pmg_status st = slots_check(h, ws);
  if (st != PMG_OK) return st;
  if (slot0 < 0 || n < 1 || slot0 + n > ws->max_rhs) return fail(PMG_ERR_ARG, "invalid slot range");
  if (ws->slot_pending) return fail(PMG_ERR_BUSY, "a cycle is pending: call pmg_slots_wait first");
  Ctx c{h, ws, static_cast<cudaStream_t>(stream)};
  return slots_release_impl(c, slot0, n);
}

pmg_status pmg_autotune(pmg_handle h, pmg_ws ws, void* stream) {
  pmg_status st = check_ws(h, ws);
  if (st != PMG_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Ctx c{h, ws, s};
  const bool prof = ws->prof;
  ws->prof = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    ws->prof = prof;
    return fail(PMG_ERR_CUDA, "event creation failed");
  }
  pmg_status err = PMG_OK;
  // best of three timed runs after one warm-up run, in ms
  auto timeit = [&](auto&& fn) -> double {
    double best = 1e300;
    for (int rep = 0; rep < 4 && err == PMG_OK; ++rep) {
      if ((err = begin_launches(c)) != PMG_OK) break;
      cudaEventRecord(e0, s);
      fn();
      cudaEventRecord(e1, s);
      if ((err = finish_launches(c)) != PMG_OK) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) best = std::min(best, double(ms));
    }
    return best;
  };
  auto fill = [&](auto* p, long long n) {
    using T = std::remove_pointer_t<decltype(p)>;
    pmgk::k_fill<T><<<grid_for(n, 256, h->sms * 16), 256, 0, s>>>(n, T(1), p);
  };
  auto pick = [&](unsigned char& slot, std::initializer_list<unsigned char> cands, auto&& fn) {
    double best = 1e300;
    unsigned char arg = slot;
    for (unsigned char v : cands) {
      slot = v;
      const double t = timeit(fn);
      if (t < best) { best = t; arg = v; }
    }
    slot = arg;
  };
  // single-vector solves and sweeps: the windowed kernel, the ring kernel and
  // every chain configuration of the clustered kernel
  auto pick_single = [&](unsigned char& var, unsigned char& cfg, bool ring_ok, bool wave_ok, auto&& fn) {
    double best = 1e300;
    unsigned char bv = var, bc = cfg;
    auto trial = [&](unsigned char v, unsigned char k) {
      var = v;
      cfg = k;
      const double t = timeit(fn);
      if (t < best) { best = t; bv = v; bc = k; }
    };
    trial(kVarLp2, cfg);
    if (ring_ok) trial(kVarRing, cfg);
    if (wave_ok) trial(kVarWave, cfg);
    for (int k = 0; k < kNumLp4Cfgs; ++k) trial(kVarCluster, (unsigned char)k);
    var = bv;
    cfg = bc;
  };
  const size_t cap = kLpSmemCap;
  for (size_t l = 0; l < h->dl.size() && err == PMG_OK; ++l) {
    const DevPLevel& D = h->dl[l];
    const int L = int(l);
    fill(ws->f[l], D.N);
    const bool ring_ok = size_t(D.Lc64.nx + 64) * 32 * sizeof(double) <= cap;
    pick_single(h->ptune[l].sL, h->ptune[l].cL, ring_ok, false, [&] { lsolve(c, L, ws->f[l], ws->y[l]); });
    pick_single(h->ptune[l].sU, h->ptune[l].cU, ring_ok, false, [&] { usolve(c, L, ws->f[l], ws->e[l], ws->u[l]); });
    if (ws->R) {
      const long long nR = (long long)D.N * ws->R;
      double* b64 = ws->bf[l];
      float* b32 = reinterpret_cast<float*>(ws->br[l]);
      fill(b64, nR);
      fill(b32, nR);
      for (int up = 0; up < 2; ++up) {
        unsigned char& s64 = up ? h->ptune[l].bU[0] : h->ptune[l].bL[0];
        unsigned char& s32 = up ? h->ptune[l].bU[1] : h->ptune[l].bL[1];
        pick(s64, {kVarRing, kVarLines}, [&] { b_tri<double>(c, L, up, s64, b64, ws->by[l]); });
        pick(s32, {kVarRing, kVarLines},
             [&] { b_tri<float>(c, L, up, s32, b32, reinterpret_cast<float*>(ws->bt[l])); });
      }
    }
  }
  for (size_t j = 0; j + 1 < h->dh.size() && err == PMG_OK; ++j) {
    const DevHLevel& D = h->dh[j];
    const int J = int(j);
    fill(ws->hb[j], D.N);
    fill(ws->hx[j], D.N);
    const bool ring_ok = size_t(D.Loc.nx + 64) * 32 * sizeof(double) <= cap;
    const bool wave_ok = D.wave_f != nullptr;
    pick_single(h->htune[j].gF, h->htune[j].cF, ring_ok, wave_ok, [&] { gs(c, J, false, ws->hb[j], ws->hx[j]); });
    pick_single(h->htune[j].gB, h->htune[j].cB, ring_ok, wave_ok, [&] { gs(c, J, true, ws->hb[j], ws->hx[j]); });
    if (ws->R) {
      const long long nR = (long long)D.N * ws->R;
      fill(ws->bhb[j], nR);
      fill(ws->bhx[j], nR);
      pick(h->htune[j].bF, {kVarRing, kVarLines}, [&] { b_gs(c, J, false, ws->bhb[j], ws->bhx[j]); });
      pick(h->htune[j].bB, {kVarRing, kVarLines}, [&] { b_gs(c, J, true, ws->bhb[j], ws->bhx[j]); });
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ws->prof = prof;
  ++h->tune_epoch;
  return err;
}

pmg_status pmg_set_kernels(pmg_handle h, const int* tune_p, const int* tune_h) {
  if (!h || !tune_p || !tune_h) return fail(PMG_ERR_ARG, "null argument");
  if (!h->uploaded) return fail(PMG_ERR_STATE, "hierarchy not uploaded");
  auto field = [](int v, int k) { return (unsigned char)((v >> (2 * k)) & 3); };
  auto single_ok = [](unsigned char f) { return f != kVarLines; };
  auto batched_ok = [](unsigned char f) { return f == kVarRing || f == kVarLines; };
  for (size_t l = 0; l < h->dl.size(); ++l) {
    const int v = tune_p[l];
    if (!single_ok(field(v, 0)) || !single_ok(field(v, 1)))
      return fail(PMG_ERR_ARG, "single-vector solves take variant 0, 1 or 3");
    for (int k = 2; k < 6; ++k)
      if (!batched_ok(field(v, k))) return fail(PMG_ERR_ARG, "batched solves take variant 1 or 2");
  }
  for (size_t j = 0; j < h->dh.size(); ++j) {
    const int v = tune_h[j];
    if (!batched_ok(field(v, 2)) || !batched_ok(field(v, 3))) return fail(PMG_ERR_ARG, "invalid sweep variant");
  }
  for (size_t l = 0; l < h->dl.size(); ++l) {
    const int v = tune_p[l];
    PTune& t = h->ptune[l];
    t.sL = field(v, 0); t.sU = field(v, 1);
    t.bL[0] = field(v, 2); t.bU[0] = field(v, 3); t.bL[1] = field(v, 4); t.bU[1] = field(v, 5);
    t.cL = (v >> 12) & 7; t.cU = (v >> 15) & 7;
  }
  for (size_t j = 0; j < h->dh.size(); ++j) {
    const int v = tune_h[j];
    HTune& t = h->htune[j];
    t.gF = field(v, 0); t.gB = field(v, 1); t.bF = field(v, 2); t.bB = field(v, 3);
    t.cF = (v >> 8) & 7; t.cB = (v >> 11) & 7;
  }
  ++h->tune_epoch;
  return PMG_OK;
}

pmg_status pmg_apply(pmg_handle h, pmg_ws ws, int op, int level, const double* x, const double* b, double* y,
                     void* stream) {
  pmg_status st = check_ws(h, ws);
  if (st != PMG_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Ctx c{h, ws, s};
  const int nlev = int(h->dl.size()), nh = int(h->dh.size());
  const bool plevel_op = op <= PMG_OP_VCYCLE && op != PMG_OP_COARSE_SOLVE;
  if (plevel_op && (level < 0 || level >= nlev)) return fail(PMG_ERR_ARG, "level out of range");
  if (!plevel_op && op != PMG_OP_COARSE_SOLVE && (level < 0 || level >= nh)) return fail(PMG_ERR_ARG, "level out of range");
  st = begin_launches(c);
  if (st != PMG_OK) return st;
  switch (op) {
    case PMG_OP_RESIDUAL:
      residual(c, level, b, x, y);
      break;
    case PMG_OP_SMOOTH: {
      const int N = h->dl[level].N;
      if (y != x) PMG_CUDA(cudaMemcpyAsync(y, x, size_t(N) * sizeof(double), cudaMemcpyDeviceToDevice, s));
      residual(c, level, b, y, ws->r[level]);
      smooth_from_residual(c, level, ws->r[level], y);
      break;
    }
    case PMG_OP_LSOLVE:
      lsolve(c, level, b, y);
      break;
    case PMG_OP_USOLVE:
      usolve(c, level, b, y, nullptr);
      break;
    case PMG_OP_RESTRICT:
      restrict_to(c, level, x, y);
      break;
    case PMG_OP_PROLONG_ADD:
      prolong_add(c, level, x, b, y);
      break;
    case PMG_OP_COARSE_SOLVE:
      coarse_solve(c, b, y);
      break;
    case PMG_OP_VCYCLE: {
      const int N = h->dl[level].N;
      if (y != x) PMG_CUDA(cudaMemcpyAsync(y, x, size_t(N) * sizeof(double), cudaMemcpyDeviceToDevice, s));
      vcycle(c, level, b, y, nullptr);
      break;
    }
    case PMG_OP_GS_FWD:
    case PMG_OP_GS_BWD: {
      const int N = h->dh[level].N;
      if (y != x) PMG_CUDA(cudaMemcpyAsync(y, x, size_t(N) * sizeof(double), cudaMemcpyDeviceToDevice, s));
      gs(c, level, op == PMG_OP_GS_BWD, b, y);
      break;
    }
    case PMG_OP_HMG_VCYCLE: {
      const int N = h->dh[level].N;
      if (y != x) PMG_CUDA(cudaMemcpyAsync(y, x, size_t(N) * sizeof(double), cudaMemcpyDeviceToDevice, s));
      hmg_vcycle(c, level, b, y);
      break;
    }
    default:
      return fail(PMG_ERR_ARG, "unknown op");
  }
  return finish_launches(c);
}

pmg_status pmg_export_csr(pmg_handle h, int which, int level, int* nr, int* nc, long long* nnz, int* rp, int* ci,
                          double* v) {
  if (!h || !nr || !nc || !nnz) return fail(PMG_ERR_ARG, "null argument");
  const auto& H = h->H;
  pmgl::Csr tmp;
  const pmgl::Csr* a = nullptr;
  if (which >= 0 && which <= 3) {
    if (level < 0 || level >= int(H.lev.size())) return fail(PMG_ERR_ARG, "level out of range");
    const auto& L = H.lev[size_t(level)];
    if (which == 0) a = &L.A;
    if (which == 1) a = &L.L;
    if (which == 3) a = &L.Praw;
    if (which == 2) {
      // U with its diagonal first in each row
      tmp.nr = tmp.nc = L.N;
      tmp.rp.assign(size_t(L.N) + 1, 0);
      for (int i = 0; i < L.N; ++i) {
        tmp.ci.push_back(i);
        tmp.v.push_back(L.udiag[size_t(i)]);
        for (int t = L.U.rp[i]; t < L.U.rp[i + 1]; ++t) { tmp.ci.push_back(L.U.ci[t]); tmp.v.push_back(L.U.v[t]); }
        tmp.rp[size_t(i) + 1] = int(tmp.ci.size());
      }
      a = &tmp;
    }
  } else if (which == 4) {
    if (level < 0 || level >= int(H.hl.size())) return fail(PMG_ERR_ARG, "level out of range");
    a = &H.hl[size_t(level)].A;
  } else {
    return fail(PMG_ERR_ARG, "unknown matrix");
  }
  *nr = a->nr;
  *nc = a->nc;
  *nnz = a->nnz();
  if (rp) {
    if (!ci || !v) return fail(PMG_ERR_ARG, "null output array");
    std::memcpy(rp, a->rp.data(), a->rp.size() * sizeof(int));
    std::memcpy(ci, a->ci.data(), a->ci.size() * sizeof(int));
    std::memcpy(v, a->v.data(), a->v.size() * sizeof(double));
  }
  return PMG_OK;
}

pmg_status pmg_export_lumped(pmg_handle h, int level, double* out) {
  if (!h || !out) return fail(PMG_ERR_ARG, "null argument");
  const auto& H = h->H;
  if (level >= 0 && level < int(H.lev.size())) {
    std::memcpy(out, H.lev[size_t(level)].ML.data(), H.lev[size_t(level)].ML.size() * sizeof(double));
    return PMG_OK;
  }
  if (level == int(H.lev.size())) {
    std::memcpy(out, H.ML1.data(), H.ML1.size() * sizeof(double));
    return PMG_OK;
  }
  return fail(PMG_ERR_ARG, "level out of range");
}

pmg_status pmg_l2_error(pmg_handle h, const double* u_host, double* err) {
  if (!h || !u_host || !err) return fail(PMG_ERR_ARG, "null argument");
  *err = pmgl::l2_error(h->H, u_host);
  return PMG_OK;
}

pmg_status pmg_ws_profile(pmg_ws ws, int enable) {
  if (!ws) return fail(PMG_ERR_ARG, "null workspace");
  ws->prof = enable != 0;
  return PMG_OK;
}

pmg_status pmg_ws_stats(pmg_ws ws, pmg_stats_t* out, int reset) {
  if (!ws || !out) return fail(PMG_ERR_ARG, "null argument");
  for (int k = 0; k < PMG_NKERN; ++k) {
    out->ms[k] = ws->prof_ms[k];
    out->launches[k] = ws->prof_n[k];
    out->bytes[k] = ws->prof_bytes[k];
  }
  out->total_launches = ws->launches;
  out->graph_launches = ws->graph_launches;
  if (reset) {
    for (int k = 0; k < PMG_NKERN; ++k) { ws->prof_ms[k] = 0; ws->prof_n[k] = 0; ws->prof_bytes[k] = 0; }
    ws->launches = 0;
    ws->graph_launches = 0;
  }
  return PMG_OK;
}

pmg_status pmg_ws_destroy(pmg_ws ws) {
  delete ws;
  return PMG_OK;
}

pmg_status pmg_destroy(pmg_handle h) {
  delete h;
  return PMG_OK;
}

const char* pmg_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free forward solve.
//
// Some callers cannot allocate device memory: code running inside a memory
// pool or arena that was sized up front, plug-ins whose host application owns
// every cudaMalloc, or code that must not allocate once a real-time loop has
// started.  pmg_lsolve_noalloc serves them: it runs the sync-free forward
// substitution kernel with its scratch (per-row ready flags, the row counter
// and the error word) in a fixed device array that belongs to this library
// and exists on every GPU that loads it, so the call itself allocates nothing.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocMaxRows = 1 << 20;     // largest system the fixed scratch serves
constexpr int kNoAllocHeader = 64;           // counter and error word, padded to 256 bytes

// [0]: row counter, [1]: error word, [64 .. 64 + n): ready flags.
static __device__ __align__(256) unsigned g_noalloc_scratch[kNoAllocHeader + kNoAllocMaxRows];

struct NoAllocDevice {
  bool ready = false;
  unsigned* scratch = nullptr;  // device address of g_noalloc_scratch on this device
  int sms = 0;
};
constexpr int kNoAllocMaxDevices = 64;
NoAllocDevice g_noalloc_devices[kNoAllocMaxDevices];
std::mutex g_noalloc_mutex;

// Resolves the device address of the scratch array for the current device
// (once per device, with that device current).
pmg_status noalloc_device(NoAllocDevice** out) {
  int dev = 0;
  PMG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(PMG_ERR_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  NoAllocDevice& d = g_noalloc_devices[dev];
  if (!d.ready) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(PMG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(PMG_ERR_CUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
    d.scratch = static_cast<unsigned*>(ptr);
    d.sms = sms;
    d.ready = true;
  }
  *out = &d;
  return PMG_OK;
}

}  // namespace

extern "C" pmg_status pmg_lsolve_noalloc(int n, const int* rp_dev, const int* ci_dev, const double* v_dev,
                                         const double* b_dev, double* y_dev, void* stream) {
  if (n < 0 || (n > 0 && (!rp_dev || !ci_dev || !v_dev || !b_dev || !y_dev)))
    return fail(PMG_ERR_ARG, "pmg_lsolve_noalloc: negative n or a null device pointer");
  if (n > kNoAllocMaxRows)
    return fail(PMG_ERR_ARG, "pmg_lsolve_noalloc: n = " + std::to_string(n) + " exceeds the fixed scratch limit of " +
                                 std::to_string(kNoAllocMaxRows) + " rows");
  if (n == 0) return PMG_OK;
  NoAllocDevice* d = nullptr;
  pmg_status st = noalloc_device(&d);
  if (st != PMG_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned* counter = d->scratch;
  unsigned* err = d->scratch + 1;
  unsigned* flags = d->scratch + kNoAllocHeader;
  // the previous call's counter, error word and flags are still in the array
  PMG_CUDA(cudaMemsetAsync(d->scratch, 0, (size_t(kNoAllocHeader) + size_t(n)) * sizeof(unsigned), s));
  pmgk::Csr L{n, rp_dev, ci_dev, v_dev};
  pmgk::k_lsolve<<<d->sms * 4, 256, 0, s>>>(L, b_dev, y_dev, flags, 1u, counter, err);
  PMG_CUDA(cudaGetLastError());
  unsigned herr = 0;
  PMG_CUDA(cudaMemcpyAsync(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  PMG_CUDA(cudaStreamSynchronize(s));
  if (herr) return fail(PMG_ERR_TIMEOUT, "a device-side dependency wait expired");
  return PMG_OK;
}
