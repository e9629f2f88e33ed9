// Context, setup, multigrid cycle (Algorithm 1), PCG (Sec. 4) and the C ABI of igamg.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <type_traits>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/igamg.h"
#include "host_math.h"
#include "kernels.cuh"
#include "tc_gemm.cuh"
#include "topology.h"

using namespace igamg;

namespace {

struct Fail {
  igamg_status code;
  std::string msg;
};

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      throw Fail{e_ == cudaErrorMemoryAllocation ? IGAMG_ERR_OOM : IGAMG_ERR_CUDA,       \
                 std::string(#call) + ": " + cudaGetErrorString(e_)};                   \
  } while (0)

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Device allocation registry of a context.
struct DevMem {
  std::vector<void*> ptrs;
  std::vector<size_t> sizes;  // bytes of each allocation
  template <class T>
  T* alloc(size_t count) {
    void* p = nullptr;
    if (count == 0) count = 1;
    CK(cudaMalloc(&p, count * sizeof(T)));
    ptrs.push_back(p);
    sizes.push_back(count * sizeof(T));
    return static_cast<T*>(p);
  }
  template <class T>
  T* upload(const std::vector<T>& h, cudaStream_t s) {
    T* d = alloc<T>(h.size());
    if (!h.empty()) CK(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return d;
  }
  void truncate(size_t mark) {  // frees the allocations made after `mark`
    for (size_t i = mark; i < ptrs.size(); ++i) cudaFree(ptrs[i]);
    ptrs.resize(mark);
    sizes.resize(mark);
  }
  size_t bytes() const {
    size_t b = 0;
    for (size_t x : sizes) b += x;
    return b;
  }
  void release() { truncate(0); }
};

struct Smoother1D {  // subspace-corrected mass smoother data of one direction signature
  int len = 0;
  std::vector<double> U;   // len x len, columns = M-orthonormal basis [U~, U^G]
  std::vector<double> mu;  // len
  double* dU = nullptr;
};

template <class T>
struct GemmSetT {
  GemmDescT<T>* d = nullptr;
  std::vector<GemmDescT<T>> h;  // host copy (FP64 sets are translated into lower precision)
  int batch = 0, maxM = 0, maxN = 0;
  int R = 0;                    // FMA tile factor (0: size heuristic; the autotuner may set it)
  double flops = 0, bytes = 0;  // algorithmic work of one launch
};
using GemmSet = GemmSetT<double>;

template <class T>
struct ModeSetT {  // one mode-product stage of the 3D interiors (all interiors of a level)
  ModeDescT<T>* d = nullptr;
  std::vector<ModeDescT<T>> h;
  int batch = 0, max_n = 0;
  int64_t max_fibres = 0;
};

template <class T>
struct TcSet {
  TcDesc<T, T>* d = nullptr;
  std::vector<TcDesc<T, T>> h;
  int batch = 0, maxM = 0, maxN = 0;
  double flops = 0;       // algorithmic (the GEMMs' own)
  double exec_flops = 0;  // BF16 MMA work issued
  double dig_bytes = 0;   // digit pass: B read, digit planes and exponents written
  // digit scratch of the set: sizes and per-descriptor offsets; the descriptors are uploaded
  // once the context's scratch is bound (bind_tc)
  int64_t dig_elems = 0, tau_elems = 0, tiles = 0, panels = 0;
  int *tstart_d = nullptr, *pstart_d = nullptr;  // tile and panel prefixes (device)
  std::vector<int64_t> dig_off, tau_off;
  bool side = false;      // launched on the interface stream (its own scratch)
};

// Numeric data of one level in one precision: the vectors and the descriptor sets the
// cycle launches.  FP64 data are built by the setup; lower-precision data are twins of them.
// Fibre-major stacked tensor-core stage of the 2D interiors (FP64): one descriptor per group
// of patches sharing the stage's basis and sizes, their fibres stacked along the MMA's M side.
struct StackSet {
  std::vector<TcStack<double, double>> h;
  std::vector<std::vector<const double*>> hX, hE;  // host copies of each descriptor's tables
  std::vector<std::vector<double*>> hC;
  TcStack<double, double>* d = nullptr;  // uploaded by bind_stack
  int batch = 0;
  int64_t tiles = 0, panels = 0, dig_elems = 0, tau_elems = 0;
  std::vector<int64_t> dig_off, tau_off;
  int *tstart_d = nullptr, *pstart_d = nullptr;
  double flops = 0, exec_flops = 0, dig_bytes = 0;
};

template <class T>
struct Num {
  const void* band = nullptr;  // band coefficients of the cycle: T, or __nv_bfloat16 when bf16
  bool bf16 = false;
  const T* band_op = nullptr;  // band coefficients of the Krylov operator (always type T)
  PatchDev* pd_pair = nullptr; // 3D BF16 cycle bands in the paired layout: patch offsets into it
  PatchDev* pd_blk = nullptr;  // 3D FP32 bands in the tap-blocked layout: patch offsets into it
  KronDevT<T>* kd = nullptr;   // rectangle patches: Kronecker-sum operator per patch
  T *F = nullptr, *U = nullptr, *R = nullptr;
  GemmSetT<T> st0F, st0R, st1, st2, st3;            // 2D interiors
  TcSet<T> tc0F, tc0R, tc1, tc2, tc3;               // interiors on the tensor cores (2D: 4
  TcSet<T> tc4, tc5;                                // stages; 3D: tc0F, tc1..tc5 = 6 stages)
  TcSet<T> tq0, tq1, tq2, tq3;                      // 3D faces on the tensor cores
  StackSet sk0F, sk0R, sk1, sk2, sk3;               // 2D interiors, stacked (FP64 engine)
  ModeSetT<T> fm[4];                                // 3D faces as mode products (FMA engine)
  FdSmallT<T>* fsmall = nullptr;                    // small 2D interiors, one block each
  SmoothSmallT<T> ssmall{};                         // + edges and vertices in the same launch
  FdRowsT<T>* frows = nullptr;                      // 2D interiors by row blocks (two launches)
  int nfrows = 0, frows_n0 = 0, frows_n1 = 0;
  bool use_rows = false;
  double ssmall_flops = 0;
  int nfsmall = 0;
  bool use_fused = false;
  double fsmall_flops = 0;
  bool use_tc = false;
  GemmSetT<T> m0f, m1f, m2f, m0b, m1b, m2b;         // 3D interiors
  ModeSetT<T> md[6];                                // the same six products as mode products
  Fd3SmallT<T>* fd3 = nullptr;                      // small 3D interiors: the six in one launch
  int nfd3 = 0;
  Iface3SmallT<T> i3s{};                            // small 3D interface pieces: one launch
  bool i3_ok = false;
  T* cX = nullptr;                                  // compact 3D interior tensor
  T *G = nullptr, *Z = nullptr, *vscale = nullptr;  // interface nodes
  GemmSetT<T> edgeA, edgeB, face0, face1, face2, face3;
  XferT<T>* rpass[3] = {nullptr, nullptr, nullptr};
  Xfer2T<T>* r2 = nullptr;
  Xfer2T<T>* p2 = nullptr;
  XferT<T>* ppass[3] = {nullptr, nullptr, nullptr};
  T *tA = nullptr, *tB = nullptr;
};

struct Level {
  LevelTopo topo;
  std::vector<PatchDev> pd_h;
  PatchDev* pd = nullptr;
  int max_n[3] = {1, 1, 1}, max_p = 1;
  int uniform_p = 0;  // the degree shared by every patch and direction, else 0
  int64_t* l2g = nullptr;
  int64_t *g2t_ptr = nullptr, *g2t = nullptr;
  double* band = nullptr;  // FP64 band coefficients (none when kron)
  bool kron = false;       // every patch a rectangle: A applied as a Kronecker sum of 1D K, M
  unsigned char* active = nullptr;  // kron: 1 for non-eliminated tile nodes
  std::vector<KronDevT<double>> kd_h;
  int64_t band_doubles = 0;  // size of a band array in this layout (mass bands of the rhs)
  bool tc_ok = false;        // tensor-core FD stage sets built (the FD engine may switch)
  bool fused_ok = false;     // every 2D interior fits the one-block FD kernel
  bool small_ok = false;     // ... and every edge too: the whole smoother is one launch
  std::vector<FdRowsT<double>> fr_h;
  std::vector<EdgeSmallT<double>> es_h;
  std::vector<FaceSmallT<double>> f3s_h;       // 3D small interface pieces, host copies
  std::vector<EdgeSmallT<double>> e3s_h;
  int64_t v3_beg = 0, v3_end = 0;
  std::vector<FdSmallT<double>> fs_h;
  Num<double> n64;
  Num<float> n32;
  // 3D interior boxes (shared by all precisions)
  BoxDev* boxes = nullptr;
  int nbox = 0;
  int64_t max_box = 0;
  // interface nodes (shared)
  int64_t n_if = 0;
  int64_t *if_ptr = nullptr, *if_idx = nullptr;
  // transfer from level l-1 (valid for level >= 1): host descriptors per pass
  std::vector<XferT<double>> rp_h[3], pp_h[3];
  std::vector<Xfer2T<double>> r2_h, p2_h;  // 2D: both passes fused (when the tables allow)
  std::vector<Fd3SmallT<double>> fd3_h;      // 3D small interiors (kFd3SmallN), host copy
  int64_t box_vol = 0;                        // 3D interior nodes of the level
  int x2_rout0 = 0, x2_rout1 = 0, x2_pout0 = 0, x2_pout1 = 0, x2_rw1 = 0, x2_pw1 = 0;
  int64_t rmax[3] = {0, 0, 0}, pmax[3] = {0, 0, 0};
  double apply_flops = 0, band_bytes = 0, xfer_flops = 0, xfer_bytes = 0;
};

template <class T> Num<T>& num(Level& L);
template <> Num<double>& num<double>(Level& L) { return L.n64; }
template <> Num<float>& num<float>(Level& L) { return L.n32; }

}  // namespace

namespace igamg {
struct Lockstep;
void lockstep_free(Lockstep* k);
// One more set of a context's work arrays, for solving several right-hand sides of one
// problem together: every array the cycle and the PCG write (the registered work arrays, the
// Krylov vectors, the tensor-core digit scratch) once more; the constant arrays are shared.
struct WorkCopy {
  std::vector<std::tuple<const double*, int64_t, double*>> tw;  // (context's array, count, this copy's), by base
  double *X = nullptr, *Pv = nullptr, *W = nullptr, *Bt = nullptr, *Rr = nullptr;
  __nv_bfloat16* dig[2] = {nullptr, nullptr};
  int* tau[2] = {nullptr, nullptr};
  __nv_bfloat16* sdig = nullptr;  // stacked stages' digit scratch
  int* stau = nullptr;
};
}  // namespace igamg

struct igamg_ctx {
  cudaStream_t stream = nullptr;
  igamg_options opt{};
  ProblemDesc pd;
  std::vector<Level> lv;
  DevMem mem;
  double* A0inv = nullptr;
  int64_t N0 = 0;
  double *X = nullptr, *Pv = nullptr, *W = nullptr, *Bt = nullptr, *gtmp = nullptr;
  float *X32 = nullptr, *P32 = nullptr, *W32 = nullptr, *Zold32 = nullptr;  // inner (low-precision) PCG vectors
  double* Rr = nullptr;                                    // FP64 residual of the refinement
  bool low = false;                                        // low-precision numerics built
  bool low_bf16 = false;                                   // bands stored in BF16
  bool verbose = false;                                    // IGAMG_VERBOSE set: log refinement steps
  // FP64 device arrays referenced by the cycle: (base, count, constant?) for the twins
  std::vector<std::tuple<double*, int64_t, bool>> reg;
  std::vector<int64_t> band_count;                         // band doubles per level
  std::map<std::tuple<int, int>, std::pair<double*, double*>> kron_1d;  // (m, p) -> banded K, M
  int* tc_err = nullptr;                                   // device flag: tensor-core wait timed out
  // PCG iteration body replayed as a CUDA graph (index 0 FP64, 1 FP32 inner), captured on a
  // private stream (the legacy stream cannot capture) and launched on `stream`
  // slot 2 * index + (1 while profiling): the plain graph and the one with timing nodes
  // are kept side by side, so switching the profiler between solves costs no capture
  // (index 2 FP64 and 3 low-precision cycle alone, for igamg_cycle_time)
  static constexpr int kGraphSlots = 8;
  cudaGraphExec_t iter_graph[kGraphSlots] = {};
  unsigned graph_key[kGraphSlots] = {};                   // profiling mode it was captured in
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> graph_ev[kGraphSlots];  // timing nodes inside it
  int64_t graph_launch[kGraphSlots][8] = {};              // per-replay launch accounting
  double graph_flops[kGraphSlots][8] = {}, graph_bytes[kGraphSlots][8] = {};
  cudaStream_t cap_stream = nullptr;
  // the interface pieces of a smoothing step run on a second stream, concurrently with the
  // patch interiors (disjoint pieces, Eq. additive); forked and joined by events
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  int capturing = -1, pending_graph = -1;
  std::map<const void*, const void*> tc_bf16_twin;         // S=7 slices -> S=1 slices of the same matrix
  double *partials = nullptr, *scal = nullptr;
  double* h_scal = nullptr;  // pinned
  std::string err;
  double t_setup_ms = 0, t_assemble_ms = 0;
  // per-class launch accounting (igamg_profile_*)
  bool prof = false;
  unsigned prof_mask = 0;  // classes whose launches get timing events
  int64_t prof_launch[8] = {0};
  double prof_ms[8] = {0}, prof_flops[8] = {0}, prof_bytes[8] = {0};
  std::vector<cudaEvent_t> ev_free;
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> ev_open;
  int cur_cls = -1;
  cudaEvent_t cur_start = nullptr;
  // several right-hand sides solved together (igamg_solve_multi): the FP64 digit scratch
  // sizes, the work-array copies 1.., and the lockstep engines by number of right-hand sides
  int64_t dig64[2] = {0, 0}, tau64[2] = {0, 0};
  int64_t sdig = 0, stau = 0;  // digit scratch of the stacked 2D stages
  std::deque<igamg::WorkCopy> copies;  // stable addresses: the engines point into it
  std::map<int, igamg::Lockstep*> multi;
};

static thread_local std::string g_setup_error = "no error";

namespace igamg {
// A 2D patch whose bilinear map is affine with orthogonal Jacobian columns (a rectangle,
// any orientation) has the constant metric C = |det J| J^{-1} J^{-T} = diag(c0, c1) with
// c_j = |det J| / |J e_j|^2 (Sec. 2: the patch stiffness integrand grad^T C grad).
bool rect_metric(const double* X, double* c0, double* c1) {
  double a[2] = {X[2] - X[0], X[3] - X[1]}, b[2] = {X[4] - X[0], X[5] - X[1]};
  double la = std::hypot(a[0], a[1]), lb = std::hypot(b[0], b[1]);
  double gap = std::hypot(X[6] - X[0] - a[0] - b[0], X[7] - X[1] - a[1] - b[1]);
  if (!(la > 0 && lb > 0) || gap > 1e-14 * (la + lb) || std::fabs(a[0] * b[0] + a[1] * b[1]) > 1e-14 * la * lb)
    return false;
  double det = std::fabs(a[0] * b[1] - a[1] * b[0]);
  *c0 = det / (la * la);
  *c1 = det / (lb * lb);
  return true;
}

// Message returned by igamg_last_error(NULL) on this thread.
void set_context_free_error(const std::string& msg) { g_setup_error = msg; }
// Stream a context launches on (the batch layer lends contexts to its worker streams).
cudaStream_t ctx_stream(const igamg_ctx* c) { return c->stream; }
void ctx_set_stream(igamg_ctx* c, cudaStream_t s) { c->stream = s; }
// Device memory the context holds (its own allocations).
size_t ctx_device_bytes(const igamg_ctx* c) { return c->mem.bytes(); }
// Scheduling weight of one solve: finest-level tile nodes times (degree + 2).
double ctx_work_estimate(const igamg_ctx* c) {
  const LevelTopo& T = c->lv.back().topo;
  return double(T.T) * (c->pd.p[0] + 2);
}
}  // namespace igamg

namespace {

double* reg_const(igamg_ctx* c, double* p, size_t n) {
  c->reg.emplace_back(p, int64_t(n), true);
  return p;
}
double* reg_work(igamg_ctx* c, double* p, int64_t n) {
  c->reg.emplace_back(p, n, false);
  return p;
}

enum { CLS_APPLY = 0, CLS_FD = 1, CLS_IFACE = 2, CLS_TRANSFER = 3, CLS_COARSE = 4, CLS_VECTOR = 5, CLS_TENSOR_EXEC = 6,
       CLS_TC_KERNEL = 7 };

cudaEvent_t prof_event(igamg_ctx* c) {
  if (!c->ev_free.empty()) {
    cudaEvent_t e = c->ev_free.back();
    c->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e;
  CK(cudaEventCreate(&e));
  return e;
}

// Brackets one launch of class `cls` (and of the sub-account `sub`, e.g. the tensor-core
// kernel inside the FD classes, or -1) with algorithmic work (flops, bytes).  The event pair
// is recorded when either class is timed; its time goes to the classes that are.
struct ProfScope {
  igamg_ctx* c;
  int code = 0xFF;  // timed main class (low 4 bits) and sub-account (high 4 bits); 15 = none
  cudaEvent_t a = nullptr;
  ProfScope(igamg_ctx* c_, int cls, double flops, double bytes, int launches = 1, int sub = -1) : c(c_) {
    if (!c->prof) return;
    c->prof_launch[cls] += launches;
    c->prof_flops[cls] += flops;
    c->prof_bytes[cls] += bytes;
    if (sub >= 0) {
      c->prof_launch[sub] += launches;
      c->prof_flops[sub] += flops;
      c->prof_bytes[sub] += bytes;
    }
    const bool tm = (c->prof_mask >> cls) & 1u, ts = sub >= 0 && ((c->prof_mask >> sub) & 1u);
    if (!tm && !ts) return;
    code = (tm ? cls : 15) | ((ts ? sub : 15) << 4);
    a = prof_event(c);
    record(a);
  }
  void record(cudaEvent_t e) {
    // inside a graph capture the event becomes a record node that fires on every replay
    if (c->capturing >= 0) CK(cudaEventRecordWithFlags(e, c->stream, cudaEventRecordExternal));
    else CK(cudaEventRecord(e, c->stream));
  }
  ~ProfScope() noexcept(false) {
    if (!a) return;
    cudaEvent_t b = prof_event(c);
    record(b);
    if (c->capturing >= 0) c->graph_ev[c->capturing].emplace_back(code, a, b);
    else c->ev_open.emplace_back(code, a, b);
  }
};

void prof_add_ms(igamg_ctx* c, int code, float ms) {
  if ((code & 15) != 15) c->prof_ms[code & 15] += ms;
  if ((code >> 4) != 15) c->prof_ms[code >> 4] += ms;
}

// Folds completed event pairs into the per-class totals (stream must be synchronised).
void prof_collect(igamg_ctx* c) {
  for (auto& t : c->ev_open) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, std::get<1>(t), std::get<2>(t)));
    prof_add_ms(c, std::get<0>(t), ms);
    c->ev_free.push_back(std::get<1>(t));
    c->ev_free.push_back(std::get<2>(t));
  }
  c->ev_open.clear();
  if (c->pending_graph >= 0) {  // timing nodes of the last graph replay
    for (auto& t : c->graph_ev[c->pending_graph]) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, std::get<1>(t), std::get<2>(t)));
      prof_add_ms(c, std::get<0>(t), ms);
    }
    c->pending_graph = -1;
  }
}

void drop_graph(igamg_ctx* c, int gi) {
  if (c->iter_graph[gi]) CK(cudaGraphExecDestroy(c->iter_graph[gi]));
  c->iter_graph[gi] = nullptr;
  for (auto& t : c->graph_ev[gi]) {
    c->ev_free.push_back(std::get<1>(t));
    c->ev_free.push_back(std::get<2>(t));
  }
  c->graph_ev[gi].clear();
}

// Runs `body` as the replay of a graph captured from it on the first call (and again when
// the profiling mode changed).  The body must launch onto c->stream only and touch the same
// buffers with the same host arguments every time.
template <class F>
void graph_run(igamg_ctx* c, int index, F&& body) {
  const unsigned key = c->prof ? (0x100u | c->prof_mask) : 0u;
  const int gi = 2 * index + (c->prof ? 1 : 0);
  if (c->iter_graph[gi] && c->graph_key[gi] != key) drop_graph(c, gi);
  if (!c->iter_graph[gi]) {
    if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    int64_t l0[8];
    double f0[8], b0[8];
    std::copy(c->prof_launch, c->prof_launch + 8, l0);
    std::copy(c->prof_flops, c->prof_flops + 8, f0);
    std::copy(c->prof_bytes, c->prof_bytes + 8, b0);
    cudaStream_t user = c->stream;
    c->stream = c->cap_stream;
    c->capturing = gi;
    cudaGraph_t g = nullptr;
    try {
      CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
      body();
      CK(cudaStreamEndCapture(c->stream, &g));
    } catch (...) {
      cudaGraph_t dead = nullptr;
      cudaStreamEndCapture(c->stream, &dead);
      if (dead) cudaGraphDestroy(dead);
      c->stream = user;
      c->capturing = -1;
      throw;
    }
    c->stream = user;
    c->capturing = -1;
    CK(cudaGraphInstantiate(&c->iter_graph[gi], g, 0));
    CK(cudaGraphDestroy(g));
    c->graph_key[gi] = key;
    for (int k = 0; k < 8; ++k) {  // the capture launched nothing: count per replay instead
      c->graph_launch[gi][k] = c->prof_launch[k] - l0[k];
      c->graph_flops[gi][k] = c->prof_flops[k] - f0[k];
      c->graph_bytes[gi][k] = c->prof_bytes[k] - b0[k];
    }
    std::copy(l0, l0 + 8, c->prof_launch);
    std::copy(f0, f0 + 8, c->prof_flops);
    std::copy(b0, b0 + 8, c->prof_bytes);
  }
  CK(cudaGraphLaunch(c->iter_graph[gi], c->stream));
  if (c->prof) {
    for (int k = 0; k < 8; ++k) {
      c->prof_launch[k] += c->graph_launch[gi][k];
      c->prof_flops[k] += c->graph_flops[gi][k];
      c->prof_bytes[k] += c->graph_bytes[gi][k];
    }
    c->pending_graph = gi;
  }
}

template <class T>
double gemm_flops(const std::vector<GemmDescT<T>>& v) {
  double f = 0;
  for (auto& d : v) f += 2.0 * d.M * double(d.N) * d.K;
  return f;
}

template <class T>
void set_gemm(igamg_ctx* c, GemmSetT<T>& gs, const std::vector<GemmDescT<T>>& v) {
  gs.h = v;
  gs.batch = int(v.size());
  gs.maxM = gs.maxN = 0;
  for (auto& d : v) {
    gs.maxM = std::max(gs.maxM, d.M);
    gs.maxN = std::max(gs.maxN, d.N);
  }
  gs.d = v.empty() ? nullptr : c->mem.upload(v, c->stream);
  gs.flops = gemm_flops(v);
  gs.bytes = 0;
  for (auto& d : v) gs.bytes += 8.0 * (double(d.M) * d.K + double(d.K) * d.N + 2.0 * d.M * d.N);
}

template <class T>
void set_mode(igamg_ctx* c, ModeSetT<T>& ms, const std::vector<ModeDescT<T>>& v) {
  ms.h = v;
  ms.batch = int(v.size());
  ms.max_fibres = 0;
  ms.max_n = 0;
  for (auto& d : v) ms.max_fibres = std::max(ms.max_fibres, d.fibres), ms.max_n = std::max(ms.max_n, d.n);
  ms.d = v.empty() ? nullptr : c->mem.upload(v, c->stream);
}

// One mode-product stage with the work accounting of the GEMM stage it replaces.
template <class T>
void run_mode(igamg_ctx* c, const ModeSetT<T>& ms, const GemmSetT<T>& gs, int epi, int cls = CLS_FD) {
  ProfScope ps(c, cls, gs.flops, gs.bytes * sizeof(T) / 8.0);
  CK(launch_mode_product<T>(c->stream, ms.d, ms.batch, ms.max_fibres, ms.max_n, epi));
}

template <class T>
void run_gemm(igamg_ctx* c, const GemmSetT<T>& gs, bool ta, bool tb, int epi, double alpha, int cls) {
  if (!gs.batch) return;
  ProfScope ps(c, cls, gs.flops, gs.bytes * sizeof(T) / 8.0);
  CK(launch_gemm<T>(c->stream, gs.d, gs.batch, gs.maxM, gs.maxN, ta, tb, epi, T(alpha), gs.R));
}

template <class T>
void set_tc(igamg_ctx*, TcSet<T>& ts, const std::vector<TcDesc<T, T>>& v, bool side = false) {
  constexpr int S = sizeof(T) == 8 ? 7 : 1;
  ts.h = v;
  ts.batch = int(v.size());
  ts.maxM = ts.maxN = 0;
  ts.flops = ts.exec_flops = ts.dig_bytes = 0;
  ts.dig_elems = ts.tau_elems = ts.tiles = 0;
  ts.dig_off.clear();
  ts.tau_off.clear();
  ts.side = side;
  for (auto& d : v) {
    ts.maxM = std::max(ts.maxM, d.M);
    ts.maxN = std::max(ts.maxN, d.N);
    ts.flops += 2.0 * d.M * double(d.N) * d.K;
    ts.exec_flops += tc_exec_flops(d.M, d.N, d.K, S);
    ts.dig_off.push_back(ts.dig_elems);
    ts.tau_off.push_back(ts.tau_elems);
    ts.dig_elems += tc_dig_elems(d.N, d.K, S);
    ts.tau_elems += tc_tau_elems(d.N, S);
    ts.dig_bytes += double(d.N) * d.K * (sizeof(T) + 2.0 * S) + 4.0 * tc_tau_elems(d.N, S);
  }
  ts.d = nullptr;  // uploaded by bind_tc
}

void set_stack(StackSet& ss, const std::vector<TcStack<double, double>>& v) {
  ss.h = v;
  ss.batch = int(v.size());
  ss.flops = ss.exec_flops = ss.dig_bytes = 0;
  ss.dig_elems = ss.tau_elems = 0;
  ss.dig_off.clear();
  ss.tau_off.clear();
  for (auto& d : v) {
    const double M = double(d.P) * d.F;
    ss.flops += 2.0 * M * d.N * d.K;
    ss.exec_flops += tc_stack_exec_flops(d.P, d.F, d.N, d.K);
    ss.dig_off.push_back(ss.dig_elems);
    ss.tau_off.push_back(ss.tau_elems);
    ss.dig_elems += tc_stack_dig_elems(d.P, d.F, d.K);
    ss.tau_elems += int64_t(d.P) * d.F;
    ss.dig_bytes += M * d.K * (8.0 + 2.0 * 7) + 4.0 * M;
  }
  ss.d = nullptr;  // uploaded by bind_stack
}

// Every tensor-core set of precision T gets the digit scratch of its stream: the sets
// launched on the solve's stream run one after another and share one buffer, the interface
// (face) sets on the side stream share another.  Then the descriptors are uploaded.
template <class T>
void bind_tc(igamg_ctx* c) {
  std::vector<TcSet<T>*> sets;
  for (Level& L : c->lv) {
    Num<T>& N = num<T>(L);
    for (TcSet<T>* p : {&N.tc0F, &N.tc0R, &N.tc1, &N.tc2, &N.tc3, &N.tc4, &N.tc5, &N.tq0, &N.tq1, &N.tq2, &N.tq3})
      if (p->batch && !p->d) sets.push_back(p);
  }
  int64_t dig[2] = {0, 0}, tau[2] = {0, 0};
  for (TcSet<T>* p : sets) {
    dig[p->side] = std::max(dig[p->side], p->dig_elems);
    tau[p->side] = std::max(tau[p->side], p->tau_elems);
  }
  __nv_bfloat16* dbase[2] = {nullptr, nullptr};
  int* tbase[2] = {nullptr, nullptr};
  for (int k = 0; k < 2; ++k) {
    if (dig[k]) dbase[k] = c->mem.alloc<__nv_bfloat16>(size_t(dig[k]));
    if (tau[k]) tbase[k] = c->mem.alloc<int>(size_t(tau[k]));
    if (sizeof(T) == 8) c->dig64[k] = dig[k], c->tau64[k] = tau[k];
  }
  for (TcSet<T>* p : sets) {
    for (int i = 0; i < p->batch; ++i) {
      p->h[i].Bdig = dbase[p->side] + p->dig_off[i];
      p->h[i].Btau = tbase[p->side] ? tbase[p->side] + p->tau_off[i] : nullptr;
    }
    p->d = c->mem.upload(p->h, c->stream);
    std::vector<int> ts, ps;
    tc_prefixes(p->h, sizeof(T) == 8 ? 7 : 1, ts, ps);
    p->tiles = ts.back();
    p->panels = ps.back();
    p->tstart_d = c->mem.upload(ts, c->stream);
    p->pstart_d = c->mem.upload(ps, c->stream);
  }
}

// The stacked sets of every level share one digit scratch (they run one after another on
// the solve's stream).
void bind_stack(igamg_ctx* c) {
  std::vector<StackSet*> sets;
  for (Level& L : c->lv)
    for (StackSet* p : {&L.n64.sk0F, &L.n64.sk0R, &L.n64.sk1, &L.n64.sk2, &L.n64.sk3})
      if (p->batch && !p->d) sets.push_back(p);
  int64_t dig = 0, tau = 0;
  for (StackSet* p : sets) {
    dig = std::max(dig, p->dig_elems);
    tau = std::max(tau, p->tau_elems);
  }
  if (sets.empty()) return;
  c->sdig = dig;
  c->stau = tau;
  __nv_bfloat16* dbase = c->mem.alloc<__nv_bfloat16>(size_t(std::max<int64_t>(dig, 1)));
  int* tbase = c->mem.alloc<int>(size_t(std::max<int64_t>(tau, 1)));
  for (StackSet* p : sets) {
    for (int i = 0; i < p->batch; ++i) {
      p->h[i].Xdig = dbase + p->dig_off[i];
      p->h[i].Xtau = tbase + p->tau_off[i];
    }
    p->d = c->mem.upload(p->h, c->stream);
    std::vector<int> ts, ps;
    tc_stack_prefixes(p->h, ts, ps);
    p->tiles = ts.back();
    p->panels = ps.back();
    p->tstart_d = c->mem.upload(ts, c->stream);
    p->pstart_d = c->mem.upload(ps, c->stream);
  }
}

void run_stack(igamg_ctx* c, const StackSet& ss, int epi, double alpha, int cls = CLS_FD) {
  if (!ss.batch) return;
  if (!ss.d) throw Fail{IGAMG_ERR_NUMERIC, "stacked tensor-core set without scratch"};
  {
    ProfScope ps(c, cls, 0.0, ss.dig_bytes);
    CK(launch_tc_digits_stack(c->stream, ss.d, ss.batch, ss.pstart_d, ss.panels));
  }
  if (c->prof) c->prof_flops[CLS_TENSOR_EXEC] += ss.exec_flops;
  ProfScope ps(c, cls, ss.flops, 0.0, 1, CLS_TC_KERNEL);
  CK(launch_gemm_tc_stack(c->stream, ss.d, ss.batch, ss.tstart_d, ss.tiles, epi, alpha, c->tc_err));
}

template <class T>
void run_tc(igamg_ctx* c, const TcSet<T>& ts, int epi, double alpha, int cls = CLS_FD) {
  if (!ts.batch) return;
  if (!ts.d) throw Fail{IGAMG_ERR_NUMERIC, "tensor-core set without scratch"};
  {
    ProfScope ps(c, cls, 0.0, ts.dig_bytes);
    if constexpr (std::is_same<T, double>::value)
      CK((launch_tc_digits<7, double, double>(c->stream, ts.d, ts.batch, ts.pstart_d, ts.panels)));
    else
      CK((launch_tc_digits<1, float, float>(c->stream, ts.d, ts.batch, ts.pstart_d, ts.panels)));
  }
  if (c->prof) c->prof_flops[CLS_TENSOR_EXEC] += ts.exec_flops;
  ProfScope ps(c, cls, ts.flops, 0.0, 1, CLS_TC_KERNEL);
  if constexpr (std::is_same<T, double>::value)
    CK((launch_gemm_tc<7, double, double>(c->stream, ts.d, ts.batch, ts.tstart_d, ts.tiles, epi, alpha, c->tc_err)));
  else
    CK((launch_gemm_tc<1, float, float>(c->stream, ts.d, ts.batch, ts.tstart_d, ts.tiles, epi, float(alpha),
                                        c->tc_err)));
}

// ---------------------------------------------------------------- setup helpers

// Subspace-corrected mass smoother on one direction (Sec. 3 names it for the patch
// interiors; this library reads it as follows): S~ = splines of the index set with odd
// derivatives < p vanishing at kept (Neumann) ends and even derivatives 2..<p vanishing at
// dropped (interface / Dirichlet) ends; S^G its M-orthogonal complement; the FD basis is an
// M-orthonormal basis of S~ followed by the (K, M) eigenvectors on S^G, with
// mu = sigma on S~ and lambda + sigma on S^G.
Smoother1D build_scms(int m, int p, bool drop_lo, bool drop_hi, double sigma) {
  Mat M, K;
  mass_stiffness_1d(m, p, M, K);
  int n = m + p;
  std::vector<int> I;
  for (int i = drop_lo ? 1 : 0; i < (drop_hi ? n - 1 : n); ++i) I.push_back(i);
  int len = int(I.size());
  Mat MI = submatrix(M, n, I), KI = submatrix(K, n, I);
  // constraint rows (normalised)
  std::vector<double> t = uniform_knots(m, p);
  std::vector<std::vector<double>> rows;
  std::vector<double> der((p + 1) * (p + 1));
  for (int end = 0; end < 2; ++end) {
    bool dropped = end == 0 ? drop_lo : drop_hi;
    double x = end == 0 ? 0.0 : 1.0;
    int span = find_span(t, p, x);
    nonzero_basis(t, p, span, x, p, der.data());
    for (int r = dropped ? 2 : 1; r < p; r += 2) {
      std::vector<double> row(len, 0.0);
      double mx = 0.0;
      for (int j = 0; j <= p; ++j) {
        int gi = span - p + j;
        auto it = std::find(I.begin(), I.end(), gi);
        if (it != I.end()) {
          row[it - I.begin()] = der[r * (p + 1) + j];
          mx = std::max(mx, std::fabs(der[r * (p + 1) + j]));
        }
      }
      if (mx > 0) {
        for (double& v : row) v /= mx;
        rows.push_back(row);
      }
    }
  }
  // orthonormal basis of range(C^T) by Gram-Schmidt (twice), completed to R^len
  std::vector<std::vector<double>> Q;
  auto orth_add = [&](std::vector<double> v, double tol) {
    double n0 = 0;
    for (double a : v) n0 += a * a;
    n0 = std::sqrt(n0);
    for (int pass = 0; pass < 2; ++pass)
      for (auto& q : Q) {
        double d = 0;
        for (int i = 0; i < len; ++i) d += q[i] * v[i];
        for (int i = 0; i < len; ++i) v[i] -= d * q[i];
      }
    double nn = 0;
    for (double a : v) nn += a * a;
    nn = std::sqrt(nn);
    if (nn <= tol * n0 || nn == 0.0) return false;
    for (double& a : v) a /= nn;
    Q.push_back(v);
    return true;
  };
  for (auto& r : rows) orth_add(r, 1e-10);
  int rank = int(Q.size());
  for (int i = 0; i < len && int(Q.size()) < len; ++i) {
    std::vector<double> e(len, 0.0);
    e[i] = 1.0;
    orth_add(e, 1e-6);
  }
  int nt = len - rank;  // dim S~
  Smoother1D out;
  out.len = len;
  out.U.assign(size_t(len) * len, 0.0);
  out.mu.assign(len, sigma);
  // S~ block: Z = Q[rank..], U~ = Z L^{-T} with Z^T M Z = L L^T
  if (nt > 0) {
    Mat Zm(size_t(len) * nt);
    for (int a = 0; a < nt; ++a)
      for (int i = 0; i < len; ++i) Zm[size_t(i) * nt + a] = Q[rank + a][i];
    Mat MZ = matmul(MI, Zm, len, len, nt);
    Mat G = matmul(Zm, MZ, nt, len, nt, true, false);
    if (!cholesky(nt, G)) throw Fail{IGAMG_ERR_NUMERIC, "SCMS Cholesky failed"};
    // U~ = Z L^{-T}: solve L^T rows... column a of U~ = Z * (L^{-T})[:, a]
    Mat Linv_T(size_t(nt) * nt, 0.0);  // L^{-T}
    for (int a = 0; a < nt; ++a) {
      std::vector<double> e(nt, 0.0);
      e[a] = 1.0;
      // solve L^T y = e
      for (int i = nt - 1; i >= 0; --i) {
        double v = e[i];
        for (int k = i + 1; k < nt; ++k) v -= G[size_t(k) * nt + i] * e[k];
        e[i] = v / G[size_t(i) * nt + i];
      }
      for (int i = 0; i < nt; ++i) Linv_T[size_t(i) * nt + a] = e[i];
    }
    Mat Ut = matmul(Zm, Linv_T, len, nt, nt);
    for (int i = 0; i < len; ++i)
      for (int a = 0; a < nt; ++a) out.U[size_t(i) * len + a] = Ut[size_t(i) * nt + a];
  }
  if (rank > 0) {
    // W = M^{-1} Qc (range(C^T) basis), eigen of (W^T K W, W^T M W)
    Mat Lm = MI;
    if (!cholesky(len, Lm)) throw Fail{IGAMG_ERR_NUMERIC, "mass Cholesky failed"};
    Mat Wm(size_t(len) * rank);
    for (int a = 0; a < rank; ++a)
      for (int i = 0; i < len; ++i) Wm[size_t(i) * rank + a] = Q[a][i];
    cholesky_solve_many(len, Lm, Wm, rank);
    Mat KW = matmul(KI, Wm, len, len, rank), MW = matmul(MI, Wm, len, len, rank);
    Mat Kr = matmul(Wm, KW, rank, len, rank, true, false), Mr = matmul(Wm, MW, rank, len, rank, true, false);
    std::vector<double> lam;
    Mat Y;
    if (!generalized_eigen(rank, Kr, Mr, lam, Y)) throw Fail{IGAMG_ERR_NUMERIC, "SCMS eigen failed"};
    Mat UG = matmul(Wm, Y, len, rank, rank);
    for (int i = 0; i < len; ++i)
      for (int a = 0; a < rank; ++a) out.U[size_t(i) * len + nt + a] = UG[size_t(i) * rank + a];
    for (int a = 0; a < rank; ++a) out.mu[nt + a] = lam[a] + sigma;
  }
  return out;
}

struct Tables1D {  // Gauss points and basis tables of one (m, p) spline space
  std::vector<double> xq, wq, B, dB;
};

Tables1D tables_1d(int m, int p) {
  Tables1D t;
  int nq = p + 1;
  std::vector<double> xg(nq), wg(nq), kn = uniform_knots(m, p), d(2 * (p + 1));
  gauss_legendre(nq, xg.data(), wg.data());
  t.xq.resize(size_t(m) * nq);
  t.wq.resize(size_t(m) * nq);
  t.B.resize(size_t(m) * nq * (p + 1));
  t.dB.resize(size_t(m) * nq * (p + 1));
  for (int e = 0; e < m; ++e)
    for (int q = 0; q < nq; ++q) {
      double x = (e + xg[q]) / m;
      t.xq[size_t(e) * nq + q] = x;
      t.wq[size_t(e) * nq + q] = wg[q] / m;
      nonzero_basis(kn, p, p + e, x, 1, d.data());
      for (int a = 0; a <= p; ++a) {
        t.B[(size_t(e) * nq + q) * (p + 1) + a] = d[a];
        t.dB[(size_t(e) * nq + q) * (p + 1) + a] = d[p + 1 + a];
      }
    }
  return t;
}

struct DevTables {  // device copies of one Tables1D
  double *xq, *wq, *B, *dB;
};

// Edge (1D) smoother of an interface piece: (h/p)^{d-1} K + (h/p)^{d-3} M on the interior
// indices of the edge's knot vector, applied by its generalised eigenvectors.
void edge_fd(int d, int m, int p, Mat& U, std::vector<double>& dinv) {
  Mat Mm, Km;
  mass_stiffness_1d(m, p, Mm, Km);
  std::vector<int> I;
  for (int i = 1; i < m + p - 1; ++i) I.push_back(i);
  int len = int(I.size());
  Mat MI = submatrix(Mm, m + p, I), KI = submatrix(Km, m + p, I);
  std::vector<double> lam;
  if (!generalized_eigen(len, KI, MI, lam, U)) throw Fail{IGAMG_ERR_NUMERIC, "edge eigen failed"};
  double h = 1.0 / m, a = std::pow(h / p, d - 1), b = std::pow(h / p, d - 3);
  dinv.resize(len);
  for (int q = 0; q < len; ++q) dinv[q] = 1.0 / (a * lam[q] + b);
}

void assemble_level(igamg_ctx* c, Level& L, std::map<std::tuple<int, int>, DevTables>& dtabs,
                    std::map<std::tuple<int, int>, Tables1D>& tabs, double* dcorn, bool mass, double* band) {
  const int d = c->pd.dim, K = c->pd.K;
  for (int k = 0; k < K; ++k) {
    const PatchDev& P = L.pd_h[k];
    ElemAsm ea{};
    ea.dim = d;
    ea.p = P.p[0];
    ea.mass = mass ? 1 : 0;
    int64_t nn = 1;
    for (int j = 0; j < 3; ++j) {
      ea.n[j] = P.n[j];
      ea.m[j] = P.m[j];
      ea.color[j] = 0;
    }
    for (int j = 0; j < d; ++j) {
      nn *= P.n[j];
      if (P.p[j] != P.p[0]) throw Fail{IGAMG_ERR_UNSUPPORTED, "direction-dependent degree"};
      auto key = std::make_tuple(P.m[j], P.p[j]);
      if (!tabs.count(key)) tabs[key] = tables_1d(P.m[j], P.p[j]);
      if (!dtabs.count(key)) {
        const Tables1D& tb = tabs[key];
        dtabs[key] = DevTables{c->mem.upload(tb.xq, c->stream), c->mem.upload(tb.wq, c->stream),
                               c->mem.upload(tb.B, c->stream), c->mem.upload(tb.dB, c->stream)};
      }
      const DevTables& t = dtabs[key];
      ea.xq[j] = t.xq;
      ea.wq[j] = t.wq;
      ea.B[j] = t.B;
      ea.dB[j] = t.dB;
    }
    ea.off = P.off;
    ea.band_off = P.band_off;
    ea.nn = nn;
    ea.corners = dcorn + size_t(k) * (1 << d) * d;
    ea.l2g = L.l2g;
    ea.band = band;
    CK(launch_assemble_elem(c->stream, ea));
  }
}

// Row-banded copy [n][2p+1] of a dense symmetric n x n banded 1D matrix.
std::vector<double> row_band(const Mat& A, int n, int p) {
  std::vector<double> b(size_t(n) * (2 * p + 1), 0.0);
  for (int i = 0; i < n; ++i)
    for (int t = 0; t <= 2 * p; ++t) {
      int j = i - p + t;
      if (j >= 0 && j < n) b[size_t(i) * (2 * p + 1) + t] = A[size_t(i) * n + j];
    }
  return b;
}

// Interior sizes from which the tensor-core FD is built (a candidate of the autotuner) and
// from which it is used when the autotuner is off.
constexpr int kTcMinLen = 32, kTcMinLenStatic = 96;

void build_levels(igamg_ctx* c) {
  cudaStream_t s = c->stream;
  const int d = c->pd.dim, K = c->pd.K;
  const int NL = c->pd.levels;
  for (int k = 0; k < K; ++k) {
    int lim = d == 2 ? 10 : 4;
    if (c->pd.p[k * d] > lim)
      throw Fail{IGAMG_ERR_UNSUPPORTED, "degree above " + std::to_string(lim) + " in " + std::to_string(d) + "D"};
  }
  c->lv.resize(NL);
  std::map<std::tuple<int, int, int, int, double>, Smoother1D> scms;  // (m,p,lo,hi,sigma)
  std::map<std::tuple<int, int>, Tables1D> tabs;
  std::map<std::tuple<int, int>, DevTables> dtabs;
  double* dcorn = c->mem.upload(c->pd.corners, s);
  auto get_scms = [&](int m, int p, bool lo, bool hi, double sigma) -> Smoother1D* {
    auto key = std::make_tuple(m, p, int(lo), int(hi), sigma);
    if (!scms.count(key)) scms[key] = build_scms(m, p, lo, hi, sigma);
    Smoother1D* S = &scms[key];
    if (!S->dU) S->dU = reg_const(c, c->mem.upload(S->U, s), S->U.size());
    return S;
  };
  for (int l = 0; l < NL; ++l) {
    Level& L = c->lv[l];
    int code = 0;
    std::string e = build_level(c->pd, l, L.topo, &code);
    if (!e.empty()) throw Fail{igamg_status(code), e};
    const LevelTopo& T = L.topo;
    int64_t band_total = 0;
    L.pd_h.resize(K);
    for (int k = 0; k < K; ++k) {
      PatchDev& P = L.pd_h[k];
      P.off = T.off[k];
      int64_t nn = T.off[k + 1] - T.off[k], nb = 1;
      for (int j = 0; j < 3; ++j) {
        P.n[j] = j < d ? T.n[k * d + j] : 1;
        P.p[j] = j < d ? c->pd.p[k * d + j] : 0;
        P.m[j] = j < d ? (c->pd.m[k * d + j] >> (NL - 1 - l)) : 1;
        if (j < d) nb *= 2 * P.p[j] + 1;
        L.max_n[j] = std::max(L.max_n[j], P.n[j]);
        L.max_p = std::max(L.max_p, P.p[j]);
      }
      P.band_off = band_total;
      band_total += nn * nb;
      L.apply_flops += 2.0 * double(nn) * nb;
      L.band_bytes += 8.0 * double(nn) * nb;
    }
    L.uniform_p = L.max_p;
    for (int q = 0; q < K * d; ++q)
      if (c->pd.p[q] != L.max_p) L.uniform_p = 0;
    L.pd = c->mem.upload(L.pd_h, s);
    L.l2g = c->mem.upload(T.l2g, s);
    L.g2t_ptr = c->mem.upload(T.g2t_ptr, s);
    L.g2t = c->mem.upload(T.g2t, s);
    L.band_doubles = band_total;
    // rectangle patches (2D, above the coarsest level): no bands, Kronecker-sum apply
    L.kron = d == 2 && l > 0 && c->opt.apply_engine == 0;
    std::vector<double> cc(2 * K);
    for (int k = 0; k < K && L.kron; ++k)
      L.kron = rect_metric(c->pd.corners.data() + size_t(k) * 8, &cc[2 * k], &cc[2 * k + 1]);
    if (L.kron) {
      std::vector<unsigned char> act(T.T);
      for (int64_t t = 0; t < T.T; ++t) act[t] = T.l2g[t] >= 0 ? 1 : 0;
      L.active = c->mem.upload(act, s);
      L.apply_flops = 0;
      L.band_bytes = 0;
      for (int k = 0; k < K; ++k) {
        const PatchDev& P = L.pd_h[k];
        KronDevT<double> kd{P.off, P.n[0], P.n[1], P.p[0], P.p[1], nullptr, nullptr, nullptr, nullptr,
                            cc[2 * k], cc[2 * k + 1]};
        const double* KM[2][2];
        for (int j = 0; j < 2; ++j) {
          auto key = std::make_tuple(P.m[j], P.p[j]);
          if (!c->kron_1d.count(key)) {
            Mat M1, K1;
            mass_stiffness_1d(P.m[j], P.p[j], M1, K1);
            int n = P.m[j] + P.p[j];
            std::vector<double> kb = row_band(K1, n, P.p[j]), mb = row_band(M1, n, P.p[j]);
            c->kron_1d[key] = {reg_const(c, c->mem.upload(kb, s), kb.size()),
                               reg_const(c, c->mem.upload(mb, s), mb.size())};
          }
          KM[j][0] = c->kron_1d[key].first;
          KM[j][1] = c->kron_1d[key].second;
        }
        kd.K0 = KM[0][0];
        kd.M0 = KM[0][1];
        kd.K1 = KM[1][0];
        kd.M1 = KM[1][1];
        L.kd_h.push_back(kd);
        double nn = double(P.n[0]) * P.n[1];
        L.apply_flops += nn * 4.0 * (2 * P.p[0] + 1 + 2 * P.p[1] + 1);  // 4d(2p+1) per node
      }
      L.n64.kd = c->mem.upload(L.kd_h, s);
      band_total = 0;
    }
    L.band = band_total ? c->mem.alloc<double>(band_total) : nullptr;
    L.n64.F = reg_work(c, c->mem.alloc<double>(T.T), T.T);
    L.n64.U = reg_work(c, c->mem.alloc<double>(T.T), T.T);
    L.n64.R = reg_work(c, c->mem.alloc<double>(T.T), T.T);
    CK(cudaMemsetAsync(L.n64.F, 0, T.T * sizeof(double), s));
    CK(cudaMemsetAsync(L.n64.U, 0, T.T * sizeof(double), s));
    CK(cudaMemsetAsync(L.n64.R, 0, T.T * sizeof(double), s));
    L.n64.band = L.band;
    L.n64.band_op = L.band;
    c->band_count.push_back(band_total);
    double ta0 = now_ms();
    if (!L.kron) {
      CK(cudaMemsetAsync(L.band, 0, band_total * sizeof(double), s));
      assemble_level(c, L, dtabs, tabs, dcorn, false, L.band);
    }
    CK(cudaStreamSynchronize(s));
    c->t_assemble_ms += now_ms() - ta0;
    if (l == 0) continue;

    // ---------------- patch-interior smoother
    std::map<std::string, double*> dinv_cache;
    // digit slices of an FD basis (or its transpose) for the tensor-core contractions,
    // uploaded once per (basis, orientation)
    struct Sl { const __nv_bfloat16* a; const int* e; int nkb; };
    std::map<std::pair<const Smoother1D*, int>, Sl> sl;
    auto slices = [&](const Smoother1D* S, int tr) -> Sl {
      auto key = std::make_pair(S, tr);
      if (!sl.count(key)) {
        int n = S->len;
        std::vector<double> A(size_t(n) * n);
        for (int i = 0; i < n; ++i)
          for (int k = 0; k < n; ++k) A[size_t(i) * n + k] = tr ? S->U[size_t(k) * n + i] : S->U[size_t(i) * n + k];
        std::vector<uint16_t> sv;
        std::vector<int> ev;
        slice_constant(A, n, n, 7, sv, ev);
        const __nv_bfloat16* da = reinterpret_cast<const __nv_bfloat16*>(c->mem.upload(sv, s));
        if (c->opt.precision == IGAMG_BF16) {
          std::vector<uint16_t> s1;
          std::vector<int> e1;
          slice_constant(A, n, n, 1, s1, e1);
          c->tc_bf16_twin[da] = c->mem.upload(s1, s);
        }
        sl[key] = Sl{da, c->mem.upload(ev, s), tc_kblocks(n)};
      }
      return sl[key];
    };
    // the same bases sliced as the N-side operand of the stacked (fibre-major) stages
    struct SlN { const __nv_bfloat16* w; const int* e; };
    std::map<std::pair<const Smoother1D*, int>, SlN> sln;
    auto slices_n = [&](const Smoother1D* S, int tr) -> SlN {
      auto key = std::make_pair(S, tr);
      if (!sln.count(key)) {
        int n = S->len;
        std::vector<double> A(size_t(n) * n);
        for (int i = 0; i < n; ++i)
          for (int k = 0; k < n; ++k) A[size_t(i) * n + k] = tr ? S->U[size_t(k) * n + i] : S->U[size_t(i) * n + k];
        std::vector<uint16_t> sv;
        std::vector<int> ev;
        slice_constant(A, n, n, 7, sv, ev, 32);
        sln[key] = SlN{reinterpret_cast<const __nv_bfloat16*>(c->mem.upload(sv, s)), c->mem.upload(ev, s)};
      }
      return sln[key];
    };
    if (d == 2) {
      int64_t fd_total = 0;
      std::vector<GemmDesc> s0F, s0R, s1, s2, s3;
      for (const Interior& in : T.interiors) {
        const PatchDev& P = L.pd_h[in.k];
        if (in.len[0] == 0 || in.len[1] == 0) continue;  // empty piece (p = 1, one element)
        Smoother1D* S[2];
        for (int j = 0; j < 2; ++j) {
          S[j] = get_scms(P.m[j], P.p[j], in.drop_lo[j], in.drop_hi[j], c->opt.sigma_scale * double(P.m[j]) * P.m[j]);
          if (S[j]->len != in.len[j]) throw Fail{IGAMG_ERR_NUMERIC, "smoother size mismatch"};
        }
        int n0 = in.len[0], n1 = in.len[1];
        std::string dk = std::to_string(intptr_t(S[0])) + "/" + std::to_string(intptr_t(S[1]));
        if (!dinv_cache.count(dk)) {
          std::vector<double> Dv(size_t(n0) * n1);
          for (int a = 0; a < n0; ++a)
            for (int b = 0; b < n1; ++b) Dv[size_t(a) * n1 + b] = 1.0 / (S[0]->mu[a] + S[1]->mu[b]);
          dinv_cache[dk] = reg_const(c, c->mem.upload(Dv, s), Dv.size());
        }
        double* Dinv = dinv_cache[dk];
        int64_t base = fd_total;
        fd_total += int64_t(n0) * n1;
        int64_t xoff = P.off + int64_t(in.lo[0]) * P.n[1] + in.lo[1];
        GemmDesc g0{S[0]->dU, nullptr, (double*)(intptr_t)base, nullptr, n0, P.n[1], n1, 0, n0, n1, n0};
        GemmDesc gF = g0, gR = g0;
        gF.B = L.n64.F + xoff;
        gR.B = L.n64.R + xoff;
        s0F.push_back(gF);
        s0R.push_back(gR);
        s1.push_back(GemmDesc{(double*)(intptr_t)base, S[1]->dU, (double*)(intptr_t)base, Dinv, n1, n1, n1, n1, n0, n1, n1});
        s2.push_back(GemmDesc{S[0]->dU, (double*)(intptr_t)base, (double*)(intptr_t)base, nullptr, n0, n1, n1, 0, n0, n1, n0});
        s3.push_back(GemmDesc{(double*)(intptr_t)base, S[1]->dU, L.n64.U + xoff, nullptr, n1, n1, P.n[1], 0, n0, n1, n1});
      }
      double* fdT = reg_work(c, c->mem.alloc<double>(fd_total), fd_total);
      double* fdY = reg_work(c, c->mem.alloc<double>(fd_total), fd_total);
      for (auto& g : s0F) g.C = fdT + (intptr_t)g.C;
      for (auto& g : s0R) g.C = fdT + (intptr_t)g.C;
      for (auto& g : s1) { g.A = fdT + (intptr_t)g.A; g.C = fdY + (intptr_t)g.C; }
      for (auto& g : s2) { g.B = fdY + (intptr_t)g.B; g.C = fdT + (intptr_t)g.C; }
      for (auto& g : s3) g.A = fdT + (intptr_t)g.A;
      set_gemm(c, L.n64.st0F, s0F);
      set_gemm(c, L.n64.st0R, s0R);
      set_gemm(c, L.n64.st1, s1);
      set_gemm(c, L.n64.st2, s2);
      set_gemm(c, L.n64.st3, s3);
      // row-block FD (a candidate of the autotuner), Y in the stage-1 scratch of each interior
      {
        std::vector<FdRowsT<double>> fr;
        size_t q = 0;
        int mx0 = 0, mx1 = 0;
        for (const Interior& in : T.interiors) {
          if (in.len[0] == 0 || in.len[1] == 0) continue;
          const PatchDev& P = L.pd_h[in.k];
          const int64_t xoff = P.off + int64_t(in.lo[0]) * P.n[1] + in.lo[1];
          fr.push_back(FdRowsT<double>{s0F[q].A, s1[q].B, s1[q].E, L.n64.F + xoff, L.n64.R + xoff, L.n64.U + xoff,
                                       s1[q].C, in.len[0], in.len[1], P.n[1]});
          mx0 = std::max(mx0, in.len[0]);
          mx1 = std::max(mx1, in.len[1]);
          ++q;
        }
        if (!fr.empty()) {
          L.fr_h = fr;
          L.n64.frows = c->mem.upload(fr, s);
          L.n64.nfrows = int(fr.size());
          L.n64.frows_n0 = mx0;
          L.n64.frows_n1 = mx1;
          L.n64.use_rows = c->opt.fd_engine == 4;
        }
      }
      // one-block FD for small interiors (a candidate of the autotuner)
      {
        bool ok = !s0F.empty();
        std::vector<FdSmallT<double>> fs;
        size_t q = 0;
        double fl = 0;
        for (const Interior& in : T.interiors) {
          if (in.len[0] == 0 || in.len[1] == 0) continue;
          const PatchDev& P = L.pd_h[in.k];
          const int n0 = in.len[0], n1 = in.len[1];
          ok = ok && n0 <= kFdSmallMax && n1 <= kFdSmallMax;
          const int64_t xoff = P.off + int64_t(in.lo[0]) * P.n[1] + in.lo[1];
          fs.push_back(FdSmallT<double>{s0F[q].A, s1[q].B, s1[q].E, L.n64.F + xoff, L.n64.R + xoff, L.n64.U + xoff, n0,
                                        n1, P.n[1]});
          fl += 4.0 * n0 * n1 * double(n0 + n1);
          ++q;
        }
        if (ok) {
          L.fused_ok = true;
          L.fs_h = fs;
          L.n64.fsmall = c->mem.upload(fs, s);
          L.n64.nfsmall = int(fs.size());
          L.n64.fsmall_flops = fl;
          L.n64.use_fused = c->opt.fd_engine == 3;
        }
      }
      int min_len = 1 << 30;
      for (const Interior& in : T.interiors)
        if (in.len[0] && in.len[1]) min_len = std::min(min_len, std::min(in.len[0], in.len[1]));
      // tensor cores where the interiors are large enough to amortise the slices
      int max_len = 0;
      for (const Interior& in : T.interiors) max_len = std::max(max_len, std::max(in.len[0], in.len[1]));
      // (FP64 digit sums are exact up to K = kTcMaxK)
      const bool want_tc = max_len <= kTcMaxK &&
                           (c->opt.fd_engine == 2 ? min_len >= 1 : c->opt.fd_engine == 0 && min_len >= kTcMinLen);
      if (want_tc) {
        // constant-left form: T = U0^T X, Y^T = U1^T T^T (.* Dinv), S = U0 Y, Z^T = U1 S^T
        std::vector<TcDesc<double, double>> t0F, t0R, t1, t2, t3;
        // fibre-major stacked form (the FP64 engine's): T = U0^T X kept as [n0][n1],
        // Y = (T U1) .* Dinv kept as Y^T [n1][n0], Q = Y U1^T kept as Q^T [n1][n0] in T's
        // scratch, Z = U0 Q into the tile; every stage writes fibre-contiguous rows.  Patches
        // with the same basis and sizes form one descriptor per stage.
        using SD = TcStack<double, double>;
        using SKey = std::tuple<const void*, int, int, int, int>;  // W slices, F, K, ldx, ldc
        struct SGrp {
          SD proto{};
          std::vector<const double*> X, E;
          std::vector<double*> C;
        };
        std::map<SKey, SGrp> sgrp[5];
        auto sadd = [&](int st, const SlN& w, int N, int K, const double* X, int xt, int ldx, int F, double* C, int ldc,
                        const double* E, int et, int lde) {
          SGrp& g = sgrp[st][SKey{w.w, F, K, ldx, ldc}];
          if (g.X.empty()) g.proto = SD{w.w, w.e, nullptr, nullptr, nullptr, ldx, xt, ldc, 0, lde, et, 0, F, N, K};
          g.X.push_back(X);
          g.C.push_back(C);
          g.E.push_back(E);
        };
        size_t q = 0;
        for (const Interior& in : T.interiors) {
          const PatchDev& P = L.pd_h[in.k];
          if (in.len[0] == 0 || in.len[1] == 0) continue;
          const Smoother1D* S0 = get_scms(P.m[0], P.p[0], in.drop_lo[0], in.drop_hi[0], c->opt.sigma_scale * double(P.m[0]) * P.m[0]);
          const Smoother1D* S1 = get_scms(P.m[1], P.p[1], in.drop_lo[1], in.drop_hi[1], c->opt.sigma_scale * double(P.m[1]) * P.m[1]);
          int n0 = in.len[0], n1 = in.len[1];
          const GemmDesc& g0 = s0F[q];
          const GemmDesc& g1 = s1[q];
          const GemmDesc& g3 = s3[q];
          double* Tb = g0.C;   // scratch T (n0 x n1)
          double* Yb = g1.C;   // scratch Y
          Sl a0t = slices(S0, 1), a1t = slices(S1, 1), a0 = slices(S0, 0), a1 = slices(S1, 0);
          // every stage stores its output transposed (lanes of the epilogue write consecutive
          // addresses): T and S are kept as T^T, S^T ([n1][n0]), which the next stage reads
          // row by row
          TcDesc<double, double> d0{a0t.a, a0t.e, a0t.nkb, g0.B, P.n[1], 0, Tb, n0, 1, nullptr, 0, n0, n1, n0};
          t0F.push_back(d0);
          d0.B = s0R[q].B;
          t0R.push_back(d0);
          t1.push_back(TcDesc<double, double>{a1t.a, a1t.e, a1t.nkb, Tb, n0, 0, Yb, n1, 1, g1.E, n1, n1, n0, n1});
          t2.push_back(TcDesc<double, double>{a0.a, a0.e, a0.nkb, Yb, n1, 0, Tb, n0, 1, nullptr, 0, n0, n1, n0});
          t3.push_back(TcDesc<double, double>{a1.a, a1.e, a1.nkb, Tb, n0, 0, g3.C, P.n[1], 1, nullptr, 0, n1, n0, n1});
          const SlN w0t = slices_n(S0, 1), w1t = slices_n(S1, 1), w0 = slices_n(S0, 0), w1 = slices_n(S1, 0);
          sadd(0, w0t, n0, n0, g0.B, 0, P.n[1], n1, Tb, n1, nullptr, 0, 0);
          sadd(1, w0t, n0, n0, s0R[q].B, 0, P.n[1], n1, Tb, n1, nullptr, 0, 0);
          sadd(2, w1t, n1, n1, Tb, 1, n1, n0, Yb, n0, g1.E, 1, n1);
          sadd(3, w1, n1, n1, Yb, 0, n0, n0, Tb, n0, nullptr, 0, 0);
          sadd(4, w0, n0, n0, Tb, 1, n0, n1, g3.C, P.n[1], nullptr, 0, 0);
          ++q;
        }
        StackSet* sout[5] = {&L.n64.sk0F, &L.n64.sk0R, &L.n64.sk1, &L.n64.sk2, &L.n64.sk3};
        for (int st = 0; st < 5; ++st) {
          std::vector<SD> v;
          for (auto& kv : sgrp[st]) {
            SD dd = kv.second.proto;
            dd.P = int(kv.second.X.size());
            dd.X = c->mem.upload(kv.second.X, s);
            dd.C = c->mem.upload(kv.second.C, s);
            dd.E = st == 2 ? c->mem.upload(kv.second.E, s) : nullptr;
            v.push_back(dd);
          }
          set_stack(*sout[st], v);
          for (auto& kv : sgrp[st]) {
            sout[st]->hX.push_back(kv.second.X);
            sout[st]->hC.push_back(kv.second.C);
            sout[st]->hE.push_back(kv.second.E);
          }
        }
        set_tc(c, L.n64.tc0F, t0F);
        set_tc(c, L.n64.tc0R, t0R);
        set_tc(c, L.n64.tc1, t1);
        set_tc(c, L.n64.tc2, t2);
        set_tc(c, L.n64.tc3, t3);
        L.tc_ok = true;
        // without the autotuner: the tensor cores from interiors of kTcMinLenStatic up
        L.n64.use_tc = c->opt.fd_engine == 2 || min_len >= kTcMinLenStatic;
      }
    } else {
      // 3D: compact boxes, three mode products forward, Dinv, three backward
      std::vector<BoxDev> boxes;
      std::vector<GemmDesc> f0, f1, f2, b0, b1, b2;
      int64_t tot = 0;
      struct Pend { int64_t base; int n0, n1, n2; Smoother1D* S[3]; double* Dinv; };
      std::vector<Pend> pend;
      for (const Interior& in : T.interiors) {
        const PatchDev& P = L.pd_h[in.k];
        if (in.len[0] == 0 || in.len[1] == 0 || in.len[2] == 0) continue;
        Pend pe;
        for (int j = 0; j < 3; ++j) {
          pe.S[j] = get_scms(P.m[j], P.p[j], in.drop_lo[j], in.drop_hi[j], c->opt.sigma_scale * double(P.m[j]) * P.m[j]);
          if (pe.S[j]->len != in.len[j]) throw Fail{IGAMG_ERR_NUMERIC, "smoother size mismatch"};
        }
        pe.n0 = in.len[0];
        pe.n1 = in.len[1];
        pe.n2 = in.len[2];
        std::string dk = std::to_string(intptr_t(pe.S[0])) + "/" + std::to_string(intptr_t(pe.S[1])) + "/" +
                         std::to_string(intptr_t(pe.S[2]));
        if (!dinv_cache.count(dk)) {
          std::vector<double> Dv(size_t(pe.n0) * pe.n1 * pe.n2);
          for (int a = 0; a < pe.n0; ++a)
            for (int b = 0; b < pe.n1; ++b)
              for (int q = 0; q < pe.n2; ++q)
                Dv[(size_t(a) * pe.n1 + b) * pe.n2 + q] = 1.0 / (pe.S[0]->mu[a] + pe.S[1]->mu[b] + pe.S[2]->mu[q]);
          dinv_cache[dk] = reg_const(c, c->mem.upload(Dv, s), Dv.size());
        }
        pe.Dinv = dinv_cache[dk];
        pe.base = tot;
        BoxDev bx;
        bx.tile_off = P.off;
        bx.compact_off = tot;
        for (int j = 0; j < 3; ++j) {
          bx.n[j] = P.n[j];
          bx.lo[j] = in.lo[j];
          bx.len[j] = in.len[j];
        }
        boxes.push_back(bx);
        int64_t vol = int64_t(pe.n0) * pe.n1 * pe.n2;
        L.max_box = std::max(L.max_box, vol);
        tot += vol;
        pend.push_back(pe);
      }
      L.nbox = int(boxes.size());
      L.boxes = c->mem.upload(boxes, s);
      L.box_vol = tot;
      {  // every interior small enough for the one-launch kernel
        bool ok = !pend.empty();
        std::vector<Fd3SmallT<double>> f3;
        for (size_t i = 0; i < pend.size() && ok; ++i) {
          const Pend& pe = pend[i];
          ok = std::max(pe.n0, std::max(pe.n1, pe.n2)) <= kFd3SmallN;
          Fd3SmallT<double> f{pe.S[0]->dU, pe.S[1]->dU, pe.S[2]->dU, pe.Dinv, boxes[i].tile_off, {}, {}, {}};
          for (int j = 0; j < 3; ++j) {
            f.n[j] = boxes[i].n[j];
            f.lo[j] = boxes[i].lo[j];
            f.len[j] = boxes[i].len[j];
          }
          f3.push_back(f);
        }
        if (ok) {
          L.fd3_h = f3;
          L.n64.fd3 = c->mem.upload(f3, s);
          L.n64.nfd3 = int(f3.size());
        }
      }
      L.n64.cX = reg_work(c, c->mem.alloc<double>(tot), tot);
      double* cB1 = reg_work(c, c->mem.alloc<double>(tot), tot);
      double* cB2 = reg_work(c, c->mem.alloc<double>(tot), tot);
      for (const Pend& pe : pend) {
        int n0 = pe.n0, n1 = pe.n1, n2 = pe.n2, n12 = n1 * n2;
        double *X = L.n64.cX + pe.base, *B1 = cB1 + pe.base, *B2 = cB2 + pe.base;
        const double *U0 = pe.S[0]->dU, *U1 = pe.S[1]->dU, *U2 = pe.S[2]->dU;
        f0.push_back(GemmDesc{U0, X, B1, nullptr, n0, n12, n12, 0, n0, n12, n0});
        for (int a = 0; a < n0; ++a)
          f1.push_back(GemmDesc{U1, B1 + int64_t(a) * n12, B2 + int64_t(a) * n12, nullptr, n1, n2, n2, 0, n1, n2, n1});
        f2.push_back(GemmDesc{B2, U2, B1, pe.Dinv, n2, n2, n2, n2, n0 * n1, n2, n2});
        b0.push_back(GemmDesc{U0, B1, B2, nullptr, n0, n12, n12, 0, n0, n12, n0});
        for (int a = 0; a < n0; ++a)
          b1.push_back(GemmDesc{U1, B2 + int64_t(a) * n12, B1 + int64_t(a) * n12, nullptr, n1, n2, n2, 0, n1, n2, n1});
        b2.push_back(GemmDesc{B1, U2, X, nullptr, n2, n2, n2, 0, n0 * n1, n2, n2});
      }
      // the same products as one mode-product launch per stage (matrices of at most
      // kModeMaxN rows), used instead of the GEMM stages by the FMA engine
      {
        bool ok = !pend.empty();
        std::vector<ModeDescT<double>> md[6];
        for (const Pend& pe : pend) {
          int n0 = pe.n0, n1 = pe.n1, n2 = pe.n2;
          ok = ok && std::max(n0, std::max(n1, n2)) <= kModeMaxN;
          const int64_t n12 = int64_t(n1) * n2;
          double *X = L.n64.cX + pe.base, *B1 = cB1 + pe.base, *B2 = cB2 + pe.base;
          const double *U0 = pe.S[0]->dU, *U1 = pe.S[1]->dU, *U2 = pe.S[2]->dU;
          md[0].push_back(ModeDescT<double>{U0, X, B1, nullptr, n0, 1, n12, n12});
          md[1].push_back(ModeDescT<double>{U1, B1, B2, nullptr, n1, 1, n2, int64_t(n0) * n2});
          md[2].push_back(ModeDescT<double>{U2, B2, B1, pe.Dinv, n2, 1, 1, int64_t(n0) * n1});
          md[3].push_back(ModeDescT<double>{U0, B1, B2, nullptr, n0, 0, n12, n12});
          md[4].push_back(ModeDescT<double>{U1, B2, B1, nullptr, n1, 0, n2, int64_t(n0) * n2});
          md[5].push_back(ModeDescT<double>{U2, B1, X, nullptr, n2, 0, 1, int64_t(n0) * n1});
        }
        if (ok)
          for (int j = 0; j < 6; ++j) set_mode(c, L.n64.md[j], md[j]);
      }
      set_gemm(c, L.n64.m0f, f0);
      set_gemm(c, L.n64.m1f, f1);
      set_gemm(c, L.n64.m2f, f2);
      set_gemm(c, L.n64.m0b, b0);
      set_gemm(c, L.n64.m1b, b1);
      set_gemm(c, L.n64.m2b, b2);
      int min_len = 1 << 30;
      for (const Pend& pe : pend) min_len = std::min(min_len, std::min(pe.n0, std::min(pe.n1, pe.n2)));
      int max_len = 0;
      for (const Pend& pe : pend) max_len = std::max(max_len, std::max(pe.n0, std::max(pe.n1, pe.n2)));
      const bool want_tc = !pend.empty() && max_len <= kTcMaxK &&
                           (c->opt.fd_engine == 2 ? true : c->opt.fd_engine == 0 && min_len >= kTcMinLen);
      if (want_tc) {
        // tensor cores: each stage contracts the leading mode and rotates it to the back,
        // C(i1, i2, j0) = sum_i0 U(i0, j0) X(i0, i1, i2), an n x n^2 product stored
        // transposed; three stages restore the order (j0, j1, j2), where Dinv is applied.
        std::vector<TcDesc<double, double>> tf[3], tb[3];
        for (const Pend& pe : pend) {
          const int n[3] = {pe.n0, pe.n1, pe.n2};
          const int64_t vol = int64_t(pe.n0) * pe.n1 * pe.n2;
          double *X = L.n64.cX + pe.base, *B1 = cB1 + pe.base, *B2 = cB2 + pe.base;
          double* fin[3] = {X, B1, B2};
          double* fout[3] = {B1, B2, B1};
          double* bin[3] = {B1, B2, B1};
          double* bout[3] = {B2, B1, X};
          for (int j = 0; j < 3; ++j) {
            const int m = n[j], rest = int(vol / m);
            const Sl at = slices(pe.S[j], 1), a = slices(pe.S[j], 0);
            const double* E = j == 2 ? pe.Dinv : nullptr;
            tf[j].push_back(TcDesc<double, double>{at.a, at.e, at.nkb, fin[j], rest, 0, fout[j], m, 1, E, m, m, rest, m});
            tb[j].push_back(TcDesc<double, double>{a.a, a.e, a.nkb, bin[j], rest, 0, bout[j], m, 1, nullptr, 0, m, rest, m});
          }
        }
        set_tc(c, L.n64.tc0F, tf[0]);
        set_tc(c, L.n64.tc1, tf[1]);
        set_tc(c, L.n64.tc2, tf[2]);
        set_tc(c, L.n64.tc3, tb[0]);
        set_tc(c, L.n64.tc4, tb[1]);
        set_tc(c, L.n64.tc5, tb[2]);
        L.tc_ok = true;
        L.n64.use_tc = c->opt.fd_engine == 2 || min_len >= kTcMinLenStatic;
      }
    }

    // ---------------- interface pieces: vertices; edges and faces grouped by signature
    std::map<std::tuple<int, int, int, int, int>, std::vector<int>> groups;  // (kind, m, p, len0, len1)
    for (int i = 0; i < int(T.ifaces.size()); ++i) {
      const IfacePiece& pc = T.ifaces[i];
      const PatchDev& P = L.pd_h[pc.k];
      if (pc.kind == PIECE_VERTEX) groups[std::make_tuple(0, 0, 0, 1, 1)].push_back(i);
      else {
        int j = pc.dirs[0];
        groups[std::make_tuple(pc.kind, P.m[j], P.p[j], pc.len[0], pc.len[1])].push_back(i);
      }
    }
    std::vector<int64_t> ptr{0}, idx;
    std::vector<double> vsc;
    std::vector<GemmDesc> eA, eB, q0, q1, q2, q3;
    std::vector<TcDesc<double, double>> tqd[4];
    bool face_tc = true;
    std::vector<EdgeSmallT<double>> es;
    bool edges_small = d == 2;
    std::vector<FaceSmallT<double>> fsm;  // 3D: faces for the one-launch interface smoother
    bool iface3_small = d == 3;
    int64_t vtx_beg = 0, vtx_end = 0;
    int64_t face_tot = 0;
    for (auto& kv : groups) {
      int kind = std::get<0>(kv.first);
      int64_t gbase = int64_t(vsc.size());
      for (int i : kv.second) {
        const IfacePiece& pc = T.ifaces[i];
        int64_t cnt = int64_t(pc.len[0]) * pc.len[1];
        for (int64_t q = 0; q < cnt; ++q) {
          int64_t g = T.iface_gid[pc.first + q];
          for (int64_t cc = T.g2t_ptr[g]; cc < T.g2t_ptr[g + 1]; ++cc) idx.push_back(T.g2t[cc]);
          ptr.push_back(int64_t(idx.size()));
          double vs = 0.0;
          if (kind == PIECE_VERTEX) {
            const PatchDev& P = L.pd_h[pc.k];
            double h = 1.0 / P.m[0], p = P.p[0];
            vs = 1.0 / std::pow(h / p, d - 2);
          }
          vsc.push_back(vs);
        }
      }
      int m = std::get<1>(kv.first), p = std::get<2>(kv.first);
      int len0 = std::get<3>(kv.first), len1 = std::get<4>(kv.first);
      int np = int(kv.second.size());
      if (kind == PIECE_VERTEX) {
        vtx_beg = gbase;
        vtx_end = int64_t(vsc.size());
      }
      if (kind == PIECE_EDGE && len0 > 0) {
        Mat U;
        std::vector<double> dv;
        edge_fd(d, m, p, U, dv);
        double* dU = reg_const(c, c->mem.upload(U, s), U.size());
        double* ddv = reg_const(c, c->mem.upload(dv, s), dv.size());
        edges_small = edges_small && len0 <= kFdSmallMax;
        iface3_small = iface3_small && len0 <= kIface3SmallN;
        for (int j = 0; j < np; ++j) es.push_back(EdgeSmallT<double>{dU, ddv, gbase + int64_t(j) * len0, len0});
        eA.push_back(GemmDesc{(double*)(intptr_t)gbase, dU, (double*)(intptr_t)gbase, ddv, len0, len0, len0, 0, np, len0, len0});
        eB.push_back(GemmDesc{(double*)(intptr_t)gbase, dU, (double*)(intptr_t)gbase, nullptr, len0, len0, len0, 0, np, len0, len0});
      } else if (kind == PIECE_FACE && len0 > 0 && len1 > 0) {
        // 2D subspace-corrected mass smoother of the face, D = (h/p)(mu0 + mu1 + p^2/h^2)
        double h = 1.0 / m, sigma = c->opt.sigma_scale * double(m) * m;
        Smoother1D* S0 = get_scms(m, p, true, true, sigma);
        Smoother1D* S1 = get_scms(m, p, true, true, sigma);
        std::vector<double> Dv(size_t(len0) * len1);
        for (int a = 0; a < len0; ++a)
          for (int b = 0; b < len1; ++b)
            Dv[size_t(a) * len1 + b] = 1.0 / ((h / p) * (S0->mu[a] + S1->mu[b] + double(p) * p / (h * h)));
        double* Dinv = reg_const(c, c->mem.upload(Dv, s), Dv.size());
        const bool tcf = std::max(len0, len1) <= kTcMaxK &&
                         (c->opt.fd_engine == 2 || (c->opt.fd_engine == 0 && std::min(len0, len1) >= kTcMinLen));
        face_tc = face_tc && tcf;
        Sl a0t{}, a1t{}, a0{}, a1{};
        if (tcf) {
          a0t = slices(S0, 1);
          a1t = slices(S1, 1);
          a0 = slices(S0, 0);
          a1 = slices(S1, 0);
        }
        iface3_small = iface3_small && std::max(len0, len1) <= kIface3SmallN;
        for (int f = 0; f < np; ++f) {
          int64_t off = gbase + int64_t(f) * len0 * len1, tb = face_tot + int64_t(f) * len0 * len1;
          fsm.push_back(FaceSmallT<double>{S0->dU, S1->dU, Dinv, off, len0, len1});
          q0.push_back(GemmDesc{S0->dU, (double*)(intptr_t)off, (double*)(intptr_t)tb, nullptr, len0, len1, len1, 0, len0, len1, len0});
          q1.push_back(GemmDesc{(double*)(intptr_t)tb, S1->dU, (double*)(intptr_t)tb, Dinv, len1, len1, len1, len1, len0, len1, len1});
          q2.push_back(GemmDesc{S0->dU, (double*)(intptr_t)tb, (double*)(intptr_t)tb, nullptr, len0, len1, len1, 0, len0, len1, len0});
          q3.push_back(GemmDesc{(double*)(intptr_t)tb, S1->dU, (double*)(intptr_t)off, nullptr, len1, len1, len1, 0, len0, len1, len1});
          if (tcf) {  // the interior formulation on the face block (offsets resolved below)
            using TD = TcDesc<double, double>;
            // outputs stored transposed, as for the interiors (T^T and S^T in fT)
            tqd[0].push_back(TD{a0t.a, a0t.e, a0t.nkb, (double*)(intptr_t)off, len1, 0, (double*)(intptr_t)tb, len0, 1,
                                nullptr, 0, len0, len1, len0});
            tqd[1].push_back(TD{a1t.a, a1t.e, a1t.nkb, (double*)(intptr_t)tb, len0, 0, (double*)(intptr_t)tb, len1, 1,
                                Dinv, len1, len1, len0, len1});
            tqd[2].push_back(TD{a0.a, a0.e, a0.nkb, (double*)(intptr_t)tb, len1, 0, (double*)(intptr_t)tb, len0, 1,
                                nullptr, 0, len0, len1, len0});
            tqd[3].push_back(TD{a1.a, a1.e, a1.nkb, (double*)(intptr_t)tb, len0, 0, (double*)(intptr_t)off, len1, 1,
                                nullptr, 0, len1, len0, len1});
          }
        }
        face_tot += int64_t(np) * len0 * len1;
      }
    }
    L.n_if = int64_t(vsc.size());
    L.if_ptr = c->mem.upload(ptr, s);
    L.if_idx = c->mem.upload(idx, s);
    L.n64.vscale = reg_const(c, c->mem.upload(vsc, s), vsc.size());
    if (iface3_small && L.n_if > 0) {  // every face and edge small: the one-launch interface smoother
      L.f3s_h = fsm;
      L.e3s_h = es;
      L.v3_beg = vtx_beg;
      L.v3_end = vtx_end;
      Iface3SmallT<double>& q = L.n64.i3s;
      q.faces = fsm.empty() ? nullptr : c->mem.upload(fsm, s);
      q.nfaces = int(fsm.size());
      q.edges = es.empty() ? nullptr : c->mem.upload(es, s);
      q.nedges = int(es.size());
      q.ptr = L.if_ptr;
      q.idx = L.if_idx;
      q.vscale = L.n64.vscale;
      q.vbeg = vtx_beg;
      q.vend = vtx_end;
      q.u = L.n64.U;
      L.n64.i3_ok = true;
    }
    L.n64.G = reg_work(c, c->mem.alloc<double>(L.n_if), L.n_if);
    L.n64.Z = reg_work(c, c->mem.alloc<double>(L.n_if), L.n_if);
    double* Yif = reg_work(c, c->mem.alloc<double>(L.n_if), L.n_if);
    double* fT = reg_work(c, c->mem.alloc<double>(face_tot), face_tot);
    double* fY = reg_work(c, c->mem.alloc<double>(face_tot), face_tot);
    CK(cudaMemsetAsync(L.n64.Z, 0, std::max<int64_t>(L.n_if, 1) * sizeof(double), s));
    for (auto& g : eA) { g.A = L.n64.G + (intptr_t)g.A; g.C = Yif + (intptr_t)g.C; }
    for (auto& g : eB) { g.A = Yif + (intptr_t)g.A; g.C = L.n64.Z + (intptr_t)g.C; }
    for (auto& g : q0) { g.B = L.n64.G + (intptr_t)g.B; g.C = fT + (intptr_t)g.C; }
    for (auto& g : q1) { g.A = fT + (intptr_t)g.A; g.C = fY + (intptr_t)g.C; }
    for (auto& g : q2) { g.B = fY + (intptr_t)g.B; g.C = fT + (intptr_t)g.C; }
    for (auto& g : q3) { g.A = fT + (intptr_t)g.A; g.C = L.n64.Z + (intptr_t)g.C; }
    set_gemm(c, L.n64.edgeA, eA);
    set_gemm(c, L.n64.edgeB, eB);
    if (L.fused_ok && edges_small) {  // the whole smoother of this level in one launch
      L.small_ok = true;
      L.es_h = es;
      SmoothSmallT<double>& q = L.n64.ssmall;
      q.fd = L.n64.fsmall;
      q.nfd = L.n64.nfsmall;
      q.edges = es.empty() ? nullptr : c->mem.upload(es, s);
      q.nedges = int(es.size());
      q.ptr = L.if_ptr;
      q.idx = L.if_idx;
      q.vscale = L.n64.vscale;
      q.vbeg = vtx_beg;
      q.vend = vtx_end;
      q.vF = L.n64.F;
      q.vR = L.n64.R;
      q.u = L.n64.U;
      double fl = L.n64.fsmall_flops;
      for (const auto& e : es) fl += 4.0 * e.len * double(e.len);
      L.n64.ssmall_flops = fl;
    }
    set_gemm(c, L.n64.face0, q0);
    set_gemm(c, L.n64.face1, q1);
    set_gemm(c, L.n64.face2, q2);
    set_gemm(c, L.n64.face3, q3);
    if (!q0.empty()) {  // the same four products as mode products (faces of <= kModeMaxN)
      bool ok = true;
      std::vector<ModeDescT<double>> fm[4];
      for (size_t f = 0; f < q0.size(); ++f) {
        const int len0 = q0[f].M, len1 = q0[f].N;
        ok = ok && std::max(len0, len1) <= kModeMaxN;
        fm[0].push_back(ModeDescT<double>{q0[f].A, q0[f].B, q0[f].C, nullptr, len0, 1, len1, len1});
        fm[1].push_back(ModeDescT<double>{q1[f].B, q1[f].A, q1[f].C, q1[f].E, len1, 1, 1, len0});
        fm[2].push_back(ModeDescT<double>{q2[f].A, q2[f].B, q2[f].C, nullptr, len0, 0, len1, len1});
        fm[3].push_back(ModeDescT<double>{q3[f].B, q3[f].A, q3[f].C, nullptr, len1, 0, 1, len0});
      }
      if (ok)
        for (int j = 0; j < 4; ++j) set_mode(c, L.n64.fm[j], fm[j]);
    }
    if (face_tc && !q0.empty()) {
      // stage 0 reads G, 1 reads T writes Y, 2 reads Y writes T, 3 reads T writes Z
      for (auto& t : tqd[0]) { t.B = L.n64.G + (intptr_t)t.B; t.C = fT + (intptr_t)t.C; }
      for (auto& t : tqd[1]) { t.B = fT + (intptr_t)t.B; t.C = fY + (intptr_t)t.C; }
      for (auto& t : tqd[2]) { t.B = fY + (intptr_t)t.B; t.C = fT + (intptr_t)t.C; }
      for (auto& t : tqd[3]) { t.B = fT + (intptr_t)t.B; t.C = L.n64.Z + (intptr_t)t.C; }
      set_tc(c, L.n64.tq0, tqd[0], true);
      set_tc(c, L.n64.tq1, tqd[1], true);
      set_tc(c, L.n64.tq2, tqd[2], true);
      set_tc(c, L.n64.tq3, tqd[3], true);
    }

    // ---------------- transfers from level l-1 (one 1D pass per direction)
    const Level& C = c->lv[l - 1];
    std::map<std::tuple<int, int>, std::vector<void*>> ptabs;
    std::map<std::tuple<int, int>, std::pair<std::vector<int>, std::vector<int>>> pstart_h;  // rs, ps
    auto tables = [&](int mc, int p) -> std::vector<void*>& {
      auto key = std::make_tuple(mc, p);
      if (!ptabs.count(key)) {
        Mat P = prolongation_1d(mc, p);
        int nf = 2 * mc + p, nc = mc + p, wp = 0, wr = 0;
        std::vector<int> ps(nf), rs(nc);
        for (int i = 0; i < nf; ++i) {
          int lo = nc, hi = -1;
          for (int jj = 0; jj < nc; ++jj)
            if (P[size_t(i) * nc + jj] != 0.0) { lo = std::min(lo, jj); hi = std::max(hi, jj); }
          ps[i] = hi < 0 ? 0 : lo;
          wp = std::max(wp, hi - lo + 1);
        }
        for (int jj = 0; jj < nc; ++jj) {
          int lo = nf, hi = -1;
          for (int i = 0; i < nf; ++i)
            if (P[size_t(i) * nc + jj] != 0.0) { lo = std::min(lo, i); hi = std::max(hi, i); }
          rs[jj] = hi < 0 ? 0 : lo;
          wr = std::max(wr, hi - lo + 1);
        }
        std::vector<double> pw(size_t(nf) * wp, 0.0), rw(size_t(nc) * wr, 0.0);
        for (int i = 0; i < nf; ++i)
          for (int a = 0; a < wp && ps[i] + a < nc; ++a) pw[size_t(i) * wp + a] = P[size_t(i) * nc + ps[i] + a];
        for (int jj = 0; jj < nc; ++jj)
          for (int a = 0; a < wr && rs[jj] + a < nf; ++a) rw[size_t(jj) * wr + a] = P[size_t(rs[jj] + a) * nc + jj];
        ptabs[key] = {reg_const(c, c->mem.upload(rw, s), rw.size()), c->mem.upload(rs, s),
                      reg_const(c, c->mem.upload(pw, s), pw.size()), c->mem.upload(ps, s),
                      (void*)(intptr_t)wr, (void*)(intptr_t)wp};
        pstart_h[key] = {rs, ps};
      }
      return ptabs[key];
    };
    std::vector<XferT<double>> rp[3], pp[3];
    int64_t tAsz = 0, tBsz = 0;
    for (int k = 0; k < K; ++k) {
      const PatchDev &Pf = L.pd_h[k], &Pc = C.pd_h[k];
      // restriction: dims go fine -> coarse one at a time: shape after pass j has coarse
      // sizes in directions <= j
      int shp[3];
      for (int j = 0; j < 3; ++j) shp[j] = Pf.n[j];
      int64_t in_off = Pf.off;
      for (int j = 0; j < d; ++j) {
        auto& tb = tables(Pc.m[j], Pc.p[j]);
        XferT<double> x{};
        x.outer = 1;
        for (int i = 0; i < j; ++i) x.outer *= shp[i];
        x.inner = 1;
        for (int i = j + 1; i < d; ++i) x.inner *= shp[i];
        x.nin = Pf.n[j];
        x.nout = Pc.n[j];
        x.width = int((intptr_t)tb[4]);
        x.wt = (const double*)tb[0];
        x.st = (const int*)tb[1];
        x.in_off = in_off;
        int64_t outsz = int64_t(x.outer) * x.nout * x.inner;
        if (j == d - 1) x.out_off = Pc.off;
        else if (j % 2 == 0) { x.out_off = tAsz; }
        else { x.out_off = tBsz; }
        rp[j].push_back(x);
        L.rmax[j] = std::max(L.rmax[j], outsz);
        shp[j] = Pc.n[j];
        in_off = x.out_off;
        L.xfer_flops += 2.0 * double(outsz) * x.width;
        L.xfer_bytes += 8.0 * double(outsz);
        if (j < d - 1) { if (j % 2 == 0) tAsz += outsz; else tBsz += outsz; }
      }
    }
    int64_t rA = tAsz, rB = tBsz;
    tAsz = tBsz = 0;
    for (int k = 0; k < K; ++k) {
      const PatchDev &Pf = L.pd_h[k], &Pc = C.pd_h[k];
      int shp[3];
      for (int j = 0; j < 3; ++j) shp[j] = Pc.n[j];
      int64_t in_off = Pc.off;
      for (int j = 0; j < d; ++j) {
        auto& tb = tables(Pc.m[j], Pc.p[j]);
        XferT<double> x{};
        x.outer = 1;
        for (int i = 0; i < j; ++i) x.outer *= shp[i];
        x.inner = 1;
        for (int i = j + 1; i < d; ++i) x.inner *= shp[i];
        x.nin = Pc.n[j];
        x.nout = Pf.n[j];
        x.width = int((intptr_t)tb[5]);
        x.wt = (const double*)tb[2];
        x.st = (const int*)tb[3];
        x.in_off = in_off;
        int64_t outsz = int64_t(x.outer) * x.nout * x.inner;
        if (j == d - 1) x.out_off = Pf.off;
        else if (j % 2 == 0) x.out_off = tAsz;
        else x.out_off = tBsz;
        pp[j].push_back(x);
        L.pmax[j] = std::max(L.pmax[j], outsz);
        shp[j] = Pf.n[j];
        in_off = x.out_off;
        L.xfer_flops += 2.0 * double(outsz) * x.width;
        L.xfer_bytes += 8.0 * double(outsz);
        if (j < d - 1) { if (j % 2 == 0) tAsz += outsz; else tBsz += outsz; }
      }
    }
    int64_t na = std::max(rA, tAsz), nb2 = std::max(rB, tBsz);
    L.n64.tA = reg_work(c, c->mem.alloc<double>(na), na);
    L.n64.tB = reg_work(c, c->mem.alloc<double>(nb2), nb2);
    for (int j = 0; j < d; ++j) {
      L.rp_h[j] = rp[j];
      L.pp_h[j] = pp[j];
      L.n64.rpass[j] = c->mem.upload(rp[j], s);
      L.n64.ppass[j] = c->mem.upload(pp[j], s);
    }
    if (d == 2) {
      // both passes in one launch; each block's input columns must fit its shared buffer
      // (2 x 32 + width): checked on the start tables
      auto fits = [](const std::vector<int>& st, int nout, int width) {
        for (int o = 0; o < nout; o += 32) {
          const int e = std::min(o + 32, nout) - 1;
          if (st[e] + width - st[o] > 64 + width) return false;
        }
        return true;
      };
      bool ok = true;
      std::vector<Xfer2T<double>> r2, p2;
      for (int k = 0; k < K; ++k) {
        const PatchDev &Pf = L.pd_h[k], &Pc = C.pd_h[k];
        auto& t0 = tables(Pc.m[0], Pc.p[0]);
        auto& t1 = tables(Pc.m[1], Pc.p[1]);
        const auto& h1 = pstart_h[std::make_tuple(Pc.m[1], Pc.p[1])];
        const int wr0 = int((intptr_t)t0[4]), wr1 = int((intptr_t)t1[4]);
        const int wp0 = int((intptr_t)t0[5]), wp1 = int((intptr_t)t1[5]);
        ok = ok && fits(h1.first, Pc.n[1], wr1) && fits(h1.second, Pf.n[1], wp1);
        r2.push_back(Xfer2T<double>{Pf.off, Pc.off, Pf.n[0], Pf.n[1], Pc.n[0], Pc.n[1], (const double*)t0[0],
                                    (const double*)t1[0], (const int*)t0[1], (const int*)t1[1], wr0, wr1});
        p2.push_back(Xfer2T<double>{Pc.off, Pf.off, Pc.n[0], Pc.n[1], Pf.n[0], Pf.n[1], (const double*)t0[2],
                                    (const double*)t1[2], (const int*)t0[3], (const int*)t1[3], wp0, wp1});
        L.x2_rout0 = std::max(L.x2_rout0, Pc.n[0]);
        L.x2_rout1 = std::max(L.x2_rout1, Pc.n[1]);
        L.x2_pout0 = std::max(L.x2_pout0, Pf.n[0]);
        L.x2_pout1 = std::max(L.x2_pout1, Pf.n[1]);
        L.x2_rw1 = std::max(L.x2_rw1, wr1);
        L.x2_pw1 = std::max(L.x2_pw1, wp1);
      }
      if (ok) {
        L.r2_h = r2;
        L.p2_h = p2;
        L.n64.r2 = c->mem.upload(r2, s);
        L.n64.p2 = c->mem.upload(p2, s);
      }
    }
  }
  bind_tc<double>(c);
  bind_stack(c);
  // coarse solver: dense A_0 from the level-0 bands, Cholesky, explicit inverse
  Level& L0 = c->lv[0];
  const LevelTopo& T0 = L0.topo;
  int64_t N0 = T0.N;
  if (N0 > 20000) throw Fail{IGAMG_ERR_UNSUPPORTED, "coarse problem too large for the dense solver"};
  int64_t bsz = 0;
  for (int k = 0; k < K; ++k) {
    int64_t nb = 1;
    for (int j = 0; j < d; ++j) nb *= 2 * L0.pd_h[k].p[j] + 1;
    bsz = std::max(bsz, L0.pd_h[k].band_off + (T0.off[k + 1] - T0.off[k]) * nb);
  }
  std::vector<double> hb(bsz);
  CK(cudaMemcpyAsync(hb.data(), L0.band, bsz * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  Mat A0(size_t(N0) * N0, 0.0);
  for (int k = 0; k < K; ++k) {
    const PatchDev& P = L0.pd_h[k];
    int64_t nn = T0.off[k + 1] - T0.off[k];
    int W[3] = {1, 1, 1}, nt = 1;
    for (int j = 0; j < d; ++j) { W[j] = 2 * P.p[j] + 1; nt *= W[j]; }
    for (int64_t li = 0; li < nn; ++li) {
      int64_t gi = T0.l2g[P.off + li];
      if (gi < 0) continue;
      int ii[3] = {0, 0, 0};
      int64_t r = li;
      for (int j = d - 1; j >= 0; --j) { ii[j] = int(r % P.n[j]); r /= P.n[j]; }
      for (int t = 0; t < nt; ++t) {
        int tt[3] = {0, 0, 0}, rr = t;
        for (int j = d - 1; j >= 0; --j) { tt[j] = rr % W[j]; rr /= W[j]; }
        int64_t lj = 0;
        bool ok = true;
        for (int j = 0; j < d; ++j) {
          int jj = ii[j] + tt[j] - P.p[j];
          ok = ok && jj >= 0 && jj < P.n[j];
          lj = lj * P.n[j] + jj;
        }
        if (!ok) continue;
        int64_t gj = T0.l2g[P.off + lj];
        if (gj < 0) continue;
        A0[size_t(gi) * N0 + gj] += hb[P.band_off + int64_t(t) * nn + li];
      }
    }
  }
  Mat Lc = A0;
  if (!cholesky(int(N0), Lc)) throw Fail{IGAMG_ERR_NUMERIC, "coarse Cholesky failed (A_0 not SPD)"};
  Mat inv(size_t(N0) * N0, 0.0);
  for (int64_t i = 0; i < N0; ++i) inv[size_t(i) * N0 + i] = 1.0;
  cholesky_solve_many(int(N0), Lc, inv, int(N0));
  c->N0 = N0;
  c->A0inv = c->mem.upload(inv, s);
  // PCG vectors
  const Level& Lf = c->lv.back();
  int64_t Tf = Lf.topo.T;
  c->X = c->mem.alloc<double>(Tf);
  c->Pv = c->mem.alloc<double>(Tf);
  c->W = c->mem.alloc<double>(Tf);
  c->Bt = c->mem.alloc<double>(Tf);
  c->Rr = c->mem.alloc<double>(Tf);
  int64_t gmaxN = 0;
  for (auto& L : c->lv) gmaxN = std::max(gmaxN, L.topo.N);
  c->gtmp = c->mem.alloc<double>(gmaxN);
  c->partials = c->mem.alloc<double>(RED_BLOCKS);
  c->tc_err = c->mem.alloc<int>(1);
  CK(cudaMemsetAsync(c->tc_err, 0, sizeof(int), s));
  c->scal = c->mem.alloc<double>(16);
  CK(cudaMemsetAsync(c->scal, 0, 16 * sizeof(double), s));
  CK(cudaMallocHost(&c->h_scal, 16 * sizeof(double)));
  CK(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------- cycle

template <class T>
void residual(igamg_ctx* c, int l, const T* f, const T* u, T* r, bool krylov = false) {
  Level& L = c->lv[l];
  Num<T>& N = num<T>(L);
  const bool bf = N.bf16 && !krylov;
  double bb = bf ? 0.25 : double(sizeof(T)) / 8.0;  // band bytes relative to FP64
  if (L.kron) {
    ProfScope ps(c, CLS_APPLY, L.apply_flops, (double(sizeof(T)) * (f ? 3 : 2) + 1.0) * L.topo.T);
    CK(launch_kron_apply_2d<T>(c->stream, N.kd, c->pd.K, L.max_n[0], L.max_n[1], L.max_p, L.active, u, f, r));
    return;
  }
  ProfScope ps(c, CLS_APPLY, L.apply_flops, L.band_bytes * bb + double(sizeof(T)) * L.topo.T * (f ? 3 : 2));
  if (bf) {
    if constexpr (std::is_same<T, float>::value) {
      const __nv_bfloat16* band = static_cast<const __nv_bfloat16*>(N.band);
      if (c->pd.dim == 2)
        CK((launch_band_apply_2d<float, __nv_bfloat16>(c->stream, L.pd, c->pd.K, L.max_n[0], L.max_n[1], L.max_p,
                                                         band, u, f, r, L.uniform_p)));
      else if (N.pd_pair)
        CK(launch_band_apply_3d_pair<__nv_bfloat16>(c->stream, N.pd_pair, c->pd.K, L.max_n, L.uniform_p, band, u, f,
                                                    r));
      else
        CK((launch_band_apply_3d<float, __nv_bfloat16>(c->stream, L.pd, c->pd.K, L.max_n, L.max_p, band, u, f, r,
                                                         L.uniform_p)));
    }
    return;
  }
  const T* band = krylov ? N.band_op : static_cast<const T*>(N.band);
  if constexpr (std::is_same<T, float>::value) {
    if (c->pd.dim == 3 && N.pd_blk) {  // FP32 bands in the tap-blocked layout
      CK(launch_band_apply_3d_blk(c->stream, N.pd_blk, c->pd.K, L.max_n, L.uniform_p, band, u, f, r));
      return;
    }
  }
  if (c->pd.dim == 2)
    CK((launch_band_apply_2d<T, T>(c->stream, L.pd, c->pd.K, L.max_n[0], L.max_n[1], L.max_p, band, u, f, r,
                                   L.uniform_p)));
  else
    CK((launch_band_apply_3d<T, T>(c->stream, L.pd, c->pd.K, L.max_n, L.max_p, band, u, f, r, L.uniform_p)));
}

// Makes c->stream another stream for the scope (launch helpers use c->stream).
struct OnStream {
  igamg_ctx* c;
  cudaStream_t prev;
  OnStream(igamg_ctx* c_, cudaStream_t s) : c(c_), prev(c_->stream) { c->stream = s; }
  ~OnStream() { c->stream = prev; }
};

// Interface pieces of a smoothing step: edges (1D FD), faces (2D FD) and vertices, with the
// gather of the copies before and the scatter after (Sigma of Eq. ops6).
template <class T>
void smooth_interface(igamg_ctx* c, Level& L, Num<T>& N, const T* v, double tau, bool add) {
  if (N.i3_ok) {  // small 3D level: gather, face and edge FD, vertices and scatter in one launch
    ProfScope ps(c, CLS_IFACE, N.face0.flops + N.face1.flops + N.face2.flops + N.face3.flops + N.edgeA.flops +
                                   N.edgeB.flops + 2.0 * L.n_if,
                 4.0 * sizeof(T) * L.n_if);
    CK(launch_iface3_small<T>(c->stream, N.i3s, v, T(tau), add ? 1 : 0));
    return;
  }
  {
    ProfScope ps(c, CLS_IFACE, 0.0, 2.0 * sizeof(T) * L.n_if);
    CK(launch_iface_gather<T>(c->stream, L.n_if, L.if_ptr, L.if_idx, v, N.G));
  }
  run_gemm(c, N.edgeA, false, false, EPI_COLSCALE, 1.0, CLS_IFACE);
  run_gemm(c, N.edgeB, false, true, EPI_STORE, 1.0, CLS_IFACE);
  if (N.use_tc && N.tq0.batch) {  // faces follow the interiors' engine
    run_tc(c, N.tq0, EPI_STORE, 1.0, CLS_IFACE);
    run_tc(c, N.tq1, EPI_MUL, 1.0, CLS_IFACE);
    run_tc(c, N.tq2, EPI_STORE, 1.0, CLS_IFACE);
    run_tc(c, N.tq3, EPI_STORE, 1.0, CLS_IFACE);
  } else if (N.fm[0].batch) {
    run_mode(c, N.fm[0], N.face0, EPI_STORE, CLS_IFACE);
    run_mode(c, N.fm[1], N.face1, EPI_MUL, CLS_IFACE);
    run_mode(c, N.fm[2], N.face2, EPI_STORE, CLS_IFACE);
    run_mode(c, N.fm[3], N.face3, EPI_STORE, CLS_IFACE);
  } else {
    run_gemm(c, N.face0, true, false, EPI_STORE, 1.0, CLS_IFACE);
    run_gemm(c, N.face1, false, false, EPI_MUL, 1.0, CLS_IFACE);
    run_gemm(c, N.face2, false, false, EPI_STORE, 1.0, CLS_IFACE);
    run_gemm(c, N.face3, false, true, EPI_STORE, 1.0, CLS_IFACE);
  }
  {
    ProfScope ps(c, CLS_IFACE, 2.0 * L.n_if, 3.0 * sizeof(T) * L.n_if);
    CK(launch_iface_scatter<T>(c->stream, L.n_if, L.if_ptr, L.if_idx, N.Z, N.G, N.vscale, T(tau), add ? 1 : 0, N.U));
  }
}

// u (=|+=) tau L^{-1} v for a distributed v (F or R of the level): patch interiors by
// fast diagonalisation, faces by their 2D and edges by their 1D fast diagonalisation,
// vertices by scaling (Eq. additive; the pieces are disjoint, so the sum is a set of
// independent blocks).
template <class T>
void smooth(igamg_ctx* c, int l, bool from_F, bool add) {
  Level& L = c->lv[l];
  Num<T>& N = num<T>(L);
  const T* v = from_F ? N.F : N.R;
  double tau = c->opt.tau;
  int epi = add ? EPI_ADD : EPI_ASSIGN;
  if (c->pd.dim == 2 && N.use_fused && L.small_ok) {  // interiors, edges and vertices: one launch
    ProfScope ps(c, CLS_FD, N.ssmall_flops, 0.0);
    CK(launch_smooth_small<T>(c->stream, N.ssmall, from_F ? 1 : 0, T(tau), add ? 1 : 0));
    return;
  }
  // the interface pieces on the side stream, concurrently with the interiors below
  const bool fork = L.n_if > 0 && c->side;
  if (fork) {
    CK(cudaEventRecord(c->fork_ev, c->stream));
    CK(cudaStreamWaitEvent(c->side, c->fork_ev, 0));
    OnStream os(c, c->side);
    smooth_interface<T>(c, L, N, v, tau, add);
  }
  if (c->pd.dim == 2 && N.use_rows) {
    for (int pass = 1; pass <= 2; ++pass) {
      ProfScope ps(c, CLS_FD, 2.0 * N.st1.flops, 0.0);  // two of the four products per pass
      CK(launch_fd_rows<T>(c->stream, N.frows, N.nfrows, N.frows_n0, N.frows_n1, pass, from_F ? 1 : 0, T(tau),
                           add ? 1 : 0));
    }
  } else if (c->pd.dim == 2 && N.use_fused) {
    ProfScope ps(c, CLS_FD, N.fsmall_flops, 0.0);
    CK(launch_fd_small<T>(c->stream, N.fsmall, N.nfsmall, from_F ? 1 : 0, T(tau), add ? 1 : 0));
  } else if (c->pd.dim == 2 && N.use_tc) {
    bool stacked = false;
    if constexpr (std::is_same<T, double>::value) {
      if (N.sk1.batch) {  // FP64: the fibre-major stacked stages
        run_stack(c, from_F ? N.sk0F : N.sk0R, EPI_STORE, 1.0);
        run_stack(c, N.sk1, EPI_MUL, 1.0);
        run_stack(c, N.sk2, EPI_STORE, 1.0);
        run_stack(c, N.sk3, epi, tau);
        stacked = true;
      }
    }
    if (!stacked) {
      run_tc(c, from_F ? N.tc0F : N.tc0R, EPI_STORE, 1.0);
      run_tc(c, N.tc1, EPI_MUL, 1.0);
      run_tc(c, N.tc2, EPI_STORE, 1.0);
      run_tc(c, N.tc3, epi, tau);
    }
  } else if (c->pd.dim == 2) {
    run_gemm(c, from_F ? N.st0F : N.st0R, true, false, EPI_STORE, 1.0, CLS_FD);
    run_gemm(c, N.st1, false, false, EPI_MUL, 1.0, CLS_FD);
    run_gemm(c, N.st2, false, false, EPI_STORE, 1.0, CLS_FD);
    run_gemm(c, N.st3, false, true, epi, tau, CLS_FD);
  } else if (L.nbox && N.fd3 && !N.use_tc) {  // small interiors: one launch, same arithmetic
    const double fl = N.m0f.flops + N.m1f.flops + N.m2f.flops + N.m0b.flops + N.m1b.flops + N.m2b.flops;
    ProfScope ps(c, CLS_FD, fl, 2.0 * sizeof(T) * L.box_vol);
    CK(launch_fd3_small<T>(c->stream, N.fd3, N.nfd3, v, N.U, T(tau), add ? 1 : 0));
  } else if (L.nbox) {
    {
      ProfScope ps(c, CLS_FD, 0.0, 2.0 * sizeof(T) * L.max_box * L.nbox);
      CK(launch_box_copy<T>(c->stream, L.boxes, L.nbox, L.max_box, v, N.cX, 1, T(1), 0));
    }
    if (N.use_tc) {
      run_tc(c, N.tc0F, EPI_STORE, 1.0);
      run_tc(c, N.tc1, EPI_STORE, 1.0);
      run_tc(c, N.tc2, EPI_MUL, 1.0);
      run_tc(c, N.tc3, EPI_STORE, 1.0);
      run_tc(c, N.tc4, EPI_STORE, 1.0);
      run_tc(c, N.tc5, EPI_STORE, 1.0);
    } else if (N.md[0].batch) {
      run_mode(c, N.md[0], N.m0f, EPI_STORE);
      run_mode(c, N.md[1], N.m1f, EPI_STORE);
      run_mode(c, N.md[2], N.m2f, EPI_MUL);
      run_mode(c, N.md[3], N.m0b, EPI_STORE);
      run_mode(c, N.md[4], N.m1b, EPI_STORE);
      run_mode(c, N.md[5], N.m2b, EPI_STORE);
    } else {
      run_gemm(c, N.m0f, true, false, EPI_STORE, 1.0, CLS_FD);
      run_gemm(c, N.m1f, true, false, EPI_STORE, 1.0, CLS_FD);
      run_gemm(c, N.m2f, false, false, EPI_MUL, 1.0, CLS_FD);
      run_gemm(c, N.m0b, false, false, EPI_STORE, 1.0, CLS_FD);
      run_gemm(c, N.m1b, false, false, EPI_STORE, 1.0, CLS_FD);
      run_gemm(c, N.m2b, false, true, EPI_STORE, 1.0, CLS_FD);
    }
    ProfScope ps(c, CLS_FD, 0.0, 2.0 * sizeof(T) * L.max_box * L.nbox);
    CK(launch_box_copy<T>(c->stream, L.boxes, L.nbox, L.max_box, N.cX, N.U, 0, T(tau), add ? 1 : 0));
  }
  if (fork) {
    CK(cudaEventRecord(c->join_ev, c->side));
    CK(cudaStreamWaitEvent(c->stream, c->join_ev, 0));
  } else if (L.n_if > 0) {
    smooth_interface<T>(c, L, N, v, tau, add);
  }
}

// r_{l-1} = P_l^T r_l (distributed -> distributed), one direction at a time.
template <class T>
void restrict_to_coarse(igamg_ctx* c, int l, const T* rf) {
  Level& L = c->lv[l];
  Level& C = c->lv[l - 1];
  Num<T>& N = num<T>(L);
  const int d = c->pd.dim, K = c->pd.K;
  if (N.r2) {
    ProfScope pr(c, CLS_TRANSFER, L.xfer_flops / 3, L.xfer_bytes / 3 * sizeof(T) / 8.0, 1);
    CK(launch_transfer_2d<T>(c->stream, N.r2, K, L.x2_rout0, L.x2_rout1, L.x2_rw1, rf, num<T>(C).F, 0, C.l2g));
    return;
  }
  ProfScope pr(c, CLS_TRANSFER, L.xfer_flops / 3, L.xfer_bytes / 3 * sizeof(T) / 8.0, d);
  const T* in = rf;
  for (int j = 0; j < d; ++j) {
    T* out = j == d - 1 ? num<T>(C).F : (j % 2 == 0 ? N.tA : N.tB);
    CK(launch_transfer_1d<T>(c->stream, N.rpass[j], K, L.rmax[j], in, out, 0, j == d - 1 ? C.l2g : nullptr));
    in = out;
  }
}

// u_l += P_l u_{l-1} (accumulated -> accumulated).
template <class T>
void prolong_add(igamg_ctx* c, int l) {
  Level& L = c->lv[l];
  Level& C = c->lv[l - 1];
  Num<T>& N = num<T>(L);
  const int d = c->pd.dim, K = c->pd.K;
  if (N.p2) {
    ProfScope pp(c, CLS_TRANSFER, 2 * L.xfer_flops / 3, 2 * L.xfer_bytes / 3 * sizeof(T) / 8.0, 1);
    CK(launch_transfer_2d<T>(c->stream, N.p2, K, L.x2_pout0, L.x2_pout1, L.x2_pw1, num<T>(C).U, N.U, 1, nullptr));
    return;
  }
  ProfScope pp(c, CLS_TRANSFER, 2 * L.xfer_flops / 3, 2 * L.xfer_bytes / 3 * sizeof(T) / 8.0, d);
  const T* in = num<T>(C).U;
  for (int j = 0; j < d; ++j) {
    T* out = j == d - 1 ? N.U : (j % 2 == 0 ? N.tA : N.tB);
    CK(launch_transfer_1d<T>(c->stream, N.ppass[j], K, L.pmax[j], in, out, j == d - 1 ? 1 : 0, nullptr));
    in = out;
  }
}

// Exact coarsest solve, always in FP64 (the inverse is applied in FP64 to the gathered
// coarse residual whatever the vector precision).
template <class T>
void coarse_solve(igamg_ctx* c) {
  Level& L0 = c->lv[0];
  ProfScope ps(c, CLS_COARSE, 2.0 * double(c->N0) * c->N0, 8.0 * double(c->N0) * c->N0);
  CK(launch_coarse_solve<T>(c->stream, c->N0, L0.g2t_ptr, L0.g2t, c->A0inv, num<T>(L0).F, num<T>(L0).U));
}

// Algorithm 1 on level l >= 1: f = F_l (distributed), u = U_l (accumulated).
template <class T>
void multigrid(igamg_ctx* c, int l, bool zero_init) {
  Level& L = c->lv[l];
  Num<T>& N = num<T>(L);
  const int nu = c->opt.nu, mu = c->opt.mu;
  for (int i = 0; i < nu; ++i) {
    if (zero_init && i == 0) {
      smooth<T>(c, l, true, false);  // u = 0: the residual is f itself
    } else {
      residual<T>(c, l, N.F, N.U, N.R);
      smooth<T>(c, l, false, true);
    }
  }
  residual<T>(c, l, N.F, N.U, N.R);
  restrict_to_coarse<T>(c, l, N.R);
  if (l == 1) {
    coarse_solve<T>(c);
  } else {
    for (int j = 0; j < mu; ++j) multigrid<T>(c, l - 1, j == 0);
  }
  prolong_add<T>(c, l);
  for (int i = 0; i < nu; ++i) {
    residual<T>(c, l, N.F, N.U, N.R);
    smooth<T>(c, l, false, true);
  }
}

// z = U_L = Multigrid(L, 0, F_L)
template <class T>
void precondition(igamg_ctx* c) {
  int Lf = int(c->lv.size()) - 1;
  if (Lf == 0) coarse_solve<T>(c);
  else multigrid<T>(c, Lf, true);
}

int level_index(const igamg_ctx* c, int level) {
  int NL = int(c->lv.size());
  if (level == -1) return NL - 1;
  if (level < 0 || level >= NL) throw Fail{IGAMG_ERR_ARG, "level out of range"};
  return level;
}

void to_dist(igamg_ctx* c, int l, const double* xg, double* xt) {
  Level& L = c->lv[l];
  ProfScope ps(c, CLS_VECTOR, 0.0, 16.0 * L.topo.N);
  CK(cudaMemsetAsync(xt, 0, L.topo.T * sizeof(double), c->stream));
  CK(launch_global_to_tile<double>(c->stream, L.topo.N, L.g2t_ptr, L.g2t, xg, xt, 1));
}
void to_acc(igamg_ctx* c, int l, const double* xg, double* xt) {
  Level& L = c->lv[l];
  ProfScope ps(c, CLS_VECTOR, 0.0, 16.0 * L.topo.N);
  CK(cudaMemsetAsync(xt, 0, L.topo.T * sizeof(double), c->stream));
  CK(launch_global_to_tile<double>(c->stream, L.topo.N, L.g2t_ptr, L.g2t, xg, xt, 0));
}
void from_acc(igamg_ctx* c, int l, const double* xt, double* xg) {
  Level& L = c->lv[l];
  ProfScope ps(c, CLS_VECTOR, 0.0, 16.0 * L.topo.N);
  CK(launch_tile_to_global<double>(c->stream, L.topo.N, L.g2t_ptr, L.g2t, xt, xg, 0));
}
void from_dist(igamg_ctx* c, int l, const double* xt, double* xg) {
  Level& L = c->lv[l];
  ProfScope ps(c, CLS_VECTOR, 0.0, 16.0 * L.topo.N);
  CK(launch_tile_to_global<double>(c->stream, L.topo.N, L.g2t_ptr, L.g2t, xt, xg, 1));
}

double read_scalar(igamg_ctx* c, int i) {
  CK(cudaMemcpyAsync(c->h_scal + i, c->scal + i, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (c->prof) prof_collect(c);
  return c->h_scal[i];
}

template <class T>
void vdot(igamg_ctx* c, const T* a, const T* b, int64_t n, double* out) {
  ProfScope ps(c, CLS_VECTOR, 2.0 * n, 2.0 * sizeof(T) * n, 2);
  CK(launch_dot<T>(c->stream, a, b, n, c->partials, out));
}

template <class T>
void vnorm_dist(igamg_ctx* c, int l, const T* v, double* out) {
  Level& L = c->lv[l];
  ProfScope ps(c, CLS_VECTOR, 2.0 * L.topo.N, double(sizeof(T)) * L.topo.T, 2);
  CK(launch_norm2_dist<T>(c->stream, L.topo.N, L.g2t_ptr, L.g2t, v, c->partials, out));
}

// PCG (Sec. 4) in precision T on the tile layout of the finest level: r = F_L and w
// distributed; x, z = U_L, p accumulated.  The residual r must be set on entry, x is
// zeroed.  Stops when ||r|| <= tol * ||r_0|| (tol > 0) or after max_iter iterations.
// scal: 0 rz, 1 pw, 2 rz_new, 3 rr.  Returns the iterations and the final ratio.
template <class T>
int pcg_core(igamg_ctx* c, T* x, T* p, T* w, double tol, int max_iter, double* rel_out, bool* stalled) {
  const int Lf = int(c->lv.size()) - 1;
  Level& L = c->lv[Lf];
  Num<T>& N = num<T>(L);
  const int64_t T_ = L.topo.T;
  const bool flexible = sizeof(T) < 8;  // low-precision cycle: Polak-Ribiere beta
  cudaStream_t s = c->stream;
  CK(cudaMemsetAsync(x, 0, T_ * sizeof(T), s));
  vnorm_dist<T>(c, Lf, N.F, c->scal + 3);
  double rr0 = read_scalar(c, 3);
  if (!std::isfinite(rr0)) throw Fail{IGAMG_ERR_NUMERIC, "non-finite initial residual"};
  *rel_out = 0.0;
  *stalled = false;
  if (rr0 == 0.0) return 0;
  int it = 0;
  double rel = 1.0;
  std::vector<double> hist{1.0};
  precondition<T>(c);
  CK(cudaMemcpyAsync(p, N.U, T_ * sizeof(T), cudaMemcpyDeviceToDevice, s));
  if (flexible) CK(cudaMemcpyAsync(c->Zold32, N.U, T_ * sizeof(T), cudaMemcpyDeviceToDevice, s));
  vdot<T>(c, N.F, N.U, T_, c->scal + 0);
  // one PCG step after the convergence check: z = B r, beta, p, w = A p, alpha, x, r, ||r||
  auto body = [&](bool with_precondition) {
    cudaStream_t s = c->stream;  // the capture stream while a graph is recorded
    if (with_precondition) {
      precondition<T>(c);
      vdot<T>(c, N.F, N.U, T_, c->scal + 2);
      if (flexible) {
        if constexpr (std::is_same<T, float>::value) {
          vdot<T>(c, N.F, c->Zold32, T_, c->scal + 4);
          ProfScope ps(c, CLS_VECTOR, 2.0 * T_, 4.0 * sizeof(T) * T_, 2);
          CK(launch_fcg_p(s, T_, c->scal, p, N.U, c->Zold32));
        }
      } else {
        ProfScope ps(c, CLS_VECTOR, 2.0 * T_, 3.0 * sizeof(T) * T_, 2);
        CK(launch_pcg_p<T>(s, T_, c->scal, p, N.U));
      }
    }
    residual<T>(c, Lf, nullptr, p, w, true);
    if (flexible) {  // keep the low-precision residual free of cancellation between copies
      ProfScope ps(c, CLS_VECTOR, 0.0, 3.0 * sizeof(T) * L.n_if);
      CK(launch_canonicalize<T>(s, L.n_if, L.if_ptr, L.if_idx, w));
    }
    vdot<T>(c, p, w, T_, c->scal + 1);
    {
      ProfScope ps(c, CLS_VECTOR, 4.0 * T_, 6.0 * sizeof(T) * T_);
      CK(launch_pcg_xr<T>(s, T_, c->scal, x, N.F, p, w));
    }
    vnorm_dist<T>(c, Lf, N.F, c->scal + 3);
  };
  const int gi = sizeof(T) == 8 ? 0 : 1;
  while (!(tol > 0 && rel <= tol) && it < max_iter) {
    if (it == 0) {
      body(false);
    } else if (c->opt.graphs) {
      // the step touches fixed buffers only: capture it once, replay it every iteration
      graph_run(c, gi, [&] { body(true); });
    } else {
      body(true);
    }
    ++it;
    double rr = read_scalar(c, 3);
    if (!std::isfinite(rr)) throw Fail{IGAMG_ERR_NUMERIC, "non-finite residual in PCG"};
    rel = std::sqrt(rr / rr0);
    hist.push_back(rel);
    // low precision: stop once the last 8 iterations gained less than a factor 2
    if (flexible && it >= 8 && rel > 0.5 * hist[it - 8]) {
      *stalled = true;
      break;
    }
  }
  *rel_out = rel;
  return it;
}

void check_tc(igamg_ctx* c) {
  int e = 0;
  CK(cudaMemcpy(&e, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) throw Fail{IGAMG_ERR_TIMEOUT, "a tensor-core contraction timed out waiting for its MMAs"};
}

// FP64 PCG from x (global) with rhs b (global).
igamg_status pcg(igamg_ctx* c, const double* b, double* x, double tol, igamg_result* res) {
  double t0 = now_ms();
  const int Lf = int(c->lv.size()) - 1;
  Level& L = c->lv[Lf];
  const int64_t T = L.topo.T;
  cudaStream_t s = c->stream;
  to_dist(c, Lf, b, c->Bt);
  to_acc(c, Lf, x, c->X);
  // solve A d = b - A x0 from d = 0, then x = x0 + d (Rr holds x0)
  residual<double>(c, Lf, c->Bt, c->X, L.n64.F, true);
  CK(cudaMemcpyAsync(c->Rr, c->X, T * sizeof(double), cudaMemcpyDeviceToDevice, s));
  double rel = 0.0;
  bool stalled = false;
  int it = pcg_core<double>(c, c->X, c->Pv, c->W, tol, c->opt.max_iter, &rel, &stalled);
  CK(launch_axpby(s, T, 1.0, c->Rr, 1.0, c->X));
  from_acc(c, Lf, c->X, x);
  CK(cudaStreamSynchronize(s));
  check_tc(c);
  if (c->prof) prof_collect(c);
  if (res) {
    res->iters = it;
    res->outer_iters = 1;
    res->relres = rel;
    res->t_setup_ms = c->t_setup_ms;
    res->t_assemble_ms = c->t_assemble_ms;
    res->t_solve_ms = now_ms() - t0;
  }
  return (tol > 0 && rel > tol) ? IGAMG_ERR_NOT_CONVERGED : IGAMG_OK;
}

// FP64 iterative refinement around a low-precision PCG (the precision variant):
// r = b - A x in FP64; the inner PCG (FP32 vectors, FP32 or BF16 bands, FP32 smoother
// contractions, FP64 coarse solve) reduces the scaled residual by inner_tol; x += d.
igamg_status pcg_refined(igamg_ctx* c, const double* b, double* x, double tol, igamg_result* res) {
  double t0 = now_ms();
  const int Lf = int(c->lv.size()) - 1;
  Level& L = c->lv[Lf];
  const int64_t T = L.topo.T;
  cudaStream_t s = c->stream;
  to_dist(c, Lf, b, c->Bt);
  to_acc(c, Lf, x, c->X);
  int total = 0, outer = 0;
  double rel = 1.0, rr0 = -1.0;
  igamg_status st = IGAMG_OK;
  while (true) {
    residual<double>(c, Lf, c->Bt, c->X, c->Rr, true);
    vnorm_dist<double>(c, Lf, c->Rr, c->scal + 3);
    double rr = read_scalar(c, 3);
    if (!std::isfinite(rr)) throw Fail{IGAMG_ERR_NUMERIC, "non-finite residual in refinement"};
    if (rr0 < 0) rr0 = rr;
    rel = rr0 > 0 ? std::sqrt(rr / rr0) : 0.0;
    if (rr0 == 0.0 || (tol > 0 && rel <= tol)) break;
    if (total >= c->opt.max_iter || outer >= 60) { st = tol > 0 ? IGAMG_ERR_NOT_CONVERGED : IGAMG_OK; break; }
    // canonical distributed form, then the scaled FP32 residual (norm 1)
    CK(launch_canonicalize<double>(s, L.n_if, L.if_ptr, L.if_idx, c->Rr));
    double scale = 1.0 / std::sqrt(rr);
    CK(launch_convert_f64_f32(s, T, c->Rr, scale, L.n32.F));
    double irel = 0.0;
    bool stalled = false;
    int it = pcg_core<float>(c, c->X32, c->P32, c->W32, c->opt.inner_tol, c->opt.max_iter - total, &irel, &stalled);
    total += it;
    ++outer;
    if (c->verbose)
      std::fprintf(stderr, "[igamg] refinement %d: ||r||/||r0|| = %.3e, inner %d its, inner reduction %.3e%s\n", outer,
                   rel, it, irel, stalled ? " (stalled)" : "");
    CK(launch_add_scaled_f32(s, T, c->X32, 1.0 / scale, c->X));
    if (it == 0) { st = IGAMG_ERR_NUMERIC; break; }
  }
  from_acc(c, Lf, c->X, x);
  CK(cudaStreamSynchronize(s));
  check_tc(c);
  if (c->prof) prof_collect(c);
  if (res) {
    res->iters = total;
    res->outer_iters = outer;
    res->relres = rel;
    res->t_setup_ms = c->t_setup_ms;
    res->t_assemble_ms = c->t_assemble_ms;
    res->t_solve_ms = now_ms() - t0;
  }
  return st;
}

// ---------------------------------------------------------------- FD autotuner

// Per level, the patch-interior FD contractions run on the candidate that times fastest on
// this device: the FMA GEMM with an 8R x 8R output tile per block (R = 1, 2, 4) or the
// tensor cores (where their stage sets were built).  A level's choice depends only on its
// interior shapes and degrees, so it is kept process-wide under that signature: later
// contexts with the same shapes (a batch of similar problems) reuse it without timing, and
// two contexts in one process always make the same choice.
struct FdChoice {
  bool tc;
  int R;
};
std::mutex g_tune_mu;
std::map<std::string, FdChoice> g_tune_cache;

std::string fd_signature(const igamg_ctx* c, const Level& L) {
  std::string k = "d" + std::to_string(c->pd.dim) + (L.tc_ok ? "t" : "f") + (L.fused_ok ? "s" : "") + "r";
  for (const Interior& in : L.topo.interiors) {
    k += "|" + std::to_string(c->pd.p[in.k * c->pd.dim]);
    for (int j = 0; j < c->pd.dim; ++j) k += "x" + std::to_string(in.len[j]);
  }
  return k;
}

void apply_choice(Level& L, const FdChoice& ch) {
  Num<double>& N = L.n64;
  N.use_tc = ch.tc && L.tc_ok;
  N.use_fused = ch.R == -1 && L.fused_ok;  // R = -1: the one-block kernel
  N.use_rows = ch.R == -2 && N.nfrows > 0;  // R = -2: the row-block kernel
  for (GemmSet* g : {&N.st0F, &N.st0R, &N.st1, &N.st2, &N.st3, &N.m0f, &N.m1f, &N.m2f, &N.m0b, &N.m1b, &N.m2b})
    g->R = ch.R > 0 ? ch.R : 0;
}

void autotune(igamg_ctx* c) {
  cudaStream_t s = c->stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (int l = 1; l < int(c->lv.size()); ++l) {
    Level& L = c->lv[l];
    if (!L.n64.st0F.batch && !L.n64.m0f.batch) continue;  // no patch interiors on this level
    const std::string key = fd_signature(c, L);
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        apply_choice(L, it->second);
        continue;
      }
    }
    std::vector<FdChoice> cand{{false, 1}, {false, 2}, {false, 4}};
    if (L.tc_ok) cand.push_back({true, 0});
    if (L.fused_ok) cand.push_back({false, -1});
    if (L.n64.nfrows && c->pd.dim == 2) cand.push_back({false, -2});
    FdChoice best{false, 0};
    float best_ms = 1e30f;
    // each candidate: a warm-up, then the best of three timings of two smoothers (the best
    // of several short timings is robust to other work sharing the GPU)
    for (const FdChoice& ch : cand) {
      apply_choice(L, ch);
      smooth<double>(c, l, true, false);
      float ms = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        CK(cudaEventRecord(e0, s));
        for (int r = 0; r < 2; ++r) smooth<double>(c, l, true, false);
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, e0, e1));
        ms = std::min(ms, 1.5f * t);  // per three smoothers, as reported
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = ch;
      }
    }
    if (c->verbose)
      std::fprintf(stderr, "[igamg] autotune level %d: %s R=%d (%.3f ms per smoother)\n", l,
                   best.tc ? "tensor" : best.R == -1 ? "one-block" : best.R == -2 ? "row-block" : "fma", best.R,
                   best_ms / 3);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    // a context that tuned the same signature concurrently may have stored first: use
    // the stored choice, so that every context of the process agrees
    apply_choice(L, g_tune_cache.emplace(key, best).first->second);
  }
  CK(cudaEventDestroy(e0));
  CK(cudaEventDestroy(e1));
  CK(cudaMemsetAsync(c->lv.back().n64.U, 0, c->lv.back().topo.T * sizeof(double), s));
  check_tc(c);
}

// The FP32 twin of a level picks its own engine: FP32 FMA GEMMs and single BF16 tensor-core
// products (one slice pair instead of 28) weigh differently than their FP64 counterparts, so
// the FP64 choice is only the starting point.  Same candidates and timing rule as autotune().
void apply_choice_low(Level& L, const FdChoice& ch) {
  Num<float>& N = L.n32;
  N.use_tc = ch.tc && N.tc1.batch > 0;
  N.use_fused = ch.R == -1 && L.fused_ok;
  N.use_rows = ch.R == -2 && N.nfrows > 0;
  for (GemmSetT<float>* g : {&N.st0F, &N.st0R, &N.st1, &N.st2, &N.st3, &N.m0f, &N.m1f, &N.m2f, &N.m0b, &N.m1b, &N.m2b})
    g->R = ch.R > 0 ? ch.R : 0;
}

void autotune_low(igamg_ctx* c) {
  cudaStream_t s = c->stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (int l = 1; l < int(c->lv.size()); ++l) {
    Level& L = c->lv[l];
    Num<float>& N = L.n32;
    if (!N.st0F.batch && !N.m0f.batch) continue;  // no patch interiors on this level
    const std::string key = fd_signature(c, L) + (c->low_bf16 ? "|bf16" : "|f32");
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        apply_choice_low(L, it->second);
        continue;
      }
    }
    std::vector<FdChoice> cand{{false, 1}, {false, 2}, {false, 4}};
    if (N.tc1.batch) cand.push_back({true, 0});
    if (L.fused_ok) cand.push_back({false, -1});
    if (N.nfrows && c->pd.dim == 2) cand.push_back({false, -2});
    FdChoice best{false, 0};
    float best_ms = 1e30f;
    for (const FdChoice& ch : cand) {
      apply_choice_low(L, ch);
      smooth<float>(c, l, true, false);
      float ms = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        CK(cudaEventRecord(e0, s));
        for (int r = 0; r < 2; ++r) smooth<float>(c, l, true, false);
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, e0, e1));
        ms = std::min(ms, 1.5f * t);
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = ch;
      }
    }
    if (c->verbose)
      std::fprintf(stderr, "[igamg] autotune level %d (%s): %s R=%d (%.3f ms per smoother)\n", l,
                   c->low_bf16 ? "bf16" : "fp32",
                   best.tc ? "tensor" : best.R == -1 ? "one-block" : best.R == -2 ? "row-block" : "fma", best.R,
                   best_ms / 3);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    apply_choice_low(L, g_tune_cache.emplace(key, best).first->second);
  }
  CK(cudaEventDestroy(e0));
  CK(cudaEventDestroy(e1));
  CK(cudaMemsetAsync(c->lv.back().n32.U, 0, c->lv.back().topo.T * sizeof(float), s));
  check_tc(c);
}

// Twins of the FP64 numerics in FP32 (bands in FP32 or BF16): every registered FP64 array
// gets an FP32 copy (constants converted, work buffers allocated) and every FP64
// descriptor is translated pointer by pointer.
void build_low(igamg_ctx* c, bool bf16_bands) {
  cudaStream_t s = c->stream;
  std::vector<std::tuple<double*, int64_t, float*>> tw;
  for (auto& r : c->reg) {
    double* base = std::get<0>(r);
    int64_t n = std::get<1>(r);
    float* f = c->mem.alloc<float>(std::max<int64_t>(n, 1));
    if (std::get<2>(r)) CK(launch_convert_f64_f32(s, n, base, 1.0, f));
    else CK(cudaMemsetAsync(f, 0, std::max<int64_t>(n, 1) * sizeof(float), s));
    tw.emplace_back(base, n, f);
  }
  std::sort(tw.begin(), tw.end(), [](const auto& a, const auto& b) { return std::get<0>(a) < std::get<0>(b); });
  auto tr = [&](const double* p) -> float* {
    if (!p) return nullptr;
    auto it = std::upper_bound(tw.begin(), tw.end(), p,
                               [](const double* q, const auto& e) { return q < std::get<0>(e); });
    if (it == tw.begin()) throw Fail{IGAMG_ERR_NUMERIC, "untracked array in a descriptor"};
    --it;
    int64_t off = p - std::get<0>(*it);
    if (off < 0 || off > std::get<1>(*it)) throw Fail{IGAMG_ERR_NUMERIC, "untracked array in a descriptor"};
    return std::get<2>(*it) + off;
  };
  auto tr_set = [&](const GemmSet& g, GemmSetT<float>& out) {
    std::vector<GemmDescT<float>> v;
    for (const GemmDesc& d : g.h)
      v.push_back(GemmDescT<float>{tr(d.A), tr(d.B), tr(d.C), tr(d.E), d.lda, d.ldb, d.ldc, d.lde, d.M, d.N, d.K});
    set_gemm(c, out, v);
    out.R = g.R;
  };
  for (size_t l = 0; l < c->lv.size(); ++l) {
    Level& L = c->lv[l];
    Num<double>& A = L.n64;
    Num<float>& B = L.n32;
    B.F = tr(A.F);
    B.U = tr(A.U);
    B.R = tr(A.R);
    B.cX = tr(A.cX);
    B.G = tr(A.G);
    B.Z = tr(A.Z);
    B.vscale = tr(A.vscale);
    B.tA = tr(A.tA);
    B.tB = tr(A.tB);
    int64_t nb = c->band_count[l];
    const bool finest = l + 1 == c->lv.size();
    float* b32 = nullptr;
    if (L.kron) {  // FP32 1D factors in every variant (no bands to round to BF16)
      std::vector<KronDevT<float>> kf;
      for (const auto& k : L.kd_h)
        kf.push_back(KronDevT<float>{k.off, k.n0, k.n1, k.p0, k.p1, tr(k.K0), tr(k.M0), tr(k.K1), tr(k.M1),
                                     float(k.c0), float(k.c1)});
      B.kd = c->mem.upload(kf, s);
    }
    // 3D BF16 bands of one degree: the paired layout (rows padded to even length, one
    // bfloat162 load per tap and node pair; FP32 bands stay flat: paired float2 loads
    // measured slower)
    const bool pair = bf16_bands && !L.kron && c->pd.dim == 3 && L.uniform_p >= 2 && L.uniform_p <= 4;
    const int taps = (2 * L.uniform_p + 1) * (2 * L.uniform_p + 1) * (2 * L.uniform_p + 1);
    int64_t ptot = 0, pmaxe = 0;
    if (pair) {
      std::vector<PatchDev> pp = L.pd_h;
      for (auto& q : pp) {
        const int64_t ne = int64_t(q.n[0]) * q.n[1] * band_row_even(q.n[2]);
        q.band_off = ptot;
        ptot += taps * ne;
        pmaxe = std::max(pmaxe, ne);
      }
      B.pd_pair = c->mem.upload(pp, s);
    }
    if (!L.kron && (!bf16_bands || finest)) {  // FP32 bands: the cycle's (FP32 mode) and the Krylov operator's
      if (c->pd.dim == 3 && L.uniform_p >= 2 && L.uniform_p <= 4) {
        // tap-blocked layout: all taps of 32 consecutive nodes contiguous
        const int tp = (2 * L.uniform_p + 1) * (2 * L.uniform_p + 1) * (2 * L.uniform_p + 1);
        std::vector<PatchDev> pb = L.pd_h;
        int64_t tot = 0, maxn = 0;
        for (auto& q : pb) {
          const int64_t nn = int64_t(q.n[0]) * q.n[1] * q.n[2];
          q.band_off = tot;
          tot += (nn + 31) / 32 * 32 * tp;
          maxn = std::max(maxn, nn);
        }
        b32 = c->mem.alloc<float>(size_t(std::max<int64_t>(tot, 1)));
        B.pd_blk = c->mem.upload(pb, s);
        CK(launch_band_blk_f32(s, L.pd, B.pd_blk, int(pb.size()), tp, maxn, L.band, b32));
      } else {
        b32 = c->mem.alloc<float>(nb);
        CK(launch_convert_f64_f32(s, nb, L.band, 1.0, b32));
      }
      B.band_op = b32;
    }
    if (bf16_bands && !L.kron && pair) {
      __nv_bfloat16* bb = c->mem.alloc<__nv_bfloat16>(size_t(std::max<int64_t>(ptot, 1)));
      CK(launch_band_pair<__nv_bfloat16>(s, L.pd, B.pd_pair, int(L.pd_h.size()), taps, pmaxe, L.band, bb));
      B.band = bb;
      B.bf16 = true;
    } else if (bf16_bands && !L.kron) {
      __nv_bfloat16* bb = c->mem.alloc<__nv_bfloat16>(nb);
      CK(launch_convert_f64_bf16(s, nb, L.band, bb));
      B.band = bb;
      B.bf16 = true;
    } else {
      B.band = b32;
    }
    if (bf16_bands && L.tc_ok && (A.use_tc || c->opt.fd_engine == 0)) {  // BF16 operands: one MMA per product
      auto tr_tc = [&](const TcSet<double>& g, TcSet<float>& out) {
        std::vector<TcDesc<float, float>> v;
        for (const auto& d : g.h) {
          auto it = c->tc_bf16_twin.find(d.Aslices);
          if (it == c->tc_bf16_twin.end()) throw Fail{IGAMG_ERR_NUMERIC, "missing BF16 basis slices"};
          v.push_back(TcDesc<float, float>{static_cast<const __nv_bfloat16*>(it->second), nullptr, d.nkb, tr(d.B), d.ldb,
                                            d.tb, tr(d.C), d.ldc, d.tc, tr(d.E), d.lde, d.M, d.N, d.K});
        }
        set_tc(c, out, v, g.side);
      };
      tr_tc(A.tc0F, B.tc0F); tr_tc(A.tc0R, B.tc0R); tr_tc(A.tc1, B.tc1); tr_tc(A.tc2, B.tc2); tr_tc(A.tc3, B.tc3);
      tr_tc(A.tc4, B.tc4); tr_tc(A.tc5, B.tc5);
      tr_tc(A.tq0, B.tq0); tr_tc(A.tq1, B.tq1); tr_tc(A.tq2, B.tq2); tr_tc(A.tq3, B.tq3);
      B.use_tc = true;
    }
    if (!L.fr_h.empty()) {
      std::vector<FdRowsT<float>> fr;
      for (const auto& f : L.fr_h)
        fr.push_back(FdRowsT<float>{tr(f.U0), tr(f.U1), tr(f.Dinv), tr(f.vF), tr(f.vR), tr(f.u), tr(f.Y), f.n0, f.n1,
                                    f.ld});
      B.frows = c->mem.upload(fr, s);
      B.nfrows = int(fr.size());
      B.frows_n0 = A.frows_n0;
      B.frows_n1 = A.frows_n1;
      B.use_rows = A.use_rows;
    }
    if (L.fused_ok) {
      std::vector<FdSmallT<float>> fs;
      for (const auto& f : L.fs_h)
        fs.push_back(FdSmallT<float>{tr(f.U0), tr(f.U1), tr(f.Dinv), tr(f.vF), tr(f.vR), tr(f.u), f.n0, f.n1, f.ld});
      B.fsmall = c->mem.upload(fs, s);
      B.nfsmall = int(fs.size());
      B.fsmall_flops = A.fsmall_flops;
      B.use_fused = A.use_fused;
      if (L.small_ok) {
        std::vector<EdgeSmallT<float>> es;
        for (const auto& e : L.es_h) es.push_back(EdgeSmallT<float>{tr(e.U), tr(e.dinv), e.first, e.len});
        SmoothSmallT<float>& q = B.ssmall;
        const SmoothSmallT<double>& a = A.ssmall;
        q.fd = B.fsmall;
        q.nfd = B.nfsmall;
        q.edges = es.empty() ? nullptr : c->mem.upload(es, s);
        q.nedges = int(es.size());
        q.ptr = a.ptr;
        q.idx = a.idx;
        q.vscale = tr(a.vscale);
        q.vbeg = a.vbeg;
        q.vend = a.vend;
        q.vF = tr(a.vF);
        q.vR = tr(a.vR);
        q.u = tr(a.u);
        B.ssmall_flops = A.ssmall_flops;
      }
    }
    tr_set(A.st0F, B.st0F); tr_set(A.st0R, B.st0R); tr_set(A.st1, B.st1); tr_set(A.st2, B.st2);
    tr_set(A.st3, B.st3);
    tr_set(A.m0f, B.m0f); tr_set(A.m1f, B.m1f); tr_set(A.m2f, B.m2f);
    tr_set(A.m0b, B.m0b); tr_set(A.m1b, B.m1b); tr_set(A.m2b, B.m2b);
    auto tr_mode = [&](const ModeSetT<double>& a, ModeSetT<float>& b) {
      if (!a.batch) return;
      std::vector<ModeDescT<float>> v;
      for (const auto& d : a.h)
        v.push_back(ModeDescT<float>{tr(d.Mat), tr(d.X), tr(d.Y), tr(d.E), d.n, d.mtr, d.inner, d.fibres});
      set_mode(c, b, v);
    };
    for (int j = 0; j < 6; ++j) tr_mode(A.md[j], B.md[j]);
    if (!L.fd3_h.empty()) {
      std::vector<Fd3SmallT<float>> f3;
      for (const auto& f : L.fd3_h) {
        Fd3SmallT<float> g{tr(f.U0), tr(f.U1), tr(f.U2), tr(f.Dinv), f.tile_off, {}, {}, {}};
        for (int j = 0; j < 3; ++j) {
          g.n[j] = f.n[j];
          g.lo[j] = f.lo[j];
          g.len[j] = f.len[j];
        }
        f3.push_back(g);
      }
      B.fd3 = c->mem.upload(f3, s);
      B.nfd3 = int(f3.size());
    }
    for (int j = 0; j < 4; ++j) tr_mode(A.fm[j], B.fm[j]);
    if (A.i3_ok) {
      std::vector<FaceSmallT<float>> f3;
      for (const auto& f : L.f3s_h) f3.push_back(FaceSmallT<float>{tr(f.U0), tr(f.U1), tr(f.Dinv), f.first, f.len0, f.len1});
      std::vector<EdgeSmallT<float>> e3;
      for (const auto& e : L.e3s_h) e3.push_back(EdgeSmallT<float>{tr(e.U), tr(e.dinv), e.first, e.len});
      Iface3SmallT<float>& q = B.i3s;
      q.faces = f3.empty() ? nullptr : c->mem.upload(f3, s);
      q.nfaces = int(f3.size());
      q.edges = e3.empty() ? nullptr : c->mem.upload(e3, s);
      q.nedges = int(e3.size());
      q.ptr = L.if_ptr;
      q.idx = L.if_idx;
      q.vscale = tr(A.vscale);
      q.vbeg = L.v3_beg;
      q.vend = L.v3_end;
      q.u = tr(A.U);
      B.i3_ok = true;
    }
    tr_set(A.edgeA, B.edgeA); tr_set(A.edgeB, B.edgeB);
    tr_set(A.face0, B.face0); tr_set(A.face1, B.face1); tr_set(A.face2, B.face2); tr_set(A.face3, B.face3);
    if (!L.r2_h.empty()) {
      std::vector<Xfer2T<float>> r2, p2;
      for (const auto& x : L.r2_h)
        r2.push_back(Xfer2T<float>{x.in_off, x.out_off, x.nin0, x.nin1, x.nout0, x.nout1, tr(x.w0), tr(x.w1), x.st0,
                                   x.st1, x.width0, x.width1});
      for (const auto& x : L.p2_h)
        p2.push_back(Xfer2T<float>{x.in_off, x.out_off, x.nin0, x.nin1, x.nout0, x.nout1, tr(x.w0), tr(x.w1), x.st0,
                                   x.st1, x.width0, x.width1});
      B.r2 = c->mem.upload(r2, s);
      B.p2 = c->mem.upload(p2, s);
    }
    for (int j = 0; j < 3; ++j) {
      if (L.rp_h[j].empty()) continue;
      std::vector<XferT<float>> rp, pp;
      for (auto& x : L.rp_h[j]) rp.push_back(XferT<float>{x.in_off, x.out_off, x.outer, x.inner, x.nin, x.nout, x.width, tr(x.wt), x.st});
      for (auto& x : L.pp_h[j]) pp.push_back(XferT<float>{x.in_off, x.out_off, x.outer, x.inner, x.nin, x.nout, x.width, tr(x.wt), x.st});
      B.rpass[j] = c->mem.upload(rp, s);
      B.ppass[j] = c->mem.upload(pp, s);
    }
  }
  int64_t Tf = c->lv.back().topo.T;
  c->X32 = c->mem.alloc<float>(Tf);
  c->P32 = c->mem.alloc<float>(Tf);
  c->W32 = c->mem.alloc<float>(Tf);
  c->Zold32 = c->mem.alloc<float>(Tf);
  bind_tc<float>(c);
  c->low = true;
  c->low_bf16 = bf16_bands;
  CK(cudaStreamSynchronize(s));
}

template <class F>
igamg_status guarded(igamg_ctx* c, F&& f) {
  if (!c) return IGAMG_ERR_ARG;
  try {
    igamg_status st = f();
    if (st != IGAMG_OK && st != IGAMG_ERR_NOT_CONVERGED) return st;
    if (st == IGAMG_ERR_NOT_CONVERGED) c->err = "PCG did not reach the tolerance within max_iter";
    return st;
  } catch (const Fail& e) {
    c->err = e.msg;
    return e.code;
  } catch (const std::exception& e) {
    c->err = e.what();
    return IGAMG_ERR_ARG;
  }
}

}  // namespace

// ---------------------------------------------------------------- lockstep batches
//
// Many independent problems solved by PCG in lockstep, every step of Algorithm 1 one launch
// over all problems: the stiffness applies, smoother pieces, transfers and coarse solves of
// every problem at the same depth below its finest level (depth d = level L_q - d of problem
// q), and the PCG vector operations of all problems.  The launches take job lists built once
// from the problems' own descriptors, so each problem runs exactly the arithmetic of its
// single solve (same kernels per entry, same reduction partitions) and its iterates are
// bit-identical to solving it alone; a problem that has converged keeps its iterate (its
// updates are masked) while the others continue.  One PCG iteration of the whole batch is
// one CUDA graph replay.  Scope: 2D problems whose patches are rectangles (Kronecker apply),
// FP64, V-cycles; other batches use the worker-stream path.
namespace igamg {

struct LockGemmGroup {  // FMA GEMM stage descriptors of one tile factor R
  GemmDesc* d = nullptr;
  int batch = 0, maxM = 0, maxN = 0, R = 0;
  double flops = 0;
};
struct LockTcStage {  // one tensor-core stage over the problems that use the tensor cores
  TcDesc<double, double>* d = nullptr;
  int *tstart = nullptr, *pstart = nullptr;
  int batch = 0;
  int64_t tiles = 0, panels = 0;
  double exec_flops = 0, flops = 0;
};
struct LockStackStage {  // one stacked (fibre-major) tensor-core stage over the problems
  TcStack<double, double>* d = nullptr;
  int *tstart = nullptr, *pstart = nullptr;
  int batch = 0;
  int64_t tiles = 0, panels = 0;
  double exec_flops = 0, flops = 0;
};
struct LockSmooth {  // the smoother of one depth, one direction (from F, assign / from R, add)
  // one-launch small-level smoothers
  SmoothSmallT<double>* small = nullptr;
  int* small_start = nullptr;
  int nsmall = 0, small_blocks = 0;
  // interface pieces of the other problems
  NodeJobT<double>* gather = nullptr;
  NodeJobT<double>* scatter = nullptr;
  int niface = 0;
  int64_t max_if = 0;
  std::vector<LockGemmGroup> edgeA, edgeB;
  // interiors by engine
  FdRowsT<double>* rows = nullptr;
  int nrows = 0, rows_n0 = 0, rows_n1 = 0;
  FdSmallT<double>* fsmall = nullptr;
  int nfsmall = 0;
  LockTcStage tc[4];
  LockStackStage sk[4];
  std::vector<LockGemmGroup> st[4];
  double flops = 0;  // algorithmic FLOPs of the kernels outside the GEMM groups and stages
};
struct LockDepth {
  KronJobT<double>* res = nullptr;  // r = f - A u on this depth's levels
  int nres = 0, res_n0 = 0, res_n1 = 0, res_p = 0;
  double res_flops = 0, x_flops = 0, coarse_flops = 0;
  LockSmooth sm[2];                 // [0] from F, assign (zero initial guess); [1] from R, add
  Xfer2JobT<double>* rst = nullptr;
  Xfer2JobT<double>* pro = nullptr;
  int nx = 0, r_out0 = 0, r_out1 = 0, r_w1 = 0, p_out0 = 0, p_out1 = 0, p_w1 = 0;
  NodeJobT<double>* coarse = nullptr;  // problems whose next level is the coarsest
  int ncoarse = 0;
  int64_t coarse_n = 0;
};

// One right-hand side of a lockstep solve: a context and the work arrays it runs on (its
// own, or one of its copies when several right-hand sides of one problem run together).
struct LockMember {
  igamg_ctx* c = nullptr;
  const WorkCopy* w = nullptr;  // nullptr: the context's own arrays
  // this member's array for an array of the context (constant arrays map to themselves)
  double* tr(const double* p) const {
    if (!w || !p) return const_cast<double*>(p);
    auto it = std::upper_bound(w->tw.begin(), w->tw.end(), p,
                               [](const double* q, const auto& e) { return q < std::get<0>(e); });
    if (it == w->tw.begin()) throw Fail{IGAMG_ERR_NUMERIC, "untracked array in a descriptor"};
    --it;
    const int64_t off = p - std::get<0>(*it);
    if (off < 0 || off > std::get<1>(*it)) throw Fail{IGAMG_ERR_NUMERIC, "untracked array in a descriptor"};
    return std::get<2>(*it) + off;
  }
  double* X() const { return w ? w->X : c->X; }
  double* Pv() const { return w ? w->Pv : c->Pv; }
  double* W() const { return w ? w->W : c->W; }
  double* Bt() const { return w ? w->Bt : c->Bt; }
  double* Rr() const { return w ? w->Rr : c->Rr; }
};

struct Lockstep {
  std::vector<igamg_ctx*> ctx;
  std::vector<LockMember> mb;
  DevMem mem;
  int nprob = 0, depths = 0, nu = 1;
  double tau = 0.25;
  std::vector<LockDepth> dep;
  // finest-level Krylov apply w = A p, and the operands of the PCG vector steps
  KronJobT<double>* kry = nullptr;
  int nkry = 0, kry_n0 = 0, kry_n1 = 0, kry_p = 0;
  double kry_flops = 0, vec_flops = 0;
  VecJobT<double>* v_fu = nullptr;   // dot(F, U) / copy U -> p (a = F or p, b = U)
  VecJobT<double>* v_pw = nullptr;   // dot(p, w)
  VecJobT<double>* v_xr = nullptr;   // x += alpha p, r -= alpha w
  VecJobT<double>* v_pz = nullptr;   // p = U + beta p
  VecJobT<double>* v_nrm = nullptr;  // norm of the distributed residual F
  VecJobT<double>* v_cpu = nullptr;  // p = U
  int64_t max_T = 0;
  double* partials = nullptr;        // nprob x RED_BLOCKS
  double* scal = nullptr;            // nprob x 8 PCG scalars
  double* h_scal = nullptr;          // pinned mirror
  int* active = nullptr;
  int* h_active = nullptr;           // pinned mirror
  int* err = nullptr;                // tensor-core timeout flag
  cudaStream_t cap = nullptr;
  cudaGraphExec_t iter = nullptr;
  // accounting: launches and algorithmic FLOPs of the last solve (per graph replay: the
  // counts of its capture)
  int64_t launches = 0, it_launches = 0;
  double flops = 0, it_flops = 0, mma_flops = 0, it_mma_flops = 0;
};

namespace {

template <class V>
V* lk_upload(Lockstep* k, const std::vector<V>& h) {
  if (h.empty()) return nullptr;
  V* d = k->mem.alloc<V>(h.size());
  CK(cudaMemcpy(d, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice));
  return d;
}

using MemberGemm = std::pair<const GemmSet*, const LockMember*>;
using MemberTc = std::pair<const TcSet<double>*, const LockMember*>;
using MemberStack = std::pair<const StackSet*, const LockMember*>;

// The stacked descriptors of every member at one stage (a copy's own tables and scratch).
void lk_stack_stage(Lockstep* k, const std::vector<MemberStack>& sets, LockStackStage& out) {
  std::vector<TcStack<double, double>> h;
  for (const auto& sm : sets) {
    const StackSet* t = sm.first;
    const LockMember& m = *sm.second;
    for (int i = 0; i < t->batch; ++i) {
      TcStack<double, double> d = t->h[i];
      if (m.w) {
        std::vector<const double*> X, E;
        std::vector<double*> C;
        for (const double* p : t->hX[i]) X.push_back(m.tr(p));
        for (double* p : t->hC[i]) C.push_back(m.tr(p));
        for (const double* p : t->hE[i]) E.push_back(m.tr(p));
        d.X = lk_upload(k, X);
        d.C = lk_upload(k, C);
        d.E = t->h[i].E ? lk_upload(k, E) : nullptr;
        d.Xdig = m.w->sdig + t->dig_off[i];
        d.Xtau = m.w->stau + t->tau_off[i];
      }
      h.push_back(d);
    }
    out.exec_flops += t->exec_flops;
    out.flops += t->flops;
  }
  if (h.empty()) return;
  std::vector<int> ts, ps;
  tc_stack_prefixes(h, ts, ps);
  out.batch = int(h.size());
  out.tiles = ts.back();
  out.panels = ps.back();
  out.d = lk_upload(k, h);
  out.tstart = lk_upload(k, ts);
  out.pstart = lk_upload(k, ps);
}

void lk_gemm_groups(Lockstep* k, const std::vector<MemberGemm>& sets, std::vector<LockGemmGroup>& out) {
  std::map<int, std::vector<GemmDesc>> byR;
  for (const auto& gm : sets) {
    const GemmSet* g = gm.first;
    const LockMember& m = *gm.second;
    if (!g->batch) continue;
    for (GemmDesc d : g->h) {
      d.A = m.tr(d.A);
      d.B = m.tr(d.B);
      d.C = m.tr(d.C);
      d.E = m.tr(d.E);
      byR[g->R].push_back(d);
    }
  }
  for (auto& kv : byR) {
    LockGemmGroup gg;
    gg.R = kv.first;
    gg.batch = int(kv.second.size());
    for (auto& d : kv.second) {
      gg.maxM = std::max(gg.maxM, d.M);
      gg.maxN = std::max(gg.maxN, d.N);
    }
    gg.flops = gemm_flops(kv.second);
    gg.d = lk_upload(k, kv.second);
    out.push_back(gg);
  }
}

void lk_tc_stage(Lockstep* k, const std::vector<MemberTc>& sets, LockTcStage& out) {
  std::vector<TcDesc<double, double>> h;
  for (const auto& tm : sets) {
    const TcSet<double>* t = tm.first;
    const LockMember& m = *tm.second;
    for (int i = 0; i < t->batch; ++i) {
      TcDesc<double, double> d = t->h[i];
      if (m.w) {  // the copy's inputs, outputs and digit scratch
        d.B = m.tr(d.B);
        d.C = m.tr(d.C);
        d.E = m.tr(d.E);
        d.Bdig = m.w->dig[t->side] + t->dig_off[i];
        d.Btau = m.w->tau[t->side] ? m.w->tau[t->side] + t->tau_off[i] : nullptr;
      }
      h.push_back(d);
    }
    out.exec_flops += t->exec_flops;
    out.flops += t->flops;
  }
  if (h.empty()) return;
  std::vector<int> ts, ps;
  tc_prefixes(h, 7, ts, ps);
  out.batch = int(h.size());
  out.tiles = ts.back();
  out.panels = ps.back();
  out.d = lk_upload(k, h);
  out.tstart = lk_upload(k, ts);
  out.pstart = lk_upload(k, ps);
}

}  // namespace

void lockstep_free(Lockstep* k) {
  if (!k) return;
  if (k->iter) cudaGraphExecDestroy(k->iter);
  if (k->cap) cudaStreamDestroy(k->cap);
  if (k->h_scal) cudaFreeHost(k->h_scal);
  if (k->h_active) cudaFreeHost(k->h_active);
  k->mem.release();
  delete k;
}

// The one-launch small-level smoother of member m (the copy's arrays for a copy).
SmoothSmallT<double> lk_small(Lockstep* k, const LockMember& m, const Level& L) {
  const SmoothSmallT<double>& a = L.n64.ssmall;
  if (!m.w) return a;
  SmoothSmallT<double> q = a;
  std::vector<FdSmallT<double>> fs;
  for (const auto& f : L.fs_h)
    fs.push_back(FdSmallT<double>{f.U0, f.U1, f.Dinv, m.tr(f.vF), m.tr(f.vR), m.tr(f.u), f.n0, f.n1, f.ld});
  q.fd = lk_upload(k, fs);
  q.vF = m.tr(a.vF);
  q.vR = m.tr(a.vR);
  q.u = m.tr(a.u);
  return q;  // the edge pieces read and write only through vF, vR and u
}

// The lockstep engine of a batch, or NULL (with the reason) when a problem is outside its
// scope.  Called after every context is set up (their engines chosen and descriptors built).
// `mb` lists the right-hand sides: distinct problems, or one problem and its work copies;
// with fp64_of_low a precision-variant context runs its FP64 numerics.
Lockstep* lockstep_build(const std::vector<LockMember>& mb, std::string* why, bool fp64_of_low) {
  auto no = [&](const std::string& w) -> Lockstep* {
    if (why) *why = w;
    return nullptr;
  };
  if (mb.empty()) return no("empty batch");
  std::vector<igamg_ctx*> ctx;
  for (const auto& m : mb) ctx.push_back(m.c);
  const igamg_options& o0 = ctx[0]->opt;
  for (igamg_ctx* c : ctx) {
    if (c->pd.dim != 2) return no("3D problem");
    if (!fp64_of_low && (c->opt.precision != IGAMG_FP64 || c->low)) return no("precision variant");
    if (c->opt.mu != 1 || c->opt.nu != o0.nu || c->opt.tau != o0.tau) return no("cycle options differ");
    if (c->lv.size() < 2) return no("single-level hierarchy");
    for (size_t l = 1; l < c->lv.size(); ++l) {
      const Level& L = c->lv[l];
      if (!L.kron || !L.n64.r2 || !L.n64.p2) return no("non-rectangle patch or transfer layout");
    }
  }
  Lockstep* k = new Lockstep();
  try {
    k->ctx = ctx;
    k->mb = mb;
    k->nprob = int(ctx.size());
    k->nu = o0.nu;
    k->tau = o0.tau;
    for (igamg_ctx* c : ctx) k->depths = std::max(k->depths, int(c->lv.size()) - 1);
    k->dep.resize(k->depths);
    for (int d = 0; d < k->depths; ++d) {
      LockDepth& D = k->dep[d];
      std::vector<KronJobT<double>> res;
      std::vector<Xfer2JobT<double>> rst, pro;
      std::vector<NodeJobT<double>> coarse;
      struct Side {
        std::vector<SmoothSmallT<double>> small;
        std::vector<int> small_start{0};
        std::vector<NodeJobT<double>> gather, scatter;
        std::vector<MemberGemm> eA, eB, st[4];
        std::vector<MemberTc> tc[4];
        std::vector<MemberStack> sk[4];
        std::vector<FdRowsT<double>> rows;
        std::vector<FdSmallT<double>> fsmall;
      } sd[2];
      for (const LockMember& m : k->mb) {
        igamg_ctx* c = m.c;
        const int l = int(c->lv.size()) - 1 - d;
        if (l < 1) continue;
        Level& L = c->lv[l];
        Level& C = c->lv[l - 1];
        Num<double>& N = L.n64;
        for (const auto& kd : L.kd_h) res.push_back(KronJobT<double>{kd, L.active, m.tr(N.U), m.tr(N.F), m.tr(N.R)});
        D.res_flops += L.apply_flops;
        D.x_flops += L.xfer_flops / 3;  // restriction; the prolongation is 2/3 of xfer_flops
        D.res_n0 = std::max(D.res_n0, L.max_n[0]);
        D.res_n1 = std::max(D.res_n1, L.max_n[1]);
        D.res_p = std::max(D.res_p, L.max_p);
        for (const auto& x : L.r2_h) rst.push_back(Xfer2JobT<double>{x, m.tr(N.R), m.tr(C.n64.F), C.l2g});
        for (const auto& x : L.p2_h) pro.push_back(Xfer2JobT<double>{x, m.tr(C.n64.U), m.tr(N.U), nullptr});
        D.r_out0 = std::max(D.r_out0, L.x2_rout0);
        D.r_out1 = std::max(D.r_out1, L.x2_rout1);
        D.r_w1 = std::max(D.r_w1, L.x2_rw1);
        D.p_out0 = std::max(D.p_out0, L.x2_pout0);
        D.p_out1 = std::max(D.p_out1, L.x2_pout1);
        D.p_w1 = std::max(D.p_w1, L.x2_pw1);
        if (l == 1) {
          Level& L0 = c->lv[0];
          NodeJobT<double> j{};
          j.n = c->N0;
          j.ptr = L0.g2t_ptr;
          j.idx = L0.g2t;
          j.v = m.tr(L0.n64.F);
          j.u = m.tr(L0.n64.U);
          j.Ainv = c->A0inv;
          coarse.push_back(j);
          D.coarse_n = std::max(D.coarse_n, c->N0);
          D.coarse_flops += 2.0 * double(c->N0) * c->N0;
        }
        for (int dir = 0; dir < 2; ++dir) {  // 0: from F (assign), 1: from R (add)
          Side& S = sd[dir];
          const double* v = m.tr(dir == 0 ? N.F : N.R);
          if (N.use_fused && L.small_ok) {
            D.sm[dir].flops += N.ssmall_flops;
            S.small.push_back(lk_small(k, m, L));
            const SmoothSmallT<double>& q = N.ssmall;
            S.small_start.push_back(S.small_start.back() + q.nfd + q.nedges + (q.vend > q.vbeg ? 1 : 0));
            continue;
          }
          if (L.n_if > 0) {
            NodeJobT<double> g{};
            g.n = L.n_if;
            g.ptr = L.if_ptr;
            g.idx = L.if_idx;
            g.v = v;
            g.G = m.tr(N.G);
            S.gather.push_back(g);
            NodeJobT<double> t{};
            t.n = L.n_if;
            t.ptr = L.if_ptr;
            t.idx = L.if_idx;
            t.Z = m.tr(N.Z);
            t.G = m.tr(N.G);
            t.vscale = N.vscale;
            t.u = m.tr(N.U);
            S.scatter.push_back(t);
            S.eA.push_back({&N.edgeA, &m});
            S.eB.push_back({&N.edgeB, &m});
            LockSmooth& LS = D.sm[dir];
            LS.max_if = std::max(LS.max_if, L.n_if);
          }
          // The tensor cores wherever their stage sets were built and the interiors exceed
          // the one-block size: a problem timed alone may lose with few tiles, but the
          // lockstep launches hold the tiles of every problem at this depth.
          const bool tc = N.tc0F.batch && (N.use_tc || (c->opt.fd_engine == 0 && L.tc_ok && !L.fused_ok));
          if (tc && N.sk1.batch) {  // the stacked stages, as a single solve runs them
            S.sk[0].push_back({dir == 0 ? &N.sk0F : &N.sk0R, &m});
            S.sk[1].push_back({&N.sk1, &m});
            S.sk[2].push_back({&N.sk2, &m});
            S.sk[3].push_back({&N.sk3, &m});
          } else if (tc) {
            S.tc[0].push_back({dir == 0 ? &N.tc0F : &N.tc0R, &m});
            S.tc[1].push_back({&N.tc1, &m});
            S.tc[2].push_back({&N.tc2, &m});
            S.tc[3].push_back({&N.tc3, &m});
          } else if (N.use_rows) {
            D.sm[dir].flops += 4.0 * N.st1.flops;
            for (const auto& f : L.fr_h)
              S.rows.push_back(FdRowsT<double>{f.U0, f.U1, f.Dinv, m.tr(f.vF), m.tr(f.vR), m.tr(f.u), m.tr(f.Y),
                                               f.n0, f.n1, f.ld});
            D.sm[dir].rows_n0 = std::max(D.sm[dir].rows_n0, N.frows_n0);
            D.sm[dir].rows_n1 = std::max(D.sm[dir].rows_n1, N.frows_n1);
          } else if (N.use_fused) {
            D.sm[dir].flops += N.fsmall_flops;
            for (const auto& f : L.fs_h)
              S.fsmall.push_back(FdSmallT<double>{f.U0, f.U1, f.Dinv, m.tr(f.vF), m.tr(f.vR), m.tr(f.u), f.n0, f.n1,
                                                  f.ld});
          } else {
            S.st[0].push_back({dir == 0 ? &N.st0F : &N.st0R, &m});
            S.st[1].push_back({&N.st1, &m});
            S.st[2].push_back({&N.st2, &m});
            S.st[3].push_back({&N.st3, &m});
          }
        }
      }
      D.res = lk_upload(k, res);
      D.nres = int(res.size());
      D.rst = lk_upload(k, rst);
      D.pro = lk_upload(k, pro);
      D.nx = int(rst.size());
      if (pro.size() != rst.size()) throw Fail{IGAMG_ERR_NUMERIC, "lockstep: transfer job lists differ"};
      D.coarse = lk_upload(k, coarse);
      D.ncoarse = int(coarse.size());
      for (int dir = 0; dir < 2; ++dir) {
        Side& S = sd[dir];
        LockSmooth& LS = D.sm[dir];
        LS.small = lk_upload(k, S.small);
        LS.nsmall = int(S.small.size());
        LS.small_start = LS.nsmall ? lk_upload(k, S.small_start) : nullptr;
        LS.small_blocks = S.small_start.back();
        LS.gather = lk_upload(k, S.gather);
        LS.scatter = lk_upload(k, S.scatter);
        LS.niface = int(S.gather.size());
        lk_gemm_groups(k, S.eA, LS.edgeA);
        lk_gemm_groups(k, S.eB, LS.edgeB);
        LS.rows = lk_upload(k, S.rows);
        LS.nrows = int(S.rows.size());
        LS.fsmall = lk_upload(k, S.fsmall);
        LS.nfsmall = int(S.fsmall.size());
        for (int st = 0; st < 4; ++st) {
          lk_tc_stage(k, S.tc[st], LS.tc[st]);
          lk_stack_stage(k, S.sk[st], LS.sk[st]);
          lk_gemm_groups(k, S.st[st], LS.st[st]);
        }
      }
    }
    // finest level: Krylov apply and PCG vectors (scalars of problem q at scal[8 q ..])
    k->scal = k->mem.alloc<double>(size_t(8) * k->nprob);
    CK(cudaMemset(k->scal, 0, sizeof(double) * 8 * k->nprob));
    k->partials = k->mem.alloc<double>(size_t(RED_BLOCKS) * k->nprob);
    k->active = k->mem.alloc<int>(size_t(k->nprob));
    k->err = k->mem.alloc<int>(1);
    CK(cudaMemset(k->err, 0, sizeof(int)));
    CK(cudaMallocHost(&k->h_scal, sizeof(double) * 8 * k->nprob));
    CK(cudaMallocHost(&k->h_active, sizeof(int) * k->nprob));
    std::vector<KronJobT<double>> kry;
    std::vector<VecJobT<double>> fu, pw, xr, pz, nrm, cpu;
    for (int q = 0; q < k->nprob; ++q) {
      const LockMember& m = k->mb[q];
      igamg_ctx* c = m.c;
      Level& L = c->lv.back();
      Num<double>& N = L.n64;
      for (const auto& kd : L.kd_h) kry.push_back(KronJobT<double>{kd, L.active, m.Pv(), nullptr, m.W()});
      k->kry_flops += L.apply_flops;
      k->vec_flops += 12.0 * double(L.topo.T);  // two dots, the x, r and p updates, the norm
      k->kry_n0 = std::max(k->kry_n0, L.max_n[0]);
      k->kry_n1 = std::max(k->kry_n1, L.max_n[1]);
      k->kry_p = std::max(k->kry_p, L.max_p);
      const int64_t T = L.topo.T;
      k->max_T = std::max(k->max_T, T);
      double* sc = k->scal + 8 * q;
      double *F = m.tr(N.F), *U = m.tr(N.U);
      fu.push_back(VecJobT<double>{T, sc, nullptr, nullptr, F, U, nullptr, nullptr});
      pw.push_back(VecJobT<double>{T, sc, nullptr, nullptr, m.Pv(), m.W(), nullptr, nullptr});
      xr.push_back(VecJobT<double>{T, sc, nullptr, nullptr, m.X(), F, m.Pv(), m.W()});
      pz.push_back(VecJobT<double>{T, sc, nullptr, nullptr, m.Pv(), nullptr, U, nullptr});
      nrm.push_back(VecJobT<double>{L.topo.N, sc, L.g2t_ptr, L.g2t, F, nullptr, nullptr, nullptr});
      cpu.push_back(VecJobT<double>{T, sc, nullptr, nullptr, m.Pv(), U, nullptr, nullptr});
    }
    k->kry = lk_upload(k, kry);
    k->nkry = int(kry.size());
    k->v_fu = lk_upload(k, fu);
    k->v_pw = lk_upload(k, pw);
    k->v_xr = lk_upload(k, xr);
    k->v_pz = lk_upload(k, pz);
    k->v_nrm = lk_upload(k, nrm);
    k->v_cpu = lk_upload(k, cpu);
    CK(cudaStreamCreateWithFlags(&k->cap, cudaStreamNonBlocking));
  } catch (const Fail& f) {
    lockstep_free(k);
    return no(f.msg);
  }
  return k;
}

namespace {

void lk_count(Lockstep* k, int launches, double flops, double mma = 0.0) {
  k->launches += launches;
  k->flops += flops;
  k->mma_flops += mma;
}

void lk_res(Lockstep* k, cudaStream_t s, const LockDepth& D) {
  if (!D.nres) return;
  CK(launch_kron_apply_2d_b<double>(s, D.res, D.nres, D.res_n0, D.res_n1, D.res_p));
  lk_count(k, 1, D.res_flops);
}

// One smoothing step of every problem at one depth: the small-level one-launch smoothers,
// then the interface pieces and the interiors of the others, each by the engine its own
// solve uses (the pieces are disjoint, so their order does not change any result).
void lk_smooth(Lockstep* k, cudaStream_t s, const LockSmooth& S, bool from_F, bool add) {
  const double tau = k->tau;
  const int fF = from_F ? 1 : 0, ad = add ? 1 : 0;
  lk_count(k, (S.nsmall ? 1 : 0) + (S.niface ? 2 : 0) + (S.nrows ? 2 : 0) + (S.nfsmall ? 1 : 0), S.flops);
  CK(launch_smooth_small_b<double>(s, S.small, S.small_start, S.nsmall, S.small_blocks, fF, tau, ad));
  if (S.niface) {
    CK(launch_iface_gather_b<double>(s, S.gather, S.niface, S.max_if));
    for (const auto& g : S.edgeA) {
      CK(launch_gemm<double>(s, g.d, g.batch, g.maxM, g.maxN, false, false, EPI_COLSCALE, 1.0, g.R));
      lk_count(k, 1, g.flops);
    }
    for (const auto& g : S.edgeB) {
      CK(launch_gemm<double>(s, g.d, g.batch, g.maxM, g.maxN, false, true, EPI_STORE, 1.0, g.R));
      lk_count(k, 1, g.flops);
    }
    CK(launch_iface_scatter_b<double>(s, S.scatter, S.niface, S.max_if, tau, ad));
  }
  for (int pass = 1; pass <= 2 && S.nrows; ++pass)
    CK(launch_fd_rows<double>(s, S.rows, S.nrows, S.rows_n0, S.rows_n1, pass, fF, tau, ad));
  if (S.nfsmall) CK(launch_fd_small<double>(s, S.fsmall, S.nfsmall, fF, tau, ad));
  const int epi3 = add ? EPI_ADD : EPI_ASSIGN;
  const int tepi[4] = {EPI_STORE, EPI_MUL, EPI_STORE, epi3};
  for (int st = 0; st < 4; ++st) {
    const LockTcStage& t = S.tc[st];
    if (!t.batch) continue;
    CK((launch_tc_digits<7, double, double>(s, t.d, t.batch, t.pstart, t.panels)));
    CK((launch_gemm_tc<7, double, double>(s, t.d, t.batch, t.tstart, t.tiles, tepi[st], st == 3 ? tau : 1.0, k->err)));
    lk_count(k, 2, t.flops, t.exec_flops);
  }
  for (int st = 0; st < 4; ++st) {
    const LockStackStage& t = S.sk[st];
    if (!t.batch) continue;
    CK(launch_tc_digits_stack(s, t.d, t.batch, t.pstart, t.panels));
    CK(launch_gemm_tc_stack(s, t.d, t.batch, t.tstart, t.tiles, tepi[st], st == 3 ? tau : 1.0, k->err));
    lk_count(k, 2, t.flops, t.exec_flops);
  }
  const bool ta[4] = {true, false, false, false}, tb[4] = {false, false, false, true};
  for (int st = 0; st < 4; ++st)
    for (const auto& g : S.st[st]) {
      CK(launch_gemm<double>(s, g.d, g.batch, g.maxM, g.maxN, ta[st], tb[st], tepi[st], st == 3 ? tau : 1.0, g.R));
      lk_count(k, 1, g.flops);
    }
}

// z = Multigrid(L_q, 0, r) for every problem (Algorithm 1, V-cycle), depth by depth.
void lk_cycle(Lockstep* k, cudaStream_t s) {
  for (int d = 0; d < k->depths; ++d) {
    const LockDepth& D = k->dep[d];
    for (int i = 0; i < k->nu; ++i) {
      if (i == 0) {
        lk_smooth(k, s, D.sm[0], true, false);  // u = 0: the residual is f itself
      } else {
        lk_res(k, s, D);
        lk_smooth(k, s, D.sm[1], false, true);
      }
    }
    lk_res(k, s, D);
    CK(launch_transfer_2d_b<double>(s, D.rst, D.nx, D.r_out0, D.r_out1, D.r_w1, 0));
    CK(launch_coarse_solve_b<double>(s, D.coarse, D.ncoarse, D.coarse_n));
    lk_count(k, 1 + (D.ncoarse ? 1 : 0), D.x_flops + D.coarse_flops);
  }
  for (int d = k->depths - 1; d >= 0; --d) {
    const LockDepth& D = k->dep[d];
    CK(launch_transfer_2d_b<double>(s, D.pro, D.nx, D.p_out0, D.p_out1, D.p_w1, 1));
    lk_count(k, 1, 2.0 * D.x_flops);
    for (int i = 0; i < k->nu; ++i) {
      lk_res(k, s, D);
      lk_smooth(k, s, D.sm[1], false, true);
    }
  }
}

// One PCG step of every problem (updates masked for the problems that have stopped): z = B r,
// beta, p, w = A p, alpha, x, r, ||r||.
void lk_body(Lockstep* k, cudaStream_t s, bool with_precondition) {
  if (with_precondition) {
    lk_cycle(k, s);
    CK(launch_dot_b<double>(s, k->v_fu, k->nprob, 2, k->partials));
    CK(launch_pcg_p_b<double>(s, k->v_pz, k->nprob, k->max_T, k->active));
    lk_count(k, 4, 0.0);
  }
  CK(launch_kron_apply_2d_b<double>(s, k->kry, k->nkry, k->kry_n0, k->kry_n1, k->kry_p));
  CK(launch_dot_b<double>(s, k->v_pw, k->nprob, 1, k->partials));
  CK(launch_pcg_xr_b<double>(s, k->v_xr, k->nprob, k->max_T, k->active));
  CK(launch_norm2_dist_b<double>(s, k->v_nrm, k->nprob, 3, k->partials));
  lk_count(k, 6, k->kry_flops + k->vec_flops);
}

}  // namespace

// Solves every problem of the batch from x[q] (in: x_0, out: x) for rhs b[q] to the relative
// tolerance tol, in lockstep on stream s; res and status (may be NULL) per problem.
igamg_status lockstep_solve(Lockstep* k, cudaStream_t s, const double* const* b, double* const* x, double tol,
                            igamg_result* res, igamg_status* status) {
  const double t0 = now_ms();
  const int n = k->nprob;
  std::vector<igamg_status> st(n, IGAMG_OK);
  std::vector<int> its(n, 0);
  std::vector<double> rr0(n, 0.0), rel(n, 1.0);
  k->launches = 0;
  k->flops = k->mma_flops = 0.0;
  try {
    // per-solve jobs: the caller's global vectors into the tile layout, and back
    std::vector<NodeJobT<double>> gd, ga, back;
    std::vector<VecJobT<double>> zero, keep, fin;
    std::vector<KronJobT<double>> r0;
    int64_t maxN = 0;
    int n0 = 0, n1 = 0, pm = 0;
    for (int q = 0; q < n; ++q) {
      const LockMember& m = k->mb[q];
      igamg_ctx* c = m.c;
      Level& L = c->lv.back();
      const int64_t T = L.topo.T, N = L.topo.N;
      maxN = std::max(maxN, N);
      NodeJobT<double> j{};
      j.n = N;
      j.ptr = L.g2t_ptr;
      j.idx = L.g2t;
      j.G = const_cast<double*>(b[q]);
      j.u = m.Bt();
      gd.push_back(j);
      j.G = x[q];
      j.u = m.X();
      ga.push_back(j);
      NodeJobT<double> bk{};
      bk.n = N;
      bk.ptr = L.g2t_ptr;
      bk.idx = L.g2t;
      bk.v = m.X();
      bk.G = x[q];
      back.push_back(bk);
      zero.push_back(VecJobT<double>{T, nullptr, nullptr, nullptr, m.Bt(), nullptr, nullptr, nullptr});
      zero.push_back(VecJobT<double>{T, nullptr, nullptr, nullptr, m.X(), nullptr, nullptr, nullptr});
      keep.push_back(VecJobT<double>{T, nullptr, nullptr, nullptr, m.Rr(), m.X(), nullptr, nullptr});
      fin.push_back(VecJobT<double>{T, nullptr, nullptr, nullptr, m.X(), m.Rr(), nullptr, nullptr});
      for (const auto& kd : L.kd_h) r0.push_back(KronJobT<double>{kd, L.active, m.X(), m.Bt(), m.tr(L.n64.F)});
      n0 = std::max(n0, L.max_n[0]);
      n1 = std::max(n1, L.max_n[1]);
      pm = std::max(pm, L.max_p);
    }
    DevMem tmp;
    auto up = [&](auto& h) {
      using V = typename std::decay<decltype(h)>::type::value_type;
      V* d = tmp.alloc<V>(h.size());
      CK(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice, s));
      return d;
    };
    struct Guard {
      DevMem& m;
      cudaStream_t s;
      ~Guard() {
        cudaStreamSynchronize(s);
        m.release();
      }
    } guard{tmp, s};
    auto* d_gd = up(gd);
    auto* d_ga = up(ga);
    auto* d_back = up(back);
    auto* d_zero = up(zero);
    auto* d_keep = up(keep);
    auto* d_fin = up(fin);
    auto* d_r0 = up(r0);
    // d = solution of A d = b - A x0 from d = 0; x = x0 + d (Rr holds x0)
    CK(launch_copy_b<double>(s, d_zero, 2 * n, k->max_T, 1));
    CK(launch_global_to_tile_b<double>(s, d_gd, n, maxN, 1));
    CK(launch_global_to_tile_b<double>(s, d_ga, n, maxN, 0));
    CK(launch_kron_apply_2d_b<double>(s, d_r0, int(r0.size()), n0, n1, pm));
    CK(launch_copy_b<double>(s, d_keep, n, k->max_T, 0));
    CK(launch_copy_b<double>(s, d_zero + 0, 2 * n, k->max_T, 1));  // Bt and X: X = 0 (Bt no longer needed)
    CK(launch_norm2_dist_b<double>(s, k->v_nrm, n, 3, k->partials));
    CK(cudaMemcpyAsync(k->h_scal, k->scal, sizeof(double) * 8 * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int live = 0;
    for (int q = 0; q < n; ++q) {
      rr0[q] = k->h_scal[8 * q + 3];
      if (!std::isfinite(rr0[q])) st[q] = IGAMG_ERR_NUMERIC;
      const bool go = st[q] == IGAMG_OK && rr0[q] != 0.0 && k->ctx[q]->opt.max_iter > 0 && !(tol > 0 && 1.0 <= tol);
      k->h_active[q] = go ? 1 : 0;
      live += go;
      if (rr0[q] == 0.0) rel[q] = 0.0;
    }
    if (live) {
      CK(cudaMemcpyAsync(k->active, k->h_active, sizeof(int) * n, cudaMemcpyHostToDevice, s));
      lk_cycle(k, s);
      CK(launch_copy_b<double>(s, k->v_cpu, n, k->max_T, 0));
      CK(launch_dot_b<double>(s, k->v_fu, n, 0, k->partials));
    }
    bool first = true;
    while (live) {
      if (first) {
        lk_body(k, s, false);
        first = false;
      } else {
        if (!k->iter) {  // the step touches fixed buffers only: captured once, replayed
          const int64_t l0 = k->launches;
          const double f0 = k->flops, m0 = k->mma_flops;
          cudaGraph_t g = nullptr;
          CK(cudaStreamBeginCapture(k->cap, cudaStreamCaptureModeRelaxed));
          try {
            lk_body(k, k->cap, true);
          } catch (...) {
            cudaGraph_t dead = nullptr;
            cudaStreamEndCapture(k->cap, &dead);
            if (dead) cudaGraphDestroy(dead);
            throw;
          }
          CK(cudaStreamEndCapture(k->cap, &g));
          CK(cudaGraphInstantiate(&k->iter, g, 0));
          CK(cudaGraphDestroy(g));
          k->it_launches = k->launches - l0;  // the capture launched nothing: count per replay
          k->it_flops = k->flops - f0;
          k->it_mma_flops = k->mma_flops - m0;
          k->launches = l0;
          k->flops = f0;
          k->mma_flops = m0;
        }
        CK(cudaGraphLaunch(k->iter, s));
        lk_count(k, int(k->it_launches), k->it_flops, k->it_mma_flops);
      }
      CK(cudaMemcpyAsync(k->h_scal, k->scal, sizeof(double) * 8 * n, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      bool changed = false;
      for (int q = 0; q < n; ++q) {
        if (!k->h_active[q]) continue;
        ++its[q];
        const double rr = k->h_scal[8 * q + 3];
        if (!std::isfinite(rr)) {
          st[q] = IGAMG_ERR_NUMERIC;
        } else {
          rel[q] = std::sqrt(rr / rr0[q]);
          if (!((tol > 0 && rel[q] <= tol) || its[q] >= k->ctx[q]->opt.max_iter)) continue;
        }
        k->h_active[q] = 0;
        --live;
        changed = true;
      }
      if (changed && live) CK(cudaMemcpyAsync(k->active, k->h_active, sizeof(int) * n, cudaMemcpyHostToDevice, s));
    }
    CK(launch_copy_b<double>(s, d_fin, n, k->max_T, 2));
    CK(launch_tile_to_global_b<double>(s, d_back, n, maxN, 0));
    CK(cudaStreamSynchronize(s));
    int e = 0;
    CK(cudaMemcpy(&e, k->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) throw Fail{IGAMG_ERR_TIMEOUT, "a tensor-core contraction timed out waiting for its MMAs"};
  } catch (const Fail& f) {
    set_context_free_error("lockstep batch: " + f.msg);
    for (int q = 0; q < n; ++q) {
      if (status) status[q] = f.code;
      if (res) res[q] = igamg_result{};
    }
    return f.code;
  }
  const double t = now_ms() - t0;
  igamg_status worst = IGAMG_OK;
  for (int q = 0; q < n; ++q) {
    if (st[q] == IGAMG_OK && tol > 0 && rel[q] > tol) st[q] = IGAMG_ERR_NOT_CONVERGED;
    if (status) status[q] = st[q];
    if (res) {
      igamg_result& r = res[q];
      r.iters = its[q];
      r.outer_iters = 1;
      r.relres = rel[q];
      r.t_setup_ms = k->ctx[q]->t_setup_ms;
      r.t_assemble_ms = k->ctx[q]->t_assemble_ms;
      r.t_solve_ms = t;
    }
    if (st[q] != IGAMG_OK && (worst == IGAMG_OK || worst == IGAMG_ERR_NOT_CONVERGED)) worst = st[q];
  }
  return worst;
}

void lockstep_stats(const Lockstep* k, int64_t* launches, double* flops, double* mma_flops) {
  *launches = k->launches;
  *flops = k->flops;
  *mma_flops = k->mma_flops;
}

Lockstep* lockstep_build(const std::vector<igamg_ctx*>& ctx, std::string* why) {
  std::vector<LockMember> mb;
  for (igamg_ctx* c : ctx) mb.push_back(LockMember{c, nullptr});
  return lockstep_build(mb, why, false);
}

// Whether the lockstep engine can run several right-hand sides of this context together
// (2D, every level above the coarsest made of rectangle patches with fused transfers,
// V-cycle); a precision-variant context qualifies and runs its FP64 numerics.
bool ctx_multi_ok(const igamg_ctx* c) {
  if (c->pd.dim != 2 || c->opt.mu != 1 || c->lv.size() < 2) return false;
  for (size_t l = 1; l < c->lv.size(); ++l) {
    const Level& L = c->lv[l];
    if (!L.kron || !L.n64.r2 || !L.n64.p2) return false;
  }
  return true;
}

namespace {

// Work copies 1 .. n-1 of a context: every registered work array with its current content
// (so that a copy starts in the state of the context), the Krylov vectors and the FP64
// digit scratch; allocated once and kept until the context is freed.
void ensure_copies(igamg_ctx* c, int n) {
  const cudaStream_t s = c->stream;
  const int64_t Tf = c->lv.back().topo.T;
  while (int(c->copies.size()) < n - 1) {
    WorkCopy w;
    for (const auto& r : c->reg) {
      double* base = std::get<0>(r);
      const int64_t cnt = std::get<1>(r);
      double* p = base;
      if (!std::get<2>(r)) {
        p = c->mem.alloc<double>(size_t(std::max<int64_t>(cnt, 1)));
        if (cnt > 0) CK(cudaMemcpyAsync(p, base, size_t(cnt) * sizeof(double), cudaMemcpyDeviceToDevice, s));
      }
      w.tw.emplace_back(base, cnt, p);
    }
    std::sort(w.tw.begin(), w.tw.end(), [](const auto& a, const auto& b) { return std::get<0>(a) < std::get<0>(b); });
    w.X = c->mem.alloc<double>(size_t(Tf));
    w.Pv = c->mem.alloc<double>(size_t(Tf));
    w.W = c->mem.alloc<double>(size_t(Tf));
    w.Bt = c->mem.alloc<double>(size_t(Tf));
    w.Rr = c->mem.alloc<double>(size_t(Tf));
    for (int k = 0; k < 2; ++k) {
      if (c->dig64[k]) w.dig[k] = c->mem.alloc<__nv_bfloat16>(size_t(c->dig64[k]));
      if (c->tau64[k]) w.tau[k] = c->mem.alloc<int>(size_t(c->tau64[k]));
    }
    if (c->sdig) w.sdig = c->mem.alloc<__nv_bfloat16>(size_t(c->sdig));
    if (c->stau) w.stau = c->mem.alloc<int>(size_t(c->stau));
    c->copies.push_back(std::move(w));
  }
  CK(cudaStreamSynchronize(s));
}

}  // namespace

// nrhs right-hand sides of one context solved together by the lockstep engine over the
// context and nrhs - 1 work copies (one launch per step for all of them, the operator's
// constant arrays shared); NULL when the context is outside the engine's scope.  Engines are
// kept per nrhs.
Lockstep* multi_engine(igamg_ctx* c, int nrhs) {
  auto it = c->multi.find(nrhs);
  if (it != c->multi.end()) return it->second;
  Lockstep* k = nullptr;
  if (ctx_multi_ok(c)) {
    ensure_copies(c, nrhs);
    std::vector<LockMember> mb{LockMember{c, nullptr}};
    for (int q = 1; q < nrhs; ++q) mb.push_back(LockMember{c, &c->copies[size_t(q - 1)]});
    std::string why;
    k = lockstep_build(mb, &why, true);
  }
  c->multi[nrhs] = k;
  return k;
}

}  // namespace igamg

extern "C" {

igamg_status igamg_default_options(igamg_options* opt) {
  if (!opt) return IGAMG_ERR_ARG;
  opt->tau = 0.25;
  opt->sigma_scale = 5.0;
  opt->nu = 1;
  opt->mu = 1;
  opt->max_iter = 500;
  opt->precision = IGAMG_FP64;
  opt->inner_tol = 1e-4;
  opt->fd_engine = 0;
  opt->batch_engine = 0;
  opt->graphs = 1;
  opt->apply_engine = 0;
  opt->autotune = 1;
  return IGAMG_OK;
}

igamg_status igamg_setup(const igamg_problem* prob, const igamg_options* opt, void* cuda_stream,
                         igamg_ctx** out) {
  if (!out) return IGAMG_ERR_ARG;
  *out = nullptr;
  if (!prob) { g_setup_error = "problem is NULL"; return IGAMG_ERR_ARG; }
  igamg_ctx* c = new igamg_ctx();
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->verbose = std::getenv("IGAMG_VERBOSE") != nullptr;
  igamg_default_options(&c->opt);
  if (opt) c->opt = *opt;
  double t0 = now_ms();
  try {
    if (c->opt.precision < IGAMG_FP64 || c->opt.precision > IGAMG_BF16) throw Fail{IGAMG_ERR_ARG, "bad precision"};
    if (c->opt.fd_engine < 0 || c->opt.fd_engine > 4) throw Fail{IGAMG_ERR_ARG, "bad fd_engine"};
    if (c->opt.precision != IGAMG_FP64 && !(c->opt.inner_tol > 0 && c->opt.inner_tol < 1))
      throw Fail{IGAMG_ERR_ARG, "inner_tol must be in (0, 1)"};
    if (c->opt.nu < 1 || c->opt.mu < 1 || c->opt.mu > 2 || c->opt.max_iter < 0 || !(c->opt.tau > 0))
      throw Fail{IGAMG_ERR_ARG, "bad options"};
    // the interface stream exists before the autotuner times smoothers
    CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming));
    int code = 0;
    std::string e = parse_problem(prob->dim, prob->num_patches, prob->degree, prob->num_knots, prob->knots,
                                  prob->geo_degree, prob->geo_num_ctrl, prob->geo_ctrl, prob->side_bc,
                                  prob->num_levels, c->pd, &code);
    if (!e.empty()) throw Fail{igamg_status(code), e};
    build_levels(c);
    if (c->opt.autotune && c->opt.fd_engine == 0) autotune(c);
    if (c->opt.precision != IGAMG_FP64) {
      build_low(c, c->opt.precision == IGAMG_BF16);
      if (c->opt.autotune && c->opt.fd_engine == 0) autotune_low(c);
    }
  } catch (const Fail& e) {
    g_setup_error = e.msg;
    if (c->side) {
      cudaStreamSynchronize(c->side);
      cudaStreamDestroy(c->side);
    }
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    if (c->join_ev) cudaEventDestroy(c->join_ev);
    if (c->stream) cudaStreamSynchronize(c->stream);
    c->mem.release();
    if (c->h_scal) cudaFreeHost(c->h_scal);
    delete c;
    return e.code;
  }
  c->t_setup_ms = now_ms() - t0;
  *out = c;
  return IGAMG_OK;
}

igamg_status igamg_num_dofs(const igamg_ctx* c, int level, int64_t* n) {
  if (!c || !n) return IGAMG_ERR_ARG;
  int NL = int(c->lv.size());
  int l = level == -1 ? NL - 1 : level;
  if (l < 0 || l >= NL) return IGAMG_ERR_ARG;
  *n = c->lv[l].topo.N;
  return IGAMG_OK;
}

igamg_status igamg_device_bytes(const igamg_ctx* c, int64_t* bytes) {
  if (!c || !bytes) return IGAMG_ERR_ARG;
  *bytes = int64_t(c->mem.bytes());
  return IGAMG_OK;
}

igamg_status igamg_num_local(const igamg_ctx* c, int level, int64_t* n) {
  if (!c || !n) return IGAMG_ERR_ARG;
  int NL = int(c->lv.size());
  int l = level == -1 ? NL - 1 : level;
  if (l < 0 || l >= NL) return IGAMG_ERR_ARG;
  *n = c->lv[l].topo.T;
  return IGAMG_OK;
}

igamg_status igamg_dof_map(const igamg_ctx* c, int level, int64_t* l2g) {
  if (!c || !l2g) return IGAMG_ERR_ARG;
  int NL = int(c->lv.size());
  int l = level == -1 ? NL - 1 : level;
  if (l < 0 || l >= NL) return IGAMG_ERR_ARG;
  std::memcpy(l2g, c->lv[l].topo.l2g.data(), c->lv[l].topo.T * sizeof(int64_t));
  return IGAMG_OK;
}

igamg_status igamg_greville_points(const igamg_ctx* c, int level, double* xyz) {
  if (!c || !xyz) return IGAMG_ERR_ARG;
  int NL = int(c->lv.size());
  int l = level == -1 ? NL - 1 : level;
  if (l < 0 || l >= NL) return IGAMG_ERR_ARG;
  const LevelTopo& T = c->lv[l].topo;
  const int d = c->pd.dim, nc = 1 << d;
  for (int64_t g = 0; g < T.N; ++g) {
    int64_t t = T.g2t[T.g2t_ptr[g]];
    int k = int(std::upper_bound(T.off.begin(), T.off.end(), t) - T.off.begin()) - 1;
    int64_t li = t - T.off[k];
    double xi[3] = {0, 0, 0};
    for (int j = d - 1; j >= 0; --j) {
      int n = T.n[k * d + j], p = c->pd.p[k * d + j], m = n - p;
      int i = int(li % n);
      li /= n;
      std::vector<double> kn = uniform_knots(m, p);
      double s = 0.0;
      for (int q = 1; q <= p; ++q) s += kn[i + q];
      xi[j] = s / p;
    }
    for (int a = 0; a < d; ++a) {
      double v = 0.0;
      for (int cc = 0; cc < nc; ++cc) {
        double w = 1.0;
        for (int j = 0; j < d; ++j) w *= ((cc >> j) & 1) ? xi[j] : 1.0 - xi[j];
        v += w * c->pd.corners[(size_t(k) * nc + cc) * d + a];
      }
      xyz[g * d + a] = v;
    }
  }
  return IGAMG_OK;
}

igamg_status igamg_apply(igamg_ctx* c, int level, const double* x, double* y) {
  return guarded(c, [&]() {
    if (!x || !y) throw Fail{IGAMG_ERR_ARG, "NULL vector"};
    int l = level_index(c, level);
    Level& L = c->lv[l];
    to_acc(c, l, x, L.n64.U);
    residual<double>(c, l, nullptr, L.n64.U, L.n64.R);
    from_dist(c, l, L.n64.R, y);
    return IGAMG_OK;
  });
}

igamg_status igamg_smooth(igamg_ctx* c, int level, const double* r, double* z) {
  return guarded(c, [&]() {
    if (!r || !z) throw Fail{IGAMG_ERR_ARG, "NULL vector"};
    int l = level_index(c, level);
    if (l < 1) throw Fail{IGAMG_ERR_ARG, "the smoother exists on levels >= 1"};
    Level& L = c->lv[l];
    to_dist(c, l, r, L.n64.R);
    CK(cudaMemsetAsync(L.n64.U, 0, L.topo.T * sizeof(double), c->stream));
    smooth<double>(c, l, false, false);
    CK(launch_axpby(c->stream, L.topo.T, 0.0, L.n64.U, 1.0 / c->opt.tau, L.n64.U));
    from_acc(c, l, L.n64.U, z);
    return IGAMG_OK;
  });
}

igamg_status igamg_restrict(igamg_ctx* c, int level, const double* r, double* rc) {
  return guarded(c, [&]() {
    if (!r || !rc) throw Fail{IGAMG_ERR_ARG, "NULL vector"};
    int l = level_index(c, level);
    if (l < 1) throw Fail{IGAMG_ERR_ARG, "restriction needs level >= 1"};
    Level& L = c->lv[l];
    Level& C = c->lv[l - 1];
    to_dist(c, l, r, L.n64.R);
    restrict_to_coarse<double>(c, l, L.n64.R);
    from_dist(c, l - 1, C.n64.F, rc);
    return IGAMG_OK;
  });
}

igamg_status igamg_prolong(igamg_ctx* c, int level, const double* uc, double* u) {
  return guarded(c, [&]() {
    if (!uc || !u) throw Fail{IGAMG_ERR_ARG, "NULL vector"};
    int l = level_index(c, level);
    if (l < 1) throw Fail{IGAMG_ERR_ARG, "prolongation needs level >= 1"};
    Level& L = c->lv[l];
    Level& C = c->lv[l - 1];
    to_acc(c, l - 1, uc, C.n64.U);
    CK(cudaMemsetAsync(L.n64.U, 0, L.topo.T * sizeof(double), c->stream));
    prolong_add<double>(c, l);
    from_acc(c, l, L.n64.U, u);
    return IGAMG_OK;
  });
}

igamg_status igamg_coarse_solve(igamg_ctx* c, const double* r, double* x) {
  return guarded(c, [&]() {
    if (!r || !x) throw Fail{IGAMG_ERR_ARG, "NULL vector"};
    to_dist(c, 0, r, c->lv[0].n64.F);
    coarse_solve<double>(c);
    from_acc(c, 0, c->lv[0].n64.U, x);
    return IGAMG_OK;
  });
}

igamg_status igamg_precondition(igamg_ctx* c, const double* r, double* z) {
  return guarded(c, [&]() {
    if (!r || !z) throw Fail{IGAMG_ERR_ARG, "NULL vector"};
    int Lf = int(c->lv.size()) - 1;
    to_dist(c, Lf, r, c->lv[Lf].n64.F);
    precondition<double>(c);
    from_acc(c, Lf, c->lv[Lf].n64.U, z);
    return IGAMG_OK;
  });
}

igamg_status igamg_cycle_time(igamg_ctx* c, const double* r, int reps, double* ms, double* bytes) {
  return guarded(c, [&]() {
    if (!r || !ms || reps < 1) throw Fail{IGAMG_ERR_ARG, "bad arguments"};
    const int Lf = int(c->lv.size()) - 1;
    Level& L = c->lv[Lf];
    cudaStream_t s = c->stream;
    const bool low = c->low;
    to_dist(c, Lf, r, L.n64.F);
    if (low) {
      CK(launch_canonicalize<double>(s, L.n_if, L.if_ptr, L.if_idx, L.n64.F));
      CK(launch_convert_f64_f32(s, L.topo.T, L.n64.F, 1.0, L.n32.F));
    }
    auto cycle = [&]() {
      if (low) precondition<float>(c);
      else precondition<double>(c);
    };
    // algorithmic bytes of one cycle: one cycle launched one by one with the counters on
    const bool prof0 = c->prof;
    const unsigned mask0 = c->prof_mask;
    double b0[8];
    std::copy(c->prof_bytes, c->prof_bytes + 8, b0);
    c->prof = true;
    c->prof_mask = 0;
    cycle();
    double by = 0.0;
    for (int k = 0; k < 6; ++k) by += c->prof_bytes[k] - b0[k];
    std::copy(b0, b0 + 8, c->prof_bytes);
    c->prof = false;
    // the cycle as the solve runs it: captured once as a graph, replayed
    graph_run(c, low ? 3 : 2, cycle);
    graph_run(c, low ? 3 : 2, cycle);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, s));
    for (int i = 0; i < reps; ++i) graph_run(c, low ? 3 : 2, cycle);
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->prof = prof0;
    c->prof_mask = mask0;
    check_tc(c);
    *ms = double(t) / reps;
    if (bytes) *bytes = by;
    return IGAMG_OK;
  });
}

igamg_status igamg_rhs_from_coefs(igamg_ctx* c, const double* coef, double* rhs) {
  return guarded(c, [&]() -> igamg_status {
    if (!coef || !rhs) throw Fail{IGAMG_ERR_ARG, "NULL vector"};
    // b = M_geo c: assemble the geometry mass bands of the finest level into a temporary
    // band array (same layout as the stiffness), apply them patch-locally, sum the copies.
    int Lf = int(c->lv.size()) - 1;
    Level& L = c->lv[Lf];
    cudaStream_t s = c->stream;
    double* mband = nullptr;
    CK(cudaMallocAsync(&mband, size_t(L.band_doubles) * sizeof(double), s));
    CK(cudaMemsetAsync(mband, 0, size_t(L.band_doubles) * sizeof(double), s));
    size_t mark = c->mem.ptrs.size();
    std::map<std::tuple<int, int>, Tables1D> tabs;
    std::map<std::tuple<int, int>, DevTables> dtabs;
    double* dcorn = c->mem.upload(c->pd.corners, s);
    assemble_level(c, L, dtabs, tabs, dcorn, true, mband);
    to_acc(c, Lf, coef, L.n64.U);
    if (c->pd.dim == 2)
      CK((launch_band_apply_2d<double, double>(s, L.pd, c->pd.K, L.max_n[0], L.max_n[1], L.max_p, mband, L.n64.U,
                                                nullptr, L.n64.R)));
    else
      CK((launch_band_apply_3d<double, double>(s, L.pd, c->pd.K, L.max_n, L.max_p, mband, L.n64.U, nullptr,
                                                L.n64.R)));
    from_dist(c, Lf, L.n64.R, rhs);
    CK(cudaFreeAsync(mband, s));
    CK(cudaStreamSynchronize(s));
    c->mem.truncate(mark);  // temporary tables
    return IGAMG_OK;
  });
}

igamg_status igamg_fd_apply(int n0, int n1, const double* U0, const double* U1, const double* Dinv,
                            const double* R, int ldr, double tau, double* Z, int ldz, double* scratch,
                            void* cuda_stream) {
  if (n0 < 1 || n1 < 1 || ldr < n1 || ldz < n1 || !U0 || !U1 || !Dinv || !R || !Z || !scratch) {
    g_setup_error = "igamg_fd_apply: sizes must be >= 1, strides >= n1, pointers non-NULL";
    return IGAMG_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  double* T = scratch;
  double* Y = scratch + int64_t(n0) * n1;
  try {
    CK(launch_gemm_one(s, GemmDesc{U0, R, T, nullptr, n0, ldr, n1, 0, n0, n1, n0}, true, false, EPI_STORE, 1.0));
    CK(launch_gemm_one(s, GemmDesc{T, U1, Y, Dinv, n1, n1, n1, n1, n0, n1, n1}, false, false, EPI_MUL, 1.0));
    CK(launch_gemm_one(s, GemmDesc{U0, Y, T, nullptr, n0, n1, n1, 0, n0, n1, n0}, false, false, EPI_STORE, 1.0));
    CK(launch_gemm_one(s, GemmDesc{T, U1, Z, nullptr, n1, n1, ldz, 0, n0, n1, n1}, false, true, EPI_ASSIGN, tau));
  } catch (const Fail& e) {
    g_setup_error = e.msg;
    return e.code;
  }
  return IGAMG_OK;
}

igamg_status igamg_profile_enable(igamg_ctx* c, int enable) {
  return guarded(c, [&]() {
    CK(cudaStreamSynchronize(c->stream));
    prof_collect(c);
    c->prof = enable != 0;
    c->prof_mask = unsigned(enable);
    for (int i = 0; i < 8; ++i) {
      c->prof_launch[i] = 0;
      c->prof_ms[i] = c->prof_flops[i] = c->prof_bytes[i] = 0.0;
    }
    return IGAMG_OK;
  });
}

igamg_status igamg_profile_read(igamg_ctx* c, int cls, int64_t* launches, double* ms, double* flops,
                                double* bytes) {
  return guarded(c, [&]() {
    if (cls < 0 || cls >= 8 || !launches || !ms || !flops || !bytes) throw Fail{IGAMG_ERR_ARG, "bad arguments"};
    CK(cudaStreamSynchronize(c->stream));
    prof_collect(c);
    *launches = c->prof_launch[cls];
    *ms = c->prof_ms[cls];
    *flops = c->prof_flops[cls];
    *bytes = c->prof_bytes[cls];
    return IGAMG_OK;
  });
}

igamg_status igamg_solve(igamg_ctx* c, const double* b, double* x, double tol, igamg_result* res) {
  return guarded(c, [&]() {
    if (!b || !x || !(tol >= 0)) throw Fail{IGAMG_ERR_ARG, "bad arguments"};
    return c->low ? pcg_refined(c, b, x, tol, res) : pcg(c, b, x, tol, res);
  });
}

igamg_status igamg_solve_multi(igamg_ctx* c, int nrhs, const double* const* b, double* const* x, double tol,
                               igamg_result* res, igamg_status* status) {
  if (!c) return IGAMG_ERR_ARG;
  if (nrhs < 1 || !b || !x || !(tol >= 0)) {
    c->err = "igamg_solve_multi: need nrhs >= 1, b and x arrays, tol >= 0";
    return IGAMG_ERR_ARG;
  }
  for (int q = 0; q < nrhs; ++q)
    if (!b[q] || !x[q]) {
      c->err = "igamg_solve_multi: null right-hand side or solution pointer";
      return IGAMG_ERR_ARG;
    }
  igamg::Lockstep* k = nullptr;
  if (nrhs > 1) {  // an engine that cannot be built (e.g. no memory for the copies): one at a time
    if (guarded(c, [&]() {
          k = igamg::multi_engine(c, nrhs);
          return IGAMG_OK;
        }) != IGAMG_OK) {
      k = nullptr;
      c->multi[nrhs] = nullptr;  // not retried for this count
      cudaGetLastError();        // a failed allocation leaves no error for the next launch check
    }
  }
  if (!k) {  // one at a time
    igamg_status worst = IGAMG_OK;
    for (int q = 0; q < nrhs; ++q) {
      igamg_result r{};
      igamg_status st = igamg_solve(c, b[q], x[q], tol, &r);
      if (res) res[q] = r;
      if (status) status[q] = st;
      if (st != IGAMG_OK && (worst == IGAMG_OK || worst == IGAMG_ERR_NOT_CONVERGED)) worst = st;
    }
    return worst;
  }
  igamg_status st = igamg::lockstep_solve(k, c->stream, b, x, tol, res, status);
  if (st != IGAMG_OK && st != IGAMG_ERR_NOT_CONVERGED) c->err = igamg_last_error(nullptr);
  return st;
}

igamg_status igamg_solve_host(igamg_ctx* c, const double* bh, double* xh, double tol, igamg_result* res) {
  return guarded(c, [&]() {
    if (!bh || !xh || !(tol >= 0)) throw Fail{IGAMG_ERR_ARG, "bad arguments"};
    int64_t N = c->lv.back().topo.N;
    double t0 = now_ms();
    double *db = nullptr, *dx = nullptr;
    CK(cudaMallocAsync(&db, N * sizeof(double), c->stream));
    CK(cudaMallocAsync(&dx, N * sizeof(double), c->stream));
    CK(cudaMemcpyAsync(db, bh, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(dx, xh, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    igamg_status st = c->low ? pcg_refined(c, db, dx, tol, res) : pcg(c, db, dx, tol, res);
    CK(cudaMemcpyAsync(xh, dx, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaFreeAsync(db, c->stream));
    CK(cudaFreeAsync(dx, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (res) res->t_solve_ms = now_ms() - t0;
    return st;
  });
}

igamg_status igamg_sync(igamg_ctx* c) {
  return guarded(c, [&]() {
    CK(cudaStreamSynchronize(c->stream));
    return IGAMG_OK;
  });
}

igamg_status igamg_free(igamg_ctx* c) {
  if (!c) return IGAMG_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  for (int gi = 0; gi < igamg_ctx::kGraphSlots; ++gi) {
    if (c->iter_graph[gi]) cudaGraphExecDestroy(c->iter_graph[gi]);
    for (auto& t : c->graph_ev[gi]) {
      cudaEventDestroy(std::get<1>(t));
      cudaEventDestroy(std::get<2>(t));
    }
  }
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaStreamDestroy(c->side);
  }
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->join_ev) cudaEventDestroy(c->join_ev);
  for (auto& t : c->ev_open) {
    cudaEventDestroy(std::get<1>(t));
    cudaEventDestroy(std::get<2>(t));
  }
  for (cudaEvent_t e : c->ev_free) cudaEventDestroy(e);
  for (auto& kv : c->multi) igamg::lockstep_free(kv.second);
  c->mem.release();
  if (c->h_scal) cudaFreeHost(c->h_scal);
  delete c;
  return IGAMG_OK;
}

const char* igamg_last_error(const igamg_ctx* c) {
  if (!c) return g_setup_error.c_str();
  return c->err.empty() ? "no error" : c->err.c_str();
}

}  // extern "C"
