// Context, setup, multigrid cycle (Algorithm 1), PCG (Sec. 4) and the C ABI of igamg.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/igamg.h"
#include "host_math.h"
#include "kernels.cuh"
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
  template <class T>
  T* alloc(size_t count) {
    void* p = nullptr;
    if (count == 0) count = 1;
    CK(cudaMalloc(&p, count * sizeof(T)));
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  template <class T>
  T* upload(const std::vector<T>& h, cudaStream_t s) {
    T* d = alloc<T>(h.size());
    if (!h.empty()) CK(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return d;
  }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
  }
};

struct Smoother1D {  // subspace-corrected mass smoother data of one direction signature
  int len = 0;
  std::vector<double> U;   // len x len, columns = M-orthonormal basis [U~, U^G]
  std::vector<double> mu;  // len
  double* dU = nullptr;
};

struct GemmSet {
  GemmDesc* d = nullptr;
  int batch = 0, maxM = 0, maxN = 0;
  double flops = 0, bytes = 0;  // algorithmic work of one launch
};

struct Level {
  LevelTopo topo;
  std::vector<PatchDev> pd_h;
  PatchDev* pd = nullptr;
  int max_n[3] = {1, 1, 1}, max_p = 1;
  int64_t* l2g = nullptr;
  int64_t *g2t_ptr = nullptr, *g2t = nullptr;
  double* band = nullptr;
  double *F = nullptr, *U = nullptr, *R = nullptr;
  // interior smoother: stage GEMMs; stage 0 reads F or R
  GemmSet st0F, st0R, st1, st2, st3;
  double *fdT = nullptr, *fdY = nullptr;
  // interface pieces
  int64_t n_if = 0;
  int64_t *if_ptr = nullptr, *if_idx = nullptr;
  double *G = nullptr, *Z = nullptr, *Yif = nullptr, *vscale = nullptr;
  GemmSet edgeA, edgeB;  // 1D FD of edge groups
  // transfer from level-1 (valid for level >= 1)
  TransferDev* td = nullptr;
  double* ttmp = nullptr;
  int max_nf = 0, max_nc = 0;
  double apply_flops = 0, band_bytes = 0, xfer_flops = 0, xfer_bytes = 0;
};

}  // namespace

struct igamg_ctx {
  cudaStream_t stream = nullptr;
  igamg_options opt{};
  ProblemDesc pd;
  std::vector<Level> lv;
  DevMem mem;
  double* A0inv = nullptr;
  int64_t N0 = 0;
  double *X = nullptr, *Pv = nullptr, *W = nullptr, *Bt = nullptr, *gtmp = nullptr;
  double *partials = nullptr, *scal = nullptr;
  double* h_scal = nullptr;  // pinned
  std::string err;
  double t_setup_ms = 0, t_assemble_ms = 0;
  // per-class launch accounting (igamg_profile_*)
  bool prof = false;
  int64_t prof_launch[8] = {0};
  double prof_ms[8] = {0}, prof_flops[8] = {0}, prof_bytes[8] = {0};
  std::vector<cudaEvent_t> ev_free;
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> ev_open;
  int cur_cls = -1;
  cudaEvent_t cur_start = nullptr;
};

static thread_local std::string g_setup_error = "no error";

namespace igamg {
// Message returned by igamg_last_error(NULL) on this thread.
void set_context_free_error(const std::string& msg) { g_setup_error = msg; }
}  // namespace igamg

namespace {

enum { CLS_APPLY = 0, CLS_FD = 1, CLS_IFACE = 2, CLS_TRANSFER = 3, CLS_COARSE = 4, CLS_VECTOR = 5 };

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

// Brackets one launch of class `cls` with algorithmic work (flops, bytes).
struct ProfScope {
  igamg_ctx* c;
  int cls;
  cudaEvent_t a = nullptr;
  ProfScope(igamg_ctx* c_, int cls_, double flops, double bytes, int launches = 1) : c(c_), cls(cls_) {
    if (!c->prof) return;
    c->prof_launch[cls] += launches;
    c->prof_flops[cls] += flops;
    c->prof_bytes[cls] += bytes;
    a = prof_event(c);
    CK(cudaEventRecord(a, c->stream));
  }
  ~ProfScope() noexcept(false) {
    if (!a) return;
    cudaEvent_t b = prof_event(c);
    CK(cudaEventRecord(b, c->stream));
    c->ev_open.emplace_back(cls, a, b);
  }
};

// Folds completed event pairs into the per-class totals (stream must be synchronised).
void prof_collect(igamg_ctx* c) {
  for (auto& t : c->ev_open) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, std::get<1>(t), std::get<2>(t)));
    c->prof_ms[std::get<0>(t)] += ms;
    c->ev_free.push_back(std::get<1>(t));
    c->ev_free.push_back(std::get<2>(t));
  }
  c->ev_open.clear();
}

double gemm_flops(const std::vector<GemmDesc>& v) {
  double f = 0;
  for (auto& d : v) f += 2.0 * d.M * double(d.N) * d.K;
  return f;
}

void set_gemm(igamg_ctx* c, GemmSet& gs, const std::vector<GemmDesc>& v) {
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

void run_gemm(igamg_ctx* c, const GemmSet& gs, bool ta, bool tb, int epi, double alpha, int cls) {
  if (!gs.batch) return;
  ProfScope ps(c, cls, gs.flops, gs.bytes);
  CK(launch_gemm(c->stream, gs.d, gs.batch, gs.maxM, gs.maxN, ta, tb, epi, alpha));
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

void build_levels(igamg_ctx* c) {
  cudaStream_t s = c->stream;
  const int d = c->pd.dim, K = c->pd.K;
  if (d != 2) throw Fail{IGAMG_ERR_UNSUPPORTED, "this build solves 2D problems only"};
  const int NL = c->pd.levels;
  c->lv.resize(NL);
  std::map<std::tuple<int, int, int, int, double>, Smoother1D> scms;  // (m,p,lo,hi,sigma)
  std::map<std::tuple<int, int>, Tables1D> tabs;
  for (int l = 0; l < NL; ++l) {
    Level& L = c->lv[l];
    int code = 0;
    std::string e = build_level(c->pd, l, L.topo, &code);
    if (!e.empty()) throw Fail{igamg_status(code), e};
    const LevelTopo& T = L.topo;
    // patch descriptors and bands
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
    L.pd = c->mem.upload(L.pd_h, s);
    L.l2g = c->mem.upload(T.l2g, s);
    L.g2t_ptr = c->mem.upload(T.g2t_ptr, s);
    L.g2t = c->mem.upload(T.g2t, s);
    L.band = c->mem.alloc<double>(band_total);
    L.F = c->mem.alloc<double>(T.T);
    L.U = c->mem.alloc<double>(T.T);
    L.R = c->mem.alloc<double>(T.T);
    CK(cudaMemsetAsync(L.F, 0, T.T * sizeof(double), s));
    CK(cudaMemsetAsync(L.U, 0, T.T * sizeof(double), s));
    CK(cudaMemsetAsync(L.R, 0, T.T * sizeof(double), s));
    // assembly (Eq. model:bil) patch by patch
    double ta0 = now_ms();
    {
      int64_t gmax = 0;
      for (auto& P : L.pd_h) gmax = std::max(gmax, int64_t(P.m[0]) * (P.p[0] + 1) * P.m[1] * (P.p[1] + 1) * 4);
      double* G = c->mem.alloc<double>(gmax);
      double* dcorn = c->mem.alloc<double>(c->pd.corners.size());
      CK(cudaMemcpyAsync(dcorn, c->pd.corners.data(), c->pd.corners.size() * sizeof(double),
                         cudaMemcpyHostToDevice, s));
      std::map<std::tuple<int, int>, std::vector<double*>> dtabs;
      for (int k = 0; k < K; ++k) {
        const PatchDev& P = L.pd_h[k];
        double* tp[2][4];
        for (int j = 0; j < 2; ++j) {
          auto key = std::make_tuple(P.m[j], P.p[j]);
          if (!tabs.count(key)) tabs[key] = tables_1d(P.m[j], P.p[j]);
          if (!dtabs.count(key)) {
            const Tables1D& tb = tabs[key];
            dtabs[key] = {c->mem.upload(tb.xq, s), c->mem.upload(tb.wq, s), c->mem.upload(tb.B, s),
                          c->mem.upload(tb.dB, s)};
          }
          for (int q = 0; q < 4; ++q) tp[j][q] = dtabs[key][q];
        }
        if (P.p[0] != P.p[1]) throw Fail{IGAMG_ERR_UNSUPPORTED, "direction-dependent degree"};
        CK(launch_geom_factors_2d(s, dcorn + size_t(k) * 4 * 2, P.m[0], P.m[1], P.p[0] + 1, tp[0][0],
                                  tp[0][1], tp[1][0], tp[1][1], G));
        CK(launch_assemble_2d(s, P, G, tp[0][2], tp[0][3], tp[1][2], tp[1][3], L.l2g, 0, L.band));
      }
      CK(cudaStreamSynchronize(s));
    }
    c->t_assemble_ms += now_ms() - ta0;
    // smoother (levels >= 1)
    if (l >= 1) {
      // interiors
      int64_t fd_total = 0;
      std::vector<GemmDesc> s0F, s0R, s1, s2, s3;
      std::map<std::tuple<int, int, int, int, int, int>, double*> dinv_cache;
      for (const Interior& in : T.interiors) {
        const PatchDev& P = L.pd_h[in.k];
        if (in.len[0] == 0 || in.len[1] == 0) continue;  // empty piece (p = 1, one element)
        Smoother1D* S[2];
        for (int j = 0; j < 2; ++j) {
          double sigma = c->opt.sigma_scale * double(P.m[j]) * double(P.m[j]);
          auto key = std::make_tuple(P.m[j], P.p[j], int(in.drop_lo[j]), int(in.drop_hi[j]), sigma);
          if (!scms.count(key)) scms[key] = build_scms(P.m[j], P.p[j], in.drop_lo[j], in.drop_hi[j], sigma);
          S[j] = &scms[key];
          if (!S[j]->dU) S[j]->dU = c->mem.upload(S[j]->U, s);
          if (S[j]->len != in.len[j]) throw Fail{IGAMG_ERR_NUMERIC, "smoother size mismatch"};
        }
        int n0 = in.len[0], n1 = in.len[1];
        auto dk = std::make_tuple(P.m[0], P.p[0], int(in.drop_lo[0]) + 2 * int(in.drop_hi[0]), P.m[1], P.p[1],
                                  int(in.drop_lo[1]) + 2 * int(in.drop_hi[1]));
        if (!dinv_cache.count(dk)) {
          std::vector<double> Dv(size_t(n0) * n1);
          for (int a = 0; a < n0; ++a)
            for (int b = 0; b < n1; ++b) Dv[size_t(a) * n1 + b] = 1.0 / (S[0]->mu[a] + S[1]->mu[b]);
          dinv_cache[dk] = c->mem.upload(Dv, s);
        }
        double* Dinv = dinv_cache[dk];
        int64_t base = fd_total;
        fd_total += int64_t(n0) * n1;
        int64_t xoff = P.off + int64_t(in.lo[0]) * P.n[1] + in.lo[1];
        // stage descriptors: pointers to T/Y scratch are patched after allocation
        GemmDesc g0{S[0]->dU, nullptr, (double*)(intptr_t)base, nullptr, n0, P.n[1], n1, 0, n0, n1, n0};
        GemmDesc gF = g0, gR = g0;
        gF.B = L.F + xoff;
        gR.B = L.R + xoff;
        s0F.push_back(gF);
        s0R.push_back(gR);
        s1.push_back(GemmDesc{(double*)(intptr_t)base, S[1]->dU, (double*)(intptr_t)base, Dinv, n1, n1, n1, n1,
                              n0, n1, n1});
        s2.push_back(GemmDesc{S[0]->dU, (double*)(intptr_t)base, (double*)(intptr_t)base, nullptr, n0, n1, n1, 0,
                              n0, n1, n0});
        s3.push_back(GemmDesc{(double*)(intptr_t)base, S[1]->dU, L.U + xoff, nullptr, n1, n1, P.n[1], 0, n0, n1,
                              n1});
      }
      L.fdT = c->mem.alloc<double>(fd_total);
      L.fdY = c->mem.alloc<double>(fd_total);
      for (auto& g : s0F) g.C = L.fdT + (intptr_t)g.C;
      for (auto& g : s0R) g.C = L.fdT + (intptr_t)g.C;
      for (auto& g : s1) { g.A = L.fdT + (intptr_t)g.A; g.C = L.fdY + (intptr_t)g.C; }
      for (auto& g : s2) { g.B = L.fdY + (intptr_t)g.B; g.C = L.fdT + (intptr_t)g.C; }
      for (auto& g : s3) g.A = L.fdT + (intptr_t)g.A;
      set_gemm(c, L.st0F, s0F);
      set_gemm(c, L.st0R, s0R);
      set_gemm(c, L.st1, s1);
      set_gemm(c, L.st2, s2);
      set_gemm(c, L.st3, s3);
      // interface pieces, grouped: vertices, then edges by (m, p, len)
      std::map<std::tuple<int, int, int, int>, std::vector<int>> groups;  // (kind, m, p, len)
      for (int i = 0; i < int(T.ifaces.size()); ++i) {
        const IfacePiece& pc = T.ifaces[i];
        if (pc.kind == PIECE_VERTEX) groups[std::make_tuple(0, 0, 0, 1)].push_back(i);
        else {
          const PatchDev& P = L.pd_h[pc.k];
          int j = pc.dirs[0];
          groups[std::make_tuple(1, P.m[j], P.p[j], pc.len[0])].push_back(i);
        }
      }
      std::vector<int64_t> ptr{0}, idx;
      std::vector<double> vsc;
      std::vector<GemmDesc> eA, eB;
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
            if (kind == 0) {
              const PatchDev& P = L.pd_h[pc.k];
              double h = 1.0 / P.m[0], p = P.p[0];
              vs = 1.0 / std::pow(h / p, d - 2);
            }
            vsc.push_back(vs);
          }
        }
        if (kind == 1) {
          int m = std::get<1>(kv.first), p = std::get<2>(kv.first), len = std::get<3>(kv.first);
          Mat Mm, Km;
          mass_stiffness_1d(m, p, Mm, Km);
          std::vector<int> I;
          for (int i = 1; i < m + p - 1; ++i) I.push_back(i);
          Mat MI = submatrix(Mm, m + p, I), KI = submatrix(Km, m + p, I);
          std::vector<double> lam;
          Mat U;
          if (!generalized_eigen(len, KI, MI, lam, U)) throw Fail{IGAMG_ERR_NUMERIC, "edge eigen failed"};
          double h = 1.0 / m, a = std::pow(h / p, d - 1), b = std::pow(h / p, d - 3);
          std::vector<double> dv(len);
          for (int q = 0; q < len; ++q) dv[q] = 1.0 / (a * lam[q] + b);
          double* dU = c->mem.upload(U, s);
          double* ddv = c->mem.upload(dv, s);
          int np = int(kv.second.size());
          // Y = (R U) colscale dinv ; Z = Y U^T   (R: np x len, row per piece)
          eA.push_back(GemmDesc{(double*)(intptr_t)gbase, dU, (double*)(intptr_t)gbase, ddv, len, len, len, 0, np,
                                len, len});
          eB.push_back(GemmDesc{(double*)(intptr_t)gbase, dU, (double*)(intptr_t)gbase, nullptr, len, len, len, 0,
                                np, len, len});
        }
      }
      L.n_if = int64_t(vsc.size());
      L.if_ptr = c->mem.upload(ptr, s);
      L.if_idx = c->mem.upload(idx, s);
      L.vscale = c->mem.upload(vsc, s);
      L.G = c->mem.alloc<double>(L.n_if);
      L.Z = c->mem.alloc<double>(L.n_if);
      L.Yif = c->mem.alloc<double>(L.n_if);
      CK(cudaMemsetAsync(L.Z, 0, std::max<int64_t>(L.n_if, 1) * sizeof(double), s));
      for (auto& g : eA) { g.A = L.G + (intptr_t)g.A; g.C = L.Yif + (intptr_t)g.C; }
      for (auto& g : eB) { g.A = L.Yif + (intptr_t)g.A; g.C = L.Z + (intptr_t)g.C; }
      set_gemm(c, L.edgeA, eA);
      set_gemm(c, L.edgeB, eB);
      // transfers from level l-1
      const Level& C = c->lv[l - 1];
      std::map<std::tuple<int, int>, std::vector<void*>> ptabs;
      std::vector<TransferDev> tds(K);
      int64_t ttot = 0;
      for (int k = 0; k < K; ++k) {
        TransferDev& td = tds[k];
        td.off_f = L.pd_h[k].off;
        td.off_c = C.pd_h[k].off;
        td.off_t = ttot;
        for (int j = 0; j < 3; ++j) {
          td.nf[j] = L.pd_h[k].n[j];
          td.nc[j] = C.pd_h[k].n[j];
          td.rw[j] = td.pw[j] = nullptr;
          td.rs[j] = td.ps[j] = nullptr;
          td.wr[j] = td.wp[j] = 0;
          if (j >= d) continue;
          int mc = C.pd_h[k].m[j], p = C.pd_h[k].p[j];
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
            ptabs[key] = {c->mem.upload(rw, s), c->mem.upload(rs, s), c->mem.upload(pw, s), c->mem.upload(ps, s),
                          (void*)(intptr_t)wr, (void*)(intptr_t)wp};
          }
          auto& v = ptabs[key];
          td.rw[j] = (const double*)v[0];
          td.rs[j] = (const int*)v[1];
          td.pw[j] = (const double*)v[2];
          td.ps[j] = (const int*)v[3];
          td.wr[j] = int((intptr_t)v[4]);
          td.wp[j] = int((intptr_t)v[5]);
        }
        ttot += int64_t(td.nc[0]) * td.nf[1];
        L.xfer_flops += 2.0 * (double(td.nc[0]) * td.nf[1] * td.wr[0] + double(td.nc[0]) * td.nc[1] * td.wr[1]);
        L.xfer_bytes += 8.0 * (double(td.nf[0]) * td.nf[1] + double(td.nc[0]) * td.nc[1]);
        L.max_nf = std::max(L.max_nf, std::max(td.nf[0], td.nf[1]));
        L.max_nc = std::max(L.max_nc, std::max(td.nc[0], td.nc[1]));
      }
      L.td = c->mem.upload(tds, s);
      L.ttmp = c->mem.alloc<double>(ttot);
    }
  }
  // coarse solver: dense A_0 from the level-0 bands, Cholesky, explicit inverse
  Level& L0 = c->lv[0];
  const LevelTopo& T0 = L0.topo;
  int64_t N0 = T0.N;
  if (N0 > 20000) throw Fail{IGAMG_ERR_UNSUPPORTED, "coarse problem too large for the dense solver"};
  int64_t bsz = 0;
  for (int k = 0; k < K; ++k) bsz = std::max(bsz, L0.pd_h[k].band_off + (T0.off[k + 1] - T0.off[k]) *
                                                   int64_t(2 * L0.pd_h[k].p[0] + 1) * (2 * L0.pd_h[k].p[1] + 1));
  std::vector<double> hb(bsz);
  CK(cudaMemcpyAsync(hb.data(), L0.band, bsz * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  Mat A0(size_t(N0) * N0, 0.0);
  for (int k = 0; k < K; ++k) {
    const PatchDev& P = L0.pd_h[k];
    int64_t nn = int64_t(P.n[0]) * P.n[1];
    int w1 = 2 * P.p[1] + 1;
    for (int i0 = 0; i0 < P.n[0]; ++i0)
      for (int i1 = 0; i1 < P.n[1]; ++i1) {
        int64_t gi = T0.l2g[P.off + int64_t(i0) * P.n[1] + i1];
        if (gi < 0) continue;
        for (int t0 = 0; t0 <= 2 * P.p[0]; ++t0)
          for (int t1 = 0; t1 < w1; ++t1) {
            int j0 = i0 + t0 - P.p[0], j1 = i1 + t1 - P.p[1];
            if (j0 < 0 || j0 >= P.n[0] || j1 < 0 || j1 >= P.n[1]) continue;
            int64_t gj = T0.l2g[P.off + int64_t(j0) * P.n[1] + j1];
            if (gj < 0) continue;
            A0[size_t(gi) * N0 + gj] += hb[P.band_off + int64_t(t0 * w1 + t1) * nn + int64_t(i0) * P.n[1] + i1];
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
  int64_t gmaxN = 0;
  for (auto& L : c->lv) gmaxN = std::max(gmaxN, L.topo.N);
  c->gtmp = c->mem.alloc<double>(gmaxN);
  c->partials = c->mem.alloc<double>(RED_BLOCKS);
  c->scal = c->mem.alloc<double>(16);
  CK(cudaMemsetAsync(c->scal, 0, 16 * sizeof(double), s));
  CK(cudaMallocHost(&c->h_scal, 16 * sizeof(double)));
  CK(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------- cycle

void residual(igamg_ctx* c, int l, const double* f, const double* u, double* r) {
  Level& L = c->lv[l];
  ProfScope ps(c, CLS_APPLY, L.apply_flops, L.band_bytes + 8.0 * L.topo.T * (f ? 3 : 2));
  CK(launch_band_apply_2d(c->stream, L.pd, c->pd.K, L.max_n[0], L.max_n[1], L.max_p, L.band, u, f, r));
}

// u (=|+=) tau L^{-1} v for a distributed v (F or R of the level): patch interiors by
// fast diagonalisation, edges by their 1D fast diagonalisation, vertices by scaling
// (Eq. additive; the pieces are disjoint, so the sum is a set of independent blocks).
void smooth(igamg_ctx* c, int l, bool from_F, bool add) {
  Level& L = c->lv[l];
  const double* v = from_F ? L.F : L.R;
  double tau = c->opt.tau;
  int epi = add ? EPI_ADD : EPI_ASSIGN;
  run_gemm(c, from_F ? L.st0F : L.st0R, true, false, EPI_STORE, 1.0, CLS_FD);
  run_gemm(c, L.st1, false, false, EPI_MUL, 1.0, CLS_FD);
  run_gemm(c, L.st2, false, false, EPI_STORE, 1.0, CLS_FD);
  run_gemm(c, L.st3, false, true, epi, tau, CLS_FD);
  if (L.n_if == 0) return;
  {
    ProfScope ps(c, CLS_IFACE, 0.0, 16.0 * L.n_if);
    CK(launch_iface_gather(c->stream, L.n_if, L.if_ptr, L.if_idx, v, L.G));
  }
  run_gemm(c, L.edgeA, false, false, EPI_COLSCALE, 1.0, CLS_IFACE);
  run_gemm(c, L.edgeB, false, true, EPI_STORE, 1.0, CLS_IFACE);
  {
    ProfScope ps(c, CLS_IFACE, 2.0 * L.n_if, 24.0 * L.n_if);
    CK(launch_iface_scatter(c->stream, L.n_if, L.if_ptr, L.if_idx, L.Z, L.G, L.vscale, tau, add ? 1 : 0, L.U));
  }
}

void coarse_solve(igamg_ctx* c) {
  Level& L0 = c->lv[0];
  ProfScope ps(c, CLS_COARSE, 2.0 * double(c->N0) * c->N0, 8.0 * double(c->N0) * c->N0);
  CK(launch_coarse_solve(c->stream, c->N0, L0.g2t_ptr, L0.g2t, c->A0inv, L0.F, L0.U));
}

// Algorithm 1 on level l >= 1: f = F_l (distributed), u = U_l (accumulated).
void multigrid(igamg_ctx* c, int l, bool zero_init) {
  Level& L = c->lv[l];
  const int nu = c->opt.nu, mu = c->opt.mu;
  for (int i = 0; i < nu; ++i) {
    if (zero_init && i == 0) {
      smooth(c, l, true, false);  // u = 0: the residual is f itself
    } else {
      residual(c, l, L.F, L.U, L.R);
      smooth(c, l, false, true);
    }
  }
  residual(c, l, L.F, L.U, L.R);
  Level& C = c->lv[l - 1];
  {
    ProfScope pr(c, CLS_TRANSFER, L.xfer_flops, L.xfer_bytes, 2);
    CK(launch_restrict_2d(c->stream, L.td, c->pd.K, L.max_nf, L.max_nc, L.R, L.ttmp, C.F, C.l2g, C.topo.T));
  }
  if (l == 1) {
    coarse_solve(c);
  } else {
    for (int j = 0; j < mu; ++j) multigrid(c, l - 1, j == 0);
  }
  {
    ProfScope pp(c, CLS_TRANSFER, 2.0 * L.xfer_flops, 2.0 * L.xfer_bytes, 2);
    CK(launch_prolong_2d(c->stream, L.td, c->pd.K, L.max_nf, L.max_nc, C.U, L.ttmp, L.U));
  }
  for (int i = 0; i < nu; ++i) {
    residual(c, l, L.F, L.U, L.R);
    smooth(c, l, false, true);
  }
}

// z = U_L = Multigrid(L, 0, F_L)
void precondition(igamg_ctx* c) {
  int Lf = int(c->lv.size()) - 1;
  if (Lf == 0) coarse_solve(c);
  else multigrid(c, Lf, true);
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
  CK(launch_global_to_tile(c->stream, L.topo.N, L.g2t_ptr, L.g2t, xg, xt, 1));
}
void to_acc(igamg_ctx* c, int l, const double* xg, double* xt) {
  Level& L = c->lv[l];
  ProfScope ps(c, CLS_VECTOR, 0.0, 16.0 * L.topo.N);
  CK(cudaMemsetAsync(xt, 0, L.topo.T * sizeof(double), c->stream));
  CK(launch_global_to_tile(c->stream, L.topo.N, L.g2t_ptr, L.g2t, xg, xt, 0));
}
void from_acc(igamg_ctx* c, int l, const double* xt, double* xg) {
  Level& L = c->lv[l];
  ProfScope ps(c, CLS_VECTOR, 0.0, 16.0 * L.topo.N);
  CK(launch_tile_to_global(c->stream, L.topo.N, L.g2t_ptr, L.g2t, xt, xg, 0));
}
void from_dist(igamg_ctx* c, int l, const double* xt, double* xg) {
  Level& L = c->lv[l];
  ProfScope ps(c, CLS_VECTOR, 0.0, 16.0 * L.topo.N);
  CK(launch_tile_to_global(c->stream, L.topo.N, L.g2t_ptr, L.g2t, xt, xg, 1));
}

double read_scalar(igamg_ctx* c, int i) {
  CK(cudaMemcpyAsync(c->h_scal + i, c->scal + i, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (c->prof) prof_collect(c);
  return c->h_scal[i];
}

void vdot(igamg_ctx* c, const double* a, const double* b, int64_t T, double* out) {
  ProfScope ps(c, CLS_VECTOR, 2.0 * T, 16.0 * T, 2);
  CK(launch_dot(c->stream, a, b, T, c->partials, out));
}

void vnorm_dist(igamg_ctx* c, int l, const double* v, double* out) {
  Level& L = c->lv[l];
  ProfScope ps(c, CLS_VECTOR, 2.0 * L.topo.N, 8.0 * L.topo.T, 2);
  CK(launch_norm2_dist(c->stream, L.topo.N, L.g2t_ptr, L.g2t, v, c->partials, out));
}

// PCG (Sec. 4): r, w distributed; x, z, p accumulated.  scal: 0 rz, 1 pw, 2 rz_new, 3 rr.
igamg_status pcg(igamg_ctx* c, const double* b, double* x, double tol, igamg_result* res) {
  double t0 = now_ms();
  const int Lf = int(c->lv.size()) - 1;
  Level& L = c->lv[Lf];
  const int64_t T = L.topo.T;
  cudaStream_t s = c->stream;
  to_dist(c, Lf, b, c->Bt);
  to_acc(c, Lf, x, c->X);
  residual(c, Lf, c->Bt, c->X, L.F);
  vnorm_dist(c, Lf, L.F, c->scal + 3);
  double rr0 = read_scalar(c, 3);
  if (!std::isfinite(rr0)) throw Fail{IGAMG_ERR_NUMERIC, "non-finite initial residual"};
  int it = 0;
  double rel = 0.0;
  igamg_status st = IGAMG_OK;
  if (rr0 > 0.0) {
    precondition(c);
    CK(cudaMemcpyAsync(c->Pv, L.U, T * sizeof(double), cudaMemcpyDeviceToDevice, s));
    vdot(c, L.F, L.U, T, c->scal + 0);
    rel = 1.0;
    while (true) {
      if (tol > 0 && rel <= tol) break;
      if (it >= c->opt.max_iter) { st = tol > 0 ? IGAMG_ERR_NOT_CONVERGED : IGAMG_OK; break; }
      residual(c, Lf, nullptr, c->Pv, c->W);
      vdot(c, c->Pv, c->W, T, c->scal + 1);
      {
        ProfScope ps(c, CLS_VECTOR, 4.0 * T, 48.0 * T);
        CK(launch_pcg_xr(s, T, c->scal, c->X, L.F, c->Pv, c->W));
      }
      ++it;
      vnorm_dist(c, Lf, L.F, c->scal + 3);
      double rr = read_scalar(c, 3);
      if (!std::isfinite(rr)) throw Fail{IGAMG_ERR_NUMERIC, "non-finite residual in PCG"};
      rel = std::sqrt(rr / rr0);
      if (tol > 0 && rel <= tol) break;
      if (it >= c->opt.max_iter) continue;
      precondition(c);
      vdot(c, L.F, L.U, T, c->scal + 2);
      {
        ProfScope ps(c, CLS_VECTOR, 2.0 * T, 24.0 * T, 2);
        CK(launch_pcg_p(s, T, c->scal, c->Pv, L.U));
      }
    }
  }
  from_acc(c, Lf, c->X, x);
  CK(cudaStreamSynchronize(s));
  if (c->prof) prof_collect(c);
  if (res) {
    res->iters = it;
    res->relres = rel;
    res->t_setup_ms = c->t_setup_ms;
    res->t_assemble_ms = c->t_assemble_ms;
    res->t_solve_ms = now_ms() - t0;
  }
  return st;
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

extern "C" {

igamg_status igamg_default_options(igamg_options* opt) {
  if (!opt) return IGAMG_ERR_ARG;
  opt->tau = 0.25;
  opt->sigma_scale = 5.0;
  opt->nu = 1;
  opt->mu = 1;
  opt->max_iter = 500;
  opt->precision = IGAMG_FP64;
  return IGAMG_OK;
}

igamg_status igamg_setup(const igamg_problem* prob, const igamg_options* opt, void* cuda_stream,
                         igamg_ctx** out) {
  if (!out) return IGAMG_ERR_ARG;
  *out = nullptr;
  if (!prob) { g_setup_error = "problem is NULL"; return IGAMG_ERR_ARG; }
  igamg_ctx* c = new igamg_ctx();
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  igamg_default_options(&c->opt);
  if (opt) c->opt = *opt;
  double t0 = now_ms();
  try {
    if (c->opt.precision != IGAMG_FP64) throw Fail{IGAMG_ERR_UNSUPPORTED, "only FP64 is accepted"};
    if (c->opt.nu < 1 || c->opt.mu < 1 || c->opt.mu > 2 || c->opt.max_iter < 0 || !(c->opt.tau > 0))
      throw Fail{IGAMG_ERR_ARG, "bad options"};
    int code = 0;
    std::string e = parse_problem(prob->dim, prob->num_patches, prob->degree, prob->num_knots, prob->knots,
                                  prob->geo_degree, prob->geo_num_ctrl, prob->geo_ctrl, prob->side_bc,
                                  prob->num_levels, c->pd, &code);
    if (!e.empty()) throw Fail{igamg_status(code), e};
    build_levels(c);
  } catch (const Fail& e) {
    g_setup_error = e.msg;
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

igamg_status igamg_apply(igamg_ctx* c, int level, const double* x, double* y) {
  return guarded(c, [&]() {
    if (!x || !y) throw Fail{IGAMG_ERR_ARG, "NULL vector"};
    int l = level_index(c, level);
    Level& L = c->lv[l];
    to_acc(c, l, x, L.U);
    residual(c, l, nullptr, L.U, L.R);
    from_dist(c, l, L.R, y);
    return IGAMG_OK;
  });
}

igamg_status igamg_smooth(igamg_ctx* c, int level, const double* r, double* z) {
  return guarded(c, [&]() {
    if (!r || !z) throw Fail{IGAMG_ERR_ARG, "NULL vector"};
    int l = level_index(c, level);
    if (l < 1) throw Fail{IGAMG_ERR_ARG, "the smoother exists on levels >= 1"};
    Level& L = c->lv[l];
    to_dist(c, l, r, L.R);
    CK(cudaMemsetAsync(L.U, 0, L.topo.T * sizeof(double), c->stream));
    smooth(c, l, false, false);
    CK(launch_axpby(c->stream, L.topo.T, 0.0, L.U, 1.0 / c->opt.tau, L.U));
    from_acc(c, l, L.U, z);
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
    to_dist(c, l, r, L.R);
    CK(launch_restrict_2d(c->stream, L.td, c->pd.K, L.max_nf, L.max_nc, L.R, L.ttmp, C.F, C.l2g, C.topo.T));
    from_dist(c, l - 1, C.F, rc);
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
    to_acc(c, l - 1, uc, C.U);
    CK(cudaMemsetAsync(L.U, 0, L.topo.T * sizeof(double), c->stream));
    CK(launch_prolong_2d(c->stream, L.td, c->pd.K, L.max_nf, L.max_nc, C.U, L.ttmp, L.U));
    from_acc(c, l, L.U, u);
    return IGAMG_OK;
  });
}

igamg_status igamg_coarse_solve(igamg_ctx* c, const double* r, double* x) {
  return guarded(c, [&]() {
    if (!r || !x) throw Fail{IGAMG_ERR_ARG, "NULL vector"};
    to_dist(c, 0, r, c->lv[0].F);
    coarse_solve(c);
    from_acc(c, 0, c->lv[0].U, x);
    return IGAMG_OK;
  });
}

igamg_status igamg_precondition(igamg_ctx* c, const double* r, double* z) {
  return guarded(c, [&]() {
    if (!r || !z) throw Fail{IGAMG_ERR_ARG, "NULL vector"};
    int Lf = int(c->lv.size()) - 1;
    to_dist(c, Lf, r, c->lv[Lf].F);
    precondition(c);
    from_acc(c, Lf, c->lv[Lf].U, z);
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
    size_t bytes = size_t(L.band_bytes);
    CK(cudaMallocAsync(&mband, bytes, s));
    int64_t gmax = 0;
    for (auto& P : L.pd_h) gmax = std::max(gmax, int64_t(P.m[0]) * (P.p[0] + 1) * P.m[1] * (P.p[1] + 1) * 4);
    double *G = nullptr, *dcorn = nullptr;
    CK(cudaMallocAsync(&G, gmax * sizeof(double), s));
    CK(cudaMallocAsync(&dcorn, c->pd.corners.size() * sizeof(double), s));
    CK(cudaMemcpyAsync(dcorn, c->pd.corners.data(), c->pd.corners.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    std::map<std::tuple<int, int>, std::vector<double*>> dt;
    std::vector<double*> tmp_tabs;
    for (int k = 0; k < c->pd.K; ++k) {
      const PatchDev& P = L.pd_h[k];
      double* tp[2][4];
      for (int j = 0; j < 2; ++j) {
        auto key = std::make_tuple(P.m[j], P.p[j]);
        if (!dt.count(key)) {
          Tables1D tb = tables_1d(P.m[j], P.p[j]);
          std::vector<double*> v;
          for (auto* src : {&tb.xq, &tb.wq, &tb.B, &tb.dB}) {
            double* d = nullptr;
            CK(cudaMallocAsync(&d, src->size() * sizeof(double), s));
            CK(cudaMemcpyAsync(d, src->data(), src->size() * sizeof(double), cudaMemcpyHostToDevice, s));
            v.push_back(d);
            tmp_tabs.push_back(d);
          }
          CK(cudaStreamSynchronize(s));  // host tables go out of scope
          dt[key] = v;
        }
        for (int q = 0; q < 4; ++q) tp[j][q] = dt[key][q];
      }
      CK(launch_geom_factors_2d(s, dcorn + size_t(k) * 8, P.m[0], P.m[1], P.p[0] + 1, tp[0][0], tp[0][1],
                                tp[1][0], tp[1][1], G));
      CK(launch_assemble_2d(s, P, G, tp[0][2], tp[0][3], tp[1][2], tp[1][3], L.l2g, 1, mband));
    }
    to_acc(c, Lf, coef, L.U);
    CK(launch_band_apply_2d(s, L.pd, c->pd.K, L.max_n[0], L.max_n[1], L.max_p, mband, L.U, nullptr, L.R));
    from_dist(c, Lf, L.R, rhs);
    for (double* d : tmp_tabs) CK(cudaFreeAsync(d, s));
    CK(cudaFreeAsync(G, s));
    CK(cudaFreeAsync(dcorn, s));
    CK(cudaFreeAsync(mband, s));
    CK(cudaStreamSynchronize(s));
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
    return pcg(c, b, x, tol, res);
  });
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
    igamg_status st = pcg(c, db, dx, tol, res);
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
  for (auto& t : c->ev_open) {
    cudaEventDestroy(std::get<1>(t));
    cudaEventDestroy(std::get<2>(t));
  }
  for (cudaEvent_t e : c->ev_free) cudaEventDestroy(e);
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
