// FP64 device kernels of the multi-patch multigrid solver (2D tiles).
//
// Layout: a level vector is the concatenation of per-patch tiles (C order, last direction
// fastest); a global dof shared by several patches has one copy per owner (Sec. 4: the
// processor-local parts of accumulated/distributed vectors, here all on one device).
// Band storage of A_{l,k}: band[band_off + t * nn + node] with t the flattened offset
// (j - i + p) over (2p+1)^d, tap-major so that a warp reads 32 consecutive rows of one tap.
#include "kernels.cuh"

namespace igamg {

namespace {
constexpr int AX = 32, AY = 8;  // band-apply block: 32 x 8 outputs

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order block reduction of one value per thread (blockDim.x == 256).
__device__ double block_sum_256(double v, double* sh) {
  int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (t < s) sh[t] += sh[t + s];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}
}  // namespace

// ---------------------------------------------------------------- setup: assembly

__global__ void k_geom_factors_2d(const double* __restrict__ cr, int m0, int m1, int nq0, int nq1,
                                  const double* __restrict__ xq0, const double* __restrict__ wq0,
                                  const double* __restrict__ xq1, const double* __restrict__ wq1,
                                  double* __restrict__ G) {
  int Q1 = m1 * nq1;
  int64_t total = int64_t(m0) * nq0 * Q1;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < total;
       q += int64_t(gridDim.x) * blockDim.x) {
    int a = int(q / Q1), b = int(q % Q1);
    double s = xq0[a], t = xq1[b], w = wq0[a] * wq1[b];
    // bilinear map: corners c = c0 + 2 c1, phi_0 = 1 - x, phi_1 = x
    double J00 = 0, J01 = 0, J10 = 0, J11 = 0;
    for (int c = 0; c < 4; ++c) {
      int c0 = c & 1, c1 = c >> 1;
      double ds = c0 ? 1.0 : -1.0, dt = c1 ? 1.0 : -1.0;
      double ps = c0 ? s : 1.0 - s, pt = c1 ? t : 1.0 - t;
      J00 += cr[2 * c] * ds * pt;
      J10 += cr[2 * c + 1] * ds * pt;
      J01 += cr[2 * c] * ps * dt;
      J11 += cr[2 * c + 1] * ps * dt;
    }
    double det = J00 * J11 - J01 * J10;
    double ad = fabs(det);
    double* g = G + 4 * q;
    g[0] = w * (J11 * J11 + J01 * J01) / ad;
    g[1] = -w * (J11 * J10 + J01 * J00) / ad;
    g[2] = w * (J10 * J10 + J00 * J00) / ad;
    g[3] = w * ad;
  }
}

cudaError_t launch_geom_factors_2d(cudaStream_t s, const double* corners, int m0, int m1, int nq,
                                   const double* xq0, const double* wq0, const double* xq1,
                                   const double* wq1, double* G) {
  k_geom_factors_2d<<<1216, 256, 0, s>>>(corners, m0, m1, nq, nq, xq0, wq0, xq1, wq1, G);
  return cudaGetLastError();
}

// One thread per row (i0, i1) of one patch; loops over the (2p+1)^2 taps and the Gauss
// points of the elements shared by the two supports.
__global__ void k_assemble_2d(PatchDev pd, const double* __restrict__ G,
                              const double* __restrict__ B0, const double* __restrict__ dB0,
                              const double* __restrict__ B1, const double* __restrict__ dB1,
                              const int64_t* __restrict__ l2g, int mass, double* __restrict__ band) {
  int i1 = blockIdx.x * blockDim.x + threadIdx.x;
  int i0 = blockIdx.y;
  const int n0 = pd.n[0], n1 = pd.n[1], p0 = pd.p[0], p1 = pd.p[1];
  const int m0 = pd.m[0], m1 = pd.m[1], nq0 = p0 + 1, nq1 = p1 + 1, w1 = 2 * p1 + 1;
  if (i1 >= n1) return;
  const int64_t nn = int64_t(n0) * n1, node = int64_t(i0) * n1 + i1;
  const bool active = l2g[pd.off + node] >= 0;
  const int64_t Q1 = int64_t(m1) * nq1;
  for (int t0 = 0; t0 <= 2 * p0; ++t0)
    for (int t1 = 0; t1 < w1; ++t1) {
      int j0 = i0 + t0 - p0, j1 = i1 + t1 - p1;
      double acc = 0.0;
      if (active && j0 >= 0 && j0 < n0 && j1 >= 0 && j1 < n1) {
        int e0lo = max(max(i0, j0) - p0, 0), e0hi = min(min(i0, j0), m0 - 1);
        int e1lo = max(max(i1, j1) - p1, 0), e1hi = min(min(i1, j1), m1 - 1);
        for (int e0 = e0lo; e0 <= e0hi; ++e0) {
          int a0 = i0 - e0, b0 = j0 - e0;
          for (int q0 = 0; q0 < nq0; ++q0) {
            int64_t Q0 = int64_t(e0) * nq0 + q0;
            double vi0 = B0[Q0 * (p0 + 1) + a0], di0 = dB0[Q0 * (p0 + 1) + a0];
            double vj0 = B0[Q0 * (p0 + 1) + b0], dj0 = dB0[Q0 * (p0 + 1) + b0];
            double f00 = di0 * dj0, f01 = di0 * vj0, f10 = vi0 * dj0, f11 = vi0 * vj0;
            for (int e1 = e1lo; e1 <= e1hi; ++e1) {
              int a1 = i1 - e1, b1 = j1 - e1;
              for (int q1 = 0; q1 < nq1; ++q1) {
                int64_t Qb = int64_t(e1) * nq1 + q1;
                double vi1 = B1[Qb * (p1 + 1) + a1], di1 = dB1[Qb * (p1 + 1) + a1];
                double vj1 = B1[Qb * (p1 + 1) + b1], dj1 = dB1[Qb * (p1 + 1) + b1];
                const double* g = G + 4 * (Q0 * Q1 + Qb);
                if (mass)
                  acc += g[3] * f11 * vi1 * vj1;
                else
                  acc += g[0] * f00 * vi1 * vj1 + g[1] * (f01 * vi1 * dj1 + f10 * di1 * vj1) +
                         g[2] * f11 * di1 * dj1;
              }
            }
          }
        }
      }
      band[pd.band_off + int64_t(t0 * w1 + t1) * nn + node] = acc;
    }
}

cudaError_t launch_assemble_2d(cudaStream_t s, const PatchDev& pd, const double* G,
                               const double* B0, const double* dB0, const double* B1,
                               const double* dB1, const int64_t* l2g_tile, int mass,
                               double* band) {
  dim3 grid((pd.n[1] + 63) / 64, pd.n[0]);
  k_assemble_2d<<<grid, 64, 0, s>>>(pd, G, B0, dB0, B1, dB1, l2g_tile, mass, band);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- stiffness apply

// y = f - A u (f != NULL) or y = A u, per patch tile; u staged in shared memory with a
// halo of p in every direction (zero outside the tile).
__global__ void __launch_bounds__(AX * AY) k_band_apply_2d(const PatchDev* __restrict__ pds,
                                                           const double* __restrict__ band,
                                                           const double* __restrict__ u,
                                                           const double* __restrict__ f,
                                                           double* __restrict__ y) {
  extern __shared__ double su[];
  const PatchDev pd = pds[blockIdx.z];
  const int n0 = pd.n[0], n1 = pd.n[1], p0 = pd.p[0], p1 = pd.p[1];
  const int i0b = blockIdx.y * AY, i1b = blockIdx.x * AX;
  if (i0b >= n0 || i1b >= n1) return;
  const int H0 = AY + 2 * p0, H1 = AX + 2 * p1;
  const double* ut = u + pd.off;
  for (int idx = threadIdx.y * AX + threadIdx.x; idx < H0 * H1; idx += AX * AY) {
    int r = idx / H1, c = idx % H1;
    int g0 = i0b - p0 + r, g1 = i1b - p1 + c;
    su[idx] = (g0 >= 0 && g0 < n0 && g1 >= 0 && g1 < n1) ? ut[int64_t(g0) * n1 + g1] : 0.0;
  }
  __syncthreads();
  const int i0 = i0b + threadIdx.y, i1 = i1b + threadIdx.x;
  if (i0 >= n0 || i1 >= n1) return;
  const int64_t nn = int64_t(n0) * n1, node = int64_t(i0) * n1 + i1;
  const double* bp = band + pd.band_off + node;
  const int w1 = 2 * p1 + 1;
  double acc = 0.0;
  for (int t0 = 0; t0 <= 2 * p0; ++t0) {
    const double* srow = su + (threadIdx.y + t0) * H1 + threadIdx.x;
    const double* brow = bp + int64_t(t0 * w1) * nn;
    for (int t1 = 0; t1 < w1; ++t1) acc = fma(__ldg(brow + int64_t(t1) * nn), srow[t1], acc);
  }
  y[pd.off + node] = f ? f[pd.off + node] - acc : acc;
}

cudaError_t launch_band_apply_2d(cudaStream_t s, const PatchDev* pd_dev, int K, int max_n0,
                                 int max_n1, int max_p, const double* band, const double* u,
                                 const double* f, double* y) {
  dim3 grid((max_n1 + AX - 1) / AX, (max_n0 + AY - 1) / AY, K);
  size_t sm = sizeof(double) * (AY + 2 * max_p) * (AX + 2 * max_p);
  k_band_apply_2d<<<grid, dim3(AX, AY), sm, s>>>(pd_dev, band, u, f, y);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- batched FP64 GEMM

// C = op(A) op(B) with an epilogue, one output tile of 8R x 8R per block of 64 threads;
// thread (tx, ty) owns rows ty + 8r and columns tx + 8c (r, c < R).  Rows/columns of the
// tile beyond M/N and the k-slab beyond K are skipped warp-uniformly, so ragged sizes
// (e.g. 258 = 8*32 + 2) waste FP64 work only at 8-granularity.
namespace {
constexpr int GK = 16;

template <int R>
__device__ __forceinline__ void gemm_tile(const GemmDesc& d, int ta, int tb, int epi, double alpha,
                                          int bx, int by) {
  constexpr int BT = 8 * R;
  const int i0 = by * BT, j0 = bx * BT;
  if (i0 >= d.M || j0 >= d.N) return;
  __shared__ double As[GK][BT + 1];
  __shared__ double Bs[GK][BT + 1];
  const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
  const int wty = (tid >> 5) * 4;  // smallest ty of this warp
  int rv = 0, cv = 0;              // warp-uniform counts of live micro-rows / micro-columns
#pragma unroll
  for (int r = 0; r < R; ++r) rv += (i0 + wty + 8 * r < d.M) ? 1 : 0;
#pragma unroll
  for (int c = 0; c < R; ++c) cv += (j0 + 8 * c < d.N) ? 1 : 0;
  double acc[R][R];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) acc[r][c] = 0.0;
  for (int k0 = 0; k0 < d.K; k0 += GK) {
    for (int idx = tid; idx < BT * GK; idx += 64) {
      int i, kk;
      if (ta) { i = idx % BT; kk = idx / BT; } else { kk = idx % GK; i = idx / GK; }
      int gi = i0 + i, gk = k0 + kk;
      double v = 0.0;
      if (gi < d.M && gk < d.K) v = ta ? d.A[int64_t(gk) * d.lda + gi] : d.A[int64_t(gi) * d.lda + gk];
      As[kk][i] = v;
      int j;
      if (tb) { kk = idx % GK; j = idx / GK; } else { j = idx % BT; kk = idx / BT; }
      int gj = j0 + j;
      gk = k0 + kk;
      v = 0.0;
      if (gj < d.N && gk < d.K) v = tb ? d.B[int64_t(gj) * d.ldb + gk] : d.B[int64_t(gk) * d.ldb + gj];
      Bs[kk][j] = v;
    }
    __syncthreads();
    const int kmax = min(GK, d.K - k0);
    for (int kk = 0; kk < kmax; ++kk) {
      double a[R], b[R];
#pragma unroll
      for (int r = 0; r < R; ++r) a[r] = As[kk][ty + 8 * r];
#pragma unroll
      for (int c = 0; c < R; ++c) b[c] = Bs[kk][tx + 8 * c];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (r < rv) {
#pragma unroll
          for (int c = 0; c < R; ++c)
            if (c < cv) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    int gi = i0 + ty + 8 * r;
    if (gi >= d.M) continue;
#pragma unroll
    for (int c = 0; c < R; ++c) {
      int gj = j0 + tx + 8 * c;
      if (gj >= d.N) continue;
      double v = acc[r][c];
      double* cp = d.C + int64_t(gi) * d.ldc + gj;
      switch (epi) {
        case EPI_MUL: *cp = v * d.E[int64_t(gi) * d.lde + gj]; break;
        case EPI_ROWSCALE: *cp = v * d.E[gi]; break;
        case EPI_COLSCALE: *cp = v * d.E[gj]; break;
        case EPI_ASSIGN: *cp = alpha * v; break;
        case EPI_ADD: *cp = fma(alpha, v, *cp); break;
        default: *cp = v;
      }
    }
  }
}
}  // namespace

template <int R>
__global__ void __launch_bounds__(64) k_gemm_f64(const GemmDesc* __restrict__ descs, int ta, int tb, int epi,
                                                 double alpha) {
  gemm_tile<R>(descs[blockIdx.z], ta, tb, epi, alpha, blockIdx.x, blockIdx.y);
}

template <int R>
__global__ void __launch_bounds__(64) k_gemm_f64_one(GemmDesc d, int ta, int tb, int epi, double alpha) {
  gemm_tile<R>(d, ta, tb, epi, alpha, blockIdx.x, blockIdx.y);
}

// Tile edge 8R: 32 when the 32-wide grid already fills the GPU twice, else 16, else 8.
static int pick_r(int maxM, int maxN, int batch) {
  auto tiles = [&](int bt) { return int64_t((maxM + bt - 1) / bt) * ((maxN + bt - 1) / bt) * batch; };
  if (tiles(32) >= 2 * 152) return 4;
  if (tiles(16) >= 152) return 2;
  return 1;
}

cudaError_t launch_gemm(cudaStream_t s, const GemmDesc* d_desc, int batch, int maxM, int maxN,
                        bool transA, bool transB, int epi, double alpha) {
  if (batch <= 0) return cudaSuccess;
  int R = pick_r(maxM, maxN, batch), bt = 8 * R;
  dim3 grid((maxN + bt - 1) / bt, (maxM + bt - 1) / bt, batch);
  if (R == 4) k_gemm_f64<4><<<grid, 64, 0, s>>>(d_desc, transA, transB, epi, alpha);
  else if (R == 2) k_gemm_f64<2><<<grid, 64, 0, s>>>(d_desc, transA, transB, epi, alpha);
  else k_gemm_f64<1><<<grid, 64, 0, s>>>(d_desc, transA, transB, epi, alpha);
  return cudaGetLastError();
}

cudaError_t launch_gemm_one(cudaStream_t s, const GemmDesc& d, bool transA, bool transB, int epi,
                            double alpha) {
  int R = pick_r(d.M, d.N, 1), bt = 8 * R;
  dim3 grid((d.N + bt - 1) / bt, (d.M + bt - 1) / bt, 1);
  if (R == 4) k_gemm_f64_one<4><<<grid, 64, 0, s>>>(d, transA, transB, epi, alpha);
  else if (R == 2) k_gemm_f64_one<2><<<grid, 64, 0, s>>>(d, transA, transB, epi, alpha);
  else k_gemm_f64_one<1><<<grid, 64, 0, s>>>(d, transA, transB, epi, alpha);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- interface pieces

__global__ void k_iface_gather(int64_t n, const int64_t* __restrict__ ptr, const int64_t* __restrict__ idx,
                               const double* __restrict__ v, double* __restrict__ G) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    double s = 0.0;
    for (int64_t c = ptr[i]; c < ptr[i + 1]; ++c) s += v[idx[c]];
    G[i] = s;
  }
}

__global__ void k_iface_scatter(int64_t n, const int64_t* __restrict__ ptr, const int64_t* __restrict__ idx,
                                const double* __restrict__ Z, const double* __restrict__ G,
                                const double* __restrict__ vs, double tau, int add, double* __restrict__ u) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    double val = tau * fma(vs[i], G[i], Z[i]);
    for (int64_t c = ptr[i]; c < ptr[i + 1]; ++c) {
      int64_t t = idx[c];
      u[t] = add ? u[t] + val : val;
    }
  }
}

static int grid_for(int64_t n, int threads, int cap = 4 * 152 * 8) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  return int(g < cap ? g : cap);
}

cudaError_t launch_iface_gather(cudaStream_t s, int64_t n_nodes, const int64_t* ptr,
                                const int64_t* idx, const double* v, double* G) {
  if (n_nodes <= 0) return cudaSuccess;
  k_iface_gather<<<grid_for(n_nodes, 256), 256, 0, s>>>(n_nodes, ptr, idx, v, G);
  return cudaGetLastError();
}

cudaError_t launch_iface_scatter(cudaStream_t s, int64_t n_nodes, const int64_t* ptr,
                                 const int64_t* idx, const double* Z, const double* G,
                                 const double* vscale, double tau, int add, double* u) {
  if (n_nodes <= 0) return cudaSuccess;
  k_iface_scatter<<<grid_for(n_nodes, 256), 256, 0, s>>>(n_nodes, ptr, idx, Z, G, vscale, tau, add, u);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- transfers (Sec. 3)

// Restriction P^T (distributed -> distributed), direction 0 then direction 1:
// tmp[i0c][j1] = sum_w rw0[i0c][w] rf[rs0[i0c]+w][j1];  rc[i0c][i1c] = sum_w rw1[i1c][w] tmp[i0c][rs1[i1c]+w]
__global__ void k_restrict_a(const TransferDev* __restrict__ tds, const double* __restrict__ rf,
                             double* __restrict__ tmp) {
  const TransferDev td = tds[blockIdx.z];
  int j1 = blockIdx.x * blockDim.x + threadIdx.x, i0c = blockIdx.y;
  if (i0c >= td.nc[0] || j1 >= td.nf[1]) return;
  const int W = td.wr[0];
  const double* w = td.rw[0] + int64_t(i0c) * W;
  int r0 = td.rs[0][i0c];
  double acc = 0.0;
  for (int a = 0; a < W; ++a) {
    int j0 = r0 + a;
    if (j0 < td.nf[0]) acc = fma(w[a], rf[td.off_f + int64_t(j0) * td.nf[1] + j1], acc);
  }
  tmp[td.off_t + int64_t(i0c) * td.nf[1] + j1] = acc;
}

__global__ void k_restrict_b(const TransferDev* __restrict__ tds, const double* __restrict__ tmp,
                             double* __restrict__ rc, const int64_t* __restrict__ l2g_c) {
  const TransferDev td = tds[blockIdx.z];
  int i1c = blockIdx.x * blockDim.x + threadIdx.x, i0c = blockIdx.y;
  if (i0c >= td.nc[0] || i1c >= td.nc[1]) return;
  const int W = td.wr[1];
  const double* w = td.rw[1] + int64_t(i1c) * W;
  int r1 = td.rs[1][i1c];
  const double* row = tmp + td.off_t + int64_t(i0c) * td.nf[1];
  double acc = 0.0;
  for (int a = 0; a < W; ++a) {
    int j1 = r1 + a;
    if (j1 < td.nf[1]) acc = fma(w[a], row[j1], acc);
  }
  int64_t t = td.off_c + int64_t(i0c) * td.nc[1] + i1c;
  rc[t] = l2g_c[t] >= 0 ? acc : 0.0;
}

// Prolongation P (accumulated -> accumulated, added into uf), direction 1 then 0:
// tmp[i0c][j1] = sum_w pw1[j1][w] uc[i0c][ps1[j1]+w];  uf[j0][j1] += sum_w pw0[j0][w] tmp[ps0[j0]+w][j1]
__global__ void k_prolong_a(const TransferDev* __restrict__ tds, const double* __restrict__ uc,
                            double* __restrict__ tmp) {
  const TransferDev td = tds[blockIdx.z];
  int j1 = blockIdx.x * blockDim.x + threadIdx.x, i0c = blockIdx.y;
  if (i0c >= td.nc[0] || j1 >= td.nf[1]) return;
  const int W = td.wp[1];
  const double* w = td.pw[1] + int64_t(j1) * W;
  int c1 = td.ps[1][j1];
  const double* row = uc + td.off_c + int64_t(i0c) * td.nc[1];
  double acc = 0.0;
  for (int a = 0; a < W; ++a) {
    int i1c = c1 + a;
    if (i1c < td.nc[1]) acc = fma(w[a], row[i1c], acc);
  }
  tmp[td.off_t + int64_t(i0c) * td.nf[1] + j1] = acc;
}

__global__ void k_prolong_b(const TransferDev* __restrict__ tds, const double* __restrict__ tmp,
                            double* __restrict__ uf) {
  const TransferDev td = tds[blockIdx.z];
  int j1 = blockIdx.x * blockDim.x + threadIdx.x, j0 = blockIdx.y;
  if (j0 >= td.nf[0] || j1 >= td.nf[1]) return;
  const int W = td.wp[0];
  const double* w = td.pw[0] + int64_t(j0) * W;
  int c0 = td.ps[0][j0];
  double acc = 0.0;
  for (int a = 0; a < W; ++a) {
    int i0c = c0 + a;
    if (i0c < td.nc[0]) acc = fma(w[a], tmp[td.off_t + int64_t(i0c) * td.nf[1] + j1], acc);
  }
  uf[td.off_f + int64_t(j0) * td.nf[1] + j1] += acc;
}

cudaError_t launch_restrict_2d(cudaStream_t s, const TransferDev* td, int K, int max_nf,
                               int max_nc, const double* rf, double* tmp, double* rc,
                               const int64_t* l2g_c, int64_t Tc) {
  (void)Tc;
  k_restrict_a<<<dim3((max_nf + 127) / 128, max_nc, K), 128, 0, s>>>(td, rf, tmp);
  k_restrict_b<<<dim3((max_nc + 127) / 128, max_nc, K), 128, 0, s>>>(td, tmp, rc, l2g_c);
  return cudaGetLastError();
}

cudaError_t launch_prolong_2d(cudaStream_t s, const TransferDev* td, int K, int max_nf,
                              int max_nc, const double* uc, double* tmp, double* uf) {
  k_prolong_a<<<dim3((max_nf + 127) / 128, max_nc, K), 128, 0, s>>>(td, uc, tmp);
  k_prolong_b<<<dim3((max_nf + 127) / 128, max_nf, K), 128, 0, s>>>(td, tmp, uf);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- coarse solve (Sec. 4)

__global__ void k_coarse_solve(int64_t N0, const int64_t* __restrict__ ptr, const int64_t* __restrict__ idx,
                               const double* __restrict__ Ainv, const double* __restrict__ f,
                               double* __restrict__ x) {
  extern __shared__ double g[];
  for (int64_t i = threadIdx.x; i < N0; i += blockDim.x) {
    double s = 0.0;
    for (int64_t c = ptr[i]; c < ptr[i + 1]; ++c) s += f[idx[c]];
    g[i] = s;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int64_t r = int64_t(blockIdx.x) * nw + warp; r < N0; r += int64_t(gridDim.x) * nw) {
    double acc = 0.0;
    for (int64_t c = lane; c < N0; c += 32) acc = fma(Ainv[r * N0 + c], g[c], acc);
    acc = warp_sum(acc);
    acc = __shfl_sync(0xffffffffu, acc, 0);
    for (int64_t c = ptr[r] + lane; c < ptr[r + 1]; c += 32) x[idx[c]] = acc;
  }
}

cudaError_t launch_coarse_solve(cudaStream_t s, int64_t N0, const int64_t* ptr,
                                const int64_t* idx, const double* A0inv, const double* f,
                                double* x) {
  if (N0 <= 0) return cudaSuccess;
  int blocks = int((N0 + 7) / 8);
  if (blocks > 152) blocks = 152;
  k_coarse_solve<<<blocks, 256, sizeof(double) * N0, s>>>(N0, ptr, idx, A0inv, f, x);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- global <-> tiles

__global__ void k_global_to_tile(int64_t N, const int64_t* __restrict__ ptr, const int64_t* __restrict__ idx,
                                 const double* __restrict__ xg, double* __restrict__ xt, int first_only) {
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < N; g += int64_t(gridDim.x) * blockDim.x) {
    double v = xg[g];
    for (int64_t c = ptr[g]; c < ptr[g + 1]; ++c) xt[idx[c]] = (first_only && c > ptr[g]) ? 0.0 : v;
  }
}

__global__ void k_tile_to_global(int64_t N, const int64_t* __restrict__ ptr, const int64_t* __restrict__ idx,
                                 const double* __restrict__ xt, double* __restrict__ xg, int sum_copies) {
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < N; g += int64_t(gridDim.x) * blockDim.x) {
    double v = xt[idx[ptr[g]]];
    if (sum_copies)
      for (int64_t c = ptr[g] + 1; c < ptr[g + 1]; ++c) v += xt[idx[c]];
    xg[g] = v;
  }
}

cudaError_t launch_global_to_tile(cudaStream_t s, int64_t N, const int64_t* ptr,
                                  const int64_t* idx, const double* xg, double* xt, int first_only) {
  if (N <= 0) return cudaSuccess;
  k_global_to_tile<<<grid_for(N, 256), 256, 0, s>>>(N, ptr, idx, xg, xt, first_only);
  return cudaGetLastError();
}

cudaError_t launch_tile_to_global(cudaStream_t s, int64_t N, const int64_t* ptr,
                                  const int64_t* idx, const double* xt, double* xg, int sum_copies) {
  if (N <= 0) return cudaSuccess;
  k_tile_to_global<<<grid_for(N, 256), 256, 0, s>>>(N, ptr, idx, xt, xg, sum_copies);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- reductions, PCG

__global__ void __launch_bounds__(256) k_dot_partial(const double* __restrict__ a, const double* __restrict__ b,
                                                     int64_t n, double* __restrict__ partials) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t i = blockIdx.x * int64_t(256) + threadIdx.x; i < n; i += int64_t(gridDim.x) * 256)
    s = fma(a[i], b[i], s);
  s = block_sum_256(s, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_norm2_dist_partial(int64_t N, const int64_t* __restrict__ ptr,
                                                            const int64_t* __restrict__ idx,
                                                            const double* __restrict__ v,
                                                            double* __restrict__ partials) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t g = blockIdx.x * int64_t(256) + threadIdx.x; g < N; g += int64_t(gridDim.x) * 256) {
    double c = 0.0;
    for (int64_t k = ptr[g]; k < ptr[g + 1]; ++k) c += v[idx[k]];
    s = fma(c, c, s);
  }
  s = block_sum_256(s, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_reduce_final(const double* __restrict__ partials, int nb,
                                                      double* __restrict__ out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += 256) s += partials[i];
  s = block_sum_256(s, sh);
  if (threadIdx.x == 0) *out = s;
}

cudaError_t launch_dot(cudaStream_t s, const double* a, const double* b, int64_t n,
                       double* partials, double* out) {
  k_dot_partial<<<RED_BLOCKS, 256, 0, s>>>(a, b, n, partials);
  k_reduce_final<<<1, 256, 0, s>>>(partials, RED_BLOCKS, out);
  return cudaGetLastError();
}

cudaError_t launch_norm2_dist(cudaStream_t s, int64_t N, const int64_t* ptr, const int64_t* idx,
                              const double* v, double* partials, double* out) {
  k_norm2_dist_partial<<<RED_BLOCKS, 256, 0, s>>>(N, ptr, idx, v, partials);
  k_reduce_final<<<1, 256, 0, s>>>(partials, RED_BLOCKS, out);
  return cudaGetLastError();
}

__global__ void k_pcg_xr(int64_t n, const double* __restrict__ scal, double* __restrict__ x,
                         double* __restrict__ r, const double* __restrict__ p, const double* __restrict__ w) {
  const double alpha = scal[0] / scal[1];
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    r[i] = fma(-alpha, w[i], r[i]);
  }
}

__global__ void k_pcg_p(int64_t n, const double* __restrict__ scal, double* __restrict__ p,
                        const double* __restrict__ z) {
  const double beta = scal[2] / scal[0];
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

__global__ void k_scalar_shift(double* scal) { scal[0] = scal[2]; }

__global__ void k_axpby(int64_t n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

cudaError_t launch_pcg_xr(cudaStream_t s, int64_t n, const double* scal, double* x, double* r,
                          const double* p, const double* w) {
  k_pcg_xr<<<grid_for(n, 256), 256, 0, s>>>(n, scal, x, r, p, w);
  return cudaGetLastError();
}

cudaError_t launch_pcg_p(cudaStream_t s, int64_t n, double* scal, double* p, const double* z) {
  k_pcg_p<<<grid_for(n, 256), 256, 0, s>>>(n, scal, p, z);
  k_scalar_shift<<<1, 1, 0, s>>>(scal);
  return cudaGetLastError();
}

cudaError_t launch_axpby(cudaStream_t s, int64_t n, double a, const double* x, double b, double* y) {
  k_axpby<<<grid_for(n, 256), 256, 0, s>>>(n, a, x, b, y);
  return cudaGetLastError();
}

}  // namespace igamg
