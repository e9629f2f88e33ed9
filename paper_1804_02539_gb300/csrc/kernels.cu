// Device kernels of the multi-patch multigrid solver (2D and 3D tiles; FP64, and FP32 /
// BF16-band twins for the precision variant), except the tensor-core GEMM (tc_gemm.cu).
//
// Layout: a level vector is the concatenation of per-patch tiles (C order, last direction
// fastest); a global dof shared by several patches has one copy per owner (Sec. 4: the
// processor-local parts of accumulated/distributed vectors, here all on one device).
// Band storage of A_{l,k}: band[band_off + t * nn + node] with t the flattened offset
// (j - i + p) over (2p+1)^d, tap-major so that a warp reads 32 consecutive rows of one tap.
#include "kernels.cuh"

#include <map>
#include <mutex>
#include <utility>

namespace igamg {

cudaError_t ensure_smem(const void* func, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;  // within the default limit
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> set;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = set[std::make_pair(dev, func)];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  if (e == cudaSuccess) cur = bytes;
  return e;
}


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

// ---------------------------------------------------------------- stiffness apply

// y = f - A u (f != NULL) or y = A u, per patch tile; u staged in shared memory with a
// halo of p in every direction (zero outside the tile).  TV: vector/accumulator type,
// TB: band storage type (FP64, FP32 or BF16 bands; BF16 and FP32 accumulate in FP32).
template <class T> __device__ __forceinline__ float to_acc(T v);
template <> __device__ __forceinline__ float to_acc<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_acc<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// Band coefficients are read once per apply.  The 2D apply loads FP32 and BF16 bands
// without L1 allocation and with 256-byte L2 prefetch (its tap planes are read along long
// rows); the 3D apply, whose row blocks span 32 nodes of short rows, keeps plain loads
// (the prefetch measured slower there).  FP64 bands (FP64-pipe bound) use the read-only path.
__device__ __forceinline__ float ld_band_stream(const float* p) {
  float v;
  asm("ld.global.nc.L1::no_allocate.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_band_stream(const __nv_bfloat16* p) {
  unsigned short r;
  asm("ld.global.nc.L1::no_allocate.L2::256B.b16 %0, [%1];" : "=h"(r) : "l"(p));
  return __bfloat162float(__ushort_as_bfloat16(r));
}

template <class TV, class TB>
__device__ __forceinline__ TV band_val(const TB* p) {
  if constexpr (sizeof(TV) == sizeof(TB) && std::is_same<TV, TB>::value) return __ldg(p);
  else return TV(to_acc<TB>(*p));
}
template <class TV, class TB>
__device__ __forceinline__ TV band_val_stream(const TB* p) {
  if constexpr (std::is_same<TB, double>::value) return TV(__ldg(p));
  else return TV(ld_band_stream(p));
}

// P > 0: every patch has degree P (taps unrolled; one partial sum per tap row, so a thread
// runs 2P+1 independent FMA chains); P = 0: any degrees.
template <class TV, class TB, int P>
__global__ void __launch_bounds__(AX * AY) k_band_apply_2d(const PatchDev* __restrict__ pds,
                                                           const TB* __restrict__ band,
                                                           const TV* __restrict__ u,
                                                           const TV* __restrict__ f,
                                                           TV* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TV* su = reinterpret_cast<TV*>(smraw);
  const PatchDev pd = pds[blockIdx.z];
  const int n0 = pd.n[0], n1 = pd.n[1];
  const int p0 = P ? P : pd.p[0], p1 = P ? P : pd.p[1];
  const int i0b = blockIdx.y * AY, i1b = blockIdx.x * AX;
  if (i0b >= n0 || i1b >= n1) return;
  const int H0 = AY + 2 * p0, H1 = AX + 2 * p1;
  const TV* ut = u + pd.off;
  for (int idx = threadIdx.y * AX + threadIdx.x; idx < H0 * H1; idx += AX * AY) {
    int r = idx / H1, c = idx % H1;
    int g0 = i0b - p0 + r, g1 = i1b - p1 + c;
    su[idx] = (g0 >= 0 && g0 < n0 && g1 >= 0 && g1 < n1) ? ut[int64_t(g0) * n1 + g1] : TV(0);
  }
  __syncthreads();
  const int i0 = i0b + threadIdx.y, i1 = i1b + threadIdx.x;
  if (i0 >= n0 || i1 >= n1) return;
  const int64_t nn = int64_t(n0) * n1, node = int64_t(i0) * n1 + i1;
  const TB* bp = band + pd.band_off + node;
  TV acc = 0;
  if constexpr (P > 0) {
    constexpr int W = 2 * P + 1;
    TV part[W];
#pragma unroll
    for (int t0 = 0; t0 < W; ++t0) {
      const TV* srow = su + (threadIdx.y + t0) * H1 + threadIdx.x;
      part[t0] = TV(0);
#pragma unroll
      for (int t1 = 0; t1 < W; ++t1)
        part[t0] = fma(band_val_stream<TV, TB>(bp + int64_t(t0 * W + t1) * nn), srow[t1], part[t0]);
    }
#pragma unroll
    for (int t0 = 0; t0 < W; ++t0) acc += part[t0];
  } else {
    const int w1 = 2 * p1 + 1;
    for (int t0 = 0; t0 <= 2 * p0; ++t0) {
      const TV* srow = su + (threadIdx.y + t0) * H1 + threadIdx.x;
      const TB* brow = bp + int64_t(t0 * w1) * nn;
      for (int t1 = 0; t1 < w1; ++t1) acc = fma(band_val_stream<TV, TB>(brow + int64_t(t1) * nn), srow[t1], acc);
    }
  }
  y[pd.off + node] = f ? f[pd.off + node] - acc : acc;
}

template <class TV, class TB, int P>
static void launch_apply_2d_p(cudaStream_t s, dim3 grid, size_t sm, const PatchDev* pd_dev, const TB* band,
                              const TV* u, const TV* f, TV* y) {
  k_band_apply_2d<TV, TB, P><<<grid, dim3(AX, AY), sm, s>>>(pd_dev, band, u, f, y);
}

template <class TV, class TB>
cudaError_t launch_band_apply_2d(cudaStream_t s, const PatchDev* pd_dev, int K, int max_n0,
                                 int max_n1, int max_p, const TB* band, const TV* u,
                                 const TV* f, TV* y, int uniform_p) {
  dim3 grid((max_n1 + AX - 1) / AX, (max_n0 + AY - 1) / AY, K);
  size_t sm = sizeof(TV) * (AY + 2 * max_p) * (AX + 2 * max_p);
  switch (uniform_p) {
    case 1: launch_apply_2d_p<TV, TB, 1>(s, grid, sm, pd_dev, band, u, f, y); break;
    case 2: launch_apply_2d_p<TV, TB, 2>(s, grid, sm, pd_dev, band, u, f, y); break;
    case 3: launch_apply_2d_p<TV, TB, 3>(s, grid, sm, pd_dev, band, u, f, y); break;
    case 4: launch_apply_2d_p<TV, TB, 4>(s, grid, sm, pd_dev, band, u, f, y); break;
    case 5: launch_apply_2d_p<TV, TB, 5>(s, grid, sm, pd_dev, band, u, f, y); break;
    case 6: launch_apply_2d_p<TV, TB, 6>(s, grid, sm, pd_dev, band, u, f, y); break;
    default: launch_apply_2d_p<TV, TB, 0>(s, grid, sm, pd_dev, band, u, f, y);
  }
  return cudaGetLastError();
}
template cudaError_t launch_band_apply_2d<double, double>(cudaStream_t, const PatchDev*, int, int, int, int,
                                                          const double*, const double*, const double*, double*, int);
template cudaError_t launch_band_apply_2d<float, float>(cudaStream_t, const PatchDev*, int, int, int, int,
                                                        const float*, const float*, const float*, float*, int);
template cudaError_t launch_band_apply_2d<float, __nv_bfloat16>(cudaStream_t, const PatchDev*, int, int, int, int,
                                                                const __nv_bfloat16*, const float*, const float*,
                                                                float*, int);

// ---------------------------------------------------------------- Kronecker-sum apply

// One block computes KY x AX outputs of one rectangle patch.  Pass 1 contracts the u halo
// (KY + 2p0 rows) along direction 1 with M_1 and K_1; pass 2 contracts those along
// direction 0 with K_0 and M_0: 4(2p1+1)(1 + 2p0/KY) + 4(2p0+1) flops per output and no
// operator traffic beyond the 1D bands (L1-resident).
constexpr int KY = 16;

size_t kron_apply_smem(int elem_size, int max_p) {
  return size_t(elem_size) * ((KY + 2 * max_p) * (AX + 2 * max_p) + 2 * (KY + 2 * max_p) * AX);
}

template <class T>
__device__ __forceinline__ void kron_apply_block(const KronDevT<T>& kd, const unsigned char* __restrict__ active,
                                                 const T* __restrict__ u, const T* __restrict__ f,
                                                 T* __restrict__ y, unsigned char* smraw) {
  const int n0 = kd.n0, n1 = kd.n1, p0 = kd.p0, p1 = kd.p1;
  const int i0b = blockIdx.y * KY, i1b = blockIdx.x * AX;
  if (i0b >= n0 || i1b >= n1) return;
  const int H0 = KY + 2 * p0, H1 = AX + 2 * p1;
  T* su = reinterpret_cast<T*>(smraw);
  T* sa = su + H0 * H1;  // M_1-contracted halo rows
  T* sb = sa + H0 * AX;  // K_1-contracted halo rows
  const int tid = threadIdx.y * AX + threadIdx.x;
  const T* ut = u + kd.off;
  const unsigned char* at = active + kd.off;
  for (int idx = tid; idx < H0 * H1; idx += AX * AY) {
    int r = idx / H1, cc = idx % H1;
    int g0 = i0b - p0 + r, g1 = i1b - p1 + cc;
    T v = T(0);
    if (g0 >= 0 && g0 < n0 && g1 >= 0 && g1 < n1) {
      int64_t node = int64_t(g0) * n1 + g1;
      if (at[node]) v = ut[node];
    }
    su[idx] = v;
  }
  __syncthreads();
  const int w1 = 2 * p1 + 1, w0 = 2 * p0 + 1;
  {
    const int cx = threadIdx.x, i1 = i1b + cx;
    const T* mrow = kd.M1 + int64_t(min(i1, n1 - 1)) * w1;
    const T* krow = kd.K1 + int64_t(min(i1, n1 - 1)) * w1;
    for (int r = threadIdx.y; r < H0; r += AY) {
      const T* srow = su + r * H1 + cx;
      T a = T(0), b = T(0);
      for (int t = 0; t < w1; ++t) {
        T v = srow[t];
        a = fma(mrow[t], v, a);
        b = fma(krow[t], v, b);
      }
      sa[r * AX + cx] = a;
      sb[r * AX + cx] = b;
    }
  }
  __syncthreads();
  const int i1 = i1b + threadIdx.x;
  if (i1 >= n1) return;
  for (int r = threadIdx.y; r < KY; r += AY) {
    const int i0 = i0b + r;
    if (i0 >= n0) break;
    const T* krow = kd.K0 + int64_t(i0) * w0;
    const T* mrow = kd.M0 + int64_t(i0) * w0;
    T a = T(0), b = T(0);
    for (int t = 0; t < w0; ++t) {
      a = fma(krow[t], sa[(r + t) * AX + threadIdx.x], a);
      b = fma(mrow[t], sb[(r + t) * AX + threadIdx.x], b);
    }
    const int64_t node = kd.off + int64_t(i0) * n1 + i1;
    T acc = active[node] ? kd.c0 * a + kd.c1 * b : T(0);
    y[node] = f ? f[node] - acc : acc;
  }
}

template <class T>
__global__ void __launch_bounds__(AX * AY) k_kron_apply_2d(const KronDevT<T>* __restrict__ kds,
                                                           const unsigned char* __restrict__ active,
                                                           const T* __restrict__ u, const T* __restrict__ f,
                                                           T* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char smraw[];
  kron_apply_block<T>(kds[blockIdx.z], active, u, f, y, smraw);
}

// The same apply over patch jobs of many levels or problems (each with its own vectors).
template <class T>
__global__ void __launch_bounds__(AX * AY) k_kron_apply_2d_b(const KronJobT<T>* __restrict__ jobs) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const KronJobT<T> j = jobs[blockIdx.z];
  kron_apply_block<T>(j.kd, j.active, j.u, j.f, j.y, smraw);
}

template <class T>
cudaError_t launch_kron_apply_2d_b(cudaStream_t s, const KronJobT<T>* jobs, int njobs, int max_n0, int max_n1,
                                   int max_p) {
  if (njobs <= 0) return cudaSuccess;
  dim3 grid((max_n1 + AX - 1) / AX, (max_n0 + KY - 1) / KY, njobs);
  size_t sm = kron_apply_smem(sizeof(T), max_p);
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(k_kron_apply_2d_b<T>), sm);
  if (e != cudaSuccess) return e;
  k_kron_apply_2d_b<T><<<grid, dim3(AX, AY), sm, s>>>(jobs);
  return cudaGetLastError();
}
template cudaError_t launch_kron_apply_2d_b<double>(cudaStream_t, const KronJobT<double>*, int, int, int, int);

template <class T>
cudaError_t launch_kron_apply_2d(cudaStream_t s, const KronDevT<T>* kd, int K, int max_n0, int max_n1, int max_p,
                                 const unsigned char* active, const T* u, const T* f, T* y) {
  dim3 grid((max_n1 + AX - 1) / AX, (max_n0 + KY - 1) / KY, K);
  size_t sm = kron_apply_smem(sizeof(T), max_p);
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(k_kron_apply_2d<T>), sm);
  if (e != cudaSuccess) return e;
  k_kron_apply_2d<T><<<grid, dim3(AX, AY), sm, s>>>(kd, active, u, f, y);
  return cudaGetLastError();
}
template cudaError_t launch_kron_apply_2d<double>(cudaStream_t, const KronDevT<double>*, int, int, int, int,
                                                  const unsigned char*, const double*, const double*, double*);
template cudaError_t launch_kron_apply_2d<float>(cudaStream_t, const KronDevT<float>*, int, int, int, int,
                                                 const unsigned char*, const float*, const float*, float*);

// ---------------------------------------------------------------- small-interior FD

template <class T>
__device__ void fd_small_block(const FdSmallT<T>& d, int from_F, T tau, int add, T* U0, T* U1, T* X, T* Tm) {
  const int n0 = d.n0, n1 = d.n1, tid = threadIdx.x;
  const T* v = from_F ? d.vF : d.vR;
  for (int i = tid; i < n0 * n0; i += 256) U0[i] = d.U0[i];
  for (int i = tid; i < n1 * n1; i += 256) U1[i] = d.U1[i];
  for (int i = tid; i < n0 * n1; i += 256) X[i] = v[int64_t(i / n1) * d.ld + i % n1];
  __syncthreads();
  for (int i = tid; i < n0 * n1; i += 256) {  // T = U0^T X
    const int a = i / n1, b = i % n1;
    T acc = 0;
    for (int k = 0; k < n0; ++k) acc = fma(U0[k * n0 + a], X[k * n1 + b], acc);
    Tm[i] = acc;
  }
  __syncthreads();
  for (int i = tid; i < n0 * n1; i += 256) {  // Y = (T U1) .* Dinv
    const int a = i / n1, b = i % n1;
    T acc = 0;
    for (int k = 0; k < n1; ++k) acc = fma(Tm[a * n1 + k], U1[k * n1 + b], acc);
    X[i] = acc * d.Dinv[i];
  }
  __syncthreads();
  for (int i = tid; i < n0 * n1; i += 256) {  // S = U0 Y
    const int a = i / n1, b = i % n1;
    T acc = 0;
    for (int k = 0; k < n0; ++k) acc = fma(U0[a * n0 + k], X[k * n1 + b], acc);
    Tm[i] = acc;
  }
  __syncthreads();
  for (int i = tid; i < n0 * n1; i += 256) {  // u (=|+=) tau S U1^T
    const int a = i / n1, b = i % n1;
    T acc = 0;
    for (int k = 0; k < n1; ++k) acc = fma(Tm[a * n1 + k], U1[b * n1 + k], acc);
    T* up = d.u + int64_t(a) * d.ld + b;
    *up = add ? fma(tau, acc, *up) : tau * acc;
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_fd_small(const FdSmallT<T>* __restrict__ ds, int from_F, T tau, int add) {
  constexpr int M = kFdSmallMax;
  __shared__ T U0[M * M], U1[M * M], X[M * M], Tm[M * M];
  fd_small_block<T>(ds[blockIdx.x], from_F, tau, add, U0, U1, X, Tm);
}

// Block b of the one-launch small-level smoother of one level (interiors, edges, vertices).
template <class T>
__device__ void smooth_small_block(const SmoothSmallT<T>& p, int b, int from_F, T tau, int add, T* U0, T* U1, T* X,
                                   T* Tm) {
  const int tid = threadIdx.x;
  const T* v = from_F ? p.vF : p.vR;
  if (b < p.nfd) {
    fd_small_block<T>(p.fd[b], from_F, tau, add, U0, U1, X, Tm);
    return;
  }
  if (b < p.nfd + p.nedges) {
    const EdgeSmallT<T> e = p.edges[b - p.nfd];
    const int n = e.len;
    for (int i = tid; i < n * n; i += 256) U0[i] = e.U[i];
    for (int i = tid; i < n; i += 256) {  // gather: the sum of the copies
      const int64_t g = e.first + i;
      T acc = 0;
      for (int64_t c = p.ptr[g]; c < p.ptr[g + 1]; ++c) acc += v[p.idx[c]];
      X[i] = acc;
    }
    __syncthreads();
    for (int j = tid; j < n; j += 256) {  // y = (g^T U) .* dinv
      T acc = 0;
      for (int i = 0; i < n; ++i) acc = fma(X[i], U0[i * n + j], acc);
      Tm[j] = acc * e.dinv[j];
    }
    __syncthreads();
    for (int i = tid; i < n; i += 256) {  // z = U y, scattered to every copy
      T acc = 0;
      for (int j = 0; j < n; ++j) acc = fma(Tm[j], U0[i * n + j], acc);
      const T val = tau * acc;
      const int64_t g = e.first + i;
      for (int64_t c = p.ptr[g]; c < p.ptr[g + 1]; ++c) {
        T* up = p.u + p.idx[c];
        *up = add ? *up + val : val;
      }
    }
    return;
  }
  for (int64_t g = p.vbeg + tid; g < p.vend; g += 256) {  // vertices
    T acc = 0;
    for (int64_t c = p.ptr[g]; c < p.ptr[g + 1]; ++c) acc += v[p.idx[c]];
    const T val = tau * (p.vscale[g] * acc);
    for (int64_t c = p.ptr[g]; c < p.ptr[g + 1]; ++c) {
      T* up = p.u + p.idx[c];
      *up = add ? *up + val : val;
    }
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_smooth_small(const SmoothSmallT<T> p, int from_F, T tau, int add) {
  constexpr int M = kFdSmallMax;
  __shared__ T U0[M * M], U1[M * M], X[M * M], Tm[M * M];
  smooth_small_block<T>(p, blockIdx.x, from_F, tau, add, U0, U1, X, Tm);
}

// The small-level smoothers of many levels (of different problems) in one launch: block b
// belongs to job j with bstart[j] <= b < bstart[j + 1].
template <class T>
__global__ void __launch_bounds__(256) k_smooth_small_b(const SmoothSmallT<T>* __restrict__ jobs,
                                                        const int* __restrict__ bstart, int njobs, int from_F, T tau,
                                                        int add) {
  constexpr int M = kFdSmallMax;
  __shared__ T U0[M * M], U1[M * M], X[M * M], Tm[M * M];
  int lo = 0, hi = njobs;
  const int b = blockIdx.x;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (bstart[mid] <= b) lo = mid;
    else hi = mid;
  }
  const SmoothSmallT<T> p = jobs[lo];
  smooth_small_block<T>(p, b - bstart[lo], from_F, tau, add, U0, U1, X, Tm);
}

template <class T>
cudaError_t launch_smooth_small_b(cudaStream_t s, const SmoothSmallT<T>* jobs, const int* bstart, int njobs,
                                  int total_blocks, int from_F, T tau, int add) {
  if (njobs <= 0 || total_blocks <= 0) return cudaSuccess;
  k_smooth_small_b<T><<<total_blocks, 256, 0, s>>>(jobs, bstart, njobs, from_F, tau, add);
  return cudaGetLastError();
}
template cudaError_t launch_smooth_small_b<double>(cudaStream_t, const SmoothSmallT<double>*, const int*, int, int, int,
                                                   double, int);

template <class T>
cudaError_t launch_smooth_small(cudaStream_t s, const SmoothSmallT<T>& p, int from_F, T tau, int add) {
  const int blocks = p.nfd + p.nedges + (p.vend > p.vbeg ? 1 : 0);
  if (blocks <= 0) return cudaSuccess;
  k_smooth_small<T><<<blocks, 256, 0, s>>>(p, from_F, tau, add);
  return cudaGetLastError();
}
template cudaError_t launch_smooth_small<double>(cudaStream_t, const SmoothSmallT<double>&, int, double, int);
template cudaError_t launch_smooth_small<float>(cudaStream_t, const SmoothSmallT<float>&, int, float, int);

template <class T>
cudaError_t launch_fd_small(cudaStream_t s, const FdSmallT<T>* d, int count, int from_F, T tau, int add) {
  if (count <= 0) return cudaSuccess;
  k_fd_small<T><<<count, 256, 0, s>>>(d, from_F, tau, add);
  return cudaGetLastError();
}
template cudaError_t launch_fd_small<double>(cudaStream_t, const FdSmallT<double>*, int, int, double, int);
template cudaError_t launch_fd_small<float>(cudaStream_t, const FdSmallT<float>*, int, int, float, int);

// ---------------------------------------------------------------- row-block FD

constexpr int FR_RB = 8;  // rows per block

template <class T>
__global__ void __launch_bounds__(256) k_fd_rows(const FdRowsT<T>* __restrict__ ds, int pass, int from_F, T tau,
                                                 int add) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* rowsS = reinterpret_cast<T*>(smraw);  // FR_RB x n1: this block's rows of T (pass 1) or S (pass 2)
  const FdRowsT<T> d = ds[blockIdx.y];
  const int n0 = d.n0, n1 = d.n1, a0 = blockIdx.x * FR_RB;
  if (a0 >= n0) return;
  const int rb = min(FR_RB, n0 - a0), tid = threadIdx.x;
  // first product: rows a0.. of U0^T X (pass 1) or U0 Y (pass 2), contracted over all n0 rows
  const T* src = pass == 1 ? (from_F ? d.vF : d.vR) : d.Y;
  const int lds = pass == 1 ? d.ld : n1;
  for (int o = tid; o < rb * n1; o += 256) {
    const int r = o / n1, b = o % n1, a = a0 + r;
    T acc = 0;
    for (int k = 0; k < n0; ++k) {
      const T u0 = pass == 1 ? d.U0[k * n0 + a] : d.U0[a * n0 + k];
      acc = fma(u0, src[int64_t(k) * lds + b], acc);
    }
    rowsS[r * n1 + b] = acc;
  }
  __syncthreads();
  // second product: these rows times U1 (pass 1, then .* Dinv into Y) or U1^T (pass 2, into u)
  for (int o = tid; o < rb * n1; o += 256) {
    const int r = o / n1, b = o % n1, a = a0 + r;
    T acc = 0;
    for (int k = 0; k < n1; ++k) {
      const T u1 = pass == 1 ? d.U1[k * n1 + b] : d.U1[b * n1 + k];
      acc = fma(rowsS[r * n1 + k], u1, acc);
    }
    if (pass == 1) {
      d.Y[a * n1 + b] = acc * d.Dinv[a * n1 + b];
    } else {
      T* up = d.u + int64_t(a) * d.ld + b;
      *up = add ? fma(tau, acc, *up) : tau * acc;
    }
  }
}

template <class T>
cudaError_t launch_fd_rows(cudaStream_t s, const FdRowsT<T>* d, int count, int max_n0, int max_n1, int pass,
                           int from_F, T tau, int add) {
  if (count <= 0) return cudaSuccess;
  const size_t sm = sizeof(T) * FR_RB * size_t(max_n1);
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(k_fd_rows<T>), sm);
  if (e != cudaSuccess) return e;
  dim3 grid((max_n0 + FR_RB - 1) / FR_RB, count);
  k_fd_rows<T><<<grid, 256, sm, s>>>(d, pass, from_F, tau, add);
  return cudaGetLastError();
}
template cudaError_t launch_fd_rows<double>(cudaStream_t, const FdRowsT<double>*, int, int, int, int, int, double,
                                            int);
template cudaError_t launch_fd_rows<float>(cudaStream_t, const FdRowsT<float>*, int, int, int, int, int, float, int);

// ---------------------------------------------------------------- batched GEMM

// C = op(A) op(B) with an epilogue, one output tile of 8R x 8R per block of 64 threads;
// thread (tx, ty) owns rows ty + 8r and columns tx + 8c (r, c < R).  Rows/columns of the
// tile beyond M/N and the k-slab beyond K are skipped warp-uniformly, so ragged sizes
// (e.g. 258 = 8*32 + 2) waste FMA work only at 8-granularity.  T = double (FP64 path) or
// float (FP32 inner solves).
namespace {
constexpr int GK = 16;

template <int R, class T>
__device__ __forceinline__ void gemm_tile(const GemmDescT<T>& d, int ta, int tb, int epi, T alpha,
                                          int bx, int by) {
  constexpr int BT = 8 * R;
  const int i0 = by * BT, j0 = bx * BT;
  if (i0 >= d.M || j0 >= d.N) return;
  __shared__ T As[GK][BT + 1];
  __shared__ T Bs[GK][BT + 1];
  const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
  const int wty = (tid >> 5) * 4;  // smallest ty of this warp
  int rv = 0, cv = 0;              // warp-uniform counts of live micro-rows / micro-columns
#pragma unroll
  for (int r = 0; r < R; ++r) rv += (i0 + wty + 8 * r < d.M) ? 1 : 0;
#pragma unroll
  for (int c = 0; c < R; ++c) cv += (j0 + 8 * c < d.N) ? 1 : 0;
  T acc[R][R];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) acc[r][c] = T(0);
  for (int k0 = 0; k0 < d.K; k0 += GK) {
    for (int idx = tid; idx < BT * GK; idx += 64) {
      int i, kk;
      if (ta) { i = idx % BT; kk = idx / BT; } else { kk = idx % GK; i = idx / GK; }
      int gi = i0 + i, gk = k0 + kk;
      T v = T(0);
      if (gi < d.M && gk < d.K) v = ta ? d.A[int64_t(gk) * d.lda + gi] : d.A[int64_t(gi) * d.lda + gk];
      As[kk][i] = v;
      int j;
      if (tb) { kk = idx % GK; j = idx / GK; } else { j = idx % BT; kk = idx / BT; }
      int gj = j0 + j;
      gk = k0 + kk;
      v = T(0);
      if (gj < d.N && gk < d.K) v = tb ? d.B[int64_t(gj) * d.ldb + gk] : d.B[int64_t(gk) * d.ldb + gj];
      Bs[kk][j] = v;
    }
    __syncthreads();
    const int kmax = min(GK, d.K - k0);
    for (int kk = 0; kk < kmax; ++kk) {
      T a[R], b[R];
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
      T v = acc[r][c];
      T* cp = d.C + int64_t(gi) * d.ldc + gj;
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

template <int R, class T>
__global__ void __launch_bounds__(64) k_gemm(const GemmDescT<T>* __restrict__ descs, int ta, int tb, int epi,
                                             T alpha) {
  gemm_tile<R, T>(descs[blockIdx.z], ta, tb, epi, alpha, blockIdx.x, blockIdx.y);
}

template <int R, class T>
__global__ void __launch_bounds__(64) k_gemm_one(GemmDescT<T> d, int ta, int tb, int epi, T alpha) {
  gemm_tile<R, T>(d, ta, tb, epi, alpha, blockIdx.x, blockIdx.y);
}

// Tile edge 8R: 32 when the 32-wide grid already fills the GPU twice, else 16, else 8.
static int pick_r(int maxM, int maxN, int batch) {
  auto tiles = [&](int bt) { return int64_t((maxM + bt - 1) / bt) * ((maxN + bt - 1) / bt) * batch; };
  if (tiles(32) >= 2 * 152) return 4;
  if (tiles(16) >= 152) return 2;
  return 1;
}

template <class T>
cudaError_t launch_gemm(cudaStream_t s, const GemmDescT<T>* d_desc, int batch, int maxM, int maxN,
                        bool transA, bool transB, int epi, T alpha, int R) {
  if (batch <= 0) return cudaSuccess;
  if (R != 1 && R != 2 && R != 4) R = pick_r(maxM, maxN, batch);
  const int bt = 8 * R;
  dim3 grid((maxN + bt - 1) / bt, (maxM + bt - 1) / bt, batch);
  if (R == 4) k_gemm<4, T><<<grid, 64, 0, s>>>(d_desc, transA, transB, epi, alpha);
  else if (R == 2) k_gemm<2, T><<<grid, 64, 0, s>>>(d_desc, transA, transB, epi, alpha);
  else k_gemm<1, T><<<grid, 64, 0, s>>>(d_desc, transA, transB, epi, alpha);
  return cudaGetLastError();
}
template cudaError_t launch_gemm<double>(cudaStream_t, const GemmDescT<double>*, int, int, int, bool, bool, int, double,
                                         int);
template cudaError_t launch_gemm<float>(cudaStream_t, const GemmDescT<float>*, int, int, int, bool, bool, int, float,
                                        int);

cudaError_t launch_gemm_one(cudaStream_t s, const GemmDesc& d, bool transA, bool transB, int epi,
                            double alpha) {
  int R = pick_r(d.M, d.N, 1), bt = 8 * R;
  dim3 grid((d.N + bt - 1) / bt, (d.M + bt - 1) / bt, 1);
  if (R == 4) k_gemm_one<4, double><<<grid, 64, 0, s>>>(d, transA, transB, epi, alpha);
  else if (R == 2) k_gemm_one<2, double><<<grid, 64, 0, s>>>(d, transA, transB, epi, alpha);
  else k_gemm_one<1, double><<<grid, 64, 0, s>>>(d, transA, transB, epi, alpha);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- interface pieces

template <class T>
__global__ void k_iface_gather(int64_t n, const int64_t* __restrict__ ptr, const int64_t* __restrict__ idx,
                               const T* __restrict__ v, T* __restrict__ G) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    T s = 0;
    for (int64_t c = ptr[i]; c < ptr[i + 1]; ++c) s += v[idx[c]];
    G[i] = s;
  }
}

template <class T>
__global__ void k_iface_scatter(int64_t n, const int64_t* __restrict__ ptr, const int64_t* __restrict__ idx,
                                const T* __restrict__ Z, const T* __restrict__ G,
                                const T* __restrict__ vs, T tau, int add, T* __restrict__ u) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    T val = tau * fma(vs[i], G[i], Z[i]);
    for (int64_t c = ptr[i]; c < ptr[i + 1]; ++c) {
      int64_t t = idx[c];
      u[t] = add ? u[t] + val : val;
    }
  }
}

// Canonical distributed form: for every interface node the sum of its copies goes to the
// first copy and the other copies become zero (same global vector, no cancellation
// between copies).
template <class T>
__global__ void k_canonicalize(int64_t n, const int64_t* __restrict__ ptr, const int64_t* __restrict__ idx,
                               T* __restrict__ v) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    T s = 0;
    for (int64_t c = ptr[i]; c < ptr[i + 1]; ++c) s += v[idx[c]];
    v[idx[ptr[i]]] = s;
    for (int64_t c = ptr[i] + 1; c < ptr[i + 1]; ++c) v[idx[c]] = T(0);
  }
}

static int grid_for(int64_t n, int threads, int cap = 4 * 152 * 8) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  return int(g < cap ? g : cap);
}

template <class T>
cudaError_t launch_iface_gather(cudaStream_t s, int64_t n_nodes, const int64_t* ptr,
                                const int64_t* idx, const T* v, T* G) {
  if (n_nodes <= 0) return cudaSuccess;
  k_iface_gather<T><<<grid_for(n_nodes, 256), 256, 0, s>>>(n_nodes, ptr, idx, v, G);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_iface_scatter(cudaStream_t s, int64_t n_nodes, const int64_t* ptr,
                                 const int64_t* idx, const T* Z, const T* G,
                                 const T* vscale, T tau, int add, T* u) {
  if (n_nodes <= 0) return cudaSuccess;
  k_iface_scatter<T><<<grid_for(n_nodes, 256), 256, 0, s>>>(n_nodes, ptr, idx, Z, G, vscale, tau, add, u);
  return cudaGetLastError();
}
template <class T>
cudaError_t launch_canonicalize(cudaStream_t s, int64_t n_nodes, const int64_t* ptr, const int64_t* idx, T* v) {
  if (n_nodes <= 0) return cudaSuccess;
  k_canonicalize<T><<<grid_for(n_nodes, 256), 256, 0, s>>>(n_nodes, ptr, idx, v);
  return cudaGetLastError();
}
template cudaError_t launch_canonicalize<double>(cudaStream_t, int64_t, const int64_t*, const int64_t*, double*);
template cudaError_t launch_canonicalize<float>(cudaStream_t, int64_t, const int64_t*, const int64_t*, float*);

#define INST_IF(T)                                                                                          \
  template cudaError_t launch_iface_gather<T>(cudaStream_t, int64_t, const int64_t*, const int64_t*, const T*, T*); \
  template cudaError_t launch_iface_scatter<T>(cudaStream_t, int64_t, const int64_t*, const int64_t*, const T*,     \
                                               const T*, const T*, T, int, T*);
INST_IF(double)
INST_IF(float)

// ---------------------------------------------------------------- coarse solve (Sec. 4)

// x_copies = A0^{-1} (sum of copies of f), in FP64 whatever the vector type T.
template <class T>
__global__ void k_coarse_solve(int64_t N0, const int64_t* __restrict__ ptr, const int64_t* __restrict__ idx,
                               const double* __restrict__ Ainv, const T* __restrict__ f, T* __restrict__ x) {
  extern __shared__ double g[];
  for (int64_t i = threadIdx.x; i < N0; i += blockDim.x) {
    double s = 0.0;
    for (int64_t c = ptr[i]; c < ptr[i + 1]; ++c) s += double(f[idx[c]]);
    g[i] = s;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int64_t r = int64_t(blockIdx.x) * nw + warp; r < N0; r += int64_t(gridDim.x) * nw) {
    double acc = 0.0;
    for (int64_t c = lane; c < N0; c += 32) acc = fma(Ainv[r * N0 + c], g[c], acc);
    acc = warp_sum(acc);
    acc = __shfl_sync(0xffffffffu, acc, 0);
    for (int64_t c = ptr[r] + lane; c < ptr[r + 1]; c += 32) x[idx[c]] = T(acc);
  }
}

template <class T>
cudaError_t launch_coarse_solve(cudaStream_t s, int64_t N0, const int64_t* ptr,
                                const int64_t* idx, const double* A0inv, const T* f, T* x) {
  if (N0 <= 0) return cudaSuccess;
  int blocks = int((N0 + 7) / 8);
  if (blocks > 152) blocks = 152;
  k_coarse_solve<T><<<blocks, 256, sizeof(double) * N0, s>>>(N0, ptr, idx, A0inv, f, x);
  return cudaGetLastError();
}
template cudaError_t launch_coarse_solve<double>(cudaStream_t, int64_t, const int64_t*, const int64_t*,
                                                 const double*, const double*, double*);
template cudaError_t launch_coarse_solve<float>(cudaStream_t, int64_t, const int64_t*, const int64_t*,
                                                const double*, const float*, float*);

// ---------------------------------------------------------------- global <-> tiles

template <class T>
__global__ void k_global_to_tile(int64_t N, const int64_t* __restrict__ ptr, const int64_t* __restrict__ idx,
                                 const T* __restrict__ xg, T* __restrict__ xt, int first_only) {
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < N; g += int64_t(gridDim.x) * blockDim.x) {
    T v = xg[g];
    for (int64_t c = ptr[g]; c < ptr[g + 1]; ++c) xt[idx[c]] = (first_only && c > ptr[g]) ? T(0) : v;
  }
}

template <class T>
__global__ void k_tile_to_global(int64_t N, const int64_t* __restrict__ ptr, const int64_t* __restrict__ idx,
                                 const T* __restrict__ xt, T* __restrict__ xg, int sum_copies) {
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < N; g += int64_t(gridDim.x) * blockDim.x) {
    T v = xt[idx[ptr[g]]];
    if (sum_copies)
      for (int64_t c = ptr[g] + 1; c < ptr[g + 1]; ++c) v += xt[idx[c]];
    xg[g] = v;
  }
}

template <class T>
cudaError_t launch_global_to_tile(cudaStream_t s, int64_t N, const int64_t* ptr,
                                  const int64_t* idx, const T* xg, T* xt, int first_only) {
  if (N <= 0) return cudaSuccess;
  k_global_to_tile<T><<<grid_for(N, 256), 256, 0, s>>>(N, ptr, idx, xg, xt, first_only);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_tile_to_global(cudaStream_t s, int64_t N, const int64_t* ptr,
                                  const int64_t* idx, const T* xt, T* xg, int sum_copies) {
  if (N <= 0) return cudaSuccess;
  k_tile_to_global<T><<<grid_for(N, 256), 256, 0, s>>>(N, ptr, idx, xt, xg, sum_copies);
  return cudaGetLastError();
}
template cudaError_t launch_global_to_tile<double>(cudaStream_t, int64_t, const int64_t*, const int64_t*,
                                                   const double*, double*, int);
template cudaError_t launch_tile_to_global<double>(cudaStream_t, int64_t, const int64_t*, const int64_t*,
                                                   const double*, double*, int);

// ---------------------------------------------------------------- reductions, PCG

// Partial sums in FP64 whatever the vector type (deterministic fixed grid).
template <class T>
__global__ void __launch_bounds__(256) k_dot_partial(const T* __restrict__ a, const T* __restrict__ b,
                                                     int64_t n, double* __restrict__ partials) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t i = blockIdx.x * int64_t(256) + threadIdx.x; i < n; i += int64_t(gridDim.x) * 256)
    s = fma(double(a[i]), double(b[i]), s);
  s = block_sum_256(s, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

template <class T>
__global__ void __launch_bounds__(256) k_norm2_dist_partial(int64_t N, const int64_t* __restrict__ ptr,
                                                            const int64_t* __restrict__ idx,
                                                            const T* __restrict__ v,
                                                            double* __restrict__ partials) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t g = blockIdx.x * int64_t(256) + threadIdx.x; g < N; g += int64_t(gridDim.x) * 256) {
    double c = 0.0;
    for (int64_t k = ptr[g]; k < ptr[g + 1]; ++k) c += double(v[idx[k]]);
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

template <class T>
cudaError_t launch_dot(cudaStream_t s, const T* a, const T* b, int64_t n, double* partials, double* out) {
  k_dot_partial<T><<<RED_BLOCKS, 256, 0, s>>>(a, b, n, partials);
  k_reduce_final<<<1, 256, 0, s>>>(partials, RED_BLOCKS, out);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_norm2_dist(cudaStream_t s, int64_t N, const int64_t* ptr, const int64_t* idx,
                              const T* v, double* partials, double* out) {
  k_norm2_dist_partial<T><<<RED_BLOCKS, 256, 0, s>>>(N, ptr, idx, v, partials);
  k_reduce_final<<<1, 256, 0, s>>>(partials, RED_BLOCKS, out);
  return cudaGetLastError();
}
template cudaError_t launch_dot<double>(cudaStream_t, const double*, const double*, int64_t, double*, double*);
template cudaError_t launch_dot<float>(cudaStream_t, const float*, const float*, int64_t, double*, double*);
template cudaError_t launch_norm2_dist<double>(cudaStream_t, int64_t, const int64_t*, const int64_t*,
                                               const double*, double*, double*);
template cudaError_t launch_norm2_dist<float>(cudaStream_t, int64_t, const int64_t*, const int64_t*,
                                              const float*, double*, double*);

template <class T>
__global__ void k_pcg_xr(int64_t n, const double* __restrict__ scal, T* __restrict__ x,
                         T* __restrict__ r, const T* __restrict__ p, const T* __restrict__ w) {
  __shared__ T alpha_s;  // one FP64 division per block, not per thread
  if (threadIdx.x == 0) alpha_s = T(scal[0] / scal[1]);
  __syncthreads();
  const T alpha = alpha_s;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    r[i] = fma(-alpha, w[i], r[i]);
  }
}

template <class T>
__global__ void k_pcg_p(int64_t n, const double* __restrict__ scal, T* __restrict__ p,
                        const T* __restrict__ z) {
  __shared__ T beta_s;
  if (threadIdx.x == 0) beta_s = T(scal[2] / scal[0]);
  __syncthreads();
  const T beta = beta_s;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

__global__ void k_scalar_shift(double* scal) { scal[0] = scal[2]; }

template <class T>
cudaError_t launch_pcg_xr(cudaStream_t s, int64_t n, const double* scal, T* x, T* r, const T* p, const T* w) {
  k_pcg_xr<T><<<grid_for(n, 256), 256, 0, s>>>(n, scal, x, r, p, w);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_pcg_p(cudaStream_t s, int64_t n, double* scal, T* p, const T* z) {
  k_pcg_p<T><<<grid_for(n, 256), 256, 0, s>>>(n, scal, p, z);
  k_scalar_shift<<<1, 1, 0, s>>>(scal);
  return cudaGetLastError();
}
template cudaError_t launch_pcg_xr<double>(cudaStream_t, int64_t, const double*, double*, double*, const double*,
                                           const double*);
template cudaError_t launch_pcg_xr<float>(cudaStream_t, int64_t, const double*, float*, float*, const float*,
                                          const float*);
template cudaError_t launch_pcg_p<double>(cudaStream_t, int64_t, double*, double*, const double*);
template cudaError_t launch_pcg_p<float>(cudaStream_t, int64_t, double*, float*, const float*);

// ---------------------------------------------------------------- cross-problem batches
// Node-list and vector kernels over job lists: blockIdx.y is the job, blockIdx.x and the
// threads stride over the job's nodes exactly as the single-problem kernels stride over
// theirs, so every entry is computed with the same arithmetic.

template <class T>
__global__ void k_iface_gather_b(const NodeJobT<T>* __restrict__ jobs) {
  const NodeJobT<T> j = jobs[blockIdx.y];
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < j.n; i += int64_t(gridDim.x) * blockDim.x) {
    T s = 0;
    for (int64_t c = j.ptr[i]; c < j.ptr[i + 1]; ++c) s += j.v[j.idx[c]];
    j.G[i] = s;
  }
}

template <class T>
__global__ void k_iface_scatter_b(const NodeJobT<T>* __restrict__ jobs, T tau, int add) {
  const NodeJobT<T> j = jobs[blockIdx.y];
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < j.n; i += int64_t(gridDim.x) * blockDim.x) {
    T val = tau * fma(j.vscale[i], j.G[i], j.Z[i]);
    for (int64_t c = j.ptr[i]; c < j.ptr[i + 1]; ++c) {
      int64_t t = j.idx[c];
      j.u[t] = add ? j.u[t] + val : val;
    }
  }
}

template <class T>
cudaError_t launch_iface_gather_b(cudaStream_t s, const NodeJobT<T>* jobs, int njobs, int64_t max_n) {
  if (njobs <= 0 || max_n <= 0) return cudaSuccess;
  k_iface_gather_b<T><<<dim3(grid_for(max_n, 256), njobs), 256, 0, s>>>(jobs);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_iface_scatter_b(cudaStream_t s, const NodeJobT<T>* jobs, int njobs, int64_t max_n, T tau,
                                   int add) {
  if (njobs <= 0 || max_n <= 0) return cudaSuccess;
  k_iface_scatter_b<T><<<dim3(grid_for(max_n, 256), njobs), 256, 0, s>>>(jobs, tau, add);
  return cudaGetLastError();
}

// One block per job: x_copies = Ainv (sum of copies of v), warp per row as k_coarse_solve.
template <class T>
__global__ void k_coarse_solve_b(const NodeJobT<T>* __restrict__ jobs) {
  extern __shared__ double g[];
  const NodeJobT<T> j = jobs[blockIdx.y];
  const int64_t N0 = j.n;
  for (int64_t i = threadIdx.x; i < N0; i += blockDim.x) {
    double s = 0.0;
    for (int64_t c = j.ptr[i]; c < j.ptr[i + 1]; ++c) s += double(j.v[j.idx[c]]);
    g[i] = s;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int64_t r = int64_t(blockIdx.x) * nw + warp; r < N0; r += int64_t(gridDim.x) * nw) {
    double acc = 0.0;
    for (int64_t c = lane; c < N0; c += 32) acc = fma(j.Ainv[r * N0 + c], g[c], acc);
    acc = warp_sum(acc);
    acc = __shfl_sync(0xffffffffu, acc, 0);
    for (int64_t c = j.ptr[r] + lane; c < j.ptr[r + 1]; c += 32) j.u[j.idx[c]] = T(acc);
  }
}

template <class T>
cudaError_t launch_coarse_solve_b(cudaStream_t s, const NodeJobT<T>* jobs, int njobs, int64_t max_n) {
  if (njobs <= 0 || max_n <= 0) return cudaSuccess;
  int blocks = int((max_n + 7) / 8);
  if (blocks > 16) blocks = 16;
  const size_t sm = sizeof(double) * size_t(max_n);
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(k_coarse_solve_b<T>), sm);
  if (e != cudaSuccess) return e;
  k_coarse_solve_b<T><<<dim3(blocks, njobs), 256, sm, s>>>(jobs);
  return cudaGetLastError();
}

template <class T>
__global__ void k_global_to_tile_b(const NodeJobT<T>* __restrict__ jobs, int first_only) {
  const NodeJobT<T> j = jobs[blockIdx.y];
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < j.n; g += int64_t(gridDim.x) * blockDim.x) {
    T v = j.G[g];
    for (int64_t c = j.ptr[g]; c < j.ptr[g + 1]; ++c) j.u[j.idx[c]] = (first_only && c > j.ptr[g]) ? T(0) : v;
  }
}

template <class T>
__global__ void k_tile_to_global_b(const NodeJobT<T>* __restrict__ jobs, int sum_copies) {
  const NodeJobT<T> j = jobs[blockIdx.y];
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < j.n; g += int64_t(gridDim.x) * blockDim.x) {
    T v = j.v[j.idx[j.ptr[g]]];
    if (sum_copies)
      for (int64_t c = j.ptr[g] + 1; c < j.ptr[g + 1]; ++c) v += j.v[j.idx[c]];
    j.G[g] = v;
  }
}

template <class T>
cudaError_t launch_global_to_tile_b(cudaStream_t s, const NodeJobT<T>* jobs, int njobs, int64_t max_n, int first_only) {
  if (njobs <= 0 || max_n <= 0) return cudaSuccess;
  k_global_to_tile_b<T><<<dim3(grid_for(max_n, 256), njobs), 256, 0, s>>>(jobs, first_only);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_tile_to_global_b(cudaStream_t s, const NodeJobT<T>* jobs, int njobs, int64_t max_n, int sum_copies) {
  if (njobs <= 0 || max_n <= 0) return cudaSuccess;
  k_tile_to_global_b<T><<<dim3(grid_for(max_n, 256), njobs), 256, 0, s>>>(jobs, sum_copies);
  return cudaGetLastError();
}

// Reductions: the single-problem grid of RED_BLOCKS blocks per job (blockIdx.x), partials in
// partials[j * RED_BLOCKS + b], then one block per job in the same order as k_reduce_final.
template <class T>
__global__ void __launch_bounds__(256) k_dot_partial_b(const VecJobT<T>* __restrict__ jobs, double* __restrict__ partials) {
  __shared__ double sh[256];
  const VecJobT<T> j = jobs[blockIdx.y];
  double s = 0.0;
  for (int64_t i = blockIdx.x * int64_t(256) + threadIdx.x; i < j.n; i += int64_t(gridDim.x) * 256)
    s = fma(double(j.a[i]), double(j.b[i]), s);
  s = block_sum_256(s, sh);
  if (threadIdx.x == 0) partials[int64_t(blockIdx.y) * RED_BLOCKS + blockIdx.x] = s;
}

template <class T>
__global__ void __launch_bounds__(256) k_norm2_dist_partial_b(const VecJobT<T>* __restrict__ jobs,
                                                              double* __restrict__ partials) {
  __shared__ double sh[256];
  const VecJobT<T> j = jobs[blockIdx.y];
  double s = 0.0;
  for (int64_t g = blockIdx.x * int64_t(256) + threadIdx.x; g < j.n; g += int64_t(gridDim.x) * 256) {
    double c = 0.0;
    for (int64_t k = j.ptr[g]; k < j.ptr[g + 1]; ++k) c += double(j.a[j.idx[k]]);
    s = fma(c, c, s);
  }
  s = block_sum_256(s, sh);
  if (threadIdx.x == 0) partials[int64_t(blockIdx.y) * RED_BLOCKS + blockIdx.x] = s;
}

template <class T>
__global__ void __launch_bounds__(256) k_reduce_final_b(const VecJobT<T>* __restrict__ jobs,
                                                        const double* __restrict__ partials, int out) {
  __shared__ double sh[256];
  const double* pj = partials + int64_t(blockIdx.x) * RED_BLOCKS;
  double s = 0.0;
  for (int i = threadIdx.x; i < RED_BLOCKS; i += 256) s += pj[i];
  s = block_sum_256(s, sh);
  if (threadIdx.x == 0) jobs[blockIdx.x].scal[out] = s;
}

template <class T>
cudaError_t launch_dot_b(cudaStream_t s, const VecJobT<T>* jobs, int njobs, int out, double* partials) {
  if (njobs <= 0) return cudaSuccess;
  k_dot_partial_b<T><<<dim3(RED_BLOCKS, njobs), 256, 0, s>>>(jobs, partials);
  k_reduce_final_b<T><<<njobs, 256, 0, s>>>(jobs, partials, out);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_norm2_dist_b(cudaStream_t s, const VecJobT<T>* jobs, int njobs, int out, double* partials) {
  if (njobs <= 0) return cudaSuccess;
  k_norm2_dist_partial_b<T><<<dim3(RED_BLOCKS, njobs), 256, 0, s>>>(jobs, partials);
  k_reduce_final_b<T><<<njobs, 256, 0, s>>>(jobs, partials, out);
  return cudaGetLastError();
}

template <class T>
__global__ void k_pcg_xr_b(const VecJobT<T>* __restrict__ jobs, const int* __restrict__ active) {
  if (!active[blockIdx.y]) return;
  const VecJobT<T> j = jobs[blockIdx.y];
  __shared__ T alpha_s;
  if (threadIdx.x == 0) alpha_s = T(j.scal[0] / j.scal[1]);
  __syncthreads();
  const T alpha = alpha_s;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < j.n; i += int64_t(gridDim.x) * blockDim.x) {
    j.a[i] = fma(alpha, j.c[i], j.a[i]);
    j.b[i] = fma(-alpha, j.d[i], j.b[i]);
  }
}

template <class T>
__global__ void k_pcg_p_b(const VecJobT<T>* __restrict__ jobs, const int* __restrict__ active) {
  if (!active[blockIdx.y]) return;
  const VecJobT<T> j = jobs[blockIdx.y];
  __shared__ T beta_s;
  if (threadIdx.x == 0) beta_s = T(j.scal[2] / j.scal[0]);
  __syncthreads();
  const T beta = beta_s;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < j.n; i += int64_t(gridDim.x) * blockDim.x)
    j.a[i] = fma(beta, j.a[i], j.c[i]);
}

template <class T>
__global__ void k_scalar_shift_b(const VecJobT<T>* __restrict__ jobs, const int* __restrict__ active, int njobs) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < njobs && active[q]) jobs[q].scal[0] = jobs[q].scal[2];
}

template <class T>
cudaError_t launch_pcg_xr_b(cudaStream_t s, const VecJobT<T>* jobs, int njobs, int64_t max_n, const int* active) {
  if (njobs <= 0 || max_n <= 0) return cudaSuccess;
  k_pcg_xr_b<T><<<dim3(grid_for(max_n, 256), njobs), 256, 0, s>>>(jobs, active);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_pcg_p_b(cudaStream_t s, const VecJobT<T>* jobs, int njobs, int64_t max_n, const int* active) {
  if (njobs <= 0 || max_n <= 0) return cudaSuccess;
  k_pcg_p_b<T><<<dim3(grid_for(max_n, 256), njobs), 256, 0, s>>>(jobs, active);
  k_scalar_shift_b<T><<<(njobs + 255) / 256, 256, 0, s>>>(jobs, active, njobs);
  return cudaGetLastError();
}

// mode 0: a = b; mode 1: a = 0; mode 2: a = 1 * b + 1 * a (the axpby of the solve's end)
template <class T>
__global__ void k_copy_b(const VecJobT<T>* __restrict__ jobs, int mode) {
  const VecJobT<T> j = jobs[blockIdx.y];
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < j.n; i += int64_t(gridDim.x) * blockDim.x) {
    if (mode == 0) j.a[i] = j.b[i];
    else if (mode == 1) j.a[i] = T(0);
    else j.a[i] = 1.0 * j.b[i] + 1.0 * j.a[i];
  }
}

template <class T>
cudaError_t launch_copy_b(cudaStream_t s, const VecJobT<T>* jobs, int njobs, int64_t max_n, int mode) {
  if (njobs <= 0 || max_n <= 0) return cudaSuccess;
  k_copy_b<T><<<dim3(grid_for(max_n, 256), njobs), 256, 0, s>>>(jobs, mode);
  return cudaGetLastError();
}

template cudaError_t launch_iface_gather_b<double>(cudaStream_t, const NodeJobT<double>*, int, int64_t);
template cudaError_t launch_iface_scatter_b<double>(cudaStream_t, const NodeJobT<double>*, int, int64_t, double, int);
template cudaError_t launch_coarse_solve_b<double>(cudaStream_t, const NodeJobT<double>*, int, int64_t);
template cudaError_t launch_global_to_tile_b<double>(cudaStream_t, const NodeJobT<double>*, int, int64_t, int);
template cudaError_t launch_tile_to_global_b<double>(cudaStream_t, const NodeJobT<double>*, int, int64_t, int);
template cudaError_t launch_dot_b<double>(cudaStream_t, const VecJobT<double>*, int, int, double*);
template cudaError_t launch_norm2_dist_b<double>(cudaStream_t, const VecJobT<double>*, int, int, double*);
template cudaError_t launch_pcg_xr_b<double>(cudaStream_t, const VecJobT<double>*, int, int64_t, const int*);
template cudaError_t launch_pcg_p_b<double>(cudaStream_t, const VecJobT<double>*, int, int64_t, const int*);
template cudaError_t launch_copy_b<double>(cudaStream_t, const VecJobT<double>*, int, int64_t, int);

// Flexible CG (Polak-Ribiere): beta = (rz_new - (r_new, z_old)) / rz_old; scal[5] = beta,
// scal[0] = rz_new.
__global__ void k_fcg_beta(double* scal) {
  scal[5] = (scal[2] - scal[4]) / scal[0];
  scal[0] = scal[2];
}

template <class T>
__global__ void k_p_update(int64_t n, const double* __restrict__ beta_p, T* __restrict__ p, const T* __restrict__ z,
                           T* __restrict__ zold) {
  const T beta = T(*beta_p);
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    T zi = z[i];
    p[i] = fma(beta, p[i], zi);
    zold[i] = zi;
  }
}

cudaError_t launch_fcg_p(cudaStream_t s, int64_t n, double* scal, float* p, const float* z, float* zold) {
  k_fcg_beta<<<1, 1, 0, s>>>(scal);
  k_p_update<float><<<grid_for(n, 256), 256, 0, s>>>(n, scal + 5, p, z, zold);
  return cudaGetLastError();
}

__global__ void k_axpby(int64_t n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

cudaError_t launch_axpby(cudaStream_t s, int64_t n, double a, const double* x, double b, double* y) {
  k_axpby<<<grid_for(n, 256), 256, 0, s>>>(n, a, x, b, y);
  return cudaGetLastError();
}

// Precision conversions of whole vectors: dst = scale * src.
template <class TD, class TS>
__global__ void k_convert(int64_t n, const TS* __restrict__ src, double scale, TD* __restrict__ dst) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    dst[i] = TD(double(src[i]) * scale);
}
// x64 += scale * d32 (iterative refinement update)
__global__ void k_add_scaled_f32(int64_t n, const float* __restrict__ d, double scale, double* __restrict__ x) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i] = fma(scale, double(d[i]), x[i]);
}

cudaError_t launch_convert_f64_f32(cudaStream_t s, int64_t n, const double* src, double scale, float* dst) {
  k_convert<float, double><<<grid_for(n, 256), 256, 0, s>>>(n, src, scale, dst);
  return cudaGetLastError();
}
cudaError_t launch_convert_f64_bf16(cudaStream_t s, int64_t n, const double* src, __nv_bfloat16* dst) {
  k_convert<__nv_bfloat16, double><<<grid_for(n, 256), 256, 0, s>>>(n, src, 1.0, dst);
  return cudaGetLastError();
}
cudaError_t launch_add_scaled_f32(cudaStream_t s, int64_t n, const float* d, double scale, double* x) {
  k_add_scaled_f32<<<grid_for(n, 256), 256, 0, s>>>(n, d, scale, x);
  return cudaGetLastError();
}

}  // namespace igamg

// ================================================================ dimension-generic kernels

namespace igamg {

// ---------------------------------------------------------------- element assembly

// Element matrices of the patch form a_k (Eq. model:bil) by sum factorisation over the
// Gauss points of one element, added into the band storage.  Elements of one colour
// (e_j mod (p+1) fixed in every direction) share no row, so a colour is assembled without
// atomics and the summation order is fixed.  One block (128 threads) per element.
// Geometry factors are evaluated on the fly from the multilinear map.
template <int D>
__global__ void __launch_bounds__(128) k_assemble_elem(ElemAsm ea) {
  constexpr int NC = 1 << D;
  extern __shared__ double sm[];
  const int P = ea.p + 1, Q = ea.p + 1;
  int PD = 1, QD = 1;
  for (int j = 0; j < D; ++j) { PD *= P; QD *= Q; }
  // element index of this block within the colour
  int e[3] = {0, 0, 0};
  {
    int64_t r = blockIdx.x;
    for (int j = D - 1; j >= 0; --j) {
      int cnt = (ea.m[j] - ea.color[j] + P - 1) / P;
      e[j] = ea.color[j] + P * int(r % cnt);
      r /= cnt;
    }
  }
  // shared layout
  double* Fv = sm;                      // [D][Q][P]
  double* Fd = Fv + D * Q * P;          // [D][Q][P]
  double* Cq = Fd + D * Q * P;          // [D*D or 1][QD]
  const int nterm = ea.mass ? 1 : D * D;
  double* A = Cq + nterm * QD;          // [PD][PD]
  double* S1 = A + PD * PD;             // [Q][P^2]^(D-1) ... sized by host
  double* S2 = S1 + Q * (D == 3 ? P * P * P * P : P * P);
  const int tid = threadIdx.x;
  for (int i = tid; i < D * Q * P; i += blockDim.x) {
    int j = i / (Q * P), qa = i % (Q * P);
    const double* Bt = ea.B[j] + int64_t(e[j]) * Q * P;
    const double* dBt = ea.dB[j] + int64_t(e[j]) * Q * P;
    Fv[i] = Bt[qa];
    Fd[i] = dBt[qa];
  }
  for (int i = tid; i < PD * PD; i += blockDim.x) A[i] = 0.0;
  // geometry factors at the element's Gauss points
  for (int q = tid; q < QD; q += blockDim.x) {
    int qi[3] = {0, 0, 0};
    int r = q;
    for (int j = D - 1; j >= 0; --j) { qi[j] = r % Q; r /= Q; }
    double xi[3], w = 1.0;
    for (int j = 0; j < D; ++j) {
      xi[j] = ea.xq[j][e[j] * Q + qi[j]];
      w *= ea.wq[j][e[j] * Q + qi[j]];
    }
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int c = 0; c < NC; ++c)
      for (int j = 0; j < D; ++j) {
        double f = ((c >> j) & 1) ? 1.0 : -1.0;
        for (int i = 0; i < D; ++i)
          if (i != j) f *= ((c >> i) & 1) ? xi[i] : 1.0 - xi[i];
        for (int a = 0; a < D; ++a) J[a][j] += f * ea.corners[c * D + a];
      }
    double det, Ji[3][3];
    if (D == 2) {
      det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      Ji[0][0] = J[1][1] / det; Ji[0][1] = -J[0][1] / det;
      Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
    } else {
      double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
      double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
      double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
      det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
      Ji[0][0] = c00 / det;
      Ji[1][0] = c01 / det;
      Ji[2][0] = c02 / det;
      Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
      Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
      Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
      Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
      Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
      Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    }
    double ad = fabs(det);
    if (ea.mass) {
      Cq[q] = w * ad;
    } else {
      for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) {
          double s = 0.0;
          for (int i = 0; i < D; ++i) s += Ji[a][i] * Ji[b][i];  // (J^{-1} J^{-T})_ab
          Cq[(a * D + b) * QD + q] = w * ad * s;
        }
    }
  }
  __syncthreads();
  // sum factorisation, term by term: F_j[q][a][b] = X_j(a, q) Y_j(b, q) with X/Y the value
  // or the derivative table depending on whether j is the derivative direction of the
  // test / trial function.
  for (int term = 0; term < nterm; ++term) {
    const int al = ea.mass ? -1 : term / D, be = ea.mass ? -1 : term % D;
    const double* C = Cq + term * QD;
    const double* X[3];
    const double* Y[3];
    for (int j = 0; j < D; ++j) {
      X[j] = (j == al ? Fd : Fv) + j * Q * P;
      Y[j] = (j == be ? Fd : Fv) + j * Q * P;
    }
    const int P2 = P * P;
    if (D == 2) {
      // S1[q0][a1 b1] = sum_q1 C[q0 q1] X1[q1 a1] Y1[q1 b1]
      for (int i = tid; i < Q * P2; i += blockDim.x) {
        int q0 = i / P2, ab = i % P2, a1 = ab / P, b1 = ab % P;
        double s = 0.0;
        for (int q1 = 0; q1 < Q; ++q1) s += C[q0 * Q + q1] * X[1][q1 * P + a1] * Y[1][q1 * P + b1];
        S1[i] = s;
      }
      __syncthreads();
      // A[(a0 a1),(b0 b1)] += sum_q0 S1[q0][a1 b1] X0[q0 a0] Y0[q0 b0]
      for (int i = tid; i < PD * PD; i += blockDim.x) {
        int row = i / PD, col = i % PD;
        int a0 = row / P, a1 = row % P, b0 = col / P, b1 = col % P;
        double s = 0.0;
        for (int q0 = 0; q0 < Q; ++q0) s += S1[q0 * P2 + a1 * P + b1] * X[0][q0 * P + a0] * Y[0][q0 * P + b0];
        A[i] += s;
      }
      __syncthreads();
    } else {
      const int P4 = P2 * P2;
      // S2[q0 q1][a2 b2] = sum_q2 C[q0 q1 q2] X2[q2 a2] Y2[q2 b2]
      for (int i = tid; i < Q * Q * P2; i += blockDim.x) {
        int qq = i / P2, ab = i % P2, a2 = ab / P, b2 = ab % P;
        double s = 0.0;
        for (int q2 = 0; q2 < Q; ++q2) s += C[qq * Q + q2] * X[2][q2 * P + a2] * Y[2][q2 * P + b2];
        S2[i] = s;
      }
      __syncthreads();
      // S1[q0][a1 b1 a2 b2] = sum_q1 S2[q0 q1][a2 b2] X1[q1 a1] Y1[q1 b1]
      for (int i = tid; i < Q * P4; i += blockDim.x) {
        int q0 = i / P4, rem = i % P4, ab1 = rem / P2, ab2 = rem % P2, a1 = ab1 / P, b1 = ab1 % P;
        double s = 0.0;
        for (int q1 = 0; q1 < Q; ++q1) s += S2[(q0 * Q + q1) * P2 + ab2] * X[1][q1 * P + a1] * Y[1][q1 * P + b1];
        S1[i] = s;
      }
      __syncthreads();
      for (int i = tid; i < PD * PD; i += blockDim.x) {
        int row = i / PD, col = i % PD;
        int a0 = row / P2, a1 = (row / P) % P, a2 = row % P;
        int b0 = col / P2, b1 = (col / P) % P, b2 = col % P;
        int rem = ((a1 * P + b1) * P + a2) * P + b2;
        double s = 0.0;
        for (int q0 = 0; q0 < Q; ++q0) s += S1[q0 * P4 + rem] * X[0][q0 * P + a0] * Y[0][q0 * P + b0];
        A[i] += s;
      }
      __syncthreads();
    }
  }
  // add the element matrix into the band rows (Dirichlet rows stay zero)
  const int W = 2 * ea.p + 1;
  for (int i = tid; i < PD * PD; i += blockDim.x) {
    int row = i / PD, col = i % PD;
    int a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
    int r = row, c = col;
    for (int j = D - 1; j >= 0; --j) { a[j] = r % P; r /= P; b[j] = c % P; c /= P; }
    int64_t node = 0;
    int t = 0;
    for (int j = 0; j < D; ++j) {
      node = node * ea.n[j] + (e[j] + a[j]);
      t = t * W + (b[j] - a[j] + ea.p);
    }
    if (ea.l2g[ea.off + node] < 0) continue;
    ea.band[ea.band_off + int64_t(t) * ea.nn + node] += A[i];
  }
}

size_t elem_asm_smem(int D, int p, bool mass) {
  int P = p + 1, PD = 1, QD = 1;
  for (int j = 0; j < D; ++j) { PD *= P; QD *= P; }
  size_t n = 2 * D * P * P + (mass ? 1 : D * D) * QD + PD * PD;
  n += (D == 3) ? (P * P * P * P * P + P * P * P * P) : P * P * P;
  return n * sizeof(double);
}

cudaError_t launch_assemble_elem(cudaStream_t s, const ElemAsm& base) {
  const int D = base.dim, P = base.p + 1;
  size_t smem = elem_asm_smem(D, base.p, base.mass);
  cudaError_t e;
  if (D == 2) e = ensure_smem(reinterpret_cast<const void*>(k_assemble_elem<2>), smem);
  else e = ensure_smem(reinterpret_cast<const void*>(k_assemble_elem<3>), smem);
  if (e != cudaSuccess) return e;
  int ncol = 1;
  for (int j = 0; j < D; ++j) ncol *= P;
  for (int col = 0; col < ncol; ++col) {
    ElemAsm ea = base;
    int r = col;
    int64_t cnt = 1;
    for (int j = D - 1; j >= 0; --j) {
      ea.color[j] = r % P;
      r /= P;
      int c = (ea.m[j] - ea.color[j] + P - 1) / P;
      cnt *= c > 0 ? c : 0;
    }
    if (cnt == 0) continue;
    if (D == 2) k_assemble_elem<2><<<unsigned(cnt), 128, smem, s>>>(ea);
    else k_assemble_elem<3><<<unsigned(cnt), 128, smem, s>>>(ea);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------- 3D stiffness apply

namespace {
constexpr int BX3 = 32, BY3 = 4, BZ3 = 2;
}

// P > 0: every patch of the launch has degree P in all directions (the tap loops are
// unrolled, so a thread has a plane of (2P+1)^2 band loads in flight; one FMA chain, which
// measured faster than per-row partial sums here); P = 0: any degrees.
template <class TV, class TB, int P>
__global__ void __launch_bounds__(BX3 * BY3 * BZ3) k_band_apply_3d(const PatchDev* __restrict__ pds,
                                                                   const TB* __restrict__ band,
                                                                   const TV* __restrict__ u,
                                                                   const TV* __restrict__ f,
                                                                   TV* __restrict__ y, int tiles1) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TV* su = reinterpret_cast<TV*>(smraw);
  const PatchDev pd = pds[blockIdx.z];
  const int n0 = pd.n[0], n1 = pd.n[1], n2 = pd.n[2];
  const int p0 = P ? P : pd.p[0], p1 = P ? P : pd.p[1], p2 = P ? P : pd.p[2];
  const int i0b = (blockIdx.y / tiles1) * BZ3, i1b = (blockIdx.y % tiles1) * BY3, i2b = blockIdx.x * BX3;
  if (i0b >= n0 || i1b >= n1 || i2b >= n2) return;
  const int H0 = BZ3 + 2 * p0, H1 = BY3 + 2 * p1, H2 = BX3 + 2 * p2;
  const TV* ut = u + pd.off;
  const int tid = (threadIdx.z * BY3 + threadIdx.y) * BX3 + threadIdx.x;
  for (int idx = tid; idx < H0 * H1 * H2; idx += BX3 * BY3 * BZ3) {
    int a = idx / (H1 * H2), rem = idx % (H1 * H2), b = rem / H2, c = rem % H2;
    int g0 = i0b - p0 + a, g1 = i1b - p1 + b, g2 = i2b - p2 + c;
    su[idx] = (g0 >= 0 && g0 < n0 && g1 >= 0 && g1 < n1 && g2 >= 0 && g2 < n2)
                  ? ut[(int64_t(g0) * n1 + g1) * n2 + g2] : TV(0);
  }
  __syncthreads();
  const int i0 = i0b + threadIdx.z, i1 = i1b + threadIdx.y, i2 = i2b + threadIdx.x;
  if (i0 >= n0 || i1 >= n1 || i2 >= n2) return;
  const int64_t nn = int64_t(n0) * n1 * n2, node = (int64_t(i0) * n1 + i1) * n2 + i2;
  const TB* bp = band + pd.band_off + node;
  TV acc = 0;
  if constexpr (P > 0) {
    constexpr int W = 2 * P + 1;
#pragma unroll 1
    for (int t0 = 0; t0 < W; ++t0) {
      const TB* bq = bp + int64_t(t0 * W * W) * nn;
#pragma unroll
      for (int t1 = 0; t1 < W; ++t1) {
        const TV* srow = su + ((threadIdx.z + t0) * H1 + threadIdx.y + t1) * H2 + threadIdx.x;
#pragma unroll
        for (int t2 = 0; t2 < W; ++t2) acc = fma(band_val<TV, TB>(bq + int64_t(t1 * W + t2) * nn), srow[t2], acc);
      }
    }
  } else {
    const int w1 = 2 * p1 + 1, w2 = 2 * p2 + 1;
    int t = 0;
    for (int t0 = 0; t0 <= 2 * p0; ++t0)
      for (int t1 = 0; t1 < w1; ++t1) {
        const TV* srow = su + ((threadIdx.z + t0) * H1 + threadIdx.y + t1) * H2 + threadIdx.x;
        for (int t2 = 0; t2 < w2; ++t2, ++t) acc = fma(band_val<TV, TB>(bp + int64_t(t) * nn), srow[t2], acc);
      }
  }
  y[pd.off + node] = f ? f[pd.off + node] - acc : acc;
}

// ---------------------------------------------------------------- tap-blocked FP32 3D apply

__global__ void k_band_blk_f32(const PatchDev* __restrict__ spd, const PatchDev* __restrict__ dpd, int taps,
                               const double* __restrict__ src, float* __restrict__ dst) {
  const PatchDev a = spd[blockIdx.z], b = dpd[blockIdx.z];
  const int t = blockIdx.y;
  if (t >= taps) return;
  const int64_t nn = int64_t(a.n[0]) * a.n[1] * a.n[2], nr = (nn + 31) / 32 * 32;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < nr; i += int64_t(gridDim.x) * blockDim.x)
    dst[b.band_off + ((i >> 5) * taps + t) * 32 + (i & 31)] = i < nn ? float(double(src[a.band_off + t * nn + i]) * 1.0)
                                                                     : 0.0f;
}

cudaError_t launch_band_blk_f32(cudaStream_t s, const PatchDev* src_pd, const PatchDev* dst_pd, int K, int taps,
                                int64_t max_nodes, const double* src, float* dst) {
  if (K <= 0 || taps <= 0 || max_nodes <= 0) return cudaSuccess;
  const int64_t g = std::min<int64_t>((max_nodes + 31 + 255) / 256, 1024);
  k_band_blk_f32<<<dim3(unsigned(g), unsigned(taps), unsigned(K)), 256, 0, s>>>(src_pd, dst_pd, taps, src, dst);
  return cudaGetLastError();
}

template <int P>
__global__ void __launch_bounds__(BX3 * BY3 * BZ3) k_band_apply_3d_blk(const PatchDev* __restrict__ pds,
                                                                       const float* __restrict__ band,
                                                                       const float* __restrict__ u,
                                                                       const float* __restrict__ f,
                                                                       float* __restrict__ y, int tiles1) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float* su = reinterpret_cast<float*>(smraw);
  constexpr int W = 2 * P + 1, TAPS = W * W * W;
  const PatchDev pd = pds[blockIdx.z];
  const int n0 = pd.n[0], n1 = pd.n[1], n2 = pd.n[2];
  const int i0b = (blockIdx.y / tiles1) * BZ3, i1b = (blockIdx.y % tiles1) * BY3, i2b = blockIdx.x * BX3;
  if (i0b >= n0 || i1b >= n1 || i2b >= n2) return;
  constexpr int H0 = BZ3 + 2 * P, H1 = BY3 + 2 * P, H2 = BX3 + 2 * P;
  const float* ut = u + pd.off;
  const int tid = (threadIdx.z * BY3 + threadIdx.y) * BX3 + threadIdx.x;
  for (int idx = tid; idx < H0 * H1 * H2; idx += BX3 * BY3 * BZ3) {
    const int a = idx / (H1 * H2), rem = idx % (H1 * H2), b = rem / H2, c = rem % H2;
    const int g0 = i0b - P + a, g1 = i1b - P + b, g2 = i2b - P + c;
    su[idx] = (g0 >= 0 && g0 < n0 && g1 >= 0 && g1 < n1 && g2 >= 0 && g2 < n2) ? ut[(int64_t(g0) * n1 + g1) * n2 + g2]
                                                                                : 0.0f;
  }
  __syncthreads();
  const int i0 = i0b + threadIdx.z, i1 = i1b + threadIdx.y, i2 = i2b + threadIdx.x;
  if (i0 >= n0 || i1 >= n1 || i2 >= n2) return;
  const int64_t node = (int64_t(i0) * n1 + i1) * n2 + i2;
  const float* bp = band + pd.band_off + (node >> 5) * (int64_t(TAPS) * 32) + (node & 31);
  float acc = 0.f;
#pragma unroll 1
  for (int t0 = 0; t0 < W; ++t0) {
#pragma unroll
    for (int t1 = 0; t1 < W; ++t1) {
      const float* srow = su + ((threadIdx.z + t0) * H1 + threadIdx.y + t1) * H2 + threadIdx.x;
      const float* bq = bp + (t0 * W + t1) * W * 32;
#pragma unroll
      for (int t2 = 0; t2 < W; ++t2) acc = fma(__ldg(bq + t2 * 32), srow[t2], acc);
    }
  }
  y[pd.off + node] = f ? f[pd.off + node] - acc : acc;
}

cudaError_t launch_band_apply_3d_blk(cudaStream_t s, const PatchDev* pd_dev, int K, const int* max_n, int p,
                                     const float* band, const float* u, const float* f, float* y) {
  const int t1 = (max_n[1] + BY3 - 1) / BY3, t0 = (max_n[0] + BZ3 - 1) / BZ3;
  const dim3 grid((max_n[2] + BX3 - 1) / BX3, t0 * t1, K), block(BX3, BY3, BZ3);
  const size_t sm = sizeof(float) * (BZ3 + 2 * p) * (BY3 + 2 * p) * (BX3 + 2 * p);
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = ensure_smem(reinterpret_cast<const void*>(kern), sm);
    if (e != cudaSuccess) return e;
    kern<<<grid, block, sm, s>>>(pd_dev, band, u, f, y, t1);
    return cudaGetLastError();
  };
  switch (p) {
    case 2: return go(k_band_apply_3d_blk<2>);
    case 3: return go(k_band_apply_3d_blk<3>);
    case 4: return go(k_band_apply_3d_blk<4>);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------- paired BF16 3D apply

template <class TB>
__global__ void k_band_pair(const PatchDev* __restrict__ spd, const PatchDev* __restrict__ dpd, int taps,
                            const double* __restrict__ src, TB* __restrict__ dst) {
  const PatchDev a = spd[blockIdx.z], b = dpd[blockIdx.z];
  const int n2 = a.n[2], n2e = band_row_even(n2), t = blockIdx.y;
  if (t >= taps) return;
  const int64_t nn = int64_t(a.n[0]) * a.n[1] * n2, ne = int64_t(a.n[0]) * a.n[1] * n2e;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < ne; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t row = i / n2e;
    const int i2 = int(i - row * n2e);
    dst[b.band_off + t * ne + i] = i2 < n2 ? TB(double(src[a.band_off + t * nn + row * n2 + i2]) * 1.0) : TB(0.0f);
  }
}

template <class TB>
cudaError_t launch_band_pair(cudaStream_t s, const PatchDev* src_pd, const PatchDev* dst_pd, int K, int taps,
                             int64_t max_nodes, const double* src, TB* dst) {
  if (K <= 0 || taps <= 0 || max_nodes <= 0) return cudaSuccess;
  const int64_t g = std::min<int64_t>((max_nodes + 255) / 256, 1024);
  k_band_pair<TB><<<dim3(unsigned(g), unsigned(taps), unsigned(K)), 256, 0, s>>>(src_pd, dst_pd, taps, src, dst);
  return cudaGetLastError();
}
template cudaError_t launch_band_pair<__nv_bfloat16>(cudaStream_t, const PatchDev*, const PatchDev*, int, int, int64_t,
                                                     const double*, __nv_bfloat16*);
template cudaError_t launch_band_pair<float>(cudaStream_t, const PatchDev*, const PatchDev*, int, int, int64_t,
                                             const double*, float*);

__device__ __forceinline__ float2 pair_val(const __nv_bfloat16* p) {
  return __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(p)));
}
__device__ __forceinline__ float2 pair_val(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }

// Block: 32 x 4 x 2 threads, 64 x 4 x 2 nodes (two adjacent nodes of a row per thread); the
// u halo in shared memory as in k_band_apply_3d.  (16 x 8 x 2 threads spanning 32 nodes of
// a row measured slower on the 67-node rows of the 3D benchmark.)
constexpr int PBX = 32, PBY = 4, PBZ = 2;
template <class TB, int P>
__global__ void __launch_bounds__(PBX * PBY * PBZ) k_band_apply_3d_pair(const PatchDev* __restrict__ pds,
                                                                        const TB* __restrict__ band,
                                                                        const float* __restrict__ u,
                                                                        const float* __restrict__ f,
                                                                        float* __restrict__ y, int tiles1) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float* su = reinterpret_cast<float*>(smraw);
  constexpr int W = 2 * P + 1, BXN = 2 * PBX;
  const PatchDev pd = pds[blockIdx.z];
  const int n0 = pd.n[0], n1 = pd.n[1], n2 = pd.n[2], n2e = band_row_even(n2);
  const int i0b = (blockIdx.y / tiles1) * PBZ, i1b = (blockIdx.y % tiles1) * PBY, i2b = blockIdx.x * BXN;
  if (i0b >= n0 || i1b >= n1 || i2b >= n2) return;
  constexpr int H0 = PBZ + 2 * P, H1 = PBY + 2 * P, H2 = BXN + 2 * P;
  const float* ut = u + pd.off;
  const int tid = (threadIdx.z * PBY + threadIdx.y) * PBX + threadIdx.x;
  for (int idx = tid; idx < H0 * H1 * H2; idx += PBX * PBY * PBZ) {
    const int a = idx / (H1 * H2), rem = idx % (H1 * H2), b = rem / H2, c = rem % H2;
    const int g0 = i0b - P + a, g1 = i1b - P + b, g2 = i2b - P + c;
    su[idx] = (g0 >= 0 && g0 < n0 && g1 >= 0 && g1 < n1 && g2 >= 0 && g2 < n2) ? ut[(int64_t(g0) * n1 + g1) * n2 + g2]
                                                                                : 0.0f;
  }
  __syncthreads();
  const int i0 = i0b + threadIdx.z, i1 = i1b + threadIdx.y, i2 = i2b + 2 * threadIdx.x;
  if (i0 >= n0 || i1 >= n1 || i2 >= n2) return;
  const int64_t ne = int64_t(n0) * n1 * n2e, nodep = (int64_t(i0) * n1 + i1) * n2e + i2;
  const TB* bp = band + pd.band_off + nodep;  // node pair: 2 x sizeof(TB) aligned (nodep, ne even)
  float acc0 = 0.f, acc1 = 0.f;
#pragma unroll 1
  for (int t0 = 0; t0 < W; ++t0) {
#pragma unroll
    for (int t1 = 0; t1 < W; ++t1) {
      const float* srow = su + ((threadIdx.z + t0) * H1 + threadIdx.y + t1) * H2 + 2 * threadIdx.x;
      const TB* bq = bp + int64_t((t0 * W + t1) * W) * ne;
#pragma unroll
      for (int t2 = 0; t2 < W; ++t2) {
        const float2 w = pair_val(bq + int64_t(t2) * ne);
        acc0 = fma(w.x, srow[t2], acc0);
        acc1 = fma(w.y, srow[t2 + 1], acc1);
      }
    }
  }
  const int64_t node = pd.off + (int64_t(i0) * n1 + i1) * n2 + i2;
  y[node] = f ? f[node] - acc0 : acc0;
  if (i2 + 1 < n2) y[node + 1] = f ? f[node + 1] - acc1 : acc1;
}

template <class TB>
cudaError_t launch_band_apply_3d_pair(cudaStream_t s, const PatchDev* pd_dev, int K, const int* max_n, int p,
                                      const TB* band, const float* u, const float* f, float* y) {
  const int t1 = (max_n[1] + PBY - 1) / PBY, t0 = (max_n[0] + PBZ - 1) / PBZ;
  const dim3 grid((max_n[2] + 2 * PBX - 1) / (2 * PBX), t0 * t1, K), block(PBX, PBY, PBZ);
  const size_t sm = sizeof(float) * (PBZ + 2 * p) * (PBY + 2 * p) * (2 * PBX + 2 * p);
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = ensure_smem(reinterpret_cast<const void*>(kern), sm);
    if (e != cudaSuccess) return e;
    kern<<<grid, block, sm, s>>>(pd_dev, band, u, f, y, t1);
    return cudaGetLastError();
  };
  switch (p) {
    case 2: return go(k_band_apply_3d_pair<TB, 2>);
    case 3: return go(k_band_apply_3d_pair<TB, 3>);
    case 4: return go(k_band_apply_3d_pair<TB, 4>);
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t launch_band_apply_3d_pair<__nv_bfloat16>(cudaStream_t, const PatchDev*, int, const int*, int,
                                                              const __nv_bfloat16*, const float*, const float*, float*);
template cudaError_t launch_band_apply_3d_pair<float>(cudaStream_t, const PatchDev*, int, const int*, int, const float*,
                                                      const float*, const float*, float*);

template <class TV, class TB, int P>
static cudaError_t launch_apply_3d_p(cudaStream_t s, dim3 grid, size_t sm, const PatchDev* pd_dev, const TB* band,
                                     const TV* u, const TV* f, TV* y, int t1) {
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(k_band_apply_3d<TV, TB, P>), sm);
  if (e != cudaSuccess) return e;
  k_band_apply_3d<TV, TB, P><<<grid, dim3(BX3, BY3, BZ3), sm, s>>>(pd_dev, band, u, f, y, t1);
  return cudaGetLastError();
}

template <class TV, class TB>
cudaError_t launch_band_apply_3d(cudaStream_t s, const PatchDev* pd_dev, int K, const int* max_n, int max_p,
                                 const TB* band, const TV* u, const TV* f, TV* y, int uniform_p) {
  int t1 = (max_n[1] + BY3 - 1) / BY3, t0 = (max_n[0] + BZ3 - 1) / BZ3;
  dim3 grid((max_n[2] + BX3 - 1) / BX3, t0 * t1, K);
  size_t sm = sizeof(TV) * (BZ3 + 2 * max_p) * (BY3 + 2 * max_p) * (BX3 + 2 * max_p);
  switch (uniform_p) {
    case 2: return launch_apply_3d_p<TV, TB, 2>(s, grid, sm, pd_dev, band, u, f, y, t1);
    case 3: return launch_apply_3d_p<TV, TB, 3>(s, grid, sm, pd_dev, band, u, f, y, t1);
    case 4: return launch_apply_3d_p<TV, TB, 4>(s, grid, sm, pd_dev, band, u, f, y, t1);
    default: return launch_apply_3d_p<TV, TB, 0>(s, grid, sm, pd_dev, band, u, f, y, t1);
  }
}template cudaError_t launch_band_apply_3d<double, double>(cudaStream_t, const PatchDev*, int, const int*, int,
                                                          const double*, const double*, const double*, double*, int);
template cudaError_t launch_band_apply_3d<float, float>(cudaStream_t, const PatchDev*, int, const int*, int,
                                                        const float*, const float*, const float*, float*, int);
template cudaError_t launch_band_apply_3d<float, __nv_bfloat16>(cudaStream_t, const PatchDev*, int, const int*, int,
                                                                const __nv_bfloat16*, const float*, const float*,
                                                                float*, int);

// ---------------------------------------------------------------- 1D transfer along one direction

// out[i_<j, o, i_>j] (=|+=) sum_w wt[o][w] in[i_<j, st[o] + w, i_>j] for one patch per
// blockIdx.y; shapes/offsets from XferT.  Restriction uses the column band of P_l,
// prolongation its row band.  mask: zero outputs whose node is eliminated (coarse
// Dirichlet after restriction).
template <class T>
__global__ void k_transfer_1d(const XferT<T>* __restrict__ xs, const T* __restrict__ in,
                              T* __restrict__ out, int add, const int64_t* __restrict__ mask) {
  const XferT<T> x = xs[blockIdx.y];
  const int64_t total = int64_t(x.outer) * x.nout * x.inner;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    int64_t oi = i / (int64_t(x.nout) * x.inner), rem = i % (int64_t(x.nout) * x.inner);
    int o = int(rem / x.inner), ii = int(rem % x.inner);
    const T* w = x.wt + int64_t(o) * x.width;
    int s0 = x.st[o];
    const T* src = in + x.in_off + (oi * x.nin) * x.inner + ii;
    T acc = 0;
    for (int a = 0; a < x.width; ++a) {
      int k = s0 + a;
      if (k < x.nin) acc = fma(w[a], src[int64_t(k) * x.inner], acc);
    }
    int64_t t = x.out_off + i;
    if (mask && mask[t] < 0) acc = 0;
    out[t] = add ? out[t] + acc : acc;
  }
}

template <class T>
cudaError_t launch_transfer_1d(cudaStream_t s, const XferT<T>* xs, int npatch, int64_t max_out,
                               const T* in, T* out, int add, const int64_t* mask) {
  int64_t g = (max_out + 255) / 256;
  if (g > 1024) g = 1024;
  if (g < 1) g = 1;
  k_transfer_1d<T><<<dim3(unsigned(g), npatch), 256, 0, s>>>(xs, in, out, add, mask);
  return cudaGetLastError();
}
template cudaError_t launch_transfer_1d<double>(cudaStream_t, const XferT<double>*, int, int64_t, const double*,
                                                double*, int, const int64_t*);
template cudaError_t launch_transfer_1d<float>(cudaStream_t, const XferT<float>*, int, int64_t, const float*, float*,
                                               int, const int64_t*);

// ---------------------------------------------------------------- fused 2D transfer

constexpr int XB1 = 32, XB0 = 8;  // outputs per block: 8 rows x 32 columns

template <class T>
__device__ __forceinline__ void transfer2d_block(const Xfer2T<T>& x, const T* __restrict__ in, T* __restrict__ out,
                                                 int add, const int64_t* __restrict__ mask, unsigned char* smraw) {
  T* mid = reinterpret_cast<T*>(smraw);  // XB0 x W: the dir-0 pass on the block's input columns
  const int o0b = blockIdx.y * XB0, o1b = blockIdx.x * XB1;
  if (o0b >= x.nout0 || o1b >= x.nout1) return;
  const int o1e = min(o1b + XB1, x.nout1) - 1;
  const int c1lo = x.st1[o1b], c1hi = min(x.st1[o1e] + x.width1, x.nin1);  // input columns used
  const int W = c1hi - c1lo;
  const T* src = in + x.in_off;
  for (int idx = threadIdx.x; idx < XB0 * W; idx += 256) {
    const int r = idx / W, cc = idx % W, o0 = o0b + r;
    T acc = 0;
    if (o0 < x.nout0) {
      const int s0 = x.st0[o0];
      const T* w = x.w0 + int64_t(o0) * x.width0;
      for (int a = 0; a < x.width0; ++a)
        if (s0 + a < x.nin0) acc = fma(w[a], src[int64_t(s0 + a) * x.nin1 + c1lo + cc], acc);
    }
    mid[idx] = acc;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < XB0 * XB1; idx += 256) {
    const int r = idx / XB1, cx = idx % XB1, o0 = o0b + r, o1 = o1b + cx;
    if (o0 >= x.nout0 || o1 >= x.nout1) continue;
    const int s1 = x.st1[o1];
    const T* w = x.w1 + int64_t(o1) * x.width1;
    T acc = 0;
    for (int b = 0; b < x.width1; ++b)
      if (s1 + b < x.nin1) acc = fma(w[b], mid[r * W + s1 - c1lo + b], acc);
    const int64_t t = x.out_off + int64_t(o0) * x.nout1 + o1;
    if (mask && mask[t] < 0) acc = 0;
    out[t] = add ? out[t] + acc : acc;
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_transfer_2d(const Xfer2T<T>* __restrict__ xs, const T* __restrict__ in,
                                                     T* __restrict__ out, int add, const int64_t* __restrict__ mask) {
  extern __shared__ __align__(16) unsigned char smraw[];
  transfer2d_block<T>(xs[blockIdx.z], in, out, add, mask, smraw);
}

template <class T>
__global__ void __launch_bounds__(256) k_transfer_2d_b(const Xfer2JobT<T>* __restrict__ jobs, int add) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const Xfer2JobT<T> j = jobs[blockIdx.z];
  transfer2d_block<T>(j.x, j.in, j.out, add, j.mask, smraw);
}

template <class T>
cudaError_t launch_transfer_2d_b(cudaStream_t s, const Xfer2JobT<T>* jobs, int njobs, int max_out0, int max_out1,
                                 int max_width1, int add) {
  if (njobs <= 0) return cudaSuccess;
  const size_t sm = sizeof(T) * XB0 * size_t(2 * XB1 + max_width1);
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(k_transfer_2d_b<T>), sm);
  if (e != cudaSuccess) return e;
  dim3 grid((max_out1 + XB1 - 1) / XB1, (max_out0 + XB0 - 1) / XB0, njobs);
  k_transfer_2d_b<T><<<grid, 256, sm, s>>>(jobs, add);
  return cudaGetLastError();
}
template cudaError_t launch_transfer_2d_b<double>(cudaStream_t, const Xfer2JobT<double>*, int, int, int, int, int);

template <class T>
cudaError_t launch_transfer_2d(cudaStream_t s, const Xfer2T<T>* xs, int npatch, int max_out0, int max_out1,
                               int max_width1, const T* in, T* out, int add, const int64_t* mask) {
  // the input columns of 32 consecutive outputs: at most 2 per output step plus one width
  const size_t sm = sizeof(T) * XB0 * size_t(2 * XB1 + max_width1);
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(k_transfer_2d<T>), sm);
  if (e != cudaSuccess) return e;
  dim3 grid((max_out1 + XB1 - 1) / XB1, (max_out0 + XB0 - 1) / XB0, npatch);
  k_transfer_2d<T><<<grid, 256, sm, s>>>(xs, in, out, add, mask);
  return cudaGetLastError();
}
template cudaError_t launch_transfer_2d<double>(cudaStream_t, const Xfer2T<double>*, int, int, int, int,
                                                const double*, double*, int, const int64_t*);
template cudaError_t launch_transfer_2d<float>(cudaStream_t, const Xfer2T<float>*, int, int, int, int, const float*,
                                               float*, int, const int64_t*);

// ---------------------------------------------------------------- mode products

// Shared-memory layout of one block: the n x n matrix as rows of odd stride (the two row
// groups a warp reads fall in different banks), then n rows of kModeCH fibres with stride
// kModeLDX (16-byte rows: each thread reads its four fibres as one vector).
constexpr int kModeCH = 64, kModeLDX = kModeCH + 4;
__host__ __device__ inline int mode_ldm(int n) { return (n & 1) ? n + 2 : n + 1; }
template <class T>
__host__ __device__ inline int mode_xoff(int n) {  // element offset of the fibre tile
  constexpr int al = 16 / int(sizeof(T));
  return (n * mode_ldm(n) + al - 1) / al * al;
}

__device__ __forceinline__ void cp_async_elem(float* s, const float* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(unsigned(__cvta_generic_to_shared(s))), "l"(g)
               : "memory");
}
__device__ __forceinline__ void cp_async_elem(double* s, const double* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(unsigned(__cvta_generic_to_shared(s))), "l"(g)
               : "memory");
}
__device__ __forceinline__ void ld4(const float* p, float (&b)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  b[0] = v.x, b[1] = v.y, b[2] = v.z, b[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&b)[4]) {
  const double2 v0 = reinterpret_cast<const double2*>(p)[0], v1 = reinterpret_cast<const double2*>(p)[1];
  b[0] = v0.x, b[1] = v0.y, b[2] = v1.x, b[3] = v1.y;
}
__device__ __forceinline__ void st4(float* p, const float (&b)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(b[0], b[1], b[2], b[3]);
}
__device__ __forceinline__ void st4(double* p, const double (&b)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(b[0], b[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(b[2], b[3]);
}

// One block: the matrix and kModeCH fibres copied to shared memory with asynchronous
// element copies (all of a thread's copies in flight at once), each thread then RPT rows
// (i = rg + 16 t) x 4 adjacent fibres in registers, one FMA chain per output over
// k = 0..n-1.  The output tile goes back through shared memory.  Fibres that run along
// memory (inner > 1) are moved with lanes along the fibres; fibres contiguous in memory
// (inner == 1) with each warp on an 8 (k) x 4 (fibre) patch, which keeps both the global
// accesses (32-byte pieces) and the shared-memory accesses (32 distinct banks) whole.
template <class T, int RPT>
__global__ void __launch_bounds__(256) k_mode_product(const ModeDescT<T>* __restrict__ ds, int epi) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const ModeDescT<T> d = ds[blockIdx.y];
  const int64_t c0 = int64_t(blockIdx.x) * kModeCH;
  if (c0 >= d.fibres) return;
  const int n = d.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cw = int(d.fibres - c0 < kModeCH ? d.fibres - c0 : int64_t(kModeCH));
  const int ldm = mode_ldm(n);
  T* Ms = reinterpret_cast<T*>(smraw);
  T* Xs = Ms + mode_xoff<T>(n);
  const T* __restrict__ X = d.X;
  const T* __restrict__ Mat = d.Mat;
  T* __restrict__ Y = d.Y;
  const T* __restrict__ E = d.E;
  if (d.mtr) {
    for (int idx = tid; idx < n * n; idx += 256) {
      const int k = idx / n, i = idx - k * n;
      cp_async_elem(Ms + i * ldm + k, Mat + idx);
    }
  } else {
    for (int idx = tid; idx < n * n; idx += 256) {
      const int i = idx / n, k = idx - i * n;
      cp_async_elem(Ms + i * ldm + k, Mat + idx);
    }
  }
  const int64_t inner = d.inner, slab = int64_t(n) * inner;
  const int nkb = (n + 7) >> 3;
  int64_t off = 0;  // inner > 1: this thread's fibre c0 + tid % kModeCH stays fixed
  if (inner > 1) {
    const int cl = tid % kModeCH;
    const int64_t c = c0 + cl;
    off = (c / inner) * slab + c % inner;
    for (int k = tid / kModeCH; k < n; k += 256 / kModeCH) {
      if (cl < cw) cp_async_elem(Xs + k * kModeLDX + cl, X + off + int64_t(k) * inner);
      else Xs[k * kModeLDX + cl] = T(0);
    }
  } else {
    const int kk = lane & 7, cc = lane >> 3;
    for (int tile = warp; tile < nkb * (kModeCH / 4); tile += 8) {
      const int k = (tile % nkb) * 8 + kk, cl = (tile / nkb) * 4 + cc;
      if (k >= n) continue;
      if (cl < cw) cp_async_elem(Xs + k * kModeLDX + cl, X + (c0 + cl) * n + k);
      else Xs[k * kModeLDX + cl] = T(0);
    }
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  const int cg = tid & 15, rg = tid >> 4;
  T acc[RPT][4];
  int rowoff[RPT];
#pragma unroll
  for (int t = 0; t < RPT; ++t) {
    const int i = rg + 16 * t;
    rowoff[t] = (i < n ? i : 0) * ldm;
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[t][u] = T(0);
  }
#pragma unroll 4
  for (int k = 0; k < n; ++k) {
    T b[4];
    ld4(Xs + k * kModeLDX + cg * 4, b);
#pragma unroll
    for (int t = 0; t < RPT; ++t) {
      const T a = Ms[rowoff[t] + k];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[t][u] = fma(a, b[u], acc[t][u]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < RPT; ++t) {
    const int i = rg + 16 * t;
    if (i < n) st4(Xs + i * kModeLDX + cg * 4, acc[t]);
  }
  __syncthreads();
  const bool mul = epi == EPI_MUL;
  if (inner > 1) {
    const int cl = tid % kModeCH;
    if (cl < cw) {
#pragma unroll 4
      for (int i = tid / kModeCH; i < n; i += 256 / kModeCH) {
        const int64_t a = off + int64_t(i) * inner;
        const T v = Xs[i * kModeLDX + cl];
        Y[a] = mul ? v * E[a] : v;
      }
    }
  } else {
    const int kk = lane & 7, cc = lane >> 3;
#pragma unroll 2
    for (int tile = warp; tile < nkb * (kModeCH / 4); tile += 8) {
      const int i = (tile % nkb) * 8 + kk, cl = (tile / nkb) * 4 + cc;
      if (i >= n || cl >= cw) continue;
      const int64_t a = (c0 + cl) * n + i;
      const T v = Xs[i * kModeLDX + cl];
      Y[a] = mul ? v * E[a] : v;
    }
  }
}

template <class T>
cudaError_t launch_mode_product(cudaStream_t s, const ModeDescT<T>* d, int batch, int64_t max_fibres, int max_n,
                                int epi) {
  if (batch <= 0 || max_fibres <= 0) return cudaSuccess;
  if (max_n < 1 || max_n > kModeMaxN) return cudaErrorInvalidValue;
  const size_t sm = sizeof(T) * (size_t(mode_xoff<T>(max_n)) + size_t(max_n) * kModeLDX);
  const dim3 grid(unsigned((max_fibres + kModeCH - 1) / kModeCH), unsigned(batch));
  const int rpt = (max_n + 15) / 16;
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = ensure_smem(reinterpret_cast<const void*>(kern), sm);
    if (e != cudaSuccess) return e;
    kern<<<grid, 256, sm, s>>>(d, epi);
    return cudaGetLastError();
  };
  switch (rpt) {
    case 1: return go(k_mode_product<T, 1>);
    case 2: return go(k_mode_product<T, 2>);
    case 3: return go(k_mode_product<T, 3>);
    case 4: return go(k_mode_product<T, 4>);
    default: return go(k_mode_product<T, 5>);
  }
}
template cudaError_t launch_mode_product<double>(cudaStream_t, const ModeDescT<double>*, int, int64_t, int, int);
template cudaError_t launch_mode_product<float>(cudaStream_t, const ModeDescT<float>*, int, int64_t, int, int);

// ---------------------------------------------------------------- small 3D interiors in one launch

// One mode product of a box held in shared memory: Y(..., i, ...) = sum_k M(i, k) X(..., k, ...)
// along mode `mode` of the n0 x n1 x n2 box, M(i, k) = mtr ? Mat[k n + i] : Mat[i n + k]
// (Mat in shared memory), optionally times E; one FMA chain per output over k in order.
template <class T>
__device__ void fd3_mode(const T* X, T* Y, const T* Mat, int mtr, int mode, const int* n, const T* E) {
  const int n0 = n[0], n1 = n[1], n2 = n[2], total = n0 * n1 * n2, nm = n[mode];
  const int stride = mode == 0 ? n1 * n2 : (mode == 1 ? n2 : 1);
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int q = idx % n2, b = (idx / n2) % n1, a = idx / (n1 * n2);
    const int i = mode == 0 ? a : (mode == 1 ? b : q);
    const int base = idx - i * stride;  // element with the contracted index at 0
    T acc = T(0);
    for (int k = 0; k < nm; ++k) {
      const T m = mtr ? Mat[k * nm + i] : Mat[i * nm + k];
      acc = fma(m, X[base + k * stride], acc);
    }
    Y[idx] = E ? acc * E[idx] : acc;
  }
  __syncthreads();
}

template <class T>
__global__ void __launch_bounds__(256) k_fd3_small(const Fd3SmallT<T>* __restrict__ ds, const T* __restrict__ v,
                                                   T* __restrict__ u, T tau, int add) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const Fd3SmallT<T> d = ds[blockIdx.x];
  const int n0 = d.len[0], n1 = d.len[1], n2 = d.len[2], total = n0 * n1 * n2;
  constexpr int NN = kFd3SmallN * kFd3SmallN * kFd3SmallN;
  T* X = reinterpret_cast<T*>(smraw);
  T* Y = X + NN;
  T* M0 = Y + NN;
  T* M1 = M0 + kFd3SmallN * kFd3SmallN;
  T* M2 = M1 + kFd3SmallN * kFd3SmallN;
  const int tid = threadIdx.x;
  for (int i = tid; i < n0 * n0; i += blockDim.x) M0[i] = d.U0[i];
  for (int i = tid; i < n1 * n1; i += blockDim.x) M1[i] = d.U1[i];
  for (int i = tid; i < n2 * n2; i += blockDim.x) M2[i] = d.U2[i];
  auto tile = [&](int idx) {
    const int q = idx % n2, b = (idx / n2) % n1, a = idx / (n1 * n2);
    return d.tile_off + ((int64_t(a + d.lo[0]) * d.n[1] + (b + d.lo[1])) * d.n[2] + (q + d.lo[2]));
  };
  for (int idx = tid; idx < total; idx += blockDim.x) X[idx] = v[tile(idx)];
  __syncthreads();
  const int nn[3] = {n0, n1, n2};
  fd3_mode(X, Y, M0, 1, 0, nn, static_cast<const T*>(nullptr));
  fd3_mode(Y, X, M1, 1, 1, nn, static_cast<const T*>(nullptr));
  fd3_mode(X, Y, M2, 1, 2, nn, d.Dinv);
  fd3_mode(Y, X, M0, 0, 0, nn, static_cast<const T*>(nullptr));
  fd3_mode(X, Y, M1, 0, 1, nn, static_cast<const T*>(nullptr));
  fd3_mode(Y, X, M2, 0, 2, nn, static_cast<const T*>(nullptr));
  for (int idx = tid; idx < total; idx += blockDim.x) {
    const int64_t t = tile(idx);
    u[t] = add ? fma(tau, X[idx], u[t]) : tau * X[idx];
  }
}

template <class T>
cudaError_t launch_fd3_small(cudaStream_t s, const Fd3SmallT<T>* d, int n, const T* v, T* u, T tau, int add) {
  if (n <= 0) return cudaSuccess;
  const size_t sm = sizeof(T) * (2 * size_t(kFd3SmallN) * kFd3SmallN * kFd3SmallN + 3 * size_t(kFd3SmallN) * kFd3SmallN);
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(k_fd3_small<T>), sm);
  if (e != cudaSuccess) return e;
  k_fd3_small<T><<<n, 256, sm, s>>>(d, v, u, tau, add);
  return cudaGetLastError();
}
template cudaError_t launch_fd3_small<double>(cudaStream_t, const Fd3SmallT<double>*, int, const double*, double*,
                                              double, int);
template cudaError_t launch_fd3_small<float>(cudaStream_t, const Fd3SmallT<float>*, int, const float*, float*, float,
                                             int);

// ---------------------------------------------------------------- small 3D interface pieces in one launch

template <class T>
__global__ void __launch_bounds__(256) k_iface3_small(const Iface3SmallT<T> p, const T* __restrict__ v, T tau,
                                                      int add) {
  constexpr int M = kIface3SmallN;
  __shared__ T U0[M * M], U1[M * M], X[M * M], Tm[M * M];
  const int tid = threadIdx.x, b = blockIdx.x;
  auto scatter = [&](int64_t g, T val) {
    for (int64_t c = p.ptr[g]; c < p.ptr[g + 1]; ++c) {
      T* up = p.u + p.idx[c];
      *up = add ? *up + val : val;
    }
  };
  auto gather = [&](int64_t g) {
    T acc = 0;
    for (int64_t c = p.ptr[g]; c < p.ptr[g + 1]; ++c) acc += v[p.idx[c]];
    return acc;
  };
  if (b < p.nfaces) {
    const FaceSmallT<T> f = p.faces[b];
    const int n0 = f.len0, n1 = f.len1, nn = n0 * n1;
    for (int i = tid; i < n0 * n0; i += 256) U0[i] = f.U0[i];
    for (int i = tid; i < n1 * n1; i += 256) U1[i] = f.U1[i];
    for (int i = tid; i < nn; i += 256) X[i] = gather(f.first + i);
    __syncthreads();
    for (int i = tid; i < nn; i += 256) {  // T = U0^T G
      const int a = i / n1, c = i % n1;
      T acc = 0;
      for (int k = 0; k < n0; ++k) acc = fma(U0[k * n0 + a], X[k * n1 + c], acc);
      Tm[i] = acc;
    }
    __syncthreads();
    for (int i = tid; i < nn; i += 256) {  // Y = (T U1) .* Dinv
      const int r = i / n1, j = i % n1;
      T acc = 0;
      for (int k = 0; k < n1; ++k) acc = fma(U1[k * n1 + j], Tm[r * n1 + k], acc);
      X[i] = acc * f.Dinv[i];
    }
    __syncthreads();
    for (int i = tid; i < nn; i += 256) {  // S = U0 Y
      const int a = i / n1, c = i % n1;
      T acc = 0;
      for (int k = 0; k < n0; ++k) acc = fma(U0[a * n0 + k], X[k * n1 + c], acc);
      Tm[i] = acc;
    }
    __syncthreads();
    for (int i = tid; i < nn; i += 256) {  // Z = S U1^T, scattered
      const int r = i / n1, j = i % n1;
      T acc = 0;
      for (int k = 0; k < n1; ++k) acc = fma(U1[j * n1 + k], Tm[r * n1 + k], acc);
      scatter(f.first + i, tau * acc);
    }
    return;
  }
  if (b < p.nfaces + p.nedges) {
    const EdgeSmallT<T> e = p.edges[b - p.nfaces];
    const int n = e.len;
    for (int i = tid; i < n * n; i += 256) U0[i] = e.U[i];
    for (int i = tid; i < n; i += 256) X[i] = gather(e.first + i);
    __syncthreads();
    for (int j = tid; j < n; j += 256) {  // y = (g^T U) .* dinv
      T acc = 0;
      for (int i = 0; i < n; ++i) acc = fma(X[i], U0[i * n + j], acc);
      Tm[j] = acc * e.dinv[j];
    }
    __syncthreads();
    for (int i = tid; i < n; i += 256) {  // z = U y, scattered
      T acc = 0;
      for (int j = 0; j < n; ++j) acc = fma(Tm[j], U0[i * n + j], acc);
      scatter(e.first + i, tau * acc);
    }
    return;
  }
  for (int64_t g = p.vbeg + tid; g < p.vend; g += 256) scatter(g, tau * (p.vscale[g] * gather(g)));
}

template <class T>
cudaError_t launch_iface3_small(cudaStream_t s, const Iface3SmallT<T>& p, const T* v, T tau, int add) {
  const int blocks = p.nfaces + p.nedges + (p.vend > p.vbeg ? 1 : 0);
  if (blocks <= 0) return cudaSuccess;
  k_iface3_small<T><<<blocks, 256, 0, s>>>(p, v, tau, add);
  return cudaGetLastError();
}
template cudaError_t launch_iface3_small<double>(cudaStream_t, const Iface3SmallT<double>&, const double*, double,
                                                 int);
template cudaError_t launch_iface3_small<float>(cudaStream_t, const Iface3SmallT<float>&, const float*, float, int);

// ---------------------------------------------------------------- interior box gather/scatter

// Compact copy of every patch-interior box (3D FD works on compact tensors) and the
// scatter of tau * Z back into the boxes.
template <class T>
__global__ void k_box_copy(const BoxDev* __restrict__ boxes, const T* __restrict__ src, T* __restrict__ dst,
                           int to_compact, T tau, int add) {
  const BoxDev b = boxes[blockIdx.y];
  const int64_t total = int64_t(b.len[0]) * b.len[1] * b.len[2];
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    int64_t i0 = i / (int64_t(b.len[1]) * b.len[2]), rem = i % (int64_t(b.len[1]) * b.len[2]);
    int i1 = int(rem / b.len[2]), i2 = int(rem % b.len[2]);
    int64_t t = b.tile_off + ((i0 + b.lo[0]) * b.n[1] + (i1 + b.lo[1])) * int64_t(b.n[2]) + (i2 + b.lo[2]);
    int64_t c = b.compact_off + i;
    if (to_compact) dst[c] = src[t];
    else dst[t] = add ? fma(tau, src[c], dst[t]) : tau * src[c];
  }
}

template <class T>
cudaError_t launch_box_copy(cudaStream_t s, const BoxDev* boxes, int nbox, int64_t max_box, const T* src,
                            T* dst, int to_compact, T tau, int add) {
  if (nbox <= 0) return cudaSuccess;
  int64_t g = (max_box + 255) / 256;
  if (g > 1024) g = 1024;
  if (g < 1) g = 1;
  k_box_copy<T><<<dim3(unsigned(g), nbox), 256, 0, s>>>(boxes, src, dst, to_compact, tau, add);
  return cudaGetLastError();
}
template cudaError_t launch_box_copy<double>(cudaStream_t, const BoxDev*, int, int64_t, const double*, double*, int,
                                             double, int);
template cudaError_t launch_box_copy<float>(cudaStream_t, const BoxDev*, int, int64_t, const float*, float*, int,
                                            float, int);

}  // namespace igamg
