// Device kernels of the multigrid-preconditioned CG and their launchers (FP64, and the FP32
// twins of the precision variant).
// Every launcher takes the stream explicitly and returns the launch status.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

namespace igamg {

// Raises `func`'s dynamic shared memory limit on the current device to at least `bytes` and
// never lowers it, so launches of the same kernel from concurrent host threads with
// smaller needs stay valid.
cudaError_t ensure_smem(const void* func, size_t bytes);

// Per-patch descriptor of one level's tile layout and band storage.
struct PatchDev {
  int64_t off;       // tile offset (nodes)
  int64_t band_off;  // offset of the patch's band block (doubles)
  int n[3];          // basis sizes per direction (n[2] = 1 in 2D)
  int p[3];          // degrees per direction
  int m[3];          // intervals per direction
};

// Batched GEMM descriptor: C = op(A) op(B), M x N with inner dimension K (row-major).
template <class T>
struct GemmDescT {
  const T* A;
  const T* B;
  T* C;
  const T* E;  // epilogue operand (matrix M x N with lde, or vector of length M / N)
  int lda, ldb, ldc, lde;
  int M, N, K;
};
using GemmDesc = GemmDescT<double>;

enum GemmEpilogue { EPI_STORE = 0, EPI_MUL = 1, EPI_ROWSCALE = 2, EPI_ASSIGN = 3, EPI_ADD = 4, EPI_COLSCALE = 5 };

// Element-by-element assembly of one patch (the colour loop is inside the launcher).
struct ElemAsm {
  int dim, p, mass;
  int n[3], m[3], color[3];
  int64_t off, band_off, nn;
  const double* corners;       // [2^d * d] of this patch
  const double* xq[3];         // [m * (p+1)] Gauss points per element
  const double* wq[3];
  const double* B[3];          // [m][p+1 q][p+1 a]
  const double* dB[3];
  const int64_t* l2g;          // level l2g (tile indexed)
  double* band;
};
cudaError_t launch_assemble_elem(cudaStream_t s, const ElemAsm& ea);
size_t elem_asm_smem(int D, int p, bool mass);

// y = f - A u per tile (residual) or y = A u when f == NULL (apply).  TV vector type,
// TB band storage type: (double, double), (float, float), (float, __nv_bfloat16).
// uniform_p: the common degree of every patch (selects an unrolled kernel for 1..6), or 0.
template <class TV, class TB>
cudaError_t launch_band_apply_2d(cudaStream_t s, const PatchDev* pd_dev, int K, int max_n0, int max_n1, int max_p,
                                 const TB* band, const TV* u, const TV* f, TV* y, int uniform_p = 0);
// Rectangle patch with constant metric C = |det J| J^{-1} J^{-T} = diag(c0, c1): the stiffness
// is the Kronecker sum A = c0 K_0 (x) M_1 + c1 M_0 (x) K_1 of the 1D stiffness K_j and mass
// M_j on (0,1).  The 1D matrices are stored row-banded, [n_j][2p_j+1] with entry (i, t) =
// X(i, i - p_j + t) (0 outside the matrix).
template <class T>
struct KronDevT {
  int64_t off;  // tile offset (nodes)
  int n0, n1, p0, p1;
  const T *K0, *M0, *K1, *M1;
  T c0, c1;
};
// y = f - A u (f != NULL) or y = A u per tile; rows and columns of eliminated (Dirichlet)
// nodes, active[node] == 0, are dropped: their u is read as 0 and their y is f or 0.
template <class T>
cudaError_t launch_kron_apply_2d(cudaStream_t s, const KronDevT<T>* kd, int K, int max_n0, int max_n1, int max_p,
                                 const unsigned char* active, const T* u, const T* f, T* y);
size_t kron_apply_smem(int elem_size, int max_p);

// uniform_p: the common degree of every patch and direction (selects an unrolled kernel
// for 2, 3, 4), or 0.
template <class TV, class TB>
cudaError_t launch_band_apply_3d(cudaStream_t s, const PatchDev* pd_dev, int K, const int* max_n, int max_p,
                                 const TB* band, const TV* u, const TV* f, TV* y, int uniform_p = 0);

template <class T>
cudaError_t launch_gemm(cudaStream_t s, const GemmDescT<T>* d_desc, int batch, int maxM, int maxN,
                        bool transA, bool transB, int epi, T alpha, int R = 0);
// One FP64 GEMM with the descriptor passed by value (no device-side descriptor array).
cudaError_t launch_gemm_one(cudaStream_t s, const GemmDesc& d, bool transA, bool transB, int epi,
                            double alpha);

// Interface pieces: gather sums of the copies of every interface node from a
// distributed vector; scatter tau * (Z + vscale * G) to every copy of an accumulated vector.
template <class T>
cudaError_t launch_iface_gather(cudaStream_t s, int64_t n_nodes, const int64_t* ptr, const int64_t* idx,
                                const T* v, T* G);
template <class T>
cudaError_t launch_iface_scatter(cudaStream_t s, int64_t n_nodes, const int64_t* ptr, const int64_t* idx,
                                 const T* Z, const T* G, const T* vscale, T tau, int add, T* u);

// Canonical distributed form of v on the interface nodes (sum of copies in the first copy).
template <class T>
cudaError_t launch_canonicalize(cudaStream_t s, int64_t n_nodes, const int64_t* ptr, const int64_t* idx, T* v);

// One direction of a tensor transfer: out has `nout` entries along the direction, in has
// `nin`; outer/inner are the products of the sizes before/after it.
template <class T>
struct XferT {
  int64_t in_off, out_off;
  int outer, inner, nin, nout, width;
  const T* wt;   // [nout][width]
  const int* st; // [nout]
};
template <class T>
cudaError_t launch_transfer_1d(cudaStream_t s, const XferT<T>* xs, int npatch, int64_t max_out, const T* in, T* out,
                               int add, const int64_t* mask);

// Both 1D passes of a 2D transfer in one launch: out = T1 (T0 in) per patch tile, with
// T_j(o, i) = w_j[o][a] for i = st_j[o] + a (a < width_j); the intermediate rows of a block
// live in shared memory.  Restriction (mask: zero where mask < 0) and prolongation (add).
template <class T>
struct Xfer2T {
  int64_t in_off, out_off;
  int nin0, nin1, nout0, nout1;
  const T *w0, *w1;
  const int *st0, *st1;
  int width0, width1;
};
template <class T>
cudaError_t launch_transfer_2d(cudaStream_t s, const Xfer2T<T>* xs, int npatch, int max_out0, int max_out1,
                               int max_width1, const T* in, T* out, int add, const int64_t* mask);

// Interior box of a tile <-> compact tensor.
// Whole patch-interior smoother of one small 2D interior in one block (the four FD
// contractions in shared memory): u (=|+=) tau U0 ((U0^T v U1) .* Dinv) U1^T.
constexpr int kFdSmallMax = 32;
template <class T>
struct FdSmallT {
  const T *U0, *U1, *Dinv;  // n0 x n0, n1 x n1 (columns = FD basis), n0 x n1
  const T *vF, *vR;         // the interior block in the F and R tiles (row stride ld)
  T* u;                     // the interior block in the U tile
  int n0, n1, ld;
};
template <class T>
cudaError_t launch_fd_small(cudaStream_t s, const FdSmallT<T>* d, int count, int from_F, T tau, int add);

// Patch-interior FD of a 2D level in two launches over blocks of RB rows: pass 1 computes
// rows of T = U0^T X and then of Y = (T U1) .* Dinv; pass 2 rows of S = U0 Y and then of
// u (=|+=) tau S U1^T.  Y is a scratch n0 x n1 block per interior.
template <class T>
struct FdRowsT {
  const T *U0, *U1, *Dinv;
  const T *vF, *vR;  // interior block in the F and R tiles (row stride ld)
  T* u;              // interior block in the U tile
  T* Y;              // scratch, n0 x n1 contiguous
  int n0, n1, ld;
};
template <class T>
cudaError_t launch_fd_rows(cudaStream_t s, const FdRowsT<T>* d, int count, int max_n0, int max_n1, int pass,
                           int from_F, T tau, int add);

// The whole smoother of a small 2D level in one launch: blocks [0, nfd) are the interiors
// (as launch_fd_small), the next nedges blocks one edge each (gather of the copies, 1D FD
// with U (len x len, columns = basis) and dinv, scatter tau z to the copies), the last
// block the vertices (z = vscale * gathered value).  Interface nodes are numbered as the
// gather/scatter CSR (ptr, idx) numbers them.
template <class T>
struct EdgeSmallT {
  const T *U, *dinv;
  int64_t first;  // first interface node of the edge
  int len;
};
template <class T>
struct SmoothSmallT {
  const FdSmallT<T>* fd;
  int nfd;
  const EdgeSmallT<T>* edges;
  int nedges;
  const int64_t *ptr, *idx;
  const T* vscale;
  int64_t vbeg, vend;  // vertex nodes
  const T *vF, *vR;    // level vectors (tiles)
  T* u;
};
template <class T>
cudaError_t launch_smooth_small(cudaStream_t s, const SmoothSmallT<T>& p, int from_F, T tau, int add);

struct BoxDev {
  int64_t tile_off, compact_off;
  int n[3], lo[3], len[3];
};
template <class T>
cudaError_t launch_box_copy(cudaStream_t s, const BoxDev* boxes, int nbox, int64_t max_box, const T* src, T* dst,
                            int to_compact, T tau, int add);

// Product of a small dense n x n matrix along one mode of a tensor (the FD contractions of
// the 3D interiors): for every fibre c and row i,
//   Y(i, c) = sum_k M(i, k) X(k, c),   M(i, k) = mtr ? Mat[k * n + i] : Mat[i * n + k],
// with X(k, c) at X[off(c) + k * inner], off(c) = (c / inner) * n * inner + c % inner (the
// tensor viewed as outer x n x inner; `fibres` = outer * inner), Y laid out like X, and
// E (EPI_MUL) like Y.  Every output is one FMA chain over k = 0..n-1 in order, as in
// launch_gemm.  n <= kModeMaxN.
template <class T>
struct ModeDescT {
  const T* Mat;
  const T* X;
  T* Y;
  const T* E;
  int n, mtr;
  int64_t inner, fibres;
};
constexpr int kModeMaxN = 80;

// FP32/BF16 bands of 3D patches in the paired layout: per patch (PatchDev.band_off in band
// elements) the (2p+1)^3 tap planes of n0 x n1 x n2e nodes, n2e = n2 rounded up to even
// (padding zero), so that every node pair (2x, 2x+1) of a row is one aligned 2-element load.
__host__ __device__ inline int band_row_even(int n2) { return (n2 + 1) & ~1; }
// Copies the FP64 bands (layout of `src_pd`) into the paired layout of `dst_pd` (TB = float
// or __nv_bfloat16, rounded as the flat conversions round).
template <class TB>
cudaError_t launch_band_pair(cudaStream_t s, const PatchDev* src_pd, const PatchDev* dst_pd, int K, int taps,
                             int64_t max_nodes, const double* src, TB* dst);
// FP32 bands of 3D patches in the tap-blocked layout: per patch (PatchDev.band_off in floats)
// blocks of 32 consecutive nodes (flat order), each holding its (2p+1)^3 taps x 32 nodes, so
// that a warp's loads of all taps of a row segment stream through contiguous memory:
// element (t, node) at band_off + ((node / 32) taps + t) 32 + node % 32 (padding zero).
cudaError_t launch_band_blk_f32(cudaStream_t s, const PatchDev* src_pd, const PatchDev* dst_pd, int K, int taps,
                                int64_t max_nodes, const double* src, float* dst);
// The 3D apply on tap-blocked FP32 bands (uniform degree 2..4), same tap order and FMA chain
// as launch_band_apply_3d (bit-identical results).
cudaError_t launch_band_apply_3d_blk(cudaStream_t s, const PatchDev* pd_dev, int K, const int* max_n, int p,
                                     const float* band, const float* u, const float* f, float* y);
// The 3D apply on paired bands (every patch of degree p = uniform_p in 2..4): each thread
// computes two adjacent nodes of a row from one 2-element load per tap, FP32 accumulation
// in the tap order of launch_band_apply_3d (bit-identical results).
template <class TB>
cudaError_t launch_band_apply_3d_pair(cudaStream_t s, const PatchDev* pd_dev, int K, const int* max_n, int p,
                                      const TB* band, const float* u, const float* f, float* y);

// Interior fast diagonalisation of one small 3D patch interior (every length <= kFd3SmallN):
// the box of the tile (tile_off, tile extents n, first index lo, lengths len) and the FD
// operands U0, U1, U2 (len x len) and Dinv (len0 x len1 x len2).
template <class T>
struct Fd3SmallT {
  const T *U0, *U1, *U2, *Dinv;
  int64_t tile_off;
  int n[3], lo[3], len[3];
};
constexpr int kFd3SmallN = 16;

// The interface pieces of a small 3D level in one launch (faces and edges of length <=
// kIface3SmallN; a face costs one block 4 n^3 FMAs, less than the eight launches it replaces
// at these sizes): block per face (gather of the sum of its nodes' copies, the face's 2D fast
// diagonalisation Z = U0 ((U0^T G U1) .* Dinv) U1^T, tau-scatter to every copy), block per
// edge (1D: z = U ((g^T U) .* dinv)), and one block for the vertices (z = vscale g); the FMA
// order of the gather, face/edge and scatter launches it replaces.
constexpr int kIface3SmallN = 24;
template <class T>
struct FaceSmallT {
  const T *U0, *U1, *Dinv;
  int64_t first;  // first interface node of the face (row-major len0 x len1)
  int len0, len1;
};
template <class T>
struct Iface3SmallT {
  const FaceSmallT<T>* faces;
  int nfaces;
  const EdgeSmallT<T>* edges;
  int nedges;
  const int64_t *ptr, *idx;  // interface node -> its copies in the level vectors
  const T* vscale;
  int64_t vbeg, vend;        // vertex nodes
  T* u;
};
template <class T>
cudaError_t launch_iface3_small(cudaStream_t s, const Iface3SmallT<T>& p, const T* v, T tau, int add);
// u = (add ? u + tau z : tau z) on every interior box, z = L^{-1} v restricted to the box:
// one block per interior, the six mode products (transposed bases, Dinv, bases) in shared
// memory with the FMA order of launch_mode_product, so the result equals the box copy +
// mode products + box copy path bit for bit.
template <class T>
cudaError_t launch_fd3_small(cudaStream_t s, const Fd3SmallT<T>* d, int n, const T* v, T* u, T tau, int add);
template <class T>
cudaError_t launch_mode_product(cudaStream_t s, const ModeDescT<T>* d, int batch, int64_t max_fibres, int max_n,
                                int epi);

// Coarse solve in FP64: x_copies = A0inv * (sum of copies of f) for the N0 level-0 dofs.
template <class T>
cudaError_t launch_coarse_solve(cudaStream_t s, int64_t N0, const int64_t* ptr, const int64_t* idx,
                                const double* A0inv, const T* f, T* x);

// Global <-> tile conversions (g2t CSR of copies per global dof).
template <class T>
cudaError_t launch_global_to_tile(cudaStream_t s, int64_t N, const int64_t* ptr, const int64_t* idx, const T* xg,
                                  T* xt, int first_only);
template <class T>
cudaError_t launch_tile_to_global(cudaStream_t s, int64_t N, const int64_t* ptr, const int64_t* idx, const T* xt,
                                  T* xg, int sum_copies);

// Deterministic reductions (FP64 partials): fixed grid of RED_BLOCKS partial sums, then one block.
constexpr int RED_BLOCKS = 1216;  // 8 x 152 SMs: enough loads in flight to stream HBM
template <class T>
cudaError_t launch_dot(cudaStream_t s, const T* a, const T* b, int64_t n, double* partials, double* out);
// sum over active dofs of (sum of copies of v)^2 for a distributed vector v
template <class T>
cudaError_t launch_norm2_dist(cudaStream_t s, int64_t N, const int64_t* ptr, const int64_t* idx, const T* v,
                              double* partials, double* out);

// PCG updates with scalars kept on the device: scal[0]=rz, scal[1]=pw, scal[2]=rz_new.
template <class T>
cudaError_t launch_pcg_xr(cudaStream_t s, int64_t n, const double* scal, T* x, T* r, const T* p, const T* w);
template <class T>
cudaError_t launch_pcg_p(cudaStream_t s, int64_t n, double* scal, T* p, const T* z);
cudaError_t launch_axpby(cudaStream_t s, int64_t n, double a, const double* x, double b, double* y);
// Flexible CG direction update: beta from scal[2] (r.z new), scal[4] (r.z_old), scal[0]
// (r.z old); p = z + beta p; z_old = z.
cudaError_t launch_fcg_p(cudaStream_t s, int64_t n, double* scal, float* p, const float* z, float* zold);

// Precision conversions for iterative refinement.
cudaError_t launch_convert_f64_f32(cudaStream_t s, int64_t n, const double* src, double scale, float* dst);
cudaError_t launch_convert_f64_bf16(cudaStream_t s, int64_t n, const double* src, __nv_bfloat16* dst);
cudaError_t launch_add_scaled_f32(cudaStream_t s, int64_t n, const float* d, double scale, double* x);

// ---------------------------------------------------------------- cross-problem batches
// The kernels above over job lists whose entries carry their own vectors, so that one
// launch covers the patches, levels or vectors of many independent problems.  Every job is
// computed with exactly the arithmetic of the single-problem kernel (the results do not
// depend on what else the launch holds).
template <class T>
struct KronJobT {  // one rectangle patch of one level
  KronDevT<T> kd;
  const unsigned char* active;
  const T* u;
  const T* f;  // NULL: y = A u
  T* y;
};
template <class T>
cudaError_t launch_kron_apply_2d_b(cudaStream_t s, const KronJobT<T>* jobs, int njobs, int max_n0, int max_n1,
                                   int max_p);
// Small-level smoothers of many levels: job j owns blocks [bstart[j], bstart[j+1]).
template <class T>
cudaError_t launch_smooth_small_b(cudaStream_t s, const SmoothSmallT<T>* jobs, const int* bstart, int njobs,
                                  int total_blocks, int from_F, T tau, int add);
template <class T>
struct Xfer2JobT {  // one patch tile of a 2D transfer
  Xfer2T<T> x;
  const T* in;
  T* out;
  const int64_t* mask;
};
template <class T>
cudaError_t launch_transfer_2d_b(cudaStream_t s, const Xfer2JobT<T>* jobs, int njobs, int max_out0, int max_out1,
                                 int max_width1, int add);
// Node lists of one level: interface gather (G = sums of copies of v), scatter (u (=|+=)
// tau (Z + vscale G) to every copy), coarse solves and global <-> tile conversions.
template <class T>
struct NodeJobT {
  int64_t n;
  const int64_t *ptr, *idx;
  const T* v;          // gather / coarse: the distributed input
  T* G;                // gathered sums (interface) / global vector (conversions)
  const T* Z;
  const T* vscale;
  T* u;                // scatter / coarse: the accumulated output
  const double* Ainv;  // coarse solve: the explicit inverse (n x n)
};
template <class T>
cudaError_t launch_iface_gather_b(cudaStream_t s, const NodeJobT<T>* jobs, int njobs, int64_t max_n);
template <class T>
cudaError_t launch_iface_scatter_b(cudaStream_t s, const NodeJobT<T>* jobs, int njobs, int64_t max_n, T tau,
                                   int add);
template <class T>
cudaError_t launch_coarse_solve_b(cudaStream_t s, const NodeJobT<T>* jobs, int njobs, int64_t max_n);
// global -> tile (G -> u, first_only) and tile -> global (v -> G, sum_copies)
template <class T>
cudaError_t launch_global_to_tile_b(cudaStream_t s, const NodeJobT<T>* jobs, int njobs, int64_t max_n, int first_only);
template <class T>
cudaError_t launch_tile_to_global_b(cudaStream_t s, const NodeJobT<T>* jobs, int njobs, int64_t max_n, int sum_copies);
// Vectors of many problems.  Reductions keep the single-problem partition (RED_BLOCKS
// partials per job in `partials` + j * RED_BLOCKS, then one block per job).
template <class T>
struct VecJobT {
  int64_t n;
  double* scal;      // the job's PCG scalars (also the reduction output base)
  const int64_t *ptr, *idx;  // norm of a distributed vector: copies per active dof (n dofs)
  T *a, *b, *c, *d;  // operands (meaning per kernel)
};
template <class T>
cudaError_t launch_dot_b(cudaStream_t s, const VecJobT<T>* jobs, int njobs, int out, double* partials);
template <class T>
cudaError_t launch_norm2_dist_b(cudaStream_t s, const VecJobT<T>* jobs, int njobs, int out, double* partials);
// x += alpha p, r -= alpha w (a = x, b = r, c = p, d = w) for the jobs with active[j] != 0
template <class T>
cudaError_t launch_pcg_xr_b(cudaStream_t s, const VecJobT<T>* jobs, int njobs, int64_t max_n, const int* active);
// p = z + beta p, then scal[0] = scal[2] (a = p, c = z) for the active jobs
template <class T>
cudaError_t launch_pcg_p_b(cudaStream_t s, const VecJobT<T>* jobs, int njobs, int64_t max_n, const int* active);
// a = b (copy), a = 0 (b == NULL), or b += a (axpy_into: b = 1 * a + 1 * b)
template <class T>
cudaError_t launch_copy_b(cudaStream_t s, const VecJobT<T>* jobs, int njobs, int64_t max_n, int mode);

}  // namespace igamg
