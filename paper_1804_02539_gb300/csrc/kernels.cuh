// Device kernels of the multigrid-preconditioned CG (FP64 path) and their launchers.
// Every launcher takes the stream explicitly and returns the launch status.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace igamg {

// Per-patch descriptor of one level's tile layout and band storage.
struct PatchDev {
  int64_t off;       // tile offset (nodes)
  int64_t band_off;  // offset of the patch's band block (doubles)
  int n[3];          // basis sizes per direction (n[2] = 1 in 2D)
  int p[3];          // degrees per direction
  int m[3];          // intervals per direction
};

// Batched GEMM descriptor: C = op(A) op(B), M x N with inner dimension K (row-major).
struct GemmDesc {
  const double* A;
  const double* B;
  double* C;
  const double* E;  // epilogue operand (matrix M x N with lde, or vector of length M)
  int lda, ldb, ldc, lde;
  int M, N, K;
};

enum GemmEpilogue { EPI_STORE = 0, EPI_MUL = 1, EPI_ROWSCALE = 2, EPI_ASSIGN = 3, EPI_ADD = 4, EPI_COLSCALE = 5 };

// Element-by-element assembly of one patch (any colour loop inside the launcher).
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

// 3D band apply (same contract as the 2D one).
cudaError_t launch_band_apply_3d(cudaStream_t s, const PatchDev* pd_dev, int K, const int* max_n, int max_p,
                                 const double* band, const double* u, const double* f, double* y);

// One direction of a tensor transfer: out has `nout` entries along the direction, in has
// `nin`; outer/inner are the products of the sizes before/after it.
struct Xfer1D {
  int64_t in_off, out_off;
  int outer, inner, nin, nout, width;
  const double* wt;  // [nout][width]
  const int* st;     // [nout]
};
cudaError_t launch_transfer_1d(cudaStream_t s, const Xfer1D* xs, int npatch, int64_t max_out,
                               const double* in, double* out, int add, const int64_t* mask);

// Interior box of a tile <-> compact tensor.
struct BoxDev {
  int64_t tile_off, compact_off;
  int n[3], lo[3], len[3];
};
cudaError_t launch_box_copy(cudaStream_t s, const BoxDev* boxes, int nbox, int64_t max_box, const double* src,
                            double* dst, int to_compact, double tau, int add);

// y = f - A u per tile (residual) or y = A u when f == NULL (apply).
cudaError_t launch_band_apply_2d(cudaStream_t s, const PatchDev* pd_dev, int K, int max_n0,
                                 int max_n1, int max_p, const double* band, const double* u,
                                 const double* f, double* y);

cudaError_t launch_gemm(cudaStream_t s, const GemmDesc* d_desc, int batch, int maxM, int maxN,
                        bool transA, bool transB, int epi, double alpha);
// One GEMM with the descriptor passed by value (no device-side descriptor array).
cudaError_t launch_gemm_one(cudaStream_t s, const GemmDesc& d, bool transA, bool transB, int epi,
                            double alpha);

// Interface pieces: gather sums of the copies of every interface node from a
// distributed vector; scatter tau * value to every copy of an accumulated vector.
cudaError_t launch_iface_gather(cudaStream_t s, int64_t n_nodes, const int64_t* ptr,
                                const int64_t* idx, const double* v, double* G);
cudaError_t launch_iface_scatter(cudaStream_t s, int64_t n_nodes, const int64_t* ptr,
                                 const int64_t* idx, const double* Z, const double* G,
                                 const double* vscale, double tau, int add, double* u);

// Coarse solve: x_copies = A0inv * (sum of copies of f) for the N0 level-0 dofs.
cudaError_t launch_coarse_solve(cudaStream_t s, int64_t N0, const int64_t* ptr,
                                const int64_t* idx, const double* A0inv, const double* f,
                                double* x);

// Global <-> tile conversions (g2t CSR of copies per global dof).
cudaError_t launch_global_to_tile(cudaStream_t s, int64_t N, const int64_t* ptr,
                                  const int64_t* idx, const double* xg, double* xt, int first_only);
cudaError_t launch_tile_to_global(cudaStream_t s, int64_t N, const int64_t* ptr,
                                  const int64_t* idx, const double* xt, double* xg, int sum_copies);

// Deterministic reductions: fixed grid of `nblocks` partial sums, then one block.
constexpr int RED_BLOCKS = 304;  // 2 x 152 SMs
cudaError_t launch_dot(cudaStream_t s, const double* a, const double* b, int64_t n,
                       double* partials, double* out);
// sum over active dofs of (sum of copies of v)^2 for a distributed vector v
cudaError_t launch_norm2_dist(cudaStream_t s, int64_t N, const int64_t* ptr, const int64_t* idx,
                              const double* v, double* partials, double* out);

// PCG updates with scalars kept on the device: scal[0]=rz, scal[1]=pw, scal[2]=rz_new.
cudaError_t launch_pcg_xr(cudaStream_t s, int64_t n, const double* scal, double* x, double* r,
                          const double* p, const double* w);
cudaError_t launch_pcg_p(cudaStream_t s, int64_t n, double* scal, double* p, const double* z);
cudaError_t launch_axpby(cudaStream_t s, int64_t n, double a, const double* x, double b, double* y);

}  // namespace igamg
