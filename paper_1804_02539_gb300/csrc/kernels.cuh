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

// Transfer descriptor (fine level l, coarse level l-1) of one patch; 1D tables per direction.
struct TransferDev {
  int64_t off_f, off_c, off_t;  // fine/coarse tile offsets, temp offset
  int nf[3], nc[3];
  const double* rw[3];  // restriction weights [nc * wr] (column j of P: fine rows rs[j]..)
  const int* rs[3];     // [nc] first fine row of column j
  const double* pw[3];  // prolongation weights [nf * wp] (row i of P: coarse cols ps[i]..)
  const int* ps[3];     // [nf]
  int wr[3], wp[3];
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

// Geometry factors at all Gauss points of a patch: 4 values per point,
// w|detJ|(J^{-1}J^{-T})_{00,01,11} and w|detJ| (2D).
cudaError_t launch_geom_factors_2d(cudaStream_t s, const double* corners, int m0, int m1, int nq,
                                   const double* xq0, const double* wq0, const double* xq1,
                                   const double* wq1, double* G);
// Band coefficients of the patch stiffness (mass=0) or geometry mass (mass=1) matrix.
cudaError_t launch_assemble_2d(cudaStream_t s, const PatchDev& pd, const double* G,
                               const double* B0, const double* dB0, const double* B1,
                               const double* dB1, const int64_t* l2g_tile, int mass,
                               double* band);

// y = beta*f - A u per tile (f may be NULL, then y = -A u if beta... see launcher), i.e.
// residual (f != NULL) or apply (f == NULL, y = A u).
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

cudaError_t launch_restrict_2d(cudaStream_t s, const TransferDev* td, int K, int max_nf,
                               int max_nc, const double* rf, double* tmp, double* rc,
                               const int64_t* l2g_c, int64_t Tc);
cudaError_t launch_prolong_2d(cudaStream_t s, const TransferDev* td, int K, int max_nf,
                              int max_nc, const double* uc, double* tmp, double* uf);

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
