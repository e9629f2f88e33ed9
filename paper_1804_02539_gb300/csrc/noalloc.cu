// igamg_fd_apply_noalloc: the fast-diagonalisation apply of igamg_fd_apply, with its
// scratch in a fixed device array instead of caller-provided memory, for callers that
// cannot allocate device memory themselves.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/igamg.h"
#include "kernels.cuh"

namespace igamg {
void set_context_free_error(const std::string& msg);  // defined with igamg_last_error
}

namespace {

// Largest tile accepted: n0 * n1 <= 512 * 512.  The scratch holds two such tiles (the
// intermediate U0^T R and its product with U1), 2 * 262144 doubles = 4 MiB, and stays
// resident on every device that loads this library until the process exits.
constexpr int64_t kMaxTile = 512 * 512;
__device__ __align__(256) double g_fd_scratch[2 * kMaxTile];

// Device address of the scratch array on the current device.  In host code the name
// g_fd_scratch is only a host-side stand-in, never a device pointer, so the address is
// looked up with the device current.  The lookup runs on every call (it is cheap once the
// library's device code is loaded), so a device reset between calls, which may move the
// array, never leaves a stale address behind.
cudaError_t scratch_on_current_device(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_fd_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

igamg_status fail(igamg_status st, const std::string& msg) {
  igamg::set_context_free_error(msg);  // reported by igamg_last_error(NULL)
  return st;
}

}  // namespace

extern "C" igamg_status igamg_fd_apply_noalloc(int n0, int n1, const double* U0, const double* U1,
                                                const double* Dinv, const double* R, int ldr, double tau,
                                                double* Z, int ldz, void* cuda_stream) {
  using namespace igamg;
  if (n0 < 1 || n1 < 1 || ldr < n1 || ldz < n1 || !U0 || !U1 || !Dinv || !R || !Z)
    return fail(IGAMG_ERR_ARG, "igamg_fd_apply_noalloc: sizes must be >= 1, strides >= n1, pointers non-NULL");
  if (int64_t(n0) * n1 > kMaxTile)
    return fail(IGAMG_ERR_ARG, "igamg_fd_apply_noalloc: n0*n1 = " + std::to_string(int64_t(n0) * n1) +
                                   " exceeds the fixed scratch limit of 262144 (512 x 512); use igamg_fd_apply");
  double* T = nullptr;
  cudaError_t e = scratch_on_current_device(&T);
  if (e != cudaSuccess)
    return fail(IGAMG_ERR_CUDA, std::string("igamg_fd_apply_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  double* Y = T + int64_t(n0) * n1;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // Every element of T and Y is written before it is read, so the contents left by an
  // earlier call never matter and nothing needs clearing.
  // the four products in order; a failed launch stops the sequence, so no later product reads
  // scratch that was not written
  const GemmDesc g[4] = {GemmDesc{U0, R, T, nullptr, n0, ldr, n1, 0, n0, n1, n0},
                         GemmDesc{T, U1, Y, Dinv, n1, n1, n1, n1, n0, n1, n1},
                         GemmDesc{U0, Y, T, nullptr, n0, n1, n1, 0, n0, n1, n0},
                         GemmDesc{T, U1, Z, nullptr, n1, n1, ldz, 0, n0, n1, n1}};
  const bool ta[4] = {true, false, false, false}, tb[4] = {false, false, false, true};
  const int epi[4] = {EPI_STORE, EPI_MUL, EPI_STORE, EPI_ASSIGN};
  for (int k = 0; k < 4; ++k) {
    const cudaError_t x = launch_gemm_one(s, g[k], ta[k], tb[k], epi[k], k == 3 ? tau : 1.0);
    if (x != cudaSuccess)
      return fail(IGAMG_ERR_CUDA, std::string("igamg_fd_apply_noalloc: launch: ") + cudaGetErrorString(x));
  }
  return IGAMG_OK;
}
