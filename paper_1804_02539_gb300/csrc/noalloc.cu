// igamg_fd_apply_noalloc: the fast-diagonalisation apply of igamg_fd_apply, with its
// scratch in a fixed device array instead of caller-provided memory, for callers that
// cannot allocate device memory themselves.
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
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

std::mutex g_mu;
std::map<int, double*> g_scratch_addr;  // device ordinal -> device address of g_fd_scratch

// Device address of the scratch array on the current device.  In host code the name
// g_fd_scratch is only a host-side stand-in, never a device pointer, so the address is
// looked up once per device (with that device current) and cached.
cudaError_t scratch_on_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_scratch_addr.find(dev);
  if (it != g_scratch_addr.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_fd_scratch);
  if (e != cudaSuccess) return e;
  g_scratch_addr[dev] = static_cast<double*>(p);
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
  cudaError_t r[4];
  r[0] = launch_gemm_one(s, GemmDesc{U0, R, T, nullptr, n0, ldr, n1, 0, n0, n1, n0}, true, false, EPI_STORE, 1.0);
  r[1] = launch_gemm_one(s, GemmDesc{T, U1, Y, Dinv, n1, n1, n1, n1, n0, n1, n1}, false, false, EPI_MUL, 1.0);
  r[2] = launch_gemm_one(s, GemmDesc{U0, Y, T, nullptr, n0, n1, n1, 0, n0, n1, n0}, false, false, EPI_STORE, 1.0);
  r[3] = launch_gemm_one(s, GemmDesc{T, U1, Z, nullptr, n1, n1, ldz, 0, n0, n1, n1}, false, true, EPI_ASSIGN, tau);
  for (cudaError_t x : r)
    if (x != cudaSuccess)
      return fail(IGAMG_ERR_CUDA, std::string("igamg_fd_apply_noalloc: launch: ") + cudaGetErrorString(x));
  return IGAMG_OK;
}
