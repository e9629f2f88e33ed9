// Tensor-core GEMMs of the smoother contractions (tcgen05, BF16 operands in shared memory,
// FP32 accumulators in TMEM): C = A B with A a constant, pre-sliced matrix and B varying.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "kernels.cuh"

namespace igamg {

template <class TB, class TC>
struct TcDesc {
  const __nv_bfloat16* Aslices;  // [M/128 tiles][K blocks][S][128 x 32] in core-matrix layout
  const int* Aexp;               // [M] row scale exponents (S > 1)
  int nkb;                       // K blocks of A (tc_kblocks(K))
  const TB* B;                   // B(k, n) = tb ? B[n * ldb + k] : B[k * ldb + n]
  int ldb, tb;
  TC* C;                         // C(i, j) at tc ? C[j * ldc + i] : C[i * ldc + j]
  int ldc, tc;
  const TC* E;                   // EPI_MUL operand, indexed like C with stride lde
  int lde;
  int M, N, K;
  // scratch written by the digit pass and read by the GEMM: B's digit planes
  // [N/TBN tiles][K blocks][S][TBN x 32] (core-matrix layout) and its column exponents [N]
  __nv_bfloat16* Bdig = nullptr;
  int* Btau = nullptr;
};

// Scratch sizes of one descriptor (BF16 elements of Bdig, ints of Btau) for S slices.
int64_t tc_dig_elems(int N, int K, int S);
inline int64_t tc_tau_elems(int N, int S) { return S > 1 ? N : 0; }

// S = 7: FP64-accurate digit-slice product (TB = TC = double), for K <= kTcMaxK (every single
// digit product summed over K stays an exact FP32 integer); S = 1: BF16 product with FP32
// accumulation (TB = TC = float).
constexpr int kTcMaxK = 1023;
// Two launches: the digit pass (B's digit planes and column exponents into Bdig/Btau, every
// element once) and the GEMM (both operands by bulk copies).  tile_start / panel_start are
// device copies of the prefixes tc_prefixes computes (batch + 1 entries), tiles / panels
// their totals.  Any number of descriptors; C must not alias B or E; the digit pass must
// have run on the same stream since B last changed.  err: device flag set when an mbarrier
// wait times out.
template <int S, class TB, class TC>
cudaError_t launch_tc_digits(cudaStream_t s, const TcDesc<TB, TC>* d_desc, int batch, const int* panel_start,
                             int64_t panels);
template <int S, class TB, class TC>
cudaError_t launch_gemm_tc(cudaStream_t s, const TcDesc<TB, TC>* d_desc, int batch, const int* tile_start,
                           int64_t tiles, int epi, TC alpha, int* err);
// Prefix sums over descriptors of their output tiles (GEMM work items) and of their
// 32-column (S = 7) or 128-column (S = 1) panels of B (digit-pass work items).
template <class TB, class TC>
void tc_prefixes(const std::vector<TcDesc<TB, TC>>& h, int S, std::vector<int>& tile_start,
                 std::vector<int>& panel_start);
// Output tiles of one M x N product (the GEMM's work items).
int64_t tc_tiles(int M, int N, int S);

// K blocks of the slice layout for inner dimension K.
int tc_kblocks(int K);
// BF16 MMA FLOPs one launch issues for an M x N x K product with S digit slices.
double tc_exec_flops(int M, int N, int K, int S);

// Host: slices of a constant row-major M x K matrix in the layout TcDesc::Aslices expects.
// S = 7 gives integer digits and the row exponents; S = 1 gives BF16 roundings.
void slice_constant(const std::vector<double>& A, int M, int K, int S, std::vector<uint16_t>& slices,
                    std::vector<int>& exps);

}  // namespace igamg
