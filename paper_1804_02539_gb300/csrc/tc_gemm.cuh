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

// Fibre-major stacked product (FP64, S = 7): the varying operand on the MMA's M side.  For
// each of P patches p sharing one constant W (N x K, sliced at setup in 32-row tiles):
//   C_p(i, j) = sum_k W(i, k) X_p(k, j),   i < N, j < F,
// X_p(k, j) = xt ? X_p[j * ldx + k] : X_p[k * ldx + j],  C_p(i, j) = ct ? C_p[j * ldc + i]
// : C_p[i * ldc + j], E_p(i, j) likewise with et and lde (EPI_MUL operand).  The P F fibres
// are stacked along M, so the 128-row MMA tiles are padded once per set instead of once per
// patch, and an epilogue lane owns one fibre (ct = 0 stores are coalesced).
template <class TB, class TC>
struct TcStack {
  const __nv_bfloat16* Wslices;  // [N/32 tiles][K blocks][S][32 x 32] in core-matrix layout
  const int* Wexp;               // [N] row scale exponents of W
  const TB* const* X;            // [P] varying operands
  TC* const* C;                  // [P] outputs
  const TC* const* E;            // [P] EPI_MUL operands (may be NULL when unused)
  int ldx, xt, ldc, ct, lde, et;
  int P, F, N, K;
  // scratch written by the digit pass and read by the GEMM: the stacked fibres' digit planes
  // [ceil(P F / 128)][K blocks][S][128 x 32] and their exponents [P F]
  __nv_bfloat16* Xdig = nullptr;
  int* Xtau = nullptr;
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
// The same two launches for stacked descriptors (S = 7, TB = TC = double): panels are 32-fibre
// groups of the stacked M, tiles 128 fibres x 32 rows of W.
cudaError_t launch_tc_digits_stack(cudaStream_t s, const TcStack<double, double>* d_desc, int batch,
                                   const int* panel_start, int64_t panels);
cudaError_t launch_gemm_tc_stack(cudaStream_t s, const TcStack<double, double>* d_desc, int batch,
                                 const int* tile_start, int64_t tiles, int epi, double alpha, int* err);
void tc_stack_prefixes(const std::vector<TcStack<double, double>>& h, std::vector<int>& tile_start,
                       std::vector<int>& panel_start);
// Scratch of one stacked descriptor (BF16 elements of Xdig; ints of Xtau = P F), and the
// BF16 MMA FLOPs one launch issues for it.
int64_t tc_stack_dig_elems(int P, int F, int K);
double tc_stack_exec_flops(int P, int F, int N, int K);
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
// tile_rows = 128 gives TcDesc::Aslices (the M side), 32 gives TcStack::Wslices (the N side).
void slice_constant(const std::vector<double>& A, int M, int K, int S, std::vector<uint16_t>& slices,
                    std::vector<int>& exps, int tile_rows = 128);

}  // namespace igamg
