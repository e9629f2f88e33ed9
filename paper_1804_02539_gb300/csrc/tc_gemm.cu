// Tensor-core (tcgen05) GEMMs for the fast-diagonalisation contractions of the smoother.
//
//   C = A B   with A a constant matrix (an FD basis U or U^T, sliced at setup) and B a
//   varying operand (the residual tile or an intermediate), M x N x K.
//
// S == 1: BF16 operands, FP32 accumulation in TMEM (the BF16 precision variant).
// S == 7: FP64-accurate product from BF16 digit slices (the error-free splitting scheme of
//   Ozaki et al.): every row i of A is written as 2^{sigma_i} sum_s A_s 2^{-7s} and every
//   column j of B as 2^{tau_j} sum_t B_t 2^{-7t}, with integer digits |A_s|, |B_t| <= 127
//   (exact in BF16).  Every product A_s B_t is exact in FP32 (|A_s B_t| < 2^14); the pairs
//   with s + t = q accumulate into TMEM accumulator q, and the epilogue forms
//       C_ij = 2^{sigma_i + tau_j} sum_{q=2..S+1} D_q(i,j) 2^{-7q}
//   (pairs with s + t > S + 1 are below 2^{-49} of the row and column maxima and are
//   dropped).  An accumulator stays an exact integer while its partial sums are below
//   2^24, which the worst case guarantees for (q - 1) K 127^2 < 2^24; beyond that FP32
//   rounds by at most 2^-24 of the partial sum, i.e. by < 2^{-24 - 7(q-2)} relative to the
//   leading diagonal's scale, which for K <= kTcMaxK stays at or below the 2^-49 digit
//   truncation for the diagonals where it can occur (q >= 5 at K > 255).
//
// The epilogue recombines the diagonals in 64-bit integers (units of 2^-49 of the row and
// column scales), converts once to FP64 and applies the smoother's epilogue.
//
// Two kernels per product set.
//   Digit pass (k_tc_digits): one CTA per 32-column panel of B (per descriptor), one warp
//   per 4 columns; the warp loads its columns over all of K (up to 288 rows at once, held in
//   registers), reduces the column exponents tau_j with shuffles and writes, per K block, the
//   digit planes in the canonical no-swizzle K-major core-matrix layout of an MMA operand.
//   Every element of B is sliced once per launch, however many row tiles read it.
//   GEMM (k_gemm_tc, persistent, warp-specialised): one CTA per SM walks the tiles (128 rows
//   of A x TBN columns of B over every descriptor of the batch) with a static stride;
//     warp 0       bulk TMA copies of A's pre-sliced K blocks ([S][128 x 32]) and of B's
//                  digit-plane blocks ([S][TBN x 32]) into a ring of stages (one mbarrier
//                  with the expected bytes of both);
//     warp 1       one thread issues the MMAs: for digit slice A_s, ONE MMA with the digit
//                  planes B_1..B_{8-s} stacked along N (N = (8 - s) TBN), whose output
//                  columns are exactly the accumulators of diagonals s+1 .. 8, which are
//                  contiguous in TMEM (7 MMAs per 16-wide K step instead of 28; each slice
//                  of A is read from shared memory once per K step);
//     warps 2..17  the epilogue, four warps per TMEM lane quarter (a quarter of the columns
//                  each; all 7 diagonals of a warp's columns in one round of TMEM loads).
//   Two accumulator sets in TMEM (2 x 7 x 32 of the 512 columns) let the epilogue of one
//   tile run while the MMAs of the next are issued.  Every tile runs on the tensor cores,
//   including the ragged remainders of M, N and K (padded with zero digits).
//   Synchronisation is by mbarriers only (no block barrier inside the tile loop); every wait
//   is bounded and a timeout is decided warp-uniformly, sets a shared abort flag and the
//   device error flag, and every role then leaves its loop; the MMA thread waits (bounded)
//   for its last MMAs and the TMA thread for its last copies before the TMEM is freed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "kernels.cuh"
#include "tc_gemm.cuh"

namespace igamg {

namespace {
constexpr int TBM = 128, TBK = 32;  // rows of a tile; K block of one pipeline stage
constexpr int NT = 576;             // 18 warps: TMA, MMA, 16 epilogue (4 per TMEM lane quarter)
constexpr int kEpiThreads = 512;
constexpr int kDigThreads = 256;    // digit pass: 8 warps per 32-column panel
constexpr int kDigRegBlocks = 9;    // K blocks a digit-pass lane holds in registers (288 rows; S = 7)
constexpr int WAIT_LIMIT = 1 << 24;

template <int S> struct TcCfg;
template <> struct TcCfg<7> {
  static constexpr int TBN = 32;       // columns of a tile
  static constexpr int ACC = 7 * 32;   // TMEM columns of one accumulator set (7 diagonals)
  static constexpr uint32_t TCOLS = 512;
  static constexpr int NST = 3;        // pipeline stages
};
template <> struct TcCfg<1> {
  static constexpr int TBN = 128;
  static constexpr int ACC = 128;
  static constexpr uint32_t TCOLS = 256;
  static constexpr int NST = 4;
};

template <int S>
constexpr size_t tc_smem_bytes() {
  using CF = TcCfg<S>;
  return size_t(CF::NST) * S * (TBM + CF::TBN) * TBK * 2  // A and B stages (BF16)
         + (2 * CF::NST + 8) * 8                           // mbarriers
         + 16                                              // TMEM slot, abort flag
         + 1024;                                           // alignment
}

__device__ __forceinline__ uint32_t sptr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= uint64_t((saddr >> 4) & 0x3FFF);
  d |= uint64_t(128 >> 4) << 16;              // leading byte offset: next core matrix along K
  d |= uint64_t((TBK / 8 * 128) >> 4) << 32;  // stride byte offset: next 8-row group
  d |= uint64_t(1) << 46;                     // descriptor version
  return d;
}

// element (r, k) of a [rows x 32] K-major no-swizzle tile
__device__ __forceinline__ int core_off(int r, int k) { return ((r >> 3) * (TBK / 8) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7); }

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
               :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar));
}
__device__ __forceinline__ void mbar_init(uint32_t mbar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(mbar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(mbar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t phase) {
  uint32_t done;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(done) : "r"(mbar), "r"(phase) : "memory");
  return done != 0;
}
// Bounded wait for the completion of phase `phase` of an mbarrier; gives up early when
// another role has raised the abort flag.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase, const volatile int* abort) {
  for (int it = 0; it < WAIT_LIMIT; ++it) {
    if (mbar_try(mbar, phase)) return true;
    if ((it & 1023) == 1023 && *abort) return false;
  }
  return false;
}

// Bounded wait for work this thread issued itself (its copies or MMAs), which completes
// whatever the other roles do: it does not give up on the abort flag.
__device__ __forceinline__ bool mbar_wait_own(uint32_t mbar, uint32_t phase) {
  for (int it = 0; it < WAIT_LIMIT; ++it)
    if (mbar_try(mbar, phase)) return true;
  return false;
}

__device__ __forceinline__ void tmem_ld8_issue(uint32_t ta, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(ta));
}
// Waits for all of the thread's outstanding TMEM loads (56 registers of 7 x8 loads).
__device__ __forceinline__ void tmem_ld_wait56(uint32_t (*r)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0][0]), "+r"(r[0][1]), "+r"(r[0][2]), "+r"(r[0][3]), "+r"(r[0][4]), "+r"(r[0][5]), "+r"(r[0][6]),
                 "+r"(r[0][7]), "+r"(r[1][0]), "+r"(r[1][1]), "+r"(r[1][2]), "+r"(r[1][3]), "+r"(r[1][4]), "+r"(r[1][5]),
                 "+r"(r[1][6]), "+r"(r[1][7]), "+r"(r[2][0]), "+r"(r[2][1]), "+r"(r[2][2]), "+r"(r[2][3]), "+r"(r[2][4]),
                 "+r"(r[2][5]), "+r"(r[2][6]), "+r"(r[2][7]), "+r"(r[3][0]), "+r"(r[3][1]), "+r"(r[3][2]), "+r"(r[3][3]),
                 "+r"(r[3][4]), "+r"(r[3][5]), "+r"(r[3][6]), "+r"(r[3][7]), "+r"(r[4][0]), "+r"(r[4][1]), "+r"(r[4][2]),
                 "+r"(r[4][3]), "+r"(r[4][4]), "+r"(r[4][5]), "+r"(r[4][6]), "+r"(r[4][7]), "+r"(r[5][0]), "+r"(r[5][1]),
                 "+r"(r[5][2]), "+r"(r[5][3]), "+r"(r[5][4]), "+r"(r[5][5]), "+r"(r[5][6]), "+r"(r[5][7]), "+r"(r[6][0]),
                 "+r"(r[6][1]), "+r"(r[6][2]), "+r"(r[6][3]), "+r"(r[6][4]), "+r"(r[6][5]), "+r"(r[6][6]), "+r"(r[6][7]));
}

__device__ __forceinline__ void tmem_ld16_issue(uint32_t ta, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(ta));
}
// Waits for the thread's outstanding TMEM loads; the registers are operands so that no use
// of them is scheduled before the wait.
__device__ __forceinline__ void tmem_ld_wait(uint32_t* r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]));
}

// Exponent e of |x| (x = m 2^(e-52), m < 2^53) and 53-bit integer mantissa.
__device__ __forceinline__ void split_f64(double x, int& e, uint64_t& m, bool& neg) {
  uint64_t b = uint64_t(__double_as_longlong(x));
  neg = (b >> 63) != 0;
  int eb = int((b >> 52) & 0x7FF);
  uint64_t f = b & ((uint64_t(1) << 52) - 1);
  if (eb == 0) {  // zero / subnormal: treat as the smallest normal exponent
    e = -1022;
    m = f;
  } else {
    e = eb - 1023;
    m = f | (uint64_t(1) << 52);
  }
}

// v 2^sh for an integer |v| < 2^62, rounded to nearest even like a conversion to FP64
// followed by an exact power-of-two scaling, with integer operations only (this part's FP64
// pipe is the slowest unit on the path).
__device__ __forceinline__ double scaled_i64_to_f64(long long v, int sh) {
  if (v == 0) return 0.0;
  const uint64_t sign = v < 0 ? (uint64_t(1) << 63) : 0;
  const uint64_t a = v < 0 ? uint64_t(-v) : uint64_t(v);
  int e = 63 - __clzll(a);  // leading bit position
  uint64_t m;
  if (e <= 52) {
    m = a << (52 - e);
  } else {  // drop e - 52 low bits, round to nearest even
    const int d = e - 52;
    const uint64_t rem = a & ((uint64_t(1) << d) - 1), half = uint64_t(1) << (d - 1);
    m = a >> d;
    if (rem > half || (rem == half && (m & 1))) {
      ++m;
      if (m == (uint64_t(1) << 53)) {
        m >>= 1;
        ++e;
      }
    }
  }
  const uint64_t frac = m & ((uint64_t(1) << 52) - 1);
  const int eb = e + 1023 + sh;
  if (eb > 0 && eb < 2047) return __longlong_as_double(static_cast<long long>(sign | (uint64_t(eb) << 52) | frac));
  return ldexp(__longlong_as_double(static_cast<long long>(sign | (uint64_t(e + 1023) << 52) | frac)), sh);
}

// The descriptor q holding tile t (tile prefix `start` of `batch` descriptors): the last q
// with start[q] <= t (descriptors without tiles are skipped).
__device__ __forceinline__ int tile_desc(const int* start, int batch, int t) {
  int lo = 0, hi = batch;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (start[mid] <= t) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <class TB>
__device__ __forceinline__ TB ld_b(const TB* B, int ldb, int tb, int k, int n) {
  return __ldg(tb ? B + int64_t(n) * ldb + k : B + int64_t(k) * ldb + n);
}

// BF16 bit pattern of an integer 0 <= d < 256 (exact in BF16): 2^23 + d is an FP32 whose
// low mantissa bits are d, and subtracting 2^23 leaves d exactly; its upper 16 bits are the
// BF16 encoding.  Full-rate integer and FP32 operations only.
__device__ __forceinline__ uint32_t bf16_of_small(uint32_t d) {
  return __float_as_uint(__uint_as_float(0x4B000000u | d) - 8388608.0f) >> 16;
}

// Digit planes of two FP64 values (consecutive k) against column scale tau: for plane s the
// BF16 pair (digit of x1 << 16 | digit of x0), digits of F = |x| 2^{49 - tau} < 2^49.
__device__ __forceinline__ void digit_pairs7(double x0, double x1, int tau, uint32_t* pk) {
  uint32_t hi[2], lo[2], sg[2];
  const double xs[2] = {x0, x1};
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    int e;
    uint64_t m;
    bool neg;
    split_f64(xs[u], e, m, neg);
    const int sh = (e - 52) - tau + 49;
    uint64_t F = 0;
    if (sh >= 0) F = sh < 11 ? (m << sh) : 0;  // cannot happen when |x| < 2^tau
    else if (sh > -64) F = m >> (-sh);
    hi[u] = uint32_t(F >> 28);                 // bits 28..48: digits 1..3
    lo[u] = uint32_t(F) & 0x0FFFFFFFu;         // bits 0..27: digits 4..7
    sg[u] = neg ? 0x8000u : 0u;
  }
#pragma unroll
  for (int sq = 0; sq < 7; ++sq) {
    uint32_t d0, d1;
    if (sq < 3) {
      d0 = (hi[0] >> (7 * (2 - sq))) & 127u;
      d1 = (hi[1] >> (7 * (2 - sq))) & 127u;
    } else {
      d0 = (lo[0] >> (7 * (6 - sq))) & 127u;
      d1 = (lo[1] >> (7 * (6 - sq))) & 127u;
    }
    pk[sq] = (bf16_of_small(d0) | sg[0]) | ((bf16_of_small(d1) | sg[1]) << 16);
  }
}

}  // namespace

template <int S, class TB, class TC>
__global__ void __launch_bounds__(kDigThreads) k_tc_digits(const TcDesc<TB, TC>* __restrict__ descs, int batch,
                                                           const int* __restrict__ pstart) {
  using CF = TcCfg<S>;
  constexpr int TBN = CF::TBN, BSZ = S * TBN * TBK, NG = TBN / 32;
  // K blocks held in registers at once: all of K up to 288 with S = 7 (the exponent pass and
  // the digits use one load), two blocks with S = 1 (no exponents)
  constexpr int RB = S > 1 ? kDigRegBlocks : 2;
  const int total = pstart[batch];  // panel prefix over the descriptors (tc_prefixes)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cl = 4 * warp + (lane >> 3);  // this lane's column within a 32-column group
  const int kq = lane & 7;                // K quad: k = 4 kq .. 4 kq + 3 of a block
  for (int pnl = blockIdx.x; pnl < total; pnl += gridDim.x) {
    const int q = tile_desc(pstart, batch, pnl);
    const TcDesc<TB, TC>& d = descs[q];
    const int nt = pnl - pstart[q], j0 = nt * TBN, K = d.K, N = d.N, nkb = (K + TBK - 1) / TBK;
    const TB* B = d.B;
    const int ldb = d.ldb, tb = d.tb;
    __nv_bfloat16* out = d.Bdig + int64_t(nt) * nkb * BSZ;
    const int nch = (nkb + RB - 1) / RB;  // register chunks of K blocks
    TB v[RB][NG][4];
    auto load_chunk = [&](int ch) {
#pragma unroll
      for (int b = 0; b < RB; ++b)
#pragma unroll
        for (int gq = 0; gq < NG; ++gq)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const int gk = (ch * RB + b) * TBK + 4 * kq + kk, gj = j0 + gq * 32 + cl;
            v[b][gq][kk] = (gj < N && gk < K) ? ld_b(B, ldb, tb, gk, gj) : TB(0);
          }
    };
    int tau = 0;
    if constexpr (S > 1) {
      // tau_j = 1 + the largest exponent in column j over all of K (zero columns: -1022)
      int emax = 0;
      for (int ch = 0; ch < nch; ++ch) {
        load_chunk(ch);
#pragma unroll
        for (int b = 0; b < RB; ++b)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            emax = max(emax, int((uint64_t(__double_as_longlong(double(v[b][0][kk]))) >> 52) & 0x7FF));
      }
      emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 1));
      emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 2));
      emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 4));
      tau = emax ? emax - 1023 + 1 : -1022;
      if (kq == 0 && j0 + cl < N) d.Btau[j0 + cl] = tau;
    }
    for (int ch = 0; ch < nch; ++ch) {
      if (S == 1 || nch > 1) load_chunk(ch);  // one chunk: still in registers from the tau pass
#pragma unroll
      for (int b = 0; b < RB; ++b) {
        const int kb = ch * RB + b;
        if (kb >= nkb) break;
        __nv_bfloat16* blk = out + int64_t(kb) * BSZ;
#pragma unroll
        for (int gq = 0; gq < NG; ++gq) {
          uint32_t pk[S][2];
          if constexpr (S == 1) {
            __nv_bfloat162 h0 = __floats2bfloat162_rn(float(v[b][gq][0]), float(v[b][gq][1]));
            __nv_bfloat162 h1 = __floats2bfloat162_rn(float(v[b][gq][2]), float(v[b][gq][3]));
            pk[0][0] = *reinterpret_cast<uint32_t*>(&h0);
            pk[0][1] = *reinterpret_cast<uint32_t*>(&h1);
          } else {
            uint32_t a[7], c[7];
            digit_pairs7(double(v[b][gq][0]), double(v[b][gq][1]), tau, a);
            digit_pairs7(double(v[b][gq][2]), double(v[b][gq][3]), tau, c);
#pragma unroll
            for (int sq = 0; sq < S; ++sq) {
              pk[sq][0] = a[sq];
              pk[sq][1] = c[sq];
            }
          }
#pragma unroll
          for (int sq = 0; sq < S; ++sq)
            *reinterpret_cast<uint2*>(blk + core_off(sq * TBN + gq * 32 + cl, 4 * kq)) = make_uint2(pk[sq][0], pk[sq][1]);
        }
      }
    }
  }
}

// Digit pass of stacked descriptors: one CTA per 32-fibre panel of the stacked M (fibre
// m = p F + j of patch p); 16 warps: warp w takes 4 fibres (w & 7) and the K blocks
// kb = w >> 3, (w >> 3) + 2, ... (two warps per fibre group, so that twice as many warps
// hide the latency of the integer digit arithmetic), a lane 4 consecutive k of each of its
// blocks.  The fibre exponent is the maximum over both halves (shared memory); digit planes
// go to the M-side layout [M tile][K block][S][128 x 32], exponents to Xtau[m].  A panel
// never straddles an M tile (128 is a multiple of 32).
constexpr int kDigStackThreads = 512, kDigStackRB = 5;  // K blocks a lane keeps in registers
__global__ void __launch_bounds__(kDigStackThreads) k_tc_digits_stack(const TcStack<double, double>* __restrict__ descs,
                                                                       int batch, const int* __restrict__ pstart) {
  constexpr int S = 7, ASZ = S * TBM * TBK, RB = kDigStackRB;
  __shared__ int s_emax[2][32];
  const int total = pstart[batch];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cl = 4 * (warp & 7) + (lane >> 3);  // this lane's fibre within the panel
  const int kg = warp >> 3;                      // K blocks kg, kg + 2, ...
  const int kq = lane & 7;                       // K quad: k = 4 kq .. 4 kq + 3 of a block
  for (int pnl = blockIdx.x; pnl < total; pnl += gridDim.x) {
    const int q = tile_desc(pstart, batch, pnl);
    const TcStack<double, double>& d = descs[q];
    const int M = d.P * d.F, K = d.K, nkb = (K + TBK - 1) / TBK;
    const int gm = (pnl - pstart[q]) * 32 + cl;
    const bool valid = gm < M;
    const int p = valid ? gm / d.F : 0, j = valid ? gm - p * d.F : 0;
    const double* X = valid ? d.X[p] : nullptr;
    __nv_bfloat16* out = d.Xdig + int64_t(gm / TBM) * nkb * ASZ;
    const int row = gm % TBM;
    const int mine = nkb > kg ? (nkb - kg + 1) / 2 : 0;  // K blocks of this warp
    const bool keep = mine <= RB;                        // all of them fit in registers
    double v[RB][4];
    auto load_block = [&](int b, int kb) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const int gk = kb * TBK + 4 * kq + kk;
        v[b][kk] = (valid && gk < K) ? ld_b(X, d.ldx, d.xt, gk, j) : 0.0;
      }
    };
    int emax = 0;
    for (int c0 = 0; c0 < mine; c0 += RB) {
#pragma unroll
      for (int b = 0; b < RB; ++b)
        if (c0 + b < mine) load_block(b, kg + 2 * (c0 + b));
#pragma unroll
      for (int b = 0; b < RB; ++b)
        if (c0 + b < mine)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            emax = max(emax, int((uint64_t(__double_as_longlong(v[b][kk])) >> 52) & 0x7FF));
    }
    emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 1));
    emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 2));
    emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 4));
    if (kq == 0) s_emax[kg][cl] = emax;
    __syncthreads();
    emax = max(s_emax[0][cl], s_emax[1][cl]);
    const int tau = emax ? emax - 1023 + 1 : -1022;
    if (kg == 0 && kq == 0 && valid) d.Xtau[gm] = tau;
    for (int c0 = 0; c0 < mine; c0 += RB) {
      if (!keep) {  // reload (K beyond the register blocks)
#pragma unroll
        for (int b = 0; b < RB; ++b)
          if (c0 + b < mine) load_block(b, kg + 2 * (c0 + b));
      }
#pragma unroll
      for (int b = 0; b < RB; ++b) {
        if (c0 + b >= mine) break;
        const int kb = kg + 2 * (c0 + b);
        __nv_bfloat16* blk = out + int64_t(kb) * ASZ;
        uint32_t a[7], c[7];
        digit_pairs7(v[b][0], v[b][1], tau, a);
        digit_pairs7(v[b][2], v[b][3], tau, c);
#pragma unroll
        for (int sq = 0; sq < S; ++sq)
          *reinterpret_cast<uint2*>(blk + core_off(sq * TBM + row, 4 * kq)) = make_uint2(a[sq], c[sq]);
      }
    }
    __syncthreads();  // s_emax is reused by the next panel
  }
}

// D = TcDesc: A (M side) the constant pre-sliced matrix, B (N side) the varying digit planes;
// D = TcStack (fibre-major): A the stacked fibres' digit planes, B the constant's slices.
template <int S, class TB, class TC, class D>
__global__ void __launch_bounds__(NT, 1) k_gemm_tc(const D* __restrict__ descs, int batch,
                                                 const int* __restrict__ tstart, int epi, TC alpha,
                                                 int* __restrict__ err) {
  constexpr bool FM = std::is_same<D, TcStack<TB, TC>>::value;
  using CF = TcCfg<S>;
  constexpr int TBN = CF::TBN, NST = CF::NST, ACC = CF::ACC;
  constexpr int ASZ = S * TBM * TBK, BSZ = S * TBN * TBK;  // BF16 elements of one stage
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(smem);
  __nv_bfloat16* Bs = As + NST * ASZ;
  uint64_t* bars = reinterpret_cast<uint64_t*>(Bs + NST * BSZ);
  uint64_t* full = bars;             // [NST] A and B copies landed (expect_tx)
  uint64_t* empty = full + NST;      // [NST] MMAs reading the stage done (commit)
  uint64_t* accf = empty + NST;      // [2] accumulator set complete (commit)
  uint64_t* acce = accf + 2;         // [2] accumulator set read by the epilogue (every epilogue thread)
  uint64_t* fin = acce + 2;          // [1] every MMA of this CTA done (commit)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(fin + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < NST; ++i) {
      mbar_init(sptr(full + i), 1);
      mbar_init(sptr(empty + i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(sptr(accf + i), 1);
      mbar_init(sptr(acce + i), kEpiThreads);
    }
    mbar_init(sptr(fin), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  const int total = tstart[batch];  // tile prefix over the descriptors (tc_prefixes)
  if (int(blockIdx.x) >= total) return;  // block-uniform, before any TMEM is held
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(sptr(tslot)), "r"(CF::TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  auto fail = [&](int code) {
    *abort_flag = 1;
    atomicExch(err, code);
  };

  if (warp == 0) {
    // ---------------- one bulk copy of A's pre-sliced [S][128 x 32] block and one of B's
    // digit-plane block [S][TBN x 32] per stage
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
        const int q = tile_desc(tstart, batch, t);
        const D& d = descs[q];
        const int tiles_n = (d.N + TBN - 1) / TBN, r = t - tstart[q], mt = r / tiles_n, nt = r % tiles_n;
        const int nkb = (d.K + TBK - 1) / TBK;
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int st = int(g % NST);
          if (g >= NST && !mbar_wait(sptr(empty + st), (g / NST - 1) & 1u, abort_flag)) {
            fail(1);
            ok = false;
            break;
          }
          const uint32_t abytes = uint32_t(ASZ) * 2u, bbytes = uint32_t(BSZ) * 2u;
          const __nv_bfloat16 *asrc, *bsrc;
          if constexpr (FM) {
            asrc = d.Xdig + (int64_t(mt) * nkb + kb) * ASZ;
            bsrc = d.Wslices + (int64_t(nt) * nkb + kb) * BSZ;
          } else {
            asrc = d.Aslices + (int64_t(mt) * d.nkb + kb) * ASZ;
            bsrc = d.Bdig + (int64_t(nt) * nkb + kb) * BSZ;
          }
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(sptr(full + st)),
                       "r"(abytes + bbytes));
          asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                       :: "r"(sptr(As + st * ASZ)), "l"(asrc), "r"(abytes), "r"(sptr(full + st)) : "memory");
          asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                       :: "r"(sptr(Bs + st * BSZ)), "l"(bsrc), "r"(bbytes), "r"(sptr(full + st)) : "memory");
        }
      }
      // the copies of the last stages (the latest use of each) have landed before the CTA
      // may exit, also after an abort
      for (uint32_t h = g > NST ? g - NST : 0; h < g; ++h) mbar_wait_own(sptr(full + h % NST), (h / NST) & 1u);
    }
  } else if (warp == 1) {
    // ---------------- MMA issue (one thread)
    if (lane == 0) {
      uint32_t g = 0;
      int i = 0;
      bool ok = true, any = false;
      constexpr uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(TBM >> 4) << 24);
      for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++i) {
        const int q = tile_desc(tstart, batch, t);
        const int K = descs[q].K;
        const int nkb = (K + TBK - 1) / TBK;
        const int b = i & 1;
        if (i >= 2 && !mbar_wait(sptr(acce + b), ((i >> 1) - 1) & 1u, abort_flag)) {
          fail(1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t acc0 = tmem + uint32_t(b * ACC);
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int st = int(g % NST);
          if (!mbar_wait(sptr(full + st), (g / NST) & 1u, abort_flag)) {
            fail(2);
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const bool two = K - kb * TBK > 16;  // second 16-wide K step of this block present
          const uint64_t a0 = smem_desc(sptr(As + st * ASZ)), b0 = smem_desc(sptr(Bs + st * BSZ));
#pragma unroll
          for (int kk = 0; kk < TBK / 16; ++kk) {
            if (kk > 0 && !two) continue;
            if constexpr (S == 1) {
              mma_bf16(acc0, a0 + uint64_t(kk * 16), b0 + uint64_t(kk * 16), idesc0 | (uint32_t(TBN >> 3) << 17),
                       (kb > 0 || kk > 0) ? 1u : 0u);
            } else {
#pragma unroll
              for (int sa = 1; sa <= S; ++sa) {
                // slice A_sa times the planes B_1..B_{8-sa} stacked along N: the outputs are
                // the accumulators of diagonals sa+1 .. S+1, contiguous from column (sa-1) TBN
                const uint32_t n = uint32_t(S + 1 - sa) * TBN;
                const uint64_t da = a0 + uint64_t(((sa - 1) * TBM * TBK * 2) >> 4) + uint64_t(kk * 16);
                // the first MMA of a tile (slice 1 spans every accumulator) overwrites
                mma_bf16(acc0 + uint32_t((sa - 1) * TBN), da, b0 + uint64_t(kk * 16), idesc0 | ((n >> 3) << 17),
                         (kb > 0 || kk > 0 || sa > 1) ? 1u : 0u);
              }
            }
          }
          mma_commit(sptr(empty + st));
          any = true;
        }
        if (!ok) break;
        mma_commit(sptr(accf + b));
      }
      // every MMA this thread issued is complete before the accumulators are released
      if (any) {
        mma_commit(sptr(fin));
        mbar_wait_own(sptr(fin), 0u);
      }
    }
  } else {
    // ---------------- epilogue: four warps per TMEM lane quarter (a quarter of the tile's
    // columns each), one row per lane
    using TA = typename std::conditional<S == 1, float, double>::type;  // epilogue arithmetic
    const int ew = warp - 2, quarter = warp & 3, part = ew >> 2;
    constexpr int CW = TBN / 4;  // columns of one epilogue warp
    int i = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x, ++i) {
      const int q = tile_desc(tstart, batch, t);
      const D& d = descs[q];
      const int tiles_n = (d.N + TBN - 1) / TBN, r = t - tstart[q];
      const int i0 = (r / tiles_n) * TBM, j0 = (r % tiles_n) * TBN;
      const int b = i & 1;
      const bool ok = mbar_wait(sptr(accf + b), (i >> 1) & 1u, abort_flag);
      if (__any_sync(0xffffffffu, !ok)) {
        fail(1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int gi = i0 + quarter * 32 + lane;
      int rows, sig = 0;
      if constexpr (FM) rows = d.P * d.F;
      else rows = d.M;
      if constexpr (S > 1) {
        if (gi < rows) {
          if constexpr (FM) sig = d.Xtau[gi];
          else sig = d.Aexp[gi];
        }
      }
      int fp = 0, fj = 0;  // stacked: the lane's patch and fibre
      if constexpr (FM) {
        if (gi < rows) {
          fp = gi / d.F;
          fj = gi - fp * d.F;
        }
      }
      const uint32_t trow = tmem + (uint32_t(quarter * 32) << 16) + uint32_t(b * ACC);
      constexpr int CC = S == 1 ? 16 : 8;  // columns per chunk
#pragma unroll 1
      for (int c0 = part * CW; c0 < (part + 1) * CW; c0 += CC) {
        TA acc[CC];
        if constexpr (S == 1) {
          uint32_t rr[16];
          tmem_ld16_issue(trow + uint32_t(c0), rr);
          tmem_ld_wait(rr);
#pragma unroll
          for (int u = 0; u < 16; ++u) acc[u] = __uint_as_float(rr[u]);
        } else {
          // column scales of this chunk (loads in flight during the TMEM reads)
          int tj[8];
#pragma unroll
          const int* cexp;
          if constexpr (FM) cexp = d.Wexp;
          else cexp = d.Btau;
#pragma unroll
          for (int u = 0; u < 8; ++u) tj[u] = j0 + c0 + u < d.N ? __ldg(cexp + j0 + c0 + u) : 0;
          // the 7 diagonals of these 8 columns in one round of TMEM loads, then the exact
          // integer recombination sum_q D_q 2^{7(7-q)} (q = 2..7) plus D_8 / 2^7 in units of
          // 2^-49, and the rounding to FP64 with the power-of-two scale 2^{sigma + tau - 49}
          uint32_t rr[7][8];
#pragma unroll
          for (int dg = 0; dg < 7; ++dg) tmem_ld8_issue(trow + uint32_t(dg * TBN + c0), rr[dg]);
          tmem_ld_wait56(rr);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            long long iacc = 0;
#pragma unroll
            for (int dg = 0; dg < 7; ++dg) {
              const int qd = dg + 2;
              const long long iv = __float2int_rn(__uint_as_float(rr[dg][u]));  // |D_q| < 2^24 in practice
              iacc += qd <= 7 ? (iv << (7 * (7 - qd))) : (iv >> 7);
            }
            acc[u] = scaled_i64_to_f64(iacc, sig + tj[u] - 49);
          }
        }
        if (c0 + CC >= (part + 1) * CW) {
          // every TMEM value of this warp's columns is in registers: hand them back
          asm volatile("tcgen05.fence::before_thread_sync;");
          mbar_arrive(sptr(acce + b));
        }
        if (gi < rows) {
          // epilogue operands first (loads in flight), then the stores
          TA e[CC];
          if constexpr (FM) {
            // this lane's fibre: C and E addresses of column gj are base + gj * step
            TC* Cp = d.C[fp];
            TC* cb = d.ct ? Cp + int64_t(fj) * d.ldc : Cp + fj;
            const int64_t cst = d.ct ? 1 : d.ldc;
            const TC* eb = nullptr;
            int64_t est = 0;
            if (epi == EPI_MUL) {
              const TC* Ep = d.E[fp];
              eb = d.et ? Ep + int64_t(fj) * d.lde : Ep + fj;
              est = d.et ? 1 : d.lde;
            }
#pragma unroll
            for (int u = 0; u < CC; ++u) {
              const int gj = j0 + c0 + u;
              e[u] = TA(0);
              if (gj < d.N) {
                if (epi == EPI_MUL) e[u] = TA(eb[gj * est]);
                else if (epi == EPI_ADD) e[u] = TA(cb[gj * cst]);
              }
            }
#pragma unroll
            for (int u = 0; u < CC; ++u) {
              const int gj = j0 + c0 + u;
              if (gj >= d.N) continue;
              const TA v = acc[u];
              TC* cp = cb + gj * cst;
              switch (epi) {
                case EPI_MUL: *cp = TC(v * e[u]); break;
                case EPI_ASSIGN: *cp = TC(TA(alpha) * v); break;
                case EPI_ADD: *cp = TC(fma(TA(alpha), v, e[u])); break;
                default: *cp = TC(v);
              }
            }
          } else {
            const bool needs = epi == EPI_MUL || epi == EPI_ADD;
#pragma unroll
            for (int u = 0; u < CC; ++u) {
              const int gj = j0 + c0 + u;
              e[u] = TA(0);
              if (needs && gj < d.N) {
                if (epi == EPI_MUL) e[u] = TA(d.E[d.tc ? int64_t(gj) * d.lde + gi : int64_t(gi) * d.lde + gj]);
                else e[u] = TA(d.C[d.tc ? int64_t(gj) * d.ldc + gi : int64_t(gi) * d.ldc + gj]);
              }
            }
#pragma unroll
            for (int u = 0; u < CC; ++u) {
              const int gj = j0 + c0 + u;
              if (gj >= d.N) continue;
              const TA v = acc[u];
              TC* cp = d.C + (d.tc ? int64_t(gj) * d.ldc + gi : int64_t(gi) * d.ldc + gj);
              switch (epi) {
                case EPI_MUL: *cp = TC(v * e[u]); break;
                case EPI_ASSIGN: *cp = TC(TA(alpha) * v); break;
                case EPI_ADD: *cp = TC(fma(TA(alpha), v, e[u])); break;
                default: *cp = TC(v);
              }
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(CF::TCOLS));
}

namespace {
int sm_count() {
  static std::mutex mu;
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  std::lock_guard<std::mutex> lk(mu);
  if (!cache[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    cache[dev] = n;
  }
  return cache[dev];
}
}  // namespace

template <int S, class TB, class TC>
cudaError_t launch_tc_digits(cudaStream_t s, const TcDesc<TB, TC>* d_desc, int batch, const int* panel_start,
                             int64_t panels) {
  if (batch <= 0 || panels <= 0) return cudaSuccess;
  const int grid = int(std::min<int64_t>(panels, 4 * int64_t(sm_count())));
  k_tc_digits<S, TB, TC><<<grid, kDigThreads, 0, s>>>(d_desc, batch, panel_start);
  return cudaGetLastError();
}

template <int S, class TB, class TC>
cudaError_t launch_gemm_tc(cudaStream_t s, const TcDesc<TB, TC>* d_desc, int batch, const int* tile_start,
                           int64_t tiles, int epi, TC alpha, int* err) {
  if (batch <= 0 || tiles <= 0) return cudaSuccess;
  const size_t smem = tc_smem_bytes<S>();
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(k_gemm_tc<S, TB, TC, TcDesc<TB, TC>>), smem);
  if (e != cudaSuccess) return e;
  // persistent CTAs, at most one per SM: the fewest that give every CTA the same largest
  // number of tiles as one per SM would, so that SMs left over serve the work running
  // concurrently on the interface stream
  const int64_t nsm = sm_count(), per = (tiles + nsm - 1) / nsm;
  const int grid = int(std::min<int64_t>((tiles + per - 1) / per, nsm));
  k_gemm_tc<S, TB, TC, TcDesc<TB, TC>><<<grid, NT, smem, s>>>(d_desc, batch, tile_start, epi, alpha, err);
  return cudaGetLastError();
}

cudaError_t launch_gemm_tc_stack(cudaStream_t s, const TcStack<double, double>* d_desc, int batch,
                                 const int* tile_start, int64_t tiles, int epi, double alpha, int* err) {
  if (batch <= 0 || tiles <= 0) return cudaSuccess;
  using SD = TcStack<double, double>;
  const size_t smem = tc_smem_bytes<7>();
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(k_gemm_tc<7, double, double, SD>), smem);
  if (e != cudaSuccess) return e;
  const int64_t nsm = sm_count(), per = (tiles + nsm - 1) / nsm;
  const int grid = int(std::min<int64_t>((tiles + per - 1) / per, nsm));
  k_gemm_tc<7, double, double, SD><<<grid, NT, smem, s>>>(d_desc, batch, tile_start, epi, alpha, err);
  return cudaGetLastError();
}

cudaError_t launch_tc_digits_stack(cudaStream_t s, const TcStack<double, double>* d_desc, int batch,
                                   const int* panel_start, int64_t panels) {
  if (batch <= 0 || panels <= 0) return cudaSuccess;
  const int grid = int(std::min<int64_t>(panels, 4 * int64_t(sm_count())));
  k_tc_digits_stack<<<grid, kDigStackThreads, 0, s>>>(d_desc, batch, panel_start);
  return cudaGetLastError();
}

void tc_stack_prefixes(const std::vector<TcStack<double, double>>& h, std::vector<int>& tile_start,
                       std::vector<int>& panel_start) {
  tile_start.assign(h.size() + 1, 0);
  panel_start.assign(h.size() + 1, 0);
  for (size_t q = 0; q < h.size(); ++q) {
    const int64_t M = int64_t(h[q].P) * h[q].F;
    const bool any = M > 0 && h[q].N > 0 && h[q].K > 0;
    tile_start[q + 1] = tile_start[q] + (any ? int(tc_tiles(int(M), h[q].N, 7)) : 0);
    panel_start[q + 1] = panel_start[q] + (any ? int((M + 31) / 32) : 0);
  }
}

int64_t tc_stack_dig_elems(int P, int F, int K) {
  const int64_t M = int64_t(P) * F;
  if (M <= 0 || K <= 0) return 0;
  return (M + TBM - 1) / TBM * ((K + TBK - 1) / TBK) * 7 * TBM * TBK;
}

double tc_stack_exec_flops(int P, int F, int N, int K) { return tc_exec_flops(P * F, N, K, 7); }
template cudaError_t launch_tc_digits<7, double, double>(cudaStream_t, const TcDesc<double, double>*, int, const int*,
                                                         int64_t);
template cudaError_t launch_tc_digits<1, float, float>(cudaStream_t, const TcDesc<float, float>*, int, const int*,
                                                       int64_t);
template cudaError_t launch_gemm_tc<7, double, double>(cudaStream_t, const TcDesc<double, double>*, int, const int*,
                                                       int64_t, int, double, int*);
template cudaError_t launch_gemm_tc<1, float, float>(cudaStream_t, const TcDesc<float, float>*, int, const int*, int64_t,
                                                     int, float, int*);

template <class TB, class TC>
void tc_prefixes(const std::vector<TcDesc<TB, TC>>& h, int S, std::vector<int>& tile_start,
                 std::vector<int>& panel_start) {
  const int tbn = S == 1 ? TcCfg<1>::TBN : TcCfg<7>::TBN;
  tile_start.assign(h.size() + 1, 0);
  panel_start.assign(h.size() + 1, 0);
  for (size_t q = 0; q < h.size(); ++q) {
    const bool any = h[q].M > 0 && h[q].N > 0 && h[q].K > 0;
    tile_start[q + 1] = tile_start[q] + (any ? int(tc_tiles(h[q].M, h[q].N, S)) : 0);
    panel_start[q + 1] = panel_start[q] + (any ? (h[q].N + tbn - 1) / tbn : 0);
  }
}
template void tc_prefixes<double, double>(const std::vector<TcDesc<double, double>>&, int, std::vector<int>&,
                                          std::vector<int>&);
template void tc_prefixes<float, float>(const std::vector<TcDesc<float, float>>&, int, std::vector<int>&,
                                        std::vector<int>&);

int64_t tc_tiles(int M, int N, int S) {
  if (M <= 0 || N <= 0) return 0;
  const int tbn = S == 1 ? TcCfg<1>::TBN : TcCfg<7>::TBN;
  return int64_t((M + TBM - 1) / TBM) * ((N + tbn - 1) / tbn);
}

namespace {
uint16_t bf16_bits_rn(float f) {
  uint32_t b;
  std::memcpy(&b, &f, 4);
  uint32_t r = b + 0x7FFFu + ((b >> 16) & 1u);
  return uint16_t(r >> 16);
}
}  // namespace

int tc_kblocks(int K) { return (K + TBK - 1) / TBK; }

int64_t tc_dig_elems(int N, int K, int S) {
  if (N <= 0 || K <= 0) return 0;
  const int tbn = S == 1 ? TcCfg<1>::TBN : TcCfg<7>::TBN;
  return int64_t((N + tbn - 1) / tbn) * ((K + TBK - 1) / TBK) * S * tbn * TBK;
}

double tc_exec_flops(int M, int N, int K, int S) {
  if (M <= 0 || N <= 0 || K <= 0) return 0.0;
  const int tbn = S == 1 ? TcCfg<1>::TBN : TcCfg<7>::TBN;
  const double tiles = double((M + TBM - 1) / TBM) * ((N + tbn - 1) / tbn);
  const int pairs = S == 1 ? 1 : S * (S + 1) / 2;  // digit-slice pairs (N-stacked MMAs)
  double ksteps = 0;
  for (int k0 = 0; k0 < K; k0 += TBK) ksteps += std::min(TBK, K - k0 + 15) / 16;
  return tiles * pairs * ksteps * 2.0 * TBM * tbn * 16;
}

void slice_constant(const std::vector<double>& A, int M, int K, int S, std::vector<uint16_t>& slices,
                    std::vector<int>& exps, int tile_rows) {
  const int R = tile_rows, mt = (M + R - 1) / R, nkb = (K + TBK - 1) / TBK;
  slices.assign(size_t(mt) * nkb * S * R * TBK, 0);
  exps.assign(M, 0);
  for (int i = 0; i < M; ++i) {
    double mx = 0.0;
    for (int k = 0; k < K; ++k) mx = std::max(mx, std::fabs(A[size_t(i) * K + k]));
    int e = -1022;
    if (mx > 0) std::frexp(mx, &e);  // mx = f 2^e, f in [0.5, 1): |a| < 2^e
    exps[i] = e;
    for (int k = 0; k < K; ++k) {
      double a = A[size_t(i) * K + k];
      size_t base = ((size_t(i / R) * nkb + k / TBK) * S) * R * TBK;
      int r = i % R, kk = k % TBK;
      size_t off = size_t(((r >> 3) * (TBK / 8) + (kk >> 3)) * 64 + (r & 7) * 8 + (kk & 7));
      if (S == 1) {
        slices[base + off] = bf16_bits_rn(float(a));
        continue;
      }
      double F = std::floor(std::ldexp(std::fabs(a), 7 * S - e));  // < 2^(7S), exact
      uint64_t Fi = uint64_t(F);
      for (int s = 1; s <= S; ++s) {
        float dgt = float((Fi >> (7 * (S - s))) & 127u);
        if (a < 0) dgt = -dgt;
        slices[base + size_t(s - 1) * R * TBK + off] = bf16_bits_rn(dgt);
      }
    }
  }
}

}  // namespace igamg
