// Tensor-core (tcgen05) GEMMs for the fast-diagonalisation contractions of the smoother.
//
//   C = A B   with A a constant matrix (an FD basis U or U^T, sliced at setup) and B a
//   varying operand (the residual tile or an intermediate), M x N x K.
//
// S == 1: BF16 operands, FP32 accumulation in TMEM (the BF16 precision variant).
// S == 7: FP64-accurate product from BF16 digit slices (the error-free splitting scheme of
//   Ozaki et al.): every row i of A is written as 2^{sigma_i} sum_s A_s 2^{-7s} and every
//   column j of B as 2^{tau_j} sum_t B_t 2^{-7t}, with integer digits |A_s|, |B_t| <= 127
//   (exact in BF16).  A digit product summed over K <= 1023 stays below 2^24, so each
//   tcgen05.mma of one slice pair is exact in FP32; the pairs with s + t = q accumulate
//   into TMEM accumulator q, and the epilogue forms
//       C_ij = 2^{sigma_i + tau_j} sum_{q=2..S+1} D_q(i,j) 2^{-7q}
//   in FP64 (pairs with s + t > S + 1 are below 2^{-56} relative and are dropped).
//
// The epilogue recombines the diagonals exactly in 64-bit integers (units of 2^-49 of the
// row and column scales), converts once to FP64 and applies the smoother's epilogue.
//
// Block: 512 threads (16 warps, 4 per TMEM lane quarter), one 128 x 64 output tile.  A
// pre-pass finds the column exponents of the tile's 64-column panel.  Then a two-stage
// pipeline over K blocks of 32: A's slices, pre-arranged on the host in the canonical
// no-swizzle K-major layout (core matrices of 8 rows x 16 bytes; LBO = 128 B between core
// matrices along K, SBO = 512 B between 8-row groups), arrive by one bulk TMA copy per
// stage; B's digits are produced by all threads from register-prefetched operands; one
// thread issues the MMAs of a block and commits them to the stage's mbarrier while the
// others stage the next block.  Every mbarrier wait is bounded.  Tiles with at most 32
// valid rows or columns skip the tensor cores and use FMAs on the FP64 basis; such tiles
// are scheduled after the full ones.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "kernels.cuh"
#include "tc_gemm.cuh"

namespace igamg {

namespace {
constexpr int TBM = 128, TBN = 64, TBK = 32;  // K block of one pipeline stage
constexpr int NT = 512;  // threads per CTA: 16 warps, 4 per TMEM lane quarter
constexpr int WAIT_LIMIT = 1 << 24;
constexpr int kLightRows = 32;  // a tile with this few valid rows or columns skips the tensor cores

__device__ __forceinline__ uint32_t sptr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= uint64_t((saddr >> 4) & 0x3FFF);
  d |= uint64_t(128 >> 4) << 16;   // leading byte offset: next core matrix along K
  d |= uint64_t((TBK / 8 * 128) >> 4) << 32;  // stride byte offset: next 8-row group
  d |= uint64_t(1) << 46;          // descriptor version
  return d;
}

// element (r, k) of a [rows x 64] K-major no-swizzle tile
__device__ __forceinline__ int core_off(int r, int k) { return ((r >> 3) * (TBK / 8) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7); }

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
               :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  uint32_t done = 0;
  for (int it = 0; it < WAIT_LIMIT && !done; ++it)
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(mbar), "r"(phase));
  return done != 0;
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

template <int S>
__device__ __forceinline__ void digits_f64(double x, int tau, float* dig) {
  int e;
  uint64_t m;
  bool neg;
  split_f64(x, e, m, neg);
  // fixed point F = |x| 2^{7S - tau}, |x| = m 2^{e - 52}
  int sh = (e - 52) - tau + 7 * S;
  uint64_t F = 0;
  if (sh >= 0) F = sh < 11 ? (m << sh) : 0;  // cannot happen when |x| < 2^tau
  else if (sh > -64) F = m >> (-sh);
#pragma unroll
  for (int s = 1; s <= S; ++s) {
    float d = float(uint32_t(F >> (7 * (S - s))) & 127u);
    dig[s - 1] = neg ? -d : d;
  }
}
}  // namespace

template <int S, class TB, class TC>
__global__ void __launch_bounds__(NT, 1) k_gemm_tc(const TcDesc<TB, TC>* __restrict__ descs, int epi, TC alpha,
                                                 int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // two pipeline stages, each [S][128 x TBK] of A and [S][64 x TBK] of B
  constexpr int ASZ = S * TBM * TBK, BSZ = S * TBN * TBK;
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(smem);
  __nv_bfloat16* Bs = As + 2 * ASZ;
  int* tauS = reinterpret_cast<int*>(Bs + 2 * BSZ);                           // [64]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(tauS + TBN);                    // [2] MMAs of a stage done
  uint64_t* abar = mbar + 2;                                                  // [2] A bulk copy landed
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 4);
  const TcDesc<TB, TC> d = descs[blockIdx.x];
  // tile blockIdx.y of this product; the tiles that run on the tensor cores come first, so
  // that (with the batch as the fastest grid dimension) they fill the first waves and the
  // light tiles (few valid rows or columns, FMA path) the remainder
  const int tiles_m = (d.M + TBM - 1) / TBM, tiles_n = (d.N + TBN - 1) / TBN;
  int t = blockIdx.y;
  if (t >= tiles_m * tiles_n) return;
  int Mh = tiles_m, Nh = tiles_n;
  if (d.Af) {
    Mh = d.M / TBM + (d.M % TBM > kLightRows ? 1 : 0);
    Nh = d.N / TBN + (d.N % TBN > kLightRows ? 1 : 0);
  }
  int mt, nt;
  if (t < Mh * Nh) {
    mt = t / Nh;
    nt = t % Nh;
  } else {  // the k-th light tile in row-major order
    int k = t - Mh * Nh;
    mt = 0;
    nt = 0;
    for (int q = 0; q < tiles_m * tiles_n; ++q) {
      const int a = q / tiles_n, b = q % tiles_n;
      if (a < Mh && b < Nh) continue;
      if (k-- == 0) { mt = a; nt = b; break; }
    }
  }
  const int i0 = mt * TBM, j0 = nt * TBN;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rows = min(TBM, d.M - i0), cols = min(TBN, d.N - j0);
  if (d.Af && (rows <= kLightRows || cols <= kLightRows)) {
    // a tile of a few remainder rows or columns: plain FMAs over K instead of MMAs on a
    // mostly empty 128 x 64 tile (this also keeps such tiles out of the waves of full ones)
    for (int o = tid; o < rows * cols; o += NT) {
      const int gi = i0 + o / cols, gj = j0 + o % cols;
      TC acc = TC(0);
      for (int k = 0; k < d.K; ++k) {
        const TC a = TC(d.tra ? d.Af[int64_t(k) * d.lda + gi] : d.Af[int64_t(gi) * d.lda + k]);
        const TC b = TC(d.tb ? d.B[int64_t(gj) * d.ldb + k] : d.B[int64_t(k) * d.ldb + gj]);
        acc = fma(a, b, acc);
      }
      TC* cp = d.C + (d.tc ? int64_t(gj) * d.ldc + gi : int64_t(gi) * d.ldc + gj);
      switch (epi) {
        case EPI_MUL: *cp = acc * d.E[d.tc ? int64_t(gj) * d.lde + gi : int64_t(gi) * d.lde + gj]; break;
        case EPI_ASSIGN: *cp = alpha * acc; break;
        case EPI_ADD: *cp = fma(alpha, acc, *cp); break;
        default: *cp = acc;
      }
    }
    return;
  }
  const int quarter = warp & 3, colgrp = warp >> 2;  // TMEM lanes 32*quarter.., columns 16*colgrp..
  constexpr int NACC = S == 1 ? 1 : S;      // accumulators: diagonals q = 2..S+1
  constexpr uint32_t TCOLS = S == 1 ? 64 : 512;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(sptr(tslot)), "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int q = 0; q < 4; ++q) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(sptr(mbar + q)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // column scales of B: tau_j = 1 + the largest exponent in column j of op(B) over all of K
  // (bit extraction; zero columns give -1022).  Every CTA of a column panel reads the panel
  // once here (L2-resident for the panel's other CTAs), eight loads in flight per thread.
  if constexpr (S > 1) {
    if (tid < TBN) tauS[tid] = 0;  // biased exponent field while reducing
    __syncthreads();
    int n, kq;
    if (d.tb) { n = tid >> 3; kq = tid & 7; }  // 8 lanes along k of one column
    else { n = tid & 63; kq = tid >> 6; }      // 32 lanes along the columns
    const int gn = j0 + n;
    int emax = 0;
    if (gn < d.N) {
      for (int k0 = kq; k0 < d.K; k0 += 64) {
        TB v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int k = k0 + 8 * u;
          v[u] = k < d.K ? __ldg(d.tb ? d.B + int64_t(gn) * d.ldb + k : d.B + int64_t(k) * d.ldb + gn) : TB(0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          emax = max(emax, int((uint64_t(__double_as_longlong(double(v[u]))) >> 52) & 0x7FF));
      }
    }
    atomicMax(&tauS[n], emax);
    __syncthreads();
    if (tid < TBN) tauS[tid] = tauS[tid] ? tauS[tid] - 1023 + 1 : -1022;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(TBN >> 3) << 17) | (uint32_t(TBM >> 4) << 24);
  const int nkb = (d.K + TBK - 1) / TBK;
  // B staging: thread -> (column bn, 4 consecutive k at bk).  Bits of tid, high to low:
  // bn / 8 (3), k chunk of 8 (2), bn % 8 (3), half chunk (1).  A half-warp stores 16
  // distinct 8-byte pieces of one 128-byte core matrix per digit plane (conflict-free), and
  // the loads are 32-byte sectors fully used for either storage order of B.
  const int bn = ((tid >> 6) << 3) | ((tid >> 1) & 7);
  const int bk = ((tid >> 4) & 3) * 8 + (tid & 1) * 4;
  const int gj = j0 + bn;
  TB xv[4];
  auto load_b = [&](int k0) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const int gk = k0 + bk + kk;
      xv[kk] = (gj < d.N && gk < d.K) ? __ldg(d.tb ? d.B + int64_t(gj) * d.ldb + gk : d.B + int64_t(gk) * d.ldb + gj)
                                      : TB(0);
    }
  };
  // digit planes of the registers into stage st of B
  auto stage_b = [&](int st) {
    uint32_t pk[S][2];
#pragma unroll
    for (int kk = 0; kk < 4; kk += 2) {
      float d0[S], d1[S];
      if constexpr (S == 1) {
        d0[0] = float(xv[kk]);
        d1[0] = float(xv[kk + 1]);
      } else {
        digits_f64<S>(double(xv[kk]), tauS[bn], d0);
        digits_f64<S>(double(xv[kk + 1]), tauS[bn], d1);
      }
#pragma unroll
      for (int q = 0; q < S; ++q) {
        __nv_bfloat162 h = __floats2bfloat162_rn(d0[q], d1[q]);
        pk[q][kk >> 1] = *reinterpret_cast<uint32_t*>(&h);
      }
    }
    const int off = core_off(bn, bk);
#pragma unroll
    for (int q = 0; q < S; ++q)
      *reinterpret_cast<uint2*>(Bs + st * BSZ + q * TBN * TBK + off) = make_uint2(pk[q][0], pk[q][1]);
  };
  // A: the pre-sliced block [S][128 x TBK] is contiguous: one bulk (TMA) copy per stage
  auto copy_a = [&](int kb, int st) {
    const uint32_t bytes = uint32_t(ASZ) * sizeof(__nv_bfloat16);
    const __nv_bfloat16* src = d.Aslices + (int64_t(mt) * d.nkb + kb) * ASZ;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(sptr(abar + st)), "r"(bytes));
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(sptr(As + st * ASZ)), "l"(src), "r"(bytes), "r"(sptr(abar + st)) : "memory");
  };
  bool ok = true;
  // prologue: stage 0 holds block 0; the registers hold block 1
  if (tid == 0) copy_a(0, 0);
  load_b(0);
  stage_b(0);
  if (nkb > 1) load_b(TBK);
  for (int kb = 0; kb < nkb && ok; ++kb) {
    const int st = kb & 1;
    const uint32_t par = uint32_t(kb >> 1) & 1u;  // completion count parity of stage st's barriers
    if (!mbar_wait(sptr(abar + st), par)) {
      ok = false;
      if (tid == 0) atomicExch(err, 2);
      break;
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const bool two = d.K - kb * TBK > 16;  // second 16-wide K step of this block present
      const uint64_t a0 = smem_desc(sptr(As + st * ASZ)), b0 = smem_desc(sptr(Bs + st * BSZ));
#pragma unroll
      for (int s = 1; s <= S; ++s)
#pragma unroll
        for (int t = 1; t + s <= (S == 1 ? 2 : S + 1); ++t) {
          const uint32_t acc_col = S == 1 ? 0 : uint32_t(s + t - 2) * TBN;
#pragma unroll
          for (int kk = 0; kk < TBK / 16; ++kk) {
            if (kk > 0 && !two) continue;
            // descriptors differ from the stage's by the operand offsets (address field, 16 B units)
            const uint64_t da = a0 + uint64_t(((s - 1) * TBM * TBK * 2) >> 4) + uint64_t(kk * 16);
            const uint64_t db = b0 + uint64_t(((t - 1) * TBN * TBK * 2) >> 4) + uint64_t(kk * 16);
            // the first contribution to accumulator s + t (pair (1, q-1), first K step)
            // overwrites it
            const uint32_t accum = (kb > 0 || kk > 0 || s > 1) ? 1u : 0u;
            mma_bf16(tmem + acc_col, da, db, idesc, accum);
          }
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(sptr(mbar + st)));
    }
    // while these MMAs run: stage the next block into the other buffers, once the MMAs
    // that read them (block kb - 1) are complete
    if (kb + 1 < nkb) {
      if (kb >= 1 && !mbar_wait(sptr(mbar + (st ^ 1)), uint32_t((kb - 1) >> 1) & 1u)) {
        ok = false;
        if (tid == 0) atomicExch(err, 1);
        break;
      }
      if (tid == 0) copy_a(kb + 1, st ^ 1);
      stage_b(st ^ 1);
      if (kb + 2 < nkb) load_b((kb + 2) * TBK);
    }
  }
  // the last commit arrives after every MMA of this thread is complete
  if (ok && !mbar_wait(sptr(mbar + ((nkb - 1) & 1)), uint32_t((nkb - 1) >> 1) & 1u)) {
    ok = false;
    if (tid == 0) atomicExch(err, 1);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    const int gi = i0 + quarter * 32 + lane;
    int sig = 0;
    if (S > 1 && gi < d.M) sig = d.Aexp[gi];
    const int c0 = colgrp * 16;
    const uint32_t trow = tmem + (uint32_t(quarter * 32) << 16) + uint32_t(c0);
    double acc[16];
    if constexpr (S == 1) {
      uint32_t r[16];
      tmem_ld16_issue(trow, r);
      tmem_ld_wait(r);
#pragma unroll
      for (int q = 0; q < 16; ++q) acc[q] = __uint_as_float(r[q]);
    } else {
      // exact integer recombination: sum_q D_q 2^{7(7-q)} (q = 2..7) plus D_8 / 2^7, in
      // units of 2^-49; |sum| < 2^58.  One int64 -> FP64 conversion, then the power-of-two
      // scale 2^{sigma + tau - 49} is added to the exponent bits.  The TMEM load of the next
      // diagonal is in flight while one is converted.
      long long iacc[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) iacc[q] = 0;
      uint32_t r[2][16];
      tmem_ld16_issue(trow, r[0]);
      tmem_ld_wait(r[0]);
#pragma unroll
      for (int dg = 0; dg < NACC; ++dg) {
        if (dg + 1 < NACC) tmem_ld16_issue(trow + uint32_t(dg + 1) * TBN, r[(dg + 1) & 1]);
        const int qd = dg + 2;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          long long iv = __float2int_rn(__uint_as_float(r[dg & 1][q]));  // exact: |D_q| < 2^24
          iacc[q] += qd <= 7 ? (iv << (7 * (7 - qd))) : (iv >> 7);
        }
        if (dg + 1 < NACC) tmem_ld_wait(r[(dg + 1) & 1]);
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        double x = __ll2double_rn(iacc[q]);
        int sh = sig + tauS[c0 + q] - 49;
        long long b = __double_as_longlong(x);
        if (x != 0.0) {
          int eb = int((b >> 52) & 0x7FF) + sh;
          x = (eb > 0 && eb < 2047) ? __longlong_as_double(b + ((long long)sh << 52)) : ldexp(x, sh);
        }
        acc[q] = x;
      }
    }
    if (gi < d.M) {
      // epilogue operands first (16 loads in flight), then the stores
      double e[16];
      const bool needs = epi == EPI_MUL || epi == EPI_ADD;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int gj = j0 + c0 + q;
        e[q] = 0.0;
        if (needs && gj < d.N) {
          if (epi == EPI_MUL) e[q] = double(d.E[d.tc ? int64_t(gj) * d.lde + gi : int64_t(gi) * d.lde + gj]);
          else e[q] = double(d.C[d.tc ? int64_t(gj) * d.ldc + gi : int64_t(gi) * d.ldc + gj]);
        }
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int gj = j0 + c0 + q;
        if (gj >= d.N) continue;
        const double v = acc[q];
        TC* cp = d.C + (d.tc ? int64_t(gj) * d.ldc + gi : int64_t(gi) * d.ldc + gj);
        switch (epi) {
          case EPI_MUL: *cp = TC(v * e[q]); break;
          case EPI_ASSIGN: *cp = TC(double(alpha) * v); break;
          case EPI_ADD: *cp = TC(fma(double(alpha), v, e[q])); break;
          default: *cp = TC(v);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TCOLS));
}

template <int S, class TB, class TC>
cudaError_t launch_gemm_tc(cudaStream_t s, const TcDesc<TB, TC>* d_desc, int batch, int maxM, int maxN, int epi,
                           TC alpha, int* err) {
  if (batch <= 0) return cudaSuccess;
  size_t smem = 2 * size_t(S) * (TBM + TBN) * TBK * sizeof(__nv_bfloat16) + TBN * sizeof(int) + 64 + 1024;
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(k_gemm_tc<S, TB, TC>), smem);
  if (e != cudaSuccess) return e;
  dim3 grid(batch, ((maxN + TBN - 1) / TBN) * ((maxM + TBM - 1) / TBM));
  k_gemm_tc<S, TB, TC><<<grid, NT, smem, s>>>(d_desc, epi, alpha, err);
  return cudaGetLastError();
}
template cudaError_t launch_gemm_tc<7, double, double>(cudaStream_t, const TcDesc<double, double>*, int, int, int, int,
                                                       double, int*);
template cudaError_t launch_gemm_tc<1, float, float>(cudaStream_t, const TcDesc<float, float>*, int, int, int, int, float,
                                                     int*);

namespace {
uint16_t bf16_bits_rn(float f) {
  uint32_t b;
  std::memcpy(&b, &f, 4);
  uint32_t r = b + 0x7FFFu + ((b >> 16) & 1u);
  return uint16_t(r >> 16);
}
}  // namespace

int tc_kblocks(int K) { return (K + TBK - 1) / TBK; }

double tc_exec_flops(int M, int N, int K, int S) {
  const double tiles = double((M + TBM - 1) / TBM) * ((N + TBN - 1) / TBN);
  const int pairs = S == 1 ? 1 : S * (S + 1) / 2;
  double ksteps = 0;
  for (int k0 = 0; k0 < K; k0 += TBK) ksteps += std::min(TBK, K - k0 + 15) / 16;
  return tiles * pairs * ksteps * 2.0 * TBM * TBN * 16;
}

void slice_constant(const std::vector<double>& A, int M, int K, int S, std::vector<uint16_t>& slices,
                    std::vector<int>& exps) {
  const int mt = (M + TBM - 1) / TBM, nkb = (K + TBK - 1) / TBK;
  slices.assign(size_t(mt) * nkb * S * TBM * TBK, 0);
  exps.assign(M, 0);
  for (int i = 0; i < M; ++i) {
    double mx = 0.0;
    for (int k = 0; k < K; ++k) mx = std::max(mx, std::fabs(A[size_t(i) * K + k]));
    int e = -1022;
    if (mx > 0) std::frexp(mx, &e);  // mx = f 2^e, f in [0.5, 1): |a| < 2^e
    exps[i] = e;
    for (int k = 0; k < K; ++k) {
      double a = A[size_t(i) * K + k];
      size_t base = ((size_t(i / TBM) * nkb + k / TBK) * S) * TBM * TBK;
      int r = i % TBM, kk = k % TBK;
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
        slices[base + size_t(s - 1) * TBM * TBK + off] = bf16_bits_rn(dgt);
      }
    }
  }
}

}  // namespace igamg
