// FP64-class tensor-core GEMM from exact BF16 digit-plane products
// (tcgen05 + TMA + TMEM, sm_103a).  The number format is described in
// gemm_oz.h.
//
// One CTA computes a 128 x 96 tile of C over its K range with 12 warps:
// warp 0 issues TMA loads of all 6 digit planes of A and B for a 32-wide K
// tile (84 KB per stage, 2 stages, 64-byte swizzle), warp 1 issues the 21
// plane products per K tile (tcgen05.mma M=128 N=96 K=16) into five TMEM
// accumulators of 96 columns, and warps 4..11 fold the accumulators into
// 64-bit integer sums held in registers (one row and 48 columns per thread)
// after every 1024 K values.  At the end the CTA writes C itself (alpha,
// beta, row and column scales) or, when K is split over several CTAs, adds
// its integer sums into a workspace that a second kernel converts.  Every wait
// is bounded by a 2-second %globaltimer budget; on expiry the kernel records
// an error code, waits (bounded) for its own copies and MMAs in flight, frees
// its TMEM and returns.
#include <algorithm>
#include <climits>
#include <cmath>
#include <mutex>

#include "fpconv.cuh"
#include "gemm_oz.h"
#include "matview.cuh"
#include "tc_ptx.cuh"

namespace ascc {
namespace oz {
namespace {

using namespace tc::ptx;

constexpr int BM = 128, BN = 96, BK = 32, STAGES = 2, NTHREADS = 384;
constexpr int NFOLD = 8;                         // fold warps: 4 lane quarters x 2 column halves
constexpr int HALF = BN / 2;                     // columns per fold thread
constexpr int PITCH = BN + 1;                    // int64 epilogue tile pitch (odd)
constexpr int KCT = 32;                          // K tiles per exact chunk (1024 K values)
constexpr int A_TILE = BM * BK * 2;              // one plane of A, 8 KB
constexpr int B_TILE = BN * BK * 2;              // one plane of B, 6 KB
constexpr int A_BYTES = NSLICE * A_TILE;         // 48 KB
constexpr int STAGE_BYTES = A_BYTES + NSLICE * B_TILE;  // 84 KB
// accumulators: exact groups s + t = 0, 1, 2, 3 and the tail 4..5 (weights
// 2^-28 and 2^-35), whose FP32 sums the tensor core truncates
constexpr int NACC = 5;
constexpr int TMEM_COLS = 512;                   // NACC * BN = 480 rounded to a power of two
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
constexpr int L = NSLICE * BETA;                 // 42 bits per scaled value
constexpr int UNIT = 4 * BETA;                   // fold unit 2^-28
static_assert(NACC * BN <= TMEM_COLS, "TMEM holds 512 columns");
static_assert(BM * PITCH * 8 <= STAGES * STAGE_BYTES, "the epilogue tile reuses the ring");
static_assert(NTHREADS % BN == 0, "whole rows per store pass");
static_assert(A_TILE % 512 == 0 && B_TILE % 512 == 0, "64-byte swizzle atoms are 512 bytes");
// |digit| <= 64, so a group of g + 1 <= 4 products sums to at most 1024 * 4 * 4096 = 2^24 per
// chunk: every partial sum is an integer multiple of 2^(-7 g) that FP32 holds exactly
static_assert((long long)KCT * BK * 4 * 64 * 64 <= (1ll << 24), "group chunk sums must stay exact");

// One element of the chunk fold, in units of 2^-28: groups 0..3 are exact
// integers (times 2^(-7 g)); the tail is rounded once to the unit.
__device__ __forceinline__ long long fold_high(uint32_t a0, uint32_t a1, uint32_t a2) {
  const long long i0 = __float2int_rn(__uint_as_float(a0));
  const long long i1 = __float2int_rn(__uint_as_float(a1) * 128.f);
  const long long i2 = __float2int_rn(__uint_as_float(a2) * 16384.f);
  return i0 * (1ll << 28) + i1 * (1ll << 21) + i2 * (1ll << 14);
}
__device__ __forceinline__ long long fold_low(uint32_t a3, uint32_t a4) {
  const long long i3 = __float2int_rn(__uint_as_float(a3) * 2097152.f);
  const long long it = __float2ll_rn(__uint_as_float(a4) * 268435456.f);
  return i3 * (1ll << 7) + it;
}

// One output of the digit products: the exact integer sum v scaled by
// 2^(a + b - 2 BETA - UNIT) (the row and column exponents), times alpha, plus
// beta times the old value.  The conversion, and for beta = 0 a power-of-two
// alpha, run in integer arithmetic with the FP64 expression's result.
__device__ __forceinline__ double digit_out(long long v, int32_t a, int32_t b, const Pow2& p2,
                                            double alpha, double beta, double old) {
  if (a == kNonFinite || b == kNonFinite) {
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    return beta == 0.0 ? alpha * nan : fma(alpha, nan, beta * old);
  }
  const int sh = a + b - (2 * BETA + UNIT);
  double val;
  if (beta == 0.0 && p2.ok && i64_to_f64_scaled(v, sh + p2.e, p2.neg, val)) return val;
  if (!i64_to_f64_scaled(v, sh, 0u, val)) val = i64_scaled_fp64(v, sh);
  return beta == 0.0 ? alpha * val : fma(alpha, val, beta * old);
}

__global__ void __launch_bounds__(NTHREADS, 1)
gemm_oz_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
               int M, int N, int num_kt, int kt_chunk, unsigned long long* __restrict__ ws,
               const int32_t* __restrict__ ea, const int32_t* __restrict__ eb, double alpha,
               double beta, double* __restrict__ C, long long ldc, int* err) {
  const Pow2 p2 = pow2_of(alpha);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint32_t* tmem_holder = (uint32_t*)(bars + 2 * STAGES + 3);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES),
                 acc_full = smem_u32(bars + 2 * STAGES), acc_empty = smem_u32(bars + 2 * STAGES + 1),
                 drained = smem_u32(bars + 2 * STAGES + 2);
  __shared__ int abort_flag;
  __shared__ int mma_consumed;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    mma_consumed = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, NFOLD * 32);
    mbar_init(drained, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_holder)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_holder;
  const int kt0 = blockIdx.z * kt_chunk;
  const int nkt = max(0, min(kt_chunk, num_kt - kt0));
  const int nchunks = (nkt + KCT - 1) / KCT;

  if (warp == 0 && lane == 0) {
    // TMA producer: all planes of A and B for one K tile per stage
    int issued = 0;
    for (int it = 0; it < nkt; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (uint32_t)((it / STAGES) & 1);
      if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, err, 11)) {
        abort_flag = 1;
        break;
      }
      if (*(volatile int*)&abort_flag) break;
      const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
      const int kx = (kt0 + it) * BK;
      mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
      tma_load_3d(sa, &amap, full0 + 8 * s, kx, m0, 0);
      tma_load_3d(sa + A_BYTES, &bmap, full0 + 8 * s, kx, n0, 0);
      issued = it + 1;
    }
    if (*(volatile int*)&abort_flag) {
      // let the copies still in flight land before the CTA exits
      const int first = max(*(volatile int*)&mma_consumed, issued - STAGES);
      for (int j = first; j < issued; ++j)
        mbar_wait(full0 + 8 * (j % STAGES), (uint32_t)((j / STAGES) & 1), err, 11);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: 21 plane products per K tile, accumulator by s + t
    constexpr uint32_t idesc = tc::ptx::idesc_bf16(BM, BN);
    for (int it = 0; it < nkt; ++it) {
      const int kc = it % KCT, chunk = it / KCT;
      if (kc == 0 && chunk > 0) {
        // the fold of the previous chunk must have drained the accumulators
        if (!mbar_wait(acc_empty, (uint32_t)((chunk - 1) & 1), err, 12)) {
          abort_flag = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      }
      const int s = it % STAGES;
      const uint32_t ph = (uint32_t)((it / STAGES) & 1);
      if (!mbar_wait(full0 + 8 * s, ph, err, 13)) {
        abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = smem_u32(smem + s * STAGE_BYTES), sb = sa + A_BYTES;
      uint32_t seen = 0;
#pragma unroll
      for (int u = 0; u < NSLICE; ++u) {
#pragma unroll
        for (int w = 0; u + w < NSLICE; ++w) {
          const int acc = min(u + w, NACC - 1);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t ad = sw64_desc(sa + u * A_TILE + kk * 32);
            const uint64_t bd = sw64_desc(sb + w * B_TILE + kk * 32);
            const uint32_t en = (kc == 0 && kk == 0 && !((seen >> acc) & 1u)) ? 0u : 1u;
            mma_bf16(tmem + (uint32_t)(acc * BN), ad, bd, idesc, en);
          }
          seen |= 1u << acc;
        }
      }
      mma_commit(empty0 + 8 * s);
      *(volatile int*)&mma_consumed = it + 1;
      if (kc == KCT - 1 || it == nkt - 1) mma_commit(acc_full);
    }
    // every MMA of this CTA has completed before TMEM is released
    mma_commit(drained);
    mbar_wait(drained, 0, err, 15);
  } else if (warp >= 4) {
    // fold: TMEM lanes [32 q, 32 q + 32) hold rows m0 + 32 q + lane; this
    // warp takes the columns [c_lo, c_lo + HALF) of them
    const int q = (warp - 4) & 3, c_lo = ((warp - 4) >> 2) * HALF;
    const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c_lo;
    long long acc[HALF];
#pragma unroll
    for (int j = 0; j < HALF; ++j) acc[j] = 0;
    bool ok_all = true;
    for (int chunk = 0; chunk < nchunks; ++chunk) {
      const bool ok = mbar_wait(acc_full, (uint32_t)(chunk & 1), err, 14);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (!__all_sync(0xffffffffu, ok) || *(volatile int*)&abort_flag) {
        abort_flag = 1;
        ok_all = false;
        break;
      }
#pragma unroll
      for (int cb = 0; cb < HALF / 8; ++cb) {
        // two passes (groups 0..2, then 3 and the tail) keep few values live
        uint32_t r0[8], r1[8], r2[8];
        tmem_ld8_nowait(taddr + 0 * BN + cb * 8, r0);
        tmem_ld8_nowait(taddr + 1 * BN + cb * 8, r1);
        tmem_ld8_nowait(taddr + 2 * BN + cb * 8, r2);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[cb * 8 + j] += fold_high(r0[j], r1[j], r2[j]);
        tmem_ld8_nowait(taddr + 3 * BN + cb * 8, r0);
        tmem_ld8_nowait(taddr + 4 * BN + cb * 8, r1);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[cb * 8 + j] += fold_low(r0[j], r1[j]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(acc_empty);
    }
    // park the integer sums in the idle ring (every MMA and copy has completed)
    if (ok_all && nchunks > 0) {
      long long* tile = reinterpret_cast<long long*>(smem);
#pragma unroll
      for (int j = 0; j < HALF; ++j) tile[(q * 32 + lane) * PITCH + c_lo + j] = acc[j];
    }
  }
  // all warps: coalesced rows of C (scale, alpha, beta) or of the split-K
  // integer workspace
  const bool go = __syncthreads_and(!*(volatile int*)&abort_flag) != 0;
  if (go && nchunks > 0) {
    const long long* tile = reinterpret_cast<const long long*>(smem);
    const int rows = min(BM, M - m0);
    constexpr int RPP = NTHREADS / BN;  // rows per pass
    const int c = threadIdx.x % BN, col = n0 + c;
    if (col < N) {
      const int32_t b = eb[col];
      if (gridDim.z == 1) {
        // RB rows per thread at a time: their row exponents and old values of
        // C are loaded before the first store (RB loads in flight, not one
        // round trip to memory per row)
        constexpr int RB = 8;
        for (int r0 = threadIdx.x / BN; r0 < rows; r0 += RB * RPP) {
          int32_t a[RB];
          double old[RB];
#pragma unroll
          for (int u = 0; u < RB; ++u) {
            const int rr = r0 + u * RPP;
            a[u] = rr < rows ? ea[m0 + rr] : 0;
            old[u] = (rr < rows && beta != 0.0) ? C[(long long)(m0 + rr) * ldc + col] : 0.0;
          }
#pragma unroll
          for (int u = 0; u < RB; ++u) {
            const int rr = r0 + u * RPP;
            if (rr < rows) {
              const long long v = tile[rr * PITCH + c];
              C[(long long)(m0 + rr) * ldc + col] =
                  digit_out(v, a[u], b, p2, alpha, beta, old[u]);
            }
          }
        }
      } else {
        for (int rr = threadIdx.x / BN; rr < rows; rr += RPP) {
          const long long v = tile[rr * PITCH + c], row = m0 + rr;
          atomicAdd(ws + row * N + col, (unsigned long long)v);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// C = alpha * 2^(e_i + f_j - 42) * ws + beta * C; NaN where a row or column
// held a non-finite value.
__global__ void oz_finish_kernel(double* __restrict__ C, long long ldc,
                                 const long long* __restrict__ ws, const int32_t* __restrict__ ea,
                                 const int32_t* __restrict__ eb, long long M, long long N,
                                 double alpha, double beta) {
  const Pow2 p2 = pow2_of(alpha);
  const long long total = M * N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long m = idx / N, n = idx % N;
    const int32_t a = ea[m], b = eb[n];
    double* c = C + m * ldc + n;
    *c = digit_out(ws[idx], a, b, p2, alpha, beta, beta != 0.0 ? *c : 0.0);
  }
}

// |x| as the integer bit pattern of a double (monotone in |x|; NaN and the
// infinities sort above every finite value).
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// rint(x 2^sh) for |x 2^sh| < 2^41 from the bits of x: integer arithmetic
// only (round half away from zero), no FP64 instruction.
__device__ __forceinline__ long long scaled_int(double x, int sh) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ef = (int)((b >> 52) & 0x7ff);
  unsigned long long m = b & 0xfffffffffffffull;
  int e2 = -1074;  // x = m 2^e2
  if (ef != 0) {
    m |= 1ull << 52;
    e2 = ef - 1075;
  }
  const int s = e2 + sh;
  long long q;
  if (s >= 0) {
    q = (long long)(m << s);  // no overflow: |q| < 2^41
  } else if (s > -64) {
    const int r = -s;
    q = (long long)((m >> r) + ((m >> (r - 1)) & 1ull));
  } else {
    q = 0;
  }
  return (b >> 63) ? -q : q;
}

// Digit split in three passes over runs of 8 values of one row (any row
// length keeps the whole GPU busy):
//  1. the largest high word of |x| per row (exponent and top mantissa bits)
//     by atomicMax into exps (as unsigned), zeroed before;
//  2. that word -> the row exponent e (max |x| < 2^(e - 1)), in place;
//  3. the balanced digits of rint(x 2^(42 - e)) in integer arithmetic,
//     16-byte stores per plane.
// A row whose largest |x| is below 2^-1054 (a subnormal with no bit in the
// high word) counts as zero.
template <typename I>
__global__ void oz_rowmax_kernel(unsigned* __restrict__ hmax, const double* __restrict__ in,
                                 long long rows, long long K, long long ld, long long Kp) {
  const I runs = (I)(Kp / 8), total = (I)rows * runs;
  for (I idx = blockIdx.x * (I)blockDim.x + threadIdx.x; idx < total;
       idx += (I)gridDim.x * blockDim.x) {
    const I rq = idx / runs;
    const long long r = rq, k0 = (long long)(idx - rq * runs) * 8;
    const double* x = in + r * ld + k0;
    unsigned m = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (k0 + j < K) m = max(m, (unsigned)(abs_bits(x[j]) >> 32));
    // one atomic per warp when its 32 runs share a row (long rows), else per run
    const unsigned active = __activemask();
    const long long r0 = __shfl_sync(active, r, __ffs(active) - 1);
    if (active == 0xffffffffu && __all_sync(active, r == r0)) {
      for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(active, m, off));
      if ((threadIdx.x & 31) == 0 && m) atomicMax(hmax + r, m);
    } else if (m) {
      atomicMax(hmax + r, m);
    }
  }
}

__global__ void oz_exponent_kernel(int32_t* __restrict__ exps, long long rows) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows;
       r += (long long)gridDim.x * blockDim.x) {
    const unsigned h = (unsigned)exps[r];
    int e = 0;
    if (h >= 0x7ff00000u) {
      e = kNonFinite;
    } else if (h >= 0x00100000u) {
      e = (int)(h >> 20) - 1021;  // normal: max |x| in [2^(E-1023), 2^(E-1022))
    } else if (h != 0) {
      e = (31 - __clz(h)) + 32 - 1072;  // subnormal: leading mantissa bit
    }
    exps[r] = e;
  }
}

template <typename I>
__global__ void oz_digits_kernel(__nv_bfloat16* __restrict__ out, const int32_t* __restrict__ exps,
                                 const double* __restrict__ in, long long rows, long long K,
                                 long long ld, long long Kp, long long plane_stride) {
  const I runs = (I)(Kp / 8), total = (I)rows * runs;
  for (I idx = blockIdx.x * (I)blockDim.x + threadIdx.x; idx < total;
       idx += (I)gridDim.x * blockDim.x) {
    const I rq = idx / runs;
    const long long r = rq, k0 = (long long)(idx - rq * runs) * 8;
    const int e = exps[r];
    const double* x = in + r * ld + k0;
    __align__(16) __nv_bfloat16 dig[NSLICE][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      long long q = 0;
      if (e != kNonFinite && k0 + j < K) q = scaled_int(x[j], L - e);  // |q| <= 2^41
#pragma unroll
      for (int s = NSLICE - 1; s >= 1; --s) {
        const long long d = ((q + 64) & 127) - 64;
        q = (q - d) >> BETA;
        dig[s][j] = __float2bfloat16_rn(ldexpf((float)d, -BETA * s));
      }
      dig[0][j] = __float2bfloat16_rn((float)q);
    }
#pragma unroll
    for (int s = 0; s < NSLICE; ++s)
      *reinterpret_cast<uint4*>(out + (long long)s * plane_stride + r * Kp + k0) =
          *reinterpret_cast<const uint4*>(dig[s]);
  }
}

// The first and third steps reading a strided tensor through a MatView.
template <typename I>
__global__ void oz_rowmax_view_kernel(unsigned* __restrict__ hmax, const double* __restrict__ in,
                                      MatView v, long long rows, long long K, long long Kp,
                                      bool fast) {
  const I runs = (I)(Kp / 8), total = (I)rows * runs;
  for (I idx = blockIdx.x * (I)blockDim.x + threadIdx.x; idx < total;
       idx += (I)gridDim.x * blockDim.x) {
    const I rq = idx / runs;
    const long long r = rq, k0 = (long long)(idx - rq * runs) * 8;
    double x[8];
    matview_run8<I>(v, in + matview_row<I>(v, rq), k0, K, fast, x);
    unsigned m = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) m = max(m, (unsigned)(abs_bits(x[j]) >> 32));
    const unsigned active = __activemask();
    const long long r0 = __shfl_sync(active, r, __ffs(active) - 1);
    if (active == 0xffffffffu && __all_sync(active, r == r0)) {
      for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(active, m, off));
      if ((threadIdx.x & 31) == 0 && m) atomicMax(hmax + r, m);
    } else if (m) {
      atomicMax(hmax + r, m);
    }
  }
}

template <typename I>
__global__ void oz_digits_view_kernel(__nv_bfloat16* __restrict__ out,
                                      const int32_t* __restrict__ exps,
                                      const double* __restrict__ in, MatView v, long long rows,
                                      long long K, long long Kp, long long plane_stride,
                                      bool fast) {
  const I runs = (I)(Kp / 8), total = (I)rows * runs;
  for (I idx = blockIdx.x * (I)blockDim.x + threadIdx.x; idx < total;
       idx += (I)gridDim.x * blockDim.x) {
    const I rq = idx / runs;
    const long long r = rq, k0 = (long long)(idx - rq * runs) * 8;
    const int e = exps[r];
    double x[8];
    matview_run8<I>(v, in + matview_row<I>(v, rq), k0, K, fast, x);
    __align__(16) __nv_bfloat16 dig[NSLICE][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      long long q = 0;
      if (e != kNonFinite && k0 + j < K) q = scaled_int(x[j], L - e);
#pragma unroll
      for (int s = NSLICE - 1; s >= 1; --s) {
        const long long d = ((q + 64) & 127) - 64;
        q = (q - d) >> BETA;
        dig[s][j] = __float2bfloat16_rn(ldexpf((float)d, -BETA * s));
      }
      dig[0][j] = __float2bfloat16_rn((float)q);
    }
#pragma unroll
    for (int s = 0; s < NSLICE; ++s)
      *reinterpret_cast<uint4*>(out + (long long)s * plane_stride + r * Kp + k0) =
          *reinterpret_cast<const uint4*>(dig[s]);
  }
}

// The first and third steps for a view whose contiguous dimension is on the
// row side: 64 x 32 tiles transposed through shared memory; thread (row mi,
// run kr) holds eight values of one row.
__global__ void __launch_bounds__(256) oz_rowmax_view_t_kernel(
    unsigned* __restrict__ hmax, const double* __restrict__ in, MatView v, long long rows,
    long long K, long long Kp) {
  __shared__ double tile[kViewTileK][kViewTileM + 1];
  __shared__ long long roff[kViewTileM], coff[kViewTileK];
  const long long ntm = (rows + kViewTileM - 1) / kViewTileM, ntk = Kp / kViewTileK;
  for (long long tix = blockIdx.x; tix < ntm * ntk; tix += gridDim.x) {
    const long long m0 = (tix / ntk) * kViewTileM, k0 = (tix % ntk) * kViewTileK;
    matview_load_tile_t(v, in, rows, K, m0, k0, tile, roff, coff);
    const int mi = threadIdx.x >> 2, kr = (threadIdx.x & 3) * 8;
    unsigned m = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) m = max(m, (unsigned)(abs_bits(tile[kr + j][mi]) >> 32));
    // the four runs of a row are neighbouring lanes
    m = max(m, __shfl_xor_sync(0xffffffffu, m, 1));
    m = max(m, __shfl_xor_sync(0xffffffffu, m, 2));
    if ((threadIdx.x & 3) == 0 && m0 + mi < rows && m) atomicMax(hmax + m0 + mi, m);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) oz_digits_view_t_kernel(
    __nv_bfloat16* __restrict__ out, const int32_t* __restrict__ exps,
    const double* __restrict__ in, MatView v, long long rows, long long K, long long Kp,
    long long plane_stride) {
  __shared__ double tile[kViewTileK][kViewTileM + 1];
  __shared__ long long roff[kViewTileM], coff[kViewTileK];
  const long long ntm = (rows + kViewTileM - 1) / kViewTileM, ntk = Kp / kViewTileK;
  for (long long tix = blockIdx.x; tix < ntm * ntk; tix += gridDim.x) {
    const long long m0 = (tix / ntk) * kViewTileM, k0 = (tix % ntk) * kViewTileK;
    matview_load_tile_t(v, in, rows, K, m0, k0, tile, roff, coff);
    const int mi = threadIdx.x >> 2, kr = (threadIdx.x & 3) * 8;
    if (m0 + mi < rows) {
      const int e = exps[m0 + mi];
      __align__(16) __nv_bfloat16 dig[NSLICE][8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        long long q = 0;
        if (e != kNonFinite) q = scaled_int(tile[kr + j][mi], L - e);
#pragma unroll
        for (int s = NSLICE - 1; s >= 1; --s) {
          const long long d = ((q + 64) & 127) - 64;
          q = (q - d) >> BETA;
          dig[s][j] = __float2bfloat16_rn(ldexpf((float)d, -BETA * s));
        }
        dig[0][j] = __float2bfloat16_rn((float)q);
      }
#pragma unroll
      for (int s = 0; s < NSLICE; ++s)
        *reinterpret_cast<uint4*>(out + (long long)s * plane_stride + (m0 + mi) * Kp + k0 + kr) =
            *reinterpret_cast<const uint4*>(dig[s]);
    }
    __syncthreads();
  }
}

CUtensorMap make_map3(const __nv_bfloat16* base, int64_t rows, int64_t Kp, int64_t plane_stride,
                      int box_rows) {
  CUtensorMap m;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)NSLICE};
  cuuint64_t strides[2] = {(cuuint64_t)(Kp * 2), (cuuint64_t)(plane_stride * 2)};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, (cuuint32_t)NSLICE};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = tc::encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base, dims, strides,
                               box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(ASCC_ERR_CUDA, "cuTensorMapEncodeTiled (digit planes) failed");
  return m;
}

int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (int)std::max<int64_t>(g, 1);
}

}  // namespace

int64_t padded_k(int64_t K) { return (K + BK - 1) / BK * BK; }

void split(cudaStream_t s, __nv_bfloat16* planes, int32_t* exps, const double* in, int64_t rows,
           int64_t K, int64_t ld, int64_t plane_stride) {
  if (rows <= 0) return;
  const int64_t Kp = padded_k(K);
  if (plane_stride <= 0) plane_stride = rows * Kp;
  const int64_t runs = rows * (Kp / 8);
  const int g = (int)std::min<int64_t>((runs + 255) / 256, 152 * 16);
  ASCC_CUDA(cudaMemsetAsync(exps, 0, sizeof(int32_t) * (size_t)rows, s));
  if (runs + 256ll * g < (1ll << 32)) {
    oz_rowmax_kernel<uint32_t><<<g, 256, 0, s>>>(reinterpret_cast<unsigned*>(exps), in, rows, K,
                                                 ld, Kp);
    oz_exponent_kernel<<<grid_for(rows), 256, 0, s>>>(exps, rows);
    oz_digits_kernel<uint32_t><<<g, 256, 0, s>>>(planes, exps, in, rows, K, ld, Kp, plane_stride);
  } else {
    oz_rowmax_kernel<long long><<<g, 256, 0, s>>>(reinterpret_cast<unsigned*>(exps), in, rows, K,
                                                  ld, Kp);
    oz_exponent_kernel<<<grid_for(rows), 256, 0, s>>>(exps, rows);
    oz_digits_kernel<long long><<<g, 256, 0, s>>>(planes, exps, in, rows, K, ld, Kp,
                                                  plane_stride);
  }
  count_launch(3);
  check_launch("oz_split");
}

void split_view(cudaStream_t s, __nv_bfloat16* planes, int32_t* exps, const double* in,
                const MatView& v, int64_t plane_stride) {
  ASCC_REQUIRE(v.nm >= 1 && v.nm <= 4 && v.nk >= 1 && v.nk <= 4, "oz split_view: 1..4 dims");
  const int64_t rows = v.rows(), K = v.cols();
  if (rows <= 0) return;
  const int64_t Kp = padded_k(K);
  if (plane_stride <= 0) plane_stride = rows * Kp;
  ASCC_CUDA(cudaMemsetAsync(exps, 0, sizeof(int32_t) * (size_t)rows, s));
  if (v.kstr[v.nk - 1] != 1) {
    const int64_t tiles = (rows + kViewTileM - 1) / kViewTileM * (Kp / kViewTileK);
    const int gt = (int)std::min<int64_t>(tiles, 152 * 8);
    oz_rowmax_view_t_kernel<<<gt, 256, 0, s>>>(reinterpret_cast<unsigned*>(exps), in, v, rows, K,
                                               Kp);
    oz_exponent_kernel<<<grid_for(rows), 256, 0, s>>>(exps, rows);
    oz_digits_view_t_kernel<<<gt, 256, 0, s>>>(planes, exps, in, v, rows, K, Kp, plane_stride);
    count_launch(3);
    check_launch("oz_split_view_t");
    return;
  }
  const bool fast = v.kext[v.nk - 1] % 8 == 0;
  const int64_t runs = rows * (Kp / 8);
  const int g = (int)std::min<int64_t>((runs + 255) / 256, 152 * 16);
  if (runs + 256ll * g < (1ll << 32)) {
    oz_rowmax_view_kernel<uint32_t><<<g, 256, 0, s>>>(reinterpret_cast<unsigned*>(exps), in, v,
                                                      rows, K, Kp, fast);
    oz_exponent_kernel<<<grid_for(rows), 256, 0, s>>>(exps, rows);
    oz_digits_view_kernel<uint32_t><<<g, 256, 0, s>>>(planes, exps, in, v, rows, K, Kp,
                                                      plane_stride, fast);
  } else {
    oz_rowmax_view_kernel<long long><<<g, 256, 0, s>>>(reinterpret_cast<unsigned*>(exps), in, v,
                                                       rows, K, Kp, fast);
    oz_exponent_kernel<<<grid_for(rows), 256, 0, s>>>(exps, rows);
    oz_digits_view_kernel<long long><<<g, 256, 0, s>>>(planes, exps, in, v, rows, K, Kp,
                                                       plane_stride, fast);
  }
  count_launch(3);
  check_launch("oz_split_view");
}

int splitk_for(int64_t M, int64_t N, int64_t K, bool fill) {
  if (!fill) return 1;
  const int64_t tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  const int64_t num_kt = (K + BK - 1) / BK;
  // each slice keeps at least two exact chunks; among those, the split whose
  // CTA count fills the last wave best (one CTA per SM), the smaller on ties
  const int64_t zmax = std::max<int64_t>(1, std::min<int64_t>(64, num_kt / (2 * KCT)));
  int best = 1;
  double best_eff = 0.0;
  for (int64_t z = 1; z <= zmax; ++z) {
    const int64_t ctas = tiles * z;
    const int64_t waves = (ctas + 151) / 152;
    const double eff = (double)ctas / (double)(waves * 152);
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = (int)z;
    }
  }
  return best;
}

void gemm(cudaStream_t s, int64_t M, int64_t N, int64_t K, double alpha, const __nv_bfloat16* A,
          const int32_t* ea, int64_t a_plane_stride, const __nv_bfloat16* B, const int32_t* eb,
          int64_t b_plane_stride, double beta, double* C, int64_t ldc, long long* ws, int* err,
          int splitk) {
  ASCC_REQUIRE(M > 0 && N > 0 && K > 0, "oz::gemm: empty");
  ASCC_REQUIRE(splitk >= 1 && (splitk == 1 || ws), "oz::gemm: split K needs a workspace");
  static std::once_flag attr_once;
  cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [&] {
    attr_err = cudaFuncSetAttribute(gemm_oz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    SMEM_BYTES);
  });
  ASCC_CUDA(attr_err);
  const int64_t Kp = padded_k(K);
  if (a_plane_stride <= 0) a_plane_stride = M * Kp;
  if (b_plane_stride <= 0) b_plane_stride = N * Kp;
  const CUtensorMap am = make_map3(A, M, Kp, a_plane_stride, BM);
  const CUtensorMap bm = make_map3(B, N, Kp, b_plane_stride, BN);
  count_flops(2.0 * (double)M * N * K);
  const int num_kt = (int)(Kp / BK);
  // slices of whole exact chunks
  int kt_chunk = (num_kt + splitk - 1) / splitk;
  kt_chunk = (kt_chunk + KCT - 1) / KCT * KCT;
  const int z = (num_kt + kt_chunk - 1) / kt_chunk;
  dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((N + BN - 1) / BN), (unsigned)z);
  ASCC_REQUIRE(grid.y <= 65535, "oz::gemm: N too large");
  if (z > 1) ASCC_CUDA(cudaMemsetAsync(ws, 0, ws_bytes(M, N), s));
  gemm_oz_kernel<<<grid, NTHREADS, SMEM_BYTES, s>>>(am, bm, (int)M, (int)N, num_kt, kt_chunk,
                                                    reinterpret_cast<unsigned long long*>(ws), ea,
                                                    eb, alpha, beta, C, (long long)ldc, err);
  count_launch();
  check_launch("gemm_oz");
  if (z > 1) {
    oz_finish_kernel<<<grid_for(M * N), 256, 0, s>>>(C, (long long)ldc, ws, ea, eb, M, N, alpha,
                                                     beta);
    count_launch();
    check_launch("oz_finish");
  }
}

}  // namespace oz
}  // namespace ascc
