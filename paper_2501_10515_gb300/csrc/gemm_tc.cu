// Split-precision tensor-core GEMM for sm_103a (tcgen05 + TMA + TMEM).
//
//   C (FP64, row-major) = alpha * sum_{(u,w) in segs} A_u B_w^T + beta * C
//
// A_u [M][Kp] and B_w [N][Kp] are BF16, K-major (row-major with K
// contiguous), Kp a multiple of 64.  A FP64 operand x is rounded to FP32
// (f) and carried as f = x0 + x1 + x2 (x0 = bf16(f), x1 = bf16(f - x0),
// x2 = bf16(f - x0 - x1), the subtractions exact in FP32);
// the products x0 y0, x0 y1, x1 y0 (, x0 y2, x1 y1, x2 y0) recover 16 (24)
// significant bits, each product exact in the FP32 accumulator.
//
// One CTA computes a 128 x BN tile: warp 0 issues TMA loads into a
// STAGES-deep shared-memory ring, warp 1 issues tcgen05.mma (M=128, N=BN,
// K=16) into a TMEM accumulator, and all four warps read TMEM back
// (tcgen05.ld 32x32b) for the FP64 epilogue.  Every wait is bounded by a
// 2-second %globaltimer budget; on expiry the kernel records an error code,
// skips the remaining work, frees its TMEM and returns.
#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>

#include "fpconv.cuh"
#include "gemm_tc.h"
#include "matview.cuh"
#include "tc_ptx.cuh"

namespace ascc {
namespace tc {
namespace {

constexpr int BM = 128, BN = 256, BK = 64, NTHREADS = 128;
constexpr int TK = 32;                           // K tile of the ring (64-byte swizzle rows)
constexpr int EPI_BYTES = BM * (BN + 1) * 4;     // FP32 epilogue tile (odd pitch)

// Ring geometry per split level: every stage holds all LEVEL planes of A
// (128 x 32) and of B (256 x 32) for one K tile, so the plane products of a
// K tile reuse the loaded tiles.
template <int LEVEL>
struct Ring {
  static constexpr int A_TILE = BM * TK * 2;     // 8 KB
  static constexpr int B_TILE = BN * TK * 2;     // 16 KB
  static constexpr int A_BYTES = LEVEL * A_TILE;
  static constexpr int STAGE_BYTES = LEVEL * (A_TILE + B_TILE);
  static constexpr int STAGES = LEVEL == 3 ? 3 : LEVEL == 2 ? 4 : 6;
  static constexpr int RING_BYTES = STAGES * STAGE_BYTES;
  static constexpr int BODY = RING_BYTES > EPI_BYTES ? RING_BYTES : EPI_BYTES;
  static constexpr int SMEM_BYTES = BODY + 1024 /*align*/ + 256 /*barriers*/;
  // plane products (u of A, w of B), the small planes first; the leading
  // product (0, 0) has a TMEM accumulator of its own and the cross products
  // share a second one, so that the large running sum is rounded once per K
  // step (the tensor core's FP32 accumulation truncates)
  static constexpr int NPROD = LEVEL == 1 ? 1 : LEVEL == 2 ? 3 : 6;
  static constexpr int NACC = LEVEL == 1 ? 1 : 2;
  static constexpr int TMEM_COLS = NACC == 1 ? 256 : 512;
  __host__ __device__ static constexpr int pa(int i) {
    return LEVEL == 1 ? 0 : LEVEL == 2 ? (i == 0 ? 1 : 0) : (i == 0 ? 2 : i == 1 || i == 3 ? 1 : 0);
  }
  __host__ __device__ static constexpr int pb(int i) {
    return LEVEL == 1 ? 0 : LEVEL == 2 ? (i == 1 ? 1 : 0) : (i == 2 ? 2 : i == 1 || i == 4 ? 1 : 0);
  }
  static_assert(SMEM_BYTES <= 227 * 1024, "shared memory per CTA");
};

using namespace ptx;

template <int LEVEL>
__global__ void __launch_bounds__(NTHREADS, 1)
gemm_tc_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
               int M, int N, int num_kt, int kt_chunk, double alpha, double beta,
               double* __restrict__ C, long long ldc, float* __restrict__ ws, int* err) {
  using G = Ring<LEVEL>;
  constexpr int STAGES = G::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + G::BODY);
  uint32_t* tmem_holder = (uint32_t*)(bars + 2 * STAGES + 2);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES),
                 done = smem_u32(bars + 2 * STAGES);
  __shared__ int abort_flag;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_holder)),
                 "r"(G::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_holder;
  // split K: this CTA covers the K tiles [kt0, kt0 + nkt)
  const int kt0 = blockIdx.z * kt_chunk;
  const int nkt = max(0, min(kt_chunk, num_kt - kt0));
  const int total = nkt;

  if (warp == 0 && lane == 0) {
    // TMA producer: all planes of A and B of one K tile per stage
    for (int it = 0; it < total; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (uint32_t)((it / STAGES) & 1);
      if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, err, 1)) {
        abort_flag = 1;
        break;
      }
      if (*(volatile int*)&abort_flag) break;
      const int kx = (kt0 + it) * TK;
      const uint32_t sa = smem_u32(smem + s * G::STAGE_BYTES);
      mbar_expect_tx(full0 + 8 * s, G::STAGE_BYTES);
      tma_load_3d(sa, &amap, full0 + 8 * s, kx, m0, 0);
      tma_load_3d(sa + G::A_BYTES, &bmap, full0 + 8 * s, kx, n0, 0);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: every plane product of the K tile from the same stage
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    for (int it = 0; it < total; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (uint32_t)((it / STAGES) & 1);
      if (!mbar_wait(full0 + 8 * s, ph, err, 2)) {
        abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = smem_u32(smem + s * G::STAGE_BYTES), sb = sa + G::A_BYTES;
#pragma unroll
      for (int p = 0; p < G::NPROD; ++p) {
        // accumulator 0: the leading product; 1: the cross products (the
        // first of them is p = 0)
        const bool lead = G::pa(p) == 0 && G::pb(p) == 0;
        const uint32_t acc = (G::NACC == 2 && !lead) ? 256u : 0u;
        const bool first = it == 0 && (lead || p == 0);
#pragma unroll
        for (int kk = 0; kk < TK / 16; ++kk) {
          const uint64_t ad = sw64_desc(sa + G::pa(p) * G::A_TILE + kk * 32);
          const uint64_t bd = sw64_desc(sb + G::pb(p) * G::B_TILE + kk * 32);
          mma_bf16(tmem + acc, ad, bd, idesc, (first && kk == 0) ? 0u : 1u);
        }
      }
      mma_commit(empty0 + 8 * s);
    }
    mma_commit(done);
  }
  __syncwarp();
  // epilogue: TMEM lanes [32 warp, 32 warp + 32) hold rows m0 + 32 warp + lane.
  // The tile goes through shared memory (the ring is idle once every MMA has
  // completed) so that the FP64 (or FP32 partial) stores are coalesced rows.
  const bool ok = mbar_wait(done, 0, err, 3);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool go = __syncthreads_and(ok && !*(volatile int*)&abort_flag) != 0;
  if (go) {
    constexpr int PITCH = BN + 1;  // odd pitch: conflict-free column writes
    float* tile = reinterpret_cast<float*>(smem);
    const int lrow = warp * 32 + lane;
    if (total > 0) {
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
      for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(taddr + c0, r);
        if (G::NACC == 2) {
          uint32_t q[16];
          tmem_ld16(taddr + 256 + c0, q);
#pragma unroll
          for (int j = 0; j < 16; ++j)
            tile[lrow * PITCH + c0 + j] = __uint_as_float(r[j]) + __uint_as_float(q[j]);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) tile[lrow * PITCH + c0 + j] = __uint_as_float(r[j]);
        }
      }
    }
    __syncthreads();
    const int rows = min(BM, M - m0), cols = min(BN, N - n0);
    if (ws || beta == 0.0) {
      // store-only: split-K partials (summed later) or alpha * tile, one loop
      // per kind of store
      const Pow2 p2 = pow2_of(alpha);
      // groups of U rows: a thread reads its U staged values before the
      // first of their stores, so that U stores are in flight at a time
      // (one warp per SM sub-partition has no other work to hide latency)
      auto rows_loop = [&](auto put) {
        constexpr int U = 4;
        int rr = 0;
        for (; rr + U <= rows; rr += U) {
          for (int c = threadIdx.x; c < cols; c += NTHREADS) {
            float a[U];
#pragma unroll
            for (int u = 0; u < U; ++u) a[u] = total > 0 ? tile[(rr + u) * PITCH + c] : 0.f;
#pragma unroll
            for (int u = 0; u < U; ++u) put(a[u], (long long)(m0 + rr + u), n0 + c);
          }
        }
        for (; rr < rows; ++rr) {
          const long long row = m0 + rr;
          for (int c = threadIdx.x; c < cols; c += NTHREADS)
            put(total > 0 ? tile[rr * PITCH + c] : 0.f, row, n0 + c);
        }
      };
      if (ws)
        rows_loop([&](float a, long long row, int col) {
          ws[((long long)blockIdx.z * M + row) * N + col] = a;
        });
      else if (p2.ok)
        rows_loop([&](float a, long long row, int col) {
          C[row * ldc + col] = f32_to_f64_pow2(a, p2, alpha);
        });
      else
        rows_loop([&](float a, long long row, int col) {
          C[row * ldc + col] = alpha * f32_to_f64(a);
        });
    } else {
      const bool beta1 = beta == 1.0;  // kernel-uniform: beta * old = old
      // C = alpha * tile + beta * C: the old values of RB rows are loaded
      // before the first store, so that each thread has RB loads in flight
      // instead of one round trip to memory per row
      constexpr int RB = 16;
      auto rmw = [&](auto combine) {
        for (int r0 = 0; r0 < rows; r0 += RB) {
          for (int c = threadIdx.x; c < cols; c += NTHREADS) {
            double old[RB];
#pragma unroll
            for (int u = 0; u < RB; ++u)
              old[u] = (r0 + u < rows) ? C[(long long)(m0 + r0 + u) * ldc + n0 + c] : 0.0;
#pragma unroll
            for (int u = 0; u < RB; ++u) {
              if (r0 + u < rows) {
                const float a = total > 0 ? tile[(r0 + u) * PITCH + c] : 0.f;
                C[(long long)(m0 + r0 + u) * ldc + n0 + c] = combine(a, old[u]);
              }
            }
          }
        }
      };
      if (beta1)
        rmw([&](float a, double o) { return fma(alpha, f32_to_f64(a), o); });
      else
        rmw([&](float a, double o) { return fma(alpha, (double)a, beta * o); });
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(G::TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Persistent variant for narrow products (N <= 128): 128 x 64 tiles, one CTA
// per SM looping over the (M tile, N tile, K chunk) work items.  Warps 0-3
// move accumulators out of TMEM (warp w reads lanes [32 w, 32 w + 32)), warp 4
// issues the TMA loads, warp 5 the MMAs.  The ring runs on across work items,
// and two TMEM accumulator sets let the epilogue of one tile overlap the MMAs
// of the next; the epilogue stages its tile in a shared-memory buffer of its
// own.  Every wait is bounded; after a timeout all roles stop and the kernel
// frees its TMEM and returns.
// The tile is 128 x NB with NB = 64 (thin products) or 128 (products whose
// K chunk is short, where the epilogue of a tile would otherwise not overlap
// any MMA work).
constexpr int NWARPS_N = 6;

template <int LEVEL, int NB>
struct NarrowRing {
  static constexpr int A_TILE = BM * TK * 2;     // 8 KB
  static constexpr int B_TILE = NB * TK * 2;     // 4 or 8 KB
  static constexpr int A_BYTES = LEVEL * A_TILE;
  static constexpr int STAGE_BYTES = LEVEL * (A_TILE + B_TILE);
  static constexpr int STAGES = NB == 64 ? (LEVEL == 3 ? 4 : LEVEL == 2 ? 6 : 8)
                                         : (LEVEL == 3 ? 3 : LEVEL == 2 ? 4 : 6);
  static constexpr int RING_BYTES = STAGES * STAGE_BYTES;
  static constexpr int EPI = BM * (NB + 1) * 4;
  static constexpr int OFFS = (BM + NB) * 8;     // a tile's row and column offsets (output view)
  static constexpr int SMEM_BYTES = RING_BYTES + EPI + OFFS + 1024 + 512;
  static constexpr int NACC = Ring<LEVEL>::NACC;
  static constexpr int ACC_COLS = NACC * NB;      // one accumulator set
  static constexpr int TMEM_COLS = 2 * ACC_COLS;  // two sets (a power of 2)
  static_assert(SMEM_BYTES <= 227 * 1024, "shared memory per CTA");
  static_assert(TMEM_COLS <= 512, "TMEM columns");
};

template <int LEVEL, int NB>
__global__ void __launch_bounds__(32 * NWARPS_N, 1)
gemm_tc_narrow_kernel(const __grid_constant__ CUtensorMap amap,
                      const __grid_constant__ CUtensorMap bmap, int M, int N, int num_kt,
                      int kt_chunk, int splitk, double alpha, double beta,
                      double* __restrict__ C, long long ldc, float* __restrict__ ws, int* err,
                      int trans, const __grid_constant__ MatView cview, int has_view) {
  using G = NarrowRing<LEVEL, NB>;
  using R = Ring<LEVEL>;
  constexpr int STAGES = G::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* epi = reinterpret_cast<float*>(smem + G::RING_BYTES);
  long long* voff = reinterpret_cast<long long*>(smem + G::RING_BYTES + G::EPI);  // [BM + NB]
  uint64_t* bars = (uint64_t*)(smem + G::RING_BYTES + G::EPI + G::OFFS);
  // bars: full[STAGES], empty[STAGES], acc_full[2], acc_empty[2]
  uint32_t* tmem_holder = (uint32_t*)(bars + 2 * STAGES + 4);
  __shared__ int abort_flag, epi_fail;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES),
                 accf0 = smem_u32(bars + 2 * STAGES), acce0 = smem_u32(bars + 2 * STAGES + 2);
  const int mt = (M + BM - 1) / BM, nt = (N + NB - 1) / NB;
  const int items = mt * nt * splitk;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    epi_fail = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, 4 * 32);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_holder)),
                 "r"(G::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_holder;

  auto decode = [&](int w, int& m0, int& n0, int& kt0, int& nkt) {
    const int mi = w % mt, rest = w / mt, ni = rest % nt, kz = rest / nt;
    m0 = mi * BM;
    n0 = ni * NB;
    kt0 = kz * kt_chunk;
    nkt = max(0, min(kt_chunk, num_kt - kt0));
  };

  if (warp == 4 && lane == 0) {
    // TMA producer: the ring runs on across work items
    int it = 0;
    for (int w = blockIdx.x; w < items && !*(volatile int*)&abort_flag; w += gridDim.x) {
      int m0, n0, kt0, nkt;
      decode(w, m0, n0, kt0, nkt);
      for (int j = 0; j < nkt; ++j, ++it) {
        const int s = it % STAGES;
        const uint32_t ph = (uint32_t)((it / STAGES) & 1);
        if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, err, 11) || *(volatile int*)&abort_flag) {
          abort_flag = 1;
          break;
        }
        const int kx = (kt0 + j) * TK;
        const uint32_t sa = smem_u32(smem + s * G::STAGE_BYTES);
        mbar_expect_tx(full0 + 8 * s, G::STAGE_BYTES);
        tma_load_3d(sa, &amap, full0 + 8 * s, kx, m0, 0);
        tma_load_3d(sa + G::A_BYTES, &bmap, full0 + 8 * s, kx, n0, 0);
      }
    }
  } else if (warp == 5 && lane == 0) {
    // MMA issuer: one accumulator set per work item, alternating
    constexpr uint32_t idesc = idesc_bf16(BM, NB);
    int it = 0, tc = 0;
    for (int w = blockIdx.x; w < items && !*(volatile int*)&abort_flag; w += gridDim.x, ++tc) {
      int m0, n0, kt0, nkt;
      decode(w, m0, n0, kt0, nkt);
      const int buf = tc & 1;
      const uint32_t aph = (uint32_t)((tc >> 1) & 1);
      if (!mbar_wait(acce0 + 8 * buf, aph ^ 1u, err, 12)) {
        abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t tacc = tmem + (uint32_t)(buf * G::ACC_COLS);
      bool stop = false;
      for (int j = 0; j < nkt; ++j, ++it) {
        const int s = it % STAGES;
        const uint32_t ph = (uint32_t)((it / STAGES) & 1);
        if (!mbar_wait(full0 + 8 * s, ph, err, 13)) {
          abort_flag = 1;
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sa = smem_u32(smem + s * G::STAGE_BYTES), sb = sa + G::A_BYTES;
#pragma unroll
        for (int p = 0; p < R::NPROD; ++p) {
          const bool lead = R::pa(p) == 0 && R::pb(p) == 0;
          const uint32_t acc = (R::NACC == 2 && !lead) ? (uint32_t)NB : 0u;
          const bool first = j == 0 && (lead || p == 0);
#pragma unroll
          for (int kk = 0; kk < TK / 16; ++kk) {
            const uint64_t ad = sw64_desc(sa + R::pa(p) * G::A_TILE + kk * 32);
            const uint64_t bd = sw64_desc(sb + R::pb(p) * G::B_TILE + kk * 32);
            mma_bf16(tacc + acc, ad, bd, idesc, (first && kk == 0) ? 0u : 1u);
          }
        }
        mma_commit(empty0 + 8 * s);
      }
      if (stop) break;
      mma_commit(accf0 + 8 * buf);
    }
  } else if (warp < 4) {
    // epilogue: row lrow of each tile; TMEM -> registers -> staging tile ->
    // coalesced global stores (FP64 C, or FP32 split-K partials)
    const int lrow = warp * 32 + lane;
    const int t = threadIdx.x;  // 0..127
    const Pow2 p2 = pow2_of(alpha);
    const int smode = ws            ? 0
                      : beta == 1.0 ? kStoreBeta1
                      : beta != 0.0 ? kStoreBeta
                      : p2.ok       ? kStorePow2
                                    : kStoreScaled;
    int tc = 0;
    for (int w = blockIdx.x; w < items; w += gridDim.x, ++tc) {
      int m0, n0, kt0, nkt;
      decode(w, m0, n0, kt0, nkt);
      const int buf = tc & 1;
      const uint32_t aph = (uint32_t)((tc >> 1) & 1);
      const bool ok = mbar_wait(accf0 + 8 * buf, aph, err, 14);
      // all 128 epilogue threads agree before they touch the staging tile
      if (!ok) epi_fail = 1;
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (*(volatile int*)&epi_fail || *(volatile int*)&abort_flag) {
        abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t taddr = tmem + (uint32_t)(buf * G::ACC_COLS) + ((uint32_t)(warp * 32) << 16);
      constexpr int PITCH = NB + 1;
      if (nkt > 0) {
#pragma unroll
        for (int c0 = 0; c0 < NB; c0 += 16) {
          uint32_t r[16];
          if (R::NACC == 2) {
            // both accumulators' columns in flight before one wait
            uint32_t q[16];
            tmem_ld16_nowait(taddr + c0, r);
            tmem_ld16_nowait(taddr + NB + c0, q);
            tmem_wait_ld();
#pragma unroll
            for (int jj = 0; jj < 16; ++jj)
              epi[lrow * PITCH + c0 + jj] = __uint_as_float(r[jj]) + __uint_as_float(q[jj]);
          } else {
            tmem_ld16(taddr + c0, r);
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) epi[lrow * PITCH + c0 + jj] = __uint_as_float(r[jj]);
          }
        }
      } else {
        for (int c = 0; c < NB; ++c) epi[lrow * PITCH + c] = 0.f;
      }
      // the accumulator set is free for the MMA warp again
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(acce0 + 8 * buf);
      asm volatile("bar.sync 1, 128;" ::: "memory");
      const int rows = min(BM, M - m0), cols = min(NB, N - n0);
      const int kz = w / (mt * nt);
      // (r, c) of the caller's C: tile row rr, column c; or, for the
      // exchanged product, tile row t is column m0 + t of the caller's C
      // (row n0 + c) and consecutive threads write consecutive columns
      // each thread reads U staged values before the first of their stores,
      // so that U stores are in flight at a time (one epilogue warp per SM
      // sub-partition has no other work to hide their latency)
      auto tile_loop = [&](auto put) {
        constexpr int U = 4;
        if (!trans) {
          // 128 / NB rows per pass, NB columns each
          constexpr int RP = 128 / NB;
          const int c = t % NB;
          if (c < cols) {
            int rr = t / NB;
            for (; rr + (U - 1) * RP < rows; rr += U * RP) {
              float a[U];
#pragma unroll
              for (int u = 0; u < U; ++u) a[u] = epi[(rr + u * RP) * PITCH + c];
#pragma unroll
              for (int u = 0; u < U; ++u)
                put(a[u], (long long)(m0 + rr + u * RP), (long long)(n0 + c));
            }
            for (; rr < rows; rr += RP)
              put(epi[rr * PITCH + c], (long long)(m0 + rr), (long long)(n0 + c));
          }
        } else if (t < rows) {
          int c = 0;
          for (; c + U <= cols; c += U) {
            float a[U];
#pragma unroll
            for (int u = 0; u < U; ++u) a[u] = epi[t * PITCH + c + u];
#pragma unroll
            for (int u = 0; u < U; ++u) put(a[u], (long long)(n0 + c + u), (long long)(m0 + t));
          }
          for (; c < cols; ++c) put(epi[t * PITCH + c], (long long)(n0 + c), (long long)(m0 + t));
        }
      };
      const long long Mo = trans ? N : M, No = trans ? M : N;
      // element (r, c) of the caller's C: row-major with ldc, or through the
      // output view (rows over its M dimensions, columns over its others),
      // whose offsets for this tile's rows and columns are formed once
      const long long r0 = trans ? n0 : m0, c0 = trans ? m0 : n0;
      const int nr = trans ? NB : BM, nc = trans ? BM : NB;
      if (has_view) {
        const long long Mc = trans ? N : M, Nc = trans ? M : N;  // the caller's C
        for (int i = t; i < nr; i += 128)
          voff[i] = r0 + i < Mc ? matview_row<uint32_t>(cview, (uint32_t)(r0 + i)) : 0;
        for (int j = t; j < nc; j += 128) {
          long long off = 0;
          if (c0 + j < Nc) {
            uint32_t q = (uint32_t)(c0 + j);
            for (int d = cview.nk - 1; d >= 0; --d) {
              const uint32_t e = (uint32_t)cview.kext[d], qq = q / e;
              off += (long long)(q - qq * e) * cview.kstr[d];
              q = qq;
            }
          }
          voff[nr + j] = off;
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
      }
      auto at = [&](long long r, long long c) -> long long {
        return has_view ? voff[r - r0] + voff[nr + (c - c0)] : r * ldc + c;
      };
      // C = combine(tile value, old C) over the same elements and in the same
      // order as tile_loop; each thread loads the old values of V elements
      // before the first of their stores (the elements of a tile are distinct
      // outputs), so that V loads are in flight instead of one round trip per
      // element
      auto tile_rmw = [&](auto combine) {
        constexpr int V = 8;
        if (!trans) {
          constexpr int RP = 128 / NB;
          const int c = t % NB;
          if (c < cols) {
            int rr = t / NB;
            for (; rr + (V - 1) * RP < rows; rr += V * RP) {
              long long o[V];
              double old[V];
#pragma unroll
              for (int u = 0; u < V; ++u)
                o[u] = at((long long)(m0 + rr + u * RP), (long long)(n0 + c));
#pragma unroll
              for (int u = 0; u < V; ++u) old[u] = C[o[u]];
#pragma unroll
              for (int u = 0; u < V; ++u)
                C[o[u]] = combine(epi[(rr + u * RP) * PITCH + c], old[u]);
            }
            for (; rr < rows; rr += RP) {
              const long long o = at((long long)(m0 + rr), (long long)(n0 + c));
              C[o] = combine(epi[rr * PITCH + c], C[o]);
            }
          }
        } else if (t < rows) {
          int c = 0;
          for (; c + V <= cols; c += V) {
            long long o[V];
            double old[V];
#pragma unroll
            for (int u = 0; u < V; ++u) o[u] = at((long long)(n0 + c + u), (long long)(m0 + t));
#pragma unroll
            for (int u = 0; u < V; ++u) old[u] = C[o[u]];
#pragma unroll
            for (int u = 0; u < V; ++u) C[o[u]] = combine(epi[t * PITCH + c + u], old[u]);
          }
          for (; c < cols; ++c) {
            const long long o = at((long long)(n0 + c), (long long)(m0 + t));
            C[o] = combine(epi[t * PITCH + c], C[o]);
          }
        }
      };
      if (smode == 0)
        tile_loop([&](float a, long long r, long long c) { ws[((long long)kz * Mo + r) * No + c] = a; });
      else if (smode == kStorePow2)
        tile_loop([&](float a, long long r, long long c) {
          C[at(r, c)] = f32_to_f64_pow2(a, p2, alpha);
        });
      else if (smode == kStoreScaled)
        tile_loop([&](float a, long long r, long long c) { C[at(r, c)] = alpha * f32_to_f64(a); });
      else if (smode == kStoreBeta1)
        tile_rmw([&](float a, double o) { return fma(alpha, f32_to_f64(a), o); });
      else
        tile_rmw([&](float a, double o) { return fma(alpha, (double)a, beta * o); });
      asm volatile("bar.sync 1, 128;" ::: "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 5) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(G::TMEM_COLS)
                 : "memory");
  }
}

// One step of the compensated split-K sum: hi + x by Fast2Sum, its rounding
// error into lo.
__device__ __forceinline__ void comp_add(float& hi, float& lo, float x) {
  const float t = hi + x;
  lo += (fabsf(hi) >= fabsf(x)) ? (hi - t) + x : (x - t) + hi;
  hi = t;
}

// The output of a compensated sum hi + lo, alpha (hi + lo) (+ beta c), with
// the FP32 -> FP64 conversions in integer arithmetic: no FP64 operation for a
// power-of-two alpha and lo = 0, one addition when lo != 0; another alpha
// multiplies in FP64 (equal to the plain FP64 expression, signed zeros aside).
template <int MODE>
__device__ __forceinline__ double reduce_out(float hi, float lo, const Pow2& p2, double alpha,
                                             double beta, const double* c) {
  if (MODE == kStorePow2) {
    const double h = f32_to_f64_pow2(hi, p2, alpha);
    return lo == 0.f ? h : h + f32_to_f64_pow2(lo, p2, alpha);
  }
  const double acc = f32_to_f64(hi) + f32_to_f64(lo);
  if (MODE == kStoreScaled) return alpha * acc;
  if (MODE == kStoreBeta1) return fma(alpha, acc, *c);
  return fma(alpha, acc, beta * *c);
}

// C = alpha * sum_z ws[z] + beta * C.  The FP32 partials are summed in FP32
// with a compensation term (Fast2Sum), i.e. to about 2^-48 relative, in a
// fixed order, and converted to FP64 once: the FP64 units are the scarce
// ones on this part.
template <int MODE>
__global__ void splitk_reduce_kernel(double* __restrict__ C, long long ldc,
                                     const float* __restrict__ ws, long long M, long long N,
                                     int nz, double alpha, double beta) {
  const Pow2 p2 = pow2_of(alpha);
  const long long total = M * N;
  for (long long m = blockIdx.y; m < M; m += gridDim.y) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
      const long long idx = m * N + n;
      float hi = 0.f, lo = 0.f;
      for (int z = 0; z < nz; ++z) comp_add(hi, lo, ws[(long long)z * total + idx]);
      double* c = C + m * ldc + n;
      *c = reduce_out<MODE>(hi, lo, p2, alpha, beta, c);
    }
  }
}

// The same sums when N is a multiple of 4 and the partials are 16-byte
// aligned: each thread takes four neighbouring columns with 16-byte loads and
// keeps four K-chunks in flight.  Every element is summed in the same order as
// above, so the results are identical.
template <int MODE>
__global__ void splitk_reduce4_kernel(double* __restrict__ C, long long ldc,
                                      const float* __restrict__ ws, long long M, long long N,
                                      int nz, double alpha, double beta) {
  const Pow2 p2 = pow2_of(alpha);
  const long long n4 = N / 4, total4 = M * n4;
  const float4* __restrict__ w4 = reinterpret_cast<const float4*>(ws);
  for (long long m = blockIdx.y; m < M; m += gridDim.y) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4;
         q += (long long)gridDim.x * blockDim.x) {
      const long long idx4 = m * n4 + q;
      float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
      int z = 0;
      for (; z + 4 <= nz; z += 4) {
        float4 x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = w4[(long long)(z + u) * total4 + idx4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          comp_add(hi[0], lo[0], x[u].x);
          comp_add(hi[1], lo[1], x[u].y);
          comp_add(hi[2], lo[2], x[u].z);
          comp_add(hi[3], lo[3], x[u].w);
        }
      }
      for (; z < nz; ++z) {
        const float4 x = w4[(long long)z * total4 + idx4];
        comp_add(hi[0], lo[0], x.x);
        comp_add(hi[1], lo[1], x.y);
        comp_add(hi[2], lo[2], x.z);
        comp_add(hi[3], lo[3], x.w);
      }
      double* c = C + m * ldc + 4 * q;
#pragma unroll
      for (int e = 0; e < 4; ++e) c[e] = reduce_out<MODE>(hi[e], lo[e], p2, alpha, beta, c + e);
    }
  }
}

// The same sums written through an output view: element (m, n) of the
// product goes to C + matview_row(v, m) + (offset of n over the view's
// column dimensions).  by_rows: consecutive threads take consecutive rows
// (when the view's rows, not its columns, are the contiguous side).
template <int MODE>
__global__ void splitk_reduce_view_kernel(double* __restrict__ C, MatView v,
                                          const float* __restrict__ ws, long long M, long long N,
                                          int nz, double alpha, double beta, bool by_rows) {
  const Pow2 p2 = pow2_of(alpha);
  const long long total = M * N;
  const long long outer = by_rows ? N : M, inner = by_rows ? M : N;
  for (long long o = blockIdx.y; o < outer; o += gridDim.y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < inner;
         i += (long long)gridDim.x * blockDim.x) {
      const long long m = by_rows ? i : o, n = by_rows ? o : i;
      const long long idx = m * N + n;
      float hi = 0.f, lo = 0.f;
      for (int z = 0; z < nz; ++z) comp_add(hi, lo, ws[(long long)z * total + idx]);
      long long off = matview_row<uint32_t>(v, (uint32_t)m);
      uint32_t r = (uint32_t)n;
      for (int d = v.nk - 1; d >= 0; --d) {
        const uint32_t e = (uint32_t)v.kext[d], q = r / e;
        off += (long long)(r - q * e) * v.kstr[d];
        r = q;
      }
      double* c = C + off;
      *c = reduce_out<MODE>(hi, lo, p2, alpha, beta, c);
    }
  }
}

// FP64 [rows][K] (row stride ld) -> nsplit BF16 planes [nsplit][rows][Kp], zero padded.
// The value is rounded to FP32 once (24 significant bits, as many as three
// planes hold) and split with exact FP32 subtractions.  Each thread converts a
// run of 8 consecutive values of one row and writes 16 bytes per plane.
template <typename I>
__global__ void split_bf16_kernel(__nv_bfloat16* __restrict__ out, const double* __restrict__ in,
                                  long long rows, long long K, long long ld, long long Kp,
                                  int nsplit, long long plane_stride) {
  const I runs = (I)(Kp / 8), total = (I)rows * runs;
  for (I idx = blockIdx.x * (I)blockDim.x + threadIdx.x; idx < total;
       idx += (I)gridDim.x * blockDim.x) {
    const I rq = idx / runs;
    const long long r = rq, k0 = (long long)(idx - rq * runs) * 8;
    const double* x = in + r * ld + k0;
    float f[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) f[j] = (k0 + j < K) ? f64_to_f32_rn(x[j]) : 0.f;
    for (int s = 0; s < nsplit; ++s) {
      __align__(16) __nv_bfloat16 h[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        h[j] = __float2bfloat16_rn(f[j]);
        f[j] -= __bfloat162float(h[j]);
      }
      *reinterpret_cast<uint4*>(out + (long long)s * plane_stride + r * Kp + k0) =
          *reinterpret_cast<const uint4*>(h);
    }
  }
}

// The same from a strided tensor read through a MatView (no permuted copy).
template <typename I>
__global__ void split_bf16_view_kernel(__nv_bfloat16* __restrict__ out,
                                       const double* __restrict__ in, MatView v, long long rows,
                                       long long K, long long Kp, int nsplit,
                                       long long plane_stride, bool fast) {
  const I runs = (I)(Kp / 8), total = (I)rows * runs;
  for (I idx = blockIdx.x * (I)blockDim.x + threadIdx.x; idx < total;
       idx += (I)gridDim.x * blockDim.x) {
    const I rq = idx / runs;
    const long long r = rq, k0 = (long long)(idx - rq * runs) * 8;
    double x[8];
    matview_run8<I>(v, in + matview_row<I>(v, rq), k0, K, fast, x);
    float f[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) f[j] = f64_to_f32_rn(x[j]);
    for (int s = 0; s < nsplit; ++s) {
      __align__(16) __nv_bfloat16 h[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        h[j] = __float2bfloat16_rn(f[j]);
        f[j] -= __bfloat162float(h[j]);
      }
      *reinterpret_cast<uint4*>(out + (long long)s * plane_stride + r * Kp + k0) =
          *reinterpret_cast<const uint4*>(h);
    }
  }
}

// The same for a view whose contiguous dimension is on the row side: one
// 64 x 32 tile per block pass, transposed through shared memory.
__global__ void __launch_bounds__(256) split_bf16_view_t_kernel(
    __nv_bfloat16* __restrict__ out, const double* __restrict__ in, MatView v, long long rows,
    long long K, long long Kp, int nsplit, long long plane_stride) {
  __shared__ double tile[kViewTileK][kViewTileM + 1];
  __shared__ long long roff[kViewTileM], coff[kViewTileK];
  const long long ntm = (rows + kViewTileM - 1) / kViewTileM, ntk = Kp / kViewTileK;
  for (long long tix = blockIdx.x; tix < ntm * ntk; tix += gridDim.x) {
    const long long m0 = (tix / ntk) * kViewTileM, k0 = (tix % ntk) * kViewTileK;
    matview_load_tile_t(v, in, rows, K, m0, k0, tile, roff, coff);
    const int mi = threadIdx.x >> 2, kr = (threadIdx.x & 3) * 8;
    float f[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) f[j] = f64_to_f32_rn(tile[kr + j][mi]);
    if (m0 + mi < rows) {
      for (int s = 0; s < nsplit; ++s) {
        __align__(16) __nv_bfloat16 h[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          h[j] = __float2bfloat16_rn(f[j]);
          f[j] -= __bfloat162float(h[j]);
        }
        *reinterpret_cast<uint4*>(out + (long long)s * plane_stride + (m0 + mi) * Kp + k0 + kr) =
            *reinterpret_cast<const uint4*>(h);
      }
    }
    __syncthreads();  // the tile is rewritten by the next pass
  }
}

struct SplitJob {
  __nv_bfloat16* out;
  const double* in;
  MatView v;
  long long rows, K, Kp, plane_stride;
  int nsplit, mode, fast, blocks;
};

// Both operand splits of one product in one launch: blocks [0, j0.blocks) take
// the first job, the rest the second; each job is a view read in runs of 8
// (mode 1, which covers plain [rows][K] operands) or in transposing tiles
// (mode 2).  32-bit index arithmetic (the host checks the sizes).
__global__ void __launch_bounds__(256) split_pair_kernel(SplitJob j0, SplitJob j1) {
  __shared__ double tile[kViewTileK][kViewTileM + 1];
  __shared__ long long roff[kViewTileM], coff[kViewTileK];
  const bool second = blockIdx.x >= (unsigned)j0.blocks;
  const SplitJob& j = second ? j1 : j0;
  const uint32_t bid = second ? blockIdx.x - (unsigned)j0.blocks : blockIdx.x;
  const uint32_t nb = (uint32_t)j.blocks;
  if (j.mode == 2) {
    const long long ntm = (j.rows + kViewTileM - 1) / kViewTileM, ntk = j.Kp / kViewTileK;
    for (long long tix = bid; tix < ntm * ntk; tix += nb) {
      const long long m0 = (tix / ntk) * kViewTileM, k0 = (tix % ntk) * kViewTileK;
      matview_load_tile_t(j.v, j.in, j.rows, j.K, m0, k0, tile, roff, coff);
      const int mi = threadIdx.x >> 2, kr = (threadIdx.x & 3) * 8;
      float f[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) f[q] = f64_to_f32_rn(tile[kr + q][mi]);
      if (m0 + mi < j.rows) {
        for (int s = 0; s < j.nsplit; ++s) {
          __align__(16) __nv_bfloat16 h[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            h[q] = __float2bfloat16_rn(f[q]);
            f[q] -= __bfloat162float(h[q]);
          }
          *reinterpret_cast<uint4*>(j.out + (long long)s * j.plane_stride + (m0 + mi) * j.Kp +
                                    k0 + kr) = *reinterpret_cast<const uint4*>(h);
        }
      }
      __syncthreads();  // the tile is rewritten by the next pass
    }
    return;
  }
  const uint32_t runs = (uint32_t)(j.Kp / 8), total = (uint32_t)j.rows * runs;
  for (uint32_t idx = bid * 256u + threadIdx.x; idx < total; idx += nb * 256u) {
    const uint32_t rq = idx / runs;
    const long long r = rq, k0 = (long long)(idx - rq * runs) * 8;
    double x[8];
    matview_run8<uint32_t>(j.v, j.in + matview_row<uint32_t>(j.v, rq), k0, j.K, j.fast != 0, x);
    float f[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) f[q] = f64_to_f32_rn(x[q]);
    for (int s = 0; s < j.nsplit; ++s) {
      __align__(16) __nv_bfloat16 h[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        h[q] = __float2bfloat16_rn(f[q]);
        f[q] -= __bfloat162float(h[q]);
      }
      *reinterpret_cast<uint4*>(j.out + (long long)s * j.plane_stride + r * j.Kp + k0) =
          *reinterpret_cast<const uint4*>(h);
    }
  }
}

// Self-test of the bounded wait: one thread waits, with the kernels' wait
// function and a budget of limit_ns, on the first phase of an mbarrier that
// nothing arrives at; the budget runs out, the code goes to err, the kernel
// returns.
__global__ void wait_selftest_kernel(int* err, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  const uint32_t b = smem_u32(&bar);
  mbar_init(b, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  mbar_wait_ns(b, 0, err, 99, limit_ns);
}

// 3-D map over the planes [level][rows][Kp] (plane stride in elements): one
// box brings all planes of a 32-wide K tile, 64-byte swizzle.
CUtensorMap make_planes_map(const __nv_bfloat16* base, int64_t rows, int64_t Kp,
                            int64_t plane_stride, int level, int box_rows) {
  CUtensorMap m;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)level};
  cuuint64_t strides[2] = {(cuuint64_t)(Kp * 2), (cuuint64_t)(plane_stride * 2)};
  cuuint32_t box[3] = {(cuuint32_t)TK, (cuuint32_t)box_rows, (cuuint32_t)level};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base, dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(ASCC_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return m;
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  if (!fn) throw Error(ASCC_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  return fn;
}

int64_t padded_k(int64_t K) { return (K + BK - 1) / BK * BK; }

void split_bf16(cudaStream_t s, __nv_bfloat16* out, const double* in, int64_t rows, int64_t K,
                int64_t ld, int nsplit, int64_t plane_stride) {
  const int64_t Kp = padded_k(K), total = rows * Kp;
  if (total == 0) return;
  if (plane_stride <= 0) plane_stride = total;
  const int g = (int)std::min<int64_t>((rows * (Kp / 8) + 255) / 256, 152 * 16);
  if (rows * (Kp / 8) + 256ll * g < (1ll << 32))
    split_bf16_kernel<uint32_t><<<g, 256, 0, s>>>(out, in, rows, K, ld, Kp, nsplit, plane_stride);
  else
    split_bf16_kernel<long long><<<g, 256, 0, s>>>(out, in, rows, K, ld, Kp, nsplit, plane_stride);
  count_launch();
  check_launch("split_bf16");
}

void split_bf16_view(cudaStream_t s, __nv_bfloat16* out, const double* in, const MatView& v,
                     int nsplit, int64_t plane_stride) {
  ASCC_REQUIRE(v.nm >= 1 && v.nm <= 4 && v.nk >= 1 && v.nk <= 4, "split_bf16_view: 1..4 dims");
  const int64_t rows = v.rows(), K = v.cols(), Kp = padded_k(K), total = rows * Kp;
  if (total == 0) return;
  if (plane_stride <= 0) plane_stride = total;
  if (v.kstr[v.nk - 1] != 1) {
    const int64_t tiles = (rows + kViewTileM - 1) / kViewTileM * (Kp / kViewTileK);
    const int g = (int)std::min<int64_t>(tiles, 152 * 8);
    split_bf16_view_t_kernel<<<g, 256, 0, s>>>(out, in, v, rows, K, Kp, nsplit, plane_stride);
    count_launch();
    check_launch("split_bf16_view_t");
    return;
  }
  const bool fast = v.kext[v.nk - 1] % 8 == 0;
  const int g = (int)std::min<int64_t>((rows * (Kp / 8) + 255) / 256, 152 * 16);
  if (rows * (Kp / 8) + 256ll * g < (1ll << 32))
    split_bf16_view_kernel<uint32_t><<<g, 256, 0, s>>>(out, in, v, rows, K, Kp, nsplit,
                                                       plane_stride, fast);
  else
    split_bf16_view_kernel<long long><<<g, 256, 0, s>>>(out, in, v, rows, K, Kp, nsplit,
                                                        plane_stride, fast);
  count_launch();
  check_launch("split_bf16_view");
}

void split_bf16_pair(cudaStream_t s, const SplitSpec* a, const SplitSpec* b) {
  SplitJob job[2];
  const SplitSpec* spec[2] = {a, b};
  int n = 0;
  bool fits = true;
  for (int q = 0; q < 2; ++q) {
    if (!spec[q]) continue;
    const MatView& v = spec[q]->v;
    ASCC_REQUIRE(v.nm >= 1 && v.nm <= 4 && v.nk >= 1 && v.nk <= 4, "split_bf16_pair: 1..4 dims");
    SplitJob& j = job[n];
    j.out = spec[q]->out;
    j.in = spec[q]->in;
    j.v = v;
    j.rows = v.rows();
    j.K = v.cols();
    j.Kp = padded_k(j.K);
    j.plane_stride = j.rows * j.Kp;
    j.nsplit = spec[q]->nsplit;
    j.mode = v.kstr[v.nk - 1] != 1 ? 2 : 1;
    j.fast = v.kext[v.nk - 1] % 8 == 0 ? 1 : 0;
    if (j.mode == 2) {
      const int64_t tiles = (j.rows + kViewTileM - 1) / kViewTileM * (j.Kp / kViewTileK);
      j.blocks = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, 152 * 8));
    } else {
      const int64_t runs = j.rows * (j.Kp / 8);
      j.blocks = (int)std::max<int64_t>(1, std::min<int64_t>((runs + 255) / 256, 152 * 16));
      fits = fits && runs + 256ll * j.blocks < (1ll << 32);
    }
    fits = fits && j.rows < (1ll << 31) && j.K < (1ll << 31);
    if (j.rows * j.Kp > 0) ++n;
  }
  if (n == 0) return;
  if (!fits) {
    // beyond 32-bit indices: the separate kernels (64-bit paths)
    for (int q = 0; q < 2; ++q)
      if (spec[q]) split_bf16_view(s, spec[q]->out, spec[q]->in, spec[q]->v, spec[q]->nsplit);
    return;
  }
  if (n == 1) {
    job[1] = job[0];
    job[1].blocks = 0;
  }
  split_pair_kernel<<<job[0].blocks + job[1].blocks, 256, 0, s>>>(job[0], job[1]);
  count_launch();
  check_launch("split_bf16_pair");
}

int wait_selftest(cudaStream_t s, int limit_ms) {
  int* err = nullptr;
  ASCC_CUDA(cudaMalloc(&err, sizeof(int)));
  ASCC_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  wait_selftest_kernel<<<1, 32, 0, s>>>(err, (unsigned long long)limit_ms * 1000000ull);
  count_launch();
  check_launch("wait_selftest");
  int h = 0;
  ASCC_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  ASCC_CUDA(cudaStreamSynchronize(s));
  ASCC_CUDA(cudaFree(err));
  return h;
}

int products_for(int level) { return level == 1 ? 1 : level == 2 ? 3 : 6; }

// Products with at most this many columns run on the persistent 128 x 64
// kernel; those with at most NARROW_M rows (and more columns) run on it with
// the operands exchanged and the tile stored transposed.
// Other products whose K (chunk) is at most SHORT_K run on the persistent
// kernel with 128 x 128 tiles: there the epilogue of a tile takes as long as
// its MMAs, and the persistent kernel overlaps the two.
constexpr int64_t NARROW_N = 128, NARROW_M = 64, SHORT_K = 1024;

int splitk_for(int64_t M, int64_t N, int64_t K, int fill) {
  // K chunks of at most 2048 (FP32 accumulation error ~ 2^-24 sqrt(K/16) per chunk),
  // and at least `fill` work items when K allows (fill the GPU for small M x N)
  const bool swap = M <= NARROW_M && N > NARROW_N;
  if (swap) std::swap(M, N);
  const int64_t bn = N <= NARROW_N ? 64 : padded_k(K) <= SHORT_K ? 128 : BN;
  const int64_t tiles = ((M + BM - 1) / BM) * ((N + bn - 1) / bn);
  const int64_t num_kt = (K + BK - 1) / BK;
  int64_t z = (K + 2047) / 2048;
  while (tiles * z < fill && z < num_kt) ++z;
  return (int)std::min<int64_t>(std::max<int64_t>(z, 1), std::min<int64_t>(num_kt, 512));
}

namespace {
std::mutex g_tune_mu;
std::map<uint64_t, int> g_tune;

int ilog2_ceil(int64_t x) {
  int r = 0;
  while ((int64_t(1) << r) < x) ++r;
  return r;
}

// The tile shape for this product: the tuned one of its class, tuning the
// class first when allowed (see autotuned_classes in gemm_tc.h).
int tuned_tile(cudaStream_t s, int64_t M, int64_t N, int64_t K, int level,
               const __nv_bfloat16* A, const __nv_bfloat16* B, int splitk, float* ws,
               int64_t b_plane_stride, int* err) {
  static const bool on = [] {
    const char* e = std::getenv("ASCC_AUTOTUNE");
    return !(e && e[0] == '0');
  }();
  if (!on) return kTileRules;
  const double flops = 2.0 * (double)M * N * K;
  if (M * N > (int64_t(1) << 25) || flops < 1e8) return kTileRules;
  // M <= 64 < N runs with the operands exchanged, which changes the order of
  // the tensor core's sums: those products keep the size rules
  if (M <= NARROW_M && N > NARROW_N) return kTileRules;
  const int64_t kc = (padded_k(K) + splitk - 1) / splitk;
  const uint64_t key = (uint64_t)level | (uint64_t)ilog2_ceil(M) << 4 |
                       (uint64_t)ilog2_ceil(N) << 10 | (uint64_t)ilog2_ceil(kc) << 16 |
                       (uint64_t)(splitk > 1) << 22;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
    return kTileRules;
  // candidates: every shape; scratch output, beta = 0, the caller's planes and
  // split-K workspace (all on this stream, before the caller's own product)
  double* Cs = nullptr;
  ASCC_CUDA(cudaMallocAsync(&Cs, sizeof(double) * (size_t)(M * N), s));
  const int cands[3] = {kTileWide, kTile128, kTile64};
  float best = 1e30f;
  int pick = kTileRules;
  cudaEvent_t e0, e1;
  ASCC_CUDA(cudaEventCreate(&e0));
  ASCC_CUDA(cudaEventCreate(&e1));
  for (int c : cands) {
    gemm_split(s, M, N, K, level, 1.0, A, B, 0.0, Cs, N, err, splitk, ws, b_plane_stride,
               nullptr, c);  // warm-up
    ASCC_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < 2; ++r)
      gemm_split(s, M, N, K, level, 1.0, A, B, 0.0, Cs, N, err, splitk, ws, b_plane_stride,
                 nullptr, c);
    ASCC_CUDA(cudaEventRecord(e1, s));
    ASCC_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    ASCC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  ASCC_CUDA(cudaEventDestroy(e0));
  ASCC_CUDA(cudaEventDestroy(e1));
  ASCC_CUDA(cudaFreeAsync(Cs, s));
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = pick;
  return pick;
}
}  // namespace

int64_t autotuned_classes() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return (int64_t)g_tune.size();
}

void gemm_split(cudaStream_t s, int64_t M, int64_t N, int64_t K, int level, double alpha,
                const __nv_bfloat16* A, const __nv_bfloat16* B, double beta, double* C, int64_t ldc,
                int* err, int splitk, float* ws, int64_t b_plane_stride, const MatView* cview,
                int tile) {
  if (tile == kTileAuto) tile = tuned_tile(s, M, N, K, level, A, B, splitk, ws, b_plane_stride, err);
  ASCC_REQUIRE(level >= 1 && level <= 3, "split level 1..3");
  ASCC_REQUIRE(!cview || ws, "gemm_split: an output view needs a workspace");
  ASCC_REQUIRE(M > 0 && N > 0 && K > 0, "gemm_split: empty");
  ASCC_REQUIRE(splitk >= 1 && (splitk == 1 || ws), "gemm_split: split-K needs a workspace");
  static std::once_flag attr_once;
  cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [&] {
    attr_err = cudaFuncSetAttribute(gemm_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    Ring<1>::SMEM_BYTES);
    if (attr_err == cudaSuccess)
      attr_err = cudaFuncSetAttribute(gemm_tc_kernel<2>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      Ring<2>::SMEM_BYTES);
    if (attr_err == cudaSuccess)
      attr_err = cudaFuncSetAttribute(gemm_tc_kernel<3>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      Ring<3>::SMEM_BYTES);
  });
  ASCC_CUDA(attr_err);
  const int64_t Kp = padded_k(K);
  const int num_kt = (int)(Kp / TK);
  const int kt_chunk = (num_kt + splitk - 1) / splitk;
  bool swap = M <= NARROW_M && N > NARROW_N;
  bool thin = N <= NARROW_N || swap;
  bool shortk = !thin && (int64_t)kt_chunk * TK <= SHORT_K;
  if (tile == kTileWide) {
    swap = thin = shortk = false;
  } else if (tile == kTile128) {
    swap = thin = false;
    shortk = true;
  } else if (tile == kTile64) {
    thin = true;
    shortk = false;
  }
  const bool narrow = thin || shortk;   // the persistent kernel
  const int nbt = thin ? 64 : 128;      // its tile width
  const int64_t bstride = b_plane_stride > 0 ? b_plane_stride : N * Kp;
  const CUtensorMap am = swap ? make_planes_map(B, N, Kp, bstride, level, BM)
                              : make_planes_map(A, M, Kp, M * Kp, level, BM);
  const CUtensorMap bm = swap ? make_planes_map(A, M, Kp, M * Kp, level, nbt)
                              : make_planes_map(B, N, Kp, bstride, level, narrow ? nbt : BN);
  count_flops(2.0 * (double)M * N * K);
  // the persistent kernel writes an output view itself when K is not split
  const bool epi_view = cview && narrow && splitk == 1;
  float* wsp = (splitk > 1 || (cview && !epi_view)) ? ws : nullptr;
  MatView vnone;
  const MatView& vpass = epi_view ? *cview : vnone;
  if (narrow) {
    static std::once_flag narrow_once;
    cudaError_t e = cudaSuccess;
    std::call_once(narrow_once, [&] {
      auto set = [&](const void* f, int bytes) {
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
      };
      set((const void*)gemm_tc_narrow_kernel<1, 64>, NarrowRing<1, 64>::SMEM_BYTES);
      set((const void*)gemm_tc_narrow_kernel<2, 64>, NarrowRing<2, 64>::SMEM_BYTES);
      set((const void*)gemm_tc_narrow_kernel<3, 64>, NarrowRing<3, 64>::SMEM_BYTES);
      set((const void*)gemm_tc_narrow_kernel<1, 128>, NarrowRing<1, 128>::SMEM_BYTES);
      set((const void*)gemm_tc_narrow_kernel<2, 128>, NarrowRing<2, 128>::SMEM_BYTES);
      set((const void*)gemm_tc_narrow_kernel<3, 128>, NarrowRing<3, 128>::SMEM_BYTES);
    });
    ASCC_CUDA(e);
    const int64_t Mk = swap ? N : M, Nk = swap ? M : N;  // the kernel's product
    const int64_t items = ((Mk + BM - 1) / BM) * ((Nk + nbt - 1) / nbt) * splitk;
    ASCC_REQUIRE(items < (1ll << 31), "gemm_split: too many tiles");
    const unsigned grid = (unsigned)std::min<int64_t>(items, 152);
    const int threads = 32 * NWARPS_N, tr = swap ? 1 : 0;
#define ASCC_NARROW(LV, NBV)                                                                  \
  gemm_tc_narrow_kernel<LV, NBV><<<grid, threads, NarrowRing<LV, NBV>::SMEM_BYTES, s>>>(       \
      am, bm, (int)Mk, (int)Nk, num_kt, kt_chunk, splitk, alpha, beta, C, (long long)ldc, wsp, \
      err, tr, vpass, epi_view ? 1 : 0)
    if (nbt == 64) {
      if (level == 1)
        ASCC_NARROW(1, 64);
      else if (level == 2)
        ASCC_NARROW(2, 64);
      else
        ASCC_NARROW(3, 64);
    } else {
      if (level == 1)
        ASCC_NARROW(1, 128);
      else if (level == 2)
        ASCC_NARROW(2, 128);
      else
        ASCC_NARROW(3, 128);
    }
#undef ASCC_NARROW
    count_launch();
    check_launch("gemm_tc_narrow");
  }
  dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((N + BN - 1) / BN), (unsigned)splitk);
  ASCC_REQUIRE(grid.y <= 65535, "gemm_split: N too large");
  float* w = wsp;
  if (narrow) {
    // launched above
  } else if (level == 1)
    gemm_tc_kernel<1><<<grid, NTHREADS, Ring<1>::SMEM_BYTES, s>>>(
        am, bm, (int)M, (int)N, num_kt, kt_chunk, alpha, beta, C, (long long)ldc, w, err);
  else if (level == 2)
    gemm_tc_kernel<2><<<grid, NTHREADS, Ring<2>::SMEM_BYTES, s>>>(
        am, bm, (int)M, (int)N, num_kt, kt_chunk, alpha, beta, C, (long long)ldc, w, err);
  else
    gemm_tc_kernel<3><<<grid, NTHREADS, Ring<3>::SMEM_BYTES, s>>>(
        am, bm, (int)M, (int)N, num_kt, kt_chunk, alpha, beta, C, (long long)ldc, w, err);
  if (!narrow) {
    count_launch();
    check_launch("gemm_tc");
  }
  if (cview && !epi_view) {
    const MatView& v = *cview;
    ASCC_REQUIRE(M < (1ll << 32) && N < (1ll << 32), "gemm_split: output view too large");
    const bool by_rows = v.kstr[v.nk - 1] != 1 && v.mstr[v.nm - 1] == 1;
    const int64_t outer = by_rows ? N : M, inner = by_rows ? M : N;
    const unsigned gy = (unsigned)std::min<int64_t>(outer, 65535);
    const unsigned gx = (unsigned)std::min<int64_t>((inner + 255) / 256, 64);
    const int mode = host_store_mode(alpha, beta);
#define ASCC_RV(MD)                                                                        \
  splitk_reduce_view_kernel<MD><<<dim3(gx, gy), 256, 0, s>>>(C, v, ws, M, N, splitk, alpha, \
                                                             beta, by_rows)
    if (mode == kStorePow2)
      ASCC_RV(kStorePow2);
    else if (mode == kStoreScaled)
      ASCC_RV(kStoreScaled);
    else if (mode == kStoreBeta1)
      ASCC_RV(kStoreBeta1);
    else
      ASCC_RV(kStoreBeta);
#undef ASCC_RV
    count_launch();
    check_launch("splitk_reduce_view");
  } else if (splitk > 1) {
    const unsigned gy = (unsigned)std::min<int64_t>(M, 65535);
    if (N % 4 == 0 && (reinterpret_cast<uintptr_t>(ws) & 15) == 0) {
      const unsigned gx = (unsigned)std::min<int64_t>((N / 4 + 255) / 256, 64);
      const int mode = host_store_mode(alpha, beta);
#define ASCC_R4(MD)                                                                          \
  splitk_reduce4_kernel<MD><<<dim3(gx, gy), 256, 0, s>>>(C, (long long)ldc, ws, M, N, splitk, \
                                                         alpha, beta)
      if (mode == kStorePow2)
        ASCC_R4(kStorePow2);
      else if (mode == kStoreScaled)
        ASCC_R4(kStoreScaled);
      else if (mode == kStoreBeta1)
        ASCC_R4(kStoreBeta1);
      else
        ASCC_R4(kStoreBeta);
#undef ASCC_R4
    } else {
      const unsigned gx = (unsigned)std::min<int64_t>((N + 255) / 256, 64);
      const int mode = host_store_mode(alpha, beta);
#define ASCC_R1(MD)                                                                        \
  splitk_reduce_kernel<MD><<<dim3(gx, gy), 256, 0, s>>>(C, (long long)ldc, ws, M, N, splitk, \
                                                        alpha, beta)
      if (mode == kStorePow2)
        ASCC_R1(kStorePow2);
      else if (mode == kStoreScaled)
        ASCC_R1(kStoreScaled);
      else if (mode == kStoreBeta1)
        ASCC_R1(kStoreBeta1);
      else
        ASCC_R1(kStoreBeta);
#undef ASCC_R1
    }
    count_launch();
    check_launch("splitk_reduce");
  }
}

}  // namespace tc
}  // namespace ascc
