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
#include <mutex>

#include "gemm_tc.h"
#include "tc_ptx.cuh"

namespace ascc {
namespace tc {
namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4, NTHREADS = 128;
constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int TMEM_COLS = 256;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
static_assert(BM * (BN + 1) * 4 <= STAGES * STAGE_BYTES, "the epilogue tile reuses the ring");

struct Segs {
  int n;
  int a[6];
  int b[6];
};

using namespace ptx;

__global__ void __launch_bounds__(NTHREADS, 1)
gemm_tc_kernel(const __grid_constant__ CUtensorMap a0, const __grid_constant__ CUtensorMap a1,
               const __grid_constant__ CUtensorMap a2, const __grid_constant__ CUtensorMap b0,
               const __grid_constant__ CUtensorMap b1, const __grid_constant__ CUtensorMap b2,
               Segs segs, int M, int N, int num_kt, int kt_chunk, double alpha, double beta,
               double* __restrict__ C, long long ldc, float* __restrict__ ws, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + STAGES * STAGE_BYTES);
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
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_holder;
  // split K: this CTA covers k-tiles [kt0, kt0 + nkt) of every segment
  const int kt0 = blockIdx.z * kt_chunk;
  const int nkt = max(0, min(kt_chunk, num_kt - kt0));
  const int total = segs.n * nkt;

  if (warp == 0 && lane == 0) {
    // TMA producer
    const CUtensorMap* am[3] = {&a0, &a1, &a2};
    const CUtensorMap* bm[3] = {&b0, &b1, &b2};
    for (int it = 0; it < total; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (uint32_t)((it / STAGES) & 1);
      if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, err, 1)) {
        abort_flag = 1;
        break;
      }
      if (*(volatile int*)&abort_flag) break;
      const int seg = it / nkt, kt = kt0 + it % nkt;
      const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
      mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
      tma_load_2d(sa, am[segs.a[seg]], full0 + 8 * s, kt * BK, m0);
      tma_load_2d(sa + A_BYTES, bm[segs.b[seg]], full0 + 8 * s, kt * BK, n0);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    for (int it = 0; it < total; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (uint32_t)((it / STAGES) & 1);
      if (!mbar_wait(full0 + 8 * s, ph, err, 2)) {
        abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint64_t ad = sw128_desc(sa + kk * 32);
        const uint64_t bd = sw128_desc(sa + A_BYTES + kk * 32);
        mma_bf16(tmem, ad, bd, idesc, (it > 0 || kk > 0) ? 1u : 0u);
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
#pragma unroll
        for (int j = 0; j < 16; ++j) tile[lrow * PITCH + c0 + j] = __uint_as_float(r[j]);
      }
    }
    __syncthreads();
    const int rows = min(BM, M - m0);
    for (int rr = 0; rr < rows; ++rr) {
      const long long row = m0 + rr;
      for (int c = threadIdx.x; c < BN; c += NTHREADS) {
        const int col = n0 + c;
        if (col >= N) break;
        const float a = total > 0 ? tile[rr * PITCH + c] : 0.f;
        if (ws) {
          // split-K partial, summed later
          ws[((long long)blockIdx.z * M + row) * N + col] = a;
        } else {
          double* cp = C + row * ldc + col;
          const double acc = (double)a;
          *cp = (beta == 0.0) ? alpha * acc : fma(alpha, acc, beta * *cp);
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

// C = alpha * sum_z ws[z] + beta * C.  The FP32 partials are summed in FP32
// with a compensation term (Fast2Sum), i.e. to about 2^-48 relative, in a
// fixed order, and converted to FP64 once: the FP64 units are the scarce
// ones on this part.
__global__ void splitk_reduce_kernel(double* __restrict__ C, long long ldc,
                                     const float* __restrict__ ws, long long M, long long N,
                                     int nz, double alpha, double beta) {
  const long long total = M * N;
  for (long long m = blockIdx.y; m < M; m += gridDim.y) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
      const long long idx = m * N + n;
      float hi = 0.f, lo = 0.f;
      for (int z = 0; z < nz; ++z) {
        const float x = ws[(long long)z * total + idx];
        const float t = hi + x;
        lo += (fabsf(hi) >= fabsf(x)) ? (hi - t) + x : (x - t) + hi;
        hi = t;
      }
      const double acc = (double)hi + (double)lo;
      double* c = C + m * ldc + n;
      *c = (beta == 0.0) ? alpha * acc : fma(alpha, acc, beta * *c);
    }
  }
}

// FP64 [rows][K] (row stride ld) -> nsplit BF16 planes [nsplit][rows][Kp], zero padded.
// The value is rounded to FP32 once (24 significant bits, as many as three
// planes hold) and split with exact FP32 subtractions.  Each thread converts a
// run of 8 consecutive values of one row and writes 16 bytes per plane.
__global__ void split_bf16_kernel(__nv_bfloat16* __restrict__ out, const double* __restrict__ in,
                                  long long rows, long long K, long long ld, long long Kp,
                                  int nsplit, long long plane_stride) {
  const long long runs = Kp / 8, total = rows * runs;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long r = idx / runs, k0 = (idx - r * runs) * 8;
    const double* x = in + r * ld + k0;
    float f[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) f[j] = (k0 + j < K) ? (float)x[j] : 0.f;
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

CUtensorMap make_map(const __nv_bfloat16* base, int64_t rows, int64_t Kp, int box_rows) {
  CUtensorMap m;
  cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(Kp * 2)};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
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
  split_bf16_kernel<<<g, 256, 0, s>>>(out, in, rows, K, ld, Kp, nsplit, plane_stride);
  count_launch();
  check_launch("split_bf16");
}

int products_for(int level) { return level == 1 ? 1 : level == 2 ? 3 : 6; }

int splitk_for(int64_t M, int64_t N, int64_t K) {
  // K chunks of at most 2048 (FP32 accumulation error ~ 2^-24 sqrt(K/16) per chunk),
  // and enough CTAs to fill the GPU for small M x N
  const int64_t tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  const int64_t num_kt = (K + BK - 1) / BK;
  int64_t z = (K + 2047) / 2048;
  while (tiles * z < 2 * 152 && z < num_kt) ++z;
  return (int)std::min<int64_t>(std::max<int64_t>(z, 1), std::min<int64_t>(num_kt, 512));
}

void gemm_split(cudaStream_t s, int64_t M, int64_t N, int64_t K, int level, double alpha,
                const __nv_bfloat16* A, const __nv_bfloat16* B, double beta, double* C, int64_t ldc,
                int* err, int splitk, float* ws, int64_t b_plane_stride) {
  ASCC_REQUIRE(level >= 1 && level <= 3, "split level 1..3");
  ASCC_REQUIRE(M > 0 && N > 0 && K > 0, "gemm_split: empty");
  ASCC_REQUIRE(splitk >= 1 && (splitk == 1 || ws), "gemm_split: split-K needs a workspace");
  static std::once_flag attr_once;
  cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [&] {
    attr_err = cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    SMEM_BYTES);
  });
  ASCC_CUDA(attr_err);
  const int64_t Kp = padded_k(K);
  CUtensorMap am[3], bm[3];
  for (int u = 0; u < 3; ++u) {
    const int uu = u < level ? u : 0;
    am[u] = make_map(A + (int64_t)uu * M * Kp, M, Kp, BM);
    bm[u] = make_map(B + (int64_t)uu * (b_plane_stride > 0 ? b_plane_stride : N * Kp), N, Kp, BN);
  }
  // products with the small planes first (accumulated before the large ones)
  Segs sg;
  if (level == 1) {
    sg = {1, {0}, {0}};
  } else if (level == 2) {
    sg = {3, {1, 0, 0}, {0, 1, 0}};
  } else {
    sg = {6, {2, 1, 0, 1, 0, 0}, {0, 1, 2, 0, 1, 0}};
  }
  count_flops(2.0 * (double)M * N * K);
  const int num_kt = (int)(Kp / BK);
  const int kt_chunk = (num_kt + splitk - 1) / splitk;
  dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((N + BN - 1) / BN), (unsigned)splitk);
  ASCC_REQUIRE(grid.y <= 65535, "gemm_split: N too large");
  gemm_tc_kernel<<<grid, NTHREADS, SMEM_BYTES, s>>>(am[0], am[1], am[2], bm[0], bm[1], bm[2], sg,
                                                    (int)M, (int)N, num_kt, kt_chunk, alpha, beta,
                                                    C, (long long)ldc, splitk > 1 ? ws : nullptr,
                                                    err);
  count_launch();
  check_launch("gemm_tc");
  if (splitk > 1) {
    const unsigned gx = (unsigned)std::min<int64_t>((N + 255) / 256, 64);
    const unsigned gy = (unsigned)std::min<int64_t>(M, 65535);
    splitk_reduce_kernel<<<dim3(gx, gy), 256, 0, s>>>(C, (long long)ldc, ws, M, N, splitk, alpha,
                                                     beta);
    count_launch();
    check_launch("splitk_reduce");
  }
}

}  // namespace tc
}  // namespace ascc
