// Split-precision BF16 tensor-core GEMM (tcgen05/TMA/TMEM) for sm_103a.
#pragma once

#include <cuda_bf16.h>

#include "common.h"

namespace ascc {
namespace tc {

// Kp: K rounded up to the 64-element K tile of the kernel.
int64_t padded_k(int64_t K);

// Number of BF16 x BF16 products a split level uses (1, 3 or 6).
int products_for(int level);

// out[s * plane_stride + r * Kp + k] = s-th BF16 plane of in[r][k] (row stride
// ld), zero padded to Kp; s < nsplit; plane_stride <= 0 means rows * Kp.
// x = sum_s plane_s up to the FP32 rounding of x and the last plane's rounding.
void split_bf16(cudaStream_t s, __nv_bfloat16* out, const double* in, int64_t rows, int64_t K,
                int64_t ld, int nsplit, int64_t plane_stride = 0);

// The same planes of a strided tensor read as the matrix v (rows v.rows(),
// K = v.cols()), without a permuted copy.
void split_bf16_view(cudaStream_t s, __nv_bfloat16* out, const double* in, const MatView& v,
                     int nsplit, int64_t plane_stride = 0);

// One split for split_bf16_pair: the planes [nsplit][v.rows()][Kp] of `in`
// read as the matrix v (a plain [rows][K] operand with row stride ld is the
// view nm = nk = 1, mstr = ld, kstr = 1).
struct SplitSpec {
  __nv_bfloat16* out;
  const double* in;
  MatView v;
  int nsplit;
};
// Both splits of one product in one launch (either may be null).
void split_bf16_pair(cudaStream_t s, const SplitSpec* a, const SplitSpec* b);

// C[M][N] (FP64, row stride ldc) = alpha * A B^T + beta * C with A [level][M][Kp] and
// B [level][N][Kp] BF16 planes from split_bf16 (K-major).  err: device int that
// receives a nonzero code if a bounded wait inside the kernel gives up.
// splitk > 1 splits K over the grid: each chunk's FP32 accumulator goes to
// ws [splitk][M][N] (FP32) and the chunks are summed in FP64 afterwards, which
// bounds the FP32 accumulation error by the chunk length.
// b_plane_stride: elements between B's planes (<= 0: N * Kp, i.e. packed planes),
// so that a row block of a larger plane set can serve as B.
// cview: C written through a view (rows over its M dimensions, columns over
// its column dimensions; ldc unused), the partials always going through ws.
// tile: the kernel's tile shape (TileShape).  For a given splitk every shape
// accumulates each element over the same K tiles in the same order, so the
// choice does not change the result, except that kTile64 (and the size rules)
// exchange the operands for M <= 64 < N, which changes the order of the
// tensor core's sums; the autotuner leaves those products to the rules.
enum TileShape {
  kTileRules = -1,  // the size rules alone (no tuning: no allocation, no sync)
  kTileAuto = 0,    // the autotuner's choice for the shape class, else the rules
  kTileWide = 1,    // 128 x 256, one tile per CTA
  kTile128 = 2,     // persistent, 128 x 128
  kTile64 = 3       // persistent, 128 x 64 (operands exchanged for M <= 64 < N)
};
void gemm_split(cudaStream_t s, int64_t M, int64_t N, int64_t K, int level, double alpha,
                const __nv_bfloat16* A, const __nv_bfloat16* B, double beta, double* C,
                int64_t ldc, int* err, int splitk = 1, float* ws = nullptr,
                int64_t b_plane_stride = 0, const MatView* cview = nullptr,
                int tile = kTileAuto);

// Autotuner of the tile shape (ASCC_AUTOTUNE=0 turns it off): the first
// product of a shape class (level, and M, N, K per chunk and split-K rounded
// to powers of two) on a stream that is not being captured runs once per
// candidate shape into scratch memory, timed with CUDA events, and the
// fastest is kept for the class.  Products above 2^25 output elements or
// below 10^8 flops keep the size rules.  Returns the number of classes tuned.
int64_t autotuned_classes();

// Runs one bounded wait that cannot complete (see ascc_selftest_bounded_wait)
// with a budget of limit_ms and returns the code it recorded (0: none).
int wait_selftest(cudaStream_t s, int limit_ms);

// Number of K chunks the residual engine uses for an M x N x K product.
// fill: the work items (tiles x chunks) aimed for; fewer chunks leave the SMs
// to concurrent launches.
int splitk_for(int64_t M, int64_t N, int64_t K, int fill = 2 * 152);

}  // namespace tc
}  // namespace ascc
