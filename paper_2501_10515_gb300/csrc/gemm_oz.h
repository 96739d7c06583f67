// FP64-class GEMM on the BF16 tensor cores by exact integer-slice products
// (the error-free splitting of Ozaki, Ogita and Oishi, with BF16 digits and
// exact FP32 accumulation over bounded K chunks) for sm_103a.
//
// Each row r of an FP64 operand X [rows][K] is scaled by its own power of two
// 2^e_r (max_k |X_rk| < 2^(e_r - 1)) and rounded to a 42-bit integer
// q = rint(X 2^(42 - e_r)), which is written as NSLICE = 6 balanced base-2^7
// digits d_0..d_5 (|d_s| <= 64, exact in BF16).  Plane s stores d_s 2^(-7 s),
// so that X = 2^(e_r - 7) sum_s plane_s up to the 2^(-42) rounding of q.
//
// The product sum_k X_ik Y_jk is assembled from the plane products (s, t)
// with s + t <= 5.  Products of equal s + t = g share one power of two, so
// their K sum is an integer multiple of 2^(-7 g); over a chunk of 1024 K
// values it stays within 2^24 for g <= 3 and the FP32 tensor-core
// accumulator holds it exactly (whatever its rounding mode).  Groups 0..3 get
// one TMEM accumulator each; the groups 4 and 5 (weights 2^-28 and 2^-35)
// share a fifth, whose FP32 rounding (truncating, on this hardware) stays far
// below the digit truncation.  After each chunk the accumulators are folded
// into a 64-bit integer sum in units of 2^-28 (exact for groups 0..3), so the
// only roundings are the digit truncation, the tail accumulator and the final
// conversion to FP64.  Integer partial sums make the result independent of
// the order in which K chunks (and split-K slices) arrive.
//
// Accuracy: 1e-12 to 5e-12 of |A||B| elementwise for rows of even magnitude
// (42-bit fixed point relative to each row's largest entry, products with
// s + t >= 6 left out).
#pragma once

#include <cuda_bf16.h>

#include "common.h"

namespace ascc {
namespace oz {

constexpr int NSLICE = 6;  // digit planes per operand
constexpr int BETA = 7;    // bits per digit
// exponent marking a row that holds a NaN or an infinity
constexpr int32_t kNonFinite = -0x40000000;

// K rounded up to the 32-element K tile of the kernel.
int64_t padded_k(int64_t K);

// Writes the NSLICE digit planes of in [rows][K] (row stride ld) to
// planes[s * plane_stride + r * Kp + k] (zero padded to Kp) and the row
// exponents e_r to exps[r]; plane_stride <= 0 means rows * Kp.
void split(cudaStream_t s, __nv_bfloat16* planes, int32_t* exps, const double* in, int64_t rows,
           int64_t K, int64_t ld, int64_t plane_stride = 0);

// The same from a strided tensor read as the matrix v (rows v.rows(), K =
// v.cols()), without a permuted copy.
void split_view(cudaStream_t s, __nv_bfloat16* planes, int32_t* exps, const double* in,
                const MatView& v, int64_t plane_stride = 0);

// Workspace of gemm(): one 64-bit integer per element of C.
inline size_t ws_bytes(int64_t M, int64_t N) { return sizeof(long long) * (size_t)(M * N); }

// C[M][N] (row stride ldc) = alpha * A B^T + beta * C from the planes of
// A [M][K] and B [N][K] (split()), K split over `splitk` CTAs.  err receives
// a nonzero code if a bounded wait inside the kernel gives up.
void gemm(cudaStream_t s, int64_t M, int64_t N, int64_t K, double alpha, const __nv_bfloat16* A,
          const int32_t* ea, int64_t a_plane_stride, const __nv_bfloat16* B, const int32_t* eb,
          int64_t b_plane_stride, double beta, double* C, int64_t ldc, long long* ws, int* err,
          int splitk = 1);

// Number of K slices that fills the GPU's SMs most evenly for an M x N x K product.
// (fill = false: one slice, the SMs left to concurrent launches.)
int splitk_for(int64_t M, int64_t N, int64_t K, bool fill = true);

// Number of BF16 x BF16 plane products per K step.
constexpr int products() { return NSLICE * (NSLICE + 1) / 2; }

}  // namespace oz
}  // namespace ascc
