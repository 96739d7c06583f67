// Device-side addressing of a MatView (common.h): the offset of a row and the
// eight values of a column run, for the kernels that split an operand into
// BF16 planes straight from a permuted tensor.
#pragma once

#include "common.h"

namespace ascc {

// I: the type of the index arithmetic (32-bit whenever the extents allow:
// a 64-bit division is a long instruction sequence).
template <typename I = long long>
__device__ __forceinline__ long long matview_row(const MatView& v, I r) {
  long long off = 0;
  for (int d = v.nm - 1; d >= 0; --d) {
    const I e = (I)v.mext[d];
    const I q = r / e;
    off += (long long)(r - q * e) * v.mstr[d];
    r = q;
  }
  return off;
}

// x[j] = element (row, k0 + j) for k0 + j < K, else 0; row points at the
// row's first element.  When the last column dimension is contiguous and a
// multiple of 8 long (fast), a run that starts at a multiple of 8 stays in it.
template <typename I = long long>
__device__ __forceinline__ void matview_run8(const MatView& v, const double* __restrict__ row,
                                             long long k0, long long K, bool fast, double* x) {
  long long idx[4] = {0, 0, 0, 0};
  long long off = 0;
  I rem = (I)k0;
  for (int d = v.nk - 1; d >= 0; --d) {
    const I e = (I)v.kext[d];
    const I q = rem / e;
    idx[d] = (long long)(rem - q * e);
    off += idx[d] * v.kstr[d];
    rem = q;
  }
  if (fast && k0 + 8 <= K) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = row[off + j];
    return;
  }
  const int L = v.nk - 1;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    x[j] = (k0 + j < K) ? row[off] : 0.0;
    int d = L;
    ++idx[d];
    off += v.kstr[d];
    while (d > 0 && idx[d] == v.kext[d]) {
      off -= v.kext[d] * v.kstr[d];
      idx[d] = 0;
      --d;
      ++idx[d];
      off += v.kstr[d];
    }
  }
}

}  // namespace ascc

namespace ascc {

// Transposing tile loader for views whose contiguous dimension is on the
// row side: a 64-row x 32-column tile of the matrix goes through shared memory
// (tile[k][m], zero outside the matrix), read with consecutive threads on
// consecutive rows.  Block of 256 threads; roff / coff are scratch tables of
// 64 and 32 offsets (-1 outside).
constexpr int kViewTileM = 64, kViewTileK = 32;

__device__ __forceinline__ void matview_load_tile_t(const MatView& v, const double* __restrict__ in,
                                                    long long rows, long long K, long long m0,
                                                    long long k0,
                                                    double (*tile)[kViewTileM + 1],
                                                    long long* roff, long long* coff) {
  const int t = threadIdx.x;
  if (t < kViewTileM) roff[t] = (m0 + t < rows) ? matview_row(v, m0 + t) : -1;
  if (t >= 128 && t < 128 + kViewTileK) {
    const int c = t - 128;
    long long k = k0 + c, off = -1;
    if (k < K) {
      off = 0;
      for (int d = v.nk - 1; d >= 0; --d) {
        const long long q = k / v.kext[d];
        off += (k - q * v.kext[d]) * v.kstr[d];
        k = q;
      }
    }
    coff[c] = off;
  }
  __syncthreads();
  const int mi = t & (kViewTileM - 1), kq = t >> 6;
  const long long r = roff[mi];
#pragma unroll
  for (int i = 0; i < kViewTileK / 4; ++i) {
    const int k = kq + 4 * i;
    const long long c = coff[k];
    tile[k][mi] = (r >= 0 && c >= 0) ? in[r + c] : 0.0;
  }
  __syncthreads();
}

}  // namespace ascc
