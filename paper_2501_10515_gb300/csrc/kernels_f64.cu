// FP64 kernels of the residual engine: a tiled DFMA GEMM, strided copies,
// reductions and the elementwise steps of the amplitude update.
#include <algorithm>
#include <atomic>

#include "kernels.h"

namespace ascc {

static std::atomic<int64_t> g_launches{0};
static std::atomic<double> g_flops{0.0};
namespace {
thread_local int64_t tl_launches = 0;
thread_local double tl_flops = 0.0;
}  // namespace
void count_launch(int64_t n) {
  g_launches += n;
  tl_launches += n;
}
int64_t launch_total() { return g_launches.load(); }
int64_t thread_launches() { return tl_launches; }
void count_flops(double f) {
  tl_flops += f;
  double cur = g_flops.load();
  while (!g_flops.compare_exchange_weak(cur, cur + f)) {
  }
}
double flop_total() { return g_flops.load(); }
double thread_flops() { return tl_flops; }
void check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    throw Error(ASCC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

namespace k {
namespace {

constexpr int TM = 64, TN = 64, TK = 16, NT = 256;

// 64x64 output tile per block, 4x4 per thread (strided), K in steps of 16.
template <bool TA, bool TB>
__global__ void __launch_bounds__(NT)
gemm_f64_kernel(int64_t M, int64_t N, int64_t K, double alpha,
                const double* __restrict__ A, int64_t lda, int64_t sA,
                const double* __restrict__ B, int64_t ldb, int64_t sB,
                double beta, double* __restrict__ C, int64_t ldc, int64_t sC) {
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  const int64_t bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int64_t m0 = (int64_t)blockIdx.y * TM, n0 = (int64_t)blockIdx.x * TN;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int64_t k0 = 0; k0 < K; k0 += TK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int idx = tid + NT * r;
      int mm, kk;
      if (!TA) { mm = idx / TK; kk = idx % TK; } else { kk = idx / TM; mm = idx % TM; }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      double val = 0.0;
      if (gm < M && gk < K) val = TA ? A[gk * lda + gm] : A[gm * lda + gk];
      As[kk][mm] = val;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int idx = tid + NT * r;
      int nn, kk;
      if (!TB) { kk = idx / TN; nn = idx % TN; } else { nn = idx / TK; kk = idx % TK; }
      const int64_t gn = n0 + nn, gk = k0 + kk;
      double val = 0.0;
      if (gn < N && gk < K) val = TB ? B[gn * ldb + gk] : B[gk * ldb + gn];
      Bs[kk][nn] = val;
    }
    __syncthreads();
    auto step = [&](int kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    };
    if (K - k0 >= TK) {
#pragma unroll
      for (int kk = 0; kk < TK; ++kk) step(kk);
    } else {
      // last, partial K tile: the zero-filled rows would only add 0 * 0 on
      // the FP64 units, the scarce ones on this part (a K = 1 outer product
      // would pay 16 times its work)
      const int kn = (int)(K - k0);
      for (int kk = 0; kk < kn; ++kk) step(kk);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
    // the row's four old values of C are loaded before its first store
    double old[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gn = n0 + tx + 16 * j;
      old[j] = (beta != 0.0 && gn < N) ? C[gm * ldc + gn] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      C[gm * ldc + gn] = (beta == 0.0) ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * old[j]);
    }
  }
}

// C = alpha * sum_z ws[z] + beta * C for z slices of M x N (fixed summation order).
__global__ void reduce_slices_kernel(double* C, int64_t ldc, const double* ws, int64_t M,
                                     int64_t N, int z, double alpha, double beta) {
  const int64_t total = M * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int q = 0; q < z; ++q) acc += ws[(int64_t)q * total + idx];
    const int64_t m = idx / N, n = idx % N;
    double* c = C + m * ldc + n;
    *c = (beta == 0.0) ? alpha * acc : fma(alpha, acc, beta * *c);
  }
}

struct Strides {
  int nd;
  int64_t shape[8];
  int64_t istride[8];
  int64_t ostride[8];
};

__global__ void strided_copy_kernel(double* __restrict__ out, const double* __restrict__ in,
                                    int64_t total, Strides st, double alpha, double beta) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = idx, ioff = 0, ooff = 0;
    for (int d = st.nd - 1; d >= 0; --d) {
      const int64_t c = rem % st.shape[d];
      rem /= st.shape[d];
      ioff += c * st.istride[d];
      ooff += c * st.ostride[d];
    }
    const double val = alpha * in[ioff];
    out[ooff] = (beta == 0.0) ? val : val + beta * out[ooff];
  }
}

// Row-wise copy: the last dimension is walked by the threads (len values per
// row, `per` rows per block pass), the outer index is decomposed once per row.
// Long rows are cut into nseg segments of seglen values, so that a few long
// rows still spread over the whole GPU.  PLAIN (alpha = 1, beta = 0) moves the
// bits without FP64 arithmetic.  I is the type of the row-index arithmetic:
// 32-bit whenever rows * nseg < 2^31 (the divisions are then a few times
// cheaper), 64-bit otherwise.
template <bool PLAIN, typename I>
__global__ void copy_rows_kernel(double* __restrict__ out, const double* __restrict__ in,
                                 int64_t rows, int len, int per, Strides st, int64_t is_last,
                                 int64_t os_last, double alpha, double beta, int nseg,
                                 int seglen) {
  const int sub = threadIdx.x / (blockDim.x / per), t = threadIdx.x % (blockDim.x / per);
  const int width = blockDim.x / per;
  const I units = (I)rows * (I)nseg;
  for (I u = (I)blockIdx.x * per + sub; u < units; u += (I)gridDim.x * per) {
    const I row = u / (I)nseg;
    const int jb = (int)(u - row * (I)nseg) * seglen;
    const int je = min(len, jb + seglen);
    I rem = row;
    int64_t ioff = 0, ooff = 0;
    for (int d = st.nd - 1; d >= 0; --d) {
      const I sh = (I)st.shape[d];
      const I c = rem % sh;
      rem /= sh;
      ioff += (int64_t)c * st.istride[d];
      ooff += (int64_t)c * st.ostride[d];
    }
    // four independent loads in flight per thread
    for (int j0 = jb + t; j0 < je; j0 += 4 * width) {
      // the four inputs (and, with beta, the four old outputs) are loaded
      // before the first store
      double v[4], old[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = j0 + q * width;
        v[q] = (j < je) ? in[ioff + j * is_last] : 0.0;
        old[q] = (!PLAIN && beta != 0.0 && j < je) ? out[ooff + j * os_last] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = j0 + q * width;
        if (j < je) {
          double* o = out + ooff + j * os_last;
          if (PLAIN) *o = v[q];
          else *o = (beta == 0.0) ? alpha * v[q] : fma(alpha, v[q], beta * old[q]);
        }
      }
    }
  }
}

// Tiled transpose: dimension a is contiguous in the input and the last
// dimension b in the output; 32 x 32 tiles go through shared memory so that
// both the loads and the stores are coalesced.  The other dimensions (st)
// are decomposed once per tile, in 32-bit arithmetic (I) whenever the tile
// count is below 2^31.
template <bool PLAIN, typename I>
__global__ void copy_transpose_kernel(double* __restrict__ out, const double* __restrict__ in,
                                      int64_t na, int64_t nb, int64_t outer, Strides st,
                                      int64_t is_b, int64_t os_a, double alpha, double beta) {
  __shared__ double tile[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const I ta_n = (I)((na + 31) / 32), tb_n = (I)((nb + 31) / 32);
  const I ntiles = (I)outer * ta_n * tb_n;
  for (I tid = blockIdx.x; tid < ntiles; tid += gridDim.x) {
    const I tq = tid / tb_n;
    const I tb = tid - tq * tb_n, ta = tq % ta_n, q = tq / ta_n;
    I rem = q;
    int64_t ioff = 0, ooff = 0;
    for (int d = st.nd - 1; d >= 0; --d) {
      const I sh = (I)st.shape[d];
      const I c = rem % sh;
      rem /= sh;
      ioff += (int64_t)c * st.istride[d];
      ooff += (int64_t)c * st.ostride[d];
    }
    const int64_t a0 = (int64_t)ta * 32, b0 = (int64_t)tb * 32;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t a = a0 + tx, b = b0 + ty + 8 * i;
      if (a < na && b < nb) tile[ty + 8 * i][tx] = in[ioff + a + b * is_b];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t b = b0 + tx, a = a0 + ty + 8 * i;
      if (a < na && b < nb) {
        const double v = tile[tx][ty + 8 * i];
        double* o = out + ooff + a * os_a + b;
        if (PLAIN) *o = v;
        else *o = (beta == 0.0) ? alpha * v : fma(alpha, v, beta * *o);
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

// One (x, y) column per thread: its K values of A stay in registers and all J
// outputs are formed from W in shared memory; the old values of C are loaded
// eight at a time before their stores.  Reads A once and C once: HBM-bound
// in FP32, FP64-unit-bound in FP64.
template <typename CT>
__global__ void axis_matrix_kernel(double* __restrict__ C, const double* __restrict__ A,
                                   const double* __restrict__ W, int64_t X, int K, int J,
                                   int64_t Y, double alpha, double beta) {
  __shared__ CT w[32 * 32];
  for (int e = threadIdx.x; e < K * J; e += blockDim.x) w[e] = (CT)W[e];
  __syncthreads();
  const int64_t total = X * Y;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = idx / Y, y = idx - x * Y;
    const double* a = A + x * (int64_t)K * Y + y;
    double* c = C + x * (int64_t)J * Y + y;
    CT av[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) av[k] = k < K ? (CT)a[k * Y] : CT(0);
    for (int j0 = 0; j0 < J; j0 += 8) {
      double old[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        old[u] = (beta != 0.0 && j0 + u < J) ? c[(int64_t)(j0 + u) * Y] : 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + u;
        if (j < J) {
          CT acc = CT(0);
#pragma unroll
          for (int k = 0; k < 32; ++k)
            if (k < K) acc = fma_t(av[k], w[k * J + j], acc);
          const double r = (double)acc;
          c[(int64_t)j * Y] = (beta == 0.0) ? alpha * r : fma(alpha, r, beta * old[u]);
        }
      }
    }
  }
}

__global__ void gemv_rows_kernel(int64_t M, int64_t K, double alpha, const double* __restrict__ A,
                                 int64_t lda, const double* __restrict__ x, double beta,
                                 double* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  for (int64_t m = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; m < M;
       m += (int64_t)gridDim.x * blockDim.x / 32) {
    const double* a = A + m * lda;
    double acc = 0.0;
    for (int64_t k = lane; k < K; k += 32) acc = fma(a[k], x[k], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) y[m] = (beta == 0.0) ? alpha * acc : fma(alpha, acc, beta * y[m]);
  }
}

// Short rows (K <= 8): one thread per row.
__global__ void gemv_short_kernel(int64_t M, int64_t K, double alpha, const double* __restrict__ A,
                                  int64_t lda, const double* __restrict__ x, double beta,
                                  double* __restrict__ y) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
       m += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t k = 0; k < K; ++k) acc = fma(A[m * lda + k], x[k], acc);
    y[m] = (beta == 0.0) ? alpha * acc : fma(alpha, acc, beta * y[m]);
  }
}

// out = alpha * a * b + beta * out over an nd-dimensional box walked in the
// output's row-major order (astride / bstride 0 where a label is absent).
struct OuterStrides {
  int nd;
  int64_t shape[8], astride[8], bstride[8], ostride[8];
};

template <typename I>
__global__ void outer_kernel(double* __restrict__ out, const double* __restrict__ a,
                             const double* __restrict__ b, int64_t total, OuterStrides st,
                             double alpha, double beta) {
  for (I idx = blockIdx.x * (I)blockDim.x + threadIdx.x; idx < (I)total;
       idx += (I)gridDim.x * blockDim.x) {
    I rem = idx;
    int64_t ao = 0, bo = 0, oo = 0;
    for (int d = st.nd - 1; d >= 0; --d) {
      const I e = (I)st.shape[d], q = rem / e;
      const int64_t c = (int64_t)(rem - q * e);
      rem = q;
      ao += c * st.astride[d];
      bo += c * st.bstride[d];
      oo += c * st.ostride[d];
    }
    const double val = alpha * a[ao] * b[bo];
    out[oo] = (beta == 0.0) ? val : val + beta * out[oo];
  }
}

__global__ void gemv_cols_kernel(int64_t M, int64_t K, double alpha, const double* __restrict__ A,
                                 int64_t lda, const double* __restrict__ x, double beta,
                                 double* __restrict__ y) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
       m += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t k = 0; k < K; ++k) acc = fma(A[k * lda + m], x[k], acc);
    y[m] = (beta == 0.0) ? alpha * acc : fma(alpha, acc, beta * y[m]);
  }
}

// Transposed matrix-vector product, first pass: block (x, y) sums rows
// [y kchunk, (y+1) kchunk) of A (K x M, row stride lda) times x for 32
// consecutive columns (one per lane, coalesced), 8 rows at a time, into
// part[y][m]; gemv_t_reduce adds the chunks in a fixed order.
__global__ void gemv_t_partial(int64_t M, int64_t K, const double* __restrict__ A, int64_t lda,
                               const double* __restrict__ x, int64_t kchunk,
                               double* __restrict__ part) {
  __shared__ double sh[8][33];
  const int64_t m = blockIdx.x * 32 + threadIdx.x;
  const int64_t k0 = blockIdx.y * kchunk, k1 = min(K, k0 + kchunk);
  double acc = 0.0;
  if (m < M)
    for (int64_t k = k0 + threadIdx.y; k < k1; k += 8) acc = fma(A[k * lda + m], x[k], acc);
  sh[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && m < M) {
    double t = 0.0;
    for (int r = 0; r < 8; ++r) t += sh[r][threadIdx.x];
    part[blockIdx.y * M + m] = t;
  }
}

// Row matrix-vector product for few, long rows, first pass: block (c, m)
// sums chunk c of row m (256 threads, a fixed tree order) into part[c][m].
__global__ void gemv_n_partial(int64_t M, int64_t K, const double* __restrict__ A, int64_t lda,
                               const double* __restrict__ x, int64_t kchunk,
                               double* __restrict__ part) {
  __shared__ double sh[8];
  const int64_t m = blockIdx.y, k0 = blockIdx.x * kchunk, k1 = min(K, k0 + kchunk);
  const double* a = A + m * lda;
  double acc = 0.0;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) acc = fma(a[k], x[k], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sh[w];
    part[blockIdx.x * M + m] = t;
  }
}

__global__ void gemv_t_reduce(int64_t M, int nchunk, const double* __restrict__ part,
                              double alpha, double beta, double* __restrict__ y) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
       m += (int64_t)gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int c = 0; c < nchunk; ++c) t += part[c * M + m];
    y[m] = (beta == 0.0) ? alpha * t : fma(alpha, t, beta * y[m]);
  }
}

__global__ void fill_kernel(double* x, double v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}

__global__ void axpby_kernel(double* y, const double* x, double a, double b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (b == 0.0) ? a * x[i] : fma(a, x[i], b * y[i]);
}

constexpr int RB = 256;       // reduction block
constexpr int RG = 4 * 152;   // reduction grid (4 blocks per SM)

__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  v = (threadIdx.x < blockDim.x / 32) ? sh[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double nanmax(double a, double b) {
  return (b > a || b != b) ? b : a;  // keeps NaN
}

__device__ double block_max(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  v = (threadIdx.x < blockDim.x / 32) ? sh[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// partial[row][block] = sum over this block's grid-stride share of x . Y[row]
__global__ void dot_rows_partial(const double* __restrict__ x, const double* __restrict__ Y,
                                 int64_t ldy, int64_t n, double* __restrict__ partial) {
  __shared__ double sh[32];
  const int row = blockIdx.y;
  const double* y = Y + row * ldy;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc = fma(x[i], y[i], acc);
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[row * gridDim.x + blockIdx.x] = acc;
}

__global__ void sum_partials(const double* __restrict__ partial, int parts, double* out) {
  __shared__ double sh[32];
  const int row = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < parts; i += blockDim.x) acc += partial[row * parts + i];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) out[row] = acc;
}

__global__ void maxabs_partial(const double* __restrict__ x, int64_t n, double* partial) {
  __shared__ double sh[32];
  double m = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double a = fabs(x[i]);
    m = (a > m || a != a) ? a : m;  // propagate NaN
  }
  m = block_max(m, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = m;
}

__global__ void max_partials(const double* partial, int parts, double* out) {
  __shared__ double sh[32];
  double m = 0.0;
  for (int i = threadIdx.x; i < parts; i += blockDim.x) {
    const double a = partial[i];
    m = (a > m || a != a) ? a : m;
  }
  m = block_max(m, sh);
  if (threadIdx.x == 0) out[0] = m;
}

__global__ void lincomb_kernel(double* y, const double* X, int64_t ldx, const double* c,
                               int m, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int kk = 0; kk < m; ++kk) acc = fma(c[kk], X[kk * ldx + i], acc);
    y[i] = acc;
  }
}

// DIIS on the device (one thread; m <= 32).  Stores the new Gram row of slot
// a.slot[a.cnt-1] (row[q] = e_new . e_q for every slot q) into gram[m][m];
// with a.solve set, solves the bordered system
//   [[G/s + 1e-12 I, 1], [1, 0]] [c; l] = [0; 1],  s = max |diag G|,
// over the active slots (in a.slot order) by Gaussian elimination with
// partial pivoting and writes c to coef[slot] (0 for inactive slots).  A
// degenerate or non-finite system sets *fail = 1 and coef = e_new.
__global__ void diis_kernel(double* gram, const double* row, DiisArgs a, double* coef,
                            double* fail) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int m = a.m, cnt = a.cnt, nw = a.slot[cnt - 1];
  for (int q = 0; q < cnt; ++q) {
    const int sq = a.slot[q];
    gram[nw * m + sq] = row[sq];
    gram[sq * m + nw] = row[sq];
  }
  if (!a.solve) return;
  for (int q = 0; q < m; ++q) coef[q] = 0.0;
  double A[33 * 33], b[33], x[33];
  const int nn = cnt + 1;
  double scale = 0.0;
  for (int i = 0; i < cnt; ++i) scale = fmax(scale, fabs(gram[a.slot[i] * m + a.slot[i]]));
  bool ok = scale > 0.0 && isfinite(scale);
  if (ok) {
    for (int i = 0; i < nn * nn; ++i) A[i] = 0.0;
    for (int i = 0; i < nn; ++i) b[i] = 0.0;
    for (int i = 0; i < cnt; ++i) {
      for (int j = 0; j < cnt; ++j)
        A[i * nn + j] = gram[a.slot[i] * m + a.slot[j]] / scale + (i == j ? 1e-12 : 0.0);
      A[i * nn + cnt] = 1.0;
      A[cnt * nn + i] = 1.0;
    }
    b[cnt] = 1.0;
    for (int col = 0; col < nn && ok; ++col) {
      int piv = col;
      for (int r = col + 1; r < nn; ++r)
        if (fabs(A[r * nn + col]) > fabs(A[piv * nn + col])) piv = r;
      if (fabs(A[piv * nn + col]) < 1e-300) {
        ok = false;
        break;
      }
      if (piv != col) {
        for (int j = 0; j < nn; ++j) {
          const double t = A[col * nn + j];
          A[col * nn + j] = A[piv * nn + j];
          A[piv * nn + j] = t;
        }
        const double t = b[col];
        b[col] = b[piv];
        b[piv] = t;
      }
      for (int r = col + 1; r < nn; ++r) {
        const double f = A[r * nn + col] / A[col * nn + col];
        for (int j = col; j < nn; ++j) A[r * nn + j] = __dsub_rn(A[r * nn + j], __dmul_rn(f, A[col * nn + j]));
        b[r] = __dsub_rn(b[r], __dmul_rn(f, b[col]));
      }
    }
    if (ok) {
      for (int r = nn - 1; r >= 0; --r) {
        double acc = b[r];
        for (int j = r + 1; j < nn; ++j) acc = __dsub_rn(acc, __dmul_rn(A[r * nn + j], x[j]));
        x[r] = acc / A[r * nn + r];
      }
      for (int i = 0; i < nn; ++i) ok = ok && isfinite(x[i]);
    }
  }
  if (ok) {
    for (int i = 0; i < cnt; ++i) coef[a.slot[i]] = x[i];
  } else {
    coef[nw] = 1.0;
    *fail = 1.0;
  }
}

// L = 1 + x - t1m - t1m x ;  R = 1 - x + t1m - x t1m   (t1m[o+a][i] = t1[i][a])
__global__ void build_LR_kernel(double* L, double* R, const double* t1, int o, int v,
                                int hole, int particle, double xv) {
  const int n = o + v;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * n;
       idx += gridDim.x * blockDim.x) {
    const int r = idx / n, c = idx % n;
    double l = (r == c) ? 1.0 : 0.0, rr = l;
    if (r >= o && c < o) {  // virtual row, occupied column: -t1m / +t1m
      const double t = t1[c * v + (r - o)];
      l -= t;
      rr += t;
    }
    if (hole >= 0) {
      const int p = o + particle;
      if (r == hole && c == p) { l += xv; rr -= xv; }
      if (r >= o && c == p) l -= t1[hole * v + (r - o)] * xv;      // (t1m x)[o+a][p]
      if (r == hole && c < o) rr -= xv * t1[c * v + particle];     // (x t1m)[h][i]
    }
    L[idx] = l;
    R[idx] = rr;
  }
}

__global__ void tilde_kernel(double* u, const double* t, int o, int v) {
  const int64_t vv = (int64_t)v * v, total = (int64_t)o * o * vv;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ab = idx % vv, ij = idx / vv;
    const int64_t i = ij / o, j = ij % o;
    u[idx] = 2.0 * t[idx] - t[(j * o + i) * vv + ab];
  }
}

__global__ void mixed_mask_kernel(double* m, const double* t, int o, int v, int hole,
                                  int particle) {
  const int64_t total = (int64_t)o * o * v * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = idx;
    const int b = (int)(r % v); r /= v;
    const int a = (int)(r % v); r /= v;
    const int j = (int)(r % o); r /= o;
    const int i = (int)r;
    const int cnt = (i == hole) + (j == hole) + (a == particle) + (b == particle);
    m[idx] = (cnt >= 1 && cnt <= 3) ? t[idx] : 0.0;
  }
}

__device__ __forceinline__ int64_t pair_row(int i, int j, int o) {
  return (int64_t)i * o - (int64_t)i * (i - 1) / 2 + (j - i);
}

__global__ void gather_pairs_kernel(double* tpair, const double* t, int o, int64_t vv) {
  const int64_t npair = (int64_t)o * (o + 1) / 2, total = npair * vv;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = idx / vv, c = idx % vv;
    // invert p = i o - i (i - 1) / 2 + (j - i) by walking i (o is small)
    int i = 0;
    int64_t base = 0;
    while (base + (o - i) <= p) {
      base += o - i;
      ++i;
    }
    const int j = i + (int)(p - base);
    tpair[idx] = t[((int64_t)i * o + j) * vv + c];
  }
}

__global__ void scatter_pairs_kernel(double* Y, const double* Yvv, int o, int v, int n) {
  const int64_t vv = (int64_t)v * v, total = (int64_t)o * o * vv;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = idx;
    const int b = (int)(r % v); r /= v;
    const int a = (int)(r % v); r /= v;
    const int j = (int)(r % o);
    const int i = (int)(r / o);
    const double y = (i <= j) ? Yvv[pair_row(i, j, o) * vv + (int64_t)a * v + b]
                              : Yvv[pair_row(j, i, o) * vv + (int64_t)b * v + a];
    Y[(((int64_t)i * o + j) * n + o + a) * v + b] = y;
  }
}

// Denominators: bare eps for the primary amplitudes (every index h or p) of a
// one-CSF state and for the ground state; eps_eff (h and p at their mean) for
// all other amplitudes of a one-CSF state.
__global__ void jacobi_kernel(double* tn, double* e, const double* t, const double* r,
                              const double* eps, const double* eps_eff, int o, int v, int hole,
                              int particle, const int32_t* t3idx, int64_t n3) {
  const int64_t n1 = (int64_t)o * v, n2 = n1 * n1, total = n1 + n2 + n3;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    double D;
    if (idx < n1) {
      const int i = (int)(idx / v), a = (int)(idx % v);
      const double* ee = (i == hole && a == particle) ? eps : eps_eff;
      D = ee[i] - ee[o + a];
    } else if (idx < n1 + n2) {
      int64_t q = idx - n1;
      const int b = (int)(q % v); q /= v;
      const int a = (int)(q % v); q /= v;
      const int j = (int)(q % o); q /= o;
      const int i = (int)q;
      const bool prim = i == hole && j == hole && a == particle && b == particle;
      const double* ee = prim ? eps : eps_eff;
      D = ee[i] + ee[j] - ee[o + a] - ee[o + b];
    } else {
      const int32_t* ix = t3idx + 6 * (idx - n1 - n2);
      D = eps_eff[ix[0]] + eps_eff[ix[1]] + eps_eff[ix[2]] - eps_eff[o + ix[3]] -
          eps_eff[o + ix[4]] - eps_eff[o + ix[5]];
    }
    const double step = r[idx] / D;
    tn[idx] = t[idx] + step;
    e[idx] = step;
  }
}

// Pair step of a one-CSF state: (t1[i][a], t2[i][h][a][p]) solve a 2 x 2
// model Jacobian [[-D1, c F_hp], [q, -D2]] (see jacobi_pairs in kernels.h).
__global__ void pair_step_kernel(double* tn, double* e, const double* t, const double* r,
                                 const double* eps_eff, const double* F, int o, int v, int hole,
                                 int particle) {
  const int n = o + v;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= o * v) return;
  const int i = idx / v, a = idx % v, h = hole, p = particle;
  const int64_t n1 = (int64_t)o * v, vv = (int64_t)v * v;
  const double fhp = F[(int64_t)h * n + o + p], fph = F[(int64_t)(o + p) * n + h];
  double J00, J01, J10, J11;
  if (i == h && a == p) {
    J00 = 0.0; J01 = fhp; J10 = 2.0 * fhp; J11 = 0.0;
  } else {
    const bool mixed = (i == h) || (a == p);
    J00 = -(eps_eff[i] - eps_eff[o + a]);
    J11 = -(eps_eff[i] + eps_eff[h] - eps_eff[o + a] - eps_eff[o + p]);
    J01 = (mixed ? 1.0 : 2.0) * fhp;
    J10 = mixed ? fph : 0.0;
  }
  const double det = J00 * J11 - J01 * J10;
  const double mx = fmax(fmax(fabs(J00), fabs(J01)), fmax(fabs(J10), fabs(J11)));
  if (!(fabs(det) > 1e-12 * mx * mx)) return;  // keep the diagonal step
  const int64_t q1 = (int64_t)i * v + a;
  const int64_t q2 = n1 + (((int64_t)i * o + h) * v + a) * v + p;
  const int64_t q2s = n1 + (((int64_t)h * o + i) * v + p) * v + a;
  const double r1 = r[q1], r2 = r[q2];
  const double d1 = -(J11 * r1 - J01 * r2) / det;
  const double d2 = -(-J10 * r1 + J00 * r2) / det;
  tn[q1] = t[q1] + d1;
  e[q1] = d1;
  tn[q2] = t[q2] + d2;
  e[q2] = d2;
  if (q2s != q2) {
    tn[q2s] = t[q2s] + d2;
    e[q2s] = d2;
  }
  (void)vv;
}

// out[r][j] = M[r][cols[j]] - (r == cols[j]) for an n x n matrix M.
__global__ void cols_minus_identity_kernel(double* out, const double* M, int n, int c0, int nlo,
                                           int extra, int nc) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * nc;
       idx += gridDim.x * blockDim.x) {
    const int r = idx / nc, j = idx % nc;
    const int c = j < nlo ? c0 + j : extra;
    out[idx] = M[(int64_t)r * n + c] - (r == c ? 1.0 : 0.0);
  }
}

__global__ void diag_sum_kernel(double* d, const double* B, int naux, int n, int o) {
  const int P = blockIdx.x * blockDim.x + threadIdx.x;
  if (P >= naux) return;
  const double* b = B + (int64_t)P * n * n;
  double acc = 0.0;
  for (int kk = 0; kk < o; ++kk) acc += b[kk * n + kk];
  d[P] = acc;
}

__global__ void reference_energy_kernel(double* out, const double* h, int n, const double* g,
                                        int o) {
  __shared__ double sh[32];
  double acc = 0.0;
  const int64_t o2 = (int64_t)o * o;
  for (int64_t idx = threadIdx.x; idx < o2; idx += blockDim.x) {
    const int64_t i = idx / o, j = idx % o;
    // g[i][i][j][j] and g[i][j][j][i] of an o^4 block
    acc += 2.0 * g[((i * o + i) * o + j) * o + j] - g[((i * o + j) * o + j) * o + i];
  }
  for (int i = threadIdx.x; i < o; i += blockDim.x) acc += 2.0 * h[(int64_t)i * n + i];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) out[0] = acc;
}

int grid_for(int64_t n, int block = 256) {
  int64_t g = (n + block - 1) / block;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

void gemm_f64(cudaStream_t s, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
              const double* A, int64_t lda, int64_t sA, const double* B, int64_t ldb,
              int64_t sB, double beta, double* C, int64_t ldc, int64_t sC, int64_t batch) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (K <= 0) {
    // an empty contraction: C = beta C on a contiguous batch of M x N blocks
    ASCC_REQUIRE(ldc == N && (batch == 1 || sC == M * N), "gemm_f64: K = 0 needs contiguous C");
    if (beta == 0.0) fill(s, C, 0.0, M * N * batch);
    else axpby(s, C, C, 0.0, beta, M * N * batch);
    return;
  }
  count_flops(2.0 * (double)M * (double)N * (double)K * (double)batch);
  // split K over the grid when the output has too few 64 x 64 tiles to fill the
  // GPU: K is cut into z equal chunks (z divides K), each chunk's product goes
  // to its own FP64 slice and the slices are summed in a fixed order
  const int64_t tiles = ((M + TM - 1) / TM) * ((N + TN - 1) / TN);
  if (batch == 1 && tiles < 152 && K >= 256) {
    int64_t zmax = std::min<int64_t>(2 * 152 / tiles, K / 64);
    int64_t z = 1;
    for (int64_t c = zmax; c >= 2; --c)
      if (K % c == 0) {
        z = c;
        break;
      }
    if (z >= 2) {
      const int64_t kc = K / z;
      double* ws = nullptr;
      ASCC_CUDA(cudaMallocAsync(&ws, sizeof(double) * (size_t)(z * M * N), s));
      gemm_f64(s, ta, tb, M, N, kc, 1.0, A, lda, ta ? kc * lda : kc, B, ldb, tb ? kc : kc * ldb,
               0.0, ws, N, M * N, z);
      count_flops(-2.0 * (double)M * (double)N * (double)K);  // counted above already
      reduce_slices_kernel<<<grid_for(M * N), 256, 0, s>>>(C, ldc, ws, M, N, (int)z, alpha, beta);
      count_launch();
      check_launch("reduce_slices");
      ASCC_CUDA(cudaFreeAsync(ws, s));
      return;
    }
  }
  dim3 grid((unsigned)((N + TN - 1) / TN), (unsigned)((M + TM - 1) / TM), 1);
  for (int64_t b0 = 0; b0 < batch; b0 += 65535) {
    const int64_t nb = std::min<int64_t>(65535, batch - b0);
    grid.z = (unsigned)nb;
    const double* Ab = A + b0 * sA;
    const double* Bb = B + b0 * sB;
    double* Cb = C + b0 * sC;
    if (!ta && !tb)
      gemm_f64_kernel<false, false><<<grid, NT, 0, s>>>(M, N, K, alpha, Ab, lda, sA, Bb, ldb, sB, beta, Cb, ldc, sC);
    else if (ta && !tb)
      gemm_f64_kernel<true, false><<<grid, NT, 0, s>>>(M, N, K, alpha, Ab, lda, sA, Bb, ldb, sB, beta, Cb, ldc, sC);
    else if (!ta && tb)
      gemm_f64_kernel<false, true><<<grid, NT, 0, s>>>(M, N, K, alpha, Ab, lda, sA, Bb, ldb, sB, beta, Cb, ldc, sC);
    else
      gemm_f64_kernel<true, true><<<grid, NT, 0, s>>>(M, N, K, alpha, Ab, lda, sA, Bb, ldb, sB, beta, Cb, ldc, sC);
    count_launch();
  }
  check_launch("gemm_f64");
}

void outer(cudaStream_t s, double* out, const int64_t* out_stride, const double* a,
           const int64_t* a_stride, const double* b, const int64_t* b_stride, int nd,
           const int64_t* shape, double alpha, double beta) {
  ASCC_REQUIRE(nd >= 0 && nd <= 8, "outer: 0..8 dimensions");
  OuterStrides st;
  st.nd = 0;
  int64_t total = 1;
  for (int d = 0; d < nd; ++d) {
    total *= shape[d];
    if (shape[d] == 1) continue;
    st.shape[st.nd] = shape[d];
    st.astride[st.nd] = a_stride[d];
    st.bstride[st.nd] = b_stride[d];
    st.ostride[st.nd] = out_stride[d];
    ++st.nd;
  }
  if (total == 0) return;
  const int g = grid_for(total);
  if (total + 256ll * g < (1ll << 32))
    outer_kernel<uint32_t><<<g, 256, 0, s>>>(out, a, b, total, st, alpha, beta);
  else
    outer_kernel<int64_t><<<g, 256, 0, s>>>(out, a, b, total, st, alpha, beta);
  count_launch();
  check_launch("outer");
}

void strided_copy(cudaStream_t s, double* out, const int64_t* out_stride, const double* in,
                  const int64_t* in_stride, int nd, const int64_t* shape, double alpha,
                  double beta) {
  ASCC_REQUIRE(nd >= 1 && nd <= 8, "strided_copy: 1..8 dimensions");
  // drop unit dimensions
  int64_t sh[8], is[8], os[8];
  int m = 0;
  int64_t total = 1;
  for (int d = 0; d < nd; ++d) {
    total *= shape[d];
    if (shape[d] == 1) continue;
    sh[m] = shape[d];
    is[m] = in_stride[d];
    os[m] = out_stride[d];
    ++m;
  }
  if (total == 0) return;
  if (m == 0) {
    sh[0] = 1;
    is[0] = os[0] = 1;
    m = 1;
  }
  // merge neighbouring dimensions that are contiguous on both sides
  {
    int w = 0;
    for (int d = 1; d < m; ++d) {
      if (is[w] == is[d] * sh[d] && os[w] == os[d] * sh[d] && sh[w] * sh[d] <= (1ll << 30)) {
        sh[w] *= sh[d];
        is[w] = is[d];
        os[w] = os[d];
      } else {
        ++w;
        sh[w] = sh[d];
        is[w] = is[d];
        os[w] = os[d];
      }
    }
    m = w + 1;
  }
  const bool plain = alpha == 1.0 && beta == 0.0;
  const int last = m - 1;
  // the input-contiguous dimension, if it is not the last one
  int a = -1;
  for (int d = 0; d < last; ++d)
    if (is[d] == 1) a = d;
  if (os[last] == 1 && is[last] != 1 && a >= 0 && out != in && sh[last] >= 8 && sh[a] >= 8) {
    Strides st;
    st.nd = 0;
    int64_t outer = 1;
    for (int d = 0; d < last; ++d) {
      if (d == a) continue;
      st.shape[st.nd] = sh[d];
      st.istride[st.nd] = is[d];
      st.ostride[st.nd] = os[d];
      ++st.nd;
      outer *= sh[d];
    }
    const int64_t tiles = outer * ((sh[a] + 31) / 32) * ((sh[last] + 31) / 32);
    const int g = (int)std::min<int64_t>(tiles, 152 * 16);
    const bool narrow = tiles < ((int64_t)1 << 31);
    if (plain && narrow)
      copy_transpose_kernel<true, uint32_t><<<g, dim3(32, 8), 0, s>>>(
          out, in, sh[a], sh[last], outer, st, is[last], os[a], alpha, beta);
    else if (plain)
      copy_transpose_kernel<true, int64_t><<<g, dim3(32, 8), 0, s>>>(
          out, in, sh[a], sh[last], outer, st, is[last], os[a], alpha, beta);
    else if (narrow)
      copy_transpose_kernel<false, uint32_t><<<g, dim3(32, 8), 0, s>>>(
          out, in, sh[a], sh[last], outer, st, is[last], os[a], alpha, beta);
    else
      copy_transpose_kernel<false, int64_t><<<g, dim3(32, 8), 0, s>>>(
          out, in, sh[a], sh[last], outer, st, is[last], os[a], alpha, beta);
  } else if (os[last] == 1 || is[last] == 1) {
    // rows along the last dimension (coalesced on at least one side)
    Strides st;
    st.nd = last;
    int64_t rows = 1;
    for (int d = 0; d < last; ++d) {
      st.shape[d] = sh[d];
      st.istride[d] = is[d];
      st.ostride[d] = os[d];
      rows *= sh[d];
    }
    const int len = (int)sh[last];
    // threads per row: about four values each, 32..256; the rest of the block
    // takes further rows
    int width = 32;
    while (width < 256 && 4 * width < len) width *= 2;
    const int per = 256 / width;
    // fewer rows than the 2432 blocks of a full grid: cut the rows into
    // segments of at least 1024 values (a multiple of one 4 x 256 pass)
    int nseg = 1, seglen = len;
    if (per == 1 && rows < 152 * 16 && len > 2048) {
      const int64_t want = std::min<int64_t>((152 * 16 + rows - 1) / rows, (len + 1023) / 1024);
      seglen = (int)(((len + want - 1) / want + 1023) / 1024 * 1024);
      nseg = (len + seglen - 1) / seglen;
    }
    const int64_t blocks = (rows * nseg + per - 1) / per;
    const int g = (int)std::min<int64_t>(blocks, 152 * 16);
    // 32-bit row arithmetic needs rows * nseg plus one grid stride below 2^31
    const bool narrow = rows * nseg + (int64_t)g * per < ((int64_t)1 << 31);
    if (plain && narrow)
      copy_rows_kernel<true, uint32_t><<<g, 256, 0, s>>>(out, in, rows, len, per, st, is[last],
                                                         os[last], alpha, beta, nseg, seglen);
    else if (plain)
      copy_rows_kernel<true, int64_t><<<g, 256, 0, s>>>(out, in, rows, len, per, st, is[last],
                                                        os[last], alpha, beta, nseg, seglen);
    else if (narrow)
      copy_rows_kernel<false, uint32_t><<<g, 256, 0, s>>>(out, in, rows, len, per, st, is[last],
                                                          os[last], alpha, beta, nseg, seglen);
    else
      copy_rows_kernel<false, int64_t><<<g, 256, 0, s>>>(out, in, rows, len, per, st, is[last],
                                                         os[last], alpha, beta, nseg, seglen);
  } else {
    Strides st;
    st.nd = m;
    for (int d = 0; d < m; ++d) {
      st.shape[d] = sh[d];
      st.istride[d] = is[d];
      st.ostride[d] = os[d];
    }
    strided_copy_kernel<<<grid_for(total), 256, 0, s>>>(out, in, total, st, alpha, beta);
  }
  count_launch();
  check_launch("strided_copy");
}

void axis_matrix(cudaStream_t s, bool fp32, double* C, const double* A, const double* W,
                 int64_t X, int K, int J, int64_t Y, double alpha, double beta) {
  ASCC_REQUIRE(K >= 1 && K <= 32 && J >= 1 && J <= 32, "axis_matrix: K and J in 1..32");
  const int64_t total = X * Y;
  if (total <= 0) return;
  count_flops(2.0 * (double)total * K * J);
  const int g = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  if (fp32)
    axis_matrix_kernel<float><<<g, 256, 0, s>>>(C, A, W, X, K, J, Y, alpha, beta);
  else
    axis_matrix_kernel<double><<<g, 256, 0, s>>>(C, A, W, X, K, J, Y, alpha, beta);
  count_launch();
  check_launch("axis_matrix");
}

void gemv_f64(cudaStream_t s, bool ta, int64_t M, int64_t K, double alpha, const double* A,
              int64_t lda, const double* x, double beta, double* y) {
  if (M <= 0) return;
  if (ta && K > 64) {
    // K split over the grid so that a long, narrow product still fills the GPU
    const int64_t gx = (M + 31) / 32;
    int64_t nchunk = std::max<int64_t>(1, std::min<int64_t>((152 * 8 + gx - 1) / gx, (K + 63) / 64));
    nchunk = std::min<int64_t>(nchunk, 4096);
    const int64_t kchunk = (K + nchunk - 1) / nchunk;
    nchunk = (K + kchunk - 1) / kchunk;
    double* part = nullptr;
    ASCC_CUDA(cudaMallocAsync(&part, sizeof(double) * (size_t)(nchunk * M), s));
    gemv_t_partial<<<dim3((unsigned)gx, (unsigned)nchunk), dim3(32, 8), 0, s>>>(M, K, A, lda, x,
                                                                               kchunk, part);
    gemv_t_reduce<<<grid_for(M), 256, 0, s>>>(M, (int)nchunk, part, alpha, beta, y);
    ASCC_CUDA(cudaFreeAsync(part, s));
    count_launch(2);
    check_launch("gemv_t");
    return;
  }
  if (!ta && M < 152 * 16 && K >= 2048) {
    // few long rows (down to a single dot product): chunks of each row over
    // the grid, summed in a fixed order
    const int64_t want = (152 * 8 + M - 1) / M;
    int64_t nchunk = std::max<int64_t>(1, std::min<int64_t>(want, K / 2048));
    const int64_t kchunk = (K + nchunk - 1) / nchunk;
    nchunk = (K + kchunk - 1) / kchunk;
    double* part = nullptr;
    ASCC_CUDA(cudaMallocAsync(&part, sizeof(double) * (size_t)(nchunk * M), s));
    gemv_n_partial<<<dim3((unsigned)nchunk, (unsigned)M), 256, 0, s>>>(M, K, A, lda, x, kchunk,
                                                                      part);
    gemv_t_reduce<<<grid_for(M), 256, 0, s>>>(M, (int)nchunk, part, alpha, beta, y);
    ASCC_CUDA(cudaFreeAsync(part, s));
    count_launch(2);
    check_launch("gemv_n");
    return;
  }
  if (ta)
    gemv_cols_kernel<<<grid_for(M), 256, 0, s>>>(M, K, alpha, A, lda, x, beta, y);
  else if (K <= 8)
    gemv_short_kernel<<<grid_for(M), 256, 0, s>>>(M, K, alpha, A, lda, x, beta, y);
  else
    gemv_rows_kernel<<<(int)std::min<int64_t>((M * 32 + 255) / 256, 152 * 16), 256, 0, s>>>(
        M, K, alpha, A, lda, x, beta, y);
  count_launch();
  check_launch("gemv_f64");
}

void fill(cudaStream_t s, double* x, double v, int64_t n) {
  if (n <= 0) return;
  fill_kernel<<<grid_for(n), 256, 0, s>>>(x, v, n);
  count_launch();
  check_launch("fill");
}

void axpby(cudaStream_t s, double* y, const double* x, double a, double b, int64_t n) {
  if (n <= 0) return;
  axpby_kernel<<<grid_for(n), 256, 0, s>>>(y, x, a, b, n);
  count_launch();
  check_launch("axpby");
}

void dot_rows(cudaStream_t s, const double* x, const double* Y, int64_t ldy, int rows, int64_t n,
              double* out, double* work) {
  if (rows <= 0) return;
  dim3 g(RG, rows);
  dot_rows_partial<<<g, RB, 0, s>>>(x, Y, ldy, n, work);
  sum_partials<<<rows, RB, 0, s>>>(work, RG, out);
  count_launch(2);
  check_launch("dot_rows");
}

void maxabs(cudaStream_t s, const double* x, int64_t n, double* out, double* work) {
  maxabs_partial<<<RG, RB, 0, s>>>(x, n, work);
  max_partials<<<1, RB, 0, s>>>(work, RG, out);
  count_launch(2);
  check_launch("maxabs");
}

void diis(cudaStream_t s, double* gram, const double* row, const DiisArgs& a, double* coef,
          double* fail) {
  diis_kernel<<<1, 32, 0, s>>>(gram, row, a, coef, fail);
  count_launch();
  check_launch("diis");
}

void lincomb(cudaStream_t s, double* y, const double* X, int64_t ldx, const double* c, int m,
             int64_t n) {
  lincomb_kernel<<<grid_for(n), 256, 0, s>>>(y, X, ldx, c, m, n);
  count_launch();
  check_launch("lincomb");
}

void build_LR(cudaStream_t s, double* L, double* R, const double* t1, int o, int v, int hole,
              int particle, double xval) {
  const int n = o + v;
  build_LR_kernel<<<grid_for((int64_t)n * n), 256, 0, s>>>(L, R, t1, o, v, hole, particle, xval);
  count_launch();
  check_launch("build_LR");
}

void tilde(cudaStream_t s, double* u, const double* t, int o, int v) {
  tilde_kernel<<<grid_for((int64_t)o * o * v * v), 256, 0, s>>>(u, t, o, v);
  count_launch();
  check_launch("tilde");
}

void gather_pairs(cudaStream_t s, double* tpair, const double* t, int o, int64_t vv) {
  const int64_t total = (int64_t)o * (o + 1) / 2 * vv;
  if (!total) return;
  gather_pairs_kernel<<<grid_for(total), 256, 0, s>>>(tpair, t, o, vv);
  count_launch();
  check_launch("gather_pairs");
}

void scatter_pairs(cudaStream_t s, double* Y, const double* Yvv, int o, int v, int n) {
  const int64_t total = (int64_t)o * o * v * v;
  if (!total) return;
  scatter_pairs_kernel<<<grid_for(total), 256, 0, s>>>(Y, Yvv, o, v, n);
  count_launch();
  check_launch("scatter_pairs");
}

void mixed_mask(cudaStream_t s, double* m, const double* t, int o, int v, int hole, int particle) {
  mixed_mask_kernel<<<grid_for((int64_t)o * o * v * v), 256, 0, s>>>(m, t, o, v, hole, particle);
  count_launch();
  check_launch("mixed_mask");
}

void jacobi(cudaStream_t s, double* tn, double* e, const double* t, const double* r,
            const double* eps, const double* eps_eff, int o, int v, int hole, int particle,
            const int32_t* t3idx, int64_t n3) {
  const int64_t total = (int64_t)o * v + (int64_t)o * o * v * v + n3;
  jacobi_kernel<<<grid_for(total), 256, 0, s>>>(tn, e, t, r, eps, eps_eff, o, v, hole, particle,
                                                t3idx, n3);
  count_launch();
  check_launch("jacobi");
}

void cols_minus_identity(cudaStream_t s, double* out, const double* M, int n, int nlo, int extra,
                         int nc) {
  cols_minus_identity_kernel<<<grid_for((int64_t)n * nc), 256, 0, s>>>(out, M, n, 0, nlo, extra,
                                                                        nc);
  count_launch();
  check_launch("cols_minus_identity");
}

void jacobi_pairs(cudaStream_t s, double* tn, double* e, const double* t, const double* r,
                  const double* eps_eff, const double* F, int o, int v, int hole, int particle) {
  if (hole < 0) return;
  pair_step_kernel<<<(o * v + 127) / 128, 128, 0, s>>>(tn, e, t, r, eps_eff, F, o, v, hole,
                                                       particle);
  count_launch();
  check_launch("pair_step");
}

void diag_sum(cudaStream_t s, double* d, const double* B, int naux, int n, int o) {
  diag_sum_kernel<<<(naux + 127) / 128, 128, 0, s>>>(d, B, naux, n, o);
  count_launch();
  check_launch("diag_sum");
}

void reference_energy(cudaStream_t s, double* out, const double* h, int n, const double* goooo,
                      int o) {
  reference_energy_kernel<<<1, 256, 0, s>>>(out, h, n, goooo, o);
  count_launch();
  check_launch("reference_energy");
}

}  // namespace k
}  // namespace ascc
