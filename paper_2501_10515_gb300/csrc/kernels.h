// Launchers of the FP64 device kernels used by the residual engine.
#pragma once

#include "common.h"

namespace ascc {
namespace k {

// C[b] = alpha * op(A[b]) * op(B[b]) + beta * C[b], row-major, batch strides in
// elements (stride 0 broadcasts an operand).  op(A) is M x K, op(B) is K x N.
void gemm_f64(cudaStream_t s, bool ta, bool tb, int64_t M, int64_t N, int64_t K,
              double alpha, const double* A, int64_t lda, int64_t sA,
              const double* B, int64_t ldb, int64_t sB, double beta, double* C,
              int64_t ldc, int64_t sC, int64_t batch);

// y[m] = alpha * sum_k op(A)[m][k] x[k] + beta * y[m] (op(A) is M x K;
// ta: A stored K x M).  A warp per row (ta = false) or a thread per row.
// C[x][j][y] = alpha sum_k A[x][k][y] W[k][j] + beta C[x][j][y] (row-major;
// K, J <= 32): a small matrix applied along one axis of a large tensor, read
// and written in place.  fp32 = false sums in FP64 in ascending k (the order
// of gemm_f64); fp32 = true rounds A and W to FP32 and sums in FP32.
void axis_matrix(cudaStream_t s, bool fp32, double* C, const double* A, const double* W,
                 int64_t X, int K, int J, int64_t Y, double alpha, double beta);
void gemv_f64(cudaStream_t s, bool ta, int64_t M, int64_t K, double alpha, const double* A,
              int64_t lda, const double* x, double beta, double* y);

// out[strided] = alpha * a[strided] * b[strided] + beta * out over an
// nd-dimensional box (an outer product, or a scaled copy when b's strides are 0).
void outer(cudaStream_t s, double* out, const int64_t* out_stride, const double* a,
           const int64_t* a_stride, const double* b, const int64_t* b_stride, int nd,
           const int64_t* shape, double alpha, double beta);

// out[strided] = alpha * in[strided] + beta * out over an nd-dimensional
// index box `shape` (strides in elements, one per dimension).
void strided_copy(cudaStream_t s, double* out, const int64_t* out_stride,
                  const double* in, const int64_t* in_stride, int nd,
                  const int64_t* shape, double alpha, double beta);

void fill(cudaStream_t s, double* x, double v, int64_t n);
void axpby(cudaStream_t s, double* y, const double* x, double a, double b, int64_t n);  // y = a x + b y

// Deterministic reductions; results land in device memory.
void dot_rows(cudaStream_t s, const double* x, const double* Y, int64_t ldy,
              int rows, int64_t n, double* out, double* work);  // out[r] = x . Y[r]
void maxabs(cudaStream_t s, const double* x, int64_t n, double* out, double* work);

// DIIS step on the device (Sec. III.B): slot[cnt-1] is the newest slot, the
// others the active history in age order; see diis_kernel.
struct DiisArgs {
  int m, cnt, solve;
  int slot[32];
};
void diis(cudaStream_t s, double* gram, const double* row, const DiisArgs& a, double* coef,
          double* fail);

// y = sum_k c[k] * X[k]  (c in device memory)
void lincomb(cudaStream_t s, double* y, const double* X, int64_t ldx,
             const double* c, int m, int64_t n);

// Dressing matrices L = (1 - t1)(1 + x), R = (1 - x)(1 + t1) as n x n row-major
// (x[h][o+p] = xval; hole < 0 means x = 0).
void build_LR(cudaStream_t s, double* L, double* R, const double* t1, int o,
              int v, int hole, int particle, double xval);

// u = 2 t - t^(i<->j) for t[o][o][v][v]
void tilde(cudaStream_t s, double* u, const double* t, int o, int v);

// m = t where 1 <= #primary spatial indices <= 3, else 0 (Eq. pnm split).
void mixed_mask(cudaStream_t s, double* m, const double* t, int o, int v,
                int hole, int particle);

// Jacobi step (Sec. III.B): tn = t + r / D and e = tn - t over the packed
// vector [t1 | t2 | t3'].  D uses eps for the primary amplitudes of a one-CSF
// state (hole >= 0) and eps_eff (h and p at their mean) for the others.
void jacobi(cudaStream_t s, double* tn, double* e, const double* t,
            const double* r, const double* eps, const double* eps_eff, int o,
            int v, int hole, int particle, const int32_t* t3idx, int64_t n3);

// out[r][j] = M[r][c_j] - delta(r, c_j) for the columns c_j = j (j < nlo) and
// c_j = extra (j = nlo, when nc = nlo + 1) of an n x n matrix M.
void cols_minus_identity(cudaStream_t s, double* out, const double* M, int n, int nlo, int extra,
                         int nc);

// Overwrites the steps of the pairs (t1[i][a], t2[i][h][a][p] = t2[h][i][p][a])
// of a one-CSF state with the solution of the 2 x 2 model Jacobian
//   [[-D1, c F_hp], [q, -D2]]  (c = 2, q = 0 if i != h and a != p; c = 1,
//   q = F_ph if exactly one of them is primary; [[0, F_hp], [2 F_hp, 0]] for
//   (h, p)), D from eps_eff and F the dressed Fock matrix (n x n).  A
//   near-singular pair keeps its diagonal step.  No-op for hole < 0.
void jacobi_pairs(cudaStream_t s, double* tn, double* e, const double* t, const double* r,
                  const double* eps_eff, const double* F, int o, int v, int hole, int particle);

// Pair-symmetric ladder operands (t_ji^dc = t_ij^cd, (ac|bd) = (bd|ac) give
// Y_ji^{ba} = Y_ij^{ab}): gather_pairs packs the rows t[i][j][:] (vv values)
// of the pairs i <= j, row p = i o - i (i - 1) / 2 + (j - i); scatter_pairs
// writes Y[i][j][o+a][b] (Y [o][o][n][v]) from the pair products
// Yvv[p][a][b], transposing a and b for i > j.
void gather_pairs(cudaStream_t s, double* tpair, const double* t, int o, int64_t vv);
void scatter_pairs(cudaStream_t s, double* Y, const double* Yvv, int o, int v, int n);

// d[P] = sum_k B[P][k][k]
void diag_sum(cudaStream_t s, double* d, const double* B, int naux, int n, int o);

// out[0] = 2 sum_i h[i][i] + sum_ij (2 g[i][i][j][j] - g[i][j][j][i]) for
// g = oooo block (o^4) and h n x n.
void reference_energy(cudaStream_t s, double* out, const double* h, int n,
                      const double* goooo, int o);

}  // namespace k
}  // namespace ascc
