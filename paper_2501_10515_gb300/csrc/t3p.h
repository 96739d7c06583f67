// The mixed-triples slice T3' of a one-CSF state (arXiv 2501.10515,
// Sec. II.B.1): the alpha-beta-beta triples with at least three primary spin
// orbitals among h-up, h-down, p-up, p-down, their residual R3' and their
// contributions to R1 and R2, with the partial linearisation of Sec. II.C.
//
// Storage.  The packed amplitudes (the order of ascc_t3p_indices: (i, j < k,
// a, b < c) lexicographic) are unpacked into four dense blocks that
// partition the slice by the set of primary spin orbitals an element holds:
//   TA[k][b][c] = t3[h,h,k,p,b,c]            [o][v][v]  (antisymmetric in b, c)
//   TB[k][a][c] = t3[h,h,k,a,p,c], a != p    [o][v][v]
//   TC[j][k][c] = t3[h,j,k,p,p,c], j,k != h  [o][o][v]  (antisymmetric in j, k)
//   TD[i][k][c] = t3[i,h,k,p,p,c], i != h    [o][o][v]
// (zero at every excluded position), and R3' is formed in the same blocks.
//
// Evaluation.  A generated program (t3p_program.inc, written by gen_t3p.py
// from the spin-orbital triples equations) of dense contractions over these
// blocks, the dressed Fock matrix, the dressed DF factor and t2, run through
// the engine's einsum planner.  Contractions that share a large operand with
// the same indices contracted are stacked into one product: their other
// operands are copied into the rows of a stack S, W = X . S^T is one GEMM,
// and each member's result is copied out of its columns of W.  Its four sections are run with the t2
// operand bound to:
//   pro  (R1, R2 from T3'; R3' from [H,T3'])      no t2
//   lin  (R3' from [H,T2])                         T2
//   quad (R3' from 1/2[[H,T2],T2])                 T2, and for PLASCC again
//                                                  with T2^M and weight -1
//   mix  (R3' from [[H,T2],T3'])                   T2 (ASCC) or T2 - T2^M (PLASCC)
#pragma once

#include "engine.h"

namespace ascc {

struct T3pTensor {
  int kind;          // 0 base operand, 1 slice of a base operand, 2 intermediate
  int base;          // base operand index (kinds 0, 1)
  const char* spec;  // slice selector, one character per base dimension
  const char* dims;  // o / v / P per dimension; # = the rows of a stack
  int section;
  const char* rows;  // stacks: '+'-separated dims of each member's rows
};

struct T3pOp {
  int section;
  // 0 slice, 1 contraction into `out`, 2 contraction accumulated into an
  // output, 3 member operand `a` into its rows of stack `out`, 4 member's
  // columns of stacked product `a` into `out` or (out < 0) into an output
  int kind;
  int out, a, b;
  const char* spec;  // einsum labels of a, b and the result; kinds 3, 4: a permutation
  double alpha;
  int base;          // slice: the base operand; accumulate: the output base operand
  const char* outspec;
  int member;        // kinds 3, 4: the member's index in its stack
};

// Base operands of the program, in the order of its tables.
enum T3pBase { T3P_F = 0, T3P_B, T3P_T2, T3P_TS, T3P_TA, T3P_TB, T3P_TC, T3P_TD, T3P_R1,
               T3P_R2, T3P_RA, T3P_RB, T3P_RC, T3P_RD, T3P_NBASE };
enum T3pSection { T3P_PRO = 0, T3P_LIN, T3P_QUAD, T3P_MIX };

// Streams, per-stream planners, events and private output copies of a
// concurrent run (T3pProgram::run_streams); owned by the caller.
struct T3pStreams {
  std::vector<cudaStream_t> streams;          // [0] is the caller's stream
  std::vector<std::unique_ptr<Einsum>> es;    // one planner per stream
  std::vector<cudaEvent_t> op_events;         // one per op
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;              // one per stream
  double* priv = nullptr;                     // [streams][block_elements]
};

// Streams of a concurrent T3' run: ASCC_T3P_STREAMS if set (1 = one
// stream), else the default.
int t3p_streams();

class T3pProgram {
 public:
  // o, v, naux: sizes; h, p: the primary hole and particle; nstreams: the
  // streams a concurrent run may use (the workspace and the plan depend on it).
  T3pProgram(int o, int v, int naux, int h, int p, int nstreams = 1);
  ~T3pProgram();
  T3pProgram(const T3pProgram&) = delete;
  T3pProgram& operator=(const T3pProgram&) = delete;
  // Device workspace of the intermediates (elements of double), with
  // intermediates whose lifetimes do not overlap sharing memory.
  int64_t workspace_elements() const { return ws_elems_; }
  // Runs one section; base[T3pBase] points at the base operands (t2 / ts of
  // the binding of that section); scale multiplies every accumulation.
  void run(Einsum& es, cudaStream_t s, int section, double* const* base, double scale,
           double* ws) const;
  // The same on several streams (dependencies by events, deterministic sums).
  void run_streams(T3pStreams& ex, int section, double* const* base, double scale,
                   double* ws) const;
  int nstreams() const { return nstreams_; }
  // Pairs of ops of a section whose memory footprints conflict but that the
  // stream plan leaves unordered (0 for a race-free plan); drop_waits checks
  // the plan without its event waits (a test of the checker itself).
  int64_t plan_hazards(bool drop_waits = false) const;
  // Pairs of intermediates whose workspace ranges overlap while both are live
  // (0 for a correct placement); collapse places every tensor at offset 0
  // (a test of the check itself).
  int64_t placement_clobbers(bool collapse = false) const;
  // room of each planner's plane cache during a run
  size_t cache_bytes() const {
    return (size_t)std::min<int64_t>(int64_t(1) << 30, ws_elems_ / 2) / 256 * 256;
  }
  int op_count() const;
  // Sizes of the four blocks (elements) and the offsets of TA..TD (RA..RD)
  // in one concatenated buffer.
  int64_t block_elements() const { return blk_off_[4]; }
  bool profiling() const { return profile_path_ != nullptr; }
  int64_t block_offset(int b) const { return blk_off_[b]; }

 private:
  std::vector<int64_t> base_shape(int b) const;
  int64_t dims_extent(const char* dims) const;      // product of o / v / P extents
  int64_t stack_rows(const char* rows, int upto) const;  // rows of the first `upto` members
  void select(int b, const char* spec, int64_t* offset, std::vector<int64_t>& shape,
              std::vector<int64_t>& stride) const;
  void stack_copy(const T3pOp& op, cudaStream_t s, double* const* base, double* const* outb,
                  double scale, double* ws) const;
  void exec_op(int q, Einsum& es, cudaStream_t s, double* const* base, double* const* outb,
               double scale, double* ws, double* tmp) const;
  void plan_streams();
  int o_, v_, n_, naux_, h_, p_;
  std::vector<std::vector<int64_t>> shape_;
  std::vector<int64_t> offset_;  // element offset of each slice / intermediate
  int64_t ws_elems_ = 0, acc_off_ = 0, acc_len_ = 0;
  int nstreams_ = 1;
  std::vector<int> op_stream_;            // planned stream of each op
  std::vector<std::vector<int>> deps_;    // ops each op waits for (latest per stream)
  int64_t blk_off_[5];
  // per-op timing when ASCC_T3P_PROFILE names an output file
  const char* profile_path_ = nullptr;
  mutable std::vector<cudaEvent_t> prof_ev_;
  mutable std::vector<double> prof_ms_;
  mutable std::vector<int> prof_n_;
};

namespace k {
// Packed slice <-> blocks.  dst[q] = element offset of amplitude q in the
// concatenated [TA|TB|TC|TD] buffer, sgn[q] its sign; dst2/sgn2 the
// antisymmetric partner position in TA or TC (-1 if none).
void t3p_unpack(cudaStream_t s, double* blocks, int64_t nblk, const double* t3,
                const int64_t* dst, const int64_t* dst2, const signed char* sgn, int64_t n3);
void t3p_gather(cudaStream_t s, double* r3, const double* blocks, const int64_t* dst,
                const signed char* sgn, int64_t n3);
// out[i] += sum_k part[k * n + i], k = 0..nparts-1 in order
void sum_rows(cudaStream_t s, double* out, const double* part, int64_t n, int nparts);
}  // namespace k

}  // namespace ascc
