// Residual engine of libascc: the einsum planner, the per-molecule bare
// integrals, the per-state amplitude iteration.
#pragma once

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.h"

namespace ascc {

// Contracts two dense row-major tensors on the device: C = alpha A.B + beta C
// with single-character index labels ("ijcd,acbd->ijab").  Labels shared by
// A, B and C are batched, labels of A and C (B and C) form the GEMM rows
// (columns), labels of A and B only are summed.  Operands are permuted into
// GEMM order only when their layout is not already usable.
class Einsum {
 public:
  explicit Einsum(cudaStream_t s) : s_(s) {}
  void operator()(const char* spec, double alpha, const T& A, const T& B, double beta,
                  const T& C) const;
  // C = alpha * permute(A) + beta * C, spec "kilj->klij"
  void perm(const char* spec, double alpha, const T& A, double beta, const T& C) const;
  // level 0: FP64 DFMA GEMM.  level 1..3: unbatched contractions of at least
  // min_flops run on the BF16 tensor cores with operands split into `level`
  // BF16 planes (1, 3 or 6 products); level 4: the same contractions as exact
  // digit-plane products (FP64-class); err receives kernel timeout codes.
  void set_split(int level, int* err, double min_flops = 4e7) {
    level_ = level;
    err_ = err;
    min_flops_ = min_flops;
  }
  int level() const { return level_; }
  int* err() const { return err_; }
  double min_flops() const { return min_flops_; }
  // Scratch of the tensor-core path, grown on demand and reused by every call
  // on this stream (calls on one stream never overlap).
  void* scratch(int which, size_t bytes) const;
  // While frozen (a CUDA graph capture), the scratch must not be reallocated:
  // a request beyond its size is an error instead.
  void freeze(bool on) const { frozen_ = on; }
  // Plane cache of the tensor-core path.  set_keys names the operands of the
  // next call (-1: none): a key promises that the operand's values stay the
  // same until the next cache_reset, so that planes split from it with the
  // same arrangement and level are reused.  cache_reset empties the cache and
  // gives it `bytes` of room (kept when it already has that much).
  void set_keys(int64_t a, int64_t b) const {
    key_a_ = a;
    key_b_ = b;
  }
  void cache_reset(size_t bytes) const;
  // Work items a split-K product aims for (tiles x K chunks); 0: no chunks
  // beyond the accuracy rule (launches on concurrent streams fill the SMs).
  void set_fill(int items) const { fill_ = items; }
  int fill() const { return fill_; }

 private:
  struct CacheEntry {
    int64_t key;
    std::string sig;
    size_t off;
  };
  mutable std::vector<CacheEntry> cache_;
  mutable DevBuf cache_buf_;
  mutable size_t cache_used_ = 0;
  mutable int64_t key_a_ = -1, key_b_ = -1;
  mutable int fill_ = 2 * 152;
  cudaStream_t s_;
  mutable bool frozen_ = false;
  int level_ = 0;
  int* err_ = nullptr;
  double min_flops_ = 4e7;
  mutable DevBuf scratch_[5];
};

// Copies a strided box of `in` into `out` (both with explicit strides).
void box_copy(cudaStream_t s, double* out, std::vector<int64_t> ostride, const double* in,
              std::vector<int64_t> istride, std::vector<int64_t> shape, double alpha = 1.0,
              double beta = 0.0);

// Bare integrals of one molecule, shared by all of its states.
struct Molecule {
  int o = 0, v = 0, n = 0, naux = 0;
  cudaStream_t stream = nullptr;
  std::vector<double> eps_host;
  OT eps;    // [n]
  OT B;      // [naux][n][n] bare DF factor
  OT hcore;  // [n][n] core Hamiltonian with diag(eps) as Fock matrix
  OT Bvv;    // [naux][v][v]
  OT Bnv;    // [naux][n][v]
  OT Gext;   // [n][v][v][v], Gext[x][b][c][d] = (xc|bd)
  DevBuf Gext_bf16;  // [3][n v][v^2 padded] BF16 planes of Gext (mixed precision)
  DevBuf Gext_oz;    // [6][n v][v^2 padded to 32] BF16 digit planes of Gext
  DevBuf Gext_oz_exp;  // int32 [n v] row exponents of Gext_oz
  // The ladder block is built on first use by a state of that precision.
  void ensure_fp64_ladder();
  void ensure_bf16_ladder();
  void ensure_oz_ladder();
  int build_level_ = 0;
  std::mutex mu_;
  // build_level 0 builds the bare integrals in FP64; 1..3 on the BF16 tensor
  // cores with that split level (used when the first state is mixed precision).
  Molecule(int o, int v, int naux, const double* eps_h, const double* B_src, bool on_device,
           cudaStream_t s, int build_level = 0);
  DevBuf err;  // int: timeout codes of tensor-core launches made for the molecule
  size_t bytes() const;
};

class T3pProgram;
struct T3pStreams;

struct Options {
  int precision = ASCC_FP64;
  int linearize = 1;
  int triples = 0;
  int pl_hole = -1, pl_particle = -1;
  double r_tol = 1e-8, e_tol = 1e-10;
  int max_iter = 200, diis_dim = 16, diis_start = 3;
  int polish_iter = 50;
  double polish_tol = 1e-6;
  int ladder_stream = 0;  // 1: rebuild (xc|bd) chunks per residual; -1: store; 0: auto
};

// One state (ground or one-CSF excited) of a molecule.
class State {
 public:
  // xsign = -1 runs the second ansatz of Sec. II.D (S -> -S).
  State(std::shared_ptr<Molecule> mol, int hole, int particle, double beta, const Options& opt,
        cudaStream_t s, double xsign = 1.0);
  ~State();

  int64_t n1() const { return (int64_t)o_ * v_; }
  int64_t n2() const { return (int64_t)o_ * o_ * v_ * v_; }
  int64_t n3() const { return (int64_t)t3idx_host_.size() / 6; }
  int64_t namp() const { return n1() + n2() + n3(); }
  const std::vector<int32_t>& t3_indices() const { return t3idx_host_; }

  // Residual of packed device amplitudes t -> packed device residual r and
  // device scalar energy.
  void residual(const double* t, double* r, double* energy);
  // Precision of a stand-alone residual call: FP64, or the polishing split
  // level in mixed precision.
  void prepare_eval() {
    es_.set_split(opt_.precision == ASCC_MIXED_BF16 ? 3 : opt_.precision == ASCC_FP64_TC ? 4 : 0,
                  err_.as<int>(), tc_min_flops_);
  }
  ascc_status solve(ascc_result* res);
  // Checkpoint of the iteration state: amplitudes, the DIIS history (slot
  // ids in age order, their (t, e) pairs and Gram matrix), the iteration
  // counters and the mixed-precision phase with its correction, so that a
  // loaded state continues exactly as the saved one would have.
  int64_t checkpoint_bytes() const;
  void checkpoint_save(void* buf, int64_t bytes);
  void checkpoint_load(const void* buf, int64_t bytes);
  // Iteration control: reset() loads the zeroth-order guess and clears the
  // DIIS history; iterate() runs up to max_steps residual evaluations from
  // the current amplitudes and history (Sec. III.B).
  void reset();
  ascc_status iterate(int max_steps, ascc_result* res);
  // Profiling of the dense ladder GEMM (CUDA events on the state's stream).
  void set_profiling(bool on) { profile_ = on; }
  void profile(double* ladder_ms, int64_t* ladder_launches, double* ladder_flops,
               double* ladder_mma_flops = nullptr);
  void initial_guess(std::vector<double>& t) const;

  double* amplitudes() { return t_.p(); }
  cudaStream_t stream() const { return s_; }
  std::shared_ptr<Molecule> molecule() const { return mol_; }
  const Options& options() const { return opt_; }
  double reference_energy();

 private:
  void build_state_integrals();
  void dress(const double* t1);
  void ladder(const T& t2, const T& r2);
  // the ladder GEMMs against (xc|bd) chunks rebuilt in this call
  void ladder_streamed(const T& t2);
  void quad_terms(const T& t, const T& u, const T& Z, const T& r2, double sign);
  // T3' slice: its residual R3' and its contributions to R1 and R2
  void triples(const T& t2, const double* t3, const T& r1, const T& r2, double* r3);
  void setup_triples();
  // one section of the T3' program, replayed from a CUDA graph captured on its
  // second run with the same level, operands and weight
  void run_t3(int section, double* const* base, double scale);
  struct T3Graph {
    cudaGraphExec_t exec = nullptr;
    bool failed = false;
    int64_t launches = 0;
    double flops = 0.0;
  };
  std::map<std::vector<uint64_t>, T3Graph> t3_graphs_;
  bool t3_use_graphs_ = true;
  // streams of the concurrent T3' run (empty: one stream) and the private
  // copies of the R3' blocks it accumulates into
  std::unique_ptr<T3pStreams> t3x_;
  OT t3priv_;
  void foo_term(const T& t, const double* W, double alpha, const T& Z);

  std::shared_ptr<Molecule> mol_;
  Options opt_;
  // iteration state
  std::vector<int> slots_;  // active DIIS slots, oldest first
  int next_slot_ = 0, iter_ = 0;
  bool have_prev_ = false, done_ = false;
  double e_prev_ = 0.0, e_last_ = 0.0, r_last_ = 0.0;
  ascc_status status_ = ASCC_ERR_NOT_CONVERGED;
  // profiling
  bool profile_ = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events_;
  double ladder_ms_ = 0.0, ladder_flops_ = 0.0, ladder_mma_flops_ = 0.0;
  int64_t ladder_launches_ = 0;
  cudaStream_t s_;
  int o_, v_, n_, naux_;
  int hole_, particle_;  // -1 for the ground state
  int lh_, lp_;          // primary labels used by the partial linearisation
  double beta_, xval_, xsign_ = 1.0;
  int nu_;               // v (+1 with the hole slot of an excited state)
  Einsum es_;
  std::vector<int32_t> t3idx_host_;
  DevBuf t3idx_;         // int32 [n3][6]
  // T3' program, packed-slice <-> block maps, blocks of t3 and of R3', its
  // workspace and the t2 - t2^(i<->j) operand of each binding
  std::unique_ptr<T3pProgram> t3p_;
  DevBuf t3dst_, t3dst2_, t3sgn_;
  OT t3blk_, r3blk_, t3ws_, t3ts_, t3nm_;
  // per-state constant integrals of the ladder corrections
  OT Gh1, Gh2, Gh3, GooP;
  // amplitudes, residual, DIIS
  OT t_, r_, hist_t_, hist_e_, scal_, work_, coef_, eps_eff_, gram_;
  DevBuf err_;           // int: device-side timeout codes of the tensor-core GEMM
  bool polish_ = false, need_refresh_ = false, have_corr_ = false;
  // mixed precision: the defect-corrected polishing gave way to FP64-class
  // residuals throughout (it stalled); polish_its_ counts its iterations
  bool fallback_ = false;
  int polish_its_ = 0;
  // stall detection of the low-precision phase of a digit-planes-only state:
  // the best max|R| since its last halving and the steps since
  double best_r_ = 0.0;
  int stall_n_ = 0;
  int fp64_evals_ = 0;
  OT corr_;  // FP64-minus-polishing residual correction (mixed precision)
  double tc_min_flops_ = 4e7;  // contractions below this stay FP64 (ASCC_TC_MIN_FLOPS overrides)
  int iter_low_ = 0;
  int level_for_phase() const;
  // per-iteration workspace
  OT L_, R_, LamC_, RhoC_, rowsC_, colsC_, Bhat_, hhat_, F_, dP_, J_, K_, Boo_, Bov_, Bvo_, Bvv_, Bno_, Bon_;
  OT goooo_, gooov_, goovv_, govov_, gvovo_, gvoov_, gvvoo_, Lvoov_, Lovov_;
  OT u_, m_, um_, Z_, WC_, WD_, Wq_, Fvv_, Foo_, X_, Y_, Yfull_, Z1_, tt_, Yoo_, YC_, Z1C_;
  OT tpair_, Yvv_, Yov_;  // pair-symmetric ladder operands
  // streamed ladder: chunk buffers and the t operand's planes
  bool stream_ladder_ = false;
  // mixed precision with the block stored as digit planes only: the ladder
  // is an exact digit-plane product in every phase
  bool ladder_digits_ = false;
  int64_t stream_chunk_bytes_ = (int64_t)1 << 30;
  OT stream_ac_, stream_gc_;
  DevBuf stream_a_, stream_ae_, stream_b_, stream_be_;
};

}  // namespace ascc
