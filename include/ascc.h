/*
 * ascc.h -- C ABI of the GB300 implementation of the Aufbau-suppressed
 * coupled-cluster (ASCC / PLASCC) amplitude-residual hot path.
 *
 * Method (arXiv 2501.10515, "Improving Aufbau Suppressed Coupled Cluster
 * Through Perturbative Analysis"):
 *   wave function      exp(-S^+) exp(T) |phi0>                    (Sec. II.A, Eq. ogascc)
 *   one-CSF S          (1/sqrt2)(p_up^+ h_up + p_dn^+ h_dn)         (Eq. 1CSF-S)
 *   working equations  E = <phi0| exp(-T) Hbar exp(T) |phi0>,
 *                      0 = <mu|   exp(-T) Hbar exp(T) |phi0>,
 *                      Hbar = exp(S^+) H exp(-S^+)                  (Eqs. energy, amp, sim)
 *   cluster operator   T1 + T2 (+ the mixed-triples slice T3')      (Sec. II.B.1)
 *   PLASCC             drop terms with >= 2 powers of T2^M / T3'    (Sec. II.C)
 *   solver             diagonal-Jacobian update with DIIS           (Sec. III.B)
 *
 * Conventions
 *   o, v      numbers of occupied / virtual spatial orbitals, n = o + v.
 *   eps[n]    orbital energies; the Fock matrix of the reference is diag(eps).
 *   B         density-fitting factor B[P][p][q], P < naux, symmetric in (p,q);
 *             (pq|rs) = sum_P B[P][p][q] B[P][r][s] (chemists' notation).
 *   t1[i][a]  alpha single amplitudes, row-major [o][v].
 *   t2[i][j][a][b]  alpha-beta double amplitudes, row-major [o][o][v][v];
 *             callers pass pair-symmetric t2 (t2[i][j][a][b] = t2[j][i][b][a]).
 *   t3p[k]    the T3' slice: alpha-beta-beta triples t[i][j][k][a][b][c]
 *             (j<k, b<c) with at least three of {h up, h dn, p up, p dn}
 *             among their spin-orbital indices, in the order returned by
 *             ascc_t3p_indices (lexicographic in (i,j,k,a,b,c)).
 *   Residuals have the layouts of the amplitudes they belong to.
 *
 * Errors: every function returns an ascc_status and never throws across the
 * ABI.  ascc_last_error() returns a thread-local message for the last failure.
 * Memory: inputs are copied; all device memory belongs to the context and is
 * released by ascc_destroy.  Device pointers are CUDA global-memory addresses
 * on the context's device; host pointers are ordinary (pageable or pinned)
 * memory.
 */
#ifndef ASCC_H
#define ASCC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ascc_ctx ascc_ctx;

typedef enum {
  ASCC_OK = 0,
  ASCC_ERR_INVALID = 1,        /* bad argument or unsupported option            */
  ASCC_ERR_OOM = 2,            /* device allocation failed                      */
  ASCC_ERR_CUDA = 3,           /* a CUDA runtime call failed                    */
  ASCC_ERR_NOT_CONVERGED = 4,  /* iteration cap reached                         */
  ASCC_ERR_DIVERGED = 5,       /* non-finite energy or residual                 */
  ASCC_ERR_TIMEOUT = 6         /* a bounded device wait gave up                 */
} ascc_status;

/* Precision of the residual contractions.
 *   ASCC_FP64        every contraction in FP64 (DFMA).
 *   ASCC_MIXED_BF16  large contractions on the BF16 tensor cores, 3 then 6
 *                    split products (the occupied Fock-like terms, an o x o
 *                    matrix along one index, as FP32 sums), with defect
 *                    correction from FP64-class evaluations (ASCC_FP64_TC
 *                    contractions); the accepted amplitudes satisfy the FP64
 *                    equations to r_tol.
 *   ASCC_FP64_TC     every large contraction as exact BF16 digit-plane
 *                    products on the tensor cores (ascc_gemm_fp64_tc, error
 *                    1e-12 to 5e-12 of |A||B|); iterations follow the FP64 path. */
enum { ASCC_FP64 = 0, ASCC_MIXED_BF16 = 1, ASCC_FP64_TC = 2 };

typedef struct {
  int32_t n_csf;     /* 0 = ground state (S = 0); 1 = one-CSF excited state     */
                     /* (two-CSF states, Sec. II.B.2, are not built on the GPU:  */
                     /*  n_csf = 2 returns ASCC_ERR_INVALID)                      */
  int32_t hole;      /* occupied index h in [0, o) of S (n_csf = 1)              */
  int32_t particle;  /* virtual index p in [0, v) of S (n_csf = 1)               */
  double beta;       /* T^P(0) = beta S + gamma S^2, gamma = -beta^2/2 (Eq.
                        TP-guess, Sec. II.D); 0 means: from alpha and ansatz   */
  double alpha;      /* Aufbau weight of the target reference (Sec. II.D)       */
  int32_t ansatz;    /* 0: beta = 1/(1+alpha) with S as given; 1: the second
                        ansatz, the hole orbital's sign flipped (alpha -> -alpha,
                        beta = 1/(1-alpha)), run as S -> -S in these orbitals   */
  int32_t reserved;
} ascc_excitation;

typedef struct {
  int32_t precision;   /* ASCC_FP64, ASCC_MIXED_BF16 or ASCC_FP64_TC            */
  int32_t linearize;   /* 0 = ASCC, 1 = PLASCC (Sec. II.C)                      */
  int32_t triples;     /* 1 = include T3' for n_csf = 1 (Sec. II.B.1)           */
  int32_t pl_hole;     /* primary pair used to split a ground-state solve for   */
  int32_t pl_particle; /*   PLASCC (Sec. II.C: same removal in the ground state) */
  double r_tol;        /* convergence: max |R| <= r_tol ...                     */
  double e_tol;        /*   ... and |E - E_prev| <= e_tol (Sec. III.A)          */
  int32_t max_iter;    /* iteration cap                                         */
  int32_t diis_dim;    /* DIIS history length (<= 32)                           */
  int32_t diis_start;  /* pairs needed before extrapolating                     */
  int32_t polish_iter; /* reserved                                             */
  double polish_tol;   /* mixed precision: max |R| at which the 3-product phase */
                       /*   hands over to the FP64-corrected polishing phase     */
  int32_t ladder_stream; /* the bare (xc|bd) block of the particle-particle ladder:
                            1 = rebuilt in ~1 GB x-chunks inside every residual
                            (no stored block; about twice the ladder work),
                            -1 = stored once per molecule, 0 = stored unless its
                            planes would take more than 60 % of the free device
                            memory when the state is created                    */
  int32_t reserved2;
} ascc_options;

typedef struct {
  double energy;      /* converged total energy E (Eq. energy)                 */
  double e_ref;       /* <phi0|Hbar|phi0>                                      */
  double max_resid;   /* max |R| at the last evaluation                        */
  int32_t iterations; /* residual evaluations performed                        */
  int32_t status;     /* ascc_status of the solve                              */
  int32_t iterations_low;   /* of which in low precision (mixed precision)     */
  int32_t fp64_evaluations; /* FP64-class residuals of the polishing phase
                               (mixed precision)                               */
} ascc_result;

/* Fills *opt with defaults: FP64, PLASCC, triples off, r_tol 1e-8, e_tol 1e-10,
 * max_iter 200, DIIS 16 / start 3, polish 1e-6.  Returns ASCC_OK. */
ascc_status ascc_default_options(ascc_options* opt);

/* Creates a context for one state of one molecule (Secs. II.A-II.B).
 *   o, v, naux  sizes (o >= 1, v >= 1, naux >= 1).
 *   eps         [o+v] orbital energies; host memory; copied.
 *   B           [naux][n][n] DF factor; host memory if b_on_device == 0,
 *               else device memory on the current device; copied.
 *   exc         excitation (NULL = ground state).
 *   opt         options (NULL = defaults).
 *   stream      cudaStream_t the context works on; NULL = a library-owned
 *               stream.
 * Builds the bare integral blocks the residual needs (once per context).
 * On failure *out is set to NULL. */
ascc_status ascc_create(ascc_ctx** out, int32_t o, int32_t v, int32_t naux,
                        const double* eps, const double* B, int32_t b_on_device,
                        const ascc_excitation* exc, const ascc_options* opt,
                        void* stream);

/* Creates a second state of the molecule held by `base` (another excitation
 * or the ground state), sharing its bare integrals on the device.  The
 * molecule's memory lives until every context using it is destroyed. */
ascc_status ascc_create_sibling(ascc_ctx** out, const ascc_ctx* base,
                                const ascc_excitation* exc,
                                const ascc_options* opt, void* stream);

/* Number of T3' amplitudes of this state (0 for the ground state or when
 * triples are off). */
int64_t ascc_t3p_size(const ascc_ctx* ctx);

/* Writes the [ascc_t3p_size][6] index list (i,j,k,a,b,c) of T3' to host
 * memory idx. */
ascc_status ascc_t3p_indices(const ascc_ctx* ctx, int32_t* idx);

/* One residual evaluation (Eqs. energy, amp over Hbar; PLASCC if the
 * context's options say so) at caller-given amplitudes.
 *   t1, t2, t3p  inputs; r1, r2, r3p, energy outputs (any may be NULL
 *   except t1, t2; t3p may be NULL when ascc_t3p_size is 0).
 *   t2 [o][o][v][v] must have the pair symmetry of closed-shell spin-adapted
 *   doubles, t2[i][j][a][b] = t2[j][i][b][a]: the particle-particle ladder
 *   is evaluated for the pairs i <= j only and the rest follows from it.
 * ascc_residual takes host buffers; ascc_residual_device takes device
 * buffers and does not synchronise the stream. */
ascc_status ascc_residual(ascc_ctx* ctx, const double* t1, const double* t2,
                          const double* t3p, double* r1, double* r2,
                          double* r3p, double* energy);
ascc_status ascc_residual_device(ascc_ctx* ctx, const double* t1,
                                 const double* t2, const double* t3p,
                                 double* r1, double* r2, double* r3p,
                                 double* energy);

/* Energy (Eq. energy) at caller-given host amplitudes. */
ascc_status ascc_energy(ascc_ctx* ctx, const double* t1, const double* t2,
                        double* energy);

/* Solves the amplitude equations from the zeroth-order guess (Eq. TP-guess)
 * with the Jacobi + DIIS iteration (Sec. III.B).  Fills *res (host).
 * Returns ASCC_OK on convergence, ASCC_ERR_NOT_CONVERGED or
 * ASCC_ERR_DIVERGED otherwise (res is filled in every case). */
ascc_status ascc_solve(ascc_ctx* ctx, ascc_result* res);

/* The two ansatz choices of Sec. II.D for an excitation with Aufbau weight
 * alpha: the state as created and the same state with the hole orbital's
 * sign flipped (alpha -> -alpha, S -> -S), sharing the molecule's integrals.
 * Both are solved from their zeroth-order guesses; the reported energy is
 * their mean, or the energy of the one that converged when the other did
 * not (Sec. III.A).  The second state is created on the first call and kept
 * by the context.  Returns ASCC_OK when at least one converged (res->energy
 * set, res->converged = 1 or 2), else the first choice's status with
 * res->energy = NaN.  ctx must hold a one-CSF excited state. */
typedef struct {
  double energy;          /* reported energy: mean, or the converged one      */
  int32_t converged;      /* how many of the two converged (0, 1, 2)           */
  int32_t reserved;
  ascc_result first;      /* ansatz 0: beta = 1/(1+alpha)                      */
  ascc_result second;     /* ansatz 1: beta = 1/(1-alpha), hole sign flipped   */
} ascc_two_ansatz_result;
ascc_status ascc_solve_two_ansatz(ascc_ctx* ctx, ascc_two_ansatz_result* res);

/* Step-wise solve (Sec. III.B).  ascc_reset loads the zeroth-order guess
 * (Eq. TP-guess) and clears the DIIS history; ascc_iterate continues from the
 * current amplitudes and history for at most max_steps residual evaluations
 * and fills *res.  Returns ASCC_OK once converged, ASCC_ERR_NOT_CONVERGED
 * while still iterating or at the cap, ASCC_ERR_DIVERGED on non-finite
 * values.  ascc_solve = ascc_reset + ascc_iterate(max_iter + 1). */
ascc_status ascc_reset(ascc_ctx* ctx);
ascc_status ascc_iterate(ascc_ctx* ctx, int32_t max_steps, ascc_result* res);

/* Profiling of the dense particle-particle ladder contraction: when enabled,
 * each launch is bracketed by CUDA events on the context's stream.
 * ascc_get_profile reports the summed event time (ms) of the dominant
 * ladder launch (the GEMM of the o(o+1)/2 pair rows against the v^2 virtual
 * rows of (xc|bd), with its split-K reduction; the whole ladder when the
 * block is streamed), the number of such launches and their flops:
 * 2 (o(o+1)/2) v^4 each (2 v^2 (o^3 v + o(o+1)/2 v^2) when streamed), and the
 * same times the plane products the tensor cores execute. */
typedef struct {
  double ladder_ms;
  double ladder_flops;
  int64_t ladder_launches;
  int64_t launches;   /* kernel launches of this library since the context was made */
  double gemm_flops;  /* flops (2 m n k) of all contractions since the context was made,
                         one product each whatever the precision                   */
  double ladder_mma_flops; /* ladder_flops times the BF16 plane products per step
                              (equal to ladder_flops on the FP64 path)             */
} ascc_profile;
ascc_status ascc_set_profiling(ascc_ctx* ctx, int32_t enable);
ascc_status ascc_get_profile(ascc_ctx* ctx, ascc_profile* out);

/* Split-precision tensor-core GEMM used by the mixed-precision residual:
 *   C = alpha * A B^T + beta * C,
 * A [M][K], B [N][K], C [M][N]: row-major FP64 device buffers.  Each operand
 * is split into `level` BF16 planes (x = x0 + x1 + ..., level 1..3) and the
 * 1, 3 or 6 leading plane products run as tcgen05 BF16 MMAs with FP32
 * accumulation; relative accuracy is about 4e-3, 2e-5 and 1e-7 respectively
 * (the paper's own code is FP64 NumPy; this is the GB300 precision device
 * behind ASCC_MIXED_BF16).  stream: cudaStream_t or NULL (default stream);
 * the call does not synchronise.  Returns ASCC_ERR_TIMEOUT if a bounded wait
 * inside the kernel gave up (checked at the next call on the same stream
 * after synchronisation by the caller). */
ascc_status ascc_gemm_split_bf16(int64_t M, int64_t N, int64_t K, int32_t level,
                                 double alpha, const double* A, const double* B,
                                 double beta, double* C, void* stream);

/* The same product with an explicit tile shape of the tcgen05 kernel:
 *   tile = 1: 128 x 256 tiles, one per CTA; 2: a persistent kernel (one CTA
 *   per SM looping over tiles) with 128 x 128 tiles; 3: the persistent kernel
 *   with 128 x 64 tiles (for M <= 64 < N the operands exchanged, the tile
 *   stored transposed); -1: the size rules (what ascc_gemm_split_bf16 uses);
 *   0: the autotuner's choice for the product's shape class, which runs the
 *   three shapes once each, timed, the first time a class is seen on a
 *   stream that is not being captured (that call allocates scratch for one
 *   output and synchronises the stream; products above 2^25 output elements
 *   or below 1e8 flops keep the size rules; ASCC_AUTOTUNE=0 turns tuning off).
 * Every tile shape accumulates each element over the same K tiles in the
 * same order, so the result does not depend on `tile`, with one exception:
 * for M <= 64 < N, tile 3 and the size rules exchange the operands, which
 * changes the order of the tensor core's sums (the autotuner leaves such
 * products to the size rules).  The residual engine's tensor-core
 * contractions use tile = 0. */
ascc_status ascc_gemm_split_bf16_tiled(int64_t M, int64_t N, int64_t K, int32_t level,
                                       double alpha, const double* A, const double* B,
                                       double beta, double* C, void* stream, int32_t tile);

/* Number of shape classes the tile autotuner has timed in this process. */
int64_t ascc_autotuned_classes(void);

/* Self-test of the bounded device waits that guard every tensor-core kernel:
 * one thread of a one-block kernel waits, with the kernels' own wait
 * function but a budget of limit_ms (1..2000) milliseconds, on an mbarrier
 * phase that nothing completes.  The budget runs out, the kernel records a
 * code and returns, and the call returns ASCC_ERR_TIMEOUT, the status a
 * tensor-core GEMM whose wait gave up reports; the context stays usable.
 * Synchronises `stream` (NULL: the default stream). */
ascc_status ascc_selftest_bounded_wait(int32_t limit_ms, void* stream);

/* Race and placement check of the T3' program (host only, no device call):
 * builds the program of a state of size o, v, naux on `nstreams` streams and
 * returns the number of op pairs of a section whose memory footprints
 * conflict (a write against a read or write of overlapping workspace, or two
 * accumulations into R1 or R2) but that neither stream order nor the plan's
 * event waits order, plus the number of intermediate pairs that share
 * workspace while both are live; 0 means race-free and correctly placed.
 * mode 0: the plan as built; 1: without its event waits; 2: with every
 * intermediate placed at offset 0 (modes 1 and 2 test the checks themselves).
 * Returns -1 on bad arguments. */
int64_t ascc_t3p_plan_check(int32_t o, int32_t v, int32_t naux, int32_t nstreams,
                            int32_t mode);

/* FP64-class GEMM on the BF16 tensor cores (the contraction device behind
 * ASCC_FP64_TC and the polishing evaluations of ASCC_MIXED_BF16):
 *   C = alpha * A B^T + beta * C,
 * A [M][K], B [N][K], C [M][N]: row-major FP64 device buffers.  Each row is
 * scaled by a power of two and rounded to a 42-bit integer held as six
 * 7-bit BF16 digit planes (error-free splitting of Ozaki, Ogita and Oishi);
 * the 21 leading plane products run as tcgen05 BF16 MMAs whose grouped FP32
 * sums are exact over chunks of 1024 K values and are folded into 64-bit
 * integers.  Error: 1e-12 to 5e-12 of |A||B| elementwise for rows of even
 * magnitude (each row is a 42-bit fixed-point number relative to its largest
 * entry, and the plane products with s + t >= 6 are left out); a row or
 * column holding a NaN or an infinity gives NaN.  Results do not depend on
 * the K split.  stream: cudaStream_t or NULL; the call does not synchronise
 * (it allocates its operand planes and workspace stream-ordered).  Returns
 * ASCC_ERR_TIMEOUT if a bounded wait of an earlier call gave up. */
ascc_status ascc_gemm_fp64_tc(int64_t M, int64_t N, int64_t K, double alpha,
                              const double* A, const double* B, double beta,
                              double* C, void* stream);

/* The same product as ascc_gemm_split_bf16 (same operand split, same K
 * split, same FP32 partial sums), for callers that cannot allocate device
 * memory when they need it: a process whose GPU memory has been handed in
 * full to another pool (e.g. a framework's caching allocator that reserved
 * the device up front) has none left for cudaMalloc, and code that must not
 * enter the CUDA allocator (cudaMalloc / cudaFree may synchronise the whole
 * device) cannot use the stream-ordered scratch of ascc_gemm_split_bf16.
 * This entry point calls no cudaMalloc/cudaFree and no allocating library
 * routine: the BF16 operand planes and the split-K partials live in a fixed
 * 32 MiB device array per GPU (held by every GPU that loads the library
 * until the process exits).  The paper has no counterpart; it is a property
 * of this library's tensor-core GEMM.
 *   Limit: 2 * level * (M + N) * ceil(K / 64) * 64 bytes (rounded up to 256)
 *   plus 4 * z * M * N bytes of partials when K is split in z chunks (z as
 *   ascc_gemm_split_bf16 chooses it) must not exceed 32 MiB; larger requests
 *   return ASCC_ERR_INVALID without touching the GPU.
 *   The first call on a device looks up the array's device address (with
 *   that device current).
 *   Each call ends by reading its device timeout flag back to the host, so
 *   it synchronises `stream` before returning; a bounded wait that gave up
 *   returns ASCC_ERR_TIMEOUT.
 *   All calls share the array, which keeps the last call's contents: calls
 *   that overlap on the GPU (different streams, or threads calling at the
 *   same time) race on it. */
ascc_status ascc_gemm_split_bf16_noalloc(int64_t M, int64_t N, int64_t K,
                                         int32_t level, double alpha,
                                         const double* A, const double* B,
                                         double beta, double* C, void* stream);

/* ------------------------------------------------------------------ serving
 * A request server for streams of ASCC solves of different molecules and
 * states on one GPU.  Worker threads, each on its own CUDA stream, admit the
 * oldest queued request whose device footprint (ascc_footprint_bytes) fits
 * beside the requests already running (a request at the head of the queue
 * that does not fit yet does not hold back smaller ones), build its bare
 * integrals once, solve its states (ground state first if listed; a ground
 * state takes the primary pair of the request's first excitation for PLASCC)
 * and free the memory, so requests that arrive while others run are admitted
 * as memory frees up and their work overlaps on the device.  With
 * ASCC_MIXED_BF16, a state whose mixed solve ends ASCC_ERR_NOT_CONVERGED is
 * solved again on the FP64-class path (ASCC_FP64_TC) from the initial guess;
 * its result then carries that solve's status and energy and the iterations
 * of both.  Times are seconds since creation. */
typedef struct ascc_server ascc_server;
typedef struct {
  int64_t request_id;
  int32_t state_index; /* index into the request's state list; -1: request failed */
  int32_t status;      /* ascc_status of the solve                              */
  double energy;
  int32_t iterations;
  int32_t worker;
  double t_arrival, t_start, t_end;
} ascc_serve_result;

/* memory_budget: device bytes the admitted requests may use together;
 * max_active: worker threads (1..64); opt: solve options (NULL = defaults). */
ascc_status ascc_server_create(ascc_server** out, size_t memory_budget,
                               int32_t max_active, const ascc_options* opt);
/* Queues one request (host eps [o+v] and B [naux][n][n] are copied; the
 * arrival time is the submission time).  Thread-safe.  A request whose
 * ascc_footprint_bytes exceeds the server's memory budget is refused with
 * ASCC_ERR_OOM (nothing is queued).  Workers admit the oldest queued request
 * that fits beside the running ones. */
ascc_status ascc_server_submit(ascc_server* srv, int32_t o, int32_t v,
                               int32_t naux, const double* eps, const double* B,
                               int32_t n_states, const ascc_excitation* states,
                               int64_t* request_id);
/* Blocks until every submitted request has finished. */
ascc_status ascc_server_drain(ascc_server* srv);
int64_t ascc_server_result_count(ascc_server* srv);
/* Copies the per-state results (completion order) to out[capacity]. */
ascc_status ascc_server_results(ascc_server* srv, ascc_serve_result* out,
                                int64_t capacity);
void ascc_server_destroy(ascc_server* srv);

/* Amplitudes in and out (host buffers, FP64).  ascc_set_state replaces the
 * amplitudes and keeps the DIIS history and counters as they are; for an
 * exact resume use the checkpoint calls below. */
ascc_status ascc_get_state(ascc_ctx* ctx, double* t1, double* t2, double* t3p);
ascc_status ascc_set_state(ascc_ctx* ctx, const double* t1, const double* t2,
                           const double* t3p);

/* Checkpoint of a solve in progress: the amplitudes, the DIIS history (the
 * stored amplitude / error pairs in age order, their Gram matrix and slot
 * ids), the iteration counters and, in mixed precision, the polishing phase
 * with its residual correction.  A state loaded into a context created with
 * the same molecule, excitation and options continues (ascc_iterate) exactly
 * as the saved one would have: bitwise, since every kernel of the iteration
 * is deterministic.  The blob is host memory of ascc_checkpoint_size bytes
 * (it grows with the DIIS history, up to 2 diis_dim + 1 amplitude vectors);
 * loading checks the sizes, excitation and options and returns
 * ASCC_ERR_INVALID for a blob of another state. */
ascc_status ascc_checkpoint_size(const ascc_ctx* ctx, int64_t* bytes);
ascc_status ascc_checkpoint_save(ascc_ctx* ctx, void* buf, int64_t bytes);
ascc_status ascc_checkpoint_load(ascc_ctx* ctx, const void* buf, int64_t bytes);

/* Device bytes a context of this shape needs (bare integrals + state). */
size_t ascc_footprint_bytes(int32_t o, int32_t v, int32_t naux,
                            const ascc_options* opt);

/* Number of kernel launches issued by this context since creation. */
int64_t ascc_launch_count(const ascc_ctx* ctx);

void ascc_destroy(ascc_ctx* ctx);
const char* ascc_status_string(ascc_status s);
const char* ascc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ASCC_H */
