// C ABI of libascc (declared in include/ascc.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>

#include "engine.h"
#include "gemm_oz.h"
#include "gemm_tc.h"
#include "kernels.h"
#include "t3p.h"

using namespace ascc;

struct ascc_ctx {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::unique_ptr<State> state;
  std::unique_ptr<State> partner;  // the other ansatz of Sec. II.D, built on first use
  ascc_excitation exc{};
  bool has_exc = false;
  int64_t launches0 = 0;
  double flops0 = 0.0;
  ~ascc_ctx() {
    if (stream) cudaStreamSynchronize(stream);
    partner.reset();
    state.reset();
    if (stream) cudaStreamSynchronize(stream);
    if (own_stream && stream) cudaStreamDestroy(stream);
    // the stream-ordered pool keeps freed blocks (its release threshold is
    // unbounded, so that iterations reuse them): hand back what no other
    // state holds, for the device's other users
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess)
      cudaMemPoolTrimTo(pool, 0);
  }
};

namespace {
thread_local std::string g_err;
}  // namespace

void ascc::record_error(const std::string& msg) { g_err = msg; }

namespace {

template <class F>
ascc_status guard(F&& f) {
  try {
    return f();
  } catch (const Error& e) {
    g_err = e.what();
    return e.status;
  } catch (const std::bad_alloc&) {
    g_err = "host allocation failed";
    return ASCC_ERR_OOM;
  } catch (const std::exception& e) {
    g_err = e.what();
    return ASCC_ERR_INVALID;
  }
}

Options to_options(const ascc_options* o) {
  Options r;
  if (!o) return r;
  r.precision = o->precision;
  r.linearize = o->linearize;
  r.triples = o->triples;
  r.pl_hole = o->pl_hole;
  r.pl_particle = o->pl_particle;
  r.r_tol = o->r_tol;
  r.e_tol = o->e_tol;
  r.max_iter = o->max_iter;
  r.diis_dim = o->diis_dim;
  r.diis_start = o->diis_start;
  r.polish_iter = o->polish_iter;
  r.polish_tol = o->polish_tol;
  r.ladder_stream = o->ladder_stream;
  return r;
}

void prepare_pool() {
  int dev = 0;
  ASCC_CUDA(cudaGetDevice(&dev));
  cudaMemPool_t pool;
  ASCC_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t thr = UINT64_MAX;
  ASCC_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
}

void check_exc(const ascc_excitation* exc, int o, int v, int& hole, int& particle, double& beta,
               double& xsign) {
  hole = -1;
  particle = -1;
  beta = 1.0;
  xsign = 1.0;
  if (!exc || exc->n_csf == 0) return;
  ASCC_REQUIRE(exc->n_csf == 1, "only one-CSF excitations are supported");
  ASCC_REQUIRE(exc->hole >= 0 && exc->hole < o, "hole out of range");
  ASCC_REQUIRE(exc->particle >= 0 && exc->particle < v, "particle out of range");
  ASCC_REQUIRE(exc->ansatz == 0 || exc->ansatz == 1, "ansatz must be 0 or 1");
  ASCC_REQUIRE(std::isfinite(exc->alpha) && std::fabs(exc->alpha) < 1.0, "|alpha| must be < 1");
  hole = exc->hole;
  particle = exc->particle;
  xsign = exc->ansatz == 1 ? -1.0 : 1.0;
  if (exc->beta != 0.0)
    beta = exc->beta;
  else
    beta = exc->ansatz == 1 ? 1.0 / (1.0 - exc->alpha) : 1.0 / (1.0 + exc->alpha);
  ASCC_REQUIRE(std::isfinite(beta) && beta > 0.0, "beta must be positive");
}

ascc_status make_ctx(ascc_ctx** out, std::shared_ptr<Molecule> mol, const ascc_excitation* exc,
                     const ascc_options* opt, cudaStream_t stream, bool own) {
  auto ctx = std::make_unique<ascc_ctx>();
  ctx->stream = stream;
  ctx->own_stream = own;
  ctx->launches0 = launch_total();
  ctx->flops0 = flop_total();
  int hole, particle;
  double beta, xsign;
  check_exc(exc, mol->o, mol->v, hole, particle, beta, xsign);
  Options o = to_options(opt);
  if (o.pl_hole >= mol->o || o.pl_particle >= mol->v) throw Error(ASCC_ERR_INVALID, "pl labels");
  ctx->state = std::make_unique<State>(std::move(mol), hole, particle, beta, o, stream, xsign);
  if (exc) {
    ctx->exc = *exc;
    ctx->has_exc = true;
  }
  ASCC_CUDA(cudaStreamSynchronize(stream));
  *out = ctx.release();
  return ASCC_OK;
}
}  // namespace

extern "C" {

ascc_status ascc_default_options(ascc_options* opt) {
  if (!opt) return ASCC_ERR_INVALID;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = ASCC_FP64;
  opt->linearize = 1;
  opt->triples = 0;
  opt->pl_hole = -1;
  opt->pl_particle = -1;
  opt->r_tol = 1e-8;
  opt->e_tol = 1e-10;
  opt->max_iter = 200;
  opt->diis_dim = 16;
  opt->diis_start = 3;
  opt->polish_iter = 50;
  opt->polish_tol = 1e-6;
  opt->ladder_stream = 0;
  opt->reserved2 = 0;
  return ASCC_OK;
}

ascc_status ascc_create(ascc_ctx** out, int32_t o, int32_t v, int32_t naux, const double* eps,
                        const double* B, int32_t b_on_device, const ascc_excitation* exc,
                        const ascc_options* opt, void* stream) {
  if (out) *out = nullptr;
  return guard([&]() -> ascc_status {
    ASCC_REQUIRE(out && eps && B, "null argument");
    ASCC_REQUIRE(o >= 1 && v >= 1 && naux >= 1, "sizes must be positive");
    prepare_pool();
    cudaStream_t s = (cudaStream_t)stream;
    bool own = false;
    if (!s) {
      ASCC_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      own = true;
    }
    try {
      const int build_level = (opt && opt->precision == ASCC_MIXED_BF16) ? 3 : 0;
      auto mol = std::make_shared<Molecule>(o, v, naux, eps, B, b_on_device != 0, s, build_level);
      return make_ctx(out, std::move(mol), exc, opt, s, own);
    } catch (...) {
      if (own) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
      }
      throw;
    }
  });
}

ascc_status ascc_create_sibling(ascc_ctx** out, const ascc_ctx* base, const ascc_excitation* exc,
                                const ascc_options* opt, void* stream) {
  if (out) *out = nullptr;
  return guard([&]() -> ascc_status {
    ASCC_REQUIRE(out && base && base->state, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    bool own = false;
    if (!s) {
      ASCC_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      own = true;
    }
    // the molecule's buffers were produced on the base stream
    ASCC_CUDA(cudaStreamSynchronize(base->stream));
    return make_ctx(out, base->state->molecule(), exc, opt, s, own);
  });
}

int64_t ascc_t3p_size(const ascc_ctx* ctx) { return ctx && ctx->state ? ctx->state->n3() : 0; }

ascc_status ascc_t3p_indices(const ascc_ctx* ctx, int32_t* idx) {
  return guard([&]() -> ascc_status {
    ASCC_REQUIRE(ctx && ctx->state && (idx || ctx->state->n3() == 0), "null argument");
    const auto& v = ctx->state->t3_indices();
    if (!v.empty()) std::memcpy(idx, v.data(), v.size() * sizeof(int32_t));
    return ASCC_OK;
  });
}

ascc_status ascc_residual_device(ascc_ctx* ctx, const double* t1, const double* t2,
                                 const double* t3p, double* r1, double* r2, double* r3p,
                                 double* energy) {
  return guard([&]() -> ascc_status {
    ASCC_REQUIRE(ctx && ctx->state && t1 && t2, "null argument");
    State& S = *ctx->state;
    ASCC_REQUIRE(S.n3() == 0 || t3p, "t3p required");
    cudaStream_t s = ctx->stream;
    const int64_t n1 = S.n1(), n2 = S.n2(), n3 = S.n3(), N = S.namp();
    OT tv({N}, s), rv({N}, s), e({1}, s);
    ASCC_CUDA(cudaMemcpyAsync(tv.p(), t1, n1 * 8, cudaMemcpyDeviceToDevice, s));
    ASCC_CUDA(cudaMemcpyAsync(tv.p() + n1, t2, n2 * 8, cudaMemcpyDeviceToDevice, s));
    if (n3) ASCC_CUDA(cudaMemcpyAsync(tv.p() + n1 + n2, t3p, n3 * 8, cudaMemcpyDeviceToDevice, s));
    S.prepare_eval();
    S.residual(tv.p(), rv.p(), e.p());
    if (r1) ASCC_CUDA(cudaMemcpyAsync(r1, rv.p(), n1 * 8, cudaMemcpyDeviceToDevice, s));
    if (r2) ASCC_CUDA(cudaMemcpyAsync(r2, rv.p() + n1, n2 * 8, cudaMemcpyDeviceToDevice, s));
    if (r3p && n3)
      ASCC_CUDA(cudaMemcpyAsync(r3p, rv.p() + n1 + n2, n3 * 8, cudaMemcpyDeviceToDevice, s));
    if (energy) ASCC_CUDA(cudaMemcpyAsync(energy, e.p(), 8, cudaMemcpyDeviceToDevice, s));
    return ASCC_OK;
  });
}

ascc_status ascc_residual(ascc_ctx* ctx, const double* t1, const double* t2, const double* t3p,
                          double* r1, double* r2, double* r3p, double* energy) {
  return guard([&]() -> ascc_status {
    ASCC_REQUIRE(ctx && ctx->state && t1 && t2, "null argument");
    State& S = *ctx->state;
    ASCC_REQUIRE(S.n3() == 0 || t3p, "t3p required");
    cudaStream_t s = ctx->stream;
    const int64_t n1 = S.n1(), n2 = S.n2(), n3 = S.n3(), N = S.namp();
    OT tv({N}, s), rv({N}, s), e({1}, s);
    ASCC_CUDA(cudaMemcpyAsync(tv.p(), t1, n1 * 8, cudaMemcpyHostToDevice, s));
    ASCC_CUDA(cudaMemcpyAsync(tv.p() + n1, t2, n2 * 8, cudaMemcpyHostToDevice, s));
    if (n3) ASCC_CUDA(cudaMemcpyAsync(tv.p() + n1 + n2, t3p, n3 * 8, cudaMemcpyHostToDevice, s));
    S.prepare_eval();
    S.residual(tv.p(), rv.p(), e.p());
    if (r1) ASCC_CUDA(cudaMemcpyAsync(r1, rv.p(), n1 * 8, cudaMemcpyDeviceToHost, s));
    if (r2) ASCC_CUDA(cudaMemcpyAsync(r2, rv.p() + n1, n2 * 8, cudaMemcpyDeviceToHost, s));
    if (r3p && n3)
      ASCC_CUDA(cudaMemcpyAsync(r3p, rv.p() + n1 + n2, n3 * 8, cudaMemcpyDeviceToHost, s));
    if (energy) ASCC_CUDA(cudaMemcpyAsync(energy, e.p(), 8, cudaMemcpyDeviceToHost, s));
    ASCC_CUDA(cudaStreamSynchronize(s));
    return ASCC_OK;
  });
}

ascc_status ascc_energy(ascc_ctx* ctx, const double* t1, const double* t2, double* energy) {
  return guard([&]() -> ascc_status {
    ASCC_REQUIRE(ctx && ctx->state && energy, "null argument");
    State& S = *ctx->state;
    std::vector<double> t3(S.n3(), 0.0);
    const double* t3p = S.n3() ? t3.data() : nullptr;
    if (S.n3()) {
      // the energy has no T3' term; read the stored slice to keep it consistent
      ASCC_CUDA(cudaMemcpyAsync(t3.data(), S.amplitudes() + S.n1() + S.n2(), S.n3() * 8,
                                cudaMemcpyDeviceToHost, ctx->stream));
      ASCC_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    return ascc_residual(ctx, t1, t2, t3p, nullptr, nullptr, nullptr, energy);
  });
}

ascc_status ascc_solve(ascc_ctx* ctx, ascc_result* res) {
  return guard([&]() -> ascc_status {
    ASCC_REQUIRE(ctx && ctx->state, "null argument");
    const double eref = ctx->state->reference_energy();
    ascc_status st = ctx->state->solve(res);
    if (res) res->e_ref = eref;
    if (st != ASCC_OK) g_err = st == ASCC_ERR_DIVERGED ? "diverged" : "not converged";
    return st;
  });
}

ascc_status ascc_solve_two_ansatz(ascc_ctx* ctx, ascc_two_ansatz_result* res) {
  return guard([&]() -> ascc_status {
    ASCC_REQUIRE(ctx && ctx->state && res, "null argument");
    ASCC_REQUIRE(ctx->has_exc && ctx->exc.n_csf == 1, "the two ansatz choices need an excited state");
    State& S = *ctx->state;
    if (!ctx->partner) {
      // the same state with the hole orbital's sign flipped: S -> -S and
      // alpha -> -alpha (beta' = 1 / (1 - alpha) for the first choice's
      // beta = 1 / (1 + alpha))
      ascc_excitation e = ctx->exc;
      e.ansatz = 1 - e.ansatz;
      e.beta = 0.0;
      int hole, particle;
      double beta, xsign;
      check_exc(&e, S.molecule()->o, S.molecule()->v, hole, particle, beta, xsign);
      ctx->partner = std::make_unique<State>(S.molecule(), hole, particle, beta, S.options(),
                                             ctx->stream, xsign);
    }
    State* first = ctx->exc.ansatz == 0 ? ctx->state.get() : ctx->partner.get();
    State* second = ctx->exc.ansatz == 0 ? ctx->partner.get() : ctx->state.get();
    std::memset(res, 0, sizeof(*res));
    first->solve(&res->first);
    second->solve(&res->second);
    const bool a = res->first.status == ASCC_OK, b = res->second.status == ASCC_OK;
    res->converged = (int32_t)a + (int32_t)b;
    if (a && b) {
      res->energy = 0.5 * (res->first.energy + res->second.energy);
    } else if (a || b) {
      res->energy = a ? res->first.energy : res->second.energy;
    } else {
      res->energy = NAN;
      g_err = "neither ansatz converged";
      return (ascc_status)res->first.status;
    }
    return ASCC_OK;
  });
}

ascc_status ascc_checkpoint_size(const ascc_ctx* ctx, int64_t* bytes) {
  return guard([&]() -> ascc_status {
    ASCC_REQUIRE(ctx && ctx->state && bytes, "null argument");
    *bytes = ctx->state->checkpoint_bytes();
    return ASCC_OK;
  });
}

ascc_status ascc_checkpoint_save(ascc_ctx* ctx, void* buf, int64_t bytes) {
  return guard([&]() -> ascc_status {
    ASCC_REQUIRE(ctx && ctx->state && buf, "null argument");
    ctx->state->checkpoint_save(buf, bytes);
    return ASCC_OK;
  });
}

ascc_status ascc_checkpoint_load(ascc_ctx* ctx, const void* buf, int64_t bytes) {
  return guard([&]() -> ascc_status {
    ASCC_REQUIRE(ctx && ctx->state && buf, "null argument");
    ctx->state->checkpoint_load(buf, bytes);
    return ASCC_OK;
  });
}

ascc_status ascc_reset(ascc_ctx* ctx) {
  return guard([&]() -> ascc_status {
    ASCC_REQUIRE(ctx && ctx->state, "null argument");
    ctx->state->reset();
    return ASCC_OK;
  });
}

ascc_status ascc_iterate(ascc_ctx* ctx, int32_t max_steps, ascc_result* res) {
  return guard([&]() -> ascc_status {
    ASCC_REQUIRE(ctx && ctx->state && max_steps >= 0, "bad argument");
    return ctx->state->iterate(max_steps, res);
  });
}

ascc_status ascc_set_profiling(ascc_ctx* ctx, int32_t enable) {
  return guard([&]() -> ascc_status {
    ASCC_REQUIRE(ctx && ctx->state, "null argument");
    ctx->state->set_profiling(enable != 0);
    return ASCC_OK;
  });
}

ascc_status ascc_get_profile(ascc_ctx* ctx, ascc_profile* out) {
  return guard([&]() -> ascc_status {
    ASCC_REQUIRE(ctx && ctx->state && out, "null argument");
    ctx->state->profile(&out->ladder_ms, &out->ladder_launches, &out->ladder_flops,
                        &out->ladder_mma_flops);
    out->launches = launch_total() - ctx->launches0;
    out->gemm_flops = flop_total() - ctx->flops0;
    return ASCC_OK;
  });
}

ascc_status ascc_gemm_split_bf16(int64_t M, int64_t N, int64_t K, int32_t level, double alpha,
                                 const double* A, const double* B, double beta, double* C,
                                 void* stream) {
  return ascc_gemm_split_bf16_tiled(M, N, K, level, alpha, A, B, beta, C, stream, -1);
}

ascc_status ascc_gemm_split_bf16_tiled(int64_t M, int64_t N, int64_t K, int32_t level,
                                       double alpha, const double* A, const double* B, double beta,
                                       double* C, void* stream, int32_t tile) {
  return guard([&]() -> ascc_status {
    ASCC_REQUIRE(tile >= -1 && tile <= 3, "tile must be -1, 0, 1, 2 or 3");
    ASCC_REQUIRE(A && B && C && M > 0 && N > 0 && K > 0, "bad argument");
    ASCC_REQUIRE(level >= 1 && level <= 3, "level must be 1, 2 or 3");
    cudaStream_t s = (cudaStream_t)stream;
    static int* err = nullptr;
    if (!err) {
      ASCC_CUDA(cudaMalloc(&err, sizeof(int)));
      ASCC_CUDA(cudaMemset(err, 0, sizeof(int)));
    }
    int h = 0;
    ASCC_CUDA(cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
      cudaMemset(err, 0, sizeof(int));
      throw Error(ASCC_ERR_TIMEOUT, "tensor-core GEMM wait timed out");
    }
    const int64_t Kp = tc::padded_k(K);
    DevBuf pa(sizeof(__nv_bfloat16) * (size_t)(level * M * Kp), s);
    DevBuf pb(sizeof(__nv_bfloat16) * (size_t)(level * N * Kp), s);
    tc::split_bf16(s, pa.as<__nv_bfloat16>(), A, M, K, K, level);
    tc::split_bf16(s, pb.as<__nv_bfloat16>(), B, N, K, K, level);
    const int z = tc::splitk_for(M, N, K);
    DevBuf ws(z > 1 ? sizeof(float) * (size_t)(z * M * N) : 0, s);
    tc::gemm_split(s, M, N, K, level, alpha, pa.as<__nv_bfloat16>(), pb.as<__nv_bfloat16>(), beta,
                   C, N, err, z, ws.as<float>(), 0, nullptr, tile);
    return ASCC_OK;
  });
}

ascc_status ascc_gemm_fp64_tc(int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                              const double* B, double beta, double* C, void* stream) {
  return guard([&]() -> ascc_status {
    ASCC_REQUIRE(A && B && C && M > 0 && N > 0 && K > 0, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    static int* err = nullptr;
    if (!err) {
      ASCC_CUDA(cudaMalloc(&err, sizeof(int)));
      ASCC_CUDA(cudaMemset(err, 0, sizeof(int)));
    }
    int h = 0;
    ASCC_CUDA(cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
      cudaMemset(err, 0, sizeof(int));
      throw Error(ASCC_ERR_TIMEOUT, "tensor-core GEMM wait timed out");
    }
    const int64_t Kq = oz::padded_k(K);
    DevBuf pa(sizeof(__nv_bfloat16) * (size_t)(oz::NSLICE * M * Kq), s);
    DevBuf pb(sizeof(__nv_bfloat16) * (size_t)(oz::NSLICE * N * Kq), s);
    DevBuf ea(sizeof(int32_t) * (size_t)M, s), eb(sizeof(int32_t) * (size_t)N, s);
    DevBuf ws(oz::ws_bytes(M, N), s);
    oz::split(s, pa.as<__nv_bfloat16>(), ea.as<int32_t>(), A, M, K, K);
    oz::split(s, pb.as<__nv_bfloat16>(), eb.as<int32_t>(), B, N, K, K);
    oz::gemm(s, M, N, K, alpha, pa.as<__nv_bfloat16>(), ea.as<int32_t>(), 0,
             pb.as<__nv_bfloat16>(), eb.as<int32_t>(), 0, beta, C, N, ws.as<long long>(), err,
             oz::splitk_for(M, N, K));
    return ASCC_OK;
  });
}

ascc_status ascc_get_state(ascc_ctx* ctx, double* t1, double* t2, double* t3p) {
  return guard([&]() -> ascc_status {
    ASCC_REQUIRE(ctx && ctx->state, "null argument");
    State& S = *ctx->state;
    cudaStream_t s = ctx->stream;
    if (t1) ASCC_CUDA(cudaMemcpyAsync(t1, S.amplitudes(), S.n1() * 8, cudaMemcpyDeviceToHost, s));
    if (t2)
      ASCC_CUDA(cudaMemcpyAsync(t2, S.amplitudes() + S.n1(), S.n2() * 8, cudaMemcpyDeviceToHost, s));
    if (t3p && S.n3())
      ASCC_CUDA(cudaMemcpyAsync(t3p, S.amplitudes() + S.n1() + S.n2(), S.n3() * 8,
                                cudaMemcpyDeviceToHost, s));
    ASCC_CUDA(cudaStreamSynchronize(s));
    return ASCC_OK;
  });
}

ascc_status ascc_set_state(ascc_ctx* ctx, const double* t1, const double* t2, const double* t3p) {
  return guard([&]() -> ascc_status {
    ASCC_REQUIRE(ctx && ctx->state && t1 && t2, "null argument");
    State& S = *ctx->state;
    cudaStream_t s = ctx->stream;
    ASCC_CUDA(cudaMemcpyAsync(S.amplitudes(), t1, S.n1() * 8, cudaMemcpyHostToDevice, s));
    ASCC_CUDA(cudaMemcpyAsync(S.amplitudes() + S.n1(), t2, S.n2() * 8, cudaMemcpyHostToDevice, s));
    if (S.n3()) {
      ASCC_REQUIRE(t3p, "t3p required");
      ASCC_CUDA(cudaMemcpyAsync(S.amplitudes() + S.n1() + S.n2(), t3p, S.n3() * 8,
                                cudaMemcpyHostToDevice, s));
    }
    ASCC_CUDA(cudaStreamSynchronize(s));
    return ASCC_OK;
  });
}

size_t ascc_footprint_bytes(int32_t o, int32_t v, int32_t naux, const ascc_options* opt) {
  // molecule: B, hcore, Bvv, Bnv, ladder block (FP64 or 3 BF16 planes) and its
  // build chunk; state: amplitudes, residual, DIIS history, per-iteration
  // workspace and the einsum temporaries (a few o^2 v^2 / o^2 n^2 tensors).
  const double n = o + v, O = o, V = v, P = naux;
  const int prec = opt ? opt->precision : ASCC_FP64;
  const bool mixed = prec == ASCC_MIXED_BF16, digits = prec != ASCC_FP64;
  const int m = opt ? opt->diis_dim : 16;
  const double kp = std::ceil(V * V / 64.0) * 64.0, kq = std::ceil(V * V / 32.0) * 32.0;
  double mol = 8.0 * (P * n * n + n * n + P * V * V + P * n * V);
  // ladder blocks: FP64 (+ its build temporary), or the BF16 split planes
  // (mixed) and the six digit planes (mixed, FP64_TC) with ~2 GB of build chunks
  const bool stream = opt && opt->ladder_stream == 1;
  if (stream) {
    // rebuilt per residual: one ~1 GB FP64 chunk, its permutation temporary and planes
    mol += 3.5 * (double)(1 << 30);
  } else {
    if (!digits) mol += 8.0 * n * V * V * V * 2.0;
    if (mixed) mol += 2.0 * 3.0 * n * V * kp;
    if (digits) mol += 2.0 * 6.0 * n * V * kq + 4.0 * n * V + 2.2e9;
  }
  const double o2v2 = O * O * V * V, namp = O * V + o2v2;
  double state = 8.0 * (namp * (2.0 * m + 4.0) + P * n * n * 1.2 + 24.0 * o2v2 +
                        O * O * n * n * 3.0 + O * O * n * V * 4.0);
  if (mixed) state += 2.0 * 3.0 * (O * O + n * V) * kp;  // operand planes of the ladder
  // digit planes of the ladder's t operand, the integer workspace, and the
  // planes of the largest generic contraction (o v x o v x o v)
  if (digits) state += 2.0 * 6.0 * O * O * kq + 8.0 * o2v2 + 2.0 * 6.0 * 2.0 * o2v2 + 8.0 * o2v2;
  if (opt && opt->triples) {
    // T3' blocks of t3 and R3', their workspace (intermediates of the
    // generated program, sized for the worst primary pair) and the t2 - t2^T
    // operands
    const int ns = t3p_streams();
    T3pProgram prog(o, v, naux, 0, 0, ns);
    state += 8.0 * ((2.0 + (ns > 1 ? ns : 0)) * prog.block_elements() +
                    prog.workspace_elements() + 2.0 * o2v2) +
             (double)ns * prog.cache_bytes();
  }
  return (size_t)((mol + state) * 1.1);
}

int64_t ascc_launch_count(const ascc_ctx* ctx) {
  return ctx ? launch_total() - ctx->launches0 : 0;
}

void ascc_destroy(ascc_ctx* ctx) { delete ctx; }

int64_t ascc_autotuned_classes(void) { return tc::autotuned_classes(); }

ascc_status ascc_selftest_bounded_wait(int32_t limit_ms, void* stream) {
  return guard([&]() -> ascc_status {
    ASCC_REQUIRE(limit_ms >= 1 && limit_ms <= 2000, "limit_ms in 1..2000");
    const int code = tc::wait_selftest((cudaStream_t)stream, limit_ms);
    if (code != 0)
      throw Error(ASCC_ERR_TIMEOUT, "bounded wait gave up (code " + std::to_string(code) + ")");
    return ASCC_OK;
  });
}

int64_t ascc_t3p_plan_check(int32_t o, int32_t v, int32_t naux, int32_t nstreams,
                            int32_t mode) {
  try {
    if (o < 2 || v < 2 || naux < 1 || nstreams < 1 || nstreams > 16 || mode < 0 || mode > 2)
      return -1;
    T3pProgram prog(o, v, naux, o - 1, 0, nstreams);
    return prog.plan_hazards(mode == 1) + prog.placement_clobbers(mode == 2);
  } catch (const std::exception& e) {
    record_error(e.what());
    return -1;
  }
}

const char* ascc_status_string(ascc_status s) {
  switch (s) {
    case ASCC_OK: return "ok";
    case ASCC_ERR_INVALID: return "invalid argument";
    case ASCC_ERR_OOM: return "out of device memory";
    case ASCC_ERR_CUDA: return "CUDA error";
    case ASCC_ERR_NOT_CONVERGED: return "not converged";
    case ASCC_ERR_DIVERGED: return "diverged";
    case ASCC_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

const char* ascc_last_error(void) { return g_err.c_str(); }

}  // extern "C"
