// Residual engine: einsum planner, bare integrals, and the ASCC/PLASCC
// residual and Jacobi+DIIS iteration on one GPU (FP64 path).
//
// Formulation (arXiv 2501.10515, Sec. II.A): the working equations are the
// ground-state CC equations over Hbar = exp(S^+) H exp(-S^+).  Both S^+ and
// T1 act as one-body orbital transforms, so per iteration the engine forms
//     B-hat^P = L B^P R,   L = (1 - t1)(1 + x),  R = (1 - x)(1 + t1),
// (x[h][p] = 1/sqrt2, Eq. 1CSF-S) and evaluates the closed-shell doubles-only
// CC equations of that non-Hermitian two-body Hamiltonian.  All blocks except
// the particle-particle ladder come from B-hat by density fitting; the
// ladder uses the bare (xc|bd) integrals, built once per molecule, with the
// L and R dressings applied to the output and to the amplitudes.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>

#include "engine.h"
#include "gemm_oz.h"
#include "gemm_tc.h"
#include "kernels.h"
#include "t3p.h"

namespace ascc {

namespace {
std::vector<int64_t> row_major_strides(const std::vector<int64_t>& shape) {
  std::vector<int64_t> st(shape.size());
  int64_t acc = 1;
  for (int d = (int)shape.size() - 1; d >= 0; --d) {
    st[d] = acc;
    acc *= shape[d];
  }
  return st;
}

struct Spec {
  std::string a, b, c;
};

Spec parse(const char* spec, bool two) {
  std::string s(spec);
  Spec r;
  auto arrow = s.find("->");
  ASCC_REQUIRE(arrow != std::string::npos, "einsum: missing ->");
  r.c = s.substr(arrow + 2);
  std::string lhs = s.substr(0, arrow);
  if (two) {
    auto comma = lhs.find(',');
    ASCC_REQUIRE(comma != std::string::npos, "einsum: two operands expected");
    r.a = lhs.substr(0, comma);
    r.b = lhs.substr(comma + 1);
  } else {
    r.a = lhs;
  }
  return r;
}
}  // namespace

void box_copy(cudaStream_t s, double* out, std::vector<int64_t> ostride, const double* in,
              std::vector<int64_t> istride, std::vector<int64_t> shape, double alpha,
              double beta) {
  k::strided_copy(s, out, ostride.data(), in, istride.data(), (int)shape.size(), shape.data(),
                  alpha, beta);
}

void Einsum::cache_reset(size_t bytes) const {
  cache_.clear();
  cache_used_ = 0;
  if (cache_buf_.bytes() < bytes && !frozen_) cache_buf_.alloc(bytes, s_);
}

void* Einsum::scratch(int which, size_t bytes) const {
  DevBuf& b = scratch_[which];
  if (b.bytes() < bytes) {
    ASCC_REQUIRE(!frozen_, "einsum scratch would grow during a graph capture");
    b.alloc(bytes + bytes / 8, s_);
  }
  return b.as<void>();
}

void Einsum::perm(const char* spec, double alpha, const T& A, double beta, const T& C) const {
  Spec sp = parse(spec, false);
  ASCC_REQUIRE((int)sp.a.size() == A.nd() && (int)sp.c.size() == C.nd(), "perm: rank");
  auto ast = row_major_strides(A.shape);
  std::vector<int64_t> istride, shape;
  for (char ch : sp.c) {
    auto pos = sp.a.find(ch);
    ASCC_REQUIRE(pos != std::string::npos, "perm: label");
    istride.push_back(ast[pos]);
    shape.push_back(A.shape[pos]);
  }
  for (int d = 0; d < C.nd(); ++d) ASCC_REQUIRE(C.shape[d] == shape[d], "perm: shape");
  box_copy(s_, C.p, row_major_strides(C.shape), A.p, istride, shape, alpha, beta);
}

namespace {
// X (labels xl, row-major) as the matrix [rows ml][cols kl]: each side's
// dimensions in label order, unit dimensions dropped and neighbours that are
// contiguous in X merged.  False when a side needs more than 4 dimensions or
// neither side's last dimension is contiguous (its reads would not coalesce;
// a contiguous row side is read by the transposing split kernels).
bool matrix_view(const T& X, const std::string& xl, const std::string& ml, const std::string& kl,
                 MatView& v, bool any_layout = false) {
  const auto st = row_major_strides(X.shape);
  auto side = [&](const std::string& l, int64_t* ext, int64_t* str, int& n) {
    n = 0;
    for (char ch : l) {
      const auto pos = xl.find(ch);
      const int64_t e = X.shape[pos], s = st[pos];
      if (e == 1) continue;
      if (n > 0 && str[n - 1] == s * e) {
        ext[n - 1] *= e;
        str[n - 1] = s;
        continue;
      }
      if (n == 4) return false;
      ext[n] = e;
      str[n] = s;
      ++n;
    }
    if (n == 0) {
      ext[0] = 1;
      str[0] = 0;
      n = 1;
    }
    return true;
  };
  if (!side(ml, v.mext, v.mstr, v.nm) || !side(kl, v.kext, v.kstr, v.nk)) return false;
  return any_layout || v.kstr[v.nk - 1] == 1 || v.mstr[v.nm - 1] == 1;
}
}  // namespace

void Einsum::operator()(const char* spec, double alpha, const T& A, const T& B, double beta,
                        const T& C) const {
  // the operand keys hold for this call only
  const int64_t key_a = key_a_, key_b = key_b_;
  key_a_ = key_b_ = -1;
  Spec sp = parse(spec, true);
  ASCC_REQUIRE((int)sp.a.size() == A.nd() && (int)sp.b.size() == B.nd() &&
                   (int)sp.c.size() == C.nd(),
               std::string("einsum rank mismatch: ") + spec);
  std::map<char, int64_t> size;
  for (int d = 0; d < A.nd(); ++d) size[sp.a[d]] = A.shape[d];
  for (int d = 0; d < B.nd(); ++d) {
    auto it = size.find(sp.b[d]);
    ASCC_REQUIRE(it == size.end() || it->second == B.shape[d], std::string("einsum size: ") + spec);
    size[sp.b[d]] = B.shape[d];
  }
  for (int d = 0; d < C.nd(); ++d)
    ASCC_REQUIRE(size.count(sp.c[d]) && size[sp.c[d]] == C.shape[d],
                 std::string("einsum out: ") + spec);
  auto in = [](const std::string& s, char c) { return s.find(c) != std::string::npos; };
  std::string bat, Ml, Nl, Kl;
  for (char ch : sp.c) {
    if (in(sp.a, ch) && in(sp.b, ch)) bat += ch;
    else if (in(sp.a, ch)) Ml += ch;
    else Nl += ch;
  }
  for (char ch : sp.a) {
    if (in(sp.b, ch) && !in(sp.c, ch)) Kl += ch;
    ASCC_REQUIRE(in(sp.b, ch) || in(sp.c, ch), std::string("einsum: lone label in ") + spec);
  }
  for (char ch : sp.b)
    ASCC_REQUIRE(in(sp.a, ch) || in(sp.c, ch), std::string("einsum: lone label in ") + spec);
  auto prod = [&](const std::string& l) {
    int64_t p = 1;
    for (char ch : l) p *= size[ch];
    return p;
  };
  // an output laid out [batch][N][M]: the same product with the operands
  // exchanged writes it directly
  if (sp.c != bat + Ml + Nl && sp.c == bat + Nl + Ml) {
    const std::string sw = sp.b + "," + sp.a + "->" + sp.c;
    key_a_ = key_b;
    key_b_ = key_a;
    (*this)(sw.c_str(), alpha, B, A, beta, C);
    return;
  }
  const int64_t nb = prod(bat), Ms = prod(Ml), Ns = prod(Nl), Ks = prod(Kl);
  auto shape_of = [&](const std::string& l) {
    std::vector<int64_t> sh;
    for (char ch : l) sh.push_back(size[ch]);
    return sh;
  };

  const std::string cl = bat + Ml + Nl;
  if (Ks == 1 && C.nd() <= 8) {
    // no contraction (an outer product or a scaled copy): written in place
    const auto ast = row_major_strides(A.shape), bst = row_major_strides(B.shape);
    const auto cst = row_major_strides(C.shape);
    std::vector<int64_t> as(C.nd(), 0), bs(C.nd(), 0);
    for (int d = 0; d < C.nd(); ++d) {
      const auto pa = sp.a.find(sp.c[d]), pb = sp.b.find(sp.c[d]);
      if (pa != std::string::npos) as[d] = ast[pa];
      if (pb != std::string::npos) bs[d] = bst[pb];
    }
    k::outer(s_, C.p, cst.data(), A.p, as.data(), B.p, bs.data(), C.nd(), C.shape.data(), alpha,
             beta);
    return;
  }
  if (level_ > 0 && nb == 1 && Ms > 1 && Ns > 1 && 2.0 * Ms * Ns * Ks >= min_flops_) {
    // tensor-core path: A as [M][K], B as [N][K] (K contiguous), split into
    // BF16 planes (or digit planes at level 4).  An operand in another layout
    // is split through a strided view when one of its sides is contiguous,
    // else permuted first; planes of a keyed operand come from the cache when
    // the same arrangement was split before.
    const bool oz_level = level_ == 4;
    const int64_t Kp = oz_level ? oz::padded_k(Ks) : tc::padded_k(Ks);
    const int nplanes = oz_level ? oz::NSLICE : level_;
    struct Planes {
      __nv_bfloat16* p = nullptr;
      int32_t* e = nullptr;
    };
    // BF16 splits are collected (job) and launched together after both operands
    tc::SplitSpec jobs[2];
    int njobs = 0;
    OT keep[2];  // permuted copies that a collected split still reads
    auto planes = [&](const T& X, const std::string& xl, const std::string& ml, int64_t key,
                      int which) {
      const int64_t rows = prod(ml);
      const size_t pbytes = sizeof(__nv_bfloat16) * (size_t)(nplanes * rows * Kp);
      const size_t ebytes = oz_level ? sizeof(int32_t) * (size_t)rows : 0;
      std::string sig;
      if (key >= 0) {
        sig = std::to_string(level_) + ":";
        for (char ch : ml) sig += std::to_string(xl.find(ch)) + ",";
        sig += "|";
        for (char ch : Kl) sig += std::to_string(xl.find(ch)) + ",";
        for (const auto& c : cache_)
          if (c.key == key && c.sig == sig) {
            Planes r;
            r.p = reinterpret_cast<__nv_bfloat16*>(cache_buf_.as<char>() + c.off);
            if (oz_level) r.e = reinterpret_cast<int32_t*>(cache_buf_.as<char>() + c.off + pbytes);
            return r;
          }
      }
      Planes r;
      const size_t need = (pbytes + ebytes + 255) / 256 * 256;
      if (key >= 0 && cache_buf_.bytes() > 0 && cache_used_ + need <= cache_buf_.bytes()) {
        r.p = reinterpret_cast<__nv_bfloat16*>(cache_buf_.as<char>() + cache_used_);
        if (oz_level) r.e = reinterpret_cast<int32_t*>(cache_buf_.as<char>() + cache_used_ + pbytes);
        cache_.push_back({key, sig, cache_used_});
        cache_used_ += need;
      } else {
        r.p = static_cast<__nv_bfloat16*>(scratch(which, pbytes));
        if (oz_level) r.e = static_cast<int32_t*>(scratch(3 + which, ebytes));
      }
      MatView vx;
      auto plain = [&](const double* src) {
        MatView pv;
        pv.nm = pv.nk = 1;
        pv.mext[0] = rows;
        pv.mstr[0] = Ks;
        pv.kext[0] = Ks;
        pv.kstr[0] = 1;
        jobs[njobs++] = tc::SplitSpec{r.p, src, pv, level_};
      };
      if (xl == ml + Kl) {
        if (oz_level)
          oz::split(s_, r.p, r.e, X.p, rows, Ks, Ks);
        else
          plain(X.p);
      } else if (matrix_view(X, xl, ml, Kl, vx)) {
        if (oz_level)
          oz::split_view(s_, r.p, r.e, X.p, vx);
        else
          jobs[njobs++] = tc::SplitSpec{r.p, X.p, vx, level_};
      } else {
        OT& Xt = keep[which];
        Xt.make(shape_of(ml + Kl), s_);
        perm((xl + "->" + ml + Kl).c_str(), 1.0, X, 0.0, Xt.t);
        if (oz_level)
          oz::split(s_, r.p, r.e, Xt.p(), rows, Ks, Ks);
        else
          plain(Xt.p());
      }
      return r;
    };
    const Planes qa = planes(A, sp.a, Ml, key_a, 0), qb = planes(B, sp.b, Nl, key_b, 1);
    if (njobs > 0) tc::split_bf16_pair(s_, &jobs[0], njobs > 1 ? &jobs[1] : nullptr);
    if (oz_level) {
      // exact digit-plane products (FP64-class)
      auto* ws = static_cast<long long*>(scratch(2, oz::ws_bytes(Ms, Ns)));
      const int z = oz::splitk_for(Ms, Ns, Ks, fill_ > 0);
      if (sp.c == cl) {
        oz::gemm(s_, Ms, Ns, Ks, alpha, qa.p, qa.e, 0, qb.p, qb.e, 0, beta, C.p, Ns, ws, err_, z);
      } else {
        OT Ct(shape_of(cl), s_);
        oz::gemm(s_, Ms, Ns, Ks, 1.0, qa.p, qa.e, 0, qb.p, qb.e, 0, 0.0, Ct.p(), Ns, ws, err_, z);
        perm((cl + "->" + sp.c).c_str(), alpha, Ct.t, beta, C);
      }
      return;
    }
    const __nv_bfloat16 *pa = qa.p, *pb = qb.p;
    const int z = tc::splitk_for(Ms, Ns, Ks, fill_);
    // an output in another layout is written through a view by the reduction
    MatView vc;
    const bool view_c = sp.c != cl && matrix_view(C, sp.c, Ml, Nl, vc, true);
    float* ws = (z > 1 || view_c)
                    ? static_cast<float*>(scratch(2, sizeof(float) * (size_t)(z * Ms * Ns)))
                    : nullptr;
    if (sp.c == cl) {
      tc::gemm_split(s_, Ms, Ns, Ks, level_, alpha, pa, pb, beta, C.p, Ns, err_, z, ws);
    } else if (view_c) {
      tc::gemm_split(s_, Ms, Ns, Ks, level_, alpha, pa, pb, beta, C.p, 0, err_, z, ws, 0, &vc);
    } else {
      OT Ct(shape_of(cl), s_);
      tc::gemm_split(s_, Ms, Ns, Ks, level_, 1.0, pa, pb, 0.0, Ct.p(), Ns, err_, z, ws);
      perm((cl + "->" + sp.c).c_str(), alpha, Ct.t, beta, C);
    }
    return;
  }
  // FP64 paths: operand A in (bat, M, K) or (bat, K, M), B in (bat, K, N) or
  // (bat, N, K); other layouts are permuted first
  bool ta = false;
  const double* Ap = A.p;
  OT Atmp;
  if (sp.a == bat + Ml + Kl) {
    ta = false;
  } else if (sp.a == bat + Kl + Ml) {
    ta = true;
  } else {
    std::string want = bat + Ml + Kl;
    Atmp.make(shape_of(want), s_);
    perm((sp.a + "->" + want).c_str(), 1.0, A, 0.0, Atmp.t);
    Ap = Atmp.p();
  }
  bool tb = false;
  const double* Bp = B.p;
  OT Btmp;
  if (sp.b == bat + Kl + Nl) {
    tb = false;
  } else if (sp.b == bat + Nl + Kl) {
    tb = true;
  } else {
    std::string want = bat + Kl + Nl;
    Btmp.make(shape_of(want), s_);
    perm((sp.b + "->" + want).c_str(), 1.0, B, 0.0, Btmp.t);
    Bp = Btmp.p();
  }
  const int64_t lda = ta ? Ms : Ks, ldb = tb ? Ks : Ns;
  if (Ms == 1 && Ns > 1 && nb == 1 && Ks > 0) {
    // vector-matrix product: a matrix-vector product with B as the matrix
    if (sp.c == cl) {
      k::gemv_f64(s_, !tb, Ns, Ks, alpha, Bp, ldb, Ap, beta, C.p);
    } else {
      OT Ct(shape_of(cl), s_);
      k::gemv_f64(s_, !tb, Ns, Ks, 1.0, Bp, ldb, Ap, 0.0, Ct.p());
      perm((cl + "->" + sp.c).c_str(), alpha, Ct.t, beta, C);
    }
    return;
  }
  if (Ns == 1 && nb == 1 && Ks > 0) {
    // matrix-vector product: memory-bound, FP64 on every path
    if (sp.c == cl) {
      k::gemv_f64(s_, ta, Ms, Ks, alpha, Ap, lda, Bp, beta, C.p);
    } else {
      OT Ct(shape_of(cl), s_);
      k::gemv_f64(s_, ta, Ms, Ks, 1.0, Ap, lda, Bp, 0.0, Ct.p());
      perm((cl + "->" + sp.c).c_str(), alpha, Ct.t, beta, C);
    }
    return;
  }
  if (sp.c == cl) {
    k::gemm_f64(s_, ta, tb, Ms, Ns, Ks, alpha, Ap, lda, Ms * Ks, Bp, ldb, Ks * Ns, beta, C.p, Ns,
                Ms * Ns, nb);
  } else {
    OT Ct(shape_of(cl), s_);
    k::gemm_f64(s_, ta, tb, Ms, Ns, Ks, 1.0, Ap, lda, Ms * Ks, Bp, ldb, Ks * Ns, 0.0, Ct.p(), Ns,
                Ms * Ns, nb);
    perm((cl + "->" + sp.c).c_str(), alpha, Ct.t, beta, C);
  }
}

// ---------------------------------------------------------------- Molecule
Molecule::Molecule(int o_, int v_, int naux_, const double* eps_h, const double* B_src,
                   bool on_device, cudaStream_t s, int build_level)
    : o(o_), v(v_), n(o_ + v_), naux(naux_), stream(s) {
  err.alloc(sizeof(int), s);
  err.zero();
  eps_host.assign(eps_h, eps_h + n);
  eps.make({n}, s);
  ASCC_CUDA(cudaMemcpyAsync(eps.p(), eps_h, sizeof(double) * n, cudaMemcpyHostToDevice, s));
  B.make({naux, n, n}, s);
  ASCC_CUDA(cudaMemcpyAsync(B.p(), B_src, sizeof(double) * (size_t)naux * n * n,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  Einsum es(s);
  // core Hamiltonian: h = diag(eps) - sum_i [2 (pq|ii) - (pi|iq)]
  OT d({naux}, s), J({n, n}, s), K({n, n}, s), Bno({naux, n, o}, s), Bon({naux, o, n}, s);
  k::diag_sum(s, d.p(), B.p(), naux, n, o);
  es("Ppq,P->pq", 1.0, B.t, d.t, 0.0, J.t);
  box_copy(s, Bno.p(), {(int64_t)n * o, o, 1}, B.p(), {(int64_t)n * n, n, 1}, {naux, n, o});
  box_copy(s, Bon.p(), {(int64_t)o * n, n, 1}, B.p(), {(int64_t)n * n, n, 1}, {naux, o, n});
  es("Ppk,Pkq->pq", 1.0, Bno.t, Bon.t, 0.0, K.t);
  hcore.make({n, n}, s);
  k::fill(s, hcore.p(), 0.0, (int64_t)n * n);
  box_copy(s, hcore.p(), {n + 1}, eps.p(), {1}, {n});  // diagonal
  k::axpby(s, hcore.p(), J.p(), -2.0, 1.0, (int64_t)n * n);
  k::axpby(s, hcore.p(), K.p(), 1.0, 1.0, (int64_t)n * n);
  // bare blocks for the ladder
  Bvv.make({naux, v, v}, s);
  box_copy(s, Bvv.p(), {(int64_t)v * v, v, 1}, B.p() + (int64_t)o * n + o, {(int64_t)n * n, n, 1},
           {naux, v, v});
  Bnv.make({naux, n, v}, s);
  box_copy(s, Bnv.p(), {(int64_t)n * v, v, 1}, B.p() + o, {(int64_t)n * n, n, 1}, {naux, n, v});
  build_level_ = build_level;
}

// Gext[x][b][c][d] = (xc|bd) = sum_P B[P][x][o+c] B[P][o+b][o+d], in FP64.
void Molecule::ensure_fp64_ladder() {
  std::lock_guard<std::mutex> lock(mu_);
  if (Gext.buf.bytes()) return;
  Einsum es(stream);
  Gext.make({n, v, v, v}, stream);
  es.set_split(0, err.as<int>(), 0.0);
  // x-chunks keep the GEMM's permutation temporary at ~1 GB
  const int64_t v3 = (int64_t)v * v * v;
  int64_t xc = std::max<int64_t>(1, ((int64_t)1 << 27) / v3);
  xc = std::min<int64_t>(xc, n);
  OT Ac({naux, xc, v}, stream);
  for (int64_t x0 = 0; x0 < n; x0 += xc) {
    const int64_t nx = std::min<int64_t>(xc, n - x0);
    T a(Ac.p(), {naux, nx, v}), gch(Gext.p() + x0 * v3, {nx, v, v, v});
    box_copy(stream, Ac.p(), {nx * v, v, 1}, Bnv.p() + x0 * v, {(int64_t)n * v, v, 1},
             {naux, nx, v});
    es("Pxc,Pbd->xbcd", 1.0, a, Bvv.t, 0.0, gch);
  }
  ASCC_CUDA(cudaStreamSynchronize(stream));
}

// BF16 planes of Gext for the mixed-precision ladder, built x-chunk by
// x-chunk (from the FP64 block when it exists, else on the tensor cores with
// the finest split) so that the FP64 block never has to exist in full.
void Molecule::ensure_bf16_ladder() {
  std::lock_guard<std::mutex> lock(mu_);
  if (Gext_bf16.bytes()) return;
  const int64_t rows = (int64_t)n * v, K = (int64_t)v * v, Kp = tc::padded_k(K);
  Gext_bf16.alloc(sizeof(__nv_bfloat16) * (size_t)(3 * rows * Kp), stream);
  if (Gext.buf.bytes()) {
    tc::split_bf16(stream, Gext_bf16.as<__nv_bfloat16>(), Gext.p(), rows, K, K, 3, rows * Kp);
    ASCC_CUDA(cudaStreamSynchronize(stream));
    return;
  }
  Einsum es(stream);
  es.set_split(build_level_ > 0 ? build_level_ : 3, err.as<int>(), 0.0);
  const int64_t v3 = (int64_t)v * v * v;
  int64_t xc = std::max<int64_t>(1, ((int64_t)1 << 27) / v3);  // ~1 GB FP64 per chunk
  xc = std::min<int64_t>(xc, n);
  OT Ac({naux, xc, v}, stream), Gc({xc, v, v, v}, stream);
  for (int64_t x0 = 0; x0 < n; x0 += xc) {
    const int64_t nx = std::min<int64_t>(xc, n - x0);
    T a(Ac.p(), {naux, nx, v}), gch(Gc.p(), {nx, v, v, v});
    box_copy(stream, Ac.p(), {nx * v, v, 1}, Bnv.p() + x0 * v, {(int64_t)n * v, v, 1},
             {naux, nx, v});
    es("Pxc,Pbd->xbcd", 1.0, a, Bvv.t, 0.0, gch);
    tc::split_bf16(stream, Gext_bf16.as<__nv_bfloat16>() + x0 * v * Kp, Gc.p(), nx * v, K, K, 3,
                   rows * Kp);
  }
  int h = 0;
  ASCC_CUDA(cudaMemcpyAsync(&h, err.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, stream));
  ASCC_CUDA(cudaStreamSynchronize(stream));
  if (h) throw Error(ASCC_ERR_TIMEOUT, "tensor-core GEMM wait timed out while building (xc|bd)");
}

// Digit planes of Gext for FP64-class tensor-core ladders, built x-chunk by
// x-chunk with FP64-class contractions (or split from the FP64 block when it
// exists).
void Molecule::ensure_oz_ladder() {
  std::lock_guard<std::mutex> lock(mu_);
  if (Gext_oz.bytes()) return;
  const int64_t rows = (int64_t)n * v, K = (int64_t)v * v, Kq = oz::padded_k(K);
  Gext_oz.alloc(sizeof(__nv_bfloat16) * (size_t)(oz::NSLICE * rows * Kq), stream);
  Gext_oz_exp.alloc(sizeof(int32_t) * (size_t)rows, stream);
  auto* planes = Gext_oz.as<__nv_bfloat16>();
  auto* exps = Gext_oz_exp.as<int32_t>();
  if (Gext.buf.bytes()) {
    oz::split(stream, planes, exps, Gext.p(), rows, K, K, rows * Kq);
    ASCC_CUDA(cudaStreamSynchronize(stream));
    return;
  }
  Einsum es(stream);
  es.set_split(4, err.as<int>(), 0.0);
  const int64_t v3 = (int64_t)v * v * v;
  int64_t xc = std::max<int64_t>(1, ((int64_t)1 << 27) / v3);  // ~1 GB FP64 per chunk
  xc = std::min<int64_t>(xc, n);
  OT Ac({naux, xc, v}, stream), Gc({xc, v, v, v}, stream);
  for (int64_t x0 = 0; x0 < n; x0 += xc) {
    const int64_t nx = std::min<int64_t>(xc, n - x0);
    T a(Ac.p(), {naux, nx, v}), gch(Gc.p(), {nx, v, v, v});
    box_copy(stream, Ac.p(), {nx * v, v, 1}, Bnv.p() + x0 * v, {(int64_t)n * v, v, 1},
             {naux, nx, v});
    es("Pxc,Pbd->xbcd", 1.0, a, Bvv.t, 0.0, gch);
    oz::split(stream, planes + x0 * v * Kq, exps + x0 * v, Gc.p(), nx * v, K, K, rows * Kq);
  }
  int h = 0;
  ASCC_CUDA(cudaMemcpyAsync(&h, err.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, stream));
  ASCC_CUDA(cudaStreamSynchronize(stream));
  if (h) throw Error(ASCC_ERR_TIMEOUT, "tensor-core GEMM wait timed out while building (xc|bd)");
}

size_t Molecule::bytes() const {
  return eps.buf.bytes() + B.buf.bytes() + hcore.buf.bytes() + Bvv.buf.bytes() +
         Bnv.buf.bytes() + Gext.buf.bytes() + Gext_bf16.bytes() + Gext_oz.bytes() +
         Gext_oz_exp.bytes();
}

// ---------------------------------------------------------------- State
namespace {
std::vector<int32_t> t3p_index(int o, int v, int h, int p) {
  // alpha-beta-beta triples (i, j<k, a, b<c) with >= 3 primary spin orbitals
  // (Sec. II.B.1), in lexicographic order of (i, j, k, a, b, c).
  std::vector<int32_t> out;
  if (h < 0) return out;
  for (int i = 0; i < o; ++i)
    for (int j = 0; j < o; ++j)
      for (int kk = j + 1; kk < o; ++kk) {
        const int occ = (i == h) + (j == h || kk == h);
        if (occ == 0) continue;
        for (int a = 0; a < v; ++a) {
          const int have = occ + (a == p);
          if (have < 2) continue;
          for (int b = 0; b < v; ++b)
            for (int c = b + 1; c < v; ++c) {
              if (have >= 3 || b == p || c == p) {
                const int32_t row[6] = {i, j, kk, a, b, c};
                out.insert(out.end(), row, row + 6);
              }
            }
        }
      }
  return out;
}
}  // namespace

State::State(std::shared_ptr<Molecule> mol, int hole, int particle, double beta,
             const Options& opt, cudaStream_t s, double xsign)
    : mol_(std::move(mol)), opt_(opt), s_(s), es_(s) {
  o_ = mol_->o; v_ = mol_->v; n_ = mol_->n; naux_ = mol_->naux;
  hole_ = hole; particle_ = particle;
  beta_ = beta == 0.0 ? 1.0 : beta;
  xsign_ = xsign < 0 ? -1.0 : 1.0;
  xval_ = hole_ >= 0 ? xsign_ / std::sqrt(2.0) : 0.0;
  lh_ = hole_ >= 0 ? hole_ : opt_.pl_hole;
  lp_ = hole_ >= 0 ? particle_ : opt_.pl_particle;
  if (lh_ < 0) opt_.linearize = 0;
  ASCC_REQUIRE(opt_.precision == ASCC_FP64 || opt_.precision == ASCC_MIXED_BF16 ||
                   opt_.precision == ASCC_FP64_TC,
               "precision must be ASCC_FP64, ASCC_MIXED_BF16 or ASCC_FP64_TC");
  ASCC_REQUIRE(opt_.diis_dim >= 1 && opt_.diis_dim <= 32, "diis_dim in 1..32");
  if (opt_.triples && hole_ >= 0) t3idx_host_ = t3p_index(o_, v_, hole_, particle_);
  if (const char* env = std::getenv("ASCC_NO_GRAPHS")) t3_use_graphs_ = env[0] == '0';
  nu_ = v_ + (hole_ >= 0 ? 1 : 0);
  const int64_t N = namp();
  t_.make({N}, s);
  r_.make({N}, s);
  hist_t_.make({opt_.diis_dim, N}, s);
  hist_e_.make({opt_.diis_dim, N}, s);
  scal_.make({64}, s);
  work_.make({(int64_t)32 * 4 * 152 + 64}, s);
  coef_.make({32}, s);
  gram_.make({32 * 32}, s);
  const int o = o_, v = v_, n = n_, P = naux_;
  L_.make({n, n}, s); R_.make({n, n}, s);
  {
    const int nc = o + (hole_ >= 0 ? 1 : 0);
    LamC_.make({n, nc}, s); RhoC_.make({n, nc}, s);
    rowsC_.make({P, nc, n}, s); colsC_.make({P, n, nc}, s);
  }
  Bhat_.make({P, n, n}, s);
  hhat_.make({n, n}, s); F_.make({n, n}, s);
  dP_.make({P}, s); J_.make({n, n}, s); K_.make({n, n}, s);
  Boo_.make({P, o, o}, s); Bov_.make({P, o, v}, s); Bvo_.make({P, v, o}, s);
  Bvv_.make({P, v, v}, s); Bno_.make({P, n, o}, s); Bon_.make({P, o, n}, s);
  goooo_.make({o, o, o, o}, s); gooov_.make({o, o, o, v}, s); goovv_.make({o, o, v, v}, s);
  govov_.make({o, v, o, v}, s); gvovo_.make({v, o, v, o}, s); gvoov_.make({v, o, o, v}, s);
  gvvoo_.make({v, v, o, o}, s); Lvoov_.make({v, o, o, v}, s); Lovov_.make({o, v, o, v}, s);
  u_.make({o, o, v, v}, s); Z_.make({o, o, v, v}, s);
  WC_.make({o, o, v, v}, s); WD_.make({v, o, o, v}, s); Wq_.make({o, o, o, o}, s);
  Fvv_.make({v, v}, s); Foo_.make({o, o}, s); X_.make({P, o, v}, s);
  Y_.make({o, o, n, v}, s);
  tpair_.make({(int64_t)o * (o + 1) / 2, (int64_t)v * v}, s);
  Yvv_.make({(int64_t)o * (o + 1) / 2, (int64_t)v * v}, s);
  Yov_.make({(int64_t)o * o, (int64_t)o * v}, s); Yfull_.make({o, o, n, n}, s); Z1_.make({o, o, n, v}, s);
  {
    const int nc = o + (hole_ >= 0 ? 1 : 0);
    YC_.make({o, o, n, nc}, s); Z1C_.make({o, o, nc, v}, s);
  }
  tt_.make({o, o, nu_, nu_}, s); Yoo_.make({o, o, o, o}, s);
  if (opt_.linearize) {
    m_.make({o, o, v, v}, s);
    um_.make({o, o, v, v}, s);
  }
  err_.alloc(sizeof(int), s);
  err_.zero();
  if (opt_.precision == ASCC_MIXED_BF16) corr_.make({namp()}, s);
  if (const char* env = std::getenv("ASCC_TC_MIN_FLOPS")) tc_min_flops_ = std::atof(env);
  {
    // Jacobi denominators: the hole and particle of a one-CSF state are half
    // occupied in S phi0; their mean energy enters the non-primary amplitudes.
    std::vector<double> ee = mol_->eps_host;
    if (hole_ >= 0) {
      const double m = 0.5 * (ee[hole_] + ee[o_ + particle_]);
      ee[hole_] = m;
      ee[o_ + particle_] = m;
    }
    eps_eff_.make({n_}, s);
    ASCC_CUDA(cudaMemcpyAsync(eps_eff_.p(), ee.data(), sizeof(double) * n_, cudaMemcpyHostToDevice, s));
    ASCC_CUDA(cudaStreamSynchronize(s));
  }
  ASCC_CUDA(cudaStreamSynchronize(mol_->stream));
  if (const char* env = std::getenv("ASCC_LADDER_CHUNK_MB"))
    stream_chunk_bytes_ = std::max<int64_t>(1, std::atoll(env)) << 20;
  {
    // store the (xc|bd) blocks once per molecule, or rebuild chunks per residual
    const double rows = (double)n_ * v_, K = (double)v_ * v_;
    const double kp = std::ceil(K / 64.0) * 64.0, kq = std::ceil(K / 32.0) * 32.0;
    double need = 0.0;
    const bool have = mol_->Gext.buf.bytes() || mol_->Gext_bf16.bytes() || mol_->Gext_oz.bytes();
    if (opt_.precision == ASCC_MIXED_BF16) need = rows * (6.0 * kp + 12.0 * kq);
    else if (opt_.precision == ASCC_FP64_TC) need = rows * 12.0 * kq;
    else need = rows * 16.0 * K;
    const bool mixed = opt_.precision == ASCC_MIXED_BF16;
    if (opt_.ladder_stream == 1) {
      stream_ladder_ = true;
    } else if (opt_.ladder_stream == 0 && !have) {
      size_t freeb = 0, totalb = 0;
      ASCC_CUDA(cudaMemGetInfo(&freeb, &totalb));
      {
        // blocks the stream-ordered pool holds but no allocation uses are free too
        int dev = 0;
        cudaMemPool_t pool;
        uint64_t reserved = 0, used = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess &&
            cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) ==
                cudaSuccess &&
            cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess &&
            reserved > used)
          freeb += (size_t)(reserved - used);
      }
      if (need > 0.6 * (double)freeb) {
        // mixed precision whose two forms of the block do not fit: the digit
        // planes alone (the exact ladder in every phase), else streaming
        if (mixed && rows * 12.0 * kq <= 0.6 * (double)freeb)
          ladder_digits_ = true;
        else
          stream_ladder_ = true;
      }
    } else if (mixed && have && mol_->Gext_oz.bytes() && !mol_->Gext_bf16.bytes()) {
      ladder_digits_ = true;  // a sibling of a state that stored the digit planes alone
    }
  }
  if (stream_ladder_) {
    // nothing stored: ladder_streamed() rebuilds the block in x-chunks
  } else if (opt_.precision == ASCC_MIXED_BF16) {
    if (!ladder_digits_) mol_->ensure_bf16_ladder();
    mol_->ensure_oz_ladder();  // FP64-class polishing evaluations
  } else if (opt_.precision == ASCC_FP64_TC) {
    mol_->ensure_oz_ladder();
  } else {
    mol_->ensure_fp64_ladder();
  }
  build_state_integrals();
  if (n3() > 0) setup_triples();
}

// Packed T3' order -> positions in the blocks TA..TD (see t3p.h): h is moved
// into the j slot and p into the b slot, each swap flipping the sign; TA and
// TC also receive the antisymmetric partner (c, b) / (k, j).
void State::setup_triples() {
  const int o = o_, v = v_, h = hole_, p = particle_;
  const int ns = t3p_streams();
  t3p_ = std::make_unique<T3pProgram>(o, v, naux_, h, p, ns);
  const int64_t N3 = n3();
  std::vector<int64_t> dst(N3), dst2(N3);
  std::vector<signed char> sgn(N3);
  const int64_t oA = t3p_->block_offset(0), oB = t3p_->block_offset(1),
                oC = t3p_->block_offset(2), oD = t3p_->block_offset(3);
  for (int64_t q = 0; q < N3; ++q) {
    const int32_t* x = &t3idx_host_[6 * q];
    int i = x[0], j = x[1], kk = x[2], a = x[3], b = x[4], c = x[5];
    int sg = 1;
    int64_t d1 = -1, d2 = -1;
    if (i == h && (j == h || kk == h)) {
      if (j != h) { std::swap(j, kk); sg = -sg; }
      if (a == p) {
        d1 = oA + ((int64_t)kk * v + b) * v + c;
        d2 = oA + ((int64_t)kk * v + c) * v + b;
      } else {
        if (b != p) { std::swap(b, c); sg = -sg; }
        d1 = oB + ((int64_t)kk * v + a) * v + c;
      }
    } else if (i == h) {
      if (b != p) { std::swap(b, c); sg = -sg; }
      d1 = oC + ((int64_t)j * o + kk) * v + c;
      d2 = oC + ((int64_t)kk * o + j) * v + c;
    } else {
      if (j != h) { std::swap(j, kk); sg = -sg; }
      if (b != p) { std::swap(b, c); sg = -sg; }
      d1 = oD + ((int64_t)i * o + kk) * v + c;
    }
    dst[q] = d1;
    dst2[q] = d2;
    sgn[q] = (signed char)sg;
  }
  t3dst_.alloc(sizeof(int64_t) * N3, s_);
  t3dst2_.alloc(sizeof(int64_t) * N3, s_);
  t3sgn_.alloc(N3, s_);
  t3idx_.alloc(sizeof(int32_t) * 6 * N3, s_);
  ASCC_CUDA(cudaMemcpyAsync(t3dst_.as<int64_t>(), dst.data(), sizeof(int64_t) * N3,
                            cudaMemcpyHostToDevice, s_));
  ASCC_CUDA(cudaMemcpyAsync(t3dst2_.as<int64_t>(), dst2.data(), sizeof(int64_t) * N3,
                            cudaMemcpyHostToDevice, s_));
  ASCC_CUDA(cudaMemcpyAsync(t3sgn_.as<signed char>(), sgn.data(), N3, cudaMemcpyHostToDevice, s_));
  ASCC_CUDA(cudaMemcpyAsync(t3idx_.as<int32_t>(), t3idx_host_.data(), sizeof(int32_t) * 6 * N3,
                            cudaMemcpyHostToDevice, s_));
  t3blk_.make({t3p_->block_elements()}, s_);
  r3blk_.make({t3p_->block_elements()}, s_);
  t3ws_.make({t3p_->workspace_elements()}, s_);
  if (ns > 1) {
    t3x_ = std::make_unique<T3pStreams>();
    T3pStreams& x = *t3x_;
    x.streams.push_back(s_);
    for (int k = 1; k < ns; ++k) {
      cudaStream_t st;
      ASCC_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      x.streams.push_back(st);
    }
    for (int k = 0; k < ns; ++k) x.es.push_back(std::make_unique<Einsum>(x.streams[k]));
    x.op_events.resize(t3p_->op_count());
    for (auto& e : x.op_events) ASCC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ASCC_CUDA(cudaEventCreateWithFlags(&x.fork, cudaEventDisableTiming));
    x.join.resize(ns);
    for (auto& e : x.join) ASCC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    t3priv_.make({(int64_t)ns * t3p_->block_elements()}, s_);
    x.priv = t3priv_.p();
  }
  t3ts_.make({o, o, v, v}, s_);
  if (opt_.linearize) t3nm_.make({o, o, v, v}, s_);
  ASCC_CUDA(cudaStreamSynchronize(s_));
}

void State::run_t3(int section, double* const* base, double scale) {
  const T3pProgram& P = *t3p_;
  double* ws = t3ws_.p();
  const bool conc = t3x_ && !P.profiling();
  if (conc)
    for (auto& e : t3x_->es) e->set_split(es_.level(), es_.err(), es_.min_flops());
  auto direct = [&] {
    if (conc)
      P.run_streams(*t3x_, section, base, scale, ws);
    else
      P.run(es_, s_, section, base, scale, ws);
  };
  auto freeze = [&](bool on) {
    es_.freeze(on);
    if (t3x_)
      for (auto& e : t3x_->es) e->freeze(on);
  };
  if (!t3_use_graphs_ || P.profiling()) {
    direct();
    return;
  }
  std::vector<uint64_t> key = {(uint64_t)section, (uint64_t)es_.level()};
  uint64_t sb;
  std::memcpy(&sb, &scale, sizeof(sb));
  key.push_back(sb);
  for (int b = 0; b < T3P_NBASE; ++b) key.push_back((uint64_t)(uintptr_t)base[b]);
  auto it = t3_graphs_.find(key);
  if (it == t3_graphs_.end()) {
    // first run of this form: direct, which also sizes the einsum scratch
    // (callers that pass new buffers on every call do not grow the cache)
    if (t3_graphs_.size() >= 64) {
      for (auto& kv : t3_graphs_)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
      t3_graphs_.clear();
    }
    t3_graphs_.emplace(key, T3Graph{});
    direct();
    return;
  }
  T3Graph& g = it->second;
  if (!g.exec && !g.failed) {
    const int64_t l0 = thread_launches();
    const double f0 = thread_flops();
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(s_, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      freeze(true);
      try {
        direct();
      } catch (const std::exception&) {
        ok = false;
      }
      freeze(false);
      ok = cudaStreamEndCapture(s_, &graph) == cudaSuccess && ok && graph;
    }
    // the captured launches did not run
    g.launches = thread_launches() - l0;
    g.flops = thread_flops() - f0;
    count_launch(-g.launches);
    count_flops(-g.flops);
    if (ok && cudaGraphInstantiate(&g.exec, graph, 0) != cudaSuccess) g.exec = nullptr;
    if (graph) cudaGraphDestroy(graph);
    if (!g.exec) {
      g.failed = true;
      cudaGetLastError();
    }
  }
  if (g.exec) {
    ASCC_CUDA(cudaGraphLaunch(g.exec, s_));
    count_launch(g.launches);
    count_flops(g.flops);
  } else {
    direct();
  }
}

// R3' and the T3' terms of R1 and R2 by the generated program (t3p.h); the
// partially linearised state drops the T2^M T2^M and T2^M T3' parts of R3'
// (Sec. II.C).
void State::triples(const T& t2, const double* t3, const T& r1, const T& r2, double* r3) {
  const T3pProgram& P = *t3p_;
  const int64_t nb = P.block_elements(), N3 = n3();
  k::t3p_unpack(s_, t3blk_.p(), nb, t3, t3dst_.as<int64_t>(), t3dst2_.as<int64_t>(),
                t3sgn_.as<signed char>(), N3);
  k::fill(s_, r3blk_.p(), 0.0, nb);
  double* base[T3P_NBASE] = {};
  base[T3P_F] = F_.p();
  base[T3P_B] = Bhat_.p();
  for (int b = 0; b < 4; ++b) {
    base[T3P_TA + b] = t3blk_.p() + P.block_offset(b);
    base[T3P_RA + b] = r3blk_.p() + P.block_offset(b);
  }
  base[T3P_R1] = r1.p;
  base[T3P_R2] = r2.p;
  double* ws = t3ws_.p();
  auto bind = [&](double* t) {
    // ts = t - t^(i<->j), the same-spin doubles of the singlet
    es_.perm("ijab->jiab", -1.0, T(t, {o_, o_, v_, v_}), 0.0, t3ts_.t);
    k::axpby(s_, t3ts_.p(), t, 1.0, 1.0, n2());
    base[T3P_T2] = t;
    base[T3P_TS] = t3ts_.p();
  };
  run_t3(T3P_PRO, base, 1.0);
  bind(t2.p);
  run_t3(T3P_LIN, base, 1.0);
  run_t3(T3P_QUAD, base, 1.0);
  if (opt_.linearize) {
    bind(m_.p());
    run_t3(T3P_QUAD, base, -1.0);
    k::axpby(s_, t3nm_.p(), t2.p, 1.0, 0.0, n2());
    k::axpby(s_, t3nm_.p(), m_.p(), -1.0, 1.0, n2());
    bind(t3nm_.p());
  }
  run_t3(T3P_MIX, base, 1.0);
  k::t3p_gather(s_, r3, r3blk_.p(), t3dst_.as<int64_t>(), t3sgn_.as<signed char>(), N3);
}

// Mixed precision: 3 BF16 products (16 significant bits) until max|R| reaches
// polish_tol, then 6 products (24 bits) with a defect correction: the residual
// is R6(t) + [R64(t0) - R6(t0)] with R64 the FP64-class (digit-plane)
// residual, refreshed at hand-over and whenever the corrected iteration
// converges, so that the accepted amplitudes satisfy the FP64 equations.
int State::level_for_phase() const {
  if (opt_.precision == ASCC_FP64_TC || fallback_) return 4;
  if (opt_.precision != ASCC_MIXED_BF16) return 0;
  return polish_ ? 3 : 2;
}

State::~State() {
  for (auto& kv : t3_graphs_)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  if (t3x_) {
    T3pStreams& x = *t3x_;
    cudaStreamSynchronize(s_);
    x.es.clear();
    for (auto& e : x.op_events) cudaEventDestroy(e);
    for (auto& e : x.join) cudaEventDestroy(e);
    if (x.fork) cudaEventDestroy(x.fork);
    for (size_t k = 1; k < x.streams.size(); ++k) cudaStreamDestroy(x.streams[k]);
  }
  for (auto& ev : events_) {
    cudaEventDestroy(ev.first);
    cudaEventDestroy(ev.second);
  }
}

void State::build_state_integrals() {
  const int o = o_, v = v_, n = n_, P = naux_, nu = nu_;
  Molecule& M = *mol_;
  // Goo[k][l][u][w] = (k u | l w), u, w over the virtuals plus the hole slot
  OT Bou({P, o, nu}, s_);
  box_copy(s_, Bou.p(), {(int64_t)o * nu, nu, 1}, M.B.p() + o, {(int64_t)n * n, n, 1}, {P, o, v});
  if (hole_ >= 0)
    box_copy(s_, Bou.p() + v, {(int64_t)o * nu, nu}, M.B.p() + hole_, {(int64_t)n * n, n},
             {P, o});
  GooP.make({o, o, nu, nu}, s_);
  es_("Pku,Plw->kluw", 1.0, Bou.t, Bou.t, 0.0, GooP.t);
  if (hole_ < 0) return;
  const int h = hole_;
  // Bh[P][x] = B[P][x][h]; Bvh[P][b] = B[P][o+b][h]
  OT Bh({P, n}, s_), Bvh({P, v}, s_);
  box_copy(s_, Bh.p(), {n, 1}, M.B.p() + h, {(int64_t)n * n, n}, {P, n});
  box_copy(s_, Bvh.p(), {v, 1}, M.B.p() + (int64_t)o * n + h, {(int64_t)n * n, n}, {P, v});
  Gh1.make({n, v, v}, s_);  // (x h | b d)
  es_("Px,Pbd->xbd", 1.0, Bh.t, M.Bvv.t, 0.0, Gh1.t);
  Gh2.make({n, v, v}, s_);  // (x c | b h) at [x][b][c]
  es_("Pxc,Pb->xbc", 1.0, M.Bnv.t, Bvh.t, 0.0, Gh2.t);
  Gh3.make({n, v}, s_);     // (x h | b h)
  es_("Px,Pb->xb", 1.0, Bh.t, Bvh.t, 0.0, Gh3.t);
}

void State::initial_guess(std::vector<double>& t) const {
  // Eq. TP-guess: t1[h][p] = beta/sqrt2, t2[h][h][p][p] = -beta^2/2; else 0
  // (t1[h][p] = -beta/sqrt2 for the second ansatz, S -> -S).
  t.assign((size_t)namp(), 0.0);
  if (hole_ < 0) return;
  t[(size_t)hole_ * v_ + particle_] = xsign_ * beta_ / std::sqrt(2.0);
  const int64_t i2 = (((int64_t)hole_ * o_ + hole_) * v_ + particle_) * v_ + particle_;
  t[(size_t)(n1() + i2)] = -0.5 * beta_ * beta_;
}

// B-hat = L B R and h-hat = L h R with the S^+ and T1 orbital transforms.
// L = 1 + Lambda and R = 1 + Rho have non-zero off-identity columns only in
// C = {occupied} (+ {p} for a one-CSF state), so
//   B-hat = B1 + (B1 Rho_C) scattered into the columns C,  B1 = B + Lambda_C B[C, :],
// which costs 4 n^2 |C| per DF index instead of 4 n^3.
void State::dress(const double* t1) {
  const int n = n_, P = naux_, o = o_;
  Molecule& M = *mol_;
  k::build_LR(s_, L_.p(), R_.p(), t1, o_, v_, hole_, particle_, xval_);
  const int64_t nn = (int64_t)n * n;
  const int nc = o + (hole_ >= 0 ? 1 : 0);
  const int pcol = hole_ >= 0 ? o + particle_ : -1;
  k::cols_minus_identity(s_, LamC_.p(), L_.p(), n, o, pcol, nc);
  k::cols_minus_identity(s_, RhoC_.p(), R_.p(), n, o, pcol, nc);
  auto apply = [&](const double* src, double* dst, int batch) {
    // rows C of src
    box_copy(s_, rowsC_.p(), {(int64_t)nc * n, n, 1}, src, {nn, n, 1}, {batch, o, n});
    if (pcol >= 0)
      box_copy(s_, rowsC_.p() + (int64_t)o * n, {(int64_t)nc * n, 1}, src + (int64_t)pcol * n,
               {nn, 1}, {batch, n});
    ASCC_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * nn * batch, cudaMemcpyDeviceToDevice, s_));
    if (es_.level() > 0 && batch > 1) {
      // tensor-core states: both K = |C| products as single FP64-class
      // digit-plane GEMMs over all DF indices (FP64 DFMA is the scarce unit)
      const int lev = es_.level();
      es_.set_split(4, err_.as<int>(), tc_min_flops_);
      T lam(LamC_.p(), {n, nc}), rho(RhoC_.p(), {n, nc});
      T rows(rowsC_.p(), {batch, nc, n}), cols(colsC_.p(), {batch, n, nc}), d(dst, {batch, n, n});
      es_("pk,Pkq->Ppq", 1.0, lam, rows, 1.0, d);
      es_("Ppq,qj->Ppj", 1.0, d, rho, 0.0, cols);
      es_.set_split(lev, err_.as<int>(), tc_min_flops_);
    } else {
      k::gemm_f64(s_, false, false, n, n, nc, 1.0, LamC_.p(), nc, 0, rowsC_.p(), n,
                  (int64_t)nc * n, 1.0, dst, n, nn, batch);
      k::gemm_f64(s_, false, false, n, nc, n, 1.0, dst, n, nn, RhoC_.p(), nc, 0, 0.0, colsC_.p(),
                  nc, (int64_t)n * nc, batch);
    }
    box_copy(s_, dst, {nn, n, 1}, colsC_.p(), {(int64_t)n * nc, nc, 1}, {batch, n, o}, 1.0, 1.0);
    if (pcol >= 0)
      box_copy(s_, dst + pcol, {nn, n}, colsC_.p() + o, {(int64_t)n * nc, nc}, {batch, n}, 1.0,
               1.0);
  };
  apply(M.B.p(), Bhat_.p(), P);
  apply(M.hcore.p(), hhat_.p(), 1);
  const int v = v_;
  const std::vector<int64_t> bs = {nn, n, 1};
  box_copy(s_, Boo_.p(), {(int64_t)o * o, o, 1}, Bhat_.p(), bs, {P, o, o});
  box_copy(s_, Bov_.p(), {(int64_t)o * v, v, 1}, Bhat_.p() + o, bs, {P, o, v});
  box_copy(s_, Bvo_.p(), {(int64_t)v * o, o, 1}, Bhat_.p() + (int64_t)o * n, bs, {P, v, o});
  box_copy(s_, Bvv_.p(), {(int64_t)v * v, v, 1}, Bhat_.p() + (int64_t)o * n + o, bs, {P, v, v});
  box_copy(s_, Bno_.p(), {(int64_t)n * o, o, 1}, Bhat_.p(), bs, {P, n, o});
  box_copy(s_, Bon_.p(), {(int64_t)o * n, n, 1}, Bhat_.p(), bs, {P, o, n});
  // Fock matrix of H-hat: F = h + 2 J - K.  F enters R1 and R2 with O(1)
  // weight, so it (and the oooo block of the reference energy) is built in
  // FP64, or with the FP64-class digit-plane products when the state uses
  // the tensor cores.
  const int lev = es_.level();
  es_.set_split(lev ? 4 : 0, err_.as<int>(), tc_min_flops_);
  k::diag_sum(s_, dP_.p(), Bhat_.p(), P, n, o);
  es_("Ppq,P->pq", 1.0, Bhat_.t, dP_.t, 0.0, J_.t);
  es_("Ppk,Pkq->pq", 1.0, Bno_.t, Bon_.t, 0.0, K_.t);
  es_("Pij,Pkl->ijkl", 1.0, Boo_.t, Boo_.t, 0.0, goooo_.t);
  es_.set_split(lev, err_.as<int>(), tc_min_flops_);
  k::axpby(s_, F_.p(), hhat_.p(), 1.0, 0.0, nn);
  k::axpby(s_, F_.p(), J_.p(), 2.0, 1.0, nn);
  k::axpby(s_, F_.p(), K_.p(), -1.0, 1.0, nn);
  // integral blocks (pq|rs)-hat = sum_P B-hat[P][p][q] B-hat[P][r][s]
  es_("Pij,Pka->ijka", 1.0, Boo_.t, Bov_.t, 0.0, gooov_.t);
  es_("Pij,Pab->ijab", 1.0, Boo_.t, Bvv_.t, 0.0, goovv_.t);
  es_("Pia,Pjb->iajb", 1.0, Bov_.t, Bov_.t, 0.0, govov_.t);
  es_("Pai,Pbj->aibj", 1.0, Bvo_.t, Bvo_.t, 0.0, gvovo_.t);
  es_("Pai,Pjb->aijb", 1.0, Bvo_.t, Bov_.t, 0.0, gvoov_.t);
  es_("Pab,Pij->abij", 1.0, Bvv_.t, Boo_.t, 0.0, gvvoo_.t);
  // L_aikc = 2 g_aikc - g_acki ; L_ldkc = 2 g_ldkc - g_lckd
  k::axpby(s_, Lvoov_.p(), gvoov_.p(), 2.0, 0.0, gvoov_.t.size());
  es_.perm("acki->aikc", -1.0, gvvoo_.t, 1.0, Lvoov_.t);
  k::axpby(s_, Lovov_.p(), govov_.p(), 2.0, 0.0, govov_.t.size());
  es_.perm("lckd->ldkc", -1.0, govov_.t, 1.0, Lovov_.t);
}

// Particle-particle ladder sum_cd g-hat_acbd t_ij^cd with g-hat dressed by L
// (output indices a, b) and R (summed indices c, d): the bare (xc|bd) carry
// the dense O(o^2 v^4) part, the hole-slot terms of R (c or d = p, Eq.
// 1CSF-S) and the occupied rows of L are O(N^5) corrections.
void State::ladder(const T& t2, const T& r2) {
  const int o = o_, v = v_, n = n_, nu = nu_;
  Molecule& M = *mol_;
  const int64_t vv = (int64_t)v * v;
  // Y[i][j][x][b] = sum_cd t[i][j][c][d] (xc|bd)
  // profiling brackets the dominant launch: the virtual-row GEMM (kernel and
  // its split-K reduction), or the whole streamed ladder
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  auto prof_begin = [&]() {
    if (!profile_) return;
    ASCC_CUDA(cudaEventCreate(&ev0));
    ASCC_CUDA(cudaEventCreate(&ev1));
    ASCC_CUDA(cudaEventRecord(ev0, s_));
  };
  auto prof_end = [&]() {
    if (profile_) ASCC_CUDA(cudaEventRecord(ev1, s_));
  };
  // (xc|bd) = (bd|xc) and t_ji^dc = t_ij^cd give Y_ji^{ab} = Y_ij^{ba} for the
  // virtual rows x = o+a: those come from the o(o+1)/2 pairs i <= j only; the
  // occupied rows x = k need every pair.
  const int64_t npair = (int64_t)o * (o + 1) / 2, ovr = (int64_t)o * v, vvr = vv;
  k::gather_pairs(s_, tpair_.p(), t2.p, o, vv);
  if (stream_ladder_) {
    prof_begin();
    ladder_streamed(t2);
    prof_end();
  } else if (es_.level() == 4 || (ladder_digits_ && es_.level() > 0)) {
    // exact digit-plane products (also in the low-precision phase of a mixed
    // state that holds the block as digit planes only)
    const int64_t K = vv, Kq = oz::padded_k(K), rows = (int64_t)n * v;
    const __nv_bfloat16* G = M.Gext_oz.as<__nv_bfloat16>();
    const int32_t* eG = M.Gext_oz_exp.as<int32_t>();
    auto* pa = static_cast<__nv_bfloat16*>(
        es_.scratch(0, sizeof(__nv_bfloat16) * (size_t)(oz::NSLICE * (int64_t)o * o * Kq)));
    auto* ea = static_cast<int32_t*>(es_.scratch(3, sizeof(int32_t) * (size_t)o * o));
    // occupied rows: all pairs
    oz::split(s_, pa, ea, t2.p, (int64_t)o * o, K, K);
    auto* ws = static_cast<long long*>(es_.scratch(2, oz::ws_bytes((int64_t)o * o, ovr)));
    oz::gemm(s_, (int64_t)o * o, ovr, K, 1.0, pa, ea, 0, G, eG, rows * Kq, 0.0, Yov_.p(), ovr, ws,
             err_.as<int>(), oz::splitk_for((int64_t)o * o, ovr, K));
    // virtual rows: pairs i <= j
    oz::split(s_, pa, ea, tpair_.p(), npair, K, K);
    ws = static_cast<long long*>(es_.scratch(2, oz::ws_bytes(npair, vvr)));
    prof_begin();
    oz::gemm(s_, npair, vvr, K, 1.0, pa, ea, 0, G + ovr * Kq, eG + ovr, rows * Kq, 0.0, Yvv_.p(),
             vvr, ws, err_.as<int>(), oz::splitk_for(npair, vvr, K));
    prof_end();
  } else if (es_.level() > 0) {
    const int lev = es_.level();
    const int64_t K = vv, Kp = tc::padded_k(K), rows = (int64_t)n * v;
    // planes of Gext are stored [3][rows][Kp]; the kernel reads planes 0..lev-1
    const __nv_bfloat16* G = M.Gext_bf16.as<__nv_bfloat16>();
    auto* pa = static_cast<__nv_bfloat16*>(
        es_.scratch(0, sizeof(__nv_bfloat16) * (size_t)(lev * (int64_t)o * o * Kp)));
    // occupied rows: all pairs
    tc::split_bf16(s_, pa, t2.p, (int64_t)o * o, K, K, lev);
    int z = tc::splitk_for((int64_t)o * o, ovr, K);
    float* ws = z > 1 ? static_cast<float*>(
                            es_.scratch(2, sizeof(float) * (size_t)(z * (int64_t)o * o * ovr)))
                      : nullptr;
    tc::gemm_split(s_, (int64_t)o * o, ovr, K, lev, 1.0, pa, G, 0.0, Yov_.p(), ovr, err_.as<int>(),
                   z, ws, rows * Kp);
    // virtual rows: pairs i <= j
    tc::split_bf16(s_, pa, tpair_.p(), npair, K, K, lev);
    z = tc::splitk_for(npair, vvr, K);
    ws = z > 1 ? static_cast<float*>(es_.scratch(2, sizeof(float) * (size_t)(z * npair * vvr)))
               : nullptr;
    prof_begin();
    tc::gemm_split(s_, npair, vvr, K, lev, 1.0, pa, G + ovr * Kp, 0.0, Yvv_.p(), vvr,
                   err_.as<int>(), z, ws, rows * Kp);
    prof_end();
  } else {
    const double* G = M.Gext.p();
    k::gemm_f64(s_, false, true, (int64_t)o * o, ovr, vv, 1.0, t2.p, vv, 0, G, vv, 0, 0.0,
                Yov_.p(), ovr, 0, 1);
    prof_begin();
    k::gemm_f64(s_, false, true, npair, vvr, vv, 1.0, tpair_.p(), vv, 0, G + ovr * vv, vv,
                0, 0.0, Yvv_.p(), vvr, 0, 1);
    prof_end();
  }
  // Y[i][j][k][b] = Yov[ij][k b];  Y[i][j][o+a][b] from the pair products
  box_copy(s_, Y_.p(), {(int64_t)n * v, 1}, Yov_.p(), {ovr, 1}, {(int64_t)o * o, ovr});
  k::scatter_pairs(s_, Y_.p(), Yvv_.p(), o, v, n);
  if (profile_) {
    events_.push_back({ev0, ev1});
    ladder_launches_ += 1;
    const double fl = stream_ladder_
                          ? 2.0 * (double)vv * ((double)o * o * o * v + (double)npair * vv)
                          : 2.0 * (double)npair * vvr * vv;
    ladder_flops_ += fl;
    ladder_mma_flops_ += fl * ((es_.level() == 4 || ladder_digits_) ? oz::products()
                               : es_.level() > 0 ? tc::products_for(es_.level())
                                                 : 1);
  }
  // R-dressed amplitudes tt[i][j][u][w], u, w over the virtuals (+ hole slot)
  const int64_t s4[4] = {(int64_t)o * vv, vv, v, 1};
  box_copy(s_, tt_.p(), {(int64_t)o * nu * nu, (int64_t)nu * nu, nu, 1}, t2.p,
           {s4[0], s4[1], s4[2], s4[3]}, {o, o, v, v});
  if (hole_ >= 0) {
    const int p = particle_;
    const double x = xval_;
    OT tpd({o, o, v}, s_), tcp({o, o, v}, s_), tpp({o, o}, s_);
    box_copy(s_, tpd.p(), {(int64_t)o * v, v, 1}, t2.p + (int64_t)p * v, {s4[0], s4[1], 1},
             {o, o, v});
    box_copy(s_, tcp.p(), {(int64_t)o * v, v, 1}, t2.p + p, {s4[0], s4[1], v}, {o, o, v});
    box_copy(s_, tpp.p(), {o, 1}, t2.p + (int64_t)p * v + p, {s4[0], s4[1]}, {o, o});
    es_("ijd,xbd->ijxb", -x, tpd.t, Gh1.t, 1.0, Y_.t);
    es_("ijc,xbc->ijxb", -x, tcp.t, Gh2.t, 1.0, Y_.t);
    es_("ij,xb->ijxb", x * x, tpp.t, Gh3.t, 1.0, Y_.t);
    const int64_t so = (int64_t)o * nu * nu;
    box_copy(s_, tt_.p() + (int64_t)v * nu, {so, (int64_t)nu * nu, 1}, tpd.p(),
             {(int64_t)o * v, v, 1}, {o, o, v}, -x);
    box_copy(s_, tt_.p() + v, {so, (int64_t)nu * nu, nu}, tcp.p(), {(int64_t)o * v, v, 1},
             {o, o, v}, -x);
    box_copy(s_, tt_.p() + (int64_t)v * nu + v, {so, (int64_t)nu * nu}, tpp.p(), {o, 1}, {o, o},
             x * x);
  }
  // Y_oo[i][j][k][l] = sum_uw tt[i][j][u][w] (k u | l w)
  es_("ijuw,kluw->ijkl", 1.0, tt_.t, GooP.t, 0.0, Yoo_.t);
  // Yfull[i][j][t][v'] over all orbitals t, v'
  const int64_t fs[4] = {(int64_t)o * n * n, (int64_t)n * n, n, 1};
  box_copy(s_, Yfull_.p() + o, {fs[0], fs[1], fs[2], 1}, Y_.p(),
           {(int64_t)o * n * v, (int64_t)n * v, v, 1}, {o, o, n, v});
  // Yfull[i][j][o+a][l] = Y[j][i][l][a]
  box_copy(s_, Yfull_.p() + (int64_t)o * n, {fs[0], fs[1], n, 1}, Y_.p(),
           {(int64_t)n * v, (int64_t)o * n * v, 1, v}, {o, o, v, o});
  box_copy(s_, Yfull_.p(), {fs[0], fs[1], n, 1}, Yoo_.p(),
           {(int64_t)o * o * o, (int64_t)o * o, o, 1}, {o, o, o, o});
  // r2[i][j][a][b] += sum_{t,v'} L[o+a][t] L[o+b][v'] Yfull[i][j][t][v'] with
  // L[o+a][.] = e_{o+a} + Lambda[o+a][C] (columns C = occupied + p only):
  //   Z1 = Yfull[.., V] + Yfull[.., C] Lambda_V^T,  r2 += Z1[V, ..] + Lambda_V Z1[C, ..]
  const int nc = o + (hole_ >= 0 ? 1 : 0);
  const int pcol = hole_ >= 0 ? o + particle_ : -1;
  const double* LamV = LamC_.p() + (int64_t)o * nc;  // rows o..n-1 of (L - 1)[:, C]
  const int64_t oo = (int64_t)o * o;
  box_copy(s_, Z1_.p(), {v, 1}, Yfull_.p() + o, {n, 1}, {oo * n, v});
  box_copy(s_, YC_.p(), {nc, 1}, Yfull_.p(), {n, 1}, {oo * n, o});
  if (pcol >= 0) box_copy(s_, YC_.p() + o, {nc}, Yfull_.p() + pcol, {n}, {oo * n});
  const int lev = es_.level();
  if (lev > 0) {
    // tensor-core states: the K = |C| products as FP64-class digit planes
    es_.set_split(4, err_.as<int>(), tc_min_flops_);
    es_("mk,ak->ma", 1.0, T(YC_.p(), {oo * n, nc}), T((double*)LamV, {v, nc}), 1.0,
        T(Z1_.p(), {oo * n, v}));
  } else {
    k::gemm_f64(s_, false, true, oo * n, v, nc, 1.0, YC_.p(), nc, 0, LamV, nc, 0, 1.0, Z1_.p(), v,
                0, 1);
  }
  box_copy(s_, r2.p, {vv, 1}, Z1_.p() + (int64_t)o * v, {(int64_t)n * v, 1}, {oo, vv}, 1.0, 1.0);
  box_copy(s_, Z1C_.p(), {(int64_t)nc * v, v, 1}, Z1_.p(), {(int64_t)n * v, v, 1}, {oo, o, v});
  if (pcol >= 0)
    box_copy(s_, Z1C_.p() + (int64_t)o * v, {(int64_t)nc * v, 1}, Z1_.p() + (int64_t)pcol * v,
             {(int64_t)n * v, 1}, {oo, v});
  if (lev > 0) {
    es_("ak,xkb->xab", 1.0, T((double*)LamV, {v, nc}), T(Z1C_.p(), {oo, nc, v}), 1.0,
        T(r2.p, {oo, v, v}));
    es_.set_split(lev, err_.as<int>(), tc_min_flops_);
  } else {
    k::gemm_f64(s_, false, false, v, v, nc, 1.0, LamV, nc, 0, Z1C_.p(), v, (int64_t)nc * v, 1.0,
                r2.p, v, vv, oo);
  }
}

// The ladder GEMMs with the bare block rebuilt chunk by chunk: for x in a
// chunk of orbitals, (xc|bd) = sum_P B[P][x][o+c] B[P][o+b][o+d] is built with
// FP64-class contractions (6 products for the 3-product phase), split for the
// state's precision and multiplied into the Yov (occupied x, all pairs) or Yvv
// (virtual x, pairs i <= j) columns of that chunk.  Nothing of size n v^3 is
// kept between calls.
void State::ladder_streamed(const T& t2) {
  const int o = o_, v = v_, n = n_, P = naux_;
  Molecule& M = *mol_;
  const int lev = es_.level();
  const int64_t vv = (int64_t)v * v, v3 = vv * v, ovr = (int64_t)o * v, vvr = vv;
  const int64_t npair = (int64_t)o * (o + 1) / 2, oo = (int64_t)o * o;
  int64_t xc = std::max<int64_t>(1, stream_chunk_bytes_ / (8 * v3));
  xc = std::min<int64_t>(xc, n);
  if (!stream_gc_.buf.bytes() || stream_gc_.t.shape[0] < xc) {
    stream_ac_.make({P, xc, v}, s_);
    stream_gc_.make({xc, v, v, v}, s_);
  }
  // the t operands (all pairs, pairs i <= j) in the state's number format, once
  const bool digits = lev == 4;
  const int64_t Kp = digits ? oz::padded_k(vv) : tc::padded_k(vv);
  const int planes = digits ? oz::NSLICE : lev;
  __nv_bfloat16 *a_occ = nullptr, *a_vir = nullptr;
  int32_t *e_occ = nullptr, *e_vir = nullptr;
  if (lev > 0) {
    const size_t need = sizeof(__nv_bfloat16) * (size_t)(planes * (oo + npair) * Kp);
    if (stream_a_.bytes() < need) stream_a_.alloc(need, s_);
    a_occ = stream_a_.as<__nv_bfloat16>();
    a_vir = a_occ + (int64_t)planes * oo * Kp;
    if (digits) {
      if (stream_ae_.bytes() < sizeof(int32_t) * (size_t)(oo + npair))
        stream_ae_.alloc(sizeof(int32_t) * (size_t)(oo + npair), s_);
      e_occ = stream_ae_.as<int32_t>();
      e_vir = e_occ + oo;
      oz::split(s_, a_occ, e_occ, t2.p, oo, vv, vv);
      oz::split(s_, a_vir, e_vir, tpair_.p(), npair, vv, vv);
    } else {
      tc::split_bf16(s_, a_occ, t2.p, oo, vv, vv, lev);
      tc::split_bf16(s_, a_vir, tpair_.p(), npair, vv, vv, lev);
    }
  }
  const int build = lev == 2 ? 3 : 4;
  for (int g = 0; g < 2; ++g) {
    const int64_t xbeg = g == 0 ? 0 : o, xend = g == 0 ? o : n;
    const int64_t rows_a = g == 0 ? oo : npair, ldc = g == 0 ? ovr : vvr;
    for (int64_t x0 = xbeg; x0 < xend; x0 += xc) {
      const int64_t nx = std::min<int64_t>(xc, xend - x0), rows = nx * v;
      box_copy(s_, stream_ac_.p(), {nx * v, v, 1}, M.Bnv.p() + x0 * v, {(int64_t)n * v, v, 1},
               {P, nx, v});
      es_.set_split(build, err_.as<int>(), 0.0);
      es_("Pxc,Pbd->xbcd", 1.0, T(stream_ac_.p(), {P, nx, v}), M.Bvv.t, 0.0,
          T(stream_gc_.p(), {nx, v, v, v}));
      es_.set_split(lev, err_.as<int>(), tc_min_flops_);
      double* C = (g == 0 ? Yov_.p() : Yvv_.p()) + (x0 - xbeg) * v;
      if (lev == 0) {
        k::gemm_f64(s_, false, true, rows_a, rows, vv, 1.0, g == 0 ? t2.p : tpair_.p(), vv, 0,
                    stream_gc_.p(), vv, 0, 0.0, C, ldc, 0, 1);
        continue;
      }
      const size_t bneed = sizeof(__nv_bfloat16) * (size_t)(planes * rows * Kp);
      if (stream_b_.bytes() < bneed) stream_b_.alloc(bneed, s_);
      auto* bp = stream_b_.as<__nv_bfloat16>();
      if (digits) {
        if (stream_be_.bytes() < sizeof(int32_t) * (size_t)rows)
          stream_be_.alloc(sizeof(int32_t) * (size_t)rows, s_);
        oz::split(s_, bp, stream_be_.as<int32_t>(), stream_gc_.p(), rows, vv, vv);
        auto* ws = static_cast<long long*>(es_.scratch(2, oz::ws_bytes(rows_a, rows)));
        oz::gemm(s_, rows_a, rows, vv, 1.0, g == 0 ? a_occ : a_vir, g == 0 ? e_occ : e_vir, 0, bp,
                 stream_be_.as<int32_t>(), 0, 0.0, C, ldc, ws, err_.as<int>(),
                 oz::splitk_for(rows_a, rows, vv));
      } else {
        tc::split_bf16(s_, bp, stream_gc_.p(), rows, vv, vv, lev);
        const int z = tc::splitk_for(rows_a, rows, vv);
        float* ws = z > 1 ? static_cast<float*>(
                                es_.scratch(2, sizeof(float) * (size_t)(z * rows_a * rows)))
                          : nullptr;
        tc::gemm_split(s_, rows_a, rows, vv, lev, 1.0, g == 0 ? a_occ : a_vir, bp, 0.0, C, ldc,
                       err_.as<int>(), z, ws);
      }
    }
  }
}

// Terms bilinear in T2 with intermediates built from (t, u = 2t - t^T) and
// contracted with t; added to Z (permuted part) and r2 with factor sign.
void State::quad_terms(const T& t, const T& u, const T& Z, const T& r2, double sign) {
  // hole-hole ladder, quadratic part: sum_kl t_kl^ab sum_cd t_ij^cd g_kcld
  es_("ijcd,kcld->klij", 1.0, t, govov_.t, 0.0, Wq_.t);
  es_("klab,klij->ijab", sign, t, Wq_.t, 1.0, r2);
  // crossed ring: X_kiac = -1/2 sum_ld t_li^ad g_kdlc
  es_("liad,kdlc->kiac", -0.5, t, govov_.t, 0.0, WC_.t);
  es_("kjbc,kiac->ijab", -0.5 * sign, t, WC_.t, 1.0, Z);
  es_("kibc,kjac->ijab", -1.0 * sign, t, WC_.t, 1.0, Z);
  // ring: Y_aikc = 1/2 sum_ld u_il^ad L_ldkc
  es_("ilad,ldkc->aikc", 0.5, u, Lovov_.t, 0.0, WD_.t);
  es_("jkbc,aikc->ijab", 0.5 * sign, u, WD_.t, 1.0, Z);
  // Fock-like: F'_bc = -sum u_kl^bd g_ldkc, F'_kj = sum u_lj^cd g_kdlc
  es_("klbd,ldkc->bc", -1.0, u, govov_.t, 0.0, Fvv_.t);
  es_("ljcd,kdlc->kj", 1.0, u, govov_.t, 0.0, Foo_.t);
  es_("ijac,bc->ijab", sign, t, Fvv_.t, 1.0, Z);
  foo_term(t, Foo_.p(), -sign, Z);
}

// Z_ijab += alpha sum_k t_ikab W_kj: an o x o matrix applied along the second
// index, in place (tensor-core tiles would be mostly padding at N = K = o).
// FP64 sums on the FP64 and FP64-class paths, FP32 sums at the split-BF16
// levels (at least as accurate as their products).
void State::foo_term(const T& t, const double* W, double alpha, const T& Z) {
  const int lev = es_.level();
  if (o_ <= 32) {
    k::axis_matrix(s_, lev >= 1 && lev <= 3, Z.p, t.p, W, o_, o_, o_, (int64_t)v_ * v_, alpha,
                   1.0);
  } else {
    es_("ikab,kj->ijab", alpha, t, T(const_cast<double*>(W), {o_, o_}), 1.0, Z);
  }
}

void State::residual(const double* tv, double* rv, double* energy) {
  const int o = o_, v = v_;
  const int64_t n1 = this->n1(), n2 = this->n2();
  T t1((double*)tv, {o, v}), t2((double*)tv + n1, {o, o, v, v});
  T r1(rv, {o, v}), r2(rv + n1, {o, o, v, v});
  dress(t1.p);
  k::tilde(s_, u_.p(), t2.p, o, v);
  const int n = n_;
  // ---- singles (alpha projection)
  box_copy(s_, r1.p, {v, 1}, F_.p() + (int64_t)o * n, {1, n}, {o, v});  // F_ai
  es_("Pkc,kicd->Pid", 1.0, Bov_.t, u_.t, 0.0, X_.t);
  es_("Pad,Pid->ia", 1.0, Bvv_.t, X_.t, 1.0, r1);                         // sum u g_adkc
  es_("klac,kilc->ia", -1.0, u_.t, gooov_.t, 1.0, r1);
  // contractions with the Fock matrix carry O(1) x O(t) products: FP64, or
  // the FP64-class digit-plane products on the tensor-core paths
  const int lev = es_.level();
  es_.set_split(lev ? 4 : 0, err_.as<int>(), tc_min_flops_);
  {
    OT Fov({o, v}, s_);
    box_copy(s_, Fov.p(), {v, 1}, F_.p() + o, {n, 1}, {o, v});
    es_("ikac,kc->ia", 1.0, u_.t, Fov.t, 1.0, r1);
  }
  es_.set_split(lev, err_.as<int>(), tc_min_flops_);
  // ---- doubles (alpha-beta projection)
  es_.perm("aibj->ijab", 1.0, gvovo_.t, 0.0, r2);
  ladder(t2, r2);
  es_("klab,kilj->ijab", 1.0, t2, goooo_.t, 1.0, r2);
  k::fill(s_, Z_.p(), 0.0, n2);
  es_("kjbc,kiac->ijab", -0.5, t2, goovv_.t, 1.0, Z_.t);
  es_("kibc,kjac->ijab", -1.0, t2, goovv_.t, 1.0, Z_.t);
  es_("jkbc,aikc->ijab", 0.5, u_.t, Lvoov_.t, 1.0, Z_.t);
  es_.set_split(lev ? 4 : 0, err_.as<int>(), tc_min_flops_);
  {
    OT Fvv({v, v}, s_), Foo({o, o}, s_);
    box_copy(s_, Fvv.p(), {v, 1}, F_.p() + (int64_t)o * n + o, {n, 1}, {v, v});
    box_copy(s_, Foo.p(), {o, 1}, F_.p(), {n, 1}, {o, o});
    es_("ijac,bc->ijab", 1.0, t2, Fvv.t, 1.0, Z_.t);
    foo_term(t2, Foo.p(), -1.0, Z_.t);
  }
  es_.set_split(lev, err_.as<int>(), tc_min_flops_);
  quad_terms(t2, u_.t, Z_.t, r2, 1.0);
  if (opt_.linearize) {
    // PLASCC (Sec. II.C): remove the terms bilinear in the mixed doubles
    k::mixed_mask(s_, m_.p(), t2.p, o, v, lh_, lp_);
    k::tilde(s_, um_.p(), m_.p(), o, v);
    quad_terms(m_.t, um_.t, Z_.t, r2, -1.0);
  }
  es_.perm("ijab->jiba", 1.0, Z_.t, 1.0, r2);
  k::axpby(s_, r2.p, Z_.p(), 1.0, 1.0, n2);
  if (n3() > 0) triples(t2, tv + n1 + n2, r1, r2, rv + n1 + n2);
  // ---- energy: <phi0|H-hat|phi0> + sum t_ij^ab L_iajb
  k::reference_energy(s_, scal_.p() + 8, hhat_.p(), n, goooo_.p(), o);
  {
    OT Lp({o, o, v, v}, s_);
    es_.perm("iajb->ijab", 1.0, Lovov_.t, 0.0, Lp.t);
    k::dot_rows(s_, t2.p, Lp.p(), 0, 1, n2, scal_.p() + 9, work_.p());
  }
  k::axpby(s_, energy, scal_.p() + 8, 1.0, 0.0, 1);
  k::axpby(s_, energy, scal_.p() + 9, 1.0, 1.0, 1);
}

double State::reference_energy() {
  OT z({n1()}, s_);
  k::fill(s_, z.p(), 0.0, n1());
  dress(z.p());
  k::reference_energy(s_, scal_.p() + 10, hhat_.p(), n_, goooo_.p(), o_);
  double e = 0.0;
  ASCC_CUDA(cudaMemcpyAsync(&e, scal_.p() + 10, sizeof(double), cudaMemcpyDeviceToHost, s_));
  ASCC_CUDA(cudaStreamSynchronize(s_));
  return e;
}

void State::reset() {
  const int64_t N = namp();
  std::vector<double> guess;
  initial_guess(guess);
  ASCC_CUDA(cudaMemcpyAsync(t_.p(), guess.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s_));
  const int m = opt_.diis_dim;
  k::fill(s_, hist_t_.p(), 0.0, (int64_t)m * N);
  k::fill(s_, hist_e_.p(), 0.0, (int64_t)m * N);
  slots_.clear();
  k::fill(s_, gram_.p(), 0.0, (int64_t)m * m);
  k::fill(s_, scal_.p(), 0.0, 64);
  next_slot_ = 0;
  iter_ = 0;
  iter_low_ = 0;
  best_r_ = 0.0;
  stall_n_ = 0;
  fp64_evals_ = 0;
  polish_ = false;
  need_refresh_ = false;
  have_corr_ = false;
  fallback_ = false;
  polish_its_ = 0;
  have_prev_ = false;
  done_ = false;
  status_ = ASCC_ERR_NOT_CONVERGED;
  ASCC_CUDA(cudaStreamSynchronize(s_));
}

// One pass per residual evaluation: residual, convergence test, Jacobi step,
// DIIS extrapolation (rules fixed in the oracle's solver docstring).
ascc_status State::iterate(int max_steps, ascc_result* res) {
  const int64_t N = namp();
  const int m = opt_.diis_dim;
  for (int step = 0; step < max_steps && !done_; ++step) {
    const int lev = level_for_phase();
    bool refreshed = false;
    if (lev == 3 && need_refresh_) {
      // polishing: the FP64-class residual (exact digit-plane products on the
      // tensor cores) and the 6-product residual at the same amplitudes; their
      // difference corrects the following iterations (defect correction), and
      // this step itself uses the FP64-class residual
      es_.set_split(4, err_.as<int>(), tc_min_flops_);
      residual(t_.p(), r_.p(), scal_.p());
      es_.set_split(3, err_.as<int>(), tc_min_flops_);
      residual(t_.p(), corr_.p(), scal_.p() + 2);
      k::axpby(s_, corr_.p(), r_.p(), 1.0, -1.0, N);            // corr = R64 - R3
      k::axpby(s_, scal_.p() + 3, scal_.p(), 1.0, 0.0, 1);
      k::axpby(s_, scal_.p() + 3, scal_.p() + 2, -1.0, 1.0, 1);  // E64 - E3
      need_refresh_ = false;
      have_corr_ = true;
      refreshed = true;
      ++fp64_evals_;
    } else {
      es_.set_split(lev, err_.as<int>(), tc_min_flops_);
      residual(t_.p(), r_.p(), scal_.p());
      if (lev == 3 && have_corr_) {
        k::axpby(s_, r_.p(), corr_.p(), 1.0, 1.0, N);
        k::axpby(s_, scal_.p(), scal_.p() + 3, 1.0, 1.0, 1);
      }
    }
    k::maxabs(s_, r_.p(), N, scal_.p() + 1, work_.p());
    // the one host readback of an iteration: E, max|R|, the DIIS failure flag
    // of the previous step and the device timeout code
    double h2[8];
    int kerr = 0;
    ASCC_CUDA(cudaMemcpyAsync(h2, scal_.p(), 8 * sizeof(double), cudaMemcpyDeviceToHost, s_));
    ASCC_CUDA(cudaMemcpyAsync(&kerr, err_.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, s_));
    ASCC_CUDA(cudaStreamSynchronize(s_));
    if (kerr != 0)
      throw Error(ASCC_ERR_TIMEOUT, "tensor-core GEMM wait timed out (code " +
                                        std::to_string(kerr) + ")");
    e_last_ = h2[0];
    r_last_ = h2[1];
    if (h2[6] != 0.0) {
      // the previous extrapolation failed: keep only the newest pair
      if (!slots_.empty()) slots_.assign(1, slots_.back());
      k::fill(s_, scal_.p() + 6, 0.0, 1);
    }
    const int it = iter_++;
    if (lev == 2) ++iter_low_;
    if (lev == 2 && std::isfinite(r_last_)) {
      bool hand = r_last_ <= opt_.polish_tol;
      if (!hand && ladder_digits_ && r_last_ <= 10.0 * opt_.polish_tol) {
        // a state that polishes with FP64-class steps (ladder as digit planes
        // only) whose low-precision noise floor lies above polish_tol: hand
        // over once max|R| has not halved for 8 steps
        if (best_r_ == 0.0 || r_last_ < 0.5 * best_r_) {
          best_r_ = r_last_;
          stall_n_ = 0;
        } else if (++stall_n_ >= 8) {
          hand = true;
        }
      }
      if (hand) {
        // hand over to the polishing precision and re-evaluate (with an
        // FP64-class correction) before testing convergence.  The DIIS history
        // is kept: its error vectors carry the coarser residual but age out
        // within diis_dim steps, and slowly converging states need the long
        // history.  A state with the ladder as digit planes only polishes with
        // FP64-class residuals throughout (no 6-product phase).
        polish_ = true;
        need_refresh_ = true;
        have_prev_ = false;
        best_r_ = 0.0;
        stall_n_ = 0;
        if (ladder_digits_) fallback_ = true;
      }
    }
    if (!std::isfinite(e_last_) || !std::isfinite(r_last_)) {
      status_ = ASCC_ERR_DIVERGED;
      done_ = true;
      break;
    }
    if (have_prev_ && r_last_ <= opt_.r_tol && std::fabs(e_last_ - e_prev_) <= opt_.e_tol) {
      if (lev == 3 && !refreshed) {
        // converged on the corrected residual: confirm with a fresh FP64 one
        need_refresh_ = true;
        continue;
      }
      status_ = ASCC_OK;
      done_ = true;
      break;
    }
    if (lev == 3 && ++polish_its_ >= 30 + opt_.diis_dim) {
      // the corrected iteration stalls (slowly converging states): continue with
      // FP64-class residuals in every step; the history of corrected residuals
      // is kept (they are FP64-class up to the drift of the correction)
      fallback_ = true;
    }
    if (it >= opt_.max_iter) {
      status_ = ASCC_ERR_NOT_CONVERGED;
      done_ = true;
      break;
    }
    e_prev_ = e_last_;
    have_prev_ = true;
    int slot;
    if ((int)slots_.size() < m) {
      slot = next_slot_++;
    } else {
      slot = slots_.front();
      slots_.erase(slots_.begin());
    }
    slots_.push_back(slot);
    double* tn = hist_t_.p() + (int64_t)slot * N;
    double* en = hist_e_.p() + (int64_t)slot * N;
    k::jacobi(s_, tn, en, t_.p(), r_.p(), mol_->eps.p(), eps_eff_.p(), o_, v_, hole_, particle_,
              n3() ? t3idx_.as<int32_t>() : nullptr, n3());
    k::jacobi_pairs(s_, tn, en, t_.p(), r_.p(), eps_eff_.p(), F_.p(), o_, v_, hole_, particle_);
    k::dot_rows(s_, en, hist_e_.p(), N, m, N, scal_.p() + 32, work_.p());
    // Gram row, bordered solve and extrapolation stay on the device; a failed
    // solve leaves t = tn and is seen at the next readback
    k::DiisArgs da{};
    da.m = m;
    da.cnt = (int)slots_.size();
    da.solve = da.cnt >= opt_.diis_start;
    for (int q = 0; q < da.cnt; ++q) da.slot[q] = slots_[q];
    k::diis(s_, gram_.p(), scal_.p() + 32, da, coef_.p(), scal_.p() + 6);
    if (da.solve)
      k::lincomb(s_, t_.p(), hist_t_.p(), N, coef_.p(), m, N);
    else
      k::axpby(s_, t_.p(), tn, 1.0, 0.0, N);
  }
  if (res) {
    res->energy = e_last_;
    res->max_resid = r_last_;
    res->iterations = iter_;
    res->status = done_ ? status_ : ASCC_ERR_NOT_CONVERGED;
    res->iterations_low = iter_low_;
    res->fp64_evaluations = fp64_evals_;
    res->e_ref = 0.0;
  }
  return done_ ? status_ : ASCC_ERR_NOT_CONVERGED;
}

namespace {
constexpr int64_t kCkptMagic = 0x5450434b43435341LL;  // "ASCCKCPT"
constexpr int kCkptHeader = 24;
}  // namespace

int64_t State::checkpoint_bytes() const {
  const int64_t N = namp(), m = opt_.diis_dim, cnt = (int64_t)slots_.size();
  int64_t words = kCkptHeader + cnt + 3 + 8 + m * m + N + 2 * cnt * N;
  if (opt_.precision == ASCC_MIXED_BF16) words += N;
  return 8 * words;
}

void State::checkpoint_save(void* buf, int64_t bytes) {
  ASCC_REQUIRE(buf && bytes >= checkpoint_bytes(), "checkpoint buffer too small");
  const int64_t N = namp(), m = opt_.diis_dim, cnt = (int64_t)slots_.size();
  auto* w = static_cast<int64_t*>(buf);
  const int64_t flags = (int64_t)have_prev_ | (int64_t)done_ << 1 | (int64_t)polish_ << 2 |
                        (int64_t)need_refresh_ << 3 | (int64_t)have_corr_ << 4 |
                        (int64_t)fallback_ << 5;
  const int64_t head[kCkptHeader] = {kCkptMagic, 1, o_, v_, n3(), opt_.precision, opt_.linearize,
                                     m, cnt, next_slot_, iter_, iter_low_, fp64_evals_,
                                     polish_its_, flags, (int64_t)status_, hole_, particle_,
                                     lh_, lp_, (int64_t)(xsign_ < 0), stall_n_, 0, 0};
  int64_t best_bits;
  std::memcpy(&best_bits, &best_r_, sizeof(best_bits));
  std::memcpy(w, head, sizeof(head));
  w[23] = best_bits;
  for (int64_t q = 0; q < cnt; ++q) w[kCkptHeader + q] = slots_[q];
  auto* d = reinterpret_cast<double*>(w + kCkptHeader + cnt);
  d[0] = e_prev_;
  d[1] = e_last_;
  d[2] = r_last_;
  d += 3;
  ASCC_CUDA(cudaMemcpyAsync(d, scal_.p(), 8 * sizeof(double), cudaMemcpyDeviceToHost, s_));
  d += 8;
  ASCC_CUDA(cudaMemcpyAsync(d, gram_.p(), sizeof(double) * m * m, cudaMemcpyDeviceToHost, s_));
  d += m * m;
  ASCC_CUDA(cudaMemcpyAsync(d, t_.p(), sizeof(double) * N, cudaMemcpyDeviceToHost, s_));
  d += N;
  for (int64_t q = 0; q < cnt; ++q) {
    const int64_t sl = slots_[q];
    ASCC_CUDA(cudaMemcpyAsync(d, hist_t_.p() + sl * N, sizeof(double) * N, cudaMemcpyDeviceToHost,
                              s_));
    d += N;
    ASCC_CUDA(cudaMemcpyAsync(d, hist_e_.p() + sl * N, sizeof(double) * N, cudaMemcpyDeviceToHost,
                              s_));
    d += N;
  }
  if (opt_.precision == ASCC_MIXED_BF16)
    ASCC_CUDA(cudaMemcpyAsync(d, corr_.p(), sizeof(double) * N, cudaMemcpyDeviceToHost, s_));
  ASCC_CUDA(cudaStreamSynchronize(s_));
}

void State::checkpoint_load(const void* buf, int64_t bytes) {
  ASCC_REQUIRE(buf && bytes >= 8 * kCkptHeader, "checkpoint buffer too small");
  const auto* w = static_cast<const int64_t*>(buf);
  const int64_t N = namp(), m = opt_.diis_dim, cnt = w[8];
  ASCC_REQUIRE(w[0] == kCkptMagic && w[1] == 1, "not a checkpoint of this library");
  ASCC_REQUIRE(w[2] == o_ && w[3] == v_ && w[4] == n3() && w[5] == opt_.precision &&
                   w[6] == opt_.linearize && w[7] == m && w[16] == hole_ &&
                   w[17] == particle_ && w[18] == lh_ && w[19] == lp_ &&
                   w[20] == (int64_t)(xsign_ < 0),
               "checkpoint of a different state or options");
  ASCC_REQUIRE(cnt >= 0 && cnt <= m, "checkpoint: bad DIIS history length");
  int64_t words = kCkptHeader + cnt + 3 + 8 + m * m + N + 2 * cnt * N;
  if (opt_.precision == ASCC_MIXED_BF16) words += N;
  ASCC_REQUIRE(bytes >= 8 * words, "checkpoint buffer too small");
  slots_.clear();
  for (int64_t q = 0; q < cnt; ++q) {
    const int64_t sl = w[kCkptHeader + q];
    ASCC_REQUIRE(sl >= 0 && sl < m, "checkpoint: bad DIIS slot");
    slots_.push_back((int)sl);
  }
  next_slot_ = (int)w[9];
  iter_ = (int)w[10];
  iter_low_ = (int)w[11];
  fp64_evals_ = (int)w[12];
  polish_its_ = (int)w[13];
  const int64_t flags = w[14];
  have_prev_ = flags & 1;
  done_ = (flags >> 1) & 1;
  polish_ = (flags >> 2) & 1;
  need_refresh_ = (flags >> 3) & 1;
  have_corr_ = (flags >> 4) & 1;
  fallback_ = (flags >> 5) & 1;
  status_ = (ascc_status)w[15];
  stall_n_ = (int)w[21];
  std::memcpy(&best_r_, &w[23], sizeof(best_r_));
  const auto* d = reinterpret_cast<const double*>(w + kCkptHeader + cnt);
  e_prev_ = d[0];
  e_last_ = d[1];
  r_last_ = d[2];
  d += 3;
  ASCC_CUDA(cudaMemcpyAsync(scal_.p(), d, 8 * sizeof(double), cudaMemcpyHostToDevice, s_));
  d += 8;
  ASCC_CUDA(cudaMemcpyAsync(gram_.p(), d, sizeof(double) * m * m, cudaMemcpyHostToDevice, s_));
  d += m * m;
  ASCC_CUDA(cudaMemcpyAsync(t_.p(), d, sizeof(double) * N, cudaMemcpyHostToDevice, s_));
  d += N;
  for (int64_t q = 0; q < cnt; ++q) {
    const int64_t sl = slots_[q];
    ASCC_CUDA(cudaMemcpyAsync(hist_t_.p() + sl * N, d, sizeof(double) * N, cudaMemcpyHostToDevice,
                              s_));
    d += N;
    ASCC_CUDA(cudaMemcpyAsync(hist_e_.p() + sl * N, d, sizeof(double) * N, cudaMemcpyHostToDevice,
                              s_));
    d += N;
  }
  if (opt_.precision == ASCC_MIXED_BF16)
    ASCC_CUDA(cudaMemcpyAsync(corr_.p(), d, sizeof(double) * N, cudaMemcpyHostToDevice, s_));
  ASCC_CUDA(cudaStreamSynchronize(s_));
}

ascc_status State::solve(ascc_result* res) {
  reset();
  return iterate(opt_.max_iter + 1, res);
}

void State::profile(double* ladder_ms, int64_t* ladder_launches, double* ladder_flops,
                    double* ladder_mma_flops) {
  for (auto& ev : events_) {
    ASCC_CUDA(cudaEventSynchronize(ev.second));
    float ms = 0.f;
    ASCC_CUDA(cudaEventElapsedTime(&ms, ev.first, ev.second));
    ladder_ms_ += ms;
    cudaEventDestroy(ev.first);
    cudaEventDestroy(ev.second);
  }
  events_.clear();
  if (ladder_ms) *ladder_ms = ladder_ms_;
  if (ladder_launches) *ladder_launches = ladder_launches_;
  if (ladder_flops) *ladder_flops = ladder_flops_;
  if (ladder_mma_flops) *ladder_mma_flops = ladder_mma_flops_;
}

}  // namespace ascc
