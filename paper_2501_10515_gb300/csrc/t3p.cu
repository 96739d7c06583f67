// Executor of the generated T3' program (see t3p.h) and the kernels that move
// the packed slice into its dense blocks and back.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "kernels.h"
#include "t3p.h"

namespace ascc {

namespace {
#include "t3p_program.inc"

int64_t round_up(int64_t x, int64_t q) { return (x + q - 1) / q * q; }

std::vector<int64_t> rm_strides(const std::vector<int64_t>& shape) {
  std::vector<int64_t> st(shape.size());
  int64_t acc = 1;
  for (int d = (int)shape.size() - 1; d >= 0; --d) {
    st[d] = acc;
    acc *= shape[d];
  }
  return st;
}
}  // namespace

T3pProgram::T3pProgram(int o, int v, int naux, int h, int p, int nstreams)
    : o_(o), v_(v), n_(o + v), naux_(naux), h_(h), p_(p), nstreams_(std::max(1, nstreams)) {
  profile_path_ = std::getenv("ASCC_T3P_PROFILE");
  blk_off_[0] = 0;
  blk_off_[1] = (int64_t)o * v * v;
  blk_off_[2] = blk_off_[1] + (int64_t)o * v * v;
  blk_off_[3] = blk_off_[2] + (int64_t)o * o * v;
  blk_off_[4] = blk_off_[3] + (int64_t)o * o * v;
  auto extent = [&](char c) -> int64_t {
    return c == 'o' ? o : c == 'v' ? v : c == 'P' ? naux : (int64_t)(o + v);
  };
  shape_.resize(kT3pTensorCount);
  for (int t = 0; t < kT3pTensorCount; ++t)
    for (const char* c = kT3pTensors[t].dims; *c; ++c)
      shape_[t].push_back(*c == '#' ? stack_rows(kT3pTensors[t].rows, 1 << 30) : extent(*c));
  // lifetimes over the run order (pro, lin, quad, mix; quad may run twice on
  // the same allocation), then first-fit placement
  std::vector<int> def(kT3pTensorCount, -1), last(kT3pTensorCount, -1);
  int64_t acc_max = 1;
  for (int q = 0; q < kT3pOpCount; ++q) {
    const T3pOp& op = kT3pOps[q];
    if (op.out >= 0 && def[op.out] < 0) def[op.out] = q;
    if (op.a >= 0) last[op.a] = q;
    if (op.b >= 0) last[op.b] = q;
    if (op.kind == 2) {
      int64_t e = 1;
      for (const char* c = op.outspec; *c; ++c)
        if (*c == 'o' || *c == 'v') e *= extent(*c);
      acc_max = std::max(acc_max, e);
    }
  }
  // the quad section runs twice under partial linearisation: whatever it reads
  // from earlier sections must outlive its last op
  int quad_end = -1;
  for (int q = 0; q < kT3pOpCount; ++q)
    if (kT3pOps[q].section == T3P_QUAD) quad_end = q;
  for (int q = 0; q < kT3pOpCount; ++q) {
    const T3pOp& op = kT3pOps[q];
    if (op.section != T3P_QUAD) continue;
    for (int t : {op.a, op.b})
      if (t >= 0 && kT3pTensors[t].section != T3P_QUAD) last[t] = std::max(last[t], quad_end);
  }
  // on several streams an op may run while ops before it still do: memory is
  // not handed on before a window of later ops has been issued (the stream
  // plan then adds the waits for what is still shared)
  const int window = nstreams_ > 1 ? 48 : 0;
  struct Slot { int64_t off, size; int s, e; };
  std::vector<Slot> placed;
  std::vector<int> order;
  for (int t = 0; t < kT3pTensorCount; ++t)
    if (kT3pTensors[t].kind != 0 && def[t] >= 0) order.push_back(t);
  std::sort(order.begin(), order.end(), [&](int a, int b) { return def[a] < def[b]; });
  offset_.assign(kT3pTensorCount, -1);
  int64_t peak = 0;
  for (int t : order) {
    int64_t sz = 1;
    for (auto d : shape_[t]) sz *= d;
    sz = round_up(std::max<int64_t>(sz, 1), 32);
    const int s = def[t], e = std::max(last[t], def[t]) + window;
    std::vector<std::pair<int64_t, int64_t>> live;
    for (const Slot& sl : placed)
      if (!(sl.e < s || sl.s > e)) live.push_back({sl.off, sl.size});
    std::sort(live.begin(), live.end());
    int64_t off = 0;
    for (auto& lv : live) {
      if (off + sz <= lv.first) break;
      off = std::max(off, lv.first + lv.second);
    }
    placed.push_back({off, sz, s, e});
    offset_[t] = off;
    peak = std::max(peak, off + sz);
  }
  acc_off_ = round_up(peak, 32);
  acc_len_ = round_up(acc_max, 32);
  ws_elems_ = acc_off_ + acc_len_ * nstreams_;
  if (nstreams_ > 1) plan_streams();
}

int T3pProgram::op_count() const { return kT3pOpCount; }

// Race check of the stream plan, from memory footprints alone (independent
// of how plan_streams derives its dependencies): two ops of a section
// conflict when one writes workspace memory the other reads or writes, or
// both accumulate into R1 or R2 (RA..RD and the temporaries are per stream).
// Each conflict must be ordered by stream order or by the event waits:
// vector clocks over the streams record, for every op, the latest op of each
// stream known to be complete when it starts.
// Placement check, from the op table alone (independent of the constructor's
// liveness): the sections run as pro, lin, quad, quad (the second run for
// PLASCC), mix; a tensor is live from a write to its last read before its next
// write (writes with no read between them, the rows of a stack, extend one
// interval); two tensors whose workspace ranges overlap must never be live at
// once.  collapse: every tensor placed at offset 0 (a test of the check).
int64_t T3pProgram::placement_clobbers(bool collapse) const {
  const int T = kT3pTensorCount;
  std::vector<int> seq;
  for (int sec : {T3P_PRO, T3P_LIN, T3P_QUAD, T3P_QUAD, T3P_MIX})
    for (int q = 0; q < kT3pOpCount; ++q)
      if (kT3pOps[q].section == sec) seq.push_back(q);
  struct Iv { int b, e; };
  std::vector<std::vector<Iv>> iv(T);
  std::vector<bool> read_since(T, true);
  for (int pos = 0; pos < (int)seq.size(); ++pos) {
    const T3pOp& op = kT3pOps[seq[pos]];
    for (int t : {op.a, op.b})
      if (t >= 0 && offset_[t] >= 0 && !iv[t].empty()) {
        iv[t].back().e = pos;
        read_since[t] = true;
      }
    if (op.out >= 0 && offset_[op.out] >= 0) {
      const int t = op.out;
      if (iv[t].empty() || read_since[t])
        iv[t].push_back({pos, pos});
      else
        iv[t].back().e = pos;
      read_since[t] = false;
    }
  }
  auto size_of = [&](int t) {
    int64_t e = 1;
    for (auto d : shape_[t]) e *= d;
    return std::max<int64_t>(e, 1);
  };
  int64_t clobbers = 0;
  for (int x = 0; x < T; ++x) {
    if (offset_[x] < 0 || iv[x].empty()) continue;
    const int64_t xb = collapse ? 0 : offset_[x], xe = xb + size_of(x);
    for (int y = x + 1; y < T; ++y) {
      if (offset_[y] < 0 || iv[y].empty()) continue;
      const int64_t yb = collapse ? 0 : offset_[y], ye = yb + size_of(y);
      if (!(xb < ye && yb < xe)) continue;
      bool clash = false;
      for (const Iv& a : iv[x]) {
        for (const Iv& b : iv[y])
          if (a.b <= b.e && b.b <= a.e) {
            clash = true;
            break;
          }
        if (clash) break;
      }
      if (clash) ++clobbers;
    }
  }
  return clobbers;
}

int64_t T3pProgram::plan_hazards(bool drop_waits) const {
  const int Q = kT3pOpCount, ns = nstreams_;
  if (ns <= 1 || op_stream_.empty()) return 0;
  auto size_of = [&](int t) {
    int64_t e = 1;
    for (auto d : shape_[t]) e *= d;
    return std::max<int64_t>(e, 1);
  };
  struct Fp { int64_t b, e; bool w; };
  std::vector<std::vector<Fp>> fp(Q);
  std::vector<int> r12(Q, -1);
  for (int q = 0; q < Q; ++q) {
    const T3pOp& op = kT3pOps[q];
    if (op.out >= 0 && offset_[op.out] >= 0)
      fp[q].push_back({offset_[op.out], offset_[op.out] + size_of(op.out), true});
    for (int t : {op.a, op.b})
      if (t >= 0 && offset_[t] >= 0) fp[q].push_back({offset_[t], offset_[t] + size_of(t), false});
    if ((op.kind == 2 || (op.kind == 4 && op.out < 0)) && (op.base == T3P_R1 || op.base == T3P_R2))
      r12[q] = op.base;
  }
  std::vector<std::vector<int>> vc(Q, std::vector<int>(ns, -1));
  std::vector<int> last(ns, -1);
  int section = -1;
  int64_t hazards = 0;
  std::vector<int> members;
  for (int q = 0; q < Q; ++q) {
    const T3pOp& op = kT3pOps[q];
    if (op.section != section) {
      section = op.section;
      std::fill(last.begin(), last.end(), -1);
      members.clear();
    }
    const int st = op_stream_[q];
    std::vector<int>& c = vc[q];
    if (last[st] >= 0) c = vc[last[st]];
    if (!drop_waits)
      for (int d : deps_[q])
        if (kT3pOps[d].section == section)
          for (int k = 0; k < ns; ++k) c[k] = std::max(c[k], vc[d][k]);
    c[st] = q;
    for (int p : members) {
      const int sp = op_stream_[p];
      if (sp == st || c[sp] >= p) continue;  // ordered
      bool clash = r12[p] >= 0 && r12[p] == r12[q];
      for (const Fp& x : fp[p]) {
        if (clash) break;
        for (const Fp& y : fp[q])
          if ((x.w || y.w) && x.b < y.e && y.b < x.e) {
            clash = true;
            break;
          }
      }
      if (clash) ++hazards;
    }
    members.push_back(q);
    last[st] = q;
  }
  return hazards;
}

int t3p_streams() {
  if (const char* env = std::getenv("ASCC_T3P_STREAMS")) {
    const int n = std::atoi(env);
    return std::min(std::max(n, 1), 16);
  }
  return 6;
}

// Stream plan: dependencies of every op (writers of what it reads; earlier
// users of any workspace range it writes), then a list schedule in program
// order on estimated op times, each op on the stream where it can start
// first; accumulations into R1 / R2 stay on stream 0.
void T3pProgram::plan_streams() {
  const int T = kT3pTensorCount, Q = kT3pOpCount;
  std::vector<int64_t> size(T, 0);
  for (int t = 0; t < T; ++t) {
    int64_t e = 1;
    for (auto d : shape_[t]) e *= d;
    size[t] = e;
  }
  std::vector<std::vector<int>> writers(T), users(T);
  for (int q = 0; q < Q; ++q) {
    const T3pOp& op = kT3pOps[q];
    if (op.out >= 0) {
      writers[op.out].push_back(q);
      users[op.out].push_back(q);
    }
    if (op.a >= 0) users[op.a].push_back(q);
    if (op.b >= 0) users[op.b].push_back(q);
  }
  // tensors whose workspace ranges overlap
  std::vector<std::vector<int>> overlap(T);
  for (int t = 0; t < T; ++t) {
    if (offset_[t] < 0) continue;
    const int64_t a0 = offset_[t], a1 = offset_[t] + std::max<int64_t>(size[t], 1);
    for (int u = 0; u < T; ++u) {
      if (u == t || offset_[u] < 0) continue;
      const int64_t b0 = offset_[u], b1 = offset_[u] + std::max<int64_t>(size[u], 1);
      if (a0 < b1 && b0 < a1) overlap[t].push_back(u);
    }
  }
  std::vector<std::vector<int>> full(Q);
  for (int q = 0; q < Q; ++q) {
    const T3pOp& op = kT3pOps[q];
    auto add = [&](int d) {
      if (d < q && kT3pOps[d].section == op.section) full[q].push_back(d);
    };
    for (int t : {op.a, op.b})
      if (t >= 0)
        for (int w : writers[t]) add(w);
    if (op.out >= 0) {
      for (int u : users[op.out])
        if (u < q && kT3pOps[u].kind == 3) add(u);  // earlier rows of a stack
      for (int y : overlap[op.out])
        for (int u : users[y]) add(u);
    }
  }
  // estimated time of an op (s): launch gaps plus data movement plus flops
  auto cost = [&](int q) {
    const T3pOp& op = kT3pOps[q];
    double bytes = 0.0, flops = 0.0;
    for (int t : {op.a, op.b, op.out})
      if (t >= 0) bytes += 8.0 * (double)size[t];
    if (op.kind == 1 || op.kind == 2) {
      double f = 2.0;
      const std::string sp(op.spec);
      std::string seen;
      const auto arrow = sp.find("->");
      const auto comma = sp.find(',');
      const std::string la = sp.substr(0, comma), lb = sp.substr(comma + 1, arrow - comma - 1);
      for (int side = 0; side < 2; ++side) {
        const std::string& l = side ? lb : la;
        const int t = side ? op.b : op.a;
        const std::vector<int64_t> sh = kT3pTensors[t].kind == 0
                                            ? base_shape(kT3pTensors[t].base)
                                            : shape_[t];
        for (size_t d = 0; d < l.size() && d < sh.size(); ++d)
          if (seen.find(l[d]) == std::string::npos) {
            seen += l[d];
            f *= (double)sh[d];
          }
      }
      flops = f;
    }
    return 6e-6 + bytes / 3e12 + flops / 2e14;
  };
  op_stream_.assign(Q, 0);
  deps_.assign(Q, {});
  std::vector<double> finish(Q, 0.0), ready(nstreams_, 0.0);
  int section = -1;
  for (int q = 0; q < Q; ++q) {
    const T3pOp& op = kT3pOps[q];
    if (op.section != section) {
      section = op.section;
      std::fill(ready.begin(), ready.end(), 0.0);
    }
    double est = 0.0;
    for (int d : full[q]) est = std::max(est, finish[d]);
    const bool to_r12 = (op.kind == 2 || (op.kind == 4 && op.out < 0)) &&
                        (op.base == T3P_R1 || op.base == T3P_R2);
    int best = 0;
    if (!to_r12) {
      double bt = 1e300;
      for (int k = 0; k < nstreams_; ++k) {
        const double t0 = std::max(est, ready[k]);
        if (t0 < bt - 1e-12) {
          bt = t0;
          best = k;
        }
      }
    }
    op_stream_[q] = best;
    finish[q] = std::max(est, ready[best]) + cost(q);
    ready[best] = finish[q];
    // keep the latest dependency on each other stream
    std::vector<int> latest(nstreams_, -1);
    for (int d : full[q])
      if (op_stream_[d] != best) latest[op_stream_[d]] = std::max(latest[op_stream_[d]], d);
    for (int k = 0; k < nstreams_; ++k)
      if (latest[k] >= 0) deps_[q].push_back(latest[k]);
  }
}

int64_t T3pProgram::dims_extent(const char* dims) const {
  int64_t e = 1;
  for (const char* c = dims; *c && *c != '+'; ++c)
    e *= *c == 'o' ? o_ : *c == 'v' ? v_ : *c == 'P' ? naux_ : (int64_t)n_;
  return e;
}

int64_t T3pProgram::stack_rows(const char* rows, int upto) const {
  int64_t r = 0;
  int m = 0;
  const char* c = rows;
  while (m < upto) {
    r += dims_extent(c);
    ++m;
    while (*c && *c != '+') ++c;
    if (!*c) break;
    ++c;
  }
  return r;
}

std::vector<int64_t> T3pProgram::base_shape(int b) const {
  switch (b) {
    case T3P_F: return {n_, n_};
    case T3P_B: return {naux_, n_, n_};
    case T3P_T2: case T3P_TS: case T3P_R2: return {o_, o_, v_, v_};
    case T3P_TA: case T3P_TB: case T3P_RA: case T3P_RB: return {o_, v_, v_};
    case T3P_TC: case T3P_TD: case T3P_RC: case T3P_RD: return {o_, o_, v_};
    case T3P_R1: return {o_, v_};
  }
  throw Error(ASCC_ERR_INVALID, "T3' program: unknown base operand");
}

// Offset, extents and strides of the box of base operand b that a selector
// picks: 'h' / 'p' fix a dimension at the primary hole / particle, 'o' / 'v'
// take the occupied / virtual range of an all-orbital dimension (or the whole
// dimension of an occupied / virtual one), 'P' the whole DF dimension.
void T3pProgram::select(int b, const char* spec, int64_t* offset, std::vector<int64_t>& shape,
                        std::vector<int64_t>& stride) const {
  const std::vector<int64_t> bs = base_shape(b);
  ASCC_REQUIRE(std::strlen(spec) == bs.size(), "T3' program: selector rank");
  std::vector<int64_t> st(bs.size());
  int64_t acc = 1;
  for (int d = (int)bs.size() - 1; d >= 0; --d) {
    st[d] = acc;
    acc *= bs[d];
  }
  *offset = 0;
  shape.clear();
  stride.clear();
  for (size_t d = 0; d < bs.size(); ++d) {
    const bool all = b == T3P_F || (b == T3P_B && d > 0);  // dimensions over all orbitals
    const char c = spec[d];
    if (c == 'h') {
      *offset += h_ * st[d];
    } else if (c == 'p') {
      *offset += ((all ? o_ : 0) + p_) * st[d];
    } else if (c == 'o') {
      shape.push_back(o_);
      stride.push_back(st[d]);
    } else if (c == 'v') {
      *offset += (all ? o_ : 0) * st[d];
      shape.push_back(v_);
      stride.push_back(st[d]);
    } else {
      shape.push_back(bs[d]);
      stride.push_back(st[d]);
    }
  }
}

// Contractions of at least this many flops run on the tensor cores when the
// state uses them: most of the program's products are small (an o x v x v
// block against a v x v one), and the FP64 units would serialise them.
// (ASCC_T3P_TC_MIN_FLOPS overrides it.)
// Split-K work-item target of the program's products (ASCC_T3P_SPLITK_FILL
// overrides it): the sections run on several streams, whose launches fill
// the SMs that a product leaves.
int t3p_fill() {
  static const int v = [] {
    const char* env = std::getenv("ASCC_T3P_SPLITK_FILL");
    return env ? std::atoi(env) : 76;
  }();
  return v;
}

double tc_min_flops() {
  static const double v = [] {
    const char* env = std::getenv("ASCC_T3P_TC_MIN_FLOPS");
    return env ? std::atof(env) : 1e6;
  }();
  return v;
}

// One op.  base: the operands; outb: where accumulations into the output
// blocks go (the outputs themselves, or a stream's private copies); tmp: room
// for a product that lands in a slice of an output.
void T3pProgram::exec_op(int q, Einsum& es, cudaStream_t s, double* const* base,
                         double* const* outb, double scale, double* ws, double* tmp) const {
  const T3pOp& op = kT3pOps[q];
  auto tensor = [&](int t) -> T {
    const T3pTensor& d = kT3pTensors[t];
    if (d.kind == 0) return T(base[d.base], base_shape(d.base));
    return T(ws + offset_[t], shape_[t]);
  };
  auto pack = [](std::vector<int64_t>& shape, std::vector<int64_t>& a, std::vector<int64_t>& b) {
    if (shape.empty()) {
      shape = {1};
      a = {1};
      b = {1};
    }
  };
  if (op.kind == 0) {
    int64_t off;
    std::vector<int64_t> shape, stride;
    select(op.base, kT3pTensors[op.out].spec, &off, shape, stride);
    std::vector<int64_t> ost = rm_strides(shape);
    pack(shape, stride, ost);
    box_copy(s, ws + offset_[op.out], ost, base[op.base] + off, stride, shape);
  } else if (op.kind == 1) {
    es.set_keys(op.a, op.b);
    es(op.spec, op.alpha, tensor(op.a), tensor(op.b), 0.0, tensor(op.out));
  } else if (op.kind == 3 || op.kind == 4) {
    stack_copy(op, s, base, outb, scale, ws);
  } else {
    int64_t off;
    std::vector<int64_t> shape, stride;
    select(op.base, op.outspec, &off, shape, stride);
    es.set_keys(op.a, op.b);
    if (off == 0 && shape == base_shape(op.base)) {
      es(op.spec, op.alpha * scale, tensor(op.a), tensor(op.b), 1.0, T(outb[op.base], shape));
      return;
    }
    es(op.spec, op.alpha * scale, tensor(op.a), tensor(op.b), 0.0, T(tmp, shape));
    std::vector<int64_t> ost = rm_strides(shape);
    pack(shape, stride, ost);
    box_copy(s, outb[op.base] + off, stride, tmp, ost, shape, 1.0, 1.0);
  }
}

void T3pProgram::run(Einsum& es, cudaStream_t s, int section, double* const* base,
                     double scale, double* ws) const {
  const double min0 = es.min_flops();
  if (es.level() > 0) es.set_split(es.level(), es.err(), std::min(min0, tc_min_flops()));
  // every tensor of a section is written once before it is read, so its
  // planes stay valid for the rest of the section
  es.cache_reset(cache_bytes());
  const int fill0 = es.fill();
  es.set_fill(t3p_fill());
  // optional per-op timing (ASCC_T3P_PROFILE=<file>): CUDA events around
  // every op, summed per op and written to the file when the program is freed
  const bool prof = profile_path_ != nullptr;
  if (prof && prof_ev_.empty()) {
    prof_ev_.resize(2 * kT3pOpCount);
    for (auto& e : prof_ev_) ASCC_CUDA(cudaEventCreate(&e));
    prof_ms_.assign(kT3pOpCount, 0.0);
    prof_n_.assign(kT3pOpCount, 0);
  }
  for (int q = 0; q < kT3pOpCount; ++q) {
    if (kT3pOps[q].section != section) continue;
    if (prof) ASCC_CUDA(cudaEventRecord(prof_ev_[2 * q], s));
    exec_op(q, es, s, base, base, scale, ws, ws + acc_off_);
    if (prof) ASCC_CUDA(cudaEventRecord(prof_ev_[2 * q + 1], s));
  }
  es.set_split(es.level(), es.err(), min0);
  es.set_fill(fill0);
  if (prof) {
    ASCC_CUDA(cudaStreamSynchronize(s));
    for (int q = 0; q < kT3pOpCount; ++q) {
      if (kT3pOps[q].section != section) continue;
      float ms = 0.f;
      ASCC_CUDA(cudaEventElapsedTime(&ms, prof_ev_[2 * q], prof_ev_[2 * q + 1]));
      prof_ms_[q] += ms;
      prof_n_[q] += 1;
    }
  }
}

// The same section spread over the streams of `ex` (ex.streams[0] is the
// caller's stream): each op on its planned stream after the ops it depends
// on (producers of its operands, earlier users of the memory it writes);
// accumulations into RA..RD go to the stream's private copies, summed into
// the outputs in stream order at the end; R1 / R2 accumulate on stream 0.
void T3pProgram::run_streams(T3pStreams& ex, int section, double* const* base, double scale,
                             double* ws) const {
  const int ns = (int)ex.streams.size();
  cudaStream_t s0 = ex.streams[0];
  const int64_t nb = block_elements();
  k::fill(s0, ex.priv, 0.0, nb * ns);
  ASCC_CUDA(cudaEventRecord(ex.fork, s0));
  for (int k = 1; k < ns; ++k) ASCC_CUDA(cudaStreamWaitEvent(ex.streams[k], ex.fork, 0));
  std::vector<double> min0(ns);
  for (int k = 0; k < ns; ++k) {
    Einsum& e = *ex.es[k];
    min0[k] = e.min_flops();
    if (e.level() > 0) e.set_split(e.level(), e.err(), std::min(min0[k], tc_min_flops()));
    e.cache_reset(cache_bytes());
    e.set_fill(t3p_fill());
  }
  std::vector<double*> outb(T3P_NBASE * ns);
  for (int k = 0; k < ns; ++k) {
    for (int b = 0; b < T3P_NBASE; ++b) outb[k * T3P_NBASE + b] = base[b];
    for (int b = 0; b < 4; ++b) outb[k * T3P_NBASE + T3P_RA + b] = ex.priv + k * nb + blk_off_[b];
  }
  for (int q = 0; q < kT3pOpCount; ++q) {
    if (kT3pOps[q].section != section) continue;
    const int st = op_stream_[q] % ns;
    cudaStream_t s = ex.streams[st];
    for (int d : deps_[q])
      if (kT3pOps[d].section == section && op_stream_[d] % ns != st)
        ASCC_CUDA(cudaStreamWaitEvent(s, ex.op_events[d], 0));
    exec_op(q, *ex.es[st], s, base, outb.data() + st * T3P_NBASE, scale, ws,
            ws + acc_off_ + st * acc_len_);
    ASCC_CUDA(cudaEventRecord(ex.op_events[q], s));
  }
  for (int k = 0; k < ns; ++k) {
    Einsum& e = *ex.es[k];
    e.set_split(e.level(), e.err(), min0[k]);
  }
  for (int k = 1; k < ns; ++k) {
    ASCC_CUDA(cudaEventRecord(ex.join[k], ex.streams[k]));
    ASCC_CUDA(cudaStreamWaitEvent(s0, ex.join[k], 0));
  }
  k::sum_rows(s0, base[T3P_RA], ex.priv, nb, ns);
}

T3pProgram::~T3pProgram() {
  if (profile_path_ && !prof_ms_.empty()) {
    if (FILE* f = std::fopen(profile_path_, "w")) {
      std::fprintf(f, "op,section,kind,a_dims,b_dims,out_dims,spec,calls,ms\n");
      auto dims = [&](int t) { return t >= 0 ? kT3pTensors[t].dims : ""; };
      for (int q = 0; q < kT3pOpCount; ++q) {
        const T3pOp& op = kT3pOps[q];
        std::fprintf(f, "%d,%d,%d,%s,%s,%s,%s,%d,%.6f\n", q, op.section, op.kind, dims(op.a),
                     dims(op.b), op.out >= 0 ? dims(op.out) : op.outspec, op.spec, prof_n_[q],
                     prof_ms_[q]);
      }
      std::fclose(f);
    }
  }
  for (auto& e : prof_ev_) cudaEventDestroy(e);
}

namespace {
// the dims of member m of a '+'-separated rows string
std::string member_dims(const char* rows, int m) {
  const char* c = rows;
  for (int q = 0; q < m; ++q) {
    while (*c && *c != '+') ++c;
    if (*c) ++c;
  }
  std::string d;
  while (*c && *c != '+') d += *c++;
  return d;
}

}  // namespace

// Kind 3: member operand Y (labels: spec before ->) into rows [off, off + N_m)
// of the stack S[#][K...], in the order spec after -> (the member's free
// labels, then the contracted ones).  Kind 4: the member's columns of the
// stacked product W[F...][#] (labels: F, then the member's free labels) into
// its intermediate, or accumulated into an output block.
void T3pProgram::stack_copy(const T3pOp& op, cudaStream_t s, double* const* base,
                            double* const* outb, double scale, double* ws) const {
  const std::string spec(op.spec);
  const auto arrow = spec.find("->");
  const std::string lhs = spec.substr(0, arrow), rhs = spec.substr(arrow + 2);
  auto ext = [&](char c) -> int64_t {
    return c == 'o' ? o_ : c == 'v' ? v_ : c == 'P' ? naux_ : (int64_t)n_;
  };
  if (op.kind == 3) {
    const T3pTensor& S = kT3pTensors[op.out];
    const std::string gd = member_dims(S.rows, op.member);
    const int64_t off = stack_rows(S.rows, op.member);
    std::vector<int64_t> kshape(shape_[op.out].begin() + 1, shape_[op.out].end());
    int64_t kprod = 1;
    for (auto d : kshape) kprod *= d;
    std::vector<int64_t> gshape;
    for (char c : gd) gshape.push_back(ext(c));
    std::vector<int64_t> dst = rm_strides(gshape), kst = rm_strides(kshape);
    for (auto& x : dst) x *= kprod;
    dst.insert(dst.end(), kst.begin(), kst.end());
    const T3pTensor& Yd = kT3pTensors[op.a];
    const std::vector<int64_t> yshape = Yd.kind == 0 ? base_shape(Yd.base) : shape_[op.a];
    const std::vector<int64_t> yst = rm_strides(yshape);
    const double* y = Yd.kind == 0 ? base[Yd.base] : ws + offset_[op.a];
    std::vector<int64_t> src, shape;
    for (char c : rhs) {
      const auto q = lhs.find(c);
      src.push_back(yst[q]);
      shape.push_back(yshape[q]);
    }
    if (shape.empty()) {
      shape = {1};
      src = {1};
      dst = {1};
    }
    box_copy(s, ws + offset_[op.out] + off * kprod, dst, y, src, shape);
    return;
  }
  const T3pTensor& W = kT3pTensors[op.a];
  const std::string fd(W.dims, std::strlen(W.dims) - 1);
  const std::string gd = member_dims(W.rows, op.member);
  const int64_t off = stack_rows(W.rows, op.member);
  const int64_t ntot = shape_[op.a].back();
  std::vector<int64_t> fshape, gshape;
  for (char c : fd) fshape.push_back(ext(c));
  for (char c : gd) gshape.push_back(ext(c));
  std::vector<int64_t> fst = rm_strides(fshape), gst = rm_strides(gshape);
  for (auto& x : fst) x *= ntot;
  std::vector<int64_t> lab_st(fst), lab_ext(fshape);
  lab_st.insert(lab_st.end(), gst.begin(), gst.end());
  lab_ext.insert(lab_ext.end(), gshape.begin(), gshape.end());
  ASCC_REQUIRE(lab_st.size() == lhs.size(), "T3' program: unstack labels");
  std::vector<int64_t> src, shape;
  for (char c : rhs) {
    const auto q = lhs.find(c);
    src.push_back(lab_st[q]);
    shape.push_back(lab_ext[q]);
  }
  const double* w = ws + offset_[op.a] + off;
  if (op.out >= 0) {
    ASCC_REQUIRE(shape_[op.out] == shape, "T3' program: unstack result shape");
    std::vector<int64_t> dst = rm_strides(shape_[op.out]);
    if (shape.empty()) {
      shape = {1};
      src = {1};
      dst = {1};
    }
    box_copy(s, ws + offset_[op.out], dst, w, src, shape, op.alpha, 0.0);
    return;
  }
  int64_t boff;
  std::vector<int64_t> bshape, bstride;
  select(op.base, op.outspec, &boff, bshape, bstride);
  ASCC_REQUIRE(bshape == shape, "T3' program: unstack output box");
  if (shape.empty()) {
    shape = {1};
    src = {1};
    bstride = {1};
  }
  box_copy(s, outb[op.base] + boff, bstride, w, src, shape, op.alpha * scale, 1.0);
}

namespace k {
namespace {
__global__ void t3p_unpack_kernel(double* __restrict__ blocks, const double* __restrict__ t3,
                                  const int64_t* __restrict__ dst,
                                  const int64_t* __restrict__ dst2,
                                  const signed char* __restrict__ sgn, int64_t n3) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n3;
       q += (int64_t)gridDim.x * blockDim.x) {
    const double x = t3[q] * (double)sgn[q];
    blocks[dst[q]] = x;
    if (dst2[q] >= 0) blocks[dst2[q]] = -x;
  }
}

__global__ void t3p_gather_kernel(double* __restrict__ r3, const double* __restrict__ blocks,
                                  const int64_t* __restrict__ dst,
                                  const signed char* __restrict__ sgn, int64_t n3) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n3;
       q += (int64_t)gridDim.x * blockDim.x)
    r3[q] = blocks[dst[q]] * (double)sgn[q];
}

int blocks_for(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
}
}  // namespace

void t3p_unpack(cudaStream_t s, double* blocks, int64_t nblk, const double* t3,
                const int64_t* dst, const int64_t* dst2, const signed char* sgn, int64_t n3) {
  fill(s, blocks, 0.0, nblk);
  if (n3 == 0) return;
  t3p_unpack_kernel<<<blocks_for(n3), 256, 0, s>>>(blocks, t3, dst, dst2, sgn, n3);
  count_launch();
  check_launch("t3p_unpack");
}

namespace {
__global__ void sum_rows_kernel(double* __restrict__ out, const double* __restrict__ part,
                                int64_t n, int nparts) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double t = out[i];
    for (int k = 0; k < nparts; ++k) t += part[k * n + i];
    out[i] = t;
  }
}
}  // namespace

void sum_rows(cudaStream_t s, double* out, const double* part, int64_t n, int nparts) {
  if (n <= 0) return;
  sum_rows_kernel<<<blocks_for(n), 256, 0, s>>>(out, part, n, nparts);
  count_launch();
  check_launch("sum_rows");
}

void t3p_gather(cudaStream_t s, double* r3, const double* blocks, const int64_t* dst,
                const signed char* sgn, int64_t n3) {
  if (n3 == 0) return;
  t3p_gather_kernel<<<blocks_for(n3), 256, 0, s>>>(r3, blocks, dst, sgn, n3);
  count_launch();
  check_launch("t3p_gather");
}
}  // namespace k

}  // namespace ascc
