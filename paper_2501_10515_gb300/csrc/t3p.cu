// Executor of the generated T3' program (see t3p.h) and the kernels that move
// the packed slice into its dense blocks and back.
#include <algorithm>
#include <cstring>

#include "kernels.h"
#include "t3p.h"

namespace ascc {

namespace {
#include "t3p_program.inc"

int64_t round_up(int64_t x, int64_t q) { return (x + q - 1) / q * q; }
}  // namespace

T3pProgram::T3pProgram(int o, int v, int naux, int h, int p)
    : o_(o), v_(v), n_(o + v), naux_(naux), h_(h), p_(p) {
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
    for (const char* c = kT3pTensors[t].dims; *c; ++c) shape_[t].push_back(extent(*c));
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
    const int s = def[t], e = std::max(last[t], def[t]);
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
  ws_elems_ = acc_off_ + round_up(acc_max, 32);
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
constexpr double kTcMinFlops = 1e6;

void T3pProgram::run(Einsum& es, cudaStream_t s, int section, double* const* base,
                     double scale, double* ws) const {
  const double min0 = es.min_flops();
  if (es.level() > 0) es.set_split(es.level(), es.err(), std::min(min0, kTcMinFlops));
  auto tensor = [&](int t) -> T {
    const T3pTensor& d = kT3pTensors[t];
    if (d.kind == 0) return T(base[d.base], base_shape(d.base));
    return T(ws + offset_[t], shape_[t]);
  };
  for (int q = 0; q < kT3pOpCount; ++q) {
    const T3pOp& op = kT3pOps[q];
    if (op.section != section) continue;
    if (op.kind == 0) {
      int64_t off;
      std::vector<int64_t> shape, stride;
      select(op.base, kT3pTensors[op.out].spec, &off, shape, stride);
      std::vector<int64_t> ost(shape.size());
      int64_t acc = 1;
      for (int d = (int)shape.size() - 1; d >= 0; --d) {
        ost[d] = acc;
        acc *= shape[d];
      }
      if (shape.empty()) {
        shape = {1};
        stride = {1};
        ost = {1};
      }
      box_copy(s, ws + offset_[op.out], ost, base[op.base] + off, stride, shape);
    } else if (op.kind == 1) {
      es(op.spec, op.alpha, tensor(op.a), tensor(op.b), 0.0, tensor(op.out));
    } else {
      int64_t off;
      std::vector<int64_t> shape, stride;
      select(op.base, op.outspec, &off, shape, stride);
      const bool whole = off == 0 && shape == base_shape(op.base);
      if (whole) {
        es(op.spec, op.alpha * scale, tensor(op.a), tensor(op.b), 1.0,
           T(base[op.base], shape));
        continue;
      }
      double* tmp = ws + acc_off_;
      es(op.spec, op.alpha * scale, tensor(op.a), tensor(op.b), 0.0, T(tmp, shape));
      std::vector<int64_t> ost(shape.size());
      int64_t acc = 1;
      for (int d = (int)shape.size() - 1; d >= 0; --d) {
        ost[d] = acc;
        acc *= shape[d];
      }
      if (shape.empty()) {
        shape = {1};
        stride = {1};
        ost = {1};
      }
      box_copy(s, base[op.base] + off, stride, tmp, ost, shape, 1.0, 1.0);
    }
  }
  es.set_split(es.level(), es.err(), min0);
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

void t3p_gather(cudaStream_t s, double* r3, const double* blocks, const int64_t* dst,
                const signed char* sgn, int64_t n3) {
  if (n3 == 0) return;
  t3p_gather_kernel<<<blocks_for(n3), 256, 0, s>>>(r3, blocks, dst, sgn, n3);
  count_launch();
  check_launch("t3p_gather");
}
}  // namespace k

}  // namespace ascc
