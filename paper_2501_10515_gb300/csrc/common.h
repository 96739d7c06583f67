// Shared host/device utilities of libascc: status plumbing, device buffers,
// dense row-major tensors and the launch counter.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/ascc.h"

namespace ascc {

// An exception carrying an ascc_status; caught at the C ABI boundary.
struct Error : std::runtime_error {
  ascc_status status;
  Error(ascc_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define ASCC_CUDA(call)                                                          \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      throw ::ascc::Error(e_ == cudaErrorMemoryAllocation ? ASCC_ERR_OOM         \
                                                           : ASCC_ERR_CUDA,      \
                          std::string(#call) + ": " + cudaGetErrorString(e_) +   \
                              " (" __FILE__ ":" + std::to_string(__LINE__) + ")"); \
    }                                                                            \
  } while (0)

#define ASCC_REQUIRE(cond, msg)                                                  \
  do {                                                                           \
    if (!(cond)) throw ::ascc::Error(ASCC_ERR_INVALID, (msg));                   \
  } while (0)

// Kernel launch bookkeeping: every launch goes through count_launch() so the
// context can report how many of its own kernels ran.
void count_launch(int64_t n = 1);
int64_t launch_total();
void count_flops(double f);
double flop_total();
// the same counts for the calling thread only (exact deltas around a capture)
int64_t thread_launches();
double thread_flops();
void check_launch(const char* what);
// Stores the message returned by ascc_last_error() on this thread.
void record_error(const std::string& msg);

// Stream-ordered device buffer.
class DevBuf {
 public:
  DevBuf() = default;
  DevBuf(size_t bytes, cudaStream_t s) { alloc(bytes, s); }
  ~DevBuf() { release(); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept { swap(o); }
  DevBuf& operator=(DevBuf&& o) noexcept {
    release();
    swap(o);
    return *this;
  }
  void alloc(size_t bytes, cudaStream_t s) {
    release();
    stream_ = s;
    bytes_ = bytes;
    if (bytes) ASCC_CUDA(cudaMallocAsync(&ptr_, bytes, s));
  }
  void release() {
    if (ptr_) cudaFreeAsync(ptr_, stream_);
    ptr_ = nullptr;
    bytes_ = 0;
  }
  template <class T = double>
  T* as() const { return static_cast<T*>(ptr_); }
  size_t bytes() const { return bytes_; }
  void zero() const {
    if (bytes_) ASCC_CUDA(cudaMemsetAsync(ptr_, 0, bytes_, stream_));
  }

 private:
  void swap(DevBuf& o) {
    std::swap(ptr_, o.ptr_);
    std::swap(bytes_, o.bytes_);
    std::swap(stream_, o.stream_);
  }
  void* ptr_ = nullptr;
  size_t bytes_ = 0;
  cudaStream_t stream_ = nullptr;
};

// A dense row-major FP64 tensor view (does not own memory).
struct T {
  double* p = nullptr;
  std::vector<int64_t> shape;
  T() = default;
  T(double* ptr, std::vector<int64_t> s) : p(ptr), shape(std::move(s)) {}
  int64_t size() const {
    int64_t n = 1;
    for (auto d : shape) n *= d;
    return n;
  }
  int nd() const { return (int)shape.size(); }
};

// An owned tensor.
struct OT {
  DevBuf buf;
  T t;
  OT() = default;
  OT(std::vector<int64_t> shape, cudaStream_t s) { make(std::move(shape), s); }
  void make(std::vector<int64_t> shape, cudaStream_t s) {
    int64_t n = 1;
    for (auto d : shape) n *= d;
    buf.alloc(sizeof(double) * (size_t)n, s);
    t = T(buf.as<double>(), std::move(shape));
  }
  double* p() const { return t.p; }
  operator const T&() const { return t; }
};

// A strided tensor read as a matrix: row r = (r_0, .., r_{nm-1}) and column
// k = (k_0, .., k_{nk-1}) in row-major digit order over mext / kext; the
// element is at sum_d r_d mstr[d] + sum_d k_d kstr[d] (in elements).
struct MatView {
  int nm = 0, nk = 0;
  int64_t mext[4] = {}, mstr[4] = {}, kext[4] = {}, kstr[4] = {};
  int64_t rows() const {
    int64_t n = 1;
    for (int d = 0; d < nm; ++d) n *= mext[d];
    return n;
  }
  int64_t cols() const {
    int64_t n = 1;
    for (int d = 0; d < nk; ++d) n *= kext[d];
    return n;
  }
};

}  // namespace ascc
