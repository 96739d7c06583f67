// A variant of the split-precision tensor-core GEMM that allocates nothing.
//
// Some callers cannot call cudaMalloc at the time they need the product:
// code running inside a CUDA stream capture that must not create memory
// nodes, real-time loops that forbid allocator calls (which may synchronise
// or page), or hosts whose device memory is fully handed out up front to a
// framework's own pool.  For them the BF16 operand planes live in a fixed
// file-scope device array instead of stream-ordered scratch.
#include <cuda_bf16.h>

#include <mutex>

#include "gemm_tc.h"

namespace {

// Capacity of the shared scratch: level * (M + N) * Kp BF16 values must fit.
constexpr size_t kScratchBytes = 32u << 20;  // 32 MiB per device, held until exit

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];
static __device__ __align__(256) int g_scratch_err;

struct Scratch {
  void* planes = nullptr;
  int* err = nullptr;
};

constexpr int kMaxDevices = 64;
std::mutex g_mu;
Scratch g_dev[kMaxDevices];

// Device addresses of the scratch on the current device.  The first call on a
// device resolves them with cudaGetSymbolAddress (the host-side names are only
// stand-ins); later calls reuse the cached addresses.
Scratch scratch_for_current_device() {
  int dev = 0;
  ASCC_CUDA(cudaGetDevice(&dev));
  ASCC_REQUIRE(dev >= 0 && dev < kMaxDevices, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  Scratch& s = g_dev[dev];
  if (!s.planes) {
    void* p = nullptr;
    void* e = nullptr;
    ASCC_CUDA(cudaGetSymbolAddress(&p, g_scratch));
    ASCC_CUDA(cudaGetSymbolAddress(&e, g_scratch_err));
    s.planes = p;
    s.err = static_cast<int*>(e);
  }
  return s;
}

}  // namespace

using namespace ascc;

namespace {
template <class F>
ascc_status guarded(F&& f) {
  try {
    return f();
  } catch (const Error& e) {
    record_error(e.what());
    return e.status;
  } catch (const std::exception& e) {
    record_error(e.what());
    return ASCC_ERR_INVALID;
  }
}
}  // namespace

extern "C" ascc_status ascc_gemm_split_bf16_noalloc(int64_t M, int64_t N, int64_t K,
                                                    int32_t level, double alpha, const double* A,
                                                    const double* B, double beta, double* C,
                                                    void* stream) {
  return guarded([&]() -> ascc_status {
    ASCC_REQUIRE(A && B && C && M > 0 && N > 0 && K > 0, "bad argument");
    ASCC_REQUIRE(level >= 1 && level <= 3, "level must be 1, 2 or 3");
    const int64_t Kp = tc::padded_k(K);
    const double need = 2.0 * level * ((double)M + (double)N) * (double)Kp;
    if (need > (double)kScratchBytes)
      throw Error(ASCC_ERR_INVALID,
                  "ascc_gemm_split_bf16_noalloc: level*(M+N)*ceil64(K) BF16 values need " +
                      std::to_string((long long)need) + " bytes; the fixed scratch holds " +
                      std::to_string((long long)kScratchBytes));
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc = scratch_for_current_device();
    // report a timeout of the previous call on this device, then clear the flag
    int prev = 0;
    ASCC_CUDA(cudaMemcpyAsync(&prev, sc.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    ASCC_CUDA(cudaStreamSynchronize(s));
    ASCC_CUDA(cudaMemsetAsync(sc.err, 0, sizeof(int), s));
    if (prev) throw Error(ASCC_ERR_TIMEOUT, "a previous no-alloc GEMM wait timed out");
    __nv_bfloat16* pa = static_cast<__nv_bfloat16*>(sc.planes);
    __nv_bfloat16* pb = pa + (int64_t)level * M * Kp;
    tc::split_bf16(s, pa, A, M, K, K, level);
    tc::split_bf16(s, pb, B, N, K, K, level);
    tc::gemm_split(s, M, N, K, level, alpha, pa, pb, beta, C, N, sc.err);
    return ASCC_OK;
  });
}
