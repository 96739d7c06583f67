// A variant of the split-precision tensor-core GEMM that allocates nothing.
//
// Some callers cannot allocate device memory when they need the product: a
// process whose GPU memory has been handed in full to another pool (a
// framework's caching allocator that reserved the device up front) has none
// left for cudaMalloc, and code that must not enter the CUDA allocator at all
// (cudaMalloc / cudaFree may synchronise the whole device) cannot use the
// stream-ordered scratch of ascc_gemm_split_bf16.  For them the BF16 operand
// planes and the FP32 split-K partials live in a fixed file-scope device
// array instead.
#include <cuda_bf16.h>

#include <cmath>
#include <mutex>

#include "gemm_tc.h"

namespace {

// Capacity of the shared scratch: level * (M + N) * Kp BF16 values plus the
// split-K partials (z * M * N FP32 values when K is split in z chunks).
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
    // the K split of ascc_gemm_split_bf16, so that both give the same product
    const int z = tc::splitk_for(M, N, K);
    const double planes = 2.0 * level * ((double)M + (double)N) * (double)Kp;
    const double plane_bytes = std::ceil(planes / 256.0) * 256.0;
    const double need = plane_bytes + (z > 1 ? 4.0 * z * (double)M * (double)N : 0.0);
    if (need > (double)kScratchBytes)
      throw Error(ASCC_ERR_INVALID,
                  "ascc_gemm_split_bf16_noalloc: the operand planes and split-K partials need " +
                      std::to_string((long long)need) + " bytes; the fixed scratch holds " +
                      std::to_string((long long)kScratchBytes));
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc = scratch_for_current_device();
    auto* pa = static_cast<__nv_bfloat16*>(sc.planes);
    __nv_bfloat16* pb = pa + (int64_t)level * M * Kp;
    float* ws = z > 1 ? reinterpret_cast<float*>(static_cast<unsigned char*>(sc.planes) +
                                                 (size_t)plane_bytes)
                      : nullptr;
    ASCC_CUDA(cudaMemsetAsync(sc.err, 0, sizeof(int), s));
    tc::split_bf16(s, pa, A, M, K, K, level);
    tc::split_bf16(s, pb, B, N, K, K, level);
    tc::gemm_split(s, M, N, K, level, alpha, pa, pb, beta, C, N, sc.err, z, ws, 0, nullptr,
                   tc::kTileRules);
    // this call's bounded device waits: read the flag back (synchronises s)
    int flag = 0;
    ASCC_CUDA(cudaMemcpyAsync(&flag, sc.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    ASCC_CUDA(cudaStreamSynchronize(s));
    if (flag) throw Error(ASCC_ERR_TIMEOUT, "ascc_gemm_split_bf16_noalloc: a device wait timed out");
    return ASCC_OK;
  });
}
