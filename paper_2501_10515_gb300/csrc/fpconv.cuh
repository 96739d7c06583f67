// FP32 <-> FP64 conversions in integer arithmetic.  The FP64 pipe of this part
// executes about two operations per clock per SM, so a conversion per element
// there (F2F), not memory, bounds the plane splits and the FP64 epilogues of
// the tensor-core GEMMs.  Each function gives exactly the IEEE-754 result of
// the plain expression it replaces; the rare operands outside the normal
// range take that expression in a separate (not inlined) function, so that
// the compiler does not evaluate it for every element.
#pragma once

#include <cstdint>

namespace ascc {

static __device__ __noinline__ float f64_to_f32_cast(double x) { return (float)x; }
static __device__ __noinline__ double f32_scaled_fp64(float x, double alpha) {
  return alpha * (double)x;
}
static __device__ __noinline__ double i64_scaled_fp64(long long q, int sh) {
  return ldexp((double)q, sh);
}

// (float)x, round to nearest even: the 52-bit significand is cut to 23 bits
// and rounded up when the dropped bits exceed half an ulp, or equal it and the
// kept value is odd; a carry out of the significand increments the exponent
// (up to infinity, as the rounding requires).
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const uint64_t u = (uint64_t)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(u >> 32);
  const uint32_t sign = hi & 0x80000000u;
  if ((u << 1) == 0) return __uint_as_float(sign);
  const int ef = (int)((hi >> 20) & 0x7ff) - 1023 + 127;
  if (ef < 1 || ef > 254) return f64_to_f32_cast(x);  // FP32 subnormal, overflow, inf, nan
  // significand bits 51..29 kept (20 from the high word, 3 from the low),
  // bits 28..0 dropped
  const uint32_t lo = (uint32_t)u;
  uint32_t r = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t rem = lo & 0x1fffffffu;
  r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;
  return __uint_as_float(sign | (((uint32_t)ef << 23) + r));
}

// alpha = (-1)^neg 2^e exactly (ok), read from its bits.
struct Pow2 {
  bool ok;
  int e;
  uint32_t neg;
};

__device__ __forceinline__ Pow2 pow2_of(double alpha) {
  const uint64_t u = (uint64_t)__double_as_longlong(alpha);
  const int ex = (int)((u >> 52) & 0x7ff);
  Pow2 p;
  p.neg = (uint32_t)(u >> 63);
  p.e = ex - 1023;
  p.ok = (u & 0xfffffffffffffull) == 0 && ex > 0 && ex < 2047;
  return p;
}

// (double)x, built from the bits of x (exact).
__device__ __forceinline__ double f32_to_f64(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t ex = (u >> 23) & 0xffu;
  if ((u & 0x7fffffffu) == 0) return __hiloint2double((int)(u & 0x80000000u), 0);
  if (ex == 0 || ex == 255) return f32_scaled_fp64(x, 1.0);  // subnormal, inf, nan
  const uint32_t m = u & 0x7fffffu;
  return __hiloint2double(
      (int)((u & 0x80000000u) | ((ex + (1023 - 127)) << 20) | (m >> 3)), (int)(m << 29));
}

// alpha * (double)x for alpha = (-1)^p.neg 2^p.e: the exponent of alpha is
// added to that of x (exact); results outside the normal range take the FP64
// product.
__device__ __forceinline__ double f32_to_f64_pow2(float x, const Pow2& p, double alpha) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t ex = (u >> 23) & 0xffu;
  const uint32_t s = ((u >> 31) ^ p.neg) << 31;
  if ((u & 0x7fffffffu) == 0) return __hiloint2double((int)s, 0);
  const int e = (int)ex + (1023 - 127) + p.e;
  if (ex == 0 || ex == 255 || e <= 0 || e >= 2047) return f32_scaled_fp64(x, alpha);
  const uint32_t m = u & 0x7fffffu;
  return __hiloint2double((int)(s | ((uint32_t)e << 20) | (m >> 3)), (int)(m << 29));
}

// How an epilogue writes alpha * acc (+ beta * C), decided once per kernel so
// that no per-element select evaluates an FP64 operation it does not need:
// beta = 0 with a power-of-two alpha (integer arithmetic only), beta = 0 with
// another alpha (one FP64 product), beta = 1 (one FP64 fma: beta * C = C),
// other beta (FP64 fma of alpha acc and beta C).
enum StoreMode { kStorePow2 = 1, kStoreScaled = 2, kStoreBeta = 3, kStoreBeta1 = 4 };

inline int host_store_mode(double alpha, double beta) {
  if (beta == 1.0) return kStoreBeta1;
  if (beta != 0.0) return kStoreBeta;
  uint64_t u;
  __builtin_memcpy(&u, &alpha, sizeof(u));
  const int ex = (int)((u >> 52) & 0x7ff);
  return ((u & 0xfffffffffffffull) == 0 && ex > 0 && ex < 2047) ? kStorePow2 : kStoreScaled;
}

// (double)q * 2^sh with the sign flipped when neg: the cast's round to nearest
// even of |q| to 53 bits, then the exponent; false (and nothing written) when
// the result is not a normal FP64 number.
__device__ __forceinline__ bool i64_to_f64_scaled(long long q, int sh, uint32_t neg,
                                                  double& out) {
  if (q == 0) {
    out = __hiloint2double((int)(neg << 31), 0);
    return true;
  }
  const uint64_t sgn = (uint64_t)((q < 0 ? 1u : 0u) ^ neg) << 63;
  const uint64_t m = q < 0 ? (uint64_t)(-(q + 1)) + 1u : (uint64_t)q;
  const int nb = 64 - __clzll((long long)m);
  int e = nb - 1 + sh;
  uint64_t mant;
  if (nb <= 53) {
    mant = m << (53 - nb);
  } else {
    const int r = nb - 53;
    mant = m >> r;
    const uint64_t rem = m & ((1ull << r) - 1), half = 1ull << (r - 1);
    if (rem > half || (rem == half && (mant & 1u))) ++mant;
    if (mant >> 53) {
      mant >>= 1;
      ++e;
    }
  }
  const int be = e + 1023;
  if (be <= 0 || be >= 2047) return false;
  out = __longlong_as_double((long long)(sgn | ((uint64_t)be << 52) | (mant & 0xfffffffffffffull)));
  return true;
}

}  // namespace ascc
