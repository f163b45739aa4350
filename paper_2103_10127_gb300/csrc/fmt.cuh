// Reduced-precision storage formats of the stored subdomain inverses, shared
// by the apply kernels and their packing kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <type_traits>

#include "common.cuh"

namespace rav {

// ---------------------------------------------------------------------------
// Reduced-precision storage: round-to-nearest-even to a binary format with p
// significand bits, minimum normal exponent emin, saturating at vmax.
__device__ inline double round_fmt(double v, int p, int emin, double vmax) {
  if (v == 0.0 || !isfinite(v)) return v;
  int E;
  frexp(v, &E);
  int e = E - 1;
  if (e < emin) e = emin;
  const double quantum = ldexp(1.0, e - (p - 1));
  double q = rint(v / quantum) * quantum;
  q = q > vmax ? vmax : (q < -vmax ? -vmax : q);
  return q;
}

template <typename T>
struct Fmt;
template <>
struct Fmt<double> {
  static __device__ double enc(double v) { return v; }
  static __device__ double dec(double v, const float*) { return v; }
  static constexpr bool scaled = false;
};
template <>
struct Fmt<float> {
  static __device__ float enc(double v) { return (float)round_fmt(v, 24, -126, 3.4028234663852886e38); }
  static __device__ float dec(float v, const float*) { return v; }
  static constexpr bool scaled = false;
};
template <>
struct Fmt<__nv_bfloat16> {
  static __device__ __nv_bfloat16 enc(double v) {
    return __float2bfloat16_rn((float)round_fmt(v, 8, -126, 3.3895313892515355e38));
  }
  static __device__ float dec(__nv_bfloat16 v, const float*) { return __bfloat162float(v); }
  static constexpr bool scaled = false;
};
struct fp8_t {
  uint8_t bits;
};
__device__ __forceinline__ fp8_t ld_stream(const fp8_t* p) {
  fp8_t r;
  r.bits = __ldcs(reinterpret_cast<const unsigned char*>(p));
  return r;
}
template <>
struct Fmt<fp8_t> {
  static __device__ fp8_t enc(double v) {
    const float q = (float)round_fmt(v, 4, -6, 448.0);
    fp8_t r;
    r.bits = (uint8_t)__nv_cvt_float_to_fp8(q, __NV_SATFINITE, __NV_E4M3);
    return r;
  }
  static __device__ float dec(fp8_t v, const float* lut) { return lut[v.bits]; }
  static constexpr bool scaled = true;
};

// Accumulation type of an apply reading storage type T: fp64 for fp64
// storage, fp32 for every reduced format.
template <typename T>
using AccT = typename std::conditional<std::is_same<T, double>::value, double, float>::type;

}  // namespace rav
