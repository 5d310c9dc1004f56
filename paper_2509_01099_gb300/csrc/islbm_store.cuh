// Storage types of the population arrays and their compute type.
//
// Every storage form holds the deviation from the rest state (f_i - w_i for the
// flow populations, g_i - t_i T0 for the temperature populations); FP64 computes
// in double, the other forms in float.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace islbm {

template <typename S>
struct Store;

template <>
struct Store<double> {
  using R = double;
  static __device__ __forceinline__ R ld(const double* p) { return __ldg(p); }
  static __device__ __forceinline__ void st(double* p, R v) { *p = v; }
  static __device__ __forceinline__ void st_sr(double* p, R v, unsigned) { *p = v; }
};

template <>
struct Store<float> {
  using R = float;
  static __device__ __forceinline__ R ld(const float* p) { return __ldg(p); }
  static __device__ __forceinline__ void st(float* p, R v) { *p = v; }
  static __device__ __forceinline__ void st_sr(float* p, R v, unsigned) { *p = v; }
};

// Stochastic rounding of the 16-bit stores of the time step.  Near a steady
// state the per-step change of a population (e.g. the buoyancy increment
// g beta T w_i ~ 1e-6) is below half an FP16 / BF16 ulp of the stored
// deviation; round-to-nearest then discards it on every step and the flow
// stalls.  Adding uniform random bits below the kept mantissa and truncating
// rounds up with probability equal to the discarded fraction, so the
// expected stored value is exact.  `r` supplies 32 random bits.
__device__ __forceinline__ __half sr_to_fp16(float v, unsigned r) {
  const float a = fabsf(v);
  // FP16 normal range: the 13 mantissa bits dropped by the truncating conversion
  // receive random bits first (adding to the bit pattern keeps the sign)
  const float vn = __uint_as_float(__float_as_uint(v) + (r >> 19));
  // FP16 subnormal range: the grid is 2^-24; add a uniform fraction of it to |v|
  const float vs = copysignf(a + (float)(r >> 8) * 3.5527136788005009e-15f, v);
  return __float2half_rz(a >= 6.103515625e-05f ? vn : vs);
}

template <>
struct Store<__half> {
  using R = float;
  static __device__ __forceinline__ R ld(const __half* p) { return __half2float(__ldg(p)); }
  static __device__ __forceinline__ void st(__half* p, R v) { *p = __float2half_rn(v); }
  static __device__ __forceinline__ void st_sr(__half* p, R v, unsigned r) {
    *p = sr_to_fp16(v, r);
  }
};

template <>
struct Store<__nv_bfloat16> {
  using R = float;
  static __device__ __forceinline__ R ld(const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(p));
  }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, R v) {
    *p = __float2bfloat16_rn(v);
  }
  static __device__ __forceinline__ void st_sr(__nv_bfloat16* p, R v, unsigned r) {
    // BF16 is the upper half of the FP32 pattern: add random bits to the lower
    // half (the carry rounds away from zero with the dropped fraction's
    // probability) and keep the upper half
    *p = __ushort_as_bfloat16((unsigned short)((__float_as_uint(v) + (r >> 16)) >> 16));
  }
};

// Random bits for the stochastic rounding: a counter-based hash of (node, step)
// (the murmur3 finalizer), then a linear congruential sequence per store.
__device__ __forceinline__ unsigned sr_seed(unsigned long long node, unsigned step) {
  unsigned h = (unsigned)node * 0x9e3779b1u ^ (unsigned)(node >> 32) ^ (step * 0x85ebca77u);
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}
__device__ __forceinline__ unsigned sr_next(unsigned& r) {
  r = r * 1664525u + 1013904223u;
  return r;
}

// FP64 block reduction helpers shared by the reduction kernels.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

}  // namespace islbm
