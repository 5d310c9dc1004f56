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
};

template <>
struct Store<float> {
  using R = float;
  static __device__ __forceinline__ R ld(const float* p) { return __ldg(p); }
  static __device__ __forceinline__ void st(float* p, R v) { *p = v; }
};

template <>
struct Store<__half> {
  using R = float;
  static __device__ __forceinline__ R ld(const __half* p) { return __half2float(__ldg(p)); }
  static __device__ __forceinline__ void st(__half* p, R v) { *p = __float2half_rn(v); }
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
};

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
