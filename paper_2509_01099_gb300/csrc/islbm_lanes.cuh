// Arithmetic on one node (float, double) or on two nodes at once (float2: the
// paired FP32 instructions of sm_100 and later, one issue slot for both
// nodes).  The collision is written once against these helpers.
#pragma once

#include <cuda_runtime.h>

namespace islbm {

// The scalar forms leave the compiler free to fuse a product into a following
// sum (fewer instructions in the one-node-per-thread kernels); the paired forms
// round every operation as written.
__device__ __forceinline__ float ladd(float a, float b) { return a + b; }
__device__ __forceinline__ float lsub(float a, float b) { return a - b; }
__device__ __forceinline__ float lmul(float a, float b) { return a * b; }
__device__ __forceinline__ float lfma(float a, float b, float c) { return fmaf(a, b, c); }
// 1 / rho of the collision: FP64 divides; FP32 takes the hardware reciprocal
// (within 2 ulp for the densities ~1 of a weakly compressible flow, far below
// the rounding of the FP32 step)
__device__ __forceinline__ float lrcp(float a) { return __fdividef(1.0f, a); }

__device__ __forceinline__ double ladd(double a, double b) { return a + b; }
__device__ __forceinline__ double lsub(double a, double b) { return a - b; }
__device__ __forceinline__ double lmul(double a, double b) { return a * b; }
__device__ __forceinline__ double lfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double lrcp(double a) { return 1.0 / a; }

__device__ __forceinline__ float2 ladd(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as b * (-1) + a: the product is exact, so this rounds like a - b
__device__ __forceinline__ float2 lsub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 lmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 lfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 lrcp(float2 a) {
  return make_float2(__fdividef(1.0f, a.x), __fdividef(1.0f, a.y));
}

// Three-point interpolation sum w0 a + w1 b + w2 c (t.x a + t.y b + t.z c for
// a packed table), with its roundings
// fixed (no freedom left to the compiler's multiply-add fusion, so every build
// of a kernel computes the same bits).
__device__ __forceinline__ float lin3(float w0, float w1, float w2, float a, float b, float c) {
  return fmaf(w2, c, fmaf(w1, b, __fmul_rn(w0, a)));
}
__device__ __forceinline__ double lin3(double w0, double w1, double w2, double a, double b,
                                       double c) {
  return fma(w2, c, fma(w1, b, __dmul_rn(w0, a)));
}
__device__ __forceinline__ float dot3(float4 t, float a, float b, float c) {
  return lin3(t.x, t.y, t.z, a, b, c);
}

// A scalar (a constant or a parameter) as a lane value.
template <typename L>
struct Lanes;
template <>
struct Lanes<float> {
  using S = float;
  static __device__ __forceinline__ float bc(float v) { return v; }
};
template <>
struct Lanes<double> {
  using S = double;
  static __device__ __forceinline__ double bc(double v) { return v; }
};
template <>
struct Lanes<float2> {
  using S = float;
  static __device__ __forceinline__ float2 bc(float v) { return make_float2(v, v); }
};

}  // namespace islbm
