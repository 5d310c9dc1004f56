// Storage types of the population arrays and their compute type.
//
// Every storage form holds the deviation from the rest state (f_i - w_i for the
// flow populations, g_i - t_i T0 for the temperature populations); FP64 computes
// in double, the other forms in float.  The non-equilibrium form (Neq16) splits
// that deviation into FP32 moments and 16-bit remainders (below).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

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

// Non-equilibrium 16-bit storage (2-D).  Per node the buffer holds the
// collision invariants and momentum of the stored post-collision state in FP32,
//   m = (drho, jx, jy, Tr) = (sum_i d_i, sum_i e_ix d_i, sum_i e_iy d_i, sum_i g_i),
// with d_i = f_i - w_i, and per population the part that m does not fix,
//   r_i = d_i - E_i(m),
// where E_i(m) is the equilibrium deviation of those moments (the second-order
// Hermite form of Sec. 2.1 for the flow, N^-1 n_eq for the temperature).  After
// a collision that part is the relaxed non-equilibrium population plus the
// force term, orders of magnitude below d_i, so 16 bits of it resolve the
// state far more finely than 16 bits of d_i: r_i is kept as FP16 of
// r_i * 2^12 (the scale lifts it out of FP16's subnormal range), rounded to
// nearest.  The slowly varying part lives in the FP32 moments, so no
// stochastic rounding is needed.  Layout: 14 planes of FP16 remainders, then 4
// planes of FP32 moments, all with the same plane stride in elements.
struct Neq16 {
  unsigned short bits;
};

template <>
struct Store<Neq16> {
  using R = float;
};

template <typename S>
struct is_neq : std::false_type {};
template <>
struct is_neq<Neq16> : std::true_type {};

constexpr float kNeqScale = 4096.f;
constexpr float kNeqUnscale = 1.f / 4096.f;

// FP32 moment planes of a Neq16 buffer (after the 14 remainder planes).
__device__ __forceinline__ const float* neq_moments(const Neq16* s, long long P) {
  return reinterpret_cast<const float*>(s + 14 * P);
}
__device__ __forceinline__ float* neq_moments(Neq16* s, long long P) {
  return reinterpret_cast<float*>(s + 14 * P);
}

// E_i(m): equilibrium deviations of the moments m of a D2Q9 + D2Q5 node,
//   E_i = w_i (drho + 3 e_i.j + rho (9/2 (e_i.u)^2 - 3/2 u^2)), u = j / rho,
//   E^g_0 = t_0 Tr, E^g_i = t_i Tr + (e_i.u) Tr / 2 (i = 1..4),
// with t_0 = (1 - a_T)/5, t_i = (4 + a_T)/20 (the temperature equilibrium's
// rest weights).  Direction order as the 2-D kernels.
__device__ __forceinline__ void neq_eq2(float drho, float jx, float jy, float Tr, float t0,
                                        float ti, float (&e)[9], float (&q)[5]) {
  const float rho = 1.f + drho;
  const float inv = __frcp_rn(rho);
  const float ux = jx * inv, uy = jy * inv;
  const float a = drho - 1.5f * rho * (ux * ux + uy * uy);
  const float h = 4.5f * rho;
  const float rx = h * ux * ux, ry = h * uy * uy;
  const float sp = ux + uy, sm = uy - ux;
  const float rp = h * sp * sp, rm = h * sm * sm;
  const float jp = 3.f * (jx + jy), jm = 3.f * (jy - jx);
  constexpr float w0 = 4.f / 9.f, w1 = 1.f / 9.f, w5 = 1.f / 36.f;
  e[0] = w0 * a;
  e[1] = w1 * (a + rx + 3.f * jx);
  e[3] = w1 * (a + rx - 3.f * jx);
  e[2] = w1 * (a + ry + 3.f * jy);
  e[4] = w1 * (a + ry - 3.f * jy);
  e[5] = w5 * (a + rp + jp);
  e[7] = w5 * (a + rp - jp);
  e[6] = w5 * (a + rm + jm);
  e[8] = w5 * (a + rm - jm);
  const float hx = 0.5f * ux * Tr, hy = 0.5f * uy * Tr, tt = ti * Tr;
  q[0] = t0 * Tr;
  q[1] = tt + hx;
  q[3] = tt - hx;
  q[2] = tt + hy;
  q[4] = tt - hy;
}

// Deviations d_i, d^g_i of one node from its moments and stored remainders.
__device__ __forceinline__ void neq_decode2(float drho, float jx, float jy, float Tr,
                                            const unsigned short (&r)[14], float t0, float ti,
                                            float (&f)[9], float (&g)[5]) {
  neq_eq2(drho, jx, jy, Tr, t0, ti, f, g);
#pragma unroll
  for (int i = 0; i < 9; ++i)
    f[i] = fmaf(__half2float(__ushort_as_half(r[i])), kNeqUnscale, f[i]);
#pragma unroll
  for (int i = 0; i < 5; ++i)
    g[i] = fmaf(__half2float(__ushort_as_half(r[9 + i])), kNeqUnscale, g[i]);
}

// Moments and remainders of one node's deviations (the inverse of the above,
// exact up to the rounding of the remainders).
__device__ __forceinline__ void neq_encode2(const float (&f)[9], const float (&g)[5], float t0,
                                            float ti, float (&m)[4], unsigned short (&r)[14]) {
  m[0] = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
  m[1] = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
  m[2] = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
  m[3] = (g[0] + g[1]) + (g[2] + g[3]) + g[4];
  float e[9], q[5];
  neq_eq2(m[0], m[1], m[2], m[3], t0, ti, e, q);
#pragma unroll
  for (int i = 0; i < 9; ++i) r[i] = __half_as_ushort(__float2half_rn((f[i] - e[i]) * kNeqScale));
#pragma unroll
  for (int i = 0; i < 5; ++i)
    r[9 + i] = __half_as_ushort(__float2half_rn((g[i] - q[i]) * kNeqScale));
}

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
