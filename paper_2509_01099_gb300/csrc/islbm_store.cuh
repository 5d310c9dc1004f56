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
// Hermite form of Sec. 2.1 for the flow, N^-1 n_eq for the temperature, both
// with rho = 1 in their quadratic terms).  After
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

// Arithmetic of the non-equilibrium form, one node (float) or two (float2,
// the paired FP32 instructions), every operation rounded as written: the
// encode and decode of a node give the same bits in every kernel.
__device__ __forceinline__ float nq_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float nq_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float nq_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float nq_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float nq_bc(float v, float) { return v; }
__device__ __forceinline__ float2 nq_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as b * (-1) + a: the product is exact, so this rounds like a - b
__device__ __forceinline__ float2 nq_sub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 nq_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 nq_fma(float2 a, float2 b, float2 c) {
  return __ffma2_rn(a, b, c);
}
__device__ __forceinline__ float2 nq_bc(float v, float2) { return make_float2(v, v); }

// E_i(m): the equilibrium deviations of the moments m of a D2Q9 + D2Q5 node,
// with rho = 1 in the quadratic terms (no division: the difference from the
// equilibrium, drho u^2 ~ 1e-7, is carried by the remainder),
//   E_i = w_i (drho + 3 e_i.j + 9/2 (e_i.j)^2 - 3/2 j^2),
//   E^g_0 = t_0 Tr, E^g_i = t_i Tr + (e_i.j) Tr / 2 (i = 1..4),
// with t_0 = (1 - a_T)/5, t_i = (4 + a_T)/20 (the temperature equilibrium's
// rest weights).  Direction order as the 2-D kernels.
template <typename L>
__device__ __forceinline__ void neq_eq2(L drho, L jx, L jy, L Tr, float t0, float ti,
                                        L (&e)[9], L (&q)[5]) {
  auto c = [](float v) { return nq_bc(v, L{}); };
  const L jsq = nq_fma(jx, jx, nq_mul(jy, jy));
  const L a = nq_fma(c(-1.5f), jsq, drho);   // drho - 3/2 j^2
  const L sp = nq_add(jx, jy), sm = nq_sub(jy, jx);
  const L ax = nq_fma(nq_mul(c(4.5f), jx), jx, a);
  const L ay = nq_fma(nq_mul(c(4.5f), jy), jy, a);
  const L ap = nq_fma(nq_mul(c(4.5f), sp), sp, a);
  const L am = nq_fma(nq_mul(c(4.5f), sm), sm, a);
  const L jx3 = nq_mul(c(3.f), jx), jy3 = nq_mul(c(3.f), jy);
  const L jp = nq_mul(c(3.f), sp), jm = nq_mul(c(3.f), sm);
  const L w0 = c(4.f / 9.f), w1 = c(1.f / 9.f), w5 = c(1.f / 36.f);
  e[0] = nq_mul(w0, a);
  e[1] = nq_mul(w1, nq_add(ax, jx3));
  e[3] = nq_mul(w1, nq_sub(ax, jx3));
  e[2] = nq_mul(w1, nq_add(ay, jy3));
  e[4] = nq_mul(w1, nq_sub(ay, jy3));
  e[5] = nq_mul(w5, nq_add(ap, jp));
  e[7] = nq_mul(w5, nq_sub(ap, jp));
  e[6] = nq_mul(w5, nq_add(am, jm));
  e[8] = nq_mul(w5, nq_sub(am, jm));
  const L hx = nq_mul(nq_mul(c(0.5f), jx), Tr), hy = nq_mul(nq_mul(c(0.5f), jy), Tr);
  const L tt = nq_mul(c(ti), Tr);
  q[0] = nq_mul(c(t0), Tr);
  q[1] = nq_add(tt, hx);
  q[3] = nq_sub(tt, hx);
  q[2] = nq_add(tt, hy);
  q[4] = nq_sub(tt, hy);
}

// The moments (drho, jx, jy, Tr) of one node's deviations.
template <typename L>
__device__ __forceinline__ void neq_moments2(const L (&f)[9], const L (&g)[5], L (&m)[4]) {
  m[0] = nq_add(nq_add(nq_add(nq_add(f[0], f[1]), nq_add(f[2], f[3])),
                       nq_add(nq_add(f[4], f[5]), nq_add(f[6], f[7]))),
                f[8]);
  m[1] = nq_add(nq_add(nq_sub(f[1], f[3]), nq_sub(f[5], f[6])), nq_sub(f[8], f[7]));
  m[2] = nq_sub(nq_add(nq_sub(f[2], f[4]), nq_add(f[5], f[6])), nq_add(f[7], f[8]));
  m[3] = nq_add(nq_add(nq_add(g[0], g[1]), nq_add(g[2], g[3])), g[4]);
}

// Deviations d_i, d^g_i of one node from its moments and stored remainders.
__device__ __forceinline__ void neq_decode2(float drho, float jx, float jy, float Tr,
                                            const unsigned short (&r)[14], float t0, float ti,
                                            float (&f)[9], float (&g)[5]) {
  neq_eq2<float>(drho, jx, jy, Tr, t0, ti, f, g);
#pragma unroll
  for (int i = 0; i < 9; ++i)
    f[i] = __fmaf_rn(__half2float(__ushort_as_half(r[i])), kNeqUnscale, f[i]);
#pragma unroll
  for (int i = 0; i < 5; ++i)
    g[i] = __fmaf_rn(__half2float(__ushort_as_half(r[9 + i])), kNeqUnscale, g[i]);
}

// The same for two nodes: remainders as half2 pairs (node a in the low half).
__device__ __forceinline__ void neq_decode2x2(float2 drho, float2 jx, float2 jy, float2 Tr,
                                              const unsigned (&r)[14], float t0, float ti,
                                              float2 (&f)[9], float2 (&g)[5]) {
  neq_eq2<float2>(drho, jx, jy, Tr, t0, ti, f, g);
  const float2 u = make_float2(kNeqUnscale, kNeqUnscale);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const __half2 h = *reinterpret_cast<const __half2*>(&r[i]);
    f[i] = __ffma2_rn(__half22float2(h), u, f[i]);
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const __half2 h = *reinterpret_cast<const __half2*>(&r[9 + i]);
    g[i] = __ffma2_rn(__half22float2(h), u, g[i]);
  }
}

// Moments and remainders of one node's deviations (the inverse of the above,
// exact up to the rounding of the remainders).
__device__ __forceinline__ void neq_encode2(const float (&f)[9], const float (&g)[5], float t0,
                                            float ti, float (&m)[4], unsigned short (&r)[14]) {
  neq_moments2<float>(f, g, m);
  float e[9], q[5];
  neq_eq2<float>(m[0], m[1], m[2], m[3], t0, ti, e, q);
#pragma unroll
  for (int i = 0; i < 9; ++i)
    r[i] = __half_as_ushort(__float2half_rn(__fmul_rn(__fsub_rn(f[i], e[i]), kNeqScale)));
#pragma unroll
  for (int i = 0; i < 5; ++i)
    r[9 + i] = __half_as_ushort(__float2half_rn(__fmul_rn(__fsub_rn(g[i], q[i]), kNeqScale)));
}

// The remainders of two nodes (node a in the low halves) for given moments m
// (the collision's post-collision moments: exact up to rounding, which the
// remainders then carry).
__device__ __forceinline__ void neq_remainders2x2(const float2 (&f)[9], const float2 (&g)[5],
                                                  const float2 (&m)[4], float t0, float ti,
                                                  unsigned (&r)[14]) {
  float2 e[9], q[5];
  neq_eq2<float2>(m[0], m[1], m[2], m[3], t0, ti, e, q);
  const float2 s = make_float2(kNeqScale, kNeqScale);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float2 v = __fmul2_rn(nq_sub(f[i], e[i]), s);
    const __half2 h = __floats2half2_rn(v.x, v.y);
    r[i] = *reinterpret_cast<const unsigned*>(&h);
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const float2 v = __fmul2_rn(nq_sub(g[i], q[i]), s);
    const __half2 h = __floats2half2_rn(v.x, v.y);
    r[9 + i] = *reinterpret_cast<const unsigned*>(&h);
  }
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
