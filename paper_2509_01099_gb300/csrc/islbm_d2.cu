// 2-D kernels: D2Q9 flow + D2Q5 temperature populations (Sec. 2.1 - 2.3).
//
// Storage: one plane per population, [q][y][x] with a padded x pitch; planes
// 0..8 hold the flow populations, 9..13 the temperature populations, in the
// velocity order
//   D2Q9: (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
//   D2Q5: (0,0) (1,0) (0,1) (-1,0) (0,-1).
// The stored state of time t is the post-collision deviation f_i^+ - w_i
// (g_i^+, the temperature populations carrying T - T_s with T_s the mean wall
// temperature).  One step therefore pulls the post-collision values
// through the virtual streaming + quadratic interpolation (Sec. 2.2) or the
// wall rules (Sec. 2.3), forms the macroscopic moments and collides (Sec. 2.1),
// which is the paper's collide -> stream -> interpolate cycle with the state
// stored after the collision instead of before it.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <vector>

#include "islbm_internal.h"
#include "islbm_lanes.cuh"
#include "islbm_store.cuh"
#include "islbm_tma.cuh"

namespace islbm {
namespace {

template <typename R>
struct P2 {
  int nx, ny, pitch;
  int y0, y1;           // rows the step computes: [y0, y1) (all rows unless a slab is set)
  long long plane;
  const int* bx[2];
  const R* wx[2];
  const int* by[2];
  const R* wy[2];
  const float4* px[2];  // packed FP32 tables of the tiled kernel
  const float4* py[2];
  // The temperature populations carry T - T_s (T_s: mean wall temperature);
  // the buoyancy force is rho g beta (T - T_ref) = rho g beta (T - T_s + Fb).
  R gbeta, s_e, s_eps, s_q, s_nu, q_j, q_e, q_nu, a_T;
  R Ts, Fb;             // T_s and T_s - T_ref
  R abb_hot, abb_cold;  // omega (T_w - T_s) of the anti-bounce-back rule
  unsigned step;        // step counter (seeds the stochastic rounding of 16-bit stores)
};

// Rest weights w_i of the D2Q9 populations.
template <typename R>
__device__ __forceinline__ R wrest(int i) {
  return i == 0 ? R(4.0 / 9.0) : (i < 5 ? R(1.0 / 9.0) : R(1.0 / 36.0));
}

// Rest weights (t_0, t_i) of the D2Q5 temperature equilibrium, (1 - a_T)/5 and
// (4 + a_T)/20.
__device__ __forceinline__ void trest(float aT, float& t0, float& ti) {
  t0 = (1.f - aT) * 0.2f;
  ti = (4.f + aT) * 0.05f;
}

// The 14 stored deviations of one node (flow d_i = f_i - w_i, temperature
// g_i), read or written as a whole: population by population, or for the
// non-equilibrium form through its moments (islbm_store.cuh).
template <typename S>
struct NodeIO {
  using R = typename Store<S>::R;
  static __device__ __forceinline__ void load(const S* __restrict__ s, size_t idx, long long P,
                                              float, R (&f)[9], R (&g)[5]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = Store<S>::ld(s + i * P + idx);
#pragma unroll
    for (int i = 0; i < 5; ++i) g[i] = Store<S>::ld(s + (9 + i) * P + idx);
  }
  static __device__ __forceinline__ void store(S* __restrict__ s, size_t idx, long long P, float,
                                               const R (&f)[9], const R (&g)[5]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) Store<S>::st(s + i * P + idx, f[i]);
#pragma unroll
    for (int i = 0; i < 5; ++i) Store<S>::st(s + (9 + i) * P + idx, g[i]);
  }
};

template <>
struct NodeIO<Neq16> {
  static __device__ __forceinline__ void load(const Neq16* __restrict__ s, size_t idx,
                                              long long P, float aT, float (&f)[9],
                                              float (&g)[5]) {
    const unsigned short* h = reinterpret_cast<const unsigned short*>(s);
    const float* m = neq_moments(s, P);
    unsigned short r[14];
#pragma unroll
    for (int i = 0; i < 14; ++i) r[i] = __ldg(h + i * P + idx);
    float t0, ti;
    trest(aT, t0, ti);
    neq_decode2(__ldg(m + idx), __ldg(m + P + idx), __ldg(m + 2 * P + idx),
                __ldg(m + 3 * P + idx), r, t0, ti, f, g);
  }
  static __device__ __forceinline__ void store(Neq16* __restrict__ s, size_t idx, long long P,
                                               float aT, const float (&f)[9],
                                               const float (&g)[5]) {
    float t0, ti;
    trest(aT, t0, ti);
    float m[4];
    unsigned short r[14];
    neq_encode2(f, g, t0, ti, m, r);
    unsigned short* h = reinterpret_cast<unsigned short*>(s);
    float* mm = neq_moments(s, P);
#pragma unroll
    for (int i = 0; i < 14; ++i) h[i * P + idx] = r[i];
#pragma unroll
    for (int k = 0; k < 4; ++k) mm[k * P + idx] = m[k];
  }
};

// MRT collision in deviation form (Sec. 2.1), of one node (L = R) or of two
// nodes at once (L = float2, R = float: paired FP32 instructions).
//   m = M f with the Lallemand-Luo rows (rho, e, eps, jx, qx, jy, qy, pxx, pxy);
//   m+ = m - S (m - m_eq) + (I - S/2) M F~ with the printed m_eq and M F~;
//   f+ = f + M^-1 (m+ - m), M^-1 = M^T diag(1/|row_k|^2).
//   g: n = N g with rows (T, jx, jy, -4+5|c|^2, cx^2-cy^2), n+ = n - Q (n - n_eq).
// The buoyancy F = rho g beta (T - T_ref) acts along +y; u = (sum e f + F/2)/rho.
// The populations carry T - T_s, which is also the temperature of the
// equilibrium fluxes u T and of a_T T.
// Returns rho, u and T of the pre-collision state, and in m_o the moments of
// the post-collision state: drho, jx, jy + F_y, T - T_s.
template <typename L, typename R>
__device__ __forceinline__ void collide_m(L (&f)[9], L (&g)[5], const P2<R>& p, L& rho_o,
                                          L& ux_o, L& uy_o, L& T_o, L (&m_o)[4]) {
  using K = Lanes<L>;
  auto c = [](double v) { return K::bc((typename K::S)v); };
  // pre-collision moments
  const L d13 = lsub(f[1], f[3]), d56 = lsub(f[5], f[6]), d87 = lsub(f[8], f[7]);
  const L d24 = lsub(f[2], f[4]), p56 = ladd(f[5], f[6]), p78 = ladd(f[7], f[8]);
  const L drho = ladd(ladd(ladd(ladd(f[0], f[1]), ladd(f[2], f[3])),
                           ladd(ladd(f[4], f[5]), ladd(f[6], f[7]))), f[8]);
  const L rho = ladd(c(1), drho);
  const L jx = ladd(ladd(d13, d56), d87);
  const L jy = lsub(ladd(d24, p56), p78);
  const L Tr = ladd(ladd(ladd(g[0], g[1]), ladd(g[2], g[3])), g[4]);  // T - T_s
  const L Fy = lmul(lmul(rho, K::bc(p.gbeta)), ladd(Tr, K::bc(p.Fb)));
  const L inv = lrcp(rho);
  const L ux = lmul(jx, inv);
  const L uy = lmul(lfma(c(0.5), Fy, jy), inv);
  const L ux2 = lmul(ux, ux), uy2 = lmul(uy, uy);
  const L rusq = lmul(rho, ladd(ux2, uy2));
  const L uF = lmul(uy, Fy);

  const L sax = ladd(ladd(f[1], f[2]), ladd(f[3], f[4]));
  const L sdg = ladd(p56, p78);
  const L m1 = lfma(c(2), sdg, lsub(lmul(c(-4), f[0]), sax));
  const L m2 = lfma(c(-2), sax, lfma(c(4), f[0], sdg));
  const L m4 = lfma(c(-2), d13, ladd(d56, d87));
  const L m6 = lfma(c(-2), d24, lsub(p56, p78));
  const L m7 = lsub(ladd(f[1], f[3]), ladd(f[2], f[4]));
  const L m8 = lsub(ladd(f[5], f[7]), ladd(f[6], f[8]));

  // moment increments; the deviation form moves M w = (1,-2,1,0,...) into m_eq
  const R he = R(1) - R(0.5) * p.s_e, heps = R(1) - R(0.5) * p.s_eps;
  const R hq = R(1) - R(0.5) * p.s_q, hnu = R(1) - R(0.5) * p.s_nu;
  const L dm1 = lfma(K::bc(-p.s_e), lfma(c(-3), rusq, lfma(c(2), drho, m1)),
                     lmul(K::bc(R(6) * he), uF));
  const L dm2 = lfma(K::bc(-p.s_eps), lfma(c(3), rusq, lsub(m2, drho)),
                     lmul(K::bc(R(-6) * heps), uF));
  const L dm4 = lmul(K::bc(-p.s_q), lfma(rho, ux, m4));
  const L dm5 = Fy;  // j_y gains exactly F_y (independent of s_j)
  const L dm6 = lfma(K::bc(-p.s_q), lfma(rho, uy, m6), lmul(K::bc(-hq), Fy));
  const L dm7 = lfma(K::bc(-p.s_nu), lfma(rho, lsub(uy2, ux2), m7),
                     lmul(K::bc(R(-2) * hnu), uF));
  const L dm8 = lfma(K::bc(-p.s_nu), lsub(m8, lmul(lmul(rho, ux), uy)),
                     lmul(K::bc(hnu), lmul(ux, Fy)));

  // f+ = f + M^-1 dm
  const L a1 = lmul(dm1, c(1.0 / 36.0)), a2 = lmul(dm2, c(1.0 / 36.0));
  const L a4 = lmul(dm4, c(1.0 / 12.0)), a5 = lmul(dm5, c(1.0 / 6.0));
  const L a6 = lmul(dm6, c(1.0 / 12.0)), a7 = lmul(dm7, c(0.25)), a8 = lmul(dm8, c(0.25));
  const L cax = lsub(lmul(c(-2), a2), a1);   // -a1 - 2 a2
  const L cdg = lfma(c(2), a1, a2);          // 2 a1 + a2
  f[0] = lfma(c(4), lsub(a2, a1), f[0]);
  const L t13 = ladd(cax, a7);
  f[1] = ladd(f[1], lfma(c(-2), a4, t13));
  f[3] = ladd(f[3], lfma(c(2), a4, t13));
  const L t24 = lsub(cax, a7), v24 = lfma(c(-2), a6, a5);   // a5 - 2 a6
  f[2] = ladd(f[2], ladd(t24, v24));
  f[4] = ladd(f[4], lsub(t24, v24));
  const L w56 = ladd(a5, a6), p48 = ladd(a4, a8), m48 = lsub(a4, a8);
  const L cp = ladd(cdg, w56), cm = lsub(cdg, w56);
  f[5] = ladd(f[5], ladd(cp, p48));
  f[6] = ladd(f[6], lsub(cp, p48));
  f[7] = ladd(f[7], lsub(cm, m48));
  f[8] = ladd(f[8], ladd(cm, m48));

  const L n1 = lsub(g[1], g[3]), n2 = lsub(g[2], g[4]);
  const L n3 = lfma(c(-4), g[0], ladd(ladd(g[1], g[2]), ladd(g[3], g[4])));
  const L n4 = lsub(ladd(g[1], g[3]), ladd(g[2], g[4]));
  const L b1 = lmul(K::bc(R(-0.5) * p.q_j), lsub(n1, lmul(ux, Tr)));
  const L b2 = lmul(K::bc(R(-0.5) * p.q_j), lsub(n2, lmul(uy, Tr)));
  const L b3 = lmul(K::bc(R(-0.05) * p.q_e), lsub(n3, lmul(K::bc(p.a_T), Tr)));
  const L b4 = lmul(K::bc(R(-0.25) * p.q_nu), n4);
  g[0] = lfma(c(-4), b3, g[0]);
  const L s34 = ladd(b3, b4), d34 = lsub(b3, b4);
  g[1] = ladd(g[1], ladd(b1, s34));
  g[3] = ladd(g[3], lsub(s34, b1));
  g[2] = ladd(g[2], ladd(b2, d34));
  g[4] = ladd(g[4], lsub(d34, b2));

  rho_o = rho;
  ux_o = ux;
  uy_o = uy;
  T_o = Tr;
  m_o[0] = drho;
  m_o[1] = jx;
  m_o[2] = ladd(jy, Fy);
  m_o[3] = Tr;
}

template <typename L, typename R>
__device__ __forceinline__ void collide(L (&f)[9], L (&g)[5], const P2<R>& p, L& rho_o,
                                        L& ux_o, L& uy_o, L& T_o) {
  L m[4];
  collide_m(f, g, p, rho_o, ux_o, uy_o, T_o, m);
}

// Interpolated pull of one population (Sec. 2.2): the value at node (x, y) is
// the tensor-product quadratic Lagrange interpolant of the post-collision
// values at the departure point (X_x - cx, Y_y - cy).  On the uniform mesh the
// interpolant is a pure shift.
template <typename S, typename R, int CX, int CY, bool UNI>
__device__ __forceinline__ R pull(const S* __restrict__ pl, int x, int y, const P2<R>& p) {
  using St = Store<S>;
  if (CX == 0 && CY == 0) return St::ld(pl + (size_t)y * p.pitch + x);
  if (UNI) return St::ld(pl + (size_t)(y - CY) * p.pitch + (x - CX));
  if (CY == 0) {
    constexpr int k = CX > 0 ? 0 : 1;
    const int b = __ldg(p.bx[k] + x);
    const R* w = p.wx[k] + 3 * x;
    const S* r = pl + (size_t)y * p.pitch + b;
    return lin3(__ldg(w), __ldg(w + 1), __ldg(w + 2), St::ld(r), St::ld(r + 1), St::ld(r + 2));
  }
  if (CX == 0) {
    constexpr int k = CY > 0 ? 0 : 1;
    const int b = __ldg(p.by[k] + y);
    const R* w = p.wy[k] + 3 * y;
    const S* r = pl + (size_t)b * p.pitch + x;
    return lin3(__ldg(w), __ldg(w + 1), __ldg(w + 2), St::ld(r), St::ld(r + p.pitch),
                St::ld(r + 2 * (size_t)p.pitch));
  }
  constexpr int kx = CX > 0 ? 0 : 1;
  constexpr int ky = CY > 0 ? 0 : 1;
  const int bx = __ldg(p.bx[kx] + x);
  const int by = __ldg(p.by[ky] + y);
  const R* wx = p.wx[kx] + 3 * x;
  const R* wy = p.wy[ky] + 3 * y;
  const R wx0 = __ldg(wx), wx1 = __ldg(wx + 1), wx2 = __ldg(wx + 2);
  R acc = R(0);
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const S* r = pl + (size_t)(by + l) * p.pitch + bx;
    acc = lfma(__ldg(wy + l), lin3(wx0, wx1, wx2, St::ld(r), St::ld(r + 1), St::ld(r + 2)), acc);
  }
  return acc;
}

template <typename S, bool UNI>
__global__ void __launch_bounds__(256)
    k_step(const S* __restrict__ fin, S* __restrict__ fout, P2<typename Store<S>::R> p) {
  using R = typename Store<S>::R;
  using St = Store<S>;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = p.y0 + (int)(blockIdx.y * blockDim.y + threadIdx.y);
  if (x >= p.nx || y >= p.y1) return;
  const size_t idx = (size_t)y * p.pitch + x;
  const long long P = p.plane;
  // departure point behind the west / east / south / north wall
  const bool wW = (x == 0), wE = (x == p.nx - 1), wS = (y == 0), wN = (y == p.ny - 1);
  R f[9], g[5];
  // flow: half-way bounce-back f_i = f_ibar^+ at the wall (Sec. 2.3)
  f[0] = St::ld(fin + idx);
  f[1] = wW ? St::ld(fin + 3 * P + idx) : pull<S, R, 1, 0, UNI>(fin + 1 * P, x, y, p);
  f[2] = wS ? St::ld(fin + 4 * P + idx) : pull<S, R, 0, 1, UNI>(fin + 2 * P, x, y, p);
  f[3] = wE ? St::ld(fin + 1 * P + idx) : pull<S, R, -1, 0, UNI>(fin + 3 * P, x, y, p);
  f[4] = wN ? St::ld(fin + 2 * P + idx) : pull<S, R, 0, -1, UNI>(fin + 4 * P, x, y, p);
  f[5] = (wW || wS) ? St::ld(fin + 7 * P + idx) : pull<S, R, 1, 1, UNI>(fin + 5 * P, x, y, p);
  f[6] = (wE || wS) ? St::ld(fin + 8 * P + idx) : pull<S, R, -1, 1, UNI>(fin + 6 * P, x, y, p);
  f[7] = (wE || wN) ? St::ld(fin + 5 * P + idx) : pull<S, R, -1, -1, UNI>(fin + 7 * P, x, y, p);
  f[8] = (wW || wN) ? St::ld(fin + 6 * P + idx) : pull<S, R, 1, -1, UNI>(fin + 8 * P, x, y, p);
  // temperature: anti-bounce-back on the isothermal x-walls, bounce-back on the
  // adiabatic y-walls (Sec. 2.3)
  const S* gin = fin + 9 * P;
  g[0] = St::ld(gin + idx);
  g[1] = wW ? p.abb_hot - St::ld(gin + 3 * P + idx) : pull<S, R, 1, 0, UNI>(gin + 1 * P, x, y, p);
  g[2] = wS ? St::ld(gin + 4 * P + idx) : pull<S, R, 0, 1, UNI>(gin + 2 * P, x, y, p);
  g[3] = wE ? p.abb_cold - St::ld(gin + 1 * P + idx) : pull<S, R, -1, 0, UNI>(gin + 3 * P, x, y, p);
  g[4] = wN ? St::ld(gin + 2 * P + idx) : pull<S, R, 0, -1, UNI>(gin + 4 * P, x, y, p);

  R rho, ux, uy, T;
  collide(f, g, p, rho, ux, uy, T);
  unsigned r = sr_seed(idx, p.step);
#pragma unroll
  for (int i = 0; i < 9; ++i) St::st_sr(fout + i * P + idx, f[i], sr_next(r));
#pragma unroll
  for (int i = 0; i < 5; ++i) St::st_sr(fout + (9 + i) * P + idx, g[i], sr_next(r));
}

// Equilibrium (Sec. 2.1) of given fields, then the collision.  The flow
// equilibrium is the second-order Hermite form w_i rho (1 + 3 e.u + 9/2 (e.u)^2
// - 3/2 u^2), which has exactly the printed moments; the temperature
// equilibrium is N^-1 n_eq: g_0 = t_0 T, g_i = t_i T + (e_i.u) T / 2 with
// t_0 = (1 - a_T)/5, t_i = (4 + a_T)/20.
template <typename S>
__global__ void k_init_fields(S* __restrict__ fout, P2<typename Store<S>::R> p,
                              const double* __restrict__ rho_in, const double* __restrict__ T_in,
                              const double* __restrict__ u_in, const double* __restrict__ v_in) {
  using R = typename Store<S>::R;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const size_t node = (size_t)y * p.nx + x;
  const R rho = rho_in ? R(rho_in[node]) : R(1);
  const R T = R(T_in[node] - (double)p.Ts);   // T - T_s
  const R ux = u_in ? R(u_in[node]) : R(0);
  const R uy = v_in ? R(v_in[node]) : R(0);
  const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const R usq = ux * ux + uy * uy;
  R f[9], g[5];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const R eu = R(ex[i]) * ux + R(ey[i]) * uy;
    f[i] = wrest<R>(i) * (rho * (R(1) + R(3) * eu + R(4.5) * eu * eu - R(1.5) * usq) - R(1));
  }
  const R t0 = (R(1) - p.a_T) * R(0.2), ti = (R(4) + p.a_T) * R(0.05);
  const R Tr = T;
  g[0] = t0 * Tr;
#pragma unroll
  for (int i = 1; i < 5; ++i) g[i] = ti * Tr + R(0.5) * (R(ex[i]) * ux + R(ey[i]) * uy) * T;
  R r_, a_, b_, c_;
  collide(f, g, p, r_, a_, b_, c_);
  NodeIO<S>::store(fout, (size_t)y * p.pitch + x, p.plane, (float)p.a_T, f, g);
}

// Full FP64 pre-collision populations ([q][node]) -> deviations -> collision.
template <typename S>
__global__ void k_init_pops(S* __restrict__ fout, P2<typename Store<S>::R> p,
                            const double* __restrict__ fin, const double* __restrict__ gin) {
  using R = typename Store<S>::R;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const size_t nodes = (size_t)p.nx * p.ny;
  const size_t node = (size_t)y * p.nx + x;
  R f[9], g[5];
#pragma unroll
  for (int i = 0; i < 9; ++i) f[i] = R(fin[i * nodes + node] - wrest<double>(i));
#pragma unroll
  for (int i = 0; i < 5; ++i) g[i] = R(gin[i * nodes + node]);
  R r_, a_, b_, c_;
  collide(f, g, p, r_, a_, b_, c_);
  NodeIO<S>::store(fout, (size_t)y * p.pitch + x, p.plane, (float)p.a_T, f, g);
}

// Macroscopic state of a node from the stored post-collision deviations, in
// FP64: rho and T are collision invariants; the collision adds F to the
// momentum, so u = (sum e f^+ - F/2)/rho.
struct NodeState {
  double rho, ux, uy, T;
};

template <typename S>
__device__ __forceinline__ NodeState node_state(const S* __restrict__ s, size_t idx,
                                                long long P, float aT, double gbeta, double Ts,
                                                double Tref) {
  typename Store<S>::R fr[9], gr[5];
  NodeIO<S>::load(s, idx, P, aT, fr, gr);
  double f[9], g[5];
#pragma unroll
  for (int i = 0; i < 9; ++i) f[i] = (double)fr[i];
#pragma unroll
  for (int i = 0; i < 5; ++i) g[i] = (double)gr[i];
  NodeState n;
  const double drho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
  n.rho = 1.0 + drho;
  const double jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
  const double jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
  const double Tr = (g[0] + g[1]) + (g[2] + g[3]) + g[4];
  n.T = Tr + Ts;
  const double Fy = n.rho * gbeta * (n.T - Tref);
  n.ux = jx / n.rho;
  n.uy = (jy - 0.5 * Fy) / n.rho;
  return n;
}

template <typename S>
__global__ void k_fields(const S* __restrict__ s, P2<typename Store<S>::R> p, double gbeta,
                         double Ts, double Tref, double* rho, double* T, double* u, double* v) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const NodeState n = node_state(s, (size_t)y * p.pitch + x, p.plane, (float)p.a_T, gbeta, Ts,
                                 Tref);
  const size_t node = (size_t)y * p.nx + x;
  if (rho) rho[node] = n.rho;
  if (T) T[node] = n.T;
  if (u) u[node] = n.ux;
  if (v) v[node] = n.uy;
}

template <typename S>
__global__ void k_pops(const S* __restrict__ s, P2<typename Store<S>::R> p, double* f,
                       double* g) {
  using R = typename Store<S>::R;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const size_t nodes = (size_t)p.nx * p.ny, node = (size_t)y * p.nx + x;
  R fr[9], gr[5];
  NodeIO<S>::load(s, (size_t)y * p.pitch + x, p.plane, (float)p.a_T, fr, gr);
#pragma unroll
  for (int i = 0; i < 9; ++i) f[i * nodes + node] = (double)fr[i] + wrest<double>(i);
#pragma unroll
  for (int i = 0; i < 5; ++i) g[i * nodes + node] = (double)gr[i];
}

// Population sums and velocity of one node in the compute type of the storage
// (FP32 for FP32 / 16-bit storage, FP64 for FP64 storage): the reductions
// accumulate in FP64, but the node's own arithmetic needs no more precision
// than the state it reads (FP64 arithmetic runs at a small fraction of the
// FP32 rate on this GPU).  drho, the density's deviation from 1, keeps the
// mass accumulation free of the rounding of 1 + drho.
template <typename R>
struct NodeC {
  R drho, ux, uy, T;
};

template <typename S>
__device__ __forceinline__ NodeC<typename Store<S>::R> node_state_c(
    const S* __restrict__ s, size_t idx, long long P, float aT, typename Store<S>::R gbeta,
    typename Store<S>::R Ts, typename Store<S>::R Tref) {
  using R = typename Store<S>::R;
  R f[9], g[5];
  NodeIO<S>::load(s, idx, P, aT, f, g);
  NodeC<R> n;
  n.drho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
  const R rho = R(1) + n.drho;
  const R jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
  const R jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
  const R Tr = (g[0] + g[1]) + (g[2] + g[3]) + g[4];
  n.T = Tr + Ts;
  const R Fy = rho * gbeta * (n.T - Tref);
  n.ux = jx / rho;
  n.uy = (jy - R(0.5) * Fy) / rho;
  return n;
}

// Reductions of the current state (Sec. 3, Eq. (17), Eq. (18)): per-block FP64
// partial sums of the midpoint-rule weighted contributions of every node; the
// nodes in the planes next to the isothermal walls and on the centre line add
// the temperature sums from which the host finishes Eq. (17) and Nu_middle.
// A block takes whole rows (of the slab when one is set), its threads the
// columns.
template <typename S>
__global__ void __launch_bounds__(256)
    k_reduce(const S* __restrict__ s, P2<typename Store<S>::R> p, double gbeta, double Ts,
             double T0,
             const double* __restrict__ Wx, const double* __restrict__ Wy, double* partial) {
  using R = typename Store<S>::R;
  double acc[RED_COUNT];
#pragma unroll
  for (int k = 0; k < RED_COUNT; ++k) acc[k] = 0.0;
  const int mL = (p.nx % 2 == 0) ? p.nx / 2 - 1 : (p.nx - 1) / 2 - 1;  // left column of the centre pair
  const int mR = (p.nx % 2 == 0) ? p.nx / 2 : (p.nx + 1) / 2;           // right column
  const int mC = (p.nx % 2 == 0) ? -1 : (p.nx - 1) / 2;                  // centre column (odd n)
  const R gb = R(gbeta), ts = R(Ts), t0 = R(T0);
  for (int y = p.y0 + (int)blockIdx.x; y < p.y1; y += (int)gridDim.x) {
    const double wy = Wy[y];
    for (int x = threadIdx.x; x < p.nx; x += blockDim.x) {
      const NodeC<R> n = node_state_c(s, (size_t)y * p.pitch + x, p.plane, (float)p.a_T, gb, ts, t0);
      const double W = Wx[x] * wy;
      const R u2 = n.ux * n.ux + n.uy * n.uy;
      const R sp = sqrt(u2);
      const R uT = n.ux * (n.T - t0);
      acc[RED_MASS] += W * (1.0 + (double)n.drho);
      acc[RED_UT] += W * (double)uT;
      acc[RED_SPEED] += W * (double)sp;
      acc[RED_UV2] += W * (double)u2;
      acc[RED_U2] += W * (double)u2;
      const double T = (double)n.T;
      if (x == 0) acc[RED_HOT1] += wy * T;
      if (x == 1) acc[RED_HOT2] += wy * T;
      if (x == p.nx - 1) acc[RED_COLD1] += wy * T;
      if (x == p.nx - 2) acc[RED_COLD2] += wy * T;
      if (x == mL) acc[RED_MIDTL] += wy * T;
      if (x == mR) acc[RED_MIDTR] += wy * T;
      if (mC < 0 && (x == mL || x == mR)) acc[RED_MIDCONV] += 0.5 * wy * (double)uT;
      if (x == mC) acc[RED_MIDCONV] += wy * (double)uT;
      const bool finite = isfinite(n.drho) && isfinite(n.ux) && isfinite(n.uy) && isfinite(n.T);
      if (!finite) acc[RED_NONFINITE] += 1.0;
      acc[RED_MAXSPEED] = fmax(acc[RED_MAXSPEED], finite ? (double)sp : 0.0);
    }
  }
  __shared__ double sh[8][RED_COUNT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < RED_COUNT; ++k) {
    const double v = (k == RED_MAXSPEED) ? warp_max(acc[k]) : warp_sum(acc[k]);
    if (lane == 0) sh[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < RED_COUNT) {
    const int k = threadIdx.x;
    double v = sh[0][k];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      v = (k == RED_MAXSPEED) ? fmax(v, sh[w][k]) : v + sh[w][k];
    partial[(size_t)blockIdx.x * RED_STRIDE + k] = v;
  }
}

// Steady-state criterion (Sec. 3): sum |u(t) - u(t0)|_2, sum |u(t0)|_2,
// sum |T*(t) - T*(t0)|, sum |T*(t0)| over the nodes, against the snapshot of
// (u, v, T*) taken at the previous check, which is then replaced by the
// current fields.  Partial sums per block in slots 0..3 (the others zero).
// Without a snapshot (have_snap = 0) the old values count as zero and the
// buffer is only written.
template <typename S>
__global__ void __launch_bounds__(256)
    k_steady(const S* __restrict__ s, P2<typename Store<S>::R> p, double gbeta, double Ts,
             double T0, double dT, int have_snap, double* snap, double* partial) {
  double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  const long long nodes = (long long)p.nx * p.ny;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nodes;
       k += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(k / p.nx), x = (int)(k - (long long)y * p.nx);
    const NodeState n = node_state(s, (size_t)y * p.pitch + x, p.plane, (float)p.a_T, gbeta, Ts,
                                   T0);
    const double Tn = (n.T - T0) / dT;
    double ou = 0.0, ov = 0.0, oT = 0.0;
    if (have_snap) {
      ou = snap[k];
      ov = snap[nodes + k];
      oT = snap[2 * nodes + k];
    }
    a0 += sqrt((n.ux - ou) * (n.ux - ou) + (n.uy - ov) * (n.uy - ov));
    a1 += sqrt(ou * ou + ov * ov);
    a2 += fabs(Tn - oT);
    a3 += fabs(oT);
    snap[k] = n.ux;
    snap[nodes + k] = n.uy;
    snap[2 * nodes + k] = Tn;
  }
  __shared__ double sh[8][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  a0 = warp_sum(a0); a1 = warp_sum(a1); a2 = warp_sum(a2); a3 = warp_sum(a3);
  if (lane == 0) { sh[warp][0] = a0; sh[warp][1] = a1; sh[warp][2] = a2; sh[warp][3] = a3; }
  __syncthreads();
  if (threadIdx.x < RED_STRIDE) {
    double v = 0.0;
    if (threadIdx.x < 4)
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[w][threadIdx.x];
    partial[(size_t)blockIdx.x * RED_STRIDE + threadIdx.x] = v;
  }
}

// One warp per slot sums the block partials in a fixed order (deterministic).
__global__ void k_finish(const double* __restrict__ partial, int blocks, double* out) {
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k >= RED_COUNT) return;
  double v = 0.0;
  for (int b = lane; b < blocks; b += 32) {
    const double x = partial[(size_t)b * RED_STRIDE + k];
    v = (k == RED_MAXSPEED) ? fmax(v, x) : v + x;
  }
  v = (k == RED_MAXSPEED) ? warp_max(v) : warp_sum(v);
  if (lane == 0) out[k] = v;
}

template <typename R>
P2<R> make_params(const Solver& s) {
  P2<R> p;
  p.nx = s.n[0];
  p.ny = s.n[1];
  p.y0 = s.row_end > 0 ? s.row_begin : 0;
  p.y1 = s.row_end > 0 ? s.row_end : s.n[1];
  p.pitch = s.pitch;
  p.plane = s.plane;
  for (int k = 0; k < 2; ++k) {
    p.bx[k] = s.dax[0].base[k];
    p.wx[k] = static_cast<const R*>(s.dax[0].w[k]);
    p.by[k] = s.dax[1].base[k];
    p.wy[k] = static_cast<const R*>(s.dax[1].w[k]);
    p.px[k] = s.dax[0].packed[k];
    p.py[k] = s.dax[1].packed[k];
  }
  const Physics& h = s.ph;
  p.gbeta = R(h.gbeta);
  p.Ts = R(h.Ts);
  p.Fb = R(h.Ts - h.T0);
  p.s_e = R(h.s_e);
  p.s_eps = R(h.s_eps);
  p.s_q = R(h.s_q);
  p.s_nu = R(h.s_nu);
  p.q_j = R(h.q_j);
  p.q_e = R(h.q_e);
  p.q_nu = R(h.q_nu);
  p.a_T = R(h.a_T);
  p.abb_hot = R(h.omega * (h.T_hot - h.Ts));
  p.abb_cold = R(h.omega * (h.T_cold - h.Ts));
  p.step = (unsigned)s.time;
  return p;
}

// rows of the step: the slab [row_begin, row_end) when one is set
int step_rows(const Solver& s) { return s.row_end > 0 ? s.row_end - s.row_begin : s.n[1]; }


// ---------------------------------------------------------------------------
// Tiled step (FP32 compute, any 32/16-bit storage, centred stencil).
//
// A CTA owns a 64 x (4R) tile.  All 14 population planes of the tile plus a
// one-node halo (rounded out to a 16-byte chunk in x) are staged in shared
// memory with cp.async, so every global value is fetched once by a coalesced
// 16-byte copy.  Thread (c, rg) owns column c and the R rows rg*R .. rg*R+R-1:
// the quadratic interpolation is applied axis by axis (Sec. 2.2): R+2 rows are
// interpolated in x once and reused by the R outputs of the y pass.  Tiles that
// touch a y-wall take the general per-node path.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n)
               : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}


constexpr int kFixedOrder = INT_MAX;   // k0 of k_step_tma: no tile is claimed
constexpr int kTX = 64;       // tile width
constexpr int kRG = 4;        // row groups per tile
constexpr int kThreads = kTX * kRG;

template <typename S, int R>
struct TileGeom {
  static constexpr int TY = R * kRG;
  static constexpr int HX = 16 / (int)sizeof(S);      // halo columns: one 16-byte chunk
  static constexpr int SW = kTX + 2 * HX;              // staged row width
  static constexpr int SH = TY + 2;                    // staged rows
  static constexpr int CPR = SW / HX;                  // chunks per staged row
  static constexpr int PLANE = SH * SW;                // staged elements per population
  static constexpr size_t smem_bytes() {
    return (size_t)14 * PLANE * sizeof(S) + (size_t)2 * TY * sizeof(float4);
  }
};

// Compute phase of one staged tile: interpolated pull / walls -> collision ->
// store.  `sm` holds the 14 staged planes (rows ry0.., columns x0-HX..).  The
// packed interpolation tables (unused on a uniform mesh) come from `wxp` /
// `wxm`, the x tables of the tile's first column, and `wyp` / `wym`, the y
// tables of its first row (shared or global memory).
// O: the storage type written (S, or Neq16 when S = float holds a decoded tile).
template <typename S, int R, bool UNI, typename O = S>
__device__ __forceinline__ void tile_body(const S* __restrict__ sm, const float4* wxp,
                                          const float4* wxm, const float4* wyp,
                                          const float4* wym, int x0, int y0, int ry0,
                                          O* __restrict__ fout, const P2<float>& p) {
  using G = TileGeom<S, R>;
  constexpr int TY = G::TY, HX = G::HX, SW = G::SW;
  const int cx0 = x0 - HX;
  const int c = threadIdx.x % kTX, rg = threadIdx.x / kTX;
  const int x = x0 + c;
  if (x >= p.nx) return;
  const int col = x - cx0;
  const bool wW = (x == 0), wE = (x == p.nx - 1);
  float4 tp = make_float4(0.f, 0.f, 0.f, 0.f), tm = tp;
  int bp = col - 1, bm = col - 1;
  if (!UNI) {
    tp = wxp[c];
    tm = wxm[c];
    bp = __float_as_int(tp.w) - cx0;
    bm = __float_as_int(tm.w) - cx0;
  }
  auto rd = [&](int pl, int row, int cl) -> float {
    if (!(ISLBM_IN_WINDOW(row, G::SH) && ISLBM_IN_WINDOW(cl, SW))) row = cl = 0;
    return to_f(sm[(size_t)pl * G::PLANE + row * SW + cl]);
  };
  // x-interpolated value of plane pl in staged row `row` for direction cx
  auto xi = [&](int pl, int row, int cx) -> float {
    if (UNI) return rd(pl, row, col - cx);
    const float4 t = cx > 0 ? tp : tm;
    const int b = cx > 0 ? bp : bm;
    return dot3(t, rd(pl, row, b), rd(pl, row, b + 1), rd(pl, row, b + 2));
  };

  const int yr0 = y0 + rg * R;            // first output row of the thread
  const int lr0 = yr0 - ry0;              // its staged row
  const bool fast = (y0 >= 1) && (y0 + TY <= p.ny - 1);
  float f[9][R], g[5][R];

  if (fast) {
    // rows yr0-1 .. yr0+R are staged rows lr0-1 .. lr0+R
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int lr = lr0 + m;
      f[0][m] = rd(0, lr, col);
      g[0][m] = rd(9, lr, col);
      f[1][m] = wW ? rd(3, lr, col) : xi(1, lr, +1);
      f[3][m] = wE ? rd(1, lr, col) : xi(3, lr, -1);
      g[1][m] = wW ? p.abb_hot - rd(12, lr, col) : xi(10, lr, +1);
      g[3][m] = wE ? p.abb_cold - rd(10, lr, col) : xi(12, lr, -1);
    }
    // planes moving in y: window of R+2 (x-interpolated) rows, then the y pass
    auto ypass = [&](int pl, int cx, int cy, float (&out)[R]) {
      float h[R + 2];
#pragma unroll
      for (int l = 0; l < R + 2; ++l) h[l] = (cx == 0) ? rd(pl, lr0 - 1 + l, col) : xi(pl, lr0 - 1 + l, cx);
#pragma unroll
      for (int m = 0; m < R; ++m) {
        if (UNI) {
          out[m] = h[m + 1 - cy];
        } else {
          const float4 q = (cy > 0 ? wyp : wym)[rg * R + m];
          out[m] = dot3(q, h[m], h[m + 1], h[m + 2]);
        }
      }
    };
    ypass(2, 0, +1, f[2]);
    ypass(4, 0, -1, f[4]);
    ypass(5, +1, +1, f[5]);
    ypass(6, -1, +1, f[6]);
    ypass(7, -1, -1, f[7]);
    ypass(8, +1, -1, f[8]);
    ypass(11, 0, +1, g[2]);
    ypass(13, 0, -1, g[4]);
    // half-way bounce-back where the departure point lies behind an x-wall
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int lr = lr0 + m;
      if (wW) {
        f[5][m] = rd(7, lr, col);
        f[8][m] = rd(6, lr, col);
      }
      if (wE) {
        f[6][m] = rd(8, lr, col);
        f[7][m] = rd(5, lr, col);
      }
    }
  } else {
    // general path: y-walls and clamped stencils, node by node; rows beyond
    // the mesh hold zeros (collided with their pair row, never stored)
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int y = yr0 + m;
      const int lr = y - ry0;
      if (y >= p.y1) {
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i][m] = 0.f;
#pragma unroll
        for (int i = 0; i < 5; ++i) g[i][m] = 0.f;
        continue;
      }
      const bool wS = (y == 0), wN = (y == p.ny - 1);
      float4 qp = make_float4(0.f, 0.f, 0.f, 0.f), qm = qp;
      int brp = 0, brm = 0;
      if (!UNI) {
        qp = wyp[rg * R + m];
        qm = wym[rg * R + m];
        brp = __float_as_int(qp.w) - ry0;
        brm = __float_as_int(qm.w) - ry0;
      }
      auto ypull = [&](int pl, int cx, int cy) -> float {
        if (UNI) return (cx == 0) ? rd(pl, lr - cy, col) : xi(pl, lr - cy, cx);
        const float4 q = cy > 0 ? qp : qm;
        const int br = cy > 0 ? brp : brm;
        if (cx == 0) return dot3(q, rd(pl, br, col), rd(pl, br + 1, col), rd(pl, br + 2, col));
        return dot3(q, xi(pl, br, cx), xi(pl, br + 1, cx), xi(pl, br + 2, cx));
      };
      f[0][m] = rd(0, lr, col);
      g[0][m] = rd(9, lr, col);
      f[1][m] = wW ? rd(3, lr, col) : xi(1, lr, +1);
      f[3][m] = wE ? rd(1, lr, col) : xi(3, lr, -1);
      f[2][m] = wS ? rd(4, lr, col) : ypull(2, 0, +1);
      f[4][m] = wN ? rd(2, lr, col) : ypull(4, 0, -1);
      f[5][m] = (wW || wS) ? rd(7, lr, col) : ypull(5, +1, +1);
      f[6][m] = (wE || wS) ? rd(8, lr, col) : ypull(6, -1, +1);
      f[7][m] = (wE || wN) ? rd(5, lr, col) : ypull(7, -1, -1);
      f[8][m] = (wW || wN) ? rd(6, lr, col) : ypull(8, +1, -1);
      g[1][m] = wW ? p.abb_hot - rd(12, lr, col) : xi(10, lr, +1);
      g[3][m] = wE ? p.abb_cold - rd(10, lr, col) : xi(12, lr, -1);
      g[2][m] = wS ? rd(13, lr, col) : ypull(11, 0, +1);
      g[4][m] = wN ? rd(11, lr, col) : ypull(13, 0, -1);
    }
  }

  // ---- collide and store: rows m, m+1 in one paired collision ----
  static_assert(R % 2 == 0, "rows are collided in pairs");
#pragma unroll
  for (int m = 0; m < R; m += 2) {
    const int y = yr0 + m;
    if (y >= p.y1) break;
    float2 fn[9], gn[5];
#pragma unroll
    for (int i = 0; i < 9; ++i) fn[i] = make_float2(f[i][m], f[i][m + 1]);
#pragma unroll
    for (int i = 0; i < 5; ++i) gn[i] = make_float2(g[i][m], g[i][m + 1]);
    float2 rho, ux, uy, T, mm[4];
    collide_m(fn, gn, p, rho, ux, uy, T, mm);
    const size_t idx = (size_t)y * p.pitch + x;
    if constexpr (is_neq<O>::value) {
      // rows y (low halves) and y + 1 (high halves) encoded together
      float t0, ti;
      trest(p.a_T, t0, ti);
      unsigned rr[14];
      neq_remainders2x2(fn, gn, mm, t0, ti, rr);
      unsigned short* h = reinterpret_cast<unsigned short*>(fout);
      float* mo = neq_moments(fout, p.plane);
#pragma unroll
      for (int i = 0; i < 14; ++i) h[(size_t)i * p.plane + idx] = (unsigned short)(rr[i] & 0xFFFFu);
#pragma unroll
      for (int k = 0; k < 4; ++k) mo[(size_t)k * p.plane + idx] = mm[k].x;
      if (y + 1 < p.y1) {
        const size_t idx1 = idx + p.pitch;
#pragma unroll
        for (int i = 0; i < 14; ++i) h[(size_t)i * p.plane + idx1] = (unsigned short)(rr[i] >> 16);
#pragma unroll
        for (int k = 0; k < 4; ++k) mo[(size_t)k * p.plane + idx1] = mm[k].y;
      }
    } else {
      unsigned r = sr_seed(idx, p.step);
#pragma unroll
      for (int i = 0; i < 9; ++i)
        Store<S>::st_sr(fout + (size_t)i * p.plane + idx, fn[i].x, sr_next(r));
#pragma unroll
      for (int i = 0; i < 5; ++i)
        Store<S>::st_sr(fout + (size_t)(9 + i) * p.plane + idx, gn[i].x, sr_next(r));
      if (y + 1 < p.y1) {
        const size_t idx1 = idx + p.pitch;
        unsigned r1 = sr_seed(idx1, p.step);
#pragma unroll
        for (int i = 0; i < 9; ++i)
          Store<S>::st_sr(fout + (size_t)i * p.plane + idx1, fn[i].y, sr_next(r1));
#pragma unroll
        for (int i = 0; i < 5; ++i)
          Store<S>::st_sr(fout + (size_t)(9 + i) * p.plane + idx1, gn[i].y, sr_next(r1));
      }
    }
  }
}

template <typename S, int R, bool UNI>
__global__ void __launch_bounds__(kThreads, 2)
    k_step_tiled(const S* __restrict__ fin, S* __restrict__ fout, P2<float> p) {
  using G = TileGeom<S, R>;
  constexpr int TY = G::TY, HX = G::HX, SW = G::SW, SH = G::SH, CPR = G::CPR;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  S* sm = reinterpret_cast<S*>(smem_raw);
  float4* wyt = reinterpret_cast<float4*>(smem_raw + (size_t)14 * G::PLANE * sizeof(S));

  const int x0 = blockIdx.x * kTX, y0 = p.y0 + (int)blockIdx.y * TY;
  const int cx0 = x0 - HX;
  const int ry0 = max(0, min(y0 - 1, p.ny - 3));
  // ---- stage the tile + halo of every plane ----
  constexpr int CPP = SH * CPR;
  for (int k = threadIdx.x; k < 14 * CPP; k += kThreads) {
    const int pl = k / CPP;
    const int r = k - pl * CPP;
    const int row = r / CPR;
    const int ch = r - row * CPR;
    const int gy = ry0 + row, gx = cx0 + ch * HX;
    const bool ok = gy < p.ny && gx >= 0 && gx + HX <= p.pitch;
    const S* src = ok ? fin + (size_t)pl * p.plane + (size_t)gy * p.pitch + gx : fin;
    cp_async16(sm + (size_t)pl * G::PLANE + row * SW + ch * HX, src, ok);
  }
  if (!UNI && threadIdx.x < 2 * TY) {
    const int k = threadIdx.x / TY, yy = y0 + threadIdx.x % TY;
    wyt[threadIdx.x] = yy < p.ny ? __ldg(p.py[k] + yy) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  cp_async_wait_all();
  __syncthreads();
  tile_body<S, R, UNI>(sm, p.px[0] + x0, p.px[1] + x0, wyt, wyt + TY, x0, y0, ry0, fout, p);
}

// ---------------------------------------------------------------------------
// Persistent TMA-pipelined step.  One CTA per SM slot; a single thread issues,
// for each tile, one 3-D TMA copy (box SW x SH x 14 planes, out-of-range parts
// zero-filled) plus four bulk copies of the tile's packed interpolation tables
// (x tables of its columns, y tables of its rows) into one of STAGES
// shared-memory stages, all tracked by one mbarrier, so the copies of the next
// tiles are in flight while the current tile is computed and the compute
// reads nothing but shared memory.
//
// Tile order.  The tile of a CTA's k-th stage use is blockIdx.x + k * gridDim.x
// for k < k0 (k0 >= STAGES, and k0 * gridDim.x <= the tile count, so these
// tiles all exist).  From use k0 on, each tile is claimed from a device counter
// STAGES uses ahead of its use (tiles k0 * gridDim.x and up), so SMs that run
// ahead take more tiles: with k0 = STAGES on large meshes, where a CTA walks
// hundreds of tiles, the claimed order keeps the tiles in flight a compact band
// of rows (the fixed stride lets the CTAs drift apart); with k0 a tile or two
// short of the CTA's share on small meshes, only the last tiles are claimed and
// even out the SMs' finishing times.  k0 = INT_MAX: the fixed stride
// throughout.  The last CTA to finish resets the counter.  A tile index at or
// beyond the tile count ends the CTA's walk.
//
// Every mbarrier wait is bounded: on timeout the CTA records an error flag,
// drains its outstanding copies (again bounded) and leaves through the same
// exit, so the counter is still reset.
//
// sched[0]: error flag; sched[1]: tiles claimed; sched[2]: CTAs finished
// (sched[1], sched[2] are zero between launches).
// ---------------------------------------------------------------------------

// Shared-memory stage of k_step_tma: the staged planes, then the tables
// (x+, x- of kTX columns; y+, y- of TY rows; float4 each).
template <typename S, int R>
struct TmaStage {
  using Staged = S;                                    // type of the planes the compute reads
  static constexpr unsigned PLANES = (unsigned)(14 * TileGeom<S, R>::PLANE * sizeof(S));
  static constexpr unsigned LOADED = PLANES;           // bytes the copies bring
  static constexpr unsigned TABLES = (unsigned)((2 * kTX + 2 * TileGeom<S, R>::TY) * 16);
  static constexpr unsigned BYTES = PLANES + TABLES;
  static constexpr unsigned EXTRA = 0;                 // shared memory behind the ring
  static_assert(PLANES % 128 == 0 && BYTES % 128 == 0, "stages keep the TMA's 128-byte alignment");
};

// Non-equilibrium storage: the copies bring the FP16 remainders (box of
// kTX + 16 columns from x0 - 8, one 16-byte chunk of halo each side) and the
// FP32 moments (kTX + 8 columns from x0 - 4) into the stage; the decode writes
// the FP32 deviations, in the layout of TileGeom<float, R> that tile_body
// reads, into one buffer of DECODED bytes behind the ring (EXTRA).
template <int R>
struct TmaStage<Neq16, R> {
  using Staged = float;
  using G = TileGeom<float, R>;
  static constexpr int HW = kTX + 16;                  // remainder row width (halves)
  static constexpr unsigned RAW_H = (unsigned)(14 * G::SH * HW * 2);
  static constexpr unsigned M_OFF = (RAW_H + 127u) / 128u * 128u;
  static constexpr unsigned RAW_M = (unsigned)(4 * G::SH * G::SW * 4);
  static constexpr unsigned LOADED = RAW_H + RAW_M;
  static constexpr unsigned PLANES = (M_OFF + RAW_M + 127u) / 128u * 128u;
  static constexpr unsigned TABLES = (unsigned)((2 * kTX + 2 * G::TY) * 16);
  static constexpr unsigned BYTES = PLANES + TABLES;
  static constexpr unsigned DECODED = (unsigned)(14 * G::PLANE * 4);
  static constexpr unsigned EXTRA = (DECODED + 127u) / 128u * 128u;
  static_assert(BYTES % 128 == 0 && M_OFF % 128 == 0, "TMA destinations stay 128-byte aligned");
  static_assert(G::SW == kTX + 8, "the moment box covers the decoded window");
};

// Decode of a staged Neq16 tile into the FP32 buffer `out` (see
// TmaStage<Neq16, R>), two neighbouring columns per thread and pass.  The
// caller's next CTA-wide barrier publishes the buffer.  Nodes outside the mesh
// were zero-filled by the copy and decode to zero deviations, as the FP32
// stage holds there.
template <int R>
__device__ __forceinline__ void neq_decode_tile(const unsigned char* stage, float* out_f,
                                                float aT) {
  using ST = TmaStage<Neq16, R>;
  using G = typename ST::G;
  constexpr int NODES = G::PLANE, SW = G::SW, HW = ST::HW;
  constexpr int PAIRS = NODES / 2;
  static_assert(SW % 2 == 0 && HW % 2 == 0, "node pairs share one 32-bit word");
  const unsigned* rh = reinterpret_cast<const unsigned*>(stage);
  const float2* rm = reinterpret_cast<const float2*>(stage + ST::M_OFF);
  float2* out = reinterpret_cast<float2*>(out_f);
  float t0, ti;
  trest(aT, t0, ti);
  for (int q = threadIdx.x; q < PAIRS; q += kThreads) {   // nodes 2q, 2q + 1 of the window
    const int n = 2 * q;
    const int row = n / SW, c = n - row * SW;
    unsigned r[14];
#pragma unroll
    for (int i = 0; i < 14; ++i) r[i] = rh[((i * G::SH + row) * HW + c + 4) / 2];
    float2 f[9], g[5];
    neq_decode2x2(rm[q], rm[(NODES + n) / 2], rm[(2 * NODES + n) / 2], rm[(3 * NODES + n) / 2],
                  r, t0, ti, f, g);
#pragma unroll
    for (int i = 0; i < 9; ++i) out[(i * NODES + n) / 2] = f[i];
#pragma unroll
    for (int i = 0; i < 5; ++i) out[((9 + i) * NODES + n) / 2] = g[i];
  }
}

// CTAs per SM that the shared memory of a k_step_tma instantiation allows (two
// when its ring fits in half of the 228 KB); the register budget follows.
template <typename S, int R, int STAGES>
constexpr int tma_ctas_per_sm() {
  return (size_t)STAGES * TmaStage<S, R>::BYTES + TmaStage<S, R>::EXTRA + 1536 <= 114 * 1024
             ? 2
             : 1;
}

// tmap_m: the moment planes of a Neq16 buffer (unused for the other forms).
template <typename S, int R, int STAGES>
__global__ void __launch_bounds__(kThreads, (tma_ctas_per_sm<S, R, STAGES>()))
    k_step_tma(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap tmap_m,
               S* __restrict__ fout, P2<float> p, int* sched, int k0) {
  static_assert(STAGES >= 2, "a claimed tile is published by the barriers of the next use");
  using ST = TmaStage<S, R>;
  using SS = typename ST::Staged;
  using G = TileGeom<SS, R>;
  constexpr int TY = G::TY, HX = G::HX;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* dec = reinterpret_cast<float*>(smem_raw + (size_t)STAGES * ST::BYTES);   // Neq16
  uint64_t* bars =
      reinterpret_cast<uint64_t*>(smem_raw + (size_t)STAGES * ST::BYTES + ST::EXTRA);
  __shared__ int tile_of[STAGES];   // claimed tile of each stage (uses from k0 on)
  const int ntx = (p.nx + kTX - 1) / kTX, nty = (p.y1 - p.y0 + TY - 1) / TY;
  const int ntiles = ntx * nty;
  const int stride = STAGES * (int)gridDim.x;
  auto tile_origin = [&](int t, int& x0, int& y0, int& ry0) {
    const int ty = t / ntx;
    x0 = (t - ty * ntx) * kTX;
    y0 = p.y0 + ty * TY;
    ry0 = max(0, min(y0 - 1, p.ny - 3));
  };
  auto tables = [&](int st) {
    return reinterpret_cast<float4*>(smem_raw + (size_t)st * ST::BYTES + ST::PLANES);
  };
  auto issue = [&](int t, int st) {
    int x0, y0, ry0;
    tile_origin(t, x0, y0, ry0);
    // the tables of the tile's columns and rows that lie inside the mesh
    const unsigned xb = 16u * (unsigned)min(kTX, p.nx - x0);
    const unsigned yb = 16u * (unsigned)min(TY, p.ny - y0);
    float4* tab = tables(st);
    unsigned char* dst = smem_raw + (size_t)st * ST::BYTES;
    mbar_expect_tx(&bars[st], ST::LOADED + 2 * (xb + yb));
    if constexpr (is_neq<S>::value) {
      tma_load_3d(dst, &tmap, x0 - 8, ry0, 0, &bars[st]);
      tma_load_3d(dst + ST::M_OFF, &tmap_m, x0 - HX, ry0, 0, &bars[st]);
    } else {
      tma_load_3d(dst, &tmap, x0 - HX, ry0, 0, &bars[st]);
    }
    bulk_load(tab, p.px[0] + x0, xb, &bars[st]);
    bulk_load(tab + kTX, p.px[1] + x0, xb, &bars[st]);
    bulk_load(tab + 2 * kTX, p.py[0] + y0, yb, &bars[st]);
    bulk_load(tab + 2 * kTX + TY, p.py[1] + y0, yb, &bars[st]);
  };
  // Tile of the k-th stage use.  A claimed tile is written by thread 0 right
  // after the CTA-wide barrier that ends use k - STAGES; the barriers of use
  // k - STAGES + 1 (STAGES >= 2) publish it to the other threads.
  auto tile_at = [&](int k) {
    return k < k0 ? (int)blockIdx.x + k * (int)gridDim.x : tile_of[k % STAGES];
  };
  if constexpr (is_neq<S>::value) {
  if (threadIdx.x == 0) {
    asm volatile("prefetch.tensormap [%0];\n" ::"l"(&tmap) : "memory");
    asm volatile("prefetch.tensormap [%0];\n" ::"l"(&tmap_m) : "memory");
    for (int st = 0; st < STAGES; ++st) mbar_init(&bars[st], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int st = 0; st < STAGES; ++st) {
      const int t = blockIdx.x + st * gridDim.x;
      if (t < ntiles) issue(t, st);
    }
  for (int k = 0;; ++k) {
    const int t = tile_at(k);
    if (t >= ntiles) break;
    const int st = k % STAGES;
    // the tile for this stage's next use; a claim is made now so that its
    // latency overlaps the compute (the value is needed when the stage frees up)
    int next = t + stride;
    if (k + STAGES >= k0 && threadIdx.x == 0) next = k0 * (int)gridDim.x + atomicAdd(&sched[1], 1);
    const bool ok = mbar_wait(&bars[st], (unsigned)(k / STAGES) & 1u);
    // FP16NEQ: decode before the barrier, which then also publishes the decoded
    // tile (a thread whose wait gave up decodes stale data that is never used)
    if constexpr (is_neq<S>::value) neq_decode_tile<R>(smem_raw + (size_t)st * ST::BYTES, dec, p.a_T);
    if (__syncthreads_or(!ok)) {
      // a copy did not arrive: flag it, drain what is still in flight, leave
      if (threadIdx.x == 0) {
        atomicExch(&sched[0], 1);
        for (int j = 0; j < STAGES; ++j) {
          const int kk = k + j;
          if (tile_at(kk) < ntiles) mbar_wait(&bars[kk % STAGES], (unsigned)(kk / STAGES) & 1u);
        }
      }
      break;
    }
    int x0, y0, ry0;
    tile_origin(t, x0, y0, ry0);
    const SS* sm = reinterpret_cast<const SS*>(smem_raw + (size_t)st * ST::BYTES);
    if constexpr (is_neq<S>::value) sm = dec;
    const float4* tab = tables(st);
    tile_body<SS, R, false, S>(sm, tab, tab + kTX, tab + 2 * kTX, tab + 2 * kTX + TY, x0, y0,
                               ry0, fout, p);
    __syncthreads();   // every thread is done with stage st
    if (threadIdx.x == 0) {
      if (k + STAGES >= k0) tile_of[st] = next;
      if (next < ntiles) {
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        issue(next, st);
      }
    }
  }
  } else {
    // FP32 and 16-bit storage: a "full" and an "empty" mbarrier per stage and
    // no CTA-wide barrier in the loop.  Every warp waits for a stage's copies
    // itself, computes its part of the tile and arrives on the stage's empty
    // barrier; thread 0 refills the stage once all warps have arrived.  Warps
    // run up to STAGES - 1 tiles apart instead of meeting twice per tile.
    // In the claimed order a stage's tile index is written by thread 0 before
    // the arrival that completes the stage's phase, so a warp reads it after
    // its wait; with no tile left the phase is completed by a plain arrival.
    // A wait that fails raises the CTA's abort flag (every other wait then
    // gives up at once) and the error flag; thread 0 drains the stages it
    // filled before it leaves.
    uint64_t* full = bars;
    uint64_t* empty = bars + STAGES;
    volatile int* abort = reinterpret_cast<volatile int*>(bars + 2 * STAGES);
    if (threadIdx.x == 0) {
      asm volatile("prefetch.tensormap [%0];\n" ::"l"(&tmap) : "memory");
      for (int st = 0; st < STAGES; ++st) {
        mbar_init(&full[st], 1);
        mbar_init(&empty[st], kThreads / 32);
      }
      *abort = 0;
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    int filled = 0;   // thread 0: stage uses filled so far (copies or a plain arrival)
    int seen = 0;     // thread 0: stage uses whose phase it has seen complete
    if (threadIdx.x == 0)
      for (int st = 0; st < STAGES; ++st) {
        const int t = blockIdx.x + st * gridDim.x;
        if (t < ntiles) {
          issue(t, st);
          filled = st + 1;
        }
      }
    const unsigned lane = threadIdx.x & 31u;
    auto fail = [&]() {
      if (!*abort) atomicExch(&sched[0], 1);
      *abort = 1;
    };
    for (int k = 0;; ++k) {
      const int st = k % STAGES;
      const unsigned ph = (unsigned)(k / STAGES) & 1u;
      const bool fixed = k < k0;
      int t = (int)blockIdx.x + k * (int)gridDim.x;
      if (fixed && t >= ntiles) break;
      if (!__all_sync(0xffffffffu, mbar_wait_or_abort(&full[st], ph, abort))) {
        if (lane == 0) fail();
        break;
      }
      if (threadIdx.x == 0) seen = k + 1;
      if (!fixed) {
        t = tile_of[st];
        if (t >= ntiles) break;
      }
      // the tile of this stage's next use; a claim is made now so that its
      // latency overlaps the compute
      int next = t + stride;
      const bool claim = k + STAGES >= k0;   // the use k + STAGES takes a claimed tile
      if (claim && threadIdx.x == 0) next = k0 * (int)gridDim.x + atomicAdd(&sched[1], 1);
      int x0, y0, ry0;
      tile_origin(t, x0, y0, ry0);
      const float4* tab = tables(st);
      tile_body<SS, R, false, S>(reinterpret_cast<const SS*>(smem_raw + (size_t)st * ST::BYTES),
                                 tab, tab + kTX, tab + 2 * kTX, tab + 2 * kTX + TY, x0, y0, ry0,
                                 fout, p);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
      int pfail = 0;
      if (threadIdx.x == 0 && (next < ntiles || claim)) {
        // refill stage st for use k + STAGES once every warp is done with use k
        if (!mbar_wait_or_abort(&empty[st], ph, abort)) {
          fail();
          pfail = 1;
        } else {
          if (claim) tile_of[st] = next;
          if (next < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            issue(next, st);
          } else {
            mbar_arrive(&full[st]);   // no tile left: complete the phase with no bytes
          }
          filled = k + STAGES + 1;
        }
      }
      if (__shfl_sync(0xffffffffu, pfail, 0)) break;
    }
    // copies still in flight land before the CTA's shared memory is released
    if (threadIdx.x == 0)
      for (int u = seen; u < filled; ++u) mbar_wait(&full[u % STAGES], (unsigned)(u / STAGES) & 1u);
  }
  if (k0 != kFixedOrder && threadIdx.x == 0) {
    // every claim of this CTA is done; the last CTA out resets the counters
    __threadfence();
    if (atomicAdd(&sched[2], 1) == (int)gridDim.x - 1) {
      atomicExch(&sched[1], 0);
      atomicExch(&sched[2], 0);
    }
  }
}

// ---------------------------------------------------------------------------
// Batched persistent step: many cavities of different sizes in one launch.
// The work list holds (cavity, tile) items; each cavity brings its own
// parameters, output buffers and TMA descriptors (in global memory).
// ---------------------------------------------------------------------------

template <typename S>
struct alignas(128) BatchCav {
  CUtensorMap map[2];      // descriptors of the cavity's two buffers
  CUtensorMap mapm[2];     // Neq16: descriptors of their moment planes
  P2<float> p;
  S* out[2];               // output buffer when reading buffer 0 / 1
};

// Two CTAs per SM fit the shared memory of every 8-row form (FP16NEQ's
// decoded tile included); the register budget is held to that.
template <typename S, int R, int STAGES>
__global__ void __launch_bounds__(kThreads, (R == 2 ? 2 : 1))
    k_step_tma_batch(const BatchCav<S>* __restrict__ cavs, const int2* __restrict__ items,
                     int nitems, int parity, unsigned step, int* err) {
  using ST = TmaStage<S, R>;
  using SS = typename ST::Staged;
  using G = TileGeom<SS, R>;
  constexpr int TY = G::TY, HX = G::HX;
  constexpr unsigned BUF = ST::PLANES;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* dec = reinterpret_cast<float*>(smem_raw + (size_t)STAGES * BUF);   // Neq16
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (size_t)STAGES * BUF + ST::EXTRA);
  auto origin = [&](const P2<float>& p, int t, int& x0, int& y0, int& ry0) {
    const int ntx = (p.nx + kTX - 1) / kTX;
    const int ty = t / ntx;
    x0 = (t - ty * ntx) * kTX;
    y0 = ty * TY;
    ry0 = max(0, min(y0 - 1, p.ny - 3));
  };
  auto issue = [&](int item, int st) {
    const int2 it = items[item];
    const BatchCav<S>& cv = cavs[it.x];
    int x0, y0, ry0;
    origin(cv.p, it.y, x0, y0, ry0);
    unsigned char* dst = smem_raw + (size_t)st * BUF;
    mbar_expect_tx(&bars[st], ST::LOADED);
    if constexpr (is_neq<S>::value) {
      tma_load_3d(dst, &cv.map[parity], x0 - 8, ry0, 0, &bars[st]);
      tma_load_3d(dst + ST::M_OFF, &cv.mapm[parity], x0 - HX, ry0, 0, &bars[st]);
    } else {
      tma_load_3d(dst, &cv.map[parity], x0 - HX, ry0, 0, &bars[st]);
    }
  };
  if constexpr (is_neq<S>::value) {
  if (threadIdx.x == 0) {
    for (int st = 0; st < STAGES; ++st) mbar_init(&bars[st], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int st = 0; st < STAGES; ++st) {
      const int i = blockIdx.x + st * gridDim.x;
      if (i < nitems) issue(i, st);
    }
  for (int k = 0;; ++k) {
    const int i = blockIdx.x + k * gridDim.x;
    if (i >= nitems) break;
    const int st = k % STAGES;
    const bool ok = mbar_wait(&bars[st], (unsigned)(k / STAGES) & 1u);
    const int2 it = items[i];
    const BatchCav<S>& cv = cavs[it.x];
    // FP16NEQ: decode before the barrier, which then also publishes the decoded tile
    if constexpr (is_neq<S>::value) neq_decode_tile<R>(smem_raw + (size_t)st * BUF, dec, cv.p.a_T);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicExch(err, 1);
        for (int j = 0; j < STAGES; ++j) {
          const int kk = k + j;
          if (blockIdx.x + kk * gridDim.x < nitems)
            mbar_wait(&bars[kk % STAGES], (unsigned)(kk / STAGES) & 1u);
        }
      }
      return;
    }
    P2<float> p = cv.p;
    p.step = step;
    int x0, y0, ry0;
    origin(p, it.y, x0, y0, ry0);
    const SS* sm = reinterpret_cast<const SS*>(smem_raw + (size_t)st * BUF);
    if constexpr (is_neq<S>::value) sm = dec;
    tile_body<SS, R, false, S>(sm, p.px[0] + x0, p.px[1] + x0, p.py[0] + y0, p.py[1] + y0, x0,
                               y0, ry0, cv.out[parity], p);
    __syncthreads();
    if (threadIdx.x == 0) {
      const int in = i + STAGES * gridDim.x;
      if (in < nitems) {
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        issue(in, st);
      }
    }
  }
  } else {
    // FP32 and 16-bit storage: full / empty mbarriers per stage and no
    // CTA-wide barrier in the loop, as in k_step_tma.
    uint64_t* full = bars;
    uint64_t* empty = bars + STAGES;
    volatile int* abort = reinterpret_cast<volatile int*>(bars + 2 * STAGES);
    if (threadIdx.x == 0) {
      for (int st = 0; st < STAGES; ++st) {
        mbar_init(&full[st], 1);
        mbar_init(&empty[st], kThreads / 32);
      }
      *abort = 0;
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    int filled = 0, seen = 0;   // thread 0: stage uses filled / seen complete
    if (threadIdx.x == 0)
      for (int st = 0; st < STAGES; ++st) {
        const int i = blockIdx.x + st * gridDim.x;
        if (i < nitems) {
          issue(i, st);
          filled = st + 1;
        }
      }
    const unsigned lane = threadIdx.x & 31u;
    auto fail = [&]() {
      if (!*abort) atomicExch(err, 1);
      *abort = 1;
    };
    for (int k = 0;; ++k) {
      const int i = blockIdx.x + k * gridDim.x;
      if (i >= nitems) break;
      const int st = k % STAGES;
      const unsigned ph = (unsigned)(k / STAGES) & 1u;
      if (!__all_sync(0xffffffffu, mbar_wait_or_abort(&full[st], ph, abort))) {
        if (lane == 0) fail();
        break;
      }
      if (threadIdx.x == 0) seen = k + 1;
      const int2 it = items[i];
      const BatchCav<S>& cv = cavs[it.x];
      P2<float> p = cv.p;
      p.step = step;
      int x0, y0, ry0;
      origin(p, it.y, x0, y0, ry0);
      tile_body<SS, R, false, S>(reinterpret_cast<const SS*>(smem_raw + (size_t)st * BUF),
                                 p.px[0] + x0, p.px[1] + x0, p.py[0] + y0, p.py[1] + y0, x0, y0,
                                 ry0, cv.out[parity], p);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
      int pfail = 0;
      const int in = i + STAGES * gridDim.x;
      if (threadIdx.x == 0 && in < nitems) {
        // refill stage st once every warp is done with it
        if (!mbar_wait_or_abort(&empty[st], ph, abort)) {
          fail();
          pfail = 1;
        } else {
          asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
          issue(in, st);
          filled = k + STAGES + 1;
        }
      }
      if (__shfl_sync(0xffffffffu, pfail, 0)) break;
    }
    if (threadIdx.x == 0)
      for (int u = seen; u < filled; ++u) mbar_wait(&full[u % STAGES], (unsigned)(u / STAGES) & 1u);
  }
}

template <typename S, int R, bool UNI>
cudaError_t launch_tiled(const Solver& s, const S* in, S* out, const P2<float>& p) {
  using G = TileGeom<S, R>;
  const cudaError_t e = launch_setup_once(
      reinterpret_cast<const void*>(k_step_tiled<S, R, UNI>),
      [](const void* k, int*) {
        return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)TileGeom<S, R>::smem_bytes());
      },
      nullptr);
  if (e != cudaSuccess) return e;
  const dim3 grid((s.n[0] + kTX - 1) / kTX, (step_rows(s) + G::TY - 1) / G::TY);
  k_step_tiled<S, R, UNI><<<grid, kThreads, G::smem_bytes(), s.stream>>>(in, out, p);
  return cudaGetLastError();
}


// Tiles per CTA from which k_step_tma claims every tile after the first
// STAGES.  Measured on the FP32 1024^2 .. 8192^2 cavities: at 27 tiles per CTA
// (2048^2) the fixed stride is 2% faster, at 108 (4096^2) the claimed order
// is 1.2x faster and at 8192^2 1.5x.
constexpr int kClaimAllTilesPerCta = 64;

// Tuning override of the tile order: ISLBM_TMA_SCHEDULE=fixed / claimed /
// tail (unset: automatic).
int tma_schedule_override() {
  static const int v = [] {
    const char* e = std::getenv("ISLBM_TMA_SCHEDULE");
    if (!e) return -1;
    if (std::strcmp(e, "fixed") == 0) return 0;
    if (std::strcmp(e, "claimed") == 0) return 1;
    if (std::strcmp(e, "tail") == 0) return 2;
    return -1;
  }();
  return v;
}

// k0 of k_step_tma (the first claimed stage use): claimed throughout on large
// meshes, the fixed stride below that.  The `tail` order (the fixed stride one
// tile short of the CTAs' common share, then claimed tiles) was measured
// slower than the fixed stride at 1024^2 (41.4k against 44.5k MLUPS) and
// 2048^2, so it is only an option.
int tma_first_claim(int ntiles, int grid, int stages) {
  const int per_cta = ntiles / grid;
  int mode = tma_schedule_override();
  if (mode < 0) mode = per_cta >= kClaimAllTilesPerCta ? 1 : 0;
  if (mode == 1) return per_cta >= stages ? stages : kFixedOrder;
  if (mode == 2) return per_cta - 1 >= stages ? per_cta - 1 : kFixedOrder;
  return kFixedOrder;
}

template <typename S, int R, int STAGES>
cudaError_t launch_tma(const Solver& s, int cur, S* out, const P2<float>& p) {
  using G = TileGeom<typename TmaStage<S, R>::Staged, R>;
  constexpr size_t smem = (size_t)STAGES * TmaStage<S, R>::BYTES + TmaStage<S, R>::EXTRA + 64;
  int blocks_per_sm = 0;
  const cudaError_t e = launch_setup_once(
      reinterpret_cast<const void*>(k_step_tma<S, R, STAGES>),
      [](const void* k, int* bps) {
        cudaError_t e2 = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem);
        if (e2 == cudaSuccess)
          e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k, kThreads, smem);
        return e2;
      },
      &blocks_per_sm);
  if (e != cudaSuccess) return e;
  if (blocks_per_sm < 1) return cudaErrorInvalidConfiguration;
  const int ntiles = ((s.n[0] + kTX - 1) / kTX) * ((step_rows(s) + G::TY - 1) / G::TY);
  const int grid = std::min(ntiles, s.sm_count * blocks_per_sm);
  // claimed tiles pay off once a CTA walks more than a few dozen tiles
  const int k0 = tma_first_claim(ntiles, grid, STAGES);
  k_step_tma<S, R, STAGES><<<grid, kThreads, smem, s.stream>>>(
      *reinterpret_cast<const CUtensorMap*>(s.tmap[cur]),
      *reinterpret_cast<const CUtensorMap*>(s.tmap_m[cur]), out, p, s.derr, k0);
  return cudaGetLastError();
}

dim3 block2() { return dim3(32, 8); }
dim3 grid2(const Solver& s) { return dim3((s.n[0] + 31) / 32, (s.n[1] + 7) / 8); }
dim3 grid2_step(const Solver& s) { return dim3((s.n[0] + 31) / 32, (step_rows(s) + 7) / 8); }

// Dispatch on the storage type.
template <template <typename> class Fn, typename... A>
cudaError_t dispatch(Solver& s, A... a) {
  switch (s.precision) {
    case ISLBM_FP64: return Fn<double>::run(s, a...);
    case ISLBM_FP32: return Fn<float>::run(s, a...);
    case ISLBM_FP16DEV: return Fn<__half>::run(s, a...);
    case ISLBM_BF16DEV: return Fn<__nv_bfloat16>::run(s, a...);
    case ISLBM_FP16NEQ: return Fn<Neq16>::run(s, a...);
  }
  return cudaErrorInvalidValue;
}

template <typename S>
struct StepFn {
  static cudaError_t run(Solver& s) {
    using R = typename Store<S>::R;
    const P2<R> p = make_params<R>(s);
    S* out = static_cast<S*>(s.buf[s.cur ^ 1]);
    if constexpr (is_neq<S>::value) {
      // the non-equilibrium form is decoded per staged tile: pipelined kernels only
      switch (s.variant) {
        case KV_TMA_R2S2: return launch_tma<S, 2, 2>(s, s.cur, out, p);
        case KV_TMA_R2S3: return launch_tma<S, 2, 3>(s, s.cur, out, p);
        default: return cudaErrorInvalidValue;
      }
    } else {
      const S* in = static_cast<const S*>(s.buf[s.cur]);
      if constexpr (!std::is_same<S, double>::value) {
        // the tiled kernels cover the centred stencil (their halo is one node);
        // on the uniform mesh the direct pure-shift kernel is the default
        if (s.stencil == ISLBM_STENCIL_CENTRED) {
          switch (s.variant) {
            case KV_TILED: return launch_tiled<S, 4, false>(s, in, out, p);
            case KV_TMA_R4S2: return launch_tma<S, 4, 2>(s, s.cur, out, p);
            case KV_TMA_R2S2: return launch_tma<S, 2, 2>(s, s.cur, out, p);
            case KV_TMA_R2S3: return launch_tma<S, 2, 3>(s, s.cur, out, p);
            case KV_TMA_R4S3: return launch_tma<S, 4, 3>(s, s.cur, out, p);
            default: break;
          }
        }
      }
      if (s.uniform)
        k_step<S, true><<<grid2_step(s), block2(), 0, s.stream>>>(in, out, p);
      else
        k_step<S, false><<<grid2_step(s), block2(), 0, s.stream>>>(in, out, p);
      return cudaGetLastError();
    }
  }
};

template <typename S>
struct InitFieldsFn {
  static cudaError_t run(Solver& s, const double* rho, const double* T, const double* u,
                         const double* v) {
    using R = typename Store<S>::R;
    k_init_fields<S><<<grid2(s), block2(), 0, s.stream>>>(static_cast<S*>(s.buf[s.cur]),
                                                         make_params<R>(s), rho, T, u, v);
    return cudaGetLastError();
  }
};

template <typename S>
struct InitPopsFn {
  static cudaError_t run(Solver& s, const double* f, const double* g) {
    using R = typename Store<S>::R;
    k_init_pops<S><<<grid2(s), block2(), 0, s.stream>>>(static_cast<S*>(s.buf[s.cur]),
                                                       make_params<R>(s), f, g);
    return cudaGetLastError();
  }
};

template <typename S>
struct FieldsFn {
  static cudaError_t run(Solver& s, double* rho, double* T, double* u, double* v) {
    using R = typename Store<S>::R;
    k_fields<S><<<grid2(s), block2(), 0, s.stream>>>(static_cast<const S*>(s.buf[s.cur]),
                                                    make_params<R>(s), s.ph.gbeta, s.ph.Ts, s.ph.T0, rho,
                                                    T, u, v);
    return cudaGetLastError();
  }
};

template <typename S>
struct PopsFn {
  static cudaError_t run(Solver& s, double* f, double* g) {
    using R = typename Store<S>::R;
    k_pops<S><<<grid2(s), block2(), 0, s.stream>>>(static_cast<const S*>(s.buf[s.cur]),
                                                  make_params<R>(s), f, g);
    return cudaGetLastError();
  }
};

template <typename S>
struct ReduceFn {
  static cudaError_t run(Solver& s) {
    using R = typename Store<S>::R;
    k_reduce<S><<<s.red_blocks, 256, 0, s.stream>>>(
        static_cast<const S*>(s.buf[s.cur]), make_params<R>(s), s.ph.gbeta, s.ph.Ts, s.ph.T0,
        s.dax[0].W, s.dax[1].W, s.dscratch);
    return cudaGetLastError();
  }
};

template <typename S>
struct SteadyFn {
  static cudaError_t run(Solver& s) {
    using R = typename Store<S>::R;
    k_steady<S><<<s.red_blocks, 256, 0, s.stream>>>(
        static_cast<const S*>(s.buf[s.cur]), make_params<R>(s), s.ph.gbeta, s.ph.Ts, s.ph.T0,
        s.ph.dT, s.snap_valid ? 1 : 0, s.dsnap, s.dscratch);
    return cudaGetLastError();
  }
};

}  // namespace

cudaError_t launch_step(Solver& s) {
  if (s.dim == 3) return launch_step_3d(s);
  cudaError_t e = dispatch<StepFn>(s);
  if (e == cudaSuccess) s.cur ^= 1;
  return e;
}

cudaError_t launch_init_fields(Solver& s, const double* rho, const double* T, const double* u0,
                               const double* u1, const double* u2) {
  if (s.dim == 3) return launch_init_fields_3d(s, rho, T, u0, u1, u2);
  return dispatch<InitFieldsFn>(s, rho, T, u0, u1);
}

cudaError_t launch_init_populations(Solver& s, const double* f, const double* g) {
  if (s.dim == 3) return launch_init_populations_3d(s, f, g);
  return dispatch<InitPopsFn>(s, f, g);
}

cudaError_t launch_fields(Solver& s, double* rho, double* T, double* u0, double* u1,
                          double* u2) {
  if (s.dim == 3) return launch_fields_3d(s, rho, T, u0, u1, u2);
  return dispatch<FieldsFn>(s, rho, T, u0, u1);
}

cudaError_t launch_populations(Solver& s, double* f, double* g) {
  if (s.dim == 3) return launch_populations_3d(s, f, g);
  return dispatch<PopsFn>(s, f, g);
}

cudaError_t launch_reduce(Solver& s) {
  cudaError_t e = (s.dim == 3) ? launch_reduce_3d(s) : dispatch<ReduceFn>(s);
  if (e != cudaSuccess) return e;
  return launch_finish_reduce(s);
}

cudaError_t launch_steady(Solver& s) {
  cudaError_t e = (s.dim == 3) ? launch_steady_3d(s) : dispatch<SteadyFn>(s);
  if (e != cudaSuccess) return e;
  return launch_finish_reduce(s);
}

cudaError_t launch_finish_reduce(Solver& s) {
  k_finish<<<1, 32 * RED_COUNT, 0, s.stream>>>(s.dscratch, s.red_blocks, s.dresult);
  return cudaGetLastError();
}

// ---- batched step ----
namespace {

template <typename S, int R>
struct BatchGroupImpl : BatchGroup {
  BatchCav<S>* dcavs = nullptr;
  int2* ditems = nullptr;
  int ncav = 0, nitems = 0, grid = 0;
  size_t smem = 0;
  DevAllocator mem;
  cudaStream_t stream = nullptr;
  ~BatchGroupImpl() override {
    dev_free(mem, dcavs, stream);
    dev_free(mem, ditems, stream);
    cudaStreamSynchronize(stream);
  }
  cudaError_t launch(cudaStream_t st, int parity, unsigned step, int* err) override {
    k_step_tma_batch<S, R, 2><<<grid, kThreads, smem, st>>>(dcavs, ditems, nitems, parity, step,
                                                           err);
    return cudaGetLastError();
  }
};

template <typename S, int R>
cudaError_t make_group_impl(const std::vector<Solver*>& members, int sm_count,
                            cudaStream_t stream, BatchGroup** out) {
  using G = TileGeom<typename TmaStage<S, R>::Staged, R>;
  auto* g = new BatchGroupImpl<S, R>();
  g->smem = (size_t)2 * TmaStage<S, R>::PLANES + TmaStage<S, R>::EXTRA + 64;
  cudaError_t e = cudaFuncSetAttribute(k_step_tma_batch<S, R, 2>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g->smem);
  int bps = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_step_tma_batch<S, R, 2>, kThreads,
                                                      g->smem);
  std::vector<BatchCav<S>> cavs(members.size());
  std::vector<int2> items;
  for (size_t c = 0; c < members.size() && e == cudaSuccess; ++c) {
    Solver& m = *members[c];
    std::memcpy(&cavs[c].map[0], m.tmap[0], sizeof(CUtensorMap));
    std::memcpy(&cavs[c].map[1], m.tmap[1], sizeof(CUtensorMap));
    std::memcpy(&cavs[c].mapm[0], m.tmap_m[0], sizeof(CUtensorMap));
    std::memcpy(&cavs[c].mapm[1], m.tmap_m[1], sizeof(CUtensorMap));
    cavs[c].p = make_params<float>(m);
    cavs[c].out[0] = static_cast<S*>(m.buf[1]);
    cavs[c].out[1] = static_cast<S*>(m.buf[0]);
    const int ntiles = ((m.n[0] + kTX - 1) / kTX) * ((m.n[1] + G::TY - 1) / G::TY);
    for (int t = 0; t < ntiles; ++t) items.push_back(make_int2((int)c, t));
  }
  g->ncav = (int)members.size();
  g->nitems = (int)items.size();
  g->grid = std::max(1, std::min(g->nitems, sm_count * std::max(bps, 1)));
  g->mem = current_allocator();
  g->stream = stream;
  if (e == cudaSuccess)
    e = dev_alloc(g->mem, reinterpret_cast<void**>(&g->dcavs), cavs.size() * sizeof(BatchCav<S>),
                  stream);
  if (e == cudaSuccess)
    e = dev_alloc(g->mem, reinterpret_cast<void**>(&g->ditems), items.size() * sizeof(int2),
                  stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->dcavs, cavs.data(), cavs.size() * sizeof(BatchCav<S>),
                        cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->ditems, items.data(), items.size() * sizeof(int2),
                        cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    delete g;
    return e;
  }
  *out = g;
  return cudaSuccess;
}

template <int R>
cudaError_t make_group_r(const std::vector<Solver*>& m, int precision, int sm, cudaStream_t st,
                         BatchGroup** out) {
  switch (precision) {
    case ISLBM_FP32: return make_group_impl<float, R>(m, sm, st, out);
    case ISLBM_FP16DEV: return make_group_impl<__half, R>(m, sm, st, out);
    case ISLBM_BF16DEV: return make_group_impl<__nv_bfloat16, R>(m, sm, st, out);
    case ISLBM_FP16NEQ:
      if constexpr (R == 2) return make_group_impl<Neq16, R>(m, sm, st, out);
      break;
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t make_batch_group(const std::vector<Solver*>& members, int tile_rows, int precision,
                             int sm_count, cudaStream_t stream, BatchGroup** out) {
  if (tile_rows == 2) return make_group_r<2>(members, precision, sm_count, stream, out);
  if (tile_rows == 4) return make_group_r<4>(members, precision, sm_count, stream, out);
  return cudaErrorInvalidValue;
}

}  // namespace islbm

namespace islbm {
int bounds_flag_d2(int reset) {
#ifdef ISLBM_BOUNDS_CHECK
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_bounds_flag, sizeof(int)) != cudaSuccess) return -1;
  if (reset) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_bounds_flag, &zero, sizeof(int));
  }
  return v;
#else
  (void)reset;
  return 0;
#endif
}
}  // namespace islbm
