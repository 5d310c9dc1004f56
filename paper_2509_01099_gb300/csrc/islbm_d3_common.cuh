// Shared pieces of the 3-D step kernels: parameters, rest weights and the
// D3Q19 / D3Q7 MRT collision (Sec. 2.1, Sec. 4).
#pragma once

#include "islbm_internal.h"
#include "islbm_lanes.cuh"
#include "islbm_store.cuh"

namespace islbm {
namespace {

template <typename R>
struct P3 {
  int nx, ny, nz, pitch;
  long long plane;
  const int* b[3][2];
  const R* w[3][2];
  const float4* pk[3][2];   // packed FP32 tables (w0, w1, w2, base) of the pipelined kernel
  // temperature populations carry T - T_s; force rho g beta (T - T_s + Fb)
  R gbeta, s_e, s_eps, s_q, s_nu, s_pi, s_m, q_j, q_e, q_nu, a_T;
  R Ts, Fb;
  R abb_hot, abb_cold;
  unsigned step;   // seeds the stochastic rounding of 16-bit stores
};

template <typename R>
__device__ __forceinline__ R wrest3(int i) {
  return i == 0 ? R(1.0 / 3.0) : (i < 7 ? R(1.0 / 18.0) : R(1.0 / 36.0));
}

// MRT collision of one node in deviation form (Sec. 2.1), d'Humieres moment basis
// (rho, e, eps, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww, pxy, pyz, pxz,
// mx, my, mz) with the printed m_eq and M F~; f+ = f + M^T diag(1/|row|^2) dm.
// Temperature: D3Q7 rows (T, jx, jy, jz, -6+7|c|^2, 3cx^2-|c|^2, cy^2-cz^2).
template <typename R>
__device__ __forceinline__ void collide3(R (&f)[19], R (&g)[7], const P3<R>& p, R& rho_o,
                                         R& ux_o, R& uy_o, R& uz_o, R& T_o) {
  const R sax = ((f[1] + f[2]) + (f[3] + f[4])) + (f[5] + f[6]);
  const R exy = (f[7] + f[8]) + (f[9] + f[10]);
  const R exz = (f[11] + f[12]) + (f[13] + f[14]);
  const R eyz = (f[15] + f[16]) + (f[17] + f[18]);
  const R sed = exy + exz + eyz;
  const R drho = f[0] + sax + sed;
  const R rho = R(1) + drho;
  // odd combinations of the edge populations
  const R xy_x = (f[7] - f[8]) + (f[9] - f[10]);    // sum cx over xy edges
  const R xy_y = (f[7] - f[8]) - (f[9] - f[10]);    // sum cy over xy edges
  const R xz_x = (f[11] - f[12]) + (f[13] - f[14]);
  const R xz_z = (f[11] - f[12]) - (f[13] - f[14]);
  const R yz_y = (f[15] - f[16]) + (f[17] - f[18]);
  const R yz_z = (f[15] - f[16]) - (f[17] - f[18]);
  const R jx = (f[1] - f[2]) + xy_x + xz_x;
  const R jy = (f[3] - f[4]) + xy_y + yz_y;
  const R jz = (f[5] - f[6]) + xz_z + yz_z;
  const R Tr = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + g[6]);
  const R T = Tr;   // T - T_s
  const R Fy = rho * p.gbeta * (Tr + p.Fb);
  const R inv = lrcp(rho);
  const R ux = jx * inv, uy = (jy + R(0.5) * Fy) * inv, uz = jz * inv;
  const R ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
  const R rusq = rho * (ux2 + uy2 + uz2);
  const R uF = uy * Fy;

  const R m1 = R(-30) * f[0] - R(11) * sax + R(8) * sed;
  const R m2 = R(12) * f[0] - R(4) * sax + sed;
  const R m4 = R(-4) * (f[1] - f[2]) + xy_x + xz_x;
  const R m6 = R(-4) * (f[3] - f[4]) + xy_y + yz_y;
  const R m8 = R(-4) * (f[5] - f[6]) + xz_z + yz_z;
  const R axx = f[1] + f[2], ayy = f[3] + f[4], azz = f[5] + f[6];
  const R m9 = R(2) * axx - (ayy + azz) + (exy + exz) - R(2) * eyz;
  const R m10 = R(-4) * axx + R(2) * (ayy + azz) + (exy + exz) - R(2) * eyz;
  const R m11 = (ayy - azz) + (exy - exz);
  const R m12 = R(-2) * (ayy - azz) + (exy - exz);
  const R m13 = (f[7] + f[8]) - (f[9] + f[10]);
  const R m14 = (f[15] + f[16]) - (f[17] + f[18]);
  const R m15 = (f[11] + f[12]) - (f[13] + f[14]);
  const R m16 = xy_x - xz_x;
  const R m17 = yz_y - xy_y;
  const R m18 = xz_z - yz_z;

  const R pxx = R(2) * ux2 - uy2 - uz2, pww = uy2 - uz2;
  const R dm1 = -p.s_e * (m1 + R(11) * drho - R(19) * rusq) + (R(1) - R(0.5) * p.s_e) * R(38) * uF;
  const R dm2 = -p.s_eps * (m2 - R(3) * drho + R(5.5) * rusq) - (R(1) - R(0.5) * p.s_eps) * R(11) * uF;
  const R dm4 = -p.s_q * (m4 + R(2.0 / 3.0) * rho * ux);
  const R dm5 = Fy;
  const R dm6 = -p.s_q * (m6 + R(2.0 / 3.0) * rho * uy) - (R(1) - R(0.5) * p.s_q) * R(2.0 / 3.0) * Fy;
  const R dm8 = -p.s_q * (m8 + R(2.0 / 3.0) * rho * uz);
  const R dm9 = -p.s_nu * (m9 - rho * pxx) - (R(1) - R(0.5) * p.s_nu) * R(2) * uF;
  const R dm10 = -p.s_pi * (m10 + R(0.5) * rho * pxx) + (R(1) - R(0.5) * p.s_pi) * uF;
  const R dm11 = -p.s_nu * (m11 - rho * pww) + (R(1) - R(0.5) * p.s_nu) * R(2) * uF;
  const R dm12 = -p.s_pi * (m12 + R(0.5) * rho * pww) - (R(1) - R(0.5) * p.s_pi) * uF;
  const R dm13 = -p.s_nu * (m13 - rho * ux * uy) + (R(1) - R(0.5) * p.s_nu) * ux * Fy;
  const R dm14 = -p.s_nu * (m14 - rho * uy * uz) + (R(1) - R(0.5) * p.s_nu) * uz * Fy;
  const R dm15 = -p.s_nu * (m15 - rho * ux * uz);
  const R dm16 = -p.s_m * m16, dm17 = -p.s_m * m17, dm18 = -p.s_m * m18;

  const R a1 = dm1 * R(1.0 / 2394.0), a2 = dm2 * R(1.0 / 252.0);
  const R a4 = dm4 * R(1.0 / 40.0), a5 = dm5 * R(0.1), a6 = dm6 * R(1.0 / 40.0);
  const R a8 = dm8 * R(1.0 / 40.0);
  const R a9 = dm9 * R(1.0 / 36.0), a10 = dm10 * R(1.0 / 72.0);
  const R a11 = dm11 * R(1.0 / 12.0), a12 = dm12 * R(1.0 / 24.0);
  const R a13 = dm13 * R(0.25), a14 = dm14 * R(0.25), a15 = dm15 * R(0.25);
  const R a16 = dm16 * R(0.125), a17 = dm17 * R(0.125), a18 = dm18 * R(0.125);

  const R cax = R(-11) * a1 - R(4) * a2;
  const R ced = R(8) * a1 + a2;
  f[0] += R(-30) * a1 + R(12) * a2;
  const R xx = R(2) * a9 - R(4) * a10;                 // x-axis pair, even part
  const R yy = -a9 + R(2) * a10 + a11 - R(2) * a12;    // y-axis pair
  const R zz = -a9 + R(2) * a10 - a11 + R(2) * a12;    // z-axis pair
  f[1] += cax + xx - R(4) * a4;
  f[2] += cax + xx + R(4) * a4;
  f[3] += cax + yy + a5 - R(4) * a6;
  f[4] += cax + yy - a5 + R(4) * a6;
  f[5] += cax + zz - R(4) * a8;
  f[6] += cax + zz + R(4) * a8;
  const R exy_e = ced + a9 + a10 + a11 + a12;          // even part of the xy edges
  const R exz_e = ced + a9 + a10 - a11 - a12;
  const R eyz_e = ced - R(2) * a9 - R(2) * a10;
  const R px = a4, py = a5 + a6, pz = a8;                // odd parts (jx = jz = 0 increments)
  f[7] += exy_e + px + py + a13 + a16 - a17;
  f[8] += exy_e - px - py + a13 - a16 + a17;
  f[9] += exy_e + px - py - a13 + a16 + a17;
  f[10] += exy_e - px + py - a13 - a16 - a17;
  f[11] += exz_e + px + pz + a15 - a16 + a18;
  f[12] += exz_e - px - pz + a15 + a16 - a18;
  f[13] += exz_e + px - pz - a15 - a16 - a18;
  f[14] += exz_e - px + pz - a15 + a16 + a18;
  f[15] += eyz_e + py + pz + a14 + a17 - a18;
  f[16] += eyz_e - py - pz + a14 - a17 + a18;
  f[17] += eyz_e + py - pz - a14 + a17 + a18;
  f[18] += eyz_e - py + pz - a14 - a17 - a18;

  const R n1 = g[1] - g[2], n2 = g[3] - g[4], n3 = g[5] - g[6];
  const R n4 = R(-6) * g[0] + ((g[1] + g[2]) + (g[3] + g[4])) + (g[5] + g[6]);
  const R n5 = R(2) * (g[1] + g[2]) - ((g[3] + g[4]) + (g[5] + g[6]));
  const R n6 = (g[3] + g[4]) - (g[5] + g[6]);
  const R b1 = R(-0.5) * p.q_j * (n1 - ux * T);
  const R b2 = R(-0.5) * p.q_j * (n2 - uy * T);
  const R b3 = R(-0.5) * p.q_j * (n3 - uz * T);
  const R b4 = -p.q_e * (n4 - p.a_T * Tr) * R(1.0 / 42.0);
  const R b5 = -p.q_nu * n5 * R(1.0 / 12.0);
  const R b6 = R(-0.25) * p.q_nu * n6;
  g[0] += R(-6) * b4;
  g[1] += b1 + b4 + R(2) * b5;
  g[2] += -b1 + b4 + R(2) * b5;
  g[3] += b2 + b4 - b5 + b6;
  g[4] += -b2 + b4 - b5 + b6;
  g[5] += b3 + b4 - b5 - b6;
  g[6] += -b3 + b4 - b5 - b6;
  rho_o = rho;
  ux_o = ux;
  uy_o = uy;
  uz_o = uz;
  T_o = T;
}

template <typename R>
P3<R> make_params3(const Solver& s) {
  P3<R> p;
  p.nx = s.n[0];
  p.ny = s.n[1];
  p.nz = s.n[2];
  p.pitch = s.pitch;
  p.plane = s.plane;
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 2; ++k) {
      p.b[a][k] = s.dax[a].base[k];
      p.w[a][k] = static_cast<const R*>(s.dax[a].w[k]);
      p.pk[a][k] = s.dax[a].packed[k];
    }
  const Physics& h = s.ph;
  p.gbeta = R(h.gbeta);
  p.Ts = R(h.Ts);
  p.Fb = R(h.Ts - h.T0);
  p.s_e = R(h.s_e);
  p.s_eps = R(h.s_eps);
  p.s_q = R(h.s_q);
  p.s_nu = R(h.s_nu);
  p.s_pi = R(h.s_pi);
  p.s_m = R(h.s_m);
  p.q_j = R(h.q_j);
  p.q_e = R(h.q_e);
  p.q_nu = R(h.q_nu);
  p.a_T = R(h.a_T);
  p.abb_hot = R(h.omega * (h.T_hot - h.Ts));
  p.abb_cold = R(h.omega * (h.T_cold - h.Ts));
  p.step = (unsigned)s.time;
  return p;
}

}  // namespace
}  // namespace islbm
