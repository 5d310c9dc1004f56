// 3-D kernels: D3Q19 flow + D3Q7 temperature populations (Sec. 2.1 - 2.3, Sec. 4).
//
// Storage: one plane per population, [q][z][y][x] with a padded x pitch;
// planes 0..18 hold the flow populations, 19..25 the temperature populations,
// in the velocity order
//   D3Q19: 0 | +x -x +y -y +z -z | (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0)
//          (1,0,1) (-1,0,-1) (1,0,-1) (-1,0,1) (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1)
//   D3Q7:  0 | +x -x +y -y +z -z
// As in 2-D, the stored state is the post-collision deviation, and one step is
// pull (interpolated virtual streaming or wall rule) -> macroscopic moments ->
// MRT collision -> store.  Hot wall at x = 0, cold wall at x = 1, the y and z
// walls adiabatic; gravity along -y.
#include "islbm_internal.h"
#include "islbm_store.cuh"
#include "islbm_d3_common.cuh"

namespace islbm {
namespace {

// Separable quadratic interpolation of one population at node (x, y, z)
// (Sec. 2.2).  At most two axes move for D3Q19.
template <typename S, typename R, int CX, int CY, int CZ, bool UNI>
__device__ __forceinline__ R pull3(const S* __restrict__ pl, int x, int y, int z,
                                   const P3<R>& p) {
  using St = Store<S>;
  const size_t sy = p.pitch, sz = (size_t)p.pitch * p.ny;
  if (UNI || (CX == 0 && CY == 0 && CZ == 0))
    return St::ld(pl + (size_t)(z - CZ) * sz + (size_t)(y - CY) * sy + (x - CX));
  // the (up to) two moving axes
  int base0 = 0, base1 = 0;
  const R* w0 = nullptr;
  const R* w1 = nullptr;
  size_t st0 = 0, st1 = 0;
  size_t origin = (size_t)z * sz + (size_t)y * sy + x;
  int na = 0;
  if (CX != 0) {
    constexpr int k = CX > 0 ? 0 : 1;
    base0 = __ldg(p.b[0][k] + x);
    w0 = p.w[0][k] + 3 * x;
    st0 = 1;
    origin -= x;
    na = 1;
  }
  if (CY != 0) {
    constexpr int k = CY > 0 ? 0 : 1;
    const int b = __ldg(p.b[1][k] + y);
    const R* w = p.w[1][k] + 3 * y;
    origin -= (size_t)y * sy;
    if (na == 0) { base0 = b; w0 = w; st0 = sy; na = 1; }
    else { base1 = b; w1 = w; st1 = sy; na = 2; }
  }
  if (CZ != 0) {
    constexpr int k = CZ > 0 ? 0 : 1;
    const int b = __ldg(p.b[2][k] + z);
    const R* w = p.w[2][k] + 3 * z;
    origin -= (size_t)z * sz;
    if (na == 0) { base0 = b; w0 = w; st0 = sz; na = 1; }
    else { base1 = b; w1 = w; st1 = sz; na = 2; }
  }
  const S* o = pl + origin + (size_t)base0 * st0;
  const R a0 = __ldg(w0), a1 = __ldg(w0 + 1), a2 = __ldg(w0 + 2);
  if (na == 1) return lin3(a0, a1, a2, St::ld(o), St::ld(o + st0), St::ld(o + 2 * st0));
  o += (size_t)base1 * st1;
  R acc = R(0);
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const S* r = o + l * st1;
    acc = lfma(__ldg(w1 + l), lin3(a0, a1, a2, St::ld(r), St::ld(r + st0), St::ld(r + 2 * st0)),
               acc);
  }
  return acc;
}

template <typename S, bool UNI>
__global__ void __launch_bounds__(256)
    k_step3(const S* __restrict__ fin, S* __restrict__ fout, P3<typename Store<S>::R> p) {
  using R = typename Store<S>::R;
  using St = Store<S>;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= p.nx || y >= p.ny) return;
  const size_t idx = ((size_t)z * p.ny + y) * p.pitch + x;
  const long long P = p.plane;
  const bool wxm = x == 0, wxp = x == p.nx - 1, wym = y == 0, wyp = y == p.ny - 1;
  const bool wzm = z == 0, wzp = z == p.nz - 1;
  R f[19], g[7];
#define BB(i, o) St::ld(fin + (o) * P + idx)
#define PL(i, cx, cy, cz) pull3<S, R, cx, cy, cz, UNI>(fin + (i) * P, x, y, z, p)
  f[0] = St::ld(fin + idx);
  f[1] = wxm ? BB(1, 2) : PL(1, 1, 0, 0);
  f[2] = wxp ? BB(2, 1) : PL(2, -1, 0, 0);
  f[3] = wym ? BB(3, 4) : PL(3, 0, 1, 0);
  f[4] = wyp ? BB(4, 3) : PL(4, 0, -1, 0);
  f[5] = wzm ? BB(5, 6) : PL(5, 0, 0, 1);
  f[6] = wzp ? BB(6, 5) : PL(6, 0, 0, -1);
  f[7] = (wxm || wym) ? BB(7, 8) : PL(7, 1, 1, 0);
  f[8] = (wxp || wyp) ? BB(8, 7) : PL(8, -1, -1, 0);
  f[9] = (wxm || wyp) ? BB(9, 10) : PL(9, 1, -1, 0);
  f[10] = (wxp || wym) ? BB(10, 9) : PL(10, -1, 1, 0);
  f[11] = (wxm || wzm) ? BB(11, 12) : PL(11, 1, 0, 1);
  f[12] = (wxp || wzp) ? BB(12, 11) : PL(12, -1, 0, -1);
  f[13] = (wxm || wzp) ? BB(13, 14) : PL(13, 1, 0, -1);
  f[14] = (wxp || wzm) ? BB(14, 13) : PL(14, -1, 0, 1);
  f[15] = (wym || wzm) ? BB(15, 16) : PL(15, 0, 1, 1);
  f[16] = (wyp || wzp) ? BB(16, 15) : PL(16, 0, -1, -1);
  f[17] = (wym || wzp) ? BB(17, 18) : PL(17, 0, 1, -1);
  f[18] = (wyp || wzm) ? BB(18, 17) : PL(18, 0, -1, 1);
  g[0] = St::ld(fin + 19 * P + idx);
  g[1] = wxm ? p.abb_hot - BB(20, 21) : PL(20, 1, 0, 0);
  g[2] = wxp ? p.abb_cold - BB(21, 20) : PL(21, -1, 0, 0);
  g[3] = wym ? BB(22, 23) : PL(22, 0, 1, 0);
  g[4] = wyp ? BB(23, 22) : PL(23, 0, -1, 0);
  g[5] = wzm ? BB(24, 25) : PL(24, 0, 0, 1);
  g[6] = wzp ? BB(25, 24) : PL(25, 0, 0, -1);
#undef BB
#undef PL
  R rho, ux, uy, uz, T;
  collide3(f, g, p, rho, ux, uy, uz, T);
  unsigned r = sr_seed(idx, p.step);
#pragma unroll
  for (int i = 0; i < 19; ++i) St::st_sr(fout + i * P + idx, f[i], sr_next(r));
#pragma unroll
  for (int i = 0; i < 7; ++i) St::st_sr(fout + (19 + i) * P + idx, g[i], sr_next(r));
}

__device__ __constant__ int kE3[19][3] = {
    {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1}, {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1}, {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

// Equilibrium (Sec. 2.1) of given fields, then the collision: the second-order
// Hermite flow equilibrium (whose moments are the printed m_eq) and
// g_0 = t_0 T, g_i = t_i T + (e_i.u) T / 2 with t_0 = (1-a_T)/7, t_i = (6+a_T)/42.
template <typename S>
__global__ void k_init_fields3(S* __restrict__ fout, P3<typename Store<S>::R> p,
                               const double* __restrict__ rho_in, const double* __restrict__ T_in,
                               const double* __restrict__ u_in, const double* __restrict__ v_in,
                               const double* __restrict__ w_in) {
  using R = typename Store<S>::R;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= p.nx || y >= p.ny) return;
  const size_t node = ((size_t)z * p.ny + y) * p.nx + x;
  const R rho = rho_in ? R(rho_in[node]) : R(1);
  const R T = R(T_in[node] - (double)p.Ts);   // T - T_s
  const R ux = u_in ? R(u_in[node]) : R(0);
  const R uy = v_in ? R(v_in[node]) : R(0);
  const R uz = w_in ? R(w_in[node]) : R(0);
  const R usq = ux * ux + uy * uy + uz * uz;
  R f[19], g[7];
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const R eu = R(kE3[i][0]) * ux + R(kE3[i][1]) * uy + R(kE3[i][2]) * uz;
    f[i] = wrest3<R>(i) * (rho * (R(1) + R(3) * eu + R(4.5) * eu * eu - R(1.5) * usq) - R(1));
  }
  const R t0 = (R(1) - p.a_T) / R(7), ti = (R(6) + p.a_T) / R(42);
  const R Tr = T;
  g[0] = t0 * Tr;
#pragma unroll
  for (int i = 1; i < 7; ++i)
    g[i] = ti * Tr + R(0.5) * (R(kE3[i][0]) * ux + R(kE3[i][1]) * uy + R(kE3[i][2]) * uz) * T;
  R r_, a_, b_, c_, d_;
  collide3(f, g, p, r_, a_, b_, c_, d_);
  const size_t idx = ((size_t)z * p.ny + y) * p.pitch + x;
#pragma unroll
  for (int i = 0; i < 19; ++i) Store<S>::st(fout + i * p.plane + idx, f[i]);
#pragma unroll
  for (int i = 0; i < 7; ++i) Store<S>::st(fout + (19 + i) * p.plane + idx, g[i]);
}

template <typename S>
__global__ void k_init_pops3(S* __restrict__ fout, P3<typename Store<S>::R> p,
                             const double* __restrict__ fin, const double* __restrict__ gin) {
  using R = typename Store<S>::R;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= p.nx || y >= p.ny) return;
  const size_t nodes = (size_t)p.nx * p.ny * p.nz;
  const size_t node = ((size_t)z * p.ny + y) * p.nx + x;
  R f[19], g[7];
#pragma unroll
  for (int i = 0; i < 19; ++i) f[i] = R(fin[i * nodes + node] - wrest3<double>(i));
#pragma unroll
  for (int i = 0; i < 7; ++i) g[i] = R(gin[i * nodes + node]);
  R r_, a_, b_, c_, d_;
  collide3(f, g, p, r_, a_, b_, c_, d_);
  const size_t idx = ((size_t)z * p.ny + y) * p.pitch + x;
#pragma unroll
  for (int i = 0; i < 19; ++i) Store<S>::st(fout + i * p.plane + idx, f[i]);
#pragma unroll
  for (int i = 0; i < 7; ++i) Store<S>::st(fout + (19 + i) * p.plane + idx, g[i]);
}

struct NodeState3 {
  double rho, ux, uy, uz, T;
};

template <typename S>
__device__ __forceinline__ NodeState3 node_state3(const S* __restrict__ s, size_t idx,
                                                  long long P, double gbeta, double Ts,
                                                  double Tref) {
  double f[19], g[7];
#pragma unroll
  for (int i = 0; i < 19; ++i) f[i] = (double)Store<S>::ld(s + i * P + idx);
#pragma unroll
  for (int i = 0; i < 7; ++i) g[i] = (double)Store<S>::ld(s + (19 + i) * P + idx);
  double drho = 0, jx = 0, jy = 0, jz = 0, Tr = 0;
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    drho += f[i];
    jx += kE3[i][0] * f[i];
    jy += kE3[i][1] * f[i];
    jz += kE3[i][2] * f[i];
  }
#pragma unroll
  for (int i = 0; i < 7; ++i) Tr += g[i];
  NodeState3 n;
  n.rho = 1.0 + drho;
  n.T = Tr + Ts;
  const double Fy = n.rho * gbeta * (n.T - Tref);
  n.ux = jx / n.rho;
  n.uy = (jy - 0.5 * Fy) / n.rho;
  n.uz = jz / n.rho;
  return n;
}

template <typename S>
__global__ void k_fields3(const S* __restrict__ s, P3<typename Store<S>::R> p, double gbeta,
                          double Ts, double Tref, double* rho, double* T, double* u, double* v,
                          double* w) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= p.nx || y >= p.ny) return;
  const NodeState3 n =
      node_state3(s, ((size_t)z * p.ny + y) * p.pitch + x, p.plane, gbeta, Ts, Tref);
  const size_t node = ((size_t)z * p.ny + y) * p.nx + x;
  if (rho) rho[node] = n.rho;
  if (T) T[node] = n.T;
  if (u) u[node] = n.ux;
  if (v) v[node] = n.uy;
  if (w) w[node] = n.uz;
}

template <typename S>
__global__ void k_pops3(const S* __restrict__ s, P3<typename Store<S>::R> p, double* f,
                        double* g) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= p.nx || y >= p.ny) return;
  const size_t nodes = (size_t)p.nx * p.ny * p.nz;
  const size_t node = ((size_t)z * p.ny + y) * p.nx + x;
  const size_t idx = ((size_t)z * p.ny + y) * p.pitch + x;
#pragma unroll
  for (int i = 0; i < 19; ++i)
    f[i * nodes + node] = (double)Store<S>::ld(s + i * p.plane + idx) + wrest3<double>(i);
#pragma unroll
  for (int i = 0; i < 7; ++i) g[i * nodes + node] = (double)Store<S>::ld(s + (19 + i) * p.plane + idx);
}

// Population sums and velocity of one node in the compute type of the storage
// (as the 2-D node_state_c): FP64 accumulation, arithmetic at the state's own
// precision.
template <typename R>
struct NodeC3 {
  R drho, ux, uy, uz, T;
};

template <typename S>
__device__ __forceinline__ NodeC3<typename Store<S>::R> node_state3_c(
    const S* __restrict__ s, size_t idx, long long P, typename Store<S>::R gbeta,
    typename Store<S>::R Ts, typename Store<S>::R Tref) {
  using R = typename Store<S>::R;
  R f[19], g[7];
#pragma unroll
  for (int i = 0; i < 19; ++i) f[i] = Store<S>::ld(s + i * P + idx);
#pragma unroll
  for (int i = 0; i < 7; ++i) g[i] = Store<S>::ld(s + (19 + i) * P + idx);
  R drho = 0, jx = 0, jy = 0, jz = 0, Tr = 0;
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    drho += f[i];
    jx += R(kE3[i][0]) * f[i];
    jy += R(kE3[i][1]) * f[i];
    jz += R(kE3[i][2]) * f[i];
  }
#pragma unroll
  for (int i = 0; i < 7; ++i) Tr += g[i];
  NodeC3<R> n;
  n.drho = drho;
  const R rho = R(1) + drho;
  n.T = Tr + Ts;
  const R Fy = rho * gbeta * (n.T - Tref);
  n.ux = jx / rho;
  n.uy = (jy - R(0.5) * Fy) / rho;
  n.uz = jz / rho;
  return n;
}

// Reductions (Sec. 4): FP64 volume sums and the wall-plane temperature sums of
// Eq. (17) with the wall-plane weights W_y W_z.  A block takes whole rows
// (y, z), its threads the columns.
template <typename S>
__global__ void __launch_bounds__(256)
    k_reduce3(const S* __restrict__ s, P3<typename Store<S>::R> p, double gbeta, double Ts,
              double T0,
              const double* __restrict__ Wx, const double* __restrict__ Wy,
              const double* __restrict__ Wz, double* partial) {
  using R = typename Store<S>::R;
  double acc[RED_COUNT];
#pragma unroll
  for (int k = 0; k < RED_COUNT; ++k) acc[k] = 0.0;
  const int rows = p.ny * p.nz;
  const R gb = R(gbeta), ts = R(Ts), t0 = R(T0);
  for (int row = (int)blockIdx.x; row < rows; row += (int)gridDim.x) {
    const int z = row / p.ny, y = row - z * p.ny;
    const double wp = Wy[y] * Wz[z];
    const size_t base = ((size_t)z * p.ny + y) * p.pitch;
    for (int x = threadIdx.x; x < p.nx; x += blockDim.x) {
      const NodeC3<R> n = node_state3_c(s, base + x, p.plane, gb, ts, t0);
      const double W = Wx[x] * wp;
      const R uv2 = n.ux * n.ux + n.uy * n.uy;
      const R u2 = uv2 + n.uz * n.uz;
      const R sp = sqrt(u2);
      acc[RED_MASS] += W * (1.0 + (double)n.drho);
      acc[RED_UT] += W * (double)(n.ux * (n.T - t0));
      acc[RED_SPEED] += W * (double)sp;
      acc[RED_UV2] += W * (double)uv2;
      acc[RED_U2] += W * (double)u2;
      const double T = (double)n.T;
      if (x == 0) acc[RED_HOT1] += wp * T;
      if (x == 1) acc[RED_HOT2] += wp * T;
      if (x == p.nx - 1) acc[RED_COLD1] += wp * T;
      if (x == p.nx - 2) acc[RED_COLD2] += wp * T;
      const bool finite = isfinite(n.drho) && isfinite(n.ux) && isfinite(n.uy) &&
                          isfinite(n.uz) && isfinite(n.T);
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

// Steady-state criterion (Sec. 3) in 3-D, as the 2-D kernel with (u, v, w, T*).
template <typename S>
__global__ void __launch_bounds__(256)
    k_steady3(const S* __restrict__ s, P3<typename Store<S>::R> p, double gbeta, double Ts,
              double T0, double dT, int have_snap, double* snap, double* partial) {
  double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  const long long nodes = (long long)p.nx * p.ny * p.nz;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nodes;
       k += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(k % p.nx);
    const long long r = k / p.nx;
    const int y = (int)(r % p.ny), z = (int)(r / p.ny);
    const NodeState3 n =
        node_state3(s, ((size_t)z * p.ny + y) * p.pitch + x, p.plane, gbeta, Ts, T0);
    const double Tn = (n.T - T0) / dT;
    double ou = 0.0, ov = 0.0, ow = 0.0, oT = 0.0;
    if (have_snap) {
      ou = snap[k];
      ov = snap[nodes + k];
      ow = snap[2 * nodes + k];
      oT = snap[3 * nodes + k];
    }
    a0 += sqrt((n.ux - ou) * (n.ux - ou) + (n.uy - ov) * (n.uy - ov) + (n.uz - ow) * (n.uz - ow));
    a1 += sqrt(ou * ou + ov * ov + ow * ow);
    a2 += fabs(Tn - oT);
    a3 += fabs(oT);
    snap[k] = n.ux;
    snap[nodes + k] = n.uy;
    snap[2 * nodes + k] = n.uz;
    snap[3 * nodes + k] = Tn;
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

dim3 block3() { return dim3(32, 8, 1); }
dim3 grid3(const Solver& s) { return dim3((s.n[0] + 31) / 32, (s.n[1] + 7) / 8, s.n[2]); }

template <template <typename> class Fn, typename... A>
cudaError_t dispatch3(Solver& s, A... a) {
  switch (s.precision) {
    case ISLBM_FP64: return Fn<double>::run(s, a...);
    case ISLBM_FP32: return Fn<float>::run(s, a...);
    case ISLBM_FP16DEV: return Fn<__half>::run(s, a...);
    case ISLBM_BF16DEV: return Fn<__nv_bfloat16>::run(s, a...);
  }
  return cudaErrorInvalidValue;
}

template <typename S>
struct Step3 {
  static cudaError_t run(Solver& s) {
    using R = typename Store<S>::R;
    const auto p = make_params3<R>(s);
    const S* in = static_cast<const S*>(s.buf[s.cur]);
    S* out = static_cast<S*>(s.buf[s.cur ^ 1]);
    if (s.uniform)
      k_step3<S, true><<<grid3(s), block3(), 0, s.stream>>>(in, out, p);
    else
      k_step3<S, false><<<grid3(s), block3(), 0, s.stream>>>(in, out, p);
    return cudaGetLastError();
  }
};

template <typename S>
struct InitFields3 {
  static cudaError_t run(Solver& s, const double* rho, const double* T, const double* u,
                         const double* v, const double* w) {
    using R = typename Store<S>::R;
    k_init_fields3<S><<<grid3(s), block3(), 0, s.stream>>>(static_cast<S*>(s.buf[s.cur]),
                                                          make_params3<R>(s), rho, T, u, v, w);
    return cudaGetLastError();
  }
};

template <typename S>
struct InitPops3 {
  static cudaError_t run(Solver& s, const double* f, const double* g) {
    using R = typename Store<S>::R;
    k_init_pops3<S><<<grid3(s), block3(), 0, s.stream>>>(static_cast<S*>(s.buf[s.cur]),
                                                        make_params3<R>(s), f, g);
    return cudaGetLastError();
  }
};

template <typename S>
struct Fields3 {
  static cudaError_t run(Solver& s, double* rho, double* T, double* u, double* v, double* w) {
    using R = typename Store<S>::R;
    k_fields3<S><<<grid3(s), block3(), 0, s.stream>>>(static_cast<const S*>(s.buf[s.cur]),
                                                     make_params3<R>(s), s.ph.gbeta, s.ph.Ts,
                                                     s.ph.T0, rho, T, u, v, w);
    return cudaGetLastError();
  }
};

template <typename S>
struct Pops3 {
  static cudaError_t run(Solver& s, double* f, double* g) {
    using R = typename Store<S>::R;
    k_pops3<S><<<grid3(s), block3(), 0, s.stream>>>(static_cast<const S*>(s.buf[s.cur]),
                                                   make_params3<R>(s), f, g);
    return cudaGetLastError();
  }
};

template <typename S>
struct Reduce3 {
  static cudaError_t run(Solver& s) {
    using R = typename Store<S>::R;
    k_reduce3<S><<<s.red_blocks, 256, 0, s.stream>>>(
        static_cast<const S*>(s.buf[s.cur]), make_params3<R>(s), s.ph.gbeta, s.ph.Ts, s.ph.T0,
        s.dax[0].W, s.dax[1].W, s.dax[2].W, s.dscratch);
    return cudaGetLastError();
  }
};

template <typename S>
struct Steady3 {
  static cudaError_t run(Solver& s) {
    using R = typename Store<S>::R;
    k_steady3<S><<<s.red_blocks, 256, 0, s.stream>>>(
        static_cast<const S*>(s.buf[s.cur]), make_params3<R>(s), s.ph.gbeta, s.ph.Ts, s.ph.T0,
        s.ph.dT, s.snap_valid ? 1 : 0, s.dsnap, s.dscratch);
    return cudaGetLastError();
  }
};

}  // namespace

cudaError_t launch_step_3d(Solver& s) {
  cudaError_t e = s.variant == KV_TMA_3D  ? launch_step_3d_tma(s)
                  : is_zm3d(s.variant)     ? launch_step_3d_zm(s)
                                           : dispatch3<Step3>(s);
  if (e == cudaSuccess) s.cur ^= 1;
  return e;
}

cudaError_t launch_init_fields_3d(Solver& s, const double* rho, const double* T,
                                  const double* u0, const double* u1, const double* u2) {
  return dispatch3<InitFields3>(s, rho, T, u0, u1, u2);
}

cudaError_t launch_init_populations_3d(Solver& s, const double* f, const double* g) {
  return dispatch3<InitPops3>(s, f, g);
}

cudaError_t launch_fields_3d(Solver& s, double* rho, double* T, double* u0, double* u1,
                             double* u2) {
  return dispatch3<Fields3>(s, rho, T, u0, u1, u2);
}

cudaError_t launch_populations_3d(Solver& s, double* f, double* g) {
  return dispatch3<Pops3>(s, f, g);
}

cudaError_t launch_reduce_3d(Solver& s) { return dispatch3<Reduce3>(s); }

cudaError_t launch_steady_3d(Solver& s) { return dispatch3<Steady3>(s); }

}  // namespace islbm
