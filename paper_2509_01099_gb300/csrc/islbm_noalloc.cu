// Reductions for callers that cannot allocate device memory.
//
// islbm_reduce_noalloc computes what islbm_reduce computes (Nu, Re, mass, ...)
// for a 2-D cavity state that lives entirely in the caller's device memory,
// without a handle and without allocating anything.  Its scratch (per-block
// partial sums and the finished result) is the file-scope device array below:
// every GPU that loads the library holds it until the process exits.
#include <cmath>
#include <cstring>

#include "islbm_internal.h"
#include "islbm_store.cuh"

namespace islbm {
void set_last_error_static(const char* msg);
}

namespace {

constexpr int kNodesPerBlock = 16384;   // nodes reduced by one block
constexpr int kMaxBlocks = 8192;        // partial rows in the scratch array
constexpr long long kMaxNodes = (long long)kNodesPerBlock * kMaxBlocks;   // 134,217,728
constexpr int kRow = islbm::RED_STRIDE;  // doubles per partial row
constexpr int kResults = 12;            // finished values written by the last kernel

// 8193 rows of 16 doubles: the partials of at most kMaxBlocks blocks, then the
// result row.  1 MiB.
static __device__ __align__(256) double g_noalloc_scratch[(kMaxBlocks + 1) * kRow];

// Per-node sums of the full FP64 post-collision populations ([9][ny][nx] and
// [5][ny][nx]), same slots as the handle's reduction.  Lattice coordinates and
// the Eq. (18) widths come from the ghost-node meshes: W_j = (xi_{j+1} - xi_{j-1}) / (2 lu),
// with each axis's own lattice unit lu = xi_1 - xi_0 (the finish kernel rejects
// meshes whose axes differ in it).
__global__ void __launch_bounds__(256)
    k_noalloc_partials(const double* __restrict__ f, const double* __restrict__ g, int nx,
                       int ny, const double* __restrict__ xi_x, const double* __restrict__ xi_y,
                       double u_f, double Ts, double T0, double* scratch) {
  using namespace islbm;
  double acc[RED_COUNT];
#pragma unroll
  for (int k = 0; k < RED_COUNT; ++k) acc[k] = 0.0;
  const long long nodes = (long long)nx * ny;
  const long long begin = (long long)blockIdx.x * kNodesPerBlock;
  const long long end = begin + kNodesPerBlock < nodes ? begin + kNodesPerBlock : nodes;
  const double lu = xi_x[1] - xi_x[0], lu_y = xi_y[1] - xi_y[0];
  // g beta = u_f^2 / L, L the cavity height in lattice units (Table 1)
  const double gbeta = u_f * u_f / ((xi_y[ny] - xi_y[1]) / lu_y + 1.0);
  const int mL = (nx % 2 == 0) ? nx / 2 - 1 : (nx - 1) / 2 - 1;
  const int mR = (nx % 2 == 0) ? nx / 2 : (nx + 1) / 2;
  const int mC = (nx % 2 == 0) ? -1 : (nx - 1) / 2;
  for (long long k = begin + threadIdx.x; k < end; k += blockDim.x) {
    const int y = (int)(k / nx), x = (int)(k - (long long)y * nx);
    double rho = 0, jx = 0, jy = 0, T = 0;
    const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const double v = f[(size_t)i * nodes + k];
      rho += v;
      jx += ex[i] * v;
      jy += ey[i] * v;
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) T += g[(size_t)i * nodes + k];
    T += Ts;                      // the populations carry T - T_s
    const double Tr = T - T0;
    const double Fy = rho * gbeta * Tr;
    const double ux = jx / rho, uy = (jy - 0.5 * Fy) / rho;
    const double wx = (xi_x[x + 2] - xi_x[x]) / (2.0 * lu);
    const double wy = (xi_y[y + 2] - xi_y[y]) / (2.0 * lu_y);
    const double W = wx * wy;
    const double u2 = ux * ux + uy * uy, sp = sqrt(u2);
    acc[RED_MASS] += W * rho;
    acc[RED_UT] += W * ux * Tr;
    acc[RED_SPEED] += W * sp;
    acc[RED_UV2] += W * u2;
    acc[RED_U2] += W * u2;
    if (x == 0) acc[RED_HOT1] += wy * T;
    if (x == 1) acc[RED_HOT2] += wy * T;
    if (x == nx - 1) acc[RED_COLD1] += wy * T;
    if (x == nx - 2) acc[RED_COLD2] += wy * T;
    if (x == mL) acc[RED_MIDTL] += wy * T;
    if (x == mR) acc[RED_MIDTR] += wy * T;
    if (mC < 0 && (x == mL || x == mR)) acc[RED_MIDCONV] += 0.5 * wy * ux * Tr;
    if (x == mC) acc[RED_MIDCONV] += wy * ux * Tr;
    const bool finite = isfinite(rho) && isfinite(ux) && isfinite(uy) && isfinite(T);
    if (!finite) acc[RED_NONFINITE] += 1.0;
    acc[RED_MAXSPEED] = fmax(acc[RED_MAXSPEED], finite ? sp : 0.0);
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
    for (int w = 1; w < 8; ++w) v = (k == RED_MAXSPEED) ? fmax(v, sh[w][k]) : v + sh[w][k];
    scratch[(size_t)blockIdx.x * kRow + k] = v;   // every slot the finish reads is written here
  }
}

struct Phys {
  double Ra, Pr, u_f, T_hot, T_cold, T0, dT;
};

// Fixed-order sum of the partial rows, then the finished values (Sec. 3,
// Eq. (17), Eq. (18)) into the result row.  Its last entry flags meshes that
// islbm_create would refuse: not strictly increasing, or axes with different
// lattice units.
__global__ void k_noalloc_finish(double* scratch, int blocks, int nx, int ny,
                                 const double* __restrict__ xi_x, const double* __restrict__ xi_y,
                                 Phys ph) {
  using namespace islbm;
  __shared__ double sums[RED_COUNT];
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = threadIdx.x; j <= nx; j += blockDim.x)
    if (!(xi_x[j + 1] > xi_x[j])) bad = 1;
  for (int j = threadIdx.x; j <= ny; j += blockDim.x)
    if (!(xi_y[j + 1] > xi_y[j])) bad = 1;
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k < RED_COUNT) {
    double v = 0.0;
    for (int b = lane; b < blocks; b += 32) {
      const double x = scratch[(size_t)b * kRow + k];
      v = (k == RED_MAXSPEED) ? fmax(v, x) : v + x;
    }
    v = (k == RED_MAXSPEED) ? warp_max(v) : warp_sum(v);
    if (lane == 0) sums[k] = v;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double lu = xi_x[1] - xi_x[0], lu_y = xi_y[1] - xi_y[0];
  double* res = scratch + (size_t)kMaxBlocks * kRow;
  res[11] = (bad || !(fabs(lu_y - lu) <= 1e-9 * lu)) ? 1.0 : 0.0;
  auto X = [&](const double* xi, int j) { return (xi[j] - xi[0]) / (xi == xi_y ? lu_y : lu); };
  const double Lx = X(xi_x, nx) - X(xi_x, 1) + 1.0;
  const double L = X(xi_y, ny) - X(xi_y, 1) + 1.0;
  const double vol = Lx * L, area = L;
  const double sq = sqrt(ph.Ra * ph.Pr);
  res[0] = sq * sums[RED_UT] / (ph.u_f * ph.dT * vol) + 1.0;
  double q = (X(xi_x, 2) - X(xi_x, 1)) / (X(xi_x, 1) - X(xi_x, 0));
  double den = q * (2 * q + 1);
  const double hot = -4 * q * (q + 1) / den * ph.T_hot * area +
                     (2 * q + 1) * (2 * q + 1) / den * sums[RED_HOT1] - sums[RED_HOT2] / den;
  q = (X(xi_x, nx) - X(xi_x, nx - 1)) / (X(xi_x, nx + 1) - X(xi_x, nx));
  den = q * (2 * q + 1);
  const double cold = 4 * q * (q + 1) / den * ph.T_cold * area -
                      (2 * q + 1) * (2 * q + 1) / den * sums[RED_COLD1] + sums[RED_COLD2] / den;
  res[1] = -hot * L / (ph.dT * area);
  res[2] = -cold * L / (ph.dT * area);
  const double inv_dx = (nx % 2 == 0)
                            ? 1.0 / (X(xi_x, nx / 2 + 1) - X(xi_x, nx / 2))
                            : 1.0 / (X(xi_x, (nx + 1) / 2 + 1) - X(xi_x, (nx + 1) / 2 - 1));
  res[3] = (sq * sums[RED_MIDCONV] / (ph.u_f * ph.dT) -
            L * (sums[RED_MIDTR] - sums[RED_MIDTL]) * inv_dx / ph.dT) / L;
  res[4] = sqrt(ph.Ra / ph.Pr) * sqrt(sums[RED_U2] / vol) / ph.u_f;
  res[5] = sqrt(ph.Ra / ph.Pr) * sqrt(sums[RED_UV2] / vol) / ph.u_f;
  res[10] = sqrt(ph.Ra / ph.Pr) * sums[RED_SPEED] / (ph.u_f * vol);
  res[6] = sums[RED_MASS];
  res[7] = 0.5 * sums[RED_U2];
  res[8] = sums[RED_MAXSPEED] / ph.u_f;
  res[9] = sums[RED_NONFINITE];
}

}  // namespace

extern "C" islbm_status islbm_reduce_noalloc(const double* f, const double* g, int nx, int ny,
                                             const double* xi_x, const double* xi_y, double Ra,
                                             double Pr, const islbm_params* opt, void* stream,
                                             islbm_reductions* out) {
  using islbm::set_last_error_static;
  if (!f || !g || !xi_x || !xi_y || !out) {
    set_last_error_static("islbm_reduce_noalloc: NULL argument");
    return ISLBM_ERR_ARG;
  }
  if (nx < 4 || ny < 4) {
    set_last_error_static("islbm_reduce_noalloc: need at least 4 nodes per axis");
    return ISLBM_ERR_ARG;
  }
  if ((long long)nx * ny > kMaxNodes) {
    set_last_error_static(
        "islbm_reduce_noalloc: state too large for the static scratch "
        "(at most 134217728 nodes = 8192 blocks of 16384)");
    return ISLBM_ERR_ARG;
  }
  if (!(Ra > 0) || !(Pr > 0)) {
    set_last_error_static("islbm_reduce_noalloc: Ra and Pr must be positive");
    return ISLBM_ERR_ARG;
  }
  islbm_params prm;
  islbm_default_params(&prm);
  if (opt) prm = *opt;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
    set_last_error_static("islbm_reduce_noalloc: no usable CUDA device");
    return ISLBM_ERR_CUDA;
  }
  // The host-side name of the array is only a stand-in: the kernels need its
  // device address on the current device.  It is looked up on every call (cheap
  // once the module is loaded), so a context created again after
  // cudaDeviceReset, where the array may have moved, is served correctly.
  void* sym = nullptr;
  if (cudaGetSymbolAddress(&sym, g_noalloc_scratch) != cudaSuccess || !sym) {
    set_last_error_static("islbm_reduce_noalloc: cudaGetSymbolAddress failed");
    return ISLBM_ERR_CUDA;
  }
  double* scratch = static_cast<double*>(sym);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long nodes = (long long)nx * ny;
  const int blocks = (int)((nodes + kNodesPerBlock - 1) / kNodesPerBlock);
  const double u_f = prm.Ma / std::sqrt(3.0);
  Phys ph;
  ph.Ra = Ra;
  ph.Pr = Pr;
  ph.u_f = u_f;
  ph.T_hot = prm.T_hot;
  ph.T_cold = prm.T_cold;
  ph.T0 = prm.reference == ISLBM_TREF_COLD ? prm.T_cold : 0.5 * (prm.T_hot + prm.T_cold);
  ph.dT = prm.T_hot != prm.T_cold ? prm.T_hot - prm.T_cold : 1.0;
  k_noalloc_partials<<<blocks, 256, 0, st>>>(f, g, nx, ny, xi_x, xi_y, u_f,
                                             0.5 * (prm.T_hot + prm.T_cold), ph.T0, scratch);
  k_noalloc_finish<<<1, 32 * islbm::RED_COUNT, 0, st>>>(scratch, blocks, nx, ny, xi_x, xi_y, ph);
  double res[kResults];
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(res, scratch + (size_t)kMaxBlocks * kRow, sizeof(res),
                      cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    set_last_error_static("islbm_reduce_noalloc: kernel launch or copy failed");
    return ISLBM_ERR_CUDA;
  }
  if (res[11] != 0.0) {
    set_last_error_static(
        "islbm_reduce_noalloc: meshes must be strictly increasing and share one lattice unit");
    return ISLBM_ERR_ARG;
  }
  std::memset(out, 0, sizeof(*out));
  out->Nu = res[0];
  out->Nu_hot = res[1];
  out->Nu_cold = res[2];
  out->Nu_middle = res[3];
  out->Re = res[4];
  out->Re_uv = res[5];
  out->mass = res[6];
  out->ke = res[7];
  out->max_speed = res[8];
  out->nonfinite = res[9];
  out->Re_mean = res[10];
  if (res[9] > 0 || !std::isfinite(res[0])) {
    set_last_error_static("islbm_reduce_noalloc: non-finite values in the state");
    return ISLBM_ERR_DIVERGED;
  }
  return ISLBM_OK;
}
