// Pipelined 3-D step kernel (D3Q19 + D3Q7; Sec. 2.1 - 2.3, Sec. 4).
//
// A CTA owns a 32 x 4 x 2 tile of nodes (one node per consumer thread) and
// walks its share of the tiles persistently.  The 26 population planes of a
// tile are staged in opposite pairs (0), (1,2), (3,4), ... (17,18), (19),
// (20,21), (22,23), (24,25): one 4-D TMA copy per pair brings the tile plus a
// one-node halo along the axes the pair moves on (rounded out to a 16-byte
// chunk in x; one descriptor per box shape) into a ring of shared-memory
// slots.  A producer warp issues the copies as slots
// free up; the eight consumer warps take each pair as it lands, pull both
// populations of their node by the separable quadratic interpolation of
// Sec. 2.2 (or the wall rules of Sec. 2.3, which read the opposite population
// of the same pair), and after the last pair collide and store.  The copy of a
// pair is tracked by a "full" mbarrier (transaction bytes) and its release by
// an "empty" mbarrier (one arrival per consumer warp).  Every wait is bounded:
// a wait that gives up raises the CTA's abort flag and the device error flag,
// the producer stops issuing and waits (bounded) for its copies in flight,
// and the CTA returns.
//
// The interpolation stencils are node-centred (base = node - 1, clamped at the
// walls), so the staged window of a tile starts one node before it, shifted
// inwards at the far walls: it needs n_y >= tile height + 2 and n_z >= tile
// depth + 2 (step_3d_tma_fits).
#include "islbm_d3_common.cuh"
#include "islbm_tma.cuh"

namespace islbm {
namespace {

constexpr int kT3X = 32, kT3Y = 4, kT3Z = 2;
constexpr int kConsumers3 = kT3X * kT3Y * kT3Z;   // one consumer thread per node of a tile
constexpr int kConsumerWarps3 = kConsumers3 / 32;
constexpr int kThreads3 = kConsumers3 + 32;       // + one producer warp
constexpr int kPairs3 = 14;
constexpr int kStages3 = 7;
constexpr int kGroup3 = 2;                        // pairs pulled together by the consumers
static_assert(kPairs3 % kGroup3 == 0 && kStages3 >= 2 * kGroup3, "ring too short for a group");

template <typename S>
struct Geom3 {
  static constexpr int HX = 16 / (int)sizeof(S);
  // window extents with a halo on every axis
  static constexpr int SW = kT3X + 2 * HX, SH = kT3Y + 2, SD = kT3Z + 2;
  // a slot holds the largest pair box in use: no D3Q19 / D3Q7 velocity moves
  // along all three axes, so a box has halos on at most two
  static constexpr unsigned XY = 2u * SW * SH * kT3Z * (unsigned)sizeof(S);
  static constexpr unsigned XZ = 2u * SW * kT3Y * SD * (unsigned)sizeof(S);
  static constexpr unsigned YZ = 2u * kT3X * SH * SD * (unsigned)sizeof(S);
  static constexpr unsigned SLOT = XY > XZ ? (XY > YZ ? XY : YZ) : (XZ > YZ ? XZ : YZ);
  // ring slots, then the barriers (and the abort flag), then the packed
  // interpolation tables of the three axes when they fit
  static constexpr size_t ring_bytes() { return (size_t)kStages3 * SLOT; }
  // full[kStages3], empty[kStages3] and the abort flag, rounded up to 128 bytes
  static constexpr size_t bar_bytes() {
    return (2 * kStages3 * sizeof(uint64_t) + sizeof(int) + 127) / 128 * 128;
  }
  static size_t smem_bytes(size_t table_bytes) { return ring_bytes() + bar_bytes() + table_bytes; }
};
static_assert(Geom3<float>::SLOT % 128 == 0 && Geom3<__half>::SLOT % 128 == 0,
              "TMA destinations must stay 128-byte aligned");
static_assert(Geom3<float>::bar_bytes() >= 2 * kStages3 * sizeof(uint64_t) + sizeof(int),
              "the barrier area must hold both barrier arrays and the abort flag");

// Box of a pair whose populations move along x / y / z (HXa, HYa, HZa): a
// one-node halo only along the moving axes (x rounded out to 16 bytes).
template <typename S, bool HXa, bool HYa, bool HZa>
struct Box3 {
  static constexpr int W = kT3X + (HXa ? 2 * Geom3<S>::HX : 0);
  static constexpr int H = kT3Y + (HYa ? 2 : 0);
  static constexpr int D = kT3Z + (HZa ? 2 : 0);
  static constexpr int POP = W * H * D;
  static constexpr unsigned BYTES = 2u * POP * (unsigned)sizeof(S);
};

// box type of pair j: bit 0 x, bit 1 y, bit 2 z
__host__ __device__ constexpr int pair_type(int j) {
  return (j == 0 || j == 10) ? 0
         : (j == 1 || j == 11) ? 1
         : (j == 2 || j == 12) ? 2
         : (j == 3 || j == 13) ? 4
         : (j == 4 || j == 5)  ? 3
         : (j == 6 || j == 7)  ? 5
                               : 6;
}

template <typename S>
__host__ __device__ constexpr unsigned box_bytes(int type) {
  return 2u * (unsigned)(kT3X + ((type & 1) ? 2 * Geom3<S>::HX : 0)) *
         (unsigned)(kT3Y + ((type & 2) ? 2 : 0)) * (unsigned)(kT3Z + ((type & 4) ? 2 : 0)) *
         (unsigned)sizeof(S);
}

template <typename S>
constexpr bool boxes_fit_slot() {
  for (int q = 0; q < kPairs3; ++q)
    if (pair_type(q) == 7 || box_bytes<S>(pair_type(q)) > Geom3<S>::SLOT) return false;
  return true;
}
static_assert(boxes_fit_slot<float>() && boxes_fit_slot<__half>() &&
                  boxes_fit_slot<__nv_bfloat16>(),
              "every pair box fits a ring slot");

// One TMA descriptor per box type (index = type bits) of the input buffer.
struct alignas(64) Maps3 {
  CUtensorMap m[7];
};

// first population of pair j
__device__ __forceinline__ int pair_first(int j) {
  return j == 0 ? 0 : (j <= 9 ? 2 * j - 1 : (j == 10 ? 19 : 2 * j - 2));
}

// Bounded wait (the limits of mbar_wait) that also gives up as soon as another
// thread raised the abort flag.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, unsigned phase,
                                              const volatile int* abort) {
  if (mbar_try_wait(bar, phase)) return true;
  const unsigned long long t0 = global_ns();
  for (int i = 0; i < kWaitMaxPolls; ++i) {
    if (mbar_try_wait(bar, phase)) return true;
    if ((i & 63) == 63 && (*abort || global_ns() - t0 > kWaitLimitNs)) return false;
  }
  return false;
}

// Geometry of one node inside a staged window.
template <typename R>
struct Node3 {
  int lxh, lyh, lzh;              // node position in a window with a halo on that axis
  int lxn, lyn, lzn;              // ... and without
  float4 tx[2], ty[2], tz[2];     // packed tables (+ / - direction) per axis
  int bx[2], by[2], bz[2];        // stencil bases in halo-window coordinates
};

// Value of the node itself in a plane staged with box (HXa, HYa, HZa).
template <typename S, typename R, bool HXa, bool HYa, bool HZa>
__device__ __forceinline__ R own_w(const S* __restrict__ pl, const Node3<R>& n) {
  using B = Box3<S, HXa, HYa, HZa>;
  const int x = HXa ? n.lxh : n.lxn, y = HYa ? n.lyh : n.lyn, z = HZa ? n.lzh : n.lzn;
  if (!(ISLBM_IN_WINDOW(z, B::D) && ISLBM_IN_WINDOW(y, B::H) && ISLBM_IN_WINDOW(x, B::W)))
    return R(0);
  return (R)to_f(pl[(z * B::H + y) * B::W + x]);
}

// Pull of population plane `pl` moving with (CX, CY, CZ) at the node; the same
// operation order as the direct kernel's pull3 (first moving axis inside).
template <typename S, typename R, int CX, int CY, int CZ, bool UNI>
__device__ __forceinline__ R pull_w(const S* __restrict__ pl, const Node3<R>& n) {
  using B = Box3<S, CX != 0, CY != 0, CZ != 0>;
  auto at = [&](int z, int y, int x) -> R {
    if (!(ISLBM_IN_WINDOW(z, B::D) && ISLBM_IN_WINDOW(y, B::H) && ISLBM_IN_WINDOW(x, B::W)))
      return R(0);
    return (R)to_f(pl[(z * B::H + y) * B::W + x]);
  };
  // node coordinates in this box (halo coordinates along the moving axes)
  const int lx = CX != 0 ? n.lxh : n.lxn, ly = CY != 0 ? n.lyh : n.lyn;
  const int lz = CZ != 0 ? n.lzh : n.lzn;
  if (UNI || (CX == 0 && CY == 0 && CZ == 0)) return at(lz - CZ, ly - CY, lx - CX);
  constexpr int kx = CX > 0 ? 0 : 1, ky = CY > 0 ? 0 : 1, kz = CZ > 0 ? 0 : 1;
  if (CX != 0 && CY == 0 && CZ == 0) {
    const float4 t = n.tx[kx];
    const int b = n.bx[kx];
    return dot3(t, at(lz, ly, b), at(lz, ly, b + 1), at(lz, ly, b + 2));
  }
  if (CX == 0 && CY != 0 && CZ == 0) {
    const float4 t = n.ty[ky];
    const int b = n.by[ky];
    return dot3(t, at(lz, b, lx), at(lz, b + 1, lx), at(lz, b + 2, lx));
  }
  if (CX == 0 && CY == 0 && CZ != 0) {
    const float4 t = n.tz[kz];
    const int b = n.bz[kz];
    return dot3(t, at(b, ly, lx), at(b + 1, ly, lx), at(b + 2, ly, lx));
  }
  R acc = R(0);
  if (CZ == 0) {   // x inside, y outside
    const float4 a = n.tx[kx], w = n.ty[ky];
    const int b0 = n.bx[kx], b1 = n.by[ky];
    const R wl[3] = {w.x, w.y, w.z};
#pragma unroll
    for (int l = 0; l < 3; ++l)
      acc = lfma(wl[l], dot3(a, at(lz, b1 + l, b0), at(lz, b1 + l, b0 + 1), at(lz, b1 + l, b0 + 2)),
                 acc);
  } else if (CY == 0) {   // x inside, z outside
    const float4 a = n.tx[kx], w = n.tz[kz];
    const int b0 = n.bx[kx], b1 = n.bz[kz];
    const R wl[3] = {w.x, w.y, w.z};
#pragma unroll
    for (int l = 0; l < 3; ++l)
      acc = lfma(wl[l], dot3(a, at(b1 + l, ly, b0), at(b1 + l, ly, b0 + 1), at(b1 + l, ly, b0 + 2)),
                 acc);
  } else {   // y inside, z outside
    const float4 a = n.ty[ky], w = n.tz[kz];
    const int b0 = n.by[ky], b1 = n.bz[kz];
    const R wl[3] = {w.x, w.y, w.z};
#pragma unroll
    for (int l = 0; l < 3; ++l)
      acc = lfma(wl[l], dot3(a, at(b1 + l, b0, lx), at(b1 + l, b0 + 1, lx), at(b1 + l, b0 + 2, lx)),
                 acc);
  }
  return acc;
}

// three CTAs per SM (72 registers a thread): the consumers are latency-bound,
// and the third CTA gives 24 consumer warps per SM (measured 1.14x over two)
constexpr int kMinBlocks3 = kThreads3 <= 320 ? 3 : 1;
static_assert(kT3X % 32 == 0 && kConsumers3 % 32 == 0, "tiles are whole warps along x");

template <typename S, bool UNI>
__global__ void __launch_bounds__(kThreads3, kMinBlocks3)
    k_step3_tma(const __grid_constant__ Maps3 maps, S* __restrict__ fout, P3<float> p,
                int* err, int tables_in_smem) {
  using G = Geom3<S>;
  using St = Store<S>;
  using R = float;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + G::ring_bytes());
  uint64_t* empty = full + kStages3;
  volatile int* abort = reinterpret_cast<volatile int*>(empty + kStages3);
  // packed tables [axis][direction][node] in shared memory (read once per CTA)
  // layout: x+ x- y+ y- z+ z-, each n_axis entries
  float4* tab = reinterpret_cast<float4*>(smem_raw + G::ring_bytes() + G::bar_bytes());
  const int toff[3] = {0, 2 * p.nx, 2 * (p.nx + p.ny)};
  if (tables_in_smem) {
    const int na[3] = {p.nx, p.ny, p.nz};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int k = 0; k < 2; ++k)
        for (int i = threadIdx.x; i < na[a]; i += blockDim.x)
          tab[toff[a] + k * na[a] + i] = __ldg(p.pk[a][k] + i);
  }

  const int ntx = (p.nx + kT3X - 1) / kT3X, nty = (p.ny + kT3Y - 1) / kT3Y;
  const int ntz = (p.nz + kT3Z - 1) / kT3Z;
  const int ntiles = ntx * nty * ntz;
  auto origin = [&](int t, int& x0, int& y0, int& z0, int& sy0, int& sz0) {
    const int tz = t / (ntx * nty);
    const int r = t - tz * ntx * nty;
    const int ty = r / ntx;
    x0 = (r - ty * ntx) * kT3X;
    y0 = ty * kT3Y;
    z0 = tz * kT3Z;
    sy0 = max(0, min(y0 - 1, p.ny - G::SH));
    sz0 = max(0, min(z0 - 1, p.nz - G::SD));
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages3; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps3);
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == kConsumerWarps3) {
    // ---------------- producer ----------------
    if (lane == 0) {
      unsigned j = 0;   // pair jobs issued (32-bit: cheap slot and phase arithmetic)
      bool stop = false;
      for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
        int x0, y0, z0, sy0, sz0;
        origin(t, x0, y0, z0, sy0, sz0);
        for (int q = 0; q < kPairs3; ++q, ++j) {
          const int s = (int)(j % (unsigned)kStages3);
          if (j >= (unsigned)kStages3 &&
              !wait_or_abort(&empty[s], ((j / (unsigned)kStages3) - 1u) & 1u, abort)) {
            if (!*abort) atomicExch(err, 1);
            *abort = 1;
            stop = true;
            break;
          }
          if (*abort) {
            stop = true;
            break;
          }
          const int ty = pair_type(q);
          mbar_expect_tx(&full[s], box_bytes<S>(ty));
          tma_load_4d(smem_raw + (size_t)s * G::SLOT, &maps.m[ty], (ty & 1) ? x0 - G::HX : x0,
                      (ty & 2) ? sy0 : y0, (ty & 4) ? sz0 : z0, pair_first(q), &full[s]);
        }
      }
      // wait (bounded) for the last copy issued into every slot
      for (int s = 0; s < kStages3 && (unsigned)s < j; ++s) {
        const unsigned last = j - 1u - ((j - 1u - (unsigned)s) % (unsigned)kStages3);
        mbar_wait(&full[s], (last / (unsigned)kStages3) & 1u);
      }
    }
  } else {
    // ---------------- consumers ----------------
    const int c = threadIdx.x % kT3X, ry = (threadIdx.x / kT3X) % kT3Y;
    const int rz = threadIdx.x / (kT3X * kT3Y);
    const long long P = p.plane;
    // ring slot and completed ring cycles at the first pair of the current tile
    unsigned s0 = 0, c0 = 0;
    bool stop = false;
    for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
      int x0, y0, z0, sy0, sz0;
      origin(t, x0, y0, z0, sy0, sz0);
      const int x = x0 + c, y = y0 + ry, z = z0 + rz;
      const bool valid = x < p.nx && y < p.ny && z < p.nz;
      const int xc = min(x, p.nx - 1), yc = min(y, p.ny - 1), zc = min(z, p.nz - 1);
      Node3<R> n;
      n.lxh = xc - (x0 - G::HX);
      n.lyh = yc - sy0;
      n.lzh = zc - sz0;
      n.lxn = xc - x0;
      n.lyn = yc - y0;
      n.lzn = zc - z0;
      if (!UNI) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          if (tables_in_smem) {
            n.tx[k] = tab[toff[0] + k * p.nx + xc];
            n.ty[k] = tab[toff[1] + k * p.ny + yc];
            n.tz[k] = tab[toff[2] + k * p.nz + zc];
          } else {
            n.tx[k] = __ldg(p.pk[0][k] + xc);
            n.ty[k] = __ldg(p.pk[1][k] + yc);
            n.tz[k] = __ldg(p.pk[2][k] + zc);
          }
          n.bx[k] = __float_as_int(n.tx[k].w) - (x0 - G::HX);
          n.by[k] = __float_as_int(n.ty[k].w) - sy0;
          n.bz[k] = __float_as_int(n.tz[k].w) - sz0;
        }
      }
      const bool wxm = xc == 0, wxp = xc == p.nx - 1, wym = yc == 0, wyp = yc == p.ny - 1;
      const bool wzm = zc == 0, wzp = zc == p.nz - 1;
      R f[19], g[7];
      // ring slot and phase of pair q of this tile
      auto slot_of = [&](int q) { return (s0 + (unsigned)q) % (unsigned)kStages3; };
      auto phase_of = [&](int q) { return (c0 + (s0 + (unsigned)q) / (unsigned)kStages3) & 1u; };
#pragma unroll
      for (int qg = 0; qg < kPairs3; qg += kGroup3) {
        // wait for every pair of the group, then pull them together (their
        // shared-memory reads are independent, which gives each warp more
        // loads in flight)
        bool ok = true;
#pragma unroll
        for (int u = 0; u < kGroup3; ++u) {
          ok = ok && wait_or_abort(&full[slot_of(qg + u)], phase_of(qg + u), abort);
        }
        if (!ok) {
          if (!*abort) atomicExch(err, 1);
          *abort = 1;
          stop = true;
          break;
        }
#pragma unroll
        for (int u = 0; u < kGroup3; ++u) {
        const int q = qg + u;
        const int s = (int)slot_of(q);
        const S* a = reinterpret_cast<const S*>(smem_raw + (size_t)s * G::SLOT);
#define PW(pl, cx, cy, cz) pull_w<S, R, cx, cy, cz, UNI>(pl, n)
#define PAIR(X, Y, Z)                                  \
  constexpr bool hx = X, hy = Y, hz = Z;               \
  const S* b = a + Box3<S, hx, hy, hz>::POP;           \
  auto own = [&](const S* pl) -> R { return own_w<S, R, hx, hy, hz>(pl, n); };
        switch (q) {
          case 0: { PAIR(false, false, false) (void)b; f[0] = own(a); } break;
          case 1: {
            PAIR(true, false, false)
            f[1] = wxm ? own(b) : PW(a, 1, 0, 0);
            f[2] = wxp ? own(a) : PW(b, -1, 0, 0);
          } break;
          case 2: {
            PAIR(false, true, false)
            f[3] = wym ? own(b) : PW(a, 0, 1, 0);
            f[4] = wyp ? own(a) : PW(b, 0, -1, 0);
          } break;
          case 3: {
            PAIR(false, false, true)
            f[5] = wzm ? own(b) : PW(a, 0, 0, 1);
            f[6] = wzp ? own(a) : PW(b, 0, 0, -1);
          } break;
          case 4: {
            PAIR(true, true, false)
            f[7] = (wxm || wym) ? own(b) : PW(a, 1, 1, 0);
            f[8] = (wxp || wyp) ? own(a) : PW(b, -1, -1, 0);
          } break;
          case 5: {
            PAIR(true, true, false)
            f[9] = (wxm || wyp) ? own(b) : PW(a, 1, -1, 0);
            f[10] = (wxp || wym) ? own(a) : PW(b, -1, 1, 0);
          } break;
          case 6: {
            PAIR(true, false, true)
            f[11] = (wxm || wzm) ? own(b) : PW(a, 1, 0, 1);
            f[12] = (wxp || wzp) ? own(a) : PW(b, -1, 0, -1);
          } break;
          case 7: {
            PAIR(true, false, true)
            f[13] = (wxm || wzp) ? own(b) : PW(a, 1, 0, -1);
            f[14] = (wxp || wzm) ? own(a) : PW(b, -1, 0, 1);
          } break;
          case 8: {
            PAIR(false, true, true)
            f[15] = (wym || wzm) ? own(b) : PW(a, 0, 1, 1);
            f[16] = (wyp || wzp) ? own(a) : PW(b, 0, -1, -1);
          } break;
          case 9: {
            PAIR(false, true, true)
            f[17] = (wym || wzp) ? own(b) : PW(a, 0, 1, -1);
            f[18] = (wyp || wzm) ? own(a) : PW(b, 0, -1, 1);
          } break;
          case 10: { PAIR(false, false, false) (void)b; g[0] = own(a); } break;
          case 11: {
            PAIR(true, false, false)
            g[1] = wxm ? p.abb_hot - own(b) : PW(a, 1, 0, 0);
            g[2] = wxp ? p.abb_cold - own(a) : PW(b, -1, 0, 0);
          } break;
          case 12: {
            PAIR(false, true, false)
            g[3] = wym ? own(b) : PW(a, 0, 1, 0);
            g[4] = wyp ? own(a) : PW(b, 0, -1, 0);
          } break;
          default: {
            PAIR(false, false, true)
            g[5] = wzm ? own(b) : PW(a, 0, 0, 1);
            g[6] = wzp ? own(a) : PW(b, 0, 0, -1);
          } break;
        }
#undef PAIR
#undef PW
        }
        __syncwarp();
        if (lane == 0)
#pragma unroll
          for (int u = 0; u < kGroup3; ++u) mbar_arrive(&empty[slot_of(qg + u)]);
      }
      if (stop) break;
      {
        const unsigned e = s0 + (unsigned)kPairs3;
        s0 = e % (unsigned)kStages3;
        c0 += e / (unsigned)kStages3;
      }
      if (valid) {
        R rho, ux, uy, uz, T;
        collide3(f, g, p, rho, ux, uy, uz, T);
        const size_t idx = ((size_t)z * p.ny + y) * p.pitch + x;
        unsigned r = sr_seed(idx, p.step);
#pragma unroll
        for (int i = 0; i < 19; ++i) St::st_sr(fout + i * P + idx, f[i], sr_next(r));
#pragma unroll
        for (int i = 0; i < 7; ++i) St::st_sr(fout + (19 + i) * P + idx, g[i], sr_next(r));
      }
    }
  }
  __syncthreads();   // the producer has drained its copies before the CTA leaves
}

template <typename S, bool UNI>
cudaError_t launch3_tma(Solver& s, int blocks) {
  using G = Geom3<S>;
  // the tables go to shared memory when the CTAs per SM still fit
  constexpr size_t kMaxSmem = kMinBlocks3 == 3 ? 74 * 1024 : 227 * 1024;
  const size_t table_bytes = (size_t)2 * (s.n[0] + s.n[1] + s.n[2]) * sizeof(float4);
  const int in_smem = G::smem_bytes(table_bytes) <= kMaxSmem ? 1 : 0;
  const size_t smem = G::smem_bytes(in_smem ? table_bytes : 0);
  const cudaError_t e = launch_setup_once(
      reinterpret_cast<const void*>(k_step3_tma<S, UNI>),
      [](const void* k, int*) {
        return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kMaxSmem);
      },
      nullptr);
  if (e != cudaSuccess) return e;
  S* out = static_cast<S*>(s.buf[s.cur ^ 1]);
  const Maps3* maps = reinterpret_cast<const Maps3*>(s.tmap3[s.cur]);
  k_step3_tma<S, UNI><<<blocks, kThreads3, smem, s.stream>>>(*maps, out, make_params3<float>(s),
                                                             s.derr, in_smem);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch3_tma_any(Solver& s) {
  const long long tiles = (long long)((s.n[0] + kT3X - 1) / kT3X) * ((s.n[1] + kT3Y - 1) / kT3Y) *
                          ((s.n[2] + kT3Z - 1) / kT3Z);
  const int blocks = (int)std::min<long long>(tiles, (long long)kMinBlocks3 * s.sm_count);
  return s.uniform ? launch3_tma<S, true>(s, blocks) : launch3_tma<S, false>(s, blocks);
}

}  // namespace

cudaError_t launch_step_3d_tma(Solver& s) {
  switch (s.precision) {
    case ISLBM_FP32: return launch3_tma_any<float>(s);
    case ISLBM_FP16DEV: return launch3_tma_any<__half>(s);
    case ISLBM_BF16DEV: return launch3_tma_any<__nv_bfloat16>(s);
  }
  return cudaErrorInvalidValue;
}

int bounds_flag_d3(int reset) {
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

bool step_3d_tma_fits(int ny, int nz) { return ny >= kT3Y + 2 && nz >= kT3Z + 2; }

void step_3d_tma_box(int elem, int type, unsigned (&box)[4]) {
  const int hx = 16 / elem;
  box[0] = (unsigned)(kT3X + ((type & 1) ? 2 * hx : 0));
  box[1] = (unsigned)(kT3Y + ((type & 2) ? 2 : 0));
  box[2] = (unsigned)(kT3Z + ((type & 4) ? 2 : 0));
  box[3] = 2;
}

}  // namespace islbm
