// Z-marching pipelined 3-D step kernel (D3Q19 + D3Q7; Sec. 2.1 - 2.3, Sec. 4).
//
// A CTA owns a column of nodes: a TX x TY tile of the (x, y) plane, over a
// chunk of consecutive z levels, and marches through the chunk one level per
// step.  Every consumer thread keeps one (x, y) position for the whole chunk,
// so its interpolation tables, wall flags and shared-memory offsets are set up
// once per column, and everything that depends on z (the z weights, the z
// walls, the staged levels in use) is the same for the whole CTA.
//
// Staging.  The 26 population planes fall into seven groups by the axes they
// move along, each fetched by one TMA box per level:
//   R  (planes 0, 19)           no halo          B ring
//   X  (1, 2, 20, 21)           x halo           B ring
//   Y  (3, 4, 22, 23)           y halo           B ring
//   XY (7 .. 10)                x and y halos    B ring
//   Z  (5, 6, 24, 25)           -                A ring
//   XZ (11 .. 14)               x halo           A ring
//   YZ (15 .. 18)               y halo           A ring
// (x halos are rounded out to a 16-byte chunk.)  The groups that move in z
// need the three levels of the node-centred z stencil (base = z - 1, clamped
// at the walls); they go through the A ring, whose slots hold one level each
// and are reused once no pending step reads them.  The other groups are read
// at the node's own level only and go through the B ring, one slot per step.
// A producer warp issues each step's copies on one "full" mbarrier
// (transaction bytes) as soon as the slots they overwrite are released through
// the per-step "empty" mbarriers (one arrival per consumer warp).
//
// Chunks are handed out round robin in chunk-major order: at any time the
// CTAs work on neighbouring columns of the same band of levels, so the halo
// rows and columns they share are fetched from DRAM once and served by L2.
//
// Every wait is bounded (one second of the global timer): a wait that gives
// up raises the CTA's abort flag and the device error flag, the producer stops
// issuing and waits (bounded) for its copies in flight, and the CTA returns.
//
// The operations and their order are those of the direct kernel's pull3 and
// collide3, so the two kernels compute the same bits.  The kernel needs the
// node-centred stencil (the stencil base of both directions of an axis is
// node - 1, clamped to the axis).
#include <algorithm>
#include <cstdlib>

#include "islbm_d3_common.cuh"
#include "islbm_tma.cuh"

namespace islbm {
namespace {

constexpr int kZmTX = 32;

// staging groups: index of the TMA descriptor of each
enum ZmGroup { ZG_R = 0, ZG_X, ZG_Y, ZG_XY, ZG_Z, ZG_XZ, ZG_YZ, ZG_COUNT };

__host__ __device__ constexpr int zm_planes(int g) { return g == ZG_R ? 2 : 4; }
__host__ __device__ constexpr bool zm_hx(int g) { return g == ZG_X || g == ZG_XY || g == ZG_XZ; }
__host__ __device__ constexpr bool zm_hy(int g) { return g == ZG_Y || g == ZG_XY || g == ZG_YZ; }
// first plane of a group
__host__ __device__ constexpr int zm_first(int g) {
  return g == ZG_R ? 0 : g == ZG_X ? 1 : g == ZG_Y ? 3 : g == ZG_XY ? 7 : g == ZG_Z ? 5
         : g == ZG_XZ ? 11 : 15;
}
// stride between the two plane pairs of the R, X, Y and Z groups (flow plane
// and temperature plane: 19 planes apart); the XY, XZ and YZ groups are four
// consecutive planes
__host__ __device__ constexpr bool zm_split(int g) {
  return g == ZG_R || g == ZG_X || g == ZG_Y || g == ZG_Z;
}

template <typename S, int TY>
struct ZmGeom {
  static constexpr int TX = kZmTX;
  static constexpr int HX = 16 / (int)sizeof(S);
  static constexpr int WX = TX + 2 * HX;   // width of a box with an x halo
  static constexpr int HY = TY + 2;        // height of a box with a y halo
  static constexpr int width(int g) { return zm_hx(g) ? WX : TX; }
  static constexpr int height(int g) { return zm_hy(g) ? HY : TY; }
  static constexpr int plane_elems(int g) { return width(g) * height(g); }
  static constexpr unsigned bytes(int g) {
    return (unsigned)(zm_planes(g) * plane_elems(g)) * (unsigned)sizeof(S);
  }
  // byte offsets of the groups inside a B slot (R, X, Y, XY) and an A slot
  // (Z, XZ, YZ)
  static constexpr unsigned off(int g) {
    return g == ZG_R ? 0u
           : g == ZG_X ? bytes(ZG_R)
           : g == ZG_Y ? bytes(ZG_R) + bytes(ZG_X)
           : g == ZG_XY ? bytes(ZG_R) + bytes(ZG_X) + bytes(ZG_Y)
           : g == ZG_Z ? 0u
           : g == ZG_XZ ? bytes(ZG_Z)
                        : bytes(ZG_Z) + bytes(ZG_XZ);
  }
  static constexpr unsigned B_SLOT = bytes(ZG_R) + bytes(ZG_X) + bytes(ZG_Y) + bytes(ZG_XY);
  static constexpr unsigned A_SLOT = bytes(ZG_Z) + bytes(ZG_XZ) + bytes(ZG_YZ);
};

// Ring configuration of one instantiation: tile height, A and B ring depths,
// CTAs per SM the shared memory is sized for.
template <typename S, int TY, int DA, int DB>
struct ZmCfg {
  using G = ZmGeom<S, TY>;
  static constexpr int kConsumers = kZmTX * TY;
  static constexpr int kConsumerWarps = kConsumers / 32;
  static constexpr int kThreads = kConsumers + 32;   // + one producer warp
  static constexpr size_t a_bytes() { return (size_t)DA * G::A_SLOT; }
  static constexpr size_t b_bytes() { return (size_t)DB * G::B_SLOT; }
  // full[DB], empty[DB] and the abort flag, rounded up to 128 bytes
  static constexpr size_t bar_bytes() {
    return (2 * DB * sizeof(uint64_t) + sizeof(int) + 127) / 128 * 128;
  }
  static constexpr size_t smem_bytes() { return a_bytes() + b_bytes() + bar_bytes(); }
  static_assert(DA >= 3, "the A ring holds the three levels of a z stencil");
  static_assert(DB >= 1, "the B ring needs a slot");
  static_assert(G::A_SLOT % 128 == 0 && G::B_SLOT % 128 == 0,
                "TMA destinations must stay 128-byte aligned");
  static_assert(G::bytes(ZG_R) % 128 == 0 && G::bytes(ZG_X) % 128 == 0 &&
                    G::bytes(ZG_Y) % 128 == 0 && G::bytes(ZG_XY) % 128 == 0 &&
                    G::bytes(ZG_Z) % 128 == 0 && G::bytes(ZG_XZ) % 128 == 0,
                "every group box starts 128-byte aligned inside its slot");
  static_assert(kConsumers % 32 == 0, "tiles are whole warps along x");
};

struct alignas(128) ZmMaps {
  CUtensorMap m[ZG_COUNT];
};

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, int c4, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
      "r"(smem_u32(bar))
      : "memory");
}

// Bounded wait that also gives up as soon as another thread raised the abort
// flag (the limits of mbar_wait).
__device__ __forceinline__ bool zm_wait(uint64_t* bar, unsigned phase, const volatile int* abort) {
  if (mbar_try_wait(bar, phase)) return true;
  const unsigned long long t0 = global_ns();
  for (int i = 0; i < kWaitMaxPolls; ++i) {
    if (mbar_try_wait(bar, phase)) return true;
    if ((i & 63) == 63 && (*abort || global_ns() - t0 > kWaitLimitNs)) return false;
  }
  return false;
}

// One staged value: plane `pl` of a group box of width W and height H, row y,
// column x (window coordinates).
template <typename S, int W, int H>
__device__ __forceinline__ float zat(const S* __restrict__ box, int pl, int y, int x) {
  if (!(ISLBM_IN_WINDOW(y, H) && ISLBM_IN_WINDOW(x, W))) return 0.f;
  return to_f(box[(pl * H + y) * W + x]);
}

// Node-centred stencil base of an axis of n nodes: node - 1, clamped.
__host__ __device__ __forceinline__ int zm_base(int j, int n) { return max(0, min(j - 1, n - 3)); }

// The schedule both roles walk: chunk-major items, round robin over the CTAs.
struct ZmSched {
  int ncx, ncol, nitems, zc, ny, nz;
  // column origin (x0, y0), first row of the y-halo window (wy0: one row
  // before the tile, moved inwards on a ragged last tile so that the window
  // still holds every stencil row), and the chunk's levels [z0, z1)
  __device__ __forceinline__ void item(int t, int& x0, int& y0, int& wy0, int& z0, int& z1,
                                       int ty) const {
    const int chunk = t / ncol;
    const int col = t - chunk * ncol;
    const int cy = col / ncx;
    x0 = (col - cy * ncx) * kZmTX;
    y0 = cy * ty;
    wy0 = min(y0 - 1, ny - (ty + 2));
    z0 = chunk * zc;
    z1 = min(z0 + zc, nz);
  }
};

template <typename S, int TY, int DA, int DB, int MINB>
__global__ void __launch_bounds__(ZmCfg<S, TY, DA, DB>::kThreads, MINB)
    k_step3_zm(const __grid_constant__ ZmMaps maps, S* __restrict__ fout, P3<float> p,
               int* err, ZmSched sc) {
  using C = ZmCfg<S, TY, DA, DB>;
  using G = typename C::G;
  using St = Store<S>;
  using R = float;
  constexpr int TX = kZmTX;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* ringA = smem_raw;
  unsigned char* ringB = smem_raw + C::a_bytes();
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + C::a_bytes() + C::b_bytes());
  uint64_t* empty = full + DB;
  volatile int* abort = reinterpret_cast<volatile int*>(empty + DB);

  if (threadIdx.x == 0) {
    for (int s = 0; s < DB; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], C::kConsumerWarps);
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nz = p.nz;
  if (warp == C::kConsumerWarps) {
    // ---------------- producer ----------------
    if (lane == 0) {
      unsigned s = 0;      // steps issued
      unsigned a = 0;      // A levels issued
      unsigned done = 0;   // consumer steps known to be complete
      unsigned use[DA];    // last step that reads the level in each A slot (+1; 0 = none)
#pragma unroll
      for (int i = 0; i < DA; ++i) use[i] = 0;
      bool stop = false;
      // wait until consumer step `t` is complete (steps complete in order)
      auto wait_done = [&](unsigned t) -> bool {
        while (done <= t) {
          if (!zm_wait(&empty[done % DB], (done / DB) & 1u, abort)) return false;
          ++done;
        }
        return true;
      };
      auto fail = [&]() {
        if (!*abort) atomicExch(err, 1);
        *abort = 1;
        stop = true;
      };
      for (int t = blockIdx.x; t < sc.nitems && !stop; t += gridDim.x) {
        int x0, y0, wy0, z0, z1;
        sc.item(t, x0, y0, wy0, z0, z1, TY);
        const int b0 = zm_base(z0, nz);
        int next_level = b0;   // next A level of this column to fetch
        const unsigned a_item = a;
        for (int z = z0; z < z1 && !stop; ++z, ++s) {
          // the B slot of this step was last read by step s - DB
          if (s >= (unsigned)DB && !wait_done(s - DB)) { fail(); break; }
          const int bz = zm_base(z, nz);
          const int last = bz + 2;   // A levels b(z) .. b(z) + 2 must be staged
          // the A slots that receive the new levels must be released first
          for (int L = next_level; L <= last; ++L) {
            const unsigned q = a + (unsigned)(L - next_level);
            const unsigned u = use[q % DA];
            if (u != 0 && !wait_done(u - 1)) { fail(); break; }
          }
          if (stop) break;
          if (*abort) { stop = true; break; }
          const int sb = (int)(s % DB);
          const unsigned nnew = (unsigned)(last - next_level + 1);
          mbar_expect_tx(&full[sb], G::B_SLOT + nnew * G::A_SLOT);
          unsigned char* B = ringB + (size_t)sb * G::B_SLOT;
          tma_load_4d(B + G::off(ZG_R), &maps.m[ZG_R], x0, y0, z, 0, &full[sb]);
          tma_load_5d(B + G::off(ZG_X), &maps.m[ZG_X], x0 - G::HX, y0, z, 0, 0, &full[sb]);
          tma_load_5d(B + G::off(ZG_Y), &maps.m[ZG_Y], x0, wy0, z, 0, 0, &full[sb]);
          tma_load_4d(B + G::off(ZG_XY), &maps.m[ZG_XY], x0 - G::HX, wy0, z, 0, &full[sb]);
          for (int L = next_level; L <= last; ++L, ++a) {
            unsigned char* A = ringA + (size_t)(a % DA) * G::A_SLOT;
            tma_load_5d(A + G::off(ZG_Z), &maps.m[ZG_Z], x0, y0, L, 0, 0, &full[sb]);
            tma_load_4d(A + G::off(ZG_XZ), &maps.m[ZG_XZ], x0 - G::HX, y0, L, 0, &full[sb]);
            tma_load_4d(A + G::off(ZG_YZ), &maps.m[ZG_YZ], x0, wy0, L, 0, &full[sb]);
          }
          next_level = last + 1;
          // this step reads the levels b(z) .. b(z) + 2
          const unsigned lo = a_item + (unsigned)(bz - b0);
#pragma unroll
          for (int m = 0; m < 3; ++m) use[(lo + m) % DA] = s + 1;
        }
      }
      // wait (bounded) for the copies of the last steps issued
      for (unsigned t = s > (unsigned)DB ? s - DB : 0u; t < s; ++t)
        mbar_wait(&full[t % DB], (t / DB) & 1u);
    }
  } else {
    // ---------------- consumers ----------------
    const int c = threadIdx.x % TX, ry = threadIdx.x / TX;
    const long long P = p.plane;
    const size_t zstride = (size_t)p.pitch * p.ny;
    unsigned s = 0, a = 0;
    bool stop = false;
    for (int t = blockIdx.x; t < sc.nitems && !stop; t += gridDim.x) {
      int x0, y0, wy0, z0, z1;
      sc.item(t, x0, y0, wy0, z0, z1, TY);
      const int x = x0 + c, y = y0 + ry;
      const bool valid = x < p.nx && y < p.ny;
      const int xc = min(x, p.nx - 1), yc = min(y, p.ny - 1);
      // window coordinates: own position without / with the halo, stencil bases
      const int lxn = xc - x0, lyn = yc - y0;
      const int lxh = lxn + G::HX, lyh = yc - wy0;
      const int bxh = zm_base(xc, p.nx) - (x0 - G::HX);
      const int byh = zm_base(yc, p.ny) - wy0;
      const float4 tx0 = __ldg(p.pk[0][0] + xc), tx1 = __ldg(p.pk[0][1] + xc);
      const float4 ty0 = __ldg(p.pk[1][0] + yc), ty1 = __ldg(p.pk[1][1] + yc);
      const bool wxm = xc == 0, wxp = xc == p.nx - 1, wym = yc == 0, wyp = yc == p.ny - 1;
      const int b0 = zm_base(z0, nz);
      size_t idx = ((size_t)z0 * p.ny + y) * p.pitch + x;
      for (int z = z0; z < z1; ++z, ++s, idx += zstride) {
        const int sb = (int)(s % DB);
        if (!zm_wait(&full[sb], (s / DB) & 1u, abort)) {
          if (!*abort) atomicExch(err, 1);
          *abort = 1;
          stop = true;
          break;
        }
        const int bz = zm_base(z, nz);
        const unsigned lo = a + (unsigned)(bz - b0);
        const S* B = reinterpret_cast<const S*>(ringB + (size_t)sb * G::B_SLOT);
        const S* A0 = reinterpret_cast<const S*>(ringA + (size_t)(lo % DA) * G::A_SLOT);
        const S* A1 = reinterpret_cast<const S*>(ringA + (size_t)((lo + 1) % DA) * G::A_SLOT);
        const S* A2 = reinterpret_cast<const S*>(ringA + (size_t)((lo + 2) % DA) * G::A_SLOT);
        const int oz = z - bz;   // own level among the three: 0 at z = 0, 2 at the top
        const S* Ao = oz == 0 ? A0 : (oz == 1 ? A1 : A2);
        const float4 tz0 = __ldg(p.pk[2][0] + z), tz1 = __ldg(p.pk[2][1] + z);
        const bool wzm = z == 0, wzp = z == nz - 1;

        const S* bR = B + G::off(ZG_R) / sizeof(S);
        const S* bX = B + G::off(ZG_X) / sizeof(S);
        const S* bY = B + G::off(ZG_Y) / sizeof(S);
        const S* bXY = B + G::off(ZG_XY) / sizeof(S);
        constexpr int oZ = G::off(ZG_Z) / sizeof(S), oXZ = G::off(ZG_XZ) / sizeof(S);
        constexpr int oYZ = G::off(ZG_YZ) / sizeof(S);
        constexpr int WX = G::WX, HY = G::HY;

        // own value (bounce-back partners) in each group
        auto ownR = [&](int pl) { return zat<S, TX, TY>(bR, pl, lyn, lxn); };
        auto ownX = [&](int pl) { return zat<S, WX, TY>(bX, pl, lyn, lxh); };
        auto ownY = [&](int pl) { return zat<S, TX, HY>(bY, pl, lyh, lxn); };
        auto ownXY = [&](int pl) { return zat<S, WX, HY>(bXY, pl, lyh, lxh); };
        auto ownZ = [&](int pl) { return zat<S, TX, TY>(Ao + oZ, pl, lyn, lxn); };
        auto ownXZ = [&](int pl) { return zat<S, WX, TY>(Ao + oXZ, pl, lyn, lxh); };
        auto ownYZ = [&](int pl) { return zat<S, TX, HY>(Ao + oYZ, pl, lyh, lxn); };
        // one-axis pulls
        auto pullX = [&](int pl, float4 w) {
          return dot3(w, zat<S, WX, TY>(bX, pl, lyn, bxh), zat<S, WX, TY>(bX, pl, lyn, bxh + 1),
                      zat<S, WX, TY>(bX, pl, lyn, bxh + 2));
        };
        auto pullY = [&](int pl, float4 w) {
          return dot3(w, zat<S, TX, HY>(bY, pl, byh, lxn), zat<S, TX, HY>(bY, pl, byh + 1, lxn),
                      zat<S, TX, HY>(bY, pl, byh + 2, lxn));
        };
        auto pullZ = [&](int pl, float4 w) {
          return dot3(w, zat<S, TX, TY>(A0 + oZ, pl, lyn, lxn), zat<S, TX, TY>(A1 + oZ, pl, lyn, lxn),
                      zat<S, TX, TY>(A2 + oZ, pl, lyn, lxn));
        };
        // two-axis pulls: the first moving axis inside, the second outside
        auto pullXY = [&](int pl, float4 wx, float4 wy) {
          const R wl[3] = {wy.x, wy.y, wy.z};
          R acc = R(0);
#pragma unroll
          for (int l = 0; l < 3; ++l)
            acc = lfma(wl[l],
                       dot3(wx, zat<S, WX, HY>(bXY, pl, byh + l, bxh),
                            zat<S, WX, HY>(bXY, pl, byh + l, bxh + 1),
                            zat<S, WX, HY>(bXY, pl, byh + l, bxh + 2)),
                       acc);
          return acc;
        };
        auto pullXZ = [&](int pl, float4 wx, float4 wz) {
          const R wl[3] = {wz.x, wz.y, wz.z};
          const S* lv[3] = {A0 + oXZ, A1 + oXZ, A2 + oXZ};
          R acc = R(0);
#pragma unroll
          for (int l = 0; l < 3; ++l)
            acc = lfma(wl[l],
                       dot3(wx, zat<S, WX, TY>(lv[l], pl, lyn, bxh),
                            zat<S, WX, TY>(lv[l], pl, lyn, bxh + 1),
                            zat<S, WX, TY>(lv[l], pl, lyn, bxh + 2)),
                       acc);
          return acc;
        };
        auto pullYZ = [&](int pl, float4 wy, float4 wz) {
          const R wl[3] = {wz.x, wz.y, wz.z};
          const S* lv[3] = {A0 + oYZ, A1 + oYZ, A2 + oYZ};
          R acc = R(0);
#pragma unroll
          for (int l = 0; l < 3; ++l)
            acc = lfma(wl[l],
                       dot3(wy, zat<S, TX, HY>(lv[l], pl, byh, lxn),
                            zat<S, TX, HY>(lv[l], pl, byh + 1, lxn),
                            zat<S, TX, HY>(lv[l], pl, byh + 2, lxn)),
                       acc);
          return acc;
        };

        R f[19], g[7];
        // group planes: R (f0, g0), X (f1, f2, g1, g2), Y (f3, f4, g3, g4),
        // Z (f5, f6, g5, g6), XY (f7 .. f10), XZ (f11 .. f14), YZ (f15 .. f18)
        f[0] = ownR(0);
        g[0] = ownR(1);
        f[1] = wxm ? ownX(1) : pullX(0, tx0);
        f[2] = wxp ? ownX(0) : pullX(1, tx1);
        g[1] = wxm ? p.abb_hot - ownX(3) : pullX(2, tx0);
        g[2] = wxp ? p.abb_cold - ownX(2) : pullX(3, tx1);
        f[3] = wym ? ownY(1) : pullY(0, ty0);
        f[4] = wyp ? ownY(0) : pullY(1, ty1);
        g[3] = wym ? ownY(3) : pullY(2, ty0);
        g[4] = wyp ? ownY(2) : pullY(3, ty1);
        f[5] = wzm ? ownZ(1) : pullZ(0, tz0);
        f[6] = wzp ? ownZ(0) : pullZ(1, tz1);
        g[5] = wzm ? ownZ(3) : pullZ(2, tz0);
        g[6] = wzp ? ownZ(2) : pullZ(3, tz1);
        f[7] = (wxm || wym) ? ownXY(1) : pullXY(0, tx0, ty0);
        f[8] = (wxp || wyp) ? ownXY(0) : pullXY(1, tx1, ty1);
        f[9] = (wxm || wyp) ? ownXY(3) : pullXY(2, tx0, ty1);
        f[10] = (wxp || wym) ? ownXY(2) : pullXY(3, tx1, ty0);
        f[11] = (wxm || wzm) ? ownXZ(1) : pullXZ(0, tx0, tz0);
        f[12] = (wxp || wzp) ? ownXZ(0) : pullXZ(1, tx1, tz1);
        f[13] = (wxm || wzp) ? ownXZ(3) : pullXZ(2, tx0, tz1);
        f[14] = (wxp || wzm) ? ownXZ(2) : pullXZ(3, tx1, tz0);
        f[15] = (wym || wzm) ? ownYZ(1) : pullYZ(0, ty0, tz0);
        f[16] = (wyp || wzp) ? ownYZ(0) : pullYZ(1, ty1, tz1);
        f[17] = (wym || wzp) ? ownYZ(3) : pullYZ(2, ty0, tz1);
        f[18] = (wyp || wzm) ? ownYZ(2) : pullYZ(3, ty1, tz0);
        // every staged value of this step is in registers: release the slots
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[sb]);
        if (valid) {
          R rho, ux, uy, uz, T;
          collide3(f, g, p, rho, ux, uy, uz, T);
          unsigned r = sr_seed(idx, p.step);
#pragma unroll
          for (int i = 0; i < 19; ++i) St::st_sr(fout + i * P + idx, f[i], sr_next(r));
#pragma unroll
          for (int i = 0; i < 7; ++i) St::st_sr(fout + (19 + i) * P + idx, g[i], sr_next(r));
        }
      }
      if (stop) break;
      // A levels this column fetched: b(z0) .. b(z1 - 1) + 2
      a += (unsigned)(zm_base(z1 - 1, nz) + 3 - b0);
    }
  }
  __syncthreads();   // the producer has drained its copies before the CTA leaves
}

// ---- launch configurations ----
// (S, TY, DA, DB, CTAs per SM the shared memory and registers are sized for)
template <typename S, int TY, int DA, int DB, int MINB>
struct ZmLaunch {
  using C = ZmCfg<S, TY, DA, DB>;
  static const void* fn() { return reinterpret_cast<const void*>(k_step3_zm<S, TY, DA, DB, MINB>); }
  static cudaError_t setup(const void* k, int* per_sm) {
    cudaError_t e =
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_bytes());
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, C::kThreads, C::smem_bytes());
    if (e != cudaSuccess) return e;
    *per_sm = std::max(n, 1);
    return cudaSuccess;
  }
  static cudaError_t run(Solver& s, int zc_override) {
    int per_sm = 1;
    cudaError_t e = launch_setup_once(fn(), &ZmLaunch::setup, &per_sm);
    if (e != cudaSuccess) return e;
    ZmSched sc;
    sc.ncx = (s.n[0] + kZmTX - 1) / kZmTX;
    sc.ncol = sc.ncx * ((s.n[1] + TY - 1) / TY);
    sc.ny = s.n[1];
    sc.nz = s.n[2];
    const long long slots = (long long)per_sm * s.sm_count;
    // chunk length: the one with the least estimated time, counting each
    // column start as about one level of work (its two extra A levels and
    // the pipeline restart)
    int best = s.n[2];
    double best_cost = 1e300;
    for (int zc = 4; zc <= s.n[2] + 3; zc += 4) {
      const int zcc = std::min(zc, s.n[2]);
      const long long items = (long long)sc.ncol * ((s.n[2] + zcc - 1) / zcc);
      const long long rounds = (items + slots - 1) / slots;
      const double cost = (double)rounds * (zcc + 1.0);
      if (cost < best_cost - 1e-9) {
        best_cost = cost;
        best = zcc;
      }
      if (zcc == s.n[2]) break;
    }
    sc.zc = zc_override > 0 ? std::min(zc_override, s.n[2]) : best;
    sc.nitems = sc.ncol * ((s.n[2] + sc.zc - 1) / sc.zc);
    const int blocks = (int)std::min<long long>(sc.nitems, slots);
    S* out = static_cast<S*>(s.buf[s.cur ^ 1]);
    const ZmMaps* maps = reinterpret_cast<const ZmMaps*>(s.tmap3[s.cur]);
    k_step3_zm<S, TY, DA, DB, MINB><<<blocks, C::kThreads, C::smem_bytes(), s.stream>>>(
        *maps, out, make_params3<float>(s), s.derr, sc);
    return cudaGetLastError();
  }
};

// Tuning override of the chunk length (levels per column item; 0 = automatic).
int zm_chunk_override() {
  static const int v = [] {
    const char* e = std::getenv("ISLBM_ZM_CHUNK");
    return e ? std::max(0, std::atoi(e)) : 0;
  }();
  return v;
}

template <typename S>
cudaError_t launch_zm(Solver& s) {
  const int zc = zm_chunk_override();
  switch (s.variant) {
    case KV_ZM3D_T4: return ZmLaunch<S, 4, 6, 2, 3>::run(s, zc);
    default: return ZmLaunch<S, 8, 4, 2, 2>::run(s, zc);
  }
}

}  // namespace

cudaError_t launch_step_3d_zm(Solver& s) {
  switch (s.precision) {
    case ISLBM_FP32: return launch_zm<float>(s);
    case ISLBM_FP16DEV: return launch_zm<__half>(s);
    case ISLBM_BF16DEV: return launch_zm<__nv_bfloat16>(s);
  }
  return cudaErrorInvalidValue;
}

int bounds_flag_zm(int reset) {
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

int zm_tile_rows(int variant) { return variant == KV_ZM3D_T4 ? 4 : 8; }

// TMA box (x, y, z, planes[, plane pairs]) of staging group g.
int step_3d_zm_box(int elem, int variant, int g, unsigned (&box)[5]) {
  const int ty = zm_tile_rows(variant);
  const int hx = 16 / elem;
  box[0] = (unsigned)(kZmTX + (zm_hx(g) ? 2 * hx : 0));
  box[1] = (unsigned)(ty + (zm_hy(g) ? 2 : 0));
  box[2] = 1;
  if (zm_split(g)) {
    box[3] = 2;
    box[4] = g == ZG_R ? 1u : 2u;
    return g == ZG_R ? 4 : 5;
  }
  box[3] = 4;
  box[4] = 1;
  return 4;
}

int step_3d_zm_first_plane(int g) { return zm_first(g); }
int step_3d_zm_split(int g) { return zm_split(g) ? 1 : 0; }

}  // namespace islbm
