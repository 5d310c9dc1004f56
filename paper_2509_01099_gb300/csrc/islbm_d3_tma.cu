// Pipelined 3-D step kernel (D3Q19 + D3Q7; Sec. 2.1 - 2.3, Sec. 4).
//
// A CTA owns a 32 x 4 x 2 tile of nodes (one node per consumer thread) and
// walks its share of the tiles persistently.  The 26 population planes of a
// tile are staged in opposite pairs (0), (1,2), (3,4), ... (17,18), (19),
// (20,21), (22,23), (24,25): one 4-D TMA copy per pair brings the tile plus a
// one-node halo on every side (rounded out to a 16-byte chunk in x) into a
// ring of shared-memory slots.  A producer warp issues the copies as slots
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
// inwards at the far walls: it needs n_y >= 6 and n_z >= 4.
#include "islbm_d3_common.cuh"
#include "islbm_tma.cuh"

namespace islbm {
namespace {

constexpr int kT3X = 32, kT3Y = 4, kT3Z = 2;
constexpr int kConsumers3 = kT3X * kT3Y * kT3Z;   // 256
constexpr int kConsumerWarps3 = kConsumers3 / 32;
constexpr int kThreads3 = kConsumers3 + 32;       // + one producer warp
constexpr int kPairs3 = 14;
constexpr int kStages3 = 6;

template <typename S>
struct Geom3 {
  static constexpr int HX = 16 / (int)sizeof(S);
  static constexpr int SW = kT3X + 2 * HX, SH = kT3Y + 2, SD = kT3Z + 2;
  static constexpr int POP = SW * SH * SD;                      // staged elements per population
  static constexpr unsigned SLOT = 2u * POP * (unsigned)sizeof(S);   // bytes per pair
  static constexpr size_t smem_bytes() {
    return (size_t)kStages3 * SLOT + 2 * kStages3 * sizeof(uint64_t) + 16;
  }
};
static_assert(Geom3<float>::SLOT % 128 == 0 && Geom3<__half>::SLOT % 128 == 0,
              "TMA destinations must stay 128-byte aligned");

// first population of pair j
__device__ __forceinline__ int pair_first(int j) {
  return j == 0 ? 0 : (j <= 9 ? 2 * j - 1 : (j == 10 ? 19 : 2 * j - 2));
}

// Bounded wait that also gives up as soon as another thread raised the abort flag.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, unsigned phase,
                                              const volatile int* abort) {
  for (int i = 0; i < (1 << 22); ++i) {
    if (mbar_try_wait(bar, phase)) return true;
    if (*abort) return false;
  }
  return false;
}

// Geometry of one node inside a staged window.
template <typename R>
struct Node3 {
  int lx, ly, lz;                 // node position in the window
  float4 tx[2], ty[2], tz[2];     // packed tables (+ / - direction) per axis
  int bx[2], by[2], bz[2];        // stencil bases in window coordinates
};

// Pull of population plane `pl` moving with (CX, CY, CZ) at the node; the same
// operation order as the direct kernel's pull3 (first moving axis inside).
template <typename S, typename R, int CX, int CY, int CZ, bool UNI>
__device__ __forceinline__ R pull_w(const S* __restrict__ pl, const Node3<R>& n) {
  using G = Geom3<S>;
  auto at = [&](int z, int y, int x) -> R { return (R)to_f(pl[(z * G::SH + y) * G::SW + x]); };
  if (UNI || (CX == 0 && CY == 0 && CZ == 0)) return at(n.lz - CZ, n.ly - CY, n.lx - CX);
  constexpr int kx = CX > 0 ? 0 : 1, ky = CY > 0 ? 0 : 1, kz = CZ > 0 ? 0 : 1;
  if (CX != 0 && CY == 0 && CZ == 0) {
    const float4 t = n.tx[kx];
    const int b = n.bx[kx];
    return t.x * at(n.lz, n.ly, b) + t.y * at(n.lz, n.ly, b + 1) + t.z * at(n.lz, n.ly, b + 2);
  }
  if (CX == 0 && CY != 0 && CZ == 0) {
    const float4 t = n.ty[ky];
    const int b = n.by[ky];
    return t.x * at(n.lz, b, n.lx) + t.y * at(n.lz, b + 1, n.lx) + t.z * at(n.lz, b + 2, n.lx);
  }
  if (CX == 0 && CY == 0 && CZ != 0) {
    const float4 t = n.tz[kz];
    const int b = n.bz[kz];
    return t.x * at(b, n.ly, n.lx) + t.y * at(b + 1, n.ly, n.lx) + t.z * at(b + 2, n.ly, n.lx);
  }
  R acc = R(0);
  if (CZ == 0) {   // x inside, y outside
    const float4 a = n.tx[kx], w = n.ty[ky];
    const int b0 = n.bx[kx], b1 = n.by[ky];
    const R wl[3] = {w.x, w.y, w.z};
#pragma unroll
    for (int l = 0; l < 3; ++l)
      acc += wl[l] * (a.x * at(n.lz, b1 + l, b0) + a.y * at(n.lz, b1 + l, b0 + 1) +
                      a.z * at(n.lz, b1 + l, b0 + 2));
  } else if (CY == 0) {   // x inside, z outside
    const float4 a = n.tx[kx], w = n.tz[kz];
    const int b0 = n.bx[kx], b1 = n.bz[kz];
    const R wl[3] = {w.x, w.y, w.z};
#pragma unroll
    for (int l = 0; l < 3; ++l)
      acc += wl[l] * (a.x * at(b1 + l, n.ly, b0) + a.y * at(b1 + l, n.ly, b0 + 1) +
                      a.z * at(b1 + l, n.ly, b0 + 2));
  } else {   // y inside, z outside
    const float4 a = n.ty[ky], w = n.tz[kz];
    const int b0 = n.by[ky], b1 = n.bz[kz];
    const R wl[3] = {w.x, w.y, w.z};
#pragma unroll
    for (int l = 0; l < 3; ++l)
      acc += wl[l] * (a.x * at(b1 + l, b0, n.lx) + a.y * at(b1 + l, b0 + 1, n.lx) +
                      a.z * at(b1 + l, b0 + 2, n.lx));
  }
  return acc;
}

template <typename S, bool UNI>
__global__ void __launch_bounds__(kThreads3, 2)
    k_step3_tma(const __grid_constant__ CUtensorMap tmap, S* __restrict__ fout, P3<float> p,
                int* err) {
  using G = Geom3<S>;
  using St = Store<S>;
  using R = float;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + (size_t)kStages3 * G::SLOT);
  uint64_t* empty = full + kStages3;
  volatile int* abort = reinterpret_cast<volatile int*>(empty + kStages3);

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
      long long j = 0;
      bool stop = false;
      for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
        int x0, y0, z0, sy0, sz0;
        origin(t, x0, y0, z0, sy0, sz0);
        for (int q = 0; q < kPairs3; ++q, ++j) {
          const int s = (int)(j % kStages3);
          if (j >= kStages3 &&
              !wait_or_abort(&empty[s], (unsigned)((j / kStages3) - 1) & 1u, abort)) {
            if (!*abort) atomicExch(err, 1);
            *abort = 1;
            stop = true;
            break;
          }
          if (*abort) {
            stop = true;
            break;
          }
          mbar_expect_tx(&full[s], G::SLOT);
          tma_load_4d(smem_raw + (size_t)s * G::SLOT, &tmap, x0 - G::HX, sy0, sz0, pair_first(q),
                      &full[s]);
        }
      }
      // wait (bounded) for the last copy issued into every slot
      for (int s = 0; s < kStages3 && s < j; ++s) {
        const long long last = j - 1 - ((j - 1 - s) % kStages3);
        mbar_wait(&full[s], (unsigned)(last / kStages3) & 1u);
      }
    }
  } else {
    // ---------------- consumers ----------------
    const int c = threadIdx.x & 31, ry = (threadIdx.x >> 5) & (kT3Y - 1);
    const int rz = threadIdx.x / (kT3X * kT3Y);
    const long long P = p.plane;
    long long j = 0;
    bool stop = false;
    for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
      int x0, y0, z0, sy0, sz0;
      origin(t, x0, y0, z0, sy0, sz0);
      const int x = x0 + c, y = y0 + ry, z = z0 + rz;
      const bool valid = x < p.nx && y < p.ny && z < p.nz;
      const int xc = min(x, p.nx - 1), yc = min(y, p.ny - 1), zc = min(z, p.nz - 1);
      Node3<R> n;
      n.lx = xc - (x0 - G::HX);
      n.ly = yc - sy0;
      n.lz = zc - sz0;
      if (!UNI) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          n.tx[k] = __ldg(p.pk[0][k] + xc);
          n.ty[k] = __ldg(p.pk[1][k] + yc);
          n.tz[k] = __ldg(p.pk[2][k] + zc);
          n.bx[k] = __float_as_int(n.tx[k].w) - (x0 - G::HX);
          n.by[k] = __float_as_int(n.ty[k].w) - sy0;
          n.bz[k] = __float_as_int(n.tz[k].w) - sz0;
        }
      }
      const bool wxm = xc == 0, wxp = xc == p.nx - 1, wym = yc == 0, wyp = yc == p.ny - 1;
      const bool wzm = zc == 0, wzp = zc == p.nz - 1;
      R f[19], g[7];
      const int here = (n.lz * G::SH + n.ly) * G::SW + n.lx;
#pragma unroll
      for (int q = 0; q < kPairs3; ++q) {
        const int s = (int)((j + q) % kStages3);
        if (!wait_or_abort(&full[s], (unsigned)((j + q) / kStages3) & 1u, abort)) {
          if (!*abort) atomicExch(err, 1);
          *abort = 1;
          stop = true;
          break;
        }
        const S* a = reinterpret_cast<const S*>(smem_raw + (size_t)s * G::SLOT);
        const S* b = a + G::POP;
        auto own = [&](const S* pl) -> R { return (R)to_f(pl[here]); };
#define PW(pl, cx, cy, cz) pull_w<S, R, cx, cy, cz, UNI>(pl, n)
        switch (q) {
          case 0: f[0] = own(a); break;
          case 1:
            f[1] = wxm ? own(b) : PW(a, 1, 0, 0);
            f[2] = wxp ? own(a) : PW(b, -1, 0, 0);
            break;
          case 2:
            f[3] = wym ? own(b) : PW(a, 0, 1, 0);
            f[4] = wyp ? own(a) : PW(b, 0, -1, 0);
            break;
          case 3:
            f[5] = wzm ? own(b) : PW(a, 0, 0, 1);
            f[6] = wzp ? own(a) : PW(b, 0, 0, -1);
            break;
          case 4:
            f[7] = (wxm || wym) ? own(b) : PW(a, 1, 1, 0);
            f[8] = (wxp || wyp) ? own(a) : PW(b, -1, -1, 0);
            break;
          case 5:
            f[9] = (wxm || wyp) ? own(b) : PW(a, 1, -1, 0);
            f[10] = (wxp || wym) ? own(a) : PW(b, -1, 1, 0);
            break;
          case 6:
            f[11] = (wxm || wzm) ? own(b) : PW(a, 1, 0, 1);
            f[12] = (wxp || wzp) ? own(a) : PW(b, -1, 0, -1);
            break;
          case 7:
            f[13] = (wxm || wzp) ? own(b) : PW(a, 1, 0, -1);
            f[14] = (wxp || wzm) ? own(a) : PW(b, -1, 0, 1);
            break;
          case 8:
            f[15] = (wym || wzm) ? own(b) : PW(a, 0, 1, 1);
            f[16] = (wyp || wzp) ? own(a) : PW(b, 0, -1, -1);
            break;
          case 9:
            f[17] = (wym || wzp) ? own(b) : PW(a, 0, 1, -1);
            f[18] = (wyp || wzm) ? own(a) : PW(b, 0, -1, 1);
            break;
          case 10: g[0] = own(a); break;
          case 11:
            g[1] = wxm ? p.abb_hot - own(b) : PW(a, 1, 0, 0);
            g[2] = wxp ? p.abb_cold - own(a) : PW(b, -1, 0, 0);
            break;
          case 12:
            g[3] = wym ? own(b) : PW(a, 0, 1, 0);
            g[4] = wyp ? own(a) : PW(b, 0, -1, 0);
            break;
          default:
            g[5] = wzm ? own(b) : PW(a, 0, 0, 1);
            g[6] = wzp ? own(a) : PW(b, 0, 0, -1);
            break;
        }
#undef PW
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
      }
      if (stop) break;
      j += kPairs3;
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
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_step3_tma<S, UNI>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)G::smem_bytes());
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const S* in = static_cast<const S*>(s.buf[s.cur]);
  (void)in;
  S* out = static_cast<S*>(s.buf[s.cur ^ 1]);
  const CUtensorMap* map = reinterpret_cast<const CUtensorMap*>(s.tmap[s.cur]);
  k_step3_tma<S, UNI><<<blocks, kThreads3, G::smem_bytes(), s.stream>>>(*map, out,
                                                                       make_params3<float>(s),
                                                                       s.derr);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch3_tma_any(Solver& s) {
  const long long tiles = (long long)((s.n[0] + kT3X - 1) / kT3X) * ((s.n[1] + kT3Y - 1) / kT3Y) *
                          ((s.n[2] + kT3Z - 1) / kT3Z);
  const int blocks = (int)std::min<long long>(tiles, 2LL * s.sm_count);
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

size_t step_3d_tma_box(int elem, unsigned (&box)[4]) {
  const int hx = 16 / elem;
  box[0] = (unsigned)(kT3X + 2 * hx);
  box[1] = kT3Y + 2;
  box[2] = kT3Z + 2;
  box[3] = 2;
  return (size_t)box[0] * box[1] * box[2] * box[3] * elem;
}

}  // namespace islbm
