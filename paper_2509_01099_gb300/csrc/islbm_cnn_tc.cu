// BF16 GEMM of the warm-start network on the fifth-generation tensor cores:
// tcgen05.mma with its FP32 accumulator in tensor memory (TMEM).
//
//   C[M,N] (+)= op(A)[M,K] op(B)[K,N] (+ bias[N]),  A, B in BF16, C in FP32,
//   with the operand orientations of islbm_cnn_gemm_bf16 (transA / transB).
//
// A CTA of 4 warps owns a 128 x BN tile of C (BN = 16 .. 256).  Operand tiles
// of 64 k-values are staged in shared memory in the no-swizzle K-major layout
// the MMA reads through its matrix descriptors: 8 x 8 core matrices of 8 rows
// of 16 bytes, the core matrices of a row group 128 bytes apart along k and
// the row groups 1024 bytes apart.  Operands that are K-major in global memory
// (A with transA = 0, B with transB = 1) are copied 16 bytes at a time with
// cp.async; the others are read as 8 x 8 blocks (eight 16-byte rows along M or
// N) and transposed in registers into whole core matrices.  Two stages: while thread 0 issues the four MMAs (K = 16 each)
// of one stage and commits them to that stage's mbarrier, the CTA stages the
// next one.  After the last stage every warp reads its 32 rows of the
// accumulator (tcgen05.ld) and writes them out.  Split K (for products whose
// output tiles alone cannot fill the GPU) writes partial tiles to a workspace
// that a second kernel adds up in a fixed order, so results are deterministic.
//
// The paper has no counterpart; the network predicts a steady cavity state
// that initialises the solver.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "islbm_internal.h"
#include "islbm_tma.cuh"

namespace islbm {
namespace {

constexpr int kTcBM = 128, kTcBK = 64, kTcThreads = 128, kTcStages = 2;

// device flag: a bounded wait of the tcgen05 GEMM gave up (read by
// islbm_cnn_check_timeout)
__device__ int g_tc_timeout = 0;

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// Shared-memory matrix descriptor, no swizzle: start address, leading (k)
// and stride (row-group) byte offsets, all in 16-byte units; bits 46-47 hold
// the descriptor version 1.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N / 8 and M / 16.
__host__ __device__ constexpr uint32_t tc_idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::
                   "r"(smem_u32(bar))
               : "memory");
}

// 16 consecutive FP32 columns of the calling thread's TMEM lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void cp_async16z(void* dst, const void* src, bool ok) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "r"(ok ? 16 : 0)
               : "memory");
}

// byte offset of element (row r, k) in a K-major no-swizzle tile of 64 k
__device__ __forceinline__ uint32_t tc_off(int r, int k) {
  return (uint32_t)(((r >> 3) * 8 + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Stage rows [r0, r0 + ROWS) x k [k0, k0 + 64) of an operand into the tile at
// `dst`.  kmajor: element (r, k) at src[r * ld + k]; else at src[k * ld + r].
// Out-of-range elements (r >= R, k >= kend) are zero.
template <int ROWS>
__device__ __forceinline__ void tc_stage(unsigned char* dst, const __nv_bfloat16* __restrict__ src,
                                         int ld, bool kmajor, int r0, int R, int k0, int kend) {
  if (kmajor) {
    // 16-byte chunks along k: row r, chunk c covers k0 + 8c .. +7
    for (int e = threadIdx.x; e < ROWS * 8; e += kTcThreads) {
      const int r = e >> 3, c = e & 7;
      const int gr = r0 + r, gk = k0 + 8 * c;
      const bool ok = gr < R && gk + 8 <= kend;
      unsigned char* d = dst + tc_off(r, 8 * c);
      if (ok || gr >= R || gk >= kend) {
        cp_async16z(d, ok ? static_cast<const void*>(src + (size_t)gr * ld + gk) : src, ok);
      } else {   // a chunk cut by the end of k
        __nv_bfloat16 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
          v[j] = gk + j < kend ? src[(size_t)gr * ld + gk + j] : __float2bfloat16(0.f);
        *reinterpret_cast<uint4*>(d) = *reinterpret_cast<const uint4*>(v);
      }
    }
  } else {
    // 8 x 8 blocks: eight 16-byte rows along r (one per k), transposed in
    // registers into the eight 16-byte rows along k of one core matrix
    for (int e = threadIdx.x; e < (ROWS / 8) * 8; e += kTcThreads) {
      const int rb = e >> 3, kb = e & 7;
      const int gr = r0 + 8 * rb, gk = k0 + 8 * kb;
      uint32_t w[8][4];   // w[kk]: r-pairs (0,1) (2,3) (4,5) (6,7) at k = gk + kk
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        if (gk + kk < kend && gr + 8 <= R) {
          const uint4 q = __ldg(reinterpret_cast<const uint4*>(src + (size_t)(gk + kk) * ld + gr));
          w[kk][0] = q.x;
          w[kk][1] = q.y;
          w[kk][2] = q.z;
          w[kk][3] = q.w;
        } else {
          __nv_bfloat16 v[8];
#pragma unroll
          for (int j = 0; j < 8; ++j)
            v[j] = (gk + kk < kend && gr + j < R) ? src[(size_t)(gk + kk) * ld + gr + j]
                                                   : __float2bfloat16(0.f);
          const uint4 q = *reinterpret_cast<const uint4*>(v);
          w[kk][0] = q.x;
          w[kk][1] = q.y;
          w[kk][2] = q.z;
          w[kk][3] = q.w;
        }
      }
      unsigned char* core = dst + (uint32_t)((rb * 8 + kb) * 128);
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) {
        // row rr of the core matrix: k-pairs (0,1) .. (6,7) at r = gr + rr
        const unsigned sel = (rr & 1) ? 0x7632u : 0x5410u;
        uint4 o;
        o.x = __byte_perm(w[0][rr >> 1], w[1][rr >> 1], sel);
        o.y = __byte_perm(w[2][rr >> 1], w[3][rr >> 1], sel);
        o.z = __byte_perm(w[4][rr >> 1], w[5][rr >> 1], sel);
        o.w = __byte_perm(w[6][rr >> 1], w[7][rr >> 1], sel);
        *reinterpret_cast<uint4*>(core + rr * 16) = o;
      }
    }
  }
}

template <int BN>
struct TcGeom {
  static constexpr unsigned A_BYTES = kTcBM * kTcBK * 2;   // 16 KB
  static constexpr unsigned B_BYTES = BN * kTcBK * 2;
  static constexpr unsigned STAGE = A_BYTES + B_BYTES;
  static constexpr unsigned TMEM_COLS = BN < 32 ? 32 : BN;   // a power of two >= 32
  static constexpr size_t smem_bytes() { return (size_t)kTcStages * STAGE + 64; }
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "M = 128 MMAs take N = 16 .. 256");
  static_assert((BN & (BN - 1)) == 0, "the TMEM allocation is a power of two");
  static_assert(STAGE % 128 == 0, "stages stay 128-byte aligned");
};

// out == nullptr: write C (bias / accumulate as asked); else the split's
// partial tile into out[blockIdx.z][M][N].
template <int BN>
__global__ void __launch_bounds__(kTcThreads)
    k_gemm_tc(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ B,
              float* __restrict__ C, const float* __restrict__ bias, int M, int N, int K, int lda,
              int ldb, int ldc, int transA, int transB, int accumulate, int kchunk,
              float* __restrict__ partial) {
  using G = TcGeom<BN>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + kTcStages * G::STAGE);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + kTcStages);
  int* abort = reinterpret_cast<int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kTcBM, n0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) mbar_init(&bars[s], 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(G::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  constexpr uint32_t idesc = tc_idesc(kTcBM, BN);

  const int ntiles = (kend - kbeg + kTcBK - 1) / kTcBK;
  for (int t = 0; t < ntiles; ++t) {
    const int st = t % kTcStages;
    unsigned char* sA = smem_raw + st * G::STAGE;
    unsigned char* sB = sA + G::A_BYTES;
    if (t >= kTcStages) {
      // the MMAs that read this stage two tiles ago have completed
      const bool ok = mbar_wait(&bars[st], (unsigned)((t / kTcStages) - 1) & 1u);
      if (!ok) *abort = 1;
    }
    __syncthreads();
    if (*abort) break;
    const int k0 = kbeg + t * kTcBK;
    tc_stage<kTcBM>(sA, A, lda, transA == 0, m0, M, k0, kend);
    tc_stage<BN>(sB, B, ldb, transB != 0, n0, N, k0, kend);
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
      for (int ks = 0; ks < kTcBK / 16; ++ks)
        tc_mma(tmem, tc_desc(a0 + 256u * ks, 128u, 1024u), tc_desc(b0 + 256u * ks, 128u, 1024u),
               idesc, (t > 0 || ks > 0) ? 1u : 0u);
      tc_commit(&bars[st]);
    }
  }
  // the last commit covers every MMA issued before it
  bool ok = !*abort;
  if (ok && ntiles > 0) {
    const int t = ntiles - 1;
    ok = mbar_wait(&bars[t % kTcStages], (unsigned)(t / kTcStages) & 1u);
  }
  if (!ok) {
    atomicExch(&g_tc_timeout, 1);
    // wait (bounded) for the MMAs still in flight before the tile is freed
    for (int t = max(0, ntiles - kTcStages); t < ntiles; ++t)
      mbar_wait(&bars[t % kTcStages], (unsigned)(t / kTcStages) & 1u);
  }
  tc_fence_after();
  if (ok) {
    // rows 32 warp .. +31 of the accumulator live in TMEM lanes 32 warp .. +31
    const int row = m0 + 32 * warp + lane;
    const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      tc_ld16(taddr + (uint32_t)c0, v);
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = n0 + c0 + j;
          if (col >= N) continue;
          if (partial) {
            partial[((size_t)blockIdx.z * M + row) * N + col] = v[j];
          } else {
            float r = v[j];
            if (bias) r += bias[col];
            float* dst = C + (size_t)row * ldc + col;
            *dst = accumulate ? *dst + r : r;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(G::TMEM_COLS)
                 : "memory");
  }
}

// C (+)= sum over the splits of the partial tiles, in split order (+ bias).
__global__ void k_splitk_sum(const float* __restrict__ partial, int split, int M, int N,
                             float* __restrict__ C, int ldc, const float* __restrict__ bias,
                             int accumulate) {
  const long long total = (long long)M * N;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < split; ++z) s += partial[(size_t)z * total + e];
    const int m = (int)(e / N), n = (int)(e - (long long)m * N);
    if (bias) s += bias[n];
    float* dst = C + (size_t)m * ldc + n;
    *dst = accumulate ? *dst + s : s;
  }
}

// Split-K workspace, one per device, grown on demand (the device is idle while
// a buffer is replaced).
std::mutex g_ws_mutex;
float* g_ws[64] = {nullptr};
size_t g_ws_bytes[64] = {0};
DevAllocator g_ws_mem[64];

}  // namespace

cudaError_t cnn_splitk_workspace(size_t bytes, float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_ws_mutex);
  if (g_ws_bytes[dev] < bytes) {
    // the old buffer may still be read by work in flight on any stream
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    if (g_ws[dev]) dev_free(g_ws_mem[dev], g_ws[dev], nullptr);
    g_ws[dev] = nullptr;
    g_ws_bytes[dev] = 0;
    g_ws_mem[dev] = current_allocator();
    e = dev_alloc(g_ws_mem[dev], reinterpret_cast<void**>(&g_ws[dev]), bytes, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    g_ws_bytes[dev] = bytes;
  }
  *out = g_ws[dev];
  return cudaSuccess;
}

cudaError_t launch_splitk_sum(const float* partial, int split, int M, int N, float* C, int ldc,
                              const float* bias, int accumulate, cudaStream_t stream) {
  const long long n = (long long)M * N;
  const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
  k_splitk_sum<<<blocks, 256, 0, stream>>>(partial, split, M, N, C, ldc, bias, accumulate);
  return cudaGetLastError();
}

namespace {

template <int BN>
cudaError_t run_tc(const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, const float* bias,
                   int M, int N, int K, int lda, int ldb, int ldc, int transA, int transB,
                   int accumulate, cudaStream_t stream, int sms) {
  using G = TcGeom<BN>;
  const cudaError_t e0 = launch_setup_once(
      reinterpret_cast<const void*>(k_gemm_tc<BN>),
      [](const void* k, int*) {
        return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)TcGeom<BN>::smem_bytes());
      },
      nullptr);
  if (e0 != cudaSuccess) return e0;
  const int gx = (N + BN - 1) / BN, gy = (M + kTcBM - 1) / kTcBM;
  const long long tiles = (long long)gx * gy;
  // split K when the output tiles alone leave most SMs idle
  int split = 1;
  if (tiles < 2LL * sms && K >= 8 * kTcBK) {
    split = (int)std::min<long long>((2LL * sms + tiles - 1) / tiles, K / (4 * kTcBK));
    split = std::max(split, 1);
  }
  const int kchunk = ((K + split - 1) / split + kTcBK - 1) / kTcBK * kTcBK;
  split = (K + kchunk - 1) / kchunk;
  float* part = nullptr;
  if (split > 1) {
    const cudaError_t e = cnn_splitk_workspace((size_t)split * M * N * sizeof(float), &part);
    if (e != cudaSuccess) return e;
  }
  const dim3 grid(gx, gy, split);
  k_gemm_tc<BN><<<grid, kTcThreads, G::smem_bytes(), stream>>>(
      A, B, C, bias, M, N, K, lda, ldb, ldc, transA, transB, accumulate, kchunk, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || split == 1) return e;
  return launch_splitk_sum(part, split, M, N, C, ldc, bias, accumulate, stream);
}

}  // namespace

bool cnn_gemm_tc_supported(const void* A, const void* B, int M, int N, int K, int lda, int ldb) {
  (void)M;
  (void)N;
  (void)K;
  // 16-byte chunks of both operands: leading dimensions in multiples of 8
  // elements and 16-byte aligned bases
  return lda % 8 == 0 && ldb % 8 == 0 && (reinterpret_cast<uintptr_t>(A) & 15u) == 0 &&
         (reinterpret_cast<uintptr_t>(B) & 15u) == 0;
}

cudaError_t launch_cnn_gemm_tc(const void* A, const void* B, float* C, const float* bias, int M,
                               int N, int K, int lda, int ldb, int ldc, int transA, int transB,
                               int accumulate, cudaStream_t stream, int sms) {
  const auto* a = static_cast<const __nv_bfloat16*>(A);
  const auto* b = static_cast<const __nv_bfloat16*>(B);
#define ISLBM_TC(BNV) \
  run_tc<BNV>(a, b, C, bias, M, N, K, lda, ldb, ldc, transA, transB, accumulate, stream, sms)
  if (N <= 16) return ISLBM_TC(16);
  if (N <= 32) return ISLBM_TC(32);
  if (N <= 64) return ISLBM_TC(64);
  if (N <= 128) return ISLBM_TC(128);
  return ISLBM_TC(256);
#undef ISLBM_TC
}

int cnn_tc_timeout_flag(int reset) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_timeout, sizeof(int)) != cudaSuccess) return -1;
  if (reset && v) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_tc_timeout, &zero, sizeof(int));
  }
  return v;
}

}  // namespace islbm
