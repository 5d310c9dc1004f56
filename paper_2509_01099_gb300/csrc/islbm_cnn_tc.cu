// BF16 GEMM of the warm-start network on the fifth-generation tensor cores:
// tcgen05.mma with its FP32 accumulator in tensor memory (TMEM).
//
//   C[M,N] (+)= op(A)[M,K] op(B)[K,N] (+ bias[N]),  A, B in BF16, C in FP32,
//   with the operand orientations of islbm_cnn_gemm_bf16 (transA / transB).
//
// A CTA of 4 warps owns a 128 x BN tile of C (BN = 16, 32 or 64).  Operand tiles
// of 64 k-values move by TMA into a ring of kTcStages shared-memory stages, in
// the no-swizzle core-matrix layouts the MMA reads through its matrix
// descriptors.  An operand that is K-major in global memory (A with transA =
// 0, B with transB = 1) arrives as one box of 64 k x rows in the 128-byte
// swizzled layout; an MN-major one as boxes of 8 rows x 64 k (no swizzle, core
// matrices of 8 k-rows of 16 bytes), one per group of 8 rows, and the MMA reads
// it MN-major (the transpose bits of the instruction descriptor).  Warp 0 issues the copies, warp 1 the
// MMAs (K = 16 each) and their commits, which free a stage once its MMAs are
// done; after the last stage every warp reads its 32 rows of the accumulator
// (tcgen05.ld) and writes them out through shared memory in whole row
// segments.  Split K (for products whose output tiles alone cannot fill the
// GPU) writes partial tiles to a workspace that a second kernel adds up in a
// fixed order, so results are deterministic.
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

constexpr int kTcBM = 128, kTcBK = 64, kTcThreads = 128, kTcStages = 4;

// device flag: a bounded wait of the tcgen05 GEMM gave up (read by
// islbm_cnn_check_timeout)
__device__ int g_tc_timeout = 0;

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// Shared-memory matrix descriptor: start address, leading byte offset
// (between core matrices adjacent along k; unused by the 128-byte swizzle) and
// stride byte offset (between core matrices, or 8-row swizzle atoms, adjacent
// along M or N), all in 16-byte units; bits 46-47 hold the descriptor version
// 1 and bits 61-63 the layout: 0 no swizzle, 2 the 128-byte swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo,
                                            uint32_t layout) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((uint64_t)layout << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, A / B
// MN-major when a_mn / b_mn (bits 15 / 16), N / 8 and M / 16.
__host__ __device__ constexpr uint32_t tc_idesc(int m, int n, int a_mn, int b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
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

template <int BN>
struct TcGeom {
  static constexpr unsigned A_BYTES = kTcBM * kTcBK * 2;   // 16 KB
  static constexpr unsigned B_BYTES = BN * kTcBK * 2;
  static constexpr unsigned STAGE = A_BYTES + B_BYTES;
  static constexpr unsigned TMEM_COLS = BN < 32 ? 32 : BN;   // a power of two >= 32
  // stages, then full[S], empty[S], done, the TMEM address and the abort word
  static constexpr size_t smem_bytes() { return (size_t)kTcStages * STAGE + 8 * (2 * kTcStages + 1) + 16; }
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "M = 128 MMAs take N = 16 .. 256");
  static_assert((BN & (BN - 1)) == 0, "the TMEM allocation is a power of two");
  static_assert(STAGE % 1024 == 0, "stages stay 1024-byte aligned");
  static_assert(STAGE >= 4 * 32 * 17 * 4, "the epilogue's patches fit in a stage");
};

// Shared-memory layout of an operand tile of `rows` rows x 64 k in a stage.
// K-major: one TMA box of 64 k x rows with the 128-byte swizzle, i.e. rows of
// 128 bytes whose 16-byte chunks are permuted by (row mod 8); 8-row atoms lie
// 1024 bytes apart (stride offset) and the next 16 k start 32 bytes further.
// MN-major: boxes of 8 rows x 64 k without swizzle, 1024 bytes apart (stride
// offset), the k groups of 8 lying 128 bytes apart inside them (leading
// offset); the next 16 k start 256 bytes further.
__device__ __forceinline__ void tc_layout(bool mn, uint32_t& lbo, uint32_t& sbo, uint32_t& k16,
                                          uint32_t& layout) {
  if (mn) {
    lbo = 128u;
    sbo = 1024u;
    k16 = 256u;
    layout = 0u;
  } else {
    lbo = 16u;
    sbo = 1024u;
    k16 = 32u;
    layout = 2u;
  }
}

// The copies of one operand tile: rows r0 .. r0 + rows - 1, k k0 .. k0 + 63.
__device__ __forceinline__ void tc_issue(const CUtensorMap* map, bool mn, int rows,
                                         unsigned char* dst, int r0, int k0, uint64_t* bar) {
  if (mn) {
    for (int g = 0; g < rows / 8; ++g) tma_load_2d(dst + g * 1024, map, r0 + 8 * g, k0, bar);
  } else {
    tma_load_2d(dst, map, k0, r0, bar);
  }
}

// ta / tb: TMA descriptors of A and B (2-D, BF16; see tc_issue); a_mn / b_mn:
// the operand is MN-major in global memory.  partial == nullptr: write C (bias
// / accumulate as asked); else the split's partial tile into
// partial[blockIdx.z][M][N].
template <int BN>
__global__ void __launch_bounds__(kTcThreads)
    k_gemm_tc(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
              float* __restrict__ C, const float* __restrict__ bias, int M, int N, int K,
              int ldc, int a_mn, int b_mn, int accumulate, int kchunk,
              float* __restrict__ partial) {
  using G = TcGeom<BN>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + kTcStages * G::STAGE);
  uint64_t* empty = full + kTcStages;
  uint64_t* done = empty + kTcStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* abort = reinterpret_cast<int*>(tmem_slot + 1);
  int* issued = abort + 1;     // tiles whose copies were issued
  int* consumed = issued + 1;  // tiles whose MMAs were issued
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kTcBM, n0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
  const int ntiles = (kend - kbeg + kTcBK - 1) / kTcBK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *abort = 0;
    *issued = 0;
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("prefetch.tensormap [%0];\n" ::"l"(&ta) : "memory");
    asm volatile("prefetch.tensormap [%0];\n" ::"l"(&tb) : "memory");
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

  if (threadIdx.x == 0) {
    // producer: a stage is refilled once the MMAs that read it have completed
    int t = 0;
    for (; t < ntiles; ++t) {
      const int st = t % kTcStages;
      if (t >= kTcStages &&
          !mbar_wait(&empty[st], (unsigned)((t / kTcStages) - 1) & 1u)) {
        atomicExch(abort, 1);
        break;
      }
      if (*reinterpret_cast<volatile int*>(abort)) break;
      unsigned char* sA = smem_raw + st * G::STAGE;
      mbar_expect_tx(&full[st], G::STAGE);
      const int k0 = kbeg + t * kTcBK;
      tc_issue(&ta, a_mn != 0, kTcBM, sA, m0, k0, &full[st]);
      tc_issue(&tb, b_mn != 0, BN, sA + G::A_BYTES, n0, k0, &full[st]);
    }
    *issued = t;
  } else if (threadIdx.x == 32) {
    // MMA issuer: four MMAs of K = 16 per stage, committed to the stage's
    // `empty` barrier; the last commit also arrives on `done`
    constexpr uint32_t base = tc_idesc(kTcBM, BN, 0, 0);
    const uint32_t idesc = base | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16);
    uint32_t alb, asb, ak, al, blb, bsb, bk, bl;
    tc_layout(a_mn != 0, alb, asb, ak, al);
    tc_layout(b_mn != 0, blb, bsb, bk, bl);
    int t = 0;
    for (; t < ntiles; ++t) {
      const int st = t % kTcStages;
      if (!mbar_wait(&full[st], (unsigned)(t / kTcStages) & 1u)) {
        atomicExch(abort, 1);
        break;
      }
      tc_fence_after();
      const uint32_t a0 = smem_u32(smem_raw + st * G::STAGE), b0 = a0 + G::A_BYTES;
#pragma unroll
      for (int ks = 0; ks < kTcBK / 16; ++ks)
        tc_mma(tmem, tc_desc(a0 + ak * ks, alb, asb, al), tc_desc(b0 + bk * ks, blb, bsb, bl),
               idesc, (t > 0 || ks > 0) ? 1u : 0u);
      tc_commit(&empty[st]);
    }
    *consumed = t;
    tc_commit(done);   // arrives once every MMA issued above has completed
  }
  // every thread: the accumulator is complete (or the block gave up); the
  // verdict is the block's, so that every warp takes the same path below
  const bool ok = __syncthreads_and(mbar_wait(done, 0u) ? 1 : 0) &&
                  !*reinterpret_cast<volatile int*>(abort);
  if (!ok && threadIdx.x == 0) {
    atomicExch(&g_tc_timeout, 1);
    // copies issued but never consumed may still land: wait for them (bounded)
    for (int t = *consumed; t < *issued; ++t)
      mbar_wait(&full[t % kTcStages], (unsigned)(t / kTcStages) & 1u);
  }
  tc_fence_after();
  __syncthreads();   // the operand stages are free
  if (ok) {
    // rows 32 warp .. +31 of the accumulator live in TMEM lanes 32 warp .. +31.
    // Each 32 x 16 chunk goes through the warp's patch of shared memory so
    // that a store instruction writes two rows of 16 consecutive columns
    // instead of one column of 32 rows.
    float* patch = reinterpret_cast<float*>(smem_raw) + warp * (32 * 17);
    const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
    const int half = lane >> 4, cl = lane & 15;
    float* out = partial ? partial + (size_t)blockIdx.z * M * N : C;
    const int ld = partial ? N : ldc;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      tc_ld16(taddr + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) patch[lane * 17 + j] = v[j];
      __syncwarp();
      const int col = n0 + c0 + cl;
      const float b = (!partial && bias && col < N) ? bias[col] : 0.f;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int rl = 2 * i + half;             // row of the patch
        const int row = m0 + 32 * warp + rl;
        if (row < M && col < N) {
          float r = patch[rl * 17 + cl];
          float* dst = out + (size_t)row * ld + col;
          if (!partial) {
            r += b;
            if (accumulate) r += *dst;
          }
          *dst = r;
        }
      }
      __syncwarp();
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

typedef CUresult (*TcEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                               const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                               const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                               CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

TcEncodeFn tc_encode_fn() {
  static TcEncodeFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<TcEncodeFn>(f);
  }();
  return fn;
}

// 2-D descriptor of a row-major BF16 operand of `nrows` rows (stride ld
// elements) and `ncols` columns: K-major (columns = k) with boxes of 64 k x
// `rows` rows and the 128-byte swizzle, or MN-major (columns = M or N) with
// boxes of 8 x 64 k, no swizzle.
cudaError_t tc_map(CUtensorMap* map, const void* base, int nrows, int ncols, int ld, bool mn,
                   int rows) {
  TcEncodeFn fn = tc_encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {(cuuint64_t)ncols, (cuuint64_t)nrows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {mn ? 8u : 64u, mn ? 64u : (cuuint32_t)rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        mn ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

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
  // A: M x K row-major (transA = 0, K-major) or K x M (MN-major); B: N x K
  // (transB = 1, K-major) or K x N (MN-major)
  const bool a_mn = transA != 0, b_mn = transB == 0;
  CUtensorMap ta, tb;
  cudaError_t e = a_mn ? tc_map(&ta, A, K, M, lda, true, kTcBM)
                       : tc_map(&ta, A, M, K, lda, false, kTcBM);
  if (e == cudaSuccess)
    e = b_mn ? tc_map(&tb, B, K, N, ldb, true, BN) : tc_map(&tb, B, N, K, ldb, false, BN);
  if (e != cudaSuccess) return e;
  const int gx = (N + BN - 1) / BN, gy = (M + kTcBM - 1) / kTcBM;
  const long long tiles = (long long)gx * gy;
  // split K when the output tiles alone leave most SMs idle; a split is a
  // whole number of 64-wide k stages, so no copy crosses into the next split
  int split = 1;
  if (tiles < 2LL * sms && K >= 8 * kTcBK) {
    split = (int)std::min<long long>((2LL * sms + tiles - 1) / tiles, K / (4 * kTcBK));
    split = std::max(split, 1);
  }
  const int kchunk = ((K + split - 1) / split + kTcBK - 1) / kTcBK * kTcBK;
  split = (K + kchunk - 1) / kchunk;
  float* part = nullptr;
  if (split > 1) {
    e = cnn_splitk_workspace((size_t)split * M * N * sizeof(float), &part);
    if (e != cudaSuccess) return e;
  }
  const dim3 grid(gx, gy, split);
  k_gemm_tc<BN><<<grid, kTcThreads, G::smem_bytes(), stream>>>(
      ta, tb, C, bias, M, N, K, ldc, a_mn ? 1 : 0, b_mn ? 1 : 0, accumulate, kchunk, part);
  e = cudaGetLastError();
  if (e != cudaSuccess || split == 1) return e;
  return launch_splitk_sum(part, split, M, N, C, ldc, bias, accumulate, stream);
}

}  // namespace

bool cnn_gemm_tc_supported(const void* A, const void* B, int M, int N, int K, int lda, int ldb) {
  (void)M;
  (void)N;
  (void)K;
  // TMA copies of both operands: leading dimensions in multiples of 8
  // elements (16-byte strides) and 16-byte aligned bases
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
  // tiles of up to 64 columns: a 128 x 64 tile in four stages leaves room for
  // two blocks per SM, and wide products (the data gradients, N = 9 C_in up to
  // 576) then spread over more blocks
  if (N <= 16) return ISLBM_TC(16);
  if (N <= 32) return ISLBM_TC(32);
  return ISLBM_TC(64);
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
