// Kernels of the warm-start network: a BF16 tensor-core GEMM with FP32
// accumulation (forward, backward-data and backward-weight products of the
// fully connected and 3x3 convolution layers, the convolutions as im2col
// GEMMs), and the elementwise pieces around it (NHWC layout throughout).
// The paper has no counterpart; the network predicts a steady cavity state
// that initialises the solver.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "islbm_internal.h"

namespace {

// ---------------------------------------------------------------------------
// C[M,N] (+)= op(A)[M,K] op(B)[K,N] (+ bias[N]).  A, B in BF16, C in FP32.
//   transA = 0: A is M x K row-major (lda >= K); 1: A is K x M row-major.
//   transB = 0: B is K x N row-major (ldb >= N); 1: B is N x K row-major.
// 128 threads = 4 warps in 2 x 2, block tile 64 x 64, k-step 32; each warp
// computes 32 x 32 with mma.sync.m16n8k16 (2 x 4 fragments).  Tiles are
// staged in shared memory in the fragment-friendly orientation (A as [m][k],
// B as [n][k]); out-of-range elements are zero.
// ---------------------------------------------------------------------------
constexpr int GM = 64, GN = 64, GK = 32;
constexpr int SPAD = 8;   // row padding (bf16) against bank conflicts

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4],
                                               const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128)
    k_gemm_bf16(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ B,
                float* __restrict__ C, const float* __restrict__ bias, int M, int N, int K,
                int lda, int ldb, int ldc, int transA, int transB, int accumulate, int kchunk,
                float* __restrict__ partial) {
  __shared__ __nv_bfloat16 sA[GM][GK + SPAD];
  __shared__ __nv_bfloat16 sB[GN][GK + SPAD];
  const int m0 = blockIdx.y * GM, n0 = blockIdx.x * GN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int grp = lane >> 2, tig = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
  const __nv_bfloat16 zero = __float2bfloat16(0.f);
  // split-K: block z covers k in [z kchunk, (z + 1) kchunk) and adds its part
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  for (int k0 = kbeg; k0 < kend; k0 += GK) {
    // stage A tile as [m][k] and B tile as [n][k]
    for (int e = threadIdx.x; e < GM * GK; e += 128) {
      const int mm = transA ? (e % GM) : (e / GK);
      const int kk = transA ? (e / GM) : (e % GK);
      const int gm = m0 + mm, gk = k0 + kk;
      __nv_bfloat16 v = zero;
      if (gm < M && gk < kend) v = transA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
      sA[mm][kk] = v;
    }
    for (int e = threadIdx.x; e < GN * GK; e += 128) {
      const int nn = transB ? (e / GK) : (e % GN);
      const int kk = transB ? (e % GK) : (e / GN);
      const int gn = n0 + nn, gk = k0 + kk;
      __nv_bfloat16 v = zero;
      if (gn < N && gk < kend) v = transB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
      sB[nn][kk] = v;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < GK; ks += 16) {
      uint32_t af[2][4], bf[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + 16 * i + grp;
        const int c = ks + 2 * tig;
        af[i][0] = pack_bf16(sA[r][c], sA[r][c + 1]);
        af[i][1] = pack_bf16(sA[r + 8][c], sA[r + 8][c + 1]);
        af[i][2] = pack_bf16(sA[r][c + 8], sA[r][c + 9]);
        af[i][3] = pack_bf16(sA[r + 8][c + 8], sA[r + 8][c + 9]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = wn + 8 * j + grp;
        const int c = ks + 2 * tig;
        bf[j][0] = pack_bf16(sB[n][c], sB[n][c + 1]);
        bf[j][1] = pack_bf16(sB[n][c + 8], sB[n][c + 9]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16_16816(acc[i][j], af[i], bf[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int gm = m0 + wm + 16 * i + grp + (r >= 2 ? 8 : 0);
        const int gn = n0 + wn + 8 * j + 2 * tig + (r & 1);
        if (gm < M && gn < N) {
          float v = acc[i][j][r];
          if (partial) {   // split K: this split's part, summed in a fixed order later
            partial[((size_t)blockIdx.z * M + gm) * N + gn] = v;
            continue;
          }
          if (bias) v += bias[gn];
          float* dst = C + (size_t)gm * ldc + gn;
          *dst = accumulate ? *dst + v : v;
        }
      }
}

// 3x3 'same' im2col of an NHWC FP32 tensor into BF16 rows [b,y,x][dy][dx][c],
// zero-padded to kpad columns.
__global__ void k_im2col(const float* __restrict__ in, __nv_bfloat16* __restrict__ col, int Bn,
                         int H, int W, int C, int kpad) {
  const long long total = (long long)Bn * H * W * kpad;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e % kpad);
    const long long pix = e / kpad;
    float v = 0.f;
    if (k < 9 * C) {
      const int c = k % C, tap = k / C;
      const int dy = tap / 3 - 1, dx = tap % 3 - 1;
      const int x = (int)(pix % W);
      const long long r = pix / W;
      const int y = (int)(r % H), b = (int)(r / H);
      const int yy = y + dy, xx = x + dx;
      if (yy >= 0 && yy < H && xx >= 0 && xx < W)
        v = in[(((long long)b * H + yy) * W + xx) * C + c];
    }
    col[e] = __float2bfloat16(v);
  }
}

// Adjoint of k_im2col: din[b,y,x,c] = sum over the 9 taps of dcol at the
// neighbour that read (y, x) (a gather, no atomics).
__global__ void k_col2im(const float* __restrict__ dcol, float* __restrict__ din, int Bn, int H,
                         int W, int C, int kpad) {
  const long long total = (long long)Bn * H * W * C;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    const long long pix = e / C;
    const int x = (int)(pix % W);
    const long long r = pix / W;
    const int y = (int)(r % H), b = (int)(r / H);
    float s = 0.f;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int dy = tap / 3 - 1, dx = tap % 3 - 1;
      const int oy = y - dy, ox = x - dx;   // output pixel whose tap read (y, x)
      if (oy >= 0 && oy < H && ox >= 0 && ox < W)
        s += dcol[(((long long)b * H + oy) * W + ox) * kpad + tap * C + c];
    }
    din[e] = s;
  }
}

__global__ void k_upsample2x(const float* __restrict__ in, float* __restrict__ out, int Bn, int H,
                             int W, int C) {
  const long long total = (long long)Bn * 4 * H * W * C;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    const long long pix = e / C;
    const int x = (int)(pix % (2 * W));
    const long long r = pix / (2 * W);
    const int y = (int)(r % (2 * H)), b = (int)(r / (2 * H));
    out[e] = in[(((long long)b * H + y / 2) * W + x / 2) * C + c];
  }
}

__global__ void k_upsample2x_back(const float* __restrict__ dout, float* __restrict__ din, int Bn,
                                  int H, int W, int C) {
  const long long total = (long long)Bn * H * W * C;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    const long long pix = e / C;
    const int x = (int)(pix % W);
    const long long r = pix / W;
    const int y = (int)(r % H), b = (int)(r / H);
    const long long W2 = 2LL * W;
    const long long base = (((long long)b * 2 * H + 2 * y) * W2 + 2 * x) * C + c;
    din[e] = dout[base] + dout[base + C] + dout[base + W2 * C] + dout[base + W2 * C + C];
  }
}

__global__ void k_tanh(float* __restrict__ x, long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    x[e] = tanhf(x[e]);
}

// dx = dy * (1 - y^2) for y = tanh(x)
__global__ void k_tanh_back(const float* __restrict__ y, float* __restrict__ dy, long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    dy[e] = dy[e] * (1.f - y[e] * y[e]);
}

__global__ void k_to_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    y[e] = __float2bfloat16(x[e]);
}

// Column sums of an M x N row-major matrix (bias gradients).  Block (32, 8):
// 32 columns, 8 row lanes; block (x, y) sums rows [y * kColsumRows, ...) of its
// columns into partial[y][n]; the chunks are then added in a fixed order, so
// the sums do not depend on scheduling.
constexpr int kColsumRows = 2048;
__global__ void k_colsum(const float* __restrict__ x, float* __restrict__ partial, int M, int N) {
  const int n = blockIdx.x * 32 + threadIdx.x;
  const long long m0 = (long long)blockIdx.y * kColsumRows;
  const long long m1 = m0 + kColsumRows < M ? m0 + kColsumRows : M;
  float s = 0.f;
  if (n < N)
    for (long long m = m0 + threadIdx.y; m < m1; m += 8) s += x[m * N + n];
  __shared__ float sh[8][33];
  sh[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && n < N) {
    float t = 0.f;
#pragma unroll
    for (int r = 0; r < 8; ++r) t += sh[r][threadIdx.x];
    partial[(size_t)blockIdx.y * N + n] = t;
  }
}

// mean squared error over n values with weights w (per channel, period C):
// loss partials per block and the gradient 2 w (y - t) / n
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t,
                      const float* __restrict__ wc, int C, float* __restrict__ dy,
                      double* __restrict__ partial, long long n) {
  double acc = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const float w = wc ? wc[e % C] : 1.f;
    const float d = y[e] - t[e];
    acc += (double)w * d * d;
    dy[e] = 2.f * w * d / (float)n;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double sh[8];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    partial[blockIdx.x] = s;
  }
}

// Adam (Kingma & Ba) on FP32 master weights; also writes the BF16 copy
__global__ void k_adam(float* __restrict__ w, __nv_bfloat16* __restrict__ wb,
                       const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.f - b1) * gg;
    const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    const float upd = lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    const float nw = w[e] - upd;
    w[e] = nw;
    if (wb) wb[e] = __float2bfloat16(nw);
  }
}

// Solver fields (FP64, one array per field) <-> network channels (NHWC FP32):
// y = ((T - T_mid) / T_scale, u / u_scale, v / u_scale).
__global__ void k_pack_fields(const double* __restrict__ T, const double* __restrict__ u,
                              const double* __restrict__ v, long long nodes, double T_mid,
                              double T_scale, double u_scale, float* __restrict__ y) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nodes;
       k += (long long)gridDim.x * blockDim.x) {
    y[3 * k] = (float)((T[k] - T_mid) / T_scale);
    y[3 * k + 1] = (float)(u[k] / u_scale);
    y[3 * k + 2] = (float)(v[k] / u_scale);
  }
}

__global__ void k_unpack_fields(const float* __restrict__ y, long long nodes, double T_mid,
                                double T_scale, double u_scale, double* __restrict__ T,
                                double* __restrict__ u, double* __restrict__ v) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nodes;
       k += (long long)gridDim.x * blockDim.x) {
    T[k] = T_mid + T_scale * (double)y[3 * k];
    u[k] = u_scale * (double)y[3 * k + 1];
    v[k] = u_scale * (double)y[3 * k + 2];
  }
}

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)(g > 4 * 1024 ? 4 * 1024 : (g < 1 ? 1 : g));
}

islbm_status launched(cudaError_t e) {
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? ISLBM_OK : ISLBM_ERR_CUDA;
}

#define CNN_STREAM static_cast<cudaStream_t>(stream)

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    sms = 1;
  return sms;
}

}  // namespace

namespace {

islbm_status gemm_mma_sync(const void* A, const void* B, float* C, const float* bias, int M,
                           int N, int K, int lda, int ldb, int ldc, int transA, int transB,
                           int accumulate, void* stream) {
  const int gx = (N + GN - 1) / GN, gy = (M + GM - 1) / GM;
  // split K over blockIdx.z when the output tiles alone do not fill the GPU
  const int sms = device_sms();
  const long long tiles = (long long)gx * gy;
  int split = 1;
  if (tiles < 2LL * sms && K >= 16 * GK) {
    split = (int)((2LL * sms + tiles - 1) / tiles);
    split = std::min(split, K / (8 * GK));
    split = std::max(split, 1);
  }
  const int kchunk = ((K + split - 1) / split + GK - 1) / GK * GK;
  split = (K + kchunk - 1) / kchunk;
  float* part = nullptr;
  if (split > 1 &&
      islbm::cnn_splitk_workspace((size_t)split * M * N * sizeof(float), &part) != cudaSuccess)
    return ISLBM_ERR_OOM;
  const dim3 grid(gx, gy, split);
  k_gemm_bf16<<<grid, 128, 0, CNN_STREAM>>>(static_cast<const __nv_bfloat16*>(A),
                                            static_cast<const __nv_bfloat16*>(B), C, bias, M, N,
                                            K, lda, ldb, ldc, transA, transB, accumulate, kchunk,
                                            part);
  if (split > 1) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return launched(e);
    return launched(
        islbm::launch_splitk_sum(part, split, M, N, C, ldc, bias, accumulate, CNN_STREAM));
  }
  return launched(cudaSuccess);
}

}  // namespace

extern "C" islbm_status islbm_cnn_gemm_bf16_ex(const void* A, const void* B, float* C,
                                               const float* bias, int M, int N, int K, int lda,
                                               int ldb, int ldc, int transA, int transB,
                                               int accumulate, int path, void* stream) {
  if (!A || !B || !C || M <= 0 || N <= 0 || K <= 0 || ldc < N ||
      lda < (transA ? M : K) || ldb < (transB ? K : N) || path < 0 || path > 2)
    return ISLBM_ERR_ARG;
  const bool tc_ok = islbm::cnn_gemm_tc_supported(A, B, M, N, K, lda, ldb);
  if (path == 2 && !tc_ok) return ISLBM_ERR_ARG;
  // path 0: the tensor-core kernel, except for products with K <= 32 (the
  // data gradients of the narrow layers): a 128 x 64 tile then does too little
  // work for its setup, and the mma.sync kernel is faster (measured on GB300)
  if (path == 1 || !tc_ok || (path == 0 && K <= 32))
    return gemm_mma_sync(A, B, C, bias, M, N, K, lda, ldb, ldc, transA, transB, accumulate,
                         stream);
  return launched(islbm::launch_cnn_gemm_tc(A, B, C, bias, M, N, K, lda, ldb, ldc, transA, transB,
                                            accumulate, CNN_STREAM, device_sms()));
}

extern "C" islbm_status islbm_cnn_gemm_bf16(const void* A, const void* B, float* C,
                                            const float* bias, int M, int N, int K, int lda,
                                            int ldb, int ldc, int transA, int transB,
                                            int accumulate, void* stream) {
  return islbm_cnn_gemm_bf16_ex(A, B, C, bias, M, N, K, lda, ldb, ldc, transA, transB,
                                accumulate, 0, stream);
}

extern "C" islbm_status islbm_cnn_check_timeout(int reset, int* timed_out) {
  if (!timed_out) return ISLBM_ERR_ARG;
  const int v = islbm::cnn_tc_timeout_flag(reset);
  if (v < 0) return ISLBM_ERR_CUDA;
  *timed_out = v;
  return ISLBM_OK;
}

extern "C" islbm_status islbm_cnn_im2col(const float* in, void* col, int Bn, int H, int W, int C,
                                         int kpad, void* stream) {
  if (!in || !col || kpad < 9 * C) return ISLBM_ERR_ARG;
  const long long n = (long long)Bn * H * W * kpad;
  k_im2col<<<grid_for(n), 256, 0, CNN_STREAM>>>(in, static_cast<__nv_bfloat16*>(col), Bn, H, W,
                                                C, kpad);
  return launched(cudaSuccess);
}

extern "C" islbm_status islbm_cnn_col2im(const float* dcol, float* din, int Bn, int H, int W,
                                         int C, int kpad, void* stream) {
  if (!dcol || !din || kpad < 9 * C) return ISLBM_ERR_ARG;
  const long long n = (long long)Bn * H * W * C;
  k_col2im<<<grid_for(n), 256, 0, CNN_STREAM>>>(dcol, din, Bn, H, W, C, kpad);
  return launched(cudaSuccess);
}

extern "C" islbm_status islbm_cnn_upsample2x(const float* in, float* out, int Bn, int H, int W,
                                             int C, int backward, void* stream) {
  if (!in || !out) return ISLBM_ERR_ARG;
  if (!backward) {
    const long long n = 4LL * Bn * H * W * C;
    k_upsample2x<<<grid_for(n), 256, 0, CNN_STREAM>>>(in, out, Bn, H, W, C);
  } else {
    const long long n = (long long)Bn * H * W * C;   // H, W of the small tensor
    k_upsample2x_back<<<grid_for(n), 256, 0, CNN_STREAM>>>(in, out, Bn, H, W, C);
  }
  return launched(cudaSuccess);
}

extern "C" islbm_status islbm_cnn_tanh(float* x, long long n, void* stream) {
  if (!x) return ISLBM_ERR_ARG;
  k_tanh<<<grid_for(n), 256, 0, CNN_STREAM>>>(x, n);
  return launched(cudaSuccess);
}

extern "C" islbm_status islbm_cnn_tanh_back(const float* y, float* dy, long long n, void* stream) {
  if (!y || !dy) return ISLBM_ERR_ARG;
  k_tanh_back<<<grid_for(n), 256, 0, CNN_STREAM>>>(y, dy, n);
  return launched(cudaSuccess);
}

extern "C" islbm_status islbm_cnn_to_bf16(const float* x, void* y, long long n, void* stream) {
  if (!x || !y) return ISLBM_ERR_ARG;
  k_to_bf16<<<grid_for(n), 256, 0, CNN_STREAM>>>(x, static_cast<__nv_bfloat16*>(y), n);
  return launched(cudaSuccess);
}

extern "C" islbm_status islbm_cnn_colsum(const float* x, float* out, int M, int N, int accumulate,
                                         void* stream) {
  if (!x || !out || M <= 0 || N <= 0) return ISLBM_ERR_ARG;
  const int chunks = (M + kColsumRows - 1) / kColsumRows;
  float* part = nullptr;
  if (islbm::cnn_splitk_workspace((size_t)chunks * N * sizeof(float), &part) != cudaSuccess)
    return ISLBM_ERR_OOM;
  const dim3 grid((N + 31) / 32, chunks);
  k_colsum<<<grid, dim3(32, 8), 0, CNN_STREAM>>>(x, part, M, N);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return launched(e);
  return launched(islbm::launch_splitk_sum(part, chunks, 1, N, out, N, nullptr, accumulate,
                                           CNN_STREAM));
}

extern "C" islbm_status islbm_cnn_mse(const float* y, const float* t, const float* wc, int C,
                                      float* dy, double* partial, int blocks, long long n,
                                      void* stream) {
  if (!y || !t || !dy || !partial || blocks <= 0) return ISLBM_ERR_ARG;
  k_mse<<<blocks, 256, 0, CNN_STREAM>>>(y, t, wc, C, dy, partial, n);
  return launched(cudaSuccess);
}

extern "C" islbm_status islbm_cnn_adam(float* w, void* wb, const float* g, float* m, float* v,
                                       long long n, float lr, float b1, float b2, float eps,
                                       long long t, void* stream) {
  if (!w || !g || !m || !v || t < 1) return ISLBM_ERR_ARG;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  k_adam<<<grid_for(n), 256, 0, CNN_STREAM>>>(w, static_cast<__nv_bfloat16*>(wb), g, m, v, n, lr,
                                              b1, b2, eps, c1, c2);
  return launched(cudaSuccess);
}

extern "C" islbm_status islbm_cnn_pack_fields(const double* T, const double* u, const double* v,
                                              long long nodes, double T_mid, double T_scale,
                                              double u_scale, float* y, void* stream) {
  if (!T || !u || !v || !y || nodes <= 0 || !(T_scale != 0.0) || !(u_scale != 0.0))
    return ISLBM_ERR_ARG;
  k_pack_fields<<<grid_for(nodes), 256, 0, CNN_STREAM>>>(T, u, v, nodes, T_mid, T_scale, u_scale,
                                                         y);
  return launched(cudaSuccess);
}

extern "C" islbm_status islbm_cnn_unpack_fields(const float* y, long long nodes, double T_mid,
                                                double T_scale, double u_scale, double* T,
                                                double* u, double* v, void* stream) {
  if (!T || !u || !v || !y || nodes <= 0) return ISLBM_ERR_ARG;
  k_unpack_fields<<<grid_for(nodes), 256, 0, CNN_STREAM>>>(y, nodes, T_mid, T_scale, u_scale, T,
                                                           u, v);
  return launched(cudaSuccess);
}
