// Host side of the C ABI declared in include/islbm.h.
//
// Set-up follows the paper: meshes (Sec. 2.3, Table 1), lattice-unit
// parameters (Sec. 2.1, Sec. 3), per-axis quadratic Lagrange tables for the
// virtual streaming (Sec. 2.2, built once in FP64), and the finishing of the
// Nu / Re reductions (Sec. 3, Sec. 4, Eq. (17), Eq. (18)).
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "islbm_internal.h"

using namespace islbm;

namespace {

// Last error of the calling thread, in a fixed buffer (copying a message into
// it allocates nothing).
thread_local char g_last_error[512] = {0};

void copy_last_error(const char* msg) {
  std::strncpy(g_last_error, msg, sizeof(g_last_error) - 1);
  g_last_error[sizeof(g_last_error) - 1] = 0;
}

islbm_status fail(Solver* s, islbm_status st, const std::string& msg) {
  if (s) s->err = msg;
  copy_last_error(msg.c_str());
  return st;
}

islbm_status cuda_fail(Solver* s, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(s, e == cudaErrorMemoryAllocation ? ISLBM_ERR_OOM : ISLBM_ERR_CUDA, m);
}

#define CK(s, call)                                   \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(s, e_, #call); \
  } while (0)

// Mirror a mesh so that xi[n+1-j] = 1 - xi[j] holds exactly.
void make_symmetric(double* xi, int n) {
  for (int j = (n + 2) / 2; j <= n + 1; ++j) xi[j] = 1.0 - xi[n + 1 - j];
}

// Lattice coordinates X_j = (xi_j - xi_0)/(xi_1 - xi_0) (1 l.u. = minimal
// resolution, Table 1); integer to rounding means the uniform mesh.
std::vector<double> lattice_coords(const double* xi, int n, bool* uniform) {
  std::vector<double> X(n + 2);
  const double lu = xi[1] - xi[0];
  double dev = 0.0;
  for (int j = 0; j < n + 2; ++j) {
    X[j] = (xi[j] - xi[0]) / lu;
    dev = std::fmax(dev, std::fabs(X[j] - std::nearbyint(X[j])));
  }
  *uniform = dev < 1e-9;
  if (*uniform)
    for (int j = 0; j < n + 2; ++j) X[j] = std::nearbyint(X[j]);
  return X;
}

// Per-axis interpolation tables (Sec. 2.2).  For direction c the value at node
// j is the quadratic Lagrange interpolant through nodes b, b+1, b+2 evaluated
// at the departure point X_j - c.  A departure point behind a half-way wall
// (j = 1 with c = +1, j = n with c = -1) is flagged with base -1.
void build_axis(Axis& a, const double* xi, int n, int stencil) {
  a.n = n;
  a.X = lattice_coords(xi, n, &a.uniform);
  a.W.resize(n);
  for (int j = 1; j <= n; ++j) a.W[j - 1] = 0.5 * (a.X[j + 1] - a.X[j - 1]);  // Eq. (18)
  for (int k = 0; k < 2; ++k) {
    const int c = k == 0 ? +1 : -1;
    a.base[k].assign(n, -1);
    a.w[k].assign(3 * n, 0.0);
    for (int j = 1; j <= n; ++j) {
      if ((j == 1 && c == +1) || (j == n && c == -1)) continue;
      int b = stencil == ISLBM_STENCIL_UPWIND ? j - 1 - c : j - 1;
      b = b < 1 ? 1 : (b > n - 2 ? n - 2 : b);
      const double d = a.X[j] - c;
      const double x0 = a.X[b], x1 = a.X[b + 1], x2 = a.X[b + 2];
      a.base[k][j - 1] = b - 1;
      a.w[k][3 * (j - 1) + 0] = (d - x1) * (d - x2) / ((x0 - x1) * (x0 - x2));
      a.w[k][3 * (j - 1) + 1] = (d - x0) * (d - x2) / ((x1 - x0) * (x1 - x2));
      a.w[k][3 * (j - 1) + 2] = (d - x0) * (d - x1) / ((x2 - x0) * (x2 - x1));
    }
  }
}

islbm_status check_mesh(const double* xi, int n, const char* name, double* lu) {
  if (!xi) return fail(nullptr, ISLBM_ERR_ARG, std::string(name) + " is NULL");
  if (n < 4) return fail(nullptr, ISLBM_ERR_ARG, std::string(name) + ": need at least 4 nodes");
  for (int j = 0; j <= n; ++j)
    if (!(xi[j + 1] > xi[j]) || !std::isfinite(xi[j + 1]))
      return fail(nullptr, ISLBM_ERR_ARG, std::string(name) + " is not strictly increasing");
  const double lo = xi[1] - xi[0], hi = xi[n + 1] - xi[n];
  if (std::fabs(lo - hi) > 1e-9 * lo)
    return fail(nullptr, ISLBM_ERR_ARG,
                std::string(name) + ": ghost spacing differs at the two ends");
  for (int j = 1; j < n; ++j)
    if (xi[j + 1] - xi[j] < lo * (1.0 - 1e-9))
      return fail(nullptr, ISLBM_ERR_ARG,
                  std::string(name) + ": a fluid spacing is below one lattice unit");
  *lu = lo;
  return ISLBM_OK;
}

// Simple FNV-1a over the configuration, for checkpoints.
unsigned long long fnv(const void* data, size_t n, unsigned long long h) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; ++i) h = (h ^ p[i]) * 1099511628211ull;
  return h;
}

// TMA descriptors of the two population buffers for the pipelined 2-D kernels:
// a 3-D tensor (x over the padded pitch, y, population plane) with a box of
// one staged tile (64 + 2 halo chunks wide, 4R + 2 rows, all 14 planes).
std::string encode_tensor_maps(Solver* s) {
  typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                               const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                               const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                               CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return "cuTensorMapEncodeTiled is not available";
  const int R = (s->variant == KV_TMA_R2S2 || s->variant == KV_TMA_R2S3) ? 2 : 4;
  const int hx = 16 / (int)s->elem;
  const CUtensorMapDataType dt =
      s->precision == ISLBM_FP32
          ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
          : (s->precision == ISLBM_FP16DEV || s->precision == ISLBM_FP16NEQ
                 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
  if (s->dim == 3 && is_zm3d(s->variant)) {
    // z-marching kernels: one descriptor per staging group.  Its base is the
    // group's first plane; the dimensions are (x over the padded pitch, y, z,
    // planes of the group[, the flow / temperature pair 19 planes apart]).
    for (int b = 0; b < 2; ++b)
      for (int g = 0; g < 7; ++g) {
        unsigned bx[5];
        const int rank = step_3d_zm_box((int)s->elem, s->variant, g, bx);
        const bool split = step_3d_zm_split(g) != 0;
        const cuuint64_t dims[5] = {(cuuint64_t)s->pitch, (cuuint64_t)s->n[1], (cuuint64_t)s->n[2],
                                    (cuuint64_t)(split ? 2 : 4), 2};
        const cuuint64_t plane_bytes = (cuuint64_t)s->plane * s->elem;
        // R (rank 4, split): the second "plane" is the temperature rest plane
        const cuuint64_t strides[4] = {(cuuint64_t)s->pitch * s->elem,
                                       (cuuint64_t)s->pitch * s->n[1] * s->elem,
                                       (split && rank == 4) ? 19 * plane_bytes : plane_bytes,
                                       19 * plane_bytes};
        const cuuint32_t box[5] = {bx[0], bx[1], bx[2], bx[3], bx[4]};
        const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
        void* base = static_cast<char*>(s->buf[b]) + (size_t)step_3d_zm_first_plane(g) * plane_bytes;
        CUresult r = reinterpret_cast<EncodeFn>(fn)(
            reinterpret_cast<CUtensorMap*>(s->tmap3[b][g]), dt, (cuuint32_t)rank, base, dims,
            strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
          return "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
      }
    return "";
  }
  if (s->dim == 3) {
    // 4-D view [population][z][y][x] of a buffer; a box holds a tile of two planes
    // with a halo along the axes in the bits of its type (1 x, 2 y, 4 z)
    const cuuint64_t dims[4] = {(cuuint64_t)s->pitch, (cuuint64_t)s->n[1], (cuuint64_t)s->n[2],
                                (cuuint64_t)(s->qf + s->qg)};
    const cuuint64_t strides[3] = {(cuuint64_t)s->pitch * s->elem,
                                   (cuuint64_t)s->pitch * s->n[1] * s->elem,
                                   (cuuint64_t)s->plane * s->elem};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int b = 0; b < 2; ++b)
      for (int type = 0; type < 7; ++type) {
        unsigned b4[4];
        step_3d_tma_box((int)s->elem, type, b4);
        const cuuint32_t box[4] = {b4[0], b4[1], b4[2], b4[3]};
        CUresult r = reinterpret_cast<EncodeFn>(fn)(
            reinterpret_cast<CUtensorMap*>(s->tmap3[b][type]), dt, 4, s->buf[b], dims, strides,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
          return "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
      }
    return "";
  }
  const cuuint64_t dims[3] = {(cuuint64_t)s->pitch, (cuuint64_t)s->n[1], 14};
  const cuuint64_t strides[2] = {(cuuint64_t)s->pitch * s->elem, (cuuint64_t)s->plane * s->elem};
  const cuuint32_t box[3] = {(cuuint32_t)(64 + 2 * hx), (cuuint32_t)(4 * R + 2), 14};
  const cuuint32_t estr[3] = {1, 1, 1};
  for (int b = 0; b < 2; ++b) {
    CUresult r = reinterpret_cast<EncodeFn>(fn)(
        reinterpret_cast<CUtensorMap*>(s->tmap[b]), dt, 3, s->buf[b], dims, strides, box, estr,
        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    // FP16NEQ: the 4 FP32 moment planes after the 14 remainder planes, a box
    // of the tile with one 16-byte chunk (4 columns) of halo on each side
    const cuuint64_t mdims[3] = {(cuuint64_t)s->pitch, (cuuint64_t)s->n[1], 4};
    const cuuint64_t mstrides[2] = {(cuuint64_t)s->pitch * 4, (cuuint64_t)s->plane * 4};
    const cuuint32_t mbox[3] = {64 + 8, (cuuint32_t)(4 * R + 2), 4};
    void* mbase = static_cast<char*>(s->buf[b]) + (size_t)14 * s->plane * s->elem;
    if (s->precision == ISLBM_FP16NEQ) {
      r = reinterpret_cast<EncodeFn>(fn)(
          reinterpret_cast<CUtensorMap*>(s->tmap_m[b]), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, mbase,
          mdims, mstrides, mbox, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS)
        return "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    } else {
      std::memcpy(s->tmap_m[b], s->tmap[b], sizeof(s->tmap_m[b]));
    }
  }
  return "";
}

}  // namespace

namespace {
std::mutex g_alloc_mutex;
islbm::DevAllocator g_alloc;
}  // namespace

islbm::DevAllocator islbm::current_allocator() {
  std::lock_guard<std::mutex> lock(g_alloc_mutex);
  return g_alloc;
}

cudaError_t islbm::dev_alloc(const DevAllocator& a, void** p, size_t bytes,
                             cudaStream_t stream) {
  *p = nullptr;
  if (a.alloc) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    *p = a.alloc(bytes, dev, stream, a.ctx);
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
  }
  return cudaMallocAsync(p, bytes, stream);
}

void islbm::dev_free(const DevAllocator& a, void* p, cudaStream_t stream) {
  if (!p) return;
  if (a.alloc) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (a.release) a.release(p, dev, stream, a.ctx);
    return;
  }
  cudaFreeAsync(p, stream);
}

extern "C" islbm_status islbm_set_allocator(islbm_alloc_fn alloc, islbm_free_fn release,
                                            void* ctx) {
  if ((alloc == nullptr) != (release == nullptr))
    return fail(nullptr, ISLBM_ERR_ARG, "islbm_set_allocator: give both functions or neither");
  std::lock_guard<std::mutex> lock(g_alloc_mutex);
  g_alloc.alloc = alloc;
  g_alloc.release = release;
  g_alloc.ctx = ctx;
  return ISLBM_OK;
}

cudaError_t islbm::launch_setup_once(const void* kernel,
                                     cudaError_t (*setup)(const void*, int*), int* value) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(kernel, dev);
  auto it = done.find(key);
  if (it == done.end()) {
    int v = 1;
    e = setup(kernel, &v);
    if (e != cudaSuccess) return e;
    it = done.emplace(key, v).first;
  }
  if (value) *value = it->second;
  return cudaSuccess;
}

namespace {

// Report (and clear) a timeout recorded by a pipelined kernel.  Synchronises.
islbm_status check_device_flag(Solver* s) {
  int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, s->derr, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "reading the device error flag");
  if (flag) {
    cudaMemsetAsync(s->derr, 0, sizeof(int), s->stream);
    return fail(s, ISLBM_ERR_TIMEOUT, "a bounded wait in the step kernel gave up");
  }
  return ISLBM_OK;
}

islbm_status finish_reductions(Solver* s, islbm_reductions* out) {
  const double* r = s->hresult;
  const Physics& h = s->ph;
  const double L = h.L;
  // the averages divide by the measure of the cavity and of a side wall
  // (L^d and L^(d-1) for the square / cubic cavity)
  double vol = 1.0, area = 1.0;
  for (int a = 0; a < s->dim; ++a) {
    const Axis& A = s->ax[a];
    const double La = A.X[A.n] - A.X[1] + 1.0;
    vol *= La;
    if (a > 0) area *= La;
  }
  const double dT = h.dT;
  islbm_reductions o;
  std::memset(&o, 0, sizeof(o));
  // <Nu> = sqrt(Ra Pr) <u* T*>_V + 1 (Sec. 3, Sec. 4); <Re> = sqrt(Ra/Pr) times
  // the root-mean-square speed (the reading that reproduces Table 2), the
  // volume-averaged speed as Re_mean, and the (u, v) root-mean-square as Re_uv
  const double sra = std::sqrt(h.Ra / h.Pr);
  o.Nu = std::sqrt(h.Ra * h.Pr) * r[RED_UT] / (h.u_f * dT * vol) + 1.0;
  o.Re = sra * std::sqrt(r[RED_U2] / vol) / h.u_f;
  o.Re_uv = sra * std::sqrt(r[RED_UV2] / vol) / h.u_f;
  o.Re_mean = sra * r[RED_SPEED] / (h.u_f * vol);
  o.mass = r[RED_MASS];
  o.ke = 0.5 * r[RED_U2];
  // Nu_hot / Nu_cold = -<dT*/dx*> with dT*/dx* = (L/dT) dT/dX by Eq. (17); the
  // wall-plane sums of T are linear in the node values.
  const double hot = h.hot_cw * h.T_hot * area + h.hot_c1 * r[RED_HOT1] + h.hot_c2 * r[RED_HOT2];
  const double cold =
      h.cold_cw * h.T_cold * area + h.cold_c1 * r[RED_COLD1] + h.cold_c2 * r[RED_COLD2];
  o.Nu_hot = -hot * L / (dT * area);
  o.Nu_cold = -cold * L / (dT * area);
  if (s->dim == 2) {
    const double conv = std::sqrt(h.Ra * h.Pr) * r[RED_MIDCONV] / (h.u_f * dT);
    const double cond = L * (r[RED_MIDTR] - r[RED_MIDTL]) * h.mid_inv_dx / dT;
    o.Nu_middle = (conv - cond) / L;
  } else {
    o.Nu_middle = NAN;
  }
  o.max_speed = r[RED_MAXSPEED] / h.u_f;
  o.nonfinite = r[RED_NONFINITE];
  o.time = s->time;
  *out = o;
  if (o.nonfinite > 0 || !std::isfinite(o.Nu) || !std::isfinite(o.mass))
    return fail(s, ISLBM_ERR_DIVERGED, "non-finite values in the state");
  return ISLBM_OK;
}

}  // namespace

// ============================================================================
// mesh helpers
// ============================================================================

extern "C" islbm_status islbm_mesh_uniform(int n, double* xi) {
  if (n < 4 || !xi) return fail(nullptr, ISLBM_ERR_ARG, "islbm_mesh_uniform: n >= 4 and xi");
  for (int j = 0; j <= n + 1; ++j) xi[j] = (j - 0.5) / n;   // Eq. (14b) + ghost nodes
  make_symmetric(xi, n);
  return ISLBM_OK;
}

extern "C" islbm_status islbm_mesh_erf(int n, double a, double* xi) {
  if (n < 4 || !xi || !(a > 0))
    return fail(nullptr, ISLBM_ERR_ARG, "islbm_mesh_erf: n >= 4, a > 0 and xi");
  const double den = std::erf(0.5 * a);
  for (int j = 0; j <= n + 1; ++j)
    xi[j] = 0.5 * (std::erf(a * (double(j) / (n + 1) - 0.5)) / den + 1.0);
  make_symmetric(xi, n);
  return ISLBM_OK;
}

extern "C" islbm_status islbm_mesh_tanh(int n, double a, double* xi) {
  if (n < 4 || !xi || !(a > 0))
    return fail(nullptr, ISLBM_ERR_ARG, "islbm_mesh_tanh: n >= 4, a > 0 and xi");
  const double den = std::tanh(0.5 * a);
  for (int j = 0; j <= n + 1; ++j)
    xi[j] = 0.5 * (std::tanh(a * (double(j) / (n + 1) - 0.5)) / den + 1.0);
  make_symmetric(xi, n);
  return ISLBM_OK;
}

extern "C" void islbm_default_params(islbm_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->Ma = 0.1;
  p->T_hot = 0.5;
  p->T_cold = -0.5;
  p->stencil = ISLBM_STENCIL_CENTRED;
  p->reference = ISLBM_TREF_COLD;
}

// ============================================================================
// create / destroy
// ============================================================================

extern "C" islbm_status islbm_create(const double* xi_x, int nx, const double* xi_y, int ny,
                                     const double* xi_z, int nz, double Ra, double Pr,
                                     int lattice, int precision, const islbm_params* opt,
                                     void* stream, islbm_t* out) {
  if (!out) return fail(nullptr, ISLBM_ERR_ARG, "islbm_create: out is NULL");
  *out = nullptr;
  if (lattice != ISLBM_D2Q9_D2Q5 && lattice != ISLBM_D3Q19_D3Q7)
    return fail(nullptr, ISLBM_ERR_ARG, "islbm_create: unknown lattice");
  if (precision < ISLBM_FP64 || precision > ISLBM_FP16NEQ)
    return fail(nullptr, ISLBM_ERR_ARG, "islbm_create: unknown precision");
  const int dim = lattice == ISLBM_D2Q9_D2Q5 ? 2 : 3;
  if ((dim == 2) != (xi_z == nullptr))
    return fail(nullptr, ISLBM_ERR_ARG, "islbm_create: xi_z must be NULL exactly for the 2-D lattice");
  if (!(Ra > 0) || !(Pr > 0) || !std::isfinite(Ra) || !std::isfinite(Pr))
    return fail(nullptr, ISLBM_ERR_ARG, "islbm_create: Ra and Pr must be positive");
  islbm_params prm;
  islbm_default_params(&prm);
  if (opt) prm = *opt;
  if (!(prm.Ma > 0)) return fail(nullptr, ISLBM_ERR_ARG, "islbm_create: Ma must be positive");
  if (prm.stencil != ISLBM_STENCIL_CENTRED && prm.stencil != ISLBM_STENCIL_UPWIND)
    return fail(nullptr, ISLBM_ERR_ARG, "islbm_create: unknown stencil");
  if (prm.kernel < 0 || prm.kernel >= KV_COUNT ||
      (dim == 2 && (prm.kernel == KV_TMA_3D || is_zm3d(prm.kernel))))
    return fail(nullptr, ISLBM_ERR_ARG, "islbm_create: unknown kernel variant");
  if (precision == ISLBM_FP16NEQ &&
      (dim != 2 || prm.stencil != ISLBM_STENCIL_CENTRED ||
       (prm.kernel != KV_AUTO && prm.kernel != KV_TMA_R2S2 && prm.kernel != KV_TMA_R2S3)))
    return fail(nullptr, ISLBM_ERR_ARG,
                "islbm_create: FP16NEQ storage needs the 2-D lattice, the centred stencil and "
                "kernel variant 0, 4 or 5");
  const double* xis[3] = {xi_x, xi_y, xi_z};
  const int ns[3] = {nx, ny, dim == 3 ? nz : 1};
  const char* names[3] = {"xi_x", "xi_y", "xi_z"};
  double lu[3] = {0, 0, 0};
  for (int a = 0; a < dim; ++a) {
    islbm_status st = check_mesh(xis[a], ns[a], names[a], &lu[a]);
    if (st != ISLBM_OK) return st;
  }
  for (int a = 1; a < dim; ++a)
    if (std::fabs(lu[a] - lu[0]) > 1e-9 * lu[0])
      return fail(nullptr, ISLBM_ERR_ARG, "islbm_create: axes use different lattice units");

  islbm_solver* s = new (std::nothrow) islbm_solver();
  if (!s) return fail(nullptr, ISLBM_ERR_OOM, "islbm_create: host allocation");
  s->dim = dim;
  s->lattice = lattice;
  s->precision = precision;
  s->stencil = prm.stencil;
  s->stream = static_cast<cudaStream_t>(stream);
  s->qf = dim == 2 ? 9 : 19;
  s->qg = dim == 2 ? 5 : 7;
  s->uniform = true;
  for (int a = 0; a < 3; ++a) s->n[a] = ns[a];
  for (int a = 0; a < dim; ++a) {
    build_axis(s->ax[a], xis[a], ns[a], prm.stencil);
    s->uniform = s->uniform && s->ax[a].uniform;
  }
  s->nodes = (long long)s->n[0] * s->n[1] * s->n[2];

  // ---- physics (Sec. 2.1, Sec. 3, Table 1) ----
  Physics& h = s->ph;
  const Axis& ay = s->ax[1];
  h.Ra = Ra;
  h.Pr = Pr;
  h.Ma = prm.Ma;
  h.L = ay.X[ay.n] - ay.X[1] + 1.0;   // distance between the half-way walls
  h.u_f = prm.Ma / std::sqrt(3.0);
  h.nu = h.u_f * h.L * std::sqrt(Pr / Ra);
  h.alpha = h.u_f * h.L / std::sqrt(Pr * Ra);
  h.gbeta = h.u_f * h.u_f / h.L;
  h.T_hot = prm.T_hot;
  h.T_cold = prm.T_cold;
  if (prm.reference != ISLBM_TREF_MEAN && prm.reference != ISLBM_TREF_COLD) {
    delete s;
    return fail(nullptr, ISLBM_ERR_ARG, "islbm_create: unknown reference temperature");
  }
  h.T0 = prm.reference == ISLBM_TREF_COLD ? prm.T_cold : 0.5 * (prm.T_hot + prm.T_cold);
  h.Ts = 0.5 * (prm.T_hot + prm.T_cold);
  h.dT = (prm.T_hot != prm.T_cold) ? prm.T_hot - prm.T_cold : 1.0;
  h.s_nu = 1.0 / (3.0 * h.nu + 0.5);
  const double magic = 8.0 * (2.0 - h.s_nu) / (8.0 - h.s_nu);
  h.s_e = prm.s_e > 0 ? prm.s_e : h.s_nu;
  h.s_eps = prm.s_eps > 0 ? prm.s_eps : h.s_nu;
  h.s_pi = prm.s_pi > 0 ? prm.s_pi : h.s_nu;
  h.s_q = prm.s_q > 0 ? prm.s_q : magic;
  h.s_m = prm.s_m > 0 ? prm.s_m : magic;
  h.q_j = prm.q_j > 0 ? prm.q_j : 3.0 - std::sqrt(3.0);
  h.q_e = prm.q_e > 0 ? prm.q_e : 1.0;
  h.q_nu = prm.q_nu > 0 ? prm.q_nu : 1.0;
  if (dim == 2) {
    h.a_T = 20.0 * std::sqrt(3.0) * h.alpha - 4.0;
    h.omega = (4.0 + h.a_T) / 10.0;
    if (!(h.a_T > -4.0 && h.a_T <= 1.0)) {
      delete s;
      return fail(nullptr, ISLBM_ERR_ARG, "islbm_create: a_T outside (-4, 1] (diffusivity too large)");
    }
  } else {
    h.a_T = 42.0 * std::sqrt(3.0) * h.alpha - 6.0;
    h.omega = (6.0 + h.a_T) / 21.0;
    if (!(h.a_T > -6.0 && h.a_T <= 1.0)) {
      delete s;
      return fail(nullptr, ISLBM_ERR_ARG, "islbm_create: a_T outside (-6, 1] (diffusivity too large)");
    }
  }
  // Eq. (17) coefficients with Delta = 1 l.u. and q = (X_2 - X_1)/(X_1 - X_0)
  const Axis& ax = s->ax[0];
  const int N = ax.n;
  {
    const double q = (ax.X[2] - ax.X[1]) / (ax.X[1] - ax.X[0]);
    const double den = q * (2 * q + 1);
    h.hot_cw = -4 * q * (q + 1) / den;
    h.hot_c1 = (2 * q + 1) * (2 * q + 1) / den;
    h.hot_c2 = -1.0 / den;
  }
  {
    const double q = (ax.X[N] - ax.X[N - 1]) / (ax.X[N + 1] - ax.X[N]);
    const double den = q * (2 * q + 1);
    h.cold_cw = 4 * q * (q + 1) / den;
    h.cold_c1 = -(2 * q + 1) * (2 * q + 1) / den;
    h.cold_c2 = 1.0 / den;
  }
  if (N % 2 == 0)
    h.mid_inv_dx = 1.0 / (ax.X[N / 2 + 1] - ax.X[N / 2]);
  else
    h.mid_inv_dx = 1.0 / (ax.X[(N + 1) / 2 + 1] - ax.X[(N + 1) / 2 - 1]);

  // ---- device and memory ----
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    delete s;
    return fail(nullptr, ISLBM_ERR_CUDA, "islbm_create: no CUDA device");
  }
  cudaGetDevice(&s->device);
  cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device);
  // step-kernel variant: the pipelined TMA kernel for stretched 2-D meshes in
  // FP32 / 16-bit storage, the direct kernel otherwise
  // (and the 3-D pipelined kernel for stretched 3-D meshes)
  if (prm.kernel != KV_AUTO)
    s->variant = prm.kernel;
  else if (dim == 2 && precision == ISLBM_FP16NEQ)
    s->variant = KV_TMA_R2S2;   // decoded per staged tile: pipelined kernels only
  else if (dim == 2)
    s->variant = (precision != ISLBM_FP64 && !s->uniform)
                     ? (precision == ISLBM_FP32 ? KV_TMA_R2S2 : KV_TMA_R4S2)
                     : KV_DIRECT;
  else
    s->variant = s->uniform ? KV_DIRECT : KV_ZM3D;
  if (precision == ISLBM_FP64 || prm.stencil != ISLBM_STENCIL_CENTRED)
    s->variant = KV_DIRECT;
  if (dim == 3 && s->variant == KV_TMA_3D && !step_3d_tma_fits(s->n[1], s->n[2]))
    s->variant = KV_DIRECT;
  if (dim == 3 && s->variant != KV_TMA_3D && !is_zm3d(s->variant)) s->variant = KV_DIRECT;
  s->elem = precision == ISLBM_FP64 ? 8 : (precision == ISLBM_FP32 ? 4 : 2);
  s->pitch = (s->n[0] + 31) / 32 * 32;
  s->plane = (long long)s->pitch * s->n[1] * s->n[2];
  // FP16NEQ: 14 planes of FP16 remainders, then 4 planes of FP32 moments
  s->state_bytes = precision == ISLBM_FP16NEQ
                       ? (size_t)s->plane * (14 * 2 + 4 * 4)
                       : (size_t)(s->qf + s->qg) * s->plane * s->elem;
  const size_t pop_bytes = s->state_bytes;
  const size_t rsize = precision == ISLBM_FP64 ? 8 : 4;
  size_t tab_bytes = 0;
  for (int a = 0; a < dim; ++a) {
    const int n = s->n[a];
    tab_bytes += 2 * (((size_t)n * 4 + 255) / 256 * 256);
    tab_bytes += 2 * (((size_t)3 * n * rsize + 255) / 256 * 256);
    tab_bytes += ((size_t)n * 8 + 255) / 256 * 256;
    tab_bytes += 2 * (((size_t)n * 16 + 255) / 256 * 256);
  }
  tab_bytes += 256;
  s->red_blocks = 4 * 152;
  auto cleanup = [&](islbm_status st, const std::string& m) {
    islbm_destroy(s);
    return fail(nullptr, st, m);
  };
  cudaError_t e;
  s->mem = current_allocator();
  auto dmalloc = [&](void** p, size_t bytes) { return dev_alloc(s->mem, p, bytes, s->stream); };
  for (int b = 0; b < 2; ++b) {
    e = dmalloc(&s->buf[b], pop_bytes);
    if (e != cudaSuccess) return cleanup(ISLBM_ERR_OOM, "islbm_create: population buffers");
    // pooled allocators hand back memory with old contents: start from zeros
    // so that no step or reduction ever sees values it did not write
    e = cudaMemsetAsync(s->buf[b], 0, pop_bytes, s->stream);
    if (e != cudaSuccess) return cleanup(ISLBM_ERR_CUDA, "islbm_create: population buffers");
  }
  e = dmalloc(&s->dtables, tab_bytes);
  if (e != cudaSuccess) return cleanup(ISLBM_ERR_OOM, "islbm_create: tables");
  e = dmalloc(reinterpret_cast<void**>(&s->dscratch),
              (size_t)s->red_blocks * RED_STRIDE * sizeof(double));
  if (e != cudaSuccess) return cleanup(ISLBM_ERR_OOM, "islbm_create: reduction scratch");
  e = dmalloc(reinterpret_cast<void**>(&s->dresult), RED_STRIDE * sizeof(double));
  if (e != cudaSuccess) return cleanup(ISLBM_ERR_OOM, "islbm_create: reduction result");
  e = cudaMallocHost(&s->hresult, RED_STRIDE * sizeof(double));
  if (e != cudaSuccess) return cleanup(ISLBM_ERR_OOM, "islbm_create: pinned result");
  e = dmalloc(reinterpret_cast<void**>(&s->derr), kDerrInts * sizeof(int));
  if (e != cudaSuccess) return cleanup(ISLBM_ERR_OOM, "islbm_create: error flag");
  e = cudaMemsetAsync(s->derr, 0, kDerrInts * sizeof(int), s->stream);
  if (e != cudaSuccess) return cleanup(ISLBM_ERR_CUDA, "islbm_create: error flag");
  if (s->variant >= KV_TMA_R4S2) {
    const std::string m = encode_tensor_maps(s);
    if (!m.empty()) return cleanup(ISLBM_ERR_CUDA, "islbm_create: " + m);
  }
  // pack the tables on the host and copy once
  std::vector<char> host(tab_bytes, 0);
  size_t off = 0;
  char* dbase = static_cast<char*>(s->dtables);
  for (int a = 0; a < dim; ++a) {
    const Axis& A = s->ax[a];
    const int n = A.n;
    for (int k = 0; k < 2; ++k) {
      off = (off + 255) & ~size_t(255);
      std::memcpy(host.data() + off, A.base[k].data(), (size_t)n * 4);
      s->dax[a].base[k] = reinterpret_cast<const int*>(dbase + off);
      off += (size_t)n * 4;
      off = (off + 255) & ~size_t(255);
      for (int i = 0; i < 3 * n; ++i) {
        if (rsize == 8) {
          double v = A.w[k][i];
          std::memcpy(host.data() + off + (size_t)i * 8, &v, 8);
        } else {
          float v = (float)A.w[k][i];
          std::memcpy(host.data() + off + (size_t)i * 4, &v, 4);
        }
      }
      s->dax[a].w[k] = dbase + off;
      off += (size_t)3 * n * rsize;
    }
    off = (off + 255) & ~size_t(255);
    std::memcpy(host.data() + off, A.W.data(), (size_t)n * 8);
    s->dax[a].W = reinterpret_cast<const double*>(dbase + off);
    off += (size_t)n * 8;
    // packed FP32 tables of the tiled kernels: wall entries get zero weights
    // and a stencil base inside the axis
    for (int k = 0; k < 2; ++k) {
      off = (off + 255) & ~size_t(255);
      for (int j = 0; j < n; ++j) {
        int b = A.base[k][j];
        float w4[4] = {(float)A.w[k][3 * j], (float)A.w[k][3 * j + 1], (float)A.w[k][3 * j + 2], 0.f};
        if (b < 0) {
          b = std::min(std::max(j - 1, 0), n - 3);
          w4[0] = w4[1] = w4[2] = 0.f;
        }
        std::memcpy(&w4[3], &b, 4);
        std::memcpy(host.data() + off + (size_t)j * 16, w4, 16);
      }
      s->dax[a].packed[k] = reinterpret_cast<const float4*>(dbase + off);
      off += (size_t)n * 16;
    }
  }
  e = cudaMemcpyAsync(s->dtables, host.data(), tab_bytes, cudaMemcpyHostToDevice, s->stream);
  if (e != cudaSuccess) return cleanup(ISLBM_ERR_CUDA, "islbm_create: table upload");
  e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cleanup(ISLBM_ERR_CUDA, "islbm_create: table upload");

  // configuration fingerprint for checkpoints
  unsigned long long fp = 1469598103934665603ull;
  int cfg[6] = {dim, lattice, precision, s->n[0], s->n[1], s->n[2]};
  fp = fnv(cfg, sizeof(cfg), fp);
  double phys[4] = {Ra, Pr, prm.Ma, h.L};
  fp = fnv(phys, sizeof(phys), fp);
  for (int a = 0; a < dim; ++a) fp = fnv(s->ax[a].X.data(), s->ax[a].X.size() * 8, fp);
  s->fingerprint = fp;

  // rest state rho = 1, u = 0, T = T0: all deviations vanish
  for (int b = 0; b < 2; ++b) {
    e = cudaMemsetAsync(s->buf[b], 0, pop_bytes, s->stream);
    if (e != cudaSuccess) return cleanup(ISLBM_ERR_CUDA, "islbm_create: memset");
  }
  *out = s;
  return ISLBM_OK;
}

extern "C" void islbm_destroy(islbm_t s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  for (int b = 0; b < 2; ++b)
    if (s->graph[b]) cudaGraphExecDestroy(s->graph[b]);
  if (s->side) {
    cudaStreamSynchronize(s->side);
    cudaStreamDestroy(s->side);
  }
  if (s->ev_in) cudaEventDestroy(s->ev_in);
  if (s->ev_out) cudaEventDestroy(s->ev_out);
  for (int b = 0; b < 2; ++b) dev_free(s->mem, s->buf[b], s->stream);
  dev_free(s->mem, s->dtables, s->stream);
  dev_free(s->mem, s->dscratch, s->stream);
  dev_free(s->mem, s->dresult, s->stream);
  dev_free(s->mem, s->dfield, s->stream);
  dev_free(s->mem, s->derr, s->stream);
  dev_free(s->mem, s->dsnap, s->stream);
  dev_free(s->mem, s->davg, s->stream);
  cudaStreamSynchronize(s->stream);   // the frees are stream-ordered
  if (s->hresult) cudaFreeHost(s->hresult);
  delete s;
}

extern "C" const char* islbm_last_error(islbm_t s) {
  return s ? s->err.c_str() : g_last_error;
}

namespace islbm {
void set_last_error_static(const char* msg) { copy_last_error(msg); }
}  // namespace islbm

extern "C" islbm_status islbm_info(islbm_t s, islbm_info_t* o) {
  if (!s || !o) return fail(s, ISLBM_ERR_ARG, "islbm_info: NULL argument");
  std::memset(o, 0, sizeof(*o));
  o->dim = s->dim;
  for (int a = 0; a < 3; ++a) o->n[a] = s->n[a];
  o->q_flow = s->qf;
  o->q_temp = s->qg;
  o->uniform = s->uniform ? 1 : 0;
  o->precision = s->precision;
  const Physics& h = s->ph;
  o->L = h.L;
  o->u_f = h.u_f;
  o->nu = h.nu;
  o->alpha = h.alpha;
  o->gbeta = h.gbeta;
  o->s_nu = h.s_nu;
  o->a_T = h.a_T;
  o->omega = h.omega;
  o->steps_per_tf = h.L / h.u_f;
  o->bytes_per_update = 2.0 * (double)s->state_bytes / (double)s->plane;
  o->time = s->time;
  o->kernel = s->variant;
  o->sm_count = s->sm_count;
  return ISLBM_OK;
}

// ============================================================================
// state in / out
// ============================================================================

static islbm_status ensure_field_buffer(Solver* s) {
  if (s->dfield) return ISLBM_OK;
  const size_t q = (size_t)(s->qf + s->qg);
  const size_t need = std::max<size_t>(5, q) * (size_t)s->nodes * sizeof(double);
  cudaError_t e = dev_alloc(s->mem, reinterpret_cast<void**>(&s->dfield), need, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "field staging buffer");
  return ISLBM_OK;
}

extern "C" islbm_status islbm_set_fields_device(islbm_t s, const double* rho, const double* T,
                                                const double* u, const double* v,
                                                const double* w) {
  if (!s) return fail(nullptr, ISLBM_ERR_ARG, "islbm_set_fields: NULL handle");
  if (!T) return fail(s, ISLBM_ERR_ARG, "islbm_set_fields: T is required");
  if (s->dim == 2 && w) return fail(s, ISLBM_ERR_ARG, "islbm_set_fields: w must be NULL in 2-D");
  CK(s, launch_init_fields(*s, rho, T, u, v, w));
  s->time = 0;
  s->snap_valid = false;
  return ISLBM_OK;
}

extern "C" islbm_status islbm_set_fields(islbm_t s, const double* rho, const double* T,
                                         const double* u, const double* v, const double* w) {
  if (!s) return fail(nullptr, ISLBM_ERR_ARG, "islbm_set_fields: NULL handle");
  if (!T) return fail(s, ISLBM_ERR_ARG, "islbm_set_fields: T is required");
  if (s->dim == 2 && w) return fail(s, ISLBM_ERR_ARG, "islbm_set_fields: w must be NULL in 2-D");
  islbm_status st = ensure_field_buffer(s);
  if (st != ISLBM_OK) return st;
  const size_t n = (size_t)s->nodes;
  const double* src[5] = {rho, T, u, v, w};
  double* dst[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  for (int k = 0; k < 5; ++k) {
    if (!src[k]) continue;
    dst[k] = s->dfield + k * n;
    CK(s, cudaMemcpyAsync(dst[k], src[k], n * sizeof(double), cudaMemcpyHostToDevice, s->stream));
  }
  CK(s, launch_init_fields(*s, dst[0], dst[1], dst[2], dst[3], dst[4]));
  CK(s, cudaStreamSynchronize(s->stream));
  s->time = 0;
  s->snap_valid = false;
  return ISLBM_OK;
}

extern "C" islbm_status islbm_set_populations(islbm_t s, const double* f, const double* g) {
  if (!s || !f || !g) return fail(s, ISLBM_ERR_ARG, "islbm_set_populations: NULL argument");
  islbm_status st = ensure_field_buffer(s);
  if (st != ISLBM_OK) return st;
  const size_t n = (size_t)s->nodes;
  double* df = s->dfield;
  double* dg = s->dfield + (size_t)s->qf * n;
  CK(s, cudaMemcpyAsync(df, f, (size_t)s->qf * n * 8, cudaMemcpyHostToDevice, s->stream));
  CK(s, cudaMemcpyAsync(dg, g, (size_t)s->qg * n * 8, cudaMemcpyHostToDevice, s->stream));
  CK(s, launch_init_populations(*s, df, dg));
  CK(s, cudaStreamSynchronize(s->stream));
  s->time = 0;
  s->snap_valid = false;
  return ISLBM_OK;
}

// Capture kGraphSteps consecutive steps starting from buffer `parity` into a
// graph on the private stream.
static cudaError_t build_graph(Solver* s, int parity) {
  cudaError_t e;
  if (!s->side) {
    e = cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    e = cudaEventCreateWithFlags(&s->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  const cudaStream_t user = s->stream;
  const int cur = s->cur;
  const long long t0 = s->time;
  s->stream = s->side;
  s->cur = parity;
  e = cudaStreamBeginCapture(s->side, cudaStreamCaptureModeThreadLocal);
  cudaError_t le = cudaSuccess;
  if (e == cudaSuccess) {
    // each captured step gets its own step index (it seeds the stochastic
    // rounding of 16-bit stores; replays repeat the 64 indices)
    for (int k = 0; k < kGraphSteps && le == cudaSuccess; ++k, ++s->time) le = launch_step(*s);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s->side, &g);
    if (e == cudaSuccess && le == cudaSuccess) e = cudaGraphInstantiate(&s->graph[parity], g, 0);
    if (g) cudaGraphDestroy(g);
    if (le != cudaSuccess) e = le;
  }
  s->stream = user;
  s->cur = cur;
  s->time = t0;
  return e;
}

extern "C" islbm_status islbm_step(islbm_t s, long long n) {
  NvtxRange range("islbm_step");
  if (!s) return fail(nullptr, ISLBM_ERR_ARG, "islbm_step: NULL handle");
  if (n < 0) return fail(s, ISLBM_ERR_ARG, "islbm_step: negative step count");
  // whole blocks of kGraphSteps steps are replayed from a captured graph
  while (s->use_graphs && n >= kGraphSteps) {
    if (!s->graph[s->cur]) {
      const cudaError_t e = build_graph(s, s->cur);
      if (e != cudaSuccess) {   // fall back to plain launches for this handle
        s->use_graphs = false;
        cudaGetLastError();
        break;
      }
    }
    CK(s, cudaEventRecord(s->ev_in, s->stream));
    CK(s, cudaStreamWaitEvent(s->side, s->ev_in, 0));
    {
      NvtxRange replay("islbm_graph_replay");
      CK(s, cudaGraphLaunch(s->graph[s->cur], s->side));
    }
    CK(s, cudaEventRecord(s->ev_out, s->side));
    CK(s, cudaStreamWaitEvent(s->stream, s->ev_out, 0));
    n -= kGraphSteps;
    s->time += kGraphSteps;
  }
  for (long long k = 0; k < n; ++k) {
    CK(s, launch_step(*s));
    ++s->time;
  }
  return ISLBM_OK;
}

extern "C" islbm_status islbm_get_fields_device(islbm_t s, double* rho, double* T, double* u,
                                                double* v, double* w) {
  if (!s) return fail(nullptr, ISLBM_ERR_ARG, "islbm_get_fields: NULL handle");
  if (s->dim == 2 && w) return fail(s, ISLBM_ERR_ARG, "islbm_get_fields: w must be NULL in 2-D");
  CK(s, launch_fields(*s, rho, T, u, v, w));
  return ISLBM_OK;
}

extern "C" islbm_status islbm_get_fields(islbm_t s, double* rho, double* T, double* u,
                                         double* v, double* w) {
  if (!s) return fail(nullptr, ISLBM_ERR_ARG, "islbm_get_fields: NULL handle");
  if (s->dim == 2 && w) return fail(s, ISLBM_ERR_ARG, "islbm_get_fields: w must be NULL in 2-D");
  islbm_status st = ensure_field_buffer(s);
  if (st != ISLBM_OK) return st;
  const size_t n = (size_t)s->nodes;
  double* dst[5] = {rho, T, u, v, w};
  double* dev[5];
  for (int k = 0; k < 5; ++k) dev[k] = dst[k] ? s->dfield + k * n : nullptr;
  CK(s, launch_fields(*s, dev[0], dev[1], dev[2], dev[3], dev[4]));
  for (int k = 0; k < 5; ++k)
    if (dst[k])
      CK(s, cudaMemcpyAsync(dst[k], dev[k], n * 8, cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  return ISLBM_OK;
}

// ---- time averages (FP64 accumulators on the device) ----

namespace {
__global__ void k_accumulate(double* __restrict__ acc, const double* __restrict__ src,
                             long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    acc[i] += src[i];
}
__global__ void k_scale(double* __restrict__ dst, const double* __restrict__ src, double c,
                        long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = c * src[i];
}
int elementwise_grid(long long n) { return (int)std::min<long long>((n + 255) / 256, 4096); }
}  // namespace

extern "C" islbm_status islbm_average_reset(islbm_t s) {
  if (!s) return fail(nullptr, ISLBM_ERR_ARG, "islbm_average_reset: NULL handle");
  const size_t bytes = (size_t)(s->dim + 1) * (size_t)s->nodes * sizeof(double);
  if (!s->davg) {
    cudaError_t e = dev_alloc(s->mem, reinterpret_cast<void**>(&s->davg), bytes, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "time-average accumulators");
  }
  CK(s, cudaMemsetAsync(s->davg, 0, bytes, s->stream));
  s->avg_count = 0;
  return ISLBM_OK;
}

extern "C" islbm_status islbm_average_add(islbm_t s) {
  if (!s) return fail(nullptr, ISLBM_ERR_ARG, "islbm_average_add: NULL handle");
  if (!s->davg) {
    const islbm_status st = islbm_average_reset(s);
    if (st != ISLBM_OK) return st;
  }
  islbm_status st = ensure_field_buffer(s);
  if (st != ISLBM_OK) return st;
  const size_t n = (size_t)s->nodes;
  // dfield holds [rho][T][u][v][w]; T, u, v (, w) are contiguous from dfield + n
  double* f = s->dfield;
  CK(s, launch_fields(*s, nullptr, f + n, f + 2 * n, f + 3 * n, s->dim == 3 ? f + 4 * n : nullptr));
  const long long m = (long long)(s->dim + 1) * (long long)n;
  k_accumulate<<<elementwise_grid(m), 256, 0, s->stream>>>(s->davg, f + n, m);
  CK(s, cudaGetLastError());
  ++s->avg_count;
  return ISLBM_OK;
}

extern "C" islbm_status islbm_average_get(islbm_t s, double* T, double* u, double* v, double* w,
                                          long long* count) {
  if (!s) return fail(nullptr, ISLBM_ERR_ARG, "islbm_average_get: NULL handle");
  if (s->dim == 2 && w) return fail(s, ISLBM_ERR_ARG, "islbm_average_get: w must be NULL in 2-D");
  if (count) *count = s->avg_count;
  if (s->avg_count <= 0) return fail(s, ISLBM_ERR_ARG, "islbm_average_get: nothing accumulated");
  islbm_status st = ensure_field_buffer(s);
  if (st != ISLBM_OK) return st;
  const size_t n = (size_t)s->nodes;
  const long long m = (long long)(s->dim + 1) * (long long)n;
  k_scale<<<elementwise_grid(m), 256, 0, s->stream>>>(s->dfield, s->davg, 1.0 / (double)s->avg_count, m);
  CK(s, cudaGetLastError());
  double* dst[4] = {T, u, v, w};
  for (int k = 0; k < s->dim + 1; ++k)
    if (dst[k])
      CK(s, cudaMemcpyAsync(dst[k], s->dfield + k * n, n * 8, cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  return ISLBM_OK;
}

extern "C" islbm_status islbm_get_populations(islbm_t s, double* f, double* g) {
  if (!s || !f || !g) return fail(s, ISLBM_ERR_ARG, "islbm_get_populations: NULL argument");
  islbm_status st = ensure_field_buffer(s);
  if (st != ISLBM_OK) return st;
  const size_t n = (size_t)s->nodes;
  double* df = s->dfield;
  double* dg = s->dfield + (size_t)s->qf * n;
  CK(s, launch_populations(*s, df, dg));
  CK(s, cudaMemcpyAsync(f, df, (size_t)s->qf * n * 8, cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaMemcpyAsync(g, dg, (size_t)s->qg * n * 8, cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  return ISLBM_OK;
}

extern "C" islbm_status islbm_reduce(islbm_t s, islbm_reductions* out) {
  NvtxRange range("islbm_reduce");
  if (!s || !out) return fail(s, ISLBM_ERR_ARG, "islbm_reduce: NULL argument");
  if (s->row_end > 0)
    return fail(s, ISLBM_ERR_ARG,
                "islbm_reduce: the handle steps a slab; combine islbm_reduce_sums over the "
                "slabs and finish them with islbm_finish_sums");
  {
    const islbm_status st = check_device_flag(s);
    if (st != ISLBM_OK) return st;
  }
  CK(s, launch_reduce(*s));
  CK(s, cudaMemcpyAsync(s->hresult, s->dresult, RED_STRIDE * sizeof(double),
                        cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  return finish_reductions(s, out);
}

extern "C" islbm_status islbm_steady_change(islbm_t s, double* du, double* dT) {
  NvtxRange range("islbm_steady_change");
  if (!s || !du || !dT) return fail(s, ISLBM_ERR_ARG, "islbm_steady_change: NULL argument");
  if (!s->dsnap) {
    const size_t n = (size_t)(s->dim + 1) * (size_t)s->nodes * sizeof(double);
    cudaError_t e = dev_alloc(s->mem, reinterpret_cast<void**>(&s->dsnap), n, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "steady-state snapshot");
    s->snap_valid = false;
  }
  {
    const islbm_status st = check_device_flag(s);
    if (st != ISLBM_OK) return st;
  }
  CK(s, launch_steady(*s));
  CK(s, cudaMemcpyAsync(s->hresult, s->dresult, RED_STRIDE * sizeof(double),
                        cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  const double* r = s->hresult;
  if (!s->snap_valid) {
    *du = *dT = INFINITY;
  } else {
    *du = r[1] > 0 ? r[0] / r[1] : (r[0] > 0 ? INFINITY : 0.0);
    *dT = r[3] > 0 ? r[2] / r[3] : (r[2] > 0 ? INFINITY : 0.0);
  }
  s->snap_valid = true;
  if (!std::isfinite(r[0]) || !std::isfinite(r[2]))
    return fail(s, ISLBM_ERR_DIVERGED, "non-finite values in the state");
  return ISLBM_OK;
}

extern "C" islbm_status islbm_run_to_steady(islbm_t s, double tol, long long interval,
                                            long long max_steps, long long* steps_done,
                                            double* du_out, double* dT_out) {
  if (!s) return fail(nullptr, ISLBM_ERR_ARG, "islbm_run_to_steady: NULL handle");
  if (!(tol > 0) || interval <= 0 || max_steps < 0)
    return fail(s, ISLBM_ERR_ARG, "islbm_run_to_steady: tol > 0, interval > 0, max_steps >= 0");
  double du = INFINITY, dT = INFINITY;
  long long done = 0;
  islbm_status st = islbm_steady_change(s, &du, &dT);   // snapshot of the starting state
  while (st == ISLBM_OK && done < max_steps) {
    const long long n = std::min(interval, max_steps - done);
    st = islbm_step(s, n);
    if (st != ISLBM_OK) break;
    done += n;
    st = islbm_steady_change(s, &du, &dT);
    if (st == ISLBM_OK && n == interval && du < tol && dT < tol) break;
  }
  if (steps_done) *steps_done = done;
  if (du_out) *du_out = du;
  if (dT_out) *dT_out = dT;
  if (st != ISLBM_OK) return st;
  if (!(du < tol && dT < tol))
    return fail(s, ISLBM_ERR_NOT_CONVERGED, "islbm_run_to_steady: step budget exhausted");
  return ISLBM_OK;
}

extern "C" islbm_status islbm_nusselt(islbm_t s, islbm_nu* out) {
  if (!out) return fail(s, ISLBM_ERR_ARG, "islbm_nusselt: NULL argument");
  islbm_reductions r;
  islbm_status st = islbm_reduce(s, &r);
  out->vol = r.Nu;
  out->hot = r.Nu_hot;
  out->cold = r.Nu_cold;
  out->middle = r.Nu_middle;
  return st;
}

extern "C" islbm_status islbm_reynolds(islbm_t s, double* re) {
  if (!re) return fail(s, ISLBM_ERR_ARG, "islbm_reynolds: NULL argument");
  islbm_reductions r;
  islbm_status st = islbm_reduce(s, &r);
  *re = r.Re;
  return st;
}

extern "C" islbm_status islbm_mass(islbm_t s, double* m) {
  if (!m) return fail(s, ISLBM_ERR_ARG, "islbm_mass: NULL argument");
  islbm_reductions r;
  islbm_status st = islbm_reduce(s, &r);
  *m = r.mass;
  return st;
}

extern "C" islbm_status islbm_synchronize(islbm_t s) {
  if (!s) return fail(nullptr, ISLBM_ERR_ARG, "islbm_synchronize: NULL handle");
  CK(s, cudaStreamSynchronize(s->stream));
  return check_device_flag(s);
}

// ============================================================================
// checkpoints
// ============================================================================

namespace {
struct CkptHeader {
  char magic[8];
  unsigned long long fingerprint;
  long long time;
  long long bytes;
};
}  // namespace

extern "C" islbm_status islbm_save(islbm_t s, const char* path) {
  if (!s || !path) return fail(s, ISLBM_ERR_ARG, "islbm_save: NULL argument");
  const size_t bytes = s->state_bytes;
  std::vector<char> host(bytes);
  CK(s, cudaMemcpyAsync(host.data(), s->buf[s->cur], bytes, cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return fail(s, ISLBM_ERR_IO, std::string("islbm_save: cannot open ") + path);
  CkptHeader hd;
  std::memcpy(hd.magic, "ISLBMCK1", 8);
  hd.fingerprint = s->fingerprint;
  hd.time = s->time;
  hd.bytes = (long long)bytes;
  bool ok = std::fwrite(&hd, sizeof(hd), 1, fp) == 1 && std::fwrite(host.data(), 1, bytes, fp) == bytes;
  ok = (std::fclose(fp) == 0) && ok;
  if (!ok) return fail(s, ISLBM_ERR_IO, std::string("islbm_save: short write to ") + path);
  return ISLBM_OK;
}

extern "C" islbm_status islbm_load(islbm_t s, const char* path) {
  if (!s || !path) return fail(s, ISLBM_ERR_ARG, "islbm_load: NULL argument");
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return fail(s, ISLBM_ERR_IO, std::string("islbm_load: cannot open ") + path);
  CkptHeader hd;
  const size_t bytes = s->state_bytes;
  if (std::fread(&hd, sizeof(hd), 1, fp) != 1 || std::memcmp(hd.magic, "ISLBMCK1", 8) != 0) {
    std::fclose(fp);
    return fail(s, ISLBM_ERR_IO, "islbm_load: not a checkpoint");
  }
  if (hd.fingerprint != s->fingerprint || hd.bytes != (long long)bytes) {
    std::fclose(fp);
    return fail(s, ISLBM_ERR_IO, "islbm_load: checkpoint of another configuration");
  }
  std::vector<char> host(bytes);
  const bool ok = std::fread(host.data(), 1, bytes, fp) == bytes;
  std::fclose(fp);
  if (!ok) return fail(s, ISLBM_ERR_IO, "islbm_load: truncated checkpoint");
  CK(s, cudaMemcpyAsync(s->buf[s->cur], host.data(), bytes, cudaMemcpyHostToDevice, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  s->time = hd.time;
  s->snap_valid = false;
  return ISLBM_OK;
}

extern "C" islbm_status islbm_debug_bounds(int reset, int* flagged) {
  if (!flagged) return fail(nullptr, ISLBM_ERR_ARG, "islbm_debug_bounds: NULL argument");
  const int a = bounds_flag_d2(reset), b = bounds_flag_d3(reset), c = bounds_flag_zm(reset);
  if (a < 0 || b < 0 || c < 0)
    return fail(nullptr, ISLBM_ERR_CUDA, "islbm_debug_bounds: reading the flags");
  *flagged = (a | b | c) ? 1 : 0;
  return ISLBM_OK;
}

// ============================================================================
// 2-D slab decomposition: row range, halo rows, partial sums
// ============================================================================

static_assert(RED_MAXSPEED == ISLBM_SUM_MAX_SLOT && RED_STRIDE == ISLBM_REDUCTION_SUMS,
              "the C ABI's description of the partial sums matches the reduction slots");

static void drop_graphs(Solver* s) {
  if (s->side) cudaStreamSynchronize(s->side);
  for (int b = 0; b < 2; ++b)
    if (s->graph[b]) {
      cudaGraphExecDestroy(s->graph[b]);
      s->graph[b] = nullptr;
    }
}

extern "C" islbm_status islbm_set_row_range(islbm_t s, int row_begin, int row_end) {
  if (!s) return fail(nullptr, ISLBM_ERR_ARG, "islbm_set_row_range: NULL handle");
  if (s->dim != 2) return fail(s, ISLBM_ERR_ARG, "islbm_set_row_range: 2-D cavities only");
  if (s->precision == ISLBM_FP16NEQ)
    return fail(s, ISLBM_ERR_ARG, "islbm_set_row_range: not for FP16NEQ storage");
  if (row_begin < 0 || row_end > s->n[1] || row_begin >= row_end)
    return fail(s, ISLBM_ERR_ARG, "islbm_set_row_range: need 0 <= row_begin < row_end <= n_y");
  drop_graphs(s);   // captured steps carry the old range
  if (row_begin == 0 && row_end == s->n[1]) {
    s->row_begin = s->row_end = 0;
  } else {
    s->row_begin = row_begin;
    s->row_end = row_end;
  }
  return ISLBM_OK;
}

static islbm_status rows_args(Solver* s, int row0, int nrows, const void* p, const char* name) {
  if (!s) return fail(nullptr, ISLBM_ERR_ARG, std::string(name) + ": NULL handle");
  if (s->dim != 2) return fail(s, ISLBM_ERR_ARG, std::string(name) + ": 2-D cavities only");
  if (s->precision == ISLBM_FP16NEQ)
    return fail(s, ISLBM_ERR_ARG, std::string(name) + ": not for FP16NEQ storage");
  if (!p) return fail(s, ISLBM_ERR_ARG, std::string(name) + ": NULL buffer");
  if (row0 < 0 || nrows <= 0 || row0 + nrows > s->n[1])
    return fail(s, ISLBM_ERR_ARG, std::string(name) + ": rows outside the mesh");
  return ISLBM_OK;
}

extern "C" islbm_status islbm_get_rows(islbm_t s, int row0, int nrows, void* dst) {
  const islbm_status st = rows_args(s, row0, nrows, dst, "islbm_get_rows");
  if (st != ISLBM_OK) return st;
  const size_t width = (size_t)nrows * s->pitch * s->elem;
  const char* src = static_cast<const char*>(s->buf[s->cur]) + (size_t)row0 * s->pitch * s->elem;
  CK(s, cudaMemcpy2DAsync(dst, width, src, (size_t)s->plane * s->elem, width, s->qf + s->qg,
                          cudaMemcpyDefault, s->stream));
  return ISLBM_OK;
}

extern "C" islbm_status islbm_set_rows(islbm_t s, int row0, int nrows, const void* src) {
  const islbm_status st = rows_args(s, row0, nrows, src, "islbm_set_rows");
  if (st != ISLBM_OK) return st;
  const size_t width = (size_t)nrows * s->pitch * s->elem;
  char* dst = static_cast<char*>(s->buf[s->cur]) + (size_t)row0 * s->pitch * s->elem;
  CK(s, cudaMemcpy2DAsync(dst, (size_t)s->plane * s->elem, src, width, width, s->qf + s->qg,
                          cudaMemcpyDefault, s->stream));
  s->snap_valid = false;
  return ISLBM_OK;
}

extern "C" islbm_status islbm_reduce_sums(islbm_t s, double* sums) {
  NvtxRange range("islbm_reduce_sums");
  if (!s || !sums) return fail(s, ISLBM_ERR_ARG, "islbm_reduce_sums: NULL argument");
  {
    const islbm_status st = check_device_flag(s);
    if (st != ISLBM_OK) return st;
  }
  CK(s, launch_reduce(*s));
  CK(s, cudaMemcpyAsync(s->hresult, s->dresult, RED_STRIDE * sizeof(double),
                        cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  std::memcpy(sums, s->hresult, RED_STRIDE * sizeof(double));
  return ISLBM_OK;
}

extern "C" islbm_status islbm_finish_sums(islbm_t s, const double* sums, islbm_reductions* out) {
  if (!s || !sums || !out) return fail(s, ISLBM_ERR_ARG, "islbm_finish_sums: NULL argument");
  std::memcpy(s->hresult, sums, RED_STRIDE * sizeof(double));
  return finish_reductions(s, out);
}
