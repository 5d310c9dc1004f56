// Internal declarations of the GB300 ISLBM library (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <string>
#include <vector>

#include "../../include/islbm.h"

namespace islbm {

// Debug builds (ISLBM_BOUNDS_CHECK, build(debug=True)) check every staged
// shared-memory index of the pipelined kernels: an index outside its window
// raises the translation unit's bounds flag (read by islbm_debug_bounds) and
// reads element 0 instead; nothing traps.  Release builds compile the check
// away.
#ifdef __CUDACC__
#ifdef ISLBM_BOUNDS_CHECK
static __device__ int g_bounds_flag = 0;
__device__ __forceinline__ bool in_window(int v, int n) {
  if ((unsigned)v < (unsigned)n) return true;
  atomicOr(&g_bounds_flag, 1);
  return false;
}
#define ISLBM_IN_WINDOW(v, n) ::islbm::in_window((v), (n))
#else
#define ISLBM_IN_WINDOW(v, n) true
#endif
#endif
// bounds flags of the kernel translation units (always 0 in release builds);
// reset != 0 clears them
int bounds_flag_d2(int reset);
int bounds_flag_d3(int reset);
int bounds_flag_zm(int reset);

// Device memory of the library: through the allocator registered with
// islbm_set_allocator, else cudaMallocAsync / cudaFreeAsync on the stream of
// the owner.  An owner records the allocator its memory came from (a later
// registration does not change how that memory is freed).
struct DevAllocator {
  islbm_alloc_fn alloc = nullptr;
  islbm_free_fn release = nullptr;
  void* ctx = nullptr;
};
DevAllocator current_allocator();
cudaError_t dev_alloc(const DevAllocator& a, void** p, size_t bytes, cudaStream_t stream);
void dev_free(const DevAllocator& a, void* p, cudaStream_t stream);

// One-time launch setup of a kernel (shared-memory attribute, occupancy query),
// run once per (kernel, current device) under a lock; *value receives what the
// setup stored (e.g. CTAs per SM).
cudaError_t launch_setup_once(const void* kernel, cudaError_t (*setup)(const void*, int*),
                              int* value);

// NVTX range for profilers (nsys / ncu ranges); a no-op when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Reduction accumulator slots (FP64).  The finished vector is copied to the host.
enum RedSlot {
  RED_MASS = 0,   // sum rho W
  RED_UT,         // sum u (T - T0) W
  RED_SPEED,      // sum |u| W
  RED_UV2,        // sum (u^2 + v^2) W
  RED_U2,         // sum |u|^2 W
  RED_HOT1,       // sum T W_perp on the first fluid plane next to the hot wall
  RED_HOT2,       // ... on the second plane
  RED_COLD1,      // sum T W_perp on the last fluid plane (cold wall)
  RED_COLD2,      // ... on the one before it
  RED_MIDCONV,    // sum u (T - T0) W_y on the centre line (2-D; halved per column for even n)
  RED_MIDTL,      // sum T W_y on the column left of the centre (2-D)
  RED_MIDTR,      // sum T W_y on the column right of the centre (2-D)
  RED_NONFINITE,  // count of non-finite nodes
  RED_MAXSPEED,   // max |u| (max-reduced)
  RED_COUNT
};

constexpr int RED_STRIDE = 16;   // doubles per block partial (>= RED_COUNT)

// Step-kernel variants of the FP32/16-bit paths (islbm_params.kernel).
enum KernelVariant {
  KV_AUTO = 0,      // chosen by the library (islbm_create)
  KV_DIRECT = 1,    // one thread per node, interpolation from global memory
  KV_TILED = 2,     // cp.async staging of a 64 x 16 tile, one tile per CTA
  KV_TMA_R4S2 = 3,  // persistent, TMA double buffer, 64 x 16 tiles
  KV_TMA_R2S2 = 4,  // persistent, TMA double buffer, 64 x 8 tiles
  KV_TMA_R2S3 = 5,  // persistent, TMA triple buffer, 64 x 8 tiles
  KV_TMA_R4S3 = 6,  // persistent, TMA triple buffer, 64 x 16 tiles
  KV_TMA_3D = 7,    // 3-D: persistent, warp-specialised TMA ring of population pairs
  KV_ZM3D = 8,      // 3-D: z-marching columns of 32 x 8 nodes, TMA rings of levels
  KV_ZM3D_T4 = 9,   // 3-D: z-marching columns of 32 x 4 nodes
  KV_COUNT
};

// Per-axis tables, built once on the host in FP64.
struct Axis {
  int n = 0;
  std::vector<double> X;       // lattice coordinates of ghost + fluid nodes (n + 2)
  std::vector<double> W;       // midpoint-rule widths of the fluid nodes (n)
  std::vector<int> base[2];    // [0]: c = +1, [1]: c = -1; first stencil node (0-based), -1 at a wall
  std::vector<double> w[2];    // 3 Lagrange weights per fluid node
  bool uniform = false;
};

// Device view of one axis.  Weights are stored in the compute type.
struct DevAxis {
  const int* base[2];
  const void* w[2];
  const double* W;
  const float4* packed[2];  // FP32 (w0, w1, w2, base as int bits); walls: zero weights
};

// Lattice-unit physics of a handle.
struct Physics {
  double Ra, Pr, Ma, L, u_f, nu, alpha, gbeta, dT;
  double s_nu, s_e, s_eps, s_q, s_pi, s_m;
  double q_j, q_e, q_nu, a_T, omega;
  double T_hot, T_cold, T0;   // T0: reference of the buoyancy force and of T*
  double Ts;                  // storage offset of the temperature populations (mean wall T)
  // wall-derivative coefficients (Eq. (17)): dT/dX = cw*T_w + c1*T_1 + c2*T_2
  double hot_cw, hot_c1, hot_c2, cold_cw, cold_c1, cold_c2;
  double mid_inv_dx;  // 1/(X_{m+1}-X_m) (even n) or 1/(X_{m+1}-X_{m-1}) (odd n)
};

constexpr int kDerrInts = 4;

struct Solver {
  int dim = 2, lattice = 0, precision = 1, stencil = 0;
  int n[3] = {1, 1, 1};
  int qf = 9, qg = 5;
  bool uniform = false;
  cudaStream_t stream = nullptr;
  int device = 0;
  size_t elem = 4;          // bytes per stored population value (FP16NEQ: per remainder)
  size_t state_bytes = 0;   // bytes of one state buffer
  int pitch = 0;            // x pitch in elements
  long long plane = 0;      // elements per population plane
  long long nodes = 0;
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;              // buffer holding the current (post-collision) state
  long long time = 0;
  Physics ph{};
  Axis ax[3];
  void* dtables = nullptr;
  DevAxis dax[3]{};
  double* dscratch = nullptr;     // reduction partials [blocks][RED_COUNT]
  int red_blocks = 0;
  double* dresult = nullptr;      // finished reduction vector
  double* hresult = nullptr;      // pinned host copy
  double* dfield = nullptr;       // staging for field upload / download (5 * nodes)
  double* dsnap = nullptr;        // steady-state snapshot (u, v[, w], T*), allocated on first use
  double* davg = nullptr;         // time-average accumulators (T, u, v[, w]), FP64
  long long avg_count = 0;        // states accumulated since the last reset
  bool snap_valid = false;
  std::string err;
  DevAllocator mem;               // where this handle's device memory comes from
  unsigned long long fingerprint = 0;
  int variant = KV_DIRECT;        // step kernel of the 2-D FP32/16-bit path
  // 2-D slab of a domain decomposition: steps and reductions cover rows
  // [row_begin, row_end) only (row_end == 0: every row)
  int row_begin = 0, row_end = 0;
  int sm_count = 0;
  // device words of the pipelined kernels: [0] error flag, [1] tiles claimed,
  // [2] CTAs finished (the 2-D TMA kernel's dynamic schedule; zero between launches)
  int* derr = nullptr;
  alignas(128) unsigned char tmap[2][128];   // TMA descriptors of buf[0] / buf[1]
  alignas(128) unsigned char tmap_m[2][128]; // FP16NEQ: of their moment planes
  alignas(128) unsigned char tmap3[2][7][128];   // 3-D: one descriptor per box shape
  // CUDA graphs of kGraphSteps steps, one per starting buffer, replayed on a
  // private stream that is ordered against `stream` with events
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  cudaStream_t side = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  bool use_graphs = true;
};

constexpr int kGraphSteps = 64;   // even: a replay leaves the buffer parity unchanged

// ---- kernel launchers (islbm_d2.cu / islbm_d3.cu) ----
// Equilibrium initialisation followed by a collision; fields are device arrays
// (rho may be null -> 1; u[2] null in 2-D).  Writes buf[cur].
cudaError_t launch_init_fields(Solver& s, const double* rho, const double* T, const double* u0,
                               const double* u1, const double* u2);
// Collide full FP64 populations (device, [q][node]) and store them into buf[cur].
cudaError_t launch_init_populations(Solver& s, const double* f, const double* g);
// One fused step: buf[cur] -> buf[cur ^ 1].
cudaError_t launch_step(Solver& s);
// Macroscopic fields of the current state into device arrays (any may be null).
cudaError_t launch_fields(Solver& s, double* rho, double* T, double* u0, double* u1, double* u2);
// Full FP64 post-collision populations of the current state, [q][node] device arrays.
cudaError_t launch_populations(Solver& s, double* f, double* g);
// Reductions of the current state into s.dresult (RED_COUNT doubles).
cudaError_t launch_reduce(Solver& s);

cudaError_t launch_init_fields_3d(Solver& s, const double* rho, const double* T,
                                  const double* u0, const double* u1, const double* u2);
cudaError_t launch_init_populations_3d(Solver& s, const double* f, const double* g);
cudaError_t launch_step_3d(Solver& s);
cudaError_t launch_step_3d_tma(Solver& s);
// TMA box (x, y, z, planes) of the 3-D pipelined kernel for a pair moving along
// the axes in the bits of `type` (1 x, 2 y, 4 z)
void step_3d_tma_box(int elem, int type, unsigned (&box)[4]);
// whether the 3-D pipelined kernel's staged window fits the mesh
bool step_3d_tma_fits(int ny, int nz);
// z-marching 3-D kernels (KV_ZM3D, KV_ZM3D_T4)
cudaError_t launch_step_3d_zm(Solver& s);
// TMA box of staging group g (0..6) of a z-marching variant; returns the rank
// of its descriptor (4 or 5)
int step_3d_zm_box(int elem, int variant, int g, unsigned (&box)[5]);
// first plane of staging group g, and whether the group is two plane pairs
// 19 planes apart (flow and temperature) rather than consecutive planes
int step_3d_zm_first_plane(int g);
int step_3d_zm_split(int g);
inline bool is_zm3d(int variant) { return variant == KV_ZM3D || variant == KV_ZM3D_T4; }
cudaError_t launch_fields_3d(Solver& s, double* rho, double* T, double* u0, double* u1,
                             double* u2);
cudaError_t launch_populations_3d(Solver& s, double* f, double* g);
cudaError_t launch_reduce_3d(Solver& s);

// Deterministic final sum of the per-block partials (islbm_d2.cu).
cudaError_t launch_finish_reduce(Solver& s);
// Steady-state sums against the snapshot (which is then refreshed); slots 0..3 of dresult.
cudaError_t launch_steady(Solver& s);
cudaError_t launch_steady_3d(Solver& s);

}  // namespace islbm

namespace islbm {
// tcgen05 GEMM of the warm-start network (islbm_cnn_tc.cu)
bool cnn_gemm_tc_supported(const void* A, const void* B, int M, int N, int K, int lda, int ldb);
cudaError_t launch_cnn_gemm_tc(const void* A, const void* B, float* C, const float* bias, int M,
                               int N, int K, int lda, int ldb, int ldc, int transA, int transB,
                               int accumulate, cudaStream_t stream, int sms);
// the tcgen05 GEMM's timeout flag (-1: not readable); reset != 0 clears it
int cnn_tc_timeout_flag(int reset);
// split-K partial tiles of the network GEMMs: a per-device workspace grown on
// demand, and the fixed-order sum of the partials into C
cudaError_t cnn_splitk_workspace(size_t bytes, float** out);
cudaError_t launch_splitk_sum(const float* partial, int split, int M, int N, float* C, int ldc,
                              const float* bias, int accumulate, cudaStream_t stream);

// One launch configuration of the batched step: the cavities sharing a tile
// height, with their device-side parameter records and work list.
struct BatchGroup {
  virtual ~BatchGroup() {}
  virtual cudaError_t launch(cudaStream_t stream, int parity, unsigned step, int* err) = 0;
};
cudaError_t make_batch_group(const std::vector<Solver*>& members, int tile_rows, int precision,
                             int sm_count, cudaStream_t stream, BatchGroup** out);
}  // namespace islbm

// The opaque handle of the C ABI is the solver itself.
struct islbm_solver : public islbm::Solver {};
