/*
 * islbm.h -- C ABI of the GB300 interpolation-supplemented lattice Boltzmann
 * solver for side-heated cavity convection.
 *
 * Method: Xu, Zhao, Xu & Jiang, "Interpolation-supplemented lattice Boltzmann
 * simulation of thermal convection on non-uniform meshes", Int. J. Heat Mass
 * Transfer (2025).  Section references below are to that paper.
 *
 * Conventions shared by every entry point
 *   - Every call returns an islbm_status; ISLBM_OK is 0.  On failure the
 *     message is available from islbm_last_error(handle) (or
 *     islbm_last_error(NULL) when there is no handle yet).
 *   - Grids are stored x fastest: node (x, y[, z]) of a field lives at
 *     index x + nx*(y + ny*z).  Population arrays are [q][z][y][x].
 *   - "Host" pointers are caller-owned host memory, read or written before the
 *     call returns.  "Device" pointers are caller-owned CUDA device memory on
 *     the device of the handle; the call enqueues work on the handle's stream
 *     and returns without waiting.
 *   - The library owns the device memory of a handle (two population buffers,
 *     the interpolation tables and a small reduction scratch area), allocated
 *     in islbm_create and freed in islbm_destroy.
 *   - Calls on one handle are not thread-safe; different handles are
 *     independent.
 *   - There is no CPU fallback: without a CUDA device islbm_create returns
 *     ISLBM_ERR_CUDA.
 *   - Temperatures are given in the units of the wall temperatures
 *     (islbm_params.T_hot = +1/2, T_cold = -1/2 by default, so dT = 1); the
 *     paper's T* = (T - T0)/dT uses the reference T0 of islbm_params.reference
 *     (default: the cold wall, so T* = T + 1/2 lies in [0, 1]).  Velocities
 *     are in lattice units (l.u. per time step); u* = u / u_f with u_f from
 *     islbm_info.
 */
#ifndef ISLBM_H
#define ISLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define ISLBM_API __attribute__((visibility("default")))
#else
#define ISLBM_API
#endif

typedef struct islbm_solver* islbm_t;

typedef enum {
  ISLBM_OK = 0,
  ISLBM_ERR_ARG = 1,           /* invalid argument; nothing was changed            */
  ISLBM_ERR_CUDA = 2,          /* CUDA error, or no usable GPU                     */
  ISLBM_ERR_OOM = 3,           /* device allocation failed                         */
  ISLBM_ERR_DIVERGED = 4,      /* a reduction found a non-finite value             */
  ISLBM_ERR_NOT_CONVERGED = 5, /* steady state not reached within the step budget  */
  ISLBM_ERR_TIMEOUT = 6,       /* a bounded device wait gave up                    */
  ISLBM_ERR_IO = 7             /* checkpoint file missing, short or mismatched     */
} islbm_status;

/* Lattice pair (Sec. 2.1): D2Q9 flow + D2Q5 temperature, or D3Q19 + D3Q7. */
typedef enum { ISLBM_D2Q9_D2Q5 = 0, ISLBM_D3Q19_D3Q7 = 1 } islbm_lattice;

/* Storage type of the populations.  Collision and interpolation run in FP64
 * for ISLBM_FP64 and in FP32 otherwise.  All forms store the deviation from
 * the rest state, f_i - w_i (flow) and g_i (temperature, T0 = 0); FP16DEV and
 * BF16DEV store those deviations in 16 bits (stochastically rounded).
 * ISLBM_FP16NEQ (2-D only, the centred stencil, kernel variants 4 and 5 of
 * islbm_params.kernel; ISLBM_ERR_ARG otherwise, and for the slab calls) splits each node's deviations into its moments (drho, jx, jy, T) in
 * FP32 and, per population, the remainder beyond the equilibrium of those
 * moments in FP16 (scaled by 2^12, rounded to nearest): 44 bytes a node
 * against 56 (FP32) and 28 (FP16DEV), with the remainder, which carries the
 * stress and heat flux, resolved to about 1e-8 instead of 1e-5. */
typedef enum {
  ISLBM_FP64 = 0,
  ISLBM_FP32 = 1,
  ISLBM_FP16DEV = 2,
  ISLBM_BF16DEV = 3,
  ISLBM_FP16NEQ = 4
} islbm_precision;

/* Interpolation stencil of the virtual streaming (Sec. 2.2): three nodes
 * centred on the target node (moved inwards at the walls), or shifted one node
 * upwind of the streaming direction. */
typedef enum { ISLBM_STENCIL_CENTRED = 0, ISLBM_STENCIL_UPWIND = 1 } islbm_stencil;

/* Optional parameters.  Fill with islbm_default_params and override.  A rate
 * <= 0 selects the default:
 *   s_e = s_eps = s_pi = s_nu, s_q = s_m = 8(2 - s_nu)/(8 - s_nu),
 *   q_j = 3 - sqrt(3) (implied by the a_T formulas of Sec. 2.1), q_e = q_nu = 1. */
typedef struct {
  double Ma;          /* Mach number of the free-fall velocity, Sec. 3 (0.1)    */
  double T_hot;       /* wall temperatures in T* units (+0.5, -0.5)             */
  double T_cold;
  double s_e, s_eps, s_q, s_pi, s_m;   /* flow MRT rates (Sec. 2.1)            */
  double q_j, q_e, q_nu;               /* temperature MRT rates (Sec. 2.1)     */
  int stencil;        /* islbm_stencil                                          */
  int kernel;         /* step-kernel variant of the FP32/16-bit paths: 0 = chosen
                         by the library; 1 direct (one thread per node); 2-D:
                         2 tiled (cp.async tile staging); 3-6 persistent TMA
                         pipelines (64x16 / 64x8 tiles, 2 / 3 stages: 3 = 16
                         rows 2 stages, 4 = 8 rows 2 stages, 5 = 8 rows 3
                         stages, 6 = 16 rows 3 stages); 3-D: 7 persistent TMA
                         ring of opposite-population pairs (32x4x2 tiles, needs
                         n_y >= 6, n_z >= 4); 8 / 9 z-marching columns of
                         32x8 / 32x4 nodes with TMA rings of z levels.  2-6 in
                         3-D and every variant for FP64 or the upwind stencil
                         run the direct kernel; 7-9 in 2-D are ISLBM_ERR_ARG. */
  int reference;      /* reference temperature T0 of the buoyancy force and of T*
                         (Sec. 2.1): ISLBM_TREF_COLD = the cold wall (default;
                         reproduces the asymmetric centre values of Table 3),
                         ISLBM_TREF_MEAN = mean of the wall temperatures          */
  int reserved[5];
} islbm_params;

/* Choices of the reference temperature T0 (islbm_params.reference). */
enum { ISLBM_TREF_MEAN = 0, ISLBM_TREF_COLD = 1 };

/* Derived lattice-unit parameters of a handle. */
typedef struct {
  int dim;            /* 2 or 3                                                 */
  int n[3];           /* fluid nodes per axis (n[2] = 1 in 2-D)                 */
  int q_flow, q_temp; /* 9/5 or 19/7                                            */
  int uniform;        /* 1 if every axis is the uniform mesh (pure shift)       */
  int precision;      /* islbm_precision                                        */
  double L;           /* cavity height in l.u. (Table 1)                        */
  double u_f;         /* free-fall velocity Ma/sqrt(3) in l.u./step (Sec. 3)    */
  double nu, alpha;   /* viscosity and diffusivity in lattice units            */
  double gbeta;       /* g beta in lattice units, dT = 1                        */
  double s_nu, a_T, omega;
  double steps_per_tf;   /* time steps per free-fall time, L/u_f (Sec. 3)       */
  double bytes_per_update; /* algorithmic HBM bytes of one node update          */
  long long time;     /* steps taken since the last set_* call                  */
  int kernel;         /* step-kernel variant in use (see islbm_params.kernel)    */
  int sm_count;       /* streaming multiprocessors of the device                */
} islbm_info_t;

/* Reductions of the current state (Sec. 3 and Sec. 4), accumulated in FP64. */
typedef struct {
  double Nu;          /* <Nu> = sqrt(Ra Pr) <u* T*>_V + 1                        */
  double Nu_hot;      /* minus the wall average of dT/dx (starred units), hot wall, Eq. (17) */
  double Nu_cold;     /* the same on the cold wall, Eq. (17)                      */
  double Nu_middle;   /* line average of sqrt(Ra Pr) u T - dT/dx (starred units) at x = 1/2 (2-D; NaN in 3-D) */
  double Re;          /* <Re> = sqrt(Ra/Pr) sqrt(<|u*|^2>_V): root-mean-square speed,
                         the form that reproduces the Re of Table 2              */
  double Re_uv;       /* same with u*^2 + v*^2 only (the printed 3-D components) */
  double Re_mean;     /* sqrt(Ra/Pr) <|u*|>_V, the volume-averaged speed         */
  double mass;        /* sum rho W (l.u.^d)                                      */
  double ke;          /* 1/2 sum |u|^2 W                                         */
  double max_speed;   /* max |u| / u_f                                           */
  double nonfinite;   /* number of nodes with a non-finite rho, u or T           */
  long long time;
} islbm_reductions;

/* ---- mesh helpers (Sec. 2.3) ------------------------------------------------
 * Fill xi[0 .. n+1] (host, caller-owned, n+2 doubles) with a mesh in
 * ghost-node form: xi[1..n] are the fluid nodes, xi[0] and xi[n+1] lie one
 * lattice unit beyond the first and last fluid node, so the half-way walls sit
 * at (xi[0]+xi[1])/2 and (xi[n]+xi[n+1])/2.
 *   uniform: xi_j = (j - 0.5)/n (Eq. (14b)); ghosts at -0.5/n and 1 + 0.5/n.
 *   erf:     xi_j = (erf[a(j/(n+1) - 1/2)]/erf(a/2) + 1)/2 (Sec. 2.3).
 *   tanh:    the same form with tanh in place of erf.
 * Requires n >= 4 and a > 0.  The result is exactly symmetric. */
ISLBM_API islbm_status islbm_mesh_uniform(int n, double* xi);
ISLBM_API islbm_status islbm_mesh_erf(int n, double a, double* xi);
ISLBM_API islbm_status islbm_mesh_tanh(int n, double a, double* xi);

/* Fill *p with the defaults listed at islbm_params. */
ISLBM_API void islbm_default_params(islbm_params* p);

/* Create a cavity solver (Sec. 2.1-2.3, Sec. 3).
 *   xi_x, xi_y, xi_z: host meshes in ghost-node form of nx+2, ny+2, nz+2
 *     doubles (copied).  xi_z = NULL for the 2-D lattice.  All axes must share
 *     the lattice unit xi[1]-xi[0] (to 1e-9 relative), have equal ghost
 *     spacing at both ends, and increase strictly.  A mesh whose spacings are
 *     all one lattice unit is streamed by a pure shift.
 *   Ra, Pr > 0; lattice: islbm_lattice; precision: islbm_precision.
 *   opt: NULL for the defaults.
 *   stream: cudaStream_t to enqueue all work on (NULL = the legacy stream).
 * The cavity height L (Table 1) sets nu = u_f L sqrt(Pr/Ra),
 * alpha = u_f L / sqrt(Pr Ra), g beta = u_f^2 / L.  Fails with ISLBM_ERR_ARG
 * if 1/s_nu <= 1/2 or a_T lies outside its admissible range
 * (-4 < a_T <= 1 for D2Q5, -6 < a_T <= 1 for D3Q7).
 * The new solver holds the rest state rho = 1, u = 0, T = 0.  *out receives
 * the handle (caller owns it; release with islbm_destroy). */
ISLBM_API islbm_status islbm_create(const double* xi_x, int nx, const double* xi_y, int ny,
                                    const double* xi_z, int nz, double Ra, double Pr,
                                    int lattice, int precision, const islbm_params* opt,
                                    void* stream, islbm_t* out);

/* Release every resource of the handle (synchronises its stream).  NULL is a no-op. */
ISLBM_API void islbm_destroy(islbm_t h);

/* Last error message of the handle, or of the calling thread when h is NULL. */
ISLBM_API const char* islbm_last_error(islbm_t h);

/* Derived parameters of the handle (host struct, filled on return). */
ISLBM_API islbm_status islbm_info(islbm_t h, islbm_info_t* out);

/* Equilibrium initialisation (Sec. 2.1): f = f^eq(rho, u), g = g^eq(T, u),
 * followed by the local collision.  Host arrays of n_x*n_y[*n_z] doubles; rho
 * may be NULL (rho = 1), w must be NULL in 2-D.  Resets the step counter. */
ISLBM_API islbm_status islbm_set_fields(islbm_t h, const double* rho, const double* T,
                                        const double* u, const double* v, const double* w);

/* As islbm_set_fields with device pointers (asynchronous on the handle's stream). */
ISLBM_API islbm_status islbm_set_fields_device(islbm_t h, const double* rho, const double* T,
                                               const double* u, const double* v,
                                               const double* w);

/* Initialise from full pre-collision populations: host arrays f[q_flow][z][y][x]
 * and g[q_temp][z][y][x] in FP64, in the velocity order of the paper's
 * lattices as listed in the library's documentation.  The temperature
 * populations carry T - T_s, T_s the mean of the wall temperatures (zero for
 * the default walls).  The library collides them and stores the result.
 * Resets the step counter. */
ISLBM_API islbm_status islbm_set_populations(islbm_t h, const double* f, const double* g);

/* Advance n >= 0 ISLBM time steps (Sec. 2.2): virtual streaming with
 * quadratic interpolation and wall conditions (Sec. 2.3) followed by the
 * local MRT collisions (Sec. 2.1), one fused kernel per step.  Asynchronous:
 * returns after enqueueing. */
ISLBM_API islbm_status islbm_step(islbm_t h, long long n);

/* Macroscopic fields of the current time step (Sec. 2.1): rho, T*, u, v[, w],
 * each n_x*n_y[*n_z] doubles in host memory.  Any pointer may be NULL; w must
 * be NULL in 2-D.  Synchronises the stream. */
ISLBM_API islbm_status islbm_get_fields(islbm_t h, double* rho, double* T, double* u,
                                        double* v, double* w);

/* As islbm_get_fields into device buffers (asynchronous). */
ISLBM_API islbm_status islbm_get_fields_device(islbm_t h, double* rho, double* T, double* u,
                                               double* v, double* w);

/* The stored state: full post-collision populations f+ and g+ of the current
 * time step (FP64 host arrays, layout as islbm_set_populations).  Synchronises. */
ISLBM_API islbm_status islbm_get_populations(islbm_t h, double* f, double* g);

/* Nu, Re, mass and kinetic energy of the current time step (Sec. 3 / Sec. 4),
 * weighted with the midpoint rule of Eq. (18).  Synchronises.  Returns
 * ISLBM_ERR_DIVERGED (with *out filled) if any node is non-finite. */
ISLBM_API islbm_status islbm_reduce(islbm_t h, islbm_reductions* out);

/* Steady-state criterion of Sec. 3: *du = sum_i |u(t) - u(t')|_2 / sum_i |u(t')|_2
 * and *dT = sum_i |T*(t) - T*(t')| / sum_i |T*(t')|, with t' the time of the
 * previous call (the paper compares states 2000 steps apart).  The first call
 * after creation or a set_* / load only records the state and returns +inf.
 * Allocates a snapshot of (d+1) doubles per node on first use.  Synchronises. */
ISLBM_API islbm_status islbm_steady_change(islbm_t h, double* du, double* dT);

/* Advance in blocks of `interval` steps until both steady-state changes of
 * islbm_steady_change fall below `tol` (the paper uses 1e-9 with interval 2000,
 * Sec. 3), or `max_steps` have been taken (then ISLBM_ERR_NOT_CONVERGED).
 * steps_done / du / dT (host, may be NULL) receive the steps taken and the last
 * changes.  Synchronises after every block. */
ISLBM_API islbm_status islbm_run_to_steady(islbm_t h, double tol, long long interval,
                                           long long max_steps, long long* steps_done,
                                           double* du, double* dT);

/* Time averages of the fields in FP64 device accumulators (for flows that keep
 * oscillating; not in the paper, whose runs are steady).  islbm_average_reset
 * zeroes them (allocating (d+1) doubles per node on first use);
 * islbm_average_add adds the current T, u, v (, w) (asynchronous);
 * islbm_average_get writes the means to host arrays of n_x*n_y[*n_z] doubles
 * (any may be NULL; w must be NULL in 2-D), *count (may be NULL) receives the
 * number of states averaged; ISLBM_ERR_ARG when nothing was accumulated.
 * Synchronises.  set_* and load leave the accumulators untouched. */
ISLBM_API islbm_status islbm_average_reset(islbm_t h);
ISLBM_API islbm_status islbm_average_add(islbm_t h);
ISLBM_API islbm_status islbm_average_get(islbm_t h, double* T, double* u, double* v, double* w,
                                         long long* count);

/* Convenience views of islbm_reduce. */
typedef struct { double vol, hot, cold, middle; } islbm_nu;
ISLBM_API islbm_status islbm_nusselt(islbm_t h, islbm_nu* out);
ISLBM_API islbm_status islbm_reynolds(islbm_t h, double* re);
ISLBM_API islbm_status islbm_mass(islbm_t h, double* m);

/* Wait for all work enqueued on the handle. */
ISLBM_API islbm_status islbm_synchronize(islbm_t h);

/* Checkpoint: write / read the stored populations, the step counter and a
 * fingerprint of the mesh and parameters.  islbm_load fails with ISLBM_ERR_IO
 * if the file is short or was written by a handle with another configuration. */
ISLBM_API islbm_status islbm_save(islbm_t h, const char* path);
ISLBM_API islbm_status islbm_load(islbm_t h, const char* path);

/* ---- batched cavities (a sweep of independent problems) ----------------------
 * A batch advances many 2-D cavities of different sizes and Rayleigh numbers
 * together: one persistent kernel launch per step (per tile height) walks a
 * work list of (cavity, tile) items over all of them, and blocks of steps are
 * replayed from CUDA graphs.  Each cavity is an ordinary solver handle owned
 * by the batch (islbm_batch_member): set its fields, read its fields and
 * reductions through the single-cavity entry points, but advance it only with
 * islbm_batch_step. */
typedef enum { ISLBM_MESH_UNIFORM = 0, ISLBM_MESH_ERF = 1, ISLBM_MESH_TANH = 2 } islbm_mesh_kind;
typedef struct {
  int n;          /* fluid nodes per axis (square cavity)           */
  int mesh;       /* islbm_mesh_kind                                 */
  double a;       /* stretching parameter (erf / tanh)               */
  double Ra, Pr;
} islbm_cavity;
typedef struct islbm_batch* islbm_batch_t;

/* Time the 2-D step-kernel variants (islbm_params.kernel 1..6) of one square mesh
 * with CUDA events on `stream` (30 steps after 5 warm-up steps each) and
 * return the fastest in *best; us_per_step (host, may be NULL) receives
 * ISLBM_KERNEL_VARIANTS entries (+inf for variants that cannot run).  Results
 * are cached per (n, mesh, a, precision) for the life of the process.
 * FP32 / FP16DEV / BF16DEV / FP16NEQ (which runs variants 4 and 5 only). */
#define ISLBM_KERNEL_VARIANTS 10
ISLBM_API islbm_status islbm_autotune(int n, int mesh, double a, int precision, void* stream,
                                      int* best, double* us_per_step);

/* Create a batch of `count` cavities (host array, copied) with one storage
 * precision (FP32 / FP16DEV / BF16DEV / FP16NEQ).  opt: common parameters
 * (NULL = defaults).  autotune != 0 chooses each mesh size's tile height with
 * islbm_autotune (FP16NEQ: always 8 rows); otherwise 8-row tiles.  stream:
 * shared by all members. */
ISLBM_API islbm_status islbm_batch_create(int count, const islbm_cavity* cavities, int precision,
                                          const islbm_params* opt, int autotune, void* stream,
                                          islbm_batch_t* out);
ISLBM_API void islbm_batch_destroy(islbm_batch_t b);
/* The solver handle of cavity i (owned by the batch). */
ISLBM_API islbm_status islbm_batch_member(islbm_batch_t b, int i, islbm_t* out);
/* Tile height (rows) used for cavity i: 8 or 16 (0 for a bad index). */
ISLBM_API int islbm_batch_tile_rows(islbm_batch_t b, int i);
/* Advance every cavity by n steps (asynchronous). */
ISLBM_API islbm_status islbm_batch_step(islbm_batch_t b, long long n);
/* Wait for the batch; reports a timeout of a bounded wait as ISLBM_ERR_TIMEOUT. */
ISLBM_API islbm_status islbm_batch_synchronize(islbm_batch_t b);
/* Step in blocks of `interval` until every cavity meets the steady criterion of
 * Sec. 3 (islbm_steady_change below tol) or max_steps have been taken;
 * steps_to_steady (host, count entries, may be NULL) receives each cavity's
 * step count at which it first met it (-1: not reached).  A cavity that has
 * met the criterion is taken out of the work list (its state is kept and no
 * further steps are spent on it); all cavities are advanced again when the
 * call returns. */
ISLBM_API islbm_status islbm_batch_run_to_steady(islbm_batch_t b, double tol, long long interval,
                                                 long long max_steps, long long* steps_to_steady);

/* Steady-Nu criterion for flows that settle to a statistically steady state
 * (a persistent oscillation on a coarse mesh never meets the field criterion
 * above): every `sample` steps each cavity's volume-averaged Nu and Re
 * (islbm_reduce) are recorded; after every `window` samples their window
 * means are formed, and a cavity is steady at the end of the first window
 * whose mean Nu differs from the previous window's by at most tol * |mean|.
 * steps_to_steady, nu_mean, re_mean (host, count entries each, may be NULL)
 * receive the step count (-1: not reached) and the window means of that
 * window (of the last window for a cavity that did not converge).  Steps
 * continue in whole samples until every cavity is steady or the next sample
 * would pass max_steps (then ISLBM_ERR_NOT_CONVERGED).  As in
 * islbm_batch_run_to_steady, steady cavities leave the work list until the
 * call returns.  ISLBM_ERR_ARG for
 * tol <= 0, sample <= 0 or window < 2.  Not in the paper, whose runs are
 * converged with the field criterion. */
ISLBM_API islbm_status islbm_batch_run_to_steady_nu(islbm_batch_t b, double tol, long long sample,
                                                    int window, long long max_steps,
                                                    long long* steps_to_steady, double* nu_mean,
                                                    double* re_mean);

/* ---- warm-start network kernels ----------------------------------------------
 * Not part of the paper's method: these kernels train and evaluate a small
 * convolutional network that predicts the steady cavity state from
 * (log Ra, Pr, stretching) so that islbm_set_fields can start the solver near
 * it.  All pointers are device pointers; every call is asynchronous on
 * `stream`, returns ISLBM_ERR_ARG for NULL pointers or bad sizes (nothing
 * launched) and ISLBM_ERR_CUDA if the launch fails.  Tensors are NHWC, FP32
 * unless stated; "bf16" buffers hold __nv_bfloat16. */
/* C[M,N] (+)= op(A) op(B) (+ bias[N]) on the tensor cores, BF16 operands with
 * FP32 accumulation.  transA = 0: A is M x K row-major with leading dimension
 * lda; 1: A is K x M row-major.  transB = 0: B is K x N row-major; 1: N x K.
 * accumulate != 0 adds to C.  A, B: bf16; C, bias: FP32 (bias may be NULL).
 * Path: when lda and ldb are multiples of 8 and A, B are 16-byte aligned, the
 * fifth-generation tensor cores (tcgen05.mma, accumulator in tensor memory;
 * 128 x 16 / 32 / 64 tiles, operands copied by TMA in 64-wide k stages),
 * except when K <= 32; else the warp-level mma.sync kernel.
 * When the output tiles are too few to fill the GPU the K range is split and
 * the splits' partial tiles are added in a fixed order, so results do not
 * depend on scheduling.  The partial tiles live in one split-K workspace per
 * device, allocated through the registered allocator and grown on demand
 * (the device is synchronised while it grows): calls that split K, and
 * islbm_cnn_colsum, must not run concurrently on different streams of one
 * device.  ISLBM_ERR_ARG also for ldc < N or a leading dimension of A or B
 * shorter than its row; ISLBM_ERR_OOM when the workspace cannot grow. */
ISLBM_API islbm_status islbm_cnn_gemm_bf16(const void* A, const void* B, float* C,
                                           const float* bias, int M, int N, int K, int lda,
                                           int ldb, int ldc, int transA, int transB,
                                           int accumulate, void* stream);
/* The same product with the path chosen: 0 as islbm_cnn_gemm_bf16, 1 the
 * mma.sync kernel, 2 the tcgen05 kernel (ISLBM_ERR_ARG when its conditions
 * above do not hold). */
ISLBM_API islbm_status islbm_cnn_gemm_bf16_ex(const void* A, const void* B, float* C,
                                              const float* bias, int M, int N, int K, int lda,
                                              int ldb, int ldc, int transA, int transB,
                                              int accumulate, int path, void* stream);
/* *timed_out = 1 if a bounded mbarrier wait of the tcgen05 GEMM gave up since
 * the last reset (its output tile is then not written); reset != 0 clears the
 * flag.  Reads device memory (synchronous). */
ISLBM_API islbm_status islbm_cnn_check_timeout(int reset, int* timed_out);
/* 3x3 zero-padded im2col of in[B,H,W,C] into bf16 rows col[B*H*W][kpad]
 * ordered [dy][dx][c]; kpad >= 9C, the extra columns are zero. */
ISLBM_API islbm_status islbm_cnn_im2col(const float* in, void* col, int B, int H, int W, int C,
                                        int kpad, void* stream);
/* Adjoint of islbm_cnn_im2col: din[B,H,W,C] from dcol[B*H*W][kpad] (written, not added). */
ISLBM_API islbm_status islbm_cnn_col2im(const float* dcol, float* din, int B, int H, int W,
                                        int C, int kpad, void* stream);
/* Nearest-neighbour 2x upsampling of in[B,H,W,C] into out[B,2H,2W,C]; with
 * backward != 0 the adjoint: in is the gradient [B,2H,2W,C], out [B,H,W,C]. */
ISLBM_API islbm_status islbm_cnn_upsample2x(const float* in, float* out, int B, int H, int W,
                                            int C, int backward, void* stream);
/* x = tanh(x) in place; and dy *= 1 - y^2 (y = tanh output). */
ISLBM_API islbm_status islbm_cnn_tanh(float* x, long long n, void* stream);
ISLBM_API islbm_status islbm_cnn_tanh_back(const float* y, float* dy, long long n, void* stream);
/* FP32 -> bf16 copy of n values. */
ISLBM_API islbm_status islbm_cnn_to_bf16(const float* x, void* y, long long n, void* stream);
/* out[N] (+)= column sums of the M x N row-major x.  Chunks of 2048 rows are
 * summed in the split-K workspace and added in a fixed order (deterministic);
 * ISLBM_ERR_OOM when the workspace cannot grow. */
ISLBM_API islbm_status islbm_cnn_colsum(const float* x, float* out, int M, int N, int accumulate,
                                        void* stream);
/* Weighted mean squared error of y against t (n values, channel weights wc of
 * period C, NULL = 1): dy = 2 wc (y - t) / n, and `blocks` partial sums of
 * wc (y - t)^2 in partial[blocks] (FP64; their sum / n is the loss). */
ISLBM_API islbm_status islbm_cnn_mse(const float* y, const float* t, const float* wc, int C,
                                     float* dy, double* partial, int blocks, long long n,
                                     void* stream);
/* One Adam step (Kingma & Ba) of n FP32 weights w with gradient g and moments
 * m, v at step t >= 1; wb (may be NULL) receives the bf16 copy of w. */
ISLBM_API islbm_status islbm_cnn_adam(float* w, void* wb, const float* g, float* m, float* v,
                                      long long n, float lr, float beta1, float beta2,
                                      float eps, long long t, void* stream);

/* Solver fields <-> network channels for `nodes` nodes (the 2-D node order of
 * islbm_get_fields_device): y[3k..3k+2] = ((T - T_mid) / T_scale,
 * u / u_scale, v / u_scale) with T, u, v FP64 device arrays and y FP32 NHWC;
 * unpack is the inverse.  ISLBM_ERR_ARG for NULL pointers, nodes <= 0 or a
 * zero scale (pack). */
ISLBM_API islbm_status islbm_cnn_pack_fields(const double* T, const double* u, const double* v,
                                             long long nodes, double T_mid, double T_scale,
                                             double u_scale, float* y, void* stream);
ISLBM_API islbm_status islbm_cnn_unpack_fields(const float* y, long long nodes, double T_mid,
                                               double T_scale, double u_scale, double* T,
                                               double* u, double* v, void* stream);

/* Debug builds only (compiled with ISLBM_BOUNDS_CHECK): *flagged = 1 if any
 * staged shared-memory index of the pipelined step kernels fell outside its
 * window since the last reset (the access read element 0 instead; nothing
 * traps).  reset != 0 clears the flags.  Release builds always report 0.
 * The paper has no counterpart: this is a bounds checker for the kernels. */
ISLBM_API islbm_status islbm_debug_bounds(int reset, int* flagged);

/* Self-test of the bounded device waits of the pipelined step kernels (the
 * paper has no counterpart): one CTA waits on an mbarrier that nothing
 * arrives at, gives up after the same limit as the step kernels (one second
 * of the GPU's global timer), raises a device flag and returns.  Returns
 * ISLBM_ERR_TIMEOUT when the flag was raised (the expected outcome),
 * ISLBM_OK if the wait somehow completed, ISLBM_ERR_CUDA / ISLBM_ERR_OOM on a
 * CUDA failure.  Synchronises `stream`; the context stays usable. */
ISLBM_API islbm_status islbm_selftest_wait_timeout(void* stream);

/* Self-test of the CTA abort flag of the barrier-free pipelined loops (the
 * paper has no counterpart): in one CTA, warp 0 waits on an mbarrier that
 * nothing arrives at until the wait limit and then raises the CTA's abort
 * flag; the other warps make three waits on another such mbarrier, each of
 * which gives up at its own limit or as soon as the flag is up.
 * *failed_waits (host) receives the failed waits of warp 1 (3 expected), *ms
 * (host) their total time in milliseconds (about one wait limit, 1000 ms,
 * when the flag ends the second and third waits; three limits without it).
 * Returns ISLBM_ERR_TIMEOUT when warp 0's wait gave up (the expected outcome),
 * ISLBM_ERR_ARG for a null pointer, ISLBM_ERR_CUDA / ISLBM_ERR_OOM on a CUDA
 * failure.  Synchronises `stream`; the context stays usable. */
ISLBM_API islbm_status islbm_selftest_wait_abort(void* stream, int* failed_waits, int* ms);

/* ---- device memory --------------------------------------------------------------
 * Every device allocation of the library (a handle's population buffers,
 * tables, scratch and staging buffers, a batch's work lists, the network
 * GEMM's split-K workspace) goes through the allocator registered here, or,
 * when none is, cudaMallocAsync / cudaFreeAsync on the owner's stream (the
 * handle's or the batch's; the legacy stream for the workspace).  alloc
 * returns a device pointer of at least `bytes` bytes on device `device` for
 * use on `stream` (NULL on failure, which the calling entry point reports as
 * ISLBM_ERR_OOM); release returns one.  A handle keeps the allocator it was
 * created with: registering another later does not change how its memory is
 * freed.  Both functions or neither (NULL, NULL restores the default);
 * ISLBM_ERR_ARG otherwise.  Not a method of the paper: memory plumbing.  The
 * Python binding registers torch's caching allocator when torch has CUDA. */
typedef void* (*islbm_alloc_fn)(size_t bytes, int device, void* stream, void* ctx);
typedef void (*islbm_free_fn)(void* ptr, int device, void* stream, void* ctx);
ISLBM_API islbm_status islbm_set_allocator(islbm_alloc_fn alloc, islbm_free_fn release,
                                           void* ctx);

/* ---- 2-D slab decomposition ---------------------------------------------------
 * The time step of Sec. 2.2 needs, at a node, the post-collision populations
 * of its own row and of the rows next to it (the y stencil of the quadratic
 * interpolation, or the bounce-back partner at a wall).  A cavity split into
 * slabs of rows therefore exchanges one halo row on each side per step.  These
 * calls let one handle per rank (each holding the whole mesh) step only its
 * slab; the ranks move the halo rows between them (a copy, NCCL or any other
 * transport) between steps, and combine the partial sums of the reductions.
 * The paper runs one GPU; the split is this library's.
 *
 * islbm_set_row_range: subsequent islbm_step calls compute rows
 * [row_begin, row_end) of a 2-D cavity only (0 <= row_begin < row_end <= n_y;
 * the whole range restores the default).  Rows outside keep whatever they
 * held; the caller must refresh rows row_begin - 1 and row_end (where they
 * exist) from the ranks that own them before every step.  islbm_reduce then
 * returns ISLBM_ERR_ARG: use islbm_reduce_sums and islbm_finish_sums.
 * ISLBM_ERR_ARG for 3-D handles or an empty or out-of-mesh range. */
ISLBM_API islbm_status islbm_set_row_range(islbm_t h, int row_begin, int row_end);

/* Copy rows [row0, row0 + nrows) of the current (post-collision) state out of
 * / into the handle: all Q_f + Q_g = 14 planes in the storage type (8, 4 or 2
 * bytes a value), laid out [plane][row][x over the padded pitch]:
 * 14 * nrows * pitch * bytes in all (pitch = n_x rounded up to 32, from
 * islbm_info's bytes_per_update and n).  `dst` / `src` may be host or device
 * memory (caller-owned).  Stream-ordered: the call returns after enqueueing the
 * copy on the handle's stream; synchronise that stream before reading a host
 * `dst` or reusing a host `src`.  ISLBM_ERR_ARG for 3-D handles, NULL
 * buffers or rows outside the mesh. */
ISLBM_API islbm_status islbm_get_rows(islbm_t h, int row0, int nrows, void* dst);
ISLBM_API islbm_status islbm_set_rows(islbm_t h, int row0, int nrows, const void* src);

/* The raw FP64 sums behind islbm_reduce over the handle's rows (all rows, or
 * the slab of islbm_set_row_range): ISLBM_REDUCTION_SUMS doubles into the
 * caller's host array `sums` (synchronises the stream).  Sums over disjoint
 * slabs add up to the whole cavity's, except entry ISLBM_SUM_MAX_SLOT, a
 * maximum.  islbm_finish_sums turns combined sums into the finished values of
 * Sec. 3 / Sec. 4, Eq. (17), Eq. (18) (as islbm_reduce; ISLBM_ERR_DIVERGED for
 * non-finite nodes). */
#define ISLBM_REDUCTION_SUMS 16
#define ISLBM_SUM_MAX_SLOT 13
ISLBM_API islbm_status islbm_reduce_sums(islbm_t h, double* sums);
ISLBM_API islbm_status islbm_finish_sums(islbm_t h, const double* sums, islbm_reductions* out);

/* ---- reductions without allocation ------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers of
 * this library that cannot allocate device memory: code that runs while its
 * memory pool is fully reserved, hosts that hand the library only buffers they
 * already own, or loops where an allocation (and the device synchronisation it
 * can cause) is not allowed.  islbm_reduce_noalloc computes the same
 * quantities as islbm_reduce for a 2-D cavity state that lives entirely in the
 * caller's device memory, with no handle, and calls no cudaMalloc, cudaFree or
 * other allocating routine.
 *   f, g: device, full FP64 post-collision populations [9][ny][nx] and
 *     [5][ny][nx] in the velocity order of islbm_set_populations (the layout
 *     islbm_get_populations writes to the host).
 *   nx, ny: fluid nodes per axis, at least 4 each; nx*ny at most 134217728.
 *   xi_x, xi_y: device, the meshes (nx+2 and ny+2 doubles, ghost-node form as
 *     for islbm_create: strictly increasing, one lattice unit xi_1 - xi_0
 *     shared by both axes).  The library cannot see the sizes of f, g, xi_x
 *     and xi_y: they must hold the counts above (the Python binding checks
 *     them before the call).
 *   Ra, Pr, opt (Ma, T_hot, T_cold; NULL = defaults): as for islbm_create.
 *   stream: cudaStream_t for the two kernels (NULL = legacy stream).
 *   out: host struct, filled on return (the call synchronises the stream).
 * Its scratch is one file-scope device array of 1 MiB (per-block partial sums
 * of at most 8192 blocks plus the result), held by every GPU that loads the
 * library until the process exits.  Every value a call reads from it is
 * written earlier in the same call.  Every call looks up the array's device
 * address on the current device (cudaGetSymbolAddress) before it launches.
 * The call synchronises its stream and copies the result to host memory, so
 * it cannot be used inside a stream capture.  All calls share the array:
 * calls that overlap on the GPU (e.g. on two streams) race, so serialise
 * them.  Returns ISLBM_ERR_ARG for NULL pointers or sizes outside the limits
 * above (nothing launched) and for meshes that are not strictly increasing or
 * whose axes differ in lattice unit (found on the device; no result is
 * returned), ISLBM_ERR_DIVERGED if a node is non-finite, ISLBM_ERR_CUDA on a
 * launch failure; the message is available from islbm_last_error(NULL). */
ISLBM_API islbm_status islbm_reduce_noalloc(const double* f, const double* g, int nx, int ny,
                                            const double* xi_x, const double* xi_y, double Ra,
                                            double Pr, const islbm_params* opt, void* stream,
                                            islbm_reductions* out);

#ifdef __cplusplus
}
#endif

#endif /* ISLBM_H */
