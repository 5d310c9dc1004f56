// Batched cavities and the tile-shape autotuner (C ABI: include/islbm.h).
//
// A batch owns one solver per cavity (buffers, tables, TMA descriptors) and
// advances all of them with one persistent kernel launch per tile shape and
// step, walking a work list of (cavity, tile) items; blocks of steps are
// replayed from CUDA graphs.  The autotuner times the step-kernel variants of
// a mesh with CUDA events and remembers the fastest.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "islbm_internal.h"

using namespace islbm;

namespace islbm {
void set_last_error_static(const char* msg);
}

struct islbm_batch {
  std::vector<islbm_t> members;
  std::vector<char> active;              // members still advanced by islbm_batch_step
  std::vector<int> rows;                 // rows per thread (2 or 4) of each member's tiles
  std::vector<BatchGroup*> groups;
  cudaStream_t stream = nullptr;
  int precision = ISLBM_FP32;
  int parity = 0;                        // buffer read by the next step (all members)
  long long time = 0;
  int* derr = nullptr;
  islbm::DevAllocator mem;               // where derr came from
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  cudaStream_t side = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  bool use_graphs = true;
  std::string err;
};

namespace {

islbm_status bfail(islbm_batch* b, islbm_status st, const std::string& m) {
  if (b) b->err = m;
  set_last_error_static(m.c_str());
  return st;
}

std::string member_error(islbm_t m) {
  const char* e = islbm_last_error(m);
  return e ? std::string(e) : std::string();
}

islbm_status make_mesh(int kind, int n, double a, std::vector<double>& xi) {
  xi.resize((size_t)n + 2);
  if (kind == ISLBM_MESH_UNIFORM) return islbm_mesh_uniform(n, xi.data());
  if (kind == ISLBM_MESH_ERF) return islbm_mesh_erf(n, a, xi.data());
  if (kind == ISLBM_MESH_TANH) return islbm_mesh_tanh(n, a, xi.data());
  return ISLBM_ERR_ARG;
}

// one batched step on `st` (all groups), then the members' bookkeeping
cudaError_t batch_launch(islbm_batch* b, cudaStream_t st) {
  for (BatchGroup* g : b->groups) {
    const cudaError_t e = g->launch(st, b->parity, (unsigned)b->time, b->derr);
    if (e != cudaSuccess) return e;
  }
  b->parity ^= 1;
  return cudaSuccess;
}

cudaError_t build_batch_graph(islbm_batch* b, int parity) {
  cudaError_t e;
  if (!b->side) {
    if ((e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming)) != cudaSuccess) return e;
  }
  const int saved = b->parity;
  const long long t0 = b->time;
  b->parity = parity;
  e = cudaStreamBeginCapture(b->side, cudaStreamCaptureModeThreadLocal);
  cudaError_t le = cudaSuccess;
  if (e == cudaSuccess) {
    for (int k = 0; k < kGraphSteps && le == cudaSuccess; ++k, ++b->time) le = batch_launch(b, b->side);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->side, &g);
    if (e == cudaSuccess && le == cudaSuccess) e = cudaGraphInstantiate(&b->graph[parity], g, 0);
    if (g) cudaGraphDestroy(g);
    if (le != cudaSuccess) e = le;
  }
  b->parity = saved;
  b->time = t0;
  return e;
}

void sync_members(islbm_batch* b, long long steps) {
  for (size_t i = 0; i < b->members.size(); ++i)
    if (b->active[i]) {
      b->members[i]->cur = b->parity;
      b->members[i]->time += steps;
    }
}

// (Re)build the work lists of the active members, one group per tile height;
// the captured graphs belong to the old lists and are dropped.
cudaError_t rebuild_groups(islbm_batch* b) {
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return e;
  if (b->side && (e = cudaStreamSynchronize(b->side)) != cudaSuccess) return e;
  for (int k = 0; k < 2; ++k)
    if (b->graph[k]) {
      cudaGraphExecDestroy(b->graph[k]);
      b->graph[k] = nullptr;
    }
  for (BatchGroup* g : b->groups) delete g;
  b->groups.clear();
  for (int rows : {2, 4}) {
    std::vector<Solver*> grp;
    for (size_t i = 0; i < b->members.size(); ++i)
      if (b->active[i] && b->rows[i] == rows) grp.push_back(b->members[i]);
    if (grp.empty()) continue;
    BatchGroup* g = nullptr;
    e = make_batch_group(grp, rows, b->precision, b->members[0]->sm_count, b->stream, &g);
    if (e != cudaSuccess) return e;
    b->groups.push_back(g);
  }
  return cudaSuccess;
}

// Advance every member again: a retired member's state is copied into the
// buffer the batch reads next, so that all members share one parity.
islbm_status reactivate_all(islbm_batch* b) {
  bool changed = false;
  for (size_t i = 0; i < b->members.size(); ++i) {
    if (b->active[i]) continue;
    islbm_t m = b->members[i];
    if (m->cur != b->parity) {
      const size_t bytes = m->state_bytes;
      const cudaError_t e = cudaMemcpyAsync(m->buf[b->parity], m->buf[m->cur], bytes,
                                            cudaMemcpyDeviceToDevice, b->stream);
      if (e != cudaSuccess)
        return bfail(b, ISLBM_ERR_CUDA, std::string("batch reactivate: ") + cudaGetErrorString(e));
      m->cur = b->parity;
    }
    b->active[i] = 1;
    changed = true;
  }
  if (!changed) return ISLBM_OK;
  const cudaError_t e = rebuild_groups(b);
  return e == cudaSuccess ? ISLBM_OK
                          : bfail(b, ISLBM_ERR_CUDA, std::string("batch regroup: ") + cudaGetErrorString(e));
}

// Stop advancing the members flagged in `retire` (a converged cavity keeps its state).
islbm_status retire(islbm_batch* b, const std::vector<char>& retire_now) {
  bool changed = false;
  for (size_t i = 0; i < b->members.size(); ++i)
    if (retire_now[i] && b->active[i]) {
      b->active[i] = 0;
      changed = true;
    }
  if (!changed) return ISLBM_OK;
  const cudaError_t e = rebuild_groups(b);
  return e == cudaSuccess ? ISLBM_OK
                          : bfail(b, ISLBM_ERR_CUDA, std::string("batch regroup: ") + cudaGetErrorString(e));
}

// ---- autotuner ----
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, long long, int>, std::vector<double>> g_tune_cache;

}  // namespace

extern "C" islbm_status islbm_autotune(int n, int mesh, double a, int precision, void* stream,
                                       int* best, double* us_per_step) {
  if (n < 4 || !best || precision < ISLBM_FP32 || precision > ISLBM_FP16NEQ)
    return bfail(nullptr, ISLBM_ERR_ARG, "islbm_autotune: n >= 4, 16/32-bit precision, best");
  const auto key = std::make_tuple(n, mesh, (long long)std::llround(a * 1e6), precision);
  std::vector<double> times;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) times = it->second;
  }
  if (times.empty()) {
    std::vector<double> xi;
    if (make_mesh(mesh, n, a, xi) != ISLBM_OK)
      return bfail(nullptr, ISLBM_ERR_ARG, "islbm_autotune: bad mesh");
    times.assign(KV_COUNT, INFINITY);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
      return bfail(nullptr, ISLBM_ERR_CUDA, "islbm_autotune: events");
    for (int k = KV_DIRECT; k < KV_COUNT; ++k) {
      islbm_params prm;
      islbm_default_params(&prm);
      prm.kernel = k;
      islbm_t h = nullptr;
      if (islbm_create(xi.data(), n, xi.data(), n, nullptr, 0, 1e7, 0.71, ISLBM_D2Q9_D2Q5,
                       precision, &prm, stream, &h) != ISLBM_OK)
        continue;
      h->use_graphs = false;
      const int warm = 5, runs = 30;
      bool ok = islbm_step(h, warm) == ISLBM_OK;
      ok = ok && cudaEventRecord(e0, st) == cudaSuccess;
      ok = ok && islbm_step(h, runs) == ISLBM_OK;
      ok = ok && cudaEventRecord(e1, st) == cudaSuccess;
      ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
      float ms = 0.f;
      if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && islbm_synchronize(h) == ISLBM_OK)
        times[k] = 1e3 * ms / runs;
      islbm_destroy(h);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = times;
  }
  int k_best = KV_DIRECT;
  for (int k = KV_DIRECT; k < KV_COUNT; ++k)
    if (times[k] < times[k_best]) k_best = k;
  *best = k_best;
  if (us_per_step)
    for (int k = 0; k < KV_COUNT; ++k) us_per_step[k] = times[k];
  return std::isfinite(times[k_best])
             ? ISLBM_OK
             : bfail(nullptr, ISLBM_ERR_CUDA, "islbm_autotune: no variant ran");
}

extern "C" islbm_status islbm_batch_create(int count, const islbm_cavity* cav, int precision,
                                           const islbm_params* opt, int autotune, void* stream,
                                           islbm_batch_t* out) {
  if (!out || !cav || count <= 0)
    return bfail(nullptr, ISLBM_ERR_ARG, "islbm_batch_create: count > 0, cavities, out");
  *out = nullptr;
  if (precision < ISLBM_FP32 || precision > ISLBM_FP16NEQ)
    return bfail(nullptr, ISLBM_ERR_ARG, "islbm_batch_create: FP32 or 16-bit storage");
  auto* b = new islbm_batch();
  b->stream = static_cast<cudaStream_t>(stream);
  b->precision = precision;
  islbm_params base;
  islbm_default_params(&base);
  if (opt) base = *opt;
  base.stencil = ISLBM_STENCIL_CENTRED;
  std::map<std::tuple<int, int, long long>, int> rows_of;   // tile height per mesh
  for (int i = 0; i < count; ++i) {
    const islbm_cavity& c = cav[i];
    std::vector<double> xi;
    if (make_mesh(c.mesh, c.n, c.a, xi) != ISLBM_OK) {
      islbm_batch_destroy(b);
      return bfail(nullptr, ISLBM_ERR_ARG, "islbm_batch_create: bad mesh of cavity " + std::to_string(i));
    }
    const auto mk = std::make_tuple(c.n, c.mesh, (long long)std::llround(c.a * 1e6));
    int rows = 2;
    auto it = rows_of.find(mk);
    if (it != rows_of.end()) {
      rows = it->second;
    } else {
      if (autotune) {
        double us[KV_COUNT];
        int bestk = 0;
        if (islbm_autotune(c.n, c.mesh, c.a, precision, stream, &bestk, us) == ISLBM_OK)
          rows = us[KV_TMA_R4S2] < us[KV_TMA_R2S2] ? 4 : 2;
      }
      rows_of[mk] = rows;
    }
    islbm_params prm = base;
    prm.kernel = rows == 4 ? KV_TMA_R4S2 : KV_TMA_R2S2;
    islbm_t h = nullptr;
    const islbm_status st = islbm_create(xi.data(), c.n, xi.data(), c.n, nullptr, 0, c.Ra, c.Pr,
                                         ISLBM_D2Q9_D2Q5, precision, &prm, stream, &h);
    if (st != ISLBM_OK) {
      islbm_batch_destroy(b);
      return bfail(nullptr, st, "islbm_batch_create: cavity " + std::to_string(i) + ": " +
                                    member_error(nullptr));
    }
    b->members.push_back(h);
    b->rows.push_back(rows);
  }
  b->active.assign(b->members.size(), 1);
  b->mem = islbm::current_allocator();
  cudaError_t e = islbm::dev_alloc(b->mem, reinterpret_cast<void**>(&b->derr), sizeof(int),
                                   b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->derr, 0, sizeof(int), b->stream);
  if (e == cudaSuccess) e = rebuild_groups(b);
  if (e != cudaSuccess) {
    islbm_batch_destroy(b);
    return bfail(nullptr, ISLBM_ERR_CUDA, std::string("islbm_batch_create: ") + cudaGetErrorString(e));
  }
  *out = b;
  return ISLBM_OK;
}

extern "C" void islbm_batch_destroy(islbm_batch_t b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (int k = 0; k < 2; ++k)
    if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
  if (b->side) {
    cudaStreamSynchronize(b->side);
    cudaStreamDestroy(b->side);
  }
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  for (BatchGroup* g : b->groups) delete g;
  for (islbm_t m : b->members) islbm_destroy(m);
  islbm::dev_free(b->mem, b->derr, b->stream);
  if (b->stream) cudaStreamSynchronize(b->stream);
  delete b;
}

extern "C" islbm_status islbm_batch_member(islbm_batch_t b, int i, islbm_t* out) {
  if (!b || !out || i < 0 || i >= (int)b->members.size())
    return bfail(b, ISLBM_ERR_ARG, "islbm_batch_member: index out of range");
  *out = b->members[i];
  return ISLBM_OK;
}

extern "C" int islbm_batch_tile_rows(islbm_batch_t b, int i) {
  return (b && i >= 0 && i < (int)b->rows.size()) ? 4 * b->rows[i] : 0;
}

extern "C" islbm_status islbm_batch_step(islbm_batch_t b, long long n) {
  NvtxRange range("islbm_batch_step");
  if (!b || n < 0) return bfail(b, ISLBM_ERR_ARG, "islbm_batch_step: handle, n >= 0");
  if (b->groups.empty()) return ISLBM_OK;   // every member retired
  while (b->use_graphs && n >= kGraphSteps) {
    if (!b->graph[b->parity] && build_batch_graph(b, b->parity) != cudaSuccess) {
      b->use_graphs = false;
      cudaGetLastError();
      break;
    }
    cudaError_t e = cudaEventRecord(b->ev_in, b->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side, b->ev_in, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->graph[b->parity], b->side);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_out, b->side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_out, 0);
    if (e != cudaSuccess)
      return bfail(b, ISLBM_ERR_CUDA, std::string("islbm_batch_step: ") + cudaGetErrorString(e));
    n -= kGraphSteps;
    b->time += kGraphSteps;
    sync_members(b, kGraphSteps);
  }
  for (long long k = 0; k < n; ++k) {
    const cudaError_t e = batch_launch(b, b->stream);
    if (e != cudaSuccess)
      return bfail(b, ISLBM_ERR_CUDA, std::string("islbm_batch_step: ") + cudaGetErrorString(e));
    ++b->time;
    sync_members(b, 1);
  }
  return ISLBM_OK;
}

extern "C" islbm_status islbm_batch_synchronize(islbm_batch_t b) {
  if (!b) return bfail(nullptr, ISLBM_ERR_ARG, "islbm_batch_synchronize: NULL handle");
  int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, b->derr, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess)
    return bfail(b, ISLBM_ERR_CUDA, std::string("islbm_batch_synchronize: ") + cudaGetErrorString(e));
  if (flag) {
    cudaMemsetAsync(b->derr, 0, sizeof(int), b->stream);
    return bfail(b, ISLBM_ERR_TIMEOUT, "a bounded wait in the batched step gave up");
  }
  return ISLBM_OK;
}

extern "C" islbm_status islbm_batch_run_to_steady(islbm_batch_t b, double tol, long long interval,
                                                  long long max_steps, long long* steps_to_steady) {
  if (!b || !(tol > 0) || interval <= 0 || max_steps < 0)
    return bfail(b, ISLBM_ERR_ARG, "islbm_batch_run_to_steady: tol > 0, interval > 0");
  const size_t n = b->members.size();
  std::vector<long long> done(n, -1);
  double du, dT;
  for (size_t i = 0; i < n; ++i) {
    if (!b->active[i]) continue;
    const islbm_status st = islbm_steady_change(b->members[i], &du, &dT);   // snapshots
    if (st != ISLBM_OK) return bfail(b, st, member_error(b->members[i]));
  }
  long long t = 0;
  size_t left = n;
  while (left > 0 && t < max_steps) {
    const long long k = std::min(interval, max_steps - t);
    islbm_status st = islbm_batch_step(b, k);
    if (st == ISLBM_OK) st = islbm_batch_synchronize(b);
    if (st != ISLBM_OK) return st;
    t += k;
    for (size_t i = 0; i < n; ++i) {
      if (!b->active[i]) continue;
      st = islbm_steady_change(b->members[i], &du, &dT);
      if (st != ISLBM_OK) return bfail(b, st, member_error(b->members[i]));
      if (done[i] < 0 && k == interval && du < tol && dT < tol) {
        done[i] = t;
        --left;
      }
    }
    std::vector<char> conv(n, 0);
    for (size_t i = 0; i < n; ++i) conv[i] = done[i] >= 0;
    st = retire(b, conv);
    if (st != ISLBM_OK) return st;
  }
  if (steps_to_steady)
    for (size_t i = 0; i < n; ++i) steps_to_steady[i] = done[i];
  const islbm_status ra = reactivate_all(b);
  if (ra != ISLBM_OK) return ra;
  return left == 0 ? ISLBM_OK
                   : bfail(b, ISLBM_ERR_NOT_CONVERGED, "islbm_batch_run_to_steady: step budget exhausted");
}

extern "C" islbm_status islbm_batch_run_to_steady_nu(islbm_batch_t b, double tol, long long sample,
                                                     int window, long long max_steps,
                                                     long long* steps_to_steady, double* nu_mean,
                                                     double* re_mean) {
  if (!b || !(tol > 0) || sample <= 0 || window < 2 || max_steps < 0)
    return bfail(b, ISLBM_ERR_ARG,
                 "islbm_batch_run_to_steady_nu: tol > 0, sample > 0, window >= 2");
  const size_t n = b->members.size();
  std::vector<long long> done(n, -1);
  std::vector<double> sum_nu(n, 0.0), sum_re(n, 0.0), prev(n, NAN), nu_out(n, NAN), re_out(n, NAN);
  long long t = 0;
  int in_window = 0;
  size_t left = n;
  while (left > 0 && t + sample <= max_steps) {
    islbm_status st = islbm_batch_step(b, sample);
    if (st == ISLBM_OK) st = islbm_batch_synchronize(b);
    if (st != ISLBM_OK) return st;
    t += sample;
    for (size_t i = 0; i < n; ++i) {
      if (!b->active[i]) continue;
      islbm_reductions r;
      st = islbm_reduce(b->members[i], &r);
      if (st != ISLBM_OK) return bfail(b, st, member_error(b->members[i]));
      sum_nu[i] += r.Nu;
      sum_re[i] += r.Re;
    }
    if (++in_window < window) continue;
    in_window = 0;
    for (size_t i = 0; i < n; ++i) {
      const double m = sum_nu[i] / window, mr = sum_re[i] / window;
      sum_nu[i] = sum_re[i] = 0.0;
      if (done[i] < 0) {
        nu_out[i] = m;
        re_out[i] = mr;
        if (std::isfinite(prev[i]) && std::fabs(m - prev[i]) <= tol * std::fabs(m)) {
          done[i] = t;
          --left;
        }
      }
      prev[i] = m;
    }
    std::vector<char> conv(n, 0);
    for (size_t i = 0; i < n; ++i) conv[i] = done[i] >= 0;
    st = retire(b, conv);
    if (st != ISLBM_OK) return st;
  }
  for (size_t i = 0; i < n; ++i) {
    if (steps_to_steady) steps_to_steady[i] = done[i];
    if (nu_mean) nu_mean[i] = nu_out[i];
    if (re_mean) re_mean[i] = re_out[i];
  }
  const islbm_status ra = reactivate_all(b);
  if (ra != ISLBM_OK) return ra;
  return left == 0 ? ISLBM_OK
                   : bfail(b, ISLBM_ERR_NOT_CONVERGED,
                           "islbm_batch_run_to_steady_nu: step budget exhausted");
}
