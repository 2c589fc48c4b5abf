// C ABI of the solver (declarations and contracts in include/tde.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "tde_internal.cuh"

namespace tde {

// Optional per-launch timing: an event pair around every kernel of a call, summed
// per kernel class by tde_profile_collect.  Off by default; never enable it while
// a stream is being captured into a graph.
struct ProfRec {
  int id;
  int step;  // merge step the launch belongs to, -1 before the first merge step
  cudaEvent_t a, b;
};
static thread_local int g_prof_step = -1;

static thread_local Tuning g_tuning;
Tuning& thread_tuning() { return g_tuning; }
static thread_local bool g_prof_on = false;
static thread_local uint32_t g_prof_mask = 0xffffffffu;  // kernel classes recorded
static thread_local std::vector<cudaEvent_t> g_pool;
static thread_local size_t g_pool_next = 0;
static thread_local std::vector<ProfRec> g_recs;
static thread_local cudaEvent_t g_open[kNumKernelIds];

static cudaEvent_t next_event() {
  if (g_pool_next == g_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    g_pool.push_back(e);
  }
  return g_pool[g_pool_next++];
}
void prof_begin(int id, cudaStream_t s) {
  if (!g_prof_on || !((g_prof_mask >> id) & 1u)) return;
  cudaEvent_t e = next_event();
  cudaEventRecord(e, s);
  g_open[id] = e;
}
void prof_end(int id, cudaStream_t s) {
  if (!g_prof_on || !((g_prof_mask >> id) & 1u)) return;
  cudaEvent_t e = next_event();
  cudaEventRecord(e, s);
  g_recs.push_back(ProfRec{id, g_prof_step, g_open[id], e});
}

__global__ void k_set_offsets(int64_t* off, int64_t n) {
  off[0] = 0;
  off[1] = n;
}

int run_solver(const Plan& plan, const Workspace& ws, const int64_t* offsets_dev,
               const double* d, const double* e, double* lambda, cudaStream_t stream) {
  if (cudaMemsetAsync(ws.status, 0, sizeof(Status), stream) != cudaSuccess) return TDE_ECUDA;
  if (cudaMemsetAsync(ws.sigma_bits, 0, 8 * size_t(plan.batch), stream) != cudaSuccess)
    return TDE_ECUDA;
  g_prof_step = -1;
  launch_plan(plan, ws, offsets_dev, stream);
  launch_scale(plan, ws, offsets_dev, d, e, stream);
  launch_leaves(plan, ws, lambda, stream);
  const LevelState state{ws.LAM, ws.BLO, ws.BHI};
  for (int s = 0; s < plan.steps; ++s) {
    g_prof_step = s;
    launch_step(plan, ws, s, lambda, stream, state, state);
  }
  g_prof_step = -1;
  return cudaGetLastError() == cudaSuccess ? TDE_OK : TDE_ECUDA;
}

// Workspace of tde_eigvecs_rows: the eigenvalue workspace, then the requested-row
// section (U, its count, the request map, and the three row arrays X, XD, AX of
// nsel x N doubles each).
static size_t carve_sel(const Plan& plan, int64_t nsel, void* base, Workspace* w, SelArgs* sa,
                        int32_t** U, int32_t** nu, int32_t** MAP) {
  size_t off = carve_workspace(plan, base, w);
  auto take = [&](size_t bytes) -> char* {
    char* ptr = base ? static_cast<char*>(base) + off : nullptr;
    off += (bytes + 255) & ~size_t(255);
    return ptr;
  };
  const size_t N = size_t(std::max<int64_t>(plan.nrows, 1));
  const size_t ns = size_t(std::max<int64_t>(nsel, 1));
  int32_t* u = reinterpret_cast<int32_t*>(take(4 * ns));
  int32_t* cnt = reinterpret_cast<int32_t*>(take(4));
  int32_t* map = reinterpret_cast<int32_t*>(take(4 * ns));
  double* X = reinterpret_cast<double*>(take(8 * ns * N));
  double* XD = reinterpret_cast<double*>(take(8 * ns * N));
  double* AX = reinterpret_cast<double*>(take(8 * ns * N));
  if (sa) {
    sa->U = u;
    sa->nu = cnt;
    sa->nsel = int32_t(nsel);
    sa->N = int64_t(N);
    sa->X = X;
    sa->XD = XD;
    sa->AX = AX;
    *U = u;
    *nu = cnt;
    *MAP = map;
  }
  return off;
}

}  // namespace tde

using namespace tde;

extern "C" {

int tde_eigvals_workspace(int64_t n, int32_t leaf, size_t* bytes) {
  if (n < 0 || bytes == nullptr) return TDE_EINVAL;
  int64_t off[2] = {0, n};
  Plan p;
  int rc = build_plan(1, off, leaf, &p);
  if (rc != TDE_OK) return rc;
  *bytes = carve_workspace(p, nullptr, nullptr);
  return TDE_OK;
}

int tde_eigvals(int64_t n, const double* d, const double* e, double* lambda, int32_t leaf,
                void* ws, size_t ws_bytes, void* stream) {
  g_launches = 0;
  if (n < 0) return TDE_EINVAL;
  if (n == 0) return TDE_OK;
  if (d == nullptr || lambda == nullptr || ws == nullptr || (n > 1 && e == nullptr))
    return TDE_EINVAL;
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return TDE_EINVAL;
  int64_t off[2] = {0, n};
  Plan p;
  int rc = build_plan(1, off, leaf, &p);
  if (rc != TDE_OK) return rc;
  Workspace w;
  size_t need = carve_workspace(p, ws, &w);
  if (ws_bytes < need) return TDE_EWORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_set_offsets<<<1, 1, 0, s>>>(w.offsets, n);
  g_launches += 1;
  return run_solver(p, w, w.offsets, d, e, lambda, s);
}

int tde_eigvals_batched_workspace(int64_t batch, const int64_t* offsets_host, int32_t leaf,
                                  size_t* bytes) {
  if (bytes == nullptr) return TDE_EINVAL;
  Plan p;
  int rc = build_plan(batch, offsets_host, leaf, &p);
  if (rc != TDE_OK) return rc;
  *bytes = carve_workspace(p, nullptr, nullptr);
  return TDE_OK;
}

int tde_eigvals_batched(int64_t batch, const int64_t* offsets_host, const int64_t* offsets_dev,
                        const double* d, const double* e, double* lambda, int32_t leaf,
                        void* ws, size_t ws_bytes, void* stream) {
  g_launches = 0;
  Plan p;
  int rc = build_plan(batch, offsets_host, leaf, &p);
  if (rc != TDE_OK) return rc;
  if (p.nrows == 0) return TDE_OK;
  if (offsets_dev == nullptr || d == nullptr || lambda == nullptr || ws == nullptr ||
      (p.nrows > 1 && e == nullptr))
    return TDE_EINVAL;
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return TDE_EINVAL;
  Workspace w;
  size_t need = carve_workspace(p, ws, &w);
  if (ws_bytes < need) return TDE_EWORKSPACE;
  return run_solver(p, w, offsets_dev, d, e, lambda, static_cast<cudaStream_t>(stream));
}

int tde_get_info(const void* ws, void* stream, int32_t* info) {
  if (ws == nullptr || info == nullptr) return TDE_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Status* st = static_cast<const Status*>(ws);
  if (cudaMemcpyAsync(info, &st->info, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return TDE_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return TDE_ECUDA;
  return TDE_OK;
}

int tde_eigvecs_rows_workspace(int64_t n, int64_t nsel, int32_t leaf, size_t* bytes) {
  if (n < 0 || nsel < 0 || nsel > kMaxSel || bytes == nullptr) return TDE_EINVAL;
  int64_t off[2] = {0, n};
  Plan p;
  int rc = build_plan(1, off, leaf, &p);
  if (rc != TDE_OK) return rc;
  *bytes = carve_sel(p, nsel, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
  return TDE_OK;
}

int tde_eigvecs_rows(int64_t n, const double* d, const double* e, int64_t nsel,
                     const int64_t* rows, double* lambda, double* qrows, int32_t leaf, void* ws,
                     size_t ws_bytes, void* stream) {
  g_launches = 0;
  if (n < 0 || nsel < 0 || nsel > kMaxSel) return TDE_EINVAL;
  if (n == 0) return TDE_OK;
  if (d == nullptr || lambda == nullptr || ws == nullptr || (n > 1 && e == nullptr) ||
      (nsel > 0 && (rows == nullptr || qrows == nullptr)))
    return TDE_EINVAL;
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return TDE_EINVAL;
  int64_t off[2] = {0, n};
  Plan p;
  int rc = build_plan(1, off, leaf, &p);
  if (rc != TDE_OK) return rc;
  Workspace w;
  SelArgs sa;
  int32_t *U = nullptr, *nu = nullptr, *MAP = nullptr;
  const size_t need = carve_sel(p, nsel, ws, &w, &sa, &U, &nu, &MAP);
  if (ws_bytes < need) return TDE_EWORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(w.status, 0, sizeof(Status), s) != cudaSuccess) return TDE_ECUDA;
  if (cudaMemsetAsync(w.sigma_bits, 0, 8, s) != cudaSuccess) return TDE_ECUDA;
  k_set_offsets<<<1, 1, 0, s>>>(w.offsets, n);
  g_launches += 1;
  g_prof_step = -1;
  launch_plan(p, w, w.offsets, s);
  launch_scale(p, w, w.offsets, d, e, s);
  launch_leaves(p, w, lambda, s);
  if (nsel > 0) {
    launch_sel_prepare(sa, rows, n, U, nu, MAP, w.status, s);
    launch_sel_leaves(p, w, sa, s);
  }
  const LevelState state{w.LAM, w.BLO, w.BHI};
  for (int st = 0; st < p.steps; ++st) {
    g_prof_step = st;
    launch_step(p, w, st, lambda, s, state, state, false, nsel > 0 ? &sa : nullptr);
  }
  g_prof_step = -1;
  if (nsel > 0) launch_sel_gather(sa, MAP, nsel, n, qrows, s);
  return cudaGetLastError() == cudaSuccess ? TDE_OK : TDE_ECUDA;
}

int tde_dense_eigvals_workspace(int64_t n, int32_t leaf, size_t* bytes) {
  if (n < 0 || bytes == nullptr) return TDE_EINVAL;
  int64_t off[2] = {0, n};
  Plan p;
  int rc = build_plan(1, off, leaf, &p);
  if (rc != TDE_OK) return rc;
  *bytes = dense_workspace(n, carve_workspace(p, nullptr, nullptr));
  return TDE_OK;
}

int tde_dense_eigvals(int64_t n, const double* A, int64_t lda, double* lambda, int32_t leaf,
                      void* ws, size_t ws_bytes, void* stream) {
  g_launches = 0;
  if (n < 0) return TDE_EINVAL;
  if (n == 0) return TDE_OK;
  if (A == nullptr || lambda == nullptr || ws == nullptr || lda < n) return TDE_EINVAL;
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return TDE_EINVAL;
  int64_t off[2] = {0, n};
  Plan p;
  int rc = build_plan(1, off, leaf, &p);
  if (rc != TDE_OK) return rc;
  const size_t tri = carve_workspace(p, nullptr, nullptr);
  if (ws_bytes < dense_workspace(n, tri)) return TDE_EWORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double *d = nullptr, *e = nullptr;
  rc = dense_reduce(n, A, lda, ws, tri, &d, &e, s);
  if (rc != TDE_OK) return rc;
  Workspace w;
  carve_workspace(p, ws, &w);
  k_set_offsets<<<1, 1, 0, s>>>(w.offsets, n);
  g_launches += 1;
  return run_solver(p, w, w.offsets, d, e, lambda, s);
}

int64_t tde_last_launch_count(void) { return g_launches; }

int tde_set_tuning(int32_t warp_min_k, int32_t small_list_min) {
  if (warp_min_k < 0 || small_list_min < 0) return TDE_EINVAL;
  const Tuning d;
  g_tuning.warp_min_k = warp_min_k > 0 ? warp_min_k : d.warp_min_k;
  g_tuning.small_list_min = small_list_min > 0 ? small_list_min : d.small_list_min;
  return TDE_OK;
}

int tde_set_multipole(int32_t min_k, int32_t* previous) {
  if (min_k != 0 && min_k < 256) return TDE_EINVAL;
  if (previous != nullptr) *previous = g_tuning.multipole_min_k;
  g_tuning.multipole_min_k = min_k > 0 ? min_k : Tuning{}.multipole_min_k;
  return TDE_OK;
}

int tde_get_tuning(int32_t* out) {
  if (out == nullptr) return TDE_EINVAL;
  out[0] = g_tuning.warp_min_k;
  out[1] = g_tuning.small_list_min;
  return TDE_OK;
}

int tde_plan_query(int64_t batch, const int64_t* offsets_host, int32_t leaf, int64_t* out) {
  if (out == nullptr) return TDE_EINVAL;
  Plan p;
  int rc = build_plan(batch, offsets_host, leaf, &p);
  if (rc != TDE_OK) return rc;
  out[0] = p.steps;
  out[1] = p.nleaves;
  out[2] = p.nmerges;
  out[3] = p.cmax;
  return TDE_OK;
}

int tde_profile_enable(int on) {
  g_prof_on = on != 0;
  return TDE_OK;
}

int tde_profile_select(uint32_t mask) {
  g_prof_mask = mask != 0u ? mask : 0xffffffffu;
  return TDE_OK;
}

int tde_profile_collect_steps(int nids, int nsteps, double* ms, int64_t* launches);
int tde_profile_collect(int nids, double* ms, int64_t* launches) {
  return tde_profile_collect_steps(nids, 0, ms, launches);
}

int tde_profile_collect_steps(int nids, int nsteps, double* ms, int64_t* launches) {
  if (nids < 0 || nsteps < 0 || (nids > 0 && (ms == nullptr || launches == nullptr)))
    return TDE_EINVAL;
  const int rows = nsteps + 1;
  for (int i = 0; i < nids * rows; ++i) {
    ms[i] = 0.0;
    launches[i] = 0;
  }
  int rc = TDE_OK;
  for (const ProfRec& r : g_recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) {
      rc = TDE_ECUDA;
      continue;
    }
    float t = 0.f;
    cudaEventElapsedTime(&t, r.a, r.b);
    if (r.id < nids) {
      // row 0: every launch; row s + 1: launches of merge step s (when requested)
      ms[r.id] += t;
      launches[r.id] += 1;
      if (r.step >= 0 && r.step < nsteps) {
        ms[(r.step + 1) * nids + r.id] += t;
        launches[(r.step + 1) * nids + r.id] += 1;
      }
    }
  }
  g_recs.clear();
  g_pool_next = 0;
  return rc;
}

int tde_read_work(const void* ws, void* stream, unsigned long long* out, int n) {
  if (ws == nullptr || out == nullptr || n < 0 || n > kNumWork) return TDE_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Status* st = static_cast<const Status*>(ws);
  if (cudaMemcpyAsync(out, st->work, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, s) !=
      cudaSuccess)
    return TDE_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return TDE_ECUDA;
  return TDE_OK;
}

}  // extern "C"
