// C ABI of the solver (declarations and contracts in include/tde.h).
#include <cmath>
#include <cstring>

#include "tde_internal.cuh"

namespace tde {

__global__ void k_set_offsets(int64_t* off, int64_t n) {
  off[0] = 0;
  off[1] = n;
}

int run_solver(const Plan& plan, const Workspace& ws, const int64_t* offsets_dev,
               const double* d, const double* e, double* lambda, cudaStream_t stream) {
  if (cudaMemsetAsync(ws.status, 0, sizeof(Status), stream) != cudaSuccess) return TDE_ECUDA;
  if (cudaMemsetAsync(ws.sigma_bits, 0, 8 * size_t(plan.batch), stream) != cudaSuccess)
    return TDE_ECUDA;
  launch_plan(plan, ws, offsets_dev, stream);
  launch_scale(plan, ws, offsets_dev, d, e, stream);
  launch_leaves(plan, ws, lambda, stream);
  for (int s = 0; s < plan.steps; ++s) launch_step(plan, ws, s, lambda, stream);
  return cudaGetLastError() == cudaSuccess ? TDE_OK : TDE_ECUDA;
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

int64_t tde_last_launch_count(void) { return g_launches; }

}  // extern "C"
