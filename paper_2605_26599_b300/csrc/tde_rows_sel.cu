// Requested rows of the eigenvector matrix: Algorithm 1 with a general row list
// sigma_v ("requested local rows"; duplicate and unordered requests allowed,
// resolved by metadata).  The caller's rows ride through the tree next to the
// boundary rows; every transformation a merge applies to the columns of
// diag(Q_L, Q_R) -- the merge permutation, the deflation rotations and
// permutations, the secular eigenvectors -- is applied to each requested row
// alone (Lemma "selected-row multiplication"; appendix lemmas on column
// permutations and local rotations), so the root returns (Q)_sigma without
// forming Q.
//
// State: row u of X / XD / AX belongs to the distinct requested row U[u] and, at
// each level, holds the entries of the eigenvector row of the node containing
// U[u] over that node's columns [lo, hi) (the node's own index range).  A merge
// with tracked rows runs, besides the boundary-row kernels:
//   k_sel_form     the merge permutation of the child's row, zeros over the other
//                  child's columns (diag(Q_L, Q_R) has a zero block);
//   k_sel_deflate  negligible-z columns pass through; each close-pole rotation run
//                  is replayed with the same prefix-sum formulas as k_deflate
//                  (kept column: sum z_i x_i / sqrt(sum z_i^2); rotated-out column
//                  k: (z_k U_{<k} - W_{<k} x_k) / sqrt(W_{<k} (W_{<k} + z_k^2)));
//   k_sel_rows     x'_j = sum_i x_i zhat_i / Delta_ij / nu_j for the active roots,
//                  up to four rows of one merge per pole sweep;
//   k_sel_place    the ascending order of the parent's eigenvalues.
// z-hat is built at root merges too.  Cost: one extra multiply-add per (pole,
// root) pair and requested row over the merges on the row's path to the root,
// O(n^2) per row in total.
#include <algorithm>

#include "tde_internal.cuh"

namespace tde {

constexpr int kSelRowsPerSweep = 4;

// Sort the requests by row (bitonic, one block), keep the distinct valid rows in
// U and map each request to its row's index.  Rows outside [0, n) set the
// device status to TDE_EINVAL and map to -1 (their output rows are zero).
__global__ void __launch_bounds__(kMaxSel) k_sel_prepare(const int64_t* __restrict__ rows, int nsel,
                                                         int64_t n, int32_t* U, int32_t* nu,
                                                         int32_t* MAP, Status* st) {
  __shared__ unsigned long long key[kMaxSel];
  __shared__ int sm[kMaxSel / 32];
  const int t = threadIdx.x;
  unsigned long long k = ~0ull;  // padding sorts last
  if (t < nsel) {
    const int64_t r = rows[t];
    const bool ok = r >= 0 && r < n;
    if (!ok) set_status(st, TDE_EINVAL);
    k = (static_cast<unsigned long long>(ok ? r : 0x7fffffffLL) << 32) | unsigned(t);
  }
  key[t] = k;
  __syncthreads();
  for (int size = 2; size <= kMaxSel; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const int partner = t ^ stride;
      if (partner > t) {
        const bool up = (t & size) == 0;
        const unsigned long long a = key[t], b = key[partner];
        if ((a > b) == up) {
          key[t] = b;
          key[partner] = a;
        }
      }
      __syncthreads();
    }
  }
  const int row = (t < nsel) ? int(key[t] >> 32) : 0x7fffffff;
  const bool valid = row != 0x7fffffff;
  const int prow = (t > 0 && t < nsel) ? int(key[t - 1] >> 32) : -1;
  const int first = (valid && row != prow) ? 1 : 0;
  int total;
  const int ex = block_excl_scan<kMaxSel>(first, sm, &total);
  if (first) U[ex] = row;
  if (t >= total && t < nsel) U[t] = 0x7fffffff;
  if (t < nsel) MAP[int(key[t] & 0xffffffffu)] = valid ? ex + first - 1 : -1;
  if (t == 0) *nu = total;
}

// The merge of this step that holds requested row u, or -1.
__device__ __forceinline__ int64_t sel_merge(const SelArgs& sa, const Merge* M, int64_t cnt, int u,
                                             Merge* m) {
  if (u >= *sa.nu) return -1;
  const int r = sa.U[u];
  const int64_t g = find_merge(M, cnt, r);
  *m = M[g];
  return (r >= m->lo && r < m->hi) ? g : -1;
}

// first index in U[0..nu) holding a row >= r
__device__ __forceinline__ int sel_lower(const SelArgs& sa, int r) {
  int lo = 0, hi = *sa.nu;
  while (lo < hi) {
    const int md = (lo + hi) >> 1;
    if (sa.U[md] < r)
      lo = md + 1;
    else
      hi = md;
  }
  return lo;
}

__global__ void k_sel_form(SelArgs sa, const Merge* __restrict__ M, int64_t cnt,
                           const double* __restrict__ LAM) {
  const int u = blockIdx.y;
  Merge m;
  if (sel_merge(sa, M, cnt, u, &m) < 0) return;
  const bool left = sa.U[u] < m.mid;
  const double* x = sa.X + int64_t(u) * sa.N;
  double* xd = sa.XD + int64_t(u) * sa.N;
  for (int p = m.lo + blockIdx.x * blockDim.x + threadIdx.x; p < m.hi; p += gridDim.x * blockDim.x) {
    const double lam = LAM[p];
    if (p < m.mid) {
      const int out = m.lo + (p - m.lo) + count_less(LAM + m.mid, m.hi - m.mid, lam);
      xd[out] = left ? x[p] : 0.0;
    } else {
      const int out = m.lo + (p - m.mid) + count_leq(LAM + m.lo, m.mid - m.lo, lam);
      xd[out] = left ? 0.0 : x[p];
    }
  }
}

struct SelDeflateArgs {
  const Merge* M;
  int64_t cnt;
  const MState* ms;
  const double* Z;
  const int32_t *SURV, *OUTIDX, *ACTMAP;
  const uint8_t *PFLAG, *RFLAG;
};

// One warp per requested row: the survivors in chunks of 32 with a segmented
// inclusive scan of (z^2, z x) that restarts at every run head.
__global__ void k_sel_deflate(SelArgs sa, SelDeflateArgs a) {
  const int lane = threadIdx.x & 31;
  const int u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (u >= sa.nsel) return;
  Merge m;
  const int64_t g = sel_merge(sa, a.M, a.cnt, u, &m);
  if (g < 0) return;
  const int lo = m.lo, n0 = m.hi - m.lo, S = a.ms[g].surv;
  const double* xd = sa.XD + int64_t(u) * sa.N + lo;
  double* ax = sa.AX + int64_t(u) * sa.N + lo;
  for (int i = lane; i < n0; i += 32)
    if (a.PFLAG[lo + i] == 1) ax[a.OUTIDX[lo + i]] = xd[i];
  double cw = 0.0, cv = 0.0;  // carry: inclusive (z^2, z x) of the previous chunk's last survivor
  for (int c0 = 0; c0 < S; c0 += 32) {
    const int k = c0 + lane;
    const bool valid = k < S;
    int pos = 0;
    bool head = false;
    double zk = 0.0, xk = 0.0;
    if (valid) {
      pos = a.SURV[lo + k] - lo;
      head = a.RFLAG[lo + k] != 0;
      zk = a.Z[lo + pos];
      xk = xd[pos];
    }
    const double wk = zk * zk, vk = zk * xk;
    double w = wk, v = vk;
    bool h = head;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double wo = __shfl_up_sync(0xffffffffu, w, o);
      const double vo = __shfl_up_sync(0xffffffffu, v, o);
      const bool ho = __shfl_up_sync(0xffffffffu, h, o);
      if (lane >= o) {
        if (!h) {
          w += wo;
          v += vo;
        }
        h = h || ho;
      }
    }
    if (!h) {  // no run head at or before this lane in the chunk: the carry continues
      w += cw;
      v += cv;
    }
    const double pw_up = __shfl_up_sync(0xffffffffu, w, 1);
    const double pv_up = __shfl_up_sync(0xffffffffu, v, 1);
    const double pw = lane == 0 ? cw : pw_up, pv = lane == 0 ? cv : pv_up;
    if (valid && !head) {  // rotated out against the run prefix
      const double sc = 1.0 / sqrt(pw * (pw + wk));
      ax[a.OUTIDX[lo + pos]] = (zk * pv - pw * xk) * sc;
    }
    const bool runend = valid && (k == S - 1 || a.RFLAG[lo + k + 1] != 0);
    if (runend) ax[a.ACTMAP[lo + k]] = head ? xk : v / sqrt(w);
    cw = __shfl_sync(0xffffffffu, w, 31);
    cv = __shfl_sync(0xffffffffu, v, 31);
  }
}

struct SelRowsArgs {
  const Merge* M;
  int64_t cnt;
  const MState* ms;
  const double *AD, *ZH, *DORG, *TAU;
  Status* st;
};

// Block row y = requested row u; a block works only if u starts a group of up to
// four consecutive requested rows of the same merge.  One warp per active root.
__global__ void __launch_bounds__(128) k_sel_rows(SelArgs sa, SelRowsArgs a) {
  const int u = blockIdx.y;
  Merge m;
  const int64_t g = sel_merge(sa, a.M, a.cnt, u, &m);
  if (g < 0) return;
  const int first = sel_lower(sa, m.lo);
  if ((u - first) % kSelRowsPerSweep != 0) return;
  const int nr = min(kSelRowsPerSweep, sel_lower(sa, m.hi) - u);
  const int lo = m.lo, K = a.ms[g].K;
  const int lane = threadIdx.x & 31;
  const double* AD = a.AD + lo;
  const double* ZH = a.ZH + lo;
  const double* x0 = sa.AX + int64_t(u) * sa.N + lo;
  const int64_t N = sa.N;
  unsigned long long sweeps = 0;
  for (int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < K;
       j += gridDim.x * (blockDim.x >> 5)) {
    const double dorg = a.DORG[lo + j], tau = a.TAU[lo + j];
    double s2 = 0.0, c0 = 0.0, c1 = 0.0, c2 = 0.0, c3 = 0.0;
    for (int i = lane; i < K; i += 32) {
      const double t = ZH[i] * rcp_refined((AD[i] - dorg) - tau);
      s2 = fma(t, t, s2);
      c0 = fma(x0[i], t, c0);
      if (nr > 1) c1 = fma(x0[N + i], t, c1);
      if (nr > 2) c2 = fma(x0[2 * N + i], t, c2);
      if (nr > 3) c3 = fma(x0[3 * N + i], t, c3);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      c0 += __shfl_xor_sync(0xffffffffu, c0, o);
      c1 += __shfl_xor_sync(0xffffffffu, c1, o);
      c2 += __shfl_xor_sync(0xffffffffu, c2, o);
      c3 += __shfl_xor_sync(0xffffffffu, c3, o);
    }
    if (lane == 0) {
      const double inv = 1.0 / sqrt(s2);
      double* out = sa.XD + int64_t(u) * N + lo + j;
      out[0] = c0 * inv;
      if (nr > 1) out[N] = c1 * inv;
      if (nr > 2) out[2 * N] = c2 * inv;
      if (nr > 3) out[3 * N] = c3 * inv;
    }
    sweeps += unsigned(K);
  }
  if (lane == 0 && sweeps) {
    atomicAdd(&a.st->work[kWorkSelSweepPairs], sweeps);
    atomicAdd(&a.st->work[kWorkSelRowPairs], sweeps * unsigned(nr));
  }
}

__global__ void k_sel_place(SelArgs sa, const Merge* __restrict__ M, int64_t cnt,
                            const MState* __restrict__ ms, const double* __restrict__ LAMA,
                            const double* __restrict__ AD) {
  const int u = blockIdx.y;
  Merge m;
  const int64_t g = sel_merge(sa, M, cnt, u, &m);
  if (g < 0) return;
  const int lo = m.lo, K = ms[g].K, F = (m.hi - m.lo) - K;
  const double* xd = sa.XD + int64_t(u) * sa.N;
  const double* ax = sa.AX + int64_t(u) * sa.N;
  double* x = sa.X + int64_t(u) * sa.N;
  for (int p = lo + blockIdx.x * blockDim.x + threadIdx.x; p < m.hi; p += gridDim.x * blockDim.x) {
    const int local = p - lo;
    if (local < K) {
      const int rank = local + count_less(AD + lo + K, F, LAMA[p]);
      x[lo + rank] = xd[p];
    } else {
      const int rank = (local - K) + count_leq(LAMA + lo, K, AD[p]);
      x[lo + rank] = ax[p];
    }
  }
}

__global__ void k_sel_gather(SelArgs sa, const int32_t* __restrict__ MAP, int64_t nsel, int64_t n,
                             double* qrows) {
  const int64_t total = nsel * n;
  for (int64_t f = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; f < total;
       f += int64_t(gridDim.x) * blockDim.x) {
    const int64_t q = f / n, j = f - q * n;
    const int u = MAP[q];
    qrows[f] = u >= 0 ? sa.X[int64_t(u) * sa.N + j] : 0.0;
  }
}

// ---- launchers ---------------------------------------------------------------
static int sel_grid_x(const Plan& plan, int step, int per_block) {
  const int64_t k0 = std::max<int64_t>(plan.step_maxsize[step], 1);
  return int(std::min<int64_t>((k0 + per_block - 1) / per_block, 148 * 4));
}

void launch_sel_prepare(const SelArgs& sa, const int64_t* rows, int64_t nrows_total, int32_t* U,
                        int32_t* nu, int32_t* MAP, Status* st, cudaStream_t s) {
  k_sel_prepare<<<1, kMaxSel, 0, s>>>(rows, sa.nsel, nrows_total, U, nu, MAP, st);
  g_launches += 1;
}

void launch_sel_form(const Plan& plan, const Workspace& ws, const SelArgs& sa, int step,
                     LevelState in, cudaStream_t s) {
  const dim3 grid(sel_grid_x(plan, step, 256), sa.nsel);
  k_sel_form<<<grid, 256, 0, s>>>(sa, ws.merges + plan.step_base[step], plan.step_count[step], in.lam);
  g_launches += 1;
}

void launch_sel_deflate(const Plan& plan, const Workspace& ws, const SelArgs& sa, int step,
                        cudaStream_t s) {
  SelDeflateArgs a;
  a.M = ws.merges + plan.step_base[step];
  a.cnt = plan.step_count[step];
  a.ms = ws.mstate;
  a.Z = ws.Z;
  a.SURV = ws.SURV;
  a.OUTIDX = ws.OUTIDX;
  a.ACTMAP = ws.ACTMAP;
  a.PFLAG = ws.PFLAG;
  a.RFLAG = ws.RFLAG;
  k_sel_deflate<<<(sa.nsel + 3) / 4, 128, 0, s>>>(sa, a);
  g_launches += 1;
}

void launch_sel_rows(const Plan& plan, const Workspace& ws, const SelArgs& sa, int step,
                     cudaStream_t s) {
  SelRowsArgs a;
  a.M = ws.merges + plan.step_base[step];
  a.cnt = plan.step_count[step];
  a.ms = ws.mstate;
  a.AD = ws.AD;
  a.ZH = ws.Z;
  a.DORG = reinterpret_cast<const double*>(ws.KEYA);
  a.TAU = ws.TAU;
  a.st = ws.status;
  const dim3 grid(sel_grid_x(plan, step, 4), sa.nsel);
  k_sel_rows<<<grid, 128, 0, s>>>(sa, a);
  g_launches += 1;
}

void launch_sel_place(const Plan& plan, const Workspace& ws, const SelArgs& sa, int step,
                      cudaStream_t s) {
  const dim3 grid(sel_grid_x(plan, step, 256), sa.nsel);
  k_sel_place<<<grid, 256, 0, s>>>(sa, ws.merges + plan.step_base[step], plan.step_count[step],
                                   ws.mstate, ws.D, ws.AD);
  g_launches += 1;
}

void launch_sel_gather(const SelArgs& sa, const int32_t* MAP, int64_t nsel, int64_t n,
                       double* qrows, cudaStream_t s) {
  const int64_t total = nsel * n;
  const int grid = int(std::min<int64_t>((total + 255) / 256, 148 * 16));
  k_sel_gather<<<std::max(grid, 1), 256, 0, s>>>(sa, MAP, nsel, n, qrows);
  g_launches += 1;
}

}  // namespace tde
