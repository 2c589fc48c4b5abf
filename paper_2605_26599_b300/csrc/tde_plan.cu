// Split-tree plan, workspace carving and input scaling.
//
// Tree (Sec. 3.3 balanced tree; Sec. 4.1 split tree built on the device): node
// (h, i) of a matrix of order n covers rows [floor(i n / 2^h), floor((i+1) n / 2^h)),
// so sibling sizes differ by at most one and every leaf sits at depth L, the
// smallest L with ceil(n / 2^L) <= leaf.  Merges are processed bottom-up in
// "steps": step s merges depth L_k - 1 - s of every matrix k with L_k > s, so a
// forest of uneven trees shares each level's launches (Sec. 4.1 level batching).
// The host derives only counts from the packing; the descriptors themselves are
// written by two device kernels, so a call never copies host memory.
//
// Driver preprocessing (Sec. 4.2: "splits at negligible off-diagonal entries,
// scales unreduced blocks"): every matrix is scaled by a power of two so that
// max|T| lies in [1, 2) (exact in binary floating point), and an off-diagonal with
// |e_i| <= eps sqrt|d_i| sqrt|d_{i+1}| is set to zero.  A zero coupling at a cut
// gives rho = 0, which deflates every pole of that merge, so the spectrum is the
// union of the blocks without changing the tree.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "tde_internal.cuh"

namespace tde {

thread_local int64_t g_launches = 0;

int build_plan(int64_t batch, const int64_t* off, int32_t leaf, Plan* plan) {
  if (batch < 0 || (batch > 0 && off == nullptr) || plan == nullptr) return TDE_EINVAL;
  if (batch > int64_t(kMatMask) + 1) return TDE_EINVAL;  // matrix index bits of Merge::info
  if (leaf == 0) leaf = 32;
  if (leaf < 1 || leaf > kMaxLeaf) return TDE_EINVAL;
  Plan p;
  p.batch = batch;
  p.leaf = leaf;
  p.tune = thread_tuning();
  if (batch > 0 && off[0] != 0) return TDE_EINVAL;
  for (int64_t k = 0; k < batch; ++k) {
    int64_t nk = off[k + 1] - off[k];
    if (nk < 0) return TDE_EINVAL;
    if (nk == 0) continue;
    int L = levels_of(nk, leaf);
    p.nleaves += int64_t(1) << L;
    if (L > p.steps) p.steps = L;
    if (L > kMaxSteps) return TDE_EINVAL;
    for (int s = 0; s < L; ++s) {
      const int h = L - 1 - s;
      p.step_count[s] += int64_t(1) << h;
      if (h > 0) p.step_has_nonroot[s] = true;
      const int64_t size = (nk + (int64_t(1) << h) - 1) >> h;  // ceil(n / 2^h)
      if (size > p.step_maxsize[s]) p.step_maxsize[s] = size;
    }
  }
  p.nrows = batch > 0 ? off[batch] : 0;
  if (p.nrows >= (int64_t(1) << 31) - 1024) return TDE_EINVAL;
  int64_t acc = 0;
  for (int s = 0; s < p.steps; ++s) {
    p.step_base[s] = acc;
    acc += p.step_count[s];
    p.cmax = std::max(p.cmax, p.step_count[s]);
  }
  p.nmerges = acc;
  *plan = p;
  return TDE_OK;
}

static size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

size_t carve_workspace(const Plan& plan, void* base, Workspace* ws) {
  const size_t N = size_t(std::max<int64_t>(plan.nrows, 1));
  const size_t B = size_t(std::max<int64_t>(plan.batch, 1));
  size_t off = 0;
  char* b = static_cast<char*>(base);
  auto take = [&](size_t bytes) -> void* {
    void* ptr = b ? static_cast<void*>(b + off) : nullptr;
    off += align_up(bytes);
    return ptr;
  };
  Workspace w{};
  w.status = static_cast<Status*>(take(sizeof(Status)));
  w.sigma_bits = static_cast<unsigned long long*>(take(8 * B));
  w.offsets = static_cast<int64_t*>(take(8 * (B + 1)));
  double** dbl[] = {&w.ds, &w.es, &w.LAM, &w.BLO, &w.BHI, &w.D, &w.Z, &w.RLO, &w.RHI,
                    &w.AD, &w.AZ, &w.ALO, &w.AHI, &w.TAU};
  for (double** p : dbl) *p = static_cast<double*>(take(8 * N));
  int32_t** ints[] = {&w.ORG,  &w.ROOTMAP, &w.ROOTMAP2, &w.SURV,   &w.IDXA,
                      &w.IDXB, &w.ZPOS,    &w.OUTIDX,   &w.ACTMAP, &w.KEEPIDX};
  for (int32_t** p : ints) *p = static_cast<int32_t*>(take(4 * N));
  w.PFLAG = static_cast<uint8_t*>(take(N));
  w.RFLAG = static_cast<uint8_t*>(take(N + 1));
  w.KEYA = static_cast<unsigned long long*>(take(8 * N));
  w.KEYB = static_cast<unsigned long long*>(take(8 * N));
  w.merges = static_cast<Merge*>(take(sizeof(Merge) * size_t(std::max<int64_t>(plan.nmerges, 1))));
  w.leaves = static_cast<Leaf*>(take(sizeof(Leaf) * size_t(std::max<int64_t>(plan.nleaves, 1))));
  w.mstate = static_cast<MState*>(take(sizeof(MState) * size_t(std::max<int64_t>(plan.cmax, 1))));
  w.pfx = static_cast<int32_t*>(take(4 * size_t(plan.steps + 1) * (B + 1)));
  w.bytes = off;
  if (ws) *ws = w;
  return off;
}

// ---- device plan ------------------------------------------------------------

struct PlanArgs {
  int64_t batch;
  int32_t leaf;
  int32_t steps;
  int64_t nmerges;
  int64_t nleaves;
  int64_t step_base[kMaxSteps];
};

// Block b < steps: per-matrix merge counts of step b; block b == steps: leaf
// counts.  Exclusive prefix over matrices into pfx[b][0..batch].
__global__ void k_plan_prefix(const int64_t* __restrict__ off, PlanArgs a, int32_t* pfx) {
  __shared__ int sm[8];
  const int b = blockIdx.x;
  int32_t* row = pfx + int64_t(b) * (a.batch + 1);
  int carry = 0;
  for (int64_t base = 0; base < a.batch; base += 256) {
    int64_t k = base + threadIdx.x;
    int c = 0;
    if (k < a.batch) {
      int64_t nk = off[k + 1] - off[k];
      if (nk > 0) {
        int L = levels_of(nk, a.leaf);
        if (b == a.steps)
          c = 1 << L;
        else if (L > b)
          c = 1 << (L - 1 - b);
      }
    }
    int total;
    int ex = block_excl_scan<256>(c, sm, &total);
    if (k < a.batch) row[k] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) row[a.batch] = carry;
}

__device__ __forceinline__ int64_t find_row(const int32_t* row, int64_t batch, int64_t g) {
  // largest k with row[k] <= g (row is non-decreasing; entries for empty
  // matrices repeat, so take the last of a run of equal values)
  int64_t lo = 0, hi = batch;  // row[hi] > g
  while (hi - lo > 1) {
    int64_t m = (lo + hi) >> 1;
    if (row[m] <= g)
      lo = m;
    else
      hi = m;
  }
  return lo;
}

__global__ void k_plan_fill(const int64_t* __restrict__ off, PlanArgs a,
                            const int32_t* __restrict__ pfx, Merge* merges, Leaf* leaves) {
  const int64_t total = a.nmerges + a.nleaves;
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < total;
       g += int64_t(gridDim.x) * blockDim.x) {
    if (g < a.nmerges) {
      int s = 0;
      while (s + 1 < a.steps && a.step_base[s + 1] <= g) ++s;
      int64_t local = g - a.step_base[s];
      const int32_t* row = pfx + int64_t(s) * (a.batch + 1);
      int64_t k = find_row(row, a.batch, local);
      int64_t i = local - row[k];
      int64_t o = off[k], n = off[k + 1] - o;
      int L = levels_of(n, a.leaf);
      int h = L - 1 - s;
      Merge m;
      m.lo = int32_t(o + ((i * n) >> h));
      m.hi = int32_t(o + (((i + 1) * n) >> h));
      m.mid = int32_t(o + (((2 * i + 1) * n) >> (h + 1)));
      m.info = int32_t(uint32_t(k) | (h == 0 ? kRootBit : 0u) | (i == 0 ? kLeftSpineBit : 0u) |
                       (i == (int64_t(1) << h) - 1 ? kRightSpineBit : 0u));
      merges[g] = m;
    } else {
      int64_t local = g - a.nmerges;
      const int32_t* row = pfx + int64_t(a.steps) * (a.batch + 1);
      int64_t k = find_row(row, a.batch, local);
      int64_t i = local - row[k];
      int64_t o = off[k], n = off[k + 1] - o;
      int L = levels_of(n, a.leaf);
      Leaf lf;
      lf.lo = int32_t(o + ((i * n) >> L));
      lf.hi = int32_t(o + (((i + 1) * n) >> L));
      lf.mat = int32_t(k);
      lf.flags = (lf.lo > o ? 1 : 0) | (lf.hi < o + n ? 2 : 0) | (L == 0 ? 4 : 0);
      leaves[local] = lf;
    }
  }
}

void launch_plan(const Plan& plan, const Workspace& ws, const int64_t* off, cudaStream_t s) {
  PlanArgs a{};
  a.batch = plan.batch;
  a.leaf = plan.leaf;
  a.steps = plan.steps;
  a.nmerges = plan.nmerges;
  a.nleaves = plan.nleaves;
  for (int i = 0; i < kMaxSteps; ++i) a.step_base[i] = plan.step_base[i];
  prof_begin(kKPlan, s);
  k_plan_prefix<<<plan.steps + 1, 256, 0, s>>>(off, a, ws.pfx);
  int64_t total = plan.nmerges + plan.nleaves;
  int grid = int(std::min<int64_t>((total + 255) / 256, 148 * 16));
  k_plan_fill<<<std::max(grid, 1), 256, 0, s>>>(off, a, ws.pfx, ws.merges, ws.leaves);
  prof_end(kKPlan, s);
  g_launches += 2;
}

// ---- scaling --------------------------------------------------------------

__device__ __forceinline__ int64_t matrix_of(const int64_t* off, int64_t batch, int64_t p) {
  int64_t lo = 0, hi = batch;  // off[lo] <= p < off[hi]
  while (hi - lo > 1) {
    int64_t m = (lo + hi) >> 1;
    if (off[m] <= p)
      lo = m;
    else
      hi = m;
  }
  return lo;
}

__global__ void k_sigma(const int64_t* __restrict__ off, int64_t batch, int64_t nrows,
                        const double* __restrict__ d, const double* __restrict__ e,
                        unsigned long long* sigma_bits, Status* st) {
  for (int64_t base = blockIdx.x * int64_t(blockDim.x); base < nrows;
       base += int64_t(gridDim.x) * blockDim.x) {
    int64_t p = base + threadIdx.x;
    bool valid = p < nrows;
    int64_t k = -1;
    double v = 0.0;
    if (valid) {
      k = matrix_of(off, batch, p);
      double dv = d[p];
      v = fabs(dv);
      bool fin = isfinite(dv);
      if (p + 1 < off[k + 1]) {
        double ev = e[p];
        v = fmax(v, fabs(ev));
        fin = fin && isfinite(ev);
      }
      if (!fin) {
        set_status(st, TDE_ENONFINITE);
        v = 0.0;
      }
    }
    // warp-aggregate when every lane of the warp sees the same matrix
    int64_t k0 = __shfl_sync(0xffffffffu, k, 0);
    bool uniform = __all_sync(0xffffffffu, !valid || k == k0);
    if (uniform) {
      double r = v;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
      if ((threadIdx.x & 31) == 0 && k0 >= 0)
        atomicMax(&sigma_bits[k0], (unsigned long long)__double_as_longlong(r));
    } else if (valid) {
      atomicMax(&sigma_bits[k], (unsigned long long)__double_as_longlong(v));
    }
  }
}

__device__ __forceinline__ int scale_exponent(unsigned long long bits) {
  double s = __longlong_as_double((long long)bits);
  if (!(s > 0.0) || !isfinite(s)) return 0;
  return ilogb(s);
}

__global__ void k_scale(const int64_t* __restrict__ off, int64_t batch, int64_t nrows,
                        const double* __restrict__ d, const double* __restrict__ e,
                        const unsigned long long* __restrict__ sigma_bits, double* ds,
                        double* es) {
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < nrows;
       p += int64_t(gridDim.x) * blockDim.x) {
    int64_t k = matrix_of(off, batch, p);
    int ex = scale_exponent(sigma_bits[k]);
    double dp = ldexp(d[p], -ex);
    ds[p] = dp;
    double ep = 0.0;
    if (p + 1 < off[k + 1]) {
      ep = ldexp(e[p], -ex);
      double dq = ldexp(d[p + 1], -ex);
      if (fabs(ep) <= kEps * sqrt(fabs(dp)) * sqrt(fabs(dq))) ep = 0.0;
    }
    es[p] = ep;
  }
}

void launch_scale(const Plan& plan, const Workspace& ws, const int64_t* off, const double* d,
                  const double* e, cudaStream_t s) {
  if (plan.nrows == 0) return;
  int grid = int(std::min<int64_t>((plan.nrows + 255) / 256, 148 * 8));
  prof_begin(kKScale, s);
  k_sigma<<<grid, 256, 0, s>>>(off, plan.batch, plan.nrows, d, e, ws.sigma_bits, ws.status);
  k_scale<<<grid, 256, 0, s>>>(off, plan.batch, plan.nrows, d, e, ws.sigma_bits, ws.ds, ws.es);
  prof_end(kKScale, s);
  g_launches += 2;
}

}  // namespace tde
