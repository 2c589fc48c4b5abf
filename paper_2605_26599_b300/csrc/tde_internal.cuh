// Internal declarations of the boundary-row D&C solver (sm_103a).
//
// Data layout in device memory (one workspace, sections 256-byte aligned; N = the
// packed number of rows of all matrices):
//   scaled inputs         ds, es                     2N doubles
//   boundary-row state    LAM, BLO, BHI              3N doubles (Eq. boundary-state:
//                         per node, eigenvalues ascending with the first / last
//                         eigenvector row entry of each column)
//   merge problem         D, Z, RLO, RHI             4N doubles (Eq. merge-problem,
//                         sorted by D; RLO / RHI are the rows of diag(Q_L, Q_R))
//   deflated problem      AD, AZ, ALO, AHI           4N doubles (active poles first,
//                         then the deflated eigenvalues of the merge, both sorted)
//   compact roots         TAU (N doubles) + ORG (N int32): lambda_j = AD[ORG] + TAU
//                         (Sec. 4.1 compact root representation)
//   maps                  ROOTMAP, ROOTMAP2, SURV (N int32), PFLAG, RFLAG (N bytes)
//   sort scratch          KEYA, KEYB (N uint64), IDXA, IDXB (N int32)
//   plan                  merge and leaf descriptors, per-step merge state
// Aliases once a buffer is dead within a level: LAMA (roots) -> D, ZHAT -> Z,
// parent rows of active columns -> RLO / RHI, origin poles D_org(j) -> KEYA.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tde.h"

namespace tde {

constexpr int kMaxLeaf = 64;
constexpr int kMaxSteps = 40;
constexpr double kEps = 2.220446049250313e-16;  // DBL_EPSILON = 2^-52

// One merge of the split tree: children [lo, mid) and [mid, hi) (global rows).
struct Merge {
  int32_t lo, mid, hi;
  int32_t info;  // bits 0..28: matrix index; bit 29: first node of its tree level (left
                 // spine); bit 30: last node of its level (right spine); bit 31: root merge
};
// One leaf [lo, hi) of matrix `mat`.  flags: 1 = torn at lo (d[lo] -= |e[lo-1]|),
// 2 = torn at hi (d[hi-1] -= |e[hi-1]|), 4 = the leaf is the whole matrix.
struct Leaf {
  int32_t lo, hi, mat, flags;
};
// Per-merge state of the current step.
struct MState {
  int32_t K;     // active rank after deflation
  int32_t base;  // first index of this merge's roots in its root list
  double rho;    // rho' = 2 |beta|
  double rhoinv; // 1 / rho
  double zsq;    // sum of active z^2
  int32_t big;   // 1: roots in the warp-per-root list (K >= warp_min_k)
  int32_t surv;  // survivors of the negligible-z test (active + rotation-deflated)
  double shift;  // the active poles' single-precision copies hold D - shift (their midrange)
};

// Launch-shape parameters chosen per call (tde_set_tuning; the Python autotuner
// searches them together with the leaf order):
//   warp_min_k      merges whose active rank K reaches this are solved one warp per
//                   root (per pole for z-hat); smaller ones one thread per root
//   small_list_min  below this many small-K roots in a step the thread-per-root
//                   kernels would leave SMs idle, so the warp kernels take them too
struct Tuning {
  int32_t warp_min_k = 256;
  int32_t small_list_min = 148 * 4 * 32;
  int32_t multipole_min_k = 1024;  // block expansions for merges with K >= this
};
Tuning& thread_tuning();

constexpr uint32_t kRootBit = 0x80000000u;
// Rows a merge's ancestors need (Algorithm 1: sigma_v holds exactly the rows demanded
// by ancestors): the left spine of a tree feeds only bhi upwards (its blo would
// only ever reach the root's blo, which nothing reads), the right spine only blo.
constexpr uint32_t kRightSpineBit = 0x40000000u;
constexpr uint32_t kLeftSpineBit = 0x20000000u;
constexpr uint32_t kMatMask = 0x1fffffffu;

// Work counters accumulated on the device by every call (reset per call):
enum WorkCounter {
  kWorkSecularPairs = 0,  // pole terms summed exactly in FP64 sweeps (K per sweep without
                          // the block expansion)
  kWorkSecularSweeps,     // sum over roots of the number of pole sweeps
  kWorkLownerPairs,       // Löwner factors multiplied directly (K^2 per non-root merge
                          // without the block expansion)
  kWorkRowsPairs,         // (pole, root) terms of the row sums summed exactly (K^2 per
                          // non-root merge without the block expansion)
  kWorkRoots,             // roots solved
  kWorkDeflated,          // eigenvalues deflated (small z or rotation)
  kWorkRotations,         // close-pole rotations
  kWorkLeafRotations,     // plane rotations in the leaf QR sweeps
  kWorkSorts,             // merges whose rotated deflated list needed a sort
  kWorkSortedEntries,     // entries in those sorts
  kWorkSecular32Pairs,    // sum over roots of K x (number of single-precision pole sweeps)
  kWorkSecular32Sweeps,   // sum over roots of the number of single-precision pole sweeps
  kWorkSelRowPairs,       // requested-row updates: (pole, root, requested row) triples
  kWorkSelSweepPairs,     // requested-row updates: (pole, root) pairs per sweep of up to four rows
  kWorkSecularFarBlocks,  // pole blocks taken through their series in FP64 sweeps
  kWorkRowsFarSeries,     // series evaluated for the row sums (two or three per far block:
                          // the norm and the rows the merge needs)
  kWorkLownerFarBlocks,   // pair blocks taken through their series in the Löwner products
  kWorkSecularSeriesOps,  // FP64 operations of those series evaluations (each one's FP64
  kWorkLownerSeriesOps,   // Horner head, its distance, reciprocal, argument and
  kWorkRowsSeriesOps,     // accumulation), per stage
  kNumWork
};

// A forest's small-K root list is ordered by descending K (bins of K, the last bin
// holding every K >= kOrderBins - 1), so that the roots held by the groups of one
// warp at any time have nearly equal K and their sweeps end together.
constexpr int kOrderBins = 512;

struct Status {
  int32_t info;
  uint32_t claim_next;  // next entry of a dynamically claimed work list (see claim_begin)
  uint32_t claim_done;  // blocks of the claiming launch that have finished
  int32_t pad[29];
  uint32_t root_count[kMaxSteps];      // roots of small-K merges per step
  uint32_t root_count_big[kMaxSteps];  // roots of merges with K >= warp_min_k
  unsigned long long work[kNumWork];
  uint32_t order_hist[kOrderBins];    // forests: roots of the step's small-K merges per bin of K
  uint32_t order_cursor[kOrderBins];  // next list entry of each bin (descending K)
};

// Kernel classes timed by the optional per-launch event profiler.
enum KernelId { kKPlan = 0, kKScale, kKLeaves, kKForm, kKDeflate, kKSecular, kKLowner, kKRows,
                kKPlace, kKSel, kKSelRows, kNumKernelIds };
void prof_begin(int id, cudaStream_t s);
void prof_end(int id, cudaStream_t s);

// Warp-aggregated add to a device work counter (safe under a partial warp).
__device__ __forceinline__ void work_add(Status* st, int which, unsigned v) {
  const unsigned mask = __activemask();
  const unsigned x = __reduce_add_sync(mask, v);
  if ((threadIdx.x & 31) == unsigned(__ffs(mask) - 1) && x)
    atomicAdd(&st->work[which], (unsigned long long)x);
}

struct Workspace {
  Status* status;
  unsigned long long* sigma_bits;  // per matrix, max |T| as non-negative double bits
  int64_t* offsets;                // device offsets (single-matrix calls write here)
  double *ds, *es;
  double *LAM, *BLO, *BHI;
  double *D, *Z, *RLO, *RHI;
  double *AD, *AZ, *ALO, *AHI;
  double* TAU;
  int32_t *ORG, *ROOTMAP, *ROOTMAP2, *SURV;
  int32_t* ZPOS;    // negligible-z deflated positions of a merge (deflation step 5)
  int32_t* OUTIDX;  // per merge position: index of its deflated entry in [active | deflated]
  int32_t* ACTMAP;  // per survivor: index of the active pole its run ends in
  int32_t* KEEPIDX; // per rotation-deflated position: active index of its run's kept pole
  uint8_t *PFLAG, *RFLAG;
  unsigned long long *KEYA, *KEYB;
  int32_t *IDXA, *IDXB;
  Merge* merges;   // all steps back to back
  Leaf* leaves;
  MState* mstate;  // cmax entries, reused every step
  int32_t* pfx;    // (steps + 1) x (batch + 1) plan prefix counts
  size_t bytes;
};

// Host-side plan: depends only on the packing and the leaf order.
struct Plan {
  int64_t batch = 0;
  int64_t nrows = 0;
  int32_t leaf = 32;
  int32_t steps = 0;
  int64_t nleaves = 0;
  int64_t nmerges = 0;
  int64_t cmax = 0;
  int64_t step_count[kMaxSteps] = {0};
  int64_t step_maxsize[kMaxSteps] = {0};  // largest merge order (K0) of the step
  int64_t step_base[kMaxSteps] = {0};
  bool step_has_nonroot[kMaxSteps] = {false};
  Tuning tune;
};

int build_plan(int64_t batch, const int64_t* offsets_host, int32_t leaf, Plan* plan);
size_t carve_workspace(const Plan& plan, void* base, Workspace* ws);
int run_solver(const Plan& plan, const Workspace& ws, const int64_t* offsets_dev,
               const double* d, const double* e, double* lambda, cudaStream_t stream);

// ---- device helpers -------------------------------------------------------

// Dynamic work claiming for kernels whose items differ in cost: each warp takes
// the next item index from st->claim_next; the last block to finish resets the
// counter, so consecutive launches on one stream (and graph replays) start at 0.
// At most one claiming kernel may run at a time per workspace.
__device__ __forceinline__ uint32_t claim_next_item(Status* st) {
  uint32_t r = 0;
  if ((threadIdx.x & 31) == 0) r = atomicAdd(&st->claim_next, 1u);
  return __shfl_sync(0xffffffffu, r, 0);
}
__device__ __forceinline__ void claim_finish_block(Status* st) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&st->claim_done, 1u) == gridDim.x - 1) {
      st->claim_next = 0;
      st->claim_done = 0;
      __threadfence();
    }
  }
}

__device__ __forceinline__ void set_status(Status* st, int code) {
  atomicCAS(&st->info, 0, code);
}

// Merge of a step containing row p: the last merge with lo <= p (merges of a step
// are ordered by lo).
__device__ __forceinline__ int64_t find_merge(const Merge* M, int64_t cnt, int64_t p) {
  int64_t lo = 0, hi = cnt;  // M[lo].lo <= p
  while (hi - lo > 1) {
    int64_t m = (lo + hi) >> 1;
    if (M[m].lo <= p)
      lo = m;
    else
      hi = m;
  }
  return lo;
}

// number of entries of the ascending array a[0..n) strictly below x
__device__ __forceinline__ int count_less(const double* a, int n, double x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int m = (lo + hi) >> 1;
    if (a[m] < x)
      lo = m + 1;
    else
      hi = m;
  }
  return lo;
}
// number of entries of the ascending array a[0..n) less than or equal to x
__device__ __forceinline__ int count_leq(const double* a, int n, double x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int m = (lo + hi) >> 1;
    if (a[m] <= x)
      lo = m + 1;
    else
      hi = m;
  }
  return lo;
}

// Levels of a matrix of order n with leaves of order <= leaf: the smallest L with
// ceil(n / 2^L) <= leaf (node (h, i) covers [floor(i n / 2^h), floor((i+1) n / 2^h))),
// but never so deep that a leaf would be empty (2^L <= n); with leaf = 1 and n not
// a power of two some leaves therefore hold two rows.
__host__ __device__ inline int levels_of(int64_t n, int leaf) {
  int L = 0;
  while (((n + (int64_t(1) << L) - 1) >> L) > leaf && (int64_t(2) << L) <= n) ++L;
  return L;
}

// Order-preserving map of a double to an unsigned key.
__device__ __forceinline__ unsigned long long order_key(double x) {
  unsigned long long b = __double_as_longlong(x);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_value(unsigned long long k) {
  unsigned long long b = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double(b);
}

__device__ __forceinline__ double shfl_up_d(double v, int o) {
  return __shfl_up_sync(0xffffffffu, v, o);
}

// Block-wide exclusive prefix sum of one int per thread; returns the total in
// *total.  All threads of the block must call it.  sm: NT/32 ints.
template <int NT>
__device__ __forceinline__ int block_excl_scan(int v, int* sm, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sm[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = (lane < NT / 32) ? sm[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NT / 32) sm[lane] = w;
  }
  __syncthreads();
  int before = (warp > 0) ? sm[warp - 1] : 0;
  *total = sm[NT / 32 - 1];
  __syncthreads();
  return before + x - v;
}

// Block-wide max / sum of one double per thread, returned to every thread.  The
// warp partials are combined by warp 0 alone and broadcast: FP64 work done by every
// thread of a large block would cost the SM's FP64 pipe once per thread.  All
// threads must call them.  sm: NT/32 doubles.
template <int NT>
__device__ __forceinline__ double block_max(double v, double* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double x = sm[lane < NT / 32 ? lane : 0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (lane == 0) sm[0] = x;
  }
  __syncthreads();
  const double r = sm[0];
  __syncthreads();
  return r;
}

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double x = lane < NT / 32 ? sm[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sm[0] = x;
  }
  __syncthreads();
  const double r = sm[0];
  __syncthreads();
  return r;
}

// ---- launchers (defined in the .cu files) -----------------------------------
void launch_plan(const Plan& plan, const Workspace& ws, const int64_t* offsets_dev,
                 cudaStream_t s);
void launch_scale(const Plan& plan, const Workspace& ws, const int64_t* offsets_dev,
                  const double* d, const double* e, cudaStream_t s);
void launch_leaves(const Plan& plan, const Workspace& ws, double* lambda, cudaStream_t s);
// Boundary-row state (eigenvalues, first and last eigenvector rows) of one level.
struct LevelState {
  double *lam, *blo, *bhi;
};
// Requested rows of the eigenvector matrix (Algorithm 1 with a general row list
// sigma_v; tde_rows_sel.cu).  Row u of each array belongs to the distinct
// requested row U[u] and holds, over the columns of the node containing U[u] at
// the current level (the node's row range [lo, hi) indexes its columns too), the
// entries of that node's eigenvector row.
constexpr int kMaxSel = TDE_MAX_SEL_ROWS;  // requested rows per call
struct SelArgs {
  const int32_t* U;   // distinct requested rows, ascending; entries past *nu hold INT32_MAX
  const int32_t* nu;  // number of distinct rows (device)
  int32_t nsel;       // capacity of U (requests of the call)
  int64_t N;          // stride between the rows of X, XD, AX
  double* X;          // level state (children's rows in, parent's rows out)
  double* XD;         // rows of the merge problem, then of the active roots' columns
  double* AX;         // rows of the deflated problem (active columns, then deflated)
};
void launch_sel_prepare(const SelArgs& sa, const int64_t* rows, int64_t nrows_total, int32_t* U,
                        int32_t* nu, int32_t* MAP, Status* st, cudaStream_t s);
void launch_sel_leaves(const Plan& plan, const Workspace& ws, const SelArgs& sa, cudaStream_t s);
void launch_sel_form(const Plan& plan, const Workspace& ws, const SelArgs& sa, int step,
                     LevelState in, cudaStream_t s);
void launch_sel_deflate(const Plan& plan, const Workspace& ws, const SelArgs& sa, int step,
                        cudaStream_t s);
void launch_sel_rows(const Plan& plan, const Workspace& ws, const SelArgs& sa, int step,
                     cudaStream_t s);
void launch_sel_place(const Plan& plan, const Workspace& ws, const SelArgs& sa, int step,
                      cudaStream_t s);
// Dense symmetric front end (tde_dense.cu): tri_bytes of tridiagonal-solver
// workspace (at offset 0) followed by the reduction's buffers; the reduction copies
// A (leading dimension lda) into the workspace, reduces it and returns pointers to
// d and e (e with n entries, the last zero).
size_t dense_workspace(int64_t n, size_t tri_bytes);
int dense_reduce(int64_t n, const double* A, int64_t lda, void* ws, size_t tri_bytes, double** d_out,
                 double** e_out, cudaStream_t s);
void launch_sel_gather(const SelArgs& sa, const int32_t* MAP, int64_t nsel, int64_t n,
                       double* qrows, cudaStream_t s);

// One merge step: reads the children's state from `in` and writes the parents'
// state to `out` (in == out is allowed: a merge's children occupy its own rows).
// The step's two root-list counters (Status::root_count[step], root_count_big[step])
// must be zero on entry: the deflation appends the roots of every merge to them, so
// a caller that runs a step again first clears them.
// With recompute = true only the merge internals are rebuilt (no place): used by
// the adjoint, which also forces z-hat and rows at root merges.  With `sel` the
// requested eigenvector rows are carried through the step as well (z-hat and the
// row update then run at root merges too).
// Saved secular roots of one step (tau and D_org of every active root, at the
// rows of its merge): the adjoint checkpoints them in its forward pass and
// restores them when it rebuilds the step, instead of solving again.
struct RootsCheckpoint {
  const double* tau;
  const double* dorg;
};
void launch_step(const Plan& plan, const Workspace& ws, int step, double* lambda, cudaStream_t s,
                 LevelState in, LevelState out, bool recompute = false,
                 const SelArgs* sel = nullptr, double* rows_inu = nullptr,
                 const RootsCheckpoint* roots = nullptr);
void launch_form(const Plan& plan, const Workspace& ws, int step, LevelState in, cudaStream_t s);
// secular, Lowner and boundary-row kernels of one step; returns the launch count.
// rows_inu (optional) receives 1 / nu_j, the inverse norm of every active root's
// secular eigenvector, from the row kernels.
int launch_roots(const Plan& plan, const Workspace& ws, int step, const Merge* M, cudaStream_t s,
                 bool all_merges = false, double* rows_inu = nullptr,
                 const RootsCheckpoint* roots = nullptr);

// Reciprocal in about three FP64 fused multiply-adds: a hardware approximation r0
// of 1/x refined by the third-order (Householder) step for 1/x,
// r = r0 (1 + e + e^2) with e = 1 - x r0, i.e. the geometric series of
// 1 / (1 - e) truncated after the quadratic term; the relative error drops from
// |e| to about |e|^3 plus the final rounding.
__device__ __forceinline__ double rcp_refined(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, 1.0);
  const double ee = fma(e, e, e);
  return fma(r, ee, r);
}

// Reciprocal square root in about five FP64 operations: a hardware approximation
// y0 of x^(-1/2) refined by the third-order step y = y0 (1 + e/2 + 3 e^2/8) with
// e = 1 - x y0^2, the binomial series of (1 - e)^(-1/2) truncated after the
// quadratic term; the relative error drops from about |e|/2 to (5/16)|e|^3 plus the
// final rounding.  For finite x > 0 (callers keep 1 / sqrt(x) for anything else).
__device__ __forceinline__ double rsqrt_refined(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y * y, 1.0);
  return fma(y, e * fma(e, 0.375, 0.5), y);
}

// Plane rotation of the leaf QR sweeps: (c, s) = (x, y) / r with r = sqrt(x^2 + y^2),
// formed from r^2 (one fused multiply-add) and its refined reciprocal square root
// (c = x / r, s = y / r, r = r^2 / r) instead of an IEEE square root and division,
// whose dependent latencies (hundreds of cycles each on this part's FP64 units)
// would dominate the chain of a bulge chase.  The identity (1, 0, 0) when r^2 is
// zero or below the normal range, where both entries are negligible next to the
// scaled matrix (whose largest entry lies in [1, 2)).  Every leaf QR (the forward
// solver, the requested-row leaves and the adjoint's full-Q leaves) uses this one
// function, so all of them apply bitwise the same rotations.
__device__ __forceinline__ void leaf_givens(double x, double y, double& c, double& s, double& r) {
  const double r2 = fma(x, x, y * y);
  if (r2 >= 2.2250738585072014e-308) {  // DBL_MIN
    const double inv = rsqrt_refined(r2);
    c = x * inv;
    s = y * inv;
    r = r2 * inv;
  } else {
    c = 1.0;
    s = 0.0;
    r = 0.0;
  }
}

// Similarity T <- G^T T G of one bulge-chase rotation on the 2 x 2 block
// [[ai, bi], [bi, aj]] of the leaf tridiagonal: the new diagonal pair and coupling.
// Written with explicit fused multiply-adds so that every leaf QR (forward,
// requested rows, adjoint) rounds identically.
__device__ __forceinline__ void leaf_rotate(double c, double s, double ai, double aj, double bi,
                                            double& ai_out, double& aj_out, double& bi_out) {
  const double cc = c * c, ss = s * s, cs = c * s;
  const double t = 2.0 * (cs * bi);
  ai_out = fma(cc, ai, fma(ss, aj, t));
  aj_out = fma(ss, ai, fma(cc, aj, -t));
  bi_out = fma(cs, aj - ai, (cc - ss) * bi);
}

extern thread_local int64_t g_launches;

}  // namespace tde
