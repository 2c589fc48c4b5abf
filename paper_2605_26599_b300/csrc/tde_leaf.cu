// Leaf solver (Algorithm 1, leaf branch; Sec. 4.1 "solves leaf subproblems,
// extracts only the first and last eigenvector rows"; Sec. 4.2 leaf DSTEQR('I')
// keeping two rows).
//
// Each leaf is a torn diagonal block (Eq. dc-split: the diagonal entries next to
// a cut are reduced by |beta|) of order m <= 64.  It is diagonalised by implicit
// symmetric tridiagonal QR with a Wilkinson shift: every step chases a bulge from
// the top of the unreduced block to its bottom with plane rotations G_i acting on
// rows/columns (i, i+1) as T <- G_i^T T G_i.  The eigenvector matrix is
// Q = G_1 G_2 ..., and by the selected-row lemma (Lemma "selected-row
// multiplication") its first and last rows are obtained by applying the same
// rotations to e_1^T and e_m^T only -- the leaf never forms Q.
// One thread owns one leaf (warps hold one to 32 leaves, see k_leaves); the
// outputs are the eigenvalues in ascending order with the matching first-row (blo)
// and last-row (bhi) entries.
#include <algorithm>

#include "tde_internal.cuh"

namespace tde {

// Implicit QR on a[0..m), b[0..m-1) (b[i] couples i and i+1), tracking the
// first row r0 and last row r1 of the accumulated rotation product.
// Returns false if an unreduced block needed more than 40 steps per row; adds the
// number of plane rotations applied to *rot.
// Kept out of line so that every kernel runs one compiled body: the requested-row
// leaves (k_sel_leaves) rely on reproducing the rotations of k_leaves bit for bit.
__device__ __noinline__ bool leaf_qr_two_rows(int m, double* a, double* b, double* r0, double* r1,
                                              unsigned* rot) {
  int hi = m - 1;
  int steps = 0;
  const int max_steps = 40 * m;
  while (hi > 0) {
    // unreduced block [lo, hi]: walk up while the coupling is not negligible
    int lo = hi;
    while (lo > 0) {
      double c = b[lo - 1];
      if (fabs(c) <= kEps * (fabs(a[lo - 1]) + fabs(a[lo]))) {
        b[lo - 1] = 0.0;
        break;
      }
      --lo;
    }
    if (lo == hi) {  // a[hi] has converged
      --hi;
      continue;
    }
    if (++steps > max_steps) return false;
    // Wilkinson shift: eigenvalue of the trailing 2x2 closer to a[hi]
    double bh = b[hi - 1];
    double half = 0.5 * (a[hi - 1] - a[hi]);
    double root = sqrt(half * half + bh * bh);
    double mu = a[hi] - bh * bh / (half + (half >= 0.0 ? root : -root));
    if (!isfinite(mu)) mu = a[hi];
    // first rotation from the first column of T - mu I, then chase the bulge.  The
    // entries one rotation hands to the next (the new a[i+1], b[i+1] and the tracked
    // rows' entries at column i+1) stay in registers: only entries the chase has not
    // touched yet are loaded, so the chain of rotations never waits on a local-memory
    // round trip.
    double ai = a[lo], bi = b[lo], p0 = r0[lo], p1 = r1[lo];
    double x = ai - mu, y = bi;
    *rot += unsigned(hi - lo);
    for (int i = lo; i < hi; ++i) {
      double c, s, r;
      leaf_givens(x, y, c, s, r);
      if (i > lo) b[i - 1] = r;  // the bulge is annihilated into the coupling
      const double aj = a[i + 1], q0 = r0[i + 1], q1 = r1[i + 1];
      double na, naj, nb;
      leaf_rotate(c, s, ai, aj, bi, na, naj, nb);
      a[i] = na;
      ai = naj;
      if (i + 1 < hi) {
        const double bn = b[i + 1];
        y = s * bn;  // new bulge at (i, i+2)
        bi = c * bn;
        x = nb;
      } else {
        b[i] = nb;
      }
      // Q <- Q G_i on columns (i, i+1) for the two tracked rows
      r0[i] = fma(c, p0, s * q0);
      p0 = fma(c, q0, -(s * p0));
      r1[i] = fma(c, p1, s * q1);
      p1 = fma(c, q1, -(s * p1));
    }
    a[hi] = ai;
    r0[hi] = p0;
    r1[hi] = p1;
  }
  return true;
}

// One leaf per lane of the first `per` lanes of each one-warp block.  A leaf's QR is
// a chain of dependent FP64 operations, and an FP64 warp instruction occupies the
// SM's FP64 unit for the whole warp however few lanes are active, so the host picks
// `per` to put few warps on each SM: few leaves (n = 2048, leaf 32: 64 leaves) get
// one leaf per warp, each warp alone on its SM; many leaves share warps, up to 32.
__global__ void __launch_bounds__(32) k_leaves(const Leaf* __restrict__ leaves, int64_t nleaves,
                                               int per, const double* __restrict__ ds,
                                               const double* __restrict__ es,
                                               const unsigned long long* __restrict__ sigma_bits,
                                               double* LAM, double* BLO, double* BHI, double* out,
                                               Status* st) {
  const int lane = threadIdx.x & 31;
  for (int64_t w = blockIdx.x; w * per < nleaves; w += gridDim.x) {
    const int64_t t = w * per + lane;
    if (lane >= per || t >= nleaves) continue;
    const Leaf lf = leaves[t];
    const int m = lf.hi - lf.lo;
    double a[kMaxLeaf], b[kMaxLeaf], r0[kMaxLeaf], r1[kMaxLeaf];
    for (int j = 0; j < m; ++j) {
      a[j] = ds[lf.lo + j];
      b[j] = (j + 1 < m) ? es[lf.lo + j] : 0.0;
      r0[j] = (j == 0) ? 1.0 : 0.0;
      r1[j] = (j == m - 1) ? 1.0 : 0.0;
    }
    // Cuppen tearing (Eq. 1): T = diag(T_L, T_R) + |beta| u u^T, u = e_last + sgn(beta) e_first
    if (lf.flags & 1) a[0] -= fabs(es[lf.lo - 1]);
    if (lf.flags & 2) a[m - 1] -= fabs(es[lf.hi - 1]);
    unsigned rot = 0;
    if (!leaf_qr_two_rows(m, a, b, r0, r1, &rot)) set_status(st, TDE_ENOCONV);
    work_add(st, kWorkLeafRotations, rot);
    // ascending order, rows follow their eigenvalue (insertion sort, m <= 64)
    for (int j = 1; j < m; ++j) {
      double v = a[j], p = r0[j], q = r1[j];
      int i = j - 1;
      while (i >= 0 && a[i] > v) {
        a[i + 1] = a[i];
        r0[i + 1] = r0[i];
        r1[i + 1] = r1[i];
        --i;
      }
      a[i + 1] = v;
      r0[i + 1] = p;
      r1[i + 1] = q;
    }
    if (lf.flags & 4) {
      double s = __longlong_as_double((long long)sigma_bits[lf.mat]);
      int ex = (s > 0.0 && isfinite(s)) ? ilogb(s) : 0;
      for (int j = 0; j < m; ++j) out[lf.lo + j] = ldexp(a[j], ex);
    } else {
      for (int j = 0; j < m; ++j) {
        LAM[lf.lo + j] = a[j];
        BLO[lf.lo + j] = r0[j];
        BHI[lf.lo + j] = r1[j];
      }
    }
  }
}

void launch_leaves_to(const Plan& plan, const Workspace& ws, double* lambda, cudaStream_t s,
                      LevelState out) {
  if (plan.nleaves == 0) return;
  // leaves per warp: about two warps per SM before warps take more than one leaf
  const int64_t per64 = (plan.nleaves + 2 * 148 - 1) / (2 * 148);
  const int per = int(std::min<int64_t>(32, std::max<int64_t>(1, per64)));
  int64_t grid = (plan.nleaves + per - 1) / per;
  if (grid > 148 * 64) grid = 148 * 64;
  prof_begin(kKLeaves, s);
  k_leaves<<<int(grid), 32, 0, s>>>(ws.leaves, plan.nleaves, per, ws.ds, ws.es, ws.sigma_bits,
                                    out.lam, out.blo, out.bhi, lambda, ws.status);
  prof_end(kKLeaves, s);
  g_launches += 1;
}

// Requested rows at the leaves (Algorithm 1, leaf branch: "return the requested
// rows of the leaf eigenvector matrix").  For each distinct requested row r the
// leaf holding it is diagonalised again by the same QR with the tracked rows
// e_r and e_last: the rotations depend on the leaf's (d, e) only, so they -- and
// the ascending sort -- are those of k_leaves, and the tracked row is row r of
// the very Q whose first and last rows k_leaves stored.
__global__ void k_sel_leaves(SelArgs sa, const Leaf* __restrict__ leaves, int64_t nleaves,
                             const double* __restrict__ ds, const double* __restrict__ es) {
  const int nu = *sa.nu;
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nu; u += gridDim.x * blockDim.x) {
    const int r = sa.U[u];
    int64_t lo_t = 0, hi_t = nleaves;  // last leaf with lo <= r
    while (hi_t - lo_t > 1) {
      const int64_t md = (lo_t + hi_t) >> 1;
      if (leaves[md].lo <= r)
        lo_t = md;
      else
        hi_t = md;
    }
    const Leaf lf = leaves[lo_t];
    const int m = lf.hi - lf.lo;
    double a[kMaxLeaf], b[kMaxLeaf], r0[kMaxLeaf], r1[kMaxLeaf];
    for (int j = 0; j < m; ++j) {
      a[j] = ds[lf.lo + j];
      b[j] = (j + 1 < m) ? es[lf.lo + j] : 0.0;
      r0[j] = (j == r - lf.lo) ? 1.0 : 0.0;
      r1[j] = (j == m - 1) ? 1.0 : 0.0;
    }
    if (lf.flags & 1) a[0] -= fabs(es[lf.lo - 1]);
    if (lf.flags & 2) a[m - 1] -= fabs(es[lf.hi - 1]);
    unsigned rot = 0;
    leaf_qr_two_rows(m, a, b, r0, r1, &rot);  // a failure is reported by k_leaves
    for (int j = 1; j < m; ++j) {
      double v = a[j], p = r0[j], q = r1[j];
      int i = j - 1;
      while (i >= 0 && a[i] > v) {
        a[i + 1] = a[i];
        r0[i + 1] = r0[i];
        r1[i + 1] = r1[i];
        --i;
      }
      a[i + 1] = v;
      r0[i + 1] = p;
      r1[i + 1] = q;
    }
    double* x = sa.X + int64_t(u) * sa.N + lf.lo;
    for (int j = 0; j < m; ++j) x[j] = r0[j];
  }
}

void launch_sel_leaves(const Plan& plan, const Workspace& ws, const SelArgs& sa, cudaStream_t s) {
  if (plan.nleaves == 0 || sa.nsel == 0) return;
  const int grid = (sa.nsel + 63) / 64;
  k_sel_leaves<<<grid, 64, 0, s>>>(sa, ws.leaves, plan.nleaves, ws.ds, ws.es);
  g_launches += 1;
}

void launch_leaves(const Plan& plan, const Workspace& ws, double* lambda, cudaStream_t s) {
  launch_leaves_to(plan, ws, lambda, s, LevelState{ws.LAM, ws.BLO, ws.BHI});
}

}  // namespace tde
