// Adjoint of the boundary-row D&C: d(loss)/d(d) and d(loss)/d(e) from the
// gradient of the loss with respect to the eigenvalues.
//
// Structure (a reverse sweep over the split tree, top-down):
//   1. forward recomputation with a checkpoint of the boundary-row state (lambda,
//      blo, bhi) at the input of every merge step and of the step's secular roots
//      (tau, D_org);
//   2. for every step from the top down: rebuild the step's merge internals from
//      its checkpoints (form, deflation, the saved roots, z-hat, rows at every
//      merge, root merges included), then pull the adjoints of the parents'
//      (lambda, blo, bhi) back through
//        - the ascending placement (a permutation),
//        - the secular eigen-decomposition A = diag(D) + rho' z z^T = Y L Y^T,
//          whose outputs are the roots L and the boundary rows blo = Y^T RLO,
//          bhi = Y^T RHI: the adjoint of a symmetric eigen-decomposition,
//          A_bar = Y (L_bar + F o (Y^T Y_bar)) Y^T, F_jk = 1/(l_k - l_j),
//          Y^T Y_bar = W with W_jk = blo_j blo_bar_k + bhi_j bhi_bar_k (rank two),
//          evaluated in O(K^2) through the Cauchy form of the secular
//          eigenvectors y_sj = zhat_s / (nu_j (D_s - l_j)):
//            D_bar_s = A_bar_ss = sum_j lbar_j y_sj^2 + zhat_s^2 sum_j g_j / (D_s - l_j),
//            g_j = -sum_{k != j} (W_jk - W_kj) / (nu_j nu_k (l_j - l_k)^2)
//          (partial fractions of 1 / ((D_s - l_j)(D_s - l_k))), and with
//          c = Y^T z, h_j = sum_{k != j} (W_jk - W_kj) c_k / (l_k - l_j):
//            z_bar = rho' (A_bar + A_bar^T) z = rho' Y (2 lbar o c + h),
//            rho'_bar = z^T A_bar z = sum_j (lbar_j c_j^2 + c_j h_j / 2),
//            RLO_bar = Y blo_bar, RHI_bar = Y bhi_bar;
//          root differences are formed as (D_org(j) - D_org(k)) + (tau_j - tau_k),
//        - the deflation (negligible z: pass-through; close-pole rotation runs:
//          the prefix-sum formulas reversed run by run).  A rotation drops the
//          coupling kappa_m = u_keep^T diag(D) u_def,m between a deflated direction
//          and its run's kept pole; kappa is at most tol, so the eigenvalues do not
//          see it to first order, but d kappa / dD is O(1) and the eigenvectors
//          (hence the propagated rows) do: the first-order mixing
//          dy_j = f_m kappa y_aj / (l_j - v_m), df_m = sum_k y_k kappa y_ak / (v_m - l_k)
//          gives kappa_bar_m = sum_j y_aj [(blo_bar_j r_m + bhi_bar_j r'_m)
//          - (blo_bar_m blo_j + bhi_bar_m bhi_j)] / (l_j - v_m), pulled back
//          through kappa_m = z_m sqrt(W_{m-1}) (c_{m-1} - D_m) / sqrt(W_m W_L)
//          (W prefix sums of z^2 over the run, c the running weighted mean); its
//          terms proportional to (c - D) are of order tol and are dropped.
//          Couplings between two deflated directions of one run are not modelled.
//        - the formation of D, z, RLO, RHI from the children (a permutation; z
//          carries 1/sqrt(2) and the sign of the cut coupling beta; rho' = 2|beta|);
//   3. at the leaves: the standard adjoint of a symmetric eigen-decomposition,
//      A_bar = Q (diag(lambda_bar) + F o (Q^T Q_bar)) Q^T with F_jk = 1/(l_k - l_j),
//      Q_bar nonzero only in the first and last rows, then d_bar_i = A_bar_ii,
//      e_bar_i = 2 A_bar_i,i+1, and the tearing d_cut -= |beta| gives
//      e_bar_cut -= sgn(beta) (d_bar of the two torn diagonal entries).
// Deflation decisions, the tree and the scaling are constants of the
// differentiation (eigenvalue derivatives are scale invariant).
// Memory.  Reversing merge step s needs the boundary-row state at its input
// (level s).  Two layouts, chosen from the caller's workspace size:
//   * slots (the default, O(n)): S checkpoint slots of one level state each
//     (3 n doubles; S = 4 by default, at least 1).  Levels are reversed by
//     bisection: to reverse steps [lo, hi) from the state of level lo, the state
//     of level mid = lo + ceil((hi - lo) / 2) is recomputed forward into the next
//     slot, [mid, hi) is reversed from it, then [lo, mid); with no slot left the
//     steps of a segment are reversed one by one, each from a forward
//     recomputation into the scratch level.  The first forward pass already stores
//     the levels of the schedule's first descent (0, L/2, 3L/4, ...), so the costly
//     top steps are never recomputed.  Each reversed step solves its secular roots
//     again while rebuilding its merge;
//   * levels (when the workspace holds them): the state at every level and every
//     step's roots (tau, D_org) are checkpointed in the forward pass (5 n doubles
//     per step, O(n log n)); the rebuild restores the roots instead of solving.
// Both give the same gradient.  Every other buffer is O(n).
#include <algorithm>

#include "tde_internal.cuh"

namespace tde {

constexpr int kMaxBwdLeaf = 32;

struct AdjWorkspace {
  Workspace fw;
  int slots;                           // checkpoint slots (levels layout: one per step)
  bool levels;                         // every level's state and roots checkpointed
  double* CK;                          // slots x 3 x N level states
  double* CR;                          // levels layout: steps x 2 x N saved roots (tau, D_org)
  double *GL, *GBL, *GBH;              // adjoint of the current level's state
  double *ALB, *ABL, *ABH;             // adjoints of a merge's [active | deflated] outputs
  double *RLT, *RAL, *RBE, *RGA, *RINU, *RC;  // per active root: g, h, scratch, 1/nu, 2 lbar c + h
  double *PDB, *PZB, *PRLB, *PRHB;     // adjoints of the active poles
  double *MDB, *MZB, *MRLB, *MRHB;     // adjoints at the sorted merge positions
  double* RHOBAR;                      // per merge of a step: adjoint of rho'
  double* KBAR;                        // per rotation-deflated position: adjoint of its coupling
  double* LAMOUT;                      // eigenvalues when the caller passes none
  size_t bytes;
};

static size_t align_up_adj(size_t x) { return (x + 255) & ~size_t(255); }

constexpr int kDefaultSlots = 4;

// Workspace of the adjoint: the forward workspace, the checkpoints (levels layout
// when levels is true, else `slots` level states), then the O(n) adjoint arrays.
size_t carve_adjoint(const Plan& plan, void* base, AdjWorkspace* aw, bool levels, int slots) {
  AdjWorkspace w{};
  size_t off = carve_workspace(plan, base, &w.fw);
  off = align_up_adj(off);
  const size_t N = size_t(std::max<int64_t>(plan.nrows, 1));
  const int steps = std::max(plan.steps, 1);
  w.levels = levels;
  w.slots = levels ? steps : std::max(1, std::min(slots, steps));
  char* b = static_cast<char*>(base);
  auto take = [&](size_t bytes) -> double* {
    double* p = b ? reinterpret_cast<double*>(b + off) : nullptr;
    off += align_up_adj(bytes);
    return p;
  };
  w.CK = take(8 * N * 3 * size_t(w.slots));
  w.CR = levels ? take(8 * N * 2 * size_t(steps)) : nullptr;
  double** arrs[] = {&w.GL,  &w.GBL, &w.GBH, &w.ALB,  &w.ABL, &w.ABH, &w.RLT,  &w.RAL,
                     &w.RBE, &w.RGA, &w.RINU, &w.RC,  &w.PDB, &w.PZB, &w.PRLB, &w.PRHB,
                     &w.MDB, &w.MZB, &w.MRLB, &w.MRHB, &w.KBAR, &w.LAMOUT};
  for (double** p : arrs) *p = take(8 * N);
  w.RHOBAR = take(8 * size_t(std::max<int64_t>(plan.cmax, 1)));
  w.bytes = off;
  if (aw) *aw = w;
  return off;
}


struct AdjArgs {
  const Merge* M;
  int64_t cnt;
  int64_t nrows;
  const MState* ms;
  const int32_t *ROOTMAP, *ROOTMAP2;
  const uint32_t *count, *count2;
  const double *LAMA, *AD, *AZ, *ALO, *AHI, *TAU, *DORG, *ZHAT, *ROWLO, *ROWHI;
  const double *D, *Z, *RLO, *RHI;  // the merge problem (restored before the deflation adjoint)
  const double* es;
  const int32_t *SURV, *OUTIDX, *ACTMAP, *KEEPIDX;
  const uint8_t *PFLAG, *RFLAG;
  LevelState in;  // children's state (checkpoint of this step)
  AdjWorkspace w;
  double* grad_e;
};

// parents' adjoints (ascending order) -> [active | deflated] order of each merge
__global__ void k_adj_place(AdjArgs a) {
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < a.nrows;
       p += int64_t(gridDim.x) * blockDim.x) {
    const int64_t g = find_merge(a.M, a.cnt, p);
    const Merge m = a.M[g];
    if (p < m.lo || p >= m.hi) continue;
    const int K = a.ms[g].K, lo = m.lo, F = (m.hi - m.lo) - K, local = int(p - lo);
    int rank;
    if (local < K)
      rank = local + count_less(a.AD + lo + K, F, a.LAMA[p]);
    else
      rank = (local - K) + count_leq(a.LAMA + lo, K, a.AD[p]);
    const int src = lo + rank;
    a.w.ALB[p] = a.w.GL[src];
    a.w.ABL[p] = a.w.GBL[src];
    a.w.ABH[p] = a.w.GBH[src];
  }
}

__device__ __forceinline__ double adj_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per active root j, a sweep over the other roots k of its merge: g_j and h_j,
// and the merge's rho' adjoint sum_j (lbar_j c_j^2 + c_j h_j / 2).  1 / nu_j comes
// from the recomputed row kernels; c_j = zhat^T y_j = (1 / nu_j) sum_s zhat_s^2 /
// (D_s - l_j) = -1 / (rho' nu_j), because the roots solve the secular equation
// of zhat exactly (that is how zhat is built).  Per pair: the root difference,
// a refined reciprocal and W_jk - W_kj; the factors of j are applied after the
// sum.  Lane 0 also stores 2 lbar_j c_j + h_j, the z_bar coefficient of root j.
// G lanes per root (an aligned power of two; G = 32: a warp), over the small-K
// root list (big = 0) or the large-K one (big = 1).
template <int G>
__device__ __forceinline__ double adj_group_sum(double v, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

template <int G>
__global__ void __launch_bounds__(128) k_adj_pairs(AdjArgs a, int big) {
  const uint32_t total = big ? *a.count2 : *a.count;
  const int lane = threadIdx.x & 31, gl = lane & (G - 1);
  const unsigned mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const uint32_t grp = (blockIdx.x * blockDim.x + threadIdx.x) / G;
  const uint32_t ngrp = (gridDim.x * blockDim.x) / G;
  for (uint32_t r = grp; r < total; r += ngrp) {
    const int g = big ? a.ROOTMAP2[r] : a.ROOTMAP[r];
    const MState ms = a.ms[g];
    const int K = ms.K, j = int(r) - ms.base, lo = a.M[g].lo;
    const double oj = a.DORG[lo + j], tj = a.TAU[lo + j];
    const double bl = a.ROWLO[lo + j], bh = a.ROWHI[lo + j];
    const double gbl = a.w.ABL[lo + j], gbh = a.w.ABH[lo + j];
    double gs = 0.0, hs = 0.0;
    for (int k = gl; k < K; k += G) {
      if (k == j) continue;
      const double idl = rcp_refined((oj - a.DORG[lo + k]) + (tj - a.TAU[lo + k]));  // 1/(l_j - l_k)
      const double wd = fma(bl, a.w.ABL[lo + k], bh * a.w.ABH[lo + k]) -
                        fma(a.ROWLO[lo + k], gbl, a.ROWHI[lo + k] * gbh);  // W_jk - W_kj
      const double u = wd * a.w.RINU[lo + k] * idl;
      gs = fma(u, idl, gs);
      hs += u;
    }
    gs = adj_group_sum<G>(gs, mask);
    hs = adj_group_sum<G>(hs, mask);
    if (gl == 0) {
      const double inuj = a.w.RINU[lo + j];
      const double gj = -inuj * gs;      // -sum_k W' / (nu_j nu_k (l_j - l_k)^2)
      const double hj = hs / ms.rho;     // sum_k W' c_k / (l_k - l_j) with c_k = -inu_k / rho'
      const double c = -inuj / ms.rho;
      const double lb = a.w.ALB[lo + j];
      a.w.RLT[lo + j] = gj;
      a.w.RAL[lo + j] = hj;
      a.w.RC[lo + j] = fma(2.0 * lb, c, hj);
      atomicAdd(&a.w.RHOBAR[g], lb * c * c + 0.5 * c * hj);
    }
  }
}

// Per active pole s: adjoints of D_s, z_s (through zhat ~ z), RLO_s, RHI_s, as
// sums over the roots j with y_sj = t_sj / nu_j, t_sj = zhat_s / (D_s - l_j):
//   D_bar = sum lbar_j y^2 + zhat_s sum g_j t,  z_bar = rho' sum y (2 lbar_j c_j + h_j),
//   RLO_bar = sum blo_bar_j y,  RHI_bar = sum bhi_bar_j y.
template <int G>
__global__ void __launch_bounds__(128) k_adj_poles(AdjArgs a, int big) {
  const uint32_t total = big ? *a.count2 : *a.count;
  const int lane = threadIdx.x & 31, gl = lane & (G - 1);
  const unsigned mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const uint32_t grp = (blockIdx.x * blockDim.x + threadIdx.x) / G;
  const uint32_t ngrp = (gridDim.x * blockDim.x) / G;
  for (uint32_t r = grp; r < total; r += ngrp) {
    const int g = big ? a.ROOTMAP2[r] : a.ROOTMAP[r];
    const MState ms = a.ms[g];
    const int K = ms.K, i = int(r) - ms.base, lo = a.M[g].lo;
    const double Di = a.AD[lo + i], zh = a.ZHAT[lo + i];
    double s1 = 0.0, s2 = 0.0, zb = 0.0, rlb = 0.0, rhb = 0.0;
    for (int j = gl; j < K; j += G) {
      const double t = zh * rcp_refined((Di - a.DORG[lo + j]) - a.TAU[lo + j]);
      const double y = t * a.w.RINU[lo + j];
      s1 = fma(y * a.w.ALB[lo + j], y, s1);
      s2 = fma(t, a.w.RLT[lo + j], s2);
      zb = fma(y, a.w.RC[lo + j], zb);
      rlb = fma(a.w.ABL[lo + j], y, rlb);
      rhb = fma(a.w.ABH[lo + j], y, rhb);
    }
    s1 = adj_group_sum<G>(s1, mask);
    s2 = adj_group_sum<G>(s2, mask);
    zb = adj_group_sum<G>(zb, mask);
    rlb = adj_group_sum<G>(rlb, mask);
    rhb = adj_group_sum<G>(rhb, mask);
    if (gl == 0) {
      a.w.PDB[lo + i] = fma(zh, s2, s1);
      a.w.PZB[lo + i] = ms.rho * zb;
      a.w.PRLB[lo + i] = rlb;
      a.w.PRHB[lo + i] = rhb;
    }
  }
}

// Per rotation-deflated position: kappa_bar (see the header) by a sweep over the
// active roots of its merge (one warp per position).
__global__ void k_adj_kappa(AdjArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  // 32 positions per warp round: a ballot of the rotation-deflated ones, each
  // then swept by the whole warp
  for (int64_t base = warp * 32; base < a.nrows; base += nwarps * 32) {
    const int64_t pl = base + lane;
    unsigned cand = __ballot_sync(0xffffffffu, pl < a.nrows && a.PFLAG[pl] == 2);
    while (cand) {
      const int64_t p = base + (__ffs(cand) - 1);
      cand &= cand - 1;
      const int64_t g = find_merge(a.M, a.cnt, p);
      const Merge m = a.M[g];
      if (p < m.lo || p >= m.hi) continue;  // a row outside this step's merges
      const int lo = m.lo;
      const int K = a.ms[g].K;
      const int idx = lo + a.OUTIDX[p];
      const int ia = lo + a.KEEPIDX[p];
      const double v = a.AD[idx], rl = a.ALO[idx], rh = a.AHI[idx];
      const double gbl = a.w.ABL[idx], gbh = a.w.ABH[idx];
      const double Da = a.AD[ia], za = a.ZHAT[ia];
      double kb = 0.0;
      for (int j = lane; j < K; j += 32) {
        const double oj = a.DORG[lo + j], tj = a.TAU[lo + j];
        const double y = za * rcp_refined((Da - oj) - tj) * a.w.RINU[lo + j];
        const double num = (a.w.ABL[lo + j] * rl + a.w.ABH[lo + j] * rh) -
                           (gbl * a.ROWLO[lo + j] + gbh * a.ROWHI[lo + j]);
        kb = fma(y * num, rcp_refined((oj - v) + tj), kb);
      }
      kb = adj_warp_sum(kb);
      if (lane == 0) a.w.KBAR[p] = kb;
    }
  }
}

// Deflation adjoint of one merge (one block per merge).  Negligible-z entries pass
// their adjoints through; every rotation run (survivors k0..kL, kept pole = the
// z^2-weighted mean, deflated entries = cross-weighted means, rows rotated) is
// reversed by one thread through its prefix sums W, S = sum D w, U = sum z R.
__global__ void k_adj_deflate(AdjArgs a) {
  for (int64_t g = blockIdx.x; g < a.cnt; g += gridDim.x) {
    const Merge m = a.M[g];
    const int lo = m.lo, n0 = m.hi - m.lo;
    const double* D = a.D + lo;
    const double* Z = a.Z + lo;
    const double* RL = a.RLO + lo;
    const double* RH = a.RHI + lo;
    int S = 0;  // survivors = positions not deflated for a negligible z
    for (int p = threadIdx.x; p < n0; p += blockDim.x) {
      if (a.PFLAG[lo + p] == 1) {
        const int idx = lo + a.OUTIDX[lo + p];
        a.w.MDB[lo + p] = a.w.ALB[idx];
        a.w.MZB[lo + p] = 0.0;
        a.w.MRLB[lo + p] = a.w.ABL[idx];
        a.w.MRHB[lo + p] = a.w.ABH[idx];
      }
    }
    {
      int c = 0;
      for (int p = threadIdx.x; p < n0; p += blockDim.x) c += a.PFLAG[lo + p] != 1 ? 1 : 0;
      __shared__ int s_cnt;
      if (threadIdx.x == 0) s_cnt = 0;
      __syncthreads();
      atomicAdd(&s_cnt, c);
      __syncthreads();
      S = s_cnt;
      __syncthreads();
    }
    double* PW = a.w.RLT + lo;  // per-survivor prefix scratch (the root scalars are dead)
    double* PS = a.w.RAL + lo;
    double* PUL = a.w.RBE + lo;
    double* PUH = a.w.RGA + lo;
    for (int k0 = threadIdx.x; k0 < S; k0 += blockDim.x) {
      if (a.RFLAG[lo + k0] == 0) continue;  // not a run start
      int kL = k0;
      while (kL + 1 < S && a.RFLAG[lo + kL + 1] == 0) ++kL;
      const int L = kL - k0;
      const int act = lo + a.ACTMAP[lo + kL];
      if (L == 0) {
        const int p = a.SURV[lo + k0] - lo;
        a.w.MDB[lo + p] = a.w.PDB[act];
        a.w.MZB[lo + p] = a.w.PZB[act];
        a.w.MRLB[lo + p] = a.w.PRLB[act];
        a.w.MRHB[lo + p] = a.w.PRHB[act];
        continue;
      }
      // forward prefix sums
      double W = 0.0, Sx = 0.0, UL = 0.0, UH = 0.0;
      for (int q = 0; q <= L; ++q) {
        const int p = a.SURV[lo + k0 + q] - lo;
        const double z = Z[p], w = z * z;
        W += w;
        Sx += D[p] * w;
        UL += z * RL[p];
        UH += z * RH[p];
        PW[k0 + q] = W;
        PS[k0 + q] = Sx;
        PUL[k0 + q] = UL;
        PUH[k0 + q] = UH;
      }
      // adjoint of the kept pole (prefix L)
      const double cbar = a.w.PDB[act], zabar = a.w.PZB[act];
      const double ralbar = a.w.PRLB[act], rahbar = a.w.PRHB[act];
      const double za = sqrt(W);
      double aW = -cbar * Sx / (W * W) + zabar / (2.0 * za) -
                  (ralbar * UL + rahbar * UH) / (2.0 * za * za * za);
      double aS = cbar / W;
      double aUL = ralbar / za, aUH = rahbar / za;
      double GW = 0.0, GS = 0.0, GUL = 0.0, GUH = 0.0;
      for (int q = L; q >= 0; --q) {
        const int p = a.SURV[lo + k0 + q] - lo;
        const double Dm = D[p], zm = Z[p], wm = zm * zm, Rl = RL[p], Rh = RH[p];
        GW += aW;
        GS += aS;
        GUL += aUL;
        GUH += aUH;
        double wbar = GW + GS * Dm;
        double dbar = GS * wm;
        double zbar = GUL * Rl + GUH * Rh;
        double rlbar = GUL * zm, rhbar = GUH * zm;
        aW = aS = aUL = aUH = 0.0;
        if (q >= 1) {  // deflated entry q uses prefix q-1
          // dropped coupling to the kept pole: kappa = Km (c_{q-1} - D_q)
          {
            const double Pw = PW[k0 + q - 1];
            const double Km = zm * sqrt(Pw) / sqrt(PW[k0 + q] * W);
            const double kb = a.w.KBAR[lo + p] * Km;
            dbar -= kb;
            aS += kb / Pw;                                // c = S / W over prefix q-1
            aW -= kb * PS[k0 + q - 1] / (Pw * Pw);
          }
          const int idx = lo + a.OUTIDX[lo + p];
          const double vbar = a.w.ALB[idx], rbl = a.w.ABL[idx], rbh = a.w.ABH[idx];
          const double P = PW[k0 + q - 1], Sp = PS[k0 + q - 1];
          const double Upl = PUL[k0 + q - 1], Uph = PUH[k0 + q - 1];
          const double Q = P + wm;
          const double v = (wm * (Sp / P) + P * Dm) / Q;
          const double sig = 1.0 / sqrt(P * Q);
          const double numl = zm * Upl - P * Rl, numh = zm * Uph - P * Rh;
          const double dsig_dP = -sig * (Q + P) / (2.0 * P * Q);
          const double dsig_dw = -sig / (2.0 * Q);
          // value
          aW += vbar * (Dm - wm * Sp / (P * P) - v) / Q;
          aS += vbar * (wm / P) / Q;
          wbar += vbar * (Sp / P - v) / Q;
          dbar += vbar * P / Q;
          // rows
          aW += rbl * (-Rl * sig + numl * dsig_dP) + rbh * (-Rh * sig + numh * dsig_dP);
          aUL += rbl * zm * sig;
          aUH += rbh * zm * sig;
          wbar += (rbl * numl + rbh * numh) * dsig_dw;
          zbar += (rbl * Upl + rbh * Uph) * sig;
          rlbar += -P * sig * rbl;
          rhbar += -P * sig * rbh;
        }
        zbar += 2.0 * zm * wbar;
        a.w.MDB[lo + p] = dbar;
        a.w.MZB[lo + p] = zbar;
        a.w.MRLB[lo + p] = rlbar;
        a.w.MRHB[lo + p] = rhbar;
      }
    }
    if (threadIdx.x == 0) {
      // rho' = 2 |beta|, beta = e at the cut
      const double beta = a.es[m.mid - 1];
      const double sg = beta >= 0.0 ? 1.0 : -1.0;
      atomicAdd(&a.grad_e[m.mid - 1], 2.0 * sg * a.w.RHOBAR[g]);
    }
    __syncthreads();
  }
}

// merge-position adjoints -> the children's (lambda, blo, bhi) adjoints
__global__ void k_adj_form(AdjArgs a) {
  const double inv_sqrt2 = 0.70710678118654752440;
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < a.nrows;
       p += int64_t(gridDim.x) * blockDim.x) {
    const Merge m = a.M[find_merge(a.M, a.cnt, p)];
    if (p < m.lo || p >= m.hi) continue;
    const double beta = a.es[m.mid - 1];
    const double sgn = beta >= 0.0 ? 1.0 : -1.0;
    const double x = a.in.lam[p];
    if (p < m.mid) {
      const int out = m.lo + int(p - m.lo) + count_less(a.in.lam + m.mid, m.hi - m.mid, x);
      a.w.GL[p] = a.w.MDB[out];
      a.w.GBH[p] = a.w.MZB[out] * inv_sqrt2;
      a.w.GBL[p] = a.w.MRLB[out];
    } else {
      const int out = m.lo + int(p - m.mid) + count_leq(a.in.lam + m.lo, m.mid - m.lo, x);
      a.w.GL[p] = a.w.MDB[out];
      a.w.GBL[p] = sgn * a.w.MZB[out] * inv_sqrt2;
      a.w.GBH[p] = a.w.MRHB[out];
    }
  }
}

// ---------------------------------------------------------------------------
// Leaves: full eigen-decomposition of the torn leaf by the same implicit QR with
// all rotations accumulated into Q (m <= 32), then the symmetric eigen adjoint.
__device__ bool leaf_qr_full(int m, double* a, double* b, double* Q) {
  int hi = m - 1, steps = 0;
  while (hi > 0) {
    int lo = hi;
    while (lo > 0) {
      if (fabs(b[lo - 1]) <= kEps * (fabs(a[lo - 1]) + fabs(a[lo]))) {
        b[lo - 1] = 0.0;
        break;
      }
      --lo;
    }
    if (lo == hi) {
      --hi;
      continue;
    }
    if (++steps > 40 * m) return false;
    const double bh = b[hi - 1];
    const double half = 0.5 * (a[hi - 1] - a[hi]);
    const double root = sqrt(half * half + bh * bh);
    double mu = a[hi] - bh * bh / (half + (half >= 0.0 ? root : -root));
    if (!isfinite(mu)) mu = a[hi];
    double x = a[lo] - mu, y = b[lo];
    for (int i = lo; i < hi; ++i) {
      double c, s, r;
      leaf_givens(x, y, c, s, r);  // the same rotation as the forward leaf solver
      if (i > lo) b[i - 1] = r;
      leaf_rotate(c, s, a[i], a[i + 1], b[i], a[i], a[i + 1], b[i]);
      if (i + 1 < hi) {
        const double bn = b[i + 1];
        y = s * bn;
        b[i + 1] = c * bn;
        x = b[i];
      }
      for (int r0 = 0; r0 < m; ++r0) {  // the tracked rows' update of the forward, every row
        const double p = Q[r0 * kMaxBwdLeaf + i], q = Q[r0 * kMaxBwdLeaf + i + 1];
        Q[r0 * kMaxBwdLeaf + i] = fma(c, p, s * q);
        Q[r0 * kMaxBwdLeaf + i + 1] = fma(c, q, -(s * p));
      }
    }
  }
  return true;
}

__global__ void k_adj_leaves(const Leaf* __restrict__ leaves, int64_t nleaves,
                             const double* __restrict__ ds, const double* __restrict__ es,
                             const double* __restrict__ GL, const double* __restrict__ GBL,
                             const double* __restrict__ GBH, LevelState fwd, double* grad_d,
                             double* grad_e, Status* st) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < nleaves;
       t += int64_t(gridDim.x) * blockDim.x) {
    const Leaf lf = leaves[t];
    const int m = lf.hi - lf.lo;
    double a[kMaxBwdLeaf], b[kMaxBwdLeaf], Q[kMaxBwdLeaf * kMaxBwdLeaf];
    for (int j = 0; j < m; ++j) {
      a[j] = ds[lf.lo + j];
      b[j] = (j + 1 < m) ? es[lf.lo + j] : 0.0;
      for (int k = 0; k < m; ++k) Q[j * kMaxBwdLeaf + k] = (j == k) ? 1.0 : 0.0;
    }
    if (lf.flags & 1) a[0] -= fabs(es[lf.lo - 1]);
    if (lf.flags & 2) a[m - 1] -= fabs(es[lf.hi - 1]);
    if (!leaf_qr_full(m, a, b, Q)) set_status(st, TDE_ENOCONV);
    // ascending order; the columns of Q follow their eigenvalue
    for (int j = 0; j < m; ++j) {
      int best = j;
      for (int k = j + 1; k < m; ++k)
        if (a[k] < a[best]) best = k;
      if (best != j) {
        const double tv = a[j];
        a[j] = a[best];
        a[best] = tv;
        for (int r = 0; r < m; ++r) {
          const double tq = Q[r * kMaxBwdLeaf + j];
          Q[r * kMaxBwdLeaf + j] = Q[r * kMaxBwdLeaf + best];
          Q[r * kMaxBwdLeaf + best] = tq;
        }
      }
    }
    // eigenvector signs are arbitrary: align every column with the rows the
    // forward pass stored (the row adjoints refer to those), using the larger of
    // the two boundary entries
    if (!(lf.flags & 4)) {
      for (int k = 0; k < m; ++k) {
        const double f0 = fwd.blo[lf.lo + k], f1 = fwd.bhi[lf.lo + k];
        const double q0 = Q[0 * kMaxBwdLeaf + k], q1 = Q[(m - 1) * kMaxBwdLeaf + k];
        const bool flip = fabs(f0) >= fabs(f1) ? (q0 * f0 < 0.0) : (q1 * f1 < 0.0);
        if (flip)
          for (int r = 0; r < m; ++r) Q[r * kMaxBwdLeaf + k] = -Q[r * kMaxBwdLeaf + k];
      }
    }
    // H = Q G with G_jk = lbar_j [j == k] + (Q_0j blobar_k + Q_{m-1}j bhibar_k) / (l_k - l_j)
    double hprev[kMaxBwdLeaf];
    for (int i = 0; i < m; ++i) {
      double hrow[kMaxBwdLeaf];
      for (int k = 0; k < m; ++k) {
        double s0 = 0.0, s1 = 0.0;
        for (int j = 0; j < m; ++j) {
          if (j == k || a[k] == a[j]) continue;
          const double f = Q[i * kMaxBwdLeaf + j] / (a[k] - a[j]);
          s0 += f * Q[0 * kMaxBwdLeaf + j];
          s1 += f * Q[(m - 1) * kMaxBwdLeaf + j];
        }
        hrow[k] = Q[i * kMaxBwdLeaf + k] * GL[lf.lo + k] + GBL[lf.lo + k] * s0 +
                  GBH[lf.lo + k] * s1;
      }
      double dbar = 0.0;
      for (int k = 0; k < m; ++k) dbar += hrow[k] * Q[i * kMaxBwdLeaf + k];
      grad_d[lf.lo + i] = dbar;
      if (i > 0) {  // e between rows i-1 and i: A_bar(i-1, i) + A_bar(i, i-1)
        double eb = 0.0;
        for (int k = 0; k < m; ++k)
          eb += hprev[k] * Q[i * kMaxBwdLeaf + k] + hrow[k] * Q[(i - 1) * kMaxBwdLeaf + k];
        atomicAdd(&grad_e[lf.lo + i - 1], eb);
      }
      if (i == 0 && (lf.flags & 1)) {
        const double c = es[lf.lo - 1];
        atomicAdd(&grad_e[lf.lo - 1], -(c >= 0.0 ? 1.0 : -1.0) * dbar);
      }
      if (i == m - 1 && (lf.flags & 2)) {
        const double c = es[lf.hi - 1];
        atomicAdd(&grad_e[lf.hi - 1], -(c >= 0.0 ? 1.0 : -1.0) * dbar);
      }
      for (int k = 0; k < m; ++k) hprev[k] = hrow[k];
    }
  }
}

__global__ void k_adj_init(int64_t nrows, const double* __restrict__ grad_lambda, double* GL,
                           double* GBL, double* GBH, double* grad_e) {
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < nrows;
       p += int64_t(gridDim.x) * blockDim.x) {
    GL[p] = grad_lambda[p];
    GBL[p] = 0.0;
    GBH[p] = 0.0;
    grad_e[p] = 0.0;
  }
}

void launch_leaves_to(const Plan& plan, const Workspace& ws, double* lambda, cudaStream_t s,
                      LevelState out);

// Reverses merge step st: rebuilds its merge internals from the state `in` of
// level st (the roots restored from `roots` when given, else solved again) and
// pulls the adjoints of the parents' state back to the children's.
static void adjoint_step(const Plan& plan, const AdjWorkspace& w, int st, LevelState in,
                         const RootsCheckpoint* roots, double* lambda, double* grad_e,
                         cudaStream_t s) {
  const Workspace& ws = w.fw;
  const int64_t N = plan.nrows;
  const Merge* M = ws.merges + plan.step_base[st];
  const int64_t cnt = plan.step_count[st];
  cudaMemsetAsync(&ws.status->root_count[st], 0, 4, s);
  cudaMemsetAsync(&ws.status->root_count_big[st], 0, 4, s);
  cudaMemsetAsync(w.RHOBAR, 0, 8 * size_t(cnt), s);
  const LevelState scratch{ws.LAM, ws.BLO, ws.BHI};
  launch_step(plan, ws, st, lambda, s, in, scratch, /*recompute=*/true, nullptr, w.RINU, roots);
  AdjArgs a;
  a.M = M;
  a.cnt = cnt;
  a.nrows = N;
  a.ms = ws.mstate;
  a.ROOTMAP = ws.ROOTMAP;
  a.ROOTMAP2 = ws.ROOTMAP2;
  a.count = &ws.status->root_count[st];
  a.count2 = &ws.status->root_count_big[st];
  a.LAMA = ws.D;
  a.AD = ws.AD;
  a.AZ = ws.AZ;
  a.ALO = ws.ALO;
  a.AHI = ws.AHI;
  a.TAU = ws.TAU;
  a.DORG = reinterpret_cast<const double*>(ws.KEYA);
  a.ZHAT = ws.Z;
  a.ROWLO = ws.RLO;
  a.ROWHI = ws.RHI;
  a.D = ws.D;
  a.Z = ws.Z;
  a.RLO = ws.RLO;
  a.RHI = ws.RHI;
  a.es = ws.es;
  a.SURV = ws.SURV;
  a.OUTIDX = ws.OUTIDX;
  a.ACTMAP = ws.ACTMAP;
  a.KEEPIDX = ws.KEEPIDX;
  a.PFLAG = ws.PFLAG;
  a.RFLAG = ws.RFLAG;
  a.in = in;
  a.w = w;
  a.grad_e = grad_e;
  const int flat = int(std::min<int64_t>((N + 255) / 256, 148 * 8));
  const int ggrid = int(std::min<int64_t>((N * 4 + 127) / 128, 148 * 16));
  k_adj_place<<<flat, 256, 0, s>>>(a);
  k_adj_pairs<4><<<ggrid, 128, 0, s>>>(a, 0);
  k_adj_pairs<32><<<148 * 8, 128, 0, s>>>(a, 1);
  k_adj_poles<4><<<ggrid, 128, 0, s>>>(a, 0);
  k_adj_poles<32><<<148 * 8, 128, 0, s>>>(a, 1);
  k_adj_kappa<<<148 * 8, 128, 0, s>>>(a);
  launch_form(plan, ws, st, in, s);  // restore D, z, RLO, RHI of the merge problem
  const int dgrid = int(std::min<int64_t>(cnt, 148 * 8));
  k_adj_deflate<<<dgrid, 256, 0, s>>>(a);
  k_adj_form<<<flat, 256, 0, s>>>(a);
  g_launches += 9;
}

// Copies level state a to b (three arrays of n doubles).
static int copy_state(LevelState src, LevelState dst, int64_t N, cudaStream_t s) {
  const size_t bytes = 8 * size_t(N);
  if (cudaMemcpyAsync(dst.lam, src.lam, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(dst.blo, src.blo, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(dst.bhi, src.bhi, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return TDE_ECUDA;
  return TDE_OK;
}

// Bisection schedule of the slots layout (see the file header).
struct Reverser {
  const Plan& plan;
  const AdjWorkspace& w;
  double* lambda;
  double* grad_e;
  cudaStream_t s;
  int rc = TDE_OK;
  LevelState slot(int k) const {
    const int64_t N = plan.nrows;
    double* base = w.CK + size_t(k) * 3 * size_t(N);
    return LevelState{base, base + N, base + 2 * N};
  }
  // the state of level `to` into dst (in place), from the state of level `from` in src;
  // each recomputed step's root lists start empty again (its deflation appends to them)
  void forward(LevelState src, int from, LevelState dst, int to) {
    if (rc == TDE_OK) rc = copy_state(src, dst, plan.nrows, s);
    for (int k = from; k < to; ++k) {
      if (cudaMemsetAsync(&w.fw.status->root_count[k], 0, 4, s) != cudaSuccess ||
          cudaMemsetAsync(&w.fw.status->root_count_big[k], 0, 4, s) != cudaSuccess)
        rc = TDE_ECUDA;
      launch_step(plan, w.fw, k, lambda, s, dst, dst);
    }
  }
  static int mid_of(int lo, int hi) { return lo + (hi - lo + 1) / 2; }
  // reverses steps [lo, hi) from the state of level lo held in slot sl; slots
  // sl + 1 ... hold the first descent's levels when `primed` (filled by the first
  // forward pass), else they are free
  void run(int lo, int hi, int sl, bool primed) {
    if (hi <= lo) return;
    if (hi - lo == 1) {
      adjoint_step(plan, w, lo, slot(sl), nullptr, lambda, grad_e, s);
      return;
    }
    if (sl + 1 >= w.slots) {  // no free slot: each step from a recomputation into the scratch level
      const LevelState scratch{w.fw.LAM, w.fw.BLO, w.fw.BHI};
      for (int st = hi - 1; st > lo; --st) {
        forward(slot(sl), lo, scratch, st);
        adjoint_step(plan, w, st, scratch, nullptr, lambda, grad_e, s);
      }
      adjoint_step(plan, w, lo, slot(sl), nullptr, lambda, grad_e, s);
      return;
    }
    const int mid = mid_of(lo, hi);
    if (!primed) forward(slot(sl), lo, slot(sl + 1), mid);
    run(mid, hi, sl + 1, primed);
    run(lo, mid, sl, false);
  }
};

int run_adjoint(const Plan& plan, const AdjWorkspace& w, const int64_t* offsets_dev,
                const double* d, const double* e, const double* grad_lambda, double* lambda,
                double* grad_d, double* grad_e, cudaStream_t s) {
  const Workspace& ws = w.fw;
  const int64_t N = plan.nrows;
  if (lambda == nullptr) lambda = w.LAMOUT;
  if (cudaMemsetAsync(ws.status, 0, sizeof(Status), s) != cudaSuccess) return TDE_ECUDA;
  if (cudaMemsetAsync(ws.sigma_bits, 0, 8 * size_t(plan.batch), s) != cudaSuccess)
    return TDE_ECUDA;
  const LevelState scratch{ws.LAM, ws.BLO, ws.BHI};
  Reverser rv{plan, w, lambda, grad_e, s};
  // 1. forward pass: the eigenvalues, and the checkpoints
  launch_plan(plan, ws, offsets_dev, s);
  launch_scale(plan, ws, offsets_dev, d, e, s);
  launch_leaves_to(plan, ws, lambda, s, plan.steps > 0 ? rv.slot(0) : scratch);
  if (w.levels) {
    for (int st = 0; st < plan.steps; ++st) {
      const LevelState out = st + 1 < plan.steps ? rv.slot(st + 1) : scratch;
      launch_step(plan, ws, st, lambda, s, rv.slot(st), out);
      double* cr = w.CR + size_t(st) * 2 * size_t(N);
      if (cudaMemcpyAsync(cr, ws.TAU, 8 * size_t(N), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
          cudaMemcpyAsync(cr + N, ws.KEYA, 8 * size_t(N), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return TDE_ECUDA;
    }
  } else if (plan.steps > 0) {
    // in place on the scratch level; the levels of the schedule's first descent
    // (0, then mid of [previous, steps), ...) are copied into slots 1, 2, ...
    if (copy_state(rv.slot(0), scratch, N, s) != TDE_OK) return TDE_ECUDA;
    int next_slot = 1, lo = 0;
    int want = (w.slots > 1 && plan.steps > 1) ? Reverser::mid_of(0, plan.steps) : -1;
    for (int st = 0; st < plan.steps; ++st) {
      launch_step(plan, ws, st, lambda, s, scratch, scratch);
      if (st + 1 == want) {
        if (copy_state(scratch, rv.slot(next_slot), N, s) != TDE_OK) return TDE_ECUDA;
        ++next_slot;
        lo = want;
        want = (next_slot < w.slots && plan.steps - lo > 1) ? Reverser::mid_of(lo, plan.steps) : -1;
      }
    }
  }
  const int flat = int(std::min<int64_t>((N + 255) / 256, 148 * 8));
  k_adj_init<<<flat, 256, 0, s>>>(N, grad_lambda, w.GL, w.GBL, w.GBH, grad_e);
  g_launches += 1;
  // 2. reverse sweep
  if (w.levels) {
    for (int st = plan.steps - 1; st >= 0; --st) {
      const double* cr = w.CR + size_t(st) * 2 * size_t(N);
      const RootsCheckpoint roots{cr, cr + N};
      adjoint_step(plan, w, st, rv.slot(st), &roots, lambda, grad_e, s);
    }
  } else {
    rv.run(0, plan.steps, 0, true);
    if (rv.rc != TDE_OK) return rv.rc;
  }
  // 3. leaves
  const int lgrid = int(std::min<int64_t>((plan.nleaves + 63) / 64, 148 * 32));
  const LevelState leafstate = plan.steps > 0 ? rv.slot(0) : scratch;
  k_adj_leaves<<<std::max(lgrid, 1), 64, 0, s>>>(ws.leaves, plan.nleaves, ws.ds, ws.es, w.GL,
                                                  w.GBL, w.GBH, leafstate, grad_d, grad_e,
                                                  ws.status);
  g_launches += 1;
  return cudaGetLastError() == cudaSuccess ? TDE_OK : TDE_ECUDA;
}

// Bytes of the slots layout with `slots` checkpoint slots, and of the levels layout.
static int backward_sizes(int64_t batch, const int64_t* offsets_host, int32_t leaf, int slots,
                          Plan* p, size_t* slots_bytes, size_t* levels_bytes) {
  int rc = build_plan(batch, offsets_host, leaf, p);
  if (rc != TDE_OK) return rc;
  if (p->leaf > kMaxBwdLeaf) return TDE_EINVAL;
  if (slots_bytes) *slots_bytes = carve_adjoint(*p, nullptr, nullptr, false, slots);
  if (levels_bytes) *levels_bytes = carve_adjoint(*p, nullptr, nullptr, true, 0);
  return TDE_OK;
}

}  // namespace tde

using namespace tde;

extern "C" int tde_eigvals_backward_workspace(int64_t batch, const int64_t* offsets_host,
                                              int32_t leaf, size_t* bytes) {
  if (bytes == nullptr) return TDE_EINVAL;
  Plan p;
  return backward_sizes(batch, offsets_host, leaf, kDefaultSlots, &p, bytes, nullptr);
}

extern "C" int tde_eigvals_backward_workspace_slots(int64_t batch, const int64_t* offsets_host,
                                                    int32_t leaf, int32_t slots, size_t* bytes) {
  if (bytes == nullptr || slots < 0) return TDE_EINVAL;
  Plan p;
  size_t sb = 0, lb = 0;
  const int rc = backward_sizes(batch, offsets_host, leaf, slots == 0 ? 1 : slots, &p, &sb, &lb);
  if (rc != TDE_OK) return rc;
  *bytes = (slots == 0 || slots >= p.steps) ? lb : sb;
  return TDE_OK;
}

extern "C" int tde_eigvals_backward(int64_t batch, const int64_t* offsets_host,
                                    const int64_t* offsets_dev, const double* d, const double* e,
                                    const double* grad_lambda, double* lambda, double* grad_d,
                                    double* grad_e, int32_t leaf, void* ws, size_t ws_bytes,
                                    void* stream) {
  g_launches = 0;
  Plan p;
  size_t one = 0, lb = 0;
  int rc = backward_sizes(batch, offsets_host, leaf, 1, &p, &one, &lb);
  if (rc != TDE_OK) return rc;
  if (p.nrows == 0) return TDE_OK;
  if (offsets_dev == nullptr || d == nullptr || grad_lambda == nullptr || grad_d == nullptr ||
      grad_e == nullptr || ws == nullptr || (p.nrows > 1 && e == nullptr))
    return TDE_EINVAL;
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return TDE_EINVAL;
  if (ws_bytes < one) return TDE_EWORKSPACE;
  // the levels layout when it fits, else as many slots as fit
  const bool levels = ws_bytes >= lb;
  int slots = 1;
  if (!levels)
    while (slots + 1 < std::max(p.steps, 1) &&
           carve_adjoint(p, nullptr, nullptr, false, slots + 1) <= ws_bytes)
      ++slots;
  AdjWorkspace w;
  carve_adjoint(p, ws, &w, levels, slots);
  return run_adjoint(p, w, offsets_dev, d, e, grad_lambda, lambda, grad_d, grad_e,
                     static_cast<cudaStream_t>(stream));
}
