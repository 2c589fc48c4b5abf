// One merge level of the boundary-row D&C (Algorithm 1, internal-node branch;
// Sec. 4.1 GPU implementation).  Every kernel covers all merges of one step.
//
//   k_form     D = Lambda_L (+) Lambda_R by a merge of the two sorted child
//              spectra; z = concat(bhi(Q_L), s blo(Q_R)) / sqrt(2), rho' = 2|beta|
//              (Eq. merge-problem, Lemma "boundary sufficiency"); the rows of
//              diag(Q_L, Q_R) that feed the parent's boundary rows are
//              RLO = [blo(Q_L), 0] and RHI = [0, bhi(Q_R)].
//   k_deflate  deflation (Sec. 4.1: negligible z, close poles, Givens rotations on
//              z and on the two rows, compaction, active / deflated maps; the
//              rotations and permutations commute with row selection by the
//              appendix lemmas on column permutations and local rotations).
//   k_secular  the K roots of 1 + rho' sum z_i^2 / (D_i - lambda) (Sec. 4.1 root
//              solve), each stored compactly as lambda_j = D_org + tau_j
//              (Sec. 4.1 compact root representation; appendix "compact delta
//              reconstruction": Delta_i = (D_i - D_org) - tau).
//   k_lowner   z-hat from the computed roots (appendix "WPROD product chains"):
//              zhat_i^2 = prod_j (lambda_j - D_i) / (rho' prod_{j!=i} (D_j - D_i)),
//              evaluated as a product of positive ratios.
//   k_rows     parent boundary rows of each active column j (Sec. 4.1,
//              R_parent(:, j) = R_child y_j with y_j(i) = zhat_i / Delta_ij
//              normalised): two streamed dot products per root, no Y formed.
//   k_place    the parent's eigenvalues in ascending order (active roots merged
//              with the deflated eigenvalues), with their boundary rows; at a
//              root merge only the eigenvalues, unscaled, into the output.
#include <algorithm>

#include <cooperative_groups.h>

#include "tde_internal.cuh"

namespace tde {

namespace cg = cooperative_groups;

constexpr int kNT = 256;  // threads of the per-merge deflation block (small merges)

// ---------------------------------------------------------------------------
__global__ void k_form(const Merge* __restrict__ M, int64_t cnt, int64_t nrows,
                       const double* __restrict__ LAM, const double* __restrict__ BLO,
                       const double* __restrict__ BHI, const double* __restrict__ es, double* D,
                       double* Z, double* RLO, double* RHI) {
  const double inv_sqrt2 = 0.70710678118654752440;
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < nrows;
       p += int64_t(gridDim.x) * blockDim.x) {
    const Merge m = M[find_merge(M, cnt, p)];
    if (p < m.lo || p >= m.hi) continue;
    const double beta = es[m.mid - 1];
    const double sgn = beta >= 0.0 ? 1.0 : -1.0;
    const double x = LAM[p];
    if (p < m.mid) {
      int out = m.lo + int(p - m.lo) + count_less(LAM + m.mid, m.hi - m.mid, x);
      D[out] = x;
      Z[out] = BHI[p] * inv_sqrt2;
      RLO[out] = BLO[p];
      RHI[out] = 0.0;
    } else {
      int out = m.lo + int(p - m.mid) + count_leq(LAM + m.lo, m.mid - m.lo, x);
      D[out] = x;
      Z[out] = sgn * BLO[p] * inv_sqrt2;
      RLO[out] = 0.0;
      RHI[out] = BHI[p];
    }
  }
}

// ---------------------------------------------------------------------------
// Close-pole rotations as prefix sums.  Rotating a pole (D_p, z_p) against
// (D_j, z_j) so that the z-direction keeps all of z leaves a kept pole
// (w_p D_p + w_j D_j) / (w_p + w_j) with z = sqrt(w_p + w_j), w = z^2, and a
// deflated pole (w_j D_p + w_p D_j) / (w_p + w_j); the dropped coupling is
// z_p z_j (D_p - D_j) / (w_p + w_j).  Chaining rotations along a run a..k of
// consecutive survivors therefore keeps the run's z^2-weighted mean and total
// weight W, and the kept column of the rows is U / sqrt(W) with U = sum z R.
// A survivor j continues the run (is rotated into it) iff the dropped coupling
// is at most tol:  |sqrt(W) z_j (D_j - c)| <= tol (W + w_j), c = DW / W, which
// is tested squared: w_j (W D_j - DW)^2 <= tol^2 W (W + w_j)^2.
//
// The walks below evaluate this rule and the run sums at several call sites, and
// re-use decisions of earlier walks wherever the carry is unchanged, so every
// product and sum of them is rounded explicitly (__dmul_rn / __dadd_rn are never
// contracted into an FMA): each inlined copy computes the same bits, and a
// decision close to the threshold cannot differ between two walks of one input.
__device__ __forceinline__ bool continues_run(double W, double DW, double Dj, double wj,
                                              double tol2) {
  const double a = fma(W, Dj, -DW);
  const double s = __dadd_rn(W, wj);
  return __dmul_rn(__dmul_rn(wj, a), a) <= __dmul_rn(__dmul_rn(__dmul_rn(tol2, W), s), s);
}

struct T4 {
  double w, dw, ulo, uhi;
};
__device__ __forceinline__ T4 t4_add(const T4& a, const T4& b) {
  return T4{a.w + b.w, a.dw + b.dw, a.ulo + b.ulo, a.uhi + b.uhi};
}
__device__ __forceinline__ T4 t4_shfl_up(const T4& v, int o) {
  return T4{shfl_up_d(v.w, o), shfl_up_d(v.dw, o), shfl_up_d(v.ulo, o), shfl_up_d(v.uhi, o)};
}
__device__ __forceinline__ T4 t4_shfl_xor(const T4& v, int o) {
  return T4{__shfl_xor_sync(0xffffffffu, v.w, o), __shfl_xor_sync(0xffffffffu, v.dw, o),
            __shfl_xor_sync(0xffffffffu, v.ulo, o), __shfl_xor_sync(0xffffffffu, v.uhi, o)};
}

// Run boundaries of survivors [begin, end) (one warp).  The sequential rule -- walk
// the survivors in ascending order and let each one join the current run if the
// test passes -- is evaluated 32 survivors at a time: every lane first assumes the
// run of its predecessor is that predecessor alone, the assumed runs are summed
// with a segmented scan, the test is re-evaluated against them, and the first
// lane whose decision changes is fixed; lanes before it are already exact.
// (cW, cDW) carries the (W, DW) of the run open at `begin` (`have` = one is open)
// and returns the one open at the end.  With `stop_when_equal`, a chunk whose
// decisions equal those already in rflag and which contains a run start ends the
// walk early (returns false): from that start on the old decisions are exact.
// RFLAG[k] = 1 iff survivor k starts a run.
__device__ bool run_segment(int begin, int end, const int32_t* surv, const double* D,
                            const double* Z, double tol2, uint8_t* rflag, double& cW,
                            double& cDW, bool have, bool stop_when_equal) {
  const int lane = threadIdx.x & 31;
  for (int base = begin; base < end; base += 32) {
    const int k = base + lane;
    const bool valid = k < end;
    double Dk = 0.0, wk = 0.0;
    if (valid) {
      int pos = surv[k];
      Dk = D[pos];
      double zk = Z[pos];
      wk = __dmul_rn(zk, zk);
    }
    const double Dp = shfl_up_d(Dk, 1), wp = shfl_up_d(wk, 1);
    bool guess;
    if (lane == 0)
      guess = valid && have && continues_run(cW, cDW, Dk, wk, tol2);
    else
      guess = valid && continues_run(wp, __dmul_rn(Dp, wp), Dk, wk, tol2);
    int start = 0;
    double W = 0.0, DWv = 0.0;
    for (int iter = 0; iter <= 32; ++iter) {
      W = wk;
      DWv = __dmul_rn(Dk, wk);
      if (lane == 0 && guess) {
        W = __dadd_rn(W, cW);
        DWv = __dadd_rn(DWv, cDW);
      }
      bool h = !guess;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        double Wo = shfl_up_d(W, o), DWo = shfl_up_d(DWv, o);
        bool ho = __shfl_up_sync(0xffffffffu, h, o);
        if (lane >= o) {
          if (!h) {
            W = __dadd_rn(W, Wo);
            DWv = __dadd_rn(DWv, DWo);
          }
          h = h || ho;
        }
      }
      const double Wpre = shfl_up_d(W, 1), DWpre = shfl_up_d(DWv, 1);
      bool truth = guess;
      if (lane > 0) truth = valid && continues_run(Wpre, DWpre, Dk, wk, tol2);
      unsigned mis = __ballot_sync(0xffffffffu, valid && lane >= start && truth != guess);
      if (mis == 0) break;
      int f = __ffs(mis) - 1;
      if (lane == f) guess = truth;
      start = f + 1;
    }
    const uint8_t flag = guess ? 0 : 1;
    bool same = true;
    if (stop_when_equal && valid) same = rflag[k] == flag;
    const bool all_same = __all_sync(0xffffffffu, same);
    const bool any_start = __any_sync(0xffffffffu, valid && flag == 1);
    if (valid) rflag[k] = flag;
    int last = min(31, end - 1 - base);
    cW = __shfl_sync(0xffffffffu, W, last);
    cDW = __shfl_sync(0xffffffffu, DWv, last);
    have = true;
    if (stop_when_equal && all_same && any_start) return false;
  }
  return true;
}

// Run boundaries of all S survivors by the warps of the block.  Long lists are cut
// into one segment per warp; each warp walks its segment assuming the segment's
// first survivor is tested against its predecessor alone, then warp 0 re-walks the
// segments in order with the true carry until the decisions agree again (skipping
// those whose true carry is the assumed one).
template <int NT>
__device__ void run_boundaries(int S, const int32_t* surv, const double* D, const double* Z,
                               double tol2, uint8_t* rflag, double* s_cw, double* s_cdw) {
  constexpr int NW = NT / 32;
  const int warp = threadIdx.x >> 5;
  if (S < 64 * NW) {
    if (warp == 0) {
      double cW = 0.0, cDW = 0.0;
      run_segment(0, S, surv, D, Z, tol2, rflag, cW, cDW, false, false);
    }
    return;
  }
  const int seg = ((S + NW - 1) / NW + 31) & ~31;
  {
    const int b = warp * seg, e = min(S, b + seg);
    double cW = 0.0, cDW = 0.0;
    bool have = false;
    if (b < e) {
      if (b > 0) {  // speculative carry: the predecessor alone
        const int pos = surv[b - 1];
        const double z = Z[pos];
        cW = __dmul_rn(z, z);
        cDW = __dmul_rn(D[pos], cW);
        have = true;
      }
      run_segment(b, e, surv, D, Z, tol2, rflag, cW, cDW, have, false);
    }
    if ((threadIdx.x & 31) == 0) {
      s_cw[warp] = cW;
      s_cdw[warp] = cDW;
    }
  }
  __syncthreads();
  if (warp == 0) {
    for (int w = 1; w < NW; ++w) {
      const int b = w * seg, e = min(S, b + seg);
      if (b >= e) break;
      double cW = s_cw[w - 1], cDW = s_cdw[w - 1];
      // the speculative carry again (same expression, same bits): a segment whose
      // true carry equals it is already exact
      const double z = Z[surv[b - 1]], sW = __dmul_rn(z, z), sDW = __dmul_rn(D[surv[b - 1]], sW);
      if (__double_as_longlong(cW) == __double_as_longlong(sW) &&
          __double_as_longlong(cDW) == __double_as_longlong(sDW))
        continue;
      const bool completed = run_segment(b, e, surv, D, Z, tol2, rflag, cW, cDW, true, true);
      if (completed && (threadIdx.x & 31) == 0) {
        s_cw[w] = cW;
        s_cdw[w] = cDW;
      }
      __syncwarp();
    }
  }
}

// Block merge sort of keys (with int payload) in global scratch; n entries.
// Tiles of kTile are sorted in shared memory (bitonic), then merged pairwise.
// Returns a pointer to the buffer (A or B) holding the result.
constexpr int kTile = 1024;

// Bitonic sort of one tile [t0, t0 + len) of KA / IA in shared memory, in place.
__device__ void sort_tile(int t0, int len, unsigned long long* KA, int32_t* IA,
                          unsigned long long* skey, int32_t* sidx) {
  int p2 = 1;
  while (p2 < len) p2 <<= 1;
  for (int i = threadIdx.x; i < p2; i += blockDim.x) {
    skey[i] = (i < len) ? KA[t0 + i] : ~0ull;
    sidx[i] = (i < len) ? IA[t0 + i] : -1;
  }
  __syncthreads();
  for (int size = 2; size <= p2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < p2; i += blockDim.x) {
        int j = i ^ stride;
        if (j > i) {
          bool up = (i & size) == 0;
          unsigned long long ki = skey[i], kj = skey[j];
          if ((ki > kj) == up) {
            skey[i] = kj;
            skey[j] = ki;
            int32_t x = sidx[i];
            sidx[i] = sidx[j];
            sidx[j] = x;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    KA[t0 + i] = skey[i];
    IA[t0 + i] = sidx[i];
  }
  __syncthreads();
}

// Entries [first, n) with stride `step` of one pairwise merge pass (runs of
// `width` sorted entries in src, pairs merged into dst): each entry finds its place
// by a binary search in its partner run (ties: the left run first).
__device__ void merge_pass(int n, int width, int first, int step, const unsigned long long* src_k,
                           const int32_t* src_i, unsigned long long* dst_k, int32_t* dst_i) {
  for (int e = first; e < n; e += step) {
    int run = e / width;
    int run_lo = run * width;
    int pair_lo = (run & ~1) * width;
    int partner_lo = (run & 1) ? pair_lo : pair_lo + width;
    int partner_len = max(0, min(width, n - partner_lo));
    unsigned long long key = src_k[e];
    int lo = 0, hi = partner_len;
    if (run & 1) {  // right run: partner entries <= key come first
      while (lo < hi) {
        int m = (lo + hi) >> 1;
        if (src_k[partner_lo + m] <= key) lo = m + 1; else hi = m;
      }
    } else {  // left run: partner entries < key come first
      while (lo < hi) {
        int m = (lo + hi) >> 1;
        if (src_k[partner_lo + m] < key) lo = m + 1; else hi = m;
      }
    }
    int dst = pair_lo + (e - run_lo) + lo;
    dst_k[dst] = key;
    dst_i[dst] = src_i[e];
  }
}

__device__ int block_sort(int n, unsigned long long* KA, int32_t* IA, unsigned long long* KB,
                          int32_t* IB, unsigned long long* skey, int32_t* sidx) {
  for (int t0 = 0; t0 < n; t0 += kTile) sort_tile(t0, min(kTile, n - t0), KA, IA, skey, sidx);
  int which = 0;
  unsigned long long *src_k = KA, *dst_k = KB;
  int32_t *src_i = IA, *dst_i = IB;
  for (int width = kTile; width < n; width <<= 1) {
    merge_pass(n, width, threadIdx.x, blockDim.x, src_k, src_i, dst_k, dst_i);
    __syncthreads();
    unsigned long long* tk = src_k;
    src_k = dst_k;
    dst_k = tk;
    int32_t* ti = src_i;
    src_i = dst_i;
    dst_i = ti;
    which ^= 1;
  }
  return which;
}

struct DeflateArgs {
  const Merge* M;
  int64_t cnt;
  int step;
  const double* es;
  double *D, *Z, *RLO, *RHI;
  double *AD, *AZ, *ALO, *AHI;
  int32_t *SURV, *ROOTMAP, *ROOTMAP2, *IDXA, *IDXB, *ZPOS, *OUTIDX, *ACTMAP, *KEEPIDX;
  uint8_t *PFLAG, *RFLAG;
  unsigned long long *KEYA, *KEYB;
  MState* ms;
  Status* st;
  int32_t warp_min_k;
  int32_t order_small;  // forests: small-K merges get their list range from k_order_assign
};


// One CTA of NT threads per merge: 64 for steps whose merges have at most 64 rows,
// 256 up to 8192 rows and 1024 above (where steps with few merges take the
// cluster kernel instead); a CTA walks its merge in NT-row chunks.
template <int NT>
__global__ void __launch_bounds__(NT) k_deflate(DeflateArgs a) {
  __shared__ int sm_int[NT / 32];
  __shared__ double sm_dbl[NT / 32];
  __shared__ T4 s_agg[NT / 32];
  __shared__ int s_aggh[NT / 32];
  __shared__ T4 s_pre[NT / 32];
  __shared__ T4 s_incl[NT];
  __shared__ unsigned long long s_key[kTile];
  __shared__ int32_t s_idx[kTile];
  __shared__ int s_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int64_t g = blockIdx.x; g < a.cnt; g += gridDim.x) {
    const Merge m = a.M[g];
    const int lo = m.lo, n0 = m.hi - m.lo;
    const double rho = 2.0 * fabs(a.es[m.mid - 1]);
    double* D = a.D + lo;
    double* Z = a.Z + lo;
    double* RLO = a.RLO + lo;
    double* RHI = a.RHI + lo;
    uint8_t* PFLAG = a.PFLAG + lo;
    int32_t* SURV = a.SURV + lo;
    uint8_t* RFLAG = a.RFLAG + lo;

    // 1. tol = 8 eps max(max|D|, max|z|)   (D is sorted)
    double zm = 0.0;
    for (int i = tid; i < n0; i += NT) zm = fmax(zm, fabs(Z[i]));
    zm = block_max<NT>(zm, sm_dbl);
    const double dmax = fmax(fabs(D[0]), fabs(D[n0 - 1]));
    const double tol = 8.0 * kEps * fmax(dmax, zm);
    const double tol2 = tol * tol;

    // 2. negligible z: rho' |z_i| <= tol deflates pole i with its rows unchanged
    int S = 0;
    for (int c0 = 0; c0 < n0; c0 += NT) {
      int i = c0 + tid;
      int keep = 0;
      if (i < n0) {
        keep = rho * fabs(Z[i]) > tol ? 1 : 0;
        PFLAG[i] = keep ? 0 : 1;
      }
      int total;
      int ex = block_excl_scan<NT>(keep, sm_int, &total);
      if (keep) SURV[S + ex] = lo + i;
      S += total;
    }
    __syncthreads();

    // 3. close poles: run boundaries over the survivors
    __shared__ double s_cw[NT / 32], s_cdw[NT / 32];
    run_boundaries<NT>(S, SURV, a.D, a.Z, tol2, RFLAG, s_cw, s_cdw);
    __syncthreads();

    // 4. emit: continuing survivors deflate in place, run ends become active poles
    T4 carry{0.0, 0.0, 0.0, 0.0};
    int K = 0;
    double zsq = 0.0;
    for (int c0 = 0; c0 < S; c0 += NT) {
      const int k = c0 + tid;
      const bool valid = k < S;
      int pos = 0;
      bool head = true;
      double Dk = 0.0, zk = 0.0, rl = 0.0, rh = 0.0;
      T4 own{0.0, 0.0, 0.0, 0.0};
      if (valid) {
        pos = SURV[k] - lo;
        head = RFLAG[k] != 0;
        Dk = D[pos];
        zk = Z[pos];
        rl = RLO[pos];
        rh = RHI[pos];
        double wk = zk * zk;
        own = T4{wk, Dk * wk, zk * rl, zk * rh};
      }
      // block segmented inclusive scan with carry-in (warps past S hold no survivor)
      T4 v = own;
      bool h = head;
      if (c0 + warp * 32 < S) {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          T4 vo = t4_shfl_up(v, o);
          bool ho = __shfl_up_sync(0xffffffffu, h, o);
          if (lane >= o) {
            if (!h) v = t4_add(v, vo);
            h = h || ho;
          }
        }
      }
      if (lane == 31) {
        s_agg[warp] = v;
        s_aggh[warp] = h ? 1 : 0;
      }
      __syncthreads();
      if (warp == 0) {  // prefix of each warp: carry, then the warp aggregates before it
        T4 inc = lane < NT / 32 ? s_agg[lane] : T4{0.0, 0.0, 0.0, 0.0};
        bool hh = lane < NT / 32 ? s_aggh[lane] != 0 : true;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          T4 vo = t4_shfl_up(inc, o);
          bool ho = __shfl_up_sync(0xffffffffu, hh, o);
          if (lane >= o) {
            if (!hh) inc = t4_add(inc, vo);
            hh = hh || ho;
          }
        }
        const T4 pv = t4_shfl_up(inc, 1);
        const bool ph = __shfl_up_sync(0xffffffffu, hh, 1);
        if (lane < NT / 32) s_pre[lane] = lane == 0 ? carry : (ph ? pv : t4_add(carry, pv));
      }
      __syncthreads();
      if (!h) v = t4_add(v, s_pre[warp]);
      s_incl[tid] = v;
      __syncthreads();
      const T4 prev = (tid > 0) ? s_incl[tid - 1] : carry;
      bool runend = false;
      if (valid) runend = (k == S - 1) || RFLAG[k + 1] != 0;
      int ex_total;
      int act = block_excl_scan<NT>(runend ? 1 : 0, sm_int, &ex_total);
      double zact2 = 0.0;
      if (valid && !head) {
        // deflated by rotation against the run prefix `prev`
        double Wp = prev.w, wk = own.w;
        double c = prev.dw / Wp;
        double val = (wk * c + Wp * Dk) / (Wp + wk);
        double sc = 1.0 / sqrt(Wp * (Wp + wk));
        D[pos] = val;
        RLO[pos] = (zk * prev.ulo - Wp * rl) * sc;
        RHI[pos] = (zk * prev.uhi - Wp * rh) * sc;
        PFLAG[pos] = 2;
        a.KEEPIDX[lo + pos] = K + act;  // its run ends in the next run end, active index K + act
      }
      if (valid && runend) {
        a.ACTMAP[lo + k] = K + act;
        double ad, az, al, ah;
        if (head) {
          ad = Dk;
          az = zk;
          al = rl;
          ah = rh;
        } else {
          double W = v.w;
          az = sqrt(W);
          ad = v.dw / W;
          double inv = 1.0 / az;
          al = v.ulo * inv;
          ah = v.uhi * inv;
        }
        int idx = lo + K + act;
        a.AD[idx] = ad;
        a.AZ[idx] = az;
        a.ALO[idx] = al;
        a.AHI[idx] = ah;
        zact2 = az * az;
      }
      zsq += block_sum<NT>(zact2, sm_dbl);
      K += ex_total;
      // carry: inclusive value of the last survivor of this chunk
      int last = min(NT - 1, S - 1 - c0);
      carry = s_incl[last];
      __syncthreads();
    }

    // 5. deflated eigenvalues: those deflated for a negligible z (PFLAG 1) keep the
    //    ascending order of D; rotated ones (PFLAG 2) may be out of order.  Collect
    //    the positions of each kind, in position order.
    int32_t* ZPOS = a.ZPOS + lo;  // SURV stays intact for the adjoint
    int32_t* RPOS = a.IDXA + lo;
    int FZ = 0, FR = 0;
    for (int c0 = 0; c0 < n0; c0 += NT) {
      const int i = c0 + tid;
      const int pf = i < n0 ? PFLAG[i] : 0;
      const int both = (pf == 1 ? 1 : 0) | (pf == 2 ? (1 << 16) : 0);
      int total;
      const int ex = block_excl_scan<NT>(both, sm_int, &total);
      if (pf == 1) ZPOS[FZ + (ex & 0xffff)] = i;
      if (pf == 2) RPOS[FR + (ex >> 16)] = i;
      FZ += total & 0xffff;
      FR += total >> 16;
    }
    if (tid == 0) s_flag = 0;
    __syncthreads();
    // 6. sort the rotated ones by value if they are out of order
    for (int k = tid; k + 1 < FR; k += NT)
      if (D[RPOS[k]] > D[RPOS[k + 1]]) s_flag = 1;
    __syncthreads();
    if (s_flag) {
      if (tid == 0) {
        atomicAdd(&a.st->work[kWorkSorts], 1ull);
        atomicAdd(&a.st->work[kWorkSortedEntries], (unsigned long long)FR);
      }
      for (int k = tid; k < FR; k += NT) a.KEYA[lo + k] = order_key(D[RPOS[k]]);
      __syncthreads();
      const int which = block_sort(FR, a.KEYA + lo, a.IDXA + lo, a.KEYB + lo, a.IDXB + lo, s_key, s_idx);
      if (which) RPOS = a.IDXB + lo;
    }
    __syncthreads();
    // 7. merge the two ascending lists into AD / ALO / AHI after the K active poles
    for (int k = tid; k < FZ; k += NT) {
      const int pos = ZPOS[k];
      const double x = D[pos];
      int l = 0, h = FR;  // rotated entries strictly below x come first
      while (l < h) {
        const int md = (l + h) >> 1;
        if (D[RPOS[md]] < x) l = md + 1; else h = md;
      }
      const int dst = lo + K + k + l;
      a.AD[dst] = x;
      a.ALO[dst] = RLO[pos];
      a.AHI[dst] = RHI[pos];
      a.OUTIDX[lo + pos] = K + k + l;
    }
    for (int k = tid; k < FR; k += NT) {
      const int pos = RPOS[k];
      const double x = D[pos];
      int l = 0, h = FZ;  // negligible-z entries at or below x come first
      while (l < h) {
        const int md = (l + h) >> 1;
        if (D[ZPOS[md]] <= x) l = md + 1; else h = md;
      }
      const int dst = lo + K + k + l;
      a.AD[dst] = x;
      a.ALO[dst] = RLO[pos];
      a.AHI[dst] = RHI[pos];
      a.OUTIDX[lo + pos] = K + k + l;
    }
    __syncthreads();
    // 8. single-precision copies of the active poles for the first stage of the
    //    secular solver: D_i - shift as an unevaluated float pair hi + lo (about 48
    //    bits relative to the spread of the merge's poles, not to their magnitude:
    //    the offsets D_i - D_org the solver forms are shift-invariant) and z_i
    //    rounded to float.  KEYB / IDXB held the sort scratch until here.
    const double shift = K > 0 ? 0.5 * (a.AD[lo] + a.AD[lo + K - 1]) : 0.0;
    {
      float2* AD32 = reinterpret_cast<float2*>(a.KEYB) + lo;
      float* AZ32 = reinterpret_cast<float*>(a.IDXB) + lo;
      for (int k = tid; k < K; k += NT) {
        const double x = a.AD[lo + k] - shift;
        const float hi = __double2float_rn(x);
        AD32[k] = make_float2(hi, __double2float_rn(x - double(hi)));
        AZ32[k] = __double2float_rn(a.AZ[lo + k]);
      }
    }
    // 9. roots of this merge get a contiguous range of one of the step's two root
    //    lists: merges with K >= warp_min_k are solved one warp per root.  In a
    //    forest a small-K merge only counts its roots into its bin of K here, and
    //    k_order_assign gives it its range once the step's histogram is complete.
    __shared__ int s_base;
    const bool big = K >= a.warp_min_k;
    const bool ordered = a.order_small != 0 && !big;
    if (tid == 0) {
      s_base = K > 0 ? int(atomicAdd(big ? &a.st->root_count_big[a.step] : &a.st->root_count[a.step],
                                     unsigned(K)))
                     : 0;
      if (ordered && K > 0) atomicAdd(&a.st->order_hist[min(K, kOrderBins - 1)], unsigned(K));
      MState st;
      st.K = K;
      st.base = ordered ? 0 : s_base;
      st.rho = rho;
      st.rhoinv = 1.0 / rho;
      st.zsq = zsq;
      st.big = big ? 1 : 0;
      st.surv = S;
      st.shift = shift;
      a.ms[g] = st;
      atomicAdd(&a.st->work[kWorkDeflated], (unsigned long long)(n0 - K));
      atomicAdd(&a.st->work[kWorkRotations], (unsigned long long)(S - K));
    }
    __syncthreads();
    int32_t* rmap = big ? a.ROOTMAP2 : a.ROOTMAP;
    if (!ordered)
      for (int j = tid; j < K; j += NT) rmap[s_base + j] = int32_t(g);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Deflation of a few large merges by thread-block clusters: the C CTAs of a
// cluster share one merge, so its element-wise work (the FP64 run sums, rotations
// and compaction of steps 2-5, 7-9 of k_deflate) is spread over C SMs instead of
// one.  The steps, the run boundaries and the deflation decisions are those of
// k_deflate; the segmented run sums are associated by CTA, so the rotated values
// can differ from k_deflate's in the last bits (glued Wilkinson blocks, n = 2048:
// eigenvalues within 8.9e-16).  What changes is how the sequential pieces are cut:
//   * compactions (steps 2 and 5) count per CTA slice, exchange the counts and
//     write at the exclusive prefix of the CTAs before;
//   * run boundaries (step 3): each warp of the cluster walks one segment of the
//     survivors speculatively (k_deflate's rule), then all segments re-check their
//     start against their predecessor's final carry in parallel rounds until no
//     carry changes.  Segment 0 is exact, and a round in which segment s re-walks
//     against an exact predecessor makes it exact, so at most one round per
//     segment is needed (usually one in all);
//   * the segmented run sums (step 4) take as carry-in the sum from the last run
//     start in the CTAs before, from per-CTA aggregates;
//   * the sort of rotated eigenvalues (step 6) is spread over the C CTAs (cluster_sort).
// Values a CTA publishes live in its shared memory (ClusterSlot) and are read
// through distributed shared memory after a cluster barrier; each field is
// written once per merge and the merge loop ends with a barrier before reuse.
struct ClusterSlot {
  double zmax, zsq;
  T4 agg;
  int nkeep, nend, has_head, nz, nr, unsorted, which, base;
  int changed[2];
};

// Cluster barrier ordering this thread's global writes before the other CTAs' reads
// (the barrier's arrive has release and its wait acquire semantics at cluster
// scope, which covers global memory).
__device__ __forceinline__ void cluster_sync_mem(cg::cluster_group& cl) { cl.sync(); }

// block_sort over the C CTAs of a cluster: CTA r sorts the tiles r, r + C, ... and
// takes the entries r NT + tid, stride C NT, of every merge pass; cluster barriers
// (which order the global writes) separate the passes.  Same passes, same result.
__device__ int cluster_sort(cg::cluster_group& cl, int r, int C, int n, unsigned long long* KA,
                            int32_t* IA, unsigned long long* KB, int32_t* IB,
                            unsigned long long* skey, int32_t* sidx) {
  for (int t0 = r * kTile; t0 < n; t0 += C * kTile) sort_tile(t0, min(kTile, n - t0), KA, IA, skey, sidx);
  cluster_sync_mem(cl);
  int which = 0;
  unsigned long long *src_k = KA, *dst_k = KB;
  int32_t *src_i = IA, *dst_i = IB;
  for (int width = kTile; width < n; width <<= 1) {
    merge_pass(n, width, r * int(blockDim.x) + int(threadIdx.x), C * int(blockDim.x), src_k, src_i,
               dst_k, dst_i);
    cluster_sync_mem(cl);
    unsigned long long* tk = src_k;
    src_k = dst_k;
    dst_k = tk;
    int32_t* ti = src_i;
    src_i = dst_i;
    dst_i = ti;
    which ^= 1;
  }
  return which;
}

// Sum of an int field over the ranks before r and over all C ranks, computed by
// every warp on its own (lane q reads rank q).
template <class F>
__device__ __forceinline__ void cluster_scan_int(cg::cluster_group& cl, ClusterSlot& slot, int C,
                                                 int r, F field, int* before, int* total) {
  const int lane = threadIdx.x & 31;
  int v = lane < C ? field(*cl.map_shared_rank(&slot, lane)) : 0;
  int b = lane < r ? v : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v += __shfl_xor_sync(0xffffffffu, v, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  *before = b;
  *total = v;
}

template <int NT>
__device__ __forceinline__ int block_max_int(int v, int* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = __reduce_max_sync(0xffffffffu, v);
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  const int r = __reduce_max_sync(0xffffffffu, sm[lane < NT / 32 ? lane : 0]);
  __syncthreads();
  return r;
}

template <int NT>
__global__ void __launch_bounds__(NT, 1) k_deflate_cluster(DeflateArgs a) {
  constexpr int NW = NT / 32;
  __shared__ int sm_int[NW];
  __shared__ double sm_dbl[NW];
  __shared__ T4 s_agg[NW];
  __shared__ int s_aggh[NW];
  __shared__ T4 s_pre[NW];
  __shared__ T4 s_incl[NT];
  __shared__ unsigned long long s_key[kTile];
  __shared__ int32_t s_idx[kTile];
  __shared__ double s_cw[2][NW], s_cdw[2][NW];
  __shared__ T4 s_carry;
  __shared__ ClusterSlot slot;
  cg::cluster_group cl = cg::this_cluster();
  const int C = int(cl.num_blocks()), r = int(cl.block_rank());
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t ncl = gridDim.x / C;

  for (int64_t g = blockIdx.x / C; g < a.cnt; g += ncl) {
    const Merge m = a.M[g];
    const int lo = m.lo, n0 = m.hi - m.lo;
    const double rho = 2.0 * fabs(a.es[m.mid - 1]);
    double* D = a.D + lo;
    double* Z = a.Z + lo;
    double* RLO = a.RLO + lo;
    double* RHI = a.RHI + lo;
    uint8_t* PFLAG = a.PFLAG + lo;
    int32_t* SURV = a.SURV + lo;
    uint8_t* RFLAG = a.RFLAG + lo;
    const int L = (n0 + C - 1) / C;  // positions of this CTA: [eb, ee)
    const int eb = min(n0, r * L), ee = min(n0, eb + L);

    // 1. tol = 8 eps max(max|D|, max|z|)
    double zm = 0.0;
    for (int i = eb + tid; i < ee; i += NT) zm = fmax(zm, fabs(Z[i]));
    zm = block_max<NT>(zm, sm_dbl);
    if (tid == 0) slot.zmax = zm;
    cl.sync();
    zm = lane < C ? cl.map_shared_rank(&slot, lane)->zmax : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) zm = fmax(zm, __shfl_xor_sync(0xffffffffu, zm, o));
    const double dmax = fmax(fabs(D[0]), fabs(D[n0 - 1]));
    const double tol = 8.0 * kEps * fmax(dmax, zm);
    const double tol2 = tol * tol;

    // 2. negligible z, compacted into SURV at the survivors of the CTAs before
    int cnt = 0;
    for (int c0 = eb; c0 < ee; c0 += NT) {
      const int i = c0 + tid;
      int keep = 0;
      if (i < ee) {
        keep = rho * fabs(Z[i]) > tol ? 1 : 0;
        PFLAG[i] = keep ? 0 : 1;
      }
      cnt += __syncthreads_count(keep);
    }
    if (tid == 0) slot.nkeep = cnt;
    cl.sync();
    int off, S;
    cluster_scan_int(cl, slot, C, r, [](const ClusterSlot& x) { return x.nkeep; }, &off, &S);
    for (int c0 = eb; c0 < ee; c0 += NT) {
      const int i = c0 + tid;
      const int keep = (i < ee && rho * fabs(Z[i]) > tol) ? 1 : 0;
      int total;
      const int ex = block_excl_scan<NT>(keep, sm_int, &total);
      if (keep) SURV[off + ex] = lo + i;
      off += total;
    }
    cluster_sync_mem(cl);

    // 3. run boundaries: speculative walk per warp segment, then parallel rounds in
    //    which a segment walks again only when the carry it receives differs (bit for
    //    bit) from the one it last walked with: the same carry gives the same
    //    decisions and the same carry out, and the walk is FP64-bound
    {
      const int NS = C * NW;
      const int seg = ((S + NS - 1) / NS + 31) & ~31;
      const int sid = r * NW + warp;
      const int b = min(S, sid * seg), e = min(S, b + seg);
      double cW = 0.0, cDW = 0.0;
      double inW = 0.0, inDW = 0.0;  // carry of the segment's last walk
      if (b < e) {
        bool have = false;
        if (b > 0) {
          const int pos = SURV[b - 1];
          const double z = a.Z[pos];
          cW = __dmul_rn(z, z);
          cDW = __dmul_rn(a.D[pos], cW);
          have = true;
        }
        inW = cW;
        inDW = cDW;
        run_segment(b, e, SURV, a.D, a.Z, tol2, RFLAG, cW, cDW, have, false);
      }
      if (lane == 0) {
        s_cw[0][warp] = cW;
        s_cdw[0][warp] = cDW;
      }
      cluster_sync_mem(cl);
      int cur = 0;
      bool converged = false;
      for (int round = 0; round <= NS; ++round) {
        double nW = s_cw[cur][warp], nDW = s_cdw[cur][warp];
        bool changed = false;
        if (b < e && sid > 0) {
          const int pr = (sid - 1) / NW, pw = (sid - 1) % NW;
          double W = cl.map_shared_rank(&s_cw[cur][0], pr)[pw];
          double DW = cl.map_shared_rank(&s_cdw[cur][0], pr)[pw];
          const bool same_in = __double_as_longlong(W) == __double_as_longlong(inW) &&
                               __double_as_longlong(DW) == __double_as_longlong(inDW);
          inW = W;
          inDW = DW;
          if (!same_in && run_segment(b, e, SURV, a.D, a.Z, tol2, RFLAG, W, DW, true, true)) {
            changed = __double_as_longlong(W) != __double_as_longlong(nW) ||
                      __double_as_longlong(DW) != __double_as_longlong(nDW);
            nW = W;
            nDW = DW;
          }
        }
        if (lane == 0) {
          s_cw[cur ^ 1][warp] = nW;
          s_cdw[cur ^ 1][warp] = nDW;
        }
        const int any = __syncthreads_or(changed ? 1 : 0);
        if (tid == 0) slot.changed[round & 1] = any;
        cluster_sync_mem(cl);
        int anyc = lane < C ? cl.map_shared_rank(&slot, lane)->changed[round & 1] : 0;
        anyc = __any_sync(0xffffffffu, anyc != 0) ? 1 : 0;
        cur ^= 1;
        if (!anyc) {
          converged = true;
          break;
        }
      }
      if (!converged && r == 0 && tid == 0) set_status(a.st, TDE_ENOCONV);
    }

    // 4. emit over this CTA's survivors [sb, se): the carry-in is the run sum from
    //    the last run start in the CTAs before
    const int LS = (S + C - 1) / C;
    const int sb = min(S, r * LS), se = min(S, sb + LS);
    {
      int hl = -1, nend = 0;
      for (int c0 = sb; c0 < se; c0 += NT) {
        const int k = c0 + tid;
        bool end = false;
        if (k < se) {
          if (RFLAG[k] != 0) hl = k;
          end = (k == S - 1) || RFLAG[k + 1] != 0;
        }
        nend += __syncthreads_count(end ? 1 : 0);
      }
      hl = block_max_int<NT>(hl, sm_int);
      T4 acc{0.0, 0.0, 0.0, 0.0};
      for (int k = max(hl, sb) + tid; k < se; k += NT) {
        const int pos = SURV[k] - lo;
        const double zk = Z[pos], wk = zk * zk;
        acc = t4_add(acc, T4{wk, D[pos] * wk, zk * RLO[pos], zk * RHI[pos]});
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc = t4_add(acc, t4_shfl_xor(acc, o));
      if (lane == 0) s_agg[warp] = acc;
      __syncthreads();
      if (warp == 0) {
        T4 x = lane < NW ? s_agg[lane] : T4{0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = t4_add(x, t4_shfl_xor(x, o));
        acc = x;
      }
      if (tid == 0) {
        slot.agg = acc;
        slot.has_head = hl >= 0 ? 1 : 0;
        slot.nend = nend;
      }
    }
    cl.sync();
    if (tid == 0) {
      T4 c{0.0, 0.0, 0.0, 0.0};
      for (int q = r - 1; q >= 0; --q) {
        const ClusterSlot* p = cl.map_shared_rank(&slot, q);
        c = t4_add(p->agg, c);
        if (p->has_head) break;
      }
      s_carry = c;
    }
    int K, Ktot;
    cluster_scan_int(cl, slot, C, r, [](const ClusterSlot& x) { return x.nend; }, &K, &Ktot);
    __syncthreads();
    T4 carry = s_carry;
    double zsq = 0.0;
    for (int c0 = sb; c0 < se; c0 += NT) {
      const int k = c0 + tid;
      const bool valid = k < se;
      int pos = 0;
      bool head = true;
      double Dk = 0.0, zk = 0.0, rl = 0.0, rh = 0.0;
      T4 own{0.0, 0.0, 0.0, 0.0};
      if (valid) {
        pos = SURV[k] - lo;
        head = RFLAG[k] != 0;
        Dk = D[pos];
        zk = Z[pos];
        rl = RLO[pos];
        rh = RHI[pos];
        double wk = zk * zk;
        own = T4{wk, Dk * wk, zk * rl, zk * rh};
      }
      T4 v = own;
      bool h = head;
      if (c0 + warp * 32 < se) {  // warps past the slice hold no survivor
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          T4 vo = t4_shfl_up(v, o);
          bool ho = __shfl_up_sync(0xffffffffu, h, o);
          if (lane >= o) {
            if (!h) v = t4_add(v, vo);
            h = h || ho;
          }
        }
      }
      if (lane == 31) {
        s_agg[warp] = v;
        s_aggh[warp] = h ? 1 : 0;
      }
      __syncthreads();
      if (warp == 0) {
        T4 inc = lane < NW ? s_agg[lane] : T4{0.0, 0.0, 0.0, 0.0};
        bool hh = lane < NW ? s_aggh[lane] != 0 : true;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          T4 vo = t4_shfl_up(inc, o);
          bool ho = __shfl_up_sync(0xffffffffu, hh, o);
          if (lane >= o) {
            if (!hh) inc = t4_add(inc, vo);
            hh = hh || ho;
          }
        }
        const T4 pv = t4_shfl_up(inc, 1);
        const bool ph = __shfl_up_sync(0xffffffffu, hh, 1);
        if (lane < NW) s_pre[lane] = lane == 0 ? carry : (ph ? pv : t4_add(carry, pv));
      }
      __syncthreads();
      if (!h) v = t4_add(v, s_pre[warp]);
      s_incl[tid] = v;
      __syncthreads();
      const T4 prev = (tid > 0) ? s_incl[tid - 1] : carry;
      bool runend = false;
      if (valid) runend = (k == S - 1) || RFLAG[k + 1] != 0;
      int ex_total;
      int act = block_excl_scan<NT>(runend ? 1 : 0, sm_int, &ex_total);
      double zact2 = 0.0;
      if (valid && !head) {
        double Wp = prev.w, wk = own.w;
        double c = prev.dw / Wp;
        double val = (wk * c + Wp * Dk) / (Wp + wk);
        double sc = 1.0 / sqrt(Wp * (Wp + wk));
        D[pos] = val;
        RLO[pos] = (zk * prev.ulo - Wp * rl) * sc;
        RHI[pos] = (zk * prev.uhi - Wp * rh) * sc;
        PFLAG[pos] = 2;
        a.KEEPIDX[lo + pos] = K + act;
      }
      if (valid && runend) {
        a.ACTMAP[lo + k] = K + act;
        double ad, az, al, ah;
        if (head) {
          ad = Dk;
          az = zk;
          al = rl;
          ah = rh;
        } else {
          double W = v.w;
          az = sqrt(W);
          ad = v.dw / W;
          double inv = 1.0 / az;
          al = v.ulo * inv;
          ah = v.uhi * inv;
        }
        int idx = lo + K + act;
        a.AD[idx] = ad;
        a.AZ[idx] = az;
        a.ALO[idx] = al;
        a.AHI[idx] = ah;
        zact2 = az * az;
      }
      zsq += block_sum<NT>(zact2, sm_dbl);
      K += ex_total;
      int last = min(NT - 1, se - 1 - c0);
      carry = s_incl[last];
      __syncthreads();
    }
    if (tid == 0) slot.zsq = zsq;
    cluster_sync_mem(cl);
    K = Ktot;
    if (r == 0 && tid == 0) {  // only the thread writing the merge state needs it
      zsq = 0.0;
      for (int q = 0; q < C; ++q) zsq += cl.map_shared_rank(&slot, q)->zsq;
    }

    // 5. deflated positions of each kind, in position order, over the CTA slices
    int32_t* ZPOS = a.ZPOS + lo;
    int32_t* RPOS = a.IDXA + lo;
    {
      int nz = 0, nr = 0;
      for (int c0 = eb; c0 < ee; c0 += NT) {
        const int i = c0 + tid;
        const int pf = i < ee ? PFLAG[i] : 0;
        nz += __syncthreads_count(pf == 1);
        nr += __syncthreads_count(pf == 2);
      }
      if (tid == 0) {
        slot.nz = nz;
        slot.nr = nr;
      }
    }
    cl.sync();
    int FZ, FR, oz, orr;
    cluster_scan_int(cl, slot, C, r, [](const ClusterSlot& x) { return x.nz; }, &oz, &FZ);
    cluster_scan_int(cl, slot, C, r, [](const ClusterSlot& x) { return x.nr; }, &orr, &FR);
    for (int c0 = eb; c0 < ee; c0 += NT) {
      const int i = c0 + tid;
      const int pf = i < ee ? PFLAG[i] : 0;
      const int both = (pf == 1 ? 1 : 0) | (pf == 2 ? (1 << 16) : 0);
      int total;
      const int ex = block_excl_scan<NT>(both, sm_int, &total);
      if (pf == 1) ZPOS[oz + (ex & 0xffff)] = i;
      if (pf == 2) RPOS[orr + (ex >> 16)] = i;
      oz += total & 0xffff;
      orr += total >> 16;
    }
    cluster_sync_mem(cl);

    // 6. sort the rotated ones by value if they are out of order (CTA 0)
    {
      int bad = 0;
      for (int k = r * NT + tid; k + 1 < FR; k += C * NT)
        if (D[RPOS[k]] > D[RPOS[k + 1]]) bad = 1;
      bad = __syncthreads_or(bad);
      if (tid == 0) slot.unsorted = bad;
    }
    cl.sync();
    int unsorted = lane < C ? cl.map_shared_rank(&slot, lane)->unsorted : 0;
    unsorted = __any_sync(0xffffffffu, unsorted != 0) ? 1 : 0;
    if (unsorted) {
      if (r == 0 && tid == 0) {
        atomicAdd(&a.st->work[kWorkSorts], 1ull);
        atomicAdd(&a.st->work[kWorkSortedEntries], (unsigned long long)FR);
      }
      for (int k = r * NT + tid; k < FR; k += C * NT) a.KEYA[lo + k] = order_key(D[RPOS[k]]);
      cluster_sync_mem(cl);
      const int which =
          cluster_sort(cl, r, C, FR, a.KEYA + lo, a.IDXA + lo, a.KEYB + lo, a.IDXB + lo, s_key, s_idx);
      if (which) RPOS = a.IDXB + lo;
    }

    // 7. merge the two ascending lists after the K active poles
    for (int k = r * NT + tid; k < FZ; k += C * NT) {
      const int pos = ZPOS[k];
      const double x = D[pos];
      int l = 0, h = FR;
      while (l < h) {
        const int md = (l + h) >> 1;
        if (D[RPOS[md]] < x) l = md + 1; else h = md;
      }
      const int dst = lo + K + k + l;
      a.AD[dst] = x;
      a.ALO[dst] = RLO[pos];
      a.AHI[dst] = RHI[pos];
      a.OUTIDX[lo + pos] = K + k + l;
    }
    for (int k = r * NT + tid; k < FR; k += C * NT) {
      const int pos = RPOS[k];
      const double x = D[pos];
      int l = 0, h = FZ;
      while (l < h) {
        const int md = (l + h) >> 1;
        if (D[ZPOS[md]] <= x) l = md + 1; else h = md;
      }
      const int dst = lo + K + k + l;
      a.AD[dst] = x;
      a.ALO[dst] = RLO[pos];
      a.AHI[dst] = RHI[pos];
      a.OUTIDX[lo + pos] = K + k + l;
    }
    cluster_sync_mem(cl);  // KEYB / IDXB (sort scratch, RPOS) are reused below

    // 8. single-precision pole copies (k_deflate step 8)
    const double shift = K > 0 ? 0.5 * (a.AD[lo] + a.AD[lo + K - 1]) : 0.0;
    {
      float2* AD32 = reinterpret_cast<float2*>(a.KEYB) + lo;
      float* AZ32 = reinterpret_cast<float*>(a.IDXB) + lo;
      for (int k = r * NT + tid; k < K; k += C * NT) {
        const double x = a.AD[lo + k] - shift;
        const float hi = __double2float_rn(x);
        AD32[k] = make_float2(hi, __double2float_rn(x - double(hi)));
        AZ32[k] = __double2float_rn(a.AZ[lo + k]);
      }
    }
    // 9. root list range and merge state (CTA 0), then the root map (a forest's
    //    small-K merge takes its range from k_order_assign instead)
    const bool big = K >= a.warp_min_k;
    const bool ordered = a.order_small != 0 && !big;
    if (r == 0 && tid == 0) {
      const int base = K > 0 ? int(atomicAdd(big ? &a.st->root_count_big[a.step]
                                                 : &a.st->root_count[a.step],
                                             unsigned(K)))
                             : 0;
      if (ordered && K > 0) atomicAdd(&a.st->order_hist[min(K, kOrderBins - 1)], unsigned(K));
      MState st;
      st.K = K;
      st.base = ordered ? 0 : base;
      st.rho = rho;
      st.rhoinv = 1.0 / rho;
      st.zsq = zsq;
      st.big = big ? 1 : 0;
      st.surv = S;
      st.shift = shift;
      a.ms[g] = st;
      slot.base = base;
      atomicAdd(&a.st->work[kWorkDeflated], (unsigned long long)(n0 - K));
      atomicAdd(&a.st->work[kWorkRotations], (unsigned long long)(S - K));
    }
    cl.sync();
    const int base = cl.map_shared_rank(&slot, 0)->base;
    int32_t* rmap = big ? a.ROOTMAP2 : a.ROOTMAP;
    if (!ordered)
      for (int j = r * NT + tid; j < K; j += C * NT) rmap[base + j] = int32_t(g);
    cl.sync();  // the slots are rewritten by the next merge
  }
}

// ---------------------------------------------------------------------------
__global__ void k_place(const Merge* __restrict__ M, int64_t cnt, int64_t nrows,
                        const MState* __restrict__ ms, const double* __restrict__ LAMA,
                        const double* __restrict__ ROWLO, const double* __restrict__ ROWHI,
                        const double* __restrict__ AD, const double* __restrict__ ALO,
                        const double* __restrict__ AHI,
                        const unsigned long long* __restrict__ sigma_bits, double* LAM,
                        double* BLO, double* BHI, double* out) {
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < nrows;
       p += int64_t(gridDim.x) * blockDim.x) {
    const int64_t g = find_merge(M, cnt, p);
    const Merge m = M[g];
    if (p < m.lo || p >= m.hi) continue;
    const int K = ms[g].K, lo = m.lo, F = (m.hi - m.lo) - K;
    const int local = int(p - lo);
    double x, rl, rh;
    int rank;
    if (local < K) {
      x = LAMA[p];
      rank = local + count_less(AD + lo + K, F, x);
      rl = ROWLO[p];
      rh = ROWHI[p];
    } else {
      x = AD[p];
      rank = (local - K) + count_leq(LAMA + lo, K, x);
      rl = ALO[p];
      rh = AHI[p];
    }
    const int dst = lo + rank;
    if (uint32_t(m.info) & kRootBit) {
      double s = __longlong_as_double((long long)sigma_bits[uint32_t(m.info) & kMatMask]);
      int ex = (s > 0.0 && isfinite(s)) ? ilogb(s) : 0;
      out[dst] = ldexp(x, ex);
    } else {
      LAM[dst] = x;
      BLO[dst] = rl;
      BHI[dst] = rh;
    }
  }
}

// ---------------------------------------------------------------------------
void launch_form(const Plan& plan, const Workspace& ws, int step, LevelState in, cudaStream_t s) {
  const Merge* M = ws.merges + plan.step_base[step];
  const int64_t nrows = plan.nrows;
  const int flat_grid = int(std::min<int64_t>((nrows + 255) / 256, 148 * 8));
  k_form<<<flat_grid, 256, 0, s>>>(M, plan.step_count[step], nrows, in.lam, in.blo, in.bhi, ws.es,
                                   ws.D, ws.Z, ws.RLO, ws.RHI);
}

// Cluster size for steps with few large merges: as many CTAs per merge as fill the
// SMs once (at most 16, the non-portable maximum, if a 16-CTA cluster of
// 1024-thread CTAs fits this device; 8 otherwise).  0 selects the one-CTA kernels.
static int deflate_cluster_size(int64_t cnt, int64_t maxsize) {
  // fit[k]: how many clusters of 2^k CTAs this device runs at once (queried once)
  static int fit[5] = {-1, 0, 0, 0, 0};
  if (fit[0] < 0) {
    fit[0] = 0;
    const bool np = cudaFuncSetAttribute(k_deflate_cluster<1024>,
                                         cudaFuncAttributeNonPortableClusterSizeAllowed,
                                         1) == cudaSuccess;
    for (int k = 1; k <= 4; ++k) {
      if (k == 4 && !np) break;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(1u << k);
      cfg.blockDim = dim3(1024);
      cudaLaunchAttribute at;
      at.id = cudaLaunchAttributeClusterDimension;
      at.val.clusterDim.x = 1u << k;
      at.val.clusterDim.y = 1;
      at.val.clusterDim.z = 1;
      cfg.attrs = &at;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, k_deflate_cluster<1024>, &cfg) == cudaSuccess)
        fit[k] = n;
    }
    cudaGetLastError();  // a refused query leaves no sticky error
  }
  if (maxsize < 1024 || cnt < 1) return 0;
  // the largest cluster size whose clusters for all cnt merges run in one wave
  for (int k = 4; k >= 1; --k)
    if (fit[k] >= cnt) return 1 << k;
  return 0;
}

// ---------------------------------------------------------------------------
// A forest's small-K root list in descending order of K.  The deflation kernels
// count each small-K merge's roots into its bin of K (Status::order_hist);
// k_order_cursor turns that histogram into each bin's first list entry and
// clears it for the next step, and k_order_assign gives every small-K merge of
// the step its contiguous range (one atomic on its bin's cursor) and writes the
// root map.  Which merges share a bin, and in which order, changes no result: a
// root depends only on its own merge, wherever it sits in the list.
__global__ void __launch_bounds__(kOrderBins) k_order_cursor(Status* st) {
  __shared__ uint32_t s[kOrderBins];
  const int t = threadIdx.x;
  const int bin = kOrderBins - 1 - t;  // position t holds the t-th largest bin
  const uint32_t v = st->order_hist[bin];
  st->order_hist[bin] = 0u;
  s[t] = v;
  __syncthreads();
  for (int o = 1; o < kOrderBins; o <<= 1) {  // inclusive scan over positions
    const uint32_t add = t >= o ? s[t - o] : 0u;
    __syncthreads();
    s[t] += add;
    __syncthreads();
  }
  st->order_cursor[bin] = s[t] - v;
}

__global__ void __launch_bounds__(256) k_order_assign(int64_t cnt, MState* __restrict__ ms,
                                                       Status* st, int32_t* __restrict__ ROOTMAP) {
  __shared__ int s_base[256], s_K[256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t g0 = int64_t(blockIdx.x) * 256; g0 < cnt; g0 += int64_t(gridDim.x) * 256) {
    const int64_t g = g0 + threadIdx.x;
    int K = 0, base = 0;
    if (g < cnt) {
      const MState m = ms[g];
      if (m.K > 0 && !m.big) {
        K = m.K;
        base = int(atomicAdd(&st->order_cursor[min(K, kOrderBins - 1)], unsigned(K)));
        ms[g].base = base;
      }
    }
    s_base[threadIdx.x] = base;
    s_K[threadIdx.x] = K;
    __syncthreads();
    for (int q = warp; q < 256; q += 8) {  // the root map, one warp per merge
      const int Kq = s_K[q], bq = s_base[q];
      for (int jj = lane; jj < Kq; jj += 32) ROOTMAP[bq + jj] = int32_t(g0 + q);
    }
    __syncthreads();
  }
}

void launch_deflate(const DeflateArgs& da, int64_t maxsize, cudaStream_t s) {
  const int64_t cnt = da.cnt;
  const int c = deflate_cluster_size(cnt, maxsize);
  if (c > 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(cnt * c));
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = unsigned(c);
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_deflate_cluster<1024>, da);
    return;
  }
  if (maxsize > 8192)
    k_deflate<1024><<<int(std::min<int64_t>(cnt, 148 * 8)), 1024, 0, s>>>(da);
  else if (maxsize > 64)
    k_deflate<kNT><<<int(std::min<int64_t>(cnt, 148 * 8)), kNT, 0, s>>>(da);
  else
    k_deflate<64><<<int(std::min<int64_t>(cnt, 148 * 32)), 64, 0, s>>>(da);
}

void launch_step(const Plan& plan, const Workspace& ws, int step, double* lambda, cudaStream_t s,
                 LevelState in, LevelState out, bool recompute, const SelArgs* sel,
                 double* rows_inu, const RootsCheckpoint* roots) {
  const Merge* M = ws.merges + plan.step_base[step];
  const int64_t cnt = plan.step_count[step];
  const int64_t nrows = plan.nrows;
  const int flat_grid = int(std::min<int64_t>((nrows + 255) / 256, 148 * 8));
  prof_begin(kKForm, s);
  launch_form(plan, ws, step, in, s);
  prof_end(kKForm, s);
  if (sel) {
    prof_begin(kKSel, s);
    launch_sel_form(plan, ws, *sel, step, in, s);
    prof_end(kKSel, s);
  }
  DeflateArgs da;
  da.M = M;
  da.cnt = cnt;
  da.step = step;
  da.es = ws.es;
  da.D = ws.D;
  da.Z = ws.Z;
  da.RLO = ws.RLO;
  da.RHI = ws.RHI;
  da.AD = ws.AD;
  da.AZ = ws.AZ;
  da.ALO = ws.ALO;
  da.AHI = ws.AHI;
  da.SURV = ws.SURV;
  da.ROOTMAP = ws.ROOTMAP;
  da.ROOTMAP2 = ws.ROOTMAP2;
  da.ZPOS = ws.ZPOS;
  da.OUTIDX = ws.OUTIDX;
  da.ACTMAP = ws.ACTMAP;
  da.KEEPIDX = ws.KEEPIDX;
  da.IDXA = ws.IDXA;
  da.IDXB = ws.IDXB;
  da.PFLAG = ws.PFLAG;
  da.RFLAG = ws.RFLAG;
  da.KEYA = ws.KEYA;
  da.KEYB = ws.KEYB;
  da.ms = ws.mstate;
  da.st = ws.status;
  da.warp_min_k = plan.tune.warp_min_k;
  da.order_small = (plan.batch > 1 && cnt > 0) ? 1 : 0;
  prof_begin(kKDeflate, s);
  launch_deflate(da, plan.step_maxsize[step], s);
  if (da.order_small) {
    k_order_cursor<<<1, kOrderBins, 0, s>>>(ws.status);
    k_order_assign<<<int(std::min<int64_t>((cnt + 255) / 256, 148 * 8)), 256, 0, s>>>(
        cnt, ws.mstate, ws.status, ws.ROOTMAP);
  }
  prof_end(kKDeflate, s);
  if (sel) {
    prof_begin(kKSel, s);
    launch_sel_deflate(plan, ws, *sel, step, s);
    prof_end(kKSel, s);
  }
  // form, deflate + roots
  int launches = 2 + (da.order_small ? 2 : 0) +
                 launch_roots(plan, ws, step, M, s, recompute || sel != nullptr, rows_inu, roots);
  if (sel) {
    prof_begin(kKSelRows, s);
    launch_sel_rows(plan, ws, *sel, step, s);
    prof_end(kKSelRows, s);
  }
  if (recompute) {
    g_launches += launches;
    return;
  }
  ++launches;  // place
  prof_begin(kKPlace, s);
  k_place<<<flat_grid, 256, 0, s>>>(M, cnt, nrows, ws.mstate, ws.D, ws.RLO, ws.RHI, ws.AD,
                                    ws.ALO, ws.AHI, ws.sigma_bits, out.lam, out.blo, out.bhi,
                                    lambda);
  prof_end(kKPlace, s);
  if (sel) {
    prof_begin(kKSel, s);
    launch_sel_place(plan, ws, *sel, step, s);
    prof_end(kKSel, s);
  }
  g_launches += launches;
}

}  // namespace tde
