// Root-level kernels of one merge step: the secular solve, the Lowner z-hat and
// the boundary-row update (Sec. 4.1; Algorithm 1, "solve the local secular
// equations ... compute (Q_v)_sigma by selected-row updates").
//
// All three are sweeps over the K active poles of a merge for each of its K roots
// (or, for z-hat, over the K roots for each pole), so a merge costs O(K^2) FP64
// work on O(K) data that stays in L1/L2.  On this part FP64 is the scarce
// resource (an FP64 instruction occupies the pipe for the whole warp whether or
// not its lanes are active), so the kernels keep every lane busy:
//   * merges whose active rank K >= warp_min_k (known only on the device, after
//     deflation; the deflation kernel files their roots in a second list): one
//     warp per root (per pole for z-hat); the 32 lanes stride over the poles and
//     the partial sums are combined with shuffles, so the whole warp shares one
//     root's iteration count;
//   * smaller merges: four lanes of a warp per root (one thread per root below
//     order 24), the roots of a warp moving in warp-synchronous rounds.
// Reciprocals use rcp_refined (three fused multiply-adds) instead of IEEE
// division.
#include <algorithm>

#include "tde_internal.cuh"

namespace tde {

struct RootArgs {
  const Merge* M;
  const MState* ms;
  const int32_t* ROOTMAP;   // roots of merges with K < warp_min_k
  const int32_t* ROOTMAP2;  // roots of merges with K >= warp_min_k
  const uint32_t* count;    // lengths of the two lists (device)
  const uint32_t* count2;
  const double *AD, *AZ, *ALO, *AHI;
  const float2* AD32;  // alias KEYB: active D minus the merge's midrange as an unevaluated
                       // float pair (hi, lo)
  const float* AZ32;   // alias IDXB: active z rounded to float
  double* TAU;
  int32_t* ORG;
  double* LAMA;           // aliases D: lambda_j of the active roots
  double* ZHAT;           // aliases Z
  double *ROWLO, *ROWHI;  // alias RLO, RHI: parent rows of the active columns
  double* DORG;           // alias KEYA: D_org(j) of every active root
  double* MPD;            // alias Z: pole-block centres, radii and moments (secular)
  double* MPR;            // alias KEYB: Löwner's pair-block moments, then (after Löwner)
                          // the boundary rows' block moments
  int32_t mp_min_k;       // merges with K >= this use the block expansion
  Status* st;
  uint32_t small_list_min;  // shorter small-K lists go to the warp kernels
  int all_merges;           // also build z-hat and rows at root merges (adjoint)
  double* RINU;             // optional: 1 / nu_j of every active root (adjoint)
};

// ---------------------------------------------------------------------------
// Secular equation.  For root j (0-based) of the active problem with sorted
// distinct poles D and nonzero z, w(lambda) = 1/rho' + sum_i z_i^2 / (D_i - lambda)
// has one root in (D_j, D_{j+1}) for j < K-1 and one in (D_{K-1}, D_{K-1} + rho' zsq)
// for the last root.  In shifted coordinates lambda = D_org + tau with
// Delta_i = (D_i - D_org) - tau the two poles that bracket the root keep full
// relative accuracy.
//
// Each iteration evaluates w and its derivatives and takes the root of a rational
// model C + S1 / (Delta_jl - eta) + S2 / (Delta_jr - eta) of w around the current
// point, kept inside a bisection bracket:
//   * third-order model: S1, S2 and C fitted to w, w' and w''/2 = sum z^2/Delta^3
//     (the fitted weights are nonnegative in exact arithmetic for every root but
//     the last);
//   * two-term model: S1 = Delta_jl^2 psi', S2 = Delta_jr^2 phi' with psi / phi the
//     poles left (i <= jl) and right of the root (each side's derivative attributed
//     to its nearest pole); if a step fails to shrink |w| tenfold, the origin pole
//     gets its exact residue z_org^2 and the other pole the rest of w' from then on
//     -- this rescues roots pressed against a pole with a tiny z.
//
// Two precisions.  On this part an FP64 instruction costs about forty times the
// issue slots of an FP32 one, so every root starts with a single-precision stage:
// pole offsets from an unevaluated float pair per pole (D_i - shift = hi + lo with
// the merge's midrange as shift, about 48 bits, so D_i - D_org keeps its relative
// accuracy), hardware reciprocal approximations and a compensated sum for w, all
// in units of the root's interval width so that the sums stay in the float range.  It starts at the midpoint of the
// interval (whose sign of w chooses the origin, the nearer pole), iterates the
// third-order model until the step is below 2^-10 |tau| and ends with one sweep at
// the final tau, which also supplies w'' there.  Where the model has no root in the
// bracket (a root pressed against an origin pole of tiny z), the step goes straight
// to z_org^2 / (the rest of w) instead of bisecting.  The FP64 stage starts from that
// tau with the whole interval as bracket; each FP64 sweep gives w and w' to full
// accuracy, w'' comes from a single-precision sweep at the same point (its error
// enters the step at second order), and a third-order step below 2^-18 |tau| is
// accepted without another sweep (the error it leaves is of order
// (2^-18)^3 |tau|), a two-term step below 2^-27 |tau| likewise (order
// (2^-27)^2 |tau|).  Anything non-finite or a negative fitted weight sends a step
// to the two-term model.  A root whose interval is narrower than 2^-28 of the
// shifted pole magnitude |D - shift| (where the float pair cannot resolve the
// offsets), or whose single-precision stage fails, starts in FP64 at the midpoint
// and iterates with the two-term model only.  Convergence: |w| below eps times a running bound on the
// rounding error of its evaluation, 8 (|psi| + |phi|) + 1/rho' + |tau| (psi' + phi').
struct SecSums {
  double psi, dpsi, phi, dphi;
};

// single-precision sums: psi, phi (compensated), their derivatives, and
// hw = sum z^2 / Delta^3 over all poles
struct Sec32 {
  float psi, dpsi, phi, dphi, hw;
};

struct SecState {
  int org, jl, jr;
  bool exact;  // origin pole weighted by its exact residue
  double tau, tlo, thi, w, wprev, dorg, ol, orr, rhoinv, zorg2;
  SecSums s;
};

// FP64 start at the interval midpoint: sec_init_point sets the evaluation point
// (origin j, or K-1 for the last root, and the half width), the caller sweeps
// there, and sec_init_finish picks the origin (the nearer pole) from the sign of
// w and sets the half-interval bracket.
__device__ __forceinline__ void sec_init_point(const double* D, int K, int j, double rho,
                                               double rhoinv, double zsq, SecState& q) {
  q.rhoinv = rhoinv;
  if (j < K - 1) {
    q.jl = j;
    q.jr = j + 1;
    q.dorg = D[j];
    q.tau = 0.5 * (D[j + 1] - D[j]);
  } else {
    q.jl = K - 2;
    q.jr = K - 1;
    q.org = K - 1;
    q.dorg = D[K - 1];
    q.tau = 0.5 * (rho * zsq);
  }
}

__device__ __forceinline__ void sec_init_finish(const double* D, const double* Z, int K, int j,
                                                double rho, double zsq, SecState& q) {
  q.w = q.rhoinv + q.s.psi + q.s.phi;
  if (j < K - 1) {
    const double half = q.tau;
    if (q.w >= 0.0) {
      q.org = j;
      q.tlo = 0.0;
      q.thi = half;
    } else {
      q.org = j + 1;
      q.tau = -half;
      q.tlo = -half;
      q.thi = 0.0;
    }
  } else {
    const double upper = rho * zsq;
    if (q.w >= 0.0) {
      q.tlo = 0.0;
      q.thi = q.tau;
    } else {
      q.tlo = q.tau;
      q.thi = upper;
    }
  }
  q.dorg = D[q.org];
  q.zorg2 = Z[q.org] * Z[q.org];
  q.ol = D[q.jl] - q.dorg;
  q.orr = D[q.jr] - q.dorg;
  q.exact = false;
  q.wprev = 0.0;
}

// Weights of the third-order model at poles a = Delta_jl, b = Delta_jr from
// w' = dw and w''/2 = hw, as P1 = S1 / a^2 = a (hw b - dw) / (b - a) and
// P2 = S2 / b^2 = b (dw - hw a) / (b - a).  False if either is negative or not
// finite.  T is double (FP64 stage) or float (single-precision stage).
__device__ __forceinline__ double fast_rcp(double x) { return rcp_refined(x); }
__device__ __forceinline__ float fast_rcp(float x) { return __fdividef(1.0f, x); }

template <class T>
__device__ __forceinline__ bool fit3(T a, T b, T dw, T hw, T* P1, T* P2) {
  const T inv = fast_rcp(b - a);
  const T p1 = a * (hw * b - dw) * inv;
  const T p2 = b * (dw - hw * a) * inv;
  if (!(p1 >= T(0) && p2 >= T(0) && isfinite(p1 + p2))) return false;
  *P1 = p1;
  *P2 = p2;
  return true;
}

// Root eta of the model w(tau + eta) ~ C + S1 / (a - eta) + S2 / (b - eta) with
// S1 = P1 a^2, S2 = P2 b^2 and value w at eta = 0, such that tau + eta lies in
// (tlo, thi); the smaller one if both roots do.  False if neither does (or on
// non-finite values).  Reciprocals need no correct rounding here: a step is an
// approximation whose own error is relative to its size.
template <class T>
__device__ __forceinline__ bool model_root(T w, T a, T b, T P1, T P2, T tau, T tlo, T thi, T* eta) {
  const T C = w - P1 * a - P2 * b;
  const T A = C * (a + b) + P1 * a * a + P2 * b * b;
  const T Bq = a * b * w;
  if (C == T(0)) {
    if (A == T(0)) return false;
    *eta = Bq * fast_rcp(A);
    return true;
  }
  const T disc = A * A - T(4) * Bq * C;
  const T sq = sqrt(disc > T(0) ? disc : T(0));
  const T qq = T(0.5) * (A >= T(0) ? A + sq : A - sq);
  const T r1 = qq * fast_rcp(C);
  const T r2 = (qq != T(0)) ? Bq * fast_rcp(qq) : r1;
  const bool ok1 = (tau + r1 > tlo) && (tau + r1 < thi);
  const bool ok2 = (tau + r2 > tlo) && (tau + r2 < thi);
  if (ok1 && ok2) {
    *eta = fabs(r1) < fabs(r2) ? r1 : r2;
    return true;
  }
  if (ok1 || ok2) {
    *eta = ok1 ? r1 : r2;
    return true;
  }
  return false;
}

// One FP64 iteration; hw = w''/2 at tau when `third`.  Returns 1 if tau moved and
// needs a new sweep, 0 if converged.
__device__ __forceinline__ int sec_step(SecState& q, double hw, bool third) {
  const double erretm =
      8.0 * (fabs(q.s.psi) + fabs(q.s.phi)) + q.rhoinv + fabs(q.tau) * (q.s.dpsi + q.s.dphi);
  if (fabs(q.w) <= kEps * erretm) return 0;
  if (q.w > 0.0)
    q.thi = fmin(q.thi, q.tau);
  else
    q.tlo = fmax(q.tlo, q.tau);
  if (q.thi - q.tlo <= 2.0 * kEps * fmax(fabs(q.tlo), fabs(q.thi))) return 0;
  // Short last step: with w''/2 known and the Newton step -w / w' below 2^-20 |tau|,
  // the second-order step eta = -w / (w' + (w''/2) eta_N) of the Taylor model
  // w + w' eta + (w''/2) eta^2 is final.  The origin pole sits at distance |tau|
  // and every other one farther, so the dropped cubic term moves eta by at most
  // |eta| (eta / tau)^2 < 2^-40 |eta|, and the float rounding of w''/2 by
  // 2^-24 |eta / tau| |eta|: both below 2^-60 |tau|.
  if (third) {
    const double dw = q.s.dpsi + q.s.dphi;
    if (fabs(q.w) <= 0x1p-20 * fabs(q.tau) * dw) {
      const double eta = -(q.w * dw) * rcp_refined(fma(dw, dw, -hw * q.w));
      const double ntau = q.tau + eta;
      if (ntau > q.tlo && ntau < q.thi) {
        q.tau = ntau;
        return 0;
      }
    }
  }
  const double a = q.ol - q.tau, b = q.orr - q.tau;  // Delta of the two model poles
  if (q.wprev != 0.0 && fabs(q.w) > 0.1 * fabs(q.wprev)) q.exact = true;
  q.wprev = q.w;
  double P1, P2;
  const bool cubic = third && fit3(a, b, q.s.dpsi + q.s.dphi, hw, &P1, &P2);
  if (!cubic) {
    P1 = q.s.dpsi;
    P2 = q.s.dphi;
    if (q.exact) {
      const double dw = q.s.dpsi + q.s.dphi;
      const double e = (q.org == q.jl) ? q.zorg2 * fast_rcp(a * a) : q.zorg2 * fast_rcp(b * b);
      if (e <= dw) {
        P1 = (q.org == q.jl) ? e : dw - e;
        P2 = dw - P1;
      }
    }
  }
  double eta = 0.0;
  const bool have = model_root(q.w, a, b, P1, P2, q.tau, q.tlo, q.thi, &eta);
  double ntau = q.tau + eta;
  const bool model = have && ntau > q.tlo && ntau < q.thi;
  if (!model) ntau = 0.5 * (q.tlo + q.thi);
  if (ntau == q.tau) return 0;
  q.tau = ntau;
  if (model && fabs(eta) <= (cubic ? 0x1p-18 : 0x1p-27) * fabs(ntau)) return 0;
  return 1;
}

constexpr int kMaxSweeps = 64;
constexpr int kMaxSweeps32 = 24;

// Single-precision stage for root j, all of it in float, as steps that a driver
// interleaves with its sweeps (`sw32(org, jl, tau, inv)` evaluates the sums):
//   s32_begin   applicability and the first point (interval midpoint); the stage is
//               skipped where the float copies cannot resolve the interval
//               (`sw32.resolves`)
//   s32_first   after the first sweep: the origin (nearer pole) and its bracket
//   s32_step    one model step; false when the stage stops (w at the float
//               resolution, no move, non-finite)
//   s32_after   after the sweep at the new point: stop below 2^-10 |tau| or at
//               kMaxSweeps32 sweeps
//   s32_finish  for a finite w and tau inside the interval fills q for the FP64
//               stage (origin, tau, the whole interval as bracket) and *hw with
//               w''/2 at tau; *hw_ok is false where w''/2 overflowed the float range
//               (a root within about 2^-40 S of its origin), and the FP64 stage
//               then starts from tau with the two-term model
// The stage works in units of S, the power of two at or below the root's interval
// width (offsets and tau divided by S, w and its sums multiplied by S, so the
// derivative sums of poles closer than 2^-40 stay inside the float range); inv is
// 1/S.
struct Stage32 {
  int org, jl, jr, sweeps;
  bool live;
  float rhoinv, tau, tlo, thi, lo_int, hi_int, ol, orr, gap, inv;
  float zorg2;  // z_org^2 of the origin pole (its residue, in the stage's units too)
  double dorg, S, Sinv;
  Sec32 s;
};

template <class Sweep32>
__device__ __forceinline__ bool s32_begin(const double* D, int K, int j, double rho,
                                          double rhoinv, double zsq, const Sweep32& sw32,
                                          Stage32& st) {
  st.jl = (j < K - 1) ? j : K - 2;
  st.jr = st.jl + 1;
  const double width = (j < K - 1) ? D[st.jr] - D[st.jl] : rho * zsq;
  if (!(width >= 0x1p-90 && width <= 0x1p90) || !sw32.resolves(st.jl, st.jr, j == K - 1, width))
    return false;
  // S = 2^ex and its inverse built from the exponent bits (width is a normal
  // double in [2^-90, 2^90]), so that every scaling below is an exact multiply
  const int ex = int((__double_as_longlong(width) >> 52) & 0x7ff) - 1023;
  st.S = __longlong_as_double((long long)(1023 + ex) << 52);
  st.Sinv = __longlong_as_double((long long)(1023 - ex) << 52);
  st.inv = __int_as_float((127 - ex) << 23);
  st.rhoinv = float(st.S * rhoinv);
  st.sweeps = 0;
  st.live = false;
  if (j < K - 1) {
    st.gap = float(width * st.Sinv);
    st.org = j;
    st.tau = 0.5f * st.gap;
  } else {
    st.org = K - 1;
    st.hi_int = float(width * st.Sinv);
    st.lo_int = 0.0f;
    st.tau = 0.5f * st.hi_int;
    st.tlo = 0.0f;
    st.thi = st.hi_int;
  }
  return true;
}

__device__ __forceinline__ void s32_first(const double* D, const double* Z, int K, int j,
                                          Stage32& st) {
  st.sweeps = 1;
  if (j < K - 1) {
    const float h32 = st.tau;
    if (st.rhoinv + st.s.psi + st.s.phi >= 0.0f) {
      st.org = j;
      st.tlo = 0.0f;
      st.thi = h32;
      st.lo_int = 0.0f;
      st.hi_int = st.gap;
    } else {
      st.org = j + 1;
      st.tau = h32 - st.gap;
      st.tlo = st.tau;
      st.thi = 0.0f;
      st.lo_int = -st.gap;
      st.hi_int = 0.0f;
    }
  }
  st.dorg = D[st.org];
  st.ol = float((D[st.jl] - st.dorg) * st.Sinv);
  st.orr = float((D[st.jr] - st.dorg) * st.Sinv);
  st.zorg2 = float(Z[st.org] * Z[st.org]);
  st.live = true;
}

__device__ __forceinline__ bool s32_step(Stage32& st, float* eta_out, bool* have_out) {
  const float w = st.rhoinv + st.s.psi + st.s.phi;
  if (!isfinite(w)) {
    st.live = false;
    return false;
  }
  // w at the resolution of the float sums: tau is as good as this stage gets (a
  // model step would be below the rounding of tau), stop here with s at tau
  if (fabsf(w) <= 0x1p-22f * (st.rhoinv + fabsf(st.s.psi) + fabsf(st.s.phi))) {
    st.live = false;
    return false;
  }
  if (w > 0.0f)
    st.thi = fminf(st.thi, st.tau);
  else
    st.tlo = fmaxf(st.tlo, st.tau);
  const float a = st.ol - st.tau, b = st.orr - st.tau;
  float P1, P2;
  if (!fit3(a, b, st.s.dpsi + st.s.dphi, st.s.hw, &P1, &P2)) {
    P1 = st.s.dpsi;
    P2 = st.s.dphi;
  }
  float eta = 0.0f;
  const bool have = model_root(w, a, b, P1, P2, st.tau, st.tlo, st.thi, &eta);
  float nt = have ? st.tau + eta : 0.5f * (st.tlo + st.thi);
  if (!have) {
    // A root pressed against an origin pole of tiny z: that pole's term is invisible
    // in the sums until tau nears z^2 / w, so the fitted model finds no root in the
    // bracket.  With the rest of w about constant near the pole, the root sits at
    // t = z_org^2 / (w + z_org^2 / tau): taken when it lies in the bracket and below
    // half of |tau| (a ratio, so t keeps its relative accuracy in float).
    const float t = st.zorg2 / (w + st.zorg2 / st.tau);
    if (t > st.tlo && t < st.thi && fabsf(t) < 0.5f * fabsf(st.tau)) nt = t;
  }
  if (nt == st.tau || !(nt > st.lo_int && nt < st.hi_int)) {  // no move: s is at tau
    st.live = false;
    return false;
  }
  st.tau = nt;
  *eta_out = eta;
  *have_out = have;
  return true;
}

__device__ __forceinline__ void s32_after(Stage32& st, float eta, bool have) {
  ++st.sweeps;
  if ((have && fabsf(eta) <= 0x1p-10f * fabsf(st.tau)) || st.sweeps >= kMaxSweeps32) st.live = false;
}

// w''/2 in natural units from its value in the stage's units (S^3 w''/2)
__device__ __forceinline__ double hw_natural(const Stage32& st, float hws) {
  return double(hws) * (st.Sinv * st.Sinv * st.Sinv);
}

// single-precision sweep at the FP64 stage's tau, for w''/2 (natural units)
template <class Sweep32>
__device__ __forceinline__ double hw_at(const Sweep32& sw32, const Stage32& st, const SecState& q) {
  return hw_natural(st, sw32(q.org, q.jl, float(q.tau * st.Sinv), st.inv).hw);
}

__device__ __forceinline__ bool s32_finish(const double* D, const double* Z, double rhoinv,
                                           const Stage32& st, SecState& q, double* hw,
                                           bool* hw_ok) {
  *hw_ok = isfinite(st.s.hw);  // overflows for a root within ~2^-40 S of its origin
  if (!(isfinite(st.rhoinv + st.s.psi + st.s.phi) && st.tau > st.lo_int && st.tau < st.hi_int))
    return false;
  q.org = st.org;
  q.jl = st.jl;
  q.jr = st.jr;
  q.tau = double(st.tau) * st.S;
  q.tlo = double(st.lo_int) * st.S;
  q.thi = double(st.hi_int) * st.S;
  q.rhoinv = rhoinv;
  q.dorg = st.dorg;
  q.zorg2 = Z[st.org] * Z[st.org];
  q.ol = D[st.jl] - st.dorg;
  q.orr = D[st.jr] - st.dorg;
  q.exact = false;
  q.wprev = 0.0;
  *hw = hw_natural(st, st.s.hw);
  return true;
}

// Solves root j; returns the number of FP64 pole sweeps (*n32 the single-precision
// ones), *ok = false if capped.  One root per caller (a warp or a thread).
template <class Sweep, class Sweep32>
__device__ int secular_root(const double* D, const double* Z, int K, int j, double rho,
                            double rhoinv, double zsq, Sweep& sweep, Sweep32& sw32, int* org_out,
                            double* tau_out, bool* ok, int* n32) {
  *ok = true;
  *n32 = 0;
  if (K == 1) {
    *org_out = 0;
    *tau_out = rho * Z[0] * Z[0];
    return 0;
  }
  SecState q;
  double hw = 0.0;
  Stage32 st;
  bool third = false, handed = false;
  if (s32_begin(D, K, j, rho, rhoinv, zsq, sw32, st)) {
    st.s = sw32(st.org, st.jl, st.tau, st.inv);
    s32_first(D, Z, K, j, st);
    for (;;) {
      float eta = 0.0f;
      bool have = false;
      if (!s32_step(st, &eta, &have)) break;
      st.s = sw32(st.org, st.jl, st.tau, st.inv);
      s32_after(st, eta, have);
      if (!st.live) break;
    }
    *n32 = st.sweeps;
    bool hw_ok;
    handed = s32_finish(D, Z, rhoinv, st, q, &hw, &hw_ok);
    third = handed && hw_ok;
  }
  if (handed) {
    q.s = sweep(q.dorg, q.tau, q.jl);
    q.w = q.rhoinv + q.s.psi + q.s.phi;
  } else {
    sec_init_point(D, K, j, rho, rhoinv, zsq, q);
    q.s = sweep(q.dorg, q.tau, q.jl);
    sec_init_finish(D, Z, K, j, rho, zsq, q);
  }
  int sweeps = 1;
  while (sec_step(q, hw, third) == 1) {
    if (sweeps >= kMaxSweeps) {
      *ok = false;
      break;
    }
    if (third) {
      hw = hw_at(sw32, st, q);
      ++*n32;
    }
    q.s = sweep(q.dorg, q.tau, q.jl);
    q.w = q.rhoinv + q.s.psi + q.s.phi;
    ++sweeps;
  }
  *org_out = q.org;
  *tau_out = q.tau;
  return sweeps;
}

// Warp-synchronous form for kernels in which one warp solves several roots at a
// time (one thread or G lanes per root; `valid` false for lanes without a root).
// Every phase change and loop exit is a warp vote, so the roots of a warp run
// each kind of sweep in the same rounds: an FP64 instruction costs the whole
// warp's issue slot however few lanes are active, and roots at different phases
// would otherwise pay for one another's sweeps.  Same steps and stopping rules as
// secular_root; all 32 lanes must call it together.
template <class Sweep, class Sweep32>
__device__ int secular_root_sync(const double* D, const double* Z, int K, int j, double rho,
                                 double rhoinv, double zsq, bool valid, Sweep& sweep, Sweep32& sw32,
                                 int* org_out, double* tau_out, bool* ok, int* n32) {
  constexpr unsigned kFull = 0xffffffffu;
  *ok = true;
  *n32 = 0;
  const bool act = valid && K > 1;
  Stage32 st;
  st.live = false;
  const bool in32 = act && s32_begin(D, K, j, rho, rhoinv, zsq, sw32, st);
  if (in32) {
    st.s = sw32(st.org, st.jl, st.tau, st.inv);
    s32_first(D, Z, K, j, st);
  }
  for (;;) {
    float eta = 0.0f;
    bool have = false;
    const bool need = in32 && st.live && s32_step(st, &eta, &have);
    if (!__any_sync(kFull, need)) break;
    if (need) {
      st.s = sw32(st.org, st.jl, st.tau, st.inv);
      s32_after(st, eta, have);
    }
  }
  SecState q;
  q.org = 0;
  q.tau = 0.0;
  double hw = 0.0;
  bool third = false, handed = false;
  if (in32) {
    *n32 = st.sweeps;
    bool hw_ok;
    handed = s32_finish(D, Z, rhoinv, st, q, &hw, &hw_ok);
    third = handed && hw_ok;
  }
  if (act && !handed) sec_init_point(D, K, j, rho, rhoinv, zsq, q);
  if (act) q.s = sweep(q.dorg, q.tau, q.jl);
  if (act) {
    if (handed)
      q.w = q.rhoinv + q.s.psi + q.s.phi;
    else
      sec_init_finish(D, Z, K, j, rho, zsq, q);
  }
  int sweeps = act ? 1 : 0;
  bool go = act;
  for (;;) {
    if (go) {
      if (sec_step(q, hw, third) == 0) {
        go = false;
      } else if (sweeps >= kMaxSweeps) {
        *ok = false;
        go = false;
      }
    }
    if (!__any_sync(kFull, go)) break;
    if (go && third) {
      hw = hw_at(sw32, st, q);
      ++*n32;
    }
    if (go) {
      q.s = sweep(q.dorg, q.tau, q.jl);
      q.w = q.rhoinv + q.s.psi + q.s.phi;
      ++sweeps;
    }
  }
  if (valid && K == 1) {
    *org_out = 0;
    *tau_out = rho * Z[0] * Z[0];
    return 0;
  }
  *org_out = q.org;
  *tau_out = q.tau;
  return sweeps;
}

// Block expansion of the FP64 sums (merges with K >= mp_min_k, warp-per-root
// kernel).  The K poles are cut into nb = K / 128 blocks of consecutive poles (the
// last one takes the remainder).  Per block, k_block_moments stores its centre m,
// its radius r (largest |D_i - m|) and the normalised moments
//   M'_k = sum_{i in block} z_i^2 ((D_i - m) / r)^k,
// so that for lambda outside the block, with t = 1 / (m - lambda) and x = -r t,
//   sum z_i^2 / (D_i - lambda)   = t   sum_k M'_k x^k,
//   sum z_i^2 / (D_i - lambda)^2 = t^2 sum_k (k + 1) M'_k x^k.
// A sweep takes a block through these series when r <= |m - lambda| / 3 (|x| <= 1/3):
// with 35 terms the dropped part is below 3^-35 (1 + 1/3) / (1 - 1/3) < 2^-54 of the
// block's own sum_i |z_i^2 / (D_i - lambda)|, under the rounding bound of the
// convergence test.  A round of 32 blocks all within 1/4 of their distance stops
// after 27 terms (4^-27 (5/3) < 2^-53), all within 1/16 after 14 (16^-14 = 2^-56),
// all within 1/64 after 10 (64^-10 = 2^-60).
// Only the head of each series runs in FP64: from term H on, Horner's rule runs in
// float on float copies of the same moments and enters the FP64 chain as its
// starting value.  The float part's error, about 3 x 2^-24 |x|^H of M'_0, stays
// below 2^-55 for the value with H = 21 / 17 / 9 / 6 (x within 1/3, 1/4, 1/16, 1/64),
// and below 2^-40 for the derivative with H = 14 / 11 / 6 / 4.  The derivative only shapes the
// step and the error bound: a relative error of 2^-40 moves the last step
// (|eta| <= 2^-18 |tau|) by under 2^-58 |tau|.
// Every other block (the root's own and its neighbours) is summed exactly.  The
// block lies wholly on one side of lambda, so it adds to psi or phi as a whole.
// m - lambda is formed as (m - D_org) - tau, like every Delta.
constexpr int kMpBlock = 128;  // poles per block
constexpr int kMpTerms = 35;   // series terms (radius <= 1/3 of the distance)
constexpr int kMpMid = 27;     // enough when radius <= 1/4 of the distance
constexpr int kMpShort = 14;   // enough when radius <= 1/16 of the distance (16^-14 = 2^-56)
constexpr int kMpTiny = 10;    // enough when radius <= 1/64 of the distance (64^-10 = 2^-60)
// FP64 heads of the value and derivative series, tiers 0..3 (1/64, 1/16, 1/4, 1/3)
constexpr int kHv0 = 6, kHv1 = 9, kHv2 = 17, kHv3 = 21;
constexpr int kHd0 = 4, kHd1 = 6, kHd2 = 11, kHd3 = 14;
constexpr int kMpFields = 3 + kHv3 + kHd3;     // m, r, 3 r, M'_k (k < 21), (k + 1) M'_k (k < 14)
// FP64 operations of a far block besides its heads (work counter): m - lambda 2,
// reciprocal 1, x 1, accumulation 3 (t val, t^2, t^2 der)
constexpr int kSecSeriesOverhead = 7;

// Far test and series tier of a round of 32 blocks (warp vote over the lanes whose
// block, of radius r at distance |dm| from the point, is far): far when 3 r <= |dm|;
// tier 0 if all far blocks of the round are within 1/64 of their distance, 1 if
// within 1/16, 2 if within 1/4, else 3.  The tests compare the bit patterns of non-negative doubles
// (ordered like their values), so that they take no FP64 instruction: adding
// j << 52 multiplies a normal double by 2^j; r3 is the stored 3 r.
struct FarTest {
  bool far;
  int tier;
};
__device__ __forceinline__ FarTest far_test_bits(double dm, double r, double r3, bool valid) {
  const long long db = __double_as_longlong(dm) & 0x7fffffffffffffffLL;
  const long long rb = __double_as_longlong(r);
  FarTest ft;
  ft.far = valid && db >= __double_as_longlong(r3);
  if (__all_sync(0xffffffffu, !ft.far || db >= rb + (6LL << 52)))
    ft.tier = 0;
  else if (__all_sync(0xffffffffu, !ft.far || db >= rb + (4LL << 52)))
    ft.tier = 1;
  else if (__all_sync(0xffffffffu, !ft.far || db >= rb + (2LL << 52)))
    ft.tier = 2;
  else
    ft.tier = 3;
  return ft;
}

// The value and derivative series of one far block (N terms, FP64 heads HV and
// HD): float Horner over the tails (fa: M'_k, fb: (k + 1) M'_k), then FP64 Horner
// over the heads (ca, cb) from the tails' values.
template <int N, int HV, int HD>
__device__ __forceinline__ void series_mixed(const double* ca, const double* cb, const float* fa,
                                             const float* fb, int nb, double x, double& val,
                                             double& der) {
  static_assert(HD <= HV && HV < N, "heads inside the series");
  const float xf = __double2float_rn(x);
  float tv = fa[(N - 1) * nb], td = fb[(N - 1) * nb];
#pragma unroll
  for (int k = N - 2; k >= HD; --k) {
    if (k >= HV) tv = fmaf(tv, xf, fa[k * nb]);
    td = fmaf(td, xf, fb[k * nb]);
  }
  double v = double(tv), d = double(td);
#pragma unroll
  for (int k = HV - 1; k >= 0; --k) {
    v = fma(v, x, ca[k * nb]);
    if (k < HD) d = fma(d, x, cb[k * nb]);
  }
  val = v;
  der = d;
}
static_assert(kMpFields <= kMpBlock, "block data must fit the merge's rows (fields x K / 128 <= K)");

// Float data of the blocks, placed after the FP64 data (field q of block b at
// BF[q nb + b], BF = (float*)(MPD + lo + 38 nb)): the centre minus the merge's
// midrange as a float pair, the radius, the normalised moments M'_k and
// (k + 1) M'_k (k < 35; the tails of the FP64 series and the single-precision
// stage's w and w') and (k + 1)(k + 2) / 2 M'_k (k < 18, its w''/2).  In the stage's
// units (offsets / S, sums x S) a far block with d = (m - lambda) / S and
// x = -(r / S) / d adds
//   w: (1/d) sum M'_k x^k,  w': (1/d)^2 sum (k + 1) M'_k x^k,
//   w''/2: (1/d)^3 sum (k + 1)(k + 2)/2 M'_k x^k,
// far blocks (|x| <= 1/3) take 18 terms, rounds within 1/16 10: the dropped part
// stays below 2^-27 of the block's terms, under the rounding of the float sums.
// The normalisation keeps every float in range.
constexpr int kMfTerms = 35;  // float M'_k and (k + 1) M'_k
constexpr int kMf32 = 18;     // terms of the single-precision stage: 3^-18 x 2 < 2^-27
constexpr int kMfShort = 10;  // radius <= 1/16: 16^-10 = 2^-40
constexpr int kMfFields = 3 + 2 * kMfTerms + kMf32;  // centre hi, lo, radius, three series
static_assert(2 * kMpFields + kMfFields <= 2 * kMpBlock, "both block data sets fit the merge's rows");

// Block data of the merge at lo lives coefficient-major in MPD + lo: field q of
// block b at [q * nb + b] (84 nb <= K entries, inside the merge's rows).
__device__ __forceinline__ int mp_blocks(int K, int mp_min_k) {
  return K >= mp_min_k ? K / kMpBlock : 0;
}

// Superblocks: sbs consecutive blocks (the last one takes the remainder) with the
// same kind of data, at most 32 per merge.  A sweep first takes every superblock
// that is far from the point through its series (one superblock per lane), then
// goes block by block over the superblocks it did not take whole, 32 blocks per
// round.  The secular sums and the Löwner products use sbs = 8 in merges of 65 to
// 256 blocks (16 up to 512, 32 up to 1024 blocks): the near superblocks (the
// point's own and its neighbours) then hold about 24 blocks, one round, so a sweep
// takes two rounds of series where one block per lane would take nb / 32.  The
// row sums keep 32-block superblocks from 192 blocks: their block data (121
// doubles per block) leave no room for smaller ones inside the merge's rows.
// Their data follow the blocks' float data (field q of superblock s at [q nsb + s]).
constexpr int kSbMin = 65;       // from here the superblock round saves block rounds
constexpr int kSbRows = 32;      // superblock size of the row sums
constexpr int kSbRowsMin = 192;  // and their threshold (below it the round costs what it saves)
static_assert(kSbRows == 32, "the row sums' block rounds coincide with their superblocks");
__device__ __forceinline__ int sb_size(int nb) { return nb <= 256 ? 8 : nb <= 512 ? 16 : 32; }
__device__ __forceinline__ int sb_count(int nb, int sbs, int min_nb) {
  if (nb < min_nb || sbs == 0) return 0;
  const int nsb = (nb + sbs - 1) / sbs;
  return nsb <= 32 ? nsb : 0;
}
// superblocks of the secular sums and Löwner products
__device__ __forceinline__ int sb_count(int nb) { return sb_count(nb, sb_size(nb), kSbMin); }
// superblocks of the row sums
__device__ __forceinline__ int sb_count_rows(int nb) { return sb_count(nb, kSbRows, kSbRowsMin); }

// The blocks a sweep takes one by one after its superblock round: those of the
// superblocks it did not take whole (all blocks without superblocks), in
// ascending order; entry idx of the list is block kept_block(k, idx).
struct KeptBlocks {
  unsigned keep;  // superblocks not taken whole
  int sbs, count;
};
__device__ __forceinline__ KeptBlocks kept_blocks(int nsb, int sbs, unsigned sfar, int nb) {
  KeptBlocks k;
  if (nsb == 0) {
    k.keep = 0u;
    k.sbs = 0;
    k.count = nb;
    return k;
  }
  k.sbs = sbs;
  k.keep = (nsb >= 32 ? 0xffffffffu : (1u << nsb) - 1u) & ~sfar;
  k.count = __popc(k.keep) * sbs;
  if ((k.keep >> (nsb - 1)) & 1u) k.count -= nsb * sbs - nb;  // the last superblock is short
  return k;
}
// block of list entry idx, or -1 past the end of the list
__device__ __forceinline__ int kept_block(const KeptBlocks& k, int idx) {
  if (idx >= k.count) return -1;
  if (k.sbs == 0) return idx;
  unsigned m = k.keep;
  for (int q = idx / k.sbs; q > 0; --q) m &= m - 1;  // skip the kept superblocks before it
  return (__ffs(m) - 1) * k.sbs + idx % k.sbs;
}
__device__ __forceinline__ double* sb_data(double* MPD_lo, int nb) {
  return MPD_lo + kMpFields * nb + (kMfFields * nb + 1) / 2;
}

// In place, v_k <- sum_{q<=k} C(k, q) a^(k-q) v_q (k < N): N - 1 passes of
// v_j += a v_(j-1) from the top down, pass i starting at j = i (Pascal's rule).
template <int N>
__device__ __forceinline__ void binomial_shift(double (&v)[N], double a) {
#pragma unroll
  for (int i = 1; i < N; ++i) {
#pragma unroll
    for (int j = N - 1; j >= i; --j) v[j] = fma(a, v[j - 1], v[j]);
  }
}
// per 8 blocks (1024 rows, the smallest superblock): their data and one
// superblock's, each at most kMpFields + (kMfFields + 1) / 2 + 1 doubles
static_assert((8 + 1) * (kMpFields + (kMfFields + 1) / 2 + 1) <= 8 * kMpBlock,
              "block and superblock data fit the merge's rows");

// one thread evaluates all K poles
struct ThreadSweep {
  const double* __restrict__ D;
  const double* __restrict__ Z;
  int K;
  __device__ __forceinline__ SecSums operator()(double dorg, double tau, int jl) const {
    SecSums s{0.0, 0.0, 0.0, 0.0};
    for (int i = 0; i < K; ++i) {
      const double zi = Z[i];
      const double t = zi * rcp_refined((D[i] - dorg) - tau);
      const bool left = i <= jl;
      const double zl = left ? zi : 0.0, zr = left ? 0.0 : zi;
      const double tl = left ? t : 0.0, tr = left ? 0.0 : t;
      s.psi = fma(zl, t, s.psi);
      s.dpsi = fma(tl, t, s.dpsi);
      s.phi = fma(zr, t, s.phi);
      s.dphi = fma(tr, t, s.dphi);
    }
    return s;
  }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp sums of four values in six FP64 additions instead of twenty: the first
// exchange leaves lanes 0-15 the partial sums of a, b and lanes 16-31 those of c,
// d, the second one value per lane quarter (a, b, c, d in lanes 0-7, 8-15, 16-23,
// 24-31), three more finish each quarter, and shuffles broadcast the totals.
__device__ __forceinline__ void warp_sum4(double& a, double& b, double& c, double& d) {
  const int lane = threadIdx.x & 31;
  const bool hi16 = lane & 16, hi8 = lane & 8;
  double x0 = hi16 ? c : a, x1 = hi16 ? d : b;
  const double y0 = hi16 ? a : c, y1 = hi16 ? b : d;
  x0 += __shfl_xor_sync(0xffffffffu, y0, 16);
  x1 += __shfl_xor_sync(0xffffffffu, y1, 16);
  double z = hi8 ? x1 : x0;
  z += __shfl_xor_sync(0xffffffffu, hi8 ? x0 : x1, 8);
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
  a = __shfl_sync(0xffffffffu, z, 0);
  b = __shfl_sync(0xffffffffu, z, 8);
  c = __shfl_sync(0xffffffffu, z, 16);
  d = __shfl_sync(0xffffffffu, z, 24);
}

// Warp sums of V values per lane by recursive halving: at each exchange (lane
// offsets 16, 8, 4, 2, 1) a lane keeps the upper or lower half of its list (an odd
// list gains a zero) and adds its partner's copy of that half, so the five
// exchanges take about V FP64 additions instead of 5 V.  Afterwards v[j], j <
// warp_halved_len(V), holds the total of entry halving_index<V>(lane, j), or
// padding where that is -1.
__host__ __device__ constexpr int halved(int L) { return (L + 1) / 2; }
__host__ __device__ constexpr int warp_halved_len(int V) { return halved(halved(halved(halved(halved(V))))); }

template <int L, int V>
__device__ __forceinline__ void halve_step(double (&v)[V], int o, bool up) {
  constexpr int H = halved(L);
#pragma unroll
  for (int j = 0; j < H; ++j) {
    const double lo = v[j];
    const double hi = (j + H < L) ? v[j + H] : 0.0;
    v[j] = (up ? hi : lo) + __shfl_xor_sync(0xffffffffu, up ? lo : hi, o);
  }
}

template <int V>
__device__ __forceinline__ void warp_sum_halving(double (&v)[V], int lane) {
  constexpr int L1 = halved(V), L2 = halved(L1), L3 = halved(L2), L4 = halved(L3);
  halve_step<V>(v, 16, lane & 16);
  halve_step<L1>(v, 8, lane & 8);
  halve_step<L2>(v, 4, lane & 4);
  halve_step<L3>(v, 2, lane & 2);
  halve_step<L4>(v, 1, lane & 1);
}

// Entry held in slot j after warp_sum_halving: undo the exchanges from the last
// one, adding the kept half's offset; a slot that was padding at any exchange is -1.
template <int V>
__device__ __forceinline__ int halving_index(int lane, int j) {
  constexpr int L1 = halved(V), L2 = halved(L1), L3 = halved(L2), L4 = halved(L3), L5 = halved(L4);
  int k = j + ((lane & 1) ? L5 : 0);
  if (k >= L4) return -1;
  k += (lane & 2) ? L4 : 0;
  if (k >= L3) return -1;
  k += (lane & 4) ? L3 : 0;
  if (k >= L2) return -1;
  k += (lane & 8) ? L2 : 0;
  if (k >= L1) return -1;
  k += (lane & 16) ? L1 : 0;
  return k < V ? k : -1;
}

// the 32 lanes of a warp stride over the poles (left and right ranges separately)
// Sum of z_i^2 / Delta_i and (z_i / Delta_i)^2 over i = b + lane, b + lane + 32, ...
// below e, four independent chains per lane.
__device__ __forceinline__ void lane_sums(const double* __restrict__ D, const double* __restrict__ Z,
                                          int b, int e, int lane, double dorg, double tau,
                                          double& sum, double& dsum) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0, d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
  int i = b + lane;
  for (; i + 96 < e; i += 128) {
    const double z0 = Z[i], z1 = Z[i + 32], z2 = Z[i + 64], z3 = Z[i + 96];
    const double t0 = z0 * rcp_refined((D[i] - dorg) - tau);
    const double t1 = z1 * rcp_refined((D[i + 32] - dorg) - tau);
    const double t2 = z2 * rcp_refined((D[i + 64] - dorg) - tau);
    const double t3 = z3 * rcp_refined((D[i + 96] - dorg) - tau);
    a0 = fma(z0, t0, a0);
    d0 = fma(t0, t0, d0);
    a1 = fma(z1, t1, a1);
    d1 = fma(t1, t1, d1);
    a2 = fma(z2, t2, a2);
    d2 = fma(t2, t2, d2);
    a3 = fma(z3, t3, a3);
    d3 = fma(t3, t3, d3);
  }
  for (; i < e; i += 32) {
    const double z0 = Z[i];
    const double t0 = z0 * rcp_refined((D[i] - dorg) - tau);
    a0 = fma(z0, t0, a0);
    d0 = fma(t0, t0, d0);
  }
  sum = (a0 + a1) + (a2 + a3);
  dsum = (d0 + d1) + (d2 + d3);
}

// Adds the terms of poles b + lane, b + lane + 32, ... below e to two chains of
// z^2 / Delta and two of (z / Delta)^2 (the block-expanded sweep keeps them over
// all its near blocks and combines them once).
__device__ __forceinline__ void lane_acc(const double* __restrict__ D, const double* __restrict__ Z,
                                         int b, int e, int lane, double dorg, double tau,
                                         double& a0, double& a1, double& d0, double& d1) {
  int i = b + lane;
  for (; i + 32 < e; i += 64) {
    const double z0 = Z[i], z1 = Z[i + 32];
    const double t0 = z0 * rcp_refined((D[i] - dorg) - tau);
    const double t1 = z1 * rcp_refined((D[i + 32] - dorg) - tau);
    a0 = fma(z0, t0, a0);
    d0 = fma(t0, t0, d0);
    a1 = fma(z1, t1, a1);
    d1 = fma(t1, t1, d1);
  }
  if (i < e) {
    const double z0 = Z[i];
    const double t0 = z0 * rcp_refined((D[i] - dorg) - tau);
    a0 = fma(z0, t0, a0);
    d0 = fma(t0, t0, d0);
  }
}

// All 32 lanes sum one root.  With nb > 0 (block expansion) lane l takes blocks
// l, l + 32, ...: a far block through its series, and the near blocks found in
// each round of 32 are summed exactly by the whole warp.  `pairs` and `blocks`
// count the exact pole terms and the series evaluations (work counters).
struct WarpSweep {
  const double* __restrict__ D;
  const double* __restrict__ Z;
  int K;
  int lane;
  int nb;
  const double* __restrict__ MP;
  const float* __restrict__ MF;
  mutable unsigned long long pairs;
  mutable unsigned blocks;
  mutable unsigned sops;
  int nsb;                         // superblocks (0: none)
  const double* __restrict__ SP;   // their FP64 data
  const float* __restrict__ SF;    // and float data
  // One far block (or superblock) of data C / F with nc entries per field at lane
  // slot b: adds its series to p, dp (left of lambda) or f, df.
  __device__ __forceinline__ void far_series(const double* C, const float* F, int nc, int b,
                                             double dm, double rb, int tier, double& p,
                                             double& dp, double& f, double& df) const {
    const double t = rcp_refined(dm), x = -rb * t;
    const double* ca = C + 3 * nc + b;
    const double* cb = C + (3 + kHv3) * nc + b;
    const float* fa = F + 3 * nc + b;
    const float* fb = F + (3 + kMfTerms) * nc + b;
    double val, der;
    if (tier == 0)
      series_mixed<kMpTiny, kHv0, kHd0>(ca, cb, fa, fb, nc, x, val, der);
    else if (tier == 1)
      series_mixed<kMpShort, kHv1, kHd1>(ca, cb, fa, fb, nc, x, val, der);
    else if (tier == 2)
      series_mixed<kMpMid, kHv2, kHd2>(ca, cb, fa, fb, nc, x, val, der);
    else
      series_mixed<kMpTerms, kHv3, kHd3>(ca, cb, fa, fb, nc, x, val, der);
    if (dm > 0.0) {
      f = fma(t, val, f);
      df = fma(t * t, der, df);
    } else {
      p = fma(t, val, p);
      dp = fma(t * t, der, dp);
    }
  }
  __device__ __forceinline__ SecSums operator()(double dorg, double tau, int jl) const {
    double p = 0.0, dp = 0.0, f = 0.0, df = 0.0;
    if (nb == 0) {
      lane_sums(D, Z, 0, jl + 1, lane, dorg, tau, p, dp);
      lane_sums(D, Z, jl + 1, K, lane, dorg, tau, f, df);
      pairs += unsigned(K);
    } else {
      double pa0 = 0.0, pa1 = 0.0, pd0 = 0.0, pd1 = 0.0;  // near poles left of lambda
      double fa0 = 0.0, fa1 = 0.0, fd0 = 0.0, fd1 = 0.0;  // and right of it
      // one round: the lane's block (or superblock) b of data C / F with nc entries
      // per field through its series if it is far from the point
      auto far_round = [&](const double* C, const float* F, int nc, int b, bool valid) -> bool {
        const double dm = valid ? (C[b] - dorg) - tau : 1.0;  // m - lambda
        const double rb = valid ? C[nc + b] : 0.0;
        const FarTest ft = far_test_bits(dm, rb, valid ? C[2 * nc + b] : 0.0, valid);
        if (ft.far) far_series(C, F, nc, b, dm, rb, ft.tier, p, dp, f, df);
        const unsigned nfar = __popc(__ballot_sync(0xffffffffu, ft.far));
        blocks += nfar;
        sops += nfar * unsigned(kSecSeriesOverhead + (ft.tier == 0   ? kHv0 + kHd0
                                                      : ft.tier == 1 ? kHv1 + kHd1
                                                      : ft.tier == 2 ? kHv2 + kHd2
                                                                     : kHv3 + kHd3));
        return ft.far;
      };
      unsigned sfar = 0;  // superblocks taken whole
      if (nsb > 0) sfar = __ballot_sync(0xffffffffu, far_round(SP, SF, nsb, lane, lane < nsb));
      const KeptBlocks kb = kept_blocks(nsb, sb_size(nb), sfar, nb);
      for (int base = 0; base < kb.count; base += 32) {
        const int b = kept_block(kb, base + lane);
        const bool far = far_round(MP, MF, nb, b < 0 ? 0 : b, b >= 0);
        unsigned nm = __ballot_sync(0xffffffffu, b >= 0 && !far);
        while (nm) {
          const int bb = __shfl_sync(0xffffffffu, b, __ffs(nm) - 1);
          nm &= nm - 1;
          const int i0 = bb * kMpBlock, i1 = (bb == nb - 1) ? K : i0 + kMpBlock;
          const int mid = min(max(jl + 1, i0), i1);
          lane_acc(D, Z, i0, mid, lane, dorg, tau, pa0, pa1, pd0, pd1);
          lane_acc(D, Z, mid, i1, lane, dorg, tau, fa0, fa1, fd0, fd1);
          pairs += unsigned(i1 - i0);
        }
      }
      p += pa0 + pa1;
      dp += pd0 + pd1;
      f += fa0 + fa1;
      df += fd0 + fd1;
    }
    SecSums s;
    warp_sum4(p, dp, f, df);
    s.psi = p;
    s.dpsi = dp;
    s.phi = f;
    s.dphi = df;
    return s;
  }
};

// G lanes (a power of two below 32, aligned) share one root: they stride over the
// poles with the left / right split uniform inside the group and combine with
// shuffles restricted to the group, so groups of one warp may diverge safely.
template <int G, class T>
__device__ __forceinline__ T group_sum(T v, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

// Group sums of four values (G >= 4 lanes): the first exchange leaves the lower
// half of the group the partial sums of a, b and the upper half those of c, d, the
// second one value per quarter, the rest finish each quarter, and shuffles within
// the group broadcast the totals (3 FP64 additions for G = 4 instead of 8).
template <int G>
__device__ __forceinline__ void group_sum4(double& a, double& b, double& c, double& d,
                                           unsigned mask) {
  static_assert(G >= 4 && G <= 32, "four quarters");
  const int gl = threadIdx.x & (G - 1);
  const bool h = gl & (G / 2), q = gl & (G / 4);
  double x0 = h ? c : a, x1 = h ? d : b;
  const double y0 = h ? a : c, y1 = h ? b : d;
  x0 += __shfl_xor_sync(mask, y0, G / 2);
  x1 += __shfl_xor_sync(mask, y1, G / 2);
  double z = q ? x1 : x0;
  z += __shfl_xor_sync(mask, q ? x0 : x1, G / 4);
#pragma unroll
  for (int o = G / 8; o > 0; o >>= 1) z += __shfl_xor_sync(mask, z, o);
  a = __shfl_sync(mask, z, 0, G);
  b = __shfl_sync(mask, z, G / 4, G);
  c = __shfl_sync(mask, z, G / 2, G);
  d = __shfl_sync(mask, z, 3 * G / 4, G);
}

template <int G>
__device__ __forceinline__ void group_lane_sums(const double* __restrict__ D,
                                                const double* __restrict__ Z, int b, int e, int gl,
                                                double dorg, double tau, double& sum, double& dsum) {
  double a0 = 0.0, a1 = 0.0, d0 = 0.0, d1 = 0.0;
  int i = b + gl;
  for (; i + G < e; i += 2 * G) {
    const double z0 = Z[i], z1 = Z[i + G];
    const double t0 = z0 * rcp_refined((D[i] - dorg) - tau);
    const double t1 = z1 * rcp_refined((D[i + G] - dorg) - tau);
    a0 = fma(z0, t0, a0);
    d0 = fma(t0, t0, d0);
    a1 = fma(z1, t1, a1);
    d1 = fma(t1, t1, d1);
  }
  for (; i < e; i += G) {
    const double z0 = Z[i];
    const double t0 = z0 * rcp_refined((D[i] - dorg) - tau);
    a0 = fma(z0, t0, a0);
    d0 = fma(t0, t0, d0);
  }
  sum = a0 + a1;
  dsum = d0 + d1;
}

template <int G>
struct GroupSweep {
  const double* __restrict__ D;
  const double* __restrict__ Z;
  int K;
  int gl;
  unsigned mask;
  __device__ __forceinline__ SecSums operator()(double dorg, double tau, int jl) const {
    double p, dp, f, df;
    group_lane_sums<G>(D, Z, 0, jl + 1, gl, dorg, tau, p, dp);
    group_lane_sums<G>(D, Z, jl + 1, K, gl, dorg, tau, f, df);
    group_sum4<G>(p, dp, f, df, mask);
    SecSums s;
    s.psi = p;
    s.dpsi = dp;
    s.phi = f;
    s.dphi = df;
    return s;
  }
};

// ---- single-precision sweeps -------------------------------------------------
__device__ __forceinline__ float rcp_approx32(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Terms of poles b + l0, b + l0 + st, ... below e at offset tau from the origin
// pole ho, in single precision and in units of S = 1 / inv: with Delta the pole's
// offset divided by S, w = sum z^2/Delta (compensated: c carries the negated low
// part lost so far), dw = sum z^2/Delta^2, hw = sum z^2/Delta^3, and
// Delta = ((hi_i - hi_o) + (lo_i - lo_o)) inv - tau: the hi difference is exact for
// nearby poles, so the offset keeps about 24 bits relative to its own size.
__device__ __forceinline__ void range32(const float2* __restrict__ H, const float* __restrict__ Z,
                                        int b, int e, int l0, int st, float2 ho, float tau,
                                        float inv, float& w, float& dw, float& hw) {
  float s = 0.f, c = 0.f, d = 0.f, h = 0.f;
  for (int i = b + l0; i < e; i += st) {
    const float2 p = H[i];
    const float z = Z[i];
    const float del = fmaf((p.x - ho.x) + (p.y - ho.y), inv, -tau);
    const float r = rcp_approx32(del);
    const float t = z * r;
    const float y = fmaf(z, t, -c);
    const float ns = s + y;
    c = (ns - s) - y;
    s = ns;
    d = fmaf(t, t, d);
    h = fmaf(t, t * r, h);
  }
  w = s - c;
  dw = d;
  hw = h;
}

// range32 with four terms formed before they are added, in range32's order (the
// same sums bit for bit): more independent work per lane for the short loops of the
// group sweeps.
__device__ __forceinline__ void range32_x4(const float2* __restrict__ H, const float* __restrict__ Z,
                                           int b, int e, int l0, int st, float2 ho, float tau,
                                           float inv, float& w, float& dw, float& hw) {
  float s = 0.f, c = 0.f, d = 0.f, h = 0.f;
  int i = b + l0;
  for (; i + 3 * st < e; i += 4 * st) {
    float zz[4], tt[4], rr[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float2 p = H[i + u * st];
      zz[u] = Z[i + u * st];
      const float del = fmaf((p.x - ho.x) + (p.y - ho.y), inv, -tau);
      rr[u] = rcp_approx32(del);
      tt[u] = zz[u] * rr[u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float y = fmaf(zz[u], tt[u], -c);
      const float ns = s + y;
      c = (ns - s) - y;
      s = ns;
      d = fmaf(tt[u], tt[u], d);
      h = fmaf(tt[u], tt[u] * rr[u], h);
    }
  }
  for (; i < e; i += st) {
    const float2 p = H[i];
    const float z = Z[i];
    const float del = fmaf((p.x - ho.x) + (p.y - ho.y), inv, -tau);
    const float r = rcp_approx32(del);
    const float t = z * r;
    const float y = fmaf(z, t, -c);
    const float ns = s + y;
    c = (ns - s) - y;
    s = ns;
    d = fmaf(t, t, d);
    h = fmaf(t, t * r, h);
  }
  w = s - c;
  dw = d;
  hw = h;
}

// Float copies of the active poles.  `resolves`: whether they resolve the interval
// of the given width between poles jl < jr (or, for the last root, above jr): the
// width must reach 2^-28 of the shifted pole magnitudes |D - shift|.
struct Copies32 {
  const float2* __restrict__ H;
  const float* __restrict__ Z;
  int K;
  __device__ __forceinline__ bool resolves(int jl, int jr, bool, double width) const {
    return width >= 0x1p-28 * double(fmaxf(fabsf(H[jl].x), fabsf(H[jr].x)));
  }
};

struct ThreadSweep32 : Copies32 {
  __device__ __forceinline__ Sec32 operator()(int org, int jl, float tau, float inv) const {
    const float2 ho = H[org];
    Sec32 s;
    float hl, hr;
    range32(H, Z, 0, jl + 1, 0, 1, ho, tau, inv, s.psi, s.dpsi, hl);
    range32(H, Z, jl + 1, K, 0, 1, ho, tau, inv, s.phi, s.dphi, hr);
    s.hw = hl + hr;
    return s;
  }
};

template <int G>
struct GroupSweep32 : Copies32 {
  int gl;
  unsigned mask;
  __device__ __forceinline__ Sec32 operator()(int org, int jl, float tau, float inv) const {
    const float2 ho = H[org];
    float p, dp, hl, f, df, hr;
    range32_x4(H, Z, 0, jl + 1, gl, G, ho, tau, inv, p, dp, hl);
    range32_x4(H, Z, jl + 1, K, gl, G, ho, tau, inv, f, df, hr);
    Sec32 s;
    s.psi = group_sum<G>(p, mask);
    s.dpsi = group_sum<G>(dp, mask);
    s.phi = group_sum<G>(f, mask);
    s.dphi = group_sum<G>(df, mask);
    s.hw = group_sum<G>(hl + hr, mask);
    return s;
  }
};

// Single-precision sums of the warp kernel (all 32 lanes on one root).  With nb > 0
// a sweep first takes the far superblocks (nsb > 0; one per lane), then goes block
// by block over the superblocks it did not take whole, 32 blocks per round: far
// blocks through their float series, near blocks term by term by the whole warp.
struct WarpSweep32 : Copies32 {
  int lane;
  int nb;
  const float* __restrict__ BF;
  int nsb;                         // superblocks (0: none)
  const float* __restrict__ SF;    // their float data (the blocks' layout, nsb entries per field)
  // lane's block (or superblock) b of float data F with nc entries per field, at
  // offset d (units of S) from the point: far -> its series into (p, dp) or (f, df), h
  __device__ __forceinline__ bool far_series32(const float* F, int nc, int b, bool valid, float2 ho,
                                               float tau, float inv, float& p, float& dp, float& f,
                                               float& df, float& h) const {
    const float d = valid ? fmaf((F[b] - ho.x) + (F[nc + b] - ho.y), inv, -tau) : 1.f;
    const float rs = valid ? F[2 * nc + b] * inv : 0.f;
    const bool far = valid && 3.f * rs <= fabsf(d);
    const bool tail = __all_sync(0xffffffffu, !far || 16.f * rs <= fabsf(d));
    if (far) {
      const float q = rcp_approx32(d), x = -rs * q;
      const float* A = F + 3 * nc + b;
      float va, vb, vc;
      if (tail) {
        va = A[(kMfShort - 1) * nc];
        vb = A[(kMfTerms + kMfShort - 1) * nc];
        vc = A[(2 * kMfTerms + kMfShort - 1) * nc];
#pragma unroll
        for (int k = kMfShort - 2; k >= 0; --k) {
          va = fmaf(va, x, A[k * nc]);
          vb = fmaf(vb, x, A[(kMfTerms + k) * nc]);
          vc = fmaf(vc, x, A[(2 * kMfTerms + k) * nc]);
        }
      } else {
        va = A[(kMf32 - 1) * nc];
        vb = A[(kMfTerms + kMf32 - 1) * nc];
        vc = A[(2 * kMfTerms + kMf32 - 1) * nc];
#pragma unroll
        for (int k = kMf32 - 2; k >= 0; --k) {
          va = fmaf(va, x, A[k * nc]);
          vb = fmaf(vb, x, A[(kMfTerms + k) * nc]);
          vc = fmaf(vc, x, A[(2 * kMfTerms + k) * nc]);
        }
      }
      const float q2 = q * q;
      if (d > 0.f) {
        f = fmaf(q, va, f);
        df = fmaf(q2, vb, df);
      } else {
        p = fmaf(q, va, p);
        dp = fmaf(q2, vb, dp);
      }
      h = fmaf(q2 * q, vc, h);
    }
    return far;
  }
  __device__ __forceinline__ Sec32 operator()(int org, int jl, float tau, float inv) const {
    const float2 ho = H[org];
    float p = 0.f, dp = 0.f, f = 0.f, df = 0.f, h = 0.f;
    if (nb == 0) {
      float hl, hr;
      range32(H, Z, 0, jl + 1, lane, 32, ho, tau, inv, p, dp, hl);
      range32(H, Z, jl + 1, K, lane, 32, ho, tau, inv, f, df, hr);
      h = hl + hr;
    } else {
      unsigned sfar = 0;  // superblocks taken whole
      if (nsb > 0)
        sfar = __ballot_sync(0xffffffffu, far_series32(SF, nsb, lane, lane < nsb, ho, tau, inv, p, dp,
                                                        f, df, h));
      const KeptBlocks kb = kept_blocks(nsb, sb_size(nb), sfar, nb);
      for (int base = 0; base < kb.count; base += 32) {
        const int b = kept_block(kb, base + lane);
        const bool far = far_series32(BF, nb, b < 0 ? 0 : b, b >= 0, ho, tau, inv, p, dp, f, df, h);
        unsigned nm = __ballot_sync(0xffffffffu, b >= 0 && !far);
        while (nm) {
          const int bb = __shfl_sync(0xffffffffu, b, __ffs(nm) - 1);
          nm &= nm - 1;
          const int i0 = bb * kMpBlock, i1 = (bb == nb - 1) ? K : i0 + kMpBlock;
          const int mid = min(max(jl + 1, i0), i1);
          float w, dw, hw;
          range32(H, Z, i0, mid, lane, 32, ho, tau, inv, w, dw, hw);
          p += w;
          dp += dw;
          h += hw;
          range32(H, Z, mid, i1, lane, 32, ho, tau, inv, w, dw, hw);
          f += w;
          df += dw;
          h += hw;
        }
      }
    }
    Sec32 s;
    s.psi = group_sum<32>(p, 0xffffffffu);
    s.dpsi = group_sum<32>(dp, 0xffffffffu);
    s.phi = group_sum<32>(f, 0xffffffffu);
    s.dphi = group_sum<32>(df, 0xffffffffu);
    s.hw = group_sum<32>(h, 0xffffffffu);
    return s;
  }
};

// ---- kernels ------------------------------------------------------------------
__device__ __forceinline__ void secular_store(const RootArgs& a, int lo, int j, int org, double tau,
                                              int sweeps, int K, bool ok, bool leader) {
  if (leader) {
    if (!ok) set_status(a.st, TDE_ENOCONV);
    const double dorg = a.AD[lo + org];
    a.TAU[lo + j] = tau;
    a.ORG[lo + j] = org;
    a.DORG[lo + j] = dorg;
    a.LAMA[lo + j] = dorg + tau;
  }
}

// per-thread tallies of the device work counters, flushed once per thread
struct SecTally {
  unsigned long long pairs = 0, sops = 0;
  unsigned sweeps = 0, pairs32 = 0, sweeps32 = 0, roots = 0, blocks = 0;
  __device__ __forceinline__ void add(int n64, int n32, int K) {
    add_counted((unsigned long long)n64 * unsigned(K), 0u, 0u, n64, n32, K);
  }
  // FP64 work given as exact pole terms and block series evaluations (and their
  // FP64 operations)
  __device__ __forceinline__ void add_counted(unsigned long long exact, unsigned nblocks,
                                              unsigned nops, int n64, int n32, int K) {
    pairs += exact;
    blocks += nblocks;
    sops += nops;
    sweeps += unsigned(n64);
    pairs32 += unsigned(n32) * unsigned(K);
    sweeps32 += unsigned(n32);
    roots += 1;
  }
  __device__ __forceinline__ void flush(Status* st) const {
    if (!roots) return;
    atomicAdd(&st->work[kWorkSecularPairs], pairs);
    if (blocks) atomicAdd(&st->work[kWorkSecularFarBlocks], (unsigned long long)blocks);
    if (sops) atomicAdd(&st->work[kWorkSecularSeriesOps], sops);
    atomicAdd(&st->work[kWorkSecularSweeps], (unsigned long long)sweeps);
    atomicAdd(&st->work[kWorkSecular32Pairs], (unsigned long long)pairs32);
    atomicAdd(&st->work[kWorkSecular32Sweeps], (unsigned long long)sweeps32);
    atomicAdd(&st->work[kWorkRoots], (unsigned long long)roots);
  }
};

// Root r of the warp kernels' list: the large-K list, then the small-K list when
// that one is too short for the thread kernels.
__device__ __forceinline__ uint32_t warp_list_total(const RootArgs& a) {
  const uint32_t small = *a.count;
  return *a.count2 + (small < a.small_list_min ? small : 0u);
}
// Merge of entry r of that combined list; *in_list receives r's index within its
// own list, which is what a merge's `base` refers to.
__device__ __forceinline__ int warp_list_merge(const RootArgs& a, uint32_t r, int* in_list) {
  const uint32_t nb = *a.count2;
  if (r < nb) {
    *in_list = int(r);
    return a.ROOTMAP2[r];
  }
  *in_list = int(r - nb);
  return a.ROOTMAP[r - nb];
}

// Block centres, radii and moments (BlockFar) of the merges whose roots
// k_secular_warp solves and whose K reaches mp_min_k, one warp per block: warps
// walk that kernel's root list 32 roots at a time, and root j = 128 b stands for
// block b.
__global__ void __launch_bounds__(128) k_block_moments(RootArgs a) {
  const uint32_t total = warp_list_total(a);
  const int lane = threadIdx.x & 31;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t base = gw * 32; base < total; base += nw * 32) {
    const uint32_t r = base + lane;
    int g = 0, j = 0, nb = 0;
    bool head = false;
    if (r < total) {
      int rl;
      g = warp_list_merge(a, r, &rl);
      const MState ms = a.ms[g];
      j = rl - ms.base;
      nb = mp_blocks(ms.K, a.mp_min_k);
      head = nb > 0 && (j % kMpBlock) == 0 && j / kMpBlock < nb;
    }
    unsigned hm = __ballot_sync(0xffffffffu, head);
    while (hm) {
      const int src = __ffs(hm) - 1;
      hm &= hm - 1;
      const int gg = __shfl_sync(0xffffffffu, g, src), b = __shfl_sync(0xffffffffu, j, src) / kMpBlock;
      const int nbb = __shfl_sync(0xffffffffu, nb, src);
      const int lo = a.M[gg].lo, K = a.ms[gg].K;
      const double* D = a.AD + lo;
      const double* Z = a.AZ + lo;
      const int i0 = b * kMpBlock, i1 = (b == nbb - 1) ? K : i0 + kMpBlock;
      const double m = 0.5 * (D[i0] + D[i1 - 1]);
      const double rad = fmax(m - D[i0], D[i1 - 1] - m);
      double mo[kMfTerms];  // normalised: sum z^2 ((D_i - m) / r)^k
#pragma unroll
      for (int k = 0; k < kMfTerms; ++k) mo[k] = 0.0;
      const double rinv = rad > 0.0 ? 1.0 / rad : 0.0;
      for (int i = i0 + lane; i < i1; i += 32) {
        const double y = (D[i] - m) * rinv;
        double pn = Z[i] * Z[i];
#pragma unroll
        for (int k = 0; k < kMfTerms; ++k) {
          mo[k] += pn;
          pn *= y;
        }
      }
      warp_sum_halving(mo, lane);
      double* MP = a.MPD + lo;
      float* BF = reinterpret_cast<float*>(MP + kMpFields * nbb);
      if (lane == 0) {
        MP[b] = m;
        MP[nbb + b] = rad;
        MP[2 * nbb + b] = 3.0 * rad;
        const double c = m - a.ms[gg].shift;
        const float ch = __double2float_rn(c);
        BF[b] = ch;
        BF[nbb + b] = __double2float_rn(c - double(ch));
        BF[2 * nbb + b] = __double2float_rn(rad);
      }
#pragma unroll
      for (int jj = 0; jj < warp_halved_len(kMfTerms); ++jj) {
        const int k = halving_index<kMfTerms>(lane, jj);
        if (k >= 0) {
          const double m0 = mo[jj], m1 = double(k + 1) * m0;
          if (k < kHv3) MP[(3 + k) * nbb + b] = m0;
          if (k < kHd3) MP[(3 + kHv3 + k) * nbb + b] = m1;
          BF[(3 + k) * nbb + b] = __double2float_rn(m0);
          BF[(3 + kMfTerms + k) * nbb + b] = __double2float_rn(m1);
          if (k < kMf32)
            BF[(3 + 2 * kMfTerms + k) * nbb + b] = __double2float_rn(0.5 * double(k + 2) * m1);
        }
      }
    }
  }
}

// Superblock data from the block data (one warp per superblock, lane = block): with
// the superblock's centre m_S and radius R, a = (m_b - m_S) / R and c = r_b / R
// (|a| + c <= 1), its normalised moments are the exact binomial translation
//   M'_k = sum_b sum_{j<=k} C(k, j) a^(k-j) c^j M'^b_j,
// summed over the blocks; each term is bounded by the block's M'_0, so the shift
// adds no cancellation.  M'^b_j comes from the FP64 heads for j < 21 (which alone
// make the superblock's FP64 heads) and from the float copies above.
__global__ void __launch_bounds__(128) k_super_moments(RootArgs a) {
  const uint32_t total = warp_list_total(a);
  const int lane = threadIdx.x & 31;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t base = gw * 32; base < total; base += nw * 32) {
    const uint32_t r = base + lane;
    int g = 0, j = 0, nsb = 0, nb = 0;
    bool head = false;
    if (r < total) {
      int rl;
      g = warp_list_merge(a, r, &rl);
      const MState ms = a.ms[g];
      j = rl - ms.base;
      nb = mp_blocks(ms.K, a.mp_min_k);
      nsb = sb_count(nb);
      const int sbp = sb_size(nb) * kMpBlock;  // poles per superblock
      head = nsb > 0 && (j % sbp) == 0 && j / sbp < nsb;
    }
    unsigned hm = __ballot_sync(0xffffffffu, head);
    while (hm) {
      const int src = __ffs(hm) - 1;
      hm &= hm - 1;
      const int gg = __shfl_sync(0xffffffffu, g, src);
      const int nbb = __shfl_sync(0xffffffffu, nb, src), nss = __shfl_sync(0xffffffffu, nsb, src);
      const int sbs = sb_size(nbb), sbp = sbs * kMpBlock;
      const int sb = __shfl_sync(0xffffffffu, j, src) / sbp;
      const int lo = a.M[gg].lo, K = a.ms[gg].K;
      const double* D = a.AD + lo;
      const int i0 = sb * sbp, i1 = (sb == nss - 1) ? K : i0 + sbp;
      const double m = 0.5 * (D[i0] + D[i1 - 1]);
      const double rad = fmax(m - D[i0], D[i1 - 1] - m);
      const double rinv = rad > 0.0 ? 1.0 / rad : 0.0;
      const double* MP = a.MPD + lo;
      const float* BF = reinterpret_cast<const float*>(MP + kMpFields * nbb);
      double* SP = sb_data(a.MPD + lo, nbb);
      float* SF = reinterpret_cast<float*>(SP + kMpFields * nss);
      const int b = sb * sbs + lane;
      double S[kMfTerms];
#pragma unroll
      for (int k = 0; k < kMfTerms; ++k) S[k] = 0.0;
      if (b < nbb && lane < sbs) {
        const double av = (MP[b] - m) * rinv, cv = MP[nbb + b] * rinv;
        double cj = 1.0;  // S_q = c^q M'^b_q, then shifted by a
#pragma unroll
        for (int q = 0; q < kMfTerms; ++q) {
          const double mj = q < kHv3 ? MP[(3 + q) * nbb + b] : double(BF[(3 + q) * nbb + b]);
          S[q] = cj * mj;
          cj *= cv;
        }
        binomial_shift(S, av);
      }
      warp_sum_halving(S, lane);
      if (lane == 0) {
        SP[sb] = m;
        SP[nss + sb] = rad;
        SP[2 * nss + sb] = 3.0 * rad;
        const double c = m - a.ms[gg].shift;  // the single-precision stage's centre pair
        const float ch = __double2float_rn(c);
        SF[sb] = ch;
        SF[nss + sb] = __double2float_rn(c - double(ch));
        SF[2 * nss + sb] = __double2float_rn(rad);
      }
#pragma unroll
      for (int jj = 0; jj < warp_halved_len(kMfTerms); ++jj) {
        const int k = halving_index<kMfTerms>(lane, jj);
        if (k >= 0) {
          const double m0 = S[jj], m1 = double(k + 1) * m0;
          if (k < kHv3) SP[(3 + k) * nss + sb] = m0;
          if (k < kHd3) SP[(3 + kHv3 + k) * nss + sb] = m1;
          SF[(3 + k) * nss + sb] = __double2float_rn(m0);
          SF[(3 + kMfTerms + k) * nss + sb] = __double2float_rn(m1);
          if (k < kMf32)
            SF[(3 + 2 * kMfTerms + k) * nss + sb] = __double2float_rn(0.5 * double(k + 2) * m1);
        }
      }
    }
  }
}

// One thread per root.  The loop over roots advances a whole warp at a time (32
// consecutive roots), which keeps every lane in step for the warp votes of
// secular_root_sync.
__global__ void k_secular_thread(RootArgs a) {
  const uint32_t total = *a.count;
  if (total < a.small_list_min) return;  // the warp kernel takes a short list
  const int lane = threadIdx.x & 31;
  SecTally tally;
  for (uint32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < total;
       base += gridDim.x * blockDim.x) {
    const uint32_t r = base + lane;
    const bool valid = r < total;
    const int g = valid ? a.ROOTMAP[r] : 0;
    const MState ms = valid ? a.ms[g] : MState{};
    const int j = int(r) - ms.base, lo = valid ? a.M[g].lo : 0, K = valid ? ms.K : 0;
    ThreadSweep sw{a.AD + lo, a.AZ + lo, K};
    ThreadSweep32 sw32{{a.AD32 + lo, a.AZ32 + lo, K}};
    int org = 0, n32 = 0;
    double tau = 0.0;
    bool ok = true;
    const int sweeps = secular_root_sync(a.AD + lo, a.AZ + lo, K, j, ms.rho, ms.rhoinv, ms.zsq, valid, sw,
                                         sw32, &org, &tau, &ok, &n32);
    if (valid) {
      secular_store(a, lo, j, org, tau, sweeps, K, ok, true);
      tally.add(sweeps, n32, K);
    }
  }
  tally.flush(a.st);
}

// ---------------------------------------------------------------------------
// Small-K roots with refill (a forest's thread-per-root steps).  Warp-synchronous
// rounds (secular_root_sync) keep the roots of a warp in step, so a warp pays for as
// many sweeps of each kind as its slowest root needs, and the FP64 units take a warp
// instruction's full time however few lanes it carries.
// Here each group of G lanes runs its root through the same steps as a state
// machine and claims the next root of the list as soon as its root is done.  A pass
// of the loop gives every group that needs one a single-precision sweep; FP64
// sweeps wait until no group is in its single-precision stage and no idle group can
// still claim a root, and then run for every waiting group at once, so that the
// FP64 passes stay as full as the warp-synchronous rounds.  A root's operations and
// their order are those of secular_root_sync, so its result is the same bit for bit.
enum : int { kRootIdle = 0, kRootF32First, kRootF32, kRootF64Init, kRootF64, kRootF64Wait };

template <int G>
struct SmallSweeps {
  __device__ static GroupSweep<G> f64(const RootArgs& a, int lo, int K, int gl, unsigned mask) {
    return GroupSweep<G>{a.AD + lo, a.AZ + lo, K, gl, mask};
  }
  __device__ static GroupSweep32<G> f32(const RootArgs& a, int lo, int K, int gl, unsigned mask) {
    return GroupSweep32<G>{{a.AD32 + lo, a.AZ32 + lo, K}, gl, mask};
  }
};
template <>
struct SmallSweeps<1> {
  __device__ static ThreadSweep f64(const RootArgs& a, int lo, int K, int, unsigned) {
    return ThreadSweep{a.AD + lo, a.AZ + lo, K};
  }
  __device__ static ThreadSweep32 f32(const RootArgs& a, int lo, int K, int, unsigned) {
    return ThreadSweep32{{a.AD32 + lo, a.AZ32 + lo, K}};
  }
};

// The roots of the small-K list (total entries), claimed through st->claim_next
// (the caller resets it with claim_finish_block).  All 32 lanes call it together.
template <int G>
__device__ void secular_roots_refill(const RootArgs& a, uint32_t total, SecTally& tally) {
  constexpr unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31, gl = lane & (G - 1), first = lane & ~(G - 1);
  const unsigned mask = ((G == 32) ? kFull : ((1u << G) - 1u)) << first;
  const bool leader = gl == 0;
  const unsigned below = (1u << lane) - 1u;
  int phase = kRootIdle;
  bool more = true;  // the list may still hold unclaimed roots (warp-uniform)
  int lo = 0, K = 0, j = 0, n32 = 0, sweeps = 0;
  double rho = 0.0, rhoinv = 0.0, zsq = 0.0, hw = 0.0;
  bool third = false, handed = false, ok = true;
  const double *D = a.AD, *Z = a.AZ;
  Stage32 st;
  st.live = false;
  st.org = 0;
  st.jl = 0;
  st.tau = 0.0f;
  st.inv = 1.0f;
  SecState q;
  q.org = 0;
  q.jl = 0;
  q.tau = 0.0;
  q.dorg = 0.0;
  for (;;) {
    // 1. idle groups claim the next entries of the list
    const unsigned idle = __ballot_sync(kFull, leader && phase == kRootIdle);
    if (more && idle) {
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(&a.st->claim_next, unsigned(__popc(idle)));
      base = __shfl_sync(kFull, base, 0);
      more = base + unsigned(__popc(idle)) < total;
      const uint32_t r = __shfl_sync(kFull, base + unsigned(__popc(idle & below)), first);
      if (phase == kRootIdle && r < total) {
        const int g = a.ROOTMAP[r];
        const MState ms = a.ms[g];
        lo = a.M[g].lo;
        K = ms.K;
        j = int(r) - ms.base;
        rho = ms.rho;
        rhoinv = ms.rhoinv;
        zsq = ms.zsq;
        D = a.AD + lo;
        Z = a.AZ + lo;
        n32 = 0;
        sweeps = 0;
        hw = 0.0;
        third = handed = false;
        ok = true;
        if (K <= 1) {  // a single pole: the root is D_0 + rho z_0^2
          secular_store(a, lo, j, 0, rho * Z[0] * Z[0], 0, K, true, leader);
          tally.add(0, 0, K);
        } else if (s32_begin(D, K, j, rho, rhoinv, zsq, SmallSweeps<G>::f32(a, lo, K, gl, mask), st)) {
          phase = kRootF32First;
        } else {
          st.live = false;
          sec_init_point(D, K, j, rho, rhoinv, zsq, q);
          phase = kRootF64Init;
        }
      }
    }
    if (!__any_sync(kFull, phase != kRootIdle)) {
      if (!more) break;
      continue;
    }
    // 2. the steps that decide this pass's sweeps
    bool step32 = false, have = false, hand = false, go = false, done = false;
    float eta = 0.0f;
    if (phase == kRootF32) {
      step32 = st.live && s32_step(st, &eta, &have);
      hand = !step32;
    } else if (phase == kRootF64) {
      if (sec_step(q, hw, third) == 0) {
        done = true;
      } else if (sweeps >= kMaxSweeps) {
        ok = false;
        done = true;
      } else {
        go = true;  // w''/2 at the new point now (third-order steps), the sweep when due
        phase = kRootF64Wait;
      }
    }
    // 3. single-precision sweeps: the stage's, and w''/2 at the FP64 stage's point
    const bool want_hw = go && third;
    const bool s32 = phase == kRootF32First || step32 || want_hw;
    if (__any_sync(kFull, s32) && s32) {
      const Sec32 r32 = SmallSweeps<G>::f32(a, lo, K, gl, mask)(
          want_hw ? q.org : st.org, want_hw ? q.jl : st.jl,
          want_hw ? float(q.tau * st.Sinv) : st.tau, st.inv);
      if (want_hw) {
        hw = hw_natural(st, r32.hw);
        ++n32;
      } else {
        st.s = r32;
        if (phase == kRootF32First) {
          s32_first(D, Z, K, j, st);
          phase = kRootF32;
        } else {
          s32_after(st, eta, have);
        }
      }
    }
    // 4. hand-over to the FP64 stage (or its midpoint start)
    if (hand) {
      n32 = st.sweeps;
      bool hw_ok;
      handed = s32_finish(D, Z, rhoinv, st, q, &hw, &hw_ok);
      third = handed && hw_ok;
      if (!handed) sec_init_point(D, K, j, rho, rhoinv, zsq, q);
      phase = kRootF64Init;
    }
    // 5. FP64 sweeps (the stage's first, and the iterations') of all waiting groups,
    //    once no group is in the single-precision stage or could still claim a root
    const bool waits = phase == kRootF64Init || phase == kRootF64Wait;
    const bool busy32 = phase == kRootF32First || phase == kRootF32 || (more && phase == kRootIdle);
    if (__any_sync(kFull, waits) && !__any_sync(kFull, busy32) && waits) {
      q.s = SmallSweeps<G>::f64(a, lo, K, gl, mask)(q.dorg, q.tau, q.jl);
      if (phase == kRootF64Init) {
        if (handed)
          q.w = q.rhoinv + q.s.psi + q.s.phi;
        else
          sec_init_finish(D, Z, K, j, rho, zsq, q);
        sweeps = 1;
        phase = kRootF64;
      } else {
        q.w = q.rhoinv + q.s.psi + q.s.phi;
        ++sweeps;
        phase = kRootF64;
      }
    }
    // 6. finished roots
    if (done) {
      secular_store(a, lo, j, q.org, q.tau, sweeps, K, ok, leader);
      tally.add(sweeps, n32, K);
      phase = kRootIdle;
    }
  }
}

// The small-K list with refill (G lanes per root; one thread per root for G = 1),
// 444 blocks of 128 threads claiming roots from the list.
template <int G>
__global__ void __launch_bounds__(128) k_secular_small(RootArgs a) {
  const uint32_t total = *a.count;
  if (total < a.small_list_min) return;  // the warp kernel takes a short list
  SecTally tally;
  secular_roots_refill<G>(a, total, tally);
  if ((threadIdx.x & (G - 1)) == 0) tally.flush(a.st);
  claim_finish_block(a.st);
}

// Warp-cooperative form for the warp kernel: lane l owns one root (its own merge,
// origin, bracket and model state), and every sweep is summed by the whole warp,
// one root at a time.  Each round the warp sweeps, in turn, every root that needs a
// sweep (ballot), broadcasting its point (origin, tau, jl) and its merge; lane l
// keeps the sums of its own root (the warp reductions are butterflies, so every
// lane holds the same totals).  The per-root scalar work (the model step,
// convergence test, the stage hand-over) then runs once for all 32 roots, lane
// parallel, instead of once per root at warp width: on this part an FP64
// instruction occupies the pipe for the whole warp however few lanes are active.
// Same steps and stopping rules as secular_root; all 32 lanes must call it.
// `co` supplies the cooperative sweeps: sweep32(src, org, jl, tau, inv) and
// sweep64(src, dorg, tau, jl) sum the root of lane src.  G < 32: the sweeps are
// summed by groups of G lanes instead of the whole warp; a pass then takes G
// rounds, in round i every group sums the root of its i-th lane, and the roots'
// scalar work still runs once for all 32 roots.
template <int G, class Coop, class Copies>
__device__ int secular_root_coop(const double* D, const double* Z, int K, int j, double rho,
                                 double rhoinv, double zsq, bool valid, const Copies& cp, Coop& co,
                                 int* org_out, double* tau_out, bool* ok, int* n32) {
  static_assert(G == 32 || (G >= 2 && G <= 16 && (G & (G - 1)) == 0), "lanes per sweep");
  constexpr unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int first = lane & ~(G - 1);
  const unsigned gm = (G == 32) ? kFull : (((1u << (G & 31)) - 1u) << first);
  *ok = true;
  *n32 = 0;
  const bool act = valid && K > 1;
  Stage32 st;
  st.live = false;
  st.org = 0;
  st.jl = 0;
  st.tau = 0.0f;
  st.inv = 1.0f;
  // cooperative single-precision sweeps of the flagged lanes at (org, jl, tf, st.inv)
  auto sweep32_all = [&](bool flag, int org, int jl, float tf, Sec32& out) {
    if constexpr (G == 32) {
      unsigned m = __ballot_sync(kFull, flag);
      while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const Sec32 s = co.sweep32(src, __shfl_sync(kFull, org, src), __shfl_sync(kFull, jl, src),
                                   __shfl_sync(kFull, tf, src), __shfl_sync(kFull, st.inv, src));
        if (lane == src) out = s;
      }
    } else {
#pragma unroll 1
      for (int i = 0; i < G; ++i) {
        const int src = first + i;
        const bool f = __shfl_sync(kFull, flag, src);  // uniform within each group
        if (!__any_sync(kFull, f)) continue;
        if (f) {
          const Sec32 s = co.sweep32(src, __shfl_sync(gm, org, src), __shfl_sync(gm, jl, src),
                                     __shfl_sync(gm, tf, src), __shfl_sync(gm, st.inv, src));
          if (lane == src) out = s;
        }
      }
    }
  };
  const bool in32 = act && s32_begin(D, K, j, rho, rhoinv, zsq, cp, st);
  sweep32_all(in32, st.org, st.jl, st.tau, st.s);
  if (in32) s32_first(D, Z, K, j, st);
  for (;;) {
    float eta = 0.0f;
    bool have = false;
    const bool need = in32 && st.live && s32_step(st, &eta, &have);
    if (!__any_sync(kFull, need)) break;
    sweep32_all(need, st.org, st.jl, st.tau, st.s);
    if (need) s32_after(st, eta, have);
  }
  SecState q;
  q.org = 0;
  q.jl = 0;
  q.tau = 0.0;
  q.dorg = 0.0;
  double hw = 0.0;
  bool third = false, handed = false;
  if (in32) {
    *n32 = st.sweeps;
    bool hw_ok;
    handed = s32_finish(D, Z, rhoinv, st, q, &hw, &hw_ok);
    third = handed && hw_ok;
  }
  if (act && !handed) sec_init_point(D, K, j, rho, rhoinv, zsq, q);
  // cooperative FP64 sweeps of the flagged lanes at (q.dorg, q.tau, q.jl)
  auto sweep64_all = [&](bool flag) {
    if constexpr (G == 32) {
      unsigned m = __ballot_sync(kFull, flag);
      while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const SecSums s = co.sweep64(src, __shfl_sync(kFull, q.dorg, src), __shfl_sync(kFull, q.tau, src),
                                     __shfl_sync(kFull, q.jl, src));
        if (lane == src) q.s = s;
      }
    } else {
#pragma unroll 1
      for (int i = 0; i < G; ++i) {
        const int src = first + i;
        const bool f = __shfl_sync(kFull, flag, src);
        if (!__any_sync(kFull, f)) continue;
        if (f) {
          const SecSums s = co.sweep64(src, __shfl_sync(gm, q.dorg, src), __shfl_sync(gm, q.tau, src),
                                       __shfl_sync(gm, q.jl, src));
          if (lane == src) q.s = s;
        }
      }
    }
  };
  sweep64_all(act);
  if (act) {
    if (handed)
      q.w = q.rhoinv + q.s.psi + q.s.phi;
    else
      sec_init_finish(D, Z, K, j, rho, zsq, q);
  }
  int sweeps = act ? 1 : 0;
  bool go = act;
  for (;;) {
    if (go) {
      if (sec_step(q, hw, third) == 0) {
        go = false;
      } else if (sweeps >= kMaxSweeps) {
        *ok = false;
        go = false;
      }
    }
    if (!__any_sync(kFull, go)) break;
    // w''/2 at the new point from a single-precision sweep (third-order steps)
    const bool h3 = go && third;
    Sec32 s3;
    sweep32_all(h3, q.org, q.jl, h3 ? float(q.tau * st.Sinv) : 0.0f, s3);
    if (h3) {
      hw = hw_natural(st, s3.hw);
      ++*n32;
    }
    sweep64_all(go);
    if (go) {
      q.w = q.rhoinv + q.s.psi + q.s.phi;
      ++sweeps;
    }
  }
  if (valid && K == 1) {
    *org_out = 0;
    *tau_out = rho * Z[0] * Z[0];
    return 0;
  }
  *org_out = q.org;
  *tau_out = q.tau;
  return sweeps;
}

// Cooperative sweeps of the warp kernel: the root of lane src lives in the merge at
// row lo (order K, nb pole blocks, nsb superblocks), broadcast from that lane; the
// FP64 work counters accumulate warp-uniformly.
struct WarpCoop {
  const RootArgs* a;
  int lane, lo, K, nb;
  unsigned long long pairs = 0;
  unsigned blocks = 0, sops = 0;
  __device__ __forceinline__ void merge_of(int src, int& slo, int& sK, int& snb) const {
    slo = __shfl_sync(0xffffffffu, lo, src);
    sK = __shfl_sync(0xffffffffu, K, src);
    snb = __shfl_sync(0xffffffffu, nb, src);
  }
  __device__ __forceinline__ Sec32 sweep32(int src, int org, int jl, float tau, float inv) const {
    int slo, sK, snb;
    merge_of(src, slo, sK, snb);
    const float* mf = reinterpret_cast<const float*>(a->MPD + slo + kMpFields * snb);
    const int nsb = sb_count(snb);
    const double* sp = sb_data(a->MPD + slo, snb);
    const WarpSweep32 sw{{a->AD32 + slo, a->AZ32 + slo, sK}, lane, snb, mf, nsb,
                         reinterpret_cast<const float*>(sp + kMpFields * nsb)};
    return sw(org, jl, tau, inv);
  }
  __device__ __forceinline__ SecSums sweep64(int src, double dorg, double tau, int jl) {
    int slo, sK, snb;
    merge_of(src, slo, sK, snb);
    const float* mf = reinterpret_cast<const float*>(a->MPD + slo + kMpFields * snb);
    const int nsb = sb_count(snb);
    const double* sp = sb_data(a->MPD + slo, snb);
    const WarpSweep sw{a->AD + slo, a->AZ + slo, sK, lane, snb, a->MPD + slo, mf, 0ull, 0u, 0u, nsb, sp,
                       reinterpret_cast<const float*>(sp + kMpFields * nsb)};
    const SecSums s = sw(dorg, tau, jl);
    pairs += sw.pairs;
    blocks += sw.blocks;
    sops += sw.sops;
    return s;
  }
};

// The warp kernel takes its list in tiles of T consecutive entries, one root per
// lane (lanes T..31 idle in the scalar steps, busy in every sweep).  T is the
// power of two at or below a quarter of the list length per launched warp, capped
// at 32: a warp sweeps the roots of its tile one after another, so larger tiles
// would leave warps without work on short lists (whose sweeps are latency-bound)
// and leave a tail of whole tiles at the end of long ones; with about four tiles
// per warp the claims still balance, and T = 32 cuts the per-root scalar work
// 32-fold.  Roots differ in cost (one to several sweeps in each precision),
// so warps claim tiles one at a time instead of a fixed stride, which would leave
// a tail.  Within a merge the list alternates between the two ends of the
// spectrum and moves inward (entry q is root q / 2 from the bottom for even q,
// from the top for odd q), so the costly roots (narrow gaps, many sweeps, at the
// ends) are claimed first and the cheap middle roots form the tail.
__global__ void __launch_bounds__(128, 3) k_secular_warp(RootArgs a) {
  const uint32_t total = warp_list_total(a);
  const uint32_t per_warp = total / (4 * ((gridDim.x * blockDim.x) >> 5));
  const uint32_t T = per_warp >= 32 ? 32u : per_warp >= 16 ? 16u : per_warp >= 8 ? 8u
                   : per_warp >= 4 ? 4u : per_warp >= 2 ? 2u : 1u;
  const uint32_t tiles = (total + T - 1) / T;
  const int lane = threadIdx.x & 31;
  unsigned long long pairs = 0, sops = 0, pairs32 = 0;  // pairs, sops: warp-uniform
  unsigned blocks = 0, sweeps64 = 0, sweeps32 = 0, roots = 0;
  for (uint32_t t = claim_next_item(a.st); t < tiles; t = claim_next_item(a.st)) {
    const uint32_t r = t * T + uint32_t(lane);
    const bool valid = uint32_t(lane) < T && r < total;
    int rl = 0, g = 0;
    if (valid) g = warp_list_merge(a, r, &rl);
    const MState ms = valid ? a.ms[g] : MState{};
    const int q = rl - ms.base, lo = valid ? a.M[g].lo : 0, K = valid ? ms.K : 0;
    const int j = (q & 1) ? K - 1 - (q >> 1) : (q >> 1);
    WarpCoop co{&a, lane, lo, K, mp_blocks(K, a.mp_min_k)};
    const Copies32 cp{a.AD32 + lo, a.AZ32 + lo, K};
    int org = 0, n32 = 0;
    double tau = 0.0;
    bool ok = true;
    const int sweeps = secular_root_coop<32>(a.AD + lo, a.AZ + lo, K, j, ms.rho, ms.rhoinv, ms.zsq,
                                             valid, cp, co, &org, &tau, &ok, &n32);
    if (valid) {
      secular_store(a, lo, j, org, tau, sweeps, K, ok, true);
      sweeps64 += unsigned(sweeps);
      sweeps32 += unsigned(n32);
      pairs32 += (unsigned long long)n32 * unsigned(K);
      roots += 1;
    }
    pairs += co.pairs;
    blocks += co.blocks;
    sops += co.sops;
  }
  // per-lane tallies summed over the warp, one atomic per counter per warp
  sweeps64 = __reduce_add_sync(0xffffffffu, sweeps64);
  sweeps32 = __reduce_add_sync(0xffffffffu, sweeps32);
  roots = __reduce_add_sync(0xffffffffu, roots);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) pairs32 += __shfl_xor_sync(0xffffffffu, pairs32, o);
  if (lane == 0 && roots) {
    atomicAdd(&a.st->work[kWorkSecularPairs], pairs);
    if (blocks) atomicAdd(&a.st->work[kWorkSecularFarBlocks], (unsigned long long)blocks);
    if (sops) atomicAdd(&a.st->work[kWorkSecularSeriesOps], sops);
    atomicAdd(&a.st->work[kWorkSecularSweeps], (unsigned long long)sweeps64);
    atomicAdd(&a.st->work[kWorkSecular32Pairs], pairs32);
    atomicAdd(&a.st->work[kWorkSecular32Sweeps], (unsigned long long)sweeps32);
    atomicAdd(&a.st->work[kWorkRoots], (unsigned long long)roots);
  }
  claim_finish_block(a.st);
}

// Cooperative sweeps by groups of G lanes (small merges: plain sums over all K
// poles, no block expansion): the root of lane src, in src's group, lives in the
// merge at row lo of order K, broadcast within the group.
template <int G>
struct GroupCoop {
  const RootArgs* a;
  int gl, lo, K;
  unsigned gm;
  __device__ __forceinline__ Sec32 sweep32(int src, int org, int jl, float tau, float inv) const {
    const int slo = __shfl_sync(gm, lo, src), sK = __shfl_sync(gm, K, src);
    const GroupSweep32<G> sw{{a->AD32 + slo, a->AZ32 + slo, sK}, gl, gm};
    return sw(org, jl, tau, inv);
  }
  __device__ __forceinline__ SecSums sweep64(int src, double dorg, double tau, int jl) const {
    const int slo = __shfl_sync(gm, lo, src), sK = __shfl_sync(gm, K, src);
    const GroupSweep<G> sw{a->AD + slo, a->AZ + slo, sK, gl, gm};
    return sw(dorg, tau, jl);
  }
};

// The small-K list in tiles, one root per lane: warps claim tiles of T consecutive
// entries, every sweep is summed by a group of G lanes (G rounds per pass, see
// secular_root_coop), and the roots' scalar work (model steps, convergence tests,
// stage hand-over) runs lane-parallel for the whole tile instead of on every lane
// of a root's group.  Entry k of a tile sits in group k mod (32 / G), so a tile of
// 32 / G entries fills every group's first round; T is 32 where the list gives each
// warp at least two tiles of 32 / G, else 16, else 32 / G.  Same steps and sums as
// the warp-synchronous rounds of four-lane groups and as k_secular_small<G>, so the
// same roots bit for bit.  A forest sorts its list by K first, so a tile's roots have
// nearly equal K.
template <int G>
__global__ void __launch_bounds__(128) k_secular_lanes(RootArgs a) {
  const uint32_t total = *a.count;
  if (total < a.small_list_min) {  // the warp kernel takes a short list
    claim_finish_block(a.st);
    return;
  }
  constexpr uint32_t kGroups = 32 / G;
  const uint32_t per_warp = total / (4 * ((gridDim.x * blockDim.x) >> 5));
  const uint32_t T = per_warp >= 8 ? 32u : per_warp >= 4 ? 16u : kGroups;
  const uint32_t tiles = (total + T - 1) / T;
  const int lane = threadIdx.x & 31, gl = lane & (G - 1);
  const unsigned gm = ((1u << G) - 1u) << (lane & ~(G - 1));
  const uint32_t k = uint32_t(gl) * kGroups + uint32_t(lane / G);  // this lane's tile entry
  SecTally tally;
  for (uint32_t t = claim_next_item(a.st); t < tiles; t = claim_next_item(a.st)) {
    const uint32_t r = t * T + k;
    const bool valid = k < T && r < total;
    const int g = valid ? a.ROOTMAP[r] : 0;
    const MState ms = valid ? a.ms[g] : MState{};
    const int j = int(r) - ms.base, lo = valid ? a.M[g].lo : 0, K = valid ? ms.K : 0;
    GroupCoop<G> co{&a, gl, lo, K, gm};
    const Copies32 cp{a.AD32 + lo, a.AZ32 + lo, K};
    int org = 0, n32 = 0;
    double tau = 0.0;
    bool ok = true;
    const int sweeps = secular_root_coop<G>(a.AD + lo, a.AZ + lo, K, j, ms.rho, ms.rhoinv, ms.zsq,
                                            valid, cp, co, &org, &tau, &ok, &n32);
    if (valid) {
      secular_store(a, lo, j, org, tau, sweeps, K, ok, true);
      tally.add(sweeps, n32, K);
    }
  }
  tally.flush(a.st);
  claim_finish_block(a.st);
}

// ---------------------------------------------------------------------------
// z-hat of pole i from all K roots (appendix "WPROD product chains"):
//   zhat_i^2 = (lambda_K - D_i) / rho' * prod_{j<i} (lambda_j - D_i) / (D_j - D_i)
//              * prod_{i<=j<K-1} (lambda_j - D_i) / (D_{j+1} - D_i)
// (1-based K), every factor positive and below one by interlacing, so the partial
// products neither overflow nor underflow before the full product does.
// lambda_j - D_i = (D_org(j) - D_i) + tau_j keeps the near factors accurate.
//
// The factors are accumulated as two separate products (numerators and
// denominators, five FP64 operations per pair instead of a division) kept as a
// mantissa in [1, 2) and an integer binary exponent, renormalised every eight
// factors by integer operations on the exponent field.  Every factor lies in
// (1e-38, 16) (distinct poles and roots of a scaled matrix), so eight of them
// cannot leave the normal range.
struct MantExp {
  double m;
  int e;
};

__device__ __forceinline__ void me_renorm(MantExp& x) {
  const int hi = __double2hiint(x.m);
  const int ex = (hi >> 20) & 0x7ff;
  if (ex == 0 || ex == 0x7ff) return;  // zero, subnormal or non-finite: leave as is
  x.e += ex - 1023;
  x.m = __hiloint2double((hi & 0x800fffff) | (1023 << 20), __double2loint(x.m));
}

__device__ __forceinline__ void me_mul(MantExp& x, const MantExp& y) {
  x.m *= y.m;
  x.e += y.e;
  me_renorm(x);
}

// num / den as one double (the result is O(1) or below: it is a z-hat square).  A
// renormalised mantissa lies in [1, 2) (biased exponent 1023), where the refined
// reciprocal needs no range care; anything else takes a division.
__device__ __forceinline__ double me_ratio(const MantExp& num, const MantExp& den) {
  const bool unit = ((__double2hiint(den.m) >> 20) & 0x7ff) == 1023;
  return ldexp(unit ? num.m * rcp_refined(den.m) : num.m / den.m, num.e - den.e);
}

__device__ __forceinline__ void lowner_pair(const double* AD, const double* DORG, const double* TAU,
                                            int i, double Di, int j, double& num, double& den) {
  num *= (DORG[j] - Di) + TAU[j];
  den *= (j < i ? AD[j] : AD[j + 1]) - Di;
}

__device__ __forceinline__ void lowner_store(const RootArgs& a, int lo, int i, double Di, int K,
                                             double rhoinv, MantExp num, MantExp den,
                                             double slog = 0.0) {
  const double last = ((a.DORG[lo + K - 1] - Di) + a.TAU[lo + K - 1]) * rhoinv;
  const double z2 = me_ratio(num, den) * last * (slog != 0.0 ? exp(slog) : 1.0);
  a.ZHAT[lo + i] = copysign(sqrt(fmax(z2, 0.0)), a.AZ[lo + i]);
}

__global__ void k_lowner_thread(RootArgs a) {
  const uint32_t total = *a.count;
  if (total < a.small_list_min) return;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < total; r += gridDim.x * blockDim.x) {
    const int g = a.ROOTMAP[r];
    const Merge m = a.M[g];
    if ((uint32_t(m.info) & kRootBit) && !a.all_merges) continue;
    const MState ms = a.ms[g];
    const int K = ms.K, i = int(r) - ms.base, lo = m.lo;
    const double* AD = a.AD + lo;
    const double* DORG = a.DORG + lo;
    const double* TAU = a.TAU + lo;
    const double Di = AD[i];
    MantExp num{1.0, 0}, den{1.0, 0};
    int j = 0;
    for (; j + 8 <= K - 1; j += 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) lowner_pair(AD, DORG, TAU, i, Di, j + u, num.m, den.m);
      me_renorm(num);
      me_renorm(den);
    }
    for (; j < K - 1; ++j) lowner_pair(AD, DORG, TAU, i, Di, j, num.m, den.m);
    me_renorm(num);
    me_renorm(den);
    lowner_store(a, lo, i, Di, K, ms.rhoinv, num, den);
    work_add(a.st, kWorkLownerPairs, unsigned(K));
  }
}

// Block expansion of the Löwner products (merges with K >= mp_min_k).  In log form
// zhat_i^2 = (lambda_K - D_i) / rho' exp(sum_j log f_j), f_j = (lambda_j - D_i) /
// (P_j - D_i) with P_j = D_j for j < i and D_{j+1} for j >= i.  The K - 1 pairs
// are cut into the blocks of the secular expansion (pairs j in [128 b, 128 b +
// 128), the last block up to K - 1); block b spans [D_b0, D_b1] around its centre
// m with radius r.  For D_i far from it (r <= |D_i - m| / 3) its pairs sum to
//   sum_j log f_j = -w sum_{k>=0} c_k x^k,  w = 1 / (D_i - m),  x = r w,
//   c_k = G_{k+1} / ((k + 1) r^k),
//   G_k = sum_j (lambda_j - m)^k - (P_j - m)^k = sum_j a_j h_{k-1}(lambda_j - m, P_j - m),
// a_j = lambda_j - P_j and h the complete homogeneous sum, so G_k carries no
// cancellation and |c_k| <= sum_j |a_j|; the block lies wholly on one side of D_i,
// so P_j = D_j (left, set L) or D_{j+1} (right, set R) for all its pairs.  With 35
// terms (27 for rounds within 1/4, 14 within 1/16, 10 within 1/64) the dropped part
// is below 2^-53 of sum_j |a_j| / |D_i - m| <= 1 (absolute, in the log), and the far
// blocks' sum enters zhat^2 through one exp.  As in the secular sweep only the first
// 21 / 17 / 9 / 6 terms run in FP64 and the rest in float (error below 2^-55 of the
// same bound).
// Near blocks multiply their factors directly.
constexpr int kMlTerms = 35;   // far: radius <= 1/3 of the distance; 27 within 1/4, 14 within 1/16
constexpr int kMlSeriesOverhead = 4;  // FP64 operations besides the head: D_i - m, 1/., x, accumulation
constexpr int kMlHead = kHv3;  // FP64 coefficients stored per side
constexpr int kTailBase = kHv0;  // float copies start at this term (every tier's head reaches it)
constexpr int kMlFields = 3 + 2 * kMlHead;                // m, r, 3 r, c^L_k, c^R_k (k < 21)
constexpr int kMlFloats = 2 * (kMlTerms - kTailBase);     // c^L_k, c^R_k (6 <= k < 35) as floats
static_assert(2 * kMlFields + kMlFloats <= 2 * kMpBlock, "block data must fit the merge's rows");
// superblocks of pair blocks (same rule as the secular sums; data after the blocks')
static_assert((8 + 1) * (kMlFields + (kMlFloats + 1) / 2 + 1) <= 8 * kMpBlock,
              "block and superblock data fit the merge's rows");
__device__ __forceinline__ double* lowner_sb_data(double* MPR_lo, int nb) {
  return MPR_lo + kMlFields * nb + (kMlFloats * nb + 1) / 2;
}

// One series of N terms with an FP64 head of H terms (coefficients c[k * nb]) and
// a float tail (coefficients f[(k - kTailBase) * nb]), at x.
template <int N, int H>
__device__ __forceinline__ double series1_mixed(const double* c, const float* f, int nb, double x) {
  static_assert(H >= kTailBase && H < N, "head inside the series");
  const float xf = __double2float_rn(x);
  float tv = f[(N - 1 - kTailBase) * nb];
#pragma unroll
  for (int k = N - 2; k >= H; --k) tv = fmaf(tv, xf, f[(k - kTailBase) * nb]);
  double v = double(tv);
#pragma unroll
  for (int k = H - 1; k >= 0; --k) v = fma(v, x, c[k * nb]);
  return v;
}

__device__ __forceinline__ int lowner_block_end(int b, int nb, int K) {
  return b == nb - 1 ? K - 1 : (b + 1) * kMpBlock;
}

__global__ void __launch_bounds__(128) k_lowner_moments(RootArgs a) {
  const uint32_t total = warp_list_total(a);
  const int lane = threadIdx.x & 31;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t base = gw * 32; base < total; base += nw * 32) {
    const uint32_t r = base + lane;
    int g = 0, j = 0, nb = 0;
    bool head = false;
    if (r < total) {
      int rl;
      g = warp_list_merge(a, r, &rl);
      const Merge m = a.M[g];
      const MState ms = a.ms[g];
      j = rl - ms.base;
      nb = ((uint32_t(m.info) & kRootBit) && !a.all_merges) ? 0 : mp_blocks(ms.K, a.mp_min_k);
      head = nb > 0 && (j % kMpBlock) == 0 && j / kMpBlock < nb;
    }
    unsigned hm = __ballot_sync(0xffffffffu, head);
    while (hm) {
      const int src = __ffs(hm) - 1;
      hm &= hm - 1;
      const int gg = __shfl_sync(0xffffffffu, g, src), b = __shfl_sync(0xffffffffu, j, src) / kMpBlock;
      const int nbb = __shfl_sync(0xffffffffu, nb, src);
      const int lo = a.M[gg].lo, K = a.ms[gg].K;
      const double* D = a.AD + lo;
      const double* DORG = a.DORG + lo;
      const double* TAU = a.TAU + lo;
      const int j0 = b * kMpBlock, j1 = lowner_block_end(b, nbb, K);
      const double m = 0.5 * (D[j0] + D[j1]);
      const double rad = fmax(m - D[j0], D[j1] - m);
      const double rinv = rad > 0.0 ? 1.0 / rad : 0.0;
      double* MP = a.MPR + lo;
      float* MF = reinterpret_cast<float*>(MP + kMlFields * nbb);
      if (lane == 0) {
        MP[b] = m;
        MP[nbb + b] = rad;
        MP[2 * nbb + b] = 3.0 * rad;
      }
      for (int side = 0; side < 2; ++side) {  // L: partner D_j, R: partner D_{j+1}
        double gk[kMlTerms];  // G_{k+1} / r^k
#pragma unroll
        for (int k = 0; k < kMlTerms; ++k) gk[k] = 0.0;
        for (int jj = j0 + lane; jj < j1; jj += 32) {
          const double P = D[jj + side];
          const double u = ((DORG[jj] - m) + TAU[jj]) * rinv, v = (P - m) * rinv;
          const double aj = (DORG[jj] - P) + TAU[jj];
          double h = 1.0, vk = 1.0;
#pragma unroll
          for (int k = 0; k < kMlTerms; ++k) {  // G_{k+1} / r^k += a h_k(u, v)
            gk[k] = fma(aj, h, gk[k]);
            vk *= v;
            h = fma(u, h, vk);
          }
        }
        warp_sum_halving(gk, lane);
#pragma unroll
        for (int jj = 0; jj < warp_halved_len(kMlTerms); ++jj) {
          const int k = halving_index<kMlTerms>(lane, jj);
          if (k >= 0) {
            const double c = gk[jj] / double(k + 1);
            if (k < kMlHead) MP[(3 + side * kMlHead + k) * nbb + b] = c;
            if (k >= kTailBase)
              MF[(side * (kMlTerms - kTailBase) + k - kTailBase) * nbb + b] = __double2float_rn(c);
          }
        }
      }
    }
  }
}

// Superblock coefficients of the Löwner log sums from those of its pair blocks: with
// a = (m_b - m_S) / R and c = r_b / R, c^S_k = sum_b sum_{q<=k} C(k, q) a^(k-q) c^q c^b_q
// on each side (G_(k+1) translated to the new centre and rescaled; |a| + c <= 1).
__global__ void __launch_bounds__(64) k_lowner_super(RootArgs a) {  // 2 warps: L, R
  const uint32_t total = warp_list_total(a);
  const int lane = threadIdx.x & 31;
  const int side = threadIdx.x >> 5;  // the block's warps share the roots, one side each
  const uint32_t gw = blockIdx.x, nw = gridDim.x;
  for (uint32_t base = gw * 32; base < total; base += nw * 32) {
    const uint32_t r = base + lane;
    int g = 0, j = 0, nb = 0, nsb = 0;
    bool head = false;
    if (r < total) {
      int rl;
      g = warp_list_merge(a, r, &rl);
      const Merge mg = a.M[g];
      const MState ms = a.ms[g];
      j = rl - ms.base;
      nb = ((uint32_t(mg.info) & kRootBit) && !a.all_merges) ? 0 : mp_blocks(ms.K, a.mp_min_k);
      nsb = sb_count(nb);
      const int sbp = sb_size(nb) * kMpBlock;  // pairs per superblock
      head = nsb > 0 && (j % sbp) == 0 && j / sbp < nsb;
    }
    unsigned hm = __ballot_sync(0xffffffffu, head);
    while (hm) {
      const int src = __ffs(hm) - 1;
      hm &= hm - 1;
      const int gg = __shfl_sync(0xffffffffu, g, src);
      const int nbb = __shfl_sync(0xffffffffu, nb, src), nss = __shfl_sync(0xffffffffu, nsb, src);
      const int sbs = sb_size(nbb), sbp = sbs * kMpBlock;
      const int sb = __shfl_sync(0xffffffffu, j, src) / sbp;
      const int lo = a.M[gg].lo, K = a.ms[gg].K;
      const double* D = a.AD + lo;
      const int j0 = sb * sbp, j1 = (sb == nss - 1) ? K - 1 : j0 + sbp;
      const double m = 0.5 * (D[j0] + D[j1]);
      const double rad = fmax(m - D[j0], D[j1] - m);
      const double rinv = rad > 0.0 ? 1.0 / rad : 0.0;
      const double* MP = a.MPR + lo;
      const float* MF = reinterpret_cast<const float*>(MP + kMlFields * nbb);
      double* SP = lowner_sb_data(a.MPR + lo, nbb);
      float* SF = reinterpret_cast<float*>(SP + kMlFields * nss);
      const int b = sb * sbs + lane;
      const bool mine = b < nbb && lane < sbs;
      if (lane == 0 && side == 0) {
        SP[sb] = m;
        SP[nss + sb] = rad;
        SP[2 * nss + sb] = 3.0 * rad;
      }
      {
        double S[kMlTerms];
#pragma unroll
        for (int k = 0; k < kMlTerms; ++k) S[k] = 0.0;
        if (mine) {
          const double av = (MP[b] - m) * rinv, cv = MP[nbb + b] * rinv;
          double cq = 1.0;
#pragma unroll
          for (int q = 0; q < kMlTerms; ++q) {
            const double c = q < kMlHead ? MP[(3 + side * kMlHead + q) * nbb + b]
                                         : double(MF[(side * (kMlTerms - kTailBase) + q - kTailBase) * nbb + b]);
            S[q] = cq * c;
            cq *= cv;
          }
          binomial_shift(S, av);
        }
        warp_sum_halving(S, lane);
#pragma unroll
        for (int jj = 0; jj < warp_halved_len(kMlTerms); ++jj) {
          const int k = halving_index<kMlTerms>(lane, jj);
          if (k >= 0) {
            if (k < kMlHead) SP[(3 + side * kMlHead + k) * nss + sb] = S[jj];
            if (k >= kTailBase)
              SF[(side * (kMlTerms - kTailBase) + k - kTailBase) * nss + sb] = __double2float_rn(S[jj]);
          }
        }
      }
    }
  }
}

// A warp takes tiles of T consecutive poles (T = the poles per warp, at most 32;
// tile t goes to warp t mod the warp count): it forms each pole's products and
// far-block log sum cooperatively as before and leaves them in lane u (the pole's
// place in the tile), and the closing scalar work -- the ratio, exp of the log
// sum, the square root -- runs once per tile for all its poles instead of at warp
// width per pole.
__global__ void k_lowner_warp(RootArgs a) {
  const uint32_t total = warp_list_total(a);
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t per = (total + nwarps - 1) / nwarps;
  const uint32_t T = per >= 32 ? 32u : (per == 0 ? 1u : per);
  const uint32_t tiles = (total + T - 1) / T;
  unsigned pairs = 0, series = 0;
  unsigned long long sops = 0;
  for (uint32_t t = warp; t < tiles; t += nwarps) {
    // this lane's pole of the tile: its merge and sums, stored after the tile
    bool keep = false;
    int k_lo = 0, k_i = 0, k_K = 0;
    double k_Di = 0.0, k_rhoinv = 0.0, k_slog = 0.0;
    MantExp k_num{1.0, 0}, k_den{1.0, 0};
    const uint32_t r_end = min(total, (t + 1) * T);
    for (uint32_t r = t * T; r < r_end; ++r) {
      int rl;
      const int g = warp_list_merge(a, r, &rl);
      const Merge m = a.M[g];
      if ((uint32_t(m.info) & kRootBit) && !a.all_merges) continue;
      const MState ms = a.ms[g];
      const int K = ms.K, i = rl - ms.base, lo = m.lo;
      const double* AD = a.AD + lo;
      const double* DORG = a.DORG + lo;
      const double* TAU = a.TAU + lo;
      const double Di = AD[i];
      MantExp num{1.0, 0}, den{1.0, 0};
      double slog = 0.0;  // far blocks' log sum (block expansion)
      const int nb = mp_blocks(K, a.mp_min_k);
      if (nb == 0) {
        int j = lane;
        for (; j + 7 * 32 < K - 1; j += 8 * 32) {
#pragma unroll
          for (int u = 0; u < 8; ++u) lowner_pair(AD, DORG, TAU, i, Di, j + 32 * u, num.m, den.m);
          me_renorm(num);
          me_renorm(den);
        }
        for (; j < K - 1; j += 32) lowner_pair(AD, DORG, TAU, i, Di, j, num.m, den.m);
        me_renorm(num);
        me_renorm(den);
        pairs += unsigned(K);
      } else {
        const double* MP = a.MPR + lo;
        const float* MF = reinterpret_cast<const float*>(MP + kMlFields * nb);
        const int nsb = sb_count(nb);
        const double* SP = lowner_sb_data(a.MPR + lo, nb);
        const float* SF = reinterpret_cast<const float*>(SP + kMlFields * nsb);
        // one round: the lane's pair block (or superblock) b of data C / F with nc
        // entries per field through its log series if it is far from D_i
        auto far_round = [&](const double* C, const float* F, int nc, int b, bool valid) -> bool {
          const double dm = valid ? Di - C[b] : 1.0;
          const double rb = valid ? C[nc + b] : 0.0;
          const FarTest ft = far_test_bits(dm, rb, valid ? C[2 * nc + b] : 0.0, valid);
          if (ft.far) {
            const double w = rcp_refined(dm), x = rb * w;
            const int side = dm < 0.0 ? 1 : 0;  // right of D_i: R
            const double* c = C + (3 + side * kMlHead) * nc + b;
            const float* f = F + side * (kMlTerms - kTailBase) * nc + b;
            double val;
            if (ft.tier == 0)
              val = series1_mixed<kMpTiny, kHv0>(c, f, nc, x);
            else if (ft.tier == 1)
              val = series1_mixed<kMpShort, kHv1>(c, f, nc, x);
            else if (ft.tier == 2)
              val = series1_mixed<kMpMid, kHv2>(c, f, nc, x);
            else
              val = series1_mixed<kMlTerms, kHv3>(c, f, nc, x);
            slog = fma(-w, val, slog);
          }
          const unsigned nfar = __popc(__ballot_sync(0xffffffffu, ft.far));
          series += nfar;
          sops += nfar * unsigned(kMlSeriesOverhead + (ft.tier == 0   ? kHv0
                                                       : ft.tier == 1 ? kHv1
                                                       : ft.tier == 2 ? kHv2
                                                                      : kHv3));
          return ft.far;
        };
        unsigned sfar = 0;  // superblocks taken whole
        if (nsb > 0) sfar = __ballot_sync(0xffffffffu, far_round(SP, SF, nsb, lane, lane < nsb));
        const KeptBlocks kb = kept_blocks(nsb, sb_size(nb), sfar, nb);
        for (int base = 0; base < kb.count; base += 32) {
          const int b = kept_block(kb, base + lane);
          const bool far = far_round(MP, MF, nb, b < 0 ? 0 : b, b >= 0);
          unsigned nm = __ballot_sync(0xffffffffu, b >= 0 && !far);
          while (nm) {
            const int bb = __shfl_sync(0xffffffffu, b, __ffs(nm) - 1);
            nm &= nm - 1;
            const int j0 = bb * kMpBlock, j1 = lowner_block_end(bb, nb, K);
            for (int j = j0 + lane; j < j1; j += 32) lowner_pair(AD, DORG, TAU, i, Di, j, num.m, den.m);
            me_renorm(num);  // at most four factors per lane since the last renormalisation
            me_renorm(den);
            pairs += unsigned(j1 - j0);
          }
        }
        slog = warp_sum(slog);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        MantExp pn{__shfl_xor_sync(0xffffffffu, num.m, o), __shfl_xor_sync(0xffffffffu, num.e, o)};
        MantExp pd{__shfl_xor_sync(0xffffffffu, den.m, o), __shfl_xor_sync(0xffffffffu, den.e, o)};
        me_mul(num, pn);
        me_mul(den, pd);
      }
      if (uint32_t(lane) == r - t * T) {
        keep = true;
        k_lo = lo;
        k_i = i;
        k_K = K;
        k_Di = Di;
        k_rhoinv = ms.rhoinv;
        k_slog = slog;
        k_num = num;
        k_den = den;
      }
    }
    if (keep) lowner_store(a, k_lo, k_i, k_Di, k_K, k_rhoinv, k_num, k_den, k_slog);
  }
  if (lane == 0 && pairs) atomicAdd(&a.st->work[kWorkLownerPairs], (unsigned long long)pairs);
  if (lane == 0 && series) atomicAdd(&a.st->work[kWorkLownerFarBlocks], (unsigned long long)series);
  if (lane == 0 && sops) atomicAdd(&a.st->work[kWorkLownerSeriesOps], sops);
}

// ---------------------------------------------------------------------------
// Parent boundary rows of active column j (Sec. 4.1): with y_j(i) proportional to
// zhat_i / Delta_ij, R_parent(:, j) = R_child y_j / ||zhat / Delta_:j||.  Only the
// rows the merge's ancestors need are formed (kLeftSpineBit / kRightSpineBit;
// both when all_merges asks for every merge's full state): MODE 3 both rows,
// 1 the low row only, 2 the high row only -- 8 instead of 9 FP64 instructions
// per pair on the two spines of every tree.
__device__ __forceinline__ int rows_mode(const RootArgs& a, const Merge& m) {
  if (a.all_merges) return 3;
  const uint32_t f = uint32_t(m.info);
  return ((f & kLeftSpineBit) ? 0 : 1) | ((f & kRightSpineBit) ? 0 : 2);
}

template <int MODE>
__device__ __forceinline__ void rows_thread_sweep(const double* AD, const double* ZH, const double* AL,
                                                  const double* AH, int K, double dorg, double tau,
                                                  double& s2, double& sl, double& sh) {
  s2 = sl = sh = 0.0;
  for (int i = 0; i < K; ++i) {
    const double t = ZH[i] * rcp_refined((AD[i] - dorg) - tau);
    s2 = fma(t, t, s2);
    if (MODE & 1) sl = fma(AL[i], t, sl);
    if (MODE & 2) sh = fma(AH[i], t, sh);
  }
}

__global__ void k_rows_thread(RootArgs a) {
  const uint32_t total = *a.count;
  if (total < a.small_list_min) return;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < total; r += gridDim.x * blockDim.x) {
    const int g = a.ROOTMAP[r];
    const Merge m = a.M[g];
    if ((uint32_t(m.info) & kRootBit) && !a.all_merges) continue;
    const MState ms = a.ms[g];
    const int K = ms.K, j = int(r) - ms.base, lo = m.lo;
    const double* AD = a.AD + lo;
    const double* ZH = a.ZHAT + lo;
    const double* AL = a.ALO + lo;
    const double* AH = a.AHI + lo;
    const double dorg = a.DORG[lo + j];
    const double tau = a.TAU[lo + j];
    double s2, sl, sh;
    switch (rows_mode(a, m)) {
      case 1: rows_thread_sweep<1>(AD, ZH, AL, AH, K, dorg, tau, s2, sl, sh); break;
      case 2: rows_thread_sweep<2>(AD, ZH, AL, AH, K, dorg, tau, s2, sl, sh); break;
      default: rows_thread_sweep<3>(AD, ZH, AL, AH, K, dorg, tau, s2, sl, sh); break;
    }
    const double inv = 1.0 / sqrt(s2);
    if (a.RINU) a.RINU[lo + j] = inv;
    a.ROWLO[lo + j] = sl * inv;
    a.ROWHI[lo + j] = sh * inv;
    work_add(a.st, kWorkRowsPairs, unsigned(K));
  }
}

// lanes stride over the poles, two independent chains per lane
template <int MODE>
__device__ __forceinline__ void rows_warp_sweep(const double* AD, const double* ZH, const double* AL,
                                                const double* AH, int K, int lane, double dorg,
                                                double tau, double& s2o, double& slo, double& sho) {
  double s2 = 0.0, sl = 0.0, sh = 0.0, s2b = 0.0, slb = 0.0, shb = 0.0;
  int i = lane;
  for (; i + 32 < K; i += 64) {
    const double t0 = ZH[i] * rcp_refined((AD[i] - dorg) - tau);
    const double t1 = ZH[i + 32] * rcp_refined((AD[i + 32] - dorg) - tau);
    s2 = fma(t0, t0, s2);
    if (MODE & 1) sl = fma(AL[i], t0, sl);
    if (MODE & 2) sh = fma(AH[i], t0, sh);
    s2b = fma(t1, t1, s2b);
    if (MODE & 1) slb = fma(AL[i + 32], t1, slb);
    if (MODE & 2) shb = fma(AH[i + 32], t1, shb);
  }
  for (; i < K; i += 32) {
    const double t0 = ZH[i] * rcp_refined((AD[i] - dorg) - tau);
    s2 = fma(t0, t0, s2);
    if (MODE & 1) sl = fma(AL[i], t0, sl);
    if (MODE & 2) sh = fma(AH[i], t0, sh);
  }
  double a = s2 + s2b, l = (MODE & 1) ? sl + slb : 0.0, h = (MODE & 2) ? sh + shb : 0.0, u = 0.0;
  warp_sum4(a, l, h, u);
  s2o = a;
  slo = l;
  sho = h;
}

// Block expansion of the row sums (merges with K >= mp_min_k): with the blocks of
// the secular expansion, t = 1 / (m - lambda_j) and x = -r t, a block far from
// lambda_j (r <= |m - lambda_j| / 3) adds
//   t^2 sum_k (k + 1) A_k x^k  to  sum zhat_i^2 / Delta_ij^2,   A_k = sum zhat^2 y^k,
//   t   sum_k L_k x^k          to  sum ALO_i zhat_i / Delta_ij,  L_k = sum zhat ALO y^k,
//   t   sum_k H_k x^k          to  sum AHI_i zhat_i / Delta_ij,  H_k = sum zhat AHI y^k,
// y = (D_i - m) / r, with 40 terms (32 for rounds within 1/4 of their distance, 16
// within 1/16, 10 within 1/64): the dropped part stays below 2^-55 of the sum of the
// block's |terms| for the squared kernel and below 2^-60 for the others.  The first
// 24 / 19 / 9 / 6 terms of the squared kernel and 21 / 17 / 9 / 6 of the others run
// in FP64, the rest in float: the float part's error, about 3 (k + 1) 2^-24 |x|^k from the head's
// end k on, stays below 2^-55 of the same sums.
constexpr int kMrTerms = 40;  // far: radius <= 1/3 of the distance
constexpr int kMrMid = 32;    // radius <= 1/4
constexpr int kMrShort = 16;  // radius <= 1/16 of the distance: 17 x 16^-16 < 2^-59
constexpr int kMrTiny = 10;   // radius <= 1/64 of the distance: 11 x 64^-10 < 2^-56
constexpr int kMrHa0 = 6, kMrHa1 = 9, kMrHa2 = 19, kMrHa3 = 24;  // FP64 heads of the squared kernel
constexpr int kMrHl0 = kHv0, kMrHl1 = kHv1, kMrHl2 = kHv2, kMrHl3 = kHv3;  // and of the two rows
constexpr int kMrFields = 3 + kMrHa3 + 2 * kMrHl3;  // m, r, 3 r, (k + 1) A_k, L_k, H_k (heads)
constexpr int kMrTail = kMrTerms - kTailBase;       // float terms per kernel (6 <= k < 40)
static_assert(2 * kMrFields + 3 * kMrTail <= 2 * kMpBlock, "block data must fit the merge's rows");
// superblocks (same rule as the secular sums; data after the blocks')
static_assert((kSbRows + 1) * (kMrFields + (3 * kMrTail + 1) / 2 + 1) <= kSbRows * kMpBlock,
              "block and superblock data fit the merge's rows");
__device__ __forceinline__ double* rows_sb_data(double* MPR_lo, int nb) {
  return MPR_lo + kMrFields * nb + (3 * kMrTail * nb + 1) / 2;
}

// Moments of the row sums, one warp per block (found as in k_block_moments).
__global__ void __launch_bounds__(128) k_rows_moments(RootArgs a) {
  const uint32_t total = warp_list_total(a);
  const int lane = threadIdx.x & 31;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t base = gw * 32; base < total; base += nw * 32) {
    const uint32_t r = base + lane;
    int g = 0, j = 0, nb = 0;
    bool head = false;
    if (r < total) {
      int rl;
      g = warp_list_merge(a, r, &rl);
      const Merge m = a.M[g];
      const MState ms = a.ms[g];
      j = rl - ms.base;
      nb = ((uint32_t(m.info) & kRootBit) && !a.all_merges) ? 0 : mp_blocks(ms.K, a.mp_min_k);
      head = nb > 0 && (j % kMpBlock) == 0 && j / kMpBlock < nb;
    }
    unsigned hm = __ballot_sync(0xffffffffu, head);
    while (hm) {
      const int src = __ffs(hm) - 1;
      hm &= hm - 1;
      const int gg = __shfl_sync(0xffffffffu, g, src), b = __shfl_sync(0xffffffffu, j, src) / kMpBlock;
      const int nbb = __shfl_sync(0xffffffffu, nb, src);
      const int lo = a.M[gg].lo, K = a.ms[gg].K;
      const double* D = a.AD + lo;
      const double* ZH = a.ZHAT + lo;
      const int i0 = b * kMpBlock, i1 = (b == nbb - 1) ? K : i0 + kMpBlock;
      const double m = 0.5 * (D[i0] + D[i1 - 1]);
      const double rad = fmax(m - D[i0], D[i1 - 1] - m);
      const double rinv = rad > 0.0 ? 1.0 / rad : 0.0;
      double* MP = a.MPR + lo;
      float* MF = reinterpret_cast<float*>(MP + kMrFields * nbb);
      if (lane == 0) {
        MP[b] = m;
        MP[nbb + b] = rad;
        MP[2 * nbb + b] = 3.0 * rad;
      }
      for (int which = 0; which < 3; ++which) {  // zhat^2 (stored times k + 1), zhat ALO, zhat AHI
        const double* W = which == 1 ? a.ALO + lo : a.AHI + lo;
        double mo[kMrTerms];
#pragma unroll
        for (int k = 0; k < kMrTerms; ++k) mo[k] = 0.0;
        for (int i = i0 + lane; i < i1; i += 32) {
          const double y = (D[i] - m) * rinv;
          double pw = ZH[i] * (which == 0 ? ZH[i] : W[i]);
#pragma unroll
          for (int k = 0; k < kMrTerms; ++k) {
            mo[k] += pw;
            pw *= y;
          }
        }
        const int head = which == 0 ? kMrHa3 : kMrHl3;
        const int off = which == 0 ? 0 : kMrHa3 + (which - 1) * kMrHl3;
        warp_sum_halving(mo, lane);
#pragma unroll
        for (int jj = 0; jj < warp_halved_len(kMrTerms); ++jj) {
          const int k = halving_index<kMrTerms>(lane, jj);
          if (k >= 0) {
            const double v = which == 0 ? double(k + 1) * mo[jj] : mo[jj];
            if (k < head) MP[(3 + off + k) * nbb + b] = v;
            if (k >= kTailBase) MF[(which * kMrTail + k - kTailBase) * nbb + b] = __double2float_rn(v);
          }
        }
      }
    }
  }
}

// Superblock moments of the row sums from the blocks' (binomial translation of
// A'_k, L'_k, H'_k as for the secular moments; A is stored times k + 1).
__global__ void __launch_bounds__(96) k_rows_super(RootArgs a) {  // 3 warps: A, L, H
  const uint32_t total = warp_list_total(a);
  const int lane = threadIdx.x & 31;
  const int which = threadIdx.x >> 5;  // the block's warps share the roots, one weight each
  const uint32_t gw = blockIdx.x, nw = gridDim.x;
  constexpr int kSbPoles = kSbRows * kMpBlock;
  for (uint32_t base = gw * 32; base < total; base += nw * 32) {
    const uint32_t r = base + lane;
    int g = 0, j = 0, nb = 0, nsb = 0;
    bool head = false;
    if (r < total) {
      int rl;
      g = warp_list_merge(a, r, &rl);
      const Merge mg = a.M[g];
      const MState ms = a.ms[g];
      j = rl - ms.base;
      nb = ((uint32_t(mg.info) & kRootBit) && !a.all_merges) ? 0 : mp_blocks(ms.K, a.mp_min_k);
      nsb = sb_count_rows(nb);
      head = nsb > 0 && (j % kSbPoles) == 0 && j / kSbPoles < nsb;
    }
    unsigned hm = __ballot_sync(0xffffffffu, head);
    while (hm) {
      const int src = __ffs(hm) - 1;
      hm &= hm - 1;
      const int gg = __shfl_sync(0xffffffffu, g, src);
      const int sb = __shfl_sync(0xffffffffu, j, src) / kSbPoles;
      const int nbb = __shfl_sync(0xffffffffu, nb, src), nss = __shfl_sync(0xffffffffu, nsb, src);
      const int lo = a.M[gg].lo, K = a.ms[gg].K;
      const double* D = a.AD + lo;
      const int i0 = sb * kSbPoles, i1 = (sb == nss - 1) ? K : i0 + kSbPoles;
      const double m = 0.5 * (D[i0] + D[i1 - 1]);
      const double rad = fmax(m - D[i0], D[i1 - 1] - m);
      const double rinv = rad > 0.0 ? 1.0 / rad : 0.0;
      const double* MP = a.MPR + lo;
      const float* MF = reinterpret_cast<const float*>(MP + kMrFields * nbb);
      double* SP = rows_sb_data(a.MPR + lo, nbb);
      float* SF = reinterpret_cast<float*>(SP + kMrFields * nss);
      const int b = sb * kSbRows + lane;
      const bool mine = b < nbb && lane < kSbRows;
      if (lane == 0 && which == 0) {
        SP[sb] = m;
        SP[nss + sb] = rad;
        SP[2 * nss + sb] = 3.0 * rad;
      }
      {  // A (stored times k + 1), L, H
        const int head = which == 0 ? kMrHa3 : kMrHl3;
        const int off = which == 0 ? 0 : kMrHa3 + (which - 1) * kMrHl3;
        double S[kMrTerms];
#pragma unroll
        for (int k = 0; k < kMrTerms; ++k) S[k] = 0.0;
        if (mine) {
          const double av = (MP[b] - m) * rinv, cv = MP[nbb + b] * rinv;
          double cq = 1.0;
#pragma unroll
          for (int q = 0; q < kMrTerms; ++q) {
            double c = q < head ? MP[(3 + off + q) * nbb + b]
                                : double(MF[(which * kMrTail + q - kTailBase) * nbb + b]);
            if (which == 0) c *= 1.0 / double(q + 1);
            S[q] = cq * c;
            cq *= cv;
          }
          binomial_shift(S, av);
        }
        warp_sum_halving(S, lane);
#pragma unroll
        for (int jj = 0; jj < warp_halved_len(kMrTerms); ++jj) {
          const int k = halving_index<kMrTerms>(lane, jj);
          if (k >= 0) {
            const double v = which == 0 ? double(k + 1) * S[jj] : S[jj];
            if (k < head) SP[(3 + off + k) * nss + sb] = v;
            if (k >= kTailBase) SF[(which * kMrTail + k - kTailBase) * nss + sb] = __double2float_rn(v);
          }
        }
      }
    }
  }
}

// The row sums' series of one far block at x: N terms, FP64 heads HA (squared
// kernel) and HL (row kernels), float tails.
template <int MODE, int N, int HA, int HL>
__device__ __forceinline__ void rows_mixed(const double* __restrict__ MP,
                                           const float* __restrict__ MF, int nb, int b, double x,
                                           double& va, double& vl, double& vh) {
  static_assert(HL <= HA && HL >= kTailBase && HA < N, "heads inside the series");
  const double* CA = MP + 3 * nb + b;
  const double* CL = MP + (3 + kMrHa3) * nb + b;
  const double* CH = MP + (3 + kMrHa3 + kMrHl3) * nb + b;
  const float* FA = MF + b;
  const float* FL = MF + kMrTail * nb + b;
  const float* FH = MF + 2 * kMrTail * nb + b;
  const float xf = __double2float_rn(x);
  float ta = FA[(N - 1 - kTailBase) * nb], tl = 0.f, th = 0.f;
  if (MODE & 1) tl = FL[(N - 1 - kTailBase) * nb];
  if (MODE & 2) th = FH[(N - 1 - kTailBase) * nb];
#pragma unroll
  for (int k = N - 2; k >= HL; --k) {
    if (k >= HA) ta = fmaf(ta, xf, FA[(k - kTailBase) * nb]);
    if (MODE & 1) tl = fmaf(tl, xf, FL[(k - kTailBase) * nb]);
    if (MODE & 2) th = fmaf(th, xf, FH[(k - kTailBase) * nb]);
  }
  double a = double(ta), l = double(tl), h = double(th);
#pragma unroll
  for (int k = HA - 1; k >= 0; --k) {
    a = fma(a, x, CA[k * nb]);
    if (k < HL) {
      if (MODE & 1) l = fma(l, x, CL[k * nb]);
      if (MODE & 2) h = fma(h, x, CH[k * nb]);
    }
  }
  va = a;
  vl = l;
  vh = h;
}

// Row sums of one root with the block expansion (all 32 lanes): far blocks one per
// lane through their series, near blocks term by term by the whole warp.
template <int MODE>
__device__ __forceinline__ void rows_warp_sweep_blocks(const double* AD, const double* ZH,
                                                       const double* AL, const double* AH, int K,
                                                       int nb, const double* __restrict__ MP,
                                                       int lane, double dorg, double tau,
                                                       double& s2o, double& slo, double& sho,
                                                       unsigned& exact, unsigned& series,
                                                       unsigned long long& sops) {
  const float* MF = reinterpret_cast<const float*>(MP + kMrFields * nb);
  const int nsb = sb_count_rows(nb);
  const double* SP = rows_sb_data(const_cast<double*>(MP), nb);
  const float* SF = reinterpret_cast<const float*>(SP + kMrFields * nsb);
  double s2 = 0.0, sl = 0.0, sh = 0.0;
  unsigned sfar = 0;  // superblocks taken whole (their rounds are skipped below)
  if (nsb > 0) {
    const int sb = lane;
    const double dm = sb < nsb ? (SP[sb] - dorg) - tau : 1.0;
    const double rb = sb < nsb ? SP[nsb + sb] : 0.0;
    const FarTest ft = far_test_bits(dm, rb, sb < nsb ? SP[2 * nsb + sb] : 0.0, sb < nsb);
    if (ft.far) {
      const double t = rcp_refined(dm), x = -rb * t;
      double va, vl = 0.0, vh = 0.0;
      if (ft.tier == 0)
        rows_mixed<MODE, kMrTiny, kMrHa0, kMrHl0>(SP, SF, nsb, sb, x, va, vl, vh);
      else if (ft.tier == 1)
        rows_mixed<MODE, kMrShort, kMrHa1, kMrHl1>(SP, SF, nsb, sb, x, va, vl, vh);
      else if (ft.tier == 2)
        rows_mixed<MODE, kMrMid, kMrHa2, kMrHl2>(SP, SF, nsb, sb, x, va, vl, vh);
      else
        rows_mixed<MODE, kMrTerms, kMrHa3, kMrHl3>(SP, SF, nsb, sb, x, va, vl, vh);
      s2 = fma(t * t, va, s2);
      if (MODE & 1) sl = fma(t, vl, sl);
      if (MODE & 2) sh = fma(t, vh, sh);
    }
    sfar = __ballot_sync(0xffffffffu, ft.far);
    const unsigned nfar = __popc(sfar), chains = MODE == 3 ? 3u : 2u;
    series += nfar * chains;
    const unsigned ha = ft.tier == 0 ? kMrHa0 : ft.tier == 1 ? kMrHa1 : ft.tier == 2 ? kMrHa2 : kMrHa3;
    const unsigned hl = ft.tier == 0 ? kMrHl0 : ft.tier == 1 ? kMrHl1 : ft.tier == 2 ? kMrHl2 : kMrHl3;
    sops += nfar * (ha + (chains - 1) * hl + 5 + chains);
  }
  for (int b0 = 0; b0 < nb; b0 += 32) {
    if ((sfar >> (b0 / kSbRows)) & 1u) continue;  // the round went through its superblock
    const int b = b0 + lane;
    bool near = false;
    const double dm = b < nb ? (MP[b] - dorg) - tau : 1.0;  // m - lambda
    const double rb = b < nb ? MP[nb + b] : 0.0;
    const FarTest ft = far_test_bits(dm, rb, b < nb ? MP[2 * nb + b] : 0.0, b < nb);
    if (b < nb) {
      if (ft.far) {
        const double t = rcp_refined(dm), x = -rb * t;
        double va, vl = 0.0, vh = 0.0;
        if (ft.tier == 0)
          rows_mixed<MODE, kMrTiny, kMrHa0, kMrHl0>(MP, MF, nb, b, x, va, vl, vh);
        else if (ft.tier == 1)
          rows_mixed<MODE, kMrShort, kMrHa1, kMrHl1>(MP, MF, nb, b, x, va, vl, vh);
        else if (ft.tier == 2)
          rows_mixed<MODE, kMrMid, kMrHa2, kMrHl2>(MP, MF, nb, b, x, va, vl, vh);
        else
          rows_mixed<MODE, kMrTerms, kMrHa3, kMrHl3>(MP, MF, nb, b, x, va, vl, vh);
        s2 = fma(t * t, va, s2);
        if (MODE & 1) sl = fma(t, vl, sl);
        if (MODE & 2) sh = fma(t, vh, sh);
      } else {
        near = true;
      }
    }
    unsigned nm = __ballot_sync(0xffffffffu, near);
    const unsigned nfar = unsigned(min(32, nb - b0) - __popc(nm)), chains = MODE == 3 ? 3u : 2u;
    series += nfar * chains;
    const unsigned ha = ft.tier == 0 ? kMrHa0 : ft.tier == 1 ? kMrHa1 : ft.tier == 2 ? kMrHa2 : kMrHa3;
    const unsigned hl = ft.tier == 0 ? kMrHl0 : ft.tier == 1 ? kMrHl1 : ft.tier == 2 ? kMrHl2 : kMrHl3;
    // heads, then m - lambda 2, reciprocal 1, x 1, t^2 1 and one accumulation per chain
    sops += nfar * (ha + (chains - 1) * hl + 5 + chains);
    while (nm) {
      const int bb = b0 + __ffs(nm) - 1;
      nm &= nm - 1;
      const int i0 = bb * kMpBlock, i1 = (bb == nb - 1) ? K : i0 + kMpBlock;
      for (int i = i0 + lane; i < i1; i += 32) {
        const double t0 = ZH[i] * rcp_refined((AD[i] - dorg) - tau);
        s2 = fma(t0, t0, s2);
        if (MODE & 1) sl = fma(AL[i], t0, sl);
        if (MODE & 2) sh = fma(AH[i], t0, sh);
      }
      exact += unsigned(i1 - i0);
    }
  }
  double l = (MODE & 1) ? sl : 0.0, h = (MODE & 2) ? sh : 0.0, u = 0.0;
  warp_sum4(s2, l, h, u);
  s2o = s2;
  slo = l;
  sho = h;
}

__global__ void k_rows_warp(RootArgs a) {
  const uint32_t total = warp_list_total(a);
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned pairs = 0, series = 0;
  unsigned long long sops = 0;
  for (uint32_t r = warp; r < total; r += nwarps) {
    int rl;
    const int g = warp_list_merge(a, r, &rl);
    const Merge m = a.M[g];
    if ((uint32_t(m.info) & kRootBit) && !a.all_merges) continue;
    const MState ms = a.ms[g];
    const int K = ms.K, j = rl - ms.base, lo = m.lo;
    const double* AD = a.AD + lo;
    const double* ZH = a.ZHAT + lo;
    const double* AL = a.ALO + lo;
    const double* AH = a.AHI + lo;
    const double dorg = a.DORG[lo + j];
    const double tau = a.TAU[lo + j];
    double s2, sl, sh;
    const int nb = mp_blocks(K, a.mp_min_k);
    if (nb > 0) {
      const double* MP = a.MPR + lo;
      switch (rows_mode(a, m)) {
        case 1: rows_warp_sweep_blocks<1>(AD, ZH, AL, AH, K, nb, MP, lane, dorg, tau, s2, sl, sh, pairs, series, sops); break;
        case 2: rows_warp_sweep_blocks<2>(AD, ZH, AL, AH, K, nb, MP, lane, dorg, tau, s2, sl, sh, pairs, series, sops); break;
        default: rows_warp_sweep_blocks<3>(AD, ZH, AL, AH, K, nb, MP, lane, dorg, tau, s2, sl, sh, pairs, series, sops); break;
      }
    } else {
      switch (rows_mode(a, m)) {
        case 1: rows_warp_sweep<1>(AD, ZH, AL, AH, K, lane, dorg, tau, s2, sl, sh); break;
        case 2: rows_warp_sweep<2>(AD, ZH, AL, AH, K, lane, dorg, tau, s2, sl, sh); break;
        default: rows_warp_sweep<3>(AD, ZH, AL, AH, K, lane, dorg, tau, s2, sl, sh); break;
      }
      pairs += unsigned(K);
    }
    if (lane == 0) {
      const double inv = (s2 > 0.0 && s2 < 0x1p1000) ? rsqrt_refined(s2) : 1.0 / sqrt(s2);
      if (a.RINU) a.RINU[lo + j] = inv;
      a.ROWLO[lo + j] = sl * inv;
      a.ROWHI[lo + j] = sh * inv;
    }
  }
  if (lane == 0 && pairs) atomicAdd(&a.st->work[kWorkRowsPairs], (unsigned long long)pairs);
  if (lane == 0 && series) atomicAdd(&a.st->work[kWorkRowsFarSeries], (unsigned long long)series);
  if (lane == 0 && sops) atomicAdd(&a.st->work[kWorkRowsSeriesOps], sops);
}

// Restores the saved roots of one step: tau, D_org and lambda = D_org + tau (the
// same expression the secular kernels store) at the active rows of every merge.
__global__ void k_restore_roots(const Merge* __restrict__ M, int64_t cnt, int64_t nrows,
                                const MState* __restrict__ ms, RootsCheckpoint ck, double* TAU,
                                double* DORG, double* LAMA) {
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < nrows;
       p += int64_t(gridDim.x) * blockDim.x) {
    const int64_t g = find_merge(M, cnt, p);
    const Merge m = M[g];
    if (p < m.lo || p >= m.hi || p - m.lo >= ms[g].K) continue;
    const double tau = ck.tau[p], dorg = ck.dorg[p];
    TAU[p] = tau;
    DORG[p] = dorg;
    LAMA[p] = dorg + tau;
  }
}

int launch_roots(const Plan& plan, const Workspace& ws, int step, const Merge* M, cudaStream_t s,
                 bool all_merges, double* rows_inu, const RootsCheckpoint* roots) {
  RootArgs ra;
  ra.RINU = rows_inu;
  ra.M = M;
  ra.ms = ws.mstate;
  ra.ROOTMAP = ws.ROOTMAP;
  ra.ROOTMAP2 = ws.ROOTMAP2;
  ra.count = &ws.status->root_count[step];
  ra.count2 = &ws.status->root_count_big[step];
  ra.AD = ws.AD;
  ra.AZ = ws.AZ;
  ra.ALO = ws.ALO;
  ra.AHI = ws.AHI;
  ra.AD32 = reinterpret_cast<const float2*>(ws.KEYB);
  ra.AZ32 = reinterpret_cast<const float*>(ws.IDXB);
  ra.MPD = ws.Z;
  ra.MPR = reinterpret_cast<double*>(ws.KEYB);
  ra.mp_min_k = plan.tune.multipole_min_k;
  ra.TAU = ws.TAU;
  ra.ORG = ws.ORG;
  ra.LAMA = ws.D;
  ra.ZHAT = ws.Z;
  ra.ROWLO = ws.RLO;
  ra.ROWHI = ws.RHI;
  ra.DORG = reinterpret_cast<double*>(ws.KEYA);
  ra.st = ws.status;
  ra.small_list_min = uint32_t(plan.tune.small_list_min);
  ra.all_merges = all_merges ? 1 : 0;
  // The thread kernels cover the small-K list when it is long enough to fill the
  // GPU; the warp kernels cover the large-K list and a short small-K list.  Which
  // case applies is known only on the device, so both always launch.
  const int64_t nrows = plan.nrows;
  const int tgrid = int(std::min<int64_t>((nrows + 127) / 128, 148 * 8));
  const int wgrid = 148 * 8;
  // lanes per root for the small-K list, from the largest merge order of the step
  const int64_t k0 = plan.step_maxsize[step];
  const int G = k0 <= 24 ? 1 : 4;
  int launches = 2;
  prof_begin(kKSecular, s);
  if (roots) {
    const int fgrid = int(std::min<int64_t>((nrows + 255) / 256, 148 * 8));
    k_restore_roots<<<fgrid, 256, 0, s>>>(M, plan.step_count[step], nrows, ws.mstate, *roots, ws.TAU,
                                          reinterpret_cast<double*>(ws.KEYA), ws.D);
    launches = 1;
  } else {
  if (plan.step_maxsize[step] >= ra.mp_min_k) {
    k_block_moments<<<int(std::min<int64_t>((nrows + 127) / 128, 148 * 8)), 128, 0, s>>>(ra);
    ++launches;
    if (plan.step_maxsize[step] >= int64_t(kSbMin) * kMpBlock) {  // superblocks possible
      k_super_moments<<<int(std::min<int64_t>((nrows + 127) / 128, 148 * 8)), 128, 0, s>>>(ra);
      ++launches;
    }
  }
  // The small-K list: four-lane roots in tiles of one root per lane with four-lane
  // sweeps, whose scalar steps run once per root instead of on all four lanes of its
  // group (4096 Lanczos-style tridiagonals: 192 -> 168.5 ms per solve, where the list
  // is also sorted by K; n = 65536, four families: 35.98 -> 35.80 ms over the
  // solver's stages, unsorted, since the two ordering launches per step cost a
  // single matrix more than they gain).  Steps of merges of at most 24 rows take one
  // thread per root: the refill kernel in a forest, warp-synchronous rounds in a
  // single matrix.  All of them give the same roots bit for bit.
  if (G == 4)
    k_secular_lanes<4><<<148 * 4, 128, 0, s>>>(ra);  // four blocks of 128 threads per SM
  else if (plan.batch > 1)
    k_secular_small<1><<<148 * 4, 128, 0, s>>>(ra);
  else
    k_secular_thread<<<tgrid, 128, 0, s>>>(ra);
  // three resident blocks per SM (168 registers per thread); each warp claims tiles
  k_secular_warp<<<148 * 3, 128, 0, s>>>(ra);
  }
  prof_end(kKSecular, s);
  if (plan.step_has_nonroot[step] || all_merges) {
    prof_begin(kKLowner, s);
    if (plan.step_maxsize[step] >= ra.mp_min_k) {
      k_lowner_moments<<<int(std::min<int64_t>((nrows + 127) / 128, 148 * 8)), 128, 0, s>>>(ra);
      ++launches;
      if (plan.step_maxsize[step] >= int64_t(kSbMin) * kMpBlock) {
        k_lowner_super<<<int(std::min<int64_t>((nrows + 31) / 32, 148 * 32)), 64, 0, s>>>(ra);
        ++launches;
      }
    }
    k_lowner_thread<<<tgrid, 128, 0, s>>>(ra);
    k_lowner_warp<<<wgrid, 128, 0, s>>>(ra);
    prof_end(kKLowner, s);
    prof_begin(kKRows, s);
    if (plan.step_maxsize[step] >= ra.mp_min_k) {
      k_rows_moments<<<int(std::min<int64_t>((nrows + 127) / 128, 148 * 8)), 128, 0, s>>>(ra);
      ++launches;
      if (plan.step_maxsize[step] >= int64_t(kSbRowsMin) * kMpBlock) {
        k_rows_super<<<int(std::min<int64_t>((nrows + 31) / 32, 148 * 32)), 96, 0, s>>>(ra);
        ++launches;
      }
    }
    k_rows_thread<<<tgrid, 128, 0, s>>>(ra);
    k_rows_warp<<<wgrid, 128, 0, s>>>(ra);
    prof_end(kKRows, s);
    launches += 4;
  }
  return launches;
}

__global__ void k_check_reciprocal(int64_t n, const double* __restrict__ x, double* out) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    out[i] = rcp_refined(x[i]);
}

__global__ void k_check_rsqrt(int64_t n, const double* __restrict__ x, double* out) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    out[i] = rsqrt_refined(x[i]);
}

}  // namespace tde

extern "C" int tde_check_rsqrt(int64_t n, const double* x, double* out, void* stream) {
  using namespace tde;
  if (n < 0 || (n > 0 && (x == nullptr || out == nullptr))) return TDE_EINVAL;
  if (n == 0) return TDE_OK;
  const int grid = int(std::min<int64_t>((n + 255) / 256, 148 * 8));
  k_check_rsqrt<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(n, x, out);
  return cudaGetLastError() == cudaSuccess ? TDE_OK : TDE_ECUDA;
}

extern "C" int tde_check_reciprocal(int64_t n, const double* x, double* out, void* stream) {
  using namespace tde;
  if (n < 0 || (n > 0 && (x == nullptr || out == nullptr))) return TDE_EINVAL;
  if (n == 0) return TDE_OK;
  const int grid = int(std::min<int64_t>((n + 255) / 256, 148 * 8));
  k_check_reciprocal<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(n, x, out);
  return cudaGetLastError() == cudaSuccess ? TDE_OK : TDE_ECUDA;
}
