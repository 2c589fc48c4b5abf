// Dense symmetric front end: A = Q T Q^T by Householder reflections, then the
// eigenvalues of T by the boundary-row solver (the dense EVD pipeline of Sec. 2:
// reduce to tridiagonal form, then solve the tridiagonal problem; the
// "reduced dense" workload of Sec. 5).  Eigenvalues only: Q is not kept.
//
// Column j (0-based, lower triangle, column-major with leading dimension n):
//   x = A[j+1:, j];  H_j = I - tau v v^T with v[0] = 1 maps x to (beta, 0, ..., 0)
//   e_j = beta,  d_j = A[j, j]
//   y = A22 v  (A22 = A[j+1:, j+1:]),  w = tau y - (tau^2 / 2)(y^T v) v
//   A22 <- A22 - v w^T - w v^T.
// On this part an FP64 fused multiply-add costs about as much time as 13 bytes of
// HBM traffic, so even this unblocked (matrix-vector) form is bound by the FP64
// pipe rather than by memory, and the two passes of a column are fused instead of
// blocked: one sweep over the trailing lower triangle applies column j's rank-2
// update and accumulates column j+1's product y (four FMAs per stored element,
// one read and one write).  Column j+1 itself is updated beforehand by a
// single-block kernel that also builds its reflector.
#include <algorithm>

#include "tde_internal.cuh"

namespace tde {

constexpr int kDenseTile = 64;  // rows x columns of one tile of the fused sweep
constexpr int kColThreads = 1024;

struct DenseArgs {
  double* A;   // n x n, column-major, lower triangle used
  int64_t n;
  double* V;   // two reflector vectors (ping-pong), n each
  double* W;   // two update vectors w, n each
  double* Y;   // two products y, n each
  double* tau; // [2]
  double* P;   // per tile of the sweep: 64 row partial sums, then 64 column partial sums
  double* d;   // [n]
  double* e;   // [n]
  unsigned* done;  // blocks of the current k_dense_reduce launch that have finished
};

__device__ __forceinline__ double block_reduce_sum(double v, double* sm) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sm[threadIdx.x] : 0.0;
  if (warp == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sm[0] = v;
  }
  __syncthreads();
  const double r = sm[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ double block_reduce_max(double v, double* sm) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sm[threadIdx.x] : 0.0;
  if (warp == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) sm[0] = v;
  }
  __syncthreads();
  const double r = sm[0];
  __syncthreads();
  return r;
}

// Column step j (one block, any multiple of 32 threads): finish column j-1's update
// vector w from its product y, apply column j-1's rank-2 update to column j, store
// d_j, build column j's reflector (v, tau, e_j).  Buffers of column j use slot
// j & 1.  Three passes over the column: y.v; then w, the column update and the sums
// for the norm of the new subdiagonal part (v_{j-1}[0] = 1, so w[0] is known to every
// thread after the first pass); then v.  The reflector's scalars (a hypot and two
// divisions) are formed by one thread and broadcast: issued by every warp they
// would cost the FP64 unit once per warp.  y is read past L1 (__ldcg): when the
// step runs in the last block of k_dense_reduce, other blocks of that launch wrote it.
__device__ void column_step(const DenseArgs& a, int64_t j, double* sm) {
  const int64_t n = a.n;
  const int t = threadIdx.x, nt = blockDim.x;
  const int cur = int(j & 1), prv = cur ^ 1;
  double* col = a.A + j * n;  // column j
  const int64_t m = n - j - 1;  // length of x = A[j+1:, j]
  double* x = col + j + 1;
  double ss = 0.0, mx = 0.0;  // sum of squares and max |x_i| over i >= 1
  if (j > 0) {
    // w_{j-1} = tau y + alpha v with alpha = -(tau^2/2)(y.v), over rows j .. n-1 (index r - j)
    const int64_t mm = n - j;
    const double tp = a.tau[prv];
    const double* __restrict__ v = a.V + prv * n;
    const double* y = a.Y + prv * n;
    double* __restrict__ w = a.W + prv * n;
    double* __restrict__ cj = col + j;
    double dot = 0.0;
#pragma unroll 4
    for (int64_t i = t; i < mm; i += nt) dot = fma(__ldcg(y + i), v[i], dot);
    dot = block_reduce_sum(dot, sm);
    const double alpha = -0.5 * tp * tp * dot;
    const double w0 = fma(alpha, v[0], tp * __ldcg(y));
    // A[r, j] -= v[r-j] w[0] + w[r-j] v[0] (v[0] = 1); rows r > j+1 feed the norm
#pragma unroll 4
    for (int64_t i = t; i < mm; i += nt) {
      const double wi = fma(alpha, v[i], tp * __ldcg(y + i));
      w[i] = wi;
      const double c = cj[i] - fma(v[i], w0, wi);
      cj[i] = c;
      if (i >= 2) {
        ss = fma(c, c, ss);
        mx = fmax(mx, fabs(c));
      }
    }
  } else {
    for (int64_t i = t + 1; i < m; i += nt) {
      const double c = x[i];
      ss = fma(c, c, ss);
      mx = fmax(mx, fabs(c));
    }
  }
  ss = block_reduce_sum(ss, sm);
  mx = block_reduce_max(mx, sm);
  if (t == 0) a.d[j] = col[j];
  if (j + 1 >= n) return;
  // reflector of x (length m), LAPACK's convention:
  // beta = -sign(alpha) ||x||, tau = (beta - alpha) / beta, v = [1, x[1:] / (alpha - beta)]
  if (mx > 0.0 && !(ss > 0x1p-900 && ss < 0x1p900)) {
    // the plain sum of squares under- or overflowed: recompute it scaled by max |x_i|
    const double inv = 1.0 / mx;
    double s2 = 0.0;
    for (int64_t i = t + 1; i < m; i += nt) {
      const double q = x[i] * inv;
      s2 = fma(q, q, s2);
    }
    ss = block_reduce_sum(s2, sm) * mx * mx;
  }
  if (t == 0) {
    const double alpha = x[0];
    const double xnorm = sqrt(ss);
    double tau = 0.0, beta = alpha, scale = 0.0;
    if (mx > 0.0) {
      beta = -copysign(hypot(alpha, xnorm), alpha);
      tau = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    sm[0] = scale;
    a.tau[cur] = tau;
    a.e[j] = beta;
  }
  __syncthreads();
  const double scale = sm[0];
  double* __restrict__ v = a.V + cur * n;
  const double* __restrict__ xr = x;
#pragma unroll 4
  for (int64_t i = t; i < m; i += nt) v[i] = (i == 0) ? 1.0 : xr[i] * scale;
}

__global__ void __launch_bounds__(kColThreads) k_dense_column(DenseArgs a, int64_t j) {
  __shared__ double sm[32];
  column_step(a, j, sm);
}

// Fused sweep for column j over the trailing lower triangle B = A[j+1:, j+1:]
// (order m = n - j - 1): B <- B - vp wp^T - wp vp^T with column j-1's (vp, wp)
// (skipped for j = 0), then y += B v_j, taking both triangles' contributions from
// the stored lower one.  Tile (bi, bk), bi >= bk, of 64 x 64 per block of 256
// threads; thread (tx, ty), tx, ty in [0, 16), owns rows tx + 16 rr and columns
// ty + 16 cc (rr, cc in [0, 4)), so 16 threads read 16 consecutive rows of a
// column and every stored element costs four FMAs: two for the update, one into
// the thread's row sum and one into its column sum.  The 16 partial sums of each
// row and column are combined in shared memory and written to the tile's slot of
// P; k_dense_reduce adds the slots in a fixed order (no atomics: the reduction is
// bitwise reproducible).
__global__ void __launch_bounds__(256) k_dense_sweep(DenseArgs a, int64_t j) {
  __shared__ double s_v[kDenseTile], s_vp[kDenseTile], s_wp[kDenseTile];
  __shared__ double s_rv[kDenseTile], s_rvp[kDenseTile], s_rwp[kDenseTile];
  __shared__ double s_red[16][kDenseTile + 1];
  const int64_t n = a.n, m = n - j - 1;
  // tile index t -> (bi, bk) with bi >= bk and t = bi (bi + 1) / 2 + bk
  const int64_t tt = blockIdx.x;
  int64_t bi = int64_t((sqrt(8.0 * double(tt) + 1.0) - 1.0) * 0.5);
  while (bi * (bi + 1) / 2 > tt) --bi;
  while ((bi + 1) * (bi + 2) / 2 <= tt) ++bi;
  const int64_t bk = tt - bi * (bi + 1) / 2;
  const int cur = int(j & 1), prv = cur ^ 1;
  const bool upd = j > 0;
  // column j's vectors are indexed from row j+1 (B's row 0), column j-1's from row j
  const double* v = a.V + cur * n;
  const double* vp = a.V + prv * n + 1;
  const double* wp = a.W + prv * n + 1;
  const int64_t i0 = bi * kDenseTile, k0 = bk * kDenseTile;
  {
    const int q = threadIdx.x & 63, which = threadIdx.x >> 6;
    const int64_t idx = (which < 2 ? i0 : k0) + q;
    const bool ok = idx < m;
    if (which == 0) {
      s_rv[q] = ok ? v[idx] : 0.0;
      s_rvp[q] = (ok && upd) ? vp[idx] : 0.0;
    } else if (which == 1) {
      s_rwp[q] = (ok && upd) ? wp[idx] : 0.0;
    } else if (which == 2) {
      s_v[q] = ok ? v[idx] : 0.0;
      s_vp[q] = (ok && upd) ? vp[idx] : 0.0;
    } else {
      s_wp[q] = (ok && upd) ? wp[idx] : 0.0;
    }
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const bool diag = bi == bk;
  double* base = a.A + (j + 1) * n + (j + 1);  // B(0, 0)
  double yr[4] = {0.0, 0.0, 0.0, 0.0}, yc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int cc = 0; cc < 4; ++cc) {
    const int kk = ty + 16 * cc;
    const int64_t k = k0 + kk;
    const double vk = s_v[kk], vpk = s_vp[kk], wpk = s_wp[kk];
    double* colp = base + k * n + i0;
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const int ii = tx + 16 * rr;
      const int64_t i = i0 + ii;
      if (i < m && k < m && (!diag || ii >= kk)) {
        double* p = colp + ii;
        const double b = fma(-s_rvp[ii], wpk, fma(-s_rwp[ii], vpk, *p));
        *p = b;
        yr[rr] = fma(b, vk, yr[rr]);
        if (!diag || ii != kk) yc[cc] = fma(b, s_rv[ii], yc[cc]);
      }
    }
  }
  double* slot = a.P + tt * (2 * kDenseTile);
  // row totals: 16 column groups (ty) per row
#pragma unroll
  for (int rr = 0; rr < 4; ++rr) s_red[ty][tx + 16 * rr] = yr[rr];
  __syncthreads();
  if (threadIdx.x < kDenseTile) {
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < 16; ++q) acc += s_red[q][threadIdx.x];
    slot[threadIdx.x] = acc;
  }
  __syncthreads();
  // column totals: 16 row groups (tx) per column
#pragma unroll
  for (int cc = 0; cc < 4; ++cc) s_red[tx][ty + 16 * cc] = yc[cc];
  __syncthreads();
  if (threadIdx.x < kDenseTile) {
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < 16; ++q) acc += s_red[q][threadIdx.x];
    slot[kDenseTile + threadIdx.x] = acc;
  }
}

// y_i of column j's sweep: the row totals of the tiles in i's tile row (bk <= b)
// plus the column totals of the tiles in i's tile column (bi >= b), b = i / 64.
// One block per tile row b; its 256 threads are 64 rows x 4 interleaved chunks of
// that list, combined in a fixed order.
__global__ void __launch_bounds__(256) k_dense_reduce(DenseArgs a, int64_t j) {
  __shared__ double s_acc[4][kDenseTile];
  const int64_t m = a.n - j - 1;
  const int64_t T = (m + kDenseTile - 1) / kDenseTile;
  const int64_t b = blockIdx.x;
  const int r = threadIdx.x & 63, c = threadIdx.x >> 6;
  double acc = 0.0;
  // entries q = 0 .. T: q <= b is the row total of tile (b, q); q > b the column
  // total of tile (q - 1, b)
  for (int64_t q = c; q <= T; q += 4) {
    if (q <= b)
      acc += a.P[(b * (b + 1) / 2 + q) * (2 * kDenseTile) + r];
    else
      acc += a.P[((q - 1) * q / 2 + b) * (2 * kDenseTile) + kDenseTile + r];
  }
  s_acc[c][r] = acc;
  __syncthreads();
  const int64_t i = b * kDenseTile + threadIdx.x;
  if (threadIdx.x < kDenseTile && i < m)
    a.Y[int(j & 1) * a.n + i] = (s_acc[0][threadIdx.x] + s_acc[1][threadIdx.x]) +
                                (s_acc[2][threadIdx.x] + s_acc[3][threadIdx.x]);
  // the last block of the launch to finish takes column j + 1's step, which needs
  // every row of y (the ticket orders it after the other blocks' writes; no block
  // waits for another)
  __shared__ unsigned s_ticket;
  __shared__ double sm[32];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_ticket = atomicAdd(a.done, 1u);
  __syncthreads();
  if (s_ticket != gridDim.x - 1) return;
  __threadfence();
  column_step(a, j + 1, sm);
  if (threadIdx.x == 0) *a.done = 0u;  // ready for the next launch on this stream
}

// ---- driver -------------------------------------------------------------------
size_t dense_workspace(int64_t n, size_t tri_bytes) {
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t N = size_t(std::max<int64_t>(n, 1));
  const size_t T = (N + kDenseTile - 1) / kDenseTile;
  return al(tri_bytes) + al(8 * N * N) + 6 * al(8 * N) + al(16) + 2 * al(8 * N) + al(16) +
         al(8 * (T * (T + 1) / 2) * 2 * kDenseTile);
}

// The tridiagonal solver's workspace comes first, so that its status word sits
// at the start of the caller's workspace like for every other entry point.
int dense_reduce(int64_t n, const double* A, int64_t lda, void* ws, size_t tri_bytes, double** d_out,
                 double** e_out, cudaStream_t s) {
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t N = size_t(n);
  char* p = static_cast<char*>(ws) + al(tri_bytes);
  DenseArgs a;
  a.n = n;
  a.A = reinterpret_cast<double*>(p);
  p += al(8 * N * N);
  a.V = reinterpret_cast<double*>(p);
  p += 2 * al(8 * N);
  a.W = reinterpret_cast<double*>(p);
  p += 2 * al(8 * N);
  a.Y = reinterpret_cast<double*>(p);
  p += 2 * al(8 * N);
  a.tau = reinterpret_cast<double*>(p);
  p += al(16);
  a.d = reinterpret_cast<double*>(p);
  p += al(8 * N);
  a.e = reinterpret_cast<double*>(p);
  p += al(8 * N);
  a.done = reinterpret_cast<unsigned*>(p);
  p += al(16);
  a.P = reinterpret_cast<double*>(p);  // last: its size follows from the tile count
  *d_out = a.d;
  *e_out = a.e;
  if (cudaMemcpy2DAsync(a.A, 8 * N, A, 8 * size_t(lda), 8 * N, N, cudaMemcpyDeviceToDevice, s) !=
      cudaSuccess)
    return TDE_ECUDA;
  if (cudaMemsetAsync(a.e, 0, 8 * N, s) != cudaSuccess) return TDE_ECUDA;
  if (cudaMemsetAsync(a.done, 0, 16, s) != cudaSuccess) return TDE_ECUDA;
  // column 0's step, then per column j: the sweep and the reduction of its product,
  // whose last block takes column j + 1's step
  k_dense_column<<<1, kColThreads, 0, s>>>(a, 0);
  g_launches += 1;
  for (int64_t j = 0; j + 1 < n; ++j) {
    const int64_t m = n - j - 1;
    const int64_t T = (m + kDenseTile - 1) / kDenseTile;
    k_dense_sweep<<<unsigned(T * (T + 1) / 2), 256, 0, s>>>(a, j);
    k_dense_reduce<<<unsigned(T), 256, 0, s>>>(a, j);
    g_launches += 2;
  }
  return cudaGetLastError() == cudaSuccess ? TDE_OK : TDE_ECUDA;
}

}  // namespace tde
