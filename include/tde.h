/*
 * tde.h -- C ABI of the B300 (sm_103a) boundary-row divide-and-conquer solver for
 * all eigenvalues of real symmetric tridiagonal matrices T = tridiag(e, d, e),
 * in IEEE double precision.
 *
 * Method: the eigenvalue-only boundary-row D&C of arxiv 2605.26599 ("Reducing
 * Internal State in Eigenvalue-Only Divide-and-Conquer Tridiagonal
 * Eigensolvers").  T is torn at balanced cut points into a rank-one modification
 * of two children (Eq. 1 / Eq. dc-split); each child keeps only its eigenvalues
 * and the first and last rows of its eigenvector matrix (the boundary-row state,
 * Eq. boundary-state); a merge forms diag(D) + rho z z^T from the child spectra and
 * boundary rows (Eq. merge-problem), deflates it, solves the secular equation
 * for every root, and propagates only the two boundary rows to the parent
 * (Algorithm 1; Sec. 4.1).  The root merge solves roots only.
 *
 * Conventions shared by every entry point
 *  - All array pointers are DEVICE pointers to float64 data unless a name ends
 *    in _host.  Arrays are dense and contiguous, 8-byte aligned.  The caller owns
 *    every buffer; no entry point allocates device memory.
 *  - ws is caller-provided device workspace, 256-byte aligned, of at least the
 *    size returned by the matching *_workspace query.  Its contents need no
 *    initialisation and are clobbered.  Two calls that run concurrently must not
 *    share a workspace.
 *  - stream is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    Every compute entry point only enqueues work on that stream and returns
 *    without synchronising; it performs no host<->device copy, so a call can be
 *    captured into a CUDA graph.
 *  - leaf is the largest leaf order of the split tree (1..64; 0 selects 32).
 *  - Return value: TDE_OK, or a negative code for invalid arguments, a too-small
 *    workspace or a failed launch (nothing has been enqueued for EINVAL/EWORKSPACE).
 *    Numerical failures found on the device (no convergence, non-finite input)
 *    are recorded in a status word inside ws and read with tde_get_info().
 *  - d, e and offsets are read-only; outputs are written once per call.
 */
#ifndef TDE_H_
#define TDE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TDE_OK = 0,
  TDE_EINVAL = -1,      /* invalid argument (null pointer, negative size, bad leaf) */
  TDE_ECUDA = -2,       /* a CUDA launch or API call failed */
  TDE_EWORKSPACE = -3,  /* ws_bytes smaller than the workspace query */
  TDE_ENOCONV = 1,      /* device: a leaf QL or secular iteration hit its cap */
  TDE_ENONFINITE = 2,   /* device: d or e holds a NaN or an infinity */
  TDE_ETIMEOUT = 3      /* device: a bounded wait gave up (reserved) */
} tde_status;

/* Bytes of workspace tde_eigvals needs for order n with the given leaf order.
 * Host-only; O(n) (about 200 n bytes).  Defined by the O(n) boundary-row state
 * contract of Sec. 3.3 / Sec. 4.2. */
int tde_eigvals_workspace(int64_t n, int32_t leaf, size_t* bytes);

/* All eigenvalues of one tridiagonal (Sec. 3.1 problem setting).
 *   n       order, n >= 0 (n = 0 is a no-op)
 *   d       [n]   diagonal
 *   e       [n-1] off-diagonal (e[i] couples rows i and i+1); may be NULL if n <= 1
 *   lambda  [n]   output, eigenvalues in ascending order
 * Internally scales T by the power of two 2^-floor(log2 max|T|) (exact; the
 * eigenvalues are unscaled exactly), sets negligible off-diagonals
 * (|e_i| <= eps sqrt|d_i| sqrt|d_{i+1}|) to zero (Sec. 4.2 driver), solves the
 * leaves by implicit QR keeping two eigenvector rows, and merges level by level. */
int tde_eigvals(int64_t n, const double* d, const double* e, double* lambda, int32_t leaf,
                void* ws, size_t ws_bytes, void* stream);

/* Maximum number of requested rows of one tde_eigvecs_rows call. */
#define TDE_MAX_SEL_ROWS 1024

/* Bytes of workspace tde_eigvecs_rows needs for order n, nsel requested rows and
 * the given leaf order: the tde_eigvals workspace plus about 24 nsel n bytes. */
int tde_eigvecs_rows_workspace(int64_t n, int64_t nsel, int32_t leaf, size_t* bytes);

/* Eigenvalues and requested rows of the eigenvector matrix (Algorithm 1 with a
 * general requested row list sigma: the requested rows are carried through the
 * merge tree beside the boundary rows and updated by the selected-row lemma, so
 * Q itself is never formed).
 *   n, d, e, lambda, leaf   as for tde_eigvals
 *   nsel    number of requests, 0 <= nsel <= TDE_MAX_SEL_ROWS (0: eigenvalues only)
 *   rows    [nsel] device int64, row indices in [0, n), any order, repeats allowed
 *   qrows   [nsel * n] device output, row-major: qrows[q * n + j] = Q[rows[q]][j],
 *           where Q is orthogonal, T = Q diag(lambda) Q^T and column j belongs to
 *           lambda[j].  All requested rows come from the same Q, so every column's
 *           sign is consistent across them (the sign itself is arbitrary).
 *   ws      tde_eigvecs_rows_workspace bytes, 256-byte aligned, caller-owned
 * Argument errors return TDE_EINVAL before any launch.  A requested row outside
 * [0, n) sets the device status (tde_get_info) to TDE_EINVAL and its output row to
 * zeros.  Cost: the eigenvalue solve plus O(n^2) per distinct requested row. */
int tde_eigvecs_rows(int64_t n, const double* d, const double* e, int64_t nsel,
                     const int64_t* rows, double* lambda, double* qrows, int32_t leaf, void* ws,
                     size_t ws_bytes, void* stream);

/* Bytes of workspace tde_dense_eigvals needs: 8 n^2 for the reduced copy of A, a
 * few n-vectors, and the tridiagonal solver's workspace. */
int tde_dense_eigvals_workspace(int64_t n, int32_t leaf, size_t* bytes);

/* All eigenvalues of a dense symmetric matrix (the dense pipeline of Sec. 2: an
 * orthogonal reduction A = Q T Q^T to tridiagonal form, then the boundary-row
 * solver on T; Q is not kept).
 *   A       [lda * n] device, read only; column j is A[j * lda .. j * lda + n).
 *           Only the lower triangle of that column-major layout is read (the upper
 *           triangle of a row-major array), so a full symmetric matrix may be passed
 *           in either order.
 *   lambda  [n] output, ascending
 *   ws      tde_dense_eigvals_workspace bytes, 256-byte aligned, caller-owned
 * Householder reflections, one column at a time: an FP64 sweep over the trailing
 * lower triangle per column (4 FMAs per stored element), so about (2/3) n^3 FMAs. */
int tde_dense_eigvals(int64_t n, const double* A, int64_t lda, double* lambda, int32_t leaf,
                      void* ws, size_t ws_bytes, void* stream);

/* Workspace for tde_eigvals_batched with the given packing (host offsets). */
int tde_eigvals_batched_workspace(int64_t batch, const int64_t* offsets_host, int32_t leaf,
                                  size_t* bytes);

/* Eigenvalues of `batch` independent tridiagonals packed back to back (the
 * level-synchronous schedule of Sec. 4.1 applied to a forest: every level of
 * every tree runs in the same launches).
 *   offsets_host [batch+1] host copy of the packing, offsets[0] = 0,
 *                non-decreasing; matrix k owns rows offsets[k] .. offsets[k+1]-1
 *   offsets_dev  [batch+1] the same values in device memory (int64)
 *   d, e, lambda [offsets[batch]] packed; e[offsets[k+1]-1] is ignored
 * The plan (tree shapes and launch sizes) is derived from offsets_host on the
 * host; a CUDA graph captured from this call stays valid while the packing is
 * unchanged. */
int tde_eigvals_batched(int64_t batch, const int64_t* offsets_host, const int64_t* offsets_dev,
                        const double* d, const double* e, double* lambda, int32_t leaf,
                        void* ws, size_t ws_bytes, void* stream);

/* Workspace for tde_eigvals_backward with the given packing (leaf <= 32): the
 * default O(n) layout with 4 checkpoint slots (see tde_eigvals_backward). */
int tde_eigvals_backward_workspace(int64_t batch, const int64_t* offsets_host, int32_t leaf,
                                   size_t* bytes);

/* Workspace for tde_eigvals_backward with `slots` checkpoint slots (slots >= 1;
 * slots = 0, or at least the number of merge steps, gives the levels layout that
 * checkpoints every level).  More slots trade memory for less recomputation. */
int tde_eigvals_backward_workspace_slots(int64_t batch, const int64_t* offsets_host, int32_t leaf,
                                         int32_t slots, size_t* bytes);

/* Gradient of a loss of the eigenvalues with respect to d and e (reverse mode),
 * for a packed batch as in tde_eigvals_batched (batch = 1 with offsets {0, n} for
 * one matrix).
 *   grad_lambda [N]  dL/dlambda, aligned with the ascending eigenvalues
 *   lambda      [N]  output: the eigenvalues (may be NULL)
 *   grad_d      [N]  output: dL/dd
 *   grad_e      [N]  output: dL/de (entry at the last row of each matrix is 0)
 * Method: implicit differentiation of every merge, in a reverse sweep over the
 * merge steps (top-down) that rebuilds each merge from the boundary-row state at
 * its input and pulls the adjoints back through the placement, the secular
 * eigen-decomposition (implicit differentiation of every root and of the Cauchy
 * form of the boundary rows), the deflation and the formation of the merge
 * problem; the leaves use the adjoint of their full eigen-decomposition and the
 * tearing d -= |beta| of Eq. (1).  Deflation decisions and the tree are constants
 * of the differentiation.  Simple (distinct) eigenvalues are assumed.
 * Workspace, chosen from ws_bytes: with the size of
 * tde_eigvals_backward_workspace (or of tde_eigvals_backward_workspace_slots for S
 * slots) the states of S levels are checkpointed and the others recomputed
 * forward in a bisection schedule, each rebuilt merge solving its roots again:
 * O(n) memory for a fixed S.  A workspace of the levels layout
 * (tde_eigvals_backward_workspace_slots with slots = 0) checkpoints every level
 * and every step's roots (O(n log n)) and recomputes nothing.  Both layouts give
 * the same gradient.  Sizes below the one-slot layout return TDE_EWORKSPACE. */
int tde_eigvals_backward(int64_t batch, const int64_t* offsets_host, const int64_t* offsets_dev,
                         const double* d, const double* e, const double* grad_lambda,
                         double* lambda, double* grad_d, double* grad_e, int32_t leaf,
                         void* ws, size_t ws_bytes, void* stream);

/* Reads the device status word of a workspace used by a previous call on
 * `stream` (synchronises that stream).  *info receives 0 or a positive
 * tde_status code.  The word is reset at the start of every compute call. */
int tde_get_info(const void* ws, void* stream, int32_t* info);

/* Measured FP64 fused multiply-add throughput of the current device, in FMA
 * instructions per second (every lane of every warp issuing independent
 * chains); the denominator of the solver's FP64 roofline.  Blocks the host for
 * about 50 ms.  Returns TDE_OK and writes *fma_per_s. */
int tde_measure_fp64_peak(double* fma_per_s);

/* Launch-shape tuning for subsequent calls on this thread (0 restores a default):
 *   warp_min_k      merges whose active rank reaches this solve one warp per root
 *                   (default 256); smaller ones sum each root's sweeps over four
 *                   lanes of a warp (one root per lane for its other steps), or
 *                   take one thread per root below order 24;
 *   small_list_min  a step with fewer small-merge roots than this hands them to the
 *                   warp-per-root kernels too (default 18944 = 148 SMs x 4 warps x 32).
 * They change the time, and the eigenvalues only at the level of rounding (the
 * kernels sum in different orders, and only the warp-per-root kernels use the
 * block expansion of tde_set_multipole). */
int tde_set_tuning(int32_t warp_min_k, int32_t small_list_min);

/* Threshold of the block expansion for subsequent calls on this thread: in merges
 * whose active rank K reaches min_k (and that the warp-per-root kernels solve), the
 * FP64 secular sweeps, the Lowner products (in log form) and the boundary-row sums
 * take distant blocks of 128 poles through series of the block's normalised
 * moments instead of term by term; the series length follows the block's
 * separation (radius / distance <= 1/64, 1/16, 1/4, 1/3: 10, 14, 27, 35 terms for
 * the secular and Lowner sums, 10, 16, 32, 40 for the row sums), which keeps the
 * series error below the rounding of the sums it replaces.  Merges of 192 or more
 * blocks also take distant superblocks of 32 blocks.  min_k = 0 restores the
 * default (1024); any other value below 256 is TDE_EINVAL; a value above every K
 * turns the expansion off.  *previous (if not NULL) receives the value in force
 * before the call. */
int tde_set_multipole(int32_t min_k, int32_t* previous);
/* out[0] = warp_min_k, out[1] = small_list_min of this thread. */
int tde_get_tuning(int32_t* out);

/* Host-only description of the split-tree plan for a packing (no device work):
 * out[0] merge steps (tree levels), out[1] leaves, out[2] merges, out[3] the
 * largest number of merges in one step.  Node (h, i) of a matrix of order n covers
 * rows [floor(i n / 2^h), floor((i+1) n / 2^h)); leaves sit at depth L, the
 * smallest L with ceil(n / 2^L) <= leaf, capped so that 2^L <= n (Sec. 3.3
 * balanced tree). */
int tde_plan_query(int64_t batch, const int64_t* offsets_host, int32_t leaf, int64_t* out);

/* Applies the solver's device reciprocal (a hardware approximation refined by the
 * third-order step r (1 + e + e^2), e = 1 - x r) to x[0..n) -> out[0..n), device
 * arrays, on `stream`.  Exposed so tests can compare it with IEEE 1/x. */
int tde_check_reciprocal(int64_t n, const double* x, double* out, void* stream);

/* Applies the solver's device reciprocal square root (a hardware approximation y0
 * of x^(-1/2) refined by the third-order step y0 (1 + e/2 + 3 e^2/8),
 * e = 1 - x y0^2; used for the boundary-row normalisation) to x[0..n) -> out[0..n),
 * device arrays, on `stream`.  Defined for finite x > 0.  Exposed so tests can
 * compare it with CUDA's rsqrt and with IEEE 1/sqrt(x).  TDE_EINVAL for n < 0 or
 * null arrays with n > 0. */
int tde_check_rsqrt(int64_t n, const double* x, double* out, void* stream);

/* Number of kernel launches the last compute call on this thread enqueued. */
int64_t tde_last_launch_count(void);

/* Per-kernel timing for measurement.  With profiling enabled, every compute call
 * on this thread records a CUDA event pair around each kernel launch; collect
 * synchronises on those events, writes per-kernel-class milliseconds and launch
 * counts into ms[0..nids) / launches[0..nids) (classes: 0 plan, 1 scale, 2 leaves,
 * 3 form, 4 deflate, 5 secular, 6 lowner, 7 rows, 8 place, 9 requested-row form,
 * deflation and placement, 10 requested-row update) and clears the record.
 * Do not enable it while the stream is being captured into a CUDA graph. */
int tde_profile_enable(int on);
/* Kernel classes the profiler records on this thread: bit c of mask selects class c
 * (numbering as above); 0 selects every class (the default).  Recording fewer
 * classes puts fewer event records between the kernels of a timed region. */
int tde_profile_select(uint32_t mask);
int tde_profile_collect(int nids, double* ms, int64_t* launches);
/* Like tde_profile_collect, with a per-merge-step breakdown: ms and launches hold
 * (nsteps + 1) rows of nids entries; row 0 is the total, row s + 1 the launches of
 * merge step s (bottom-up level s of the split tree). */
int tde_profile_collect_steps(int nids, int nsteps, double* ms, int64_t* launches);

/* Copies the workspace's device work counters (synchronises `stream`):
 * out[0] pole terms summed exactly in FP64 secular sweeps (K per sweep of a root,
 * fewer where the block expansion takes distant blocks through their series),
 * out[1] FP64 secular sweeps, out[2] Lowner factors multiplied directly (K per
 * pole without the block expansion), out[3] boundary-row terms summed
 * exactly (K per root without the block expansion),
 * out[4] roots solved, out[5] deflated eigenvalues, out[6] close-pole rotations,
 * out[7] leaf plane rotations, out[8] merges whose rotated deflated eigenvalues
 * needed sorting, out[9] entries sorted, out[10] single-precision secular pole
 * sweeps x K, out[11] single-precision secular sweeps, out[12] requested-row
 * updates as (pole, root, row) triples, out[13] their (pole, root) sweeps (one per
 * group of up to four rows of a merge), out[14] pole blocks taken through their
 * series in FP64 secular sweeps, out[15] series evaluated for the boundary-row sums
 * (two or three per far pole block), out[16] pair blocks taken through their series in the
 * Lowner products, out[17..19] the FP64 operations of the series evaluations of
 * the secular sweeps, Lowner products and boundary rows (each far block's FP64
 * Horner head plus its distance, reciprocal, argument and accumulation; the
 * float tails are not counted).  n <= 20 entries are copied.  The counters are
 * reset at the start of every compute call that uses the workspace. */
int tde_read_work(const void* ws, void* stream, unsigned long long* out, int n);

/* Largest order tde_eigvals_noalloc accepts. */
#define TDE_NOALLOC_MAX_N 16384

/* tde_eigvals without a caller workspace, for callers that cannot allocate
 * device memory (for instance code handed device pointers by a framework that
 * owns every allocation).  The paper has no counterpart; it is a convenience of
 * this library.  The workspace is a 4 MiB array compiled into the library, kept
 * on every GPU that loads it until the process exits.  d, e, lambda, leaf and
 * stream mean what they mean for tde_eigvals; n must not exceed
 * TDE_NOALLOC_MAX_N (TDE_EWORKSPACE otherwise, nothing enqueued), for any leaf
 * order.  No memory is allocated.  The first call on a device looks up the
 * array's device address in the device's primary context and caches it; make
 * that first call before any stream capture, and do not use this entry point
 * after cudaDeviceReset or from a non-primary context (the array may have moved).
 * All calls share the one array: calls that overlap on the GPU race and must be
 * serialised by the caller.  Numerical failures found on the device are read
 * with tde_noalloc_get_info. */
int tde_eigvals_noalloc(int64_t n, const double* d, const double* e, double* lambda,
                        int32_t leaf, void* stream);

/* Device status word of the last tde_eigvals_noalloc call on the current device
 * that enqueued work (n >= 1), read on `stream` (synchronises it; use the
 * stream of that call or one ordered after it).  *info receives 0 or a positive
 * tde_status code, as tde_get_info does for a caller workspace.  Allocates
 * nothing.  The paper has no counterpart. */
int tde_noalloc_get_info(void* stream, int32_t* info);

#ifdef __cplusplus
}
#endif
#endif /* TDE_H_ */
