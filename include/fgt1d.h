/*
 * fgt1d.h -- C ABI of the GB300 (sm_103a) sum-of-exponentials fast Gauss transform.
 *
 * The transform (eqs. 1.1-1.2 of Jiang, "A fast Gauss transform in one dimension
 * using sum-of-exponentials approximations", arXiv:1909.09825):
 *
 *     u_i = sum_{j=1..N} exp(-(x_i - y_j)^2 / (4 delta)) alpha_j,   i = 1..M,
 *
 * is evaluated with the SOE approximation of eq. 1.3,
 *     G(x; delta) ~ S_n(x; delta) = Re sum_{k=1..n_e} W_k exp(-tau_k |x| / sqrt(delta)),
 * (n_e = n/2 conjugate pairs, W_k = 2 w_k; Sec. 4), whose nodes come from the
 * Caratheodory-Fejer near-best rational approximation of e^z on (-inf, 0]
 * (Sec. 2.3, eqs. 2.10-2.14; Sec. 3.3).  The sources and targets are merged and
 * sorted (Sec. 4) and the split sums h+ / h- of eqs. 4.3-4.4 are swept with the
 * forward and backward recurrences of eqs. 4.5-4.6, then evaluated (eq. 4.1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Arrays named x, y, alpha, u, grad_* and perm are DEVICE pointers unless the
 *    name ends in _host; they are owned by the caller, contiguous, float64
 *    (perm: uint32).  They must stay valid until the stream work completes.
 *  - Merged order: the merged point q < N is source j = q (coordinate y[q]);
 *    q >= N is target i = q - N (coordinate x[q - N]).  The stable sort orders by
 *    coordinate, ties by q, so a source equal to a target precedes it and is
 *    counted in h+ (eq. 4.4 uses y_j <= x_i).  -0.0 is treated as +0.0.
 *  - `workspace` is a caller-allocated device buffer of at least the size returned
 *    by the matching *_workspace_size call, 256-byte aligned.  One workspace must
 *    not be used by two calls that can overlap on the GPU.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Compute entry
 *    points are asynchronous: they enqueue work and return.  Argument errors are
 *    returned immediately; conditions found on the device (a NaN/Inf coordinate,
 *    an expired bounded wait, a bad batch item) are recorded in the workspace and
 *    returned by fgt1d_check, which synchronises the stream.
 *  - Return value: FGT1D_OK (0) or one of the FGT1D_E* codes below.
 *  - P = M + N must be below 2^31.  M = 0 is a no-op; N = 0 writes u = 0.
 *  - Inter-block waits are bounded: a wait that runs past its bound (about 2 s of SM
 *    clock by default) records FGT1D_ETIMEOUT for fgt1d_check and the kernels end.
 *    Two environment variables, read at every call, exist to test this path without a
 *    GPU fault: FGT1D_SPIN_LIMIT_CYCLES (a positive integer of SM clock cycles)
 *    replaces the bound, and FGT1D_FAULT=sweep_timeout or sort_timeout makes one wait
 *    of the forward sweep or of each prefix sort pass run out (tile 0 is never
 *    processed).
 *    After an expired sort wait the results are not written.  Leave both unset in use.
 */
#ifndef FGT1D_H
#define FGT1D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fgt1d_plan_s* fgt1d_plan; /* opaque, host memory owned by the library */
typedef void* fgt1d_stream;              /* a cudaStream_t */

/* status codes */
#define FGT1D_OK 0
#define FGT1D_EINVAL 1        /* bad argument: delta <= 0 or not finite, eps out of range,
                                 negative size, P >= 2^31, NULL pointer with nonzero size */
#define FGT1D_EUNSUPPORTED 2  /* eps below the smallest E_n reachable, or FP32 with eps < 1e-6 */
#define FGT1D_ENONFINITE 3    /* a coordinate was NaN or infinite (found on the device) */
#define FGT1D_ENOMEM 4        /* host allocation failed */
#define FGT1D_ETIMEOUT 5      /* a bounded inter-block wait gave up (found on the device) */
#define FGT1D_ECUDA 6         /* a CUDA runtime call failed */
#define FGT1D_EWORKSPACE 7    /* workspace NULL, misaligned or smaller than required */
#define FGT1D_ETOOLARGE 8     /* problem larger than the fixed scratch of fgt1d_execute_noalloc */

/* plan flags */
#define FGT1D_FP64 0u         /* FP64 accuracy at every step (recurrences, gaps, carries in
                                 FP64; each multiplier rounded once to FP64 from exact
                                 partial sums formed partly on the FP32 pipe) */
#define FGT1D_FP32 1u         /* bulk recurrences in FP32 complex, FP64 coordinate differences
                                 and inter-tile carries; requires eps >= 1e-6 */
#define FGT1D_EXACT_SELF 2u   /* a source at exactly a target's coordinate contributes
                                 G(0) = 1 instead of S_n(0) (the paper's codes use S_n(0)) */
#define FGT1D_F32X2 4u        /* recurrences in double-float (pairs of FP32, ~48-bit
                                 significand) with FP64 tile carries, within ~32x the FP64
                                 path's rounding; gradients use the FP64 path */

#define FGT1D_MAX_TERMS 8     /* largest n_e a plan can hold */
#define FGT1D_MAX_N 16        /* largest CF order n (Sec. 3.3; n <= 14 built in FP64, n = 16
                                 in double-double arithmetic) */

/* Step a0, the SOE generator (Sec. 2.3 eqs. 2.10-2.13, Sec. 3.3; eq. 3.1 for E_n).
 * Builds the CF type (n-1, n) approximation of e^z on (-inf, 0] for even n in
 * [2, FGT1D_MAX_N] on the host (FP64 up to n = 14; n = 16 in double-double, as the
 * paper builds its largest orders in extended precision) and converts it with eq. 2.11.
 * Outputs: *n_e = n/2; tau_k = sqrt(z_k) (one of each conjugate pair, Im tau_k > 0,
 * ascending Re tau_k, delta-free) and W_k = 2 w_k in caller host arrays of length
 * >= FGT1D_MAX_TERMS; *E_n = max |G(x;1) - S_n(x;1)| over the sampled grid (x = 0,
 * 1e5 log-spaced points in [1e-5, 1e2], and uniform grids on [0, 12] and [0, 1e-3]).
 * Errors: FGT1D_EINVAL for odd or out-of-range n or NULL outputs. */
int fgt1d_soe_cf(int n, int* n_e, double* tau_re, double* tau_im, double* w_re, double* w_im,
                 double* E_n);

/* Plan for bandwidth delta and accuracy eps: picks the smallest even n with
 * E_n <= eps (Sec. 3.3), keeps half of the conjugate pairs (Sec. 4) and
 * precomputes the per-term constants.  flags: FGT1D_FP64, FGT1D_FP32 or FGT1D_F32X2,
 * optionally or-ed with FGT1D_EXACT_SELF (honoured by fgt1d_execute, fgt1d_execute_host,
 * fgt1d_execute_noalloc, fgt1d_execute_self and fgt1d_geometry_apply; the batched
 * transform and fgt1d_backward ignore it).
 * Errors: FGT1D_EINVAL (delta <= 0/non-finite, eps not in (0, 0.5), unknown flags or
 * both FP32 and F32X2, out == NULL), FGT1D_EUNSUPPORTED (eps < E_n of FGT1D_MAX_N, or
 * FP32 with eps < 1e-6), FGT1D_ENOMEM. */
int fgt1d_plan_create(double delta, double eps, unsigned flags, fgt1d_plan* out);

/* Plan from a caller-given halved SOE (tau_k, W_k), k < n_e <= FGT1D_MAX_TERMS, with
 * Re tau_k > 0 (so every multiplier has modulus <= 1, eq. 2.3).  Used to run the
 * transform with any SOE, e.g. the hyperbolic-contour one of Sec. 3.4.  E_n is
 * recorded as NaN (unknown).  Errors as fgt1d_plan_create, plus FGT1D_EINVAL for
 * Re tau_k <= 0 or non-finite values. */
int fgt1d_plan_create_soe(double delta, int n_e, const double* tau_re, const double* tau_im,
                          const double* w_re, const double* w_im, unsigned flags, fgt1d_plan* out);

/* Reads a plan back.  Any output pointer may be NULL; the node arrays need room for
 * n_e values.  *n is the CF order (0 for a plan built from a given SOE). */
int fgt1d_plan_info(fgt1d_plan plan, int* n, int* n_e, double* E_n, double* delta,
                    unsigned* flags, double* tau_re, double* tau_im, double* w_re, double* w_im);

void fgt1d_plan_destroy(fgt1d_plan plan);

/* Device workspace bytes needed by fgt1d_execute for these sizes. */
int fgt1d_workspace_size(fgt1d_plan plan, int64_t M, int64_t N, size_t* bytes);

/* Steps a1-a7 (Sec. 4): the transform of eq. 1.1 for device arrays x[M] (targets),
 * y[N] (sources), alpha[N]; writes u[M] in the original target order.  Stream-ordered;
 * device-side errors are reported by fgt1d_check. */
int fgt1d_execute(fgt1d_plan plan, const double* x, int64_t M, const double* y,
                  const double* alpha, int64_t N, double* u, void* workspace, size_t ws_bytes,
                  fgt1d_stream stream);

/* fgt1d_execute that also records four caller-created CUDA events (cudaEvent_t,
 * any may be NULL) on `stream`: events[0] before the sort, events[1] after the sort,
 * events[2] after the forward sweep kernel, events[3] after the backward sweep kernel.
 * Used to time each stage on the launching stream. */
int fgt1d_execute_profiled(fgt1d_plan plan, const double* x, int64_t M, const double* y,
                           const double* alpha, int64_t N, double* u, void* workspace, size_t ws_bytes,
                           fgt1d_stream stream, void* const* events);

/* Same transform for HOST arrays (pageable or pinned): copies x, y, alpha to the
 * device, runs fgt1d_execute, copies u back and synchronises the stream.  The
 * workspace (device) must hold fgt1d_workspace_size_host bytes; it also carries the
 * device copies of the inputs and output.  Returns the device status like fgt1d_check. */
int fgt1d_workspace_size_host(fgt1d_plan plan, int64_t M, int64_t N, size_t* bytes);
int fgt1d_execute_host(fgt1d_plan plan, const double* x_host, int64_t M, const double* y_host,
                       const double* alpha_host, int64_t N, double* u_host, void* workspace,
                       size_t ws_bytes, fgt1d_stream stream);

/* fgt1d_execute_host without the final synchronisation (no counterpart in the paper):
 * the copies in, the transform and the copy of u out are enqueued on `stream` (the
 * strengths' copy on a second stream that the transform waits for) and the call
 * returns.  The host arrays must stay valid, and u_host unread, until the stream's work
 * is done; fgt1d_check(workspace, ws_bytes, stream) then waits and returns the device
 * status.  With pinned host arrays, calls on two streams with two workspaces overlap
 * one transform's copies with the other's kernels.  Arguments and argument errors as
 * fgt1d_execute_host (M = 0 and N = 0 are handled on the host at once). */
int fgt1d_execute_host_async(fgt1d_plan plan, const double* x_host, int64_t M, const double* y_host,
                             const double* alpha_host, int64_t N, double* u_host, void* workspace,
                             size_t ws_bytes, fgt1d_stream stream);

/* A batch of B independent transforms of uneven sizes and bandwidths in one pass of
 * the same kernels (the same method per item; the paper treats one transform).  Item b
 * has targets x[x_off[b] .. x_off[b+1]), sources y and strengths alpha at
 * [y_off[b] .. y_off[b+1]), bandwidth delta[b] (device array of B values, or NULL for
 * the plan's delta; the plan fixes eps and thus n_e), and writes u[x_off[b] ..
 * x_off[b+1]).  x_off and y_off are DEVICE arrays of B + 1 non-decreasing offsets in
 * [0, M_total] and [0, N_total]; they are read on the device, so the call can be captured
 * in a CUDA graph and replayed with new offsets, bandwidths and data.  Every item's
 * merged points are padded to whole 4096-point tiles; the workspace
 * (fgt1d_batched_workspace_size, an upper bound for any offsets with these totals)
 * therefore grows by at most one tile per item.  An item with bad offsets or a delta
 * that is not positive and finite is skipped and reported by fgt1d_check as
 * FGT1D_EINVAL.  Requires (M_total + N_total) / 4096 + B < 2^19. */
int fgt1d_batched_workspace_size(fgt1d_plan plan, int B, int64_t M_total, int64_t N_total, size_t* bytes);
int fgt1d_execute_batched(fgt1d_plan plan, int B, const int64_t* x_off, const int64_t* y_off,
                          const double* delta, const double* x, int64_t M_total, const double* y,
                          const double* alpha, int64_t N_total, double* u, void* workspace, size_t ws_bytes,
                          fgt1d_stream stream);

/* Identical targets and sources (Fig. 4.1's case): u_i = sum_j G(x_i - x_j) alpha_j for
 * the N points x (device), strengths alpha[N] and output u[N] (device, original order).
 * The N points are sorted once (not 2N merged points); the forward state is inclusive
 * and the backward state exclusive, so the self term and every coincident pair get
 * S_n(0) as in Fig. 4.1; with FGT1D_EXACT_SELF they get G(0) = 1 (each u_i gains
 * (1 - S_n(0)) times the total strength of the points at exactly x_i, itself included).
 * Workspace: fgt1d_self_workspace_size.  FP64 and FP32 plans (F32X2 plans return
 * FGT1D_EUNSUPPORTED).  N = 0 is a no-op.  Errors as fgt1d_execute. */
int fgt1d_self_workspace_size(fgt1d_plan plan, int64_t N, size_t* bytes);
int fgt1d_execute_self(fgt1d_plan plan, const double* x, int64_t N, const double* alpha, double* u,
                       void* workspace, size_t ws_bytes, fgt1d_stream stream);

/* Fixed geometry (Sec. 5: when the transform is applied many times to fixed points
 * with different strength vectors, pre-sort the points and store every exponential in
 * a table).  fgt1d_geometry_bind sorts the merged points of targets x[M] and sources
 * y[N] (steps a1-a2) and fills the multiplier table exp(-tau_k s (z_p - z_{p-1}))
 * for every merged point p and term k (step a4), all kept in the workspace;
 * fgt1d_geometry_apply then runs steps a3 and a5-a7 for a strength vector alpha[N]
 * (device) into u[M] (device, original target order), reading the multipliers from the
 * table: no sort and no exponential.  FP32 plans keep the sorted points without a table
 * (their sweeps form a multiplier in a few FP32 multiply-adds, cheaper than reading
 * it): their apply skips the sort only.  The workspace (fgt1d_geometry_workspace_size,
 * 256-byte aligned) belongs to the geometry until it is bound again or used by another
 * call; apply must get the same plan, tile shape and sizes as the bind (the workspace
 * carries a tag of M, N, delta, the nodes, the tile shape (the table's layout) and the
 * precision (its entries); a mismatch or an unbound workspace runs nothing and
 * fgt1d_check returns FGT1D_EINVAL).  Both calls are stream-ordered and graph-capturable;
 * apply calls sharing a workspace must not overlap.  Every precision: FP64, F32X2 (the
 * table then holds double-float entries rounded from the FP64 multipliers) and FP32;
 * FGT1D_EXACT_SELF allowed.  Errors: FGT1D_EINVAL,
 * FGT1D_EWORKSPACE, FGT1D_ECUDA; a NaN/Inf coordinate found by bind is reported by
 * fgt1d_check as FGT1D_ENONFINITE. */
int fgt1d_geometry_workspace_size(fgt1d_plan plan, int64_t M, int64_t N, size_t* bytes);
int fgt1d_geometry_bind(fgt1d_plan plan, const double* x, int64_t M, const double* y, int64_t N,
                        void* workspace, size_t ws_bytes, fgt1d_stream stream);
int fgt1d_geometry_apply(fgt1d_plan plan, int64_t M, int64_t N, const double* alpha, double* u,
                         void* workspace, size_t ws_bytes, fgt1d_stream stream);

/* Sweep tile shape and its autotuner.  Every sweep tile holds 4096 merged points (the
 * chunk of the associative scan, Sec. 4 recurrences split per tile); a tile runs as
 * `threads` threads of 4096 / threads consecutive points each.  threads = 128 (32
 * points per thread) or 256 (16 points per thread); 0 selects the default, 256 (the
 * gradient sweeps of fgt1d_backward then use 128 for plans with n_e > 5).  Results
 * differ between shapes only by rounding.  fgt1d_plan_get_tile returns the shape of the
 * transform sweeps (never 0).  Not thread-safe
 * with a concurrent execute on the same plan.  Errors: FGT1D_EINVAL. */
int fgt1d_plan_set_tile(fgt1d_plan plan, int threads);
int fgt1d_plan_get_tile(fgt1d_plan plan, int* threads);

/* Times every tile shape on the caller's own workload and keeps the fastest in the
 * plan (no counterpart in the paper).  With x_off == NULL the workload is one
 * transform (fgt1d_execute with M = M_total, N = N_total; B must be 1), otherwise the
 * batch of fgt1d_execute_batched (same arguments).  Each shape runs once untimed and
 * then `reps` (>= 1) times, timed with CUDA events on `stream`; u is overwritten and the
 * call synchronises the stream, so it cannot be captured in a graph (capture the
 * execute calls after it).  *threads_out (may be NULL) receives the chosen shape and
 * ms_out (may be NULL, room for 2) the mean milliseconds of shapes 128 and 256.  If
 * the environment variable FGT1D_TILE_THREADS is 128 or 256 that shape is taken
 * without timing (ms_out gets -1).  If FGT1D_TUNE_CACHE names a file, a choice stored
 * there for the same precision, n_e, floor(log2(M_total + N_total)) and kind (single or
 * batched) is taken without timing (ms_out gets -1), and a timed choice is appended to
 * it (text lines "<precision flags> <n_e> <log2 size> <batched> <threads> <ms>"; the
 * file belongs to one GPU model).  Errors: those of the execute call, or the device
 * status as fgt1d_check reports it; the plan keeps its previous shape on error. */
int fgt1d_autotune(fgt1d_plan plan, int B, const int64_t* x_off, const int64_t* y_off, const double* delta,
                   const double* x, int64_t M_total, const double* y, const double* alpha, int64_t N_total,
                   double* u, void* workspace, size_t ws_bytes, int reps, fgt1d_stream stream, int* threads_out,
                   float* ms_out);

/* The transform of fgt1d_execute for callers that cannot allocate device memory (no
 * counterpart in the paper).  Takes only the inputs and the output: its scratch is a
 * fixed 16 MiB array in the library's device memory, held on every GPU that loads the
 * library until the process exits, which fits any plan with M + N <= 65,536 points;
 * more points return FGT1D_ETOOLARGE.  Pointer rules and errors as fgt1d_execute
 * (a NULL array with a nonzero size returns FGT1D_EINVAL before any GPU work).  The
 * first call on a device with M > 0 and N > 0 looks up the array's address (once per
 * device, that device current; a failed lookup returns FGT1D_ECUDA and is retried by
 * the next call): make it before any stream capture.  All calls share the array, so
 * calls whose GPU work can overlap race and must be ordered by the caller.
 * Device-side conditions (NaN/Inf coordinates, an expired wait) are not reported by
 * this entry point. */
int fgt1d_execute_noalloc(fgt1d_plan plan, const double* x, int64_t M, const double* y,
                          const double* alpha, int64_t N, double* u, fgt1d_stream stream);

/* Range partition of one transform over several devices or processes (no counterpart
 * in the paper, whose Sec. 6 only remarks that the method parallelises over modes).  The
 * recurrences of eqs. 4.5-4.6 are affine in the state, so a contiguous range of the
 * sorted coordinate line -- a "segment", holding every target and source whose
 * coordinate falls in it -- can be transformed alone and corrected afterwards by the
 * states entering it from both sides.  Segments are ordered along the line (g = 0 ..
 * G-1) and must not interleave: every point of segment g lies at or right of every
 * point of segment g-1 (points with equal coordinates belong to one segment).
 *
 * Boundary record of a segment, FGT1D_SEGMENT_DOUBLES(n_e) doubles:
 *   [0, n_e) Re F_k, [n_e, 2 n_e) Im F_k: F_k = sum over the segment's sources of
 *            alpha_j exp(-tau_k (z_last - y_j) / sqrt(delta)), the forward state of
 *            eq. 4.5 at its last point;
 *   [2 n_e, 4 n_e) Re G_k, Im G_k: G_k = sum over its sources of alpha_j
 *            exp(-tau_k (y_j - z_first) / sqrt(delta)), the backward state of eq. 4.6 at
 *            its first point with that point's own strength included;
 *   [4 n_e] z_first, [4 n_e + 1] z_last: its smallest and largest coordinate (NaN for a
 *            segment without points).
 * A carry record has the same size: Re/Im F_in (the forward state at z_prev, the last
 * point of the segments to the left), Re/Im G_in (the backward state, inclusive, at
 * z_next, the first point of the segments to the right), z_prev, z_next (NaN: none).
 *
 * fgt1d_segment_execute: the transform of the segment's targets x[M] and sources y[N],
 *   alpha[N] (device) with zero entering states into u[M] (device), and its boundary
 *   record into `boundary` (device).  Any of M, N may be 0 (a segment without targets
 *   still reports its sources' states).  Workspace: fgt1d_workspace_size(plan, M, N);
 *   it keeps the segment's sorted points for fgt1d_segment_apply.
 * fgt1d_segment_compose: HOST arithmetic on the boundary records of all G segments
 *   (`boundaries`, host, G records in order): writes segment g's carry record (host).
 *   Each step across a segment multiplies by exp(-tau_k d / sqrt(delta)) of a span d
 *   between two FP64 coordinates, computed directly.  FGT1D_EINVAL if the segments are
 *   not ordered or a record is not finite.
 * fgt1d_segment_apply: u[i] += Re sum_k W_k (F_in,k exp(-tau_k (x_i - z_prev)/sqrt(delta))
 *   + G_in,k exp(-tau_k (z_next - x_i)/sqrt(delta))) for every target of the segment,
 *   with `carry` a DEVICE copy of its carry record, the workspace of the preceding
 *   fgt1d_segment_execute (same plan and sizes, not used by another call in between),
 *   and u as written by it.  Terms below 2^-60 of the carry are skipped.
 * Together: execute on every segment, gather the G boundary records, compose, apply;
 * u then equals the transform of all points (up to rounding).  Errors as
 * fgt1d_execute; FP64, FP32 and F32X2 plans (the carries are FP64 in each). */
#define FGT1D_SEGMENT_DOUBLES(n_e) (4 * (n_e) + 2)
int fgt1d_segment_execute(fgt1d_plan plan, const double* x, int64_t M, const double* y,
                          const double* alpha, int64_t N, double* u, double* boundary,
                          void* workspace, size_t ws_bytes, fgt1d_stream stream);
int fgt1d_segment_compose(fgt1d_plan plan, int G, int g, const double* boundaries, double* carry);
int fgt1d_segment_apply(fgt1d_plan plan, int64_t M, int64_t N, const double* carry, double* u,
                        void* workspace, size_t ws_bytes, fgt1d_stream stream);

/* Gradients of L = sum_i grad_u[i] u_i for the transform computed by fgt1d_execute
 * (the SOE operator of eq. 1.3 with the plan's nodes; the paper has no gradients):
 *   grad_alpha[j] = sum_i grad_u[i] S(x_i - y_j)      (the transform with roles swapped)
 *   grad_x[i]     = grad_u[i] sum_j alpha_j S'(x_i - y_j)
 *   grad_y[j]     = -alpha_j sum_i grad_u[i] S'(x_i - y_j)
 *   grad_delta[0] = sum_ij grad_u[i] alpha_j dS(x_i - y_j; delta)/d delta
 * with S' taken as 0 at coincident points (S has a cusp there).  Each sum runs on the
 * same sorted recurrences as the transform (eqs. 4.5-4.6) with a second evaluation
 * channel Re sum_k V_k (h+ - h-), V_k = -tau_k W_k / sqrt(delta); grad_delta uses the
 * scale invariance sum x dL/dx + sum y dL/dy + 2 delta dL/ddelta = 0.  Device arrays:
 * grad_u[M]; outputs grad_x[M], grad_y[N], grad_alpha[N], grad_delta[1], any of which
 * may be NULL (not computed).  When grad_x or grad_delta is requested, the second sum
 * (targets y, sources x) reuses the first one's sorted points and multipliers.
 * Workspace from fgt1d_backward_workspace_size.  Stream-ordered like fgt1d_execute. */
int fgt1d_backward_workspace_size(fgt1d_plan plan, int64_t M, int64_t N, size_t* bytes);
int fgt1d_backward(fgt1d_plan plan, const double* x, int64_t M, const double* y, const double* alpha,
                   int64_t N, const double* grad_u, double* grad_x, double* grad_y, double* grad_alpha,
                   double* grad_delta, void* workspace, size_t ws_bytes, fgt1d_stream stream);

/* Steps a1-a2 alone (Sec. 4, first step; Sec. 5 sorting): the stable sort of the
 * merged points.  perm[p] (device, uint32, length M + N) receives the merged index at
 * sorted position p.  Workspace from fgt1d_sort_workspace_size.  Like every entry point
 * that sorts, it detects sources and targets that each arrive in non-decreasing order
 * (Sec. 5's pre-sorted points) and then merges the two runs in one pass instead of
 * running the radix passes; the permutation is the same either way.  The radix passes
 * sort 32-bit keys that are a non-decreasing function of the coordinate within its
 * item's range and fix up the few runs of equal keys; when a run of more than 32
 * distinct coordinates shares one key (a cluster narrower than the range / 2^32), the
 * full 64-bit sort runs instead, with the same result. */
int fgt1d_sort_workspace_size(int64_t M, int64_t N, size_t* bytes);
int fgt1d_sort_merged(const double* x, int64_t M, const double* y, int64_t N, uint32_t* perm,
                      void* workspace, size_t ws_bytes, fgt1d_stream stream);

/* Measures the pipes that bound this library's kernels on the current device (no
 * counterpart in the paper): 16 independent chains per thread of FP64 FMA, FP32 FMA and the
 * special-function unit's ex2.approx and sin.approx on every SM, each timed with CUDA
 * events on `stream` (best of two after a warm-up launch).  out (host, >= 10 doubles):
 * out[0], out[1] FP64 FMA per second and per SM per clock cycle; out[2], out[3] the same
 * for FP32 FMA; out[4], out[5] ex2; out[6], out[7] sin; out[8] the number of SMs; out[9]
 * the SM clock in MHz during the FP64 run (from the cycle counter and the global timer).
 * One FMA is two floating-point operations.  Allocates a few bytes of device memory and
 * synchronises the stream.  Errors: FGT1D_EINVAL (out NULL), FGT1D_ECUDA. */
int fgt1d_measure_peaks(double* out, fgt1d_stream stream);

/* Synchronises `stream`, then returns and clears the device status recorded in the
 * workspace by the previous compute calls: FGT1D_OK, FGT1D_EINVAL (a bad batch item),
 * FGT1D_ENONFINITE, FGT1D_ETIMEOUT, or FGT1D_ECUDA if the stream reported an error. */
int fgt1d_check(void* workspace, size_t ws_bytes, fgt1d_stream stream);

/* Human-readable text of a status code (static storage). */
const char* fgt1d_strerror(int status);

/* Library version: major * 10000 + minor * 100 + patch. */
int fgt1d_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FGT1D_H */
