/*
 * CPU oracle for the 1D Gauss transform and its SOE fast algorithm.
 *
 * TEST INFRASTRUCTURE ONLY: plain, slow, FP64, single-threaded unless an
 * OpenMP thread count is passed.  It shares no code with the CUDA library and
 * includes none of its headers.  Compile with -ffp-contract=off so that every
 * product is rounded on its own (no FMA contraction).
 *
 *   o1_direct      eqs. 1.1-1.2: u_i = sum_j alpha_j exp(-(x_i - y_j)^2 / (4 delta)),
 *                  Neumaier-compensated sum over j.
 *   o2_soe_direct  eqs. 1.3 and 4.1-4.2: u_i = sum_j alpha_j Re sum_k W_k
 *                  exp(-tau_k |x_i - y_j| / sqrt(delta)) over the halved node set.
 *   o3_recurrence  Sec. 4: stable sort of the merged points (sources first on
 *                  equal coordinates, eq. 4.4 puts y_j = x_i in h^+), forward
 *                  recurrence eq. 4.5 and backward recurrence eq. 4.6 with the
 *                  exponentials of consecutive gaps, evaluation eq. 4.1 and
 *                  unpermutation.
 *   o3_recurrence_par / o3_sort_merged_par  the same algorithm and sort on several
 *                  host cores (coordinate segments with directly computed span carries).
 *   o3_segment_boundary / o3_carry_apply  a segment's boundary states and the entering
 *                  states' contribution to its targets, as direct sums.
 *   o1_grad / o2_grad  direct O(MN) gradients of L = sum_i g_i u_i with respect to
 *                  alpha, x, y and delta, for the Gaussian and for the SOE kernel.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MAX_TERMS 16

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_openmp_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Neumaier's compensated addition: adds t to (*sum, *comp). */
static inline void neumaier_add(double* sum, double* comp, double t) {
    double s2 = *sum + t;
    if (fabs(*sum) >= fabs(t)) *comp += (*sum - s2) + t;
    else *comp += (t - s2) + *sum;
    *sum = s2;
}

/* O1: direct Gauss transform, eqs. 1.1-1.2. */
void o1_direct(const double* x, int64_t M, const double* y, const double* alpha, int64_t N,
               double delta, double* u, int nthreads) {
    set_threads(nthreads);
    const double four_delta = 4.0 * delta;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) if (nthreads != 1)
#endif
    for (int64_t i = 0; i < M; ++i) {
        double sum = 0.0, comp = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            double d = x[i] - y[j];
            neumaier_add(&sum, &comp, alpha[j] * exp(-(d * d) / four_delta));
        }
        u[i] = sum + comp;
    }
}

/* Real part of W e^{-tau r} for r >= 0: Re(W) e^{-a r} cos(b r) + Im(W) e^{-a r} sin(b r),
 * with tau = a + i b. */
static inline double soe_term(double tre, double tim, double wre, double wim, double r) {
    double mag = exp(-tre * r);
    return mag * (wre * cos(tim * r) + wim * sin(tim * r));
}

/* S_n(d; delta) = Re sum_k W_k exp(-tau_k |d| / sqrt(delta)), eq. 1.3 (halved set). */
static double soe_kernel(int n_e, const double* tre, const double* tim, const double* wre,
                         const double* wim, double d, double sqrt_delta) {
    double r = fabs(d) / sqrt_delta;
    double s = 0.0;
    for (int k = 0; k < n_e; ++k) s += soe_term(tre[k], tim[k], wre[k], wim[k], r);
    return s;
}

/* O2: direct SOE sum, eqs. 1.3, 4.1-4.2. */
void o2_soe_direct(const double* x, int64_t M, const double* y, const double* alpha, int64_t N,
                   double delta, int n_e, const double* tre, const double* tim, const double* wre,
                   const double* wim, double* u, int nthreads) {
    set_threads(nthreads);
    const double sd = sqrt(delta);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) if (nthreads != 1)
#endif
    for (int64_t i = 0; i < M; ++i) {
        double sum = 0.0, comp = 0.0;
        for (int64_t j = 0; j < N; ++j)
            neumaier_add(&sum, &comp, alpha[j] * soe_kernel(n_e, tre, tim, wre, wim, x[i] - y[j], sd));
        u[i] = sum + comp;
    }
}

/* ---- O3: the paper's algorithm ------------------------------------------------------ */

/* Merged point q: q < N is source j = q (coordinate y[q]); q >= N is target i = q - N. */
typedef struct {
    const double* x;
    const double* y;
    int64_t N;
} merged_t;

static inline double merged_coord(const merged_t* m, int64_t q) {
    return q < m->N ? m->y[q] : m->x[q - m->N];
}

/* Stable merge sort of merged indices by coordinate (ties keep the merged order). */
static void merge_sort(int64_t* a, int64_t* tmp, int64_t n, const merged_t* m) {
    for (int64_t width = 1; width < n; width *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * width) {
            int64_t mid = lo + width < n ? lo + width : n;
            int64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            int64_t i = lo, j = mid, k = lo;
            while (i < mid && j < hi) {
                /* take from the right run only if strictly smaller: stability */
                if (merged_coord(m, a[j]) < merged_coord(m, a[i])) tmp[k++] = a[j++];
                else tmp[k++] = a[i++];
            }
            while (i < mid) tmp[k++] = a[i++];
            while (j < hi) tmp[k++] = a[j++];
        }
        memcpy(a, tmp, (size_t)n * sizeof(int64_t));
    }
}

/* Sorted merged permutation (bit-exact reference for the GPU sort).
 * Returns 0, or -1 if a coordinate is NaN or infinite, -2 on allocation failure. */
int o3_sort_merged(const double* x, int64_t M, const double* y, int64_t N, int64_t* perm) {
    int64_t P = M + N;
    merged_t m = {x, y, N};
    for (int64_t q = 0; q < P; ++q) {
        if (!isfinite(merged_coord(&m, q))) return -1;
        perm[q] = q;
    }
    int64_t* tmp = (int64_t*)malloc((size_t)(P > 0 ? P : 1) * sizeof(int64_t));
    if (!tmp) return -2;
    merge_sort(perm, tmp, P, &m);
    free(tmp);
    return 0;
}

/* O3: sort, forward pass (eq. 4.5), backward pass (eq. 4.6), evaluation (eq. 4.1),
 * unpermute.  exact_self != 0 adds (1 - S_n(0)) alpha_j for every source that shares
 * the coordinate of a target, so that coincident pairs get G(0) = 1 instead of S_n(0).
 * perm_out (may be NULL) receives the sorted merged order.  Returns 0 or the error of
 * o3_sort_merged. */
int o3_recurrence(const double* x, int64_t M, const double* y, const double* alpha, int64_t N,
                  double delta, int n_e, const double* tre, const double* tim, const double* wre,
                  const double* wim, int exact_self, double* u, int64_t* perm_out) {
    int64_t P = M + N;
    if (n_e < 1 || n_e > ORACLE_MAX_TERMS) return -3;
    int64_t* perm = perm_out ? perm_out : (int64_t*)malloc((size_t)(P > 0 ? P : 1) * sizeof(int64_t));
    if (!perm) return -2;
    int rc = o3_sort_merged(x, M, y, N, perm);
    if (rc) {
        if (!perm_out) free(perm);
        return rc;
    }
    merged_t m = {x, y, N};
    const double sd = sqrt(delta);
    double* hre = (double*)calloc((size_t)(M > 0 ? M : 1) * n_e, sizeof(double)); /* h^+ at targets */
    double* him = (double*)calloc((size_t)(M > 0 ? M : 1) * n_e, sizeof(double));
    if (!hre || !him) { free(hre); free(him); if (!perm_out) free(perm); return -2; }
    double Fr[ORACLE_MAX_TERMS], Fi[ORACLE_MAX_TERMS];
    for (int k = 0; k < n_e; ++k) Fr[k] = Fi[k] = 0.0;
    /* forward: h^+_p = e^{-t_k (z_p - z_{p-1}) / sqrt(delta)} h^+_{p-1} + alpha_p [source] */
    for (int64_t p = 0; p < P; ++p) {
        int64_t q = perm[p];
        double z = merged_coord(&m, q);
        if (p > 0) {
            double gap = z - merged_coord(&m, perm[p - 1]);
            for (int k = 0; k < n_e; ++k) {
                double mag = exp(-tre[k] * gap / sd), ang = tim[k] * gap / sd;
                double er = mag * cos(ang), ei = -mag * sin(ang);
                double nr = er * Fr[k] - ei * Fi[k], ni = er * Fi[k] + ei * Fr[k];
                Fr[k] = nr; Fi[k] = ni;
            }
        }
        if (q < N) {
            for (int k = 0; k < n_e; ++k) Fr[k] += alpha[q];
        } else {
            int64_t i = q - N;
            for (int k = 0; k < n_e; ++k) { hre[i * n_e + k] = Fr[k]; him[i * n_e + k] = Fi[k]; }
        }
    }
    /* backward: h^-_p = e^{-t_k (z_{p+1} - z_p) / sqrt(delta)} (h^-_{p+1} + alpha_{p+1} [source]) */
    double Br[ORACLE_MAX_TERMS], Bi[ORACLE_MAX_TERMS];
    for (int k = 0; k < n_e; ++k) Br[k] = Bi[k] = 0.0;
    double s0 = 0.0;
    for (int k = 0; k < n_e; ++k) s0 += wre[k];
    for (int64_t p = P - 1; p >= 0; --p) {
        int64_t q = perm[p];
        if (q >= N) {
            int64_t i = q - N;
            double acc = 0.0;
            for (int k = 0; k < n_e; ++k)
                acc += wre[k] * (hre[i * n_e + k] + Br[k]) - wim[k] * (him[i * n_e + k] + Bi[k]);
            if (exact_self) {
                /* sources that share this coordinate sit just before the target run */
                double zi = x[i], same = 0.0;
                for (int64_t r = p - 1; r >= 0 && merged_coord(&m, perm[r]) == zi; --r)
                    if (perm[r] < N) same += alpha[perm[r]];
                acc += (1.0 - s0) * same;
            }
            u[i] = acc;
        } else {
            for (int k = 0; k < n_e; ++k) Br[k] += alpha[q];
        }
        if (p > 0) {
            double gap = merged_coord(&m, q) - merged_coord(&m, perm[p - 1]);
            for (int k = 0; k < n_e; ++k) {
                double mag = exp(-tre[k] * gap / sd), ang = tim[k] * gap / sd;
                double er = mag * cos(ang), ei = -mag * sin(ang);
                double nr = er * Br[k] - ei * Bi[k], ni = er * Bi[k] + ei * Br[k];
                Br[k] = nr; Bi[k] = ni;
            }
        }
    }
    free(hre); free(him);
    if (!perm_out) free(perm);
    return 0;
}

/* O3 for identical targets and sources (Fig. 4.1): sort the N points once (stable),
 * forward pass h+_i = beta_i + e_{i-1} h+_{i-1} (inclusive), backward pass
 * h-_i = e_i (beta_{i+1} + h-_{i+1}) (exclusive), u = Re sum_k W_k (h+ + h-), unpermute;
 * beta is alpha in sorted order and e_i = exp(-t_k (x_{i+1} - x_i) / sqrt(delta)) for
 * consecutive sorted points.  exact_self != 0 adds (1 - S_n(0)) times the strengths of
 * all points at x_i (the point itself included), so that the self pair and every
 * coincident pair get G(0) = 1 instead of S_n(0).  Returns 0 or the error of
 * o3_sort_merged. */
int o3_recurrence_self(const double* x, const double* alpha, int64_t N, double delta, int n_e, const double* tre,
                       const double* tim, const double* wre, const double* wim, int exact_self, double* u) {
    if (n_e < 1 || n_e > ORACLE_MAX_TERMS) return -3;
    int64_t* perm = (int64_t*)malloc((size_t)(N > 0 ? N : 1) * sizeof(int64_t));
    double* hre = (double*)calloc((size_t)(N > 0 ? N : 1) * n_e, sizeof(double));
    double* him = (double*)calloc((size_t)(N > 0 ? N : 1) * n_e, sizeof(double));
    if (!perm || !hre || !him) { free(perm); free(hre); free(him); return -2; }
    int rc = o3_sort_merged(NULL, 0, x, N, perm); /* the points as sources only */
    if (rc) { free(perm); free(hre); free(him); return rc; }
    const double sd = sqrt(delta);
    double Fr[ORACLE_MAX_TERMS], Fi[ORACLE_MAX_TERMS];
    for (int64_t i = 0; i < N; ++i) {
        for (int k = 0; k < n_e; ++k) {
            double nr = 0.0, ni = 0.0;
            if (i > 0) {
                double gap = x[perm[i]] - x[perm[i - 1]];
                double mag = exp(-tre[k] * gap / sd), ang = tim[k] * gap / sd;
                double er = mag * cos(ang), ei = -mag * sin(ang);
                nr = er * Fr[k] - ei * Fi[k];
                ni = er * Fi[k] + ei * Fr[k];
            }
            Fr[k] = nr + alpha[perm[i]];
            Fi[k] = ni;
            hre[i * n_e + k] = Fr[k];
            him[i * n_e + k] = Fi[k];
        }
    }
    double Br[ORACLE_MAX_TERMS], Bi[ORACLE_MAX_TERMS];
    for (int k = 0; k < n_e; ++k) Br[k] = Bi[k] = 0.0;
    for (int64_t i = N - 1; i >= 0; --i) {
        if (i < N - 1) {
            double gap = x[perm[i + 1]] - x[perm[i]];
            for (int k = 0; k < n_e; ++k) {
                double mag = exp(-tre[k] * gap / sd), ang = tim[k] * gap / sd;
                double er = mag * cos(ang), ei = -mag * sin(ang);
                double cr = Br[k] + alpha[perm[i + 1]], ci = Bi[k];
                Br[k] = er * cr - ei * ci;
                Bi[k] = er * ci + ei * cr;
            }
        }
        double acc = 0.0;
        for (int k = 0; k < n_e; ++k)
            acc += wre[k] * (hre[i * n_e + k] + Br[k]) - wim[k] * (him[i * n_e + k] + Bi[k]);
        if (exact_self) {
            /* the run of equal coordinates around sorted position i, both directions */
            double zi = x[perm[i]], same = alpha[perm[i]], s0 = 0.0;
            for (int64_t r = i - 1; r >= 0 && x[perm[r]] == zi; --r) same += alpha[perm[r]];
            for (int64_t r = i + 1; r < N && x[perm[r]] == zi; ++r) same += alpha[perm[r]];
            for (int k = 0; k < n_e; ++k) s0 += wre[k];
            acc += (1.0 - s0) * same;
        }
        u[perm[i]] = acc;
    }
    free(perm); free(hre); free(him);
    return 0;
}

/* ---- O3 on several host cores -----------------------------------------------------------
 * The same algorithm split over coordinate segments, for the multi-core CPU baseline and
 * for checking the GPU element by element at full size in seconds.
 *
 * Sort: the merged points as (coordinate, merged index) records; T contiguous chunks of
 * the merged order are sorted in parallel by a stable merge sort, then adjacent sorted
 * runs are merged pairwise (left run first on equal coordinates), so the order is the
 * stable one of o3_sort_merged, bit for bit.
 *
 * Recurrences: eqs. 4.5-4.6 are affine in the state, so a segment [b, e) of the sorted
 * points can be swept with zero state entering it and corrected afterwards.  Pass 1
 * (parallel over segments) gives each segment's forward aggregate at its last point and
 * its backward aggregate at its first point (that point's own strength included).
 * The carries are then composed in order, each step multiplying by the exponential of a
 * span computed directly from two FP64 coordinates (no product over points).  Pass 2
 * (parallel over segments) sweeps each segment again from its true entering state,
 * as o3_recurrence does, and evaluates eq. 4.1 at its targets. */

typedef struct {
    double z;
    int64_t q;
} zrec_t;

/* stable merge of sorted runs a[0, na) and b[0, nb) into out: a first on ties */
static void merge_runs(const zrec_t* a, int64_t na, const zrec_t* b, int64_t nb, zrec_t* out) {
    int64_t i = 0, j = 0, k = 0;
    while (i < na && j < nb) {
        if (b[j].z < a[i].z) out[k++] = b[j++];
        else out[k++] = a[i++];
    }
    while (i < na) out[k++] = a[i++];
    while (j < nb) out[k++] = b[j++];
}

static void merge_sort_rec(zrec_t* a, zrec_t* tmp, int64_t n) {
    for (int64_t width = 1; width < n; width *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * width) {
            int64_t mid = lo + width < n ? lo + width : n;
            int64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            merge_runs(a + lo, mid - lo, a + mid, hi - mid, tmp + lo);
        }
        memcpy(a, tmp, (size_t)n * sizeof(zrec_t));
    }
}

/* Sorted records of the merged points with nthreads threads (0: OpenMP default).
 * Returns 0, -1 for a NaN or infinite coordinate, -2 on allocation failure. */
static int sort_records_par(const double* x, int64_t M, const double* y, int64_t N, zrec_t* r, int nthreads) {
    const int64_t P = M + N;
    int bad = 0;
    for (int64_t q = 0; q < P; ++q) {
        r[q].z = q < N ? y[q] : x[q - N];
        r[q].q = q;
        if (!isfinite(r[q].z)) bad = 1;
    }
    if (bad) return -1;
    if (P < 2) return 0;
    zrec_t* tmp = (zrec_t*)malloc((size_t)P * sizeof(zrec_t));
    if (!tmp) return -2;
    int T = 1;
#ifdef _OPENMP
    T = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
    int64_t nch = 1;
    while (nch < T && nch * 2 <= P) nch *= 2; /* a power of two, for the pairwise rounds */
    const int64_t len = (P + nch - 1) / nch;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(T)
#endif
    for (int64_t c = 0; c < nch; ++c) {
        int64_t lo = c * len, hi = lo + len < P ? lo + len : P;
        if (lo < hi) merge_sort_rec(r + lo, tmp + lo, hi - lo);
    }
    zrec_t *src = r, *dst = tmp;
    for (int64_t w = len; w < P; w *= 2) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(T)
#endif
        for (int64_t lo = 0; lo < P; lo += 2 * w) {
            int64_t mid = lo + w < P ? lo + w : P;
            int64_t hi = lo + 2 * w < P ? lo + 2 * w : P;
            merge_runs(src + lo, mid - lo, src + mid, hi - mid, dst + lo);
        }
        zrec_t* t = src;
        src = dst;
        dst = t;
    }
    if (src != r) memcpy(r, src, (size_t)P * sizeof(zrec_t));
    free(tmp);
    return 0;
}

/* The stable merged order of o3_sort_merged, computed on several threads. */
int o3_sort_merged_par(const double* x, int64_t M, const double* y, int64_t N, int64_t* perm, int nthreads) {
    const int64_t P = M + N;
    zrec_t* r = (zrec_t*)malloc((size_t)(P > 0 ? P : 1) * sizeof(zrec_t));
    if (!r) return -2;
    int rc = sort_records_par(x, M, y, N, r, nthreads);
    if (rc == 0)
        for (int64_t p = 0; p < P; ++p) perm[p] = r[p].q;
    free(r);
    return rc;
}

/* e^{-tau_k d / sqrt(delta)} for a coordinate distance d >= 0 */
static inline void decay(double tre, double tim, double d, double sd, double* er, double* ei) {
    double mag = exp(-tre * d / sd), ang = tim * d / sd;
    *er = mag * cos(ang);
    *ei = -mag * sin(ang);
}

/* O3 over nseg coordinate segments on nthreads threads (0: OpenMP default); exact_self
 * as in o3_recurrence.  perm_out (may be NULL) receives the sorted merged order.
 * Returns 0, or -1 (NaN/Inf coordinate), -2 (allocation), -3 (bad n_e). */
int o3_recurrence_par(const double* x, int64_t M, const double* y, const double* alpha, int64_t N,
                      double delta, int n_e, const double* tre, const double* tim, const double* wre,
                      const double* wim, int exact_self, int nseg, int nthreads, double* u, int64_t* perm_out) {
    const int64_t P = M + N;
    if (n_e < 1 || n_e > ORACLE_MAX_TERMS) return -3;
    if (M == 0) return 0;
    if (nseg < 1) nseg = 1;
    if (nseg > P) nseg = (int)P;
    int T = 1;
#ifdef _OPENMP
    T = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
    zrec_t* r = (zrec_t*)malloc((size_t)P * sizeof(zrec_t));
    /* per segment: forward aggregate (last point) and backward aggregate (first point),
     * then the composed carries */
    double* agg = (double*)calloc((size_t)nseg * n_e * 4, sizeof(double));
    double* car = (double*)calloc((size_t)nseg * n_e * 4, sizeof(double));
    if (!r || !agg || !car) { free(r); free(agg); free(car); return -2; }
    int rc = sort_records_par(x, M, y, N, r, nthreads);
    if (rc) { free(r); free(agg); free(car); return rc; }
    if (perm_out)
        for (int64_t p = 0; p < P; ++p) perm_out[p] = r[p].q;
    const double sd = sqrt(delta);
    double s0 = 0.0;
    for (int k = 0; k < n_e; ++k) s0 += wre[k];
#define SEG_LO(g) ((int64_t)(((__int128)P * (g)) / nseg))
    /* pass 1: aggregates with zero entering state */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(T)
#endif
    for (int g = 0; g < nseg; ++g) {
        const int64_t b = SEG_LO(g), e = SEG_LO(g + 1);
        for (int k = 0; k < n_e; ++k) {
            double Fr = 0.0, Fi = 0.0, Br = 0.0, Bi = 0.0, er, ei, t;
            for (int64_t p = b; p < e; ++p) {
                if (p > b) {
                    decay(tre[k], tim[k], r[p].z - r[p - 1].z, sd, &er, &ei);
                    t = er * Fr - ei * Fi; Fi = er * Fi + ei * Fr; Fr = t;
                }
                if (r[p].q < N) Fr += alpha[r[p].q];
            }
            for (int64_t p = e - 1; p >= b; --p) {
                if (p < e - 1) {
                    decay(tre[k], tim[k], r[p + 1].z - r[p].z, sd, &er, &ei);
                    t = er * Br - ei * Bi; Bi = er * Bi + ei * Br; Br = t;
                }
                if (r[p].q < N) Br += alpha[r[p].q]; /* inclusive of the first point */
            }
            double* a = agg + ((size_t)g * n_e + k) * 4;
            a[0] = Fr; a[1] = Fi; a[2] = Br; a[3] = Bi;
        }
    }
    /* carries: car[g] = forward state at the last point of segment g - 1 and the
     * (inclusive) backward state at the first point of segment g + 1, each composed
     * from the aggregates with direct span exponentials */
    for (int k = 0; k < n_e; ++k) {
        double Fr = 0.0, Fi = 0.0, er, ei, t;
        for (int g = 0; g < nseg; ++g) {
            double* c = car + ((size_t)g * n_e + k) * 4;
            c[0] = Fr; c[1] = Fi;
            const double* a = agg + ((size_t)g * n_e + k) * 4;
            if (g > 0) {
                decay(tre[k], tim[k], r[SEG_LO(g + 1) - 1].z - r[SEG_LO(g) - 1].z, sd, &er, &ei);
                t = er * Fr - ei * Fi; Fi = er * Fi + ei * Fr; Fr = t;
            }
            Fr += a[0]; Fi += a[1];
        }
        double Br = 0.0, Bi = 0.0;
        for (int g = nseg - 1; g >= 0; --g) {
            double* c = car + ((size_t)g * n_e + k) * 4;
            c[2] = Br; c[3] = Bi;
            const double* a = agg + ((size_t)g * n_e + k) * 4;
            if (g < nseg - 1) {
                decay(tre[k], tim[k], r[SEG_LO(g + 1)].z - r[SEG_LO(g)].z, sd, &er, &ei);
                t = er * Br - ei * Bi; Bi = er * Bi + ei * Br; Br = t;
            }
            Br += a[2]; Bi += a[3];
        }
    }
    /* pass 2: each segment from its true entering states; evaluation at targets */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(T)
#endif
    for (int g = 0; g < nseg; ++g) {
        const int64_t b = SEG_LO(g), e = SEG_LO(g + 1);
        for (int64_t p = b; p < e; ++p)
            if (r[p].q >= N) u[r[p].q - N] = 0.0;
        for (int k = 0; k < n_e; ++k) {
            const double* c = car + ((size_t)g * n_e + k) * 4;
            double Fr = c[0], Fi = c[1], er, ei, t;
            for (int64_t p = b; p < e; ++p) {
                if (p > 0) {
                    decay(tre[k], tim[k], r[p].z - r[p - 1].z, sd, &er, &ei);
                    t = er * Fr - ei * Fi; Fi = er * Fi + ei * Fr; Fr = t;
                }
                if (r[p].q < N) Fr += alpha[r[p].q];
                else u[r[p].q - N] += wre[k] * Fr - wim[k] * Fi;
            }
            /* backward: h-_p = e^{-t (z_{p+1} - z_p)} (h-_{p+1} + alpha_{p+1} [source]);
             * entering the segment's last point from the next segment's inclusive state */
            double Br = 0.0, Bi = 0.0;
            if (e < P) {
                decay(tre[k], tim[k], r[e].z - r[e - 1].z, sd, &er, &ei);
                Br = er * c[2] - ei * c[3];
                Bi = er * c[3] + ei * c[2];
            }
            for (int64_t p = e - 1; p >= b; --p) {
                if (r[p].q >= N) u[r[p].q - N] += wre[k] * Br - wim[k] * Bi;
                if (p > b) {
                    double cr = Br + (r[p].q < N ? alpha[r[p].q] : 0.0), ci = Bi;
                    decay(tre[k], tim[k], r[p].z - r[p - 1].z, sd, &er, &ei);
                    Br = er * cr - ei * ci;
                    Bi = er * ci + ei * cr;
                }
            }
        }
        if (exact_self) {
            /* sources that share a target's coordinate sit just before it (stable order);
             * the run may start in an earlier segment */
            for (int64_t p = b; p < e; ++p) {
                if (r[p].q < N) continue;
                double same = 0.0;
                for (int64_t q = p - 1; q >= 0 && r[q].z == r[p].z; --q)
                    if (r[q].q < N) same += alpha[r[q].q];
                u[r[p].q - N] += (1.0 - s0) * same;
            }
        }
    }
#undef SEG_LO
    free(r); free(agg); free(car);
    return 0;
}

/* ---- segments of a range-partitioned transform (plain definitions) ---------------------
 * A segment holds the targets x[M] and sources y[N] of one coordinate range.  Its
 * boundary record (4 n_e + 2 doubles): F_k = sum_j alpha_j e^{-t_k (z_last - y_j)/sqrt(delta)}
 * (real parts, then imaginary parts), G_k = sum_j alpha_j e^{-t_k (y_j - z_first)/sqrt(delta)}
 * (real, imaginary), z_first, z_last (the smallest and largest coordinate of all its
 * points; NaN when it has none).  Direct O(N n_e) sums: eqs. 4.3-4.4 at the segment's
 * ends. */
void o3_segment_boundary(const double* x, int64_t M, const double* y, const double* alpha, int64_t N,
                         double delta, int n_e, const double* tre, const double* tim, double* out) {
    double zf = NAN, zl = NAN;
    for (int64_t i = 0; i < M; ++i) {
        if (isnan(zf) || x[i] < zf) zf = x[i];
        if (isnan(zl) || x[i] > zl) zl = x[i];
    }
    for (int64_t j = 0; j < N; ++j) {
        if (isnan(zf) || y[j] < zf) zf = y[j];
        if (isnan(zl) || y[j] > zl) zl = y[j];
    }
    const double sd = sqrt(delta);
    for (int k = 0; k < n_e; ++k) {
        double Fr = 0.0, Fi = 0.0, Gr = 0.0, Gi = 0.0, er, ei;
        for (int64_t j = 0; j < N; ++j) {
            decay(tre[k], tim[k], zl - y[j], sd, &er, &ei);
            Fr += alpha[j] * er;
            Fi += alpha[j] * ei;
            decay(tre[k], tim[k], y[j] - zf, sd, &er, &ei);
            Gr += alpha[j] * er;
            Gi += alpha[j] * ei;
        }
        out[k] = Fr; out[n_e + k] = Fi; out[2 * n_e + k] = Gr; out[3 * n_e + k] = Gi;
    }
    out[4 * n_e] = zf;
    out[4 * n_e + 1] = zl;
}

/* u_i += Re sum_k W_k (F_k e^{-t_k (x_i - z_prev)/sqrt(delta)} + G_k e^{-t_k (z_next - x_i)/sqrt(delta)})
 * for a carry record (F, G, z_prev, z_next; a NaN coordinate means no neighbour):
 * the states entering the segment, carried to each target by eqs. 4.5-4.6. */
void o3_carry_apply(const double* x, int64_t M, double delta, int n_e, const double* tre, const double* tim,
                    const double* wre, const double* wim, const double* carry, double* u) {
    const double sd = sqrt(delta), zp = carry[4 * n_e], zn = carry[4 * n_e + 1];
    for (int64_t i = 0; i < M; ++i) {
        double acc = 0.0;
        for (int k = 0; k < n_e; ++k) {
            double er, ei, hr = 0.0, hi = 0.0;
            if (!isnan(zp)) {
                decay(tre[k], tim[k], x[i] - zp, sd, &er, &ei);
                hr += er * carry[k] - ei * carry[n_e + k];
                hi += er * carry[n_e + k] + ei * carry[k];
            }
            if (!isnan(zn)) {
                decay(tre[k], tim[k], zn - x[i], sd, &er, &ei);
                hr += er * carry[2 * n_e + k] - ei * carry[3 * n_e + k];
                hi += er * carry[3 * n_e + k] + ei * carry[2 * n_e + k];
            }
            acc += wre[k] * hr - wim[k] * hi;
        }
        u[i] += acc;
    }
}

/* ---- direct gradients ------------------------------------------------------------------
 * L = sum_i g_i u_i.  For a kernel K(d), d = x_i - y_j:
 *   dL/dalpha_j = sum_i g_i K(d);  dL/dx_i = g_i sum_j alpha_j K'(d);
 *   dL/dy_j = -alpha_j sum_i g_i K'(d);  dL/ddelta = sum_ij g_i alpha_j dK/ddelta.
 * Gaussian: K = e^{-d^2/(4 delta)}, K' = -d/(2 delta) K, dK/ddelta = d^2/(4 delta^2) K.
 * SOE: K = Re sum W_k e^{-tau_k s |d|}, s = delta^{-1/2};
 *   K' = Re sum W_k (-tau_k s sgn d) e^{...} with sgn 0 = 0 (the cusp at d = 0 is given
 *   the symmetric value 0, which is also G'(0));
 *   dK/ddelta = Re sum W_k tau_k |d| s / (2 delta) e^{...}.
 */
void o1_grad(const double* x, int64_t M, const double* y, const double* alpha, int64_t N,
             double delta, const double* g, double* gx, double* gy, double* galpha, double* gdelta) {
    double gd = 0.0;
    for (int64_t j = 0; j < N; ++j) { gy[j] = 0.0; galpha[j] = 0.0; }
    for (int64_t i = 0; i < M; ++i) {
        double sx = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            double d = x[i] - y[j];
            double K = exp(-(d * d) / (4.0 * delta));
            double Kp = -d / (2.0 * delta) * K;
            galpha[j] += g[i] * K;
            sx += alpha[j] * Kp;
            gy[j] -= alpha[j] * g[i] * Kp;
            gd += g[i] * alpha[j] * (d * d) / (4.0 * delta * delta) * K;
        }
        gx[i] = g[i] * sx;
    }
    *gdelta = gd;
}

void o2_grad(const double* x, int64_t M, const double* y, const double* alpha, int64_t N,
             double delta, int n_e, const double* tre, const double* tim, const double* wre,
             const double* wim, const double* g, double* gx, double* gy, double* galpha,
             double* gdelta) {
    const double s = 1.0 / sqrt(delta);
    double gd = 0.0;
    for (int64_t j = 0; j < N; ++j) { gy[j] = 0.0; galpha[j] = 0.0; }
    for (int64_t i = 0; i < M; ++i) {
        double sx = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            double d = x[i] - y[j];
            double r = fabs(d) * s;
            double sg = d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0);
            double K = 0.0, Kp = 0.0, Kd = 0.0;
            for (int k = 0; k < n_e; ++k) {
                double mag = exp(-tre[k] * r);
                double er = mag * cos(tim[k] * r), ei = -mag * sin(tim[k] * r); /* e^{-tau r} */
                double wer = wre[k] * er - wim[k] * ei, wei = wre[k] * ei + wim[k] * er; /* W e^{-tau r} */
                K += wer;
                /* Re(W tau e^{-tau r}) */
                double wt = wer * tre[k] - wei * tim[k];
                Kp += -s * sg * wt;
                Kd += wt * fabs(d) * s / (2.0 * delta);
            }
            galpha[j] += g[i] * K;
            sx += alpha[j] * Kp;
            gy[j] -= alpha[j] * g[i] * Kp;
            gd += g[i] * alpha[j] * Kd;
        }
        gx[i] = g[i] * sx;
    }
    *gdelta = gd;
}
