/*
 * FP64 CPU oracle for the seismic saliency method (Shafiq, Long, Di, AlRegib,
 * "A novel attention model for salient structure detection in seismic volumes").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's CPU
 * baseline leg load this library.  It shares no code with the CUDA path.
 *
 * Each routine is the plain definition from the paper, written out voxel by voxel
 * in double precision, with no blocking, fusion or reordering:
 *   - local spectrum of an n x n x n cube around a voxel: Sec. 2 step 1 and
 *     Eq. 2 (separable DFT K = D_t (x) D_x (x) D_y applied to the cube C_n);
 *   - spectral projection F_m = F * P_m / sqrt(i^2+j^2+k^2): Eq. 1, with the
 *     zero-frequency bin left out (Sec. 2, text after Eq. 2);
 *   - feature E_m = mean over the cube's bins of |F_m| (Sec. 2 step 3), or, as the alternative
 *     reading of that garbled step, the mean of |F_m|^2 (the projected spectral energy);
 *   - directional center-surround S_m (Eq. 3);
 *   - sequential LMS / NLMS / RLS weight adaptation (Sec. 2, text around Eq. 4);
 *   - the analytic adjoints of the feature and center-surround steps (used to
 *     check gradients; the paper itself has no backward pass).
 *
 * Readings of points the paper leaves open (all configurable by argument):
 *   window offsets u in [-n/2, n/2-1] per axis around the voxel (stride 1);
 *   signed bin index i = k for k < n/2, else k - n;  i <-> f_t, j <-> f_x, k <-> f_y;
 *   E_m = (1/n^3) * sum over bins k != 0 of r_m(k) |F[k]|  (feature 0), or
 *   E_m = (1/n^3) * sum over bins k != 0 of r_m(k)^2 |F[k]|^2  (feature 1, energy);
 *   borders: symmetric (edge sample repeated), periodic or zero extension.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum { BND_SYMMETRIC = 0, BND_PERIODIC = 1, BND_ZERO = 2 };

/* Relative magnitude (to the window L1 norm) at or below which a bin is treated as F = 0 in the
   adjoint: 2^-40.  The reason is FP64 arithmetic alone: a bin that is exactly zero (a mirror-
   symmetric or aliased window under the border extension) comes out of the FP64 DFT of this file
   at no more than about 3n 2^-53 times the L1 norm (three one-axis sums of n terms each, twiddles
   rounded to 2^-53), below 2^-45 for n <= 32, while |F| / L1 of a bin that is not zero is whatever
   the data make it.  So the band only catches zeros of the
   mathematics, where the subgradient of |F| is taken as 0. */
#define KINK_TAU (1.0 / 1099511627776.0)

/* Boundary extension of one axis.  Returns -1 where the zero extension applies. */
static long ext_index(long i, long N, int mode) {
    if (i >= 0 && i < N) return i;
    if (mode == BND_PERIODIC) {
        long r = i % N;
        return r < 0 ? r + N : r;
    }
    if (mode == BND_ZERO) return -1;
    /* symmetric with the edge sample repeated: -1 -> 0, -2 -> 1, N -> N-1 */
    long P = 2 * N;
    long r = i % P;
    if (r < 0) r += P;
    return r < N ? r : P - 1 - r;
}

static long ext_flat(long t, long x, long y, long T, long X, long Y, int mode) {
    long a = ext_index(t, T, mode), b = ext_index(x, X, mode), c = ext_index(y, Y, mode);
    if (a < 0 || b < 0 || c < 0) return -1;
    return (a * X + b) * Y + c;
}

static int signed_bin(int k, int n) { return k < n / 2 ? k : k - n; }

static double taper_1d(int u, int n, int taper) {
    if (taper == 0) return 1.0;                      /* rectangular: the cube as is */
    return 0.5 - 0.5 * cos(2.0 * M_PI * u / n);      /* periodic Hann (option) */
}

/* Projection ratio r_m(k) = P_m / sqrt(i^2+j^2+k^2) of Eq. 1 for m = 0 (t), 1 (x), 2 (y). */
static double proj_ratio(int m, int i, int j, int k) {
    double r2 = (double)i * i + (double)j * j + (double)k * k;
    double p2 = (m == 0) ? (double)j * j + (double)k * k
              : (m == 1) ? (double)i * i + (double)k * k
                         : (double)i * i + (double)j * j;
    return sqrt(p2) / sqrt(r2);
}

typedef struct {
    int n;
    double *w, *a1re, *a1im, *a2re, *a2im, *fre, *fim;
    double *cs, *sn; /* cos, sin of 2 pi m / n */
} work_t;

static int work_init(work_t* W, int n) {
    size_t n3 = (size_t)n * n * n;
    W->n = n;
    W->w = malloc(n3 * sizeof(double));
    W->a1re = malloc(n3 * sizeof(double));
    W->a1im = malloc(n3 * sizeof(double));
    W->a2re = malloc(n3 * sizeof(double));
    W->a2im = malloc(n3 * sizeof(double));
    W->fre = malloc(n3 * sizeof(double));
    W->fim = malloc(n3 * sizeof(double));
    W->cs = malloc(n * sizeof(double));
    W->sn = malloc(n * sizeof(double));
    if (!W->w || !W->a1re || !W->a1im || !W->a2re || !W->a2im || !W->fre || !W->fim || !W->cs || !W->sn)
        return -1;
    for (int m = 0; m < n; ++m) {
        W->cs[m] = cos(2.0 * M_PI * m / n);
        W->sn[m] = sin(2.0 * M_PI * m / n);
    }
    return 0;
}

static void work_free(work_t* W) {
    free(W->w); free(W->a1re); free(W->a1im); free(W->a2re); free(W->a2im);
    free(W->fre); free(W->fim); free(W->cs); free(W->sn);
}

#define IDX3(a, b, c, n) (((size_t)(a) * (n) + (b)) * (n) + (c))

/*
 * Local spectrum of the cube around voxel (t,x,y):
 *   F[k] = sum_u h(u) Vext[t+u_t-n/2, x+u_x-n/2, y+u_y-n/2] exp(-2 pi i k.u / n),
 * u, k in [0,n)^3, computed as three one-axis DFTs (Eq. 2).  Result in W->fre/fim,
 * indexed [k_t][k_x][k_y].
 */
static void local_spectrum(const double* V, long T, long X, long Y, int n, int mode, int taper,
                           long t, long x, long y, work_t* W) {
    const int h2 = n / 2;
    for (int ut = 0; ut < n; ++ut)
        for (int ux = 0; ux < n; ++ux)
            for (int uy = 0; uy < n; ++uy) {
                long q = ext_flat(t + ut - h2, x + ux - h2, y + uy - h2, T, X, Y, mode);
                double v = q < 0 ? 0.0 : V[q];
                W->w[IDX3(ut, ux, uy, n)] =
                    v * taper_1d(ut, n, taper) * taper_1d(ux, n, taper) * taper_1d(uy, n, taper);
            }
    /* DFT along t */
    for (int kt = 0; kt < n; ++kt)
        for (int ux = 0; ux < n; ++ux)
            for (int uy = 0; uy < n; ++uy) {
                double re = 0.0, im = 0.0;
                for (int ut = 0; ut < n; ++ut) {
                    int m = (kt * ut) % n;
                    double v = W->w[IDX3(ut, ux, uy, n)];
                    re += v * W->cs[m];
                    im -= v * W->sn[m];
                }
                W->a1re[IDX3(kt, ux, uy, n)] = re;
                W->a1im[IDX3(kt, ux, uy, n)] = im;
            }
    /* DFT along x */
    for (int kt = 0; kt < n; ++kt)
        for (int kx = 0; kx < n; ++kx)
            for (int uy = 0; uy < n; ++uy) {
                double re = 0.0, im = 0.0;
                for (int ux = 0; ux < n; ++ux) {
                    int m = (kx * ux) % n;
                    double ar = W->a1re[IDX3(kt, ux, uy, n)], ai = W->a1im[IDX3(kt, ux, uy, n)];
                    /* (ar + i ai)(cos - i sin) */
                    re += ar * W->cs[m] + ai * W->sn[m];
                    im += ai * W->cs[m] - ar * W->sn[m];
                }
                W->a2re[IDX3(kt, kx, uy, n)] = re;
                W->a2im[IDX3(kt, kx, uy, n)] = im;
            }
    /* DFT along y */
    for (int kt = 0; kt < n; ++kt)
        for (int kx = 0; kx < n; ++kx)
            for (int ky = 0; ky < n; ++ky) {
                double re = 0.0, im = 0.0;
                for (int uy = 0; uy < n; ++uy) {
                    int m = (ky * uy) % n;
                    double ar = W->a2re[IDX3(kt, kx, uy, n)], ai = W->a2im[IDX3(kt, kx, uy, n)];
                    re += ar * W->cs[m] + ai * W->sn[m];
                    im += ai * W->cs[m] - ar * W->sn[m];
                }
                W->fre[IDX3(kt, kx, ky, n)] = re;
                W->fim[IDX3(kt, kx, ky, n)] = im;
            }
}

/* Step 2 + 3: E_m = (1/n^3) sum_{k != 0} |F_m[k]| with F_m = r_m F (Eq. 1, DC excluded); with
   feature 1 the squared magnitude |F_m[k]|^2 = r_m(k)^2 |F[k]|^2 is averaged instead. */
static void features_from_spectrum(const work_t* W, int feature, double E[3]) {
    const int n = W->n;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int kt = 0; kt < n; ++kt)
        for (int kx = 0; kx < n; ++kx)
            for (int ky = 0; ky < n; ++ky) {
                if (kt == 0 && kx == 0 && ky == 0) continue;
                int i = signed_bin(kt, n), j = signed_bin(kx, n), k = signed_bin(ky, n);
                size_t b = IDX3(kt, kx, ky, n);
                double mag2 = W->fre[b] * W->fre[b] + W->fim[b] * W->fim[b];
                for (int m = 0; m < 3; ++m) {
                    double r = proj_ratio(m, i, j, k);
                    acc[m] += feature == 1 ? r * r * mag2 : r * sqrt(mag2);
                }
            }
    double inv = 1.0 / ((double)n * n * n);
    for (int m = 0; m < 3; ++m) E[m] = acc[m] * inv;
}

static int check_common(long T, long X, long Y, int n, int mode) {
    if (T <= 0 || X <= 0 || Y <= 0) return -1;
    if (n < 2 || (n & 1)) return -2;
    if (mode < 0 || mode > 2) return -3;
    return 0;
}

/* One voxel's full local spectrum F (interleaved re,im; [k_t][k_x][k_y][2]). */
int sal_oracle_local_spectrum(const double* V, long T, long X, long Y, int n, int mode, int taper,
                              long t, long x, long y, double* F) {
    int rc = check_common(T, X, Y, n, mode);
    if (rc) return rc;
    work_t W;
    if (work_init(&W, n)) { work_free(&W); return -4; }
    local_spectrum(V, T, X, Y, n, mode, taper, t, x, y, &W);
    size_t n3 = (size_t)n * n * n;
    for (size_t b = 0; b < n3; ++b) { F[2 * b] = W.fre[b]; F[2 * b + 1] = W.fim[b]; }
    work_free(&W);
    return 0;
}

/* One voxel's projected spectra F_m of Eq. 1 ([3][k_t][k_x][k_y][2]; DC set to 0). */
int sal_oracle_projected_spectra(const double* V, long T, long X, long Y, int n, int mode, int taper,
                                 long t, long x, long y, double* Fm) {
    int rc = check_common(T, X, Y, n, mode);
    if (rc) return rc;
    work_t W;
    if (work_init(&W, n)) { work_free(&W); return -4; }
    local_spectrum(V, T, X, Y, n, mode, taper, t, x, y, &W);
    size_t n3 = (size_t)n * n * n;
    for (int m = 0; m < 3; ++m)
        for (int kt = 0; kt < n; ++kt)
            for (int kx = 0; kx < n; ++kx)
                for (int ky = 0; ky < n; ++ky) {
                    size_t b = IDX3(kt, kx, ky, n);
                    double r = 0.0;
                    if (kt || kx || ky) r = proj_ratio(m, signed_bin(kt, n), signed_bin(kx, n), signed_bin(ky, n));
                    Fm[2 * (m * n3 + b)] = W.fre[b] * r;
                    Fm[2 * (m * n3 + b) + 1] = W.fim[b] * r;
                }
    work_free(&W);
    return 0;
}

/* Features E [3][T][X][Y] of every voxel. */
int sal_oracle_features(const double* V, long T, long X, long Y, int n, int mode, int taper, int feature,
                        double* E, int nthreads) {
    int rc = check_common(T, X, Y, n, mode);
    if (rc) return rc;
    if (feature < 0 || feature > 1) return -5;
    const long N = T * X * Y;
    int fail = 0;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
    {
        work_t W;
        int ok = work_init(&W, n) == 0;
        if (!ok) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(static)
        for (long p = 0; p < N; ++p) {
            if (!ok) continue;
            long t = p / (X * Y), x = (p / Y) % X, y = p % Y;
            double e[3];
            local_spectrum(V, T, X, Y, n, mode, taper, t, x, y, &W);
            features_from_spectrum(&W, feature, e);
            for (int m = 0; m < 3; ++m) E[m * N + p] = e[m];
        }
        work_free(&W);
    }
    return fail ? -4 : 0;
}

/* Features at listed voxels: pts [count][3] (t,x,y) -> Eout [count][3]. */
int sal_oracle_features_at(const double* V, long T, long X, long Y, int n, int mode, int taper, int feature,
                           const int64_t* pts, long count, double* Eout, int nthreads) {
    int rc = check_common(T, X, Y, n, mode);
    if (rc) return rc;
    if (feature < 0 || feature > 1) return -5;
    int fail = 0;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
    {
        work_t W;
        int ok = work_init(&W, n) == 0;
        if (!ok) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 4)
        for (long s = 0; s < count; ++s) {
            if (!ok) continue;
            local_spectrum(V, T, X, Y, n, mode, taper, pts[3 * s], pts[3 * s + 1], pts[3 * s + 2], &W);
            features_from_spectrum(&W, feature, &Eout[3 * s]);
        }
        work_free(&W);
    }
    return fail ? -4 : 0;
}

/*
 * Conditioning of the |F| adjoint (test helper, no step of the method): for every voxel p, the
 * number of non-DC bins of its cube whose magnitude lies in (lo * L1, hi * L1], L1 = sum_u
 * |h(u) Vext[p+u-n/2]|.  The direction F / |F| that the adjoint of step 3 needs is ill-conditioned
 * for small |F|: an arithmetic with unit rounding e computes it with an error of about
 * e L1 / |F|, so windows holding such bins bound the agreement any lower precision can reach.
 * counts [T][X][Y] is overwritten.
 */
int sal_oracle_band_count(const double* V, long T, long X, long Y, int n, int mode, int taper,
                          double lo, double hi, int32_t* counts, int nthreads) {
    int rc = check_common(T, X, Y, n, mode);
    if (rc) return rc;
    const long N = T * X * Y;
    const size_t n3 = (size_t)n * n * n;
    int fail = 0;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
    {
        work_t W;
        int ok = work_init(&W, n) == 0;
        if (!ok) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(static)
        for (long p = 0; p < N; ++p) {
            if (!ok) continue;
            long t = p / (X * Y), x = (p / Y) % X, y = p % Y;
            local_spectrum(V, T, X, Y, n, mode, taper, t, x, y, &W);
            double l1 = 0.0;
            for (size_t b = 0; b < n3; ++b) l1 += fabs(W.w[b]);
            int c = 0;
            for (size_t b = 1; b < n3; ++b) {
                double mag = sqrt(W.fre[b] * W.fre[b] + W.fim[b] * W.fim[b]);
                if (mag > lo * l1 && mag <= hi * l1) ++c;
            }
            counts[p] = c;
        }
        work_free(&W);
    }
    return fail ? -4 : 0;
}

/*
 * Directional center-surround, Eq. 3:
 *   S_m[p] = (1/Q) sum_{o} | E_m[p] - w_o * Eext_m[p + o] |,   Q = number of offsets.
 * E, S: [3][T][X][Y]; off [Q][3] (dt,dx,dy); w [Q].
 */
int sal_oracle_center_surround(const double* E, long T, long X, long Y, int mode, int Q,
                               const int* off, const double* w, double* S, int nthreads) {
    if (T <= 0 || X <= 0 || Y <= 0 || Q <= 0 || mode < 0 || mode > 2) return -1;
    const long N = T * X * Y;
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
    for (long p = 0; p < N; ++p) {
        long t = p / (X * Y), x = (p / Y) % X, y = p % Y;
        for (int m = 0; m < 3; ++m) {
            const double* Em = E + m * N;
            double acc = 0.0;
            for (int o = 0; o < Q; ++o) {
                long q = ext_flat(t + off[3 * o], x + off[3 * o + 1], y + off[3 * o + 2], T, X, Y, mode);
                double nb = q < 0 ? 0.0 : Em[q];
                acc += fabs(Em[p] - w[o] * nb);
            }
            S[m * N + p] = acc / Q;
        }
    }
    return 0;
}

/*
 * Adjoint of Eq. 3 (weights w_o and E both variables).  With d = E[p] - w_o Eext[p+o]
 * and sgn(0) = 0:  gE[p] += sgn(d) gS[p] / Q;  gE[ext(p+o)] -= sgn(d) gS[p] w_o / Q;
 * gw[o] -= sgn(d) gS[p] Eext[p+o] / Q.  gE [3][T][X][Y] and gw [Q] are overwritten.
 */
int sal_oracle_center_surround_adjoint(const double* E, long T, long X, long Y, int mode, int Q,
                                       const int* off, const double* w, const double* gS,
                                       double* gE, double* gw) {
    if (T <= 0 || X <= 0 || Y <= 0 || Q <= 0 || mode < 0 || mode > 2) return -1;
    const long N = T * X * Y;
    memset(gE, 0, 3 * N * sizeof(double));
    memset(gw, 0, Q * sizeof(double));
    for (int m = 0; m < 3; ++m) {
        const double* Em = E + m * N;
        double* gEm = gE + m * N;
        for (long p = 0; p < N; ++p) {
            long t = p / (X * Y), x = (p / Y) % X, y = p % Y;
            double g = gS[m * N + p] / Q;
            if (g == 0.0) continue;
            for (int o = 0; o < Q; ++o) {
                long q = ext_flat(t + off[3 * o], x + off[3 * o + 1], y + off[3 * o + 2], T, X, Y, mode);
                double nb = q < 0 ? 0.0 : Em[q];
                double d = Em[p] - w[o] * nb;
                double s = d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0);
                gEm[p] += s * g;
                if (q >= 0) gEm[q] -= s * g * w[o];
                gw[o] -= s * g * nb;
            }
        }
    }
    return 0;
}

/*
 * Adjoint of the feature step.  For each voxel p, with F_p recomputed,
 *   U[k] = (1/n^3) (sum_m gE_m[p] r_m(k)) F_p[k] / |F_p[k]|       (feature 0), or
 *   U[k] = (2/n^3) (sum_m gE_m[p] r_m(k)^2) F_p[k]                 (feature 1, energy)
 *   (0 at DC and where |F| <= 2^-40 sum_u |h(u) Vext[p+u-n/2]|, i.e. F = 0 up to FP64 rounding:
 *   the zero subgradient of |F|),
 *   gVext[p + u - n/2] += h(u) Re sum_k U[k] exp(+2 pi i k.u / n),
 * then the extension is folded back onto V (zero extension drops).  gV [T][X][Y] is
 * overwritten.  Per-thread accumulators are summed in thread order.
 */
int sal_oracle_features_adjoint(const double* V, long T, long X, long Y, int n, int mode, int taper, int feature,
                                const double* gE, double* gV, int nthreads) {
    int rc = check_common(T, X, Y, n, mode);
    if (rc) return rc;
    if (feature < 0 || feature > 1) return -5;
    const long N = T * X * Y;
    const int h2 = n / 2;
    const size_t n3 = (size_t)n * n * n;
    int nth = nthreads > 0 ? nthreads : omp_get_max_threads();
    double* acc = calloc((size_t)nth * N, sizeof(double));
    if (!acc) return -4;
    int fail = 0;
#pragma omp parallel num_threads(nth)
    {
        int tid = omp_get_thread_num();
        double* g = acc + (size_t)tid * N;
        work_t W;
        int ok = work_init(&W, n) == 0;
        double *ure = malloc(n3 * sizeof(double)), *uim = malloc(n3 * sizeof(double));
        double *b2re = malloc(n3 * sizeof(double)), *b2im = malloc(n3 * sizeof(double));
        double *b1re = malloc(n3 * sizeof(double)), *b1im = malloc(n3 * sizeof(double));
        if (!ok || !ure || !uim || !b2re || !b2im || !b1re || !b1im) {
            ok = 0;
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(static)
        for (long p = 0; p < N; ++p) {
            if (!ok) continue;
            double ge[3] = {gE[p], gE[N + p], gE[2 * N + p]};
            if (ge[0] == 0.0 && ge[1] == 0.0 && ge[2] == 0.0) continue;
            long t = p / (X * Y), x = (p / Y) % X, y = p % Y;
            local_spectrum(V, T, X, Y, n, mode, taper, t, x, y, &W);
            /* |F| has no direction at F = 0 (a kink): bins whose magnitude is at or below
               KINK_TAU times the window's L1 norm (zero up to the FP64 rounding of the DFT)
               take the zero subgradient. */
            double l1 = 0.0;
            for (size_t b = 0; b < n3; ++b) l1 += fabs(W.w[b]);
            const double thr = KINK_TAU * l1;
            for (int kt = 0; kt < n; ++kt)
                for (int kx = 0; kx < n; ++kx)
                    for (int ky = 0; ky < n; ++ky) {
                        size_t b = IDX3(kt, kx, ky, n);
                        double mag = sqrt(W.fre[b] * W.fre[b] + W.fim[b] * W.fim[b]);
                        ure[b] = uim[b] = 0.0;
                        if (kt == 0 && kx == 0 && ky == 0) continue;
                        int i = signed_bin(kt, n), j = signed_bin(kx, n), k = signed_bin(ky, n);
                        double c = 0.0;
                        if (feature == 1) {
                            /* d |F|^2 / d(Re F, Im F) = 2 (Re F, Im F): smooth, no kink */
                            for (int m = 0; m < 3; ++m) {
                                double r = proj_ratio(m, i, j, k);
                                c += ge[m] * r * r;
                            }
                            c *= 2.0 / (double)n3;
                        } else {
                            if (mag <= thr) continue;
                            for (int m = 0; m < 3; ++m) c += ge[m] * proj_ratio(m, i, j, k);
                            c /= (double)n3 * mag;
                        }
                        ure[b] = c * W.fre[b];
                        uim[b] = c * W.fim[b];
                    }
            /* inverse along y: B2[kt][kx][uy] = sum_ky U exp(+2 pi i ky uy / n) */
            for (int kt = 0; kt < n; ++kt)
                for (int kx = 0; kx < n; ++kx)
                    for (int uy = 0; uy < n; ++uy) {
                        double re = 0.0, im = 0.0;
                        for (int ky = 0; ky < n; ++ky) {
                            int m = (ky * uy) % n;
                            double ar = ure[IDX3(kt, kx, ky, n)], ai = uim[IDX3(kt, kx, ky, n)];
                            re += ar * W.cs[m] - ai * W.sn[m];
                            im += ai * W.cs[m] + ar * W.sn[m];
                        }
                        b2re[IDX3(kt, kx, uy, n)] = re;
                        b2im[IDX3(kt, kx, uy, n)] = im;
                    }
            /* inverse along x */
            for (int kt = 0; kt < n; ++kt)
                for (int ux = 0; ux < n; ++ux)
                    for (int uy = 0; uy < n; ++uy) {
                        double re = 0.0, im = 0.0;
                        for (int kx = 0; kx < n; ++kx) {
                            int m = (kx * ux) % n;
                            double ar = b2re[IDX3(kt, kx, uy, n)], ai = b2im[IDX3(kt, kx, uy, n)];
                            re += ar * W.cs[m] - ai * W.sn[m];
                            im += ai * W.cs[m] + ar * W.sn[m];
                        }
                        b1re[IDX3(kt, ux, uy, n)] = re;
                        b1im[IDX3(kt, ux, uy, n)] = im;
                    }
            /* inverse along t, real part, then scatter through the extension */
            for (int ut = 0; ut < n; ++ut)
                for (int ux = 0; ux < n; ++ux)
                    for (int uy = 0; uy < n; ++uy) {
                        double re = 0.0;
                        for (int kt = 0; kt < n; ++kt) {
                            int m = (kt * ut) % n;
                            re += b1re[IDX3(kt, ux, uy, n)] * W.cs[m] - b1im[IDX3(kt, ux, uy, n)] * W.sn[m];
                        }
                        re *= taper_1d(ut, n, taper) * taper_1d(ux, n, taper) * taper_1d(uy, n, taper);
                        long q = ext_flat(t + ut - h2, x + ux - h2, y + uy - h2, T, X, Y, mode);
                        if (q >= 0) g[q] += re;
                    }
        }
        work_free(&W);
        free(ure); free(uim); free(b2re); free(b2im); free(b1re); free(b1im);
    }
    for (long p = 0; p < N; ++p) {
        double s = 0.0;
        for (int th = 0; th < nth; ++th) s += acc[(size_t)th * N + p];
        gV[p] = s;
    }
    free(acc);
    return fail ? -4 : 0;
}

/*
 * Sequential adaptive filters of Sec. 2 (Eq. 4 and the text after it), one pass over
 * the samples in array order.  x_p = (Xs[0][p], Xs[1][p], Xs[2][p]); desired D[p].
 * e_p = D[p] - W.x_p is the a-priori error; err2 (nullable) receives e_p^2.
 *   LMS:  W += mu e x
 *   NLMS: W += mu e x / (eps + |x|^2)
 *   RLS:  k = P x / (lambda + x'Px);  W += k e;  P = (P - k x'P) / lambda,  P0 = I/delta.
 */
int sal_oracle_lms(const double* Xs, const double* D, long N, double mu, double* W, double* err2) {
    for (long p = 0; p < N; ++p) {
        double x[3] = {Xs[p], Xs[N + p], Xs[2 * N + p]};
        double e = D[p] - (W[0] * x[0] + W[1] * x[1] + W[2] * x[2]);
        if (err2) err2[p] = e * e;
        for (int m = 0; m < 3; ++m) W[m] += mu * e * x[m];
    }
    return 0;
}

int sal_oracle_nlms(const double* Xs, const double* D, long N, double mu, double eps, double* W,
                    double* err2) {
    for (long p = 0; p < N; ++p) {
        double x[3] = {Xs[p], Xs[N + p], Xs[2 * N + p]};
        double e = D[p] - (W[0] * x[0] + W[1] * x[1] + W[2] * x[2]);
        double nx = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
        if (err2) err2[p] = e * e;
        for (int m = 0; m < 3; ++m) W[m] += mu * e * x[m] / (eps + nx);
    }
    return 0;
}

int sal_oracle_rls(const double* Xs, const double* D, long N, double lambda, double delta, double* W,
                   double* err2) {
    double P[3][3] = {{1.0 / delta, 0, 0}, {0, 1.0 / delta, 0}, {0, 0, 1.0 / delta}};
    for (long p = 0; p < N; ++p) {
        double x[3] = {Xs[p], Xs[N + p], Xs[2 * N + p]};
        double Px[3], xP[3];
        for (int a = 0; a < 3; ++a) {
            Px[a] = P[a][0] * x[0] + P[a][1] * x[1] + P[a][2] * x[2];
            xP[a] = x[0] * P[0][a] + x[1] * P[1][a] + x[2] * P[2][a];
        }
        double den = lambda + x[0] * Px[0] + x[1] * Px[1] + x[2] * Px[2];
        double k[3] = {Px[0] / den, Px[1] / den, Px[2] / den};
        double e = D[p] - (W[0] * x[0] + W[1] * x[1] + W[2] * x[2]);
        if (err2) err2[p] = e * e;
        for (int a = 0; a < 3; ++a) W[a] += k[a] * e;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) P[a][b] = (P[a][b] - k[a] * xP[b]) / lambda;
    }
    return 0;
}
