/*
 * sal.h — C ABI of the GB300 (sm_103a) seismic saliency library, libsal.so.
 *
 * Method: Shafiq, Long, Di, AlRegib, "A novel attention model for salient structure
 * detection in seismic volumes" (Applied Computing and Intelligence, 2021).  The
 * paper's problem statement (Sec. 2): given a seismic volume V of size T x X x Y
 * (T time/depth, X crossline, Y inline), compute a saliency map S of the same size
 * by (1) a local 3D DFT of an n^3 cube around every voxel (Eq. 2), (2) a spectral
 * projection of each local spectrum onto the t, x and y dimensions (Eq. 1),
 * (3) per-dimension features E_m, (4) a directional center-surround comparison
 * giving S_m (Eq. 3, Fig. 4) and (5) a weighted combination of S_t, S_x, S_y with
 * equal, given or template-fitted weights (Eq. 4).
 *
 * Conventions for every entry point:
 *   - Volumes are C-contiguous float32 [T][X][Y] (Y fastest).  Stacked maps are
 *     [3][T][X][Y] with the planes in the order t, x, y.
 *   - All data pointers are DEVICE pointers owned by the caller, unless a comment
 *     says otherwise.  The handle owns only its constant tables and scratch.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     stream-ordered and asynchronous: they return after enqueueing the work.
 *   - Every call returns a sal_status.  Argument errors are reported before any
 *     work is enqueued.  Errors found on the device set an error word that the
 *     next call on the handle reports as SAL_ERR_DEVICE_CHECK.  Nothing traps on
 *     the device.  sal_last_error() gives a one-line message for the last error.
 *   - Results are deterministic for a fixed handle configuration: reductions
 *     use fixed-order trees, never floating-point atomics.
 *   - A handle is not thread-safe: calls on one handle must not overlap in time.
 */
#ifndef SAL_H
#define SAL_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sal_handle sal_handle;

typedef enum {
    SAL_OK = 0,
    SAL_ERR_INVALID_ARG = 1,   /* null pointer, bad size, bad parameter          */
    SAL_ERR_UNSUPPORTED = 2,   /* valid but not built (e.g. a window size)        */
    SAL_ERR_OOM = 3,           /* scratch does not fit the HBM budget or device   */
    SAL_ERR_CUDA = 4,          /* a CUDA runtime call or launch failed            */
    SAL_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up              */
    SAL_ERR_DEVICE_CHECK = 6   /* a device-side check set the error word          */
} sal_status;

typedef enum { SAL_FP32 = 0, SAL_BF16 = 1, SAL_FP16 = 2 } sal_precision;

/* Border extension of V (for the DFT cubes) and of E (for the center-surround). */
typedef enum {
    SAL_BND_SYMMETRIC = 0,  /* edge sample repeated: -1 -> 0, -2 -> 1, T -> T-1 */
    SAL_BND_PERIODIC = 1,
    SAL_BND_ZERO = 2
} sal_boundary;

typedef struct {
    int n;                  /* cube side of the local DFT (Sec. 2 step 1, Eq. 2): n in
                               {2,4,8,16,32} for SAL_FP32, {8,16,32} for BF16/FP16; the
                               backward calls are built for n <= 16                      */
    int stride;             /* window stride s: 1 = a cube around every voxel; s > 1 with
                               s < n/2 (windows overlapping by more than half, Sec. 2
                               step 1) = cubes only at voxels whose indices are all
                               multiples of s, E interpolated trilinearly in between
                               (held past the last lattice point of an axis); the
                               backward goes through the interpolation's adjoint and the
                               cubes of the lattice voxels                           */
    int taper;              /* 0 = rectangular (the cube as is), 1 = periodic Hann    */
    int boundary;           /* sal_boundary                                           */
    int feature;            /* 0 = E_m = (1/n^3) sum_{k != 0} r_m(k) |F[k]| (step 3: the mean
                               of |F_m| over the cube's bins); 1 = E_m = (1/n^3) sum_{k != 0}
                               r_m(k)^2 |F[k]|^2 (the mean of |F_m|^2, the energy reading of
                               that garbled step); both forward and backward, all precisions;
                               2 = E_m = (1/n^3) sum_u |f_m[u]|, f_m the inverse DFT of F_m (its
                               spatial-domain reading): FP32, n in {2, 4, 8, 16}, stride 1,
                               forward and backward (other combinations:
                               SAL_ERR_UNSUPPORTED at sal_create)                        */
    /* Directional center-surround window (Eq. 3, Fig. 4): Q = n_offsets neighbours
       o = (dt,dx,dy), |dt|,|dx|,|dy| <= 8, with weight w_o = alpha[dir_id[o]] * gauss_w[o].
       Host pointers; copied by sal_create.  n_offsets = 0: sal_create builds the window
       itself from the direction fields at the end of this struct (sal_directional_window);
       offsets, gauss_w, dir_id and n_dirs are then ignored. */
    int n_offsets;          /* Q, 0 or 1 <= Q <= 64                                    */
    const int* offsets;     /* [Q][3]                                                  */
    const float* gauss_w;   /* [Q]  Gaussian factor of each neighbour                  */
    const int* dir_id;      /* [Q]  direction group of each neighbour, < n_dirs        */
    int n_dirs;             /* 1 <= n_dirs <= 16                                       */
    const float* alpha;     /* [n_dirs] per-direction weights (host); with n_offsets = 0
                               it may be NULL (all 1)                                   */
    int prec;               /* sal_precision of the local DFT contraction              */
    double ls_delta;        /* ridge delta of the template fit (G + delta I)^-1 b      */
    size_t hbm_budget_bytes;/* upper bound on the handle's device scratch (0 = none)   */
    /* Used when n_offsets = 0 (see sal_directional_window): */
    int n_directions;       /* 0 with directions NULL: the three directions of Fig. 4  */
    const int* directions;  /* [n_directions][3] direction vectors (host)              */
    int radius;             /* R: neighbours s d for s = +-1 .. +-R                    */
    double sigma;           /* sigma of the Gaussian factors                           */
} sal_params;

/* The directional window of Eq. 3 and Fig. 4 (host only, no device work).  For each direction
 * vector d_i (directions [n_directions][3]; with n_directions = 0 and directions NULL, the three
 * directions of Fig. 4: t (1,0,0), x (0,1,0) and t-x (1,1,0)), the neighbours o = s d_i for
 * s = -R .. -1, 1 .. R in that order, with Gaussian factor gauss_w = exp(-|o|^2 / (2 sigma^2))
 * (Eq. 3's w before the per-direction weight alpha) and direction id i.  Q = 2 R n_directions
 * neighbours are written to offsets [Q][3], gauss_w [Q] and dir_id [Q] (host arrays of capacity
 * `cap` neighbours) and Q to *n_offsets.  SAL_ERR_INVALID_ARG if R < 1, sigma is not finite and
 * positive, n_directions is not in [1, 16] (or 0 with directions NULL), a direction is zero, a
 * component of some o exceeds +-8, or Q exceeds cap or 64.  sal_create calls it when
 * sal_params.n_offsets is 0. */
sal_status sal_directional_window(int n_directions, const int* directions, int radius, double sigma, int cap,
                                  int* n_offsets, int* offsets, float* gauss_w, int* dir_id);

/* Creates a handle for volumes of size T x X x Y on the current CUDA device.
 * Validates `p`, builds the DFT tables and allocates scratch (E, S_m and gradient
 * planes, reduction partials) within p->hbm_budget_bytes.  *out receives the
 * handle; on error *out is NULL.  Synchronous. */
sal_status sal_create(const sal_params* p, int T, int X, int Y, sal_handle** out);

/* Frees the handle and its scratch.  NULL is accepted.  Synchronises the device. */
sal_status sal_destroy(sal_handle* h);

/* Bytes of device scratch the handle holds (host pointer `bytes`). */
sal_status sal_workspace_size(const sal_handle* h, size_t* bytes);

/* Replaces the per-direction weights alpha[n_dirs] (host pointer).  Takes effect
 * for calls enqueued after it returns. */
sal_status sal_set_alpha(sal_handle* h, const float* alpha);

/* Steps 1-3 (Sec. 2; Eq. 2 local DFT, Eq. 1 projection, step 3 feature):
 *   E[m][p] = (1/n^3) sum_{k != 0} r_m(k) |F_p[k]|,  m in {t,x,y},
 *   F_p[k] = sum_u h(u) Vext[p + u - n/2] exp(-2 pi i k.u / n),  u,k in [0,n)^3,
 *   r_t = sqrt(j^2+k^2)/|kappa|, r_x = sqrt(i^2+k^2)/|kappa|, r_y = sqrt(i^2+j^2)/|kappa|,
 * with signed bins (i,j,k) and the zero-frequency bin left out.
 * V: [T][X][Y] float32 (device).  E: [3][T][X][Y] float32 (device, written). */
sal_status sal_local_spectra_project(sal_handle* h, const float* V, float* E, void* stream);

/* Step 4, directional center-surround (Eq. 3):
 *   S3[m][p] = (1/Q) sum_o | E[m][p] - w_o * Eext[m][p + o] |.
 * E: [3][T][X][Y] (device).  S3: [3][T][X][Y] raw maps (device, written). */
sal_status sal_center_surround(sal_handle* h, const float* E, float* S3, void* stream);

/* Step 5, combination (Eq. 4): each S_m is min-max normalised to [0,1] (a flat map
 * becomes 0); the weights are W_in (device [3]) if D is NULL and W_in is not, equal
 * (1/3) if both are NULL, or, if D (device [T][X][Y], the desired map) is given, the
 * least-squares fit W = (G + delta I)^-1 b with G = sum_p x_p x_p^T, b = sum_p x_p D_p,
 * x_p = (S^_t, S^_x, S^_y)(p), accumulated in FP64.  S = minmax(sum_m W_m S^_m).
 * W_out: device [3], receives the weights used (nullable).  S: [T][X][Y] (written). */
sal_status sal_combine(sal_handle* h, const float* S3, const float* D, const float* W_in,
                       float* W_out, float* S, void* stream);

/* Steps 1-5 in one call.  S3_opt and E_opt (nullable, device [3][T][X][Y]) receive
 * the intermediate maps when given; otherwise the handle's scratch holds them. */
sal_status sal_saliency(sal_handle* h, const float* V, const float* D, const float* W_in,
                        float* S, float* S3_opt, float* E_opt, float* W_out, void* stream);

/* Gradient of L = sum_p gS[p] * S[p] for S = sal_saliency(V, weights W) with the
 * min-max bounds of the forward pass held constant (the paper has no backward pass;
 * this is the adjoint of Eq. 1-4).  Recomputes the forward pass and the local
 * spectra brick by brick; no spectra are stored.
 * V: [T][X][Y], W: device [3] (the weights of the forward pass), gS: [T][X][Y].
 * Outputs (device, each nullable): gV [T][X][Y], gW [3], galpha [n_dirs]. */
sal_status sal_saliency_backward(sal_handle* h, const float* V, const float* W, const float* gS,
                                 float* gV, float* gW, float* galpha, void* stream);

/* Allocation-free form of sal_combine, for callers that cannot allocate device memory: code
 * that runs under a caller-owned memory pool or arena, inside a region where new allocations
 * are forbidden, or on a path where an allocation and the synchronisation it may bring are not
 * acceptable.  It needs no handle (sal_create allocates) and calls no cudaMalloc or cudaFree.
 * The paper has no counterpart.  It computes what sal_combine computes, with the same arguments
 * and results (ls_delta as in sal_params), on the current device: S3, S and the non-NULL D, W_in,
 * W_out must be device memory of that device (else SAL_ERR_INVALID_ARG before any work).
 * Its reduction scratch is one file-scope device array of about 0.6 MiB that every GPU that
 * loads the library holds until the process exits.  Limit: T*X*Y <= 16,777,216 voxels; larger
 * volumes return SAL_ERR_UNSUPPORTED before any work.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current and keeps it for the
 * process: make that first call before any stream capture, and do not call it on a device after
 * a cudaDeviceReset of that device in the same process (the kept address would be stale).  All
 * calls share the array: calls that overlap on the GPU (other streams, other threads) race and
 * give wrong results.  Errors are reported by sal_last_error(NULL), which a successful call
 * clears. */
sal_status sal_combine_noalloc(int T, int X, int Y, const float* S3, const float* D, const float* W_in,
                               double ls_delta, float* W_out, float* S, void* stream);

/* The paper's adaptive weight update for step 5 (Eq. 4 and the adaptive scheme with LMS, NLMS and
 * RLS, run as the sequential filters the paper describes; NLMS is its choice for all results).
 * x_p = (S^_t, S^_x, S^_y)(p) are the min-max normalised maps of S3 (a flat map gives 0), d_p = D[p];
 * the voxels are visited inline sections (y) outermost, then x, then t; e = d - W.x and
 *   LMS:  W += mu e x                      (W0 = (1/3, 1/3, 1/3))
 *   NLMS: W += mu e x / (eps + |x|^2)      (W0 = (1/3, 1/3, 1/3))
 *   RLS:  k = P x / (lambda + x'P x); W += k e; P = (P - k x'P) / lambda   (W0 = 0, P0 = I / delta)
 * in FP64.  sections = 0: one recursion over the whole volume; sections = N > 0: the weights are
 * re-adapted for every block of N inline sections (each block its own recursion from W0), as the
 * paper allows.  The recursion is sequential by nature: one warp per block.
 * S3: [3][T][X][Y] raw maps; D: [T][X][Y]; W_out: device [ceil(Y / N)][3] (one row when
 * sections = 0); err2 (nullable): device [T*X*Y], the squared error e^2 of every step in filter
 * order.  The weights of a block can be passed to sal_combine as W_in. */
typedef enum { SAL_ADAPT_LMS = 0, SAL_ADAPT_NLMS = 1, SAL_ADAPT_RLS = 2 } sal_adapt_method;
typedef struct {
    sal_adapt_method method;
    double mu;       /* LMS / NLMS step size (0.5) */
    double eps;      /* NLMS regulariser (1e-8) */
    double lambda;   /* RLS forgetting factor (1) */
    double delta;    /* RLS P0 = I / delta (1e-6) */
    int sections;    /* inline sections per block; 0 = whole volume */
} sal_adapt_params;
sal_status sal_adapt_weights(sal_handle* h, const float* S3, const float* D, const sal_adapt_params* p,
                             float* W_out, float* err2, void* stream);

/* Stepwise backward calls (adjoints of the three forward steps; the fused call above is
 * their composition).  The paper has no backward pass: these follow from Eq. 1-4.
 *
 * sal_local_spectra_project_backward: gV = (dE/dV)^T gE for E = sal_local_spectra_project(V):
 *   gVext[p + u - n/2] += Re sum_k h(u) exp(+2 pi i k.u / n) (sum_m gE_m[p] r_m(k)/n^3) F_p[k]/|F_p[k]|
 *   folded back through the border extension.  V, gV: [T][X][Y]; gE: [3][T][X][Y].
 *   The first backward call on a handle allocates its backward scratch. */
sal_status sal_local_spectra_project_backward(sal_handle* h, const float* V, const float* gE, float* gV,
                                              void* stream);

/* sal_center_surround_backward: adjoint of Eq. 3 with respect to E and the per-direction
 * weights: gE = (dS3/dE)^T gS3 (nullable), galpha[d] = sum_{o in d} gauss_w[o] dL/dw_o
 * (nullable).  sgn(0) = 0 at the kinks of |.|.  E, gS3, gE: [3][T][X][Y]. */
sal_status sal_center_surround_backward(sal_handle* h, const float* E, const float* gS3, float* gE, float* galpha,
                                        void* stream);

/* sal_combine_backward: adjoint of Eq. 4 and the two min-max normalisations (bounds held
 * constant) for S = sal_combine(S3, W): gS3[m] = W_m gS / ((max C - min C)(max S_m - min S_m)),
 * gW (nullable, device [3]).  S3, gS3: [3][T][X][Y]; W: device [3]; gS: [T][X][Y]. */
sal_status sal_combine_backward(sal_handle* h, const float* S3, const float* W, const float* gS, float* gS3,
                                float* gW, void* stream);

/* Check of the failure detection (the paper has no counterpart).  The tensor-core kernels bound every
 * wait on an mbarrier; a wait that gives up sets the handle's error word, the CTA leaves, and the next
 * call on the handle returns SAL_ERR_TIMEOUT and clears the word.  This call makes such a wait give
 * up on purpose: one CTA waits on an mbarrier to which no arrival is ever made, through the same
 * bounded helper, with `tries` tries (1 <= tries <= 2^20; SAL_ERR_INVALID_ARG otherwise), then sets
 * the error word and returns.  Nothing faults, traps or spins without bound, and the CUDA context and
 * the handle stay usable.  Enqueued on `stream`; returns SAL_OK once enqueued. */
sal_status sal_check_bounded_wait(sal_handle* h, unsigned tries, void* stream);

/* Measured issue rate of the MUFU pipe (the paper has no counterpart: the roofline denominator of the
 * |F| epilogues).  op 0: sqrt.approx.f32, op 1: rsqrt.approx.f32, the instructions those epilogues
 * issue once per bin.  Runs 8 CTAs of 256 threads per SM of the current device, each thread 16
 * independent chains of 2048 operations, on the legacy default stream, synchronously, after one
 * warm-up launch, timed with CUDA events; allocates and frees a small output buffer.
 * *ops_per_second receives operations per second over the whole device, *sm_count (nullable) the
 * device's SM count.  Errors are reported by sal_last_error(NULL). */
sal_status sal_measure_mufu_rate(int op, double* ops_per_second, int* sm_count);

/* Measured cost of one tensor-core MMA (tcgen05.mma, kind::f16, M = 128, K = 16, FP16 operands, FP32
 * accumulation) with n_cols = 16, 32, 64, 128 or 256 columns, in SM clock cycles: the instruction
 * rate of the tensor pipe, which bounds the local-spectrum kernels' narrow MMAs (N = 16 .. 64) rather
 * than their flops.  Not part of the paper's method (the measurement behind the tensor-core kernels'
 * roofline).  One CTA per SM of the current device; one elected thread issues 4096 MMAs back to back on
 * constant operands in shared memory into one tensor-memory accumulator, commits them and waits
 * (bounded); runs on the legacy default stream, synchronously, after one warm-up launch, and allocates
 * and frees two small device buffers.  *cycles_per_mma receives the mean over the SMs of the cycles
 * from the first issue to completion divided by 4096, *sm_count (nullable) the device's SM count.
 * SAL_ERR_UNSUPPORTED on a device without 5th-generation tensor cores; SAL_ERR_TIMEOUT if the bounded
 * wait gave up.  Errors are reported by sal_last_error(NULL). */
sal_status sal_measure_mma_rate(int n_cols, double* cycles_per_mma, int* sm_count);

/* Number of kernels this library has launched in the process so far (all handles and
 * entry points), for accounting; host pointer `count`. */
sal_status sal_launch_count(unsigned long long* count);

/* Message of the last error on the handle ("" if none).  h may be NULL (then the
 * last sal_create error of this thread is returned).  The string lives until the
 * next call on the handle. */
const char* sal_last_error(const sal_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* SAL_H */
