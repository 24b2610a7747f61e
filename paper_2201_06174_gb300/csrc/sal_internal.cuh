// Internal declarations shared by the libsal.so translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "sal.h"

namespace sal {

constexpr int kMaxOffsets = 64;
constexpr int kMaxDirs = 16;
constexpr int kMaxHalo = 8;      // |dt|,|dx|,|dy| bound of a center-surround offset
constexpr int kMaxN = 32;        // largest DFT side the tables hold
constexpr int kRedBlocks = 1216; // fixed fan-in of the grid-stride reductions (8 blocks per SM of a
                                 // 152-SM part); the results do not depend on the device

// Center-surround window of Eq. 3, passed by value as a kernel parameter.
struct Stencil {
    int Q;
    int n_dirs;
    float invQ;
    int halo[3];              // max |offset component| per axis (t, x, y)
    int off[kMaxOffsets][3];
    float g[kMaxOffsets];     // Gaussian factor of each neighbour
    int dir[kMaxOffsets];     // direction group
    float w[kMaxOffsets];     // effective weight alpha[dir] * g
};

// Real DFT twiddles with the taper folded in: c[k][u] = h(u) cos(2 pi k u / n),
// s[k][u] = h(u) sin(2 pi k u / n), for k in [0, n/2], u in [0, n).
struct TwiddleTable {
    int n;
    float c[kMaxN / 2 + 1][kMaxN];
    float s[kMaxN / 2 + 1][kMaxN];
};

enum : int { BND_SYMMETRIC = 0, BND_PERIODIC = 1, BND_ZERO = 2 };

// Border extension of one axis; -1 where the zero extension applies.
__host__ __device__ __forceinline__ int ext_index(int i, int n, int mode) {
    if ((unsigned)i < (unsigned)n) return i;
    if (mode == BND_PERIODIC) {
        int r = i % n;
        return r < 0 ? r + n : r;
    }
    if (mode == BND_ZERO) return -1;
    int P = 2 * n;  // symmetric, edge sample repeated
    int r = i % P;
    if (r < 0) r += P;
    return r < n ? r : P - 1 - r;
}

// Scratch for the volume-wide reductions (device memory owned by the handle).
struct Reduce {
    float* mm_part;     // [kRedBlocks][8]  per-block min/max partials
    double* g_part;     // [kRedBlocks][16] per-block FP64 partial sums
    float* norm;        // [16]: lo[3], inv[3], W[3], loC, invC, flags
    double* wsum;       // [16]: reduced FP64 sums (Gram, gradient of W)
};

// ---- K1: local spectra + projection + features ----------------------------------------------
// feat: 0 = the mean of |F_m| (step 3), 1 = the mean of |F_m|^2 (energy reading).  stride s: cubes only
// at voxels whose indices are multiples of s; E is then the lattice [3][ceil(T/s)][ceil(X/s)][ceil(Y/s)].
bool spectra_f32_supported(int n);
cudaError_t spectra_f32_prepare(int n);
// taper 0 (rect) at stride 1 takes the sliding form of stage 3 for n >= 8
// wtab: the Eq. 1 weight table of the FP32 kernels (f32_weight_table_fill), device memory
cudaError_t spectra_f32_launch(int n, const TwiddleTable& tw, const float* wtab, const float* V, float* E, int T,
                               int X, int Y, int bnd, int feat, int stride, int taper, cudaStream_t s);
size_t f32_weight_table_floats(int n);
// The spatial-domain reading of the feature step (FP32, n in {2, 4, 8, 16}, stride 1): per-window separable
// FFTs in shared memory (spatial_f32_prepare sets their shared-memory limits; once per device).  rtab: the
// Eq. 1 ratio table (spatial_weight_table_fill, host; 16-byte aligned device copy).
bool spatial_f32_supported(int n);
size_t spatial_weight_table_floats(int n);
void spatial_weight_table_fill(int n, float* out);
cudaError_t spatial_f32_prepare();
cudaError_t spatial_f32_launch(int n, const float* rtab, const float* V, float* E, int T, int X, int Y, int bnd,
                               int taper, cudaStream_t s);
void f32_weight_table_fill(int n, int feat, float* out);   // host
// The lattice features of stride s to every voxel of E [3][T][X][Y] (trilinear, held past the last point),
// and its adjoint: the lattice points of gEl (full-size, zero elsewhere) gather the gradients gE.
cudaError_t upsample_launch(const float* Ec, float* E, int T, int X, int Y, int stride, cudaStream_t s);
cudaError_t upsample_adjoint_launch(const float* gE, float* gEl, int T, int X, int Y, int stride, cudaStream_t s);
// V [rows][Y] -> Vp [rows][Ypad] (Ypad >= Y; the padding columns are not written)
cudaError_t pad_rows_launch(const float* V, float* Vp, long long rows, int Y, int Ypad, cudaStream_t s);

// K1 for the 32^3 window: FP32 on the SIMT pipes, or on the tensor cores (BF16 fmt = 1, FP16 fmt = 0)
cudaError_t spectra_f32_n32_prepare();
// taper 0 (rect) at stride 1 takes the sliding form of stage 3
cudaError_t spectra_f32_n32_launch(const TwiddleTable& tw, const float* V, float* E, int T, int X, int Y, int bnd,
                                   int feat, int stride, int taper, cudaStream_t s);
cudaError_t spectra_tc32_prepare(int fmt);
cudaError_t spectra_tc32_launch(int fmt, const TwiddleTable& tw, const float* V, float* E, int T, int X, int Y,
                                int bnd, int feat, int stride, int* err, cudaStream_t s);

// K1 on the tensor cores (BF16 fmt = 1, FP16 fmt = 0); err: device-visible error word.  The constant
// operands (twiddles in the operand layouts, Eq. 1 weights) are built once per handle into `tables`.
bool spectra_tc_supported(int n);
size_t spectra_tc_tables_bytes(int n);
cudaError_t spectra_tc_prepare(int n, int fmt);
cudaError_t spectra_tc_tables_build(int n, int fmt, const TwiddleTable& tw, int feat, void* tables, cudaStream_t s);
// Vt (nullable): a copy of V with rows of Yt >= Y floats, Yt a multiple of 4, which the TMA staging of interior
// bricks reads through one tensor copy per brick when V's own rows are not a multiple of 16 bytes.
cudaError_t spectra_tc_launch(int n, int fmt, const void* tables, const float* V, float* E, int T, int X, int Y,
                              int bnd, int feat, int stride, const float* Vt, int Yt, int* err, cudaStream_t s);

// ---- K3a: sequential adaptive weights (LMS / NLMS / RLS) over inline-section blocks -------------
// Per-map bounds of S3 into r.norm (lo at 0..2, 1/(hi-lo) at 3..5; 0 for a flat map).
cudaError_t minmax_bounds_launch(const float* S3, long long N, const Reduce& r, cudaStream_t s);
// Normalised maps from S3 and r.norm; one chain per block of `sections` inline sections (0: one chain);
// W_out [blocks][3]; err2 (nullable) the squared error of every step in filter order.
cudaError_t adapt_launch(const float* S3, const float* D, int T, int X, int Y, int method, double mu, double eps,
                         double lambda, double delta, int sections, const float* norm, float* W_out, float* err2,
                         cudaStream_t s);

// ---- K2: directional center-surround ----------------------------------------------------------
// Once per device: the shared-memory size limit of the ring-staged K2 (windows whose ring fits 96 KB).
cudaError_t dcs_prepare();
cudaError_t dcs_launch(const float* E, float* S3, int T, int X, int Y, int bnd, const Stencil& st,
                       float* mm_part, cudaStream_t s);

// ---- K3: normalisation + combination ----------------------------------------------------------
int red_blocks(long long NV);  // grid of the grid-stride reduction kernels (<= kRedBlocks)
cudaError_t combine_launch(const float* S3, const float* D, const float* W_in, float* W_out, float* S,
                           long long N, double delta, bool s3_partials_ready, const Reduce& r, cudaStream_t s);

// ---- K4/K5 and the backward reductions ---------------------------------------------------------
// Brick of the spectral adjoint: outputs x0 in [xs*BX, xs*BX+BX), y0 in [ys*BY, ys*BY+BY) at one t0;
// its block of gVext is [u_t in n][XH = BX+n-1][YH = BY+n-1] floats.
struct SpectraAdjointGeometry {
    int BY;            // outputs per brick along y
    int YH;            // y extent of a brick's block
    int BX;            // outputs per brick along x
    int XH;            // x extent of a brick's block
    int block_floats;  // n * slice: scratch floats per brick
    int slice;         // floats per u_t slice of a block: XH * YH rounded up to a multiple of 4 (16-byte rows)
};
cudaError_t spectra_adjoint_f32_prepare(int n);
SpectraAdjointGeometry spectra_adjoint_f32_geometry(int n);
// bricks of t0 = t_begin + r t_step, r < t_count (t_step s > 1: the lattice planes of stride-s windows)
// taper 0 (rect) runs both y-passes as sliding recursions for n = 8, 16.  lists (nullable; device scratch of
// spectra_adjoint_f32_list_bytes): the small bins of the abs(F) reading are listed per CTA there and
// resolved by a second, grid-wide pass; without it each CTA resolves its own.
size_t spectra_adjoint_f32_list_bytes(int n, int X, int Y, int t_count);
cudaError_t spectra_adjoint_f32_launch(int n, const TwiddleTable& tw, const float* wtab, const float* V,
                                       const float* gE, float* blocks, int T, int X, int Y, int bnd, int feat,
                                       int t_begin, int t_step, int t_count, int taper, int* lists, cudaStream_t s);
// K5 on the tensor cores (FP16 operands: fmt must be 0); its constant operands are built once per handle
cudaError_t spectra_adjoint_tc_prepare(int n, int fmt);
size_t spectra_adjoint_tc_tables_bytes(int n);
cudaError_t spectra_adjoint_tc_tables_build(int n, const TwiddleTable& tw, int feat, void* tables, cudaStream_t s);
SpectraAdjointGeometry spectra_adjoint_tc_geometry(int n);
// The adjoint of the spatial-domain reading: brick blocks of the same layout as K5's (geometry below), bricks
// of the planes t_begin .. t_begin + t_count - 1 (stride 1)
SpectraAdjointGeometry spatial_adjoint_f32_geometry(int n);
cudaError_t spatial_adjoint_f32_launch(int n, const float* rtab, const float* V, const float* gE, float* blocks,
                                       int T, int X, int Y, int bnd, int t_begin, int t_count, int taper,
                                       cudaStream_t s);
cudaError_t spectra_adjoint_tc_launch(int n, int fmt, const TwiddleTable& tw, const void* tables, const float* V,
                                      const float* gE, float* blocks, int T, int X, int Y, int bnd, int feat,
                                      int t_begin, int t_step, int t_count, const float* Vt, int Yt, int* err,
                                      cudaStream_t s);
cudaError_t backward_weights_launch(const float* S3, const float* gS, long long N, const Reduce& r, double* part,
                                    float* coef, float* gW, cudaStream_t s);
// gS with map stride gms: the raw-map gradient of map m at p is coef[m] * gS[m * gms + p].  Windows whose
// plane ring fits shared memory run tiled when the tiles fill two waves of the GPU (dcs_adjoint_prepare
// sets the size limit and reads the SM count; once per device).
cudaError_t dcs_adjoint_prepare();
// gS with map stride gms: the raw-map gradient of map m at p is coef[m] * gS[m * gms + p]
cudaError_t dcs_adjoint_launch(const float* E, const float* gS, long long gms, const float* coef, float* gE, int T,
                               int X, int Y, int bnd, const Stencil& st, cudaStream_t s);
cudaError_t dcs_galpha_launch(const float* E, const float* gS, long long gms, const float* coef, int T, int X, int Y,
                              int bnd, const Stencil& st, double* part, float* galpha, cudaStream_t s);
// Both at once: the tiled kernel also sums the weight-gradient terms (one FP64 partial per tile and offset into
// tile_part, tile_part_bytes long) when the window has at most 18 offsets and the partials fit; otherwise the
// two launches above.  gE and galpha must both be given.
cudaError_t dcs_adjoint_galpha_launch(const float* E, const float* gS, long long gms, const float* coef, float* gE,
                                      int T, int X, int Y, int bnd, const Stencil& st, double* tile_part,
                                      size_t tile_part_bytes, double* part, float* galpha, cudaStream_t s);
cudaError_t expand_gradient_launch(const float* gS, const float* coef, float* gS3, long long N, cudaStream_t s);
// Overlap-add of one slab's brick blocks into gV through the scratch `ext` (gather_ext_floats floats):
// first along t (contiguous slices), then across the bricks that overlap each voxel.
size_t gather_ext_floats(int n, SpectraAdjointGeometry g, int X, int Y, int t_count, int t_step);
cudaError_t gather_add_launch(const float* blocks, float* ext, float* gV, int T, int X, int Y, int bnd, int n,
                              SpectraAdjointGeometry g, int t_begin, int t_count, int t_step, cudaStream_t s);

// One CTA waits, through the tensor-core kernels' bounded mbarrier wait, on a barrier that nobody
// arrives at, gives up after `tries` tries and sets the error word (failure-detection check).
cudaError_t wait_check_launch(int* err, unsigned tries, cudaStream_t s);

// SM count of the current device (cudaDevAttrMultiProcessorCount; 1 if the query fails).
int device_sms();

// Process-wide count of kernels launched by the library (sal_launch_count).
void note_launches(int k);

// Message for sal_last_error(NULL) from entry points that have no handle.
void set_unbound_error(const std::string& msg);

}  // namespace sal
