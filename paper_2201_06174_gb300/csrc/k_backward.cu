// Backward pass of the combination and center-surround steps, and the overlap-add gather of the
// spectral adjoint (the paper has no backward pass; this is the adjoint of Eq. 3 and Eq. 4 with
// the min-max bounds of the forward pass held constant).
//
//   S = (C - loC) invC,  C = sum_m W_m S^_m,  S^_m = (S_m - lo_m) inv_m
//   gW_m = invC inv_m sum_p gS[p] (S_m[p] - lo_m)            (FP64 sums, fixed order)
//   gS_m = coef_m gS,  coef_m = W_m invC inv_m
// Center-surround (Eq. 3), d_{p,o} = E[p] - w_o Eext[p+o], sgn(0) = 0:
//   gE[q] = (1/Q) [ gS_m[q] sum_o sgn(d_{q,o}) - sum_o w_o sum_{p: ext(p+o) = q} gS_m[p] sgn(d_{p,o}) ]
//   gw_o  = -(1/Q) sum_m sum_p gS_m[p] sgn(d_{p,o}) Eext_m[p+o],   galpha_d = sum_{o in d} g_o gw_o
// Every output is formed by gathering, so no atomics are used and results are deterministic.
#include <cfloat>

#include "sal_internal.cuh"

namespace sal {
namespace {

constexpr int kThreads = 256;
constexpr int kYChunk = 128;   // voxels of a row per warp work item of the stencil kernels
constexpr size_t kTileSmemMax = 96 * 1024;   // plane ring of the tiled center-surround adjoint
enum : int { N_LO = 0, N_INV = 3, N_W = 6, N_LOC = 9, N_INVC = 10 };

__device__ __forceinline__ int floordiv(int a, int b) {  // b > 0
    int q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}
__device__ __forceinline__ int ceildiv(int a, int b) { return -floordiv(-a, b); }

__device__ __forceinline__ float sgnf(float d) { return (d > 0.f) ? 1.f : ((d < 0.f) ? -1.f : 0.f); }

// Positions p in [0, N) with ext(p + o) == q: the range [o, N + o) is shorter than one period,
// so each family of preimages contributes at most one (at most two in all).
__device__ __forceinline__ int pre_offset(int q, int o, int N, int mode, int* out) {
    // extended positions i' in [o, N + o) that map to q
    const int lo = o, hi = N + o;
    int c = 0;
    if (mode == BND_ZERO) {
        if (q >= lo && q < hi) out[c++] = q - o;
    } else if (mode == BND_PERIODIC) {
        for (int i = q + N * ceildiv(lo - q, N); i < hi; i += N) out[c++] = i - o;
    } else {
        const int P = 2 * N;
        for (int i = q + P * ceildiv(lo - q, P); i < hi; i += P) out[c++] = i - o;
        const int r = P - 1 - q;
        for (int i = r + P * ceildiv(lo - r, P); i < hi; i += P) out[c++] = i - o;
    }
    return c;
}

// pre_offset without divisions when N >= abs(o) (the general form otherwise); same positions, same order:
// the direct preimage q - o, then the reflections below and above the volume (symmetric); the one
// wrapped position (periodic).
__device__ __forceinline__ int pre_offset_near(int q, int o, int N, int mode, int* out) {
    if (N < (o < 0 ? -o : o)) return pre_offset(q, o, N, mode, out);
    int c = 0;
    const int p = q - o;
    if (mode == BND_ZERO) {
        if ((unsigned)p < (unsigned)N) out[c++] = p;
    } else if (mode == BND_PERIODIC) {
        out[c++] = p < 0 ? p + N : (p >= N ? p - N : p);   // p in [-N, 2N): exactly one wrap lands
    } else {
        const int lo = -1 - q - o, hi = 2 * N - 1 - q - o;
        if ((unsigned)p < (unsigned)N) out[c++] = p;
        if ((unsigned)lo < (unsigned)N) out[c++] = lo;
        if ((unsigned)hi < (unsigned)N) out[c++] = hi;
    }
    return c;
}

// Extended positions i' in [lo, hi) with ext(i') == q.
__device__ __forceinline__ int pre_range(int q, int N, int mode, int lo, int hi, int* out, int cap) {
    int c = 0;
    if (mode == BND_ZERO) {
        if (q >= lo && q < hi) out[c++] = q;
    } else if (mode == BND_PERIODIC) {
        for (int i = q + N * ceildiv(lo - q, N); i < hi && c < cap; i += N) out[c++] = i;
    } else {
        const int P = 2 * N;
        for (int i = q + P * ceildiv(lo - q, P); i < hi && c < cap; i += P) out[c++] = i;
        const int r = P - 1 - q;
        for (int i = r + P * ceildiv(lo - r, P); i < hi && c < cap; i += P) out[c++] = i;
    }
    return c;
}

// FP64 partials of sum_p gS[p] (S_m[p] - lo_m), m = 0..2.
__global__ void __launch_bounds__(kThreads)
kb_weights_partial(const float* __restrict__ S3, const float* __restrict__ gS, long long NV,
                   const float* __restrict__ norm, double* __restrict__ part) {
    const float lo0 = norm[N_LO], lo1 = norm[N_LO + 1], lo2 = norm[N_LO + 2];
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (long long p = (long long)blockIdx.x * kThreads + threadIdx.x; p < NV; p += (long long)gridDim.x * kThreads) {
        const double g = (double)__ldg(gS + p);
        a0 += g * (double)(__ldg(S3 + p) - lo0);
        a1 += g * (double)(__ldg(S3 + NV + p) - lo1);
        a2 += g * (double)(__ldg(S3 + 2 * NV + p) - lo2);
    }
    __shared__ double red[3][kThreads];
    red[0][threadIdx.x] = a0;
    red[1][threadIdx.x] = a1;
    red[2][threadIdx.x] = a2;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 3) part[blockIdx.x * 64 + threadIdx.x] = red[threadIdx.x][0];
}

// gW and the per-map coefficients coef_m = W_m invC inv_m.  One block.
__global__ void __launch_bounds__(kThreads)
kb_weights_finalize(const double* __restrict__ part, int nparts, const float* __restrict__ norm,
                    float* __restrict__ coef, float* __restrict__ gW) {
    __shared__ double s[3][kThreads];
    for (int c = 0; c < 3; ++c) {
        double a = 0.0;
        for (int i = threadIdx.x; i < nparts; i += kThreads) a += part[i * 64 + c];
        s[c][threadIdx.x] = a;
    }
    __syncthreads();
    for (int st = kThreads / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st)
            for (int c = 0; c < 3; ++c) s[c][threadIdx.x] += s[c][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x < 3) {
        const int m = threadIdx.x;
        const double invC = norm[N_INVC], inv = norm[N_INV + m];
        coef[m] = (float)((double)norm[N_W + m] * invC * inv);
        if (gW) gW[m] = (float)(invC * inv * s[m][0]);
    }
}

// One voxel q = (t, x, y) of the center-surround adjoint through the border extension: q as the center of
// each comparison (neighbour ext(q + o)) and as the neighbour (every p with ext(p + o) = q).
__device__ __forceinline__ void dcs_adjoint_border(const float* __restrict__ E, const float* __restrict__ gS,
                                                   long long gms, int T, int X, int Y, int bnd, const Stencil& st,
                                                   const float* s_w, int t, int x, int y, const float (&eq)[3],
                                                   const float (&gq)[3], float (&acc)[3]) {
    const long long NV = (long long)T * X * Y;
    for (int o = 0; o < st.Q; ++o) {
        const int dt = st.off[o][0], dx = st.off[o][1], dy = st.off[o][2];
        const float w = s_w[o];
        // q as the center of the comparison
        const int tt = ext_index(t + dt, T, bnd), xx = ext_index(x + dx, X, bnd), yy = ext_index(y + dy, Y, bnd);
        const bool ok = (tt | xx | yy) >= 0;
        const long long nq = ok ? ((long long)tt * X + xx) * Y + yy : 0;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const float nb = ok ? __ldg(E + m * NV + nq) : 0.f;
            acc[m] += sgnf(fmaf(-w, nb, eq[m])) * gq[m];
        }
        // q as the neighbour: p with ext(p + o) = q
        int pt[2], px[2], py[2];
        const int nt = pre_offset_near(t, dt, T, bnd, pt);
        const int nx = pre_offset_near(x, dx, X, bnd, px);
        const int ny = pre_offset_near(y, dy, Y, bnd, py);
        for (int a = 0; a < nt; ++a)
            for (int b = 0; b < nx; ++b)
                for (int c = 0; c < ny; ++c) {
                    const long long p = ((long long)pt[a] * X + px[b]) * Y + py[c];
#pragma unroll
                    for (int m = 0; m < 3; ++m)
                        acc[m] -= w * sgnf(fmaf(-w, eq[m], __ldg(E + m * NV + p))) * __ldg(gS + m * gms + p);
                }
    }
}

// K4: gradient of the features through Eq. 3 (gather form).  One warp per 128 voxels of a (t, x) row;
// voxels the stencil halo away from every border read their neighbours q + o and their preimages q - o
// at linear offsets, the others go through the border extension.
__global__ void __launch_bounds__(kThreads)
k4_dcs_adjoint(const float* __restrict__ E, const float* __restrict__ gS, long long gms, const float* __restrict__ coef,
               float* __restrict__ gE, int T, int X, int Y, int bnd, const __grid_constant__ Stencil st) {
    constexpr int kWarps = kThreads / 32;
    // gradient of the raw map m at p: coef[m] * gS[m * gms + p]
    const long long NV = (long long)T * X * Y;
    const float c0 = coef[0], c1 = coef[1], c2 = coef[2];
    __shared__ long long s_lin[kMaxOffsets];
    __shared__ float s_w[kMaxOffsets];
    for (int o = threadIdx.x; o < st.Q; o += kThreads) {
        s_lin[o] = ((long long)st.off[o][0] * X + st.off[o][1]) * Y + st.off[o][2];
        s_w[o] = st.w[o];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int Q = st.Q;
    const int ht = st.halo[0], hx = st.halo[1], hy = st.halo[2];
    const int nyc = (Y + kYChunk - 1) / kYChunk;
    for (long long it = (long long)blockIdx.x * kWarps + wid; it < (long long)T * X * nyc;
         it += (long long)gridDim.x * kWarps) {
        const long long r = it / nyc;
        const int yc = (int)(it - r * nyc) * kYChunk, ye = min(Y, yc + kYChunk);
        const int t = (int)(r / X), x = (int)(r - (long long)t * X);
        const bool row_inner = t >= ht && t < T - ht && x >= hx && x < X - hx;
        for (int y = yc + lane; y < ye; y += 32) {
            const long long q = r * Y + y;
            float eq[3], gq[3], acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                eq[m] = __ldg(E + m * NV + q);
                gq[m] = __ldg(gS + m * gms + q);
            }
            if (row_inner && y >= hy && y < Y - hy) {
                // the neighbour is q + o and the only preimage of q under offset o is q - o
#pragma unroll 2
                for (int o = 0; o < Q; ++o) {
                    const long long d = s_lin[o];
                    const float w = s_w[o];
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        const float nb = __ldg(E + m * NV + q + d);
                        const float pe = __ldg(E + m * NV + q - d), pg = __ldg(gS + m * gms + q - d);
                        acc[m] += sgnf(fmaf(-w, nb, eq[m])) * gq[m];
                        acc[m] -= w * sgnf(fmaf(-w, eq[m], pe)) * pg;
                    }
                }
            } else {
                dcs_adjoint_border(E, gS, gms, T, X, Y, bnd, st, s_w, t, x, y, eq, gq, acc);
            }
            gE[q] = acc[0] * c0 * st.invQ;
            gE[NV + q] = acc[1] * c1 * st.invQ;
            gE[2 * NV + q] = acc[2] * c2 * st.invQ;
        }
    }
}

// K4, tiled: one block per tile of 16 x 16 (x, y) columns and up to 8 planes along t (a thread per
// column).  E and gS of the tile and its halo stream through a ring of 2 h_t + 1 planes in shared memory
// (border extension applied at load), so each value is read from global memory once per tile instead of
// once per neighbour; the next plane is fetched into registers while the current one is computed.  Voxels
// the stencil halo away from every border do exactly the arithmetic of the row kernel on the staged
// values; the others (several preimages, or none) take the border path, also on the staged values.
constexpr int kTX = 16, kTY = 16, kTileT = 8;
constexpr int kPre = 2;   // plane elements per thread prefetched into registers (the rest loaded at store)
static_assert(kTX * kTY == kThreads, "one column per thread");

__host__ __device__ inline size_t dcs_tile_smem_bytes(int ht, int hx, int hy) {
    return (size_t)(2 * ht + 1) * 6 * (kTX + 2 * hx) * (kTY + 2 * hy) * sizeof(float);
}

// Geometry of the staged planes of one tile: ring slot b of plane t, planes t - h_t .. t + h_t, columns
// [x0 - h_x, x0 + kTX + h_x) x [y0 - h_y, y0 + kTY + h_y).
struct TileRing {
    const float* ring;
    int R, PL, PE, TXH, TYH, ht, hx, hy, x0, y0;
    __device__ __forceinline__ int slot(int b, int dt) const {   // |dt| <= h_t: one wrap at most
        int sl = b + dt;
        sl += sl < 0 ? R : 0;
        sl -= sl >= R ? R : 0;
        return sl;
    }
};

// The per-voxel border path of the tiled kernel, in the order of dcs_adjoint_border (same sums, same
// result): the neighbour ext(q + o) is staged for every voxel of the tile; each preimage p comes from the
// ring when it lies in the staged region (always, for symmetric and zero extension: a reflected preimage
// is within the halo of q) and from global memory otherwise (periodic wrap across the volume).
__device__ __forceinline__ void dcs_adjoint_border_tile(const float* __restrict__ E, const float* __restrict__ gS,
                                                        long long gms, int T, int X, int Y, int bnd,
                                                        const TileRing& tr, const int (*s_d)[3], const float* s_w,
                                                        int Q, int b, int t, int x, int y, const float (&eq)[3],
                                                        const float (&gq)[3], float (&acc)[3]) {
    const long long NV = (long long)T * X * Y;
    for (int o = 0; o < Q; ++o) {
        const int dt = s_d[o][0], dx = s_d[o][1], dy = s_d[o][2];
        const float w = s_w[o];
        const float* nb_p = tr.ring + (size_t)tr.slot(b, dt) * tr.PL + (x - tr.x0 + tr.hx + dx) * tr.TYH +
                            (y - tr.y0 + tr.hy + dy);
#pragma unroll
        for (int m = 0; m < 3; ++m) acc[m] += sgnf(fmaf(-w, nb_p[m * tr.PE], eq[m])) * gq[m];
        int pt[2], px[2], py[2];
        const int nt = pre_offset_near(t, dt, T, bnd, pt);
        const int nx = pre_offset_near(x, dx, X, bnd, px);
        const int ny = pre_offset_near(y, dy, Y, bnd, py);
        for (int a = 0; a < nt; ++a)
            for (int c = 0; c < nx; ++c)
                for (int e = 0; e < ny; ++e) {
                    const int rt = pt[a] - t, rx = px[c] - tr.x0 + tr.hx, ry = py[e] - tr.y0 + tr.hy;
                    float pe[3], pg[3];
                    if (rt >= -tr.ht && rt <= tr.ht && rx >= 0 && rx < tr.TXH && ry >= 0 && ry < tr.TYH) {
                        const float* pp = tr.ring + (size_t)tr.slot(b, rt) * tr.PL + rx * tr.TYH + ry;
#pragma unroll
                        for (int m = 0; m < 3; ++m) {
                            pe[m] = pp[m * tr.PE];
                            pg[m] = pp[(3 + m) * tr.PE];
                        }
                    } else {
                        const long long g = ((long long)pt[a] * X + px[c]) * Y + py[e];
#pragma unroll
                        for (int m = 0; m < 3; ++m) {
                            pe[m] = __ldg(E + m * NV + g);
                            pg[m] = __ldg(gS + m * gms + g);
                        }
                    }
#pragma unroll
                    for (int m = 0; m < 3; ++m) acc[m] -= w * sgnf(fmaf(-w, eq[m], pe[m])) * pg[m];
                }
    }
}

// GW: also the per-tile partials of the per-offset weight gradients (the sums of k4_gw_partial, for windows of
// at most kGwMax offsets): each thread sums its voxels' terms over the tile's planes in registers, a fixed
// shuffle tree sums the warp, the warps are summed in order in FP64 into tpart[tile][o].
constexpr int kGwMax = 18;

template <bool GW>
__global__ void __launch_bounds__(kThreads, GW ? 2 : 3)   // 3 blocks per SM: 59 KB of ring each (default window)
k4_dcs_adjoint_tiled(const float* __restrict__ E, const float* __restrict__ gS, long long gms,
                     const float* __restrict__ coef, float* __restrict__ gE, int T, int X, int Y, int bnd,
                     const __grid_constant__ Stencil st, double* __restrict__ tpart) {
    extern __shared__ float s_ring[];   // [2 h_t + 1][6][TXH][TYH]: E_t, E_x, E_y, gS_t, gS_x, gS_y
    __shared__ float s_w[kMaxOffsets];
    __shared__ int s_d[kMaxOffsets][3];
    const long long NV = (long long)T * X * Y;
    const int ht = st.halo[0], hx = st.halo[1], hy = st.halo[2];
    const int R = 2 * ht + 1, TXH = kTX + 2 * hx, TYH = kTY + 2 * hy, PE = TXH * TYH, PL = 6 * PE;
    for (int o = threadIdx.x; o < st.Q; o += kThreads) {
        s_w[o] = st.w[o];
        s_d[o][0] = st.off[o][0];
        s_d[o][1] = st.off[o][1];
        s_d[o][2] = st.off[o][2];
    }
    const int ntx = (X + kTX - 1) / kTX, nty = (Y + kTY - 1) / kTY;
    const int tyi = blockIdx.x % nty, txi = (blockIdx.x / nty) % ntx, tti = blockIdx.x / (nty * ntx);
    const int x0 = txi * kTX, y0 = tyi * kTY, ta = tti * kTileT, tb = min(T, ta + kTileT);
    const int lx = threadIdx.x / kTY, ly = threadIdx.x % kTY;
    const int x = x0 + lx, y = y0 + ly;
    const float c0 = coef[0], c1 = coef[1], c2 = coef[2];
    const int Q = st.Q;
    float gw[GW ? kGwMax : 1];
#pragma unroll
    for (int o = 0; o < (GW ? kGwMax : 1); ++o) gw[o] = 0.f;
    const float cm[3] = {c0, c1, c2};
    const bool col_ok = x < X && y < Y;
    const bool col_inner = x >= hx && x < X - hx && y >= hy && y < Y - hy;
    // global index of element i (< PE) of extended plane gt, or -1 outside a zero-extended volume
    auto src = [&](int gt, int i) -> long long {
        const int ix = i / TYH, iy = i - ix * TYH;
        const int gx = ext_index(x0 - hx + ix, X, bnd), gy = ext_index(y0 - hy + iy, Y, bnd);
        return (gt | gx | gy) >= 0 ? ((long long)gt * X + gx) * Y + gy : -1;
    };
    float pre[kPre][6];
    auto fetch = [&](int tp) {   // the first kPre * kThreads elements of plane tp into registers
        const int gt = ext_index(tp, T, bnd);
#pragma unroll
        for (int k = 0; k < kPre; ++k) {
            const int i = threadIdx.x + k * kThreads;
            const long long g = i < PE ? src(gt, i) : -1;
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                pre[k][m] = g >= 0 ? __ldg(E + m * NV + g) : 0.f;
                pre[k][3 + m] = g >= 0 ? __ldg(gS + m * gms + g) : 0.f;
            }
        }
    };
    auto store = [&](int tp) {   // registers into the ring slot of plane tp; the rest of the plane directly
        int sl = tp % R;
        sl += sl < 0 ? R : 0;
        float* dst = s_ring + (size_t)sl * PL;
#pragma unroll
        for (int k = 0; k < kPre; ++k) {
            const int i = threadIdx.x + k * kThreads;
            if (i < PE) {
#pragma unroll
                for (int c = 0; c < 6; ++c) dst[c * PE + i] = pre[k][c];
            }
        }
        const int gt = ext_index(tp, T, bnd);
        for (int i = threadIdx.x + kPre * kThreads; i < PE; i += kThreads) {
            const long long g = src(gt, i);
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                dst[m * PE + i] = g >= 0 ? __ldg(E + m * NV + g) : 0.f;
                dst[(3 + m) * PE + i] = g >= 0 ? __ldg(gS + m * gms + g) : 0.f;
            }
        }
    };
    for (int tp = ta - ht; tp <= ta + ht; ++tp) {   // planes ta - h_t .. ta + h_t
        fetch(tp);
        store(tp);
    }
    __syncthreads();
    int b = ta % R;   // ring slot of plane t, advanced step by step
    for (int t = ta; t < tb; ++t, b = b + 1 == R ? 0 : b + 1) {
        const bool more = t + 1 < tb;   // block-uniform
        if (more) fetch(t + 1 + ht);
        // every thread reaches the same two barriers of each step; only columns inside the volume compute
        if (col_ok) {
            const long long q = ((long long)t * X + x) * Y + y;
            float eq[3], gq[3], acc[3] = {0.f, 0.f, 0.f};
            const float* here = s_ring + (size_t)b * PL + (lx + hx) * TYH + (ly + hy);
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                eq[m] = here[m * PE];
                gq[m] = here[(3 + m) * PE];
            }
            // one offset of the interior path: the neighbour is q + o and the only preimage of q under offset
            // o is q - o; returns this voxel's term of the weight gradient of o (GW)
            auto interior = [&](int o) -> float {
                const int dt = s_d[o][0], dx = s_d[o][1], dy = s_d[o][2];
                const float w = s_w[o];
                // slots of planes t + dt and t - dt (|dt| <= h_t < R: one wrap at most)
                int sn = b + dt, sp = b - dt;
                sn += sn < 0 ? R : 0;
                sn -= sn >= R ? R : 0;
                sp += sp < 0 ? R : 0;
                sp -= sp >= R ? R : 0;
                const float* nb_p = s_ring + (size_t)sn * PL + (lx + hx + dx) * TYH + (ly + hy + dy);
                const float* pr_p = s_ring + (size_t)sp * PL + (lx + hx - dx) * TYH + (ly + hy - dy);
                float g = 0.f;
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const float nb = nb_p[m * PE];
                    const float pe = pr_p[m * PE], pg = pr_p[(3 + m) * PE];
                    const float own = sgnf(fmaf(-w, nb, eq[m])) * gq[m];
                    acc[m] += own;
                    acc[m] -= w * sgnf(fmaf(-w, eq[m], pe)) * pg;
                    if (GW) g = fmaf(own * cm[m], nb, g);
                }
                return g;
            };
            if (col_inner && t >= ht && t < T - ht) {
                if (GW) {
#pragma unroll
                    for (int o = 0; o < kGwMax; ++o)
                        if (o < Q) gw[o] += interior(o);
                } else {
#pragma unroll 2
                    for (int o = 0; o < Q; ++o) interior(o);
                }
            } else {
                const TileRing tr{s_ring, R, PL, PE, TXH, TYH, ht, hx, hy, x0, y0};
                dcs_adjoint_border_tile(E, gS, gms, T, X, Y, bnd, tr, s_d, s_w, Q, b, t, x, y, eq, gq, acc);
                if (GW) {
                    // the weight-gradient terms take the extended neighbour ext(q + o), staged for every voxel
#pragma unroll
                    for (int o = 0; o < kGwMax; ++o) {
                        if (o < Q) {
                            const float w = s_w[o];
                            const float* nb_p = s_ring + (size_t)tr.slot(b, s_d[o][0]) * PL +
                                                (lx + hx + s_d[o][1]) * TYH + (ly + hy + s_d[o][2]);
                            float g = 0.f;
#pragma unroll
                            for (int m = 0; m < 3; ++m) {
                                const float nb = nb_p[m * PE];
                                g = fmaf(sgnf(fmaf(-w, nb, eq[m])) * gq[m] * cm[m], nb, g);
                            }
                            gw[o] += g;
                        }
                    }
                }
            }
            gE[q] = acc[0] * c0 * st.invQ;
            gE[NV + q] = acc[1] * c1 * st.invQ;
            gE[2 * NV + q] = acc[2] * c2 * st.invQ;
        }
        __syncthreads();   // plane t - h_t is no longer read: its slot takes plane t + 1 + h_t
        if (more) store(t + 1 + ht);
        __syncthreads();
    }
    if (GW) {
        __shared__ double s_gw[kThreads / 32][kGwMax];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int o = 0; o < kGwMax; ++o) {
            float v = gw[o];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
            if (lane == 0) s_gw[wid][o] = (double)v;
        }
        __syncthreads();
        if (threadIdx.x < Q) {
            double a = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) a += s_gw[w][threadIdx.x];
            tpart[(size_t)blockIdx.x * Q + threadIdx.x] = a;
        }
    }
}

// Sums of the per-tile weight-gradient partials, one block per offset (fixed order: strided threads, then a
// tree), into part[o] (the single partial the finalize kernel then reads).
__global__ void __launch_bounds__(kThreads)
k4_gw_tiles_sum(const double* __restrict__ tpart, long long ntiles, int Q, double* __restrict__ part) {
    __shared__ double red[kThreads / 32];
    const int o = blockIdx.x;
    double a = 0.0;
    for (long long i = threadIdx.x; i < ntiles; i += kThreads) a += tpart[i * Q + o];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) a += __shfl_xor_sync(0xffffffffu, a, d);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
        part[o] = t;
    }
}

// FP64 partials of gw_o (before the -1/Q factor): one warp per 128 voxels of a (t, x) row, 4 per lane; for each offset the warp sums its voxels' terms (fixed shuffle tree) into a
// warp-private FP64 accumulator, and the warps' accumulators are summed in warp order.
__global__ void __launch_bounds__(kThreads)
k4_gw_partial(const float* __restrict__ E, const float* __restrict__ gS, long long gms, const float* __restrict__ coef,
              int T, int X, int Y, int bnd, const __grid_constant__ Stencil st, double* __restrict__ part) {
    constexpr int kWarps = kThreads / 32, kJ = 4;
    const long long NV = (long long)T * X * Y;
    const float c[3] = {coef[0], coef[1], coef[2]};
    __shared__ double wacc[kWarps][kMaxOffsets];
    __shared__ long long s_lin[kMaxOffsets];
    __shared__ float s_w[kMaxOffsets];
    for (int o = threadIdx.x; o < st.Q; o += kThreads) {
        s_lin[o] = ((long long)st.off[o][0] * X + st.off[o][1]) * Y + st.off[o][2];
        s_w[o] = st.w[o];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = lane; o < kMaxOffsets; o += 32) wacc[wid][o] = 0.0;
    __syncthreads();
    const int Q = st.Q;
    const int ht = st.halo[0], hx = st.halo[1], hy = st.halo[2];
    static_assert(32 * kJ == kYChunk, "one chunk per work item");
    const int nyc = (Y + kYChunk - 1) / kYChunk;
    for (long long it = (long long)blockIdx.x * kWarps + wid; it < (long long)T * X * nyc;
         it += (long long)gridDim.x * kWarps) {
        const long long r = it / nyc;
        const int t = (int)(r / X), x = (int)(r - (long long)t * X);
        const bool row_inner = t >= ht && t < T - ht && x >= hx && x < X - hx;
        {
            const int y0 = (int)(it - r * nyc) * kYChunk;   // warp-uniform
            float ep[kJ][3], gp[kJ][3];
            bool live[kJ], inner[kJ];
#pragma unroll
            for (int j = 0; j < kJ; ++j) {
                const int y = y0 + 32 * j + lane;
                live[j] = y < Y;
                inner[j] = row_inner && y >= hy && y < Y - hy;
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    ep[j][m] = live[j] ? __ldg(E + m * NV + r * Y + y) : 0.f;
                    gp[j][m] = live[j] ? c[m] * __ldg(gS + m * gms + r * Y + y) : 0.f;
                }
            }
            for (int o = 0; o < Q; ++o) {
                const float w = s_w[o];
                float s = 0.f;
#pragma unroll
                for (int j = 0; j < kJ; ++j) {
                    if (!live[j]) continue;
                    const int y = y0 + 32 * j + lane;
                    long long nq;
                    if (inner[j]) {
                        nq = r * Y + y + s_lin[o];
                    } else {
                        const int tt = ext_index(t + st.off[o][0], T, bnd), xx = ext_index(x + st.off[o][1], X, bnd),
                                  yy = ext_index(y + st.off[o][2], Y, bnd);
                        if ((tt | xx | yy) < 0) continue;
                        nq = ((long long)tt * X + xx) * Y + yy;
                    }
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        const float nb = __ldg(E + m * NV + nq);
                        s = fmaf(sgnf(fmaf(-w, nb, ep[j][m])) * gp[j][m], nb, s);
                    }
                }
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
                if (lane == 0) wacc[wid][o] += (double)s;
            }
        }
    }
    __syncthreads();
    for (int o = threadIdx.x; o < st.Q; o += kThreads) {
        double a = 0.0;
        for (int w = 0; w < kWarps; ++w) a += wacc[w][o];
        part[blockIdx.x * 64 + o] = a;
    }
}

// galpha_d = sum_{o in d} g_o gw_o, gw_o = -(1/Q) sum_blocks part[block][o].  One block; one warp per
// offset sums its partials in a fixed order (strided lanes, then a shuffle tree).
__global__ void __launch_bounds__(kThreads)
k4_galpha_finalize(const double* __restrict__ part, int nparts, const __grid_constant__ Stencil st,
                   float* __restrict__ galpha) {
    __shared__ double gw[kMaxOffsets];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = wid; o < st.Q; o += kThreads / 32) {
        double a = 0.0;
        for (int i = lane; i < nparts; i += 32) a += part[i * 64 + o];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) a += __shfl_xor_sync(0xffffffffu, a, d);
        if (lane == 0) gw[o] = -a / st.Q;
    }
    __syncthreads();
    if (threadIdx.x < st.n_dirs) {
        double a = 0.0;
        for (int o = 0; o < st.Q; ++o)
            if (st.dir[o] == (int)threadIdx.x) a += (double)st.g[o] * gw[o];
        galpha[threadIdx.x] = (float)a;
    }
}

// Overlap-add of the spectral adjoint, in two passes.  The bricks of t0 = t_begin + r t_step, r < t_count
// (t_step > 1: the lattice planes of stride-s windows), hold blocks [u_t][x'][y'] (u_t < n, x' < XH,
// y' < YH); brick (xs, sg) covers x_ext in [xs*BX - n/2, xs*BX - n/2 + XH), y_ext likewise with BY, YH;
// slice u_t of brick t0 lies at t_ext = t0 - n/2 + u_t.
//   pass 1 (along t): ext[i][brick][x'][y'] = sum over t0 of the slices at t_ext = t_begin - n/2 + i, for
//     every extended plane i < t_step (t_count - 1) + n -- contiguous slices, read once;
//   pass 2 (across bricks): gV[q] += sum of ext over the extended positions (t_ext, x_ext, y_ext) that
//     map to q and the bricks that hold them.
// Both passes sum in a fixed order, so the result is deterministic.
// Pass 1: one warp per (plane i, brick) row of `slice` contiguous floats (slice4 = slice / 4 16-byte groups:
// the blocks' slices are padded to a multiple of 4 floats), lanes along the row.
__global__ void __launch_bounds__(kThreads)
k5_gather_t(const float4* __restrict__ blocks, float4* __restrict__ ext, int n, int nb, int slice4, int t_count,
            int t_step) {
    constexpr int kWarps = kThreads / 32;
    const int lane = threadIdx.x & 31;
    const long long bsz = (long long)n * slice4;
    const long long rows = (long long)(t_step * (t_count - 1) + n) * nb;
    // from the slice of brick r to that of brick r + 1 on the same plane: the next t0's block, u_t - t_step
    const long long rstep = (long long)nb * bsz - (long long)t_step * slice4;
    for (long long w = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5); w < rows;
         w += (long long)gridDim.x * kWarps) {
        const int brick = (int)(w % nb), i = (int)(w / nb);
        // the bricks r whose slice u_t = i - t_step r (< n) lands on plane i, in increasing r
        const int r_lo = i >= n ? (i - n + t_step) / t_step : 0;
        const int nr = min(t_count - 1, i / t_step) - r_lo + 1;   // at most 16 (n <= 16)
        const float4* src = blocks + ((long long)r_lo * nb + brick) * bsz + (long long)(i - t_step * r_lo) * slice4;
        float4* dst = ext + w * slice4;
        for (int e = lane; e < slice4; e += 32) {
            float4 v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = j < nr ? __ldg(src + j * rstep + e) : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                sum.x += v[j].x;
                sum.y += v[j].y;
                sum.z += v[j].z;
                sum.w += v[j].w;
            }
            dst[e] = sum;
        }
    }
}

// Pass 2: one thread per voxel; block (32 y, 8 x) of plane t = t_lo + blockIdx.z.
__global__ void __launch_bounds__(kThreads)
k5_gather_xy(const float* __restrict__ ext, float* __restrict__ gV, int T, int X, int Y, int bnd, int n, int BX,
             int XH, int BY, int YH, int slice, int t_begin, int t_count, int t_step, int t_lo) {
    const int h2 = n / 2;
    const int nseg = (Y + BY - 1) / BY;
    const int nxs = (X + BX - 1) / BX;
    const int nb = nxs * nseg;
    const int te_lo = t_begin - h2, te_hi = t_begin + t_step * (t_count - 1) + h2;   // extended planes of this slab
    const int t = t_lo + blockIdx.z, x = blockIdx.y * 8 + threadIdx.y, y = blockIdx.x * 32 + threadIdx.x;
    if (x >= X || y >= Y) return;
    const long long q = ((long long)t * X + x) * Y + y;
    if (t >= h2 && t < T - h2 && x >= h2 && x < X - h2 && y >= h2 && y < Y - h2) {
        // interior voxel: its only extended position is itself
        if (t < te_lo || t >= te_hi) return;
        const int xa = max(0, ceildiv(x + h2 - XH + 1, BX)), xb = min(nxs - 1, floordiv(x + h2, BX));
        const int sa = max(0, ceildiv(y + h2 - YH + 1, BY)), sb = min(nseg - 1, floordiv(y + h2, BY));
        const float* plane = ext + (long long)(t - te_lo) * nb * slice;
        float sum = 0.f;
        if (xb - xa < 4 && sb - sa < 2) {
            // up to 4 x 2 bricks (the tensor-core geometries): every load issued before the sums, which run in
            // the loop order below (x brick outer, y segment inner)
            float v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int xs = xa + k / 2, sg = sa + k % 2;
                v[k] = xs <= xb && sg <= sb ? __ldg(plane + (long long)(xs * nseg + sg) * slice + (x - xs * BX + h2) * YH +
                                                   (y - sg * BY + h2))
                                            : 0.f;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (xa + k / 2 <= xb && sa + k % 2 <= sb) sum += v[k];
        } else {
            for (int xs = xa; xs <= xb; ++xs)
                for (int sg = sa; sg <= sb; ++sg)
                    sum += __ldg(plane + (long long)(xs * nseg + sg) * slice + (x - xs * BX + h2) * YH +
                                 (y - sg * BY + h2));
        }
        gV[q] += sum;
        return;
    }
    int et[40], ex[40], ey[40];
    const int nt = pre_range(t, T, bnd, te_lo, te_hi, et, 40);
    if (nt == 0) return;
    const int nx = pre_range(x, X, bnd, -h2, X + h2 - 1, ex, 40);
    const int ny = pre_range(y, Y, bnd, -h2, Y + h2 - 1, ey, 40);
    float sum = 0.f;
    for (int a = 0; a < nt; ++a) {
        const float* plane = ext + (long long)(et[a] - te_lo) * nb * slice;
        for (int b = 0; b < nx; ++b) {
            const int xe = ex[b];
            const int xa = max(0, ceildiv(xe + h2 - XH + 1, BX)), xb = min(nxs - 1, floordiv(xe + h2, BX));
            for (int xs = xa; xs <= xb; ++xs) {
                const int ux = xe - xs * BX + h2;
                for (int c = 0; c < ny; ++c) {
                    const int ye = ey[c];
                    const int sa = max(0, ceildiv(ye + h2 - YH + 1, BY));
                    const int sb = min(nseg - 1, floordiv(ye + h2, BY));
                    for (int sg = sa; sg <= sb; ++sg)
                        sum += __ldg(plane + (long long)(xs * nseg + sg) * slice + ux * YH + (ye - sg * BY + h2));
                }
            }
        }
    }
    gV[q] += sum;
}

// gS3[m][p] = coef[m] * gS[p]
__global__ void __launch_bounds__(kThreads)
kb_expand(const float* __restrict__ gS, const float* __restrict__ coef, float* __restrict__ gS3, long long NV) {
    const float c0 = coef[0], c1 = coef[1], c2 = coef[2];
    for (long long p = (long long)blockIdx.x * kThreads + threadIdx.x; p < NV; p += (long long)gridDim.x * kThreads) {
        const float g = __ldg(gS + p);
        gS3[p] = c0 * g;
        gS3[NV + p] = c1 * g;
        gS3[2 * NV + p] = c2 * g;
    }
}

}  // namespace

cudaError_t expand_gradient_launch(const float* gS, const float* coef, float* gS3, long long N, cudaStream_t s) {
    kb_expand<<<red_blocks(N), kThreads, 0, s>>>(gS, coef, gS3, N);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t backward_weights_launch(const float* S3, const float* gS, long long N, const Reduce& r, double* part,
                                    float* coef, float* gW, cudaStream_t s) {
    const int nb = red_blocks(N);
    kb_weights_partial<<<nb, kThreads, 0, s>>>(S3, gS, N, r.norm, part);
    kb_weights_finalize<<<1, kThreads, 0, s>>>(part, nb, r.norm, coef, gW);
    note_launches(2);
    return cudaGetLastError();
}

// The tiled kernel holds one block per tile for all its planes; with fewer tiles than two waves of
// resident blocks (3 per SM) it leaves SMs idle, and the row kernel, whose warps cover every row, is faster.
static int g_tiled_min_blocks = 2 * 3 * 152;   // set from the device's SM count by dcs_adjoint_prepare

cudaError_t dcs_adjoint_prepare() {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_tiled_min_blocks = 2 * 3 * sms;
    e = cudaFuncSetAttribute(k4_dcs_adjoint_tiled<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kTileSmemMax);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k4_dcs_adjoint_tiled<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kTileSmemMax);
}

cudaError_t dcs_adjoint_launch(const float* E, const float* gS, long long gms, const float* coef, float* gE, int T,
                               int X, int Y, int bnd, const Stencil& st, cudaStream_t s) {
    const long long NV = (long long)T * X * Y;
    const size_t smem = dcs_tile_smem_bytes(st.halo[0], st.halo[1], st.halo[2]);
    const long long nblk = (long long)((T + kTileT - 1) / kTileT) * ((X + kTX - 1) / kTX) * ((Y + kTY - 1) / kTY);
    // the tiled kernel when its plane ring fits (dcs_adjoint_prepare), its tiles fill the GPU and their
    // count fits a one-dimensional grid; the row kernel otherwise
    if (smem <= kTileSmemMax && nblk >= g_tiled_min_blocks && nblk <= 0x7fffffffLL) {
        k4_dcs_adjoint_tiled<false><<<(int)nblk, kThreads, smem, s>>>(E, gS, gms, coef, gE, T, X, Y, bnd, st, nullptr);
        note_launches(1);
        return cudaGetLastError();
    }
    k4_dcs_adjoint<<<red_blocks(NV), kThreads, 0, s>>>(E, gS, gms, coef, gE, T, X, Y, bnd, st);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t dcs_adjoint_galpha_launch(const float* E, const float* gS, long long gms, const float* coef, float* gE,
                                      int T, int X, int Y, int bnd, const Stencil& st, double* tile_part,
                                      size_t tile_part_bytes, double* part, float* galpha, cudaStream_t s) {
    const size_t smem = dcs_tile_smem_bytes(st.halo[0], st.halo[1], st.halo[2]);
    const long long nblk = (long long)((T + kTileT - 1) / kTileT) * ((X + kTX - 1) / kTX) * ((Y + kTY - 1) / kTY);
    const bool fused = smem <= kTileSmemMax && nblk >= g_tiled_min_blocks && nblk <= 0x7fffffffLL &&
                       st.Q <= kGwMax && tile_part && (size_t)nblk * st.Q * sizeof(double) <= tile_part_bytes;
    if (!fused) {
        cudaError_t e = dcs_galpha_launch(E, gS, gms, coef, T, X, Y, bnd, st, part, galpha, s);
        if (e != cudaSuccess) return e;
        return dcs_adjoint_launch(E, gS, gms, coef, gE, T, X, Y, bnd, st, s);
    }
    k4_dcs_adjoint_tiled<true><<<(int)nblk, kThreads, smem, s>>>(E, gS, gms, coef, gE, T, X, Y, bnd, st, tile_part);
    k4_gw_tiles_sum<<<st.Q, kThreads, 0, s>>>(tile_part, nblk, st.Q, part);
    k4_galpha_finalize<<<1, kThreads, 0, s>>>(part, 1, st, galpha);
    note_launches(3);
    return cudaGetLastError();
}

cudaError_t dcs_galpha_launch(const float* E, const float* gS, long long gms, const float* coef, int T, int X, int Y,
                              int bnd, const Stencil& st, double* part, float* galpha, cudaStream_t s) {
    const long long NV = (long long)T * X * Y;
    const int nb = red_blocks(NV);
    k4_gw_partial<<<nb, kThreads, 0, s>>>(E, gS, gms, coef, T, X, Y, bnd, st, part);
    k4_galpha_finalize<<<1, kThreads, 0, s>>>(part, nb, st, galpha);
    note_launches(2);
    return cudaGetLastError();
}

size_t gather_ext_floats(int n, SpectraAdjointGeometry g, int X, int Y, int t_count, int t_step) {
    const size_t nb = (size_t)((X + g.BX - 1) / g.BX) * ((Y + g.BY - 1) / g.BY);
    return (size_t)(t_step * (t_count - 1) + n) * nb * g.slice;
}

cudaError_t gather_add_launch(const float* blocks, float* ext, float* gV, int T, int X, int Y, int bnd, int n,
                              SpectraAdjointGeometry g, int t_begin, int t_count, int t_step, cudaStream_t s) {
    if (n > 16 || t_step < 1) return cudaErrorInvalidValue;   // pass 1 unrolls up to 16 bricks per plane
    const int nb = ((X + g.BX - 1) / g.BX) * ((Y + g.BY - 1) / g.BY);
    const long long e_total = (long long)gather_ext_floats(n, g, X, Y, t_count, t_step);
    if (g.slice % 4 != 0) return cudaErrorInvalidValue;   // pass 1 moves 16-byte groups
    const long long rows1 = e_total / g.slice;   // (plane, brick) rows, a warp each
    long long b1 = (rows1 + kThreads / 32 - 1) / (kThreads / 32);
    const long long cap1 = 8LL * device_sms();   // grid-stride: 8 blocks per SM
    if (b1 > cap1) b1 = cap1;
    if (b1 < 1) b1 = 1;
    k5_gather_t<<<(int)b1, kThreads, 0, s>>>(reinterpret_cast<const float4*>(blocks), reinterpret_cast<float4*>(ext),
                                             n, nb, g.slice / 4, t_count, t_step);
    // planes the slab reaches: extended t in [t_begin - n/2, t_begin + t_step (t_count - 1) + n/2); a slab
    // whose extension leaves the volume may wrap (periodic) or reflect (symmetric) onto any edge plane
    const int h2 = n / 2;
    int t_lo = t_begin - h2, t_hi = t_begin + t_step * (t_count - 1) + h2;
    if (t_lo < 0 || t_hi > T) {
        t_lo = 0;
        t_hi = T;
    }
    static_assert(kThreads == 32 * 8, "pass 2 blocks are 32 y x 8 x");
    const dim3 grid2((Y + 31) / 32, (X + 7) / 8, t_hi - t_lo);   // T, X <= 65535 (checked at create)
    k5_gather_xy<<<grid2, dim3(32, 8), 0, s>>>(ext, gV, T, X, Y, bnd, n, g.BX, g.XH, g.BY, g.YH, g.slice, t_begin,
                                              t_count, t_step, t_lo);
    note_launches(2);
    return cudaGetLastError();
}

}  // namespace sal
