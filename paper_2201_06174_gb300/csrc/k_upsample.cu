// Features of stride-s windows back to every voxel (the ">50% overlap" of Sec. 2 step 1 read as cubes
// only at voxels whose indices are multiples of s, s < n/2).  Along each axis a voxel i between the
// lattice points a = s floor(i/s) and a + s takes (1 - f) E(a) + f E(a + s), f = (i - a)/s; past the last
// lattice point of the axis it takes that point's value.  Applied along all three axes (trilinear).
// HBM-bound: each output voxel is written once (12 B); the lattice (1/s^3 of that) is read from L2.  The
// adjoint (for the backward) gathers every voxel's gradient back onto the lattice with the same weights.
#include "sal_internal.cuh"

namespace sal {
namespace {

constexpr int kThreads = 256;

// Lattice index and weight of the upper neighbour along one axis (L lattice points).
__device__ __forceinline__ void axis_weights(int i, int s, int L, int& a, int& b, float& f) {
    a = i / s;
    const int r = i - a * s;
    b = a + 1 < L ? a + 1 : a;
    f = b == a ? 0.f : (float)r / (float)s;
}

// One warp per (t, x) row, lanes along y.
__global__ void __launch_bounds__(kThreads)
k1_upsample(const float* __restrict__ Ec, float* __restrict__ E, int T, int X, int Y, int s) {
    constexpr int kWarps = kThreads / 32;
    const int Tc = (T + s - 1) / s, Xc = (X + s - 1) / s, Yc = (Y + s - 1) / s;
    const long long NV = (long long)T * X * Y, NVc = (long long)Tc * Xc * Yc;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (long long r = (long long)blockIdx.x * kWarps + wid; r < (long long)T * X; r += (long long)gridDim.x * kWarps) {
        const int t = (int)(r / X), x = (int)(r - (long long)t * X);
        int ta, tb, xa, xb;
        float ft, fx;
        axis_weights(t, s, Tc, ta, tb, ft);
        axis_weights(x, s, Xc, xa, xb, fx);
        const long long c00 = ((long long)ta * Xc + xa) * Yc, c01 = ((long long)ta * Xc + xb) * Yc;
        const long long c10 = ((long long)tb * Xc + xa) * Yc, c11 = ((long long)tb * Xc + xb) * Yc;
        for (int y = lane; y < Y; y += 32) {
            int ya, yb;
            float fy;
            axis_weights(y, s, Yc, ya, yb, fy);
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const float* e = Ec + m * NVc;
                // along y, then x, then t
                const float v00 = fmaf(fy, __ldg(e + c00 + yb) - __ldg(e + c00 + ya), __ldg(e + c00 + ya));
                const float v01 = fmaf(fy, __ldg(e + c01 + yb) - __ldg(e + c01 + ya), __ldg(e + c01 + ya));
                const float v10 = fmaf(fy, __ldg(e + c10 + yb) - __ldg(e + c10 + ya), __ldg(e + c10 + ya));
                const float v11 = fmaf(fy, __ldg(e + c11 + yb) - __ldg(e + c11 + ya), __ldg(e + c11 + ya));
                const float v0 = fmaf(fx, v01 - v00, v00), v1 = fmaf(fx, v11 - v10, v10);
                E[m * NV + r * Y + y] = fmaf(ft, v1 - v0, v0);
            }
        }
    }
}

// Adjoint weight of voxel i for lattice point c along one axis (L lattice points): 1 - f if c is its lower
// point, f if its upper one (1 past the last lattice point).
__device__ __forceinline__ float axis_adjoint_weight(int i, int c, int s, int L) {
    int a, b;
    float f;
    axis_weights(i, s, L, a, b, f);
    return (a == c ? 1.f - f : 0.f) + (b == c && b != a ? f : 0.f);
}

// Transpose of k1_upsample: each lattice point c gathers, in a fixed order, the gradients of the voxels
// interpolated from it, and writes them at its own voxel of gEl [3][T][X][Y] (the other voxels of gEl
// are left as they are: zero).
__global__ void __launch_bounds__(kThreads)
k5_upsample_adjoint(const float* __restrict__ gE, float* __restrict__ gEl, int T, int X, int Y, int s) {
    const int Tc = (T + s - 1) / s, Xc = (X + s - 1) / s, Yc = (Y + s - 1) / s;
    const long long NV = (long long)T * X * Y, NVc = (long long)Tc * Xc * Yc;
    for (long long c = (long long)blockIdx.x * kThreads + threadIdx.x; c < NVc; c += (long long)gridDim.x * kThreads) {
        const int yc = (int)(c % Yc), xc = (int)((c / Yc) % Xc), tc = (int)(c / ((long long)Xc * Yc));
        // voxels interpolated from this lattice point, per axis: (c - 1) s < i < (c + 1) s, and every
        // voxel past the last lattice point
        const int t_lo = max(0, s * (tc - 1) + 1), t_hi = tc == Tc - 1 ? T - 1 : min(T - 1, s * (tc + 1) - 1);
        const int x_lo = max(0, s * (xc - 1) + 1), x_hi = xc == Xc - 1 ? X - 1 : min(X - 1, s * (xc + 1) - 1);
        const int y_lo = max(0, s * (yc - 1) + 1), y_hi = yc == Yc - 1 ? Y - 1 : min(Y - 1, s * (yc + 1) - 1);
        float acc[3] = {0.f, 0.f, 0.f};
        for (int t = t_lo; t <= t_hi; ++t) {
            const float wt = axis_adjoint_weight(t, tc, s, Tc);
            for (int x = x_lo; x <= x_hi; ++x) {
                const float wtx = wt * axis_adjoint_weight(x, xc, s, Xc);
                const long long row = ((long long)t * X + x) * Y;
                for (int y = y_lo; y <= y_hi; ++y) {
                    const float w = wtx * axis_adjoint_weight(y, yc, s, Yc);
#pragma unroll
                    for (int m = 0; m < 3; ++m) acc[m] = fmaf(w, __ldg(gE + m * NV + row + y), acc[m]);
                }
            }
        }
        const long long v = ((long long)(s * tc) * X + s * xc) * Y + s * yc;
#pragma unroll
        for (int m = 0; m < 3; ++m) gEl[m * NV + v] = acc[m];
    }
}

}  // namespace

cudaError_t upsample_adjoint_launch(const float* gE, float* gEl, int T, int X, int Y, int stride, cudaStream_t s) {
    if (stride < 2) return cudaErrorInvalidValue;
    const long long NVc = (long long)((T + stride - 1) / stride) * ((X + stride - 1) / stride) *
                          ((Y + stride - 1) / stride);
    long long nb = (NVc + kThreads - 1) / kThreads;
    const long long cap = 32LL * device_sms();   // grid-stride: 32 blocks per SM
    if (nb > cap) nb = cap;
    if (nb < 1) nb = 1;
    k5_upsample_adjoint<<<(int)nb, kThreads, 0, s>>>(gE, gEl, T, X, Y, stride);
    note_launches(1);
    return cudaGetLastError();
}

// One warp per row of V, lanes along y (coalesced on both sides); HBM-bound, 8 B per voxel.
__global__ void __launch_bounds__(kThreads)
k_pad_rows(const float* __restrict__ V, float* __restrict__ Vp, long long rows, int Y, int Ypad) {
    constexpr int kWarps = kThreads / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (long long r = (long long)blockIdx.x * kWarps + wid; r < rows; r += (long long)gridDim.x * kWarps) {
        const float* src = V + r * Y;
        float* dst = Vp + r * Ypad;
        for (int y = lane; y < Y; y += 32) dst[y] = __ldg(src + y);
    }
}

cudaError_t pad_rows_launch(const float* V, float* Vp, long long rows, int Y, int Ypad, cudaStream_t s) {
    if (Y < 1 || Ypad < Y || rows < 1) return cudaErrorInvalidValue;
    long long nb = (rows + kThreads / 32 - 1) / (kThreads / 32);
    const long long cap = 16LL * device_sms();
    if (nb > cap) nb = cap;
    k_pad_rows<<<(int)nb, kThreads, 0, s>>>(V, Vp, rows, Y, Ypad);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t upsample_launch(const float* Ec, float* E, int T, int X, int Y, int stride, cudaStream_t s) {
    if (stride < 1) return cudaErrorInvalidValue;
    const long long rows = (long long)T * X;
    long long nb = (rows + kThreads / 32 - 1) / (kThreads / 32);
    if (nb > kRedBlocks) nb = kRedBlocks;
    if (nb < 1) nb = 1;
    k1_upsample<<<(int)nb, kThreads, 0, s>>>(Ec, E, T, X, Y, stride);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace sal
