// Features of stride-s windows back to every voxel (the ">50% overlap" of Sec. 2 step 1 read as cubes
// only at voxels whose indices are multiples of s, s < n/2).  Along each axis a voxel i between the
// lattice points a = s floor(i/s) and a + s takes (1 - f) E(a) + f E(a + s), f = (i - a)/s; past the last
// lattice point of the axis it takes that point's value.  Applied along all three axes (trilinear).
// HBM-bound: each output voxel is written once (12 B); the lattice (1/s^3 of that) is read from L2.
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

}  // namespace

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
