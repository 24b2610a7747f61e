// K2: directional center-surround comparison (Sec. 2 step 4, Eq. 3; windows of Fig. 4)
//   S_m[p] = (1/Q) sum_o | E_m[p] - w_o * Eext_m[p + o] |,   m in {t, x, y},
// in compensated FP32: each difference is formed by one FMA (fmaf(-w, e_nb, e_c): the product is
// not rounded before the subtraction) and the Q distances are summed with Kahan compensation.
// HBM-bound: 12 B read + 12 B written per voxel; neighbours come from L1/L2.  One warp per 128 voxels of
// a (t, x) row;
// voxels the halo away from every border take the stencil as linear offsets, the others go through the
// border extension.  Fused per-block min/max of each S_m for the normalisation in K3.
#include <cfloat>

#include "sal_internal.cuh"

namespace sal {
namespace {

constexpr int kThreads = 256;
constexpr int kYChunk = 128;   // voxels of a row per warp work item

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__global__ void __launch_bounds__(kThreads)
k2_dcs(const float* __restrict__ E, float* __restrict__ S3, int T, int X, int Y, int bnd,
       const __grid_constant__ Stencil st, float* __restrict__ mm_part) {
    constexpr int kWarps = kThreads / 32;
    const long long NV = (long long)T * X * Y;
    // linear offset of each neighbour: the whole comparison of a voxel at least the halo away from every
    // border reads E at p + s_lin[o]
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
    float mn[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, mx[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    // one warp per 128-voxel chunk of a (t, x) row, lanes along y
    const int nyc = (Y + kYChunk - 1) / kYChunk;
    for (long long it = (long long)blockIdx.x * kWarps + wid; it < (long long)T * X * nyc;
         it += (long long)gridDim.x * kWarps) {
        const long long r = it / nyc;
        const int yc = (int)(it - r * nyc) * kYChunk, ye = min(Y, yc + kYChunk);
        const int t = (int)(r / X), x = (int)(r - (long long)t * X);
        const bool row_inner = t >= ht && t < T - ht && x >= hx && x < X - hx;
        for (int y = yc + lane; y < ye; y += 32) {
            const long long p = r * Y + y;
            float ec[3], acc[3] = {0.f, 0.f, 0.f}, cmp[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int m = 0; m < 3; ++m) ec[m] = __ldg(E + m * NV + p);
            if (row_inner && y >= hy && y < Y - hy) {
#pragma unroll 2
                for (int o = 0; o < Q; ++o) {
                    const float* e = E + p + s_lin[o];
                    const float w = s_w[o];
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        // Kahan: acc + cmp carries the sum to about twice the FP32 precision
                        const float yv = fabsf(fmaf(-w, __ldg(e + m * NV), ec[m])) - cmp[m];
                        const float tv = acc[m] + yv;
                        cmp[m] = (tv - acc[m]) - yv;
                        acc[m] = tv;
                    }
                }
            } else {
                for (int o = 0; o < Q; ++o) {
                    const int tt = ext_index(t + st.off[o][0], T, bnd);
                    const int xx = ext_index(x + st.off[o][1], X, bnd);
                    const int yy = ext_index(y + st.off[o][2], Y, bnd);
                    const bool ok = tt >= 0 && xx >= 0 && yy >= 0;
                    const long long q = ok ? ((long long)tt * X + xx) * Y + yy : 0;
                    const float w = s_w[o];
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        const float nb = ok ? __ldg(E + m * NV + q) : 0.f;
                        const float yv = fabsf(fmaf(-w, nb, ec[m])) - cmp[m];
                        const float tv = acc[m] + yv;
                        cmp[m] = (tv - acc[m]) - yv;
                        acc[m] = tv;
                    }
                }
            }
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const float s = acc[m] * st.invQ;
                S3[m * NV + p] = s;
                mn[m] = fminf(mn[m], s);
                mx[m] = fmaxf(mx[m], s);
            }
        }
    }
    __shared__ float red[kThreads / 32][6];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        float a = warp_min(mn[m]), b = warp_max(mx[m]);
        if (lane == 0) {
            red[wid][m] = a;
            red[wid][3 + m] = b;
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int c = threadIdx.x;
        float v = red[0][c];
        for (int w = 1; w < kThreads / 32; ++w) v = c < 3 ? fminf(v, red[w][c]) : fmaxf(v, red[w][c]);
        mm_part[blockIdx.x * 8 + c] = v;
    }
}

}  // namespace

cudaError_t dcs_launch(const float* E, float* S3, int T, int X, int Y, int bnd, const Stencil& st,
                       float* mm_part, cudaStream_t s) {
    const long long NV = (long long)T * X * Y;
    const int blocks = red_blocks(NV);  // K3 reduces exactly this many min/max partials
    k2_dcs<<<blocks, kThreads, 0, s>>>(E, S3, T, X, Y, bnd, st, mm_part);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace sal
