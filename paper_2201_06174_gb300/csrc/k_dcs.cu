// K2: directional center-surround comparison (Sec. 2 step 4, Eq. 3; windows of Fig. 4)
//   S_m[p] = (1/Q) sum_o | E_m[p] - w_o * Eext_m[p + o] |,   m in {t, x, y},
// in compensated FP32: each difference is formed by one FMA (fmaf(-w, e_nb, e_c): the product is
// not rounded before the subtraction) and the Q distances are summed with Kahan compensation.
// HBM-class: 12 B read + 12 B written per voxel.  Two forms with the same per-voxel sums: k2_dcs_tiled
// (windows whose plane ring fits 96 KB of shared memory, the default among them, on volumes with at least
// a wave of tiles) stages E in tiles with their halos; k2_dcs, one warp per 128 voxels of a (t, x) row,
// reads the neighbours from L1/L2 (voxels the halo away from every border at linear offsets, the others
// through the border extension).
// Both fuse the per-block min/max of each S_m for the normalisation in K3.
#include <algorithm>
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

// K2, ring-staged: the same sums, with E read from global memory about once per tile.  A tile is 16 x 16
// (x, y) columns (a thread each) and up to 16 planes along t; E of the tile and its halo streams through a
// ring of 2 h_t + 1 planes in shared memory with the border extension applied at load, so every voxel,
// at the border or not, reads its neighbours ext(p + o) from the ring in the order of the offsets (the
// result is that of k2_dcs bit for bit).  The next plane is fetched into registers while the current one
// is computed.  Blocks are persistent over the tiles (as many as fit on the GPU at once); each keeps the
// min/max of its outputs, and partial slots beyond the grid get neutral values (K3 reads a fixed count).
constexpr int kTX = 16, kTY = 16, kTT = 16;
constexpr int kPre = 2;   // plane elements per thread prefetched into registers (the rest loaded at store)
static_assert(kTX * kTY == kThreads, "one column per thread");

__host__ __device__ inline size_t ring_bytes(int ht, int hx, int hy) {
    return (size_t)(2 * ht + 1) * 3 * (kTX + 2 * hx) * (kTY + 2 * hy) * sizeof(float);
}

__global__ void __launch_bounds__(kThreads)
k2_dcs_tiled(const float* __restrict__ E, float* __restrict__ S3, int T, int X, int Y, int bnd,
             const __grid_constant__ Stencil st, float* __restrict__ mm_part, int nparts) {
    extern __shared__ float s_ring[];   // [2 h_t + 1][3][TXH][TYH]
    __shared__ float s_w[kMaxOffsets];
    __shared__ int s_d[kMaxOffsets][3];
    const long long NV = (long long)T * X * Y;
    const int ht = st.halo[0], hx = st.halo[1], hy = st.halo[2];
    const int R = 2 * ht + 1, TXH = kTX + 2 * hx, TYH = kTY + 2 * hy, PE = TXH * TYH, PL = 3 * PE;
    for (int o = threadIdx.x; o < st.Q; o += kThreads) {
        s_w[o] = st.w[o];
        s_d[o][0] = st.off[o][0];
        s_d[o][1] = st.off[o][1];
        s_d[o][2] = st.off[o][2];
    }
    const int Q = st.Q;
    const int ntx = (X + kTX - 1) / kTX, nty = (Y + kTY - 1) / kTY, ntt = (T + kTT - 1) / kTT;
    const long long ntiles = (long long)ntx * nty * ntt;
    const int lx = threadIdx.x / kTY, ly = threadIdx.x % kTY;
    float mn[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, mx[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    __syncthreads();
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int tyi = (int)(tile % nty), txi = (int)((tile / nty) % ntx), tti = (int)(tile / ((long long)nty * ntx));
        const int x0 = txi * kTX, y0 = tyi * kTY, ta = tti * kTT, tb = min(T, ta + kTT);
        const int x = x0 + lx, y = y0 + ly;
        const bool col_ok = x < X && y < Y;
        // global index of element i (< PE) of extended plane gt, or -1 outside a zero-extended volume
        auto src = [&](int gt, int i) -> long long {
            const int ix = i / TYH, iy = i - ix * TYH;
            const int gx = ext_index(x0 - hx + ix, X, bnd), gy = ext_index(y0 - hy + iy, Y, bnd);
            return (gt | gx | gy) >= 0 ? ((long long)gt * X + gx) * Y + gy : -1;
        };
        float pre[kPre][3];
        auto fetch = [&](int tp) {   // the first kPre * kThreads elements of plane tp into registers
            const int gt = ext_index(tp, T, bnd);
#pragma unroll
            for (int k = 0; k < kPre; ++k) {
                const int i = threadIdx.x + k * kThreads;
                const long long g = i < PE ? src(gt, i) : -1;
#pragma unroll
                for (int m = 0; m < 3; ++m) pre[k][m] = g >= 0 ? __ldg(E + m * NV + g) : 0.f;
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
                    for (int m = 0; m < 3; ++m) dst[m * PE + i] = pre[k][m];
                }
            }
            const int gt = ext_index(tp, T, bnd);
            for (int i = threadIdx.x + kPre * kThreads; i < PE; i += kThreads) {
                const long long g = src(gt, i);
#pragma unroll
                for (int m = 0; m < 3; ++m) dst[m * PE + i] = g >= 0 ? __ldg(E + m * NV + g) : 0.f;
            }
        };
        for (int tp = ta - ht; tp <= ta + ht; ++tp) {   // planes ta - h_t .. ta + h_t
            fetch(tp);
            store(tp);
        }
        __syncthreads();
        int b = ta % R;   // ring slot of plane t
        for (int t = ta; t < tb; ++t, b = b + 1 == R ? 0 : b + 1) {
            const bool more = t + 1 < tb;   // block-uniform
            if (more) fetch(t + 1 + ht);
            if (col_ok) {
                const float* here = s_ring + (size_t)b * PL + (lx + hx) * TYH + (ly + hy);
                float ec[3], acc[3] = {0.f, 0.f, 0.f}, cmp[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int m = 0; m < 3; ++m) ec[m] = here[m * PE];
#pragma unroll 2
                for (int o = 0; o < Q; ++o) {
                    int sl = b + s_d[o][0];   // |dt| <= h_t < R: one wrap at most
                    sl += sl < 0 ? R : 0;
                    sl -= sl >= R ? R : 0;
                    const float* nb = s_ring + (size_t)sl * PL + (lx + hx + s_d[o][1]) * TYH + (ly + hy + s_d[o][2]);
                    const float w = s_w[o];
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        // Kahan: acc + cmp carries the sum to about twice the FP32 precision
                        const float yv = fabsf(fmaf(-w, nb[m * PE], ec[m])) - cmp[m];
                        const float tv = acc[m] + yv;
                        cmp[m] = (tv - acc[m]) - yv;
                        acc[m] = tv;
                    }
                }
                const long long p = ((long long)t * X + x) * Y + y;
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const float sv = acc[m] * st.invQ;
                    S3[m * NV + p] = sv;
                    mn[m] = fminf(mn[m], sv);
                    mx[m] = fmaxf(mx[m], sv);
                }
            }
            __syncthreads();   // plane t - h_t is no longer read: its slot takes plane t + 1 + h_t
            if (more) store(t + 1 + ht);
            __syncthreads();
        }
    }
    __shared__ float red[kThreads / 32][6];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const float a = warp_min(mn[m]), c = warp_max(mx[m]);
        if (lane == 0) {
            red[wid][m] = a;
            red[wid][3 + m] = c;
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int c = threadIdx.x;
        float v = red[0][c];
        for (int w = 1; w < kThreads / 32; ++w) v = c < 3 ? fminf(v, red[w][c]) : fmaxf(v, red[w][c]);
        mm_part[blockIdx.x * 8 + c] = v;
    }
    // the slots of the partials no block of this grid fills: neutral (min +inf-like, max -inf-like)
    if (blockIdx.x == 0)
        for (int i = gridDim.x * 8 + threadIdx.x; i < nparts * 8; i += kThreads)
            mm_part[i] = (i % 8) < 3 ? FLT_MAX : -FLT_MAX;
}

constexpr size_t kRingMax = 96 * 1024;   // windows whose ring is larger take the row kernel

}  // namespace

cudaError_t dcs_prepare() {
    return cudaFuncSetAttribute(k2_dcs_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingMax);
}

cudaError_t dcs_launch(const float* E, float* S3, int T, int X, int Y, int bnd, const Stencil& st,
                       float* mm_part, cudaStream_t s) {
    const long long NV = (long long)T * X * Y;
    const int nparts = red_blocks(NV);  // K3 reduces exactly this many min/max partials
    const size_t smem = ring_bytes(st.halo[0], st.halo[1], st.halo[2]);
    int per_sm = 0;
    if (smem <= kRingMax) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k2_dcs_tiled, kThreads, smem);
        if (e != cudaSuccess) return e;
    }
    const long long ntiles = (long long)((T + kTT - 1) / kTT) * ((X + kTX - 1) / kTX) * ((Y + kTY - 1) / kTY);
    const long long wave = (long long)std::max(per_sm, 1) * device_sms();
    // the ring kernel when its tiles fill at least one wave of resident blocks; with fewer it would leave
    // SMs idle, and the row kernel, whose warps cover every row, is faster
    if (smem <= kRingMax && per_sm > 0 && ntiles >= wave) {
        long long grid = std::min<long long>(wave, nparts);
        k2_dcs_tiled<<<(int)grid, kThreads, smem, s>>>(E, S3, T, X, Y, bnd, st, mm_part, nparts);
        note_launches(1);
        return cudaGetLastError();
    }
    k2_dcs<<<nparts, kThreads, 0, s>>>(E, S3, T, X, Y, bnd, st, mm_part);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace sal
