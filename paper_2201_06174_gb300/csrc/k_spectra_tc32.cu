// K1-TC for the 32^3 window (Sec. 2 steps 1-3; Eq. 2, Eq. 1): stage 3 (the DFT along y of every
// (k_t, k_x) row) on the tensor cores, as for the smaller windows, with the shapes of n = 32:
//   rows m = (x0 - xb) * 32 + k_x, 4 positions x 32 k_x = 128;
//   B = the 32 paired twiddle columns [cos k = 0..16 | sin k = 1..15] over 32 taps: two K steps;
//   one output y0 = 64 TMEM columns (real part of A x B | imaginary part of A x B);
//   the halo brick is staged in FP16 after a per-brick 1/max|V| scale (the FP32 brick of a 32^3
//   window exceeds shared memory); stages 1-2 accumulate in FP32 on the SIMT pipes.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "spectra_f32_common.cuh"
#include "tc_sm100.cuh"

namespace sal {
namespace {

using f32::bin_mag;
using f32::Tw;

constexpr int N = 32, H = N / 2 + 1, P = 128 / N, BY = 16;
constexpr int XH = P + N - 1, YH = BY + N - 1;
constexpr int KROWS = BY + N - 1;                        // window start + 32 taps
constexpr uint32_t SBO_A = KROWS * 16;
constexpr int kThreads = 256;
constexpr uint32_t kTmemCols = 512;                      // 8 outputs x 64 columns
constexpr uint32_t kWaitLimit = 1u << 22;

constexpr size_t IN_B = (size_t)N * XH * YH * 2;         // FP16 halo
constexpr size_t G1_B = (size_t)XH * YH * 8;
constexpr size_t A_B = (size_t)16 * SBO_A;
constexpr size_t B_B = 2048;
constexpr size_t WT_B = (size_t)N * H * 3 * 4;
constexpr size_t OFF_G1 = (IN_B + 127) / 128 * 128;
constexpr size_t OFF_A = (OFF_G1 + G1_B + 127) / 128 * 128;
constexpr size_t OFF_B = OFF_A + 2 * A_B;
constexpr size_t OFF_WT = OFF_B + B_B;
constexpr size_t OFF_MISC = OFF_WT + WT_B;
constexpr size_t SMEM = OFF_MISC + 64 + (kThreads / 32) * 4;
static_assert(SMEM <= 227 * 1024, "shared memory");

template <int FMT> struct Pack;
template <> struct Pack<1> {
    __device__ static uint16_t one(float a) {
        __nv_bfloat16 v = __float2bfloat16_rn(a);
        return *reinterpret_cast<uint16_t*>(&v);
    }
};
template <> struct Pack<0> {
    __device__ static uint16_t one(float a) {
        __half v = __float2half_rn(a);
        return *reinterpret_cast<uint16_t*>(&v);
    }
};

template <int FMT, bool EN>
__global__ void __launch_bounds__(kThreads, 1)
k1_spectra_tc32(const float* __restrict__ V, float* __restrict__ E, int T, int X, int Y, int bnd, int stride,
                const __grid_constant__ Tw<N> tw, int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    __half* s_in = reinterpret_cast<__half*>(smem);                     // [N][XH][YH], scaled
    float2* s_g1 = reinterpret_cast<float2*>(smem + OFF_G1);            // [XH][YH]
    unsigned char* s_are = smem + OFF_A;
    unsigned char* s_aim = smem + OFF_A + A_B;
    unsigned char* s_b = smem + OFF_B;                                  // [32 n][32 k], K-major
    float* s_wt = reinterpret_cast<float*>(smem + OFF_WT);              // [k_x][k][3] of this tile
    uint64_t* s_mbar = reinterpret_cast<uint64_t*>(smem + OFF_MISC);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + OFF_MISC + 8);
    int* s_fail = reinterpret_cast<int*>(smem + OFF_MISC + 16);
    float* s_red = reinterpret_cast<float*>(smem + OFF_MISC + 64);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int yb = blockIdx.x * BY, xb = blockIdx.y * P, t0 = blockIdx.z * stride;   // stride s: planes t0 = k s

    if (warp == 0) tc::tmem_alloc(tc::smem_u32(s_tmem), kTmemCols);
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(s_mbar), 1);
        *s_fail = 0;
    }
    for (int i = tid; i < 32 * 32; i += kThreads) {
        const int n = i / 32, k = i % 32;
        float v = 0.f;
        if (n < H) v = tw.c[n][k];
        else v = tw.s[n - H + 1][k];
        *reinterpret_cast<uint16_t*>(s_b + (n / 8) * 512 + (k / 8) * 128 + (n % 8) * 16 + (k % 8) * 2) =
            Pack<FMT>::one(v);
    }
    for (int i = tid; i < (int)(2 * A_B / 16); i += kThreads)
        reinterpret_cast<uint4*>(s_are)[i] = make_uint4(0u, 0u, 0u, 0u);
    // the halo's maximum first (two passes over global memory; the second converts to FP16)
    float vmax = 0.f;
    for (int r = tid; r < N * XH * YH; r += kThreads) {
        const int yy = r % YH, xx = (r / YH) % XH, ut = r / (YH * XH);
        const int gt = ext_index(t0 - N / 2 + ut, T, bnd);
        const int gx = ext_index(xb - N / 2 + xx, X, bnd);
        const int gy = ext_index(yb - N / 2 + yy, Y, bnd);
        if ((gt | gx | gy) >= 0) vmax = fmaxf(vmax, fabsf(__ldg(V + ((size_t)gt * X + gx) * Y + gy)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    if (lane == 0) s_red[warp] = vmax;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *s_tmem;
    float bmax = 0.f;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) bmax = fmaxf(bmax, s_red[w]);
    const float scale = bmax > 0.f ? bmax : 1.f;
    const float inv_scale = 1.f / scale;
    for (int r = tid; r < N * XH * YH; r += kThreads) {
        const int yy = r % YH, xx = (r / YH) % XH, ut = r / (YH * XH);
        const int gt = ext_index(t0 - N / 2 + ut, T, bnd);
        const int gx = ext_index(xb - N / 2 + xx, X, bnd);
        const int gy = ext_index(yb - N / 2 + yy, Y, bnd);
        float v = 0.f;
        if ((gt | gx | gy) >= 0) v = __ldg(V + ((size_t)gt * X + gx) * Y + gy);
        s_in[r] = __float2half_rn(v * inv_scale);
    }

    const int q = warp & 3, half = warp >> 2;
    const int m = 32 * q + lane;
    const int x0l = m / N, kx = m % N;
    float acc[8][3];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i][0] = acc[i][1] = acc[i][2] = 0.f;
    const uint32_t idesc = tc::idesc_f16(FMT, 128, 32, 1, 0);
    const uint32_t bsm = tc::smem_u32(s_b), are = tc::smem_u32(s_are), aim = tc::smem_u32(s_aim);
    uint32_t phase = 0;

    for (int kt = 0; kt < H; ++kt) {
        float cr[N], sr[N];
#pragma unroll
        for (int u = 0; u < N; ++u) {
            cr[u] = tw.c[kt][u];
            sr[u] = tw.s[kt][u];
        }
        __syncthreads();   // the halo is staged; the previous tile is done with s_g1 and s_wt
        for (int i = tid; i < N * H; i += kThreads) {
            const int k = i % H, x = i / H;
            const int ii = kt, j = x < N / 2 ? x : x - N;
            const float mult = (kt == 0 || 2 * kt == N) ? 1.f : 2.f;
            float w0, w1, w2;
            f32::bin_weights<EN>(ii, j, k, mult / (float)(N * N * N), w0, w1, w2);
            s_wt[i * 3 + 0] = w0;
            s_wt[i * 3 + 1] = w1;
            s_wt[i * 3 + 2] = w2;
        }
        for (int it = tid; it < XH * YH; it += kThreads) {
            float Pv = 0.f, Qv = 0.f;
#pragma unroll
            for (int u = 0; u < N; ++u) {
                const float v = __half2float(s_in[u * XH * YH + it]);
                Pv = fmaf(v, cr[u], Pv);
                Qv = fmaf(v, sr[u], Qv);
            }
            s_g1[it] = make_float2(Pv, -Qv);
        }
        __syncthreads();
        // stage 2 -> A operand: row m = xl * 32 + k_x at K row y (2-byte stores)
        for (int it = tid; it < P * YH; it += kThreads) {
            const int xl = it / YH, y = it % YH;
            float2 g[N];
#pragma unroll
            for (int u = 0; u < N; ++u) g[u] = s_g1[(xl + u) * YH + y];
            unsigned char* rowre = s_are + (size_t)(xl * 4) * SBO_A + (size_t)y * 16;
            unsigned char* rowim = s_aim + (size_t)(xl * 4) * SBO_A + (size_t)y * 16;
#pragma unroll
            for (int k = 0; k < H; ++k) {
                float pr = 0.f, pi = 0.f, qr = 0.f, qi = 0.f;
#pragma unroll
                for (int u = 0; u < N; ++u) {
                    pr = fmaf(g[u].x, tw.c[k][u], pr);
                    pi = fmaf(g[u].y, tw.c[k][u], pi);
                    if (k != 0 && 2 * k != N) {
                        qr = fmaf(g[u].x, tw.s[k][u], qr);
                        qi = fmaf(g[u].y, tw.s[k][u], qi);
                    }
                }
                const size_t oa = (size_t)(k / 8) * SBO_A + (k % 8) * 2;
                *reinterpret_cast<uint16_t*>(rowre + oa) = Pack<FMT>::one(pr + qi);
                *reinterpret_cast<uint16_t*>(rowim + oa) = Pack<FMT>::one(pi - qr);
                if (k != 0 && 2 * k != N) {
                    const int kb = N - k;
                    const size_t ob = (size_t)(kb / 8) * SBO_A + (kb % 8) * 2;
                    *reinterpret_cast<uint16_t*>(rowre + ob) = Pack<FMT>::one(pr - qi);
                    *reinterpret_cast<uint16_t*>(rowim + ob) = Pack<FMT>::one(pi + qr);
                }
            }
        }
        tc::fence_async_smem();
        __syncthreads();
        float wt[3][H];
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const float* w = s_wt + (kx * H + k) * 3;
            wt[0][k] = w[0];
            wt[1][k] = w[1];
            wt[2][k] = w[2];
        }
        for (int pass = 0; pass < 2; ++pass) {
            if (tid == 0 && !*s_fail) {
                tc::fence_after_sync();
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint32_t y0 = pass * 8 + j;
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint64_t bd = tc::desc_noswizzle(bsm + ks * 256, 128, 512);
                        tc::mma_f16(tmem + j * 64, tc::desc_noswizzle(are + (y0 + 16 * ks) * 16, 128, SBO_A), bd,
                                    idesc, ks);
                        tc::mma_f16(tmem + j * 64 + 32, tc::desc_noswizzle(aim + (y0 + 16 * ks) * 16, 128, SBO_A), bd,
                                    idesc, ks);
                    }
                }
                tc::mma_commit(tc::smem_u32(s_mbar));
            }
            const int failed_before = *s_fail;
            const bool ok = failed_before ? false : tc::mbar_wait(tc::smem_u32(s_mbar), phase, kWaitLimit);
            const int bad = __syncthreads_or(!ok);
            if (bad && tid == 0 && !failed_before) {
                atomicOr(err, 1);
                *s_fail = 1;
            }
            phase ^= 1u;
            tc::fence_after_sync();
            if (!bad) {
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int j = half + 2 * jj;
                    float vr[32], vi[32];
                    tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(j * 64), vr);
                    tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(j * 64 + 32), vi);
                    float e0 = 0.f, e1 = 0.f, e2 = 0.f;
#pragma unroll
                    for (int k = 0; k < H; ++k) {
                        const float pr = vr[k], pi = vi[k];
                        float a;
                        if (k == 0 || 2 * k == N) {
                            a = bin_mag<EN>(fmaf(pr, pr, pi * pi));
                        } else {
                            const float qr = vr[H + k - 1], qi = vi[H + k - 1];
                            const float ar = pr + qi, ai = pi - qr, br = pr - qi, bi = pi + qr;
                            a = bin_mag<EN>(fmaf(ar, ar, ai * ai)) + bin_mag<EN>(fmaf(br, br, bi * bi));
                        }
                        e0 = fmaf(wt[0][k], a, e0);
                        e1 = fmaf(wt[1][k], a, e1);
                        e2 = fmaf(wt[2][k], a, e2);
                    }
                    acc[pass * 4 + jj][0] += e0;
                    acc[pass * 4 + jj][1] += e1;
                    acc[pass * 4 + jj][2] += e2;
                }
            }
            tc::fence_before_sync();
            __syncthreads();
        }
    }

    // E: [3][T][X][Y], or the lattice [3][Tc][Xc][Yc] (ceil(T / s) ...) for stride s > 1
    const int Xc = (X + stride - 1) / stride, Yc = (Y + stride - 1) / stride;
    const size_t NV = (size_t)((T + stride - 1) / stride) * Xc * Yc;
    const int x = xb + x0l;
    const float out_scale = EN ? scale * scale : scale;   // the features of the unscaled brick
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int y0 = (i / 4) * 8 + half + 2 * (i % 4);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float s = acc[i][c];
#pragma unroll
            for (int o = 1; o < N; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            const int y = yb + y0;
            if (kx == 0 && x < X && y < Y && !*s_fail) {
                if (stride == 1)
                    E[c * NV + ((size_t)t0 * X + x) * Y + y] = s * out_scale;
                else if (x % stride == 0 && y % stride == 0)   // the lattice (a rare path)
                    E[c * NV + ((size_t)(t0 / stride) * Xc + x / stride) * Yc + y / stride] = s * out_scale;
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

template <int FMT, bool EN>
cudaError_t prepare32() {
    return cudaFuncSetAttribute(k1_spectra_tc32<FMT, EN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
}

}  // namespace

cudaError_t spectra_tc32_prepare(int fmt) {
    cudaError_t e = fmt == 1 ? prepare32<1, false>() : prepare32<0, false>();
    if (e != cudaSuccess) return e;
    return fmt == 1 ? prepare32<1, true>() : prepare32<0, true>();
}

cudaError_t spectra_tc32_launch(int fmt, const TwiddleTable& t, const float* V, float* E, int T, int X, int Y,
                                int bnd, int feat, int stride, int* err, cudaStream_t s) {
    if (stride < 1) return cudaErrorInvalidConfiguration;
    dim3 grid((Y + BY - 1) / BY, (X + P - 1) / P, (T + stride - 1) / stride);
    const Tw<N> tw = f32::make_tw<N>(t);
    const int st = stride;
    if (fmt == 1 && feat == 1) k1_spectra_tc32<1, true><<<grid, kThreads, SMEM, s>>>(V, E, T, X, Y, bnd, st, tw, err);
    else if (fmt == 1) k1_spectra_tc32<1, false><<<grid, kThreads, SMEM, s>>>(V, E, T, X, Y, bnd, st, tw, err);
    else if (feat == 1) k1_spectra_tc32<0, true><<<grid, kThreads, SMEM, s>>>(V, E, T, X, Y, bnd, st, tw, err);
    else k1_spectra_tc32<0, false><<<grid, kThreads, SMEM, s>>>(V, E, T, X, Y, bnd, st, tw, err);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace sal
