// K1-F32 for the 32^3 window (Sec. 2 steps 1-3; Eq. 2, Eq. 1) on the SIMT pipes in FP32.
//
// The 32^3 cube makes the all-k_t intermediates of the smaller windows too large for shared
// memory, so the CTA streams over k_t tiles (0 .. 16): for each k_t it forms
//   G1[x][y]    = sum_u h(u) exp(-2 pi i k_t u / 32) V[t0-16+u][x][y]      (stage 1, t)
//   G2[k_x][y]  = sum_u h(u) exp(-2 pi i k_x u / 32) G1[u][y]              (stage 2, x)
//   F(y0)[k_y]  = sum_u h(u) exp(-2 pi i k_y u / 32) G2[k_x][y0 - 16 + u]  (stage 3, y)
// and accumulates E_m over tiles.  One CTA = one brick (t0, x0, y0 .. y0 + 7): 256 threads, warp w
// owns output y0 = w, lane = k_x; the sum over k_x is a warp shuffle; the sum over k_t stays in
// registers across tiles.  The halo brick (32 x 32 x 39 floats) lives in shared memory.
#include "spectra_f32_common.cuh"

namespace sal {
namespace {

using f32::bin_mag;
using f32::Tw;

constexpr int N = 32, H = N / 2 + 1, BY = 8, YH = BY + N - 1, NT = 256;
constexpr size_t IN_B = (size_t)N * N * YH * 4;
constexpr size_t G_B = (size_t)N * YH * 8;
constexpr size_t WT_B = (size_t)N * H * 3 * 4;
constexpr size_t SMEM = IN_B + 2 * G_B + WT_B;

template <bool EN>
__global__ void __launch_bounds__(NT, 1)
k1_spectra_f32_n32(const float* __restrict__ V, float* __restrict__ E, int T, int X, int Y, int bnd, int stride,
                   const __grid_constant__ Tw<N> tw) {
    extern __shared__ __align__(16) unsigned char smem[];
    float* s_in = reinterpret_cast<float*>(smem);                         // [N][N][YH]
    float2* s_g1 = reinterpret_cast<float2*>(smem + IN_B);                // [N][YH]
    float2* s_g2 = reinterpret_cast<float2*>(smem + IN_B + G_B);          // [N][YH]
    float* s_wt = reinterpret_cast<float*>(smem + IN_B + 2 * G_B);        // [k_x][k][3] of this tile

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // stride s: cubes only at indices that are multiples of s
    const int yb = blockIdx.x * BY, x0 = blockIdx.y * stride, t0 = blockIdx.z * stride;

    for (int r = tid; r < N * N * YH; r += NT) {
        const int yy = r % YH, ux = (r / YH) % N, ut = r / (YH * N);
        const int gt = ext_index(t0 - N / 2 + ut, T, bnd);
        const int gx = ext_index(x0 - N / 2 + ux, X, bnd);
        const int gy = ext_index(yb - N / 2 + yy, Y, bnd);
        float v = 0.f;
        if ((gt | gx | gy) >= 0) v = __ldg(V + ((size_t)gt * X + gx) * Y + gy);
        s_in[r] = v;
    }
    float e0 = 0.f, e1 = 0.f, e2 = 0.f;       // this lane's (k_x) partial E of output y0 = warp
    const int kx = lane, y0 = warp;

    for (int kt = 0; kt < H; ++kt) {
        float cr[N], sr[N];
#pragma unroll
        for (int u = 0; u < N; ++u) {
            cr[u] = tw.c[kt][u];
            sr[u] = tw.s[kt][u];
        }
        __syncthreads();  // previous tile done with s_g1, s_g2, s_wt (and the halo is staged)
        // projection weights of (k_t, k_x, |k_y|) for this tile
        for (int i = tid; i < N * H; i += NT) {
            const int k = i % H, x = i / H;
            const int ii = kt, j = x < N / 2 ? x : x - N;
            const float mult = (kt == 0 || 2 * kt == N) ? 1.f : 2.f;
            float w0, w1, w2;
            f32::bin_weights<EN>(ii, j, k, mult / (float)(N * N * N), w0, w1, w2);
            s_wt[i * 3 + 0] = w0;
            s_wt[i * 3 + 1] = w1;
            s_wt[i * 3 + 2] = w2;
        }
        // stage 1 (t) for this k_t
        for (int it = tid; it < N * YH; it += NT) {
            float P = 0.f, Q = 0.f;
#pragma unroll
            for (int u = 0; u < N; ++u) {
                const float v = s_in[u * N * YH + it];
                P = fmaf(v, cr[u], P);
                Q = fmaf(v, sr[u], Q);
            }
            s_g1[it] = make_float2(P, -Q);
        }
        __syncthreads();
        // stage 2 (x): item (y, group of k); F[k] = P - iQ and F[n-k] = P + iQ
        for (int it = tid; it < YH * 4; it += NT) {
            const int y = it % YH, grp = it / YH;
            float2 g[N];
#pragma unroll
            for (int u = 0; u < N; ++u) g[u] = s_g1[u * YH + y];
#pragma unroll
            for (int k = 0; k < H; ++k) {
                if ((k % 4) != grp && !(k == N / 2 && grp == 0)) continue;
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
                s_g2[k * YH + y] = make_float2(pr + qi, pi - qr);
                if (k != 0 && 2 * k != N) s_g2[(N - k) * YH + y] = make_float2(pr - qi, pi + qr);
            }
        }
        __syncthreads();
        // stage 3 (y) + projection/feature epilogue: warp = y0, lane = k_x
        if (stride == 1 || (yb + y0) % stride == 0) {
            float pr[H], pi[H], qr[H], qi[H];
#pragma unroll
            for (int k = 0; k < H; ++k) pr[k] = pi[k] = qr[k] = qi[k] = 0.f;
            const float2* row = s_g2 + kx * YH + y0;
#pragma unroll
            for (int u = 0; u < N; ++u) {
                const float2 g = row[u];
#pragma unroll
                for (int k = 0; k < H; ++k) {
                    pr[k] = fmaf(g.x, tw.c[k][u], pr[k]);
                    pi[k] = fmaf(g.y, tw.c[k][u], pi[k]);
                    if (k != 0 && 2 * k != N) {
                        qr[k] = fmaf(g.x, tw.s[k][u], qr[k]);
                        qi[k] = fmaf(g.y, tw.s[k][u], qi[k]);
                    }
                }
            }
            const float* w = s_wt + kx * H * 3;
#pragma unroll
            for (int k = 0; k < H; ++k) {
                float a;
                if (k == 0 || 2 * k == N) {
                    a = bin_mag<EN>(fmaf(pr[k], pr[k], pi[k] * pi[k]));
                } else {
                    const float ar = pr[k] + qi[k], ai = pi[k] - qr[k];
                    const float br = pr[k] - qi[k], bi = pi[k] + qr[k];
                    a = bin_mag<EN>(fmaf(ar, ar, ai * ai)) + bin_mag<EN>(fmaf(br, br, bi * bi));
                }
                e0 = fmaf(w[k * 3 + 0], a, e0);
                e1 = fmaf(w[k * 3 + 1], a, e1);
                e2 = fmaf(w[k * 3 + 2], a, e2);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e0 += __shfl_xor_sync(0xffffffffu, e0, o);
        e1 += __shfl_xor_sync(0xffffffffu, e1, o);
        e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    }
    // E: [3][T][X][Y], or the lattice [3][Tc][Xc][Yc] (ceil(T / s) ...) for stride s > 1
    const int y = yb + y0;
    if (lane == 0 && y < Y && (stride == 1 || y % stride == 0)) {
        const int Xc = (X + stride - 1) / stride, Yc = (Y + stride - 1) / stride;
        const size_t NV = (size_t)((T + stride - 1) / stride) * Xc * Yc;
        const size_t p = ((size_t)(t0 / stride) * Xc + x0 / stride) * Yc + y / stride;
        E[p] = e0;
        E[NV + p] = e1;
        E[2 * NV + p] = e2;
    }
}

}  // namespace

cudaError_t spectra_f32_n32_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k1_spectra_f32_n32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k1_spectra_f32_n32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
}

cudaError_t spectra_f32_n32_launch(const TwiddleTable& t, const float* V, float* E, int T, int X, int Y, int bnd,
                                   int feat, int stride, cudaStream_t s) {
    if (stride < 1) return cudaErrorInvalidConfiguration;
    dim3 grid((Y + BY - 1) / BY, (X + stride - 1) / stride, (T + stride - 1) / stride);
    if (feat == 1)
        k1_spectra_f32_n32<true><<<grid, NT, SMEM, s>>>(V, E, T, X, Y, bnd, stride, f32::make_tw<N>(t));
    else
        k1_spectra_f32_n32<false><<<grid, NT, SMEM, s>>>(V, E, T, X, Y, bnd, stride, f32::make_tw<N>(t));
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace sal
