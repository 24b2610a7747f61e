// K1-F32 for the 32^3 window (Sec. 2 steps 1-3; Eq. 2, Eq. 1) on the SIMT pipes in FP32.
//
// The 32^3 cube makes the all-k_t intermediates of the smaller windows too large for shared
// memory, so the CTA streams over k_t tiles (0 .. 16): for each k_t it forms
//   G1[x][y]    = sum_u h(u) exp(-2 pi i k_t u / 32) V[t0-16+u][x][y]      (stage 1, t)
//   G2[k_x][y]  = sum_u h(u) exp(-2 pi i k_x u / 32) G1[u][y]              (stage 2, x)
//   F(y0)[k_y]  = sum_u h(u) exp(-2 pi i k_y u / 32) G2[k_x][y0 - 16 + u]  (stage 3, y)
// and accumulates E_m over tiles.  One CTA = one brick (t0, x0, y0 .. y0 + 7): 256 threads, lane = k_x.
// Direct form: warp w owns output y0 = w; the sum over k_x is a warp shuffle; the sum over k_t stays in
// registers across tiles.  Sliding form (rect taper, stride 1): warp w owns the k_y pairs (k, 32 - k) with
// k = w, w + 8 (and 16 for warp 0) for all 8 outputs: the first by the direct sum, the others by
//   F_{y0+1}[k] = e^{2 pi i k / 32} (F_{y0}[k] - G2[y0 - 16] + G2[y0 + 16]),
// each thread keeping the partial E of the 8 outputs across tiles; the brick is staged minus one of its
// voxels (only the DC bin moves), so a constant region stays exactly zero.  The halo brick
// (32 x 32 x 39 floats) lives in shared memory.
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

template <bool EN, bool SL>
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

    const float vshift = SL ? __ldg(V + ((size_t)t0 * X + x0) * Y + yb) : 0.f;
    // the halo brick a (u_t, u_x) row of YH samples per warp, RU rows in flight: each lane samples y = lane and
    // lane + 32, its two border-extended source columns fixed for the brick
    {
        constexpr int ROWS = N * N, RU = 4;
        const int gy0 = ext_index(yb - N / 2 + lane, Y, bnd);
        const int gy1 = lane + 32 < YH ? ext_index(yb - N / 2 + lane + 32, Y, bnd) : -1;
        for (int r0 = warp * RU; r0 < ROWS; r0 += (NT / 32) * RU) {
            float v0[RU], v1[RU];
#pragma unroll
            for (int a = 0; a < RU; ++a) {   // loads first
                const int r = r0 + a;
                const int gt = ext_index(t0 - N / 2 + r / N, T, bnd);
                const int gx = ext_index(x0 - N / 2 + r % N, X, bnd);
                v0[a] = v1[a] = 0.f;
                if ((gt | gx) >= 0) {
                    const float* row = V + ((size_t)gt * X + gx) * Y;
                    if (gy0 >= 0) v0[a] = __ldg(row + gy0);
                    if (gy1 >= 0) v1[a] = __ldg(row + gy1);
                }
            }
#pragma unroll
            for (int a = 0; a < RU; ++a) {   // s_in[u_t][u_x][y], row r = u_t N + u_x
                s_in[(r0 + a) * YH + lane] = v0[a] - vshift;
                if (lane + 32 < YH) s_in[(r0 + a) * YH + lane + 32] = v1[a] - vshift;
            }
        }
    }
    float e0 = 0.f, e1 = 0.f, e2 = 0.f;       // direct form: this lane's (k_x) partial E of output y0 = warp
    float es[SL ? BY : 1][3];                 // sliding form: this lane's partial E of the 8 outputs
#pragma unroll
    for (int o = 0; o < (SL ? BY : 1); ++o) es[o][0] = es[o][1] = es[o][2] = 0.f;
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
        if (SL) {
            // stage 3 (y) by the sliding recursion: warp = group of k_y pairs, lane = k_x, all 8 outputs
            const float2* row = s_g2 + kx * YH;
            const float* w = s_wt + kx * H * 3;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int k = q == 2 ? 16 : warp + 8 * q;   // pair index (k, 32 - k); 16 only for warp 0
                if (q == 2 && warp != 0) break;
                const bool self = k == 0 || k == 16;
                float pr = 0.f, pi = 0.f, qr = 0.f, qi = 0.f;
#pragma unroll 8
                for (int u = 0; u < N; ++u) {
                    const float2 g = row[u];
                    pr = fmaf(g.x, tw.c[k][u], pr);
                    pi = fmaf(g.y, tw.c[k][u], pi);
                    qr = fmaf(g.x, tw.s[k][u], qr);
                    qi = fmaf(g.y, tw.s[k][u], qi);
                }
                // F[k] = P - iQ, F[32-k] = P + iQ (self-paired bins: Q = 0 up to rounding, F = P)
                float ar = self ? pr : pr + qi, ai = self ? pi : pi - qr;
                float br = pr - qi, bi = pi + qr;
                const float c = tw.c[k][1], sn = tw.s[k][1];   // e^{2 pi i k/32}; the pair's twiddle has -sn
                const float w0 = w[k * 3 + 0], w1 = w[k * 3 + 1], w2 = w[k * 3 + 2];
#pragma unroll
                for (int o = 0; o < BY; ++o) {
                    if (o > 0) {
                        const float2 a = row[o - 1], b = row[o - 1 + N];   // sample leaving, sample entering
                        const float dr = b.x - a.x, di = b.y - a.y;
                        const float xr = ar + dr, xi = ai + di;
                        ar = fmaf(c, xr, -sn * xi);
                        ai = fmaf(sn, xr, c * xi);
                        if (!self) {
                            const float yr = br + dr, yi = bi + di;
                            br = fmaf(c, yr, sn * yi);
                            bi = fmaf(-sn, yr, c * yi);
                        }
                    }
                    float a = bin_mag<EN>(fmaf(ar, ar, ai * ai));
                    if (!self) a += bin_mag<EN>(fmaf(br, br, bi * bi));
                    es[o][0] = fmaf(w0, a, es[o][0]);
                    es[o][1] = fmaf(w1, a, es[o][1]);
                    es[o][2] = fmaf(w2, a, es[o][2]);
                }
            }
        }
        // stage 3 (y) + projection/feature epilogue: warp = y0, lane = k_x
        if (!SL && (stride == 1 || (yb + y0) % stride == 0)) {
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
    if (SL) {
        // sum over k_x (lanes), then over the k_y groups (warps, in order) through shared memory
        float* s_red = reinterpret_cast<float*>(s_g1);   // [8 warps][BY][3]
#pragma unroll
        for (int o = 0; o < BY; ++o)
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                float v = es[o][m];
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
                es[o][m] = v;
            }
        __syncthreads();   // last tile done with s_g1
        if (lane == 0)
#pragma unroll
            for (int o = 0; o < BY; ++o)
#pragma unroll
                for (int m = 0; m < 3; ++m) s_red[(warp * BY + o) * 3 + m] = es[o][m];
        __syncthreads();
        // lane 0 of warp y0 writes output y0
        e0 = e1 = e2 = 0.f;
        for (int w = 0; w < NT / 32; ++w) {
            e0 += s_red[(w * BY + y0) * 3 + 0];
            e1 += s_red[(w * BY + y0) * 3 + 1];
            e2 += s_red[(w * BY + y0) * 3 + 2];
        }
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            e0 += __shfl_xor_sync(0xffffffffu, e0, o);
            e1 += __shfl_xor_sync(0xffffffffu, e1, o);
            e2 += __shfl_xor_sync(0xffffffffu, e2, o);
        }
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
    cudaError_t e = cudaFuncSetAttribute(k1_spectra_f32_n32<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k1_spectra_f32_n32<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k1_spectra_f32_n32<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k1_spectra_f32_n32<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    return e;
}

cudaError_t spectra_f32_n32_launch(const TwiddleTable& t, const float* V, float* E, int T, int X, int Y, int bnd,
                                   int feat, int stride, int taper, cudaStream_t s) {
    if (stride < 1) return cudaErrorInvalidConfiguration;
    dim3 grid((Y + BY - 1) / BY, (X + stride - 1) / stride, (T + stride - 1) / stride);
    const Tw<N> tw = f32::make_tw<N>(t);
    const bool sl = taper == 0 && stride == 1;
    if (feat == 1 && sl) k1_spectra_f32_n32<true, true><<<grid, NT, SMEM, s>>>(V, E, T, X, Y, bnd, stride, tw);
    else if (feat == 1) k1_spectra_f32_n32<true, false><<<grid, NT, SMEM, s>>>(V, E, T, X, Y, bnd, stride, tw);
    else if (sl) k1_spectra_f32_n32<false, true><<<grid, NT, SMEM, s>>>(V, E, T, X, Y, bnd, stride, tw);
    else k1_spectra_f32_n32<false, false><<<grid, NT, SMEM, s>>>(V, E, T, X, Y, bnd, stride, tw);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace sal
