// Building blocks of the FP32 (SIMT) local-spectrum kernels, shared by the forward K1 and the
// adjoint K5: brick staging with border extension, the separable sliding DFT stages along t and
// x (Eq. 2), and the per-row projection weights of Eq. 1.
//
// Brick of one CTA: outputs (t0, x0, y_start .. y_start+BY-1); halo
//   V[t0-n/2 .. t0+n/2-1][x0-n/2 .. x0+n/2-1][y_start-n/2 .. y_start+BY+n/2-2]  ([N][N][YH] floats)
// Stage 1:  G1[k_t][x][y]   = sum_u h(u) exp(-2 pi i k_t u / n) V[..u..][x][y],   k_t in [0, n/2]
// Stage 2:  G2[k_t][k_x][y] = sum_u h(u) exp(-2 pi i k_x u / n) G1[k_t][u][y],      k_x in [0, n)
// Each one-axis DFT pairs bins k and n-k: with P = sum g c(k,u), Q = sum g s(k,u),
// F[k] = P - iQ and F[n-k] = P + iQ.
#pragma once

#include "sal_internal.cuh"

namespace sal {
namespace f32 {

// Square root and reciprocal square root on the MUFU pipe (one instruction each, relative
// error about 2^-22, far inside the 1e-5 budget of the FP32 form).
__device__ __forceinline__ float fast_sqrt(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float fast_rsqrt(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Eq. 1 weights of one bin (signed indices i, j, k; only their squares enter) with the multiplicity of
// its k_t and the 1/n^3 of the mean folded in (mult_over_n3): r_m = P_m / |k| for the feature of step 3
// (the mean of |F_m| = r_m |F|), or r_m^2 for the energy reading (the mean of |F_m|^2 = r_m^2 |F|^2);
// zero at DC.
template <bool EN>
__host__ __device__ __forceinline__ void bin_weights(int i, int j, int k, float mult_over_n3, float& w0, float& w1,
                                                     float& w2) {
    const float r2 = (float)(i * i + j * j + k * k);
    w0 = w1 = w2 = 0.f;
    if (r2 > 0.f) {
        const float p0 = (float)(j * j + k * k), p1 = (float)(i * i + k * k), p2 = (float)(i * i + j * j);
        if (EN) {
            const float inv = mult_over_n3 / r2;
            w0 = p0 * inv;
            w1 = p1 * inv;
            w2 = p2 * inv;
        } else {
            const float inv = mult_over_n3 / sqrtf(r2);
            w0 = sqrtf(p0) * inv;
            w1 = sqrtf(p1) * inv;
            w2 = sqrtf(p2) * inv;
        }
    }
}

// The per-bin quantity the feature averages, from |F|^2: |F| (step 3) or |F|^2 (energy).
template <bool EN>
__device__ __forceinline__ float bin_mag(float m2) {
    if (EN) return m2;
    return fast_sqrt(m2);
}

// Adjoint of the per-bin quantity: the factor sc with Gamma = sc F for the bin weight rho = sum_m gE_m w_m:
// d|F| = F / |F| (zero subgradient where |F|^2 <= thr2, the kink band), d|F|^2 = 2 F (smooth).
template <bool EN>
__device__ __forceinline__ float bin_adjoint_scale(float rho, float m2, float thr2) {
    if (EN) return 2.f * rho;
    return m2 > thr2 ? rho * fast_rsqrt(m2) : 0.f;
}

// Twiddles with the taper folded in: c[k][u] = h(u) cos(2 pi k u / n), s[k][u] = h(u) sin(...).
template <int N> struct Tw {
    float c[N / 2 + 1][N];
    float s[N / 2 + 1][N];
};

template <int N>
inline Tw<N> make_tw(const TwiddleTable& t) {
    Tw<N> w;
    for (int k = 0; k <= N / 2; ++k)
        for (int u = 0; u < N; ++u) {
            w.c[k][u] = t.c[k][u];
            w.s[k][u] = t.s[k][u];
        }
    return w;
}

template <int N_, int BY_, int NT_> struct Brick {
    static constexpr int N = N_, BY = BY_, NT = NT_;
    static constexpr int H = N / 2 + 1;
    static constexpr int YH = BY + N - 1;          // y extent of the halo brick
    static constexpr int ROWS = H * N;             // (k_t, k_x) rows of stage 3
    static constexpr int IN_FLOATS = N * N * YH;
    static constexpr int G_FLOAT2 = H * N * YH;
    static_assert(NT % 32 == 0 && NT >= YH, "staging maps one y position per thread");

    // Halo brick of V into s_in [N][N][YH], border extension applied per axis, minus vshift (a constant
    // over the brick moves only the DC bin of a rect-tapered cube).
    __device__ static void stage_brick(const float* __restrict__ V, float* s_in, int T, int X, int Y, int bnd,
                                       int t0, int x0, int y_start, float vshift = 0.f) {
        constexpr int RSTEP = NT / YH;
        constexpr int ITERS = (N * N + RSTEP - 1) / RSTEP;   // rows per thread: all loads issued, then stored
        const int tid = threadIdx.x;
        const int yy = tid % YH;
        const int r0 = tid / YH;
        const int gy = ext_index(y_start - N / 2 + yy, Y, bnd);
        if (r0 < RSTEP) {
            float v[ITERS];
#pragma unroll
            for (int i = 0; i < ITERS; ++i) {
                const int r = r0 + i * RSTEP;
                v[i] = 0.f;
                if (r < N * N) {
                    const int ut = r / N, ux = r % N;
                    const int gt = ext_index(t0 - N / 2 + ut, T, bnd);
                    const int gx = ext_index(x0 - N / 2 + ux, X, bnd);
                    if ((gt | gx | gy) >= 0) v[i] = __ldg(V + ((size_t)gt * X + gx) * Y + gy);
                }
            }
#pragma unroll
            for (int i = 0; i < ITERS; ++i) {
                const int r = r0 + i * RSTEP;
                if (r < N * N) s_in[r * YH + yy] = v[i] - vshift;
            }
        }
    }

    // Stage 1: DFT along t of the real cube, bins k_t in [0, n/2].  s_in -> s_g1 [H][N][YH].
    __device__ static void stage1(const float* s_in, float2* s_g1, const Tw<N>& tw) {
        for (int it = threadIdx.x; it < N * YH; it += NT) {
            const int ux = it / YH, yy = it % YH;
            float v[N];
#pragma unroll
            for (int u = 0; u < N; ++u) v[u] = s_in[(u * N + ux) * YH + yy];
#pragma unroll
            for (int k = 0; k < H; ++k) {
                float P = 0.f, Q = 0.f;
#pragma unroll
                for (int u = 0; u < N; ++u) {
                    P = fmaf(v[u], tw.c[k][u], P);
                    Q = fmaf(v[u], tw.s[k][u], Q);
                }
                s_g1[(k * N + ux) * YH + yy] = make_float2(P, -Q);
            }
        }
    }

    // Stage 2: DFT along x (complex input), all k_x.  s_g1 -> s_g2 [H][N][YH].
    __device__ static void stage2(const float2* s_g1, float2* s_g2, const Tw<N>& tw) {
        for (int it = threadIdx.x; it < H * YH; it += NT) {
            const int kt = it / YH, yy = it % YH;
            float2 g[N];
#pragma unroll
            for (int u = 0; u < N; ++u) g[u] = s_g1[(kt * N + u) * YH + yy];
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
                s_g2[(kt * N + k) * YH + yy] = make_float2(pr + qi, pi - qr);
                if (k != 0 && 2 * k != N) s_g2[(kt * N + (N - k)) * YH + yy] = make_float2(pr - qi, pi + qr);
            }
        }
    }

    // Projection weights of one stage-3 row (k_t, k_x) for |k_y| = k in [0, n/2], from the handle's table
    // [3][H][ROWS] (f32_weight_table): wt[m][k] = r_m(k_t, k_x, k) (or r_m^2, energy) * multiplicity(k_t)
    // / n^3, zero at DC (Eq. 1).
    __device__ static void row_weights(const float* __restrict__ wtab, int row, float (&wt)[3][H]) {
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int k = 0; k < H; ++k) wt[m][k] = __ldg(wtab + (m * H + k) * ROWS + row);
    }
};

// The table row_weights reads, [3][h][h n] (rows k_t n + k_x), for window n and the feature reading
// (EN: energy), computed on the host with bin_weights (correctly rounded square roots and division, as on
// the device).
template <bool EN>
inline void f32_weight_table(int n, float* out) {
    const int h = n / 2 + 1, rows = h * n;
    for (int row = 0; row < rows; ++row) {
        const int kt = row / n, kx = row % n;
        const int j = kx < n / 2 ? kx : kx - n;
        const float mult = (kt == 0 || 2 * kt == n) ? 1.f : 2.f;
        const float scale = mult / (float)(n * n * n);
        for (int k = 0; k < h; ++k) {
            float w[3];
            bin_weights<EN>(kt, j, k, scale, w[0], w[1], w[2]);
            for (int m = 0; m < 3; ++m) out[(m * h + k) * rows + row] = w[m];
        }
    }
}

}  // namespace f32
}  // namespace sal
