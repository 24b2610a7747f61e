// The spatial-domain reading of the feature step (Sec. 2 step 3; Eq. 1, Eq. 2), FP32, n in {2, 4, 8, 16}:
//   E_m[p] = (1/n^3) sum_u |f_m[u]|,   f_m = IDFT(r_m DFT(w)),
// w the (tapered) cube of voxel p, r_m = P_m / |k| the projection ratio of Eq. 1 (zero at DC), and its
// adjoint  dE_m/dw = (1/n^3) A_m sign(f_m),  A_m = IDFT diag(r_m) DFT (real and symmetric: r_m is even in k).
//
// One window per group of n^2 threads (256 / n^2 windows per CTA at a time); the window's complex 3-D arrays
// live in shared memory (float2 [t][x][y], rows padded to n + 1 elements so that the lines of all three axes
// fall on distinct banks), and each thread transforms one line at a time in registers (radix-2 FFT,
// decimation in time).  The Eq. 1 ratios come from a table built on the host.
// The separable 3-D transform is three passes of line FFTs; the pass along t holds a complete spectrum line,
// so the Eq. 1 weights and the first inverse pass run in the same registers.  Since every f_m is real, maps
// 0 and 1 share one complex inverse transform: IDFT((r_0 + i r_1) F) = f_0 + i f_1.
//
// Forward: 9 line FFTs per thread and window.  Backward: the same forward recompute, the signs s_m, then
//   sum_m gE_m A_m s_m = Re IDFT( (gE_0 r_0 - i gE_1 r_1) DFT(s_0 + i s_1) + gE_2 r_2 DFT(s_2) ) / n^3
// (A_m real: Re IDFT(r_m DFT(s_0 + i s_1)) = A_m s_0 and Re IDFT(-i r_m DFT(s_0 + i s_1)) = A_m s_1), 18 line
// FFTs; each window's gradient, times the taper, is added (in a fixed window order) into its brick's block
// in shared memory, and the bricks' blocks go through the same overlap-add as the spectral adjoint.
#include <cmath>

#include "sal_internal.cuh"

namespace sal {
namespace {

constexpr int kThreads = 256;
constexpr int kBX = 8, kBY = 8;   // windows per brick along x and y (a brick is one voxel deep in t)

// e^{-2 pi i k / 16} = c16(k) - i s16(k), k < 8: the 16th roots of unity (cos(pi/8) = sqrt(2 + sqrt(2)) / 2,
// sin(pi/8) = sqrt(2 - sqrt(2)) / 2, cos(pi/4) = sqrt(2) / 2), enough for every line length n <= 16
__host__ __device__ constexpr float c16(int k) {
    return k == 0 ? 1.f
         : k == 1 ? 0.923879532511286756f
         : k == 2 ? 0.707106781186547524f
         : k == 3 ? 0.382683432365089772f
         : k == 4 ? 0.f
         : k == 5 ? -0.382683432365089772f
         : k == 6 ? -0.707106781186547524f
                  : -0.923879532511286756f;
}
__host__ __device__ constexpr float s16(int k) {
    return k == 0 ? 0.f
         : k == 1 ? 0.382683432365089772f
         : k == 2 ? 0.707106781186547524f
         : k == 3 ? 0.923879532511286756f
         : k == 4 ? 1.f
         : k == 5 ? 0.923879532511286756f
         : k == 6 ? 0.707106781186547524f
                  : 0.382683432365089772f;
}

template <int N>
__host__ __device__ constexpr int log2c() {
    return N <= 1 ? 0 : 1 + log2c<N / 2>();
}

template <int N>
__host__ __device__ constexpr int bitrev(int i) {
    int r = 0;
    for (int b = 0; b < log2c<N>(); ++b) r |= ((i >> b) & 1) << (log2c<N>() - 1 - b);
    return r;
}

// In-place DFT of one line of N <= 16 points held in registers: X[k] = sum_j x[j] e^{-/+ 2 pi i j k / N}
// (+ for INV; no 1/N).  Radix-2 decimation in time: bit-reversed reorder, then log2 N butterfly stages; every
// index is a template constant, so the line stays in registers.
template <int N, int I>
__device__ __forceinline__ void bitrev_swap(float (&re)[N], float (&im)[N]) {
    if constexpr (I < N) {
        constexpr int J = bitrev<N>(I);
        if constexpr (J > I) {
            const float a = re[I], b = im[I];
            re[I] = re[J];
            im[I] = im[J];
            re[J] = a;
            im[J] = b;
        }
        bitrev_swap<N, I + 1>(re, im);
    }
}

// One butterfly (a, a + LEN/2) of the stage of length LEN with the twiddle e^{-/+ 2 pi i J / LEN}.
template <int N, bool INV, int LEN, int A, int J>
__device__ __forceinline__ void butterfly(float (&re)[N], float (&im)[N]) {
    constexpr int B = A + LEN / 2, K = J * (16 / LEN);
    float vr, vi;
    if constexpr (K == 0) {
        vr = re[B];
        vi = im[B];
    } else if constexpr (K == 4) {   // -i (forward) or +i (inverse)
        vr = INV ? -im[B] : im[B];
        vi = INV ? re[B] : -re[B];
    } else {
        constexpr float c = c16(K), s = INV ? s16(K) : -s16(K);
        vr = fmaf(re[B], c, -im[B] * s);
        vi = fmaf(re[B], s, im[B] * c);
    }
    re[B] = re[A] - vr;
    im[B] = im[A] - vi;
    re[A] += vr;
    im[A] += vi;
}

template <int N, bool INV, int LEN, int I>   // I: butterfly index within the stage, I < N / 2
__device__ __forceinline__ void stage(float (&re)[N], float (&im)[N]) {
    if constexpr (I < N / 2) {
        constexpr int H = LEN / 2, A = (I / H) * LEN + I % H;
        butterfly<N, INV, LEN, A, I % H>(re, im);
        stage<N, INV, LEN, I + 1>(re, im);
    }
}

template <int N, bool INV, int LEN>
__device__ __forceinline__ void stages(float (&re)[N], float (&im)[N]) {
    if constexpr (LEN <= N) {
        stage<N, INV, LEN, 0>(re, im);
        stages<N, INV, 2 * LEN>(re, im);
    }
}

template <int N, bool INV>
__device__ __forceinline__ void fft_line(float (&re)[N], float (&im)[N]) {
    bitrev_swap<N, 0>(re, im);
    stages<N, INV, 2>(re, im);
}

// Shared-memory layout of one window's complex array: float2 (re, im) elements [t][x][y], rows of N + 1
// elements.  A half-warp's 8-byte accesses along any of the three axes then fall on distinct bank pairs
// (N = 16: lines along y step 17 elements, along x and t the 16 lanes of a half-warp run along y).
template <int N>
struct Lay {
    static constexpr int ROW = N + 1, PLANE = N * ROW, WIN = N * PLANE;
    static constexpr int LINES = N * N, WPC = kThreads / LINES;   // lines per window, windows per CTA
};

// First element and stride of line l along axis AX (0 = t, 1 = x, 2 = y): AX 2: l = (t, x); AX 1: l = (t, y);
// AX 0: l = (x, y).
template <int N, int AX>
__device__ __forceinline__ int line_base(int l) {
    return AX == 2 ? l * Lay<N>::ROW
         : AX == 1 ? (l / N) * Lay<N>::PLANE + (l % N)
                   : (l / N) * Lay<N>::ROW + (l % N);
}
template <int N, int AX>
__device__ __forceinline__ constexpr int line_stride() {
    return AX == 2 ? 1 : AX == 1 ? Lay<N>::ROW : Lay<N>::PLANE;
}

template <int N, int AX>
__device__ __forceinline__ void load_line(const float2* __restrict__ a, int l, float (&re)[N], float (&im)[N]) {
    const int b = line_base<N, AX>(l);
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const float2 v = a[b + j * line_stride<N, AX>()];
        re[j] = v.x;
        im[j] = v.y;
    }
}
template <int N, int AX>
__device__ __forceinline__ void store_line(float2* __restrict__ a, int l, const float (&re)[N], const float (&im)[N]) {
    const int b = line_base<N, AX>(l);
#pragma unroll
    for (int j = 0; j < N; ++j) a[b + j * line_stride<N, AX>()] = make_float2(re[j], im[j]);
}

// One pass of line FFTs along AX over an array, in place.
template <int N, int AX, bool INV>
__device__ __forceinline__ void fft_pass(float2* a, int l) {
    float re[N], im[N];
    load_line<N, AX>(a, l, re, im);
    fft_line<N, INV>(re, im);
    store_line<N, AX>(a, l, re, im);
}

// Eq. 1 ratio table: entry (|s_t| (N/2 + 1) + |s_x|) (N/2 + 1) + |s_y| holds (r_0, r_1, r_2, 0) of the bins with
// signed indices +-s (r_m depends on squared indices only); built on the host (spatial_weight_table_fill).
template <int N>
__device__ __forceinline__ int abs_bin(int k) {
    return k <= N / 2 ? k : N - k;
}

// The periodic Hann taper h(u) = 0.5 - 0.5 cos(2 pi u / n) = sin^2(pi u / n), u < n, into shared memory; the
// barrier orders it before every use.
template <int N>
__device__ __forceinline__ void stage_taper(float* s_h) {
    if (threadIdx.x < N) {
        const float s = sinpif((float)threadIdx.x / (float)N);
        s_h[threadIdx.x] = s * s;
    }
    __syncthreads();
}

// The spectrum line l = (k_x, k_y) along t, taken to (r_0 + i r_1) F and r_2 F and transformed back along t.
template <int N>
__device__ __forceinline__ void weigh_and_invert_t(int l, const float4* __restrict__ rtab, float (&re)[N],
                                                   float (&im)[N], float (&ar)[N], float (&ai)[N]) {
    constexpr int H = N / 2 + 1;
    const float4* row = rtab + abs_bin<N>(l / N) * H + abs_bin<N>(l % N);
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const float4 r = __ldg(row + abs_bin<N>(k) * H * H);
        const float fr = re[k], fi = im[k];
        ar[k] = r.x * fr - r.y * fi;   // (r_0 + i r_1)(fr + i fi)
        ai[k] = r.x * fi + r.y * fr;
        re[k] = r.z * fr;
        im[k] = r.z * fi;
    }
    fft_line<N, true>(ar, ai);
    fft_line<N, true>(re, im);
}

// Sum of three values over the N^2 threads of a window group (fixed order); the group's thread 0 gets it.
// N >= 8: a barrier inside (every thread of the CTA calls it).
template <int N>
__device__ __forceinline__ void group_sum3(float& a0, float& a1, float& a2, float (*s_red)[3], int l) {
    constexpr int W = Lay<N>::LINES < 32 ? Lay<N>::LINES : 32;
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if constexpr (Lay<N>::LINES > 32) {
        constexpr int WPW = Lay<N>::LINES / 32;   // warps per window
        const int warp = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) {
            s_red[warp][0] = a0;
            s_red[warp][1] = a1;
            s_red[warp][2] = a2;
        }
        __syncthreads();
        if (l == 0) {
            a0 = a1 = a2 = 0.f;
            for (int w = warp; w < warp + WPW; ++w) {
                a0 += s_red[w][0];
                a1 += s_red[w][1];
                a2 += s_red[w][2];
            }
        }
    }
}

template <int N>
constexpr int arrays_bytes() {
    return 2 * Lay<N>::WPC * Lay<N>::WIN * (int)sizeof(float2);   // F and G
}

// Forward: one CTA per run of YB consecutive windows along y of one (t, x) row.  Their halo
// [n][n][YB + n - 1] of V (border extension applied) is loaded once with coalesced loads, and each window's
// first pass (along y) reads its rows from it; groups of n^2 threads take WPC windows at a time.
template <int N>
struct Seg {
    static constexpr int YB = Lay<N>::WPC > 16 ? Lay<N>::WPC : 16;   // windows per CTA
    static constexpr int HROW = YB + N - 1, HALO = N * N * HROW;
};

template <int N>
constexpr int fwd_smem_bytes() {
    return arrays_bytes<N>() + Seg<N>::HALO * (int)sizeof(float);
}

template <int N, bool HANN>
__global__ void __launch_bounds__(kThreads, 2)
k1_spatial_f32(const float* __restrict__ V, const float4* __restrict__ rtab, float* __restrict__ E, int T, int X,
               int Y, int bnd) {
    using L = Lay<N>;
    using S = Seg<N>;
    extern __shared__ __align__(16) float smem[];
    __shared__ float s_red[kThreads / 32][3];
    __shared__ float s_h[16];
    float2* F = reinterpret_cast<float2*>(smem);
    float2* G = F + L::WPC * L::WIN;
    float* halo = reinterpret_cast<float*>(G + L::WPC * L::WIN);
    const int g = threadIdx.x / L::LINES, l = threadIdx.x % L::LINES;
    float2* Fg = F + g * L::WIN;
    float2* Gg = G + g * L::WIN;
    const int t = blockIdx.z, x = blockIdx.y, y0 = blockIdx.x * S::YB;
    if (HANN && threadIdx.x < N) {
        const float s = sinpif((float)threadIdx.x / (float)N);   // h(u) = 0.5 - 0.5 cos(2 pi u / n)
        s_h[threadIdx.x] = s * s;
    }
    for (int i = threadIdx.x; i < S::HALO; i += kThreads) {
        const int yy = i % S::HROW, r = i / S::HROW;   // r = u_t n + u_x
        const int gt = ext_index(t - N / 2 + r / N, T, bnd), gx = ext_index(x - N / 2 + r % N, X, bnd);
        const int gy = ext_index(y0 - N / 2 + yy, Y, bnd);
        halo[i] = (gt | gx | gy) >= 0 ? __ldg(V + ((size_t)gt * X + gx) * Y + gy) : 0.f;
    }
    __syncthreads();
    const size_t NV = (size_t)T * X * Y;
    const float* hl = halo + l * S::HROW;   // this thread's row (u_t, u_x) = (l / n, l % n)
    const float hrow = HANN ? s_h[l / N] * s_h[l % N] : 1.f;
#pragma unroll 1
    for (int it = 0; it < S::YB / L::WPC; ++it) {
        const int wy = it * L::WPC + g, y = y0 + wy;   // windows past the row's end compute and store nothing
        float re[N], im[N], ar[N], ai[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            re[j] = HANN ? hl[wy + j] * (hrow * s_h[j]) : hl[wy + j];
            im[j] = 0.f;
        }
        fft_line<N, false>(re, im);
        store_line<N, 2>(Fg, l, re, im);
        __syncthreads();
        fft_pass<N, 1, false>(Fg, l);
        __syncthreads();
        load_line<N, 0>(Fg, l, re, im);
        fft_line<N, false>(re, im);   // F complete on this (k_x, k_y) line
        weigh_and_invert_t<N>(l, rtab, re, im, ar, ai);
        store_line<N, 0>(Gg, l, ar, ai);   // G: (r_0 + i r_1) F, F: r_2 F, both inverted along t
        store_line<N, 0>(Fg, l, re, im);
        __syncthreads();
        fft_pass<N, 1, true>(Gg, l);
        fft_pass<N, 1, true>(Fg, l);
        __syncthreads();
        load_line<N, 2>(Gg, l, ar, ai);
        load_line<N, 2>(Fg, l, re, im);
        fft_line<N, true>(ar, ai);   // n^3 (f_0 + i f_1) on this (u_t, u_x) line
        fft_line<N, true>(re, im);   // n^3 f_2
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            a0 += fabsf(ar[j]);
            a1 += fabsf(ai[j]);
            a2 += fabsf(re[j]);
        }
        group_sum3<N>(a0, a1, a2, s_red, l);
        if (l == 0 && y < Y) {
            constexpr float sc = 1.f / ((float)(N * N * N) * (float)(N * N * N));   // 1/n^3 IDFT, 1/n^3 mean
            const size_t q = ((size_t)t * X + x) * Y + y;
            E[q] = a0 * sc;
            E[NV + q] = a1 * sc;
            E[2 * NV + q] = a2 * sc;
        }
        __syncthreads();   // the next windows' first pass overwrites F
    }
}

// Loads the window of voxel (t, x, y) along line l = (u_t, u_x) (border extension, taper applied) and
// transforms it along y: the first forward pass, straight from V.
template <int N, bool HANN>
__device__ __forceinline__ void load_window_line(const float* __restrict__ V, int T, int X, int Y, int bnd, int t,
                                                 int x, int y, int l, const float* __restrict__ h, float (&re)[N],
                                                 float (&im)[N]) {
    const int ut = l / N, ux = l % N;
    const int gt = ext_index(t - N / 2 + ut, T, bnd), gx = ext_index(x - N / 2 + ux, X, bnd);
    const bool row_ok = (gt | gx) >= 0;
    const float* row = V + ((size_t)(row_ok ? gt : 0) * X + (row_ok ? gx : 0)) * Y;
    const float hrow = HANN ? h[ut] * h[ux] : 1.f;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const int gy = ext_index(y - N / 2 + j, Y, bnd);
        const float v = row_ok && gy >= 0 ? __ldg(row + gy) : 0.f;
        re[j] = HANN ? v * (hrow * h[j]) : v;
        im[j] = 0.f;
    }
    fft_line<N, false>(re, im);
}

// Backward: one CTA per brick (kBX x kBY windows of one t plane); the brick's block [u_t][x'][y'] (x' < XH,
// y' < YH, u_t slices of SLICE floats) collects the windows' gradients and goes to `blocks`.
template <int N>
struct BrickGeo {
    static constexpr int XH = kBX + N - 1, YH = kBY + N - 1, SLICE = (XH * YH + 3) / 4 * 4;
    static constexpr int BLOCK = N * SLICE;
};

template <int N, bool HANN>
__global__ void __launch_bounds__(kThreads, 2)
k5_spatial_adjoint_f32(const float* __restrict__ V, const float4* __restrict__ rtab, const float* __restrict__ gE,
                       float* __restrict__ blocks, int T, int X, int Y, int bnd, int t_begin) {
    using L = Lay<N>;
    using G = BrickGeo<N>;
    constexpr int H = N / 2 + 1;
    extern __shared__ __align__(16) float smem[];
    __shared__ float s_h[16];
    stage_taper<N>(s_h);
    const int g = threadIdx.x / L::LINES, l = threadIdx.x % L::LINES;
    float2* Fg = reinterpret_cast<float2*>(smem) + g * L::WIN;
    float2* Gg = reinterpret_cast<float2*>(smem) + (L::WPC + g) * L::WIN;
    float* blk = smem + 4 * L::WPC * L::WIN;
    for (int i = threadIdx.x; i < G::BLOCK; i += kThreads) blk[i] = 0.f;   // ordered before the first add by the
                                                                          // passes' barriers
    const int nseg = (Y + kBY - 1) / kBY;
    const int xs = blockIdx.x / nseg, sg = blockIdx.x % nseg, t = t_begin + blockIdx.y;
    const long long NV = (long long)T * X * Y;
    const int ut = l / N, ux = l % N;   // this thread's line of the last pass (along y)
    const float4* rrow = rtab + abs_bin<N>(l / N) * H + abs_bin<N>(l % N);   // its (k_x, k_y) line in the t passes
#pragma unroll 1
    for (int it = 0; it < kBX * kBY / L::WPC; ++it) {
        const int wi = it * L::WPC + g, wx = wi / kBY, wy = wi % kBY;
        const int x = xs * kBX + wx, y = sg * kBY + wy;
        const bool valid = x < X && y < Y;
        const long long q = ((long long)t * X + min(x, X - 1)) * Y + min(y, Y - 1);
        const float e0 = __ldg(gE + q), e1 = __ldg(gE + NV + q), e2 = __ldg(gE + 2 * NV + q);
        float re[N], im[N], ar[N], ai[N];
        // forward recompute: f_0 + i f_1 and f_2 (times n^3)
        load_window_line<N, HANN>(V, T, X, Y, bnd, t, min(x, X - 1), min(y, Y - 1), l, s_h, re, im);
        store_line<N, 2>(Fg, l, re, im);
        __syncthreads();
        fft_pass<N, 1, false>(Fg, l);
        __syncthreads();
        load_line<N, 0>(Fg, l, re, im);
        fft_line<N, false>(re, im);
        weigh_and_invert_t<N>(l, rtab, re, im, ar, ai);
        store_line<N, 0>(Gg, l, ar, ai);
        store_line<N, 0>(Fg, l, re, im);
        __syncthreads();
        fft_pass<N, 1, true>(Gg, l);
        fft_pass<N, 1, true>(Fg, l);
        __syncthreads();
        load_line<N, 2>(Gg, l, ar, ai);
        load_line<N, 2>(Fg, l, re, im);
        fft_line<N, true>(ar, ai);
        fft_line<N, true>(re, im);
        // the signs (sign(0) = 0), s_0 + i s_1 and s_2, transformed forward along y in the same registers
#pragma unroll
        for (int j = 0; j < N; ++j) {
            ar[j] = ar[j] > 0.f ? 1.f : ar[j] < 0.f ? -1.f : 0.f;
            ai[j] = ai[j] > 0.f ? 1.f : ai[j] < 0.f ? -1.f : 0.f;
            re[j] = re[j] > 0.f ? 1.f : re[j] < 0.f ? -1.f : 0.f;
            im[j] = 0.f;
        }
        fft_line<N, false>(ar, ai);
        fft_line<N, false>(re, im);
        store_line<N, 2>(Gg, l, ar, ai);
        store_line<N, 2>(Fg, l, re, im);
        __syncthreads();
        fft_pass<N, 1, false>(Gg, l);
        fft_pass<N, 1, false>(Fg, l);
        __syncthreads();
        // along t: Z = DFT(s_0 + i s_1) and S_2 = DFT(s_2) complete on this (k_x, k_y) line; the combined
        // spectrum U = (e_0 r_0 - i e_1 r_1) Z + e_2 r_2 S_2, inverted along t
        load_line<N, 0>(Gg, l, ar, ai);
        load_line<N, 0>(Fg, l, re, im);
        fft_line<N, false>(ar, ai);
        fft_line<N, false>(re, im);
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const float4 r = __ldg(rrow + abs_bin<N>(k) * H * H);
            const float a = e0 * r.x, b = e1 * r.y, c = e2 * r.z;
            const float ur = a * ar[k] + b * ai[k] + c * re[k];
            const float ui = a * ai[k] - b * ar[k] + c * im[k];
            re[k] = ur;
            im[k] = ui;
        }
        fft_line<N, true>(re, im);
        store_line<N, 0>(Fg, l, re, im);
        __syncthreads();
        fft_pass<N, 1, true>(Fg, l);
        __syncthreads();
        load_line<N, 2>(Fg, l, re, im);
        fft_line<N, true>(re, im);
        // gw = h3 (1/n^3) sum_m gE_m A_m s_m = h3 Re(IDFT(U)) / n^6 on this (u_t, u_x) line
        constexpr float sc = 1.f / ((float)(N * N * N) * (float)(N * N * N));
        const float hrow = HANN ? s_h[ut] * s_h[ux] : 1.f;
        float* dst = blk + ut * G::SLICE + (wx + ux) * G::YH + wy;
        // the windows of this iteration overlap: one group at a time, in window order
#pragma unroll 1
        for (int r = 0; r < L::WPC; ++r) {
            if (r == g && valid) {
#pragma unroll
                for (int j = 0; j < N; ++j) dst[j] += re[j] * (sc * (HANN ? hrow * s_h[j] : 1.f));
            }
            __syncthreads();
        }
    }
    float4* out = reinterpret_cast<float4*>(blocks + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * G::BLOCK);
    const float4* src = reinterpret_cast<const float4*>(blk);
    for (int i = threadIdx.x; i < G::BLOCK / 4; i += kThreads) out[i] = src[i];
}

template <int N>
constexpr int adjoint_smem_bytes() {
    return arrays_bytes<N>() + BrickGeo<N>::BLOCK * (int)sizeof(float);
}

template <int N, bool HANN>
cudaError_t set_attrs() {
    cudaError_t e = cudaFuncSetAttribute(k1_spatial_f32<N, HANN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         fwd_smem_bytes<N>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k5_spatial_adjoint_f32<N, HANN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                adjoint_smem_bytes<N>());
}

template <int N>
SpectraAdjointGeometry geometry_n() {
    using G = BrickGeo<N>;
    return SpectraAdjointGeometry{kBY, G::YH, kBX, G::XH, G::BLOCK, G::SLICE};
}

template <int N, bool HANN>
cudaError_t fwd_n(const float* V, const float4* rtab, float* E, int T, int X, int Y, int bnd, cudaStream_t s) {
    const dim3 grid((Y + Seg<N>::YB - 1) / Seg<N>::YB, X, T);   // T, X <= 65535 (checked at create)
    k1_spatial_f32<N, HANN><<<grid, kThreads, fwd_smem_bytes<N>(), s>>>(V, rtab, E, T, X, Y, bnd);
    return cudaGetLastError();
}

template <int N, bool HANN>
cudaError_t adj_n(const float* V, const float4* rtab, const float* gE, float* blocks, int T, int X, int Y, int bnd, int t_begin,
                  int t_count, cudaStream_t s) {
    const long long nb = (long long)((X + kBX - 1) / kBX) * ((Y + kBY - 1) / kBY);
    if (nb > 0x7fffffffLL || t_count > 65535) return cudaErrorInvalidValue;
    k5_spatial_adjoint_f32<N, HANN><<<dim3((unsigned)nb, t_count), kThreads, adjoint_smem_bytes<N>(), s>>>(
        V, rtab, gE, blocks, T, X, Y, bnd, t_begin);
    return cudaGetLastError();
}

}  // namespace

bool spatial_f32_supported(int n) { return n == 2 || n == 4 || n == 8 || n == 16; }

size_t spatial_weight_table_floats(int n) {
    const size_t h = (size_t)n / 2 + 1;
    return 4 * h * h * h;
}

void spatial_weight_table_fill(int n, float* out) {
    // r_m = P_m / |k| of Eq. 1 over the absolute signed indices a_t, a_x, a_y <= n/2 (zero at DC), in FP64,
    // rounded once: P_0^2 = a_x^2 + a_y^2, P_1^2 = a_t^2 + a_y^2, P_2^2 = a_t^2 + a_x^2
    const int h = n / 2 + 1;
    for (int at = 0; at < h; ++at)
        for (int ax = 0; ax < h; ++ax)
            for (int ay = 0; ay < h; ++ay) {
                const double r2 = (double)at * at + (double)ax * ax + (double)ay * ay;
                float* e = out + 4 * ((size_t)(at * h + ax) * h + ay);
                e[0] = r2 > 0 ? (float)std::sqrt(((double)ax * ax + (double)ay * ay) / r2) : 0.f;
                e[1] = r2 > 0 ? (float)std::sqrt(((double)at * at + (double)ay * ay) / r2) : 0.f;
                e[2] = r2 > 0 ? (float)std::sqrt(((double)at * at + (double)ax * ax) / r2) : 0.f;
                e[3] = 0.f;
            }
}

cudaError_t spatial_f32_prepare() {
    cudaError_t e;
    if ((e = set_attrs<2, false>()) != cudaSuccess || (e = set_attrs<2, true>()) != cudaSuccess ||
        (e = set_attrs<4, false>()) != cudaSuccess || (e = set_attrs<4, true>()) != cudaSuccess ||
        (e = set_attrs<8, false>()) != cudaSuccess || (e = set_attrs<8, true>()) != cudaSuccess ||
        (e = set_attrs<16, false>()) != cudaSuccess || (e = set_attrs<16, true>()) != cudaSuccess)
        return e;
    return cudaSuccess;
}

SpectraAdjointGeometry spatial_adjoint_f32_geometry(int n) {
    switch (n) {
        case 2: return geometry_n<2>();
        case 4: return geometry_n<4>();
        case 8: return geometry_n<8>();
        default: return geometry_n<16>();
    }
}

cudaError_t spatial_f32_launch(int n, const float* rtab, const float* V, float* E, int T, int X, int Y, int bnd, int taper,
                               cudaStream_t s) {
    const float4* rt = reinterpret_cast<const float4*>(rtab);
    cudaError_t e;
    switch (n * 2 + (taper ? 1 : 0)) {
        case 4: e = fwd_n<2, false>(V, rt, E, T, X, Y, bnd, s); break;
        case 5: e = fwd_n<2, true>(V, rt, E, T, X, Y, bnd, s); break;
        case 8: e = fwd_n<4, false>(V, rt, E, T, X, Y, bnd, s); break;
        case 9: e = fwd_n<4, true>(V, rt, E, T, X, Y, bnd, s); break;
        case 16: e = fwd_n<8, false>(V, rt, E, T, X, Y, bnd, s); break;
        case 17: e = fwd_n<8, true>(V, rt, E, T, X, Y, bnd, s); break;
        case 32: e = fwd_n<16, false>(V, rt, E, T, X, Y, bnd, s); break;
        case 33: e = fwd_n<16, true>(V, rt, E, T, X, Y, bnd, s); break;
        default: return cudaErrorInvalidValue;
    }
    if (e == cudaSuccess) note_launches(1);
    return e;
}

cudaError_t spatial_adjoint_f32_launch(int n, const float* rtab, const float* V, const float* gE, float* blocks, int T, int X, int Y,
                                       int bnd, int t_begin, int t_count, int taper, cudaStream_t s) {
    const float4* rt = reinterpret_cast<const float4*>(rtab);
    cudaError_t e;
    switch (n * 2 + (taper ? 1 : 0)) {
        case 4: e = adj_n<2, false>(V, rt, gE, blocks, T, X, Y, bnd, t_begin, t_count, s); break;
        case 5: e = adj_n<2, true>(V, rt, gE, blocks, T, X, Y, bnd, t_begin, t_count, s); break;
        case 8: e = adj_n<4, false>(V, rt, gE, blocks, T, X, Y, bnd, t_begin, t_count, s); break;
        case 9: e = adj_n<4, true>(V, rt, gE, blocks, T, X, Y, bnd, t_begin, t_count, s); break;
        case 16: e = adj_n<8, false>(V, rt, gE, blocks, T, X, Y, bnd, t_begin, t_count, s); break;
        case 17: e = adj_n<8, true>(V, rt, gE, blocks, T, X, Y, bnd, t_begin, t_count, s); break;
        case 32: e = adj_n<16, false>(V, rt, gE, blocks, T, X, Y, bnd, t_begin, t_count, s); break;
        case 33: e = adj_n<16, true>(V, rt, gE, blocks, T, X, Y, bnd, t_begin, t_count, s); break;
        default: return cudaErrorInvalidValue;
    }
    if (e == cudaSuccess) note_launches(1);
    return e;
}

}  // namespace sal
