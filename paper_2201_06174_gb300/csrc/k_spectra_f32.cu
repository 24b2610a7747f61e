// K1-F32: local 3D DFT around every voxel, spectral projection and feature, in FP32 on
// the SIMT pipes (Sec. 2 steps 1-3; Eq. 2 separable DFT, Eq. 1 projection).
//
// One CTA owns a line of BY output voxels (t0, x0, y_start .. y_start+BY-1).  It stages the
// halo brick V[t0-n/2 .. t0+n/2-1][x0-n/2 .. x0+n/2-1][y_start-n/2 .. y_start+BY+n/2-2] in
// shared memory (border extension applied at load) and runs the separable sliding DFT:
//   stage 1 (t, real input):  G1[k_t][x][y]  = sum_u c/s(k_t,u) V[t0-n/2+u][x][y],   k_t in [0,n/2]
//   stage 2 (x, complex):     G2[k_t][k_x][y] = sum_u c/s(k_x,u) G1[k_t][u][y],      k_x in [0,n)
//   stage 3 (y, complex):     F[k_t][k_x][k_y](y0) = sum_u c/s(k_y,u) G2[k_t][k_x][y0-n/2+u]
// Hermitian symmetry of a real cube keeps only k_t in [0, n/2] (multiplicity 2 for
// 0 < k_t < n/2).  Each one-axis DFT pairs bins k and n-k: with P = sum g cos, Q = sum g sin,
// F[k] = P - iQ and F[n-k] = P + iQ, which halves the multiplies.
// Sliding form of stage 3 (rect taper, n >= 8, one cube per voxel; the brick is staged minus one of its
// voxels): each thread takes the first output of its chunk by the direct sum and every later one by the
// recursion of the sliding DFT,
//   F_{y0+1}[k_y] = e^{2 pi i k_y / n} (F_{y0}[k_y] - G2[y0 - n/2] + G2[y0 + n/2])
// (the window drops its first sample, gains the next, and its phase origin moves by one), which
// costs O(1) per bin and output instead of O(n).
// Stage 3 is fused with the feature epilogue: |F| per bin (|F|^2 for the energy reading), weighted by
// the projection ratios r_m(k) of Eq. 1 (r_m^2 for the energy; zero at DC), summed over k_y in registers and over (k_t,k_x) rows through
// shared memory in a fixed order.  Per-voxel spectra never leave the SM.
#include "spectra_f32_common.cuh"

namespace sal {
namespace {

using f32::bin_mag;
using f32::Tw;

template <int N> struct Cfg;
template <> struct Cfg<2>  { static constexpr int BY = 32, YC = 1, MINB = 4; };
template <> struct Cfg<4>  { static constexpr int BY = 32, YC = 2, MINB = 4; };
template <> struct Cfg<8>  { static constexpr int BY = 64, YC = 8, MINB = 2; };
template <> struct Cfg<16> { static constexpr int BY = 32, YC = 16, MINB = 2; };

template <int N> struct Geo {
    static constexpr int H = N / 2 + 1;
    static constexpr int BY = Cfg<N>::BY;
    static constexpr int YC = Cfg<N>::YC;
    static constexpr int ROWS = H * N;             // (k_t, k_x) rows of stage 3
    static constexpr int NT = ROWS * (BY / YC);    // threads per CTA
    using B = f32::Brick<N, BY, NT>;
    static constexpr int YH = B::YH;
    static constexpr int PART_FLOATS = BY * 3 * ROWS;
    // region 1: G1 (stages 1-2), then the partial sums (stage 3, reduction); region 2: the halo brick
    // (staging, stage 1), then G2 (stages 2-3).  Each stage reads one region and writes the other.
    static constexpr size_t G_BYTES = (size_t)B::G_FLOAT2 * 8, IN_BYTES = (size_t)B::IN_FLOATS * 4;
    static constexpr size_t R1 = G_BYTES > (size_t)PART_FLOATS * 4 ? G_BYTES : (size_t)PART_FLOATS * 4;
    static constexpr size_t R2 = IN_BYTES > G_BYTES ? IN_BYTES : G_BYTES;
    static constexpr size_t SMEM = R1 + R2;
    static_assert(BY % YC == 0, "BY/YC");
    static_assert(NT <= 1024, "threads");
};

// Stage-3 forms: direct sum per output; direct on the lattice of multiples of `stride` (stride > 1);
// sliding recursion along y (rect taper, stride 1).
enum : int { kDirect = 0, kLattice = 1, kSliding = 2 };

// EN: the energy reading of the feature
template <int N, bool EN, int MODE>
__global__ void __launch_bounds__(Geo<N>::NT, Cfg<N>::MINB)
k1_spectra_f32(const float* __restrict__ V, float* __restrict__ E, int T, int X, int Y, int bnd, int stride,
               const float* __restrict__ wtab, const __grid_constant__ Tw<N> tw) {
    constexpr bool STR = MODE == kLattice;
    static_assert(MODE != kSliding || N >= 8, "the sliding form pays from n = 8");
    using G = Geo<N>;
    using B = typename G::B;
    constexpr int H = G::H, BY = G::BY, YC = G::YC, YH = G::YH, ROWS = G::ROWS, NT = G::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* s_g1 = reinterpret_cast<float2*>(smem_raw);                              // [H][N][YH]    region 1
    float* s_part = reinterpret_cast<float*>(smem_raw);                              // [BY][3][ROWS] region 1
    float* s_in = reinterpret_cast<float*>(smem_raw + G::R1);                        // [N][N][YH]    region 2
    float2* s_g2 = reinterpret_cast<float2*>(smem_raw + G::R1);                      // [H][N][YH]    region 2

    const int tid = threadIdx.x;
    const int y_start = blockIdx.x * BY;
    const int x0 = blockIdx.y * stride;   // stride s: cubes only at indices that are multiples of s
    const int t0 = blockIdx.z * stride;

    // Sliding form: the brick minus one of its voxels.  Every non-DC bin is unchanged (rect taper), and a
    // constant region stages exact zeros, whose spectra the recursion keeps at zero; without the shift the
    // rounding residues of its non-DC bins would be rotated differently at each output.
    const float vshift = MODE == kSliding ? __ldg(V + ((size_t)t0 * X + x0) * Y + y_start) : 0.f;
    B::stage_brick(V, s_in, T, X, Y, bnd, t0, x0, y_start, vshift);
    __syncthreads();
    B::stage1(s_in, s_g1, tw);
    __syncthreads();
    B::stage2(s_g1, s_g2, tw);
    __syncthreads();

    // ---- stage 3 + projection/feature epilogue ----------------------------------------------
    const int row = tid % ROWS;           // (k_t, k_x)
    const int ych = tid / ROWS;           // chunk of YC outputs
    float wt[3][H];                       // r_m(k_t,k_x,+-k_y) (r_m^2: energy) * multiplicity / n^3
    B::row_weights(wtab, row, wt);
    const float2* grow = s_g2 + (size_t)row * YH;
    if (MODE == kSliding) {
        float fr[N], fi[N];   // F[k_y] of the current output, all n bins
        {
            const float2* g0 = grow + ych * YC;
            float pr[H], pi[H], qr[H], qi[H];
#pragma unroll
            for (int k = 0; k < H; ++k) pr[k] = pi[k] = qr[k] = qi[k] = 0.f;
#pragma unroll
            for (int u = 0; u < N; ++u) {
                const float2 g = g0[u];
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
#pragma unroll
            for (int k = 0; k < H; ++k) {
                if (k == 0 || 2 * k == N) {
                    fr[k] = pr[k];
                    fi[k] = pi[k];
                } else {
                    fr[k] = pr[k] + qi[k];       // F[k]   = P - iQ
                    fi[k] = pi[k] - qr[k];
                    fr[N - k] = pr[k] - qi[k];   // F[n-k] = P + iQ
                    fi[N - k] = pi[k] + qr[k];
                }
            }
        }
        for (int j = 0; j < YC; ++j) {
            const int yl = ych * YC + j;
            if (j > 0) {
                const float2 a = grow[yl - 1], b = grow[yl - 1 + N];   // sample leaving, sample entering
                const float dr = b.x - a.x, di = b.y - a.y;
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    // e^{2 pi i k / n}: the twiddles at u = 1 (rect taper), sine negated above n/2
                    const float c = k <= N / 2 ? tw.c[k][1] : tw.c[N - k][1];
                    const float sn = k <= N / 2 ? tw.s[k][1] : -tw.s[N - k][1];
                    const float xr = fr[k] + dr, xi = fi[k] + di;
                    fr[k] = fmaf(c, xr, -sn * xi);
                    fi[k] = fmaf(sn, xr, c * xi);
                }
            }
            float e0 = 0.f, e1 = 0.f, e2 = 0.f;
#pragma unroll
            for (int k = 0; k < H; ++k) {
                float a = bin_mag<EN>(fmaf(fr[k], fr[k], fi[k] * fi[k]));
                if (k != 0 && 2 * k != N) a += bin_mag<EN>(fmaf(fr[N - k], fr[N - k], fi[N - k] * fi[N - k]));
                e0 = fmaf(wt[0][k], a, e0);
                e1 = fmaf(wt[1][k], a, e1);
                e2 = fmaf(wt[2][k], a, e2);
            }
            s_part[(yl * 3 + 0) * ROWS + row] = e0;
            s_part[(yl * 3 + 1) * ROWS + row] = e1;
            s_part[(yl * 3 + 2) * ROWS + row] = e2;
        }
    }
    for (int yl = ych * YC; MODE != kSliding && yl < ych * YC + YC; ++yl) {
        if (STR && (y_start + yl) % stride != 0) continue;
        float pr[H], pi[H], qr[H], qi[H];
#pragma unroll
        for (int k = 0; k < H; ++k) pr[k] = pi[k] = qr[k] = qi[k] = 0.f;
#pragma unroll
        for (int u = 0; u < N; ++u) {
            const float2 g = grow[yl + u];
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
        float e0 = 0.f, e1 = 0.f, e2 = 0.f;
#pragma unroll
        for (int k = 0; k < H; ++k) {
            float a;
            if (k == 0 || 2 * k == N) {
                a = bin_mag<EN>(fmaf(pr[k], pr[k], pi[k] * pi[k]));
            } else {
                const float ar = pr[k] + qi[k], ai = pi[k] - qr[k];   // F[k]   = P - iQ
                const float br = pr[k] - qi[k], bi = pi[k] + qr[k];   // F[n-k] = P + iQ
                a = bin_mag<EN>(fmaf(ar, ar, ai * ai)) + bin_mag<EN>(fmaf(br, br, bi * bi));
            }
            e0 = fmaf(wt[0][k], a, e0);
            e1 = fmaf(wt[1][k], a, e1);
            e2 = fmaf(wt[2][k], a, e2);
        }
        s_part[(yl * 3 + 0) * ROWS + row] = e0;
        s_part[(yl * 3 + 1) * ROWS + row] = e1;
        s_part[(yl * 3 + 2) * ROWS + row] = e2;
    }
    __syncthreads();

    // ---- fixed-order reduction over the (k_t, k_x) rows ---------------------------------------
    // E: [3][T][X][Y], or the lattice [3][Tc][Xc][Yc] (ceil(T / s) ...) for stride s > 1
    const int Xc = (X + stride - 1) / stride, Yc = (Y + stride - 1) / stride;
    const size_t NVc = (size_t)((T + stride - 1) / stride) * Xc * Yc;
    const int lane = tid & 31, warp = tid >> 5;
    for (int it = warp; it < BY * 3; it += NT / 32) {
        const int yl = it / 3, m = it % 3;
        const int y = y_start + yl;
        if (STR && y % stride != 0) continue;
        const float* p = s_part + (size_t)(yl * 3 + m) * ROWS;
        float acc = 0.f;
        for (int r = lane; r < ROWS; r += 32) acc += p[r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0 && y < Y) {
            if (STR) E[m * NVc + ((size_t)(t0 / stride) * Xc + x0 / stride) * Yc + y / stride] = acc;
            else E[m * NVc + ((size_t)t0 * X + x0) * Y + y] = acc;
        }
    }
}

template <int N, bool EN, int MODE>
cudaError_t prepare_one() {
    return cudaFuncSetAttribute(k1_spectra_f32<N, EN, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Geo<N>::SMEM);
}

template <int N> constexpr bool kHasSliding = N >= 8;

template <int N>
cudaError_t prepare() {
    cudaError_t e = prepare_one<N, false, kDirect>();
    if (e == cudaSuccess) e = prepare_one<N, true, kDirect>();
    if (e == cudaSuccess) e = prepare_one<N, false, kLattice>();
    if (e == cudaSuccess) e = prepare_one<N, true, kLattice>();
    if constexpr (kHasSliding<N>) {
        if (e == cudaSuccess) e = prepare_one<N, false, kSliding>();
        if (e == cudaSuccess) e = prepare_one<N, true, kSliding>();
    }
    return e;
}

template <int N, int MODE>
void launch_mode(const Tw<N>& tw, const float* wtab, dim3 grid, const float* V, float* E, int T, int X, int Y,
                 int bnd, int feat, int stride, cudaStream_t s) {
    using G = Geo<N>;
    if (feat == 1) k1_spectra_f32<N, true, MODE><<<grid, G::NT, G::SMEM, s>>>(V, E, T, X, Y, bnd, stride, wtab, tw);
    else k1_spectra_f32<N, false, MODE><<<grid, G::NT, G::SMEM, s>>>(V, E, T, X, Y, bnd, stride, wtab, tw);
}

template <int N>
cudaError_t launch(const TwiddleTable& t, const float* wtab, const float* V, float* E, int T, int X, int Y,
                   int bnd, int feat, int stride, bool rect, cudaStream_t s) {
    using G = Geo<N>;
    dim3 grid((Y + G::BY - 1) / G::BY, (X + stride - 1) / stride, (T + stride - 1) / stride);
    const Tw<N> tw = f32::make_tw<N>(t);
    if (stride > 1) {
        launch_mode<N, kLattice>(tw, wtab, grid, V, E, T, X, Y, bnd, feat, stride, s);
    } else if constexpr (kHasSliding<N>) {
        if (rect) launch_mode<N, kSliding>(tw, wtab, grid, V, E, T, X, Y, bnd, feat, 1, s);
        else launch_mode<N, kDirect>(tw, wtab, grid, V, E, T, X, Y, bnd, feat, 1, s);
    } else {
        launch_mode<N, kDirect>(tw, wtab, grid, V, E, T, X, Y, bnd, feat, 1, s);
    }
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace

bool spectra_f32_supported(int n) { return n == 2 || n == 4 || n == 8 || n == 16; }

size_t f32_weight_table_floats(int n) {
    const int h = n / 2 + 1;
    return (size_t)3 * h * h * n;
}

void f32_weight_table_fill(int n, int feat, float* out) {
    if (feat == 1) f32::f32_weight_table<true>(n, out);
    else f32::f32_weight_table<false>(n, out);
}

cudaError_t spectra_f32_prepare(int n) {
    switch (n) {
        case 2: return prepare<2>();
        case 4: return prepare<4>();
        case 8: return prepare<8>();
        case 16: return prepare<16>();
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t spectra_f32_launch(int n, const TwiddleTable& tw, const float* wtab, const float* V, float* E, int T,
                               int X, int Y, int bnd, int feat, int stride, int taper, cudaStream_t s) {
    if (T > 65535 || X > 65535 || stride < 1) return cudaErrorInvalidConfiguration;
    const bool rect = taper == 0;
    switch (n) {
        case 2: return launch<2>(tw, wtab, V, E, T, X, Y, bnd, feat, stride, rect, s);
        case 4: return launch<4>(tw, wtab, V, E, T, X, Y, bnd, feat, stride, rect, s);
        case 8: return launch<8>(tw, wtab, V, E, T, X, Y, bnd, feat, stride, rect, s);
        case 16: return launch<16>(tw, wtab, V, E, T, X, Y, bnd, feat, stride, rect, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sal
