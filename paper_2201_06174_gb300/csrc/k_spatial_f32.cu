// K1 for the spatial-domain reading of the feature step (Sec. 2 step 3; Eq. 1, Eq. 2), FP32, n <= 8:
//   E_m[p] = (1/n^3) sum_u |f_m[u]|,   f_m = IDFT(r_m DFT(w)),
// w the (tapered) cube of voxel p.  IDFT diag(r_m) DFT is the circulant of the real kernel
// h_m = IDFT(r_m) (r_m is even in k), so f_m[u] = sum_v w[v] h_m[(u - v) mod n]: n^6 FMAs per map and
// voxel, evaluated directly (a first form: exact, not fast).  One CTA per 128 consecutive voxels of a
// (t, x) row: the halo [n][n][128 + n - 1] of V in shared memory (border extension applied at load), the
// three kernels h_m and the taper beside it (from the handle's table); one thread per voxel.
#include <cmath>

#include "sal_internal.cuh"

namespace sal {
namespace {

constexpr int kThreads = 128;

template <int N, bool HANN>
__global__ void __launch_bounds__(kThreads)
k1_spatial_f32(const float* __restrict__ V, float* __restrict__ E, int T, int X, int Y, int bnd,
               const float* __restrict__ tab) {
    constexpr int N3 = N * N * N, YH = kThreads + N - 1;
    static_assert((N & (N - 1)) == 0 && N <= 8, "power-of-two windows up to 8");
    __shared__ float s_in[N][N][YH];
    __shared__ float s_h[3][N3];   // h_m[u_t][u_x][u_y], 1/n^3 of the inverse DFT included
    __shared__ float s_tp[N3];     // taper h(u_t) h(u_x) h(u_y)
    const int t = blockIdx.z, x = blockIdx.y, y0 = blockIdx.x * kThreads;
    for (int i = threadIdx.x; i < 4 * N3; i += kThreads) {
        if (i < 3 * N3) s_h[i / N3][i % N3] = __ldg(tab + i);
        else s_tp[i - 3 * N3] = __ldg(tab + i);
    }
    for (int i = threadIdx.x; i < N * N * YH; i += kThreads) {
        const int yy = i % YH, ux = (i / YH) % N, ut = i / (YH * N);
        const int gt = ext_index(t - N / 2 + ut, T, bnd), gx = ext_index(x - N / 2 + ux, X, bnd);
        const int gy = ext_index(y0 - N / 2 + yy, Y, bnd);
        s_in[ut][ux][yy] = (gt | gx | gy) >= 0 ? __ldg(V + ((size_t)gt * X + gx) * Y + gy) : 0.f;
    }
    __syncthreads();   // the only barrier: threads past the row's end leave after it
    const int yl = threadIdx.x, y = y0 + yl;
    if (y >= Y) return;
    const size_t NV = (size_t)T * X * Y, q = ((size_t)t * X + x) * Y + y;
#pragma unroll 1
    for (int m = 0; m < 3; ++m) {
        float acc = 0.f;
#pragma unroll 1
        for (int u = 0; u < N3; ++u) {
            const int ut = u / (N * N), ux = (u / N) % N, uy = u % N;
            float f = 0.f;
#pragma unroll 1
            for (int vt = 0; vt < N; ++vt)
#pragma unroll 1
                for (int vx = 0; vx < N; ++vx) {
                    const float* hrow = s_h[m] + ((ut - vt) & (N - 1)) * N * N + ((ux - vx) & (N - 1)) * N;
                    const float* wrow = &s_in[vt][vx][yl];
                    const float* trow = s_tp + (vt * N + vx) * N;
#pragma unroll
                    for (int vy = 0; vy < N; ++vy) {
                        const float w = HANN ? wrow[vy] * trow[vy] : wrow[vy];
                        f = fmaf(w, hrow[(uy - vy) & (N - 1)], f);
                    }
                }
            acc += fabsf(f);
        }
        E[m * NV + q] = acc * (1.f / N3);
    }
}

template <int N, bool HANN>
void launch_n(const float* V, float* E, int T, int X, int Y, int bnd, const float* tab, cudaStream_t s) {
    const dim3 grid((Y + kThreads - 1) / kThreads, X, T);   // T, X <= 65535 (checked at create)
    k1_spatial_f32<N, HANN><<<grid, kThreads, 0, s>>>(V, E, T, X, Y, bnd, tab);
}

}  // namespace

bool spatial_f32_supported(int n) { return n == 2 || n == 4 || n == 8; }

size_t spatial_table_floats(int n) { return (size_t)4 * n * n * n; }

void spatial_table_fill(int n, int taper, float* out) {
    // h_m[u] = (1/n^3) sum_k r_m(k) cos(2 pi k.u / n) (the sine part cancels: r_m is even in k), r_m the
    // Eq. 1 ratio over signed bin indices (zero at DC); then the taper over the cube
    const int n3 = n * n * n;
    auto sgn = [n](int k) { return k < n / 2 ? k : k - n; };
    for (int m = 0; m < 3; ++m)
        for (int u = 0; u < n3; ++u) {
            const int ut = u / (n * n), ux = (u / n) % n, uy = u % n;
            double a = 0.0;
            for (int k = 0; k < n3; ++k) {
                const int kt = k / (n * n), kx = (k / n) % n, ky = k % n;
                const double i = sgn(kt), j = sgn(kx), l = sgn(ky);
                const double r = std::sqrt(i * i + j * j + l * l);
                if (r == 0.0) continue;
                const double P = m == 0 ? std::sqrt(j * j + l * l) : m == 1 ? std::sqrt(i * i + l * l)
                                                                        : std::sqrt(i * i + j * j);
                a += P / r * std::cos(2.0 * M_PI * (double)(kt * ut + kx * ux + ky * uy) / n);
            }
            out[m * n3 + u] = (float)(a / n3);
        }
    for (int u = 0; u < n3; ++u) {
        const int c[3] = {u / (n * n), (u / n) % n, u % n};
        double w = 1.0;
        for (int a = 0; a < 3; ++a) w *= taper ? 0.5 - 0.5 * std::cos(2.0 * M_PI * c[a] / n) : 1.0;
        out[3 * n3 + u] = (float)w;
    }
}

cudaError_t spatial_f32_launch(int n, const float* tab, const float* V, float* E, int T, int X, int Y, int bnd,
                               int taper, cudaStream_t s) {
    switch (n * 2 + (taper ? 1 : 0)) {
        case 4: launch_n<2, false>(V, E, T, X, Y, bnd, tab, s); break;
        case 5: launch_n<2, true>(V, E, T, X, Y, bnd, tab, s); break;
        case 8: launch_n<4, false>(V, E, T, X, Y, bnd, tab, s); break;
        case 9: launch_n<4, true>(V, E, T, X, Y, bnd, tab, s); break;
        case 16: launch_n<8, false>(V, E, T, X, Y, bnd, tab, s); break;
        case 17: launch_n<8, true>(V, E, T, X, Y, bnd, tab, s); break;
        default: return cudaErrorInvalidValue;
    }
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace sal
