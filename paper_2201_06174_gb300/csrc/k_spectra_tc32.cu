// K1-TC for the 32^3 window (Sec. 2 steps 1-3; Eq. 2, Eq. 1): stage 3 (the DFT along y of every
// (k_t, k_x) row) on the tensor cores, as for the smaller windows, with the shapes of n = 32:
//   rows m = (x0 - xb) * 32 + k_x, 4 positions x 32 k_x = 128;
//   B = the 32 twiddle columns over 32 taps (two K steps), each bin's cosine and sine side by side:
//     column 0: cos k = 0, column 1: cos k = 16 (the self-paired bins), columns 2j, 2j + 1: cos j, sin j;
//   one output y0 = 64 TMEM columns (real part of A x B | imaginary part of A x B), read back in halves of
//     16 columns that hold whole (cos, sin) pairs;
//   the halo brick is staged in FP16 after a per-brick 1/max|V| scale (the FP32 brick of a 32^3
//   window exceeds shared memory);
//   stage 1 (t) per k_t on the SIMT pipes (FP32 sums over the 32 taps), written as the stage-2 B operand
//     B2[(re|im, y)][(cos|sin, x)] = [[G1r, G1i], [G1i, -G1r]] (16-bit, K-major, x over a 40-row halo);
//   stage 2 (x) on the tensor cores as in the smaller windows: A2 = the Toeplitz twiddles
//     h(x - x0) [cos | sin](2 pi k_x (x - x0) / n), built once per CTA, so one MMA chain (K = 80, N = 96)
//     gives Re G2 and Im G2 of every (x0, k_x) row and halo column y; D2 is rounded into the stage-3 A.
// 16 warps (one CTA per SM: the halo fills shared memory): the SIMT stage needs the warps to hide its
// latency; in the epilogue the four warps of a tensor-memory lane quarter take two outputs of each pass.
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
constexpr int kThreads = 512;
constexpr uint32_t kTmemCols = 512;                      // 8 outputs x 64 columns
constexpr uint32_t kWaitLimit = 1u << 22;

constexpr int XHP = 40;                                  // x halo rows of stage 2 (>= XH, multiple of 8)
constexpr int YP = 48;                                   // y columns of stage 2 (>= YH, multiple of 8)
constexpr int K2 = 2 * XHP;                              // stage-2 K: cos taps | sin taps
constexpr int N2 = 2 * YP;                               // stage-2 N: re | im over y
constexpr uint32_t SBO_K2 = K2 / 8 * 128;                // 8-row group stride of the K-major A2 / B2
constexpr size_t IN_B = (size_t)N * XH * YH * 2;         // FP16 halo
constexpr size_t B2_B = (size_t)N2 / 8 * SBO_K2;         // stage-2 B (one k_t)
constexpr size_t A2_B = (size_t)16 * SBO_K2;             // stage-2 A (128 rows)
constexpr size_t A_B = (size_t)16 * SBO_A;
constexpr size_t B_B = 2048;
constexpr size_t WT_B = (size_t)N * H * 3 * 4;
constexpr size_t OFF_B2 = (IN_B + 127) / 128 * 128;
constexpr size_t OFF_A2 = OFF_B2 + B2_B;
constexpr size_t OFF_A = OFF_A2 + A2_B;
constexpr size_t OFF_B = OFF_A + 2 * A_B;
constexpr size_t OFF_WT = OFF_B + B_B;
constexpr size_t OFF_MISC = OFF_WT + 2 * WT_B;                 // the weight table, double-buffered by k_t
constexpr size_t SMEM = OFF_MISC + 64 + (kThreads / 32) * 4;
static_assert(SMEM <= 227 * 1024, "shared memory");
static_assert(XH <= XHP && YH <= YP && N2 <= 256 && N2 % 16 == 0, "stage-2 shapes");
static_assert(OFF_B2 % 128 == 0 && OFF_A2 % 128 == 0 && OFF_A % 16 == 0, "operand alignment");

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
    unsigned char* s_b2 = smem + OFF_B2;                                // stage-2 B (K-major)
    unsigned char* s_a2 = smem + OFF_A2;                                // stage-2 A (K-major)
    unsigned char* s_are = smem + OFF_A;
    unsigned char* s_aim = smem + OFF_A + A_B;
    unsigned char* s_b = smem + OFF_B;                                  // [32 n][32 k], K-major
    float* s_wt = reinterpret_cast<float*>(smem + OFF_WT);              // [2][k_x][k][3]: tiles k_t, k_t + 1
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
        const float v = n == 0 ? tw.c[0][k] : n == 1 ? tw.c[N / 2][k] : (n & 1) ? tw.s[n / 2][k] : tw.c[n / 2][k];
        *reinterpret_cast<uint16_t*>(s_b + (n / 8) * 512 + (k / 8) * 128 + (n % 8) * 16 + (k % 8) * 2) =
            Pack<FMT>::one(v);
    }
    for (int i = tid; i < (int)(2 * A_B / 16); i += kThreads)
        reinterpret_cast<uint4*>(s_are)[i] = make_uint4(0u, 0u, 0u, 0u);
    // B2 rows and columns past the halo stay zero (A2 is zero there too, but 0 x garbage could be NaN)
    for (int i = tid; i < (int)(B2_B / 16); i += kThreads)
        reinterpret_cast<uint4*>(s_b2)[i] = make_uint4(0u, 0u, 0u, 0u);
    // A2[(x0l, k_x)][k2]: k2 < XHP: cos, else sin, of (k_x, x - x0l), x = k2 % XHP; zero outside the window
    for (int i = tid; i < 128 * K2; i += kThreads) {
        const int mm = i / K2, k2 = i % K2;
        const int x0 = mm / N, kxx = mm % N, u = k2 % XHP - x0;
        float v = 0.f;
        if (u >= 0 && u < N) {
            const bool lo = kxx <= N / 2;
            const int kk = lo ? kxx : N - kxx;
            v = k2 < XHP ? tw.c[kk][u] : (lo ? tw.s[kk][u] : -tw.s[kk][u]);
        }
        *reinterpret_cast<uint16_t*>(s_a2 + (mm / 8) * SBO_K2 + (k2 / 8) * 128 + (mm % 8) * 16 + (k2 % 8) * 2) =
            Pack<FMT>::one(v);
    }
    // The halo brick, two passes over global memory (its maximum, then the scaled FP16 copy): a warp per
    // (u_t, x) row of YH samples, each lane samples y = lane and lane + 32 (its two border-extended source
    // columns fixed for the whole brick), RU rows in flight per warp.
    constexpr int ROWS = N * XH, RU = 4;
    const int gy0 = ext_index(yb - N / 2 + lane, Y, bnd);
    const int gy1 = lane + 32 < YH ? ext_index(yb - N / 2 + lane + 32, Y, bnd) : -1;
    auto halo_rows = [&](auto&& use) {
        for (int r0 = warp * RU; r0 < ROWS; r0 += (kThreads / 32) * RU) {
            float v0[RU], v1[RU];
#pragma unroll
            for (int a = 0; a < RU; ++a) {   // loads first
                const int r = r0 + a;
                v0[a] = v1[a] = 0.f;
                if (r < ROWS) {
                    const int gt = ext_index(t0 - N / 2 + r / XH, T, bnd);
                    const int gx = ext_index(xb - N / 2 + r % XH, X, bnd);
                    if ((gt | gx) >= 0) {
                        const float* row = V + ((size_t)gt * X + gx) * Y;
                        if (gy0 >= 0) v0[a] = __ldg(row + gy0);
                        if (gy1 >= 0) v1[a] = __ldg(row + gy1);
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < RU; ++a)
                if (r0 + a < ROWS) use(r0 + a, v0[a], v1[a]);
        }
    };
    float vmax = 0.f;
    halo_rows([&](int, float a, float b) { vmax = fmaxf(vmax, fmaxf(fabsf(a), fabsf(b))); });
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
    halo_rows([&](int r, float a, float b) {   // s_in[u][x][y], row r = u XH + x
        s_in[(size_t)r * YH + lane] = __float2half_rn(a * inv_scale);
        if (lane + 32 < YH) s_in[(size_t)r * YH + lane + 32] = __float2half_rn(b * inv_scale);
    });

    const int q = warp & 3, sub = warp >> 2;   // lane quarter; outputs sub and sub + 4 of each pass
    const int m = 32 * q + lane;
    const int x0l = m / N, kx = m % N;
    float acc[4][3];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = acc[i][2] = 0.f;
    const uint32_t idesc = tc::idesc_f16(FMT, 128, 32, 1, 0);
    const uint32_t bsm = tc::smem_u32(s_b), are = tc::smem_u32(s_are), aim = tc::smem_u32(s_aim);
    uint32_t phase = 0;

    // The SIMT part of tile kt: its Eq. 1 weight table (buffer kt % 2) and stage 1 (t) into the stage-2 B
    // operand.  Tile 0 runs before the loop; tile kt + 1 runs while the last stage-3 MMAs of tile kt execute.
    auto prep_tile = [&](int kt) {
        float cr[N], sr[N];
#pragma unroll
        for (int u = 0; u < N; ++u) {
            cr[u] = tw.c[kt][u];
            sr[u] = tw.s[kt][u];
        }
        float* wtab = s_wt + (kt & 1) * (N * H * 3);
        for (int i = tid; i < N * H; i += kThreads) {
            const int k = i % H, x = i / H;
            const int ii = kt, j = x < N / 2 ? x : x - N;
            const float mult = (kt == 0 || 2 * kt == N) ? 1.f : 2.f;
            float w0, w1, w2;
            f32::bin_weights<EN>(ii, j, k, mult / (float)(N * N * N), w0, w1, w2);
            wtab[i * 3 + 0] = w0;
            wtab[i * 3 + 1] = w1;
            wtab[i * 3 + 2] = w2;
        }
        // stage 1 (t): G1 = P - iQ of every halo position, into B2 (K-major: byte(ncol, k2) = (ncol/8) SBO_K2 +
        // (k2/8) 128 + (ncol%8) 16 + (k2%8) 2; ncol = y (re) or YP + y (im), k2 = x (cos) or XHP + x (sin))
        for (int it = tid; it < XH * YH; it += kThreads) {
            float Pv = 0.f, Qv = 0.f;
#pragma unroll
            for (int u = 0; u < N; ++u) {
                const float v = __half2float(s_in[u * XH * YH + it]);
                Pv = fmaf(v, cr[u], Pv);
                Qv = fmaf(v, sr[u], Qv);
            }
            const int x = it / YH, y = it % YH;
            const size_t o_re = (size_t)(y / 8) * SBO_K2 + (y % 8) * 16;
            const size_t o_im = (size_t)((YP + y) / 8) * SBO_K2 + ((YP + y) % 8) * 16;
            const size_t k_c = (size_t)(x / 8) * 128 + (x % 8) * 2;
            const size_t k_s = (size_t)((XHP + x) / 8) * 128 + ((XHP + x) % 8) * 2;
            *reinterpret_cast<uint16_t*>(s_b2 + o_re + k_c) = Pack<FMT>::one(Pv);
            *reinterpret_cast<uint16_t*>(s_b2 + o_re + k_s) = Pack<FMT>::one(-Qv);
            *reinterpret_cast<uint16_t*>(s_b2 + o_im + k_c) = Pack<FMT>::one(-Qv);
            *reinterpret_cast<uint16_t*>(s_b2 + o_im + k_s) = Pack<FMT>::one(-Pv);
        }
        tc::fence_async_smem();
    };
    __syncthreads();   // the halo is staged
    prep_tile(0);

    for (int kt = 0; kt < H; ++kt) {
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        // stage 2 (x) on the tensor cores: D2[(x0, k_x)][(re | im, y)] = A2 B2 in tensor-memory columns [0, N2)
        {
            if (tid == 0 && !*s_fail) {
                tc::fence_after_sync();
                const uint32_t idesc2 = tc::idesc_f16(FMT, 128, N2, 0, 0);
                const uint64_t a2d = tc::desc_noswizzle(tc::smem_u32(s_a2), 128, SBO_K2);
                const uint64_t b2d = tc::desc_noswizzle(tc::smem_u32(s_b2), 128, SBO_K2);
#pragma unroll
                for (int ks = 0; ks < K2 / 16; ++ks)
                    tc::mma_f16(tmem, tc::desc_add(a2d, 256 * ks), tc::desc_add(b2d, 256 * ks), idesc2, ks > 0 ? 1u : 0u);
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
            // D2 -> the stage-3 A operands (row m at K row y, 2-byte stores): three warps per lane quarter, one
            // 32-column chunk each (columns [0, YP): real part over y, [YP, 2 YP): imaginary part)
            if (!bad && sub < 3) {
                float v[32];
                tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * sub), v);
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int c = 32 * sub + i, part = c / YP, y = c % YP;
                    if (y < YH) {
                        unsigned char* dst = (part ? s_aim : s_are) + (size_t)(m / 8) * SBO_A + (size_t)y * 16 + (m % 8) * 2;
                        *reinterpret_cast<uint16_t*>(dst) = Pack<FMT>::one(v[i]);
                    }
                }
            }
            tc::fence_async_smem();
            tc::fence_before_sync();
            __syncthreads();
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
            // under the last MMAs of this tile: the next tile's weights and stage 1 (B2 and the other weight
            // buffer are free: this tile's stage-2 MMAs have completed)
            if (pass == 1 && kt + 1 < H) prep_tile(kt + 1);
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
                float wt[3][H];   // this lane's Eq. 1 weights for (k_t, k_x), |k_y| = 0 .. n/2
                const float* wtab = s_wt + (kt & 1) * (N * H * 3);
#pragma unroll
                for (int k = 0; k < H; ++k) {
                    const float* w = wtab + (kx * H + k) * 3;
                    wt[0][k] = w[0];
                    wt[1][k] = w[1];
                    wt[2][k] = w[2];
                }
#pragma unroll
                for (int jj = 0; jj < 2; ++jj) {
                    const int j = sub + 4 * jj;
                    float e0 = 0.f, e1 = 0.f, e2 = 0.f;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {   // columns 16 h .. 16 h + 15: bins k = 8 h .. 8 h + 7
                        float vr[16], vi[16];
                        tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(j * 64 + 16 * h), vr);
                        tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(j * 64 + 32 + 16 * h), vi);
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            const int k = 8 * h + c;
                            const float pr = vr[2 * c], pi = vi[2 * c], qr = vr[2 * c + 1], qi = vi[2 * c + 1];
                            if (k == 0) {   // columns 0, 1: the self-paired bins 0 and n/2
                                const float a0 = bin_mag<EN>(fmaf(pr, pr, pi * pi));
                                const float a1 = bin_mag<EN>(fmaf(qr, qr, qi * qi));
                                e0 = fmaf(wt[0][0], a0, fmaf(wt[0][H - 1], a1, e0));
                                e1 = fmaf(wt[1][0], a0, fmaf(wt[1][H - 1], a1, e1));
                                e2 = fmaf(wt[2][0], a0, fmaf(wt[2][H - 1], a1, e2));
                            } else {        // bins k and n - k: P = pr + i pi, Q = qr + i qi
                                const float ar = pr + qi, ai = pi - qr, br = pr - qi, bi = pi + qr;
                                const float a = bin_mag<EN>(fmaf(ar, ar, ai * ai)) + bin_mag<EN>(fmaf(br, br, bi * bi));
                                e0 = fmaf(wt[0][k], a, e0);
                                e1 = fmaf(wt[1][k], a, e1);
                                e2 = fmaf(wt[2][k], a, e2);
                            }
                        }
                    }
                    acc[pass * 2 + jj][0] += e0;
                    acc[pass * 2 + jj][1] += e1;
                    acc[pass * 2 + jj][2] += e2;
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
    for (int i = 0; i < 4; ++i) {
        const int y0 = (i / 2) * 8 + sub + 4 * (i % 2);
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
