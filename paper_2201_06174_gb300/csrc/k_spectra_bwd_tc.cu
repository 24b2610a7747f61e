// K5-TC: adjoint of the local-spectrum feature step (backward of Sec. 2 steps 1-3; Eq. 1, Eq. 2)
// with both dense contractions along y on the tensor cores (tcgen05.mma, BF16/FP16 operands,
// FP32 accumulation in tensor memory).  Same brick as K1-TC: t0, x0 in [xb, xb + P), P = 128/n,
// y0 in [yb, yb + 16).  For each k_t tile:
//   stages 1-2 (SIMT, FP32) and the forward stage-3 MMAs, as in K1-TC (spectra recomputed);
//   Gamma (epilogue from TMEM): Gamma[k] = (sum_m gE_m wt_m(k)) F[k]/|F[k]| (zero subgradient where
//     |F| <= 2^-19 of the window's L1 norm), folded into the pair coefficients of the inverse DFT:
//     A_k = Gamma[k] + Gamma[n-k], B_k = i (Gamma[k] - Gamma[n-k]) (self-paired bins: A_k = Gamma[k]);
//   inverse along y on the tensor cores: one MMA per output y0 and real/imaginary part with
//     B_{y0}[y][j] = T[j][y - y0] (the twiddle table shifted to the window of y0), all y0
//     accumulating into one TMEM accumulator -- the overlap-add over the sliding windows happens in
//     the accumulator: Gamma_G2[row][y] = sum_y0 sum_j Gamma'_{y0}[row][j] T[j][y - y0];
//   adjoint of stage 2 (x) and of stage 1 (t) on the SIMT pipes, accumulated over k_t tiles into
//     the brick's block of gVext [u_t][x][y] in shared memory, written to scratch at the end; the
//     fixed-order gather kernel sums the overlapping blocks.
// Low-precision operands are FP16 (3 more mantissa bits than BF16: the direction F/|F| of small bins
// amplifies operand rounding), scaled per brick (1/max|V| for the forward, n^3 / (8 max|gE|) for
// Gamma') and unscaled in FP32.  Every wait on the tensor cores is bounded.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "spectra_f32_common.cuh"
#include "tc_sm100.cuh"

namespace sal {
namespace {

using f32::fast_rsqrt;
using f32::Tw;

constexpr int kThreads = 512;             // 16 warps: 4 per TMEM lane quarter
constexpr int kGroups = kThreads / 128;   // warp groups sharing a lane quarter
constexpr int kBY = 16;
constexpr int kKRows = kBY + 15;
constexpr uint32_t kTmemCols = 512;       // [0,256) forward F of 8 outputs; [256,320) inverse re/im
constexpr uint32_t kInvCol = 256;
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr float kKinkTau = 1.0f / 524288.0f;  // zero-subgradient band of |F| (2^-19 of the window L1 norm)
constexpr int kZStride = 33;              // float2 stride of a row of Gamma_G2 / z (bank spread)

template <int N> struct BtGeo {
    static constexpr int H = N / 2 + 1;
    static constexpr int P = 128 / N;
    static constexpr int XH = P + N - 1;
    static constexpr int YH = kBY + N - 1;
    static constexpr uint32_t SBO_A = kKRows * 16;
    static constexpr size_t IN_B = (size_t)N * XH * YH * 4;
    static constexpr size_t G1_B = (size_t)XH * YH * 8;
    static constexpr size_t A_B = (size_t)16 * SBO_A;
    static constexpr size_t BINV_B = (size_t)kBY * 1024;
    static constexpr size_t WT_B = (size_t)H * N * H * 3 * 4;
    static constexpr size_t GAM_B0 = (size_t)4 * 2 * 4096;                 // 4 outputs x re/im x 128x16 operand
    static constexpr size_t Z_B = (size_t)128 * kZStride * 8;               // Gamma_G2 / z rows
    static constexpr size_t GAM_B = GAM_B0 > Z_B ? GAM_B0 : Z_B;
    static constexpr size_t OFF_G1 = IN_B;
    static constexpr size_t OFF_A = (OFF_G1 + G1_B + 127) / 128 * 128;
    static constexpr size_t OFF_B = OFF_A + 2 * A_B;
    static constexpr size_t OFF_BINV = OFF_B + 512;
    static constexpr size_t OFF_WT = OFF_BINV + BINV_B;
    static constexpr size_t OFF_GAM = (OFF_WT + WT_B + 127) / 128 * 128;
    static constexpr size_t OFF_GV = OFF_GAM + GAM_B;
    static constexpr size_t OFF_GE = OFF_GV + IN_B;
    static constexpr size_t OFF_L1 = OFF_GE + (size_t)3 * P * kBY * 4;
    static constexpr size_t OFF_MISC = OFF_L1 + (size_t)P * kBY * 4;
    static constexpr size_t SMEM_USED = OFF_MISC + 64 + 2 * (kThreads / 32) * 4;
    static_assert(4 % kGroups == 0, "operand slots per warp group");
    // one CTA per SM: it holds all 512 tensor-memory columns
    static constexpr size_t SMEM = SMEM_USED > (size_t)120 * 1024 ? SMEM_USED : (size_t)120 * 1024;
    static constexpr int BLOCK_FLOATS = N * XH * YH;
    static_assert(SMEM <= 227 * 1024, "shared memory");
    static_assert(2 * H - 2 <= 16 && YH <= 31, "operand shapes");
};

template <int FMT> struct Pack;
template <> struct Pack<1> {
    __device__ static uint32_t two(float a, float b) {
        __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&v);
    }
    __device__ static uint16_t one(float a) {
        __nv_bfloat16 v = __float2bfloat16_rn(a);
        return *reinterpret_cast<uint16_t*>(&v);
    }
};
template <> struct Pack<0> {
    __device__ static uint32_t two(float a, float b) {
        __half2 v = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&v);
    }
    __device__ static uint16_t one(float a) {
        __half v = __float2half_rn(a);
        return *reinterpret_cast<uint16_t*>(&v);
    }
};

// Twiddle row j of the paired inverse/forward tables: cos of k = j (j < H), sin of k = j - H + 1.
template <int N>
__device__ __forceinline__ float pair_twiddle(const Tw<N>& tw, int j, int u) {
    constexpr int H = N / 2 + 1;
    if (u < 0 || u >= N) return 0.f;
    if (j < H) return tw.c[j][u];
    if (j < 2 * H - 2) return tw.s[j - H + 1][u];
    return 0.f;
}

template <int N, int FMT>
__global__ void __launch_bounds__(kThreads, 1)
k5_spectra_adjoint_tc(const float* __restrict__ V, const float* __restrict__ gE, float* __restrict__ blocks,
                      int T, int X, int Y, int bnd, int t_begin, const __grid_constant__ Tw<N> tw,
                      int* __restrict__ err) {
    using G = BtGeo<N>;
    constexpr int H = G::H, P = G::P, XH = G::XH, YH = G::YH;
    extern __shared__ __align__(128) unsigned char smem[];
    float* s_in = reinterpret_cast<float*>(smem);
    float2* s_g1 = reinterpret_cast<float2*>(smem + G::OFF_G1);
    float* s_col = reinterpret_cast<float*>(smem + G::OFF_G1);          // L1 column sums (set-up only)
    unsigned char* s_are = smem + G::OFF_A;
    unsigned char* s_aim = smem + G::OFF_A + G::A_B;
    unsigned char* s_b = smem + G::OFF_B;
    unsigned char* s_binv = smem + G::OFF_BINV;
    float* s_wt = reinterpret_cast<float*>(smem + G::OFF_WT);
    unsigned char* s_gam = smem + G::OFF_GAM;                            // Gamma' operands
    float2* s_z = reinterpret_cast<float2*>(smem + G::OFF_GAM);          // Gamma_G2 / z (aliases)
    float* s_gv = reinterpret_cast<float*>(smem + G::OFF_GV);            // [N][XH][YH]
    float* s_ge = reinterpret_cast<float*>(smem + G::OFF_GE);            // [3][P][16]
    float* s_l1 = reinterpret_cast<float*>(smem + G::OFF_L1);            // [P][16]
    uint64_t* s_mbar = reinterpret_cast<uint64_t*>(smem + G::OFF_MISC);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + G::OFF_MISC + 8);
    int* s_fail = reinterpret_cast<int*>(smem + G::OFF_MISC + 16);
    float* s_red = reinterpret_cast<float*>(smem + G::OFF_MISC + 64);    // [2][warps]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int yb = blockIdx.x * kBY;
    const int xb = blockIdx.y * P;
    const int t0 = t_begin + blockIdx.z;
    const size_t NV = (size_t)T * X * Y;

    // ---- set-up -----------------------------------------------------------------------------------
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(s_tmem), kTmemCols);
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(s_mbar), 1);
        *s_fail = 0;
    }
    for (int i = tid; i < 256; i += kThreads) {
        const int n = i / 16, k = i % 16;
        *reinterpret_cast<uint16_t*>(s_b + (n / 8) * 256 + (k / 8) * 128 + (n % 8) * 16 + (k % 8) * 2) =
            Pack<FMT>::one(pair_twiddle<N>(tw, n, k));
    }
    for (int i = tid; i < kBY * 32 * 16; i += kThreads) {   // B_{y0}[y][j] = T[j][y - y0]
        const int j = i % 16, y = (i / 16) % 32, y0 = i / 512;
        *reinterpret_cast<uint16_t*>(s_binv + y0 * 1024 + (y / 8) * 256 + (j / 8) * 128 + (y % 8) * 16 + (j % 8) * 2) =
            Pack<FMT>::one(pair_twiddle<N>(tw, j, y - y0));
    }
    for (int i = tid; i < H * N * H; i += kThreads) {
        const int k = i % H, kx = (i / H) % N, kt = i / (H * N);
        const int ii = kt, j = kx < N / 2 ? kx : kx - N;
        const float mult = (kt == 0 || 2 * kt == N) ? 1.f : 2.f;
        const float r2 = (float)(ii * ii + j * j + k * k);
        float w0 = 0.f, w1 = 0.f, w2 = 0.f;
        if (r2 > 0.f) {
            const float inv = mult / (float)(N * N * N) / sqrtf(r2);
            w0 = sqrtf((float)(j * j + k * k)) * inv;
            w1 = sqrtf((float)(ii * ii + k * k)) * inv;
            w2 = sqrtf((float)(ii * ii + j * j)) * inv;
        }
        s_wt[i * 3 + 0] = w0;
        s_wt[i * 3 + 1] = w1;
        s_wt[i * 3 + 2] = w2;
    }
    for (int i = tid; i < (int)(2 * G::A_B / 16); i += kThreads)
        reinterpret_cast<uint4*>(s_are)[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = tid; i < N * XH * YH; i += kThreads) s_gv[i] = 0.f;
    float vmax = 0.f, gmax = 0.f;
    for (int r = tid; r < N * XH * YH; r += kThreads) {
        const int yy = r % YH, xx = (r / YH) % XH, ut = r / (YH * XH);
        const int gt = ext_index(t0 - N / 2 + ut, T, bnd);
        const int gx = ext_index(xb - N / 2 + xx, X, bnd);
        const int gy = ext_index(yb - N / 2 + yy, Y, bnd);
        float v = 0.f;
        if ((gt | gx | gy) >= 0) v = __ldg(V + ((size_t)gt * X + gx) * Y + gy);
        s_in[r] = v;
        vmax = fmaxf(vmax, fabsf(v));
    }
    for (int i = tid; i < 3 * P * kBY; i += kThreads) {
        const int y0 = i % kBY, xl = (i / kBY) % P, m = i / (kBY * P);
        const int x = xb + xl, y = yb + y0;
        const float g = (x < X && y < Y) ? __ldg(gE + m * NV + ((size_t)t0 * X + x) * Y + y) : 0.f;
        s_ge[i] = g;
        gmax = fmaxf(gmax, fabsf(g));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
    }
    if (lane == 0) {
        s_red[warp] = vmax;
        s_red[kThreads / 32 + warp] = gmax;
    }
    __syncthreads();
    // window L1 norms (the kink band of |F|): column sums over t, then a box over x and y
    for (int it = tid; it < XH * YH; it += kThreads) {
        float a = 0.f;
#pragma unroll
        for (int u = 0; u < N; ++u) a = fmaf(tw.c[0][u], fabsf(s_in[u * XH * YH + it]), a);
        s_col[it] = a;
    }
    __syncthreads();
    for (int i = tid; i < P * kBY; i += kThreads) {
        const int y0 = i % kBY, xl = i / kBY;
        float a = 0.f;
        for (int ux = 0; ux < N; ++ux)
#pragma unroll
            for (int uy = 0; uy < N; ++uy) a = fmaf(tw.c[0][ux] * tw.c[0][uy], s_col[(xl + ux) * YH + y0 + uy], a);
        s_l1[i] = a;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *s_tmem;
    float bmax = 0.f, bgmax = 0.f;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) {
        bmax = fmaxf(bmax, s_red[w]);
        bgmax = fmaxf(bgmax, s_red[kThreads / 32 + w]);
    }
    const float inv_scale = 1.f / (bmax > 0.f ? bmax : 1.f);
    const float sigma = bgmax > 0.f ? (float)(N * N * N) / (8.f * bgmax) : 1.f;  // Gamma' operand scale

    const int q = warp & 3, grp = warp >> 2;   // lane quarter, warp group
    const int m = 32 * q + lane;                 // TMEM lane = stage-3 row (x0l, k_x)
    const int x0l = m / N, kx = m % N;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    const uint32_t idesc_f = tc::idesc_f16(FMT, 128, 16, 1, 0);
    const uint32_t idesc_i = tc::idesc_f16(FMT, 128, 32, 0, 0);
    const uint64_t bdesc = tc::desc_noswizzle(tc::smem_u32(s_b), 128, 256);
    const uint32_t are = tc::smem_u32(s_are), aim = tc::smem_u32(s_aim);
    const uint32_t gam = tc::smem_u32(s_gam), binv = tc::smem_u32(s_binv);
    uint32_t phase = 0;

    // CTA-uniform bounded wait on the MMA barrier; false once the CTA has given up
    auto wait_mma = [&]() -> bool {
        const int failed_before = *s_fail;
        const bool ok = failed_before ? false : tc::mbar_wait(tc::smem_u32(s_mbar), phase, kWaitLimit);
        const int bad = __syncthreads_or(!ok);
        if (bad && tid == 0 && !failed_before) {
            atomicOr(err, 1);
            *s_fail = 1;
        }
        phase ^= 1u;
        tc::fence_after_sync();
        return !bad;
    };

    for (int kt = 0; kt < H; ++kt) {
        float cr[N], sr[N];
#pragma unroll
        for (int u = 0; u < N; ++u) {
            cr[u] = tw.c[kt][u];
            sr[u] = tw.s[kt][u];
        }
        // ---- stages 1 and 2 (forward recompute) ---------------------------------------------------
        for (int it = tid; it < XH * YH; it += kThreads) {
            float Pv = 0.f, Qv = 0.f;
#pragma unroll
            for (int u = 0; u < N; ++u) {
                const float v = s_in[u * XH * YH + it];
                Pv = fmaf(v, cr[u], Pv);
                Qv = fmaf(v, sr[u], Qv);
            }
            s_g1[it] = make_float2(Pv, -Qv);
        }
        __syncthreads();
        for (int it = tid; it < P * YH; it += kThreads) {
            const int xl = it / YH, y = it % YH;
            float2 g[N];
#pragma unroll
            for (int u = 0; u < N; ++u) g[u] = s_g1[(xl + u) * YH + y];
            float fr[N], fi[N];
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
                fr[k] = (pr + qi) * inv_scale;
                fi[k] = (pi - qr) * inv_scale;
                if (k != 0 && 2 * k != N) {
                    fr[N - k] = (pr - qi) * inv_scale;
                    fi[N - k] = (pi + qr) * inv_scale;
                }
            }
#pragma unroll
            for (int c = 0; c < N / 8; ++c) {
                const size_t off = (size_t)(xl * (N / 8) + c) * G::SBO_A + (size_t)y * 16;
                uint4 vr, vi;
                vr.x = Pack<FMT>::two(fr[8 * c + 0], fr[8 * c + 1]);
                vr.y = Pack<FMT>::two(fr[8 * c + 2], fr[8 * c + 3]);
                vr.z = Pack<FMT>::two(fr[8 * c + 4], fr[8 * c + 5]);
                vr.w = Pack<FMT>::two(fr[8 * c + 6], fr[8 * c + 7]);
                vi.x = Pack<FMT>::two(fi[8 * c + 0], fi[8 * c + 1]);
                vi.y = Pack<FMT>::two(fi[8 * c + 2], fi[8 * c + 3]);
                vi.z = Pack<FMT>::two(fi[8 * c + 4], fi[8 * c + 5]);
                vi.w = Pack<FMT>::two(fi[8 * c + 6], fi[8 * c + 7]);
                *reinterpret_cast<uint4*>(s_are + off) = vr;
                *reinterpret_cast<uint4*>(s_aim + off) = vi;
            }
        }
        tc::fence_async_smem();
        __syncthreads();
        float wt[3][H];
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const float* w = s_wt + ((kt * N + kx) * H + k) * 3;
            wt[0][k] = w[0];
            wt[1][k] = w[1];
            wt[2][k] = w[2];
        }
        // ---- forward stage 3, Gamma, inverse stage 3 on the tensor cores ---------------------------
        for (int pass = 0; pass < 2; ++pass) {
            if (tid == 0 && !*s_fail) {
                tc::fence_after_sync();
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint32_t y0 = pass * 8 + j;
                    tc::mma_f16(tmem + j * 32, tc::desc_noswizzle(are + y0 * 16, 128, G::SBO_A), bdesc, idesc_f, 0);
                    tc::mma_f16(tmem + j * 32 + 16, tc::desc_noswizzle(aim + y0 * 16, 128, G::SBO_A), bdesc, idesc_f,
                                0);
                }
                tc::mma_commit(tc::smem_u32(s_mbar));
            }
            bool ok = wait_mma();
            for (int batch = 0; batch < 2; ++batch) {
                if (ok) {
#pragma unroll
                    for (int jj = 0; jj < 4 / kGroups; ++jj) {
                        const int slot = grp * (4 / kGroups) + jj;  // operand slot in this batch
                        const int j = batch * 4 + slot;            // TMEM output slot of this pass
                        const int y0 = pass * 8 + j;
                        float v[32];
                        tc::tmem_ld32(tmem + lane_base + (uint32_t)(j * 32), v);
                        const int gi = x0l * kBY + y0;
                        const float g0 = s_ge[gi], g1 = s_ge[P * kBY + gi], g2 = s_ge[2 * P * kBY + gi];
                        const float thr = kKinkTau * s_l1[gi] * inv_scale;
                        const float thr2 = fmaxf(thr * thr, 1e-30f);
                        float gr[16], gim[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) gr[i] = gim[i] = 0.f;
#pragma unroll
                        for (int k = 0; k < H; ++k) {
                            const float rho = sigma * fmaf(g0, wt[0][k], fmaf(g1, wt[1][k], g2 * wt[2][k]));
                            const float pr = v[k], pi = v[16 + k];
                            if (k == 0 || 2 * k == N) {
                                const float m2 = fmaf(pr, pr, pi * pi);
                                const float sc = m2 > thr2 ? rho * fast_rsqrt(m2) : 0.f;
                                gr[k] = sc * pr;
                                gim[k] = sc * pi;
                            } else {
                                const float qr = v[H + k - 1], qi = v[16 + H + k - 1];
                                const float ar = pr + qi, ai = pi - qr, br = pr - qi, bi = pi + qr;
                                const float m2a = fmaf(ar, ar, ai * ai), m2b = fmaf(br, br, bi * bi);
                                const float sa = m2a > thr2 ? rho * fast_rsqrt(m2a) : 0.f;
                                const float sb = m2b > thr2 ? rho * fast_rsqrt(m2b) : 0.f;
                                const float gar = sa * ar, gai = sa * ai, gbr = sb * br, gbi = sb * bi;
                                gr[k] = gar + gbr;                 // A_k
                                gim[k] = gai + gbi;
                                gr[H + k - 1] = gbi - gai;         // B_k = i (Gamma_a - Gamma_b)
                                gim[H + k - 1] = gar - gbr;
                            }
                        }
                        // K-major operand rows: (m/8)*256 + (j/8)*128 + (m%8)*16 + (j%8)*2
                        unsigned char* pre = s_gam + slot * 8192 + (m / 8) * 256 + (m % 8) * 16;
                        unsigned char* pim = pre + 4096;
#pragma unroll
                        for (int c = 0; c < 2; ++c) {
                            uint4 wr, wi;
                            wr.x = Pack<FMT>::two(gr[8 * c + 0], gr[8 * c + 1]);
                            wr.y = Pack<FMT>::two(gr[8 * c + 2], gr[8 * c + 3]);
                            wr.z = Pack<FMT>::two(gr[8 * c + 4], gr[8 * c + 5]);
                            wr.w = Pack<FMT>::two(gr[8 * c + 6], gr[8 * c + 7]);
                            wi.x = Pack<FMT>::two(gim[8 * c + 0], gim[8 * c + 1]);
                            wi.y = Pack<FMT>::two(gim[8 * c + 2], gim[8 * c + 3]);
                            wi.z = Pack<FMT>::two(gim[8 * c + 4], gim[8 * c + 5]);
                            wi.w = Pack<FMT>::two(gim[8 * c + 6], gim[8 * c + 7]);
                            *reinterpret_cast<uint4*>(pre + c * 128) = wr;
                            *reinterpret_cast<uint4*>(pim + c * 128) = wi;
                        }
                    }
                }
                tc::fence_async_smem();
                tc::fence_before_sync();
                __syncthreads();
                if (tid == 0 && !*s_fail) {
                    tc::fence_after_sync();
#pragma unroll
                    for (int slot = 0; slot < 4; ++slot) {
                        const uint32_t y0 = pass * 8 + batch * 4 + slot;
                        const uint64_t bd = tc::desc_noswizzle(binv + y0 * 1024, 128, 256);
                        tc::mma_f16(tmem + kInvCol, tc::desc_noswizzle(gam + slot * 8192, 128, 256), bd, idesc_i,
                                    y0 > 0 ? 1u : 0u);
                        tc::mma_f16(tmem + kInvCol + 32, tc::desc_noswizzle(gam + slot * 8192 + 4096, 128, 256), bd,
                                    idesc_i, y0 > 0 ? 1u : 0u);
                    }
                    tc::mma_commit(tc::smem_u32(s_mbar));
                }
                ok = wait_mma() && ok;
            }
            tc::fence_before_sync();
            __syncthreads();
        }
        // ---- Gamma_G2[row][y] from the accumulator (unscaled) ----------------------------------------
        if (grp == 0 && !*s_fail) {
            float vr[32], vi[32];
            tc::tmem_ld32(tmem + lane_base + kInvCol, vr);
            tc::tmem_ld32(tmem + lane_base + kInvCol + 32, vi);
            const float is = 1.f / sigma;
#pragma unroll
            for (int y = 0; y < YH; ++y) s_z[m * kZStride + y] = make_float2(vr[y] * is, vi[y] * is);
        }
        tc::fence_before_sync();
        __syncthreads();
        // ---- adjoint of stage 2 (x): z[x0l][u][y] in place ------------------------------------------
        for (int it = tid; it < P * YH; it += kThreads) {
            const int xl = it / YH, y = it % YH;
            float ar[H], ai[H], br[H], bi[H];
#pragma unroll
            for (int k = 0; k < H; ++k) {
                const float2 a = s_z[(xl * N + k) * kZStride + y];
                if (k == 0 || 2 * k == N) {
                    ar[k] = a.x; ai[k] = a.y; br[k] = bi[k] = 0.f;
                } else {
                    const float2 b = s_z[(xl * N + (N - k)) * kZStride + y];
                    ar[k] = a.x + b.x;
                    ai[k] = a.y + b.y;
                    br[k] = b.y - a.y;
                    bi[k] = a.x - b.x;
                }
            }
#pragma unroll
            for (int u = 0; u < N; ++u) {
                float zr = 0.f, zi = 0.f;
#pragma unroll
                for (int k = 0; k < H; ++k) {
                    zr = fmaf(ar[k], tw.c[k][u], zr);
                    zi = fmaf(ai[k], tw.c[k][u], zi);
                    if (k != 0 && 2 * k != N) {
                        zr = fmaf(br[k], tw.s[k][u], zr);
                        zi = fmaf(bi[k], tw.s[k][u], zi);
                    }
                }
                s_z[(xl * N + u) * kZStride + y] = make_float2(zr, zi);
            }
        }
        __syncthreads();
        // ---- overlap over x0 and adjoint of stage 1 (t), accumulated over k_t -------------------------
        for (int it = tid; it < XH * YH; it += kThreads) {
            const int x = it / YH, y = it % YH;
            float gr = 0.f, gi = 0.f;
            const int xa = x - N + 1 > 0 ? x - N + 1 : 0, xe = x < P - 1 ? x : P - 1;
            for (int xl = xa; xl <= xe; ++xl) {
                const float2 z = s_z[(xl * N + (x - xl)) * kZStride + y];
                gr += z.x;
                gi += z.y;
            }
#pragma unroll
            for (int u = 0; u < N; ++u) {
                float* o = s_gv + (u * XH + x) * YH + y;
                *o = fmaf(gr, cr[u], fmaf(-gi, sr[u], *o));
            }
        }
        __syncthreads();
    }

    // ---- the brick's block of gVext to scratch ---------------------------------------------------------
    const size_t cta = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    float* blk = blocks + cta * G::BLOCK_FLOATS;
    const bool good = *s_fail == 0;
    for (int i = tid; i < G::BLOCK_FLOATS; i += kThreads) blk[i] = good ? s_gv[i] : 0.f;
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

template <int N, int FMT>
cudaError_t prepare_nf() {
    return cudaFuncSetAttribute(k5_spectra_adjoint_tc<N, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)BtGeo<N>::SMEM);
}

template <int N, int FMT>
cudaError_t launch_nf(const TwiddleTable& t, const float* V, const float* gE, float* blocks, int T, int X, int Y,
                      int bnd, int t_begin, int t_count, int* err, cudaStream_t s) {
    using G = BtGeo<N>;
    dim3 grid((Y + kBY - 1) / kBY, (X + G::P - 1) / G::P, t_count);
    k5_spectra_adjoint_tc<N, FMT><<<grid, kThreads, G::SMEM, s>>>(V, gE, blocks, T, X, Y, bnd, t_begin,
                                                                   f32::make_tw<N>(t), err);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t spectra_adjoint_tc_prepare(int n, int fmt) {
    if (fmt != 0) return cudaErrorInvalidValue;  // built with FP16 operands only
    if (n == 8) return prepare_nf<8, 0>();
    if (n == 16) return prepare_nf<16, 0>();
    return cudaErrorInvalidValue;
}

SpectraAdjointGeometry spectra_adjoint_tc_geometry(int n) {
    if (n == 8) return {kBY, BtGeo<8>::YH, BtGeo<8>::P, BtGeo<8>::XH, BtGeo<8>::BLOCK_FLOATS};
    if (n == 16) return {kBY, BtGeo<16>::YH, BtGeo<16>::P, BtGeo<16>::XH, BtGeo<16>::BLOCK_FLOATS};
    return {0, 0, 0, 0, 0};
}

cudaError_t spectra_adjoint_tc_launch(int n, int fmt, const TwiddleTable& tw, const float* V, const float* gE,
                                      float* blocks, int T, int X, int Y, int bnd, int t_begin, int t_count, int* err,
                                      cudaStream_t s) {
    if (fmt != 0) return cudaErrorInvalidValue;
    if (n == 8) return launch_nf<8, 0>(tw, V, gE, blocks, T, X, Y, bnd, t_begin, t_count, err, s);
    if (n == 16) return launch_nf<16, 0>(tw, V, gE, blocks, T, X, Y, bnd, t_begin, t_count, err, s);
    return cudaErrorInvalidValue;
}

}  // namespace sal
