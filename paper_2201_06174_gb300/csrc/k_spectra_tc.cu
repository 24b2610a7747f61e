// K1-TC: local 3D DFT + projection + feature (Sec. 2 steps 1-3; Eq. 2, Eq. 1) with the dominant
// contraction -- stage 3, the DFT along y of every (k_t, k_x) row -- on the 5th-generation tensor
// cores (tcgen05.mma, kind::f16, BF16 or FP16 operands, FP32 accumulation in tensor memory).
//
// CTA brick: t0, x0 in [xb, xb + P) with P = 128/n, y0 in [yb, yb + 16).
// For each k_t tile (k_t = 0 .. n/2):
//   stage 1 (SIMT, FP32):  G1[x][y]     = sum_u h(u) exp(-2 pi i k_t u / n) V[t0-n/2+u][x][y]
//   stage 2 (SIMT, FP32):  G2[x0][k_x][y] = sum_u h(u) exp(-2 pi i k_x u / n) G1[x0-n/2+u][y]
//            rounded (after a per-brick scale 1/max|V|) to BF16/FP16 into the A operand:
//            row m = (x0 - xb) * n + k_x (128 rows), K = y, MN-major, no swizzle, 16-byte K rows
//   stage 3 (tensor cores): per output y0, D = A[:, y0 .. y0+15] x B, B = [cos | sin] twiddles
//            (pairing k_y with n-k_y: P = sum g cos, Q = sum g sin, F = P -+ iQ); the window of y0
//            is the same descriptor moved by 16*y0 bytes.  Real and imaginary parts of A are two
//            MMAs of N = 16 columns into tensor memory.
//   epilogue (tcgen05.ld): |F| for every bin, weighted by r_m of Eq. 1 (table in shared memory),
//            summed over k_y in registers, over k_t across tiles, over k_x by warp shuffles.
// Every wait on the tensor cores is bounded; on timeout the CTA sets the error word and leaves
// after releasing its tensor memory.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "spectra_f32_common.cuh"
#include "tc_sm100.cuh"

namespace sal {
namespace {

using f32::fast_sqrt;
using f32::Tw;

constexpr int kThreads = 256;
constexpr int kBY = 16;                 // outputs per CTA along y
constexpr int kKRows = kBY + 15;        // K rows of the A operand: window start + 16 taps
constexpr uint32_t kTmemCols = 256;     // 8 outputs x (16 + 16) FP32 columns
constexpr uint32_t kWaitLimit = 1u << 22;

template <int N> struct TcGeo {
    static constexpr int H = N / 2 + 1;
    static constexpr int P = 128 / N;          // x0 positions per CTA
    static constexpr int XH = P + N - 1;       // x extent of the halo
    static constexpr int YH = kBY + N - 1;     // y extent of the halo
    static constexpr uint32_t SBO_A = kKRows * 16;           // bytes between 8-row groups of A
    static constexpr size_t IN_B = (size_t)N * XH * YH * 4;
    static constexpr size_t G1_B = (size_t)XH * YH * 8;
    static constexpr size_t A_B = (size_t)16 * SBO_A;        // one of A_re / A_im
    static constexpr size_t B_B = 512;
    static constexpr size_t WT_B = (size_t)H * N * H * 3 * 4;
    static constexpr size_t OFF_G1 = IN_B;
    static constexpr size_t OFF_A = (OFF_G1 + G1_B + 127) / 128 * 128;
    static constexpr size_t OFF_B = OFF_A + 2 * A_B;
    static constexpr size_t OFF_WT = OFF_B + B_B;
    static constexpr size_t OFF_MISC = OFF_WT + WT_B;
    static constexpr size_t SMEM_USED = OFF_MISC + 64 + kThreads / 32 * 4;
    // at most two CTAs per SM: two x 256 tensor-memory columns fill the 512 of an SM
    static constexpr size_t SMEM = SMEM_USED > (size_t)80 * 1024 ? SMEM_USED : (size_t)80 * 1024;
    static_assert(2 * H - 2 <= 16, "B columns");
    static_assert(YH <= kKRows, "window rows");
};

template <int FMT> struct Pack;
template <> struct Pack<1> {  // BF16
    __device__ static uint32_t two(float a, float b) {
        __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&v);
    }
    __device__ static uint16_t one(float a) {
        __nv_bfloat16 v = __float2bfloat16_rn(a);
        return *reinterpret_cast<uint16_t*>(&v);
    }
};
template <> struct Pack<0> {  // FP16
    __device__ static uint32_t two(float a, float b) {
        __half2 v = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&v);
    }
    __device__ static uint16_t one(float a) {
        __half v = __float2half_rn(a);
        return *reinterpret_cast<uint16_t*>(&v);
    }
};

template <int N, int FMT>
__global__ void __launch_bounds__(kThreads, 2)
k1_spectra_tc(const float* __restrict__ V, float* __restrict__ E, int T, int X, int Y, int bnd,
              const __grid_constant__ Tw<N> tw, int* __restrict__ err) {
    using G = TcGeo<N>;
    constexpr int H = G::H, P = G::P, XH = G::XH, YH = G::YH;
    extern __shared__ __align__(128) unsigned char smem[];
    float* s_in = reinterpret_cast<float*>(smem);                       // [N][XH][YH]
    float2* s_g1 = reinterpret_cast<float2*>(smem + G::OFF_G1);         // [XH][YH]
    unsigned char* s_are = smem + G::OFF_A;                             // A real part
    unsigned char* s_aim = smem + G::OFF_A + G::A_B;                    // A imaginary part
    unsigned char* s_b = smem + G::OFF_B;                               // B [16 x 16], K-major
    float* s_wt = reinterpret_cast<float*>(smem + G::OFF_WT);           // [k_t][k_x][k][3]
    uint64_t* s_mbar = reinterpret_cast<uint64_t*>(smem + G::OFF_MISC);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + G::OFF_MISC + 8);
    int* s_fail = reinterpret_cast<int*>(smem + G::OFF_MISC + 16);
    float* s_red = reinterpret_cast<float*>(smem + G::OFF_MISC + 64);   // [warps]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int yb = blockIdx.x * kBY;
    const int xb = blockIdx.y * P;
    const int t0 = blockIdx.z;

    // ---- set-up: tensor memory, mbarrier, B operand, weight table, halo brick ------------------
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(s_tmem), kTmemCols);
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(s_mbar), 1);
        *s_fail = 0;
    }
    for (int i = tid; i < 256; i += kThreads) {
        const int n = i / 16, k = i % 16;
        float v = 0.f;
        if (k < N) {
            if (n < H) v = tw.c[n][k];
            else if (n < 2 * H - 2) v = tw.s[n - H + 1][k];
        }
        *reinterpret_cast<uint16_t*>(s_b + (n / 8) * 256 + (k / 8) * 128 + (n % 8) * 16 + (k % 8) * 2) =
            Pack<FMT>::one(v);
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
    // A rows beyond the halo (read by the last windows, multiplied by zero twiddles) stay zero
    for (int i = tid; i < (int)(2 * G::A_B / 16); i += kThreads)
        reinterpret_cast<uint4*>(s_are)[i] = make_uint4(0u, 0u, 0u, 0u);
    float vmax = 0.f;
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
    const float scale = bmax > 0.f ? bmax : 1.f;     // per-brick scale of the low-precision operand
    const float inv_scale = 1.f / scale;

    // epilogue mapping: TMEM lane quarter q, row m = 32 q + lane, output slots of this warp
    const int q = warp & 3, half = warp >> 2;
    const int m = 32 * q + lane;
    const int x0l = m / N, kx = m % N;
    float acc[8][3];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i][0] = acc[i][1] = acc[i][2] = 0.f;

    const uint32_t idesc = tc::idesc_f16(FMT, 128, 16, 1, 0);
    const uint64_t bdesc = tc::desc_noswizzle(tc::smem_u32(s_b), 128, 256);
    const uint32_t are = tc::smem_u32(s_are), aim = tc::smem_u32(s_aim);
    uint32_t phase = 0;

    for (int kt = 0; kt < H; ++kt) {
        // ---- stage 1 for this k_t ------------------------------------------------------------
        {
            float cr[N], sr[N];
#pragma unroll
            for (int u = 0; u < N; ++u) {
                cr[u] = tw.c[kt][u];
                sr[u] = tw.s[kt][u];
            }
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
        }
        __syncthreads();
        // ---- stage 2 -> A operand (low precision) --------------------------------------------
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
        // this lane's projection weights for (k_t, k_x), |k_y| = 0 .. n/2
        float wt[3][H];
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const float* w = s_wt + ((kt * N + kx) * H + k) * 3;
            wt[0][k] = w[0];
            wt[1][k] = w[1];
            wt[2][k] = w[2];
        }
        // ---- stage 3 on the tensor cores, two passes of 8 outputs --------------------------------
        for (int pass = 0; pass < 2; ++pass) {
            if (tid == 0 && !*s_fail) {
                tc::fence_after_sync();
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint32_t y0 = pass * 8 + j;
                    const uint64_t ar = tc::desc_noswizzle(are + y0 * 16, 128, G::SBO_A);
                    const uint64_t ai = tc::desc_noswizzle(aim + y0 * 16, 128, G::SBO_A);
                    tc::mma_f16(tmem + j * 32, ar, bdesc, idesc, 0);
                    tc::mma_f16(tmem + j * 32 + 16, ai, bdesc, idesc, 0);
                }
                tc::mma_commit(tc::smem_u32(s_mbar));
            }
            // the give-up decision is CTA-uniform: the TMEM loads below are warp-collective
            const int failed_before = *s_fail;  // written only before the previous barrier
            const bool ok = failed_before ? false : tc::mbar_wait(tc::smem_u32(s_mbar), phase, kWaitLimit);
            const int bad = __syncthreads_or(!ok);
            if (bad && tid == 0 && !failed_before) {
                atomicOr(err, 1);
                *s_fail = 1;  // read by every thread only after the barrier that ends this pass
            }
            phase ^= 1u;
            tc::fence_after_sync();
            if (!bad) {
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int j = half + 2 * jj;
                    float v[32];
                    tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(j * 32), v);
                    float e0 = 0.f, e1 = 0.f, e2 = 0.f;
#pragma unroll
                    for (int k = 0; k < H; ++k) {
                        const float pr = v[k], pi = v[16 + k];
                        float a;
                        if (k == 0 || 2 * k == N) {
                            a = fast_sqrt(fmaf(pr, pr, pi * pi));
                        } else {
                            const float qr = v[H + k - 1], qi = v[16 + H + k - 1];
                            const float ar = pr + qi, ai = pi - qr, br = pr - qi, bi = pi + qr;
                            a = fast_sqrt(fmaf(ar, ar, ai * ai)) + fast_sqrt(fmaf(br, br, bi * bi));
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

    // ---- sum over the n lanes of each x0 (k_x), write E -------------------------------------------
    const size_t NV = (size_t)T * X * Y;
    const int x = xb + x0l;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int y0 = (i / 4) * 8 + half + 2 * (i % 4);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float s = acc[i][c];
#pragma unroll
            for (int o = 1; o < N; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            const int y = yb + y0;
            if (kx == 0 && x < X && y < Y && !*s_fail) E[c * NV + ((size_t)t0 * X + x) * Y + y] = s * scale;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

template <int N, int FMT>
cudaError_t prepare_nf() {
    return cudaFuncSetAttribute(k1_spectra_tc<N, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)TcGeo<N>::SMEM);
}

template <int N, int FMT>
cudaError_t launch_nf(const TwiddleTable& t, const float* V, float* E, int T, int X, int Y, int bnd, int* err,
                      cudaStream_t s) {
    using G = TcGeo<N>;
    dim3 grid((Y + kBY - 1) / kBY, (X + G::P - 1) / G::P, T);
    k1_spectra_tc<N, FMT><<<grid, kThreads, G::SMEM, s>>>(V, E, T, X, Y, bnd, f32::make_tw<N>(t), err);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace

bool spectra_tc_supported(int n) { return n == 8 || n == 16; }

cudaError_t spectra_tc_prepare(int n, int fmt) {
    if (n == 8) return fmt == 1 ? prepare_nf<8, 1>() : prepare_nf<8, 0>();
    if (n == 16) return fmt == 1 ? prepare_nf<16, 1>() : prepare_nf<16, 0>();
    return cudaErrorInvalidValue;
}

cudaError_t spectra_tc_launch(int n, int fmt, const TwiddleTable& tw, const float* V, float* E, int T, int X, int Y,
                              int bnd, int* err, cudaStream_t s) {
    if (n == 8) return fmt == 1 ? launch_nf<8, 1>(tw, V, E, T, X, Y, bnd, err, s)
                                : launch_nf<8, 0>(tw, V, E, T, X, Y, bnd, err, s);
    if (n == 16) return fmt == 1 ? launch_nf<16, 1>(tw, V, E, T, X, Y, bnd, err, s)
                                 : launch_nf<16, 0>(tw, V, E, T, X, Y, bnd, err, s);
    return cudaErrorInvalidValue;
}

}  // namespace sal
