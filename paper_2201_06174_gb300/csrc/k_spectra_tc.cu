// K1-TC: local 3D DFT + projection + feature (Sec. 2 steps 1-3; Eq. 2, Eq. 1) with all three
// separable DFT stages on the 5th-generation tensor cores (tcgen05.mma, kind::f16, BF16 or FP16
// operands, FP32 accumulation in tensor memory).  Only the abs(F) / Eq. 1 epilogue runs on the SIMT
// pipes.
//
// CTA brick: t0, x0 in [xb, xb + P) with P = 128/n, y0 in [yb, yb + 16).  Positions of the halo are
// pos = x * YP + y (x < 24, y < YP = 8 ceil(YH / 8)).
//   stage 1 (t), once for all k_t:  D1[pos][c] = sum_u V[t0-n/2+u][x][y] T1[u][c],
//            c = [cos k_t = 0..n/2 | sin k_t = 1..n/2-1]; A = the brick scaled by 1/max|V| and
//            rounded to 16 bits (MN-major: 8 consecutive y per 16-byte row), one MMA per 128 positions.
//            D1 is read back once and scattered into one stage-2 B operand per k_t:
//            G1 = P - iQ  ->  B2[(re|im, y)][(cos|sin, x)] = [[G1r, G1i], [G1i, -G1r]].
//   stage 2 (x), per k_t:  D2[(x0, k_x)][(re|im, y)] = sum_x A2[(x0, k_x)][(cos|sin, x)] B2[..][..],
//            A2 = the Toeplitz twiddles h(x - x0) [cos | sin](2 pi k_x (x - x0) / n): the sliding
//            window along x is built into A2, so G2 = sum (c - i s)(G1r + i G1i) for all 16 k_x.
//            D2 is rounded to 16 bits into the stage-3 A operands (real, imaginary), MN-major with
//            16-byte K rows: the window of output y0 is the same descriptor moved by 16 y0 bytes.
//   stage 3 (y), per k_t and output y0:  D3[(x0, k_x)][(re|im, k_y)] = Are(y0) B3a + Aim(y0) B3b,
//            B3a = [c | -s], B3b = [s | c] over all k_y: the accumulator holds Re F and Im F.
//   epilogue (tcgen05.ld): abs(F) per bin, bins k_y and n - k_y summed (same Eq. 1 ratios), weighted
//            by r_m / |k| of Eq. 1, summed over k_y in registers, over k_t across tiles, over k_x by
//            warp shuffles; E = sum * max|V|.
// Every wait on the tensor cores is bounded; on timeout the CTA sets the error word and leaves after
// releasing its tensor memory.
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
constexpr int kKRows = kBY + 15;        // K rows of the stage-3 A operand: window start + 16 taps
constexpr int kXHP = 24;                // halo rows along x staged (>= P + n - 1, multiple of 8)
constexpr int kK2 = 2 * kXHP;           // stage-2 K: 24 cos taps + 24 sin taps
constexpr uint32_t kTmemCols = 256;     // two 128-column accumulator buffers
constexpr uint32_t kWaitLimit = 1u << 22;

template <int N> struct TcGeo {
    static constexpr int H = N / 2 + 1;
    static constexpr int P = 128 / N;          // x0 positions per CTA
    static constexpr int XH = P + N - 1;       // x extent of the halo
    static constexpr int YH = kBY + N - 1;     // y extent of the halo
    static constexpr int YG = (YH + 7) / 8;
    static constexpr int YP = 8 * YG;          // y positions per halo row
    static constexpr int NB1 = (kXHP * YP + 127) / 128;   // stage-1 MMAs (128 positions each)
    static constexpr int N2 = 2 * YP;          // stage-2 N: re | im over y
    static constexpr int N3 = 2 * N;           // stage-3 N per output: re | im over k_y
    static constexpr int OPC = 32 / N3;        // outputs per 32-column TMEM chunk (1 or 2)
    static constexpr int OPP = 128 / N3;       // outputs per pass (one 128-column buffer)
    static constexpr int PASSES = kBY / OPP;   // 4 (n = 16) or 2 (n = 8), alternating buffers
    static constexpr uint32_t SBO_A3 = kKRows * 16;
    static constexpr uint32_t SBO_K2 = kK2 / 8 * 128;    // 8-row group stride of the K-major A2 / B2
    static constexpr size_t A1_B = (size_t)NB1 * 4096;
    static constexpr size_t B2_B = (size_t)N2 / 8 * SBO_K2;   // one k_t tile
    static constexpr size_t B2ALL_B = (size_t)H * B2_B;
    static constexpr size_t R0_B = A1_B > B2ALL_B ? A1_B : B2ALL_B;   // A1 then the B2 tiles (aliased)
    // constant operands, built once per handle and bulk-copied into every CTA:
    // [A2 | B1 | B3a | B3b | Eq. 1 weight table]
    static constexpr size_t A2_B = (size_t)16 * SBO_K2;
    static constexpr size_t B3_B = (size_t)N3 / 8 * 256;
    static constexpr size_t WT_B = ((size_t)H * H * H * 3 * 4 + 15) / 16 * 16;
    static constexpr size_t TAB_B1 = A2_B;
    static constexpr size_t TAB_B3A = TAB_B1 + 512;
    static constexpr size_t TAB_B3B = TAB_B3A + B3_B;
    static constexpr size_t TAB_WT = TAB_B3B + B3_B;
    static constexpr size_t TAB_B = TAB_WT + WT_B;
    static constexpr size_t A3_B = (size_t)16 * SBO_A3;
    static constexpr size_t OFF_TAB = (R0_B + 127) / 128 * 128;
    static constexpr size_t OFF_A3 = OFF_TAB + TAB_B;
    static constexpr size_t OFF_MISC = OFF_A3 + 2 * A3_B;
    static constexpr size_t SMEM = OFF_MISC + 64 + kThreads / 32 * 4;
    static constexpr int STAGE_ITEMS = 16 * NB1 * 16;   // (u, 8-position group) items of the A1 fill
    static constexpr int STAGE_PER_THREAD = (STAGE_ITEMS + kThreads - 1) / kThreads;
    static_assert(XH <= kXHP && YH <= 32 && YP <= 32, "halo");
    static_assert(2 * H - 2 <= 16, "stage-1 columns");
    static_assert(NB1 * 16 <= (int)kTmemCols && N2 <= 128, "tensor memory");
    static_assert(PASSES * OPP == kBY && PASSES % 2 == 0 && PASSES * OPC * 2 == 8, "passes");
    static_assert(TAB_B % 16 == 0 && OFF_TAB % 16 == 0 && OFF_A3 % 16 == 0, "bulk copy alignment");
    static_assert(SMEM <= 113 * 1024, "two CTAs per SM");
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

// Twiddles of any bin k in [0, n): h(u) cos(2 pi k u / n) and h(u) sin(2 pi k u / n); 0 outside [0, n).
template <int N> __device__ __forceinline__ float twc(const Tw<N>& tw, int k, int u) {
    if (u < 0 || u >= N) return 0.f;
    return k <= N / 2 ? tw.c[k][u] : tw.c[N - k][u];
}
template <int N> __device__ __forceinline__ float tws(const Tw<N>& tw, int k, int u) {
    if (u < 0 || u >= N) return 0.f;
    return k <= N / 2 ? tw.s[k][u] : -tw.s[N - k][u];
}

// The constant operands of one (n, operand type): A2 (Toeplitz stage-2 twiddles, K-major), B1
// (stage-1 twiddles), B3a / B3b (stage-3 twiddles), the Eq. 1 weight table [k_t][|k_x|][|k_y|][3].
template <int N, int FMT>
__global__ void k1_tc_tables(const __grid_constant__ Tw<N> tw, unsigned char* __restrict__ out) {
    using G = TcGeo<N>;
    constexpr int H = G::H;
    unsigned char* a2 = out;
    unsigned char* b1 = out + G::TAB_B1;
    unsigned char* b3a = out + G::TAB_B3A;
    unsigned char* b3b = out + G::TAB_B3B;
    float* wt = reinterpret_cast<float*>(out + G::TAB_WT);
    const int tid = threadIdx.x;
    // B1[c][u]: c < H: cos k_t = c; H <= c < 2H-2: sin k_t = c-H+1.  byte = (c/8)256 + (u/8)128 + (c%8)16 + (u%8)2
    for (int i = tid; i < 256; i += blockDim.x) {
        const int c = i / 16, u = i % 16;
        float v = 0.f;
        if (c < H) v = twc<N>(tw, c, u);
        else if (c < 2 * H - 2) v = tws<N>(tw, c - H + 1, u);
        *reinterpret_cast<uint16_t*>(b1 + (c / 8) * 256 + (u / 8) * 128 + (c % 8) * 16 + (u % 8) * 2) =
            Pack<FMT>::one(v);
    }
    // B3a[ncol][u] = [c | -s], B3b[ncol][u] = [s | c] over k_y = ncol % n (K-major, K = u)
    for (int i = tid; i < G::N3 * 16; i += blockDim.x) {
        const int ncol = i / 16, u = i % 16, k = ncol % N;
        const bool re = ncol < N;
        const float c = twc<N>(tw, k, u), sn = tws<N>(tw, k, u);
        const size_t off = (ncol / 8) * 256 + (u / 8) * 128 + (ncol % 8) * 16 + (u % 8) * 2;
        *reinterpret_cast<uint16_t*>(b3a + off) = Pack<FMT>::one(re ? c : -sn);
        *reinterpret_cast<uint16_t*>(b3b + off) = Pack<FMT>::one(re ? sn : c);
    }
    // A2[(x0l, k_x)][k2]: k2 < 24: cos, else sin, of (k_x, x - x0l) with x = k2 % 24 (K-major)
    for (int i = tid; i < 128 * kK2; i += blockDim.x) {
        const int m = i / kK2, k2 = i % kK2;
        const int x0l = m / N, kx = m % N, x = k2 % kXHP, u = x - x0l;
        const float v = k2 < kXHP ? twc<N>(tw, kx, u) : tws<N>(tw, kx, u);
        *reinterpret_cast<uint16_t*>(a2 + (m / 8) * G::SBO_K2 + (k2 / 8) * 128 + (m % 8) * 16 + (k2 % 8) * 2) =
            Pack<FMT>::one(v);
    }
    // Eq. 1 weights r_m(k) / |k| (k_t multiplicity folded in) over (k_t, |k_x|, |k_y|)
    for (int i = tid; i < H * H * H; i += blockDim.x) {
        const int k = i % H, aj = (i / H) % H, kt = i / (H * H);
        const float mult = (kt == 0 || 2 * kt == N) ? 1.f : 2.f;
        const float r2 = (float)(kt * kt + aj * aj + k * k);
        float w0 = 0.f, w1 = 0.f, w2 = 0.f;
        if (r2 > 0.f) {
            const float inv = mult / (float)(N * N * N) / sqrtf(r2);
            w0 = sqrtf((float)(aj * aj + k * k)) * inv;
            w1 = sqrtf((float)(kt * kt + k * k)) * inv;
            w2 = sqrtf((float)(kt * kt + aj * aj)) * inv;
        }
        wt[i * 3 + 0] = w0;
        wt[i * 3 + 1] = w1;
        wt[i * 3 + 2] = w2;
    }
}

template <int N, int FMT>
__global__ void __launch_bounds__(kThreads, 2)
k1_spectra_tc(const float* __restrict__ V, float* __restrict__ E, int T, int X, int Y, int bnd,
              const unsigned char* __restrict__ tables, int* __restrict__ err) {
    using G = TcGeo<N>;
    constexpr int H = G::H, P = G::P, XH = G::XH, YH = G::YH, YG = G::YG, YP = G::YP;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* s_a1 = smem;                              // stage-1 A (MN-major), then:
    unsigned char* s_b2 = smem;                              // stage-2 B tiles, one per k_t (K-major)
    unsigned char* s_tab = smem + G::OFF_TAB;                // constant operands (bulk copy)
    unsigned char* s_are = smem + G::OFF_A3;                 // stage-3 A, real part (MN-major)
    unsigned char* s_aim = smem + G::OFF_A3 + G::A3_B;       // stage-3 A, imaginary part
    const float* s_wt = reinterpret_cast<const float*>(s_tab + G::TAB_WT);   // [k_t][|k_x|][|k_y|][3]
    // mbarriers: [0], [1] accumulator buffer full (MMA commit), [2] constant operands landed
    uint64_t* s_mbar = reinterpret_cast<uint64_t*>(smem + G::OFF_MISC);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + G::OFF_MISC + 48);
    int* s_fail = reinterpret_cast<int*>(smem + G::OFF_MISC + 52);
    float* s_red = reinterpret_cast<float*>(smem + G::OFF_MISC + 64);   // [warps]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int yb = blockIdx.x * kBY;
    const int xb = blockIdx.y * P;
    const int t0 = blockIdx.z;

    // ---- set-up: tensor memory, mbarriers, constant operands (bulk copy), stage-3 A zero rows --------
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(s_tmem), kTmemCols);
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(&s_mbar[0]), 1);
        tc::mbar_init(tc::smem_u32(&s_mbar[1]), 1);
        tc::mbar_init(tc::smem_u32(&s_mbar[2]), 1);
        *s_fail = 0;
        tc::mbar_arrive_expect_tx(tc::smem_u32(&s_mbar[2]), (uint32_t)G::TAB_B);
        tc::bulk_g2s(tc::smem_u32(s_tab), tables, (uint32_t)G::TAB_B, tc::smem_u32(&s_mbar[2]));
    }
    // stage-3 A rows beyond the halo (read by the last windows, multiplied by zero twiddles) stay zero
    for (int i = tid; i < (int)(2 * G::A3_B / 16); i += kThreads)
        reinterpret_cast<uint4*>(s_are)[i] = make_uint4(0u, 0u, 0u, 0u);

    // ---- the halo brick: registers -> max|V| -> 16-bit stage-1 A operand ---------------------------
    // item = (u, g): 8 positions pos = 8g .. 8g+7 (x = g / YG, y = 8 (g % YG) + i) at tap u
    const int ty = yb - N / 2;
    const bool interior = t0 - N / 2 >= 0 && t0 + N / 2 <= T && xb - N / 2 >= 0 && xb - N / 2 + XH <= X && ty >= 0 &&
                          ty + YP <= Y && (Y & 3) == 0 && (reinterpret_cast<uintptr_t>(V) & 15) == 0;
    float vals[G::STAGE_PER_THREAD][8];
    float vmax = 0.f;
#pragma unroll
    for (int r = 0; r < G::STAGE_PER_THREAD; ++r) {
        const int item = tid + r * kThreads;
        const int u = item / (G::NB1 * 16), g = item % (G::NB1 * 16);
        const int x = g / YG, y8 = 8 * (g % YG);
        const bool live = item < G::STAGE_ITEMS && u < N && x < XH;
#pragma unroll
        for (int i = 0; i < 8; ++i) vals[r][i] = 0.f;
        if (interior) {
            if (live) {
                const float* src = V + ((size_t)(t0 - N / 2 + u) * X + (xb - N / 2 + x)) * Y + ty + y8;
                const float4 a = __ldg(reinterpret_cast<const float4*>(src));
                const float4 b = __ldg(reinterpret_cast<const float4*>(src + 4));
                vals[r][0] = a.x; vals[r][1] = a.y; vals[r][2] = a.z; vals[r][3] = a.w;
                vals[r][4] = b.x; vals[r][5] = b.y; vals[r][6] = b.z; vals[r][7] = b.w;
            }
        } else {
            const int gt = ext_index(t0 - N / 2 + u, T, bnd);
            const int gx = ext_index(xb - N / 2 + x, X, bnd);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int gy = ext_index(ty + y8 + i, Y, bnd);
                if (live && y8 + i < YH && (gt | gx | gy) >= 0) vals[r][i] = __ldg(V + ((size_t)gt * X + gx) * Y + gy);
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (y8 + i >= YH) vals[r][i] = 0.f;     // positions past the halo (their outputs are not used)
            vmax = fmaxf(vmax, fabsf(vals[r][i]));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    if (lane == 0) s_red[warp] = vmax;
    __syncthreads();
    float bmax = 0.f;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) bmax = fmaxf(bmax, s_red[w]);
    const float scale = bmax > 0.f ? bmax : 1.f;     // per-brick scale of the low-precision operands
    const float inv_scale = 1.f / scale;
#pragma unroll
    for (int r = 0; r < G::STAGE_PER_THREAD; ++r) {
        const int item = tid + r * kThreads;
        if (item < G::STAGE_ITEMS) {
            const int u = item / (G::NB1 * 16), g = item % (G::NB1 * 16);
            uint4 w;
            w.x = Pack<FMT>::two(vals[r][0] * inv_scale, vals[r][1] * inv_scale);
            w.y = Pack<FMT>::two(vals[r][2] * inv_scale, vals[r][3] * inv_scale);
            w.z = Pack<FMT>::two(vals[r][4] * inv_scale, vals[r][5] * inv_scale);
            w.w = Pack<FMT>::two(vals[r][6] * inv_scale, vals[r][7] * inv_scale);
            // MN-major: byte(pos, u) = (pos/8) 256 + (u/8) 128 + (u%8) 16 + (pos%8) 2
            *reinterpret_cast<uint4*>(s_a1 + g * 256 + (u / 8) * 128 + (u % 8) * 16) = w;
        }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *s_tmem;

    // Every wait is CTA-uniform: thread 0 polls the mbarrier (bounded), the barrier that follows spreads
    // a give-up (after which no MMA is issued and no tensor memory is read) and, in the k_t loop, also
    // marks that every warp finished the previous pass.
    auto wait_cta = [&](int b, uint32_t parity) -> bool {
        const int failed_before = *s_fail;  // written only before an earlier barrier
        bool ok = true;
        if (tid == 0) ok = failed_before ? false : tc::mbar_wait(tc::smem_u32(&s_mbar[b]), parity, kWaitLimit);
        const int bad = __syncthreads_or(!ok || failed_before);
        if (bad && tid == 0 && !failed_before) {
            atomicOr(err, 1);
            *s_fail = 1;  // read by every thread only after a later barrier
        }
        tc::fence_after_sync();
        return !bad;
    };

    const int q = warp & 3, half = warp >> 2;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    const uint32_t idesc1 = tc::idesc_f16(FMT, 128, 16, 1, 0);
    const uint32_t idesc2 = tc::idesc_f16(FMT, 128, G::N2, 0, 0);
    const uint32_t idesc3 = tc::idesc_f16(FMT, 128, G::N3, 1, 0);
    const uint32_t tab = tc::smem_u32(s_tab), b2base = tc::smem_u32(s_b2);
    const uint32_t are = tc::smem_u32(s_are), aim = tc::smem_u32(s_aim);
    const uint64_t b3a = tc::desc_noswizzle(tab + (uint32_t)G::TAB_B3A, 128, 256);
    const uint64_t b3b = tc::desc_noswizzle(tab + (uint32_t)G::TAB_B3B, 128, 256);
    // stage 2 of tile kt into buffer 0 (columns [0, N2)); completion on full[0]
    auto issue_s2 = [&](int kt) {
        const uint32_t b2 = b2base + (uint32_t)(kt * G::B2_B);
#pragma unroll
        for (int s = 0; s < kK2 / 16; ++s)
            tc::mma_f16(tmem, tc::desc_noswizzle(tab + 256 * s, 128, G::SBO_K2),
                        tc::desc_noswizzle(b2 + 256 * s, 128, G::SBO_K2), idesc2, s > 0 ? 1u : 0u);
        tc::mma_commit(tc::smem_u32(&s_mbar[0]));
    };
    // stage 3 of one pass (OPP outputs) into buffer pass % 2; completion on full[pass % 2]
    auto issue_s3 = [&](int pass) {
        const uint32_t col = (uint32_t)(128 * (pass & 1));
#pragma unroll
        for (int j = 0; j < G::OPP; ++j) {
            const uint32_t y0 = pass * G::OPP + j;
            tc::mma_f16(tmem + col + j * G::N3, tc::desc_noswizzle(are + y0 * 16, 128, G::SBO_A3), b3a, idesc3, 0);
            tc::mma_f16(tmem + col + j * G::N3, tc::desc_noswizzle(aim + y0 * 16, 128, G::SBO_A3), b3b, idesc3, 1);
        }
        tc::mma_commit(tc::smem_u32(&s_mbar[pass & 1]));
    };
    // D2 (buffer 0) -> stage-3 A operands: warps of half 0 take the real columns, half 1 the imaginary
    auto convert_d2 = [&]() {
        float v[32];
        tc::tmem_ld32(tmem + lane_base + (uint32_t)(half * YP), v);
        const int m = 32 * q + lane;
        unsigned char* dst = (half ? s_aim : s_are) + (m / 8) * G::SBO_A3 + (m % 8) * 2;
#pragma unroll
        for (int y = 0; y < YH; ++y) *reinterpret_cast<uint16_t*>(dst + y * 16) = Pack<FMT>::one(v[y]);
        tc::fence_async_smem();
    };

    // ---- stage 1 on the tensor cores, all k_t at once (after the constant operands landed) ----------
    bool ok = wait_cta(2, 0);
    if (tid == 0 && ok) {
        const uint64_t b1 = tc::desc_noswizzle(tab + (uint32_t)G::TAB_B1, 128, 256);
#pragma unroll
        for (int i = 0; i < G::NB1; ++i)
            tc::mma_f16(tmem + 16 * i, tc::desc_noswizzle(tc::smem_u32(s_a1) + 4096 * i, 128, 256), b1, idesc1, 0);
        tc::mma_commit(tc::smem_u32(&s_mbar[0]));
    }
    ok = wait_cta(0, 0);
    uint32_t ph0 = 1, ph1 = 0;   // next phase parities of the two buffer barriers
    // D1 -> one stage-2 B tile per k_t (the A1 region is free once the stage-1 MMAs completed)
    if (ok) {
        for (int i = half; i < G::NB1; i += 2) {
            float v[32];
            tc::tmem_ld32(tmem + lane_base + (uint32_t)(16 * i), v);   // columns 16 i .. 16 i + 15 used
            const int pos = 128 * i + 32 * q + lane;
            const int x = pos / YP, y = pos % YP;
            if (x < kXHP) {
                // K-major: byte(ncol, k2) = (ncol/8) SBO_K2 + (k2/8) 128 + (ncol%8) 16 + (k2%8) 2
                const size_t o_re = (size_t)(y / 8) * G::SBO_K2 + (y % 8) * 16;
                const size_t o_im = (size_t)((YP + y) / 8) * G::SBO_K2 + ((YP + y) % 8) * 16;
                const size_t k_c = (size_t)(x / 8) * 128 + (x % 8) * 2;
                const size_t k_s = (size_t)((kXHP + x) / 8) * 128 + ((kXHP + x) % 8) * 2;
#pragma unroll
                for (int kt = 0; kt < H; ++kt) {
                    const float g1r = v[kt];
                    const float g1i = (kt == 0 || 2 * kt == N) ? 0.f : -v[H - 1 + kt];
                    unsigned char* b2 = s_b2 + (size_t)kt * G::B2_B;
                    *reinterpret_cast<uint16_t*>(b2 + o_re + k_c) = Pack<FMT>::one(g1r);
                    *reinterpret_cast<uint16_t*>(b2 + o_re + k_s) = Pack<FMT>::one(g1i);
                    *reinterpret_cast<uint16_t*>(b2 + o_im + k_c) = Pack<FMT>::one(g1i);
                    *reinterpret_cast<uint16_t*>(b2 + o_im + k_s) = Pack<FMT>::one(-g1r);
                }
            }
        }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && !*s_fail) {
        tc::fence_after_sync();
        issue_s2(0);
    }
    ok = wait_cta(0, ph0);
    ph0 ^= 1u;
    if (ok) convert_d2();
    tc::fence_before_sync();
    __syncthreads();

    // epilogue mapping: TMEM lane quarter q, row m = 32 q + lane
    const int m = 32 * q + lane;
    const int x0l = m / N, kx = m % N;
    const int ajx = kx <= N / 2 ? kx : N - kx;
    float acc[8][3];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i][0] = acc[i][1] = acc[i][2] = 0.f;

    // ---- the k_t loop: one CTA barrier per pass; the MMAs of a pass are issued one pass ahead --------
    for (int kt = 0; kt < H; ++kt) {
        if (tid == 0 && !*s_fail) {
            tc::fence_after_sync();
            issue_s3(0);
            issue_s3(1);
        }
        // this lane's Eq. 1 weights for (k_t, |k_x|), |k_y| = 0 .. n/2
        float wt[3][H];
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const float* w = s_wt + ((kt * H + ajx) * H + k) * 3;
            wt[0][k] = w[0];
            wt[1][k] = w[1];
            wt[2][k] = w[2];
        }
#pragma unroll
        for (int pass = 0; pass < G::PASSES; ++pass) {
            const int b = pass & 1;
            // pass complete in buffer b, and every warp done with the previous pass (buffer b ^ 1)
            const bool full = wait_cta(b, b ? ph1 : ph0);
            if (b) ph1 ^= 1u; else ph0 ^= 1u;
            if (tid == 0 && !*s_fail && pass >= 1) {
                if (pass + 1 < G::PASSES) issue_s3(pass + 1);
                else if (kt + 1 < H) issue_s2(kt + 1);       // buffer 0 free: stage 2 of the next tile
            }
            if (full) {
                // chunks half and half + 2 of this buffer, both loads in flight before the wait
                uint32_t r[2][32];
                tc::tmem_ld32_async(tmem + lane_base + (uint32_t)(128 * b + 32 * half), r[0]);
                tc::tmem_ld32_async(tmem + lane_base + (uint32_t)(128 * b + 32 * (half + 2)), r[1]);
                tc::tmem_wait_ld(r[0]);
                tc::tmem_wait_ld(r[1]);
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) {
#pragma unroll
                    for (int o = 0; o < G::OPC; ++o) {
                        float e0 = 0.f, e1 = 0.f, e2 = 0.f;
#pragma unroll
                        for (int k = 0; k < H; ++k) {
                            const float re = __uint_as_float(r[cc][o * G::N3 + k]);
                            const float im = __uint_as_float(r[cc][o * G::N3 + N + k]);
                            float sm = fast_sqrt(fmaf(re, re, im * im));
                            if (k != 0 && 2 * k != N) {
                                const float re2 = __uint_as_float(r[cc][o * G::N3 + N - k]);
                                const float im2 = __uint_as_float(r[cc][o * G::N3 + 2 * N - k]);
                                sm += fast_sqrt(fmaf(re2, re2, im2 * im2));
                            }
                            e0 = fmaf(wt[0][k], sm, e0);
                            e1 = fmaf(wt[1][k], sm, e1);
                            e2 = fmaf(wt[2][k], sm, e2);
                        }
                        const int slot = (pass * 2 + cc) * G::OPC + o;
                        acc[slot][0] += e0;
                        acc[slot][1] += e1;
                        acc[slot][2] += e2;
                    }
                }
            }
            tc::fence_before_sync();
        }
        if (kt + 1 < H) {
            // stage 2 of kt + 1 done (and with it every stage-3 MMA of kt): A3 may be rewritten
            ok = wait_cta(0, ph0);
            ph0 ^= 1u;
            if (ok) convert_d2();
            tc::fence_before_sync();
            __syncthreads();
        }
    }
    __syncthreads();

    // ---- sum over the n lanes of each x0 (k_x), write E -------------------------------------------
    const size_t NV = (size_t)T * X * Y;
    const int x = xb + x0l;
    const bool good = *s_fail == 0;
#pragma unroll
    for (int pass = 0; pass < G::PASSES; ++pass)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc)
#pragma unroll
            for (int o = 0; o < G::OPC; ++o) {
                const int slot = (pass * 2 + cc) * G::OPC + o;
                const int y0 = pass * G::OPP + (half + 2 * cc) * G::OPC + o;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float s = acc[slot][c];
#pragma unroll
                    for (int w = 1; w < N; w <<= 1) s += __shfl_xor_sync(0xffffffffu, s, w);
                    const int y = yb + y0;
                    if (kx == 0 && x < X && y < Y && good) E[c * NV + ((size_t)t0 * X + x) * Y + y] = s * scale;
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
cudaError_t tables_nf(const TwiddleTable& t, void* dst, cudaStream_t s) {
    k1_tc_tables<N, FMT><<<1, 256, 0, s>>>(f32::make_tw<N>(t), static_cast<unsigned char*>(dst));
    note_launches(1);
    return cudaGetLastError();
}

template <int N, int FMT>
cudaError_t launch_nf(const void* tables, const float* V, float* E, int T, int X, int Y, int bnd, int* err,
                      cudaStream_t s) {
    using G = TcGeo<N>;
    dim3 grid((Y + kBY - 1) / kBY, (X + G::P - 1) / G::P, T);
    k1_spectra_tc<N, FMT><<<grid, kThreads, G::SMEM, s>>>(V, E, T, X, Y, bnd,
                                                          static_cast<const unsigned char*>(tables), err);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace

bool spectra_tc_supported(int n) { return n == 8 || n == 16; }

size_t spectra_tc_tables_bytes(int n) {
    if (n == 8) return TcGeo<8>::TAB_B;
    if (n == 16) return TcGeo<16>::TAB_B;
    return 0;
}

cudaError_t spectra_tc_prepare(int n, int fmt) {
    if (n == 8) return fmt == 1 ? prepare_nf<8, 1>() : prepare_nf<8, 0>();
    if (n == 16) return fmt == 1 ? prepare_nf<16, 1>() : prepare_nf<16, 0>();
    return cudaErrorInvalidValue;
}

cudaError_t spectra_tc_tables_build(int n, int fmt, const TwiddleTable& tw, void* dst, cudaStream_t s) {
    if (n == 8) return fmt == 1 ? tables_nf<8, 1>(tw, dst, s) : tables_nf<8, 0>(tw, dst, s);
    if (n == 16) return fmt == 1 ? tables_nf<16, 1>(tw, dst, s) : tables_nf<16, 0>(tw, dst, s);
    return cudaErrorInvalidValue;
}

cudaError_t spectra_tc_launch(int n, int fmt, const void* tables, const float* V, float* E, int T, int X, int Y,
                              int bnd, int* err, cudaStream_t s) {
    if (n == 8) return fmt == 1 ? launch_nf<8, 1>(tables, V, E, T, X, Y, bnd, err, s)
                                : launch_nf<8, 0>(tables, V, E, T, X, Y, bnd, err, s);
    if (n == 16) return fmt == 1 ? launch_nf<16, 1>(tables, V, E, T, X, Y, bnd, err, s)
                                 : launch_nf<16, 0>(tables, V, E, T, X, Y, bnd, err, s);
    return cudaErrorInvalidValue;
}

}  // namespace sal
