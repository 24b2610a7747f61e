// K1-TC: local 3D DFT + projection + feature (Sec. 2 steps 1-3; Eq. 2, Eq. 1) with all three
// separable DFT stages on the 5th-generation tensor cores (tcgen05.mma, kind::f16, BF16 or FP16
// operands, FP32 accumulation in tensor memory); the stages are described in tc_spectra_common.cuh.
// Only the abs(F) / Eq. 1 epilogue runs on the SIMT pipes: abs(F) per bin, bins k_y and n - k_y summed
// (same Eq. 1 ratios), weighted by r_m / |k| of Eq. 1, summed over k_y in registers, over k_t across
// tiles, over k_x by warp shuffles; E = sum * max|V|.
// Warp-specialised: one producer warp issues every MMA; eight consumer warps read the accumulators and
// run the epilogue.  Two 128-column accumulator buffers alternate; producer and consumers meet only on
// mbarriers (buffer full: MMA commit; buffer empty and stage-3 A written: one arrival per consumer
// warp), so the tensor core runs up to two passes ahead and no CTA-wide barrier sits in the k_t loop.
// Every wait is bounded; on timeout the CTA sets the error word, stops issuing and leaves after
// releasing its tensor memory.
#include "tc_spectra_common.cuh"

namespace sal {
namespace {

using f32::bin_mag;
using f32::Tw;
using tcs::kBY;
using tcs::kK2;
using tcs::kWaitLimit;
using tcs::Pack;

constexpr int kConsumers = 8;           // consumer warps: 2 per tensor-memory lane quarter
constexpr int kThreads = 32 * (kConsumers + 1);   // + one producer warp
constexpr uint32_t kTmemCols = 256;     // two 128-column accumulator buffers

template <int N> struct TcGeo : tcs::FwdGeo<N> {
    using F = tcs::FwdGeo<N>;
    static constexpr size_t OFF_TAB = F::R0_B;
    static constexpr size_t OFF_A3 = OFF_TAB + F::TAB_B;
    static constexpr size_t OFF_MISC = OFF_A3 + 2 * F::A3_B;
    static constexpr size_t SMEM = OFF_MISC + 80 + 16 * 4;
    static_assert(F::NB1 * 16 <= (int)kTmemCols, "tensor memory");
    static_assert(F::PASSES * F::OPC * 2 == 8, "accumulator slots");
    static_assert(SMEM <= 113 * 1024, "two CTAs per SM");
};

template <int N, int FMT>
__global__ void k1_tc_tables(const __grid_constant__ Tw<N> tw, unsigned char* __restrict__ out, int feat) {
    tcs::build_fwd_tables<N, FMT>(tw, out, threadIdx.x, blockDim.x, feat);
}

// EN: the energy reading of the feature (|F|^2 per bin; the weight table then holds r_m^2)
template <int N, int FMT, bool EN>
__global__ void __launch_bounds__(kThreads, 2)
k1_spectra_tc(const float* __restrict__ V, float* __restrict__ E, int T, int X, int Y, int bnd, int stride,
              const unsigned char* __restrict__ tables, int* __restrict__ err,
              const __grid_constant__ CUtensorMap tmap, int smode) {
    using G = TcGeo<N>;
    constexpr int H = G::H, P = G::P;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* s_a1 = smem;                              // stage-1 A (MN-major), then:
    unsigned char* s_b2 = smem;                              // stage-2 B tiles, one per k_t (K-major)
    unsigned char* s_tab = smem + G::OFF_TAB;                // constant operands (bulk copy)
    unsigned char* s_are = smem + G::OFF_A3;                 // stage-3 A, real part (MN-major)
    unsigned char* s_aim = smem + G::OFF_A3 + G::A3_B;       // stage-3 A, imaginary part
    const float* s_wt = reinterpret_cast<const float*>(s_tab + G::TAB_WT);   // [k_t][|k_x|][|k_y|][3]
    // mbarriers: [0], [1] buffer full (MMA commit); [2], [3] buffer empty (one arrival per consumer warp);
    // [4] stage-3 A written, [5] stage-2 B tiles written (one arrival per consumer warp); [6] constants;
    // [7] the brick's TMA copies landed
    uint64_t* s_mbar = reinterpret_cast<uint64_t*>(smem + G::OFF_MISC);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + G::OFF_MISC + 64);
    int* s_fail = reinterpret_cast<int*>(smem + G::OFF_MISC + 68);
    float* s_red = reinterpret_cast<float*>(smem + G::OFF_MISC + 80);   // [warps]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int yb = blockIdx.x * kBY;
    const int xb = blockIdx.y * P;
    const int t0 = blockIdx.z * stride;   // stride s: only the planes t0 = multiple of s

    // ---- set-up: tensor memory, mbarriers, constant operands (bulk copy), stage-3 A zero rows --------
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(s_tmem), kTmemCols);
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(&s_mbar[0]), 1);
        tc::mbar_init(tc::smem_u32(&s_mbar[1]), 1);
        tc::mbar_init(tc::smem_u32(&s_mbar[2]), kConsumers);
        tc::mbar_init(tc::smem_u32(&s_mbar[3]), kConsumers);
        tc::mbar_init(tc::smem_u32(&s_mbar[4]), kConsumers);
        tc::mbar_init(tc::smem_u32(&s_mbar[5]), kConsumers);
        tc::mbar_init(tc::smem_u32(&s_mbar[6]), 1);
        tc::mbar_init(tc::smem_u32(&s_mbar[7]), 1);
        *s_fail = 0;
        tc::mbar_arrive_expect_tx(tc::smem_u32(&s_mbar[6]), (uint32_t)G::TAB_B);
        tc::bulk_g2s(tc::smem_u32(s_tab), tables, (uint32_t)G::TAB_B, tc::smem_u32(&s_mbar[6]));
    }
    // an interior brick: its copies go to the TMA unit first (warp 0), the rest of the set-up overlaps them
    const bool tma = tcs::tma_brick<N>(smode, T, X, Y, t0, xb, yb);
    if (tma && warp == 0)
        tcs::stage_issue<N>(smode, &tmap, V, X, Y, t0, xb, yb, smem + G::STG_OFF, tc::smem_u32(&s_mbar[7]), lane);
    // stage-3 A rows beyond the halo (read by the last windows, multiplied by zero twiddles) stay zero
    for (int i = tid; i < (int)(2 * G::A3_B / 16); i += kThreads)
        reinterpret_cast<uint4*>(s_are)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();   // mbarriers initialised before anyone waits on them

    // ---- the halo brick as the 16-bit stage-1 A operand ----------------------------------------------
    const float scale = tcs::stage_brick<N, FMT, kThreads>(V, T, X, Y, bnd, t0, xb, yb, s_a1, s_red, tid, tma,
                                                           smem + G::STG_OFF, smode, tc::smem_u32(&s_mbar[7]), err,
                                                           s_fail);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *s_tmem;
    volatile int* v_fail = s_fail;
    auto give_up = [&]() {
        atomicOr(err, 1);
        atomicExch(s_fail, 1);
    };

    const int q = warp & 3, half = (warp >> 2) & 1;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;

    if (warp == kConsumers) {
        // ============================ producer warp: one elected lane issues every MMA ========================
        {
            const uint32_t idesc1 = tc::idesc_f16(FMT, 128, 16, 1, 0);
            const uint32_t idesc2 = tc::idesc_f16(FMT, 128, G::N2, 0, 0);
            const uint32_t idesc3 = tc::idesc_f16(FMT, 128, G::N3, 1, 0);
            const uint32_t tab = tc::smem_u32(s_tab), b2base = tc::smem_u32(s_b2);
            const uint32_t are = tc::smem_u32(s_are), aim = tc::smem_u32(s_aim);
            const uint64_t b3a = tc::desc_noswizzle(tab + (uint32_t)G::TAB_B3A, 128, 256);
            const uint64_t b3b = tc::desc_noswizzle(tab + (uint32_t)G::TAB_B3B, 128, 256);
            // warp-uniform bounded wait; a give-up (here or in a consumer) stops all further issue
            auto pwait = [&](int b, uint32_t parity) -> bool {
                bool ok = !*v_fail && tc::mbar_wait(tc::smem_u32(&s_mbar[b]), parity, kWaitLimit);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok && lane == 0 && !*v_fail) give_up();
                tc::fence_after_sync();
                return ok;
            };
            // base descriptors; windows and K steps are the same descriptors moved (desc_add)
            const uint64_t a2d = tc::desc_noswizzle(tab, 128, G::SBO_K2);
            const uint64_t b2d = tc::desc_noswizzle(b2base, 128, G::SBO_K2);
            const uint64_t ared = tc::desc_noswizzle(are, 128, G::SBO_A3);
            const uint64_t aimd = tc::desc_noswizzle(aim, 128, G::SBO_A3);
            auto issue_s2 = [&](int kt) {
                const uint64_t b2 = tc::desc_add(b2d, (uint32_t)(kt * G::B2_B));
                if (tc::elect_one()) {
#pragma unroll
                    for (int s = 0; s < kK2 / 16; ++s)
                        tc::mma_f16(tmem, tc::desc_add(a2d, 256 * s), tc::desc_add(b2, 256 * s), idesc2,
                                    s > 0 ? 1u : 0u);
                    tc::mma_commit(tc::smem_u32(&s_mbar[0]));
                }
                __syncwarp();
            };
            auto issue_s3 = [&](int pass) {
                const uint32_t col = (uint32_t)(128 * (pass & 1));
                if (tc::elect_one()) {
#pragma unroll
                    for (int j = 0; j < G::OPP; ++j) {
                        const uint32_t y0 = pass * G::OPP + j;
                        tc::mma_f16(tmem + col + j * G::N3, tc::desc_add(ared, y0 * 16), b3a, idesc3, 0);
                        tc::mma_f16(tmem + col + j * G::N3, tc::desc_add(aimd, y0 * 16), b3b, idesc3, 1);
                    }
                    tc::mma_commit(tc::smem_u32(&s_mbar[pass & 1]));
                }
                __syncwarp();
            };
            bool alive = pwait(6, 0);
            if (alive) {   // stage 1, all k_t at once
                const uint64_t b1 = tc::desc_noswizzle(tab + (uint32_t)G::TAB_B1, 128, 256);
                const uint64_t a1 = tc::desc_noswizzle(tc::smem_u32(s_a1), 128, 256);
                if (tc::elect_one()) {
#pragma unroll
                    for (int i = 0; i < G::NB1; ++i) tc::mma_f16(tmem + 16 * i, tc::desc_add(a1, 4096 * i), b1, idesc1, 0);
                    tc::mma_commit(tc::smem_u32(&s_mbar[0]));
                }
                __syncwarp();
            }
            alive = alive && pwait(5, 0);             // the stage-2 B tiles are written
            if (alive) issue_s2(0);
            uint32_t pa = 0, pe0 = 0, pe1 = 0;
            for (int kt = 0; kt < H && alive; ++kt) {
                alive = pwait(4, pa);                 // A3(kt) written; buffer 0 (D2) read
                pa ^= 1u;
                if (!alive) break;
                issue_s3(0);
                if (kt > 0) {
                    alive = pwait(3, pe1);            // buffer 1 released by the last pass of kt - 1
                    pe1 ^= 1u;
                    if (!alive) break;
                }
                issue_s3(1);
#pragma unroll
                for (int pass = 2; pass < G::PASSES; ++pass) {
                    const int b = pass & 1;
                    alive = pwait(2 + b, b ? pe1 : pe0);   // pass - 2 released buffer b
                    if (b) pe1 ^= 1u; else pe0 ^= 1u;
                    if (!alive) break;
                    issue_s3(pass);
                }
                if (!alive || kt + 1 == H) break;
                alive = pwait(2, pe0);                // pass PASSES - 2 released buffer 0
                pe0 ^= 1u;
                if (alive) issue_s2(kt + 1);
            }
        }
        __syncwarp();
    }

    // ================================ consumer warps ===============================================
    const int m = 32 * q + lane;
    const int x0l = m / N, kx = m % N;
    const int ajx = kx <= N / 2 ? kx : N - kx;
    float acc[8][3];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i][0] = acc[i][1] = acc[i][2] = 0.f;
    if (warp < kConsumers) {
        // warp-uniform bounded wait
        auto cwait = [&](int b, uint32_t parity) -> bool {
            bool ok = !*v_fail && tc::mbar_wait(tc::smem_u32(&s_mbar[b]), parity, kWaitLimit);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok && lane == 0 && !*v_fail) give_up();
            tc::fence_after_sync();
            return ok;
        };
        auto arrive = [&](int b) {
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(tc::smem_u32(&s_mbar[b]));
        };
        uint32_t pf0 = 0, pf1 = 0;
        // D1 -> one stage-2 B tile per k_t (the A1 region is free once the stage-1 MMAs completed)
        if (cwait(0, pf0)) tcs::d1_to_b2<N, FMT>(tmem, s_b2, q, lane, half, 2);
        pf0 ^= 1u;
        tc::fence_async_smem();
        arrive(5);
        // D2 of the first tile -> stage-3 A operands (half 0: real columns, half 1: imaginary)
        if (cwait(0, pf0)) tcs::d2_to_a3<N, FMT>(tmem, s_are, s_aim, q, lane, half);
        pf0 ^= 1u;
        arrive(4);
        for (int kt = 0; kt < H; ++kt) {
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
                const bool full = cwait(b, b ? pf1 : pf0);
                if (b) pf1 ^= 1u; else pf0 ^= 1u;
                if (pass == G::PASSES - 1 && kt + 1 < H) {
                    // the last pass's buffer is full, so every stage-3 MMA of kt has completed and A3 is free: the
                    // D2 of kt + 1 (its stage-2 MMAs followed this pass's) goes into A3 before this pass's
                    // epilogue, and the first stage-3 MMAs of kt + 1 run under that epilogue
                    if (cwait(0, pf0)) tcs::d2_to_a3<N, FMT>(tmem, s_are, s_aim, q, lane, half);
                    pf0 ^= 1u;
                    arrive(4);
                }
                if (full) {
#pragma unroll
                    for (int cc = 0; cc < 2; ++cc) {   // chunks half and half + 2 of this buffer
                        float v[32];
                        tc::tmem_ld32(tmem + lane_base + (uint32_t)(128 * b + 32 * (half + 2 * cc)), v);
#pragma unroll
                        for (int o = 0; o < G::OPC; ++o) {
                            // |F|^2 of bins (2j, 2j+1) with packed FP32 pairs (two rounded FMAs per
                            // instruction), then |F| per bin, bins k and n - k summed (same Eq. 1 ratios)
                            float mg[N];
#pragma unroll
                            for (int j = 0; j < N / 2; ++j) {
                                const float2 re = make_float2(v[o * G::N3 + 2 * j], v[o * G::N3 + 2 * j + 1]);
                                const float2 im = make_float2(v[o * G::N3 + N + 2 * j], v[o * G::N3 + N + 2 * j + 1]);
                                const float2 m2 = __ffma2_rn(re, re, __fmul2_rn(im, im));
                                mg[2 * j] = bin_mag<EN>(m2.x);
                                mg[2 * j + 1] = bin_mag<EN>(m2.y);
                            }
                            float sm[H];
#pragma unroll
                            for (int k = 0; k < H; ++k) sm[k] = (k == 0 || 2 * k == N) ? mg[k] : mg[k] + mg[N - k];
                            // the weighted sums over |k_y|, two partial sums per map in one packed pair
                            float2 a0 = make_float2(0.f, 0.f), a1 = a0, a2 = a0;
#pragma unroll
                            for (int k = 0; k + 1 < H; k += 2) {
                                const float2 s2 = make_float2(sm[k], sm[k + 1]);
                                a0 = __ffma2_rn(make_float2(wt[0][k], wt[0][k + 1]), s2, a0);
                                a1 = __ffma2_rn(make_float2(wt[1][k], wt[1][k + 1]), s2, a1);
                                a2 = __ffma2_rn(make_float2(wt[2][k], wt[2][k + 1]), s2, a2);
                            }
                            float e0 = a0.x + a0.y, e1 = a1.x + a1.y, e2 = a2.x + a2.y;
                            if (H & 1) {
                                e0 = fmaf(wt[0][H - 1], sm[H - 1], e0);
                                e1 = fmaf(wt[1][H - 1], sm[H - 1], e1);
                                e2 = fmaf(wt[2][H - 1], sm[H - 1], e2);
                            }
                            const int slot = (pass * 2 + cc) * G::OPC + o;
                            acc[slot][0] += e0;
                            acc[slot][1] += e1;
                            acc[slot][2] += e2;
                        }
                    }
                }
                arrive(2 + b);                                 // this warp is done with buffer b
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();

    // ---- sum over the n lanes of each x0 (k_x), write E -------------------------------------------
    // E: [3][T][X][Y], or the lattice [3][Tc][Xc][Yc] (ceil(T / s) ...) for stride s > 1
    const int Xc = (X + stride - 1) / stride, Yc = (Y + stride - 1) / stride;
    const size_t NV = (size_t)((T + stride - 1) / stride) * Xc * Yc;
    const int x = xb + x0l;
    const bool good = *s_fail == 0 && warp < kConsumers;   // the producer warp holds no results
    const float out_scale = EN ? scale * scale : scale;     // the features of the unscaled brick
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
                    if (kx == 0 && x < X && y < Y && good) {
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

template <int N, int FMT>
cudaError_t prepare_nf() {
    cudaError_t e = cudaFuncSetAttribute(k1_spectra_tc<N, FMT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)TcGeo<N>::SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k1_spectra_tc<N, FMT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)TcGeo<N>::SMEM);
}

template <int N, int FMT>
cudaError_t tables_nf(const TwiddleTable& t, int feat, void* dst, cudaStream_t s) {
    k1_tc_tables<N, FMT><<<1, 256, 0, s>>>(f32::make_tw<N>(t), static_cast<unsigned char*>(dst), feat);
    note_launches(1);
    return cudaGetLastError();
}

template <int N, int FMT>
cudaError_t launch_nf(const void* tables, const float* V, float* E, int T, int X, int Y, int bnd, int feat, int stride,
                      const float* Vt, int Yt, int* err, cudaStream_t s) {
    using G = TcGeo<N>;
    dim3 grid((Y + kBY - 1) / kBY, (X + G::P - 1) / G::P, (T + stride - 1) / stride);
    const unsigned char* tab = static_cast<const unsigned char*>(tables);
    CUtensorMap tmap;
    const int smode = tcs::brick_stage_mode<N>(V, T, X, Y, &tmap, true, Vt, Yt);
    if (feat == 1)
        k1_spectra_tc<N, FMT, true><<<grid, kThreads, G::SMEM, s>>>(V, E, T, X, Y, bnd, stride, tab, err, tmap, smode);
    else
        k1_spectra_tc<N, FMT, false><<<grid, kThreads, G::SMEM, s>>>(V, E, T, X, Y, bnd, stride, tab, err, tmap, smode);
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

cudaError_t spectra_tc_tables_build(int n, int fmt, const TwiddleTable& tw, int feat, void* dst, cudaStream_t s) {
    if (n == 8) return fmt == 1 ? tables_nf<8, 1>(tw, feat, dst, s) : tables_nf<8, 0>(tw, feat, dst, s);
    if (n == 16) return fmt == 1 ? tables_nf<16, 1>(tw, feat, dst, s) : tables_nf<16, 0>(tw, feat, dst, s);
    return cudaErrorInvalidValue;
}

cudaError_t spectra_tc_launch(int n, int fmt, const void* tables, const float* V, float* E, int T, int X, int Y,
                              int bnd, int feat, int stride, const float* Vt, int Yt, int* err, cudaStream_t s) {
    if (stride < 1) return cudaErrorInvalidConfiguration;
    if (n == 8) return fmt == 1 ? launch_nf<8, 1>(tables, V, E, T, X, Y, bnd, feat, stride, Vt, Yt, err, s)
                                : launch_nf<8, 0>(tables, V, E, T, X, Y, bnd, feat, stride, Vt, Yt, err, s);
    if (n == 16) return fmt == 1 ? launch_nf<16, 1>(tables, V, E, T, X, Y, bnd, feat, stride, Vt, Yt, err, s)
                                 : launch_nf<16, 0>(tables, V, E, T, X, Y, bnd, feat, stride, Vt, Yt, err, s);
    return cudaErrorInvalidValue;
}

}  // namespace sal
