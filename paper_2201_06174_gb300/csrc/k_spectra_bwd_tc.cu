// K5-TC: adjoint of the local-spectrum feature step (backward of Sec. 2 steps 1-3; Eq. 1, Eq. 2) with
// every dense contraction on the 5th-generation tensor cores (tcgen05.mma, kind::f16, FP16 operands,
// FP32 accumulation in tensor memory).  Same brick as K1-TC: t0, x0 in [xb, xb + P), P = 128/n,
// y0 in [yb, yb + 16).
//   forward recompute: stages 1-3 as in K1-TC (tc_spectra_common.cuh): the spectra are recomputed
//     brick by brick, never stored;
//   Gamma (epilogue from tensor memory): Gamma[k] = (sum_m gE_m wt_m(k)) F[k]/|F[k]| -- the gradient of
//     L = sum gE . E with respect to (Re F, Im F) -- with the zero subgradient where |F| <= 2^-19 of the
//     window's L1 norm (FP16 operands put the direction of smaller bins at the level of their rounding;
//     the 16-bit forms answer to the 1e-2 bar) (the energy reading: Gamma[k] = 2 (sum_m gE_m wt_m(k)) F[k], wt holding r_m^2);
//     rounded to FP16 (scaled by sigma = n^3 / (8 max|gE|)) into the operand [(x0, k_x)][(re | im, k_y)]
//     of one output;
//   adjoint of stage 3 (y): Gamma of bins k and n - k folded into pair coefficients (A = G[k] + G[n-k],
//     B = G[k] - G[n-k]; the twiddles of n - k are those of k with the sine negated):
//       dG2r[y] = sum_y0 [A_r | B_i] Tinv_re(y - y0),  Tinv_re = [c_k | -s_k],
//       dG2i[y] = sum_y0 [A_i | B_r] Tinv_im(y - y0),  Tinv_im = [c_k |  s_k],
//     one MMA (K = 16) per part and output, all outputs accumulating into one accumulator -- the
//     overlap-add over the sliding windows happens in the accumulator.  Tinv is one table of rows
//     y - y0 + 15 (K-major with 16-byte rows), so the window of output y0 is the same descriptor moved
//     by 16 (15 - y0) bytes;
//   adjoint of stage 2 (x): the stage-2 twiddle matrix A2 [(x0,k_x)][(cos|sin, x)] read as an MN-major
//     operand is its transpose; with B_c = [dG2r | dG2i] and B_s = [-dG2i | dG2r] (dG2 rounded to FP16),
//     D[x][(re|im, y)] = A2_cos^T B_c + A2_sin^T B_s is dG1 = (sum c dG2r - s dG2i, sum c dG2i + s dG2r)
//     directly (two MMA chains of K = 128, the sin rows selected by moving the start 24 rows);
//   adjoint of stage 1 (t) on the tensor cores as well: dG1 (scaled, FP16) is written as an MN-major
//     A operand [pos][(re, im, 0...)] and D_t[pos][u_t] += A_t B_t(k_t), B_t = [c | -s](k_t, u_t),
//     accumulates the brick's block of gVext over all k_t in tensor memory; at the end it is written to
//     scratch [u_t][x][y] and the fixed-order gather kernel sums the overlapping blocks.
// Warp-specialised: two issuing warps (one for the forward recompute's MMAs, one for the adjoint's MMAs and
// the dG1 moves, so that neither chain of waits holds back the other), sixteen consumer warps compute Gamma
// and move the adjoint operands; they meet only on mbarriers, and the stage-3 MMAs of the next k_t tile are
// issued while the consumers still read back the adjoint of the current one.
// FP16 operands in both 16-bit forms (3 more mantissa bits than BF16: the direction F/|F| of small bins
// amplifies operand rounding).  Every wait on the tensor cores is bounded; on timeout the CTA sets the
// error word, skips the remaining MMAs and writes a zero block.
#include "tc_spectra_common.cuh"

namespace sal {
namespace {

using f32::fast_rsqrt;
using f32::Tw;
using tcs::kBY;
using tcs::kK2;
using tcs::kWaitLimit;
using tcs::kXHP;
using tcs::Pack;

constexpr int kFmt = 0;                   // FP16 operands
constexpr int kConsumers = 16;            // consumer warps: 4 per tensor-memory lane quarter
constexpr int kThreads = 32 * (kConsumers + 2);   // + the adjoint and the forward issuing warps
constexpr int kBars = 16;                 // mbarriers
constexpr uint32_t kTmemCols = 512;       // [0,256) forward buffers; [256,320) dG2; [320,384) dG1; [384,480) gV
constexpr uint32_t kColY = 256;
constexpr uint32_t kColX = 320;
constexpr uint32_t kColT = 384;
constexpr float kDxScale = 1.f / 64.f;    // keeps the FP16 copy of dG1 far from the FP16 range limit
constexpr float kKinkTau = 1.0f / 524288.0f;  // zero-subgradient band of |F| (2^-19 of the window L1 norm)
constexpr int kTR = 48;                   // rows of the shifted inverse twiddle tables (y - y0 + 15)

template <int N> struct BtGeo : tcs::FwdGeo<N> {
    using F = tcs::FwdGeo<N>;
    static constexpr int KG = 2 * N;                          // Gamma K: re | im over k_y
    static constexpr uint32_t SBO_G = KG / 8 * 128;           // 8-row group stride of a Gamma operand
    static constexpr size_t SLOT_B = (size_t)16 * SBO_G;      // one output (128 rows)
    static constexpr size_t GSET_B = (size_t)F::OPP * SLOT_B; // one pass
    static constexpr int PK = 2 * F::H - 2;                   // pair coefficients per part (n)
    static constexpr uint32_t TI_LBO = kTR * 16;              // K-group stride of a shifted table
    static constexpr size_t TI_B = (size_t)2 * TI_LBO;        // K = 16 per table
    static constexpr uint32_t IM_OFF = PK == 16 ? 256u : 0u;  // K offset of the imaginary-part operand
    static constexpr size_t TAB_TRE = F::TAB_B;
    static constexpr size_t TAB_TIM = TAB_TRE + TI_B;
    static constexpr size_t TAB_BT = TAB_TIM + TI_B;          // B_t per k_t: [u][(re, im, 0...)], 512 B each
    static constexpr size_t TAB5_B = TAB_BT + (size_t)F::H * 512;
    static constexpr size_t BDG_B = (size_t)8 * 2048;         // one dG2 operand [K = 128][N = 64], MN-major
    static constexpr int SLICE = (F::XH * F::YH + 3) / 4 * 4;   // u_t slices of the block, 16-byte aligned
    static constexpr int BLOCK_FLOATS = N * SLICE;
    static constexpr size_t OFF_TAB = F::R0_B;
    static constexpr size_t OFF_A3 = OFF_TAB + TAB5_B;
    static constexpr size_t OFF_G = (OFF_A3 + 2 * F::A3_B + 127) / 128 * 128;   // two Gamma sets
    static constexpr size_t G_B = 2 * GSET_B;
    static constexpr size_t OFF_BC = OFF_G + G_B;                // B_c | B_s (their own region)
    static constexpr size_t OFF_AT = OFF_BC + 2 * BDG_B;         // t-adjoint A operand [pos][16], MN-major
    static constexpr size_t OFF_GE = OFF_AT + F::A1_B;
    static constexpr size_t OFF_L1 = OFF_GE + (size_t)3 * F::P * kBY * 4;
    static constexpr size_t OFF_MISC = (OFF_L1 + (size_t)F::P * kBY * 4 + 15) / 16 * 16;
    static constexpr size_t SMEM = OFF_MISC + 8 * kBars + 16 + 2 * 32 * 4;
    static_assert((size_t)(kXHP * F::YP + F::XH * kBY) * 4 <= G_B, "L1 sums fit in the Gamma region");
    static_assert(TAB5_B % 16 == 0 && OFF_A3 % 16 == 0 && OFF_AT % 16 == 0, "alignment");
    static_assert(kColT + 16 * F::NB1 <= kTmemCols, "tensor memory");
    static_assert(OFF_BC % 128 == 0, "B_c | B_s alignment");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

// The adjoint's constant operands: the forward tables, then the shifted inverse-y twiddles of the pair
// coefficients, byte(row, K) = row 16 + (K/8) TI_LBO + (K%8) 2, d = row - 15, K = 16 per table:
//   re table: kk < H: c(kk, d); H <= kk < 2H-2: -s(kk-H+1, d)   (multiplies [A_r | B_i])
//   im table: kk < H: c(kk, d); H <= kk < 2H-2:  s(kk-H+1, d)   (multiplies [A_i | B_r])
// with kk = K for n = 16; for n = 8 the operand holds both parts in one K = 16 row ([re | im], 8 each), so
// the re table is zero in K 8..15 and the im table holds its entries at K = 8 + kk (zero below).
template <int N>
__global__ void k5_tc_tables(const __grid_constant__ Tw<N> tw, unsigned char* __restrict__ out, int feat) {
    using G = BtGeo<N>;
    constexpr int H = G::H;
    tcs::build_fwd_tables<N, kFmt>(tw, out, threadIdx.x, blockDim.x, feat);
    unsigned char* tre = out + G::TAB_TRE;
    unsigned char* tim = out + G::TAB_TIM;
    for (int i = threadIdx.x; i < kTR * 16; i += blockDim.x) {
        const int row = i / 16, K = i % 16, d = row - 15;
        auto coef = [&](int kk, bool im_part) -> float {
            if (kk < 0 || kk >= 2 * H - 2) return 0.f;
            if (kk < H) return tcs::twc<N>(tw, kk, d);
            const float sv = tcs::tws<N>(tw, kk - H + 1, d);
            return im_part ? sv : -sv;
        };
        const float vre = G::PK == 16 ? coef(K, false) : (K < 8 ? coef(K, false) : 0.f);
        const float vim = G::PK == 16 ? coef(K, true) : (K >= 8 ? coef(K - 8, true) : 0.f);
        const size_t off = (size_t)row * 16 + (K / 8) * G::TI_LBO + (K % 8) * 2;
        *reinterpret_cast<uint16_t*>(tre + off) = Pack<kFmt>::one(vre);
        *reinterpret_cast<uint16_t*>(tim + off) = Pack<kFmt>::one(vim);
    }
    // B_t(k_t)[u][k] (K-major, N = u): k = 0: c(k_t, u), k = 1: -s(k_t, u), other K rows zero
    unsigned char* bt = out + G::TAB_BT;
    for (int i = threadIdx.x; i < G::H * 256; i += blockDim.x) {
        const int kt = i / 256, u = (i / 16) % 16, k = i % 16;
        const float v = k == 0 ? tcs::twc<N>(tw, kt, u) : (k == 1 ? -tcs::tws<N>(tw, kt, u) : 0.f);
        *reinterpret_cast<uint16_t*>(bt + kt * 512 + (u / 8) * 256 + (k / 8) * 128 + (u % 8) * 16 + (k % 8) * 2) =
            Pack<kFmt>::one(v);
    }
}

// EN: the energy reading of the feature: Gamma = 2 rho F (no kink band).  The operand holds
// sigma (2 / n^3) rho F of the staged brick (whose |F| is at most n^3, so the FP16 operand stays in the
// range of the feature's unit directions) and the block is scaled back by n^3 max|V| / sigma.
template <int N, bool EN>
__global__ void __launch_bounds__(kThreads, 1)
k5_spectra_adjoint_tc(const float* __restrict__ V, const float* __restrict__ gE, float* __restrict__ blocks,
                      int T, int X, int Y, int bnd, int t_begin, int t_step,
                      const unsigned char* __restrict__ tables,
                      const __grid_constant__ Tw<N> tw, int* __restrict__ err,
                      const __grid_constant__ CUtensorMap tmap, int smode) {
    using G = BtGeo<N>;
    constexpr int H = G::H, P = G::P, XH = G::XH, YH = G::YH, YP = G::YP;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* s_a1 = smem;                                  // stage-1 A, then the stage-2 B tiles
    unsigned char* s_b2 = smem;
    unsigned char* s_tab = smem + G::OFF_TAB;
    unsigned char* s_are = smem + G::OFF_A3;
    unsigned char* s_aim = smem + G::OFF_A3 + G::A3_B;
    unsigned char* s_g = smem + G::OFF_G;                        // Gamma operands, two sets
    unsigned char* s_bc = smem + G::OFF_BC;                      // B_c = [dG2r | dG2i] (after the y adjoint)
    unsigned char* s_bs = s_bc + G::BDG_B;                       // B_s = [-dG2i | dG2r]
    float* s_col = reinterpret_cast<float*>(smem + G::OFF_G);    // L1 column sums (set-up only)
    unsigned char* s_at = smem + G::OFF_AT;                      // t-adjoint A operand
    float* s_ge = reinterpret_cast<float*>(smem + G::OFF_GE);    // [3][P][16]
    float* s_l1 = reinterpret_cast<float*>(smem + G::OFF_L1);    // [P][16]
    const float* s_wt = reinterpret_cast<const float*>(s_tab + G::TAB_WT);
    // mbarriers (arrival counts): [0], [1] forward buffer full (MMA commit); [2], [3] forward buffer read
    // (16 warps); [4] stage-3 A written (16); [5] stage-2 B tiles written (16); [6], [7] Gamma set written
    // (16); [8] dG2 complete (commit); [9] B_c | B_s written (16); [10] dG1 complete (commit; the
    // adjoint issuing warp alone waits on it); [11] the brick's TMA copies landed; [12] constant operands landed
    // (bulk copy); [13] the brick's gV block complete; [14], [15] the adjoint-y MMAs that read Gamma set 0 / 1
    // complete (commit: the set may be rewritten)
    uint64_t* s_mbar = reinterpret_cast<uint64_t*>(smem + G::OFF_MISC);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + G::OFF_MISC + 8 * kBars);
    int* s_fail = reinterpret_cast<int*>(smem + G::OFF_MISC + 8 * kBars + 4);
    float* s_red = reinterpret_cast<float*>(smem + G::OFF_MISC + 8 * kBars + 16);  // [2][32]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int q = warp & 3, grp = (warp >> 2) & 3;
    const int yb = blockIdx.x * kBY;
    const int xb = blockIdx.y * P;
    const int t0 = t_begin + blockIdx.z * t_step;   // t_step s > 1: the lattice planes of stride-s windows
    const size_t NV = (size_t)T * X * Y;

    // ---- set-up ------------------------------------------------------------------------------------
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(s_tmem), kTmemCols);
    if (tid == 0) {
        const uint32_t counts[kBars] = {1, 1, kConsumers, kConsumers, kConsumers, kConsumers, kConsumers, kConsumers,
                                        1, kConsumers, 1, 1, 1, 1, 1, 1};
        for (int b = 0; b < kBars; ++b) tc::mbar_init(tc::smem_u32(&s_mbar[b]), counts[b]);
        *s_fail = 0;
        tc::mbar_arrive_expect_tx(tc::smem_u32(&s_mbar[12]), (uint32_t)G::TAB5_B);
        tc::bulk_g2s(tc::smem_u32(s_tab), tables, (uint32_t)G::TAB5_B, tc::smem_u32(&s_mbar[12]));
    }
    // an interior brick: its copies go to the TMA unit first (warp 0), the rest of the set-up overlaps them
    const bool tma = tcs::tma_brick<N>(smode, T, X, Y, t0, xb, yb);
    if (tma && warp == 0)
        tcs::stage_issue<N>(smode, &tmap, V, X, Y, t0, xb, yb, smem + G::STG_OFF, tc::smem_u32(&s_mbar[11]), lane);
    for (int i = tid; i < (int)(2 * G::A3_B / 16); i += kThreads)
        reinterpret_cast<uint4*>(s_are)[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = tid; i < (int)(G::A1_B / 16); i += kThreads)       // K rows 2..15 of A_t stay zero
        reinterpret_cast<uint4*>(s_at)[i] = make_uint4(0u, 0u, 0u, 0u);
    float gmax = 0.f;
    for (int i = tid; i < 3 * P * kBY; i += kThreads) {
        const int y0 = i % kBY, xl = (i / kBY) % P, m = i / (kBY * P);
        const int x = xb + xl, y = yb + y0;
        const float g = (x < X && y < Y) ? __ldg(gE + m * NV + ((size_t)t0 * X + x) * Y + y) : 0.f;
        s_ge[i] = g;
        gmax = fmaxf(gmax, fabsf(g));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
    if (lane == 0) s_red[32 + warp] = gmax;
    __syncthreads();   // mbarriers initialised before anyone waits on them
    const float scale = tcs::stage_brick<N, kFmt, kThreads>(V, T, X, Y, bnd, t0, xb, yb, s_a1, s_red, tid, tma,
                                                            smem + G::STG_OFF, smode, tc::smem_u32(&s_mbar[11]), err,
                                                            s_fail);
    // the direction F/|F| does not depend on the brick scale; the energy's Gamma = 2 rho F does (F of the
    // unscaled brick = scale x F of the staged one): that factor is applied to the block at the end
    float bgmax = 0.f;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) bgmax = fmaxf(bgmax, s_red[32 + w]);
    const float sigma = bgmax > 0.f ? (float)(N * N * N) / (8.f * bgmax) : 1.f;   // Gamma operand scale
    // per-bin factor of the operand: sigma rho / |F| (feature), sigma (2 / n^3) rho (energy)
    const float sigma_op = EN ? sigma * (2.f / (float)(N * N * N)) : sigma;
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    // window L1 norms (the kink band of |F|), in the units of the scaled brick: column sums over t of
    // h(u) |V|, then a box over x and y with h(u_x) h(u_y)
    for (int pos = tid; pos < kXHP * YP; pos += kThreads) {
        float a = 0.f;
#pragma unroll
        for (int u = 0; u < N; ++u) {
            const __half hv = *reinterpret_cast<const __half*>(s_a1 + (pos / 8) * 256 + (u / 8) * 128 + (u % 8) * 16 +
                                                               (pos % 8) * 2);
            a = fmaf(tw.c[0][u], fabsf(__half2float(hv)), a);
        }
        s_col[pos] = a;
    }
    __syncthreads();
    // box over y (h(u_y)), rows x of the halo, kept in the upper part of the column-sum area
    float* s_row = s_col + kXHP * YP;
    for (int i = tid; i < XH * kBY; i += kThreads) {
        const int y0 = i % kBY, x = i / kBY;
        float a = 0.f;
#pragma unroll
        for (int uy = 0; uy < N; ++uy) a = fmaf(tw.c[0][uy], s_col[x * YP + y0 + uy], a);
        s_row[i] = a;
    }
    __syncthreads();
    for (int i = tid; i < P * kBY; i += kThreads) {
        const int y0 = i % kBY, xl = i / kBY;
        float a = 0.f;
#pragma unroll
        for (int ux = 0; ux < N; ++ux) a = fmaf(tw.c[0][ux], s_row[(xl + ux) * kBY + y0], a);
        s_l1[i] = a;
    }
    __syncthreads();   // L1 norms visible; the column-sum area (Gamma region) free again
    tc::fence_after_sync();
    const uint32_t tmem = *s_tmem;
    volatile int* v_fail = s_fail;
    auto give_up = [&]() {
        atomicOr(err, 1);
        atomicExch(s_fail, 1);
    };
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;

    if (warp >= kConsumers) {
        // ====== issuing warps: in each, one elected lane issues the MMAs.  The adjoint warp (lane quarter 0 of
        // tensor memory) also moves dG1 into the t-adjoint operand, so the consumers never wait for the
        // adjoint of stage 2 ======
        {
            const bool adjoint = warp == kConsumers;
            const bool leader = lane == 0;
            const uint32_t idesc1 = tc::idesc_f16(kFmt, 128, 16, 1, 0);
            const uint32_t idesc2 = tc::idesc_f16(kFmt, 128, G::N2, 0, 0);
            const uint32_t idesc3 = tc::idesc_f16(kFmt, 128, G::N3, 1, 0);
            const uint32_t idescy = tc::idesc_f16(kFmt, 128, 32, 0, 0);
            const uint32_t idescx = tc::idesc_f16(kFmt, 128, 64, 1, 1);
            const uint32_t idesct = tc::idesc_f16(kFmt, 128, 16, 1, 0);
            const uint32_t tab = tc::smem_u32(s_tab), b2base = tc::smem_u32(s_b2);
            const uint32_t are = tc::smem_u32(s_are), aim = tc::smem_u32(s_aim);
            const uint32_t gbase = tc::smem_u32(s_g), bc = tc::smem_u32(s_bc), bs = tc::smem_u32(s_bs);
            const uint32_t at = tc::smem_u32(s_at);
            const uint64_t b3a = tc::desc_noswizzle(tab + (uint32_t)G::TAB_B3A, 128, 256);
            const uint64_t b3b = tc::desc_noswizzle(tab + (uint32_t)G::TAB_B3B, 128, 256);
            uint32_t ph = 0;   // expected phase parity of each mbarrier, one bit each
            auto commit = [&](int b) {
                if (tc::elect_one()) tc::mma_commit(tc::smem_u32(&s_mbar[b]));
                __syncwarp();
            };
            // warp-uniform bounded wait; a give-up (here or in a consumer) stops all further issue
            auto pwait = [&](int b) -> bool {
                bool ok = !*v_fail && tc::mbar_wait(tc::smem_u32(&s_mbar[b]), (ph >> b) & 1u, kWaitLimit);
                ph ^= 1u << b;
                ok = __all_sync(0xffffffffu, ok);
                if (!ok && leader && !*v_fail) give_up();
                tc::fence_after_sync();
                return ok;
            };
            // base descriptors; windows, slots and K steps are the same descriptors moved (desc_add)
            const uint64_t a2d = tc::desc_noswizzle(tab, 128, G::SBO_K2);
            const uint64_t b2d = tc::desc_noswizzle(b2base, 128, G::SBO_K2);
            const uint64_t ared = tc::desc_noswizzle(are, 128, G::SBO_A3);
            const uint64_t aimd = tc::desc_noswizzle(aim, 128, G::SBO_A3);
            const uint64_t gd = tc::desc_noswizzle(gbase, 128, G::SBO_G);
            const uint64_t tred = tc::desc_noswizzle(tab + (uint32_t)G::TAB_TRE, G::TI_LBO, 128);
            const uint64_t timd = tc::desc_noswizzle(tab + (uint32_t)G::TAB_TIM, G::TI_LBO, 128);
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
            // adjoint of stage 3 for the outputs of one pass (Gamma set pass % 2), accumulating into kColY
            auto issue_inv_y = [&](int pass) {
                const uint32_t set = (uint32_t)((pass & 1) * G::GSET_B);
                if (tc::elect_one()) {
#pragma unroll
                    for (int j = 0; j < G::OPP; ++j) {
                        const uint32_t y0 = pass * G::OPP + j;
                        const uint32_t slot = set + (uint32_t)(j * G::SLOT_B);
                        const uint32_t shift = (15u - y0) * 16u;
                        const uint32_t accum = y0 > 0 ? 1u : 0u;
                        tc::mma_f16(tmem + kColY, tc::desc_add(gd, slot), tc::desc_add(tred, shift), idescy, accum);
                        tc::mma_f16(tmem + kColY + 32, tc::desc_add(gd, slot + G::IM_OFF), tc::desc_add(timd, shift),
                                    idescy, accum);
                    }
                }
                __syncwarp();
            };
            if (!adjoint) {
                // ---- forward issue: stage 1 once, then stage 2 per k_t and stage 3 per pass ----------------
                bool alive = pwait(12);
                if (alive) {   // stage 1, all k_t at once
                    const uint64_t b1 = tc::desc_noswizzle(tab + (uint32_t)G::TAB_B1, 128, 256);
                    const uint64_t a1 = tc::desc_noswizzle(tc::smem_u32(s_a1), 128, 256);
                    if (tc::elect_one()) {
#pragma unroll
                        for (int i = 0; i < G::NB1; ++i)
                            tc::mma_f16(tmem + 16 * i, tc::desc_add(a1, 4096 * i), b1, idesc1, 0);
                        tc::mma_commit(tc::smem_u32(&s_mbar[0]));
                    }
                    __syncwarp();
                }
                alive = alive && pwait(5);
                if (alive) issue_s2(0);
                alive = alive && pwait(4);
                if (alive) {
                    issue_s3(0);
                    issue_s3(1);
                }
                for (int kt = 0; kt < H && alive; ++kt) {
#pragma unroll
                    for (int pass = 0; pass < G::PASSES; ++pass) {
                        const int b = pass & 1;
                        if (pass + 2 < G::PASSES) {
                            if (!(alive = pwait(2 + b))) break;   // the pass read buffer b
                            issue_s3(pass + 2);
                        } else if (pass + 2 == G::PASSES && kt + 1 < H) {
                            if (!(alive = pwait(2))) break;       // buffer 0 released
                            issue_s2(kt + 1);
                        }
                    }
                    if (!alive || kt + 1 == H) break;
                    if (!(alive = pwait(4))) break;               // A3(kt + 1) written (buffer 0's D2 read)
                    issue_s3(0);
                    if (!(alive = pwait(3))) break;               // buffer 1 released by the last pass of kt
                    issue_s3(1);
                }
            } else {
                // ---- adjoint issue: y per pass, x per k_t, t per k_t (with the dG1 moves) ------------------
                // ---- dG1 of tile ktp -> the t-adjoint operand, then the t-adjoint MMAs.  Run after the adjoint-y
                // MMAs of the next tile's first pass are issued, so the wait for the adjoint-x MMAs does not hold them
                // back; it still precedes the next adjoint-x (which rewrites dG1) and the next conversion (which
                // rewrites the operand), both later in this warp's program order.
                auto finish_t = [&](int ktp) -> bool {
                    // ---- dG1 (rows x = lane) -> the t-adjoint A operand, K rows 0 (re) and 1 (im) -------------------
                    // (the t-adjoint MMAs of tile ktp - 1 precede the adjoint-x MMAs of ktp: complete once dG1 is)
                    if (!pwait(10)) return false;
                    uint32_t d0[32], d1[32];      // columns 0..31: re over y; 32..63: im over y
                    tc::tmem_ld32_async(tmem + kColX, d0);
                    tc::tmem_ld32_async(tmem + kColX + 32u, d1);
                    tc::tmem_wait_ld(d0);
                    tc::tmem_wait_ld(d1);
    #pragma unroll
                    for (int c = 0; c < 4; ++c) {   // columns 16 c ..: re over y (c = 0, 1), im over y (c = 2, 3)
                        float v[16];
    #pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] = __uint_as_float((c < 2 ? d0 : d1)[16 * (c & 1) + i]);
                        const int k = c >> 1;
                        if (lane < kXHP) {
    #pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const int y8 = 16 * (c & 1) + 8 * h;
                                if (y8 < YP) {
                                    // MN-major: byte(pos, k) = (pos/8) 256 + (k/8) 128 + (k%8) 16 + (pos%8) 2, pos = x YP + y
                                    uint4 w;
                                    w.x = Pack<kFmt>::two(kDxScale * v[8 * h + 0], kDxScale * v[8 * h + 1]);
                                    w.y = Pack<kFmt>::two(kDxScale * v[8 * h + 2], kDxScale * v[8 * h + 3]);
                                    w.z = Pack<kFmt>::two(kDxScale * v[8 * h + 4], kDxScale * v[8 * h + 5]);
                                    w.w = Pack<kFmt>::two(kDxScale * v[8 * h + 6], kDxScale * v[8 * h + 7]);
                                    *reinterpret_cast<uint4*>(s_at + ((lane * YP + y8) / 8) * 256 + k * 16) = w;
                                }
                            }
                        }
                    }
                    tc::fence_async_smem();
                    tc::fence_before_sync();
                    __syncwarp();
                    tc::fence_after_sync();
                    // ---- adjoint of stage 1: gV block += A_t B_t(k_t), accumulated over k_t in tensor memory ----
                    const uint64_t btd = tc::desc_noswizzle(tab + (uint32_t)(G::TAB_BT + 512 * ktp), 128, 256);
                    const uint64_t atd = tc::desc_noswizzle(at, 128, 256);
                    if (tc::elect_one()) {
    #pragma unroll
                        for (int i = 0; i < G::NB1; ++i)
                            tc::mma_f16(tmem + kColT + 16 * i, tc::desc_add(atd, 4096 * i), btd, idesct, ktp > 0 ? 1u : 0u);
                    }
                    __syncwarp();
                    return true;
                };
                bool alive = pwait(12);
                for (int kt = 0; kt < H && alive; ++kt) {
#pragma unroll
                    for (int pass = 0; pass < G::PASSES; ++pass) {
                        const int b = pass & 1;
                        if (!(alive = pwait(6 + b))) break;       // Gamma of this pass written
                        issue_inv_y(pass);
                        commit(14 + b);                           // Gamma set b read once these complete
                        if (pass == G::PASSES - 1) commit(8);
                        if (pass == 0 && kt > 0 && !(alive = finish_t(kt - 1))) break;
                    }
                    if (!alive) break;
                    // ---- adjoint of stage 2: dG1 = A2_cos^T B_c + A2_sin^T B_s (A2 read MN-major) -----------
                    if (!(alive = pwait(9))) break;
                    const uint64_t a2t = tc::desc_noswizzle(tab, G::SBO_K2, 128);   // A2 read MN-major: A2^T
                    const uint64_t bcd = tc::desc_noswizzle(bc, 128, 2048), bsd = tc::desc_noswizzle(bs, 128, 2048);
                    if (tc::elect_one()) {
#pragma unroll
                        for (int s = 0; s < 8; ++s) {
                            tc::mma_f16(tmem + kColX, tc::desc_add(a2t, 1536 * s), tc::desc_add(bcd, 256 * s), idescx,
                                        s > 0 ? 1u : 0u);
                            tc::mma_f16(tmem + kColX, tc::desc_add(a2t, (kXHP / 8) * 128 + 1536 * s),
                                        tc::desc_add(bsd, 256 * s), idescx, 1u);
                        }
                        tc::mma_commit(tc::smem_u32(&s_mbar[10]));
                    }
                    __syncwarp();
                }
                if (alive) alive = finish_t(H - 1);
                if (alive) commit(13);
            }
        }
        __syncwarp();
    } else {
        // ================================ consumer warps ===============================================
        uint32_t ph = 0;   // expected phase parity of each mbarrier, one bit each
        // warp-uniform bounded wait
        auto cwait = [&](int b) -> bool {
            bool ok = !*v_fail && tc::mbar_wait(tc::smem_u32(&s_mbar[b]), (ph >> b) & 1u, kWaitLimit);
            ph ^= 1u << b;
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
        const int m = 32 * q + lane;
        const int x0l = m / N, kx = m % N;
        const int ajx = kx <= N / 2 ? kx : N - kx;
        bool ok = cwait(0);
        if (ok) tcs::d1_to_b2<N, kFmt>(tmem, s_b2, q, lane, grp, 4);
        tc::fence_async_smem();
        arrive(5);
        ok = cwait(0);
        if (ok && grp < 2) tcs::d2_to_a3<N, kFmt>(tmem, s_are, s_aim, q, lane, grp);
        arrive(4);
        // this lane's Eq. 1 weights for (k_t, |k_x|), in pairs of |k_y| (2 kk, 2 kk + 1) for packed FP32; those
        // of the next tile are read before the tile boundary's waits, which then cover the loads
        constexpr int HP = (H + 1) / 2;
        float2 wt[3][HP];
        auto load_wt = [&](int kt) {
#pragma unroll
            for (int kk = 0; kk < HP; ++kk) {
                const float* w = s_wt + ((kt * H + ajx) * H + 2 * kk) * 3;
                const bool two = 2 * kk + 1 < H;
                wt[0][kk] = make_float2(w[0], two ? w[3] : 0.f);
                wt[1][kk] = make_float2(w[1], two ? w[4] : 0.f);
                wt[2][kk] = make_float2(w[2], two ? w[5] : 0.f);
            }
        };
        load_wt(0);
        for (int kt = 0; kt < H; ++kt) {
#pragma unroll
            for (int pass = 0; pass < G::PASSES; ++pass) {
                const int b = pass & 1;
                // Gamma set b is rewritten only once the adjoint-y MMAs that read it two passes ago completed
                const bool full = cwait(b);
                const bool set_free = kt * G::PASSES + pass < 2 || cwait(14 + b);
                if (full && set_free) {
                    float v[32];
                    tc::tmem_ld32(tmem + lane_base + (uint32_t)(128 * b + 32 * grp), v);
#pragma unroll
                    for (int o = 0; o < G::OPC; ++o) {
                        const int j = grp * G::OPC + o;
                        const int y0 = pass * G::OPP + j;
                        const int gi = x0l * kBY + y0;
                        const float g0 = s_ge[gi], g1 = s_ge[P * kBY + gi], g2 = s_ge[2 * P * kBY + gi];
                        const float thr = kKinkTau * s_l1[gi];
                        const float thr2 = fmaxf(thr * thr, 1e-30f);
                        // rho of |k_y| = 2 kk, 2 kk + 1 (packed; sigma folded into the three gE factors)
                        const float2 gs0 = make_float2(sigma_op * g0, sigma_op * g0);
                        const float2 gs1 = make_float2(sigma_op * g1, sigma_op * g1);
                        const float2 gs2 = make_float2(sigma_op * g2, sigma_op * g2);
                        float2 rho[HP];
#pragma unroll
                        for (int kk = 0; kk < HP; ++kk)
                            rho[kk] = __ffma2_rn(gs0, wt[0][kk], __ffma2_rn(gs1, wt[1][kk], __fmul2_rn(gs2, wt[2][kk])));
                        auto rho_of = [&](int k) -> float {
                            const int a = k <= N / 2 ? k : N - k;
                            return (a & 1) ? rho[a / 2].y : rho[a / 2].x;
                        };
                        // bins (2j, 2j+1) in packed FP32 pairs (two rounded operations per instruction).  The
                        // kink band as a 0/1 factor: |F|^2 carries 1e-30 (far below every band) so that the
                        // reciprocal square root stays finite where the factor is 0
                        const float2 tiny = make_float2(1e-30f, 1e-30f);
                        float gr[N], gim[N];
#pragma unroll
                        for (int j = 0; j < N / 2; ++j) {
                            const int k0 = 2 * j, k1 = 2 * j + 1;
                            const float2 re = make_float2(v[o * G::N3 + k0], v[o * G::N3 + k1]);
                            const float2 im = make_float2(v[o * G::N3 + N + k0], v[o * G::N3 + N + k1]);
                            const float2 r = make_float2(rho_of(k0), rho_of(k1));
                            float2 sc = r;
                            if (!EN) {
                                const float2 m2 = __ffma2_rn(re, re, __ffma2_rn(im, im, tiny));
                                const float2 on = make_float2(m2.x > thr2 ? 1.f : 0.f, m2.y > thr2 ? 1.f : 0.f);
                                sc = __fmul2_rn(__fmul2_rn(r, on), make_float2(fast_rsqrt(m2.x), fast_rsqrt(m2.y)));
                            }
                            const float2 a = __fmul2_rn(sc, re), c = __fmul2_rn(sc, im);
                            gr[k0] = a.x;
                            gr[k1] = a.y;
                            gim[k0] = c.x;
                            gim[k1] = c.y;
                        }
                        // pair coefficients of bins k and n - k (same twiddles up to the sign of the sine):
                        // re part [A_r | B_i], im part [A_i | B_r], A = G[k] + G[n-k], B = G[k] - G[n-k]
                        float pr[G::PK], pi[G::PK];
#pragma unroll
                        for (int k = 0; k < H; ++k) {
                            const bool self = k == 0 || 2 * k == N;
                            pr[k] = self ? gr[k] : gr[k] + gr[N - k];
                            pi[k] = self ? gim[k] : gim[k] + gim[N - k];
                            if (!self) {
                                pr[H - 1 + k] = gim[k] - gim[N - k];
                                pi[H - 1 + k] = gr[k] - gr[N - k];
                            }
                        }
                        // K-major operand: byte(m, k) = (m/8) SBO_G + (k/8) 128 + (m%8) 16 + (k%8) 2, k = [re | im]
                        unsigned char* dst = s_g + b * G::GSET_B + j * G::SLOT_B + (m / 8) * G::SBO_G + (m % 8) * 16;
#pragma unroll
                        for (int c = 0; c < G::PK / 8; ++c) {
                            uint4 wr, wi;
                            wr.x = Pack<kFmt>::two(pr[8 * c + 0], pr[8 * c + 1]);
                            wr.y = Pack<kFmt>::two(pr[8 * c + 2], pr[8 * c + 3]);
                            wr.z = Pack<kFmt>::two(pr[8 * c + 4], pr[8 * c + 5]);
                            wr.w = Pack<kFmt>::two(pr[8 * c + 6], pr[8 * c + 7]);
                            wi.x = Pack<kFmt>::two(pi[8 * c + 0], pi[8 * c + 1]);
                            wi.y = Pack<kFmt>::two(pi[8 * c + 2], pi[8 * c + 3]);
                            wi.z = Pack<kFmt>::two(pi[8 * c + 4], pi[8 * c + 5]);
                            wi.w = Pack<kFmt>::two(pi[8 * c + 6], pi[8 * c + 7]);
                            *reinterpret_cast<uint4*>(dst + c * 128) = wr;
                            *reinterpret_cast<uint4*>(dst + (G::PK / 8 + c) * 128) = wi;
                        }
                    }
                }
                tc::fence_async_smem();
                arrive(2 + b);   // buffer b read (released only now: an earlier release costs registers)
                arrive(6 + b);   // Gamma set b written
            }
            if (kt + 1 < H) {
                load_wt(kt + 1);
                // stage 2 of kt + 1 done (and with it every stage-3 MMA of kt): A3 may be rewritten
                ok = cwait(0);
                if (ok && grp < 2) tcs::d2_to_a3<N, kFmt>(tmem, s_are, s_aim, q, lane, grp);
                arrive(4);
            }
            // ---- dG2 (all adjoint-y MMAs of kt done) -> B_c | B_s (FP16, MN-major [K = m][N = 64]) -------
            if (cwait(8)) {
                // warp group grp: columns 16 grp .. 16 grp + 15 of (re y 0..31 | im y 0..31) -> B_c at the same
                // columns, B_s at the other half (re -> the im slot, im -> the re slot, negated)
                float v[16];
                tc::tmem_ld16(tmem + lane_base + kColY + (uint32_t)(16 * grp), v);
                const float sgn = grp < 2 ? 1.f : -1.f;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int n = 16 * grp + 8 * h, ns = (n + 32) % 64;
                    uint4 w, ws;
                    w.x = Pack<kFmt>::two(v[8 * h + 0], v[8 * h + 1]);
                    w.y = Pack<kFmt>::two(v[8 * h + 2], v[8 * h + 3]);
                    w.z = Pack<kFmt>::two(v[8 * h + 4], v[8 * h + 5]);
                    w.w = Pack<kFmt>::two(v[8 * h + 6], v[8 * h + 7]);
                    ws.x = Pack<kFmt>::two(sgn * v[8 * h + 0], sgn * v[8 * h + 1]);
                    ws.y = Pack<kFmt>::two(sgn * v[8 * h + 2], sgn * v[8 * h + 3]);
                    ws.z = Pack<kFmt>::two(sgn * v[8 * h + 4], sgn * v[8 * h + 5]);
                    ws.w = Pack<kFmt>::two(sgn * v[8 * h + 6], sgn * v[8 * h + 7]);
                    const size_t row = (size_t)(m / 8) * 128 + (m % 8) * 16;
                    *reinterpret_cast<uint4*>(s_bc + (n / 8) * 2048 + row) = w;
                    *reinterpret_cast<uint4*>(s_bs + (ns / 8) * 2048 + row) = ws;
                }
            }
            tc::fence_async_smem();
            arrive(9);
        }
        // ---- the brick's block of gVext (tensor memory) to scratch [u_t][x][y] --------------------------------
        ok = cwait(13);
        const size_t cta = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        float* blk = blocks + cta * G::BLOCK_FLOATS;
        const float out_scale = EN ? (float)(N * N * N) * scale / (sigma * kDxScale) : 1.f / (sigma * kDxScale);
        for (int i = grp; i < G::NB1; i += 4) {
            float v[16];
            if (ok) tc::tmem_ld16(tmem + lane_base + kColT + (uint32_t)(16 * i), v);
            const int pos = 128 * i + m, x = pos / YP, y = pos % YP;
            if (x < XH && y < YH) {
#pragma unroll
                for (int u = 0; u < N; ++u) blk[u * G::SLICE + x * YH + y] = ok ? v[u] * out_scale : 0.f;
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

template <int N>
cudaError_t prepare_n() {
    cudaError_t e = cudaFuncSetAttribute(k5_spectra_adjoint_tc<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)BtGeo<N>::SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k5_spectra_adjoint_tc<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)BtGeo<N>::SMEM);
}

template <int N>
cudaError_t tables_n(const TwiddleTable& t, int feat, void* dst, cudaStream_t s) {
    k5_tc_tables<N><<<1, 256, 0, s>>>(f32::make_tw<N>(t), static_cast<unsigned char*>(dst), feat);
    note_launches(1);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_n(const TwiddleTable& t, const void* tables, const float* V, const float* gE, float* blocks, int T,
                     int X, int Y, int bnd, int feat, int t_begin, int t_step, int t_count, const float* Vt, int Yt,
                     int* err, cudaStream_t s) {
    using G = BtGeo<N>;
    dim3 grid((Y + kBY - 1) / kBY, (X + G::P - 1) / G::P, t_count);
    const unsigned char* tab = static_cast<const unsigned char*>(tables);
    CUtensorMap tmap;
    const int smode = tcs::brick_stage_mode<N>(V, T, X, Y, &tmap, false, Vt, Yt);
    if (feat == 1)
        k5_spectra_adjoint_tc<N, true><<<grid, kThreads, G::SMEM, s>>>(V, gE, blocks, T, X, Y, bnd, t_begin, t_step,
                                                                       tab, f32::make_tw<N>(t), err, tmap, smode);
    else
        k5_spectra_adjoint_tc<N, false><<<grid, kThreads, G::SMEM, s>>>(V, gE, blocks, T, X, Y, bnd, t_begin, t_step,
                                                                        tab, f32::make_tw<N>(t), err, tmap, smode);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t spectra_adjoint_tc_prepare(int n, int fmt) {
    if (fmt != 0) return cudaErrorInvalidValue;  // built with FP16 operands only
    if (n == 8) return prepare_n<8>();
    if (n == 16) return prepare_n<16>();
    return cudaErrorInvalidValue;
}

size_t spectra_adjoint_tc_tables_bytes(int n) {
    if (n == 8) return BtGeo<8>::TAB5_B;
    if (n == 16) return BtGeo<16>::TAB5_B;
    return 0;
}

cudaError_t spectra_adjoint_tc_tables_build(int n, const TwiddleTable& tw, int feat, void* dst, cudaStream_t s) {
    if (n == 8) return tables_n<8>(tw, feat, dst, s);
    if (n == 16) return tables_n<16>(tw, feat, dst, s);
    return cudaErrorInvalidValue;
}

SpectraAdjointGeometry spectra_adjoint_tc_geometry(int n) {
    if (n == 8) return {kBY, BtGeo<8>::YH, BtGeo<8>::P, BtGeo<8>::XH, BtGeo<8>::BLOCK_FLOATS, BtGeo<8>::SLICE};
    if (n == 16) return {kBY, BtGeo<16>::YH, BtGeo<16>::P, BtGeo<16>::XH, BtGeo<16>::BLOCK_FLOATS, BtGeo<16>::SLICE};
    return {0, 0, 0, 0, 0, 0};
}

cudaError_t spectra_adjoint_tc_launch(int n, int fmt, const TwiddleTable& tw, const void* tables, const float* V,
                                      const float* gE, float* blocks, int T, int X, int Y, int bnd, int feat,
                                      int t_begin, int t_step, int t_count, const float* Vt, int Yt, int* err,
                                      cudaStream_t s) {
    if (fmt != 0 || t_step < 1) return cudaErrorInvalidValue;
    if (n == 8)
        return launch_n<8>(tw, tables, V, gE, blocks, T, X, Y, bnd, feat, t_begin, t_step, t_count, Vt, Yt, err, s);
    if (n == 16)
        return launch_n<16>(tw, tables, V, gE, blocks, T, X, Y, bnd, feat, t_begin, t_step, t_count, Vt, Yt, err, s);
    return cudaErrorInvalidValue;
}

}  // namespace sal
