// Shared pieces of the tensor-core forms of the local-spectrum kernels (K1-TC forward, K5-TC adjoint):
// brick geometry, 16-bit packing, twiddles of any bin, the constant operands in their shared-memory
// layouts, the staging of the halo brick as the stage-1 A operand (Eq. 2 applied separably), and the
// scatter of the stage-1 result into one stage-2 B operand per k_t.
//
// CTA brick: t0, x0 in [xb, xb + P) with P = 128/n, y0 in [yb, yb + 16).  Positions of the halo are
// pos = x * YP + y (x < 24, y < YP = 8 ceil(YH / 8)).
//   stage 1 (t), once for all k_t:  D1[pos][c] = sum_u V[t0-n/2+u][x][y] T1[u][c],
//            c = [cos k_t = 0..n/2 | sin k_t = 1..n/2-1]; A = the brick scaled by 1/max|V| and
//            rounded to 16 bits (MN-major: 8 consecutive y per 16-byte row), one MMA per 128 positions.
//            G1 = P - iQ is scattered into one stage-2 B operand per k_t:
//            B2[(re|im, y)][(cos|sin, x)] = [[G1r, G1i], [G1i, -G1r]].
//   stage 2 (x), per k_t:  D2[(x0, k_x)][(re|im, y)] = sum_x A2[(x0, k_x)][(cos|sin, x)] B2,
//            A2 = the Toeplitz twiddles h(x - x0) [cos | sin](2 pi k_x (x - x0) / n): the sliding
//            window along x is built into A2.  D2 is rounded to 16 bits into the stage-3 A operands
//            (real, imaginary), MN-major with 16-byte K rows: the window of output y0 is the same
//            descriptor moved by 16 y0 bytes.
//   stage 3 (y), per output y0:  D3[(x0, k_x)][(re|im, k_y)] = Are(y0) B3a + Aim(y0) B3b,
//            B3a = [c | -s], B3b = [s | c] over all k_y: the accumulator holds Re F and Im F.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "spectra_f32_common.cuh"
#include "tc_sm100.cuh"

namespace sal {
namespace tcs {

using f32::Tw;

constexpr int kBY = 16;                 // outputs per CTA along y
constexpr int kKRows = kBY + 15;        // K rows of the stage-3 A operand: window start + 16 taps
constexpr int kXHP = 24;                // halo rows along x staged (>= P + n - 1, multiple of 8)
constexpr int kK2 = 2 * kXHP;           // stage-2 K: 24 cos taps + 24 sin taps
constexpr uint32_t kWaitLimit = 1u << 22;

template <int N> struct FwdGeo {
    static constexpr int H = N / 2 + 1;
    static constexpr int P = 128 / N;          // x0 positions per CTA
    static constexpr int XH = P + N - 1;       // x extent of the halo
    static constexpr int YH = kBY + N - 1;     // y extent of the halo
    static constexpr int YG = (YH + 7) / 8;
    static constexpr int YP = 8 * YG;          // y positions per halo row
    static constexpr int NB1 = (kXHP * YP + 127) / 128;   // stage-1 MMAs (128 positions each)
    static constexpr int N2 = 2 * YP;          // stage-2 N: re | im over y
    static constexpr int N3 = 2 * N;           // stage-3 N per output: re | im over k_y
    static constexpr int OPC = 32 / N3;        // outputs per 32-column tensor-memory chunk (1 or 2)
    static constexpr int OPP = 128 / N3;       // outputs per pass (one 128-column buffer)
    static constexpr int PASSES = kBY / OPP;   // 4 (n = 16) or 2 (n = 8), alternating buffers
    static constexpr uint32_t SBO_A3 = kKRows * 16;
    static constexpr uint32_t SBO_K2 = kK2 / 8 * 128;    // 8-row group stride of the K-major A2 / B2
    static constexpr size_t A1_B = (size_t)NB1 * 4096;
    static constexpr size_t B2_B = (size_t)N2 / 8 * SBO_K2;   // one k_t tile
    static constexpr size_t B2ALL_B = (size_t)H * B2_B;
    static constexpr size_t R0_B = ((A1_B > B2ALL_B ? A1_B : B2ALL_B) + 127) / 128 * 128;  // A1, then B2 tiles
    // forward constant operands: [A2 | B1 | B3a | B3b | Eq. 1 weight table]
    static constexpr size_t A2_B = (size_t)16 * SBO_K2;
    static constexpr size_t B3_B = (size_t)N3 / 8 * 256;
    static constexpr size_t WT_B = ((size_t)H * H * H * 3 * 4 + 15) / 16 * 16;
    static constexpr size_t TAB_B1 = A2_B;
    static constexpr size_t TAB_B3A = TAB_B1 + 512;
    static constexpr size_t TAB_B3B = TAB_B3A + B3_B;
    static constexpr size_t TAB_WT = TAB_B3B + B3_B;
    static constexpr size_t TAB_B = TAB_WT + WT_B;
    static constexpr size_t A3_B = (size_t)16 * SBO_A3;
    static constexpr int STAGE_ITEMS = 16 * NB1 * 16;   // (u, 8-position group) items of the A1 fill
    // FP32 landing area of an interior brick's TMA copies, at the end of region 0 (the stage-1 A operand,
    // written after every thread has read its samples, may overlap it): one tensor box [u][x][YP y], or
    // one bulk copy per (u, x) row of RB = YP + 4 floats from the 16-byte boundary at or below its start
    static constexpr int RB = YP + 4;
    static constexpr size_t STG_TENSOR_B = (size_t)N * XH * YP * 4;
    static constexpr size_t STG_ROWS_B = (size_t)N * XH * RB * 4;
    static constexpr size_t STG_B = STG_TENSOR_B > STG_ROWS_B ? STG_TENSOR_B : STG_ROWS_B;
    static constexpr size_t STG_OFF = (R0_B - STG_B) / 128 * 128;
    static_assert(XH <= kXHP && YH <= 32 && YP <= 32, "halo");
    static_assert(2 * H - 2 <= 16, "stage-1 columns");
    static_assert(N2 <= 128, "stage-2 accumulator");
    static_assert(PASSES * OPP == kBY && PASSES % 2 == 0, "passes");
    static_assert(TAB_B % 16 == 0 && A3_B % 16 == 0, "bulk copy alignment");
    static_assert(STG_B <= R0_B && (RB * 4) % 16 == 0 && (YP * 4) % 16 == 0, "TMA landing area");
};

// How the interior bricks of a launch reach shared memory (bricks whose halo leaves the volume always take
// the SIMT loads, which apply the border extension): SIMT loads; one tiled tensor copy per brick (a 3-D
// tensor map over V, usable when a row of V is a multiple of 16 bytes); or one bulk copy per (u_t, x)
// row of the brick (any row length).  Both copies run on the TMA unit, plain (no multicast).
enum : int { kStageSimt = 0, kStageTensor = 1, kStageRows = 2 };

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

// The forward constant operands of one (n, operand type) into `out` (TAB_B bytes): A2 (Toeplitz
// stage-2 twiddles, K-major), B1 (stage-1 twiddles), B3a / B3b (stage-3 twiddles), the Eq. 1 weight
// table [k_t][|k_x|][|k_y|][3] (r_m, or r_m^2 for the energy reading feat = 1, with the k_t multiplicity
// and the 1/n^3 of the mean folded in).
template <int N, int FMT>
__device__ void build_fwd_tables(const Tw<N>& tw, unsigned char* out, int tid, int nt, int feat) {
    using G = FwdGeo<N>;
    constexpr int H = G::H;
    unsigned char* a2 = out;
    unsigned char* b1 = out + G::TAB_B1;
    unsigned char* b3a = out + G::TAB_B3A;
    unsigned char* b3b = out + G::TAB_B3B;
    float* wt = reinterpret_cast<float*>(out + G::TAB_WT);
    // B1[c][u]: c < H: cos k_t = c; H <= c < 2H-2: sin k_t = c-H+1.  byte = (c/8)256 + (u/8)128 + (c%8)16 + (u%8)2
    for (int i = tid; i < 256; i += nt) {
        const int c = i / 16, u = i % 16;
        float v = 0.f;
        if (c < H) v = twc<N>(tw, c, u);
        else if (c < 2 * H - 2) v = tws<N>(tw, c - H + 1, u);
        *reinterpret_cast<uint16_t*>(b1 + (c / 8) * 256 + (u / 8) * 128 + (c % 8) * 16 + (u % 8) * 2) =
            Pack<FMT>::one(v);
    }
    // B3a[ncol][u] = [c | -s], B3b[ncol][u] = [s | c] over k_y = ncol % n (K-major, K = u)
    for (int i = tid; i < G::N3 * 16; i += nt) {
        const int ncol = i / 16, u = i % 16, k = ncol % N;
        const bool re = ncol < N;
        const float c = twc<N>(tw, k, u), sn = tws<N>(tw, k, u);
        const size_t off = (ncol / 8) * 256 + (u / 8) * 128 + (ncol % 8) * 16 + (u % 8) * 2;
        *reinterpret_cast<uint16_t*>(b3a + off) = Pack<FMT>::one(re ? c : -sn);
        *reinterpret_cast<uint16_t*>(b3b + off) = Pack<FMT>::one(re ? sn : c);
    }
    // A2[(x0l, k_x)][k2]: k2 < 24: cos, else sin, of (k_x, x - x0l) with x = k2 % 24 (K-major)
    for (int i = tid; i < 128 * kK2; i += nt) {
        const int m = i / kK2, k2 = i % kK2;
        const int x0l = m / N, kx = m % N, x = k2 % kXHP, u = x - x0l;
        const float v = k2 < kXHP ? twc<N>(tw, kx, u) : tws<N>(tw, kx, u);
        *reinterpret_cast<uint16_t*>(a2 + (m / 8) * G::SBO_K2 + (k2 / 8) * 128 + (m % 8) * 16 + (k2 % 8) * 2) =
            Pack<FMT>::one(v);
    }
    for (int i = tid; i < H * H * H; i += nt) {
        const int k = i % H, aj = (i / H) % H, kt = i / (H * H);
        const float mult = (kt == 0 || 2 * kt == N) ? 1.f : 2.f;
        float w0, w1, w2;
        if (feat == 1) f32::bin_weights<true>(kt, aj, k, mult / (float)(N * N * N), w0, w1, w2);
        else f32::bin_weights<false>(kt, aj, k, mult / (float)(N * N * N), w0, w1, w2);
        wt[i * 3 + 0] = w0;
        wt[i * 3 + 1] = w1;
        wt[i * 3 + 2] = w2;
    }
}

// Host: the staging mode of a launch over V [T][X][Y] and, for kStageTensor, its tensor map (3-D, dims
// {Y, X, T}, box {YP, XH, n} floats, no swizzle, no multicast).  A tensor map needs 16-byte row strides
// (Y a multiple of 4); other row lengths take the row copies; a V not 16-byte aligned the SIMT loads.
// allow_rows = false: a kernel whose brick staging is not hidden by a second CTA on the SM (the adjoint)
// takes the SIMT loads instead of the row copies, whose many small transfers cost it more than the loads.
// Vt, Yt: a row-padded copy of V (Yt >= Y, a multiple of 4): the tensor map then reads the copy, and every
// interior brick takes one tensor copy whatever Y is (the border bricks keep the SIMT loads from V).
template <int N>
inline int brick_stage_mode(const float* V, int T, int X, int Y, CUtensorMap* tmap, bool allow_rows,
                            const float* Vt = nullptr, int Yt = 0) {
    using G = FwdGeo<N>;
    *tmap = CUtensorMap{};
    const int rows = allow_rows ? kStageRows : kStageSimt;
    // the tensor map reads the row-padded copy when there is one (same samples, rows of Yt floats)
    const float* src = Vt ? Vt : V;
    const int ys = Vt ? Yt : Y;
    if (Vt && (ys < Y || (ys & 3) != 0)) return kStageSimt;
    if ((reinterpret_cast<uintptr_t>(src) & 15) != 0) return kStageSimt;
    if ((ys & 3) != 0) return rows;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }();
    if (!encode) return rows;
    const cuuint64_t dims[3] = {(cuuint64_t)Y, (cuuint64_t)X, (cuuint64_t)T};
    const cuuint64_t strides[2] = {(cuuint64_t)ys * 4, (cuuint64_t)X * ys * 4};
    const cuuint32_t box[3] = {(cuuint32_t)G::YP, (cuuint32_t)G::XH, (cuuint32_t)N};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode(tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(src), dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? kStageTensor : rows;
}

// Whether the brick at (t0, xb, yb) is staged by the TMA unit in mode `smode`: its halo (YP samples per
// row) lies inside the volume; the row copies also must not read past the end of V (each reads up to
// 3 samples beyond its row's halo).
template <int N>
__device__ __forceinline__ bool tma_brick(int smode, int T, int X, int Y, int t0, int xb, int yb) {
    using G = FwdGeo<N>;
    const int ty = yb - N / 2;
    const bool inside = t0 - N / 2 >= 0 && t0 + N / 2 <= T && xb - N / 2 >= 0 && xb - N / 2 + G::XH <= X &&
                        ty >= 0 && ty + G::YP <= Y;
    if (smode == kStageTensor) return inside;
    if (smode != kStageRows || !inside) return false;
    const size_t last = ((size_t)(t0 + N / 2 - 1) * X + (xb - N / 2 + G::XH - 1)) * Y + ty + G::YP + 3;
    return last < (size_t)T * X * Y;
}

// Issue of an interior brick's TMA copies into s_stage, completion counted on mbar (initialised with one
// arrival); one warp, all lanes.  Lane 0 sets the expected byte count before any copy is issued.
template <int N>
__device__ void stage_issue(int smode, const CUtensorMap* tmap, const float* __restrict__ V, int X, int Y, int t0,
                            int xb, int yb, unsigned char* s_stage, uint32_t mbar, int lane) {
    using G = FwdGeo<N>;
    const int ty = yb - N / 2;
    if (lane == 0)
        tc::mbar_arrive_expect_tx(mbar, (uint32_t)(smode == kStageTensor ? G::STG_TENSOR_B : G::STG_ROWS_B));
    __syncwarp();
    if (smode == kStageTensor) {
        if (lane == 0) tc::tma_load_3d(tc::smem_u32(s_stage), tmap, ty, xb - N / 2, t0 - N / 2, mbar);
    } else {
        for (int r = lane; r < N * G::XH; r += 32) {
            const int u = r / G::XH, x = r % G::XH;
            const size_t f = ((size_t)(t0 - N / 2 + u) * X + (xb - N / 2 + x)) * Y + ty;
            tc::bulk_g2s(tc::smem_u32(s_stage + (size_t)r * G::RB * 4), V + (f & ~(size_t)3), (uint32_t)(G::RB * 4),
                         mbar);
        }
    }
}

// The halo brick as the 16-bit stage-1 A operand, scaled by 1/max|V|; returns max|V| (1 for an all-zero
// brick).  item = (u, g): 8 positions pos = 8g .. 8g+7 (x = g / YG, y = 8 (g % YG) + i) at tap u.
// Bricks staged by the TMA unit (tma_brick; stage_issue has issued their copies) read their samples from
// s_stage once mbar completes (a bounded wait: on timeout the error word and *s_fail are set and the
// brick is taken as zero); the others load them from V, applying the border extension.  Contains one
// __syncthreads.
template <int N, int FMT, int NT>
__device__ float stage_brick(const float* __restrict__ V, int T, int X, int Y, int bnd, int t0, int xb, int yb,
                             unsigned char* s_a1, float* s_red, int tid, bool tma, const unsigned char* s_stage,
                             int smode, uint32_t mbar, int* err, int* s_fail) {
    using G = FwdGeo<N>;
    constexpr int XH = G::XH, YH = G::YH, YG = G::YG, YP = G::YP;
    constexpr int PER = (G::STAGE_ITEMS + NT - 1) / NT;
    const int lane = tid & 31, warp = tid >> 5;
    const int ty = yb - N / 2;
    bool landed = false;
    if (tma) {
        landed = tc::mbar_wait(mbar, 0, kWaitLimit);
        if (!landed) {
            atomicOr(err, 1);
            atomicExch(s_fail, 1);
        }
    }
    const float* stg = reinterpret_cast<const float*>(s_stage);
    const bool interior = t0 - N / 2 >= 0 && t0 + N / 2 <= T && xb - N / 2 >= 0 && xb - N / 2 + XH <= X && ty >= 0 &&
                          ty + YP <= Y;
    float vals[PER][8];
    float vmax = 0.f;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const int item = tid + r * NT;
        const int u = item / (G::NB1 * 16), g = item % (G::NB1 * 16);
        const int x = g / YG, y8 = 8 * (g % YG);
        const bool live = item < G::STAGE_ITEMS && u < N && x < XH;
#pragma unroll
        for (int i = 0; i < 8; ++i) vals[r][i] = 0.f;
        if (tma) {
            if (live && landed) {
                if (smode == kStageTensor) {
                    // rows of YP floats from a 128-byte aligned base: two 16-byte reads
                    const float4* row = reinterpret_cast<const float4*>(stg + (size_t)(u * XH + x) * YP + y8);
                    const float4 a = row[0], b = row[1];
                    vals[r][0] = a.x; vals[r][1] = a.y; vals[r][2] = a.z; vals[r][3] = a.w;
                    vals[r][4] = b.x; vals[r][5] = b.y; vals[r][6] = b.z; vals[r][7] = b.w;
                } else {
                    const size_t f = ((size_t)(t0 - N / 2 + u) * X + (xb - N / 2 + x)) * Y + ty;
                    const float* row = stg + (size_t)(u * XH + x) * G::RB + (f & 3);
#pragma unroll
                    for (int i = 0; i < 8; ++i) vals[r][i] = row[y8 + i];
                }
            }
        } else if (interior) {
            // the halo inside the volume: direct loads, no border extension
            if (live) {
                const float* src = V + ((size_t)(t0 - N / 2 + u) * X + (xb - N / 2 + x)) * Y + ty + y8;
#pragma unroll
                for (int i = 0; i < 8; ++i) vals[r][i] = __ldg(src + i);
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
    for (int w = 0; w < NT / 32; ++w) bmax = fmaxf(bmax, s_red[w]);
    const float scale = bmax > 0.f ? bmax : 1.f;
    const float inv_scale = 1.f / scale;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const int item = tid + r * NT;
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
    return scale;
}

// D1 (tensor memory columns [16 i, 16 i + 16) of stage-1 block i) -> one stage-2 B tile per k_t.
// Blocks i = grp, grp + ngrp, ... are read by the warps of group grp (lane quarter q).
template <int N, int FMT>
__device__ void d1_to_b2(uint32_t tmem, unsigned char* s_b2, int q, int lane, int grp, int ngrp) {
    using G = FwdGeo<N>;
    constexpr int H = G::H, YP = G::YP;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    for (int i = grp; i < G::NB1; i += ngrp) {
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

// D2 (tensor memory columns [0, N2)) -> the stage-3 A operands: part 0 = real columns, 1 = imaginary.
template <int N, int FMT>
__device__ void d2_to_a3(uint32_t tmem, unsigned char* s_are, unsigned char* s_aim, int q, int lane, int part) {
    using G = FwdGeo<N>;
    float v[32];
    tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(part * G::YP), v);
    const int m = 32 * q + lane;
    unsigned char* dst = (part ? s_aim : s_are) + (m / 8) * G::SBO_A3 + (m % 8) * 2;
#pragma unroll
    for (int y = 0; y < G::YH; ++y) *reinterpret_cast<uint16_t*>(dst + y * 16) = Pack<FMT>::one(v[y]);
    tc::fence_async_smem();
}

}  // namespace tcs
}  // namespace sal
