// K5-F32: adjoint of the local-spectrum feature step (the backward of Sec. 2 steps 1-3).
//
// For L = sum_p sum_m gE_m[p] E_m[p] with E_m[p] = sum_{k in half} wt_m(k) |F_p[k]| (wt holds
// r_m of Eq. 1, the Hermitian multiplicity of k_t and 1/n^3), the gradient with respect to the
// (extended) input is
//   gVext[p + u - n/2] += Re sum_{k in half} h(u) exp(+2 pi i k.u / n) Gamma_p[k],
//   Gamma_p[k] = (sum_m gE_m[p] wt_m(k)) F_p[k] / |F_p[k]|,
// with Gamma = 0 at DC and where F_p[k] = 0 (|F| has no direction there: the zero subgradient), i.e. the
// transposes of the three sliding DFT stages applied to Gamma in reverse order.
//
// The direction F / |F| is ill-conditioned for small |F|: FP32 computes F to about 2^-26 of the window's
// L1 norm A_p = sum_u |h(u) Vext[p + u - n/2]| (which bounds every |F_p[k]|), so a bin with |F| near that
// level has no usable FP32 direction.  Such bins are resolved exactly:
//   - bins that vanish for every input, because the border extension makes the coefficient of every
//     source sample of one axis vanish (a mirror-symmetric window along an axis zeroes its Nyquist bin,
//     a window folded onto few samples zeroes more), are found on the host by integer arithmetic on the
//     window's index map (axis_vanish_mask) and take Gamma = 0;
//   - every other bin with FP32 |F| <= 2^-16 A_p and a non-zero weight is recomputed by one warp as a
//     direct sum over its cube in float-float arithmetic (pairs of FP32 values, error about 2^-46 A_p;
//     resolve_small_bins), and takes Gamma = 0 if |F| <= 2^-36 A_p, else its float-float direction.
// Bins above 2^-16 A_p carry an FP32 direction error of at most about 2^-10.
// Spectra are recomputed brick by brick (the forward stages of K1), never stored.
//
// One CTA = one brick (t0, x0, y_start .. y_start+BY-1), same mapping as K1:
//   1. stage brick, forward stages 1 and 2 (shared with K1);
//   2. per (row, y0): forward stage 3 -> Gamma -> inverse DFT along y (pairing k, n-k), added
//      into a private accumulation window of the thread (thread-interleaved shared memory); for the rect
//      cube at n = 8, 16 both y-passes slide over the thread's run of outputs (see SL below);
//   3. windows of the y-chunks summed into Gamma_G2[k_t][k_x][y];
//   4. adjoint of stage 2 (x) -> Gamma_G1[k_t][u_x][y];
//   5. adjoint of stage 1 (t), real part -> the brick's block [u_t][u_x][y] of gVext, written to
//      scratch; a separate gather kernel sums the overlapping blocks in a fixed order.
#include "spectra_f32_common.cuh"

namespace sal {
namespace {

using f32::Tw;

constexpr float kSmallBin = 1.0f / 65536.0f;       // FP32 |F| / A_p at or below which a bin is resolved exactly
constexpr float kZeroBin = 1.0f / 68719476736.0f;  // float-float max(|Re F|, |Im F|) / A_p at or below which F = 0
constexpr int kListQ = 32;   // small bins a CTA may hand to the listed-bin passes (more: it resolves them itself)
// Layout of the listed-bin scratch of one launch of ncta CTAs (ints): [0] the number of listed bins, [4 ..)
// the work list (cta << 5 | entry, in no particular order), then per CTA kListStride ints: [0] its count,
// [1 .. Q] its entries (owner | output << 10 | bin << 14, in the in-kernel resolve's order), [1 + Q ..) the
// (Re, Im) of each entry's Gamma, written by the exact pass.
constexpr int kListStride = 1 + 3 * kListQ;
__host__ __device__ constexpr size_t list_cta_offset(long long ncta) { return 4 + (size_t)ncta * kListQ; }

// Float-float constants of the exact recompute: cos, sin of 2 pi m / n and the taper h(u), each as a pair
// (hi, lo) of FP32 values whose sum is the double-precision value.
template <int N> struct Exact2f {
    float ch[N], cl[N], sh[N], sl[N], hh[N], hl[N];
};

// Masks of the bins that vanish for every input, per axis (t, x, y): bit k of the mask of position p
// (the cube's samples p - n/2 .. p + n/2 - 1 of that axis) is set when bin k of that axis vanishes.
// Positions whose cube lies inside the axis never vanish; the others are p < n (entries 0 .. n-1) and
// p >= L - n (entries n .. 2n-1).
struct VanishTab {
    uint16_t m[3][32];
    int L[3];
};

__device__ __forceinline__ uint32_t vanish_mask(const VanishTab& v, int a, int p, int n) {
    const int L = v.L[a];
    if (p - n / 2 >= 0 && p + n / 2 - 1 < L) return 0u;
    return p < n ? v.m[a][p] : v.m[a][n + (p - (L - n))];
}

// Host: does bin k of the one-axis cube at position p (axis length L) vanish for every input?  The bin is
// sum_m h(m) w^(k m) x[src(m)] (w = exp(-2 pi i / n)), so it vanishes for all x iff, for each source
// sample j, the coefficient sum_{m: src(m) = j} h(m) w^(k m) is 0.  With n a power of two, w has minimal
// polynomial w^(n/2) + 1, so the coefficient is zero iff its coordinates on w^0 .. w^(n/2-1)
// (w^(e + n/2) = -w^e) are; they are integers for the rect taper (h = 1) and, scaled by 4, for the
// periodic Hann taper (4 h(m) w^(km) = 2 w^(km) - w^(km+m) - w^(km-m)).  Exact: no rounding enters.
inline bool axis_bin_vanishes(int n, int p, int L, int bnd, int taper, int k) {
    if (p - n / 2 >= 0 && p + n / 2 - 1 < L) return false;
    int src[32];
    for (int m = 0; m < n; ++m) src[m] = ext_index(p - n / 2 + m, L, bnd);
    for (int m = 0; m < n; ++m) {
        if (src[m] < 0) continue;
        bool first = true;
        for (int q = 0; q < m; ++q) first = first && src[q] != src[m];
        if (!first) continue;
        int a[16] = {0};
        for (int q = m; q < n; ++q) {
            if (src[q] != src[m]) continue;
            const int e0 = (k * q) % n;
            const int es[3] = {e0, (e0 + q) % n, (e0 - q + n) % n};
            const int vs[3] = {taper ? 2 : 1, taper ? -1 : 0, taper ? -1 : 0};
            for (int r = 0; r < 3; ++r) {
                if (es[r] < n / 2) a[es[r]] += vs[r];
                else a[es[r] - n / 2] -= vs[r];
            }
        }
        for (int e = 0; e < n / 2; ++e)
            if (a[e] != 0) return false;
    }
    return true;
}

inline uint16_t axis_vanish_mask(int n, int p, int L, int bnd, int taper) {
    uint16_t mk = 0;
    for (int k = 0; k < n; ++k)
        if (axis_bin_vanishes(n, p, L, bnd, taper, k)) mk = (uint16_t)(mk | (1u << k));
    return mk;
}

inline VanishTab make_vanish_tab(int n, int T, int X, int Y, int bnd, int taper) {
    VanishTab v{};
    const int L[3] = {T, X, Y};
    for (int a = 0; a < 3; ++a) {
        v.L[a] = L[a];
        for (int p = 0; p < n && p < L[a]; ++p) v.m[a][p] = axis_vanish_mask(n, p, L[a], bnd, taper);
        for (int p = L[a] - n > 0 ? L[a] - n : 0; p < L[a]; ++p)
            v.m[a][n + (p - (L[a] - n))] = axis_vanish_mask(n, p, L[a], bnd, taper);
    }
    return v;
}

// Float-float arithmetic (an unevaluated sum hi + lo of two FP32 values): the error-free transformations
// two-sum (Knuth) and the FMA product residual, with the usual renormalisation.
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ff_fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    return ff_fast_two_sum(s, e + a.lo + b.lo);
}
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ FF ff_mul1(float a, FF b) {   // a exact in FP32
    const float p = a * b.hi;
    return ff_fast_two_sum(p, fmaf(a, b.lo, fmaf(a, b.hi, -p)));
}

template <int N> struct BCfg;
template <> struct BCfg<2>  { static constexpr int BY = 32, YC = 1, MINB = 4; };
template <> struct BCfg<4>  { static constexpr int BY = 32, YC = 2, MINB = 4; };
template <> struct BCfg<8>  { static constexpr int BY = 32, YC = 4, MINB = 2; };
template <> struct BCfg<16> { static constexpr int BY = 16, YC = 8, MINB = 2; };

template <int N> struct BGeo {
    static constexpr int H = N / 2 + 1;
    static constexpr int BY = BCfg<N>::BY;
    static constexpr int YC = BCfg<N>::YC;
    static constexpr int ROWS = H * N;
    static constexpr int NT = ROWS * (BY / YC);
    using B = f32::Brick<N, BY, NT>;
    static constexpr int YH = B::YH;
    static constexpr int WIN = YC + N - 1;                       // private window (complex values)
    static constexpr size_t IN_BYTES = (size_t)B::IN_FLOATS * 4;
    static constexpr size_t G_BYTES = (size_t)B::G_FLOAT2 * 8;
    static constexpr size_t WIN_BYTES = (size_t)NT * WIN * 8;
    static constexpr size_t A0 = IN_BYTES + G_BYTES;
    static constexpr size_t A_BYTES = A0 > WIN_BYTES ? A0 : WIN_BYTES;   // s_in+s_g1 | windows | Gamma_G1
    static constexpr size_t SMALL_OFF = A_BYTES + G_BYTES + (size_t)4 * BY * 4 + (size_t)YH * 4;
    // [YC][NT] uint16 masks of the small bins each thread leaves to the exact recompute, then the source
    // rows of the cube along t and x ([N] + [N] ints, -1 outside a zero-extended volume)
    static constexpr size_t IDX_OFF = (SMALL_OFF + (size_t)YC * NT * 2 + 15) / 16 * 16;
    static constexpr size_t WB_OFF = IDX_OFF + (size_t)2 * N * 4;   // [NT / 32] owners of small bins, per warp
    static constexpr size_t SMEM = WB_OFF + (size_t)(NT / 32 + 1) * 4;   // + the CTA's list decision
    static_assert(N <= 16, "16-bit masks of small bins");
    static constexpr int SLICE = (N * YH + 3) / 4 * 4;           // u_t slices of the block, 16-byte aligned
    static constexpr int BLOCK_FLOATS = N * SLICE;               // scratch block per CTA
    static_assert(BY % YC == 0 && NT <= 1024, "geometry");
};

// The small bins left by step 2 (s_small[yi][owner] bit k_y: output yi of the owner's run, bin k_y of its
// (k_t, k_x) row), each owner's bins by one warp (the owners dealt round-robin to the CTA's warps in thread
// order): the lanes split the n^3 terms of the direct sum
// F = sum_u h(u) Vext[p + u - n/2] w^(k.u) (each lane a fixed u_y, four independent float-float
// accumulators, the loads of four terms issued before their arithmetic) and reduce it; Gamma = rho F / |F|
// (0 if max(|Re F|, |Im F|) <= 2^-36 A_p) and its inverse DFT along y, h(u) Gamma exp(+2 pi i k_y u / n),
// go into the owner's private window.
template <int N, int NT, int YC, int BY, int H, int ROWS>
__device__ __noinline__ void resolve_small_bins(const float* __restrict__ V, int X, int Y, int bnd, int y_start,
                                                int taper, const uint16_t* s_small, const int* s_src, float2* s_win,
                                                const float* s_ge, const float* s_l1,
                                                const float* __restrict__ wtab, const Tw<N>& tw,
                                                const Exact2f<N>& ex, unsigned* s_wbits) {
    constexpr int N3 = N * N * N, PER = N3 >= 32 ? N3 / 32 : 1, STEP = 32 / N;   // terms per lane, (ut, ux) step
    constexpr int U = PER >= 4 ? 4 : PER;                                          // independent accumulators
    const int tid = threadIdx.x, lane = tid & 31;
    // lane's fixed u_y and its first (u_t, u_x) pair: term e = lane + 32 i has u_y = lane % N and
    // (u_t, u_x) = divmod(lane / N + STEP i, N)
    const int uy = lane % N, r0 = lane / N;
    const bool live = lane < N3;   // n = 2: 8 terms, lanes 8.. idle
    // the owners (threads with small bins) in thread order, dealt round-robin to the CTA's warps: an owner's bins
    // are processed by one warp in a fixed order (the same sums in the same order whichever warp it is), and
    // owners that cluster in one warp no longer hold the rest of the CTA at the next barrier
    constexpr int NW = NT / 32;
    const int warp = tid >> 5;
    bool mine = false;
    for (int yi = 0; yi < YC; ++yi) mine = mine || s_small[yi * NT + tid] != 0;
    const unsigned wb = __ballot_sync(0xffffffffu, mine);
    if (lane == 0) s_wbits[warp] = wb;
    __syncthreads();   // every owner's masks and every warp's owner bits visible
    int idx = 0;   // index of the next owner in thread order
    for (int w = 0; w < NW; ++w) {
        unsigned todo = s_wbits[w];
        while (todo) {
            const int o = 32 * w + __ffs(todo) - 1;
            todo &= todo - 1;
            if (idx++ % NW != warp) continue;
            const int row = o % ROWS, kt = row / N, kx = row % N, ych = o / ROWS;
            for (int yi = 0; yi < YC; ++yi) {
                unsigned msk = s_small[yi * NT + o];
                const int yl = ych * YC + yi;
                const int gy = ext_index(y_start + yl - N / 2 + uy, Y, bnd);
                while (msk) {
                    const int ky = __ffs(msk) - 1;
                    msk &= msk - 1;
                    FF re[U], im[U];
    #pragma unroll
                    for (int a = 0; a < U; ++a) re[a] = im[a] = FF{0.f, 0.f};
                    const FF hy = {ex.hh[uy], ex.hl[uy]};
                    for (int i0 = 0; i0 < PER; i0 += U) {
                        float v[U];
                        int ph[U];
                        FF h2[U];
    #pragma unroll
                        for (int a = 0; a < U; ++a) {   // loads first, then the arithmetic
                            const int rr = live ? r0 + STEP * (i0 + a) : 0, ut = rr / N, ux = rr % N;
                            const int gt = s_src[ut], gx = s_src[N + ux];
                            v[a] = (live && (gt | gx | gy) >= 0) ? __ldg(V + ((size_t)gt * X + gx) * Y + gy) : 0.f;
                            ph[a] = (kt * ut + kx * ux + ky * uy) % N;
                            h2[a] = taper ? ff_mul(FF{ex.hh[ut], ex.hl[ut]}, FF{ex.hh[ux], ex.hl[ux]}) : FF{1.f, 0.f};
                        }
    #pragma unroll
                        for (int a = 0; a < U; ++a) {
                            FF c = {ex.ch[ph[a]], ex.cl[ph[a]]}, sn = {-ex.sh[ph[a]], -ex.sl[ph[a]]};
                            if (taper) {
                                const FF h3 = ff_mul(h2[a], hy);
                                c = ff_mul(h3, c);
                                sn = ff_mul(h3, sn);
                            }
                            re[a] = ff_add(re[a], ff_mul1(v[a], c));
                            im[a] = ff_add(im[a], ff_mul1(v[a], sn));
                        }
                    }
    #pragma unroll
                    for (int a = 1; a < U; ++a) {
                        re[0] = ff_add(re[0], re[a]);
                        im[0] = ff_add(im[0], im[a]);
                    }
                    FF fre = re[0], fim = im[0];
    #pragma unroll
                    for (int d = 16; d > 0; d >>= 1) {
                        const FF r2 = {__shfl_xor_sync(0xffffffffu, fre.hi, d), __shfl_xor_sync(0xffffffffu, fre.lo, d)};
                        const FF i2 = {__shfl_xor_sync(0xffffffffu, fim.hi, d), __shfl_xor_sync(0xffffffffu, fim.lo, d)};
                        fre = ff_add(fre, r2);
                        fim = ff_add(fim, i2);
                    }
                    const float mx = fmaxf(fabsf(fre.hi), fabsf(fim.hi));
                    if (mx > kZeroBin * s_l1[yl] && lane < N) {
                        const int k = ky <= N / 2 ? ky : N - ky;
                        const float rho = fmaf(s_ge[yl], __ldg(wtab + k * ROWS + row),
                                               fmaf(s_ge[BY + yl], __ldg(wtab + (H + k) * ROWS + row),
                                                    s_ge[2 * BY + yl] * __ldg(wtab + (2 * H + k) * ROWS + row)));
                        const float fr = fre.hi / mx, fi = fim.hi / mx;      // scaled first: no underflow
                        const float sc = rho / sqrtf(fmaf(fr, fr, fi * fi));
                        const float gr = sc * fr, gi = sc * fi;
                        const int u = lane;
                        const float c = tw.c[k][u], sn = ky <= N / 2 ? tw.s[k][u] : -tw.s[k][u];
                        float2* w = s_win + (yi + u) * NT + o;
                        float2 acc = *w;
                        acc.x += gr * c - gi * sn;
                        acc.y += gr * sn + gi * c;
                        *w = acc;
                    }
                    __syncwarp();
                }
            }
        }
    }
}

// The CTA's small bins as a list for the listed-bin pass: entries (owner, output, bin) in the order the
// in-kernel resolve would take them (owners in thread order, then outputs, then bins), list[0] = their
// count.  Returns (CTA-uniform) whether the list holds them all; a CTA with more than kListQ writes a count
// of 0 and resolves its bins itself.  Contains one __syncthreads.
template <int NT, int YC>
__device__ bool list_small_bins(const uint16_t* s_small, unsigned* s_wbits, int* __restrict__ list,
                                int* __restrict__ work, int* __restrict__ nwork, long long cta) {
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    bool mine = false;
    for (int yi = 0; yi < YC; ++yi) mine = mine || s_small[yi * NT + tid] != 0;
    const unsigned wb = __ballot_sync(0xffffffffu, mine);
    if (lane == 0) s_wbits[warp] = wb;
    __syncthreads();
    if (tid == 0) {
        int cnt = 0;
        for (int w = 0; w < NW; ++w) {
            for (unsigned todo = s_wbits[w]; todo; todo &= todo - 1) {
                const int o = 32 * w + __ffs(todo) - 1;
                for (int yi = 0; yi < YC; ++yi)
                    for (unsigned msk = s_small[yi * NT + o]; msk; msk &= msk - 1) {
                        if (cnt < kListQ) list[1 + cnt] = o | (yi << 10) | ((__ffs(msk) - 1) << 14);
                        ++cnt;
                    }
            }
        }
        const bool fits = cnt <= kListQ;
        list[0] = fits ? cnt : 0;
        s_wbits[NW] = fits ? 1u : 0u;
        if (fits && cnt > 0) {   // the exact pass takes the bins in any order: each writes its own slot
            const int base = atomicAdd(nwork, cnt);
            for (int e = 0; e < cnt; ++e) work[base + e] = (int)(cta << 5) | e;
        }
    }
    __syncthreads();
    return s_wbits[NW] != 0u;
}

// The listed bins' exact pass: one warp per listed bin (a grid-stride loop over the work list).  Each is
// recomputed exactly as the in-kernel resolve does (the direct sum F = sum_u h(u) Vext[...] w^(k.u) in
// float-float arithmetic, lanes splitting the n^3 terms; A_p = sum_u h(u) |Vext| alongside), and its
// Gamma = rho F / |F| (0 if max(|Re F|, |Im F|) <= 2^-36 A_p) is written to the bin's slot of its CTA's list.
template <int N>
__global__ void __launch_bounds__(256)
k5_listed_exact_f32(const float* __restrict__ V, const float* __restrict__ gE, int* __restrict__ lists,
                    long long ncta, int T, int X, int Y, int bnd, int t_begin, int t_step,
                    const float* __restrict__ wtab, int taper, const __grid_constant__ Exact2f<N> ex) {
    using G = BGeo<N>;
    constexpr int H = G::H, BY = G::BY, YC = G::YC, ROWS = G::ROWS;
    constexpr int N3 = N * N * N, PER = N3 >= 32 ? N3 / 32 : 1, STEP = 32 / N;
    constexpr int U = PER >= 4 ? 4 : PER;   // terms whose loads are issued together
    // the float-float constants in shared memory: the lanes index them by their own phase, which the
    // parameter space would serve one distinct address at a time
    __shared__ float s_ex[6][N];
    __shared__ int s_rows[8][2][N];   // per warp: the cube's source rows along t and x of its current bin
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < 6 * N; i += blockDim.x) {
        const int a = i / N, m = i % N;
        s_ex[a][m] = a == 0 ? ex.ch[m] : a == 1 ? ex.cl[m] : a == 2 ? ex.sh[m] : a == 3 ? ex.sl[m]
                   : a == 4 ? ex.hh[m] : ex.hl[m];
    }
    __syncthreads();
    const int nw = lists[0];
    const int* work = lists + 4;
    int* ctal = lists + list_cta_offset(ncta);
    const int nseg = (Y + BY - 1) / BY;
    const size_t NV = (size_t)T * X * Y;
    const int uy = lane % N, r0 = lane / N;
    const bool live = lane < N3;
    const int wstride = gridDim.x * (blockDim.x / 32);
    for (int w = blockIdx.x * (blockDim.x / 32) + wib; w < nw; w += wstride) {
        const int item = work[w];
        const long long cta = item >> 5;
        const int e = item & 31;
        int* L = ctal + cta * kListStride;
        const int ent = L[1 + e];
        const int y_start = (int)(cta % nseg) * BY;
        const int x0 = (int)((cta / nseg) % X);
        const int t0 = t_begin + (int)(cta / ((long long)nseg * X)) * t_step;
        const int o = ent & 1023, yi = (ent >> 10) & 15, ky = (ent >> 14) & 15;
        const int row = o % ROWS, kt = row / N, kx = row % N, ych = o / ROWS;
        const int yl = ych * YC + yi;
        const int gy = ext_index(y_start + yl - N / 2 + uy, Y, bnd);
        if (lane < 2 * N)
            s_rows[wib][lane / N][lane % N] = lane < N ? ext_index(t0 - N / 2 + lane, T, bnd)
                                                       : ext_index(x0 - N / 2 + lane - N, X, bnd);
        __syncwarp();
        const FF hy = {s_ex[4][uy], s_ex[5][uy]};
        FF re = {0.f, 0.f}, im = {0.f, 0.f};
        float a1 = 0.f;   // the window's L1 norm, FP32 (it only places the 2^-36 band)
        for (int i0 = 0; i0 < PER; i0 += U) {
            float v[U];
            int tx[U];
#pragma unroll
            for (int a = 0; a < U; ++a) {   // loads first
                const int rr = live ? r0 + STEP * (i0 + a) : 0, ut = rr / N, ux = rr % N;
                const int gt = s_rows[wib][0][ut], gx = s_rows[wib][1][ux];
                v[a] = (live && (gt | gx | gy) >= 0) ? __ldg(V + ((size_t)gt * X + gx) * Y + gy) : 0.f;
                tx[a] = rr;
            }
#pragma unroll
            for (int a = 0; a < U; ++a) {
                const int ut = tx[a] / N, ux = tx[a] % N;
                const int ph = (kt * ut + kx * ux + ky * uy) % N;
                FF c = {s_ex[0][ph], s_ex[1][ph]}, sn = {-s_ex[2][ph], -s_ex[3][ph]};
                if (taper) {
                    const FF h3 = ff_mul(ff_mul(FF{s_ex[4][ut], s_ex[5][ut]}, FF{s_ex[4][ux], s_ex[5][ux]}), hy);
                    c = ff_mul(h3, c);
                    sn = ff_mul(h3, sn);
                    a1 = fmaf(h3.hi, fabsf(v[a]), a1);
                } else {
                    a1 += fabsf(v[a]);
                }
                re = ff_add(re, ff_mul1(v[a], c));
                im = ff_add(im, ff_mul1(v[a], sn));
            }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            const FF r2 = {__shfl_xor_sync(0xffffffffu, re.hi, d), __shfl_xor_sync(0xffffffffu, re.lo, d)};
            const FF i2 = {__shfl_xor_sync(0xffffffffu, im.hi, d), __shfl_xor_sync(0xffffffffu, im.lo, d)};
            re = ff_add(re, r2);
            im = ff_add(im, i2);
            a1 += __shfl_xor_sync(0xffffffffu, a1, d);
        }
        float gr = 0.f, gim = 0.f;
        const float mx = fmaxf(fabsf(re.hi), fabsf(im.hi));
        if (mx > kZeroBin * a1) {
            const int k = ky <= N / 2 ? ky : N - ky;
            const size_t gi = ((size_t)t0 * X + x0) * Y + y_start + yl;
            const float rho = fmaf(__ldg(gE + gi), __ldg(wtab + k * ROWS + row),
                                   fmaf(__ldg(gE + NV + gi), __ldg(wtab + (H + k) * ROWS + row),
                                        __ldg(gE + 2 * NV + gi) * __ldg(wtab + (2 * H + k) * ROWS + row)));
            const float fr = re.hi / mx, fi = im.hi / mx;      // scaled first: no underflow
            const float sc = rho / sqrtf(fmaf(fr, fr, fi * fi));
            gr = sc * fr;
            gim = sc * fi;
        }
        if (lane == 0) {
            float* gam = reinterpret_cast<float*>(L + 1 + kListQ);
            gam[2 * e] = gr;
            gam[2 * e + 1] = gim;
        }
        __syncwarp();   // the next bin rewrites this warp's source rows
    }
}

// The listed bins' apply pass: one warp per CTA of the main kernel's launch adds its listed bins, in list
// order, to the brick's block; the three adjoint stages of one bin are the outer product
//   block[u_t][u_x][y_l + u_y] += Re( Gamma h(u_t) h(u_x) h(u_y) e^{+2 pi i (k_t u_t + k_x u_x + k_y u_y) / n} ).
// Each block element is owned by one lane per bin; the warp syncs between bins (they overlap along y).
template <int N>
__global__ void __launch_bounds__(256)
k5_listed_apply_f32(float* __restrict__ blocks, const int* __restrict__ lists, long long ncta,
                    const __grid_constant__ Tw<N> tw) {
    using G = BGeo<N>;
    constexpr int YC = G::YC, YH = G::YH, ROWS = G::ROWS;
    constexpr int N3 = N * N * N, PER = N3 >= 32 ? N3 / 32 : 1, STEP = 32 / N;
    __shared__ float s_c[N / 2 + 1][N], s_s[N / 2 + 1][N];   // the lanes index them by their own taps
    for (int i = threadIdx.x; i < (N / 2 + 1) * N; i += blockDim.x) {
        s_c[i / N][i % N] = tw.c[i / N][i % N];
        s_s[i / N][i % N] = tw.s[i / N][i % N];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long cta = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (cta >= ncta) return;
    const int* L = lists + list_cta_offset(ncta) + cta * kListStride;
    const int cnt = L[0];
    if (cnt <= 0) return;
    const float* gam = reinterpret_cast<const float*>(L + 1 + kListQ);
    float* blk = blocks + cta * G::BLOCK_FLOATS;
    const int uy = lane % N, r0 = lane / N;
    const bool live = lane < N3;
    for (int e = 0; e < cnt; ++e) {
        const float gr = gam[2 * e], gim = gam[2 * e + 1];
        if (gr != 0.f || gim != 0.f) {   // warp-uniform
            const int ent = L[1 + e];
            const int o = ent & 1023, yi = (ent >> 10) & 15, ky = (ent >> 14) & 15;
            const int row = o % ROWS, kt = row / N, kx = row % N, ych = o / ROWS;
            const int yl = ych * YC + yi;
            // h(u) e^{+i theta} of each axis from the twiddle table (the taper is in it): bins above n/2 take the
            // conjugate of their mirror
            const int kxa = kx <= N / 2 ? kx : N - kx, kya = ky <= N / 2 ? ky : N - ky;
            const float sx = kx <= N / 2 ? 1.f : -1.f, sy = ky <= N / 2 ? 1.f : -1.f;
            const float eyr = s_c[kya][uy], eyi = sy * s_s[kya][uy];
            const float gyr = gr * eyr - gim * eyi, gyi = gr * eyi + gim * eyr;   // Gamma e_y
            constexpr int UB = PER >= 8 ? 8 : PER;   // block elements read, then written, together
            for (int i0 = 0; i0 < PER; i0 += UB) {
                float cur[UB];
                size_t off[UB];
#pragma unroll
                for (int a = 0; a < UB; ++a) {
                    const int rr = r0 + STEP * (i0 + a);
                    off[a] = (size_t)(rr / N) * G::SLICE + (rr % N) * YH + yl + uy;
                    cur[a] = (live && rr < N * N) ? blk[off[a]] : 0.f;
                }
#pragma unroll
                for (int a = 0; a < UB; ++a) {
                    const int rr = r0 + STEP * (i0 + a);
                    if (!live || rr >= N * N) continue;
                    const int ut = rr / N, ux = rr % N;
                    const float etr = s_c[kt][ut], eti = s_s[kt][ut];
                    const float exr = s_c[kxa][ux], exi = sx * s_s[kxa][ux];
                    const float txr = etr * exr - eti * exi, txi = etr * exi + eti * exr;
                    blk[off[a]] = cur[a] + (gyr * txr - gyi * txi);
                }
            }
        }
        __syncwarp();   // the next bin's window overlaps this one's along y
    }
}

// EN: the energy reading of the feature (Gamma = 2 rho F, no kink band).  SL: both y-passes slide (rect
// taper, n = 8, 16).  With the phase anchored at the start y_r of the thread's run,
//   Ft_j[k] = F_{y_r + j}[k] w^(k j) = sum_{y = j}^{j + n - 1} G2[y_r + y] w^(k y),   w = e^(-2 pi i / n),
// the forward recompute is Ft_0 by the direct sum, then Ft_{j+1} = Ft_j + (G2[y_r + j + n] - G2[y_r + j]) w^(k j),
// and |Ft| = |F|, so Gamma~_j = Gamma(Ft_j) = Gamma_j w^(k j) (the direction and the energy reading alike).
// The inverse along y of the run, dG2[y_r + p] = sum_{j <= p < j + n} sum_k Gamma_j[k] e^(2 pi i k (p - j)/n),
// is then z(P, p) = sum_k P[k] e^(2 pi i k p / n) of the sum P of Gamma~_j over the outputs j whose window
// holds p: for a run of YC <= n outputs, with the prefix sums P_i = sum_{j <= i} Gamma~_j,
//   p < YC - 1:  z(P_p, p);     YC - 1 <= p < n:  z(P_{YC-1}, p);     p = n + i:  z(P_{YC-1}, i) - z(P_i, i),
// (z has period n in p): YC + n - 1 point evaluations of n bins per run instead of YC n.
// The brick is staged as is: the small-bin level below is relative to the raw window's L1 norm.
template <int N, bool EN, bool SL>
__global__ void __launch_bounds__(BGeo<N>::NT, BCfg<N>::MINB)
k5_spectra_adjoint_f32(const float* __restrict__ V, const float* __restrict__ gE, float* __restrict__ blocks,
                       int T, int X, int Y, int bnd, int t_begin, int t_step, const float* __restrict__ wtab,
                       int taper, const __grid_constant__ Tw<N> tw, const __grid_constant__ Exact2f<N> ex,
                       const __grid_constant__ VanishTab vt, int* __restrict__ lists) {
    using G = BGeo<N>;
    using B = typename G::B;
    constexpr int H = G::H, BY = G::BY, YC = G::YC, YH = G::YH, ROWS = G::ROWS, NT = G::NT, WIN = G::WIN;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* s_in = reinterpret_cast<float*>(smem_raw);
    float2* s_g1 = reinterpret_cast<float2*>(smem_raw + G::IN_BYTES);
    float2* s_win = reinterpret_cast<float2*>(smem_raw);                 // [WIN][NT] after stage 2
    float2* s_gg1 = reinterpret_cast<float2*>(smem_raw);                 // Gamma_G1 [H][N][YH] after step 3
    float2* s_g2 = reinterpret_cast<float2*>(smem_raw + G::A_BYTES);     // G2, then Gamma_G2 [H][N][YH]
    float* s_ge = reinterpret_cast<float*>(smem_raw + G::A_BYTES + G::G_BYTES);  // [3][BY]
    float* s_l1 = s_ge + 3 * BY;                                                 // [BY] window L1 norms
    float* s_col = s_l1 + BY;                                                    // [YH] column sums
    uint16_t* s_small = reinterpret_cast<uint16_t*>(smem_raw + G::SMALL_OFF);    // [YC][NT]
    int* s_src = reinterpret_cast<int*>(smem_raw + G::IDX_OFF);                   // [2][N] cube rows along t, x

    const int tid = threadIdx.x;
    const int y_start = blockIdx.x * BY;
    const int x0 = blockIdx.y;
    const int t0 = t_begin + blockIdx.z * t_step;   // t_step s > 1: the lattice planes of stride-s windows
    const size_t NV = (size_t)T * X * Y;

    if (!EN)
        for (int i = tid; i < 2 * N; i += NT)
            s_src[i] = i < N ? ext_index(t0 - N / 2 + i, T, bnd) : ext_index(x0 - N / 2 + i - N, X, bnd);
    B::stage_brick(V, s_in, T, X, Y, bnd, t0, x0, y_start);
    for (int i = tid; i < 3 * BY; i += NT) {
        const int m = i / BY, yl = i % BY, y = y_start + yl;
        s_ge[i] = y < Y ? __ldg(gE + m * NV + ((size_t)t0 * X + x0) * Y + y) : 0.f;
    }
    __syncthreads();
    // window L1 norms A[y0] = sum_u h(u_t) h(u_x) h(u_y) |V|, as column sums then a y box sum
    for (int yy = tid; yy < YH; yy += NT) {
        float a = 0.f;
        for (int r = 0; r < N * N; ++r) a = fmaf(tw.c[0][r / N] * tw.c[0][r % N], fabsf(s_in[r * YH + yy]), a);
        s_col[yy] = a;
    }
    B::stage1(s_in, s_g1, tw);
    __syncthreads();
    for (int yl = tid; yl < BY; yl += NT) {
        float a = 0.f;
#pragma unroll
        for (int u = 0; u < N; ++u) a = fmaf(tw.c[0][u], s_col[yl + u], a);
        s_l1[yl] = a;
    }
    B::stage2(s_g1, s_g2, tw);
    __syncthreads();

    // ---- step 2: forward stage 3, Gamma, inverse along y into the private window -------------
    const int row = tid % ROWS;
    const int ych = tid / ROWS;
    float wt[3][H];
    B::row_weights(wtab, row, wt);
    if constexpr (!SL) {   // the sliding inverse writes every window position itself
#pragma unroll
        for (int j = 0; j < WIN; ++j) s_win[j * NT + tid] = make_float2(0.f, 0.f);
    }
    static_assert(!SL || YC <= N, "the sliding inverse needs runs of at most n outputs");
    const float2* grow = s_g2 + (size_t)row * YH;
    float fr[N], fi[N];   // F[k_y] of the current output, all n bins (SL: Ft, the run-anchored phase)
    // SL: prefix sums over the run's outputs of the pair coefficients below (the pairing is linear)
    float par[H], pai[H], pbr[H], pbi[H];
#pragma unroll
    for (int k = 0; k < H; ++k) par[k] = pai[k] = pbr[k] = pbi[k] = 0.f;
    // z(P, p): sum_k P[k] e^(2 pi i k p / n) from the pair coefficients of P, at run position p (mod n)
    auto z_at = [&](int p, float& zr, float& zi) {
        zr = 0.f;
        zi = 0.f;
#pragma unroll
        for (int k = 0; k < H; ++k) {
            zr = fmaf(par[k], tw.c[k][p], zr);
            zi = fmaf(pai[k], tw.c[k][p], zi);
            if (k != 0 && 2 * k != N) {
                zr = fmaf(pbr[k], tw.s[k][p], zr);
                zi = fmaf(pbi[k], tw.s[k][p], zi);
            }
        }
    };
    // the whole row vanishes when its k_t or its k_x does
    const bool row_vanishes =
        !EN && (((vanish_mask(vt, 0, t0, N) >> (row / N)) | (vanish_mask(vt, 1, x0, N) >> (row % N))) & 1u);
    for (int yi = 0; yi < YC; ++yi) {
        const int yl = ych * YC + yi;
        if (!SL || yi == 0) {
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
        } else {
            // Ft_yi = Ft_{yi-1} + (entering - leaving) w^(k (yi - 1)), w^(k m) = c - i sn
            const float2 a = grow[yl - 1], b = grow[yl - 1 + N];   // sample leaving, sample entering
            const float dr = b.x - a.x, di = b.y - a.y;
            const int m = yi - 1;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const float c = k <= N / 2 ? tw.c[k][m] : tw.c[N - k][m];
                const float sn = k <= N / 2 ? tw.s[k][m] : -tw.s[N - k][m];
                fr[k] = fmaf(dr, c, fmaf(di, sn, fr[k]));
                fi[k] = fmaf(di, c, fmaf(-dr, sn, fi[k]));
            }
        }
        const float g0 = s_ge[yl], g1 = s_ge[BY + yl], g2 = s_ge[2 * BY + yl];
        const float thr = kSmallBin * s_l1[yl];
        const float thr2 = fmaxf(thr * thr, 1e-30f);   // also keeps subnormal |F|^2 away from rsqrt
        unsigned small = 0u;                            // bins at or below thr: Gamma left to the FP64 recompute
        // A_k = Gamma[k] + Gamma[n-k], B_k = i (Gamma[k] - Gamma[n-k]); self-paired bins: A_k = Gamma[k]
        float ar[H], ai[H], br[H], bi[H];
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const float rho = fmaf(g0, wt[0][k], fmaf(g1, wt[1][k], g2 * wt[2][k]));
            if (k == 0 || 2 * k == N) {
                const float m2 = fmaf(fr[k], fr[k], fi[k] * fi[k]);
                const float sc = f32::bin_adjoint_scale<EN>(rho, m2, thr2);
                if (!EN && m2 <= thr2 && rho != 0.f) small |= 1u << k;
                ar[k] = sc * fr[k];
                ai[k] = sc * fi[k];
                br[k] = bi[k] = 0.f;
            } else {
                const float far = fr[k], fai = fi[k];            // F[k]
                const float hr = fr[N - k], hi = fi[N - k];      // F[n-k]
                const float m2a = fmaf(far, far, fai * fai), m2b = fmaf(hr, hr, hi * hi);
                const float sa = f32::bin_adjoint_scale<EN>(rho, m2a, thr2);
                const float sb = f32::bin_adjoint_scale<EN>(rho, m2b, thr2);
                if (!EN && rho != 0.f) {
                    if (m2a <= thr2) small |= 1u << k;
                    if (m2b <= thr2) small |= 1u << (N - k);
                }
                const float gar = sa * far, gai = sa * fai, gbr = sb * hr, gbi = sb * hi;
                ar[k] = gar + gbr;
                ai[k] = gai + gbi;
                br[k] = gbi - gai;        // i * (Gamma_a - Gamma_b)
                bi[k] = gar - gbr;
            }
        }
        if (!EN) {
            // bins that vanish for every input keep Gamma = 0; so does an all-zero cube (A_p = 0)
            if (small != 0u && (row_vanishes || !(s_l1[yl] > 0.f))) small = 0u;
            if (small != 0u) small &= ~vanish_mask(vt, 2, y_start + yl, N);
            s_small[yi * NT + tid] = (uint16_t)small;
        }
        if constexpr (SL) {
            // P_yi = P_{yi-1} + Gamma~_yi; position yi takes z(P_yi, yi), position n + yi its negative (the
            // full sum's value is added below)
#pragma unroll
            for (int k = 0; k < H; ++k) {
                par[k] += ar[k];
                pai[k] += ai[k];
                pbr[k] += br[k];
                pbi[k] += bi[k];
            }
            if (yi < YC - 1) {
                float zr, zi;
                z_at(yi, zr, zi);
                s_win[yi * NT + tid] = make_float2(zr, zi);
                s_win[(N + yi) * NT + tid] = make_float2(-zr, -zi);
            }
        } else {
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
                float2* w = s_win + (yi + u) * NT + tid;
                float2 acc = *w;
                acc.x += zr;
                acc.y += zi;
                *w = acc;
            }
        }
    }
    if constexpr (SL) {
        // the full sum P_{YC-1}: positions YC - 1 .. n - 1 take z(P_{YC-1}, p); positions n + i add z(P_{YC-1}, i)
#pragma unroll
        for (int p = 0; p < N; ++p) {
            float zr, zi;
            z_at(p, zr, zi);
            if (p < YC - 1) {
                float2* w = s_win + (N + p) * NT + tid;
                float2 acc = *w;
                acc.x += zr;
                acc.y += zi;
                *w = acc;
            } else {
                s_win[p * NT + tid] = make_float2(zr, zi);
            }
        }
    }
    if (!EN) {
        // the small bins go to the listed-bin pass when a list is given and they fit in it
        unsigned* s_wbits = reinterpret_cast<unsigned*>(smem_raw + G::WB_OFF);
        const size_t cta = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        const size_t ncta = (size_t)gridDim.x * gridDim.y * gridDim.z;
        const bool listed = lists && list_small_bins<NT, YC>(s_small, s_wbits,
                                                             lists + list_cta_offset(ncta) + cta * kListStride,
                                                             lists + 4, lists, (long long)cta);
        if (!listed)
            resolve_small_bins<N, NT, YC, BY, H, ROWS>(V, X, Y, bnd, y_start, taper, s_small, s_src, s_win, s_ge,
                                                       s_l1, wtab, tw, ex, s_wbits);
    }
    __syncthreads();

    // ---- step 3: sum the y-chunk windows into Gamma_G2[row][y] ---------------------------------
    for (int it = tid; it < ROWS * YH; it += NT) {
        const int r = it % ROWS, y = it / ROWS;   // rows fastest: window reads are consecutive
        float sr = 0.f, si = 0.f;
#pragma unroll
        for (int c = 0; c < BY / YC; ++c) {
            const int j = y - c * YC;
            if (j >= 0 && j < WIN) {
                const float2 v = s_win[j * NT + c * ROWS + r];
                sr += v.x;
                si += v.y;
            }
        }
        s_g2[(size_t)r * YH + y] = make_float2(sr, si);
    }
    __syncthreads();

    // ---- step 4: adjoint of stage 2 (x): Gamma_G1[k_t][u][y] ----------------------------------
    for (int it = tid; it < H * YH; it += NT) {
        const int kt = it / YH, y = it % YH;
        float ar[H], ai[H], br[H], bi[H];
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const float2 a = s_g2[(size_t)(kt * N + k) * YH + y];
            if (k == 0 || 2 * k == N) {
                ar[k] = a.x; ai[k] = a.y; br[k] = bi[k] = 0.f;
            } else {
                const float2 b = s_g2[(size_t)(kt * N + (N - k)) * YH + y];
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
            s_gg1[(size_t)(kt * N + u) * YH + y] = make_float2(zr, zi);
        }
    }
    __syncthreads();

    // ---- step 5: adjoint of stage 1 (t), real part -> scratch block [u_t][u_x][y] -------------
    const size_t cta = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    float* blk = blocks + cta * G::BLOCK_FLOATS;
    for (int it = tid; it < N * YH; it += NT) {
        const int ux = it / YH, y = it % YH;
        float2 g[H];
#pragma unroll
        for (int k = 0; k < H; ++k) g[k] = s_gg1[(size_t)(k * N + ux) * YH + y];
#pragma unroll
        for (int u = 0; u < N; ++u) {
            float z = 0.f;
#pragma unroll
            for (int k = 0; k < H; ++k) {
                z = fmaf(g[k].x, tw.c[k][u], z);
                if (k != 0 && 2 * k != N) z = fmaf(-g[k].y, tw.s[k][u], z);
            }
            blk[(size_t)u * G::SLICE + ux * YH + y] = z;
        }
    }
}

template <int N> constexpr bool kAdjointSliding = N >= 8;

template <int N>
cudaError_t prepare_n() {
    constexpr int smem = (int)BGeo<N>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(k5_spectra_adjoint_f32<N, false, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k5_spectra_adjoint_f32<N, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if constexpr (kAdjointSliding<N>) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k5_spectra_adjoint_f32<N, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k5_spectra_adjoint_f32<N, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem);
    }
    return e;
}

// The float-float constants of the exact recompute of small bins: cos, sin (2 pi m / n) and the taper
// (rect, or the periodic Hann window 1/2 - cos(2 pi u / n) / 2), from the host's double-precision libm,
// each split into an FP32 head and the FP32 rounding of the remainder.
template <int N>
Exact2f<N> make_exact2f(int taper) {
    Exact2f<N> e;
    auto split = [](double v, float& hi, float& lo) {
        hi = (float)v;
        lo = (float)(v - (double)hi);
    };
    for (int m = 0; m < N; ++m) {
        const double a = 2.0 * 3.14159265358979323846 * m / N;
        split(cos(a), e.ch[m], e.cl[m]);
        split(sin(a), e.sh[m], e.sl[m]);
        split(taper ? 0.5 - 0.5 * cos(a) : 1.0, e.hh[m], e.hl[m]);
    }
    return e;
}

template <int N, bool SL>
void launch_sl(const TwiddleTable& t, const float* wtab, dim3 grid, const float* V, const float* gE, float* blocks,
               int T, int X, int Y, int bnd, int feat, int t_begin, int t_step, int taper, int* lists,
               cudaStream_t s) {
    using G = BGeo<N>;
    if (feat == 1) {
        k5_spectra_adjoint_f32<N, true, SL><<<grid, G::NT, G::SMEM, s>>>(
            V, gE, blocks, T, X, Y, bnd, t_begin, t_step, wtab, taper, f32::make_tw<N>(t), make_exact2f<N>(taper),
            VanishTab{}, nullptr);
        return;
    }
    k5_spectra_adjoint_f32<N, false, SL><<<grid, G::NT, G::SMEM, s>>>(
        V, gE, blocks, T, X, Y, bnd, t_begin, t_step, wtab, taper, f32::make_tw<N>(t), make_exact2f<N>(taper),
        make_vanish_tab(N, T, X, Y, bnd, taper), lists);
    if (lists) {
        const long long ncta = (long long)grid.x * grid.y * grid.z;
        k5_listed_exact_f32<N><<<8 * device_sms(), 256, 0, s>>>(V, gE, lists, ncta, T, X, Y, bnd, t_begin, t_step,
                                                                 wtab, taper, make_exact2f<N>(taper));
        k5_listed_apply_f32<N><<<(unsigned)((ncta + 7) / 8), 256, 0, s>>>(blocks, lists, ncta, f32::make_tw<N>(t));
        note_launches(2);
    }
}

template <int N>
cudaError_t launch_n(const TwiddleTable& t, const float* wtab, const float* V, const float* gE, float* blocks, int T,
                     int X, int Y, int bnd, int feat, int t_begin, int t_step, int t_count, int taper, int* lists,
                     cudaStream_t s) {
    using G = BGeo<N>;
    dim3 grid((Y + G::BY - 1) / G::BY, X, t_count);
    if (lists && feat != 1) {   // the work-list counter starts at zero
        const cudaError_t e = cudaMemsetAsync(lists, 0, sizeof(int), s);
        if (e != cudaSuccess) return e;
    }
    if constexpr (kAdjointSliding<N>) {
        if (taper == 0)
            launch_sl<N, true>(t, wtab, grid, V, gE, blocks, T, X, Y, bnd, feat, t_begin, t_step, taper, lists, s);
        else
            launch_sl<N, false>(t, wtab, grid, V, gE, blocks, T, X, Y, bnd, feat, t_begin, t_step, taper, lists, s);
    } else {
        launch_sl<N, false>(t, wtab, grid, V, gE, blocks, T, X, Y, bnd, feat, t_begin, t_step, taper, lists, s);
    }
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t spectra_adjoint_f32_prepare(int n) {
    switch (n) {
        case 2: return prepare_n<2>();
        case 4: return prepare_n<4>();
        case 8: return prepare_n<8>();
        case 16: return prepare_n<16>();
        default: return cudaErrorInvalidValue;
    }
}

SpectraAdjointGeometry spectra_adjoint_f32_geometry(int n) {
    switch (n) {
        case 2: return {BGeo<2>::BY, BGeo<2>::YH, 1, 2, BGeo<2>::BLOCK_FLOATS, BGeo<2>::SLICE};
        case 4: return {BGeo<4>::BY, BGeo<4>::YH, 1, 4, BGeo<4>::BLOCK_FLOATS, BGeo<4>::SLICE};
        case 8: return {BGeo<8>::BY, BGeo<8>::YH, 1, 8, BGeo<8>::BLOCK_FLOATS, BGeo<8>::SLICE};
        case 16: return {BGeo<16>::BY, BGeo<16>::YH, 1, 16, BGeo<16>::BLOCK_FLOATS, BGeo<16>::SLICE};
        default: return {0, 0, 0, 0, 0, 0};
    }
}

size_t spectra_adjoint_f32_list_bytes(int n, int X, int Y, int t_count) {
    const int by = n == 16 ? BGeo<16>::BY : BGeo<8>::BY;   // 32 for n <= 8
    const long long ncta = (long long)((Y + by - 1) / by) * X * t_count;
    return (list_cta_offset(ncta) + (size_t)ncta * kListStride) * sizeof(int);
}

cudaError_t spectra_adjoint_f32_launch(int n, const TwiddleTable& tw, const float* wtab, const float* V,
                                       const float* gE, float* blocks, int T, int X, int Y, int bnd, int feat,
                                       int t_begin, int t_step, int t_count, int taper, int* lists, cudaStream_t s) {
    if (t_step < 1 || taper < 0 || taper > 1) return cudaErrorInvalidValue;
    switch (n) {
        case 2:
            return launch_n<2>(tw, wtab, V, gE, blocks, T, X, Y, bnd, feat, t_begin, t_step, t_count, taper, lists, s);
        case 4:
            return launch_n<4>(tw, wtab, V, gE, blocks, T, X, Y, bnd, feat, t_begin, t_step, t_count, taper, lists, s);
        case 8:
            return launch_n<8>(tw, wtab, V, gE, blocks, T, X, Y, bnd, feat, t_begin, t_step, t_count, taper, lists, s);
        case 16:
            return launch_n<16>(tw, wtab, V, gE, blocks, T, X, Y, bnd, feat, t_begin, t_step, t_count, taper, lists,
                                s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sal
