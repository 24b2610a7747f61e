// K3: normalisation and combination of the three saliency maps (Sec. 2 step 5, Eq. 4).
//   S^_m = (S_m - min S_m) / (max S_m - min S_m)   (a flat map becomes 0)
//   W    = equal (1/3), given, or the least-squares fit to a desired map D:
//          W = (G + delta I)^-1 b,  G = sum_p x_p x_p^T,  b = sum_p x_p D_p,  x_p = S^(p),
//          G and b accumulated in FP64 (per-thread, then per-block trees, then a fixed-order
//          sum of the block partials) and solved on the device by one thread;
//   S    = minmax(sum_m W_m S^_m).
// All passes are grid-stride, HBM-bound and deterministic (no floating-point atomics).
#include <cfloat>
#include <cmath>
#include <mutex>
#include <string>

#include "sal_internal.cuh"

namespace sal {
namespace {

constexpr int kThreads = 256;

enum : int { N_LO = 0, N_INV = 3, N_W = 6, N_LOC = 9, N_INVC = 10 };

__device__ __forceinline__ float flat_inv(float lo, float hi) {
    const float span = hi - lo;
    return (span > 1e-30f * fmaxf(1.f, fabsf(hi))) ? 1.f / span : 0.f;
}

// Reduces per-block min/max partials (layout [part][8]: min at c, max at 3+c) of `nmaps`
// maps; writes lo and 1/(hi-lo) (0 for a flat map).  One block.
__global__ void __launch_bounds__(kThreads)
k3_minmax_finalize(const float* __restrict__ mm_part, int nparts, int nmaps, float* __restrict__ lo,
                   float* __restrict__ inv) {
    __shared__ float smin[3][kThreads], smax[3][kThreads];
    for (int m = 0; m < nmaps; ++m) {
        float a = FLT_MAX, b = -FLT_MAX;
        for (int i = threadIdx.x; i < nparts; i += kThreads) {
            a = fminf(a, mm_part[i * 8 + m]);
            b = fmaxf(b, mm_part[i * 8 + 3 + m]);
        }
        smin[m][threadIdx.x] = a;
        smax[m][threadIdx.x] = b;
    }
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int m = 0; m < nmaps; ++m) {
                smin[m][threadIdx.x] = fminf(smin[m][threadIdx.x], smin[m][threadIdx.x + s]);
                smax[m][threadIdx.x] = fmaxf(smax[m][threadIdx.x], smax[m][threadIdx.x + s]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int m = 0; m < nmaps; ++m) {
            lo[m] = smin[m][0];
            inv[m] = flat_inv(smin[m][0], smax[m][0]);
        }
}

// FP64 partial Gram matrix and right-hand side of the template fit.
__global__ void __launch_bounds__(kThreads)
k3_gram(const float* __restrict__ S3, const float* __restrict__ D, long long NV, const float* __restrict__ norm,
        double* __restrict__ g_part) {
    const float lo0 = norm[N_LO], lo1 = norm[N_LO + 1], lo2 = norm[N_LO + 2];
    const float iv0 = norm[N_INV], iv1 = norm[N_INV + 1], iv2 = norm[N_INV + 2];
    double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (long long p = (long long)blockIdx.x * kThreads + threadIdx.x; p < NV; p += (long long)gridDim.x * kThreads) {
        const double x0 = (double)((__ldg(S3 + p) - lo0) * iv0);
        const double x1 = (double)((__ldg(S3 + NV + p) - lo1) * iv1);
        const double x2 = (double)((__ldg(S3 + 2 * NV + p) - lo2) * iv2);
        const double d = (double)__ldg(D + p);
        acc[0] += x0 * x0; acc[1] += x0 * x1; acc[2] += x0 * x2;
        acc[3] += x1 * x1; acc[4] += x1 * x2; acc[5] += x2 * x2;
        acc[6] += x0 * d;  acc[7] += x1 * d;  acc[8] += x2 * d;
    }
    __shared__ double red[9][kThreads];
    for (int c = 0; c < 9; ++c) red[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int c = 0; c < 9; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 9) g_part[blockIdx.x * 16 + threadIdx.x] = red[threadIdx.x][0];
}

// Chooses the weights: mode 0 equal, 1 given (W_in), 2 least squares from the Gram partials.
__global__ void __launch_bounds__(kThreads)
k3_weights(const double* __restrict__ g_part, int nparts, const float* __restrict__ W_in, int mode, double delta,
           float* __restrict__ norm, float* __restrict__ W_out, double* __restrict__ wsum) {
    __shared__ double s[9][kThreads];
    if (mode == 2) {
        for (int c = 0; c < 9; ++c) {
            double a = 0.0;
            for (int i = threadIdx.x; i < nparts; i += kThreads) a += g_part[i * 16 + c];
            s[c][threadIdx.x] = a;
        }
        __syncthreads();
        for (int st = kThreads / 2; st > 0; st >>= 1) {
            if (threadIdx.x < st)
                for (int c = 0; c < 9; ++c) s[c][threadIdx.x] += s[c][threadIdx.x + st];
            __syncthreads();
        }
    }
    if (threadIdx.x != 0) return;
    double W[3];
    if (mode == 0) {
        W[0] = W[1] = W[2] = 1.0 / 3.0;
    } else if (mode == 1) {
        for (int m = 0; m < 3; ++m) W[m] = (double)W_in[m];
    } else {
        double A[3][4] = {{s[0][0] + delta, s[1][0], s[2][0], s[6][0]},
                          {s[1][0], s[3][0] + delta, s[4][0], s[7][0]},
                          {s[2][0], s[4][0], s[5][0] + delta, s[8][0]}};
        for (int c = 0; c < 9; ++c) wsum[c] = s[c][0];
        // Gaussian elimination with partial pivoting.
        for (int c = 0; c < 3; ++c) {
            int piv = c;
            for (int r = c + 1; r < 3; ++r)
                if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
            if (piv != c)
                for (int k = 0; k < 4; ++k) {
                    double tmp = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = tmp;
                }
            const double d = A[c][c];
            for (int r = c + 1; r < 3; ++r) {
                const double f = d != 0.0 ? A[r][c] / d : 0.0;
                for (int k = c; k < 4; ++k) A[r][k] -= f * A[c][k];
            }
        }
        for (int c = 2; c >= 0; --c) {
            double v = A[c][3];
            for (int k = c + 1; k < 3; ++k) v -= A[c][k] * W[k];
            W[c] = A[c][c] != 0.0 ? v / A[c][c] : 0.0;
        }
    }
    for (int m = 0; m < 3; ++m) {
        norm[N_W + m] = (float)W[m];
        if (W_out) W_out[m] = (float)W[m];
    }
}

__global__ void __launch_bounds__(kThreads)
k3_combine(const float* __restrict__ S3, long long NV, const float* __restrict__ norm, float* __restrict__ S,
           float* __restrict__ mm_part) {
    const float lo0 = norm[N_LO], lo1 = norm[N_LO + 1], lo2 = norm[N_LO + 2];
    const float a0 = norm[N_INV] * norm[N_W], a1 = norm[N_INV + 1] * norm[N_W + 1], a2 = norm[N_INV + 2] * norm[N_W + 2];
    float mn = FLT_MAX, mx = -FLT_MAX;
    for (long long p = (long long)blockIdx.x * kThreads + threadIdx.x; p < NV; p += (long long)gridDim.x * kThreads) {
        float c = (__ldg(S3 + p) - lo0) * a0;
        c = fmaf(__ldg(S3 + NV + p) - lo1, a1, c);
        c = fmaf(__ldg(S3 + 2 * NV + p) - lo2, a2, c);
        S[p] = c;
        mn = fminf(mn, c);
        mx = fmaxf(mx, c);
    }
    __shared__ float smin[kThreads], smax[kThreads];
    smin[threadIdx.x] = mn;
    smax[threadIdx.x] = mx;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            smin[threadIdx.x] = fminf(smin[threadIdx.x], smin[threadIdx.x + s]);
            smax[threadIdx.x] = fmaxf(smax[threadIdx.x], smax[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        mm_part[blockIdx.x * 8] = smin[0];
        mm_part[blockIdx.x * 8 + 3] = smax[0];
    }
}

// Per-block min/max partials of the three S_m planes (used when S3 did not come from K2).
__global__ void __launch_bounds__(kThreads)
k3_minmax3(const float* __restrict__ S3, long long NV, float* __restrict__ mm_part) {
    float mn[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, mx[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (long long p = (long long)blockIdx.x * kThreads + threadIdx.x; p < NV; p += (long long)gridDim.x * kThreads)
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const float v = __ldg(S3 + m * NV + p);
            mn[m] = fminf(mn[m], v);
            mx[m] = fmaxf(mx[m], v);
        }
    __shared__ float smin[3][kThreads], smax[3][kThreads];
    for (int m = 0; m < 3; ++m) {
        smin[m][threadIdx.x] = mn[m];
        smax[m][threadIdx.x] = mx[m];
    }
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int m = 0; m < 3; ++m) {
                smin[m][threadIdx.x] = fminf(smin[m][threadIdx.x], smin[m][threadIdx.x + s]);
                smax[m][threadIdx.x] = fmaxf(smax[m][threadIdx.x], smax[m][threadIdx.x + s]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 3) {
        mm_part[blockIdx.x * 8 + threadIdx.x] = smin[threadIdx.x][0];
        mm_part[blockIdx.x * 8 + 3 + threadIdx.x] = smax[threadIdx.x][0];
    }
}

__global__ void __launch_bounds__(kThreads)
k3_normalize(float* __restrict__ S, long long NV, const float* __restrict__ norm) {
    const float lo = norm[N_LOC], inv = norm[N_INVC];
    for (long long p = (long long)blockIdx.x * kThreads + threadIdx.x; p < NV; p += (long long)gridDim.x * kThreads)
        S[p] = (S[p] - lo) * inv;
}

}  // namespace

int red_blocks(long long NV) {
    long long b = (NV + kThreads - 1) / kThreads;
    return (int)(b < kRedBlocks ? b : kRedBlocks);
}

cudaError_t minmax_bounds_launch(const float* S3, long long N, const Reduce& r, cudaStream_t s) {
    const int nb = red_blocks(N);
    k3_minmax3<<<nb, kThreads, 0, s>>>(S3, N, r.mm_part);
    k3_minmax_finalize<<<1, kThreads, 0, s>>>(r.mm_part, nb, 3, r.norm + N_LO, r.norm + N_INV);
    note_launches(2);
    return cudaGetLastError();
}

cudaError_t combine_launch(const float* S3, const float* D, const float* W_in, float* W_out, float* S,
                           long long N, double delta, bool s3_partials_ready, const Reduce& r, cudaStream_t s) {
    const int nb = red_blocks(N);
    // min/max partials of S3: written by K2 (same block count) when it produced S3
    if (!s3_partials_ready) k3_minmax3<<<nb, kThreads, 0, s>>>(S3, N, r.mm_part);
    k3_minmax_finalize<<<1, kThreads, 0, s>>>(r.mm_part, nb, 3, r.norm + N_LO, r.norm + N_INV);
    int mode = D ? 2 : (W_in ? 1 : 0);
    if (mode == 2) k3_gram<<<nb, kThreads, 0, s>>>(S3, D, N, r.norm, r.g_part);
    k3_weights<<<1, kThreads, 0, s>>>(r.g_part, nb, W_in, mode, delta, r.norm, W_out, r.wsum);
    k3_combine<<<nb, kThreads, 0, s>>>(S3, N, r.norm, S, r.mm_part);
    k3_minmax_finalize<<<1, kThreads, 0, s>>>(r.mm_part, nb, 1, r.norm + N_LOC, r.norm + N_INVC);
    k3_normalize<<<nb, kThreads, 0, s>>>(S, N, r.norm);
    note_launches(5 + (s3_partials_ready ? 0 : 1) + (mode == 2 ? 1 : 0));
    return cudaGetLastError();
}

}  // namespace sal

// ---- Allocation-free combination --------------------------------------------------------------
// sal_combine_noalloc runs the same K3 kernels as sal_combine, but its reduction scratch is a
// file-scope device array instead of memory the handle obtains from cudaMalloc.  It serves
// callers that must not allocate device memory: code running under a caller-owned memory pool
// or arena, inside a region that forbids new allocations, or on a path where an allocation
// (and the implicit synchronisation it can bring) is not acceptable.
namespace {

constexpr long long kNoAllocVoxPerBlock = 4096;  // 256 threads x 16 voxels per partial slot
constexpr int kNoAllocSlots = 4096;              // partial slots held by the static array
constexpr long long kNoAllocMaxVoxels = kNoAllocVoxPerBlock * kNoAllocSlots;  // 16,777,216

struct NoAllocScratch {
    double g_part[kNoAllocSlots * 16];
    double wsum[16];
    float mm_part[kNoAllocSlots * 8];
    float norm[16];
};

// Host code must not use this name as a device address: on the host it is only a stand-in.
// The device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

constexpr int kNoAllocMaxDevices = 64;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};
std::mutex g_noalloc_mu;

// True when p is device (or managed) memory that the current device dev can address as its own.
bool on_device(const void* p, int dev) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" sal_status sal_combine_noalloc(int T, int X, int Y, const float* S3, const float* D, const float* W_in,
                                          double ls_delta, float* W_out, float* S, void* stream) {
    sal::set_unbound_error("");
    if (T < 1 || X < 1 || Y < 1) {
        sal::set_unbound_error("sal_combine_noalloc: T, X, Y must be >= 1");
        return SAL_ERR_INVALID_ARG;
    }
    const long long N = (long long)T * X * Y;
    if (N > kNoAllocMaxVoxels) {
        sal::set_unbound_error("sal_combine_noalloc: volume of " + std::to_string(N) +
                               " voxels exceeds the static scratch limit of 16777216 voxels");
        return SAL_ERR_UNSUPPORTED;
    }
    if (!S3 || !S) {
        sal::set_unbound_error("sal_combine_noalloc: S3 and S must not be NULL");
        return SAL_ERR_INVALID_ARG;
    }
    if (!(ls_delta >= 0.0) || !std::isfinite(ls_delta)) {
        sal::set_unbound_error("sal_combine_noalloc: ls_delta must be finite and >= 0");
        return SAL_ERR_INVALID_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        sal::set_unbound_error(std::string("sal_combine_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return SAL_ERR_CUDA;
    }
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        sal::set_unbound_error("sal_combine_noalloc: device ordinal beyond 63");
        return SAL_ERR_UNSUPPORTED;
    }
    // every buffer must live on the current device: the kernels launch there
    const void* bufs[5] = {S3, S, D, W_in, W_out};
    const char* names[5] = {"S3", "S", "D", "W_in", "W_out"};
    for (int i = 0; i < 5; ++i)
        if (bufs[i] && !on_device(bufs[i], dev)) {
            sal::set_unbound_error(std::string("sal_combine_noalloc: ") + names[i] +
                                   " is not device memory of the current device " + std::to_string(dev));
            return SAL_ERR_INVALID_ARG;
        }
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            e = cudaGetSymbolAddress(&g_noalloc_addr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_noalloc_addr[dev] = nullptr;
                sal::set_unbound_error(std::string("sal_combine_noalloc: cudaGetSymbolAddress: ") +
                                       cudaGetErrorString(e));
                return SAL_ERR_CUDA;
            }
        }
        base = g_noalloc_addr[dev];
    }
    NoAllocScratch* scr = static_cast<NoAllocScratch*>(base);
    sal::Reduce r{};
    r.mm_part = scr->mm_part;
    r.g_part = scr->g_part;
    r.norm = scr->norm;
    r.wsum = scr->wsum;
    // Every partial slot a kernel reads was written earlier in this call, so the leftovers
    // of a previous call need no clearing.
    const int nb = (int)((N + kNoAllocVoxPerBlock - 1) / kNoAllocVoxPerBlock);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    sal::k3_minmax3<<<nb, sal::kThreads, 0, s>>>(S3, N, r.mm_part);
    sal::k3_minmax_finalize<<<1, sal::kThreads, 0, s>>>(r.mm_part, nb, 3, r.norm + sal::N_LO, r.norm + sal::N_INV);
    const int mode = D ? 2 : (W_in ? 1 : 0);
    if (mode == 2) sal::k3_gram<<<nb, sal::kThreads, 0, s>>>(S3, D, N, r.norm, r.g_part);
    sal::k3_weights<<<1, sal::kThreads, 0, s>>>(r.g_part, nb, W_in, mode, ls_delta, r.norm, W_out, r.wsum);
    sal::k3_combine<<<nb, sal::kThreads, 0, s>>>(S3, N, r.norm, S, r.mm_part);
    sal::k3_minmax_finalize<<<1, sal::kThreads, 0, s>>>(r.mm_part, nb, 1, r.norm + sal::N_LOC, r.norm + sal::N_INVC);
    sal::k3_normalize<<<nb, sal::kThreads, 0, s>>>(S, N, r.norm);
    sal::note_launches(6 + (mode == 2 ? 1 : 0));
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        sal::set_unbound_error(std::string("sal_combine_noalloc: launch: ") + cudaGetErrorString(e));
        return SAL_ERR_CUDA;
    }
    return SAL_OK;
}
