// Host side of the C ABI declared in include/sal.h: parameter validation, handle-owned tables
// and scratch, and stream-ordered launches of the kernels K1 (local spectra + features),
// K2 (center-surround) and K3 (normalisation + combination).
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <atomic>
#include <cstring>
#include <string>
#include <vector>

#include "sal_internal.cuh"

struct sal_handle {
    int device = 0;
    int T = 0, X = 0, Y = 0;
    long long N = 0;
    int n = 0, taper = 0, boundary = 0, feature = 0, prec = 0, stride = 1;
    double ls_delta = 1e-6;
    size_t budget = 0;
    sal::Stencil st{};
    std::vector<float> alpha;
    sal::TwiddleTable tw{};
    float* E = nullptr;      // [3][N] feature scratch
    float* Ec = nullptr;     // [3][Tc][Xc][Yc] lattice features of stride > 1
    float* S3 = nullptr;     // [3][N] raw center-surround scratch
    sal::Reduce red{};
    void* small = nullptr;   // one allocation holding the reduction scratch
    void* tc_tables = nullptr;  // constant tensor-core operands of K1 (BF16/FP16 forms)
    void* adj_tables = nullptr; // constant tensor-core operands of K5 (FP16)
    float* f32_wt = nullptr;    // Eq. 1 weight table of the FP32 K1 / K5 (n <= 16)
    float* sp_tab = nullptr;    // spatial-domain reading: the Eq. 1 ratio table
    float* vpad = nullptr;      // V with rows padded to ypad floats (tensor-core forms, Y not a multiple of 4)
    int ypad = 0;
    // backward scratch, allocated by the first sal_saliency_backward call
    float* gE = nullptr;     // [3][N]
    double* bpart = nullptr; // [kRedBlocks][64]
    float* blocks = nullptr; // brick blocks of the spectral adjoint for one slab of t0
    size_t blocks_bytes = 0; //   (also the per-tile partials of the center-surround adjoint, which runs before)
    float* gext = nullptr;   // the blocks summed along t, per extended plane of the slab
    float* gEl = nullptr;    // stride > 1: the feature gradient gathered onto the lattice voxels (zero elsewhere)
    int slab_t = 0;
    volatile int* err_host = nullptr;  // mapped host word set by bounded device waits that gave up
    int* err_dev = nullptr;
    size_t bytes = 0;
    std::string last;
};

namespace {

thread_local std::string g_create_error;

sal_status fail(sal_handle* h, sal_status s, const std::string& msg) {
    if (h) h->last = msg; else g_create_error = msg;
    return s;
}

sal_status cuda_fail(sal_handle* h, cudaError_t e, const char* where) {
    return fail(h, SAL_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

void free_scratch(sal_handle* h) {
    if (h->E) cudaFree(h->E);
    if (h->S3) cudaFree(h->S3);
    if (h->Ec) cudaFree(h->Ec);
    h->Ec = nullptr;
    if (h->small) cudaFree(h->small);
    if (h->tc_tables) cudaFree(h->tc_tables);
    if (h->adj_tables) cudaFree(h->adj_tables);
    h->tc_tables = h->adj_tables = nullptr;
    if (h->f32_wt) cudaFree(h->f32_wt);
    h->f32_wt = nullptr;
    if (h->sp_tab) cudaFree(h->sp_tab);
    h->sp_tab = nullptr;
    if (h->vpad) cudaFree(h->vpad);
    h->vpad = nullptr;
    if (h->err_host) cudaFreeHost((void*)h->err_host);
    h->err_host = nullptr;
    h->err_dev = nullptr;
    if (h->gE) cudaFree(h->gE);
    if (h->bpart) cudaFree(h->bpart);
    if (h->blocks) cudaFree(h->blocks);
    if (h->gext) cudaFree(h->gext);
    if (h->gEl) cudaFree(h->gEl);
    h->E = h->S3 = h->gE = h->blocks = h->gext = h->gEl = nullptr;
    h->small = nullptr;
    h->bpart = nullptr;
}

void build_twiddles(sal_handle* h) {
    const int n = h->n;
    h->tw.n = n;
    for (int k = 0; k <= n / 2; ++k)
        for (int u = 0; u < n; ++u) {
            const int m = (k * u) % n;
            const double hu = h->taper ? 0.5 - 0.5 * std::cos(2.0 * M_PI * u / n) : 1.0;
            h->tw.c[k][u] = (float)(hu * std::cos(2.0 * M_PI * m / n));
            h->tw.s[k][u] = (float)(hu * std::sin(2.0 * M_PI * m / n));
        }
}

void refresh_weights(sal_handle* h) {
    for (int o = 0; o < h->st.Q; ++o) h->st.w[o] = h->alpha[h->st.dir[o]] * h->st.g[o];
}

sal_status check_handle(sal_handle* h) {
    if (!h) return SAL_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    h->last.clear();
    if (h->err_host && *h->err_host) {
        *h->err_host = 0;
        return fail(h, SAL_ERR_TIMEOUT, "a bounded tensor-core wait gave up in an earlier call; its outputs are invalid");
    }
    return SAL_OK;
}

// The row-padded copy of V the tensor-core kernels' TMA staging reads (one tensor copy per interior brick),
// refreshed from V on every call; null (and no work) when V's rows are already a multiple of 16 bytes.
const float* padded_copy(sal_handle* h, const float* V, cudaStream_t st, cudaError_t& e) {
    e = cudaSuccess;
    if (!h->vpad) return nullptr;
    e = sal::pad_rows_launch(V, h->vpad, (long long)h->T * h->X, h->Y, h->ypad, st);
    return e == cudaSuccess ? h->vpad : nullptr;
}

// K1 in the handle's precision: FP32 on the SIMT pipes, or BF16/FP16 on the tensor cores.  With stride
// s > 1 the cubes sit on the lattice of multiples of s (into the handle's lattice scratch) and E is
// interpolated from them.
cudaError_t launch_k1(sal_handle* h, const float* V, float* E, cudaStream_t st) {
    const int s = h->stride;
    float* out = s > 1 ? h->Ec : E;
    cudaError_t e;
    if (h->feature == 2) {
        e = sal::spatial_f32_launch(h->n, h->sp_tab, V, E, h->T, h->X, h->Y, h->boundary, h->taper, st);
    } else if (h->n == 32) {
        e = h->prec == SAL_FP32
                ? sal::spectra_f32_n32_launch(h->tw, V, out, h->T, h->X, h->Y, h->boundary, h->feature, s, h->taper, st)
                : sal::spectra_tc32_launch(h->prec == SAL_BF16 ? 1 : 0, h->tw, V, out, h->T, h->X, h->Y, h->boundary,
                                           h->feature, s, h->err_dev, st);
    } else if (h->prec == SAL_FP32) {
        e = sal::spectra_f32_launch(h->n, h->tw, h->f32_wt, V, out, h->T, h->X, h->Y, h->boundary, h->feature, s,
                                    h->taper, st);
    } else {
        const float* vt = padded_copy(h, V, st, e);
        if (e == cudaSuccess)
            e = sal::spectra_tc_launch(h->n, h->prec == SAL_BF16 ? 1 : 0, h->tc_tables, V, out, h->T, h->X, h->Y,
                                       h->boundary, h->feature, s, vt, h->ypad, h->err_dev, st);
    }
    if (e != cudaSuccess || s == 1) return e;
    return sal::upsample_launch(h->Ec, E, h->T, h->X, h->Y, s, st);
}

}  // namespace

void sal::set_unbound_error(const std::string& msg) { g_create_error = msg; }

int sal::device_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || sms < 1)
        return 1;
    return sms;
}

static std::atomic<unsigned long long> g_launches{0};
void sal::note_launches(int k) { g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed); }

extern "C" {

sal_status sal_directional_window(int n_directions, const int* directions, int radius, double sigma, int cap,
                                  int* n_offsets, int* offsets, float* gauss_w, int* dir_id) {
    // the t, x and t-x directions of Fig. 4
    static const int kFig4[3][3] = {{1, 0, 0}, {0, 1, 0}, {1, 1, 0}};
    if (!n_offsets || !offsets || !gauss_w || !dir_id)
        return fail(nullptr, SAL_ERR_INVALID_ARG, "window output arrays must not be NULL");
    if (n_directions == 0 && directions == nullptr) {
        n_directions = 3;
        directions = &kFig4[0][0];
    }
    if (n_directions < 1 || n_directions > sal::kMaxDirs || !directions)
        return fail(nullptr, SAL_ERR_INVALID_ARG, "n_directions must be in [1, 16] with directions given");
    if (radius < 1) return fail(nullptr, SAL_ERR_INVALID_ARG, "radius must be >= 1");
    if (!(sigma > 0.0) || !std::isfinite(sigma))
        return fail(nullptr, SAL_ERR_INVALID_ARG, "sigma must be finite and > 0");
    const long long Q = 2LL * radius * n_directions;
    if (Q > sal::kMaxOffsets || Q > cap)
        return fail(nullptr, SAL_ERR_INVALID_ARG, "the window holds " + std::to_string(Q) + " neighbours (limit " +
                                                      std::to_string(std::min(cap, sal::kMaxOffsets)) + ")");
    int q = 0;
    for (int d = 0; d < n_directions; ++d) {
        const int* v = directions + 3 * d;
        if (v[0] == 0 && v[1] == 0 && v[2] == 0) return fail(nullptr, SAL_ERR_INVALID_ARG, "a direction is zero");
        for (int sgn = -radius; sgn <= radius; ++sgn) {
            if (sgn == 0) continue;
            long long r2 = 0;
            for (int a = 0; a < 3; ++a) {
                const long long c = (long long)sgn * v[a];
                if (c < -sal::kMaxHalo || c > sal::kMaxHalo)
                    return fail(nullptr, SAL_ERR_INVALID_ARG, "a neighbour component exceeds +-8");
                offsets[3 * q + a] = (int)c;
                r2 += c * c;
            }
            gauss_w[q] = (float)std::exp(-(double)r2 / (2.0 * sigma * sigma));
            dir_id[q] = d;
            ++q;
        }
    }
    *n_offsets = q;
    g_create_error.clear();
    return SAL_OK;
}

sal_status sal_create(const sal_params* p_in, int T, int X, int Y, sal_handle** out) {
    g_create_error.clear();
    if (!out) return fail(nullptr, SAL_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!p_in) return fail(nullptr, SAL_ERR_INVALID_ARG, "params is NULL");
    // n_offsets = 0: the window of Eq. 3 / Fig. 4 is built here from the direction fields
    sal_params pw = *p_in;
    int w_offs[3 * sal::kMaxOffsets], w_dir[sal::kMaxOffsets];
    float w_g[sal::kMaxOffsets];
    std::vector<float> w_alpha;
    if (p_in->n_offsets == 0) {
        const sal_status ws = sal_directional_window(p_in->n_directions, p_in->directions, p_in->radius,
                                                     p_in->sigma, sal::kMaxOffsets, &pw.n_offsets, w_offs, w_g,
                                                     w_dir);
        if (ws != SAL_OK) return ws;
        pw.offsets = w_offs;
        pw.gauss_w = w_g;
        pw.dir_id = w_dir;
        pw.n_dirs = p_in->n_directions == 0 && p_in->directions == nullptr ? 3 : p_in->n_directions;
        if (!p_in->alpha) {
            w_alpha.assign(pw.n_dirs, 1.0f);
            pw.alpha = w_alpha.data();
        }
    }
    const sal_params* p = &pw;
    if (T < 1 || X < 1 || Y < 1) return fail(nullptr, SAL_ERR_INVALID_ARG, "T, X, Y must be >= 1");
    if (T > 65535 || X > 65535) return fail(nullptr, SAL_ERR_UNSUPPORTED, "T and X must be <= 65535");
    if (p->n < 2 || (p->n & 1) || p->n > sal::kMaxN)
        return fail(nullptr, SAL_ERR_INVALID_ARG, "n must be even, 2 <= n <= 32");
    if (p->stride < 1 || (p->stride > 1 && 2 * p->stride >= p->n))
        return fail(nullptr, SAL_ERR_INVALID_ARG, "stride must be 1 or satisfy 1 < stride < n/2 (overlap > 50%)");
    if (p->taper != 0 && p->taper != 1) return fail(nullptr, SAL_ERR_INVALID_ARG, "taper must be 0 or 1");
    if (p->boundary < 0 || p->boundary > 2) return fail(nullptr, SAL_ERR_INVALID_ARG, "bad boundary");
    if (p->feature < 0 || p->feature > 2)
        return fail(nullptr, SAL_ERR_INVALID_ARG,
                    "feature must be 0 (mean of |F_m|), 1 (mean of |F_m|^2) or 2 (mean of |IDFT(F_m)|)");
    if (p->feature == 2 && (p->prec != SAL_FP32 || !sal::spatial_f32_supported(p->n) || p->stride != 1))
        return fail(nullptr, SAL_ERR_UNSUPPORTED, "feature 2 is built for FP32, n in {2, 4, 8, 16}, stride 1");
    if (p->prec < 0 || p->prec > 2) return fail(nullptr, SAL_ERR_INVALID_ARG, "bad precision");
    if (!sal::spectra_f32_supported(p->n) && p->n != 32)
        return fail(nullptr, SAL_ERR_UNSUPPORTED, "FP32 path is built for n in {2,4,8,16,32}");
    if (p->prec != SAL_FP32 && !sal::spectra_tc_supported(p->n) && p->n != 32)
        return fail(nullptr, SAL_ERR_UNSUPPORTED, "BF16/FP16 tensor-core path is built for n in {8,16,32}");
    if (p->n_offsets < 1 || p->n_offsets > sal::kMaxOffsets)
        return fail(nullptr, SAL_ERR_INVALID_ARG, "n_offsets must be in [1, 64]");
    if (p->n_dirs < 1 || p->n_dirs > sal::kMaxDirs)
        return fail(nullptr, SAL_ERR_INVALID_ARG, "n_dirs must be in [1, 16]");
    if (!p->offsets || !p->gauss_w || !p->dir_id || !p->alpha)
        return fail(nullptr, SAL_ERR_INVALID_ARG, "stencil arrays must not be NULL");
    if (!(p->ls_delta >= 0.0) || !std::isfinite(p->ls_delta))
        return fail(nullptr, SAL_ERR_INVALID_ARG, "ls_delta must be finite and >= 0");

    sal_handle* h = new sal_handle();
    h->T = T; h->X = X; h->Y = Y;
    h->N = (long long)T * X * Y;
    h->n = p->n; h->taper = p->taper; h->boundary = p->boundary; h->feature = p->feature; h->stride = p->stride;
    h->prec = p->prec; h->ls_delta = p->ls_delta; h->budget = p->hbm_budget_bytes;
    h->st.Q = p->n_offsets;
    h->st.n_dirs = p->n_dirs;
    h->st.invQ = 1.0f / (float)p->n_offsets;
    for (int o = 0; o < p->n_offsets; ++o) {
        for (int a = 0; a < 3; ++a) {
            const int v = p->offsets[3 * o + a];
            if (v < -sal::kMaxHalo || v > sal::kMaxHalo) {
                delete h;
                return fail(nullptr, SAL_ERR_INVALID_ARG, "stencil offset component beyond +-8");
            }
            h->st.off[o][a] = v;
            h->st.halo[a] = std::max(h->st.halo[a], v < 0 ? -v : v);
        }
        if (p->dir_id[o] < 0 || p->dir_id[o] >= p->n_dirs) {
            delete h;
            return fail(nullptr, SAL_ERR_INVALID_ARG, "dir_id out of range");
        }
        if (!std::isfinite(p->gauss_w[o])) {
            delete h;
            return fail(nullptr, SAL_ERR_INVALID_ARG, "gauss_w must be finite");
        }
        h->st.dir[o] = p->dir_id[o];
        h->st.g[o] = p->gauss_w[o];
    }
    h->alpha.assign(p->alpha, p->alpha + p->n_dirs);
    for (float a : h->alpha)
        if (!std::isfinite(a)) {
            delete h;
            return fail(nullptr, SAL_ERR_INVALID_ARG, "alpha must be finite");
        }
    refresh_weights(h);
    build_twiddles(h);

    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) { delete h; return cuda_fail(nullptr, e, "cudaGetDevice"); }
    if (h->n == 32) {
        // forward only: the backward of the 32^3 window is not built
        e = h->prec == SAL_FP32 ? sal::spectra_f32_n32_prepare() : sal::spectra_tc32_prepare(h->prec == SAL_BF16 ? 1 : 0);
    } else {
        e = sal::spectra_f32_prepare(h->n);
        if (e == cudaSuccess) e = sal::spectra_adjoint_f32_prepare(h->n);
        if (e == cudaSuccess && h->prec != SAL_FP32) e = sal::spectra_tc_prepare(h->n, h->prec == SAL_BF16 ? 1 : 0);
        if (e == cudaSuccess && h->prec != SAL_FP32) e = sal::spectra_adjoint_tc_prepare(h->n, 0);
    }
    if (e == cudaSuccess && h->feature == 2) e = sal::spatial_f32_prepare();
    if (e == cudaSuccess) e = sal::dcs_prepare();
    if (e == cudaSuccess) e = sal::dcs_adjoint_prepare();
    if (e != cudaSuccess) { delete h; return cuda_fail(nullptr, e, "kernel attributes"); }

    const size_t plane3 = (size_t)3 * h->N * sizeof(float);
    const size_t small = (size_t)sal::kRedBlocks * 8 * sizeof(float) + (size_t)sal::kRedBlocks * 16 * sizeof(double)
                         + 32 * sizeof(float) + 16 * sizeof(double) + 256;
    const bool tc_fwd = h->prec != SAL_FP32 && sal::spectra_tc_supported(h->n);
    const size_t tab_bytes = tc_fwd ? sal::spectra_tc_tables_bytes(h->n) : 0;
    const size_t adj_bytes = tc_fwd ? sal::spectra_adjoint_tc_tables_bytes(h->n) : 0;
    const bool f32_tab = h->prec == SAL_FP32 && sal::spectra_f32_supported(h->n) && h->feature != 2;
    const size_t wt_bytes = f32_tab ? sal::f32_weight_table_floats(h->n) * sizeof(float) : 0;
    const size_t sp_bytes = h->feature == 2 ? sal::spatial_weight_table_floats(h->n) * sizeof(float) : 0;
    const int sc = p->stride;
    const size_t ec_bytes = sc > 1 ? (size_t)3 * ((T + sc - 1) / sc) * ((X + sc - 1) / sc) * ((Y + sc - 1) / sc) *
                                         sizeof(float)
                                   : 0;
    // the tensor-core forms stage interior bricks by TMA from a row-padded copy when rows are not 16-byte multiples
    const int ypad = (Y + 3) & ~3;
    const size_t vpad_bytes = tc_fwd && h->feature != 2 && ypad != Y ? (size_t)T * X * ypad * sizeof(float) : 0;
    const size_t need = 2 * plane3 + small + tab_bytes + adj_bytes + ec_bytes + wt_bytes + sp_bytes + vpad_bytes;
    if (h->budget && need > h->budget) {
        delete h;
        return fail(nullptr, SAL_ERR_OOM, "scratch (" + std::to_string(need) + " B) exceeds hbm_budget_bytes");
    }
    if ((e = cudaMalloc(&h->E, plane3)) != cudaSuccess || (e = cudaMalloc(&h->S3, plane3)) != cudaSuccess ||
        (e = cudaMalloc(&h->small, small)) != cudaSuccess ||
        (ec_bytes && (e = cudaMalloc(&h->Ec, ec_bytes)) != cudaSuccess) ||
        (vpad_bytes && (e = cudaMalloc(&h->vpad, vpad_bytes)) != cudaSuccess)) {
        free_scratch(h);
        delete h;
        cudaGetLastError();
        return fail(nullptr, SAL_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    {
        void* hp = nullptr;
        if ((e = cudaHostAlloc(&hp, sizeof(int), cudaHostAllocMapped)) != cudaSuccess ||
            (e = cudaHostGetDevicePointer((void**)&h->err_dev, hp, 0)) != cudaSuccess) {
            if (hp) cudaFreeHost(hp);
            free_scratch(h);
            delete h;
            return cuda_fail(nullptr, e, "error word");
        }
        h->err_host = static_cast<volatile int*>(hp);
        *h->err_host = 0;
    }
    h->ypad = h->vpad ? ypad : 0;
    char* b = static_cast<char*>(h->small);
    h->red.g_part = reinterpret_cast<double*>(b);
    b += (size_t)sal::kRedBlocks * 16 * sizeof(double);
    h->red.wsum = reinterpret_cast<double*>(b);
    b += 16 * sizeof(double);
    h->red.mm_part = reinterpret_cast<float*>(b);
    b += (size_t)sal::kRedBlocks * 8 * sizeof(float);
    h->red.norm = reinterpret_cast<float*>(b);
    {
        // norm layout: [0..10] bounds and weights, [12..14] gradient coefficients, [16..18] ones
        float init[32] = {0.f};
        init[16] = init[17] = init[18] = 1.f;
        if ((e = cudaMemcpy(h->red.norm, init, sizeof(init), cudaMemcpyHostToDevice)) != cudaSuccess) {
            free_scratch(h);
            delete h;
            return cuda_fail(nullptr, e, "cudaMemcpy");
        }
    }
    if (tc_fwd) {
        if ((e = cudaMalloc(&h->tc_tables, tab_bytes)) != cudaSuccess) {
            free_scratch(h);
            delete h;
            cudaGetLastError();
            return fail(nullptr, SAL_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        if ((e = cudaMalloc(&h->adj_tables, adj_bytes)) != cudaSuccess) {
            free_scratch(h);
            delete h;
            cudaGetLastError();
            return fail(nullptr, SAL_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        if ((e = sal::spectra_tc_tables_build(h->n, h->prec == SAL_BF16 ? 1 : 0, h->tw, h->feature, h->tc_tables,
                                              0)) != cudaSuccess ||
            (e = sal::spectra_adjoint_tc_tables_build(h->n, h->tw, h->feature, h->adj_tables, 0)) != cudaSuccess ||
            (e = cudaStreamSynchronize(0)) != cudaSuccess) {
            free_scratch(h);
            delete h;
            return cuda_fail(nullptr, e, "tensor-core tables");
        }
    }
    if (f32_tab) {
        std::vector<float> wt(sal::f32_weight_table_floats(h->n));
        sal::f32_weight_table_fill(h->n, h->feature, wt.data());
        if ((e = cudaMalloc(&h->f32_wt, wt_bytes)) != cudaSuccess) {
            free_scratch(h);
            delete h;
            cudaGetLastError();
            return fail(nullptr, SAL_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        if ((e = cudaMemcpy(h->f32_wt, wt.data(), wt_bytes, cudaMemcpyHostToDevice)) != cudaSuccess) {
            free_scratch(h);
            delete h;
            return cuda_fail(nullptr, e, "cudaMemcpy");
        }
    }
    if (sp_bytes) {
        std::vector<float> rt(sal::spatial_weight_table_floats(h->n));
        sal::spatial_weight_table_fill(h->n, rt.data());
        if ((e = cudaMalloc(&h->sp_tab, sp_bytes)) != cudaSuccess) {
            free_scratch(h);
            delete h;
            cudaGetLastError();
            return fail(nullptr, SAL_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        if ((e = cudaMemcpy(h->sp_tab, rt.data(), sp_bytes, cudaMemcpyHostToDevice)) != cudaSuccess) {
            free_scratch(h);
            delete h;
            return cuda_fail(nullptr, e, "cudaMemcpy");
        }
    }
    h->bytes = need;
    *out = h;
    return SAL_OK;
}

sal_status sal_destroy(sal_handle* h) {
    if (!h) return SAL_OK;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    free_scratch(h);
    delete h;
    return SAL_OK;
}

sal_status sal_workspace_size(const sal_handle* h, size_t* bytes) {
    if (!h || !bytes) return SAL_ERR_INVALID_ARG;
    *bytes = h->bytes;
    return SAL_OK;
}

sal_status sal_check_bounded_wait(sal_handle* h, unsigned tries, void* stream) {
    sal_status st = check_handle(h);
    if (st != SAL_OK) return st;
    if (tries < 1 || tries > (1u << 20)) return fail(h, SAL_ERR_INVALID_ARG, "tries must be in [1, 2^20]");
    cudaError_t e = sal::wait_check_launch(h->err_dev, tries, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(h, e, "wait check launch");
    return SAL_OK;
}

sal_status sal_set_alpha(sal_handle* h, const float* alpha) {
    if (!h) return SAL_ERR_INVALID_ARG;
    if (!alpha) return fail(h, SAL_ERR_INVALID_ARG, "alpha is NULL");
    for (int d = 0; d < h->st.n_dirs; ++d)
        if (!std::isfinite(alpha[d])) return fail(h, SAL_ERR_INVALID_ARG, "alpha must be finite");
    h->alpha.assign(alpha, alpha + h->st.n_dirs);
    refresh_weights(h);
    return SAL_OK;
}

sal_status sal_local_spectra_project(sal_handle* h, const float* V, float* E, void* stream) {
    sal_status s = check_handle(h);
    if (s != SAL_OK) return s;
    if (!V || !E) return fail(h, SAL_ERR_INVALID_ARG, "V and E must not be NULL");
    cudaError_t e = launch_k1(h, V, E, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SAL_OK : cuda_fail(h, e, "local_spectra_project launch");
}

sal_status sal_center_surround(sal_handle* h, const float* E, float* S3, void* stream) {
    sal_status s = check_handle(h);
    if (s != SAL_OK) return s;
    if (!E || !S3) return fail(h, SAL_ERR_INVALID_ARG, "E and S3 must not be NULL");
    cudaError_t e = sal::dcs_launch(E, S3, h->T, h->X, h->Y, h->boundary, h->st, h->red.mm_part,
                                    static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SAL_OK : cuda_fail(h, e, "center_surround launch");
}

sal_status sal_combine(sal_handle* h, const float* S3, const float* D, const float* W_in, float* W_out, float* S,
                       void* stream) {
    sal_status s = check_handle(h);
    if (s != SAL_OK) return s;
    if (!S3 || !S) return fail(h, SAL_ERR_INVALID_ARG, "S3 and S must not be NULL");
    cudaError_t e = sal::combine_launch(S3, D, W_in, W_out, S, h->N, h->ls_delta, false, h->red,
                                        static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SAL_OK : cuda_fail(h, e, "combine launch");
}

sal_status sal_saliency(sal_handle* h, const float* V, const float* D, const float* W_in, float* S, float* S3_opt,
                        float* E_opt, float* W_out, void* stream) {
    sal_status s = check_handle(h);
    if (s != SAL_OK) return s;
    if (!V || !S) return fail(h, SAL_ERR_INVALID_ARG, "V and S must not be NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float* E = E_opt ? E_opt : h->E;
    float* S3 = S3_opt ? S3_opt : h->S3;
    cudaError_t e = launch_k1(h, V, E, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "local_spectra_project launch");
    e = sal::dcs_launch(E, S3, h->T, h->X, h->Y, h->boundary, h->st, h->red.mm_part, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "center_surround launch");
    e = sal::combine_launch(S3, D, W_in, W_out, S, h->N, h->ls_delta, true, h->red, st);
    return e == cudaSuccess ? SAL_OK : cuda_fail(h, e, "combine launch");
}

namespace {

constexpr size_t kBlocksCap = (size_t)2 << 30;  // brick-block scratch of the spectral adjoint (per slab)

// Brick geometry of the spectral adjoint in the handle's precision.
sal::SpectraAdjointGeometry adjoint_geometry(const sal_handle* h) {
    if (h->feature == 2) return sal::spatial_adjoint_f32_geometry(h->n);
    return h->prec == SAL_FP32 ? sal::spectra_adjoint_f32_geometry(h->n) : sal::spectra_adjoint_tc_geometry(h->n);
}

sal_status ensure_backward_scratch(sal_handle* h) {
    if (h->n == 32) return fail(h, SAL_ERR_UNSUPPORTED, "the backward is built for n in {2,4,8,16}");
    if (h->gE) return SAL_OK;
    const sal::SpectraAdjointGeometry g = adjoint_geometry(h);
    const int nseg = (h->Y + g.BY - 1) / g.BY;
    const size_t per_t = (size_t)((h->X + g.BX - 1) / g.BX) * nseg * g.block_floats * sizeof(float);
    // the overlap-add's scratch: one brick-summed plane per extended plane of the slab (s (slab - 1) + n,
    // s the stride: the bricks of a slab sit on the lattice planes)
    const int sc = h->stride;
    const size_t per_ext = sal::gather_ext_floats(h->n, g, h->X, h->Y, 1, 1) / h->n * sizeof(float);
    const size_t ext_fixed = (size_t)(h->n - sc) * per_ext;
    const int planes = (h->T + sc - 1) / sc;   // lattice planes (every plane at stride 1)
    size_t cap = kBlocksCap;
    const size_t plane3 = (size_t)3 * h->N * sizeof(float);
    const size_t lat3 = sc > 1 ? plane3 : 0;
    const size_t bpart = (size_t)sal::kRedBlocks * 64 * sizeof(double);
    if (h->budget) {
        const size_t used = h->bytes + plane3 + lat3 + bpart + ext_fixed;
        if (used + per_t + sc * per_ext > h->budget)
            return fail(h, SAL_ERR_OOM, "backward scratch exceeds hbm_budget_bytes");
        cap = std::min(cap, h->budget - used);
    }
    int slab = (int)std::max<size_t>(1, std::min<size_t>((size_t)planes, cap / (per_t + sc * per_ext)));
    const size_t ext_bytes = sal::gather_ext_floats(h->n, g, h->X, h->Y, slab, sc) * sizeof(float);
    cudaError_t e;
    if ((e = cudaMalloc(&h->gE, plane3)) != cudaSuccess || (e = cudaMalloc(&h->bpart, bpart)) != cudaSuccess ||
        (e = cudaMalloc(&h->blocks, per_t * slab)) != cudaSuccess ||
        (e = cudaMalloc(&h->gext, ext_bytes)) != cudaSuccess ||
        (lat3 && (e = cudaMalloc(&h->gEl, lat3)) != cudaSuccess)) {
        if (h->gE) cudaFree(h->gE);
        if (h->bpart) cudaFree(h->bpart);
        if (h->blocks) cudaFree(h->blocks);
        if (h->gext) cudaFree(h->gext);
        h->gE = h->blocks = h->gext = nullptr;
        h->bpart = nullptr;
        cudaGetLastError();
        return fail(h, SAL_ERR_OOM, std::string("backward scratch cudaMalloc: ") + cudaGetErrorString(e));
    }
    h->slab_t = slab;   // lattice planes per slab
    h->blocks_bytes = per_t * slab;
    h->bytes += plane3 + lat3 + bpart + per_t * slab + ext_bytes;
    return SAL_OK;
}

// gV = (dE/dV)^T gE through the brick blocks of K5 and the fixed-order overlap-add, slab by slab.
sal_status spectral_adjoint(sal_handle* h, const float* V, const float* gE, float* gV, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(gV, 0, (size_t)h->N * sizeof(float), st)) != cudaSuccess)
        return cuda_fail(h, e, "spectral adjoint: memset");
    const int sc = h->stride;
    if (sc > 1) {
        // stride s: the gradient of the interpolated features back onto the lattice voxels; the cubes of
        // the other voxels were never taken, so only the bricks of the lattice planes run
        if ((e = cudaMemsetAsync(h->gEl, 0, (size_t)3 * h->N * sizeof(float), st)) != cudaSuccess ||
            (e = sal::upsample_adjoint_launch(gE, h->gEl, h->T, h->X, h->Y, sc, st)) != cudaSuccess)
            return cuda_fail(h, e, "spectral adjoint: interpolation adjoint");
        gE = h->gEl;
    }
    const sal::SpectraAdjointGeometry g = adjoint_geometry(h);
    const int planes = (h->T + sc - 1) / sc;
    const float* vt = nullptr;
    if (h->prec != SAL_FP32) {
        vt = padded_copy(h, V, st, e);
        if (e != cudaSuccess) return cuda_fail(h, e, "spectral adjoint: padded copy");
    }
    // the FP32 adjoint lists its small bins in the overlap-add's plane buffer, free until the gather runs
    const size_t ext_bytes = sal::gather_ext_floats(h->n, g, h->X, h->Y, h->slab_t, sc) * sizeof(float);
    int* lists = h->prec == SAL_FP32 && h->feature == 0 &&
                         sal::spectra_adjoint_f32_list_bytes(h->n, h->X, h->Y, h->slab_t) <= ext_bytes
                     ? reinterpret_cast<int*>(h->gext)
                     : nullptr;
    for (int p0 = 0; p0 < planes; p0 += h->slab_t) {
        const int cnt = std::min(h->slab_t, planes - p0), t_begin = p0 * sc;
        e = h->feature == 2
                ? sal::spatial_adjoint_f32_launch(h->n, h->sp_tab, V, gE, h->blocks, h->T, h->X, h->Y, h->boundary, t_begin, cnt,
                                                  h->taper, st)
            : h->prec == SAL_FP32
                ? sal::spectra_adjoint_f32_launch(h->n, h->tw, h->f32_wt, V, gE, h->blocks, h->T, h->X, h->Y,
                                                  h->boundary, h->feature, t_begin, sc, cnt, h->taper, lists, st)
                // the adjoint's 16-bit operands are FP16 in both 16-bit forms: the direction F/|F| of
                // small bins amplifies operand rounding, and FP16 carries 3 more mantissa bits
                : sal::spectra_adjoint_tc_launch(h->n, 0, h->tw, h->adj_tables, V, gE, h->blocks, h->T, h->X, h->Y,
                                                 h->boundary, h->feature, t_begin, sc, cnt, vt, h->ypad, h->err_dev,
                                                 st);
        if (e != cudaSuccess) return cuda_fail(h, e, "spectral adjoint");
        if ((e = sal::gather_add_launch(h->blocks, h->gext, gV, h->T, h->X, h->Y, h->boundary, h->n, g, t_begin, cnt,
                                        sc, st)) != cudaSuccess)
            return cuda_fail(h, e, "spectral adjoint: overlap-add");
    }
    return SAL_OK;
}

}  // namespace

sal_status sal_saliency_backward(sal_handle* h, const float* V, const float* W, const float* gS, float* gV,
                                 float* gW, float* galpha, void* stream) {
    sal_status s = check_handle(h);
    if (s != SAL_OK) return s;
    if (!V || !W || !gS) return fail(h, SAL_ERR_INVALID_ARG, "V, W and gS must not be NULL");
    if ((s = ensure_backward_scratch(h)) != SAL_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    // forward recompute: features, raw maps, normalisation bounds for the given weights
    if ((e = launch_k1(h, V, h->E, st)) != cudaSuccess) return cuda_fail(h, e, "backward: local_spectra_project");
    if ((e = sal::dcs_launch(h->E, h->S3, h->T, h->X, h->Y, h->boundary, h->st, h->red.mm_part, st)) != cudaSuccess)
        return cuda_fail(h, e, "backward: center_surround");
    // the combined map itself is not needed: gE's first plane holds it until K4 overwrites it
    if ((e = sal::combine_launch(h->S3, nullptr, W, nullptr, h->gE, h->N, h->ls_delta, true, h->red, st)) !=
        cudaSuccess)
        return cuda_fail(h, e, "backward: combine");
    float* coef = h->red.norm + 12;
    if ((e = sal::backward_weights_launch(h->S3, gS, h->N, h->red, h->bpart, coef, gW, st)) != cudaSuccess)
        return cuda_fail(h, e, "backward: weights");
    if (galpha && gV) {
        // one pass for both gradients (the brick scratch holds the per-tile partials until K5 needs it)
        if ((e = sal::dcs_adjoint_galpha_launch(h->E, gS, 0, coef, h->gE, h->T, h->X, h->Y, h->boundary, h->st,
                                                reinterpret_cast<double*>(h->blocks), h->blocks_bytes, h->bpart,
                                                galpha, st)) != cudaSuccess)
            return cuda_fail(h, e, "backward: center_surround adjoint and alpha");
        return spectral_adjoint(h, V, h->gE, gV, st);
    }
    if (galpha &&
        (e = sal::dcs_galpha_launch(h->E, gS, 0, coef, h->T, h->X, h->Y, h->boundary, h->st, h->bpart, galpha, st)) !=
            cudaSuccess)
        return cuda_fail(h, e, "backward: alpha");
    if (!gV) return SAL_OK;
    if ((e = sal::dcs_adjoint_launch(h->E, gS, 0, coef, h->gE, h->T, h->X, h->Y, h->boundary, h->st, st)) !=
        cudaSuccess)
        return cuda_fail(h, e, "backward: center_surround adjoint");
    return spectral_adjoint(h, V, h->gE, gV, st);
}

sal_status sal_local_spectra_project_backward(sal_handle* h, const float* V, const float* gE, float* gV,
                                              void* stream) {
    sal_status s = check_handle(h);
    if (s != SAL_OK) return s;
    if (!V || !gE || !gV) return fail(h, SAL_ERR_INVALID_ARG, "V, gE and gV must not be NULL");
    if ((s = ensure_backward_scratch(h)) != SAL_OK) return s;
    return spectral_adjoint(h, V, gE, gV, static_cast<cudaStream_t>(stream));
}

sal_status sal_center_surround_backward(sal_handle* h, const float* E, const float* gS3, float* gE, float* galpha,
                                        void* stream) {
    sal_status s = check_handle(h);
    if (s != SAL_OK) return s;
    if (!E || !gS3) return fail(h, SAL_ERR_INVALID_ARG, "E and gS3 must not be NULL");
    if ((s = ensure_backward_scratch(h)) != SAL_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    const float* ones = h->red.norm + 16;
    if (galpha && gE) {
        if ((e = sal::dcs_adjoint_galpha_launch(E, gS3, h->N, ones, gE, h->T, h->X, h->Y, h->boundary, h->st,
                                                reinterpret_cast<double*>(h->blocks), h->blocks_bytes, h->bpart,
                                                galpha, st)) != cudaSuccess)
            return cuda_fail(h, e, "center_surround_backward");
        return SAL_OK;
    }
    if (galpha && (e = sal::dcs_galpha_launch(E, gS3, h->N, ones, h->T, h->X, h->Y, h->boundary, h->st, h->bpart,
                                             galpha, st)) != cudaSuccess)
        return cuda_fail(h, e, "center_surround_backward: alpha");
    if (gE && (e = sal::dcs_adjoint_launch(E, gS3, h->N, ones, gE, h->T, h->X, h->Y, h->boundary, h->st, st)) !=
                  cudaSuccess)
        return cuda_fail(h, e, "center_surround_backward");
    return SAL_OK;
}

sal_status sal_adapt_weights(sal_handle* h, const float* S3, const float* D, const sal_adapt_params* p,
                             float* W_out, float* err2, void* stream) {
    sal_status s = check_handle(h);
    if (s != SAL_OK) return s;
    if (!S3 || !D || !p || !W_out) return fail(h, SAL_ERR_INVALID_ARG, "S3, D, params and W_out must not be NULL");
    if (p->method != SAL_ADAPT_LMS && p->method != SAL_ADAPT_NLMS && p->method != SAL_ADAPT_RLS)
        return fail(h, SAL_ERR_INVALID_ARG, "unknown adaptive method");
    if (p->sections < 0) return fail(h, SAL_ERR_INVALID_ARG, "sections must be >= 0");
    if (!std::isfinite(p->mu) || !std::isfinite(p->eps) || !(p->eps >= 0.0) || !std::isfinite(p->lambda) ||
        !(p->lambda > 0.0) || !std::isfinite(p->delta) || !(p->delta > 0.0))
        return fail(h, SAL_ERR_INVALID_ARG, "mu, eps >= 0, lambda > 0 and delta > 0 must be finite");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if ((e = sal::minmax_bounds_launch(S3, h->N, h->red, st)) != cudaSuccess) return cuda_fail(h, e, "adapt: bounds");
    if ((e = sal::adapt_launch(S3, D, h->T, h->X, h->Y, (int)p->method, p->mu, p->eps, p->lambda, p->delta,
                               p->sections, h->red.norm, W_out, err2, st)) != cudaSuccess)
        return cuda_fail(h, e, "adapt");
    return SAL_OK;
}

sal_status sal_combine_backward(sal_handle* h, const float* S3, const float* W, const float* gS, float* gS3,
                                float* gW, void* stream) {
    sal_status s = check_handle(h);
    if (s != SAL_OK) return s;
    if (!S3 || !W || !gS || !gS3) return fail(h, SAL_ERR_INVALID_ARG, "S3, W, gS and gS3 must not be NULL");
    if ((s = ensure_backward_scratch(h)) != SAL_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    // bounds of the forward combination; its map goes to gS3's first plane until overwritten
    if ((e = sal::combine_launch(S3, nullptr, W, nullptr, gS3, h->N, h->ls_delta, false, h->red, st)) != cudaSuccess)
        return cuda_fail(h, e, "combine_backward: bounds");
    float* coef = h->red.norm + 12;
    if ((e = sal::backward_weights_launch(S3, gS, h->N, h->red, h->bpart, coef, gW, st)) != cudaSuccess)
        return cuda_fail(h, e, "combine_backward: weights");
    if ((e = sal::expand_gradient_launch(gS, coef, gS3, h->N, st)) != cudaSuccess)
        return cuda_fail(h, e, "combine_backward: expand");
    return SAL_OK;
}

sal_status sal_launch_count(unsigned long long* count) {
    if (!count) return SAL_ERR_INVALID_ARG;
    *count = g_launches.load(std::memory_order_relaxed);
    return SAL_OK;
}

const char* sal_last_error(const sal_handle* h) {
    return h ? h->last.c_str() : g_create_error.c_str();
}

}  // extern "C"
