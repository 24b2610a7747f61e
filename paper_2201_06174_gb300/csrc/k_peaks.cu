// Measured issue rate of the MUFU (XU) pipe for the two operations the |F| epilogues use: the
// roofline denominator of the abs(F) / Gamma epilogues of K1 and K5.  Every thread runs 16
// independent dependency chains of one approximate square root (or reciprocal square root), so the
// pipe, not the latency of a chain, bounds the rate; the grid is 8 CTAs of 256 threads per SM of
// the current device (the SM count comes from the device attribute), timed with CUDA events after
// a warm-up launch.
//
// Measured cost of one tcgen05.mma (kind::f16, M = 128, K = 16) in SM cycles, by N: the tensor pipe's
// instruction rate, which binds MMAs narrower than the pipe's width long before their flops do.  One CTA
// per SM; one elected lane issues kMmaIters MMAs back to back on constant descriptors (zero operands in
// shared memory, one accumulator in tensor memory), commits them to an mbarrier and waits (bounded);
// clock64 around issue and completion gives the cycles per MMA.
#include <string>
#include <vector>

#include "sal_internal.cuh"
#include "tc_sm100.cuh"

namespace sal {
namespace {

constexpr int kChains = 16;
constexpr int kIters = 2048;

template <int OP>
__global__ void __launch_bounds__(256) k_mufu_rate(float* out) {
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = 1.5f + 0.01f * j + 1e-6f * threadIdx.x;
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) {
            if (OP == 0) asm volatile("sqrt.approx.ftz.f32 %0, %0;" : "+f"(a[j]));
            else asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(a[j]));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

constexpr int kMmaIters = 4096;
constexpr int kMmaSmem = 120 * 1024;   // more than half an SM's shared memory: one CTA per SM

template <int NC>
__global__ void __launch_bounds__(128, 1) k_mma_rate(long long* cycles, int* err) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t s_tmem;
    for (int i = threadIdx.x; i < 16 * 1024 / 16; i += 128) reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
    if (threadIdx.x < 32) tc::tmem_alloc(tc::smem_u32(&s_tmem), 512);
    if (threadIdx.x == 0) tc::mbar_init(tc::smem_u32(&mbar), 1);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    if (threadIdx.x < 32) {
        // A: 128 x 16 and B: NC x 16, K-major, no swizzle (8-row groups of 256 B), both zero
        const uint64_t ad = tc::desc_noswizzle(tc::smem_u32(smem), 128, 256);
        const uint64_t bd = tc::desc_noswizzle(tc::smem_u32(smem) + 4096u, 128, 256);
        constexpr uint32_t idesc = tc::idesc_f16(0, 128, NC, 0, 0);
        const long long c0 = clock64();
        if (tc::elect_one()) {
            for (int i = 0; i < kMmaIters; ++i) tc::mma_f16(tmem, ad, bd, idesc, i > 0 ? 1u : 0u);
            tc::mma_commit(tc::smem_u32(&mbar));
        }
        __syncwarp();
        const bool ok = tc::mbar_wait(tc::smem_u32(&mbar), 0, 1u << 24);
        const long long c1 = clock64();
        if (threadIdx.x == 0) {
            if (!ok) atomicOr(err, 1);
            cycles[blockIdx.x] = c1 - c0;
        }
        if (!ok) tc::mbar_wait(tc::smem_u32(&mbar), 0, 1u << 24);   // nothing in flight at dealloc
    }
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_dealloc(tmem, 512);
}

template <int NC>
cudaError_t mma_rate_run(int sms, long long* cycles, int* err) {
    cudaError_t e = cudaFuncSetAttribute(k_mma_rate<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMmaSmem);
    if (e != cudaSuccess) return e;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first is a warm-up
        k_mma_rate<NC><<<sms, 128, kMmaSmem>>>(cycles, err);
        note_launches(1);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace
}  // namespace sal

extern "C" sal_status sal_measure_mma_rate(int n_cols, double* cycles_per_mma, int* sm_count) {
    sal::set_unbound_error("");
    if (!cycles_per_mma || (n_cols != 16 && n_cols != 32 && n_cols != 64 && n_cols != 128 && n_cols != 256)) {
        sal::set_unbound_error("sal_measure_mma_rate: n_cols must be 16, 32, 64, 128 or 256 and cycles_per_mma not NULL");
        return SAL_ERR_INVALID_ARG;
    }
    int dev = 0, sms = 0, major = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    if (e != cudaSuccess) {
        sal::set_unbound_error(std::string("sal_measure_mma_rate: ") + cudaGetErrorString(e));
        return SAL_ERR_CUDA;
    }
    if (major < 10) {
        sal::set_unbound_error("sal_measure_mma_rate: needs a device with 5th-generation tensor cores");
        return SAL_ERR_UNSUPPORTED;
    }
    long long* cycles = nullptr;
    int* err = nullptr;
    std::vector<long long> h(sms);
    int herr = 0;
    if ((e = cudaMalloc(&cycles, sizeof(long long) * sms)) == cudaSuccess && (e = cudaMalloc(&err, sizeof(int))) == cudaSuccess &&
        (e = cudaMemset(err, 0, sizeof(int))) == cudaSuccess) {
        switch (n_cols) {
            case 16: e = sal::mma_rate_run<16>(sms, cycles, err); break;
            case 32: e = sal::mma_rate_run<32>(sms, cycles, err); break;
            case 64: e = sal::mma_rate_run<64>(sms, cycles, err); break;
            case 128: e = sal::mma_rate_run<128>(sms, cycles, err); break;
            default: e = sal::mma_rate_run<256>(sms, cycles, err); break;
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(h.data(), cycles, sizeof(long long) * sms, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    }
    if (cycles) cudaFree(cycles);
    if (err) cudaFree(err);
    if (e != cudaSuccess) {
        sal::set_unbound_error(std::string("sal_measure_mma_rate: ") + cudaGetErrorString(e));
        return SAL_ERR_CUDA;
    }
    if (herr) {
        sal::set_unbound_error("sal_measure_mma_rate: a bounded wait for the MMAs gave up");
        return SAL_ERR_TIMEOUT;
    }
    double sum = 0.0;
    for (long long c : h) sum += (double)c;
    *cycles_per_mma = sum / sms / sal::kMmaIters;
    if (sm_count) *sm_count = sms;
    return SAL_OK;
}

extern "C" sal_status sal_measure_mufu_rate(int op, double* ops_per_second, int* sm_count) {
    sal::set_unbound_error("");
    if (!ops_per_second || (op != 0 && op != 1)) {
        sal::set_unbound_error("sal_measure_mufu_rate: op must be 0 or 1 and ops_per_second not NULL");
        return SAL_ERR_INVALID_ARG;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        sal::set_unbound_error(std::string("sal_measure_mufu_rate: ") + cudaGetErrorString(e));
        return SAL_ERR_CUDA;
    }
    const int blocks = 8 * sms, threads = 256;
    float* out = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    float ms = 0.f;
    if ((e = cudaMalloc(&out, sizeof(float) * blocks * threads)) == cudaSuccess &&
        (e = cudaEventCreate(&t0)) == cudaSuccess && (e = cudaEventCreate(&t1)) == cudaSuccess) {
        auto launch = [&]() {
            if (op == 0) sal::k_mufu_rate<0><<<blocks, threads>>>(out);
            else sal::k_mufu_rate<1><<<blocks, threads>>>(out);
            sal::note_launches(1);
            return cudaGetLastError();
        };
        e = launch();                                           // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(t0);
        if (e == cudaSuccess) e = launch();
        if (e == cudaSuccess) e = cudaEventRecord(t1);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (out) cudaFree(out);
    if (e != cudaSuccess || !(ms > 0.f)) {
        sal::set_unbound_error(std::string("sal_measure_mufu_rate: ") + cudaGetErrorString(e));
        return SAL_ERR_CUDA;
    }
    *ops_per_second = (double)blocks * threads * sal::kIters * sal::kChains / (ms * 1e-3);
    if (sm_count) *sm_count = sms;
    return SAL_OK;
}
