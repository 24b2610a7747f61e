// Measured issue rate of the MUFU (XU) pipe for the two operations the |F| epilogues use: the
// roofline denominator of the abs(F) / Gamma epilogues of K1 and K5.  Every thread runs 16
// independent dependency chains of one approximate square root (or reciprocal square root), so the
// pipe, not the latency of a chain, bounds the rate; the grid is 8 CTAs of 256 threads per SM of
// the current device (the SM count comes from the device attribute), timed with CUDA events after
// a warm-up launch.
#include "sal_internal.cuh"

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

}  // namespace
}  // namespace sal

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
