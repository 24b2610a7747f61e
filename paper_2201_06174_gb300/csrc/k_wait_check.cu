// Failure-detection check of the tensor-core kernels' bounded waits.  Every mbarrier wait of those
// kernels gives up after a fixed number of tries, sets the handle's mapped error word and lets the
// CTA leave; the next call on the handle then returns SAL_ERR_TIMEOUT.  This kernel runs that same
// path on purpose and nothing else: one CTA initialises an mbarrier that expects one arrival, makes
// no arrival, waits on it through the same bounded helper with a caller-given number of tries, and on
// giving up sets the error word exactly as the tensor-core kernels do.  It allocates no tensor memory
// and issues no asynchronous copy, so there is nothing in flight when it returns.
#include "sal_internal.cuh"
#include "tc_sm100.cuh"

namespace sal {
namespace {

__global__ void __launch_bounds__(32) k_wait_check(int* __restrict__ err, uint32_t tries) {
    __shared__ __align__(8) uint64_t s_mbar;
    const uint32_t mbar = tc::smem_u32(&s_mbar);
    if (threadIdx.x == 0) tc::mbar_init(mbar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool ok = tc::mbar_wait(mbar, 0, tries);   // phase 0 never completes: no arrival is made
        if (!ok) atomicOr(err, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(mbar) : "memory");
}

}  // namespace

cudaError_t wait_check_launch(int* err, unsigned tries, cudaStream_t s) {
    k_wait_check<<<1, 32, 0, s>>>(err, tries);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace sal
