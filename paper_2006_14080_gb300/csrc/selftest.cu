// Self-test of the bounded device-side wait that every mbarrier wait of the
// tensor-core kernels goes through: one thread waits on an mbarrier that no
// thread ever completes, gives up after the limit and records the timeout in
// the plan's deferred status word, exactly as a product kernel does before
// it returns.  Nothing faults or hangs: the wait ends at the limit.
#include "common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace mri {
namespace {

__global__ void bounded_wait_probe_kernel(int *status, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        tc::mbar_init(tc::smem_u32(&bar), 1);
        tc::fence_barrier_init();
        // no arrival ever completes phase 0 of the barrier
        if (!tc::mbar_wait(tc::smem_u32(&bar), 0, &abort_flag, limit_ns)) atomicExch(status, kStatusTimeout);
    }
}

}  // namespace
}  // namespace mri

using namespace mri;

extern "C" {

MRI_API int mri_plan_selftest_wait(mri_plan *p, double limit_ms, mri_stream_t stream) {
    if (!p) return set_error("null plan"), MRI_ERR_INVALID;
    if (!(limit_ms > 0.0) || limit_ms > 1000.0) return set_error("limit_ms must be in (0, 1000]"), MRI_ERR_INVALID;
    bounded_wait_probe_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(&p->scal->status, (uint64_t)(limit_ms * 1e6));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(std::string("bounded-wait probe launch: ") + cudaGetErrorString(e)), MRI_ERR_CUDA;
    p->launches += 1;
    return MRI_OK;
}

}  // extern "C"
