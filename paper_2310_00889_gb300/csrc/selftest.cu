// Self-test of the bounded-wait path used by the pair-sum kernels.
//
// The pair-sum kernels wait on mbarriers for their bulk copies with a time limit; when a
// copy never lands they set the device error word and leave.  This kernel exercises that
// path without any fault: it initialises an mbarrier that expects bytes no copy will
// deliver, waits on it with the given limit, and records the expiry exactly as the
// pair-sum kernels do.
#include "engine.h"

namespace {

using namespace sbq;

__global__ void bounded_wait_selftest(int *err, unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        mbar_arrive_expect_tx(&bar, 16);   // 16 bytes that nothing will deliver
    __syncthreads();
    const bool timed_out = !mbar_wait_bounded(&bar, 0, limit_ns);
    if (__syncthreads_or(timed_out) && threadIdx.x == 0)
        atomicOr(err, DEV_ERR_TIMEOUT);
}

}  // namespace

extern "C" SBQ_API int sbq_selftest_bounded_wait(int64_t limit_ns, void *stream)
{
    clear_error();
    if (limit_ns <= 0 || limit_ns > 2000000000LL) {
        set_error("limit_ns must be in (0, 2e9]");
        return SBQ_EINVAL;
    }
    int *err = device_error_word();
    if (!err) {
        set_error("cannot allocate the device error word");
        return SBQ_ENOMEM;
    }
    bounded_wait_selftest<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(
        err, static_cast<unsigned long long>(limit_ns));
    SBQ_CUDA(cudaGetLastError());
    return SBQ_OK;
}
