// selftest.cu — a diagnostic of the bounded asynchronous-copy waits.
//
// The TMA-fed kernels (four-step passes, column pass) wait on an mbarrier for
// their copies a bounded number of times and, if the copies never complete,
// record a timeout in the plan's device status word and return instead of
// hanging.  This kernel exercises that path on purpose: it arms an mbarrier
// for 16 bytes that no copy will ever deliver, so its bounded wait runs out.
#include "internal.h"
#include "tma.cuh"

namespace gbfft {

__global__ void k_wait_timeout(int *status, unsigned polls) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    mbar_expect_tx(&bar, 16);  // the one arrival happens; 16 bytes never do
    if (!mbar_wait_bounded(&bar, 0, polls)) atomicExch(status, 1);
}

cudaError_t launch_wait_timeout(int *status, unsigned polls, cudaStream_t s) {
    k_wait_timeout<<<1, 32, 0, s>>>(status, polls);
    return cudaGetLastError();
}

}  // namespace gbfft
