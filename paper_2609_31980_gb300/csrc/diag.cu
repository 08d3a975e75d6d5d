// diag.cu — a check of the device-side failure handling: a bounded wait that
// is made to run out.
//
// Every wait of the query kernels on an mbarrier is bounded in time; when the
// bound is reached the kernel records FRNN_ERR_TIMEOUT in the context's status
// word and returns, so the context stays usable.  k_wait_timeout waits on a
// barrier that nothing ever completes (no thread arrives on it, no copy is
// tied to it), with the same bounded wait, and records the same status.
#include "frnn_host.h"

namespace frnn {

__global__ void k_wait_timeout(uint64_t limit_ns, int32_t* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    fence_mbar_init();
    __syncwarp();
    // phase 0 needs one arrival that never comes
    const bool done = mbar_wait_bounded(&bar, 0u, limit_ns);
    if (!done && threadIdx.x == 0) atomicOr(status, kStatusTimeout);
}

cudaError_t launch_wait_timeout(uint64_t limit_ns, int32_t* status, cudaStream_t st) {
    k_wait_timeout<<<1, 32, 0, st>>>(limit_ns, status);
    return cudaGetLastError();
}

}  // namespace frnn
