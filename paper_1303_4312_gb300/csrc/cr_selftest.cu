// cr_selftest.cu -- test hook for the bounded waits of the merge kernels.
//
// Every mbarrier wait in the tile-merge kernel gives up after a wall-clock
// limit, records CR_ETIMEOUT in the workspace status word and lets the kernel
// return, so a lost copy or a missing arrival can never hang the GPU.  This
// entry point exercises exactly that path on purpose and safely: one thread
// initialises an mbarrier that expects one arrival, never arrives, and waits
// on it with the same bounded wait (mbar_wait) and the caller's limit.  The
// wait must run out, the status word must read CR_ETIMEOUT afterwards, and
// the context stays usable.  The paper has no counterpart.
#include <cuda_runtime.h>

#include "../../include/corank.h"
#include "cr_device.cuh"

namespace {

__global__ void bounded_wait_kernel(void* ws, uint64_t limit_ns, uint64_t* elapsed_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    cr::mbar_init(&bar, 1);
    cr::fence_barrier_init();
    const uint64_t t0 = cr::global_timer_ns();
    const bool done = cr::mbar_wait(&bar, 0, limit_ns);   // nothing ever arrives
    const uint64_t t1 = cr::global_timer_ns();
    if (elapsed_ns) *elapsed_ns = t1 - t0;
    cr::WsHeader* h = static_cast<cr::WsHeader*>(ws);
    h->status = done ? cr::kDevOk : cr::kDevTimeout;
}

}  // namespace

namespace cr {
void set_last_error(const char* msg);   // cr_abi.cu
}

extern "C" cr_status cr_selftest_bounded_wait(void* ws, size_t ws_bytes, uint64_t limit_ns,
                                              uint64_t* d_elapsed_ns, cr_stream stream) {
    if (ws == nullptr || ws_bytes < sizeof(cr::WsHeader) ||
        (reinterpret_cast<uintptr_t>(ws) & 15u) != 0) {
        cr::set_last_error("workspace NULL, too small or not 16-byte aligned");
        return CR_EINVAL;
    }
    if (limit_ns == 0 || limit_ns > 100000000ull) {   // at most 100 ms
        cr::set_last_error("limit_ns must be in [1, 10^8]");
        return CR_EINVAL;
    }
    bounded_wait_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(ws, limit_ns,
                                                                        d_elapsed_ns);
    const cudaError_t e = cudaGetLastError();
    cr::set_last_error(e == cudaSuccess ? "" : cudaGetErrorString(e));
    return e == cudaSuccess ? CR_OK : CR_ECUDA;
}
