// gtt_selftest_bounded_wait: exercises, on the GPU and without any fault, the
// expiry path of the bounded mbarrier waits that every pipelined kernel of the
// library uses (no counterpart in the paper).
#include "gtt_plan.h"
#include "gtt_tma.cuh"

namespace gtt {

// One warp waits on an mbarrier that nothing arrives on, with the pass
// kernels' try-wait primitive and a poll limit; the expiry is reported in a
// device flag the way the pass kernels report theirs.
__global__ void gtt_wait_selftest_kernel(int *flag, uint32_t polls) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = smem_addr(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);
        fence_mbar_init();
    }
    __syncwarp();
    bool done = false;
    for (uint32_t i = 0; i < polls && !done; ++i) done = mbar_try_wait(b, 0);
    if (threadIdx.x == 0) *flag = done ? 0 : 1;
}

} // namespace gtt

extern "C" gtt_status_t gtt_selftest_bounded_wait(int polls, int *expired, gtt_stream_t stream) {
    using namespace gtt;
    if (polls < 1 || polls > (1 << 20) || !expired)
        return set_error(GTT_ERR_INVALID_ARG, "polls must be in [1, 2^20] and expired non-NULL");
    *expired = 0;
    int *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(int));
    if (e != cudaSuccess) return set_error(GTT_ERR_ALLOC, "self-test flag");
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemsetAsync(d, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        gtt_wait_selftest_kernel<<<1, 32, 0, s>>>(d, (uint32_t)polls);
        e = cudaGetLastError();
    }
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_error(e, "bounded-wait self-test");
    *expired = h;
    return GTT_OK;
}
