// wait_selftest.cu -- self-test of the bounded waits every pipelined kernel uses (no counterpart
// in the paper).  One thread waits on a freshly initialised mbarrier phase that either completes
// (one arrival, the barrier's count) or never does (no arrival).  In the second case the wait
// must give up after about a second, record kDevErrTimeout in the status word and let the kernel
// return, so that the host reads PTS_ERR_TIMEOUT and the context stays usable.  The waits are
// the library's own helpers: mbar_wait_bounded (single-role kernels) and mbar_wait_or_abort
// (warp-specialised kernels, which also raise an abort flag for the other roles).
#include "tc_common.cuh"

namespace pts {
namespace {

__global__ void k_wait_selftest(int arrive, int abortable, int *status, int *completed) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    if (arrive) mbar_arrive(&bar);
    const bool ok = abortable ? mbar_wait_or_abort(&bar, 0, status, &abort_flag) : mbar_wait_bounded(&bar, 0, status);
    completed[0] = ok ? 1 : 0;
    completed[1] = abort_flag;
}

}  // namespace
}  // namespace pts

using namespace pts;

extern "C" pts_status pts_wait_selftest(int arrive, int abortable, int *completed_out) {
    if (!completed_out) return set_error(PTS_ERR_INVALID_ARG, "pts_wait_selftest: null pointer");
    DevBuf<int> buf;  // [0] status word, [1] completed, [2] abort flag as the kernel left it
    PTS_TRY(buf.ensure(3, "wait self-test"));
    PTS_CUDA_TRY(cudaMemset(buf.ptr, 0, 3 * sizeof(int)));
    count_launches(1);
    k_wait_selftest<<<1, 32>>>(arrive ? 1 : 0, abortable ? 1 : 0, buf.ptr, buf.ptr + 1);
    PTS_CUDA_TRY(cudaGetLastError());
    PTS_CUDA_TRY(cudaDeviceSynchronize());
    int h[3] = {0, 0, 0};
    PTS_CUDA_TRY(cudaMemcpy(h, buf.ptr, sizeof(h), cudaMemcpyDeviceToHost));
    *completed_out = h[1];
    if (h[0] & kDevErrTimeout) {
        if (abortable && !h[2]) return set_error(PTS_ERR_DEVICE, "pts_wait_selftest: timed out without the abort flag");
        return set_error(PTS_ERR_TIMEOUT, "pts_wait_selftest: the wait gave up");
    }
    if (h[0]) return set_error(PTS_ERR_DEVICE, "pts_wait_selftest: unexpected status bits");
    return PTS_OK;
}
