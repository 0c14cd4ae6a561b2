// Failure-detection self-test of the device-side bounded waits.  One thread
// waits, with the same bounded mbarrier wait every pipelined kernel of the
// library uses, on a barrier that nothing ever arrives at.  The wait can
// only end by its time limit: it records ADV_DEV_TIMEOUT in the model's
// status word and the kernel returns.  No copy is in flight and no tensor
// memory is held, so the context stays usable afterwards.
#include "common.cuh"
#include "selftest.cuh"

namespace adv {

__global__ void wait_timeout_check_kernel(int* status_word, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_s;
    mbar_init(&bar, 1);
    abort_s = 0;
    fence_mbar_init();
    // the wait is bounded by %globaltimer: first make sure, under an
    // iteration cap, that the timer advances (otherwise leave the status
    // word untouched, which the caller reads as a failed check)
    const uint64_t t0 = global_timer_ns();
    bool moves = false;
    for (int it = 0; it < (1 << 22) && !moves; ++it) moves = global_timer_ns() != t0;
    if (!moves) return;
    mbar_wait_bounded(&bar, 0u, status_word, &abort_s, limit_ns);   // phase 0 never completes
}

cudaError_t launch_wait_timeout_check(int* status_word, uint64_t limit_ns, cudaStream_t s) {
    wait_timeout_check_kernel<<<1, 1, 0, s>>>(status_word, limit_ns);
    adv_count_launch(1);
    return cudaGetLastError();
}

}  // namespace adv
