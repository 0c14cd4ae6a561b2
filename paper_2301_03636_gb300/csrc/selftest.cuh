#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace adv {
// One thread runs the library's bounded mbarrier wait on a barrier nothing
// arrives at; after limit_ns it records ADV_DEV_TIMEOUT in *status_word.
cudaError_t launch_wait_timeout_check(int* status_word, uint64_t limit_ns, cudaStream_t s);
}  // namespace adv
