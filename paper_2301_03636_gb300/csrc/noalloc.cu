// Tensor-core scoring for callers that cannot allocate device memory.
//
// advisor_score_variants needs a caller-provided workspace for the 16-bit
// activation image the tensor-core scorer reads.  Some callers have no way
// to provide one: code running where cudaMalloc is not allowed or not wanted
// (for example inside a host callback, a signal-safe or real-time path, or a
// plugin whose host process forbids extra device allocations after start-up).
// For them this file keeps that image in a fixed, file-scope device array
// (the "scratch"), so the call needs nothing but its inputs and outputs.
//
// The scratch is NOSCRATCH_ROWS rows of up to 128 16-bit features: 4 MiB on
// every GPU that loads the library, held until the process exits.  All calls
// on a device share it; each call overwrites it completely for its rows
// (padding rows of the last tile are written as zeros), so nothing from an
// earlier call is read.  Two calls whose kernels overlap on the GPU (e.g. on
// two streams) race on the scratch; callers must order them.
#include <mutex>

#include "noalloc.cuh"

namespace adv {

constexpr int64_t NOSCRATCH_ROWS = 16384;
constexpr int NOSCRATCH_MAX_SLABS = 2;   // F <= 128: two 64-column slabs per row
constexpr size_t NOSCRATCH_BYTES = (size_t)(NOSCRATCH_ROWS / ADV_TILE_M) * NOSCRATCH_MAX_SLABS * ADV_X_SLAB_BYTES;

static __device__ __align__(256) uint8_t g_noalloc_scratch[NOSCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (the symbol name is only a host-side handle, not a device address)
// and kept for the life of the process: the library must not outlive a reset
// of the device (cudaDeviceReset or a re-created primary context), after
// which the kept address would no longer be valid.
cudaError_t noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}
}  // namespace

}  // namespace adv


extern "C" advisor_status advisor_score_variants_noalloc(advisor_model_t m, const int32_t* d_feat_q16,
                                                         const uint8_t* d_row_status, int64_t n_rows,
                                                         advisor_precision precision, float* d_scores,
                                                         cudaStream_t stream) {
    using namespace adv;
    if (!m || n_rows < 0 || !d_feat_q16 || !d_scores || ((uintptr_t)d_feat_q16 % 16) != 0)
        return ADVISOR_ERR_INVALID_ARGUMENT;
    if (precision != ADVISOR_BF16 && precision != ADVISOR_FP16) return ADVISOR_ERR_UNSUPPORTED;
    if (n_rows > NOSCRATCH_ROWS) return ADVISOR_ERR_OUT_OF_MEMORY;   // beyond the fixed scratch
    if (n_rows == 0) return ADVISOR_OK;
    NoallocModelView v{};
    if (!adv_model_noalloc_view(m, precision == ADVISOR_BF16 ? 0 : 1, &v) || !v.ready)
        return ADVISOR_ERR_INVALID_ARGUMENT;
    if (!v.tc_ok) return ADVISOR_ERR_UNSUPPORTED;
    if (!adv_model_prepare(m, stream)) return ADVISOR_ERR_CUDA;
    if (v.nslab0 > NOSCRATCH_MAX_SLABS) return ADVISOR_ERR_UNSUPPORTED;
    void* scratch = nullptr;
    if (noalloc_scratch(&scratch) != cudaSuccess) return ADVISOR_ERR_CUDA;
    uint8_t* x = static_cast<uint8_t*>(scratch);
    const int64_t npad = ((n_rows + ADV_TILE_M - 1) / ADV_TILE_M) * ADV_TILE_M;
    const int fmt = precision == ADVISOR_BF16 ? 1 : 2;
    cudaError_t e = launch_standardize(d_feat_q16, d_row_status, n_rows, npad, x, v.nslab0, v.sa, v.sc, v.F, fmt, stream);
    if (e != cudaSuccess) return ADVISOR_ERR_CUDA;
    TcArgs a = v.tc;
    a.x_img = x;
    a.n_rows = n_rows;
    a.n_tiles = (int)(npad / ADV_TILE_M);
    a.status = d_row_status;
    a.scores = d_scores;
    a.fmt = precision == ADVISOR_BF16 ? 1 : 0;
    return launch_mlp_tc(a, v.num_sms, stream, v.tc_ctas) == cudaSuccess ? ADVISOR_OK : ADVISOR_ERR_CUDA;
}
