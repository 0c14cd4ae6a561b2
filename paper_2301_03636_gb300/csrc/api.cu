// C ABI of libadvisor (include/advisor.h): argument checks, the layouts of
// the caller-owned parameter block and workspace, and the launch sequences
// of the hot path.  No entry point allocates device memory or synchronises,
// except advisor_get_device_status.
#include <atomic>
#include <cstring>
#include <new>

#include "mlp.cuh"
#include "pack.cuh"
#include "train.cuh"
#include "noalloc.cuh"
#include "selftest.cuh"

namespace {

std::atomic<long long> g_launches{0};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
int roundup(int x, int m) { return ((x + m - 1) / m) * m; }
bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

struct WsLayout {
    size_t x_img, h_img[2], partial, feat32, status, scores, counters, seg_state, seg_start, seg_cnt;
    size_t cand_rows, y32, cand2_rows, y64, pos64, seg_thr, y16, cand_mid_rows;
    size_t train;   // start of the training region
    size_t bytes;
};

}  // namespace

extern "C" void adv_count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

struct advisor_model {
    adv::ModelLayout L;
    uint8_t* P = nullptr;
    size_t p_bytes = 0;
    uint8_t* WS = nullptr;
    size_t ws_bytes = 0;
    int64_t max_rows = 0, max_kernels = 0;
    WsLayout W{};
    adv::TrainLayout T{};
    int num_sms = 0;
    bool params_set = false;
    cudaEvent_t prof_start = nullptr, prof_stop = nullptr;   // bracket the tensor-core scorer launch
    int64_t adam_step = 0;
    int64_t saved_rows = 0;   // rows of the last advisor_forward_saved
    adv::LaunchConfig cfg{};  // launch shapes of the hot path (a plan may set them)
    bool fp8_calibrated = false;   // activation scales stored (advisor_model_calibrate_fp8)
    int saved_fmt = 0;             // precision of the last advisor_forward_saved: 0 FP32, 1 BF16, 2 FP16
    bool last_mid = false;         // the last re-scoring selection ran the FP16 middle tier
    // advisor_rank_staged: the stream that copies the descriptor chunks and the
    // events that hand each chunk to the scoring stream (created on first use)
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t stage_ev[ADVISOR_MAX_STAGES + 1] = {};
    // the master parameters changed (an optimizer step) since the derived
    // inference copies were last built: rebuilt before the next scoring call
    bool images_stale = false;
    ~advisor_model() {
        for (cudaEvent_t e : stage_ev)
            if (e) cudaEventDestroy(e);
        if (copy_stream) cudaStreamDestroy(copy_stream);
    }
};

namespace {

advisor_status cuda_status(cudaError_t e) { return e == cudaSuccess ? ADVISOR_OK : ADVISOR_ERR_CUDA; }

WsLayout ws_layout(const adv::ModelLayout& L, int64_t R, int64_t K, adv::TrainLayout* T) {
    WsLayout w{};
    size_t o = 0;
    const int64_t tiles = (R + ADV_TILE_M - 1) / ADV_TILE_M;
    auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
    w.x_img = take((size_t)tiles * L.nslab[0] * ADV_X_SLAB_BYTES);
    // models too wide for the fused scorer run layer by layer through two
    // activation images and per-chunk partial sums of the output layer
    // (every model may run layer by layer: the path a launch configuration can choose)
    const bool layered = L.n_hidden >= 1;
    for (int i = 0; i < 2; ++i) w.h_img[i] = take(layered ? (size_t)tiles * (L.nmax / 64) * ADV_X_SLAB_BYTES : 0);
    const int last_chunks = (L.npad8[L.n_hidden > 0 ? L.n_hidden - 1 : 0] + 255) / 256;
    w.partial = take(layered ? (size_t)2 * last_chunks * tiles * ADV_TILE_M * 4 : 0);
    w.feat32 = take((size_t)R * L.F * 4);
    w.status = take((size_t)R);
    w.scores = take((size_t)R * 4);
    w.counters = take(16);
    w.seg_state = take((size_t)K * 4);
    w.seg_start = take((size_t)K * 4);
    w.seg_cnt = take((size_t)K * 4);
    w.cand_rows = take((size_t)R * 8);
    w.y32 = take((size_t)R * 4);
    w.cand2_rows = take((size_t)R * 8);
    w.y64 = take((size_t)R * 8);
    w.pos64 = take((size_t)R * 4);
    w.seg_thr = take((size_t)K * 8);
    w.y16 = take((size_t)R * 4);
    w.cand_mid_rows = take((size_t)R * 8);
    w.train = o;
    const size_t tb = adv::train_layout(L, R, T);
    o = align256(o + tb);
    w.bytes = o;
    return w;
}

adv::MlpDesc mlp_desc(const advisor_model* m) {
    const adv::ModelLayout& L = m->L;
    adv::MlpDesc d{};
    d.nw = L.nw;
    for (int i = 0; i < L.nw; ++i) d.widths[i] = L.widths[i];
    const float* master = reinterpret_cast<const float*>(m->P + L.p_master);
    for (int l = 0; l < L.n_layers; ++l) {
        d.W[l] = master + L.layer_w_off[l];
        d.b[l] = master + L.layer_b_off[l];
        d.WT[l] = reinterpret_cast<const float*>(m->P + L.p_wT[l]);
        d.wt_ld[l] = (L.widths[l + 1] + 3) / 4 * 4;
    }
    d.sa = reinterpret_cast<const float*>(m->P + L.p_stdz_a);
    d.sc = reinterpret_cast<const float*>(m->P + L.p_stdz_c);
    d.mu = reinterpret_cast<const double*>(m->P + L.p_mu);
    d.sigma = reinterpret_cast<const double*>(m->P + L.p_sigma);
    return d;
}

int* status_word(advisor_model* m) { return reinterpret_cast<int*>(m->P + m->L.p_status); }

adv::TcArgs tc_args(advisor_model* m, const uint8_t* x_img, int64_t n, const uint8_t* status, float* scores,
                    int fmt_idx /* 0 bf16, 1 fp16 */) {
    const adv::ModelLayout& L = m->L;
    adv::TcArgs a{};
    a.x_img = x_img;
    for (int l = 0; l < L.n_hidden; ++l) {
        a.w_img[l] = m->P + L.p_w16[fmt_idx][l];
        a.bias[l] = reinterpret_cast<const float*>(m->P + L.p_bias_off[l]);
        a.npad[l] = L.npad[l];
        a.nslab[l] = L.nslab[l];
    }
    a.w_out = reinterpret_cast<const float*>(m->P + L.p_wout_pad);
    a.b_out = reinterpret_cast<const float*>(m->P + L.p_master) + L.layer_b_off[L.n_layers - 1];
    a.n_hidden = L.n_hidden;
    a.nmax = L.nmax;
    a.fmt = fmt_idx == 0 ? 1 : 0;   // instruction-descriptor code: 1 = BF16, 0 = F16
    a.n_rows = n;
    a.n_tiles = (int)((n + ADV_TILE_M - 1) / ADV_TILE_M);
    a.status = status;
    a.scores = scores;
    a.status_word = status_word(m);
    a.timeout_ns = 2000000000ull;
    return a;
}

bool tc_supported(const advisor_model* m) {
    const adv::ModelLayout& L = m->L;
    if (!L.tc_ok) return false;
    int nslab_max = 1;
    for (int l = 0; l < L.n_hidden; ++l) nslab_max = L.nslab[l] > nslab_max ? L.nslab[l] : nslab_max;
    return adv::mlp_tc_smem_bytes(nslab_max, L.nmax, L.n_hidden) <= 232448;
}

// Models whose hidden layers exceed the fused scorer: one launch per layer.
bool wide_supported(const advisor_model* m) { return !m->L.tc_ok && m->L.n_hidden >= 1; }
// The fused scorer for this call: the model fits it, the precision is 16-bit
// and the launch configuration does not ask for the layer-by-layer path.
bool use_fused(const advisor_model* m, advisor_precision p) {
    return tc_supported(m) && p != ADVISOR_FP8_E4M3 && !m->cfg.layer_path;
}

cudaError_t launch_wide(advisor_model* m, const uint8_t* x_img, int64_t n_rows, const uint8_t* status, float* scores,
                        int fi, cudaStream_t s, const int* n_rows_dev = nullptr);

// Rebuild the derived inference copies when an optimizer step has changed
// the masters since they were built.  Inside a stream capture the rebuild is
// recorded into the graph and the model stays marked (eager calls still
// rebuild before they score).
cudaError_t ensure_images(advisor_model* m, cudaStream_t s) {
    if (!m->images_stale) return cudaSuccess;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return cudaErrorUnknown;
    const cudaError_t e = adv::launch_repack(m->L, m->P, s);
    if (e == cudaSuccess && cs == cudaStreamCaptureStatusNone) m->images_stale = false;
    return e;
}

advisor_status check_ready(const advisor_model* m, int64_t n_rows) {
    if (!m || !m->P || !m->WS || !m->params_set) return ADVISOR_ERR_INVALID_ARGUMENT;
    if (n_rows > m->max_rows) return ADVISOR_ERR_OUT_OF_MEMORY;
    return ADVISOR_OK;
}

// Inside a stream capture the records become event nodes of the graph, so a
// replayed plan still brackets the scorer.
cudaError_t record_event(cudaEvent_t ev, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal)
                                               : cudaEventRecord(ev, s);
}

cudaError_t launch_tc_profiled(advisor_model* m, const adv::TcArgs& a, cudaStream_t s) {
    if (m->prof_start) {
        cudaError_t e = record_event(m->prof_start, s);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = adv::launch_mlp_tc(a, m->num_sms, s, m->cfg.tc_ctas);
    if (e == cudaSuccess && m->prof_stop) e = record_event(m->prof_stop, s);
    return e;
}

cudaError_t launch_wide(advisor_model* m, const uint8_t* x_img, int64_t n_rows, const uint8_t* status, float* scores,
                        int fi, cudaStream_t s, const int* n_rows_dev) {
    const adv::ModelLayout& L = m->L;
    const int tiles = (int)((n_rows + ADV_TILE_M - 1) / ADV_TILE_M);
    const bool profiled = !n_rows_dev;   // the events bracket the first-tier scorer only
    if (profiled && m->prof_start) {
        cudaError_t e = record_event(m->prof_start, s);
        if (e != cudaSuccess) return e;
    }
    const uint8_t* in = x_img;
    int last_chunks = 1;
    const bool f8 = fi == 2;   // E4M3 images: 128 K per 128-byte row
    for (int l = 0; l < L.n_hidden; ++l) {
        adv::LayerArgs a{};
        a.a_img = in;
        a.a_slabs = f8 ? L.nslab8[l] : L.nslab[l];
        a.w_img = m->P + (f8 ? L.p_w8[l] : L.p_w16[fi][l]);
        a.npad = f8 ? L.npad8[l] : L.npad[l];
        a.n_chunks = (a.npad + 255) / 256;
        a.n_tiles = tiles;
        a.n_rows_dev = n_rows_dev;
        a.bias = reinterpret_cast<const float*>(m->P + L.p_bias_off[l]);
        a.mode = l + 1 == L.n_hidden ? 1 : 0;
        a.out_img = m->WS + m->W.h_img[l & 1];
        a.w_out = reinterpret_cast<const float*>(m->P + L.p_wout_pad);
        a.partial = reinterpret_cast<float*>(m->WS + m->W.partial);
        a.fmt = f8 ? 2 : (fi == 0 ? 1 : 0);   // 2 = E4M3; instruction-descriptor codes 1 = BF16, 0 = F16
        a.fp8 = reinterpret_cast<const float*>(m->P + L.p_fp8);
        a.layer = l;
        a.status_word = status_word(m);
        a.timeout_ns = 2000000000ull;
        cudaError_t e = adv::launch_mlp_layer_tc(a, m->num_sms, s);
        if (e != cudaSuccess) return e;
        in = a.out_img;
        last_chunks = a.n_chunks;
    }
    cudaError_t e = adv::launch_sum_partials(reinterpret_cast<const float*>(m->WS + m->W.partial), 2 * last_chunks,
                                             (int64_t)tiles * ADV_TILE_M, n_rows,
                                             reinterpret_cast<const float*>(m->P + L.p_master) +
                                                 L.layer_b_off[L.n_layers - 1],
                                             status, scores, m->num_sms, s, n_rows_dev);
    if (e == cudaSuccess && profiled && m->prof_stop) e = record_event(m->prof_stop, s);
    return e;
}

// FP16 middle tier of the re-score: the tier-1 candidates (a.cand_rows,
// count counters[0]) are re-extracted from their descriptors into a compact
// FP16 image, scored on the tensor cores (y16, row counts read on the device)
// and filtered by select_mid / topn_mid into a.cand_mid_rows (counters[2]).
cudaError_t run_mid_tier(advisor_model* m, const advisor_variant_desc* desc, int64_t n_rows, adv::SelectArgs& a,
                         bool topn, cudaStream_t s) {
    const adv::ModelLayout& L = m->L;
    adv::ExtractArgs x{};
    x.desc = desc;
    x.n_rows = n_rows;
    x.n_rows_padded = ((n_rows + ADV_TILE_M - 1) / ADV_TILE_M) * ADV_TILE_M;
    x.x_img = m->WS + m->W.x_img;
    x.nslab = L.nslab[0];
    x.sa = reinterpret_cast<const float*>(m->P + L.p_stdz_a);
    x.sc = reinterpret_cast<const float*>(m->P + L.p_stdz_c);
    x.rows = a.cand_rows;
    x.count_dev = &a.counters[0];
    cudaError_t e = adv::launch_extract_list(x, L.F, 2 /* FP16 image */, m->num_sms, s);
    if (e != cudaSuccess) return e;
    float* y16 = reinterpret_cast<float*>(m->WS + m->W.y16);
    if (use_fused(m, ADVISOR_FP16)) {
        adv::TcArgs t = tc_args(m, x.x_img, n_rows, nullptr, y16, 1);
        t.n_rows_dev = &a.counters[0];
        e = adv::launch_mlp_tc(t, m->num_sms, s, m->cfg.tc_ctas);
    } else {
        e = launch_wide(m, x.x_img, n_rows, nullptr, y16, 1, s, &a.counters[0]);
    }
    if (e != cudaSuccess) return e;
    a.y16 = y16;
    a.cand_mid_rows = reinterpret_cast<int64_t*>(m->WS + m->W.cand_mid_rows);
    return topn ? adv::launch_topn_mid(a, s, m->cfg.select_block) : adv::launch_select_mid(a, s, m->cfg.select_block);
}

// The middle tier needs the descriptors (the 16-bit image is rebuilt from
// them) and a model the tensor-core scorers run.
bool mid_supported(const advisor_model* m) { return tc_supported(m) || wide_supported(m); }

// Tiered selection; `src` supplies the rows for the re-score (features or descriptors).
advisor_status do_select(advisor_model* m, const float* scores, int64_t n_rows, const int64_t* off, int64_t K,
                         adv::RowSrc src, bool rescore, float eps, float eps32, int32_t* best, double* best_score,
                         cudaStream_t s, float eps16 = -1.f, bool counters_zeroed = false, bool scores_fp32 = false) {
    if (K > m->max_kernels) return ADVISOR_ERR_OUT_OF_MEMORY;
    adv::SelectArgs a{};
    a.scores = scores;
    a.n_rows = n_rows;
    a.off = off;
    a.n_kernels = K;
    a.best = best;
    a.best_score = best_score;
    a.eps = rescore ? eps : -1.f;
    a.eps32 = eps32;
    a.counters = reinterpret_cast<int*>(m->WS + m->W.counters);
    a.seg_state = reinterpret_cast<int*>(m->WS + m->W.seg_state);
    a.seg_start = reinterpret_cast<int*>(m->WS + m->W.seg_start);
    a.seg_cnt = reinterpret_cast<int*>(m->WS + m->W.seg_cnt);
    a.cand_rows = reinterpret_cast<int64_t*>(m->WS + m->W.cand_rows);
    a.y32 = reinterpret_cast<float*>(m->WS + m->W.y32);
    a.cand2_rows = reinterpret_cast<int64_t*>(m->WS + m->W.cand2_rows);
    a.y64 = reinterpret_cast<double*>(m->WS + m->W.y64);
    a.status_word = status_word(m);
    a.eps16 = eps16;
    const bool mid = rescore && eps16 >= 0.f;
    cudaError_t e;
    if (rescore) {
        if (!counters_zeroed) {
            e = cudaMemsetAsync(a.counters, 0, 4 * sizeof(int), s);
            if (e != cudaSuccess) return ADVISOR_ERR_CUDA;
        }
        m->last_mid = mid;
    }
    e = adv::launch_select_tier1(a, s, m->cfg.select_block);
    if (e != cudaSuccess || !rescore) return cuda_status(e);
    if (mid) {
        e = run_mid_tier(m, src.desc, n_rows, a, false, s);
        if (e != cudaSuccess) return ADVISOR_ERR_CUDA;
        a.cand_rows = a.cand_mid_rows;   // the FP32 tier takes the survivors
    }
    const adv::MlpDesc md = mlp_desc(m);
    if (scores_fp32 && !mid) {
        // the first tier's scores are the plain FP32 path's, whose bound eps32 was
        // calibrated on that path: the FP32 tier reads them instead of re-scoring
        a.y32_rows = scores;
    } else {
        adv::RowSrc r1 = src;
        r1.rows = a.cand_rows;
        r1.count_dev = &a.counters[mid ? 2 : 0];
        r1.count = 0;
        e = adv::launch_mlp_fp32(md, r1, a.y32, m->num_sms, true, s, a.status_word, m->cfg.list_blocks_per_sm,
                                 m->cfg.list_chunk_kb);
        if (e != cudaSuccess) return ADVISOR_ERR_CUDA;
    }
    e = adv::launch_select_tier2(a, s, m->cfg.select_block);
    if (e != cudaSuccess) return ADVISOR_ERR_CUDA;
    adv::RowSrc r2 = src;
    r2.rows = a.cand2_rows;
    r2.count_dev = &a.counters[1];
    r2.count = 0;
    // the FP64 scorer's last block makes the final selection (no launch of its own)
    return cuda_status(adv::launch_mlp_fp64(md, r2, a.y64, m->num_sms, s, &a));
}

}  // namespace

extern "C" {

const char* advisor_status_string(advisor_status s) {
    switch (s) {
        case ADVISOR_OK: return "ok";
        case ADVISOR_ERR_INVALID_ARGUMENT: return "invalid argument";
        case ADVISOR_ERR_BAD_DESCRIPTOR: return "bad descriptor";
        case ADVISOR_ERR_OUT_OF_MEMORY: return "workspace or parameter block too small";
        case ADVISOR_ERR_CUDA: return "CUDA error";
        case ADVISOR_ERR_TIMEOUT: return "device wait timed out";
        case ADVISOR_ERR_UNSUPPORTED: return "unsupported shape or precision";
        case ADVISOR_ERR_BAD_SEGMENTS: return "malformed segment offsets";
    }
    return "unknown status";
}

int64_t advisor_launch_count(void) { return (int64_t)g_launches.load(); }

int64_t advisor_variant_count(int64_t depth) { return adv::variant_count(depth); }

advisor_status advisor_enumerate_variants(const advisor_variant_desc* d_kernels, int64_t n_kernels,
                                          advisor_variant_desc* d_variants, int64_t capacity, int64_t* d_seg_off,
                                          int64_t* d_total, cudaStream_t stream) {
    if (n_kernels < 0 || capacity < 0 || !d_seg_off || (n_kernels > 0 && !d_kernels) ||
        (capacity > 0 && !d_variants))
        return ADVISOR_ERR_INVALID_ARGUMENT;
    if (!aligned(d_kernels, 16) || !aligned(d_variants, 16)) return ADVISOR_ERR_INVALID_ARGUMENT;
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return ADVISOR_ERR_CUDA;
    return cuda_status(adv::launch_enumerate(d_kernels, n_kernels, d_variants, capacity, d_seg_off, d_total, sms,
                                             stream));
}

advisor_status advisor_model_calibrate_fp8(advisor_model_t m, const int32_t* d_feat_q16, int64_t n_rows,
                                           cudaStream_t stream) {
    if (!m || !d_feat_q16 || n_rows < 1) return ADVISOR_ERR_INVALID_ARGUMENT;
    advisor_status st = check_ready(m, n_rows);
    if (st != ADVISOR_OK) return st;
    if (!wide_supported(m)) return ADVISOR_ERR_UNSUPPORTED;
    uint8_t* TW = m->WS + m->W.train;
    cudaError_t e = adv::launch_forward_saved(m->L, m->T, TW, mlp_desc(m), d_feat_q16, n_rows, nullptr, stream);
    if (e != cudaSuccess) return ADVISOR_ERR_CUDA;
    const float* acts[ADV_MAX_LAYERS] = {};
    for (int l = 0; l < m->L.n_hidden; ++l) acts[l] = reinterpret_cast<const float*>(TW + m->T.act[l]);
    e = adv::launch_fp8_calibrate(m->L, m->P, acts, n_rows, stream);
    if (e != cudaSuccess) return ADVISOR_ERR_CUDA;
    m->fp8_calibrated = true;
    return ADVISOR_OK;
}

// Internal hooks for plans (plan.cu): which re-score tiers the last selection ran.
extern "C" int adv_model_last_mid(advisor_model_t m) { return m && m->last_mid ? 1 : 0; }
extern "C" void adv_model_set_last_mid(advisor_model_t m, int mid) {
    if (m) m->last_mid = mid != 0;
}

advisor_status advisor_get_rescore_counts_ex(advisor_model_t m, int64_t* h_counts, cudaStream_t stream) {
    if (!m || !h_counts || !m->WS) return ADVISOR_ERR_INVALID_ARGUMENT;
    int c[4] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(c, m->WS + m->W.counters, sizeof(c), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return ADVISOR_ERR_CUDA;
    h_counts[0] = m->last_mid ? c[0] : 0;   // FP16 tier
    h_counts[1] = m->last_mid ? c[2] : c[0];   // FP32 tier
    h_counts[2] = c[1];                        // FP64 tier
    return ADVISOR_OK;
}

advisor_status advisor_get_rescore_counts(advisor_model_t m, int64_t* h_counts, cudaStream_t stream) {
    if (!h_counts) return ADVISOR_ERR_INVALID_ARGUMENT;
    int64_t c[3];
    const advisor_status st = advisor_get_rescore_counts_ex(m, c, stream);
    if (st != ADVISOR_OK) return st;
    h_counts[0] = c[1];
    h_counts[1] = c[2];
    return ADVISOR_OK;
}

advisor_status advisor_model_get_launch_config(advisor_model_t m, advisor_launch_config* out) {
    if (!m || !out) return ADVISOR_ERR_INVALID_ARGUMENT;
    out->extract_block = m->cfg.extract_block;
    out->tc_ctas = m->cfg.tc_ctas;
    out->list_blocks_per_sm = m->cfg.list_blocks_per_sm;
    out->list_chunk_kb = m->cfg.list_chunk_kb;
    out->select_block = m->cfg.select_block;
    out->layer_path = m->cfg.layer_path;
    return ADVISOR_OK;
}

advisor_status advisor_model_set_launch_config(advisor_model_t m, const advisor_launch_config* c) {
    if (!m || !c) return ADVISOR_ERR_INVALID_ARGUMENT;
    adv::LaunchConfig n;
    n.extract_block = c->extract_block;
    n.tc_ctas = c->tc_ctas;
    n.list_blocks_per_sm = c->list_blocks_per_sm;
    n.list_chunk_kb = c->list_chunk_kb;
    n.select_block = c->select_block;
    n.layer_path = c->layer_path;
    if (!adv::launch_config_valid(n)) return ADVISOR_ERR_INVALID_ARGUMENT;
    m->cfg = n;
    return ADVISOR_OK;
}

advisor_status advisor_model_create(const int32_t* h_widths, int32_t n_widths, advisor_model_t* out) {
    if (!h_widths || !out || n_widths < 3 || n_widths > ADV_MAX_LAYERS) return ADVISOR_ERR_INVALID_ARGUMENT;
    const int F = h_widths[0];
    if (F != 32 && F != 33 && F != 64 && F != 128) return ADVISOR_ERR_INVALID_ARGUMENT;
    if (h_widths[n_widths - 1] != 1) return ADVISOR_ERR_INVALID_ARGUMENT;
    for (int i = 1; i + 1 < n_widths; ++i)
        if (h_widths[i] < 1 || h_widths[i] > 1024) return ADVISOR_ERR_INVALID_ARGUMENT;
    advisor_model* m = new (std::nothrow) advisor_model();
    if (!m) return ADVISOR_ERR_OUT_OF_MEMORY;
    adv::ModelLayout& L = m->L;
    L.nw = n_widths;
    for (int i = 0; i < n_widths; ++i) L.widths[i] = h_widths[i];
    L.F = F;
    L.n_layers = n_widths - 1;
    L.n_hidden = n_widths - 2;
    int64_t po = 0;
    for (int l = 0; l < L.n_layers; ++l) {
        L.layer_w_off[l] = po;
        po += (int64_t)L.widths[l + 1] * L.widths[l];
        L.layer_b_off[l] = po;
        po += L.widths[l + 1];
    }
    L.n_params = po;
    L.tc_ok = 1;
    L.nmax = 0;
    for (int l = 0; l < L.n_hidden; ++l) {
        L.kpad[l] = roundup(L.widths[l], 64);
        L.npad[l] = roundup(L.widths[l + 1], 64);
        L.nslab[l] = L.kpad[l] / 64;
        if (L.widths[l + 1] > 256) L.tc_ok = 0;
        L.nmax = L.npad[l] > L.nmax ? L.npad[l] : L.nmax;
        L.npad8[l] = roundup(L.widths[l + 1], 128);
        L.nslab8[l] = roundup(L.widths[l], 128) / 128;
    }
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
    L.p_master = take((size_t)L.n_params * 4);
    for (int l = 0; l < L.n_layers; ++l) L.p_wT[l] = take((size_t)L.widths[l] * ((L.widths[l + 1] + 3) / 4 * 4) * 4);
    for (int l = 0; l < L.n_hidden; ++l) {
        L.p_w16[0][l] = take((size_t)L.npad[l] * L.kpad[l] * 2);
        L.p_w16[1][l] = take((size_t)L.npad[l] * L.kpad[l] * 2);
        // E4M3 copies only for models that run layer by layer
        L.p_w8[l] = take(L.tc_ok ? 0 : (size_t)L.npad8[l] * L.nslab8[l] * ADV_SLAB_ROW_BYTES);
        L.p_bias_off[l] = take((size_t)L.npad8[l] * 4);
    }
    L.p_fp8 = take(32 * 4);
    L.p_wout_pad = take((size_t)L.npad8[L.n_hidden - 1] * 4);
    L.p_stdz_a = take((size_t)F * 4);
    L.p_stdz_c = take((size_t)F * 4);
    L.p_mu = take((size_t)F * 8);
    L.p_sigma = take((size_t)F * 8);
    L.p_adam_m = take((size_t)L.n_params * 4);
    L.p_adam_v = take((size_t)L.n_params * 4);
    L.p_status = take(16);
    L.p_misc = take(256);
    L.param_bytes = o;
    *out = m;
    return ADVISOR_OK;
}

advisor_status advisor_model_destroy(advisor_model_t m) {
    delete m;
    return ADVISOR_OK;
}

size_t advisor_model_param_bytes(advisor_model_t m) { return m ? m->L.param_bytes : 0; }

int64_t advisor_model_param_count(advisor_model_t m) { return m ? m->L.n_params : 0; }

size_t advisor_workspace_bytes(advisor_model_t m, int64_t max_rows, int64_t max_kernels) {
    if (!m || max_rows < 0 || max_kernels < 0) return 0;
    adv::TrainLayout t{};
    return ws_layout(m->L, max_rows < 1 ? 1 : max_rows, max_kernels < 1 ? 1 : max_kernels, &t).bytes;
}

advisor_status advisor_model_bind(advisor_model_t m, void* d_params, size_t param_bytes, void* d_workspace,
                                  size_t workspace_bytes, int64_t max_rows, int64_t max_kernels) {
    if (!m || !d_params || !d_workspace || max_rows < 1 || max_kernels < 1) return ADVISOR_ERR_INVALID_ARGUMENT;
    if (!aligned(d_params, 256) || !aligned(d_workspace, 256)) return ADVISOR_ERR_INVALID_ARGUMENT;
    if (param_bytes < m->L.param_bytes) return ADVISOR_ERR_OUT_OF_MEMORY;
    adv::TrainLayout t{};
    const WsLayout w = ws_layout(m->L, max_rows, max_kernels, &t);
    if (workspace_bytes < w.bytes) return ADVISOR_ERR_OUT_OF_MEMORY;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ADVISOR_ERR_CUDA;
    if (cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return ADVISOR_ERR_CUDA;
    if (m->P != (uint8_t*)d_params) m->params_set = false;
    m->P = (uint8_t*)d_params;
    m->p_bytes = param_bytes;
    m->WS = (uint8_t*)d_workspace;
    m->ws_bytes = workspace_bytes;
    m->max_rows = max_rows;
    m->max_kernels = max_kernels;
    m->W = w;
    m->T = t;
    return ADVISOR_OK;
}

advisor_status advisor_model_set_params(advisor_model_t m, const float* d_params_fp32, const double* d_mu,
                                        const double* d_sigma, cudaStream_t stream) {
    if (!m || !m->P || !d_params_fp32 || !d_mu || !d_sigma) return ADVISOR_ERR_INVALID_ARGUMENT;
    cudaError_t e = cudaMemsetAsync(m->P + m->L.p_status, 0, 16, stream);
    if (e != cudaSuccess) return ADVISOR_ERR_CUDA;
    e = adv::launch_set_params(m->L, m->P, d_params_fp32, d_mu, d_sigma, stream);
    if (e != cudaSuccess) return ADVISOR_ERR_CUDA;
    m->params_set = true;
    m->images_stale = false;   // set_params builds the derived copies
    m->adam_step = 0;
    m->fp8_calibrated = false;
    return ADVISOR_OK;
}

advisor_status advisor_model_get_params(advisor_model_t m, float* d_params_fp32, cudaStream_t stream) {
    if (!m || !m->P || !d_params_fp32) return ADVISOR_ERR_INVALID_ARGUMENT;
    return cuda_status(adv::launch_copy_f32(reinterpret_cast<const float*>(m->P + m->L.p_master), d_params_fp32,
                                            m->L.n_params, stream));
}

advisor_status advisor_fit_standardizer(const int32_t* d_feat_q16, const uint8_t* d_row_status, int64_t n_rows,
                                        int32_t n_features, double* d_mu, double* d_sigma, cudaStream_t stream) {
    if (!d_feat_q16 || !d_mu || !d_sigma || n_rows < 1 || n_features < 1 || n_features > 1024)
        return ADVISOR_ERR_INVALID_ARGUMENT;
    return cuda_status(adv::launch_fit_standardizer(d_feat_q16, d_row_status, n_rows, n_features, d_mu, d_sigma,
                                                    stream));
}

advisor_status advisor_extract_features(const advisor_variant_desc* d_desc, int64_t n_rows, int32_t n_features,
                                        int32_t* d_feat_q16, uint8_t* d_row_status, cudaStream_t stream) {
    if (n_rows < 0 || (n_features != 32 && n_features != 33 && n_features != 64 && n_features != 128))
        return ADVISOR_ERR_INVALID_ARGUMENT;
    if (n_rows == 0) return ADVISOR_OK;
    if (!d_desc || !d_feat_q16 || !aligned(d_desc, 16) || !aligned(d_feat_q16, 16))
        return ADVISOR_ERR_INVALID_ARGUMENT;
    adv::ExtractArgs a{};
    a.desc = d_desc;
    a.n_rows = n_rows;
    a.n_rows_padded = n_rows;
    a.feat = d_feat_q16;
    a.status = d_row_status;
    return cuda_status(adv::launch_extract(a, n_features, 0, stream));
}

advisor_status advisor_score_variants(advisor_model_t m, const int32_t* d_feat_q16, const uint8_t* d_row_status,
                                      int64_t n_rows, advisor_precision precision, float* d_scores,
                                      cudaStream_t stream) {
    if (!m || n_rows < 0 || !d_feat_q16 || !d_scores || !aligned(d_feat_q16, 16))
        return ADVISOR_ERR_INVALID_ARGUMENT;
    if (n_rows == 0) return ADVISOR_OK;
    advisor_status st = check_ready(m, n_rows);
    if (st != ADVISOR_OK) return st;
    if (ensure_images(m, stream) != cudaSuccess) return ADVISOR_ERR_CUDA;
    if (precision == ADVISOR_FP32) {
        adv::RowSrc src{d_feat_q16, nullptr, nullptr, nullptr, n_rows, d_row_status};
        return cuda_status(adv::launch_mlp_fp32(mlp_desc(m), src, d_scores, m->num_sms, false, stream));
    }
    if (precision == ADVISOR_FP8_E4M3) {
        if (!wide_supported(m)) return ADVISOR_ERR_UNSUPPORTED;
        if (!m->fp8_calibrated) return ADVISOR_ERR_INVALID_ARGUMENT;
    } else if (precision != ADVISOR_BF16 && precision != ADVISOR_FP16) {
        return ADVISOR_ERR_UNSUPPORTED;
    }
    const bool fused = use_fused(m, precision);
    if (!fused && m->L.n_hidden < 1) return ADVISOR_ERR_UNSUPPORTED;
    const int fi = precision == ADVISOR_BF16 ? 0 : (precision == ADVISOR_FP16 ? 1 : 2);
    const int64_t npad = ((n_rows + ADV_TILE_M - 1) / ADV_TILE_M) * ADV_TILE_M;
    uint8_t* x = m->WS + m->W.x_img;
    cudaError_t e = adv::launch_standardize(d_feat_q16, d_row_status, n_rows, npad, x,
                                            fi == 2 ? m->L.nslab8[0] : m->L.nslab[0],
                                            reinterpret_cast<const float*>(m->P + m->L.p_stdz_a),
                                            reinterpret_cast<const float*>(m->P + m->L.p_stdz_c), m->L.F,
                                            fi + 1, stream,
                                            reinterpret_cast<const float*>(m->P + m->L.p_fp8) + ADV_FP8_X_SCALE);
    if (e != cudaSuccess) return ADVISOR_ERR_CUDA;
    if (!fused) return cuda_status(launch_wide(m, x, n_rows, d_row_status, d_scores, fi, stream));
    return cuda_status(launch_tc_profiled(m, tc_args(m, x, n_rows, d_row_status, d_scores, fi), stream));
}

advisor_status advisor_score_variants_fp64(advisor_model_t m, const int32_t* d_feat_q16,
                                           const uint8_t* d_row_status, int64_t n_rows, double* d_scores,
                                           cudaStream_t stream) {
    if (!m || n_rows < 0 || !d_feat_q16 || !d_scores) return ADVISOR_ERR_INVALID_ARGUMENT;
    if (n_rows == 0) return ADVISOR_OK;
    if (!m->P || !m->params_set) return ADVISOR_ERR_INVALID_ARGUMENT;
    if (ensure_images(m, stream) != cudaSuccess) return ADVISOR_ERR_CUDA;
    adv::RowSrc src{d_feat_q16, nullptr, nullptr, nullptr, n_rows, d_row_status};
    return cuda_status(adv::launch_mlp_fp64(mlp_desc(m), src, d_scores, m->num_sms, stream));
}

advisor_status advisor_select_best(advisor_model_t m, const float* d_scores, int64_t n_rows,
                                   const int64_t* d_seg_off, int64_t n_kernels, const int32_t* d_feat_q16,
                                   float eps_scores, float eps_fp32, int32_t* d_best_local, double* d_best_score,
                                   cudaStream_t stream) {
    if (!m || n_rows < 0 || n_kernels < 0 || !d_best_local || !d_best_score) return ADVISOR_ERR_INVALID_ARGUMENT;
    if (n_kernels == 0) return ADVISOR_OK;
    if (!d_seg_off || (n_rows > 0 && !d_scores)) return ADVISOR_ERR_INVALID_ARGUMENT;
    const bool rescore = d_feat_q16 != nullptr && eps_scores >= 0.f;
    if (rescore && (eps_fp32 < 0.f || !aligned(d_feat_q16, 16))) return ADVISOR_ERR_INVALID_ARGUMENT;
    advisor_status st = check_ready(m, n_rows);
    if (st != ADVISOR_OK) return st;
    if (rescore && ensure_images(m, stream) != cudaSuccess) return ADVISOR_ERR_CUDA;
    adv::RowSrc src{d_feat_q16, nullptr, nullptr, nullptr, 0, nullptr};
    return do_select(m, d_scores, n_rows, d_seg_off, n_kernels, src, rescore, eps_scores, eps_fp32, d_best_local,
                     d_best_score, stream);
}

}  // extern "C"

namespace {

// a1-a5 of the ranking calls: descriptors -> scores and row status; *rs
// receives where the re-score tiers read the rows from (the FP32 path keeps
// the int32 features, the tensor-core paths re-extract from the descriptors).
//
// row0 (a multiple of the 128-row tile) scores rows row0 .. row0 + n_rows - 1
// of the arrays that d_desc, scores and status point to, into the matching
// part of the workspace; *rs still refers to the whole arrays.
advisor_status rank_scores(advisor_model* m, const advisor_variant_desc* d_desc, int64_t n_rows,
                           advisor_precision precision, float* scores, uint8_t* status, adv::RowSrc* rs,
                           cudaStream_t stream, int64_t row0 = 0) {
    *rs = adv::RowSrc{nullptr, d_desc, nullptr, nullptr, 0, nullptr};
    const adv::ModelLayout& L = m->L;
    if (precision == ADVISOR_FP32) *rs = adv::RowSrc{reinterpret_cast<int32_t*>(m->WS + m->W.feat32), nullptr,
                                                     nullptr, nullptr, 0, nullptr};
    if (n_rows == 0) return ADVISOR_OK;
    d_desc += row0;
    scores += row0;
    status += row0;
    adv::ExtractArgs a{};
    a.desc = d_desc;
    a.n_rows = n_rows;
    a.status = status;
    a.sa = reinterpret_cast<const float*>(m->P + L.p_stdz_a);
    a.sc = reinterpret_cast<const float*>(m->P + L.p_stdz_c);
    cudaError_t e;
    if (precision == ADVISOR_FP32) {
        a.n_rows_padded = n_rows;
        a.feat = reinterpret_cast<int32_t*>(m->WS + m->W.feat32) + row0 * L.F;
        e = adv::launch_extract(a, L.F, 0, stream, m->cfg.extract_block);
        if (e != cudaSuccess) return ADVISOR_ERR_CUDA;
        adv::RowSrc src{a.feat, nullptr, nullptr, nullptr, n_rows, status};
        e = adv::launch_mlp_fp32(mlp_desc(m), src, scores, m->num_sms, false, stream);
        return e == cudaSuccess ? ADVISOR_OK : ADVISOR_ERR_CUDA;
    }
    if (precision == ADVISOR_FP8_E4M3) {
        if (!wide_supported(m)) return ADVISOR_ERR_UNSUPPORTED;
        if (!m->fp8_calibrated) return ADVISOR_ERR_INVALID_ARGUMENT;
    } else if (precision != ADVISOR_BF16 && precision != ADVISOR_FP16) {
        return ADVISOR_ERR_UNSUPPORTED;
    }
    const bool fused = use_fused(m, precision);
    if (!fused && m->L.n_hidden < 1) return ADVISOR_ERR_UNSUPPORTED;
    const int fi = precision == ADVISOR_BF16 ? 0 : (precision == ADVISOR_FP16 ? 1 : 2);
    a.n_rows_padded = ((n_rows + ADV_TILE_M - 1) / ADV_TILE_M) * ADV_TILE_M;
    a.nslab = fi == 2 ? L.nslab8[0] : L.nslab[0];
    a.x_img = m->WS + m->W.x_img + (size_t)(row0 / ADV_TILE_M) * a.nslab * ADV_X_SLAB_BYTES;
    a.x8_scale = reinterpret_cast<const float*>(m->P + L.p_fp8) + ADV_FP8_X_SCALE;
    e = adv::launch_extract(a, L.F, fi + 1, stream, m->cfg.extract_block);
    if (e != cudaSuccess) return ADVISOR_ERR_CUDA;
    e = fused ? launch_tc_profiled(m, tc_args(m, a.x_img, n_rows, status, scores, fi), stream)
              : launch_wide(m, a.x_img, n_rows, status, scores, fi, stream);
    return e == cudaSuccess ? ADVISOR_OK : ADVISOR_ERR_CUDA;
}

// Top-N selection with the tiered re-score (select.cu, topn_*).
advisor_status do_select_topn(advisor_model* m, const float* scores, int64_t n_rows, const int64_t* off, int64_t K,
                              int N, adv::RowSrc src, bool rescore, float eps, float eps32, int32_t* best,
                              double* best_score, cudaStream_t s, float eps16 = -1.f,
                              bool counters_zeroed = false) {
    adv::SelectArgs a{};
    a.scores = scores;
    a.n_rows = n_rows;
    a.off = off;
    a.n_kernels = K;
    a.best = best;
    a.best_score = best_score;
    a.eps = rescore ? eps : -1.f;
    a.eps32 = eps32;
    a.counters = reinterpret_cast<int*>(m->WS + m->W.counters);
    a.seg_state = reinterpret_cast<int*>(m->WS + m->W.seg_state);
    a.seg_start = reinterpret_cast<int*>(m->WS + m->W.seg_start);
    a.seg_cnt = reinterpret_cast<int*>(m->WS + m->W.seg_cnt);
    a.cand_rows = reinterpret_cast<int64_t*>(m->WS + m->W.cand_rows);
    a.y32 = reinterpret_cast<float*>(m->WS + m->W.y32);
    a.cand2_rows = reinterpret_cast<int64_t*>(m->WS + m->W.cand2_rows);
    a.y64 = reinterpret_cast<double*>(m->WS + m->W.y64);
    a.status_word = status_word(m);
    a.top_n = N;
    a.pos64 = reinterpret_cast<int*>(m->WS + m->W.pos64);
    a.seg_thr = reinterpret_cast<double*>(m->WS + m->W.seg_thr);
    a.eps16 = eps16;
    const bool mid = rescore && eps16 >= 0.f;
    cudaError_t e;
    if (rescore) {
        if (!counters_zeroed) {
            e = cudaMemsetAsync(a.counters, 0, 4 * sizeof(int), s);
            if (e != cudaSuccess) return ADVISOR_ERR_CUDA;
        }
        m->last_mid = mid;
    }
    e = adv::launch_topn_tier1(a, s, m->cfg.select_block);
    if (e != cudaSuccess || !rescore) return cuda_status(e);
    if (mid) {
        e = run_mid_tier(m, src.desc, n_rows, a, true, s);
        if (e != cudaSuccess) return ADVISOR_ERR_CUDA;
        a.cand_rows = a.cand_mid_rows;   // the FP32 tier takes the survivors
    }
    const adv::MlpDesc md = mlp_desc(m);
    adv::RowSrc r1 = src;
    r1.rows = a.cand_rows;
    r1.count_dev = &a.counters[mid ? 2 : 0];
    r1.count = 0;
    e = adv::launch_mlp_fp32(md, r1, a.y32, m->num_sms, true, s, a.status_word, m->cfg.list_blocks_per_sm,
                             m->cfg.list_chunk_kb);
    if (e != cudaSuccess) return ADVISOR_ERR_CUDA;
    e = adv::launch_topn_tier2(a, s, m->cfg.select_block);
    if (e != cudaSuccess) return ADVISOR_ERR_CUDA;
    adv::RowSrc r2 = src;
    r2.rows = a.cand2_rows;
    r2.count_dev = &a.counters[1];
    r2.count = 0;
    e = adv::launch_mlp_fp64(md, r2, a.y64, m->num_sms, s);
    if (e != cudaSuccess) return ADVISOR_ERR_CUDA;
    return cuda_status(adv::launch_topn_final(a, s, m->cfg.select_block));
}

// Whether the device can read `p` directly: device or managed memory, or
// page-locked host memory mapped into the unified address space.
bool device_readable(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();   // clear the error state this query leaves behind
        return false;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeHost && at.devicePointer == p;
}

// Shared checks of the ranking calls.
advisor_status rank_checks(advisor_model_t m, const advisor_variant_desc* d_desc, int64_t n_rows,
                           const int64_t* d_seg_off, int64_t n_kernels, advisor_precision precision,
                           float eps_scores, float eps_fp16, float eps_fp32, const int32_t* d_best_local,
                           const double* d_best_score) {
    if (!m || n_rows < 0 || n_kernels < 0 || !d_best_local || !d_best_score) return ADVISOR_ERR_INVALID_ARGUMENT;
    if (n_kernels == 0) return ADVISOR_OK;
    if (!d_seg_off || (n_rows > 0 && (!d_desc || !aligned(d_desc, 16) || !device_readable(d_desc))))
        return ADVISOR_ERR_INVALID_ARGUMENT;
    // offsets and answers: device memory or mapped page-locked host memory
    if (!device_readable(d_seg_off) || !device_readable(d_best_local) || !device_readable(d_best_score))
        return ADVISOR_ERR_INVALID_ARGUMENT;
    advisor_status st = check_ready(m, n_rows);
    if (st != ADVISOR_OK) return st;
    if (n_kernels > m->max_kernels) return ADVISOR_ERR_OUT_OF_MEMORY;
    const bool rescore = eps_scores >= 0.f;
    if (rescore && eps_fp32 < 0.f) return ADVISOR_ERR_INVALID_ARGUMENT;
    if (eps_fp16 >= 0.f) {
        if (!rescore) return ADVISOR_ERR_INVALID_ARGUMENT;
        if (precision == ADVISOR_FP32 || !mid_supported(m)) return ADVISOR_ERR_UNSUPPORTED;
    }
    return ADVISOR_OK;
}

}  // namespace

extern "C" {

advisor_status advisor_rank_ex(advisor_model_t m, const advisor_variant_desc* d_desc, int64_t n_rows,
                               const int64_t* d_seg_off, int64_t n_kernels, advisor_precision precision,
                               float eps_scores, float eps_fp16, float eps_fp32, int32_t* d_best_local,
                               double* d_best_score, float* d_scores, uint8_t* d_row_status, cudaStream_t stream) {
    advisor_status st = rank_checks(m, d_desc, n_rows, d_seg_off, n_kernels, precision, eps_scores, eps_fp16,
                                    eps_fp32, d_best_local, d_best_score);
    if (st != ADVISOR_OK || n_kernels == 0) return st;
    if (ensure_images(m, stream) != cudaSuccess) return ADVISOR_ERR_CUDA;
    const bool rescore = eps_scores >= 0.f;
    float* scores = d_scores ? d_scores : reinterpret_cast<float*>(m->WS + m->W.scores);
    uint8_t* status = d_row_status ? d_row_status : m->WS + m->W.status;
    const bool zeroed = rescore && n_rows > 0;   // zeroed ahead, so that the kernels of the chain follow one another
    if (zeroed && cudaMemsetAsync(m->WS + m->W.counters, 0, 4 * sizeof(int), stream) != cudaSuccess)
        return ADVISOR_ERR_CUDA;
    adv::RowSrc rs{};
    st = rank_scores(m, d_desc, n_rows, precision, scores, status, &rs, stream);
    if (st != ADVISOR_OK) return st;
    return do_select(m, scores, n_rows, d_seg_off, n_kernels, rs, rescore && n_rows > 0, eps_scores, eps_fp32,
                     d_best_local, d_best_score, stream, eps_fp16 >= 0.f ? eps_fp16 : -1.f, zeroed,
                     precision == ADVISOR_FP32);
}

advisor_status advisor_rank_staged_ex(advisor_model_t m, const advisor_variant_desc* h_desc,
                                      advisor_variant_desc* d_desc, int64_t n_rows, const int64_t* d_seg_off,
                                      int64_t n_kernels, advisor_precision precision, float eps_scores,
                                      float eps_fp16, float eps_fp32, int32_t* d_best_local, double* d_best_score,
                                      float* d_scores, uint8_t* d_row_status, int32_t n_stages,
                                      cudaStream_t stream) {
    if (n_stages < 1 || n_stages > ADVISOR_MAX_STAGES) return ADVISOR_ERR_INVALID_ARGUMENT;
    advisor_status st = rank_checks(m, d_desc, n_rows, d_seg_off, n_kernels, precision, eps_scores, eps_fp16,
                                    eps_fp32, d_best_local, d_best_score);
    if (st != ADVISOR_OK || n_kernels == 0) return st;
    if (ensure_images(m, stream) != cudaSuccess) return ADVISOR_ERR_CUDA;
    if (n_rows > 0) {
        cudaPointerAttributes at{};
        if (!h_desc || cudaPointerGetAttributes(&at, h_desc) != cudaSuccess || at.type != cudaMemoryTypeHost) {
            cudaGetLastError();
            return ADVISOR_ERR_INVALID_ARGUMENT;   // the copies need page-locked host memory
        }
    }
    if (!m->copy_stream) {
        if (cudaStreamCreateWithFlags(&m->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
            m->copy_stream = nullptr;
            return ADVISOR_ERR_CUDA;
        }
        for (cudaEvent_t& e : m->stage_ev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return ADVISOR_ERR_CUDA;
    }
    const bool rescore = eps_scores >= 0.f;
    float* scores = d_scores ? d_scores : reinterpret_cast<float*>(m->WS + m->W.scores);
    uint8_t* status = d_row_status ? d_row_status : m->WS + m->W.status;
    const bool zeroed = rescore && n_rows > 0;
    if (zeroed && cudaMemsetAsync(m->WS + m->W.counters, 0, 4 * sizeof(int), stream) != cudaSuccess)
        return ADVISOR_ERR_CUDA;
    // chunks of whole 128-row tiles: the copy of chunk c + 1 overlaps the scoring of chunk c
    const int64_t tiles = (n_rows + ADV_TILE_M - 1) / ADV_TILE_M;
    const int64_t chunk = ((tiles + n_stages - 1) / n_stages) * ADV_TILE_M;
    if (cudaEventRecord(m->stage_ev[0], stream) != cudaSuccess ||
        cudaStreamWaitEvent(m->copy_stream, m->stage_ev[0], 0) != cudaSuccess)
        return ADVISOR_ERR_CUDA;
    adv::RowSrc rs{};
    int c = 0;
    for (int64_t r0 = 0; r0 < n_rows; r0 += chunk, ++c) {
        const int64_t rows = n_rows - r0 < chunk ? n_rows - r0 : chunk;
        if (cudaMemcpyAsync(d_desc + r0, h_desc + r0, (size_t)rows * sizeof(advisor_variant_desc),
                            cudaMemcpyHostToDevice, m->copy_stream) != cudaSuccess ||
            cudaEventRecord(m->stage_ev[c + 1], m->copy_stream) != cudaSuccess ||
            cudaStreamWaitEvent(stream, m->stage_ev[c + 1], 0) != cudaSuccess)
            return ADVISOR_ERR_CUDA;
        st = rank_scores(m, d_desc, rows, precision, scores, status, &rs, stream, r0);
        if (st != ADVISOR_OK) return st;
    }
    if (n_rows == 0) rank_scores(m, d_desc, 0, precision, scores, status, &rs, stream);
    else if (c == 0) return ADVISOR_ERR_CUDA;
    return do_select(m, scores, n_rows, d_seg_off, n_kernels, rs, rescore && n_rows > 0, eps_scores, eps_fp32,
                     d_best_local, d_best_score, stream, eps_fp16 >= 0.f ? eps_fp16 : -1.f, zeroed,
                     precision == ADVISOR_FP32);
}

advisor_status advisor_rank_staged(advisor_model_t m, const advisor_variant_desc* h_desc,
                                   advisor_variant_desc* d_desc, int64_t n_rows, const int64_t* d_seg_off,
                                   int64_t n_kernels, advisor_precision precision, float eps_scores,
                                   float eps_fp32, int32_t* d_best_local, double* d_best_score, float* d_scores,
                                   uint8_t* d_row_status, int32_t n_stages, cudaStream_t stream) {
    return advisor_rank_staged_ex(m, h_desc, d_desc, n_rows, d_seg_off, n_kernels, precision, eps_scores, -1.f,
                                  eps_fp32, d_best_local, d_best_score, d_scores, d_row_status, n_stages, stream);
}

advisor_status advisor_rank(advisor_model_t m, const advisor_variant_desc* d_desc, int64_t n_rows,
                            const int64_t* d_seg_off, int64_t n_kernels, advisor_precision precision,
                            float eps_scores, float eps_fp32, int32_t* d_best_local, double* d_best_score,
                            float* d_scores, uint8_t* d_row_status, cudaStream_t stream) {
    return advisor_rank_ex(m, d_desc, n_rows, d_seg_off, n_kernels, precision, eps_scores, -1.f, eps_fp32,
                           d_best_local, d_best_score, d_scores, d_row_status, stream);
}

advisor_status advisor_rank_topn_ex(advisor_model_t m, const advisor_variant_desc* d_desc, int64_t n_rows,
                                    const int64_t* d_seg_off, int64_t n_kernels, int32_t top_n,
                                    advisor_precision precision, float eps_scores, float eps_fp16, float eps_fp32,
                                    int32_t* d_best_local, double* d_best_score, float* d_scores,
                                    uint8_t* d_row_status, cudaStream_t stream) {
    if (top_n < 1 || top_n > ADVISOR_MAX_TOP_N) return ADVISOR_ERR_INVALID_ARGUMENT;
    advisor_status st = rank_checks(m, d_desc, n_rows, d_seg_off, n_kernels, precision, eps_scores, eps_fp16,
                                    eps_fp32, d_best_local, d_best_score);
    if (st != ADVISOR_OK || n_kernels == 0) return st;
    if (ensure_images(m, stream) != cudaSuccess) return ADVISOR_ERR_CUDA;
    const bool rescore = eps_scores >= 0.f;
    float* scores = d_scores ? d_scores : reinterpret_cast<float*>(m->WS + m->W.scores);
    uint8_t* status = d_row_status ? d_row_status : m->WS + m->W.status;
    const bool zeroed = rescore && n_rows > 0;
    if (zeroed && cudaMemsetAsync(m->WS + m->W.counters, 0, 4 * sizeof(int), stream) != cudaSuccess)
        return ADVISOR_ERR_CUDA;
    adv::RowSrc rs{};
    st = rank_scores(m, d_desc, n_rows, precision, scores, status, &rs, stream);
    if (st != ADVISOR_OK) return st;
    return do_select_topn(m, scores, n_rows, d_seg_off, n_kernels, top_n, rs, rescore && n_rows > 0, eps_scores,
                          eps_fp32, d_best_local, d_best_score, stream, eps_fp16 >= 0.f ? eps_fp16 : -1.f, zeroed);
}

advisor_status advisor_rank_topn(advisor_model_t m, const advisor_variant_desc* d_desc, int64_t n_rows,
                                 const int64_t* d_seg_off, int64_t n_kernels, int32_t top_n,
                                 advisor_precision precision, float eps_scores, float eps_fp32,
                                 int32_t* d_best_local, double* d_best_score, float* d_scores,
                                 uint8_t* d_row_status, cudaStream_t stream) {
    return advisor_rank_topn_ex(m, d_desc, n_rows, d_seg_off, n_kernels, top_n, precision, eps_scores, -1.f,
                                eps_fp32, d_best_local, d_best_score, d_scores, d_row_status, stream);
}

// Training precision: 0 FP32 SIMT, 1 BF16 / 2 FP16 tensor-core GEMMs; -1 unsupported.
int train_fmt(advisor_model* m, advisor_precision p) {
    if (p == ADVISOR_FP32) return 0;
    if (p != ADVISOR_BF16 && p != ADVISOR_FP16) return -1;
    return p == ADVISOR_BF16 ? 1 : 2;
}

// The fused 16-bit training forward, for models the fused scorer covers (else nullptr).
const adv::FusedFwd* fused_fwd(advisor_model* m, int fmt, adv::FusedFwd* ff) {
    if (fmt == 0 || !tc_supported(m)) return nullptr;
    const adv::ModelLayout& L = m->L;
    ff->tc = tc_args(m, nullptr, 0, nullptr, nullptr, fmt == 1 ? 0 : 1);
    ff->x_img = m->WS + m->W.x_img;
    ff->num_sms = m->num_sms;
    ff->ctas = m->cfg.tc_ctas;
    for (int l = 0; l < L.n_hidden; ++l) {
        ff->img16[0][l] = m->P + L.p_w16[0][l];
        ff->img16[1][l] = m->P + L.p_w16[1][l];
        ff->bias_pad[l] = reinterpret_cast<float*>(m->P + L.p_bias_off[l]);
    }
    ff->wout_pad = reinterpret_cast<float*>(m->P + L.p_wout_pad);
    return ff;
}

advisor_status advisor_train_step(advisor_model_t m, const int32_t* d_feat_q16, const float* d_labels,
                                  int64_t n_rows, advisor_precision precision, const float* h_adam, float* d_loss,
                                  cudaStream_t stream) {
    if (!m || !d_feat_q16 || !d_labels || !h_adam || n_rows < 1) return ADVISOR_ERR_INVALID_ARGUMENT;
    advisor_status st = check_ready(m, n_rows);
    if (st != ADVISOR_OK) return st;
    const int fmt = train_fmt(m, precision);
    if (fmt < 0) return ADVISOR_ERR_UNSUPPORTED;
    const adv::AdamHyper h{h_adam[0], h_adam[1], h_adam[2], h_adam[3], h_adam[4]};
    const int64_t step = m->adam_step + 1;
    adv::FusedFwd ff{};
    cudaError_t e = fmt == 0 ? adv::launch_train_step(m->L, m->T, m->P, m->WS + m->W.train, mlp_desc(m), d_feat_q16,
                                                      d_labels, n_rows, &h, step, nullptr, d_loss, m->num_sms, stream)
                             : adv::launch_train_step_tc(m->L, m->T, m->P, m->WS + m->W.train, mlp_desc(m), fmt,
                                                         d_feat_q16, d_labels, n_rows, &h, step, nullptr, d_loss,
                                                         stream, status_word(m), fused_fwd(m, fmt, &ff));
    if (e != cudaSuccess) return ADVISOR_ERR_CUDA;
    m->adam_step = step;
    m->images_stale = true;
    return ADVISOR_OK;
}

advisor_status advisor_train_step_ex(advisor_model_t m, const int32_t* d_feat_q16, const float* d_labels,
                                     int64_t n_rows, advisor_precision precision, const advisor_train_options* opt,
                                     float* d_loss, cudaStream_t stream) {
    if (!m || !d_feat_q16 || !d_labels || !opt || n_rows < 1) return ADVISOR_ERR_INVALID_ARGUMENT;
    if ((opt->optimizer != ADVISOR_OPT_ADAM && opt->optimizer != ADVISOR_OPT_RMSPROP) ||
        (opt->loss != ADVISOR_LOSS_MSE && opt->loss != ADVISOR_LOSS_RMSE))
        return ADVISOR_ERR_INVALID_ARGUMENT;
    advisor_status st = check_ready(m, n_rows);
    if (st != ADVISOR_OK) return st;
    const int fmt = train_fmt(m, precision);
    if (fmt < 0) return ADVISOR_ERR_UNSUPPORTED;
    adv::TrainOptions o{};
    o.optimizer = opt->optimizer;
    o.loss = opt->loss;
    o.h = adv::AdamHyper{opt->lr, opt->beta1, opt->beta2, opt->eps, opt->weight_decay};
    o.alpha = opt->alpha;
    const int64_t step = m->adam_step + 1;
    adv::FusedFwd ff{};
    cudaError_t e = adv::launch_train_step_ex(m->L, m->T, m->P, m->WS + m->W.train, mlp_desc(m), fmt, d_feat_q16,
                                              d_labels, n_rows, o, step, d_loss, stream, status_word(m),
                                              fused_fwd(m, fmt, &ff));
    if (e != cudaSuccess) return ADVISOR_ERR_CUDA;
    m->adam_step = step;
    m->images_stale = true;
    return ADVISOR_OK;
}

advisor_status advisor_loss_grad(advisor_model_t m, const int32_t* d_feat_q16, const float* d_labels,
                                 int64_t n_rows, advisor_precision precision, float* d_grad, float* d_loss,
                                 cudaStream_t stream) {
    if (!m || !d_feat_q16 || !d_labels || !d_grad || n_rows < 1) return ADVISOR_ERR_INVALID_ARGUMENT;
    advisor_status st = check_ready(m, n_rows);
    if (st != ADVISOR_OK) return st;
    const int fmt = train_fmt(m, precision);
    if (fmt < 0) return ADVISOR_ERR_UNSUPPORTED;
    adv::FusedFwd ff{};
    if (fmt != 0)
        return cuda_status(adv::launch_train_step_tc(m->L, m->T, m->P, m->WS + m->W.train, mlp_desc(m), fmt,
                                                     d_feat_q16, d_labels, n_rows, nullptr, 0, d_grad, d_loss,
                                                     stream, status_word(m), fused_fwd(m, fmt, &ff)));
    return cuda_status(adv::launch_train_step(m->L, m->T, m->P, m->WS + m->W.train, mlp_desc(m), d_feat_q16,
                                              d_labels, n_rows, nullptr, 0, d_grad, d_loss, m->num_sms, stream));
}

advisor_status advisor_model_set_profile_events(advisor_model_t m, void* ev_start, void* ev_stop) {
    if (!m || (ev_start == nullptr) != (ev_stop == nullptr)) return ADVISOR_ERR_INVALID_ARGUMENT;
    m->prof_start = static_cast<cudaEvent_t>(ev_start);
    m->prof_stop = static_cast<cudaEvent_t>(ev_stop);
    return ADVISOR_OK;
}

advisor_status advisor_forward_saved(advisor_model_t m, const int32_t* d_feat_q16, int64_t n_rows,
                                     advisor_precision precision, float* d_y, cudaStream_t stream) {
    if (!m || !d_feat_q16 || n_rows < 1) return ADVISOR_ERR_INVALID_ARGUMENT;
    advisor_status st = check_ready(m, n_rows);
    if (st != ADVISOR_OK) return st;
    const int fmt = train_fmt(m, precision);
    if (fmt < 0) return ADVISOR_ERR_UNSUPPORTED;
    adv::FusedFwd ff{};
    cudaError_t e = fmt == 0 ? adv::launch_forward_saved(m->L, m->T, m->WS + m->W.train, mlp_desc(m), d_feat_q16,
                                                         n_rows, d_y, stream)
                             : adv::launch_forward_saved_tc(m->L, m->T, m->WS + m->W.train, mlp_desc(m), fmt,
                                                            d_feat_q16, n_rows, d_y, stream, status_word(m),
                                                            fused_fwd(m, fmt, &ff));
    if (e != cudaSuccess) return ADVISOR_ERR_CUDA;
    m->saved_rows = n_rows;
    m->saved_fmt = fmt;
    return ADVISOR_OK;
}

advisor_status advisor_backward(advisor_model_t m, const float* d_dy, int64_t n_rows, float* d_grad,
                                cudaStream_t stream) {
    if (!m || !d_dy || !d_grad || n_rows < 1) return ADVISOR_ERR_INVALID_ARGUMENT;
    if (n_rows != m->saved_rows) return ADVISOR_ERR_INVALID_ARGUMENT;
    if (m->saved_fmt != 0)
        return cuda_status(adv::launch_backward_tc(m->L, m->T, m->WS + m->W.train, mlp_desc(m), m->saved_fmt,
                                                   d_dy, n_rows, d_grad, stream, status_word(m)));
    return cuda_status(adv::launch_backward(m->L, m->T, m->WS + m->W.train, mlp_desc(m), d_dy, n_rows, d_grad, stream));
}

advisor_status advisor_model_repack(advisor_model_t m, cudaStream_t stream) {
    if (!m || !m->P) return ADVISOR_ERR_INVALID_ARGUMENT;
    const advisor_status st = cuda_status(adv::launch_repack(m->L, m->P, stream));
    if (st == ADVISOR_OK) m->images_stale = false;
    return st;
}

advisor_status advisor_model_refresh(advisor_model_t m, cudaStream_t stream) {
    if (!m || !m->P) return ADVISOR_ERR_INVALID_ARGUMENT;
    return cuda_status(ensure_images(m, stream));
}

size_t advisor_model_master_offset(advisor_model_t m) { return m ? m->L.p_master : 0; }

int64_t advisor_model_get_adam_step(advisor_model_t m) { return m ? m->adam_step : -1; }

advisor_status advisor_model_set_adam_step(advisor_model_t m, int64_t step) {
    if (!m || step < 0) return ADVISOR_ERR_INVALID_ARGUMENT;
    m->adam_step = step;
    return ADVISOR_OK;
}

advisor_status advisor_get_device_status(advisor_model_t m, cudaStream_t stream) {
    if (!m || !m->P) return ADVISOR_ERR_INVALID_ARGUMENT;
    int h = 0;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return ADVISOR_ERR_CUDA;
    if (cudaMemcpy(&h, m->P + m->L.p_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return ADVISOR_ERR_CUDA;
    if (cudaMemset(m->P + m->L.p_status, 0, sizeof(int)) != cudaSuccess) return ADVISOR_ERR_CUDA;
    if (h & ADV_DEV_TIMEOUT) return ADVISOR_ERR_TIMEOUT;
    if (h & ADV_DEV_BAD_SEGMENTS) return ADVISOR_ERR_BAD_SEGMENTS;
    return ADVISOR_OK;
}

advisor_status advisor_model_check_wait_timeout(advisor_model_t m, int64_t timeout_ns, cudaStream_t stream) {
    if (!m || !m->P) return ADVISOR_ERR_INVALID_ARGUMENT;
    if (timeout_ns < 1000 || timeout_ns > 1000000000) return ADVISOR_ERR_INVALID_ARGUMENT;
    return adv::launch_wait_timeout_check(status_word(m), (uint64_t)timeout_ns, stream) == cudaSuccess
               ? ADVISOR_OK
               : ADVISOR_ERR_CUDA;
}

// Read-only view of a bound model for the no-allocation scoring entry point
// (noalloc.cu); allocates nothing.
// Rebuild stale derived copies before a no-allocation scoring call; 0 on a CUDA error.
int adv_model_prepare(advisor_model_t m, cudaStream_t stream) {
    return m && ensure_images(m, stream) == cudaSuccess ? 1 : 0;
}

int adv_model_noalloc_view(advisor_model_t m, int fmt_idx, adv::NoallocModelView* out) {
    if (!m || !out) return 0;
    out->ready = (m->P != nullptr && m->params_set) ? 1 : 0;
    out->F = m->L.F;
    out->nslab0 = m->L.n_hidden > 0 ? m->L.nslab[0] : 0;
    out->tc_ok = tc_supported(m) ? 1 : 0;
    out->num_sms = m->num_sms;
    out->tc_ctas = m->cfg.tc_ctas;
    if (!out->ready) return 1;
    out->sa = reinterpret_cast<const float*>(m->P + m->L.p_stdz_a);
    out->sc = reinterpret_cast<const float*>(m->P + m->L.p_stdz_c);
    out->tc = tc_args(m, nullptr, 0, nullptr, nullptr, fmt_idx);
    return 1;
}

}  // extern "C"
