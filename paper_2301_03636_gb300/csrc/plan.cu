// Plans: the batched ranking path (a1-a7) captured once into a CUDA graph
// and replayed, with an optional autotuner over launch shapes.
//
// Fig. 2 of arXiv 2301.03636 runs every generated variant of a kernel
// through feature extraction, the cost model and a selection; batching many
// kernels' variants into one pass makes that a fixed sequence of six
// kernels and a memset whose shapes depend only on the batch size.  Replaying
// the sequence as one graph removes the per-launch host overhead and the
// gaps between kernels.  The autotuner measures a small set of launch shapes
// (advisor_launch_config) on the caller's own data and keeps the fastest;
// the shapes never change the selections (the layer-by-layer path changes
// the last bits of the 16-bit scores, within their error bound).
//
// Besides the library's public entry points, two internal hooks are used:
// the launch counter and the model's record of which re-score tiers the
// last selection ran (where advisor_get_rescore_counts finds each tier's
// count), which every replay sets to its own plan's.
#include <algorithm>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "advisor.h"

extern "C" void adv_count_launch(int n);
extern "C" int adv_model_last_mid(advisor_model_t m);
extern "C" void adv_model_set_last_mid(advisor_model_t m, int mid);

struct advisor_plan {
    advisor_model_t model = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    advisor_launch_config cfg{};
    float replay_us = 0.f;
    int32_t kernels = 0;
    int mid = 0;   // the captured selection runs the FP16 middle tier
};

namespace {

struct RankCall {
    advisor_model_t m;
    const advisor_variant_desc* desc;
    int64_t n_rows;
    const int64_t* off;
    int64_t n_kernels;
    advisor_precision precision;
    float eps, eps16, eps32;   // eps16 < 0: no FP16 tier
    int32_t* best;
    double* best_score;
    float* scores;
    uint8_t* status;
    const advisor_variant_desc* h_desc;   // non-null: advisor_rank_staged from these host descriptors into desc
    int32_t n_stages;
};

bool same(const advisor_launch_config& a, const advisor_launch_config& b) {
    return a.extract_block == b.extract_block && a.tc_ctas == b.tc_ctas &&
           a.list_blocks_per_sm == b.list_blocks_per_sm && a.list_chunk_kb == b.list_chunk_kb &&
           a.select_block == b.select_block && a.layer_path == b.layer_path;
}

void release(cudaGraph_t g, cudaGraphExec_t x) {
    if (x) cudaGraphExecDestroy(x);
    if (g) cudaGraphDestroy(g);
}

// Capture advisor_rank on `cap` with the model's current configuration.
advisor_status capture(const RankCall& r, cudaStream_t cap, cudaGraph_t* g_out, cudaGraphExec_t* x_out,
                       int32_t* kernels) {
    *g_out = nullptr;
    *x_out = nullptr;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return ADVISOR_ERR_CUDA;
    const long long before = advisor_launch_count();
    const advisor_status st =
        r.h_desc ? advisor_rank_staged_ex(r.m, r.h_desc, const_cast<advisor_variant_desc*>(r.desc), r.n_rows, r.off,
                                          r.n_kernels, r.precision, r.eps, r.eps16, r.eps32, r.best, r.best_score,
                                          r.scores, r.status, r.n_stages, cap)
                 : advisor_rank_ex(r.m, r.desc, r.n_rows, r.off, r.n_kernels, r.precision, r.eps, r.eps16, r.eps32,
                                   r.best, r.best_score, r.scores, r.status, cap);
    // the launches were only recorded; replays account for them instead
    adv_count_launch(-(int)(advisor_launch_count() - before));
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cap, &g);
    if (st != ADVISOR_OK || e != cudaSuccess) {
        release(g, nullptr);
        cudaGetLastError();
        return st != ADVISOR_OK ? st : ADVISOR_ERR_CUDA;
    }
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) { release(g, nullptr); return ADVISOR_ERR_CUDA; }
    std::vector<cudaGraphNode_t> nodes(n);
    int32_t k = 0;
    if (n > 0 && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) { release(g, nullptr); return ADVISOR_ERR_CUDA; }
    for (size_t i = 0; i < n; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    cudaGraphExec_t x = nullptr;
    if (cudaGraphInstantiate(&x, g, 0) != cudaSuccess) {
        release(g, nullptr);
        cudaGetLastError();
        return ADVISOR_ERR_CUDA;
    }
    *g_out = g;
    *x_out = x;
    *kernels = k;
    return ADVISOR_OK;
}

// Median time of `reps` replays after `warm` unmeasured ones, in microseconds.
advisor_status time_replays(cudaGraphExec_t x, cudaStream_t s, int warm, int reps, float* us) {
    for (int i = 0; i < warm; ++i)
        if (cudaGraphLaunch(x, s) != cudaSuccess) return ADVISOR_ERR_CUDA;
    std::vector<cudaEvent_t> ev(2 * reps, nullptr);
    advisor_status st = ADVISOR_OK;
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) st = ADVISOR_ERR_CUDA;
    std::vector<float> t;
    for (int i = 0; st == ADVISOR_OK && i < reps; ++i) {
        if (cudaEventRecord(ev[2 * i], s) != cudaSuccess || cudaGraphLaunch(x, s) != cudaSuccess ||
            cudaEventRecord(ev[2 * i + 1], s) != cudaSuccess)
            st = ADVISOR_ERR_CUDA;
    }
    if (st == ADVISOR_OK && cudaStreamSynchronize(s) != cudaSuccess) st = ADVISOR_ERR_CUDA;
    for (int i = 0; st == ADVISOR_OK && i < reps; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]) != cudaSuccess) st = ADVISOR_ERR_CUDA;
        t.push_back(ms * 1000.f);
    }
    for (auto e : ev)
        if (e) cudaEventDestroy(e);
    if (st != ADVISOR_OK) return st;
    std::sort(t.begin(), t.end());
    *us = t[t.size() / 2];
    return ADVISOR_OK;
}

// Capture with `c` and time it; on any failure of this candidate (e.g. a
// shape the model's widths do not fit) the candidate is skipped.
bool try_candidate(const RankCall& r, const advisor_launch_config& c, cudaStream_t cap, cudaStream_t s,
                   float* us) {
    if (advisor_model_set_launch_config(r.m, &c) != ADVISOR_OK) return false;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    int32_t k = 0;
    if (capture(r, cap, &g, &x, &k) != ADVISOR_OK) return false;
    const advisor_status st = time_replays(x, s, 3, 15, us);
    release(g, x);
    return st == ADVISOR_OK;
}

// Autotune (optionally) and capture one ranking call into a plan.
advisor_status make_plan(const RankCall& r, int32_t autotune, cudaStream_t stream, advisor_plan_t* out) {
    advisor_model_t m = r.m;
    const int64_t n_rows = r.n_rows;
    if (!m || !out) return ADVISOR_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    advisor_launch_config saved{};
    advisor_status st = advisor_model_get_launch_config(m, &saved);
    if (st != ADVISOR_OK) return st;
    st = advisor_model_refresh(m, stream);
    if (st != ADVISOR_OK) return st;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return ADVISOR_ERR_CUDA;
    cudaStream_t cap = nullptr;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return ADVISOR_ERR_CUDA;
    advisor_launch_config best = saved;
    float best_us = 0.f;
    if (autotune) {
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        // tensor-core scorer: one CTA per SM, or the fewest CTAs that keep
        // the same number of 128-row tiles on the busiest CTA
        const int64_t tiles = (n_rows + 127) / 128;
        const int64_t per = tiles > 0 ? (tiles + sms - 1) / sms : 1;
        const int balanced = (int)((tiles + per - 1) / per);
        if (!try_candidate(r, best, cap, stream, &best_us)) {
            advisor_model_set_launch_config(m, &saved);
            cudaStreamDestroy(cap);
            return ADVISOR_ERR_CUDA;
        }
        // one setting at a time, in the order the kernels run
        for (int knob = 0; knob < 5; ++knob) {
            std::vector<advisor_launch_config> cands;
            advisor_launch_config c = best;
            if (knob == 0) {
                for (int b : {64, 128, 256}) { c.extract_block = b; cands.push_back(c); }
            } else if (knob == 1) {
                for (int t : {0, balanced}) { c.tc_ctas = t; cands.push_back(c); }
            } else if (knob == 2) {
                c.list_blocks_per_sm = 1; c.list_chunk_kb = 32; cands.push_back(c);
                c.list_blocks_per_sm = 2; c.list_chunk_kb = 16; cands.push_back(c);
                c.list_blocks_per_sm = 1; c.list_chunk_kb = 16; cands.push_back(c);
            } else if (knob == 3) {
                for (int b : {128, 256}) { c.select_block = b; cands.push_back(c); }
            } else {
                for (int lp : {0, 1}) { c.layer_path = lp; cands.push_back(c); }
            }
            for (const auto& cand : cands) {
                if (same(cand, best)) continue;
                float us = 0.f;
                if (try_candidate(r, cand, cap, stream, &us) && us < best_us) {
                    best_us = us;
                    best = cand;
                }
            }
        }
    }
    st = advisor_model_set_launch_config(m, &best);
    advisor_plan* p = nullptr;
    if (st == ADVISOR_OK) {
        p = new (std::nothrow) advisor_plan();
        if (!p) st = ADVISOR_ERR_OUT_OF_MEMORY;
    }
    if (st == ADVISOR_OK) st = capture(r, cap, &p->graph, &p->exec, &p->kernels);
    advisor_model_set_launch_config(m, &saved);
    cudaStreamDestroy(cap);
    if (st != ADVISOR_OK) {
        delete p;
        return st;
    }
    p->model = m;
    p->mid = adv_model_last_mid(m);   // set by the capture's selection
    p->cfg = best;
    p->replay_us = autotune ? best_us : 0.f;
    *out = p;
    return ADVISOR_OK;
}

}  // namespace

extern "C" {

advisor_status advisor_plan_rank_ex(advisor_model_t m, const advisor_variant_desc* d_desc, int64_t n_rows,
                                    const int64_t* d_seg_off, int64_t n_kernels, advisor_precision precision,
                                    float eps_scores, float eps_fp16, float eps_fp32, int32_t* d_best_local,
                                    double* d_best_score, float* d_scores, uint8_t* d_row_status, int32_t autotune,
                                    cudaStream_t stream, advisor_plan_t* out) {
    const RankCall r{m, d_desc, n_rows, d_seg_off, n_kernels, precision, eps_scores, eps_fp16, eps_fp32,
                     d_best_local, d_best_score, d_scores, d_row_status, nullptr, 1};
    return make_plan(r, autotune, stream, out);
}

advisor_status advisor_plan_rank(advisor_model_t m, const advisor_variant_desc* d_desc, int64_t n_rows,
                                 const int64_t* d_seg_off, int64_t n_kernels, advisor_precision precision,
                                 float eps_scores, float eps_fp32, int32_t* d_best_local, double* d_best_score,
                                 float* d_scores, uint8_t* d_row_status, int32_t autotune, cudaStream_t stream,
                                 advisor_plan_t* out) {
    return advisor_plan_rank_ex(m, d_desc, n_rows, d_seg_off, n_kernels, precision, eps_scores, -1.f, eps_fp32,
                                d_best_local, d_best_score, d_scores, d_row_status, autotune, stream, out);
}

advisor_status advisor_plan_rank_staged_ex(advisor_model_t m, const advisor_variant_desc* h_desc,
                                           advisor_variant_desc* d_desc, int64_t n_rows, const int64_t* d_seg_off,
                                           int64_t n_kernels, advisor_precision precision, float eps_scores,
                                           float eps_fp16, float eps_fp32, int32_t* d_best_local,
                                           double* d_best_score, float* d_scores, uint8_t* d_row_status,
                                           int32_t n_stages, int32_t autotune, cudaStream_t stream,
                                           advisor_plan_t* out) {
    if (!h_desc) return ADVISOR_ERR_INVALID_ARGUMENT;
    const RankCall r{m, d_desc, n_rows, d_seg_off, n_kernels, precision, eps_scores, eps_fp16, eps_fp32,
                     d_best_local, d_best_score, d_scores, d_row_status, h_desc, n_stages};
    return make_plan(r, autotune, stream, out);
}

advisor_status advisor_plan_rank_staged(advisor_model_t m, const advisor_variant_desc* h_desc,
                                        advisor_variant_desc* d_desc, int64_t n_rows, const int64_t* d_seg_off,
                                        int64_t n_kernels, advisor_precision precision, float eps_scores,
                                        float eps_fp32, int32_t* d_best_local, double* d_best_score,
                                        float* d_scores, uint8_t* d_row_status, int32_t n_stages,
                                        int32_t autotune, cudaStream_t stream, advisor_plan_t* out) {
    return advisor_plan_rank_staged_ex(m, h_desc, d_desc, n_rows, d_seg_off, n_kernels, precision, eps_scores,
                                       -1.f, eps_fp32, d_best_local, d_best_score, d_scores, d_row_status, n_stages,
                                       autotune, stream, out);
}

advisor_status advisor_plan_launch(advisor_plan_t p, cudaStream_t stream) {
    if (!p || !p->exec) return ADVISOR_ERR_INVALID_ARGUMENT;
    // derived copies an optimizer step left stale are rebuilt before the replay
    const advisor_status st = advisor_model_refresh(p->model, stream);
    if (st != ADVISOR_OK) return st;
    if (cudaGraphLaunch(p->exec, stream) != cudaSuccess) return ADVISOR_ERR_CUDA;
    adv_model_set_last_mid(p->model, p->mid);
    adv_count_launch(p->kernels);
    return ADVISOR_OK;
}

advisor_status advisor_plan_info(advisor_plan_t p, advisor_launch_config* cfg, float* replay_us,
                                 int32_t* kernels_per_replay) {
    if (!p) return ADVISOR_ERR_INVALID_ARGUMENT;
    if (cfg) *cfg = p->cfg;
    if (replay_us) *replay_us = p->replay_us;
    if (kernels_per_replay) *kernels_per_replay = p->kernels;
    return ADVISOR_OK;
}

advisor_status advisor_plan_destroy(advisor_plan_t p) {
    if (!p) return ADVISOR_OK;
    release(p->graph, p->exec);
    delete p;
    return ADVISOR_OK;
}

}  // extern "C"
