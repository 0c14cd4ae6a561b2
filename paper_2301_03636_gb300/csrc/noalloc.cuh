// Shared between api.cu and noalloc.cu: what the no-allocation scoring entry
// point needs to know about a bound model.
#pragma once
#include "mlp.cuh"

namespace adv {

// Layout facts the entry point needs from the model object (api.cu).
struct NoallocModelView {
    int F;
    int nslab0;
    const float* sa;
    const float* sc;
    TcArgs tc;   // weights, biases, output row, geometry; x_img/n_rows/scores/status filled per call
    int num_sms;
    int tc_ctas;   // the model's CTA count for the tensor-core scorer (0: one per SM)
    int tc_ok;
    int ready;
};

}  // namespace adv

// Provided by api.cu: a read-only view of a bound model (allocates nothing).
extern "C" int adv_model_noalloc_view(advisor_model_t m, int fmt_idx, adv::NoallocModelView* out);
extern "C" int adv_model_prepare(advisor_model_t m, cudaStream_t stream);
