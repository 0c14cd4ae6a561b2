// Training-mode kernels (train.cu): forward with saved activations, MSE loss
// on ln runtime, hand-written backward, Adam.
#pragma once
#include <cuda.h>   // CUtensorMap (the encoder is reached through the runtime's driver entry point)

#include "mlp.cuh"

namespace adv {

struct TrainLayout {
    size_t act[ADV_MAX_LAYERS + 1];   // act[0] = standardised input z [R][F]; act[l] = layer-l output [R][w_l]
    size_t dA, dB;                    // gradient ping-pong [R][wmax]
    size_t grad;                      // [n_params]
    size_t part;                      // split-K partial sums [splits][max(out*in + out)]
    size_t loss_part;                 // per-block loss partial sums
    size_t loss;                      // 1 float
    // 16-bit tensor-core path (train_tc.cu)
    size_t x16;                       // standardised input [R][F], 16-bit
    size_t h16[ADV_MAX_LAYERS];       // hidden-layer outputs [R][w_{l+1}], 16-bit
    size_t w16[ADV_MAX_LAYERS];       // row-major 16-bit copies of the hidden layers' weights
    size_t dz16[2];                   // dZ ping-pong [R][wmax], 16-bit
    size_t c32;                       // FP32 GEMM output [R][wmax] (aliases dB)
    size_t bias_part;                 // bias / output-row gradient partials of the 16-bit backward
    int64_t bias_part_floats;         //   (kept apart from `part`, summed in one launch at its end)
    int splits;
    int64_t rows;
    size_t bytes;
};

struct AdamHyper {
    float lr, beta1, beta2, eps, weight_decay;
};

// Bytes of the training region for up to R rows; fills *t.
size_t train_layout(const ModelLayout& L, int64_t R, TrainLayout* t);

// Forward + loss + backward; with `adam` non-null also the Adam update of the
// master weights (step counts from 1) and the repack of the derived copies.
// d_grad_out (nullable) receives the FP32 gradient, d_loss (nullable) the loss.
cudaError_t launch_train_step(const ModelLayout& L, const TrainLayout& T, uint8_t* P, uint8_t* TW,
                              const MlpDesc& md, const int32_t* feat, const float* labels, int64_t n,
                              const AdamHyper* adam, int64_t step, float* d_grad_out, float* d_loss, int num_sms,
                              cudaStream_t s);

// Forward pass keeping every layer's output in the training region; the
// output y (n floats) is copied to d_y when non-null.
cudaError_t launch_forward_saved(const ModelLayout& L, const TrainLayout& T, uint8_t* TW, const MlpDesc& md,
                                 const int32_t* feat, int64_t n, float* d_y, cudaStream_t s);
// Backward of the last saved forward (same n) from dL/dy to d_grad.
cudaError_t launch_backward(const ModelLayout& L, const TrainLayout& T, uint8_t* TW, const MlpDesc& md,
                            const float* d_dy, int64_t n, float* d_grad, cudaStream_t s);

// dL/dy (into the dA buffer) and the loss of the saved forward output.
cudaError_t launch_mse_loss(const ModelLayout& L, const TrainLayout& T, uint8_t* TW, const float* labels, int64_t n,
                            float* d_loss, cudaStream_t s);
// Adam update of the master weights (step counts from 1), then the repack.
// The optimizer kernels update the FP32 masters only; the derived inference
// copies (16-bit and E4M3 images, transposed copy, padded biases) are rebuilt
// by the caller before the next scoring call (launch_repack).
cudaError_t launch_adam_update(const ModelLayout& L, uint8_t* P, const float* grad, const AdamHyper& adam,
                               int64_t step, cudaStream_t s);

// Backward of the saved forward from dL/dy already in the dA buffer.
cudaError_t launch_backward_saved(const ModelLayout& L, const TrainLayout& T, uint8_t* TW, const MlpDesc& md,
                                  int64_t n, float* grad, cudaStream_t s);

// Optimizer and loss of a training step: optimizer 0 Adam (h), 1 RMSprop
// (h.lr, alpha, h.eps, h.weight_decay added to the gradient); loss 0 MSE
// (0.5 mean (y - t)^2), 1 RMSE (sqrt(mean (y - t)^2)).
struct TrainOptions {
    int optimizer;
    int loss;
    AdamHyper h;
    float alpha;
};
// The 16-bit training forward through the fused tensor-core scorer (for
// models it covers, hidden widths multiples of 8): one launch packs this
// step's weights (the scorer's swizzled 16-bit images, the padded biases and
// output row, and the row-major 16-bit copies the backward GEMMs use), the
// features are standardised into the scorer's image and the row-major copy,
// and the scorer writes each hidden layer's activations and the output.
struct FusedFwd {
    TcArgs tc;                              // scores -> the output y; save_act set by the forward
    uint8_t* x_img;                         // workspace image of the batch
    int num_sms, ctas;
    uint8_t* img16[2][ADV_MAX_LAYERS];      // [BF16, FP16][hidden layer] images in the parameter block
    float* bias_pad[ADV_MAX_LAYERS];
    float* wout_pad;
};

// One training step with these options; fmt 0 FP32 SIMT, 1 BF16, 2 FP16.
// ff (nullable): the fused forward for fmt 1 / 2.
cudaError_t launch_train_step_ex(const ModelLayout& L, const TrainLayout& T, uint8_t* P, uint8_t* TW,
                                 const MlpDesc& md, int fmt, const int32_t* feat, const float* labels, int64_t n,
                                 const TrainOptions& o, int64_t step, float* d_loss, cudaStream_t s, int* status_word,
                                 const FusedFwd* ff = nullptr);

// Dense GEMM on the tensor cores (gemm_tc.cu): C[m][n] = sum_k A(m,k) B(n,k),
// 16-bit operands, FP32 accumulation.  A(m, k) = A[m * lda + k] (a_mn == 0,
// K-major) or A[k * lda + m] (a_mn == 1, MN-major), likewise B.  C row-major
// with leading dimension ldc: FP32, or the operands' 16-bit type (c16, round
// to nearest).  splits > 1 splits K over CTAs: FP32 partials go to part
// ([splits][M][ldc]) and are added in split order into C.
struct TcGemm {
    // TMA tensor maps of A and B (set by launch_gemm_tc when both operands'
    // row strides are multiples of 16 bytes and their bases 16-byte aligned)
    CUtensorMap tma_a, tma_b;
    int use_tma;
    int box_b;             // B rows per K block in the TMA path (64-multiple <= 256)
    int stages;            // ring depth of the TMA path (2 .. 4; set by launch_gemm_tc)
    const uint16_t* A;
    int64_t lda;
    int a_mn;
    const uint16_t* B;
    int64_t ldb;
    int b_mn;
    int64_t M, N, K;
    void* C;
    int64_t ldc;
    int c16;
    float* part;
    int splits;
    int fmt;               // 1 BF16, 0 FP16
    int* status_word;
    uint64_t timeout_ns;
    // Masked form (c16 = 1, splits = 1): C[m][n] = 16-bit(acc) where
    // mask_h[m][n] > 0, else 0 (ReLU backward; mask_h row stride ldc), and
    // colpart[m / 128][n] = the sum over the tile's rows of the stored C
    // (bias-gradient partials, one row per 128-row tile, row stride N).
    const uint16_t* mask_h;
    float* colpart;
};
cudaError_t launch_gemm_tc(const TcGemm& g, cudaStream_t s);

// TMA tensor map of a row-major 16-bit array [rows][cols] (cols * 2 a multiple
// of 16 bytes, 16-byte aligned base): box 64 columns x box_rows rows with the
// 128-byte swizzle; fmt 1 BF16, else FP16.  False when it cannot be made.
bool encode_rows_map(CUtensorMap* map, const void* p, int64_t cols, int64_t rows, int box_rows, int fmt);

// ReLU backward through a hidden layer in one persistent kernel (the masked
// form of TcGemm, specialised): dz[r][j] = 16-bit(sum_k dza[r][k] W[k][j])
// where h[r][j] > 0, else 0, for r < n, j < fi, k < fo; and the bias-gradient
// partials colpart[p][j] (p < *parts) whose sum over p in order is
// sum_r dz[r][j].  W stays in shared memory; 128-row tiles are dealt to the
// CTAs round robin.  16-bit arrays row-major, 16-byte aligned; fo, fi
// multiples of 8 and <= 256.  Returns cudaErrorNotSupported (nothing
// launched) for shapes outside that, or when colpart_cap floats cannot hold
// the partials.
cudaError_t launch_dgrad_mask(const uint16_t* dza, int fo, const uint16_t* W, int fi, const uint16_t* h, int64_t n,
                              uint16_t* dz, float* colpart, int64_t colpart_cap, int* parts, int fmt,
                              int* status_word, cudaStream_t s);

// 16-bit operands on the tensor cores (train_tc.cu); fmt 1 BF16, 2 FP16.
cudaError_t launch_forward_saved_tc(const ModelLayout& L, const TrainLayout& T, uint8_t* TW, const MlpDesc& md,
                                    int fmt, const int32_t* feat, int64_t n, float* d_y, cudaStream_t s,
                                    int* status_word, const FusedFwd* ff = nullptr);
// MSE loss and backward of the saved 16-bit forward (y in the training region):
// the loss (to the loss buffer and d_loss, nullable) and the gradient; where the
// vectorised backward applies, dL/dy is computed inside it.
cudaError_t launch_loss_backward_tc(const ModelLayout& L, const TrainLayout& T, uint8_t* TW, const MlpDesc& md,
                                    int fmt, const float* labels, int64_t n, float* d_grad, float* d_loss,
                                    cudaStream_t s, int* status_word);
cudaError_t launch_backward_tc(const ModelLayout& L, const TrainLayout& T, uint8_t* TW, const MlpDesc& md, int fmt,
                               const float* d_dy, int64_t n, float* d_grad, cudaStream_t s, int* status_word);
cudaError_t launch_train_step_tc(const ModelLayout& L, const TrainLayout& T, uint8_t* P, uint8_t* TW,
                                 const MlpDesc& md, int fmt, const int32_t* feat, const float* labels, int64_t n,
                                 const AdamHyper* adam, int64_t step, float* d_grad_out, float* d_loss,
                                 cudaStream_t s, int* status_word, const FusedFwd* ff = nullptr);

}  // namespace adv
