// Kernel argument structures and launcher declarations shared by the
// translation units of libadvisor.
#pragma once
#include "common.cuh"

namespace adv {

// FP32 master parameters of the MLP as seen by the SIMT kernels.
struct MlpDesc {
    int nw;
    int widths[ADV_MAX_LAYERS + 1];
    const float* W[ADV_MAX_LAYERS];    // [out][in]
    const float* b[ADV_MAX_LAYERS];    // [out]
    const float* WT[ADV_MAX_LAYERS];   // [in][wt_ld] (transposed copy, rows zero-padded to wt_ld)
    int wt_ld[ADV_MAX_LAYERS];         // out rounded up to a multiple of 4
    const float* sa;                   // z = f * sa - sc (FP32 standardisation)
    const float* sc;
    const double* mu;                  // FP64 standardisation
    const double* sigma;
};

// Where the rows of a scoring call come from.
struct RowSrc {
    const int32_t* feat;               // [n][F] int32 features, or nullptr: recompute from desc
    const advisor_variant_desc* desc;
    const int64_t* rows;               // list of row indices (nullptr: identity)
    const int* count_dev;              // device-side list length (nullptr: use count)
    int64_t count;
    const uint8_t* status;             // row status (nullable), indexed by row
};

// extract.cu
struct ExtractArgs {
    const advisor_variant_desc* desc;
    int64_t n_rows;
    int64_t n_rows_padded;   // rows covered (X image rows incl. zero padding)
    int32_t* feat;           // nullable
    uint8_t* status;         // nullable
    uint8_t* x_img;          // nullable
    int nslab;               // slabs of the X image
    const float* sa;         // standardisation: z = f * sa - sc
    const float* sc;
    const float* x8_scale;   // E4M3 image (format 3): the first layer's activation scale (device)
    // gathered extraction (launch_extract_list): image position p holds
    // descriptor row rows[p] for p < min(*count_dev, n_rows)
    const int64_t* rows;
    const int* count_dev;
};
// Launch shapes of the hot path that a plan's autotuner may vary.  Every
// choice but layer_path gives bit-identical results: rows, segments and tiles
// are processed by the same per-row / per-segment code whatever the grid or
// block shape, and no summation order depends on them; layer_path changes
// the tensor-core accumulation order (results agree within the 16-bit error
// bound, and the tiered re-score keeps the selections exact).
struct LaunchConfig {
    int extract_block = 128;       // threads per block of the extraction kernel: 64, 128 or 256
    int tc_ctas = 0;               // CTAs of the persistent tensor-core scorer: 0 = one per SM
    int list_blocks_per_sm = 1;    // FP32 near-tie scorer: blocks per SM, 1 or 2
    int list_chunk_kb = 32;        // FP32 near-tie scorer: weight chunk per bulk copy, 16 or 32 KB
    int select_block = 256;        // threads per block of the selection kernels: 128 or 256
    int layer_path = 0;            // 1: run models that fit the fused scorer layer by layer instead
};
bool launch_config_valid(const LaunchConfig& c);

cudaError_t launch_extract(const ExtractArgs& a, int F, int fmt, cudaStream_t s, int block = 128);
cudaError_t launch_extract_list(const ExtractArgs& a, int F, int fmt, int num_sms, cudaStream_t s);
// x_rm (16-bit formats, F % 8 == 0): also the standardised rows row-major
// ([n][F], the same values as the image) for the training step's weight gradient.
cudaError_t launch_standardize(const int32_t* feat, const uint8_t* status, int64_t n, int64_t npad, uint8_t* x_img,
                               int nslab, const float* sa, const float* sc, int F, int fmt, cudaStream_t s,
                               const float* x8_scale = nullptr, uint16_t* x_rm = nullptr);
cudaError_t launch_fit_standardizer(const int32_t* feat, const uint8_t* status, int64_t n, int F, double* mu,
                                    double* sigma, cudaStream_t s);

// mlp_simt.cu
cudaError_t launch_mlp_fp32(const MlpDesc& m, const RowSrc& src, float* out, int num_sms, bool for_list,
                            cudaStream_t s, int* status_word = nullptr, int list_blocks_per_sm = 1,
                            int list_chunk_kb = 32);
struct SelectArgs;
// fin (nullable): the argmin's selection state; the last block then makes the
// final selection (see mlp_fp64_kernel), with fin->counters[3] zeroed beforehand
cudaError_t launch_mlp_fp64(const MlpDesc& m, const RowSrc& src, double* out, int num_sms, cudaStream_t s,
                            const SelectArgs* fin = nullptr);

// mlp_tc.cu
struct TcArgs {
    const uint8_t* x_img;                  // [n_tiles][nslab0][16 KB]
    const uint8_t* w_img[ADV_MAX_LAYERS];  // per hidden layer: [nslab_l][npad_l * 128 B]
    const float* bias[ADV_MAX_LAYERS];     // per hidden layer, padded to npad_l with zeros
    const float* w_out;                    // [npad_last], padded with zeros
    const float* b_out;                    // 1 float
    int npad[ADV_MAX_LAYERS];
    int nslab[ADV_MAX_LAYERS];
    int n_hidden;
    int nmax;
    int fmt;                               // 1 BF16, 0 F16 (instruction descriptor encoding)
    int64_t n_rows;
    int n_tiles;
    const int* n_rows_dev;                 // nullable: rows = min(*n_rows_dev, n_rows), read on the device
    const uint8_t* status;                 // nullable
    float* scores;
    int* status_word;
    unsigned long long timeout_ns;
    // training forward (nullable per layer): hidden layer l's post-ReLU 16-bit
    // activations, row-major [n_rows][save_ld[l]] (save_ld[l] a multiple of 8)
    void* save_act[ADV_MAX_LAYERS];
    int save_ld[ADV_MAX_LAYERS];
    // with use_tma_save, tm_save[l] maps save_act[l] (dims {save_ld[l], n_rows},
    // box 64 columns x 128 rows, 128-byte swizzle: one slab of the shared-memory
    // image) and every hidden layer but the last is stored from that image by TMA
    // instead of row by row from the epilogue's registers
    CUtensorMap tm_save[ADV_MAX_LAYERS];
    int use_tma_save;
};
cudaError_t launch_mlp_tc(const TcArgs& a, int num_sms, cudaStream_t s, int ctas = 0);

// One hidden layer of a wide MLP on the tensor cores (csrc/mlp_layer_tc.cu).
struct LayerArgs {
    const uint8_t* a_img;     // input image: [tile][a_slabs][128 rows x 128 B], 128B swizzle
    int a_slabs;              // input slabs (kpad / 64)
    const uint8_t* w_img;     // weights: [a_slabs][npad rows][128 B] (the packed 16-bit image)
    int npad;                 // output width rounded up to 64
    int n_chunks;             // ceil(npad / 256)
    int n_tiles;              // 128-row tiles (capacity; the stride of `partial`)
    const int* n_rows_dev;    // nullable: only the tiles of the first *n_rows_dev rows are computed
    const float* bias;        // [npad]
    int mode;                 // 0: ReLU -> out_img; 1: ReLU, dot with w_out -> partial
    uint8_t* out_img;         // mode 0: [tile][npad / 64][128 x 128 B]
    const float* w_out;       // mode 1: [npad]
    float* partial;           // mode 1: [n_chunks][2][n_tiles * 128]
    int fmt;                  // operands: 1 BF16, 0 F16 (kind::f16), 2 E4M3 (kind::f8f6f4)
    const float* fp8;         // E4M3: the model's FP8 scale block (ADV_FP8_*)
    int layer;                // E4M3: hidden-layer index (its scales)
    int* status_word;
    uint64_t timeout_ns;
};
size_t mlp_layer_tc_smem_bytes();
cudaError_t launch_mlp_layer_tc(const LayerArgs& a, int num_sms, cudaStream_t s);
cudaError_t launch_sum_partials(const float* partial, int n_parts, int64_t stride, int64_t n_rows, const float* b_out,
                                const uint8_t* status, float* scores, int num_sms, cudaStream_t s,
                                const int* n_rows_dev = nullptr);
size_t mlp_tc_smem_bytes(int nslab_max, int nmax, int n_hidden);

// select.cu
struct SelectArgs {
    const float* scores;
    int64_t n_rows;
    const int64_t* off;
    int64_t n_kernels;
    int32_t* best;
    double* best_score;
    float eps;                 // < 0: plain argmin
    float eps32;
    int* counters;             // [0] tier-1 candidates, [1] tier-2 candidates, [2] FP16-tier survivors,
                               // [3] FP64 scorer blocks done (its last block makes the final selection)
    int* seg_state;
    int* seg_start;
    int* seg_cnt;
    int64_t* cand_rows;
    float* y32;
    // non-null: the FP32 value of candidate row r is y32_rows[r] (the first tier's
    // scores were the plain FP32 path's) and y32 is not read
    const float* y32_rows;
    int64_t* cand2_rows;
    double* y64;
    int* status_word;
    // top-N selection
    int top_n;                 // N (best / best_score are [n_kernels][N])
    int* pos64;                // per FP32 candidate: its position in the FP64 list, or -1
    double* seg_thr;           // per kernel: the FP32 window bound
    // FP16 middle tier (select_mid / topn_mid): y16[i] scores cand_rows[i];
    // survivors go to cand_mid_rows, counted by counters[2]
    float eps16;
    const float* y16;
    int64_t* cand_mid_rows;
};
cudaError_t launch_select_tier1(const SelectArgs& a, cudaStream_t s, int block = 256);
cudaError_t launch_topn_tier1(const SelectArgs& a, cudaStream_t s, int block = 256);
cudaError_t launch_topn_tier2(const SelectArgs& a, cudaStream_t s, int block = 256);
cudaError_t launch_topn_final(const SelectArgs& a, cudaStream_t s, int block = 256);
cudaError_t launch_select_tier2(const SelectArgs& a, cudaStream_t s, int block = 256);
cudaError_t launch_select_mid(const SelectArgs& a, cudaStream_t s, int block = 256);
cudaError_t launch_topn_mid(const SelectArgs& a, cudaStream_t s, int block = 256);

// Variant generation (enumerate.cu).
int64_t variant_count(int64_t depth);
cudaError_t launch_enumerate(const advisor_variant_desc* kernels, int64_t K, advisor_variant_desc* out,
                             int64_t capacity, int64_t* seg_off, int64_t* total, int num_sms, cudaStream_t s);

}  // namespace adv
