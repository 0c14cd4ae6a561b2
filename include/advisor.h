/*
 * advisor.h -- C ABI of the GB300 (sm_103a) cost-model hot path of the
 * OpenMP Advisor method (arXiv 2301.03636).
 *
 * The method (Sec. 3, Fig. 2): every kernel of a program has a set of
 * generated offload variants (Sec. 4.1.3); a trained cost model predicts the
 * runtime of every variant from its features (Sec. 4.2), and the variants of
 * each kernel are sorted by predicted cost so that the best can be selected.
 * This library computes, on one GPU:
 *
 *   descriptor -> validation -> integer features -> z-score standardisation
 *   -> MLP regression (predicted ln runtime) -> per-kernel argmin,
 *
 * and trains the MLP from measured (here: synthetic) runtimes (training mode).
 *
 * Conventions for every entry point:
 *  - Memory: every device buffer belongs to the caller.  The library never
 *    allocates or frees device memory; sizes of the model's parameter block
 *    and of the scratch workspace are reported by advisor_model_param_bytes
 *    and advisor_workspace_bytes.  The model object holds host metadata only.
 *  - Pointers prefixed d_ are device pointers, h_ host pointers.  Device
 *    buffers must be 256-byte aligned (cudaMalloc and torch allocations are).
 *  - Asynchrony: calls enqueue kernels on `stream` and return without
 *    synchronising, except the few whose description says they synchronise
 *    (advisor_get_device_status, advisor_get_rescore_counts[_ex], plan
 *    creation, advisor_measure_fp32_fma_peak).
 *  - Errors: argument errors are returned immediately and nothing is
 *    enqueued.  Per-row descriptor errors are reported in d_row_status.
 *    Errors found on the device (malformed segment offsets, a wait that ran
 *    out of time) set a sticky status word read by advisor_get_device_status.
 *    A failed CUDA launch returns ADVISOR_ERR_CUDA.
 *  - Threading: a model object may be used from one host thread at a time.
 */
#ifndef ADVISOR_H
#define ADVISOR_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ADVISOR_OK = 0,
    ADVISOR_ERR_INVALID_ARGUMENT = 1,
    ADVISOR_ERR_BAD_DESCRIPTOR = 2,   /* device status: a descriptor failed validation */
    ADVISOR_ERR_OUT_OF_MEMORY = 3,    /* workspace or parameter block too small */
    ADVISOR_ERR_CUDA = 4,
    ADVISOR_ERR_TIMEOUT = 5,          /* device status: a bounded wait gave up */
    ADVISOR_ERR_UNSUPPORTED = 6,      /* shape or precision the library does not run */
    ADVISOR_ERR_BAD_SEGMENTS = 7      /* device status: segment offsets not monotone / out of range */
} advisor_status;

/* Arithmetic of the MLP scorer.  FP32: SIMT FP32 FMA ("plain" path).
 * BF16 / FP16: tcgen05 tensor cores, 16-bit operands, FP32 accumulation in
 * tensor memory, FP32 bias/ReLU epilogue, output layer in FP32.
 * FP64: SIMT FP64 with the oracle's summation order (slow; used for the
 * near-tie re-score and for error calibration).  FP8_E4M3: tensor cores
 * with E4M3 operands and per-tensor scales (kind::f8f6f4), FP32
 * accumulation and epilogue; models with a hidden width above 256 only,
 * after advisor_model_calibrate_fp8. */
typedef enum {
    ADVISOR_FP32 = 0,
    ADVISOR_BF16 = 1,
    ADVISOR_FP16 = 2,
    ADVISOR_FP64 = 3,
    ADVISOR_FP8_E4M3 = 4
} advisor_precision;

/* One generated variant of one kernel: 16 x int64 = 128 bytes, array of
 * structures, row-major.  Fields follow the per-kernel information of
 * Sec. 4.1.1 (loop nest), the data classes of Sec. 4.1.2 (mapped bytes) and
 * the five variant parameters of Sec. 4.1.3.  Valid ranges (a row outside
 * them gets a nonzero status bit and is never selected):
 *   depth 1..4; trip[i] in 1..2^24 for i < depth, trip[i] == 1 otherwise;
 *   flops_per_iter, bytes_per_iter in 1..2^32; h2d_bytes, d2h_bytes in 0..2^48;
 *   teams, threads in 1..2^24; pf_pos in 0..depth-1; dist_collapse == 0 if
 *   pf_pos == 0 else 1..pf_pos; pf_collapse in 1..depth-pf_pos; schedule 0..2;
 *   data_mode 0..1; trip product <= 2^48, trip product * flops_per_iter and
 *   trip product * bytes_per_iter <= 2^62. */
typedef struct {
    int64_t depth;          /* number of nested for loops (NUM, Sec. 4.1.3) */
    int64_t trip[4];        /* trip count of loop levels 0..3 */
    int64_t flops_per_iter; /* operations in the loop body */
    int64_t bytes_per_iter; /* bytes touched by the loop body */
    int64_t h2d_bytes;      /* mapped to the device (alloc/to/tofrom, Sec. 4.1.2) */
    int64_t d2h_bytes;      /* mapped back to the host (from/tofrom) */
    int64_t teams;
    int64_t threads;
    int64_t pf_pos;         /* loop x carrying 'parallel for' (0: combined with distribute) */
    int64_t dist_collapse;  /* collapse of 'teams distribute' */
    int64_t pf_collapse;    /* collapse of 'parallel for' */
    int64_t schedule;       /* 0 static, 1 dynamic, 2 guided */
    int64_t data_mode;      /* the two-valued data-transfer parameter */
} advisor_variant_desc;

/* Row status bits written by the extraction kernels (0 = valid). */
#define ADVISOR_ROW_BAD_DEPTH       0x01u
#define ADVISOR_ROW_BAD_TRIP        0x02u
#define ADVISOR_ROW_BAD_WORK        0x04u
#define ADVISOR_ROW_BAD_MAPPED      0x08u
#define ADVISOR_ROW_BAD_PARALLELISM 0x10u
#define ADVISOR_ROW_BAD_VARIANT     0x20u
#define ADVISOR_ROW_BAD_RANGE       0x40u

typedef struct advisor_model* advisor_model_t;

/* Text of a status code (static storage). */
const char* advisor_status_string(advisor_status s);

/* ---- model object -------------------------------------------------------- */

/* Create the host object of an MLP with layer widths widths[0..n_widths-1]
 * (Sec. 5, Exp. 3: fully connected, ReLU hidden layers, one output neuron).
 * widths[0] = number of features F (32, 33, 64 or 128), widths[n_widths-1]
 * must be 1, 3 <= n_widths <= 8, hidden widths 1..1024 (any width: the
 * tensor-core images pad to multiples of 64 with zero weights).  Hidden widths
 * up to 256 run in the fused tensor-core scorer, wider ones layer by layer. */
advisor_status advisor_model_create(const int32_t* h_widths, int32_t n_widths, advisor_model_t* out);
advisor_status advisor_model_destroy(advisor_model_t m);

/* Bytes of the caller-allocated device parameter block: FP32 master weights,
 * their packed 16-bit tensor-core copies, standardisation constants and the
 * Adam moments. */
size_t advisor_model_param_bytes(advisor_model_t m);

/* Bytes of the caller-allocated scratch workspace for calls of up to max_rows
 * rows and max_kernels kernels (16-bit activations of the tensor-core path,
 * candidate lists of the near-tie re-score, training activations). */
size_t advisor_workspace_bytes(advisor_model_t m, int64_t max_rows, int64_t max_kernels);

/* Attach the device parameter block and workspace (sizes as reported above,
 * 256-byte aligned).  Must precede set_params.  May be called again to move
 * the workspace (e.g. a larger one). */
advisor_status advisor_model_bind(advisor_model_t m, void* d_params, size_t param_bytes,
                                  void* d_workspace, size_t workspace_bytes,
                                  int64_t max_rows, int64_t max_kernels);

/* Load parameters.  d_params_fp32: the FP32 master parameters, per layer
 * W[out][in] row-major followed by b[out].  d_mu, d_sigma: the z-score
 * standardisation of the features (Sec. 5, Exp. 3): z = (feature/65536 - mu)
 * / sigma, FP64, F entries each, sigma > 0.  Packs the 16-bit copies and
 * resets the Adam state. */
advisor_status advisor_model_set_params(advisor_model_t m, const float* d_params_fp32,
                                        const double* d_mu, const double* d_sigma,
                                        cudaStream_t stream);

/* Copy the FP32 master parameters out (d_params_fp32, same layout). */
advisor_status advisor_model_get_params(advisor_model_t m, float* d_params_fp32, cudaStream_t stream);

/* Number of FP32 master parameters. */
int64_t advisor_model_param_count(advisor_model_t m);

/* Fit the standardisation on a calibration sample: mean and population
 * standard deviation of feature/65536 over the valid rows (sigma 0 -> 1).
 * d_feat_q16 [n_rows][F], d_row_status nullable.  Writes F doubles each. */
advisor_status advisor_fit_standardizer(const int32_t* d_feat_q16, const uint8_t* d_row_status,
                                        int64_t n_rows, int32_t n_features, double* d_mu,
                                        double* d_sigma, cudaStream_t stream);

/* ---- hot path ----------------------------------------------------------- */

/* a1-a2: validate descriptors and extract the F integer features of each
 * (Fig. 2 "Feature Extraction"), bit-exact.  Features are Q16.16 fixed point:
 * binary logarithms of counts, bytes and their products (digit-by-digit
 * base-2 logarithm by repeated squaring), signed differences of those,
 * one-hot and small-integer variant parameters.  d_feat_q16 [n_rows][F]
 * row-major int32; invalid rows get all-zero features.  d_row_status [n_rows]
 * (nullable) receives the ADVISOR_ROW_* bits.  F in {32, 33, 64, 128}: 32
 * base features; 33 = the base features and the number of collapsed loops
 * (dist_collapse + pf_collapse), the input width of the paper's network
 * (Sec. 5 Exp. 3, whose 33 features the paper does not list); 64 adds eight
 * features per loop level; 128 adds 64 signed differences of base features. */
advisor_status advisor_extract_features(const advisor_variant_desc* d_desc, int64_t n_rows,
                                        int32_t n_features, int32_t* d_feat_q16,
                                        uint8_t* d_row_status, cudaStream_t stream);

/* a3-a5: predicted ln runtime of every row (Fig. 2 "Predicted Runtime").
 * d_feat_q16 [n_rows][F]; d_row_status nullable (rows with nonzero status
 * score +inf); d_scores [n_rows] FP32.  precision as advisor_precision; the
 * 16-bit precisions use the workspace. */
advisor_status advisor_score_variants(advisor_model_t m, const int32_t* d_feat_q16,
                                      const uint8_t* d_row_status, int64_t n_rows,
                                      advisor_precision precision, float* d_scores,
                                      cudaStream_t stream);

/* FP64 scores of every row (d_scores [n_rows] double), each dot product
 * summed sequentially over the input index with separately rounded products
 * and sums: the FP64 reference value of the regression of Sec. 4.2.  Slow
 * (FP64 SIMT); used to measure the error bounds of the other precisions. */
advisor_status advisor_score_variants_fp64(advisor_model_t m, const int32_t* d_feat_q16,
                                           const uint8_t* d_row_status, int64_t n_rows,
                                           double* d_scores, cudaStream_t stream);

/* Variant generation (Sec. 4.1.3; the counts are Table 1): every offload
 * variant of each kernel's loop nest.  A kernel is given as a descriptor
 * whose loop-nest and work fields (depth .. threads) are used and whose
 * variant fields are ignored.  For NUM = depth collapsible loops the variants
 * are all combinations of x = the loop of 'parallel for' (0..NUM-1), the
 * 'teams distribute' collapse (0 = combined when x = 0, else 1..x), the
 * 'parallel for' collapse (1..NUM-x), the schedule (0..2) and the data mode
 * (0..1), in that order with the data mode fastest: 6, 18, 42, 84 variants
 * for NUM = 1..4, none for any other depth.  Output: d_variants (device,
 * capacity rows; rows beyond the capacity are not written), d_seg_off
 * [n_kernels + 1] (device int64: kernel k owns rows d_seg_off[k] ..
 * d_seg_off[k+1]-1, the layout advisor_rank takes) and d_total (device
 * int64, nullable: the full count, which may exceed the capacity).
 * Asynchronous on `stream`. */
int64_t advisor_variant_count(int64_t depth);
advisor_status advisor_enumerate_variants(const advisor_variant_desc* d_kernels, int64_t n_kernels,
                                          advisor_variant_desc* d_variants, int64_t capacity,
                                          int64_t* d_seg_off, int64_t* d_total, cudaStream_t stream);

/* a6-a7: per-kernel selection (Fig. 2 "sort codes based on cost and select").
 * Kernel k owns rows d_seg_off[k] .. d_seg_off[k+1]-1 (int64, non-decreasing,
 * d_seg_off[0] >= 0, last <= n_rows).  d_best_local[k] = index of the selected
 * row within kernel k (0-based), -1 if the kernel has no finite score;
 * d_best_score[k] its predicted ln runtime.  Ties go to the lowest index.
 * With d_feat_q16 == NULL the selection is the argmin of d_scores.  With
 * features, rows whose score is within 2*eps_scores of their kernel's minimum
 * are re-scored in FP32, and rows still within 2*eps_fp32 of the FP32 minimum
 * are re-scored in FP64 with the oracle's summation order, so that the
 * selection equals the FP64 argmin whenever |score - fp64| <= eps_scores and
 * |fp32 - fp64| <= eps_fp32 hold.  d_best_score then holds the value of the
 * last tier that decided the kernel. */
advisor_status advisor_select_best(advisor_model_t m, const float* d_scores, int64_t n_rows,
                                   const int64_t* d_seg_off, int64_t n_kernels,
                                   const int32_t* d_feat_q16, float eps_scores, float eps_fp32,
                                   int32_t* d_best_local, double* d_best_score,
                                   cudaStream_t stream);

/* a1-a7 in one call: descriptors -> features -> scores -> selection, the
 * features of the tensor-core path going straight to 16-bit standardised
 * activations.  d_scores and d_row_status are optional outputs (nullable).
 * Near-tie re-score as in advisor_select_best (recomputes the features of the
 * candidate rows from their descriptors); eps_scores < 0 disables it.
 * d_desc may also point to page-locked host memory (cudaHostAlloc /
 * cudaHostRegister, accessible from the device through unified addressing):
 * the kernels then read the descriptors over the CPU-GPU link while they
 * compute, instead of the caller copying them first; the host must not
 * change them until the call has completed on `stream`.  d_seg_off,
 * d_best_local and d_best_score may likewise be page-locked host memory: the
 * kernels read the offsets and write the answers there directly, and the host
 * reads the answers once the call has completed on `stream` (a serving batch
 * then needs no copy around the call).  Any of these pointers that the device
 * cannot access (e.g. pageable host memory) returns
 * ADVISOR_ERR_INVALID_ARGUMENT. */
advisor_status advisor_rank(advisor_model_t m, const advisor_variant_desc* d_desc, int64_t n_rows,
                            const int64_t* d_seg_off, int64_t n_kernels,
                            advisor_precision precision, float eps_scores, float eps_fp32,
                            int32_t* d_best_local, double* d_best_score, float* d_scores,
                            uint8_t* d_row_status, cudaStream_t stream);

/* advisor_rank with the descriptors in page-locked host memory (h_desc,
 * cudaHostAlloc / cudaHostRegister) and a caller-owned device buffer d_desc
 * of n_rows descriptors that receives them: the copy runs in n_stages chunks
 * of whole 128-row tiles (1 <= n_stages <= ADVISOR_MAX_STAGES) on a stream of
 * the model's own, and each chunk is extracted and scored on `stream` as soon
 * as it has arrived, so that the copies overlap the scoring; the selection
 * follows once every chunk is scored.  Same results as advisor_rank on
 * d_desc.  The host must not change h_desc until the call has completed on
 * `stream`.  Errors: those of advisor_rank; ADVISOR_ERR_INVALID_ARGUMENT for
 * an h_desc that is not page-locked host memory or n_stages out of range. */
#define ADVISOR_MAX_STAGES 16
advisor_status advisor_rank_staged(advisor_model_t m, const advisor_variant_desc* h_desc,
                                   advisor_variant_desc* d_desc, int64_t n_rows, const int64_t* d_seg_off,
                                   int64_t n_kernels, advisor_precision precision, float eps_scores,
                                   float eps_fp32, int32_t* d_best_local, double* d_best_score, float* d_scores,
                                   uint8_t* d_row_status, int32_t n_stages, cudaStream_t stream);

/* advisor_rank_staged with the FP16 tensor-core tier of advisor_rank_ex
 * (eps_fp16 >= 0; same argument rules as advisor_rank_ex). */
advisor_status advisor_rank_staged_ex(advisor_model_t m, const advisor_variant_desc* h_desc,
                                      advisor_variant_desc* d_desc, int64_t n_rows, const int64_t* d_seg_off,
                                      int64_t n_kernels, advisor_precision precision, float eps_scores,
                                      float eps_fp16, float eps_fp32, int32_t* d_best_local, double* d_best_score,
                                      float* d_scores, uint8_t* d_row_status, int32_t n_stages,
                                      cudaStream_t stream);

/* advisor_rank with an FP16 tensor-core tier between the first scores and
 * the FP32 re-score (a7 of Fig. 2's selection, made cheaper for wide models
 * and coarse first tiers).  eps_fp16 >= 0 enables it: the tier-1 candidates
 * are re-extracted from their descriptors into a compact FP16 image, scored
 * on the tensor cores, and only those within 2*eps_fp16 of their kernel's
 * FP16 minimum (and any whose FP16 value is not finite) go on to FP32.  The
 * selection equals the FP64 argmin whenever |score - fp64| <= eps_scores,
 * |fp16 - fp64| <= eps_fp16 and |fp32 - fp64| <= eps_fp32 hold.  Needs
 * eps_scores >= 0 (else ADVISOR_ERR_INVALID_ARGUMENT), a 16-bit or E4M3
 * first tier and a model the tensor-core scorers run (else
 * ADVISOR_ERR_UNSUPPORTED).  eps_fp16 < 0: identical to advisor_rank. */
advisor_status advisor_rank_ex(advisor_model_t m, const advisor_variant_desc* d_desc, int64_t n_rows,
                               const int64_t* d_seg_off, int64_t n_kernels, advisor_precision precision,
                               float eps_scores, float eps_fp16, float eps_fp32, int32_t* d_best_local,
                               double* d_best_score, float* d_scores, uint8_t* d_row_status,
                               cudaStream_t stream);

/* FP8 (E4M3) operands for models whose hidden layers run one launch per
 * layer (a hidden width above 256): per-tensor scales, scale = amax / 448.
 * Weight scales come from the exact amax of each weight matrix (computed by
 * set_params / repack); activation scales are static, from the amax of each
 * hidden layer's input over a calibration sample: this call runs the FP32
 * forward on d_feat_q16 [n_rows][F] (n_rows <= the bound max_rows; the
 * standardised features for the first layer, the ReLU outputs for the
 * others) and stores the scales with the model.  set_params clears them;
 * ADVISOR_FP8_E4M3 scoring before this call returns
 * ADVISOR_ERR_INVALID_ARGUMENT.  Models that fit the fused 16-bit scorer
 * (every hidden width <= 256) return ADVISOR_ERR_UNSUPPORTED. */
advisor_status advisor_model_calibrate_fp8(advisor_model_t m, const int32_t* d_feat_q16, int64_t n_rows,
                                           cudaStream_t stream);

/* Launch shapes of the hot path (the batching of many kernels' variants
 * into persistent launches).  Every setting but layer_path gives
 * bit-identical results: rows, tiles and segments run the same per-row /
 * per-segment code whatever the grid or block, and no summation order
 * depends on them. */
typedef struct {
    int32_t extract_block;      /* threads per block of the extraction kernel: 64, 128 or 256 */
    int32_t tc_ctas;            /* CTAs of the persistent tensor-core scorer (at most one per SM; 0 = one per SM) */
    int32_t list_blocks_per_sm; /* FP32 near-tie scorer: persistent 16-row blocks per SM, 1 or 2 */
    int32_t list_chunk_kb;      /* FP32 near-tie scorer: weight chunk per bulk copy, 16 or 32 (KB) */
    int32_t select_block;       /* threads per block of the selection kernels (a warp per kernel): 128 or 256 */
    int32_t layer_path;         /* 1: score models that fit the fused tensor-core kernel (hidden widths <= 256)
                                   with one launch per layer instead (0 or 1); the two paths agree within the
                                   16-bit error bound (different accumulation order), not bit for bit */
} advisor_launch_config;

/* The model's launch shapes (defaults 128, 0, 1, 32, 256, 0), used by every
 * later call.  set returns ADVISOR_ERR_INVALID_ARGUMENT for a value outside
 * the lists above and leaves the configuration unchanged. */
advisor_status advisor_model_get_launch_config(advisor_model_t m, advisor_launch_config* out);
advisor_status advisor_model_set_launch_config(advisor_model_t m, const advisor_launch_config* cfg);

/* Batching under a CUDA graph: advisor_rank with these arguments, captured
 * once into a graph ("plan") that later calls replay with one launch.  The
 * plan binds every pointer as given: a replay reads the current contents of
 * d_desc and d_seg_off (same n_rows and n_kernels) and writes the same
 * outputs, so a caller refills the input buffers in place between replays.
 * autotune != 0: first time each launch configuration of a small candidate
 * set (one setting at a time, in path order; each candidate captured and
 * replayed on `stream`, which runs the path and overwrites the outputs) and
 * capture the fastest; autotune == 0 captures the model's current
 * configuration.  Either way the model's own configuration is left as it
 * was.  Creating a plan synchronises `stream`; capture happens on a private
 * stream.  The model must stay alive, bound to the same buffers, while the
 * plan exists; profile events set on the model are recorded by every
 * replay.  Errors: those of advisor_rank, and ADVISOR_ERR_CUDA when the
 * capture or instantiation fails. */
typedef struct advisor_plan* advisor_plan_t;
advisor_status advisor_plan_rank(advisor_model_t m, const advisor_variant_desc* d_desc, int64_t n_rows,
                                 const int64_t* d_seg_off, int64_t n_kernels, advisor_precision precision,
                                 float eps_scores, float eps_fp32, int32_t* d_best_local,
                                 double* d_best_score, float* d_scores, uint8_t* d_row_status,
                                 int32_t autotune, cudaStream_t stream, advisor_plan_t* out);

/* advisor_plan_rank for advisor_rank_staged: the plan replays the staged
 * copy of h_desc into d_desc together with the ranking (refill h_desc in
 * place between replays). */
advisor_status advisor_plan_rank_staged(advisor_model_t m, const advisor_variant_desc* h_desc,
                                        advisor_variant_desc* d_desc, int64_t n_rows, const int64_t* d_seg_off,
                                        int64_t n_kernels, advisor_precision precision, float eps_scores,
                                        float eps_fp32, int32_t* d_best_local, double* d_best_score,
                                        float* d_scores, uint8_t* d_row_status, int32_t n_stages,
                                        int32_t autotune, cudaStream_t stream, advisor_plan_t* out);

/* advisor_plan_rank / advisor_plan_rank_staged with the FP16 tensor-core
 * tier of advisor_rank_ex captured into the plan (eps_fp16 >= 0; same
 * argument rules as advisor_rank_ex).  Replays give the same selections as
 * advisor_rank_ex with these arguments. */
advisor_status advisor_plan_rank_ex(advisor_model_t m, const advisor_variant_desc* d_desc, int64_t n_rows,
                                    const int64_t* d_seg_off, int64_t n_kernels, advisor_precision precision,
                                    float eps_scores, float eps_fp16, float eps_fp32, int32_t* d_best_local,
                                    double* d_best_score, float* d_scores, uint8_t* d_row_status, int32_t autotune,
                                    cudaStream_t stream, advisor_plan_t* out);
advisor_status advisor_plan_rank_staged_ex(advisor_model_t m, const advisor_variant_desc* h_desc,
                                           advisor_variant_desc* d_desc, int64_t n_rows, const int64_t* d_seg_off,
                                           int64_t n_kernels, advisor_precision precision, float eps_scores,
                                           float eps_fp16, float eps_fp32, int32_t* d_best_local,
                                           double* d_best_score, float* d_scores, uint8_t* d_row_status,
                                           int32_t n_stages, int32_t autotune, cudaStream_t stream,
                                           advisor_plan_t* out);

/* Replay the plan on `stream` (asynchronous: one graph launch). */
advisor_status advisor_plan_launch(advisor_plan_t p, cudaStream_t stream);

/* The configuration the plan was captured with; *replay_us (nullable) the
 * median replay time the autotuner measured for it (0 without autotuning);
 * *kernels_per_replay (nullable) the kernel nodes in the graph. */
advisor_status advisor_plan_info(advisor_plan_t p, advisor_launch_config* cfg, float* replay_us,
                                 int32_t* kernels_per_replay);

/* Release the graph (NULL is a no-op). */
advisor_status advisor_plan_destroy(advisor_plan_t p);

/* Top N per kernel (Fig. 2: "sort codes based on cost and select top N"):
 * advisor_rank with d_best_local / d_best_score of shape [n_kernels][top_n]
 * (row-major): entry t of kernel k is the local index and score of the
 * kernel's (t+1)-th best variant, ties to the lower index; -1 / +inf where the
 * kernel has fewer finite scores.  With eps_scores >= 0 the list equals the
 * FP64 ordering whenever |score - fp64| <= eps_scores and |fp32 - fp64| <=
 * eps_fp32: rows within 2*eps_scores of the N-th score are re-scored in FP32,
 * and those within 2*eps_fp32 of another one near the N-th FP32 value in
 * FP64; d_best_score then holds the deciding value of each entry.
 * 1 <= top_n <= ADVISOR_MAX_TOP_N. */
#define ADVISOR_MAX_TOP_N 128
advisor_status advisor_rank_topn(advisor_model_t m, const advisor_variant_desc* d_desc, int64_t n_rows,
                                 const int64_t* d_seg_off, int64_t n_kernels, int32_t top_n,
                                 advisor_precision precision, float eps_scores, float eps_fp32,
                                 int32_t* d_best_local, double* d_best_score, float* d_scores,
                                 uint8_t* d_row_status, cudaStream_t stream);

/* advisor_rank_topn with the FP16 middle tier of advisor_rank_ex: t16 = the
 * N-th smallest finite FP16 value among a kernel's tier-1 candidates (+inf
 * if fewer than N are finite); candidates above t16 + 2*eps_fp16 are dropped
 * before the FP32 tier.  Same argument rules as advisor_rank_ex. */
advisor_status advisor_rank_topn_ex(advisor_model_t m, const advisor_variant_desc* d_desc, int64_t n_rows,
                                    const int64_t* d_seg_off, int64_t n_kernels, int32_t top_n,
                                    advisor_precision precision, float eps_scores, float eps_fp16,
                                    float eps_fp32, int32_t* d_best_local, double* d_best_score,
                                    float* d_scores, uint8_t* d_row_status, cudaStream_t stream);

/* a8: one training step (Sec. 3 training mode; Sec. 5 Exp. 3): forward,
 * loss = 0.5 * mean (y - label)^2 over the n_rows rows (labels: ln runtime),
 * hand-written backward, Adam update of the FP32 master weights; the derived
 * inference copies are marked stale and rebuilt by the next scoring call or
 * plan replay (advisor_model_refresh).  precision ADVISOR_FP32 (SIMT) or
 * ADVISOR_BF16 / ADVISOR_FP16 (16-bit operands for the forward/backward
 * GEMMs, FP32 accumulation and master weights).  h_adam = {lr, beta1, beta2,
 * eps, weight_decay} (host floats, copied at call time).  d_loss (nullable)
 * receives the loss (FP32) of the forward pass before the update.  Needs
 * n_rows <= the max_rows the workspace was bound with. */
advisor_status advisor_train_step(advisor_model_t m, const int32_t* d_feat_q16, const float* d_labels,
                                  int64_t n_rows, advisor_precision precision, const float* h_adam,
                                  float* d_loss, cudaStream_t stream);

/* A training step with a choice of optimizer and loss (Sec. 5 Exp. 3 trains
 * with RMSprop and the RMSE loss): optimizer ADVISOR_OPT_ADAM (lr, beta1,
 * beta2, eps, decoupled weight_decay: the update of advisor_train_step) or
 * ADVISOR_OPT_RMSPROP (g' = g + weight_decay w; v = alpha v + (1 - alpha)
 * g'^2; w -= lr g' / (sqrt(v) + eps), v kept with the model); loss
 * ADVISOR_LOSS_MSE (0.5 mean (y - t)^2) or ADVISOR_LOSS_RMSE (sqrt(mean
 * (y - t)^2)).  d_loss (nullable) receives the loss before the update.
 * Precisions as advisor_train_step. */
#define ADVISOR_OPT_ADAM 0
#define ADVISOR_OPT_RMSPROP 1
#define ADVISOR_LOSS_MSE 0
#define ADVISOR_LOSS_RMSE 1
typedef struct {
    int32_t optimizer;
    int32_t loss;
    float lr, beta1, beta2, alpha, eps, weight_decay;
} advisor_train_options;
advisor_status advisor_train_step_ex(advisor_model_t m, const int32_t* d_feat_q16, const float* d_labels,
                                     int64_t n_rows, advisor_precision precision, const advisor_train_options* opt,
                                     float* d_loss, cudaStream_t stream);

/* Gradient only (no update): d_grad [param_count] FP32 of the same loss,
 * same layout as the master parameters.  For gradient checks. */
advisor_status advisor_loss_grad(advisor_model_t m, const int32_t* d_feat_q16, const float* d_labels,
                                 int64_t n_rows, advisor_precision precision, float* d_grad,
                                 float* d_loss, cudaStream_t stream);

/* Forward pass for training (Sec. 3 training mode), keeping every layer's
 * output in the workspace for advisor_backward.  d_y [n_rows] (nullable)
 * receives the predictions.  precision ADVISOR_FP32. */
advisor_status advisor_forward_saved(advisor_model_t m, const int32_t* d_feat_q16, int64_t n_rows,
                                     advisor_precision precision, float* d_y, cudaStream_t stream);

/* Hand-written backward of the last advisor_forward_saved (same n_rows):
 * from d_dy = dL/dy [n_rows] to the parameter gradient d_grad [param_count]
 * (layout of the master parameters).  ReLU derivative 1 for positive
 * pre-activations, 0 otherwise. */
advisor_status advisor_backward(advisor_model_t m, const float* d_dy, int64_t n_rows, float* d_grad,
                                cudaStream_t stream);

/* Rebuild the derived copies (16-bit tensor-core images, transposed copy,
 * padded biases) after the FP32 master parameters were changed in place. */
advisor_status advisor_model_repack(advisor_model_t m, cudaStream_t stream);

/* The training steps update the FP32 masters only and mark the derived
 * copies stale; every scoring call (and every plan replay) rebuilds them
 * first when they are.  This call does that rebuild now, on `stream`, and is
 * a no-op when nothing changed. */
advisor_status advisor_model_refresh(advisor_model_t m, cudaStream_t stream);

/* Byte offset of the FP32 master parameters inside the parameter block (so
 * that a caller can view them as a tensor, e.g. for an external optimizer). */
size_t advisor_model_master_offset(advisor_model_t m);

/* Adam step counter of the model (checkpoint / resume; the moments live in
 * the parameter block). */
int64_t advisor_model_get_adam_step(advisor_model_t m);
advisor_status advisor_model_set_adam_step(advisor_model_t m, int64_t step);

/* Read and clear the model's sticky device status word (synchronises
 * `stream`).  Returns ADVISOR_OK, ADVISOR_ERR_TIMEOUT, ADVISOR_ERR_BAD_SEGMENTS
 * or ADVISOR_ERR_CUDA. */
advisor_status advisor_get_device_status(advisor_model_t m, cudaStream_t stream);

/* Near-tie statistics of the last selection with re-score on this model
 * (advisor_select_best / advisor_rank with eps_scores >= 0): h_counts[0] =
 * rows re-scored in FP32, h_counts[1] = rows re-scored in FP64 (host
 * int64[2]).  A ranking call with ADVISOR_FP32 scores and no FP16 tier takes
 * its candidates' FP32 values from its own first-tier scores instead of
 * re-scoring them (the plain FP32 scores, whose bound eps_fp32 is); [0] then
 * counts those candidates.  Synchronises `stream`.  Values are undefined
 * before the first such call. */
advisor_status advisor_get_rescore_counts(advisor_model_t m, int64_t* h_counts, cudaStream_t stream);

/* As advisor_get_rescore_counts with the FP16 middle tier (host int64[3]):
 * h_counts[0] = rows re-scored in FP16 (0 when the last selection ran
 * without that tier), [1] = rows re-scored in FP32, [2] = in FP64. */
advisor_status advisor_get_rescore_counts_ex(advisor_model_t m, int64_t* h_counts, cudaStream_t stream);

/* Tensor-core scoring that allocates nothing: the computation and result
 * of advisor_score_variants with ADVISOR_BF16 or ADVISOR_FP16 on the fused
 * scorer (this call always runs the fused tensor-core kernel, with the
 * model's tc_ctas, whatever layer_path the model's launch configuration
 * sets), for callers that cannot provide device memory for a workspace
 * (code where cudaMalloc is not allowed, e.g. host callbacks or hosts that
 * forbid device allocations after start-up).  The paper has no
 * counterpart: this is an interface convenience.  The 16-bit activation
 * image lives in a fixed device array inside the library: 16,384 rows of up
 * to 128 features (4 MiB on every GPU that loads the library, held until
 * exit); n_rows beyond 16,384 returns ADVISOR_ERR_OUT_OF_MEMORY before
 * anything is enqueued.  The model must be bound and loaded (set_params);
 * its workspace is not used.  The first call on a device looks up the
 * array's device address (once per device, with that device current, kept
 * for the life of the process: the library must not outlive a reset of the
 * device), so make that first call before any stream capture.  All calls on
 * a device share the array; each call rewrites every part it reads, but
 * calls whose kernels overlap on the GPU (e.g. on two streams) race and
 * must be ordered by the caller.  ADVISOR_FP32 / ADVISOR_FP64 return
 * ADVISOR_ERR_UNSUPPORTED. */
advisor_status advisor_score_variants_noalloc(advisor_model_t m, const int32_t* d_feat_q16,
                                              const uint8_t* d_row_status, int64_t n_rows,
                                              advisor_precision precision, float* d_scores,
                                              cudaStream_t stream);

/* Measurement hook: when ev_start / ev_stop (cudaEvent_t handles created by
 * the caller with timing enabled) are non-NULL, every later launch of the
 * tensor-core scorer by this model is bracketed by cudaEventRecord on the
 * call's stream, so that the caller can time that kernel alone inside a
 * longer sequence.  Pass NULL, NULL to stop. */
advisor_status advisor_model_set_profile_events(advisor_model_t m, void* ev_start, void* ev_stop);

/* Measurement only: the FP32 FMA rate of this GPU's CUDA cores in TFLOP/s
 * (2 FLOP per FMA), measured by a launch of independent FMA chains that
 * fills every SM (fastest of three timed launches after one warm-up), the
 * denominator of the FP32 scorer's roofline.  Synchronises `stream`. */
advisor_status advisor_measure_fp32_fma_peak(double* h_tflops, cudaStream_t stream);

/* Failure-detection self-test of the device-side bounded waits: launches one
 * thread that waits, with the bounded mbarrier wait every pipelined kernel of
 * the library uses, on a barrier nothing arrives at.  After timeout_ns
 * (1,000 .. 1,000,000,000 ns, else ADVISOR_ERR_INVALID_ARGUMENT) the wait
 * gives up, records the timeout in the model's status word and the kernel
 * returns, leaving no copy in flight and no tensor memory held: the next
 * advisor_get_device_status returns ADVISOR_ERR_TIMEOUT (and clears it), and
 * the model stays usable.  Asynchronous on `stream`. */
advisor_status advisor_model_check_wait_timeout(advisor_model_t m, int64_t timeout_ns, cudaStream_t stream);

/* Number of kernels this library launched since load (host-side counter of
 * successful launches; for launch accounting in benchmarks). */
int64_t advisor_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* ADVISOR_H */
