// Variant generation on the GPU (Sec. 4.1.3; the counts are Table 1).
//
// For a kernel whose loop nest has NUM = depth collapsible for loops, the
// generated offload variants are all combinations of the position x of the
// 'parallel for' directive (loop 0 .. NUM-1), the collapse of 'teams
// distribute' (absent when x = 0, where the two directives are combined,
// else 1..x), the collapse of 'parallel for' (1..NUM-x), the schedule
// (static, dynamic, guided) and the data-transfer mode (2 values):
// 6 * (NUM + sum_{x=1}^{NUM-1} x (NUM-x)) = 6, 18, 42, 84 for NUM = 1..4.
// Order within a kernel: x, then the distribute collapse, then the
// parallel-for collapse, then the schedule, then the data mode (fastest).
//
// Two launches: one block computes every kernel's count and the exclusive
// prefix sum (the segment offsets the ranking calls take); then one warp per
// kernel writes its variants, each lane decoding its variant index.
#include "common.cuh"

namespace adv {

// (x, dc, pc) of combination c of a depth-`depth` nest, in the order above.
__device__ __forceinline__ void decode_combo(int depth, int c, int& x, int& dc, int& pc) {
    for (x = 0; x < depth; ++x) {
        const int span = depth - x;                  // parallel-for collapse choices
        const int n_dc = x == 0 ? 1 : x;             // distribute collapse choices
        if (c < n_dc * span) break;
        c -= n_dc * span;
    }
    const int span = depth - x;
    dc = x == 0 ? 0 : 1 + c / span;
    pc = 1 + c % span;
}

__host__ __device__ __forceinline__ int64_t variants_of_depth(int64_t depth) {
    if (depth < 1 || depth > 4) return 0;
    // sum over x of (x == 0 ? 1 : x) * (depth - x) combinations, 6 variants each
    int64_t c = depth;
    for (int64_t x = 1; x < depth; ++x) c += x * (depth - x);
    return 6 * c;
}

__global__ void __launch_bounds__(1024) variant_offsets_kernel(const advisor_variant_desc* __restrict__ kernels,
                                                               int64_t K, int64_t* __restrict__ seg_off,
                                                               int64_t* __restrict__ total) {
    __shared__ int64_t warp_sum[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int64_t per = (K + 1023) / 1024;
    const int64_t k0 = t * per, k1 = k0 + per < K ? k0 + per : K;
    int64_t mine = 0;
    for (int64_t k = k0; k < k1; ++k) mine += variants_of_depth(kernels[k].depth);
    // exclusive scan of the per-thread sums over the block
    int64_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_sum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int64_t ws = warp_sum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t v = __shfl_up_sync(0xffffffffu, ws, o);
            if (lane >= o) ws += v;
        }
        warp_sum[lane] = ws;   // inclusive sums of the warps
    }
    __syncthreads();
    int64_t run = incl - mine + (w > 0 ? warp_sum[w - 1] : 0);
    for (int64_t k = k0; k < k1; ++k) {
        seg_off[k] = run;
        run += variants_of_depth(kernels[k].depth);
    }
    if (t == 1023) {
        seg_off[K] = run;   // thread 1023 owns the last (possibly empty) range
        if (total) *total = run;
    }
}

__global__ void emit_variants_kernel(const advisor_variant_desc* __restrict__ kernels, int64_t K,
                                     const int64_t* __restrict__ seg_off, advisor_variant_desc* __restrict__ out,
                                     int64_t capacity) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < K; k += warps) {
        const advisor_variant_desc kd = kernels[k];
        const int depth = (int)kd.depth;
        const int n = (int)variants_of_depth(kd.depth);
        const int64_t base = seg_off[k];
        for (int v = lane; v < n; v += 32) {
            if (base + v >= capacity) break;
            int x, dc, pc;
            decode_combo(depth, v / 6, x, dc, pc);
            advisor_variant_desc o = kd;
            o.pf_pos = x;
            o.dist_collapse = dc;
            o.pf_collapse = pc;
            o.schedule = (v % 6) / 2;
            o.data_mode = v % 2;
            out[base + v] = o;
        }
    }
}

int64_t variant_count(int64_t depth) { return variants_of_depth(depth); }

cudaError_t launch_enumerate(const advisor_variant_desc* kernels, int64_t K, advisor_variant_desc* out,
                             int64_t capacity, int64_t* seg_off, int64_t* total, int num_sms, cudaStream_t s) {
    variant_offsets_kernel<<<1, 1024, 0, s>>>(kernels, K, seg_off, total);
    const int64_t blocks = (K + 7) / 8;
    const int grid = (int)(blocks < 1 ? 1 : (blocks < 16 * num_sms ? blocks : 16 * num_sms));
    emit_variants_kernel<<<grid, 256, 0, s>>>(kernels, K, seg_off, out, capacity);
    adv_count_launch(2);
    return cudaGetLastError();
}

}  // namespace adv
