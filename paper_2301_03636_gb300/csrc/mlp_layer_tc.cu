// Per-layer tensor-core scorer for MLPs whose hidden layers are too wide for
// the fused kernel (a4-a5 of the large sweep, e.g. 128-1024-1024-1024-1),
// with 16-bit operands (BF16 / FP16, kind::f16) or E4M3 operands
// (kind::f8f6f4, per-tensor scales: H = ReLU(s_x s_w acc + b), re-quantised
// with the next layer's activation scale):
// each hidden layer is one persistent launch computing
//     H_out = ReLU(H_in W^T + b)        (Sec. 4.2 regression, Sec. 5 Exp. 3 network)
// with H_in / H_out in the same tiled 16-bit image the extraction kernel
// writes (128-row tiles of 64-column slabs, 128-byte rows, 128B swizzle), so
// a layer's output is the next layer's operand as it stands.  The last hidden
// layer does not store its activations: its epilogue multiplies them by the
// output row and leaves FP32 partial sums per 128-column half-chunk, which
// adv::launch_sum_partials adds in a fixed order (plus the output bias).
//
// Work item = (128-row tile, chunk of up to 256 output columns); items are
// dealt round-robin to one CTA per SM in tile-major order, so the CTAs that
// run at the same time share A tiles and the whole weight image through L2.
// 13 warps:
//   warps 0-3   producers: the K slabs of all items form one sequence consumed
//               through stages 0,1,2,3,0,...; producer q fills stage q (one
//               16 KB A slab + one B slab of up to 32 KB), because bulk copies
//               issued by one thread complete one after another;
//   warp 4      MMA issuer (one thread) and tensor-memory owner: two FP32
//               accumulators of 256 columns, used by alternate items, so one
//               item's epilogue overlaps the next item's MMAs;
//   warps 5-12  epilogue: two warps per TMEM lane quadrant (warp % 4), each
//               taking half of the item's columns.
// All waits are bounded by %globaltimer and report ADV_DEV_TIMEOUT.
#include "mlp.cuh"

namespace adv {

constexpr int LG_STAGES = 4;
constexpr int LG_BN = 256;
constexpr int LG_EPI_WARPS = 8;
constexpr int LG_THREADS = 32 * (LG_STAGES + 1 + LG_EPI_WARPS);
constexpr uint32_t LG_B_BYTES = LG_BN * ADV_SLAB_ROW_BYTES;                 // 32 KB
constexpr uint32_t LG_STAGE_BYTES = ADV_X_SLAB_BYTES + LG_B_BYTES;          // 48 KB

// KIND: 0 F16, 1 BF16 (kind::f16), 2 E4M3 (kind::f8f6f4).
template <int FMT>
__device__ __forceinline__ uint32_t lg_relu_pack(float lo, float hi) {
    uint32_t d;
    if constexpr (FMT == 1) asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    else asm("cvt.rn.relu.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

template <int KIND>
__global__ void __launch_bounds__(LG_THREADS, 1) mlp_layer_tc_kernel(const __grid_constant__ LayerArgs a) {
    constexpr int FMT = KIND == 1 ? 1 : 0;   // instruction-descriptor format code (E4M3 shares F16's 0)
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_addr(smem_raw);
    uint8_t* base = smem_raw + ((1024u - (raw_addr & 1023u)) & 1023u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + LG_STAGES * LG_STAGE_BYTES);
    uint64_t* full = bars;                          // [LG_STAGES]
    uint64_t* empty = bars + LG_STAGES;             // [LG_STAGES]
    uint64_t* acc_full = bars + 2 * LG_STAGES;      // [2]
    uint64_t* acc_empty = acc_full + 2;             // [2]
    uint64_t* drain = acc_empty + 2;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < LG_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&acc_full[s], 1);
            mbar_init(&acc_empty[s], LG_EPI_WARPS * 32);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == LG_STAGES) {
        tmem_alloc(tmem_holder, 2 * LG_BN);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    const int G = gridDim.x, b = blockIdx.x;
    int64_t live_tiles = a.n_tiles;
    if (a.n_rows_dev) {   // a gathered list whose length an earlier kernel wrote
        const int64_t c = *a.n_rows_dev;
        const int64_t t = c > 0 ? (c + ADV_TILE_M - 1) / ADV_TILE_M : 0;
        live_tiles = t < live_tiles ? t : live_tiles;
    }
    const int64_t n_items = live_tiles * a.n_chunks;
    const int n_my = n_items > b ? (int)((n_items - b + G - 1) / G) : 0;   // items b, b+G, b+2G, ...
    const uint64_t lim = a.timeout_ns;
    const int ks = a.a_slabs;

    if (warp < LG_STAGES) {
        // ---------------- producers ----------------
        const int q = warp;
        if (lane == 0) {
            uint32_t phase = 0;
            int64_t idx = 0;
            int mine = 0;
            bool ok = true;
            for (int i = 0; i < n_my && ok; ++i) {
                const int64_t item = b + (int64_t)i * G;
                const int tile = (int)(item / a.n_chunks), chunk = (int)(item % a.n_chunks);
                const int n0 = chunk * LG_BN;
                const int bn = a.npad - n0 < LG_BN ? a.npad - n0 : LG_BN;
                const uint32_t bbytes = (uint32_t)bn * ADV_SLAB_ROW_BYTES;
                for (int k = 0; k < ks; ++k, ++idx) {
                    if (idx % LG_STAGES != q) continue;
                    if (!mbar_wait_bounded(&empty[q], phase ^ 1u, a.status_word, abort_flag, lim)) {
                        ok = false;
                        break;
                    }
                    uint8_t* st = base + q * LG_STAGE_BYTES;
                    mbar_expect_tx(&full[q], ADV_X_SLAB_BYTES + bbytes);
                    bulk_g2s(st, a.a_img + ((size_t)tile * ks + k) * ADV_X_SLAB_BYTES, ADV_X_SLAB_BYTES, &full[q]);
                    bulk_g2s(st + ADV_X_SLAB_BYTES,
                             a.w_img + ((size_t)k * a.npad + n0) * ADV_SLAB_ROW_BYTES, bbytes, &full[q]);
                    ++mine;
                    phase ^= 1u;
                }
            }
            if (mine > 0) mbar_wait_bounded(&full[q], phase ^ 1u, a.status_word, abort_flag, lim);
        }
    } else if (warp == LG_STAGES) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            int64_t idx = 0;
            bool ok = true, any = false;
            for (int i = 0; i < n_my && ok; ++i) {
                const int64_t item = b + (int64_t)i * G;
                const int chunk = (int)(item % a.n_chunks);
                const int bn = a.npad - chunk * LG_BN < LG_BN ? a.npad - chunk * LG_BN : LG_BN;
                const uint32_t idesc = f16_idesc((uint32_t)FMT, 128u, (uint32_t)bn);
                const int ab = i & 1;
                const uint32_t use = (uint32_t)(i >> 1);
                if (!mbar_wait_bounded(&acc_empty[ab], (use & 1u) ^ 1u, a.status_word, abort_flag, lim)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(ab * LG_BN);
                for (int k = 0; k < ks; ++k, ++idx) {
                    const int stage = (int)(idx % LG_STAGES);
                    const uint32_t par = (uint32_t)((idx / LG_STAGES) & 1);
                    if (!mbar_wait_bounded(&full[stage], par, a.status_word, abort_flag, lim)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint8_t* st = base + stage * LG_STAGE_BYTES;
                    const uint64_t adesc = sw128_desc(smem_addr(st));
                    const uint64_t bdesc = sw128_desc(smem_addr(st + ADV_X_SLAB_BYTES));
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {   // 32 bytes of K per instruction
                        if constexpr (KIND == 2)
                            umma_f8f6f4(d_tmem, adesc + 2u * kk, bdesc + 2u * kk, idesc, (k | kk) != 0);
                        else
                            umma_f16(d_tmem, adesc + 2u * kk, bdesc + 2u * kk, idesc, (k | kk) != 0);
                    }
                    umma_commit(&empty[stage]);
                    any = true;
                }
                if (!ok) break;
                umma_commit(&acc_full[ab]);
            }
            if (any) {   // every issued MMA has completed before tensor memory is released
                umma_commit(drain);
                mbar_wait_bounded(drain, 0, a.status_word, abort_flag, lim);
            }
        }
    } else {
        // ---------------- epilogue ----------------
        const int e = warp - (LG_STAGES + 1);       // 0..7
        const int quad = warp & 3;                  // TMEM lane quadrant
        const int half = e >> 2;                    // column half of the item
        const uint32_t r = (uint32_t)(quad * 32 + lane);
        const int out_slabs = a.npad / (KIND == 2 ? ADV_SLAB_K8 : ADV_SLAB_K);
        float acc_scale = 1.f, out_inv = 1.f;   // E4M3: dequantise the accumulator, quantise the output
        if constexpr (KIND == 2) {
            const float w_amax = __uint_as_float(reinterpret_cast<const unsigned*>(a.fp8)[ADV_FP8_W_AMAX + a.layer]);
            acc_scale = __ldg(a.fp8 + ADV_FP8_X_SCALE + a.layer) * (w_amax > 0.f ? w_amax / ADV_E4M3_MAX : 1.f);
            if (a.mode == 0) out_inv = 1.f / __ldg(a.fp8 + ADV_FP8_X_SCALE + a.layer + 1);
        }
        for (int i = 0; i < n_my; ++i) {
            const int64_t item = b + (int64_t)i * G;
            const int tile = (int)(item / a.n_chunks), chunk = (int)(item % a.n_chunks);
            const int n0 = chunk * LG_BN;
            const int bn = a.npad - n0 < LG_BN ? a.npad - n0 : LG_BN;
            const int cw = bn >> 1;                 // this warp's columns [c_lo, c_lo + cw), cw % 16 == 0
            const int c_lo = half * cw;
            const int ab = i & 1;
            const uint32_t use = (uint32_t)(i >> 1);
            const bool got = mbar_wait_bounded(&acc_full[ab], use & 1u, a.status_word, abort_flag, lim);
            __syncwarp();   // tcgen05.ld / wait are warp-collective
            if (!got) break;
            tc_fence_after();
            const uint32_t t_base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(ab * LG_BN);
            float y = 0.f;
            for (int c0 = c_lo; c0 < c_lo + cw; c0 += 16) {
                uint32_t v[16];
                tmem_ld_32x32b_x16(t_base + (uint32_t)c0, v);
                float4 bq[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) bq[u] = __ldg(reinterpret_cast<const float4*>(a.bias + n0 + c0) + u);
                tmem_wait_ld();
                const float* bf = reinterpret_cast<const float*>(bq);
                if constexpr (KIND == 2) {
#pragma unroll
                    for (int u = 0; u < 16; ++u) v[u] = __float_as_uint(__uint_as_float(v[u]) * acc_scale);
                }
                if (KIND == 2 && a.mode == 0) {
                    const int c = n0 + c0;          // first output column of these 16: one 16-byte chunk
                    uint8_t* slab = a.out_img + ((size_t)tile * out_slabs + (c >> 7)) * ADV_X_SLAB_BYTES;
                    uint32_t pk[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        float z[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            z[e] = fmaxf(__uint_as_float(v[4 * t + e]) + bf[4 * t + e], 0.f) * out_inv;
                        pk[t] = e4m3x2(z[0], z[1]) | (e4m3x2(z[2], z[3]) << 16);
                    }
                    *reinterpret_cast<uint4*>(slab + sw128_offset(r, (uint32_t)((c & 127) >> 4))) =
                        make_uint4(pk[0], pk[1], pk[2], pk[3]);
                } else if (a.mode == 0) {
                    const int c = n0 + c0;          // first output column of these 16
                    uint8_t* slab = a.out_img + ((size_t)tile * out_slabs + (c >> 6)) * ADV_X_SLAB_BYTES;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        uint32_t pk[4];
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            const int cc = 8 * h + 2 * t;
                            pk[t] = lg_relu_pack<FMT>(__uint_as_float(v[cc]) + bf[cc],
                                                      __uint_as_float(v[cc + 1]) + bf[cc + 1]);
                        }
                        const uint32_t ch = (uint32_t)(((c & 63) >> 3) + h);
                        *reinterpret_cast<uint4*>(slab + sw128_offset(r, ch)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    }
                } else {
                    const float4* w4 = reinterpret_cast<const float4*>(a.w_out + n0 + c0);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float4 wq = __ldg(w4 + u);
                        y = fmaf(fmaxf(__uint_as_float(v[4 * u + 0]) + bf[4 * u + 0], 0.f), wq.x, y);
                        y = fmaf(fmaxf(__uint_as_float(v[4 * u + 1]) + bf[4 * u + 1], 0.f), wq.y, y);
                        y = fmaf(fmaxf(__uint_as_float(v[4 * u + 2]) + bf[4 * u + 2], 0.f), wq.z, y);
                        y = fmaf(fmaxf(__uint_as_float(v[4 * u + 3]) + bf[4 * u + 3], 0.f), wq.w, y);
                    }
                }
            }
            if (a.mode == 1)
                a.partial[((size_t)chunk * 2 + half) * ((size_t)a.n_tiles * ADV_TILE_M) + (size_t)tile * ADV_TILE_M + r] = y;
            tc_fence_before();
            mbar_arrive(&acc_empty[ab]);
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == LG_STAGES) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * LG_BN);
    }
}

// scores[row] = b_out + sum over (chunk, half) of partial[chunk][half][row], in that order.
__global__ void sum_partials_kernel(const float* __restrict__ partial, int n_parts, int64_t stride, int64_t n_rows,
                                    const float* __restrict__ b_out, const uint8_t* __restrict__ status,
                                    float* __restrict__ scores, const int* __restrict__ n_rows_dev) {
    if (n_rows_dev) {
        const int64_t c = *n_rows_dev;
        n_rows = c < 0 ? 0 : (c < n_rows ? c : n_rows);
    }
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n_rows;
         row += (int64_t)gridDim.x * blockDim.x) {
        float y = 0.f;
        for (int p = 0; p < n_parts; ++p) y += partial[(size_t)p * stride + row];
        scores[row] = (status && status[row]) ? INFINITY : y + __ldg(b_out);
    }
}

size_t mlp_layer_tc_smem_bytes() {
    return (size_t)LG_STAGES * LG_STAGE_BYTES + (2 * LG_STAGES + 5) * sizeof(uint64_t) + 16 + 1024;
}

cudaError_t launch_mlp_layer_tc(const LayerArgs& a, int num_sms, cudaStream_t s) {
    if (a.n_tiles <= 0) return cudaSuccess;
    if (a.npad <= 0 || a.npad % ADV_SLAB_K != 0 || a.a_slabs <= 0 || a.n_chunks != (a.npad + LG_BN - 1) / LG_BN)
        return cudaErrorInvalidValue;
    const size_t smem = mlp_layer_tc_smem_bytes();
    if (a.fmt == 2 && (!a.fp8 || a.npad % ADV_SLAB_K8 != 0)) return cudaErrorInvalidValue;
    auto kern = a.fmt == 1 ? mlp_layer_tc_kernel<1> : (a.fmt == 2 ? mlp_layer_tc_kernel<2> : mlp_layer_tc_kernel<0>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t items = (int64_t)a.n_tiles * a.n_chunks;
    const int grid = (int)(items < num_sms ? items : num_sms);
    kern<<<grid, LG_THREADS, smem, s>>>(a);
    adv_count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_sum_partials(const float* partial, int n_parts, int64_t stride, int64_t n_rows, const float* b_out,
                                const uint8_t* status, float* scores, int num_sms, cudaStream_t s,
                                const int* n_rows_dev) {
    if (n_rows <= 0) return cudaSuccess;
    const int64_t blocks = (n_rows + 255) / 256;
    const int grid = (int)(blocks < 8 * num_sms ? blocks : 8 * num_sms);
    sum_partials_kernel<<<grid, 256, 0, s>>>(partial, n_parts, stride, n_rows, b_out, status, scores, n_rows_dev);
    adv_count_launch(1);
    return cudaGetLastError();
}

}  // namespace adv
