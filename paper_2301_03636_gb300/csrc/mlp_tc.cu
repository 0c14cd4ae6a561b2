// Tensor-core MLP scorer (a4-a5) on sm_103a: tcgen05.mma with 16-bit
// operands (BF16 or FP16) from shared memory, FP32 accumulators in tensor
// memory, bias + ReLU + 16-bit cast fused into the epilogue, and the output
// layer (one neuron, Sec. 5 Exp. 3) fused into the last hidden layer's
// epilogue in FP32.
//
// Persistent kernel, one CTA per SM, 320 threads:
//   warp 0      weight producer: streams 64-column K slabs of each hidden
//               layer's weights (pre-packed in the shared-memory image order,
//               one 1-D bulk copy per slab) through a 3-stage ring;
//   warp 1      MMA issuer (one thread) and tensor-memory owner;
//   warps 2-9   two epilogue groups of four warps; group g owns "slot" g:
//               one 128-row tile, its activation buffer in shared memory and
//               its accumulator columns in tensor memory.  Warp w reads TMEM
//               lanes 32*(w%4) .. 32*(w%4)+31, one row per thread.
// The CTA works on two tiles at once (slots 0 and 1).  Each weight slab is
// loaded once and applied to both tiles (M = 256 rows per slab), so weight
// traffic from L2 is halved; the activations never leave shared memory
// between layers.  Activation images are 64-column slabs of 128-byte rows
// with the 128B swizzle, the K-major layout the UMMA shared-memory
// descriptors read.  All waits are bounded by %globaltimer and report
// ADV_DEV_TIMEOUT instead of hanging.
#include "mlp.cuh"

namespace adv {

constexpr int TC_THREADS = 320;
constexpr int TC_STAGES = 3;

__device__ __forceinline__ uint32_t pack2_16(float a, float b, int fmt) {
    if (fmt == 1) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
    __half2 h = __floats2half2_rn(fminf(a, 65504.f), fminf(b, 65504.f));
    return *reinterpret_cast<uint32_t*>(&h);
}

__global__ void __launch_bounds__(TC_THREADS, 1) mlp_tc_kernel(const __grid_constant__ TcArgs a) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_addr(smem_raw);
    uint8_t* base = smem_raw + ((1024u - (raw_addr & 1023u)) & 1023u);

    int nslab_max = 1;
    for (int l = 0; l < a.n_hidden; ++l) nslab_max = a.nslab[l] > nslab_max ? a.nslab[l] : nslab_max;
    const uint32_t act_bytes = (uint32_t)nslab_max * ADV_X_SLAB_BYTES;
    const uint32_t wslab_bytes = (uint32_t)a.nmax * ADV_SLAB_ROW_BYTES;
    uint8_t* act[2] = {base, base + act_bytes};
    uint8_t* wst = base + 2 * act_bytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(wst + TC_STAGES * wslab_bytes);
    uint64_t* w_full = bars;
    uint64_t* w_empty = bars + TC_STAGES;
    uint64_t* x_full = bars + 2 * TC_STAGES;
    uint64_t* acc_full = x_full + 2;
    uint64_t* act_ready = acc_full + 2;
    uint64_t* drain = act_ready + 2;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

    uint32_t tmem_cols = 32;
    while (tmem_cols < 2u * (uint32_t)a.nmax) tmem_cols <<= 1;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&w_full[s], 1);
            mbar_init(&w_empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&x_full[s], 1);
            mbar_init(&acc_full[s], 1);
            mbar_init(&act_ready[s], 128);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    if (warp == 1) {
        tmem_alloc(tmem_holder, tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    const int G = gridDim.x, b = blockIdx.x;
    const int n_my = a.n_tiles > b ? (a.n_tiles - b + G - 1) / G : 0;   // tiles b, b+G, b+2G, ...
    const int n_pairs = (n_my + 1) / 2;
    const uint64_t lim = a.timeout_ns;

    if (warp == 0) {
        // ---------------- weight producer ----------------
        if (lane == 0) {
            uint32_t stage = 0, phase = 0;
            int issued = 0;
            bool ok = true;
            for (int p = 0; p < n_pairs && ok; ++p) {
                for (int l = 0; l < a.n_hidden && ok; ++l) {
                    const uint32_t sb = (uint32_t)a.npad[l] * ADV_SLAB_ROW_BYTES;
                    for (int k = 0; k < a.nslab[l]; ++k) {
                        if (!mbar_wait_bounded(&w_empty[stage], phase ^ 1u, a.status_word, abort_flag, lim)) {
                            ok = false;
                            break;
                        }
                        mbar_expect_tx(&w_full[stage], sb);
                        bulk_g2s(wst + stage * wslab_bytes, a.w_img[l] + (size_t)k * sb, sb, &w_full[stage]);
                        ++issued;
                        if (++stage == TC_STAGES) { stage = 0; phase ^= 1u; }
                    }
                }
            }
            // copies in flight end before the CTA does (they complete quickly,
            // and on the normal path the MMA thread has already consumed them)
            for (int i = 0; i < TC_STAGES && i < issued; ++i) {
                if (stage == 0) { stage = TC_STAGES; phase ^= 1u; }
                --stage;
                mbar_wait_bounded(&w_full[stage], phase, a.status_word, abort_flag, lim);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            uint32_t stage = 0, phase = 0;
            uint32_t xph[2] = {0, 0}, aph[2] = {0, 0};
            bool ok = true, any = false;
            for (int p = 0; p < n_pairs && ok; ++p) {
                const int ns = (2 * p + 1 < n_my) ? 2 : 1;
                for (int l = 0; l < a.n_hidden && ok; ++l) {
                    for (int s = 0; s < ns && ok; ++s) {
                        if (l == 0) {
                            ok = mbar_wait_bounded(&x_full[s], xph[s], a.status_word, abort_flag, lim);
                            xph[s] ^= 1u;
                        }
                        if (ok && (p > 0 || l > 0)) {
                            ok = mbar_wait_bounded(&act_ready[s], aph[s], a.status_word, abort_flag, lim);
                            aph[s] ^= 1u;
                        }
                    }
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t idesc = f16_idesc((uint32_t)a.fmt, 128u, (uint32_t)a.npad[l]);
                    for (int k = 0; k < a.nslab[l]; ++k) {
                        if (!mbar_wait_bounded(&w_full[stage], phase, a.status_word, abort_flag, lim)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t bdesc = sw128_desc(smem_addr(wst + stage * wslab_bytes));
                        for (int s = 0; s < ns; ++s) {
                            const uint64_t adesc = sw128_desc(smem_addr(act[s] + (size_t)k * ADV_X_SLAB_BYTES));
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk)
                                umma_f16(tmem + (uint32_t)(s * a.nmax), adesc + 2u * kk, bdesc + 2u * kk, idesc,
                                         (k | kk) != 0);
                        }
                        umma_commit(&w_empty[stage]);
                        any = true;
                        if (++stage == TC_STAGES) { stage = 0; phase ^= 1u; }
                    }
                    if (!ok) break;
                    for (int s = 0; s < ns; ++s) umma_commit(&acc_full[s]);
                }
            }
            if (any) {   // every issued MMA has completed before tensor memory is released
                umma_commit(drain);
                mbar_wait_bounded(drain, 0, a.status_word, abort_flag, lim);
            }
        }
    } else {
        // ---------------- epilogue groups ----------------
        const int g = (warp - 2) >> 2;              // slot
        const int quad = warp & 3;                  // TMEM lane quadrant
        const uint32_t r = (uint32_t)(quad * 32 + lane);
        const bool leader = (warp == 2 + 4 * g) && lane == 0;
        const int nslab0 = a.nslab[0];
        const uint32_t x_bytes = (uint32_t)nslab0 * ADV_X_SLAB_BYTES;
        uint8_t* my_act = act[g];
        const uint32_t t_base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(g * a.nmax);
        uint32_t accph = 0;
        int x_pending = 0;
        uint32_t xph = 0;
        auto load_x = [&](int tile) {
            mbar_expect_tx(&x_full[g], x_bytes);
            const uint8_t* src = a.x_img + (size_t)tile * x_bytes;
            for (int k = 0; k < nslab0; ++k)
                bulk_g2s(my_act + (size_t)k * ADV_X_SLAB_BYTES, src + (size_t)k * ADV_X_SLAB_BYTES,
                         ADV_X_SLAB_BYTES, &x_full[g]);
        };
        if (leader && g < n_my) { load_x(b + g * G); x_pending = 1; }
        bool ok = true;
        for (int i = g; i < n_my && ok; i += 2) {
            const int tile = b + i * G;
            const int64_t row = (int64_t)tile * ADV_TILE_M + r;
            for (int l = 0; l < a.n_hidden; ++l) {
                const bool got = mbar_wait_bounded(&acc_full[g], accph, a.status_word, abort_flag, lim);
                __syncwarp();   // tcgen05.ld / wait::ld are warp-collective (.sync.aligned)
                if (!got) { ok = false; break; }
                accph ^= 1u;
                if (l == 0) { x_pending = 0; xph ^= 1u; }   // the MMAs consumed the X tile
                tc_fence_after();
                const float* __restrict__ bias = a.bias[l];
                const int np = a.npad[l];
                if (l + 1 < a.n_hidden) {
                    for (int c0 = 0; c0 < np; c0 += 32) {
                        uint32_t v[32];
                        tmem_ld_32x32b_x32(t_base + (uint32_t)c0, v);
                        tmem_wait_ld();
                        uint8_t* slab = my_act + (size_t)(c0 >> 6) * ADV_X_SLAB_BYTES;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float4 b0 = __ldg(reinterpret_cast<const float4*>(bias + c0 + 8 * q));
                            const float4 b1 = __ldg(reinterpret_cast<const float4*>(bias + c0 + 8 * q + 4));
                            const float h0 = fmaxf(__uint_as_float(v[8 * q + 0]) + b0.x, 0.f);
                            const float h1 = fmaxf(__uint_as_float(v[8 * q + 1]) + b0.y, 0.f);
                            const float h2 = fmaxf(__uint_as_float(v[8 * q + 2]) + b0.z, 0.f);
                            const float h3 = fmaxf(__uint_as_float(v[8 * q + 3]) + b0.w, 0.f);
                            const float h4 = fmaxf(__uint_as_float(v[8 * q + 4]) + b1.x, 0.f);
                            const float h5 = fmaxf(__uint_as_float(v[8 * q + 5]) + b1.y, 0.f);
                            const float h6 = fmaxf(__uint_as_float(v[8 * q + 6]) + b1.z, 0.f);
                            const float h7 = fmaxf(__uint_as_float(v[8 * q + 7]) + b1.w, 0.f);
                            const uint4 pk = make_uint4(pack2_16(h0, h1, a.fmt), pack2_16(h2, h3, a.fmt),
                                                        pack2_16(h4, h5, a.fmt), pack2_16(h6, h7, a.fmt));
                            const uint32_t chunk = (uint32_t)(((c0 & 63) >> 3) + q);
                            *reinterpret_cast<uint4*>(slab + sw128_offset(r, chunk)) = pk;
                        }
                    }
                    fence_proxy_async_smem();   // make the generic stores visible to the tensor core
                } else {
                    // the X buffer is free: every MMA that read it has completed
                    if (leader && i + 2 < n_my) { load_x(b + (i + 2) * G); x_pending = 1; }
                    float y = 0.f;
                    for (int c0 = 0; c0 < np; c0 += 32) {
                        uint32_t v[32];
                        tmem_ld_32x32b_x32(t_base + (uint32_t)c0, v);
                        tmem_wait_ld();
#pragma unroll
                        for (int e = 0; e < 32; ++e) {
                            const float h = fmaxf(__uint_as_float(v[e]) + __ldg(bias + c0 + e), 0.f);
                            y = fmaf(h, __ldg(a.w_out + c0 + e), y);
                        }
                    }
                    y += __ldg(a.b_out);
                    if (row < a.n_rows) a.scores[row] = (a.status && a.status[row]) ? INFINITY : y;
                }
                tc_fence_before();
                mbar_arrive(&act_ready[g]);
            }
        }
        if (leader && x_pending) mbar_wait_bounded(&x_full[g], xph, a.status_word, abort_flag, lim);
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, tmem_cols);
    }
}

size_t mlp_tc_smem_bytes(int nslab_max, int nmax) {
    return (size_t)2 * nslab_max * ADV_X_SLAB_BYTES + (size_t)TC_STAGES * nmax * ADV_SLAB_ROW_BYTES +
           (2 * TC_STAGES + 7) * sizeof(uint64_t) + 16 + 1024;
}

cudaError_t launch_mlp_tc(const TcArgs& a, int num_sms, cudaStream_t s) {
    if (a.n_tiles <= 0) return cudaSuccess;
    int nslab_max = 1;
    for (int l = 0; l < a.n_hidden; ++l) nslab_max = a.nslab[l] > nslab_max ? a.nslab[l] : nslab_max;
    const size_t smem = mlp_tc_smem_bytes(nslab_max, a.nmax);
    cudaError_t e = cudaFuncSetAttribute(mlp_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = a.n_tiles < num_sms ? a.n_tiles : num_sms;
    mlp_tc_kernel<<<grid, TC_THREADS, smem, s>>>(a);
    adv_count_launch(1);
    return cudaGetLastError();
}

}  // namespace adv
