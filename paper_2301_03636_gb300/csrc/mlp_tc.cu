// Tensor-core MLP scorer (a4-a5) on sm_103a: tcgen05.mma with 16-bit
// operands (BF16 or FP16) from shared memory, FP32 accumulators in tensor
// memory, bias + ReLU + 16-bit cast fused into the epilogue, and the output
// layer (one neuron, Sec. 5 Exp. 3) fused into the last hidden layer's
// epilogue in FP32.
//
// Persistent kernel, one CTA per SM, 608 threads:
//   warps 0, 18  weight producers: stream 64-column K slabs of each hidden
//                layer's weights (pre-packed in the shared-memory image order,
//                one 1-D bulk copy of up to 32 KB per slab) through a 2-stage
//                ring, producer q owning stage q (bulk copies issued by one
//                thread complete one after another, ~450-800 cycles each).
//                Two stages leave room for the biases and the output row in
//                shared memory, which shortens the epilogue more than a third
//                stage would shorten the MMA waits;
//   warp 1       MMA issuer (one thread) and tensor-memory owner;
//   warps 2-17   sixteen epilogue warps.  Warp w reads TMEM lanes
//                32*(w%4) .. 32*(w%4)+31 (one row per thread); the four warps
//                of a lane quadrant take one quarter of the columns each.
// The CTA works on two 128-row tiles at once ("slots" 0 and 1: an activation
// buffer in shared memory and accumulator columns in tensor memory each) and
// issues each layer slot by slot.  All sixteen epilogue warps turn one slot's
// accumulator into the next layer's activations (TMEM -> registers -> bias,
// ReLU, 16-bit -> shared memory) while the tensor core computes the same
// layer for the other slot, then move on to that slot.  The activations never leave shared memory
// between layers.  Activation and weight images are 64-column slabs of
// 128-byte rows with the 128B swizzle, the K-major layout the UMMA
// shared-memory descriptors read.  All waits are bounded by %globaltimer and
// report ADV_DEV_TIMEOUT instead of hanging.
#include "mlp.cuh"

namespace adv {

constexpr int TC_STAGES = 2;
constexpr int TC_THREADS = 32 * (2 + 16 + (TC_STAGES - 1));   // producer 0, MMA, 16 epilogue, producers 1..

// ReLU + round-to-nearest + pack two FP32 values into 16-bit pairs (lo in
// the low half); FP16 saturates to the largest finite value.
template <int FMT>
__device__ __forceinline__ uint32_t relu_pack(float lo, float hi) {
    uint32_t d;
    if constexpr (FMT == 1) asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    else asm("cvt.rn.relu.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

template <int FMT, bool SAVE>
__global__ void __launch_bounds__(TC_THREADS, 1) mlp_tc_kernel(const __grid_constant__ TcArgs a) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_addr(smem_raw);
    uint8_t* base = smem_raw + ((1024u - (raw_addr & 1023u)) & 1023u);

    int nslab_max = 1;
    for (int l = 0; l < a.n_hidden; ++l) nslab_max = a.nslab[l] > nslab_max ? a.nslab[l] : nslab_max;
    const uint32_t act_bytes = (uint32_t)nslab_max * ADV_X_SLAB_BYTES;
    uint8_t* act[2] = {base, base + act_bytes};
    uint8_t* wst = base + 2 * act_bytes;
    const uint32_t stage_bytes = (uint32_t)a.nmax * ADV_SLAB_ROW_BYTES;   // one K slab of all N rows
    // biases of the hidden layers and the output row, staged once per CTA: the
    // epilogue reads them with broadcast shared loads instead of global loads
    float* bias_s = reinterpret_cast<float*>(wst + TC_STAGES * stage_bytes);   // [n_hidden + 1][nmax]
    uint64_t* bars = reinterpret_cast<uint64_t*>(bias_s + (a.n_hidden + 1) * a.nmax);
    uint64_t* w_full = bars;
    uint64_t* w_empty = bars + TC_STAGES;
    uint64_t* x_full = bars + 2 * TC_STAGES;
    uint64_t* acc_full = x_full + 2;       // [2]: the slot's layer is in TMEM
    uint64_t* act_ready = acc_full + 2;    // [2]: the slot's epilogue of the layer is done
    uint64_t* red_full = act_ready + 2;
    uint64_t* drain = red_full + 2;
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
            mbar_init(&act_ready[s], 512);
            mbar_init(&red_full[s], 384);   // column quarters 1..3 of all four lane quadrants
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    for (int i = threadIdx.x; i < (a.n_hidden + 1) * a.nmax; i += blockDim.x) {
        const int l = i / a.nmax, c = i % a.nmax;
        bias_s[i] = l < a.n_hidden ? (c < a.npad[l] ? a.bias[l][c] : 0.f)
                                   : (c < a.npad[a.n_hidden - 1] ? a.w_out[c] : 0.f);
    }
    if (warp == 1) {
        tmem_alloc(tmem_holder, tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    griddep_wait();   // the activation image (and a gathered row count) come from the kernel before
    griddep_trigger();
    int64_t n_rows = a.n_rows;
    if (a.n_rows_dev) {   // a gathered list whose length an earlier kernel wrote
        const int64_t c = *a.n_rows_dev;
        n_rows = c < 0 ? 0 : (c < n_rows ? c : n_rows);
    }
    const int n_tiles = (int)((n_rows + ADV_TILE_M - 1) / ADV_TILE_M);
    const int G = gridDim.x, b = blockIdx.x;
    const int n_my = n_tiles > b ? (n_tiles - b + G - 1) / G : 0;   // tiles b, b+G, b+2G, ...
    const int n_pairs = (n_my + 1) / 2;
    const uint64_t lim = a.timeout_ns;

    if (warp == 0 || warp >= 18) {
        // ---------------- weight producers ----------------
        // The chunks (pair, layer, slot, K slab) form one sequence that the
        // MMA thread consumes through stages 0, 1, 2, 0, ...; producer q
        // fills stage q with every chunk whose index is q modulo TC_STAGES.
        const int q = warp == 0 ? 0 : warp - 17;
        if (lane == 0) {
            uint32_t phase = 0;
            int idx = 0, mine = 0;
            bool ok = true;
            for (int p = 0; p < n_pairs && ok; ++p) {
                const int ns = (2 * p + 1 < n_my) ? 2 : 1;
                for (int l = 0; l < a.n_hidden && ok; ++l) {
                    const uint32_t sb = (uint32_t)a.npad[l] * ADV_SLAB_ROW_BYTES;   // one 64-column K slab
                    for (int s = 0; s < ns && ok; ++s) {
                        for (int k = 0; k < a.nslab[l]; ++k, ++idx) {
                            if (idx % TC_STAGES != q) continue;
                            if (!mbar_wait_bounded(&w_empty[q], phase ^ 1u, a.status_word, abort_flag, lim)) {
                                ok = false;
                                break;
                            }
                            mbar_expect_tx(&w_full[q], sb);
                            bulk_g2s(wst + q * stage_bytes, a.w_img[l] + (size_t)k * sb, sb, &w_full[q]);
                            ++mine;
                            phase ^= 1u;
                        }
                    }
                }
            }
            // this producer's last copy ends before the CTA does (on the
            // normal path the MMA thread has consumed it already)
            if (mine > 0) mbar_wait_bounded(&w_full[q], phase ^ 1u, a.status_word, abort_flag, lim);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            uint32_t stage = 0, phase = 0;
            uint32_t xph[2] = {0, 0}, aph[2] = {0, 0};
            bool ok = true, any = false;
            bool stores = false;   // TMA stores of saved activations issued (training forward)
            for (int p = 0; p < n_pairs && ok; ++p) {
                const int ns = (2 * p + 1 < n_my) ? 2 : 1;
                for (int l = 0; l < a.n_hidden && ok; ++l) {
                    const uint32_t idesc = f16_idesc((uint32_t)FMT, 128u, (uint32_t)a.npad[l]);
                    for (int s = 0; s < ns && ok; ++s) {
                        if (l == 0) {
                            ok = mbar_wait_bounded(&x_full[s], xph[s], a.status_word, abort_flag, lim);
                            xph[s] ^= 1u;
                        }
                        if (ok && (p > 0 || l > 0)) {
                            ok = mbar_wait_bounded(&act_ready[s], aph[s], a.status_word, abort_flag, lim);
                            aph[s] ^= 1u;
                        }
                        if (!ok) break;
                        tc_fence_after();
                        if constexpr (SAVE) {
                            // layer l - 1's output is complete in act[s]: store it for the backward
                            if (l >= 1 && a.use_tma_save && a.save_act[l - 1]) {
                                const int32_t row0 = (int32_t)((int64_t)(b + (2 * p + s) * G) * ADV_TILE_M);
                                for (int k = 0; k < a.nslab[l]; ++k)
                                    tma_store_2d(&a.tm_save[l - 1], act[s] + (size_t)k * ADV_X_SLAB_BYTES, 64 * k,
                                                 row0);
                                bulk_commit();
                                stores = true;
                            }
                        }
                        const uint32_t d_tmem = tmem + (uint32_t)(s * a.nmax);
                        for (int k = 0; k < a.nslab[l]; ++k) {
                            if (!mbar_wait_bounded(&w_full[stage], phase, a.status_word, abort_flag, lim)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint64_t bdesc = sw128_desc(smem_addr(wst + stage * stage_bytes));
                            const uint64_t adesc = sw128_desc(smem_addr(act[s] + (size_t)k * ADV_X_SLAB_BYTES));
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk)
                                umma_f16(d_tmem, adesc + 2u * kk, bdesc + 2u * kk, idesc, (k | kk) != 0);
                            umma_commit(&w_empty[stage]);
                            any = true;
                            if (++stage == TC_STAGES) { stage = 0; phase ^= 1u; }
                        }
                        if (!ok) break;
                        // the epilogue (or the next X load) writes act[s] once the accumulator is
                        // ready: the stores above must have read it first
                        if (SAVE && stores) bulk_wait_read<0>();
                        umma_commit(&acc_full[s]);
                    }
                }
            }
            if (any) {   // every issued MMA has completed before tensor memory is released
                umma_commit(drain);
                mbar_wait_bounded(drain, 0, a.status_word, abort_flag, lim);
            }
            if (SAVE && stores) bulk_wait_all();   // the saved activations are written before the CTA ends
        }
    } else {
        // ---------------- epilogue warps ----------------
        const int e = warp - 2;                     // 0..15
        const int j = e >> 2;                       // column quarter
        const int quad = warp & 3;                  // TMEM lane quadrant
        const uint32_t r = (uint32_t)(quad * 32 + lane);
        const bool leader = e == 0 && lane == 0;
        const int nslab0 = a.nslab[0];
        const uint32_t x_bytes = (uint32_t)nslab0 * ADV_X_SLAB_BYTES;
        uint32_t accph[2] = {0, 0}, redph[2] = {0, 0}, xph[2] = {0, 0};
        int x_pending[2] = {0, 0};
        auto load_x = [&](int s, int tile) {
            mbar_expect_tx(&x_full[s], x_bytes);
            const uint8_t* src = a.x_img + (size_t)tile * x_bytes;
            for (int k = 0; k < nslab0; ++k)
                bulk_g2s(act[s] + (size_t)k * ADV_X_SLAB_BYTES, src + (size_t)k * ADV_X_SLAB_BYTES,
                         ADV_X_SLAB_BYTES, &x_full[s]);
        };
        if (leader) {
            for (int s = 0; s < 2 && s < n_my; ++s) { load_x(s, b + s * G); x_pending[s] = 1; }
        }
        bool ok = true;
        for (int p = 0; p < n_pairs && ok; ++p) {
            const int ns = (2 * p + 1 < n_my) ? 2 : 1;
            for (int l = 0; l < a.n_hidden && ok; ++l) {
                const bool last = (l + 1 == a.n_hidden);
                const float* bias = bias_s + l * a.nmax;
                const int cw = a.npad[l] >> 2;              // this warp's columns: [cb, cb + cw), cw % 16 == 0
                const int cb = j * cw;
                for (int s = 0; s < ns; ++s) {
                    const int i = 2 * p + s;                // tile index within this CTA
                    const bool got = mbar_wait_bounded(&acc_full[s], accph[s], a.status_word, abort_flag, lim);
                    __syncwarp();   // tcgen05.ld / st / wait are warp-collective (.sync.aligned)
                    if (!got) { ok = false; break; }
                    accph[s] ^= 1u;
                    if (l == 0) { x_pending[s] = 0; xph[s] ^= 1u; }   // the MMAs consumed the X tile
                    tc_fence_after();
                    // the X buffer of this slot is free: every MMA that read it has completed
                    if (last && leader && i + 2 < n_my) { load_x(s, b + (i + 2) * G); x_pending[s] = 1; }
                    const uint32_t t_base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(s * a.nmax);
                    uint8_t* my_act = act[s];
                    float y4[4] = {0.f, 0.f, 0.f, 0.f};
                    // training: this layer's 16-bit activations also go to global memory, row-major
                    const int64_t grow = (int64_t)(b + i * G) * ADV_TILE_M + r;
                    uint8_t* save = SAVE && a.save_act[l] && grow < n_rows
                                        ? reinterpret_cast<uint8_t*>(a.save_act[l]) + (size_t)grow * a.save_ld[l] * 2
                                        : nullptr;
                    for (int c0 = cb; c0 < cb + cw; c0 += 32) {
                        const bool two = c0 + 16 < cb + cw;     // a second 16-column group in this step
                        uint32_t v0[16], v1[16];
                        tmem_ld_32x32b_x16(t_base + (uint32_t)c0, v0);
                        if (two) tmem_ld_32x32b_x16(t_base + (uint32_t)(c0 + 16), v1);
                        float4 bq[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            bq[q] = (q < 4 || two) ? reinterpret_cast<const float4*>(bias + c0)[q]
                                                   : make_float4(0.f, 0.f, 0.f, 0.f);
                        tmem_wait_ld();
                        const float* bf = reinterpret_cast<const float*>(bq);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            if (h == 1 && !two) break;
                            const uint32_t* v = h ? v1 : v0;
                            const int c = c0 + 16 * h;
                            if (!last) {
                                uint8_t* slab = my_act + (size_t)(c >> 6) * ADV_X_SLAB_BYTES;
#pragma unroll
                                for (int q = 0; q < 2; ++q) {
                                    uint32_t pk[4];
#pragma unroll
                                    for (int t = 0; t < 4; ++t) {
                                        const int cc = 8 * q + 2 * t;
                                        pk[t] = relu_pack<FMT>(__uint_as_float(v[cc]) + bf[16 * h + cc],
                                                               __uint_as_float(v[cc + 1]) + bf[16 * h + cc + 1]);
                                    }
                                    const uint32_t chunk = (uint32_t)(((c & 63) >> 3) + q);
                                    *reinterpret_cast<uint4*>(slab + sw128_offset(r, chunk)) =
                                        make_uint4(pk[0], pk[1], pk[2], pk[3]);
                                    if (SAVE && save && !a.use_tma_save && c + 8 * q < a.save_ld[l])
                                        *reinterpret_cast<uint4*>(save + (size_t)(c + 8 * q) * 2) =
                                            make_uint4(pk[0], pk[1], pk[2], pk[3]);
                                }
                            } else {
                                if (SAVE && save) {
#pragma unroll
                                    for (int q = 0; q < 2; ++q) {
                                        uint32_t pk[4];
#pragma unroll
                                        for (int t = 0; t < 4; ++t) {
                                            const int cc = 8 * q + 2 * t;
                                            pk[t] = relu_pack<FMT>(__uint_as_float(v[cc]) + bf[16 * h + cc],
                                                                   __uint_as_float(v[cc + 1]) + bf[16 * h + cc + 1]);
                                        }
                                        if (c + 8 * q < a.save_ld[l])
                                            *reinterpret_cast<uint4*>(save + (size_t)(c + 8 * q) * 2) =
                                                make_uint4(pk[0], pk[1], pk[2], pk[3]);
                                    }
                                }
                                const float4* w4 = reinterpret_cast<const float4*>(bias_s + a.n_hidden * a.nmax + c);
#pragma unroll
                                for (int u = 0; u < 4; ++u) {
                                    const float4 wq = w4[u];   // staged in shared memory
                                    const float* bb = bf + 16 * h + 4 * u;
                                    y4[0] = fmaf(fmaxf(__uint_as_float(v[4 * u + 0]) + bb[0], 0.f), wq.x, y4[0]);
                                    y4[1] = fmaf(fmaxf(__uint_as_float(v[4 * u + 1]) + bb[1], 0.f), wq.y, y4[1]);
                                    y4[2] = fmaf(fmaxf(__uint_as_float(v[4 * u + 2]) + bb[2], 0.f), wq.z, y4[2]);
                                    y4[3] = fmaf(fmaxf(__uint_as_float(v[4 * u + 3]) + bb[3], 0.f), wq.w, y4[3]);
                                }
                            }
                        }
                    }
                    if (!last) {
                        fence_proxy_async_smem();   // make the generic stores visible to the tensor core
                    } else {
                        // combine the four column quarters of each row in a fixed order: quarters
                        // 1..3 park their partial sums in their own (already read) TMEM columns
                        float y = (y4[0] + y4[1]) + (y4[2] + y4[3]);
                        if (j != 0) {
                            tmem_st_32x32b_x1(t_base + (uint32_t)cb, __float_as_uint(y));
                            tmem_wait_st();
                            tc_fence_before();
                            mbar_arrive(&red_full[s]);
                        } else {
                            const bool gr = mbar_wait_bounded(&red_full[s], redph[s], a.status_word, abort_flag, lim);
                            __syncwarp();
                            if (gr) {
                                tc_fence_after();
                                const float y1 = __uint_as_float(tmem_ld_32x32b_x1(t_base + (uint32_t)cw));
                                const float y2 = __uint_as_float(tmem_ld_32x32b_x1(t_base + (uint32_t)(2 * cw)));
                                const float y3 = __uint_as_float(tmem_ld_32x32b_x1(t_base + (uint32_t)(3 * cw)));
                                tmem_wait_ld();
                                y = ((y + y1) + y2) + y3 + __ldg(a.b_out);
                                const int64_t row = (int64_t)(b + i * G) * ADV_TILE_M + r;
                                if (row < n_rows) a.scores[row] = (a.status && a.status[row]) ? INFINITY : y;
                            }
                        }
                        redph[s] ^= 1u;
                    }
                    tc_fence_before();
                    mbar_arrive(&act_ready[s]);
                }
            }
        }
        if (leader) {
            for (int s = 0; s < 2; ++s)
                if (x_pending[s]) mbar_wait_bounded(&x_full[s], xph[s], a.status_word, abort_flag, lim);
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, tmem_cols);
    }
}

size_t mlp_tc_smem_bytes(int nslab_max, int nmax, int n_hidden) {
    return (size_t)2 * nslab_max * ADV_X_SLAB_BYTES + (size_t)TC_STAGES * nmax * ADV_SLAB_ROW_BYTES +
           (size_t)(n_hidden + 1) * nmax * sizeof(float) + (2 * TC_STAGES + 9) * sizeof(uint64_t) + 16 + 1024;
}

cudaError_t launch_mlp_tc(const TcArgs& a, int num_sms, cudaStream_t s, int ctas) {
    if (a.n_tiles <= 0) return cudaSuccess;
    int nslab_max = 1;
    for (int l = 0; l < a.n_hidden; ++l) nslab_max = a.nslab[l] > nslab_max ? a.nslab[l] : nslab_max;
    const size_t smem = mlp_tc_smem_bytes(nslab_max, a.nmax, a.n_hidden);
    bool save = false;
    for (int l = 0; l < a.n_hidden; ++l) save = save || a.save_act[l] != nullptr;
    auto kern = a.fmt == 1 ? (save ? mlp_tc_kernel<1, true> : mlp_tc_kernel<1, false>)
                           : (save ? mlp_tc_kernel<0, true> : mlp_tc_kernel<0, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int cap = (ctas > 0 && ctas < num_sms) ? ctas : num_sms;   // at most one resident CTA per SM
    const int grid = a.n_tiles < cap ? a.n_tiles : cap;
    e = launch_pdl(kern, dim3(grid), dim3(TC_THREADS), smem, s, a);
    if (e != cudaSuccess) return e;
    adv_count_launch(1);
    return cudaGetLastError();
}

}  // namespace adv
