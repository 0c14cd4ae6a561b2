// SIMT MLP scorers (Sec. 4.2 cost model, Sec. 5 Exp. 3 network):
//  - FP32 "plain" path: standardise -> ReLU hidden layers -> linear output,
//    FP32 FMA on the CUDA cores, all layers fused per tile of rows with the
//    activations resident in shared memory;
//  - FP64 re-score: one block per row, each dot product summed sequentially
//    over the input index with separately rounded products and sums (the
//    summation order of the FP64 definition), so that its value is the exact
//    FP64 reference value of that row.
// Both read rows either from int32 features or straight from descriptors,
// optionally through a device-side list of row indices (near-tie re-score).
#include "features.cuh"
#include "mlp.cuh"

namespace adv {

template <int F, bool FROM_DESC>
__device__ __forceinline__ bool fetch_row_features(const RowSrc& src, int64_t row, int32_t (&f)[F]) {
    if constexpr (FROM_DESC) {
        int64_t d[16];
        load_desc(src.desc, row, d);
        const uint32_t st = validate_row(d);
        if (st == 0) row_features<F>(d, f);
        else {
#pragma unroll
            for (int j = 0; j < F; ++j) f[j] = 0;
        }
        return st == 0 && !(src.status && src.status[row]);
    } else {
        if constexpr (F % 4 == 0) {
            const int4* p = reinterpret_cast<const int4*>(src.feat + (size_t)row * F);
#pragma unroll
            for (int j = 0; j < F / 4; ++j) {
                const int4 v = __ldg(p + j);
                f[4 * j] = v.x; f[4 * j + 1] = v.y; f[4 * j + 2] = v.z; f[4 * j + 3] = v.w;
            }
        } else {   // rows not 16-byte aligned (F = 33)
#pragma unroll
            for (int j = 0; j < F; ++j) f[j] = __ldg(src.feat + (size_t)row * F + j);
        }
        return !(src.status && src.status[row]);
    }
}

// A group of G lanes fetches one row (row < 0: none): lane g of the group
// keeps features g + G q in mine[q] (zeros for an invalid or absent row).
// Returns the row's validity; every lane of the warp must call it.
template <int F, int G, bool FROM_DESC>
__device__ __forceinline__ bool fetch_row_features_lanes(const RowSrc& src, int64_t row, int g,
                                                         int32_t (&mine)[(F + G - 1) / G]) {
    bool ok = false;
    if constexpr (FROM_DESC) {
        int64_t d[16];
        if (row >= 0) {
            load_desc(src.desc, row, d);
            ok = validate_row(d) == 0;
        }
        if (!ok) placeholder_desc(d);
        row_features_lanes<F, G>(d, g, mine);
        if (!ok) {
#pragma unroll
            for (int q = 0; q < (F + G - 1) / G; ++q) mine[q] = 0;
        }
    } else {
        if (row >= 0) {
            const int32_t* p = src.feat + (size_t)row * F;
#pragma unroll
            for (int q = 0; q < (F + G - 1) / G; ++q) mine[q] = G * q + g < F ? __ldg(p + G * q + g) : 0;
            ok = true;
        } else {
#pragma unroll
            for (int q = 0; q < (F + G - 1) / G; ++q) mine[q] = 0;
        }
    }
    return ok && !(src.status && src.status[row]);
}

// TM rows per tile, RPT rows per thread, 8 columns per thread, 256 threads.
template <int TM, int RPT, int F, bool FROM_DESC>
__global__ void __launch_bounds__(256) mlp_fp32_kernel(MlpDesc m, RowSrc src, float* __restrict__ out, int ws) {
    constexpr int RG = TM / RPT;       // row groups
    constexpr int CG = 256 / RG;       // column lanes
    constexpr int CW = CG * 8;         // columns per chunk
    constexpr int KC = 16;             // K per staged weight chunk
    static_assert(RG * CG == 256, "thread layout");
    extern __shared__ float smem_f[];
    float* act0 = smem_f;
    float* act1 = act0 + TM * ws;
    float* Wst = act1 + TM * ws;       // [KC][CW]
    __shared__ int64_t row_of[TM];
    __shared__ int row_ok[TM];

    const int tid = threadIdx.x;
    const int rg = tid / CG, cg = tid % CG;
    const int64_t count = src.count_dev ? (int64_t)*src.count_dev : src.count;
    const int64_t ntiles = (count + TM - 1) / TM;

    for (int i = tid; i < 2 * TM * ws; i += 256) act0[i] = 0.f;

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        float* in = act0;
        float* outb = act1;
        if (tid < TM) {
            const int64_t pos = tile * TM + tid;
            int64_t row = -1;
            if (pos < count) row = src.rows ? src.rows[pos] : pos;
            row_of[tid] = row;
            int ok = 0;
            if (row >= 0) {
                int32_t f[F];
                ok = fetch_row_features<F, FROM_DESC>(src, row, f) ? 1 : 0;
#pragma unroll
                for (int k = 0; k < F; ++k) in[tid * ws + k] = fmaf((float)f[k], __ldg(m.sa + k), -__ldg(m.sc + k));
            } else {
#pragma unroll
                for (int k = 0; k < F; ++k) in[tid * ws + k] = 0.f;
            }
            row_ok[tid] = ok;
        }
        __syncthreads();

        for (int l = 0; l + 2 < m.nw; ++l) {
            const int fi = m.widths[l], fo = m.widths[l + 1];
            const float* __restrict__ Wl = m.W[l];
            const float* __restrict__ bl = m.b[l];
            for (int c0 = 0; c0 < fo; c0 += CW) {
                float acc[RPT][8];
#pragma unroll
                for (int i = 0; i < RPT; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
                for (int k0 = 0; k0 < fi; k0 += KC) {
                    __syncthreads();
                    // stage W[c0 + n][k0 + kk] as Wst[kk][n]
                    for (int idx = tid; idx < KC * CW; idx += 256) {
                        const int n = idx / KC, kk = idx % KC;
                        const int gn = c0 + n, gk = k0 + kk;
                        Wst[kk * CW + n] = (gn < fo && gk < fi) ? __ldg(Wl + (size_t)gn * fi + gk) : 0.f;
                    }
                    __syncthreads();
#pragma unroll
                    for (int kk = 0; kk < KC; ++kk) {
                        float a[RPT], w[8];
#pragma unroll
                        for (int i = 0; i < RPT; ++i) a[i] = in[(rg * RPT + i) * ws + k0 + kk];
#pragma unroll
                        for (int j = 0; j < 8; ++j) w[j] = Wst[kk * CW + cg + CG * j];
#pragma unroll
                        for (int i = 0; i < RPT; ++i)
#pragma unroll
                            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], w[j], acc[i][j]);
                    }
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int c = c0 + cg + CG * j;
                    if (c < fo) {
                        const float bb = __ldg(bl + c);
#pragma unroll
                        for (int i = 0; i < RPT; ++i) outb[(rg * RPT + i) * ws + c] = fmaxf(acc[i][j] + bb, 0.f);
                    }
                }
            }
            __syncthreads();
            float* t = in; in = outb; outb = t;
        }
        // output layer: one warp per row, fixed-order reduction
        {
            const int L = m.nw - 2;
            const int fi = m.widths[L];
            const float* __restrict__ wl = m.W[L];
            const int warp = tid >> 5, lane = tid & 31;
            for (int r = warp; r < TM; r += 8) {
                float s = 0.f;
                for (int k = lane; k < fi; k += 32) s = fmaf(in[r * ws + k], __ldg(wl + k), s);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) {
                    const int64_t pos = tile * TM + r;
                    if (pos < count) out[pos] = row_ok[r] ? s + __ldg(m.b[L]) : INFINITY;
                }
            }
        }
    }
}

// 16-byte asynchronous global -> shared copy; src_bytes = 0 fills zeros.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(smem)), "l"(gmem), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// The plain FP32 scorer for hidden widths up to 256: 64-row tiles, thread t
// computes rows 8 (t / 32) .. + 7 and output neurons 8 (t % 32) .. + 7 of
// every layer.  The transposed weights WT[k][j] come into shared memory 16
// input rows at a time with asynchronous 16-byte copies, double-buffered so
// that the next chunk arrives while this one is used; per 4 input indices a
// thread reads its 8 rows' activations and the 4 x 8 weights as 16-byte
// shared loads feeding 256 FMAs.  Each output neuron is still summed over
// the input index in order with FMA, as in mlp_fp32_kernel (same values).
constexpr int T64_KC = 16;

template <int F, bool FROM_DESC>
__global__ void __launch_bounds__(256, 1) mlp_fp32_t64_kernel(MlpDesc m, RowSrc src, float* __restrict__ out, int ws) {
    constexpr int TM = 64, KC = T64_KC, CW = 256;
    extern __shared__ __align__(16) float smem_t[];
    float* act0 = smem_t;                  // [TM][ws] row-major
    float* act1 = act0 + TM * ws;
    float* wst = act1 + TM * ws;           // [2][KC][CW]
    __shared__ int row_ok[TM];
    const int tid = threadIdx.x;
    const int rg = tid >> 5, cq = tid & 31;   // rows 8 rg .. + 7, neurons 8 cq .. + 7
    const int64_t count = src.count_dev ? (int64_t)*src.count_dev : src.count;
    const int64_t ntiles = (count + TM - 1) / TM;
    for (int i = tid; i < 2 * TM * ws; i += 256) act0[i] = 0.f;

    // chunk kc0 of layer l into buffer buf: WT rows kc0 .. kc0 + KC - 1, columns 0 .. CW - 1
    auto stage = [&](int l, int kc0, int buf) {
        const int fi = m.widths[l], ld = m.wt_ld[l];
        const float* wt = m.WT[l];
        float* dst = wst + buf * KC * CW;
#pragma unroll
        for (int q = 0; q < KC * CW / 4 / 256; ++q) {
            const int piece = tid + 256 * q;           // 16-byte piece
            const int kk = piece / (CW / 4), n4 = (piece % (CW / 4)) * 4;
            const bool in = kc0 + kk < fi && n4 < ld;
            cp_async16(dst + kk * CW + n4, in ? wt + (size_t)(kc0 + kk) * ld + n4 : wt, in ? 16 : 0);
        }
        cp_async_commit();
    };

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        float* in = act0;
        float* outb = act1;
        if (tid < TM) {
            const int64_t pos = tile * TM + tid;
            int64_t row = -1;
            if (pos < count) row = src.rows ? src.rows[pos] : pos;
            int ok = 0;
            if (row >= 0) {
                int32_t f[F];
                ok = fetch_row_features<F, FROM_DESC>(src, row, f) ? 1 : 0;
#pragma unroll
                for (int k = 0; k < F; ++k) in[tid * ws + k] = fmaf((float)f[k], __ldg(m.sa + k), -__ldg(m.sc + k));
            } else {
#pragma unroll
                for (int k = 0; k < F; ++k) in[tid * ws + k] = 0.f;
            }
            row_ok[tid] = ok;
        }
        __syncthreads();
        for (int l = 0; l + 2 < m.nw; ++l) {
            const int fi = m.widths[l], fo = m.widths[l + 1];
            const int nck = (fi + KC - 1) / KC;
            float acc[8][8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
            stage(l, 0, 0);
            for (int c = 0; c < nck; ++c) {
                if (c + 1 < nck) {
                    stage(l, (c + 1) * KC, (c + 1) & 1);
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
                __syncthreads();
                const float* w = wst + (c & 1) * KC * CW + 8 * cq;
                const float* a = in + (8 * rg) * ws + c * KC;
#pragma unroll
                for (int k4 = 0; k4 < KC; k4 += 4) {
                    float av[8][4];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float4 t = *reinterpret_cast<const float4*>(a + i * ws + k4);
                        av[i][0] = t.x; av[i][1] = t.y; av[i][2] = t.z; av[i][3] = t.w;
                    }
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const float4 w0 = *reinterpret_cast<const float4*>(w + (k4 + kk) * CW);
                        const float4 w1 = *reinterpret_cast<const float4*>(w + (k4 + kk) * CW + 4);
                        const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                        for (int i = 0; i < 8; ++i)
#pragma unroll
                            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i][kk], wv[j], acc[i][j]);
                    }
                }
                __syncthreads();   // buffer c & 1 is refilled two chunks later
            }
            // bias + ReLU; columns past fo are never read by the next layer
            float bb[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) bb[j] = 8 * cq + j < fo ? __ldg(m.b[l] + 8 * cq + j) : 0.f;
            if (8 * cq < fo) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    float* o = outb + (8 * rg + i) * ws + 8 * cq;
                    *reinterpret_cast<float4*>(o) = make_float4(fmaxf(acc[i][0] + bb[0], 0.f), fmaxf(acc[i][1] + bb[1], 0.f),
                                                                fmaxf(acc[i][2] + bb[2], 0.f), fmaxf(acc[i][3] + bb[3], 0.f));
                    *reinterpret_cast<float4*>(o + 4) = make_float4(fmaxf(acc[i][4] + bb[4], 0.f), fmaxf(acc[i][5] + bb[5], 0.f),
                                                                    fmaxf(acc[i][6] + bb[6], 0.f), fmaxf(acc[i][7] + bb[7], 0.f));
                }
            }
            __syncthreads();
            float* t = in; in = outb; outb = t;
        }
        {
            const int L = m.nw - 2;
            const int fi = m.widths[L];
            const float* __restrict__ wl = m.W[L];
            const int warp = tid >> 5, lane = tid & 31;
            for (int r = warp; r < TM; r += 8) {
                float s = 0.f;
                for (int k = lane; k < fi; k += 32) s = fmaf(in[r * ws + k], __ldg(wl + k), s);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) {
                    const int64_t pos = tile * TM + r;
                    if (pos < count) out[pos] = row_ok[r] ? s + __ldg(m.b[L]) : INFINITY;
                }
            }
        }
    }
}

// The plain FP32 scorer for hidden widths up to 1,024 (the column-block loop
// would carry wider layers in 1,024-column blocks): 16-row tiles, thread t computes rows 8 (t / 128) .. + 7
// and output neurons cb + 8 (t % 128) .. + 7 of column block cb.  The
// transposed weights WT[k][j] of the block come into shared memory W16_KC
// input rows at a time with asynchronous 16-byte copies, double-buffered; per
// 4 input indices a thread reads its 8 rows' activations (the same for every
// lane of a warp: broadcasts) and 4 x 8 weights (one contiguous 1 KB row
// piece per warp) as 16-byte shared loads feeding 256 FMAs.  Each output
// neuron is summed over the input index in order with FMA, as in the other
// FP32 scorers (same values).
constexpr int W16_KC = 8;

template <int F, bool FROM_DESC>
__global__ void __launch_bounds__(256, 1) mlp_fp32_w16_kernel(MlpDesc m, RowSrc src, float* __restrict__ out, int ws) {
    constexpr int TM = 16, KC = W16_KC, CW = 1024;
    extern __shared__ __align__(16) float smem_w[];
    float* act0 = smem_w;                  // [TM][ws] row-major
    float* act1 = act0 + TM * ws;
    float* wst = act1 + TM * ws;           // [2][KC][CW]
    __shared__ int row_ok[TM];
    const int tid = threadIdx.x;
    const int rg = tid >> 7, cq = tid & 127;   // rows 8 rg .. + 7, neurons cb + 8 cq .. + 7
    const int64_t count = src.count_dev ? (int64_t)*src.count_dev : src.count;
    const int64_t ntiles = (count + TM - 1) / TM;
    for (int i = tid; i < 2 * TM * ws; i += 256) act0[i] = 0.f;

    // chunk kc0 of layer l, column block cb, into buffer buf: WT rows kc0 .. kc0 + KC - 1
    auto stage = [&](int l, int cb, int kc0, int buf) {
        const int fi = m.widths[l], ld = m.wt_ld[l];
        const float* wt = m.WT[l];
        float* dst = wst + buf * KC * CW;
#pragma unroll
        for (int q = 0; q < KC * CW / 4 / 256; ++q) {
            const int piece = tid + 256 * q;           // 16-byte piece
            const int kk = piece / (CW / 4), n4 = (piece % (CW / 4)) * 4;
            const bool in = kc0 + kk < fi && cb + n4 < ld;
            cp_async16(dst + kk * CW + n4, in ? wt + (size_t)(kc0 + kk) * ld + cb + n4 : wt, in ? 16 : 0);
        }
        cp_async_commit();
    };

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        float* in = act0;
        float* outb = act1;
        if (tid < TM) {
            const int64_t pos = tile * TM + tid;
            int64_t row = -1;
            if (pos < count) row = src.rows ? src.rows[pos] : pos;
            int ok = 0;
            if (row >= 0) {
                int32_t f[F];
                ok = fetch_row_features<F, FROM_DESC>(src, row, f) ? 1 : 0;
#pragma unroll
                for (int k = 0; k < F; ++k) in[tid * ws + k] = fmaf((float)f[k], __ldg(m.sa + k), -__ldg(m.sc + k));
            } else {
#pragma unroll
                for (int k = 0; k < F; ++k) in[tid * ws + k] = 0.f;
            }
            row_ok[tid] = ok;
        }
        __syncthreads();
        for (int l = 0; l + 2 < m.nw; ++l) {
            const int fi = m.widths[l], fo = m.widths[l + 1];
            const int nck = (fi + KC - 1) / KC;
            for (int cb = 0; cb < fo; cb += CW) {
                float acc[8][8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
                stage(l, cb, 0, 0);
                for (int c = 0; c < nck; ++c) {
                    if (c + 1 < nck) {
                        stage(l, cb, (c + 1) * KC, (c + 1) & 1);
                        cp_async_wait<1>();
                    } else {
                        cp_async_wait<0>();
                    }
                    __syncthreads();
                    const float* w = wst + (c & 1) * KC * CW + 8 * cq;
                    const float* a = in + (8 * rg) * ws + c * KC;
#pragma unroll
                    for (int k4 = 0; k4 < KC; k4 += 4) {
                        float av[8][4];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const float4 t = *reinterpret_cast<const float4*>(a + i * ws + k4);
                            av[i][0] = t.x; av[i][1] = t.y; av[i][2] = t.z; av[i][3] = t.w;
                        }
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const float4 w0 = *reinterpret_cast<const float4*>(w + (k4 + kk) * CW);
                            const float4 w1 = *reinterpret_cast<const float4*>(w + (k4 + kk) * CW + 4);
                            const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                            for (int i = 0; i < 8; ++i)
#pragma unroll
                                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i][kk], wv[j], acc[i][j]);
                        }
                    }
                    __syncthreads();   // buffer c & 1 is refilled two chunks later
                }
                // bias + ReLU; columns past fo are never read by the next layer
                const int c0 = cb + 8 * cq;
                if (c0 < fo) {
                    float bb[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) bb[j] = c0 + j < fo ? __ldg(m.b[l] + c0 + j) : 0.f;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        float* o = outb + (8 * rg + i) * ws + c0;
                        *reinterpret_cast<float4*>(o) =
                            make_float4(fmaxf(acc[i][0] + bb[0], 0.f), fmaxf(acc[i][1] + bb[1], 0.f),
                                        fmaxf(acc[i][2] + bb[2], 0.f), fmaxf(acc[i][3] + bb[3], 0.f));
                        *reinterpret_cast<float4*>(o + 4) =
                            make_float4(fmaxf(acc[i][4] + bb[4], 0.f), fmaxf(acc[i][5] + bb[5], 0.f),
                                        fmaxf(acc[i][6] + bb[6], 0.f), fmaxf(acc[i][7] + bb[7], 0.f));
                    }
                }
            }
            __syncthreads();
            float* t = in; in = outb; outb = t;
        }
        {
            const int L = m.nw - 2;
            const int fi = m.widths[L];
            const float* __restrict__ wl = m.W[L];
            const int warp = tid >> 5, lane = tid & 31;
            for (int r = warp; r < TM; r += 8) {
                float s = 0.f;
                for (int k = lane; k < fi; k += 32) s = fmaf(in[r * ws + k], __ldg(wl + k), s);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) {
                    const int64_t pos = tile * TM + r;
                    if (pos < count) out[pos] = row_ok[r] ? s + __ldg(m.b[L]) : INFINITY;
                }
            }
        }
    }
}

// FP32 scorer for short row lists (the near-tie re-score).  A block takes
// LIST_RB = 16 rows as two groups of 8 (threads 0-127 and 128-255); each
// thread computes two adjacent output neurons of its group (JP pairs, 256
// columns apart, for widths > 256), summing over the input index in order
// with FMA -- the same order as the plain FP32 path.  The transposed weights
// WT[k][j] stream through shared memory in chunks of kc rows by 1-D bulk
// copies (a ring of `stages`, one thread issuing), so the block never waits
// on single L2 loads; activations are stored transposed act[k][16] and read
// as broadcast 16-byte shared loads: two broadcasts and one 8-byte weight
// load feed 16 FMAs.  Features are computed by 16 lanes per row.
constexpr int LIST_RB = 16;

template <int JP, int F, bool FROM_DESC>
__global__ void __launch_bounds__(256, 1) mlp_fp32_list_kernel(MlpDesc m, RowSrc src, float* __restrict__ out,
                                                            int wmax4, int kc, int stages, int* status_word) {
    constexpr int RB = LIST_RB;
    constexpr int MAX_STAGES = 4;
    extern __shared__ __align__(16) float smem_l[];
    float* h0 = smem_l;                    // [wmax4][RB]
    float* h1 = h0 + wmax4 * RB;
    float* wbuf = h1 + wmax4 * RB;         // [stages][kc * wmax4]
    __shared__ uint64_t full[MAX_STAGES];
    __shared__ int row_ok[RB];
    __shared__ int abort_s;
    const int tid = threadIdx.x;
    const int nh = m.nw - 2;
    {
        // Every block streams all of the transposed weights, tile after tile,
        // and the FP64 re-score after this kernel reads them again.  Their
        // lines are requested into L2 all at once here (one line per thread
        // of the grid), while the selection kernel before is still running,
        // instead of one ring chunk after another from DRAM.
        const int64_t gt = (int64_t)blockIdx.x * blockDim.x + tid, gs = (int64_t)gridDim.x * blockDim.x;
        for (int l = 0; l < nh; ++l) {
            const char* p = reinterpret_cast<const char*>(m.WT[l]);
            const int64_t lines = ((int64_t)m.widths[l] * m.wt_ld[l] * 4 + 127) / 128;
            for (int64_t i = gt; i < lines; i += gs) prefetch_l2(p + i * 128);
        }
    }
    griddep_wait();   // the candidate list and its count come from the selection kernel before
    griddep_trigger();
    const int64_t count = src.count_dev ? (int64_t)*src.count_dev : src.count;
    const int64_t ntiles = (count + RB - 1) / RB;
    int nchunks = 0;
    for (int l = 0; l < nh; ++l) nchunks += (m.widths[l] + kc - 1) / kc;
    if (tid == 0) {
        for (int i = 0; i < stages; ++i) mbar_init(&full[i], 1);
        abort_s = 0;
        fence_mbar_init();
    }
    __syncthreads();
    // chunk c of the per-tile stream: layer l, rows k0 .. k0 + nk - 1 of WT[l]
    auto issue = [&](int c, int stage) {
        int l = 0, k0 = 0;
        for (l = 0; l < nh; ++l) {
            const int nc = (m.widths[l] + kc - 1) / kc;
            if (c < nc) { k0 = c * kc; break; }
            c -= nc;
        }
        const int fi = m.widths[l];
        const int nk = fi - k0 < kc ? fi - k0 : kc;
        const uint32_t bytes = (uint32_t)(nk * m.wt_ld[l] * 4);
        mbar_expect_tx(&full[stage], bytes);
        bulk_g2s(wbuf + (size_t)stage * kc * wmax4, m.WT[l] + (size_t)k0 * m.wt_ld[l], bytes, &full[stage]);
    };
    const int rg = tid >> 7;        // row group: rows 8 rg .. 8 rg + 7
    const int cp = tid & 127;       // column pair: 2 cp, 2 cp + 1 (+ 256 p)
    uint32_t used = 0;              // chunks consumed so far by this block (across tiles)
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        if (tid == 0)
            for (int c = 0; c < stages && c < nchunks; ++c) issue(c, (int)((used + c) % stages));
        {
            // half-warp h of warp w fetches row 2 w + h of the tile
            const int lane = tid & 31, r = 2 * (tid >> 5) + (lane >> 4), g = lane & 15;
            const int64_t pos = tile * RB + r;
            const int64_t row = pos < count ? (src.rows ? src.rows[pos] : pos) : -1;
            int32_t mine[(F + 15) / 16];
            const bool ok = fetch_row_features_lanes<F, 16, FROM_DESC>(src, row, g, mine);
#pragma unroll
            for (int q = 0; q < (F + 15) / 16; ++q) {
                const int k = 16 * q + g;
                if (k < F) h0[k * RB + r] = fmaf((float)mine[q], __ldg(m.sa + k), -__ldg(m.sc + k));
            }
            if (g == 0) row_ok[r] = ok ? 1 : 0;
        }
        __syncthreads();
        float* in = h0;
        float* ob = h1;
        int c = 0;
        for (int l = 0; l < nh; ++l) {
            const int fi = m.widths[l], fo = m.widths[l + 1], ld = m.wt_ld[l];
            // acc[p][e][i]: neuron 2 cp + 256 p + e, rows 2 i and 2 i + 1 of the group (FP32 pair)
            uint64_t acc[JP][2][4];
#pragma unroll
            for (int p = 0; p < JP; ++p)
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[p][0][i] = acc[p][1][i] = 0ull;
            for (int k0 = 0; k0 < fi; k0 += kc, ++c) {
                const int stage = (int)((used + c) % stages);
                const uint32_t par = ((used + c) / stages) & 1u;
                if (!mbar_wait_bounded(&full[stage], par, status_word, &abort_s, 2000000000ull)) break;
                const float* wk = wbuf + (size_t)stage * kc * wmax4;
                const int nk = fi - k0 < kc ? fi - k0 : kc;
                auto step = [&](int kk) {
                    // the 8 activations as row pairs (0,1) (2,3) (4,5) (6,7)
                    const ulonglong2* hv = reinterpret_cast<const ulonglong2*>(in + (k0 + kk) * RB + 8 * rg);
                    const ulonglong2 ha = hv[0], hb = hv[1];
                    const uint64_t hp[4] = {ha.x, ha.y, hb.x, hb.y};
#pragma unroll
                    for (int p = 0; p < JP; ++p) {
                        const int j = 2 * cp + 256 * p;
                        // columns past the padded width read column 0; their sums are never stored
                        const float2 w = *reinterpret_cast<const float2*>(wk + kk * ld + (j < ld ? j : 0));
                        const uint64_t wx = f32x2_dup(w.x), wy = f32x2_dup(w.y);
                        // two rows per instruction, each an IEEE FMA as fmaf computes it
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            f32x2_fma(acc[p][0][i], hp[i], wx);
                            f32x2_fma(acc[p][1][i], hp[i], wy);
                        }
                    }
                };
                int kk = 0;
                for (; kk + 16 <= nk; kk += 16) {
#pragma unroll
                    for (int u = 0; u < 16; ++u) step(kk + u);
                }
                for (; kk < nk; ++kk) step(kk);
                __syncthreads();   // every thread is done with this stage
                if (tid == 0 && c + stages < nchunks) issue(c + stages, stage);
            }
#pragma unroll
            for (int p = 0; p < JP; ++p) {
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int j = 2 * cp + 256 * p + e;
                    if (j < fo) {
                        const float bb = __ldg(m.b[l] + j);
                        float a[8];
#pragma unroll
                        for (int i = 0; i < 4; ++i) f32x2_unpack(acc[p][e][i], a[2 * i], a[2 * i + 1]);
                        float4* o4 = reinterpret_cast<float4*>(ob + j * RB + 8 * rg);
                        o4[0] = make_float4(fmaxf(a[0] + bb, 0.f), fmaxf(a[1] + bb, 0.f), fmaxf(a[2] + bb, 0.f),
                                            fmaxf(a[3] + bb, 0.f));
                        o4[1] = make_float4(fmaxf(a[4] + bb, 0.f), fmaxf(a[5] + bb, 0.f), fmaxf(a[6] + bb, 0.f),
                                            fmaxf(a[7] + bb, 0.f));
                    }
                }
            }
            __syncthreads();
            float* t = in; in = ob; ob = t;
        }
        used += (uint32_t)nchunks;
        {
            const int fi = m.widths[nh];
            const float* __restrict__ wl = m.W[nh];
            const int warp = tid >> 5, lane = tid & 31;
            for (int r = warp; r < RB; r += 8) {
                float s = 0.f;
                for (int k = lane; k < fi; k += 32) s = fmaf(in[k * RB + r], __ldg(wl + k), s);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) {
                    const int64_t pos = tile * RB + r;
                    if (pos < count) out[pos] = (row_ok[r] && !abort_s) ? s + __ldg(m.b[nh]) : INFINITY;
                }
            }
        }
    }
}

// FP64 reference-order scorer: one block per listed row.  With FIN (the
// argmin's last tier), the block that finishes last also makes the final
// selection: every kernel whose FP64 candidates these are (seg_state 2) takes
// the smallest (FP64 value, row) among them, as select_final_kernel would.
template <int F, bool FROM_DESC, bool FIN>
__global__ void __launch_bounds__(256) mlp_fp64_kernel(MlpDesc m, RowSrc src, double* __restrict__ out, int wmax,
                                                       SelectArgs fin) {
    extern __shared__ double smem_d[];
    double* h0 = smem_d;
    double* h1 = h0 + wmax;
    __shared__ int32_t fs[F];
    __shared__ int okf;
    griddep_wait();
    griddep_trigger();
    const int64_t count = src.count_dev ? (int64_t)*src.count_dev : src.count;
    for (int64_t pos = blockIdx.x; pos < count; pos += gridDim.x) {
        __syncthreads();
        const int64_t row = src.rows ? src.rows[pos] : pos;
        if (threadIdx.x < 32) {   // warp 0 fetches the row, its lanes sharing the logarithms
            const int lane = threadIdx.x;
            int32_t mine[(F + 31) / 32];
            const bool ok = fetch_row_features_lanes<F, 32, FROM_DESC>(src, row, lane, mine);
#pragma unroll
            for (int q = 0; q < (F + 31) / 32; ++q)
                if (32 * q + lane < F) fs[32 * q + lane] = mine[q];
            if (lane == 0) okf = ok ? 1 : 0;
        }
        __syncthreads();
        if (!okf) {
            if (threadIdx.x == 0) out[pos] = INFINITY;
            continue;
        }
        for (int k = threadIdx.x; k < F; k += blockDim.x)
            h0[k] = __ddiv_rn(__dsub_rn((double)fs[k] / 65536.0, m.mu[k]), m.sigma[k]);
        __syncthreads();
        double* in = h0;
        double* ob = h1;
        for (int l = 0; l + 1 < m.nw; ++l) {
            const int fi = m.widths[l], fo = m.widths[l + 1];
            const float* __restrict__ WT = m.WT[l];   // [fi][wt_ld]
            const bool hidden = (l + 2 < m.nw);
            for (int j = threadIdx.x; j < fo; j += blockDim.x) {
                double s = 0.0;
                for (int k = 0; k < fi; ++k) s = __dadd_rn(s, __dmul_rn((double)__ldg(WT + (size_t)k * m.wt_ld[l] + j), in[k]));
                s = __dadd_rn(s, (double)__ldg(m.b[l] + j));
                ob[j] = hidden ? (s > 0.0 ? s : 0.0) : s;
            }
            __syncthreads();
            double* t = in; in = ob; ob = t;
        }
        if (threadIdx.x == 0) out[pos] = in[0];
    }
    if constexpr (FIN) {
        __shared__ int last_s;
        __threadfence();   // this block's FP64 values are visible before it is counted
        __syncthreads();
        if (threadIdx.x == 0) last_s = atomicAdd(&fin.counters[3], 1) == (int)gridDim.x - 1;
        __syncthreads();
        if (!last_s) return;
        __threadfence();
        // candidate i of kernel k: the thread at k's first candidate decides k
        for (int64_t i = threadIdx.x; i < count; i += blockDim.x) {
            const int64_t row = fin.cand2_rows[i];
            int64_t lo = 0, hi = fin.n_kernels - 1;   // the last kernel whose first row is <= row
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (fin.off[mid] <= row) lo = mid;
                else hi = mid - 1;
            }
            const int64_t k = lo;
            if (fin.seg_state[k] != 2 || fin.seg_start[k] != i) continue;
            double bv = INFINITY;
            int64_t br = -1;
            for (int t = 0; t < fin.seg_cnt[k]; ++t) {
                const double v = out[i + t];
                const int64_t r = fin.cand2_rows[i + t];
                if (v < (double)INFINITY && (br < 0 || v < bv || (v == bv && r < br))) {
                    bv = v;
                    br = r;
                }
            }
            if (br >= 0) {
                fin.best[k] = (int32_t)(br - fin.off[k]);
                fin.best_score[k] = bv;
            }
            fin.seg_state[k] = 0;
        }
    }
}

// ---- launchers -----------------------------------------------------------------
static int act_stride(const MlpDesc& m) {
    int w = 0;
    for (int i = 0; i < m.nw; ++i) w = w > m.widths[i] ? w : m.widths[i];
    return ((w + 15) / 16) * 16 + 4;   // rows padded past the last K chunk, +4 against bank aliasing
}

template <int TM, int RPT, int F, bool FD>
static cudaError_t launch_fp32_t(const MlpDesc& m, const RowSrc& src, float* out, int grid, cudaStream_t s) {
    const int ws = act_stride(m);
    constexpr int CW = (256 / (TM / RPT)) * 8;
    const size_t smem = (size_t)(2 * TM * ws + 16 * CW) * sizeof(float);
    auto k = mlp_fp32_kernel<TM, RPT, F, FD>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, 256, smem, s>>>(m, src, out, ws);
    adv_count_launch(1);
    return cudaGetLastError();
}

template <int F, bool FD>
static cudaError_t launch_fp32_t64(const MlpDesc& m, const RowSrc& src, float* out, int grid, cudaStream_t s) {
    const int ws = act_stride(m);
    const size_t smem = (size_t)(2 * 64 * ws + 2 * T64_KC * 256) * sizeof(float);
    auto k = mlp_fp32_t64_kernel<F, FD>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, 256, smem, s>>>(m, src, out, ws);
    adv_count_launch(1);
    return cudaGetLastError();
}

template <bool FD>
static cudaError_t launch_fp32_t64_f(const MlpDesc& m, const RowSrc& src, float* out, int grid, cudaStream_t s) {
    switch (m.widths[0]) {
        case 32: return launch_fp32_t64<32, FD>(m, src, out, grid, s);
        case 33: return launch_fp32_t64<33, FD>(m, src, out, grid, s);
        case 64: return launch_fp32_t64<64, FD>(m, src, out, grid, s);
        case 128: return launch_fp32_t64<128, FD>(m, src, out, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int F, bool FD>
static cudaError_t launch_fp32_w16(const MlpDesc& m, const RowSrc& src, float* out, int grid, cudaStream_t s) {
    const int ws = act_stride(m);
    const size_t smem = (size_t)(2 * 16 * ws + 2 * W16_KC * 1024) * sizeof(float);
    auto k = mlp_fp32_w16_kernel<F, FD>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, 256, smem, s>>>(m, src, out, ws);
    adv_count_launch(1);
    return cudaGetLastError();
}

template <bool FD>
static cudaError_t launch_fp32_w16_f(const MlpDesc& m, const RowSrc& src, float* out, int grid, cudaStream_t s) {
    switch (m.widths[0]) {
        case 32: return launch_fp32_w16<32, FD>(m, src, out, grid, s);
        case 33: return launch_fp32_w16<33, FD>(m, src, out, grid, s);
        case 64: return launch_fp32_w16<64, FD>(m, src, out, grid, s);
        case 128: return launch_fp32_w16<128, FD>(m, src, out, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int TM, int RPT, bool FD>
static cudaError_t launch_fp32_f(const MlpDesc& m, const RowSrc& src, float* out, int grid, cudaStream_t s) {
    switch (m.widths[0]) {
        case 32: return launch_fp32_t<TM, RPT, 32, FD>(m, src, out, grid, s);
        case 33: return launch_fp32_t<TM, RPT, 33, FD>(m, src, out, grid, s);
        case 64: return launch_fp32_t<TM, RPT, 64, FD>(m, src, out, grid, s);
        case 128: return launch_fp32_t<TM, RPT, 128, FD>(m, src, out, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int F, bool FD>
static cudaError_t launch_fp32_list_t(const MlpDesc& m, const RowSrc& src, float* out, int grid, int wmax4,
                                      int* status_word, int blocks_per_sm, int chunk_kb, cudaStream_t s) {
    int kc = chunk_kb * 1024 / (wmax4 * 4);   // weight rows per bulk copy (16 or 32 KB chunks)
    kc = kc < 1 ? 1 : (kc > 32 ? 32 : kc);
    const size_t act = (size_t)2 * wmax4 * LIST_RB * sizeof(float);
    const size_t chunk = (size_t)kc * wmax4 * sizeof(float);
    // shared memory per block: at most 200 KB, or 100 KB when two blocks share an SM
    const size_t budget = blocks_per_sm > 1 ? 100 * 1024 : 200 * 1024;
    int stages = 3;
    while (stages > 2 && act + stages * chunk > budget) --stages;
    if (act + stages * chunk > budget) return cudaErrorInvalidValue;
    const size_t smem = act + stages * chunk;
    auto k = wmax4 <= 256 ? mlp_fp32_list_kernel<1, F, FD> : mlp_fp32_list_kernel<4, F, FD>;
    if (wmax4 > 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k, dim3(grid), dim3(256), smem, s, m, src, out, wmax4, kc, stages, status_word);
    if (e != cudaSuccess) return e;
    adv_count_launch(1);
    return cudaGetLastError();
}

static cudaError_t launch_fp32_list(const MlpDesc& m, const RowSrc& src, float* out, int num_sms,
                                    int* status_word, int blocks_per_sm, int chunk_kb, cudaStream_t s) {
    int wmax = 0;
    for (int i = 0; i < m.nw; ++i) wmax = wmax > m.widths[i] ? wmax : m.widths[i];
    const int wmax4 = (wmax + 3) / 4 * 4;
    const bool fd = (src.feat == nullptr);
    int grid = num_sms * blocks_per_sm;   // persistent 16-row blocks; longer lists loop
    if (!src.count_dev) {
        const int64_t tiles = (src.count + LIST_RB - 1) / LIST_RB;
        grid = (int)(tiles < 1 ? 1 : (tiles < grid ? tiles : grid));
    }
    switch (m.widths[0]) {
        case 32: return fd ? launch_fp32_list_t<32, true>(m, src, out, grid, wmax4, status_word, blocks_per_sm, chunk_kb, s) : launch_fp32_list_t<32, false>(m, src, out, grid, wmax4, status_word, blocks_per_sm, chunk_kb, s);
        case 33: return fd ? launch_fp32_list_t<33, true>(m, src, out, grid, wmax4, status_word, blocks_per_sm, chunk_kb, s) : launch_fp32_list_t<33, false>(m, src, out, grid, wmax4, status_word, blocks_per_sm, chunk_kb, s);
        case 64: return fd ? launch_fp32_list_t<64, true>(m, src, out, grid, wmax4, status_word, blocks_per_sm, chunk_kb, s) : launch_fp32_list_t<64, false>(m, src, out, grid, wmax4, status_word, blocks_per_sm, chunk_kb, s);
        case 128: return fd ? launch_fp32_list_t<128, true>(m, src, out, grid, wmax4, status_word, blocks_per_sm, chunk_kb, s) : launch_fp32_list_t<128, false>(m, src, out, grid, wmax4, status_word, blocks_per_sm, chunk_kb, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_mlp_fp32(const MlpDesc& m, const RowSrc& src, float* out, int num_sms, bool for_list,
                            cudaStream_t s, int* status_word, int list_blocks_per_sm, int list_chunk_kb) {
    int wmax = 0;
    for (int i = 1; i + 1 < m.nw; ++i) wmax = wmax > m.widths[i] ? wmax : m.widths[i];
    const bool fd = (src.feat == nullptr);
    if (!for_list && wmax <= 256) {
        const int64_t tiles = (src.count + 63) / 64;
        const int grid = (int)(tiles < 1 ? 1 : tiles);
        return fd ? launch_fp32_t64_f<true>(m, src, out, grid, s) : launch_fp32_t64_f<false>(m, src, out, grid, s);
    }
    if (for_list && status_word)
        return launch_fp32_list(m, src, out, num_sms, status_word, list_blocks_per_sm, list_chunk_kb, s);
    // wider models: 16-row tiles in 1,024-column blocks while the activations fit
    // (two 16-row buffers and the weight ring in 227 KB of shared memory)
    if (!for_list && (size_t)(2 * 16 * act_stride(m) + 2 * W16_KC * 1024) * sizeof(float) <= 227 * 1024) {
        const int64_t tiles = (src.count + 15) / 16;
        const int grid = (int)(tiles < 1 ? 1 : tiles);
        return fd ? launch_fp32_w16_f<true>(m, src, out, grid, s) : launch_fp32_w16_f<false>(m, src, out, grid, s);
    }
    int grid = num_sms * 2;
    if (!for_list) {
        const int64_t tiles = (src.count + 15) / 16;
        grid = (int)(tiles < 1 ? 1 : tiles);
    }
    return fd ? launch_fp32_f<16, 8, true>(m, src, out, grid, s) : launch_fp32_f<16, 8, false>(m, src, out, grid, s);
}

template <int F, bool FD>
static cudaError_t launch_fp64_t(const MlpDesc& m, const RowSrc& src, double* out, int grid, cudaStream_t s,
                                 const SelectArgs* fin) {
    int wmax = 0;
    for (int i = 0; i < m.nw; ++i) wmax = wmax > m.widths[i] ? wmax : m.widths[i];
    const size_t smem = (size_t)2 * wmax * sizeof(double);
    auto k = fin ? mlp_fp64_kernel<F, FD, true> : mlp_fp64_kernel<F, FD, false>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const SelectArgs none{};
    e = launch_pdl(k, dim3(grid), dim3(256), smem, s, m, src, out, wmax, fin ? *fin : none);
    if (e != cudaSuccess) return e;
    adv_count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_mlp_fp64(const MlpDesc& m, const RowSrc& src, double* out, int num_sms, cudaStream_t s,
                            const SelectArgs* fin) {
    int grid = num_sms * 4;
    if (!src.count_dev) grid = (int)(src.count < grid ? (src.count < 1 ? 1 : src.count) : grid);
    const bool fd = (src.feat == nullptr);
    switch (m.widths[0]) {
        case 32: return fd ? launch_fp64_t<32, true>(m, src, out, grid, s, fin) : launch_fp64_t<32, false>(m, src, out, grid, s, fin);
        case 33: return fd ? launch_fp64_t<33, true>(m, src, out, grid, s, fin) : launch_fp64_t<33, false>(m, src, out, grid, s, fin);
        case 64: return fd ? launch_fp64_t<64, true>(m, src, out, grid, s, fin) : launch_fp64_t<64, false>(m, src, out, grid, s, fin);
        case 128: return fd ? launch_fp64_t<128, true>(m, src, out, grid, s, fin) : launch_fp64_t<128, false>(m, src, out, grid, s, fin);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace adv
