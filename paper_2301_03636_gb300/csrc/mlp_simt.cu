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
        const int4* p = reinterpret_cast<const int4*>(src.feat + (size_t)row * F);
#pragma unroll
        for (int j = 0; j < F / 4; ++j) {
            const int4 v = __ldg(p + j);
            f[4 * j] = v.x; f[4 * j + 1] = v.y; f[4 * j + 2] = v.z; f[4 * j + 3] = v.w;
        }
        return !(src.status && src.status[row]);
    }
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

// FP64 reference-order scorer: one block per listed row.
template <int F, bool FROM_DESC>
__global__ void __launch_bounds__(256) mlp_fp64_kernel(MlpDesc m, RowSrc src, double* __restrict__ out, int wmax) {
    extern __shared__ double smem_d[];
    double* h0 = smem_d;
    double* h1 = h0 + wmax;
    __shared__ int32_t fs[F];
    __shared__ int okf;
    const int64_t count = src.count_dev ? (int64_t)*src.count_dev : src.count;
    for (int64_t pos = blockIdx.x; pos < count; pos += gridDim.x) {
        __syncthreads();
        const int64_t row = src.rows ? src.rows[pos] : pos;
        if (threadIdx.x == 0) {
            int32_t f[F];
            okf = fetch_row_features<F, FROM_DESC>(src, row, f) ? 1 : 0;
#pragma unroll
            for (int k = 0; k < F; ++k) fs[k] = f[k];
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
            const float* __restrict__ WT = m.WT[l];   // [fi][fo]
            const bool hidden = (l + 2 < m.nw);
            for (int j = threadIdx.x; j < fo; j += blockDim.x) {
                double s = 0.0;
                for (int k = 0; k < fi; ++k) s = __dadd_rn(s, __dmul_rn((double)__ldg(WT + (size_t)k * fo + j), in[k]));
                s = __dadd_rn(s, (double)__ldg(m.b[l] + j));
                ob[j] = hidden ? (s > 0.0 ? s : 0.0) : s;
            }
            __syncthreads();
            double* t = in; in = ob; ob = t;
        }
        if (threadIdx.x == 0) out[pos] = in[0];
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

template <int TM, int RPT, bool FD>
static cudaError_t launch_fp32_f(const MlpDesc& m, const RowSrc& src, float* out, int grid, cudaStream_t s) {
    switch (m.widths[0]) {
        case 32: return launch_fp32_t<TM, RPT, 32, FD>(m, src, out, grid, s);
        case 64: return launch_fp32_t<TM, RPT, 64, FD>(m, src, out, grid, s);
        case 128: return launch_fp32_t<TM, RPT, 128, FD>(m, src, out, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_mlp_fp32(const MlpDesc& m, const RowSrc& src, float* out, int num_sms, bool for_list,
                            cudaStream_t s) {
    int wmax = 0;
    for (int i = 1; i + 1 < m.nw; ++i) wmax = wmax > m.widths[i] ? wmax : m.widths[i];
    const bool fd = (src.feat == nullptr);
    if (!for_list && wmax <= 256) {
        const int64_t tiles = (src.count + 63) / 64;
        const int grid = (int)(tiles < 1 ? 1 : tiles);
        return fd ? launch_fp32_f<64, 8, true>(m, src, out, grid, s) : launch_fp32_f<64, 8, false>(m, src, out, grid, s);
    }
    if (wmax <= 256) {   // latency-oriented: 16-row tiles, 2 rows x 8 columns per thread
        const int grid = num_sms * 4;
        return fd ? launch_fp32_f<16, 2, true>(m, src, out, grid, s) : launch_fp32_f<16, 2, false>(m, src, out, grid, s);
    }
    int grid = num_sms * 2;
    if (!for_list) {
        const int64_t tiles = (src.count + 15) / 16;
        grid = (int)(tiles < 1 ? 1 : tiles);
    }
    return fd ? launch_fp32_f<16, 8, true>(m, src, out, grid, s) : launch_fp32_f<16, 8, false>(m, src, out, grid, s);
}

template <int F, bool FD>
static cudaError_t launch_fp64_t(const MlpDesc& m, const RowSrc& src, double* out, int grid, cudaStream_t s) {
    int wmax = 0;
    for (int i = 0; i < m.nw; ++i) wmax = wmax > m.widths[i] ? wmax : m.widths[i];
    const size_t smem = (size_t)2 * wmax * sizeof(double);
    auto k = mlp_fp64_kernel<F, FD>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, 256, smem, s>>>(m, src, out, wmax);
    adv_count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_mlp_fp64(const MlpDesc& m, const RowSrc& src, double* out, int num_sms, cudaStream_t s) {
    int grid = num_sms * 4;
    if (!src.count_dev) grid = (int)(src.count < grid ? (src.count < 1 ? 1 : src.count) : grid);
    const bool fd = (src.feat == nullptr);
    switch (m.widths[0]) {
        case 32: return fd ? launch_fp64_t<32, true>(m, src, out, grid, s) : launch_fp64_t<32, false>(m, src, out, grid, s);
        case 64: return fd ? launch_fp64_t<64, true>(m, src, out, grid, s) : launch_fp64_t<64, false>(m, src, out, grid, s);
        case 128: return fd ? launch_fp64_t<128, true>(m, src, out, grid, s) : launch_fp64_t<128, false>(m, src, out, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace adv
