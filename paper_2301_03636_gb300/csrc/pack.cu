// Parameter packing: FP32 master parameters -> the derived copies the
// scorers read (16-bit weight images in the tensor-core shared-memory order,
// a transposed FP32 copy, zero-padded biases and output row, FP32
// standardisation constants).
#include "mlp.cuh"
#include "pack.cuh"

namespace adv {

// Weight image of hidden layer l: slab k holds rows n = 0..npad-1 of
// W[n][64k .. 64k+63] as 16-bit values, 128 bytes per row, 16-byte chunk c
// of row n stored at chunk position c ^ (n % 8).  Padding is zero.
__global__ void pack_w16_kernel(const float* __restrict__ W, int fo, int fi, int npad, int kpad,
                                uint8_t* __restrict__ img_bf16, uint8_t* __restrict__ img_f16) {
    const int64_t total = (int64_t)npad * kpad / 8;   // 8-element chunks
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(c / (kpad / 8));
        const int kc = (int)(c % (kpad / 8));          // chunk index along K
        const int slab = kc / 8, chunk = kc % 8;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = kc * 8 + e;
            v[e] = (n < fo && k < fi) ? W[(size_t)n * fi + k] : 0.f;
        }
        uint32_t wb[4], wh[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __nv_bfloat162 hb = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
            __half2 hh = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
            wb[i] = *reinterpret_cast<uint32_t*>(&hb);
            wh[i] = *reinterpret_cast<uint32_t*>(&hh);
        }
        const size_t off = (size_t)slab * npad * ADV_SLAB_ROW_BYTES + sw128_offset((uint32_t)n, (uint32_t)chunk);
        *reinterpret_cast<uint4*>(img_bf16 + off) = make_uint4(wb[0], wb[1], wb[2], wb[3]);
        *reinterpret_cast<uint4*>(img_f16 + off) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
    }
}

// max |x| over n values, folded into *amax_bits by atomicMax on the bit
// pattern (non-negative floats order like their bit patterns).
__global__ void amax_kernel(const float* __restrict__ x, int64_t n, unsigned* amax_bits) {
    __shared__ float red[32];
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(x[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) atomicMax(amax_bits, __float_as_uint(m));
    }
}

// E4M3 weight image of a hidden layer: slab k holds rows n = 0..npad8-1 of
// W[n][128k .. 128k+127] / s as 8-bit values, 128 bytes per row, 16-byte
// chunk c of row n at chunk position c ^ (n % 8); s = amax / 448 (per-tensor
// scale, exact amax).  Padding is zero.
__global__ void pack_w8_kernel(const float* __restrict__ W, int fo, int fi, int npad8, int nslab8,
                               const unsigned* __restrict__ amax_bits, uint8_t* __restrict__ img) {
    const float amax = __uint_as_float(*amax_bits);
    const float inv = amax > 0.f ? ADV_E4M3_MAX / amax : 1.f;
    const int kchunks = nslab8 * 8;                     // 16-element chunks per row
    const int64_t total = (int64_t)npad8 * kchunks;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(c / kchunks);
        const int kc = (int)(c % kchunks);
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = kc * 16 + 4 * i + e;
                v[e] = (n < fo && k < fi) ? W[(size_t)n * fi + k] * inv : 0.f;
            }
            w[i] = e4m3x2(v[0], v[1]) | (e4m3x2(v[2], v[3]) << 16);
        }
        const size_t off = (size_t)(kc / 8) * npad8 * ADV_SLAB_ROW_BYTES + sw128_offset((uint32_t)n, (uint32_t)(kc % 8));
        *reinterpret_cast<uint4*>(img + off) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Activation scales from the calibration amax values, in place: scale =
// amax / 448 (1 when the amax is 0); then mark the model calibrated.
__global__ void fp8_finalize_kernel(float* fp8, int n_hidden) {
    if (threadIdx.x == 0) {
        for (int l = 0; l < n_hidden; ++l) {
            const float amax = __uint_as_float(reinterpret_cast<unsigned*>(fp8)[ADV_FP8_X_SCALE + l]);
            fp8[ADV_FP8_X_SCALE + l] = amax > 0.f ? amax / ADV_E4M3_MAX : 1.f;
        }
        fp8[ADV_FP8_CALIBRATED] = 1.f;
    }
}

// WT[k][n] = W[n][k], rows of ld >= fo floats, zero beyond fo.
__global__ void transpose_kernel(const float* __restrict__ W, int fo, int fi, int ld, float* __restrict__ WT) {
    const int64_t total = (int64_t)ld * fi;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(i / ld), n = (int)(i % ld);
        WT[i] = n < fo ? W[(size_t)n * fi + k] : 0.f;
    }
}

__global__ void pad_copy_kernel(const float* __restrict__ src, int n, int npad, float* __restrict__ dst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += gridDim.x * blockDim.x)
        dst[i] = i < n ? src[i] : 0.f;
}

__global__ void stdz_kernel(const double* __restrict__ mu, const double* __restrict__ sigma, int F,
                            float* __restrict__ sa, float* __restrict__ sc, double* __restrict__ mu_out,
                            double* __restrict__ sigma_out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < F) {
        const double s = sigma[k];
        sa[k] = (float)(1.0 / (65536.0 * s));
        sc[k] = (float)(mu[k] / s);
        mu_out[k] = mu[k];
        sigma_out[k] = s;
    }
}

__global__ void copy_f32_kernel(const float* __restrict__ src, float* __restrict__ dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

__global__ void zero_f32_kernel(float* __restrict__ dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = 0.f;
}

static int grid_for(int64_t n) {
    const int64_t g = (n + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

// Rebuild every derived copy from the master parameters already in the block.
cudaError_t launch_repack(const ModelLayout& L, uint8_t* P, cudaStream_t s) {
    const float* master = reinterpret_cast<const float*>(P + L.p_master);
    for (int l = 0; l < L.n_layers; ++l) {
        const int fi = L.widths[l], fo = L.widths[l + 1];
        const float* W = master + L.layer_w_off[l];
        const int ld = (fo + 3) / 4 * 4;
        transpose_kernel<<<grid_for((int64_t)ld * fi), 256, 0, s>>>(W, fo, fi, ld,
                                                                   reinterpret_cast<float*>(P + L.p_wT[l]));
        if (l < L.n_hidden) {
            const int64_t chunks = (int64_t)L.npad[l] * L.kpad[l] / 8;
            pack_w16_kernel<<<grid_for(chunks), 256, 0, s>>>(W, fo, fi, L.npad[l], L.kpad[l], P + L.p_w16[0][l],
                                                            P + L.p_w16[1][l]);
            pad_copy_kernel<<<grid_for(L.npad8[l]), 256, 0, s>>>(master + L.layer_b_off[l], fo, L.npad8[l],
                                                                reinterpret_cast<float*>(P + L.p_bias_off[l]));
            adv_count_launch(2);
            if (!L.tc_ok) {   // E4M3 copy for the layer-by-layer path
                unsigned* amax = reinterpret_cast<unsigned*>(P + L.p_fp8) + ADV_FP8_W_AMAX + l;
                cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(unsigned), s);
                if (e != cudaSuccess) return e;
                amax_kernel<<<grid_for((int64_t)fo * fi), 256, 0, s>>>(W, (int64_t)fo * fi, amax);
                pack_w8_kernel<<<grid_for((int64_t)L.npad8[l] * L.nslab8[l] * 8), 256, 0, s>>>(
                    W, fo, fi, L.npad8[l], L.nslab8[l], amax, P + L.p_w8[l]);
                adv_count_launch(2);
            }
        }
        adv_count_launch(1);
    }
    const int last = L.n_layers - 1;
    pad_copy_kernel<<<grid_for(L.npad8[last - 1]), 256, 0, s>>>(master + L.layer_w_off[last], L.widths[last],
                                                               L.npad8[last - 1],
                                                              reinterpret_cast<float*>(P + L.p_wout_pad));
    adv_count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_set_params(const ModelLayout& L, uint8_t* P, const float* params, const double* mu,
                              const double* sigma, cudaStream_t s) {
    // new parameters: the FP8 activation scales must be calibrated again
    cudaError_t e0 = cudaMemsetAsync(P + L.p_fp8, 0, 32 * sizeof(float), s);
    if (e0 != cudaSuccess) return e0;
    copy_f32_kernel<<<grid_for(L.n_params), 256, 0, s>>>(params, reinterpret_cast<float*>(P + L.p_master),
                                                         L.n_params);
    stdz_kernel<<<(L.F + 127) / 128, 128, 0, s>>>(mu, sigma, L.F, reinterpret_cast<float*>(P + L.p_stdz_a),
                                                  reinterpret_cast<float*>(P + L.p_stdz_c),
                                                  reinterpret_cast<double*>(P + L.p_mu),
                                                  reinterpret_cast<double*>(P + L.p_sigma));
    zero_f32_kernel<<<grid_for(2 * L.n_params), 256, 0, s>>>(reinterpret_cast<float*>(P + L.p_adam_m),
                                                            L.n_params);
    zero_f32_kernel<<<grid_for(2 * L.n_params), 256, 0, s>>>(reinterpret_cast<float*>(P + L.p_adam_v),
                                                            L.n_params);
    adv_count_launch(4);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_repack(L, P, s);
}

cudaError_t launch_copy_f32(const float* src, float* dst, int64_t n, cudaStream_t s) {
    copy_f32_kernel<<<grid_for(n), 256, 0, s>>>(src, dst, n);
    adv_count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_fp8_calibrate(const ModelLayout& L, uint8_t* P, const float* const* acts, int64_t n,
                                 cudaStream_t s) {
    float* fp8 = reinterpret_cast<float*>(P + L.p_fp8);
    cudaError_t e = cudaMemsetAsync(fp8 + ADV_FP8_X_SCALE, 0, ADV_MAX_LAYERS * sizeof(float), s);
    if (e != cudaSuccess) return e;
    for (int l = 0; l < L.n_hidden; ++l) {
        const int64_t cnt = n * L.widths[l];
        amax_kernel<<<grid_for(cnt), 256, 0, s>>>(acts[l], cnt, reinterpret_cast<unsigned*>(fp8) + ADV_FP8_X_SCALE + l);
        adv_count_launch(1);
    }
    fp8_finalize_kernel<<<1, 32, 0, s>>>(fp8, L.n_hidden);
    adv_count_launch(1);
    return cudaGetLastError();
}

}  // namespace adv
