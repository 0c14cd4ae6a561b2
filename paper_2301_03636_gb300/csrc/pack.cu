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
            pad_copy_kernel<<<grid_for(L.npad[l]), 256, 0, s>>>(master + L.layer_b_off[l], fo, L.npad[l],
                                                               reinterpret_cast<float*>(P + L.p_bias_off[l]));
            adv_count_launch(2);
        }
        adv_count_launch(1);
    }
    const int last = L.n_layers - 1;
    pad_copy_kernel<<<grid_for(L.npad[last - 1]), 256, 0, s>>>(master + L.layer_w_off[last], L.widths[last],
                                                              L.npad[last - 1],
                                                              reinterpret_cast<float*>(P + L.p_wout_pad));
    adv_count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_set_params(const ModelLayout& L, uint8_t* P, const float* params, const double* mu,
                              const double* sigma, cudaStream_t s) {
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

}  // namespace adv
