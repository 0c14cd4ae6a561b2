// Descriptor validation and integer feature extraction (a1-a3).
//
// Fig. 2 of arXiv 2301.03636 feeds every generated variant through "Feature
// Extraction" before the trained model; the paper does not list its
// features, so the feature set here is this library's own (documented in
// include/advisor.h): Q16.16 binary logarithms of the loop-nest counts, the
// work, the mapped bytes (Sec. 4.1.2) and the parallelism, their signed
// differences, and the variant parameters of Sec. 4.1.3.
//
// One thread per descriptor row; the 128-byte row is read with eight 16-byte
// vector loads.  Outputs: int32 features [n][F] (bit-exact), and/or the
// standardised 16-bit activations of the tensor-core scorer written straight
// into its shared-memory image layout (128-row tiles, 64-column slabs of
// 128-byte rows, 128B swizzle), so that the scorer moves them with one bulk
// copy per slab.
#include "features.cuh"
#include "mlp.cuh"

namespace adv {

// Convert 8 standardised values to 16-bit and pack them into a uint4.
template <int FMT>
__device__ __forceinline__ uint4 pack8(const float (&z)[8]) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if constexpr (FMT == 1) {
            __nv_bfloat162 h = __floats2bfloat162_rn(z[2 * i], z[2 * i + 1]);
            w[i] = *reinterpret_cast<uint32_t*>(&h);
        } else {
            __half2 h = __floats2half2_rn(fminf(fmaxf(z[2 * i], -65504.f), 65504.f),
                                          fminf(fmaxf(z[2 * i + 1], -65504.f), 65504.f));
            w[i] = *reinterpret_cast<uint32_t*>(&h);
        }
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// Write one row of the E4M3 activation image: one slab per 128 features
// (128-byte rows of 8-bit values, 16-byte chunk c = features 16c..16c+15 of
// row r at chunk position c ^ (r % 8)), standardised values times inv_s
// (the reciprocal of the first layer's per-tensor activation scale).
template <int F>
__device__ __forceinline__ void write_x_row_e4m3(uint8_t* x_img, int nslab, int64_t row, const int32_t (&f)[F],
                                                 bool valid_row, const float* __restrict__ sa,
                                                 const float* __restrict__ sc, float inv_s) {
    const int64_t tile = row / ADV_TILE_M;
    const uint32_t r = (uint32_t)(row % ADV_TILE_M);
    uint8_t* tile_base = x_img + (size_t)tile * nslab * ADV_X_SLAB_BYTES;
#pragma unroll
    for (int s = 0; s < (F + 127) / 128; ++s) {
        if (s >= nslab) break;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            uint32_t w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float z[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int k = s * 128 + c * 16 + 4 * i + e;
                    z[e] = (valid_row && k < F)
                               ? fmaf((float)f[k < F ? k : 0], __ldg(sa + (k < F ? k : 0)), -__ldg(sc + (k < F ? k : 0))) * inv_s
                               : 0.f;
                }
                w[i] = e4m3x2(z[0], z[1]) | (e4m3x2(z[2], z[3]) << 16);
            }
            *reinterpret_cast<uint4*>(tile_base + (size_t)s * ADV_X_SLAB_BYTES + sw128_offset(r, c)) =
                make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// Write one row of the 16-bit activation image: row `row` of the tile grid,
// kpad = nslab * 64 columns, features beyond F (and rows beyond n) are zero.
template <int F, int FMT>
__device__ __forceinline__ void write_x_row(uint8_t* x_img, int nslab, int64_t row, const int32_t (&f)[F],
                                            bool valid_row, const float* __restrict__ sa,
                                            const float* __restrict__ sc, uint16_t* x_rm = nullptr) {
    const int64_t tile = row / ADV_TILE_M;
    const uint32_t r = (uint32_t)(row % ADV_TILE_M);
    uint8_t* tile_base = x_img + (size_t)tile * nslab * ADV_X_SLAB_BYTES;
#pragma unroll
    for (int s = 0; s < (F + 63) / 64; ++s) {
        if (s >= nslab) break;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            float z[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int k = s * 64 + c * 8 + e;
                z[e] = (valid_row && k < F) ? fmaf((float)f[k < F ? k : 0], __ldg(sa + (k < F ? k : 0)),
                                                   -__ldg(sc + (k < F ? k : 0)))
                                            : 0.f;
            }
            const uint4 pk = pack8<FMT>(z);
            *reinterpret_cast<uint4*>(tile_base + (size_t)s * ADV_X_SLAB_BYTES + sw128_offset(r, c)) = pk;
            if constexpr (F % 8 == 0)
                if (x_rm && valid_row && s * 64 + c * 8 < F)
                    *reinterpret_cast<uint4*>(x_rm + (size_t)row * F + s * 64 + c * 8) = pk;
        }
    }
}


template <int F, int FMT>
__global__ void __launch_bounds__(256) extract_kernel(ExtractArgs a) {
    griddep_wait();
    griddep_trigger();
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= a.n_rows_padded) return;
    int32_t f[F];
    bool valid = false;
    if (row < a.n_rows) {
        int64_t d[16];
        load_desc(a.desc, row, d);
        const uint32_t st = validate_row(d);
        valid = (st == 0);
        if (valid) {
            row_features<F>(d, f);
        } else {
#pragma unroll
            for (int j = 0; j < F; ++j) f[j] = 0;
        }
        if (a.status) a.status[row] = (uint8_t)st;
        if (a.feat) {
            if constexpr (F % 4 == 0) {
                int4* dst = reinterpret_cast<int4*>(a.feat + (size_t)row * F);
#pragma unroll
                for (int j = 0; j < F / 4; ++j) dst[j] = make_int4(f[4 * j], f[4 * j + 1], f[4 * j + 2], f[4 * j + 3]);
            } else {   // rows not 16-byte aligned (F = 33)
#pragma unroll
                for (int j = 0; j < F; ++j) a.feat[(size_t)row * F + j] = f[j];
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < F; ++j) f[j] = 0;
    }
    if constexpr (FMT == 3) {
        if (a.x_img) write_x_row_e4m3<F>(a.x_img, a.nslab, row, f, valid, a.sa, a.sc, 1.f / __ldg(a.x8_scale));
    } else if constexpr (FMT != 0) {
        if (a.x_img) write_x_row<F, FMT>(a.x_img, a.nslab, row, f, valid, a.sa, a.sc);
    }
}

// Gathered extraction for the FP16 middle tier of the near-tie re-score:
// image position p holds descriptor row rows[p] for p < n = min(*count_dev,
// n_rows); positions n .. the next multiple of 128 are zero rows.  n is read
// on the device (an earlier kernel wrote it), so the launch covers the
// capacity with a grid-stride loop.  No status or int32 features are written.
template <int F, int FMT>
__global__ void __launch_bounds__(128) extract_list_kernel(ExtractArgs a) {
    int64_t n = *a.count_dev;
    n = n < 0 ? 0 : (n < a.n_rows ? n : a.n_rows);
    const int64_t padded = (n + ADV_TILE_M - 1) / ADV_TILE_M * ADV_TILE_M;
    const float inv_s = FMT == 3 ? 1.f / __ldg(a.x8_scale) : 1.f;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < padded;
         p += (int64_t)gridDim.x * blockDim.x) {
        int32_t f[F];
        bool valid = false;
        if (p < n) {
            int64_t d[16];
            load_desc(a.desc, a.rows[p], d);
            valid = validate_row(d) == 0;
            if (valid) row_features<F>(d, f);
        }
        if (!valid) {
#pragma unroll
            for (int j = 0; j < F; ++j) f[j] = 0;
        }
        if constexpr (FMT == 3) write_x_row_e4m3<F>(a.x_img, a.nslab, p, f, valid, a.sa, a.sc, inv_s);
        else write_x_row<F, FMT>(a.x_img, a.nslab, p, f, valid, a.sa, a.sc);
    }
}

// int32 features -> 16-bit standardised activation image.
template <int F, int FMT>
__global__ void __launch_bounds__(128) standardize_kernel(const int32_t* __restrict__ feat,
                                                          const uint8_t* __restrict__ status, int64_t n_rows,
                                                          int64_t n_rows_padded, uint8_t* x_img, int nslab,
                                                          const float* __restrict__ sa,
                                                          const float* __restrict__ sc,
                                                          const float* __restrict__ x8_scale, uint16_t* x_rm) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n_rows_padded) return;
    int32_t f[F];
    const bool valid = row < n_rows;
    if (valid) {
        if constexpr (F % 4 == 0) {
            const int4* src = reinterpret_cast<const int4*>(feat + (size_t)row * F);
#pragma unroll
            for (int j = 0; j < F / 4; ++j) {
                const int4 v = __ldg(src + j);
                f[4 * j] = v.x; f[4 * j + 1] = v.y; f[4 * j + 2] = v.z; f[4 * j + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < F; ++j) f[j] = __ldg(feat + (size_t)row * F + j);
        }
    } else {
#pragma unroll
        for (int j = 0; j < F; ++j) f[j] = 0;
    }
    (void)status;  // invalid rows are scored +inf by the scorer's epilogue
    if constexpr (FMT == 3) write_x_row_e4m3<F>(x_img, nslab, row, f, valid, sa, sc, 1.f / __ldg(x8_scale));
    else write_x_row<F, FMT>(x_img, nslab, row, f, valid, sa, sc, x_rm);
}

// The same image (and the optional row-major copy), one 16-byte chunk of 8
// features per thread: the 8 * nslab chunks of a row are consecutive threads,
// so that a warp's loads and stores cover whole rows (a thread per row would
// touch 32 rows with every access).  16-bit formats, F % 8 == 0, 16-byte
// aligned feat.  Same values as write_x_row.
template <int F, int FMT>
__global__ void __launch_bounds__(256) standardize_chunks_kernel(const int32_t* __restrict__ feat, int64_t n_rows,
                                                                 int64_t n_rows_padded, uint8_t* x_img, int nslab,
                                                                 const float* __restrict__ sa,
                                                                 const float* __restrict__ sc, uint16_t* x_rm) {
    static_assert(F % 8 == 0, "whole 8-feature chunks");
    const int cpr = nslab * 8;   // 16-byte chunks per image row
    const int64_t total = n_rows_padded * cpr;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t / cpr;
        const int c = (int)(t - row * cpr);   // features 8c .. 8c + 7
        const int k0 = 8 * c;
        const bool live = row < n_rows && k0 < F;
        float z[8];
        if (live) {
            const int4* src = reinterpret_cast<const int4*>(feat + (size_t)row * F + k0);
            const int4 u = __ldg(src), v = __ldg(src + 1);
            const int32_t q[8] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 8; ++e) z[e] = fmaf((float)q[e], __ldg(sa + k0 + e), -__ldg(sc + k0 + e));
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) z[e] = 0.f;
        }
        const uint4 pk = pack8<FMT>(z);
        const int64_t tile = row / ADV_TILE_M;
        const uint32_t r = (uint32_t)(row % ADV_TILE_M);
        *reinterpret_cast<uint4*>(x_img + ((size_t)tile * nslab + (c >> 3)) * ADV_X_SLAB_BYTES +
                                  sw128_offset(r, (uint32_t)(c & 7))) = pk;
        if (x_rm && live) *reinterpret_cast<uint4*>(x_rm + (size_t)row * F + k0) = pk;
    }
}

// Mean and population standard deviation of feature/65536 per column over
// the valid rows, in FP64, with a fixed reduction order.
__global__ void __launch_bounds__(256) fit_standardizer_kernel(const int32_t* __restrict__ feat,
                                                               const uint8_t* __restrict__ status,
                                                               int64_t n_rows, int F, double* mu,
                                                               double* sigma) {
    __shared__ double red[256];
    __shared__ long long cnt_s[256];
    const int j = blockIdx.x;
    double s = 0.0;
    long long c = 0;
    for (int64_t r = threadIdx.x; r < n_rows; r += blockDim.x) {
        if (status && status[r]) continue;
        s += (double)feat[(size_t)r * F + j] / 65536.0;
        ++c;
    }
    red[threadIdx.x] = s;
    cnt_s[threadIdx.x] = c;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            red[threadIdx.x] += red[threadIdx.x + w];
            cnt_s[threadIdx.x] += cnt_s[threadIdx.x + w];
        }
        __syncthreads();
    }
    const long long cnt = cnt_s[0];
    const double mean = cnt ? red[0] / (double)cnt : 0.0;
    __syncthreads();
    double v = 0.0;
    for (int64_t r = threadIdx.x; r < n_rows; r += blockDim.x) {
        if (status && status[r]) continue;
        const double e = (double)feat[(size_t)r * F + j] / 65536.0 - mean;
        v += e * e;
    }
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double sd = cnt ? sqrt(red[0] / (double)cnt) : 0.0;
        mu[j] = mean;
        sigma[j] = sd > 0.0 ? sd : 1.0;
    }
}

// ---- host launchers ------------------------------------------------------------
template <int F>
static cudaError_t launch_extract_f(const ExtractArgs& a, int fmt, cudaStream_t s, int block) {
    const int64_t rows = a.n_rows_padded;
    const unsigned grid = (unsigned)((rows + block - 1) / block);
    if (grid == 0) return cudaSuccess;
    auto k = fmt == 1 ? extract_kernel<F, 1> : fmt == 2 ? extract_kernel<F, 2> : fmt == 3 ? extract_kernel<F, 3>
                                                                                   : extract_kernel<F, 0>;
    const cudaError_t e = launch_pdl(k, dim3(grid), dim3(block), 0, s, a);
    if (e != cudaSuccess) return e;
    adv_count_launch(1);
    return cudaGetLastError();
}

template <int F>
static cudaError_t launch_extract_list_f(const ExtractArgs& a, int fmt, int num_sms, cudaStream_t s) {
    const int64_t blocks = (a.n_rows + ADV_TILE_M - 1) / ADV_TILE_M;   // 128 threads per block
    const unsigned grid = (unsigned)(blocks < 8 * num_sms ? blocks : 8 * num_sms);
    if (grid == 0) return cudaSuccess;
    if (fmt == 1) extract_list_kernel<F, 1><<<grid, 128, 0, s>>>(a);
    else if (fmt == 2) extract_list_kernel<F, 2><<<grid, 128, 0, s>>>(a);
    else if (fmt == 3) extract_list_kernel<F, 3><<<grid, 128, 0, s>>>(a);
    else return cudaErrorInvalidValue;
    adv_count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_extract_list(const ExtractArgs& a, int F, int fmt, int num_sms, cudaStream_t s) {
    if (!a.rows || !a.count_dev || !a.x_img) return cudaErrorInvalidValue;
    switch (F) {
        case 32: return launch_extract_list_f<32>(a, fmt, num_sms, s);
        case 33: return launch_extract_list_f<33>(a, fmt, num_sms, s);
        case 64: return launch_extract_list_f<64>(a, fmt, num_sms, s);
        case 128: return launch_extract_list_f<128>(a, fmt, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_extract(const ExtractArgs& a, int F, int fmt, cudaStream_t s, int block) {
    if (block != 64 && block != 128 && block != 256) return cudaErrorInvalidValue;
    switch (F) {
        case 32: return launch_extract_f<32>(a, fmt, s, block);
        case 33: return launch_extract_f<33>(a, fmt, s, block);
        case 64: return launch_extract_f<64>(a, fmt, s, block);
        case 128: return launch_extract_f<128>(a, fmt, s, block);
        default: return cudaErrorInvalidValue;
    }
}

template <int F>
static cudaError_t launch_standardize_f(const int32_t* feat, const uint8_t* status, int64_t n, int64_t npad,
                                        uint8_t* x_img, int nslab, const float* sa, const float* sc, int fmt,
                                        const float* x8_scale, uint16_t* x_rm, cudaStream_t s) {
    const unsigned grid = (unsigned)((npad + 127) / 128);
    if (grid == 0) return cudaSuccess;
    if (fmt == 3 && !x8_scale) return cudaErrorInvalidValue;
    if (x_rm && (fmt == 3 || F % 8 != 0 || ((uintptr_t)x_rm & 15) != 0)) return cudaErrorInvalidValue;
    if constexpr (F % 8 == 0) {
        if (fmt != 3 && ((uintptr_t)feat & 15) == 0) {   // a lane per 16-byte chunk
            const int64_t total = npad * nslab * 8;
            const unsigned g2 = (unsigned)((total + 255) / 256 < 65535 * 16 ? (total + 255) / 256 : 65535 * 16);
            if (fmt == 1)
                standardize_chunks_kernel<F, 1><<<g2, 256, 0, s>>>(feat, n, npad, x_img, nslab, sa, sc, x_rm);
            else
                standardize_chunks_kernel<F, 2><<<g2, 256, 0, s>>>(feat, n, npad, x_img, nslab, sa, sc, x_rm);
            adv_count_launch(1);
            return cudaGetLastError();
        }
    }
    if (fmt == 1)
        standardize_kernel<F, 1><<<grid, 128, 0, s>>>(feat, status, n, npad, x_img, nslab, sa, sc, x8_scale, x_rm);
    else if (fmt == 3)
        standardize_kernel<F, 3><<<grid, 128, 0, s>>>(feat, status, n, npad, x_img, nslab, sa, sc, x8_scale, x_rm);
    else
        standardize_kernel<F, 2><<<grid, 128, 0, s>>>(feat, status, n, npad, x_img, nslab, sa, sc, x8_scale, x_rm);
    adv_count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_standardize(const int32_t* feat, const uint8_t* status, int64_t n, int64_t npad, uint8_t* x_img,
                               int nslab, const float* sa, const float* sc, int F, int fmt, cudaStream_t s,
                               const float* x8_scale, uint16_t* x_rm) {
    switch (F) {
        case 32: return launch_standardize_f<32>(feat, status, n, npad, x_img, nslab, sa, sc, fmt, x8_scale, x_rm, s);
        case 33: return launch_standardize_f<33>(feat, status, n, npad, x_img, nslab, sa, sc, fmt, x8_scale, x_rm, s);
        case 64: return launch_standardize_f<64>(feat, status, n, npad, x_img, nslab, sa, sc, fmt, x8_scale, x_rm, s);
        case 128: return launch_standardize_f<128>(feat, status, n, npad, x_img, nslab, sa, sc, fmt, x8_scale, x_rm, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fit_standardizer(const int32_t* feat, const uint8_t* status, int64_t n, int F, double* mu,
                                    double* sigma, cudaStream_t s) {
    fit_standardizer_kernel<<<F, 256, 0, s>>>(feat, status, n, F, mu, sigma);
    adv_count_launch(1);
    return cudaGetLastError();
}

}  // namespace adv
