// Training mode with 16-bit operands on the tensor cores (Sec. 3 training
// mode, Sec. 5 Exp. 3 network): the same forward, MSE loss on ln runtime,
// hand-written backward and Adam update as the FP32 path in train.cu, with
// every layer GEMM taking BF16 (or FP16) operands and accumulating in FP32:
//   forward   C_l = H_{l-1} W_l^T (GEMM), H_l = 16-bit(ReLU(C_l + b_l)),
//             y = H_L w_out + b_out (FP32 dot per row);
//   backward  dZ_L = 16-bit(dy w_out^T masked by H_L > 0),
//             dW_l = dZ_l^T H_{l-1}  (GEMM, K = rows, split over CTAs, the
//                                     partial sums added in a fixed order),
//             db_l = column sums of dZ_l (fixed split order),
//             dZ_{l-1} = 16-bit(dZ_l W_l masked by H_{l-1} > 0);
//   Adam on the FP32 master weights, then the derived copies are rebuilt.
// The GEMMs are this library's tcgen05 kernels (gemm_tc.cu): the generic
// TMA-fed GEMM, reading the row-major operands in place as K-major or
// MN-major, for the weight gradients; the persistent ReLU-backward kernel for
// dZ_{l-1} with the bias-gradient column sums in its epilogue.  For models
// the fused scorer covers, the forward is that scorer (mlp_tc.cu) saving the
// 16-bit activations.  The bias and output-row gradient partials are summed in
// one launch at the end of the backward.  Activations are kept in 16 bits
// between layers, so the masks use the stored 16-bit values (positive iff the
// FP32 pre-activation rounded to a positive value).
#include <algorithm>
#include <type_traits>

#include "pack.cuh"
#include "train.cuh"

namespace adv {

namespace {

constexpr int TC_SPLIT_ROWS = 1024;   // rows per partial sum of the column reductions

int grid_n(int64_t n, int block = 256) {
    const int64_t g = (n + block - 1) / block;
    return (int)(g < 1 ? 1 : (g > 8192 ? 8192 : g));
}

template <typename T>
__device__ __forceinline__ T to16(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 to16<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half to16<__half>(float x) { return __float2half_rn(x); }
template <typename T>
__device__ __forceinline__ float from16(T x);
template <>
__device__ __forceinline__ float from16<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <>
__device__ __forceinline__ float from16<__half>(__half x) { return __half2float(x); }

template <typename T>
__global__ void cvt16_kernel(const float* __restrict__ src, T* __restrict__ dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = to16<T>(src[i]);
}

// x[r][k] = 16-bit(f[r][k] * sa[k] - sc[k]), the standardisation of the scorers
template <typename T>
__global__ void stdz16_kernel(const int32_t* __restrict__ feat, int64_t n, int F, const float* __restrict__ sa,
                              const float* __restrict__ sc, T* __restrict__ x) {
    const int64_t total = n * F;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(i % F);
        x[i] = to16<T>(fmaf((float)feat[i], __ldg(sa + k), -__ldg(sc + k)));
    }
}

template <typename T>
__global__ void bias_relu16_kernel(const float* __restrict__ c, int64_t n, int w, const float* __restrict__ b,
                                   T* __restrict__ h) {
    const int64_t total = n * w;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        h[i] = to16<T>(fmaxf(c[i] + __ldg(b + (int)(i % w)), 0.f));
}

// y[r] = sum_j h[r][j] w_out[j] + b_out, one warp per row, fixed order
template <typename T>
__global__ void out_dot16_kernel(const T* __restrict__ h, int64_t n, int w, const float* __restrict__ wo,
                                 const float* __restrict__ bo, float* __restrict__ y) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
        float s = 0.f;
        for (int j = lane; j < w; j += 32) s = fmaf(from16<T>(h[r * w + j]), __ldg(wo + j), s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) y[r] = s + __ldg(bo);
    }
}

// dz[r][j] = 16-bit(dy[r] w_out[j]) where h[r][j] > 0, else 0
template <typename T>
__global__ void dz_last16_kernel(const float* __restrict__ dy, const float* __restrict__ wo, const T* __restrict__ h,
                                 int64_t n, int w, T* __restrict__ dz) {
    const int64_t total = n * w;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        dz[i] = to16<T>(from16<T>(h[i]) > 0.f ? dy[i / w] * __ldg(wo + (int)(i % w)) : 0.f);
}

// dz[r][j] = 16-bit(c[r][j]) where h[r][j] > 0, else 0
template <typename T>
__global__ void mask16_kernel(const float* __restrict__ c, const T* __restrict__ h, int64_t n, int w,
                              T* __restrict__ dz) {
    const int64_t total = n * w;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        dz[i] = to16<T>(from16<T>(h[i]) > 0.f ? c[i] : 0.f);
}

// part[s][j] = sum over the rows of split s of wt[r] x[r][j] (wt null: 1), in row order
template <typename T>
__global__ void colsum16_kernel(const T* __restrict__ x, const float* __restrict__ wt, int64_t n, int w,
                                float* __restrict__ part) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.y * TC_SPLIT_ROWS;
    if (j >= w) return;
    const int64_t r1 = r0 + TC_SPLIT_ROWS < n ? r0 + TC_SPLIT_ROWS : n;
    float s = 0.f;
    for (int64_t r = r0; r < r1; ++r) s = fmaf(wt ? wt[r] : 1.f, from16<T>(x[r * w + j]), s);
    part[(size_t)blockIdx.y * w + j] = s;
}

// part[s] = sum of v over the rows of split s
__global__ void rowsum_kernel(const float* __restrict__ v, int64_t n, float* __restrict__ part) {
    __shared__ float red[32];
    const int64_t r0 = (int64_t)blockIdx.x * TC_SPLIT_ROWS;
    const int64_t r1 = r0 + TC_SPLIT_ROWS < n ? r0 + TC_SPLIT_ROWS : n;
    float s = 0.f;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) s += v[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        part[blockIdx.x] = t;
    }
}

// out[j] = sum over s of part[s][j]: eight interleaved split sequences per
// column (s = y, y + 8, ...) summed in split order, then combined in y order.
// Block (32, 8), one block per 32 columns.
__global__ void __launch_bounds__(1024) splitsum16_kernel(const float* __restrict__ part, int splits, int w,
                                                          float* __restrict__ out) {
    // 32 columns x 32 split lanes: lane y sums splits y, y + 32, ... in order,
    // then the lanes are added in order
    __shared__ float red[32][33];
    const int j = blockIdx.x * 32 + threadIdx.x;
    float s = 0.f;
    if (j < w) {
        int i = threadIdx.y;
        for (; i + 96 < splits; i += 128) {
            const float a0 = part[(size_t)i * w + j], a1 = part[(size_t)(i + 32) * w + j];
            const float a2 = part[(size_t)(i + 64) * w + j], a3 = part[(size_t)(i + 96) * w + j];
            s = (((s + a0) + a1) + a2) + a3;
        }
        for (; i < splits; i += 32) s += part[(size_t)i * w + j];
    }
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && j < w) {
        float t = 0.f;
#pragma unroll 8
        for (int y = 0; y < 32; ++y) t += red[y][threadIdx.x];
        out[j] = t;
    }
}

// Several split sums in one launch: job j sums parts[j][i][c] over i < splits[j]
// into out[j][c] for c < w[j], in the order of splitsum16_kernel.
constexpr int SS_MAX_JOBS = ADV_MAX_LAYERS + 2;
struct SplitSumJobs {
    const float* part[SS_MAX_JOBS];
    float* out[SS_MAX_JOBS];
    float* out2[SS_MAX_JOBS];   // nullable: a second copy of the result
    float div[SS_MAX_JOBS];     // the sum is divided by this
    int splits[SS_MAX_JOBS], w[SS_MAX_JOBS];
    int first_block[SS_MAX_JOBS + 1];   // blocks of job j: first_block[j] .. first_block[j + 1] - 1
    int n;
};

__global__ void __launch_bounds__(1024) splitsum_jobs_kernel(const __grid_constant__ SplitSumJobs jb) {
    __shared__ float red[32][33];
    int j = 0;
    while (j + 1 < jb.n && (int)blockIdx.x >= jb.first_block[j + 1]) ++j;
    const int w = jb.w[j], splits = jb.splits[j];
    const float* __restrict__ part = jb.part[j];
    const int c = ((int)blockIdx.x - jb.first_block[j]) * 32 + threadIdx.x;
    float s = 0.f;
    if (c < w) {
        int i = threadIdx.y;
        for (; i + 96 < splits; i += 128) {
            const float a0 = part[(size_t)i * w + c], a1 = part[(size_t)(i + 32) * w + c];
            const float a2 = part[(size_t)(i + 64) * w + c], a3 = part[(size_t)(i + 96) * w + c];
            s = (((s + a0) + a1) + a2) + a3;
        }
        for (; i < splits; i += 32) s += part[(size_t)i * w + c];
    }
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && c < w) {
        float t = 0.f;
#pragma unroll 8
        for (int y = 0; y < 32; ++y) t += red[y][threadIdx.x];
        t = t / jb.div[j];
        jb.out[j][c] = t;
        if (jb.out2[j]) jb.out2[j][c] = t;
    }
}

struct SplitSums {
    SplitSumJobs jb{};
    void add(const float* part, int splits, int w, float* out, float div = 1.f, float* out2 = nullptr) {
        jb.part[jb.n] = part;
        jb.out[jb.n] = out;
        jb.out2[jb.n] = out2;
        jb.div[jb.n] = div;
        jb.splits[jb.n] = splits;
        jb.w[jb.n] = w;
        jb.first_block[jb.n + 1] = jb.first_block[jb.n] + (w + 31) / 32;
        ++jb.n;
    }
    void launch(cudaStream_t s) const {
        if (jb.n == 0) return;
        splitsum_jobs_kernel<<<jb.first_block[jb.n], dim3(32, 32), 0, s>>>(jb);
        adv_count_launch(1);
    }
};

void splitsum(const float* part, int splits, int w, float* out, cudaStream_t s) {
    splitsum16_kernel<<<(w + 31) / 32, dim3(32, 32), 0, s>>>(part, splits, w, out);
}

// ---- vectorised forms: 8 consecutive columns (16 bytes of 16-bit values) per
// thread, 32-bit indices; used when w % 8 == 0, 256 % (w / 8) == 0 and the
// matrix has fewer than 2^31 elements.
constexpr int VEC_ROWS = 256;   // rows per block of the fused column sums

template <typename T>
__device__ __forceinline__ uint32_t pack2(float lo, float hi);
template <>
__device__ __forceinline__ uint32_t pack2<__nv_bfloat16>(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}
template <>
__device__ __forceinline__ uint32_t pack2<__half>(float lo, float hi) {
    __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}
template <typename T>
__device__ __forceinline__ void unpack8(const uint4 u, float (&f)[8]) {
    const T* h = reinterpret_cast<const T*>(&u);
#pragma unroll
    for (int i = 0; i < 8; ++i) f[i] = from16<T>(h[i]);
}
__device__ __forceinline__ void load8f(const float* p, float (&f)[8]) {
    const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
    f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w; f[4] = b.x; f[5] = b.y; f[6] = b.z; f[7] = b.w;
}
template <typename T>
__device__ __forceinline__ uint4 pack8(const float (&f)[8]) {
    return make_uint4(pack2<T>(f[0], f[1]), pack2<T>(f[2], f[3]), pack2<T>(f[4], f[5]), pack2<T>(f[6], f[7]));
}

bool vec_ok(int64_t n, int w) { return w % 8 == 0 && 256 % (w / 8) == 0 && n * w < ((int64_t)1 << 31); }

template <typename T>
__global__ void bias_relu16_vec_kernel(const float* __restrict__ c, int n, int w, const float* __restrict__ b,
                                       T* __restrict__ h) {
    const int w8 = w >> 3, total = n * w8;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < total; v += gridDim.x * blockDim.x) {
        const int j = (v % w8) << 3;
        float x[8], bb[8];
        load8f(c + (size_t)v * 8, x);
        load8f(b + j, bb);
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fmaxf(x[i] + bb[i], 0.f);
        reinterpret_cast<uint4*>(h)[v] = pack8<T>(x);
    }
}

template <typename T>
__global__ void stdz16_vec_kernel(const int32_t* __restrict__ feat, int n, int F, const float* __restrict__ sa,
                                  const float* __restrict__ sc, T* __restrict__ x) {
    const int f8 = F >> 3, total = n * f8;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < total; v += gridDim.x * blockDim.x) {
        const int k = (v % f8) << 3;
        const int4 a = reinterpret_cast<const int4*>(feat)[2 * v], bq = reinterpret_cast<const int4*>(feat)[2 * v + 1];
        const int q[8] = {a.x, a.y, a.z, a.w, bq.x, bq.y, bq.z, bq.w};
        float z[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) z[i] = fmaf((float)q[i], __ldg(sa + k + i), -__ldg(sc + k + i));
        reinterpret_cast<uint4*>(x)[v] = pack8<T>(z);
    }
}

// Last hidden layer, for a block of VEC_ROWS rows: dZ[r][j] = 16-bit(dy[r]
// w_out[j]) where h[r][j] > 0, else 0; plus the block's column sums in row
// order: part0[block][j] = sum_r dZ[r][j] (the bias gradient, of the stored
// 16-bit dZ as the GEMMs read it) and part1[block][j] = sum_r dy[r] h[r][j]
// (the output-row gradient).  With labels (the MSE loss fused in), dy[r] =
// (y[r] - t[r]) / n is computed here instead of read, and the block also
// writes part_loss[block] = sum_r (y[r] - t[r])^2 / 2 and part_dsum[block] =
// sum_r dy[r] (the output bias's gradient), rows in order.
template <typename T>
__global__ void __launch_bounds__(256) dz_last_colsum16_kernel(const float* __restrict__ dy,
                                                               const float* __restrict__ wo, const T* __restrict__ h,
                                                               int n, int w, T* __restrict__ dz,
                                                               float* __restrict__ part0, float* __restrict__ part1,
                                                               const float* __restrict__ y,
                                                               const float* __restrict__ labels,
                                                               float* __restrict__ part_loss,
                                                               float* __restrict__ part_dsum) {
    __shared__ float red0[256 * 8], red1[256 * 8];
    __shared__ float redl[256], redd[256];
    const int w8 = w >> 3;
    const int cg = threadIdx.x % w8;            // column group: columns 8 cg .. 8 cg + 7
    const int rl = threadIdx.x / w8;            // row lane
    const int lanes = 256 / w8;                 // rows per pass
    const int r0 = blockIdx.x * VEC_ROWS;
    float s0[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, s1[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float sl = 0.f, sd = 0.f;                   // this row lane's loss and dy sums (column group 0)
    float wq[8];
    load8f(wo + 8 * cg, wq);
    const int r_end = r0 + VEC_ROWS < n ? r0 + VEC_ROWS : n;
    constexpr int U = 8;   // rows whose loads are issued together (the sums still take them in order)
    for (int rb = r0 + rl; rb < r_end; rb += U * lanes) {
        uint4 hq[U];
        float ya[U], yb[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int r = rb + u * lanes;
            if (r < r_end) {
                hq[u] = reinterpret_cast<const uint4*>(h)[r * w8 + cg];
                if (labels) {
                    ya[u] = y[r];
                    yb[u] = labels[r];
                } else {
                    ya[u] = dy[r];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int r = rb + u * lanes;
            if (r >= r_end) break;
            float hv[8], o[8];
            unpack8<T>(hq[u], hv);
            float d;
            if (labels) {
                const float e = ya[u] - yb[u];
                d = e / (float)n;
                if (cg == 0) {
                    sl += 0.5f * e * e;
                    sd += d;
                }
            } else {
                d = ya[u];
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) o[i] = hv[i] > 0.f ? d * wq[i] : 0.f;
            const uint4 pk = pack8<T>(o);
            reinterpret_cast<uint4*>(dz)[r * w8 + cg] = pk;
            float q[8];
            unpack8<T>(pk, q);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                s0[i] += q[i];
                s1[i] = fmaf(d, hv[i], s1[i]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        red0[threadIdx.x * 8 + i] = s0[i];
        red1[threadIdx.x * 8 + i] = s1[i];
    }
    redl[threadIdx.x] = sl;
    redd[threadIdx.x] = sd;
    __syncthreads();
    // row lanes of each column summed in lane order
    for (int t = threadIdx.x; t < w; t += 256) {
        const int g = t >> 3, i = t & 7;
        float a0 = 0.f, a1 = 0.f;
        for (int l = 0; l < lanes; ++l) {
            a0 += red0[(l * w8 + g) * 8 + i];
            a1 += red1[(l * w8 + g) * 8 + i];
        }
        part0[(size_t)blockIdx.x * w + t] = a0;
        part1[(size_t)blockIdx.x * w + t] = a1;
    }
    if (labels && threadIdx.x == 0) {   // the row lanes' sums (column group 0 threads) in lane order
        float al = 0.f, ad = 0.f;
        for (int l = 0; l < lanes; ++l) {
            al += redl[l * w8];
            ad += redd[l * w8];
        }
        part_loss[blockIdx.x] = al;
        part_dsum[blockIdx.x] = ad;
    }
}

}  // namespace

// ---- the 16-bit training step -------------------------------------------------
namespace {

template <typename T>
struct Tc {
    const ModelLayout& L;
    const TrainLayout& T_;
    uint8_t* TW;
    const MlpDesc& md;
    int* status_word;
    static constexpr int fmt = std::is_same<T, __nv_bfloat16>::value ? 1 : 0;   // instruction-descriptor code

    T* x16() const { return reinterpret_cast<T*>(TW + T_.x16); }
    T* h16(int l) const { return reinterpret_cast<T*>(TW + T_.h16[l]); }
    T* w16(int l) const { return reinterpret_cast<T*>(TW + T_.w16[l]); }
    T* dz16(int i) const { return reinterpret_cast<T*>(TW + T_.dz16[i]); }
    float* c32() const { return reinterpret_cast<float*>(TW + T_.c32); }
    float* part() const { return reinterpret_cast<float*>(TW + T_.part); }
    float* bias_part() const { return reinterpret_cast<float*>(TW + T_.bias_part); }
    float* y() const { return reinterpret_cast<float*>(TW + T_.act[L.n_layers]); }
    float* dy() const { return reinterpret_cast<float*>(TW + T_.dA); }

    // C[M][N] = sum_k A(m,k) B(n,k) on the tensor cores (see TcGemm)
    cudaError_t gemm(const T* A, int64_t lda, int a_mn, const T* B, int64_t ldb, int b_mn, int64_t M, int64_t N,
                     int64_t K, void* C, int64_t ldc, int c16, int splits, cudaStream_t s) const {
        TcGemm g{};
        g.A = reinterpret_cast<const uint16_t*>(A);
        g.lda = lda;
        g.a_mn = a_mn;
        g.B = reinterpret_cast<const uint16_t*>(B);
        g.ldb = ldb;
        g.b_mn = b_mn;
        g.M = M;
        g.N = N;
        g.K = K;
        g.C = C;
        g.ldc = ldc;
        g.c16 = c16;
        g.part = part();
        g.splits = splits;
        g.fmt = fmt;
        g.status_word = status_word;
        g.timeout_ns = 2000000000ull;
        return launch_gemm_tc(g, s);
    }
    // dZ[n][fi] = 16-bit(dZ_above W) masked by h > 0 (ReLU backward), plus the
    // bias-gradient partials colpart[tile][fi] of the stored dZ, 128-row tiles
    cudaError_t gemm_mask(const T* dz_above, int fo, const T* W, int fi, const T* h, int64_t n, T* dz, float* colpart,
                          cudaStream_t s) const {
        TcGemm g{};
        g.A = reinterpret_cast<const uint16_t*>(dz_above);
        g.lda = fo;
        g.a_mn = 0;
        g.B = reinterpret_cast<const uint16_t*>(W);
        g.ldb = fi;
        g.b_mn = 1;
        g.M = n;
        g.N = fi;
        g.K = fo;
        g.C = dz;
        g.ldc = fi;
        g.c16 = 1;
        g.splits = 1;
        g.fmt = fmt;
        g.status_word = status_word;
        g.timeout_ns = 2000000000ull;
        g.mask_h = reinterpret_cast<const uint16_t*>(h);
        g.colpart = colpart;
        return launch_gemm_tc(g, s);
    }
    // split-K factor of the weight-gradient GEMMs: about 1,024 rows per split, at
    // most the partial-sum buffer's splits
    int dw_splits(int64_t n) const {
        const int64_t sp = (n + 1023) / 1024;
        return (int)(sp < 1 ? 1 : (sp > T_.splits ? T_.splits : sp));
    }
    // input of hidden layer l: the standardised features or the previous layer's output
    const T* in16(int l) const { return l == 0 ? x16() : h16(l - 1); }

    cudaError_t forward(const int32_t* feat, int64_t n, cudaStream_t s) const {
        for (int l = 0; l < L.n_hidden; ++l) {
            const int64_t cnt = (int64_t)L.widths[l] * L.widths[l + 1];
            cvt16_kernel<T><<<grid_n(cnt), 256, 0, s>>>(md.W[l], w16(l), cnt);
        }
        if (vec_ok(n, L.F) && L.F % 8 == 0)
            stdz16_vec_kernel<T><<<grid_n(n * L.F / 8), 256, 0, s>>>(feat, (int)n, L.F, md.sa, md.sc, x16());
        else
            stdz16_kernel<T><<<grid_n(n * L.F), 256, 0, s>>>(feat, n, L.F, md.sa, md.sc, x16());
        adv_count_launch(L.n_hidden + 1);
        for (int l = 0; l < L.n_hidden; ++l) {
            const int fi = L.widths[l], fo = L.widths[l + 1];
            // C[n][fo] = In[n][fi] W[fo][fi]^T: A = In (K-major), B = W (K-major)
            cudaError_t e = gemm(in16(l), fi, 0, w16(l), fi, 0, n, fo, fi, c32(), fo, 0, 1, s);
            if (e != cudaSuccess) return e;
            if (vec_ok(n, fo))
                bias_relu16_vec_kernel<T><<<grid_n(n * fo / 8), 256, 0, s>>>(c32(), (int)n, fo, md.b[l], h16(l));
            else
                bias_relu16_kernel<T><<<grid_n(n * fo), 256, 0, s>>>(c32(), n, fo, md.b[l], h16(l));
            adv_count_launch(1);
        }
        const int wl = L.widths[L.n_hidden];
        out_dot16_kernel<T><<<grid_n(n * 32), 256, 0, s>>>(h16(L.n_hidden - 1), n, wl, md.W[L.n_hidden],
                                                           md.b[L.n_hidden], y());
        adv_count_launch(1);
        return cudaGetLastError();
    }

    // dL/dy in dy(); gradient (master layout) into grad
    // Whether backward() takes the vectorised path, which can fuse the MSE loss in.
    bool vec_path(int64_t n) const {
        bool vec = n <= T_.rows;
        for (int l = 0; l < L.n_hidden; ++l) vec = vec && vec_ok(n, L.widths[l + 1]);
        return vec;
    }

    // dL/dy in dy(); gradient (master layout) into grad.  With labels (vectorised
    // path only), dL/dy of the MSE loss is computed from y() and the labels inside
    // the backward, and the loss goes to the loss buffer (and d_loss).
    cudaError_t backward(int64_t n, float* grad, cudaStream_t s, const float* labels = nullptr,
                         float* loss = nullptr, float* d_loss = nullptr) const {
        if (labels) return vec_path(n) ? backward_vec(n, grad, s, labels, loss, d_loss) : cudaErrorInvalidValue;
        bool vec = true;
        for (int l = 0; l < L.n_hidden; ++l) vec = vec && vec_ok(n, L.widths[l + 1]);
        // the fused reductions' partials fit the bias-partial region (sized for the workspace's rows)
        vec = vec && n <= T_.rows;
        if (vec) return backward_vec(n, grad, s);
        const int splits = (int)((n + TC_SPLIT_ROWS - 1) / TC_SPLIT_ROWS);
        const int H = L.n_hidden;
        const int wl = L.widths[H];
        // output layer: grad w_out = sum_r dy[r] H_L[r], grad b_out = sum_r dy[r]
        dim3 cg((unsigned)((wl + 127) / 128), (unsigned)splits);
        colsum16_kernel<T><<<cg, 128, 0, s>>>(h16(H - 1), dy(), n, wl, part());
        splitsum(part(), splits, wl, grad + L.layer_w_off[H], s);
        rowsum_kernel<<<splits, 256, 0, s>>>(dy(), n, part());
        splitsum(part(), splits, 1, grad + L.layer_b_off[H], s);
        dz_last16_kernel<T><<<grid_n(n * wl), 256, 0, s>>>(dy(), md.W[H], h16(H - 1), n, wl, dz16(0));
        adv_count_launch(5);
        int cur = 0;
        for (int l = H - 1; l >= 0; --l) {
            const int fi = L.widths[l], fo = L.widths[l + 1];
            // dW[fo][fi] = dZ[n][fo]^T In[n][fi]: A = dZ, B = In, both MN-major (K = the rows)
            cudaError_t e = gemm(dz16(cur), fo, 1, in16(l), fi, 1, fo, fi, n, grad + L.layer_w_off[l], fi, 0,
                                 dw_splits(n), s);
            if (e != cudaSuccess) return e;
            dim3 bg((unsigned)((fo + 127) / 128), (unsigned)splits);
            colsum16_kernel<T><<<bg, 128, 0, s>>>(dz16(cur), nullptr, n, fo, part());
            splitsum(part(), splits, fo, grad + L.layer_b_off[l], s);
            adv_count_launch(2);
            if (l == 0) break;
            // dIn[n][fi] = dZ[n][fo] W[fo][fi]: A = dZ (K-major), B = W (MN-major)
            e = gemm(dz16(cur), fo, 0, w16(l), fi, 1, n, fi, fo, c32(), fi, 0, 1, s);
            if (e != cudaSuccess) return e;
            mask16_kernel<T><<<grid_n(n * fi), 256, 0, s>>>(c32(), h16(l - 1), n, fi, dz16(cur ^ 1));
            adv_count_launch(1);
            cur ^= 1;
        }
        return cudaGetLastError();
    }

    // The same backward with the dZ producers also reducing the bias (and
    // output-row) gradients per 256-row block.
    cudaError_t backward_vec(int64_t n, float* grad, cudaStream_t s, const float* labels = nullptr,
                             float* loss = nullptr, float* d_loss = nullptr) const {
        const int blocks = (int)((n + VEC_ROWS - 1) / VEC_ROWS);
        const int nsplit = (int)((n + TC_SPLIT_ROWS - 1) / TC_SPLIT_ROWS);
        const int H = L.n_hidden;
        const int wl = L.widths[H];
        // the column-sum partials live in their own region and are summed in one
        // launch at the end: the last hidden layer's (bias p0, output row p1), the
        // output bias's (p2), then one array per lower hidden layer
        float* p0 = bias_part();
        float* p1 = p0 + (size_t)blocks * wl;
        float* p2 = p1 + (size_t)blocks * wl;   // output bias: nsplit partials, or blocks with labels
        float* pls = p2 + std::max<int64_t>(nsplit, blocks);   // the loss's partials (labels)
        float* pl = pls + blocks;
        const int64_t per_layer_rows = std::max<int64_t>((n + 127) / 128, 1024);
        SplitSums sums;
        if (labels) {
            dz_last_colsum16_kernel<T><<<blocks, 256, 0, s>>>(nullptr, md.W[H], h16(H - 1), (int)n, wl, dz16(0), p0,
                                                              p1, y(), labels, pls, p2);
            adv_count_launch(1);
            sums.add(p1, blocks, wl, grad + L.layer_w_off[H]);
            sums.add(p2, blocks, 1, grad + L.layer_b_off[H]);
            sums.add(pls, blocks, 1, loss, (float)n, d_loss);
        } else {
            dz_last_colsum16_kernel<T><<<blocks, 256, 0, s>>>(dy(), md.W[H], h16(H - 1), (int)n, wl, dz16(0), p0, p1,
                                                              nullptr, nullptr, nullptr, nullptr);
            rowsum_kernel<<<nsplit, 256, 0, s>>>(dy(), n, p2);
            adv_count_launch(2);
            sums.add(p1, blocks, wl, grad + L.layer_w_off[H]);
            sums.add(p2, nsplit, 1, grad + L.layer_b_off[H]);
        }
        sums.add(p0, blocks, wl, grad + L.layer_b_off[H - 1]);
        int cur = 0;
        for (int l = H - 1; l >= 0; --l) {
            const int fi = L.widths[l], fo = L.widths[l + 1];
            cudaError_t e = gemm(dz16(cur), fo, 1, in16(l), fi, 1, fo, fi, n, grad + L.layer_w_off[l], fi, 0,
                                 dw_splits(n), s);
            if (e != cudaSuccess) return e;
            if (l == 0) break;
            // dZ of layer l - 1 = (dZ W) masked by h > 0, rounded to 16 bits in the
            // GEMM's epilogue, with the bias gradient's per-tile column sums
            int parts = 0;
            e = launch_dgrad_mask(reinterpret_cast<const uint16_t*>(dz16(cur)), fo,
                                  reinterpret_cast<const uint16_t*>(w16(l)), fi,
                                  reinterpret_cast<const uint16_t*>(h16(l - 1)), n,
                                  reinterpret_cast<uint16_t*>(dz16(cur ^ 1)), pl, per_layer_rows * fi, &parts, fmt,
                                  status_word, s);
            if (e == cudaErrorNotSupported) {   // shapes outside the persistent kernel: the generic GEMM
                e = gemm_mask(dz16(cur), fo, w16(l), fi, h16(l - 1), n, dz16(cur ^ 1), pl, s);
                parts = (int)((n + 127) / 128);
            }
            if (e != cudaSuccess) return e;
            sums.add(pl, parts, fi, grad + L.layer_b_off[l - 1]);
            pl += (size_t)per_layer_rows * fi;
            cur ^= 1;
        }
        sums.launch(s);
        return cudaGetLastError();
    }
};

}  // namespace

// One launch per step: for every hidden layer the scorer's swizzled BF16 and
// FP16 images (as pack_w16_kernel), the row-major copy in the training format,
// the zero-padded bias, and the padded output row.
struct PackTrainArgs {
    const float* W[ADV_MAX_LAYERS];
    const float* b[ADV_MAX_LAYERS];
    int fo[ADV_MAX_LAYERS], fi[ADV_MAX_LAYERS], npad[ADV_MAX_LAYERS], kpad[ADV_MAX_LAYERS], npad8[ADV_MAX_LAYERS];
    uint8_t* img_bf16[ADV_MAX_LAYERS];
    uint8_t* img_f16[ADV_MAX_LAYERS];
    void* rm[ADV_MAX_LAYERS];
    float* bias_pad[ADV_MAX_LAYERS];
    int64_t start[ADV_MAX_LAYERS + 1];   // first chunk of each layer; start[n_hidden] = the output row's
    const float* w_out;
    int w_out_n, w_out_pad_n;
    float* wout_pad;
    int n_hidden;
};

template <typename T>
__global__ void pack_train_kernel(const __grid_constant__ PackTrainArgs p) {
    const int64_t total = p.start[p.n_hidden] + p.w_out_pad_n;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (int64_t)gridDim.x * blockDim.x) {
        if (c >= p.start[p.n_hidden]) {   // the padded output row
            const int j = (int)(c - p.start[p.n_hidden]);
            p.wout_pad[j] = j < p.w_out_n ? p.w_out[j] : 0.f;
            continue;
        }
        int l = 0;
        while (c >= p.start[l + 1]) ++l;
        const int64_t cl = c - p.start[l];
        const int fo = p.fo[l], fi = p.fi[l];
        const int64_t img_chunks = (int64_t)p.npad[l] * p.kpad[l] / 8;
        if (cl >= img_chunks) {           // the padded bias
            const int j = (int)(cl - img_chunks);
            p.bias_pad[l][j] = j < fo ? p.b[l][j] : 0.f;
            continue;
        }
        const int n = (int)(cl / (p.kpad[l] / 8));
        const int kc = (int)(cl % (p.kpad[l] / 8));
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = kc * 8 + e;
            v[e] = (n < fo && k < fi) ? p.W[l][(size_t)n * fi + k] : 0.f;
        }
        uint32_t wb[4], wh[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __nv_bfloat162 hb = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
            __half2 hh = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
            wb[i] = *reinterpret_cast<uint32_t*>(&hb);
            wh[i] = *reinterpret_cast<uint32_t*>(&hh);
        }
        const size_t off = (size_t)(kc / 8) * p.npad[l] * ADV_SLAB_ROW_BYTES + sw128_offset((uint32_t)n, (uint32_t)(kc % 8));
        *reinterpret_cast<uint4*>(p.img_bf16[l] + off) = make_uint4(wb[0], wb[1], wb[2], wb[3]);
        *reinterpret_cast<uint4*>(p.img_f16[l] + off) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
        if (n < fo) {
            T* rm = reinterpret_cast<T*>(p.rm[l]) + (size_t)n * fi;
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (kc * 8 + e < fi) rm[kc * 8 + e] = to16<T>(v[e]);
        }
    }
}

template <typename T>
static cudaError_t forward_fused(const ModelLayout& L, const TrainLayout& Tl, uint8_t* TW, const MlpDesc& md,
                                 int fmt, const int32_t* feat, int64_t n, const FusedFwd& ff, cudaStream_t s) {
    PackTrainArgs p{};
    p.n_hidden = L.n_hidden;
    int64_t at = 0;
    for (int l = 0; l < L.n_hidden; ++l) {
        p.W[l] = md.W[l];
        p.b[l] = md.b[l];
        p.fo[l] = L.widths[l + 1];
        p.fi[l] = L.widths[l];
        p.npad[l] = L.npad[l];
        p.kpad[l] = L.kpad[l];
        p.npad8[l] = L.npad8[l];
        p.img_bf16[l] = ff.img16[0][l];
        p.img_f16[l] = ff.img16[1][l];
        p.rm[l] = TW + Tl.w16[l];
        p.bias_pad[l] = ff.bias_pad[l];
        p.start[l] = at;
        at += (int64_t)L.npad[l] * L.kpad[l] / 8 + L.npad8[l];
    }
    p.start[L.n_hidden] = at;
    p.w_out = md.W[L.n_hidden];
    p.w_out_n = L.widths[L.n_hidden];
    p.w_out_pad_n = L.npad8[L.n_hidden - 1];
    p.wout_pad = ff.wout_pad;
    const int64_t total = at + p.w_out_pad_n;
    pack_train_kernel<T><<<grid_n(total), 256, 0, s>>>(p);
    T* x16 = reinterpret_cast<T*>(TW + Tl.x16);
    adv_count_launch(1);
    const int64_t npad_rows = ((n + ADV_TILE_M - 1) / ADV_TILE_M) * ADV_TILE_M;
    // the scorer's input image and, when F allows 16-byte rows, the row-major
    // copy that the first layer's weight gradient reads, in one pass
    const bool rm_fused = L.F % 8 == 0 && (Tl.x16 % 16) == 0;
    if (!rm_fused) {
        stdz16_kernel<T><<<grid_n(n * L.F), 256, 0, s>>>(feat, n, L.F, md.sa, md.sc, x16);
        adv_count_launch(1);
    }
    cudaError_t e = launch_standardize(feat, nullptr, n, npad_rows, ff.x_img, L.nslab[0], md.sa, md.sc, L.F,
                                       fmt == 1 ? 1 : 2, s, nullptr,
                                       rm_fused ? reinterpret_cast<uint16_t*>(x16) : nullptr);
    if (e != cudaSuccess) return e;
    TcArgs a = ff.tc;
    a.x_img = ff.x_img;
    a.n_rows = n;
    a.n_tiles = (int)(npad_rows / ADV_TILE_M);
    a.status = nullptr;
    a.scores = reinterpret_cast<float*>(TW + Tl.act[L.n_layers]);
    a.fmt = fmt == 1 ? 1 : 0;   // instruction-descriptor code
    a.use_tma_save = 1;
    for (int l = 0; l < L.n_hidden; ++l) {
        a.w_img[l] = ff.img16[fmt == 1 ? 0 : 1][l];
        a.save_act[l] = TW + Tl.h16[l];
        a.save_ld[l] = L.widths[l + 1];
        // the layers before the last are stored from the scorer's shared-memory image by TMA
        if (l + 1 < L.n_hidden &&
            !encode_rows_map(&a.tm_save[l], a.save_act[l], a.save_ld[l], n, ADV_TILE_M, fmt == 1 ? 1 : 2))
            a.use_tma_save = 0;
    }
    return launch_mlp_tc(a, ff.num_sms, s, ff.ctas);
}

// Whether the fused forward covers this model: the fused scorer fits and
// every hidden layer's row-major activations keep 16-byte chunks aligned.
static bool fused_forward_ok(const ModelLayout& L) {
    if (!L.tc_ok || L.n_hidden < 1) return false;
    for (int l = 0; l < L.n_hidden; ++l)
        if (L.widths[l + 1] % 8 != 0) return false;
    return true;
}

cudaError_t launch_forward_saved_tc(const ModelLayout& L, const TrainLayout& T, uint8_t* TW, const MlpDesc& md,
                                    int fmt, const int32_t* feat, int64_t n, float* d_y, cudaStream_t s,
                                    int* status_word, const FusedFwd* ff) {
    cudaError_t e;
    if (ff && fused_forward_ok(L))
        e = fmt == 1 ? forward_fused<__nv_bfloat16>(L, T, TW, md, fmt, feat, n, *ff, s)
                     : forward_fused<__half>(L, T, TW, md, fmt, feat, n, *ff, s);
    else if (fmt == 1) e = Tc<__nv_bfloat16>{L, T, TW, md, status_word}.forward(feat, n, s);
    else e = Tc<__half>{L, T, TW, md, status_word}.forward(feat, n, s);
    if (e != cudaSuccess || !d_y) return e;
    return launch_copy_f32(reinterpret_cast<const float*>(TW + T.act[L.n_layers]), d_y, n, s);
}

cudaError_t launch_backward_tc(const ModelLayout& L, const TrainLayout& T, uint8_t* TW, const MlpDesc& md, int fmt,
                               const float* d_dy, int64_t n, float* d_grad, cudaStream_t s, int* status_word) {
    if (d_dy) {
        cudaError_t e = launch_copy_f32(d_dy, reinterpret_cast<float*>(TW + T.dA), n, s);
        if (e != cudaSuccess) return e;
    }
    if (fmt == 1) return Tc<__nv_bfloat16>{L, T, TW, md, status_word}.backward(n, d_grad, s);
    return Tc<__half>{L, T, TW, md, status_word}.backward(n, d_grad, s);
}

template <typename X>
static cudaError_t loss_backward(const Tc<X>& tc, const ModelLayout& L, const TrainLayout& T, uint8_t* TW,
                                 const float* labels, int64_t n, float* grad, float* d_loss, cudaStream_t s) {
    if (tc.vec_path(n)) return tc.backward(n, grad, s, labels, reinterpret_cast<float*>(TW + T.loss), d_loss);
    const cudaError_t e = launch_mse_loss(L, T, TW, labels, n, d_loss, s);
    if (e != cudaSuccess) return e;
    return tc.backward(n, grad, s);
}

cudaError_t launch_loss_backward_tc(const ModelLayout& L, const TrainLayout& T, uint8_t* TW, const MlpDesc& md,
                                    int fmt, const float* labels, int64_t n, float* d_grad, float* d_loss,
                                    cudaStream_t s, int* status_word) {
    if (fmt == 1)
        return loss_backward(Tc<__nv_bfloat16>{L, T, TW, md, status_word}, L, T, TW, labels, n, d_grad, d_loss, s);
    return loss_backward(Tc<__half>{L, T, TW, md, status_word}, L, T, TW, labels, n, d_grad, d_loss, s);
}

cudaError_t launch_train_step_tc(const ModelLayout& L, const TrainLayout& T, uint8_t* P, uint8_t* TW,
                                 const MlpDesc& md, int fmt, const int32_t* feat, const float* labels, int64_t n,
                                 const AdamHyper* adam, int64_t step, float* d_grad_out, float* d_loss,
                                 cudaStream_t s, int* status_word, const FusedFwd* ff) {
    float* grad = d_grad_out ? d_grad_out : reinterpret_cast<float*>(TW + T.grad);
    cudaError_t e = launch_forward_saved_tc(L, T, TW, md, fmt, feat, n, nullptr, s, status_word, ff);
    if (e != cudaSuccess) return e;
    e = launch_loss_backward_tc(L, T, TW, md, fmt, labels, n, grad, d_loss, s, status_word);
    if (e != cudaSuccess || !adam) return e;
    return launch_adam_update(L, P, grad, *adam, step, s);
}

}  // namespace adv
