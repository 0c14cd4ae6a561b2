// Training mode (Sec. 3: the model is fitted to runtimes measured on the
// target; Sec. 5 Exp. 3: MLP, z-score standardised inputs).  Loss =
// 0.5 * mean (y - t)^2 on ln runtime, gradient by the hand-written backward
// of the ReLU MLP, Adam (Kingma & Ba) on the FP32 master weights.
//
// GEMMs are 128x128-tiled SIMT FP32 with generic operand strides:
//   forward   Out = In * W^T (+ b, ReLU on hidden layers)
//   dIn       dH  = dZ * W, masked by the ReLU of the layer input
//   dW, db    dW  = dZ^T * In and db = the column sums of dZ in the same
//             launch, split over rows in fixed chunks, then summed in a fixed
//             order (deterministic: the same inputs give the same bits)
// A layer with one output (or one input) column runs as a matrix-vector
// kernel instead of a 128-wide tile.
#include <cmath>

#include "features.cuh"
#include "pack.cuh"
#include "train.cuh"

namespace adv {

namespace {
constexpr int GT = 128;  // tile (rows and columns)
constexpr int GK = 8;    // K chunk
constexpr int SPLIT_ROWS = 1024;

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

struct GemmArgs {
    const float* A;
    int64_t sam, sak;
    const float* B;
    int64_t sbk, sbn;
    float* C;
    int64_t ldc;
    int64_t M, N, K;
    int64_t k_per_split;      // K range per blockIdx.z
    int64_t c_split_stride;   // element stride between split outputs
    const float* bias;        // EPI 1, 2
    const float* mask;        // EPI 3: C = mask > 0 ? acc : 0, mask(m, n) = mask[m * ldm + n]
    int64_t ldm;
    float* rowsum;            // optional: per split, sum over k of A(m, k) at rowsum[z * rowsum_stride + m]
    int64_t rowsum_stride;
};

// EPI: 0 plain, 1 bias + ReLU, 2 bias, 3 ReLU-derivative mask.
// 128 x 128 tile, 256 threads, 8 x 8 outputs per thread (rows 4 ty .. + 3 and
// 64 + 4 ty .. + 3, columns likewise with tx), K in chunks of 8 through a
// double-buffered shared-memory tile: the next chunk's global loads are in
// flight while the current one is used.  Each output is summed over k in
// increasing order with FMA (the order of the definition).  An operand whose k
// index is contiguous in memory is loaded with 8 consecutive threads along k,
// otherwise with consecutive threads along its row or column index, so that a
// warp's loads are coalesced either way.  With `rowsum`, the blocks of the
// first column tile also sum each row of A over the split's k range, in
// increasing k (the bias gradient when A is dZ transposed).
template <int EPI>
__global__ void __launch_bounds__(256, 2) gemm_kernel(GemmArgs g) {
    __shared__ __align__(16) float As[2][GK][GT + 4];
    __shared__ __align__(16) float Bs[2][GK][GT + 4];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * GT, n0 = (int64_t)blockIdx.x * GT;
    const int64_t kb = (int64_t)blockIdx.z * g.k_per_split;
    const int64_t ke = kb + g.k_per_split < g.K ? kb + g.k_per_split : g.K;
    const bool a_kc = g.sak == 1, b_kc = g.sbk == 1;
    // 16-byte loads where the operand allows them: 1 = four consecutive k of one
    // row (k contiguous), 2 = four consecutive rows or columns of one k; each
    // such piece lies wholly inside or wholly outside the operand
    auto al16 = [](const float* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    const int a_vec = (a_kc && g.sam % 4 == 0 && g.K % 4 == 0 && al16(g.A)) ? 1
                      : (g.sam == 1 && g.sak % 4 == 0 && g.M % 4 == 0 && al16(g.A)) ? 2 : 0;
    const int b_vec = (b_kc && g.sbn % 4 == 0 && g.K % 4 == 0 && al16(g.B)) ? 1
                      : (g.sbn == 1 && g.sbk % 4 == 0 && g.N % 4 == 0 && al16(g.B)) ? 2 : 0;
    // element r (0..3) of this thread's share of a 128 x 8 operand chunk (scalar loads)
    auto idx = [&](bool kc, int r, int& mn, int& kk) {
        if (kc) { mn = (tid >> 3) + 32 * r; kk = tid & 7; }
        else { mn = tid & 127; kk = (tid >> 7) + 2 * r; }
    };
    // this thread's 16-byte piece: mode 1 row tid / 2, k (tid % 2) * 4 .. + 3;
    // mode 2 k tid / 32, rows or columns (tid % 32) * 4 .. + 3
    auto vpos = [&](int mode, int& mn, int& kk) {
        if (mode == 1) { mn = tid >> 1; kk = (tid & 1) * 4; }
        else { mn = (tid & 31) * 4; kk = tid >> 5; }
    };
    float ra[4], rb[4];
    auto load_one = [&](const float* P, int64_t smn, int64_t sk, int64_t lim, int64_t o0, bool kc, int mode,
                        int64_t k0, float (&r4)[4]) {
        if (mode) {
            int mn, kk;
            vpos(mode, mn, kk);
            const int64_t x = o0 + mn, k = k0 + kk;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (x < lim && k < ke) v = *reinterpret_cast<const float4*>(P + x * smn + k * sk);
            r4[0] = v.x; r4[1] = v.y; r4[2] = v.z; r4[3] = v.w;
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                int mn, kk;
                idx(kc, r, mn, kk);
                const int64_t x = o0 + mn, k = k0 + kk;
                r4[r] = (x < lim && k < ke) ? P[x * smn + k * sk] : 0.f;
            }
        }
    };
    auto load = [&](int64_t k0) {
        load_one(g.A, g.sam, g.sak, g.M, m0, a_kc, a_vec, k0, ra);
        load_one(g.B, g.sbn, g.sbk, g.N, n0, b_kc, b_vec, k0, rb);
    };
    auto store_one = [&](float (*S)[GT + 4], bool kc, int mode, const float (&r4)[4]) {
        int mn, kk;
        if (mode == 1) {
            vpos(1, mn, kk);
#pragma unroll
            for (int j = 0; j < 4; ++j) S[kk + j][mn] = r4[j];
        } else if (mode == 2) {
            vpos(2, mn, kk);
            *reinterpret_cast<float4*>(&S[kk][mn]) = make_float4(r4[0], r4[1], r4[2], r4[3]);
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                idx(kc, r, mn, kk);
                S[kk][mn] = r4[r];
            }
        }
    };
    auto store = [&](int buf) {
        store_one(As[buf], a_kc, a_vec, ra);
        store_one(Bs[buf], b_kc, b_vec, rb);
    };
    uint64_t acc[8][4];   // row i, columns (2 jj, 2 jj + 1) as an FP32 pair
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) acc[i][jj] = 0ull;
    const bool do_rs = g.rowsum && blockIdx.x == 0 && tid < GT;   // row tid of the tile
    float accb = 0.f;
    int buf = 0;
    if (kb < ke) {
        load(kb);
        store(0);
    }
    __syncthreads();
    for (int64_t k0 = kb; k0 < ke; k0 += GK) {
        const bool more = k0 + GK < ke;
        if (more) load(k0 + GK);
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][4 * ty]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + 4 * ty]);
            const ulonglong2 b0 = *reinterpret_cast<const ulonglong2*>(&Bs[buf][kk][4 * tx]);
            const ulonglong2 b1 = *reinterpret_cast<const ulonglong2*>(&Bs[buf][kk][64 + 4 * tx]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const uint64_t b[4] = {b0.x, b0.y, b1.x, b1.y};
            // two columns per instruction, each an IEEE FMA as fmaf computes it
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint64_t a2 = f32x2_dup(a[i]);
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) f32x2_fma(acc[i][jj], a2, b[jj]);
            }
        }
        if (do_rs) {
#pragma unroll
            for (int kk = 0; kk < GK; ++kk) accb += As[buf][kk][tid];
        }
        if (more) store(buf ^ 1);   // that buffer's readers passed the barrier below last chunk
        __syncthreads();
        buf ^= 1;
    }
    if (do_rs && m0 + tid < g.M) g.rowsum[(int64_t)blockIdx.z * g.rowsum_stride + m0 + tid] = accb;
    float* C = g.C + (int64_t)blockIdx.z * g.c_split_stride;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t m = m0 + (i < 4 ? 4 * ty + i : 64 + 4 * ty + i - 4);
        if (m >= g.M) continue;
        float r[8];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) f32x2_unpack(acc[i][jj], r[2 * jj], r[2 * jj + 1]);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t n = n0 + (j < 4 ? 4 * tx + j : 64 + 4 * tx + j - 4);
            if (n >= g.N) continue;
            float v = r[j];
            if constexpr (EPI == 1) v = fmaxf(v + g.bias[n], 0.f);
            if constexpr (EPI == 2) v = v + g.bias[n];
            if constexpr (EPI == 3) v = g.mask[m * g.ldm + n] > 0.f ? v : 0.f;
            C[m * g.ldc + n] = v;
        }
    }
}

// A GEMM with one output column (N = 1: the output layer's forward) or one
// output row (M = 1: the output layer's weight gradient) as a matrix-vector
// product: one thread per output element of the split, summing over k in
// increasing order with FMA, as gemm_kernel does (same values), without the
// 127 idle columns or rows of a 128 x 128 tile.  With `rowsum` (M = 1 only),
// thread N sums A over the split instead (the output bias's gradient).
template <int EPI, bool ROW>
__global__ void __launch_bounds__(256) gemv_kernel(GemmArgs g) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // m (N = 1) or n (M = 1)
    const int64_t kb = (int64_t)blockIdx.z * g.k_per_split;
    const int64_t ke = kb + g.k_per_split < g.K ? kb + g.k_per_split : g.K;
    if (ROW && g.rowsum && t == g.N) {
        float v = 0.f;
        for (int64_t k = kb; k < ke; ++k) v += g.A[k * g.sak];
        g.rowsum[(int64_t)blockIdx.z * g.rowsum_stride] = v;
        return;
    }
    if (t >= (ROW ? g.N : g.M)) return;
    const float* A = ROW ? g.A : g.A + t * g.sam;
    const float* B = ROW ? g.B + t * g.sbn : g.B;
    float v = 0.f;
    int64_t k = kb;
    if (!ROW && g.sak == 1 && g.sbk == 1 && ((reinterpret_cast<uintptr_t>(A + kb) | reinterpret_cast<uintptr_t>(B + kb)) & 15) == 0) {
        // the row of A and the column of B as 16-byte loads, the FMAs still in k order
        for (; k + 4 <= ke; k += 4) {
            const float4 a = *reinterpret_cast<const float4*>(A + k);
            const float4 b = __ldg(reinterpret_cast<const float4*>(B + k));
            v = fmaf(a.x, b.x, v);
            v = fmaf(a.y, b.y, v);
            v = fmaf(a.z, b.z, v);
            v = fmaf(a.w, b.w, v);
        }
    }
    for (; k < ke; ++k) v = fmaf(A[k * g.sak], B[k * g.sbk], v);
    const int64_t m = ROW ? 0 : t, n = ROW ? t : 0;
    if (!ROW && g.rowsum) {   // one input column: the row's sum over the split is its only A element's
        float r = 0.f;
        for (int64_t kk = kb; kk < ke; ++kk) r += A[kk * g.sak];
        g.rowsum[(int64_t)blockIdx.z * g.rowsum_stride + m] = r;
    }
    if constexpr (EPI == 1) v = fmaxf(v + g.bias[n], 0.f);
    if constexpr (EPI == 2) v = v + g.bias[n];
    if constexpr (EPI == 3) v = g.mask[m * g.ldm + n] > 0.f ? v : 0.f;
    g.C[(int64_t)blockIdx.z * g.c_split_stride + m * g.ldc + n] = v;
}

template <int EPI>
cudaError_t gemm(const GemmArgs& g, int splits, cudaStream_t s) {
    if (g.N == 1 || g.M == 1) {
        const int64_t len = g.N == 1 ? g.M : g.N + (g.rowsum ? 1 : 0);
        dim3 grid((unsigned)((len + 255) / 256), 1, (unsigned)splits);
        if (g.N == 1) gemv_kernel<EPI, false><<<grid, 256, 0, s>>>(g);
        else gemv_kernel<EPI, true><<<grid, 256, 0, s>>>(g);
    } else {
        dim3 grid((unsigned)((g.N + GT - 1) / GT), (unsigned)((g.M + GT - 1) / GT), (unsigned)splits);
        gemm_kernel<EPI><<<grid, 256, 0, s>>>(g);
    }
    adv_count_launch(1);
    return cudaGetLastError();
}

__global__ void standardize_f32_kernel(const int32_t* __restrict__ feat, int64_t n, int F,
                                       const float* __restrict__ sa, const float* __restrict__ sc,
                                       float* __restrict__ z) {
    const int64_t total = n * F;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(i % F);
        z[i] = fmaf((float)feat[i], sa[k], -sc[k]);
    }
}

// dy = (y - t) / n and per-block sums of 0.5 (y - t)^2 (fixed order).
__global__ void __launch_bounds__(256) loss_kernel(const float* __restrict__ y, const float* __restrict__ t,
                                                   int64_t n, float* __restrict__ dy, float* __restrict__ part) {
    __shared__ float red[256];
    float s = 0.f;
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b = (int64_t)blockIdx.x * per, e = b + per < n ? b + per : n;
    for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
        const float d = y[i] - t[i];
        dy[i] = d / (float)n;
        s += 0.5f * d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// One warp: lane l sums part[l], part[l + 32], ... in order, then the lanes
// are added in a fixed tree.
__global__ void loss_final_kernel(const float* __restrict__ part, int nb, int64_t n, float* __restrict__ loss,
                                  float* __restrict__ loss_out) {
    const int lane = threadIdx.x;
    float s = 0.f;
    for (int i = lane; i < nb; i += 32) s += part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        *loss = s / (float)n;
        if (loss_out) *loss_out = s / (float)n;
    }
}

// RMSE loss (Sec. 5 Exp. 3) from the MSE path's values: loss[0] holds
// 0.5 mean e^2 and dy the MSE gradient e / n; RMSE = sqrt(2 loss[0]) goes to
// loss[1] (and loss_out) and dy becomes e / (n RMSE), in place.
__global__ void rmse_scale_kernel(float* __restrict__ dy, int64_t n, float* __restrict__ loss,
                                  float* __restrict__ loss_out) {
    const float rmse = sqrtf(2.f * loss[0]);
    const float inv = rmse > 0.f ? 1.f / rmse : 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dy[i] *= inv;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        loss[1] = rmse;
        if (loss_out) *loss_out = rmse;
    }
}

// RMSprop (Tieleman & Hinton 2012) with the weight decay added to the
// gradient: g' = g + wd w; v = alpha v + (1 - alpha) g'^2; w -= lr g' / (sqrt(v) + eps).
__global__ void rmsprop_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ v, int64_t n,
                               float lr, float alpha, float eps, float wd) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i] + wd * p[i];
        const float vi = alpha * v[i] + (1.f - alpha) * gi * gi;
        v[i] = vi;
        p[i] -= lr * gi / (sqrtf(vi) + eps);
    }
}

// grad[j] = sum over splits (in order) of part[s][j]; eight partials' loads
// are issued together, then added one after another
__global__ void split_sum_kernel(const float* __restrict__ part, int splits, int64_t stride, int64_t len,
                                 float* __restrict__ grad) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < len; j += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        int i = 0;
        for (; i + 8 <= splits; i += 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = part[(int64_t)(i + u) * stride + j];
#pragma unroll
            for (int u = 0; u < 8; ++u) s += v[u];
        }
        for (; i < splits; ++i) s += part[(int64_t)i * stride + j];
        grad[j] = s;
    }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, AdamHyper h, float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = h.beta1 * m[i] + (1.f - h.beta1) * gi;
        const float vi = h.beta2 * v[i] + (1.f - h.beta2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / c1, vh = vi / c2;
        p[i] = p[i] - h.lr * (mh / (sqrtf(vh) + h.eps) + h.weight_decay * p[i]);
    }
}

int grid1(int64_t n) {
    const int64_t g = (n + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 8192 ? 8192 : g));
}

}  // namespace

size_t train_layout(const ModelLayout& L, int64_t R, TrainLayout* t) {
    size_t o = 0;
    auto take = [&](size_t b) { size_t at = o; o = al(o + b); return at; };
    int wmax = 0;
    for (int i = 0; i < L.nw; ++i) wmax = L.widths[i] > wmax ? L.widths[i] : wmax;
    for (int l = 0; l < L.nw; ++l) t->act[l] = take((size_t)R * L.widths[l] * 4);
    t->dA = take((size_t)R * wmax * 4);
    t->dB = take((size_t)R * wmax * 4);
    t->grad = take((size_t)L.n_params * 4);
    t->splits = (int)((R + SPLIT_ROWS - 1) / SPLIT_ROWS);
    int64_t lmax = 0;
    for (int l = 0; l < L.n_layers; ++l) {
        const int64_t len = (int64_t)L.widths[l] * L.widths[l + 1];
        lmax = len > lmax ? len : lmax;
    }
    t->part = take((size_t)2 * t->splits * lmax * 4);   // room for up to twice the 1,024-row splits
    t->loss_part = take(1024 * 4);
    t->loss = take(64);
    // 16-bit tensor-core training: 16-bit activations, weights and dZ
    // ping-pong; the FP32 GEMM outputs reuse dB
    t->x16 = take((size_t)R * L.F * 2);
    for (int l = 0; l < L.n_hidden; ++l) {
        t->h16[l] = take((size_t)R * L.widths[l + 1] * 2);
        t->w16[l] = take((size_t)L.widths[l] * L.widths[l + 1] * 2);
    }
    t->dz16[0] = take((size_t)R * wmax * 2);
    t->dz16[1] = take((size_t)R * wmax * 2);
    t->c32 = t->dB;
    // partials of the 16-bit backward's column sums: the last hidden layer's
    // (bias and output row, per 256-row block), the output bias (per 1,024
    // rows, or per 256-row block with the loss fused in, which adds the loss's
    // per block), and per lower hidden layer the ReLU-backward kernel's (four
    // per CTA of up to 256 CTAs, or one per 128-row tile in the generic form)
    const int64_t tiles = (R + 127) / 128;
    t->bias_part_floats = 2 * ((R + 255) / 256) * wmax + (R + 1023) / 1024 + 2 * ((R + 255) / 256) +
                          (int64_t)L.n_hidden * (tiles > 1024 ? tiles : 1024) * wmax;
    t->bias_part = take((size_t)t->bias_part_floats * 4);
    t->rows = R;
    t->bytes = o;
    return o;
}

cudaError_t launch_forward_saved(const ModelLayout& L, const TrainLayout& T, uint8_t* TW, const MlpDesc& md,
                                 const int32_t* feat, int64_t n, float* d_y, cudaStream_t s) {
    cudaError_t e;
    auto act = [&](int l) { return reinterpret_cast<float*>(TW + T.act[l]); };
    standardize_f32_kernel<<<grid1(n * L.F), 256, 0, s>>>(feat, n, L.F, md.sa, md.sc, act(0));
    adv_count_launch(1);
    for (int l = 0; l < L.n_layers; ++l) {
        const int fi = L.widths[l], fo = L.widths[l + 1];
        GemmArgs g{};
        g.A = act(l); g.sam = fi; g.sak = 1;
        g.B = md.W[l]; g.sbk = 1; g.sbn = fi;
        g.C = act(l + 1); g.ldc = fo;
        g.M = n; g.N = fo; g.K = fi; g.k_per_split = fi; g.c_split_stride = 0;
        g.bias = md.b[l];
        e = (l + 1 < L.n_layers) ? gemm<1>(g, 1, s) : gemm<2>(g, 1, s);
        if (e != cudaSuccess) return e;
    }
    if (d_y) return launch_copy_f32(act(L.n_layers), d_y, n, s);
    return cudaGetLastError();
}

// dL/dy of loss = 0.5 mean (y - t)^2 into the gradient buffer, loss to d_loss.
cudaError_t launch_mse_loss(const ModelLayout& L, const TrainLayout& T, uint8_t* TW, const float* labels,
                              int64_t n, float* d_loss, cudaStream_t s) {
    const int nb = 256;
    loss_kernel<<<nb, 256, 0, s>>>(reinterpret_cast<float*>(TW + T.act[L.n_layers]), labels, n,
                                   reinterpret_cast<float*>(TW + T.dA), reinterpret_cast<float*>(TW + T.loss_part));
    loss_final_kernel<<<1, 32, 0, s>>>(reinterpret_cast<float*>(TW + T.loss_part), nb, n,
                                       reinterpret_cast<float*>(TW + T.loss), d_loss);
    adv_count_launch(2);
    return cudaGetLastError();
}

// Backward of the saved forward from dL/dy (already in the dA buffer) to the
// parameter gradient.
cudaError_t launch_backward_saved(const ModelLayout& L, const TrainLayout& T, uint8_t* TW, const MlpDesc& md,
                                        int64_t n, float* grad, cudaStream_t s) {
    cudaError_t e;
    auto act = [&](int l) { return reinterpret_cast<float*>(TW + T.act[l]); };
    float* dz = reinterpret_cast<float*>(TW + T.dA);
    float* dnext = reinterpret_cast<float*>(TW + T.dB);
    float* part = reinterpret_cast<float*>(TW + T.part);
    float* bpart = reinterpret_cast<float*>(TW + T.bias_part);
    int64_t lmax = 0;   // the dW partial buffer holds 2 x T.splits x lmax floats
    for (int l = 0; l < L.n_layers; ++l)
        lmax = (int64_t)L.widths[l] * L.widths[l + 1] > lmax ? (int64_t)L.widths[l] * L.widths[l + 1] : lmax;
    const int64_t part_cap = 2 * (int64_t)T.splits * lmax;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 0;
    for (int l = L.n_layers - 1; l >= 0; --l) {
        const int fi = L.widths[l], fo = L.widths[l + 1];
        float* gW = grad + L.layer_w_off[l];
        float* gb = grad + L.layer_b_off[l];
        // dW = dZ^T * In and db = column sums of dZ in one launch, split over rows
        // in fixed chunks, each summed in a fixed order.  The single-output layer's
        // matrix-vector form takes 128-row chunks (eight times the threads) where
        // its partials fit.  The tiled form takes as many chunks (whole 8-row
        // steps) as give two blocks on every SM once: 1,024-row chunks of a
        // 256 x 256 layer give 256 blocks, two on 104 SMs and one on the other 48,
        // so the launch lasts two block-times for 1.7 of work.
        int64_t rows_per = SPLIT_ROWS;
        if (fo == 1) {
            if (((n + 127) / 128) * (int64_t)fi <= part_cap) rows_per = 128;
        } else if (fi > 1 && sms > 0) {
            const int64_t tiles = (int64_t)((fo + GT - 1) / GT) * ((fi + GT - 1) / GT);
            const int64_t want = 2 * sms / tiles > 1 ? 2 * sms / tiles : 1;
            int64_t rp = ((n + want - 1) / want + 7) / 8 * 8;
            rp = rp < 64 ? 64 : rp;
            const int64_t spl = (n + rp - 1) / rp;
            if (spl * fo * fi <= part_cap && spl * fo <= T.bias_part_floats) rows_per = rp;
        }
        const int sp = (int)((n + rows_per - 1) / rows_per);
        GemmArgs g{};
        g.A = dz; g.sam = 1; g.sak = fo;
        g.B = act(l); g.sbk = fi; g.sbn = 1;
        g.C = part; g.ldc = fi;
        g.M = fo; g.N = fi; g.K = n; g.k_per_split = rows_per;
        g.c_split_stride = (int64_t)fo * fi;
        g.rowsum = bpart; g.rowsum_stride = fo;
        e = gemm<0>(g, sp, s);
        if (e != cudaSuccess) return e;
        split_sum_kernel<<<grid1((int64_t)fo * fi), 256, 0, s>>>(part, sp, (int64_t)fo * fi, (int64_t)fo * fi, gW);
        split_sum_kernel<<<grid1(fo), 256, 0, s>>>(bpart, sp, fo, fo, gb);
        adv_count_launch(2);
        if (l == 0) break;
        // dIn = dZ * W, masked by the ReLU of the input (the previous layer's output)
        GemmArgs h{};
        h.A = dz; h.sam = fo; h.sak = 1;
        h.B = md.W[l]; h.sbk = fi; h.sbn = 1;
        h.C = dnext; h.ldc = fi;
        h.M = n; h.N = fi; h.K = fo; h.k_per_split = fo; h.c_split_stride = 0;
        h.mask = act(l); h.ldm = fi;
        e = gemm<3>(h, 1, s);
        if (e != cudaSuccess) return e;
        float* t = dz; dz = dnext; dnext = t;
    }
    return cudaGetLastError();
}

cudaError_t launch_backward(const ModelLayout& L, const TrainLayout& T, uint8_t* TW, const MlpDesc& md,
                            const float* d_dy, int64_t n, float* d_grad, cudaStream_t s) {
    cudaError_t e = launch_copy_f32(d_dy, reinterpret_cast<float*>(TW + T.dA), n, s);
    if (e != cudaSuccess) return e;
    return launch_backward_saved(L, T, TW, md, n, d_grad, s);
}

cudaError_t launch_train_step(const ModelLayout& L, const TrainLayout& T, uint8_t* P, uint8_t* TW,
                              const MlpDesc& md, const int32_t* feat, const float* labels, int64_t n,
                              const AdamHyper* adam, int64_t step, float* d_grad_out, float* d_loss, int num_sms,
                              cudaStream_t s) {
    (void)num_sms;
    float* grad = d_grad_out ? d_grad_out : reinterpret_cast<float*>(TW + T.grad);
    cudaError_t e = launch_forward_saved(L, T, TW, md, feat, n, nullptr, s);
    if (e != cudaSuccess) return e;
    e = launch_mse_loss(L, T, TW, labels, n, d_loss, s);
    if (e != cudaSuccess) return e;
    e = launch_backward_saved(L, T, TW, md, n, grad, s);
    if (e != cudaSuccess || !adam) return e;
    return launch_adam_update(L, P, grad, *adam, step, s);
}

cudaError_t launch_adam_update(const ModelLayout& L, uint8_t* P, const float* grad, const AdamHyper& adam,
                               int64_t step, cudaStream_t s) {
    const float c1 = (float)(1.0 - std::pow((double)adam.beta1, (double)step));
    const float c2 = (float)(1.0 - std::pow((double)adam.beta2, (double)step));
    adam_kernel<<<grid1(L.n_params), 256, 0, s>>>(reinterpret_cast<float*>(P + L.p_master), grad,
                                                  reinterpret_cast<float*>(P + L.p_adam_m),
                                                  reinterpret_cast<float*>(P + L.p_adam_v), L.n_params, adam, c1,
                                                  c2);
    adv_count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_train_step_ex(const ModelLayout& L, const TrainLayout& T, uint8_t* P, uint8_t* TW,
                                 const MlpDesc& md, int fmt, const int32_t* feat, const float* labels, int64_t n,
                                 const TrainOptions& o, int64_t step, float* d_loss, cudaStream_t s, int* status_word,
                                 const FusedFwd* ff) {
    float* grad = reinterpret_cast<float*>(TW + T.grad);
    float* loss = reinterpret_cast<float*>(TW + T.loss);
    cudaError_t e = fmt == 0 ? launch_forward_saved(L, T, TW, md, feat, n, nullptr, s)
                             : launch_forward_saved_tc(L, T, TW, md, fmt, feat, n, nullptr, s, status_word, ff);
    if (e != cudaSuccess) return e;
    if (fmt != 0 && o.loss == 0) {   // MSE on the tensor cores: the loss goes with the backward
        e = launch_loss_backward_tc(L, T, TW, md, fmt, labels, n, grad, d_loss, s, status_word);
        if (e != cudaSuccess) return e;
        if (o.optimizer == 0) return launch_adam_update(L, P, grad, o.h, step, s);
        rmsprop_kernel<<<grid1(L.n_params), 256, 0, s>>>(reinterpret_cast<float*>(P + L.p_master), grad,
                                                         reinterpret_cast<float*>(P + L.p_adam_v), L.n_params,
                                                         o.h.lr, o.alpha, o.h.eps, o.h.weight_decay);
        adv_count_launch(1);
        return cudaGetLastError();
    }
    e = launch_mse_loss(L, T, TW, labels, n, o.loss == 1 ? nullptr : d_loss, s);
    if (e != cudaSuccess) return e;
    if (o.loss == 1) {
        rmse_scale_kernel<<<grid1(n), 256, 0, s>>>(reinterpret_cast<float*>(TW + T.dA), n, loss, d_loss);
        adv_count_launch(1);
    }
    e = fmt == 0 ? launch_backward_saved(L, T, TW, md, n, grad, s)
                 : launch_backward_tc(L, T, TW, md, fmt, nullptr, n, grad, s, status_word);
    if (e != cudaSuccess) return e;
    if (o.optimizer == 0) return launch_adam_update(L, P, grad, o.h, step, s);
    rmsprop_kernel<<<grid1(L.n_params), 256, 0, s>>>(reinterpret_cast<float*>(P + L.p_master), grad,
                                                     reinterpret_cast<float*>(P + L.p_adam_v), L.n_params, o.h.lr,
                                                     o.alpha, o.h.eps, o.h.weight_decay);
    adv_count_launch(1);
    return cudaGetLastError();
}

}  // namespace adv
