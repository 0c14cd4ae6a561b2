// Dense GEMMs of the 16-bit training step (Sec. 3 training mode, Sec. 5
// Exp. 3) on the tensor cores:
//
//   C[m][n] = sum_k A(m, k) B(n, k),  16-bit operands (BF16 or FP16), FP32
//   accumulation in tensor memory (tcgen05.mma, M = 128, N <= 256, K = 16).
//
// Each operand is read from a row-major array either as A[m][k] ("K-major":
// rows along M) or as A[k][m] ("MN-major": rows along K), and likewise B.
// A layer's training step needs
//   forward        C  = In W^T   (A = In K-major,  B = W K-major),
//   weight grad    dW = dZ^T In  (A = dZ MN-major, B = In MN-major; K = the
//                                 batch rows, split over CTAs, the partial
//                                 sums added in a fixed order),
//   input grad     dX = dZ W     (A = dZ K-major,  B = W MN-major).
// The loaders copy 16-byte chunks of 128-byte rows (64 16-bit values) into
// shared memory with the 128-byte swizzle (chunk c of row r at c ^ (r % 8)).
// The same byte pattern is a K-major operand when the rows run along M / N
// (UMMA descriptor: 8-row groups 1 KB apart) and an MN-major one when the
// rows run along K (atoms of 64 M / N values x 8 K rows, 1 KB; K groups 1 KB
// apart, M / N atoms 8 KB apart); the instruction descriptor's transpose
// bits say which.  One CTA computes a 128 x (up to) 256 tile of C over its
// range of K, through a ring of stages.  When both operands' row strides are
// multiples of 16 bytes, one thread fills the stages with 2-D TMA copies
// (cp.async.bulk.tensor, 128-byte swizzle; a {64, 128} box is a K-major
// tile, a {64, 64} box an MN-major atom; out-of-range elements read as zero)
// and another issues the MMAs; otherwise all four warps copy 16-byte chunks
// with cp.async (element by element where a chunk is not 16-byte aligned).
// The four warps then drain the accumulator (one TMEM lane quadrant each).
// Every barrier wait is bounded (ADV_DEV_TIMEOUT).
#include "mlp.cuh"
#include "train.cuh"

namespace adv {

namespace {

constexpr int GT_THREADS = 128;
constexpr int GT_M = 128;
constexpr int GT_NMAX = 256;
constexpr int GT_KB = 64;                          // K per block: one 128-byte row of 16-bit values
constexpr int GT_STAGES = 4;
constexpr uint32_t GT_A_BYTES = GT_M * 128;        // 16 KB

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// 2-D TMA load of box {x, y} (x the contiguous dimension) into shared memory,
// counted in bytes on `bar`; x * 2 bytes is a multiple of 16.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int32_t x, int32_t y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

// UMMA shared-memory descriptor of an MN-major operand with the 128-byte
// swizzle: atoms of 64 M/N values (128 B) x 8 K rows; M/N atoms `lbo` bytes
// apart, 8-row K groups `sbo` bytes apart.
__device__ __forceinline__ uint64_t mn128_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// One K block (GT_KB values of K) of an operand into shared memory.
//   K-major  (mn == 0): rows r = 0..rows-1 along M/N, 128 B each, at sw128_offset(r, c);
//   MN-major (mn == 1): atom a (64 M/N values), K row kr = 0..63, at a * 8 KB + sw128_offset(kr, c).
// Elements outside [0, nvalid) x [0, K) are zero.  16-byte chunks whose 8
// values are all in range come by cp.async when `fast` (row stride a
// multiple of 8 values, 16-byte aligned base); the rest element by element.
__device__ __forceinline__ void load_block(uint8_t* dst, const uint16_t* __restrict__ src, int64_t ld, int mn,
                                           int64_t row0, int64_t nvalid, int rows, int64_t k0, int64_t K, bool fast,
                                           int tid) {
    const int chunks = rows * 8;
    for (int i = tid; i < chunks; i += GT_THREADS) {
        uint32_t off;
        int64_t r, k;   // first element of the chunk: M/N index r, K index k
        bool along_mn;  // the chunk's 8 values run along M/N (MN-major) or along K
        if (!mn) {
            const int rr = i >> 3, c = i & 7;
            off = sw128_offset((uint32_t)rr, (uint32_t)c);
            r = row0 + rr;
            k = k0 + 8 * c;
            along_mn = false;
        } else {
            const int a = i >> 9, rem = i & 511, kr = rem >> 3, c = rem & 7;
            off = (uint32_t)a * 8192u + sw128_offset((uint32_t)kr, (uint32_t)c);
            r = row0 + a * 64 + 8 * c;
            k = k0 + kr;
            along_mn = true;
        }
        const bool all = along_mn ? (k < K && r + 8 <= nvalid) : (r < nvalid && k + 8 <= K);
        if (fast && all) {
            cp_async16(dst + off, src + (along_mn ? k * ld + r : r * ld + k));
        } else {
            uint16_t v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int64_t rr = along_mn ? r + e : r, kk = along_mn ? k : k + e;
                v[e] = (rr < nvalid && kk < K) ? src[along_mn ? kk * ld + rr : rr * ld + kk] : (uint16_t)0;
            }
            *reinterpret_cast<uint4*>(dst + off) =
                make_uint4(v[0] | (uint32_t)v[1] << 16, v[2] | (uint32_t)v[3] << 16, v[4] | (uint32_t)v[5] << 16,
                           v[6] | (uint32_t)v[7] << 16);
        }
    }
}

// Bounded wait that ignores the abort flag (draining copies already issued).
__device__ __forceinline__ bool mbar_wait_drain(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    const uint64_t t0 = global_timer_ns();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 63u && global_timer_ns() - t0 > limit_ns) return false;
    }
}

template <int FMT>
__device__ __forceinline__ uint32_t pack16x2(float lo, float hi) {
    uint32_t d;
    if constexpr (FMT == 1) asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    else asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// Sum over the warp's 32 lanes (rows) of q[0..15] (16 columns), by halving
// exchanges: after them lane L holds the total of column
// 8 b4 + 4 b3 + 2 b2 + b1 (b_i bit i of L; lanes L and L ^ 1 the same).
// The pairing is fixed, so the result is the same bits on every run.
__device__ __forceinline__ float warp_colsum16(float (&q)[16], int lane) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const bool hi = lane & 16;
        const float send = hi ? q[i] : q[i + 8], keep = hi ? q[i + 8] : q[i];
        q[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool hi = lane & 8;
        const float send = hi ? q[i] : q[i + 4], keep = hi ? q[i + 4] : q[i];
        q[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool hi = lane & 4;
        const float send = hi ? q[i] : q[i + 2], keep = hi ? q[i + 2] : q[i];
        q[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
        const bool hi = lane & 2;
        const float send = hi ? q[0] : q[1], keep = hi ? q[1] : q[0];
        q[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    return q[0] + __shfl_xor_sync(0xffffffffu, q[0], 1);
}

// Whether the 16-bit value with these bits is > 0: the bits lie in
// [1, +inf] (sign clear, not zero, not NaN).
template <int FMT>
__device__ __forceinline__ bool pos16(uint32_t bits) {
    return bits - 1u < (FMT == 1 ? 0x7F80u : 0x7C00u);
}

template <int FMT>
__device__ __forceinline__ float round16(float x) {
    const uint32_t p = pack16x2<FMT>(x, 0.f) & 0xFFFFu;
    if constexpr (FMT == 1) return __uint_as_float(p << 16);
    else return __half2float(__ushort_as_half((unsigned short)p));
}

// Masked form: whether rows of C and mask_h are read and written in 16-byte
// pieces (row stride a multiple of 8 values, 16-byte aligned bases).
__device__ __forceinline__ bool mask_vec(const TcGemm& g) {
    return g.ldc % 8 == 0 && ((uintptr_t)g.C & 15) == 0 && ((uintptr_t)g.mask_h & 15) == 0;
}

// Masked form, before the accumulator is ready: the thread's mask_h row in
// chunks 0..3 (16 values each) into registers, and the rest of the row's
// tile prefetched into L2.  Chunks that are not whole stay zero (the
// epilogue reads those element by element).
__device__ __forceinline__ void mask_preload(const TcGemm& g, int64_t m0, int64_t n0, int nt, int warp, int lane,
                                             uint4 (&hb)[4][2]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) hb[k][0] = hb[k][1] = make_uint4(0u, 0u, 0u, 0u);
    const int64_t row = m0 + 32 * warp + lane;
    if (!g.mask_h || row >= g.M || !mask_vec(g)) return;
    const uint16_t* hp = g.mask_h + row * g.ldc + n0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (16 * k + 16 <= nt) {
            hb[k][0] = reinterpret_cast<const uint4*>(hp + 16 * k)[0];
            hb[k][1] = reinterpret_cast<const uint4*>(hp + 16 * k)[1];
        }
    for (int off = 64; off < nt; off += 64) asm volatile("prefetch.global.L2 [%0];" ::"l"(hp + off));
}

// Masked epilogue (ReLU backward of the layer below): dZ = 16-bit(acc) where
// mask_h > 0, else 0, stored into C; the tile's column sums of the stored dZ
// into colpart[blockIdx.y][n0 + c] (rows in a fixed tree over the lanes, then
// the four warps in order).  `red` holds 4 x GT_NMAX floats of shared memory;
// hb holds chunks 0..3 of the row's mask (mask_preload) and is refilled four
// chunks ahead.
template <int FMT>
__device__ __forceinline__ void gemm_epilogue_mask(const TcGemm& g, uint32_t tmem, int64_t m0, int64_t n0, int nt,
                                                   int nt16, bool have_acc, bool got, int warp, int lane,
                                                   float* red, uint4 (&hb)[4][2]) {
    const int64_t row = m0 + 32 * warp + lane;
    const bool row_ok = got && row < g.M;
    const bool vec = mask_vec(g);
    const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);
    uint16_t* c16 = reinterpret_cast<uint16_t*>(g.C);
    const int colid = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
    for (int cb = 0; cb < nt16; cb += 64) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c0 = cb + 16 * k;
            if (c0 >= nt16) break;   // uniform over the CTA
            uint32_t v[16];
            if (have_acc) {
                tmem_ld_32x32b_x16(tl + (uint32_t)c0, v);
                tmem_wait_ld();
            } else {
#pragma unroll
                for (int e = 0; e < 16; ++e) v[e] = 0u;
            }
            float q[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) q[e] = 0.f;
            if (row_ok) {
                const int64_t col = n0 + c0;
                const uint16_t* hp = g.mask_h + row * g.ldc + col;
                uint16_t* dst = c16 + row * g.ldc + col;
                if (vec && c0 + 16 <= nt) {
                    const uint32_t hw[8] = {hb[k][0].x, hb[k][0].y, hb[k][0].z, hb[k][0].w,
                                            hb[k][1].x, hb[k][1].y, hb[k][1].z, hb[k][1].w};
                    if (c0 + 80 <= nt) {   // refill with chunk c0 + 64
                        hb[k][0] = reinterpret_cast<const uint4*>(hp + 64)[0];
                        hb[k][1] = reinterpret_cast<const uint4*>(hp + 64)[1];
                    }
                    uint32_t pk[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const float a = pos16<FMT>(hw[e] & 0xFFFFu) ? __uint_as_float(v[2 * e]) : 0.f;
                        const float b = pos16<FMT>(hw[e] >> 16) ? __uint_as_float(v[2 * e + 1]) : 0.f;
                        pk[e] = pack16x2<FMT>(a, b);
                    }
                    reinterpret_cast<uint4*>(dst)[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    reinterpret_cast<uint4*>(dst)[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        if constexpr (FMT == 1) {
                            q[2 * e] = __uint_as_float(pk[e] << 16);
                            q[2 * e + 1] = __uint_as_float(pk[e] & 0xFFFF0000u);
                        } else {
                            q[2 * e] = __half2float(__ushort_as_half((unsigned short)(pk[e] & 0xFFFFu)));
                            q[2 * e + 1] = __half2float(__ushort_as_half((unsigned short)(pk[e] >> 16)));
                        }
                    }
                } else {
                    for (int e = 0; e < 16 && col + e < g.N; ++e) {
                        const float x = pos16<FMT>(hp[e]) ? __uint_as_float(v[e]) : 0.f;
                        dst[e] = (uint16_t)(pack16x2<FMT>(x, 0.f) & 0xFFFFu);
                        q[e] = round16<FMT>(x);
                    }
                }
            }
            const float cs = warp_colsum16(q, lane);
            if ((lane & 1) == 0) red[warp * GT_NMAX + c0 + colid] = cs;
        }
    }
    __syncthreads();
    for (int c = 32 * warp + lane; c < nt; c += GT_THREADS) {
        const float t = ((red[c] + red[GT_NMAX + c]) + red[2 * GT_NMAX + c]) + red[3 * GT_NMAX + c];
        if (got) g.colpart[(size_t)blockIdx.y * g.N + n0 + c] = t;
    }
}

// Epilogue shared by both kernels: warp w drains TMEM lanes 32w .. 32w+31
// (rows m0 + 32w + lane) of the tile's nt16 columns into C (or the split's
// partials); zero when the tile had no K block.
template <int FMT>
__device__ __forceinline__ void gemm_epilogue(const TcGemm& g, uint32_t tmem, int64_t m0, int64_t n0, int nt16,
                                              bool have_acc, bool got, int warp, int lane) {
    const int64_t row = m0 + 32 * warp + lane;
    const bool row_ok = got && row < g.M;
    const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);
    float* c32 = g.splits > 1 ? g.part + (size_t)blockIdx.z * g.M * g.ldc : reinterpret_cast<float*>(g.C);
    uint16_t* c16 = reinterpret_cast<uint16_t*>(g.C);
    for (int c0 = 0; c0 < nt16; c0 += 16) {
        uint32_t v[16];
        if (have_acc) {
            tmem_ld_32x32b_x16(tl + (uint32_t)c0, v);
            tmem_wait_ld();
        } else {
#pragma unroll
            for (int e = 0; e < 16; ++e) v[e] = 0u;
        }
        if (!row_ok) continue;
        const int64_t col = n0 + c0;
        const bool full = col + 16 <= g.N;
        if (g.c16 && g.splits == 1) {
            uint16_t* dst = c16 + row * g.ldc + col;
            if (full && g.ldc % 8 == 0 && ((uintptr_t)dst & 15) == 0) {
                uint32_t pk[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) pk[e] = pack16x2<FMT>(__uint_as_float(v[2 * e]), __uint_as_float(v[2 * e + 1]));
                reinterpret_cast<uint4*>(dst)[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                reinterpret_cast<uint4*>(dst)[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            } else {
                for (int e = 0; e < 16 && col + e < g.N; ++e)
                    dst[e] = (uint16_t)(pack16x2<FMT>(__uint_as_float(v[e]), 0.f) & 0xFFFFu);
            }
        } else {
            float* dst = c32 + row * g.ldc + col;
            if (full && g.ldc % 4 == 0 && ((uintptr_t)dst & 15) == 0) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    reinterpret_cast<float4*>(dst)[q] = make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                                                    __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
            } else {
                for (int e = 0; e < 16 && col + e < g.N; ++e) dst[e] = __uint_as_float(v[e]);
            }
        }
    }
}

template <int FMT>
__global__ void __launch_bounds__(GT_THREADS, 1) gemm_tc_kernel(const __grid_constant__ TcGemm g) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_addr(smem_raw);
    uint8_t* base = smem_raw + ((1024u - (raw_addr & 1023u)) & 1023u);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const int64_t m0 = (int64_t)blockIdx.y * GT_M, n0 = (int64_t)blockIdx.x * GT_NMAX;
    const int nt = (int)(g.N - n0 < GT_NMAX ? g.N - n0 : GT_NMAX);   // columns of this tile
    const int nt16 = (nt + 15) & ~15;                                  // MMA N
    const int ntp = (nt + 63) & ~63;                                   // B rows loaded (64-row atoms)
    const uint32_t b_bytes = (uint32_t)ntp * 128u;
    const uint32_t stage_bytes = GT_A_BYTES + b_bytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + (size_t)GT_STAGES * stage_bytes);
    uint64_t* empty = bars;                       // [GT_STAGES] the MMAs of the stage's block are done
    uint64_t* done = bars + 2 * GT_STAGES;        // every MMA of the tile is done
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
    float* red = reinterpret_cast<float*>(bars + 2 * GT_STAGES + 2);   // masked epilogue: 4 x GT_NMAX
    const uint32_t tmem_cols = nt16 <= 32 ? 32u : nt16 <= 64 ? 64u : nt16 <= 128 ? 128u : 256u;

    if (tid == 0) {
        for (int s = 0; s < GT_STAGES; ++s) mbar_init(&empty[s], 1);
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(tmem_holder, tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    // this CTA's K blocks
    const int64_t nkb_all = (g.K + GT_KB - 1) / GT_KB;
    const int64_t per = (nkb_all + g.splits - 1) / g.splits;
    const int64_t kb0 = (int64_t)blockIdx.z * per;
    const int64_t kb1 = kb0 + per < nkb_all ? kb0 + per : nkb_all;
    const int nkb = kb1 > kb0 ? (int)(kb1 - kb0) : 0;
    const bool fast_a = g.lda % 8 == 0 && ((uintptr_t)g.A & 15) == 0;
    const bool fast_b = g.ldb % 8 == 0 && ((uintptr_t)g.B & 15) == 0;
    const uint32_t idesc = f16_idesc((uint32_t)FMT, 128u, (uint32_t)nt16) | ((uint32_t)g.a_mn << 15) |
                           ((uint32_t)g.b_mn << 16);
    const uint64_t lim = g.timeout_ns;
    uint4 hb[4][2];   // masked form: the first mask chunks of this thread's row
    mask_preload(g, m0, n0, nt, warp, lane, hb);

    auto load = [&](int j) {   // K block kb0 + j into stage j % GT_STAGES
        uint8_t* st = base + (size_t)(j % GT_STAGES) * stage_bytes;
        const int64_t k0 = (kb0 + j) * GT_KB;
        load_block(st, g.A, g.lda, g.a_mn, m0, g.M, GT_M, k0, g.K, fast_a, tid);
        load_block(st + GT_A_BYTES, g.B, g.ldb, g.b_mn, n0, g.N, ntp, k0, g.K, fast_b, tid);
    };

    bool ok = true;
    for (int j = 0; j < GT_STAGES - 1; ++j) {
        if (j < nkb) load(j);
        cp_async_commit();
    }
    for (int j = 0; j < nkb; ++j) {
        cp_async_wait<GT_STAGES - 2>();   // this thread's copies of block j have landed
        fence_proxy_async_smem();         // ... and are visible to the tensor core
        __syncthreads();                  // every thread's copies of block j
        if (tid == 0 && ok) {
            tc_fence_after();
            uint8_t* st = base + (size_t)(j % GT_STAGES) * stage_bytes;
            const uint32_t sa = smem_addr(st), sb = smem_addr(st + GT_A_BYTES);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {   // K = 16 per instruction
                const uint64_t ad = g.a_mn ? mn128_desc(sa + 2048u * kk, 8192u, 1024u) : sw128_desc(sa) + 2u * kk;
                const uint64_t bd = g.b_mn ? mn128_desc(sb + 2048u * kk, 8192u, 1024u) : sw128_desc(sb) + 2u * kk;
                umma_f16(tmem, ad, bd, idesc, (j | kk) != 0);
            }
            umma_commit(&empty[j % GT_STAGES]);
        }
        // refill the stage of block j - 1 with block j + GT_STAGES - 1 once block j - 1's MMAs are done
        const int jn = j + GT_STAGES - 1;
        if (jn < nkb) {
            if (j >= 1 && ok)
                ok = mbar_wait_bounded(&empty[(j - 1) % GT_STAGES], (uint32_t)((j - 1) / GT_STAGES) & 1u,
                                       g.status_word, abort_flag, lim);
            if (ok) load(jn);
        }
        cp_async_commit();
    }
    cp_async_wait<0>();
    if (tid == 0) {
        if (nkb > 0) umma_commit(done);
        else mbar_arrive(done);   // no K block: the tile is zero (not read from TMEM)
    }
    const bool got = mbar_wait_bounded(done, 0, g.status_word, abort_flag, lim) && ok;
    __syncwarp();
    tc_fence_after();

    if (g.mask_h) gemm_epilogue_mask<FMT>(g, tmem, m0, n0, nt, nt16, nkb > 0, got, warp, lane, red, hb);
    else gemm_epilogue<FMT>(g, tmem, m0, n0, nt16, nkb > 0, got, warp, lane);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, tmem_cols);
    }
}

// The TMA form: warp 0 lane 0 fills the stages, warp 1 lane 0 issues the
// MMAs, the four warps drain.
template <int FMT>
__global__ void __launch_bounds__(GT_THREADS, 1) gemm_tc_tma_kernel(const __grid_constant__ TcGemm g) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_addr(smem_raw);
    uint8_t* base = smem_raw + ((1024u - (raw_addr & 1023u)) & 1023u);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const int64_t m0 = (int64_t)blockIdx.y * GT_M, n0 = (int64_t)blockIdx.x * GT_NMAX;
    const int nt = (int)(g.N - n0 < GT_NMAX ? g.N - n0 : GT_NMAX);
    const int nt16 = (nt + 15) & ~15;
    const int ntp = g.box_b;                         // B rows per K block (64-multiple)
    const uint32_t b_bytes = (uint32_t)ntp * 128u;
    const uint32_t stage_bytes = GT_A_BYTES + b_bytes;
    const int NS = g.stages;                         // ring depth, 2 .. GT_STAGES
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + (size_t)NS * stage_bytes);
    uint64_t* full = bars;                           // [NS] the stage's block has landed
    uint64_t* empty = bars + GT_STAGES;              // [NS] the MMAs of the stage's block are done
    uint64_t* done = bars + 2 * GT_STAGES;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
    float* red = reinterpret_cast<float*>(bars + 2 * GT_STAGES + 2);   // masked epilogue: 4 x GT_NMAX
    const uint32_t tmem_cols = nt16 <= 32 ? 32u : nt16 <= 64 ? 64u : nt16 <= 128 ? 128u : 256u;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(tmem_holder, tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    const int64_t nkb_all = (g.K + GT_KB - 1) / GT_KB;
    const int64_t per = (nkb_all + g.splits - 1) / g.splits;
    const int64_t kb0 = (int64_t)blockIdx.z * per;
    const int64_t kb1 = kb0 + per < nkb_all ? kb0 + per : nkb_all;
    const int nkb = kb1 > kb0 ? (int)(kb1 - kb0) : 0;
    const uint64_t lim = g.timeout_ns;
    uint4 hb[4][2];   // masked form: the first mask chunks of this thread's row
    mask_preload(g, m0, n0, nt, warp, lane, hb);

    if (warp == 0 && lane == 0) {
        // ---- producer: K block j -> stage j % NS once its previous block's MMAs are done
        int issued = 0;
        for (int j = 0; j < nkb; ++j) {
            const int st = j % NS;
            if (j >= NS && !mbar_wait_bounded(&empty[st], (uint32_t)(j / NS - 1) & 1u, g.status_word, abort_flag, lim))
                break;
            uint8_t* sa = base + (size_t)st * stage_bytes;
            uint8_t* sb = sa + GT_A_BYTES;
            const int32_t k0 = (int32_t)((kb0 + j) * GT_KB);
            mbar_expect_tx(&full[st], stage_bytes);
            if (g.a_mn) {
                tma_load_2d(sa, &g.tma_a, (int32_t)m0, k0, &full[st]);
                tma_load_2d(sa + 8192, &g.tma_a, (int32_t)m0 + 64, k0, &full[st]);
            } else {
                tma_load_2d(sa, &g.tma_a, k0, (int32_t)m0, &full[st]);
            }
            if (g.b_mn) {
                for (int a = 0; a < ntp / 64; ++a) tma_load_2d(sb + 8192 * a, &g.tma_b, (int32_t)n0 + 64 * a, k0, &full[st]);
            } else {
                tma_load_2d(sb, &g.tma_b, k0, (int32_t)n0, &full[st]);
            }
            issued = j + 1;
        }
        // the copies in flight land before the CTA exits (the last fill of every stage)
        for (int j = issued > NS ? issued - NS : 0; j < issued; ++j)
            if (!mbar_wait_drain(&full[j % NS], (uint32_t)(j / NS) & 1u, lim))
                atomicOr(g.status_word, ADV_DEV_TIMEOUT);
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        const uint32_t idesc = f16_idesc((uint32_t)FMT, 128u, (uint32_t)nt16) | ((uint32_t)g.a_mn << 15) |
                               ((uint32_t)g.b_mn << 16);
        bool ok = true;
        for (int j = 0; j < nkb && ok; ++j) {
            const int st = j % NS;
            ok = mbar_wait_bounded(&full[st], (uint32_t)(j / NS) & 1u, g.status_word, abort_flag, lim);
            if (!ok) break;
            tc_fence_after();
            const uint32_t sa = smem_addr(base + (size_t)st * stage_bytes), sb = sa + GT_A_BYTES;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint64_t ad = g.a_mn ? mn128_desc(sa + 2048u * kk, 8192u, 1024u) : sw128_desc(sa) + 2u * kk;
                const uint64_t bd = g.b_mn ? mn128_desc(sb + 2048u * kk, 8192u, 1024u) : sw128_desc(sb) + 2u * kk;
                umma_f16(tmem, ad, bd, idesc, (j | kk) != 0);
            }
            umma_commit(&empty[st]);
        }
        if (nkb > 0) umma_commit(done);   // also when stopped early: the issued MMAs complete before TMEM is freed
        else mbar_arrive(done);
    }
    __syncwarp();   // the other lanes of warps 0 and 1 park here while lane 0 works
    const bool got = mbar_wait_bounded(done, 0, g.status_word, abort_flag, lim) && !*abort_flag;
    __syncwarp();
    tc_fence_after();
    if (g.mask_h) gemm_epilogue_mask<FMT>(g, tmem, m0, n0, nt, nt16, nkb > 0, got, warp, lane, red, hb);
    else gemm_epilogue<FMT>(g, tmem, m0, n0, nt16, nkb > 0, got, warp, lane);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, tmem_cols);
    }
}

// C[m][n] = sum over the splits of part[s][m][n] (FP32), in a fixed order:
// the splits in 8 consecutive groups, each summed in split order, then the
// group sums in group order.  Block of 256 threads: 32 groups of 4 columns
// (float4) x 8 split groups; needs N, ldc multiples of 4 and 16-byte aligned
// arrays (else gemm_split_sum_kernel).
__global__ void __launch_bounds__(256) gemm_split_sum4_kernel(const float* __restrict__ part, int splits, int64_t M,
                                                              int64_t N, int64_t ldc, float* __restrict__ C) {
    __shared__ float4 red[8][32];
    const int cg = threadIdx.x & 31, sg = threadIdx.x >> 5;
    const int64_t n4 = N / 4, total4 = M * n4;
    const int64_t i = (int64_t)blockIdx.x * 32 + cg;
    const size_t stride = (size_t)M * ldc;
    const int per = (splits + 7) / 8, z0 = sg * per, z1 = z0 + per < splits ? z0 + per : splits;
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < total4) {
        const int64_t m = i / n4, n = (i % n4) * 4;
        const float* p = part + m * ldc + n;
        int z = z0;
        for (; z + 4 <= z1; z += 4) {   // four loads in flight, added in split order
            const float4 a0 = *reinterpret_cast<const float4*>(p + (size_t)z * stride);
            const float4 a1 = *reinterpret_cast<const float4*>(p + (size_t)(z + 1) * stride);
            const float4 a2 = *reinterpret_cast<const float4*>(p + (size_t)(z + 2) * stride);
            const float4 a3 = *reinterpret_cast<const float4*>(p + (size_t)(z + 3) * stride);
            s.x = (((s.x + a0.x) + a1.x) + a2.x) + a3.x;
            s.y = (((s.y + a0.y) + a1.y) + a2.y) + a3.y;
            s.z = (((s.z + a0.z) + a1.z) + a2.z) + a3.z;
            s.w = (((s.w + a0.w) + a1.w) + a2.w) + a3.w;
        }
        for (; z < z1; ++z) {
            const float4 a = *reinterpret_cast<const float4*>(p + (size_t)z * stride);
            s.x += a.x;
            s.y += a.y;
            s.z += a.z;
            s.w += a.w;
        }
    }
    red[sg][cg] = s;
    __syncthreads();
    if (sg == 0 && i < total4) {
        float4 t = red[0][cg];
        for (int q = 1; q < 8; ++q) {
            t.x += red[q][cg].x;
            t.y += red[q][cg].y;
            t.z += red[q][cg].z;
            t.w += red[q][cg].w;
        }
        const int64_t m = i / n4, n = (i % n4) * 4;
        *reinterpret_cast<float4*>(C + m * ldc + n) = t;
    }
}

// The same sum for any N, ldc: one element per thread, splits in order.
__global__ void gemm_split_sum_kernel(const float* __restrict__ part, int splits, int64_t M, int64_t N, int64_t ldc,
                                      float* __restrict__ C) {
    const int64_t total = M * N;
    const size_t stride = (size_t)M * ldc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = i / N, n = i % N;
        const float* p = part + m * ldc + n;
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += p[(size_t)z * stride];
        C[m * ldc + n] = s;
    }
}


// ---- ReLU backward through a hidden layer: the persistent masked GEMM ---------
//
// Warp 0 lane 0 loads W once (KB x NA MN-major atoms: K block kb of fo, 64
// columns a of fi) and streams the 128-row K-major blocks of dza through a
// DG_SA-deep ring; warp 1 lane 0 issues the MMAs into one of two TMEM
// accumulators (tile i into buffer i % 2); warps 2..9 drain them: TMEM lane
// quadrant q = warp % 4 (rows 32 q .. 32 q + 31 of the tile), and of the
// 64-column boxes a of those rows the even ones (warps 2..5) or the odd ones
// (warps 6..9).  Rows 32 q .. 32 q + 31 of h sit in shared memory as NA TMA
// boxes {64, 32} (128-byte swizzle); a drain warp overwrites its boxes in
// place with dz and stores each back with TMA, then loads the next tile's h
// into the box as soon as the store has read it.  Column sums of the stored dz accumulate in registers
// over the CTA's tiles: lane 2u holds column 8 b4 + 4 b3 + 2 b2 + b1 of each
// 16-column chunk (b_i the bits of 2u).
constexpr int DG_THREADS = 320;
constexpr int DG_SA = 2;                  // ring depth of the dza blocks (16 KB each)

struct DgradArgs {
    CUtensorMap tm_a, tm_w, tm_h, tm_dz;
    int64_t n;
    int fo, fi;
    float* colpart;                      // [4 gridDim.x][fi]
    int* status_word;
    uint64_t timeout_ns;
};

__host__ __device__ __forceinline__ int dg_acc_cols(int fi) {   // TMEM columns of one accumulator
    const int nt16 = (fi + 15) & ~15;
    return nt16 <= 32 ? 32 : nt16 <= 64 ? 64 : nt16 <= 128 ? 128 : 256;
}

__host__ __device__ __forceinline__ size_t dg_smem_bytes(int fo, int fi) {
    const int KB = (fo + 63) / 64, NA = (fi + 63) / 64;
    return 1024 + (size_t)KB * NA * 8192 + (size_t)DG_SA * 16384 + (size_t)4 * NA * 4096 + 32 * 8;
}

template <int FMT>
__global__ void __launch_bounds__(DG_THREADS, 1) dgrad_mask_kernel(const __grid_constant__ DgradArgs g) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_addr(smem_raw);
    uint8_t* base = smem_raw + ((1024u - (raw_addr & 1023u)) & 1023u);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int KB = (g.fo + 63) / 64, NA = (g.fi + 63) / 64;
    const int nt16 = (g.fi + 15) & ~15;
    const uint32_t acc_cols = (uint32_t)dg_acc_cols(g.fi);
    uint8_t* w_s = base;                                     // KB x NA atoms of 8 KB
    uint8_t* a_s = w_s + (size_t)KB * NA * 8192;             // DG_SA x 16 KB
    uint8_t* h_s = a_s + (size_t)DG_SA * 16384;              // 4 quadrants x NA boxes of 4 KB
    uint64_t* bars = reinterpret_cast<uint64_t*>(h_s + (size_t)4 * NA * 4096);
    uint64_t* w_full = bars;                                 // W has landed
    uint64_t* a_full = bars + 1;                             // [DG_SA] a dza block has landed
    uint64_t* a_empty = a_full + DG_SA;                      // [DG_SA] its MMAs are done
    uint64_t* acc_full = a_empty + DG_SA;                    // [2] an accumulator holds a finished tile
    uint64_t* acc_empty = acc_full + 2;                      // [2] the eight drain warps have read it
    uint64_t* h_full = acc_empty + 2;                        // [4 x 4] box a of quadrant q has landed
    uint64_t* fin = h_full + 16;                             // every MMA issued has completed
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(fin + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

    const int64_t tiles = (g.n + 127) / 128;
    const int my_tiles = tiles > (int64_t)blockIdx.x ? (int)((tiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    const uint64_t lim = g.timeout_ns;

    if (tid == 0) {
        mbar_init(w_full, 1);
        for (int s = 0; s < DG_SA; ++s) {
            mbar_init(&a_full[s], 1);
            mbar_init(&a_empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 8);
        }
        for (int i = 0; i < 16; ++i) mbar_init(&h_full[i], 1);
        mbar_init(fin, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_holder, 2 * acc_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer: W once, then the dza blocks of every tile through the ring
            mbar_expect_tx(w_full, (uint32_t)(KB * NA * 8192));
            for (int kb = 0; kb < KB; ++kb)
                for (int a = 0; a < NA; ++a)
                    tma_load_2d(w_s + (size_t)(kb * NA + a) * 8192, &g.tm_w, 64 * a, 64 * kb, w_full);
            int j = 0;   // blocks issued
            bool ok = true;
            for (int i = 0; i < my_tiles && ok; ++i) {
                const int32_t row0 = (int32_t)((blockIdx.x + (int64_t)i * gridDim.x) * 128);
                for (int kb = 0; kb < KB; ++kb) {
                    const int st = j % DG_SA;
                    if (j >= DG_SA &&
                        !(ok = mbar_wait_bounded(&a_empty[st], (uint32_t)(j / DG_SA - 1) & 1u, g.status_word,
                                                 abort_flag, lim)))
                        break;
                    mbar_expect_tx(&a_full[st], 16384u);
                    tma_load_2d(a_s + (size_t)st * 16384, &g.tm_a, 64 * kb, row0, &a_full[st]);
                    ++j;
                }
            }
            // the copies in flight land before the CTA exits
            if (!mbar_wait_drain(w_full, 0, lim)) atomicOr(g.status_word, ADV_DEV_TIMEOUT);
            for (int jj = j > DG_SA ? j - DG_SA : 0; jj < j; ++jj)
                if (!mbar_wait_drain(&a_full[jj % DG_SA], (uint32_t)(jj / DG_SA) & 1u, lim))
                    atomicOr(g.status_word, ADV_DEV_TIMEOUT);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer: B = W (MN-major), A = the dza block (K-major)
            const uint32_t idesc = f16_idesc((uint32_t)FMT, 128u, (uint32_t)nt16) | (1u << 16);
            bool ok = mbar_wait_bounded(w_full, 0, g.status_word, abort_flag, lim);
            bool issued = false;
            int j = 0;
            for (int i = 0; i < my_tiles && ok; ++i) {
                const int b = i & 1;
                if (i >= 2 &&
                    !(ok = mbar_wait_bounded(&acc_empty[b], (uint32_t)((i >> 1) - 1) & 1u, g.status_word, abort_flag,
                                             lim)))
                    break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)b * acc_cols;
                for (int kb = 0; kb < KB; ++kb, ++j) {
                    const int st = j % DG_SA;
                    if (!(ok = mbar_wait_bounded(&a_full[st], (uint32_t)(j / DG_SA) & 1u, g.status_word, abort_flag,
                                                 lim)))
                        break;
                    tc_fence_after();
                    const uint32_t sa = smem_addr(a_s + (size_t)st * 16384);
                    const uint32_t sb = smem_addr(w_s + (size_t)kb * NA * 8192);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        umma_f16(d, sw128_desc(sa) + 2u * kk, mn128_desc(sb + 2048u * kk, 8192u, 1024u), idesc,
                                 (kb | kk) != 0);
                    issued = true;
                    umma_commit(&a_empty[st]);
                }
                if (!ok) break;
                umma_commit(&acc_full[b]);
            }
            if (issued) umma_commit(fin);   // arrives when every MMA above has completed
            else mbar_arrive(fin);
        }
        __syncwarp();
    } else {
        // ---- drain warps
        const int q = warp & 3, half = (warp - 2) >> 2;   // TMEM quadrant; even or odd boxes
        uint8_t* hq = h_s + (size_t)q * NA * 4096;
        uint64_t* hf = h_full + 4 * q;
        const int colid = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
        uint32_t pend = 0, par = 0;   // boxes with a load in flight, and the parity it completes
        auto load_h = [&](int a, int32_t row, int tile_i) {
            mbar_expect_tx(&hf[a], 4096u);
            tma_load_2d(hq + (size_t)a * 4096, &g.tm_h, 64 * a, row, &hf[a]);
            pend |= 1u << a;
            par = (par & ~(1u << a)) | ((uint32_t)(tile_i & 1) << a);
        };
        if (lane == 0 && my_tiles > 0)
            for (int a = half; a < NA; a += 2) load_h(a, (int32_t)(blockIdx.x * 128 + 32 * q), 0);
        float csum[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) csum[e] = 0.f;
        bool ok = true;
        for (int i = 0; i < my_tiles && ok; ++i) {
            const int64_t t = blockIdx.x + (int64_t)i * gridDim.x;
            const int32_t r0 = (int32_t)(t * 128 + 32 * q);
            const int32_t r0_next = (int32_t)((t + gridDim.x) * 128 + 32 * q);
            const bool more = i + 1 < my_tiles;
            const int b = i & 1;
            ok = __all_sync(0xffffffffu,
                            mbar_wait_bounded(&acc_full[b], (uint32_t)(i >> 1) & 1u, g.status_word, abort_flag, lim));
            if (!ok) break;
            tc_fence_after();
            const uint32_t tl = tmem + (uint32_t)b * acc_cols + ((uint32_t)(32 * q) << 16);
            int prev = -1;   // the box stored before this one
#pragma unroll
            for (int ai = 0; ai < 2; ++ai) {
                const int a = 2 * ai + half;
                if (a >= NA) break;
                ok = __all_sync(0xffffffffu,
                                mbar_wait_bounded(&hf[a], (uint32_t)i & 1u, g.status_word, abort_flag, lim));
                if (!ok) break;
                pend &= ~(1u << a);
                uint8_t* rowp = hq + (size_t)a * 4096 + (size_t)lane * 128;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int c0 = 64 * a + 16 * c;
                    if (c0 >= nt16) break;
                    uint32_t v[16];
                    tmem_ld_32x32b_x16(tl + (uint32_t)c0, v);
                    tmem_wait_ld();
                    uint4* p0 = reinterpret_cast<uint4*>(rowp + (((2 * c) ^ (lane & 7)) << 4));
                    uint4* p1 = reinterpret_cast<uint4*>(rowp + (((2 * c + 1) ^ (lane & 7)) << 4));
                    const uint4 h0 = *p0, h1 = *p1;
                    const uint32_t hw[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
                    uint32_t pk[8];
                    float qv[16];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const float x0 = pos16<FMT>(hw[e] & 0xFFFFu) ? __uint_as_float(v[2 * e]) : 0.f;
                        const float x1 = pos16<FMT>(hw[e] >> 16) ? __uint_as_float(v[2 * e + 1]) : 0.f;
                        pk[e] = pack16x2<FMT>(x0, x1);
                        if constexpr (FMT == 1) {
                            qv[2 * e] = __uint_as_float(pk[e] << 16);
                            qv[2 * e + 1] = __uint_as_float(pk[e] & 0xFFFF0000u);
                        } else {
                            qv[2 * e] = __half2float(__ushort_as_half((unsigned short)(pk[e] & 0xFFFFu)));
                            qv[2 * e + 1] = __half2float(__ushort_as_half((unsigned short)(pk[e] >> 16)));
                        }
                    }
                    *p0 = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    *p1 = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                    csum[4 * ai + c] += warp_colsum16(qv, lane);
                }
                fence_proxy_async_smem();   // the writes above, before the TMA store reads them
                __syncwarp();
                if (lane == 0) {
                    if (r0 < g.n) tma_store_2d(&g.tm_dz, hq + (size_t)a * 4096, 64 * a, r0);   // rows past n are clipped
                    bulk_commit();
                    if (prev >= 0 && more) {   // the previous box has been stored: the next tile's h into it
                        bulk_wait_read<1>();
                        load_h(prev, r0_next, i + 1);
                    }
                }
                prev = a;
            }
            if (!ok) break;
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&acc_empty[b]);
                if (prev >= 0 && more) {
                    bulk_wait_read<0>();
                    load_h(prev, r0_next, i + 1);
                }
            }
        }
        if (lane == 0) {
            bulk_wait_all();   // the dz stores are complete
            for (int a = half; a < NA; a += 2)   // loads still in flight land (only after an abort)
                if ((pend >> a) & 1u)
                    if (!mbar_wait_drain(&hf[a], (par >> a) & 1u, lim)) atomicOr(g.status_word, ADV_DEV_TIMEOUT);
        }
        if (ok) {
#pragma unroll
            for (int ai = 0; ai < 2; ++ai)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int a = 2 * ai + half, col = 64 * a + 16 * c + colid;
                    if ((lane & 1) == 0 && a < NA && col < g.fi)
                        g.colpart[((size_t)blockIdx.x * 4 + q) * g.fi + col] = csum[4 * ai + c];
                }
        }
    }
    __syncthreads();
    if (warp == 1) {
        if (!mbar_wait_drain(fin, 0, lim) && lane == 0) atomicOr(g.status_word, ADV_DEV_TIMEOUT);
        tc_fence_after();
        tmem_dealloc(tmem, 2 * acc_cols);
    }
}

}  // namespace

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once (a function-local static is
// initialised once even when several threads call this first).
EncodeTiledFn encode_fn() {
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
        return nullptr;
    }();
    return fn;
}

// Tensor map of a row-major 16-bit operand: rows of `ld` values; read as
// K-major (rows along M/N: dims {K, rows}, box {64, box_rows}) or MN-major
// (rows along K: dims {rows, K}, box {64, 64}); 128-byte swizzle, zero fill.
bool make_map(CUtensorMap* map, const uint16_t* p, int64_t ld, int mn, int64_t rows, int64_t K, int box_rows, int fmt) {
    EncodeTiledFn fn = encode_fn();
    if (!fn || ((uintptr_t)p & 15) != 0 || (ld * 2) % 16 != 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)(mn ? rows : K), (cuuint64_t)(mn ? K : rows)};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {64u, (cuuint32_t)(mn ? 64 : box_rows)};
    const cuuint32_t estr[2] = {1u, 1u};
    return fn(map, fmt == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
              const_cast<uint16_t*>(p), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool encode_rows_map(CUtensorMap* map, const void* p, int64_t cols, int64_t rows, int box_rows, int fmt) {
    return make_map(map, reinterpret_cast<const uint16_t*>(p), cols, 0, rows, cols, box_rows, fmt);
}

// Dynamic shared memory: 1 KB of alignment slack, the ring, the barriers and
// TMEM holder (2 GT_STAGES + 2 words of 8 bytes), the masked epilogue's sums.
size_t gemm_tc_smem_bytes(int64_t N, int stages) {
    const int nt = (int)(N < GT_NMAX ? N : GT_NMAX);
    const size_t ntp = (size_t)((nt + 63) & ~63);
    return 1024 + (size_t)stages * (GT_A_BYTES + ntp * 128) + (2 * GT_STAGES + 2) * 8 + 4 * GT_NMAX * 4;
}

cudaError_t launch_gemm_tc(const TcGemm& g, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    if (g.splits < 1 || (g.splits > 1 && (g.part == nullptr || g.c16))) return cudaErrorInvalidValue;
    if (g.mask_h && (!g.c16 || g.splits != 1 || g.colpart == nullptr)) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((g.N + GT_NMAX - 1) / GT_NMAX), (unsigned)((g.M + GT_M - 1) / GT_M),
                    (unsigned)g.splits);
    TcGemm t = g;
    const int64_t nround = (g.N + 63) / 64 * 64;
    t.box_b = (int)(nround < GT_NMAX ? nround : GT_NMAX);
    t.use_tma = make_map(&t.tma_a, g.A, g.lda, g.a_mn, g.M, g.K, GT_M, g.fmt) &&
                make_map(&t.tma_b, g.B, g.ldb, g.b_mn, g.N, g.K, t.box_b, g.fmt);
    // K blocks per CTA; a short K (<= 4 blocks) takes a 2-deep ring so that two
    // CTAs share an SM and one's epilogue overlaps the other's loads
    const int64_t nkb_all = (g.K + GT_KB - 1) / GT_KB;
    const int64_t per = (nkb_all + g.splits - 1) / g.splits;
    t.stages = per <= 4 ? 2 : GT_STAGES;
    cudaError_t e;
    if (t.use_tma) {
        const size_t smem = gemm_tc_smem_bytes(g.N, t.stages);
        auto kern = g.fmt == 1 ? gemm_tc_tma_kernel<1> : gemm_tc_tma_kernel<0>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, GT_THREADS, smem, s>>>(t);
    } else {
        t.stages = GT_STAGES;
        const size_t smem = gemm_tc_smem_bytes(g.N, GT_STAGES);
        auto kern = g.fmt == 1 ? gemm_tc_kernel<1> : gemm_tc_kernel<0>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, GT_THREADS, smem, s>>>(t);
    }
    adv_count_launch(1);
    e = cudaGetLastError();
    if (e != cudaSuccess || g.splits == 1) return e;
    float* C = reinterpret_cast<float*>(g.C);
    if (g.N % 4 == 0 && g.ldc % 4 == 0 && ((uintptr_t)g.part & 15) == 0 && ((uintptr_t)C & 15) == 0) {
        const int64_t total4 = g.M * (g.N / 4);
        gemm_split_sum4_kernel<<<(unsigned)((total4 + 31) / 32), 256, 0, s>>>(g.part, g.splits, g.M, g.N, g.ldc, C);
    } else {
        const int64_t total = g.M * g.N;
        const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
        gemm_split_sum_kernel<<<blocks, 256, 0, s>>>(g.part, g.splits, g.M, g.N, g.ldc, C);
    }
    adv_count_launch(1);
    return cudaGetLastError();
}


cudaError_t launch_dgrad_mask(const uint16_t* dza, int fo, const uint16_t* W, int fi, const uint16_t* h, int64_t n,
                              uint16_t* dz, float* colpart, int64_t colpart_cap, int* parts, int fmt,
                              int* status_word, cudaStream_t s) {
    if (n <= 0) {
        *parts = 0;
        return cudaSuccess;
    }
    if (fo <= 0 || fi <= 0 || fo > 256 || fi > 256 || fo % 8 != 0 || fi % 8 != 0 || (((uintptr_t)dz) & 15) != 0)
        return cudaErrorNotSupported;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (n + 127) / 128;
    int64_t grid = tiles < sms ? tiles : sms;
    if (grid * 4 * fi > colpart_cap) grid = colpart_cap / (4 * (int64_t)fi);
    if (grid < 1) return cudaErrorNotSupported;
    DgradArgs a{};
    // dza: K-major A, rows of fo values; W: MN-major B ([fo][fi], rows along K);
    // h and dz: boxes of 64 columns x 32 rows
    if (!make_map(&a.tm_a, dza, fo, 0, n, fo, 128, fmt) || !make_map(&a.tm_w, W, fi, 1, fi, fo, 64, fmt) ||
        !make_map(&a.tm_h, h, fi, 0, n, fi, 32, fmt) || !make_map(&a.tm_dz, dz, fi, 0, n, fi, 32, fmt))
        return cudaErrorNotSupported;
    a.n = n;
    a.fo = fo;
    a.fi = fi;
    a.colpart = colpart;
    a.status_word = status_word;
    a.timeout_ns = 2000000000ull;
    // a CTA holding all 512 TMEM columns gets an SM of its own: a second CTA on
    // the SM would wait in tcgen05.alloc until the first finished
    size_t smem = dg_smem_bytes(fo, fi);
    if (2 * dg_acc_cols(fi) == 512 && smem < 120 * 1024) smem = 120 * 1024;
    auto kern = fmt == 1 ? dgrad_mask_kernel<1> : dgrad_mask_kernel<0>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, DG_THREADS, smem, s>>>(a);
    adv_count_launch(1);
    *parts = (int)(4 * grid);
    return cudaGetLastError();
}

}  // namespace adv
