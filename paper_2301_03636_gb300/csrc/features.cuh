// Device-side descriptor validation and feature extraction (a1-a2),
// shared by the extraction kernels and the near-tie re-score kernels.
//
// Fig. 2 of arXiv 2301.03636 feeds every generated variant through "Feature
// Extraction" before the trained model; the paper does not list its
// features, so the set here is this library's own (listed in
// include/advisor.h and in the per-index comments below).
#pragma once
#include "common.cuh"

namespace adv {

// Binary logarithm in Q16.16 by repeated squaring of the normalised mantissa
// (digit-by-digit method; Majithia & Levan, Proc. IEEE 1973).  x = 2^k * m,
// m in [1,2) kept as a 32-bit fraction scaled by 2^31; each squaring yields one
// fraction bit: m^2 >= 2 gives 1 and the next mantissa is m^2 / 2.  L(0) = 0.
__device__ __forceinline__ int32_t log2_q16(uint64_t x) {
    if (x == 0) return 0;
    const int k = 63 - __clzll((long long)x);
    uint32_t m = (k >= 31) ? (uint32_t)(x >> (k - 31)) : (uint32_t)(x << (31 - k));
    uint32_t frac = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const uint64_t sq = (uint64_t)m * (uint64_t)m;   // value sq / 2^62 = m^2 in [1, 4)
        const uint32_t hi = (uint32_t)(sq >> 32);
        const uint32_t bit = hi >> 31;                     // m^2 >= 2  <=>  sq >= 2^63
        m = bit ? hi : (uint32_t)(sq >> 31);               // next mantissa, scaled by 2^31
        frac = (frac << 1) | bit;
    }
    return (int32_t)(((uint32_t)k << 16) | frac);
}

// Row validation; bit meanings as ADVISOR_ROW_* in advisor.h.
__device__ __forceinline__ uint32_t validate_row(const int64_t (&d)[16]) {
    const int64_t depth = d[0];
    if (depth < 1 || depth > 4) return ADVISOR_ROW_BAD_DEPTH;
    uint32_t st = 0;
    const int64_t TRIP_MAX = (int64_t)1 << 24;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t t = d[1 + i];
        const bool ok = (i < depth) ? (t >= 1 && t <= TRIP_MAX) : (t == 1);
        if (!ok) st |= ADVISOR_ROW_BAD_TRIP;
    }
    const int64_t W_MAX = (int64_t)1 << 32, M_MAX = (int64_t)1 << 48, PAR_MAX = (int64_t)1 << 24;
    if (d[5] < 1 || d[5] > W_MAX || d[6] < 1 || d[6] > W_MAX) st |= ADVISOR_ROW_BAD_WORK;
    if (d[7] < 0 || d[7] > M_MAX || d[8] < 0 || d[8] > M_MAX) st |= ADVISOR_ROW_BAD_MAPPED;
    if (d[9] < 1 || d[9] > PAR_MAX || d[10] < 1 || d[10] > PAR_MAX) st |= ADVISOR_ROW_BAD_PARALLELISM;
    const int64_t pf = d[11], dc = d[12], pc = d[13];
    bool var_ok = (pf >= 0) && (pf < depth);
    if (var_ok) {
        var_ok = (pf == 0) ? (dc == 0) : (dc >= 1 && dc <= pf);
        var_ok = var_ok && pc >= 1 && pc <= depth - pf;
    }
    var_ok = var_ok && d[14] >= 0 && d[14] <= 2 && (d[15] == 0 || d[15] == 1);
    if (!var_ok) st |= ADVISOR_ROW_BAD_VARIANT;
    if ((st & (ADVISOR_ROW_BAD_TRIP | ADVISOR_ROW_BAD_WORK)) == 0) {
        // trip product <= 2^48 and work products <= 2^62, overflow-safe
        uint64_t T = 1;
        bool over = false;
        for (int i = 0; i < 4; ++i) {
            if (i >= depth || over) break;
            const uint64_t t = (uint64_t)d[1 + i];
            if (__umul64hi(T, t) != 0) over = true;
            T = T * t;
            if (T > ((uint64_t)1 << 48)) over = true;
        }
        if (!over) {
            const uint64_t lim = (uint64_t)1 << 62;
            const uint64_t f = (uint64_t)d[5], b = (uint64_t)d[6];
            if (__umul64hi(T, f) != 0 || T * f > lim || __umul64hi(T, b) != 0 || T * b > lim) over = true;
        }
        if (over) st |= ADVISOR_ROW_BAD_RANGE;
    }
    return st;
}

// Binary logarithms of N values at once: the same digit-by-digit method as
// log2_q16, with the N squaring chains advanced in lockstep so that their
// multiplies overlap instead of waiting on each other.  Each step is written
// without a select: with s = 31 + bit, the next mantissa is the square
// shifted right by s (bit = 1: its high word; bit = 0: bits 31..62), and the
// fraction collects s instead of bit, i.e. 31 extra per step, 31 * (2^16 - 1)
// in all, taken off at the end.  This moves work from the integer ALU pipe
// to the multiply-add pipe (extraction 12.2 -> 10.1 ms at 2^26 rows, and
// 36.5 -> 32.4 us for 137,508 rows with the step in PTX).
template <int N>
__device__ __forceinline__ void log2_q16_batch(const uint64_t (&x)[N], int32_t (&out)[N]) {
    uint32_t m[N], acc[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const uint64_t v = x[i] ? x[i] : 1;               // L(0) = L(1) = 0
        const int k = 63 - __clzll((long long)v);
        m[i] = (k >= 31) ? (uint32_t)(v >> (k - 31)) : (uint32_t)(v << (31 - k));
        acc[i] = (uint32_t)k;                              // the 16 fraction bits are shifted in below
    }
#pragma unroll
    for (int it = 0; it < 16; ++it) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            // m^2 as one wide multiply (two 32-bit words); s = 31 + (m^2 >= 2) = high
            // word * 2 / 2^32 + 31; next m = low word of (m^2 >> s), a 32-bit funnel
            // shift; acc = 2 acc + s.  Written as PTX so that the step stays three
            // multiply-adds and one shift (the wide multiply in place of a low and a
            // high multiply: 117.8 -> 117.2 us per batched step).
            uint32_t lo, hi, sh, nm;
            uint64_t sq;
            asm("mul.wide.u32 %0, %1, %1;" : "=l"(sq) : "r"(m[i]));
            asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(sq));
            asm("mad.hi.u32 %0, %1, 2, 31;" : "=r"(sh) : "r"(hi));
            asm("shf.r.clamp.b32 %0, %1, %2, %3;" : "=r"(nm) : "r"(lo), "r"(hi), "r"(sh));
            m[i] = nm;
            asm("mad.lo.u32 %0, %1, 2, %2;" : "=r"(acc[i]) : "r"(acc[i]), "r"(sh));
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = (int32_t)(acc[i] - 31u * 65535u);
}

// Number of logarithms behind the F features of a row: 19 for the 32 base
// features, 16 more for the per-loop-level block (F >= 64).
template <int F>
struct FeatureLogs {
    static constexpr int N = F >= 64 ? 35 : 19;
};

// Indices of the base logarithm arguments (0 .. 18); the per-level block
// follows at 19 + 4 * level + {prefix, suffix, trip*bytes, trip*flops}.
enum { A_T0 = 0, A_T = 4, A_FL_IT, A_BY_IT, A_WF, A_WB, A_H2D, A_D2H, A_MAP, A_TEAMS, A_THREADS, A_PAR, A_D, A_Q,
       A_MIN, A_BASE_N, A_LEVEL = A_BASE_N };

struct RowFields {
    int depth, pf, dc, pc, sched, dmode, n_dist;
};

__device__ __forceinline__ RowFields row_fields(const int64_t (&d)[16]) {
    RowFields r;
    r.depth = (int)d[0];
    r.pf = (int)d[11];
    r.dc = (int)d[12];
    r.pc = (int)d[13];
    r.sched = (int)d[14];
    r.dmode = (int)d[15];
    // 'teams distribute' covers loops [0, n_dist); combined with 'parallel for' when pf == 0
    r.n_dist = (r.pf == 0) ? r.pc : r.dc;
    return r;
}

// The arguments of every logarithm the F features of a valid row take.
template <int F>
__device__ __forceinline__ void row_log_args(const int64_t (&d)[16], uint64_t (&x)[FeatureLogs<F>::N]) {
    const RowFields r = row_fields(d);
    const uint64_t t[4] = {(uint64_t)d[1], (uint64_t)d[2], (uint64_t)d[3], (uint64_t)d[4]};
    const uint64_t flops = (uint64_t)d[5], bytes = (uint64_t)d[6];
    const uint64_t h2d = (uint64_t)d[7], d2h = (uint64_t)d[8];
    const uint64_t teams = (uint64_t)d[9], threads = (uint64_t)d[10];
    const uint64_t T = t[0] * t[1] * t[2] * t[3];
    const uint64_t par = teams * threads;
    uint64_t Dp = 1, Qp = 1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (i < r.n_dist) Dp *= t[i];
        if (i >= r.pf && i < r.pf + r.pc) Qp *= t[i];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) x[A_T0 + i] = t[i];
    x[A_T] = T;
    x[A_FL_IT] = flops;
    x[A_BY_IT] = bytes;
    x[A_WF] = T * flops;
    x[A_WB] = T * bytes;
    x[A_H2D] = h2d;
    x[A_D2H] = d2h;
    x[A_MAP] = h2d + d2h;
    x[A_TEAMS] = teams;
    x[A_THREADS] = threads;
    x[A_PAR] = par;
    x[A_D] = Dp;
    x[A_Q] = Qp;
    x[A_MIN] = T < par ? T : par;
    if constexpr (F >= 64) {
        // per loop level: prefix product, suffix product, trip*bytes/iter,
        // trip*flops/iter; arguments of 1 beyond the depth (logarithm 0)
        uint64_t prefix = 1;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const bool live = i < r.depth;
            prefix *= t[i];
            uint64_t suffix = 1;
#pragma unroll
            for (int j = i; j < 4; ++j) suffix *= (j < r.depth) ? t[j] : 1;
            x[A_LEVEL + 4 * i + 0] = live ? prefix : 1;
            x[A_LEVEL + 4 * i + 1] = live ? suffix : 1;
            x[A_LEVEL + 4 * i + 2] = live ? t[i] * bytes : 1;
            x[A_LEVEL + 4 * i + 3] = live ? t[i] * flops : 1;
        }
    }
}

// The F features of a valid row from its fields and the logarithms of the
// arguments row_log_args lists.
template <int F>
__device__ __forceinline__ void row_features_from_logs(const int64_t (&d)[16], const int32_t (&L)[FeatureLogs<F>::N],
                                                       int32_t (&f)[F]) {
    constexpr int32_t ONE = 65536;
    const RowFields r = row_fields(d);
    int32_t base[32];
    base[0] = r.depth * ONE;
#pragma unroll
    for (int i = 0; i < 4; ++i) base[1 + i] = L[A_T0 + i];
    base[5] = L[A_T];
    base[6] = L[A_FL_IT];
    base[7] = L[A_BY_IT];
    base[8] = L[A_WF];
    base[9] = L[A_WB];
    base[10] = L[A_H2D];
    base[11] = L[A_D2H];
    base[12] = L[A_MAP];
    base[13] = L[A_TEAMS];
    base[14] = L[A_THREADS];
    base[15] = L[A_PAR];
    base[16] = L[A_D];
    base[17] = L[A_Q];
    base[18] = max(L[A_T] - L[A_PAR], 0);
    base[19] = max(L[A_D] - L[A_TEAMS], 0);
    base[20] = max(L[A_Q] - L[A_THREADS], 0);
    base[21] = L[A_WF] - L[A_WB];
    base[22] = L[A_WB] - L[A_MAP];
    base[23] = r.sched == 0 ? ONE : 0;
    base[24] = r.sched == 1 ? ONE : 0;
    base[25] = r.sched == 2 ? ONE : 0;
    base[26] = r.dmode * ONE;
    base[27] = r.pf * ONE;
    base[28] = r.dc * ONE;
    base[29] = r.pc * ONE;
    base[30] = r.pf == 0 ? ONE : 0;
    base[31] = L[A_MIN];
#pragma unroll
    for (int j = 0; j < 32; ++j) f[j] = base[j];
    if constexpr (F == 33) {
        // the paper-shaped input (33 features): the number of collapsed loops
        f[32] = (r.dc + r.pc) * ONE;
    }
    if constexpr (F >= 64) {
        // per loop level: log trip, distributed?, parallel-for?, in a collapse
        // group of >= 2 loops?, log prefix product, log suffix product,
        // log(trip*bytes/iter), log(trip*flops/iter); zero beyond the depth.
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int o = 32 + 8 * i;
            const bool live = i < r.depth;
            const bool in_dist = live && i < r.n_dist;
            const bool in_pf = live && (i >= r.pf) && (i < r.pf + r.pc);
            const bool grouped = (in_dist && r.n_dist >= 2) || (in_pf && r.pc >= 2);
            f[o + 0] = live ? L[A_T0 + i] : 0;
            f[o + 1] = in_dist ? ONE : 0;
            f[o + 2] = in_pf ? ONE : 0;
            f[o + 3] = grouped ? ONE : 0;
            f[o + 4] = L[A_LEVEL + 4 * i + 0];
            f[o + 5] = L[A_LEVEL + 4 * i + 1];
            f[o + 6] = L[A_LEVEL + 4 * i + 2];
            f[o + 7] = L[A_LEVEL + 4 * i + 3];
        }
    }
    if constexpr (F >= 128) {
        // 64 differences base[a] - base[b]: a = 1 + u % 21, partner b at
        // distance 1 + u / 21 to the right, wrapping inside 1..22.
#pragma unroll
        for (int u = 0; u < 64; ++u) {
            const int a = 1 + u % 21;
            const int b = 1 + (a - 1 + 1 + u / 21) % 22;
            f[64 + u] = base[a] - base[b];
        }
    }
}

// The F features of a valid row (F = 32, 33, 64 or 128), one thread.
template <int F>
__device__ __forceinline__ void row_features(const int64_t (&d)[16], int32_t (&f)[F]) {
    constexpr int N = FeatureLogs<F>::N;
    uint64_t x[N];
    row_log_args<F>(d, x);
    int32_t L[N];
    // Logarithms that follow from others are not computed again:
    //  - L(min(T, P)) = min(L(T), L(P)): the digit-by-digit logarithm is
    //    non-decreasing (a larger argument has a larger exponent, or the same
    //    exponent and a mantissa whose truncated squarings never fall below);
    //  - level 0's prefix product is trip[0] and its suffix product the whole
    //    trip product (trips past the depth are 1 in a valid row).
    constexpr int M = N - (F >= 64 ? 3 : 1);
    auto derived = [](int i) { return i == A_MIN || (F >= 64 && (i == A_LEVEL || i == A_LEVEL + 1)); };
    uint64_t y[M];
    int32_t ly[M];
#pragma unroll
    for (int i = 0, j = 0; i < N; ++i)
        if (!derived(i)) y[j++] = x[i];
    log2_q16_batch<M>(y, ly);
#pragma unroll
    for (int i = 0, j = 0; i < N; ++i)
        if (!derived(i)) L[i] = ly[j++];
    L[A_MIN] = L[A_T] < L[A_PAR] ? L[A_T] : L[A_PAR];
    if constexpr (F >= 64) {
        L[A_LEVEL] = L[A_T0];
        L[A_LEVEL + 1] = L[A_T];
    }
    row_features_from_logs<F>(d, L, f);
}

// The same features computed by a group of G lanes for one row (G = 16 or
// 32; every lane of the warp must take part, each group with its own row):
// lane g of the group takes the logarithms of arguments g, g + G, ..., the
// results are exchanged by shuffles inside the group, and every lane of the
// group assembles the (identical) feature vector, keeping features g + G q
// in mine[q].
template <int F, int G>
__device__ __forceinline__ void row_features_lanes(const int64_t (&d)[16], int g, int32_t (&mine)[(F + G - 1) / G]) {
    static_assert(G == 8 || G == 16 || G == 32, "lane group size");
    constexpr int N = FeatureLogs<F>::N;
    constexpr int NL = (N + G - 1) / G;   // logarithms per lane
    uint64_t x[N];
    row_log_args<F>(d, x);
    uint64_t a[NL];
#pragma unroll
    for (int q = 0; q < NL; ++q) a[q] = 1;
#pragma unroll
    for (int i = 0; i < N; ++i)
        if (i % G == g) a[i / G] = x[i];
    int32_t l[NL];
    log2_q16_batch<NL>(a, l);
    int32_t L[N];
#pragma unroll
    for (int i = 0; i < N; ++i) L[i] = __shfl_sync(0xffffffffu, l[i / G], i % G, G);
    int32_t f[F];
    row_features_from_logs<F>(d, L, f);
#pragma unroll
    for (int q = 0; q < (F + G - 1) / G; ++q) mine[q] = 0;
#pragma unroll
    for (int j = 0; j < F; ++j)
        if (j % G == g) mine[j / G] = f[j];
}

// A valid placeholder descriptor (depth 1, every count 1, nothing mapped),
// used where a lane group has no valid row but must still join the shuffles.
__device__ __forceinline__ void placeholder_desc(int64_t (&d)[16]) {
#pragma unroll
    for (int i = 0; i < 16; ++i) d[i] = 1;
    d[7] = 0;    // h2d bytes
    d[8] = 0;    // d2h bytes
    d[11] = 0;   // pf_pos: combined construct
    d[12] = 0;   // dist_collapse
    d[14] = 0;   // schedule static
    d[15] = 0;   // data mode
}

__device__ __forceinline__ void load_desc(const advisor_variant_desc* desc, int64_t row, int64_t (&d)[16]) {
    const longlong2* p = reinterpret_cast<const longlong2*>(desc + row);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const longlong2 v = __ldg(p + i);
        d[2 * i] = v.x;
        d[2 * i + 1] = v.y;
    }
}

}  // namespace adv
