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

// The F features of a valid row (F = 32, 64 or 128).
template <int F>
__device__ __forceinline__ void row_features(const int64_t (&d)[16], int32_t (&f)[F]) {
    constexpr int32_t ONE = 65536;
    const int depth = (int)d[0];
    const uint64_t t[4] = {(uint64_t)d[1], (uint64_t)d[2], (uint64_t)d[3], (uint64_t)d[4]};
    const uint64_t flops = (uint64_t)d[5], bytes = (uint64_t)d[6];
    const uint64_t h2d = (uint64_t)d[7], d2h = (uint64_t)d[8];
    const uint64_t teams = (uint64_t)d[9], threads = (uint64_t)d[10];
    const int pf = (int)d[11], dc = (int)d[12], pc = (int)d[13], sched = (int)d[14], dmode = (int)d[15];

    const uint64_t T = t[0] * t[1] * t[2] * t[3];
    const uint64_t work_f = T * flops, work_b = T * bytes;
    const uint64_t mapped = h2d + d2h, par = teams * threads;
    // 'teams distribute' covers loops [0, n_dist); combined with 'parallel for' when pf == 0
    const int n_dist = (pf == 0) ? pc : dc;
    uint64_t Dp = 1, Qp = 1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (i < n_dist) Dp *= t[i];
        if (i >= pf && i < pf + pc) Qp *= t[i];
    }
    const int32_t lT = log2_q16(T), lP = log2_q16(par);
    const int32_t lWF = log2_q16(work_f), lWB = log2_q16(work_b), lM = log2_q16(mapped);
    const int32_t lD = log2_q16(Dp), lQ = log2_q16(Qp);
    const int32_t lTeams = log2_q16(teams), lThreads = log2_q16(threads);

    int32_t base[32];
    base[0] = depth * ONE;
#pragma unroll
    for (int i = 0; i < 4; ++i) base[1 + i] = log2_q16(t[i]);
    base[5] = lT;
    base[6] = log2_q16(flops);
    base[7] = log2_q16(bytes);
    base[8] = lWF;
    base[9] = lWB;
    base[10] = log2_q16(h2d);
    base[11] = log2_q16(d2h);
    base[12] = lM;
    base[13] = lTeams;
    base[14] = lThreads;
    base[15] = lP;
    base[16] = lD;
    base[17] = lQ;
    base[18] = max(lT - lP, 0);
    base[19] = max(lD - lTeams, 0);
    base[20] = max(lQ - lThreads, 0);
    base[21] = lWF - lWB;
    base[22] = lWB - lM;
    base[23] = sched == 0 ? ONE : 0;
    base[24] = sched == 1 ? ONE : 0;
    base[25] = sched == 2 ? ONE : 0;
    base[26] = dmode * ONE;
    base[27] = pf * ONE;
    base[28] = dc * ONE;
    base[29] = pc * ONE;
    base[30] = pf == 0 ? ONE : 0;
    base[31] = log2_q16(T < par ? T : par);
#pragma unroll
    for (int j = 0; j < 32; ++j) f[j] = base[j];
    if constexpr (F >= 64) {
        // per loop level: log trip, distributed?, parallel-for?, in a collapse
        // group of >= 2 loops?, log prefix product, log suffix product,
        // log(trip*bytes/iter), log(trip*flops/iter); zero beyond the depth.
        uint64_t prefix = 1;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int o = 32 + 8 * i;
            if (i < depth) {
                prefix *= t[i];
                uint64_t suffix = 1;
                for (int j = i; j < depth; ++j) suffix *= t[j];
                const bool in_dist = i < n_dist;
                const bool in_pf = (i >= pf) && (i < pf + pc);
                const bool grouped = (in_dist && n_dist >= 2) || (in_pf && pc >= 2);
                f[o + 0] = log2_q16(t[i]);
                f[o + 1] = in_dist ? ONE : 0;
                f[o + 2] = in_pf ? ONE : 0;
                f[o + 3] = grouped ? ONE : 0;
                f[o + 4] = log2_q16(prefix);
                f[o + 5] = log2_q16(suffix);
                f[o + 6] = log2_q16(t[i] * bytes);
                f[o + 7] = log2_q16(t[i] * flops);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) f[o + j] = 0;
            }
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
