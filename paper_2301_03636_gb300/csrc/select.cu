// Per-kernel selection (a6) and the near-tie re-score bookkeeping (a7).
//
// Fig. 2 of arXiv 2301.03636: the predicted runtimes of the variants of a
// kernel are sorted and the best are kept; here the best one (argmin, lowest
// variant index on ties, never a row scored +inf or NaN).  One warp per
// kernel segment, lexicographic (score, row) reduction with warp shuffles.
//
// Near ties: rows within 2*eps of their kernel's minimum (eps bounds the
// scorer's error against FP64) are appended, in row order, to a candidate
// list that the FP32 scorer re-scores; rows within 2*eps32 of the FP32
// minimum go on to the FP64 scorer, whose values decide.  A kernel whose
// window holds a single row is decided at that tier.
#include "mlp.cuh"

namespace adv {

// Keep (v, r) if it beats (bv, br): smaller value, or equal value and smaller row.
__device__ __forceinline__ void lex_min(float& bv, int64_t& br, float v, int64_t r) {
    if (r >= 0 && (br < 0 || v < bv || (v == bv && r < br))) { bv = v; br = r; }
}
__device__ __forceinline__ void lex_min_d(double& bv, int64_t& br, double v, int64_t r) {
    if (r >= 0 && (br < 0 || v < bv || (v == bv && r < br))) { bv = v; br = r; }
}

__device__ __forceinline__ void warp_lex_min(float& bv, int64_t& br) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int64_t orr = __shfl_xor_sync(0xffffffffu, br, o);
        lex_min(bv, br, ov, orr);
    }
}
__device__ __forceinline__ void warp_lex_min_d(double& bv, int64_t& br) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int64_t orr = __shfl_xor_sync(0xffffffffu, br, o);
        lex_min_d(bv, br, ov, orr);
    }
}

__device__ __forceinline__ bool finite_score(float v) { return v < INFINITY; }   // false for +inf and NaN

// Append, in order, the rows r (given by lanes with `take`) to list[base + ...].
// Returns the number appended by this iteration; `done` is the running count.
__device__ __forceinline__ int append_ordered(bool take, int64_t r, int64_t* list, int base, int done) {
    const unsigned m = __ballot_sync(0xffffffffu, take);
    const int lane = threadIdx.x & 31;
    if (take) list[base + done + __popc(m & ((1u << lane) - 1u))] = r;
    return __popc(m);
}

// Tier 1 of kernel k (rows lo .. hi-1, already checked) by the whole warp.
__device__ __forceinline__ void tier1_segment_warp(const SelectArgs& a, int64_t k, int64_t lo, int64_t hi) {
    const int lane = threadIdx.x & 31;
    float bv = INFINITY;
    int64_t br = -1;
    for (int64_t r = lo + lane; r < hi; r += 32) {
        const float v = a.scores[r];
        if (finite_score(v)) lex_min(bv, br, v, r);
    }
    warp_lex_min(bv, br);
    int state = 0;
    if (br >= 0 && a.eps >= 0.f) {
        const double thr = (double)bv + 2.0 * (double)a.eps;
        int cnt = 0;
        for (int64_t r0 = lo; r0 < hi; r0 += 32) {
            const int64_t r = r0 + lane;
            const bool take = r < hi && finite_score(a.scores[r]) && (double)a.scores[r] <= thr;
            cnt += __popc(__ballot_sync(0xffffffffu, take));
        }
        if (cnt > 1) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&a.counters[0], cnt);
            base = __shfl_sync(0xffffffffu, base, 0);
            int done = 0;
            for (int64_t r0 = lo; r0 < hi; r0 += 32) {
                const int64_t r = r0 + lane;
                const bool take = r < hi && finite_score(a.scores[r]) && (double)a.scores[r] <= thr;
                done += append_ordered(take, r, a.cand_rows, base, done);
            }
            if (lane == 0) {
                a.seg_start[k] = base;
                a.seg_cnt[k] = cnt;
            }
            state = 1;
        }
    }
    if (lane == 0) {
        a.best[k] = br >= 0 ? (int32_t)(br - lo) : -1;
        a.best_score[k] = br >= 0 ? (double)bv : (double)INFINITY;
        if (a.seg_state) a.seg_state[k] = state;
    }
}

__device__ __forceinline__ bool bad_segment(const SelectArgs& a, int64_t lo, int64_t hi) {
    return lo < 0 || hi < lo || hi > a.n_rows;
}

__device__ __forceinline__ void mark_bad_segment(const SelectArgs& a, int64_t k) {
    atomicOr(a.status_word, ADV_DEV_BAD_SEGMENTS);
    a.best[k] = -1;
    a.best_score[k] = INFINITY;
    if (a.seg_state) a.seg_state[k] = 0;
}

// One warp per kernel: for few kernels, where every row should have a lane.
__global__ void __launch_bounds__(256) select_tier1_kernel(SelectArgs a) {
    griddep_wait();
    griddep_trigger();
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < a.n_kernels; k += nwarps) {
        const int64_t lo = a.off[k], hi = a.off[k + 1];
        if (bad_segment(a, lo, hi)) {
            if (lane == 0) mark_bad_segment(a, k);
            continue;
        }
        tier1_segment_warp(a, k, lo, hi);
    }
}

// One lane per kernel: for many short kernels, where a warp per kernel
// leaves the loads of each warp waiting one round trip after another.  A
// warp takes 32 consecutive kernels; each lane scans its kernel's rows in
// order (strict < keeps the lowest row on ties) and appends its candidates
// in row order; kernels longer than TIER1_LANE_MAX rows are done afterwards
// by the whole warp.
constexpr int64_t TIER1_LANE_MAX = 96;

__global__ void __launch_bounds__(256) select_tier1_lane_kernel(SelectArgs a) {
    griddep_wait();
    griddep_trigger();
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; k0 < a.n_kernels;
         k0 += nwarps * 32) {
        const int64_t k = k0 + lane;
        const bool have = k < a.n_kernels;
        int64_t lo = 0, hi = 0;
        if (have) {
            lo = a.off[k];
            hi = a.off[k + 1];
        }
        const bool bad = have && bad_segment(a, lo, hi);
        const bool longseg = have && !bad && hi - lo > TIER1_LANE_MAX;
        if (bad) mark_bad_segment(a, k);
        if (have && !bad && !longseg) {
            float bv = INFINITY;
            int64_t br = -1;
#pragma unroll 4
            for (int64_t r = lo; r < hi; ++r) {
                const float v = a.scores[r];
                if (finite_score(v) && (br < 0 || v < bv)) {
                    bv = v;
                    br = r;
                }
            }
            int state = 0;
            if (br >= 0 && a.eps >= 0.f) {
                const double thr = (double)bv + 2.0 * (double)a.eps;
                int cnt = 0;
                for (int64_t r = lo; r < hi; ++r) {
                    const float v = a.scores[r];
                    cnt += (finite_score(v) && (double)v <= thr) ? 1 : 0;
                }
                if (cnt > 1) {
                    const int base = atomicAdd(&a.counters[0], cnt);
                    int done = 0;
                    for (int64_t r = lo; r < hi; ++r) {
                        const float v = a.scores[r];
                        if (finite_score(v) && (double)v <= thr) a.cand_rows[base + done++] = r;
                    }
                    a.seg_start[k] = base;
                    a.seg_cnt[k] = cnt;
                    state = 1;
                }
            }
            a.best[k] = br >= 0 ? (int32_t)(br - lo) : -1;
            a.best_score[k] = br >= 0 ? (double)bv : (double)INFINITY;
            if (a.seg_state) a.seg_state[k] = state;
        }
        unsigned todo = __ballot_sync(0xffffffffu, longseg);
        while (todo) {
            const int j = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t kj = k0 + j;
            tier1_segment_warp(a, kj, __shfl_sync(0xffffffffu, lo, j), __shfl_sync(0xffffffffu, hi, j));
        }
    }
}

// FP32 value of the candidate at list position i
__device__ __forceinline__ float cand_y32(const SelectArgs& a, int64_t i) {
    return a.y32_rows ? a.y32_rows[a.cand_rows[i]] : a.y32[i];
}

__global__ void __launch_bounds__(256) select_tier2_kernel(SelectArgs a) {
    griddep_wait();
    griddep_trigger();
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < a.n_kernels; k += nwarps) {
        if (a.seg_state[k] != 1) continue;
        const int64_t lo = a.off[k];
        const int start = a.seg_start[k], cnt = a.seg_cnt[k];
        float bv = INFINITY;
        int64_t br = -1;
        for (int i = lane; i < cnt; i += 32) {
            const float v = cand_y32(a, start + i);
            if (finite_score(v)) lex_min(bv, br, v, a.cand_rows[start + i]);
        }
        warp_lex_min(bv, br);
        if (br < 0) {   // no finite FP32 value: keep the tier-1 decision
            if (lane == 0) a.seg_state[k] = 0;
            continue;
        }
        const double thr = (double)bv + 2.0 * (double)a.eps32;
        int cnt2 = 0;
        for (int i0 = 0; i0 < cnt; i0 += 32) {
            const int i = i0 + lane;
            const bool take = i < cnt && finite_score(cand_y32(a, start + i)) && (double)cand_y32(a, start + i) <= thr;
            cnt2 += __popc(__ballot_sync(0xffffffffu, take));
        }
        if (cnt2 > 1) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&a.counters[1], cnt2);
            base = __shfl_sync(0xffffffffu, base, 0);
            int done = 0;
            for (int i0 = 0; i0 < cnt; i0 += 32) {
                const int i = i0 + lane;
                const bool take = i < cnt && finite_score(cand_y32(a, start + i)) && (double)cand_y32(a, start + i) <= thr;
                const int64_t r = take ? a.cand_rows[start + i] : 0;
                done += append_ordered(take, r, a.cand2_rows, base, done);
            }
            if (lane == 0) {
                a.seg_start[k] = base;
                a.seg_cnt[k] = cnt2;
                a.seg_state[k] = 2;
                a.best[k] = (int32_t)(br - lo);
                a.best_score[k] = (double)bv;
            }
        } else if (lane == 0) {
            a.best[k] = (int32_t)(br - lo);
            a.best_score[k] = (double)bv;
            a.seg_state[k] = 0;
        }
    }
}

// FP16 middle tier (between tier 1 and the FP32 scorer): the tier-1
// candidates were re-scored on the tensor cores with FP16 operands (y16,
// |y16 - fp64| <= eps16).  The FP64 minimum row r* then has y16(r*) <=
// fp64(r*) + eps16 <= fp64(r16) + eps16 <= y16(r16) + 2 eps16, r16 the FP16
// minimum, so only candidates within 2*eps16 of that minimum go on to FP32.
// A candidate whose FP16 value is not finite (FP16 range exceeded) cannot be
// ruled out at this tier and always goes on.  Survivors are appended in
// candidate order to cand_mid_rows; a kernel with a single survivor is
// decided here.
__device__ __forceinline__ bool mid_keep(float v, double thr) { return !finite_score(v) || (double)v <= thr; }

__global__ void __launch_bounds__(256) select_mid_kernel(SelectArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < a.n_kernels; k += nwarps) {
        if (a.seg_state[k] != 1) continue;
        const int64_t lo = a.off[k];
        const int start = a.seg_start[k], cnt = a.seg_cnt[k];
        float bv = INFINITY;
        int64_t br = -1;
        for (int i = lane; i < cnt; i += 32) {
            const float v = a.y16[start + i];
            if (finite_score(v)) lex_min(bv, br, v, a.cand_rows[start + i]);
        }
        warp_lex_min(bv, br);
        const double thr = br >= 0 ? (double)bv + 2.0 * (double)a.eps16 : (double)INFINITY;
        int cnt2 = 0;
        for (int i0 = 0; i0 < cnt; i0 += 32) {
            const int i = i0 + lane;
            cnt2 += __popc(__ballot_sync(0xffffffffu, i < cnt && mid_keep(a.y16[start + i], thr)));
        }
        if (cnt2 > 1) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&a.counters[2], cnt2);
            base = __shfl_sync(0xffffffffu, base, 0);
            int done = 0;
            for (int i0 = 0; i0 < cnt; i0 += 32) {
                const int i = i0 + lane;
                const bool take = i < cnt && mid_keep(a.y16[start + i], thr);
                const int64_t r = take ? a.cand_rows[start + i] : 0;
                done += append_ordered(take, r, a.cand_mid_rows, base, done);
            }
            if (lane == 0) {
                a.seg_start[k] = base;
                a.seg_cnt[k] = cnt2;
            }
        } else if (lane == 0) {   // the FP16 minimum is the only survivor
            if (br >= 0) {
                a.best[k] = (int32_t)(br - lo);
                a.best_score[k] = (double)bv;
            }
            a.seg_state[k] = 0;
        }
    }
}

// ---- top N per kernel (Fig. 2: "sort codes based on cost and select top N") ----
//
// Exact against the FP64 ordering under the same error bounds as the argmin:
//   tier 1: t = the N-th smallest (score, row) of the kernel; every finite
//           row with score <= t + 2 eps is a candidate (no other row can be in
//           the FP64 top N); candidates are re-scored in FP32;
//   tier 2: t32 = the N-th smallest (FP32, row) among the candidates; those
//           with FP32 <= t32 + 2 eps32 that have another such candidate within
//           2 eps32 are re-scored in FP64 (only they can be ordered wrongly);
//   final:  the N smallest (key, row) among the candidates with FP32 <=
//           t32 + 2 eps32, key = the FP64 value where there is one, else the
//           FP32 value: two keys of different kinds belong to rows more than
//           2 eps32 apart in FP32, whose FP32 and FP64 orders agree.
// Without re-score (eps < 0) tier 1 writes the N smallest scores directly.

// The smallest finite (v, r) pair after (pv, pr) over rows lo + lane, +32, ...
__device__ __forceinline__ void next_after(const float* __restrict__ v, int64_t lo, int64_t hi, float pv, int64_t pr,
                                           float& bv, int64_t& br) {
    const int lane = threadIdx.x & 31;
    bv = INFINITY;
    br = -1;
    for (int64_t r = lo + lane; r < hi; r += 32) {
        const float x = v[r];
        if (finite_score(x) && (x > pv || (x == pv && r > pr))) lex_min(bv, br, x, r);
    }
    warp_lex_min(bv, br);
}

__global__ void __launch_bounds__(256) topn_tier1_kernel(SelectArgs a) {
    const int lane = threadIdx.x & 31;
    const int N = a.top_n;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < a.n_kernels; k += nwarps) {
        const int64_t lo = a.off[k], hi = a.off[k + 1];
        if (lo < 0 || hi < lo || hi > a.n_rows) {
            if (lane == 0) {
                atomicOr(a.status_word, ADV_DEV_BAD_SEGMENTS);
                for (int t = 0; t < N; ++t) {
                    a.best[k * N + t] = -1;
                    a.best_score[k * N + t] = INFINITY;
                }
                a.seg_state[k] = 0;
            }
            continue;
        }
        float pv = -INFINITY;
        int64_t pr = -1;
        int found = 0;
        for (int t = 0; t < N; ++t) {
            float bv;
            int64_t br;
            next_after(a.scores, lo, hi, pv, pr, bv, br);
            if (br < 0) break;
            if (lane == 0 && a.eps < 0.f) {
                a.best[k * N + t] = (int32_t)(br - lo);
                a.best_score[k * N + t] = (double)bv;
            }
            pv = bv;
            pr = br;
            ++found;
        }
        if (a.eps < 0.f || found == 0) {
            if (lane == 0) {
                for (int t = found; t < N; ++t) {
                    a.best[k * N + t] = -1;
                    a.best_score[k * N + t] = INFINITY;
                }
                a.seg_state[k] = 0;
            }
            continue;
        }
        const double thr = (double)pv + 2.0 * (double)a.eps;
        int cnt = 0;
        for (int64_t r0 = lo; r0 < hi; r0 += 32) {
            const int64_t r = r0 + lane;
            const bool take = r < hi && finite_score(a.scores[r]) && (double)a.scores[r] <= thr;
            cnt += __popc(__ballot_sync(0xffffffffu, take));
        }
        int base = 0;
        if (lane == 0) base = atomicAdd(&a.counters[0], cnt);
        base = __shfl_sync(0xffffffffu, base, 0);
        int done = 0;
        for (int64_t r0 = lo; r0 < hi; r0 += 32) {
            const int64_t r = r0 + lane;
            const bool take = r < hi && finite_score(a.scores[r]) && (double)a.scores[r] <= thr;
            done += append_ordered(take, r, a.cand_rows, base, done);
        }
        if (lane == 0) {
            a.seg_start[k] = base;
            a.seg_cnt[k] = cnt;
            a.seg_state[k] = 1;
        }
    }
}

__global__ void __launch_bounds__(256) topn_tier2_kernel(SelectArgs a) {
    const int lane = threadIdx.x & 31;
    const int N = a.top_n;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < a.n_kernels; k += nwarps) {
        if (a.seg_state[k] != 1) continue;
        const int start = a.seg_start[k], cnt = a.seg_cnt[k];
        const float* y = a.y32 + start;
        // the N-th smallest (FP32, position) among the candidates (positions follow row order)
        float pv = -INFINITY;
        int64_t pr = -1;
        for (int t = 0; t < N; ++t) {
            float bv;
            int64_t br;
            next_after(y, 0, cnt, pv, pr, bv, br);
            if (br < 0) break;
            pv = bv;
            pr = br;
        }
        const double thr = pr >= 0 ? (double)pv + 2.0 * (double)a.eps32 : -(double)INFINITY;
        const double win = 2.0 * (double)a.eps32;
        int cnt2 = 0;
        for (int i0 = 0; i0 < cnt; i0 += 32) {
            const int i = i0 + lane;
            bool take = false;
            if (i < cnt && finite_score(y[i]) && (double)y[i] <= thr) {
                for (int j = 0; j < cnt && !take; ++j)
                    take = j != i && finite_score(y[j]) && (double)y[j] <= thr &&
                           fabs((double)y[j] - (double)y[i]) <= win;
            }
            cnt2 += __popc(__ballot_sync(0xffffffffu, take));
        }
        int base = 0;
        if (lane == 0 && cnt2 > 0) base = atomicAdd(&a.counters[1], cnt2);
        base = __shfl_sync(0xffffffffu, base, 0);
        int done = 0;
        for (int i0 = 0; i0 < cnt; i0 += 32) {
            const int i = i0 + lane;
            bool take = false;
            if (i < cnt && finite_score(y[i]) && (double)y[i] <= thr) {
                for (int j = 0; j < cnt && !take; ++j)
                    take = j != i && finite_score(y[j]) && (double)y[j] <= thr &&
                           fabs((double)y[j] - (double)y[i]) <= win;
            }
            const unsigned m = __ballot_sync(0xffffffffu, take);
            if (i < cnt) a.pos64[start + i] = take ? base + done + __popc(m & ((1u << lane) - 1u)) : -1;
            if (take) a.cand2_rows[base + done + __popc(m & ((1u << lane) - 1u))] = a.cand_rows[start + i];
            done += __popc(m);
        }
        if (lane == 0) {
            a.seg_thr[k] = thr;
            a.seg_state[k] = 2;
        }
    }
}

__global__ void __launch_bounds__(256) topn_final_kernel(SelectArgs a) {
    const int lane = threadIdx.x & 31;
    const int N = a.top_n;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < a.n_kernels; k += nwarps) {
        if (a.seg_state[k] != 2) continue;
        const int64_t lo = a.off[k];
        const int start = a.seg_start[k], cnt = a.seg_cnt[k];
        const double thr = a.seg_thr[k];
        double pv = -(double)INFINITY;
        int64_t pr = -1;
        int t = 0;
        for (; t < N; ++t) {
            double bv = INFINITY;
            int64_t br = -1;
            for (int i = lane; i < cnt; i += 32) {
                const float y = a.y32[start + i];
                if (!finite_score(y) || (double)y > thr) continue;
                const int p = a.pos64[start + i];
                const double key = p >= 0 ? a.y64[p] : (double)y;
                const int64_t r = a.cand_rows[start + i];
                if (key < (double)INFINITY && (key > pv || (key == pv && r > pr))) lex_min_d(bv, br, key, r);
            }
            warp_lex_min_d(bv, br);
            if (br < 0) break;
            if (lane == 0) {
                a.best[k * N + t] = (int32_t)(br - lo);
                a.best_score[k * N + t] = bv;
            }
            pv = bv;
            pr = br;
        }
        if (lane == 0) {
            for (; t < N; ++t) {
                a.best[k * N + t] = -1;
                a.best_score[k * N + t] = INFINITY;
            }
            a.seg_state[k] = 0;
        }
    }
}

// FP16 middle tier of the top N: t16 = the N-th smallest finite (FP16, row)
// among a kernel's candidates (+inf if fewer than N are finite).  N
// candidates have FP64 <= t16 + eps16, so the N-th smallest FP64 value is at
// most that, and every FP64 top-N row has FP16 <= t16 + 2 eps16; the others
// are dropped.  Non-finite FP16 values always go on.
__global__ void __launch_bounds__(256) topn_mid_kernel(SelectArgs a) {
    const int lane = threadIdx.x & 31;
    const int N = a.top_n;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < a.n_kernels; k += nwarps) {
        if (a.seg_state[k] != 1) continue;
        const int start = a.seg_start[k], cnt = a.seg_cnt[k];
        const float* y = a.y16 + start;
        float pv = -INFINITY;
        int64_t pr = -1;
        int t = 0;
        for (; t < N; ++t) {
            float bv;
            int64_t br;
            next_after(y, 0, cnt, pv, pr, bv, br);
            if (br < 0) break;
            pv = bv;
            pr = br;
        }
        const double thr = t == N ? (double)pv + 2.0 * (double)a.eps16 : (double)INFINITY;
        int cnt2 = 0;
        for (int i0 = 0; i0 < cnt; i0 += 32) {
            const int i = i0 + lane;
            cnt2 += __popc(__ballot_sync(0xffffffffu, i < cnt && mid_keep(y[i], thr)));
        }
        int base = 0;
        if (lane == 0) base = atomicAdd(&a.counters[2], cnt2);
        base = __shfl_sync(0xffffffffu, base, 0);
        int done = 0;
        for (int i0 = 0; i0 < cnt; i0 += 32) {
            const int i = i0 + lane;
            const bool take = i < cnt && mid_keep(y[i], thr);
            const int64_t r = take ? a.cand_rows[start + i] : 0;
            done += append_ordered(take, r, a.cand_mid_rows, base, done);
        }
        if (lane == 0) {
            a.seg_start[k] = base;
            a.seg_cnt[k] = cnt2;
        }
    }
}

// One warp per segment; the kernels stride over segments, so any grid and
// any whole number of warps per block covers them.
static int select_grid(int64_t n_kernels, int block) {
    const int wpb = block / 32;
    const int64_t blocks = (n_kernels + wpb - 1) / wpb;
    return (int)(blocks < 1 ? 1 : (blocks > 65535 ? 65535 : blocks));
}

static bool select_block_ok(int block) { return block == 128 || block == 256; }

static cudaError_t counted(cudaError_t e) {
    if (e == cudaSuccess) adv_count_launch(1);
    return e;
}

// Kernels per launch from which tier 1 gives each kernel a lane instead of a warp.
constexpr int64_t TIER1_LANE_FROM = 32768;

cudaError_t launch_select_tier1(const SelectArgs& a, cudaStream_t s, int block) {
    if (!select_block_ok(block)) return cudaErrorInvalidValue;
    if (a.n_kernels >= TIER1_LANE_FROM)
        return counted(launch_pdl(select_tier1_lane_kernel, dim3(select_grid((a.n_kernels + 31) / 32, block)),
                                  dim3(block), 0, s, a));
    return counted(launch_pdl(select_tier1_kernel, dim3(select_grid(a.n_kernels, block)), dim3(block), 0, s, a));
}
cudaError_t launch_select_tier2(const SelectArgs& a, cudaStream_t s, int block) {
    if (!select_block_ok(block)) return cudaErrorInvalidValue;
    return counted(launch_pdl(select_tier2_kernel, dim3(select_grid(a.n_kernels, block)), dim3(block), 0, s, a));
}

cudaError_t launch_select_mid(const SelectArgs& a, cudaStream_t s, int block) {
    if (!select_block_ok(block) || !a.y16 || !a.cand_mid_rows) return cudaErrorInvalidValue;
    select_mid_kernel<<<select_grid(a.n_kernels, block), block, 0, s>>>(a);
    adv_count_launch(1);
    return cudaGetLastError();
}
cudaError_t launch_topn_mid(const SelectArgs& a, cudaStream_t s, int block) {
    if (!select_block_ok(block) || !a.y16 || !a.cand_mid_rows) return cudaErrorInvalidValue;
    topn_mid_kernel<<<select_grid(a.n_kernels, block), block, 0, s>>>(a);
    adv_count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_topn_tier1(const SelectArgs& a, cudaStream_t s, int block) {
    if (!select_block_ok(block)) return cudaErrorInvalidValue;
    topn_tier1_kernel<<<select_grid(a.n_kernels, block), block, 0, s>>>(a);
    adv_count_launch(1);
    return cudaGetLastError();
}
cudaError_t launch_topn_tier2(const SelectArgs& a, cudaStream_t s, int block) {
    if (!select_block_ok(block)) return cudaErrorInvalidValue;
    topn_tier2_kernel<<<select_grid(a.n_kernels, block), block, 0, s>>>(a);
    adv_count_launch(1);
    return cudaGetLastError();
}
cudaError_t launch_topn_final(const SelectArgs& a, cudaStream_t s, int block) {
    if (!select_block_ok(block)) return cudaErrorInvalidValue;
    topn_final_kernel<<<select_grid(a.n_kernels, block), block, 0, s>>>(a);
    adv_count_launch(1);
    return cudaGetLastError();
}

bool launch_config_valid(const LaunchConfig& c) {
    return (c.extract_block == 64 || c.extract_block == 128 || c.extract_block == 256) && c.tc_ctas >= 0 &&
           (c.list_blocks_per_sm == 1 || c.list_blocks_per_sm == 2) &&
           (c.list_chunk_kb == 16 || c.list_chunk_kb == 32) && select_block_ok(c.select_block) &&
           (c.layer_path == 0 || c.layer_path == 1);
}

}  // namespace adv
