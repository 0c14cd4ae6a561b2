/*
 * Plain FP64 CPU oracle of the OpenMP Advisor cost-model path:
 * descriptor validation -> integer features -> z-score standardisation ->
 * MLP regression -> per-kernel argmin, plus the FP64 gradient and an Adam step
 * for the training configuration.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it to check and to time the CUDA path.  It shares no code,
 * header, table or constant generator with the CUDA sources.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared [-fopenmp]
 * (-ffp-contract=off: every product and every sum is rounded separately, in
 * the order written below; the OpenMP pragma only splits independent rows.)
 *
 * Paper references are to arXiv 2301.03636 ("OpenMP Advisor"):
 *   Sec. 4.1.1-4.1.2  the per-kernel loop-nest and data-mapping information,
 *   Sec. 4.1.3        the five variant parameters and their valid ranges,
 *   Sec. 4.2 / Fig. 2 feature extraction -> trained model -> predicted runtime
 *                     per variant -> sort and select,
 *   Sec. 5 Exp. 3     MLP with ReLU hidden layers, z-score standardisation,
 *                     RMSE (Eq. rmse) / NRMSE (Eq. nrmse).
 * The paper lists neither its features nor its dimension reduction; the
 * feature table below is this project's reading and is written out in full.
 *
 * Parity pins: every function here is checked in tests/test_oracle_*.py
 * against hand-worked descriptors, closed forms, invariants, brute force or
 * finite differences (see the test files), and tests/test_oracle_mutants.py
 * checks that mistakes planted in copies of this file fail those pins.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>

/* ------------------------------------------------------------------------ */
/* Binary logarithm, Q16.16.                                                 */
/* Digit-by-digit base-2 logarithm by repeated squaring of the normalised    */
/* mantissa (the classical method; e.g. Majithia & Levan, "A note on base-2  */
/* logarithm computations", Proc. IEEE 1973).  For x >= 1:                    */
/*   k = floor(log2 x); m = x scaled to [1,2) as a Q1.31 fixed-point number;  */
/*   16 times: m = m*m (truncated to Q1.31); if m >= 2 emit bit 1 and halve,  */
/*   else emit bit 0.  Result = k*65536 + the 16 emitted bits.                */
/* L(0) = 0 (an absent quantity).                                             */
/* ------------------------------------------------------------------------ */
int32_t orc_log2_q16(uint64_t x)
{
    if (x == 0) return 0;
    int k = 63;
    while (((x >> k) & 1u) == 0) k--;                 /* index of the top set bit */
    uint64_t m;                                        /* value m / 2^31 in [1, 2) */
    if (k >= 31) m = x >> (k - 31);
    else         m = x << (31 - k);
    int32_t bits = 0;
    for (int i = 0; i < 16; i++) {
        m = (m * m) >> 31;                             /* m^2, still scaled by 2^31 */
        bits = bits * 2;
        if (m >= ((uint64_t)1 << 32)) {                /* m^2 >= 2 */
            bits = bits + 1;
            m = m >> 1;
        }
    }
    return (int32_t)k * 65536 + bits;
}

void orc_log2_q16_batch(const uint64_t* x, int64_t n, int32_t* out)
{
    for (int64_t i = 0; i < n; i++) out[i] = orc_log2_q16(x[i]);
}

/* ------------------------------------------------------------------------ */
/* Descriptor validation (ranges from Sec. 4.1.3; bounds chosen so that all  */
/* derived products are exact in 64-bit integers).                          */
/* ------------------------------------------------------------------------ */
enum {
    ORC_BAD_DEPTH = 1, ORC_BAD_TRIP = 2, ORC_BAD_WORK = 4, ORC_BAD_MAPPED = 8,
    ORC_BAD_PARALLELISM = 16, ORC_BAD_VARIANT = 32, ORC_BAD_RANGE = 64
};

#define P2(e) ((int64_t)1 << (e))

/* a*b if it is <= limit, else -1 (a, b >= 0). */
static int64_t mul_le(int64_t a, int64_t b, int64_t limit)
{
    unsigned __int128 p = (unsigned __int128)(uint64_t)a * (uint64_t)b;
    if (p > (unsigned __int128)(uint64_t)limit) return -1;
    return (int64_t)p;
}

uint8_t orc_validate(const int64_t* d)
{
    const int64_t depth = d[0];
    if (depth < 1 || depth > 4) return ORC_BAD_DEPTH;
    uint8_t st = 0;
    for (int i = 0; i < 4; i++) {
        int64_t t = d[1 + i];
        if (i < depth) { if (t < 1 || t > P2(24)) st |= ORC_BAD_TRIP; }
        else           { if (t != 1) st |= ORC_BAD_TRIP; }
    }
    if (d[5] < 1 || d[5] > P2(32) || d[6] < 1 || d[6] > P2(32)) st |= ORC_BAD_WORK;
    if (d[7] < 0 || d[7] > P2(48) || d[8] < 0 || d[8] > P2(48)) st |= ORC_BAD_MAPPED;
    if (d[9] < 1 || d[9] > P2(24) || d[10] < 1 || d[10] > P2(24)) st |= ORC_BAD_PARALLELISM;
    const int64_t pf_pos = d[11], dc = d[12], pc = d[13], sched = d[14], dm = d[15];
    int vok = 1;
    if (pf_pos < 0 || pf_pos > depth - 1) vok = 0;
    else {
        if (pf_pos == 0) { if (dc != 0) vok = 0; }
        else             { if (dc < 1 || dc > pf_pos) vok = 0; }
        if (pc < 1 || pc > depth - pf_pos) vok = 0;
    }
    if (sched < 0 || sched > 2) vok = 0;
    if (dm < 0 || dm > 1) vok = 0;
    if (!vok) st |= ORC_BAD_VARIANT;
    if ((st & (ORC_BAD_TRIP | ORC_BAD_WORK)) == 0) {
        int64_t T = 1;
        for (int i = 0; i < depth && T >= 0; i++) T = mul_le(T, d[1 + i], P2(48));
        if (T < 0 || mul_le(T, d[5], P2(62)) < 0 || mul_le(T, d[6], P2(62)) < 0)
            st |= ORC_BAD_RANGE;
    }
    return st;
}

/* ------------------------------------------------------------------------ */
/* Feature extraction (Fig. 2 "Feature Extraction"; our feature table).      */
/* ------------------------------------------------------------------------ */
#define Q1 65536

static int32_t imax0(int32_t a) { return a > 0 ? a : 0; }

/* Features of one valid descriptor.  F is 32, 33, 64 or 128. */
static void features_one(const int64_t* d, int F, int32_t* f)
{
    const int64_t depth = d[0];
    int64_t t[4];
    for (int i = 0; i < 4; i++) t[i] = d[1 + i];
    const int64_t flops = d[5], bytes = d[6], h2d = d[7], d2h = d[8];
    const int64_t teams = d[9], threads = d[10];
    const int64_t pf_pos = d[11], dc = d[12], pc = d[13], sched = d[14], dm = d[15];

    /* derived integers */
    int64_t T = t[0] * t[1] * t[2] * t[3];
    int64_t FL = T * flops, BY = T * bytes, MB = h2d + d2h, P = teams * threads;
    /* loop levels covered by each directive */
    int is_dist[4], is_pf[4];
    int64_t dist_n = (pf_pos == 0) ? pc : dc;          /* combined directive when pf_pos == 0 */
    for (int i = 0; i < 4; i++) {
        is_dist[i] = (i < dist_n);
        is_pf[i] = (i >= pf_pos && i < pf_pos + pc);
    }
    int64_t D = 1, Q = 1;
    for (int i = 0; i < 4; i++) {
        if (is_dist[i]) D = D * t[i];
        if (is_pf[i]) Q = Q * t[i];
    }
    int32_t LT = orc_log2_q16((uint64_t)T), LP = orc_log2_q16((uint64_t)P);
    int32_t LFL = orc_log2_q16((uint64_t)FL), LBY = orc_log2_q16((uint64_t)BY);
    int32_t LMB = orc_log2_q16((uint64_t)MB);
    int32_t LD = orc_log2_q16((uint64_t)D), LQ = orc_log2_q16((uint64_t)Q);
    int32_t Lteams = orc_log2_q16((uint64_t)teams), Lthreads = orc_log2_q16((uint64_t)threads);

    int32_t b[32];
    b[0] = (int32_t)depth * Q1;
    for (int i = 0; i < 4; i++) b[1 + i] = orc_log2_q16((uint64_t)t[i]);
    b[5] = LT;
    b[6] = orc_log2_q16((uint64_t)flops);
    b[7] = orc_log2_q16((uint64_t)bytes);
    b[8] = LFL;
    b[9] = LBY;
    b[10] = orc_log2_q16((uint64_t)h2d);
    b[11] = orc_log2_q16((uint64_t)d2h);
    b[12] = LMB;
    b[13] = Lteams;
    b[14] = Lthreads;
    b[15] = LP;
    b[16] = LD;
    b[17] = LQ;
    b[18] = imax0(LT - LP);
    b[19] = imax0(LD - Lteams);
    b[20] = imax0(LQ - Lthreads);
    b[21] = LFL - LBY;
    b[22] = LBY - LMB;
    b[23] = (sched == 0) ? Q1 : 0;
    b[24] = (sched == 1) ? Q1 : 0;
    b[25] = (sched == 2) ? Q1 : 0;
    b[26] = (int32_t)dm * Q1;
    b[27] = (int32_t)pf_pos * Q1;
    b[28] = (int32_t)dc * Q1;
    b[29] = (int32_t)pc * Q1;
    b[30] = (pf_pos == 0) ? Q1 : 0;
    b[31] = orc_log2_q16((uint64_t)(T < P ? T : P));
    for (int j = 0; j < 32 && j < F; j++) f[j] = b[j];
    if (F <= 32) return;
    if (F == 33) {   /* the paper-shaped input: the base features and the number of collapsed loops */
        f[32] = (int32_t)(dc + pc) * Q1;
        return;
    }

    /* 8 features per loop level; all zero for levels >= depth */
    for (int i = 0; i < 4; i++) {
        int32_t* g = f + 32 + 8 * i;
        if (i >= depth) { for (int j = 0; j < 8; j++) g[j] = 0; continue; }
        int64_t prefix = 1, suffix = 1;
        for (int j = 0; j <= i; j++) prefix = prefix * t[j];
        for (int j = i; j < depth; j++) suffix = suffix * t[j];
        int collapsed = (is_dist[i] && dist_n >= 2) || (is_pf[i] && pc >= 2);
        g[0] = orc_log2_q16((uint64_t)t[i]);
        g[1] = is_dist[i] ? Q1 : 0;
        g[2] = is_pf[i] ? Q1 : 0;
        g[3] = collapsed ? Q1 : 0;
        g[4] = orc_log2_q16((uint64_t)prefix);
        g[5] = orc_log2_q16((uint64_t)suffix);
        g[6] = orc_log2_q16((uint64_t)(t[i] * bytes));
        g[7] = orc_log2_q16((uint64_t)(t[i] * flops));
    }
    if (F <= 64) return;

    /* 64 signed differences of base features: pair u = 0..63 takes
       a = 1 + (u mod 21), step s = 1 + floor(u / 21), b = 1 + ((a - 1 + s) mod 22) */
    for (int u = 0; u < 64; u++) {
        int a = 1 + (u % 21);
        int s = 1 + u / 21;
        int bb = 1 + ((a - 1 + s) % 22);
        f[64 + u] = b[a] - b[bb];
    }
}

/* feat[n][F] (row-major) and status[n]; invalid rows get all-zero features.
   Returns the number of invalid rows. */
int64_t orc_extract_features(const int64_t* desc, int64_t n, int F, int32_t* feat, uint8_t* status)
{
    int64_t bad = 0;
#pragma omp parallel for schedule(static) reduction(+:bad)
    for (int64_t r = 0; r < n; r++) {
        const int64_t* d = desc + 16 * r;
        uint8_t st = orc_validate(d);
        status[r] = st;
        if (st) { memset(feat + F * r, 0, sizeof(int32_t) * (size_t)F); bad++; }
        else features_one(d, F, feat + F * r);
    }
    return bad;
}

/* ------------------------------------------------------------------------ */
/* Z-score standardisation (Sec. 5, Exp. 3): x = feature / 65536,            */
/* mu = mean, sigma = population standard deviation over the valid rows,   */
/* sigma = 1 where it is 0.                                                  */
/* ------------------------------------------------------------------------ */
void orc_fit_standardizer(const int32_t* feat, const uint8_t* status, int64_t n, int F,
                          double* mu, double* sigma)
{
    for (int j = 0; j < F; j++) {
        double s = 0.0;
        int64_t cnt = 0;
        for (int64_t r = 0; r < n; r++)
            if (!status || status[r] == 0) { s = s + (double)feat[F * r + j] / 65536.0; cnt++; }
        double m = cnt ? s / (double)cnt : 0.0;
        double v = 0.0;
        for (int64_t r = 0; r < n; r++)
            if (!status || status[r] == 0) {
                double e = (double)feat[F * r + j] / 65536.0 - m;
                v = v + e * e;
            }
        double sd = cnt ? sqrt(v / (double)cnt) : 0.0;
        mu[j] = m;
        sigma[j] = (sd > 0.0) ? sd : 1.0;
    }
}

/* ------------------------------------------------------------------------ */
/* MLP regression in FP64 (Sec. 4.2, Sec. 5 Exp. 3).                         */
/* params: FP32 master parameters, per layer W[out][in] row-major then       */
/* b[out].  Hidden layers: h' = ReLU(W h + b); the last layer is linear and  */
/* has one output (the predicted ln runtime).  Each dot product is summed    */
/* sequentially over the input index starting from 0.0, then the bias is    */
/* added.  Invalid rows score +inf.                                          */
/* ------------------------------------------------------------------------ */
static int max_width(const int32_t* widths, int nw)
{
    int w = 0;
    for (int i = 0; i < nw; i++) if (widths[i] > w) w = widths[i];
    return w;
}

static double forward_one(const int32_t* f, const int32_t* widths, int nw, const float* params,
                          const double* mu, const double* sigma, double* ha, double* hb,
                          double* pre /* nullable: all layers' pre-activations */)
{
    const int F = widths[0];
    for (int k = 0; k < F; k++) ha[k] = ((double)f[k] / 65536.0 - mu[k]) / sigma[k];
    const float* p = params;
    double* in = ha;
    double* out = hb;
    int pre_off = 0;
    for (int l = 0; l + 1 < nw; l++) {
        const int fi = widths[l], fo = widths[l + 1];
        const float* W = p;
        const float* b = p + (size_t)fo * fi;
        for (int j = 0; j < fo; j++) {
            double s = 0.0;
            for (int k = 0; k < fi; k++) s = s + (double)W[(size_t)j * fi + k] * in[k];
            s = s + (double)b[j];
            if (pre) pre[pre_off + j] = s;
            out[j] = (l + 2 < nw) ? (s > 0.0 ? s : 0.0) : s;
        }
        pre_off += fo;
        p += (size_t)fo * fi + fo;
        double* tmp = in; in = out; out = tmp;
    }
    return in[0];
}

void orc_mlp_forward(const int32_t* feat, const uint8_t* status, int64_t n, const int32_t* widths,
                     int nw, const float* params, const double* mu, const double* sigma, double* y)
{
    const int F = widths[0];
    const int W = max_width(widths, nw);
#pragma omp parallel
    {
        double* ha = (double*)malloc(sizeof(double) * (size_t)W);
        double* hb = (double*)malloc(sizeof(double) * (size_t)W);
#pragma omp for schedule(static)
        for (int64_t r = 0; r < n; r++) {
            if (status && status[r]) { y[r] = INFINITY; continue; }
            y[r] = forward_one(feat + (size_t)F * r, widths, nw, params, mu, sigma, ha, hb, NULL);
        }
        free(ha);
        free(hb);
    }
}

/* ------------------------------------------------------------------------ */
/* Per-kernel selection (Fig. 2 "sort codes based on cost and select"):      */
/* kernel k owns rows off[k] .. off[k+1]-1; best[k] is the local index of the */
/* smallest score, the lowest index on ties; -0.0 == +0.0; +inf and NaN rows  */
/* are never selected; an empty segment or one without a finite score gets   */
/* best = -1 and best_score = +inf.                                          */
/* ------------------------------------------------------------------------ */
void orc_select_best(const double* y, const int64_t* off, int64_t n_kernels,
                     int32_t* best, double* best_score)
{
    for (int64_t k = 0; k < n_kernels; k++) {
        int32_t bi = -1;
        double bs = INFINITY;
        for (int64_t r = off[k]; r < off[k + 1]; r++) {
            double v = y[r];
            if (!(v < INFINITY)) continue;              /* skips +inf and NaN */
            if (bi < 0 || v < bs) { bi = (int32_t)(r - off[k]); bs = v; }
        }
        best[k] = bi;
        best_score[k] = bs;
    }
}

/* ------------------------------------------------------------------------ */
/* Top N per kernel (Fig. 2: "sort codes based on cost and select top N").    */
/* best[k*N + t] = local index of the t-th smallest finite score of kernel k */
/* (ties to the lower local index), score[k*N + t] its value; -1 / +inf     */
/* where the kernel has fewer than t+1 finite scores.  Written as N passes   */
/* of "smallest (score, index) pair after the previous one".                 */
/* ------------------------------------------------------------------------ */
void orc_select_topn(const double* y, const int64_t* off, int64_t n_kernels, int N,
                     int32_t* best, double* score)
{
    for (int64_t k = 0; k < n_kernels; k++) {
        double pv = -INFINITY;
        int64_t pi = -1;
        for (int t = 0; t < N; t++) {
            int64_t bi = -1;
            double bv = INFINITY;
            for (int64_t r = off[k]; r < off[k + 1]; r++) {
                const double v = y[r];
                const int64_t i = r - off[k];
                if (!(v < INFINITY)) continue;                    /* skips +inf and NaN */
                if (!(v > pv || (v == pv && i > pi))) continue;   /* not after the previous pick */
                if (bi < 0 || v < bv) { bi = i; bv = v; }
            }
            best[k * N + t] = (int32_t)bi;
            score[k * N + t] = bi < 0 ? INFINITY : bv;
            if (bi >= 0) { pv = bv; pi = bi; }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Variant generation (Sec. 4.1.3, Table 1).  A kernel whose loop nest has   */
/* NUM = depth collapsible for loops (1..4) gets one variant for every       */
/* combination of                                                            */
/*   x    the loop of the 'parallel for' directive, 0 <= x < NUM;           */
/*   dc   the collapse of 'teams distribute': none (0) when x = 0, where the */
/*        two directives are combined, else 1..x;                            */
/*   pc   the collapse of 'parallel for', 1..NUM-x;                          */
/*   the schedule (static, dynamic, guided = 0, 1, 2) and the data transfer */
/*   mode (0, 1);                                                            */
/* emitted with x outermost and the data mode innermost (the library's      */
/* canonical order).  A variant copies the kernel's loop nest and work       */
/* fields (descriptor fields 0..10) and sets fields 11..15 = x, dc, pc,      */
/* schedule, data mode.                                                      */
/* ------------------------------------------------------------------------ */
int64_t orc_variant_count(int64_t depth)
{
    if (depth < 1 || depth > 4) return 0;
    int64_t combos = 0;
    for (int64_t x = 0; x < depth; x++) combos += (x == 0 ? 1 : x) * (depth - x);
    return combos * 3 * 2;
}

/* kernels[K][16] -> variants[n][16] (n = sum of the counts), seg_off[K+1]. */
int64_t orc_enumerate_variants(const int64_t* kernels, int64_t n_kernels, int64_t* out, int64_t* seg_off)
{
    int64_t n = 0;
    seg_off[0] = 0;
    for (int64_t k = 0; k < n_kernels; k++) {
        const int64_t* kd = kernels + 16 * k;
        const int64_t depth = kd[0];
        if (depth >= 1 && depth <= 4) {
            for (int64_t x = 0; x < depth; x++) {
                const int64_t dc_lo = x == 0 ? 0 : 1, dc_hi = x;
                for (int64_t dc = dc_lo; dc <= dc_hi; dc++)
                    for (int64_t pc = 1; pc <= depth - x; pc++)
                        for (int64_t sched = 0; sched < 3; sched++)
                            for (int64_t dm = 0; dm < 2; dm++) {
                                int64_t* v = out + 16 * n;
                                memcpy(v, kd, 11 * sizeof(int64_t));
                                v[11] = x;
                                v[12] = dc;
                                v[13] = pc;
                                v[14] = sched;
                                v[15] = dm;
                                n++;
                            }
            }
        }
        seg_off[k + 1] = n;
    }
    return n;
}

/* ------------------------------------------------------------------------ */
/* Training: loss = 0.5 * mean_r (y_r - t_r)^2 over the n rows (MSE on ln    */
/* runtime), its FP64 gradient with respect to every parameter (same layout  */
/* as params), and one Adam step (Kingma & Ba 2015) with decoupled weight     */
/* decay 0.  The paper trains with RMSE / RMSprop; this loss and optimizer   */
/* follow the training benchmark instead.                                    */
/* ------------------------------------------------------------------------ */
double orc_mlp_loss_grad(const int32_t* feat, const float* labels, int64_t n, const int32_t* widths,
                         int nw, const float* params, const double* mu, const double* sigma,
                         double* grad /* [param_count], overwritten */)
{
    const int F = widths[0];
    const int W = max_width(widths, nw);
    int64_t np_ = 0, nact = 0;
    for (int l = 0; l + 1 < nw; l++) { np_ += (int64_t)widths[l + 1] * widths[l] + widths[l + 1]; nact += widths[l + 1]; }
    for (int64_t i = 0; i < np_; i++) grad[i] = 0.0;
    double* pre = (double*)malloc(sizeof(double) * (size_t)nact);
    double* z0 = (double*)malloc(sizeof(double) * (size_t)F);
    double* ha = (double*)malloc(sizeof(double) * (size_t)W);
    double* hb = (double*)malloc(sizeof(double) * (size_t)W);
    double* dcur = (double*)malloc(sizeof(double) * (size_t)W);
    double* dprev = (double*)malloc(sizeof(double) * (size_t)W);
    int64_t* poff = (int64_t*)malloc(sizeof(int64_t) * (size_t)nw);
    int* aoff = (int*)malloc(sizeof(int) * (size_t)nw);
    {
        int64_t po = 0; int ao = 0;
        for (int l = 0; l + 1 < nw; l++) {
            poff[l] = po; aoff[l] = ao;
            po += (int64_t)widths[l + 1] * widths[l] + widths[l + 1];
            ao += widths[l + 1];
        }
    }
    double loss = 0.0;
    for (int64_t r = 0; r < n; r++) {
        const int32_t* f = feat + (size_t)F * r;
        double y = forward_one(f, widths, nw, params, mu, sigma, ha, hb, pre);
        for (int k = 0; k < F; k++) z0[k] = ((double)f[k] / 65536.0 - mu[k]) / sigma[k];
        double e = y - (double)labels[r];
        loss = loss + 0.5 * e * e;
        dcur[0] = e / (double)n;                         /* d loss / d y */
        for (int l = nw - 2; l >= 0; l--) {
            const int fi = widths[l], fo = widths[l + 1];
            const float* Wl = params + poff[l];
            double* gW = grad + poff[l];
            double* gb = grad + poff[l] + (int64_t)fo * fi;
            /* input activations of layer l */
            for (int j = 0; j < fo; j++) {
                double dz = dcur[j];
                gb[j] = gb[j] + dz;
                for (int k = 0; k < fi; k++) {
                    double hk = (l == 0) ? z0[k] : (pre[aoff[l - 1] + k] > 0.0 ? pre[aoff[l - 1] + k] : 0.0);
                    gW[(size_t)j * fi + k] = gW[(size_t)j * fi + k] + dz * hk;
                }
            }
            if (l == 0) break;
            for (int k = 0; k < fi; k++) {
                double s = 0.0;
                for (int j = 0; j < fo; j++) s = s + dcur[j] * (double)Wl[(size_t)j * fi + k];
                dprev[k] = (pre[aoff[l - 1] + k] > 0.0) ? s : 0.0;   /* ReLU derivative */
            }
            double* tmp = dcur; dcur = dprev; dprev = tmp;
        }
    }
    free(pre); free(z0); free(ha); free(hb); free(dcur); free(dprev); free(poff); free(aoff);
    return loss / (double)n;
}

/* One Adam step on FP64 state: m, v updated in place, returns new params in
   out_params.  step counts from 1.  Bias-corrected as in Algorithm 1 of Kingma & Ba. */
void orc_adam_step(const double* params, const double* grad, double* m, double* v, int64_t np_,
                   double lr, double beta1, double beta2, double eps, int64_t step, double* out_params)
{
    const double c1 = 1.0 - pow(beta1, (double)step);
    const double c2 = 1.0 - pow(beta2, (double)step);
    for (int64_t i = 0; i < np_; i++) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        out_params[i] = params[i] - lr * mh / (sqrt(vh) + eps);
    }
}

/* RMSprop (Tieleman & Hinton 2012, the optimizer of Sec. 5 Exp. 3) with the */
/* weight decay added to the gradient:                                        */
/*   g' = g + wd * w;  v = alpha v + (1 - alpha) g'^2;  w -= lr g' / (sqrt(v) + eps). */
void orc_rmsprop_step(const double* params, const double* grad, double* v, int64_t np_, double lr,
                      double alpha, double eps, double wd, double* out_params)
{
    for (int64_t i = 0; i < np_; i++) {
        const double g = grad[i] + wd * params[i];
        v[i] = alpha * v[i] + (1.0 - alpha) * g * g;
        out_params[i] = params[i] - lr * g / (sqrt(v[i]) + eps);
    }
}

/* The RMSE loss of Sec. 5 Exp. 3, RMSE = sqrt(mean_r (y_r - t_r)^2), and its */
/* gradient: with m = mean (y - t)^2 = 2 * (the MSE loss above),              */
/* dRMSE = dm / (2 sqrt(m)) = (gradient of the MSE loss) / RMSE (0 if RMSE = 0). */
double orc_mlp_rmse_grad(const int32_t* feat, const float* labels, int64_t n, const int32_t* widths,
                         int nw, const float* params, const double* mu, const double* sigma, double* grad)
{
    const double half_ms = orc_mlp_loss_grad(feat, labels, n, widths, nw, params, mu, sigma, grad);
    const double rmse = sqrt(2.0 * half_ms);
    int64_t np_ = 0;
    for (int l = 0; l + 1 < nw; l++) np_ += (int64_t)widths[l + 1] * widths[l] + widths[l + 1];
    for (int64_t i = 0; i < np_; i++) grad[i] = rmse > 0.0 ? grad[i] / rmse : 0.0;
    return rmse;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the parallel loops from now on (n >= 1); timing only. */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
