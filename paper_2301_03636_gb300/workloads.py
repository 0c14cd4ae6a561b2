"""Seeded synthetic inputs for the cost-model hot path.

This module only draws random inputs: loop-nest / data-mapping descriptors,
per-kernel variant counts (segment offsets), MLP weights and training labels.
It holds none of the method's arithmetic (no feature extraction, no MLP, no
selection), so that both the CUDA path and the plain CPU oracle can take their
inputs from it without sharing any computation.

Descriptor layout (one row = 16 int64 = 128 bytes), the variant parameters of
Sec. 4.1.3 plus the loop-nest and data-analysis numbers of Sec. 4.1.1-4.1.2:

    0 depth            number of nested for loops NUM (1..4)
    1..4 trip[0..3]    trip count per loop level, 1 for levels >= depth
    5 flops_per_iter   arithmetic operations in the innermost body
    6 bytes_per_iter   bytes touched by the innermost body
    7 h2d_bytes        bytes mapped host->device (alloc/to/tofrom classes)
    8 d2h_bytes        bytes mapped device->host (from/tofrom classes)
    9 teams, 10 threads
    11 pf_pos          loop x that carries 'parallel for' (0 = combined with distribute)
    12 dist_collapse   collapse of 'teams distribute' (0 iff pf_pos == 0, else 1..pf_pos)
    13 pf_collapse     collapse of 'parallel for' (1..depth-pf_pos)
    14 schedule        0 static, 1 dynamic, 2 guided
    15 data_mode       the two-valued data-transfer parameter of Sec. 4.1.3

Distributions (our reading of the workload descriptions): depth uniform 1..3,
trip counts floor(2^U(4,12)) per level, flops/iter uniform 1..32, bytes/iter
uniform 4..64, mapped bytes floor(2^U(10,28)), teams uniform 1..1024, threads
uniform over multiples of 32 in 32..1024, (pf_pos, dist_collapse, pf_collapse)
uniform over the valid combinations for the depth, schedule and data_mode
uniform.  Random numbers come from numpy's PCG64 seeded per workload.
"""
from __future__ import annotations

import dataclasses
import numpy as np

DESC_FIELDS = 16
DESC_BYTES = 128

F_DEPTH, F_TRIP0 = 0, 1
F_FLOPS, F_BYTES, F_H2D, F_D2H = 5, 6, 7, 8
F_TEAMS, F_THREADS = 9, 10
F_PF_POS, F_DIST_COLLAPSE, F_PF_COLLAPSE, F_SCHEDULE, F_DATA_MODE = 11, 12, 13, 14, 15

# Seeds of the named workloads and of the standardisation calibration sample.
SEEDS = {"plain": 1, "batched": 2, "serving": 3, "training": 4, "training_validation": 40, "sweep": 5}
CALIBRATION_SEED = 0xC0FFEE
WEIGHT_SEED_OFFSET = 100


def valid_variant_params(depth: int) -> list[tuple[int, int, int]]:
    """All (pf_pos, dist_collapse, pf_collapse) triples allowed for a loop nest
    of `depth` loops (Sec. 4.1.3): 'parallel for' at loop 0 is combined with
    'teams distribute' (no separate distribute collapse) and may collapse up
    to depth loops; at loop x >= 1 the distribute collapse is 1..x and the
    parallel-for collapse 1..depth-x."""
    out = []
    for pf_pos in range(depth):
        dist_range = [0] if pf_pos == 0 else list(range(1, pf_pos + 1))
        for dc in dist_range:
            for pc in range(1, depth - pf_pos + 1):
                out.append((pf_pos, dc, pc))
    return out


def _loguniform_int(rng, lo_exp, hi_exp, size):
    return np.floor(np.exp2(rng.uniform(lo_exp, hi_exp, size=size))).astype(np.int64)


def make_descriptors(n: int, seed: int, max_depth: int = 3) -> np.ndarray:
    """n random valid descriptors, shape (n, 16) int64, C-contiguous."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = np.ones((n, DESC_FIELDS), dtype=np.int64)
    depth = rng.integers(1, max_depth + 1, size=n)
    d[:, F_DEPTH] = depth
    trips = _loguniform_int(rng, 4.0, 12.0, (n, 4))
    lvl = np.arange(4)[None, :]
    d[:, F_TRIP0:F_TRIP0 + 4] = np.where(lvl < depth[:, None], trips, 1)
    d[:, F_FLOPS] = rng.integers(1, 33, size=n)
    d[:, F_BYTES] = rng.integers(4, 65, size=n)
    d[:, F_H2D] = _loguniform_int(rng, 10.0, 28.0, n)
    d[:, F_D2H] = _loguniform_int(rng, 10.0, 28.0, n)
    d[:, F_TEAMS] = rng.integers(1, 1025, size=n)
    d[:, F_THREADS] = 32 * rng.integers(1, 33, size=n)
    combos = {k: np.array(valid_variant_params(k), dtype=np.int64) for k in range(1, max_depth + 1)}
    pick = rng.random(n)
    for k, c in combos.items():
        sel = depth == k
        idx = np.minimum((pick[sel] * len(c)).astype(np.int64), len(c) - 1)
        d[sel, F_PF_POS:F_PF_POS + 3] = c[idx]
    d[:, F_SCHEDULE] = rng.integers(0, 3, size=n)
    d[:, F_DATA_MODE] = rng.integers(0, 2, size=n)
    return np.ascontiguousarray(d)


def counts_to_offsets(counts: np.ndarray) -> np.ndarray:
    off = np.zeros(len(counts) + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    return off


def make_segments(n_kernels: int, lo: int, hi: int, seed: int, total: int | None = None) -> np.ndarray:
    """Segment offsets [n_kernels+1] for per-kernel variant counts uniform in
    lo..hi.  With `total`, counts are rescaled to sum exactly to total while
    staying in [lo, hi] (scale, round, clamp, then +-1 on random kernels)."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    counts = rng.integers(lo, hi + 1, size=n_kernels).astype(np.int64)
    if total is not None:
        if not (lo * n_kernels <= total <= hi * n_kernels):
            raise ValueError("total out of reach for the count bounds")
        counts = np.clip(np.rint(counts * (total / counts.sum())), lo, hi).astype(np.int64)
        resid = total - int(counts.sum())
        while resid != 0:
            step = 1 if resid > 0 else -1
            ok = np.nonzero((counts + step >= lo) & (counts + step <= hi))[0]
            pick = rng.choice(ok, size=min(abs(resid), len(ok)), replace=False)
            counts[pick] += step
            resid = total - int(counts.sum())
    return counts_to_offsets(counts)


def make_query_sizes(n_queries: int, seed: int) -> np.ndarray:
    """Variant counts of serving queries: floor(2^U(2, 9)), i.e. 4..512, log-uniform."""
    rng = np.random.Generator(np.random.PCG64(seed + 31337))
    return np.minimum(_loguniform_int(rng, 2.0, 9.0, n_queries), 512)


def make_arrivals(n_queries: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Poisson arrival times (seconds from 0) at rate_per_s."""
    rng = np.random.Generator(np.random.PCG64(seed + 4242))
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n_queries))


def param_count(widths) -> int:
    return sum(widths[i + 1] * widths[i] + widths[i + 1] for i in range(len(widths) - 1))


def make_weights(widths, seed: int, init: str = "he", bias_scale: float = 0.0) -> np.ndarray:
    """FP32 master parameters, concatenated per layer as W[out][in] row-major
    followed by b[out].  init 'he' = N(0, 2/fan_in); 'glorot' = U(+-sqrt(6/(in+out)))
    (Sec. 5, Experiment 3).  Biases are 0 unless bias_scale > 0 (then U(+-bias_scale),
    used by tests to exercise the bias path).  Drawn in FP64, rounded to FP32."""
    rng = np.random.Generator(np.random.PCG64(seed + WEIGHT_SEED_OFFSET))
    parts = []
    for i in range(len(widths) - 1):
        fi, fo = widths[i], widths[i + 1]
        if init == "he":
            w = rng.normal(0.0, np.sqrt(2.0 / fi), size=(fo, fi))
        elif init == "glorot":
            a = np.sqrt(6.0 / (fi + fo))
            w = rng.uniform(-a, a, size=(fo, fi))
        else:
            raise ValueError(init)
        b = rng.uniform(-bias_scale, bias_scale, size=fo) if bias_scale > 0 else np.zeros(fo)
        parts += [w.ravel(), b]
    return np.concatenate(parts).astype(np.float32)


def make_labels(desc: np.ndarray, seed: int, noise: float = 0.1) -> np.ndarray:
    """Synthetic measured runtimes (the training-mode data of Sec. 3) as ln seconds:
    ln(max(flops/19.8e15, bytes/8e12) + mapped/5.5e10 + 5e-6) + noise*N(0,1), with
    flops = trip product * flops/iter, bytes = trip product * bytes/iter and
    mapped = h2d + d2h.  This analytic runtime stands in for the measured runtimes
    the paper collects on its clusters; it is an input, not part of the scorer."""
    rng = np.random.Generator(np.random.PCG64(seed + 5151))
    trip_prod = np.prod(desc[:, F_TRIP0:F_TRIP0 + 4].astype(np.float64), axis=1)
    flops = trip_prod * desc[:, F_FLOPS]
    byts = trip_prod * desc[:, F_BYTES]
    mapped = (desc[:, F_H2D] + desc[:, F_D2H]).astype(np.float64)
    t = np.maximum(flops / 19.8e15, byts / 8e12) + mapped / 5.5e10 + 5e-6
    return (np.log(t) + noise * rng.standard_normal(len(desc))).astype(np.float32)


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    widths: tuple
    n_kernels: int
    count_lo: int
    count_hi: int
    total_rows: int | None
    seed: int
    init: str = "he"

    @property
    def n_features(self) -> int:
        return self.widths[0]

    def offsets(self) -> np.ndarray:
        return make_segments(self.n_kernels, self.count_lo, self.count_hi, self.seed, self.total_rows)

    def descriptors(self, n_rows: int | None = None) -> np.ndarray:
        if n_rows is None:
            n_rows = int(self.offsets()[-1])
        return make_descriptors(n_rows, self.seed)

    def weights(self, bias_scale: float = 0.0) -> np.ndarray:
        return make_weights(self.widths, self.seed, self.init, bias_scale)


# The named workloads (sizes from the benchmark descriptions).
PLAIN_FP32_512 = Workload("plain_fp32_64x8", (32, 128, 128, 1), 64, 8, 8, None, SEEDS["plain"])
BATCHED_4096 = Workload("batched_4096k_f64_256x3", (64, 256, 256, 256, 1), 4096, 4, 64, None, SEEDS["batched"])
SERVING = Workload("serving_f32_128x2", (32, 128, 128, 1), 1, 4, 512, None, SEEDS["serving"])
TRAINING = Workload("train_b65536_f64_256x3", (64, 256, 256, 256, 1), 1, 65536, 65536, None, SEEDS["training"], "glorot")
LARGE_SWEEP = Workload("sweep_1m_f128_1024x3", (128, 1024, 1024, 1024, 1), 65536, 2, 64, 1 << 20, SEEDS["sweep"])

WORKLOADS = {w.name: w for w in (PLAIN_FP32_512, BATCHED_4096, SERVING, TRAINING, LARGE_SWEEP)}


def make_dslash_kernels(n_kernels: int, seed: int) -> np.ndarray:
    """Loop nests shaped like the paper's flagship kernel, the Wilson Dslash
    operator (Sec. 5, four nested site loops; Fig. plot_variants_summit runs
    L_X,L_Y,L_Z,L_T = 32,32,32,16): depth 4, trip counts a lattice L^3 x T
    drawn from a few sizes, 1,320 flops and 1,440 bytes per site (single
    precision: 8 gauge links x 72 B + 9 spinors x 96 B), the gauge field and
    source spinor mapped to the device (384 B per site) and the result spinor
    back (96 B per site), teams uniform in 1..1024, threads a multiple of 32
    in 32..1024.  Variant fields are left at their first valid value (the
    enumerator fills them).  Returns [n_kernels][16] int64."""
    rng = np.random.Generator(np.random.PCG64(seed + 4049))
    lattices = np.array([[8, 8, 8, 16], [16, 16, 16, 16], [16, 16, 16, 32], [24, 24, 24, 48], [32, 32, 32, 16],
                         [32, 32, 32, 64]], dtype=np.int64)
    d = np.zeros((n_kernels, DESC_FIELDS), dtype=np.int64)
    lat = lattices[rng.integers(0, len(lattices), size=n_kernels)]
    sites = lat.prod(axis=1)
    d[:, 0] = 4
    d[:, 1:5] = lat
    d[:, 5] = 1320
    d[:, 6] = 1440
    d[:, 7] = sites * 384
    d[:, 8] = sites * 96
    d[:, 9] = rng.integers(1, 1025, size=n_kernels)
    d[:, 10] = 32 * rng.integers(1, 33, size=n_kernels)
    d[:, 11] = 0   # combined 'teams distribute parallel for'
    d[:, 12] = 0
    d[:, 13] = 1
    return d


def calibration_descriptors(n: int = 65536) -> np.ndarray:
    """The fixed sample the z-score standardiser is fitted on (Sec. 5, Experiment 3)."""
    return make_descriptors(n, CALIBRATION_SEED)
