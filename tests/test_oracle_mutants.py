"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of oracle/advisor_oracle.c (a dropped
term, a wrong sign, index or variable, an off-by-one, a transposed operand, a
missing factor), compiles the copy into a temporary directory and runs the
oracle's pin tests against it (ADVISOR_ORACLE_LIB); at least one pin must
fail.  The unmodified source, built the same way, must pass them all.  Every
planted mistake keeps all memory accesses in bounds."""
import concurrent.futures as cf
import os
import subprocess
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "advisor_oracle.c")
PINS = ["tests/test_oracle_log2.py", "tests/test_oracle_features.py", "tests/test_oracle_mlp_select.py",
        "tests/test_oracle_variants_topn.py", "tests/test_metrics_summit.py"]

# name -> (original text, planted mistake); each original occurs exactly once
MUTANTS = {
    "log2: 15 squarings instead of 16": (
        "int32_t bits = 0;\n    for (int i = 0; i < 16; i++) {",
        "int32_t bits = 0;\n    for (int i = 0; i < 15; i++) {"),
    "log2: a squaring that lands on 2 read as below 2": (
        "if (m >= ((uint64_t)1 << 32)) {", "if (m > ((uint64_t)1 << 32)) {"),
    "log2: integer part off by one": (
        "return (int32_t)k * 65536 + bits;", "return (int32_t)(k + 1) * 65536 + bits;"),
    "features: flops-minus-bytes sign": ("b[21] = LFL - LBY;", "b[21] = LBY - LFL;"),
    "features: distributed product takes the parallel-for one": ("b[16] = LD;", "b[16] = LQ;"),
    "features: combined directive ignored": (
        "int64_t dist_n = (pf_pos == 0) ? pc : dc;", "int64_t dist_n = dc;"),
    "features: suffix product starts one level late": (
        "for (int j = i; j < depth; j++) suffix = suffix * t[j];",
        "for (int j = i + 1; j < depth; j++) suffix = suffix * t[j];"),
    "features: log of max(T, P) instead of min": (
        "b[31] = orc_log2_q16((uint64_t)(T < P ? T : P));", "b[31] = orc_log2_q16((uint64_t)(T > P ? T : P));"),
    "features: a one-loop distribute counted as collapsed": (
        "int collapsed = (is_dist[i] && dist_n >= 2) || (is_pf[i] && pc >= 2);",
        "int collapsed = (is_dist[i] && dist_n >= 1) || (is_pf[i] && pc >= 2);"),
    "features: level bytes use the flops": (
        "g[6] = orc_log2_q16((uint64_t)(t[i] * bytes));", "g[6] = orc_log2_q16((uint64_t)(t[i] * flops));"),
    "features: prefix product leaves out its own level": (
        "for (int j = 0; j <= i; j++) prefix = prefix * t[j];", "for (int j = 0; j < i; j++) prefix = prefix * t[j];"),
    "features: pair partner off by one": (
        "int bb = 1 + ((a - 1 + s) % 22);", "int bb = 1 + ((a + s) % 22);"),
    "features: pair difference reversed": ("f[64 + u] = b[a] - b[bb];", "f[64 + u] = b[bb] - b[a];"),
    "features: collapse count of the 33-feature input": (
        "f[32] = (int32_t)(dc + pc) * Q1;", "f[32] = (int32_t)pc * Q1;"),
    "validation: teams bound": (
        "if (d[9] < 1 || d[9] > P2(24) || d[10] < 1 || d[10] > P2(24)) st |= ORC_BAD_PARALLELISM;",
        "if (d[9] < 1 || d[9] > P2(25) || d[10] < 1 || d[10] > P2(24)) st |= ORC_BAD_PARALLELISM;"),
    "validation: distribute collapse may exceed the parallel-for loop": (
        "else             { if (dc < 1 || dc > pf_pos) vok = 0; }",
        "else             { if (dc < 1 || dc > pf_pos + 1) vok = 0; }"),
    "variant count: the combined case counted like the others": (
        "combos += (x == 0 ? 1 : x) * (depth - x);", "combos += (x + 1) * (depth - x);"),
    "validation: trip count bound": (
        "if (i < depth) { if (t < 1 || t > P2(24)) st |= ORC_BAD_TRIP; }",
        "if (i < depth) { if (t < 1 || t > P2(25)) st |= ORC_BAD_TRIP; }"),
    "validation: parallel-for collapse bound": (
        "if (pc < 1 || pc > depth - pf_pos) vok = 0;", "if (pc < 1 || pc > depth) vok = 0;"),
    "standardiser: n - 1 divisor": (
        "double sd = cnt ? sqrt(v / (double)cnt) : 0.0;",
        "double sd = cnt > 1 ? sqrt(v / (double)(cnt - 1)) : 0.0;"),
    "standardiser: invalid rows counted": (
        "if (!status || status[r] == 0) { s = s + (double)feat[F * r + j] / 65536.0; cnt++; }",
        "{ s = s + (double)feat[F * r + j] / 65536.0; cnt++; }"),
    "MLP: bias dropped": ("s = s + (double)b[j];\n            if (pre)", "s = s + 0.0 * (double)b[j];\n            if (pre)"),
    "MLP: weights transposed": (
        "for (int k = 0; k < fi; k++) s = s + (double)W[(size_t)j * fi + k] * in[k];",
        "for (int k = 0; k < fi; k++) s = s + (double)W[(size_t)k * fo + j] * in[k];"),
    "MLP: ReLU on the output layer": (
        "out[j] = (l + 2 < nw) ? (s > 0.0 ? s : 0.0) : s;", "out[j] = s > 0.0 ? s : 0.0;"),
    "MLP: standardisation sign": (
        "for (int k = 0; k < F; k++) ha[k] = ((double)f[k] / 65536.0 - mu[k]) / sigma[k];",
        "for (int k = 0; k < F; k++) ha[k] = ((double)f[k] / 65536.0 + mu[k]) / sigma[k];"),
    "MLP: multiplied by sigma": (
        "for (int k = 0; k < F; k++) ha[k] = ((double)f[k] / 65536.0 - mu[k]) / sigma[k];",
        "for (int k = 0; k < F; k++) ha[k] = ((double)f[k] / 65536.0 - mu[k]) * sigma[k];"),
    "argmin: ties to the higher index": (
        "if (bi < 0 || v < bs) { bi = (int32_t)(r - off[k]); bs = v; }",
        "if (bi < 0 || v <= bs) { bi = (int32_t)(r - off[k]); bs = v; }"),
    "argmin: NaN not skipped": (
        "double v = y[r];\n            if (!(v < INFINITY)) continue;",
        "double v = y[r];\n            if (v == INFINITY) continue;"),
    "top N: equal scores skipped": (
        "if (!(v > pv || (v == pv && i > pi))) continue;", "if (!(v > pv)) continue;"),
    "enumeration: collapse fields swapped": ("v[12] = dc;\n                                v[13] = pc;",
                                             "v[12] = pc;\n                                v[13] = dc;"),
    "enumeration: schedule and data mode loops swapped": (
        "for (int64_t sched = 0; sched < 3; sched++)\n                            for (int64_t dm = 0; dm < 2; dm++) {",
        "for (int64_t dm = 0; dm < 2; dm++)\n                            for (int64_t sched = 0; sched < 3; sched++) {"),
    "loss: factor 1/2 dropped": ("loss = loss + 0.5 * e * e;", "loss = loss + e * e;"),
    "gradient: bias gradient overwritten per row": ("gb[j] = gb[j] + dz;", "gb[j] = dz;"),
    "top N: a missing entry padded with the last score": (
        "score[k * N + t] = bi < 0 ? INFINITY : bv;\n            if (bi >= 0) { pv = bv; pi = bi; }",
        "score[k * N + t] = bi < 0 ? pv : bv;\n            if (bi >= 0) { pv = bv; pi = bi; }"),
    "argmin: empty segment scored 0": ("best_score[k] = bs;", "best_score[k] = bi < 0 ? 0.0 : bs;"),
    "gradient: 1/n dropped": ("dcur[0] = e / (double)n;", "dcur[0] = e;"),
    "gradient: ReLU derivative dropped": (
        "dprev[k] = (pre[aoff[l - 1] + k] > 0.0) ? s : 0.0;", "dprev[k] = s;"),
    "Adam: no bias correction": ("double mh = m[i] / c1, vh = v[i] / c2;", "double mh = m[i], vh = v[i];"),
    "Adam: gradient not squared in v": (
        "v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];", "v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i];"),
    "RMSprop: v not decayed": ("v[i] = alpha * v[i] + (1.0 - alpha) * g * g;", "v[i] = v[i] + (1.0 - alpha) * g * g;"),
    "RMSprop: weight decay dropped": ("const double g = grad[i] + wd * params[i];", "const double g = grad[i];"),
    "RMSE gradient: multiplied instead of divided": (
        "grad[i] = rmse > 0.0 ? grad[i] / rmse : 0.0;", "grad[i] = rmse > 0.0 ? grad[i] * rmse : 0.0;"),
}


def _compile(src_text, out_dir):
    os.makedirs(out_dir, exist_ok=True)
    c = os.path.join(out_dir, "advisor_oracle.c")
    so = os.path.join(out_dir, "liboracle.so")
    with open(c, "w") as f:
        f.write(src_text)
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", c, "-o", so, "-lm"]
    r = subprocess.run(base[:-1] + ["-fopenmp", "-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return so


def _run_pins(so):
    env = dict(os.environ, ADVISOR_ORACLE_LIB=so, OMP_NUM_THREADS="1")
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)


def test_pins_catch_every_planted_mistake(tmp_path):
    src = open(SRC).read()
    for name, (orig, bad) in MUTANTS.items():
        assert src.count(orig) == 1, f"{name}: the original text is not unique in the oracle source"
    jobs = {"unmodified": _compile(src, str(tmp_path / "control"))}
    for i, (name, (orig, bad)) in enumerate(MUTANTS.items()):
        jobs[name] = _compile(src.replace(orig, bad), str(tmp_path / f"m{i}"))
    with cf.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        res = dict(zip(jobs, ex.map(_run_pins, jobs.values())))
    control = res.pop("unmodified")
    assert control.returncode == 0, control.stdout[-3000:]
    missed = [name for name, r in res.items() if r.returncode != 1 or " failed" not in r.stdout]
    assert not missed, f"planted mistakes no pin caught: {missed}"
