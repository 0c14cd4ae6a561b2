"""Serving on the GPU: continuous batching of Poisson-arriving queries (one
kernel of 4..512 variants each, plain-method descriptor distribution and
network), several batches in flight; every answer equals the answer for the
same query ranked alone, and sampled answers equal the FP64 oracle's."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_03636_gb300 import advisor, serving
from paper_2301_03636_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served():
    wl = W.SERVING
    cal = torch.from_numpy(W.calibration_descriptors(16384)).cuda()
    fcal, scal = advisor.advisor_extract_features(cal, wl.n_features)
    mu, sigma = advisor.advisor_fit_standardizer(fcal, scal)
    params = wl.weights()
    base = advisor.Model(wl.widths, max_rows=16384, max_kernels=512)
    base.set_params(params, mu, sigma)
    eps = base.calibrate_eps(fcal, scal, "bf16")
    eps32 = base.calibrate_eps(fcal, scal, "fp32")
    queries = serving.make_queries(1500, 20000.0, W.SEEDS["serving"])
    # admission by device memory: 3 pipelines sharing a 144 MB budget
    done, st = serving.run_serving(base, params, mu, sigma, queries, "bf16", eps, eps32, pipelines=3,
                                   memory_budget_bytes=144 << 20)
    print("serving stats:", st)
    return dict(base=base, done=done, st=st, eps=eps, eps32=eps32, mu=mu.cpu().numpy(),
                sigma=sigma.cpu().numpy(), params=params, wl=wl)


def test_every_query_answered(gpu_lib, served):
    done = served["done"]
    assert len(done) == 1500 and len({q.qid for q in done}) == 1500
    assert all(q.status == "done" and 0 <= q.best < q.rows for q in done)
    st = served["st"]
    assert st["p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"]


def test_batches_overlap_on_the_gpu(gpu_lib, served):
    """Continuous batching, not a queue alone: at some instant at least two
    pipelines had a batch in flight on the GPU (copy-in .. copy-out intervals,
    timed by events on their streams, overlapping)."""
    st = served["st"]
    print("batches:", st["batches"], "max in flight:", st["max_batches_in_flight"],
          "rows per batch:", st["rows_per_batch_capacity"])
    assert st["max_batches_in_flight"] >= 2
    assert st["rows_per_batch_capacity"] >= 512   # the device-memory budget admits the largest query


def test_alone_equals_mix(gpu_lib, served):
    base = served["base"]
    for q in served["done"]:
        d = torch.from_numpy(q.desc).cuda()
        off = torch.tensor([0, q.rows], dtype=torch.int64, device="cuda")
        b, s = base.rank(d, off, "bf16", served["eps"], served["eps32"])
        assert int(b.item()) == q.best and float(s.item()) == q.score, q.qid


def test_sampled_answers_match_oracle(gpu_lib, served):
    wl = served["wl"]
    rng = np.random.Generator(np.random.PCG64(5))
    for q in rng.choice(served["done"], size=200, replace=False):
        best, _, _, _, _ = oracle.rank(q.desc, np.array([0, q.rows]), wl.widths, served["params"], served["mu"],
                                       served["sigma"])
        assert best[0] == q.best, q.qid
