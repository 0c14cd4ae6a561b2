"""a1-a2 on the GPU: validation status and integer features bit-exact against
the oracle, on random rows, every validation bound and invalid rows."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_03636_gb300 import advisor
from tests._cases import edge_descriptors, mixed_descriptors

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("F", [32, 64, 128])
def test_edge_rows_bit_exact(gpu_lib, F):
    d = edge_descriptors()
    f_ref, st_ref = oracle.extract_features(d, F)
    f, st = advisor.advisor_extract_features(torch.from_numpy(d).cuda(), F)
    assert np.array_equal(st.cpu().numpy(), st_ref)
    assert np.array_equal(f.cpu().numpy(), f_ref)


@pytest.mark.parametrize("F,n", [(32, 1), (64, 127), (64, 129), (128, 5000), (64, 200_003)])
def test_random_rows_bit_exact(gpu_lib, F, n):
    d = mixed_descriptors(max(n, 64), 1000 + n)[:n]
    f_ref, st_ref = oracle.extract_features(d, F)
    f, st = advisor.advisor_extract_features(torch.from_numpy(d).cuda(), F)
    assert np.array_equal(st.cpu().numpy(), st_ref)
    assert np.array_equal(f.cpu().numpy(), f_ref)


@pytest.mark.parametrize("F", [32, 33, 64])
def test_hand_worked_rows(gpu_lib, F):
    """The four hand-worked descriptors of the oracle's pins, on the GPU:
    every feature equals the value written out by hand."""
    from tests.test_oracle_features import (D1, D1_BASE, D1_LEVELS, D2, D2_BASE, D2_LEVELS, D3, D3_BASE,
                                            D3_LEVELS, D4, D4_BASE, D4_LEVELS, Q)
    d = np.stack([D1, D2, D3, D4])
    want = []
    for base, levels, collapsed in ((D1_BASE, D1_LEVELS, 1), (D2_BASE, D2_LEVELS, 2), (D3_BASE, D3_LEVELS, 3),
                                    (D4_BASE, D4_LEVELS, 4)):
        want.append(base if F == 32 else base + [collapsed * Q] if F == 33 else base + sum(levels, []))
    f, st = advisor.advisor_extract_features(torch.from_numpy(d).cuda(), F)
    assert st.cpu().numpy().tolist() == [0, 0, 0, 0]
    assert f.cpu().numpy().tolist() == want


def test_empty_call(gpu_lib):
    f, st = advisor.advisor_extract_features(torch.empty((0, 16), dtype=torch.int64, device="cuda"), 64)
    assert f.shape == (0, 64) and st.shape == (0,)


def test_fit_standardizer_matches_oracle(gpu_lib):
    d = mixed_descriptors(30_000, 5)
    f_ref, st_ref = oracle.extract_features(d, 64)
    mu_ref, sg_ref = oracle.fit_standardizer(f_ref, st_ref)
    f, st = advisor.advisor_extract_features(torch.from_numpy(d).cuda(), 64)
    mu, sg = advisor.advisor_fit_standardizer(f, st)
    assert np.allclose(mu.cpu().numpy(), mu_ref, rtol=1e-12, atol=1e-12)
    assert np.allclose(sg.cpu().numpy(), sg_ref, rtol=1e-10, atol=1e-12)
