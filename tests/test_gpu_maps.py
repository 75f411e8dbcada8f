"""GPU parity of the clique index maps, the gather H_k x and the scatter Σ H_kᵀ v_k: bit-exact."""

import numpy as np
import pytest

from sdp_inputs import config_instance
from tests import sdp_cases
from tests.gpu_support import (blocks_to_packed, make_oracle, packed_to_blocks, require_gpu,
                               setup_handle)

pytestmark = pytest.mark.gpu


def chain_case():
    """A chordal pattern that is not block-arrow: overlapping cliques of ragged sizes."""
    rng = np.random.default_rng(21)
    cliques = [np.arange(0, 3), np.arange(1, 6), np.arange(5, 12), np.array([11, 12]),
               np.arange(12, 20), np.arange(14, 21)]   # a clique path: chordal, ragged sizes
    n = 21
    P = np.zeros((n, n), bool)
    for c in cliques:
        P[np.ix_(c, c)] = True
    C = rng.standard_normal((n, n)); C = (C + C.T) * P
    C += np.diag(np.abs(C).sum(1) + 1)
    As = []
    for _ in range(5):
        A = rng.standard_normal((n, n)) * (rng.random((n, n)) < 0.4)
        A = (np.tril(A) + np.tril(A, -1).T) * P
        As.append(A)
    b = rng.standard_normal(5)
    return sdp_cases.problem_from_dense(C, As, b, cliques)


CASES = {
    "config0": lambda: sdp_cases.instance_arrays(config_instance(0)),
    "heavy_overlap": lambda: sdp_cases.random_block_arrow(l=40, d=1, h=4, m=6, seed=3),
    "chain_ragged": chain_case,
    "dense_one_clique": lambda: dict(sdp_cases.theta_c5()[0]),
}


@pytest.fixture(params=sorted(CASES), scope="module")
def case(request):
    torch, cadmm = require_gpu()
    arrs = CASES[request.param]()
    sdp = make_oracle(arrs)
    s = setup_handle(cadmm, arrs)
    yield torch, cadmm, arrs, sdp, s
    s.close()


def test_index_maps_bit_exact(case):
    torch, cadmm, arrs, sdp, s = case
    maps = cadmm.sdp_get_maps(s.h)
    lower = sdp.lower_mask()
    np.testing.assert_array_equal(maps["pat_row"], sdp.E_row[lower])
    np.testing.assert_array_equal(maps["pat_col"], sdp.E_col[lower])
    sizes = [len(c) for c in sdp.cliques]
    np.testing.assert_array_equal(maps["blk_off"], np.concatenate([[0], np.cumsum([t * (t + 1) // 2 for t in sizes])]))
    low_index = np.cumsum(lower) - 1          # full E position -> E_L position (for lower entries)
    expected = []
    for k, c in enumerate(sdp.cliques):
        t = len(c)
        for bcol in range(t):
            for a in range(bcol, t):
                expected.append(low_index[sdp.idx[k][a + bcol * t]])
    np.testing.assert_array_equal(maps["gather_idx"], np.array(expected))


def test_gather_bit_exact(case):
    torch, cadmm, arrs, sdp, s = case
    rng = np.random.default_rng(5)
    nl = s.sizes["nE_lower"]
    x_low = rng.standard_normal(nl)
    x_full = sdp.from_lower(sdp.E_row[sdp.lower_mask()], sdp.E_col[sdp.lower_mask()], x_low)
    xd = torch.tensor(x_low, device="cuda")
    out = torch.full((s.sizes["S_lower"],), np.nan, dtype=torch.float64, device="cuda")
    cadmm.sdp_gather(s.h, xd, out)
    torch.cuda.synchronize()
    ref = blocks_to_packed(sdp, [sdp.H(k, x_full) for k in range(sdp.p)])
    assert np.array_equal(out.cpu().numpy(), ref)


def test_scatter_bit_exact(case):
    torch, cadmm, arrs, sdp, s = case
    rng = np.random.default_rng(6)
    packed = rng.standard_normal(s.sizes["S_lower"]) * 10.0 ** rng.integers(-3, 4, s.sizes["S_lower"])
    out = torch.full((s.sizes["nE_lower"],), np.nan, dtype=torch.float64, device="cuda")
    cadmm.sdp_scatter(s.h, torch.tensor(packed, device="cuda"), out)
    torch.cuda.synchronize()
    ref = sdp.to_lower(sdp.HT_sum(packed_to_blocks(sdp, packed)))
    assert np.array_equal(out.cpu().numpy(), ref)
