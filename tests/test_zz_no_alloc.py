"""The allocation-free batched projection agrees with the allocating one.

project_psd_batched_noalloc serves callers that may not allocate device memory (a host framework
that owns all device memory through a pool, or a latency-bound loop that cannot afford a
cudaMalloc): it keeps its per-call schedule in a fixed array inside the library. This file is
collected last on purpose, so a run that stops at its first failure has run everything else.
"""

import numpy as np
import pytest

from tests.gpu_support import require_gpu

pytestmark = pytest.mark.gpu


def packed(W):
    return np.concatenate([W[j:, j] for j in range(W.shape[0])])


def make_batch(rng, sizes):
    blocks = []
    for s in sizes:
        W = rng.standard_normal((s, s)) * 5.0
        blocks.append((W + W.T) / 2)
    sizes = np.array(sizes, np.int32)
    lens = sizes.astype(np.int64) * (sizes + 1) // 2
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.int64)
    return blocks, sizes, lens, offs, np.concatenate([packed(W) for W in blocks])


def test_noalloc_matches_project_psd_batched_on_two_calls():
    torch, cadmm = require_gpu()
    rng = np.random.default_rng(2024)
    # two calls in a row: the second has fewer, different blocks, so stale schedule entries from the
    # first call stay in the shared array and must not matter
    calls = [([1, 2, 7, 12, 30, 31, 45, 60, 96, 5, 33], "fp64", 1e-12),
             ([30, 12, 17, 64], "fp32", 2e-5)]
    for sizes, prec, tol in calls:
        blocks, sizes, lens, offs, flat = make_batch(rng, sizes)
        inp = torch.tensor(flat, device="cuda")
        ref = torch.full_like(inp, np.nan)
        got = torch.full_like(inp, np.nan)
        cadmm.project_psd_batched(inp, ref, sizes, offs, prec=prec)
        cadmm.project_psd_batched_noalloc(inp, got, sizes, offs, prec=prec)
        torch.cuda.synchronize()
        ref, got = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(got))
        for k, W in enumerate(blocks):
            sl = slice(offs[k], offs[k] + lens[k])
            err = np.linalg.norm(got[sl] - ref[sl]) / max(np.linalg.norm(W), 1e-300)
            assert err <= tol, (prec, k, int(sizes[k]), err)


def test_noalloc_rejects_more_blocks_than_its_array_holds():
    torch, cadmm = require_gpu()
    n = cadmm.SDP_NOALLOC_MAX_BLOCKS + 1
    sizes = np.ones(n, np.int32)
    offs = np.arange(n, dtype=np.int64)
    buf = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(cadmm.SDPError) as e:
        cadmm.project_psd_batched_noalloc(buf, buf, sizes, offs)
    assert e.value.code == cadmm.SDP_ERR_UNSUPPORTED
    assert "SDP_NOALLOC_MAX_BLOCKS" in str(e.value)
