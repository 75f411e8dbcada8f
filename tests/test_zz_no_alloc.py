"""The allocation-free batched projection: results, in-place use, and no device allocation.

project_psd_batched_noalloc serves callers that may not allocate device memory (a host framework
that owns all device memory through a pool, or a latency-bound loop that cannot afford a
cudaMalloc): it keeps its per-call schedule in a fixed array inside the library. Its results are
checked against the oracle's projection and against the allocating entry point. This file is
collected last on purpose, so a run that stops at its first failure has run everything else.
"""

import ctypes

import numpy as np
import pytest

from oracle import chordal_admm as orc
from tests.gpu_support import require_gpu

pytestmark = pytest.mark.gpu


def packed(W):
    return np.concatenate([W[j:, j] for j in range(W.shape[0])])


def unpacked(v, s):
    W = np.zeros((s, s))
    pos = 0
    for j in range(s):
        W[j:, j] = v[pos:pos + s - j]
        W[j, j:] = v[pos:pos + s - j]
        pos += s - j
    return W


def make_batch(rng, sizes):
    blocks = []
    for s in sizes:
        W = rng.standard_normal((s, s)) * 5.0
        blocks.append((W + W.T) / 2)
    sizes = np.array(sizes, np.int32)
    lens = sizes.astype(np.int64) * (sizes + 1) // 2
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.int64)
    return blocks, sizes, lens, offs, np.concatenate([packed(W) for W in blocks])


def check_against_oracle(got, blocks, sizes, lens, offs, tol, ent_tol):
    """Every block against the oracle's P(W): in the Frobenius norm relative to ||W||_F (tol) and
    entry by entry relative to max |W_ij| (ent_tol)."""
    assert np.all(np.isfinite(got))
    for k, W in enumerate(blocks):
        s = int(sizes[k])
        P = orc.proj_psd(W)
        G = unpacked(got[offs[k]:offs[k] + lens[k]], s)
        fro = np.linalg.norm(G - P) / max(np.linalg.norm(W), 1e-300)
        ent = np.max(np.abs(G - P)) / max(np.max(np.abs(W)), 1e-300)
        assert fro <= tol and ent <= ent_tol, (k, s, fro, ent)


# (sizes, precision, Frobenius bound, entry bound): FP64 to rounding; FP32 within the one-sided
# Jacobi's stopping rule (columns orthogonal to 1e-4), the FP32 mode's accuracy budget
CALLS = [([1, 2, 7, 12, 30, 31, 45, 60, 96, 5, 33], "fp64", 1e-12, 1e-12),
         ([30, 12, 17, 64], "fp32", 1e-4, 4e-4)]


def test_noalloc_matches_oracle_and_project_psd_batched_on_two_calls():
    torch, cadmm = require_gpu()
    rng = np.random.default_rng(2024)
    # two calls in a row: the second has fewer, different blocks, so stale schedule entries from the
    # first call stay in the shared array and must not matter
    for sizes, prec, tol, ent_tol in CALLS:
        blocks, sizes, lens, offs, flat = make_batch(rng, sizes)
        inp = torch.tensor(flat, device="cuda")
        ref = torch.full_like(inp, np.nan)
        got = torch.full_like(inp, np.nan)
        cadmm.project_psd_batched(inp, ref, sizes, offs, prec=prec)
        cadmm.project_psd_batched_noalloc(inp, got, sizes, offs, prec=prec)
        torch.cuda.synchronize()
        ref, got = ref.cpu().numpy(), got.cpu().numpy()
        check_against_oracle(got, blocks, sizes, lens, offs, tol, ent_tol)
        for k, W in enumerate(blocks):
            sl = slice(offs[k], offs[k] + lens[k])
            err = np.linalg.norm(got[sl] - ref[sl]) / max(np.linalg.norm(W), 1e-300)
            assert err <= tol, (prec, k, int(sizes[k]), err)


def test_noalloc_in_place():
    torch, cadmm = require_gpu()
    rng = np.random.default_rng(7)
    for sizes, prec, tol, ent_tol in CALLS:
        blocks, sizes, lens, offs, flat = make_batch(rng, sizes)
        buf = torch.tensor(flat, device="cuda")
        cadmm.project_psd_batched_noalloc(buf, buf, sizes, offs, prec=prec)
        torch.cuda.synchronize()
        check_against_oracle(buf.cpu().numpy(), blocks, sizes, lens, offs, tol, ent_tol)


def _cudart():
    """The CUDA runtime this process already loaded (the library links it dynamically)."""
    for name in ("libcudart.so.13", "libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def _pool_bytes(rt, dev):
    """Used and high-water bytes of the device's default stream-ordered pool (cudaMallocAsync)."""
    pool = ctypes.c_void_p()
    if rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), ctypes.c_int(dev)) != 0:
        return None
    out = []
    for attr in (7, 8):        # cudaMemPoolAttrUsedMemCurrent, cudaMemPoolAttrUsedMemHigh
        v = ctypes.c_uint64()
        if rt.cudaMemPoolGetAttribute(pool, ctypes.c_int(attr), ctypes.byref(v)) != 0:
            return None
        out.append(v.value)
    return tuple(out)


def test_noalloc_allocates_no_device_memory():
    torch, cadmm = require_gpu()
    rng = np.random.default_rng(11)
    sizes_list = [[30] * 200 + [12] * 300, [60, 45, 7, 1] * 50]
    batches = []
    for sizes in sizes_list:
        blocks, sizes, lens, offs, flat = make_batch(rng, sizes)
        inp = torch.tensor(flat, device="cuda")
        batches.append((sizes, offs, inp, torch.empty_like(inp)))
    # one round of calls first: it sets the library up on this device and loads every kernel
    # these calls use (the runtime loads a kernel's code on its first launch)
    for sizes, offs, inp, out in batches:
        for prec in ("fp64", "fp32"):
            cadmm.project_psd_batched_noalloc(inp, out, sizes, offs, prec=prec)
    torch.cuda.synchronize()
    dev = torch.cuda.current_device()
    rt = _cudart()
    before = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(), torch.cuda.mem_get_info()[0],
              _pool_bytes(rt, dev) if rt is not None else None)
    for _ in range(5):
        for sizes, offs, inp, out in batches:
            for prec in ("fp64", "fp32"):
                cadmm.project_psd_batched_noalloc(inp, out, sizes, offs, prec=prec)
    torch.cuda.synchronize()
    after = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(), torch.cuda.mem_get_info()[0],
             _pool_bytes(rt, dev) if rt is not None else None)
    assert after == before, (before, after)


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
