"""GPU parity of the batched PSD projection (Eqs. XkUpdate, zkUpdate) against the oracle."""

import numpy as np
import pytest

from oracle import chordal_admm as orc
from tests.gpu_support import require_gpu

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 3, 5, 12, 15, 16, 17, 30, 31, 32, 33, 40, 60, 64, 95, 96]


def packed(W):
    s = W.shape[0]
    return np.concatenate([W[j:, j] for j in range(s)])


def unpacked(v, s):
    W = np.zeros((s, s))
    pos = 0
    for j in range(s):
        W[j:, j] = v[pos:pos + s - j]
        W[j, j:] = v[pos:pos + s - j]
        pos += s - j
    return W


def special_blocks(rng):
    out = []
    out.append(np.zeros((7, 7)))                                  # zero
    out.append(np.diag(rng.standard_normal(9)))                   # diagonal
    out.append(3.0 * np.eye(8))                                   # repeated eigenvalue, PSD
    out.append(-2.0 * np.eye(6))                                  # NSD
    g = rng.standard_normal(11); out.append(np.outer(g, g))       # rank one
    G = rng.standard_normal((13, 13)); out.append(-(G @ G.T))     # NSD dense
    W = rng.standard_normal((10, 10)); out.append((W + W.T) * 1e-20)   # tiny scale
    W = rng.standard_normal((10, 10)); out.append((W + W.T) * 1e20)    # huge scale
    Q, _ = np.linalg.qr(rng.standard_normal((20, 20)))
    ev = np.repeat([2.0, -1.0, 0.0, 5.0], 5)                      # clustered spectrum
    out.append((Q * ev) @ Q.T)
    return out


def batch(rng):
    blocks = []
    for s in SIZES:
        W = rng.standard_normal((s, s)) * 10.0
        blocks.append((W + W.T) / 2)
    blocks += special_blocks(rng)
    return blocks


def entry_err(P, ref, W):
    """Largest entry error relative to the largest entry of W."""
    return float(np.max(np.abs(P - ref)) / max(np.max(np.abs(W)), 1e-300))


@pytest.mark.parametrize("prec,tol,ent_tol", [("fp64", 1e-12, 1e-12), ("fp32", 1e-4, 4e-4)])
def test_project_matches_oracle(prec, tol, ent_tol):
    """The default plan on random and special blocks against the oracle. FP64: rounding. FP32:
    the one-sided eigensolvers stop once every pair of columns began a sweep orthogonal to 1e-4,
    which bounds the projection's error by about 1e-4 ||W||_F (cold starts on random and clustered
    blocks land between 1e-5 and 5e-5, by rounding; a CPU simulation of the same arithmetic shows
    the same spread); entries by four times that relative to max |W_ij|."""
    torch, cadmm = require_gpu()
    rng = np.random.default_rng(42)
    blocks = batch(rng)
    sizes = np.array([b.shape[0] for b in blocks], np.int32)
    lens = sizes.astype(np.int64) * (sizes + 1) // 2
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.int64)
    flat = np.concatenate([packed(b) for b in blocks])
    inp = torch.tensor(flat, device="cuda")
    out = torch.full_like(inp, np.nan)
    cadmm.project_psd_batched(inp, out, sizes, offs, prec=prec)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for k, W in enumerate(blocks):
        s = W.shape[0]
        P = unpacked(got[offs[k]:offs[k] + lens[k]], s)
        ref = orc.proj_psd(W)
        nW = max(np.linalg.norm(W), 1e-300)
        err = np.linalg.norm(P - ref) / nW
        assert err <= tol, (k, s, prec, err)
        assert entry_err(P, ref, W) <= ent_tol, (k, s, prec, entry_err(P, ref, W))
        if np.linalg.norm(W) > 0:
            assert np.linalg.eigvalsh(P)[0] >= -tol * nW


def test_project_in_place_and_empty():
    torch, cadmm = require_gpu()
    rng = np.random.default_rng(7)
    W = rng.standard_normal((30, 30)); W = W + W.T
    v = torch.tensor(np.concatenate([packed(W), packed(-W)]), device="cuda")
    sizes = np.array([30, 30], np.int32)
    offs = np.array([0, 465], np.int64)
    cadmm.project_psd_batched(v, v, sizes, offs, prec="fp64")
    torch.cuda.synchronize()
    got = v.cpu().numpy()
    # Moreau: W = P(W) - P(-W)
    np.testing.assert_allclose(unpacked(got[:465], 30) - unpacked(got[465:], 30), W,
                               atol=1e-12 * np.linalg.norm(W))
    cadmm.project_psd_batched(v, v, np.zeros(0, np.int32), np.zeros(0, np.int64))


@pytest.mark.parametrize("prec,tol,ent_tol", [("fp64", 1e-12, 1e-12), ("fp32", 1e-4, 4e-4)])
def test_every_variant_matches_oracle(prec, tol, ent_tol, capsys):
    """Each eigensolver kernel variant, forced on every order it accepts (random blocks, several
    per order so warp segments and CTAs hold more than one, plus the special blocks that fit),
    against the oracle's projection, in the Frobenius norm relative to ||W||_F and entry by entry
    relative to max |W_ij|. The FP32 bound is the one-sided variants' stopping rule (columns
    orthogonal to 1e-4 relative): from a cold start on a block with four 5-fold eigenvalue
    clusters they come within about 7.5e-5 of ||W||_F. On that block ||W||_F is about four times
    max |W_ij|, so its entry bound is four times the Frobenius one."""
    torch, cadmm = require_gpu()
    names = cadmm.project_variants()
    rng = np.random.default_rng(11)
    base = []
    for s in SIZES:
        for _ in range(3):
            W = rng.standard_normal((s, s))
            base.append((W + W.T) / 2)
    base += special_blocks(rng)
    tested = 0
    worst, worst_ent = {}, {}
    for v, name in enumerate(names):
        blocks = [W for W in base if cadmm.project_variant_fits(v, W.shape[0], prec)]
        if not blocks:
            continue
        sizes = np.array([b.shape[0] for b in blocks], np.int32)
        lens = sizes.astype(np.int64) * (sizes + 1) // 2
        offs = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.int64)
        inp = torch.tensor(np.concatenate([packed(b) for b in blocks]), device="cuda")
        out = torch.full_like(inp, np.nan)
        cadmm.project_psd_batched_variant(inp, out, sizes, offs, v, prec=prec)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for k, W in enumerate(blocks):
            s = W.shape[0]
            P, ref = unpacked(got[offs[k]:offs[k] + lens[k]], s), orc.proj_psd(W)
            err = np.linalg.norm(P - ref) / max(np.linalg.norm(W), 1e-300)
            ent = entry_err(P, ref, W)
            assert err <= tol and ent <= ent_tol, (name, k, s, err, ent)
            worst[name] = max(worst.get(name, 0.0), float(err))
            worst_ent[name] = max(worst_ent.get(name, 0.0), ent)
        tested += 1
    assert tested >= (4 if prec == "fp64" else 8)
    with capsys.disabled():
        print(f"\n{prec} projection variants, worst error / ||W||:", {k: f"{v:.1e}" for k, v in worst.items()})
        print(f"{prec} projection variants, worst entry error / max|W|:",
              {k: f"{v:.1e}" for k, v in worst_ent.items()})


def test_project_refuses_stream_capture():
    """project_psd_batched copies its schedule from a host buffer that lives for the call only, so
    on a capturing stream it returns SDP_ERR_UNSUPPORTED instead of recording that copy."""
    torch, cadmm = require_gpu()
    rng = np.random.default_rng(9)
    W = rng.standard_normal((12, 12)); W = W + W.T
    v = torch.tensor(packed(W), device="cuda")
    sizes, offs = np.array([12], np.int32), np.array([0], np.int64)
    cadmm.project_psd_batched(v, v, sizes, offs)          # prepares the kernels outside the capture
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        g.capture_begin()
        try:
            with pytest.raises(cadmm.SDPError) as e:
                cadmm.project_psd_batched(v, v, sizes, offs, stream=stream)
        finally:
            g.capture_end()
    assert e.value.code == cadmm.SDP_ERR_UNSUPPORTED
    assert "captured" in str(e.value)
