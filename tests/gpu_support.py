"""Helpers shared by the GPU parity tests: oracle <-> C-ABI layout conversions and setup."""

from __future__ import annotations

import numpy as np
import pytest

from oracle import chordal_admm as orc


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_06068_gb300 as cadmm
    cadmm.load_library()           # raises when the library is missing: no silent fallback
    return torch, cadmm


def make_oracle(arrs) -> orc.ChordalSDP:
    return orc.ChordalSDP(arrs["n"], arrs["cliques"], arrs["A_ptr"], arrs["A_row"], arrs["A_col"],
                          arrs["A_val"], arrs["b"], arrs["C_row"], arrs["C_col"], arrs["C_val"],
                          cones=arrs.get("cones"))


def blocks_to_packed(sdp: orc.ChordalSDP, blocks) -> np.ndarray:
    """Oracle blocks in the packed layout: clique blocks as lower triangles, cone blocks as they are."""
    out = [sdp.block_to_packed(b, len(c)) for b, c in zip(blocks[:sdp.p], sdp.cliques)]
    out += [np.asarray(b, dtype=np.float64) for b in blocks[sdp.p:]]
    return np.concatenate(out) if out else np.zeros(0)


def packed_to_blocks(sdp: orc.ChordalSDP, packed: np.ndarray):
    out, pos = [], 0
    for c in sdp.cliques:
        s = len(c)
        n = s * (s + 1) // 2
        out.append(sdp.packed_to_block(packed[pos:pos + n], s))
        pos += n
    for k in range(sdp.p, sdp.nblk):
        q = sdp.block_len(k)
        out.append(np.array(packed[pos:pos + q], dtype=np.float64))
        pos += q
    return out


def oracle_state_to_abi(sdp: orc.ChordalSDP, st: dict) -> dict:
    """Oracle iterates in the C ABI's layout (x on E_L, packed blocks)."""
    d = dict(x=sdp.to_lower(st["x"]), y=st["y"].copy(), blk_b=blocks_to_packed(sdp, st["lam"]))
    if st["form"] == "primal":
        d["blk_a"] = blocks_to_packed(sdp, st["xk"])
    else:
        d["blk_a"] = blocks_to_packed(sdp, st["zk"])
        d["blk_c"] = blocks_to_packed(sdp, st["vk"])
    return d


def rel_err(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b)), 1e-30))


def setup_handle(cadmm, arrs, form="primal", prec="fp64", rho=1.0, tol=1e-4, max_iter=2000,
                 check_every=16, flags=0):
    opts = cadmm.make_opts(rho=rho, tol=tol, max_iter=max_iter, check_every=check_every, form=form,
                           prec=prec, flags=flags)
    return cadmm.ChordalADMM(arrs, opts)
