"""Autotuner for the batched PSD projection (Eqs. XkUpdate / zkUpdate): picks, for every padded
clique order N present, the eigensolver kernel variant that runs fastest.

The variants differ in how a block is laid out on the GPU (a warp segment of 8/16/32 lanes per
block, a CTA of 4 or 8 warps per block, or the two-sided CTA kernel) and in the largest order they
take. Which is fastest depends on the order and on how many blocks run at once, so the choice is
measured, not modelled:

  - ``tune_blocks`` times every fitting variant on synthetic symmetric blocks of each order
    (cold starts, one launch per variant and order);
  - ``tune_handle`` times the projection phase of a handle's own iterations (warm starts, the
    handle's real mix of sizes), changing one order's variant at a time.

Tables are ``{N: variant}`` dicts; ``sdp_set_proj_table`` applies one to a handle, and
``save_table`` / ``load_table`` keep one as JSON.
"""

from __future__ import annotations

import json

import numpy as np

from . import (PRECS, SDP_MAX_CLIQUE, _check, load_library, project_psd_batched_variant,
               project_variant_fits, project_variants, sdp_get_maps, sdp_get_sizes, sdp_set_proj_table,
               sdp_time_phases)


def _time_ms(fn, reps: int) -> float:
    import torch
    fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return float(np.median(times))


def tune_blocks(prec="fp32", orders=None, count=4096, reps=5, seed=0) -> dict:
    """Fastest variant per even order N on ``count`` random symmetric blocks of order N."""
    import torch
    names = project_variants()
    orders = sorted(set(orders)) if orders is not None else list(range(2, SDP_MAX_CLIQUE + 1, 2))
    rng = np.random.default_rng(seed)
    table, times = {}, {}
    for N in orders:
        s = int(N)
        plen = s * (s + 1) // 2
        sizes = np.full(count, s, np.int32)
        offsets = (np.arange(count, dtype=np.int64) * plen)
        inp = torch.tensor(rng.standard_normal(count * plen), device="cuda")
        out = torch.empty_like(inp)
        cand = [v for v in range(len(names)) if project_variant_fits(v, s, prec)]
        t = {names[v]: _time_ms(lambda v=v: project_psd_batched_variant(inp, out, sizes, offsets, v, prec), reps)
             for v in cand}
        best = min(cand, key=lambda v: t[names[v]])
        table[int(N)] = int(best)
        times[int(N)] = t
    return dict(prec=prec, source="synthetic blocks", count=count, table=table, times=times)


def handle_orders(h) -> list:
    """Padded orders N of the handle's cliques, largest first."""
    sz = sdp_get_sizes(h)
    off = sdp_get_maps(h)["blk_off"]
    plen = np.diff(off)
    s = ((np.sqrt(8 * plen + 1) - 1) / 2).round().astype(np.int64)
    return sorted({int(x + (x & 1)) for x in s[: sz["p"]]}, reverse=True)


def tune_handle(h, prec="fp32", reps=3) -> dict:
    """Fastest variant per padded order, measured on the handle's own projection phase.

    Coordinate descent in one pass, largest orders first: for each order N, every fitting variant
    is tried with the other orders fixed at their current choice. The iterations run for real, so
    reset the handle afterwards."""
    names = project_variants()
    orders = handle_orders(h)
    table = {}
    times = {}

    def project_ms():
        ph = sdp_time_phases(h, reps=reps)
        return sum(v for k, v in ph.items() if k.startswith("project"))

    sdp_set_proj_table(h, prec, None)
    for N in orders:
        cand = [v for v in range(len(names)) if project_variant_fits(v, N, prec)]
        t = {}
        for v in cand:
            trial = dict(table)
            trial[N] = v
            sdp_set_proj_table(h, prec, trial)
            t[names[v]] = project_ms()
        best = min(cand, key=lambda v: t[names[v]])
        table[N] = int(best)
        times[N] = t
    sdp_set_proj_table(h, prec, table)
    return dict(prec=prec, source="handle projection phase", table=table, times=times)


def save_table(result: dict, path: str):
    with open(path, "w") as f:
        json.dump(dict(result, table={str(k): v for k, v in result["table"].items()},
                       variants=project_variants()), f, indent=1, sort_keys=True)


def load_table(path: str) -> dict:
    with open(path) as f:
        d = json.load(f)
    names = project_variants()
    # variants are stored by index; re-map through their names in case the list changed
    saved = d.get("variants", names)
    return {int(k): names.index(saved[v]) for k, v in d["table"].items() if saved[v] in names}


__all__ = ["tune_blocks", "tune_handle", "handle_orders", "save_table", "load_table", "PRECS", "_check",
           "load_library"]
