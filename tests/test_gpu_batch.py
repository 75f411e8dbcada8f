"""GPU parity of batched solves: independent block-arrow SDPs of uneven size in one handle.

A batch handle is the block-diagonal union of its problems; each problem must follow its own ADMM
iteration (Algorithms 1 and 2) exactly as a separate solve would, stop at its own first iteration
below the tolerance, and stay frozen afterwards. Instances are those of the 512-problem workload
(l ~ U{5..60}, d ~ U{4..24}, h ~ U{1..16}, m ~ U{20..300}).
"""

import numpy as np
import pytest

from oracle import chordal_admm as orc
from sdp_inputs import CONFIGS, config_instance
from tests import sdp_cases
from tests.gpu_support import make_oracle, oracle_state_to_abi, rel_err, require_gpu, setup_handle

pytestmark = pytest.mark.gpu

SAMPLE = list(range(8))
RHO = CONFIGS[2]["rho"]


@pytest.fixture(scope="module")
def batch8():
    arrs = [sdp_cases.instance_arrays(config_instance(2, i)) for i in SAMPLE]
    sdps = [make_oracle(a) for a in arrs]
    return arrs, sdps


def step(form):
    return orc.primal_iteration if form == "primal" else orc.dual_iteration


def batch_handle(cadmm, arrs, form="dual", prec="fp64", rho=RHO, tol=1e-4, max_iter=2000):
    opts = cadmm.make_opts(rho=rho, tol=tol, max_iter=max_iter, form=form, prec=prec)
    return cadmm.ChordalADMM(list(arrs), opts)


def split_state(st: dict, lay: dict, q: int) -> dict:
    e0, e1 = lay["ent_off"][q], lay["ent_off"][q + 1]
    r0, r1 = lay["row_off"][q], lay["row_off"][q + 1]
    p0, p1 = lay["pos_off"][q], lay["pos_off"][q + 1]
    return dict(x=st["x"][e0:e1], y=st["y"][r0:r1], blk_a=st["blk_a"][p0:p1], blk_b=st["blk_b"][p0:p1],
                blk_c=st["blk_c"][p0:p1])


def compare_state(gpu, sdp, st, tol):
    ref = oracle_state_to_abi(sdp, st)
    for key in ref:
        err = rel_err(gpu[key], ref[key])
        assert err <= tol, (key, err)


def test_batch_layout_and_maps_are_concatenations(batch8):
    """Offsets, E_L and the gather map of the batch are the problems' own, shifted (bit-exact)."""
    torch, cadmm = require_gpu()
    arrs, sdps = batch8
    with batch_handle(cadmm, arrs) as s:
        lay = s.batch_layout()
        maps = cadmm.sdp_get_maps(s.h)
        sz = s.sizes
    assert sz["batch"] == len(arrs)
    ent = pos = row = vtx = cl = 0
    for q, a in enumerate(arrs):
        assert (lay["vtx_off"][q], lay["row_off"][q], lay["clique_off"][q]) == (vtx, row, cl)
        assert (lay["ent_off"][q], lay["pos_off"][q]) == (ent, pos)
        with setup_handle(cadmm, a) as s1:
            m1 = cadmm.sdp_get_maps(s1.h)
            z1 = s1.sizes
        e0, e1 = ent, ent + z1["nE_lower"]
        np.testing.assert_array_equal(maps["pat_row"][e0:e1], m1["pat_row"] + vtx)
        np.testing.assert_array_equal(maps["pat_col"][e0:e1], m1["pat_col"] + vtx)
        np.testing.assert_array_equal(maps["gather_idx"][pos:pos + z1["S_lower"]], m1["gather_idx"] + ent)
        ent, pos = e1, pos + z1["S_lower"]
        row, vtx, cl = row + z1["m"], vtx + z1["n"], cl + z1["p"]
    assert (lay["ent_off"][-1], lay["pos_off"][-1], lay["row_off"][-1]) == (sz["nE_lower"], sz["S_lower"], sz["m"])


@pytest.mark.parametrize("form", ["primal", "dual"])
def test_batch_first_iteration_matches_oracle(batch8, form):
    torch, cadmm = require_gpu()
    arrs, sdps = batch8
    with batch_handle(cadmm, arrs, form=form, tol=0.0) as s:
        r = s.iterate(1)
        assert r["iters"] == 1 and r["status"] == cadmm.SDP_MAX_ITER
        st, lay, res = s.state(), s.batch_layout(), s.batch_results()
    objs = []
    for q, sdp in enumerate(sdps):
        nxt = step(form)(sdp, orc.admm_init(sdp, form), RHO)
        compare_state(split_state(st, lay, q), sdp, nxt, 1e-10)
        for key in ("eps_p", "eps_d", "obj_primal", "obj_dual"):
            assert abs(res[key][q] - nxt[key]) <= 1e-9 * max(abs(nxt[key]), 1e-6), (q, key)
        assert res["iters"][q] == 1 and res["status"][q] == cadmm.SDP_MAX_ITER
        objs.append(nxt["obj_primal"])
    # the union's objective is the sum of the problems' objectives
    assert abs(r["obj_primal"] - sum(objs)) <= 1e-9 * sum(abs(o) for o in objs)


@pytest.mark.parametrize("form", ["primal", "dual"])
def test_batch_iteration_from_oracle_state(batch8, form):
    """Upload every problem's oracle iterate after 9 iterations, take one batched GPU iteration and
    compare each problem with the oracle's 10th."""
    torch, cadmm = require_gpu()
    arrs, sdps = batch8
    sts, nxts = [], []
    for sdp in sdps:
        st = orc.admm_init(sdp, form)
        for _ in range(9):
            st = step(form)(sdp, st, RHO)
        sts.append(st)
        nxts.append(step(form)(sdp, st, RHO))
    abi = [oracle_state_to_abi(sdp, st) for sdp, st in zip(sdps, sts)]
    keys = abi[0].keys()
    cat = {k: np.concatenate([d[k] for d in abi]) for k in keys}
    with batch_handle(cadmm, arrs, form=form, tol=0.0) as s:
        cadmm.sdp_set_state(s.h, **cat)
        s.iterate(1)
        st, lay, res = s.state(), s.batch_layout(), s.batch_results()
    for q, sdp in enumerate(sdps):
        compare_state(split_state(st, lay, q), sdp, nxts[q], 1e-10)
        assert abs(res["eps_p"][q] - nxts[q]["eps_p"]) <= 1e-8 * nxts[q]["eps_p"] + 1e-12
        assert abs(res["eps_d"][q] - nxts[q]["eps_d"]) <= 1e-8 * nxts[q]["eps_d"] + 1e-12


@pytest.mark.parametrize("form,rho", [("dual", RHO), ("primal", 1.0 / RHO)])
def test_batch_fp64_solve_per_problem(batch8, form, rho):
    """Each problem stops at its own iteration (within 1 of the oracle's) with the oracle's
    objective (1e-6), and its frozen state equals a separate GPU solve of it."""
    torch, cadmm = require_gpu()
    arrs, sdps = batch8
    with batch_handle(cadmm, arrs, form=form, rho=rho, tol=1e-4, max_iter=3000) as s:
        r = s.solve()
        st, lay, res = s.state(), s.batch_layout(), s.batch_results()
    assert r["status"] == cadmm.SDP_OK
    assert r["iters"] == res["iters"].max()
    assert len(set(res["iters"].tolist())) > 1          # the problems stop at different iterations
    obj_key = "obj_primal" if form == "primal" else "obj_dual"
    for q, (a, sdp) in enumerate(zip(arrs, sdps)):
        ref = orc.admm_solve(sdp, form, rho=rho, tol=1e-4, max_iter=3000)
        assert res["status"][q] == cadmm.SDP_OK and ref["status"] == 0
        assert abs(int(res["iters"][q]) - ref["iters"]) <= 1, (q, res["iters"][q], ref["iters"])
        assert abs(res[obj_key][q] - ref[obj_key]) <= 1e-6 * abs(ref[obj_key]), q
        with setup_handle(cadmm, a, form=form, rho=rho, tol=1e-4, max_iter=3000) as s1:
            r1 = s1.solve()
            st1 = s1.state()
        if r1["iters"] == res["iters"][q]:
            mine = split_state(st, lay, q)
            for key in ("x", "y", "blk_a", "blk_b"):
                assert rel_err(mine[key], st1[key]) <= 1e-8, (q, key)


def test_batch_frozen_problems_stay_frozen(batch8):
    torch, cadmm = require_gpu()
    arrs, sdps = batch8
    with batch_handle(cadmm, arrs, form="dual", tol=1e-3) as s:
        r = s.solve()
        assert r["status"] == cadmm.SDP_OK
        st0, res0 = s.state(), s.batch_results()
        r2 = s.iterate(5)                       # every problem is frozen: nothing may change
        st1, res1 = s.state(), s.batch_results()
        assert r2["status"] == cadmm.SDP_OK
        for k in st0:
            np.testing.assert_array_equal(st0[k], st1[k])
        np.testing.assert_array_equal(res0["iters"], res1["iters"])
        s.set_opts(tol=1e-5)                     # new options unfreeze every problem
        s.iterate(3)
        st2, res2 = s.state(), s.batch_results()
        assert not np.array_equal(st2["blk_a"], st1["blk_a"])
        assert np.all(res2["status"] == cadmm.SDP_MAX_ITER)


def test_batch_nan_stays_in_its_problem(batch8):
    """A NaN planted in one problem's data stops that problem with SDP_ERR_NAN at its first
    iteration; the others still converge, and the call reports SDP_ERR_NAN."""
    torch, cadmm = require_gpu()
    arrs, sdps = batch8
    bad = 3
    arrs = list(arrs)
    a = dict(arrs[bad])
    a["b"] = a["b"].copy()
    a["b"][0] = np.nan
    arrs[bad] = a
    with batch_handle(cadmm, arrs, form="dual", tol=1e-4) as s:
        with pytest.raises(cadmm.SDPError) as e:
            s.solve()
        assert e.value.code == cadmm.SDP_ERR_NAN
        res = s.batch_results()
    assert res["status"][bad] == cadmm.SDP_ERR_NAN and res["iters"][bad] == 1
    others = [q for q in range(len(arrs)) if q != bad]
    assert np.all(res["status"][others] == cadmm.SDP_OK)


def test_batch_full_workload_fp32(capsys):
    """All 512 problems in FP32-projection mode: every one converges; sampled problems match the
    FP64 oracle's objective within 1e-4."""
    torch, cadmm = require_gpu()
    cfg = CONFIGS[2]
    arrs = [sdp_cases.instance_arrays(config_instance(2, i)) for i in range(cfg["count"])]
    with batch_handle(cadmm, arrs, form=cfg["form"], prec="fp32", rho=cfg["rho"], tol=cfg["tol"],
                      max_iter=cfg["max_iter"]) as s:
        r = s.solve()
        res = s.batch_results()
    assert r["status"] == cadmm.SDP_OK
    assert np.all(res["status"] == cadmm.SDP_OK)
    assert r["iters"] == res["iters"].max()
    with capsys.disabled():
        print(f"\nbatch of {cfg['count']}: {r['iters']} iterations, {r['seconds'] * 1e3:.1f} ms, "
              f"per-problem iterations {res['iters'].min()}..{res['iters'].max()}")
    rng = np.random.default_rng(5)
    for q in sorted(rng.choice(cfg["count"], size=4, replace=False)):
        sdp = make_oracle(arrs[q])
        ref = orc.admm_solve(sdp, "dual", rho=cfg["rho"], tol=cfg["tol"], max_iter=cfg["max_iter"])
        assert abs(res["obj_dual"][q] - ref["obj_dual"]) <= 1e-4 * abs(ref["obj_dual"]), q
        assert abs(res["obj_primal"][q] - ref["obj_primal"]) <= 1e-4 * abs(ref["obj_primal"]), q
