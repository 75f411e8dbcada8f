"""GPU parity of single ADMM iterations (Algorithms 1 and 2, FP64) against the oracle: 1e-10."""

import numpy as np
import pytest

from oracle import chordal_admm as orc
from sdp_inputs import config_instance
from tests import sdp_cases
from tests.gpu_support import make_oracle, oracle_state_to_abi, rel_err, require_gpu, setup_handle
from tests.test_gpu_maps import chain_case

pytestmark = pytest.mark.gpu

TOL = 1e-10

CASES = {
    "config0": (lambda: sdp_cases.instance_arrays(config_instance(0)), 1.0),
    "chain_ragged": (chain_case, 0.7),
    "heavy_overlap": (lambda: sdp_cases.random_block_arrow(l=40, d=1, h=4, m=6, seed=3), 2.0),
}


def compare_state(gpu, sdp, st, tol=TOL):
    ref = oracle_state_to_abi(sdp, st)
    for key in ref:
        err = rel_err(gpu[key], ref[key])
        assert err <= tol, (key, err)


def step(form):
    return orc.primal_iteration if form == "primal" else orc.dual_iteration


@pytest.mark.parametrize("form", ["primal", "dual"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_first_iteration_matches_oracle(name, form):
    torch, cadmm = require_gpu()
    make, rho = CASES[name]
    arrs = make()
    sdp = make_oracle(arrs)
    with setup_handle(cadmm, arrs, form=form, rho=rho, tol=0.0) as s:
        r = s.iterate(1)
        assert r["iters"] == 1 and r["status"] == cadmm.SDP_MAX_ITER
        st = step(form)(sdp, orc.admm_init(sdp, form), rho)
        compare_state(s.state(), sdp, st)
        for key, okey in (("eps_p", "eps_p"), ("eps_d", "eps_d"), ("obj_primal", "obj_primal"),
                          ("obj_dual", "obj_dual")):
            assert abs(r[key] - st[okey]) <= 1e-9 * max(abs(st[okey]), 1e-6), (key, r[key], st[okey])


@pytest.mark.parametrize("form", ["primal", "dual"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_iteration_from_oracle_state(name, form):
    """Load the oracle's iterate after 9 iterations, take one GPU iteration, compare with the
    oracle's 10th."""
    torch, cadmm = require_gpu()
    make, rho = CASES[name]
    arrs = make()
    sdp = make_oracle(arrs)
    st = orc.admm_init(sdp, form)
    for _ in range(9):
        st = step(form)(sdp, st, rho)
    nxt = step(form)(sdp, st, rho)
    with setup_handle(cadmm, arrs, form=form, rho=rho, tol=0.0) as s:
        cadmm.sdp_set_state(s.h, **oracle_state_to_abi(sdp, st))
        r = s.iterate(1)
        compare_state(s.state(), sdp, nxt)
        # residuals are ratios of norms; near rounding level only an absolute bound is meaningful
        assert abs(r["eps_p"] - nxt["eps_p"]) <= 1e-8 * nxt["eps_p"] + 1e-12
        assert abs(r["eps_d"] - nxt["eps_d"]) <= 1e-8 * nxt["eps_d"] + 1e-12


@pytest.mark.parametrize("form", ["primal", "dual"])
def test_thirty_iterations_track_oracle(form):
    torch, cadmm = require_gpu()
    arrs = sdp_cases.instance_arrays(config_instance(0))
    sdp = make_oracle(arrs)
    st = orc.admm_init(sdp, form)
    for _ in range(30):
        st = step(form)(sdp, st, 1.0)
    with setup_handle(cadmm, arrs, form=form, rho=1.0, tol=0.0, check_every=8) as s:
        r = s.iterate(30)
        assert r["iters"] == 30
        compare_state(s.state(), sdp, st, tol=1e-9)


@pytest.mark.parametrize("name,rho", [("small", 0.7), ("config1", 0.02), ("cones", 0.5)])
def test_primal_multipliers_reproduce_dual_blocks(name, rho):
    """Section IV's primal/dual correspondence on the GPU (the derivation and its CPU pin are in
    tests/test_oracle_scaling.py): the primal form at penalty 1/ρ, started from the state matched
    to the dual form's iterates 0..2 at penalty ρ, returns the dual form's z_k as its λ_k and
    ρ(x'_{k−2} − 2x'_{k−1}) as its x at every later iteration."""
    torch, cadmm = require_gpu()
    if name == "small":
        arrs = sdp_cases.random_block_arrow(l=3, d=3, h=2, m=5, seed=4)
    elif name == "config1":
        arrs = sdp_cases.instance_arrays(config_instance(1))
    else:
        arrs = sdp_cases.random_conic(l=2, d=3, h=2, n_free=2, n_lin=4, soc_dims=(3, 1, 40), m=6, seed=21)
    K = 12
    with setup_handle(cadmm, arrs, form="dual", rho=rho, tol=0.0) as d:
        xs, zs = [np.zeros(d.sizes["nE_lower"])], [np.zeros(d.sizes["S_lower"])]
        for _ in range(K):
            d.iterate(1)
            st = d.state()
            xs.append(st["x"])
            zs.append(st["blk_a"])
        gidx = cadmm.sdp_get_maps(d.h)["gather_idx"]
    with setup_handle(cadmm, arrs, form="primal", rho=1.0 / rho, tol=0.0) as p:
        x = rho * (xs[0] - 2.0 * xs[1])
        cadmm.sdp_set_state(p.h, x=x, y=np.zeros(len(arrs["b"])), blk_a=x[gidx] + rho * (zs[2] - zs[1]),
                            blk_b=zs[2])
        g_lam = g_x = 0.0
        for k in range(3, K + 1):
            p.iterate(1)
            st = p.state()
            g_lam = max(g_lam, float(np.max(np.abs(st["blk_b"] - zs[k])) / max(np.max(np.abs(zs[k])), 1.0)))
            xr = rho * (xs[k - 2] - 2.0 * xs[k - 1])
            g_x = max(g_x, float(np.max(np.abs(st["x"] - xr)) / max(np.max(np.abs(xr)), 1.0)))
    assert g_lam <= 1e-9 and g_x <= 1e-9, (g_lam, g_x)
