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
