"""GPU parity of the non-PSD cone blocks (free, nonnegative, second-order; Section V's product
cones, not decomposed) against the oracle, through sdp_setup_conic: single FP64 iterations within
1e-10, converged FP64 solves within 1e-6 and ±1 iteration, FP32-projection solves within 1e-4,
problems without a PSD part, and cone segments longer than one CTA's threads."""

import numpy as np
import pytest

from oracle import chordal_admm as orc
from tests import sdp_cases
from tests.gpu_support import make_oracle, oracle_state_to_abi, rel_err, require_gpu, setup_handle

pytestmark = pytest.mark.gpu


def step(form):
    return orc.primal_iteration if form == "primal" else orc.dual_iteration


def compare_state(gpu, sdp, st, tol):
    ref = oracle_state_to_abi(sdp, st)
    for key in ref:
        err = rel_err(gpu[key], ref[key])
        assert err <= tol, (key, err)


def mixed():
    return sdp_cases.random_conic(l=2, d=3, h=2, n_free=3, n_lin=5, soc_dims=(3, 4, 1), m=6, seed=21)


def pure_cones():
    return sdp_cases.random_conic(l=0, n_free=2, n_lin=7, soc_dims=(4, 2), m=5, seed=22)


def long_segments():
    # the nonnegative block spans three segments and one second-order cone has 3000 variables
    return sdp_cases.random_conic(l=3, d=2, h=2, n_free=300, n_lin=9000, soc_dims=(3000, 5, 1), m=12,
                                  seed=23, density=0.05)


CASES = {"mixed": mixed, "pure_cones": pure_cones, "long_segments": long_segments}


@pytest.mark.parametrize("form", ["primal", "dual"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_iterations_match_oracle(name, form):
    torch, cadmm = require_gpu()
    arrs = CASES[name]()
    sdp = make_oracle(arrs)
    rho = 0.8
    st = orc.admm_init(sdp, form)
    with setup_handle(cadmm, arrs, form=form, rho=rho, tol=0.0) as s:
        assert s.sizes["n_cone"] == sdp.n_cone
        assert s.sizes["nE_lower"] == int(sdp.lower_mask().sum())
        for it in range(1, 13):
            r = s.iterate(1)
            st = step(form)(sdp, st, rho)
            if it in (1, 12):
                compare_state(s.state(), sdp, st, 1e-10 if it == 1 else 1e-9)
                assert abs(r["eps_p"] - st["eps_p"]) <= 1e-8 * st["eps_p"] + 1e-12
                assert abs(r["eps_d"] - st["eps_d"]) <= 1e-8 * st["eps_d"] + 1e-12
        # load the oracle's state and take one more iteration on both sides
        cadmm.sdp_set_state(s.h, **oracle_state_to_abi(sdp, st))
        s.iterate(1)
        st = step(form)(sdp, st, rho)
        compare_state(s.state(), sdp, st, 1e-10)
        if form == "dual" and arrs["cones"]["n_free"]:
            z = s.state()["blk_a"]
            p_len = sum(len(c) * (len(c) + 1) // 2 for c in sdp.cliques)
            assert np.all(z[p_len:p_len + arrs["cones"]["n_free"]] == 0.0)   # dual cone of ℝⁿ is {0}


@pytest.mark.parametrize("form", ["primal", "dual"])
@pytest.mark.parametrize("name", ["mixed", "pure_cones"])
def test_fp64_solve_matches_oracle(name, form):
    torch, cadmm = require_gpu()
    arrs = CASES[name]()
    sdp = make_oracle(arrs)
    ref = orc.admm_solve(sdp, form, rho=1.0, tol=1e-6, max_iter=20000)
    with setup_handle(cadmm, arrs, form=form, rho=1.0, tol=1e-6, max_iter=20000) as s:
        r = s.solve()
    key = "obj_primal" if form == "primal" else "obj_dual"
    assert r["status"] == cadmm.SDP_OK and ref["status"] == 0
    assert abs(r["iters"] - ref["iters"]) <= 1, (r["iters"], ref["iters"])
    assert abs(r[key] - ref[key]) <= 1e-6 * max(1.0, abs(ref[key]))


@pytest.mark.parametrize("form", ["primal", "dual"])
def test_fp32_projection_solve(form):
    torch, cadmm = require_gpu()
    arrs = mixed()
    sdp = make_oracle(arrs)
    ref = orc.admm_solve(sdp, form, rho=1.0, tol=1e-4, max_iter=20000)
    with setup_handle(cadmm, arrs, form=form, prec="fp32", rho=1.0, tol=1e-4, max_iter=20000) as s:
        r = s.solve()
    key = "obj_primal" if form == "primal" else "obj_dual"
    assert r["status"] == cadmm.SDP_OK
    assert abs(r[key] - ref[key]) <= 1e-4 * max(1.0, abs(ref[key]))


def test_lp_as_cone_equals_lp_as_diagonal_sdp():
    """The same LP through a nonnegative block and through 1 x 1 PSD cliques: equal iterates."""
    torch, cadmm = require_gpu()
    rng = np.random.default_rng(31)
    m, nl = 8, 40
    Ac = rng.standard_normal((m, nl))
    b = Ac @ rng.uniform(0.5, 1.5, nl)
    c = Ac.T @ rng.standard_normal(m) + rng.uniform(0.5, 1.5, nl)
    cone = sdp_cases._empty_matrix_part()
    cone.update(A_ptr=np.zeros(m + 1, np.int64), b=b, cones=sdp_cases.cones_from_dense(Ac, c, n_lin=nl))
    diag = sdp_cases.lp_as_diagonal_sdp(Ac, b, c)
    out = []
    for arrs in (cone, diag):
        with setup_handle(cadmm, arrs, form="dual", rho=0.5, tol=1e-7, max_iter=20000) as s:
            r = s.solve()
            out.append((r, s.state()["x"]))
    assert out[0][0]["iters"] == out[1][0]["iters"]
    assert abs(out[0][0]["obj_dual"] - out[1][0]["obj_dual"]) <= 1e-10 * abs(out[1][0]["obj_dual"])
    np.testing.assert_allclose(out[0][1], out[1][1], rtol=0, atol=1e-12 * np.abs(out[1][1]).max())
