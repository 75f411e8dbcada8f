"""GPU whole-solve parity (converged objective, iteration count) and the solver's edge cases."""

import numpy as np
import pytest

from oracle import chordal_admm as orc
from sdp_inputs import CONFIGS, config_instance
from tests import sdp_cases
from tests.gpu_support import make_oracle, rel_err, require_gpu, setup_handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfg0():
    arrs = sdp_cases.instance_arrays(config_instance(0))
    sdp = make_oracle(arrs)
    ref = {f: orc.admm_solve(sdp, f, rho=1.0, tol=1e-4, max_iter=2000) for f in ("primal", "dual")}
    return arrs, sdp, ref


@pytest.fixture(scope="module")
def cfg1():
    cfg = CONFIGS[1]
    arrs = sdp_cases.instance_arrays(config_instance(1))
    sdp = make_oracle(arrs)
    ref = orc.admm_solve(sdp, "dual", rho=cfg["rho"], tol=cfg["tol"], max_iter=cfg["max_iter"])
    return arrs, sdp, ref


def objective(r, form):
    return r["obj_primal"] if form == "primal" else r["obj_dual"]


@pytest.mark.parametrize("form", ["primal", "dual"])
def test_config0_fp64_converges_like_oracle(cfg0, form):
    torch, cadmm = require_gpu()
    arrs, sdp, ref = cfg0
    with setup_handle(cadmm, arrs, form=form, rho=1.0, tol=1e-4, max_iter=2000) as s:
        r = s.solve()
    assert r["status"] == cadmm.SDP_OK and ref[form]["status"] == 0
    assert abs(r["iters"] - ref[form]["iters"]) <= 1
    o, oref = objective(r, form), objective(ref[form], form)
    assert abs(o - oref) <= 1e-6 * abs(oref)
    assert max(r["eps_p"], r["eps_d"]) < 1e-4


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-6), ("fp32", 1e-4)])
def test_config1_dual_converges_like_oracle(cfg1, prec, tol):
    torch, cadmm = require_gpu()
    arrs, sdp, ref = cfg1
    cfg = CONFIGS[1]
    with setup_handle(cadmm, arrs, form="dual", prec=prec, rho=cfg["rho"], tol=cfg["tol"],
                      max_iter=cfg["max_iter"]) as s:
        r = s.solve()
        X, y, Z = s.solution()
    assert r["status"] == cadmm.SDP_OK and ref["status"] == 0
    if prec == "fp64":
        assert abs(r["iters"] - ref["iters"]) <= 1
    assert abs(r["obj_dual"] - ref["obj_dual"]) <= tol * abs(ref["obj_dual"])
    assert abs(r["obj_primal"] - ref["obj_primal"]) <= tol * abs(ref["obj_primal"])
    # the dual estimate y solves A*y + Z = C with Z = Σ H_kᵀ z_k; X = -ρx satisfies A X = b
    lower = sdp.lower_mask()
    Xf = sdp.from_lower(sdp.E_row[lower], sdp.E_col[lower], X)
    np.testing.assert_allclose(sdp.A @ Xf, sdp.b, atol=1e-8 * np.abs(sdp.b).max())
    Zf = sdp.from_lower(sdp.E_row[lower], sdp.E_col[lower], Z)
    res = sdp.A.T @ y + Zf - sdp.c
    assert np.linalg.norm(res) <= 1e-2 * np.linalg.norm(sdp.c)


def test_theta_c5_on_gpu():
    torch, cadmm = require_gpu()
    arrs, opt = sdp_cases.theta_c5()
    with setup_handle(cadmm, arrs, form="primal", rho=1.0, tol=1e-10, max_iter=20000) as s:
        r = s.solve()
    assert r["status"] == cadmm.SDP_OK
    assert abs(r["obj_primal"] - opt) <= 1e-7


@pytest.mark.parametrize("form", ["primal", "dual"])
def test_trace_one_lambda_min_on_gpu(form):
    torch, cadmm = require_gpu()
    arrs, lam_min = sdp_cases.trace_one_block_arrow(l=4, d=3, h=2)
    with setup_handle(cadmm, arrs, form=form, rho=1.0, tol=1e-9, max_iter=20000) as s:
        r = s.solve()
    assert r["status"] == cadmm.SDP_OK
    assert abs(objective(r, form) - lam_min) <= 1e-6 * max(1, abs(lam_min))


def test_iteration_cap_status():
    torch, cadmm = require_gpu()
    arrs = sdp_cases.instance_arrays(config_instance(0))
    with setup_handle(cadmm, arrs, form="primal", tol=1e-14, max_iter=5) as s:
        r = s.solve()
    assert r["status"] == cadmm.SDP_MAX_ITER and r["iters"] == 5


def test_nan_input_reports_status():
    torch, cadmm = require_gpu()
    arrs = sdp_cases.instance_arrays(config_instance(0))
    arrs["b"] = arrs["b"].copy()
    arrs["b"][3] = np.nan
    with setup_handle(cadmm, arrs, form="primal", tol=1e-4, max_iter=50) as s:
        with pytest.raises(cadmm.SDPError) as e:
            s.solve()
        assert e.value.code == cadmm.SDP_ERR_NAN
        assert s.state()["y"].shape == (arrs["b"].shape[0],)     # the context stays usable


@pytest.mark.parametrize("form", ["primal", "dual"])
def test_resume_and_determinism(form):
    torch, cadmm = require_gpu()
    arrs = sdp_cases.instance_arrays(config_instance(0))
    with setup_handle(cadmm, arrs, form=form, tol=0.0, check_every=16) as s:
        s.iterate(23)
        s.iterate(27)
        a = s.state()
        s.reset()
        s.iterate(50)
        b = s.state()
    with setup_handle(cadmm, arrs, form=form, tol=0.0, check_every=1) as s:
        s.iterate(50)
        c = s.state()
    for k in a:
        assert np.array_equal(a[k], b[k]), k
        assert np.array_equal(a[k], c[k]), k


def test_switching_form_and_rho():
    torch, cadmm = require_gpu()
    arrs = sdp_cases.instance_arrays(config_instance(0))
    sdp = make_oracle(arrs)
    with setup_handle(cadmm, arrs, form="dual", rho=0.5, tol=0.0) as s:
        s.iterate(3)
        s.set_opts(form="primal", rho=10.0, tol=1e-4, max_iter=2000)
        s.reset()
        r = s.solve()
    ref = orc.admm_solve(sdp, "primal", rho=10.0, tol=1e-4, max_iter=2000)
    assert abs(r["iters"] - ref["iters"]) <= 1
    assert abs(r["obj_primal"] - ref["obj_primal"]) <= 1e-6 * abs(ref["obj_primal"])


@pytest.mark.parametrize("name", ["m", "l", "d"])
def test_sweep_first_point_converges_like_oracle(name):
    """The first point of each of the paper's block-arrow sweeps (Section V.A) at its tolerance
    1e-3, dual form, FP64: iteration count within 1 and objective within 1e-6 of the oracle."""
    torch, cadmm = require_gpu()
    from sdp_inputs import SWEEP_MAX_ITER, SWEEP_TOL, sweep_instance
    inst = sweep_instance(name, 0)
    arrs = sdp_cases.instance_arrays(inst)
    sdp = make_oracle(arrs)
    ref = orc.admm_solve(sdp, "dual", rho=0.02, tol=SWEEP_TOL, max_iter=SWEEP_MAX_ITER)
    with setup_handle(cadmm, arrs, form="dual", prec="fp64", rho=0.02, tol=SWEEP_TOL, max_iter=SWEEP_MAX_ITER) as s:
        r = s.solve()
    assert r["status"] == ref["status"]
    assert abs(r["iters"] - ref["iters"]) <= 1
    assert abs(r["obj_dual"] - ref["obj_dual"]) <= 1e-6 * abs(ref["obj_dual"])


@pytest.mark.parametrize("form", ["primal", "dual"])
def test_non_chordal_pattern_via_chordal_extension(form):
    """sdp_setup with no cliques extends the aggregate pattern itself (Section II.A); the solve then
    follows the oracle run on the oracle's extension (the same cliques) and reaches the optimum of
    the single-clique (dense) problem."""
    torch, cadmm = require_gpu()
    from oracle import chordal as och
    arrs = sdp_cases.random_sparse_sdp(n=24, m=8, seed=5)
    rows = np.concatenate([arrs["A_row"], arrs["C_row"]])
    cols = np.concatenate([arrs["A_col"], arrs["C_col"]])
    cliques, fill = och.chordal_extension(arrs["n"], rows, cols)
    assert fill > 0                                    # the pattern was not chordal
    ext = dict(arrs, cliques=[np.array(c, np.int32) for c in cliques])
    sdp = make_oracle(ext)
    ref = orc.admm_solve(sdp, form, rho=1.0, tol=1e-6, max_iter=20000)
    dense = make_oracle(dict(arrs, cliques=[np.arange(arrs["n"], dtype=np.int32)]))
    ref_dense = orc.admm_solve(dense, form, rho=1.0, tol=1e-8, max_iter=50000)
    with setup_handle(cadmm, arrs, form=form, rho=1.0, tol=1e-6, max_iter=20000) as s:
        r = s.solve()
        assert s.sizes["p"] == len(cliques)
    key = "obj_primal" if form == "primal" else "obj_dual"
    assert r["status"] == cadmm.SDP_OK and ref["status"] == 0
    assert abs(r["iters"] - ref["iters"]) <= 1
    assert abs(r[key] - ref[key]) <= 1e-6 * abs(ref[key])
    assert abs(r[key] - ref_dense[key]) <= 1e-4 * abs(ref_dense[key])


def test_projection_sweep_diagnostic(cfg0):
    """sdp_proj_sweeps: per clique, the Jacobi sweeps of the last iteration (FP32 one-sided
    eigensolver: at least one sweep, at most its cap of 20)."""
    torch, cadmm = require_gpu()
    arrs, sdp, _ = cfg0
    with setup_handle(cadmm, arrs, form="dual", prec="fp32", rho=1.0, tol=0.0) as s:
        s.iterate(20)
        sw = cadmm.sdp_proj_sweeps(s.h)
    assert sw.shape == (sdp.p,)
    assert sw.min() >= 1 and sw.max() <= 20
