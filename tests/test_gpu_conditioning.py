"""The affine step (Section III.B.1, block elimination with the cached factor of A D⁻¹ Aᵀ) on
ill-conditioned constraints: two nearly dependent rows of A make κ(A D⁻¹ Aᵀ) about 2e6 and 2e8.

Forming M = A D⁻¹ Aᵀ in FP64 already limits the affine iterate x to about κ(M)·ε: against an
extended-precision solve of the same first step, the oracle (triangular substitutions with the
Cholesky factor), an explicit M⁻¹ and the two triangular factors are equally far off (about
1.5e-10 relative at κ = 2e6, 9e-9 at κ = 2e8), because all start from M rounded to FP64. Where
they differ is the constraint residual: the explicit M⁻¹ leaves A x − b at about κ·ε, the
factors (like substitution) at about ε. Above κ₁ = 1e5 the GPU therefore takes the factors, and
these cases check that it does. Its iterates are held to the extended-precision reference: its first-step x no further from the extended-precision one than the oracle's
(plus rounding), and its iterates (x, the clique blocks, the multipliers, and Aᵀy rather than y,
whose component along the near-null direction of Aᵀ is fixed only to κ·ε) within a κ-scaled bound
of the oracle's. The converged objectives and the feasibility of x keep the well-conditioned bars
(1e-6 and 1e-10).
"""

import numpy as np
import pytest

from oracle import chordal_admm as orc
from tests import sdp_cases
from tests.gpu_support import make_oracle, oracle_state_to_abi, rel_err, require_gpu, setup_handle

pytestmark = pytest.mark.gpu


def step(form):
    return orc.primal_iteration if form == "primal" else orc.dual_iteration


def extended_first_affine_step(sdp, form, rho):
    """x and y of the first iteration from zero iterates, in extended precision (np.longdouble).
    From zero, r is exact: −c/ρ (primal form) or c (dual form; z_1 = P(0) = 0)."""
    ld = np.longdouble
    A = sdp.A.toarray().astype(ld)
    D = sdp.D.astype(ld)
    c = sdp.c.astype(ld)
    b = sdp.b.astype(ld)
    r = -c / ld(rho) if form == "primal" else c
    rhs2 = b if form == "primal" else -b / ld(rho)
    M = (A / D) @ A.T
    t = A @ (r / D) - rhs2
    m = M.shape[0]
    L = np.zeros_like(M)
    for j in range(m):
        L[j, j] = np.sqrt(M[j, j] - np.sum(L[j, :j] ** 2))
        for i in range(j + 1, m):
            L[i, j] = (M[i, j] - np.sum(L[i, :j] * L[j, :j])) / L[j, j]
    z = np.zeros(m, ld)
    for i in range(m):
        z[i] = (t[i] - np.sum(L[i, :i] * z[:i])) / L[i, i]
    y = np.zeros(m, ld)
    for i in reversed(range(m)):
        y[i] = (z[i] - np.sum(L[i + 1:, i] * y[i + 1:])) / L[i, i]
    x = (r - A.T @ y) / D
    return x, y


@pytest.mark.parametrize("form", ["primal", "dual"])
@pytest.mark.parametrize("delta", [1e-3, 1e-4])
def test_ill_conditioned_iterations_match_oracle(delta, form):
    torch, cadmm = require_gpu()
    arrs = sdp_cases.near_dependent_block_arrow(delta=delta)
    sdp = make_oracle(arrs)
    kappa = float(np.linalg.cond(sdp.M))
    assert 1e6 <= kappa <= 1e9
    rho = 1.0
    x_ext, _ = extended_first_affine_step(sdp, form, rho)
    x_ext_lower = sdp.to_lower(x_ext)
    scale = float(np.max(np.abs(x_ext_lower)))
    st = orc.admm_init(sdp, form)
    with setup_handle(cadmm, arrs, form=form, rho=rho, tol=0.0) as s:
        names = [cadmm.sdp_phase_name(s.h, i) for i in range(8)]
        assert "tri_lower" in names and "tri_upper" in names and "solve_y" not in names, names
        for it in range(30):
            st = step(form)(sdp, st, rho)
            s.iterate(1)
            gpu = s.state()
            if it == 0:
                e_gpu = float(np.max(np.abs(gpu["x"] - x_ext_lower))) / scale
                e_orc = float(np.max(np.abs(sdp.to_lower(st["x"]) - x_ext_lower))) / scale
                assert e_orc <= kappa * 1e-15 and e_gpu <= 3.0 * e_orc + 1e-13, (e_gpu, e_orc)
            ref = oracle_state_to_abi(sdp, st)
            bound = max(1e-9, kappa * 5e-16)
            for key in ref:
                if key == "y":
                    # y is determined only to about kappa eps along the near-null direction of
                    # A^T, which x never sees: compare A^T y, the part the iteration uses
                    err = rel_err(sdp.A.T @ gpu["y"], sdp.A.T @ ref["y"])
                else:
                    err = rel_err(gpu[key], ref[key])
                assert err <= bound, (it, key, err, bound)
        # the constraint residual of the affine iterate: A x = b (primal) or -b/rho (dual)
        rows, cols = sdp.E_row[sdp.lower_mask()], sdp.E_col[sdp.lower_mask()]
        x = sdp.from_lower(rows, cols, s.state()["x"])
        rhs = sdp.b if form == "primal" else -sdp.b / rho
        assert np.max(np.abs(sdp.A @ x - rhs)) <= 1e-10 * max(1.0, np.max(np.abs(rhs)))


@pytest.mark.parametrize("form", ["primal", "dual"])
@pytest.mark.parametrize("delta", [1e-3, 1e-4])
def test_ill_conditioned_solve_matches_oracle(delta, form):
    torch, cadmm = require_gpu()
    arrs = sdp_cases.near_dependent_block_arrow(delta=delta)
    sdp = make_oracle(arrs)
    rho = 1.0
    ref = orc.admm_solve(sdp, form, rho=rho, tol=1e-6, max_iter=20000)
    assert ref["status"] == 0
    with setup_handle(cadmm, arrs, form=form, rho=rho, tol=1e-6, max_iter=20000) as s:
        r = s.solve()
    assert r["status"] == cadmm.SDP_OK
    assert abs(r["iters"] - ref["iters"]) <= 1, (r["iters"], ref["iters"])
    key = "obj_primal" if form == "primal" else "obj_dual"
    assert abs(r[key] - ref[key]) <= 1e-6 * abs(ref[key]), (r[key], ref[key])


def test_well_conditioned_problem_keeps_explicit_inverse():
    torch, cadmm = require_gpu()
    arrs = sdp_cases.near_dependent_block_arrow(delta=0.3)
    assert np.linalg.cond(make_oracle(arrs).M) < 1e3
    with setup_handle(cadmm, arrs, form="dual", rho=1.0, tol=0.0) as s:
        names = [cadmm.sdp_phase_name(s.h, i) for i in range(8)]
    assert "solve_y" in names and "tri_lower" not in names, names
