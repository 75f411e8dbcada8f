"""Pins of the oracle's non-PSD cone blocks (free, nonnegative, second-order), without a GPU.

Section V says CDCS accepts products of ℝⁿ, the nonnegative orthant, second-order cones and the PSD
cone, and decomposes only the PSD one. The oracle appends the other cones' variables to x as
blocks of their own (D = 1 on them). What fixes each part, independently of its own code:

* the second-order-cone projection: the spectral formula of the cone's Jordan algebra
  (w = λ₁e₁ + λ₂e₂ with λ = t ± ‖u‖, projection max(λ₁,0)e₁ + max(λ₂,0)e₂), a generic constrained
  minimiser (scipy SLSQP) on small cones, Moreau's decomposition for a self-dual cone, and a
  hand-worked point;
* nonnegative blocks: an LP written with a nonnegative block runs the same iterates as the same LP
  written as an SDP on a diagonal pattern with 1 x 1 cliques (a 1 x 1 PSD block is a nonnegative
  number);
* second-order blocks: the optimum equals that of the same problem as an SDP on arrow matrices
  ([[t, uᵀ], [u, tI]] ⪰ 0 iff ‖u‖ ≤ t); the closed form min t s.t. u = u₀ gives ‖u₀‖;
* free blocks: the optimum equals that of the same problem with f = f⁺ − f⁻, f± ≥ 0; in the dual
  form the free block's z stays 0 (its dual cone is {0});
* primal and dual forms reach the same optimum on a mixed problem (Remark 1).
Planted mistakes (a dropped 1/2 in the SOC projection, the identity as the free block's dual
projection) make these checks fail.
"""

import numpy as np
import pytest

from oracle import chordal_admm as orc
from tests import sdp_cases

scipy_optimize = pytest.importorskip("scipy.optimize")


def conic_oracle(arrs) -> orc.ChordalSDP:
    return orc.ChordalSDP(arrs["n"], arrs["cliques"], arrs["A_ptr"], arrs["A_row"], arrs["A_col"],
                          arrs["A_val"], arrs["b"], arrs["C_row"], arrs["C_col"], arrs["C_val"],
                          cones=arrs.get("cones"))


def in_soc(x, tol=1e-12):
    return np.linalg.norm(x[1:]) <= x[0] + tol * max(1.0, np.abs(x).max())


def soc_spectral(w):
    t, u = w[0], w[1:]
    nu = np.linalg.norm(u)
    dirn = u / nu if nu > 0 else np.eye(len(u))[0] if len(u) else u
    e1 = 0.5 * np.concatenate([[1.0], dirn])
    e2 = 0.5 * np.concatenate([[1.0], -dirn])
    return max(t + nu, 0.0) * e1 + max(t - nu, 0.0) * e2


def test_soc_projection_properties():
    rng = np.random.default_rng(3)
    for trial in range(300):
        q = int(rng.integers(1, 8))
        w = rng.standard_normal(q) * rng.uniform(0.1, 10)
        if trial % 3 == 0:
            w[0] = rng.uniform(-1, 1) * np.linalg.norm(w[1:])     # the interesting region
        P = orc.proj_soc(w)
        assert in_soc(P)
        np.testing.assert_allclose(orc.proj_soc(P), P, atol=1e-13)                 # idempotent
        np.testing.assert_allclose(P - orc.proj_soc(-w), w, atol=1e-12)            # Moreau (self-dual)
        assert abs(np.dot(P, P - w)) <= 1e-11 * max(1.0, np.dot(w, w))            # orthogonality
        np.testing.assert_allclose(P, soc_spectral(w), atol=1e-12)                 # Jordan spectral form


def test_soc_projection_is_the_nearest_point():
    rng = np.random.default_rng(4)
    for trial in range(12):
        q = int(rng.integers(2, 6))
        w = rng.standard_normal(q)
        w[0] = rng.uniform(-0.8, 0.8) * np.linalg.norm(w[1:])
        cons = [{"type": "ineq", "fun": lambda x: x[0] - np.sqrt(np.dot(x[1:], x[1:]) + 1e-30)}]
        res = scipy_optimize.minimize(lambda x: np.sum((x - w) ** 2), x0=np.r_[np.linalg.norm(w) + 1, w[1:]],
                                      constraints=cons, method="SLSQP", options={"ftol": 1e-14, "maxiter": 500})
        np.testing.assert_allclose(orc.proj_soc(w), res.x, atol=1e-5)


def test_soc_projection_special_cases():
    np.testing.assert_array_equal(orc.proj_soc(np.array([5.0, 3.0, 4.0])), [5.0, 3.0, 4.0])   # inside
    np.testing.assert_array_equal(orc.proj_soc(np.array([-5.0, 3.0, 4.0])), [0.0, 0.0, 0.0])  # polar
    # hand-worked: (0, 3, 4) has ‖u‖ = 5, so a = (0 + 5)/2 and the point is a (1, 3/5, 4/5)
    np.testing.assert_allclose(orc.proj_soc(np.array([0.0, 3.0, 4.0])), [2.5, 1.5, 2.0], atol=1e-15)
    np.testing.assert_array_equal(orc.proj_soc(np.array([-2.0])), [0.0])                      # Q¹ = ℝ₊
    np.testing.assert_array_equal(orc.proj_soc(np.array([2.0])), [2.0])
    w = np.array([1.0, -2.0])
    np.testing.assert_allclose(orc.proj_cone("nonneg", w, False), [1.0, 0.0])
    np.testing.assert_array_equal(orc.proj_cone("free", w, False), w)
    np.testing.assert_array_equal(orc.proj_cone("free", w, True), [0.0, 0.0])


def random_lp(seed, m=4, nl=9):
    rng = np.random.default_rng(seed)
    Ac = rng.standard_normal((m, nl))
    x0 = rng.uniform(0.5, 1.5, nl)
    z0 = rng.uniform(0.5, 1.5, nl)
    y0 = rng.standard_normal(m)
    return Ac, Ac @ x0, Ac.T @ y0 + z0


@pytest.mark.parametrize("form", ["primal", "dual"])
def test_nonneg_block_runs_the_diagonal_sdp_iterates(form):
    Ac, b, c = random_lp(7)
    as_cone = sdp_cases._empty_matrix_part()
    as_cone.update(A_ptr=np.zeros(len(b) + 1, np.int64), b=b,
                   cones=sdp_cases.cones_from_dense(Ac, c, n_lin=Ac.shape[1]))
    cone = conic_oracle(as_cone)
    diag = conic_oracle(sdp_cases.lp_as_diagonal_sdp(Ac, b, c))
    assert cone.nblk == 1 and diag.nblk == Ac.shape[1]
    sa, sb = orc.admm_init(cone, form), orc.admm_init(diag, form)
    step = orc.primal_iteration if form == "primal" else orc.dual_iteration
    for _ in range(40):
        sa, sb = step(cone, sa, 0.7), step(diag, sb, 0.7)
        np.testing.assert_allclose(sa["x"], sb["x"], rtol=0, atol=1e-12 * max(1, np.abs(sb["x"]).max()))
        np.testing.assert_allclose(sa["y"], sb["y"], rtol=0, atol=1e-12 * max(1, np.abs(sb["y"]).max()))
        assert abs(sa["eps_p"] - sb["eps_p"]) <= 1e-12 and abs(sa["eps_d"] - sb["eps_d"]) <= 1e-12


@pytest.mark.parametrize("form", ["primal", "dual"])
def test_soc_blocks_match_the_arrow_sdp_optimum(form):
    rng = np.random.default_rng(8)
    m, nl, qd = 4, 2, [3, 4]
    nc = nl + sum(qd)
    Ac = rng.standard_normal((m, nc))
    x0, z0 = np.empty(nc), np.empty(nc)
    x0[:nl], z0[:nl] = rng.uniform(0.5, 1.5, nl), rng.uniform(0.5, 1.5, nl)
    o = nl
    for q in qd:
        for v in (x0, z0):
            u = 0.4 * rng.standard_normal(q - 1)
            v[o], v[o + 1:o + q] = np.linalg.norm(u) + 0.7, u
        o += q
    b, c = Ac @ x0, Ac.T @ rng.standard_normal(m) + z0
    as_cone = sdp_cases._empty_matrix_part()
    as_cone.update(A_ptr=np.zeros(m + 1, np.int64), b=b,
                   cones=sdp_cases.cones_from_dense(Ac, c, n_lin=nl, soc_dims=qd))
    r1 = orc.admm_solve(conic_oracle(as_cone), form, rho=1.0, tol=1e-9, max_iter=40000)
    r2 = orc.admm_solve(conic_oracle(sdp_cases.socp_as_arrow_sdp(Ac, b, c, nl, qd)), form, rho=1.0,
                        tol=1e-9, max_iter=40000)
    assert r1["status"] == 0 and r2["status"] == 0
    key = "obj_primal" if form == "primal" else "obj_dual"
    assert abs(r1[key] - r2[key]) <= 1e-6 * max(1.0, abs(r2[key]))
    if form == "primal":
        o = r1["x"][nl:]
        for q in qd:
            assert in_soc(o[:q], 1e-6)
            o = o[q:]


@pytest.mark.parametrize("form", ["primal", "dual"])
def test_soc_closed_form_norm(form):
    u0 = np.array([0.3, -1.2, 2.0])
    q = len(u0) + 1
    Ac = np.zeros((q - 1, q))
    Ac[np.arange(q - 1), np.arange(1, q)] = 1.0          # u = u0
    c = np.zeros(q)
    c[0] = 1.0                                           # min t
    arrs = sdp_cases._empty_matrix_part()
    arrs.update(A_ptr=np.zeros(q, np.int64), b=u0, cones=sdp_cases.cones_from_dense(Ac, c, soc_dims=[q]))
    r = orc.admm_solve(conic_oracle(arrs), form, rho=1.0, tol=1e-10, max_iter=20000)
    key = "obj_primal" if form == "primal" else "obj_dual"
    assert r["status"] == 0
    assert abs(r[key] - np.linalg.norm(u0)) <= 1e-7


def free_and_split(seed=9, m=4, nf=3, nl=6):
    rng = np.random.default_rng(seed)
    Af, Al = rng.standard_normal((m, nf)), rng.standard_normal((m, nl))
    f0, w0 = rng.standard_normal(nf), rng.uniform(0.5, 1.5, nl)
    y0 = rng.standard_normal(m)
    cf, cl = Af.T @ y0, Al.T @ y0 + rng.uniform(0.5, 1.5, nl)
    b = Af @ f0 + Al @ w0
    free = sdp_cases._empty_matrix_part()
    free.update(A_ptr=np.zeros(m + 1, np.int64), b=b,
                cones=sdp_cases.cones_from_dense(np.hstack([Af, Al]), np.r_[cf, cl], n_free=nf, n_lin=nl))
    split = sdp_cases._empty_matrix_part()
    split.update(A_ptr=np.zeros(m + 1, np.int64), b=b,
                 cones=sdp_cases.cones_from_dense(np.hstack([Af, -Af, Al]), np.r_[cf, -cf, cl], n_lin=2 * nf + nl))
    return free, split


@pytest.mark.parametrize("form", ["primal", "dual"])
def test_free_block_matches_the_split_problem(form):
    free, split = free_and_split()
    r1 = orc.admm_solve(conic_oracle(free), form, rho=1.0, tol=1e-9, max_iter=40000)
    r2 = orc.admm_solve(conic_oracle(split), form, rho=1.0, tol=1e-9, max_iter=40000)
    assert r1["status"] == 0 and r2["status"] == 0
    key = "obj_primal" if form == "primal" else "obj_dual"
    assert abs(r1[key] - r2[key]) <= 1e-6 * max(1.0, abs(r2[key]))
    if form == "dual":
        assert np.all(r1["zk"][0] == 0.0)                # the dual cone of ℝⁿ is {0}


def test_mixed_problem_primal_equals_dual():
    arrs = sdp_cases.random_conic(l=2, d=3, h=2, n_free=2, n_lin=4, soc_dims=(3, 2), m=6, seed=21)
    sdp = conic_oracle(arrs)
    assert sdp.kinds == ["psd", "psd", "free", "nonneg", "soc", "soc"]
    rp = orc.admm_solve(sdp, "primal", rho=1.0, tol=1e-9, max_iter=40000)
    rd = orc.admm_solve(sdp, "dual", rho=1.0, tol=1e-9, max_iter=40000)
    assert rp["status"] == 0 and rd["status"] == 0
    assert abs(rp["obj_primal"] - rd["obj_dual"]) <= 1e-6 * max(1.0, abs(rd["obj_dual"]))


def test_planted_half_in_soc_projection_is_caught(monkeypatch):
    def wrong(w):
        t, u = float(w[0]), np.asarray(w[1:])
        nu = float(np.linalg.norm(u))
        if nu <= t:
            return np.array(w, float)
        if nu <= -t:
            return np.zeros(len(w))
        a = t + nu                                         # the 1/2 dropped
        return np.concatenate([[a], (a / nu) * u])
    monkeypatch.setattr(orc, "proj_soc", wrong)
    with pytest.raises(AssertionError):
        test_soc_projection_properties()


def test_planted_identity_as_free_dual_projection_is_caught(monkeypatch):
    orig = orc.proj_cone

    def wrong(kind, w, dual):
        return np.array(w, float) if kind == "free" else orig(kind, w, dual)
    monkeypatch.setattr(orc, "proj_cone", wrong)
    with pytest.raises(AssertionError):
        test_free_block_matches_the_split_problem("dual")


def test_conic_extension_keeps_both_points_feasible():
    """The conic workload's inputs: (X0, x0) satisfies the new constraints, x0 lies inside its
    cones, and c_cone − A_coneᵀ y0 = z0 lies inside the dual cones (0 on the free variables)."""
    from sdp_inputs import config_instance, conic_extension
    inst = config_instance(0)
    qd = [3, 1, 5]
    ext = conic_extension(inst, 2, 4, qd, 2, 11)
    cn = ext["cones"]
    m, nc = len(inst.b), 2 + 4 + sum(qd)
    Ac = np.zeros((m, nc))
    for i in range(m):
        for t in range(cn["A_ptr"][i], cn["A_ptr"][i + 1]):
            Ac[i, cn["A_var"][t]] += cn["A_val"][t]
    assert np.all((Ac != 0).sum(axis=0) == 2)                       # two constraints per variable
    np.testing.assert_allclose(ext["b"] - inst.b, Ac @ ext["x0"], rtol=0, atol=1e-12)
    z = cn["c"] - Ac.T @ inst.y0
    np.testing.assert_allclose(z, ext["z0"], rtol=0, atol=1e-12)
    assert np.all(z[:2] == 0.0) and np.all(z[2:6] > 0) and np.all(ext["x0"][2:6] > 0)
    o = 6
    for q in qd:
        for v in (ext["x0"], z):
            assert np.linalg.norm(v[o + 1:o + q]) < v[o]
        o += q
