"""Pins of the CPU oracle against facts the paper and the mathematics fix (no GPU needed).

Each test checks the oracle against something other than itself: explicit Kronecker products for
H_k = E_k ⊗ E_k, closed forms, a dense LU solve of the whole KKT matrix, textbook properties of the
PSD projection, and optimal values known in closed form.
"""

import numpy as np
import pytest
import scipy.sparse

from oracle import chordal_admm as orc
from sdp_inputs import config_instance
from tests import sdp_cases


def make_sdp(arrs):
    return orc.ChordalSDP(arrs["n"], arrs["cliques"], arrs["A_ptr"], arrs["A_row"], arrs["A_col"],
                          arrs["A_val"], arrs["b"], arrs["C_row"], arrs["C_col"], arrs["C_val"])


@pytest.fixture(scope="module")
def cfg0():
    inst = config_instance(0)
    return inst, make_sdp(sdp_cases.instance_arrays(inst))


# ------------------------------------------------------------------ selectors and D (Sec. III.A)

def explicit_H(n, clique):
    """H_k = E_k ⊗ E_k as a dense matrix acting on vec(X) ∈ R^{n²} (column-major vec)."""
    s = len(clique)
    E = np.zeros((s, n))
    E[np.arange(s), clique] = 1.0
    return np.kron(E, E)


def test_selectors_match_kronecker_definition():
    arrs = sdp_cases.random_block_arrow(l=3, d=2, h=2, m=4)
    sdp = make_sdp(arrs)
    n = sdp.n
    rng = np.random.default_rng(0)
    X = rng.standard_normal((n, n))          # not symmetric: a transposed selector would show
    vecX = X.reshape(-1, order="F")
    # x on E: the entries of vec(X) at the ordered pattern pairs
    on_E = sdp.E_col * n + sdp.E_row
    x = vecX[on_E]
    for k, c in enumerate(sdp.cliques):
        Hk = explicit_H(n, c)
        # H_k x = vec(E_k X E_kᵀ) exactly (every row of H_k selects one entry)
        np.testing.assert_array_equal(sdp.H(k, x), Hk @ vecX)
        # rows of H_k are orthonormal (Sec. III.A)
        np.testing.assert_array_equal(Hk @ Hk.T, np.eye(len(c) ** 2))
        Ek = np.zeros((len(c), n)); Ek[np.arange(len(c)), c] = 1
        np.testing.assert_array_equal(sdp.H(k, x).reshape(len(c), len(c), order="F"), Ek @ X @ Ek.T)


def test_D_is_diagonal_count_and_block_arrow_closed_form():
    l, d, h = 4, 3, 2
    arrs = sdp_cases.random_block_arrow(l=l, d=d, h=h, m=4)
    sdp = make_sdp(arrs)
    n = sdp.n
    D_full = sum(explicit_H(n, c).T @ explicit_H(n, c) for c in sdp.cliques)
    # D = Σ H_kᵀ H_k is diagonal (Sec. III.B.1)
    assert np.count_nonzero(D_full - np.diag(np.diag(D_full))) == 0
    on_E = sdp.E_col * n + sdp.E_row
    np.testing.assert_array_equal(np.diag(D_full)[on_E], sdp.D)
    # block-arrow: head×head entries are covered by all l cliques, every other entry by one
    head = (sdp.E_row >= l * d) & (sdp.E_col >= l * d)
    assert np.all(sdp.D[head] == l) and np.all(sdp.D[~head] == 1)
    # |E| closed form
    assert sdp.nE == l * d * d + h * h + 2 * h * l * d


def test_scatter_is_sum_of_transposed_selectors():
    arrs = sdp_cases.random_block_arrow(l=3, d=2, h=3, m=4)
    sdp = make_sdp(arrs)
    n = sdp.n
    rng = np.random.default_rng(1)
    blocks = [rng.standard_normal(len(c) ** 2) for c in sdp.cliques]
    on_E = sdp.E_col * n + sdp.E_row
    ref = sum(explicit_H(n, c).T @ v for c, v in zip(sdp.cliques, blocks))[on_E]
    got = sdp.HT_sum(blocks)
    single = sdp.D == 1
    np.testing.assert_array_equal(got[single], ref[single])
    np.testing.assert_allclose(got, ref, rtol=1e-15, atol=1e-15)
    # brute force, ascending k from zero, one entry at a time: bit-exact
    for e in np.nonzero(~single)[0][:10]:
        acc = 0.0
        for k, c in enumerate(sdp.cliques):
            hit = np.nonzero(sdp.idx[k] == e)[0]
            for j in hit:
                acc += blocks[k][j]
        assert acc == got[e]


def test_generator_pattern_and_feasibility(cfg0):
    inst, sdp = cfg0
    l, d, h = 10, 10, 2
    nl = l * d * (d + 1) // 2 + h * (h + 1) // 2 + h * l * d
    assert len(inst.pat_row) == nl and sdp.nE == l * d * d + h * h + 2 * h * l * d
    assert all(len(c) == d + h for c in inst.cliques)
    assert inst.nnz_A == inst.m * round(0.3 * nl)
    # b = 𝒜(X0) and C = 𝒜*(y0) + Z0 hold on the vectorised data
    x0 = sdp.from_lower(inst.pat_row, inst.pat_col, inst.X0_val)
    z0 = sdp.from_lower(inst.pat_row, inst.pat_col, inst.Z0_val)
    np.testing.assert_allclose(sdp.A @ x0, inst.b, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(sdp.A.T @ inst.y0 + z0, sdp.c, rtol=1e-12, atol=1e-12)
    # Z0 ≻ 0 (diagonally dominant) and X0's clique blocks are PSD (X0 = G Gᵀ)
    Zd = np.zeros((inst.n, inst.n))
    Zd[inst.pat_row, inst.pat_col] = inst.Z0_val
    Zd = Zd + np.tril(Zd, -1).T
    assert np.linalg.eigvalsh(Zd)[0] > 0
    for k in range(sdp.p):
        s = len(sdp.cliques[k])
        assert np.linalg.eigvalsh(sdp.H(k, x0).reshape(s, s, order="F"))[0] > -1e-12


# ------------------------------------------------------------ PSD projection (Eq. XkUpdate)

def rand_sym(rng, s, scale=1.0):
    W = rng.standard_normal((s, s)) * scale
    return (W + W.T) / 2


@pytest.mark.parametrize("s", [1, 2, 5, 12, 30, 60])
def test_proj_psd_properties(s):
    rng = np.random.default_rng(s)
    for _ in range(5):
        W = rand_sym(rng, s, scale=10.0)
        P = orc.proj_psd(W)
        nW = np.linalg.norm(W)
        assert np.array_equal(P, P.T)
        assert np.linalg.eigvalsh(P)[0] >= -1e-13 * nW                        # PSD
        np.testing.assert_allclose(orc.proj_psd(P), P, atol=1e-12 * nW)       # idempotent
        np.testing.assert_allclose(P - orc.proj_psd(-W), W, atol=1e-12 * nW)  # Moreau
        assert abs(np.sum(P * (P - W))) <= 1e-11 * nW * nW                    # orthogonality
        # nearest PSD matrix: no random PSD candidate is closer
        for _ in range(5):
            G = rng.standard_normal((s, s))
            Y = G @ G.T
            assert np.linalg.norm(W - P) <= np.linalg.norm(W - Y) + 1e-12


def test_proj_psd_special_cases():
    rng = np.random.default_rng(3)
    d = rng.standard_normal(7)
    np.testing.assert_array_equal(orc.proj_psd(np.diag(d)), np.diag(np.maximum(d, 0)))
    G = rng.standard_normal((6, 6))
    S = G @ G.T
    np.testing.assert_allclose(orc.proj_psd(S), S, atol=1e-12 * np.linalg.norm(S))
    np.testing.assert_allclose(orc.proj_psd(-S), 0.0, atol=1e-12 * np.linalg.norm(S))
    g = sdp_cases.read_golden("psd_2x2.txt")
    W = np.array([float(v) for v in g["W"]]).reshape(2, 2)
    P = np.array([float(v) for v in g["P"]]).reshape(2, 2)
    np.testing.assert_allclose(orc.proj_psd(W), P, atol=1e-14)


# ---------------------------------------------------------------- KKT solve (Eq. OptCondMinY*)

def test_kkt_block_elimination_matches_dense_solve(cfg0):
    inst, sdp = cfg0
    rng = np.random.default_rng(4)
    rhs1 = rng.standard_normal(sdp.nE)
    rhs2 = rng.standard_normal(sdp.m)
    x, y = sdp.kkt_solve(rhs1, rhs2)
    A = sdp.A.toarray()
    K = np.block([[np.diag(sdp.D), A.T], [A, np.zeros((sdp.m, sdp.m))]])
    sol = np.linalg.solve(K, np.concatenate([rhs1, rhs2]))
    np.testing.assert_allclose(x, sol[:sdp.nE], rtol=1e-10, atol=1e-10 * np.abs(sol).max())
    np.testing.assert_allclose(y, sol[sdp.nE:], rtol=1e-10, atol=1e-10 * np.abs(sol).max())
    np.testing.assert_allclose(A @ x, rhs2, atol=1e-11 * np.abs(rhs2).max())
    res = K @ np.concatenate([x, y]) - np.concatenate([rhs1, rhs2])
    assert np.linalg.norm(res) <= 1e-12 * np.linalg.norm(np.concatenate([rhs1, rhs2])) * 10


def test_setup_rejects_bad_input():
    arrs = sdp_cases.random_block_arrow(l=3, d=2, h=2, m=4)
    bad = dict(arrs)
    bad["cliques"] = [c[::-1] for c in arrs["cliques"]]
    with pytest.raises(orc.OracleError) as e:
        make_sdp(bad)
    assert e.value.code == -2
    bad = dict(arrs)
    bad["cliques"] = arrs["cliques"][:-1]        # the last block's entries are no longer covered
    with pytest.raises(orc.OracleError) as e:
        make_sdp(bad)
    assert e.value.code == -2
    bad = dict(arrs)                             # duplicate constraint: A rank-deficient
    k0 = arrs["A_ptr"][1]
    bad["A_ptr"] = np.concatenate([arrs["A_ptr"], [arrs["A_ptr"][-1] + k0]])
    bad["A_row"] = np.concatenate([arrs["A_row"], arrs["A_row"][:k0]])
    bad["A_col"] = np.concatenate([arrs["A_col"], arrs["A_col"][:k0]])
    bad["A_val"] = np.concatenate([arrs["A_val"], arrs["A_val"][:k0]])
    bad["b"] = np.concatenate([arrs["b"], arrs["b"][:1]])
    with pytest.raises(orc.OracleError) as e:
        make_sdp(bad)
    assert e.value.code == -3


# ------------------------------------------------------------------ whole solves (Alg. 1, 2)

def test_trace_one_gives_lambda_min():
    arrs, lam_min = sdp_cases.trace_one_block_arrow(l=3, d=3, h=2)
    sdp = make_sdp(arrs)
    for form in ("primal", "dual"):
        r = orc.admm_solve(sdp, form, rho=1.0, tol=1e-9, max_iter=20000)
        assert r["status"] == 0
        obj = r["obj_primal"] if form == "primal" else r["obj_dual"]
        assert abs(obj - lam_min) <= 1e-6 * max(1.0, abs(lam_min))


def test_lovasz_theta_c5():
    arrs, opt = sdp_cases.theta_c5()
    sdp = make_sdp(arrs)
    r = orc.admm_solve(sdp, "primal", rho=1.0, tol=1e-10, max_iter=20000)
    assert r["status"] == 0
    assert abs(r["obj_primal"] - opt) <= 1e-7


def test_dense_and_decomposed_agree():
    """Grone's theorem: one dense clique and the clique decomposition have the same optimum."""
    arrs = sdp_cases.random_block_arrow(l=3, d=3, h=2, m=5)
    dec = make_sdp(arrs)
    dense = dict(arrs)
    dense["cliques"] = [np.arange(arrs["n"], dtype=np.int32)]
    den = make_sdp(dense)
    r1 = orc.admm_solve(dec, "primal", rho=1.0, tol=1e-9, max_iter=50000)
    r2 = orc.admm_solve(den, "primal", rho=1.0, tol=1e-9, max_iter=50000)
    assert r1["status"] == 0 and r2["status"] == 0
    assert abs(r1["obj_primal"] - r2["obj_primal"]) <= 1e-6 * max(1, abs(r2["obj_primal"]))


def test_primal_dual_remark1_and_bounds(cfg0):
    inst, sdp = cfg0
    rp = orc.admm_solve(sdp, "primal", rho=1.0, tol=1e-6, max_iter=20000)
    rd = orc.admm_solve(sdp, "dual", rho=1.0, tol=1e-6, max_iter=20000)
    assert rp["status"] == 0 and rd["status"] == 0
    # Remark 1: the decomposed dual is the dual of the decomposed primal — same optimal value
    assert abs(rp["obj_primal"] - rd["obj_dual"]) <= 1e-4 * abs(rd["obj_dual"])
    # weak duality bounds from the feasible-by-construction generator
    w = np.where(inst.pat_row != inst.pat_col, 2.0, 1.0)
    lo = float(inst.b @ inst.y0)
    hi = float(np.sum(w * inst.C_val * inst.X0_val))
    assert lo - 1e-6 <= rp["obj_primal"] <= hi + 1e-6
    # at convergence: Ax = b, the clique blocks of X are PSD, Z = Σ H_kᵀ λ_k is the dual slack
    X, y, Z = orc.primal_solution(sdp, rp, 1.0)
    np.testing.assert_allclose(sdp.A @ X, sdp.b, atol=1e-9 * np.abs(sdp.b).max())
    for k in range(sdp.p):
        s = len(sdp.cliques[k])
        lam = np.linalg.eigvalsh(rp["xk"][k].reshape(s, s, order="F"))
        assert lam[0] >= -1e-10 * abs(lam[-1])
        lam_k = np.linalg.eigvalsh(rp["lam"][k].reshape(s, s, order="F"))
        assert lam_k[0] >= -1e-10 * max(1.0, abs(lam_k[-1]))
    # dual feasibility residual of (y, Z): A*y + Z ≈ C, relative to the data
    np.testing.assert_allclose(sdp.A.T @ y + Z, sdp.c, atol=1e-3 * np.abs(sdp.c).max())


def test_primal_multipliers_are_psd_every_iteration(cfg0):
    """λ_k⁺ = λ_k + ρ(P(W) − u_k) = ρ P(−W): PSD after every primal iteration (Moreau)."""
    _, sdp = cfg0
    st = orc.admm_init(sdp, "primal")
    for _ in range(5):
        st = orc.primal_iteration(sdp, st, 1.0)
        np.testing.assert_allclose(sdp.A @ st["x"], sdp.b, atol=1e-10 * np.abs(sdp.b).max())
        for k in range(sdp.p):
            s = len(sdp.cliques[k])
            L = st["lam"][k].reshape(s, s, order="F")
            ev = np.linalg.eigvalsh(L)
            assert ev[0] >= -1e-12 * max(1.0, abs(ev[-1]))


def test_dual_multiplier_shortcut_and_sign(cfg0):
    """Eq. (MultUpdateDualSDP) with Eq. (vkEqn) substituted gives λ_k = −ρ H_k x (sign fixed)."""
    _, sdp = cfg0
    rho = 0.7
    st = orc.admm_init(sdp, "dual")
    for _ in range(4):
        st = orc.dual_iteration(sdp, st, rho)
        for k in range(sdp.p):
            scale = max(1.0, np.abs(st["lam"][k]).max(), np.abs(st["zk"][k]).max() * rho)
            np.testing.assert_allclose(st["lam_general"][k], st["lam"][k], atol=1e-12 * scale)
            if np.abs(st["u"][k]).max() > 1e-8:
                # the sign printed in Eq. (DualMultUpdate) does not satisfy the update
                assert not np.allclose(st["lam_general"][k], rho * st["u"][k], atol=1e-9 * scale)
        np.testing.assert_allclose(sdp.A @ st["x"], -sdp.b / rho, atol=1e-10 * np.abs(sdp.b).max())


def test_primal_dual_are_scaled_versions(cfg0):
    """Fig. 1 'Scaling': Algorithm 1 with ρ and Algorithm 2 with 1/ρ take the same iterations.

    The exact iterate map is not derived in the paper (parity unpinned as an identity); this checks
    the observable consequence: equal iteration counts and objectives.
    """
    _, sdp = cfg0
    rp = orc.admm_solve(sdp, "primal", rho=10.0, tol=1e-4, max_iter=2000)
    rd = orc.admm_solve(sdp, "dual", rho=0.1, tol=1e-4, max_iter=2000)
    assert abs(rp["iters"] - rd["iters"]) <= 1
    assert abs(rp["obj_primal"] - rd["obj_primal"]) <= 1e-6 * abs(rp["obj_primal"])


# ------------------------------------------------- stopping measures (Sec. III.B, Sec. IV.B)

def _stacked_selector(sdp):
    """[H_1; …; H_p] restricted to the pattern pairs E, built from E_k ⊗ E_k (dense)."""
    n = sdp.n
    on_E = sdp.E_col * n + sdp.E_row
    return np.vstack([explicit_H(n, c)[:, on_E] for c in sdp.cliques])


def _boyd_measures(A_B, B_B, c_B, xB, zB, zB_prev, yB, rho):
    """Relative primal and dual residuals of ADMM for min f(x) + g(z) s.t. A x + B z = c
    (Boyd et al. 2011, Sec. 3.3): r = A x⁺ + B z⁺ − c over max(‖A x⁺‖, ‖B z⁺‖, ‖c‖), and
    s = ρ Aᵀ B (z⁺ − z) over ‖Aᵀ y⁺‖, y the unscaled multiplier."""
    r = A_B @ xB + B_B @ zB - c_B
    s = rho * (A_B.T @ (B_B @ (zB - zB_prev)))
    return (np.linalg.norm(r), max(np.linalg.norm(A_B @ xB), np.linalg.norm(B_B @ zB), np.linalg.norm(c_B)),
            np.linalg.norm(s), np.linalg.norm(A_B.T @ yB))


@pytest.mark.parametrize("form", ["primal", "dual"])
def test_stopping_measures_match_boyd_residuals(form):
    """ε_p and ε_d are Boyd's relative residuals of the paper's splitting, assembled here from
    explicit matrices rather than from the oracle's helpers.

    Primal form (Eq. AugLagrPrimal): the first block is x, the second the stacked x_k, and the
    constraint x_k − H_k x = 0 carries λ_k, so A = −[H_k], B = I, c = 0, y = [λ_k].
    Dual form (Eq. AugLagrDual, Algorithm 2 minimising over 𝒴 before 𝒳): the first block is the
    stacked z_k, the second (y, v_k), and z_k − v_k = 0 carries λ_k, so A = I, B = [0, −I], c = 0.
    """
    arrs = sdp_cases.random_block_arrow(l=3, d=2, h=2, m=4)
    sdp = make_sdp(arrs)
    rho = 0.7                          # ≠ 1, so that a lost factor ρ shows
    H = _stacked_selector(sdp)
    nS = H.shape[0]
    st = orc.admm_init(sdp, form)
    step = orc.primal_iteration if form == "primal" else orc.dual_iteration
    for it in range(4):
        prev = st
        st = step(sdp, st, rho)
        if form == "primal":
            A_B, B_B = -H, np.eye(nS)
            xB = st["x"]
            zB, zB_prev = np.concatenate(st["xk"]), np.concatenate(prev["xk"])
        else:
            A_B = np.eye(nS)
            B_B = np.hstack([np.zeros((nS, sdp.m)), -np.eye(nS)])
            xB = np.concatenate(st["zk"])
            zB = np.concatenate([st["y"], np.concatenate(st["vk"])])
            zB_prev = np.concatenate([prev["y"], np.concatenate(prev["vk"])])
        yB = np.concatenate(st["lam"])
        rp, rp_den, rd, rd_den = _boyd_measures(A_B, B_B, np.zeros(nS), xB, zB, zB_prev, yB, rho)
        assert rp > 0 and rd > 0
        for got, want in ((st["res_p"], rp), (st["res_p_den"], rp_den), (st["res_d"], rd),
                          (st["res_d_den"], rd_den)):
            assert abs(got - want) <= 1e-13 * want, (form, it, got, want)
        assert st["eps_p"] == st["res_p"] / st["res_p_den"]
        assert st["eps_d"] == st["res_d"] / st["res_d_den"]
