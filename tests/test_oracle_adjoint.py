"""Pins of the CPU reference gradient of unrolled ADMM (oracle/adjoint.py), without a GPU.

What fixes it, independently of its own code:
  - the Daleckii–Krein derivative of P₊ against central differences of the projection (and its
    closed forms on definite and diagonal matrices);
  - the whole reverse pass against central differences of the forward iterations, for C (lower
    parameters, perturbed symmetrically) and b, on a small block-arrow problem;
  - planted mistakes in the reverse pass (a dropped b̄ term, a wrong multiplier scaling) that the
    finite-difference check must catch;
  - the cone blocks' derivatives (free, nonnegative, second-order) against central differences
    of their projections and closed forms, and the reverse pass through a problem with every cone
    kind against central differences of its forward iterations.
"""

import numpy as np
import pytest

from oracle import adjoint as adj
from oracle import chordal_admm as orc
from sdp_inputs import config_instance
from tests import sdp_cases
from tests.gpu_support import make_oracle


def sym(rng, n):
    G = rng.standard_normal((n, n))
    return 0.5 * (G + G.T)


def separated(rng, n, gap=0.3):
    """Symmetric matrix with eigenvalues at least `gap` apart and away from 0."""
    lam = np.concatenate([np.arange(1, n // 2 + 1) * gap + 0.1, -np.arange(1, n - n // 2 + 1) * gap - 0.1])
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (Q * lam) @ Q.T


def test_dk_vjp_matches_central_differences():
    rng = np.random.default_rng(1)
    for n in (2, 5, 9):
        W = separated(rng, n)
        for _ in range(3):
            E, Xb = sym(rng, n), sym(rng, n)
            h = 1e-6
            fd = np.sum(Xb * (orc.proj_psd(W + h * E) - orc.proj_psd(W - h * E))) / (2 * h)
            an = np.sum(adj.proj_psd_vjp(W, Xb) * E)
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(fd))


def test_dk_vjp_closed_forms():
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    Xb = sym(rng, 6)
    pd = (Q * np.linspace(0.5, 3.0, 6)) @ Q.T
    np.testing.assert_allclose(adj.proj_psd_vjp(pd, Xb), Xb, atol=1e-12)       # P₊ = identity near PD
    nd = -pd
    np.testing.assert_allclose(adj.proj_psd_vjp(nd, Xb), 0.0, atol=1e-12)      # P₊ = 0 near ND
    d = np.array([2.0, -1.0, 0.5, -3.0])
    G = adj.proj_psd_vjp(np.diag(d), np.ones((4, 4)))
    f = np.maximum(d, 0)
    for i in range(4):
        for j in range(4):
            want = (1.0 if d[i] > 0 else 0.0) if i == j else (f[i] - f[j]) / (d[i] - d[j])
            assert abs(G[i, j] - want) <= 1e-14


@pytest.fixture(scope="module")
def small():
    arrs = sdp_cases.random_block_arrow(l=3, d=3, h=2, m=5, seed=4)
    sdp = make_oracle(arrs)
    rng = np.random.default_rng(9)
    lower = sdp.lower_mask()
    xr_lower = rng.standard_normal(int(lower.sum()))
    x_ref = sdp.from_lower(sdp.E_row[lower], sdp.E_col[lower], xr_lower)
    return sdp, x_ref


def fd_grads(sdp, rho, T, x_ref, ic, ib, h=1e-6):
    lower = sdp.lower_mask()
    c0 = sdp.to_lower(sdp.c)
    gc = []
    for e in ic:
        cp, cm = c0.copy(), c0.copy()
        cp[e] += h
        cm[e] -= h
        gc.append((adj.loss_at(sdp, rho, T, x_ref, c_lower=cp) - adj.loss_at(sdp, rho, T, x_ref, c_lower=cm)) / (2 * h))
    gb = []
    for i in ib:
        bp, bm = sdp.b.copy(), sdp.b.copy()
        bp[i] += h
        bm[i] -= h
        gb.append((adj.loss_at(sdp, rho, T, x_ref, b=bp) - adj.loss_at(sdp, rho, T, x_ref, b=bm)) / (2 * h))
    assert lower.sum() == len(c0)
    return np.array(gc), np.array(gb)


@pytest.mark.parametrize("rho,T", [(1.0, 12), (0.5, 25)])
def test_unrolled_gradient_matches_central_differences(small, rho, T):
    sdp, x_ref = small
    L, gc, gb, _ = adj.loss_and_grad(sdp, rho, T, x_ref)
    assert np.isfinite(L)
    rng = np.random.default_rng(3)
    ic = rng.choice(len(gc), size=10, replace=False)
    ib = np.arange(sdp.m)
    fc, fb = fd_grads(sdp, rho, T, x_ref, ic, ib)
    scale = max(np.abs(gc).max(), np.abs(gb).max())
    np.testing.assert_allclose(gc[ic], fc, rtol=1e-5, atol=1e-6 * scale)
    np.testing.assert_allclose(gb, fb, rtol=1e-5, atol=1e-6 * scale)


def test_unrolled_gradient_on_a_workload_instance():
    """A few coordinates on one problem of the differentiation workload (shorter unroll)."""
    inst = config_instance(4, 0)
    sdp = make_oracle(sdp_cases.instance_arrays(inst))
    lower = sdp.lower_mask()
    x_ref = sdp.from_lower(sdp.E_row[lower], sdp.E_col[lower], inst.X0_val)
    T, rho = 8, 1.0
    L, gc, gb, _ = adj.loss_and_grad(sdp, rho, T, x_ref)
    rng = np.random.default_rng(5)
    ic = rng.choice(len(gc), size=3, replace=False)
    ib = rng.choice(sdp.m, size=3, replace=False)
    # the loss here is ~700, so a 1e-6 step leaves differences near the rounding noise of the
    # eigensolves; 1e-4 keeps truncation (O(h^2)) and rounding both below 1e-8 relative
    fc, fb = fd_grads(sdp, rho, T, x_ref, ic, ib, h=1e-4)
    scale = max(np.abs(gc).max(), np.abs(gb).max())
    np.testing.assert_allclose(gc[ic], fc, rtol=1e-5, atol=1e-6 * scale)
    np.testing.assert_allclose(gb[ib], fb, rtol=1e-5, atol=1e-6 * scale)


def test_planted_mistakes_are_caught(small, monkeypatch):
    """The finite-difference pin fails for a reverse pass that drops b̄ or mis-scales λ̄."""
    sdp, x_ref = small
    rho, T = 1.0, 10
    ib = np.arange(sdp.m)
    _, fb = fd_grads(sdp, rho, T, x_ref, [], ib)

    orig = sdp.kkt_solve

    def no_ybar(rhs1, rhs2):
        xx, yy = orig(rhs1, rhs2)
        return xx, 0.0 * yy
    bad = adj.with_data(sdp)
    monkeypatch.setattr(bad, "kkt_solve", no_ybar)
    states = adj.unrolled_forward(sdp, rho, T)
    d = states[-1]["x"] - x_ref
    _, gb_bad = adj.unrolled_backward(bad, rho, states, sdp.c + 2 * d)
    assert not np.allclose(gb_bad, fb, rtol=1e-3, atol=1e-6)

    _, gc, gb, _ = adj.loss_and_grad(sdp, rho, T, x_ref)
    np.testing.assert_allclose(gb, fb, rtol=1e-5, atol=1e-8 * np.abs(fb).max())
    # a reverse pass run with the wrong ρ (as if ρ⁻¹ and ρ were swapped) disagrees
    _, gb_rho = adj.unrolled_backward(sdp, 1.0 / 3.0, states, sdp.c + 2 * d)
    assert not np.allclose(gb_rho, fb, rtol=1e-3, atol=1e-6)


def test_cone_vjps_match_central_differences():
    """The cone blocks' derivatives: second-order (off the cone's boundary, where it is smooth)
    against central differences of the projection; inside the cone the identity, inside its polar
    zero; the nonnegative mask."""
    rng = np.random.default_rng(12)
    h = 1e-6
    for trial in range(40):
        q = int(rng.integers(2, 7))
        w = rng.standard_normal(q)
        w[0] = rng.uniform(-0.9, 0.9) * np.linalg.norm(w[1:])          # |t| < ||u||: smooth part
        E, gbar = rng.standard_normal(q), rng.standard_normal(q)
        fd = np.dot(gbar, orc.proj_soc(w + h * E) - orc.proj_soc(w - h * E)) / (2 * h)
        an = np.dot(adj.proj_soc_vjp(w, gbar), E)
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (trial, fd, an)
    w = np.array([3.0, 1.0, -1.0])
    g = rng.standard_normal(3)
    np.testing.assert_array_equal(adj.proj_soc_vjp(w, g), g)                        # inside
    np.testing.assert_array_equal(adj.proj_soc_vjp(-w, g), np.zeros(3))             # polar
    np.testing.assert_array_equal(adj.proj_cone_vjp("nonneg", np.array([1.0, -1.0]), np.array([2.0, 3.0])), [2.0, 0.0])
    np.testing.assert_array_equal(adj.proj_cone_vjp("free", np.array([1.0, -1.0]), np.array([2.0, 3.0])), [2.0, 3.0])


def test_unrolled_gradient_with_cones_matches_central_differences():
    """The reverse pass through cone blocks (free, nonnegative, second-order) on a mixed problem,
    for the cost of matrix entries and of cone variables, and for b."""
    arrs = sdp_cases.random_conic(l=2, d=3, h=2, n_free=2, n_lin=4, soc_dims=(3, 4), m=6, seed=21)
    sdp = make_oracle(arrs)
    rng = np.random.default_rng(13)
    lower = sdp.lower_mask()
    x_ref = sdp.from_lower(sdp.E_row[lower], sdp.E_col[lower], rng.standard_normal(int(lower.sum())))
    rho, T = 0.8, 15
    L, gc, gb, _ = adj.loss_and_grad(sdp, rho, T, x_ref)
    n_mat = int(lower.sum()) - sdp.n_cone
    ic = np.concatenate([rng.choice(n_mat, size=4, replace=False), n_mat + np.arange(sdp.n_cone)])
    ib = np.arange(sdp.m)
    fc, fb = fd_grads(sdp, rho, T, x_ref, ic, ib)
    scale = max(np.abs(gc).max(), np.abs(gb).max())
    np.testing.assert_allclose(gc[ic], fc, rtol=1e-5, atol=1e-6 * scale)
    np.testing.assert_allclose(gb, fb, rtol=1e-5, atol=1e-6 * scale)


def test_planted_soc_derivative_mistake_is_caught(monkeypatch):
    """A dropped ûûᵀ term in the second-order derivative fails the difference check."""
    def wrong(w, gbar):
        t, u = float(w[0]), np.asarray(w[1:])
        nu = float(np.linalg.norm(u))
        if nu <= t:
            return np.array(gbar, float)
        if nu <= -t:
            return np.zeros(len(w))
        uh, gt, gu = u / nu, float(gbar[0]), np.asarray(gbar[1:])
        return np.concatenate([[0.5 * (gt + uh @ gu)], 0.5 * gt * uh + 0.5 * (1 + t / nu) * gu])
    monkeypatch.setattr(adj, "proj_soc_vjp", wrong)
    with pytest.raises(AssertionError):
        test_cone_vjps_match_central_differences()
