"""Plain FP64 CPU reference for differentiating unrolled ADMM (Algorithm 1, primal form).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: imported by ``tests/`` and nothing else.

The paper has no derivative of its method; what is differentiated here is T iterations of
Algorithm 1 run from zero iterates, as functions of the cost ``c`` and the right-hand side ``b``.
Everything lives in the oracle's full representation (vectors on the ordered pattern pairs E,
full s×s clique blocks), where all maps are plain Euclidean linear maps:

* iteration t takes (x_k, λ_k) to
  r = Σ H_kᵀ(x_k + ρ⁻¹λ_k) − ρ⁻¹c,   [x; y] = KKT⁻¹ [r; b]   (Eq. OptCondMinYPrimal),
  u_k = H_k x,  W_k = u_k − ρ⁻¹λ_k,  x_k⁺ = P₊(W_k)   (Eq. XkUpdate),
  λ_k⁺ = λ_k + ρ(x_k⁺ − u_k)   (Eq. LambdakUpdate);
* the output is the affine iterate x of iteration T (X_T);
* reverse mode runs the transposed maps backwards. The block elimination of the KKT system is
  self-adjoint: x = S r + D⁻¹Aᵀ M⁻¹ b with S = D⁻¹ − D⁻¹AᵀM⁻¹AD⁻¹ symmetric, so the adjoint of
  (r, b) ↦ x is one more KKT solve with right-hand side [x̄; 0], returning r̄ = x and b̄ = y;
* the derivative of P₊ at a symmetric W = V diag(λ) Vᵀ is the Daleckii–Krein formula
  DP₊(W)[E] = V (Γ ∘ (Vᵀ E V)) Vᵀ with Γ_ij = (f(λ_i) − f(λ_j)) / (λ_i − λ_j), f = max(·, 0), and
  f' of the pair's mean where |λ_i − λ_j| ≤ 1e-12 max|λ| (f'(0) taken as 0). It is self-adjoint;
* cone blocks (Section V's other cones, projected in the primal form onto the cone itself): the
  free block's projection is the identity, the nonnegative one's derivative is the 0/1 mask of
  w > 0, and the second-order one's (for ‖u‖ > |t|) is ½[[1, ûᵀ], [û, (1 + t/‖u‖)I − (t/‖u‖)ûûᵀ]]
  with û = u/‖u‖ (the identity inside the cone, zero inside its polar); all are symmetric.

A full-representation gradient ḡ (∂L/∂ each ordered-pair entry) of a symmetric quantity relates
to the gradient with respect to its lower-triangle parameters (an off-diagonal parameter moves
both (i, j) and (j, i)) by ∂L/∂θ_e = ḡ_(i,j) + ḡ_(j,i) = w_e ḡ_e, w_e = 2 off the diagonal.
"""

from __future__ import annotations

import copy

import numpy as np

from .chordal_admm import ChordalSDP, _mat, _vec, admm_init, primal_iteration


def dk_gamma(lam: np.ndarray) -> np.ndarray:
    """Divided differences of f = max(·, 0) on the eigenvalues (Daleckii–Krein)."""
    f = np.maximum(lam, 0.0)
    li, lj = lam[:, None], lam[None, :]
    diff = li - lj
    close = np.abs(diff) <= 1e-12 * max(float(np.max(np.abs(lam))), 1e-300)
    mean = 0.5 * (li + lj)
    with np.errstate(divide="ignore", invalid="ignore"):
        G = (f[:, None] - f[None, :]) / diff
    return np.where(close, (mean > 0.0).astype(np.float64), G)


def proj_psd_vjp(W: np.ndarray, Xbar: np.ndarray) -> np.ndarray:
    """DP₊(W)ᵀ[X̄] = DP₊(W)[sym X̄] for symmetric W (library eigendecomposition as one step)."""
    W = 0.5 * (W + W.T)
    lam, V = np.linalg.eigh(W)
    Y = V.T @ (0.5 * (Xbar + Xbar.T)) @ V
    return V @ (dk_gamma(lam) * Y) @ V.T


def proj_soc_vjp(w: np.ndarray, gbar: np.ndarray) -> np.ndarray:
    """The derivative of the second-order projection at w applied to ḡ (it is symmetric)."""
    t, u = float(w[0]), np.asarray(w[1:], dtype=np.float64)
    nu = float(np.sqrt(np.dot(u, u)))
    if nu <= t:
        return np.array(gbar, dtype=np.float64)
    if nu <= -t:
        return np.zeros(len(w))
    uh = u / nu
    gt, gu = float(gbar[0]), np.asarray(gbar[1:], dtype=np.float64)
    r = t / nu
    out_t = 0.5 * (gt + float(np.dot(uh, gu)))
    out_u = 0.5 * gt * uh + 0.5 * ((1.0 + r) * gu - r * float(np.dot(uh, gu)) * uh)
    return np.concatenate([[out_t], out_u])


def proj_cone_vjp(kind: str, w: np.ndarray, gbar: np.ndarray) -> np.ndarray:
    """The derivative of a cone block's (primal-form) projection at w applied to ḡ."""
    if kind == "free":
        return np.array(gbar, dtype=np.float64)
    if kind == "nonneg":
        return np.where(np.asarray(w) > 0.0, gbar, 0.0)
    if kind == "soc":
        return proj_soc_vjp(w, gbar)
    raise ValueError(f"unknown cone {kind!r}")


def with_data(sdp: ChordalSDP, c_full: np.ndarray | None = None, b: np.ndarray | None = None) -> ChordalSDP:
    """A copy of the problem with a new cost and/or right-hand side (the KKT factor is unchanged:
    it depends on A and D only)."""
    out = copy.copy(sdp)
    if c_full is not None:
        out.c = np.asarray(c_full, dtype=np.float64)
    if b is not None:
        out.b = np.asarray(b, dtype=np.float64)
    return out


def unrolled_forward(sdp: ChordalSDP, rho: float, T: int) -> list:
    """States after 0..T iterations of Algorithm 1 from zero iterates."""
    states = [admm_init(sdp, "primal")]
    for _ in range(T):
        states.append(primal_iteration(sdp, states[-1], rho))
    return states


def unrolled_backward(sdp: ChordalSDP, rho: float, states: list, xbar_T: np.ndarray):
    """Reverse mode through the iterations in ``states`` (from ``unrolled_forward``).

    ``xbar_T`` is ∂L/∂x_T in the full representation. Returns (c̄, b̄): ∂L/∂c in the full
    representation through the iterations only (a loss that also uses c directly adds that term
    itself) and ∂L/∂b."""
    rinv = 1.0 / rho
    T = len(states) - 1
    K = range(sdp.nblk)
    Xb = [np.zeros(sdp.block_len(k)) for k in K]
    Lb = [np.zeros(sdp.block_len(k)) for k in K]
    cbar = np.zeros(sdp.nE)
    bbar = np.zeros(sdp.m)
    for t in range(T, 0, -1):
        prev, cur = states[t - 1], states[t]
        ub, Lpart = [], []
        for k in K:
            # λ_k⁺ = λ_k + ρ(x_k⁺ − u_k);  x_k⁺ = P(W_k);  W_k = u_k − ρ⁻¹λ_k
            Xt = Xb[k] + rho * Lb[k]
            W = cur["u"][k] - rinv * prev["lam"][k]
            if sdp.kinds[k] == "psd":
                s = len(sdp.cliques[k])
                Wb = _vec(proj_psd_vjp(_mat(W, s), _mat(Xt, s)))
            else:
                Wb = proj_cone_vjp(sdp.kinds[k], W, Xt)
            ub.append(Wb - rho * Lb[k])
            Lpart.append(Lb[k] - rinv * Wb)
        # u_k = H_k x (plus the loss term at the last iteration)
        xbar = sdp.HT_sum(ub)
        if t == T:
            xbar = xbar + xbar_T
        # x = S r + D⁻¹AᵀM⁻¹b: one KKT solve with right-hand side [x̄; 0]
        rbar, ybar = sdp.kkt_solve(xbar, np.zeros(sdp.m))
        bbar += ybar
        # r = Σ H_kᵀ(x_k + ρ⁻¹λ_k) − ρ⁻¹c
        cbar += -rinv * rbar
        Xb = [sdp.H(k, rbar) for k in K]
        Lb = [Lpart[k] + rinv * sdp.H(k, rbar) for k in K]
    return cbar, bbar


def loss_and_grad(sdp: ChordalSDP, rho: float, T: int, x_ref: np.ndarray):
    """L = ⟨C, X_T⟩ + ‖X_T − X_ref‖_F² and its gradients with respect to the lower-triangle
    parameters of C (on E_L, column-major) and to b. ``x_ref`` is in the full representation."""
    states = unrolled_forward(sdp, rho, T)
    x = states[-1]["x"]
    d = x - x_ref
    L = float(np.dot(sdp.c, x) + np.dot(d, d))
    cbar, bbar = unrolled_backward(sdp, rho, states, sdp.c + 2.0 * d)
    cbar = cbar + x                                # the loss's direct use of C
    lower = sdp.lower_mask()
    w = np.where(sdp.E_row[lower] == sdp.E_col[lower], 1.0, 2.0)
    return L, w * cbar[lower], bbar, states


def loss_at(sdp: ChordalSDP, rho: float, T: int, x_ref: np.ndarray, c_lower=None, b=None) -> float:
    """L for perturbed lower-triangle C parameters and/or b (for finite differences)."""
    c_full = None
    if c_lower is not None:
        lower = sdp.lower_mask()
        c_full = sdp.from_lower(sdp.E_row[lower], sdp.E_col[lower], c_lower)
    p = with_data(sdp, c_full, b)
    x = unrolled_forward(p, rho, T)[-1]["x"]
    d = x - x_ref
    return float(np.dot(p.c, x) + np.dot(d, d))
