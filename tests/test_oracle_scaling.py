"""Pin of the primal/dual relation (Section IV: the two decomposed ADMM algorithms are scaled
versions of each other, Algorithm 2 with penalty ρ matching Algorithm 1 with penalty 1/ρ), without
a GPU.

The exact correspondence, derived from the two algorithms (σ = 1/ρ; S, T the linear maps of the
KKT solve, x = S r + T s):
* Algorithm 1's block and multiplier steps combine, by Moreau's decomposition, into
  λ⁺ = P_{K*}(λ − σ H_k x⁺) and x_k⁺ = H_k x⁺ + (λ⁺ − λ)/σ;
* Algorithm 2's steps combine, through Eq. vkEqn and the corrected Eq. DualMultUpdate, into
  z⁺ = P_{K*}(z − H_k x⁻ + 2 H_k x), where x⁻, x are its last two affine iterates;
* with those, if λ = z at iterations n−1 and n and Algorithm 1's affine iterate is
  x_n = ρ(x'_{n−2} − 2 x'_{n−1}) (primes: Algorithm 2), both hold again at n+1 (the right-hand
  sides of the two KKT solves are then σ-multiples of each other's combination).
So Algorithm 1 started from that state reproduces Algorithm 2's z_k as its multipliers λ_k at
every later iteration. (From the zero initial iterates of both, the correspondence is not exact;
the paper's claim is about the algorithms, not about a particular start.) The test runs both
oracle algorithms independently; a planted sign error in the dual multiplier update breaks it.
"""

import numpy as np
import pytest

from oracle import chordal_admm as orc
from tests import sdp_cases
from tests.gpu_support import make_oracle


def corresponding_primal_state(sdp, D, rho, k0):
    """Algorithm 1's state at iteration k0 that corresponds to Algorithm 2's iterates D[0..k0]."""
    st = orc.admm_init(sdp, "primal")
    x = rho * (D[k0 - 2]["x"] - 2.0 * D[k0 - 1]["x"])
    lam = [z.copy() for z in D[k0]["zk"]]
    xk = [sdp.H(j, x) + rho * (D[k0]["zk"][j] - D[k0 - 1]["zk"][j]) for j in range(sdp.nblk)]
    st.update(x=x, lam=lam, xk=xk, iter=k0)
    return st


def max_gaps(sdp, rho, iters=30, k0=2):
    D = [orc.admm_init(sdp, "dual")]
    for _ in range(iters):
        D.append(orc.dual_iteration(sdp, D[-1], rho))
    st = corresponding_primal_state(sdp, D, rho, k0)
    g_lam = g_x = 0.0
    for k in range(k0 + 1, iters + 1):
        st = orc.primal_iteration(sdp, st, 1.0 / rho)
        a, b = np.concatenate(st["lam"]), np.concatenate(D[k]["zk"])
        g_lam = max(g_lam, float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1.0)))
        xr = rho * (D[k - 2]["x"] - 2.0 * D[k - 1]["x"])
        g_x = max(g_x, float(np.max(np.abs(st["x"] - xr)) / max(np.max(np.abs(xr)), 1.0)))
    return g_lam, g_x


@pytest.mark.parametrize("rho", [0.02, 0.7, 3.0])
def test_primal_multipliers_reproduce_dual_blocks(rho):
    sdp = make_oracle(sdp_cases.random_block_arrow(l=3, d=3, h=2, m=5, seed=4))
    g_lam, g_x = max_gaps(sdp, rho)
    assert g_lam <= 1e-12 and g_x <= 1e-11


def test_relation_holds_with_every_cone_kind():
    sdp = make_oracle(sdp_cases.random_conic(l=2, d=3, h=2, n_free=2, n_lin=4, soc_dims=(3, 1), m=6, seed=21))
    g_lam, g_x = max_gaps(sdp, 0.5)
    assert g_lam <= 1e-12 and g_x <= 1e-11


def test_zero_starts_do_not_correspond():
    """Both algorithms from zero: the multipliers differ (the relation needs the matched start)."""
    sdp = make_oracle(sdp_cases.random_block_arrow(l=3, d=3, h=2, m=5, seed=4))
    sp, sd = orc.admm_init(sdp, "primal"), orc.admm_init(sdp, "dual")
    gap = 0.0
    for _ in range(10):
        sp, sd = orc.primal_iteration(sdp, sp, 50.0), orc.dual_iteration(sdp, sd, 0.02)
        gap = max(gap, float(np.max(np.abs(np.concatenate(sp["lam"]) - np.concatenate(sd["zk"])))))
    assert gap > 1e-3


def test_planted_sign_error_breaks_the_relation(monkeypatch):
    orig = orc.dual_iteration

    def printed_sign(sdp, st, rho):
        out = orig(sdp, st, rho)
        out["lam"] = [-l for l in out["lam"]]          # λ_k = +ρ H_k x, as printed
        return out
    monkeypatch.setattr(orc, "dual_iteration", printed_sign)
    sdp = make_oracle(sdp_cases.random_block_arrow(l=3, d=3, h=2, m=5, seed=4))
    assert max_gaps(sdp, 0.7, iters=12)[0] > 1e-3
