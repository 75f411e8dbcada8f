"""The oracle pins bind: a planted mistake in the oracle makes at least one pin fail.

Every mistake is planted on the CPU, in the oracle, through monkeypatching; nothing here touches the
CUDA path.
"""

import numpy as np
import pytest

from oracle import chordal_admm as orc
from sdp_inputs import config_instance
from tests import sdp_cases
from tests import test_oracle_pins as pins


def _expect_pin_failure(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_projection_without_clip_is_caught(monkeypatch):
    def no_clip(W):
        W = 0.5 * (W + W.T)
        lam, V = np.linalg.eigh(W)
        return (V * lam) @ V.T
    monkeypatch.setattr(orc, "proj_psd", no_clip)
    _expect_pin_failure(pins.test_proj_psd_properties, 5)


def test_projection_clipping_wrong_side_is_caught(monkeypatch):
    def wrong_side(W):
        lam, V = np.linalg.eigh(0.5 * (W + W.T))
        return (V * np.minimum(lam, 0.0)) @ V.T
    monkeypatch.setattr(orc, "proj_psd", wrong_side)
    _expect_pin_failure(pins.test_proj_psd_special_cases)


def test_transposed_selector_is_caught(monkeypatch):
    orig = orc.ChordalSDP.__init__

    def init(self, *a, **k):
        orig(self, *a, **k)
        # swap (a, b) ↔ (b, a): each block is read row-major instead of column-major
        for i, c in enumerate(self.cliques):
            s = len(c)
            self.idx[i] = self.idx[i].reshape(s, s, order="F").T.reshape(-1, order="F")
    monkeypatch.setattr(orc.ChordalSDP, "__init__", init)
    _expect_pin_failure(pins.test_selectors_match_kronecker_definition)


def test_wrong_D_is_caught(monkeypatch):
    def kkt(self, rhs1, rhs2):
        ones = np.ones_like(self.D)
        t = self.A @ rhs1 - rhs2
        y = np.linalg.solve(self.M, t)
        return (rhs1 - self.A.T @ y) / ones, y
    monkeypatch.setattr(orc.ChordalSDP, "kkt_solve", kkt)
    inst = config_instance(0)
    inst_sdp = (inst, pins.make_sdp(sdp_cases.instance_arrays(inst)))
    _expect_pin_failure(pins.test_kkt_block_elimination_matches_dense_solve, inst_sdp)


def test_wrong_multiplier_sign_is_caught(monkeypatch):
    orig = orc.primal_iteration

    def flipped(sdp, st, rho):
        out = orig(sdp, st, rho)
        out["lam"] = [st["lam"][k] - rho * (out["xk"][k] - out["u"][k]) for k in range(sdp.p)]
        return out
    monkeypatch.setattr(orc, "primal_iteration", flipped)
    _expect_pin_failure(pins.test_trace_one_gives_lambda_min)


def test_dropped_cost_term_is_caught(monkeypatch):
    def no_cost(sdp, st, rho):
        saved = sdp.c
        sdp.c = np.zeros_like(saved)
        try:
            return orig(sdp, st, rho)
        finally:
            sdp.c = saved
    orig = orc.primal_iteration
    monkeypatch.setattr(orc, "primal_iteration", no_cost)
    _expect_pin_failure(pins.test_lovasz_theta_c5)


def test_dropped_rho_in_dual_residual_is_caught(monkeypatch):
    orig = orc.primal_iteration

    def no_rho(sdp, st, rho):
        out = orig(sdp, st, rho)
        out["res_d"] = out["res_d"] / rho
        out["eps_d"] = out["res_d"] / out["res_d_den"]
        return out
    monkeypatch.setattr(orc, "primal_iteration", no_rho)
    _expect_pin_failure(pins.test_stopping_measures_match_boyd_residuals, "primal")


def test_old_multiplier_in_dual_denominator_is_caught(monkeypatch):
    orig = orc.dual_iteration

    def old_lam(sdp, st, rho):
        out = orig(sdp, st, rho)
        out["res_d_den"] = max(float(np.sqrt(sum(float(np.dot(v, v)) for v in st["lam"]))), 1e-12)
        out["eps_d"] = out["res_d"] / out["res_d_den"]
        return out
    monkeypatch.setattr(orc, "dual_iteration", old_lam)
    _expect_pin_failure(pins.test_stopping_measures_match_boyd_residuals, "dual")


def test_primal_residual_against_wrong_iterate_is_caught(monkeypatch):
    orig = orc.dual_iteration

    def stale_v(sdp, st, rho):
        out = orig(sdp, st, rho)
        # z_k − v_k against the previous v_k instead of the one just computed
        out["res_p"] = float(np.sqrt(sum(float(np.dot(z - v, z - v)) for z, v in zip(out["zk"], st["vk"]))))
        out["eps_p"] = out["res_p"] / out["res_p_den"]
        return out
    monkeypatch.setattr(orc, "dual_iteration", stale_v)
    _expect_pin_failure(pins.test_stopping_measures_match_boyd_residuals, "dual")
