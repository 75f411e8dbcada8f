"""Full-size checks on the large block-arrow workload (l=2000, d=20, h=40: n = 40 040, 2000 cliques
of 60, m = 1000, 10 % density, 202 M nonzeros of A).

The oracle cannot run a whole iteration at this size, so one GPU iteration is checked through what
the paper fixes for every iterate: sampled clique projections against the oracle's P (Eq. zkUpdate),
the updates of v_k and lambda_k (Eqs. vkEqn, DualMultUpdate), both block rows of the KKT system
(Eq. OptCondMinYDual) via CPU sparse products, and the scatter on sampled entries (bit-exact).
"""

import numpy as np
import pytest
import scipy.sparse

from oracle import chordal_admm as orc
from sdp_inputs import CONFIGS, config_instance
from tests.gpu_support import require_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def large():
    torch, cadmm = require_gpu()
    inst = config_instance(3)
    arrs = dict(n=inst.n, cliques=inst.cliques, A_ptr=inst.A_ptr, A_row=inst.A_row, A_col=inst.A_col,
                A_val=inst.A_val, b=inst.b, C_row=inst.C_row, C_col=inst.C_col, C_val=inst.C_val)
    cfg = CONFIGS[3]
    opts = cadmm.make_opts(rho=cfg["rho"], tol=0.0, max_iter=cfg["max_iter"], form="dual", prec="fp64")
    s = cadmm.ChordalADMM(arrs, opts)
    maps = cadmm.sdp_get_maps(s.h)
    yield torch, cadmm, inst, s, maps
    s.close()


def lower_index(maps, n, rows, cols):
    keys = maps["pat_col"].astype(np.int64) * n + maps["pat_row"]
    q = np.asarray(cols, np.int64) * n + np.asarray(rows, np.int64)
    idx = np.searchsorted(keys, q)
    assert np.all(keys[idx] == q)
    return idx


def test_large_iteration_properties(large):
    torch, cadmm, inst, s, maps = large
    rho = CONFIGS[3]["rho"]
    sz = s.sizes
    nEL, SL, m = sz["nE_lower"], sz["S_lower"], sz["m"]
    s.reset()
    s.iterate(3)                       # a nonzero state reached by the method itself
    st0 = s.state()
    r = s.iterate(1)
    assert r["status"] == cadmm.SDP_MAX_ITER and r["iters"] == 4
    st1 = s.state()
    z, v_new, lam_new, x, y = st1["blk_a"], st1["blk_c"], st1["blk_b"], st1["x"], st1["y"]
    v_old, lam_old = st0["blk_c"], st0["blk_b"]
    gidx = maps["gather_idx"]
    off = maps["blk_off"]
    rinv = 1.0 / rho

    # Eqs. vkEqn and DualMultUpdate at every packed position
    u = x[gidx]
    np.testing.assert_array_equal(lam_new, -rho * u)
    np.testing.assert_allclose(v_new, (z + rinv * lam_old) + u, rtol=0, atol=1e-12 * np.abs(v_new).max())

    # Eq. zkUpdate on 12 sampled cliques against the oracle's projection (FP64)
    rng = np.random.default_rng(0)
    for k in rng.choice(len(inst.cliques), size=12, replace=False):
        sdim = len(inst.cliques[k])
        W = orc.ChordalSDP.packed_to_block(v_old[off[k]:off[k + 1]] - rinv * lam_old[off[k]:off[k + 1]], sdim)
        P = orc.proj_psd(W.reshape(sdim, sdim, order="F"))
        got = orc.ChordalSDP.packed_to_block(z[off[k]:off[k + 1]], sdim).reshape(sdim, sdim, order="F")
        assert np.linalg.norm(got - P) <= 1e-10 * max(np.linalg.norm(W), 1e-300)

    # KKT system (Eq. OptCondMinYDual): A x = -b/rho and D x + A^T y = c - sum_k H_k^T(z_k + lam_k/rho)
    w = np.where(maps["pat_row"] != maps["pat_col"], 2.0, 1.0)
    cols = lower_index(maps, inst.n, inst.A_row, inst.A_col)
    rows = np.repeat(np.arange(m), np.diff(inst.A_ptr))
    A = scipy.sparse.csr_matrix((inst.A_val, (rows, cols)), shape=(m, nEL))
    Ax = A @ (w * x)
    np.testing.assert_allclose(Ax, -rinv * inst.b, rtol=0, atol=1e-9 * np.abs(inst.b).max() * rinv)
    D = np.bincount(gidx, minlength=nEL).astype(np.float64)
    cvec = np.zeros(nEL)
    np.add.at(cvec, lower_index(maps, inst.n, inst.C_row, inst.C_col), inst.C_val)
    scat = np.bincount(gidx, weights=z + rinv * lam_old, minlength=nEL)
    r = cvec - scat
    res = D * x + A.T @ y - r
    assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(r)


def test_large_scatter_sampled_bit_exact(large):
    torch, cadmm, inst, s, maps = large
    sz = s.sizes
    rng = np.random.default_rng(1)
    blocks = rng.standard_normal(sz["S_lower"])
    out = torch.empty(sz["nE_lower"], dtype=torch.float64, device="cuda")
    cadmm.sdp_scatter(s.h, torch.tensor(blocks, device="cuda"), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    gidx = maps["gather_idx"]
    order = np.argsort(gidx, kind="stable")           # contributions of each entry, ascending clique
    starts = np.searchsorted(gidx[order], np.arange(sz["nE_lower"] + 1))
    for e in list(rng.choice(sz["nE_lower"], size=200, replace=False)) + [sz["nE_lower"] - 1]:
        acc = 0.0
        for j in range(starts[e], starts[e + 1]):
            acc = blocks[order[j]] if j == starts[e] else acc + blocks[order[j]]
        assert acc == got[e]


def test_large_phase_times(large, capsys):
    torch, cadmm, inst, s, maps = large
    s.set_opts(prec="fp32")
    s.reset()
    ph = cadmm.sdp_time_phases(s.h, reps=5)
    with capsys.disabled():
        print("\nlarge workload phases (ms):", {k: round(v, 3) for k, v in ph.items()})
    assert all(v > 0 for v in ph.values())


def test_large_fp32_projection_sampled(large):
    """The FP32 projection in the launch configuration the bench times at this size (the kernel
    the plan picks for 2000 cliques of order 60, inside the iteration graphs): one warm-started
    iteration after three, 12 sampled cliques against the oracle's FP64 P (Eq. zkUpdate), within
    the FP32 budget of the projection tests (1e-4 of ||W||_F, 4e-4 of max |W_ij| per entry)."""
    torch, cadmm, inst, s, maps = large
    rinv = 1.0 / CONFIGS[3]["rho"]
    s.set_opts(prec="fp32")
    s.reset()
    s.iterate(3)
    st0 = s.state()
    s.iterate(1)
    st1 = s.state()
    z, v_old, lam_old = st1["blk_a"], st0["blk_c"], st0["blk_b"]
    off = maps["blk_off"]
    rng = np.random.default_rng(2)
    for k in rng.choice(len(inst.cliques), size=12, replace=False):
        sdim = len(inst.cliques[k])
        W = orc.ChordalSDP.packed_to_block(v_old[off[k]:off[k + 1]] - rinv * lam_old[off[k]:off[k + 1]], sdim)
        W = W.reshape(sdim, sdim, order="F")
        P = orc.proj_psd(W)
        got = orc.ChordalSDP.packed_to_block(z[off[k]:off[k + 1]], sdim).reshape(sdim, sdim, order="F")
        assert np.linalg.norm(got - P) <= 1e-4 * np.linalg.norm(W), k
        assert np.max(np.abs(got - P)) <= 4e-4 * np.max(np.abs(W)), k
