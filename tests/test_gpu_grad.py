"""GPU reverse mode through unrolled primal ADMM (Algorithm 1) against the CPU reference gradient
(oracle/adjoint.py) and against central finite differences of the GPU forward.

The loss is L = <C, X_T> + ||X_T - X_ref||_F^2 with X_T the affine iterate after T iterations from
zero, differentiated with respect to the lower-triangle values of C and to b. Workload: 64
block-arrow SDPs with l=50, d=10, h=5 (n=505, 50 cliques of 15), m=100, T=200, checkpoints every 20.
"""

import numpy as np
import pytest

from oracle import adjoint as adj
from oracle import chordal_admm as orc
from sdp_inputs import CONFIGS, config_instance
from tests import sdp_cases
from tests.gpu_support import make_oracle, require_gpu

pytestmark = pytest.mark.gpu


def torch_loss(torch, x, c, xr, w):
    d = x - xr
    return torch.sum(w * c * x) + torch.sum(w * d * d)


def gpu_grad(cadmm, torch, handle, c0, b0, xr, T, K):
    from paper_1609_06068_gb300.autograd import lower_weights, unrolled_admm
    w = lower_weights(handle)
    c = torch.tensor(c0, device="cuda", requires_grad=True)
    b = torch.tensor(b0, device="cuda", requires_grad=True)
    x = unrolled_admm(c, b, handle, T, K)
    L = torch_loss(torch, x, c, torch.tensor(xr, device="cuda"), w)
    L.backward()
    return float(L.detach()), c.grad.cpu().numpy(), b.grad.cpu().numpy()


def gpu_loss(cadmm, torch, handle, c0, b0, xr, T, K, ent=None):
    """The loss, or (ent = (e0, e1)) the loss term of the problem owning entries e0..e1-1: the
    problems of a batch are independent, so a coordinate of one problem moves only its own term,
    and differencing that term alone keeps the rounding of the other terms out of the quotient."""
    from paper_1609_06068_gb300.autograd import lower_weights, unrolled_admm
    w = lower_weights(handle)
    with torch.no_grad():
        x = unrolled_admm(torch.tensor(c0, device="cuda"), torch.tensor(b0, device="cuda"), handle, T, K)
        sl = slice(None) if ent is None else slice(int(ent[0]), int(ent[1]))
        return float(torch_loss(torch, x[sl], torch.tensor(c0[sl], device="cuda"),
                                torch.tensor(xr[sl], device="cuda"), w[sl]))


def primal_handle(cadmm, arrs, rho):
    opts = cadmm.make_opts(rho=rho, tol=0.0, max_iter=1, form="primal", prec="fp64")
    return cadmm.ChordalADMM(arrs, opts)


@pytest.mark.parametrize("T,K", [(12, 5), (7, 20)])
def test_small_gradient_matches_oracle(T, K):
    torch, cadmm = require_gpu()
    arrs = sdp_cases.random_block_arrow(l=3, d=3, h=2, m=5, seed=4)
    sdp = make_oracle(arrs)
    rng = np.random.default_rng(9)
    lower = sdp.lower_mask()
    xr = rng.standard_normal(int(lower.sum()))
    x_ref = sdp.from_lower(sdp.E_row[lower], sdp.E_col[lower], xr)
    rho = 0.7
    L0, gc0, gb0, _ = adj.loss_and_grad(sdp, rho, T, x_ref)
    with primal_handle(cadmm, arrs, rho) as s:
        L, gc, gb = gpu_grad(cadmm, torch, s.h, sdp.to_lower(sdp.c), sdp.b, xr, T, K)
    assert abs(L - L0) <= 1e-10 * abs(L0)
    scale = max(np.abs(gc0).max(), np.abs(gb0).max())
    np.testing.assert_allclose(gc, gc0, rtol=0, atol=1e-9 * scale)
    np.testing.assert_allclose(gb, gb0, rtol=0, atol=1e-9 * scale)


@pytest.fixture(scope="module")
def workload4():
    cfg = CONFIGS[4]
    insts = [config_instance(4, i) for i in range(cfg["count"])]
    arrs = [sdp_cases.instance_arrays(x) for x in insts]
    c0 = np.concatenate([x.C_val for x in insts])
    b0 = np.concatenate([x.b for x in insts])
    xr = np.concatenate([x.X0_val for x in insts])
    return cfg, insts, arrs, c0, b0, xr


def test_workload_gradient_matches_oracle_and_differences(workload4, capsys):
    torch, cadmm = require_gpu()
    cfg, insts, arrs, c0, b0, xr = workload4
    T, K, rho = cfg["max_iter"], 20, cfg["rho"]
    import time
    with primal_handle(cadmm, arrs, rho) as s:
        lay = s.batch_layout()
        gpu_grad(cadmm, torch, s.h, c0, b0, xr, T, K)           # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L, gc, gb = gpu_grad(cadmm, torch, s.h, c0, b0, xr, T, K)
        torch.cuda.synchronize()
        t_grad = time.perf_counter() - t0
        t0 = time.perf_counter()
        gpu_loss(cadmm, torch, s.h, c0, b0, xr, T, K)
        torch.cuda.synchronize()
        t_fwd = time.perf_counter() - t0
        # CPU reference gradient on two sampled problems (the losses of the problems add up)
        for q in (0, 37):
            sdp = make_oracle(arrs[q])
            lower = sdp.lower_mask()
            x_ref = sdp.from_lower(sdp.E_row[lower], sdp.E_col[lower], insts[q].X0_val)
            _, gcq, gbq, _ = adj.loss_and_grad(sdp, rho, T, x_ref)
            e0, e1 = lay["ent_off"][q], lay["ent_off"][q + 1]
            r0, r1 = lay["row_off"][q], lay["row_off"][q + 1]
            scale = max(np.abs(gcq).max(), np.abs(gbq).max())
            np.testing.assert_allclose(gc[e0:e1], gcq, rtol=0, atol=1e-7 * scale)
            np.testing.assert_allclose(gb[r0:r1], gbq, rtol=0, atol=1e-7 * scale)
        # central differences of the GPU forward. The loss (|L| about 1e3 per problem) carries
        # FP64 rounding of about 1e-14 relative after 200 iterations, so a quotient at step h errs
        # by about 1e-14 |L| / h: at the step 1e-6 that is 1e-5 absolute, within the 1e-5 bar
        # for the components of the gradient of size 1 and more (the two largest of C and of b
        # are checked); the step 1e-4 keeps it below 1e-7 and is checked on random coordinates.
        rng = np.random.default_rng(11)
        scale = max(np.abs(gc).max(), np.abs(gb).max())
        picks = [(1e-6, "c", int(i)) for i in np.argsort(-np.abs(gc))[:2]] + \
                [(1e-6, "b", int(i)) for i in np.argsort(-np.abs(gb))[:2]] + \
                [(1e-4, "c", int(i)) for i in rng.choice(len(c0), size=4, replace=False)] + \
                [(1e-4, "b", int(i)) for i in rng.choice(len(b0), size=4, replace=False)]
        worst = {}
        for h, kind, i in picks:
            base = c0 if kind == "c" else b0
            g = gc if kind == "c" else gb
            off = lay["ent_off"] if kind == "c" else lay["row_off"]
            q = int(np.searchsorted(off, i, side="right") - 1)
            ent = (lay["ent_off"][q], lay["ent_off"][q + 1])
            p, m = base.copy(), base.copy()
            p[i] += h
            m[i] -= h
            if kind == "c":
                fd = (gpu_loss(cadmm, torch, s.h, p, b0, xr, T, K, ent) -
                      gpu_loss(cadmm, torch, s.h, m, b0, xr, T, K, ent)) / (2 * h)
            else:
                fd = (gpu_loss(cadmm, torch, s.h, c0, p, xr, T, K, ent) -
                      gpu_loss(cadmm, torch, s.h, c0, m, xr, T, K, ent)) / (2 * h)
            err = abs(fd - g[i]) / max(abs(g[i]), 1e-2 * scale)
            worst[h] = max(worst.get(h, 0.0), err)
            assert err <= 1e-5, (kind, i, h, fd, g[i])
    with capsys.disabled():
        print(f"\nunrolled T={T}, 64 problems: loss {L:.6e}, forward {t_fwd * 1e3:.1f} ms, forward+backward "
              f"{t_grad * 1e3:.1f} ms, worst finite-difference disagreement at step 1e-6 {worst[1e-6]:.2e}, "
              f"at 1e-4 {worst[1e-4]:.2e}")


@pytest.mark.parametrize("T,K", [(12, 5)])
def test_gradient_with_cones_matches_oracle(T, K):
    """Reverse mode through a problem with free, nonnegative and second-order variables (small
    and large second-order cones) against the oracle's reference gradient."""
    torch, cadmm = require_gpu()
    arrs = sdp_cases.random_conic(l=2, d=3, h=2, n_free=2, n_lin=5, soc_dims=(3, 1, 300), m=6, seed=41,
                                  soc_u_scale=5.0)
    sdp = make_oracle(arrs)
    rng = np.random.default_rng(17)
    lower = sdp.lower_mask()
    xr = rng.standard_normal(int(lower.sum()))
    x_ref = sdp.from_lower(sdp.E_row[lower], sdp.E_col[lower], xr)
    rho = 0.8
    # the second-order cones' nontrivial branch (||u|| > |t|: the point is in neither the cone nor
    # its polar) is reached by a small cone and by the large one at some forward iterate
    st = orc.admm_init(sdp, "primal")
    outside = set()
    for _ in range(T):
        nxt = orc.primal_iteration(sdp, st, rho)
        for k in range(sdp.p, sdp.nblk):
            if sdp.kinds[k] != "soc":
                continue
            w = nxt["u"][k] - st["lam"][k] / rho
            if np.linalg.norm(w[1:]) > abs(w[0]):
                outside.add(len(w))
        st = nxt
    assert 300 in outside and 3 in outside, outside     # large-cone (one CTA) and small-cone (one thread) paths
    L0, gc0, gb0, _ = adj.loss_and_grad(sdp, rho, T, x_ref)
    with primal_handle(cadmm, arrs, rho) as s:
        L, gc, gb = gpu_grad(cadmm, torch, s.h, sdp.to_lower(sdp.c), sdp.b, xr, T, K)
    assert abs(L - L0) <= 1e-10 * abs(L0)
    scale = max(np.abs(gc0).max(), np.abs(gb0).max())
    np.testing.assert_allclose(gc, gc0, rtol=0, atol=1e-9 * scale)
    np.testing.assert_allclose(gb, gb0, rtol=0, atol=1e-9 * scale)
