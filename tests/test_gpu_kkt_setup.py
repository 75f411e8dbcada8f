"""The cached KKT factorization of the affine step (Section III.B.1: block elimination with the
factor of A D⁻¹ Aᵀ) built on the device, against the same factorization built on the host
(SDP_FLAG_HOST_KKT) and against the oracle.

From m = 64 constraints the setup forms M = A D⁻¹ Aᵀ, its Cholesky factor, L⁻¹ and M⁻¹ on the
GPU in FP64. The two builds add the same products in different orders, so M differs by
rounding (about m ε relative) and the iterates by κ(M) times that: 1e-11 here, where κ is
below 1e3. Rank-deficient A must be refused the same way, and an ill-conditioned M must switch
the affine step to the triangular factors in both builds."""

import numpy as np
import pytest

from oracle import chordal_admm as orc
from tests import sdp_cases
from tests.gpu_support import make_oracle, oracle_state_to_abi, rel_err, require_gpu, setup_handle

pytestmark = pytest.mark.gpu


def step(form):
    return orc.primal_iteration if form == "primal" else orc.dual_iteration


def phases(cadmm, s):
    return [cadmm.sdp_phase_name(s.h, i) for i in range(8)]


@pytest.mark.parametrize("form", ["primal", "dual"])
@pytest.mark.parametrize("m", [64, 150])
def test_device_kkt_matches_host_and_oracle(form, m):
    torch, cadmm = require_gpu()
    arrs = sdp_cases.random_block_arrow(l=12, d=5, h=4, m=m, seed=31 + m, density=0.4)
    sdp = make_oracle(arrs)
    assert np.linalg.cond(sdp.M) < 1e3
    st = orc.admm_init(sdp, form)
    with setup_handle(cadmm, arrs, form=form, rho=0.5, tol=0.0) as dev, \
            setup_handle(cadmm, arrs, form=form, rho=0.5, tol=0.0, flags=cadmm.SDP_FLAG_HOST_KKT) as host:
        assert "solve_y" in phases(cadmm, dev) and "solve_y" in phases(cadmm, host)
        for it in range(25):
            st = step(form)(sdp, st, 0.5)
            dev.iterate(1)
            host.iterate(1)
            a, b = dev.state(), host.state()
            ref = oracle_state_to_abi(sdp, st)
            for key in ref:
                # the first iteration from zero is one affine step through M^-1: it carries the
                # difference of the two builds of M^-1 alone
                bound = 1e-12 if it == 0 else 1e-11
                assert rel_err(a[key], b[key]) <= bound, (it, key, rel_err(a[key], b[key]))
                assert rel_err(a[key], ref[key]) <= 1e-10, (it, key, rel_err(a[key], ref[key]))


def test_device_kkt_solve_matches_host():
    """A whole solve to 1e-5: the same iteration count and objectives to 1e-9."""
    torch, cadmm = require_gpu()
    arrs = sdp_cases.random_block_arrow(l=12, d=5, h=4, m=100, seed=5, density=0.4)
    out = []
    for flags in (0, cadmm.SDP_FLAG_HOST_KKT):
        with setup_handle(cadmm, arrs, form="dual", rho=1.0, tol=1e-5, max_iter=5000, flags=flags) as s:
            out.append(s.solve())
    a, b = out
    assert a["status"] == b["status"] == cadmm.SDP_OK
    assert abs(a["iters"] - b["iters"]) <= 1, (a["iters"], b["iters"])
    for key in ("obj_primal", "obj_dual"):
        assert abs(a[key] - b[key]) <= 1e-9 * max(1.0, abs(b[key])), (key, a[key], b[key])


@pytest.mark.parametrize("flags", [0, 1])
def test_device_kkt_refuses_dependent_rows(flags):
    """A constraint listed twice makes A D⁻¹ Aᵀ singular: the setup reports SDP_ERR_NOT_PD."""
    torch, cadmm = require_gpu()
    arrs = sdp_cases.random_block_arrow(l=12, d=5, h=4, m=80, seed=8, density=0.4)
    m = len(arrs["b"])
    # append row 3 of A (and b_3) as row m
    A_ptr, A_row, A_col, A_val = (np.asarray(arrs[k]) for k in ("A_ptr", "A_row", "A_col", "A_val"))
    lo, hi = int(A_ptr[3]), int(A_ptr[4])
    arrs = dict(arrs)
    arrs["A_ptr"] = np.concatenate([A_ptr, [A_ptr[-1] + (hi - lo)]]).astype(A_ptr.dtype)
    arrs["A_row"] = np.concatenate([A_row, A_row[lo:hi]]).astype(A_row.dtype)
    arrs["A_col"] = np.concatenate([A_col, A_col[lo:hi]]).astype(A_col.dtype)
    arrs["A_val"] = np.concatenate([A_val, A_val[lo:hi]]).astype(A_val.dtype)
    arrs["b"] = np.concatenate([np.asarray(arrs["b"]), [np.asarray(arrs["b"])[3]]])
    with pytest.raises(cadmm.SDPError) as e:
        setup_handle(cadmm, arrs, form="primal", flags=flags * cadmm.SDP_FLAG_HOST_KKT)
    assert e.value.code == cadmm.SDP_ERR_NOT_PD


@pytest.mark.parametrize("form", ["primal", "dual"])
def test_device_kkt_ill_conditioned_takes_factors(form):
    """Two nearly dependent constraints (κ(M) about 3e8): both builds take the two triangular
    factors, and the device build's iterates stay within a κ-scaled bound of the oracle's and
    of the host build's."""
    torch, cadmm = require_gpu()
    arrs = sdp_cases.near_dependent_block_arrow(l=12, d=5, h=4, m=80, delta=1e-4, seed=23)
    sdp = make_oracle(arrs)
    kappa = float(np.linalg.cond(sdp.M))
    assert 1e5 <= kappa <= 1e10, kappa
    bound = max(1e-9, kappa * 5e-16)
    st = orc.admm_init(sdp, form)
    with setup_handle(cadmm, arrs, form=form, rho=1.0, tol=0.0) as dev, \
            setup_handle(cadmm, arrs, form=form, rho=1.0, tol=0.0, flags=cadmm.SDP_FLAG_HOST_KKT) as host:
        for s in (dev, host):
            names = phases(cadmm, s)
            assert "tri_lower" in names and "tri_upper" in names and "solve_y" not in names, names
        for it in range(20):
            st = step(form)(sdp, st, 1.0)
            dev.iterate(1)
            host.iterate(1)
            a, b = dev.state(), host.state()
            ref = oracle_state_to_abi(sdp, st)
            for key in ref:
                if key == "y":
                    # y is fixed only to about κ ε along the near-null direction of Aᵀ
                    ea = rel_err(sdp.A.T @ a["y"], sdp.A.T @ ref["y"])
                    eb = rel_err(sdp.A.T @ a["y"], sdp.A.T @ b["y"])
                else:
                    ea, eb = rel_err(a[key], ref[key]), rel_err(a[key], b[key])
                assert ea <= bound and eb <= bound, (it, key, ea, eb, bound)
        rows, cols = sdp.E_row[sdp.lower_mask()], sdp.E_col[sdp.lower_mask()]
        x = sdp.from_lower(rows, cols, dev.state()["x"])
        rhs = sdp.b if form == "primal" else -sdp.b / 1.0
        assert np.max(np.abs(sdp.A @ x - rhs)) <= 1e-10 * max(1.0, np.max(np.abs(rhs)))


@pytest.mark.parametrize("flags", [0, 1])
def test_untidy_constraints_give_identical_iterates(flags):
    """Shuffled entries, split duplicates, explicit zeros and a cancelling pair in A: after the
    host build merges them (and, without SDP_FLAG_HOST_KKT, the device builds the A^T slices
    and the factorization from that CSR), the iterates are bit for bit those of the tidy input."""
    torch, cadmm = require_gpu()
    arrs = sdp_cases.random_block_arrow(l=30, d=5, h=4, m=70, seed=9, density=0.6)
    messy = sdp_cases.messy_constraints(arrs, seed=5)
    fl = flags * cadmm.SDP_FLAG_HOST_KKT
    with setup_handle(cadmm, arrs, form="dual", rho=0.5, tol=0.0, flags=fl) as a, \
            setup_handle(cadmm, messy, form="dual", rho=0.5, tol=0.0, flags=fl) as b:
        a.iterate(15)
        b.iterate(15)
        sa, sb = a.state(), b.state()
        for key in sa:
            assert np.array_equal(sa[key], sb[key]), key


@pytest.mark.parametrize("m,density", [(300, 0.4), (450, 0.9)])
def test_device_kkt_global_partials_match_host(m, density):
    """From m = 240 the partial sums of A D^-1 A^T no longer fit in shared memory and go to global
    memory in row bands: m = 300 with short columns stages whole slices, m = 450 with columns of
    about 400 entries stages one column at a time. The first iteration (one affine step through
    M^-1) agrees with the host build to 1e-12, later iterates to 1e-11, and with the oracle to
    1e-10."""
    torch, cadmm = require_gpu()
    arrs = sdp_cases.random_block_arrow(l=30, d=6, h=4, m=m, seed=41 + m, density=density)
    sdp = make_oracle(arrs)
    assert np.linalg.cond(sdp.M) < 1e4
    st = orc.admm_init(sdp, "dual")
    with setup_handle(cadmm, arrs, form="dual", rho=0.3, tol=0.0) as dev, \
            setup_handle(cadmm, arrs, form="dual", rho=0.3, tol=0.0, flags=cadmm.SDP_FLAG_HOST_KKT) as host:
        for it in range(6):
            st = orc.dual_iteration(sdp, st, 0.3)
            dev.iterate(1)
            host.iterate(1)
            a, b = dev.state(), host.state()
            ref = oracle_state_to_abi(sdp, st)
            for key in ref:
                bound = 1e-12 if it == 0 else 1e-11
                assert rel_err(a[key], b[key]) <= bound, (it, key, rel_err(a[key], b[key]))
                assert rel_err(a[key], ref[key]) <= 1e-10, (it, key, rel_err(a[key], ref[key]))


def test_setup_times_report_the_stages():
    """sdp_setup_times: five named stages, none negative, adding up to no more than the setup
    call's wall time; the device stage is zero when the host builds the factorization."""
    import time
    torch, cadmm = require_gpu()
    arrs = sdp_cases.random_block_arrow(l=12, d=5, h=4, m=80, seed=3, density=0.4)
    for flags in (0, cadmm.SDP_FLAG_HOST_KKT):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = setup_handle(cadmm, arrs, form="dual", flags=flags)
        wall_ms = 1e3 * (time.perf_counter() - t0)
        try:
            st = cadmm.sdp_setup_times(s.h)
        finally:
            s.close()
        assert list(st) == ["host_build", "plan", "alloc_upload", "device_kkt", "finish"]
        assert all(v >= 0.0 for v in st.values())
        assert sum(st.values()) <= wall_ms + 0.5, (st, wall_ms)
        if flags:
            assert st["device_kkt"] == 0.0
        else:
            assert st["device_kkt"] > 0.0
    assert cadmm.load_library().sdp_setup_stage_name(5) is None
