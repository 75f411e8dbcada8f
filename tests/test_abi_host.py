"""CPU checks of the C ABI: the library builds and loads, exports every function the header
declares, and its host-side validation rejects bad input before touching a GPU."""

import ctypes
import os
import re

import numpy as np
import pytest

import paper_1609_06068_gb300 as cadmm
from paper_1609_06068_gb300 import build as cbuild
from tests import sdp_cases

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "chordal_admm.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(cadmm.LIB_PATH):
        cbuild.build()
    return cadmm.load_library()


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("defined",)))


def test_header_declares_the_binding_names():
    assert header_functions() == sorted(cadmm.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7):
        assert cadmm.sdp_status_string(code) != "unknown status"
    assert cadmm.sdp_status_string(42) == "unknown status"


def _arrays():
    return sdp_cases.random_block_arrow(l=3, d=2, h=2, m=4)


def _setup_rc(arrs, opts=None, cliques=None):
    """Call sdp_setup directly and return (rc, handle); only host validation may run."""
    lib = cadmm.load_library()
    cl = cliques if cliques is not None else arrs["cliques"]
    sizes = np.array([len(c) for c in cl])
    ptr = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    vtx = np.concatenate(cl).astype(np.int32)
    A_ptr = np.asarray(arrs["A_ptr"], np.int64)
    A_row = np.asarray(arrs["A_row"], np.int32); A_col = np.asarray(arrs["A_col"], np.int32)
    A_val = np.asarray(arrs["A_val"], np.float64); b = np.asarray(arrs["b"], np.float64)
    C_row = np.asarray(arrs["C_row"], np.int32); C_col = np.asarray(arrs["C_col"], np.int32)
    C_val = np.asarray(arrs["C_val"], np.float64)
    o = opts if opts is not None else cadmm.make_opts()
    h = ctypes.c_void_p()
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    rc = lib.sdp_setup(arrs["n"], len(b), P(A_ptr), P(A_row), P(A_col), P(A_val), P(b),
                       len(C_val), P(C_row), P(C_col), P(C_val), 0, None, None,
                       len(cl), P(ptr), P(vtx), ctypes.byref(o), ctypes.byref(h))
    return rc, h


def test_setup_rejects_bad_options(lib):
    arrs = _arrays()
    assert _setup_rc(arrs, opts=cadmm.make_opts(rho=0.0))[0] == cadmm.SDP_ERR_ARG
    assert _setup_rc(arrs, opts=cadmm.make_opts(rho=-1.0))[0] == cadmm.SDP_ERR_ARG
    assert _setup_rc(arrs, opts=cadmm.make_opts(form=7))[0] == cadmm.SDP_ERR_ARG
    assert _setup_rc(arrs, opts=cadmm.make_opts(prec=3))[0] == cadmm.SDP_ERR_ARG
    assert _setup_rc(arrs, opts=cadmm.make_opts(max_iter=-1))[0] == cadmm.SDP_ERR_ARG


def test_setup_rejects_bad_cliques(lib):
    arrs = _arrays()
    rc, _ = _setup_rc(arrs, cliques=[c[::-1] for c in arrs["cliques"]])
    assert rc == cadmm.SDP_ERR_CLIQUE and "ascending" in cadmm.sdp_last_error()
    rc, _ = _setup_rc(arrs, cliques=arrs["cliques"][:-1])
    assert rc == cadmm.SDP_ERR_CLIQUE and "not covered" in cadmm.sdp_last_error()
    big = [np.arange(cadmm.SDP_MAX_CLIQUE + 1, dtype=np.int32)]
    arrs_big = dict(arrs, n=cadmm.SDP_MAX_CLIQUE + 1)
    assert _setup_rc(arrs_big, cliques=big)[0] == cadmm.SDP_ERR_UNSUPPORTED


def test_setup_rejects_rank_deficient_A(lib):
    arrs = _arrays()
    k0 = int(arrs["A_ptr"][1])
    bad = dict(arrs)
    bad["A_ptr"] = np.concatenate([arrs["A_ptr"], [arrs["A_ptr"][-1] + k0]])
    bad["A_row"] = np.concatenate([arrs["A_row"], arrs["A_row"][:k0]])
    bad["A_col"] = np.concatenate([arrs["A_col"], arrs["A_col"][:k0]])
    bad["A_val"] = np.concatenate([arrs["A_val"], arrs["A_val"][:k0]])
    bad["b"] = np.concatenate([arrs["b"], arrs["b"][:1]])
    assert _setup_rc(bad)[0] == cadmm.SDP_ERR_NOT_PD


def test_setup_rejects_upper_coordinates(lib):
    arrs = _arrays()
    bad = dict(arrs)
    bad["C_row"], bad["C_col"] = arrs["C_col"], arrs["C_row"]
    off = np.asarray(arrs["C_row"]) != np.asarray(arrs["C_col"])
    assert off.any()
    assert _setup_rc(bad)[0] == cadmm.SDP_ERR_ARG


def test_project_batched_validates_on_host(lib):
    f = lib.project_psd_batched
    sizes = np.array([3, 0], np.int32)
    offs = np.array([0, 6], np.int64)
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    dummy = ctypes.c_void_p(16)   # never dereferenced: validation fails first
    assert f(dummy, dummy, P(sizes), P(offs), 2, 0, None) == cadmm.SDP_ERR_ARG
    sizes = np.array([cadmm.SDP_MAX_CLIQUE + 1], np.int32)
    assert f(dummy, dummy, P(sizes), P(offs[:1]), 1, 0, None) == cadmm.SDP_ERR_UNSUPPORTED
    assert f(dummy, dummy, P(sizes), P(offs[:1]), 1, 5, None) == cadmm.SDP_ERR_ARG
    assert f(None, None, None, None, 0, 0, None) == cadmm.SDP_OK


def test_chordal_extension_matches_oracle():
    """The library's chordal extension (host code, no GPU) gives exactly the oracle's cliques."""
    import numpy as np
    from oracle import chordal as ch
    from sdp_inputs import config_instance
    cadmm = pytest.importorskip("paper_1609_06068_gb300")
    cadmm.load_library()
    rng = np.random.default_rng(3)
    cases = []
    inst = config_instance(1)
    cases.append((inst.n, inst.pat_row, inst.pat_col))
    for _ in range(30):
        n = int(rng.integers(1, 60))
        rows, cols = np.tril_indices(n, -1)
        keep = rng.random(len(rows)) < rng.uniform(0.01, 0.3)
        cases.append((n, rows[keep], cols[keep]))
    n = 17
    cyc = np.arange(n)
    cases.append((n, np.maximum(cyc, (cyc + 1) % n), np.minimum(cyc, (cyc + 1) % n)))
    for n, rows, cols in cases:
        got, gfill = cadmm.sdp_chordal_cliques(n, rows, cols)
        want, wfill = ch.chordal_extension(n, rows, cols)
        assert gfill == wfill
        assert [list(map(int, c)) for c in got] == [list(c) for c in want]


def _conic_rc(arrs, **cone_changes):
    cones = dict(arrs["cones"], **cone_changes)
    try:
        cadmm.sdp_setup_conic(arrs, cones, cadmm.make_opts())
    except cadmm.SDPError as exc:
        return exc.code, str(exc)
    return cadmm.SDP_OK, ""


def test_setup_conic_validates_cones_on_host(lib):
    arrs = sdp_cases.random_conic(l=2, d=2, h=1, n_free=2, n_lin=3, soc_dims=(3,), m=4, seed=5)
    assert _conic_rc(arrs, n_free=-1)[0] == cadmm.SDP_ERR_ARG
    rc, msg = _conic_rc(arrs, soc_dims=[0])
    assert rc == cadmm.SDP_ERR_ARG and "dimension" in msg
    bad_var = np.array(arrs["cones"]["A_var"])
    bad_var[0] = 2 + 3 + 3
    rc, msg = _conic_rc(arrs, A_var=bad_var)
    assert rc == cadmm.SDP_ERR_ARG and "out of range" in msg
    bad_ptr = np.array(arrs["cones"]["A_ptr"])
    bad_ptr[0] = 1
    assert _conic_rc(arrs, A_ptr=bad_ptr)[0] == cadmm.SDP_ERR_ARG
    # no PSD part and no cone variables at all
    empty = sdp_cases._empty_matrix_part()
    empty.update(A_ptr=np.zeros(2, np.int64), b=np.ones(1))
    empty["cones"] = sdp_cases.cones_from_dense(np.zeros((1, 0)), np.zeros(0))
    assert _conic_rc(empty)[0] == cadmm.SDP_ERR_ARG


def test_concurrent_setups_share_the_worker_pool(lib):
    """Host setup runs its loops on a process-wide worker pool; a second caller while the pool is
    busy runs on threads of its own. Concurrent setups (here stopped by the missing GPU after the
    host build, or completed where a GPU exists) must all return, with the same outcome as a
    serial one."""
    import threading
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("checks the host path up to the first CUDA call")
    arrs = sdp_cases.instance_arrays(__import__("sdp_inputs").config_instance(0))

    def outcome():
        try:
            cadmm.ChordalADMM(arrs, cadmm.make_opts())
            return "ok"
        except cadmm.SDPError as exc:
            return exc.code
    serial = outcome()
    results = [None] * 6
    threads = [threading.Thread(target=lambda i=i: results.__setitem__(i, outcome())) for i in range(6)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=120)
    assert not any(t.is_alive() for t in threads)
    assert results == [serial] * 6 and serial == cadmm.SDP_ERR_CUDA


def test_handle_calls_reject_null_on_host(lib):
    P = ctypes.c_void_p
    buf = (ctypes.c_int * 4)()
    assert lib.sdp_proj_sweeps(None, buf) == cadmm.SDP_ERR_ARG
    assert lib.sdp_get_sizes(None, None) == cadmm.SDP_ERR_ARG
    assert lib.sdp_setup_conic(None, None, None, ctypes.byref(P())) == cadmm.SDP_ERR_ARG


def _fork_child(q):
    arrs = sdp_cases.instance_arrays(__import__("sdp_inputs").config_instance(0))
    try:
        cadmm.ChordalADMM(arrs, cadmm.make_opts())
        q.put("ok")
    except cadmm.SDPError as exc:
        q.put(exc.code)


@pytest.mark.filterwarnings("ignore::DeprecationWarning")      # fork of a threaded process is the case tested
def test_forked_child_builds_and_exits_cleanly(lib):
    """A process forked after the worker pool started (the pool's threads do not exist in it) runs
    the host build on threads of its own and exits normally."""
    import multiprocessing as mp
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("forking after CUDA initialisation is not supported")
    arrs = sdp_cases.instance_arrays(__import__("sdp_inputs").config_instance(0))
    with pytest.raises(cadmm.SDPError):
        cadmm.ChordalADMM(arrs, cadmm.make_opts())          # starts the pool in this process
    ctx = mp.get_context("fork")
    q = ctx.Queue()
    p = ctx.Process(target=_fork_child, args=(q,))
    p.start()
    p.join(timeout=120)
    assert p.exitcode == 0
    assert q.get(timeout=5) == cadmm.SDP_ERR_CUDA


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes structs of the binding have the C header's sizes and field offsets (a mismatch
    would pass garbage through the ABI silently). gcc compiles a probe that prints them."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    structs = {"admm_opts": cadmm.admm_opts, "admm_result": cadmm.admm_result, "sdp_sizes": cadmm.sdp_sizes,
               "sdp_problem": cadmm.sdp_problem, "sdp_cones": cadmm.sdp_cones}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "chordal_admm.h"', 'int main(void) {']
    for name, cls in structs.items():
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ['    return 0;', '}']
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c_layout = {}
    for line in out:
        if line:
            name, field, value = line.split()
            c_layout[(name, field)] = int(value)
    for name, cls in structs.items():
        assert c_layout[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert c_layout[(name, field)] == getattr(cls, field).offset, (name, field)


def _oracle_of(arrs):
    from tests.gpu_support import make_oracle
    return make_oracle(arrs)


@pytest.mark.parametrize("name", ["config0", "block_arrow", "conic", "pure_cones", "theta", "non_chordal"])
def test_plan_sizes_match_the_oracle(lib, name):
    """sdp_plan (the host build alone, no GPU) against the oracle's representation: lower pattern
    entries (cone variables included), packed positions, cliques, largest clique and the stored
    nonzeros of A on the lower pattern after duplicates merge."""
    from oracle import chordal as och
    if name == "config0":
        arrs = sdp_cases.instance_arrays(__import__("sdp_inputs").config_instance(0))
    elif name == "block_arrow":
        arrs = sdp_cases.random_block_arrow(l=4, d=3, h=2, m=6, seed=2)
    elif name == "conic":
        arrs = sdp_cases.random_conic(l=2, d=3, h=2, n_free=2, n_lin=4, soc_dims=(3, 1, 40), m=6, seed=21)
    elif name == "pure_cones":
        arrs = sdp_cases.random_conic(l=0, n_free=2, n_lin=7, soc_dims=(4, 2), m=5, seed=22)
    elif name == "theta":
        arrs = sdp_cases.theta_c5()[0]
    else:
        arrs = sdp_cases.random_sparse_sdp(n=24, m=8, seed=5)
        rows = np.concatenate([arrs["A_row"], arrs["C_row"]])
        cols = np.concatenate([arrs["A_col"], arrs["C_col"]])
        cliques, _ = och.chordal_extension(arrs["n"], rows, cols)
        ref_arrs = dict(arrs, cliques=[np.array(c, np.int32) for c in cliques])
    sz = cadmm.sdp_plan(arrs, arrs.get("cones"))
    sdp = _oracle_of(ref_arrs if name == "non_chordal" else arrs)
    lower = sdp.lower_mask()
    assert sz["p"] == sdp.p and sz["n_cone"] == sdp.n_cone and sz["batch"] == 1
    assert sz["nE_lower"] == int(lower.sum())
    assert sz["S_lower"] == sum(len(c) * (len(c) + 1) // 2 for c in sdp.cliques) + sdp.n_cone
    assert sz["max_clique"] == max([len(c) for c in sdp.cliques], default=0)
    assert sz["nnz_A"] == int((sdp.A[:, np.flatnonzero(lower)] != 0).sum())


def test_plan_reports_host_errors(lib):
    arrs = sdp_cases.random_block_arrow(l=3, d=2, h=2, m=4)
    bad = dict(arrs)
    bad["b"] = np.concatenate([arrs["b"], arrs["b"][:1]])
    bad["A_ptr"] = np.concatenate([arrs["A_ptr"], arrs["A_ptr"][-1:] + 0])    # an empty constraint
    with pytest.raises(cadmm.SDPError) as exc:
        cadmm.sdp_plan(bad)
    assert exc.value.code == cadmm.SDP_ERR_NOT_PD
    with pytest.raises(cadmm.SDPError) as exc:
        cadmm.sdp_plan(dict(arrs, cliques=[np.array([1, 0], np.int32)]))
    assert exc.value.code == cadmm.SDP_ERR_CLIQUE


@pytest.mark.parametrize("case", ["short", "long"])
def test_plan_merges_untidy_constraints(lib, case):
    """Shuffled entries, split duplicates, explicit zeros and a cancelling pair leave the host
    build's count of stored nonzeros of A unchanged. "long" has constraints of more than 512
    entries, which take the radix-sort path; "short" the comparison sort."""
    if case == "short":
        arrs = sdp_cases.random_block_arrow(l=4, d=3, h=2, m=6, seed=2)
    else:
        arrs = sdp_cases.random_block_arrow(l=30, d=5, h=4, m=8, seed=4, density=0.6)
        assert np.min(np.diff(arrs["A_ptr"])) > 512
    tidy = cadmm.sdp_plan(arrs)
    messy = cadmm.sdp_plan(sdp_cases.messy_constraints(arrs))
    assert messy == tidy
