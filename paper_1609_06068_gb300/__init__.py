"""GB300 (sm_103a) hot path of chordally decomposed ADMM for sparse SDPs.

Python binding of the C ABI declared in ``include/chordal_admm.h``. Every function here has the
name of a C entry point and only marshals arguments (NumPy arrays for host data, ``torch`` CUDA
tensors for device buffers, ``torch``'s current stream by default). All computation runs in the
CUDA library ``lib/libchordal_admm.so``; when it is missing, the first call raises.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libchordal_admm.so")

SDP_OK = 0
SDP_MAX_ITER = 1
SDP_ERR_ARG = -1
SDP_ERR_CLIQUE = -2
SDP_ERR_NOT_PD = -3
SDP_ERR_CUDA = -4
SDP_ERR_NAN = -5
SDP_ERR_TIMEOUT = -6
SDP_ERR_UNSUPPORTED = -7
SDP_MAX_CLIQUE = 96
SDP_MAX_CONSTRAINTS = 16384

SDP_PRIMAL = 0
SDP_DUAL = 1
SDP_PROJ_FP64 = 0
SDP_PROJ_FP32 = 1

FORMS = {"primal": SDP_PRIMAL, "dual": SDP_DUAL}
PRECS = {"fp64": SDP_PROJ_FP64, "fp32": SDP_PROJ_FP32}

# Symbols the header declares (checked by the CPU test suite against the built library).
EXPORTS = [
    "sdp_setup", "sdp_setup_batch", "sdp_setup_conic", "sdp_batch_layout", "sdp_batch_results", "sdp_set_opts", "admm_reset", "admm_iterate", "admm_solve", "sdp_get_sizes",
    "sdp_get_solution", "sdp_get_state", "sdp_set_state", "sdp_get_maps", "sdp_gather",
    "sdp_scatter", "project_psd_batched", "sdp_time_phases", "sdp_phase_name",
    "sdp_setup_times", "sdp_setup_stage_name",
    "project_psd_batched_noalloc", "project_variant_count", "project_variant_name",
    "project_variant_fits", "project_psd_batched_variant", "sdp_set_proj_table", "sdp_set_cost",
    "sdp_set_rhs", "sdp_unrolled_forward", "sdp_unrolled_backward", "sdp_chordal_cliques", "sdp_proj_sweeps", "sdp_plan", "sdp_free",
    "sdp_status_string", "sdp_last_error",
]
SDP_NOALLOC_MAX_BLOCKS = 32768
SDP_FLAG_HOST_KKT = 1


class SDPError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {msg} (status {code})")
        self.code = code


class admm_opts(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("check_every", ctypes.c_int), ("form", ctypes.c_int), ("prec", ctypes.c_int),
                ("flags", ctypes.c_int)]


class admm_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("eps_p", ctypes.c_double),
                ("eps_d", ctypes.c_double), ("obj_primal", ctypes.c_double),
                ("obj_dual", ctypes.c_double), ("seconds", ctypes.c_double),
                ("kernel_launches", ctypes.c_longlong)]


class sdp_sizes(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("m", ctypes.c_int), ("p", ctypes.c_int),
                ("max_clique", ctypes.c_int), ("nE_lower", ctypes.c_longlong),
                ("S_lower", ctypes.c_longlong), ("nnz_A", ctypes.c_longlong), ("batch", ctypes.c_int),
                ("n_cone", ctypes.c_longlong)]


class sdp_cones(ctypes.Structure):
    _fields_ = [("n_free", ctypes.c_int), ("n_lin", ctypes.c_int), ("n_soc", ctypes.c_int),
                ("soc_dims", ctypes.c_void_p), ("A_ptr", ctypes.c_void_p), ("A_var", ctypes.c_void_p),
                ("A_val", ctypes.c_void_p), ("c", ctypes.c_void_p)]


class sdp_problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("m", ctypes.c_int), ("A_ptr", ctypes.c_void_p),
                ("A_row", ctypes.c_void_p), ("A_col", ctypes.c_void_p), ("A_val", ctypes.c_void_p),
                ("b", ctypes.c_void_p), ("C_nnz", ctypes.c_longlong), ("C_row", ctypes.c_void_p),
                ("C_col", ctypes.c_void_p), ("C_val", ctypes.c_void_p), ("pat_nnz", ctypes.c_longlong),
                ("pat_row", ctypes.c_void_p), ("pat_col", ctypes.c_void_p), ("p", ctypes.c_int),
                ("clique_ptr", ctypes.c_void_p), ("clique_vtx", ctypes.c_void_p)]


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_LL = ctypes.c_longlong


def load_library(path: str = LIB_PATH):
    """Load the CUDA library (once). Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing "
                           "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
    lib = ctypes.CDLL(path)
    sig = {
        "sdp_setup": (_I, [_I, _I, _P, _P, _P, _P, _P, _LL, _P, _P, _P, _LL, _P, _P, _I, _P, _P,
                           ctypes.POINTER(admm_opts), ctypes.POINTER(_P)]),
        "sdp_setup_batch": (_I, [_I, ctypes.POINTER(sdp_problem), ctypes.POINTER(admm_opts), ctypes.POINTER(_P)]),
        "sdp_setup_conic": (_I, [ctypes.POINTER(sdp_problem), ctypes.POINTER(sdp_cones), ctypes.POINTER(admm_opts),
                                 ctypes.POINTER(_P)]),
        "sdp_batch_layout": (_I, [_P, _P, _P, _P, _P, _P]),
        "sdp_batch_results": (_I, [_P, _P, _P, _P, _P, _P, _P]),
        "sdp_set_opts": (_I, [_P, ctypes.POINTER(admm_opts)]),
        "admm_reset": (_I, [_P, _P]),
        "admm_iterate": (_I, [_P, _I, _P, ctypes.POINTER(admm_result)]),
        "admm_solve": (_I, [_P, _P, ctypes.POINTER(admm_result)]),
        "sdp_get_sizes": (_I, [_P, ctypes.POINTER(sdp_sizes)]),
        "sdp_get_solution": (_I, [_P, _P, _P, _P]),
        "sdp_get_state": (_I, [_P, _P, _P, _P, _P, _P]),
        "sdp_set_state": (_I, [_P, _P, _P, _P, _P, _P]),
        "sdp_get_maps": (_I, [_P, _P, _P, _P, _P]),
        "sdp_gather": (_I, [_P, _P, _P, _P]),
        "sdp_scatter": (_I, [_P, _P, _P, _P]),
        "project_psd_batched": (_I, [_P, _P, _P, _P, _I, _I, _P]),
        "sdp_time_phases": (_I, [_P, _I, _P, _P, _I]),
        "sdp_phase_name": (ctypes.c_char_p, [_P, _I]),
        "sdp_setup_times": (_I, [_P, _P, _I]),
        "sdp_setup_stage_name": (ctypes.c_char_p, [_I]),
        "project_psd_batched_noalloc": (_I, [_P, _P, _P, _P, _I, _I, _P]),
        "project_variant_count": (_I, []),
        "project_variant_name": (ctypes.c_char_p, [_I]),
        "project_variant_fits": (_I, [_I, _I, _I]),
        "project_psd_batched_variant": (_I, [_P, _P, _P, _P, _I, _I, _I, _P]),
        "sdp_set_proj_table": (_I, [_P, _I, _P, _I]),
        "sdp_chordal_cliques": (_I, [_I, _LL, _P, _P, _P, _P, _P, _P, _P, _I, _LL]),
        "sdp_set_cost": (_I, [_P, _P, _P]),
        "sdp_set_rhs": (_I, [_P, _P, _P]),
        "sdp_proj_sweeps": (_I, [_P, _P]),
        "sdp_plan": (_I, [ctypes.POINTER(sdp_problem), ctypes.POINTER(sdp_cones), ctypes.POINTER(sdp_sizes)]),
        "sdp_unrolled_forward": (_I, [_P, _I, _I, _P, _P]),
        "sdp_unrolled_backward": (_I, [_P, _P, _P, _P, _P]),
        "sdp_free": (None, [_P]),
        "sdp_status_string": (ctypes.c_char_p, [_I]),
        "sdp_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, where: str, ok=(SDP_OK,)) -> int:
    if rc in ok:
        return rc
    lib = load_library()
    msg = lib.sdp_last_error().decode() or lib.sdp_status_string(rc).decode()
    raise SDPError(rc, where, msg)


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _arr(a, dtype):
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


def _stream(stream):
    """cudaStream_t of ``stream`` (a torch.cuda.Stream, an int handle, or None = torch current)."""
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, n: int | None = None, name: str = "tensor"):
    """Device pointer of a contiguous float64 CUDA tensor."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    if n is not None and t.numel() < n:
        raise ValueError(f"{name} needs at least {n} elements")
    return ctypes.c_void_p(t.data_ptr())


def make_opts(rho=1.0, tol=1e-4, max_iter=2000, check_every=16, form="primal", prec="fp64",
              flags=0) -> admm_opts:
    return admm_opts(float(rho), float(tol), int(max_iter), int(check_every),
                     FORMS.get(form, form), PRECS.get(prec, prec), int(flags))


def _result(r: admm_result) -> dict:
    return dict(iters=r.iters, status=r.status, eps_p=r.eps_p, eps_d=r.eps_d,
                obj_primal=r.obj_primal, obj_dual=r.obj_dual, seconds=r.seconds,
                kernel_launches=r.kernel_launches)


# ------------------------------------------------------------------------------- entry points

def _problem_arrays(n, A_ptr, A_row, A_col, A_val, b, C_row, C_col, C_val, cliques=None,
                    clique_ptr=None, clique_vtx=None, pat_row=None, pat_col=None):
    """The host arrays of one problem, converted to the ABI's types (kept alive by the caller)."""
    if cliques is not None:
        sizes = np.array([len(c) for c in cliques], dtype=np.int64)
        clique_ptr = np.concatenate([[0], np.cumsum(sizes)])
        clique_vtx = np.concatenate([np.asarray(c) for c in cliques]) if len(cliques) else np.zeros(0)
    elif clique_ptr is None:
        clique_ptr, clique_vtx = np.zeros(1), np.zeros(0)     # p = 0: the library's chordal extension
    d = dict(n=int(n), A_ptr=_arr(A_ptr, np.int64), A_row=_arr(A_row, np.int32), A_col=_arr(A_col, np.int32),
             A_val=_arr(A_val, np.float64), b=_arr(b, np.float64), C_row=_arr(C_row, np.int32),
             C_col=_arr(C_col, np.int32), C_val=_arr(C_val, np.float64),
             clique_ptr=_arr(clique_ptr, np.int32), clique_vtx=_arr(clique_vtx, np.int32),
             pat_row=_arr(pat_row, np.int32) if pat_row is not None else None,
             pat_col=_arr(pat_col, np.int32) if pat_col is not None else None)
    return d


def _problem_struct(d: dict) -> sdp_problem:
    pr = d["pat_row"]
    return sdp_problem(d["n"], len(d["b"]), _ptr(d["A_ptr"]), _ptr(d["A_row"]), _ptr(d["A_col"]),
                       _ptr(d["A_val"]), _ptr(d["b"]), len(d["C_val"]), _ptr(d["C_row"]), _ptr(d["C_col"]),
                       _ptr(d["C_val"]), 0 if pr is None else len(pr), _ptr(pr), _ptr(d["pat_col"]),
                       len(d["clique_ptr"]) - 1, _ptr(d["clique_ptr"]), _ptr(d["clique_vtx"]))


def sdp_setup(n, A_ptr, A_row, A_col, A_val, b, C_row, C_col, C_val, cliques=None,
              clique_ptr=None, clique_vtx=None, pat_row=None, pat_col=None, opts=None):
    """Set up the decomposed problem on the current CUDA device; returns the opaque handle."""
    lib = load_library()
    d = _problem_arrays(n, A_ptr, A_row, A_col, A_val, b, C_row, C_col, C_val, cliques, clique_ptr,
                        clique_vtx, pat_row, pat_col)
    pr = d["pat_row"]
    opts = opts if opts is not None else make_opts()
    h = ctypes.c_void_p()
    rc = lib.sdp_setup(d["n"], len(d["b"]), _ptr(d["A_ptr"]), _ptr(d["A_row"]), _ptr(d["A_col"]),
                       _ptr(d["A_val"]), _ptr(d["b"]), len(d["C_val"]), _ptr(d["C_row"]), _ptr(d["C_col"]),
                       _ptr(d["C_val"]), 0 if pr is None else len(pr), _ptr(pr), _ptr(d["pat_col"]),
                       len(d["clique_ptr"]) - 1, _ptr(d["clique_ptr"]), _ptr(d["clique_vtx"]),
                       ctypes.byref(opts), ctypes.byref(h))
    _check(rc, "sdp_setup")
    return h


def sdp_setup_batch(problems, opts=None):
    """One handle for a list of independent problems (dicts with the keyword arguments of
    ``sdp_setup``: n, A_ptr, A_row, A_col, A_val, b, C_row, C_col, C_val and cliques or
    clique_ptr/clique_vtx)."""
    lib = load_library()
    keep = [_problem_arrays(**{k: v for k, v in pr.items() if k in _PROBLEM_KEYS}) for pr in problems]
    arr = (sdp_problem * len(keep))(*[_problem_struct(d) for d in keep])
    opts = opts if opts is not None else make_opts()
    h = ctypes.c_void_p()
    _check(lib.sdp_setup_batch(len(keep), arr, ctypes.byref(opts), ctypes.byref(h)), "sdp_setup_batch")
    return h


def _cone_arrays(cones: dict) -> dict:
    nc = int(cones.get("n_free", 0)) + int(cones.get("n_lin", 0)) + int(np.sum(cones.get("soc_dims", [])))
    return dict(n_free=int(cones.get("n_free", 0)), n_lin=int(cones.get("n_lin", 0)),
                soc_dims=_arr(cones.get("soc_dims", []), np.int32), A_ptr=_arr(cones["A_ptr"], np.int64),
                A_var=_arr(cones["A_var"], np.int32), A_val=_arr(cones["A_val"], np.float64),
                c=_arr(cones["c"], np.float64) if cones.get("c") is not None else None, n_cone=nc)


def sdp_setup_conic(problem: dict, cones: dict | None, opts=None):
    """A problem with variables in free, nonnegative and second-order cones beside the PSD matrix:
    ``problem`` has sdp_setup's keyword arguments (n = 0 and cliques = [] for no PSD part),
    ``cones`` the keys n_free, n_lin, soc_dims, A_ptr, A_var, A_val and c."""
    lib = load_library()
    d = _problem_arrays(**{k: v for k, v in problem.items() if k in _PROBLEM_KEYS})
    pr = _problem_struct(d)
    cd = _cone_arrays(cones) if cones is not None else None
    cs = None if cd is None else sdp_cones(cd["n_free"], cd["n_lin"], len(cd["soc_dims"]), _ptr(cd["soc_dims"]),
                                           _ptr(cd["A_ptr"]), _ptr(cd["A_var"]), _ptr(cd["A_val"]), _ptr(cd["c"]))
    opts = opts if opts is not None else make_opts()
    h = ctypes.c_void_p()
    _check(lib.sdp_setup_conic(ctypes.byref(pr), ctypes.byref(cs) if cs is not None else None,
                               ctypes.byref(opts), ctypes.byref(h)), "sdp_setup_conic")
    return h


def sdp_plan(problem: dict, cones: dict | None = None) -> dict:
    """Host-only check and sizes of a problem (sdp_setup's arguments as a dict; cones as for
    sdp_setup_conic): the sizes a handle would have, without a GPU."""
    lib = load_library()
    d = _problem_arrays(**{k: v for k, v in problem.items() if k in _PROBLEM_KEYS})
    pr = _problem_struct(d)
    cd = _cone_arrays(cones) if cones is not None else None
    cs = None if cd is None else sdp_cones(cd["n_free"], cd["n_lin"], len(cd["soc_dims"]), _ptr(cd["soc_dims"]),
                                           _ptr(cd["A_ptr"]), _ptr(cd["A_var"]), _ptr(cd["A_val"]), _ptr(cd["c"]))
    out = sdp_sizes()
    _check(lib.sdp_plan(ctypes.byref(pr), ctypes.byref(cs) if cs is not None else None, ctypes.byref(out)),
           "sdp_plan")
    return {f: getattr(out, f) for f, _ in sdp_sizes._fields_}


_PROBLEM_KEYS = ("n", "A_ptr", "A_row", "A_col", "A_val", "b", "C_row", "C_col", "C_val", "cliques",
                 "clique_ptr", "clique_vtx", "pat_row", "pat_col")


def sdp_batch_layout(h) -> dict:
    """Offsets of each problem in the handle's vectors (arrays of batch + 1 entries)."""
    q = sdp_get_sizes(h)["batch"]
    out = dict(vtx_off=np.zeros(q + 1, np.int32), row_off=np.zeros(q + 1, np.int32),
               clique_off=np.zeros(q + 1, np.int32), ent_off=np.zeros(q + 1, np.int64),
               pos_off=np.zeros(q + 1, np.int64))
    _check(load_library().sdp_batch_layout(h, *[_ptr(out[k]) for k in
                                                ("vtx_off", "row_off", "clique_off", "ent_off", "pos_off")]),
           "sdp_batch_layout")
    return out


def sdp_batch_results(h) -> dict:
    """Per-problem iterations, status, residuals and objectives (arrays of batch entries)."""
    q = sdp_get_sizes(h)["batch"]
    out = dict(iters=np.zeros(q, np.int32), status=np.zeros(q, np.int32), eps_p=np.zeros(q),
               eps_d=np.zeros(q), obj_primal=np.zeros(q), obj_dual=np.zeros(q))
    _check(load_library().sdp_batch_results(h, *[_ptr(out[k]) for k in
                                                 ("iters", "status", "eps_p", "eps_d", "obj_primal", "obj_dual")]),
           "sdp_batch_results")
    return out


def sdp_set_opts(h, opts: admm_opts):
    _check(load_library().sdp_set_opts(h, ctypes.byref(opts)), "sdp_set_opts")


def admm_reset(h, stream=None):
    _check(load_library().admm_reset(h, _stream(stream)), "admm_reset")


def admm_iterate(h, n_iters: int, stream=None) -> dict:
    r = admm_result()
    rc = load_library().admm_iterate(h, int(n_iters), _stream(stream), ctypes.byref(r))
    _check(rc, "admm_iterate", ok=(SDP_OK, SDP_MAX_ITER))
    return _result(r)


def admm_solve(h, stream=None) -> dict:
    r = admm_result()
    rc = load_library().admm_solve(h, _stream(stream), ctypes.byref(r))
    _check(rc, "admm_solve", ok=(SDP_OK, SDP_MAX_ITER))
    return _result(r)


def sdp_get_sizes(h) -> dict:
    s = sdp_sizes()
    _check(load_library().sdp_get_sizes(h, ctypes.byref(s)), "sdp_get_sizes")
    return {f: getattr(s, f) for f, _ in sdp_sizes._fields_}


def sdp_get_solution(h):
    """(X on E_L, y, Z on E_L) as NumPy arrays."""
    sz = sdp_get_sizes(h)
    X = np.empty(sz["nE_lower"]); y = np.empty(sz["m"]); Z = np.empty(sz["nE_lower"])
    _check(load_library().sdp_get_solution(h, _ptr(X), _ptr(y), _ptr(Z)), "sdp_get_solution")
    return X, y, Z


def sdp_get_state(h) -> dict:
    sz = sdp_get_sizes(h)
    out = dict(x=np.empty(sz["nE_lower"]), y=np.empty(sz["m"]), blk_a=np.empty(sz["S_lower"]),
               blk_b=np.empty(sz["S_lower"]), blk_c=np.empty(sz["S_lower"]))
    _check(load_library().sdp_get_state(h, *(_ptr(out[k]) for k in ("x", "y", "blk_a", "blk_b", "blk_c"))),
           "sdp_get_state")
    return out


def sdp_set_state(h, x=None, y=None, blk_a=None, blk_b=None, blk_c=None):
    arrs = [None if v is None else _arr(v, np.float64) for v in (x, y, blk_a, blk_b, blk_c)]
    _check(load_library().sdp_set_state(h, *(_ptr(a) for a in arrs)), "sdp_set_state")


def sdp_proj_sweeps(h) -> np.ndarray:
    """Jacobi sweeps per clique in the handle's last iteration (diagnostic)."""
    out = np.zeros(sdp_get_sizes(h)["p"], np.int32)
    _check(load_library().sdp_proj_sweeps(h, _ptr(out)), "sdp_proj_sweeps")
    return out


def sdp_get_maps(h) -> dict:
    sz = sdp_get_sizes(h)
    out = dict(pat_row=np.empty(sz["nE_lower"], np.int32), pat_col=np.empty(sz["nE_lower"], np.int32),
               blk_off=np.empty(sz["p"] + 1, np.int64), gather_idx=np.empty(sz["S_lower"], np.int32))
    _check(load_library().sdp_get_maps(h, *(_ptr(out[k]) for k in ("pat_row", "pat_col", "blk_off", "gather_idx"))),
           "sdp_get_maps")
    return out


def sdp_gather(h, x, blocks_out, stream=None):
    sz = sdp_get_sizes(h)
    _check(load_library().sdp_gather(h, _dev_ptr(x, sz["nE_lower"], "x"),
                                      _dev_ptr(blocks_out, sz["S_lower"], "blocks_out"), _stream(stream)),
           "sdp_gather")


def sdp_scatter(h, blocks, out, stream=None):
    sz = sdp_get_sizes(h)
    _check(load_library().sdp_scatter(h, _dev_ptr(blocks, sz["S_lower"], "blocks"),
                                       _dev_ptr(out, sz["nE_lower"], "out"), _stream(stream)),
           "sdp_scatter")


def project_psd_batched(inp, out, sizes, offsets, prec="fp64", stream=None):
    """P(W) of packed lower blocks: ``inp``/``out`` float64 CUDA tensors; sizes/offsets host arrays."""
    sizes = _arr(sizes, np.int32)
    offsets = _arr(offsets, np.int64)
    if len(sizes) != len(offsets):
        raise ValueError("sizes and offsets differ in length")
    need = int((offsets + sizes.astype(np.int64) * (sizes + 1) // 2).max()) if len(sizes) else 0
    _check(load_library().project_psd_batched(_dev_ptr(inp, need, "inp"), _dev_ptr(out, need, "out"),
                                              _ptr(sizes), _ptr(offsets), len(sizes),
                                              PRECS.get(prec, prec), _stream(stream)),
           "project_psd_batched")


def project_psd_batched_noalloc(inp, out, sizes, offsets, prec="fp64", stream=None):
    """project_psd_batched without any device allocation (fixed in-library schedule array of
    SDP_NOALLOC_MAX_BLOCKS blocks; calls must not overlap on the GPU)."""
    sizes = _arr(sizes, np.int32)
    offsets = _arr(offsets, np.int64)
    if len(sizes) != len(offsets):
        raise ValueError("sizes and offsets differ in length")
    need = int((offsets + sizes.astype(np.int64) * (sizes + 1) // 2).max()) if len(sizes) else 0
    _check(load_library().project_psd_batched_noalloc(
        _dev_ptr(inp, need, "inp"), _dev_ptr(out, need, "out"), _ptr(sizes), _ptr(offsets), len(sizes),
        PRECS.get(prec, prec), _stream(stream)), "project_psd_batched_noalloc")


def project_variants() -> list:
    """Names of the projection kernel variants, by variant index."""
    lib = load_library()
    return [lib.project_variant_name(v).decode() for v in range(lib.project_variant_count())]


def project_variant_fits(variant: int, s: int, prec="fp32") -> bool:
    return bool(load_library().project_variant_fits(int(variant), int(s), PRECS.get(prec, prec)))


def project_psd_batched_variant(inp, out, sizes, offsets, variant: int, prec="fp32", stream=None):
    """project_psd_batched with every block on one kernel variant."""
    sizes = _arr(sizes, np.int32)
    offsets = _arr(offsets, np.int64)
    need = int(np.max(offsets + sizes.astype(np.int64) * (sizes + 1) // 2)) if len(sizes) else 0
    _check(load_library().project_psd_batched_variant(
        _dev_ptr(inp, need, "inp"), _dev_ptr(out, need, "out"), _ptr(sizes), _ptr(offsets), len(sizes),
        PRECS.get(prec, prec), int(variant), _stream(stream)), "project_psd_batched_variant")


def sdp_set_proj_table(h, prec, table=None):
    """Projection variant per padded block order for a handle (a dict {N: variant} or a sequence
    indexed by N; None restores the defaults)."""
    p = PRECS.get(prec, prec)
    if table is None:
        _check(load_library().sdp_set_proj_table(h, p, None, 0), "sdp_set_proj_table")
        return
    if isinstance(table, dict):
        t = np.full(SDP_MAX_CLIQUE + 1, -1, np.int32)
        for n, v in table.items():
            t[int(n)] = int(v)
    else:
        t = _arr(table, np.int32)
    _check(load_library().sdp_set_proj_table(h, p, _ptr(t), len(t)), "sdp_set_proj_table")


def sdp_chordal_cliques(n, rows, cols):
    """(cliques, fill): maximal cliques of the library's chordal extension of a pattern (host only)."""
    lib = load_library()
    r, c = _arr(rows, np.int32), _arr(cols, np.int32)
    p, nv, fill = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_longlong()
    _check(lib.sdp_chordal_cliques(int(n), len(r), _ptr(r), _ptr(c), ctypes.byref(p), ctypes.byref(nv),
                                   ctypes.byref(fill), None, None, 0, 0), "sdp_chordal_cliques")
    cp = np.zeros(p.value + 1, np.int32)
    cv = np.zeros(max(1, nv.value), np.int32)
    _check(lib.sdp_chordal_cliques(int(n), len(r), _ptr(r), _ptr(c), ctypes.byref(p), ctypes.byref(nv),
                                   ctypes.byref(fill), _ptr(cp), _ptr(cv), p.value, nv.value),
           "sdp_chordal_cliques")
    return [cv[cp[k]:cp[k + 1]].copy() for k in range(p.value)], int(fill.value)


def sdp_set_cost(h, c_lower, stream=None):
    """New cost C for the handle: a float64 CUDA tensor of its lower-pattern values (E_L order)."""
    n = sdp_get_sizes(h)["nE_lower"]
    _check(load_library().sdp_set_cost(h, _dev_ptr(c_lower, n, "c_lower"), _stream(stream)), "sdp_set_cost")


def sdp_set_rhs(h, b, stream=None):
    """New right-hand side b for the handle: a float64 CUDA tensor of m values."""
    m = sdp_get_sizes(h)["m"]
    _check(load_library().sdp_set_rhs(h, _dev_ptr(b, m, "b"), _stream(stream)), "sdp_set_rhs")


def sdp_unrolled_forward(h, T: int, ckpt_every: int = 20, x_out=None, stream=None):
    """T primal-form FP64 iterations from a reset, with checkpoints; X_T into x_out (CUDA tensor)."""
    n = sdp_get_sizes(h)["nE_lower"]
    ptr = None if x_out is None else _dev_ptr(x_out, n, "x_out")
    _check(load_library().sdp_unrolled_forward(h, int(T), int(ckpt_every), ptr, _stream(stream)),
           "sdp_unrolled_forward")


def sdp_unrolled_backward(h, xbar, cbar, bbar, stream=None):
    """Reverse mode of the last sdp_unrolled_forward: dL/dtheta_C into cbar and dL/db into bbar."""
    sz = sdp_get_sizes(h)
    _check(load_library().sdp_unrolled_backward(
        h, _dev_ptr(xbar, sz["nE_lower"], "xbar"), _dev_ptr(cbar, sz["nE_lower"], "cbar"),
        _dev_ptr(bbar, sz["m"], "bbar"), _stream(stream)), "sdp_unrolled_backward")


def sdp_time_phases(h, reps: int = 20, stream=None) -> dict:
    """Average device milliseconds of each kernel of one iteration, by kernel name."""
    lib = load_library()
    ms = np.zeros(16)
    n = lib.sdp_time_phases(h, int(reps), _stream(stream), _ptr(ms), len(ms))
    if n < 0:
        _check(n, "sdp_time_phases")
    return {lib.sdp_phase_name(h, i).decode(): float(ms[i]) for i in range(n)}


def sdp_setup_times(h) -> dict:
    """Wall-clock milliseconds of the stages of the setup call that made h, by stage name."""
    lib = load_library()
    ms = np.zeros(8)
    n = lib.sdp_setup_times(h, _ptr(ms), len(ms))
    if n < 0:
        _check(n, "sdp_setup_times")
    return {lib.sdp_setup_stage_name(i).decode(): float(ms[i]) for i in range(n)}


def sdp_phase_name(h, i: int) -> str | None:
    """Name of phase i of an iteration for the handle's current form."""
    r = load_library().sdp_phase_name(h, int(i))
    return None if r is None else r.decode()


def sdp_free(h):
    if h:
        load_library().sdp_free(h)


def sdp_status_string(code: int) -> str:
    return load_library().sdp_status_string(int(code)).decode()


def sdp_last_error() -> str:
    return load_library().sdp_last_error().decode()


class ChordalADMM:
    """Owns one handle: ``with ChordalADMM(inst_arrays, opts) as s: s.solve()``."""

    def __init__(self, arrays, opts: admm_opts | None = None):
        """``arrays``: one problem (a dict of sdp_setup's keyword arguments) or a list of them (a
        batch, set up with sdp_setup_batch)."""
        self.opts = opts if opts is not None else make_opts()
        if isinstance(arrays, dict) and arrays.get("cones") is not None:
            self.h = sdp_setup_conic(arrays, arrays["cones"], self.opts)
        elif isinstance(arrays, dict):
            self.h = sdp_setup(arrays["n"], arrays["A_ptr"], arrays["A_row"], arrays["A_col"],
                               arrays["A_val"], arrays["b"], arrays["C_row"], arrays["C_col"],
                               arrays["C_val"], cliques=arrays["cliques"], opts=self.opts)
        else:
            self.h = sdp_setup_batch(list(arrays), self.opts)
        self.sizes = sdp_get_sizes(self.h)

    def batch_layout(self):
        return sdp_batch_layout(self.h)

    def batch_results(self):
        return sdp_batch_results(self.h)

    def set_opts(self, **kw):
        d = {f: getattr(self.opts, f) for f, _ in admm_opts._fields_}
        for k, v in kw.items():
            d[k] = FORMS.get(v, PRECS.get(v, v)) if k in ("form", "prec") else v
        self.opts = admm_opts(**d)
        sdp_set_opts(self.h, self.opts)

    def reset(self, stream=None):
        admm_reset(self.h, stream)

    def iterate(self, n, stream=None):
        return admm_iterate(self.h, n, stream)

    def solve(self, stream=None):
        return admm_solve(self.h, stream)

    def state(self):
        return sdp_get_state(self.h)

    def solution(self):
        return sdp_get_solution(self.h)

    def close(self):
        if self.h:
            sdp_free(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
