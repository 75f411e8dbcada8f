"""Random SDPs with the block-arrow sparsity pattern (Section V.A and Fig. 2 of the paper).

The pattern has ``l`` diagonal blocks of size ``d`` and an arrow head of width ``h``; ``n = l*d + h``.
It is chordal and its maximal cliques are ``C_k = B_k ∪ H`` (block ``k`` plus the head), each of size
``s = d + h`` (``p = l`` cliques). Vertices are 0-based.

Data recipe (the paper gives only the pattern parameters; the values below are this project's):

* ``A_i``: symmetric, N(0,1) entries on a random ``density`` fraction of the lower-triangle pattern
  positions (diagonal included), drawn without replacement and mirrored.
* ``X0 = G Gᵀ`` with ``G`` an ``n×n`` matrix of N(0,1)/√n entries; only its values on the pattern are
  kept. ``b = 𝒜(X0)``, so the primal problem is strictly feasible.
* ``y0 ~ N(0,1)``; ``Z0`` has N(0,1) on every off-diagonal pattern entry and diagonal equal to its
  row's absolute off-diagonal sum plus one (strictly diagonally dominant, so ``Z0 ≻ 0``).
  ``C = 𝒜*(y0) + Z0``, so the dual problem is strictly feasible and the aggregate pattern is the
  full block-arrow pattern.

Random streams come from ``numpy.random.SeedSequence(seed)`` children, one per quantity (and one per
row block of ``G``), so each quantity can be drawn without holding ``G`` in memory.

Matrices are returned in lower-triangle coordinate form: for every stored entry ``row >= col``.
The lower pattern list ``pat_row/pat_col`` is in column-major order (sorted by column, then row).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# The five workloads. ``rho`` is the fixed ADMM penalty: the paper fixes none; 1.0 where the workload
# states it, otherwise the value that a scan found fastest to 1e-4 on the first instance (workload 1:
# {0.003 .. 0.3}; workload 3: {0.001 .. 1}, where 0.003 needs 561 iterations, 0.005 577, 0.002 817,
# 0.02 2007 and 0.05 and above more than 3000).
CONFIGS = {
    0: dict(name="blockarrow_l10_d10_h2_m50", l=10, d=10, h=2, m=50, density=0.30, count=1,
            max_iter=2000, tol=1e-4, form="primal", prec="fp64", rho=1.0),
    1: dict(name="blockarrow_l100_d10_h20_m200", l=100, d=10, h=20, m=200, density=0.30, count=1,
            max_iter=2000, tol=1e-4, form="dual", prec="fp32", rho=0.02),
    2: dict(name="batch512_blockarrow_l5-60_d4-24_h1-16_m20-300", l=None, d=None, h=None, m=None,
            density=0.30, count=512, max_iter=2000, tol=1e-4, form="dual", prec="fp32", rho=0.02),
    3: dict(name="blockarrow_l2000_d20_h40_m1000", l=2000, d=20, h=40, m=1000, density=0.10,
            count=1, max_iter=500, tol=1e-4, form="dual", prec="fp32", rho=0.003),
    4: dict(name="batch64_blockarrow_l50_d10_h5_m100", l=50, d=10, h=5, m=100, density=0.30,
            count=64, max_iter=200, tol=0.0, form="primal", prec="fp64", rho=1.0),
}


# The paper's three block-arrow sweeps (Section V.A): one parameter varies, the others are fixed,
# at tolerance 1e-3 and 2000 iterations. The paper's figure with the values is not reproduced
# here, so the varied values span the ranges its text describes. Point i of sweep "x" uses seed
# 9000 + 100 * ("mld".index(x)) + i.
SWEEPS = {
    "m": dict(fixed=dict(l=40, d=10, h=20), values=[50, 100, 200, 400, 700, 1000]),
    "l": dict(fixed=dict(m=1000, d=10, h=20), values=[10, 20, 40, 80, 160, 320]),
    "d": dict(fixed=dict(l=40, h=10, m=1000), values=[5, 10, 15, 20, 30, 40]),
}
SWEEP_TOL = 1e-3
SWEEP_MAX_ITER = 2000


def sweep_instance(name: str, i: int) -> "SDPInstance":
    """Point i of sweep `name` ("m", "l" or "d"), density 30 %."""
    sw = SWEEPS[name]
    params = dict(sw["fixed"])
    params[name] = sw["values"][i]
    return block_arrow_instance(density=0.30, seed=9000 + 100 * "mld".index(name) + i,
                                meta=dict(sweep=name, point=i), **params)


@dataclass
class SDPInstance:
    """One SDP ``min <C,X> s.t. <A_i,X> = b_i, X ⪰ 0`` with its chordal decomposition data."""

    n: int
    m: int
    cliques: list            # list of sorted int32 vertex arrays
    pat_row: np.ndarray      # int32, lower pattern rows (row >= col), column-major order
    pat_col: np.ndarray      # int32
    A_ptr: np.ndarray        # int64 [m+1]: constraint i owns entries A_ptr[i]:A_ptr[i+1]
    A_row: np.ndarray        # int32
    A_col: np.ndarray        # int32
    A_val: np.ndarray        # float64
    b: np.ndarray            # float64 [m]
    C_row: np.ndarray        # int32
    C_col: np.ndarray        # int32
    C_val: np.ndarray        # float64
    X0_val: np.ndarray       # float64, X0 on the lower pattern (pat order); primal feasible point
    y0: np.ndarray           # float64 [m]; (y0, Z0) is dual feasible
    Z0_val: np.ndarray       # float64, Z0 on the lower pattern (pat order)
    meta: dict = field(default_factory=dict)

    @property
    def clique_ptr(self) -> np.ndarray:
        sizes = np.array([len(c) for c in self.cliques], dtype=np.int64)
        return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)

    @property
    def clique_vtx(self) -> np.ndarray:
        return np.concatenate(self.cliques).astype(np.int32)

    @property
    def nnz_A(self) -> int:
        return int(self.A_ptr[-1])


def block_arrow_cliques(l: int, d: int, h: int) -> list:
    """Maximal cliques of the block-arrow pattern: block k plus the head, sorted ascending."""
    head = np.arange(l * d, l * d + h, dtype=np.int32)
    return [np.concatenate([np.arange(k * d, (k + 1) * d, dtype=np.int32), head]) for k in range(l)]


def _lower_pattern(n: int, cliques: list):
    """Lower-triangle pairs of the union of clique×clique, column-major order."""
    keys = []
    for c in cliques:
        c = np.asarray(c, dtype=np.int64)
        a, bb = np.tril_indices(len(c))
        keys.append(c[bb] * n + c[a])           # key = col*n + row, row >= col
    keys = np.unique(np.concatenate(keys))
    return (keys % n).astype(np.int32), (keys // n).astype(np.int32), keys


def block_arrow_instance(l: int, d: int, h: int, m: int, density: float, seed: int,
                         meta: dict | None = None) -> SDPInstance:
    n = l * d + h
    cliques = block_arrow_cliques(l, d, h)
    pat_row, pat_col, keys = _lower_pattern(n, cliques)
    nl = len(keys)
    offdiag = pat_row != pat_col
    w = np.where(offdiag, 2.0, 1.0)

    ss = np.random.SeedSequence(seed)
    s_A, s_G, s_y, s_Z = ss.spawn(4)

    # Constraint matrices, lower coordinates, CSR by constraint.
    rng_A = np.random.default_rng(s_A)
    k = int(round(density * nl))
    k = max(1, min(k, nl))
    A_pos = np.empty((m, k), dtype=np.int64)
    A_val = np.empty((m, k), dtype=np.float64)
    for i in range(m):
        pos = rng_A.choice(nl, size=k, replace=False)
        pos.sort()
        A_pos[i] = pos
        A_val[i] = rng_A.standard_normal(k)
    A_ptr = np.arange(m + 1, dtype=np.int64) * k

    # X0 = G Gᵀ on the pattern; G row blocks drawn per block and once for the head.
    g_children = s_G.spawn(l + 1)
    inv_sqrt_n = 1.0 / math.sqrt(n)
    G_head = np.random.default_rng(g_children[0]).standard_normal((h, n)) * inv_sqrt_n
    X0_val = np.empty(nl, dtype=np.float64)

    def put(rows, cols, vals):
        kk = cols.astype(np.int64) * n + rows.astype(np.int64)
        X0_val[np.searchsorted(keys, kk)] = vals

    if h > 0:
        hh = G_head @ G_head.T
        a, bb = np.tril_indices(h)
        put(l * d + a, l * d + bb, hh[a, bb])
    for blk in range(l):
        Gb = np.random.default_rng(g_children[blk + 1]).standard_normal((d, n)) * inv_sqrt_n
        bbm = Gb @ Gb.T
        a, bb = np.tril_indices(d)
        put(blk * d + a, blk * d + bb, bbm[a, bb])
        if h > 0:
            hb = G_head @ Gb.T                     # rows: head, cols: block
            hr, bc = np.meshgrid(np.arange(h), np.arange(d), indexing="ij")
            put(l * d + hr.ravel(), blk * d + bc.ravel(), hb.ravel())

    b = (A_val * (w[A_pos] * X0_val[A_pos])).sum(axis=1)

    y0 = np.random.default_rng(s_y).standard_normal(m)

    rng_Z = np.random.default_rng(s_Z)
    Z0_val = np.zeros(nl, dtype=np.float64)
    Z0_val[offdiag] = rng_Z.standard_normal(int(offdiag.sum()))
    rowsum = np.zeros(n)
    np.add.at(rowsum, pat_row[offdiag], np.abs(Z0_val[offdiag]))
    np.add.at(rowsum, pat_col[offdiag], np.abs(Z0_val[offdiag]))
    Z0_val[~offdiag] = rowsum[pat_row[~offdiag]] + 1.0

    # C = 𝒜*(y0) + Z0 on the pattern
    C_val = Z0_val + np.bincount(A_pos.ravel(), weights=(A_val * y0[:, None]).ravel(), minlength=nl)

    md = dict(l=l, d=d, h=h, density=density, seed=seed)
    if meta:
        md.update(meta)
    return SDPInstance(
        n=n, m=m, cliques=cliques, pat_row=pat_row, pat_col=pat_col,
        A_ptr=A_ptr, A_row=pat_row[A_pos.ravel()].copy(), A_col=pat_col[A_pos.ravel()].copy(),
        A_val=A_val.ravel().copy(), b=b, C_row=pat_row.copy(), C_col=pat_col.copy(), C_val=C_val,
        X0_val=X0_val, y0=y0, Z0_val=Z0_val, meta=md)


def config_seed(config: int, instance: int = 0) -> int:
    return 1000 * (config + 1) + instance


def config_shapes(config: int, instance: int = 0):
    """(l, d, h, m) of one instance of a workload; the batched workload draws them per instance."""
    cfg = CONFIGS[config]
    if config != 2:
        return cfg["l"], cfg["d"], cfg["h"], cfg["m"]
    rng = np.random.default_rng(np.random.SeedSequence([config_seed(config, instance), 7]))
    l = int(rng.integers(5, 61))
    d = int(rng.integers(4, 25))
    h = int(rng.integers(1, 17))
    m = int(rng.integers(20, 301))
    nl = l * d * (d + 1) // 2 + h * (h + 1) // 2 + h * l * d
    m = min(m, nl // 2)          # keep A D⁻¹ Aᵀ well posed on the smallest patterns
    return l, d, h, m


def config_instance(config: int, instance: int = 0, **overrides) -> SDPInstance:
    """Instance ``instance`` of workload ``config`` with seed ``1000*(config+1) + instance``."""
    cfg = CONFIGS[config]
    l, d, h, m = config_shapes(config, instance)
    params = dict(l=l, d=d, h=h, m=m, density=cfg["density"])
    params.update(overrides)
    return block_arrow_instance(seed=config_seed(config, instance),
                                meta=dict(config=config, instance=instance), **params)


# A conic workload (Section V: CDCS also accepts free, nonnegative and second-order variables,
# which are not decomposed): the n = 1020 block-arrow SDP with 10^6 nonnegative variables and
# 10^5 second-order cones of dimension 10 added, each cone variable in 2 random constraints.
# rho: a scan over {0.005 .. 2} found 1.0 fastest to 1e-4 (1658 iterations; 0.2 and below do not
# get there within 3000).
CONIC = dict(name="blockarrow_l100_d10_h20_m200+lin1e6+soc1e5x10", base=1, n_free=0, n_lin=1_000_000,
             soc_count=100_000, soc_dim=10, per_var=2, seed=7000, rho=1.0, form="dual", prec="fp32",
             iters=200)


def conic_extension(inst: SDPInstance, n_free: int, n_lin: int, soc_dims, per_var: int, seed: int) -> dict:
    """Variables in the other cones added to the SDP ``inst``: returns the new right-hand side
    ``b`` and the ``cones`` dict (n_free, n_lin, soc_dims, A_ptr, A_var, A_val, c).

    Each cone variable gets N(0,1) coefficients in ``per_var`` distinct random constraints. The
    primal point x0 is interior (free: N(0,1); nonnegative: U(0.5, 1.5); second-order: u ~
    N(0, 1/q), t = ‖u‖ + U(0.5, 1.5)) and so is the dual slack z0 (0 on the free variables, whose
    dual cone is {0}); ``b += A_cone x0`` and ``c_cone = A_coneᵀ y0 + z0`` keep (X0, x0) primal and
    (y0, Z0, z0) dual feasible."""
    soc_dims = np.asarray(soc_dims, dtype=np.int64)
    m = len(inst.b)
    nc = int(n_free + n_lin + soc_dims.sum())
    ss = np.random.SeedSequence(seed).spawn(4)
    rng_a, rng_x, rng_z, rng_r = (np.random.default_rng(s) for s in ss)
    k = min(per_var, m)
    # distinct rows per variable: uniform draws, rows with a repeat drawn again
    rows = rng_r.integers(0, m, size=(nc, k))
    while k > 1:
        srt = np.sort(rows, axis=1)
        bad = np.flatnonzero((np.diff(srt, axis=1) == 0).any(axis=1))
        if len(bad) == 0:
            break
        rows[bad] = rng_r.integers(0, m, size=(len(bad), k))
    vals = rng_a.standard_normal((nc, k))
    starts = n_free + n_lin + np.concatenate([[0], np.cumsum(soc_dims)[:-1]]).astype(np.int64)

    def interior(rng, zero_free):
        v = np.empty(nc)
        v[:n_free] = 0.0 if zero_free else rng.standard_normal(n_free)
        v[n_free:n_free + n_lin] = rng.uniform(0.5, 1.5, n_lin)
        for q in np.unique(soc_dims):                      # cones grouped by dimension
            st = starts[soc_dims == q]
            u = rng.standard_normal((len(st), q - 1)) / math.sqrt(q)
            v[st] = np.linalg.norm(u, axis=1) + rng.uniform(0.5, 1.5, len(st))
            v[st[:, None] + np.arange(1, q)[None, :]] = u
        return v

    x0 = interior(rng_x, False)
    z0 = interior(rng_z, True)
    var = np.repeat(np.arange(nc), k)
    row = rows.ravel()
    val = vals.ravel()
    order = np.lexsort((var, row))
    row, var, val = row[order], var[order], val[order]
    A_ptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(A_ptr, row + 1, 1)
    A_ptr = np.cumsum(A_ptr)
    b = inst.b + np.bincount(row, weights=val * x0[var], minlength=m)
    c = np.bincount(var, weights=val * inst.y0[row], minlength=nc) + z0
    cones = dict(n_free=int(n_free), n_lin=int(n_lin), soc_dims=soc_dims.astype(np.int32), A_ptr=A_ptr,
                 A_var=var.astype(np.int32), A_val=val, c=c)
    return dict(b=b, cones=cones, x0=x0, z0=z0)
