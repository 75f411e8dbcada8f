"""Small hand-built SDPs with known optima, used by the oracle pins and the GPU parity tests.

Each builder returns plain arrays in the C-ABI's input form: lower-triangle coordinates (row >= col),
constraints grouped by constraint (``A_ptr``), and the maximal cliques.
"""

from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name: str) -> dict:
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = vals
    return out


def lower_coo(M: np.ndarray, pattern: np.ndarray | None = None):
    """Lower-triangle coordinates of a symmetric matrix (nonzeros, or all pattern entries)."""
    n = M.shape[0]
    rows, cols = np.tril_indices(n)
    keep = (M[rows, cols] != 0) if pattern is None else pattern[rows, cols]
    rows, cols = rows[keep], cols[keep]
    order = np.lexsort((rows, cols))
    return rows[order].astype(np.int32), cols[order].astype(np.int32), M[rows[order], cols[order]]


def problem_from_dense(C: np.ndarray, As: list, b, cliques: list) -> dict:
    """Pack dense symmetric data into the coordinate form used everywhere else."""
    A_rows, A_cols, A_vals, ptr = [], [], [], [0]
    for Ai in As:
        r, c, v = lower_coo(Ai)
        A_rows.append(r); A_cols.append(c); A_vals.append(v)
        ptr.append(ptr[-1] + len(r))
    C_row, C_col, C_val = lower_coo(C)
    return dict(n=C.shape[0], cliques=[np.asarray(c, dtype=np.int32) for c in cliques],
                A_ptr=np.asarray(ptr, dtype=np.int64),
                A_row=np.concatenate(A_rows).astype(np.int32),
                A_col=np.concatenate(A_cols).astype(np.int32),
                A_val=np.concatenate(A_vals).astype(np.float64),
                b=np.asarray(b, dtype=np.float64), C_row=C_row, C_col=C_col, C_val=C_val)


def theta_c5() -> tuple[dict, float]:
    """Lovász theta of C5 as min <-J, X> s.t. tr X = 1, X_ij = 0 on edges (optimum -sqrt 5)."""
    g = read_golden("lovasz_theta_c5.txt")
    n = int(g["n"][0])
    edges = [tuple(int(t) for t in e.split("-")) for e in g["edges"]]
    C = -np.ones((n, n))
    As = [np.eye(n)]
    b = [1.0]
    for i, j in edges:
        E = np.zeros((n, n))
        E[i, j] = E[j, i] = 1.0
        As.append(E)
        b.append(0.0)
    return problem_from_dense(C, As, b, [np.arange(n)]), -float(g["theta"][0])


def block_arrow_dense_pattern(l: int, d: int, h: int) -> np.ndarray:
    n = l * d + h
    P = np.zeros((n, n), dtype=bool)
    for k in range(l):
        idx = np.r_[k * d:(k + 1) * d, l * d:n]
        P[np.ix_(idx, idx)] = True
    return P


def block_arrow_cliques(l: int, d: int, h: int) -> list:
    n = l * d + h
    return [np.r_[k * d:(k + 1) * d, l * d:n].astype(np.int32) for k in range(l)]


def trace_one_block_arrow(l=3, d=3, h=2, seed=5) -> tuple[dict, float]:
    """min <C, X> s.t. tr X = 1, X ⪰ 0 on a block-arrow C: optimum is λ_min(C)."""
    rng = np.random.default_rng(seed)
    P = block_arrow_dense_pattern(l, d, h)
    n = P.shape[0]
    C = rng.standard_normal((n, n))
    C = (C + C.T) / 2 * P
    # keep every pattern entry structurally nonzero
    C[P & (C == 0)] = 0.5
    lam_min = float(np.linalg.eigvalsh(C)[0])
    return problem_from_dense(C, [np.eye(n)], [1.0], block_arrow_cliques(l, d, h)), lam_min


def random_block_arrow(l=3, d=3, h=2, m=6, seed=11, density=0.5) -> dict:
    """A small feasible block-arrow SDP with dense data on the pattern (for dense-vs-decomposed)."""
    rng = np.random.default_rng(seed)
    P = block_arrow_dense_pattern(l, d, h)
    n = P.shape[0]
    G = rng.standard_normal((n, n)) / np.sqrt(n)
    X0 = G @ G.T
    As = []
    for _ in range(m):
        A = rng.standard_normal((n, n)) * (rng.random((n, n)) < density)
        A = np.tril(A) + np.tril(A, -1).T
        As.append(A * P)
    b = [float(np.sum(A * X0)) for A in As]
    Z = rng.standard_normal((n, n))
    Z = np.tril(Z, -1)
    Z = (Z + Z.T) * P
    Z += np.diag(np.abs(Z).sum(axis=1) + 1.0)
    y0 = rng.standard_normal(m)
    C = Z + sum(y * A for y, A in zip(y0, As))
    C[P & (C == 0)] = 1e-3
    return problem_from_dense(C, As, b, block_arrow_cliques(l, d, h))


def random_sparse_sdp(n=24, m=8, edge_density=0.12, seed=5, density=0.5) -> dict:
    """A small feasible SDP on a random non-chordal pattern (a cycle through all vertices plus
    random edges); ``cliques`` is None, so a chordal extension has to supply them."""
    rng = np.random.default_rng(seed)
    P = np.eye(n, dtype=bool)
    for i in range(n):
        j = (i + 1) % n
        P[i, j] = P[j, i] = True
    R = rng.random((n, n)) < edge_density
    R = np.tril(R, -1)
    P |= R | R.T
    G = rng.standard_normal((n, n)) / np.sqrt(n)
    X0 = G @ G.T
    As = []
    for _ in range(m):
        A = rng.standard_normal((n, n)) * (rng.random((n, n)) < density)
        A = np.tril(A) + np.tril(A, -1).T
        As.append(A * P)
    b = [float(np.sum(A * X0)) for A in As]
    Z = rng.standard_normal((n, n))
    Z = np.tril(Z, -1)
    Z = (Z + Z.T) * P
    Z += np.diag(np.abs(Z).sum(axis=1) + 1.0)
    y0 = rng.standard_normal(m)
    C = Z + sum(y * A for y, A in zip(y0, As))
    C[P & (C == 0)] = 1e-3
    d = problem_from_dense(C, As, b, [list(range(n))])
    d["cliques"] = None
    return d


def instance_arrays(inst) -> dict:
    """Coordinate arrays of a generated ``SDPInstance``."""
    return dict(n=inst.n, cliques=inst.cliques, A_ptr=inst.A_ptr, A_row=inst.A_row, A_col=inst.A_col,
                A_val=inst.A_val, b=inst.b, C_row=inst.C_row, C_col=inst.C_col, C_val=inst.C_val)


def _empty_matrix_part(n=0) -> dict:
    z32 = np.zeros(0, np.int32)
    return dict(n=n, cliques=[], A_row=z32, A_col=z32, A_val=np.zeros(0), C_row=z32, C_col=z32,
                C_val=np.zeros(0))


def random_conic(l=2, d=3, h=2, n_free=3, n_lin=5, soc_dims=(3, 4), m=6, seed=21, density=0.6,
                 soc_u_scale=0.5) -> dict:
    """A feasible problem over a block-arrow PSD part (none when l = 0) and the other cones: free,
    nonnegative and second-order variables. Built from interior points x0 (primal) and (y0, z0)
    (dual; z0 = 0 on the free variables, whose dual cone is {0}), so both have optima and they
    agree. soc_u_scale sets the size of the interior points' u parts (larger: iterates that leave
    the cones more often). Returns sdp_setup's arrays plus ``cones`` (the dict the oracle and
    sdp_setup_conic take)."""
    rng = np.random.default_rng(seed)
    soc_dims = [int(q) for q in soc_dims]
    nc = n_free + n_lin + sum(soc_dims)
    if l > 0:
        P = block_arrow_dense_pattern(l, d, h)
        n = P.shape[0]
        G = rng.standard_normal((n, n)) / np.sqrt(n)
        X0 = G @ G.T
        As = []
        for _ in range(m):
            A = rng.standard_normal((n, n)) * (rng.random((n, n)) < density)
            A = np.tril(A) + np.tril(A, -1).T
            As.append(A * P)
        Z = rng.standard_normal((n, n))
        Z = np.tril(Z, -1)
        Z = (Z + Z.T) * P
        Z += np.diag(np.abs(Z).sum(axis=1) + 1.0)
    Ac = rng.standard_normal((m, nc)) * (rng.random((m, nc)) < density)
    x0 = np.empty(nc)
    z0 = np.empty(nc)
    x0[:n_free] = rng.standard_normal(n_free)
    z0[:n_free] = 0.0
    x0[n_free:n_free + n_lin] = rng.uniform(0.5, 1.5, n_lin)
    z0[n_free:n_free + n_lin] = rng.uniform(0.5, 1.5, n_lin)
    o = n_free + n_lin
    for q in soc_dims:
        for v in (x0, z0):
            u = rng.standard_normal(q - 1) * soc_u_scale / np.sqrt(q)
            v[o] = np.linalg.norm(u) + rng.uniform(0.5, 1.5)
            v[o + 1:o + q] = u
        o += q
    y0 = rng.standard_normal(m)
    b = Ac @ x0
    c_cone = Ac.T @ y0 + z0
    if l > 0:
        b = b + np.array([float(np.sum(A * X0)) for A in As])
        C = Z + sum(y * A for y, A in zip(y0, As))
        C[P & (C == 0)] = 1e-3
        arrs = problem_from_dense(C, As, b, block_arrow_cliques(l, d, h))
    else:
        arrs = _empty_matrix_part()
        arrs.update(A_ptr=np.zeros(m + 1, np.int64), b=np.asarray(b, np.float64))
    ptr, var, val = [0], [], []
    for i in range(m):
        nz = np.flatnonzero(Ac[i])
        var.append(nz)
        val.append(Ac[i, nz])
        ptr.append(ptr[-1] + len(nz))
    arrs["cones"] = dict(n_free=n_free, n_lin=n_lin, soc_dims=soc_dims,
                         A_ptr=np.asarray(ptr, np.int64), A_var=np.concatenate(var).astype(np.int32),
                         A_val=np.concatenate(val).astype(np.float64), c=c_cone)
    return arrs


def cone_matrix(arrs) -> np.ndarray:
    """The constraint coefficients of the cone variables as a dense m x n_cone matrix."""
    cn = arrs["cones"]
    m = len(arrs["b"])
    nc = cn["n_free"] + cn["n_lin"] + sum(cn["soc_dims"])
    M = np.zeros((m, nc))
    for i in range(m):
        for t in range(cn["A_ptr"][i], cn["A_ptr"][i + 1]):
            M[i, cn["A_var"][t]] += cn["A_val"][t]
    return M


def cones_from_dense(Ac: np.ndarray, c, n_free=0, n_lin=0, soc_dims=()) -> dict:
    ptr, var, val = [0], [], []
    for i in range(Ac.shape[0]):
        nz = np.flatnonzero(Ac[i])
        var.append(nz)
        val.append(Ac[i, nz])
        ptr.append(ptr[-1] + len(nz))
    return dict(n_free=n_free, n_lin=n_lin, soc_dims=list(soc_dims), A_ptr=np.asarray(ptr, np.int64),
                A_var=np.concatenate(var).astype(np.int32) if var else np.zeros(0, np.int32),
                A_val=np.concatenate(val).astype(np.float64) if val else np.zeros(0),
                c=np.asarray(c, np.float64))


def lp_as_diagonal_sdp(Ac: np.ndarray, b, c) -> dict:
    """min cᵀw, Aw = b, w ≥ 0 as an SDP on a diagonal pattern: w_j = X_jj, singleton cliques."""
    n = Ac.shape[1]
    As = [np.diag(Ac[i]) for i in range(Ac.shape[0])]
    d = problem_from_dense(np.diag(np.asarray(c, np.float64)), As, b, [[j] for j in range(n)])
    d["cliques"] = [np.array([j], np.int32) for j in range(n)]
    return d


def socp_as_arrow_sdp(Ac: np.ndarray, b, c, n_lin: int, soc_dims) -> dict:
    """A problem over nonnegative and second-order variables as an SDP: w_j ≥ 0 is a 1 x 1 block,
    and (t, u) ∈ Q^q iff the arrow matrix [[t, uᵀ], [u, t I]] is PSD, imposed on a q x q block
    by equality constraints (equal diagonal, zero off-diagonal outside the first column)."""
    n = n_lin + sum(soc_dims)
    m0 = Ac.shape[0]
    cost = np.zeros((n, n))
    rows = [np.zeros((n, n)) for _ in range(m0)]
    bb = list(np.asarray(b, np.float64))
    cliques = []

    def put(M, var_pos, coef):
        i, j = var_pos
        if i == j:
            M[i, i] += coef
        else:
            M[i, j] += 0.5 * coef
            M[j, i] += 0.5 * coef

    pos = [(j, j) for j in range(n_lin)]
    cliques += [[j] for j in range(n_lin)]
    o = n_lin
    extra = []
    for q in soc_dims:
        pos.append((o, o))
        pos += [(o + i, o) for i in range(1, q)]
        cliques.append(list(range(o, o + q)))
        for i in range(1, q):
            E = np.zeros((n, n))
            E[o + i, o + i] = 1.0
            E[o, o] = -1.0
            extra.append(E)
            for k in range(1, i):
                E = np.zeros((n, n))
                E[o + i, o + k] = E[o + k, o + i] = 0.5
                extra.append(E)
        o += q
    for v, p in enumerate(pos):
        put(cost, p, c[v])
        for i in range(m0):
            put(rows[i], p, Ac[i, v])
    As = rows + extra
    bb += [0.0] * len(extra)
    d = problem_from_dense(cost, As, bb, cliques)
    return d


def near_dependent_block_arrow(l=4, d=3, h=2, m=8, delta=1e-4, seed=17) -> dict:
    """A feasible block-arrow SDP whose last constraint is the first one plus delta times a
    random matrix on the pattern: two nearly dependent rows of A, so that A D⁻¹ Aᵀ has condition
    number of order 1/delta²."""
    rng = np.random.default_rng(seed)
    P = block_arrow_dense_pattern(l, d, h)
    n = P.shape[0]
    G = rng.standard_normal((n, n)) / np.sqrt(n)
    X0 = G @ G.T
    As = []
    for _ in range(m - 1):
        A = rng.standard_normal((n, n)) * (rng.random((n, n)) < 0.5)
        A = np.tril(A) + np.tril(A, -1).T
        As.append(A * P)
    R = rng.standard_normal((n, n))
    R = (np.tril(R) + np.tril(R, -1).T) * P
    As.append(As[0] + delta * R)
    b = [float(np.sum(A * X0)) for A in As]
    Z = rng.standard_normal((n, n))
    Z = np.tril(Z, -1)
    Z = (Z + Z.T) * P
    Z += np.diag(np.abs(Z).sum(axis=1) + 1.0)
    y0 = rng.standard_normal(m)
    C = Z + sum(y * A for y, A in zip(y0, As))
    C[P & (C == 0)] = 1e-3
    return problem_from_dense(C, As, b, block_arrow_cliques(l, d, h))


def messy_constraints(arrs: dict, seed=3, split=0.3) -> dict:
    """The same problem with A given the untidy way a caller may give it: every constraint's
    entries shuffled, a share of them split into two halves (duplicates that add back exactly),
    explicit zeros added on the diagonal, and a pair +x, -x added on a diagonal position the
    constraint does not use (a duplicate that cancels). The merged CSR is then bit for bit that
    of the tidy problem."""
    rng = np.random.default_rng(seed)
    ptr, rows, cols, vals = (np.asarray(arrs[k]) for k in ("A_ptr", "A_row", "A_col", "A_val"))
    verts = np.unique(np.concatenate([np.asarray(c) for c in arrs["cliques"]]))
    out_r, out_c, out_v, out_p = [], [], [], [0]
    for i in range(len(ptr) - 1):
        r, c, v = rows[ptr[i]:ptr[i + 1]], cols[ptr[i]:ptr[i + 1]], vals[ptr[i]:ptr[i + 1]]
        halves = rng.random(len(v)) < split
        rr = np.concatenate([r, r[halves]])
        cc = np.concatenate([c, c[halves]])
        vv = np.concatenate([np.where(halves, v / 2, v), v[halves] / 2])
        used = set(zip(r.tolist(), c.tolist()))
        free = [int(d) for d in verts if (int(d), int(d)) not in used]
        zeros = rng.choice(verts, size=min(3, len(verts)), replace=False)
        rr = np.concatenate([rr, zeros]); cc = np.concatenate([cc, zeros]); vv = np.concatenate([vv, np.zeros(len(zeros))])
        if free:
            d = free[int(rng.integers(len(free)))]
            x = float(rng.standard_normal())
            rr = np.concatenate([rr, [d, d]]); cc = np.concatenate([cc, [d, d]]); vv = np.concatenate([vv, [x, -x]])
        perm = rng.permutation(len(vv))
        out_r.append(rr[perm]); out_c.append(cc[perm]); out_v.append(vv[perm])
        out_p.append(out_p[-1] + len(vv))
    return dict(arrs, A_ptr=np.asarray(out_p, np.int64), A_row=np.concatenate(out_r).astype(np.int32),
                A_col=np.concatenate(out_c).astype(np.int32), A_val=np.concatenate(out_v).astype(np.float64))
