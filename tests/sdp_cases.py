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
