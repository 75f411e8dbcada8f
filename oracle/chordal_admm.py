"""Plain FP64 CPU oracle of the decomposed ADMM (Algorithms 1 and 2 of the paper).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py``; never by the CUDA library. It is slow on purpose and follows the paper's notation:

* ``x = vec(X)`` lives on the ORDERED pattern pairs ``E = ∪_k C_k × C_k`` (both triangles), stacked
  column by column (Section III.A, "vec ... the stack of its columns"), so ``⟨c, x⟩ = ⟨C, X⟩``.
* ``E_k`` selects the vertices of clique ``C_k`` in ascending order (Section II.B); the block
  ``x_k = vec(E_k X E_kᵀ) = H_k x`` with ``H_k = E_k ⊗ E_k`` (Section III.A) is a full ``s×s`` block
  stored column-major, realised here as an index array into ``x``.
* ``D = Σ_k H_kᵀ H_k`` is diagonal (Section III.B.1): entry ``e`` counts the cliques covering it.

Library primitives used as single steps: ``numpy.linalg.eigh`` (eigendecomposition inside the PSD
projection), ``numpy.linalg.cholesky`` and ``scipy.linalg.solve_triangular`` (the cached factorisation
of ``A D⁻¹ Aᵀ`` and its two triangular solves), ``scipy.sparse`` products (``A v`` and ``Aᵀ y``).

Readings where the paper is silent (each one also listed in the design notes):

* Stopping measures (Section III.B, Boyd et al. 2011 §3.3 is cited but not restated):
  primal form ``ε_p = ‖[x_k − H_k x]‖ / max(‖[x_k]‖, ‖[H_k x]‖, 1e-12)`` and
  ``ε_d = ρ‖Σ H_kᵀ(x_k⁺ − x_k)‖ / max(‖Σ H_kᵀ λ_k⁺‖, 1e-12)``; dual form
  ``ε_p = ‖[z_k − v_k]‖ / max(‖[z_k]‖, ‖[v_k]‖, 1e-12)`` and
  ``ε_d = ρ‖[v_k⁺ − v_k]‖ / max(‖[λ_k⁺]‖, 1e-12)``. Norms are Euclidean over the stacked vectors.
  Iteration ``n`` stops the loop when ``max(ε_p, ε_d) < tol``. Each iteration also returns the
  four norms (``res_p``/``res_p_den``, ``res_d``/``res_d_den``) so that the tests can compare them
  with Boyd's residuals of the splitting, built from explicit matrices.
* Initial iterates are zero; the paper leaves them to the user.
* The affine step is solved by block elimination (the paper's "e.g."), with ``A D⁻¹ Aᵀ`` factored once.
* Eq. (DualMultUpdate) is printed as ``λ_k = ρ H_k x``; substituting Eq. (vkEqn) into
  Eq. (MultUpdateDualSDP) gives ``λ_k = −ρ H_k x``, which is what Algorithm 2 uses here.
* ``Σ_k H_kᵀ(·)`` adds clique contributions in ascending ``k`` starting from zero.
* ``ρ⁻¹`` is formed once as ``1/ρ`` and multiplies, as the paper writes ``ρ⁻¹λ_k`` and ``ρ⁻¹c``.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse


class OracleError(ValueError):
    """Invalid input: unsorted cliques, data outside the clique cover, or rank-deficient A."""

    def __init__(self, code: int, msg: str):
        super().__init__(msg)
        self.code = code


# ---------------------------------------------------------------------------------------------
# PSD projection, Eq. (XkUpdate) / Eq. (zkUpdate)
# ---------------------------------------------------------------------------------------------

def proj_psd(W: np.ndarray) -> np.ndarray:
    """Projection onto the PSD cone, P(W) = V max(Λ, 0) Vᵀ (Section III.B.2).

    ``W`` is a symmetric matrix (it is symmetrised first); the result is symmetrised too. The
    eigendecomposition is one library call.
    """
    W = 0.5 * (W + W.T)
    lam, V = np.linalg.eigh(W)
    X = (V * np.maximum(lam, 0.0)) @ V.T
    return 0.5 * (X + X.T)


def proj_soc(w: np.ndarray) -> np.ndarray:
    """Projection onto the second-order cone {(t, u) : ‖u‖ ≤ t} (the cone CDCS admits beside the
    PSD one, Section V): the point itself inside the cone, zero inside its polar, otherwise
    ((t + ‖u‖)/2) (1, u/‖u‖)."""
    t, u = float(w[0]), np.asarray(w[1:], dtype=np.float64)
    nu = float(np.sqrt(np.dot(u, u)))
    if nu <= t:
        return np.array(w, dtype=np.float64)
    if nu <= -t:
        return np.zeros(len(w))
    a = 0.5 * (t + nu)
    return np.concatenate([[a], (a / nu) * u])


def proj_cone(kind: str, w: np.ndarray, dual: bool) -> np.ndarray:
    """Projection onto a non-PSD cone block (primal form) or onto its dual cone (dual form).

    The free cone ℝ^q has the dual cone {0}; the nonnegative orthant and the second-order cone
    are self-dual.
    """
    if kind == "free":
        return np.zeros(len(w)) if dual else np.array(w, dtype=np.float64)
    if kind == "nonneg":
        return np.maximum(w, 0.0)
    if kind == "soc":
        return proj_soc(w)
    raise OracleError(-1, f"unknown cone {kind!r}")


def _project_item(item):
    """One block of an iteration's projections (Eqs. XkUpdate / zkUpdate): (kind, order, w, dual)."""
    kind, s, w, dual = item
    if kind == "psd":
        return _vec(proj_psd(_mat(w, s)))
    return proj_cone(kind, w, dual)


# The blocks' projections within an iteration are independent (Section III.B.2: "in parallel").
# They go through this order-preserving map, the builtin one unless a caller installs another
# (a process pool, for a timing baseline on every host core); the results do not depend on it.
_block_map = map


def set_block_map(fn) -> None:
    """Install an order-preserving map(fn, items) for the block projections (None: the builtin)."""
    global _block_map
    _block_map = map if fn is None else fn


def _project_blocks(sdp, ws, dual: bool = False) -> list:
    items = [(sdp.kinds[k], len(sdp.cliques[k]) if sdp.kinds[k] == "psd" else 0, ws[k], dual)
             for k in range(sdp.nblk)]
    return list(_block_map(_project_item, items))


def _mat(v: np.ndarray, s: int) -> np.ndarray:
    """vec⁻¹: column-major s×s matrix from its stacked columns."""
    return v.reshape(s, s, order="F")


def _vec(X: np.ndarray) -> np.ndarray:
    """vec: stack the columns of X."""
    return X.reshape(-1, order="F")


# ---------------------------------------------------------------------------------------------
# Decomposed problem data, Sections III.A and IV.A
# ---------------------------------------------------------------------------------------------

class ChordalSDP:
    """Vectorised decomposed SDP: c, A, b, the selectors H_k, D and the cached KKT factor.

    Inputs are the standard-form data (Section I): ``A_i`` and ``C`` in lower-triangle coordinate
    form (row >= col; off-diagonal entries stand for both (i,j) and (j,i)), ``b``, and the maximal
    cliques of the chordal aggregate pattern (Section III.A assumes them given).

    ``cones`` (optional) adds variables in the other cones CDCS accepts (Section V: ℝ^q, the
    nonnegative orthant, second-order cones; only the PSD cone is decomposed): a dict with
    ``n_free``, ``n_lin``, ``soc_dims`` (list), the constraint coefficients of the cone variables
    as a CSR by constraint ``A_ptr``, ``A_var``, ``A_val``, and their cost ``c`` (length
    n_free + n_lin + Σ soc_dims; variables ordered free, nonnegative, then each second-order cone
    as (t, u)). They are appended to ``x`` after the pattern pairs; each cone is one block (the
    free and the nonnegative variables one block each) whose selector picks its variables, so
    ``D`` is 1 on them. The block kinds are ``self.kinds``: "psd" for the cliques, then "free",
    "nonneg", "soc".
    """

    def __init__(self, n, cliques, A_ptr, A_row, A_col, A_val, b, C_row, C_col, C_val, cones=None):
        self.n = int(n)
        self.m = len(b)
        self.b = np.asarray(b, dtype=np.float64)
        self.cliques = [np.asarray(c, dtype=np.int64) for c in cliques]
        self.p = len(self.cliques)
        n = self.n
        for c in self.cliques:
            # E_k sorts clique vertices in the natural ordering (Section II.B).
            if len(c) == 0 or np.any(np.diff(c) <= 0) or c[0] < 0 or c[-1] >= n:
                raise OracleError(-2, "clique vertices must be distinct, ascending and in [0, n)")

        # Ordered pattern E = ∪ C_k × C_k, column-major: sort by (col, row) via key col*n + row.
        keys = np.unique(np.concatenate(
            [(c[None, :] * n + c[:, None]).ravel() for c in self.cliques])) if self.p else np.zeros(0, np.int64)
        self.keys = keys
        self.nE_mat = len(keys)
        cones = cones or {}
        nf, nl = int(cones.get("n_free", 0)), int(cones.get("n_lin", 0))
        qd = [int(q) for q in cones.get("soc_dims", [])]
        if nf < 0 or nl < 0 or any(q < 1 for q in qd):
            raise OracleError(-1, "cone sizes must be nonnegative and second-order cones non-empty")
        self.n_cone = nf + nl + sum(qd)
        # Cone variable j sits after the pattern pairs; as the diagonal pair (n + j, n + j) of a
        # virtual vertex it keeps the lower-pattern helpers below valid.
        virt = np.arange(n, n + self.n_cone, dtype=np.int64)
        self.E_row = np.concatenate([keys % n if n else keys, virt])
        self.E_col = np.concatenate([keys // n if n else keys, virt])
        self.nE = self.nE_mat + self.n_cone

        # H_k as index arrays: block entry (a, b) of vec(E_k X E_kᵀ) sits at a + b*s and selects
        # X[C_k(a), C_k(b)] (Section III.A, H_k = E_k ⊗ E_k).
        self.idx = []
        for c in self.cliques:
            s = len(c)
            a = np.tile(np.arange(s), s)          # row index within the block, fastest
            bb = np.repeat(np.arange(s), s)       # column index
            self.idx.append(np.searchsorted(keys, c[bb] * n + c[a]))

        # Cone blocks: one selector per cone over the appended variables.
        self.kinds = ["psd"] * self.p
        start = self.nE_mat
        for kind, q in [("free", nf), ("nonneg", nl)] + [("soc", q) for q in qd]:
            if q == 0:
                continue
            self.kinds.append(kind)
            self.idx.append(np.arange(start, start + q))
            start += q
        self.nblk = len(self.kinds)

        # D = Σ_k H_kᵀ H_k (Section III.B.1): diagonal, entry = number of cliques covering it.
        D = np.zeros(self.nE)
        for ix in self.idx:
            D[ix] += 1.0
        self.D = D

        # Data in vectorised form: c = vec(C) on E, A = [vec(A_1) ... vec(A_m)]ᵀ on E.
        self.c = self._full_from_lower(C_row, C_col, C_val)
        if self.n_cone:
            cc = cones.get("c")
            if cc is not None:
                self.c[self.nE_mat:] = np.asarray(cc, dtype=np.float64)
        A_ptr = np.asarray(A_ptr, dtype=np.int64)
        rows, cols, vals = [], [], []
        for i in range(self.m):
            sl = slice(A_ptr[i], A_ptr[i + 1])
            nz, v = self._full_from_lower(np.asarray(A_row)[sl], np.asarray(A_col)[sl],
                                          np.asarray(A_val)[sl], sparse=True)
            cols.append(nz)
            vals.append(v)
            rows.append(np.full(len(nz), i))
        if self.n_cone:
            cptr = np.asarray(cones["A_ptr"], dtype=np.int64)
            cvar = np.asarray(cones["A_var"], dtype=np.int64)
            cval = np.asarray(cones["A_val"], dtype=np.float64)
            if np.any(cvar < 0) or np.any(cvar >= self.n_cone):
                raise OracleError(-1, "cone variable index out of range")
            for i in range(self.m):
                sl = slice(cptr[i], cptr[i + 1])
                cols.append(self.nE_mat + cvar[sl])
                vals.append(cval[sl])
                rows.append(np.full(sl.stop - sl.start, i))
        self.A = scipy.sparse.csr_matrix(
            (np.concatenate(vals) if vals else np.zeros(0),
             (np.concatenate(rows) if rows else np.zeros(0, int),
              np.concatenate(cols) if cols else np.zeros(0, int))),
            shape=(self.m, self.nE))

        # KKT factorisation, cached before iterating (Section III.B.1): block elimination of
        # [D Aᵀ; A 0] needs the Cholesky factor of A D⁻¹ Aᵀ.
        M = (self.A @ scipy.sparse.diags(1.0 / D) @ self.A.T).toarray()
        self.M = M
        try:
            self.L = np.linalg.cholesky(M) if self.m > 0 else np.zeros((0, 0))
        except np.linalg.LinAlgError as exc:
            raise OracleError(-3, "A D^-1 A^T is not positive definite (A rank-deficient)") from exc

    # -- vectorisation helpers ----------------------------------------------------------------

    def _full_from_lower(self, rows, cols, vals, sparse=False):
        """Place lower-triangle data (i >= j) at both (i, j) and (j, i) of vec over E."""
        rows = np.asarray(rows, dtype=np.int64)
        cols = np.asarray(cols, dtype=np.int64)
        vals = np.asarray(vals, dtype=np.float64)
        if np.any(rows < cols):
            raise OracleError(-1, "coordinate data must be lower-triangular (row >= col)")
        n = self.n
        k1 = cols * n + rows
        k2 = rows * n + cols
        p1 = np.searchsorted(self.keys, k1)
        p2 = np.searchsorted(self.keys, k2)
        ok1 = (p1 < self.nE_mat) & (self.keys[np.minimum(p1, max(self.nE_mat - 1, 0))] == k1) \
            if self.nE_mat else np.zeros(len(k1), bool)
        if not np.all(ok1):
            raise OracleError(-2, "a data nonzero lies outside the union of clique blocks")
        full = np.zeros(self.nE)
        np.add.at(full, p1, vals)
        off = rows != cols
        np.add.at(full, p2[off], vals[off])
        if sparse:
            nz = np.unique(np.concatenate([p1, p2[off]]))
            return nz, full[nz]
        return full

    def lower_mask(self) -> np.ndarray:
        """Entries of E with row >= col, in column-major order (the lower pattern list)."""
        return self.E_row >= self.E_col

    def to_lower(self, x_full: np.ndarray) -> np.ndarray:
        """Values of a symmetric vec on the lower pattern, column-major order."""
        return x_full[self.lower_mask()]

    def from_lower(self, rows, cols, vals) -> np.ndarray:
        """Full vector from lower-pattern values; rows n + j (cone variable j, listed as the
        diagonal pair of a virtual vertex) go to the cone variables."""
        rows = np.asarray(rows, dtype=np.int64)
        cols = np.asarray(cols, dtype=np.int64)
        vals = np.asarray(vals, dtype=np.float64)
        cone = rows >= self.n
        full = self._full_from_lower(rows[~cone], cols[~cone], vals[~cone])
        full[self.nE_mat + (rows[cone] - self.n)] += vals[cone]
        return full

    def block_sizes(self):
        return [len(c) for c in self.cliques]

    def block_len(self, k: int) -> int:
        """Length of block k: s² for a clique (full column-major block), q for a cone."""
        return len(self.idx[k])

    def project(self, k: int, w: np.ndarray, dual: bool = False) -> np.ndarray:
        """Projection of block k (Eqs. XkUpdate / zkUpdate): P₊ on a clique block, the cone's own
        projection (its dual cone's in the dual form) on a cone block."""
        if self.kinds[k] == "psd":
            s = len(self.cliques[k])
            return _vec(proj_psd(_mat(w, s)))
        return proj_cone(self.kinds[k], w, dual)

    @staticmethod
    def block_to_packed(xk: np.ndarray, s: int) -> np.ndarray:
        """Full column-major s×s block → its lower triangle, column by column."""
        X = _mat(xk, s)
        return np.concatenate([X[j:, j] for j in range(s)])

    @staticmethod
    def packed_to_block(pk: np.ndarray, s: int) -> np.ndarray:
        X = np.zeros((s, s))
        pos = 0
        for j in range(s):
            X[j:, j] = pk[pos:pos + s - j]
            X[j, j:] = pk[pos:pos + s - j]
            pos += s - j
        return _vec(X)

    # -- the operators of the method -----------------------------------------------------------

    def H(self, k: int, x: np.ndarray) -> np.ndarray:
        """x_k = H_k x: the entries of X inside clique k (Section III.A)."""
        return x[self.idx[k]]

    def HT_sum(self, blocks) -> np.ndarray:
        """Σ_k H_kᵀ v_k, accumulating cliques in ascending k from zero (Section III.B.1)."""
        acc = np.zeros(self.nE)
        for k in range(self.nblk):
            acc[self.idx[k]] += blocks[k]
        return acc

    def kkt_solve(self, rhs1: np.ndarray, rhs2: np.ndarray):
        """Solve [D Aᵀ; A 0][x; y] = [rhs1; rhs2] (Eqs. OptCondMinYPrimal, OptCondMinYDual).

        Block elimination with the cached factor L Lᵀ = A D⁻¹ Aᵀ:
        y = (A D⁻¹ Aᵀ)⁻¹ (A D⁻¹ rhs1 − rhs2),  x = D⁻¹ (rhs1 − Aᵀ y).
        """
        t = self.A @ (rhs1 / self.D) - rhs2
        z = scipy.linalg.solve_triangular(self.L, t, lower=True)
        y = scipy.linalg.solve_triangular(self.L.T, z, lower=False)
        x = (rhs1 - self.A.T @ y) / self.D
        return x, y


# ---------------------------------------------------------------------------------------------
# Algorithms 1 and 2
# ---------------------------------------------------------------------------------------------

def _norm_blocks(blocks) -> float:
    return float(np.sqrt(sum(float(np.dot(v, v)) for v in blocks)))


def admm_init(sdp: ChordalSDP, form: str) -> dict:
    """Zero initial guesses (Algorithm 1 / 2 take them as inputs)."""
    zeros = [np.zeros(sdp.block_len(k)) for k in range(sdp.nblk)]
    st = dict(form=form, iter=0, x=np.zeros(sdp.nE), y=np.zeros(sdp.m),
              lam=[z.copy() for z in zeros])
    if form == "primal":
        st["xk"] = [z.copy() for z in zeros]
    elif form == "dual":
        st["zk"] = [z.copy() for z in zeros]
        st["vk"] = [z.copy() for z in zeros]
    else:
        raise OracleError(-1, f"unknown form {form!r}")
    return st


def primal_iteration(sdp: ChordalSDP, st: dict, rho: float) -> dict:
    """One pass of Algorithm 1: x-update, clique projections, multipliers, residuals."""
    rinv = 1.0 / rho
    # Eq. (OptCondMinYPrimal): right-hand side Σ H_kᵀ(x_k + ρ⁻¹λ_k) − ρ⁻¹c and b.
    K = range(sdp.nblk)
    r = sdp.HT_sum([st["xk"][k] + rinv * st["lam"][k] for k in K]) - rinv * sdp.c
    x, y = sdp.kkt_solve(r, sdp.b)
    # Eq. (XkUpdate): x_k = vec P_k[vec⁻¹(H_k x − ρ⁻¹λ_k)].
    u = [sdp.H(k, x) for k in K]
    xk_new = _project_blocks(sdp, [u[k] - rinv * st["lam"][k] for k in K])
    # Eq. (LambdakUpdate): λ_k += ρ (x_k − H_k x).
    lam_new = [st["lam"][k] + rho * (xk_new[k] - u[k]) for k in K]
    # Residuals (reading of Section III.B's stopping test, see module docstring).
    pri = _norm_blocks([xk_new[k] - u[k] for k in K])
    pri_den = max(_norm_blocks(xk_new), _norm_blocks(u), 1e-12)
    dres = sdp.HT_sum([xk_new[k] - st["xk"][k] for k in K])
    dual_den = max(float(np.linalg.norm(sdp.HT_sum(lam_new))), 1e-12)
    dual_num = rho * float(np.linalg.norm(dres))
    out = dict(st)
    out.update(iter=st["iter"] + 1, x=x, y=y, xk=xk_new, lam=lam_new, r=r, u=u,
               eps_p=pri / pri_den, eps_d=dual_num / dual_den,
               res_p=pri, res_p_den=pri_den, res_d=dual_num, res_d_den=dual_den,
               obj_primal=float(np.dot(sdp.c, x)), obj_dual=float(np.dot(sdp.b, -rho * y)))
    return out


def dual_iteration(sdp: ChordalSDP, st: dict, rho: float) -> dict:
    """One pass of Algorithm 2: projections, (y, x), v_k, multipliers, residuals."""
    rinv = 1.0 / rho
    # Eq. (zkUpdate): z_k = vec P_k[vec⁻¹(v_k − ρ⁻¹λ_k)].
    K = range(sdp.nblk)
    zk = _project_blocks(sdp, [st["vk"][k] - rinv * st["lam"][k] for k in K], dual=True)
    # Eq. (OptCondMinYDual): right-hand side c − Σ H_kᵀ(z_k + ρ⁻¹λ_k) and −ρ⁻¹b.
    r = sdp.c - sdp.HT_sum([zk[k] + rinv * st["lam"][k] for k in K])
    x, y = sdp.kkt_solve(r, -(rinv * sdp.b))
    # Eq. (vkEqn): v_k = z_k + ρ⁻¹λ_k + H_k x.
    u = [sdp.H(k, x) for k in K]
    vk_new = [zk[k] + rinv * st["lam"][k] + u[k] for k in K]
    # Eq. (DualMultUpdate) with the sign that Eq. (MultUpdateDualSDP) implies: λ_k = −ρ H_k x.
    lam_new = [-rho * u[k] for k in K]
    # The general update of Eq. (MultUpdateDualSDP), kept for the identity check in the tests.
    lam_general = [st["lam"][k] + rho * (zk[k] - vk_new[k]) for k in K]
    pri = _norm_blocks([zk[k] - vk_new[k] for k in K])
    pri_den = max(_norm_blocks(zk), _norm_blocks(vk_new), 1e-12)
    dres = _norm_blocks([vk_new[k] - st["vk"][k] for k in K])
    dual_den = max(_norm_blocks(lam_new), 1e-12)
    out = dict(st)
    out.update(iter=st["iter"] + 1, x=x, y=y, zk=zk, vk=vk_new, lam=lam_new, r=r, u=u,
               lam_general=lam_general,
               eps_p=pri / pri_den, eps_d=rho * dres / dual_den,
               res_p=pri, res_p_den=pri_den, res_d=rho * dres, res_d_den=dual_den,
               obj_dual=float(np.dot(sdp.b, y)), obj_primal=float(np.dot(sdp.c, -rho * x)))
    return out


def admm_solve(sdp: ChordalSDP, form: str = "primal", rho: float = 1.0, tol: float = 1e-4,
               max_iter: int = 2000, state: dict | None = None, history: bool = False) -> dict:
    """Run Algorithm 1 (primal) or 2 (dual) until max(ε_p, ε_d) < tol or ``max_iter`` iterations.

    Returns the final state plus ``iters``, ``status`` (0 converged, 1 iteration cap reached,
    -5 a non-finite residual), the residuals and both objective estimates. In the primal form the
    objective is ⟨c, x⟩ at the affine iterate and the dual estimate is bᵀ(−ρy); in the dual form it is
    bᵀy and the primal estimate ⟨c, −ρx⟩.
    """
    st = admm_init(sdp, form) if state is None else state
    step = primal_iteration if form == "primal" else dual_iteration
    hist = []
    status = 1
    for _ in range(max_iter):
        st = step(sdp, st, rho)
        if history:
            hist.append((st["eps_p"], st["eps_d"], st["obj_primal"], st["obj_dual"]))
        if not (np.isfinite(st["eps_p"]) and np.isfinite(st["eps_d"])):
            status = -5
            break
        e = max(st["eps_p"], st["eps_d"])
        if e < tol:
            status = 0
            break
    st = dict(st)
    st.update(iters=st["iter"], status=status, history=hist)
    return st


def primal_solution(sdp: ChordalSDP, st: dict, rho: float):
    """(X on E, y, Z on E) of the SDP pair from the ADMM iterates (stationarity at a fixed point).

    Primal form: X = x, y_SDP = −ρy, Z = Σ H_kᵀ λ_k. Dual form: X = −ρx, y_SDP = y,
    Z = Σ H_kᵀ z_k.
    """
    if st["form"] == "primal":
        return st["x"], -rho * st["y"], sdp.HT_sum(st["lam"])
    return -rho * st["x"], st["y"], sdp.HT_sum(st["zk"])
