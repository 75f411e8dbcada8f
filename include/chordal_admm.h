/*
 * chordal_admm.h — C ABI of the GB300 (sm_103a) hot path of chordally decomposed ADMM for sparse
 * semidefinite programs (Zheng, Fantuzzi, Papachristodoulou, Goulart, Wynn, "Fast ADMM for
 * Semidefinite Programs with Chordal Sparsity").
 *
 * Problem (Section I, Eqs. PrimalSDP / DualSDP):
 *     min <C, X>  s.t.  <A_i, X> = b_i (i = 1..m),  X PSD          (primal standard form)
 *     max <b, y>  s.t.  sum_i y_i A_i + Z = C,       Z PSD          (dual standard form)
 * with an aggregate sparsity pattern whose chordal graph has maximal cliques C_1..C_p (Section III.A).
 *
 * Conventions shared by every entry point:
 *   - Symmetric matrices are passed in lower-triangle coordinate form: entry k is (row[k], col[k],
 *     val[k]) with row >= col, 0-based; an off-diagonal entry stands for both (i,j) and (j,i).
 *     Repeated coordinates are summed.
 *   - E_L is the lower pattern: all pairs (i >= j) with i, j in a common clique, in column-major
 *     order (by column, then row). Vectors "on E_L" have one entry per such pair.
 *   - Clique blocks are stored "packed": clique k's s_k x s_k block keeps its lower triangle column
 *     by column (LAPACK 'L' packed order), blocks one after another in clique order. S_L is the
 *     total length, sum_k s_k (s_k + 1) / 2. Clique vertices must be strictly ascending (the
 *     paper's E_k sorts them in natural order, Section II.B).
 *   - Pointers are HOST pointers unless the argument says "device". The library copies host
 *     inputs; the caller keeps ownership of everything it passes.
 *   - Every function returns an int status: 0 success, > 0 a non-fatal outcome, < 0 an error
 *     (see SDP_* below). No C++ exception crosses this boundary. sdp_last_error() gives a
 *     message for the most recent error on the calling thread.
 *   - cuda_stream is a cudaStream_t passed as void* (NULL = the legacy default stream).
 */
#ifndef CHORDAL_ADMM_H
#define CHORDAL_ADMM_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------------- */
#define SDP_OK               0   /* converged (max(eps_p, eps_d) < tol) or call succeeded   */
#define SDP_MAX_ITER         1   /* iteration budget of the call used without convergence   */
#define SDP_ERR_ARG         -1   /* bad argument (size, pointer, option, row < col)          */
#define SDP_ERR_CLIQUE      -2   /* cliques unsorted / out of range, or a data nonzero is not
                                    covered by any clique block                              */
#define SDP_ERR_NOT_PD      -3   /* A D^-1 A^T not positive definite (A rank-deficient)      */
#define SDP_ERR_CUDA        -4   /* a CUDA runtime call failed                               */
#define SDP_ERR_NAN         -5   /* a residual or objective became NaN/Inf                   */
#define SDP_ERR_TIMEOUT     -6   /* a host wait on the device exceeded its time limit        */
#define SDP_ERR_UNSUPPORTED -7   /* size beyond what the kernels support (see limits below)  */

/* Limits of this build: clique size <= SDP_MAX_CLIQUE, m <= SDP_MAX_CONSTRAINTS, nnz(A) and S_L
 * below 2^31. */
#define SDP_MAX_CLIQUE       96
#define SDP_MAX_CONSTRAINTS  16384

/* ---- options ------------------------------------------------------------------------------ */
#define SDP_PRIMAL    0   /* Algorithm 1: ADMM on the decomposed primal (Eq. PrimalVectorForm) */
#define SDP_DUAL      1   /* Algorithm 2: ADMM on the decomposed dual (Eq. DualDecomposedSDPVector) */
#define SDP_PROJ_FP64 0   /* clique eigendecompositions and reconstructions in FP64            */
#define SDP_PROJ_FP32 1   /* ... in FP32; everything else stays FP64                            */

typedef struct sdp_ctx* sdp_handle;   /* opaque; owns all of its device memory */

typedef struct {
    double rho;        /* ADMM penalty rho > 0 (Eqs. AugLagrPrimal / AugLagrDual)                */
    double tol;        /* stop once max(eps_p, eps_d) < tol; tol <= 0 never stops early          */
    int max_iter;      /* iteration cap of one admm_solve call (the paper uses 2000)             */
    int check_every;   /* admm_solve reads the device stop flag every check_every iterations;
                          iterations after convergence inside that window are skipped on the
                          device, so the results of one problem do not depend on it (0 = default
                          16). A batch is re-planned at these points for the problems still
                          iterating, which can move its results by rounding.                   */
    int form;          /* SDP_PRIMAL or SDP_DUAL                                                 */
    int prec;          /* SDP_PROJ_FP64 or SDP_PROJ_FP32                                         */
    int flags;         /* 0 or SDP_FLAG_HOST_KKT                                                 */
} admm_opts;

/* By default sdp_setup and sdp_setup_conic form A D^-1 A^T, its Cholesky factor and inverse on the
 * GPU (FP64) when 64 <= m <= 4096 and no column of A on the pattern has more than 4096 nonzeros;
 * batches and other sizes take the host. SDP_FLAG_HOST_KKT keeps them on the host always (the two
 * agree to rounding; sdp_set_opts does not change where an existing handle was factored). */
#define SDP_FLAG_HOST_KKT 1

typedef struct {
    int iters;         /* iterations performed on this handle since the last admm_reset          */
    int status;        /* SDP_OK, SDP_MAX_ITER or SDP_ERR_NAN (same as the return value)         */
    double eps_p;      /* relative primal residual of the last iteration                         */
    double eps_d;      /* relative dual residual of the last iteration                           */
    double obj_primal; /* primal objective estimate <C, X>                                       */
    double obj_dual;   /* dual objective estimate <b, y>                                         */
    double seconds;    /* host wall-clock time of the call                                       */
    long long kernel_launches; /* kernels this call launched (graph nodes included; kernels of
                                  iterations after convergence start and return at once)          */
} admm_result;

typedef struct {
    int n, m, p, max_clique;
    long long nE_lower;    /* |E_L| */
    long long S_lower;     /* S_L   */
    long long nnz_A;       /* stored nonzeros of A on E_L (after merging duplicates) */
    int batch;             /* problems in the handle (1 for sdp_setup, count for sdp_setup_batch) */
    long long n_cone;      /* variables in non-PSD cones (sdp_setup_conic); they are the last
                              n_cone entries of nE_lower and positions of S_lower              */
} sdp_sizes;

/* One problem of a batch: the arguments of sdp_setup, with the same meaning, in a struct. */
typedef struct {
    int n, m;
    const long long* A_ptr;
    const int* A_row;
    const int* A_col;
    const double* A_val;
    const double* b;
    long long C_nnz;
    const int* C_row;
    const int* C_col;
    const double* C_val;
    long long pat_nnz;
    const int* pat_row;
    const int* pat_col;
    int p;
    const int* clique_ptr;
    const int* clique_vtx;
} sdp_problem;

/* Residual definitions (the paper cites Boyd et al. 2011 for them without restating; this build
 * reads them as follows, with Euclidean norms over the full symmetric vectors):
 *   primal form: eps_p = ||[x_k - H_k x]|| / max(||[x_k]||, ||[H_k x]||, 1e-12),
 *                eps_d = rho ||sum_k H_k^T (x_k+ - x_k)|| / max(||sum_k H_k^T lambda_k||, 1e-12);
 *   dual form:   eps_p = ||[z_k - v_k]|| / max(||[z_k]||, ||[v_k]||, 1e-12),
 *                eps_d = rho ||[v_k+ - v_k]|| / max(||[lambda_k]||, 1e-12).                   */

/* ---- setup (Algorithms 1-2, "Setup: chordal decomposition, KKT factorization") -------------
 * Builds the clique index maps (H_k as gather indices and their inverse as a CSR scatter map),
 * D = sum_k H_k^T H_k (Section III.B.1), A on E_L in CSR and CSC form, M = A D^-1 A^T and its
 * Cholesky factor L (computed once and cached; the per-iteration solve uses (L L^T)^-1 = L^-T L^-1
 * formed here, one product instead of two triangular ones), uploads everything to the device and
 * zeroes the iterates.
 *   n, m        matrix order and number of constraints (1 <= m <= SDP_MAX_CONSTRAINTS)
 *   A_ptr[m+1]  constraint i owns coordinates A_ptr[i] .. A_ptr[i+1]-1 of A_row/A_col/A_val
 *   b[m]        right-hand side
 *   C_*         cost matrix C, C_nnz coordinates
 *   pat_*       optional extra pattern coordinates that must be covered (may be NULL/0)
 *   clique_ptr[p+1], clique_vtx  the maximal cliques, vertices strictly ascending; p = 0 with
 *               NULL arrays: those of a chordal extension of the aggregate pattern
 *               (sdp_chordal_cliques on C, every A_i and pat_*)
 *   opts        initial options (copied)
 *   out         receives the handle on success
 * Errors: SDP_ERR_ARG, SDP_ERR_CLIQUE, SDP_ERR_NOT_PD, SDP_ERR_UNSUPPORTED, SDP_ERR_CUDA. */
int sdp_setup(int n, int m, const long long* A_ptr, const int* A_row, const int* A_col,
              const double* A_val, const double* b,
              long long C_nnz, const int* C_row, const int* C_col, const double* C_val,
              long long pat_nnz, const int* pat_row, const int* pat_col,
              int p, const int* clique_ptr, const int* clique_vtx,
              const admm_opts* opts, sdp_handle* out);

/* ---- batches of independent problems (not in the paper: many SDPs solved in one set of launches)
 * sdp_setup_batch builds one handle for `count` independent problems. The handle holds their
 * block-diagonal union: the vertices, constraints, cliques, E_L entries and packed positions of
 * problem q follow those of problem q-1 (sdp_batch_layout gives the offsets), so every vector the
 * handle reads or returns (sdp_get_state, sdp_set_state, sdp_get_solution, sdp_get_maps, the
 * device buffers of sdp_gather / sdp_scatter) is the concatenation of the problems' vectors, and
 * each problem's (A D^-1 A^T)^-1 is its own block. Every kernel of an iteration covers all problems at once;
 * no CTA works on two problems. Each problem keeps its own residuals, objectives and stop test
 * (the definitions below): a problem whose residuals fall below tol, or become NaN/Inf, is frozen
 * (its iterates stop changing) at that iteration, which is what a separate solve of it would
 * return. A call ends when every problem is frozen or its budget is used. Once half of the
 * problems are frozen, the launches are re-planned (at a stop-flag check) to cover only the rest. For a batch,
 * admm_result.status is SDP_ERR_NAN if a problem stopped on NaN/Inf, else SDP_OK if all converged,
 * else SDP_MAX_ITER; eps_p / eps_d are the maxima over the problems and the objectives their sums
 * (the objectives of the union). admm_reset, sdp_set_state and sdp_set_opts unfreeze every problem.
 * Errors as sdp_setup (the message names the failing problem); count >= 1. A handle from
 * sdp_setup behaves as a batch of one, except that it is never frozen (a later admm_iterate
 * continues from the converged state). */
int sdp_setup_batch(int count, const sdp_problem* problems, const admm_opts* opts, sdp_handle* out);

/* Offsets of each problem inside the handle's vectors, [batch + 1] host arrays each (any may be
 * NULL): vertices, constraints, cliques, E_L entries and packed positions. */
int sdp_batch_layout(sdp_handle h, int* vtx_off, int* row_off, int* clique_off, long long* ent_off,
                     long long* pos_off);

/* Per-problem outcome of the iterations so far, [batch] host arrays each (any may be NULL): the
 * iteration count (the iteration at which the problem was frozen, else all iterations run), its
 * status (SDP_OK converged, SDP_MAX_ITER, SDP_ERR_NAN), residuals and objectives of its last
 * iteration. */
int sdp_batch_results(sdp_handle h, int* iters, int* status, double* eps_p, double* eps_d,
                      double* obj_primal, double* obj_dual);

/* ---- products with other cones (Section V: CDCS accepts products of R^q, the nonnegative
 * orthant, second-order cones and the PSD cone, and decomposes only the PSD one)
 * The problem becomes  min <C, X> + c^T x  s.t.  <A_i, X> + a_i^T x = b_i,  X in S^n_+(E, ?),
 * x in R^{n_free} x R_+^{n_lin} x Q^{q_1} x ... x Q^{q_k}  with Q^q = {(t, u) : ||u|| <= t}.
 * The cone variables are appended to the pattern entries: the handle's entry vector is E_L
 * followed by them (sdp_get_maps reports cone variable j as the diagonal pair (n + j, n + j)),
 * and its packed block vector is the clique blocks followed by one block per cone (all free
 * variables one block, all nonnegative ones one block, then each second-order cone), each block
 * the cone's own variables in order, so D = 1 on them and their weight in every inner product is
 * 1. Each iteration projects these blocks onto their cone (primal form) or its dual cone (dual
 * form: {0} for the free block, the others are self-dual); the affine step, the multiplier
 * updates and the residuals are those of the SDP with the longer vectors. */
typedef struct {
    int n_free;                 /* free variables (first)                                        */
    int n_lin;                  /* nonnegative variables (next)                                  */
    int n_soc;                  /* number of second-order cones (last, in order)                 */
    const int* soc_dims;        /* [n_soc] their dimensions q_j >= 1 (t first, then u)           */
    const long long* A_ptr;     /* [m+1] constraint i owns terms A_ptr[i] .. A_ptr[i+1]-1         */
    const int* A_var;           /* cone variable of each term, 0 <= j < n_cone (duplicates add)  */
    const double* A_val;        /* coefficient of each term                                      */
    const double* c;            /* [n_cone] cost of the cone variables (NULL: zero)              */
} sdp_cones;

/* sdp_setup for a problem with cone variables beside the PSD matrix. `problem` holds the matrix
 * part as in sdp_setup (n = 0 with p = 0 and no matrix data: no PSD part at all); `cones` may be
 * NULL (then this is sdp_setup). Host pointers, copied. Not available for batches;
 * sdp_unrolled_forward / sdp_unrolled_backward take the cone blocks too (their projections'
 * derivatives: identity, the mask of w > 0, the second-order closed form).
 * Errors: as sdp_setup; SDP_ERR_ARG for negative cone sizes, a second-order cone of dimension
 * < 1, no variables at all, or a cone variable index out of range. */
int sdp_setup_conic(const sdp_problem* problem, const sdp_cones* cones, const admm_opts* opts,
                    sdp_handle* out);

/* Host-only planning of a problem (needs no GPU): runs sdp_setup_conic's host work (validation,
 * chordal extension when p = 0, index maps, A D^-1 A^T and its factorization) and reports the sizes
 * a handle would have (batch = 1), so a caller can check a problem and size its device memory
 * first. cones may be NULL. Errors: as sdp_setup_conic, except SDP_ERR_CUDA. */
int sdp_plan(const sdp_problem* problem, const sdp_cones* cones, sdp_sizes* out);

/* Chordal extension of a sparse symmetric pattern (Section II.A: a non-chordal aggregate pattern is
 * first extended to a chordal one; the paper leaves the extension to heuristics) and the maximal
 * cliques of the extension. Ordering by maximum cardinality search (ties: smallest vertex index),
 * which adds nothing to a chordal pattern; symbolic elimination in that order; maximal cliques
 * listed in elimination order of their defining vertex, vertices ascending.
 *   n, nnz, row[nnz], col[nnz]  the pattern (host; either triangle or both; diagonal ignored)
 *   p, nvtx, fill               outputs: number of cliques, total clique length, added lower pairs
 *   clique_ptr[p+1], clique_vtx[nvtx]  outputs, or NULL to ask for the sizes first
 * Host-only; needs no GPU. sdp_setup and sdp_setup_batch call it themselves when given p = 0
 * (and NULL clique arrays), on the union of the coordinates of C, every A_i and the extra pattern.
 * Errors: SDP_ERR_ARG (bad sizes or indices), SDP_ERR_ARG "too small" when the arrays passed are
 * smaller than the sizes (call with NULL first). */
int sdp_chordal_cliques(int n, long long nnz, const int* row, const int* col, int* p, long long* nvtx,
                        long long* fill, int* clique_ptr, int* clique_vtx, int capacity_p,
                        long long capacity_vtx);

/* Replace the options (rho, tol, form, precision may all change; the KKT factor does not depend
 * on them). Takes effect at the next admm_iterate / admm_solve. Does not reset the iterates. */
int sdp_set_opts(sdp_handle h, const admm_opts* opts);

/* Zero the iterates (x, y, clique blocks, multipliers) and the iteration counter. Stream-ordered. */
int admm_reset(sdp_handle h, void* cuda_stream);

/* Run up to n_iters ADMM iterations (Algorithm 1 or 2 by opts.form) from the handle's current
 * state, stopping early once max(eps_p, eps_d) < tol. Each iteration runs as captured CUDA graphs
 * on cuda_stream; the call returns after the stream has finished them.
 * Returns SDP_OK (converged), SDP_MAX_ITER (budget used), SDP_ERR_NAN, or an error. */
int admm_iterate(sdp_handle h, int n_iters, void* cuda_stream, admm_result* out);

/* admm_iterate with n_iters = opts.max_iter, from the current state (call admm_reset first for a
 * cold start). */
int admm_solve(sdp_handle h, void* cuda_stream, admm_result* out);

int sdp_get_sizes(sdp_handle h, sdp_sizes* out);

/* SDP-level solution estimates on E_L (host outputs, any may be NULL), by stationarity of the KKT
 * systems at a fixed point: primal form X = x, y = -rho*y_admm, Z = sum_k H_k^T lambda_k; dual form
 * X = -rho*x, y = y_admm, Z = sum_k H_k^T z_k. X_lower and Z_lower have nE_lower entries. */
int sdp_get_solution(sdp_handle h, double* X_lower, double* y, double* Z_lower);

/* Raw ADMM iterates (host outputs, any may be NULL): x on E_L (the affine iterate), y (m), and
 * three packed block vectors of length S_L. Primal form: blk_a = x_k, blk_b = lambda_k, blk_c
 * unused. Dual form: blk_a = z_k, blk_b = lambda_k, blk_c = v_k. */
int sdp_get_state(sdp_handle h, double* x, double* y, double* blk_a, double* blk_b, double* blk_c);

/* Set the iterates (same layout as sdp_get_state; NULL leaves a part unchanged). Used for warm
 * starts and to resume from a checkpoint. Synchronous. */
int sdp_set_state(sdp_handle h, const double* x, const double* y, const double* blk_a,
                  const double* blk_b, const double* blk_c);

/* Diagnostic: the Jacobi sweeps each clique's eigensolver took in the handle's last iteration
 * (host array [p], in clique order; 0 for a clique the iteration skipped). Synchronous. */
int sdp_proj_sweeps(sdp_handle h, int* sweeps);

/* The index maps built by sdp_setup (host outputs, any may be NULL): the lower pattern E_L as
 * (pat_row, pat_col) [nE_lower], the packed block offsets blk_off [p+1], and gather_idx [S_L]:
 * for every packed block position, the E_L index it reads (H_k as an index map). */
int sdp_get_maps(sdp_handle h, int* pat_row, int* pat_col, long long* blk_off, int* gather_idx);

/* H_k x for every clique k (Section III.A): blocks_out[device, S_L] = gather of x[device, nE_lower].
 * Exact copies. */
int sdp_gather(sdp_handle h, const double* x, double* blocks_out, void* cuda_stream);

/* sum_k H_k^T v_k (Section III.B.1): out[device, nE_lower] from blocks[device, S_L]. Each entry
 * adds its clique contributions in ascending k starting from the first; no atomics, so the result
 * is deterministic. */
int sdp_scatter(sdp_handle h, const double* blocks, double* out, void* cuda_stream);

/* Batched projection onto the PSD cone, P(W) = V max(Lambda, 0) V^T (Eqs. XkUpdate / zkUpdate):
 * in and out are DEVICE pointers to packed lower blocks (FP64); sizes[count] and offsets[count]
 * are HOST arrays giving each block's order (1 <= s <= SDP_MAX_CLIQUE) and its element offset in
 * in/out. prec selects FP64 or FP32 eigensolves (results are FP64 either way). Blocks run in one
 * launch, largest first. The call allocates a small stream-ordered device schedule, copied from a
 * host buffer of the call, so it cannot be captured in a CUDA graph: on a capturing stream it
 * returns SDP_ERR_UNSUPPORTED. in == out is allowed; blocks must not overlap otherwise. */
int project_psd_batched(const double* in, double* out, const int* sizes, const long long* offsets,
                        int count, int prec, void* cuda_stream);

/* ---- new data for an existing handle ---------------------------------------------------------
 * Replace the cost (c_lower: device array of nE_lower values, C on E_L in the handle's order, as
 * sdp_get_maps lists it) or the right-hand side (b: device array of m values). The KKT factor does
 * not depend on either, so nothing is refactored; iterates are kept. Stream-ordered. */
int sdp_set_cost(sdp_handle h, const double* c_lower, void* cuda_stream);
int sdp_set_rhs(sdp_handle h, const double* b, void* cuda_stream);

/* ---- differentiation of unrolled iterations (not in the paper) ----------------------------------
 * sdp_unrolled_forward resets the handle and runs exactly T iterations of Algorithm 1 (form must
 * be SDP_PRIMAL and prec SDP_PROJ_FP64; cliques of order <= 32), keeping the iterates
 * (x_k, lambda_k) every ckpt_every iterations in device memory owned by the handle. X_T is the
 * affine iterate x of iteration T; it is copied to x_out (device, nE_lower values; may be NULL)
 * and left in the handle (sdp_get_state).
 *
 * sdp_unrolled_backward is reverse mode through those iterations. xbar (device, nE_lower) is
 * dL/dtheta for the lower-triangle values theta of X_T (an off-diagonal theta moves X_ij and X_ji
 * together). It writes cbar (device, nE_lower): dL/dtheta_C through the iterations, where theta_C
 * are the lower-triangle values of C (a loss that uses C directly adds that term itself), and
 * bbar (device, m): dL/db. Each segment of ckpt_every iterations is recomputed from its checkpoint
 * to recover the eigenvectors of every projection; the derivative of the projection is the
 * Daleckii-Krein formula (f'(0) = 0, f' of the mean for eigenvalues closer than 1e-12 max|lambda|),
 * the KKT step is self-adjoint. Stream-ordered, returns after the stream finished. It fails with
 * SDP_ERR_ARG if the data or options changed after the forward call; it leaves the handle's
 * iterates at some recomputed step (call admm_reset before solving again). */
int sdp_unrolled_forward(sdp_handle h, int T, int ckpt_every, double* x_out, void* cuda_stream);
int sdp_unrolled_backward(sdp_handle h, const double* xbar, double* cbar, double* bbar, void* cuda_stream);

/* ---- kernel variants of the batched projection (no counterpart in the paper: implementation
 * choices, exposed so that they can be tuned). Variant v in 0 .. project_variant_count()-1 is one
 * eigensolver kernel shape (one-sided Jacobi with a warp segment or a CTA per block, two-sided
 * Jacobi with a CTA per block) with a largest padded order (s rounded up to even) and a
 * precision it accepts; project_variant_name(v) names it ("ow16": one-sided, a 16-lane warp
 * segment per block, FP32, order <= 16). project_variant_fits(v, s, prec) says whether it takes
 * blocks of order s in precision prec (1) or not (0). */
int project_variant_count(void);
const char* project_variant_name(int v);
int project_variant_fits(int v, int s, int prec);

/* project_psd_batched with every block on one given variant (device pointers as there).
 * SDP_ERR_UNSUPPORTED when the variant does not fit some block or the precision. */
int project_psd_batched_variant(const double* in, double* out, const int* sizes,
                                const long long* offsets, int count, int prec, int variant,
                                void* cuda_stream);

/* Per handle: which variant projects the cliques of padded order N in precision prec.
 * table[N] for N = 0 .. len-1 (host array; -1 or a variant that does not fit = the default for
 * that order); len <= SDP_MAX_CLIQUE + 1. NULL restores the defaults. The iteration graphs are
 * rebuilt at the next admm_iterate; iterates are unchanged. */
int sdp_set_proj_table(sdp_handle h, int prec, const int* table, int len);

/* Profiling: run one untimed iteration and then `reps` timed iterations kernel by kernel (no
 * graph) on cuda_stream, with CUDA events between the phases, all queued before the host waits
 * (so an event pair brackets the device's work, not the host's submission), and write the
 * average device milliseconds of each phase of one iteration to ms_out[0 .. count-1] in launch
 * order (count = 5 primal, 6 dual, one more each for cones, for the per-problem stop test of a
 * batch and for the triangular KKT solve, whose two solves are two phases; the projection phase
 * covers all of its launches). Returns count, or < 0 on error; max_out is the capacity of ms_out.
 * The reps + 1 iterations really run and advance the state, with the stop test disabled; the
 * call creates reps x (count + 1) CUDA events, destroyed before it returns (an event that cannot
 * be created gives SDP_ERR_CUDA). sdp_phase_name(h, i) names phase i for the handle's current
 * form (NULL when out of range). */
int sdp_time_phases(sdp_handle h, int reps, void* cuda_stream, double* ms_out, int max_out);
const char* sdp_phase_name(sdp_handle h, int i);

/* Wall-clock time of the stages of the sdp_setup* call that made h, in milliseconds (the
 * set-up that Algorithms 1 and 2 do once before iterating: the clique maps, A on the lower
 * pattern and the cached factor of A D^-1 A^T). Stage i is named by sdp_setup_stage_name(i):
 * "host_build" (index maps, A in CSR and the A^T slice layout, and the KKT factorization when it
 * is built on the host), "plan" (kernel preparation and work schedules), "alloc_upload" (device
 * allocations and host-to-device copies), "device_kkt" (the wait for the A^T slices and the KKT
 * factorization built on the device, which run while the copies after the CSR proceed; 0 when
 * they are built on the host) and "finish" (pinned control block, stream, first reset and the
 * closing device synchronization). Writes min(max_out, count) values and returns count (5), or
 * SDP_ERR_ARG for a NULL handle or a NULL ms_out with max_out > 0. sdp_setup_stage_name returns
 * NULL out of range. */
int sdp_setup_times(sdp_handle h, double* ms_out, int max_out);
const char* sdp_setup_stage_name(int i);

/* Batched PSD projection that allocates nothing (no counterpart in the paper: it exists for
 * callers, not for the method). Same arguments and results (to rounding: every block goes to the
 * kernel variant that fits the largest one) as project_psd_batched, for
 * callers that may not allocate device memory: code embedded in a host framework that owns all
 * device memory through a pool sized up front, and latency-bound loops where a cudaMalloc (which
 * may synchronize the device) is not acceptable. The per-call block schedule goes into a fixed
 * array compiled into the library (SDP_NOALLOC_MAX_BLOCKS blocks, 384 KiB, held by every GPU that
 * loads the library until the process exits) instead of an allocated buffer.
 *   - count > SDP_NOALLOC_MAX_BLOCKS returns SDP_ERR_UNSUPPORTED; other errors as for
 *     project_psd_batched.
 *   - The first call on each device looks up the array's device address and prepares the kernels;
 *     make that first call before any stream capture. After cudaDeviceReset the next call on that
 *     device repeats this set-up (every call checks the address).
 *   - sizes and offsets are host arrays (pageable or pinned), copied before the call returns:
 *     the caller may change or free them as soon as it has returned.
 *   - Every call reuses the same array, which keeps the last call's schedule. Each call
 *     overwrites every entry it reads, so nothing needs clearing, but calls that overlap on the
 *     GPU (e.g. on two streams) race on the array: order them on one stream or synchronize.
 *   - in == out is allowed (each block is read before it is written, by the same CTA).
 *   - Blocks run in the caller's order rather than largest first. */
#define SDP_NOALLOC_MAX_BLOCKS 32768
int project_psd_batched_noalloc(const double* in, double* out, const int* sizes,
                                const long long* offsets, int count, int prec, void* cuda_stream);

void sdp_free(sdp_handle h);
const char* sdp_status_string(int status);
const char* sdp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CHORDAL_ADMM_H */
