// Internal declarations shared by the host setup, the kernels and the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "../../include/chordal_admm.h"

namespace cadmm {

// Device control block: one per handle, read by every kernel of an iteration.
struct Ctrl {
    int iter;        // iterations completed since reset
    int iter_limit;  // the call stops when iter reaches this
    int done;        // nonzero: remaining kernels return immediately
    int status;      // SDP_OK / SDP_MAX_ITER / SDP_ERR_NAN once done
    unsigned int ticket;  // CTAs of the iteration's last kernel that have finished (last one finalizes)
    int active;      // batches: problems still iterating after the last iteration
    double tol;
    double eps_p, eps_d, obj_p, obj_d;
};

// Host-side result of setup: everything the device needs, in upload order.
// A vector whose resize leaves new elements uninitialized, for large arrays that are filled in
// parallel right after (the first write, not a serial zero fill, then touches each page).
template <class T>
struct DefaultInitAlloc : std::allocator<T> {
    template <class U>
    struct rebind {
        using other = DefaultInitAlloc<U>;
    };
    DefaultInitAlloc() = default;
    template <class U>
    DefaultInitAlloc(const DefaultInitAlloc<U>&) {}
    template <class U, class... Args>
    void construct(U* p, Args&&... args) {
        if constexpr (sizeof...(Args) == 0) ::new ((void*)p) U;
        else ::new ((void*)p) U(std::forward<Args>(args)...);
    }
};
template <class T>
using uvector = std::vector<T, DefaultInitAlloc<T>>;

struct HostProblem {
    int n = 0, m = 0, p = 0, smax = 0;
    int nEL = 0;        // |E_L|
    int SL = 0;         // packed block length
    long long nnz = 0;  // nonzeros of A on E_L
    std::vector<int> pat_row, pat_col;          // E_L, column-major
    std::vector<int> blk_off;                   // [p+1]
    std::vector<int> blk_size;                  // [p]
    std::vector<int> order;                     // [p] cliques by descending size
    std::vector<long long> voff;                // [p+1] eigenvector block offsets (N_k^2 each)
    std::vector<int> gather_idx;                // [SL]
    std::vector<unsigned char> pos_w;           // [SL] 1 on block diagonals, 2 elsewhere
    std::vector<int> sc_ptr;                    // [nEL+1]
    std::vector<int> sc_pos;                    // [SL]
    std::vector<int> heavy;                     // E_L entries covered by more than kHeavyCount cliques
    std::vector<double> D, dinv, wdinv, c, b;   // D, 1/D, w/D, c on E_L; b
    std::vector<unsigned char> ew;              // [nEL] weight 1 (diagonal) or 2
    std::vector<int> a_rowptr;                  // CSR of A (rows = constraints)
    uvector<int> a_col;
    uvector<double> a_val;
    std::vector<int> c_colptr;                  // CSC of A (columns = E_L entries); host only
    std::vector<unsigned short> c_row;
    std::vector<double> c_val;
    // A^T in sliced ELL form for the device: slot t of slice s holds column sell_col[32 s + t]
    // (-1: empty; a slice never spans two problems), padded to the slice's longest column;
    // element k of that column sits at sell_off[s] + 32 k + t (padding: value 0, row 0). Rows
    // are numbered within the problem.
    std::vector<int> sell_col, sell_len;        // [32 nslices], [nslices]
    std::vector<long long> sell_off;            // [nslices+1]
    std::vector<unsigned short> sell_row;
    std::vector<double> sell_val;
    std::vector<double> Minv;                   // (A D^-1 A^T)^-1: per instance an m_q x m_q row-major block
    // L^-1 (lower, row-major, per instance at the same offsets as M^-1), kept for the affine
    // step of ill-conditioned problems; LinvT = (L^-1)^T row-major, filled when kkt_tri is set.
    std::vector<double> Linv, LinvT;
    double kkt_cond = 1.0;                      // kappa_1(A D^-1 A^T) (largest over a batch)
    bool kkt_tri = false;                       // affine step by the two triangular factors
    // The factorization is left to the device (M, L, L^-1, M^-1 and kappa then come from
    // device_kkt_launch), and so is the fill of the A^T slices: sell_row and sell_val stay empty
    // here, slot_len[32 s + t] is the length of the column in slot t of slice s and col_slot[e]
    // the slot (32 s + t) of column e.
    bool kkt_on_device = false;
    std::vector<int> slot_len, col_slot;
    // Batches: instances are concatenated (block-diagonal problem); ranges are [q] .. [q+1].
    int ninst = 1;
    std::vector<int> inst_vtx, inst_cl, inst_e, inst_pos, inst_row, inst_sl;   // vertices, cliques,
                                                                      // E_L entries, positions, rows, slices
    std::vector<long long> mblk_off;                        // offsets of the M^-1 blocks
    // Non-PSD cones: n_cone variables after the E_L entries (and after the clique blocks in the
    // packed vector), projected in segments [cone_lo, cone_hi) of kind kCone*.
    int n_cone = 0;
    std::vector<int> cone_lo, cone_hi, cone_kind;
    std::vector<int> soc_pos, soc_q;            // small second-order cones: first position, dimension
};

// Kinds of cone segments, and the longest free / nonnegative segment (their projections are
// elementwise, so long runs are cut; a second-order cone is always one segment).
// kConeSocSmall segments hold up to kSmallSocPerCta second-order cones of dimension <= kSmallSoc
// (one thread each; the segment's range indexes soc_pos / soc_q), the other kinds a position range.
constexpr int kConeFree = 0, kConeNonneg = 1, kConeSoc = 2, kConeSocSmall = 3;
constexpr int kConeChunk = 4096;
constexpr int kSmallSoc = 32;
constexpr int kSmallSocPerCta = 256;

// Chordal extension of the symmetric pattern given by nnz (row, col) coordinates and the maximal
// cliques of the extension (chordal.cpp). fill = lower pairs added.
int chordal_cliques(int n, long long nnz, const int* row, const int* col, std::vector<int>& clique_ptr,
                    std::vector<int>& clique_vtx, long long& fill, std::string& err);

// Builds one HostProblem for a batch of independent problems (a block-diagonal problem). On
// failure fills err (prefixed with the failing instance) and returns the SDP_* status.
int build_host_problem_batch(int count, const sdp_problem* in, HostProblem& hp, std::string& err);

// Builds HostProblem from the ABI inputs. Returns an SDP_* status and fills err on failure.
// kkt_device: the KKT factorization may be left to device_kkt (if the problem fits its limits).
int build_host_problem(int n, int m, const long long* A_ptr, const int* A_row, const int* A_col,
                       const double* A_val, const double* b, long long C_nnz, const int* C_row,
                       const int* C_col, const double* C_val, long long pat_nnz,
                       const int* pat_row, const int* pat_col, int p, const int* clique_ptr,
                       const int* clique_vtx, const sdp_cones* cones, HostProblem& hp, std::string& err,
                       bool kkt_device = false);

// ---------------------------------------------------------------- KKT factorization on the device
// (kkt.cu) for single problems with kKktDeviceMinM <= m <= kKktDeviceMaxM: the A^T slices from
// the CSR of A, M = A D^-1 A^T from them, L, L^-1, M^-1 and kappa_1(M).
constexpr int kKktDeviceMinM = 64;
constexpr int kKktDeviceMaxM = 4096;
bool device_kkt_fits(int m, int max_col_len);
struct KktInputs {
    int m = 0, nslices = 0;
    const int* sell_col = nullptr;
    const int* sell_len = nullptr;
    const long long* sell_off = nullptr;
    const unsigned short* sell_row = nullptr;
    const double* sell_val = nullptr;
    const double* wdinv = nullptr;
    std::vector<int> slot_len_h;
    // When ell_row is set, the slices are first filled here from the CSR of A (rows ascending
    // within every column, padding 0) into ell_row / ell_val, which sell_row / sell_val name.
    const int* a_rowptr = nullptr;
    const int* a_col = nullptr;
    const double* a_val = nullptr;
    long long nnz = 0;
    int nEL = 0;
    const int* col_slot = nullptr;    // [nEL] slot 32 s + t of column e
    unsigned short* ell_row = nullptr;
    double* ell_val = nullptr;
    long long ell_size = 0;           // sell_off[nslices]
};
struct KktOutputs {
    double* L = nullptr;       // m x m: M, then its Cholesky factor in the lower triangle
    double* Linv = nullptr;    // m x m row-major, lower
    double* LinvT = nullptr;   // m x m row-major, (L^-1)^T
    double* Minv = nullptr;    // m x m row-major, symmetric
    double kappa1 = 0.0;
};
// The factorization runs on a stream of its own, so that the caller can go on uploading while it
// runs: device_kkt_launch enqueues it (SDP_OK or SDP_ERR_CUDA), device_kkt_wait waits for it and
// fills kappa1 (SDP_OK, SDP_ERR_NOT_PD when A is numerically rank-deficient, or SDP_ERR_CUDA).
// The outputs must outlive the run; KktRun's destructor waits for the stream before it frees the
// scratch, so a caller that gives up between the two calls leaves no work in flight.
struct KktRun {
    cudaStream_t st = nullptr;
    int m = 0;
    double* d_rows = nullptr;   // largest absolute row sums of M and M^-1
    int* d_notpd = nullptr;     // set by a pivot at or below 1e-12 of its diagonal entry
    std::vector<void*> bufs;
    void release();
    ~KktRun() { release(); }
};
int device_kkt_launch(const KktInputs& in, const KktOutputs& out, KktRun& run, std::string& err);
int device_kkt_wait(KktRun& run, KktOutputs& out, std::string& err);

// ---------------------------------------------------------------- kernel launch parameters

enum ProjMode { PROJ_PLAIN = 0, PROJ_PRIMAL = 1, PROJ_DUAL = 2 };

struct ProjArgs {
    const int* order;       // [count] block to process per CTA (NULL: blocks first, first + 1, ...)
    int first;
    const int* size;        // [*] block order s_k
    const long long* off;   // [*] packed element offset (64-bit for the standalone entry)
    int count;
    double rho;
    // PLAIN: in -> out.  PRIMAL: W = x[gather] - lam/rho; writes xk_new, lam, partials.
    // DUAL: W = v - lam/rho; writes z (out).
    const double* in;
    double* out;
    const double* x;
    const int* gather_idx;
    double* lam;
    const double* v;
    double* xk[2];          // primal ping-pong buffers, chosen by ctrl->iter parity
    double* part;           // [count * 4] per-clique residual partials and Jacobi sweep counts
    void* vstore;           // per-clique eigenvectors kept for warm starts (NULL: always cold)
    const long long* voff;  // [*] element offset of each clique's N x N block in vstore
    const Ctrl* ctrl;       // NULL for the standalone entry
    // Batches: a clique whose problem has stopped (inst_conv >= 0) is skipped. In the primal form
    // its current blocks are first copied to the other ping-pong buffer, once, so that both hold
    // them whatever the parity of later iterations. NULL for a single problem.
    const int* blk_inst;
    const int* inst_conv;
    int pdl;                // programmatic dependent launch inside an iteration (0 standalone)
};

// Entries covered by more cliques than this are scattered by a whole warp (in ascending clique
// order, so the sum is the same as the sequential one).
constexpr int kHeavyCount = 16;

// One CTA's share of a launch: problem q of the batch, element range [lo, hi). aux is the
// constraint (row) of a CSR chunk and unused elsewhere. No CTA spans two problems, so every
// partial sum belongs to one problem.
struct Sched {
    int q, lo, hi, aux;
};

// Projection launches: the cliques in processing order (largest first) split into runs that use
// the same kernel variant. A run [start, start + count) of `order` goes to one launch.
enum ProjVariant { PV_OS1 = 0, PV_OS2, PV_TS16, PV_TS32, PV_TS64, PV_TS96, PV_OW8, PV_OW16, PV_OW32, PV_OW64,
                   PV_WS32, PV_WS64, PV_COUNT };
constexpr int kMaxProjRuns = 64;
struct ProjPlan {
    int runs;
    int start[kMaxProjRuns], count[kMaxProjRuns], variant[kMaxProjRuns], smax[kMaxProjRuns];
    // 1: the run's stretch of `order` is start, start + 1, ... (its launch then reads no order
    // entry, one dependent load fewer before a CTA can fetch its block)
    unsigned char identity[kMaxProjRuns];
};

struct IterPtrs {
    // problem (a batch is the block-diagonal union of its problems)
    int n, m, p, nEL, SL, smax;
    int pdl;                        // launch the iteration's kernels with programmatic dependent launch
    int ninst;                      // problems in the batch (1 after sdp_setup)
    int mmax;                       // largest number of constraints of one problem
    const int* inst_cl;             // [ninst+1] first clique of each problem
    const int* inst_row;            // [ninst+1] first constraint of each problem
    const long long* mblk_off;      // [ninst+1] offset of each problem's block of M^-1
    const int* blk_inst;            // [p] problem of each clique
    // Work schedules. The two passes over A are split into warp-sized chunks (8 per CTA); the
    // other kernels give one Sched per CTA.
    const Sched* row_sched; int row_chunks; const int* row_chunk;  // CSR chunks; row_chunk[m+1]
    const Sched* tri_sched; int tri_ctas;                          // <= 8 rows of M^-1 per CTA (y solve)
    const Sched* col_sched; int col_chunks;                        // slice ranges of A^T
    int col_split;                                                 // 1: one slice per CTA, warps split it
    const Sched* pos_sched; int pos_ctas;                          // packed positions
    const Sched* ent_sched; int ent_ctas;                          // light entries, one per thread
    const Sched* heavy_sched; int heavy_ctas;                      // heavy-list ranges, one per warp
    // per problem: its first entry in each schedule that produces residual partials ([ninst+1])
    const int* inst_col_chunk; const int* inst_pos_cta; const int* inst_ent_cta; const int* inst_heavy_cta;
    double* inst_res;     // [ninst * 4]: eps_p, eps_d, obj_p, obj_d of its last iteration
    int* inst_conv;       // [ninst]: iteration at which it stopped (converged or NaN), or -1
    int* inst_stat;       // [ninst]: SDP_OK, SDP_MAX_ITER or SDP_ERR_NAN
    const int* blk_off; const long long* blk_off64; const int* blk_size; const int* order;
    const int* gather_idx; const unsigned char* pos_w;
    const int* sc_ptr; const int* sc_pos;
    const int* heavy; int n_heavy;                 // warp-per-entry scatter of heavily shared entries
    const double* D; const double* dinv; const double* wdinv; const double* c; const double* b;
    const unsigned char* ew;
    const int* a_rowptr; const int* a_col; const double* a_val;
    const int* sell_col; const int* sell_len; const long long* sell_off;    // A^T, sliced ELL
    const unsigned short* sell_row; const double* sell_val;                  // rows within the problem
    const double* Minv;                            // (A D^-1 A^T)^-1 blocks at mblk_off
    // kkt_tri: y = L^-T (L^-1 (t - rhs2)) by two triangular products with the cached factor's
    // inverse (blocks at mblk_off), z1 the intermediate; otherwise y = M^-1 (t - rhs2).
    int kkt_tri;
    const double* Linv; const double* LinvT; double* z1;
    // state
    double* x; double* y; double* r; double* rsw;
    double* xk[2]; double* lam; double* vk;
    void* vstore;         // eigenvector blocks for warm starts (projection precision)
    const long long* voff;
    double* tpart;        // [row_chunks]
    double* part_blk;     // [(p + ncs) * 4]: cliques, then cone segments
    // non-PSD cone segments (single problems only): positions [cone_lo, cone_hi), kind kCone*
    int ncs; const int* cone_lo; const int* cone_hi; const int* cone_kind;
    const int* soc_pos; const int* soc_q;         // small second-order cones (kConeSocSmall segments)
    double* part_ent;     // [max(ent_ctas + heavy_ctas, pos_ctas) * 8]
    double* part_obj;     // [col_chunks]
    Ctrl* ctrl;
};

// Launch with programmatic dependent launch when pdl is set (the kernel is scheduled while its
// predecessor finishes and waits for it in pdl_wait()); without it pdl_wait()/pdl_trigger() in
// the kernel are no-ops and it starts once its predecessor has completed.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

#ifdef __CUDACC__
// First statement of every kernel of an iteration: wait until the previous kernel in the stream
// has completed and its writes are visible.
__device__ __forceinline__ void pdl_wait() { cudaGridDependencySynchronize(); }
// Called once a CTA's main work is done: the next kernel may start launching (its CTAs then wait
// in pdl_wait). Triggering late keeps waiting CTAs off the SMs while this kernel still computes.
__device__ __forceinline__ void pdl_trigger() { cudaTriggerProgrammaticLaunchCompletion(); }
#endif

// Kernel launchers (kernels.cu / project.cu). All return cudaError_t of the launch.
cudaError_t launch_project(const ProjArgs& a, int mode, int prec, int smax, cudaStream_t st);
// One launch of a given variant over a.count blocks (a.order may point into a longer order array).
cudaError_t launch_project_variant(const ProjArgs& a, int mode, int prec, int variant, int smax, cudaStream_t st);
int project_default_variant(int s, int prec);   // the variant launch_project picks for max size s
bool project_variant_valid(int variant, int s, int prec);
// Runs of `order` (sizes non-increasing) that share a variant; table[N] (N = 1..SDP_MAX_CLIQUE+1,
// padded even order) overrides the default choice when non-NULL and valid.
ProjPlan make_proj_plan(const std::vector<int>& order, const std::vector<int>& size, int prec,
                        const int* table, int ow_min_blocks);
int proj_ow_min_blocks(int num_sms);   // blocks of order <= 32 below which a CTA per block is used
cudaError_t project_prepare();   // raises the dynamic shared-memory limit of every variant
size_t project_smem_bytes(int smax, int prec, int mode);
int project_threads(int smax);
size_t project_vstore_elems(int s);   // N*N with N = s rounded up to even
cudaError_t launch_vstore_identity(const IterPtrs& P, int prec, cudaStream_t st);

cudaError_t launch_iteration(const IterPtrs& P, const ProjPlan& plan, int form, int prec, double rho,
                             cudaStream_t st, cudaEvent_t* ev = nullptr);
int phase_count(const IterPtrs& P, int form);
const char* phase_name(int form, bool batch, bool cones, bool tri, int i);
// Condition number (1-norm) of A D^-1 A^T above which the affine step applies the Cholesky
// factor as two triangular products instead of the explicit inverse.
constexpr double kKktTriCond = 1.0e5;
cudaError_t launch_primal_rebuild_r(const IterPtrs& P, double rho, cudaStream_t st);
cudaError_t launch_gather(const IterPtrs& P, const double* x, double* blocks, cudaStream_t st);
cudaError_t launch_scatter(const IterPtrs& P, const double* blocks, double* out, cudaStream_t st);
cudaError_t launch_ctrl_arm(Ctrl* ctrl, int n_iters, double tol, cudaStream_t st);
cudaError_t launch_ctrl_reset(Ctrl* ctrl, cudaStream_t st);
cudaError_t launch_ctrl_clear(Ctrl* ctrl, cudaStream_t st);
int iteration_kernel_count(const IterPtrs& P, const ProjPlan& plan, int form);
cudaError_t launch_inst_reset(const IterPtrs& P, cudaStream_t st);   // every problem active again
// The block-elimination solve alone with right-hand side [r; 0] (r in P.r, r w/D in P.rsw):
// y = (A D^-1 A^T)^-1 A D^-1 r into P.y and x = D^-1 (r - A^T y) into P.x (form kKktZeroRhs).
constexpr int kKktZeroRhs = 2;
cudaError_t launch_kkt_adjoint(const IterPtrs& P, cudaStream_t st);
cudaError_t launch_ctrl_set_iter(Ctrl* ctrl, int it, cudaStream_t st);
// CTAs of one SM that can be resident at once for kernel 0 (spmv_rows), 1 (spmv_cols) or 2
// (update_dual) with `smem` bytes of dynamic shared memory; sizes the grids to whole waves.
int resident_ctas(int kernel, size_t smem);

// Reverse mode of unrolled primal iterations (adjoint.cu).
cudaError_t adjoint_prepare();
cudaError_t launch_form_w(const IterPtrs& P, const double* lam_prev, double rinv, double* W, cudaStream_t st);
cudaError_t launch_dk_vjp(const IterPtrs& P, int n_large, const double* W, const double* V, double* Xb,
                          double* Lb, double* ub, double rho, cudaStream_t st);
cudaError_t launch_adj_scatter(const IterPtrs& P, const double* ub, const double* xbar_T, double* xbar,
                               double* rsw, cudaStream_t st);
cudaError_t launch_adj_accum(const IterPtrs& P, const double* rbar, const double* ybar, double* cbar,
                             double* bbar, double* Xb, double* Lb, double rinv, cudaStream_t st);
cudaError_t launch_adj_finish(const IterPtrs& P, const double* cbar, const double* bbar, double* cout,
                              double* bout, cudaStream_t st);
cudaError_t launch_copy(const double* src, double* dst, long long n, cudaStream_t st);
int record_error(int code, const std::string& msg);   // sets the message sdp_last_error() returns
cudaError_t iteration_prepare();  // raises the dynamic shared-memory limit of the m-sized kernels

}  // namespace cadmm
