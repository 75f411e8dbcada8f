// Internal declarations shared by the host setup, the kernels and the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
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
    double tol;
    double eps_p, eps_d, obj_p, obj_d;
};

// Host-side result of setup: everything the device needs, in upload order.
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
    std::vector<int> a_rowptr, a_col;           // CSR of A (rows = constraints)
    std::vector<double> a_val;
    std::vector<int> c_colptr;                  // CSC of A (columns = E_L entries)
    std::vector<unsigned short> c_row;
    std::vector<double> c_val;
    std::vector<double> Linv, LinvT;            // m x m row-major
};

// Builds HostProblem from the ABI inputs. Returns an SDP_* status and fills err on failure.
int build_host_problem(int n, int m, const long long* A_ptr, const int* A_row, const int* A_col,
                       const double* A_val, const double* b, long long C_nnz, const int* C_row,
                       const int* C_col, const double* C_val, long long pat_nnz,
                       const int* pat_row, const int* pat_col, int p, const int* clique_ptr,
                       const int* clique_vtx, HostProblem& hp, std::string& err);

// ---------------------------------------------------------------- kernel launch parameters

enum ProjMode { PROJ_PLAIN = 0, PROJ_PRIMAL = 1, PROJ_DUAL = 2 };

struct ProjArgs {
    const int* order;       // [count] block to process per CTA (NULL = identity)
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
};

// Entries covered by more cliques than this are scattered by a whole warp (in ascending clique
// order, so the sum is the same as the sequential one).
constexpr int kHeavyCount = 16;

struct IterPtrs {
    // problem
    int n, m, p, nEL, SL, smax, R;      // R = CTAs per CSR row
    const int* blk_off; const long long* blk_off64; const int* blk_size; const int* order;
    const int* gather_idx; const unsigned char* pos_w;
    const int* sc_ptr; const int* sc_pos;
    const int* heavy; int n_heavy, heavy_ctas;     // warp-per-entry scatter of heavily shared entries
    const double* D; const double* dinv; const double* wdinv; const double* c; const double* b;
    const unsigned char* ew;
    const int* a_rowptr; const int* a_col; const double* a_val;
    const int* c_colptr; const unsigned short* c_row; const double* c_val;
    const double* Linv; const double* LinvT;
    // state
    double* x; double* y; double* r; double* rsw; double* z1;
    double* xk[2]; double* lam; double* vk;
    void* vstore;         // eigenvector blocks for warm starts (projection precision)
    const long long* voff;
    double* tpart;        // [m * R]
    double* part_blk;     // [p * 4]
    double* part_ent;     // [(max(ent_ctas + heavy_ctas, pos_ctas)) * 8]
    double* part_obj;     // [col_ctas]
    int ent_ctas, col_ctas, pos_ctas;
    Ctrl* ctrl;
};

// Programmatic dependent launch (a kernel scheduled while its predecessor finishes, waiting for it
// in pdl_wait()) is wired through every iteration kernel but switched off: on GB300 it made the
// captured iteration slower (FP32 projection 9.8k -> 9.0k iter/s, FP64 1.8k -> 0.9k iter/s on the
// n = 1020 block-arrow workload). With the attribute off, pdl_wait()/pdl_trigger() are no-ops.
constexpr bool kUsePDL = false;

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = kUsePDL ? 1 : 0;
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
cudaError_t project_prepare();   // raises the dynamic shared-memory limit of every variant
size_t project_smem_bytes(int smax, int prec, int mode);
int project_threads(int smax);
size_t project_vstore_elems(int s);   // N*N with N = s rounded up to even
cudaError_t launch_vstore_identity(const IterPtrs& P, int prec, cudaStream_t st);

cudaError_t launch_iteration(const IterPtrs& P, int form, int prec, double rho, cudaStream_t st,
                             cudaEvent_t* ev = nullptr);
const char* phase_name(int form, int i);
cudaError_t launch_primal_rebuild_r(const IterPtrs& P, double rho, cudaStream_t st);
cudaError_t launch_gather(const IterPtrs& P, const double* x, double* blocks, cudaStream_t st);
cudaError_t launch_scatter(const IterPtrs& P, const double* blocks, double* out, cudaStream_t st);
cudaError_t launch_ctrl_arm(Ctrl* ctrl, int n_iters, double tol, cudaStream_t st);
cudaError_t launch_ctrl_reset(Ctrl* ctrl, cudaStream_t st);
cudaError_t launch_ctrl_clear(Ctrl* ctrl, cudaStream_t st);
int iteration_kernel_count(int form);
int record_error(int code, const std::string& msg);   // sets the message sdp_last_error() returns
cudaError_t iteration_prepare();  // raises the dynamic shared-memory limit of the m-sized kernels

}  // namespace cadmm
