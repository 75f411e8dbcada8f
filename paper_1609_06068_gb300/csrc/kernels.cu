// Per-iteration kernels of the decomposed ADMM other than the PSD projection:
//   scatter      r = sum_k H_k^T(.) and the KKT right-hand side (Eqs. OptCondMinYPrimal/Dual)
//   spmv_rows    t = A (w r / D)           (block elimination, first pass over A; CSR)
//   tri_lower    z = L^-1 (t - rhs2)       (cached factor of A D^-1 A^T, Section III.B.1)
//   tri_upper    y = L^-T z
//   spmv_cols    x = (r - A^T y) / D       (second pass over A; CSC)
//   update_dual  v_k = z_k + rho^-1 lambda_k + H_k x, lambda_k = -rho H_k x (Eqs. vkEqn,
//                DualMultUpdate with the sign Eq. MultUpdateDualSDP implies)
//   finalize     residuals, objectives, stop test (one CTA, fixed-order reductions)
// Every kernel starts by reading the device control block and returns at once when the solve is
// done, so a captured graph holding several iterations can run past convergence at no cost.
// All reductions use a fixed tree, so results are bitwise reproducible run to run.
#include "sdp_internal.h"

namespace cadmm {

namespace {

constexpr int kEntThreads = 256;  // entry-wise kernels
constexpr int kRowThreads = 256;  // CSR row chunks
constexpr int kTriThreads = 256;  // triangular products (8 warps, one row per warp)
constexpr int kColThreads = 256;  // CSC columns
constexpr int kColGroup = 8;      // lanes per CSC column

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) red[warp * K + k] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double t = lane < nw ? red[lane * K + k] : 0.0;
            t = warp_sum(t);
            if (lane == 0) red[32 * K + k] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = red[32 * K + k];
}

// ---------------------------------------------------------------- scatter (primal form)
// r = sum_k H_k^T(x_k + rho^-1 lambda_k) - rho^-1 c, summed in ascending k from the first term;
// also the dual-residual pieces ||sum_k H_k^T(x_k+ - x_k)||^2 and ||sum_k H_k^T lambda_k||^2.
// use_current = 1 rebuilds r from the current blocks (after a reset or a state upload).
__global__ void __launch_bounds__(kEntThreads) k_scatter_primal(IterPtrs P, double rinv, int use_current) {
    __shared__ double red[33 * 2];
    if (P.ctrl->done) return;
    const bool odd = (P.ctrl->iter & 1) != 0;
    const double* cur = odd ? P.xk[1] : P.xk[0];
    const double* nxt = odd ? P.xk[0] : P.xk[1];
    const double* xn_buf = use_current ? cur : nxt;
    const double* xo_buf = cur;
    double v[2] = {0.0, 0.0};
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < P.nEL) {
        const int j0 = P.sc_ptr[e], j1 = P.sc_ptr[e + 1];
        double acc = 0.0, dsum = 0.0, lsum = 0.0;
        for (int j = j0; j < j1; ++j) {
            const int pos = P.sc_pos[j];
            const double xn = xn_buf[pos], xo = xo_buf[pos], l = P.lam[pos];
            const double term = __dadd_rn(xn, __dmul_rn(rinv, l));
            const double dd = xn - xo;
            if (j == j0) { acc = term; dsum = dd; lsum = l; }
            else { acc = __dadd_rn(acc, term); dsum += dd; lsum += l; }
        }
        const double re = __dsub_rn(acc, __dmul_rn(rinv, P.c[e]));
        P.r[e] = re;
        P.rsw[e] = re * P.wdinv[e];
        const double w = (double)P.ew[e];
        v[0] = w * dsum * dsum;
        v[1] = w * lsum * lsum;
    }
    if (use_current) return;
    block_sum<2>(v, red);
    if (threadIdx.x == 0) {
        P.part_ent[blockIdx.x * 8 + 0] = v[0];
        P.part_ent[blockIdx.x * 8 + 1] = v[1];
    }
}

// ---------------------------------------------------------------- scatter (dual form)
// r = c - sum_k H_k^T(z_k + rho^-1 lambda_k), ascending k from the first term.
__global__ void __launch_bounds__(kEntThreads) k_scatter_dual(IterPtrs P, double rinv) {
    if (P.ctrl->done) return;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P.nEL) return;
    const double* z = P.xk[0];
    const int j0 = P.sc_ptr[e], j1 = P.sc_ptr[e + 1];
    double acc = 0.0;
    for (int j = j0; j < j1; ++j) {
        const int pos = P.sc_pos[j];
        const double term = __dadd_rn(z[pos], __dmul_rn(rinv, P.lam[pos]));
        acc = (j == j0) ? term : __dadd_rn(acc, term);
    }
    const double re = __dsub_rn(P.c[e], acc);
    P.r[e] = re;
    P.rsw[e] = re * P.wdinv[e];
}

// ---------------------------------------------------------------- t = A (w r / D), CSR chunks
__global__ void __launch_bounds__(kRowThreads) k_spmv_rows(IterPtrs P) {
    __shared__ double red[33];
    if (P.ctrl->done) return;
    const int i = blockIdx.x / P.R, ch = blockIdx.x - (blockIdx.x / P.R) * P.R;
    const int lo0 = P.a_rowptr[i], hi0 = P.a_rowptr[i + 1];
    const long long len = hi0 - lo0;
    const int lo = lo0 + (int)(len * ch / P.R), hi = lo0 + (int)(len * (ch + 1) / P.R);
    double acc = 0.0;
#pragma unroll 4
    for (int j = lo + threadIdx.x; j < hi; j += blockDim.x) acc = fma(P.a_val[j], P.rsw[P.a_col[j]], acc);
    double v[1] = {acc};
    block_sum<1>(v, red);
    if (threadIdx.x == 0) P.tpart[blockIdx.x] = v[0];
}

// ---------------------------------------------------------------- z = L^-1 (t - rhs2)
// rhs2 = b (primal) or -rho^-1 b (dual). One warp per row of L^-1.
__global__ void __launch_bounds__(kTriThreads) k_tri_lower(IterPtrs P, double rinv, int form) {
    extern __shared__ double u[];
    if (P.ctrl->done) return;
    const int m = P.m, R = P.R;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double t = 0.0;
        for (int c = 0; c < R; ++c) t += P.tpart[i * R + c];
        const double rhs2 = form == SDP_PRIMAL ? P.b[i] : -__dmul_rn(rinv, P.b[i]);
        u[i] = t - rhs2;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int row = blockIdx.x * nw + warp; row < m; row += gridDim.x * nw) {
        const double* Lr = P.Linv + (size_t)row * m;
        double acc = 0.0;
        for (int j = lane; j <= row; j += 32) acc = fma(Lr[j], u[j], acc);
        acc = warp_sum(acc);
        if (lane == 0) P.z1[row] = acc;
    }
}

// ---------------------------------------------------------------- y = L^-T z
__global__ void __launch_bounds__(kTriThreads) k_tri_upper(IterPtrs P) {
    extern __shared__ double zs[];
    if (P.ctrl->done) return;
    const int m = P.m;
    for (int i = threadIdx.x; i < m; i += blockDim.x) zs[i] = P.z1[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int row = blockIdx.x * nw + warp; row < m; row += gridDim.x * nw) {
        const double* Lr = P.LinvT + (size_t)row * m;
        double acc = 0.0;
        for (int i = row + lane; i < m; i += 32) acc = fma(Lr[i], zs[i], acc);
        acc = warp_sum(acc);
        if (lane == 0) P.y[row] = acc;
    }
}

// ---------------------------------------------------------------- x = (r - A^T y) / D, CSC
// kColGroup lanes per column; y is staged in shared memory. Also the partial objective sums
// sum_e w_e c_e x_e of this CTA.
__global__ void __launch_bounds__(kColThreads) k_spmv_cols(IterPtrs P) {
    extern __shared__ double ys[];
    __shared__ double red[33];
    if (P.ctrl->done) return;
    for (int i = threadIdx.x; i < P.m; i += blockDim.x) ys[i] = P.y[i];
    __syncthreads();
    const int gid = threadIdx.x / kColGroup, gl = threadIdx.x % kColGroup;
    const int ngroups = blockDim.x / kColGroup;
    double obj = 0.0;
    for (int e0 = blockIdx.x * ngroups; e0 < P.nEL; e0 += gridDim.x * ngroups) {
        const int e = e0 + gid;
        const bool valid = e < P.nEL;
        double s = 0.0;
        if (valid) {
            const int lo = P.c_colptr[e], hi = P.c_colptr[e + 1];
            for (int j = lo + gl; j < hi; j += kColGroup) s = fma(P.c_val[j], ys[P.c_row[j]], s);
        }
#pragma unroll
        for (int o = kColGroup / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (valid && gl == 0) {
            const double xe = (P.r[e] - s) / P.D[e];
            P.x[e] = xe;
            obj = fma((double)P.ew[e] * P.c[e], xe, obj);
        }
    }
    double v[1] = {obj};
    block_sum<1>(v, red);
    if (threadIdx.x == 0) P.part_obj[blockIdx.x] = v[0];
}

// ---------------------------------------------------------------- dual-form multiplier update
__global__ void __launch_bounds__(kEntThreads) k_update_dual(IterPtrs P, double rho, double rinv) {
    __shared__ double red[33 * 5];
    if (P.ctrl->done) return;
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const int pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos < P.SL) {
        const double u = P.x[P.gather_idx[pos]];
        const double z = P.xk[0][pos], l = P.lam[pos], vo = P.vk[pos];
        const double vn = __dadd_rn(__dadd_rn(z, __dmul_rn(rinv, l)), u);   // Eq. vkEqn
        const double ln = __dmul_rn(-rho, u);                                // Eq. DualMultUpdate
        P.vk[pos] = vn;
        P.lam[pos] = ln;
        const double w = (double)P.pos_w[pos];
        const double d1 = z - vn, d2 = vn - vo;
        v[0] = w * d1 * d1;
        v[1] = w * z * z;
        v[2] = w * vn * vn;
        v[3] = w * d2 * d2;
        v[4] = w * ln * ln;
    }
    block_sum<5>(v, red);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 5; ++k) P.part_ent[blockIdx.x * 8 + k] = v[k];
    }
}

// ---------------------------------------------------------------- residuals and stop test
__global__ void __launch_bounds__(256) k_finalize(IterPtrs P, int form, double rho) {
    __shared__ double red[33 * 7];
    Ctrl* C = P.ctrl;
    if (C->done) return;
    double v[7] = {0, 0, 0, 0, 0, 0, 0};
    if (form == SDP_PRIMAL) {
        for (int k = threadIdx.x; k < P.p; k += blockDim.x) {
            v[0] += P.part_blk[k * 4 + 0];
            v[1] += P.part_blk[k * 4 + 1];
            v[2] += P.part_blk[k * 4 + 2];
        }
        for (int q = threadIdx.x; q < P.ent_ctas; q += blockDim.x) {
            v[3] += P.part_ent[q * 8 + 0];
            v[4] += P.part_ent[q * 8 + 1];
        }
    } else {
        for (int q = threadIdx.x; q < P.pos_ctas; q += blockDim.x)
            for (int k = 0; k < 5; ++k) v[k] += P.part_ent[q * 8 + k];
    }
    for (int q = threadIdx.x; q < P.col_ctas; q += blockDim.x) v[5] += P.part_obj[q];
    for (int i = threadIdx.x; i < P.m; i += blockDim.x) v[6] = fma(P.b[i], P.y[i], v[6]);
    block_sum<7>(v, red);
    if (threadIdx.x != 0) return;
    double eps_p, eps_d, obj_p, obj_d;
    if (form == SDP_PRIMAL) {
        eps_p = sqrt(v[0]) / fmax(fmax(sqrt(v[1]), sqrt(v[2])), 1e-12);
        eps_d = rho * sqrt(v[3]) / fmax(sqrt(v[4]), 1e-12);
        obj_p = v[5];
        obj_d = -rho * v[6];
    } else {
        eps_p = sqrt(v[0]) / fmax(fmax(sqrt(v[1]), sqrt(v[2])), 1e-12);
        eps_d = rho * sqrt(v[3]) / fmax(sqrt(v[4]), 1e-12);
        obj_d = v[6];
        obj_p = -rho * v[5];
    }
    const int it = C->iter + 1;
    C->iter = it;
    C->eps_p = eps_p;
    C->eps_d = eps_d;
    C->obj_p = obj_p;
    C->obj_d = obj_d;
    if (!isfinite(eps_p) || !isfinite(eps_d) || !isfinite(obj_p) || !isfinite(obj_d)) {
        C->status = SDP_ERR_NAN;
        C->done = 1;
    } else if (fmax(eps_p, eps_d) < C->tol) {
        C->status = SDP_OK;
        C->done = 1;
    } else if (it >= C->iter_limit) {
        C->status = SDP_MAX_ITER;
        C->done = 1;
    }
}

__global__ void k_ctrl_arm(Ctrl* C, int n_iters, double tol) {
    C->done = n_iters > 0 ? 0 : 1;
    C->status = SDP_MAX_ITER;
    C->iter_limit = C->iter + n_iters;
    C->tol = tol;
}

__global__ void k_ctrl_clear(Ctrl* C) { C->done = 0; }

__global__ void k_ctrl_reset(Ctrl* C) {
    C->iter = 0;
    C->iter_limit = 0;
    C->done = 0;
    C->status = SDP_MAX_ITER;
    C->tol = 0.0;
    C->eps_p = C->eps_d = C->obj_p = C->obj_d = 0.0;
}

__global__ void k_gather(const int* gather_idx, int SL, const double* x, double* out) {
    const int pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos < SL) out[pos] = x[gather_idx[pos]];
}

__global__ void k_scatter_plain(const int* sc_ptr, const int* sc_pos, int nEL, const double* blocks,
                                double* out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nEL) return;
    const int j0 = sc_ptr[e], j1 = sc_ptr[e + 1];
    double acc = 0.0;
    for (int j = j0; j < j1; ++j) acc = (j == j0) ? blocks[sc_pos[j]] : __dadd_rn(acc, blocks[sc_pos[j]]);
    out[e] = acc;
}

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

ProjArgs proj_args_for(const IterPtrs& P, double rho) {
    ProjArgs a{};
    a.order = P.order;
    a.size = P.blk_size;
    a.off = P.blk_off64;
    a.count = P.p;
    a.rho = rho;
    a.x = P.x;
    a.gather_idx = P.gather_idx;
    a.lam = P.lam;
    a.v = P.vk;
    a.xk[0] = P.xk[0];
    a.xk[1] = P.xk[1];
    a.part = P.part_blk;
    a.ctrl = P.ctrl;
    return a;
}

}  // namespace

int iteration_kernel_count(int form) { return form == SDP_PRIMAL ? 7 : 8; }

cudaError_t iteration_prepare() {
    // y / z / t staged in shared memory: up to SDP_MAX_CONSTRAINTS doubles.
    const int bytes = SDP_MAX_CONSTRAINTS * (int)sizeof(double);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_tri_lower, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_tri_upper, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_spmv_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// Optional per-kernel timing: when ev != nullptr, ev[i] is recorded before kernel i of the
// iteration and ev[count] after the last one.
struct Marks {
    cudaEvent_t* ev;
    cudaStream_t st;
    int i;
    void mark() {
        if (ev) cudaEventRecord(ev[i], st);
        ++i;
    }
};

cudaError_t launch_affine(const IterPtrs& P, int form, double rinv, cudaStream_t st, Marks& mk) {
    mk.mark();
    k_spmv_rows<<<P.m * P.R, kRowThreads, 0, st>>>(P);
    const int tri_ctas = cdiv(P.m, kTriThreads / 32);
    mk.mark();
    k_tri_lower<<<tri_ctas, kTriThreads, (size_t)P.m * sizeof(double), st>>>(P, rinv, form);
    mk.mark();
    k_tri_upper<<<tri_ctas, kTriThreads, (size_t)P.m * sizeof(double), st>>>(P);
    mk.mark();
    k_spmv_cols<<<P.col_ctas, kColThreads, (size_t)P.m * sizeof(double), st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_iteration(const IterPtrs& P, int form, int prec, double rho, cudaStream_t st,
                             cudaEvent_t* ev) {
    const double rinv = 1.0 / rho;
    ProjArgs a = proj_args_for(P, rho);
    Marks mk{ev, st, 0};
    cudaError_t e;
    if (form == SDP_PRIMAL) {
        if ((e = launch_affine(P, form, rinv, st, mk)) != cudaSuccess) return e;
        mk.mark();
        if ((e = launch_project(a, PROJ_PRIMAL, prec, P.smax, st)) != cudaSuccess) return e;
        mk.mark();
        k_scatter_primal<<<P.ent_ctas, kEntThreads, 0, st>>>(P, rinv, 0);
    } else {
        a.out = P.xk[0];
        mk.mark();
        if ((e = launch_project(a, PROJ_DUAL, prec, P.smax, st)) != cudaSuccess) return e;
        mk.mark();
        k_scatter_dual<<<P.ent_ctas, kEntThreads, 0, st>>>(P, rinv);
        if ((e = launch_affine(P, form, rinv, st, mk)) != cudaSuccess) return e;
        mk.mark();
        k_update_dual<<<P.pos_ctas, kEntThreads, 0, st>>>(P, rho, rinv);
    }
    mk.mark();
    k_finalize<<<1, 256, 0, st>>>(P, form, rho);
    mk.mark();
    return cudaGetLastError();
}

const char* phase_name(int form, int i) {
    static const char* primal[] = {"spmv_rows", "tri_lower", "tri_upper", "spmv_cols",
                                   "project_primal", "scatter_primal", "finalize"};
    static const char* dual[] = {"project_dual", "scatter_dual", "spmv_rows", "tri_lower",
                                 "tri_upper", "spmv_cols", "update_dual", "finalize"};
    if (form == SDP_PRIMAL) return (i >= 0 && i < 7) ? primal[i] : nullptr;
    return (i >= 0 && i < 8) ? dual[i] : nullptr;
}

cudaError_t launch_primal_rebuild_r(const IterPtrs& P, double rho, cudaStream_t st) {
    k_scatter_primal<<<P.ent_ctas, kEntThreads, 0, st>>>(P, 1.0 / rho, 1);
    return cudaGetLastError();
}

cudaError_t launch_gather(const IterPtrs& P, const double* x, double* blocks, cudaStream_t st) {
    if (P.SL > 0) k_gather<<<cdiv(P.SL, kEntThreads), kEntThreads, 0, st>>>(P.gather_idx, P.SL, x, blocks);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const IterPtrs& P, const double* blocks, double* out, cudaStream_t st) {
    if (P.nEL > 0)
        k_scatter_plain<<<cdiv(P.nEL, kEntThreads), kEntThreads, 0, st>>>(P.sc_ptr, P.sc_pos, P.nEL, blocks, out);
    return cudaGetLastError();
}

cudaError_t launch_ctrl_arm(Ctrl* ctrl, int n_iters, double tol, cudaStream_t st) {
    k_ctrl_arm<<<1, 1, 0, st>>>(ctrl, n_iters, tol);
    return cudaGetLastError();
}

cudaError_t launch_ctrl_clear(Ctrl* ctrl, cudaStream_t st) {
    k_ctrl_clear<<<1, 1, 0, st>>>(ctrl);
    return cudaGetLastError();
}

cudaError_t launch_ctrl_reset(Ctrl* ctrl, cudaStream_t st) {
    k_ctrl_reset<<<1, 1, 0, st>>>(ctrl);
    return cudaGetLastError();
}

}  // namespace cadmm
