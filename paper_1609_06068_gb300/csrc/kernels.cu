// Per-iteration kernels of the decomposed ADMM other than the PSD projection:
//   scatter      r = sum_k H_k^T(.) and the KKT right-hand side (Eqs. OptCondMinYPrimal/Dual)
//   spmv_rows    t = A (w r / D)           (block elimination, first pass over A; CSR)
//   solve_y      y = M^-1 (t - rhs2)       (M = A D^-1 A^T, inverse formed at setup from its
//                                           cached Cholesky factor, Section III.B.1)
//   spmv_cols    x = (r - A^T y) / D       (second pass over A; CSC)
//   update_dual  v_k = z_k + rho^-1 lambda_k + H_k x, lambda_k = -rho H_k x (Eqs. vkEqn,
//                DualMultUpdate with the sign Eq. MultUpdateDualSDP implies)
// For a single problem the residuals, objectives and stop test of an iteration are computed by the
// last CTA to finish the iteration's final kernel (scatter in the primal form, update in the dual
// form), reading every partial sum in a fixed order. For a batch, each CTA works on one problem
// (its Sched entry) and a separate kernel finalizes every problem, one warp each; CTAs of a problem
// that has stopped return at once.
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

// Weight 1 (diagonal) or 2 (off-diagonal) as a double, by selection: an integer-to-double
// conversion would run on GB300's narrow FP64 pipe, which already limits these kernels.
__device__ __forceinline__ double wt(unsigned char w) { return w == 1 ? 1.0 : 2.0; }

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
    __syncthreads();
}

// The same sum for a CTA of exactly NT threads, transposed: every thread parks its K values in
// shared memory (value-major, buf holds K * NT + K doubles), then warp k adds value k's NT
// partials (NT / 32 per lane in order, then the shuffle tree). GB300 issues FP64 adds at a small
// fraction of its FP32 rate, so this matters: a shuffle tree in every warp for every value issues
// K * 5 adds per warp plus a second tree, this issues K * (NT / 32 + 5) adds in all.
template <int K, int NT>
__device__ __forceinline__ void block_sum_t(double (&v)[K], double* buf) {
    static_assert(K <= NT / 32, "one warp per value");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) buf[k * NT + tid] = v[k];
    __syncthreads();
    if (warp < K) {
        const double* col = buf + warp * NT + lane;
        double s = col[0];
#pragma unroll
        for (int j = 1; j < NT / 32; ++j) s += col[32 * j];
        s = warp_sum(s);
        if (lane == 0) buf[K * NT + warp] = s;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = buf[K * NT + k];
    __syncthreads();
}

// ---------------------------------------------------------------- residuals and stop test
// Run by one whole CTA (the last to finish the iteration's final kernel).
__device__ void finalize_iteration(const IterPtrs& P, int form, double rho, int n_part) {
    __shared__ double red[7 * kEntThreads + 7];     // callers run kEntThreads threads
    Ctrl* C = P.ctrl;
    double v[7] = {0, 0, 0, 0, 0, 0, 0};
    if (form == SDP_PRIMAL) {
        for (int k = threadIdx.x; k < P.p + P.ncs; k += blockDim.x) {   // cliques, then cone segments
            v[0] += P.part_blk[k * 4 + 0];
            v[1] += P.part_blk[k * 4 + 1];
            v[2] += P.part_blk[k * 4 + 2];
        }
        for (int q = threadIdx.x; q < n_part; q += blockDim.x) {
            v[3] += P.part_ent[q * 8 + 0];
            v[4] += P.part_ent[q * 8 + 1];
        }
    } else {
        for (int q = threadIdx.x; q < n_part; q += blockDim.x)
            for (int k = 0; k < 5; ++k) v[k] += P.part_ent[q * 8 + k];
    }
    for (int q = threadIdx.x; q < P.col_chunks; q += blockDim.x) v[5] += P.part_obj[q];
    for (int i = threadIdx.x; i < P.m; i += blockDim.x) v[6] = fma(P.b[i], P.y[i], v[6]);
    block_sum_t<7, kEntThreads>(v, red);
    if (threadIdx.x >= 32) return;
    // The five square roots in lanes 0-4 and the two ratios in lanes 0-1 at once (each is a
    // chain of dependent FP64 operations; in one thread they would run one after another).
    const int lane = threadIdx.x;
    const double sq = sqrt(lane == 0 ? v[0] : lane == 1 ? v[1] : lane == 2 ? v[2] : lane == 3 ? v[3] : v[4]);
    const double q0 = __shfl_sync(0xffffffffu, sq, 0), q1 = __shfl_sync(0xffffffffu, sq, 1);
    const double q2 = __shfl_sync(0xffffffffu, sq, 2), q3 = __shfl_sync(0xffffffffu, sq, 3);
    const double q4 = __shfl_sync(0xffffffffu, sq, 4);
    const double ratio = lane == 0 ? q0 / fmax(fmax(q1, q2), 1e-12) : rho * q3 / fmax(q4, 1e-12);
    const double eps_p = __shfl_sync(0xffffffffu, ratio, 0), eps_d = __shfl_sync(0xffffffffu, ratio, 1);
    if (lane != 0) return;
    double obj_p, obj_d;
    if (form == SDP_PRIMAL) {
        obj_p = v[5];
        obj_d = -rho * v[6];
    } else {
        obj_d = v[6];
        obj_p = -rho * v[5];
    }
    const int it = C->iter + 1;
    C->iter = it;
    C->eps_p = eps_p;
    C->eps_d = eps_d;
    C->obj_p = obj_p;
    C->obj_d = obj_d;
    C->ticket = 0;
    int st = SDP_MAX_ITER;
    if (!isfinite(eps_p) || !isfinite(eps_d) || !isfinite(obj_p) || !isfinite(obj_d)) {
        st = C->status = SDP_ERR_NAN;
        C->done = 1;
    } else if (fmax(eps_p, eps_d) < C->tol) {
        st = C->status = SDP_OK;
        C->done = 1;
    } else if (it >= C->iter_limit) {
        C->status = SDP_MAX_ITER;
        C->done = 1;
    }
    P.inst_res[0] = eps_p;
    P.inst_res[1] = eps_d;
    P.inst_res[2] = obj_p;
    P.inst_res[3] = obj_d;
    P.inst_stat[0] = st;
}

// Residuals and stop test of every problem of a batch: one warp per problem sums its partials in
// a fixed order; the last CTA then sets the iteration's global outcome.
__global__ void __launch_bounds__(256) k_finalize_batch(IterPtrs P, int form, double rho) {
    __shared__ double red[33 * 4];
    __shared__ int red_i[33 * 2];
    __shared__ bool s_last;
    pdl_wait();
    Ctrl* C = P.ctrl;
    if (C->done) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = blockIdx.x * (blockDim.x >> 5) + warp;
    const int it = C->iter + 1;
    if (q < P.ninst && P.inst_conv[q] < 0) {
        double v[7] = {0, 0, 0, 0, 0, 0, 0};
        if (form == SDP_PRIMAL) {
            for (int k = P.inst_cl[q] + lane; k < P.inst_cl[q + 1]; k += 32) {
                v[0] += P.part_blk[k * 4 + 0];
                v[1] += P.part_blk[k * 4 + 1];
                v[2] += P.part_blk[k * 4 + 2];
            }
            for (int c = P.inst_ent_cta[q] + lane; c < P.inst_ent_cta[q + 1]; c += 32) {
                v[3] += P.part_ent[c * 8 + 0];
                v[4] += P.part_ent[c * 8 + 1];
            }
            for (int c = P.inst_heavy_cta[q] + lane; c < P.inst_heavy_cta[q + 1]; c += 32) {
                v[3] += P.part_ent[(P.ent_ctas + c) * 8 + 0];
                v[4] += P.part_ent[(P.ent_ctas + c) * 8 + 1];
            }
        } else {
            for (int c = P.inst_pos_cta[q] + lane; c < P.inst_pos_cta[q + 1]; c += 32)
                for (int k = 0; k < 5; ++k) v[k] += P.part_ent[c * 8 + k];
        }
        for (int c = P.inst_col_chunk[q] + lane; c < P.inst_col_chunk[q + 1]; c += 32) v[5] += P.part_obj[c];
        for (int i = P.inst_row[q] + lane; i < P.inst_row[q + 1]; i += 32) v[6] = fma(P.b[i], P.y[i], v[6]);
#pragma unroll
        for (int k = 0; k < 7; ++k) v[k] = warp_sum(v[k]);
        if (lane == 0) {
            const double eps_p = sqrt(v[0]) / fmax(fmax(sqrt(v[1]), sqrt(v[2])), 1e-12);
            const double eps_d = rho * sqrt(v[3]) / fmax(sqrt(v[4]), 1e-12);
            const double obj_p = form == SDP_PRIMAL ? v[5] : -rho * v[5];
            const double obj_d = form == SDP_PRIMAL ? -rho * v[6] : v[6];
            P.inst_res[q * 4 + 0] = eps_p;
            P.inst_res[q * 4 + 1] = eps_d;
            P.inst_res[q * 4 + 2] = obj_p;
            P.inst_res[q * 4 + 3] = obj_d;
            if (!isfinite(eps_p) || !isfinite(eps_d) || !isfinite(obj_p) || !isfinite(obj_d)) {
                P.inst_stat[q] = SDP_ERR_NAN;
                P.inst_conv[q] = it;
            } else if (fmax(eps_p, eps_d) < C->tol) {
                P.inst_stat[q] = SDP_OK;
                P.inst_conv[q] = it;
            }
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&C->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // Global outcome: residual maxima and objective sums over all problems (their last values).
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    int active = 0, nan = 0;
    for (int k = threadIdx.x; k < P.ninst; k += blockDim.x) {
        v[0] = fmax(v[0], P.inst_res[k * 4 + 0]);
        v[1] = fmax(v[1], P.inst_res[k * 4 + 1]);
        v[2] += P.inst_res[k * 4 + 2];
        v[3] += P.inst_res[k * 4 + 3];
        active += P.inst_conv[k] < 0;
        nan += P.inst_stat[k] == SDP_ERR_NAN;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v[0] = fmax(v[0], __shfl_xor_sync(0xffffffffu, v[0], o));
        v[1] = fmax(v[1], __shfl_xor_sync(0xffffffffu, v[1], o));
        v[2] += __shfl_xor_sync(0xffffffffu, v[2], o);
        v[3] += __shfl_xor_sync(0xffffffffu, v[3], o);
        active += __shfl_xor_sync(0xffffffffu, active, o);
        nan += __shfl_xor_sync(0xffffffffu, nan, o);
    }
    const int nw = blockDim.x >> 5;
    if (lane == 0) {
        for (int k = 0; k < 4; ++k) red[warp * 4 + k] = v[k];
        red_i[warp * 2 + 0] = active;
        red_i[warp * 2 + 1] = nan;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double g[4] = {0.0, 0.0, 0.0, 0.0};
    int ga = 0, gn = 0;
    for (int w = 0; w < nw; ++w) {
        g[0] = fmax(g[0], red[w * 4 + 0]);
        g[1] = fmax(g[1], red[w * 4 + 1]);
        g[2] += red[w * 4 + 2];
        g[3] += red[w * 4 + 3];
        ga += red_i[w * 2 + 0];
        gn += red_i[w * 2 + 1];
    }
    C->iter = it;
    C->eps_p = g[0];
    C->eps_d = g[1];
    C->obj_p = g[2];
    C->obj_d = g[3];
    C->ticket = 0;
    C->active = ga;
    if (ga == 0) {
        C->status = gn > 0 ? SDP_ERR_NAN : SDP_OK;
        C->done = 1;
    } else if (it >= C->iter_limit) {
        C->status = gn > 0 ? SDP_ERR_NAN : SDP_MAX_ITER;
        C->done = 1;
    }
}

// True when CTA work for problem q must be skipped: it belongs to a batch and has stopped.
__device__ __forceinline__ bool stopped(const IterPtrs& P, int q) { return P.ninst > 1 && P.inst_conv[q] >= 0; }

// After a CTA has written its partial sums: count it, and let the last one finalize.
__device__ __forceinline__ void finish_and_maybe_finalize(const IterPtrs& P, int form, double rho, int n_part) {
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&P.ctrl->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last) {
        __threadfence();
        finalize_iteration(P, form, rho, n_part);
    }
}

// ---------------------------------------------------------------- scatter (primal form)
// r = sum_k H_k^T(x_k + rho^-1 lambda_k) - rho^-1 c, summed in ascending k from the first term;
// also the dual-residual pieces ||sum_k H_k^T(x_k+ - x_k)||^2 and ||sum_k H_k^T lambda_k||^2.
// use_current = 1 rebuilds r from the current blocks (after a reset or a state upload) and skips
// the residual work. CTAs [0, ent_ctas) take one entry per thread, adding its terms in ascending
// clique order (heavily shared entries are left to the others); CTAs [ent_ctas, ent_ctas +
// heavy_ctas) take one heavily shared entry per warp: lane t adds terms t, t+32, ... and the
// lanes' sums meet in a fixed shuffle tree (deterministic; equal to the ascending sum up to
// rounding, where a sequential sum over thousands of cliques would serialize the whole warp).
__global__ void __launch_bounds__(kEntThreads) k_scatter_primal(IterPtrs P, double rinv, double rho, int use_current) {
    __shared__ double red[2 * kEntThreads + 2];
    pdl_wait();
    const bool light = (int)blockIdx.x < P.ent_ctas;
    const Sched sc = light ? P.ent_sched[blockIdx.x] : P.heavy_sched[blockIdx.x - P.ent_ctas];
    if (P.ctrl->done) return;         // the schedule entry above is read alongside the flag
    const bool odd = (P.ctrl->iter & 1) != 0;
    const double* cur = odd ? P.xk[1] : P.xk[0];
    const double* nxt = odd ? P.xk[0] : P.xk[1];
    const double* xn_buf = use_current ? cur : nxt;
    const double* xo_buf = cur;
    double v[2] = {0.0, 0.0};
    if (!use_current && stopped(P, sc.q)) return;
    if (light) {
        const int e = sc.lo + threadIdx.x;
        if (e < sc.hi) {
            const int j0 = P.sc_ptr[e], j1 = P.sc_ptr[e + 1];
            if (j1 - j0 <= kHeavyCount) {
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
                const double w = wt(P.ew[e]);
                v[0] = w * dsum * dsum;
                v[1] = w * lsum * lsum;
            }
        }
    } else {
        const int lane = threadIdx.x & 31;
        const int hw = sc.lo + (threadIdx.x >> 5);
        if (hw < sc.hi) {
            const int e = P.heavy[hw];
            const int j0 = P.sc_ptr[e], j1 = P.sc_ptr[e + 1];
            double acc = 0.0, dsum = 0.0, lsum = 0.0;
#pragma unroll 4
            for (int j = j0 + lane; j < j1; j += 32) {
                const int pos = P.sc_pos[j];
                const double xn = xn_buf[pos], xo = xo_buf[pos], l = P.lam[pos];
                acc = __dadd_rn(acc, __dadd_rn(xn, __dmul_rn(rinv, l)));
                dsum += xn - xo;
                lsum += l;
            }
            acc = warp_sum(acc);
            dsum = warp_sum(dsum);
            lsum = warp_sum(lsum);
            if (lane == 0) {
                const double re = __dsub_rn(acc, __dmul_rn(rinv, P.c[e]));
                P.r[e] = re;
                P.rsw[e] = re * P.wdinv[e];
                const double w = wt(P.ew[e]);
                v[0] = w * dsum * dsum;
                v[1] = w * lsum * lsum;
            }
        }
    }
    if (use_current) return;
    pdl_trigger();
    block_sum_t<2, kEntThreads>(v, red);
    if (threadIdx.x == 0) {
        P.part_ent[blockIdx.x * 8 + 0] = v[0];
        P.part_ent[blockIdx.x * 8 + 1] = v[1];
    }
    if (P.ninst == 1) finish_and_maybe_finalize(P, SDP_PRIMAL, rho, P.ent_ctas + P.heavy_ctas);
}

// ---------------------------------------------------------------- scatter (dual form)
// r = c - sum_k H_k^T(z_k + rho^-1 lambda_k), ascending k from the first term for light entries;
// the same split between light entries (one per thread) and heavily shared ones (one per warp,
// lane-strided partial sums and a fixed shuffle tree).
__global__ void __launch_bounds__(kEntThreads) k_scatter_dual(IterPtrs P, double rinv) {
    pdl_wait();
    const bool light = (int)blockIdx.x < P.ent_ctas;
    const Sched sc = light ? P.ent_sched[blockIdx.x] : P.heavy_sched[blockIdx.x - P.ent_ctas];
    if (P.ctrl->done) return;         // the schedule entry above is read alongside the flag
    const double* z = P.xk[0];
    if (stopped(P, sc.q)) return;
    if (light) {
        const int e = sc.lo + threadIdx.x;
        if (e >= sc.hi) return;
        const int j0 = P.sc_ptr[e], j1 = P.sc_ptr[e + 1];
        if (j1 - j0 > kHeavyCount) return;
        double acc = 0.0;
        for (int j = j0; j < j1; ++j) {
            const int pos = P.sc_pos[j];
            const double term = __dadd_rn(z[pos], __dmul_rn(rinv, P.lam[pos]));
            acc = (j == j0) ? term : __dadd_rn(acc, term);
        }
        const double re = __dsub_rn(P.c[e], acc);
        P.r[e] = re;
        P.rsw[e] = re * P.wdinv[e];
        return;
    }
    const int lane = threadIdx.x & 31;
    const int hw = sc.lo + (threadIdx.x >> 5);
    if (hw >= sc.hi) return;
    const int e = P.heavy[hw];
    const int j0 = P.sc_ptr[e], j1 = P.sc_ptr[e + 1];
    double acc = 0.0;
#pragma unroll 4
    for (int j = j0 + lane; j < j1; j += 32) {
        const int pos = P.sc_pos[j];
        acc = __dadd_rn(acc, __dadd_rn(z[pos], __dmul_rn(rinv, P.lam[pos])));
    }
    acc = warp_sum(acc);
    if (lane == 0) {
        const double re = __dsub_rn(P.c[e], acc);
        P.r[e] = re;
        P.rsw[e] = re * P.wdinv[e];
    }
}

// ---------------------------------------------------------------- t = A (w r / D), CSR chunks
// One warp per chunk of a row (no block-wide reduction); four loads in flight per lane.
__global__ void __launch_bounds__(kRowThreads) k_spmv_rows(IterPtrs P) {
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int ch = blockIdx.x * (kRowThreads / 32) + (threadIdx.x >> 5);
    if (ch >= P.row_chunks) return;
    const Sched sc = P.row_sched[ch];
    if (P.ctrl->done) return;         // the chunk above is read alongside the flag
    if (stopped(P, sc.q)) return;
    const int hi = sc.hi;
    double a0 = 0.0, a1 = 0.0;
    int j = sc.lo + lane;
    for (; j + 96 < hi; j += 128) {
        const double v0 = P.a_val[j], v1 = P.a_val[j + 32], v2 = P.a_val[j + 64], v3 = P.a_val[j + 96];
        const int c0 = P.a_col[j], c1 = P.a_col[j + 32], c2 = P.a_col[j + 64], c3 = P.a_col[j + 96];
        a0 = fma(v0, P.rsw[c0], a0);
        a1 = fma(v1, P.rsw[c1], a1);
        a0 = fma(v2, P.rsw[c2], a0);
        a1 = fma(v3, P.rsw[c3], a1);
    }
    for (; j < hi; j += 32) a0 = fma(P.a_val[j], P.rsw[P.a_col[j]], a0);
    pdl_trigger();
    const double t = warp_sum(a0 + a1);
    if (lane == 0) P.tpart[ch] = t;
}

// ---------------------------------------------------------------- y = M^-1 (t - rhs2)
// t = A (w r / D) from the row chunks' partial sums, rhs2 = b (primal), -rho^-1 b (dual) or 0
// (kKktZeroRhs: the adjoint solve). M^-1 = (A D^-1 A^T)^-1 is formed at setup from the Cholesky
// factor (L^-T L^-1), so the block elimination's two triangular products are one product: each
// CTA stages t - rhs2 of its problem in shared memory, one warp per row of M^-1.
__global__ void __launch_bounds__(kTriThreads) k_solve_y(IterPtrs P, double rinv, int form) {
    extern __shared__ double u[];
    pdl_wait();
    const Sched sc = P.tri_sched[blockIdx.x];
    if (P.ctrl->done) return;         // the schedule entry above is read alongside the flag
    if (stopped(P, sc.q)) return;
    const int r0 = P.inst_row[sc.q], m = P.inst_row[sc.q + 1] - r0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double t = 0.0;
        for (int c = P.row_chunk[r0 + i]; c < P.row_chunk[r0 + i + 1]; ++c) t += P.tpart[c];
        const double bi = P.b[r0 + i];
        const double rhs2 = form == SDP_PRIMAL ? bi : (form == SDP_DUAL ? -__dmul_rn(rinv, bi) : 0.0);
        u[i] = t - rhs2;
    }
    __syncthreads();
    const double* Mb = P.Minv + P.mblk_off[sc.q];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int grow = sc.lo + warp; grow < sc.hi; grow += nw) {
        const double* Mr = Mb + (size_t)(grow - r0) * m;
        double a0 = 0.0, a1 = 0.0;
        int j = lane;
        for (; j + 32 < m; j += 64) {
            a0 = fma(Mr[j], u[j], a0);
            a1 = fma(Mr[j + 32], u[j + 32], a1);
        }
        if (j < m) a0 = fma(Mr[j], u[j], a0);
        const double acc = warp_sum(a0 + a1);
        if (lane == 0) P.y[grow] = acc;
    }
}

// ---------------------------------------------------------------- y = L^-T (L^-1 (t - rhs2))
// The same solve for an ill-conditioned M: with the explicit M^-1, x = D^-1 (r - A^T y) misses
// A x = rhs2 by about kappa(M) eps; with the two triangular factors (the inverse of the cached
// Cholesky factor, formed by substitution at setup) by about eps. z1 = L^-1 (t - rhs2): one warp
// per row of L^-1, t - rhs2 staged in shared memory as in k_solve_y.
__global__ void __launch_bounds__(kTriThreads) k_tri_lower(IterPtrs P, double rinv, int form) {
    extern __shared__ double u[];
    pdl_wait();
    const Sched sc = P.tri_sched[blockIdx.x];
    if (P.ctrl->done) return;         // the schedule entry above is read alongside the flag
    if (stopped(P, sc.q)) return;
    const int r0 = P.inst_row[sc.q], m = P.inst_row[sc.q + 1] - r0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double t = 0.0;
        for (int c = P.row_chunk[r0 + i]; c < P.row_chunk[r0 + i + 1]; ++c) t += P.tpart[c];
        const double bi = P.b[r0 + i];
        const double rhs2 = form == SDP_PRIMAL ? bi : (form == SDP_DUAL ? -__dmul_rn(rinv, bi) : 0.0);
        u[i] = t - rhs2;
    }
    __syncthreads();
    const double* Lb = P.Linv + P.mblk_off[sc.q];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int grow = sc.lo + warp; grow < sc.hi; grow += nw) {
        const int row = grow - r0;
        const double* Lr = Lb + (size_t)row * m;
        double a0 = 0.0, a1 = 0.0;
        int j = lane;
        for (; j + 32 <= row; j += 64) {
            a0 = fma(Lr[j], u[j], a0);
            a1 = fma(Lr[j + 32], u[j + 32], a1);
        }
        if (j <= row) a0 = fma(Lr[j], u[j], a0);
        const double acc = warp_sum(a0 + a1);
        if (lane == 0) P.z1[grow] = acc;
    }
}

// y = L^-T z1: row i of L^-T is column i of L^-1, read as row i of (L^-1)^T (entries i .. m-1).
__global__ void __launch_bounds__(kTriThreads) k_tri_upper(IterPtrs P) {
    extern __shared__ double zs[];
    pdl_wait();
    const Sched sc = P.tri_sched[blockIdx.x];
    if (P.ctrl->done) return;
    if (stopped(P, sc.q)) return;
    const int r0 = P.inst_row[sc.q], m = P.inst_row[sc.q + 1] - r0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) zs[i] = P.z1[r0 + i];
    __syncthreads();
    const double* Lb = P.LinvT + P.mblk_off[sc.q];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int grow = sc.lo + warp; grow < sc.hi; grow += nw) {
        const int row = grow - r0;
        const double* Lr = Lb + (size_t)row * m;
        double a0 = 0.0, a1 = 0.0;
        int i = row + lane;
        for (; i + 32 < m; i += 64) {
            a0 = fma(Lr[i], zs[i], a0);
            a1 = fma(Lr[i + 32], zs[i + 32], a1);
        }
        if (i < m) a0 = fma(Lr[i], zs[i], a0);
        const double acc = warp_sum(a0 + a1);
        if (lane == 0) P.y[grow] = acc;
    }
}

// ---------------------------------------------------------------- x = (r - A^T y) / D
// A^T in sliced ELL form (columns ordered by length within windows of 256, so slices pad
// little): one CTA per chunk of slices of one problem, its warps taking the slices in turn, one
// lane per column, so every load of a slice is coalesced and no lane-to-lane reduction is needed.
// The problem's y is staged in shared memory: the lanes of a warp read 32 scattered rows of it per
// step, which shared memory serves in a few cycles where the L1 cache needs one pass per line.
// Also the partial objective sum_e w_e c_e x_e of the chunk.
__global__ void __launch_bounds__(kColThreads) k_spmv_cols(IterPtrs P) {
    constexpr int NW = kColThreads / 32;
    extern __shared__ double ys[];
    __shared__ double red[33];
    pdl_wait();
    const Sched sc = P.col_sched[blockIdx.x];
    if (P.ctrl->done) return;         // the schedule entry above is read alongside the flag
    if (stopped(P, sc.q)) return;
    const int r0 = P.inst_row[sc.q], m = P.inst_row[sc.q + 1] - r0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) ys[i] = P.y[r0 + i];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double obj = 0.0;
    // Slices in rounds of NW, warp w taking slot w of even rounds and slot NW-1-w of odd ones:
    // within a window the slices shorten (columns are sorted by length), so the snake order
    // pairs long slices with short ones for every warp.
    for (int base = sc.lo; base < sc.hi; base += NW) {
        const int sl = base + (((base - sc.lo) / NW) & 1 ? NW - 1 - w : w);
        if (sl >= sc.hi) continue;
        const int e = P.sell_col[32 * sl + lane], len = P.sell_len[sl];
        const double* __restrict__ val = P.sell_val + P.sell_off[sl] + lane;
        const unsigned short* __restrict__ row = P.sell_row + P.sell_off[sl] + lane;
        // eight loads in flight per lane, four independent FMA chains
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int k = 0;
        for (; k + 7 < len; k += 8) {
            double v[8];
            int q[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                v[t] = val[32 * (k + t)];
                q[t] = row[32 * (k + t)];
            }
            s0 = fma(v[0], ys[q[0]], s0);
            s1 = fma(v[1], ys[q[1]], s1);
            s2 = fma(v[2], ys[q[2]], s2);
            s3 = fma(v[3], ys[q[3]], s3);
            s0 = fma(v[4], ys[q[4]], s0);
            s1 = fma(v[5], ys[q[5]], s1);
            s2 = fma(v[6], ys[q[6]], s2);
            s3 = fma(v[7], ys[q[7]], s3);
        }
        for (; k < len; ++k) s0 = fma(val[32 * k], ys[row[32 * k]], s0);
        if (e >= 0) {
            const double xe = (P.r[e] - ((s0 + s1) + (s2 + s3))) * P.dinv[e];
            P.x[e] = xe;
            obj = fma(wt(P.ew[e]) * P.c[e], xe, obj);
        }
    }
    pdl_trigger();
    double v[1] = {obj};
    block_sum<1>(v, red);
    if (threadIdx.x == 0) P.part_obj[blockIdx.x] = v[0];
}

// The same product for problems with few slices: one CTA per slice, its 8 warps splitting the
// slice's length and their partial sums added in warp order by warp 0.
__global__ void __launch_bounds__(kColThreads) k_spmv_cols_split(IterPtrs P) {
    constexpr int NW = kColThreads / 32;
    __shared__ double part[NW][32];
    pdl_wait();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const Sched sc = P.col_sched[blockIdx.x];
    if (P.ctrl->done) return;         // the schedule entry above is read alongside the flag
    if (stopped(P, sc.q)) return;
    const int sl = sc.lo, len = P.sell_len[sl];
    const int k0 = (int)((long long)len * w / NW), k1 = (int)((long long)len * (w + 1) / NW);
    const double* __restrict__ y = P.y + P.inst_row[sc.q];
    const double* __restrict__ val = P.sell_val + P.sell_off[sl] + lane;
    const unsigned short* __restrict__ row = P.sell_row + P.sell_off[sl] + lane;
    double s0 = 0.0, s1 = 0.0;
    int k = k0;
    for (; k + 3 < k1; k += 4) {
        const double v0 = val[32 * k], v1 = val[32 * (k + 1)], v2 = val[32 * (k + 2)], v3 = val[32 * (k + 3)];
        const int r0 = row[32 * k], r1 = row[32 * (k + 1)], r2 = row[32 * (k + 2)], r3 = row[32 * (k + 3)];
        s0 = fma(v0, __ldg(y + r0), s0);
        s1 = fma(v1, __ldg(y + r1), s1);
        s0 = fma(v2, __ldg(y + r2), s0);
        s1 = fma(v3, __ldg(y + r3), s1);
    }
    for (; k < k1; ++k) s0 = fma(val[32 * k], __ldg(y + row[32 * k]), s0);
    part[w][lane] = s0 + s1;
    __syncthreads();
    if (w != 0) return;
    double s = part[0][lane];
#pragma unroll
    for (int ww = 1; ww < NW; ++ww) s += part[ww][lane];
    const int e = P.sell_col[32 * sl + lane];
    double obj = 0.0;
    if (e >= 0) {
        const double xe = (P.r[e] - s) * P.dinv[e];
        P.x[e] = xe;
        obj = wt(P.ew[e]) * P.c[e] * xe;
    }
    pdl_trigger();
    obj = warp_sum(obj);
    if (lane == 0) P.part_obj[blockIdx.x] = obj;
}

// ---------------------------------------------------------------- dual-form multiplier update
// v_k = z_k + rho^-1 lambda_k + H_k x (Eq. vkEqn), lambda_k = -rho H_k x (Eq. DualMultUpdate with
// the sign Eq. MultUpdateDualSDP implies), and the residual sums; the last CTA finalizes.
__global__ void __launch_bounds__(kEntThreads) k_update_dual(IterPtrs P, double rho, double rinv) {
    __shared__ double red[5 * kEntThreads + 5];
    pdl_wait();
    const Sched sc = P.pos_sched[blockIdx.x];
    if (P.ctrl->done) return;         // the schedule entry above is read alongside the flag
    if (stopped(P, sc.q)) return;
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    // Four positions per step, all of their loads issued before any arithmetic (one step when a
    // CTA has at most one position per thread).
    constexpr int U = 4;
    const int bd = blockDim.x;
    if (sc.hi - sc.lo <= bd) {
        const int pos = sc.lo + threadIdx.x;
        if (pos < sc.hi) {
            const double u = P.x[P.gather_idx[pos]];
            const double z = P.xk[0][pos], l = P.lam[pos], vo = P.vk[pos];
            const double vn = __dadd_rn(__dadd_rn(z, __dmul_rn(rinv, l)), u);
            const double ln = __dmul_rn(-rho, u);
            P.vk[pos] = vn;
            P.lam[pos] = ln;
            const double w = wt(P.pos_w[pos]);
            const double d1 = z - vn, d2 = vn - vo;
            v[0] = w * d1 * d1;
            v[1] = w * z * z;
            v[2] = w * vn * vn;
            v[3] = w * d2 * d2;
            v[4] = w * ln * ln;
        }
    }
    for (int base = sc.lo + threadIdx.x; base < sc.hi && sc.hi - sc.lo > bd; base += U * bd) {
        int gi[U];
        double z[U], l[U], vo[U], u[U], w[U];
#pragma unroll
        for (int t = 0; t < U; ++t) {
            const int pos = base + t * bd;
            const bool ok = pos < sc.hi;
            gi[t] = ok ? P.gather_idx[pos] : 0;
            z[t] = ok ? P.xk[0][pos] : 0.0;
            l[t] = ok ? P.lam[pos] : 0.0;
            vo[t] = ok ? P.vk[pos] : 0.0;
            w[t] = ok ? wt(P.pos_w[pos]) : 0.0;
        }
#pragma unroll
        for (int t = 0; t < U; ++t) u[t] = P.x[gi[t]];
#pragma unroll
        for (int t = 0; t < U; ++t) {
            const int pos = base + t * bd;
            const double vn = __dadd_rn(__dadd_rn(z[t], __dmul_rn(rinv, l[t])), u[t]);
            const double ln = __dmul_rn(-rho, u[t]);
            if (pos < sc.hi) {
                P.vk[pos] = vn;
                P.lam[pos] = ln;
            }
            const double d1 = z[t] - vn, d2 = vn - vo[t];
            v[0] = fma(w[t] * d1, d1, v[0]);
            v[1] = fma(w[t] * z[t], z[t], v[1]);
            v[2] = fma(w[t] * vn, vn, v[2]);
            v[3] = fma(w[t] * d2, d2, v[3]);
            v[4] = fma(w[t] * ln, ln, v[4]);
        }
    }
    pdl_trigger();
    block_sum_t<5, kEntThreads>(v, red);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 5; ++k) P.part_ent[blockIdx.x * 8 + k] = v[k];
    }
    if (P.ninst == 1) finish_and_maybe_finalize(P, SDP_DUAL, rho, (int)gridDim.x);
}

__global__ void k_ctrl_arm(Ctrl* C, int n_iters, double tol) {
    C->done = n_iters > 0 ? 0 : 1;
    C->status = SDP_MAX_ITER;
    C->iter_limit = C->iter + n_iters;
    C->tol = tol;
    C->ticket = 0;
}

__global__ void k_ctrl_clear(Ctrl* C) { C->done = 0; }

__global__ void k_ctrl_reset(Ctrl* C) {
    C->iter = 0;
    C->iter_limit = 0;
    C->done = 0;
    C->status = SDP_MAX_ITER;
    C->ticket = 0;
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

// Identity eigenvector blocks (a warm start from them is a cold start).
template <typename T>
__global__ void k_vstore_identity(T* vs, const long long* voff, const int* size, int p) {
    const int k = blockIdx.x;
    if (k >= p) return;
    const int N = size[k] + (size[k] & 1);
    T* b = vs + voff[k];
    for (int q = threadIdx.x; q < N * N; q += blockDim.x) b[q] = (q / N == q % N) ? T(1) : T(0);
}

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

ProjArgs proj_args_for(const IterPtrs& P, double rho) {
    ProjArgs a{};
    a.pdl = P.pdl;
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
    a.vstore = P.vstore;
    a.voff = P.voff;
    a.ctrl = P.ctrl;
    a.blk_inst = P.ninst > 1 ? P.blk_inst : nullptr;
    a.inst_conv = P.ninst > 1 ? P.inst_conv : nullptr;
    return a;
}

// ---------------------------------------------------------------- non-PSD cone blocks
// Section V: besides the PSD cone, CDCS accepts R^q (free), the nonnegative orthant and
// second-order cones Q^q = {(t, u) : ||u|| <= t}, and does not decompose them. Their variables are
// one block per cone after the clique blocks; each block is projected onto its cone in the primal
// form (Eq. XkUpdate) and onto the dual cone in the dual form (Eq. zkUpdate): {0} for R^q, the
// others are self-dual. The second-order projection is the point itself inside the cone, zero
// inside its polar cone, else ((t + ||u||) / 2) (1, u / ||u||). One CTA per segment: a range of
// free or nonnegative positions, one large second-order cone, or up to kSmallSocPerCta cones of
// dimension <= kSmallSoc taken by one thread each. GB300 issues FP64 at a small fraction of its
// FP32 rate, so a small cone is not spread over lanes: a lane per element would repeat the norm's
// reduction, the square root and the division for every lane of the cone. The thread reads its
// cone twice (the norm, then the result; the second pass hits L1). The epilogue is that of the
// PSD projections, with weight 1 on every position.
constexpr int kConeThreads = 256;

template <int MODE>
__device__ __forceinline__ double cone_w(const IterPtrs& P, int q, double rinv) {
    if (MODE == PROJ_PRIMAL) return __dsub_rn(P.x[P.gather_idx[q]], __dmul_rn(rinv, P.lam[q]));
    return __dsub_rn(P.vk[q], __dmul_rn(rinv, P.lam[q]));
}

// Second-order projection factors from t and ||u||: t -> t_out, u -> f u.
__device__ __forceinline__ void soc_factors(double t, double nu, double& t_out, double& f) {
    if (nu <= t) {
        t_out = t;
        f = 1.0;
    } else if (nu <= -t) {
        t_out = 0.0;
        f = 0.0;
    } else {
        t_out = 0.5 * (t + nu);
        f = t_out / nu;
    }
}

// Epilogue of one projected position xv (weight 1), shared by every cone kind.
template <int MODE>
__device__ __forceinline__ void cone_store(const IterPtrs& P, double* xk_new, int q, double xv, double rho,
                                           double (&pv)[3]) {
    if (MODE == PROJ_PRIMAL) {
        const double u = P.x[P.gather_idx[q]];
        const double d = xv - u;
        xk_new[q] = xv;
        P.lam[q] = P.lam[q] + rho * d;                         // Eq. LambdakUpdate
        pv[0] += d * d;
        pv[1] += xv * xv;
        pv[2] += u * u;
    } else {
        P.xk[0][q] = xv;                                       // z_k
    }
}

template <int MODE>
__global__ void __launch_bounds__(kConeThreads) k_project_cones(IterPtrs P, double rho, double rinv) {
    __shared__ double red[33 * 3];
    pdl_wait();
    const int sg = blockIdx.x;
    const int lo = P.cone_lo[sg], hi = P.cone_hi[sg], kind = P.cone_kind[sg];
    if (P.ctrl->done) return;         // the segment above is read alongside the flag
    double pv[3] = {0.0, 0.0, 0.0};
    double* xk_new = nullptr;
    if (MODE == PROJ_PRIMAL) xk_new = (P.ctrl->iter & 1) ? P.xk[0] : P.xk[1];
    if (kind == kConeSocSmall) {
        const int c = lo + (int)threadIdx.x;
        if (c < hi) {
            const int p0 = P.soc_pos[c], qd = P.soc_q[c];
            const double t = cone_w<MODE>(P, p0, rinv);
            double ss = 0.0;
            for (int j = 1; j < qd; ++j) {
                const double w = cone_w<MODE>(P, p0 + j, rinv);
                ss = fma(w, w, ss);
            }
            double t_out, f;
            soc_factors(t, sqrt(ss), t_out, f);
            cone_store<MODE>(P, xk_new, p0, t_out, rho, pv);
            for (int j = 1; j < qd; ++j) cone_store<MODE>(P, xk_new, p0 + j, f * cone_w<MODE>(P, p0 + j, rinv), rho, pv);
        }
    } else {
        double t_out = 0.0, f = 1.0;          // large second-order cone: t -> t_out, u -> f u
        if (kind == kConeSoc) {
            double ss[1] = {0.0};
            for (int q = lo + 1 + (int)threadIdx.x; q < hi; q += blockDim.x) {
                const double w = cone_w<MODE>(P, q, rinv);
                ss[0] = fma(w, w, ss[0]);
            }
            block_sum<1>(ss, red);
            soc_factors(cone_w<MODE>(P, lo, rinv), sqrt(ss[0]), t_out, f);
        }
        for (int q = lo + (int)threadIdx.x; q < hi; q += blockDim.x) {
            const double w = cone_w<MODE>(P, q, rinv);
            double xv;
            if (kind == kConeFree) xv = (MODE == PROJ_PRIMAL) ? w : 0.0;
            else if (kind == kConeNonneg) xv = w > 0.0 ? w : 0.0;
            else xv = (q == lo) ? t_out : f * w;
            cone_store<MODE>(P, xk_new, q, xv, rho, pv);
        }
    }
    pdl_trigger();
    if (MODE == PROJ_PRIMAL) {
        block_sum<3>(pv, red);
        if (threadIdx.x == 0) {
            double* part = P.part_blk + (size_t)(P.p + sg) * 4;
            part[0] = pv[0];
            part[1] = pv[1];
            part[2] = pv[2];
            part[3] = 0.0;
        }
    }
}

cudaError_t launch_project_cones(const IterPtrs& P, int mode, double rho, cudaStream_t st) {
    if (P.ncs <= 0) return cudaSuccess;
    if (mode == PROJ_PRIMAL)
        return launch_pdl(P.pdl != 0, k_project_cones<PROJ_PRIMAL>, dim3(P.ncs), dim3(kConeThreads), 0, st, P, rho, 1.0 / rho);
    return launch_pdl(P.pdl != 0, k_project_cones<PROJ_DUAL>, dim3(P.ncs), dim3(kConeThreads), 0, st, P, rho, 1.0 / rho);
}

// All runs of the projection plan, largest cliques first.
cudaError_t launch_project_plan(const ProjArgs& a, const IterPtrs& P, const ProjPlan& plan, int mode, int prec,
                                cudaStream_t st) {
    for (int r = 0; r < plan.runs; ++r) {
        ProjArgs b = a;
        b.order = plan.identity[r] ? nullptr : P.order + plan.start[r];
        b.first = plan.start[r];
        b.count = plan.count[r];
        const cudaError_t e = launch_project_variant(b, mode, prec, plan.variant[r], plan.smax[r], st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

__global__ void k_inst_reset(IterPtrs P) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= P.ninst) return;
    P.inst_conv[q] = -1;
    P.inst_stat[q] = SDP_MAX_ITER;
    for (int k = 0; k < 4; ++k) P.inst_res[q * 4 + k] = 0.0;
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

cudaError_t launch_affine(const IterPtrs& P, int form, double rho, double rinv, cudaStream_t st, Marks& mk) {
    cudaError_t e;
    mk.mark();
    const int warps = kRowThreads / 32;
    if ((e = launch_pdl(P.pdl != 0, k_spmv_rows, dim3(cdiv(P.row_chunks, warps)), dim3(kRowThreads), 0, st, P)) != cudaSuccess)
        return e;
    const size_t mbytes = (size_t)P.mmax * sizeof(double);   // the largest problem's y, staged
    mk.mark();
    if (P.kkt_tri) {
        if ((e = launch_pdl(P.pdl != 0, k_tri_lower, dim3(P.tri_ctas), dim3(kTriThreads), mbytes, st, P, rinv, form)) != cudaSuccess)
            return e;
        mk.mark();
        if ((e = launch_pdl(P.pdl != 0, k_tri_upper, dim3(P.tri_ctas), dim3(kTriThreads), mbytes, st, P)) != cudaSuccess) return e;
    } else if ((e = launch_pdl(P.pdl != 0, k_solve_y, dim3(P.tri_ctas), dim3(kTriThreads), mbytes, st, P, rinv, form)) != cudaSuccess) {
        return e;
    }
    mk.mark();
    if (P.col_split)
        e = launch_pdl(P.pdl != 0, k_spmv_cols_split, dim3(P.col_chunks), dim3(kColThreads), 0, st, P);
    else
        e = launch_pdl(P.pdl != 0, k_spmv_cols, dim3(P.col_chunks), dim3(kColThreads), mbytes, st, P);
    if (e != cudaSuccess) return e;
    if (form == SDP_DUAL) {
        mk.mark();
        return launch_pdl(P.pdl != 0, k_update_dual, dim3(P.pos_ctas), dim3(kEntThreads), 0, st, P, rho, rinv);
    }
    return cudaSuccess;
}

}  // namespace

int iteration_kernel_count(const IterPtrs& P, const ProjPlan& plan, int form) {
    return (form == SDP_PRIMAL ? 4 : 5) + plan.runs + (P.ncs > 0 ? 1 : 0) + (P.ninst > 1 ? 1 : 0) +
           (P.kkt_tri ? 1 : 0);
}

int phase_count(const IterPtrs& P, int form) {
    return (form == SDP_PRIMAL ? 5 : 6) + (P.ncs > 0 ? 1 : 0) + (P.ninst > 1 ? 1 : 0) + (P.kkt_tri ? 1 : 0);
}

cudaError_t iteration_prepare() {
    // y / z / t staged in shared memory: up to SDP_MAX_CONSTRAINTS doubles.
    const int bytes = SDP_MAX_CONSTRAINTS * (int)sizeof(double);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_solve_y, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_tri_lower, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_tri_upper, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_spmv_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_iteration(const IterPtrs& P, const ProjPlan& plan, int form, int prec, double rho,
                             cudaStream_t st, cudaEvent_t* ev) {
    const double rinv = 1.0 / rho;
    ProjArgs a = proj_args_for(P, rho);
    Marks mk{ev, st, 0};
    cudaError_t e;
    if (form == SDP_PRIMAL) {
        if ((e = launch_affine(P, form, rho, rinv, st, mk)) != cudaSuccess) return e;
        mk.mark();
        if ((e = launch_project_plan(a, P, plan, PROJ_PRIMAL, prec, st)) != cudaSuccess) return e;
        if (P.ncs > 0) mk.mark();
        if ((e = launch_project_cones(P, PROJ_PRIMAL, rho, st)) != cudaSuccess) return e;
        mk.mark();
        if ((e = launch_pdl(P.pdl != 0, k_scatter_primal, dim3(P.ent_ctas + P.heavy_ctas), dim3(kEntThreads), 0, st, P, rinv,
                            rho, 0)) != cudaSuccess)
            return e;
    } else {
        a.out = P.xk[0];
        mk.mark();
        if ((e = launch_project_plan(a, P, plan, PROJ_DUAL, prec, st)) != cudaSuccess) return e;
        if (P.ncs > 0) mk.mark();
        if ((e = launch_project_cones(P, PROJ_DUAL, rho, st)) != cudaSuccess) return e;
        mk.mark();
        if ((e = launch_pdl(P.pdl != 0, k_scatter_dual, dim3(P.ent_ctas + P.heavy_ctas), dim3(kEntThreads), 0, st, P,
                            rinv)) != cudaSuccess)
            return e;
        if ((e = launch_affine(P, form, rho, rinv, st, mk)) != cudaSuccess) return e;
    }
    if (P.ninst > 1) {
        mk.mark();
        const int ctas = (P.ninst + 7) / 8;
        if ((e = launch_pdl(P.pdl != 0, k_finalize_batch, dim3(ctas), dim3(256), 0, st, P, form, rho)) != cudaSuccess) return e;
    }
    mk.mark();
    return cudaGetLastError();
}

const char* phase_name(int form, bool batch, bool cones, bool tri, int i) {
    static const char* primal[] = {"spmv_rows", "solve_y", "spmv_cols", "project_primal", "project_cones",
                                   "scatter_primal+finalize", "finalize_batch"};
    static const char* dual[] = {"project_dual", "project_cones", "scatter_dual", "spmv_rows", "solve_y",
                                 "spmv_cols", "update_dual+finalize", "finalize_batch"};
    const char** list = form == SDP_PRIMAL ? primal : dual;
    const int cone_at = form == SDP_PRIMAL ? 4 : 1;
    const int solve_at = form == SDP_PRIMAL ? 1 : 4;
    const int n = (form == SDP_PRIMAL ? 5 : 6) + (cones ? 1 : 0) + (batch ? 1 : 0) + (tri ? 1 : 0);
    if (i < 0 || i >= n) return nullptr;
    // the triangular path has two phases in the slot of solve_y
    const int solve_pos = solve_at - (!cones && cone_at < solve_at ? 1 : 0);
    if (tri) {
        if (i == solve_pos) return "tri_lower";
        if (i == solve_pos + 1) return "tri_upper";
        if (i > solve_pos + 1) --i;
    }
    if (!cones && i >= cone_at) ++i;                    // no cone phase: skip its slot
    if (batch && i == (form == SDP_PRIMAL ? 5 : 6)) return form == SDP_PRIMAL ? "scatter_primal" : "update_dual";
    return list[i];
}

int resident_ctas(int kernel, size_t smem) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (kernel == 0) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_spmv_rows, kRowThreads, smem);
    if (kernel == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_spmv_cols, kColThreads, smem);
    if (kernel == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_update_dual, kEntThreads, smem);
    return e == cudaSuccess && n > 0 ? n : 1;
}

cudaError_t launch_kkt_adjoint(const IterPtrs& P, cudaStream_t st) {
    Marks mk{nullptr, st, 0};
    return launch_affine(P, kKktZeroRhs, 1.0, 1.0, st, mk);
}

__global__ void k_ctrl_set_iter(Ctrl* C, int it) { C->iter = it; }

cudaError_t launch_ctrl_set_iter(Ctrl* ctrl, int it, cudaStream_t st) {
    k_ctrl_set_iter<<<1, 1, 0, st>>>(ctrl, it);
    return cudaGetLastError();
}

cudaError_t launch_inst_reset(const IterPtrs& P, cudaStream_t st) {
    k_inst_reset<<<(P.ninst + 255) / 256, 256, 0, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_primal_rebuild_r(const IterPtrs& P, double rho, cudaStream_t st) {
    k_scatter_primal<<<P.ent_ctas + P.heavy_ctas, kEntThreads, 0, st>>>(P, 1.0 / rho, rho, 1);
    return cudaGetLastError();
}

cudaError_t launch_vstore_identity(const IterPtrs& P, int prec, cudaStream_t st) {
    if (P.vstore == nullptr || P.p <= 0) return cudaSuccess;
    if (prec == SDP_PROJ_FP32)
        k_vstore_identity<float><<<P.p, 256, 0, st>>>(static_cast<float*>(P.vstore), P.voff, P.blk_size, P.p);
    else
        k_vstore_identity<double><<<P.p, 256, 0, st>>>(static_cast<double*>(P.vstore), P.voff, P.blk_size, P.p);
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
