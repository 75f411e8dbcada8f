// Batched projection of small symmetric clique blocks onto the PSD cone (Eqs. XkUpdate, zkUpdate):
// P(W) = V diag(max(lambda, 0)) V^T, with the eigendecomposition by two-sided cyclic Jacobi.
//
// One CTA owns one clique block. The block and the eigenvector matrix V live in shared memory in
// the projection precision T (float or double). A sweep visits every index pair once in the
// round-robin ("circle") order: N/2 disjoint pairs per round, N-1 rounds (N = s rounded up to even;
// an odd block gets a zero padding row/column that never rotates). In a round, one thread per pair
// computes the rotation that zeroes a_pq (Golub & Van Loan, Sec. 8.5, symmetric Schur 2x2), then
// every thread applies J^T A J to whole 2x2 tiles (rows of pair I, columns of pair J), so the
// round needs two barriers and no intermediate copy. Sweeps stop once the off-diagonal Frobenius
// norm is below tol * ||W||_F. The reconstruction writes only the lower triangle, so the result
// is exactly symmetric; it is widened to FP64 on store.
#include <cstdio>

#include "sdp_internal.h"

namespace cadmm {

namespace {

template <typename T> struct JacobiParams;
template <> struct JacobiParams<float> {
    static constexpr float rel_tol = 1.0e-7f;
    static constexpr int max_sweeps = 24;
};
template <> struct JacobiParams<double> {
    static constexpr double rel_tol = 1.0e-15;
    static constexpr int max_sweeps = 30;
};

constexpr int kMaxPairs = SDP_MAX_CLIQUE / 2;

__device__ __forceinline__ int packed_pos(int a, int b, int s) {
    return b * s - (b * (b - 1)) / 2 + (a - b);  // column-major lower, a >= b
}

// Slot i of round r in the circle method for N players: slot 0 stays, the rest rotate.
__device__ __forceinline__ int rr_slot(int i, int r, int N) {
    return i == 0 ? 0 : 1 + ((i - 1 + r) % (N - 1));
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic CTA-wide sum of K values (fixed shuffle tree, then warp 0 over the warp sums);
// every thread receives lane 0's result.
template <typename T, int K>
__device__ __forceinline__ void block_sum_t(T (&v)[K], T* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = warp_sum_t(v[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) red[warp * K + k] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            T t = lane < nw ? red[lane * K + k] : T(0);
            t = warp_sum_t(t);
            if (lane == 0) red[32 * K + k] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = red[32 * K + k];
    __syncthreads();
}

__device__ __forceinline__ double block_max(double v, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double t = lane < nw ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
        if (lane == 0) red[32] = t;
    }
    __syncthreads();
    v = red[32];
    __syncthreads();
    return v;
}

// W_ij of one packed position: the block itself (standalone), H_k x - rho^-1 lambda_k (primal,
// Eq. XkUpdate; u = H_k x is kept in U for the multiplier update) or v_k - rho^-1 lambda_k (dual,
// Eq. zkUpdate).
template <int MODE>
__device__ __forceinline__ double load_w(const ProjArgs& a, long long off, int pos, double rinv, double* U) {
    if (MODE == PROJ_PLAIN) return a.in[off + pos];
    if (MODE == PROJ_PRIMAL) {
        const double u = a.x[a.gather_idx[off + pos]];
        U[pos] = u;
        return __dsub_rn(u, __dmul_rn(rinv, a.lam[off + pos]));
    }
    return __dsub_rn(a.v[off + pos], __dmul_rn(rinv, a.lam[off + pos]));
}

template <typename T>
__device__ __forceinline__ T t_sqrt(T x);
template <> __device__ __forceinline__ float t_sqrt<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double t_sqrt<double>(double x) { return sqrt(x); }

template <typename T, int MODE>
__global__ void __launch_bounds__(512) k_project(ProjArgs a, double rinv) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T s_c[kMaxPairs], s_s[kMaxPairs], s_t[kMaxPairs];
    __shared__ int s_p[kMaxPairs], s_q[kMaxPairs];
    __shared__ T red_t[33 * 2];
    __shared__ double red_d[33 * 3];

    if (a.ctrl != nullptr && a.ctrl->done) return;

    const int blk = a.order ? a.order[blockIdx.x] : (int)blockIdx.x;
    const int s = a.size[blk];
    const long long off = a.off[blk];
    const int N = s + (s & 1);
    const int LD = N + 1;
    const int H = N / 2;
    const int tid = threadIdx.x, nt = blockDim.x;

    T* A = reinterpret_cast<T*>(smem_raw);
    T* V = A + N * LD;
    T* dp = V + N * LD;
    const size_t ub = (size_t)(2 * N * LD + N) * sizeof(T);
    double* U = reinterpret_cast<double*>(smem_raw + ((ub + 15) & ~(size_t)15));

    double* xk_new = nullptr;
    if (MODE == PROJ_PRIMAL) xk_new = (a.ctrl->iter & 1) ? a.xk[0] : a.xk[1];

    // ---- load W into A (both triangles), V = I, zero padding
    for (int q = tid; q < N * N; q += nt) {
        const int i = q / N, j = q - (q / N) * N;
        V[i * LD + j] = (i == j) ? T(1) : T(0);
        if (i >= s || j >= s) A[i * LD + j] = T(0);
    }
    // Pass 1 finds max |W_ij|; pass 2 stores W scaled by the power of two 2^-e that brings it to
    // [1, 2), so squares and rotations stay in range in either precision. The scaling is exact
    // and is undone on the result.
    double wmax = 0.0;
    for (int q = tid; q < s * s; q += nt) {
        const int ra = q % s, cb = q / s;
        if (ra < cb) continue;
        const double w = load_w<MODE>(a, off, packed_pos(ra, cb, s), rinv, U);
        wmax = fmax(wmax, fabs(w));
    }
    wmax = block_max(wmax, red_d);
    const int e2 = (wmax > 0.0 && isfinite(wmax)) ? ilogb(wmax) : 0;
    for (int q = tid; q < s * s; q += nt) {
        const int ra = q % s, cb = q / s;
        if (ra < cb) continue;
        const int pos = packed_pos(ra, cb, s);
        const double w = (MODE == PROJ_PRIMAL) ? __dsub_rn(U[pos], __dmul_rn(rinv, a.lam[off + pos]))
                                               : load_w<MODE>(a, off, pos, rinv, U);
        const T wt = (T)ldexp(w, -e2);
        A[ra * LD + cb] = wt;
        A[cb * LD + ra] = wt;
    }
    __syncthreads();

    // ---- ||W||_F^2
    T nrm[1] = {T(0)};
    for (int q = tid; q < N * N; q += nt) {
        const T v = A[(q / N) * LD + (q % N)];
        nrm[0] += v * v;
    }
    block_sum_t<T, 1>(nrm, red_t);
    const T tol2 = JacobiParams<T>::rel_tol * JacobiParams<T>::rel_tol * nrm[0];

    // ---- cyclic Jacobi sweeps
    for (int sweep = 0; sweep < JacobiParams<T>::max_sweeps && N > 1; ++sweep) {
        T off2[1] = {T(0)};
        for (int q = tid; q < N * N; q += nt) {
            const int i = q / N, j = q - (q / N) * N;
            if (i != j) {
                const T v = A[i * LD + j];
                off2[0] += v * v;
            }
        }
        block_sum_t<T, 1>(off2, red_t);
        if (!(off2[0] > tol2)) break;

        for (int r = 0; r < N - 1; ++r) {
            if (tid < H) {
                int p = rr_slot(tid, r, N), q = rr_slot(N - 1 - tid, r, N);
                if (p > q) { const int t = p; p = q; q = t; }
                const T app = A[p * LD + p], aqq = A[q * LD + q], apq = A[p * LD + q];
                T c = T(1), sn = T(0), t = T(0);
                if (apq != T(0)) {
                    const T tau = (aqq - app) / (T(2) * apq);
                    t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + t_sqrt<T>(T(1) + tau * tau));
                    c = T(1) / t_sqrt<T>(T(1) + t * t);
                    sn = t * c;
                }
                s_p[tid] = p; s_q[tid] = q;
                s_c[tid] = c; s_s[tid] = sn; s_t[tid] = t;
            }
            __syncthreads();
            // A <- J^T A J on 2x2 tiles (I <= J; the mirror tile is written by the same thread)
            for (int w = tid; w < H * H; w += nt) {
                const int I = w / H, J = w - (w / H) * H;
                if (I > J) continue;
                const int pI = s_p[I], qI = s_q[I];
                if (I == J) {
                    const T apq = A[pI * LD + qI], t = s_t[I];
                    A[pI * LD + pI] -= t * apq;
                    A[qI * LD + qI] += t * apq;
                    A[pI * LD + qI] = T(0);
                    A[qI * LD + pI] = T(0);
                } else {
                    const int pJ = s_p[J], qJ = s_q[J];
                    const T cI = s_c[I], sI = s_s[I], cJ = s_c[J], sJ = s_s[J];
                    const T x00 = A[pI * LD + pJ], x01 = A[pI * LD + qJ];
                    const T x10 = A[qI * LD + pJ], x11 = A[qI * LD + qJ];
                    const T y00 = cI * x00 - sI * x10, y01 = cI * x01 - sI * x11;
                    const T y10 = sI * x00 + cI * x10, y11 = sI * x01 + cI * x11;
                    const T z00 = y00 * cJ - y01 * sJ, z01 = y00 * sJ + y01 * cJ;
                    const T z10 = y10 * cJ - y11 * sJ, z11 = y10 * sJ + y11 * cJ;
                    A[pI * LD + pJ] = z00; A[pI * LD + qJ] = z01;
                    A[qI * LD + pJ] = z10; A[qI * LD + qJ] = z11;
                    A[pJ * LD + pI] = z00; A[qJ * LD + pI] = z01;
                    A[pJ * LD + qI] = z10; A[qJ * LD + qI] = z11;
                }
            }
            // V <- V J
            for (int w = tid; w < N * H; w += nt) {
                const int i = w / H, J = w - (w / H) * H;
                const int pJ = s_p[J], qJ = s_q[J];
                const T c = s_c[J], sn = s_s[J];
                const T vp = V[i * LD + pJ], vq = V[i * LD + qJ];
                V[i * LD + pJ] = c * vp - sn * vq;
                V[i * LD + qJ] = sn * vp + c * vq;
            }
            __syncthreads();
        }
    }

    // ---- clip eigenvalues, rebuild the lower triangle of V diag(max(lambda,0)) V^T
    for (int i = tid; i < N; i += nt) {
        const T d = A[i * LD + i];
        dp[i] = d > T(0) ? d : T(0);
    }
    __syncthreads();

    double pv[3] = {0.0, 0.0, 0.0};
    for (int q = tid; q < s * s; q += nt) {
        const int ra = q % s, cb = q / s;
        if (ra < cb) continue;
        const T* Va = V + ra * LD;
        const T* Vb = V + cb * LD;
        T acc = T(0);
        for (int i = 0; i < N; ++i) acc += (Va[i] * dp[i]) * Vb[i];
        const double xv = ldexp((double)acc, e2);
        const int pos = packed_pos(ra, cb, s);
        if (MODE == PROJ_PRIMAL) {
            const double u = U[pos];
            const double l = a.lam[off + pos];
            const double d = xv - u;
            xk_new[off + pos] = xv;
            a.lam[off + pos] = l + a.rho * d;                  // Eq. LambdakUpdate
            const double wgt = (ra == cb) ? 1.0 : 2.0;
            pv[0] += wgt * d * d;
            pv[1] += wgt * xv * xv;
            pv[2] += wgt * u * u;
        } else {
            a.out[off + pos] = xv;
        }
    }
    if (MODE == PROJ_PRIMAL) {
        block_sum_t<double, 3>(pv, red_d);
        if (tid == 0) {
            a.part[blk * 4 + 0] = pv[0];
            a.part[blk * 4 + 1] = pv[1];
            a.part[blk * 4 + 2] = pv[2];
        }
    }
}

template <typename T, int MODE>
cudaError_t prepare_one() {
    const size_t smem =
        project_smem_bytes(SDP_MAX_CLIQUE, sizeof(T) == 4 ? SDP_PROJ_FP32 : SDP_PROJ_FP64, MODE);
    return cudaFuncSetAttribute(k_project<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
}

template <typename T, int MODE>
cudaError_t launch_one(const ProjArgs& a, int smax, cudaStream_t st) {
    const size_t smem = project_smem_bytes(smax, sizeof(T) == 4 ? SDP_PROJ_FP32 : SDP_PROJ_FP64, MODE);
    const double rinv = 1.0 / a.rho;
    k_project<T, MODE><<<a.count, project_threads(smax), smem, st>>>(a, rinv);
    return cudaGetLastError();
}

}  // namespace

size_t project_smem_bytes(int smax, int prec, int mode) {
    const int N = smax + (smax & 1);
    const int LD = N + 1;
    const size_t tsz = prec == SDP_PROJ_FP32 ? 4 : 8;
    size_t bytes = ((size_t)2 * N * LD + N) * tsz;
    bytes = (bytes + 15) & ~(size_t)15;
    if (mode == PROJ_PRIMAL) bytes += (size_t)N * (N + 1) / 2 * sizeof(double);
    return bytes;
}

int project_threads(int smax) {
    if (smax <= 16) return 64;
    if (smax <= 32) return 256;
    return 512;
}

cudaError_t project_prepare() {
    cudaError_t e;
    if ((e = prepare_one<float, PROJ_PLAIN>()) != cudaSuccess) return e;
    if ((e = prepare_one<float, PROJ_PRIMAL>()) != cudaSuccess) return e;
    if ((e = prepare_one<float, PROJ_DUAL>()) != cudaSuccess) return e;
    if ((e = prepare_one<double, PROJ_PLAIN>()) != cudaSuccess) return e;
    if ((e = prepare_one<double, PROJ_PRIMAL>()) != cudaSuccess) return e;
    return prepare_one<double, PROJ_DUAL>();
}

cudaError_t launch_project(const ProjArgs& a, int mode, int prec, int smax, cudaStream_t st) {
    if (a.count <= 0) return cudaSuccess;
    if (prec == SDP_PROJ_FP32) {
        if (mode == PROJ_PLAIN) return launch_one<float, PROJ_PLAIN>(a, smax, st);
        if (mode == PROJ_PRIMAL) return launch_one<float, PROJ_PRIMAL>(a, smax, st);
        return launch_one<float, PROJ_DUAL>(a, smax, st);
    }
    if (mode == PROJ_PLAIN) return launch_one<double, PROJ_PLAIN>(a, smax, st);
    if (mode == PROJ_PRIMAL) return launch_one<double, PROJ_PRIMAL>(a, smax, st);
    return launch_one<double, PROJ_DUAL>(a, smax, st);
}

}  // namespace cadmm
