// Reverse-mode kernels for T unrolled primal-form iterations (Algorithm 1) as functions of the cost
// c and the right-hand side b. The paper differentiates nothing; this is the transpose of each
// step of the iteration, run backwards:
//   lambda_k+ = lambda_k + rho (x_k+ - u_k), x_k+ = P(W_k), W_k = u_k - rho^-1 lambda_k,
//   u_k = H_k x, x = S r + D^-1 A^T M^-1 b, r = sum_k H_k^T (x_k + rho^-1 lambda_k) - rho^-1 c.
// Adjoints are held as gradients with respect to the full symmetric matrices, stored on their lower
// triangles (so every map keeps the form the forward kernels use); the ABI converts to gradients
// with respect to lower-triangle parameters (weight 2 off the diagonal) at its boundary.
//
// The derivative of P at W = V diag(lambda) V^T is the Daleckii-Krein formula
// V (Gamma o (V^T E V)) V^T, Gamma_ij = (f(l_i) - f(l_j)) / (l_i - l_j), f = max(., 0), and f' of the
// pair's mean where |l_i - l_j| <= 1e-12 max|l| (f'(0) = 0); it is self-adjoint. V comes from the
// forward FP64 eigensolve of the same iteration (recomputed from a checkpoint), lambda_i = v_i^T W v_i.
#include "sdp_internal.h"

namespace cadmm {

namespace {

__device__ __forceinline__ int packed_pos_a(int a, int b, int s) { return b * s - (b * (b - 1)) / 2 + (a - b); }

// W_k of iteration t from the affine iterate x of that iteration and the multipliers before it.
__global__ void k_form_w(IterPtrs P, const double* __restrict__ lam_prev, double rinv, double* __restrict__ W) {
    for (int pos = blockIdx.x * blockDim.x + threadIdx.x; pos < P.SL; pos += gridDim.x * blockDim.x)
        W[pos] = P.x[P.gather_idx[pos]] - rinv * lam_prev[pos];
}

__device__ __forceinline__ double dk_gamma(double li, double lj, double tiny) {
    const double d = li - lj;
    if (fabs(d) <= tiny) return 0.5 * (li + lj) > 0.0 ? 1.0 : 0.0;
    return (fmax(li, 0.0) - fmax(lj, 0.0)) / d;
}

// One warp segment of NR lanes per clique (N <= NR), lane c owning column c. For each clique:
// X~ = Xb + rho Lb, Wbar = DP(W)[X~], then ub = Wbar - rho Lb and Lb <- Lb - rho^-1 Wbar.
template <int NR>
struct VjpLayout {
    static constexpr int SEG = 32 / NR;
    static constexpr int BPC = 4 * SEG;
    static constexpr int LD = NR + 1;
    static constexpr int kDoubles = 3 * NR * LD + NR;     // W (then Q), X~, V tiles and lambda
    static constexpr size_t kBytes = (size_t)BPC * kDoubles * sizeof(double);
};

template <int NR>
__global__ void __launch_bounds__(128) k_dk_vjp(IterPtrs P, const int* __restrict__ order, int count,
                                                const double* __restrict__ W, const double* __restrict__ V,
                                                double* __restrict__ Xb, double* __restrict__ Lb,
                                                double* __restrict__ ub, double rho, double rinv) {
    using L = VjpLayout<NR>;
    constexpr int LD = L::LD;
    extern __shared__ __align__(16) double sm_vjp[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int seg = lane / NR, c = lane % NR;
    const int slot = warp * L::SEG + seg;
    const int idx = blockIdx.x * L::BPC + slot;
    double* Wt = sm_vjp + (size_t)slot * L::kDoubles;
    double* Xt = Wt + NR * LD;
    double* Vt = Xt + NR * LD;
    double* ls = Vt + NR * LD;
    double* Qt = Wt;                                    // W is dead once lambda is known
    int blk = -1, s = 0, N = 0;
    long long o = 0;
    if (idx < count) {
        blk = order[idx];
        s = P.blk_size[blk];
        N = s + (s & 1);
        o = P.blk_off[blk];
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        Wt[r * LD + c] = 0.0;
        Xt[r * LD + c] = 0.0;
    }
    __syncwarp();
    if (c < s)
        for (int r = c; r < s; ++r) {
            const int p = packed_pos_a(r, c, s);
            const double w = W[o + p], x = fma(rho, Lb[o + p], Xb[o + p]);
            Wt[r * LD + c] = w;
            Wt[c * LD + r] = w;
            Xt[r * LD + c] = x;
            Xt[c * LD + r] = x;
        }
    double v[NR];
    const double* Vb = V + (blk >= 0 ? P.voff[blk] : 0);
#pragma unroll
    for (int r = 0; r < NR; ++r) v[r] = (r < N && c < N) ? Vb[r * N + c] : 0.0;
#pragma unroll
    for (int r = 0; r < NR; ++r) Vt[r * LD + c] = v[r];
    __syncwarp();
    // lambda_c = v_c^T W v_c and z = X~ v_c
    double lam = 0.0, z[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        double t = 0.0, u = 0.0;
#pragma unroll
        for (int m = 0; m < NR; ++m) {
            t = fma(Wt[r * LD + m], v[m], t);
            u = fma(Xt[r * LD + m], v[m], u);
        }
        lam = fma(v[r], t, lam);
        z[r] = u;
    }
    ls[c] = lam;
    __syncwarp();
    double lmax = 0.0;
    for (int i = 0; i < N; ++i) lmax = fmax(lmax, fabs(ls[i]));
    const double tiny = 1e-12 * lmax;
    // column c of Gamma o (V^T X~ V), then column c of Q = V (Gamma o ...)
    double y[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        double t = 0.0;
#pragma unroll
        for (int r = 0; r < NR; ++r) t = fma(Vt[r * LD + i], z[r], t);
        y[i] = (i < N && c < N) ? t * dk_gamma(ls[i], lam, tiny) : 0.0;
    }
    __syncwarp();                                      // every lane is done with W before Q overwrites it
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        double t = 0.0;
#pragma unroll
        for (int i = 0; i < NR; ++i) t = fma(Vt[r * LD + i], y[i], t);
        Qt[r * LD + c] = t;
    }
    __syncwarp();
    // Wbar = Q V^T on the lower triangle, then the multiplier epilogue
    for (int cb = 0; cb < s; ++cb)
        for (int ra = cb + c; ra < s; ra += NR) {
            double t = 0.0;
            for (int i = 0; i < N; ++i) t = fma(Qt[ra * LD + i], Vt[cb * LD + i], t);
            const int p = packed_pos_a(ra, cb, s);
            const double l = Lb[o + p];
            ub[o + p] = t - rho * l;
            Lb[o + p] = l - rinv * t;
        }
}

// xbar = sum_k H_k^T ub (+ the loss gradient at the last iteration, converted from lower-parameter
// form by 1/w), and xbar w/D for the first pass over A.
__global__ void k_adj_scatter(IterPtrs P, const double* __restrict__ ub, const double* __restrict__ xbar_T,
                              double* __restrict__ xbar, double* __restrict__ rsw) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P.nEL; e += gridDim.x * blockDim.x) {
        const int j0 = P.sc_ptr[e], j1 = P.sc_ptr[e + 1];
        double acc = 0.0;
        for (int j = j0; j < j1; ++j) acc = (j == j0) ? ub[P.sc_pos[j]] : acc + ub[P.sc_pos[j]];
        if (xbar_T != nullptr) acc += xbar_T[e] * (P.ew[e] == 1 ? 1.0 : 0.5);
        xbar[e] = acc;
        rsw[e] = acc * P.wdinv[e];
    }
}

// cbar += -rho^-1 rbar, bbar += ybar, Xb = H_k rbar, Lb += rho^-1 H_k rbar.
__global__ void k_adj_accum(IterPtrs P, const double* __restrict__ rbar, const double* __restrict__ ybar,
                            double* __restrict__ cbar, double* __restrict__ bbar, double* __restrict__ Xb,
                            double* __restrict__ Lb, double rinv) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    for (int e = tid; e < P.nEL; e += nt) cbar[e] = fma(-rinv, rbar[e], cbar[e]);
    for (int i = tid; i < P.m; i += nt) bbar[i] += ybar[i];
    for (int pos = tid; pos < P.SL; pos += nt) {
        const double g = rbar[P.gather_idx[pos]];
        Xb[pos] = g;
        Lb[pos] = fma(rinv, g, Lb[pos]);
    }
}

// Lower-parameter gradients: c by its weight w, b as it is.
__global__ void k_adj_finish(IterPtrs P, const double* __restrict__ cbar, const double* __restrict__ bbar,
                             double* __restrict__ cout, double* __restrict__ bout) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    for (int e = tid; e < P.nEL; e += nt) cout[e] = (P.ew[e] == 1 ? 1.0 : 2.0) * cbar[e];
    for (int i = tid; i < P.m; i += nt) bout[i] = bbar[i];
}

__global__ void k_copy(const double* __restrict__ src, double* __restrict__ dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

inline int grid_for(long long n) { return (int)std::min<long long>(4096, std::max<long long>(1, (n + 255) / 256)); }

}  // namespace

cudaError_t adjoint_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_dk_vjp<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)VjpLayout<16>::kBytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_dk_vjp<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)VjpLayout<32>::kBytes);
}

cudaError_t launch_form_w(const IterPtrs& P, const double* lam_prev, double rinv, double* W, cudaStream_t st) {
    k_form_w<<<grid_for(P.SL), 256, 0, st>>>(P, lam_prev, rinv, W);
    return cudaGetLastError();
}

cudaError_t launch_dk_vjp(const IterPtrs& P, int n_large, const double* W, const double* V, double* Xb, double* Lb,
                          double* ub, double rho, cudaStream_t st) {
    const double rinv = 1.0 / rho;
    // P.order lists the cliques largest first: the first n_large have padded order 17..32.
    if (n_large > 0) {
        using L = VjpLayout<32>;
        k_dk_vjp<32><<<(n_large + L::BPC - 1) / L::BPC, 128, L::kBytes, st>>>(P, P.order, n_large, W, V, Xb, Lb, ub,
                                                                             rho, rinv);
    }
    const int rest = P.p - n_large;
    if (rest > 0) {
        using L = VjpLayout<16>;
        k_dk_vjp<16><<<(rest + L::BPC - 1) / L::BPC, 128, L::kBytes, st>>>(P, P.order + n_large, rest, W, V, Xb, Lb,
                                                                          ub, rho, rinv);
    }
    return cudaGetLastError();
}

cudaError_t launch_adj_scatter(const IterPtrs& P, const double* ub, const double* xbar_T, double* xbar, double* rsw,
                               cudaStream_t st) {
    k_adj_scatter<<<grid_for(P.nEL), 256, 0, st>>>(P, ub, xbar_T, xbar, rsw);
    return cudaGetLastError();
}

cudaError_t launch_adj_accum(const IterPtrs& P, const double* rbar, const double* ybar, double* cbar, double* bbar,
                             double* Xb, double* Lb, double rinv, cudaStream_t st) {
    k_adj_accum<<<grid_for(std::max<long long>(P.SL, P.nEL)), 256, 0, st>>>(P, rbar, ybar, cbar, bbar, Xb, Lb, rinv);
    return cudaGetLastError();
}

cudaError_t launch_adj_finish(const IterPtrs& P, const double* cbar, const double* bbar, double* cout, double* bout,
                              cudaStream_t st) {
    k_adj_finish<<<grid_for(P.nEL), 256, 0, st>>>(P, cbar, bbar, cout, bout);
    return cudaGetLastError();
}

cudaError_t launch_copy(const double* src, double* dst, long long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_copy<<<grid_for(n), 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

}  // namespace cadmm
