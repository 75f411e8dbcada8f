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

// Cone blocks (free, nonnegative, second-order; projected onto the cone itself in the primal
// form): the derivative of the projection is the identity (free), the mask of W > 0 (nonnegative),
// and for a second-order cone (t, u) with ||u|| > |t| the symmetric
// 1/2 [[1, uh^T], [uh, (1 + t/||u||) I - (t/||u||) uh uh^T]], uh = u / ||u|| (the identity inside
// the cone, zero inside its polar). Same epilogue as the cliques. One CTA per forward segment: a
// run of free or nonnegative positions, one large second-order cone, or up to 256 small ones (a
// thread each). Every position's X~ is read before its Lb is written.
__device__ __forceinline__ void cone_vjp_out(int pos, double wbar, double* Lb, double* ub, double rho, double rinv) {
    const double lb = Lb[pos];
    ub[pos] = wbar - rho * lb;
    Lb[pos] = lb - rinv * wbar;
}

__device__ __forceinline__ double soc_vjp_elem(bool first, double w, double g, double gt, double t, double nu,
                                               double dot) {
    if (nu <= t) return g;                      // inside the cone: identity
    if (nu <= -t) return 0.0;                   // inside the polar cone: zero
    if (first) return 0.5 * (gt + dot);
    const double r = t / nu, uh = w / nu;
    return 0.5 * gt * uh + 0.5 * ((1.0 + r) * g - r * dot * uh);
}

__global__ void __launch_bounds__(256) k_cone_vjp(IterPtrs P, const double* __restrict__ W,
                                                  const double* __restrict__ Xb, double* __restrict__ Lb,
                                                  double* __restrict__ ub, double rho, double rinv) {
    __shared__ double red[2][8];
    const int sg = blockIdx.x;
    const int lo = P.cone_lo[sg], hi = P.cone_hi[sg], kind = P.cone_kind[sg];
    if (kind == kConeSocSmall) {
        const int c = lo + (int)threadIdx.x;
        if (c >= hi) return;
        const int p0 = P.soc_pos[c], q = P.soc_q[c];
        const double t = W[p0], gt = Xb[p0] + rho * Lb[p0];
        double nn = 0.0, ug = 0.0;
        for (int j = 1; j < q; ++j) {
            const double u = W[p0 + j];
            nn = fma(u, u, nn);
            ug = fma(u, Xb[p0 + j] + rho * Lb[p0 + j], ug);
        }
        const double nu = sqrt(nn), dot = nu > 0.0 ? ug / nu : 0.0;
        cone_vjp_out(p0, soc_vjp_elem(true, t, gt, gt, t, nu, dot), Lb, ub, rho, rinv);
        for (int j = 1; j < q; ++j) {
            const double g = Xb[p0 + j] + rho * Lb[p0 + j];
            cone_vjp_out(p0 + j, soc_vjp_elem(false, W[p0 + j], g, gt, t, nu, dot), Lb, ub, rho, rinv);
        }
        return;
    }
    if (kind == kConeSoc) {
        // both sums over the cone in a fixed order: a strided partial per thread, then the warps'
        // shuffle trees and the warps in order
        double nn = 0.0, ug = 0.0;
        for (int pos = lo + 1 + (int)threadIdx.x; pos < hi; pos += blockDim.x) {
            const double u = W[pos];
            nn = fma(u, u, nn);
            ug = fma(u, Xb[pos] + rho * Lb[pos], ug);
        }
        for (int o = 16; o > 0; o >>= 1) {
            nn += __shfl_xor_sync(0xffffffffu, nn, o);
            ug += __shfl_xor_sync(0xffffffffu, ug, o);
        }
        if ((threadIdx.x & 31) == 0) {
            red[0][threadIdx.x >> 5] = nn;
            red[1][threadIdx.x >> 5] = ug;
        }
        __syncthreads();
        nn = 0.0;
        ug = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            nn += red[0][w];
            ug += red[1][w];
        }
        const double t = W[lo], gt = Xb[lo] + rho * Lb[lo];
        const double nu = sqrt(nn), dot = nu > 0.0 ? ug / nu : 0.0;
        __syncthreads();                        // every thread has read X~ at lo before it changes
        for (int pos = lo + (int)threadIdx.x; pos < hi; pos += blockDim.x) {
            const double g = Xb[pos] + rho * Lb[pos];
            cone_vjp_out(pos, soc_vjp_elem(pos == lo, W[pos], g, gt, t, nu, dot), Lb, ub, rho, rinv);
        }
        return;
    }
    for (int pos = lo + (int)threadIdx.x; pos < hi; pos += blockDim.x) {
        const double g = Xb[pos] + rho * Lb[pos];
        cone_vjp_out(pos, kind == kConeFree ? g : (W[pos] > 0.0 ? g : 0.0), Lb, ub, rho, rinv);
    }
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
    if (P.ncs > 0) k_cone_vjp<<<P.ncs, 256, 0, st>>>(P, W, Xb, Lb, ub, rho, rinv);
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
