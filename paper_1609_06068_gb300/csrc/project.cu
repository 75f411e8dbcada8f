// Batched projection of small symmetric clique blocks onto the PSD cone (Eqs. XkUpdate, zkUpdate):
// P(W) = V diag(max(lambda, 0)) V^T, with the eigendecomposition by two-sided cyclic Jacobi.
//
// One CTA owns one clique block (order s, padded to even N; a padded row/column is zero and never
// rotates). A sweep visits every index pair once in the round-robin ("circle") order: N/2 disjoint
// pairs per round, N-1 rounds. The matrix is kept in SLOT order: row/column i of the stored matrix
// belongs to the index that currently occupies slot i, round r pairs slot j with slot H+j, and
// after each round every index moves one step along a fixed ring (slot 0 stays). Because pairs sit
// at fixed slots, each thread owns fixed 2x2 tiles of A (rows of pair I, columns of pair J, I <= J)
// and fixed entries of V in registers, and every shared-memory address it touches is computed once.
// A round is: the owner of diagonal tile (I, I) computes the rotation that zeroes a_pq (Golub &
// Van Loan, symmetric Schur 2x2) and publishes (c, s); barrier; every thread applies J^T A J to its
// tiles and J to its V entries, and writes them to their next-round slots; barrier; every thread
// reloads its tiles. Sweeps stop once the off-diagonal Frobenius norm is below tol * ||W||_F.
// Eigenvector order does not matter for P(W), so the slot permutation never has to be undone.
//
// Warm start (handle path): the eigenvectors of the previous ADMM iteration's block are kept in
// HBM; the kernel forms V^T W V with them and starts Jacobi from that nearly diagonal matrix, which
// usually needs one or two sweeps. Every kWarmPeriod-th iteration starts cold from V = I so that
// rounding in V cannot accumulate. The result does not depend on the start (P is unique).
//
// W is formed in FP64 and scaled by the power of two 2^-e that brings max|W_ij| into [1, 2), then
// rounded to the projection precision T; the rebuilt lower triangle is widened and unscaled (both
// scalings are exact).
#include <algorithm>

#include "sdp_internal.h"

namespace cadmm {

namespace {

template <typename T> struct JacobiParams;
// FP32 stops at off(A) <= 1e-7 ||W||_F, about the FP32 rounding of the rebuild; the projection
// moves by at most the dropped off-diagonal part (P is 1-Lipschitz). A looser 1e-6 moved the
// converged ADMM objectives by ~1e-4 relative on the n = 1020 block-arrow workload.
template <> struct JacobiParams<float> {
    static constexpr float rel_tol = 1.0e-7f;
    static constexpr int max_sweeps = 24;
};
template <> struct JacobiParams<double> {
    static constexpr double rel_tol = 1.0e-15;
    static constexpr int max_sweeps = 30;
};

constexpr int kMaxPairs = SDP_MAX_CLIQUE / 2;
constexpr int kWarmPeriod = 8;

// Threads per CTA and register slots per thread for A tiles (KA) and V entry pairs (KV), by the
// padded order N: KA * NT >= H(H+1)/2 and KV * NT >= N*H with H = N/2.
template <int NT_, int KA_, int KV_> struct Shape {
    static constexpr int NT = NT_, KA = KA_, KV = KV_;
};
using ShapeS16 = Shape<64, 1, 2>;    // N <= 16
using ShapeS32 = Shape<256, 1, 2>;   // N <= 32
using ShapeS64 = Shape<512, 2, 4>;   // N <= 64
using ShapeS96 = Shape<512, 3, 9>;   // N <= 96

__device__ __forceinline__ int packed_pos(int a, int b, int s) {
    return b * s - (b * (b - 1)) / 2 + (a - b);  // column-major lower, a >= b
}

// Slot that the index now in slot i occupies next round: slot 0 stays; the top row 1..H-1 moves
// right, the bottom row H..N-1 moves left, and the two rows are joined into one ring.
__device__ __forceinline__ int ring_next(int i, int H, int N) {
    if (N == 2 || i == 0) return i;
    if (i < H - 1) return i + 1;
    if (i == H - 1) return N - 1;
    if (i > H) return i - 1;
    return 1;
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

// ---- Jacobi rotation that zeroes a_pq:
//   tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1+t^2),
//   s = t c; afterwards a_pp -= t a_pq, a_qq += t a_pq, a_pq = 0.
// The block is scaled so max|w| lies in [1, 2); off-diagonal entries below 1e-30 count as zero.
// FP32: the angle only has to be right to a few ulp (the residual it leaves in a_pq is of FP32
// rounding size, and later rotations remove it), so tau and t use the hardware reciprocal and
// sqrt(x) = x rsqrt(x). c = 1/sqrt(1 + t^2) is correctly rounded: c^2 + s^2 = 1 to half an ulp
// keeps V orthogonal over the thousands of rotations a warm-started block goes through (a few-ulp
// c let V drift by ~1e-5 and moved the converged ADMM objective by ~1e-4).
__device__ __forceinline__ void rotation(float app, float aqq, float apq, float& c, float& s, float& t) {
    if (fabsf(apq) < 1.0e-30f) { c = 1.f; s = 0.f; t = 0.f; return; }
    const float tau = __fdividef(aqq - app, 2.f * apq);
    const float at = fabsf(tau);
    float den;
    if (at > 1.0e15f) {
        den = 2.f * at;
    } else {
        const float x = fmaf(tau, tau, 1.f);
        den = at + x * rsqrtf(x);
    }
    t = copysignf(__fdividef(1.f, den), tau);
    c = __frsqrt_rn(fmaf(t, t, 1.f));
    s = t * c;
}

// FP64: GB300's FP64 divide and square root are long dependent chains on a narrow pipe, so the
// reciprocal and the reciprocal square root start from FP32 estimates (2^-23) and take two
// Newton steps each (error below 2^-52 before rounding).
__device__ __forceinline__ double rcp_nr(double x) {
    double r = (double)__frcp_rn((float)x);
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}
__device__ __forceinline__ double rsqrt_nr(double x) {   // x in [1, 2^60]
    double y = (double)__frsqrt_rn((float)x);
    const double h = 0.5 * x;
    y = y * fma(-h * y, y, 1.5);
    y = y * fma(-h * y, y, 1.5);
    return y;
}
__device__ __forceinline__ void rotation(double app, double aqq, double apq, double& c, double& s, double& t) {
    if (fabs(apq) < 1.0e-30) { c = 1.0; s = 0.0; t = 0.0; return; }
    const double tau = (aqq - app) * rcp_nr(2.0 * apq);
    const double at = fabs(tau);
    double den;
    if (at > 1.0e8) {
        den = 2.0 * at;                                   // sqrt(1 + tau^2) = |tau| to FP64 precision
    } else {
        const double x = fma(tau, tau, 1.0);
        den = at + x * rsqrt_nr(x);
    }
    t = copysign(rcp_nr(den), tau);
    c = rsqrt_nr(fma(t, t, 1.0));
    s = t * c;
}

// W_ij of one packed position: the block itself (standalone), H_k x - rho^-1 lambda_k (primal,
// Eq. XkUpdate) or v_k - rho^-1 lambda_k (dual, Eq. zkUpdate).
template <int MODE>
__device__ __forceinline__ double load_w(const ProjArgs& a, long long off, int pos, double rinv) {
    if (MODE == PROJ_PLAIN) return a.in[off + pos];
    // one FP64 instruction (an FP64 instruction issues at one warp instruction per 64 clocks per
    // SM partition on GB300), and one rounding instead of two
    if (MODE == PROJ_PRIMAL) return fma(-rinv, a.lam[off + pos], a.x[a.gather_idx[off + pos]]);
    return fma(-rinv, a.lam[off + pos], a.v[off + pos]);
}

// Scaling of a block by an exact power of two, 2^-e2 before the eigensolve and 2^e2 after, with
// e2 = ilogb(max |W_ij|) clamped to [-1000, 1000] so that both factors are normal doubles built
// from their exponent bits (on GB300 ldexp per element is a sequence of FP64 operations, the
// multiplication is one, and rounds the same). A block beyond that range is scaled by 2^-+1000:
// above, its FP32 values stay finite; below, its entries are under 2^-1000 and so is the error.
__device__ __forceinline__ int block_exponent(double wmax) {
    const int e = (wmax > 0.0 && isfinite(wmax)) ? ilogb(wmax) : 0;
    return e < -1000 ? -1000 : (e > 1000 ? 1000 : e);
}
__device__ __forceinline__ double pow2_exact(int k) {       // 2^k for |k| <= 1000, from its exponent bits
    return __longlong_as_double((long long)(1023 + k) << 52);
}

// x 2^-e2 rounded to FP32 (to nearest, ties to even), from the bits, with no FP64 instruction
// (on GB300 an FP64 instruction, conversions included, takes a warp 64 clocks per SM partition):
// the scaling only moves the exponent, and the rounding takes the top 24 of the 53 significand
// bits. Values that land below FP32's normal range (under 2^-126 after scaling, while the block's
// largest entry lands in [1, 2)) become zero; an infinity or a NaN stays one (unscaled).
__device__ __forceinline__ float scaled_to_float(double x, int e2) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(b >> 63) << 31;
    const int ex = (int)((b >> 52) & 0x7ff);
    const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
    const int fe = ex - e2 - 896;                        // FP32 biased exponent after scaling
    unsigned bits = sign | ((unsigned)min(max(fe, 0), 255) << 23) | (unsigned)(mant >> 29);
    const unsigned rem = (unsigned)(mant & 0x1FFFFFFFull);
    bits += (rem > 0x10000000u || (rem == 0x10000000u && (bits & 1u))) ? 1u : 0u;
    const unsigned special = sign | 0x7F800000u | (mant != 0ull ? 0x00400000u : 0u);   // inf, NaN
    bits = ex == 0x7ff ? special : (ex == 0 || fe <= 0) ? sign : bits;
    return __uint_as_float(bits);
}
// (double)f 2^e2 from the bits, with no FP64 instruction: exact for normal results; a zero or
// FP32-subnormal f (under 2^-126 of the block's scale) gives zero, an infinity or a NaN stays one,
// and a result outside the normal FP64 range becomes zero or an infinity.
__device__ __forceinline__ double float_scaled_to_double(float f, int e2) {
    const unsigned u = __float_as_uint(f);
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    const int fe = (int)((u >> 23) & 0xff);
    const unsigned long long mant = (unsigned long long)(u & 0x7FFFFFu) << 29;
    const int de = fe - 127 + 1023 + e2;
    unsigned long long bits = sign | ((unsigned long long)min(max(de, 0), 0x7ff) << 52) | mant;
    bits = (fe == 0 || de <= 0) ? sign
         : (fe == 0xff) ? (sign | 0x7FF0000000000000ull | mant)
         : (de >= 0x7ff) ? (sign | 0x7FF0000000000000ull) : bits;
    return __longlong_as_double((long long)bits);
}

// Batches: true when clique blk belongs to a problem that has stopped, so the CTA must return.
// In the primal form the iteration right after the stop copies the block's current x_k to the
// other ping-pong buffer first, so both hold it for every later parity.
// The threads t0, t0 + stride, ... share the copy.
template <int MODE>
__device__ __forceinline__ bool block_stopped(const ProjArgs& a, int blk, int s, long long off, int t0, int stride) {
    if (a.inst_conv == nullptr) return false;
    const int cv = a.inst_conv[a.blk_inst[blk]];
    if (cv < 0) return false;
    if (MODE == PROJ_PRIMAL && cv == a.ctrl->iter) {
        const int it = a.ctrl->iter;
        const double* cur = (it & 1) ? a.xk[1] : a.xk[0];
        double* nxt = (it & 1) ? a.xk[0] : a.xk[1];
        const int len = s * (s + 1) / 2;
        for (int q = t0; q < len; q += stride) nxt[off + q] = cur[off + q];
    }
    return true;
}
template <int MODE>
__device__ __forceinline__ bool block_stopped(const ProjArgs& a, int blk, int s, long long off) {
    return block_stopped<MODE>(a, blk, s, off, threadIdx.x, blockDim.x);
}

template <typename T, int MODE, class SH>
__global__ void __launch_bounds__(SH::NT) k_project(ProjArgs a, double rinv) {
    constexpr int KA = SH::KA, KV = SH::KV;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T s_c[kMaxPairs], s_s[kMaxPairs];
    __shared__ T red_t[33 * 2];
    __shared__ double red_d[33 * 4];

    pdl_wait();
    const int blk = a.order ? a.order[blockIdx.x] : a.first + (int)blockIdx.x;   // read alongside the flag
    if (a.ctrl != nullptr && a.ctrl->done) return;

    const int s = a.size[blk];
    const long long off = a.off[blk];
    if (block_stopped<MODE>(a, blk, s, off)) return;
    const int N = s + (s & 1);
    const int H = N / 2;
    const int LD = N + 1;
    const int tid = threadIdx.x;
    const int NT = SH::NT;
    const bool warm = a.vstore != nullptr && a.ctrl != nullptr && (a.ctrl->iter % kWarmPeriod) != 0;

    T* Ax = reinterpret_cast<T*>(smem_raw);   // exchange buffer for A (slot order)
    T* Vx = Ax + N * LD;                      // exchange buffer for V (rows: coordinates, cols: slots)
    T* Wb = Vx + N * LD;                      // W (warm start input / product scratch)
    T* dp = Wb + N * LD;                      // clipped eigenvalues by slot

    // ---- load W (scaled by 2^-e2) into Wb (warm) or Ax (cold), both triangles, zero padding
    double wmax = 0.0;
    for (int q = tid; q < s * s; q += NT) {
        const int ra = q % s, cb = q / s;
        if (ra < cb) continue;
        wmax = fmax(wmax, fabs(load_w<MODE>(a, off, packed_pos(ra, cb, s), rinv)));
    }
    wmax = block_max(wmax, red_d);
    const int e2 = block_exponent(wmax);
    const double down = pow2_exact(-e2), up = pow2_exact(e2);
    T* Wt = warm ? Wb : Ax;
    for (int q = tid; q < N * N; q += NT) {
        const int i = q / N, j = q - (q / N) * N;
        if (i >= s || j >= s) Wt[i * LD + j] = T(0);
    }
    for (int q = tid; q < s * s; q += NT) {
        const int ra = q % s, cb = q / s;
        if (ra < cb) continue;
        const T wt = (T)((load_w<MODE>(a, off, packed_pos(ra, cb, s), rinv)) * down);
        Wt[ra * LD + cb] = wt;
        Wt[cb * LD + ra] = wt;
    }
    // ---- V: identity (cold) or the previous eigenvectors (warm)
    T* vglob = nullptr;
    if (a.vstore != nullptr) vglob = reinterpret_cast<T*>(a.vstore) + a.voff[blk];
    for (int q = tid; q < N * N; q += NT) {
        const int i = q / N, j = q - (q / N) * N;
        Vx[i * LD + j] = warm ? vglob[q] : (i == j ? T(1) : T(0));
    }
    __syncthreads();
    if (warm) {
        // Ax = W V, then Wb = V^T Ax: the block in the basis of the previous eigenvectors.
        for (int q = tid; q < N * N; q += NT) {
            const int i = q / N, j = q - (q / N) * N;
            T acc = T(0);
            for (int k = 0; k < N; ++k) acc = fma(Wb[i * LD + k], Vx[k * LD + j], acc);
            Ax[i * LD + j] = acc;
        }
        __syncthreads();
        for (int q = tid; q < N * N; q += NT) {
            const int i = q / N, j = q - (q / N) * N;
            if (j < i) continue;
            T acc = T(0);
            for (int k = 0; k < N; ++k) acc = fma(Vx[k * LD + i], Ax[k * LD + j], acc);
            Wb[i * LD + j] = acc;
            Wb[j * LD + i] = acc;
        }
        __syncthreads();
    }
    const T* A0 = warm ? Wb : Ax;

    // ---- per-thread ownership: tiles (I, J), I <= J, and V entry pairs (row r, pair J)
    const int ntiles = H * (H + 1) / 2;
    int tI[KA], tJ[KA];
    int src[KA][4], dst[KA][4], mir[KA][4];
    T x[KA][4];
#pragma unroll
    for (int t = 0; t < KA; ++t) {
        int w = tid + t * NT, I = 0;
        tI[t] = -1;
        tJ[t] = -1;
        if (w < ntiles) {
            while (w >= H - I) { w -= H - I; ++I; }
            tI[t] = I;
            tJ[t] = I + w;
        }
        const int I0 = tI[t] < 0 ? 0 : tI[t], J0 = tJ[t] < 0 ? 0 : tJ[t];
        const int r0 = I0, r1 = H + I0, c0 = J0, c1 = H + J0;
        src[t][0] = r0 * LD + c0; src[t][1] = r0 * LD + c1;
        src[t][2] = r1 * LD + c0; src[t][3] = r1 * LD + c1;
        const int nr0 = ring_next(r0, H, N), nr1 = ring_next(r1, H, N);
        const int nc0 = ring_next(c0, H, N), nc1 = ring_next(c1, H, N);
        dst[t][0] = nr0 * LD + nc0; dst[t][1] = nr0 * LD + nc1;
        dst[t][2] = nr1 * LD + nc0; dst[t][3] = nr1 * LD + nc1;
        mir[t][0] = nc0 * LD + nr0; mir[t][1] = nc1 * LD + nr0;
        mir[t][2] = nc0 * LD + nr1; mir[t][3] = nc1 * LD + nr1;
#pragma unroll
        for (int e = 0; e < 4; ++e) x[t][e] = tI[t] >= 0 ? A0[src[t][e]] : T(0);
    }
    int vJ[KV], vsrc[KV][2], vdst[KV][2];
    T v[KV][2];
#pragma unroll
    for (int u = 0; u < KV; ++u) {
        const int w = tid + u * NT;
        vJ[u] = w < N * H ? w % H : -1;
        const int r = w < N * H ? w / H : 0, J = vJ[u] < 0 ? 0 : vJ[u];
        vsrc[u][0] = r * LD + J;
        vsrc[u][1] = r * LD + H + J;
        vdst[u][0] = r * LD + ring_next(J, H, N);
        vdst[u][1] = r * LD + ring_next(H + J, H, N);
        v[u][0] = vJ[u] >= 0 ? Vx[vsrc[u][0]] : T(0);
        v[u][1] = vJ[u] >= 0 ? Vx[vsrc[u][1]] : T(0);
    }

    // ---- ||W||_F^2 and the stopping threshold
    T nrm[1] = {T(0)};
#pragma unroll
    for (int t = 0; t < KA; ++t) {
        if (tI[t] < 0) continue;
        const T q2 = x[t][0] * x[t][0] + x[t][1] * x[t][1] + x[t][2] * x[t][2] + x[t][3] * x[t][3];
        nrm[0] += tI[t] == tJ[t] ? q2 : T(2) * q2;
    }
    block_sum_t<T, 1>(nrm, red_t);
    const T tol2 = JacobiParams<T>::rel_tol * JacobiParams<T>::rel_tol * nrm[0];

    // ---- cyclic Jacobi sweeps
    int sweeps = 0;
    for (int sweep = 0; sweep < JacobiParams<T>::max_sweeps; ++sweep) {
        T off2[1] = {T(0)};
#pragma unroll
        for (int t = 0; t < KA; ++t) {
            if (tI[t] < 0) continue;
            if (tI[t] == tJ[t]) off2[0] += x[t][1] * x[t][1] + x[t][2] * x[t][2];
            else off2[0] += T(2) * (x[t][0] * x[t][0] + x[t][1] * x[t][1] + x[t][2] * x[t][2] + x[t][3] * x[t][3]);
        }
        block_sum_t<T, 1>(off2, red_t);
        if (!(off2[0] > tol2)) break;
        ++sweeps;
        for (int r = 0; r < N - 1; ++r) {
#pragma unroll
            for (int t = 0; t < KA; ++t) {
                if (tI[t] >= 0 && tI[t] == tJ[t]) {
                    T c, sn, tt;
                    rotation(x[t][0], x[t][3], x[t][1], c, sn, tt);
                    s_c[tI[t]] = c;
                    s_s[tI[t]] = sn;
                    // J^T X J applied exactly (no a_pq := 0): an angle that is a few ulp off leaves
                    // a residual of that size in a_pq, which later rotations remove, instead of
                    // silently dropping it from the spectrum.
                    const T a00 = x[t][0], a01 = x[t][1], a11 = x[t][3];
                    const T y00 = c * a00 - sn * a01, y01 = c * a01 - sn * a11;
                    const T y10 = sn * a00 + c * a01, y11 = sn * a01 + c * a11;
                    x[t][0] = y00 * c - y01 * sn;
                    x[t][1] = y00 * sn + y01 * c;
                    x[t][2] = x[t][1];
                    x[t][3] = y10 * sn + y11 * c;
                }
            }
            __syncthreads();
#pragma unroll
            for (int t = 0; t < KA; ++t) {
                if (tI[t] < 0) continue;
                if (tI[t] != tJ[t]) {
                    const T cI = s_c[tI[t]], sI = s_s[tI[t]], cJ = s_c[tJ[t]], sJ = s_s[tJ[t]];
                    const T y00 = cI * x[t][0] - sI * x[t][2], y01 = cI * x[t][1] - sI * x[t][3];
                    const T y10 = sI * x[t][0] + cI * x[t][2], y11 = sI * x[t][1] + cI * x[t][3];
                    x[t][0] = y00 * cJ - y01 * sJ;
                    x[t][1] = y00 * sJ + y01 * cJ;
                    x[t][2] = y10 * cJ - y11 * sJ;
                    x[t][3] = y10 * sJ + y11 * cJ;
                }
                // the tile and its mirror move to the slots their indices occupy next round
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    Ax[dst[t][e]] = x[t][e];
                    Ax[mir[t][e]] = x[t][e];
                }
            }
#pragma unroll
            for (int u = 0; u < KV; ++u) {
                if (vJ[u] < 0) continue;
                const T c = s_c[vJ[u]], sn = s_s[vJ[u]];
                const T p0 = v[u][0], p1 = v[u][1];
                Vx[vdst[u][0]] = c * p0 - sn * p1;
                Vx[vdst[u][1]] = sn * p0 + c * p1;
            }
            __syncthreads();
#pragma unroll
            for (int t = 0; t < KA; ++t)
                if (tI[t] >= 0) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) x[t][e] = Ax[src[t][e]];
                }
#pragma unroll
            for (int u = 0; u < KV; ++u)
                if (vJ[u] >= 0) {
                    v[u][0] = Vx[vsrc[u][0]];
                    v[u][1] = Vx[vsrc[u][1]];
                }
        }
    }

    // ---- eigenvalues (diagonal of A, by slot), clipped; V is current in Vx
#pragma unroll
    for (int t = 0; t < KA; ++t)
        if (tI[t] >= 0 && tI[t] == tJ[t]) {
            dp[tI[t]] = x[t][0] > T(0) ? x[t][0] : T(0);
            dp[H + tI[t]] = x[t][3] > T(0) ? x[t][3] : T(0);
        }
    __syncthreads();
    if (vglob != nullptr)
        for (int q = tid; q < N * N; q += NT) vglob[q] = Vx[(q / N) * LD + (q % N)];

    // ---- rebuild the lower triangle of V diag(max(lambda, 0)) V^T and apply the epilogue
    pdl_trigger();
    double pv[3] = {0.0, 0.0, 0.0};
    double* xk_new = nullptr;
    if (MODE == PROJ_PRIMAL) xk_new = (a.ctrl->iter & 1) ? a.xk[0] : a.xk[1];
    for (int q = tid; q < s * s; q += NT) {
        const int ra = q % s, cb = q / s;
        if (ra < cb) continue;
        const T* Va = Vx + ra * LD;
        const T* Vb = Vx + cb * LD;
        T acc = T(0);
        for (int i = 0; i < N; ++i) acc = fma(Va[i] * dp[i], Vb[i], acc);
        const double xv = ((double)acc) * up;
        const int pos = packed_pos(ra, cb, s);
        if (MODE == PROJ_PRIMAL) {
            const double u = a.x[a.gather_idx[off + pos]];
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
    if (a.part != nullptr && tid == 0) a.part[blk * 4 + 3] = (double)sweeps;   // Jacobi sweeps used
}

// ---------------------------------------------------------------------------------------------
// FP32, padded order N <= 32 * CPL (CPL = 1, 2): one-sided (Hestenes) Jacobi, one CTA of 4 * CPL
// warps per clique. Larger blocks and FP64 use the two-sided kernel above.
//
// Lane j holds columns j, j + 32, ... (CPL of them) of G = B V, with B = W + sigma I and
// sigma = 2 ||W||_F, so B is positive definite and its eigenvalues are lambda(W) + sigma >= ||W||_F
// (for an indefinite W, one-sided Jacobi alone would confuse eigenvalues +mu and -mu). Warp w
// holds rows 8w .. 8w+7 of every column, in registers. A rotation of columns (i, j) makes g_i and
// g_j orthogonal (Golub & Van Loan's 2x2 formula on the Gram entries alpha = g_i.g_i,
// beta = g_j.g_j, gamma = g_i.g_j): the partner column's rows arrive by warp shuffles, the warps'
// partial gammas meet in shared memory (one barrier per round), and both ends of a pair compute
// the same rotation from the same sums. Rounds follow the round-robin schedule, so a sweep of N-1
// rounds meets every pair once. After a sweep whose largest |gamma| / sqrt(alpha beta) was below
// kOneSidedStop when it began, the columns of G are mu_j v_j: V itself is never formed, v_j =
// g_j / mu_j and lambda_j = mu_j - sigma with mu_j = ||g_j||. Warm start: G = B V_prev from the
// eigenvectors kept from the last call (recomputed from G each time, so rounding does not build up).
constexpr int kOSRows = 8;                 // rows per warp
// Cyclic Jacobi converges quadratically: a sweep that starts with every pair within
// kOneSidedStop of orthogonal leaves them within about its square divided by the relative gap of
// the shifted spectrum, which the shift 2 ||W||_F makes small for clustered eigenvalues. With
// 1e-4 the projection error stays below 1e-4 ||W|| (cold starts on 20 x 20 blocks with four
// 5-fold clusters reached 7.5e-5; 3e-4 left 1e-4 on such a block). (Looser thresholds were faster
// on the n = 1020 workload: 11.4k / 11.7k / 12.0k iterations per second at 1e-4 / 3e-4 / 1e-3.)
constexpr float kOneSidedStop = 1.0e-4f;
constexpr int kOneSidedMaxSweeps = 20;

// Round-robin partner of player i in round rd for N players (N even, n = N - 1 odd): player n
// meets player rd; every other i meets (2 rd - i) mod n, or player n when that is i itself.
__host__ __device__ constexpr int rr_partner(int i, int rd, int N) {
    if (i >= N) return i;
    const int n = N - 1;
    if (i == n) return rd;
    int j = (2 * rd - i) % n;
    if (j < 0) j += n;
    return j == i ? n : j;
}

// Partner tables of the CTA one-sided kernels, [round][player] for every even order N (32 x 32 for
// N <= 32, 64 x 64 up to 64), evaluated by the compiler: computing them in every CTA (a modulo by
// N - 1 per entry) cost about 1.5 us per projection; a CTA now copies its table with one or two
// 8-byte loads per thread.
struct PartnerTables {
    unsigned char t32[16][32 * 32];
    unsigned char t64[32][64 * 64];
};
constexpr PartnerTables make_partner_tables() {
    PartnerTables p{};
    for (int t = 0; t < 16; ++t)
        for (int q = 0; q < 32 * 32; ++q) p.t32[t][q] = (unsigned char)rr_partner(q & 31, q >> 5, 2 * (t + 1));
    for (int t = 0; t < 32; ++t)
        for (int q = 0; q < 64 * 64; ++q) p.t64[t][q] = (unsigned char)rr_partner(q & 63, q >> 6, 2 * (t + 1));
    return p;
}
__device__ __align__(16) const PartnerTables g_partner = make_partner_tables();

template <int CPL>
struct OSLayout {
    static constexpr int NP = 32 * CPL;          // players (columns) and rows
    static constexpr int NW = 4 * CPL;           // warps
    static constexpr int LD = NP + 1;
    // dynamic shared memory: W, V (floats), then the partner table (bytes)
    static constexpr size_t kMatBytes = (size_t)2 * NP * LD * sizeof(float);
    static constexpr size_t kBytes = kMatBytes + (size_t)NP * NP;
};

template <int MODE, int CPL>
__global__ void __launch_bounds__(32 * 4 * CPL, CPL == 1 ? 4 : 2) k_project_os(ProjArgs a, double rinv) {
    using L = OSLayout<CPL>;
    constexpr int NP = L::NP, NW = L::NW, LD = L::LD;
    extern __shared__ __align__(16) unsigned char smem_os[];
    float* Ws = reinterpret_cast<float*>(smem_os);           // W, then V for the rebuild
    float* Vs = Ws + NP * LD;                                // previous eigenvectors (warm start)
    unsigned char* s_partner = smem_os + L::kMatBytes;       // [round][player]
    __shared__ float s_gam[2][NW][NP];                       // partial gamma per warp, by parity
    __shared__ float s_red[NW][NP];
    __shared__ float dp[NP];
    __shared__ double red_d[33 * 3];
    __shared__ float red_f[33 * 2];

    pdl_wait();
    const int blk = a.order ? a.order[blockIdx.x] : a.first + (int)blockIdx.x;   // read alongside the flag
    if (a.ctrl != nullptr && a.ctrl->done) return;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int NT = 32 * NW;
    const int s = a.size[blk];
    const long long off = a.off[blk];
    if (block_stopped<MODE>(a, blk, s, off)) return;
    const int N = s + (s & 1);
    const int r0 = w * kOSRows;
    // Warm start whenever eigenvectors are kept (they are the identity right after a reset).
    const bool warm = a.vstore != nullptr && a.ctrl != nullptr;
    float* vglob = a.vstore != nullptr ? reinterpret_cast<float*>(a.vstore) + a.voff[blk] : nullptr;
    {
        const unsigned char* gp = CPL == 1 ? g_partner.t32[N / 2 - 1] : g_partner.t64[N / 2 - 1];
        for (int q = 8 * tid; q < NP * NP; q += 8 * NT)
            *reinterpret_cast<uint2*>(s_partner + q) = *reinterpret_cast<const uint2*>(gp + q);
    }

    // ---- W scaled by 2^-e2 into Ws (both triangles), zero outside s x s. Each thread reads its
    // entries once, all loads in flight, and keeps them until the scale is known.
    constexpr int KQ = NP * NP / (32 * NW);
    double wv[KQ];
    float vp[KQ];          // the previous eigenvectors, loaded alongside W
    double wmax = 0.0;
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
        const int q = tid + k * NT;
        const int ra = q % s, cb = q / s;
        wv[k] = (q < s * s && ra >= cb) ? load_w<MODE>(a, off, packed_pos(ra, cb, s), rinv) : 0.0;
        const int i = q / NP, j = q % NP;
        vp[k] = !warm ? 0.f : (i < N && j < N) ? vglob[i * N + j] : (i == j ? 1.f : 0.f);
    }
#pragma unroll
    for (int k = 0; k < KQ; ++k) wmax = fmax(wmax, fabs(wv[k]));
    wmax = block_max(wmax, red_d);
    const int e2 = block_exponent(wmax);
    const double down = pow2_exact(-e2), up = pow2_exact(e2);
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
        const int q = tid + k * NT;
        const int i = q / NP, j = q % NP;
        if (i >= s || j >= s) Ws[i * LD + j] = 0.f;
        if (warm) Vs[i * LD + j] = vp[k];
    }
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
        const int q = tid + k * NT;
        const int ra = q % s, cb = q / s;
        if (q < s * s && ra >= cb) {
            const float wt = (float)((wv[k]) * down);
            Ws[ra * LD + cb] = wt;
            Ws[cb * LD + ra] = wt;
        }
    }
    __syncthreads();

    // ---- shift sigma = 2 ||W||_F and the initial columns: G = B (cold) or B V_prev (warm)
    float sq[1] = {0.f};
#pragma unroll
    for (int h = 0; h < CPL; ++h)
#pragma unroll
        for (int k = 0; k < kOSRows; ++k) {
            const float wv = Ws[(r0 + k) * LD + lane + 32 * h];
            sq[0] = fmaf(wv, wv, sq[0]);
        }
    block_sum_t<float, 1>(sq, red_f);
    const float sigma = 2.f * sqrtf(sq[0]);
    float g[CPL][kOSRows];
    if (warm) {
        // G = B V_prev, summed over m in order for every entry; each V_prev entry is read once per
        // lane and each W entry once per warp (a broadcast)
#pragma unroll
        for (int h = 0; h < CPL; ++h)
#pragma unroll
            for (int k = 0; k < kOSRows; ++k) g[h][k] = sigma * Vs[(r0 + k) * LD + lane + 32 * h];
#pragma unroll 4
        for (int m = 0; m < NP; ++m) {
            float vm[CPL];
#pragma unroll
            for (int h = 0; h < CPL; ++h) vm[h] = Vs[m * LD + lane + 32 * h];
#pragma unroll
            for (int k = 0; k < kOSRows; ++k) {
                const float wrm = Ws[(r0 + k) * LD + m];
#pragma unroll
                for (int h = 0; h < CPL; ++h) g[h][k] = fmaf(wrm, vm[h], g[h][k]);
            }
        }
    } else {
#pragma unroll
        for (int h = 0; h < CPL; ++h)
#pragma unroll
            for (int k = 0; k < kOSRows; ++k) {
                const int r = r0 + k, c = lane + 32 * h;
                g[h][k] = Ws[r * LD + c] + ((r == c && c < N) ? sigma : 0.f);
            }
    }
#pragma unroll
    for (int h = 0; h < CPL; ++h)
        if (lane + 32 * h >= N) {
#pragma unroll
            for (int k = 0; k < kOSRows; ++k) g[h][k] = 0.f;
        }

    // ---- sweeps
    int sweeps = 0;
    for (int sweep = 0; sweep < kOneSidedMaxSweeps; ++sweep) {
#pragma unroll
        for (int h = 0; h < CPL; ++h) {
            float pa = 0.f;
#pragma unroll
            for (int k = 0; k < kOSRows; ++k) pa = fmaf(g[h][k], g[h][k], pa);
            s_red[w][lane + 32 * h] = pa;
        }
        __syncthreads();
        float alpha[CPL];
#pragma unroll
        for (int h = 0; h < CPL; ++h) {
            float acc = 0.f;
            for (int ww = 0; ww < NW; ++ww) acc += s_red[ww][lane + 32 * h];
            alpha[h] = acc;
        }
        float worst = 0.f;
        for (int rd = 0; rd < N - 1; ++rd) {
            int p[CPL];
            float gp[CPL][kOSRows];
            float beta[CPL];
            const int buf = rd & 1;
#pragma unroll
            for (int h = 0; h < CPL; ++h) {
                p[h] = s_partner[rd * NP + lane + 32 * h];
                const int pl = p[h] & 31, ph = p[h] >> 5;
                // the partner's alpha (lane p & 31 holds it in slot p >> 5), fetched before the
                // barrier so that it is off the round's critical path
                beta[h] = 0.f;
#pragma unroll
                for (int hs = 0; hs < CPL; ++hs) {
                    const float t = __shfl_sync(0xffffffffu, alpha[hs], pl);
                    if (hs == ph) beta[h] = t;
                }
                float pg = 0.f;
#pragma unroll
                for (int k = 0; k < kOSRows; ++k) {
                    float val = 0.f;
#pragma unroll
                    for (int hs = 0; hs < CPL; ++hs) {
                        const float t = __shfl_sync(0xffffffffu, g[hs][k], pl);
                        if (hs == ph) val = t;
                    }
                    gp[h][k] = val;
                    pg = fmaf(g[h][k], val, pg);
                }
                s_gam[buf][w][lane + 32 * h] = pg;
            }
            __syncthreads();
            float c[CPL], sg[CPL], tt[CPL], gam[CPL];
            bool first[CPL];
            float ai[CPL], aj[CPL];
#pragma unroll
            for (int h = 0; h < CPL; ++h) {
                float gsum = 0.f;
                for (int ww = 0; ww < NW; ++ww) gsum += s_gam[buf][ww][lane + 32 * h];
                gam[h] = gsum;
                const int me = lane + 32 * h;
                first[h] = me < p[h];
                ai[h] = first[h] ? alpha[h] : beta[h];
                aj[h] = first[h] ? beta[h] : alpha[h];
                float cc = 1.f, sn = 0.f, t = 0.f;
                if (p[h] != me && fabsf(gsum) > 1.0e-30f) {
                    worst = fmaxf(worst, __fdividef(gsum * gsum, fmaxf(ai[h] * aj[h], 1.0e-30f)));
                    const float zeta = __fdividef(aj[h] - ai[h], 2.f * gsum);
                    const float az = fabsf(zeta);
                    float den;
                    if (az > 1.0e15f) {
                        den = 2.f * az;
                    } else {
                        const float x = fmaf(zeta, zeta, 1.f);
                        den = az + x * rsqrtf(x);
                    }
                    t = copysignf(__fdividef(1.f, den), zeta);
                    cc = __frsqrt_rn(fmaf(t, t, 1.f));
                    sn = t * cc;
                }
                c[h] = cc;
                tt[h] = t;
                sg[h] = first[h] ? -sn : sn;     // g_i' = c g_i - s g_j (i), g_j' = s g_i + c g_j (j)
            }
#pragma unroll
            for (int h = 0; h < CPL; ++h) {
#pragma unroll
                for (int k = 0; k < kOSRows; ++k) g[h][k] = fmaf(sg[h], gp[h][k], c[h] * g[h][k]);
            }
#pragma unroll
            for (int h = 0; h < CPL; ++h)
                alpha[h] = first[h] ? ai[h] - tt[h] * gam[h] : aj[h] + tt[h] * gam[h];
        }
        ++sweeps;
        float wr = worst;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wr = fmaxf(wr, __shfl_xor_sync(0xffffffffu, wr, o));
        if (lane == 0) s_red[w][0] = wr;
        __syncthreads();
        float wmx = 0.f;
        for (int ww = 0; ww < NW; ++ww) wmx = fmaxf(wmx, s_red[ww][0]);
        __syncthreads();
        if (wmx < kOneSidedStop * kOneSidedStop) break;
    }

    // ---- mu_j = ||g_j||, lambda_j = mu_j - sigma clipped, v_j = g_j / mu_j into Ws (and HBM)
#pragma unroll
    for (int h = 0; h < CPL; ++h) {
        float pr = 0.f;
#pragma unroll
        for (int k = 0; k < kOSRows; ++k) pr = fmaf(g[h][k], g[h][k], pr);
        s_red[w][lane + 32 * h] = pr;
    }
    __syncthreads();
    for (int c = tid; c < NP; c += NT) {
        float acc = 0.f;
        for (int ww = 0; ww < NW; ++ww) acc += s_red[ww][c];
        const float mu = sqrtf(acc);
        const float lam = mu - sigma;
        dp[c] = (c < N && lam > 0.f) ? lam : 0.f;
        s_gam[0][0][c] = mu > 0.f ? 1.f / mu : 0.f;
    }
    __syncthreads();
    // V into Ws, and V diag(max(lambda, 0)) into Vs (the warm-start buffer is free now)
#pragma unroll
    for (int h = 0; h < CPL; ++h) {
        const int c = lane + 32 * h;
        const float inv = s_gam[0][0][c];
        const float dc = dp[c];
#pragma unroll
        for (int k = 0; k < kOSRows; ++k) {
            const int r = r0 + k;
            const float v = inv > 0.f ? g[h][k] * inv : (r == c ? 1.f : 0.f);
            Ws[r * LD + c] = v;
            Vs[r * LD + c] = v * dc;
            if (vglob != nullptr && c < N && r < N) vglob[r * N + c] = v;
        }
    }
    __syncthreads();

    // ---- rebuild the lower triangle of V diag(max(lambda, 0)) V^T and apply the epilogue
    pdl_trigger();
    double pv[3] = {0.0, 0.0, 0.0};
    double* xk_new = nullptr;
    if (MODE == PROJ_PRIMAL) xk_new = (a.ctrl->iter & 1) ? a.xk[0] : a.xk[1];
    // warp w takes columns w, w + NW, ...; lane j row cb + j (+ 32 h): no division, and the FP64
    // results of a column go out as consecutive stores
    for (int cb = w; cb < s; cb += NW)
#pragma unroll
    for (int h = 0; h < CPL; ++h) {
        const int ra = cb + lane + 32 * h;
        if (ra >= s) continue;
        const float* Va = Vs + ra * LD;
        const float* Wb = Ws + cb * LD;
        float acc = 0.f;
        for (int i = 0; i < N; ++i) acc = fmaf(Va[i], Wb[i], acc);
        const double xv = ((double)acc) * up;
        const int pos = packed_pos(ra, cb, s);
        if (MODE == PROJ_PRIMAL) {
            const double u = a.x[a.gather_idx[off + pos]];
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
    if (a.part != nullptr && tid == 0) a.part[blk * 4 + 3] = (double)sweeps;
}

// ---------------------------------------------------------------------------------------------
// FP32, padded order N <= 32, one CTA of four warps per clique, for launches with few cliques
// (fewer than the GPU holds warps), where a projection's time is the length of its dependent
// chain rather than its operation count. The whole CTA loads W, forms G = B V_prev, runs the
// Jacobi sweeps and rebuilds the projection. In the sweeps lane c of every warp holds column c of
// G, warp w its rows 8w .. 8w + 7, in registers: a round is 8 shuffles and 8 multiply-adds of a
// partial Gram entry per warp, one barrier to add the four partials, the 2x2 rotation and an
// 8-row column update (with all 32 rows in one warp, the 32 shuffles of a round were most of its
// time).
//
// The method is k_project_ow's (one-sided Jacobi on G = B V, B = W + sigma I, sigma = 2 ||W||_F,
// V never formed: v_j = g_j / mu_j, lambda_j = mu_j - sigma with mu_j = ||g_j||), with three
// changes on the round's critical path:
//   - the partner of round rd is updated incrementally (no division, no table lookup);
//   - the rotation takes r = sqrt(d^2 + 4 gamma^2) once, t = sign(d) 2 gamma / (|d| + r) with
//     d = alpha_j - alpha_i, which is the same t as the textbook sign(zeta) / (|zeta| + sqrt(1 +
//     zeta^2)), zeta = d / (2 gamma), with one reciprocal fewer; c = 1/sqrt(1 + t^2) from the
//     hardware estimate and one Newton-Raphson step (error about one ulp, as for a correctly
//     rounded one);
//   - a pair whose columns are already orthogonal to kWSSkip (relative) is not rotated, and a
//     round in which no pair rotates skips the column update altogether. A pair left at relative
//     Gram entry e moves P(W) by about e ||W||_F, and up to N^2/2 pairs add up in quadrature, so
//     kWSSkip = 1e-7 (about FP32 rounding of a 32-term dot product) keeps their sum near 4e-6
//     ||W||_F at order 64;
//   - each column carries a scale factor that takes the rotations' cosines, so a row of the
//     update is one FMA (fast Givens style); the factors are folded back at every sweep start;
//   - small rotations (|zeta| <= 2^-7, the usual case once a warm start is close) take the series
//     of jacobi_rot, with 2 / (alpha_j - alpha_i) formed while the Gram entry is still being
//     summed; a round whose rotations are all small has no square root or division on its chain.
// The sweeps stop after one in which every pair started within kOneSidedStop of orthogonal, as in
// the other one-sided kernels. (Stopping at any round once the last N - 1 rounds met no pair
// beyond it, instead of at sweep ends, saved under a microsecond per launch here but cost ADMM
// iterations with the order-64 kernel on workload 3: 660 against 588 to 1e-4.)
// The rotation that makes two columns of G orthogonal, for the one-sided kernels: from
// d = alpha_j - alpha_i, gamma and zeta = 2 gamma / d, the tangent t = zeta / (1 + sqrt(1 +
// zeta^2)) (= sign(d) 2 gamma / (|d| + sqrt(d^2 + 4 gamma^2)), Golub & Van Loan's smaller root),
// c = 1 / sqrt(1 + t^2) and 1/c. For |zeta| <= kSmallAngle (series = true) they come from their
// series, t = (zeta/2)(1 - zeta^2/4), c = 1 - t^2/2, 1/c = 1 + t^2/2 (truncation below 1e-9
// relative), with no division or root on the chain after gamma; otherwise from the closed forms
// (c from the hardware reciprocal square root and one Newton-Raphson step, about one ulp).
// need_full is warp-uniform: whether any lane of the warp takes the closed forms. Both ends of a
// pair see the same gamma, d and zeta, so they choose the same way and compute the same rotation.
constexpr float kSmallAngle = 0.0078125f;
struct JRot {
    float t, c, ic;
};
__device__ __forceinline__ JRot jacobi_rot(float gam, float d, float z, bool series, bool need_full) {
    JRot q;
    q.t = (0.5f * z) * fmaf(-0.25f * z, z, 1.f);
    const float t2 = q.t * q.t;
    q.c = fmaf(-0.5f, t2, 1.f);
    q.ic = fmaf(0.5f, t2, 1.f);
    if (need_full) {
        const float gg = 2.f * gam;
        const float x = fmaf(d, d, gg * gg);
        const float rr = x * rsqrtf(x);
        float t = __fdividef(gg, fabsf(d) + rr);
        t = d < 0.f ? -t : t;
        const float u = fmaf(t, t, 1.f);
        float cc = rsqrtf(u);
        cc = fmaf(0.5f * cc, fmaf(-u * cc, cc, 1.f), cc);    // Newton-Raphson step
        if (!series) {
            q.t = t;
            q.c = cc;
            q.ic = u * cc;                                   // sqrt(1 + t^2)
        }
    }
    return q;
}

constexpr int kWSLD = 36;                 // row stride (floats): 16-byte rows for float4 access
constexpr float kWSSkip = 1.0e-7f;

template <int MODE>
__global__ void __launch_bounds__(128) k_project_ws(ProjArgs a, double rinv) {
    constexpr int LD = kWSLD;
    __shared__ __align__(16) float Ws[32 * LD];   // W (scaled), later Q = V diag(lambda+)^(1/2)
    __shared__ __align__(16) float Vs[32 * LD];   // previous eigenvectors (warm start)
    __shared__ float s_gp[2][4 * 32];              // a round's partial Gram entries, by round parity
    __shared__ float s_cn[4][32];                  // partial column norms
    __shared__ int s_exp[4];
    __shared__ float s_sq[4];
    __shared__ double red_d[33 * 3];

    pdl_wait();
    const int blk = a.order ? a.order[blockIdx.x] : a.first + (int)blockIdx.x;
    // the block's descriptor is read alongside the stop flag (one round trip to memory, not two)
    const int s = a.size[blk];
    const long long off = a.off[blk];
    const long long voff = a.vstore != nullptr ? a.voff[blk] : 0;
    if (a.ctrl != nullptr && a.ctrl->done) return;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    if (block_stopped<MODE>(a, blk, s, off)) return;
    const int N = s + (s & 1);
    const bool warm = a.vstore != nullptr && a.ctrl != nullptr;
    float* vglob = a.vstore != nullptr ? reinterpret_cast<float*>(a.vstore) + voff : nullptr;

    // ---- W: warp w reads columns w, w + 4, ... of the packed lower triangle, lane j row cb + j
    // (each column a contiguous run), all loads in flight. The block's scale comes from the
    // largest exponent field, taken with integer operations.
    double wv[8];
    int emax = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int cb = w + 4 * k, ra = cb + lane;
        wv[k] = (cb < s && ra < s) ? load_w<MODE>(a, off, packed_pos(ra, cb, s), rinv) : 0.0;
    }
    float vp[8];           // previous eigenvectors: warp w rows w, w + 4, ..., lane j column j
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int r = w + 4 * k;
        vp[k] = !warm ? 0.f : (r < N && lane < N) ? vglob[r * N + lane] : (r == lane ? 1.f : 0.f);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int ex = (__double2hiint(wv[k]) >> 20) & 0x7ff;
        emax = ex > emax ? ex : emax;
    }
    emax = __reduce_max_sync(0xffffffffu, emax);
    if (lane == 0) s_exp[w] = emax;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int r = w + 4 * k;
        if (warm) Vs[r * LD + lane] = vp[k];
        // zero the padding of W: rows and columns s .. 31
        const int cb = w + 4 * k;
        if (cb >= s || lane >= s) { Ws[lane * LD + cb] = 0.f; Ws[cb * LD + lane] = 0.f; }
    }
    __syncthreads();
    emax = max(max(s_exp[0], s_exp[1]), max(s_exp[2], s_exp[3]));
    // ilogb of max |W_ij| from the biased exponent, clamped to [-1000, 1000] as in block_exponent
    // (a block whose entries are all zero or subnormal is scaled by 2^1000; a block holding an
    // infinity or a NaN goes through unscaled and shows as such in the residuals)
    const int e2 = emax == 0 ? -1000 : emax == 0x7ff ? 0 : min(max(emax - 1023, -1000), 1000);
    float sq = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int cb = w + 4 * k, ra = cb + lane;
        if (cb < s && ra < s) {
            const float wt = scaled_to_float(wv[k], e2);
            Ws[ra * LD + cb] = wt;
            Ws[cb * LD + ra] = wt;
            sq = fmaf(ra == cb ? wt : 2.f * wt, wt, sq);
        }
    }
    sq = warp_sum_t(sq);
    if (lane == 0) s_sq[w] = sq;
    __syncthreads();
    const float sigma = 2.f * sqrtf((s_sq[0] + s_sq[1]) + (s_sq[2] + s_sq[3]));

    // ---- G = B V_prev (warm) by all four warps, warp w rows 8w .. 8w + 7, lane j column j; the
    // rows stay in the warp's registers for the sweeps
    const int r0 = 8 * w;
    float g[8];
    if (warm) {
#pragma unroll
        for (int k = 0; k < 8; ++k) g[k] = sigma * Vs[(r0 + k) * LD + lane];
#pragma unroll 2
        for (int m = 0; m < 32; m += 4) {
            const float v0 = Vs[m * LD + lane], v1 = Vs[(m + 1) * LD + lane];
            const float v2 = Vs[(m + 2) * LD + lane], v3 = Vs[(m + 3) * LD + lane];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float4 wr = *reinterpret_cast<const float4*>(Ws + (r0 + k) * LD + m);
                g[k] = fmaf(wr.x, v0, g[k]);
                g[k] = fmaf(wr.y, v1, g[k]);
                g[k] = fmaf(wr.z, v2, g[k]);
                g[k] = fmaf(wr.w, v3, g[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) g[k] = lane < N ? g[k] : 0.f;
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) g[k] = lane < N ? Ws[(r0 + k) * LD + lane] + ((r0 + k == lane) ? sigma : 0.f) : 0.f;
    }

    // ---- sweeps by all four warps, lane c = column c, warp w its rows 8w .. 8w + 7. A round's
    // Gram entry is the sum of the four warps' partial sums, exchanged through shared memory with
    // one barrier (double-buffered by round parity) and added in the same order in every warp, so
    // all warps hold the same alpha, gamma, rotation and kap and take the same branches. The
    // column is kept as kap * gh: a rotation scales both columns of its pair by c, which goes into
    // kap, so the rows take one FMA each (gh' = gh -+ t (kap_partner / kap) gh_partner); every
    // sweep starts from kap = 1.
    int sweeps = 0;
    const int c = lane;
    {
        const int n = N - 1;                      // rounds per sweep (odd)
        float kap = 1.f, kinv = 1.f;
        for (int sweep = 0; sweep < kOneSidedMaxSweeps; ++sweep) {
            float ap = 0.f;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                g[k] *= kap;
                ap = fmaf(g[k], g[k], ap);
            }
            s_cn[w][c] = ap;
            __syncthreads();
            float alpha = (s_cn[0][c] + s_cn[1][c]) + (s_cn[2][c] + s_cn[3][c]);   // ||g_c||^2
            kap = 1.f;
            kinv = 1.f;
            bool big = false;                     // some pair started this sweep beyond the stop
            // round-robin partner: player n meets player rd; player i < n meets (2 rd - i) mod n,
            // or player n when that is i itself. j tracks (2 rd - c) mod n.
            int j = (c == 0 || c >= n) ? 0 : n - c;
            for (int rd = 0; rd < n; ++rd) {
                const int p = c >= N ? c : (c == n ? rd : (j == c ? n : j));
                j += 2;
                if (j >= n) j -= n;
                float gp[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) gp[k] = __shfl_sync(0xffffffffu, g[k], p);
                const float beta = __shfl_sync(0xffffffffu, alpha, p);
                const float kp = __shfl_sync(0xffffffffu, kap, p);
                const bool first = c < p;
                const float d = first ? beta - alpha : alpha - beta;   // alpha_j - alpha_i
                const float two_over_d = __fdividef(2.f, d);           // ready before gamma is
                float ga0 = 0.f, ga1 = 0.f;
#pragma unroll
                for (int k = 0; k < 8; k += 2) {
                    ga0 = fmaf(g[k], gp[k], ga0);
                    ga1 = fmaf(g[k + 1], gp[k + 1], ga1);
                }
                float* pr = s_gp[rd & 1];
                pr[w * 32 + c] = ga0 + ga1;
                __syncthreads();
                // both ends form the same product (kap * kp in the same order at both ends)
                const float kk = first ? kap * kp : kp * kap;
                const float gam = ((pr[c] + pr[32 + c]) + (pr[64 + c] + pr[96 + c])) * kk;
                const float g2 = gam * gam, ab = alpha * beta;
                const bool rot = p != c && g2 > (kWSSkip * kWSSkip) * ab;
                big |= p != c && g2 > (kOneSidedStop * kOneSidedStop) * ab;
                const float z = gam * two_over_d;                      // zeta
                const bool series = fabsf(z) <= kSmallAngle;
                if (!__any_sync(0xffffffffu, rot)) continue;
                const JRot q = jacobi_rot(gam, d, z, series, __any_sync(0xffffffffu, rot && !series));
                const float t = q.t;
                // g_i' = c g_i - s g_j (i), g_j' = s g_i + c g_j (j), with s = t c
                const float f = rot ? (first ? -t : t) * (kp * kinv) : 0.f;
#pragma unroll
                for (int k = 0; k < 8; ++k) g[k] = fmaf(f, gp[k], g[k]);
                if (rot) {
                    kap *= q.c;
                    kinv *= q.ic;
                    alpha = first ? alpha - t * gam : alpha + t * gam;
                }
            }
            ++sweeps;
            // the same in every warp (their alpha, gamma and big are equal)
            if (!__any_sync(0xffffffffu, big)) break;
        }
        // lambda_j = mu_j - sigma, v_j = g_j / mu_j; Q = V diag(max(lambda, 0))^(1/2) into Ws
        float mp = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            g[k] *= kap;
            mp = fmaf(g[k], g[k], mp);
        }
        s_cn[w][c] = mp;              // the last read of s_cn was before this sweep's barriers
        __syncthreads();
        const float mu2 = (s_cn[0][c] + s_cn[1][c]) + (s_cn[2][c] + s_cn[3][c]);
        const float mu = sqrtf(mu2);
        const float inv = mu > 0.f ? 1.f / mu : 0.f;
        const float lam = mu - sigma;
        const float qs = (c < N && lam > 0.f) ? sqrtf(lam) * inv : 0.f;
        if (vglob != nullptr && c < N) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int r = r0 + k;
                if (r < N) vglob[r * N + c] = mu > 0.f ? g[k] * inv : (r == c ? 1.f : 0.f);
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) Ws[(r0 + k) * LD + c] = g[k] * qs;
    }
    __syncthreads();

    // ---- rebuild the lower triangle of Q Q^T: warp w columns w, w + 4, ..., lane j row cb + j
    pdl_trigger();
    double pv[3] = {0.0, 0.0, 0.0};
    double* xk_new = nullptr;
    if (MODE == PROJ_PRIMAL) xk_new = (a.ctrl->iter & 1) ? a.xk[0] : a.xk[1];
    for (int cb = w; cb < s; cb += 4) {
        const int ra = cb + lane;
        if (ra >= s) continue;
        const float4* Qa = reinterpret_cast<const float4*>(Ws + ra * LD);
        const float4* Qb = reinterpret_cast<const float4*>(Ws + cb * LD);
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float4 qa = Qa[i], qb = Qb[i];
            acc[0] = fmaf(qa.x, qb.x, acc[0]);
            acc[1] = fmaf(qa.y, qb.y, acc[1]);
            acc[2] = fmaf(qa.z, qb.z, acc[2]);
            acc[3] = fmaf(qa.w, qb.w, acc[3]);
        }
        const double xv = float_scaled_to_double((acc[0] + acc[1]) + (acc[2] + acc[3]), e2);
        const int pos = packed_pos(ra, cb, s);
        if (MODE == PROJ_PRIMAL) {
            const double u = a.x[a.gather_idx[off + pos]];
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
    if (a.part != nullptr && w == 0 && lane == 0) a.part[blk * 4 + 3] = (double)sweeps;
}

// ---------------------------------------------------------------------------------------------
// FP32, padded order N <= 64, one CTA of four warps per clique: k_project_ws's method and layout
// with two columns per lane (lane c holds columns c and 32 + c, warp w rows 16w .. 16w + 15 of
// each). The sweep takes the 64 columns as two blocks of 32 and visits every pair once in 63
// rounds of disjoint pairs: 31 rounds within the blocks (the round-robin of 32 players in both
// blocks at once, so column c and column 32 + c meet partners held by the same lane) and 32
// rounds across them (column c with 32 + ((c + b) mod 32), b = 0 .. 31). Either way a lane's two
// partner columns come from one lane or two by one shuffle per row each, and the partial Gram
// entries of the four warps meet in shared memory, one barrier per round, added in the same
// order in every warp (so all warps take the same rotations and branches). Stops as
// k_project_ws does: after a sweep in which every pair started within kOneSidedStop.
constexpr int kWS64LD = 68;               // row stride (floats): 16-byte rows for float4 access

template <int MODE>
__global__ void __launch_bounds__(128) k_project_ws64(ProjArgs a, double rinv) {
    constexpr int LD = kWS64LD;
    __shared__ __align__(16) float Ws[64 * LD];   // W (scaled) (first FP64 scratch), later Q
    __shared__ __align__(16) float Vs[64 * LD];   // FP64 scratch for W, then previous eigenvectors
    __shared__ float s_gp[2][4 * 64];              // a round's partial Gram entries, by round parity
    __shared__ float s_cn[4][64];                  // partial column norms
    __shared__ int s_exp[4];
    __shared__ float s_sq[4];
    __shared__ double red_d[33 * 3];

    pdl_wait();
    const int blk = a.order ? a.order[blockIdx.x] : a.first + (int)blockIdx.x;
    const int s = a.size[blk];
    const long long off = a.off[blk];
    const long long voff = a.vstore != nullptr ? a.voff[blk] : 0;
    if (a.ctrl != nullptr && a.ctrl->done) return;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    if (block_stopped<MODE>(a, blk, s, off)) return;
    const int N = s + (s & 1);
    const bool warm = a.vstore != nullptr && a.ctrl != nullptr;
    float* vglob = a.vstore != nullptr ? reinterpret_cast<float*>(a.vstore) + voff : nullptr;

    // ---- W: the packed entries dealt to the 128 threads in turn, formed once (one FMA) into
    // FP64 scratch, the block's exponent from the bits; the tile is zeroed meanwhile
    const int len = s * (s + 1) / 2;
    double* wsc = reinterpret_cast<double*>(Vs);  // 64 x 68 floats hold the 2080 doubles of s = 64
    int emax = 0;
    for (int q = tid; q < len; q += 128) {
        const double wv = load_w<MODE>(a, off, q, rinv);
        wsc[q] = wv;
        emax = max(emax, (__double2hiint(wv) >> 20) & 0x7ff);
    }
    for (int q = tid; q < 64 * LD; q += 128) Ws[q] = 0.f;
    emax = __reduce_max_sync(0xffffffffu, emax);
    if (lane == 0) s_exp[w] = emax;
    __syncthreads();
    emax = max(max(s_exp[0], s_exp[1]), max(s_exp[2], s_exp[3]));
    // ilogb of max |W_ij| from the biased exponent, clamped to [-1000, 1000] as in block_exponent
    const int e2 = emax == 0 ? -1000 : emax == 0x7ff ? 0 : min(max(emax - 1023, -1000), 1000);
    float sq = 0.f;
    {
        int col = 0, cend = s;                        // entry q lies in column col, which ends at cend
        for (int q = tid; q < len; q += 128) {
            while (q >= cend) {
                ++col;
                cend += s - col;
            }
            const int r = col + (q - (cend - (s - col)));
            const float wt = scaled_to_float(wsc[q], e2);
            Ws[r * LD + col] = wt;
            Ws[col * LD + r] = wt;
            sq = fmaf(r == col ? wt : 2.f * wt, wt, sq);
        }
    }
    sq = warp_sum_t(sq);
    if (lane == 0) s_sq[w] = sq;
    __syncthreads();                              // W is in the tile; the scratch is free
    const float sigma = 2.f * sqrtf((s_sq[0] + s_sq[1]) + (s_sq[2] + s_sq[3]));
    if (warm)
        for (int q = tid; q < 64 * 64; q += 128) {
            const int r = q >> 6, cc = q & 63;
            Vs[r * LD + cc] = (r < N && cc < N) ? vglob[r * N + cc] : (r == cc ? 1.f : 0.f);
        }
    __syncthreads();

    // ---- G = B V_prev (warm) or B (cold): warp w rows 16w .. 16w + 15, lane c columns c, 32 + c
    const int r0 = 16 * w;
    float g[2][16];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int cc = lane + 32 * h;
        if (warm) {
#pragma unroll
            for (int k = 0; k < 16; ++k) g[h][k] = sigma * Vs[(r0 + k) * LD + cc];
            for (int m = 0; m < 64; m += 4) {
                const float v0 = Vs[m * LD + cc], v1 = Vs[(m + 1) * LD + cc];
                const float v2 = Vs[(m + 2) * LD + cc], v3 = Vs[(m + 3) * LD + cc];
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const float4 wr = *reinterpret_cast<const float4*>(Ws + (r0 + k) * LD + m);
                    g[h][k] = fmaf(wr.x, v0, g[h][k]);
                    g[h][k] = fmaf(wr.y, v1, g[h][k]);
                    g[h][k] = fmaf(wr.z, v2, g[h][k]);
                    g[h][k] = fmaf(wr.w, v3, g[h][k]);
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < 16; ++k) g[h][k] = Ws[(r0 + k) * LD + cc] + ((r0 + k == cc) ? sigma : 0.f);
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) g[h][k] = cc < N ? g[h][k] : 0.f;
    }

    // ---- sweeps (kap: the columns' scale factors, as in k_project_ws)
    int sweeps = 0;
    float kap[2] = {1.f, 1.f}, kinv[2] = {1.f, 1.f};
    {
        constexpr int n = 63;                     // rounds per sweep: 31 within the blocks, 32 across
        for (int sweep = 0; sweep < kOneSidedMaxSweeps; ++sweep) {
            bool bigs = false;                    // some pair started this sweep beyond the stop
            float ap[2] = {0.f, 0.f};
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    g[h][k] *= kap[h];
                    ap[h] = fmaf(g[h][k], g[h][k], ap[h]);
                }
            s_cn[w][lane] = ap[0];
            s_cn[w][lane + 32] = ap[1];
            __syncthreads();
            float alpha[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int cc = lane + 32 * h;
                alpha[h] = (s_cn[0][cc] + s_cn[1][cc]) + (s_cn[2][cc] + s_cn[3][cc]);
                kap[h] = 1.f;
                kinv[h] = 1.f;
            }
            int j = lane == 0 ? 0 : 31 - lane;    // within-block round-robin: (2 rd - lane) mod 31
            for (int rd = 0; rd < n; ++rd) {
                // partners: lane src[h] holds the partner of column lane + 32 h, in slot ps[h]
                int src0, src1, ps0, ps1;
                if (rd < 31) {
                    const int pl = lane == 31 ? rd : (j == lane ? 31 : j);
                    j += 2;
                    if (j >= 31) j -= 31;
                    src0 = src1 = pl;
                    ps0 = 0;
                    ps1 = 1;
                } else {
                    const int b = rd - 31;
                    src0 = (lane + b) & 31;
                    ps0 = 1;
                    src1 = (lane - b) & 31;
                    ps1 = 0;
                }
                const int p0 = src0 + 32 * ps0, p1 = src1 + 32 * ps1;   // partner columns
                // the partners' slots are the same for the whole warp in a round: slot h within the
                // blocks, the other slot across them (one shuffle per row and column)
                float gp[2][16], beta[2], kp[2];
                if (rd < 31) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        gp[0][k] = __shfl_sync(0xffffffffu, g[0][k], src0);
                        gp[1][k] = __shfl_sync(0xffffffffu, g[1][k], src1);
                    }
                    beta[0] = __shfl_sync(0xffffffffu, alpha[0], src0);
                    beta[1] = __shfl_sync(0xffffffffu, alpha[1], src1);
                    kp[0] = __shfl_sync(0xffffffffu, kap[0], src0);
                    kp[1] = __shfl_sync(0xffffffffu, kap[1], src1);
                } else {
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        gp[0][k] = __shfl_sync(0xffffffffu, g[1][k], src0);
                        gp[1][k] = __shfl_sync(0xffffffffu, g[0][k], src1);
                    }
                    beta[0] = __shfl_sync(0xffffffffu, alpha[1], src0);
                    beta[1] = __shfl_sync(0xffffffffu, alpha[0], src1);
                    kp[0] = __shfl_sync(0xffffffffu, kap[1], src0);
                    kp[1] = __shfl_sync(0xffffffffu, kap[0], src1);
                }
                float* pr = s_gp[rd & 1];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float ga0 = 0.f, ga1 = 0.f;
#pragma unroll
                    for (int k = 0; k < 16; k += 2) {
                        ga0 = fmaf(g[h][k], gp[h][k], ga0);
                        ga1 = fmaf(g[h][k + 1], gp[h][k + 1], ga1);
                    }
                    pr[w * 64 + lane + 32 * h] = ga0 + ga1;
                }
                __syncthreads();
                bool rot[2], big[2], series[2];
                float gam[2], d[2], z[2];
                bool first[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int cc = lane + 32 * h;
                    const int pc = h ? p1 : p0;
                    first[h] = cc < pc;
                    d[h] = first[h] ? beta[h] - alpha[h] : alpha[h] - beta[h];   // alpha_j - alpha_i
                    const float kk = first[h] ? kap[h] * kp[h] : kp[h] * kap[h];
                    gam[h] = ((pr[cc] + pr[64 + cc]) + (pr[128 + cc] + pr[192 + cc])) * kk;
                    const float g2 = gam[h] * gam[h], ab = alpha[h] * beta[h];
                    rot[h] = pc != cc && g2 > (kWSSkip * kWSSkip) * ab;
                    big[h] = pc != cc && g2 > (kOneSidedStop * kOneSidedStop) * ab;
                    z[h] = gam[h] * __fdividef(2.f, d[h]);                   // zeta
                    series[h] = fabsf(z[h]) <= kSmallAngle;
                }
                bigs |= big[0] || big[1];
                if (!__any_sync(0xffffffffu, rot[0] || rot[1])) continue;
                const bool need_full = __any_sync(0xffffffffu, (rot[0] && !series[0]) || (rot[1] && !series[1]));
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const JRot q = jacobi_rot(gam[h], d[h], z[h], series[h], need_full);
                    const float f = rot[h] ? (first[h] ? -q.t : q.t) * (kp[h] * kinv[h]) : 0.f;
#pragma unroll
                    for (int k = 0; k < 16; ++k) g[h][k] = fmaf(f, gp[h][k], g[h][k]);
                    if (rot[h]) {
                        kap[h] *= q.c;
                        kinv[h] *= q.ic;
                        alpha[h] = first[h] ? alpha[h] - q.t * gam[h] : alpha[h] + q.t * gam[h];
                    }
                }
            }
            ++sweeps;
            if (!__any_sync(0xffffffffu, bigs)) break;   // the same in every warp
        }
    }
    // ---- lambda_j = mu_j - sigma, v_j = g_j / mu_j; Q = V diag(max(lambda, 0))^(1/2) into Ws
    {
        float mp[2] = {0.f, 0.f};
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                g[h][k] *= kap[h];
                mp[h] = fmaf(g[h][k], g[h][k], mp[h]);
            }
        s_cn[w][lane] = mp[0];            // the last read of s_cn was before the last sweep's barriers
        s_cn[w][lane + 32] = mp[1];
        __syncthreads();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int cc = lane + 32 * h;
            const float mu2 = (s_cn[0][cc] + s_cn[1][cc]) + (s_cn[2][cc] + s_cn[3][cc]);
            const float mu = sqrtf(mu2);
            const float inv = mu > 0.f ? 1.f / mu : 0.f;
            const float lam = mu - sigma;
            const float qs = (cc < N && lam > 0.f) ? sqrtf(lam) * inv : 0.f;
            if (vglob != nullptr && cc < N) {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int r = r0 + k;
                    if (r < N) vglob[r * N + cc] = mu > 0.f ? g[h][k] * inv : (r == cc ? 1.f : 0.f);
                }
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) Ws[(r0 + k) * LD + cc] = g[h][k] * qs;
        }
    }
    __syncthreads();

    // ---- rebuild the lower triangle of Q Q^T: the packed entries dealt to the threads in turn
    pdl_trigger();
    double pv[3] = {0.0, 0.0, 0.0};
    double* xk_new = nullptr;
    if (MODE == PROJ_PRIMAL) xk_new = (a.ctrl->iter & 1) ? a.xk[0] : a.xk[1];
    const int N4 = (N + 3) & ~3;
    {
        int col = 0, cend = s;
        for (int q = tid; q < len; q += 128) {
            while (q >= cend) {
                ++col;
                cend += s - col;
            }
            const int cb = col, ra = col + (q - (cend - (s - col)));
            const float4* Qa = reinterpret_cast<const float4*>(Ws + ra * LD);
            const float4* Qb = reinterpret_cast<const float4*>(Ws + cb * LD);
            float acc0 = 0.f, acc1 = 0.f;
            for (int i = 0; i < N4 / 4; ++i) {
                const float4 x = Qa[i], y = Qb[i];
                acc0 = fmaf(x.x, y.x, acc0);
                acc1 = fmaf(x.y, y.y, acc1);
                acc0 = fmaf(x.z, y.z, acc0);
                acc1 = fmaf(x.w, y.w, acc1);
            }
            const double xv = float_scaled_to_double(acc0 + acc1, e2);
            const int pos = q;
            if (MODE == PROJ_PRIMAL) {
                const double u = a.x[a.gather_idx[off + pos]];
                const double l = a.lam[off + pos];
                const double dd = xv - u;
                xk_new[off + pos] = xv;
                a.lam[off + pos] = l + a.rho * dd;                 // Eq. LambdakUpdate
                const double wgt = (ra == cb) ? 1.0 : 2.0;
                pv[0] += wgt * dd * dd;
                pv[1] += wgt * xv * xv;
                pv[2] += wgt * u * u;
            } else {
                a.out[off + pos] = xv;
            }
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
    if (a.part != nullptr && w == 0 && lane == 0) a.part[blk * 4 + 3] = (double)sweeps;
}

// ---------------------------------------------------------------------------------------------
// FP32, padded order N <= NR (NR = 8, 16, 32): one warp segment of NR lanes per clique (32 / NR
// cliques per warp, 4 warps per CTA), lane c holding column c of G = B V in registers, so a round
// of the one-sided Jacobi iteration needs no barrier and no shared memory: the partner column
// arrives by shuffles and both ends compute the rotation from the same Gram entries. The shift is
// sigma = 2 ||W||_F, so every column of G keeps a norm mu_j = lambda_j + sigma >= ||W||_F; V is
// not tracked: G's columns converge to mu_j v_j (B = W + sigma I is positive definite and
// G = B V), so v_j = g_j / mu_j and lambda_j = mu_j - sigma. The normalized columns are kept as
// the next call's warm start (G = B V_prev). Segments of one warp stop independently; a stopped
// segment's columns are left as they are while the others finish.
template <int NR>
struct OWLayout {
    static constexpr int SEG = 32 / NR;            // cliques per warp
    static constexpr int WARPS = 4;
    static constexpr int BPC = SEG * WARPS;        // cliques per CTA
    static constexpr int LD = NR + 1;
    static constexpr size_t kBytes = (size_t)BPC * NR * LD * sizeof(float);
};

template <int NR>
__device__ __forceinline__ float seg_sum(float v) {
#pragma unroll
    for (int o = NR / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <int NR>
__device__ __forceinline__ float seg_maxf(float v) {
#pragma unroll
    for (int o = NR / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <int NR>
__device__ __forceinline__ double seg_maxd(double v) {
#pragma unroll
    for (int o = NR / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <int NR>
__device__ __forceinline__ double seg_sumd(double v) {
#pragma unroll
    for (int o = NR / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int MODE, int NR>
__global__ void __launch_bounds__(128, NR == 32 ? 4 : 0) k_project_ow(ProjArgs a, double rinv) {
    using L = OWLayout<NR>;
    constexpr int LD = L::LD;
    extern __shared__ __align__(16) unsigned char smem_ow[];
    pdl_wait();
    if (a.ctrl != nullptr && a.ctrl->done) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int seg = lane / NR, c = lane % NR, base = seg * NR;
    const int slot = warp * L::SEG + seg;
    const int idx = blockIdx.x * L::BPC + slot;
    float* Ws = reinterpret_cast<float*>(smem_ow) + (size_t)slot * NR * LD;
    int blk = -1, s = 0;
    long long off = 0;
    if (idx < a.count) {
        blk = a.order ? a.order[idx] : a.first + idx;
        s = a.size[blk];
        off = a.off[blk];
        if (block_stopped<MODE>(a, blk, s, off, c, NR)) {
            blk = -1;
            s = 0;
        }
    }
    const bool act = blk >= 0;
    const int N = s + (s & 1);
    const bool warm = act && a.vstore != nullptr && a.ctrl != nullptr;
    float* vglob = (act && a.vstore != nullptr) ? reinterpret_cast<float*>(a.vstore) + a.voff[blk] : nullptr;

    // ---- W scaled by 2^-e2 (exact) into the segment's tile, both triangles, zero padding. Up to
    // 16 rows the lane reads its column once, all loads in flight, and keeps it until the scale is
    // known; 32 doubles per lane would spill, so NR = 32 forms W twice, its packed entries dealt
    // to the lanes in turn (entries c, c + 32, ...) so that the lanes share the triangle evenly.
    // The block's exponent comes from the bits, and the scaling and rounding to FP32 take no FP64
    // instruction (FP64 instructions issue at one warp instruction per 64 clocks here).
    constexpr int KW = NR <= 16 ? NR : 1;
    double wc[KW];
    int emax = 0;
    const int len = s * (s + 1) / 2;
    if constexpr (NR <= 16) {
#pragma unroll
        for (int r = 0; r < NR; ++r)
            wc[r] = (r >= c && r < s) ? load_w<MODE>(a, off, packed_pos(r, c, s), rinv) : 0.0;
#pragma unroll
        for (int r = 0; r < NR; ++r) emax = max(emax, (__double2hiint(wc[r]) >> 20) & 0x7ff);
    } else {
        for (int q = c; q < len; q += NR) emax = max(emax, (__double2hiint(load_w<MODE>(a, off, q, rinv)) >> 20) & 0x7ff);
    }
#pragma unroll
    for (int o = NR / 2; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    // ilogb of max |W_ij| from the biased exponent, clamped to [-1000, 1000] as in block_exponent
    const int e2 = emax == 0 ? -1000 : emax == 0x7ff ? 0 : min(max(emax - 1023, -1000), 1000);
#pragma unroll
    for (int r = 0; r < NR; ++r) Ws[r * LD + c] = 0.f;
    __syncwarp();
    if constexpr (NR <= 16) {
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (r >= c && r < s) {
                const float wt = scaled_to_float(wc[r], e2);
                Ws[r * LD + c] = wt;
                Ws[c * LD + r] = wt;
            }
    } else {
        int col = 0, cend = s;                        // entry q lies in column col, which ends at cend
        for (int q = c; q < len; q += NR) {
            while (q >= cend) {
                ++col;
                cend += s - col;
            }
            const int r = col + (q - (cend - (s - col)));
            const float wt = scaled_to_float(load_w<MODE>(a, off, q, rinv), e2);
            Ws[r * LD + col] = wt;
            Ws[col * LD + r] = wt;
        }
    }
    __syncwarp();

    // ---- sigma = 2 ||W||_F and the initial columns: G = B (cold) or B V_prev (warm)
    float sq = 0.f;
#pragma unroll
    for (int r = 0; r < NR; ++r) sq = fmaf(Ws[r * LD + c], Ws[r * LD + c], sq);
    const float sigma = 2.f * sqrtf(seg_sum<NR>(sq));
    float g[NR];
    if (warm) {
        float vr[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) vr[r] = (r < N && c < N) ? vglob[r * N + c] : (r == c ? 1.f : 0.f);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            float acc = sigma * vr[r];
#pragma unroll
            for (int m = 0; m < NR; ++m) acc = fmaf(Ws[r * LD + m], vr[m], acc);
            g[r] = acc;
        }
    } else {
#pragma unroll
        for (int r = 0; r < NR; ++r) g[r] = Ws[r * LD + c] + ((r == c && c < N) ? sigma : 0.f);
    }
    if (c >= N) {
#pragma unroll
        for (int r = 0; r < NR; ++r) g[r] = 0.f;
    }

    // ---- sweeps over the round-robin schedule of N players. As in k_project_ws: the partner is
    // updated incrementally, each column carries a scale factor (a row update is one FMA), pairs
    // orthogonal to kWSSkip are not rotated, small rotations take the series, and a segment stops
    // after a sweep whose pairs all started within kOneSidedStop of orthogonal.
    int sweeps = 0;
    bool done = !act;
    const int n = N - 1;
    float kap = 1.f, kinv = 1.f;
    for (int sweep = 0; sweep < kOneSidedMaxSweeps; ++sweep) {
        if (__all_sync(0xffffffffu, done)) break;
        float alpha = 0.f;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            g[r] *= kap;
            alpha = fmaf(g[r], g[r], alpha);
        }
        kap = 1.f;
        kinv = 1.f;
        const int rounds = __reduce_max_sync(0xffffffffu, done ? 0 : n);
        bool big = false;
        int j = (c == 0 || c >= n) ? 0 : n - c;     // (2 rd - c) mod n
        for (int rd = 0; rd < rounds; ++rd) {
            const int p = (!done && c < N && rd < n) ? (c == n ? rd : (j == c ? n : j)) : c;
            j += 2;
            if (j >= n) j -= n;
            float gp[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) gp[r] = __shfl_sync(0xffffffffu, g[r], base + p);
            const float beta = __shfl_sync(0xffffffffu, alpha, base + p);
            const float kp = __shfl_sync(0xffffffffu, kap, base + p);
            const bool first = c < p;
            const float d = first ? beta - alpha : alpha - beta;   // alpha_j - alpha_i
            const float two_over_d = __fdividef(2.f, d);
            // four independent chains (both ends of a pair add in the same order, so they agree)
            float ga[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int r = 0; r < NR; ++r) ga[r & 3] = fmaf(g[r], gp[r], ga[r & 3]);
            const float kk = first ? kap * kp : kp * kap;
            const float gam = ((ga[0] + ga[1]) + (ga[2] + ga[3])) * kk;
            const float g2 = gam * gam, ab = alpha * beta;
            const bool rot = p != c && g2 > (kWSSkip * kWSSkip) * ab;
            big |= p != c && g2 > (kOneSidedStop * kOneSidedStop) * ab;
            const float z = gam * two_over_d;
            const bool series = fabsf(z) <= kSmallAngle;
            if (!__any_sync(0xffffffffu, rot)) continue;
            const JRot q = jacobi_rot(gam, d, z, series, __any_sync(0xffffffffu, rot && !series));
            // g_i' = c g_i - s g_j (i), g_j' = s g_i + c g_j (j), with s = t c
            const float f = rot ? (first ? -q.t : q.t) * (kp * kinv) : 0.f;
#pragma unroll
            for (int r = 0; r < NR; ++r) g[r] = fmaf(f, gp[r], g[r]);
            if (rot) {
                kap *= q.c;
                kinv *= q.ic;
                alpha = first ? alpha - q.t * gam : alpha + q.t * gam;
            }
        }
        if (!done) ++sweeps;
        // the segment's lanes agree on stopping
        const unsigned seg_mask = (NR == 32 ? 0xffffffffu : ((1u << NR) - 1u)) << base;
        if ((__ballot_sync(0xffffffffu, big) & seg_mask) == 0u) done = true;
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) g[r] *= kap;

    // ---- lambda_j = mu_j - sigma, v_j = g_j / mu_j; Q = V diag(max(lambda, 0))^(1/2) into the tile
    float mu2 = 0.f;
#pragma unroll
    for (int r = 0; r < NR; ++r) mu2 = fmaf(g[r], g[r], mu2);
    const float mu = sqrtf(mu2);
    const float inv = mu > 0.f ? 1.f / mu : 0.f;
    const float lam = mu - sigma;
    const float qs = (act && c < N && lam > 0.f) ? sqrtf(lam) * inv : 0.f;
    if (vglob != nullptr && c < N) {
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (r < N) vglob[r * N + c] = mu > 0.f ? g[r] * inv : (r == c ? 1.f : 0.f);
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) Ws[r * LD + c] = g[r] * qs;
    __syncwarp();

    // ---- rebuild the lower triangle of Q Q^T, column by column, and apply the epilogue
    pdl_trigger();
    double pv[3] = {0.0, 0.0, 0.0};
    double* xk_new = nullptr;
    if (MODE == PROJ_PRIMAL && act) xk_new = (a.ctrl->iter & 1) ? a.xk[0] : a.xk[1];
    // the packed entries dealt to the segment's lanes in turn, as for W
    int col = 0, cend = s;
    for (int q = c; q < len; q += NR) {
        while (q >= cend) {
            ++col;
            cend += s - col;
        }
        const int cb = col, ra = col + (q - (cend - (s - col)));
        {
            const float* Qa = Ws + ra * LD;
            const float* Qb = Ws + cb * LD;
            float acc = 0.f;
#pragma unroll 8
            for (int i = 0; i < N; ++i) acc = fmaf(Qa[i], Qb[i], acc);
            const double xv = float_scaled_to_double(acc, e2);
            const int pos = q;
            if (MODE == PROJ_PRIMAL) {
                const double u = a.x[a.gather_idx[off + pos]];
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
    }
    if (MODE == PROJ_PRIMAL) {
#pragma unroll
        for (int k = 0; k < 3; ++k) pv[k] = seg_sumd<NR>(pv[k]);
        if (act && c == 0) {
            a.part[blk * 4 + 0] = pv[0];
            a.part[blk * 4 + 1] = pv[1];
            a.part[blk * 4 + 2] = pv[2];
        }
    }
    if (act && a.part != nullptr && c == 0) a.part[blk * 4 + 3] = (double)sweeps;
}

// ---------------------------------------------------------------------------------------------
// FP32, padded order 32 < N <= 64: the same method as k_project_ow with one column per lane, but a
// block spans two warps (64 lanes), so the partner column crosses warps: every round each lane
// stores its column in the block's shared tile, the two warps meet at a named barrier, and each
// lane reads its partner's column from the tile (twice, for the Gram entry and for the update,
// which keeps register use near 64 floats). Two blocks per CTA of four warps.
constexpr int kOW64LD = 68;       // 16-byte rows: columns move through the tile as float4
constexpr size_t kOW64BlockFloats = 2 * 64 * kOW64LD + 3 * 64;   // tile, V (warm start), alpha, scale, scratch
constexpr size_t kOW64Bytes = 2 * kOW64BlockFloats * sizeof(float);

__device__ __forceinline__ void pair_sync(int pair) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + pair), "r"(64) : "memory");
}

template <int MODE>
__global__ void __launch_bounds__(128) k_project_ow64(ProjArgs a, double rinv) {
    constexpr int LD = kOW64LD;
    extern __shared__ __align__(16) unsigned char smem_ow64[];
    pdl_wait();
    if (a.ctrl != nullptr && a.ctrl->done) return;
    const int pair = threadIdx.x >> 6, c = threadIdx.x & 63;
    const int idx = blockIdx.x * 2 + pair;
    float* Ts = reinterpret_cast<float*>(smem_ow64) + (size_t)pair * kOW64BlockFloats;   // 64 x LD
    float* Vs = Ts + 64 * LD;                                                           // 64 x LD
    float* als = Vs + 64 * LD;                                                          // 64
    float* kps = als + 64;                                                              // 64
    float* red = kps + 64;                                                              // 64
    if (idx >= a.count) return;                     // both warps of the pair leave together
    const int blk = a.order ? a.order[idx] : a.first + idx;
    const int s = a.size[blk];
    const long long off = a.off[blk];
    if (block_stopped<MODE>(a, blk, s, off, c, 64)) return;
    const int N = s + (s & 1);
    const bool warm = a.vstore != nullptr && a.ctrl != nullptr;
    float* vglob = a.vstore != nullptr ? reinterpret_cast<float*>(a.vstore) + a.voff[blk] : nullptr;

    // ---- W scaled by 2^-e2 (exact) into the tile, both triangles, zero padding. The packed
    // entries are dealt to the 64 lanes in turn (lane c takes entries c, c + 64, ...), so the lanes
    // share the triangle evenly; W is formed once (one FMA) into FP64 scratch (the V tile, free
    // until the warm start fills it), the block's exponent comes from the bits, and the scaling
    // and rounding to FP32 take no FP64 instruction.
    const int len = s * (s + 1) / 2;
    double* wsc = reinterpret_cast<double*>(Vs);      // 64 x LD floats hold the 2080 doubles of s = 64
    int emax = 0;
    for (int q = c; q < len; q += 64) {
        const double wv = load_w<MODE>(a, off, q, rinv);
        wsc[q] = wv;
        emax = max(emax, (__double2hiint(wv) >> 20) & 0x7ff);
    }
    emax = __reduce_max_sync(0xffffffffu, emax);
    int* redi = reinterpret_cast<int*>(red);
    if ((c & 31) == 0) redi[c >> 5] = emax;
    for (int r = 0; r < 64; ++r) Ts[r * LD + c] = 0.f;
    pair_sync(pair);
    emax = max(redi[0], redi[1]);
    // ilogb of max |W_ij| from the biased exponent, clamped to [-1000, 1000] as in block_exponent
    const int e2 = emax == 0 ? -1000 : emax == 0x7ff ? 0 : min(max(emax - 1023, -1000), 1000);
    {
        int col = 0, cend = s;                        // entry q lies in column col, which ends at cend
        for (int q = c; q < len; q += 64) {
            while (q >= cend) {
                ++col;
                cend += s - col;
            }
            const int r = col + (q - (cend - (s - col)));
            const float wt = scaled_to_float(wsc[q], e2);
            Ts[r * LD + col] = wt;
            Ts[col * LD + r] = wt;
        }
    }
    pair_sync(pair);                                  // the scratch is read before V overwrites it
    if (warm)
        for (int r = 0; r < 64; ++r) Vs[r * LD + c] = (r < N && c < N) ? vglob[r * N + c] : (r == c ? 1.f : 0.f);
    pair_sync(pair);

    // ---- sigma = 2 ||W||_F and G = B (cold) or B V_prev (warm), column c in registers
    float sq = 0.f;
    for (int r = 0; r < 64; ++r) sq = fmaf(Ts[r * LD + c], Ts[r * LD + c], sq);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if ((c & 31) == 0) red[c >> 5] = sq;
    pair_sync(pair);
    const float sigma = 2.f * sqrtf(red[0] + red[1]);
    float g[64];
    if (warm) {
#pragma unroll
        for (int r = 0; r < 64; ++r) g[r] = sigma * Vs[r * LD + c];
        for (int m = 0; m < 64; ++m) {
            const float vm = Vs[m * LD + c];
#pragma unroll
            for (int r = 0; r < 64; ++r) g[r] = fmaf(Ts[r * LD + m], vm, g[r]);
        }
    } else {
#pragma unroll
        for (int r = 0; r < 64; ++r) g[r] = Ts[r * LD + c] + ((r == c && c < N) ? sigma : 0.f);
    }
    if (c >= N) {
#pragma unroll
        for (int r = 0; r < 64; ++r) g[r] = 0.f;
    }

    // ---- sweeps: columns meet through the tile. As in k_project_ws: incremental partners, a
    // scale factor per column (a row update is one FMA), no rotation for pairs orthogonal to
    // kWSSkip, series for small rotations, stop after a sweep that began within kOneSidedStop.
    int sweeps = 0;
    const int n = N - 1;
    float kap = 1.f, kinv = 1.f;
    for (int sweep = 0; sweep < kOneSidedMaxSweeps; ++sweep) {
        float alpha = 0.f;
#pragma unroll
        for (int r = 0; r < 64; ++r) {
            g[r] *= kap;
            alpha = fmaf(g[r], g[r], alpha);
        }
        kap = 1.f;
        kinv = 1.f;
        bool big = false;
        int j = (c == 0 || c >= n) ? 0 : n - c;     // (2 rd - c) mod n
        for (int rd = 0; rd < n; ++rd) {
            const int p = c >= N ? c : (c == n ? rd : (j == c ? n : j));
            j += 2;
            if (j >= n) j -= n;
            pair_sync(pair);                                  // the previous round's reads are done
            float4* mine = reinterpret_cast<float4*>(Ts + c * LD);
#pragma unroll
            for (int k = 0; k < 16; ++k) mine[k] = make_float4(g[4 * k], g[4 * k + 1], g[4 * k + 2], g[4 * k + 3]);
            als[c] = alpha;
            kps[c] = kap;
            pair_sync(pair);
            const float4* gp4 = reinterpret_cast<const float4*>(Ts + p * LD);
            const float beta = als[p], kp = kps[p];
            const bool first = c < p;
            const float d = first ? beta - alpha : alpha - beta;   // alpha_j - alpha_i
            const float two_over_d = __fdividef(2.f, d);
            float ga[4] = {0.f, 0.f, 0.f, 0.f};      // four chains, same order at both ends
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const float4 q = gp4[k];
                ga[0] = fmaf(g[4 * k], q.x, ga[0]);
                ga[1] = fmaf(g[4 * k + 1], q.y, ga[1]);
                ga[2] = fmaf(g[4 * k + 2], q.z, ga[2]);
                ga[3] = fmaf(g[4 * k + 3], q.w, ga[3]);
            }
            const float kk = first ? kap * kp : kp * kap;
            const float gam = ((ga[0] + ga[1]) + (ga[2] + ga[3])) * kk;
            const float g2 = gam * gam, ab = alpha * beta;
            const bool rot = p != c && g2 > (kWSSkip * kWSSkip) * ab;
            big |= p != c && g2 > (kOneSidedStop * kOneSidedStop) * ab;
            const float z = gam * two_over_d;
            const bool series = fabsf(z) <= kSmallAngle;
            if (!__any_sync(0xffffffffu, rot)) continue;        // this warp has nothing to rotate
            const JRot q = jacobi_rot(gam, d, z, series, __any_sync(0xffffffffu, rot && !series));
            const float f = rot ? (first ? -q.t : q.t) * (kp * kinv) : 0.f;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const float4 v = gp4[k];
                g[4 * k] = fmaf(f, v.x, g[4 * k]);
                g[4 * k + 1] = fmaf(f, v.y, g[4 * k + 1]);
                g[4 * k + 2] = fmaf(f, v.z, g[4 * k + 2]);
                g[4 * k + 3] = fmaf(f, v.w, g[4 * k + 3]);
            }
            if (rot) {
                kap *= q.c;
                kinv *= q.ic;
                alpha = first ? alpha - q.t * gam : alpha + q.t * gam;
            }
        }
        ++sweeps;
        const unsigned anyb = __ballot_sync(0xffffffffu, big);
        pair_sync(pair);
        if ((c & 31) == 0) red[c >> 5] = anyb ? 1.f : 0.f;
        pair_sync(pair);
        if (red[0] == 0.f && red[1] == 0.f) break;
    }
#pragma unroll
    for (int r = 0; r < 64; ++r) g[r] *= kap;

    // ---- lambda_j = mu_j - sigma, v_j = g_j / mu_j; Q = V diag(max(lambda, 0))^(1/2) into the tile
    float mu2 = 0.f;
#pragma unroll
    for (int r = 0; r < 64; ++r) mu2 = fmaf(g[r], g[r], mu2);
    const float mu = sqrtf(mu2);
    const float inv = mu > 0.f ? 1.f / mu : 0.f;
    const float lam = mu - sigma;
    const float qs = (c < N && lam > 0.f) ? sqrtf(lam) * inv : 0.f;
    if (vglob != nullptr && c < N)
        for (int r = 0; r < N; ++r) vglob[r * N + c] = mu > 0.f ? g[r] * inv : (r == c ? 1.f : 0.f);
    pair_sync(pair);
#pragma unroll
    for (int r = 0; r < 64; ++r) Ts[r * LD + c] = g[r] * qs;
    pair_sync(pair);

    // ---- rebuild the lower triangle of Q Q^T and apply the epilogue
    pdl_trigger();
    double pv[3] = {0.0, 0.0, 0.0};
    double* xk_new = nullptr;
    if (MODE == PROJ_PRIMAL) xk_new = (a.ctrl->iter & 1) ? a.xk[0] : a.xk[1];
    // the packed entries dealt to the lanes in turn, as for W; rows of Q read four at a time
    const int N4 = (N + 3) & ~3;
    int col = 0, cend = s;
    for (int q = c; q < len; q += 64) {
        while (q >= cend) {
            ++col;
            cend += s - col;
        }
        const int cb = col, ra = col + (q - (cend - (s - col)));
        {
            const float4* Qa = reinterpret_cast<const float4*>(Ts + ra * LD);
            const float4* Qb = reinterpret_cast<const float4*>(Ts + cb * LD);
            float acc0 = 0.f, acc1 = 0.f;
            for (int i = 0; i < N4 / 4; ++i) {
                const float4 x = Qa[i], y = Qb[i];
                acc0 = fmaf(x.x, y.x, acc0);
                acc1 = fmaf(x.y, y.y, acc1);
                acc0 = fmaf(x.z, y.z, acc0);
                acc1 = fmaf(x.w, y.w, acc1);
            }
            const double xv = float_scaled_to_double(acc0 + acc1, e2);
            const int pos = q;
            if (MODE == PROJ_PRIMAL) {
                const double u = a.x[a.gather_idx[off + pos]];
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
    }
    if (MODE == PROJ_PRIMAL) {
        double* rd = reinterpret_cast<double*>(Vs);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) pv[k] += __shfl_xor_sync(0xffffffffu, pv[k], o);
        }
        pair_sync(pair);
        if ((c & 31) == 0)
            for (int k = 0; k < 3; ++k) rd[(c >> 5) * 3 + k] = pv[k];
        pair_sync(pair);
        if (c == 0) {
            a.part[blk * 4 + 0] = rd[0] + rd[3];
            a.part[blk * 4 + 1] = rd[1] + rd[4];
            a.part[blk * 4 + 2] = rd[2] + rd[5];
        }
    }
    if (a.part != nullptr && c == 0) a.part[blk * 4 + 3] = (double)sweeps;
}

template <typename T, int MODE, class SH>
cudaError_t prepare_one() {
    const size_t smem = project_smem_bytes(SDP_MAX_CLIQUE, sizeof(T) == 4 ? SDP_PROJ_FP32 : SDP_PROJ_FP64, MODE);
    return cudaFuncSetAttribute(k_project<T, MODE, SH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int MODE, int CPL>
cudaError_t prepare_os() {
    return cudaFuncSetAttribute(k_project_os<MODE, CPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)OSLayout<CPL>::kBytes);
}

template <int MODE, int NR>
cudaError_t prepare_ow() {
    return cudaFuncSetAttribute(k_project_ow<MODE, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)OWLayout<NR>::kBytes);
}

template <typename T, int MODE>
cudaError_t prepare_mode() {
    cudaError_t e;
    if (sizeof(T) == 4) {
        if ((e = prepare_os<MODE, 1>()) != cudaSuccess) return e;
        if ((e = prepare_os<MODE, 2>()) != cudaSuccess) return e;
        if ((e = prepare_ow<MODE, 8>()) != cudaSuccess) return e;
        if ((e = prepare_ow<MODE, 16>()) != cudaSuccess) return e;
        if ((e = prepare_ow<MODE, 32>()) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_project_ow64<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kOW64Bytes)) != cudaSuccess)
            return e;
    }
    if ((e = prepare_one<T, MODE, ShapeS16>()) != cudaSuccess) return e;
    if ((e = prepare_one<T, MODE, ShapeS32>()) != cudaSuccess) return e;
    if ((e = prepare_one<T, MODE, ShapeS64>()) != cudaSuccess) return e;
    return prepare_one<T, MODE, ShapeS96>();
}

template <typename T, int MODE>
cudaError_t launch_mode(const ProjArgs& a, int variant, int smax, cudaStream_t st) {
    // programmatic launch inside an iteration's chain of kernels when the iteration asks for it,
    // for the FP32 kernels only (FP64 blocks measured slower with it); stand-alone projections
    // launch after their predecessor completes
    const bool pdl = sizeof(T) == 4 && MODE != PROJ_PLAIN && a.pdl != 0;
    const size_t smem = project_smem_bytes(smax, sizeof(T) == 4 ? SDP_PROJ_FP32 : SDP_PROJ_FP64, MODE);
    const double rinv = 1.0 / a.rho;
    switch (variant) {
        case PV_OS1:
            return launch_pdl(pdl, k_project_os<MODE, 1>, dim3(a.count), dim3(128), OSLayout<1>::kBytes, st,
                              a, rinv);
        case PV_OS2:
            return launch_pdl(pdl, k_project_os<MODE, 2>, dim3(a.count), dim3(256), OSLayout<2>::kBytes, st,
                              a, rinv);
        case PV_WS32:
            return launch_pdl(pdl, k_project_ws<MODE>, dim3(a.count), dim3(128), 0, st, a, rinv);
        case PV_WS64:
            return launch_pdl(pdl, k_project_ws64<MODE>, dim3(a.count), dim3(128), 0, st, a, rinv);
        case PV_OW8:
            return launch_pdl(pdl, k_project_ow<MODE, 8>,
                              dim3((a.count + OWLayout<8>::BPC - 1) / OWLayout<8>::BPC), dim3(128),
                              OWLayout<8>::kBytes, st, a, rinv);
        case PV_OW16:
            return launch_pdl(pdl, k_project_ow<MODE, 16>,
                              dim3((a.count + OWLayout<16>::BPC - 1) / OWLayout<16>::BPC), dim3(128),
                              OWLayout<16>::kBytes, st, a, rinv);
        case PV_OW64:
            return launch_pdl(pdl, k_project_ow64<MODE>, dim3((a.count + 1) / 2), dim3(128), kOW64Bytes, st,
                              a, rinv);
        case PV_OW32:
            return launch_pdl(pdl, k_project_ow<MODE, 32>,
                              dim3((a.count + OWLayout<32>::BPC - 1) / OWLayout<32>::BPC), dim3(128),
                              OWLayout<32>::kBytes, st, a, rinv);
        case PV_TS16:
            return launch_pdl(pdl, k_project<T, MODE, ShapeS16>, dim3(a.count), dim3(ShapeS16::NT), smem, st,
                              a, rinv);
        case PV_TS32:
            return launch_pdl(pdl, k_project<T, MODE, ShapeS32>, dim3(a.count), dim3(ShapeS32::NT), smem, st,
                              a, rinv);
        case PV_TS64:
            return launch_pdl(pdl, k_project<T, MODE, ShapeS64>, dim3(a.count), dim3(ShapeS64::NT), smem, st,
                              a, rinv);
        default:
            return launch_pdl(pdl, k_project<T, MODE, ShapeS96>, dim3(a.count), dim3(ShapeS96::NT), smem, st,
                              a, rinv);
    }
}

}  // namespace

size_t project_smem_bytes(int smax, int prec, int mode) {
    (void)mode;
    const int N = smax + (smax & 1);
    const int LD = N + 1;
    const size_t tsz = prec == SDP_PROJ_FP32 ? 4 : 8;
    return ((size_t)3 * N * LD + N) * tsz;
}

int project_threads(int smax) {
    const int N = smax + (smax & 1);
    if (N <= 16) return ShapeS16::NT;
    if (N <= 32) return ShapeS32::NT;
    return ShapeS64::NT;
}

size_t project_vstore_elems(int s) {
    const int N = s + (s & 1);
    return (size_t)N * N;
}

cudaError_t project_prepare() {
    cudaError_t e;

    if ((e = prepare_mode<float, PROJ_PLAIN>()) != cudaSuccess) return e;
    if ((e = prepare_mode<float, PROJ_PRIMAL>()) != cudaSuccess) return e;
    if ((e = prepare_mode<float, PROJ_DUAL>()) != cudaSuccess) return e;
    if ((e = prepare_mode<double, PROJ_PLAIN>()) != cudaSuccess) return e;
    if ((e = prepare_mode<double, PROJ_PRIMAL>()) != cudaSuccess) return e;
    return prepare_mode<double, PROJ_DUAL>();
}

int project_default_variant(int s, int prec) {
    const int N = s + (s & 1);
    if (prec == SDP_PROJ_FP32 && N <= 8) return PV_OW8;
    if (prec == SDP_PROJ_FP32 && N <= 16) return PV_OW16;
    if (prec == SDP_PROJ_FP32 && N <= 32) return PV_OW32;
    if (prec == SDP_PROJ_FP32 && N <= 64) return PV_OW64;
    if (N <= 16) return PV_TS16;
    if (N <= 32) return PV_TS32;
    if (N <= 64) return PV_TS64;
    return PV_TS96;
}

bool project_variant_valid(int variant, int s, int prec) {
    const int N = s + (s & 1);
    switch (variant) {
        case PV_OS1: return prec == SDP_PROJ_FP32 && N <= 32;
        case PV_WS32: return prec == SDP_PROJ_FP32 && N <= 32;
        case PV_WS64: return prec == SDP_PROJ_FP32 && N <= 64;
        case PV_OW8: return prec == SDP_PROJ_FP32 && N <= 8;
        case PV_OW16: return prec == SDP_PROJ_FP32 && N <= 16;
        case PV_OW32: return prec == SDP_PROJ_FP32 && N <= 32;
        case PV_OW64: return prec == SDP_PROJ_FP32 && N <= 64;
        case PV_OS2: return prec == SDP_PROJ_FP32 && N <= 64;
        case PV_TS16: return N <= 16;
        case PV_TS32: return N <= 32;
        case PV_TS64: return N <= 64;
        case PV_TS96: return N <= 96;
        default: return false;
    }
}

ProjPlan make_proj_plan(const std::vector<int>& order, const std::vector<int>& size, int prec, const int* table,
                        int ow_min_blocks) {
    // A warp segment per block pays off when there are enough blocks to fill the GPU with warps;
    // with fewer, a CTA per block finishes each block sooner (the CTA shares the load, the warm
    // start, the sweeps and the rebuild): k_project_ws up to order 32, k_project_ws64 up to 64
    // (110 us for 200 blocks of order 60, against 222 us for the CTA kernel k_project_os and 133 us
    // for the two-warp k_project_ow64).
    long long small = 0;
    for (int k : order) small += (size[k] + (size[k] & 1)) <= 64;
    const bool use_ow = small >= ow_min_blocks;
    ProjPlan pl{};
    pl.runs = 0;
    for (size_t i = 0; i < order.size(); ++i) {
        const int s = size[order[i]];
        const int N = s + (s & 1);
        int v = project_default_variant(s, prec);
        if (!use_ow && (v == PV_OW8 || v == PV_OW16 || v == PV_OW32)) v = PV_WS32;
        if (!use_ow && v == PV_OW64) v = PV_WS64;
        if (table != nullptr && project_variant_valid(table[N], s, prec)) v = table[N];
        if (pl.runs > 0 && pl.variant[pl.runs - 1] == v) {
            ++pl.count[pl.runs - 1];
            pl.smax[pl.runs - 1] = std::max(pl.smax[pl.runs - 1], s);
            continue;
        }
        if (pl.runs == kMaxProjRuns) {
            // Out of runs (only with an unusual table): the last run takes the rest with a variant
            // that fits its largest block.
            const int r = pl.runs - 1;
            ++pl.count[r];
            pl.smax[r] = std::max(pl.smax[r], s);
            if (!project_variant_valid(pl.variant[r], pl.smax[r], prec))
                pl.variant[r] = project_default_variant(pl.smax[r], prec);
            continue;
        }
        pl.start[pl.runs] = (int)i;
        pl.count[pl.runs] = 1;
        pl.variant[pl.runs] = v;
        pl.smax[pl.runs] = s;
        ++pl.runs;
    }
    for (int r = 0; r < pl.runs; ++r) {
        bool id = true;
        for (int i = pl.start[r]; i < pl.start[r] + pl.count[r] && id; ++i) id = order[i] == i;
        pl.identity[r] = id ? 1 : 0;
    }
    return pl;
}

int proj_ow_min_blocks(int num_sms) { return 4 * num_sms; }

cudaError_t launch_project_variant(const ProjArgs& a, int mode, int prec, int variant, int smax, cudaStream_t st) {
    if (a.count <= 0) return cudaSuccess;
    if (!project_variant_valid(variant, smax, prec)) return cudaErrorInvalidValue;
    if (prec == SDP_PROJ_FP32) {
        if (mode == PROJ_PLAIN) return launch_mode<float, PROJ_PLAIN>(a, variant, smax, st);
        if (mode == PROJ_PRIMAL) return launch_mode<float, PROJ_PRIMAL>(a, variant, smax, st);
        return launch_mode<float, PROJ_DUAL>(a, variant, smax, st);
    }
    if (mode == PROJ_PLAIN) return launch_mode<double, PROJ_PLAIN>(a, variant, smax, st);
    if (mode == PROJ_PRIMAL) return launch_mode<double, PROJ_PRIMAL>(a, variant, smax, st);
    return launch_mode<double, PROJ_DUAL>(a, variant, smax, st);
}

cudaError_t launch_project(const ProjArgs& a, int mode, int prec, int smax, cudaStream_t st) {
    return launch_project_variant(a, mode, prec, project_default_variant(smax, prec), smax, st);
}

}  // namespace cadmm
