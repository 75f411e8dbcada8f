// Dense FP64 part of the setup on the device: the KKT factorization that Algorithms 1 and 2 cache
// before iterating (Section III.B.1: block elimination with the factor of A D^-1 A^T).
//
//   M = A D^-1 A^T     M_ij = sum_e (w_e / D_e) A_ie A_je over the lower pattern entries e (w_e = 2
//                      off the diagonal, 1 on it), from the sliced-ELL copy of A^T already on the
//                      device. Each of G CTAs sums the outer products of a contiguous range of
//                      columns into its own m x m partial (no atomics); the partials are added in
//                      a fixed order, so M is the same on every run.
//   L L^T = M          right-looking blocked Cholesky, 32 x 32 blocks: the diagonal block in one
//                      CTA, the panel below it a row per thread, the trailing lower triangle in
//                      32 x 32 tiles. A pivot at or below 1e-12 of M's diagonal entry means A has
//                      (numerically) dependent rows.
//   L^-1               a column per warp, forward substitution against the identity.
//   M^-1 = L^-T L^-1   tiled: M^-1_ij = sum_{k >= max(i,j)} L^-1_ki L^-1_kj.
//   kappa_1(M)         ||M||_1 ||M^-1||_1 from the largest absolute row sums (both symmetric).
//
// On GB300 an FP64 FMA issues at 1.68 per clock per SM, so these steps spread over every SM;
// the host, with a handful of FP64 units, took most of a setup's time from m of a few hundred.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sdp_internal.h"

namespace cadmm {

namespace {

constexpr int kNB = 32;                  // Cholesky and product block
constexpr int kMThreads = 256;

// ------------------------------------------------------------------ M = A D^-1 A^T, partials
// CTA g: slices [s_lo[g], s_lo[g+1]); slot t of slice s is column sell_col[32 s + t] with
// slot_len[32 s + t] entries at sell_off[s] + 32 k + t. A column's entries (at most kMaxCol)
// are staged in shared memory; thread t takes rows t and len - 1 - t of the column's outer
// product (k2 <= k1), so the threads get equal shares of the triangle.
constexpr int kMaxCol = 4096;
__global__ void __launch_bounds__(kMThreads) k_kkt_partial(const int* s_lo, const int* sell_col, const int* slot_len,
                                                           const long long* sell_off, const unsigned short* sell_row,
                                                           const double* sell_val, const double* wdinv, int m,
                                                           double* part) {
    __shared__ int rs[kMaxCol];
    __shared__ double vs[kMaxCol];
    double* Mp = part + (size_t)blockIdx.x * m * m;
    for (int s = s_lo[blockIdx.x]; s < s_lo[blockIdx.x + 1]; ++s) {
        for (int t = 0; t < 32; ++t) {
            const int col = sell_col[32 * s + t];
            const int len = col < 0 ? 0 : slot_len[32 * s + t];
            if (len == 0) continue;                      // uniform across the CTA
            const double wd = wdinv[col];
            __syncthreads();                             // the previous column's products are done
            for (int k = threadIdx.x; k < len; k += blockDim.x) {
                const long long q = sell_off[s] + 32LL * k + t;
                rs[k] = sell_row[q];
                vs[k] = sell_val[q];
            }
            __syncthreads();
            const int half = (len + 1) / 2;
            for (int a = threadIdx.x; a < half; a += blockDim.x) {
                const int k1s[2] = {a, len - 1 - a};
                for (int h = 0; h < 2; ++h) {
                    const int k1 = k1s[h];
                    if (h == 1 && k1 == a) break;        // the middle row of an odd length
                    const double v1 = wd * vs[k1];
                    double* row = Mp + (size_t)rs[k1] * m;
                    for (int k2 = 0; k2 <= k1; ++k2) row[rs[k2]] = fma(v1, vs[k2], row[rs[k2]]);
                }
            }
        }
    }
}

// M (lower and upper) = sum over g of the partials' lower triangles, g ascending
__global__ void k_kkt_reduce(const double* part, int G, int m, double* M) {
    const long long mm = (long long)m * m;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < mm; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q / m), j = (int)(q % m);
        if (j > i) continue;
        double s = 0.0;
        for (int g = 0; g < G; ++g) s += part[(size_t)g * mm + q];
        M[q] = s;
        M[(size_t)j * m + i] = s;
    }
}

// ------------------------------------------------------------------ Cholesky, in place (lower)
// Diagonal block [k, k + nb): one CTA of 32 x 32 threads... (a warp per column of the block).
__global__ void __launch_bounds__(kNB * kNB / 4) k_chol_diag(double* L, const double* diag0, int m, int k, int* notpd) {
    __shared__ double a[kNB][kNB + 1];
    const int nb = min(kNB, m - k);
    for (int q = threadIdx.x; q < kNB * kNB; q += blockDim.x) {
        const int i = q / kNB, j = q % kNB;
        a[i][j] = (i < nb && j < nb && j <= i) ? L[(size_t)(k + i) * m + k + j] : 0.0;
    }
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (threadIdx.x == 0) {
            const double d = a[j][j];
            const bool ok = d > 1e-12 * diag0[k + j] && isfinite(d);
            if (!ok) atomicExch(notpd, 1);
            a[j][j] = ok ? sqrt(d) : 1.0;
        }
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) a[i][j] /= a[j][j];
        __syncthreads();
        // trailing update of the block: a_ic -= a_ij a_cj for j < c <= i
        for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
            const int i = q / nb, c = q % nb;
            if (c > j && c <= i) a[i][c] = fma(-a[i][j], a[c][j], a[i][c]);
        }
        __syncthreads();
    }
    for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
        const int i = q / nb, j = q % nb;
        if (j <= i) L[(size_t)(k + i) * m + k + j] = a[i][j];
    }
}

// Panel: rows i >= k + nb, L[i][k..k+nb) = A[i][k..k+nb) L_kk^-T (one thread per row).
__global__ void __launch_bounds__(256) k_chol_panel(double* L, int m, int k) {
    __shared__ double lk[kNB][kNB + 1];
    const int nb = min(kNB, m - k);
    for (int q = threadIdx.x; q < kNB * kNB; q += blockDim.x) {
        const int i = q / kNB, j = q % kNB;
        lk[i][j] = (i < nb && j <= i) ? L[(size_t)(k + i) * m + k + j] : 0.0;
    }
    __syncthreads();
    const int i = k + nb + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double x[kNB];
    double* row = L + (size_t)i * m + k;
#pragma unroll
    for (int c = 0; c < kNB; ++c) x[c] = c < nb ? row[c] : 0.0;
#pragma unroll
    for (int c = 0; c < kNB; ++c) {
        if (c >= nb) break;
        double s = x[c];
        for (int q = 0; q < c; ++q) s = fma(-x[q], lk[c][q], s);
        x[c] = s / lk[c][c];
    }
#pragma unroll
    for (int c = 0; c < kNB; ++c)
        if (c < nb) row[c] = x[c];
}

// Trailing update: tile (I, J), I >= J, of rows/columns >= k + nb:
// A[I][J] -= L[I][k..k+nb) L[J][k..k+nb)^T (lower tiles; the upper triangle of a diagonal tile is
// updated too and never read).
__global__ void __launch_bounds__(256) k_chol_update(double* L, int m, int k) {
    const int I = blockIdx.y, J = blockIdx.x;
    if (J > I) return;
    __shared__ double pi[kNB][kNB + 1], pj[kNB][kNB + 1];
    const int nb = min(kNB, m - k);
    const int r0 = k + nb + I * kNB, c0 = k + nb + J * kNB;
    for (int q = threadIdx.x; q < kNB * kNB; q += blockDim.x) {
        const int a = q / kNB, c = q % kNB;
        pi[a][c] = (r0 + a < m && c < nb) ? L[(size_t)(r0 + a) * m + k + c] : 0.0;
        pj[a][c] = (c0 + a < m && c < nb) ? L[(size_t)(c0 + a) * m + k + c] : 0.0;
    }
    __syncthreads();
    // thread: row a = tid / 8, columns b = (tid % 8) + 8 u, u = 0..3
    const int a = threadIdx.x / 8, b0 = threadIdx.x % 8;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c = 0; c < kNB; ++c) {
        const double x = pi[a][c];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = fma(x, pj[b0 + 8 * u][c], acc[u]);
    }
    const int i = r0 + a;
    if (i >= m) return;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int j = c0 + b0 + 8 * u;
        if (j < m && j <= i) L[(size_t)i * m + j] -= acc[u];
    }
}

// ------------------------------------------------------------------ L^-1, a column per warp
// x = L^-1 e_j by forward substitution, rows j .. m-1; the lanes split each row's dot product.
// Writes Linv (row-major, lower) and LinvT (row-major, (L^-1)^T: row j is x).
__global__ void __launch_bounds__(128) k_trinv(const double* L, int m, double* Linv, double* LinvT) {
    extern __shared__ double xs_all[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * 4 + warp;
    if (j >= m) return;
    double* x = xs_all + (size_t)warp * m;
    if (lane == 0) x[j] = 1.0 / L[(size_t)j * m + j];
    __syncwarp();
    for (int i = j + 1; i < m; ++i) {
        const double* Li = L + (size_t)i * m;
        double s0 = 0.0, s1 = 0.0;
        int q = j + lane;
        for (; q + 32 < i; q += 64) {
            s0 = fma(Li[q], x[q], s0);
            s1 = fma(Li[q + 32], x[q + 32], s1);
        }
        if (q < i) s0 = fma(Li[q], x[q], s0);
        double s = s0 + s1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) x[i] = -s / Li[i];
        __syncwarp();
    }
    for (int i = lane; i < m; i += 32) {
        const double v = i >= j ? x[i] : 0.0;
        LinvT[(size_t)j * m + i] = v;
        Linv[(size_t)i * m + j] = v;
    }
}

// ------------------------------------------------------------------ M^-1 = L^-T L^-1
// Tile (I, J), I >= J: M^-1[I rows][J rows] = sum_k LinvT[I rows][k] LinvT[J rows][k] over
// k >= I * 32 (row i of LinvT is zero before column i); mirrored into the upper triangle.
__global__ void __launch_bounds__(256) k_minv(const double* LinvT, int m, double* Minv) {
    const int I = blockIdx.y, J = blockIdx.x;
    if (J > I) return;
    __shared__ double ti[kNB][kNB + 1], tj[kNB][kNB + 1];
    const int r0 = I * kNB, c0 = J * kNB;
    const int a = threadIdx.x / 8, b0 = threadIdx.x % 8;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k0 = r0; k0 < m; k0 += kNB) {
        __syncthreads();
        for (int q = threadIdx.x; q < kNB * kNB; q += blockDim.x) {
            const int rr = q / kNB, c = q % kNB;
            ti[rr][c] = (r0 + rr < m && k0 + c < m) ? LinvT[(size_t)(r0 + rr) * m + k0 + c] : 0.0;
            tj[rr][c] = (c0 + rr < m && k0 + c < m) ? LinvT[(size_t)(c0 + rr) * m + k0 + c] : 0.0;
        }
        __syncthreads();
        for (int c = 0; c < kNB; ++c) {
            const double x = ti[a][c];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fma(x, tj[b0 + 8 * u][c], acc[u]);
        }
    }
    const int i = r0 + a;
    if (i >= m) return;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int j = c0 + b0 + 8 * u;
        if (j < m && j <= i) {
            Minv[(size_t)i * m + j] = acc[u];
            Minv[(size_t)j * m + i] = acc[u];
        }
    }
}

// Largest absolute row sum of a symmetric m x m matrix into out (one warp per row, then max).
__global__ void k_row_abs_max(const double* A, int m, double* rowsum) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= m) return;
    const double* r = A + (size_t)warp * m;
    double s = 0.0;
    for (int j = lane; j < m; j += 32) s += fabs(r[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) rowsum[warp] = s;
}

__global__ void k_diag_copy(const double* M, int m, double* diag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) diag[i] = M[(size_t)i * m + i];
}

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace

bool device_kkt_fits(int m, int max_col_len) { return m >= 1 && m <= kKktDeviceMaxM && max_col_len <= kMaxCol; }

int device_kkt(const KktInputs& in, KktOutputs& out, std::string& err) {
    const int m = in.m;
    const size_t mm = (size_t)m * m;
    cudaStream_t st = in.stream;
    int num_sms = 0, dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        err = std::string("device KKT setup: ") + cudaGetErrorString(e);
        return SDP_ERR_CUDA;
    }
    // work per slice, then G contiguous ranges of about equal work (a column of length L costs
    // L (L + 1) / 2 products)
    const int ns = in.nslices;
    std::vector<double> w(ns + 1, 0.0);
    for (int s = 0; s < ns; ++s) {
        double ws = 0.0;
        for (int t = 0; t < 32; ++t) {
            const double L = (double)in.slot_len_h[32LL * s + t];
            ws += L * (L + 1.0) / 2.0 + 1.0;
        }
        w[s + 1] = w[s] + ws;
    }
    // partial matrices: at most one per SM and at most about 2 GB of them
    const long long cap = std::max<long long>(1, (2LL << 30) / (long long)(mm * sizeof(double)));
    const int G = (int)std::max<long long>(1, std::min<long long>({(long long)num_sms, cap, (long long)std::max(1, ns)}));
    std::vector<int> s_lo(G + 1, 0);
    for (int g = 1; g < G; ++g) {
        const double target = w[ns] * g / G;
        s_lo[g] = (int)(std::lower_bound(w.begin(), w.end(), target) - w.begin());
        s_lo[g] = std::max(s_lo[g], s_lo[g - 1]);
        s_lo[g] = std::min(s_lo[g], ns);
    }
    s_lo[G] = ns;

    double* part = nullptr;
    int* d_slo = nullptr;
    int* d_slot_len = nullptr;
    double *d_diag = nullptr, *d_rows = nullptr;
    int* d_notpd = nullptr;
    auto cleanup = [&]() {
        cudaFree(part);
        cudaFree(d_slo);
        cudaFree(d_slot_len);
        cudaFree(d_diag);
        cudaFree(d_rows);
        cudaFree(d_notpd);
    };
#define KK(x)                                                                   \
    do {                                                                        \
        const cudaError_t e_ = (x);                                             \
        if (e_ != cudaSuccess) {                                                \
            cleanup();                                                          \
            err = std::string("device KKT setup: ") + cudaGetErrorString(e_);   \
            return SDP_ERR_CUDA;                                                \
        }                                                                       \
    } while (0)
    KK(cudaMalloc(&part, (size_t)G * mm * sizeof(double)));
    KK(cudaMalloc(&d_slo, sizeof(int) * (G + 1)));
    KK(cudaMalloc(&d_slot_len, sizeof(int) * std::max<size_t>(1, in.slot_len_h.size())));
    KK(cudaMalloc(&d_diag, sizeof(double) * m));
    KK(cudaMalloc(&d_rows, sizeof(double) * m * 2));
    KK(cudaMalloc(&d_notpd, sizeof(int)));
    KK(cudaMemsetAsync(part, 0, (size_t)G * mm * sizeof(double), st));
    KK(cudaMemsetAsync(d_notpd, 0, sizeof(int), st));
    KK(cudaMemcpyAsync(d_slo, s_lo.data(), sizeof(int) * (G + 1), cudaMemcpyHostToDevice, st));
    KK(cudaMemcpyAsync(d_slot_len, in.slot_len_h.data(), sizeof(int) * in.slot_len_h.size(), cudaMemcpyHostToDevice, st));

    k_kkt_partial<<<G, kMThreads, 0, st>>>(d_slo, in.sell_col, d_slot_len, in.sell_off, in.sell_row, in.sell_val,
                                           in.wdinv, m, part);
    KK(cudaGetLastError());
    k_kkt_reduce<<<std::max(1, std::min(cdiv((long long)mm, 256), 4 * num_sms)), 256, 0, st>>>(part, G, m, out.L);
    KK(cudaGetLastError());
    // M itself stays in L until the factorization overwrites it: its row sums and diagonal first
    k_row_abs_max<<<cdiv((long long)m * 32, 256), 256, 0, st>>>(out.L, m, d_rows);
    k_diag_copy<<<cdiv(m, 256), 256, 0, st>>>(out.L, m, d_diag);
    KK(cudaGetLastError());
    for (int k = 0; k < m; k += kNB) {
        k_chol_diag<<<1, kNB * kNB / 4, 0, st>>>(out.L, d_diag, m, k, d_notpd);
        const int rest = m - k - std::min(kNB, m - k);
        if (rest > 0) {
            k_chol_panel<<<cdiv(rest, 256), 256, 0, st>>>(out.L, m, k);
            const int T = cdiv(rest, kNB);
            k_chol_update<<<dim3(T, T), 256, 0, st>>>(out.L, m, k);
        }
    }
    KK(cudaGetLastError());
    const size_t xs = (size_t)4 * m * sizeof(double);
    KK(cudaFuncSetAttribute(k_trinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xs));
    k_trinv<<<cdiv(m, 4), 128, xs, st>>>(out.L, m, out.Linv, out.LinvT);
    KK(cudaGetLastError());
    const int T = cdiv(m, kNB);
    k_minv<<<dim3(T, T), 256, 0, st>>>(out.LinvT, m, out.Minv);
    KK(cudaGetLastError());
    k_row_abs_max<<<cdiv((long long)m * 32, 256), 256, 0, st>>>(out.Minv, m, d_rows + m);
    KK(cudaGetLastError());
    std::vector<double> rows(2 * (size_t)m);
    int notpd = 0;
    KK(cudaMemcpyAsync(rows.data(), d_rows, sizeof(double) * 2 * m, cudaMemcpyDeviceToHost, st));
    KK(cudaMemcpyAsync(&notpd, d_notpd, sizeof(int), cudaMemcpyDeviceToHost, st));
    KK(cudaStreamSynchronize(st));
    cleanup();
#undef KK
    if (notpd) {
        err = "A D^-1 A^T is not positive definite (A rank-deficient)";
        return SDP_ERR_NOT_PD;
    }
    double nm = 0.0, ni = 0.0;
    for (int i = 0; i < m; ++i) {
        nm = std::max(nm, rows[i]);
        ni = std::max(ni, rows[m + i]);
    }
    out.kappa1 = nm * ni;
    if (!std::isfinite(out.kappa1)) {
        err = "A D^-1 A^T is not positive definite (A rank-deficient)";
        return SDP_ERR_NOT_PD;
    }
    return SDP_OK;
}

}  // namespace cadmm
