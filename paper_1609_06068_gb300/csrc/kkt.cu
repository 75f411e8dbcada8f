// Dense FP64 part of the setup on the device: the KKT factorization that Algorithms 1 and 2 cache
// before iterating (Section III.B.1: block elimination with the factor of A D^-1 A^T).
//
//   A^T slices         from the CSR of A already on the device: every entry scattered to its
//                      column's slot, then put in row order within the slot.
//   M = A D^-1 A^T     M_ij = sum_e (w_e / D_e) A_ie A_je over the lower pattern entries e (w_e = 2
//                      off the diagonal, 1 on it), from the A^T slices. G partials each sum the
//                      outer products of a contiguous range of columns into a packed lower
//                      triangle (in shared memory when it fits, else in L2-resident global memory
//                      split into row bands, one CTA per band); no atomics, and the partials are
//                      added in a fixed order, so M is the same on every run.
//   L L^T = M          right-looking blocked Cholesky, 32 x 32 blocks: the diagonal block in one
//                      CTA, the panel below it a row per warp, the trailing lower triangle in
//                      16 x 16 tiles. A pivot at or below 1e-12 of M's diagonal entry means A has
//                      (numerically) dependent rows.
//   L^-1               a column per CTA, forward substitution in blocks of 32 rows.
//   M^-1 = L^-T L^-1   tiled: M^-1_ij = sum_{k >= max(i,j)} L^-1_ki L^-1_kj.
//   kappa_1(M)         ||M||_1 ||M^-1||_1 from the largest absolute row sums (both symmetric).
//
// On GB300 an FP64 instruction issues at one warp instruction per 64 clocks per SM partition,
// whatever the number of active lanes, so these steps keep their lanes busy and spread their
// work over every SM; the host, with a handful of FP64 units, took most of a setup's time from m
// of a few hundred.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "sdp_internal.h"

namespace cadmm {

namespace {

constexpr int kNB = 32;                  // Cholesky block
constexpr int kUT = 16;                  // trailing-update and M^-1 tile
constexpr int kMThreads = 256;
constexpr int kWarps = kMThreads / 32;

__host__ __device__ __forceinline__ long long tri_off(int i) { return (long long)i * (i + 1) / 2; }

__device__ __forceinline__ int lower_bound_s(const int* a, int n, int v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------------------ A^T slices from the CSR
// Column e of A (entry e of E_L) goes to slot col_slot[e] = 32 s + t: its k-th entry at
// sell_off[s] + 32 k + t. k_ell_scatter puts every CSR entry in its column's slot at a position
// taken with an atomic counter (any order); k_ell_rank then moves each entry to the position its
// row ranks at among the column's rows (rows are distinct within a column), so the slices come
// out with rows ascending, as a serial transpose would give them.
__global__ void k_ell_scatter(const int* a_rowptr, int m, const int* a_col, const double* a_val, long long nnz,
                              const int* col_slot, const long long* sell_off, int* cnt, unsigned short* tmp_row,
                              double* tmp_val) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nnz; q += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = m;                              // the row i with a_rowptr[i] <= q < a_rowptr[i + 1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (a_rowptr[mid] <= q) lo = mid;
            else hi = mid;
        }
        const int e = a_col[q];
        const int k = atomicAdd(cnt + e, 1);
        const int slot = col_slot[e];
        const long long pos = sell_off[slot >> 5] + 32LL * k + (slot & 31);
        tmp_row[pos] = (unsigned short)lo;
        tmp_val[pos] = a_val[q];
    }
}

__global__ void k_ell_rank(long long nslots, const int* slot_len, const long long* sell_off,
                           const unsigned short* tmp_row, const double* tmp_val, unsigned short* ell_row,
                           double* ell_val) {
    const long long slot = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (slot >= nslots) return;
    const int len = slot_len[slot];
    const long long base = sell_off[slot >> 5] + (slot & 31);
    for (int k = lane; k < len; k += 32) {
        const unsigned short r = tmp_row[base + 32LL * k];
        int rank = 0;
        for (int j = 0; j < len; ++j) rank += tmp_row[base + 32LL * j] < r ? 1 : 0;
        ell_row[base + 32LL * rank] = r;
        ell_val[base + 32LL * rank] = tmp_val[base + 32LL * k];
    }
}

// ------------------------------------------------------------------ M = A D^-1 A^T, partials
// Partial g sums the outer products of the A^T columns in its slice range [s_lo[g], s_lo[g+1])
// (slot t of slice s is column sell_col[32 s + t], with slot_len[32 s + t] entries at
// sell_off[s] + 32 k + t, rows ascending), into the packed lower triangle of an m x m matrix
// (entry (i, j), j <= i, at i (i + 1) / 2 + j).
//   kShared: m (m + 1) / 2 doubles fit in shared memory, one CTA per partial (gridDim.x = G).
//   otherwise: CTA b * G + g takes the rows in band b, [band_lo[b], band_lo[b + 1]), of partial g,
//   in global memory; G is chosen so that the G partials stay in L2.
//
// k_kkt_partial stages one column at a time; warp w takes the column's entries k1 = w, w + 8, ...
// as rows, its lanes the entries k2 <= k1 as columns, so every product of a column goes to a
// different entry and the warps need no atomics. It is the fallback for columns too long for
// k_kkt_partial_slices below.
template <bool kShared>
__global__ void __launch_bounds__(kMThreads) k_kkt_partial(const int* s_lo, int G, const int* band_lo,
                                                           const int* sell_col, const int* slot_len,
                                                           const long long* sell_off, const unsigned short* sell_row,
                                                           const double* sell_val, const double* wdinv, int m,
                                                           double* part) {
    extern __shared__ double sm[];
    const long long P = tri_off(m);
    const int g = kShared ? blockIdx.x : blockIdx.x % G;
    const int band = kShared ? 0 : blockIdx.x / G;
    double* Ms = sm;                                 // kShared: the partial, P doubles
    double* vs = kShared ? sm + P : sm;              // the staged column: m values, then m rows
    int* rs = reinterpret_cast<int*>(vs + m);
    double* Mp = kShared ? Ms : part + (size_t)g * P;
    if (kShared)
        for (long long q = threadIdx.x; q < P; q += blockDim.x) Ms[q] = 0.0;
    const int r0 = kShared ? 0 : band_lo[band], r1 = kShared ? m : band_lo[band + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int s = s_lo[g]; s < s_lo[g + 1]; ++s) {
        const long long base = sell_off[s];
        for (int t = 0; t < 32; ++t) {
            const int col = sell_col[32 * s + t];
            const int len = col < 0 ? 0 : slot_len[32 * s + t];
            if (len == 0) continue;                      // uniform across the CTA
            const double wd = wdinv[col];
            __syncthreads();                             // the previous column's products are done
            for (int k = threadIdx.x; k < len; k += blockDim.x) {
                const long long q = base + 32LL * k + t;
                rs[k] = sell_row[q];
                vs[k] = sell_val[q];
            }
            __syncthreads();
            const int p0 = kShared ? 0 : lower_bound_s(rs, len, r0);
            const int p1 = kShared ? len : lower_bound_s(rs, len, r1);
            for (int k1 = p0 + warp; k1 < p1; k1 += kWarps) {
                const double v1 = wd * vs[k1];
                double* row = Mp + tri_off(rs[k1]);
                int k2 = lane;
                // two independent read-modify-writes in flight per lane (the entries differ)
                for (; k2 + 32 <= k1; k2 += 64) {
                    const int c0 = rs[k2], c1 = rs[k2 + 32];
                    const double a0 = row[c0], a1 = row[c1];
                    row[c0] = fma(v1, vs[k2], a0);
                    row[c1] = fma(v1, vs[k2 + 32], a1);
                }
                if (k2 <= k1) row[rs[k2]] = fma(v1, vs[k2], row[rs[k2]]);
            }
        }
    }
    if (kShared) {
        __syncthreads();
        double* out = part + (size_t)g * P;
        for (long long q = threadIdx.x; q < P; q += blockDim.x) out[q] = Ms[q];
    }
}

// The same sums with whole slices staged: slice s's 32 interleaved columns are copied to shared
// memory with cp.async (values 8 bytes and row pairs 4 bytes at a time, each element row k padded
// to 33 values and 34 rows so that a lane per k reads distinct banks) while the previous slice is
// summed, two buffers deep. M row r belongs to warp r % 8: a warp takes, column by column, the
// entries k1 whose row it owns (found 32 at a time with a ballot), its lanes the k2 <= k1, so the
// warps never write the same entry and need no barrier between columns.
constexpr int kValPitch = 33, kRowPitch = 34;      // per element row k of a staged slice
struct SliceBuf {
    double* val;            // [Lcap][kValPitch]
    double* wd;             // [32] w/D of each slot's column (0 for an empty slot)
    unsigned short* row;    // [Lcap][kRowPitch]
    int* len;               // [32]
};
__host__ __device__ inline size_t slice_buf_bytes(int Lcap) {     // rounded up to 16 bytes
    const size_t b = (size_t)Lcap * (kValPitch * sizeof(double) + kRowPitch * sizeof(unsigned short)) +
                     32 * (sizeof(double) + sizeof(int));
    return (b + 15) & ~(size_t)15;
}
__device__ inline SliceBuf slice_buf_at(unsigned char* p, int Lcap) {
    SliceBuf b;
    b.val = reinterpret_cast<double*>(p);
    b.wd = b.val + (size_t)Lcap * kValPitch;
    b.row = reinterpret_cast<unsigned short*>(b.wd + 32);
    b.len = reinterpret_cast<int*>(b.row + (size_t)Lcap * kRowPitch);
    return b;
}
__device__ __forceinline__ void cp_async(void* dst, const void* src, int bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if (bytes == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// w/D of the column in every slot (0 for an empty slot), so a slice's weights are one copy
__global__ void k_slot_wd(const int* sell_col, const double* wdinv, long long nslots, double* slot_wd) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q < nslots) {
        const int c = sell_col[q];
        slot_wd[q] = c < 0 ? 0.0 : wdinv[c];
    }
}

__device__ __forceinline__ void stage_slice(const SliceBuf& b, int s, int len_s, long long base, const int* slot_len,
                                            const double* slot_wd, const unsigned short* sell_row,
                                            const double* sell_val) {
    for (int q = threadIdx.x; q < 32 * len_s; q += blockDim.x) {
        const int k = q >> 5, t = q & 31;
        cp_async(b.val + (size_t)k * kValPitch + t, sell_val + base + q, 8);
    }
    for (int q = threadIdx.x; q < 16 * len_s; q += blockDim.x) {
        const int k = q >> 4, t2 = (q & 15) * 2;
        cp_async(b.row + (size_t)k * kRowPitch + t2, sell_row + base + 32LL * k + t2, 4);
    }
    if (threadIdx.x < 32) {
        cp_async(b.wd + threadIdx.x, slot_wd + 32LL * s + threadIdx.x, 8);
        cp_async(b.len + threadIdx.x, slot_len + 32LL * s + threadIdx.x, 4);
    }
}

template <bool kShared>
__global__ void __launch_bounds__(kMThreads) k_kkt_partial_slices(const int* s_lo, int G, const int* band_lo,
                                                                  const int* slot_len, const double* slot_wd,
                                                                  const int* sell_len, const long long* sell_off,
                                                                  const unsigned short* sell_row,
                                                                  const double* sell_val, int m, int Lcap,
                                                                  double* part) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const long long P = tri_off(m);
    const int g = kShared ? blockIdx.x : blockIdx.x % G;
    const int band = kShared ? 0 : blockIdx.x / G;
    double* Ms = reinterpret_cast<double*>(smraw);
    unsigned char* bufs = smraw + (kShared ? (size_t)P * sizeof(double) : 0);
    const size_t bb = slice_buf_bytes(Lcap);
    double* Mp = kShared ? Ms : part + (size_t)g * P;
    if (kShared)
        for (long long q = threadIdx.x; q < P; q += blockDim.x) Ms[q] = 0.0;
    const int r0 = kShared ? 0 : band_lo[band], r1 = kShared ? m : band_lo[band + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sA = s_lo[g], sB = s_lo[g + 1];
    if (sA < sB) stage_slice(slice_buf_at(bufs, Lcap), sA, sell_len[sA], sell_off[sA], slot_len, slot_wd, sell_row, sell_val);
    cp_async_commit();
    for (int s = sA; s < sB; ++s) {
        if (s + 1 < sB)
            stage_slice(slice_buf_at(bufs + ((s + 1 - sA) & 1) * bb, Lcap), s + 1, sell_len[s + 1], sell_off[s + 1],
                        slot_len, slot_wd, sell_row, sell_val);
        cp_async_commit();
        cp_async_wait<1>();                          // slice s has landed (s + 1 may be in flight)
        __syncthreads();
        const SliceBuf b = slice_buf_at(bufs + ((s - sA) & 1) * bb, Lcap);
        for (int t = 0; t < 32; ++t) {
            const int len = b.len[t];
            if (len == 0) continue;
            const double wd = b.wd[t];
            const unsigned short* rw = b.row + t;        // element k at rw[k * kRowPitch]
            const double* vl = b.val + t;                // element k at vl[k * kValPitch]
            int p0 = 0, p1 = len;
            if (!kShared) {
                int lo = 0, hi = len;                    // first k with row >= r0
                while (lo < hi) { const int mid = (lo + hi) >> 1; if ((int)rw[mid * kRowPitch] < r0) lo = mid + 1; else hi = mid; }
                p0 = lo;
                hi = len;                                // first k with row >= r1
                while (lo < hi) { const int mid = (lo + hi) >> 1; if ((int)rw[mid * kRowPitch] < r1) lo = mid + 1; else hi = mid; }
                p1 = lo;
            }
            for (int kb = p0; kb < p1; kb += 32) {
                const int kl = kb + lane;
                const bool own = kl < p1 && (rw[kl * kRowPitch] & (kWarps - 1)) == warp;
                unsigned mask = __ballot_sync(0xffffffffu, own);
                while (mask) {
                    const int k1 = kb + __ffs(mask) - 1;
                    mask &= mask - 1;
                    const double v1 = wd * vl[k1 * kValPitch];
                    double* rowp = Mp + tri_off(rw[k1 * kRowPitch]);
                    int k2 = lane;
                    for (; k2 + 32 <= k1; k2 += 64) {
                        const int c0 = rw[k2 * kRowPitch], c1 = rw[(k2 + 32) * kRowPitch];
                        const double a0 = rowp[c0], a1 = rowp[c1];
                        rowp[c0] = fma(v1, vl[k2 * kValPitch], a0);
                        rowp[c1] = fma(v1, vl[(k2 + 32) * kValPitch], a1);
                    }
                    if (k2 <= k1) {
                        const int c0 = rw[k2 * kRowPitch];
                        rowp[c0] = fma(v1, vl[k2 * kValPitch], rowp[c0]);
                    }
                }
            }
        }
        __syncthreads();                             // buffer (s - sA) & 1 is refilled next
    }
    cp_async_wait<0>();
    if (kShared) {
        __syncthreads();
        double* out = part + (size_t)g * P;
        for (long long q = threadIdx.x; q < P; q += blockDim.x) out[q] = Ms[q];
    }
}

// M (lower and upper, row-major m x m) = sum over g of the packed partials, g ascending
__global__ void k_kkt_reduce(const double* part, int G, int m, double* M) {
    const long long P = tri_off(m);
    const long long mm = (long long)m * m;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < mm; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q / m), j = (int)(q % m);
        if (j > i) continue;
        const long long at = tri_off(i) + j;
        double s = 0.0;
        for (int g = 0; g < G; ++g) s += part[(size_t)g * P + at];
        M[q] = s;
        M[(size_t)j * m + i] = s;
    }
}

// ------------------------------------------------------------------ Cholesky, in place (lower)
// Diagonal block [k, k + nb): one CTA of four warps. Step j: the pivot, its reciprocal square
// root y by two Newton-Raphson steps y <- y + y (1 - d y^2) / 2 from the single-precision
// estimate (fewer FP64 instructions than a square root and a division), L_jj = d y; every thread
// computes them from shared memory. Then the column is scaled and the trailing lower triangle
// updated, its pairs (i, c), j < c <= i, listed by c descending so that step j's pairs are a
// prefix of the list and spread evenly over the threads.
constexpr int kDiagThreads = 128;
__global__ void __launch_bounds__(kDiagThreads) k_chol_diag(double* L, const double* diag0, int m, int k, int* notpd) {
    __shared__ double a[kNB][kNB + 1];
    __shared__ double d0[kNB];
    __shared__ unsigned char pair_i[kNB * (kNB - 1) / 2], pair_c[kNB * (kNB - 1) / 2];
    const int nb = min(kNB, m - k);
    for (int q = threadIdx.x; q < kNB * kNB; q += blockDim.x) {
        const int i = q / kNB, j = q % kNB;
        a[i][j] = (i < nb && j < nb && j <= i) ? L[(size_t)(k + i) * m + k + j] : 0.0;
    }
    for (int i = threadIdx.x; i < kNB; i += blockDim.x) d0[i] = i < nb ? diag0[k + i] : 1.0;
    const int npairs = nb * (nb - 1) / 2;
    for (int q = threadIdx.x; q < npairs; q += blockDim.x) {
        int c = nb - 1, base = 0;
        while (q >= base + (nb - c)) {
            base += nb - c;
            --c;
        }
        pair_i[q] = (unsigned char)(c + (q - base));
        pair_c[q] = (unsigned char)c;
    }
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        const double d = a[j][j];
        const bool ok = d > 1e-12 * d0[j] && isfinite(d);
        double ljj = 1.0, rj = 1.0;
        if (ok) {
            if (d > 1e-30 && d < 1e30) {
                double y = (double)rsqrtf((float)d);
                double r = fma(-d * y, y, 1.0);
                y = fma(0.5 * y, r, y);
                r = fma(-d * y, y, 1.0);
                y = fma(0.5 * y, r, y);
                ljj = d * y;
                rj = y;
            } else {
                ljj = sqrt(d);
                rj = 1.0 / ljj;
            }
        }
        __syncthreads();                                  // every thread has read a[j][j]
        if (threadIdx.x == 0) {
            if (!ok) atomicExch(notpd, 1);
            a[j][j] = ljj;
        }
        for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) a[i][j] *= rj;
        __syncthreads();
        const int nact = (nb - 1 - j) * (nb - j) / 2;     // pairs with c > j
        for (int q = threadIdx.x; q < nact; q += blockDim.x) {
            const int i = pair_i[q], c = pair_c[q];
            a[i][c] = fma(-a[i][j], a[c][j], a[i][c]);
        }
        __syncthreads();
    }
    for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
        const int i = q / nb, j = q % nb;
        if (j <= i) L[(size_t)(k + i) * m + k + j] = a[i][j];
    }
}

// Panel: rows i >= k + nb, L[i][k..k+nb) = A[i][k..k+nb) L_kk^-T, a row per warp with lane c
// holding entry c: for c = 0..nb-1 the owner scales its entry by 1 / L_cc, broadcasts it, and
// the lanes c' > c subtract it times L_c'c. Two FP64 instructions per step, and the rows spread
// over every SM.
constexpr int kPanelThreads = 128;
__global__ void __launch_bounds__(kPanelThreads) k_chol_panel(double* L, int m, int k) {
    __shared__ double lk[kNB][kNB + 1];
    __shared__ double rdiag[kNB];
    const int nb = min(kNB, m - k);
    for (int q = threadIdx.x; q < kNB * kNB; q += blockDim.x) {
        const int i = q / kNB, j = q % kNB;
        lk[i][j] = (i < nb && j <= i) ? L[(size_t)(k + i) * m + k + j] : 0.0;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < kNB; c += blockDim.x) rdiag[c] = c < nb ? 1.0 / lk[c][c] : 0.0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int i = k + nb + blockIdx.x * (kPanelThreads / 32) + (threadIdx.x >> 5);
    if (i >= m) return;
    double* row = L + (size_t)i * m + k;
    double x = lane < nb ? row[lane] : 0.0;
    for (int c = 0; c < nb; ++c) {
        if (lane == c) x *= rdiag[c];
        const double xc = __shfl_sync(0xffffffffu, x, c);
        if (lane > c) x = fma(-xc, lk[lane][c], x);
    }
    if (lane < nb) row[lane] = x;
}

// Trailing update: tile (I, J), I >= J, of 16 x 16 entries of rows/columns >= k + nb:
// A[I][J] -= L[I][k..k+nb) L[J][k..k+nb)^T (lower tiles; the upper triangle of a diagonal tile is
// updated too and never read). Small tiles, so that the FP64 work spreads over every SM.
__global__ void __launch_bounds__(128) k_chol_update(double* L, int m, int k) {
    const int I = blockIdx.y, J = blockIdx.x;
    if (J > I) return;
    __shared__ double pi[kUT][kNB + 1], pj[kUT][kNB + 1];
    const int nb = min(kNB, m - k);
    const int r0 = k + nb + I * kUT, c0 = k + nb + J * kUT;
    for (int q = threadIdx.x; q < kUT * kNB; q += blockDim.x) {
        const int a = q / kNB, c = q % kNB;
        pi[a][c] = (r0 + a < m && c < nb) ? L[(size_t)(r0 + a) * m + k + c] : 0.0;
        pj[a][c] = (c0 + a < m && c < nb) ? L[(size_t)(c0 + a) * m + k + c] : 0.0;
    }
    __syncthreads();
    // thread: row a = tid / 8, columns b0 and b0 + 8
    const int a = threadIdx.x / 8, b0 = threadIdx.x % 8;
    double acc0 = 0.0, acc1 = 0.0;
    for (int c = 0; c < kNB; ++c) {
        const double x = pi[a][c];
        acc0 = fma(x, pj[b0][c], acc0);
        acc1 = fma(x, pj[b0 + 8][c], acc1);
    }
    const int i = r0 + a;
    if (i >= m) return;
    const int j0 = c0 + b0, j1 = c0 + b0 + 8;
    if (j0 < m && j0 <= i) L[(size_t)i * m + j0] -= acc0;
    if (j1 < m && j1 <= i) L[(size_t)i * m + j1] -= acc1;
}

// ------------------------------------------------------------------ L^-1, a column per CTA
// x = L^-1 e_j by forward substitution in blocks of 32 rows [i0, i0 + 32): lane r of each of the
// four warps sums L[i0 + r][q] x[q] over a quarter of the finished q in [j, i0) (independent
// loads, no reductions), then warp 0 adds the quarters and solves the 32 x 32 diagonal block:
// for c = 0..31, x_c = -s_c / L_cc is broadcast and the lanes r > c add L[i0 + r][i0 + c] x_c.
// rdiag holds 1 / L_ii. Writes Linv (row-major, lower) and LinvT (row-major, (L^-1)^T: row j is
// x). Column j = blockIdx.x: the long columns (small j) start first.
constexpr int kTrinvWarps = 4;
__global__ void k_recip_diag(const double* L, int m, double* rdiag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) rdiag[i] = 1.0 / L[(size_t)i * m + i];
}

__global__ void __launch_bounds__(32 * kTrinvWarps) k_trinv(const double* L, const double* rdiag, int m,
                                                            double* Linv, double* LinvT) {
    extern __shared__ double x[];
    __shared__ double part[kTrinvWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x;
    for (int i0 = j; i0 < m; i0 += 32) {
        const int r = i0 + lane;                          // this lane's row
        // partial sums over the finished entries, a quarter of [j, i0) per warp
        const int len = i0 - j;
        const int q0 = j + (int)((long long)len * warp / kTrinvWarps);
        const int q1 = j + (int)((long long)len * (warp + 1) / kTrinvWarps);
        double s0 = 0.0, s1 = 0.0;
        if (r < m) {
            const double* Lr = L + (size_t)r * m;
            int q = q0;
            for (; q + 1 < q1; q += 2) {
                s0 = fma(Lr[q], x[q], s0);
                s1 = fma(Lr[q + 1], x[q + 1], s1);
            }
            if (q < q1) s0 = fma(Lr[q], x[q], s0);
        }
        part[warp][lane] = s0 + s1;
        __syncthreads();
        if (warp == 0) {
            double sr = 0.0;
#pragma unroll
            for (int w = 0; w < kTrinvWarps; ++w) sr += part[w][lane];
            if (r == j) sr = -1.0;                        // the unit right-hand side: x_j = 1 / L_jj
            const double rr = r < m ? rdiag[r] : 0.0;
            const double* Lr = L + (size_t)min(r, m - 1) * m + i0;
            const int nr = min(32, m - i0);
            double xr = 0.0;
            for (int c = 0; c < nr; ++c) {
                const double xc = __shfl_sync(0xffffffffu, -sr * rr, c);
                if (lane == c) xr = xc;
                if (lane > c && r < m) sr = fma(Lr[c], xc, sr);
            }
            if (r < m) x[r] = xr;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double v = i >= j ? x[i] : 0.0;
        LinvT[(size_t)j * m + i] = v;
        Linv[(size_t)i * m + j] = v;
    }
}

// ------------------------------------------------------------------ M^-1 = L^-T L^-1
// Tile (I, J) of 16 x 16, I >= J: M^-1[I rows][J rows] = sum_k LinvT[I rows][k] LinvT[J rows][k]
// over k >= 16 I (row i of LinvT is zero before column i); mirrored into the upper triangle.
__global__ void __launch_bounds__(128) k_minv(const double* LinvT, int m, double* Minv) {
    const int I = blockIdx.y, J = blockIdx.x;
    if (J > I) return;
    __shared__ double ti[kUT][kNB + 1], tj[kUT][kNB + 1];
    const int r0 = I * kUT, c0 = J * kUT;
    const int a = threadIdx.x / 8, b0 = threadIdx.x % 8;
    double acc0 = 0.0, acc1 = 0.0;
    for (int k0 = r0; k0 < m; k0 += kNB) {
        __syncthreads();
        for (int q = threadIdx.x; q < kUT * kNB; q += blockDim.x) {
            const int rr = q / kNB, c = q % kNB;
            ti[rr][c] = (r0 + rr < m && k0 + c < m) ? LinvT[(size_t)(r0 + rr) * m + k0 + c] : 0.0;
            tj[rr][c] = (c0 + rr < m && k0 + c < m) ? LinvT[(size_t)(c0 + rr) * m + k0 + c] : 0.0;
        }
        __syncthreads();
        for (int c = 0; c < kNB; ++c) {
            const double xv = ti[a][c];
            acc0 = fma(xv, tj[b0][c], acc0);
            acc1 = fma(xv, tj[b0 + 8][c], acc1);
        }
    }
    const int i = r0 + a;
    if (i >= m) return;
    const int j0 = c0 + b0, j1 = c0 + b0 + 8;
    if (j0 < m && j0 <= i) {
        Minv[(size_t)i * m + j0] = acc0;
        Minv[(size_t)j0 * m + i] = acc0;
    }
    if (j1 < m && j1 <= i) {
        Minv[(size_t)i * m + j1] = acc1;
        Minv[(size_t)j1 * m + i] = acc1;
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

bool device_kkt_fits(int m, int max_col_len) { return m >= 1 && m <= kKktDeviceMaxM && max_col_len <= m; }

void KktRun::release() {
    if (st) cudaStreamSynchronize(st);
    for (void* p : bufs) cudaFree(p);
    bufs.clear();
    if (st) cudaStreamDestroy(st);
    st = nullptr;
}

#define KK(x)                                                                   \
    do {                                                                        \
        const cudaError_t e_ = (x);                                             \
        if (e_ != cudaSuccess) {                                                \
            err = std::string("device KKT setup: ") + cudaGetErrorString(e_);   \
            return SDP_ERR_CUDA;                                                \
        }                                                                       \
    } while (0)

int device_kkt_launch(const KktInputs& in, const KktOutputs& out, KktRun& run, std::string& err) {
    const int m = in.m;
    const size_t mm = (size_t)m * m;
    run.m = m;
    int num_sms = 0, dev = 0, smem_optin = 0;
    KK(cudaStreamCreateWithFlags(&run.st, cudaStreamNonBlocking));
    KK(cudaGetDevice(&dev));
    KK(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
    KK(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaStream_t st = run.st;
    // work per slice, then G contiguous ranges of about equal work (a column of length L costs
    // L (L + 1) / 2 products)
    const int ns = in.nslices;
    std::vector<double> w(ns + 1, 0.0);
    for (int s = 0; s < ns; ++s) {
        double ws = 0.0;
        for (int t = 0; t < 32; ++t) {
            const double Lc = (double)in.slot_len_h[32LL * s + t];
            ws += Lc * (Lc + 1.0) / 2.0 + 1.0;
        }
        w[s + 1] = w[s] + ws;
    }
    // The partials: in shared memory when the packed triangle fits (one CTA per SM); otherwise
    // as many as keep them within 64 MiB of L2 (at most 4 CTAs per SM), each split into B row
    // bands of about equal triangle area. Whole slices are staged when two of them fit beside
    // the triangle, single columns otherwise.
    const long long P = (long long)m * (m + 1) / 2;
    int Lcap = 1;
    for (int v : in.slot_len_h) Lcap = std::max(Lcap, v);
    const size_t slices_bytes = 2 * slice_buf_bytes(Lcap);
    const size_t stage_bytes = (size_t)m * (sizeof(double) + sizeof(int));
    const size_t tri_bytes = (size_t)P * sizeof(double);
    const bool use_shared = tri_bytes + stage_bytes <= (size_t)smem_optin;
    const bool use_slices = (use_shared ? tri_bytes : 0) + slices_bytes <= (size_t)smem_optin;
    const size_t shared_bytes = (use_shared ? tri_bytes : 0) + (use_slices ? slices_bytes : stage_bytes);
    const long long max_ctas = use_shared ? num_sms : 4LL * num_sms;
    const long long fit = std::max<long long>(1, (64LL << 20) / (P * (long long)sizeof(double)));
    const int G = (int)std::max<long long>(1, std::min<long long>({max_ctas, fit, (long long)std::max(1, ns)}));
    const int B = use_shared ? 1 : (int)std::max<long long>(1, std::min<long long>(max_ctas / G, m / 8));
    std::vector<int> s_lo(G + 1, 0);
    for (int g = 1; g < G; ++g) {
        const double target = w[ns] * g / G;
        s_lo[g] = (int)(std::lower_bound(w.begin(), w.end(), target) - w.begin());
        s_lo[g] = std::max(s_lo[g], s_lo[g - 1]);
        s_lo[g] = std::min(s_lo[g], ns);
    }
    s_lo[G] = ns;
    // band b: rows [m sqrt(b / B), m sqrt((b + 1) / B)), the rows below i holding about i^2 / 2
    // of the triangle
    std::vector<int> band_lo(B + 1, 0);
    for (int b = 1; b < B; ++b)
        band_lo[b] = std::max(band_lo[b - 1], std::min(m, (int)std::lround(m * std::sqrt((double)b / B))));
    band_lo[B] = m;

    auto alloc = [&](auto** p, size_t bytes) {
        void* q = nullptr;
        const cudaError_t e_ = cudaMalloc(&q, std::max<size_t>(bytes, 1));
        if (e_ == cudaSuccess) {
            run.bufs.push_back(q);
            *p = static_cast<std::remove_reference_t<decltype(**p)>*>(q);
        }
        return e_;
    };
    double* part = nullptr;
    int *d_slo = nullptr, *d_band = nullptr, *d_slot_len = nullptr;
    double *d_diag = nullptr, *d_rdiag = nullptr;
    KK(alloc(&part, (size_t)G * P * sizeof(double)));
    KK(alloc(&d_slo, sizeof(int) * (G + 1)));
    KK(alloc(&d_band, sizeof(int) * (B + 1)));
    KK(alloc(&d_slot_len, sizeof(int) * in.slot_len_h.size()));
    KK(alloc(&d_diag, sizeof(double) * m));
    KK(alloc(&d_rdiag, sizeof(double) * m));
    KK(alloc(&run.d_rows, sizeof(double) * m * 2));
    KK(alloc(&run.d_notpd, sizeof(int)));
    int* d_notpd = run.d_notpd;
    double* d_rows = run.d_rows;
    if (!use_shared) KK(cudaMemsetAsync(part, 0, (size_t)G * P * sizeof(double), st));
    KK(cudaMemsetAsync(d_notpd, 0, sizeof(int), st));
    KK(cudaMemcpyAsync(d_slo, s_lo.data(), sizeof(int) * (G + 1), cudaMemcpyHostToDevice, st));
    KK(cudaMemcpyAsync(d_band, band_lo.data(), sizeof(int) * (B + 1), cudaMemcpyHostToDevice, st));
    if (!in.slot_len_h.empty())
        KK(cudaMemcpyAsync(d_slot_len, in.slot_len_h.data(), sizeof(int) * in.slot_len_h.size(), cudaMemcpyHostToDevice, st));

    // the A^T slices from the CSR
    if (in.ell_row) {
        const long long padded = in.ell_size;
        unsigned short* tmp_row = nullptr;
        double* tmp_val = nullptr;
        int* cnt = nullptr;
        KK(alloc(&tmp_row, sizeof(unsigned short) * padded));
        KK(alloc(&tmp_val, sizeof(double) * padded));
        KK(alloc(&cnt, sizeof(int) * std::max(1, in.nEL)));
        KK(cudaMemsetAsync(cnt, 0, sizeof(int) * std::max(1, in.nEL), st));
        KK(cudaMemsetAsync(in.ell_row, 0, sizeof(unsigned short) * std::max<long long>(padded, 1), st));
        KK(cudaMemsetAsync(in.ell_val, 0, sizeof(double) * std::max<long long>(padded, 1), st));
        if (in.nnz > 0) {
            const int grid = std::max(1, std::min(cdiv(in.nnz, 256), 16 * num_sms));
            k_ell_scatter<<<grid, 256, 0, st>>>(in.a_rowptr, m, in.a_col, in.a_val, in.nnz, in.col_slot, in.sell_off,
                                                cnt, tmp_row, tmp_val);
            KK(cudaGetLastError());
        }
        const long long nslots = 32LL * ns;
        if (nslots > 0) {
            k_ell_rank<<<cdiv(nslots * 32, 256), 256, 0, st>>>(nslots, d_slot_len, in.sell_off, tmp_row, tmp_val,
                                                               in.ell_row, in.ell_val);
            KK(cudaGetLastError());
        }
    }

    // M
    const int grid = use_shared ? G : G * B;
    if (use_slices) {
        const long long nslots = 32LL * ns;
        double* d_slot_wd = nullptr;
        KK(alloc(&d_slot_wd, sizeof(double) * nslots));
        if (nslots > 0) k_slot_wd<<<cdiv(nslots, 256), 256, 0, st>>>(in.sell_col, in.wdinv, nslots, d_slot_wd);
        auto* kern = use_shared ? k_kkt_partial_slices<true> : k_kkt_partial_slices<false>;
        KK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shared_bytes));
        kern<<<grid, kMThreads, shared_bytes, st>>>(d_slo, G, d_band, d_slot_len, d_slot_wd, in.sell_len, in.sell_off,
                                                    in.sell_row, in.sell_val, m, Lcap, part);
    } else {
        auto* kern = use_shared ? k_kkt_partial<true> : k_kkt_partial<false>;
        KK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shared_bytes));
        kern<<<grid, kMThreads, shared_bytes, st>>>(d_slo, G, d_band, in.sell_col, d_slot_len, in.sell_off, in.sell_row,
                                                    in.sell_val, in.wdinv, m, part);
    }
    KK(cudaGetLastError());
    k_kkt_reduce<<<std::max(1, std::min(cdiv((long long)mm, 256), 4 * num_sms)), 256, 0, st>>>(part, G, m, out.L);
    KK(cudaGetLastError());
    // M itself stays in L until the factorization overwrites it: its row sums and diagonal first
    k_row_abs_max<<<cdiv((long long)m * 32, 256), 256, 0, st>>>(out.L, m, d_rows);
    k_diag_copy<<<cdiv(m, 256), 256, 0, st>>>(out.L, m, d_diag);
    KK(cudaGetLastError());
    for (int k = 0; k < m; k += kNB) {
        k_chol_diag<<<1, kDiagThreads, 0, st>>>(out.L, d_diag, m, k, d_notpd);
        const int rest = m - k - std::min(kNB, m - k);
        if (rest > 0) {
            k_chol_panel<<<cdiv(rest, kPanelThreads / 32), kPanelThreads, 0, st>>>(out.L, m, k);
            const int T = cdiv(rest, kUT);
            k_chol_update<<<dim3(T, T), 128, 0, st>>>(out.L, m, k);
        }
    }
    KK(cudaGetLastError());
    k_recip_diag<<<cdiv(m, 256), 256, 0, st>>>(out.L, m, d_rdiag);
    k_trinv<<<m, 32 * kTrinvWarps, (size_t)m * sizeof(double), st>>>(out.L, d_rdiag, m, out.Linv, out.LinvT);
    KK(cudaGetLastError());
    const int T = cdiv(m, kUT);
    k_minv<<<dim3(T, T), 128, 0, st>>>(out.LinvT, m, out.Minv);
    KK(cudaGetLastError());
    k_row_abs_max<<<cdiv((long long)m * 32, 256), 256, 0, st>>>(out.Minv, m, d_rows + m);
    KK(cudaGetLastError());
    return SDP_OK;
}

int device_kkt_wait(KktRun& run, KktOutputs& out, std::string& err) {
    const int m = run.m;
    std::vector<double> rows(2 * (size_t)m);
    int notpd = 0;
    KK(cudaStreamSynchronize(run.st));
    KK(cudaMemcpy(rows.data(), run.d_rows, sizeof(double) * 2 * m, cudaMemcpyDeviceToHost));
    KK(cudaMemcpy(&notpd, run.d_notpd, sizeof(int), cudaMemcpyDeviceToHost));
    run.release();
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

#undef KK

}  // namespace cadmm
