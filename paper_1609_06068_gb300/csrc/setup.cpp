// Host setup of the decomposed problem (Algorithms 1-2, "Setup: chordal decomposition, KKT
// factorization"): clique index maps, D, A on the lower pattern, and the cached factor of A D^-1 A^T.
#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <atomic>
#include <functional>
#include <mutex>
#include <numeric>
#include <thread>

#include <unistd.h>

#include "sdp_internal.h"

namespace cadmm {

namespace {


int fail(std::string& err, int code, const std::string& msg) {
    err = msg;
    return code;
}

// Lower E_L index of (row, col), row >= col; -1 when the pair is not in the pattern. E_L is
// sorted by column, then row: a binary search among the rows of one column.
struct EntryIndex {
    std::vector<long long> col_start;   // [n+1]
    std::vector<int> rows;              // [|E_L|]
    // From the entries' rows and columns, sorted by column, then row.
    void build(const std::vector<int>& el_row, const std::vector<int>& el_col, long long n) {
        col_start.assign(n + 1, 0);
        rows = el_row;
        for (int c : el_col) col_start[c + 1]++;
        for (long long c = 0; c < n; ++c) col_start[c + 1] += col_start[c];
    }
    long long find(long long r, long long c) const {
        const int* lo = rows.data() + col_start[c];
        const int* hi = rows.data() + col_start[c + 1];
        const int* it = std::lower_bound(lo, hi, (int)r);
        if (it == hi || *it != r) return -1;
        return (long long)(it - rows.data());
    }
    // The same, for a row r of column c known to come after position `after` (an entry of the
    // same column with a smaller row): a few steps forward from there, then a binary search, so
    // that a run of lookups in E_L order costs about the gaps between them.
    long long find_after(long long r, long long c, long long after) const {
        const int* base = rows.data();
        const long long end = col_start[c + 1];
        long long q = after + 1;
        for (int k = 0; k < 8 && q < end && base[q] < r; ++k) ++q;
        if (q < end && base[q] < r) q = std::lower_bound(base + q, base + end, (int)r) - base;
        return (q < end && base[q] == r) ? q : -1;
    }
};

// Set on the worker threads of a batch build: each problem is then built on one thread.
thread_local bool t_serial = false;

int worker_count() { return t_serial ? 1 : (int)std::max(1u, std::thread::hardware_concurrency()); }

// Worker threads started on first use and kept for the life of the process: a setup runs a dozen
// parallel loops of a millisecond or less, where starting and joining fresh threads for each
// loop cost about as much as the loop. One caller at a time runs tasks on it (a concurrent caller,
// or a process forked from this one, which has no workers, starts threads of its own). The calling
// thread takes tasks too; the call returns once every task has run and no worker is inside the
// task loop, so the next call cannot mix with it. The pool is never destroyed: process exit ends
// its idle workers, and a forked child, whose copy of the pool has no threads behind it, has
// nothing to join at its exit.
class WorkerPool {
public:
    static WorkerPool& get() {
        static WorkerPool* pool = new WorkerPool();
        return *pool;
    }
    int threads() const { return (int)th_.size() + 1; }
    // Runs task(t) for t in [0, n); false (nothing run) when another caller holds the pool.
    bool try_run(int n, const std::function<void(int)>& task) {
        if (getpid() != pid_) return false;
        std::unique_lock<std::mutex> use(use_mu_, std::try_to_lock);
        if (!use.owns_lock()) return false;
        {
            std::lock_guard<std::mutex> lk(mu_);
            task_ = &task;
            n_ = n;
            next_.store(0);
            done_ = 0;
            ++gen_;
        }
        cv_.notify_all();
        take_tasks();
        std::unique_lock<std::mutex> lk(mu_);
        done_cv_.wait(lk, [&] { return done_ == n_ && active_ == 0; });
        task_ = nullptr;
        return true;
    }
private:
    WorkerPool() : pid_(getpid()) {
        const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
        for (int i = 0; i + 1 < hw; ++i) th_.emplace_back([this]() { worker(); });
    }
    void take_tasks() {
        for (;;) {
            const int t = next_.fetch_add(1);
            if (t >= n_) return;
            (*task_)(t);
            std::lock_guard<std::mutex> lk(mu_);
            if (++done_ == n_) done_cv_.notify_all();
        }
    }
    void worker() {
        unsigned long long seen = 0;
        for (;;) {
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return gen_ != seen; });
                seen = gen_;
                ++active_;
            }
            take_tasks();
            std::lock_guard<std::mutex> lk(mu_);
            if (--active_ == 0 && done_ == n_) done_cv_.notify_all();
        }
    }
    const pid_t pid_;
    std::vector<std::thread> th_;
    std::mutex use_mu_, mu_;
    std::condition_variable cv_, done_cv_;
    const std::function<void(int)>* task_ = nullptr;
    int n_ = 0, done_ = 0, active_ = 0;
    std::atomic<int> next_{0};
    unsigned long long gen_ = 0;
};

// Runs f(i) for i in [0, n) in up to hardware_concurrency contiguous slices.
template <typename F>
void parallel_for(int n, F f) {
    const int hw = worker_count();
    const int nt = std::max(1, std::min(hw, n));
    if (nt == 1) {
        for (int i = 0; i < n; ++i) f(i);
        return;
    }
    const std::function<void(int)> slice = [&](int t) {
        const int lo = (int)((long long)n * t / nt), hi = (int)((long long)n * (t + 1) / nt);
        for (int i = lo; i < hi; ++i) f(i);
    };
    if (WorkerPool::get().try_run(nt, slice)) return;
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t) th.emplace_back(slice, t);
    for (auto& x : th) x.join();
}

}  // namespace

// (L^-1)^T of every problem's block, row-major at the same offsets: the upper triangular product
// then reads rows, as the lower one does.
void fill_linv_t(HostProblem& hp) {
    hp.LinvT.assign(hp.Linv.size(), 0.0);
    parallel_for(hp.ninst, [&](int q) {
        const long long off = hp.mblk_off[q];
        const int mq = hp.inst_row[q + 1] - hp.inst_row[q];
        for (int i = 0; i < mq; ++i)
            for (int j = 0; j <= i; ++j) hp.LinvT[off + (size_t)j * mq + i] = hp.Linv[off + (size_t)i * mq + j];
    });
}

int build_host_problem(int n, int m, const long long* A_ptr, const int* A_row, const int* A_col,
                       const double* A_val, const double* b, long long C_nnz, const int* C_row,
                       const int* C_col, const double* C_val, long long pat_nnz,
                       const int* pat_row, const int* pat_col, int p, const int* clique_ptr,
                       const int* clique_vtx, const sdp_cones* cones, HostProblem& hp, std::string& err,
                       bool kkt_device) {
    // ---- cone variables (free, nonnegative, second-order), appended after the pattern entries
    long long nc = 0;
    if (cones) {
        if (cones->n_free < 0 || cones->n_lin < 0 || cones->n_soc < 0 || (cones->n_soc > 0 && !cones->soc_dims))
            return fail(err, SDP_ERR_ARG, "cone sizes must be nonnegative and soc_dims non-NULL");
        nc = (long long)cones->n_free + cones->n_lin;
        for (int j = 0; j < cones->n_soc; ++j) {
            if (cones->soc_dims[j] < 1) return fail(err, SDP_ERR_ARG, "second-order cone of dimension < 1");
            nc += cones->soc_dims[j];
        }
        if (nc >= (1LL << 30)) return fail(err, SDP_ERR_UNSUPPORTED, "too many cone variables");
        if (m >= 1 && !cones->A_ptr) return fail(err, SDP_ERR_ARG, "cones->A_ptr is NULL");
    }
    const bool has_psd = n > 0;
    if (n < 0 || (!has_psd && (nc == 0 || p != 0)))
        return fail(err, SDP_ERR_ARG, "n must be positive (n = 0 needs cone variables and p = 0)");
    if (m < 1 || p < 0 || !A_ptr || !b || (p > 0 && (!clique_ptr || !clique_vtx)))
        return fail(err, SDP_ERR_ARG, "m must be positive, p >= 0, and A_ptr, b, cliques non-NULL");
    if (m > SDP_MAX_CONSTRAINTS)
        return fail(err, SDP_ERR_UNSUPPORTED, "m exceeds SDP_MAX_CONSTRAINTS");
    if (C_nnz < 0 || pat_nnz < 0 || (C_nnz > 0 && (!C_row || !C_col || !C_val)) ||
        (pat_nnz > 0 && (!pat_row || !pat_col)))
        return fail(err, SDP_ERR_ARG, "bad C or pattern arrays");
    if (A_ptr[0] != 0) return fail(err, SDP_ERR_ARG, "A_ptr[0] must be 0");
    for (int i = 0; i < m; ++i)
        if (A_ptr[i + 1] < A_ptr[i]) return fail(err, SDP_ERR_ARG, "A_ptr must be non-decreasing");
    if (A_ptr[m] > 0 && (!A_row || !A_col || !A_val))
        return fail(err, SDP_ERR_ARG, "A coordinate arrays are NULL");
    if (nc > 0) {
        const long long* cp = cones->A_ptr;
        if (cp[0] != 0) return fail(err, SDP_ERR_ARG, "cones->A_ptr[0] must be 0");
        for (int i = 0; i < m; ++i)
            if (cp[i + 1] < cp[i]) return fail(err, SDP_ERR_ARG, "cones->A_ptr must be non-decreasing");
        if (cp[m] > 0 && (!cones->A_var || !cones->A_val))
            return fail(err, SDP_ERR_ARG, "cone coefficient arrays are NULL");
        for (long long t = 0; t < cp[m]; ++t)
            if (cones->A_var[t] < 0 || cones->A_var[t] >= nc)
                return fail(err, SDP_ERR_ARG, "cone variable index out of range");
    }

    // p == 0: the cliques are those of a chordal extension of the aggregate pattern (C, every A_i
    // and the extra pattern coordinates).
    std::vector<int> ext_ptr, ext_vtx;
    if (p == 0 && has_psd) {
        if (C_nnz > 0 && (!C_row || !C_col)) return fail(err, SDP_ERR_ARG, "bad C arrays");
        const long long annz = A_ptr[m];
        std::vector<int> rr, cc;
        rr.reserve((size_t)(annz + C_nnz + pat_nnz));
        cc.reserve(rr.capacity());
        auto add = [&](const int* r, const int* c, long long k) {
            for (long long t = 0; t < k; ++t) {
                rr.push_back(r[t]);
                cc.push_back(c[t]);
            }
        };
        if (annz > 0) add(A_row, A_col, annz);
        add(C_row, C_col, C_nnz);
        add(pat_row, pat_col, pat_nnz);
        long long fill = 0;
        const int rc = chordal_cliques(n, (long long)rr.size(), rr.data(), cc.data(), ext_ptr, ext_vtx, fill, err);
        if (rc) return rc;
        p = (int)ext_ptr.size() - 1;
        clique_ptr = ext_ptr.data();
        clique_vtx = ext_vtx.data();
    }

    hp = HostProblem();
    hp.n = n;
    hp.m = m;
    hp.p = p;

    // ---- cliques: E_k sorts vertices in natural order (Section II.B)
    if (clique_ptr[0] != 0) return fail(err, SDP_ERR_CLIQUE, "clique_ptr[0] must be 0");
    long long SL = 0;
    hp.blk_size.resize(p);
    hp.blk_off.resize(p + 1);
    for (int k = 0; k < p; ++k) {
        const int lo = clique_ptr[k], hi = clique_ptr[k + 1];
        const int s = hi - lo;
        if (s < 1) return fail(err, SDP_ERR_CLIQUE, "empty clique");
        if (s > SDP_MAX_CLIQUE) return fail(err, SDP_ERR_UNSUPPORTED, "clique larger than SDP_MAX_CLIQUE");
        for (int a = lo; a < hi; ++a) {
            if (clique_vtx[a] < 0 || clique_vtx[a] >= n)
                return fail(err, SDP_ERR_CLIQUE, "clique vertex out of range");
            if (a > lo && clique_vtx[a] <= clique_vtx[a - 1])
                return fail(err, SDP_ERR_CLIQUE, "clique vertices must be strictly ascending");
        }
        hp.blk_size[k] = s;
        hp.blk_off[k] = (int)SL;
        SL += (long long)s * (s + 1) / 2;
        if (SL >= (1LL << 31)) return fail(err, SDP_ERR_UNSUPPORTED, "packed block length >= 2^31");
        hp.smax = std::max(hp.smax, s);
    }
    hp.blk_off[p] = (int)SL;
    const long long SL_mat = SL;      // clique blocks; the cone blocks follow
    SL += nc;
    if (SL >= (1LL << 31)) return fail(err, SDP_ERR_UNSUPPORTED, "packed block length >= 2^31");
    hp.SL = (int)SL;
    hp.voff.resize(p + 1);
    hp.voff[0] = 0;
    for (int k = 0; k < p; ++k) {
        const long long Nk = hp.blk_size[k] + (hp.blk_size[k] & 1);
        hp.voff[k + 1] = hp.voff[k] + Nk * Nk;
    }

    // Processing order: largest cliques first (stable), so the longest eigensolves start first.
    hp.order.resize(p);
    std::iota(hp.order.begin(), hp.order.end(), 0);
    std::stable_sort(hp.order.begin(), hp.order.end(),
                     [&](int x, int y) { return hp.blk_size[x] > hp.blk_size[y]; });

    // ---- lower pattern E_L = union of lower clique pairs, column-major (by column, then row).
    // Packed positions are enumerated in storage order: clique, column b, rows a >= b.
    std::vector<int> pos_row(SL_mat), pos_col(SL_mat);
    hp.pos_w.assign(SL, 1);
    {
        long long q = 0;
        for (int k = 0; k < p; ++k) {
            const int* v = clique_vtx + clique_ptr[k];
            const int s = hp.blk_size[k];
            for (int bb = 0; bb < s; ++bb)
                for (int a = bb; a < s; ++a, ++q) {
                    pos_row[q] = v[a];
                    pos_col[q] = v[bb];
                    hp.pos_w[q] = (a == bb) ? 1 : 2;
                }
        }
    }
    // the positions ordered by column, then row (two stable counting passes, by row and then by
    // column), and repeated pairs dropped
    std::vector<int> el_row, el_col;
    {
        const int L = (int)SL_mat;
        std::vector<int> ord1(L), ord2(L);
        std::vector<int> cnt((size_t)n + 1, 0);
        for (int q = 0; q < L; ++q) cnt[pos_row[q] + 1]++;
        for (int d = 0; d < n; ++d) cnt[d + 1] += cnt[d];
        for (int q = 0; q < L; ++q) ord1[cnt[pos_row[q]]++] = q;
        std::fill(cnt.begin(), cnt.end(), 0);
        for (int q = 0; q < L; ++q) cnt[pos_col[q] + 1]++;
        for (int d = 0; d < n; ++d) cnt[d + 1] += cnt[d];
        for (int i = 0; i < L; ++i) ord2[cnt[pos_col[ord1[i]]]++] = ord1[i];
        el_row.reserve(L);
        el_col.reserve(L);
        for (int i = 0; i < L; ++i) {
            const int q = ord2[i];
            if (el_row.empty() || pos_row[q] != el_row.back() || pos_col[q] != el_col.back()) {
                el_row.push_back(pos_row[q]);
                el_col.push_back(pos_col[q]);
            }
        }
    }
    if ((long long)el_row.size() + nc >= (1LL << 31)) return fail(err, SDP_ERR_UNSUPPORTED, "|E_L| >= 2^31");
    const int nEL_mat = (int)el_row.size();
    const int nEL = nEL_mat + (int)nc;    // cone variable j is entry nEL_mat + j
    hp.nEL = nEL;
    hp.n_cone = (int)nc;
    EntryIndex index;
    index.build(el_row, el_col, std::max(n, 1));
    hp.pat_row.resize(nEL);
    hp.pat_col.resize(nEL);
    hp.ew.assign(nEL, 1);
    for (int e = 0; e < nEL_mat; ++e) {
        hp.pat_row[e] = el_row[e];
        hp.pat_col[e] = el_col[e];
        hp.ew[e] = el_row[e] == el_col[e] ? 1 : 2;
    }
    for (int j = 0; j < (int)nc; ++j) hp.pat_row[nEL_mat + j] = hp.pat_col[nEL_mat + j] = n + j;

    // ---- H_k as a gather map, and its transpose as a CSR scatter map with ascending k. The
    // block of a cone selects its own variables.
    hp.gather_idx.resize(SL);
    std::vector<int> cnt(nEL + 1, 0);
    parallel_for(p, [&](int k) {
        for (long long q = hp.blk_off[k]; q < hp.blk_off[k] + (long long)hp.blk_size[k] * (hp.blk_size[k] + 1) / 2; ++q)
            hp.gather_idx[q] = (int)index.find(pos_row[q], pos_col[q]);
    });
    for (long long j = 0; j < nc; ++j) hp.gather_idx[SL_mat + j] = nEL_mat + (int)j;
    if (nc > 0) {
        // Projection segments: every second-order cone is one; the free and the nonnegative
        // variables are cut into pieces of at most kConeChunk (their projections are elementwise).
        auto add = [&](long long lo, long long len, int kind, bool whole) {
            for (long long a = 0; a < len; a += whole ? len : kConeChunk) {
                hp.cone_lo.push_back((int)(SL_mat + lo + a));
                hp.cone_hi.push_back((int)(SL_mat + lo + std::min(len, a + (whole ? len : kConeChunk))));
                hp.cone_kind.push_back(kind);
            }
        };
        long long o = 0;
        add(o, cones->n_free, kConeFree, false);
        o += cones->n_free;
        add(o, cones->n_lin, kConeNonneg, false);
        o += cones->n_lin;
        // second-order cones: dimension <= kSmallSoc in groups (a warp each), larger ones alone
        for (int j = 0; j < cones->n_soc; ++j) {
            const int q = cones->soc_dims[j];
            if (q <= kSmallSoc) {
                hp.soc_pos.push_back((int)(SL_mat + o));
                hp.soc_q.push_back(q);
            } else {
                add(o, q, kConeSoc, true);
            }
            o += q;
        }
        const int ns = (int)hp.soc_pos.size();
        for (int a = 0; a < ns; a += kSmallSocPerCta) {
            hp.cone_lo.push_back(a);
            hp.cone_hi.push_back(std::min(ns, a + kSmallSocPerCta));
            hp.cone_kind.push_back(kConeSocSmall);
        }
    }
    for (long long q = 0; q < SL; ++q) cnt[hp.gather_idx[q] + 1]++;
    hp.sc_ptr.resize(nEL + 1);
    hp.sc_ptr[0] = 0;
    for (int e = 0; e < nEL; ++e) hp.sc_ptr[e + 1] = hp.sc_ptr[e] + cnt[e + 1];
    hp.sc_pos.resize(SL);
    {
        std::vector<int> fillp(hp.sc_ptr.begin(), hp.sc_ptr.end() - 1);
        for (long long q = 0; q < SL; ++q) hp.sc_pos[fillp[hp.gather_idx[q]]++] = (int)q;
    }
    for (int e = 0; e < nEL; ++e)
        if (hp.sc_ptr[e + 1] - hp.sc_ptr[e] > kHeavyCount) hp.heavy.push_back(e);
    // D = sum_k H_k^T H_k (Section III.B.1): number of cliques covering each entry.
    hp.D.resize(nEL);
    hp.dinv.resize(nEL);
    hp.wdinv.resize(nEL);
    for (int e = 0; e < nEL; ++e) {
        hp.D[e] = (double)(hp.sc_ptr[e + 1] - hp.sc_ptr[e]);
        hp.dinv[e] = 1.0 / hp.D[e];
        hp.wdinv[e] = (double)hp.ew[e] / hp.D[e];
    }

    // ---- cost c on E_L; every data nonzero must lie in a clique block.
    hp.c.assign(nEL, 0.0);
    for (long long t = 0; t < C_nnz; ++t) {
        const long long r = C_row[t], cc = C_col[t];
        if (r < 0 || r >= n || cc < 0 || cc >= n) return fail(err, SDP_ERR_ARG, "C index out of range");
        if (r < cc) return fail(err, SDP_ERR_ARG, "C must be given as lower coordinates (row >= col)");
        const long long e = index.find(r, cc);
        if (e < 0) {
            if (C_val[t] == 0.0) continue;
            return fail(err, SDP_ERR_CLIQUE, "a nonzero of C is not covered by the cliques");
        }
        hp.c[e] += C_val[t];
    }
    if (nc > 0 && cones->c)
        for (long long j = 0; j < nc; ++j) hp.c[nEL_mat + j] = cones->c[j];
    for (long long t = 0; t < pat_nnz; ++t) {
        const long long r = pat_row[t], cc = pat_col[t];
        if (r < 0 || r >= n || cc < 0 || cc >= n || r < cc)
            return fail(err, SDP_ERR_ARG, "pattern coordinates out of range or not lower");
        if (index.find(r, cc) < 0)
            return fail(err, SDP_ERR_CLIQUE, "a pattern entry is not covered by the cliques");
    }
    hp.b.assign(b, b + m);

    // ---- A on E_L: CSR by constraint (duplicates merged), then CSC by entry. Constraints are
    // converted in parallel tasks over contiguous ranges of constraints, each written straight
    // into the CSR arrays at its input offset (an upper bound: merging and dropping zeros only
    // shorten a constraint), then the constraints that shrank are moved down. Entries that come
    // in increasing E_L order (the usual case) are written as they are found; otherwise the
    // constraint is put in order by a stable LSD radix sort on 11-bit digits (std::stable_sort
    // for short ones), so duplicates add up in input order. The first failing constraint (lowest
    // index) decides the error.
    {
        std::vector<long long> in_off(m + 1, 0);
        for (int i = 0; i < m; ++i)
            in_off[i + 1] = in_off[i] + (A_ptr[i + 1] - A_ptr[i]) + (nc > 0 ? cones->A_ptr[i + 1] - cones->A_ptr[i] : 0);
        if (in_off[m] >= (1LL << 31)) return fail(err, SDP_ERR_UNSUPPORTED, "nnz(A) >= 2^31");
        hp.a_col.resize(in_off[m]);
        hp.a_val.resize(in_off[m]);
        const int ntask = std::max(1, std::min(m, 4 * worker_count()));
        std::vector<int> row_len(m, 0), row_err(m, SDP_OK);
        std::vector<std::string> row_msg(m);
        int ebits = 1;
        while (ebits < 31 && (1LL << ebits) < (long long)nEL) ++ebits;
        parallel_for(ntask, [&](int tk) {
            const int i0 = (int)((long long)m * tk / ntask), i1 = (int)((long long)m * (tk + 1) / ntask);
            std::vector<std::pair<int, double>> kp, kp2;       // an out-of-order constraint's entries
            std::vector<int> hist(2048);
            auto by_entry = [](const std::pair<int, double>& x, const std::pair<int, double>& y) { return x.first < y.first; };
            for (int i = i0; i < i1; ++i) {
                int* oc = hp.a_col.data() + in_off[i];
                double* ov = hp.a_val.data() + in_off[i];
                int w = 0;                                     // entries written
                bool ordered = true;                           // so far strictly increasing
                int last = -1;
                kp.clear();
                auto put = [&](int e, double v) {
                    if (ordered && e > last) {
                        last = e;
                        if (v != 0.0) {
                            oc[w] = e;
                            ov[w++] = v;
                        }
                        return;
                    }
                    if (ordered) {                             // first entry out of order: switch
                        ordered = false;
                        for (int q = 0; q < w; ++q) kp.emplace_back(oc[q], ov[q]);
                    }
                    kp.emplace_back(e, v);
                };
                long long prev_r = -1, prev_c = -1, prev_e = -1;     // last entry found
                for (long long t = A_ptr[i]; t < A_ptr[i + 1]; ++t) {
                    const long long r = A_row[t], cc = A_col[t];
                    if (r < 0 || r >= n || cc < 0 || cc >= n) { row_err[i] = SDP_ERR_ARG; row_msg[i] = "A index out of range"; return; }
                    if (r < cc) { row_err[i] = SDP_ERR_ARG; row_msg[i] = "A must be given as lower coordinates (row >= col)"; return; }
                    const long long e = (cc == prev_c && r > prev_r) ? index.find_after(r, cc, prev_e) : index.find(r, cc);
                    if (e < 0) {
                        if (A_val[t] == 0.0) continue;
                        row_err[i] = SDP_ERR_CLIQUE;
                        row_msg[i] = "a nonzero of A is not covered by the cliques";
                        return;
                    }
                    prev_r = r;
                    prev_c = cc;
                    prev_e = e;
                    put((int)e, A_val[t]);
                }
                if (nc > 0)
                    for (long long t = cones->A_ptr[i]; t < cones->A_ptr[i + 1]; ++t)
                        put(nEL_mat + cones->A_var[t], cones->A_val[t]);
                if (!ordered) {
                    const size_t cnt = kp.size();
                    if (cnt <= 512) {
                        std::stable_sort(kp.begin(), kp.end(), by_entry);
                    } else {
                        kp2.resize(cnt);
                        for (int shift = 0; shift < ebits; shift += 11) {
                            std::fill(hist.begin(), hist.end(), 0);
                            for (size_t q = 0; q < cnt; ++q) hist[(kp[q].first >> shift) & 2047]++;
                            int sum = 0;
                            for (int d = 0; d < 2048; ++d) {
                                const int c = hist[d];
                                hist[d] = sum;
                                sum += c;
                            }
                            for (size_t q = 0; q < cnt; ++q) kp2[hist[(kp[q].first >> shift) & 2047]++] = kp[q];
                            kp.swap(kp2);
                        }
                    }
                    // merge duplicates, drop zeros
                    w = 0;
                    for (size_t t = 0; t < cnt;) {
                        const int e = kp[t].first;
                        double v = kp[t].second;
                        for (++t; t < cnt && kp[t].first == e; ++t) v += kp[t].second;
                        if (v != 0.0) {
                            oc[w] = e;
                            ov[w++] = v;
                        }
                    }
                }
                row_len[i] = w;
            }
        });
        for (int i = 0; i < m; ++i)
            if (row_err[i] != SDP_OK) return fail(err, row_err[i], row_msg[i]);
        hp.a_rowptr.assign(m + 1, 0);
        for (int i = 0; i < m; ++i) hp.a_rowptr[i + 1] = hp.a_rowptr[i] + row_len[i];
        if (hp.a_rowptr[m] != in_off[m]) {
            for (int i = 0; i < m; ++i)                        // move down, in order (never upward)
                if (hp.a_rowptr[i] != in_off[i]) {
                    std::memmove(hp.a_col.data() + hp.a_rowptr[i], hp.a_col.data() + in_off[i], sizeof(int) * row_len[i]);
                    std::memmove(hp.a_val.data() + hp.a_rowptr[i], hp.a_val.data() + in_off[i], sizeof(double) * row_len[i]);
                }
            hp.a_col.resize(hp.a_rowptr[m]);
            hp.a_val.resize(hp.a_rowptr[m]);
        }
    }
    hp.nnz = (long long)hp.a_col.size();
    // CSC by a parallel transpose over column ranges: every row of the CSR lists its columns in
    // increasing order, so the entries of row i in columns [e0, e1) are one contiguous run found
    // by binary search. Each worker owns a range of columns and walks the rows in order, so every
    // column lists its rows in increasing order (as a serial transpose would) and each worker
    // writes only its own part of the output. When the device builds the KKT factorization it
    // also fills the A^T slices from the CSR (device_kkt_launch), and the host only counts the
    // columns.
    hp.c_colptr.assign(nEL + 1, 0);
    {
        const int nt = std::max(1, std::min(4 * worker_count(), nEL / 256 + 1));
        auto cols_of = [&](int t, int& e0, int& e1) {
            e0 = (int)((long long)nEL * t / nt);
            e1 = (int)((long long)nEL * (t + 1) / nt);
        };
        auto run_of = [&](int i, int e0, int e1, int& lo, int& hi) {
            const int* c0 = hp.a_col.data() + hp.a_rowptr[i];
            const int* c1 = hp.a_col.data() + hp.a_rowptr[i + 1];
            lo = (int)(std::lower_bound(c0, c1, e0) - hp.a_col.data());
            hi = (int)(std::lower_bound(c0 + (lo - hp.a_rowptr[i]), c1, e1) - hp.a_col.data());
        };
        parallel_for(nt, [&](int t) {
            int e0, e1;
            cols_of(t, e0, e1);
            for (int i = 0; i < m; ++i) {
                int lo, hi;
                run_of(i, e0, e1, lo, hi);
                for (int q = lo; q < hi; ++q) hp.c_colptr[hp.a_col[q] + 1]++;
            }
        });
        for (int e = 0; e < nEL; ++e) hp.c_colptr[e + 1] += hp.c_colptr[e];
        int max_col = 0;
        for (int e = 0; e < nEL; ++e) max_col = std::max(max_col, hp.c_colptr[e + 1] - hp.c_colptr[e]);
        hp.kkt_on_device = kkt_device && m >= kKktDeviceMinM && device_kkt_fits(m, max_col);
        if (!hp.kkt_on_device) {
            hp.c_row.resize(hp.nnz);
            hp.c_val.resize(hp.nnz);
        }
        if (!hp.kkt_on_device) parallel_for(nt, [&](int t) {
            int e0, e1;
            cols_of(t, e0, e1);
            std::vector<int> fillp(hp.c_colptr.begin() + e0, hp.c_colptr.begin() + e1);
            for (int i = 0; i < m; ++i) {
                int lo, hi;
                run_of(i, e0, e1, lo, hi);
                for (int q = lo; q < hi; ++q) {
                    const int at = fillp[hp.a_col[q] - e0]++;
                    hp.c_row[at] = (unsigned short)i;
                    hp.c_val[at] = hp.a_val[q];
                }
            }
        });
    }

    // ---- the KKT factorization: on the device (kkt.cu, after the upload) when the caller allows it
    // and the problem fits its limits (decided above); here otherwise. The device needs each A^T
    // slot's length.
    if (!hp.kkt_on_device) {
        // ---- M = A D^-1 A^T on the full symmetric vectors: M_ij = sum_e w_e A_ie A_je / D_e, with
        // w_e = 2 off the diagonal (both (i,j) and (j,i) of the pattern) and 1 on it. Columns are
        // split into a fixed number of chunks so the sum order does not depend on the machine.
        const size_t mm = (size_t)m * m;
        std::vector<double> M(mm, 0.0);
        {
            const int chunks = (m <= 2048) ? 16 : 1;
            std::vector<std::vector<double>> part(chunks);
            auto work = [&](int ch) {
                std::vector<double>& Mp = part[ch];
                Mp.assign(mm, 0.0);
                const long long e0 = (long long)nEL * ch / chunks, e1 = (long long)nEL * (ch + 1) / chunks;
                for (long long e = e0; e < e1; ++e) {
                    const double wd = hp.wdinv[e];
                    const int lo = hp.c_colptr[e], hi = hp.c_colptr[e + 1];
                    for (int s1 = lo; s1 < hi; ++s1) {
                        const double vi = wd * hp.c_val[s1];
                        double* Mi = Mp.data() + (size_t)hp.c_row[s1] * m;
                        for (int s2 = lo; s2 <= s1; ++s2) Mi[hp.c_row[s2]] += vi * hp.c_val[s2];
                    }
                }
            };
            parallel_for(chunks, work);
            // the chunks add up in a fixed order; rows of M in parallel
            parallel_for(m, [&](int i) {
                double* Mi = M.data() + (size_t)i * m;
                for (int ch = 0; ch < chunks; ++ch) {
                    const double* Pi = part[ch].data() + (size_t)i * m;
                    for (int j = 0; j < m; ++j) Mi[j] += Pi[j];
                }
            });
        }

        // ---- Cholesky M = L L^T (row-major lower, in place). A pivot at or below 1e-12 of the
        // original diagonal means A has (numerically) dependent rows.
        std::vector<double> L(mm, 0.0);
        for (int j = 0; j < m; ++j) {
            const double* Lj = L.data() + (size_t)j * m;
            double d = M[(size_t)j * m + j];
            for (int k = 0; k < j; ++k) d -= Lj[k] * Lj[k];
            if (!(d > 1e-12 * M[(size_t)j * m + j]) || !std::isfinite(d))
                return fail(err, SDP_ERR_NOT_PD, "A D^-1 A^T is not positive definite (A rank-deficient)");
            const double ljj = std::sqrt(d);
            L[(size_t)j * m + j] = ljj;
            for (int i = j + 1; i < m; ++i) {
                double* Li = L.data() + (size_t)i * m;
                double s = M[(size_t)i * m + j];
                for (int k = 0; k < j; ++k) s -= Li[k] * Lj[k];
                Li[j] = s / ljj;
            }
        }
        // ---- L^-1 (lower) by forward substitution on the unit vectors (columns are independent: in
        // parallel, each with its own work vector), then M^-1 = L^-T L^-1, so that the affine step's
        // y is one product: M^-1_ij = sum_{k >= max(i, j)} L^-1_ki L^-1_kj, k ascending.
        std::vector<double> Linv(mm, 0.0);
        parallel_for(m, [&](int j) {
            std::vector<double> xcol(m, 0.0);
            xcol[j] = 1.0 / L[(size_t)j * m + j];
            for (int i = j + 1; i < m; ++i) {
                const double* Li = L.data() + (size_t)i * m;
                double s = 0.0;
                for (int k = j; k < i; ++k) s += Li[k] * xcol[k];
                xcol[i] = -s / Li[i];
            }
            for (int i = j; i < m; ++i) Linv[(size_t)i * m + j] = xcol[i];
        });
        // (L^-1)^T row-major, so that the products below read rows
        std::vector<double> LinvTr(mm, 0.0);
        parallel_for(m, [&](int i) {
            for (int k = i; k < m; ++k) LinvTr[(size_t)i * m + k] = Linv[(size_t)k * m + i];
        });
        hp.Minv.assign(mm, 0.0);
        parallel_for(m, [&](int i) {
            const double* Ti = LinvTr.data() + (size_t)i * m;
            for (int j = 0; j <= i; ++j) {
                const double* Tj = LinvTr.data() + (size_t)j * m;
                double s = 0.0;
                for (int k = i; k < m; ++k) s += Ti[k] * Tj[k];
                hp.Minv[(size_t)i * m + j] = s;
            }
        });
        for (int i = 0; i < m; ++i)
            for (int j = i + 1; j < m; ++j) hp.Minv[(size_t)i * m + j] = hp.Minv[(size_t)j * m + i];
        // kappa_1(M) = ||M||_1 ||M^-1||_1 (both symmetric: largest absolute row sums). With the
        // explicit inverse, x = D^-1 (r - A^T y) misses A x = rhs2 by about kappa eps; with the two
        // triangular factors by about eps, as with substitution. Above kKktTriCond the affine step
        // takes the factors (one more launch per iteration).
        {
            double nm = 0.0, ni = 0.0;
            for (int i = 0; i < m; ++i) {
                double a = 0.0, bsum = 0.0;
                for (int j = 0; j < m; ++j) {
                    a += std::fabs(M[(size_t)i * m + j]);
                    bsum += std::fabs(hp.Minv[(size_t)i * m + j]);
                }
                nm = std::max(nm, a);
                ni = std::max(ni, bsum);
            }
            hp.kkt_cond = m > 0 ? nm * ni : 1.0;
            hp.kkt_tri = hp.kkt_cond > kKktTriCond;
        }
        hp.Linv.swap(Linv);
    }

    // ---- A^T as sliced ELL (32 columns per slice, one lane per column on the device). Within
    // each window of 256 consecutive columns the columns are ordered by length (longest first,
    // stable), so a slice pads to a length close to its columns' own; the window keeps the
    // per-column reads and writes of a slice within 256 consecutive entries.
    {
        constexpr int kWindow = 256;
        const int ns = (nEL + 31) / 32;
        std::vector<int> slot_col(32LL * ns, -1);
        parallel_for((nEL + kWindow - 1) / kWindow, [&](int w) {      // windows are independent
            const int w0 = w * kWindow, w1 = std::min(w0 + kWindow, nEL);
            std::vector<int> cols(w1 - w0);
            std::iota(cols.begin(), cols.end(), w0);
            std::stable_sort(cols.begin(), cols.end(), [&](int x, int y) {
                return hp.c_colptr[x + 1] - hp.c_colptr[x] > hp.c_colptr[y + 1] - hp.c_colptr[y];
            });
            for (int t = 0; t < w1 - w0; ++t) slot_col[w0 + t] = cols[t];
        });
        hp.sell_col.assign(slot_col.begin(), slot_col.end());
        hp.sell_len.resize(ns);
        hp.sell_off.resize(ns + 1);
        long long off = 0;
        for (int sl = 0; sl < ns; ++sl) {
            int len = 0;
            for (int t = 0; t < 32; ++t) {
                const int c = slot_col[32LL * sl + t];
                if (c >= 0) len = std::max(len, hp.c_colptr[c + 1] - hp.c_colptr[c]);
            }
            hp.sell_len[sl] = len;
            hp.sell_off[sl] = off;
            off += 32LL * len;
        }
        hp.sell_off[ns] = off;
        if (off >= (1LL << 31)) return fail(err, SDP_ERR_UNSUPPORTED, "padded nnz(A) >= 2^31");
        if (!hp.kkt_on_device) {
            hp.sell_val.assign(off, 0.0);
            hp.sell_row.assign(off, 0);
            parallel_for(ns, [&](int sl) {
                // in storage order (element k of the 32 slots, then k + 1, ...): the writes are
                // contiguous and the reads are 32 forward streams
                int beg[32], len[32];
                for (int t = 0; t < 32; ++t) {
                    const int c = slot_col[32LL * sl + t];
                    beg[t] = c < 0 ? 0 : hp.c_colptr[c];
                    len[t] = c < 0 ? 0 : hp.c_colptr[c + 1] - hp.c_colptr[c];
                }
                const long long base = hp.sell_off[sl];
                for (int k = 0; k < hp.sell_len[sl]; ++k)
                    for (int t = 0; t < 32; ++t)
                        if (k < len[t]) {
                            const long long q = base + 32LL * k + t;
                            hp.sell_val[q] = hp.c_val[beg[t] + k];
                            hp.sell_row[q] = hp.c_row[beg[t] + k];
                        }
            });
            std::vector<double>().swap(hp.c_val);       // the device reads the sliced form only
            std::vector<unsigned short>().swap(hp.c_row);
        } else {
            // the device fills the slices from the CSR: it needs each slot's length and each
            // column's slot
            hp.slot_len.assign(32LL * ns, 0);
            hp.col_slot.assign(nEL, 0);
            for (long long q = 0; q < 32LL * ns; ++q) {
                const int c = slot_col[q];
                if (c < 0) continue;
                hp.slot_len[q] = hp.c_colptr[c + 1] - hp.c_colptr[c];
                hp.col_slot[c] = (int)q;
            }
        }
    }

    hp.ninst = 1;
    hp.inst_sl = {0, (int)hp.sell_len.size()};
    hp.inst_vtx = {0, n};
    hp.inst_cl = {0, p};
    hp.inst_e = {0, nEL};
    hp.inst_pos = {0, hp.SL};
    hp.inst_row = {0, m};
    hp.mblk_off = {0, (long long)m * m};
    if (hp.kkt_tri) fill_linv_t(hp);
    return SDP_OK;
}

int build_host_problem_batch(int count, const sdp_problem* in, HostProblem& out, std::string& err) {
    if (count < 1 || !in) return fail(err, SDP_ERR_ARG, "count must be >= 1 and problems non-NULL");
    // Each problem is built on one thread; problems are spread over the hardware threads.
    std::vector<HostProblem> parts(count);
    std::vector<int> rcs(count, SDP_OK);
    std::vector<std::string> errs(count);
    {
        const int nt = std::max(1, std::min(worker_count(), count));
        std::vector<std::thread> th;
        std::atomic<int> next{0};
        for (int t = 0; t < nt; ++t)
            th.emplace_back([&]() {
                t_serial = true;
                for (int q = next++; q < count; q = next++) {
                    const sdp_problem& pr = in[q];
                    rcs[q] = build_host_problem(pr.n, pr.m, pr.A_ptr, pr.A_row, pr.A_col, pr.A_val, pr.b,
                                                pr.C_nnz, pr.C_row, pr.C_col, pr.C_val, pr.pat_nnz,
                                                pr.pat_row, pr.pat_col, pr.p, pr.clique_ptr, pr.clique_vtx,
                                                nullptr, parts[q], errs[q]);
                }
            });
        for (auto& x : th) x.join();
    }
    for (int q = 0; q < count; ++q)
        if (rcs[q] != SDP_OK) return fail(err, rcs[q], "problem " + std::to_string(q) + ": " + errs[q]);

    // Totals and limits of the union.
    long long n = 0, m = 0, p = 0, nEL = 0, SL = 0, nnz = 0, mm = 0;
    for (const HostProblem& h : parts) {
        n += h.n; m += h.m; p += h.p; nEL += h.nEL; SL += h.SL; nnz += h.nnz;
        mm += (long long)h.m * h.m;
    }
    if (n >= (1LL << 31) || m >= (1LL << 31) || p >= (1LL << 31))
        return fail(err, SDP_ERR_UNSUPPORTED, "batch: n, m or p >= 2^31");
    if (nEL >= (1LL << 31) || SL >= (1LL << 31) || nnz >= (1LL << 31))
        return fail(err, SDP_ERR_UNSUPPORTED, "batch: |E_L|, S_L or nnz(A) >= 2^31");

    HostProblem& hp = out;
    hp = HostProblem();
    hp.n = (int)n; hp.m = (int)m; hp.p = (int)p; hp.nEL = (int)nEL; hp.SL = (int)SL; hp.nnz = nnz;
    hp.ninst = count;
    for (auto* v : {&hp.inst_vtx, &hp.inst_cl, &hp.inst_e, &hp.inst_pos, &hp.inst_row, &hp.inst_sl})
        v->assign(count + 1, 0);
    long long sell_total = 0;
    for (const HostProblem& h : parts) sell_total += h.sell_off.back();
    if (sell_total >= (1LL << 31)) return fail(err, SDP_ERR_UNSUPPORTED, "batch: padded nnz(A) >= 2^31");
    hp.mblk_off.assign(count + 1, 0);
    for (int q = 0; q < count; ++q) {
        const HostProblem& h = parts[q];
        hp.inst_vtx[q + 1] = hp.inst_vtx[q] + h.n;
        hp.inst_cl[q + 1] = hp.inst_cl[q] + h.p;
        hp.inst_e[q + 1] = hp.inst_e[q] + h.nEL;
        hp.inst_pos[q + 1] = hp.inst_pos[q] + h.SL;
        hp.inst_row[q + 1] = hp.inst_row[q] + h.m;
        hp.inst_sl[q + 1] = hp.inst_sl[q] + (int)h.sell_len.size();
        hp.mblk_off[q + 1] = hp.mblk_off[q] + (long long)h.m * h.m;
        hp.smax = std::max(hp.smax, h.smax);
    }
    auto reserve_all = [&]() {
        hp.pat_row.reserve(nEL); hp.pat_col.reserve(nEL); hp.ew.reserve(nEL);
        hp.D.reserve(nEL); hp.dinv.reserve(nEL); hp.wdinv.reserve(nEL); hp.c.reserve(nEL);
        hp.sc_ptr.reserve(nEL + 1);
        hp.sell_col.reserve(32LL * hp.inst_sl[count]); hp.sell_len.reserve(hp.inst_sl[count]);
        hp.sell_off.reserve(hp.inst_sl[count] + 1);
        hp.sell_val.reserve(sell_total); hp.sell_row.reserve(sell_total);
        hp.blk_off.reserve(p + 1); hp.blk_size.reserve(p);
        hp.gather_idx.reserve(SL); hp.pos_w.reserve(SL); hp.sc_pos.reserve(SL);
        hp.b.reserve(m); hp.a_rowptr.reserve(m + 1);
        hp.a_col.reserve(nnz); hp.a_val.reserve(nnz);
        hp.Minv.reserve(mm);
        hp.Linv.reserve(mm);
    };
    reserve_all();
    for (const HostProblem& h : parts) {
        hp.kkt_cond = std::max(hp.kkt_cond, h.kkt_cond);
        hp.kkt_tri = hp.kkt_tri || h.kkt_tri;
    }
    hp.sc_ptr.push_back(0);
    hp.a_rowptr.push_back(0);
    // Concatenate: indices into E_L, positions, vertices and nonzeros are shifted by the totals of
    // the problems before; A^T keeps rows within the problem (each chunk reads its problem's y).
    for (int q = 0; q < count; ++q) {
        HostProblem& h = parts[q];
        const int v0 = hp.inst_vtx[q], e0 = hp.inst_e[q], s0 = hp.inst_pos[q];
        const int a0 = hp.a_rowptr.back();
        for (int e = 0; e < h.nEL; ++e) {
            hp.pat_row.push_back(h.pat_row[e] + v0);
            hp.pat_col.push_back(h.pat_col[e] + v0);
            hp.sc_ptr.push_back(h.sc_ptr[e + 1] + s0);
        }
        const long long so = hp.sell_val.size();
        for (size_t sl = 0; sl < h.sell_len.size(); ++sl) {
            hp.sell_len.push_back(h.sell_len[sl]);
            hp.sell_off.push_back(h.sell_off[sl] + so);
        }
        for (int c : h.sell_col) hp.sell_col.push_back(c >= 0 ? c + e0 : -1);
        hp.sell_val.insert(hp.sell_val.end(), h.sell_val.begin(), h.sell_val.end());
        hp.sell_row.insert(hp.sell_row.end(), h.sell_row.begin(), h.sell_row.end());
        hp.ew.insert(hp.ew.end(), h.ew.begin(), h.ew.end());
        hp.D.insert(hp.D.end(), h.D.begin(), h.D.end());
        hp.dinv.insert(hp.dinv.end(), h.dinv.begin(), h.dinv.end());
        hp.wdinv.insert(hp.wdinv.end(), h.wdinv.begin(), h.wdinv.end());
        hp.c.insert(hp.c.end(), h.c.begin(), h.c.end());
        for (int k = 0; k < h.p; ++k) {
            hp.blk_off.push_back(h.blk_off[k] + s0);
            hp.blk_size.push_back(h.blk_size[k]);
        }
        for (int t = 0; t < h.SL; ++t) {
            hp.gather_idx.push_back(h.gather_idx[t] + e0);
            hp.sc_pos.push_back(h.sc_pos[t] + s0);
        }
        hp.pos_w.insert(hp.pos_w.end(), h.pos_w.begin(), h.pos_w.end());
        for (int e : h.heavy) hp.heavy.push_back(e + e0);
        hp.b.insert(hp.b.end(), h.b.begin(), h.b.end());
        for (int i = 0; i < h.m; ++i) hp.a_rowptr.push_back(h.a_rowptr[i + 1] + a0);
        for (int c : h.a_col) hp.a_col.push_back(c + e0);
        hp.a_val.insert(hp.a_val.end(), h.a_val.begin(), h.a_val.end());
        hp.Minv.insert(hp.Minv.end(), h.Minv.begin(), h.Minv.end());
        hp.Linv.insert(hp.Linv.end(), h.Linv.begin(), h.Linv.end());
        h = HostProblem();   // release the part as soon as it is copied
    }
    hp.blk_off.push_back((int)SL);
    hp.sell_off.push_back((long long)hp.sell_val.size());
    hp.voff.assign(p + 1, 0);
    for (long long k = 0; k < p; ++k) {
        const long long Nk = hp.blk_size[k] + (hp.blk_size[k] & 1);
        hp.voff[k + 1] = hp.voff[k] + Nk * Nk;
    }
    hp.order.resize(p);
    std::iota(hp.order.begin(), hp.order.end(), 0);
    std::stable_sort(hp.order.begin(), hp.order.end(),
                     [&](int x, int y) { return hp.blk_size[x] > hp.blk_size[y]; });
    // one affine-step method for the whole batch: the triangular factors if any problem needs them
    if (hp.kkt_tri) fill_linv_t(hp);
    return SDP_OK;
}

}  // namespace cadmm
