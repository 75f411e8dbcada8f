// C ABI of the decomposed-ADMM hot path: handle lifetime, device uploads, CUDA-graph capture of
// whole iterations, and the host loop that launches graphs and polls the device stop flag.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <memory>
#include <new>
#include <type_traits>
#include <string>
#include <thread>
#include <vector>

#include "sdp_internal.h"

using cadmm::Ctrl;
using cadmm::HostProblem;
using cadmm::IterPtrs;

namespace {

thread_local std::string g_last_error;

int set_err(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return set_err(SDP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

constexpr double kWaitTimeoutSeconds = 600.0;

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// Wait for an event with a host-side time limit. The kernels contain no device-side waits, so
// this limit only guards against a device that stopped answering.
int wait_event(cudaEvent_t ev, double timeout_s) {
    const double t0 = now_s();
    for (;;) {
        const cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return SDP_OK;
        if (e != cudaErrorNotReady) return set_err(SDP_ERR_CUDA, std::string("cudaEventQuery: ") + cudaGetErrorString(e));
        if (now_s() - t0 > timeout_s) return set_err(SDP_ERR_TIMEOUT, "timed out waiting for the device");
        std::this_thread::yield();
    }
}

int check_opts(const admm_opts* o) {
    if (!o) return set_err(SDP_ERR_ARG, "opts is NULL");
    if (!(o->rho > 0.0) || o->rho != o->rho) return set_err(SDP_ERR_ARG, "rho must be positive");
    if (o->max_iter < 0 || o->check_every < 0) return set_err(SDP_ERR_ARG, "max_iter and check_every must be >= 0");
    if (o->form != SDP_PRIMAL && o->form != SDP_DUAL) return set_err(SDP_ERR_ARG, "form must be SDP_PRIMAL or SDP_DUAL");
    if (o->prec != SDP_PROJ_FP64 && o->prec != SDP_PROJ_FP32) return set_err(SDP_ERR_ARG, "prec must be SDP_PROJ_FP64 or SDP_PROJ_FP32");
    if ((o->flags & ~SDP_FLAG_HOST_KKT) != 0) return set_err(SDP_ERR_ARG, "flags must be 0 or SDP_FLAG_HOST_KKT");
    return SDP_OK;
}

}  // namespace

namespace cadmm {
int record_error(int code, const std::string& msg) { return set_err(code, msg); }
}  // namespace cadmm

// Wall-clock stages of sdp_setup*, in milliseconds (sdp_setup_times).
enum { kSetupHost = 0, kSetupPlan, kSetupUpload, kSetupKkt, kSetupFinish, kSetupStages };
const char* const kSetupStageName[kSetupStages] = {"host_build", "plan", "alloc_upload", "device_kkt", "finish"};
using SetupClock = std::chrono::steady_clock;
double ms_since(SetupClock::time_point& t) {
    const SetupClock::time_point now = SetupClock::now();
    const double ms = std::chrono::duration<double, std::milli>(now - t).count();
    t = now;
    return ms;
}

struct sdp_ctx {
    int device = 0;
    double setup_ms[kSetupStages] = {};
    admm_opts opts{};
    int n = 0, m = 0, p = 0, smax = 0, nEL = 0, SL = 0, ninst = 1;
    int n_cone = 0;               // non-PSD cone variables (last n_cone entries and positions)
    long long vstore_elems = 0;   // sum over cliques of N_k^2
    long long nnz = 0;
    // host copies needed after setup
    std::vector<int> pat_row, pat_col, blk_off, gather_idx;
    std::vector<int> inst_vtx, inst_row, inst_cl, inst_e, inst_pos;
    std::vector<int> order_h, blk_size_h;   // for rebuilding the projection plans
    int ow_min_blocks = 0;
    std::vector<int> proj_table[2];         // per precision: variant by padded order (empty = defaults)
    // What the work schedules are built from, kept so that a batch can be re-planned for the
    // problems still iterating (frozen problems then get no CTAs at all).
    struct SchedSource {
        int ninst = 1, m = 0, SL = 0, num_sms = 0;
        long long nnz = 0;
        std::vector<int> inst_row, inst_e, inst_pos, inst_sl, inst_cl, a_rowptr, sell_len, heavy;
        std::vector<long long> inst_nnz;
    } src;
    int planned = 0;                        // problems the current schedules cover
    size_t row_cap = 0, col_cap = 0;        // capacity of the CSR-chunk and A^T-chunk partial sums
    // Unrolled iterations kept for reverse mode (sdp_unrolled_forward / _backward).
    struct Adjoint {
        int T = 0, K = 0, nseg = 0, n_large = 0;
        bool valid = false;
        size_t cap_ckpt = 0, cap_seg = 0;   // doubles held by ckpt, and by Wseg + Vseg
        double* ckpt = nullptr;             // nseg x [x_k (S_L), lambda_k (S_L)]
        double* Wseg = nullptr;             // K x S_L: W_k of each iteration of a segment
        double* Vseg = nullptr;             // K x (sum N_k^2): their eigenvectors
        double *lam_prev = nullptr, *Xb = nullptr, *Lb = nullptr, *ub = nullptr;
        double *cbar = nullptr, *bbar = nullptr;
        // vectors of the adjoint KKT solve, swapped into a copy of the forward's pointers
        double *xbar = nullptr, *rsw = nullptr, *rbar = nullptr, *ybar = nullptr;
        double *tpart = nullptr, *pobj = nullptr;
        int* conv = nullptr;
        cadmm::Ctrl* ctrl = nullptr;
        std::vector<void*> seg_allocs;
    } adj;
    cadmm::ProjPlan plan[2]{};    // projection launches per precision (SDP_PROJ_FP64, SDP_PROJ_FP32)
    std::vector<void*> allocs;
    IterPtrs P{};
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t g_one = nullptr, g_chunk = nullptr;
    int chunk = 0, g_form = -1, g_prec = -1;
    double g_rho = 0.0;
    Ctrl* h_ctrl = nullptr;    // pinned, two slots
    cudaEvent_t ev[2] = {nullptr, nullptr};

    // Device arrays live as long as the handle, so small ones are carved (256-byte aligned) from
    // chunks of kChunkBytes and large ones get an allocation each: a setup makes a few dozen
    // cudaMalloc calls fewer, and sdp_free as many cudaFree calls fewer.
    static constexpr size_t kChunkBytes = size_t(4) << 20;
    char* chunk_next = nullptr;
    size_t chunk_left = 0;
    template <typename T>
    int dalloc(T** ptr, size_t count) {
        const size_t bytes = (std::max<size_t>(count, 1) * sizeof(T) + 255) & ~size_t(255);
        if (bytes > chunk_left) {
            const bool own = bytes * 4 > kChunkBytes;     // a large array: an allocation of its own
            const size_t sz = own ? bytes : kChunkBytes;
            void* p_ = nullptr;
            const cudaError_t e = cudaMalloc(&p_, sz);
            if (e != cudaSuccess) return set_err(SDP_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
            allocs.push_back(p_);
            if (own) {
                *ptr = static_cast<T*>(p_);
                return SDP_OK;
            }
            chunk_next = static_cast<char*>(p_);
            chunk_left = sz;
        }
        *ptr = reinterpret_cast<T*>(chunk_next);
        chunk_next += bytes;
        chunk_left -= bytes;
        return SDP_OK;
    }
    template <typename T, typename Alloc>
    int upload(T** ptr, const std::vector<T, Alloc>& v, size_t capacity = 0) {
        int rc = dalloc(ptr, std::max(v.size(), capacity));
        if (rc) return rc;
        if (!v.empty()) {
            const cudaError_t e = cudaMemcpy(*ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return set_err(SDP_ERR_CUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
        }
        return SDP_OK;
    }
    void destroy_graphs() {
        if (g_one) cudaGraphExecDestroy(g_one);
        if (g_chunk) cudaGraphExecDestroy(g_chunk);
        g_one = g_chunk = nullptr;
        g_form = g_prec = -1;
    }
    ~sdp_ctx() {
        cudaSetDevice(device);
        destroy_graphs();
        for (void* a : adj.seg_allocs) cudaFree(a);
        for (void* a : allocs) cudaFree(a);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
        if (h_ctrl) cudaFreeHost(h_ctrl);
    }
};

namespace {

int plan_all(sdp_ctx* h);
int maybe_replan(sdp_ctx* h, cudaStream_t st, bool* done);

int capture_graph(sdp_ctx* h, int iters, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaSuccess;
    for (int i = 0; i < iters && le == cudaSuccess; ++i)
        le = cadmm::launch_iteration(h->P, h->plan[h->opts.prec], h->opts.form, h->opts.prec, h->opts.rho,
                                     h->cap_stream);
    const cudaError_t ee = cudaStreamEndCapture(h->cap_stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return set_err(SDP_ERR_CUDA, std::string("kernel launch during capture: ") + cudaGetErrorString(le));
    }
    if (ee != cudaSuccess) return set_err(SDP_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ee));
    const cudaError_t ie = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return set_err(SDP_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
    return SDP_OK;
}

int ensure_graphs(sdp_ctx* h) {
    const int chunk = h->opts.check_every > 0 ? h->opts.check_every : 16;
    if (h->g_one && h->g_form == h->opts.form && h->g_prec == h->opts.prec && h->g_rho == h->opts.rho &&
        h->chunk == chunk)
        return SDP_OK;
    h->destroy_graphs();
    int rc = capture_graph(h, 1, &h->g_one);
    if (rc) return rc;
    rc = capture_graph(h, chunk, &h->g_chunk);
    if (rc) return rc;
    h->chunk = chunk;
    h->g_form = h->opts.form;
    h->g_prec = h->opts.prec;
    h->g_rho = h->opts.rho;
    return SDP_OK;
}

int sync_ctrl(sdp_ctx* h, cudaStream_t st, Ctrl* dst) {
    CK(cudaMemcpyAsync(dst, h->P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(h->ev[0], st));
    return wait_event(h->ev[0], kWaitTimeoutSeconds);
}

// Recompute the primal right-hand side r from the current blocks (needed after a reset, a state
// upload or a change of rho). Clears a stop flag left by a finished solve first, since every
// kernel skips its work while the flag is set.
int rebuild_r_if_primal(sdp_ctx* h, cudaStream_t st) {
    if (h->opts.form != SDP_PRIMAL) return SDP_OK;
    CK(cadmm::launch_ctrl_clear(h->P.ctrl, st));
    CK(cadmm::launch_primal_rebuild_r(h->P, h->opts.rho, st));
    return SDP_OK;
}

// Every problem of a batch iterates again (after a reset, a state upload or new options).
int unfreeze(sdp_ctx* h, cudaStream_t st) {
    CK(cadmm::launch_inst_reset(h->P, st));
    return plan_all(h);
}

int run_iterations(sdp_ctx* h, int n_iters, cudaStream_t st, admm_result* out) {
    const double t0 = now_s();
    int rc = ensure_graphs(h);
    if (rc) return rc;
    CK(cadmm::launch_ctrl_arm(h->P.ctrl, n_iters, h->opts.tol, st));
    int remaining = n_iters;
    int slot = 0, launched_chunks = 0;
    bool stop = false;
    long long launched_iters = 0;
    // Chunks of `chunk` iterations; after each chunk the stop flag is copied back, and the host
    // reads the previous chunk's flag while the current chunk runs.
    while (remaining >= h->chunk && !stop) {
        CK(cudaGraphLaunch(h->g_chunk, st));
        remaining -= h->chunk;
        launched_iters += h->chunk;
        CK(cudaMemcpyAsync(&h->h_ctrl[slot], h->P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
        CK(cudaEventRecord(h->ev[slot], st));
        if (launched_chunks > 0) {
            rc = wait_event(h->ev[slot ^ 1], kWaitTimeoutSeconds);
            if (rc) return rc;
            if (h->h_ctrl[slot ^ 1].done) stop = true;
            else if (h->ninst > 1 && h->h_ctrl[slot ^ 1].active > 0 && 2 * h->h_ctrl[slot ^ 1].active <= h->planned) {
                bool done = false;
                if ((rc = maybe_replan(h, st, &done))) return rc;
                if ((rc = ensure_graphs(h))) return rc;
                if (done) stop = true;
                launched_chunks = -1;         // the pipeline restarts after the synchronization
            }
        }
        ++launched_chunks;
        slot ^= 1;
    }
    while (remaining > 0 && !stop) {
        CK(cudaGraphLaunch(h->g_one, st));
        --remaining;
        ++launched_iters;
    }
    Ctrl c{};
    rc = sync_ctrl(h, st, &c);
    if (rc) return rc;
    if (out) {
        out->iters = c.iter;
        out->status = c.status;
        out->eps_p = c.eps_p;
        out->eps_d = c.eps_d;
        out->obj_primal = c.obj_p;
        out->obj_dual = c.obj_d;
        out->seconds = now_s() - t0;
        out->kernel_launches =
            1 + launched_iters * cadmm::iteration_kernel_count(h->P, h->plan[h->opts.prec], h->opts.form);
    }
    if (c.status == SDP_ERR_NAN) set_err(SDP_ERR_NAN, "a residual or objective became NaN/Inf");
    return c.status;
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Work schedules. No CTA (or, for the passes over A, no warp chunk) spans two problems; within a
// problem the ranges follow the element order.
struct Schedules {
    std::vector<cadmm::Sched> row, tri, col, pos, ent, heavy;
    std::vector<int> row_chunk, inst_col_chunk, inst_pos_cta, inst_ent_cta, inst_heavy_cta;
    bool col_split = false;
};


Schedules build_schedules(const sdp_ctx::SchedSource& hp, const std::vector<char>& act) {
    Schedules S;
    const int Q = hp.ninst, num_sms = hp.num_sms;
    int mmax = 1;
    long long nnz = 0, SL = 0, slices = 0;
    for (int q = 0; q < Q; ++q) {
        mmax = std::max(mmax, hp.inst_row[q + 1] - hp.inst_row[q]);
        if (!act[q]) continue;
        nnz += hp.inst_nnz[q];
        SL += hp.inst_pos[q + 1] - hp.inst_pos[q];
        slices += hp.inst_sl[q + 1] - hp.inst_sl[q];
    }
    // grids of whole waves: the CTAs each kernel can keep resident on an SM
    const long long rows_res = cadmm::resident_ctas(0, 0);
    const long long cols_res = cadmm::resident_ctas(1, (size_t)mmax * sizeof(double));
    const long long upd_res = cadmm::resident_ctas(2, 0);
    const long long nchunk = 8LL * rows_res * num_sms;
    // CSR: each row split into chunks of about nnz / nchunk nonzeros (at least 1024, at most 256
    // chunks per row); one warp per chunk.
    const long long rt = std::max<long long>(1024, (nnz + nchunk - 1) / nchunk);
    S.row_chunk.assign(hp.m + 1, 0);
    for (int q = 0; q < Q; ++q)
        for (int i = hp.inst_row[q]; i < hp.inst_row[q + 1]; ++i) {
            if (act[q]) {
                const int lo0 = hp.a_rowptr[i], hi0 = hp.a_rowptr[i + 1];
                const long long len = hi0 - lo0;
                const int R = (int)std::max<long long>(1, std::min<long long>(256, (len + rt - 1) / rt));
                for (int ch = 0; ch < R; ++ch)
                    S.row.push_back({q, lo0 + (int)(len * ch / R), lo0 + (int)(len * (ch + 1) / R), i});
            }
            S.row_chunk[i + 1] = (int)S.row.size();
        }
    // The M^-1 product (k_solve_y): 8 rows (one per warp) per CTA.
    for (int q = 0; q < Q; ++q)
        for (int r = hp.inst_row[q]; r < hp.inst_row[q + 1] && act[q]; r += 8)
            S.tri.push_back({q, r, std::min(r + 8, hp.inst_row[q + 1]), 0});
    // A^T: CTA chunks of whole slices with about nnz / (resident CTAs x SMs) stored elements (at
    // least 2048); the warps of a CTA take its slices in turn, one lane per column. With fewer
    // than 16 slices per SM in all, every slice gets a CTA of its own instead, whose warps split
    // the slice's length.
    const long long ct = std::max<long long>(2048, (nnz + cols_res * num_sms - 1) / (cols_res * num_sms));
    S.col_split = slices < 16LL * num_sms;
    S.inst_col_chunk.assign(Q + 1, 0);
    for (int q = 0; q < Q; ++q) {
        int sl = hp.inst_sl[q];
        const int s1 = act[q] ? hp.inst_sl[q + 1] : sl;
        if (S.col_split) {
            for (; sl < s1; ++sl) S.col.push_back({q, sl, sl + 1, 0});
        } else {
            while (sl < s1) {
                const int lo = sl;
                long long acc = 0;
                while (sl < s1 && (sl == lo || acc + 32LL * hp.sell_len[sl] <= ct)) {
                    acc += 32LL * hp.sell_len[sl];
                    ++sl;
                }
                S.col.push_back({q, lo, sl, 0});
            }
        }
        S.inst_col_chunk[q + 1] = (int)S.col.size();
    }
    // Light entries: 256 per CTA; heavy entries: 8 (one per warp) per CTA.
    // Packed positions per CTA of the dual update: about one wave of resident CTAs, 256..2048
    // (1..8 per thread) each.
    const int pos_per = (int)std::max<long long>(
        256, std::min<long long>(2048, (SL / (upd_res * num_sms) + 255) / 256 * 256));
    S.inst_pos_cta.assign(Q + 1, 0);
    S.inst_ent_cta.assign(Q + 1, 0);
    S.inst_heavy_cta.assign(Q + 1, 0);
    size_t h = 0;
    for (int q = 0; q < Q; ++q) {
        const size_t h0 = h;
        while (h < hp.heavy.size() && hp.heavy[h] < hp.inst_e[q + 1]) ++h;
        if (act[q]) {
            for (int lo = hp.inst_pos[q]; lo < hp.inst_pos[q + 1]; lo += pos_per)
                S.pos.push_back({q, lo, std::min(lo + pos_per, hp.inst_pos[q + 1]), 0});
            for (int lo = hp.inst_e[q]; lo < hp.inst_e[q + 1]; lo += 256)
                S.ent.push_back({q, lo, std::min(lo + 256, hp.inst_e[q + 1]), 0});
            for (size_t lo = h0; lo < h; lo += 8)
                S.heavy.push_back({q, (int)lo, (int)std::min(lo + 8, h), 0});
        }
        S.inst_pos_cta[q + 1] = (int)S.pos.size();
        S.inst_ent_cta[q + 1] = (int)S.ent.size();
        S.inst_heavy_cta[q + 1] = (int)S.heavy.size();
    }
    return S;
}

// Order of the cliques of the active problems, largest first (stable).
std::vector<int> active_order(const sdp_ctx* h, const std::vector<char>& act) {
    std::vector<int> order;
    order.reserve(h->order_h.size());
    const auto& cl = h->src.inst_cl;
    for (int k : h->order_h) {
        const int q = (int)(std::upper_bound(cl.begin(), cl.end(), k) - cl.begin()) - 1;
        if (act[q]) order.push_back(k);
    }
    return order;
}

template <typename T>
int copy_to(const T* dst, const std::vector<T>& v) {
    if (v.empty()) return SDP_OK;
    CK(cudaMemcpy(const_cast<T*>(dst), v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return SDP_OK;
}

// Point the iteration at the problems in `act`: schedules, clique order and projection plans.
// The device arrays were sized for all problems at setup, so any subset fits. The graphs hold the
// old launch shapes and are dropped (they are captured again at the next iteration call).
int apply_plan(sdp_ctx* h, const std::vector<char>& act) {
    const Schedules S = build_schedules(h->src, act);
    IterPtrs& P = h->P;
    int rc;
    if ((rc = copy_to(P.row_sched, S.row)) || (rc = copy_to(P.row_chunk, S.row_chunk)) ||
        (rc = copy_to(P.tri_sched, S.tri)) || (rc = copy_to(P.col_sched, S.col)) ||
        (rc = copy_to(P.pos_sched, S.pos)) || (rc = copy_to(P.ent_sched, S.ent)) ||
        (rc = copy_to(P.heavy_sched, S.heavy)) || (rc = copy_to(P.inst_col_chunk, S.inst_col_chunk)) ||
        (rc = copy_to(P.inst_pos_cta, S.inst_pos_cta)) || (rc = copy_to(P.inst_ent_cta, S.inst_ent_cta)) ||
        (rc = copy_to(P.inst_heavy_cta, S.inst_heavy_cta)))
        return rc;
    P.row_chunks = (int)S.row.size();
    P.tri_ctas = (int)S.tri.size();
    P.col_chunks = (int)S.col.size();
    P.col_split = S.col_split ? 1 : 0;
    P.pos_ctas = (int)S.pos.size();
    P.ent_ctas = (int)S.ent.size();
    P.heavy_ctas = (int)S.heavy.size();
    const std::vector<int> order = active_order(h, act);
    if ((rc = copy_to(P.order, order))) return rc;
    for (int prec = 0; prec < 2; ++prec)
        h->plan[prec] = cadmm::make_proj_plan(order, h->blk_size_h, prec,
                                              h->proj_table[prec].empty() ? nullptr : h->proj_table[prec].data(),
                                              h->ow_min_blocks);
    h->planned = 0;
    for (char a : act) h->planned += a ? 1 : 0;
    h->destroy_graphs();
    return SDP_OK;
}

int plan_all(sdp_ctx* h) {
    if (h->planned == h->ninst) return SDP_OK;
    return apply_plan(h, std::vector<char>(h->ninst, 1));
}

// Batches: once half of the problems the schedules cover have stopped, re-plan for the rest.
// Problems that stopped at the current iteration stay in (their primal blocks are copied to the
// other buffer by the next projection).
int maybe_replan(sdp_ctx* h, cudaStream_t st, bool* done) {
    CK(cudaStreamSynchronize(st));
    Ctrl c{};
    CK(cudaMemcpy(&c, h->P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
    *done = c.done != 0;
    if (c.done || c.active <= 0 || 2 * c.active > h->planned) return SDP_OK;
    std::vector<int> conv(h->ninst);
    CK(cudaMemcpy(conv.data(), h->P.inst_conv, sizeof(int) * h->ninst, cudaMemcpyDeviceToHost));
    std::vector<char> act(h->ninst);
    for (int q = 0; q < h->ninst; ++q) act[q] = conv[q] < 0 || conv[q] >= c.iter;
    return apply_plan(h, act);
}

// The batched projection on caller buffers: blocks largest first, one launch per run of blocks
// that share a kernel variant (variant < 0: the default for each size; else that variant for all).
int run_project_batched(const double* in, double* out, const int* sizes, const long long* offsets, int count,
                        int prec, int variant, void* cuda_stream) {
    if (count < 0) return set_err(SDP_ERR_ARG, "count must be >= 0");
    if (count == 0) return SDP_OK;
    if (!in || !out || !sizes || !offsets) return set_err(SDP_ERR_ARG, "NULL argument");
    if (prec != SDP_PROJ_FP64 && prec != SDP_PROJ_FP32) return set_err(SDP_ERR_ARG, "bad prec");
    int smax = 0;
    for (int k = 0; k < count; ++k) {
        if (sizes[k] < 1) return set_err(SDP_ERR_ARG, "block sizes must be >= 1");
        if (sizes[k] > SDP_MAX_CLIQUE) return set_err(SDP_ERR_UNSUPPORTED, "block larger than SDP_MAX_CLIQUE");
        if (offsets[k] < 0) return set_err(SDP_ERR_ARG, "offsets must be >= 0");
        smax = std::max(smax, sizes[k]);
    }
    if (variant >= 0 && !cadmm::project_variant_valid(variant, smax, prec))
        return set_err(SDP_ERR_UNSUPPORTED, "the variant does not take these blocks");
    std::vector<int> order(count);
    for (int k = 0; k < count; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sizes[a] > sizes[b]; });
    cudaStream_t st = as_stream(cuda_stream);
    // The schedule is copied from a host buffer that lives for this call only: a captured copy
    // would read it again at every replay, after it is gone. Capture is refused.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cap));
    if (cap != cudaStreamCaptureStatusNone)
        return set_err(SDP_ERR_UNSUPPORTED, "project_psd_batched cannot be captured in a CUDA graph");
    CK(cadmm::project_prepare());
    // One stream-ordered device buffer holds offsets, sizes and order.
    const size_t bytes = (size_t)count * (2 * sizeof(int) + sizeof(long long));
    std::vector<unsigned char> host(bytes);
    std::memcpy(host.data(), offsets, (size_t)count * sizeof(long long));
    std::memcpy(host.data() + (size_t)count * sizeof(long long), sizes, (size_t)count * sizeof(int));
    std::memcpy(host.data() + (size_t)count * (sizeof(long long) + sizeof(int)), order.data(),
                (size_t)count * sizeof(int));
    void* d = nullptr;
    CK(cudaMallocAsync(&d, bytes, st));
    cudaError_t e = cudaMemcpyAsync(d, host.data(), bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        cadmm::ProjArgs a{};
        a.off = static_cast<const long long*>(d);
        a.size = reinterpret_cast<const int*>(static_cast<unsigned char*>(d) + (size_t)count * sizeof(long long));
        const int* d_order = reinterpret_cast<const int*>(static_cast<unsigned char*>(d) +
                                                          (size_t)count * (sizeof(long long) + sizeof(int)));
        a.rho = 1.0;
        a.in = in;
        a.out = out;
        a.ctrl = nullptr;
        const std::vector<int> sz(sizes, sizes + count);
        cadmm::ProjPlan plan{};
        if (variant >= 0) {
            plan.runs = 1;
            plan.start[0] = 0;
            plan.count[0] = count;
            plan.variant[0] = variant;
            plan.smax[0] = smax;
        } else {
            int dev = 0, num_sms = 0;
            if (cudaGetDevice(&dev) == cudaSuccess &&
                cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
                plan = cadmm::make_proj_plan(order, sz, prec, nullptr, cadmm::proj_ow_min_blocks(num_sms));
            else
                plan = cadmm::make_proj_plan(order, sz, prec, nullptr, 0);
        }
        for (int r = 0; r < plan.runs && e == cudaSuccess; ++r) {
            a.order = d_order + plan.start[r];
            a.count = plan.count[r];
            e = cadmm::launch_project_variant(a, cadmm::PROJ_PLAIN, prec, plan.variant[r], plan.smax[r], st);
        }
    }
    // The pageable host copy above returns once the data is staged, so `host` may go away.
    const cudaError_t fe = cudaFreeAsync(d, st);
    if (e != cudaSuccess) return set_err(SDP_ERR_CUDA, std::string("project_psd_batched: ") + cudaGetErrorString(e));
    if (fe != cudaSuccess) return set_err(SDP_ERR_CUDA, std::string("cudaFreeAsync: ") + cudaGetErrorString(fe));
    return SDP_OK;
}

int create_handle(HostProblem& hp, const admm_opts* opts, sdp_handle* out, double host_ms) {
    SetupClock::time_point clk = SetupClock::now();
    sdp_ctx* h = new sdp_ctx();
    std::unique_ptr<sdp_ctx> guard(h);
    h->setup_ms[kSetupHost] = host_ms;
    CK(cudaGetDevice(&h->device));
    h->opts = *opts;
    h->n = hp.n; h->m = hp.m; h->p = hp.p; h->smax = hp.smax;
    h->nEL = hp.nEL; h->SL = hp.SL; h->nnz = hp.nnz; h->ninst = hp.ninst; h->n_cone = hp.n_cone;
    h->pat_row = hp.pat_row; h->pat_col = hp.pat_col;
    h->blk_off = hp.blk_off; h->gather_idx = hp.gather_idx;
    h->inst_vtx = hp.inst_vtx; h->inst_row = hp.inst_row; h->inst_cl = hp.inst_cl;
    h->inst_e = hp.inst_e; h->inst_pos = hp.inst_pos;
    h->order_h = hp.order;
    h->blk_size_h = hp.blk_size;
    CK(cadmm::project_prepare());
    CK(cadmm::iteration_prepare());
    CK(cadmm::adjoint_prepare());

    int num_sms = 0;
    CK(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, h->device));
    h->ow_min_blocks = cadmm::proj_ow_min_blocks(num_sms);
    h->plan[SDP_PROJ_FP64] = cadmm::make_proj_plan(hp.order, hp.blk_size, SDP_PROJ_FP64, nullptr, h->ow_min_blocks);
    h->plan[SDP_PROJ_FP32] = cadmm::make_proj_plan(hp.order, hp.blk_size, SDP_PROJ_FP32, nullptr, h->ow_min_blocks);
    {
        auto& sr = h->src;
        sr.ninst = hp.ninst;
        sr.m = hp.m;
        sr.SL = hp.SL;
        sr.nnz = hp.nnz;
        sr.num_sms = num_sms;
        sr.inst_row = hp.inst_row;
        sr.inst_e = hp.inst_e;
        sr.inst_pos = hp.inst_pos;
        sr.inst_sl = hp.inst_sl;
        sr.inst_cl = hp.inst_cl;
        sr.a_rowptr = hp.a_rowptr;
        sr.sell_len = hp.sell_len;
        sr.heavy = hp.heavy;
        sr.inst_nnz.resize(hp.ninst);
        for (int q = 0; q < hp.ninst; ++q)
            sr.inst_nnz[q] = (long long)hp.a_rowptr[hp.inst_row[q + 1]] - hp.a_rowptr[hp.inst_row[q]];
    }
    const Schedules S = build_schedules(h->src, std::vector<char>(hp.ninst, 1));
    h->planned = hp.ninst;
    h->setup_ms[kSetupPlan] = ms_since(clk);
    IterPtrs& P = h->P;
    P.n = hp.n; P.m = hp.m; P.p = hp.p; P.nEL = hp.nEL; P.SL = hp.SL; P.smax = hp.smax;
    P.ninst = hp.ninst;
    // Programmatic dependent launch hides part of each kernel's launch latency. On GB300 it paid
    // where the kernels are short (1.5e6 nonzeros of A, cliques of 30: 17.2 k -> 17.9 k FP32
    // iterations/s) and not where a pass over A takes half a millisecond (2e8 nonzeros: a batch
    // 0.8 % faster, a single problem 2 % slower).
    P.pdl = hp.nnz <= (1LL << 24) ? 1 : 0;
    P.mmax = 0;
    for (int q = 0; q < hp.ninst; ++q) P.mmax = std::max(P.mmax, hp.inst_row[q + 1] - hp.inst_row[q]);
    P.row_chunks = (int)S.row.size();
    P.tri_ctas = (int)S.tri.size();
    P.col_chunks = (int)S.col.size();
    P.col_split = S.col_split ? 1 : 0;
    P.pos_ctas = (int)S.pos.size();
    P.ent_ctas = (int)S.ent.size();
    P.heavy_ctas = (int)S.heavy.size();
    P.n_heavy = (int)hp.heavy.size();
    P.ncs = (int)hp.cone_lo.size();
    std::vector<int> blk_inst(hp.p);
    for (int q = 0; q < hp.ninst; ++q)
        for (int k = hp.inst_cl[q]; k < hp.inst_cl[q + 1]; ++k) blk_inst[k] = q;

    int rc;
    std::vector<long long> off64(hp.blk_off.begin(), hp.blk_off.end());
#define UP(field, vec)                                             \
    do {                                                           \
        auto* tmp_ = const_cast<std::remove_const_t<std::remove_pointer_t<decltype(P.field)>>*>(P.field); \
        rc = h->upload(&tmp_, vec);                                \
        if (rc) return rc;                                         \
        P.field = tmp_;                                            \
    } while (0)
    UP(inst_cl, hp.inst_cl);
    UP(inst_row, hp.inst_row);
    UP(mblk_off, hp.mblk_off);
    UP(blk_inst, blk_inst);
    // A^T slices, w/D and the CSR of A first: from them the device builds the slices' contents and
    // the KKT factorization (on a stream of its own) while the rest is uploaded
    UP(wdinv, hp.wdinv);
    UP(sell_col, hp.sell_col);
    UP(sell_len, hp.sell_len);
    UP(sell_off, hp.sell_off);
    UP(a_rowptr, hp.a_rowptr);
    UP(a_col, hp.a_col);
    UP(a_val, hp.a_val);
    const long long ell_size = hp.sell_off.empty() ? 0 : hp.sell_off.back();
    unsigned short* ell_row = nullptr;
    double* ell_val = nullptr;
    if (hp.kkt_on_device) {     // filled on the device from the CSR
        if ((rc = h->dalloc(&ell_row, (size_t)ell_size)) || (rc = h->dalloc(&ell_val, (size_t)ell_size))) return rc;
        P.sell_row = ell_row;
        P.sell_val = ell_val;
    } else {
        UP(sell_row, hp.sell_row);
        UP(sell_val, hp.sell_val);
    }
    cadmm::KktRun kkt_run;      // declared after guard: waits for its stream before h is freed
    cadmm::KktOutputs ko;
    if (hp.kkt_on_device) {
        cadmm::KktInputs ki;
        int* col_slot = nullptr;
        if ((rc = h->upload(&col_slot, hp.col_slot))) return rc;
        ki.m = hp.m;
        ki.nslices = (int)hp.sell_len.size();
        ki.sell_col = P.sell_col;
        ki.sell_len = P.sell_len;
        ki.sell_off = P.sell_off;
        ki.sell_row = P.sell_row;
        ki.sell_val = P.sell_val;
        ki.wdinv = P.wdinv;
        ki.slot_len_h.swap(hp.slot_len);
        ki.a_rowptr = P.a_rowptr;
        ki.a_col = P.a_col;
        ki.a_val = P.a_val;
        ki.nnz = hp.nnz;
        ki.nEL = hp.nEL;
        ki.col_slot = col_slot;
        ki.ell_row = ell_row;
        ki.ell_val = ell_val;
        ki.ell_size = ell_size;
        const size_t mm = (size_t)hp.m * hp.m;
        double *L = nullptr, *Li = nullptr, *LiT = nullptr, *Mi = nullptr;
        if ((rc = h->dalloc(&L, mm)) || (rc = h->dalloc(&Li, mm)) || (rc = h->dalloc(&LiT, mm)) ||
            (rc = h->dalloc(&Mi, mm)))
            return rc;
        ko.L = L;
        ko.Linv = Li;
        ko.LinvT = LiT;
        ko.Minv = Mi;
        std::string kerr;
        if ((rc = cadmm::device_kkt_launch(ki, ko, kkt_run, kerr))) return set_err(rc, kerr);
    }
    // Re-planning a batch for fewer problems splits their work more finely, so the schedules and
    // partial sums are sized for the finest split any subset can get (chunks of at least 1024
    // nonzeros per row, one slice per A^T chunk, 256 positions per update CTA).
    size_t row_cap = 0, pos_cap = 0;
    const size_t col_cap = (size_t)hp.inst_sl[hp.ninst];
    for (int i = 0; i < hp.m; ++i) {
        const long long len = hp.a_rowptr[i + 1] - hp.a_rowptr[i];
        row_cap += (size_t)std::max<long long>(1, std::min<long long>(256, (len + 1023) / 1024));
    }
    for (int q = 0; q < hp.ninst; ++q) pos_cap += (size_t)(hp.inst_pos[q + 1] - hp.inst_pos[q] + 255) / 256;
    row_cap = std::max(row_cap, S.row.size());
    pos_cap = std::max(pos_cap, S.pos.size());
    h->row_cap = row_cap;
    h->col_cap = std::max(col_cap, S.col.size());
#define UPC(field, vec, cap)                                       \
    do {                                                           \
        auto* tmp_ = const_cast<std::remove_const_t<std::remove_pointer_t<decltype(P.field)>>*>(P.field); \
        rc = h->upload(&tmp_, vec, cap);                           \
        if (rc) return rc;                                         \
        P.field = tmp_;                                            \
    } while (0)
    UPC(row_sched, S.row, row_cap);
    UP(row_chunk, S.row_chunk);
    UP(tri_sched, S.tri);
    UPC(col_sched, S.col, std::max(col_cap, S.col.size()));
    UPC(pos_sched, S.pos, pos_cap);
#undef UPC
    UP(ent_sched, S.ent);
    UP(heavy_sched, S.heavy);
    UP(inst_col_chunk, S.inst_col_chunk);
    UP(inst_pos_cta, S.inst_pos_cta);
    UP(inst_ent_cta, S.inst_ent_cta);
    UP(inst_heavy_cta, S.inst_heavy_cta);
    UP(blk_off, hp.blk_off);
    UP(blk_off64, off64);
    UP(blk_size, hp.blk_size);
    UP(voff, hp.voff);
    UP(order, hp.order);
    UP(gather_idx, hp.gather_idx);
    UP(pos_w, hp.pos_w);
    UP(sc_ptr, hp.sc_ptr);
    UP(sc_pos, hp.sc_pos);
    UP(heavy, hp.heavy);
    UP(D, hp.D);
    UP(dinv, hp.dinv);
    UP(c, hp.c);
    UP(b, hp.b);
    UP(ew, hp.ew);
    if (hp.kkt_on_device) {
        std::string kerr;
        h->setup_ms[kSetupUpload] += ms_since(clk);
        if ((rc = cadmm::device_kkt_wait(kkt_run, ko, kerr))) return set_err(rc, kerr);
        h->setup_ms[kSetupKkt] = ms_since(clk);
        P.kkt_tri = ko.kappa1 > cadmm::kKktTriCond ? 1 : 0;
        P.Minv = ko.Minv;
        P.Linv = ko.Linv;
        P.LinvT = ko.LinvT;
        if (P.kkt_tri && (rc = h->dalloc(&P.z1, (size_t)std::max(1, hp.m)))) return rc;
    } else {
        P.kkt_tri = hp.kkt_tri ? 1 : 0;
        if (hp.kkt_tri) {
            UP(Linv, hp.Linv);
            UP(LinvT, hp.LinvT);
            if ((rc = h->dalloc(&P.z1, (size_t)std::max(1, hp.m)))) return rc;
        } else {
            UP(Minv, hp.Minv);
        }
    }
    UP(cone_lo, hp.cone_lo);
    UP(cone_hi, hp.cone_hi);
    UP(cone_kind, hp.cone_kind);
    UP(soc_pos, hp.soc_pos);
    UP(soc_q, hp.soc_q);
#undef UP
    if ((rc = h->dalloc(&P.inst_res, (size_t)hp.ninst * 4))) return rc;
    if ((rc = h->dalloc(&P.inst_conv, (size_t)hp.ninst))) return rc;
    if ((rc = h->dalloc(&P.inst_stat, (size_t)hp.ninst))) return rc;
    if ((rc = h->dalloc(&P.x, hp.nEL))) return rc;
    if ((rc = h->dalloc(&P.y, hp.m))) return rc;
    if ((rc = h->dalloc(&P.r, hp.nEL))) return rc;
    if ((rc = h->dalloc(&P.rsw, hp.nEL))) return rc;
    if ((rc = h->dalloc(&P.xk[0], hp.SL))) return rc;
    if ((rc = h->dalloc(&P.xk[1], hp.SL))) return rc;
    if ((rc = h->dalloc(&P.lam, hp.SL))) return rc;
    if ((rc = h->dalloc(&P.vk, hp.SL))) return rc;
    if ((rc = h->dalloc(&P.tpart, row_cap))) return rc;
    if ((rc = h->dalloc(&P.part_blk, ((size_t)hp.p + P.ncs) * 4))) return rc;
    if ((rc = h->dalloc(&P.part_ent, std::max<size_t>(P.ent_ctas + P.heavy_ctas, pos_cap) * 8))) return rc;
    if ((rc = h->dalloc(&P.part_obj, std::max(col_cap, S.col.size())))) return rc;
    if ((rc = h->dalloc(&P.ctrl, 1))) return rc;
    {
        double* vs = nullptr;       // sized for FP64; FP32 blocks use the first half
        if ((rc = h->dalloc(&vs, (size_t)hp.voff[hp.p]))) return rc;
        P.vstore = vs;
        h->vstore_elems = hp.voff[hp.p];
    }
    h->setup_ms[kSetupUpload] += ms_since(clk);
    CK(cudaMallocHost(&h->h_ctrl, 2 * sizeof(Ctrl)));
    CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->ev[0], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->ev[1], cudaEventDisableTiming));
    guard.release();
    *out = h;
    rc = admm_reset(h, nullptr);
    if (rc) {
        delete h;
        *out = nullptr;
        return rc;
    }
    CK(cudaDeviceSynchronize());
    h->setup_ms[kSetupFinish] = ms_since(clk);
    return SDP_OK;
}

}  // namespace

extern "C" {

int sdp_setup(int n, int m, const long long* A_ptr, const int* A_row, const int* A_col,
              const double* A_val, const double* b, long long C_nnz, const int* C_row,
              const int* C_col, const double* C_val, long long pat_nnz, const int* pat_row,
              const int* pat_col, int p, const int* clique_ptr, const int* clique_vtx,
              const admm_opts* opts, sdp_handle* out) {
    try {
        if (!out) return set_err(SDP_ERR_ARG, "out is NULL");
        *out = nullptr;
        int rc = check_opts(opts);
        if (rc) return rc;
        SetupClock::time_point clk = SetupClock::now();
        HostProblem hp;
        std::string err;
        rc = cadmm::build_host_problem(n, m, A_ptr, A_row, A_col, A_val, b, C_nnz, C_row, C_col, C_val,
                                       pat_nnz, pat_row, pat_col, p, clique_ptr, clique_vtx, nullptr, hp, err,
                                       (opts->flags & SDP_FLAG_HOST_KKT) == 0);
        if (rc) return set_err(rc, err);
        return create_handle(hp, opts, out, ms_since(clk));
    } catch (const std::bad_alloc&) {
        return set_err(SDP_ERR_ARG, "host out of memory");
    } catch (...) {
        return set_err(SDP_ERR_ARG, "unexpected exception in sdp_setup");
    }
}

int sdp_setup_conic(const sdp_problem* pr, const sdp_cones* cones, const admm_opts* opts, sdp_handle* out) {
    try {
        if (!out) return set_err(SDP_ERR_ARG, "out is NULL");
        *out = nullptr;
        if (!pr) return set_err(SDP_ERR_ARG, "problem is NULL");
        int rc = check_opts(opts);
        if (rc) return rc;
        SetupClock::time_point clk = SetupClock::now();
        HostProblem hp;
        std::string err;
        rc = cadmm::build_host_problem(pr->n, pr->m, pr->A_ptr, pr->A_row, pr->A_col, pr->A_val, pr->b,
                                       pr->C_nnz, pr->C_row, pr->C_col, pr->C_val, pr->pat_nnz, pr->pat_row,
                                       pr->pat_col, pr->p, pr->clique_ptr, pr->clique_vtx, cones, hp, err,
                                       (opts->flags & SDP_FLAG_HOST_KKT) == 0);
        if (rc) return set_err(rc, err);
        return create_handle(hp, opts, out, ms_since(clk));
    } catch (const std::bad_alloc&) {
        return set_err(SDP_ERR_ARG, "host out of memory");
    } catch (...) {
        return set_err(SDP_ERR_ARG, "unexpected exception in sdp_setup_conic");
    }
}

int sdp_plan(const sdp_problem* pr, const sdp_cones* cones, sdp_sizes* out) {
    try {
        if (!pr || !out) return set_err(SDP_ERR_ARG, "NULL argument");
        HostProblem hp;
        std::string err;
        const int rc = cadmm::build_host_problem(pr->n, pr->m, pr->A_ptr, pr->A_row, pr->A_col, pr->A_val, pr->b,
                                                 pr->C_nnz, pr->C_row, pr->C_col, pr->C_val, pr->pat_nnz,
                                                 pr->pat_row, pr->pat_col, pr->p, pr->clique_ptr, pr->clique_vtx,
                                                 cones, hp, err);
        if (rc) return set_err(rc, err);
        out->n = hp.n;
        out->m = hp.m;
        out->p = hp.p;
        out->max_clique = hp.smax;
        out->nE_lower = hp.nEL;
        out->S_lower = hp.SL;
        out->nnz_A = hp.nnz;
        out->batch = 1;
        out->n_cone = hp.n_cone;
        return SDP_OK;
    } catch (const std::bad_alloc&) {
        return set_err(SDP_ERR_ARG, "host out of memory");
    } catch (...) {
        return set_err(SDP_ERR_ARG, "unexpected exception in sdp_plan");
    }
}

int sdp_setup_batch(int count, const sdp_problem* problems, const admm_opts* opts, sdp_handle* out) {
    try {
        if (!out) return set_err(SDP_ERR_ARG, "out is NULL");
        *out = nullptr;
        if (count < 1 || !problems) return set_err(SDP_ERR_ARG, "count must be >= 1 and problems non-NULL");
        int rc = check_opts(opts);
        if (rc) return rc;
        SetupClock::time_point clk = SetupClock::now();
        HostProblem hp;
        std::string err;
        rc = cadmm::build_host_problem_batch(count, problems, hp, err);
        if (rc) return set_err(rc, err);
        return create_handle(hp, opts, out, ms_since(clk));
    } catch (const std::bad_alloc&) {
        return set_err(SDP_ERR_ARG, "host out of memory");
    } catch (...) {
        return set_err(SDP_ERR_ARG, "unexpected exception in sdp_setup_batch");
    }
}

int sdp_batch_layout(sdp_handle h, int* vtx_off, int* row_off, int* clique_off, long long* ent_off,
                     long long* pos_off) {
    if (!h) return set_err(SDP_ERR_ARG, "NULL handle");
    for (int q = 0; q <= h->ninst; ++q) {
        if (vtx_off) vtx_off[q] = h->inst_vtx[q];
        if (row_off) row_off[q] = h->inst_row[q];
        if (clique_off) clique_off[q] = h->inst_cl[q];
        if (ent_off) ent_off[q] = h->inst_e[q];
        if (pos_off) pos_off[q] = h->inst_pos[q];
    }
    return SDP_OK;
}

int sdp_batch_results(sdp_handle h, int* iters, int* status, double* eps_p, double* eps_d,
                      double* obj_primal, double* obj_dual) {
    if (!h) return set_err(SDP_ERR_ARG, "NULL handle");
    CK(cudaSetDevice(h->device));
    CK(cudaDeviceSynchronize());
    const int q = h->ninst;
    Ctrl c{};
    std::vector<int> conv(q), stat(q);
    std::vector<double> res((size_t)q * 4);
    CK(cudaMemcpy(&c, h->P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(conv.data(), h->P.inst_conv, sizeof(int) * q, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(stat.data(), h->P.inst_stat, sizeof(int) * q, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(res.data(), h->P.inst_res, sizeof(double) * 4 * q, cudaMemcpyDeviceToHost));
    for (int k = 0; k < q; ++k) {
        if (iters) iters[k] = (h->ninst > 1 && conv[k] >= 0) ? conv[k] : c.iter;
        if (status) status[k] = stat[k];
        if (eps_p) eps_p[k] = res[k * 4 + 0];
        if (eps_d) eps_d[k] = res[k * 4 + 1];
        if (obj_primal) obj_primal[k] = res[k * 4 + 2];
        if (obj_dual) obj_dual[k] = res[k * 4 + 3];
    }
    return SDP_OK;
}

int sdp_chordal_cliques(int n, long long nnz, const int* row, const int* col, int* p, long long* nvtx,
                        long long* fill, int* clique_ptr, int* clique_vtx, int capacity_p,
                        long long capacity_vtx) {
    try {
        std::vector<int> cp, cv;
        long long f = 0;
        std::string err;
        const int rc = cadmm::chordal_cliques(n, nnz, row, col, cp, cv, f, err);
        if (rc) return set_err(rc, err);
        const int np = (int)cp.size() - 1;
        if (p) *p = np;
        if (nvtx) *nvtx = (long long)cv.size();
        if (fill) *fill = f;
        if (clique_ptr || clique_vtx) {
            if (!clique_ptr || !clique_vtx || capacity_p < np || capacity_vtx < (long long)cv.size())
                return set_err(SDP_ERR_ARG, "clique arrays too small (call with NULL arrays for the sizes)");
            std::copy(cp.begin(), cp.end(), clique_ptr);
            std::copy(cv.begin(), cv.end(), clique_vtx);
        }
        return SDP_OK;
    } catch (const std::bad_alloc&) {
        return set_err(SDP_ERR_ARG, "host out of memory");
    } catch (...) {
        return set_err(SDP_ERR_ARG, "unexpected exception in sdp_chordal_cliques");
    }
}

int sdp_set_opts(sdp_handle h, const admm_opts* opts) {
    if (!h) return set_err(SDP_ERR_ARG, "NULL handle");
    int rc = check_opts(opts);
    if (rc) return rc;
    CK(cudaSetDevice(h->device));
    const bool rebuild = opts->rho != h->opts.rho || opts->form != h->opts.form;
    const bool new_prec = opts->prec != h->opts.prec;
    h->opts = *opts;
    if (new_prec) CK(cadmm::launch_vstore_identity(h->P, h->opts.prec, nullptr));
    if (rebuild) {
        rc = rebuild_r_if_primal(h, nullptr);
        if (rc) return rc;
    }
    if ((rc = unfreeze(h, nullptr))) return rc;
    CK(cudaDeviceSynchronize());
    return SDP_OK;
}

int admm_reset(sdp_handle h, void* cuda_stream) {
    if (!h) return set_err(SDP_ERR_ARG, "NULL handle");
    CK(cudaSetDevice(h->device));
    cudaStream_t st = as_stream(cuda_stream);
    IterPtrs& P = h->P;
    CK(cudaMemsetAsync(P.x, 0, sizeof(double) * std::max(1, P.nEL), st));
    CK(cudaMemsetAsync(P.y, 0, sizeof(double) * P.m, st));
    CK(cudaMemsetAsync(P.r, 0, sizeof(double) * std::max(1, P.nEL), st));
    CK(cudaMemsetAsync(P.rsw, 0, sizeof(double) * std::max(1, P.nEL), st));
    for (int i = 0; i < 2; ++i) CK(cudaMemsetAsync(P.xk[i], 0, sizeof(double) * std::max(1, P.SL), st));
    CK(cudaMemsetAsync(P.lam, 0, sizeof(double) * std::max(1, P.SL), st));
    CK(cudaMemsetAsync(P.vk, 0, sizeof(double) * std::max(1, P.SL), st));
    CK(cadmm::launch_ctrl_reset(P.ctrl, st));
    CK(cadmm::launch_vstore_identity(P, h->opts.prec, st));
    int rc = unfreeze(h, st);
    if (rc) return rc;
    return rebuild_r_if_primal(h, st);
}

int admm_iterate(sdp_handle h, int n_iters, void* cuda_stream, admm_result* out) {
    if (!h) return set_err(SDP_ERR_ARG, "NULL handle");
    if (n_iters < 0) return set_err(SDP_ERR_ARG, "n_iters must be >= 0");
    CK(cudaSetDevice(h->device));
    try {
        return run_iterations(h, n_iters, as_stream(cuda_stream), out);
    } catch (...) {
        return set_err(SDP_ERR_ARG, "unexpected exception in admm_iterate");
    }
}

int admm_solve(sdp_handle h, void* cuda_stream, admm_result* out) {
    if (!h) return set_err(SDP_ERR_ARG, "NULL handle");
    return admm_iterate(h, h->opts.max_iter, cuda_stream, out);
}

int sdp_get_sizes(sdp_handle h, sdp_sizes* out) {
    if (!h || !out) return set_err(SDP_ERR_ARG, "NULL argument");
    out->n = h->n; out->m = h->m; out->p = h->p; out->max_clique = h->smax;
    out->nE_lower = h->nEL; out->S_lower = h->SL; out->nnz_A = h->nnz;
    out->batch = h->ninst;
    out->n_cone = h->n_cone;
    return SDP_OK;
}

int sdp_get_state(sdp_handle h, double* x, double* y, double* blk_a, double* blk_b, double* blk_c) {
    if (!h) return set_err(SDP_ERR_ARG, "NULL handle");
    CK(cudaSetDevice(h->device));
    CK(cudaDeviceSynchronize());
    Ctrl c{};
    CK(cudaMemcpy(&c, h->P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
    const IterPtrs& P = h->P;
    const size_t sl = sizeof(double) * P.SL;
    if (x) CK(cudaMemcpy(x, P.x, sizeof(double) * P.nEL, cudaMemcpyDeviceToHost));
    if (y) CK(cudaMemcpy(y, P.y, sizeof(double) * P.m, cudaMemcpyDeviceToHost));
    const double* a_src = h->opts.form == SDP_PRIMAL ? P.xk[c.iter & 1] : P.xk[0];
    if (blk_a) CK(cudaMemcpy(blk_a, a_src, sl, cudaMemcpyDeviceToHost));
    if (blk_b) CK(cudaMemcpy(blk_b, P.lam, sl, cudaMemcpyDeviceToHost));
    if (blk_c) CK(cudaMemcpy(blk_c, P.vk, sl, cudaMemcpyDeviceToHost));
    return SDP_OK;
}

int sdp_proj_sweeps(sdp_handle h, int* sweeps) {
    if (!h || !sweeps) return set_err(SDP_ERR_ARG, "NULL argument");
    CK(cudaSetDevice(h->device));
    CK(cudaDeviceSynchronize());
    std::vector<double> part((size_t)h->p * 4);
    if (h->p > 0) CK(cudaMemcpy(part.data(), h->P.part_blk, part.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int k = 0; k < h->p; ++k) sweeps[k] = (int)part[(size_t)k * 4 + 3];
    return SDP_OK;
}

int sdp_set_state(sdp_handle h, const double* x, const double* y, const double* blk_a,
                  const double* blk_b, const double* blk_c) {
    if (!h) return set_err(SDP_ERR_ARG, "NULL handle");
    CK(cudaSetDevice(h->device));
    CK(cudaDeviceSynchronize());
    Ctrl c{};
    CK(cudaMemcpy(&c, h->P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
    const IterPtrs& P = h->P;
    const size_t sl = sizeof(double) * P.SL;
    if (x) CK(cudaMemcpy(P.x, x, sizeof(double) * P.nEL, cudaMemcpyHostToDevice));
    if (y) CK(cudaMemcpy(P.y, y, sizeof(double) * P.m, cudaMemcpyHostToDevice));
    double* a_dst = h->opts.form == SDP_PRIMAL ? P.xk[c.iter & 1] : P.xk[0];
    if (blk_a) CK(cudaMemcpy(a_dst, blk_a, sl, cudaMemcpyHostToDevice));
    if (blk_b) CK(cudaMemcpy(P.lam, blk_b, sl, cudaMemcpyHostToDevice));
    if (blk_c) CK(cudaMemcpy(P.vk, blk_c, sl, cudaMemcpyHostToDevice));
    CK(cadmm::launch_vstore_identity(P, h->opts.prec, nullptr));
    int rc = unfreeze(h, nullptr);
    if (rc) return rc;
    rc = rebuild_r_if_primal(h, nullptr);
    if (rc) return rc;
    CK(cudaDeviceSynchronize());
    return SDP_OK;
}

int sdp_get_solution(sdp_handle h, double* X_lower, double* y, double* Z_lower) {
    if (!h) return set_err(SDP_ERR_ARG, "NULL handle");
    const int nEL = h->nEL, m = h->m, SL = h->SL;
    std::vector<double> x(nEL), ya(m), blk(SL);
    int rc = sdp_get_state(h, x.data(), ya.data(), nullptr, nullptr, nullptr);
    if (rc) return rc;
    const double rho = h->opts.rho;
    if (X_lower) {
        if (h->opts.form == SDP_PRIMAL) std::copy(x.begin(), x.end(), X_lower);
        else for (int e = 0; e < nEL; ++e) X_lower[e] = -rho * x[e];
    }
    if (y) {
        if (h->opts.form == SDP_PRIMAL) for (int i = 0; i < m; ++i) y[i] = -rho * ya[i];
        else std::copy(ya.begin(), ya.end(), y);
    }
    if (Z_lower) {
        // primal form: Z = sum_k H_k^T lambda_k; dual form: Z = sum_k H_k^T z_k
        double* d_out = nullptr;
        CK(cudaMalloc(&d_out, sizeof(double) * std::max(1, nEL)));
        const IterPtrs& P = h->P;
        Ctrl c{};
        cudaError_t e = cudaMemcpy(&c, P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost);
        const double* src = h->opts.form == SDP_PRIMAL ? P.lam : P.xk[0];
        if (e == cudaSuccess) e = cadmm::launch_scatter(P, src, d_out, nullptr);
        if (e == cudaSuccess) e = cudaMemcpy(Z_lower, d_out, sizeof(double) * nEL, cudaMemcpyDeviceToHost);
        cudaFree(d_out);
        if (e != cudaSuccess) return set_err(SDP_ERR_CUDA, std::string("sdp_get_solution: ") + cudaGetErrorString(e));
    }
    return SDP_OK;
}

int sdp_get_maps(sdp_handle h, int* pat_row, int* pat_col, long long* blk_off, int* gather_idx) {
    if (!h) return set_err(SDP_ERR_ARG, "NULL handle");
    if (pat_row) std::copy(h->pat_row.begin(), h->pat_row.end(), pat_row);
    if (pat_col) std::copy(h->pat_col.begin(), h->pat_col.end(), pat_col);
    if (blk_off) for (size_t k = 0; k < h->blk_off.size(); ++k) blk_off[k] = h->blk_off[k];
    if (gather_idx) std::copy(h->gather_idx.begin(), h->gather_idx.end(), gather_idx);
    return SDP_OK;
}

int sdp_gather(sdp_handle h, const double* x, double* blocks_out, void* cuda_stream) {
    if (!h || !x || !blocks_out) return set_err(SDP_ERR_ARG, "NULL argument");
    CK(cudaSetDevice(h->device));
    CK(cadmm::launch_gather(h->P, x, blocks_out, as_stream(cuda_stream)));
    return SDP_OK;
}

int sdp_scatter(sdp_handle h, const double* blocks, double* out, void* cuda_stream) {
    if (!h || !blocks || !out) return set_err(SDP_ERR_ARG, "NULL argument");
    CK(cudaSetDevice(h->device));
    CK(cadmm::launch_scatter(h->P, blocks, out, as_stream(cuda_stream)));
    return SDP_OK;
}

int project_psd_batched(const double* in, double* out, const int* sizes, const long long* offsets,
                        int count, int prec, void* cuda_stream) {
    return run_project_batched(in, out, sizes, offsets, count, prec, -1, cuda_stream);
}

int project_psd_batched_variant(const double* in, double* out, const int* sizes, const long long* offsets,
                                int count, int prec, int variant, void* cuda_stream) {
    if (variant < 0 || variant >= cadmm::PV_COUNT) return set_err(SDP_ERR_ARG, "no such variant");
    return run_project_batched(in, out, sizes, offsets, count, prec, variant, cuda_stream);
}

int project_variant_count(void) { return cadmm::PV_COUNT; }

const char* project_variant_name(int v) {
    static const char* names[cadmm::PV_COUNT] = {"os32", "os64", "ts16", "ts32", "ts64", "ts96",
                                                 "ow8", "ow16", "ow32", "ow64", "ws32", "ws64"};
    return (v >= 0 && v < cadmm::PV_COUNT) ? names[v] : nullptr;
}

int project_variant_fits(int v, int s, int prec) {
    if (s < 1 || s > SDP_MAX_CLIQUE) return 0;
    return cadmm::project_variant_valid(v, s, prec) ? 1 : 0;
}

int sdp_set_proj_table(sdp_handle h, int prec, const int* table, int len) {
    if (!h) return set_err(SDP_ERR_ARG, "NULL handle");
    if (prec != SDP_PROJ_FP64 && prec != SDP_PROJ_FP32) return set_err(SDP_ERR_ARG, "bad prec");
    if (table && (len < 0 || len > SDP_MAX_CLIQUE + 1)) return set_err(SDP_ERR_ARG, "len out of range");
    CK(cudaSetDevice(h->device));
    std::vector<int> t(SDP_MAX_CLIQUE + 2, -1);
    if (table)
        for (int i = 0; i < len; ++i) t[i] = table[i];
    if (table) h->proj_table[prec] = t;
    else h->proj_table[prec].clear();
    h->planned = 0;                       // re-plan every problem with the new table
    return plan_all(h);
}

int sdp_set_cost(sdp_handle h, const double* c_lower, void* cuda_stream) {
    if (!h || !c_lower) return set_err(SDP_ERR_ARG, "NULL argument");
    CK(cudaSetDevice(h->device));
    cudaStream_t st = as_stream(cuda_stream);
    CK(cudaMemcpyAsync(const_cast<double*>(h->P.c), c_lower, sizeof(double) * h->nEL, cudaMemcpyDeviceToDevice, st));
    h->adj.valid = false;
    return rebuild_r_if_primal(h, st);      // the primal right-hand side holds -c/rho
}

int sdp_set_rhs(sdp_handle h, const double* b, void* cuda_stream) {
    if (!h || !b) return set_err(SDP_ERR_ARG, "NULL argument");
    CK(cudaSetDevice(h->device));
    CK(cudaMemcpyAsync(const_cast<double*>(h->P.b), b, sizeof(double) * h->m, cudaMemcpyDeviceToDevice,
                       as_stream(cuda_stream)));
    h->adj.valid = false;
    return SDP_OK;
}

}  // extern "C"

namespace {

// Device memory for T unrolled iterations with checkpoints every K (reused when large enough).
int ensure_adjoint(sdp_ctx* h, int T, int K) {
    auto& A = h->adj;
    const size_t SL = (size_t)std::max(1, h->SL), VS = (size_t)std::max<long long>(1, h->vstore_elems);
    const int nseg = (T + K - 1) / K;
    const size_t need_ckpt = (size_t)nseg * 2 * SL, need_seg = (size_t)K * (SL + VS);
    if (A.Xb == nullptr) {
        int rc;
        if ((rc = h->dalloc(&A.lam_prev, SL)) || (rc = h->dalloc(&A.Xb, SL)) || (rc = h->dalloc(&A.Lb, SL)) ||
            (rc = h->dalloc(&A.ub, SL)) || (rc = h->dalloc(&A.cbar, h->nEL)) || (rc = h->dalloc(&A.bbar, h->m)) ||
            (rc = h->dalloc(&A.xbar, h->nEL)) || (rc = h->dalloc(&A.rsw, h->nEL)) ||
            (rc = h->dalloc(&A.rbar, h->nEL)) || (rc = h->dalloc(&A.ybar, h->m)) ||
            (rc = h->dalloc(&A.tpart, h->row_cap)) || (rc = h->dalloc(&A.pobj, h->col_cap)) ||
            (rc = h->dalloc(&A.conv, (size_t)h->ninst)) || (rc = h->dalloc(&A.ctrl, 1)))
            return rc;
        CK(cudaMemset(A.conv, 0xff, sizeof(int) * h->ninst));      // -1: no problem stopped
        CK(cudaMemset(A.ctrl, 0, sizeof(cadmm::Ctrl)));           // done = 0 for good
        A.n_large = 0;
        for (int s : h->blk_size_h) A.n_large += (s + (s & 1)) > 16;
    }
    if (need_ckpt > A.cap_ckpt || need_seg > A.cap_seg) {
        for (void* a : A.seg_allocs) cudaFree(a);
        A.seg_allocs.clear();
        A.ckpt = A.Wseg = A.Vseg = nullptr;
        A.cap_ckpt = A.cap_seg = 0;
        void* p1 = nullptr;
        void* p2 = nullptr;
        CK(cudaMalloc(&p1, need_ckpt * sizeof(double)));
        A.seg_allocs.push_back(p1);
        CK(cudaMalloc(&p2, need_seg * sizeof(double)));
        A.seg_allocs.push_back(p2);
        A.ckpt = static_cast<double*>(p1);
        A.Wseg = static_cast<double*>(p2);
        A.Vseg = A.Wseg + (size_t)K * SL;
        A.cap_ckpt = need_ckpt;
        A.cap_seg = need_seg;
    }
    A.Vseg = A.Wseg + (size_t)K * SL;
    A.T = T;
    A.K = K;
    A.nseg = nseg;
    return SDP_OK;
}

// The forward's pointers (current schedules) with the adjoint solve's vectors swapped in.
cadmm::IterPtrs adjoint_ptrs(const sdp_ctx* h) {
    const auto& A = h->adj;
    cadmm::IterPtrs AP = h->P;
    AP.r = A.xbar;
    AP.rsw = A.rsw;
    AP.x = A.rbar;
    AP.y = A.ybar;
    AP.tpart = A.tpart;
    AP.part_obj = A.pobj;
    AP.inst_conv = A.conv;
    AP.ctrl = A.ctrl;
    return AP;
}

}  // namespace

extern "C" {

int sdp_unrolled_forward(sdp_handle h, int T, int ckpt_every, double* x_out, void* cuda_stream) {
    if (!h) return set_err(SDP_ERR_ARG, "NULL handle");
    if (T < 1 || ckpt_every < 1) return set_err(SDP_ERR_ARG, "T and ckpt_every must be >= 1");
    if (h->opts.form != SDP_PRIMAL || h->opts.prec != SDP_PROJ_FP64)
        return set_err(SDP_ERR_ARG, "unrolled differentiation needs form SDP_PRIMAL and prec SDP_PROJ_FP64");
    if (h->smax > 32) return set_err(SDP_ERR_UNSUPPORTED, "unrolled differentiation takes cliques of order <= 32");
    CK(cudaSetDevice(h->device));
    cudaStream_t st = as_stream(cuda_stream);
    try {
        int rc = ensure_adjoint(h, T, ckpt_every);
        if (rc) return rc;
        auto& A = h->adj;
        A.valid = false;
        if ((rc = admm_reset(h, st))) return rc;
        const double tol = h->opts.tol;
        h->opts.tol = 0.0;                       // run exactly T iterations
        const size_t SL = h->SL;
        for (int seg = 0; seg < A.nseg && rc == SDP_OK; ++seg) {
            const int t0 = seg * A.K, n = std::min(A.K, T - t0);
            double* ck = A.ckpt + (size_t)seg * 2 * SL;
            cudaError_t e = cudaMemcpyAsync(ck, h->P.xk[t0 & 1], sizeof(double) * SL, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(ck + SL, h->P.lam, sizeof(double) * SL, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) {
                h->opts.tol = tol;
                return set_err(SDP_ERR_CUDA, std::string("checkpoint copy: ") + cudaGetErrorString(e));
            }
            admm_result res{};
            rc = run_iterations(h, n, st, &res);
            if (rc == SDP_MAX_ITER) rc = SDP_OK;
        }
        h->opts.tol = tol;
        if (rc) return rc;
        if (x_out) CK(cudaMemcpyAsync(x_out, h->P.x, sizeof(double) * h->nEL, cudaMemcpyDeviceToDevice, st));
        CK(cudaStreamSynchronize(st));
        A.valid = true;
        return SDP_OK;
    } catch (...) {
        return set_err(SDP_ERR_ARG, "unexpected exception in sdp_unrolled_forward");
    }
}

int sdp_unrolled_backward(sdp_handle h, const double* xbar, double* cbar, double* bbar, void* cuda_stream) {
    if (!h || !xbar || !cbar || !bbar) return set_err(SDP_ERR_ARG, "NULL argument");
    auto& A = h->adj;
    if (!A.valid) return set_err(SDP_ERR_ARG, "no sdp_unrolled_forward to differentiate (or data changed since)");
    if (h->opts.form != SDP_PRIMAL || h->opts.prec != SDP_PROJ_FP64)
        return set_err(SDP_ERR_ARG, "options changed since sdp_unrolled_forward");
    CK(cudaSetDevice(h->device));
    cudaStream_t st = as_stream(cuda_stream);
    const cadmm::IterPtrs& P = h->P;
    const cadmm::IterPtrs AP = adjoint_ptrs(h);
    const double rho = h->opts.rho, rinv = 1.0 / rho;
    const size_t SL = h->SL, VS = (size_t)h->vstore_elems;
    CK(cudaMemsetAsync(A.Xb, 0, sizeof(double) * std::max<size_t>(1, SL), st));
    CK(cudaMemsetAsync(A.Lb, 0, sizeof(double) * std::max<size_t>(1, SL), st));
    CK(cudaMemsetAsync(A.cbar, 0, sizeof(double) * h->nEL, st));
    CK(cudaMemsetAsync(A.bbar, 0, sizeof(double) * h->m, st));
    for (int seg = A.nseg - 1; seg >= 0; --seg) {
        const int t0 = seg * A.K, n = std::min(A.K, A.T - t0);
        // recompute the segment from its checkpoint, keeping W_k and the eigenvectors of each step
        const double* ck = A.ckpt + (size_t)seg * 2 * SL;
        CK(cadmm::launch_ctrl_set_iter(P.ctrl, t0, st));
        CK(cadmm::launch_ctrl_arm(P.ctrl, n, 0.0, st));
        CK(cudaMemcpyAsync(P.xk[t0 & 1], ck, sizeof(double) * SL, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(P.lam, ck + SL, sizeof(double) * SL, cudaMemcpyDeviceToDevice, st));
        CK(cadmm::launch_vstore_identity(P, SDP_PROJ_FP64, st));
        CK(cadmm::launch_inst_reset(P, st));
        CK(cadmm::launch_primal_rebuild_r(P, rho, st));
        for (int j = 0; j < n; ++j) {
            CK(cadmm::launch_copy(P.lam, A.lam_prev, (long long)SL, st));
            CK(cadmm::launch_iteration(P, h->plan[SDP_PROJ_FP64], SDP_PRIMAL, SDP_PROJ_FP64, rho, st));
            CK(cadmm::launch_form_w(P, A.lam_prev, rinv, A.Wseg + (size_t)j * SL, st));
            CK(cadmm::launch_copy(static_cast<const double*>(P.vstore), A.Vseg + (size_t)j * VS, (long long)VS, st));
        }
        // reverse through the segment
        for (int j = n - 1; j >= 0; --j) {
            const int t = t0 + j + 1;
            CK(cadmm::launch_dk_vjp(P, A.n_large, A.Wseg + (size_t)j * SL, A.Vseg + (size_t)j * VS, A.Xb, A.Lb,
                                    A.ub, rho, st));
            CK(cadmm::launch_adj_scatter(P, A.ub, t == A.T ? xbar : nullptr, AP.r, AP.rsw, st));
            CK(cadmm::launch_kkt_adjoint(AP, st));
            CK(cadmm::launch_adj_accum(P, AP.x, AP.y, A.cbar, A.bbar, A.Xb, A.Lb, rinv, st));
        }
    }
    CK(cadmm::launch_adj_finish(P, A.cbar, A.bbar, cbar, bbar, st));
    CK(cudaStreamSynchronize(st));
    return SDP_OK;
}

int sdp_time_phases(sdp_handle h, int reps, void* cuda_stream, double* ms_out, int max_out) {
    if (!h || reps < 1 || !ms_out) return set_err(SDP_ERR_ARG, "bad argument");
    const int count = cadmm::phase_count(h->P, h->opts.form);
    if (max_out < count) return set_err(SDP_ERR_ARG, "ms_out too small");
    CK(cudaSetDevice(h->device));
    cudaStream_t st = as_stream(cuda_stream);
    // Every repetition is queued before the device reaches it: one untimed iteration first, then
    // the timed ones with no host synchronization between them, so that an event pair brackets
    // the device's work and not the host's time to submit the launch after an idle stream.
    const size_t per = (size_t)count + 1;
    std::vector<cudaEvent_t> ev(per * (size_t)reps, nullptr);
    cudaError_t ce = cudaSuccess;
    for (size_t i = 0; i < ev.size() && ce == cudaSuccess; ++i) ce = cudaEventCreate(&ev[i]);
    std::vector<double> acc(count, 0.0);
    if (ce == cudaSuccess) ce = cadmm::launch_ctrl_arm(h->P.ctrl, reps + 1, 0.0, st);
    if (ce == cudaSuccess)
        ce = cadmm::launch_iteration(h->P, h->plan[h->opts.prec], h->opts.form, h->opts.prec, h->opts.rho, st);
    for (int r = 0; r < reps && ce == cudaSuccess; ++r)
        ce = cadmm::launch_iteration(h->P, h->plan[h->opts.prec], h->opts.form, h->opts.prec, h->opts.rho, st,
                                     ev.data() + per * (size_t)r);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    for (int r = 0; r < reps && ce == cudaSuccess; ++r)
        for (int i = 0; i < count && ce == cudaSuccess; ++i) {
            float ms = 0.f;
            ce = cudaEventElapsedTime(&ms, ev[per * r + i], ev[per * r + i + 1]);
            acc[i] += ms;
        }
    for (auto& e : ev)
        if (e != nullptr) cudaEventDestroy(e);
    if (ce != cudaSuccess) return set_err(SDP_ERR_CUDA, std::string("sdp_time_phases: ") + cudaGetErrorString(ce));
    for (int i = 0; i < count; ++i) ms_out[i] = acc[i] / reps;
    return count;
}

const char* sdp_phase_name(sdp_handle h, int i) {
    if (!h) return nullptr;
    return cadmm::phase_name(h->opts.form, h->ninst > 1, h->P.ncs > 0, h->P.kkt_tri != 0, i);
}

int sdp_setup_times(sdp_handle h, double* ms_out, int max_out) {
    if (!h) return set_err(SDP_ERR_ARG, "handle is NULL");
    if (max_out < 0 || (max_out > 0 && !ms_out)) return set_err(SDP_ERR_ARG, "ms_out is NULL");
    const int k = std::min<int>(max_out, kSetupStages);
    for (int i = 0; i < k; ++i) ms_out[i] = h->setup_ms[i];
    return kSetupStages;
}

const char* sdp_setup_stage_name(int i) { return (i >= 0 && i < kSetupStages) ? kSetupStageName[i] : nullptr; }

void sdp_free(sdp_handle h) { delete h; }

const char* sdp_status_string(int status) {
    switch (status) {
        case SDP_OK: return "converged / success";
        case SDP_MAX_ITER: return "iteration budget reached without convergence";
        case SDP_ERR_ARG: return "bad argument";
        case SDP_ERR_CLIQUE: return "cliques unsorted or not covering a data nonzero";
        case SDP_ERR_NOT_PD: return "A D^-1 A^T not positive definite (A rank-deficient)";
        case SDP_ERR_CUDA: return "CUDA error";
        case SDP_ERR_NAN: return "NaN/Inf in residuals or objective";
        case SDP_ERR_TIMEOUT: return "timed out waiting for the device";
        case SDP_ERR_UNSUPPORTED: return "size beyond the supported limits";
        default: return "unknown status";
    }
}

const char* sdp_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
