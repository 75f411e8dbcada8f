// project_psd_batched_noalloc: the batched PSD projection for callers that must not allocate
// device memory. It runs the same kernels as project_psd_batched, but the per-call block schedule
// (each block's offset and size) lives in a fixed array compiled into this library instead of a
// buffer allocated per call.
//
// Who needs it: code that runs inside a host framework which owns every byte of device memory (an
// arena or pool sized up front, so a stray cudaMalloc would fail or fragment it), and latency-bound
// loops in which a cudaMalloc, which may synchronize the whole device, is not acceptable.
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "sdp_internal.h"

namespace {

// The schedule: offsets (int64) for up to SDP_NOALLOC_MAX_BLOCKS blocks, then their sizes (int32).
// Every GPU that loads the library holds these 384 KiB until the process exits.
constexpr size_t kSchedBytes = (size_t)SDP_NOALLOC_MAX_BLOCKS * (sizeof(long long) + sizeof(int));
static __device__ __align__(256) unsigned char g_noalloc_sched[kSchedBytes];

// Host-side view: the symbol above is only a host stand-in, so its device address is looked up
// with the device current and cached here. Every call looks it up again (a table lookup in the
// runtime, no device work) and repeats the set-up when it has changed, which happens when the
// device's context was destroyed (cudaDeviceReset) and a new one created.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_sched_dev[kMaxDevices] = {};

// Host staging copy of the caller's schedule: the caller's arrays may be pinned, and a copy from
// pinned memory runs asynchronously, so they are first copied here (pageable memory: the copy
// below returns once the runtime has staged it, and this buffer may be reused at once). Host
// memory only, one buffer per calling thread.
thread_local std::vector<unsigned char> t_stage;

// Errors go to the same per-thread message that sdp_last_error() reports.
int fail(int code, const std::string& msg) { return cadmm::record_error(code, msg); }

}  // namespace

extern "C" int project_psd_batched_noalloc(const double* in, double* out, const int* sizes,
                                           const long long* offsets, int count, int prec,
                                           void* cuda_stream) {
    if (count < 0) return fail(SDP_ERR_ARG, "count must be >= 0");
    if (count > SDP_NOALLOC_MAX_BLOCKS)
        return fail(SDP_ERR_UNSUPPORTED, "count exceeds SDP_NOALLOC_MAX_BLOCKS (" +
                                             std::to_string(SDP_NOALLOC_MAX_BLOCKS) + ")");
    if (count == 0) return SDP_OK;
    if (!in || !out || !sizes || !offsets) return fail(SDP_ERR_ARG, "NULL argument");
    if (prec != SDP_PROJ_FP64 && prec != SDP_PROJ_FP32) return fail(SDP_ERR_ARG, "bad prec");
    int smax = 0;
    for (int k = 0; k < count; ++k) {
        if (sizes[k] < 1) return fail(SDP_ERR_ARG, "block sizes must be >= 1");
        if (sizes[k] > SDP_MAX_CLIQUE) return fail(SDP_ERR_UNSUPPORTED, "block larger than SDP_MAX_CLIQUE");
        if (offsets[k] < 0) return fail(SDP_ERR_ARG, "offsets must be >= 0");
        if (sizes[k] > smax) smax = sizes[k];
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(SDP_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(SDP_ERR_UNSUPPORTED, "device index beyond 63");
    void* sched = nullptr;
    {
        // The array's device address in the current context. The first call on a device (and the
        // first after its context was reset) also raises the kernels' shared-memory limit; that
        // call must happen outside any stream capture.
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_sched);
        if (e != cudaSuccess)
            return fail(SDP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        std::lock_guard<std::mutex> lock(g_mu);
        if (g_sched_dev[dev] != ptr) {
            e = cadmm::project_prepare();
            if (e != cudaSuccess)
                return fail(SDP_ERR_CUDA, std::string("project_prepare: ") + cudaGetErrorString(e));
            g_sched_dev[dev] = ptr;
        }
        sched = ptr;
    }

    // The schedule goes into the shared array as [offsets (count) | sizes (count)], through the
    // host staging buffer, in one copy. Every entry the kernel reads is overwritten here, so
    // nothing in the array has to start at zero; a call that overlaps another one on the GPU
    // would overwrite its schedule.
    const size_t off_bytes = (size_t)count * sizeof(long long);
    const size_t bytes = off_bytes + (size_t)count * sizeof(int);
    if (t_stage.size() < bytes) t_stage.resize(bytes);
    std::memcpy(t_stage.data(), offsets, off_bytes);
    std::memcpy(t_stage.data() + off_bytes, sizes, (size_t)count * sizeof(int));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    unsigned char* base = static_cast<unsigned char*>(sched);
    long long* d_off = reinterpret_cast<long long*>(base);
    int* d_size = reinterpret_cast<int*>(base + off_bytes);
    e = cudaMemcpyAsync(base, t_stage.data(), bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(SDP_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));

    cadmm::ProjArgs a{};
    a.order = nullptr;          // blocks in the caller's order
    a.size = d_size;
    a.off = d_off;
    a.count = count;
    a.rho = 1.0;
    a.in = in;
    a.out = out;
    a.ctrl = nullptr;
    e = cadmm::launch_project(a, cadmm::PROJ_PLAIN, prec, smax, st);
    if (e != cudaSuccess) return fail(SDP_ERR_CUDA, std::string("project_psd_batched_noalloc: ") + cudaGetErrorString(e));
    return SDP_OK;
}
