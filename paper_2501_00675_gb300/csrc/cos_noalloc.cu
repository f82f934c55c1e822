// cos_evaluate_static: evaluation of an existing graph that allocates no device
// memory.  All scratch -- the control block (grid-barrier counter, error word,
// result), the partial sums of the sample reduction, the per-kind coefficients,
// and one tile's node-value slabs and propagator table -- lives in one file-scope
// __device__ array of COS_STATIC_SCRATCH_BYTES, which every GPU that loads this
// library holds until the process exits.  The graph structure and the 2^{j/64}
// table come from the graph handle, the times, energies and result buffer from the
// caller.
//
// Who needs it: callers that must not call cudaMalloc/cudaFree while they evaluate --
// a host framework whose own caching allocator owns the device memory budget (an
// allocation by this library would fail or fragment its pool), and latency-bound
// serving loops, where cudaMalloc and cudaFree can synchronise the device and
// stall other streams.  They create the graph once at set-up time, then evaluate
// with their own buffers.
//
// In host code, g_static_scratch names a host-side stand-in, not device memory:
// the kernel is given the device address that cudaGetSymbolAddress returns, looked
// up once per device (and again if the device's context changes).
#include <algorithm>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include <cstdint>
#include <cuda.h>

#include "cos_internal.cuh"

namespace cosgpu {
namespace {

static __device__ __align__(256) unsigned char g_static_scratch[COS_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
struct ScratchAddr {
    void* ctx;    // the context the address belongs to
    void* ptr;    // device address of g_static_scratch in that context
};
ScratchAddr g_scratch_addr[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);

// The current context (driver entry point reached through the runtime, so the
// library needs no link-time dependency on the driver library); nullptr if unknown.
void* current_context() {
    static CtxGetCurrentFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<CtxGetCurrentFn>(f);
    }();
    CUcontext c = nullptr;
    if (fn && fn(&c) == CUDA_SUCCESS) return c;
    return nullptr;
}

// Device address of the scratch array on `device`, which must be current.  Set-up,
// once per device: cudaGetSymbolAddress (which may load the module).  The address
// is kept together with the context it was taken in and looked up again when the
// device's context differs (after cudaDeviceReset, a new primary context may load
// the module elsewhere).
int scratch_address(int device, void** out) {
    if (device < 0 || device >= kMaxDevices) return set_error(COS_ERR_INVALID, "device ordinal %d not supported", device);
    void* ctx = current_context();
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    ScratchAddr& a = g_scratch_addr[device];
    if (!a.ptr || !ctx || a.ctx != ctx) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || !ptr) {
            a.ptr = nullptr;
            return set_error(COS_ERR_CUDA, "cudaGetSymbolAddress(static scratch) failed: %s", cudaGetErrorString(e));
        }
        a.ptr = ptr;
        a.ctx = ctx;
    }
    *out = a.ptr;
    return COS_OK;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace
}  // namespace cosgpu

using namespace cosgpu;

extern "C" int cos_evaluate_static(cos_graph_t g, int32_t mode, int64_t num_samples, const double* t, int64_t t_ld,
                                   const double* eps, double beta, void* per_sample_out, double* mean_out,
                                   void* stream) {
    GraphView gv;
    int rc = graph_view(g, &gv);
    if (rc != COS_OK) return rc;
    if (mode < 0 || mode > 2) return set_error(COS_ERR_INVALID, "bad mode %d", mode);
    if (num_samples < 0) return set_error(COS_ERR_INVALID, "num_samples must be >= 0");
    if (num_samples > 0 && (!t || !per_sample_out)) return set_error(COS_ERR_INVALID, "t and per_sample_out are required");
    if (!eps) return set_error(COS_ERR_INVALID, "eps is NULL");
    if (!(beta > 0.0)) return set_error(COS_ERR_INVALID, "beta must be positive");
    const int64_t S = num_samples;
    const int64_t need_ld = (S + 127) / 128 * 128;
    if (S > 0 && t_ld < need_ld)
        return set_error(COS_ERR_INVALID, "t_ld (%lld) must be >= num_samples rounded up to a multiple of 128 (%lld)",
                         (long long)t_ld, (long long)need_ld);
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != gv.device)
        return set_error(COS_ERR_INVALID, "the graph's device (%d) must be current", gv.device);
    void* base = nullptr;
    rc = scratch_address(gv.device, &base);
    if (rc != COS_OK) return rc;

    // Carve the static array: control block, partial sums, coefficients, then one tile's working set.
    const int vec = 1;                               // 32 samples per chunk: the smallest tile
    const int64_t ch = 32 * vec;
    const size_t val = (mode == COS_MODE_FP32_MIXED) ? 4 : 8;
    const int64_t nblk = (S + kReduceBlock - 1) / kReduceBlock;
    size_t off = 0;
    const size_t ctrl_at = off;
    off += align256(sizeof(Ctrl));
    const size_t part_at = off;
    off += align256(sizeof(double) * (size_t)(nblk > 0 ? nblk : 1));
    const size_t coef_at = off;
    off += align256(sizeof(double) * 2 * (size_t)gv.K);
    if (off > (size_t)COS_STATIC_SCRATCH_BYTES)
        return set_error(COS_ERR_INVALID, "num_samples %lld exceeds the static scratch limit", (long long)S);
    const size_t per_sample = 2 * val * (size_t)gv.Wmax +
                              (mode == COS_MODE_COUNT_I64 ? 0 : val * (size_t)gv.P);
    const size_t room = (size_t)COS_STATIC_SCRATCH_BYTES - off - 5 * 256;
    int64_t tile = (int64_t)(room / per_sample) / ch * ch;
    if (tile < ch)
        return set_error(COS_ERR_INVALID,
                         "graph too large for the %d MiB static scratch (needs %zu bytes per 32-sample chunk)",
                         (int)(COS_STATIC_SCRATCH_BYTES >> 20), per_sample * (size_t)ch);
    tile = std::min<int64_t>(tile, std::max<int64_t>(need_ld, ch));
    char* b = static_cast<char*>(base);
    WalkParams p;
    memset(&p, 0, sizeof(p));
    p.ctrl = reinterpret_cast<Ctrl*>(b + ctrl_at);
    p.partials = reinterpret_cast<double*>(b + part_at);
    p.coef = reinterpret_cast<double*>(b + coef_at);
    p.slab[0] = b + off;
    off += align256(val * gv.Wmax * tile);
    p.slab[1] = b + off;
    off += align256(val * gv.Wmax * tile);
    if (mode != COS_MODE_COUNT_I64) {
        p.gtab = b + off;
        off += align256(val * gv.P * tile);
    }
    if (off > (size_t)COS_STATIC_SCRATCH_BYTES) return set_error(COS_ERR_INVALID, "static scratch layout overflow");
    p.levels = gv.levels;
    p.row_ptr = gv.row_ptr;
    p.edges = gv.edges;
    p.slot_kij = gv.slot_kij;
    p.kind_slot = gv.kind_slot;
    p.exp_tab = gv.exp_tab;
    p.L = gv.L;
    p.P = gv.P;
    p.K = gv.K;
    p.D = gv.D;
    p.t = t;
    p.eps = eps;
    p.beta = beta;
    p.S = S;
    p.t_ld = t_ld;
    p.R = per_sample_out;
    p.tile = tile;
    p.rows_per_warp = 1;
    p.wmax = (int32_t)gv.Wmax;
    p.pf_slice_bytes = INT64_MAX;   // 32-sample chunks: every parent slice is small
    p.ptab = gv.ptab;
    p.ptab_T = gv.ptab_T;
    p.ptab_tau_max = gv.ptab_tau_max;
    p.ptab_inv_h = gv.ptab ? (double)gv.ptab_T / gv.ptab_tau_max : 0.0;
    p.timeout_ns = (long long)gv.timeout_ms * 1000000LL;
    // failure-detection test hook (as in cos_evaluate): CTA 0 leaves before this barrier
    if (const char* env = getenv("COS_TEST_SKIP_BARRIER_PHASE")) p.skip_barrier_phase = atoi(env);

    int per_sm = 0, sms = 0;
    const int dev_max = max_coresident_blocks(mode, vec, 1, gv.D, gv.device);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, gv.device);
    if (dev_max <= 0 || sms <= 0) return set_error(COS_ERR_CUDA, "cannot query occupancy");
    per_sm = dev_max / sms;
    cudaStream_t st = (cudaStream_t)stream;
    // The barrier counter and the result fields start at zero on every call.  The error
    // word and its detail are not cleared here: a failure of a call made without
    // mean_out stays recorded until a call with mean_out reports (and clears) it.
    static_assert(offsetof(Ctrl, err) == sizeof(unsigned long long) && offsetof(Ctrl, mean) == 16,
                  "control block layout");
    char* cb = reinterpret_cast<char*>(p.ctrl);
    cudaError_t e = cudaMemsetAsync(cb, 0, offsetof(Ctrl, err), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cb + offsetof(Ctrl, mean), 0, sizeof(Ctrl) - offsetof(Ctrl, mean), st);
    if (e != cudaSuccess) return set_error(COS_ERR_CUDA, "clear control block: %s", cudaGetErrorString(e));
    char msg[256] = {0};
    rc = launch_walk(mode, vec, 1, p, sms * per_sm, st, msg, sizeof(msg));
    if (rc != COS_OK) return set_error(rc, "walker launch failed: %s", msg);
    if (!mean_out) return COS_OK;
    Ctrl c;
    e = cudaMemcpyAsync(&c, p.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(COS_ERR_CUDA, "read result: %s", cudaGetErrorString(e));
    if (c.err != 0) {
        // report once: clear the recorded failure so that the next call starts clean
        e = cudaMemsetAsync(cb + offsetof(Ctrl, err), 0, 2 * sizeof(int), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return set_error(COS_ERR_CUDA, "clear error word: %s", cudaGetErrorString(e));
        if (c.err == KERR_BARRIER_TIMEOUT)
            return set_error(COS_ERR_TIMEOUT,
                             "a grid barrier timed out (phase %d) in this call or in a call since the last one that "
                             "passed mean_out; the results of those calls are invalid",
                             c.err_detail);
        return set_error(COS_ERR_CUDA, "kernel reported error %d", c.err);
    }
    *mean_out = c.mean;
    if (mode == COS_MODE_COUNT_I64 && gv.count_overflow)
        return set_error(COS_ERR_OVERFLOW, "path count exceeds 2^63-1; results wrap modulo 2^64");
    return COS_OK;
}
