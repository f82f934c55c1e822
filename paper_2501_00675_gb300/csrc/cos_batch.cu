// Batched evaluation of many graphs of uneven size and sample count in one
// persistent launch.  The paper evaluates one graph per thread block and notes
// that small graphs leave most of a block idle (Sec. III "Acceleration"); here
// every graph's work is cut into the same CTA-sized items as the single-graph
// kernel and all graphs share one persistent grid.
//
// Plan: each graph contributes its coefficients task, then per window of sample
// chunks a chain of phase tasks -- per tile of samples: propagators, levels
// 1..L-1 -- then partial sums (waiting for every window) and the final mean.
// Without windows a tile is one window, so a graph is one chain.  With windows
// (Sec. II.C: levels evaluated asynchronously) the window chains of a graph are
// laid out in wavefront order (step d holds phase d - w of window w), so about L
// windows are in flight and their node values and propagators are re-read while
// still in L2.  The graphs' lists are interleaved round-robin into one task list;
// CTAs draw tickets from a global counter, a ticket names one item of one task,
// and an item waits (bounded) until the tasks it depends on have completed all
// their items.  Tickets are handed out in list order and a task only ever waits
// on earlier tasks, so the lowest pending item can always run: no co-residency is
// required.  The launch (counter reset + kernel) is captured once into a CUDA
// graph and replayed.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "cos_items.cuh"
#include "cos_tasks.cuh"

namespace cosgpu {
namespace {

struct BatchCtrl {
    unsigned long long ticket;
    int err;
    int err_task;
};

struct BatchArgs {
    const Task* tasks;
    const int32_t* joins;
    int32_t ntasks;
    int32_t pad;
    int64_t total;
    const WalkParams* params;
    unsigned* done;
    BatchCtrl* ctrl;
    long long timeout_ns;
};

template <int MODE, int V, int LAYOUT>
constexpr int batch_min_blocks() {
    if (LAYOUT == LAYOUT_ASYNC) return 4;   // no loads held in registers: a fourth CTA per SM
    // FP32 walk from the work queue: a fourth CTA per SM (64 registers) measured faster on
    // the large graph (3.74 -> 3.49 s) and the batched launch (3.02 -> 2.87 s); the
    // level-synchronous kernel keeps three (medium 2.47 -> 2.72 ms with four)
    if (MODE == COS_MODE_FP32_MIXED && LAYOUT == LAYOUT_WIDE) return 4;
    return (Traits<MODE>::kBase == COS_MODE_FP64 && V > 2) ? 2 : 3;
}

template <int MODE, int V, int LAYOUT>
__global__ void __launch_bounds__(kThreads, batch_min_blocks<MODE, V, LAYOUT>()) batch_kernel(const BatchArgs a) {
    constexpr int CHV = chunk_samples<V, LAYOUT>();
    extern __shared__ __align__(16) double smem[];
    // Tickets: thread 0 claims the next ticket while the current item runs and hands
    // it over with the end-of-item barrier (double-buffered).  A claimed ticket is
    // held only by a CTA that is running an earlier one, so the lowest unfinished
    // ticket is always running and its dependencies (earlier tasks) are complete.
    __shared__ long long s_ticket[2];
    __shared__ int s_ok;
    if (threadIdx.x == 0) s_ticket[0] = (long long)atomicAdd(&a.ctrl->ticket, 1ull);
    __syncthreads();
    int cursor = 0, buf = 0;
    int ready = -1;   // the task whose dependencies this CTA has seen complete (they stay complete)
    long long next = 0;
    for (;;) {
        const long long t = s_ticket[buf];
        if (t >= a.total) break;
        while (cursor + 1 < a.ntasks && a.tasks[cursor + 1].first <= t) ++cursor;
        const Task tk = a.tasks[cursor];
        const int item = (int)(t - tk.first);
        if (threadIdx.x == 0) next = (long long)atomicAdd(&a.ctrl->ticket, 1ull);   // used after this item
        if (cursor != ready) {   // uniform: every thread tracks the same cursor
            if (threadIdx.x == 0) {
                int ok = 1;
                const unsigned long long t0 = global_timer_ns();
                unsigned long long spin = 0;
                for (int q = -1; ok && q < tk.join_cnt; ++q) {   // the chain predecessor, then the joins
                    const int dep = q < 0 ? tk.dep : a.joins[tk.join_off + q];
                    if (dep < 0) continue;
                    const unsigned need = (unsigned)a.tasks[dep].items;
                    for (;; ++spin) {
                        if (ld_acquire_gpu_u32(a.done + dep) >= need) break;
                        if (*(volatile int*)&a.ctrl->err != 0) { ok = 0; break; }
                        if ((spin & 31) == 31 &&
                            ((long long)(global_timer_ns() - t0) > a.timeout_ns || spin > (1ull << 32))) {
                            if (atomicCAS(&a.ctrl->err, 0, KERR_BARRIER_TIMEOUT) == 0) a.ctrl->err_task = cursor;
                            ok = 0;
                            break;
                        }
                        __nanosleep(64);
                    }
                }
                s_ok = ok;
            }
            __syncthreads();
            if (!s_ok) return;
            ready = cursor;
        }
        const WalkParams& p = a.params[tk.graph];
        TileCtx tc = tile_ctx<CHV>(p, tk.tix);
        tc.c0 = tk.c0;
        switch (tk.kind) {
            case TK_COEF: item_coef(p); break;
            case TK_PROP: item_props<MODE, CHV>(p, tc, item, smem); break;
            case TK_LEVEL:
                // FP64 items are long and bound by the FP64 pipe: balance their warps' edges
                // (medium 6.56 -> 6.47 ms); the short memory-bound items of the other modes
                // lose more to the row-pointer search than they gain (large mixed +7 %)
                if (!item_level<MODE, V, LAYOUT, Traits<MODE>::kBase == COS_MODE_FP64>(p, tk.level, tc, item,
                                                                       reinterpret_cast<unsigned char*>(smem)) &&
                    (threadIdx.x & 31) == 0) {   // a bounded wait gave up: report it for the whole launch
                    const int code = *(volatile int*)&p.ctrl->err;
                    if (atomicCAS(&a.ctrl->err, 0, code ? code : KERR_BARRIER_TIMEOUT) == 0)
                        a.ctrl->err_task = code > 100 ? p.ctrl->err_detail : cursor;
                }
                break;
            case TK_PARTIALS: item_partials<MODE>(p, item); break;
            case TK_STALL: break;
            default: item_final(p); break;
        }
        if (threadIdx.x == 0) s_ticket[buf ^ 1] = next;
        __syncthreads();
        if (threadIdx.x == 0 && tk.kind != TK_STALL)   // release: the item's writes are visible first
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(a.done + cursor) : "memory");
        buf ^= 1;
    }
}

template <int MODE, int V, int LAYOUT>
const void* bk() {
    return reinterpret_cast<const void*>(&batch_kernel<MODE, V, LAYOUT>);
}

template <int LAYOUT>
const void* select_batch_layout(int mode, int vec) {
    switch (mode * 8 + vec) {
        case COS_MODE_FP64 * 8 + 1: return bk<COS_MODE_FP64, 1, LAYOUT>();
        case COS_MODE_FP64 * 8 + 2: return bk<COS_MODE_FP64, 2, LAYOUT>();
        case COS_MODE_FP64 * 8 + 4: return bk<COS_MODE_FP64, 4, LAYOUT>();
        case COS_MODE_FP32_MIXED * 8 + 1: return bk<COS_MODE_FP32_MIXED, 1, LAYOUT>();
        case COS_MODE_FP32_MIXED * 8 + 2: return bk<COS_MODE_FP32_MIXED, 2, LAYOUT>();
        case COS_MODE_FP32_MIXED * 8 + 4: return bk<COS_MODE_FP32_MIXED, 4, LAYOUT>();
        case COS_MODE_COUNT_I64 * 8 + 1: return bk<COS_MODE_COUNT_I64, 1, LAYOUT>();
        case COS_MODE_COUNT_I64 * 8 + 2: return bk<COS_MODE_COUNT_I64, 2, LAYOUT>();
        case COS_MODE_COUNT_I64 * 8 + 4: return bk<COS_MODE_COUNT_I64, 4, LAYOUT>();
        default: return nullptr;
    }
}

const void* select_batch_kernel(int mode, int vec, int layout) {
    if (mode_has_abs(mode)) {   // sums of |path| values: the wide layout only
        if (layout != 1) return nullptr;
        switch (mode * 8 + vec) {
            case kModeFp64Abs * 8 + 1: return bk<kModeFp64Abs, 1, LAYOUT_WIDE>();
            case kModeFp64Abs * 8 + 2: return bk<kModeFp64Abs, 2, LAYOUT_WIDE>();
            case kModeFp64Abs * 8 + 4: return bk<kModeFp64Abs, 4, LAYOUT_WIDE>();
            case kModeMixedAbs * 8 + 1: return bk<kModeMixedAbs, 1, LAYOUT_WIDE>();
            case kModeMixedAbs * 8 + 2: return bk<kModeMixedAbs, 2, LAYOUT_WIDE>();
            case kModeMixedAbs * 8 + 4: return bk<kModeMixedAbs, 4, LAYOUT_WIDE>();
            default: return nullptr;
        }
    }
    if (layout == 4) return select_batch_layout<LAYOUT_ASYNC>(mode, vec);
    if (layout == 3) return select_batch_layout<LAYOUT_BULK>(mode, vec);
    if (layout == 2) return select_batch_layout<LAYOUT_GROUPED>(mode, vec);
    if (layout == 1) return select_batch_layout<LAYOUT_WIDE>(mode, vec);
    return nullptr;
}

}  // namespace
}  // namespace cosgpu

using namespace cosgpu;

// Co-resident CTAs of the work-queue kernel for (mode, vec, layout) with D time variables
// over the whole device; 0 on failure.
int cosgpu::batch_coresident_blocks(int mode, int vec, int layout, int D, int device) {
    const void* k = select_batch_kernel(mode, vec, layout);
    if (!k) return 0;
    const int smem = walk_smem_bytes(mode, vec, layout, D);
    if (prepare_kernel_attrs(k, smem) != COS_OK) return 0;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    return per_sm * sms;
}

struct cos_batch {
    int device = 0;
    int32_t n = 0;
    int32_t mode = 0;        // kernel mode id (kernel_mode of the public mode)
    std::vector<cos_graph_t> graphs;
    std::vector<void*> outs;
    cos_tuning tuning{};     // batch-level overrides (samples_per_lane, rows_per_warp, ...)
    cos_tuning resolved{};
    // host plan and its pinned staging copies
    std::vector<Task> tasks;
    std::vector<WalkParams> params;
    std::vector<int> counts_overflow;
    std::vector<int32_t> joins;
    std::vector<uint64_t> member_gen;   // each member's generation when the plan was made
    Task* h_tasks = nullptr;
    int32_t* h_joins = nullptr;
    WalkParams* h_params = nullptr;
    double* h_means = nullptr;
    BatchCtrl* h_ctrl = nullptr;
    // device buffers (grow only)
    Task* d_tasks = nullptr;
    int32_t* d_joins = nullptr;
    WalkParams* d_params = nullptr;
    unsigned* d_done = nullptr;
    double* d_means = nullptr;
    BatchCtrl* d_ctrl = nullptr;
    size_t cap_tasks = 0, cap_graphs = 0, cap_joins = 0;
    int32_t ntasks = 0;
    int64_t total = 0;
    int grid = 0;
    int smem = 0;
    bool planned = false;        // host plan matches members and tuning
    bool uploaded = false;       // device copy of the plan is current
    // The staging buffers are read by host-to-device copies that run when the stream
    // reaches them; `staged` is recorded after the last such copy and waited on before
    // the host overwrites (or frees) them.  staged_* describe what they hold, so an
    // identical plan (the usual repeated evaluation) is not copied again.
    cudaEvent_t staged = nullptr;
    bool staged_valid = false;
    size_t staged_tasks = 0, staged_joins = 0, staged_params = 0;
    int launches_since_plan = 0;
    // captured launch (counter reset + kernel), built on the second launch of a plan
    cudaGraph_t cgraph = nullptr;
    cudaGraphExec_t cexec = nullptr;
};

namespace {

void drop_capture(cos_batch* b) {
    if (b->cexec) cudaGraphExecDestroy(b->cexec);
    if (b->cgraph) cudaGraphDestroy(b->cgraph);
    b->cexec = nullptr;
    b->cgraph = nullptr;
}

// Host wait until the copies that read the staging buffers have run.
int wait_staged(cos_batch* b) {
    if (!b->staged) return COS_OK;
    cudaError_t e = cudaEventSynchronize(b->staged);
    if (e != cudaSuccess) return set_error(COS_ERR_CUDA, "wait for plan upload: %s", cudaGetErrorString(e));
    return COS_OK;
}

void free_buffers(cos_batch* b) {
    drop_capture(b);
    wait_staged(b);
    if (b->staged) cudaEventDestroy(b->staged);
    b->staged = nullptr;
    b->staged_valid = false;
    cudaFree(b->d_tasks);
    cudaFree(b->d_joins);
    cudaFree(b->d_params);
    cudaFree(b->d_done);
    cudaFree(b->d_means);
    cudaFree(b->d_ctrl);
    cudaFreeHost(b->h_joins);
    cudaFreeHost(b->h_tasks);
    cudaFreeHost(b->h_params);
    cudaFreeHost(b->h_means);
    cudaFreeHost(b->h_ctrl);
    b->d_tasks = nullptr;
    b->d_joins = nullptr;
    b->d_params = nullptr;
    b->d_done = nullptr;
    b->d_means = nullptr;
    b->d_ctrl = nullptr;
    b->h_tasks = nullptr;
    b->h_joins = nullptr;
    b->h_params = nullptr;
    b->h_means = nullptr;
    b->h_ctrl = nullptr;
    b->cap_tasks = b->cap_graphs = b->cap_joins = 0;
}

int ensure_capacity(cos_batch* b, size_t ntasks, size_t ngraphs, size_t njoins) {
    cudaError_t e = cudaSuccess;
    if (njoins > b->cap_joins || ntasks > b->cap_tasks || ngraphs > b->cap_graphs) {
        const int rc = wait_staged(b);   // pending copies still read the old staging buffers
        if (rc != COS_OK) return rc;
        b->staged_valid = false;
    }
    if (njoins > b->cap_joins) {
        cudaFree(b->d_joins);
        cudaFreeHost(b->h_joins);
        b->d_joins = nullptr;
        b->h_joins = nullptr;
        const size_t cap = std::max<size_t>(njoins, 2 * b->cap_joins);
        if ((e = cudaMalloc(&b->d_joins, sizeof(int32_t) * cap)) != cudaSuccess ||
            (e = cudaMallocHost(&b->h_joins, sizeof(int32_t) * cap)) != cudaSuccess)
            return set_error(COS_ERR_OOM, "batch joins: %s", cudaGetErrorString(e));
        b->cap_joins = cap;
    }
    if (!b->d_ctrl) {
        if ((e = cudaMalloc(&b->d_ctrl, sizeof(BatchCtrl))) != cudaSuccess ||
            (e = cudaMallocHost(&b->h_ctrl, sizeof(BatchCtrl))) != cudaSuccess)
            return set_error(COS_ERR_OOM, "batch control: %s", cudaGetErrorString(e));
    }
    if (ntasks > b->cap_tasks) {
        cudaFree(b->d_tasks);
        cudaFree(b->d_done);
        cudaFreeHost(b->h_tasks);
        b->d_tasks = nullptr;
        b->d_done = nullptr;
        b->h_tasks = nullptr;
        const size_t cap = std::max<size_t>(ntasks, 2 * b->cap_tasks);
        if ((e = cudaMalloc(&b->d_tasks, sizeof(Task) * cap)) != cudaSuccess ||
            (e = cudaMalloc(&b->d_done, sizeof(unsigned) * cap)) != cudaSuccess ||
            (e = cudaMallocHost(&b->h_tasks, sizeof(Task) * cap)) != cudaSuccess)
            return set_error(COS_ERR_OOM, "batch task list: %s", cudaGetErrorString(e));
        b->cap_tasks = cap;
    }
    if (ngraphs > b->cap_graphs) {
        cudaFree(b->d_params);
        cudaFree(b->d_means);
        cudaFreeHost(b->h_params);
        cudaFreeHost(b->h_means);
        b->d_params = nullptr;
        b->d_means = nullptr;
        b->h_params = nullptr;
        b->h_means = nullptr;
        const size_t cap = std::max<size_t>(ngraphs, 2 * b->cap_graphs);
        if ((e = cudaMalloc(&b->d_params, sizeof(WalkParams) * cap)) != cudaSuccess ||
            (e = cudaMalloc(&b->d_means, 2 * sizeof(double) * cap)) != cudaSuccess ||
            (e = cudaMallocHost(&b->h_params, sizeof(WalkParams) * cap)) != cudaSuccess ||
            (e = cudaMallocHost(&b->h_means, 2 * sizeof(double) * cap)) != cudaSuccess)
            return set_error(COS_ERR_OOM, "batch parameters: %s", cudaGetErrorString(e));
        b->cap_graphs = cap;
    }
    return COS_OK;
}

// Build the interleaved task list and the per-graph parameters on the host.
int plan(cos_batch* b) {
    const int mode = b->mode;
    // one vector width and layout for the whole launch (kernel template parameters)
    cos_tuning force = b->tuning;
    if (force.samples_per_lane <= 0) force.samples_per_lane = (base_mode(mode) == COS_MODE_FP32_MIXED) ? 4 : 2;
    if (force.layout <= 0 || mode_has_abs(mode)) force.layout = 1;   // sums of |path|: wide layout only
    const int chv = force.layout == 2 ? 32 : 32 * force.samples_per_lane;   // wide and bulk: 32 * V
    cos_tuning first = force;
    b->params.assign((size_t)b->n, WalkParams{});
    b->counts_overflow.assign((size_t)b->n, 0);
    b->member_gen.assign((size_t)b->n, 0);
    // per graph: its tasks in issue order; dep and joins as indices into the same list
    std::vector<std::vector<Task>> lists((size_t)b->n);
    std::vector<std::vector<std::vector<int32_t>>> local_joins((size_t)b->n);
    for (int32_t g = 0; g < b->n; ++g) {
        cos_tuning tn;
        int rc = prepare_walk(b->graphs[(size_t)g], mode, &force, b->outs[(size_t)g], &b->params[(size_t)g], &tn);
        if (rc != COS_OK) return rc;
        if (g == 0) first = tn;
        GraphView gv;
        graph_view(b->graphs[(size_t)g], &gv);
        b->counts_overflow[(size_t)g] = gv.count_overflow;
        b->member_gen[(size_t)g] = gv.generation;
        graph_task_chain(b->params[(size_t)g], gv.widths_host, base_mode(mode), chv, force.window_chunks, g, false,
                         g == 0 && getenv("COS_TEST_STALL_TASK") != nullptr, lists[(size_t)g],
                         local_joins[(size_t)g]);
    }
    // Round-robin interleave of the graphs' lists (each list keeps its order).
    b->tasks.clear();
    b->joins.clear();
    std::vector<std::vector<int32_t>> gidx((size_t)b->n);
    size_t longest = 0;
    for (auto& l : lists) longest = std::max(longest, l.size());
    for (size_t r = 0; r < longest; ++r)
        for (int32_t g = 0; g < b->n; ++g) {
            if (r >= lists[(size_t)g].size()) continue;
            Task t = lists[(size_t)g][r];
            std::vector<int32_t>& map = gidx[(size_t)g];
            if (t.dep >= 0) t.dep = map[(size_t)t.dep];
            const std::vector<int32_t>& js = local_joins[(size_t)g][r];
            t.join_off = (int32_t)b->joins.size();
            t.join_cnt = (int32_t)js.size();
            for (int32_t q : js) b->joins.push_back(map[(size_t)q]);
            map.push_back((int32_t)b->tasks.size());
            b->tasks.push_back(t);
        }
    int64_t first_ticket = 0;
    for (auto& t : b->tasks) {
        t.first = first_ticket;
        first_ticket += t.items;
    }
    b->ntasks = (int32_t)b->tasks.size();
    b->total = first_ticket;
    b->resolved = first;
    b->resolved.samples_per_lane = force.samples_per_lane;
    b->resolved.layout = force.layout;
    b->resolved.schedule = force.window_chunks > 0 ? 2 : 1;
    b->resolved.window_chunks = force.window_chunks;
    b->resolved.prefetch = first.prefetch;
    const void* k = select_batch_kernel(mode, b->resolved.samples_per_lane, b->resolved.layout);
    if (!k) return set_error(COS_ERR_INVALID, "no batch kernel for samples_per_lane %d", b->resolved.samples_per_lane);
    int dmax = 1;
    for (const WalkParams& p : b->params) dmax = std::max(dmax, p.D);
    const int smem = walk_smem_bytes(mode, b->resolved.samples_per_lane, b->resolved.layout, dmax);
    if (prepare_kernel_attrs(k, smem) != COS_OK) return set_error(COS_ERR_CUDA, "cannot set dynamic shared memory");
    b->smem = smem;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem) != cudaSuccess || per_sm <= 0)
        return set_error(COS_ERR_CUDA, "occupancy query failed");
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    int bps = per_sm;
    if (b->tuning.blocks_per_sm > 0) bps = std::min(bps, b->tuning.blocks_per_sm);
    b->resolved.blocks_per_sm = bps;
    b->grid = sms * bps;
    int rc = ensure_capacity(b, std::max<size_t>(b->tasks.size(), 1), std::max<int32_t>(b->n, 1),
                             std::max<size_t>(b->joins.size(), 1));
    if (rc != COS_OK) return rc;
    for (int32_t g = 0; g < b->n; ++g) b->params[(size_t)g].mean_out = b->d_means + 2 * g;   // (mean R, mean A)
    drop_capture(b);
    b->planned = true;
    b->uploaded = false;
    b->launches_since_plan = 0;
    return COS_OK;
}

// Counter reset + kernel: the part of a launch that is captured and replayed.
int enqueue_run(cos_batch* b, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(b->d_done, 0, sizeof(unsigned) * std::max<int32_t>(b->ntasks, 1), st)) != cudaSuccess ||
        (e = cudaMemsetAsync(b->d_ctrl, 0, sizeof(BatchCtrl), st)) != cudaSuccess)
        return set_error(COS_ERR_CUDA, "reset batch counters: %s", cudaGetErrorString(e));
    BatchArgs a;
    a.tasks = b->d_tasks;
    a.joins = b->d_joins;
    a.ntasks = b->ntasks;
    a.pad = 0;
    a.total = b->total;
    a.params = b->d_params;
    a.done = b->d_done;
    a.ctrl = b->d_ctrl;
    a.timeout_ns = (long long)(b->resolved.timeout_ms > 0 ? b->resolved.timeout_ms : 10000) * 1000000LL;
    void* args[] = {&a};
    const void* k = select_batch_kernel(b->mode, b->resolved.samples_per_lane, b->resolved.layout);
    const size_t smem = (size_t)b->smem;
    if (b->total > 0 && (e = cudaLaunchKernel(k, dim3(b->grid), dim3(kThreads), args, smem, st)) != cudaSuccess)
        return set_error(COS_ERR_CUDA, "batch launch: %s", cudaGetErrorString(e));
    return COS_OK;
}

// Stream-ordered upload of the plan from pinned staging buffers.
int upload(cos_batch* b, cudaStream_t st) {
    const size_t nt = b->tasks.size(), nj = b->joins.size(), np = (size_t)b->n;
    // The device already holds this exact plan (the kernel only reads it).
    if (b->staged_valid && b->staged_tasks == nt && b->staged_joins == nj && b->staged_params == np &&
        (nt == 0 || memcmp(b->h_tasks, b->tasks.data(), sizeof(Task) * nt) == 0) &&
        (nj == 0 || memcmp(b->h_joins, b->joins.data(), sizeof(int32_t) * nj) == 0) &&
        (np == 0 || memcmp(b->h_params, b->params.data(), sizeof(WalkParams) * np) == 0)) {
        b->uploaded = true;
        return COS_OK;
    }
    int rc = wait_staged(b);   // an earlier upload's copies may not have run yet
    if (rc != COS_OK) return rc;
    b->staged_valid = false;
    cudaError_t e = cudaSuccess;
    if (!b->staged) e = cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming);
    if (e == cudaSuccess && !b->tasks.empty()) {
        memcpy(b->h_tasks, b->tasks.data(), sizeof(Task) * b->tasks.size());
        e = cudaMemcpyAsync(b->d_tasks, b->h_tasks, sizeof(Task) * b->tasks.size(), cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess && !b->joins.empty()) {
        memcpy(b->h_joins, b->joins.data(), sizeof(int32_t) * b->joins.size());
        e = cudaMemcpyAsync(b->d_joins, b->h_joins, sizeof(int32_t) * b->joins.size(), cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess && b->n) {
        memcpy(b->h_params, b->params.data(), sizeof(WalkParams) * b->n);
        e = cudaMemcpyAsync(b->d_params, b->h_params, sizeof(WalkParams) * b->n, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->staged, st);
    if (e != cudaSuccess) return set_error(COS_ERR_CUDA, "upload plan: %s", cudaGetErrorString(e));
    b->staged_valid = true;
    b->staged_tasks = nt;
    b->staged_joins = nj;
    b->staged_params = np;
    b->uploaded = true;
    return COS_OK;
}

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev) {
        cudaGetDevice(&prev);
        cudaSetDevice(dev);
    }
    ~DevGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

int cosgpu::launch_windowed(cos_graph_t g, cos_batch_t* cache, int mode, void* per_sample_out, const cos_tuning& tn,
                                   cudaStream_t st) {
    cos_batch* b = *cache;
    if (!b) {
        b = new (std::nothrow) cos_batch();
        if (!b) return set_error(COS_ERR_OOM, "host allocation failed");
        *cache = b;
    }
    b->mode = mode;
    int rc = cos_batch_reset(b, 1, &g, &per_sample_out);
    if (rc != COS_OK) return rc;
    b->tuning = tn;
    rc = plan(b);
    if (rc == COS_OK) rc = upload(b, st);
    if (rc == COS_OK) rc = enqueue_run(b, st);
    return rc;
}

extern "C" {

int cos_batch_create(int32_t n, const cos_graph_t* graphs, int32_t mode, void* const* per_sample_outs,
                     cos_batch_t* out) {
    if (!out) return set_error(COS_ERR_INVALID, "out is NULL");
    const int km = kernel_mode(mode);
    if (km < 0) return set_error(COS_ERR_INVALID, "bad mode %d", mode);
    cos_batch* b = new (std::nothrow) cos_batch();
    if (!b) return set_error(COS_ERR_OOM, "host allocation failed");
    b->mode = km;
    int rc = cos_batch_reset(b, n, graphs, per_sample_outs);
    if (rc != COS_OK) {
        delete b;
        return rc;
    }
    *out = b;
    return COS_OK;
}

int cos_batch_reset(cos_batch_t b, int32_t n, const cos_graph_t* graphs, void* const* per_sample_outs) {
    if (!b || n < 0 || (n > 0 && !graphs)) return set_error(COS_ERR_INVALID, "bad arguments");
    int dev = -1;
    for (int32_t g = 0; g < n; ++g) {
        GraphView gv;
        int rc = graph_view(graphs[g], &gv);
        if (rc != COS_OK) return rc;
        if (dev >= 0 && gv.device != dev) return set_error(COS_ERR_INVALID, "all graphs must be on one device");
        dev = gv.device;
        for (int32_t h = 0; h < g; ++h)
            if (graphs[h] == graphs[g]) return set_error(COS_ERR_INVALID, "graph handle %d appears twice in the batch", g);
    }
    if (b->d_ctrl && dev >= 0 && dev != b->device) return set_error(COS_ERR_INVALID, "a batch stays on one device");
    if (dev >= 0) b->device = dev;
    else cudaGetDevice(&b->device);
    b->n = n;
    b->graphs.assign(graphs, graphs + n);
    b->outs.assign((size_t)n, nullptr);
    if (per_sample_outs)
        for (int32_t g = 0; g < n; ++g) b->outs[(size_t)g] = per_sample_outs[g];
    b->planned = false;
    return COS_OK;
}

int cos_batch_set_tuning(cos_batch_t b, const cos_tuning* t) {
    if (!b || !t) return set_error(COS_ERR_INVALID, "bad arguments");
    if (t->samples_per_lane > 0 && t->samples_per_lane != 1 && t->samples_per_lane != 2 && t->samples_per_lane != 4)
        return set_error(COS_ERR_INVALID, "samples_per_lane must be 1, 2 or 4");
    if (t->rows_per_warp > 31) return set_error(COS_ERR_INVALID, "rows_per_warp must be <= 31");
    if (t->layout < 0 || t->layout > 4) return set_error(COS_ERR_INVALID, "layout must be 0, 1, 2, 3 or 4");
    if (t->window_chunks < 0) return set_error(COS_ERR_INVALID, "window_chunks must be >= 0");
    if (t->prefetch < 0 || t->prefetch > 7) return set_error(COS_ERR_INVALID, "prefetch must be 0..7");
    b->tuning = *t;
    b->planned = false;
    return COS_OK;
}

int cos_batch_get_tuning(cos_batch_t b, cos_tuning* t) {
    if (!b || !t) return set_error(COS_ERR_INVALID, "bad arguments");
    *t = b->resolved;
    return COS_OK;
}

int cos_batch_launch(cos_batch_t b, void* stream) {
    if (!b) return set_error(COS_ERR_INVALID, "batch is NULL");
    DevGuard dg(b->device);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = COS_OK;
    if (b->planned) {
        // a member whose buffers, samples or tuning changed since the plan was made:
        // the plan (and the captured graph) hold its old pointers and sizes
        for (int32_t g = 0; g < b->n && b->planned; ++g) {
            GraphView gv;
            if ((rc = graph_view(b->graphs[(size_t)g], &gv)) != COS_OK) return rc;
            if (gv.generation != b->member_gen[(size_t)g]) b->planned = false;
        }
    }
    if (!b->planned) rc = plan(b);
    if (rc != COS_OK) return rc;
    if (!b->uploaded) {
        rc = upload(b, st);
        if (rc != COS_OK) return rc;
    }
    b->launches_since_plan++;
    if (b->launches_since_plan == 1) return enqueue_run(b, st);   // a plan launched once is not worth capturing
    if (!b->cexec) {
        // second launch of the same plan: capture counter reset + kernel once, replay afterwards
        cudaStream_t cap;
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return set_error(COS_ERR_CUDA, "capture stream: %s", cudaGetErrorString(e));
        if ((e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
            cudaStreamDestroy(cap);
            return set_error(COS_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
        }
        rc = enqueue_run(b, cap);
        e = cudaStreamEndCapture(cap, &b->cgraph);
        cudaStreamDestroy(cap);
        if (rc != COS_OK) return rc;
        if (e != cudaSuccess) return set_error(COS_ERR_CUDA, "end capture: %s", cudaGetErrorString(e));
        if ((e = cudaGraphInstantiate(&b->cexec, b->cgraph, 0)) != cudaSuccess)
            return set_error(COS_ERR_CUDA, "instantiate: %s", cudaGetErrorString(e));
    }
    cudaError_t e = cudaGraphLaunch(b->cexec, st);
    if (e != cudaSuccess) return set_error(COS_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
    return COS_OK;
}

int cos_batch_results(cos_batch_t b, double* means, void* stream) {
    if (!b) return set_error(COS_ERR_INVALID, "batch is NULL");
    if (!b->planned || !b->uploaded) return set_error(COS_ERR_STATE, "batch has not been launched");
    DevGuard dg(b->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(b->h_ctrl, b->d_ctrl, sizeof(BatchCtrl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && b->n)
        e = cudaMemcpyAsync(b->h_means, b->d_means, 2 * sizeof(double) * b->n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(COS_ERR_CUDA, "batch results: %s", cudaGetErrorString(e));
    if (b->h_ctrl->err == KERR_BARRIER_TIMEOUT)
        return set_error(COS_ERR_TIMEOUT, "dependency wait timed out (task %d)", b->h_ctrl->err_task);
    if (b->h_ctrl->err != 0)
        return set_error(COS_ERR_CUDA, "batch kernel error %d (detail %d)", b->h_ctrl->err, b->h_ctrl->err_task);
    if (means) {   // [n], or [n][2] (mean R, mean A) for a batch that also sums |path| values
        const bool abs2 = mode_has_abs(b->mode);
        for (int32_t g = 0; g < b->n; ++g) {
            if (abs2) {
                means[2 * g] = b->h_means[2 * g];
                means[2 * g + 1] = b->h_means[2 * g + 1];
            } else {
                means[g] = b->h_means[2 * g];
            }
        }
    }
    if (b->mode == COS_MODE_COUNT_I64)
        for (int32_t g = 0; g < b->n; ++g)
            if (b->counts_overflow[(size_t)g])
                return set_error(COS_ERR_OVERFLOW, "graph %d: path count exceeds 2^63-1", g);
    return COS_OK;
}

int cos_batch_autotune(cos_batch_t b, void* stream, cos_tuning* best_out) {
    if (!b) return set_error(COS_ERR_INVALID, "batch is NULL");
    DevGuard dg(b->device);
    cudaStream_t st = (cudaStream_t)stream;
    const cos_tuning base = b->tuning;
    const int vecs[] = {1, 2, 4};
    const int rpws[] = {4, 8, 16, 31};
    float best_ms = 1e30f;
    cos_tuning best = base;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = COS_OK;
    const int layouts[] = {1, 2, 3, 4};
    for (int lay : layouts)
    for (int v : vecs) {
        if (mode_has_abs(b->mode) && lay != 1) continue;    // sums of |path|: wide layout only
        if (base_mode(b->mode) == COS_MODE_FP64 && v == 4) continue;   // register-heavy; never faster in FP64
        if (lay == 2 && v == 1) continue;                   // identical to the wide layout
        for (int r : rpws) {
            cos_tuning t = base;
            t.samples_per_lane = v;
            t.rows_per_warp = r;
            t.layout = lay;
            b->tuning = t;
            rc = plan(b);
            if (rc == COS_OK) rc = upload(b, st);
            if (rc != COS_OK) break;
            float ms_best = 1e30f;
            for (int rep = 0; rep < 2; ++rep) {
                cudaEventRecord(e0, st);
                rc = enqueue_run(b, st);
                cudaEventRecord(e1, st);
                if (rc != COS_OK) break;
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms_best = std::min(ms_best, ms);
            }
            if (rc != COS_OK) break;
            cudaMemcpyAsync(b->h_ctrl, b->d_ctrl, sizeof(BatchCtrl), cudaMemcpyDeviceToHost, st);
            cudaStreamSynchronize(st);
            if (b->h_ctrl->err != 0) {
                rc = set_error(COS_ERR_TIMEOUT, "autotune candidate failed (error %d)", b->h_ctrl->err);
                break;
            }
            if (ms_best < best_ms) {
                best_ms = ms_best;
                best = t;
            }
        }
        if (rc != COS_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tuning = best;
    if (rc == COS_OK) rc = plan(b);
    if (rc == COS_OK && best_out) *best_out = b->resolved;
    return rc;
}

int cos_batch_destroy(cos_batch_t b) {
    if (!b) return COS_OK;
    {
        DevGuard dg(b->device);
        free_buffers(b);
    }
    delete b;
    return COS_OK;
}

int cos_evaluate_batch(int32_t n, const cos_graph_t* graphs, const int32_t* modes, void* const* per_sample_outs,
                       double* means, void* stream) {
    if (n < 0 || (n > 0 && (!graphs || !modes))) return set_error(COS_ERR_INVALID, "bad arguments");
    for (int32_t g = 0; g < n; ++g)
        if (kernel_mode(modes[g]) < 0) return set_error(COS_ERR_INVALID, "bad mode %d for graph %d", modes[g], g);
    // one persistent launch per distinct mode (the mode is a template parameter of the
    // kernel), in order of first appearance, all enqueued before the first wait
    std::vector<int32_t> order;
    for (int32_t g = 0; g < n; ++g)
        if (std::find(order.begin(), order.end(), modes[g]) == order.end()) order.push_back(modes[g]);
    std::vector<cos_batch_t> batches(order.size(), nullptr);
    std::vector<std::vector<int32_t>> members(order.size());
    int rc = COS_OK;
    for (size_t q = 0; q < order.size() && rc == COS_OK; ++q) {
        std::vector<cos_graph_t> gs;
        std::vector<void*> outs;
        for (int32_t g = 0; g < n; ++g)
            if (modes[g] == order[q]) {
                members[q].push_back(g);
                gs.push_back(graphs[g]);
                outs.push_back(per_sample_outs ? per_sample_outs[g] : nullptr);
            }
        rc = cos_batch_create((int32_t)gs.size(), gs.data(), order[q], outs.data(), &batches[q]);
        if (rc == COS_OK) rc = cos_batch_launch(batches[q], stream);
    }
    int first_err = rc;
    for (size_t q = 0; q < order.size(); ++q) {
        if (!batches[q]) continue;
        if (first_err == COS_OK) {
            std::vector<double> m(2 * members[q].size());
            int r = cos_batch_results(batches[q], m.data(), stream);
            if (r == COS_OK || r == COS_ERR_OVERFLOW) {
                const bool abs2 = mode_has_abs(kernel_mode(order[q]));
                if (means)
                    for (size_t j = 0; j < members[q].size(); ++j) {
                        const int32_t g = members[q][j];
                        means[2 * g] = abs2 ? m[2 * j] : m[j];
                        means[2 * g + 1] = abs2 ? m[2 * j + 1] : std::nan("");
                    }
            }
            if (r != COS_OK && rc == COS_OK) rc = r;
            if (r != COS_OK && r != COS_ERR_OVERFLOW) first_err = r;
        }
        cos_batch_destroy(batches[q]);
    }
    return first_err != COS_OK ? first_err : rc;
}

}  // extern "C"
