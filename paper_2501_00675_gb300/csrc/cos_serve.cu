// Resident evaluation server: one persistent kernel keeps running while requests
// arrive, and a request admitted while it runs starts at the next free work item,
// not at the next launch.
//
// Requests are graph evaluations (Fig. 1; Sec. II.C) over counter-based uniform
// sample times drawn on the device.  The host turns each request into the same
// task chain as a batched launch (times, coefficients, per window of sample chunks
// propagators and levels 1..L-1, partial sums, final mean) and feeds the chains of
// all active requests into a task ring in device memory round-robin, one task per
// request per round (consecutive tasks are then independent, as in the batched
// plan), keeping a bounded backlog ahead of the kernel's cursor so that a new
// request joins the rotation within that backlog.  Descriptors, join entries, claim
// words and finally the published-task counter are written by host-to-device copies
// on one copy stream, so neither a claim word nor the counter is seen before what
// it announces; no kernel has to run to admit a request.  The host feeds from every submit, poll, wait and
// stats call.
//
// Claiming: a global cursor names the task whose items are handed out; a CTA reads
// the cursor and, if that task is published, takes an item by one fetch-and-add on
// the slot's claim word, (tag << 32) | (2^31 + items left): the tag is the low 32
// bits of the task's absolute index, and counting down from the bias never borrows
// into it.  The returned value names the item (or, if the slot already holds a
// later task, an item of that task, which is as good a claim); a task whose items
// are all handed out moves the cursor on.  No compare-and-swap retry is on the
// path of an item.  Items are handed out in task order except through a stale
// cursor; a CTA waits only for the dependencies of the earliest item it holds and
// sets aside an out-of-order item that is not ready (see serve_kernel), so the
// lowest unfinished item can run: no co-residency is required and an idle CTA,
// which holds nothing, may leave at any time.  Completion counters
// per ring slot are cumulative over the tasks the slot has held (a task is
// complete once its slot's counter reaches the value the host assigned, which
// every dependent carries in its own descriptor); the CTA that completes a task
// flags it in host-mapped memory, and the host reuses ring entries in order once
// they are flagged.  A published task never needs a later one, so the ring always
// drains.
//
// Every wait is bounded: dependency waits by the tuning's timeout (then the error
// is recorded and every CTA leaves), the idle poll by the server's idle time (then
// the CTA leaves; the host relaunches the kernel when work is pending and no CTA
// is left).  Completion is reported through host-mapped records (the mean, then
// the request number with a system-scope release), which the host polls.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <thread>
#include <vector>

#include "cos_items.cuh"
#include "cos_feed.h"
#include "cos_tasks.cuh"

namespace cosgpu {
namespace {

static_assert(sizeof(WalkParams) % 8 == 0, "parameters are copied as 8-byte words");

struct SvPub {          // device memory, written only by host-to-device copies
    long long tasks;    // tasks published so far
    int shutdown;       // 1: leave as soon as no published work is left
    int pad;
};

struct SvCtl {          // device memory
    long long cursor;   // task whose items are being handed out
    int err;
    int pad;
    unsigned long long stale_claims;   // claims whose slot already held a later task
};

struct SvComp {                 // host-mapped, one per request slot
    unsigned long long seq;     // request number, stored last (release, system scope)
    double mean;
};

struct SvStatus {               // host-mapped
    int err;                    // first kernel-side error (KERR_*, or a level item's code)
    int pad;
    long long err_task;         // absolute index of the task that reported it
};

struct ServeArgs {
    const SvTask* ring;
    const unsigned long long* joins;   // (ring slot << 32) | counter value, per join
    const WalkParams* params;
    unsigned long long* claim;  // [cap]: (task tag << 32) | (2^31 + items not yet handed out)
    unsigned* done;             // [cap]: items completed, cumulative over the slot's tasks
    SvCtl* ctl;
    const SvPub* pub;
    SvComp* comp;               // device alias of the mapped completion records
    SvStatus* status;           // device alias of the mapped status
    unsigned* tdone;            // device alias of the mapped task-complete flags [cap] (task tag)
    unsigned long long* cursor_out;   // device alias of the mapped cursor copy
    long long mask;
    long long jmask;
    long long timeout_ns;
    long long idle_ns;
    int test_stale;     // test hook: about one claim in test_stale reads a stale cursor (0: off)
    int pad;
};

__device__ __forceinline__ long long ld_volatile_s64(const long long* p) { return *(const volatile long long*)p; }
__device__ __forceinline__ int ld_volatile_s32(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
    return *(const volatile unsigned long long*)p;
}

__device__ __forceinline__ long long ld_acquire_gpu_s64(const long long* p) {
    long long v;
    asm volatile("ld.acquire.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Record the first error for the host and for the other CTAs.
__device__ __forceinline__ void sv_fail(const ServeArgs& a, int code, long long task) {
    if (atomicCAS(&a.ctl->err, 0, code) == 0) {
        a.status->err_task = task;
        a.status->err = code;
        __threadfence_system();
    }
}

// One attempt to claim an item (thread 0).  Returns 1 with (k, item) -- ooo set when
// the item came through a stale cursor and belongs to a task ahead of the cursor --,
// 0 when every published item is handed out, 2 when 64 tasks in a row turned out
// exhausted.
__device__ int sv_try_claim(const ServeArgs& a, long long& pub, long long& k_out, int& item_out, int& ooo) {
    for (int attempt = 0; attempt < 64; ++attempt) {
        long long k = ld_volatile_s64(&a.ctl->cursor);
        if (k >= pub) {
            pub = ld_acquire_gpu_s64(&a.pub->tasks);
            if (k >= pub) return 0;
        }
        if (a.test_stale > 0 && pub - k > 1) {
            // test hook: act on a cursor value one ring behind a published task t ahead of the
            // cursor, as a CTA would that read the cursor that long ago
            const unsigned long long h = global_timer_ns() * 0x9E3779B97F4A7C15ull + blockIdx.x;
            if ((h >> 40) % (unsigned long long)a.test_stale == 0)
                k = k + 1 + (long long)((h >> 20) % (unsigned long long)(pub - k - 1)) - (a.mask + 1);
        }
        const unsigned long long old = atomicAdd(a.claim + (k & a.mask), ~0ull);   // minus one
        const int age = (int)((unsigned)(old >> 32) - (unsigned)k);   // > 0: the slot holds a later task
        const unsigned left = (unsigned)old;
        if (age < 0) return 0;   // not yet initialised for k (cannot happen once k is published)
        if (left > 0x80000000u) {
            k_out = k + age;
            item_out = (int)(left - 0x80000001u);
            ooo = age > 0;
            if (ooo) atomicAdd(&a.ctl->stale_claims, 1ull);
            return 1;
        }
        // task k is exhausted: move the cursor on
        if (atomicCAS(reinterpret_cast<unsigned long long*>(&a.ctl->cursor), (unsigned long long)k,
                      (unsigned long long)(k + 1)) == (unsigned long long)k)   // for the host's feeder
            asm volatile("st.relaxed.sys.global.u64 [%0], %1;" ::"l"(a.cursor_out), "l"((unsigned long long)(k + 1))
                         : "memory");
    }
    return 2;
}

// sv_try_claim retried while it reports exhausted tasks skipped with work left (2),
// up to 64 times (4,096 tasks): 1 with (k, item), else 0.  Used where a CTA holds an
// item set aside, so that "nothing claimable" means no published item is unclaimed.
__device__ int sv_try_claim_settled(const ServeArgs& a, long long& pub, long long& k_out, int& item_out, int& ooo) {
    for (int r = 0; r < 64; ++r) {
        const int c = sv_try_claim(a, pub, k_out, item_out, ooo);
        if (c != 2) return c;
        if (ld_volatile_s32(&a.ctl->err) != 0) return 0;
    }
    return 0;
}

// Claim an item, waiting (bounded by the idle time) for work to be published.
// Returns 1 with (k, item), 0 to leave (shutdown, idle, or another CTA's error).
__device__ int sv_claim(const ServeArgs& a, long long& pub, long long& k_out, int& item_out, int& ooo) {
    unsigned long long t0 = global_timer_ns();
    unsigned sleep_ns = 64;
    for (unsigned long long spin = 0;; ++spin) {
        const int r = sv_try_claim(a, pub, k_out, item_out, ooo);
        if (r == 1) return 1;
        if (ld_volatile_s32(&a.ctl->err) != 0) return 0;
        if (r == 2) {   // work is there: not idle
            t0 = global_timer_ns();
            continue;
        }
        if (ld_volatile_s32(&a.pub->shutdown) != 0) return 0;
        if ((long long)(global_timer_ns() - t0) > a.idle_ns || spin > (1ull << 32)) return 0;
        __nanosleep(sleep_ns);
        sleep_ns = min(sleep_ns * 2, 8192u);
    }
}

// Request times: columns [item * kTimesPerItem, ...) of t[D][t_ld]; draws for the
// samples s < S (sample number first + s), zeros in the padding.
__device__ __forceinline__ void item_times(const WalkParams& p, unsigned long long seed, long long first, int item) {
    const int pairs = (p.D + 1) / 2;
    const long long s0 = (long long)item * kTimesPerItem;
    const long long n = min((long long)kTimesPerItem, p.t_ld - s0);
    double* t = const_cast<double*>(p.t);
    for (long long q = threadIdx.x; q < n * pairs; q += blockDim.x) {
        const int m = (int)(q / n);
        const long long s = s0 + (q - (long long)m * n);
        double x = 0.0, y = 0.0;
        if (s < p.S) uniform_time_pair(seed, (unsigned long long)(first + s), m, p.beta, x, y);
        t[(long long)(2 * m) * p.t_ld + s] = x;
        if (2 * m + 1 < p.D) t[(long long)(2 * m + 1) * p.t_ld + s] = y;
    }
}

// Dependencies of task `t` (its chain predecessor, then its joins) complete now?
__device__ __forceinline__ bool sv_deps_ready(const ServeArgs& a, int dep_slot, unsigned dep_need, long long join_off,
                                              int join_cnt) {
    for (int q = -1; q < join_cnt; ++q) {
        int dslot = dep_slot;
        unsigned need = dep_need;
        if (q >= 0) {
            const unsigned long long j = __ldcg(a.joins + ((join_off + q) & a.jmask));
            dslot = (int)(j >> 32);
            need = (unsigned)j;
        }
        if (dslot >= 0 && (int)(ld_acquire_gpu_u32(a.done + dslot) - need) < 0) return false;
    }
    return true;
}

// Wait (bounded by the timeout) until the dependencies of the task in s_tk are complete.
__device__ bool sv_wait_deps(const ServeArgs& a, const SvTask& tk) {
    const unsigned long long t0 = global_timer_ns();
    for (unsigned long long spin = 0;; ++spin) {
        if (sv_deps_ready(a, tk.dep_slot, tk.dep_need, tk.join_off, tk.join_cnt)) return true;
        if (ld_volatile_s32(&a.ctl->err) != 0) return false;
        if ((spin & 31) == 31 && ((long long)(global_timer_ns() - t0) > a.timeout_ns || spin > (1ull << 32))) {
            sv_fail(a, KERR_BARRIER_TIMEOUT, tk.self);
            return false;
        }
        __nanosleep(64);
    }
}

// A CTA holds at most three items: the current one, one claimed ahead and one set
// aside.  It only ever waits for the dependencies of the earliest item it holds
// (they are earlier still, so none is held by this CTA): when the current item is
// not ready and an item it holds is earlier, that one runs first.  An item claimed
// out of order (through a stale cursor) that is not ready is set aside -- at most
// one per CTA -- while the CTA keeps claiming in order; it runs at the first item
// boundary at which its dependencies are complete, and the CTA does not leave
// while it holds one (with no other work left it waits for them).
template <int MODE, int V>
__global__ void __launch_bounds__(kThreads, (MODE == COS_MODE_FP64 && V > 2) ? 2 : 3) serve_kernel(const ServeArgs a) {
    constexpr int CHV = chunk_samples<V, LAYOUT_WIDE>();
    extern __shared__ __align__(16) double smem[];
    __shared__ WalkParams s_p;
    __shared__ SvTask s_tk;
    __shared__ long long s_k[2];
    __shared__ int s_item[2];
    __shared__ int s_ooo[2];
    __shared__ int s_ok;
    // thread 0 only: published tasks last seen, the item claimed ahead, the item set aside
    long long pub = 0, nk = -1, dk = -1;
    int nitem = 0, nooo = 0, ditem = 0;
    if (threadIdx.x == 0) {
        long long k = -1;
        int item = 0, ooo = 0;
        if (!sv_claim(a, pub, k, item, ooo)) k = -1;
        s_k[0] = k;
        s_item[0] = item;
        s_ooo[0] = ooo;
    }
    __syncthreads();
    long long cur_k = -1, cur_seq = -1;
    int buf = 0;
    for (;;) {
        const long long k = s_k[buf];
        const int item = s_item[buf];
        if (k < 0) return;
        if (k != cur_k) {   // uniform: every thread sees the same k
            const long long s = k & a.mask;
            constexpr int TW = sizeof(SvTask) / 8;
            if (threadIdx.x < TW)
                reinterpret_cast<unsigned long long*>(&s_tk)[threadIdx.x] =
                    __ldcg(reinterpret_cast<const unsigned long long*>(a.ring + s) + threadIdx.x);
            __syncthreads();
            if (s_tk.seq != cur_seq) {
                constexpr int PW = sizeof(WalkParams) / 8;
                const unsigned long long* src = reinterpret_cast<const unsigned long long*>(a.params + s_tk.req);
                for (int w = threadIdx.x; w < PW; w += blockDim.x)
                    reinterpret_cast<unsigned long long*>(&s_p)[w] = __ldcg(src + w);
                cur_seq = s_tk.seq;
            }
            if (threadIdx.x == 0) {
                if (sv_deps_ready(a, s_tk.dep_slot, s_tk.dep_need, s_tk.join_off, s_tk.join_cnt)) {
                    s_ok = 1;
                } else if (nk >= 0 && nk < k && (dk < 0 || nk < dk)) {
                    // the item claimed ahead is earlier (this one came out of order or was set
                    // aside): run it first, keep this one as the item claimed ahead
                    const long long k2 = nk;
                    const int item2 = nitem, ooo2 = nooo;
                    nk = k, nitem = item, nooo = s_ooo[buf];
                    s_k[buf] = k2, s_item[buf] = item2, s_ooo[buf] = ooo2;
                    s_ok = 2;
                } else if (dk >= 0 && dk < k) {
                    // the item set aside is earlier: run it first, set this one aside instead
                    const long long k2 = dk;
                    const int item2 = ditem;
                    dk = k, ditem = item;
                    s_k[buf] = k2, s_item[buf] = item2, s_ooo[buf] = 0;
                    s_ok = 2;
                } else if (s_ooo[buf] && dk < 0) {
                    // ahead of the cursor and not ready: set it aside and take other work instead
                    dk = k;
                    ditem = item;
                    long long k2 = -1;
                    int item2 = 0, ooo2 = 0;
                    if (nk >= 0) {
                        k2 = nk, item2 = nitem, ooo2 = nooo;
                        nk = -1;
                    } else if (sv_try_claim_settled(a, pub, k2, item2, ooo2) != 1) {
                        k2 = -1;
                    }
                    // nothing claimable now: every published item is held by a running CTA,
                    // its dependencies among them, so run it after all
                    if (k2 < 0 && ld_volatile_s32(&a.ctl->err) == 0) {
                        k2 = dk, item2 = ditem, ooo2 = 0;
                        dk = -1;
                    }
                    s_k[buf] = k2, s_item[buf] = item2, s_ooo[buf] = ooo2;
                    s_ok = 2;
                } else {
                    // the earliest item this CTA holds: its dependencies are earlier still,
                    // so none of them is held here
                    s_ok = sv_wait_deps(a, s_tk) ? 1 : 0;
                }
            }
            __syncthreads();
            if (s_ok == 0) return;   // the launch is failing: every CTA leaves
            if (s_ok == 2) {         // this buffer now names another item: start over
                cur_k = -1;
                continue;
            }
            cur_k = k;
        }
        if (threadIdx.x == 0 && nk < 0) {   // claim the next item while this one runs
            if (sv_try_claim(a, pub, nk, nitem, nooo) != 1) nk = -1;
        }
        const WalkParams& p = s_p;
        TileCtx tc;
        if (s_tk.kind == TK_PROP || s_tk.kind == TK_LEVEL) {
            tc = tile_ctx<CHV>(p, s_tk.tix);
            tc.c0 = s_tk.c0;
        }
        switch (s_tk.kind) {
            case TK_TIMES: item_times(p, s_tk.seed, s_tk.tix, item); break;
            case TK_COEF: item_coef(p); break;
            case TK_PROP: item_props<MODE, CHV>(p, tc, item, smem); break;
            case TK_LEVEL:
                if (!item_level<MODE, V, LAYOUT_WIDE, MODE == COS_MODE_FP64>(p, s_tk.level, tc, item,
                                                                            reinterpret_cast<unsigned char*>(smem)) &&
                    (threadIdx.x & 31) == 0) {
                    const int code = *(volatile int*)&p.ctrl->err;
                    sv_fail(a, code ? code : KERR_BARRIER_TIMEOUT, k);
                }
                break;
            case TK_PARTIALS: item_partials<MODE>(p, item); break;
            case TK_FINAL: item_final(p); break;
            default: break;   // TK_STALL
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s_tk.kind != TK_STALL) {   // release: the item's writes are visible first
                unsigned old;
                asm volatile("atom.release.gpu.global.add.u32 %0, [%1], 1;"
                             : "=r"(old)
                             : "l"(a.done + (k & a.mask))
                             : "memory");
                if (old + 1u == s_tk.need)   // the task's last item: its ring entry may be reused
                    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(a.tdone + (k & a.mask)),
                                 "r"((unsigned)s_tk.self)
                                 : "memory");
            }
            if (s_tk.kind == TK_FINAL) {   // the mean (written above by this thread), then the request number
                SvComp* c = a.comp + s_tk.req;
                asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(&c->seq), "l"((unsigned long long)s_tk.seq)
                             : "memory");
            }
            // the next item: the one set aside once it can run, else the one claimed ahead,
            // else a new claim, else (no other work) the one set aside, waiting for it
            long long k2 = -1;
            int item2 = 0, ooo2 = 0;
            bool ready_aside = false;
            if (dk >= 0) {
                const SvTask* d = a.ring + (dk & a.mask);
                ready_aside = sv_deps_ready(a, __ldcg(&d->dep_slot), __ldcg(&d->dep_need), __ldcg(&d->join_off),
                                            __ldcg(&d->join_cnt));
            }
            if (ready_aside) {
                k2 = dk, item2 = ditem;
                dk = -1;
            } else if (nk >= 0) {
                k2 = nk, item2 = nitem, ooo2 = nooo;
                nk = -1;
            } else if (dk >= 0 ? sv_try_claim_settled(a, pub, k2, item2, ooo2) != 1   // holding one: no idle wait
                               : !sv_claim(a, pub, k2, item2, ooo2)) {
                k2 = -1;
            }
            if (k2 < 0 && dk >= 0 && ld_volatile_s32(&a.ctl->err) == 0) {
                k2 = dk, item2 = ditem, ooo2 = 0;
                dk = -1;
            }
            s_k[buf ^ 1] = k2;
            s_item[buf ^ 1] = item2;
            s_ooo[buf ^ 1] = ooo2;
        }
        __syncthreads();
        buf ^= 1;
    }
}

template <int MODE, int V>
const void* sk() {
    return reinterpret_cast<const void*>(&serve_kernel<MODE, V>);
}

const void* select_serve_kernel(int mode, int vec) {
    switch (mode * 8 + vec) {
        case COS_MODE_FP64 * 8 + 1: return sk<COS_MODE_FP64, 1>();
        case COS_MODE_FP64 * 8 + 2: return sk<COS_MODE_FP64, 2>();
        case COS_MODE_FP64 * 8 + 4: return sk<COS_MODE_FP64, 4>();
        case COS_MODE_FP32_MIXED * 8 + 1: return sk<COS_MODE_FP32_MIXED, 1>();
        case COS_MODE_FP32_MIXED * 8 + 2: return sk<COS_MODE_FP32_MIXED, 2>();
        case COS_MODE_FP32_MIXED * 8 + 4: return sk<COS_MODE_FP32_MIXED, 4>();
        case COS_MODE_COUNT_I64 * 8 + 1: return sk<COS_MODE_COUNT_I64, 1>();
        case COS_MODE_COUNT_I64 * 8 + 2: return sk<COS_MODE_COUNT_I64, 2>();
        case COS_MODE_COUNT_I64 * 8 + 4: return sk<COS_MODE_COUNT_I64, 4>();
        default: return nullptr;
    }
}

// Sources of the published-counter copies: a ring of kPubRing values, reused in
// blocks of kPubBlock once the copies of the block's previous use have run.
constexpr int kPubRing = 4096;
constexpr int kPubBlock = 64;

int64_t pow2_at_least(int64_t x) {
    int64_t c = 1;
    while (c < x) c <<= 1;
    return c;
}

}  // namespace
}  // namespace cosgpu

using namespace cosgpu;

struct cos_server {
    int device = 0;
    int32_t mode = 0;
    int vec = 2;
    int32_t max_D = 0;
    cos_tuning force{};
    int32_t max_req = 0;
    int64_t backlog = 0;             // tasks published ahead of the kernel's cursor at most
    int grid = 0, smem = 0;
    const void* kernel = nullptr;
    long long timeout_ns = 0, idle_ns = 0;
    int test_stale = 0;              // COS_TEST_STALE_CLAIMS (test hook)
    unsigned long long* h_stale = nullptr;   // pinned: stale-claim count read back by stats
    // device
    SvTask* d_ring = nullptr;
    unsigned long long* d_joins = nullptr;
    WalkParams* d_params = nullptr;
    unsigned long long* d_claim = nullptr;
    unsigned* d_done = nullptr;
    SvCtl* d_ctl = nullptr;
    SvPub* d_pub = nullptr;
    // pinned host mirrors (sources of the publishing copies); the ring's in fr
    FeedRing fr;
    WalkParams* h_params = nullptr;
    long long* h_pubval = nullptr;   // [kPubRing]: sources of the counter copies
    cudaEvent_t pub_ev[kPubRing / kPubBlock] = {};
    int64_t n_pub = 0;
    int* h_one = nullptr;            // 1, the shutdown flag's source
    // host-mapped records written by the kernel
    SvComp* h_comp = nullptr;
    SvComp* d_comp = nullptr;
    SvStatus* h_status = nullptr;
    SvStatus* d_status = nullptr;
    unsigned* d_tdone = nullptr;     // device alias of fr.tdone (host-mapped)
    unsigned long long* h_cursor = nullptr;
    unsigned long long* d_cursor = nullptr;
    cudaStream_t ks = nullptr, cs = nullptr;
    cudaEvent_t kdone = nullptr, cev = nullptr;
    bool running = false;
    int failed = 0;                  // cos_status once the kernel has reported an error
    int64_t next_seq = 1;
    struct Req : FeedReq {
        cos_graph_t g = nullptr;
        bool active = false, done = false;
        int overflow = 0;
        int err = 0;
        double mean = 0.0;
    };
    std::vector<Req> reqs;
    std::deque<int32_t> feeding;     // request slots with tasks left to publish, oldest first
    int64_t launches = 0, completed = 0;
};

namespace {

using Srv = cos_server;

int cuda_err(cudaError_t e, const char* what) {
    return set_error(COS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void free_server(Srv* s) {
    cudaFree(s->d_ring);
    cudaFree(s->d_joins);
    cudaFree(s->d_params);
    cudaFree(s->d_claim);
    cudaFree(s->d_done);
    cudaFree(s->d_ctl);
    cudaFree(s->d_pub);
    cudaFreeHost(s->fr.ring);
    cudaFreeHost(s->fr.joins);
    cudaFreeHost(s->h_params);
    cudaFreeHost(s->fr.claim);
    cudaFreeHost(s->h_pubval);
    cudaFreeHost(s->h_one);
    cudaFreeHost(s->h_comp);
    cudaFreeHost(s->h_status);
    cudaFreeHost(s->fr.tdone);
    cudaFreeHost(s->h_cursor);
    cudaFreeHost(s->h_stale);
    for (cudaEvent_t& e : s->pub_ev)
        if (e) cudaEventDestroy(e);
    if (s->kdone) cudaEventDestroy(s->kdone);
    if (s->cev) cudaEventDestroy(s->cev);
    if (s->ks) cudaStreamDestroy(s->ks);
    if (s->cs) cudaStreamDestroy(s->cs);
}

int map_kernel_error(int err) {
    return err == KERR_BARRIER_TIMEOUT ? COS_ERR_TIMEOUT : COS_ERR_CUDA;
}

// Has the kernel left?  Records a kernel-side error as the server's failure.
void check_kernel(Srv* s) {
    if (!s->running) return;
    const cudaError_t q = cudaEventQuery(s->kdone);
    if (q == cudaErrorNotReady) return;
    s->running = false;
    if (q != cudaSuccess) {
        s->failed = COS_ERR_CUDA;
        set_error(COS_ERR_CUDA, "resident kernel: %s", cudaGetErrorString(q));
        return;
    }
    const int err = *(volatile int*)&s->h_status->err;
    if (err != 0 && !s->failed) {
        s->failed = map_kernel_error(err);
        set_error(s->failed, "resident kernel reported error %d at task %lld", err,
                  (long long)*(volatile long long*)&s->h_status->err_task);
    }
}

// Completion records -> requests; ring entries of completed tasks, in order.
void collect(Srv* s) {
    for (int32_t r = 0; r < s->max_req; ++r) {
        Srv::Req& q = s->reqs[(size_t)r];
        if (!q.active || q.done) continue;
        if (*(volatile unsigned long long*)&s->h_comp[r].seq == (unsigned long long)q.seq) {
            __atomic_thread_fence(__ATOMIC_ACQUIRE);
            q.mean = *(volatile double*)&s->h_comp[r].mean;
            q.done = true;
            s->completed++;
        } else if (s->failed) {
            q.err = s->failed;
            q.done = true;
        }
    }
    feed_reclaim(s->fr);
    __atomic_thread_fence(__ATOMIC_ACQUIRE);
}

// Copy entries [first, first + n) of a ring of `cap` entries (wrapping) to the device.
template <typename T>
cudaError_t copy_ring(T* dst, const T* src, int64_t cap, int64_t first, int64_t n, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    while (n > 0 && e == cudaSuccess) {
        const int64_t at = first & (cap - 1);
        const int64_t m = std::min(n, cap - at);
        e = cudaMemcpyAsync(dst + at, src + at, sizeof(T) * (size_t)m, cudaMemcpyHostToDevice, st);
        first += m;
        n -= m;
    }
    return e;
}

// Publish the counter value v: its source stays untouched until the copy has run.
int publish_counter(Srv* s, long long v) {
    const int64_t n = s->n_pub++;
    const int i = (int)(n % kPubRing);
    cudaError_t e = cudaSuccess;
    if (n >= kPubRing && i % kPubBlock == 0) e = cudaEventSynchronize(s->pub_ev[i / kPubBlock]);
    if (e == cudaSuccess) {
        s->h_pubval[i] = v;
        e = cudaMemcpyAsync(&s->d_pub->tasks, s->h_pubval + i, sizeof(long long), cudaMemcpyHostToDevice, s->cs);
    }
    if (e == cudaSuccess && i % kPubBlock == kPubBlock - 1) e = cudaEventRecord(s->pub_ev[i / kPubBlock], s->cs);
    return e == cudaSuccess ? COS_OK : cuda_err(e, "publish counter");
}

// Feed the ring: one task per active request per round, oldest request first, while
// the backlog ahead of the kernel's cursor and the free ring space allow.
int feed(Srv* s) {
    if (s->feeding.empty()) return COS_OK;
    FeedRing& f = s->fr;
    const int64_t cursor = (int64_t)*(volatile unsigned long long*)s->h_cursor;
    const int64_t room = std::min(s->backlog - (f.next_task - cursor), f.cap - (f.next_task - f.tail_task));
    if (room <= 0) return COS_OK;
    const int64_t t0 = f.next_task, j0 = f.next_join;
    if (feed_round_robin(f, s->feeding, room, [s](int32_t r) -> FeedReq& { return s->reqs[(size_t)r]; }) == 0)
        return COS_OK;
    // descriptors and joins, then the claim words (a CTA that finds a new tag may run the
    // task at once), then the counter (one stream, in order)
    cudaError_t e = copy_ring(s->d_ring, f.ring, f.cap, t0, f.next_task - t0, s->cs);
    if (e == cudaSuccess) e = copy_ring(s->d_joins, f.joins, f.jcap, j0, f.next_join - j0, s->cs);
    if (e == cudaSuccess) e = copy_ring(s->d_claim, f.claim, f.cap, t0, f.next_task - t0, s->cs);
    int rc = e == cudaSuccess ? publish_counter(s, f.next_task) : cuda_err(e, "publish tasks");
    if (rc != COS_OK) s->failed = COS_ERR_CUDA;   // the mirrors have moved on: the server cannot continue
    return rc;
}

int launch(Srv* s) {
    ServeArgs a;
    a.ring = s->d_ring;
    a.joins = s->d_joins;
    a.params = s->d_params;
    a.claim = s->d_claim;
    a.done = s->d_done;
    a.ctl = s->d_ctl;
    a.pub = s->d_pub;
    a.comp = s->d_comp;
    a.status = s->d_status;
    a.tdone = s->d_tdone;
    a.cursor_out = s->d_cursor;
    a.mask = s->fr.cap - 1;
    a.jmask = s->fr.jcap - 1;
    a.timeout_ns = s->timeout_ns;
    a.idle_ns = s->idle_ns;
    a.test_stale = s->test_stale;
    a.pad = 0;
    cudaError_t e;
    if ((e = cudaEventRecord(s->cev, s->cs)) != cudaSuccess) return cuda_err(e, "record publish event");
    if ((e = cudaStreamWaitEvent(s->ks, s->cev, 0)) != cudaSuccess) return cuda_err(e, "order launch after publish");
    void* args[] = {&a};
    if ((e = cudaLaunchKernel(s->kernel, dim3((unsigned)s->grid), dim3(kThreads), args, (size_t)s->smem, s->ks)) !=
        cudaSuccess)
        return cuda_err(e, "launch resident kernel");
    if ((e = cudaEventRecord(s->kdone, s->ks)) != cudaSuccess) return cuda_err(e, "record kernel event");
    s->running = true;
    s->launches++;
    return COS_OK;
}

// Kernel exit, completions, feeding, and a relaunch when work is pending and no CTA is left.
int pump(Srv* s) {
    check_kernel(s);
    collect(s);
    if (s->failed) {
        s->feeding.clear();
        return COS_OK;
    }
    int rc = feed(s);
    if (rc != COS_OK || s->running) return rc;
    for (const Srv::Req& q : s->reqs)
        if (q.active && !q.done) return launch(s);
    return COS_OK;
}

int find_request(Srv* s, int64_t id) {
    for (int32_t r = 0; r < s->max_req; ++r)
        if (s->reqs[(size_t)r].active && s->reqs[(size_t)r].seq == id) return r;
    return -1;
}

struct DevSel {
    int prev = -1;
    explicit DevSel(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DevSel() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

int cos_server_create(int32_t mode, int32_t max_times, const cos_tuning* tuning, int32_t max_requests,
                      int64_t queue_tasks, int32_t idle_ms, cos_server_t* out) {
    if (!out) return set_error(COS_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (mode < 0 || mode > 2) return set_error(COS_ERR_INVALID, "bad mode %d", mode);
    if (max_times < 1) return set_error(COS_ERR_INVALID, "max_times must be >= 1");
    if (max_requests < 0 || queue_tasks < 0 || idle_ms < 0)
        return set_error(COS_ERR_INVALID, "max_requests, queue_tasks and idle_ms must be >= 0");
    cos_tuning t{};
    if (tuning) t = *tuning;
    if (t.samples_per_lane > 0 && t.samples_per_lane != 1 && t.samples_per_lane != 2 && t.samples_per_lane != 4)
        return set_error(COS_ERR_INVALID, "samples_per_lane must be 1, 2 or 4");
    if (t.layout > 1) return set_error(COS_ERR_INVALID, "the resident server runs the wide layout (layout 0 or 1)");
    if (t.rows_per_warp > 31) return set_error(COS_ERR_INVALID, "rows_per_warp must be <= 31");
    if (t.window_chunks < 0 || t.prefetch < 0 || t.prefetch > 7)
        return set_error(COS_ERR_INVALID, "window_chunks must be >= 0 and prefetch 0..7");
    int device = -1;
    const cudaError_t de = cudaGetDevice(&device);
    if (de != cudaSuccess) return set_error(COS_ERR_CUDA, "no usable CUDA device: %s", cudaGetErrorString(de));
    Srv* s = new (std::nothrow) Srv();
    if (!s) return set_error(COS_ERR_OOM, "host allocation failed");
    s->device = device;
    s->mode = mode;
    s->vec = t.samples_per_lane > 0 ? t.samples_per_lane : (mode == COS_MODE_FP32_MIXED ? 4 : 2);
    s->max_D = max_times;
    s->force = t;
    s->force.samples_per_lane = s->vec;
    s->force.layout = 1;
    if (s->force.rows_per_warp <= 0) s->force.rows_per_warp = 31;
    s->max_req = max_requests > 0 ? max_requests : 256;
    s->fr.cap = pow2_at_least(std::max<int64_t>(queue_tasks > 0 ? queue_tasks : 65536, 64));
    s->fr.jcap = s->fr.cap;
    s->backlog = std::min<int64_t>(s->fr.cap / 2, 16384);
    s->timeout_ns = (long long)(t.timeout_ms > 0 ? t.timeout_ms : 10000) * 1000000LL;
    s->idle_ns = (long long)(idle_ms > 0 ? idle_ms : 50) * 1000000LL;
    if (const char* env = getenv("COS_TEST_STALE_CLAIMS")) s->test_stale = std::max(0, atoi(env));
    s->kernel = select_serve_kernel(mode, s->vec);
    s->smem = walk_smem_bytes(mode, s->vec, 1, max_times);
    int rc = COS_OK;
    cudaError_t e = cudaSuccess;
    int per_sm = 0, sms = 0;
    if (!s->kernel) {
        rc = set_error(COS_ERR_INVALID, "no resident kernel for samples_per_lane %d", s->vec);
    } else if (prepare_kernel_attrs(s->kernel, s->smem) != COS_OK) {
        rc = set_error(COS_ERR_INVALID, "shared memory for %d time variables exceeds the limit", max_times);
    } else if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, s->kernel, kThreads, s->smem)) !=
                   cudaSuccess ||
               per_sm <= 0) {
        rc = set_error(COS_ERR_CUDA, "occupancy query failed");
    }
    if (rc == COS_OK) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
        const int bps = t.blocks_per_sm > 0 ? std::min(t.blocks_per_sm, per_sm) : per_sm;
        s->force.blocks_per_sm = bps;
        s->grid = sms * bps;
        const size_t nr = (size_t)s->max_req;
        const size_t cap = (size_t)s->fr.cap, jcap = (size_t)s->fr.jcap;
        if ((e = cudaMalloc(&s->d_ring, sizeof(SvTask) * cap)) != cudaSuccess ||
            (e = cudaMalloc(&s->d_joins, sizeof(unsigned long long) * jcap)) != cudaSuccess ||
            (e = cudaMalloc(&s->d_params, sizeof(WalkParams) * nr)) != cudaSuccess ||
            (e = cudaMalloc(&s->d_claim, sizeof(unsigned long long) * cap)) != cudaSuccess ||
            (e = cudaMalloc(&s->d_done, sizeof(unsigned) * cap)) != cudaSuccess ||
            (e = cudaMalloc(&s->d_ctl, sizeof(SvCtl))) != cudaSuccess ||
            (e = cudaMalloc(&s->d_pub, sizeof(SvPub))) != cudaSuccess ||
            (e = cudaMallocHost(&s->fr.ring, sizeof(SvTask) * cap)) != cudaSuccess ||
            (e = cudaMallocHost(&s->fr.joins, sizeof(unsigned long long) * jcap)) != cudaSuccess ||
            (e = cudaMallocHost(&s->h_params, sizeof(WalkParams) * nr)) != cudaSuccess ||
            (e = cudaMallocHost(&s->fr.claim, sizeof(unsigned long long) * cap)) != cudaSuccess ||
            (e = cudaMallocHost(&s->h_pubval, sizeof(long long) * kPubRing)) != cudaSuccess ||
            (e = cudaMallocHost(&s->h_one, sizeof(int))) != cudaSuccess ||
            (e = cudaMallocHost(&s->h_stale, sizeof(unsigned long long))) != cudaSuccess ||
            (e = cudaHostAlloc(&s->h_comp, sizeof(SvComp) * nr, cudaHostAllocMapped)) != cudaSuccess ||
            (e = cudaHostAlloc(&s->h_status, sizeof(SvStatus), cudaHostAllocMapped)) != cudaSuccess ||
            (e = cudaHostAlloc(&s->fr.tdone, sizeof(unsigned) * cap, cudaHostAllocMapped)) != cudaSuccess ||
            (e = cudaHostAlloc(&s->h_cursor, sizeof(unsigned long long), cudaHostAllocMapped)) != cudaSuccess ||
            (e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->d_comp), s->h_comp, 0)) != cudaSuccess ||
            (e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->d_status), s->h_status, 0)) != cudaSuccess ||
            (e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->d_tdone), s->fr.tdone, 0)) != cudaSuccess ||
            (e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->d_cursor), s->h_cursor, 0)) != cudaSuccess)
            rc = set_error(COS_ERR_OOM, "server buffers: %s", cudaGetErrorString(e));
    }
    if (rc == COS_OK) {
        memset(s->h_comp, 0, sizeof(SvComp) * (size_t)s->max_req);
        memset(s->h_status, 0, sizeof(SvStatus));
        s->fr.reset();
        *s->h_cursor = 0;
        *s->h_one = 1;
        if ((e = cudaMemset(s->d_claim, 0, sizeof(unsigned long long) * (size_t)s->fr.cap)) != cudaSuccess ||
            (e = cudaMemset(s->d_done, 0, sizeof(unsigned) * (size_t)s->fr.cap)) != cudaSuccess ||
            (e = cudaMemset(s->d_ctl, 0, sizeof(SvCtl))) != cudaSuccess ||
            (e = cudaMemset(s->d_pub, 0, sizeof(SvPub))) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&s->ks, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&s->cs, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&s->kdone, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&s->cev, cudaEventDisableTiming)) != cudaSuccess)
            rc = cuda_err(e, "server set-up");
        for (cudaEvent_t& ev : s->pub_ev)
            if (rc == COS_OK && (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
                rc = cuda_err(e, "server set-up");
        if (rc == COS_OK && (e = cudaDeviceSynchronize()) != cudaSuccess) rc = cuda_err(e, "server set-up");
    }
    if (rc != COS_OK) {
        free_server(s);
        delete s;
        return rc;
    }
    s->reqs.assign((size_t)s->max_req, Srv::Req{});
    *out = s;
    return COS_OK;
}

int cos_server_submit(cos_server_t s, cos_graph_t g, int64_t num_samples, uint64_t seed, int64_t first_sample,
                      void* per_sample_out, int64_t* request_id) {
    if (!s || !g || !request_id) return set_error(COS_ERR_INVALID, "bad arguments");
    if (!per_sample_out) return set_error(COS_ERR_INVALID, "per_sample_out is required");
    if (num_samples < 0 || first_sample < 0) return set_error(COS_ERR_INVALID, "num_samples and first_sample must be >= 0");
    DevSel dev(s->device);
    int rc = pump(s);
    if (rc != COS_OK) return rc;
    if (s->failed) return set_error(s->failed, "the server has failed; destroy it");
    GraphView gv;
    if ((rc = graph_view(g, &gv)) != COS_OK) return rc;
    if (gv.device != s->device) return set_error(COS_ERR_INVALID, "graph and server are on different devices");
    if (gv.D > s->max_D) return set_error(COS_ERR_INVALID, "graph has %d time variables; the server was made for %d", gv.D, s->max_D);
    int32_t slot = -1;
    for (int32_t r = 0; r < s->max_req; ++r) {
        const Srv::Req& q = s->reqs[(size_t)r];
        if (q.active && q.g == g) return set_error(COS_ERR_STATE, "the handle is in use by request %lld", (long long)q.seq);
        if (!q.active && slot < 0) slot = r;
    }
    if (slot < 0) return set_error(COS_ERR_BUSY, "all %d request slots are in use", s->max_req);
    SampleState undo;
    if ((rc = attach_own_samples(g, num_samples, &undo)) != COS_OK) return rc;
    WalkParams p;
    cos_tuning tn;
    rc = prepare_walk(g, s->mode, &s->force, per_sample_out, &p, &tn);
    if (rc == COS_OK && (tn.samples_per_lane != s->vec || tn.layout != 1))
        rc = set_error(COS_ERR_INVALID, "graph needs samples_per_lane %d; the server runs %d", tn.samples_per_lane, s->vec);
    if (rc != COS_OK) {
        restore_samples(g, undo);
        return rc;
    }
    p.mean_out = &s->d_comp[slot].mean;
    Srv::Req& q = s->reqs[(size_t)slot];
    q = Srv::Req{};
    graph_task_chain(p, gv.widths_host, s->mode, 32 * s->vec,
                     s->force.window_chunks > 0 ? s->force.window_chunks : tn.window_chunks, slot,
                     s->mode != COS_MODE_COUNT_I64, getenv("COS_TEST_STALL_TASK") != nullptr, q.tasks, q.joins);
    if ((int64_t)feed_max_joins(q) > s->fr.jcap) {
        const size_t need = feed_max_joins(q);
        q = Srv::Req{};
        restore_samples(g, undo);
        return set_error(COS_ERR_INVALID, "request joins %zu windows in one task; the queue holds %lld (raise queue_tasks)",
                         need, (long long)s->fr.jcap);
    }
    s->h_params[slot] = p;
    // the parameters go ahead of every counter copy that publishes one of the request's tasks
    cudaError_t e = cudaMemcpyAsync(s->d_params + slot, s->h_params + slot, sizeof(WalkParams), cudaMemcpyHostToDevice, s->cs);
    if (e != cudaSuccess) {
        q = Srv::Req{};
        restore_samples(g, undo);
        return cuda_err(e, "copy request parameters");
    }
    q.seq = s->next_seq++;
    q.g = g;
    q.active = true;
    q.seed = seed;
    q.first_sample = first_sample;
    q.overflow = s->mode == COS_MODE_COUNT_I64 && gv.count_overflow;
    q.slot_of.reserve(q.tasks.size());
    q.need_of.reserve(q.tasks.size());
    s->feeding.push_back(slot);
    *request_id = q.seq;
    return pump(s);
}

int cos_server_poll(cos_server_t s, int64_t request_id, double* mean_out) {
    if (!s) return set_error(COS_ERR_INVALID, "server is NULL");
    DevSel dev(s->device);
    const int r = find_request(s, request_id);
    if (r < 0) return set_error(COS_ERR_INVALID, "unknown or already collected request %lld", (long long)request_id);
    int rc = pump(s);
    if (rc != COS_OK) return rc;
    Srv::Req& q = s->reqs[(size_t)r];
    if (!q.done) return COS_ERR_BUSY;
    const int err = q.err, overflow = q.overflow;
    const double mean = q.mean;
    q = Srv::Req{};
    if (err) return set_error(err, "request %lld failed: %s", (long long)request_id, cos_last_error());
    if (mean_out) *mean_out = mean;
    if (overflow) return set_error(COS_ERR_OVERFLOW, "path count exceeds 2^63-1; results wrap modulo 2^64");
    return COS_OK;
}

int cos_server_wait(cos_server_t s, int64_t request_id, int32_t timeout_ms, double* mean_out) {
    if (!s) return set_error(COS_ERR_INVALID, "server is NULL");
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const int rc = cos_server_poll(s, request_id, mean_out);
        if (rc != COS_ERR_BUSY) return rc;
        const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
        if (timeout_ms >= 0 && ms > timeout_ms)
            return set_error(COS_ERR_TIMEOUT, "request %lld not complete after %d ms", (long long)request_id, timeout_ms);
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

int cos_server_stats(cos_server_t s, cos_server_info* info) {
    if (!s || !info) return set_error(COS_ERR_INVALID, "bad arguments");
    DevSel dev(s->device);
    int rc = pump(s);
    if (rc != COS_OK) return rc;
    memset(info, 0, sizeof(*info));
    info->launches = s->launches;
    info->completed = s->completed;
    for (const Srv::Req& q : s->reqs) info->in_flight += (q.active && !q.done) ? 1 : 0;
    info->queued_tasks = s->fr.next_task - s->fr.tail_task;
    info->published_tasks = s->fr.next_task;
    info->running = s->running ? 1 : 0;
    info->grid = s->grid;
    info->samples_per_lane = s->vec;
    info->failed = s->failed;
    cudaError_t e = cudaMemcpyAsync(s->h_stale, &s->d_ctl->stale_claims, sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, s->cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->cs);
    if (e != cudaSuccess) return cuda_err(e, "read claim counters");
    info->stale_claims = (int64_t)*s->h_stale;
    return COS_OK;
}

int cos_server_destroy(cos_server_t s) {
    if (!s) return COS_OK;
    int rc = COS_OK;
    {
        DevSel dev(s->device);
        // finish every submitted request (the host keeps feeding), unless the server failed
        for (;;) {
            if (pump(s) != COS_OK) break;
            bool pending = false;
            for (const Srv::Req& q : s->reqs) pending |= q.active && !q.done;
            if (!pending || s->failed) break;
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
        if (s->running) {
            // ask the CTAs to leave once the published work is done, then wait for them
            cudaError_t e = cudaMemcpyAsync(&s->d_pub->shutdown, s->h_one, sizeof(int), cudaMemcpyHostToDevice, s->cs);
            if (e == cudaSuccess) e = cudaEventSynchronize(s->kdone);
            if (e != cudaSuccess) rc = cuda_err(e, "stop resident kernel");
            s->running = false;
        }
        free_server(s);
    }
    delete s;
    return rc;
}

}  // extern "C"
