// Host side of the resident server's task ring (cos_serve.cu): the entry format the
// kernel reads, the host mirrors that the publishing copies read, and the feeder
// that stages the active requests' task chains into the ring round-robin and
// reuses ring entries in order once the kernel has flagged them complete.  Host
// code only (no CUDA calls), so that the feeder can be exercised on its own.
#pragma once

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <deque>
#include <vector>

#include "cos_tasks.cuh"

namespace cosgpu {

// One ring entry (task descriptor), as the kernel reads it.
struct SvTask {
    int64_t self;       // absolute task index (publication order); its ring slot is self & mask
    int64_t seq;        // request number (key of the CTAs' parameter cache)
    int64_t tix;        // tile index (TK_TIMES: number of the request's first sample)
    int64_t join_off;   // absolute index of the first join entry
    uint64_t seed;      // TK_TIMES: generator key
    int32_t req;        // request slot: walker parameters and completion record
    int32_t kind;
    int32_t level;
    int32_t items;
    int32_t c0;
    int32_t join_cnt;
    int32_t dep_slot;   // ring slot of the task that must be complete first, or -1 ...
    uint32_t dep_need;  // ... and the value that slot's counter has reached then
    uint32_t need;      // value of done[self & mask] once this task is complete
    int32_t pad;
};
static_assert(sizeof(SvTask) % 8 == 0, "descriptor is copied as 8-byte words");

// Claim word of a freshly published task: its tag (the low 32 bits of its absolute
// index) and, counted down from a bias of 2^31, the items not yet handed out.
inline unsigned long long claim_word(int64_t self, int32_t items) {
    return ((unsigned long long)(uint32_t)self << 32) | (0x80000000ull + (uint32_t)items);
}

// A request's task chain (graph_task_chain) and how far it has been staged.
struct FeedReq {
    int64_t seq = 0;
    uint64_t seed = 0;
    int64_t first_sample = 0;
    std::vector<Task> tasks;                 // local dep and join indices
    std::vector<std::vector<int32_t>> joins;
    size_t next = 0;                         // tasks staged so far
    std::vector<int32_t> slot_of;            // ring slot of each staged task
    std::vector<uint32_t> need_of;           // its completion value
};

// The ring as the host sees it.  The four arrays are the sources of the publishing
// copies (tdone: written by the kernel, tag of the last task completed per slot);
// the counters are absolute indices.
struct FeedRing {
    int64_t cap = 0, jcap = 0;               // powers of two
    SvTask* ring = nullptr;                  // [cap]
    unsigned long long* joins = nullptr;     // [jcap]: (slot << 32) | completion value
    unsigned long long* claim = nullptr;     // [cap]
    unsigned* tdone = nullptr;               // [cap]
    std::vector<uint32_t> slot_total;        // per slot: items of every task it has held
    std::vector<int64_t> join_end;           // per slot: next_join after its task's joins
    int64_t next_task = 0, tail_task = 0, next_join = 0, tail_join = 0;

    // Counters and per-slot bookkeeping for empty mirrors of cap / jcap entries.
    void reset() {
        slot_total.assign((size_t)cap, 0u);
        join_end.assign((size_t)cap, 0);
        next_task = tail_task = next_join = tail_join = 0;
        for (int64_t i = 0; i < cap; ++i) tdone[i] = (unsigned)(i - cap);   // no task's tag yet
    }
};

// Join entries of the request's most-joining task: it can only be staged if the
// join ring holds that many (a request needing more can never run).
inline size_t feed_max_joins(const FeedReq& q) {
    size_t m = 0;
    for (const auto& j : q.joins) m = std::max(m, j.size());
    return m;
}

// Stage task q.next of the request in slot r at ring position next_task.
inline void feed_stage(FeedRing& f, FeedReq& q, int32_t r) {
    const size_t li = q.next++;
    const Task& t = q.tasks[li];
    const int64_t self = f.next_task++;
    const int64_t at = self & (f.cap - 1);
    SvTask& e = f.ring[at];
    memset(&e, 0, sizeof(e));
    e.self = self;
    e.seq = q.seq;
    e.tix = t.kind == TK_TIMES ? q.first_sample : t.tix;
    e.seed = q.seed;
    e.req = r;
    e.kind = t.kind;
    e.level = t.level;
    e.items = t.items;
    e.c0 = t.c0;
    e.dep_slot = t.dep >= 0 ? q.slot_of[(size_t)t.dep] : -1;
    e.dep_need = t.dep >= 0 ? q.need_of[(size_t)t.dep] : 0u;
    e.join_off = f.next_join;
    e.join_cnt = (int32_t)q.joins[li].size();
    for (int32_t d : q.joins[li])
        f.joins[f.next_join++ & (f.jcap - 1)] =
            ((unsigned long long)(uint32_t)q.slot_of[(size_t)d] << 32) | q.need_of[(size_t)d];
    f.slot_total[(size_t)at] += (uint32_t)t.items;
    e.need = f.slot_total[(size_t)at];
    f.join_end[(size_t)at] = f.next_join;
    f.claim[at] = claim_word(self, t.items);
    q.slot_of.push_back((int32_t)at);
    q.need_of.push_back(e.need);
    if (t.items == 0) *(volatile unsigned*)&f.tdone[at] = (unsigned)self;   // complete as soon as published
}

// Move the tail over the tasks flagged complete, in order (their entries may be reused).
inline void feed_reclaim(FeedRing& f) {
    while (f.tail_task < f.next_task) {
        const int64_t at = f.tail_task & (f.cap - 1);
        if (*(volatile unsigned*)&f.tdone[at] != (unsigned)f.tail_task) break;
        f.tail_join = f.join_end[(size_t)at];
        f.tail_task++;
    }
}

// Stage up to `room` tasks, one per request per round in the order of `feeding`
// (request slots, oldest first), as long as the join ring has space; drop the
// requests whose chains are fully staged from `feeding`.  req_at(r) gives the
// FeedReq of request slot r.  Returns the number of tasks staged.
template <typename ReqAt>
inline int64_t feed_round_robin(FeedRing& f, std::deque<int32_t>& feeding, int64_t room, ReqAt req_at) {
    const int64_t t0 = f.next_task;
    bool progress = true;
    while (room > 0 && progress) {
        progress = false;
        for (int32_t r : feeding) {
            if (room <= 0) break;
            FeedReq& q = req_at(r);
            if (q.next >= q.tasks.size()) continue;
            if (f.next_join + (int64_t)q.joins[q.next].size() - f.tail_join > f.jcap) {
                room = 0;
                break;
            }
            feed_stage(f, q, r);
            --room;
            progress = true;
        }
    }
    for (auto it = feeding.begin(); it != feeding.end();) {
        const FeedReq& q = req_at(*it);
        it = q.next >= q.tasks.size() ? feeding.erase(it) : it + 1;
    }
    return f.next_task - t0;
}

}  // namespace cosgpu
