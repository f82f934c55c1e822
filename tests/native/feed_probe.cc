// Host-only probe of the resident server's feeder (cos_feed.h), driven against a
// simulated device.  Requests with random task chains (graph_task_chain) arrive,
// the feeder stages them round-robin into a small ring within a backlog, the
// simulated device completes staged tasks whose dependencies are complete (read
// from the staged entries, as the kernel does), flags them, and the feeder
// reclaims ring entries in order.  Every staged entry is checked against an
// independent record of the chains:
//   - the entry's fields and its claim word;
//   - its completion value (items of all tasks the slot has held);
//   - the (slot, value) of its dependency and joins;
//   - the previous occupant of the slot being complete;
//   - zero-item tasks flagged at once;
//   - the backlog and ring bounds;
//   - round-robin fairness within a feeding call.
// The run must finish every request.  Prints "ok <tasks> <requests>" or the first
// violated check.
//
// usage: feed_probe seed cap backlog max_active requests
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <deque>
#include <map>
#include <random>
#include <vector>

#include "../../paper_2501_00675_gb300/csrc/cos_feed.h"

using namespace cosgpu;

#define CHECK(cond, ...)                      \
    do {                                      \
        if (!(cond)) {                        \
            std::printf("FAIL: " __VA_ARGS__); \
            std::printf("\n");                \
            return 1;                         \
        }                                     \
    } while (0)

struct Shadow {            // independent record of a staged task
    int32_t req;
    int32_t local;
    int32_t items;
    int64_t slot;
    uint32_t need;
    bool complete;
};

int main(int argc, char** argv) {
    if (argc < 6) {
        std::fprintf(stderr, "usage: %s seed cap backlog max_active requests\n", argv[0]);
        return 2;
    }
    std::mt19937_64 rng(std::strtoull(argv[1], nullptr, 10));
    const int64_t cap = std::atoll(argv[2]);
    const int64_t backlog = std::atoll(argv[3]);
    const int max_active = std::atoi(argv[4]);
    const int total_requests = std::atoi(argv[5]);
    auto uni = [&](int64_t lo, int64_t hi) { return lo + (int64_t)(rng() % (uint64_t)(hi - lo + 1)); };

    std::vector<SvTask> ring((size_t)cap);
    std::vector<unsigned long long> joins((size_t)cap), claim((size_t)cap);
    std::vector<unsigned> tdone((size_t)cap);
    FeedRing f;
    f.cap = f.jcap = cap;
    f.ring = ring.data();
    f.joins = joins.data();
    f.claim = claim.data();
    f.tdone = tdone.data();
    f.reset();

    std::vector<FeedReq> reqs((size_t)max_active);
    std::vector<int> active((size_t)max_active, 0);
    std::vector<std::vector<int64_t>> abs_of((size_t)max_active);   // absolute index of each staged local task
    std::deque<int32_t> feeding;
    std::vector<Shadow> shadow;                  // by absolute task index
    std::vector<uint32_t> slot_sum((size_t)cap, 0);
    std::vector<uint32_t> done((size_t)cap, 0);  // the device's cumulative counters
    int submitted = 0, finished = 0;
    int64_t seq = 0, cursor = 0;
    for (int64_t step = 0; step < 2000000 && finished < total_requests; ++step) {
        // arrivals
        for (int r = 0; r < max_active && submitted < total_requests; ++r) {
            if (active[(size_t)r] || uni(0, 3) != 0) continue;
            FeedReq& q = reqs[(size_t)r];
            q = FeedReq{};
            WalkParams p{};
            p.S = uni(0, 3000);
            p.tile = 64 * uni(1, 20);
            const int chv = uni(0, 1) ? 64 : 128;
            p.K = (int32_t)uni(1, 4);
            p.rows_per_warp = (int32_t)uni(1, 31);
            p.t_ld = std::max<int64_t>(128, (p.S + 127) / 128 * 128);
            std::vector<int64_t> widths(1, 1);
            const int L = (int)uni(2, 6);
            for (int l = 1; l + 1 < L; ++l) widths.push_back(uni(1, 600));
            widths.push_back(1);
            p.L = L;
            const int mode = (int)uni(0, 2);
            graph_task_chain(p, widths.data(), mode, chv, (int)uni(0, 5), r, mode != 2, false, q.tasks, q.joins);
            if ((int64_t)feed_max_joins(q) > f.jcap) continue;   // the server refuses it at submit
            q.seq = ++seq;
            q.seed = rng();
            q.first_sample = uni(0, 1 << 20);
            abs_of[(size_t)r].clear();
            active[(size_t)r] = 1;
            feeding.push_back(r);
            ++submitted;
        }
        // feed, as the server does: within the backlog ahead of the cursor and the free ring
        const int64_t room = std::min(backlog - (f.next_task - cursor), f.cap - (f.next_task - f.tail_task));
        if (room > 0 && !feeding.empty()) {
            std::map<int32_t, size_t> before;
            for (int32_t r : feeding) before[r] = reqs[(size_t)r].next;
            const int64_t t0 = f.next_task;
            const int64_t n = feed_round_robin(f, feeding, room, [&](int32_t r) -> FeedReq& { return reqs[(size_t)r]; });
            CHECK(n <= room && f.next_task - f.tail_task <= cap, "bounds: staged %lld room %lld", (long long)n,
                  (long long)room);
            // fairness: requests that still had tasks at the end got within one task of each other
            size_t lo = SIZE_MAX, hi = 0;
            for (auto& kv : before) {
                const FeedReq& q = reqs[(size_t)kv.first];
                if (q.next >= q.tasks.size()) continue;   // ran out of tasks: may have got fewer
                const size_t got = q.next - kv.second;
                lo = std::min(lo, got), hi = std::max(hi, got);
            }
            CHECK(lo == SIZE_MAX || hi <= lo + 1, "round-robin: %zu vs %zu tasks in one call", lo, hi);
            for (int64_t t = t0; t < f.next_task; ++t) {
                const int64_t at = t & (cap - 1);
                const SvTask& e = ring[(size_t)at];
                CHECK(e.self == t, "entry %lld self %lld", (long long)t, (long long)e.self);
                CHECK(t < cap || shadow[(size_t)(t - cap)].complete, "slot %lld reused before task %lld completed",
                      (long long)at, (long long)(t - cap));
                const int32_t r = e.req;
                FeedReq& q = reqs[(size_t)r];
                const int32_t li = (int32_t)abs_of[(size_t)r].size();
                abs_of[(size_t)r].push_back(t);
                const Task& tk = q.tasks[(size_t)li];
                CHECK(e.seq == q.seq && e.kind == tk.kind && e.level == tk.level && e.items == tk.items &&
                          e.c0 == tk.c0 && e.seed == q.seed,
                      "entry %lld fields", (long long)t);
                CHECK(e.tix == (tk.kind == TK_TIMES ? q.first_sample : tk.tix), "entry %lld tix", (long long)t);
                slot_sum[(size_t)at] += (uint32_t)tk.items;
                CHECK(e.need == slot_sum[(size_t)at], "entry %lld completion value", (long long)t);
                CHECK(claim[(size_t)at] == (((unsigned long long)(uint32_t)t << 32) | (0x80000000ull + (uint32_t)tk.items)),
                      "entry %lld claim word", (long long)t);
                if (tk.dep >= 0) {
                    const Shadow& d = shadow[(size_t)abs_of[(size_t)r][(size_t)tk.dep]];
                    CHECK(e.dep_slot == d.slot && e.dep_need == d.need, "entry %lld dependency", (long long)t);
                } else {
                    CHECK(e.dep_slot == -1, "entry %lld spurious dependency", (long long)t);
                }
                CHECK(e.join_cnt == (int32_t)q.joins[(size_t)li].size(), "entry %lld join count", (long long)t);
                for (int32_t j = 0; j < e.join_cnt; ++j) {
                    const Shadow& d = shadow[(size_t)abs_of[(size_t)r][(size_t)q.joins[(size_t)li][(size_t)j]]];
                    CHECK(joins[(size_t)((e.join_off + j) & (cap - 1))] ==
                              (((unsigned long long)(uint32_t)d.slot << 32) | d.need),
                          "entry %lld join %d", (long long)t, j);
                }
                CHECK(tk.items != 0 || tdone[(size_t)at] == (unsigned)t, "zero-item task %lld not flagged", (long long)t);
                shadow.push_back(Shadow{r, li, tk.items, at, e.need, tk.items == 0});
            }
        }
        // the device: complete a few staged tasks whose dependencies are complete, as read
        // from their entries; the cursor follows the lowest task not yet complete
        for (int k = 0; k < 3; ++k) {
            const int64_t span = f.next_task - cursor;
            if (span <= 0) break;
            const int64_t t = cursor + uni(0, span - 1);
            Shadow& sh = shadow[(size_t)t];
            if (sh.complete) continue;
            const SvTask& e = ring[(size_t)(t & (cap - 1))];
            bool ready = e.dep_slot < 0 || (int32_t)(done[(size_t)e.dep_slot] - e.dep_need) >= 0;
            for (int32_t j = 0; ready && j < e.join_cnt; ++j) {
                const unsigned long long w = joins[(size_t)((e.join_off + j) & (cap - 1))];
                ready = (int32_t)(done[(size_t)(w >> 32)] - (uint32_t)w) >= 0;
            }
            if (!ready) continue;
            const Task& tk = reqs[(size_t)sh.req].tasks[(size_t)sh.local];   // the chain's own dependencies
            if (tk.dep >= 0) CHECK(shadow[(size_t)abs_of[(size_t)sh.req][(size_t)tk.dep]].complete, "ran early");
            for (int32_t d : reqs[(size_t)sh.req].joins[(size_t)sh.local])
                CHECK(shadow[(size_t)abs_of[(size_t)sh.req][(size_t)d]].complete, "ran before a join");
            done[(size_t)sh.slot] += (uint32_t)sh.items;
            CHECK(done[(size_t)sh.slot] == sh.need, "counter of task %lld", (long long)t);
            tdone[(size_t)sh.slot] = (unsigned)t;
            sh.complete = true;
        }
        while (cursor < f.next_task && shadow[(size_t)cursor].complete) ++cursor;
        feed_reclaim(f);
        CHECK(f.tail_task <= cursor, "tail %lld passed an incomplete task", (long long)f.tail_task);
        // requests whose tasks are all staged and complete finish
        for (int r = 0; r < max_active; ++r) {
            if (!active[(size_t)r]) continue;
            const FeedReq& q = reqs[(size_t)r];
            if (q.next < q.tasks.size()) continue;
            bool all = true;
            for (int64_t t : abs_of[(size_t)r]) all = all && shadow[(size_t)t].complete;
            if (all) active[(size_t)r] = 0, ++finished;
        }
    }
    CHECK(finished == total_requests, "stalled: %d of %d requests finished", finished, total_requests);
    std::printf("ok %lld %d\n", (long long)f.next_task, finished);
    return 0;
}
