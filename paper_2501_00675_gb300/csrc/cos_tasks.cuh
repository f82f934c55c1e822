// Work-queue tasks of one graph evaluation: the host-side chain builder shared by
// the batched launch (cos_batch.cu) and the resident server (cos_serve.cu).
//
// A graph contributes (optionally) a task that draws its sample times, its
// coefficients task, then per window of sample chunks a chain of phase tasks --
// per tile of samples: propagators, levels 1..L-1 -- then the partial sums
// (waiting for every window) and the final mean.  Without windows a tile is one
// window.  The window chains are laid out in wavefront order (step d holds phase
// d - w of window w), so about L windows are in flight and their node values and
// propagators are re-read while still in L2 (Sec. II.C: levels evaluated
// asynchronously).
#pragma once

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "cos_internal.cuh"

namespace cosgpu {

// TK_STALL: a test-only task (COS_TEST_STALL_TASK) that is drawn but never counted
// done, so that a dependency wait on it runs into its time limit.
// TK_TIMES: counter-based uniform sample times of a request (resident server).
enum TaskKind : int32_t {
    TK_COEF = 0, TK_PROP = 1, TK_LEVEL = 3, TK_PARTIALS = 4, TK_FINAL = 5, TK_STALL = 6, TK_TIMES = 7
};

struct Task {
    int32_t graph;      // index into the parameter array
    int32_t kind;
    int32_t level;
    int32_t dep;        // task that must be complete first (-1: none)
    int64_t tix;        // tile index
    int64_t first;      // first ticket of this task
    int32_t items;
    int32_t c0;         // first chunk of the task's window within the tile
    int32_t join_off;   // further tasks that must be complete: joins[join_off .. +join_cnt)
    int32_t join_cnt;
};

// Samples filled per TK_TIMES item (all D time rows of these sample columns).
constexpr int kTimesPerItem = 4096;

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Append the task chain of one graph evaluation to `out` (and one join list per
// task to `joins`) in issue order; dep and join entries count from the first task
// appended by this call (0).
//   p, widths    the graph's walker parameters and host level widths
//   chv          samples per chunk of the launch's kernel
//   window_chunks  > 0: windows of that many chunks; 0: one window per tile
//   graph        value of Task::graph for every task
//   times        prepend a TK_TIMES task (items cover t_ld sample columns)
//   stall        add a TK_STALL task that the final task joins (test hook)
inline void graph_task_chain(const WalkParams& p, const int64_t* widths, int mode, int chv, int window_chunks,
                             int32_t graph, bool times, bool stall, std::vector<Task>& out,
                             std::vector<std::vector<int32_t>>& joins) {
    const size_t base = out.size();
    auto make = [&](int32_t kind, int32_t level, int64_t tix, int64_t items, int32_t c0) {
        Task t;
        memset(&t, 0, sizeof(t));
        t.graph = graph;
        t.kind = kind;
        t.level = level;
        t.tix = tix;
        t.items = (int32_t)items;
        t.c0 = c0;
        t.dep = -1;
        return t;
    };
    auto emit = [&](const Task& t, std::vector<int32_t> js) {
        out.push_back(t);
        joins.push_back(std::move(js));
        return (int32_t)(out.size() - 1 - base);
    };
    int32_t first = -1;
    if (times) first = emit(make(TK_TIMES, 0, 0, div_up(p.t_ld, kTimesPerItem), 0), {});
    int32_t coef = first;
    if (mode != COS_MODE_COUNT_I64) {
        Task c = make(TK_COEF, 0, 0, 1, 0);
        c.dep = first;
        coef = emit(c, {});
    }
    const int64_t ntiles = p.S > 0 ? (p.S + p.tile - 1) / p.tile : 0;
    const int nch_max = p.S > 0 ? div_up(std::min<int64_t>(p.tile, p.S), chv) : 0;
    const int wch = window_chunks > 0 ? std::min(window_chunks, std::max(nch_max, 1)) : std::max(nch_max, 1);
    const int nw = nch_max > 0 ? div_up(nch_max, wch) : 0;
    const int rows_per_item = kWarps * p.rows_per_warp;
    std::vector<std::vector<Task>> chains((size_t)nw);
    for (int64_t tix = 0; tix < ntiles; ++tix) {
        const int64_t nsamp = std::min(p.tile, p.S - tix * p.tile);
        const int nch = div_up(nsamp, chv);
        for (int w = 0; w < nw; ++w) {
            const int c0 = w * wch;
            if (c0 >= nch) break;
            const int n_w = std::min(wch, nch - c0);
            chains[(size_t)w].push_back(
                make(TK_PROP, 0, tix, mode == COS_MODE_COUNT_I64 ? n_w : (int64_t)n_w * p.K, c0));
            for (int l = 1; l < p.L; ++l)
                chains[(size_t)w].push_back(make(TK_LEVEL, l, tix, (int64_t)n_w * div_up(widths[l], rows_per_item), c0));
        }
    }
    // wavefront: step d issues phase d - w of window w, oldest window first
    std::vector<int32_t> last((size_t)nw, coef);
    size_t maxlen = 0;
    for (auto& ch : chains) maxlen = std::max(maxlen, ch.size());
    for (size_t d = 0; d + 1 < maxlen + (size_t)nw; ++d)
        for (int w = 0; w < nw; ++w) {
            if ((size_t)w > d) break;
            const size_t ph = d - (size_t)w;
            if (ph >= chains[(size_t)w].size()) continue;
            Task t = chains[(size_t)w][ph];
            t.dep = last[(size_t)w];
            last[(size_t)w] = emit(t, {});
        }
    // the sample reduction waits for every window; the final mean for the reduction
    Task part = make(TK_PARTIALS, 0, 0, div_up(div_up(p.S, kReduceBlock), kWarps), 0);
    part.dep = coef;
    std::vector<int32_t> js;
    for (int w = 0; w < nw; ++w)
        if (last[(size_t)w] != coef) js.push_back(last[(size_t)w]);
    const int32_t ip = emit(part, std::move(js));
    Task fin = make(TK_FINAL, 0, 0, 1, 0);
    fin.dep = ip;
    std::vector<int32_t> st;
    if (stall) st.push_back(emit(make(TK_STALL, 0, 0, 1, 0), {}));
    emit(fin, std::move(st));
}

}  // namespace cosgpu
