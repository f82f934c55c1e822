// Host-only probe of the work-queue task chain builder (graph_task_chain): builds
// the chain of one graph evaluation from the parameters on the command line and
// prints one line per task, "kind level tix items c0 dep joins" (joins as a
// comma-separated list, "-" when empty), for the tests to check.
//
// usage: task_chain_probe mode S tile chv K rows_per_warp window_chunks times stall t_ld w_0 ... w_{L-1}
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_2501_00675_gb300/csrc/cos_tasks.cuh"

int main(int argc, char** argv) {
    if (argc < 12) {
        std::fprintf(stderr, "usage: %s mode S tile chv K rows_per_warp window_chunks times stall t_ld w_0 ...\n", argv[0]);
        return 2;
    }
    const int mode = std::atoi(argv[1]);
    cosgpu::WalkParams p{};
    p.S = std::atoll(argv[2]);
    p.tile = std::atoll(argv[3]);
    const int chv = std::atoi(argv[4]);
    p.K = std::atoi(argv[5]);
    p.rows_per_warp = std::atoi(argv[6]);
    const int window_chunks = std::atoi(argv[7]);
    const bool times = std::atoi(argv[8]) != 0;
    const bool stall = std::atoi(argv[9]) != 0;
    p.t_ld = std::atoll(argv[10]);
    std::vector<int64_t> widths;
    for (int a = 11; a < argc; ++a) widths.push_back(std::atoll(argv[a]));
    p.L = (int32_t)widths.size();
    std::vector<cosgpu::Task> tasks;
    std::vector<std::vector<int32_t>> joins;
    cosgpu::graph_task_chain(p, widths.data(), mode, chv, window_chunks, 0, times, stall, tasks, joins);
    for (size_t i = 0; i < tasks.size(); ++i) {
        const cosgpu::Task& t = tasks[i];
        std::printf("%d %d %lld %d %d %d ", t.kind, t.level, (long long)t.tix, t.items, t.c0, t.dep);
        if (joins[i].empty()) std::printf("-");
        for (size_t q = 0; q < joins[i].size(); ++q) std::printf(q ? ",%d" : "%d", joins[i][q]);
        std::printf("\n");
    }
    return 0;
}
