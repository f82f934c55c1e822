// Internal types shared by the host side (cos_graph.cu) and the kernels (cos_walk.cu)
// of the GB300 CoS evaluator.  Not part of the public ABI (include/cos.h is).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/cos.h"

namespace cosgpu {

// Kernel-side error codes written to Ctrl::err (0 = fine).
enum : int { KERR_NONE = 0, KERR_BARRIER_TIMEOUT = 1 };

// One level of the graph as the walker sees it.  Rows of level l are the global
// node ids [row_begin, row_begin + width); their in-edges come from level l-1,
// whose nodes are addressed by their index inside that level (src_local).
struct LevelDesc {
    int32_t row_begin;
    int32_t width;
    int32_t prev_width;
    int32_t pad;
};

// Per-launch control block in device memory: grid-barrier counter, error word,
// and the reduced result (mean and its compensated sum).
struct Ctrl {
    unsigned long long barrier;
    int err;
    int err_detail;
    double mean;
    double sum;
    double comp;
    double pad;
};

// Everything the persistent walker needs, passed by value.
struct WalkParams {
    // graph (dst-sorted CSR; Sec. II.C "Graph flattening")
    const LevelDesc* levels;   // [L]
    const int32_t* row_ptr;    // [N+1], indexed by global node id
    const int2* edges;         // [E]: (src index inside previous level, propagator slot)
    const int32_t* slot_kij;   // [3P]: (kind, i, j) per slot
    int32_t L, P, K, D;
    // samples
    const double* t;           // [D][t_ld], sample index fastest, zero padded
    const double* eps;         // [K]
    double beta;
    int64_t S;                 // number of samples
    int64_t t_ld;              // leading dimension of t (>= S, multiple of 128)
    // workspace, carved from one arena per tile
    void* slab[2];             // [nchunk][W][CH] node values, ping-pong between levels
    void* gtab;                // [nchunk][P][CH] propagator table of the tile
    double* fac_m;             // [K][D][tile] exp(-eps_k t_i)
    double* fac_p;             // [K][D][tile] exp(+eps_k t_i)
    double* coef;              // [2K]: -1/(1+e^{-beta eps_k}) (tau >= 0), 1/(1+e^{beta eps_k}) (tau < 0)
    void* R;                   // [S] sink value per sample (double, or int64 in count mode)
    double* partials;          // [ceil(S/4096)] compensated partial sums
    Ctrl* ctrl;
    int64_t tile;              // samples per tile (multiple of CH)
    int32_t rows_per_warp;
    int32_t skip_barrier_phase;  // test hook: CTA 0 leaves before this barrier (0 = off)
    long long timeout_ns;
};

constexpr int kThreads = 256;           // 8 warps per CTA
constexpr int kWarps = kThreads / 32;
constexpr int kReduceBlock = 4096;      // samples per compensated partial sum

// Device-resident view of a graph handle (read-only), for entry points that
// evaluate an existing graph with scratch memory of their own.
struct GraphView {
    const LevelDesc* levels;
    const int32_t* row_ptr;
    const int2* edges;
    const int32_t* slot_kij;
    int32_t L, P, K, D;
    int64_t Wmax;
    int device;
    int count_overflow;
};
int graph_view(cos_graph_t g, GraphView* out);
// Records a message for cos_last_error() and returns code.
int set_error(int code, const char* fmt, ...);

// Host launcher implemented in cos_walk.cu.  Returns COS_OK or COS_ERR_CUDA and
// fills msg on failure.
int launch_walk(int mode, int vec, const WalkParams& p, int grid, cudaStream_t stream, char* msg, size_t msglen);
// Co-resident persistent grid size for (mode, vec); 0 on failure.
int max_coresident_blocks(int mode, int vec, int device);
// Transpose t from [S][D] (src_ld = D) into [D][t_ld].
int launch_transpose(const double* src, int64_t S, int32_t D, double* dst, int64_t t_ld, cudaStream_t stream);

}  // namespace cosgpu
