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
// and the reduced result (mean and its compensated sum; the mean of A(s) when the
// walk also accumulates sums of |path| values).
struct Ctrl {
    unsigned long long barrier;
    int err;
    int err_detail;
    double mean;
    double sum;
    double comp;
    double mean_abs;
};

// Kernel mode ids: the public cos_mode values 0..2, and the two floating-point modes
// that also accumulate A(s) = sum of |path| in the same walk (COS_EVAL_ABS).
constexpr int kModeFp64Abs = 3;
constexpr int kModeMixedAbs = 4;
// Kernel mode id of a public mode argument (COS_EVAL_ABS folded in); -1 if invalid.
inline int kernel_mode(int mode) {
    if (mode == COS_MODE_FP64 || mode == COS_MODE_FP32_MIXED || mode == COS_MODE_COUNT_I64) return mode;
    if (mode == (COS_MODE_FP64 | COS_EVAL_ABS)) return kModeFp64Abs;
    if (mode == (COS_MODE_FP32_MIXED | COS_EVAL_ABS)) return kModeMixedAbs;
    return -1;
}
inline bool mode_has_abs(int kmode) { return kmode == kModeFp64Abs || kmode == kModeMixedAbs; }
// The arithmetic of the R walk (0, 1 or 2) of a kernel mode id.
inline int base_mode(int kmode) { return kmode >= kModeFp64Abs ? kmode - kModeFp64Abs : kmode; }

// Everything the persistent walker needs, passed by value.
struct WalkParams {
    // graph (dst-sorted CSR; Sec. II.C "Graph flattening")
    const LevelDesc* levels;   // [L]
    const int32_t* row_ptr;    // [N+1], indexed by global node id
    const int2* edges;         // [E]: (src index inside previous level, propagator slot)
    const int32_t* slot_kij;   // [3P]: (kind, i, j | sign << 30) per slot
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
    double* coef;              // [2K]: -1/(1+e^{-beta eps_k}) (tau >= 0), 1/(1+e^{beta eps_k}) (tau < 0)
    const int32_t* kind_slot;  // [K+1]: slots of kind k are [kind_slot[k], kind_slot[k+1])
    const double* exp_tab;     // [128]: 2^{j/64}, then 2^{-j/64}, j = 0..63; followed by the same
                               // 128 values as float-float (hi, lo) pairs (256 floats)
    void* R;                   // [S] sink value per sample (double, or int64 in count mode)
    double* partials;          // [ceil(S/kReduceBlock)] compensated partial sums
    // sums of |path| values in the same walk (kernel modes kModeFp64Abs, kModeMixedAbs)
    void* aslab[2];            // [nchunk][W][CH] float node values of A, as slab[]
    double* Rabs;              // [S] A(s) per sample
    double* partials_abs;      // [ceil(S/kReduceBlock)] compensated partial sums of A
    Ctrl* ctrl;
    int64_t tile;              // samples per tile (multiple of CH)
    int32_t rows_per_warp;
    int32_t skip_barrier_phase;  // test hook: CTA 0 leaves before this barrier (0 = off)
    long long timeout_ns;
    unsigned long long* trace;   // optional: [2*trace_cap] (globaltimer ns, phase id) per barrier
    int32_t trace_cap;
    int32_t wmax;                // widest level: node-value slabs are [chunk][wmax rows][chunk samples]
    double* mean_out;            // optional second destination of the mean (batched launches)
    // user-tabulated propagators (nullptr: the free-fermion formula): [K][2][ptab_T] pairs
    // (G at node m, G at node m+1 minus G at node m); half 0 on tau = m*h (tau >= 0),
    // half 1 on tau = -tau_max + m*h (tau < 0), h = tau_max/T
    const double* ptab;
    double ptab_tau_max;
    double ptab_inv_h;           // T / tau_max
    int32_t ptab_T;
    int32_t abs_weights;         // 1: every factor replaced by its absolute value (A(s) = sum of |path|)
    int64_t pf_slice_bytes;      // wide layout: L2-prefetch parents on levels whose parent slice per chunk exceeds this
    int32_t pf_bulk;             // 1: that prefetch is one bulk copy per edge run, a window of 32 edges ahead
    int32_t pf_ahead;            // line prefetch: how many batches of edges ahead (1 or 2)
};

constexpr int kThreads = 256;           // 8 warps per CTA
constexpr int kWarps = kThreads / 32;
constexpr int kReduceBlock = 1024;      // samples per compensated partial sum

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
    const int32_t* kind_slot;
    const double* exp_tab;
    const int64_t* widths_host;   // [L], host copy of the level widths
    int64_t S;                    // attached samples (-1: none)
    const double* ptab;           // tabulated propagators (see WalkParams), or nullptr
    double ptab_tau_max;
    int32_t ptab_T;
    double* t;                    // attached times [D][t_ld] (the handle's or the caller's borrowed buffer)
    int64_t t_ld;
    double beta;
    int32_t timeout_ms;           // limit of the kernels' bounded waits (the handle's tuning, else the default)
    uint64_t generation;          // changes whenever buffers, samples, tables or tuning of the handle change
};
int graph_view(cos_graph_t g, GraphView* out);
// Resolve the launch tuning of `mode` (fields of `force` > 0 override the graph's own
// tuning) and fill the walker parameters for the graph's current samples.
int prepare_walk(cos_graph_t g, int mode, const cos_tuning* force, void* per_sample_out, WalkParams* out,
                 cos_tuning* tn_out);
// Host-side sample state of a handle (what attach_own_samples changes).
struct SampleState {
    int64_t S, t_ld;
    const double* t_borrowed;
};
// Point the handle at num_samples samples of its own time buffer [D][t_ld] without any
// CUDA call (the caller fills the buffer on the device).  The handle must have had a
// sample set of at least that size attached before (which also set eps and beta);
// *undo (may be NULL) receives the previous state for restore_samples.
int attach_own_samples(cos_graph_t g, int64_t num_samples, SampleState* undo);
void restore_samples(cos_graph_t g, const SampleState& s);
// Records a message for cos_last_error() and returns code.
int set_error(int code, const char* fmt, ...);
// Windowed schedule of one graph (cos_batch.cu): plan the graph alone as a batch of
// one with the resolved tuning `tn` (window_chunks > 0), upload it and launch the
// work-queue kernel on `st`.  *cache holds the batch object between calls.
int launch_windowed(cos_graph_t g, cos_batch_t* cache, int mode, void* per_sample_out, const cos_tuning& tn,
                    cudaStream_t st);

// Host launcher implemented in cos_walk.cu.  Returns COS_OK or COS_ERR_CUDA and
// fills msg on failure.
// layout: 1 = wide, 2 = grouped (cos_tuning.layout).
int launch_walk(int mode, int vec, int layout, const WalkParams& p, int grid, cudaStream_t stream, char* msg,
                size_t msglen);
// Co-resident persistent grid size for (mode, vec, layout) with D time variables; 0 on failure.
int max_coresident_blocks(int mode, int vec, int layout, int D, int device);
// The same for the work-queue kernel (cos_batch.cu), whose register budget can differ.
int batch_coresident_blocks(int mode, int vec, int layout, int D, int device);
// Dynamic shared memory of a launch (the propagator phase keeps 32 samples x D times
// in shared memory), and the once-per-kernel opt-in to sizes above 48 KB.
int walk_smem_bytes(int mode, int vec, int layout, int D);
int prepare_kernel_attrs(const void* kernel, int smem_bytes);
// Multiply-adds per second of the current device (precision 0: double, 1: float),
// measured by a throughput kernel (cos_probe_fma_rate).
int probe_fma_rate(int precision, double* per_second, char* msg, size_t msglen);
// e^{-x} and e^{+x} with the evaluator's table-driven exponentials (self test).
int launch_exp_pair(const double* x, int64_t n, const double* tab, double* em, double* ep, cudaStream_t stream);
// Counter-based uniform times t[i][s] in [0, beta) for samples first..first+S-1.
int launch_uniform_times(uint64_t seed, int64_t first, int64_t S, int32_t D, double beta, double* t, int64_t t_ld,
                         cudaStream_t stream);
// Transpose t from [S][D] (src_ld = D) into [D][t_ld].
int launch_transpose(const double* src, int64_t S, int32_t D, double* dst, int64_t t_ld, cudaStream_t stream);

}  // namespace cosgpu
