// Metropolis walkers over the vertex times, on the device.
//
// Sec. II.B integrates the sum over diagrams over the vertex times by Monte Carlo
// sampling; Sec. II.C ("Distributing the task") runs many Markov-chain walkers on
// one GPU, and Sec. III keeps the proposal and acceptance of configurations in
// device code.  Every attached sample of a graph is a walker; one step is
//   propose (kernel): walker s draws Philox-4x32-10 words w0..w3 with counter
//     (s mod 2^32, s >> 32, n mod 2^32, 2^31 | n >> 32) and key (seed mod 2^32,
//     seed >> 32) for step n; it replaces time i = (w0 * D) >> 32 by
//     beta * (((w2 << 32 | w1) >> 11) * 2^-53) in the graph's time buffer and
//     remembers the old value;
//   evaluate: the graph's own cos_evaluate gives R' for every walker at once;
//   accept (kernel): u = (w3 + 1/2) * 2^-32; the move stays iff u * |R| < |R'|
//     (probability min(1, |R'|/|R|)), else the old time is put back; the walker's
//     current R is tallied (positive, negative) and accepted moves counted, as
//     64-bit integers, so the tallies do not depend on the order of the adds.
// The fourth counter word's top bit keeps these streams apart from
// cos_set_samples_uniform's (whose fourth word is 0).
#include <cstdio>
#include <cstring>
#include <new>

#include "cos_items.cuh"

namespace cosgpu {
namespace {

__device__ __forceinline__ uint4 walker_words(long long s, unsigned long long step, unsigned long long seed) {
    return philox4x32_10(make_uint4((unsigned)s, (unsigned)((unsigned long long)s >> 32), (unsigned)step,
                                    0x80000000u | ((unsigned)(step >> 32) & 0x7FFFFFFFu)),
                         (unsigned)seed, (unsigned)(seed >> 32));
}

__global__ void mc_propose_kernel(double* __restrict__ t, long long t_ld, long long S, int D, double beta,
                                  unsigned long long seed, unsigned long long step, double* __restrict__ old_val,
                                  int* __restrict__ old_i) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < S; s += (long long)gridDim.x * blockDim.x) {
        const uint4 w = walker_words(s, step, seed);
        const int i = (int)(((unsigned long long)w.x * (unsigned long long)D) >> 32);
        const unsigned long long x = ((((unsigned long long)w.z) << 32) | w.y) >> 11;
        double* ti = t + (long long)i * t_ld + s;
        old_i[s] = i;
        old_val[s] = *ti;
        *ti = beta * ((double)x * 0x1.0p-53);
    }
}

__global__ void mc_accept_kernel(double* __restrict__ t, long long t_ld, long long S, unsigned long long seed,
                                 unsigned long long step, const double* __restrict__ Rp, double* __restrict__ R,
                                 const double* __restrict__ old_val, const int* __restrict__ old_i,
                                 unsigned long long* __restrict__ tallies) {
    unsigned long long acc_n = 0, pos_n = 0, neg_n = 0;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < S; s += (long long)gridDim.x * blockDim.x) {
        const uint4 w = walker_words(s, step, seed);
        const double u = ((double)w.w + 0.5) * 0x1.0p-32;
        const double r = R[s], rp = Rp[s];
        double cur = r;
        if (u * fabs(r) < fabs(rp)) {
            R[s] = rp;
            cur = rp;
            ++acc_n;
        } else {
            t[(long long)old_i[s] * t_ld + s] = old_val[s];
        }
        pos_n += cur > 0.0 ? 1 : 0;
        neg_n += cur < 0.0 ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        acc_n += __shfl_down_sync(0xffffffffu, acc_n, o);
        pos_n += __shfl_down_sync(0xffffffffu, pos_n, o);
        neg_n += __shfl_down_sync(0xffffffffu, neg_n, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (acc_n) atomicAdd(tallies + 0, acc_n);
        if (pos_n) atomicAdd(tallies + 1, pos_n);
        if (neg_n) atomicAdd(tallies + 2, neg_n);
    }
}

// A step whose evaluation could not be launched: every walker takes its old time back.
__global__ void mc_restore_kernel(double* __restrict__ t, long long t_ld, long long S,
                                  const double* __restrict__ old_val, const int* __restrict__ old_i) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < S; s += (long long)gridDim.x * blockDim.x)
        t[(long long)old_i[s] * t_ld + s] = old_val[s];
}

int grid_for(long long S) {
    const long long b = (S + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

}  // namespace
}  // namespace cosgpu

using namespace cosgpu;

struct cos_mc {
    cos_graph_t g = nullptr;
    int mode = 0;
    unsigned long long seed = 0;
    unsigned long long step = 0;
    int device = 0;
    long long S = 0;
    int D = 0;
    double* R = nullptr;         // [S] current value per walker
    double* Rp = nullptr;        // [S] proposal values
    double* old_val = nullptr;   // [S] replaced time
    int* old_i = nullptr;        // [S] replaced time's index
    unsigned long long* tallies = nullptr;   // [3] accepted, positive, negative
};

namespace {

void mc_free(cos_mc* m) {
    cudaFree(m->R);
    cudaFree(m->Rp);
    cudaFree(m->old_val);
    cudaFree(m->old_i);
    cudaFree(m->tallies);
}

}  // namespace

extern "C" {

int cos_mc_create(cos_graph_t g, int32_t mode, uint64_t seed, void* stream, cos_mc_t* out) {
    if (!g || !out) return set_error(COS_ERR_INVALID, "bad arguments");
    if (mode != COS_MODE_FP64 && mode != COS_MODE_FP32_MIXED)
        return set_error(COS_ERR_INVALID, "Metropolis walkers need a floating-point mode (0 or 1)");
    GraphView gv;
    int rc = graph_view(g, &gv);
    if (rc != COS_OK) return rc;
    if (gv.S <= 0) return set_error(COS_ERR_STATE, "attach samples (the walkers' starting times) first");
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(gv.device);
    cos_mc* m = new (std::nothrow) cos_mc();
    if (!m) return set_error(COS_ERR_OOM, "host allocation failed");
    m->g = g;
    m->mode = mode;
    m->seed = seed;
    m->device = gv.device;
    m->S = gv.S;
    m->D = gv.D;
    cudaError_t e = cudaMalloc(&m->R, sizeof(double) * m->S);
    if (e == cudaSuccess) e = cudaMalloc(&m->Rp, sizeof(double) * m->S);
    if (e == cudaSuccess) e = cudaMalloc(&m->old_val, sizeof(double) * m->S);
    if (e == cudaSuccess) e = cudaMalloc(&m->old_i, sizeof(int) * m->S);
    if (e == cudaSuccess) e = cudaMalloc(&m->tallies, sizeof(unsigned long long) * 3);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->tallies, 0, sizeof(unsigned long long) * 3, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        mc_free(m);
        delete m;
        if (prev >= 0) cudaSetDevice(prev);
        return set_error(COS_ERR_OOM, "walker state: %s", cudaGetErrorString(e));
    }
    rc = cos_evaluate(g, mode, m->R, nullptr, stream);   // the starting values
    if (prev >= 0) cudaSetDevice(prev);
    if (rc != COS_OK) {
        mc_free(m);
        delete m;
        return rc;
    }
    *out = m;
    return COS_OK;
}

int cos_mc_run(cos_mc_t m, int32_t num_steps, void* stream) {
    if (!m || num_steps < 0) return set_error(COS_ERR_INVALID, "bad arguments");
    GraphView gv;
    int rc = graph_view(m->g, &gv);
    if (rc != COS_OK) return rc;
    if (gv.S != m->S || gv.D != m->D) return set_error(COS_ERR_STATE, "the graph's samples changed under the walkers");
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(m->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = grid_for(m->S);
    for (int32_t q = 0; q < num_steps && rc == COS_OK; ++q) {
        mc_propose_kernel<<<grid, 256, 0, st>>>(gv.t, gv.t_ld, m->S, m->D, gv.beta, m->seed, m->step, m->old_val,
                                                 m->old_i);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            rc = set_error(COS_ERR_CUDA, "propose: %s", cudaGetErrorString(e));
            break;
        }
        rc = cos_evaluate(m->g, m->mode, m->Rp, nullptr, stream);
        if (rc != COS_OK) {   // leave the walkers where they were
            mc_restore_kernel<<<grid, 256, 0, st>>>(gv.t, gv.t_ld, m->S, m->old_val, m->old_i);
            break;
        }
        mc_accept_kernel<<<grid, 256, 0, st>>>(gv.t, gv.t_ld, m->S, m->seed, m->step, m->Rp, m->R, m->old_val,
                                                m->old_i, m->tallies);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = set_error(COS_ERR_CUDA, "accept: %s", cudaGetErrorString(e));
        ++m->step;
    }
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
}

int cos_mc_stats(cos_mc_t m, int64_t* out, void* stream) {
    if (!m || !out) return set_error(COS_ERR_INVALID, "bad arguments");
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(m->device);
    unsigned long long h[3] = {0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(h, m->tallies, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return set_error(COS_ERR_CUDA, "walker tallies: %s", cudaGetErrorString(e));
    const int rc = cos_get_result(m->g, nullptr, stream);   // status of the last evaluation
    out[0] = (int64_t)m->step;
    out[1] = (int64_t)h[0];
    out[2] = (int64_t)h[1];
    out[3] = (int64_t)h[2];
    return rc;
}

int cos_mc_values(cos_mc_t m, double* per_walker_out, void* stream) {
    if (!m || !per_walker_out) return set_error(COS_ERR_INVALID, "bad arguments");
    cudaError_t e = cudaMemcpyAsync(per_walker_out, m->R, sizeof(double) * m->S, cudaMemcpyDefault,
                                    (cudaStream_t)stream);
    return e == cudaSuccess ? COS_OK : set_error(COS_ERR_CUDA, "walker values: %s", cudaGetErrorString(e));
}

int cos_mc_destroy(cos_mc_t m) {
    if (!m) return COS_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(m->device);
    mc_free(m);
    if (prev >= 0) cudaSetDevice(prev);
    delete m;
    return COS_OK;
}

}  // extern "C"
