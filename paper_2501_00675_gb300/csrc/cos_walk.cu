// Single-graph evaluation: one persistent cooperative kernel that, after the
// per-kind coefficients, processes the samples tile by tile:
//   1. root values and per-sample exponential factors e^{-+eps_k t_i} (double),
//   2. the propagator table G[slot][sample] of the tile,
//   3. the levels in order (Sec. II.C "Windowing": a level is complete before any
//      of its out-edges is used), a grid-wide barrier between levels, every
//      destination row summing its in-edges in CSR order,
// and finally reduces the per-sample sink values into a compensated mean.  The
// work items of each phase are in cos_items.cuh.
#include <algorithm>
#include <cstdio>

#include "cos_items.cuh"

namespace cosgpu {
namespace {

// Grid-wide barrier over all CTAs of the (co-resident, cooperative) grid.  The
// counter only grows; barrier number `epoch` completes when it reaches
// epoch * gridDim.x.  The wait gives up after p.timeout_ns (or 2^32 polls), sets
// KERR_BARRIER_TIMEOUT and makes every CTA return; a CTA that sees another's
// error also returns.  Returns false when the caller must return.
__device__ __noinline__ bool grid_sync(const WalkParams& p, unsigned long long& epoch, int phase) {
    __shared__ int s_ok;
    // Failure-detection test hook: CTA 0 returns without arriving, so every other
    // CTA's wait runs out and the launch ends with KERR_BARRIER_TIMEOUT.
    if (p.skip_barrier_phase == phase && blockIdx.x == 0) return false;
    __syncthreads();
    epoch += 1;
    if (threadIdx.x == 0) {
        const unsigned long long target = epoch * (unsigned long long)gridDim.x;
        // release: the CTA's writes (ordered before thread 0 by the block barrier) become
        // visible before the arrival is counted; the acquire loads below pair with it
        asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(&p.ctrl->barrier) : "memory");
        int ok = 1;
        const unsigned long long t0 = global_timer_ns();
        for (unsigned long long spin = 0;; ++spin) {
            if (ld_acquire_gpu(&p.ctrl->barrier) >= target) break;
            if ((spin & 15) == 15) {
                if (*(volatile int*)&p.ctrl->err != 0) {
                    ok = 0;
                    break;
                }
                const long long waited = (long long)(global_timer_ns() - t0);
                if (waited > p.timeout_ns || spin > (1ull << 32)) {
                    if (atomicCAS(&p.ctrl->err, 0, KERR_BARRIER_TIMEOUT) == 0) p.ctrl->err_detail = phase;
                    ok = 0;
                    break;
                }
            }
            if (spin >= 32) __nanosleep(32);
        }
        s_ok = ok;
        if (ok && p.trace && blockIdx.x == 0 && (long long)epoch < p.trace_cap) {
            p.trace[2 * epoch] = global_timer_ns();
            p.trace[2 * epoch + 1] = (unsigned long long)phase;
        }
    }
    __syncthreads();
    return s_ok != 0;
}


// Resident CTAs per SM the register budget is tuned for (no spills at these bounds).
template <int MODE, int V, int LAYOUT>
constexpr int min_blocks() {
    if (LAYOUT == LAYOUT_ASYNC) return 4;   // no loads held in registers: a fourth CTA per SM
    return (Traits<MODE>::kBase == COS_MODE_FP64 && V > 2) ? 2 : 3;
}

template <int MODE, int V, int LAYOUT>
__global__ void __launch_bounds__(kThreads, min_blocks<MODE, V, LAYOUT>()) walk_kernel(const WalkParams p) {
    constexpr int CHV = chunk_samples<V, LAYOUT>();
    extern __shared__ __align__(16) double smem[];
    unsigned long long epoch = 0;
    if (p.trace && blockIdx.x == 0 && threadIdx.x == 0 && p.trace_cap > 0) {
        p.trace[0] = global_timer_ns();
        p.trace[1] = 0;
    }
    if constexpr (Traits<MODE>::kBase != COS_MODE_COUNT_I64) {
        if (blockIdx.x == 0) item_coef(p);
        if (!grid_sync(p, epoch, 1)) return;
    }
    const int64_t ntiles = (p.S + p.tile - 1) / p.tile;
    for (int64_t tix = 0; tix < ntiles; ++tix) {
        const TileCtx tc = tile_ctx<CHV>(p, tix);
        const int np = prop_items<MODE>(p, tc);
        for (int it = blockIdx.x; it < np; it += gridDim.x) item_props<MODE, CHV>(p, tc, it, smem);
        if (!grid_sync(p, epoch, 2)) return;
        for (int l = 1; l < p.L; ++l) {
            const int n = level_items(p, p.levels[l], tc);
            for (int it = blockIdx.x; it < n; it += gridDim.x)
                if (!item_level<MODE, V, LAYOUT, false, 6>(p, l, tc, it, reinterpret_cast<unsigned char*>(smem))) break;
            if (!grid_sync(p, epoch, 3 + l)) return;
        }
    }
    const int n = partial_items(p);
    for (int it = blockIdx.x; it < n; it += gridDim.x) item_partials<MODE>(p, it);
    if (!grid_sync(p, epoch, 1000)) return;
    if (blockIdx.x == 0) item_final(p);
}

__global__ void transpose_kernel(const double* __restrict__ src, int64_t S, int32_t D, double* __restrict__ dst,
                                 int64_t t_ld) {
    const int64_t total = S * D;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / S, s = idx % S;
        dst[i * t_ld + s] = src[s * D + i];
    }
}

// t[2m][s], t[2m+1][s] for sample n = first + s: counter (n lo, n hi, m, 0), key = seed;
// 53 bits of each word pair scaled to [0, beta).
__global__ void uniform_times_kernel(unsigned long long seed, long long first, long long S, int D, double beta,
                                     double* __restrict__ t, long long t_ld) {
    const int pairs = (D + 1) / 2;
    const long long total = S * pairs;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(q / S);
        const long long s = q - (long long)m * S;
        double a, b;
        uniform_time_pair(seed, (unsigned long long)(first + s), m, beta, a, b);
        t[(long long)(2 * m) * t_ld + s] = a;
        if (2 * m + 1 < D) t[(long long)(2 * m + 1) * t_ld + s] = b;
    }
}

__global__ void exp_pair_kernel(const double* __restrict__ x, int64_t n, const double* __restrict__ tab,
                                double* __restrict__ em, double* __restrict__ ep) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        double a, b;
        exp_pair(x[q], tab, a, b);
        em[q] = a;
        ep[q] = b;
    }
}

// Throughput probe of the fused multiply-add pipe: every thread runs kChains
// independent dependency chains of `iters` multiply-adds each (far more chains per
// SM than the pipe's latency needs), so the launch time measures the issue rate.
// The chains' end values are stored so that nothing is optimised away.
constexpr int kChains = 8;
template <typename T>
__global__ void fma_probe_kernel(T m, T a, int iters, T* __restrict__ out) {
    T acc[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = (T)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = fma(acc[k], m, a);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += acc[k];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int MODE, int V, int LAYOUT>
const void* kernel_ptr() {
    return reinterpret_cast<const void*>(&walk_kernel<MODE, V, LAYOUT>);
}

template <int LAYOUT>
const void* select_kernel_layout(int mode, int vec) {
    switch (mode * 8 + vec) {
        case COS_MODE_FP64 * 8 + 1: return kernel_ptr<COS_MODE_FP64, 1, LAYOUT>();
        case COS_MODE_FP64 * 8 + 2: return kernel_ptr<COS_MODE_FP64, 2, LAYOUT>();
        case COS_MODE_FP64 * 8 + 4: return kernel_ptr<COS_MODE_FP64, 4, LAYOUT>();
        case COS_MODE_FP32_MIXED * 8 + 1: return kernel_ptr<COS_MODE_FP32_MIXED, 1, LAYOUT>();
        case COS_MODE_FP32_MIXED * 8 + 2: return kernel_ptr<COS_MODE_FP32_MIXED, 2, LAYOUT>();
        case COS_MODE_FP32_MIXED * 8 + 4: return kernel_ptr<COS_MODE_FP32_MIXED, 4, LAYOUT>();
        case COS_MODE_COUNT_I64 * 8 + 1: return kernel_ptr<COS_MODE_COUNT_I64, 1, LAYOUT>();
        case COS_MODE_COUNT_I64 * 8 + 2: return kernel_ptr<COS_MODE_COUNT_I64, 2, LAYOUT>();
        case COS_MODE_COUNT_I64 * 8 + 4: return kernel_ptr<COS_MODE_COUNT_I64, 4, LAYOUT>();
        default: return nullptr;
    }
}

const void* select_kernel(int mode, int vec, int layout) {
    if (mode_has_abs(mode)) {   // sums of |path| values: the wide layout only
        if (layout != 1) return nullptr;
        switch (mode * 8 + vec) {
            case kModeFp64Abs * 8 + 1: return kernel_ptr<kModeFp64Abs, 1, LAYOUT_WIDE>();
            case kModeFp64Abs * 8 + 2: return kernel_ptr<kModeFp64Abs, 2, LAYOUT_WIDE>();
            case kModeFp64Abs * 8 + 4: return kernel_ptr<kModeFp64Abs, 4, LAYOUT_WIDE>();
            case kModeMixedAbs * 8 + 1: return kernel_ptr<kModeMixedAbs, 1, LAYOUT_WIDE>();
            case kModeMixedAbs * 8 + 2: return kernel_ptr<kModeMixedAbs, 2, LAYOUT_WIDE>();
            case kModeMixedAbs * 8 + 4: return kernel_ptr<kModeMixedAbs, 4, LAYOUT_WIDE>();
            default: return nullptr;
        }
    }
    if (layout == 4) return select_kernel_layout<LAYOUT_ASYNC>(mode, vec);
    if (layout == 3) return select_kernel_layout<LAYOUT_BULK>(mode, vec);
    if (layout == 2) return select_kernel_layout<LAYOUT_GROUPED>(mode, vec);
    if (layout == 1) return select_kernel_layout<LAYOUT_WIDE>(mode, vec);
    return nullptr;
}

}  // namespace

template <int MODE>
int ring_bytes(int vec) {
    return vec == 1 ? bulk_ring_bytes<MODE, 1>() : vec == 2 ? bulk_ring_bytes<MODE, 2>() : bulk_ring_bytes<MODE, 4>();
}

int walk_smem_bytes(int mode, int vec, int layout, int D) {
    mode = base_mode(mode);
    const int props = mode == COS_MODE_COUNT_I64 ? 0 : prop_smem_bytes(D, layout == 2 ? 32 : 32 * vec);
    if (layout == 4) {
        const int ring = mode == COS_MODE_FP64 ? (vec == 1 ? async_ring_bytes<COS_MODE_FP64, 1>() : vec == 2 ? async_ring_bytes<COS_MODE_FP64, 2>() : async_ring_bytes<COS_MODE_FP64, 4>())
                         : mode == COS_MODE_FP32_MIXED ? (vec == 1 ? async_ring_bytes<COS_MODE_FP32_MIXED, 1>() : vec == 2 ? async_ring_bytes<COS_MODE_FP32_MIXED, 2>() : async_ring_bytes<COS_MODE_FP32_MIXED, 4>())
                         : (vec == 1 ? async_ring_bytes<COS_MODE_COUNT_I64, 1>() : vec == 2 ? async_ring_bytes<COS_MODE_COUNT_I64, 2>() : async_ring_bytes<COS_MODE_COUNT_I64, 4>());
        return props > ring ? props : ring;
    }
    if (layout != 3) return props;
    const int ring = mode == COS_MODE_FP64 ? ring_bytes<COS_MODE_FP64>(vec)
                     : mode == COS_MODE_FP32_MIXED ? ring_bytes<COS_MODE_FP32_MIXED>(vec)
                                                   : ring_bytes<COS_MODE_COUNT_I64>(vec);
    return props > ring ? props : ring;
}

// Opt every kernel instance into its dynamic shared-memory size.  Without the opt-in,
// dynamic and static shared memory together are limited to 48 KB, so a kernel with a
// few bytes of static shared memory needs it already below 48 KB of dynamic.
int prepare_kernel_attrs(const void* k, int smem) {
    if (smem > 40 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return COS_ERR_CUDA;
    return COS_OK;
}

int max_coresident_blocks(int mode, int vec, int layout, int D, int device) {
    const void* k = select_kernel(mode, vec, layout);
    if (!k) return 0;
    const int smem = walk_smem_bytes(mode, vec, layout, D);
    if (prepare_kernel_attrs(k, smem) != COS_OK) return 0;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    return per_sm * sms;
}

int launch_walk(int mode, int vec, int layout, const WalkParams& p, int grid, cudaStream_t stream, char* msg,
                size_t msglen) {
    const void* k = select_kernel(mode, vec, layout);
    if (!k) {
        snprintf(msg, msglen, "no kernel for mode %d, vector width %d, layout %d", mode, vec, layout);
        return COS_ERR_INVALID;
    }
    const int smem = walk_smem_bytes(mode, vec, layout, p.D);
    if (prepare_kernel_attrs(k, smem) != COS_OK) {
        snprintf(msg, msglen, "cannot set dynamic shared memory %d", smem);
        return COS_ERR_CUDA;
    }
    WalkParams copy = p;
    void* args[] = {&copy};
    cudaError_t e = cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kThreads), args, (size_t)smem, stream);
    if (e != cudaSuccess) {
        snprintf(msg, msglen, "%s", cudaGetErrorString(e));
        cudaGetLastError();
        return COS_ERR_CUDA;
    }
    return COS_OK;
}

int probe_fma_rate(int precision, double* per_second, char* msg, size_t msglen) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        snprintf(msg, msglen, "cannot query the current device");
        return COS_ERR_CUDA;
    }
    const int blocks = sms * 4, threads = 256, iters = 4096;
    const size_t n = (size_t)blocks * threads;
    void* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = COS_OK;
    float best = 1e30f;
    if (cudaMalloc(&out, n * sizeof(double)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        snprintf(msg, msglen, "probe set-up failed: %s", cudaGetErrorString(cudaGetLastError()));
        rc = COS_ERR_CUDA;
    }
    for (int rep = 0; rep < 4 && rc == COS_OK; ++rep) {   // the first run warms up
        cudaEventRecord(e0, 0);
        if (precision == 0)
            fma_probe_kernel<double><<<blocks, threads>>>(0.999999, 1e-7, iters, static_cast<double*>(out));
        else
            fma_probe_kernel<float><<<blocks, threads>>>(0.999999f, 1e-7f, iters, static_cast<float*>(out));
        cudaEventRecord(e1, 0);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            snprintf(msg, msglen, "probe kernel failed");
            rc = COS_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = std::min(best, ms);
    }
    if (rc == COS_OK) *per_second = (double)n * iters * kChains / (best * 1e-3);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    return rc;
}

int launch_exp_pair(const double* x, int64_t n, const double* tab, double* em, double* ep, cudaStream_t stream) {
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152LL * 16);
    exp_pair_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, stream>>>(x, n, tab, em, ep);
    return cudaGetLastError() == cudaSuccess ? COS_OK : COS_ERR_CUDA;
}

int launch_uniform_times(uint64_t seed, int64_t first, int64_t S, int32_t D, double beta, double* t, int64_t t_ld,
                         cudaStream_t stream) {
    const int64_t total = S * ((D + 1) / 2);
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152LL * 16);
    uniform_times_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, stream>>>(seed, first, S, D, beta, t, t_ld);
    return cudaGetLastError() == cudaSuccess ? COS_OK : COS_ERR_CUDA;
}

int launch_transpose(const double* src, int64_t S, int32_t D, double* dst, int64_t t_ld, cudaStream_t stream) {
    const int64_t total = S * D;
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((total + threads - 1) / threads, 152LL * 16);
    transpose_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), threads, 0, stream>>>(src, S, D, dst, t_ld);
    return cudaGetLastError() == cudaSuccess ? COS_OK : COS_ERR_CUDA;
}

}  // namespace cosgpu
