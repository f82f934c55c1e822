// Device side of the GB300 CoS evaluator: one persistent cooperative kernel per
// evaluation that, for every tile of samples,
//   1. forms the per-sample exponential factors exp(-+eps_k t_i)   (double),
//   2. builds the propagator table G[slot][sample] of the tile,
//   3. walks the levels in order (Sec. II.C "Windowing": a level is complete
//      before any of its out-edges is used) with a grid-wide barrier between
//      levels, each destination row summing its in-edges in CSR order,
// and finally reduces the per-sample sink values into a compensated mean.
//
// Layout (node x sample, Sec. App. A "Cache and locality"): the samples of a tile
// are split into chunks of CH = 32*V consecutive samples; lane q of a warp owns
// samples [q*V, q*V+V) of a chunk.  Node values of one level are stored
// [chunk][row][CH], the propagator table [chunk][slot][CH], so every edge of a
// warp reads one contiguous, vector-aligned run of CH values.
#include <cstdio>

#include "cos_internal.cuh"

namespace cosgpu {
namespace {

__device__ __forceinline__ unsigned long long global_timer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

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
        __threadfence();
        atomicAdd(&p.ctrl->barrier, 1ull);
        int ok = 1;
        const unsigned long long t0 = global_timer_ns();
        for (unsigned long long spin = 0;; ++spin) {
            if (ld_acquire_gpu(&p.ctrl->barrier) >= target) break;
            if (*(volatile int*)&p.ctrl->err != 0) {
                ok = 0;
                break;
            }
            if ((spin & 31) == 31) {
                const long long waited = (long long)(global_timer_ns() - t0);
                if (waited > p.timeout_ns || spin > (1ull << 32)) {
                    if (atomicCAS(&p.ctrl->err, 0, KERR_BARRIER_TIMEOUT) == 0) p.ctrl->err_detail = phase;
                    ok = 0;
                    break;
                }
            }
            __nanosleep(40);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------- vector access

template <typename T, int V>
struct alignas(sizeof(T) * V) VecT {
    T v[V];
};

template <typename T, int V>
__device__ __forceinline__ VecT<T, V> load_cg(const T* ptr) {  // L2 only: data written earlier by this kernel
    VecT<T, V> r;
    constexpr int bytes = sizeof(T) * V;
    if constexpr (bytes == 32) {
        const uint4* q = reinterpret_cast<const uint4*>(ptr);
        uint4 a = __ldcg(q), b = __ldcg(q + 1);
        memcpy(&r.v[0], &a, 16);
        memcpy(reinterpret_cast<char*>(&r.v[0]) + 16, &b, 16);
    } else if constexpr (bytes == 16) {
        uint4 a = __ldcg(reinterpret_cast<const uint4*>(ptr));
        memcpy(&r.v[0], &a, 16);
    } else if constexpr (bytes == 8) {
        uint2 a = __ldcg(reinterpret_cast<const uint2*>(ptr));
        memcpy(&r.v[0], &a, 8);
    } else {
        unsigned a = __ldcg(reinterpret_cast<const unsigned*>(ptr));
        memcpy(&r.v[0], &a, 4);
    }
    return r;
}

template <typename T, int V>
__device__ __forceinline__ VecT<T, V> load_ca(const T* ptr) {  // L1-cacheable coherent load
    return *reinterpret_cast<const VecT<T, V>*>(ptr);
}

template <typename T, int V>
__device__ __forceinline__ void store_cg(T* ptr, const VecT<T, V>& x) {
    constexpr int bytes = sizeof(T) * V;
    if constexpr (bytes == 32) {
        uint4 a, b;
        memcpy(&a, &x.v[0], 16);
        memcpy(&b, reinterpret_cast<const char*>(&x.v[0]) + 16, 16);
        __stcg(reinterpret_cast<uint4*>(ptr), a);
        __stcg(reinterpret_cast<uint4*>(ptr) + 1, b);
    } else if constexpr (bytes == 16) {
        uint4 a;
        memcpy(&a, &x.v[0], 16);
        __stcg(reinterpret_cast<uint4*>(ptr), a);
    } else if constexpr (bytes == 8) {
        uint2 a;
        memcpy(&a, &x.v[0], 8);
        __stcg(reinterpret_cast<uint2*>(ptr), a);
    } else {
        unsigned a;
        memcpy(&a, &x.v[0], 4);
        __stcg(reinterpret_cast<unsigned*>(ptr), a);
    }
}

// ---------------------------------------------------------------- mode traits

template <int MODE>
struct Traits;
template <>
struct Traits<COS_MODE_FP64> {       // everything in double
    using Val = double;
    using Prop = double;
    using SinkAcc = double;
    static constexpr bool kCount = false;
};
template <>
struct Traits<COS_MODE_FP32_MIXED> { // float propagators and products, double sink
    using Val = float;
    using Prop = float;
    using SinkAcc = double;
    static constexpr bool kCount = false;
};
template <>
struct Traits<COS_MODE_COUNT_I64> {  // unit weights, sums modulo 2^64
    using Val = unsigned long long;
    using Prop = unsigned long long;
    using SinkAcc = unsigned long long;
    static constexpr bool kCount = true;
};

__device__ __forceinline__ double madd(double p, double g, double acc) { return fma(p, g, acc); }
__device__ __forceinline__ float madd(float p, float g, float acc) { return fmaf(p, g, acc); }

// ---------------------------------------------------------------- phases

// Per-kind coefficients, per-sample exponential factors, and the root value.
template <int MODE, int V>
__device__ void phase_factors(const WalkParams& p, int64_t base, int64_t tile_n) {
    using Tr = Traits<MODE>;
    constexpr int CH = 32 * V;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
    // root: node 0 holds 1 for every sample (Fig. 1 caption)
    typename Tr::Val* root = static_cast<typename Tr::Val*>(p.slab[0]);
    for (int64_t s = gtid; s < tile_n; s += gstride) root[s] = (typename Tr::Val)1;   // [chunk][row 0][CH]
    if constexpr (!Tr::kCount) {
        for (int64_t k = gtid; k < p.K; k += gstride) {
            const double be = p.beta * p.eps[k];
            p.coef[k] = -1.0 / (1.0 + exp(-be));        // tau >= 0: -e^{-eps tau} / (1 + e^{-beta eps})
            p.coef[p.K + k] = 1.0 / (1.0 + exp(be));    // tau <  0: +e^{-eps tau} e^{-beta eps} / (1 + e^{-beta eps})
        }
        const int64_t total = (int64_t)p.K * p.D * tile_n;
        for (int64_t idx = gtid; idx < total; idx += gstride) {
            const int64_t s = idx % tile_n;
            const int64_t kd = idx / tile_n;
            const int k = (int)(kd / p.D), i = (int)(kd % p.D);
            const double x = p.eps[k] * p.t[(int64_t)i * p.t_ld + base + s];
            const double em = exp(-x);
            p.fac_m[kd * p.tile + s] = em;
            p.fac_p[kd * p.tile + s] = __drcp_rn(em);
        }
    }
    (void)CH;
}

// Propagator table of the tile: G[chunk][slot][CH] = coef(branch) * e^{-eps t_i} * e^{+eps t_j},
// formed in double and stored in the mode's propagator type (one rounding for float).
template <int MODE, int V>
__device__ void phase_gtab(const WalkParams& p, int64_t base, int64_t tile_n) {
    using Tr = Traits<MODE>;
    constexpr int CH = 32 * V;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nch = tile_n / CH;
    const int64_t total = nch * p.P * CH;
    typename Tr::Prop* gt = static_cast<typename Tr::Prop*>(p.gtab);
    for (int64_t idx = gtid; idx < total; idx += gstride) {
        const int ls = (int)(idx % CH);
        const int64_t q = (idx / CH) % p.P;
        const int64_t c = idx / ((int64_t)CH * p.P);
        const int64_t s = c * CH + ls;
        const int k = __ldg(p.slot_kij + 3 * q), i = __ldg(p.slot_kij + 3 * q + 1), j = __ldg(p.slot_kij + 3 * q + 2);
        const double ti = p.t[(int64_t)i * p.t_ld + base + s];
        const double tj = p.t[(int64_t)j * p.t_ld + base + s];
        const double cf = (ti >= tj) ? p.coef[k] : p.coef[p.K + k];   // tau = t_i - t_j >= 0 ?
        const double g = cf * p.fac_m[((int64_t)k * p.D + i) * p.tile + s] * p.fac_p[((int64_t)k * p.D + j) * p.tile + s];
        gt[idx] = (typename Tr::Prop)g;
    }
}

// One level: every destination row r of level l, for every chunk of the tile,
// sums parent x propagator over its in-edges (CSR order), one warp per row.
template <int MODE, int V>
__device__ void phase_level(const WalkParams& p, int l, int64_t base, int64_t tile_n) {
    using Tr = Traits<MODE>;
    using Val = typename Tr::Val;
    using Prop = typename Tr::Prop;
    constexpr int CH = 32 * V;
    const LevelDesc ld = p.levels[l];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nch = tile_n / CH;
    const int rows_per_item = kWarps * p.rows_per_warp;
    const int64_t nrb = (ld.width + rows_per_item - 1) / rows_per_item;
    const int64_t items = nch * nrb;
    const bool sink = (l == p.L - 1);
    const Val* parent = static_cast<const Val*>(p.slab[(l - 1) & 1]);
    Val* child = static_cast<Val*>(p.slab[l & 1]);
    const Prop* gt = static_cast<const Prop*>(p.gtab);
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int64_t c = item / nrb;
        const int64_t rb = item % nrb;
        const Val* pc = parent + c * (int64_t)ld.prev_width * CH + lane * V;
        const Prop* gc = Tr::kCount ? nullptr : gt + c * (int64_t)p.P * CH + lane * V;
        for (int rr = 0; rr < p.rows_per_warp; ++rr) {
            const int64_t r = rb * rows_per_item + (int64_t)rr * kWarps + warp;
            if (r >= ld.width) break;
            const int node = ld.row_begin + (int)r;
            const int beg = __ldg(p.row_ptr + node), end = __ldg(p.row_ptr + node + 1);
            if (sink && !Tr::kCount && MODE == COS_MODE_FP32_MIXED) {
                double acc[V];
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] = 0.0;
                for (int e0 = beg; e0 < end; e0 += 32) {
                    const int n = min(32, end - e0);
                    const int2 m = (lane < n) ? __ldg(p.edges + e0 + lane) : make_int2(0, 0);
                    for (int q = 0; q < n; ++q) {
                        const int src = __shfl_sync(0xffffffffu, m.x, q);
                        const int slot = __shfl_sync(0xffffffffu, m.y, q);
                        const VecT<Val, V> pv = load_cg<Val, V>(pc + (int64_t)src * CH);
                        const VecT<Prop, V> gv = load_ca<Prop, V>(gc + (int64_t)slot * CH);
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v] += (double)pv.v[v] * (double)gv.v[v];  // exact product
                    }
                }
                double* R = static_cast<double*>(p.R);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int64_t s = base + c * CH + lane * V + v;
                    if (s < p.S) R[s] = acc[v];
                }
                continue;
            }
            Val acc[V];
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = (Val)0;
            for (int e0 = beg; e0 < end; e0 += 32) {
                const int n = min(32, end - e0);
                const int2 m = (lane < n) ? __ldg(p.edges + e0 + lane) : make_int2(0, 0);
                int q = 0;
                for (; q + 2 <= n; q += 2) {   // two edges in flight, summed in CSR order
                    const int s0 = __shfl_sync(0xffffffffu, m.x, q), s1 = __shfl_sync(0xffffffffu, m.x, q + 1);
                    const VecT<Val, V> p0 = load_cg<Val, V>(pc + (int64_t)s0 * CH);
                    const VecT<Val, V> p1 = load_cg<Val, V>(pc + (int64_t)s1 * CH);
                    if constexpr (Tr::kCount) {
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v] += p0.v[v];
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v] += p1.v[v];
                    } else {
                        const int g0 = __shfl_sync(0xffffffffu, m.y, q), g1 = __shfl_sync(0xffffffffu, m.y, q + 1);
                        const VecT<Prop, V> w0 = load_ca<Prop, V>(gc + (int64_t)g0 * CH);
                        const VecT<Prop, V> w1 = load_ca<Prop, V>(gc + (int64_t)g1 * CH);
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v] = madd(p0.v[v], w0.v[v], acc[v]);
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v] = madd(p1.v[v], w1.v[v], acc[v]);
                    }
                }
                if (q < n) {
                    const int s0 = __shfl_sync(0xffffffffu, m.x, q);
                    const VecT<Val, V> p0 = load_cg<Val, V>(pc + (int64_t)s0 * CH);
                    if constexpr (Tr::kCount) {
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v] += p0.v[v];
                    } else {
                        const int g0 = __shfl_sync(0xffffffffu, m.y, q);
                        const VecT<Prop, V> w0 = load_ca<Prop, V>(gc + (int64_t)g0 * CH);
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v] = madd(p0.v[v], w0.v[v], acc[v]);
                    }
                }
            }
            if (sink) {
                using Out = typename Tr::SinkAcc;
                Out* R = static_cast<Out*>(p.R);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int64_t s = base + c * CH + lane * V + v;
                    if (s < p.S) R[s] = (Out)acc[v];
                }
            } else {
                VecT<Val, V> out;
#pragma unroll
                for (int v = 0; v < V; ++v) out.v[v] = acc[v];
                store_cg<Val, V>(child + (c * (int64_t)ld.width + r) * CH + lane * V, out);
            }
        }
    }
}

__device__ __forceinline__ void neumaier_add(double& sum, double& comp, double y) {
    const double u = sum + y;
    if (fabs(sum) >= fabs(y)) comp += (sum - u) + y;
    else comp += (y - u) + sum;
    sum = u;
}

// Compensated partial sums of R over blocks of kReduceBlock samples, in index order:
// lane q sums its 128 consecutive samples, lane partials are then added in lane order.
template <int MODE>
__device__ void phase_partials(const WalkParams& p) {
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nblk = (p.S + kReduceBlock - 1) / kReduceBlock;
    constexpr int per_lane = kReduceBlock / 32;
    for (int64_t b = gwarp; b < nblk; b += nwarps) {
        double sum = 0.0, comp = 0.0;
        const int64_t s0 = b * kReduceBlock + (int64_t)lane * per_lane;
        for (int q = 0; q < per_lane; ++q) {
            const int64_t s = s0 + q;
            if (s >= p.S) break;
            double x;
            if constexpr (MODE == COS_MODE_COUNT_I64) x = (double)static_cast<const long long*>(p.R)[s];
            else x = static_cast<const double*>(p.R)[s];
            neumaier_add(sum, comp, x);
        }
        const double mine = sum + comp;
        double bs = 0.0, bc = 0.0;
        for (int q = 0; q < 32; ++q) neumaier_add(bs, bc, __shfl_sync(0xffffffffu, mine, q));
        if (lane == 0) p.partials[b] = bs + bc;
    }
}

template <int MODE, int V>
__global__ void __launch_bounds__(kThreads, 2) walk_kernel(const WalkParams p) {
    constexpr int CH = 32 * V;
    unsigned long long epoch = 0;
    const int64_t ntiles = (p.S + p.tile - 1) / p.tile;
    for (int64_t tix = 0; tix < ntiles; ++tix) {
        const int64_t base = tix * p.tile;
        const int64_t n = min(p.tile, p.S - base);
        const int64_t tile_n = (n + CH - 1) / CH * CH;
        phase_factors<MODE, V>(p, base, tile_n);
        if (!grid_sync(p, epoch, 1)) return;
        if constexpr (MODE != COS_MODE_COUNT_I64) {
            phase_gtab<MODE, V>(p, base, tile_n);
            if (!grid_sync(p, epoch, 2)) return;
        }
        for (int l = 1; l < p.L; ++l) {
            phase_level<MODE, V>(p, l, base, tile_n);
            if (!grid_sync(p, epoch, 2 + l)) return;
        }
    }
    phase_partials<MODE>(p);
    if (!grid_sync(p, epoch, 1000)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t nblk = (p.S + kReduceBlock - 1) / kReduceBlock;
        double sum = 0.0, comp = 0.0;
        for (int64_t b = 0; b < nblk; ++b) neumaier_add(sum, comp, p.partials[b]);
        p.ctrl->sum = sum;
        p.ctrl->comp = comp;
        p.ctrl->mean = p.S > 0 ? (sum + comp) / (double)p.S : 0.0;
    }
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

template <int MODE, int V>
const void* kernel_ptr() {
    return reinterpret_cast<const void*>(&walk_kernel<MODE, V>);
}

const void* select_kernel(int mode, int vec) {
    switch (mode * 8 + vec) {
        case COS_MODE_FP64 * 8 + 1: return kernel_ptr<COS_MODE_FP64, 1>();
        case COS_MODE_FP64 * 8 + 2: return kernel_ptr<COS_MODE_FP64, 2>();
        case COS_MODE_FP64 * 8 + 4: return kernel_ptr<COS_MODE_FP64, 4>();
        case COS_MODE_FP32_MIXED * 8 + 1: return kernel_ptr<COS_MODE_FP32_MIXED, 1>();
        case COS_MODE_FP32_MIXED * 8 + 2: return kernel_ptr<COS_MODE_FP32_MIXED, 2>();
        case COS_MODE_FP32_MIXED * 8 + 4: return kernel_ptr<COS_MODE_FP32_MIXED, 4>();
        case COS_MODE_COUNT_I64 * 8 + 1: return kernel_ptr<COS_MODE_COUNT_I64, 1>();
        case COS_MODE_COUNT_I64 * 8 + 2: return kernel_ptr<COS_MODE_COUNT_I64, 2>();
        case COS_MODE_COUNT_I64 * 8 + 4: return kernel_ptr<COS_MODE_COUNT_I64, 4>();
        default: return nullptr;
    }
}

}  // namespace

int max_coresident_blocks(int mode, int vec, int device) {
    const void* k = select_kernel(mode, vec);
    if (!k) return 0;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, 0) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    return per_sm * sms;
}

int launch_walk(int mode, int vec, const WalkParams& p, int grid, cudaStream_t stream, char* msg, size_t msglen) {
    const void* k = select_kernel(mode, vec);
    if (!k) {
        snprintf(msg, msglen, "no kernel for mode %d, vector width %d", mode, vec);
        return COS_ERR_INVALID;
    }
    WalkParams copy = p;
    void* args[] = {&copy};
    cudaError_t e = cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kThreads), args, 0, stream);
    if (e != cudaSuccess) {
        snprintf(msg, msglen, "%s", cudaGetErrorString(e));
        cudaGetLastError();
        return COS_ERR_CUDA;
    }
    return COS_OK;
}

int launch_transpose(const double* src, int64_t S, int32_t D, double* dst, int64_t t_ld, cudaStream_t stream) {
    const int64_t total = S * D;
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((total + threads - 1) / threads, 152LL * 16);
    transpose_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), threads, 0, stream>>>(src, S, D, dst, t_ld);
    return cudaGetLastError() == cudaSuccess ? COS_OK : COS_ERR_CUDA;
}

}  // namespace cosgpu
