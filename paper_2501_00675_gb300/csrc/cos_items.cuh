// Device work items of the CoS evaluator, shared by the single-graph cooperative
// kernel (cos_walk.cu, grid barriers between phases) and the batched work-queue
// kernel (cos_batch.cu, per-graph dependency counters).  Every function below
// executes one CTA-sized unit of one phase.
//
// Layout (node x sample, App. A "Cache and locality"): the samples of a tile are
// split into chunks of CHV consecutive samples.  Node values of one level are
// stored [chunk][row][CHV] with a chunk stride of W_max rows whatever the level's
// width, so that a chunk occupies the same region at every level of one slab parity
// (windows of chunks at different levels never overlap), the propagator table
// [chunk][slot][CHV], exponential
// factors [K][D][tile].  Two level-walk layouts share this storage scheme:
//   wide    (CHV = 32*V): a warp owns one row at a time, lane q holds samples
//           [q*V, q*V+V) of the chunk; one warp instruction reads one contiguous run.
//   grouped (CHV = 32):   a warp serves V rows at once, each row owned by a group
//           of 32/V lanes holding V samples each; the parent slice of a chunk
//           (W x 32 values) stays small enough for L2.
// Either way a lane moves V values per access (16 B for float with V = 4).
#pragma once

#include <cstdint>

#include "cos_internal.cuh"

namespace cosgpu {

enum Layout : int { LAYOUT_WIDE = 0, LAYOUT_GROUPED = 1, LAYOUT_BULK = 2, LAYOUT_ASYNC = 3 };

template <int V, int LAYOUT>
__host__ __device__ constexpr int chunk_samples() {
    return LAYOUT == LAYOUT_GROUPED ? 32 : 32 * V;
}

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

__device__ __forceinline__ unsigned ld_acquire_gpu_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Philox-4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11): counter (c0..c3),
// key (k0, k1); each round multiplies c0 and c2 by the round constants and mixes the
// high halves with c1, c3 and the key, which advances by the Weyl constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, unsigned k0, unsigned k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Times 2m and 2m+1 of sample number n, uniform in [0, beta): Philox counter
// (n lo, n hi, m, 0) under the key `seed`; the top 53 bits of the word pairs
// (w1:w0) and (w3:w2) scaled by 2^-53.
__device__ __forceinline__ void uniform_time_pair(unsigned long long seed, unsigned long long n, int m, double beta,
                                                  double& a, double& b) {
    const uint4 w = philox4x32_10(make_uint4((unsigned)n, (unsigned)(n >> 32), (unsigned)m, 0u), (unsigned)seed,
                                  (unsigned)(seed >> 32));
    a = beta * ((double)((((unsigned long long)w.y << 32) | w.x) >> 11) * 0x1.0p-53);
    b = beta * ((double)((((unsigned long long)w.w << 32) | w.z) >> 11) * 0x1.0p-53);
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

// Streaming store (evict first): a level's node values are read again only by the
// next level, after the whole slab has been written, so they should not displace the
// parent runs and propagator runs that the current level re-reads from L2.
template <typename T, int V>
__device__ __forceinline__ void store_cs(T* ptr, const VecT<T, V>& x) {
    constexpr int bytes = sizeof(T) * V;
    if constexpr (bytes == 32) {
        uint4 a, b;
        memcpy(&a, &x.v[0], 16);
        memcpy(&b, reinterpret_cast<const char*>(&x.v[0]) + 16, 16);
        __stcs(reinterpret_cast<uint4*>(ptr), a);
        __stcs(reinterpret_cast<uint4*>(ptr) + 1, b);
    } else if constexpr (bytes == 16) {
        uint4 a;
        memcpy(&a, &x.v[0], 16);
        __stcs(reinterpret_cast<uint4*>(ptr), a);
    } else if constexpr (bytes == 8) {
        uint2 a;
        memcpy(&a, &x.v[0], 8);
        __stcs(reinterpret_cast<uint2*>(ptr), a);
    } else {
        unsigned a;
        memcpy(&a, &x.v[0], 4);
        __stcs(reinterpret_cast<unsigned*>(ptr), a);
    }
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

// ---------------------------------------------------------------- bulk copies (TMA engine)

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make mbarrier initialisation visible to the asynchronous (bulk copy) proxy.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this thread's earlier generic-proxy view of global memory before its later
// bulk copies (node values written by other CTAs before the last grid barrier).
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Return the memory of an mbarrier object to ordinary use (required before the shared
// memory is reused by anything but mbarrier operations or initialised again).
__device__ __forceinline__ void mbar_inval(unsigned long long* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ unsigned dynamic_smem_bytes() {
    unsigned v;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
    return v;
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bulk prefetch of `bytes` (multiple of 16, 16-byte aligned address) of global memory
// into L2 by one thread; nothing to wait for and no registers held.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// One bulk copy global -> shared of `bytes` (multiple of 16, both addresses 16-byte
// aligned), completing as transaction bytes on `bar`.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bounded wait for phase `parity` of `bar`: gives up after timeout_ns (checked every
// 64 polls), recording KERR_BARRIER_TIMEOUT; returns false then.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, const WalkParams& p) {
    unsigned long long t0 = 0;
    for (unsigned it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 63) {
            const unsigned long long now = global_timer_ns();
            if (t0 == 0) t0 = now;
            else if ((long long)(now - t0) > p.timeout_ns || it > (1u << 30)) {
                atomicCAS(&p.ctrl->err, 0, KERR_BARRIER_TIMEOUT);
                return false;
            }
        }
    }
}

// ---------------------------------------------------------------- mode traits

// kBase: the arithmetic of the R walk; kAbs: the same walk also accumulates A(s), the
// sum of |path| values, with float node values and products (a scale, not a result).
template <int MODE>
struct Traits;
template <>
struct Traits<COS_MODE_FP64> {       // everything in double
    using Val = double;
    using Prop = double;
    using SinkAcc = double;
    static constexpr bool kCount = false;
    static constexpr bool kAbs = false;
    static constexpr int kBase = COS_MODE_FP64;
};
template <>
struct Traits<COS_MODE_FP32_MIXED> { // float propagators and products, double sink
    using Val = float;
    using Prop = float;
    using SinkAcc = double;
    static constexpr bool kCount = false;
    static constexpr bool kAbs = false;
    static constexpr int kBase = COS_MODE_FP32_MIXED;
};
template <>
struct Traits<COS_MODE_COUNT_I64> {  // unit weights, sums modulo 2^64
    using Val = unsigned long long;
    using Prop = unsigned long long;
    using SinkAcc = unsigned long long;
    static constexpr bool kCount = true;
    static constexpr bool kAbs = false;
    static constexpr int kBase = COS_MODE_COUNT_I64;
};
template <>
struct Traits<kModeFp64Abs> : Traits<COS_MODE_FP64> {
    static constexpr bool kAbs = true;
};
template <>
struct Traits<kModeMixedAbs> : Traits<COS_MODE_FP32_MIXED> {
    static constexpr bool kAbs = true;
};

// |x| as a float, rounded toward zero, by 32-bit integer operations on the two halves
// of x only (no instruction of GB300's slow FP64 pipe); 0 below the float normal
// range, the largest float above it.
__device__ __forceinline__ float abs_to_float(double x) {
    const unsigned hi = (unsigned)__double2hiint(x) & 0x7fffffffu, lo = (unsigned)__double2loint(x);
    const unsigned e = hi >> 20;
    const unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29);   // top 23 of the 52 fraction bits
    const unsigned f = ((e - 1023u + 127u) << 23) | mant;
    return __uint_as_float(e < 1023u - 126u ? 0u : e > 1023u + 127u ? 0x7f7fffffu : f);
}
__device__ __forceinline__ float abs_to_float(float x) { return __uint_as_float(__float_as_uint(x) & 0x7fffffffu); }

// Bulk-copy ring of the level walk: edges in flight per warp, and the shared memory of
// one CTA: kWarps x kRing mbarriers (8 B each) first, then per warp kRing slots of
// parent run + propagator run.
constexpr int kRing = 8;
constexpr int kRingHeader = kWarps * kRing * 8;   // 512 B, a multiple of 128
static_assert(kRingHeader % 128 == 0, "ring slots must stay 128-byte aligned");

template <int MODE, int V>
__host__ __device__ constexpr int bulk_ring_bytes() {
    return kRingHeader + kWarps * kRing *
                     (32 * V * (int)sizeof(typename Traits<MODE>::Val) +
                      (Traits<MODE>::kCount ? 0 : 32 * V * (int)sizeof(typename Traits<MODE>::Prop)));
}

// Async-copy ring of the level walk (LAYOUT_ASYNC): edges in flight per warp; per warp
// kAsyncRing slots, each the warp's parent run then its propagator run (every lane
// copies and later reads only its own V values of both).
constexpr int kAsyncRing = 6;

template <int MODE, int V>
__host__ __device__ constexpr int async_ring_bytes() {
    return kWarps * kAsyncRing * 32 * V *
           ((int)sizeof(typename Traits<MODE>::Val) + (Traits<MODE>::kCount ? 0 : (int)sizeof(typename Traits<MODE>::Prop)));
}

// Per-thread asynchronous copy global -> shared of 4, 8, 16 or 32 bytes (both addresses
// aligned to the size, 16 for 32), committed by the caller as part of a group.
template <int BYTES>
__device__ __forceinline__ void cp_async_lane(void* dst, const void* src) {
    if constexpr (BYTES == 32) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst) + 16u),
                     "l"(static_cast<const char*>(src) + 16)
                     : "memory");
    } else if constexpr (BYTES == 16) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
    } else {
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES) : "memory");
    }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// Keep a computed value ahead of later volatile asm (a copy into the slot it was read from).
__device__ __forceinline__ void order_after(double& x) { asm volatile("" : "+d"(x)); }
__device__ __forceinline__ void order_after(float& x) { asm volatile("" : "+f"(x)); }
__device__ __forceinline__ void order_after(unsigned long long& x) { asm volatile("" : "+l"(x)); }

__device__ __forceinline__ double madd(double p, double g, double acc) { return fma(p, g, acc); }
__device__ __forceinline__ float madd(float p, float g, float acc) { return fmaf(p, g, acc); }

__device__ __forceinline__ void neumaier_add(double& sum, double& comp, double y) {
    const double u = sum + y;
    if (fabs(sum) >= fabs(y)) comp += (sum - u) + y;
    else comp += (y - u) + sum;
    sum = u;
}

// Samples of the tile that starts at sample `base` (tile_n = samples rounded up to the chunk).
struct TileCtx {
    int64_t base;
    int64_t tile_n;
    int nch;
    int c0;   // first chunk of the work item range (a window of chunks; 0 for a whole tile)
};

template <int CHV>
__device__ __forceinline__ TileCtx tile_ctx(const WalkParams& p, int64_t tix) {
    TileCtx tc;
    tc.base = tix * p.tile;
    const int64_t n = min(p.tile, p.S - tc.base);
    tc.tile_n = (n + CHV - 1) / CHV * CHV;
    tc.nch = (int)(tc.tile_n / CHV);
    tc.c0 = 0;
    return tc;
}

// ---------------------------------------------------------------- phase: coefficients (1 item)

// The tau >= 0 and tau < 0 prefactors of every kind.
__device__ __forceinline__ void item_coef(const WalkParams& p) {
    for (int k = threadIdx.x; k < p.K; k += blockDim.x) {
        const double be = p.beta * p.eps[k];
        p.coef[k] = -1.0 / (1.0 + exp(-be));        // tau >= 0: -e^{-eps tau} / (1 + e^{-beta eps})
        p.coef[p.K + k] = 1.0 / (1.0 + exp(be));    // tau <  0: +e^{-eps (tau+beta)} / (1 + e^{-beta eps})
    }
}

// ---------------------------------------------------------------- exponentials

// e^{-x} and e^{+x} in double precision for |x| <= 708, by the table-driven method of
// P. T. P. Tang (ACM TOMS 15, 1989): x = (64 m + j) ln2/64 + r with |r| <= ln2/128,
// e^{+-x} = 2^{+-m} 2^{+-j/64} e^{+-r}; e^{+-r} = 1 + E +- O with the even and odd parts
// of the Taylor series through r^5 (truncation below 4e-17 relative).  The 64 values
// 2^{j/64} (and 2^{-j/64}) are read from `tab` ([0..63] = 2^{j/64}, [64..127] = 2^{-j/64}).
__device__ __forceinline__ void exp_pair(double x, const double* __restrict__ tab, double& em, double& ep) {
    const double inv = 92.33248261689366;                  // 64 / ln 2 (only rounds n)
    const double c_hi = 0.01083042469326756;               // ln2/64 to 32 significant bits: n*c_hi is exact
    const double c_lo = 2.9815858269852933e-12;            // ln2/64 - c_hi
    const double nd = rint(x * inv);
    const int n = (int)nd;
    double r = fma(-nd, c_hi, x);
    r = fma(-nd, c_lo, r);
    const double r2 = r * r;
    const double even = r2 * fma(r2, fma(r2, 1.0 / 720.0, 1.0 / 24.0), 0.5);      // cosh(r) - 1
    const double odd = r * fma(r2, fma(r2, 1.0 / 120.0, 1.0 / 6.0), 1.0);         // sinh(r)
    const int j = n & 63;
    const int m = n >> 6;                                                       // floor(n / 64)
    // e^{+x} = 2^m 2^{j/64} (1 + even + odd);  e^{-x} = 2^{-m} 2^{-j/64} (1 + even - odd)
    const double tp = __ldg(tab + j), tm = __ldg(tab + 64 + j);
    const double vp = fma(tp, even + odd, tp);
    const double vm = fma(tm, even - odd, tm);
    ep = __hiloint2double(__double2hiint(vp) + (m << 20), __double2loint(vp));
    em = __hiloint2double(__double2hiint(vm) - (m << 20), __double2loint(vm));
}

// ---------------------------------------------------------------- float-float helpers

// Leading 24 significant bits of a double as a float, by truncation with 32-bit
// integer operations on the double's two halves only (no FP64 conversion; 64-bit
// integer operations occupy GB300's FP64 pipe); |x| below 2^-126 gives a signed zero.
// The callers keep |x| below 2^127.
__device__ __forceinline__ float trunc_to_float(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned e = (hi >> 20) & 0x7ffu;
    const unsigned sign = hi & 0x80000000u;
    if (e < 1023u - 126u) return __uint_as_float(sign);
    const unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29);
    return __uint_as_float(sign | ((e - 1023u + 127u) << 23) | mant);
}

// The float value f as a double, exactly, with 32-bit integer operations only (normal f or 0).
__device__ __forceinline__ double float_to_double_exact(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0) return 0.0;
    const unsigned hi = (u & 0x80000000u) | ((e - 127u + 1023u) << 20) | ((u & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)((u & 0x7u) << 29));
}

// x = hi + lo with hi, lo floats (about 48 significant bits), one DADD.
__device__ __forceinline__ float2 split_ff(double x) {
    const float hi = trunc_to_float(x);
    return make_float2(hi, trunc_to_float(x - float_to_double_exact(hi)));
}

// Product of two float-float numbers rounded to float: the exact leading product
// hi*hi plus its rounding error (FMA) plus the cross terms, summed once.
__device__ __forceinline__ float mul_ff(float2 a, float2 b) {
    const float x = a.x * b.x;
    float e = fmaf(a.x, b.x, -x);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    return x + e;
}

// Float-float product of two float-float numbers (about 46 significant bits).
__device__ __forceinline__ float2 mul_ff2(float2 a, float2 b) {
    const float x = a.x * b.x;
    float e = fmaf(a.x, b.x, -x);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float hi = x + e;
    return make_float2(hi, e - (hi - x));
}

// 2^m * (hi, lo) by exponent arithmetic; hi must stay normal (the callers keep it
// within 2^{+-100}); a lo that would leave the normal range becomes zero.
__device__ __forceinline__ float2 ldexp_ff(float2 v, int m) {
    const unsigned sh = (unsigned)m << 23;
    const float hi = __uint_as_float(__float_as_uint(v.x) + sh);
    const int elo = (int)((__float_as_uint(v.y) >> 23) & 0xffu) + m;
    const float lo = (elo <= 0 || elo >= 255) ? 0.0f : __uint_as_float(__float_as_uint(v.y) + sh);
    return make_float2(hi, lo);
}

// e^{-x} and e^{+x} as float-float values accurate to about 1e-10 relative, for
// |x| <= 30: the reduction x = (64 m + j) ln2/64 + r is done in double (one rounding
// of n, two FMAs), everything after it in FP32 -- r is below 0.0055, so its float
// rounding and the float polynomial (even and odd parts through r^4 and r^3) change
// e^{+-r} by less than 1e-9 relative; 2^{+-j/64} comes from a float-float table
// `tff` ([0..63] = 2^{j/64}, [64..127] = 2^{-j/64}, each as (hi, lo)).
__device__ __forceinline__ void exp_pair_ff(double x, const float2* __restrict__ tff, float2& em, float2& ep) {
    const float nf = rintf(trunc_to_float(x) * 92.33248261689366f);
    const double nd = (double)(int)nf;
    double r = fma(-nd, 0.01083042469326756, x);
    r = fma(-nd, 2.9815858269852933e-12, r);
    const int n = (int)nf;
    const float rf = trunc_to_float(r);
    const float r2 = rf * rf;
    const float even = r2 * fmaf(r2, 1.0f / 24.0f, 0.5f);
    const float odd = rf * fmaf(r2, 1.0f / 6.0f, 1.0f);
    const int j = n & 63, m = n >> 6;
    const float2 tp = tff[j], tm = tff[64 + j];
    // T (1 + p) = T_hi + (T_lo + T_hi p), renormalised
    const float pp = even + odd, pm = even - odd;
    const float wp = fmaf(tp.x, pp, tp.y), wm = fmaf(tm.x, pm, tm.y);
    const float hp = tp.x + wp, hm = tm.x + wm;
    ep = ldexp_ff(make_float2(hp, wp - (hp - tp.x)), m);
    em = ldexp_ff(make_float2(hm, wm - (hm - tm.x)), -m);
}

// ---------------------------------------------------------------- phase: propagators

// Item = (chunk, kind k); count mode: item = chunk (root values only).
template <int MODE>
__device__ __forceinline__ int prop_items(const WalkParams& p, const TileCtx& tc) {
    if constexpr (Traits<MODE>::kCount) return tc.nch;
    return tc.nch * p.K;
}

// Integer key of a time whose signed 64-bit order is the order of the doubles
// (non-NaN; -0 taken as +0), so that the branch test t_i >= t_j of every slot and
// sample runs on the integer pipes instead of GB300's slow FP64 pipe.  Built and
// compared with 32-bit operations on the two halves only: 64-bit integer operations
// occupy the FP64 pipe too.
__device__ __forceinline__ long long time_order_key(double t) {
    int hi = __double2hiint(t), lo = __double2loint(t);
    if (hi == (int)0x80000000 && lo == 0) hi = 0;   // -0 as +0
    if (hi < 0) {                                    // negative: reverse the magnitude order
        hi ^= 0x7fffffff;
        lo = ~lo;
    }
    return __double_as_longlong(__hiloint2double(hi, lo));
}

// a >= b for two time keys, as signed 64-bit integers (high words signed, then low
// words unsigned), by 32-bit operations.
__device__ __forceinline__ bool key_ge(long long a, long long b) {
    const double da = __longlong_as_double(a), db = __longlong_as_double(b);
    const int ah = __double2hiint(da), bh = __double2hiint(db);
    return ah > bh || (ah == bh && (unsigned)__double2loint(da) >= (unsigned)__double2loint(db));
}

// x with its sign bit flipped by shi (0 or 0x80000000) and then masked by ahi (-1, or
// 0x7fffffff for |x|), on the high word only.
__device__ __forceinline__ double sign_ops(double x, int shi, int ahi) {
    return __hiloint2double((__double2hiint(x) ^ shi) & ahi, __double2loint(x));
}

// Samples of a chunk that one pass of a propagator item keeps in shared memory.
template <int CHV>
__host__ __device__ constexpr int prop_pass_samples() {
    return CHV < 64 ? CHV : 64;
}

// Shared memory of one propagator item: times and exponentials of one pass's samples
// (at most 64 of the chunk's samples at a time).
__host__ __device__ constexpr int prop_smem_bytes(int D, int chv) { return 4 * 8 * D * (chv < 64 ? chv : 64); }

// Load the chunk's t_i for every time i, form e^{-eps_k t_i} (times the tau >= 0 and
// tau < 0 prefactors) and e^{+eps_k t_i} in shared memory, then write every propagator
// slot q = (k, i, j) of this kind:
//   G[c][q][s] = (t_i >= t_j ? coef+ : coef-) e^{-eps_k t_i} e^{+eps_k t_j}
// formed in double, rounded once to the propagator type.  The kind-k slots are the
// contiguous range [kind_slot[k], kind_slot[k+1]); bit 30 of a slot's j field marks a
// fermion-loop edge, whose factor is negated.  The first kind also writes the
// chunk's root values (node 0 holds 1, Fig. 1 caption).  The chunk's samples are
// taken in passes of at most 64 (the shared memory holds one pass).
template <int MODE, int CHV>
__device__ __forceinline__ void item_props(const WalkParams& p, const TileCtx& tc, int item, double* sm) {
    using Tr = Traits<MODE>;
    using Prop = typename Tr::Prop;
    constexpr int PCH = prop_pass_samples<CHV>();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nk = Tr::kCount ? 1 : p.K;
    const int cl = item / nk;   // chunk within the item range
    const int c = tc.c0 + cl;
    const int k = item - cl * nk;
    if (warp == 0 && k == 0)
        for (int v = lane; v < CHV; v += 32) {
            static_cast<typename Tr::Val*>(p.slab[0])[(int64_t)c * p.wmax * CHV + v] = (typename Tr::Val)1;
            if constexpr (Tr::kAbs) static_cast<float*>(p.aslab[0])[(int64_t)c * p.wmax * CHV + v] = 1.0f;
        }
    if constexpr (!Tr::kCount) {
        const int D = p.D;
        const double eps = p.eps[k], cpos = p.coef[k], cneg = p.coef[p.K + k];
        const int q0 = __ldg(p.kind_slot + k), q1 = __ldg(p.kind_slot + k + 1);
        for (int h0 = 0; h0 < CHV; h0 += PCH) {   // pass: samples [h0, h0 + PCH) of the chunk
        const int64_t s0 = tc.base + (int64_t)c * CHV + h0;
        Prop* gt = static_cast<Prop*>(p.gtab) + (int64_t)c * p.P * CHV + h0;
        if (p.ptab) {
            // user-tabulated G_k: linear interpolation on the half of the table that
            // the sign of tau selects (tau = 0 takes the tau >= 0 half), in double,
            // rounded once to the propagator type; end values outside the grid
            double* st = sm;   // [D][PCH] times
            for (int x = threadIdx.x; x < PCH * D; x += blockDim.x) {
                const int i = x / PCH, s = x - i * PCH;
                st[x] = p.t[(int64_t)i * p.t_ld + s0 + s];
            }
            __syncthreads();
            const int T = p.ptab_T;
            const double2* tk = reinterpret_cast<const double2*>(p.ptab) + (int64_t)k * 2 * T;   // (a_m, slope_m)
            for (int q = q0 + warp; q < q1; q += kWarps) {
                const int i = __ldg(p.slot_kij + 3 * q + 1), jw = __ldg(p.slot_kij + 3 * q + 2);
                const int j = jw & 0x3fffffff;
                const int shi = (jw & 0x40000000) ? (int)0x80000000 : 0;   // closes a fermion loop
                const int ahi = p.abs_weights ? 0x7fffffff : -1;            // |G| for A(s)
#pragma unroll
                for (int v = 0; v < PCH / 32; ++v) {
                    const double tau = st[i * PCH + v * 32 + lane] - st[j * PCH + v * 32 + lane];
                    const bool pos = tau >= 0.0;
                    // grid coordinate: tau/h on the tau >= 0 half, (tau + tau_max)/h = tau/h + T
                    // below; every step rounded once (no contraction)
                    const double u = __dadd_rn(__dmul_rn(tau, p.ptab_inv_h), pos ? 0.0 : (double)T);
                    int m = (int)u;
                    double f = __dsub_rn(u, (double)m);
                    if (u < 0.0) {   // before the grid: the first node's value
                        m = 0;
                        f = 0.0;
                    } else if (m >= T) {   // at or past the last node: its value
                        m = T - 1;
                        f = 1.0;
                    }
                    const double2 as = __ldg(tk + (pos ? 0 : T) + m);
                    const double g = sign_ops(__dadd_rn(as.x, __dmul_rn(f, as.y)), shi, ahi);
                    __stcg(gt + (int64_t)q * CHV + v * 32 + lane, (Prop)g);
                }
            }
            __syncthreads();   // the next pass or item reuses the shared memory
            continue;
        }
        // FP32 mode with every factor and its low half inside the normal float range
        // (|eps| beta <= 30, so factors lie within e^{+-60}): exponentials,
        // prefactors and products in float-float FP32 arithmetic (about 1e-10 relative
        // before the single rounding of G to float), instead of double operations on
        // GB300's slow FP64 pipe.
        bool use_ff = (Tr::kBase == COS_MODE_FP32_MIXED && fabs(eps) * p.beta <= 30.0);
        if (use_ff) {
            long long* sk = reinterpret_cast<long long*>(sm);             // [D][PCH] time order keys
            float2* fp_ = reinterpret_cast<float2*>(sm + PCH * D);        // [D][PCH] coef+ e^{-eps t}
            float2* fn_ = fp_ + PCH * D;                                  // [D][PCH] coef- e^{-eps t}
            float2* fe_ = fn_ + PCH * D;                                  // [D][PCH] e^{+eps t}
            const float2 cp2 = split_ff(cpos), cn2 = split_ff(cneg);
            const float2* tff = reinterpret_cast<const float2*>(p.exp_tab + 128);
            bool out_of_range = false;   // times outside [-beta, beta]: take the double path
            for (int x = threadIdx.x; x < PCH * D; x += blockDim.x) {
                const int i = x / PCH, s = x - i * PCH;
                const double t = p.t[(int64_t)i * p.t_ld + s0 + s];
                const double arg = eps * t;
                if (!(fabs(arg) <= 30.0)) {
                    out_of_range = true;
                    continue;
                }
                float2 em, ep;
                exp_pair_ff(arg, tff, em, ep);
                sk[x] = time_order_key(t);
                fp_[x] = mul_ff2(cp2, em);
                fn_[x] = mul_ff2(cn2, em);
                fe_[x] = ep;
            }
            use_ff = !__syncthreads_or(out_of_range);
            if (use_ff) {
                for (int q = q0 + warp; q < q1; q += kWarps) {
                    const int i = __ldg(p.slot_kij + 3 * q + 1), jw = __ldg(p.slot_kij + 3 * q + 2);
                    const int j = jw & 0x3fffffff;
                    const unsigned smask = (jw & 0x40000000) ? 0x80000000u : 0u;   // closes a fermion loop
                    const unsigned amask = p.abs_weights ? 0x7FFFFFFFu : 0xFFFFFFFFu;   // |G| for A(s)
#pragma unroll
                    for (int v = 0; v < PCH / 32; ++v) {
                        const int xi = i * PCH + v * 32 + lane, xj = j * PCH + v * 32 + lane;
                        const float2 a = key_ge(sk[xi], sk[xj]) ? fp_[xi] : fn_[xi];   // tau = t_i - t_j >= 0 ?
                        __stcg(reinterpret_cast<float*>(gt) + (int64_t)q * CHV + v * 32 + lane,
                               __uint_as_float((__float_as_uint(mul_ff(a, fe_[xj])) ^ smask) & amask));
                    }
                }
            }
        }
        if (!use_ff) {
            long long* sk = reinterpret_cast<long long*>(sm);   // [D][PCH] time order keys
            double* sp = sm + PCH * D;        // [D][PCH] coef+ e^{-eps t}
            double* sn = sm + 2 * PCH * D;    // [D][PCH] coef- e^{-eps t}
            double* se = sm + 3 * PCH * D;    // [D][PCH] e^{+eps t}
            for (int x = threadIdx.x; x < PCH * D; x += blockDim.x) {
                const int i = x / PCH, s = x - i * PCH;
                const double t = p.t[(int64_t)i * p.t_ld + s0 + s];
                double em, ep;
                exp_pair(eps * t, p.exp_tab, em, ep);
                sk[x] = time_order_key(t);
                sp[x] = cpos * em;
                sn[x] = cneg * em;
                se[x] = ep;
            }
            __syncthreads();
            for (int q = q0 + warp; q < q1; q += kWarps) {
                const int i = __ldg(p.slot_kij + 3 * q + 1), jw = __ldg(p.slot_kij + 3 * q + 2);
                const int j = jw & 0x3fffffff;
                // closes a fermion loop: flip the sign bit (no extra FP64 operation)
                const int shi = (jw & 0x40000000) ? (int)0x80000000 : 0;
                const int ahi = p.abs_weights ? 0x7fffffff : -1;   // |G| for A(s)
#pragma unroll
                for (int v = 0; v < PCH / 32; ++v) {
                    const int xi = i * PCH + v * 32 + lane, xj = j * PCH + v * 32 + lane;
                    const double a = key_ge(sk[xi], sk[xj]) ? sp[xi] : sn[xi];   // tau = t_i - t_j >= 0 ?
                    const double g = sign_ops(a * se[xj], shi, ahi);
                    __stcg(gt + (int64_t)q * CHV + v * 32 + lane, (Prop)g);
                }
            }
        }
        __syncthreads();   // the next pass or item reuses the shared memory
        }
    }
}

// ---------------------------------------------------------------- phase: one level

__device__ __forceinline__ int level_items(const WalkParams& p, const LevelDesc& ld, const TileCtx& tc) {
    const int rows_per_item = kWarps * p.rows_per_warp;
    return tc.nch * ((ld.width + rows_per_item - 1) / rows_per_item);
}

// Store the V accumulated samples of row r (or, in the sink level, the per-sample results).
// `off` = position of this lane's first sample inside the chunk.
template <int MODE, int V, int CHV>
__device__ __forceinline__ void store_row(const WalkParams& p, bool sink, typename Traits<MODE>::Val* child, int c,
                                          int r, const TileCtx& tc, int off,
                                          const typename Traits<MODE>::Val (&acc)[V]) {
    using Tr = Traits<MODE>;
    using Val = typename Tr::Val;
    if (sink) {
        using Out = typename Tr::SinkAcc;
        Out* R = static_cast<Out*>(p.R);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int64_t s = tc.base + (int64_t)c * CHV + off + v;
            if (s < p.S) R[s] = (Out)acc[v];
        }
    } else {
        VecT<Val, V> out;
#pragma unroll
        for (int v = 0; v < V; ++v) out.v[v] = acc[v];
        store_cs<Val, V>(child + ((int64_t)c * p.wmax + r) * CHV + off, out);
    }
}

// Sink row in FP32 mixed mode: in-edges accumulated as exact double products in double.
// pc / gc (and pa, the A values, when ABS) already point at this lane's samples of the chunk.
template <int V, int CHV, bool ABS = false>
__device__ __forceinline__ void sink_row_mixed(const WalkParams& p, const float* pc, const float* gc, int beg, int end,
                                               int c, const TileCtx& tc, int off, const float* pa = nullptr) {
    double acc[V], acca[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = acca[v] = 0.0;
    for (int e = beg; e < end; ++e) {
        const int2 m = __ldg(p.edges + e);
        const VecT<float, V> pv = load_cg<float, V>(pc + (int64_t)m.x * CHV);
        const VecT<float, V> gv = load_ca<float, V>(gc + (int64_t)m.y * CHV);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] += (double)pv.v[v] * (double)gv.v[v];   // exact product
        if constexpr (ABS) {
            const VecT<float, V> av = load_cg<float, V>(pa + (int64_t)m.x * CHV);
#pragma unroll
            for (int v = 0; v < V; ++v) acca[v] += (double)av.v[v] * (double)abs_to_float(gv.v[v]);
        }
    }
    double* R = static_cast<double*>(p.R);
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int64_t s = tc.base + (int64_t)c * CHV + off + v;
        if (s < p.S) {
            R[s] = acc[v];
            if constexpr (ABS) p.Rabs[s] = acca[v];
        }
    }
}

// Store the V accumulated A values of row r (in the sink level, the per-sample A(s)).
template <int V, int CHV>
__device__ __forceinline__ void store_row_abs(const WalkParams& p, bool sink, float* achild, int c, int r,
                                              const TileCtx& tc, int off, const float (&acc)[V]) {
    if (sink) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int64_t s = tc.base + (int64_t)c * CHV + off + v;
            if (s < p.S) p.Rabs[s] = (double)acc[v];
        }
    } else {
        VecT<float, V> out;
#pragma unroll
        for (int v = 0; v < V; ++v) out.v[v] = acc[v];
        store_cs<float, V>(achild + ((int64_t)c * p.wmax + r) * CHV + off, out);
    }
}

// Wide layout (CHV = 32*V).  Item = (chunk, block of kWarps * rows_per_warp rows),
// chunk-major.  A warp takes rows_per_warp (<= 31) consecutive rows, whose in-edges
// form one contiguous CSR range; it streams that range in windows of 32 edges
// (metadata loaded by the lanes, broadcast by shuffles), keeps U edges' parent and
// propagator loads in flight, and closes a row (store, reset) at its last in-edge.
// Every row is the sum of its in-edges in CSR order, one multiply-add per edge per
// sample.
template <int MODE, int V, bool BALANCE = false, int U_FP32 = 4>
__device__ __forceinline__ void item_level_wide(const WalkParams& p, int l, const TileCtx& tc, int item) {
    using Tr = Traits<MODE>;
    using Val = typename Tr::Val;
    using Prop = typename Tr::Prop;
    constexpr int CHV = 32 * V;
    // edges in flight per warp: 4; 3 for the FP32 walk with A, which holds three 16-byte
    // runs per edge (medium 4.13 ms with 2, 3.89 with 3, 3.98 with 4; the FP64 walk with A:
    // 9.84 ms with 2, 7.82 with 4, 9.34 with 5; the FP64 walk: 6.38 with 4, 6.48 with 5);
    // 8 for the count walk, which holds no propagator runs (medium 3.45 -> 3.13 ms); for
    // the FP32 walk, U_FP32: 4, and 6 in the level-synchronous kernel (80 registers;
    // medium 2.44 -> 2.36 ms), where the work-queue kernel (64 registers) lost with 6
    // (3.47 ms) and the resident server's kernel would spill 124 bytes
    constexpr int U = (Tr::kAbs && Tr::kBase == COS_MODE_FP32_MIXED) ? 3
                      : Tr::kCount                                 ? 8
                      : Tr::kBase == COS_MODE_FP32_MIXED           ? U_FP32
                                                                   : 4;
    const LevelDesc ld = p.levels[l];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rpw = p.rows_per_warp;
    const int rows_per_item = kWarps * rpw;
    const int nrb = (ld.width + rows_per_item - 1) / rows_per_item;
    const int cl = item / nrb;   // chunk within the item range
    const int c = tc.c0 + cl;
    const int rb = item - cl * nrb;
    const bool sink = (l == p.L - 1);
    const int off = lane * V;
    const Val* pc = static_cast<const Val*>(p.slab[(l - 1) & 1]) + (int64_t)c * p.wmax * CHV + off;
    Val* child = static_cast<Val*>(p.slab[l & 1]);
    const Prop* gc = Tr::kCount ? nullptr : static_cast<const Prop*>(p.gtab) + (int64_t)c * p.P * CHV + off;
    // sums of |path| values in the same walk: float node values of A beside those of R
    constexpr bool ABS = Tr::kAbs;
    const float* pa = ABS ? static_cast<const float*>(p.aslab[(l - 1) & 1]) + (int64_t)c * p.wmax * CHV + off : nullptr;
    float* achild = ABS ? static_cast<float*>(p.aslab[l & 1]) : nullptr;
    // levels whose parent slice per chunk is too large for L2 to keep: prefetch ahead,
    // either the next U edges' parent runs line by line (pf) or, one bulk prefetch per
    // lane, the parent runs of a whole window of 32 edges (pfb: the current window at the
    // first window of a row range, the next window at every window)
    const bool pf_level = (int64_t)ld.prev_width * (int64_t)(CHV * sizeof(Val)) > p.pf_slice_bytes;
    const bool pf = pf_level && !p.pf_bulk;
    const bool pfb = pf_level && p.pf_bulk;
    // rows [r0, r0 + nr) of the item, nr <= 31, summed by this warp in CSR order
    auto do_rows = [&](const int r0, const int nr) {
        if constexpr (Tr::kBase == COS_MODE_FP32_MIXED) {
            if (sink) {
                for (int r = r0; r < r0 + nr; ++r) {
                    const int node = ld.row_begin + r;
                    sink_row_mixed<V, CHV, ABS>(p, pc, gc, __ldg(p.row_ptr + node), __ldg(p.row_ptr + node + 1), c,
                                                tc, off, pa);
                }
                return;
            }
        }
        // lane j <= nr holds rp_j = row_ptr of row r0 + j
        const int rp = (lane <= nr) ? __ldg(p.row_ptr + ld.row_begin + r0 + lane) : 0;
        const int rp_next = __shfl_down_sync(0xffffffffu, rp, 1);
        const int beg = __shfl_sync(0xffffffffu, rp, 0);
        const int end = __shfl_sync(0xffffffffu, rp, nr);
        const unsigned nonempty = __ballot_sync(0xffffffffu, lane < nr && rp_next > rp);
        const unsigned empty = __ballot_sync(0xffffffffu, lane < nr && rp_next == rp);
        Val acc[V];
        float acca[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            acc[v] = (Val)0;
            acca[v] = 0.0f;
        }
        for (unsigned m = empty; m; m &= m - 1) {   // rows without in-edges hold 0
            store_row<MODE, V, CHV>(p, sink, child, c, r0 + __ffs(m) - 1, tc, off, acc);
            if constexpr (ABS) store_row_abs<V, CHV>(p, sink, achild, c, r0 + __ffs(m) - 1, tc, off, acca);
        }
        unsigned rows_left = nonempty;
        for (int w0 = beg; w0 < end; w0 += 32) {
            const int n = min(32, end - w0);
            const int2 meta = (lane < n) ? __ldg(p.edges + w0 + lane) : make_int2(0, 0);
            if (pfb) {
                constexpr unsigned RUNB = CHV * sizeof(Val);
                if (w0 == beg && lane < n) {
                    bulk_prefetch_l2(pc - off + (int64_t)meta.x * CHV, RUNB);
                    if constexpr (ABS) bulk_prefetch_l2(pa - off + (int64_t)meta.x * CHV, 4u * CHV);
                }
                if (w0 + 32 + lane < end) {
                    const int src2 = __ldg(&p.edges[w0 + 32 + lane].x);
                    bulk_prefetch_l2(pc - off + (int64_t)src2 * CHV, RUNB);
                    if constexpr (ABS) bulk_prefetch_l2(pa - off + (int64_t)src2 * CHV, 4u * CHV);
                }
            }
            // bit q set <=> edge w0+q is the last in-edge of its row
            const int pos = rp_next - 1 - w0;
            const unsigned ends = __reduce_or_sync(
                0xffffffffu, (lane < nr && rp_next > rp && pos >= 0 && pos < 32) ? (1u << pos) : 0u);
            for (int q0 = 0; q0 < n; q0 += U) {
                if (pf) {   // L2 prefetch of a later batch's U parent runs, one lane per 128-byte line
                    constexpr int LPL = (128 / (int)(sizeof(Val) * V)) - 1;
                    const int ahead = U * p.pf_ahead;
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int qn = q0 + ahead + u;
                        const int sn = __shfl_sync(0xffffffffu, meta.x, qn & 31);
                        if (qn < n && (lane & LPL) == 0) {
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(pc + (int64_t)sn * CHV));
                            if constexpr (ABS) asm volatile("prefetch.global.L2 [%0];" ::"l"(pa + (int64_t)sn * CHV));
                        }
                    }
                }
                VecT<Val, V> pv[U];
                VecT<Prop, V> gv[U];
                VecT<float, V> av[ABS ? U : 1];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int q = q0 + u;
                    const int src = __shfl_sync(0xffffffffu, meta.x, q & 31);
                    pv[u] = load_cg<Val, V>(pc + (int64_t)(q < n ? src : 0) * CHV);
                    if constexpr (ABS) av[u] = load_cg<float, V>(pa + (int64_t)(q < n ? src : 0) * CHV);
                    if constexpr (!Tr::kCount) {
                        const int slot = __shfl_sync(0xffffffffu, meta.y, q & 31);
                        gv[u] = load_ca<Prop, V>(gc + (int64_t)(q < n ? slot : 0) * CHV);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int q = q0 + u;
                    if (q < n) {
                        if constexpr (Tr::kCount) {
#pragma unroll
                            for (int v = 0; v < V; ++v) acc[v] += pv[u].v[v];
                        } else {
#pragma unroll
                            for (int v = 0; v < V; ++v) acc[v] = madd(pv[u].v[v], gv[u].v[v], acc[v]);
                            if constexpr (ABS) {
#pragma unroll
                                for (int v = 0; v < V; ++v)
                                    acca[v] = fmaf(av[u].v[v], abs_to_float(gv[u].v[v]), acca[v]);
                            }
                        }
                        if ((ends >> q) & 1u) {
                            const int r = r0 + __ffs(rows_left) - 1;
                            store_row<MODE, V, CHV>(p, sink, child, c, r, tc, off, acc);
                            if constexpr (ABS) store_row_abs<V, CHV>(p, sink, achild, c, r, tc, off, acca);
                            rows_left &= rows_left - 1;
#pragma unroll
                            for (int v = 0; v < V; ++v) {
                                acc[v] = (Val)0;
                                acca[v] = 0.0f;
                            }
                        }
                    }
                }
            }
        }
    };
    if constexpr (BALANCE) {
        // work-queue items end at a block barrier: split the item's rows into one
        // contiguous range per warp with about the same number of in-edges (rows stay
        // whole).  Warp w's range starts at the first row whose CSR start reaches
        // e0 + w (e1 - e0) / 8; the warp finds both of its ends in two rounds of
        // loads: every 8th row of the item (at most 31 x 8 rows), then the 8 rows of
        // the block the first round points at.
        const int ir0 = rb * rows_per_item, ir1 = min(ir0 + rows_per_item, ld.width);
        const int32_t* rp_item = p.row_ptr + ld.row_begin;
        const int e0 = __ldg(rp_item + ir0), e1 = __ldg(rp_item + ir1);
        const int ta = e0 + (int)((long long)warp * (e1 - e0) / kWarps);
        const int tz = e0 + (int)((long long)(warp + 1) * (e1 - e0) / kWarps);
        const int v1 = __ldg(rp_item + min(ir0 + 8 * lane, ir1));       // rp is non-decreasing; rp[ir1] = e1
        const int fa = __ffs(__ballot_sync(0xffffffffu, v1 >= ta)) - 1;  // first block start at or past ta
        const int fz = __ffs(__ballot_sync(0xffffffffu, v1 >= tz)) - 1;
        const int ba = ir0 + 8 * (fa - 1), bz = ir0 + 8 * (fz - 1);      // the end lies in (b, b + 8]
        const int q = lane & 7;
        // (an end decided by the first round, f = 0, leaves b = ir0 - 8: keep the load inside the item)
        const int v2 = __ldg(rp_item + min(max((lane < 8 ? ba : bz) + 1 + q, ir0), ir1));
        const unsigned ma = __ballot_sync(0xffffffffu, lane < 8 && v2 >= ta) & 0xffu;
        const unsigned mz = (__ballot_sync(0xffffffffu, lane >= 8 && lane < 16 && v2 >= tz) >> 8) & 0xffu;
        const int ra = warp == 0 ? ir0 : (fa == 0 ? ir0 : min(ba + __ffs(ma), ir1));
        const int rz = warp == kWarps - 1 ? ir1 : (fz == 0 ? ir0 : min(bz + __ffs(mz), ir1));
        for (int r0 = ra; r0 < rz; r0 += 31) do_rows(r0, min(31, rz - r0));
    } else {
        const int r0 = rb * rows_per_item + warp * rpw;
        if (r0 >= ld.width) return;
        do_rows(r0, min(rpw, ld.width - r0));
    }
}

// Grouped layout (CHV = 32).  Same items and the same per-row order as the wide
// layout; a warp's rows are split into V groups of consecutive rows and each group
// of 32/V lanes streams the CSR edge range of its own rows, metadata in windows of
// 32/V edges shuffled within the group, U edges' loads in flight per group.
template <int MODE, int V>
__device__ __forceinline__ void item_level_grouped(const WalkParams& p, int l, const TileCtx& tc, int item) {
    using Tr = Traits<MODE>;
    using Val = typename Tr::Val;
    using Prop = typename Tr::Prop;
    constexpr int CHV = 32;
    constexpr int LPR = 32 / V;   // lanes per row
    constexpr int U = 4;          // edges in flight per group
    const LevelDesc ld = p.levels[l];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gid = lane / LPR, gl = lane - gid * LPR;
    const int off = gl * V;
    const int rpw = p.rows_per_warp;
    const int rows_per_item = kWarps * rpw;
    const int nrb = (ld.width + rows_per_item - 1) / rows_per_item;
    const int cl = item / nrb;   // chunk within the item range
    const int c = tc.c0 + cl;
    const int rb = item - cl * nrb;
    const bool sink = (l == p.L - 1);
    const Val* pc = static_cast<const Val*>(p.slab[(l - 1) & 1]) + (int64_t)c * p.wmax * CHV + off;
    Val* child = static_cast<Val*>(p.slab[l & 1]);
    const Prop* gc = Tr::kCount ? nullptr : static_cast<const Prop*>(p.gtab) + (int64_t)c * p.P * CHV + off;
    const int r0 = rb * rows_per_item + warp * rpw;
    if (r0 >= ld.width) return;
    const int nr = min(rpw, ld.width - r0);
    if constexpr (Tr::kBase == COS_MODE_FP32_MIXED) {
        if (sink) {
            if (gid == 0)
                for (int r = r0; r < r0 + nr; ++r) {
                    const int node = ld.row_begin + r;
                    sink_row_mixed<V, CHV>(p, pc, gc, __ldg(p.row_ptr + node), __ldg(p.row_ptr + node + 1), c, tc, off);
                }
            return;
        }
    }
    // lane j <= nr holds rp_j = row_ptr of row r0 + j
    const int rp = (lane <= nr) ? __ldg(p.row_ptr + ld.row_begin + r0 + lane) : 0;
    const int rp_next = __shfl_down_sync(0xffffffffu, rp, 1);
    const unsigned nonempty = __ballot_sync(0xffffffffu, lane < nr && rp_next > rp);
    // rows [ga, gb) (relative to r0) belong to this lane's group
    const int ga = (gid * nr) / V, gb = ((gid + 1) * nr) / V;
    const int ebeg = __shfl_sync(0xffffffffu, rp, ga);
    const int eend = __shfl_sync(0xffffffffu, rp, gb);
    const unsigned group_rows = ((1u << gb) - 1u) & ~((1u << ga) - 1u);
    Val acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = (Val)0;
    for (unsigned m = group_rows & ~nonempty; m; m &= m - 1)   // rows without in-edges hold 0
        store_row<MODE, V, CHV>(p, sink, child, c, r0 + __ffs(m) - 1, tc, off, acc);
    unsigned rows_left = group_rows & nonempty;
    const int len = eend - ebeg;
    int maxlen = len;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) maxlen = max(maxlen, __shfl_xor_sync(0xffffffffu, maxlen, o));
    // lane j < nr: the group owning row j, and that group's first edge
    int gj = 0;
#pragma unroll
    for (int g = 1; g < V; ++g)
        if (lane >= (g * nr) / V) gj = g;
    const int ebeg_j = __shfl_sync(0xffffffffu, rp, (gj * nr) / V);
    // each group streams its edges in windows of LPR: lane gl holds the metadata of edge
    // ebeg + w0 + gl of its own group; shuffles within the group broadcast it
    for (int w0 = 0; w0 < maxlen; w0 += LPR) {
        const int2 meta = (w0 + gl < len) ? __ldg(p.edges + ebeg + w0 + gl) : make_int2(0, 0);
        // bit g*LPR + q set <=> edge w0 + q of group g closes a row
        const int pos = rp_next - 1 - (ebeg_j + w0);
        const unsigned ends = __reduce_or_sync(
            0xffffffffu, (lane < nr && rp_next > rp && pos >= 0 && pos < LPR) ? (1u << (gj * LPR + pos)) : 0u);
#pragma unroll
        for (int q0 = 0; q0 < LPR; q0 += U) {
            if (w0 + q0 >= maxlen) break;
            VecT<Val, V> pv[U];
            VecT<Prop, V> gv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = q0 + u;
                const bool valid = (w0 + q < len);
                const int src = __shfl_sync(0xffffffffu, meta.x, q, LPR);
                pv[u] = load_cg<Val, V>(pc + (int64_t)(valid ? src : 0) * CHV);
                if constexpr (!Tr::kCount) {
                    const int slot = __shfl_sync(0xffffffffu, meta.y, q, LPR);
                    gv[u] = load_ca<Prop, V>(gc + (int64_t)(valid ? slot : 0) * CHV);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = q0 + u;
                if (w0 + q < len) {
                    if constexpr (Tr::kCount) {
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v] += pv[u].v[v];
                    } else {
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v] = madd(pv[u].v[v], gv[u].v[v], acc[v]);
                    }
                    if ((ends >> (gid * LPR + q)) & 1u) {
                        store_row<MODE, V, CHV>(p, sink, child, c, r0 + __ffs(rows_left) - 1, tc, off, acc);
                        rows_left &= rows_left - 1;
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v] = (Val)0;
                    }
                }
            }
        }
    }
}

// Wide layout with a bulk-copy ring (CHV = 32*V).  Same items, rows and per-row order
// as the wide layout; instead of every lane loading its V values, lane 0 of a warp
// copies the whole parent run and propagator run of edge e + kRing into a ring slot
// in shared memory with two bulk copies (the TMA engine) completing on the slot's
// mbarrier, while the warp consumes edge e from shared memory.  kRing edges are in
// flight per warp without holding registers.  Every wait is bounded (mbar_wait); on
// a timeout the item drains its outstanding copies (bounded) and returns false.
template <int MODE, int V>
__device__ __forceinline__ bool item_level_bulk(const WalkParams& p, int l, const TileCtx& tc, int item,
                                                unsigned char* smem) {
    using Tr = Traits<MODE>;
    using Val = typename Tr::Val;
    using Prop = typename Tr::Prop;
    constexpr int CHV = 32 * V;
    constexpr unsigned RUNB = 32 * V * sizeof(Val);
    constexpr unsigned GRUNB = Tr::kCount ? 0 : 32 * V * sizeof(Prop);
    constexpr unsigned SLOTB = RUNB + GRUNB;
    const LevelDesc ld = p.levels[l];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rpw = p.rows_per_warp;
    const int rows_per_item = kWarps * rpw;
    const int nrb = (ld.width + rows_per_item - 1) / rows_per_item;
    const int cl = item / nrb;   // chunk within the item range
    const int c = tc.c0 + cl;
    const int rb = item - cl * nrb;
    const bool sink = (l == p.L - 1);
    const int off = lane * V;
    const Val* pc0 = static_cast<const Val*>(p.slab[(l - 1) & 1]) + (int64_t)c * p.wmax * CHV;
    Val* child = static_cast<Val*>(p.slab[l & 1]);
    const Prop* gc0 = Tr::kCount ? nullptr : static_cast<const Prop*>(p.gtab) + (int64_t)c * p.P * CHV;
    const int r0 = rb * rows_per_item + warp * rpw;
    if (r0 >= ld.width) return true;
    const int nr = min(rpw, ld.width - r0);
    if constexpr (Tr::kBase == COS_MODE_FP32_MIXED) {
        if (sink) {
            for (int r = r0; r < r0 + nr; ++r) {
                const int node = ld.row_begin + r;
                sink_row_mixed<V, CHV>(p, pc0 + off, gc0 + off, __ldg(p.row_ptr + node), __ldg(p.row_ptr + node + 1), c,
                                       tc, off);
            }
            return true;
        }
    }
    // lane j <= nr holds rp_j = row_ptr of row r0 + j
    const int rp = (lane <= nr) ? __ldg(p.row_ptr + ld.row_begin + r0 + lane) : 0;
    const int rp_next = __shfl_down_sync(0xffffffffu, rp, 1);
    const int beg = __shfl_sync(0xffffffffu, rp, 0);
    const int end = __shfl_sync(0xffffffffu, rp, nr);
    const unsigned nonempty = __ballot_sync(0xffffffffu, lane < nr && rp_next > rp);
    const unsigned empty = __ballot_sync(0xffffffffu, lane < nr && rp_next == rp);
    Val acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = (Val)0;
    for (unsigned m = empty; m; m &= m - 1)   // rows without in-edges hold 0
        store_row<MODE, V, CHV>(p, sink, child, c, r0 + __ffs(m) - 1, tc, off, acc);
    if (beg == end) return true;
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem) + warp * kRing;
    unsigned char* ring = smem + kRingHeader + (size_t)warp * kRing * SLOTB;
    if (lane == 0) {
#pragma unroll
        for (int r = 0; r < kRing; ++r) mbar_init(bars + r, 1);
        fence_mbar_init();
        fence_proxy_async_global();
    }
    __syncwarp();
    // metadata windows [wbase, wbase+32) and [wbase+32, wbase+64)
    int wbase = beg;
    int2 meta_a = (beg + lane < end) ? __ldg(p.edges + beg + lane) : make_int2(0, 0);
    int2 meta_b = (beg + 32 + lane < end) ? __ldg(p.edges + beg + 32 + lane) : make_int2(0, 0);
    auto ends_of = [&](int w0) {   // bit q set <=> edge w0+q is the last in-edge of its row
        const int pos = rp_next - 1 - w0;
        return __reduce_or_sync(0xffffffffu,
                                (lane < nr && rp_next > rp && pos >= 0 && pos < 32) ? (1u << pos) : 0u);
    };
    unsigned ends = ends_of(wbase);
    auto issue = [&](int e, int slot) {   // warp-uniform call; lane 0 issues the copies
        const int o = e - wbase;
        const int sa = __shfl_sync(0xffffffffu, meta_a.x, o & 31), sb = __shfl_sync(0xffffffffu, meta_b.x, o & 31);
        const int ga = __shfl_sync(0xffffffffu, meta_a.y, o & 31), gb = __shfl_sync(0xffffffffu, meta_b.y, o & 31);
        if (lane == 0) {
            const int src = o < 32 ? sa : sb;
            const int gslot = o < 32 ? ga : gb;
            unsigned char* dst = ring + (size_t)slot * SLOTB;
#ifdef COS_DEBUG_CHECKS
            // self-check (debug builds): record the first violation and skip the copy
            const unsigned long long sa_ = (unsigned long long)(pc0 + (int64_t)src * CHV);
            const unsigned long long ga_ = Tr::kCount ? 0ull : (unsigned long long)(gc0 + (int64_t)gslot * CHV);
            int bad = 0;
            if (o < 0 || o >= 64) bad = 1;
            else if (src < 0 || src >= ld.prev_width) bad = 2;
            else if (!Tr::kCount && (gslot < 0 || gslot >= p.P)) bad = 3;
            else if ((smem_u32(dst) & 15u) || (sa_ & 15ull) || (ga_ & 15ull)) bad = 4;
            else if (smem_u32(dst) - smem_u32(smem) + SLOTB > dynamic_smem_bytes()) bad = 5;
            else if (smem_u32(bars + slot) & 7u) bad = 6;
            if (bad) {   // complete the slot's phase without a copy so that every wait stays short
                if (atomicCAS(&p.ctrl->err, 0, 100 + bad) == 0) p.ctrl->err_detail = e;
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bars + slot)) : "memory");
                return;
            }
#endif
            mbar_arrive_expect_tx(bars + slot, SLOTB);
            bulk_copy_g2s(dst, pc0 + (int64_t)src * CHV, RUNB, bars + slot);
            if constexpr (!Tr::kCount) bulk_copy_g2s(dst + RUNB, gc0 + (int64_t)gslot * CHV, GRUNB, bars + slot);
        }
    };
    const int n = end - beg;
#pragma unroll
    for (int j = 0; j < kRing; ++j)
        if (j < n) issue(beg + j, j);
    unsigned rows_left = nonempty;
    for (int k = 0; k < n; ++k) {
        const int e = beg + k;
        const int slot = k & (kRing - 1);
        if (!mbar_wait(bars + slot, (unsigned)(k / kRing) & 1u, p)) {
            // drain: the copies issued for edges k+1 .. min(n, k+kRing)-1 (bounded waits)
            for (int k2 = k + 1; k2 < min(n, k + kRing); ++k2)
                (void)mbar_wait(bars + (k2 & (kRing - 1)), (unsigned)(k2 / kRing) & 1u, p);
            return false;   // the kernel stops at its next barrier; the memory is not reused
        }
        const unsigned char* src = ring + (size_t)slot * SLOTB;
        const VecT<Val, V> pv = *reinterpret_cast<const VecT<Val, V>*>(src + off * sizeof(Val));
        if constexpr (Tr::kCount) {
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] += pv.v[v];
        } else {
            const VecT<Prop, V> gv = *reinterpret_cast<const VecT<Prop, V>*>(src + RUNB + off * sizeof(Prop));
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = madd(pv.v[v], gv.v[v], acc[v]);
        }
        if ((ends >> (e - wbase)) & 1u) {
            store_row<MODE, V, CHV>(p, sink, child, c, r0 + __ffs(rows_left) - 1, tc, off, acc);
            rows_left &= rows_left - 1;
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = (Val)0;
        }
        if (e + 1 - wbase == 32) {   // slide the metadata windows
            wbase += 32;
            meta_a = meta_b;
            meta_b = (wbase + 32 + lane < end) ? __ldg(p.edges + wbase + 32 + lane) : make_int2(0, 0);
            ends = ends_of(wbase);
        }
        __syncwarp();   // every lane has read the slot before it is refilled
        if (k + kRing < n) issue(e + kRing, slot);
    }
    __syncwarp();
    if (lane == 0)   // every copy has landed: hand the memory back for other uses
#pragma unroll
        for (int r = 0; r < kRing; ++r) mbar_inval(bars + r);
    __syncwarp();
#ifdef COS_DEBUG_CHECKS
    if (*(volatile int*)&p.ctrl->err > 100) return false;
#endif
    return true;
}

// Wide layout with an async-copy ring (CHV = 32*V).  Same items, rows and per-row
// order as the wide layout.  Instead of holding a few edges' loads in registers, every
// lane copies its V values of the parent run and of the propagator run of edge
// e + kAsyncRing into a ring slot in shared memory (cp.async, one commit group per edge)
// while it consumes edge e from the ring, so kAsyncRing edges stay in flight per warp
// without registers.  A lane reads back only the values it copied itself (no
// synchronisation between lanes), and a slot is refilled only after the multiply-add
// that used its values has issued.
template <int MODE, int V>
__device__ __forceinline__ void item_level_async(const WalkParams& p, int l, const TileCtx& tc, int item,
                                                 unsigned char* smem) {
    using Tr = Traits<MODE>;
    using Val = typename Tr::Val;
    using Prop = typename Tr::Prop;
    constexpr int CHV = 32 * V;
    constexpr int R = kAsyncRing;
    constexpr int VB = V * (int)sizeof(Val);                    // bytes of a lane's parent values
    constexpr int GB = Tr::kCount ? 0 : V * (int)sizeof(Prop);  // ... and propagator values
    constexpr int SB = 32 * (VB + GB);                          // one slot of the warp's ring
    const LevelDesc ld = p.levels[l];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rpw = p.rows_per_warp;
    const int rows_per_item = kWarps * rpw;
    const int nrb = (ld.width + rows_per_item - 1) / rows_per_item;
    const int cl = item / nrb;   // chunk within the item range
    const int c = tc.c0 + cl;
    const int rb = item - cl * nrb;
    const bool sink = (l == p.L - 1);
    const int off = lane * V;
    const Val* pc = static_cast<const Val*>(p.slab[(l - 1) & 1]) + (int64_t)c * p.wmax * CHV + off;
    Val* child = static_cast<Val*>(p.slab[l & 1]);
    const Prop* gc = Tr::kCount ? nullptr : static_cast<const Prop*>(p.gtab) + (int64_t)c * p.P * CHV + off;
    const int r0 = rb * rows_per_item + warp * rpw;
    if (r0 >= ld.width) return;
    const int nr = min(rpw, ld.width - r0);
    if constexpr (Tr::kBase == COS_MODE_FP32_MIXED) {
        if (sink) {
            for (int r = r0; r < r0 + nr; ++r) {
                const int node = ld.row_begin + r;
                sink_row_mixed<V, CHV>(p, pc, gc, __ldg(p.row_ptr + node), __ldg(p.row_ptr + node + 1), c, tc, off);
            }
            return;
        }
    }
    // lane j <= nr holds rp_j = row_ptr of row r0 + j
    const int rp = (lane <= nr) ? __ldg(p.row_ptr + ld.row_begin + r0 + lane) : 0;
    const int rp_next = __shfl_down_sync(0xffffffffu, rp, 1);
    const int beg = __shfl_sync(0xffffffffu, rp, 0);
    const int end = __shfl_sync(0xffffffffu, rp, nr);
    const unsigned nonempty = __ballot_sync(0xffffffffu, lane < nr && rp_next > rp);
    const unsigned empty = __ballot_sync(0xffffffffu, lane < nr && rp_next == rp);
    Val acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = (Val)0;
    for (unsigned m = empty; m; m &= m - 1)   // rows without in-edges hold 0
        store_row<MODE, V, CHV>(p, sink, child, c, r0 + __ffs(m) - 1, tc, off, acc);
    if (beg == end) return;
    unsigned char* ring = smem + (size_t)warp * R * SB;
    unsigned char* mine_p = ring + lane * VB;            // this lane's parent values in slot 0
    unsigned char* mine_g = ring + 32 * VB + lane * GB;  // ... and its propagator values
    // metadata windows [wbase, wbase+32) and [wbase+32, wbase+64)
    int wbase = beg;
    int2 meta_a = (beg + lane < end) ? __ldg(p.edges + beg + lane) : make_int2(0, 0);
    int2 meta_b = (beg + 32 + lane < end) ? __ldg(p.edges + beg + 32 + lane) : make_int2(0, 0);
    auto ends_of = [&](int w0) {   // bit q set <=> edge w0+q is the last in-edge of its row
        const int pos = rp_next - 1 - w0;
        return __reduce_or_sync(0xffffffffu,
                                (lane < nr && rp_next > rp && pos >= 0 && pos < 32) ? (1u << pos) : 0u);
    };
    unsigned ends = ends_of(wbase);
    // copy edge e (within the two windows) into ring slot `slot`; one commit group per call
    auto issue = [&](int e, int slot) {   // warp-uniform call
        const int o = e - wbase;
        const int sa = __shfl_sync(0xffffffffu, meta_a.x, o & 31), sb = __shfl_sync(0xffffffffu, meta_b.x, o & 31);
        const int src = o < 32 ? sa : sb;
        cp_async_lane<VB>(mine_p + slot * SB, pc + (int64_t)src * CHV);
        if constexpr (!Tr::kCount) {
            const int ga = __shfl_sync(0xffffffffu, meta_a.y, o & 31), gb = __shfl_sync(0xffffffffu, meta_b.y, o & 31);
            cp_async_lane<GB>(mine_g + slot * SB, gc + (int64_t)(o < 32 ? ga : gb) * CHV);
        }
        cp_async_commit();
    };
    const int n = end - beg;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        if (j < n) issue(beg + j, j);
        else cp_async_commit();   // empty group: every iteration below waits on the same count
    }
    unsigned rows_left = nonempty;
    int slot = 0;
    for (int k = 0; k < n; ++k) {
        const int e = beg + k;
        cp_async_wait<R - 1>();   // this lane's copies of edge k have landed
        const VecT<Val, V> pv = *reinterpret_cast<const VecT<Val, V>*>(mine_p + slot * SB);
        if constexpr (Tr::kCount) {
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] += pv.v[v];
        } else {
            const VecT<Prop, V> gv = *reinterpret_cast<const VecT<Prop, V>*>(mine_g + slot * SB);
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = madd(pv.v[v], gv.v[v], acc[v]);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) order_after(acc[v]);   // the slot's values are used: it may be refilled
        if ((ends >> (e - wbase)) & 1u) {
            store_row<MODE, V, CHV>(p, sink, child, c, r0 + __ffs(rows_left) - 1, tc, off, acc);
            rows_left &= rows_left - 1;
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = (Val)0;
        }
        if (e + 1 - wbase == 32) {   // the first window is consumed: slide (edge e + R < wbase + 64 then)
            wbase += 32;
            meta_a = meta_b;
            meta_b = (wbase + 32 + lane < end) ? __ldg(p.edges + wbase + 32 + lane) : make_int2(0, 0);
            ends = ends_of(wbase);
        }
        if (k + R < n) issue(e + R, slot);
        else cp_async_commit();
        slot = slot + 1 == R ? 0 : slot + 1;
    }
    cp_async_wait<0>();   // nothing in flight into shared memory that the next item reuses
}

template <int MODE, int V, int LAYOUT, bool BALANCE = false, int U_FP32 = 4>
__device__ __forceinline__ bool item_level(const WalkParams& p, int l, const TileCtx& tc, int item,
                                           unsigned char* smem) {
    static_assert(!Traits<MODE>::kAbs || LAYOUT == LAYOUT_WIDE, "sums of |path| values: wide layout only");
    if constexpr (LAYOUT == LAYOUT_BULK) return item_level_bulk<MODE, V>(p, l, tc, item, smem);
    if constexpr (LAYOUT == LAYOUT_ASYNC) {
        item_level_async<MODE, V>(p, l, tc, item, smem);
        return true;
    }
    if constexpr (LAYOUT == LAYOUT_WIDE) item_level_wide<MODE, V, BALANCE, U_FP32>(p, l, tc, item);
    else item_level_grouped<MODE, V>(p, l, tc, item);
    return true;
}

// ---------------------------------------------------------------- phase: sample reduction

// Error-free sum of two compensated values (Knuth's TwoSum on the leading parts, the
// rounding error folded into the compensation); symmetric, so both lanes of a
// shuffle pair obtain the same result.
__device__ __forceinline__ void add_pair(double& s, double& c, double s2, double c2) {
    const double x = s + s2;
    const double z = x - s;
    const double err = (s - (x - z)) + (s2 - z);
    s = x;
    c = (c + c2) + err;
}

// Compensated sum of one value per lane: pairwise over lanes (xor tree), every lane
// ends with the same (sum, compensation).
__device__ __forceinline__ void warp_sum(double& s, double& c) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) add_pair(s, c, __shfl_xor_sync(0xffffffffu, s, o), __shfl_xor_sync(0xffffffffu, c, o));
}

// Compensated partial sums of R over blocks of kReduceBlock samples in a fixed order:
// lane q adds samples q, q+32, q+64, ... of the block with Neumaier compensation
// (coalesced loads, all issued ahead of the adds), then the lanes are combined by an
// error-free pairwise tree.  Item = kWarps consecutive blocks (one per warp).
__device__ __forceinline__ int partial_items(const WalkParams& p) {
    const int64_t nblk = (p.S + kReduceBlock - 1) / kReduceBlock;
    return (int)((nblk + kWarps - 1) / kWarps);
}

// Compensated sum of block b (kReduceBlock samples) of x, returned on every lane.
template <typename T>
__device__ __forceinline__ double block_sum(const T* __restrict__ x, int64_t S, int64_t b, int lane) {
    constexpr int per_lane = kReduceBlock / 32;
    constexpr int AHEAD = 8;
    const int64_t s0 = b * kReduceBlock + lane;
    double sum = 0.0, comp = 0.0;
#pragma unroll 1
    for (int u0 = 0; u0 < per_lane; u0 += AHEAD) {
        double v[AHEAD];
#pragma unroll
        for (int u = 0; u < AHEAD; ++u) {
            const int64_t s = s0 + (int64_t)(u0 + u) * 32;
            v[u] = s < S ? (double)x[s] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < AHEAD; ++u) neumaier_add(sum, comp, v[u]);
    }
    warp_sum(sum, comp);
    return sum + comp;
}

template <int MODE>
__device__ __forceinline__ void item_partials(const WalkParams& p, int item) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nblk = (p.S + kReduceBlock - 1) / kReduceBlock;
    const int64_t b = (int64_t)item * kWarps + warp;
    if (b >= nblk) return;
    double v;
    if constexpr (Traits<MODE>::kBase == COS_MODE_COUNT_I64) v = block_sum(static_cast<const long long*>(p.R), p.S, b, lane);
    else v = block_sum(static_cast<const double*>(p.R), p.S, b, lane);
    if (lane == 0) p.partials[b] = v;
    if constexpr (Traits<MODE>::kAbs) {
        v = block_sum(p.Rabs, p.S, b, lane);
        if (lane == 0) p.partials_abs[b] = v;
    }
}

// Compensated sum of n block partials (lane-strided Neumaier, then the lane tree).
__device__ __forceinline__ void partials_sum(const double* x, int64_t n, int lane, double& sum, double& comp) {
    sum = 0.0;
    comp = 0.0;
    for (int64_t b = lane; b < n; b += 32) neumaier_add(sum, comp, x[b]);
    warp_sum(sum, comp);
}

// Final compensated sum of the block partials by warp 0 of one CTA; the mean over
// samples (and the mean of A(s) when the walk accumulated it).
__device__ __forceinline__ void item_final(const WalkParams& p) {
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    const int64_t nblk = (p.S + kReduceBlock - 1) / kReduceBlock;
    double sum, comp;
    partials_sum(p.partials, nblk, lane, sum, comp);
    double sa = 0.0, ca = 0.0;
    if (p.partials_abs) partials_sum(p.partials_abs, nblk, lane, sa, ca);
    if (lane == 0) {
        p.ctrl->sum = sum;
        p.ctrl->comp = comp;
        p.ctrl->mean = p.S > 0 ? (sum + comp) / (double)p.S : 0.0;
        p.ctrl->mean_abs = p.S > 0 ? (sa + ca) / (double)p.S : 0.0;
        if (p.mean_out) {   // [0] the mean; [1] the mean of A(s), only when the walk accumulated it
            p.mean_out[0] = p.ctrl->mean;
            if (p.partials_abs) p.mean_out[1] = p.ctrl->mean_abs;
        }
    }
}

}  // namespace cosgpu
