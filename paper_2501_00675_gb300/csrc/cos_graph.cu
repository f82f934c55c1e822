// Host side of the C ABI: graph ingest (validation, per-level dst-sorted CSR,
// propagator slots, exact path count), sample upload, workspace management,
// evaluate dispatch and error reporting.  See include/cos.h for the contract.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "cos_internal.cuh"

using namespace cosgpu;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(COS_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    }
    return fail(COS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define COS_CUDA(call, what)                          \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

template <class T>
void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

constexpr int32_t kSignBit = 0x40000000;   // kind bit 30: the edge closes a fermion loop
constexpr int32_t kKindMask = 0x3fffffff;

// Propagator slot key of an edge row (src, dst, kind|sign, i, j).
int64_t edge_key(const int32_t* r, int32_t D) {
    const int64_t kind = r[2] & kKindMask, neg = (r[2] & kSignBit) ? 1 : 0;
    return (((kind * D) + r[3]) * D + r[4]) * 2 + neg;
}

// (kind, i, j | sign << 30) of a slot key.
void decode_key(int64_t key, int32_t D, int32_t* kij) {
    const int64_t neg = key & 1, rest = key >> 1;
    kij[0] = (int32_t)(rest / ((int64_t)D * D));
    kij[1] = (int32_t)((rest / D) % D);
    kij[2] = (int32_t)(rest % D) | (neg ? kSignBit : 0);
}

// Device arrays of one graph structure, shared by every handle created from it with
// cos_graph_share and freed with the last of them.
struct SharedArrays {
    int device = 0;
    LevelDesc* levels = nullptr;
    int32_t* row_ptr = nullptr;
    int2* edges = nullptr;
    int32_t* slot_kij = nullptr;
    int32_t* kind_slot = nullptr;
    double* exp_tab = nullptr;
    ~SharedArrays() {
        DeviceGuard dg(device);
        dfree(levels);
        dfree(row_ptr);
        dfree(edges);
        dfree(slot_kij);
        dfree(kind_slot);
        dfree(exp_tab);
    }
};

}  // namespace

struct cos_graph {
    int device = 0;
    int32_t L = 0, K = 0, D = 0;
    int64_t N = 0, E = 0, P = 0, Wmax = 0;
    std::vector<int64_t> widths, off, ecount;
    int64_t count_wrapped = 0;
    bool count_overflow = false;
    // device graph
    LevelDesc* d_levels = nullptr;
    int32_t* d_row_ptr = nullptr;
    int2* d_edges = nullptr;
    int32_t* d_slot_kij = nullptr;
    int32_t* d_kind_slot = nullptr;
    double* d_exp_tab = nullptr;
    std::shared_ptr<SharedArrays> arrays;   // owner of the four arrays above once creation succeeded
    Ctrl* d_ctrl = nullptr;
    // samples
    bool has_samples = false;
    int64_t S = 0, t_ld = 0, t_cap = 0;
    double beta = 0.0;
    double* d_t = nullptr;
    double* d_eps = nullptr;
    double* d_stage = nullptr;      // [S][D] staging for host sample-major input
    const double* t_borrowed = nullptr;   // caller's [D][t_ld] times (COS_T_BORROW)
    int64_t stage_cap = 0;
    // workspace
    void* d_arena = nullptr;
    size_t arena_bytes = 0;
    double* d_partials = nullptr;
    int64_t partial_cap = 0;
    void* d_R = nullptr;            // internal per-sample output when the caller passes none
    int64_t R_cap = 0;
    cos_tuning tuning{};
    int last_status_pending = 0;    // 1 while an evaluate has not been collected
    unsigned long long* d_trace = nullptr;   // per-barrier timestamps of the last evaluate
    int32_t trace_cap = 0;
    int last_mode = 0;              // kernel mode id of the last evaluate
    cos_batch_t wave = nullptr;     // one-graph batch of the windowed schedule (created on first use)
    int abs_next = 0;               // the next walk uses |factor| (cos_evaluate_abs)
    double* d_ptab = nullptr;       // user-tabulated propagators [K][2][ptab_T+1], or none
    int32_t ptab_T = 0;
    double ptab_tau_max = 0.0;
    int last_wave = 0;              // the last evaluate ran the windowed schedule
    // Bumped whenever something a batch plan copies from the handle may change: the
    // sample buffers, sample count or layout, the workspace, the internal result
    // buffer, the propagator tables or the tuning.  A batch re-plans when it differs.
    uint64_t generation = 0;
};

namespace {

// Bytes of workspace per sample of a tile in a given kernel mode (two node-value slabs,
// the propagator table, and two float slabs of A when the walk also sums |path| values).
size_t per_sample_bytes(const cos_graph* g, int kmode) {
    const int mode = base_mode(kmode);
    size_t val = (mode == COS_MODE_FP32_MIXED) ? 4 : 8;
    size_t gt = (mode == COS_MODE_COUNT_I64) ? 0 : val;
    size_t ab = mode_has_abs(kmode) ? 2 * sizeof(float) * (size_t)g->Wmax : 0;
    return 2 * val * (size_t)g->Wmax + gt * (size_t)g->P + ab;
}

size_t default_budget_bytes() {
    const char* env = getenv("COS_WORKSPACE_MB");
    if (env && atoll(env) > 0) return (size_t)atoll(env) << 20;
    return (size_t)16 << 30;
}

int default_vec(int kmode) { return base_mode(kmode) == COS_MODE_FP32_MIXED ? 4 : 2; }

// Carve the arena for one tile; returns false if it does not fit.
bool carve(cos_graph* g, int kmode, int64_t tile, WalkParams& p) {
    const int mode = base_mode(kmode);
    size_t val = (mode == COS_MODE_FP32_MIXED) ? 4 : 8;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off += round_up((int64_t)bytes, 256);
        return at;
    };
    size_t s0 = take(val * g->Wmax * tile);
    size_t s1 = take(val * g->Wmax * tile);
    size_t gt = 0;
    if (mode != COS_MODE_COUNT_I64) gt = take(val * g->P * tile);
    size_t a0 = 0, a1 = 0;
    if (mode_has_abs(kmode)) {
        a0 = take(sizeof(float) * g->Wmax * tile);
        a1 = take(sizeof(float) * g->Wmax * tile);
    }
    const size_t cf = take(sizeof(double) * 2 * g->K);
    if (off > g->arena_bytes) return false;
    char* base = (char*)g->d_arena;
    p.slab[0] = base + s0;
    p.slab[1] = base + s1;
    p.aslab[0] = mode_has_abs(kmode) ? (void*)(base + a0) : nullptr;
    p.aslab[1] = mode_has_abs(kmode) ? (void*)(base + a1) : nullptr;
    p.gtab = (mode != COS_MODE_COUNT_I64) ? (void*)(base + gt) : nullptr;
    p.coef = (double*)(base + cf);
    return true;
}

}  // namespace

extern "C" {

const char* cos_last_error(void) { return g_last_error.c_str(); }

int cos_create_graph(int32_t num_levels, const int64_t* level_width, const int64_t* level_edge_count,
                     const int32_t* edges, int32_t num_kinds, int32_t num_times, cos_graph_t* out) {
    if (!out) return fail(COS_ERR_INVALID, "out is NULL");
    if (!level_width || !level_edge_count) return fail(COS_ERR_INVALID, "level arrays are NULL");
    if (num_levels < 2) return fail(COS_ERR_INVALID, "num_levels must be >= 2 (got %d)", num_levels);
    if (num_kinds < 1 || num_times < 1) return fail(COS_ERR_INVALID, "num_kinds and num_times must be >= 1");
    if (num_times > 192) return fail(COS_ERR_INVALID, "num_times must be <= 192 (got %d)", num_times);
    if ((int64_t)num_kinds * num_times > (1LL << 24)) return fail(COS_ERR_INVALID, "num_kinds * num_times too large");
    const int32_t L = num_levels;
    std::vector<int64_t> off(L + 1, 0);
    int64_t E = 0, Wmax = 0;
    for (int32_t l = 0; l < L; ++l) {
        if (level_width[l] < 1) return fail(COS_ERR_INVALID, "level %d has width %lld (must be >= 1)", l, (long long)level_width[l]);
        if (level_edge_count[l] < 0) return fail(COS_ERR_INVALID, "level %d has a negative edge count", l);
        off[l + 1] = off[l] + level_width[l];
        E += level_edge_count[l];
        Wmax = std::max(Wmax, level_width[l]);
        if (off[l + 1] >= (1LL << 31) - 1 || E >= (1LL << 31) - 1)
            return fail(COS_ERR_INVALID, "graph too large (N and E must be < 2^31)");
    }
    if (level_width[0] != 1 || level_width[L - 1] != 1)
        return fail(COS_ERR_INVALID, "the first and last levels must have width 1 (root and sink)");
    if (level_edge_count[0] != 0) return fail(COS_ERR_INVALID, "level 0 (root) cannot have in-edges");
    if (E > 0 && !edges) return fail(COS_ERR_INVALID, "edges is NULL");
    const int64_t N = off[L];

    // Validate every edge against its level, and number the propagator slots.
    // slot key = ((kind * D + i) * D + j) * 2 + fermion-loop sign (kind bit 30)
    const int64_t key_space = (int64_t)num_kinds * num_times * num_times * 2;
    const bool dense = key_space <= (1LL << 22);
    std::vector<int32_t> dense_slot;
    if (dense) dense_slot.assign((size_t)key_space, -1);
    std::vector<int64_t> keys;
    if (!dense) keys.reserve((size_t)E);
    int64_t e0 = 0;
    for (int32_t l = 1; l < L; ++l) {
        for (int64_t q = e0; q < e0 + level_edge_count[l]; ++q) {
            const int32_t* r = edges + 5 * q;
            if (r[0] < off[l - 1] || r[0] >= off[l])
                return fail(COS_ERR_INVALID, "edge %lld into level %d: src %d is not in level %d", (long long)q, l, r[0], l - 1);
            if (r[1] < off[l] || r[1] >= off[l + 1])
                return fail(COS_ERR_INVALID, "edge %lld into level %d: dst %d is not in level %d", (long long)q, l, r[1], l);
            if (r[2] < 0 || (r[2] & kKindMask) >= num_kinds)
                return fail(COS_ERR_INVALID, "edge %lld: kind %d out of range [0,%d)", (long long)q, r[2] & kKindMask, num_kinds);
            if (r[3] < 0 || r[3] >= num_times || r[4] < 0 || r[4] >= num_times)
                return fail(COS_ERR_INVALID, "edge %lld: time index out of range [0,%d)", (long long)q, num_times);
            int64_t key = edge_key(r, num_times);
            if (dense) dense_slot[(size_t)key] = 0;
            else keys.push_back(key);
        }
        e0 += level_edge_count[l];
    }
    std::vector<int32_t> slot_kij;
    int64_t P = 0;
    if (dense) {
        for (int64_t key = 0; key < key_space; ++key)
            if (dense_slot[(size_t)key] == 0) dense_slot[(size_t)key] = (int32_t)P++;
        slot_kij.resize((size_t)(3 * P));
        for (int64_t key = 0; key < key_space; ++key) {
            int32_t s = dense_slot[(size_t)key];
            if (s < 0) continue;
            decode_key(key, num_times, slot_kij.data() + 3 * s);
        }
    } else {
        std::sort(keys.begin(), keys.end());
        keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
        P = (int64_t)keys.size();
        slot_kij.resize((size_t)(3 * P));
        for (int64_t s = 0; s < P; ++s) {
            decode_key(keys[(size_t)s], num_times, slot_kij.data() + 3 * s);
        }
    }

    // Rows of a level whose parent level is too wide for a chunk's parent values to
    // stay in L2 (>= 65536 nodes) are renumbered by their smallest (renumbered)
    // parent, so that consecutive rows -- one work item -- read nearby parents while
    // those are still in L2 (large mixed 3.86 -> 3.78 s per step on GB300).  Narrower
    // levels keep the input order: there the sort only groups rows of many parents
    // and unbalances statically assigned items.  Node numbers inside a level never
    // reach the results: every row keeps its in-edges and their input order, and the
    // root and the sink are alone on their levels.
    std::vector<int32_t> perm_prev(1, 0), perm;   // old local index -> new local index
    std::vector<std::pair<int64_t, int32_t>> order;
    // Per-level stable counting sort by (renumbered) destination: CSR rows in the new
    // order, in-edges of one node in input order.
    std::vector<int32_t> row_ptr((size_t)N + 1, 0);
    std::vector<int2> csr((size_t)E);
    std::vector<int64_t> cnt;
    e0 = 0;
    for (int32_t l = 1; l < L; ++l) {
        const int64_t W = level_width[l];
        order.assign((size_t)W, std::make_pair(INT64_MAX, 0));
        for (int64_t r = 0; r < W; ++r) order[(size_t)r].second = (int32_t)r;
        for (int64_t q = e0; q < e0 + level_edge_count[l]; ++q) {
            int64_t& k = order[(size_t)(edges[5 * q + 1] - off[l])].first;
            k = std::min<int64_t>(k, perm_prev[(size_t)(edges[5 * q] - off[l - 1])]);
        }
        if (level_width[l - 1] >= 65536)
            std::stable_sort(order.begin(), order.end(),
                             [](const std::pair<int64_t, int32_t>& a, const std::pair<int64_t, int32_t>& b) {
                                 return a.first < b.first;
                             });
        perm.assign((size_t)W, 0);
        for (int64_t r = 0; r < W; ++r) perm[(size_t)order[(size_t)r].second] = (int32_t)r;
        cnt.assign((size_t)W + 1, 0);
        for (int64_t q = e0; q < e0 + level_edge_count[l]; ++q)
            cnt[(size_t)perm[(size_t)(edges[5 * q + 1] - off[l])] + 1]++;
        for (int64_t r = 0; r < W; ++r) cnt[(size_t)r + 1] += cnt[(size_t)r];
        for (int64_t r = 0; r < W; ++r) row_ptr[(size_t)(off[l] + r)] = (int32_t)(e0 + cnt[(size_t)r]);
        for (int64_t q = e0; q < e0 + level_edge_count[l]; ++q) {
            const int32_t* r = edges + 5 * q;
            int64_t pos = e0 + cnt[(size_t)perm[(size_t)(r[1] - off[l])]]++;
            int64_t key = edge_key(r, num_times);
            int32_t slot = dense ? dense_slot[(size_t)key]
                                 : (int32_t)(std::lower_bound(keys.begin(), keys.end(), key) - keys.begin());
            csr[(size_t)pos] = make_int2(perm_prev[(size_t)(r[0] - off[l - 1])], slot);
        }
        e0 += level_edge_count[l];
        perm_prev.swap(perm);
    }
    row_ptr[(size_t)N] = (int32_t)E;   // (root row: row_ptr[0] = row_ptr[1] = 0)
    row_ptr[0] = 0;

    // Exact path count (unit weights), 128-bit with saturation, for the overflow flag.
    std::vector<unsigned __int128> cexact((size_t)N, 0);
    std::vector<uint64_t> cwrap((size_t)N, 0);
    cexact[0] = 1;
    cwrap[0] = 1;
    const unsigned __int128 cap = ((unsigned __int128)1) << 120;
    for (int32_t l = 1; l < L; ++l)
        for (int64_t r = off[l]; r < off[l + 1]; ++r)
            for (int32_t q = row_ptr[(size_t)r]; q < row_ptr[(size_t)r + 1]; ++q) {
                int64_t src = off[l - 1] + csr[(size_t)q].x;
                unsigned __int128 x = cexact[(size_t)r] + cexact[(size_t)src];
                cexact[(size_t)r] = x > cap ? cap : x;
                cwrap[(size_t)r] += cwrap[(size_t)src];
            }

    cos_graph* g = new (std::nothrow) cos_graph();
    if (!g) return fail(COS_ERR_OOM, "host allocation failed");
    g->L = L; g->K = num_kinds; g->D = num_times; g->N = N; g->E = E; g->P = P; g->Wmax = Wmax;
    g->widths.assign(level_width, level_width + L);
    g->ecount.assign(level_edge_count, level_edge_count + L);
    g->off = off;
    g->count_wrapped = (int64_t)cwrap[(size_t)N - 1];
    g->count_overflow = cexact[(size_t)N - 1] > (unsigned __int128)INT64_MAX;
    if (cudaGetDevice(&g->device) != cudaSuccess) {
        delete g;
        return fail(COS_ERR_CUDA, "no CUDA device");
    }
    std::vector<LevelDesc> lv((size_t)L);
    for (int32_t l = 0; l < L; ++l) {
        lv[(size_t)l].row_begin = (int32_t)off[l];
        lv[(size_t)l].width = (int32_t)level_width[l];
        lv[(size_t)l].prev_width = l ? (int32_t)level_width[l - 1] : 0;
        lv[(size_t)l].pad = 0;
    }
    auto cleanup_fail = [&](cudaError_t e, const char* what) {
        int rc = cuda_fail(e, what);
        cos_destroy(g);
        return rc;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&g->d_levels, sizeof(LevelDesc) * L)) != cudaSuccess) return cleanup_fail(e, "cudaMalloc levels");
    if ((e = cudaMalloc(&g->d_row_ptr, sizeof(int32_t) * (N + 1))) != cudaSuccess) return cleanup_fail(e, "cudaMalloc row_ptr");
    if ((e = cudaMalloc(&g->d_edges, sizeof(int2) * std::max<int64_t>(E, 1))) != cudaSuccess) return cleanup_fail(e, "cudaMalloc edges");
    if ((e = cudaMalloc(&g->d_slot_kij, sizeof(int32_t) * std::max<int64_t>(3 * P, 3))) != cudaSuccess) return cleanup_fail(e, "cudaMalloc slots");
    if ((e = cudaMalloc(&g->d_ctrl, sizeof(Ctrl))) != cudaSuccess) return cleanup_fail(e, "cudaMalloc ctrl");
    {
        // slots are numbered in (kind, i, j) order, so every kind owns one contiguous range
        std::vector<int32_t> ks((size_t)num_kinds + 1, 0);
        for (int64_t q = 0; q < P; ++q) ks[(size_t)slot_kij[3 * q] + 1]++;
        for (int32_t k = 0; k < num_kinds; ++k) ks[(size_t)k + 1] += ks[(size_t)k];
        // 2^{j/64} and 2^{-j/64}, j = 0..63, for the table-driven exponentials
        // followed by the same values as float-float pairs (hi, lo) for the FP32 path
        std::vector<double> tab(128 + 128);
        float* tff = reinterpret_cast<float*>(tab.data() + 128);
        for (int j = 0; j < 64; ++j) {
            const long double vp = std::exp2l((long double)j / 64.0L), vm = std::exp2l(-(long double)j / 64.0L);
            tab[(size_t)j] = (double)vp;
            tab[(size_t)j + 64] = (double)vm;
            const float hp = (float)vp, hm = (float)vm;
            tff[2 * j] = hp;
            tff[2 * j + 1] = (float)(vp - (long double)hp);
            tff[2 * (64 + j)] = hm;
            tff[2 * (64 + j) + 1] = (float)(vm - (long double)hm);
        }
        if ((e = cudaMalloc(&g->d_kind_slot, sizeof(int32_t) * (num_kinds + 1))) != cudaSuccess) return cleanup_fail(e, "cudaMalloc kind slots");
        if ((e = cudaMalloc(&g->d_exp_tab, sizeof(double) * tab.size())) != cudaSuccess) return cleanup_fail(e, "cudaMalloc exp table");
        if ((e = cudaMemcpy(g->d_kind_slot, ks.data(), sizeof(int32_t) * (num_kinds + 1), cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail(e, "copy kind slots");
        if ((e = cudaMemcpy(g->d_exp_tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail(e, "copy exp table");
    }
    if ((e = cudaMemcpy(g->d_levels, lv.data(), sizeof(LevelDesc) * L, cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail(e, "copy levels");
    if ((e = cudaMemcpy(g->d_row_ptr, row_ptr.data(), sizeof(int32_t) * (N + 1), cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail(e, "copy row_ptr");
    if (E && (e = cudaMemcpy(g->d_edges, csr.data(), sizeof(int2) * E, cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail(e, "copy edges");
    if (P && (e = cudaMemcpy(g->d_slot_kij, slot_kij.data(), sizeof(int32_t) * 3 * P, cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail(e, "copy slots");
    if ((e = cudaMemset(g->d_ctrl, 0, sizeof(Ctrl))) != cudaSuccess) return cleanup_fail(e, "memset ctrl");
    auto arr = std::make_shared<SharedArrays>();
    arr->device = g->device;
    arr->levels = g->d_levels;
    arr->row_ptr = g->d_row_ptr;
    arr->edges = g->d_edges;
    arr->slot_kij = g->d_slot_kij;
    arr->kind_slot = g->d_kind_slot;
    arr->exp_tab = g->d_exp_tab;
    g->arrays = std::move(arr);
    *out = g;
    return COS_OK;
}

int cos_graph_share(cos_graph_t src, cos_graph_t* out) {
    if (!src || !out) return fail(COS_ERR_INVALID, "bad arguments");
    if (!src->arrays) return fail(COS_ERR_STATE, "source graph is incomplete");
    cos_graph* g = new (std::nothrow) cos_graph();
    if (!g) return fail(COS_ERR_OOM, "host allocation failed");
    g->device = src->device;
    g->L = src->L; g->K = src->K; g->D = src->D; g->N = src->N; g->E = src->E; g->P = src->P; g->Wmax = src->Wmax;
    g->widths = src->widths;
    g->off = src->off;
    g->ecount = src->ecount;
    g->count_wrapped = src->count_wrapped;
    g->count_overflow = src->count_overflow;
    g->d_levels = src->d_levels;
    g->d_row_ptr = src->d_row_ptr;
    g->d_edges = src->d_edges;
    g->d_slot_kij = src->d_slot_kij;
    g->d_kind_slot = src->d_kind_slot;
    g->d_exp_tab = src->d_exp_tab;
    g->arrays = src->arrays;
    g->tuning = src->tuning;
    DeviceGuard dg(g->device);
    cudaError_t e = cudaMalloc(&g->d_ctrl, sizeof(Ctrl));
    if (e == cudaSuccess) e = cudaMemset(g->d_ctrl, 0, sizeof(Ctrl));
    if (e == cudaSuccess && src->d_ptab) {   // the propagator tables are copied, not shared
        const size_t bytes = sizeof(double) * 2 * 2 * (size_t)src->ptab_T * (size_t)src->K;
        e = cudaMalloc(&g->d_ptab, bytes);
        if (e == cudaSuccess) e = cudaMemcpy(g->d_ptab, src->d_ptab, bytes, cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess) {
            g->ptab_T = src->ptab_T;
            g->ptab_tau_max = src->ptab_tau_max;
        }
    }
    if (e != cudaSuccess) {
        int rc = cuda_fail(e, "cudaMalloc ctrl");
        cos_destroy(g);
        return rc;
    }
    *out = g;
    return COS_OK;
}

int cos_destroy(cos_graph_t g) {
    if (!g) return COS_OK;
    {
        DeviceGuard dg(g->device);
        if (g->wave) cos_batch_destroy(g->wave);
        g->wave = nullptr;
        dfree(g->d_ptab);
        if (g->arrays) {
            g->arrays.reset();   // frees the structure arrays with the last handle sharing them
        } else {
            dfree(g->d_levels);
            dfree(g->d_row_ptr);
            dfree(g->d_edges);
            dfree(g->d_slot_kij);
            dfree(g->d_kind_slot);
            dfree(g->d_exp_tab);
        }
        dfree(g->d_ctrl);
        dfree(g->d_t);
        dfree(g->d_eps);
        dfree(g->d_stage);
        if (g->d_arena) cudaFree(g->d_arena);
        g->d_arena = nullptr;
        dfree(g->d_partials);
        dfree(g->d_trace);
        if (g->d_R) cudaFree(g->d_R);
        g->d_R = nullptr;
    }
    delete g;
    return COS_OK;
}

int cos_graph_info(cos_graph_t g, int64_t* info, int32_t n) {
    if (!g || !info || n < 0) return fail(COS_ERR_INVALID, "bad arguments");
    const int64_t v[10] = {g->L, g->N, g->E, g->P, g->Wmax, g->count_wrapped, g->count_overflow ? 1 : 0,
                           g->K, g->D, g->device};
    for (int32_t q = 0; q < n && q < 10; ++q) info[q] = v[q];
    return COS_OK;
}

int cos_set_tuning(cos_graph_t g, const cos_tuning* t) {
    if (!g || !t) return fail(COS_ERR_INVALID, "bad arguments");
    if (t->samples_per_lane > 0 && t->samples_per_lane != 1 && t->samples_per_lane != 2 && t->samples_per_lane != 4)
        return fail(COS_ERR_INVALID, "samples_per_lane must be 1, 2 or 4");
    if (t->rows_per_warp > 31) return fail(COS_ERR_INVALID, "rows_per_warp must be <= 31");
    if (t->blocks_per_sm > 32) return fail(COS_ERR_INVALID, "blocks_per_sm must be <= 32");
    if (t->layout < 0 || t->layout > 4)
        return fail(COS_ERR_INVALID,
                    "layout must be 0 (auto), 1 (wide), 2 (grouped), 3 (wide, bulk-copy ring) or 4 (wide, async-copy ring)");
    if (t->schedule < 0 || t->schedule > 2)
        return fail(COS_ERR_INVALID, "schedule must be 0 (auto), 1 (level-synchronous) or 2 (windowed)");
    if (t->window_chunks < 0) return fail(COS_ERR_INVALID, "window_chunks must be >= 0");
    if (t->prefetch < 0 || t->prefetch > 7)
        return fail(COS_ERR_INVALID,
                    "prefetch must be 0 (auto), 1 (off), 2/4/6 (large parent slices) or 3/5/7 (always)");
    g->tuning = *t;
    g->generation++;
    return COS_OK;
}

static int resolve_tuning(cos_graph_t g, int kmode, cos_tuning* out, int64_t* tile_out) {
    const int mode = base_mode(kmode);
    cos_tuning t = g->tuning;
    if (t.samples_per_lane <= 0) t.samples_per_lane = default_vec(kmode);
    // Measured on GB300: the work queue (dynamic item assignment, dependency counters)
    // is ahead on large FP64 walks and on graphs with very wide levels; the cooperative
    // kernel on the FP32 and count walks of smaller graphs and on small evaluations,
    // where the work queue's per-call planning and upload are not amortised.
    // (with the FP32 work-queue walker at four CTAs per SM the FP32 walk of medium graphs
    // joined the FP64 one there: medium mixed 2.44 -> 2.36 ms; the level-synchronous
    // walker with six edges in flight per warp later matched it, 2.36 ms)
    const bool big = (double)g->E * (double)g->S >= 1e9;
    if (t.schedule <= 0)
        t.schedule = ((big && (mode == COS_MODE_FP64 || mode == COS_MODE_FP32_MIXED)) || g->Wmax >= 65536) ? 2 : 1;
    // level-synchronous: 8 rows per warp measured best for the FP32 walk (medium: 2.46 ms
    // against 2.50 with 16 and 2.88 with 31)
    if (t.rows_per_warp <= 0) {
        if (t.schedule == 2)   // FP32 below 65,536 nodes per level: 16 (medium 2.36 ms against 2.50 with 31)
            t.rows_per_warp = (mode == COS_MODE_FP32_MIXED && g->Wmax < 65536) ? 16 : 31;
        else
            t.rows_per_warp = mode == COS_MODE_FP64 ? 4 : mode == COS_MODE_FP32_MIXED ? 8 : 16;
    }
    if (t.layout <= 0 || mode_has_abs(kmode)) t.layout = 1;   // sums of |path| values: wide layout only
    if (t.timeout_ms <= 0) {
        const char* env = getenv("COS_TIMEOUT_MS");
        t.timeout_ms = (env && atoi(env) > 0) ? atoi(env) : 10000;
    }
    // the propagator phase keeps 4 x D x (32 * samples_per_lane) doubles in shared memory
    while (t.samples_per_lane > 1 && (t.layout == 1 || t.layout == 4) &&
           walk_smem_bytes(kmode, t.samples_per_lane, t.layout, g->D) > (160 << 10))
        t.samples_per_lane /= 2;
    // occupancy of the kernel this schedule runs (the work queue's may differ)
    int dev_max = t.schedule == 2 ? batch_coresident_blocks(kmode, t.samples_per_lane, t.layout, g->D, g->device)
                                  : max_coresident_blocks(kmode, t.samples_per_lane, t.layout, g->D, g->device);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    if (dev_max <= 0 || sms <= 0) return fail(COS_ERR_CUDA, "cannot query occupancy of the walker kernel");
    int per_sm = dev_max / sms;
    if (t.blocks_per_sm <= 0 || t.blocks_per_sm > per_sm) t.blocks_per_sm = per_sm;
    const int64_t ch = t.layout == 2 ? 32 : 32LL * t.samples_per_lane;   // samples per chunk
    int64_t need = std::max<int64_t>(round_up(std::max<int64_t>(g->S, 1), ch), ch);
    int64_t tile;
    if (t.tile_samples > 0) {
        tile = round_up(t.tile_samples, ch);
        if (mode_has_abs(kmode)) {
            // the workspace was sized for the walks without A: a fixed tile is an upper
            // bound for the walk that also keeps A's node values
            const size_t slack = (size_t)4 << 20;
            const int64_t fit = g->arena_bytes > slack ? (int64_t)((g->arena_bytes - slack) / (per_sample_bytes(g, kmode) + 1)) : 0;
            tile = std::min<int64_t>(tile, std::max<int64_t>(ch, fit / ch * ch));
        }
    } else {
        size_t psb = per_sample_bytes(g, kmode);
        const size_t slack = (size_t)4 << 20;   // alignment padding and coefficients
        int64_t fit = g->arena_bytes > slack ? (int64_t)((g->arena_bytes - slack) / (psb + 1)) : 0;
        tile = std::max<int64_t>(ch, fit / ch * ch);
        tile = std::min<int64_t>(tile, 65536);
    }
    tile = std::min(tile, need);
    t.tile_samples = (int32_t)tile;
    // four windows per tile unless asked: one window's propagator phase overlaps the
    // others' levels (medium FP64 6.67 -> 6.56 ms); small windows (kept in L2) measured slower
    if (t.window_chunks <= 0) t.window_chunks = (int32_t)std::max<int64_t>(1, (tile / ch + 3) / 4);
    if (t.prefetch <= 0) t.prefetch = 2;
    *out = t;
    *tile_out = tile;
    return COS_OK;
}

int cos_get_tuning(cos_graph_t g, int32_t mode, cos_tuning* tuning) {
    if (!g || !tuning) return fail(COS_ERR_INVALID, "bad arguments");
    const int km = kernel_mode(mode);
    if (km < 0) return fail(COS_ERR_INVALID, "bad mode %d", mode);
    int64_t tile;
    return resolve_tuning(g, km, tuning, &tile);
}

int cos_autotune(cos_graph_t g, int32_t mode, void* per_sample_out, void* stream, cos_tuning* best_out) {
    if (!g) return fail(COS_ERR_INVALID, "graph is NULL");
    const int km = kernel_mode(mode);
    if (km < 0) return fail(COS_ERR_INVALID, "bad mode %d", mode);
    if (!g->has_samples) return fail(COS_ERR_STATE, "cos_set_samples has not been called");
    DeviceGuard dg(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    const cos_tuning base = g->tuning;
    // candidates: both schedules, 8/16/31 rows per warp, the mode's two useful widths;
    // fields the caller set (> 0) stay fixed
    const int scheds[] = {1, 2};
    const int rpws[] = {8, 16, 31};
    const int vecs_fp64[] = {2, 1}, vecs_mixed[] = {4, 2}, vecs_count[] = {2, 4};
    const int* vecs = base_mode(km) == COS_MODE_FP64 ? vecs_fp64
                      : base_mode(km) == COS_MODE_FP32_MIXED ? vecs_mixed : vecs_count;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(COS_ERR_CUDA, "cannot create timing events");
    float best_ms = 1e30f;
    cos_tuning best = base;
    int rc = COS_OK;
    for (int sc : scheds)
        for (int r : rpws)
            for (int vi = 0; vi < 2 && rc == COS_OK; ++vi) {
                cos_tuning t = base;
                if (base.schedule <= 0) t.schedule = sc;
                else if (sc != scheds[0]) continue;
                if (base.rows_per_warp <= 0) t.rows_per_warp = r;
                else if (r != rpws[0]) continue;
                if (base.samples_per_lane <= 0) t.samples_per_lane = vecs[vi];
                else if (vi > 0) continue;
                g->tuning = t;
                float ms_best = 1e30f;
                for (int rep = 0; rep < 3 && rc == COS_OK; ++rep) {   // the first run warms up
                    cudaEventRecord(e0, st);
                    rc = cos_evaluate(g, mode, per_sample_out, nullptr, stream);
                    cudaEventRecord(e1, st);
                    if (rc != COS_OK) break;
                    rc = cos_get_result(g, nullptr, stream);
                    if (rc == COS_ERR_OVERFLOW) rc = COS_OK;
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0) ms_best = std::min(ms_best, ms);
                }
                if (rc == COS_OK && ms_best < best_ms) {
                    best_ms = ms_best;
                    best = t;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g->tuning = rc == COS_OK ? best : base;
    g->generation++;
    if (rc != COS_OK) return rc;
    if (best_out) {
        int64_t tile;
        return resolve_tuning(g, km, best_out, &tile);
    }
    return COS_OK;
}

int cos_set_samples(cos_graph_t g, int64_t num_samples, const double* t, int32_t t_flags, const double* eps,
                    double beta, void* stream) {
    if (!g) return fail(COS_ERR_INVALID, "graph is NULL");
    if (num_samples < 0) return fail(COS_ERR_INVALID, "num_samples must be >= 0");
    if (num_samples > 0 && !t) return fail(COS_ERR_INVALID, "t is NULL");
    if (!eps) return fail(COS_ERR_INVALID, "eps is NULL");
    if (t_flags & ~(COS_T_HOST | COS_T_SAMPLE_MAJOR | COS_T_BORROW)) return fail(COS_ERR_INVALID, "unknown t_flags bits");
    if ((t_flags & COS_T_BORROW) && (t_flags & (COS_T_HOST | COS_T_SAMPLE_MAJOR)))
        return fail(COS_ERR_INVALID, "COS_T_BORROW needs a device [D][t_ld] buffer");
    if (!(beta > 0.0) || !std::isfinite(beta)) return fail(COS_ERR_INVALID, "beta must be positive and finite");
    for (int32_t k = 0; k < g->K; ++k)
        if (!std::isfinite(eps[k]) || std::fabs(eps[k]) * beta > 600.0)
            return fail(COS_ERR_INVALID, "eps[%d] * beta must be finite with magnitude <= 600", k);
    DeviceGuard dg(g->device);
    if (!dg.ok) return fail(COS_ERR_CUDA, "cannot select device %d", g->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t S = num_samples;
    const int64_t t_ld = std::max<int64_t>(round_up(S, 128), 128);
    const int32_t D = g->D;
    const bool borrow = (t_flags & COS_T_BORROW) != 0;
    if (!borrow && t_ld * D > g->t_cap) {
        dfree(g->d_t);
        COS_CUDA(cudaMalloc(&g->d_t, sizeof(double) * t_ld * D), "cudaMalloc t");
        g->t_cap = t_ld * D;
    }
    if (!g->d_eps) COS_CUDA(cudaMalloc(&g->d_eps, sizeof(double) * g->K), "cudaMalloc eps");
    const int64_t nblk = std::max<int64_t>((S + kReduceBlock - 1) / kReduceBlock, 1);
    if (nblk > g->partial_cap) {
        dfree(g->d_partials);
        const int64_t cap = std::max<int64_t>(nblk, 4096);   // room for 4M samples without regrowth
        // two arrays: partial sums of R, then of A (when the walk also sums |path| values)
        COS_CUDA(cudaMalloc(&g->d_partials, 2 * sizeof(double) * cap), "cudaMalloc partials");
        g->partial_cap = cap;
    }
    // Workspace arena: enough for the FP64 mode over all samples, up to the budget.
    {
        size_t psb = std::max(per_sample_bytes(g, COS_MODE_FP64), per_sample_bytes(g, COS_MODE_FP32_MIXED));
        // (the walks that also sum |path| values need more per sample; their tiles shrink to fit)
        size_t want = psb * (size_t)std::max<int64_t>(round_up(std::max<int64_t>(S, 1), 128), 128) + ((size_t)8 << 20);
        size_t budget = default_budget_bytes();
        size_t minimum = psb * 128 + ((size_t)8 << 20);
        size_t bytes = std::max(std::min(want, budget), minimum);
        if (g->tuning.tile_samples > 0)   // a fixed tile fixes the workspace
            bytes = psb * (size_t)round_up(g->tuning.tile_samples, 128) + ((size_t)8 << 20);
        if (bytes > g->arena_bytes) {
            if (g->d_arena) cudaFree(g->d_arena);
            g->d_arena = nullptr;
            g->arena_bytes = 0;
            COS_CUDA(cudaMalloc(&g->d_arena, bytes), "cudaMalloc workspace");
            g->arena_bytes = bytes;
        }
    }
    COS_CUDA(cudaMemcpyAsync(g->d_eps, eps, sizeof(double) * g->K, cudaMemcpyHostToDevice, st), "copy eps");
    g->t_borrowed = borrow ? t : nullptr;
    if (!borrow) COS_CUDA(cudaMemsetAsync(g->d_t, 0, sizeof(double) * t_ld * D, st), "clear t");
    if (S > 0 && !borrow) {
        const bool host = (t_flags & COS_T_HOST) != 0;
        const bool smaj = (t_flags & COS_T_SAMPLE_MAJOR) != 0;
        if (!smaj) {
            COS_CUDA(cudaMemcpy2DAsync(g->d_t, sizeof(double) * t_ld, t, sizeof(double) * S, sizeof(double) * S, D,
                                       host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st),
                     "copy t");
        } else {
            const double* src = t;
            if (host) {
                if (S * D > g->stage_cap) {
                    dfree(g->d_stage);
                    COS_CUDA(cudaMalloc(&g->d_stage, sizeof(double) * S * D), "cudaMalloc staging");
                    g->stage_cap = S * D;
                }
                COS_CUDA(cudaMemcpyAsync(g->d_stage, t, sizeof(double) * S * D, cudaMemcpyHostToDevice, st), "copy t");
                src = g->d_stage;
            }
            int rc = launch_transpose(src, S, D, g->d_t, t_ld, st);
            if (rc != COS_OK) return fail(rc, "transpose launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        }
    }
    g->S = S;
    g->t_ld = t_ld;
    g->beta = beta;
    g->has_samples = true;
    g->generation++;
    return COS_OK;
}

int cos_set_samples_uniform(cos_graph_t g, int64_t num_samples, uint64_t seed, int64_t first_sample,
                            const double* eps, double beta, void* stream) {
    if (!g) return fail(COS_ERR_INVALID, "graph is NULL");
    if (num_samples < 0 || first_sample < 0) return fail(COS_ERR_INVALID, "num_samples and first_sample must be >= 0");
    // attach as a borrowed empty sample set first (validates eps/beta, sizes the workspace) ...
    DeviceGuard dg(g->device);
    if (!dg.ok) return fail(COS_ERR_CUDA, "cannot select device %d", g->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t t_ld = std::max<int64_t>(round_up(num_samples, 128), 128);
    if (t_ld * g->D > g->t_cap) {
        dfree(g->d_t);
        COS_CUDA(cudaMalloc(&g->d_t, sizeof(double) * t_ld * g->D), "cudaMalloc t");
        g->t_cap = t_ld * g->D;
    }
    int rc = cos_set_samples(g, num_samples, g->d_t, COS_T_BORROW, eps, beta, stream);
    if (rc != COS_OK) return rc;
    // ... then fill the graph's own time buffer with the counter-based draws
    g->t_borrowed = nullptr;
    g->generation++;
    COS_CUDA(cudaMemsetAsync(g->d_t, 0, sizeof(double) * t_ld * g->D, st), "clear t");
    if (num_samples > 0) {
        rc = launch_uniform_times(seed, first_sample, num_samples, g->D, beta, g->d_t, t_ld, st);
        if (rc != COS_OK) return fail(rc, "sampler launch failed");
    }
    return COS_OK;
}

int cos_copy_times(cos_graph_t g, double* dst, void* stream) {
    if (!g || !dst) return fail(COS_ERR_INVALID, "bad arguments");
    if (!g->has_samples) return fail(COS_ERR_STATE, "no samples attached");
    DeviceGuard dg(g->device);
    const double* src = g->t_borrowed ? g->t_borrowed : g->d_t;
    if (g->S > 0)
        COS_CUDA(cudaMemcpy2DAsync(dst, sizeof(double) * g->S, src, sizeof(double) * g->t_ld, sizeof(double) * g->S,
                                   g->D, cudaMemcpyDefault, (cudaStream_t)stream),
                 "copy times");
    return COS_OK;
}

static int collect(cos_graph_t g, double* mean_out, cudaStream_t st) {
    const bool abs2 = mode_has_abs(g->last_mode);   // mean_out holds (mean R, mean A)
    if (g->last_wave && g->wave) {   // windowed schedule: errors are in the batch's control block
        double m[2] = {0.0, 0.0};
        const int rc = cos_batch_results(g->wave, m, st);
        g->last_status_pending = 0;
        if (rc != COS_OK && rc != COS_ERR_OVERFLOW) return rc;
        if (mean_out) {
            mean_out[0] = m[0];
            if (abs2) mean_out[1] = m[1];
        }
        return rc;
    }
    Ctrl c;
    COS_CUDA(cudaMemcpyAsync(&c, g->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st), "read result");
    COS_CUDA(cudaStreamSynchronize(st), "synchronize");
    g->last_status_pending = 0;
    if (c.err == KERR_BARRIER_TIMEOUT) return fail(COS_ERR_TIMEOUT, "grid barrier timed out (phase %d)", c.err_detail);
    if (c.err != 0) return fail(COS_ERR_CUDA, "kernel reported error %d (detail %d)", c.err, c.err_detail);
    if (mean_out) {
        mean_out[0] = c.mean;
        if (abs2) mean_out[1] = c.mean_abs;
    }
    if (g->last_mode == COS_MODE_COUNT_I64 && g->count_overflow)
        return fail(COS_ERR_OVERFLOW, "path count exceeds 2^63-1; results wrap modulo 2^64");
    return COS_OK;
}

int cos_evaluate(cos_graph_t g, int32_t mode, void* per_sample_out, double* mean_out, void* stream) {
    if (!g) return fail(COS_ERR_INVALID, "graph is NULL");
    DeviceGuard dg(g->device);
    if (!dg.ok) return fail(COS_ERR_CUDA, "cannot select device %d", g->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int km = kernel_mode(mode);
    if (km < 0) return fail(COS_ERR_INVALID, "bad mode %d", mode);
    if (mode_has_abs(km) && g->abs_next)
        return fail(COS_ERR_INVALID, "COS_EVAL_ABS and cos_evaluate_abs do not combine");
    WalkParams p;
    cos_tuning tn;
    int rc = cosgpu::prepare_walk(g, km, nullptr, per_sample_out, &p, &tn);
    if (rc != COS_OK) return rc;
    if (const char* env = getenv("COS_TEST_SKIP_BARRIER_PHASE")) p.skip_barrier_phase = atoi(env);
    if (g->d_trace) {
        p.trace = g->d_trace;
        p.trace_cap = g->trace_cap;
        COS_CUDA(cudaMemsetAsync(g->d_trace, 0, sizeof(unsigned long long) * 2 * g->trace_cap, st), "reset trace");
    }
    COS_CUDA(cudaMemsetAsync(g->d_ctrl, 0, sizeof(Ctrl), st), "reset control block");
    if (tn.schedule == 2) {
        rc = launch_windowed(g, &g->wave, km, per_sample_out, tn, st);
        if (rc != COS_OK) return rc;
        g->last_wave = 1;
    } else {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
        const int grid = sms * tn.blocks_per_sm;
        char msg[256] = {0};
        rc = launch_walk(km, tn.samples_per_lane, tn.layout, p, grid, st, msg, sizeof(msg));
        if (rc != COS_OK) return fail(rc, "walker launch failed: %s", msg);
        g->last_wave = 0;
    }
    g->last_mode = km;
    g->last_status_pending = 1;
    if (mean_out) return collect(g, mean_out, st);
    return COS_OK;
}

int cos_set_trace(cos_graph_t g, int32_t capacity) {
    if (!g || capacity < 0 || capacity > (1 << 20)) return fail(COS_ERR_INVALID, "bad arguments");
    DeviceGuard dg(g->device);
    dfree(g->d_trace);
    g->trace_cap = 0;
    if (capacity > 0) {
        COS_CUDA(cudaMalloc(&g->d_trace, sizeof(unsigned long long) * 2 * capacity), "cudaMalloc trace");
        COS_CUDA(cudaMemset(g->d_trace, 0, sizeof(unsigned long long) * 2 * capacity), "clear trace");
        g->trace_cap = capacity;
    }
    return COS_OK;
}

int cos_get_trace(cos_graph_t g, int64_t* out, int32_t capacity, int32_t* count) {
    if (!g || !out || !count || capacity < 0) return fail(COS_ERR_INVALID, "bad arguments");
    *count = 0;
    if (!g->d_trace) return COS_OK;
    DeviceGuard dg(g->device);
    const int32_t n = std::min(capacity, g->trace_cap);
    std::vector<unsigned long long> h((size_t)2 * n);
    COS_CUDA(cudaMemcpy(h.data(), g->d_trace, sizeof(unsigned long long) * 2 * n, cudaMemcpyDeviceToHost), "read trace");
    int32_t c = 0;
    for (int32_t q = 0; q < n; ++q) {
        if (q > 0 && h[2 * q] == 0) break;
        out[2 * q] = (int64_t)h[2 * q];
        out[2 * q + 1] = (int64_t)h[2 * q + 1];
        c = q + 1;
    }
    *count = c;
    return COS_OK;
}

int cos_selftest_exp(cos_graph_t g, int64_t n, const double* x, double* em, double* ep, void* stream) {
    if (!g || n < 0 || (n > 0 && (!x || !em || !ep))) return fail(COS_ERR_INVALID, "bad arguments");
    DeviceGuard dg(g->device);
    if (n == 0) return COS_OK;
    int rc = launch_exp_pair(x, n, g->d_exp_tab, em, ep, (cudaStream_t)stream);
    return rc == COS_OK ? COS_OK : fail(rc, "exp self-test launch failed");
}

int cos_probe_fma_rate(int32_t precision, double* fma_per_second) {
    if ((precision != 0 && precision != 1) || !fma_per_second) return fail(COS_ERR_INVALID, "bad arguments");
    char msg[256] = {0};
    const int rc = probe_fma_rate(precision, fma_per_second, msg, sizeof(msg));
    return rc == COS_OK ? COS_OK : fail(rc, "%s", msg);
}

int cos_set_propagator_table(cos_graph_t g, int32_t T, const double* table, double tau_max) {
    if (!g) return fail(COS_ERR_INVALID, "graph is NULL");
    if (T < 0 || T > (1 << 24)) return fail(COS_ERR_INVALID, "T must be in [0, 2^24]");
    DeviceGuard dg(g->device);
    if (T == 0) {   // back to the free-fermion formula
        dfree(g->d_ptab);
        g->ptab_T = 0;
        g->ptab_tau_max = 0.0;
        g->generation++;
        return COS_OK;
    }
    if (!table) return fail(COS_ERR_INVALID, "table is NULL");
    if (!(tau_max > 0.0) || !std::isfinite(tau_max)) return fail(COS_ERR_INVALID, "tau_max must be finite and > 0");
    const size_t n = 2 * (size_t)(T + 1) * (size_t)g->K;
    for (size_t q = 0; q < n; ++q)
        if (!std::isfinite(table[q])) return fail(COS_ERR_INVALID, "table entry %zu is not finite", q);
    // device form: per kind and half, T intervals as (value at the left node, slope)
    std::vector<double> pairs(2 * 2 * (size_t)T * (size_t)g->K);
    for (size_t h = 0; h < 2 * (size_t)g->K; ++h)
        for (int32_t m = 0; m < T; ++m) {
            const double a = table[h * (T + 1) + m], b = table[h * (T + 1) + m + 1];
            pairs[2 * (h * T + m)] = a;
            pairs[2 * (h * T + m) + 1] = b - a;
        }
    double* d = nullptr;
    COS_CUDA(cudaMalloc(&d, sizeof(double) * pairs.size()), "cudaMalloc propagator table");
    cudaError_t e = cudaMemcpy(d, pairs.data(), sizeof(double) * pairs.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "copy propagator table");
    }
    dfree(g->d_ptab);
    g->d_ptab = d;
    g->ptab_T = T;
    g->ptab_tau_max = tau_max;
    g->generation++;
    return COS_OK;
}

int cos_evaluate_abs(cos_graph_t g, int32_t mode, void* per_sample_out, double* mean_out, void* stream) {
    if (!g) return fail(COS_ERR_INVALID, "graph is NULL");
    if (mode != COS_MODE_FP64 && mode != COS_MODE_FP32_MIXED)
        return fail(COS_ERR_INVALID, "the sum of |path| values needs a floating-point mode (0 or 1)");
    g->abs_next = 1;
    const int rc = cos_evaluate(g, mode, per_sample_out, mean_out, stream);
    g->abs_next = 0;
    return rc;
}

int cos_get_result(cos_graph_t g, double* mean_out, void* stream) {
    if (!g) return fail(COS_ERR_INVALID, "graph is NULL");
    DeviceGuard dg(g->device);
    return collect(g, mean_out, (cudaStream_t)stream);
}

}  // extern "C"

namespace cosgpu {

int graph_view(cos_graph_t g, GraphView* out) {
    if (!g || !out) return fail(COS_ERR_INVALID, "graph is NULL");
    out->levels = g->d_levels;
    out->row_ptr = g->d_row_ptr;
    out->edges = g->d_edges;
    out->slot_kij = g->d_slot_kij;
    out->kind_slot = g->d_kind_slot;
    out->exp_tab = g->d_exp_tab;
    out->L = g->L;
    out->P = (int32_t)g->P;
    out->K = g->K;
    out->D = g->D;
    out->Wmax = g->Wmax;
    out->device = g->device;
    out->count_overflow = g->count_overflow ? 1 : 0;
    out->widths_host = g->widths.data();
    out->S = g->has_samples ? g->S : -1;
    out->ptab = g->d_ptab;
    out->ptab_T = g->ptab_T;
    out->ptab_tau_max = g->ptab_tau_max;
    out->t = g->t_borrowed ? const_cast<double*>(g->t_borrowed) : g->d_t;
    out->t_ld = g->t_ld;
    out->beta = g->beta;
    out->generation = g->generation;
    out->timeout_ms = g->tuning.timeout_ms;
    if (out->timeout_ms <= 0) {
        const char* env = getenv("COS_TIMEOUT_MS");
        out->timeout_ms = (env && atoi(env) > 0) ? atoi(env) : 10000;
    }
    return COS_OK;
}

int prepare_walk(cos_graph_t g, int mode, const cos_tuning* force, void* per_sample_out, WalkParams* out,
                 cos_tuning* tn_out) {
    if (!g) return fail(COS_ERR_INVALID, "graph is NULL");
    if (mode < 0 || mode > kModeMixedAbs) return fail(COS_ERR_INVALID, "bad mode %d", mode);
    const bool abs2 = mode_has_abs(mode);
    if (!g->has_samples) return fail(COS_ERR_STATE, "cos_set_samples has not been called");
    if (mode_has_abs(mode) && g->tuning.tile_samples <= 0 && (!force || force->tile_samples <= 0)) {
        // the workspace was sized for the walks without A; grow it once (allocating path
        // only) so that the walk with A keeps their tile of samples
        const size_t want = std::min(per_sample_bytes(g, mode) * (size_t)std::max<int64_t>(round_up(std::max<int64_t>(g->S, 1), 128), 128) +
                                         ((size_t)8 << 20),
                                     std::max(default_budget_bytes(), g->arena_bytes));
        if (want > g->arena_bytes) {
            void* bigger = nullptr;
            if (cudaMalloc(&bigger, want) == cudaSuccess) {   // else keep the smaller workspace (smaller tiles)
                cudaFree(g->d_arena);
                g->d_arena = bigger;
                g->arena_bytes = want;
                g->generation++;
            } else {
                cudaGetLastError();
            }
        }
    }
    const cos_tuning saved = g->tuning;
    if (force) {
        if (force->samples_per_lane > 0) g->tuning.samples_per_lane = force->samples_per_lane;
        if (force->rows_per_warp > 0) g->tuning.rows_per_warp = force->rows_per_warp;
        if (force->tile_samples > 0) g->tuning.tile_samples = force->tile_samples;
        if (force->blocks_per_sm > 0) g->tuning.blocks_per_sm = force->blocks_per_sm;
        if (force->timeout_ms > 0) g->tuning.timeout_ms = force->timeout_ms;
        if (force->layout > 0) g->tuning.layout = force->layout;
        if (force->prefetch > 0) g->tuning.prefetch = force->prefetch;
    }
    cos_tuning tn;
    int64_t tile;
    int rc = resolve_tuning(g, mode, &tn, &tile);
    g->tuning = saved;
    if (rc != COS_OK) return rc;
    WalkParams& p = *out;
    memset(&p, 0, sizeof(p));
    if (!carve(g, mode, tile, p)) return fail(COS_ERR_STATE, "workspace too small for a tile of %lld samples", (long long)tile);
    p.levels = g->d_levels;
    p.row_ptr = g->d_row_ptr;
    p.edges = g->d_edges;
    p.slot_kij = g->d_slot_kij;
    p.kind_slot = g->d_kind_slot;
    p.exp_tab = g->d_exp_tab;
    p.L = g->L;
    p.P = (int32_t)g->P;
    p.K = g->K;
    p.D = g->D;
    p.t = g->t_borrowed ? g->t_borrowed : g->d_t;
    p.eps = g->d_eps;
    p.beta = g->beta;
    p.S = g->S;
    p.t_ld = g->t_ld;
    const int64_t nout = std::max<int64_t>(g->S, 1) * (abs2 ? 2 : 1);   // R, then A
    if (!per_sample_out && nout > g->R_cap) {
        // no caller buffer: the per-sample values go to an internal buffer (allocated on first need)
        if (g->d_R) cudaFree(g->d_R);
        g->d_R = nullptr;
        g->R_cap = 0;
        COS_CUDA(cudaMalloc(&g->d_R, sizeof(double) * nout), "cudaMalloc R");
        g->R_cap = nout;
        g->generation++;
    }
    p.R = per_sample_out ? per_sample_out : g->d_R;
    p.partials = g->d_partials;
    p.Rabs = abs2 ? static_cast<double*>(p.R) + g->S : nullptr;
    p.partials_abs = abs2 ? g->d_partials + g->partial_cap : nullptr;
    p.ctrl = g->d_ctrl;
    p.tile = tile;
    p.rows_per_warp = tn.rows_per_warp;
    p.wmax = (int32_t)g->Wmax;
    p.pf_slice_bytes = tn.prefetch == 1 ? INT64_MAX
                       : (tn.prefetch == 3 || tn.prefetch == 5 || tn.prefetch == 7) ? 0 : ((int64_t)32 << 20);
    p.pf_bulk = (tn.prefetch == 4 || tn.prefetch == 5) ? 1 : 0;
    p.pf_ahead = tn.prefetch >= 6 ? 2 : 1;
    p.ptab = g->d_ptab;
    p.ptab_T = g->ptab_T;
    p.ptab_tau_max = g->ptab_tau_max;
    p.ptab_inv_h = g->d_ptab ? (double)g->ptab_T / g->ptab_tau_max : 0.0;
    p.abs_weights = g->abs_next;
    p.timeout_ns = (long long)tn.timeout_ms * 1000000LL;
    if (tn_out) *tn_out = tn;
    return COS_OK;
}

int attach_own_samples(cos_graph_t g, int64_t num_samples, SampleState* undo) {
    if (!g) return fail(COS_ERR_INVALID, "graph is NULL");
    if (!g->has_samples) return fail(COS_ERR_STATE, "attach samples once (cos_set_samples*) to set eps, beta and buffers");
    if (num_samples < 0) return fail(COS_ERR_INVALID, "num_samples must be >= 0");
    const int64_t t_ld = std::max<int64_t>(round_up(num_samples, 128), 128);
    if (!g->d_t || t_ld * g->D > g->t_cap)
        return fail(COS_ERR_STATE, "the handle's time buffer holds %lld samples; attach a sample set of %lld once first",
                    (long long)(g->D > 0 ? g->t_cap / g->D : 0), (long long)num_samples);
    if (std::max<int64_t>((num_samples + kReduceBlock - 1) / kReduceBlock, 1) > g->partial_cap)
        return fail(COS_ERR_STATE, "partial-sum buffer too small for %lld samples", (long long)num_samples);
    if (undo) {
        undo->S = g->S;
        undo->t_ld = g->t_ld;
        undo->t_borrowed = g->t_borrowed;
    }
    g->S = num_samples;
    g->t_ld = t_ld;
    g->t_borrowed = nullptr;
    g->generation++;
    return COS_OK;
}

void restore_samples(cos_graph_t g, const SampleState& s) {
    g->S = s.S;
    g->t_ld = s.t_ld;
    g->t_borrowed = s.t_borrowed;
    g->generation++;
}

int set_error(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

}  // namespace cosgpu
