// C ABI of libdm: contexts, plans, argument checks, scratch management and
// the launch sequences of each call.  Host code only; kernels live in the
// other translation units.
#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "dm_internal.h"

struct dm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    uint32_t* err = nullptr;         // device error word
    uint32_t* host_err = nullptr;    // pinned copy target
    void* arena = nullptr;           // scratch, grown on demand
    size_t arena_bytes = 0;
    uint32_t* host_hist = nullptr;   // pinned, histogram read-back in dm_prepare
    size_t host_hist_words = 0;
    int64_t launches = 0;
    int deterministic = 0;           // dm_set_deterministic
    uint32_t spin_limit = dm::kSpinLimit; // dm_set_wait_limit
    int engine = DM_ENGINE_AUTO;     // dm_set_engine
    // Device buffers of dm_matmat_host (grown on demand), and the stream and
    // event its copy of Z uses to overlap the preprocessing.
    void* hx = nullptr; size_t hx_bytes = 0;
    cudaStream_t aux = nullptr;
    cudaEvent_t aux_done = nullptr;
    void* hz = nullptr; size_t hz_bytes = 0;
    void* ho = nullptr; size_t ho_bytes = 0;
    // dm_matmat_host_multi: the event after the copy of X, and one context
    // (own stream, arena and error word) per product after the first, so
    // that the products of one call run side by side.
    cudaEvent_t x_done = nullptr;
    std::vector<dm_ctx*> peers;
    std::vector<cudaStream_t> peer_streams;
    // Kernel timing (dm_profile_enable / dm_profile_read).
    struct Pending { std::string name; cudaEvent_t start, stop; int64_t launches; };
    struct Stat { int64_t launches = 0; double ms = 0; };
    bool profiling = false;
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
    std::map<std::string, Stat> stats;
    // Device buffers of destroyed plans, reused by later plans.  All use is
    // ordered on the context's stream, so a buffer handed back by
    // dm_plan_destroy can be reused by the next call without a sync.
    struct Block { void* p; size_t bytes; };
    std::vector<Block> pool;
    size_t pool_bytes = 0;
    // Lifetime: live plans and batches made from this context.  dm_destroy
    // with children still alive only marks the context destroyed (every later
    // call through it or its children fails with DM_ERR_INVALID_ARG); the
    // memory is released when the last child is destroyed.
    int64_t children = 0;
    bool destroyed = false;
};

struct dm_plan {
    dm_ctx* ctx = nullptr;
    std::vector<std::pair<void*, size_t>> owned;   // buffers from the context pool
    dm_metric metric = DM_L1;
    dm_dtype dtype = DM_F32;
    int64_t n = 0, d = 0;
    // l1
    void* xs = nullptr;
    int32_t* perm = nullptr;
    void* R = nullptr;            // R_i = sum_c (x_i(c) - mu_c), mu_c = column median
    // squared l2 and ||.||_p^p
    const void* X = nullptr;
    int64_t ldx = 0;
    void* mu = nullptr;
    int p = 0;                    // DM_LPP: the power (even: moments plan, odd: sorted plan)
    int64_t d_in = 0;             // DM_L2_EMBED: dimension of the input points (d is m)
};

struct dm_batch {
    dm_ctx* ctx = nullptr;
    dm_metric metric = DM_L1;
    dm_dtype dtype = DM_F32;
    struct Set {
        dm_plan* plan;
        const void* X; int64_t ldx;
        const void* Z; int64_t k, ldz;
        void* out; int64_t ldo;
        double cost;        // estimated bytes moved (scheduling weight)
        int lane;
    };
    std::vector<Set> sets;
    int lanes = 0;
    cudaStream_t origin = nullptr;          // capture / launch stream
    std::vector<cudaStream_t> streams;      // one per lane
    std::vector<void*> scratch;             // one per lane
    std::vector<size_t> scratch_bytes;
    cudaEvent_t fork = nullptr, done = nullptr;
    std::vector<cudaEvent_t> joins;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t launches_per_run = 0;
};

namespace {

using namespace dm;

constexpr int64_t kMaxN = (int64_t(1) << 30) - 1;
constexpr int kMaxHostProducts = 8;       // products of one dm_matmat_host_multi call

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

dm_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return DM_OK;
    if (e == cudaErrorMemoryAllocation) return DM_ERR_OOM;
    return DM_ERR_CUDA;
}

#define DM_TRY_CUDA(expr)                              \
    do {                                               \
        cudaError_t _e = (expr);                       \
        if (_e != cudaSuccess) return from_cuda(_e);   \
    } while (0)

#define DM_TRY(expr)                                   \
    do {                                               \
        dm_status _s = (expr);                         \
        if (_s != DM_OK) return _s;                    \
    } while (0)

bool valid_dtype(dm_dtype t) { return t == DM_F32 || t == DM_F64 || t == DM_I32; }
bool valid_metric(dm_metric m) { return m == DM_L1 || m == DM_L2SQ; }
// Metrics whose plan is the sorted coordinates of Algorithm 1.
bool sorted_metric(dm_metric m) { return m == DM_L1 || m == DM_TV || m == DM_L2_EMBED; }

size_t acc_size(dm_dtype t) { return t == DM_F32 ? 4 : 8; }

cudaEvent_t pool_event(dm_ctx* ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    return e;
}

// Where a launch sequence runs: the context (error word, launch count,
// timing), a stream, a scratch buffer of known size, and whether the work is
// being captured into a CUDA graph (then nothing may synchronize, allocate or
// record timing events).
struct Exec {
    dm_ctx* ctx;
    cudaStream_t stream;
    unsigned char* scratch;
    size_t scratch_bytes;
    bool graph;
};

// Brackets one group of launches with events when timing is enabled.
struct ProfScope {
    dm_ctx* ctx;
    const char* name;
    cudaStream_t stream;
    cudaEvent_t start = nullptr;
    int64_t before = 0;
    bool on;
    ProfScope(dm_ctx* c, const char* n) : ProfScope(c, n, c->stream, false) {}
    ProfScope(const Exec& e, const char* n) : ProfScope(e.ctx, n, e.stream, e.graph) {}
    ProfScope(dm_ctx* c, const char* n, cudaStream_t st, bool graph)
        : ctx(c), name(n), stream(st), on(c->profiling && !graph) {
        if (!on) return;
        start = pool_event(ctx);
        before = ctx->launches;
        if (start) cudaEventRecord(start, stream);
    }
    ~ProfScope() {
        if (!on || !start) return;
        cudaEvent_t stop = pool_event(ctx);
        if (!stop) { ctx->event_pool.push_back(start); return; }
        cudaEventRecord(stop, stream);
        ctx->pending.push_back({name, start, stop, ctx->launches - before});
    }
};

dm_status resolve_profile(dm_ctx* ctx) {
    if (ctx->pending.empty()) return DM_OK;
    DM_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    for (auto& p : ctx->pending) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, p.start, p.stop) == cudaSuccess) {
            auto& st = ctx->stats[p.name];
            st.launches += p.launches;
            st.ms += ms;
        } else {
            cudaGetLastError();
        }
        ctx->event_pool.push_back(p.start);
        ctx->event_pool.push_back(p.stop);
    }
    ctx->pending.clear();
    return DM_OK;
}
size_t up16(size_t x) { return (x + 15) & ~size_t(15); }

dm_status ensure_arena(dm_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->arena_bytes) return DM_OK;
    // Work queued on the stream may still use the old arena.
    DM_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    if (ctx->arena) cudaFree(ctx->arena);
    ctx->arena = nullptr;
    ctx->arena_bytes = 0;
    const size_t want = up16(bytes + bytes / 8);
    cudaError_t e = cudaMalloc(&ctx->arena, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->arena = nullptr;
        return DM_ERR_OOM;
    }
    ctx->arena_bytes = want;
    return DM_OK;
}

dm_status ensure_buffer(dm_ctx* ctx, void** buf, size_t* have, size_t bytes) {
    if (bytes <= *have) return DM_OK;
    DM_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    cudaError_t e = cudaMalloc(buf, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        return DM_ERR_OOM;
    }
    *have = bytes;
    return DM_OK;
}

constexpr size_t kPoolCap = size_t(8) << 30;   // cached plan buffers per context

// A device buffer of at least `bytes` for plan p: a pooled block of the same
// rounded size when one is free, else a new allocation.
dm_status plan_alloc(dm_plan* p, size_t bytes, void** out) {
    dm_ctx* ctx = p->ctx;
    bytes = (bytes + 255) & ~size_t(255);
    for (size_t i = 0; i < ctx->pool.size(); ++i) {
        if (ctx->pool[i].bytes == bytes) {
            *out = ctx->pool[i].p;
            ctx->pool_bytes -= bytes;
            ctx->pool.erase(ctx->pool.begin() + (long)i);
            p->owned.push_back({*out, bytes});
            return DM_OK;
        }
    }
    cudaError_t e = cudaMalloc(out, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        // drop the cache and retry once
        cudaStreamSynchronize(ctx->stream);
        for (auto& b : ctx->pool) cudaFree(b.p);
        ctx->pool.clear();
        ctx->pool_bytes = 0;
        e = cudaMalloc(out, bytes);
        if (e != cudaSuccess) { cudaGetLastError(); *out = nullptr; return DM_ERR_OOM; }
    }
    p->owned.push_back({*out, bytes});
    return DM_OK;
}

// Hand a plan's buffers back to the context pool (freed beyond the cap, and
// always once the context is destroyed: cudaFree waits for the device).
void plan_release(dm_plan* p) {
    dm_ctx* ctx = p->ctx;
    for (auto& ob : p->owned) {
        if (ctx->destroyed) {
            cudaFree(ob.first);
        } else if (ctx->pool_bytes + ob.second <= kPoolCap) {
            ctx->pool.push_back({ob.first, ob.second});
            ctx->pool_bytes += ob.second;
        } else {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(ob.first);
        }
    }
    p->owned.clear();
}

// Read (and clear) the device error word; the stream must be idle.
dm_status take_device_error(dm_ctx* ctx) {
    DM_TRY_CUDA(cudaMemcpyAsync(ctx->host_err, ctx->err, 4, cudaMemcpyDeviceToHost, ctx->stream));
    DM_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    const uint32_t v = *ctx->host_err;
    if (v != 0) {
        DM_TRY_CUDA(cudaMemsetAsync(ctx->err, 0, 4, ctx->stream));
        return static_cast<dm_status>(v);
    }
    return DM_OK;
}

// ------------------------------------------------------------- l1 prepare
// Scratch of the sort: [hist | counters | lookback] (zeroed), then the key
// and payload ping-pong buffers.
struct SortLayout {
    size_t hist, cnt, lb, zero_bytes, ka, kb, va, vb, total;
};

SortLayout sort_layout(dm_dtype t, int64_t n, int64_t d) {
    const size_t nd = (size_t)n * (size_t)d;
    const size_t key_bytes = key_bits(t) / 8;
    SortLayout L;
    L.hist = 0;
    L.cnt = up16(L.hist + sort_hist_words(t, d) * 4);
    L.lb = up16(L.cnt + 4 * (size_t)sort_passes(t));
    L.zero_bytes = up16(L.lb + sort_lookback_words(t, n, d) * 4);
    L.ka = L.zero_bytes;
    L.kb = up16(L.ka + nd * key_bytes);
    L.va = up16(L.kb + nd * key_bytes);
    L.vb = up16(L.va + nd * 4);
    L.total = up16(L.vb + nd * 4);
    return L;
}

dm_status alloc_l1_plan(dm_plan* p) {
    const size_t nd = (size_t)p->n * (size_t)p->d;
    DM_TRY(plan_alloc(p, nd * dtype_size(p->dtype), &p->xs));
    DM_TRY(plan_alloc(p, nd * 4, reinterpret_cast<void**>(&p->perm)));
    DM_TRY(plan_alloc(p, (size_t)p->n * acc_size(p->dtype), &p->R));
    return DM_OK;
}

// The sort of every column (Algorithm 1) and the row sums R.  Outside a
// graph, the digit histograms are read back to skip digit positions that
// are constant in every column (a stable pass over a constant digit is the
// identity) and non-finite input is reported at once; in a graph every pass
// runs and non-finite input is left in the error word for dm_sync.
dm_status prepare_l1_run(const Exec& e, dm_plan* p, const void* X, int64_t ldx) {
    dm_ctx* ctx = e.ctx;
    const dm_dtype t = p->dtype;
    const int64_t n = p->n, d = p->d;
    const int P = sort_passes(t);
    const size_t hist_words = sort_hist_words(t, d);
    const SortLayout L = sort_layout(t, n, d);
    if (e.scratch_bytes < L.total) return DM_ERR_INTERNAL;
    unsigned char* base = e.scratch;

    SortArgs a{};
    a.dtype = t;
    a.X = X; a.n = n; a.d = d; a.ldx = ldx;
    a.keys_a = base + L.ka; a.keys_b = base + L.kb;
    a.vals_a = reinterpret_cast<int32_t*>(base + L.va);
    a.vals_b = reinterpret_cast<int32_t*>(base + L.vb);
    a.hist = reinterpret_cast<uint32_t*>(base + L.hist);
    a.counters = reinterpret_cast<uint32_t*>(base + L.cnt);
    a.lookback = reinterpret_cast<uint32_t*>(base + L.lb);
    a.sorted_out = p->xs;
    a.perm_out = p->perm;
    a.err = ctx->err;
    a.spin_limit = ctx->spin_limit;

    DM_TRY_CUDA(cudaMemsetAsync(base, 0, L.zero_bytes, e.stream));
    {
        ProfScope ps(e, "sort_keygen_hist");
        DM_TRY_CUDA(sort_launch_keygen(a, e.stream, &ctx->launches));
    }
    std::vector<int> passes;
    if (e.graph) {
        for (int q = 0; q < P; ++q) passes.push_back(q);
    } else {
        if (ctx->host_hist_words < hist_words) {
            if (ctx->host_hist) cudaFreeHost(ctx->host_hist);
            ctx->host_hist = nullptr;
            ctx->host_hist_words = 0;
            DM_TRY_CUDA(cudaMallocHost(reinterpret_cast<void**>(&ctx->host_hist), hist_words * 4));
            ctx->host_hist_words = hist_words;
        }
        DM_TRY_CUDA(cudaMemcpyAsync(ctx->host_hist, a.hist, hist_words * 4, cudaMemcpyDeviceToHost,
                                    e.stream));
        DM_TRY(take_device_error(ctx));   // synchronizes
        for (int q = 0; q < P; ++q) {
            bool needed = false;
            for (int64_t c = 0; c < d && !needed; ++c) {
                const uint32_t* h = ctx->host_hist + ((size_t)c * P + q) * 256;
                bool constant = false;
                for (int b = 0; b < 256; ++b)
                    if ((int64_t)h[b] == n) { constant = true; break; }
                needed = !constant;
            }
            if (needed) passes.push_back(q);
        }
        if (passes.empty()) passes.push_back(0);   // still writes values + permutation
    }
    {
        ProfScope ps(e, "sort_onesweep");
        DM_TRY_CUDA(sort_launch_passes(a, passes.data(), (int)passes.size(), e.stream,
                                       &ctx->launches));
    }
    // R_i for the part of the query that is linear in the point (shift: the
    // median of each column, xs[c * n + n / 2]).
    {
        ProfScope ps(e, "l1_rowsum");
        DM_TRY_CUDA(rowsum_launch(t, X, n, d, ldx,
                                  static_cast<unsigned char*>(p->xs) + (size_t)(n / 2) * dtype_size(t),
                                  n, p->R, e.stream, &ctx->launches));
    }
    return DM_OK;
}

Exec ctx_exec(dm_ctx* ctx) {
    return Exec{ctx, ctx->stream, static_cast<unsigned char*>(ctx->arena), ctx->arena_bytes, false};
}

dm_status prepare_l1(dm_ctx* ctx, dm_plan* p, const void* X, int64_t ldx) {
    DM_TRY(alloc_l1_plan(p));
    DM_TRY(ensure_arena(ctx, sort_layout(p->dtype, p->n, p->d).total));
    return prepare_l1_run(ctx_exec(ctx), p, X, ldx);
}

// ------------------------------------------------------------- l2 prepare
size_t prepare_l2_scratch(dm_plan* p) {
    L2PrepArgs a{};
    a.n = p->n; a.d = p->d;
    return (size_t)l2prep_blocks(a) * p->d * 8 + 16;
}

dm_status prepare_l2_run(const Exec& e, dm_plan* p, const void* X, int64_t ldx) {
    dm_ctx* ctx = e.ctx;
    p->X = X;
    p->ldx = ldx;
    L2PrepArgs a{};
    a.dtype = p->dtype;
    a.X = X; a.n = p->n; a.d = p->d; a.ldx = ldx;
    a.mu = p->mu; a.err = ctx->err;
    if (e.scratch_bytes < prepare_l2_scratch(p)) return DM_ERR_INTERNAL;
    a.partial = e.scratch;
    ProfScope ps(e, "l2_prepare");
    DM_TRY_CUDA(l2prep_launch(a, e.stream, &ctx->launches));
    return DM_OK;
}

dm_status prepare_l2(dm_ctx* ctx, dm_plan* p, const void* X, int64_t ldx) {
    DM_TRY(plan_alloc(p, (size_t)p->d * dtype_size(p->dtype), &p->mu));
    DM_TRY(ensure_arena(ctx, prepare_l2_scratch(p)));
    return prepare_l2_run(ctx_exec(ctx), p, X, ldx);
}

void free_plan_buffers(dm_plan* p) {
    plan_release(p);
    p->xs = nullptr; p->perm = nullptr; p->R = nullptr; p->mu = nullptr;
}

// ------------------------------------------------------------------ query
// Query columns per reduce + apply round of the squared-l2 product (the
// shared memory of the reduce bounds it; wider blocks run in column chunks).
int64_t l2_chunk(const dm_plan* p, int64_t k) {
    return std::min<int64_t>(k, reduce_max_k(p->dtype, p->d));
}

// ||x - y||_p^p with odd p runs on the sorted coordinates of an l1 plan.
bool lpp_odd(const dm_plan* p) { return p->metric == DM_LPP && (p->p & 1); }

size_t matmat_scratch(const dm_plan* p, int64_t k) {
    if (lpp_odd(p)) return oddp_scratch_bytes(p->n, p->d, k, p->p);
    if (sorted_metric(p->metric)) return l1_query_scratch_bytes(p->dtype, p->n, p->d, k, p->ctx->num_sms);
    size_t feat = 0;
    int64_t D = p->d;
    if (p->metric == DM_LPP) {
        feat = up16(lpp_feature_bytes(p->dtype, p->n, p->d, p->p));
        D = p->d * p->p;
        k = std::max<int64_t>(1, std::min<int64_t>(k, reduce_max_k(p->dtype, D)));
    } else {
        k = std::max<int64_t>(1, l2_chunk(p, k));
    }
    ReduceArgs r{};
    r.dtype = p->dtype;
    r.n = p->n; r.d = D; r.k = k;
    r.num_sms = p->ctx->num_sms;
    r.engine = p->ctx->engine;
    const size_t o_res = up16((size_t)reduce_blocks(r) * (D + 2) * k * 8);
    return feat + up16(o_res + (size_t)(D + 2) * k * 8);
}

// ||x - y||_p^p for even p: powers of the centred coordinates, their moments
// against Z (the reduce kernel, in column chunks), then the binomial sum.
dm_status lpp_run(const Exec& e, dm_plan* p, const void* Z, int64_t k, int64_t ldz, void* out,
                  int64_t ldo) {
    dm_ctx* ctx = e.ctx;
    const dm_dtype t = p->dtype;
    const int64_t n = p->n, d = p->d, D = d * p->p;
    const int64_t kc = std::min<int64_t>(k, reduce_max_k(t, D));
    if (kc < 1) return DM_ERR_UNSUPPORTED;
    unsigned char* F = e.scratch;
    unsigned char* base = e.scratch + up16(lpp_feature_bytes(t, n, d, p->p));
    {
        ProfScope ps(e, "lpp_features");
        DM_TRY_CUDA(lpp_features_launch(t, p->X, n, d, p->ldx, p->mu, p->p, F, ctx->num_sms, e.stream,
                                        &ctx->launches));
    }
    for (int64_t j0 = 0; j0 < k; j0 += kc) {
        const int64_t kk = std::min<int64_t>(kc, k - j0);
        ReduceArgs r{};
        r.dtype = t;
        r.n = n; r.d = D;
        r.X = F; r.ldx = D; r.x_acc = true;
        r.mu = nullptr; r.mu_stride = 1; r.with_s = false;
        r.Z = static_cast<const unsigned char*>(Z) + (size_t)j0 * dtype_size(t);
        r.k = kk; r.ldz = ldz;
        r.num_sms = ctx->num_sms;
        r.err = ctx->err;
        r.engine = ctx->engine;
        r.spin_limit = ctx->spin_limit;
        const size_t o_res = up16((size_t)reduce_blocks(r) * (D + 2) * kk * 8);
        r.partial = base;
        r.res = base + o_res;
        {
            ProfScope ps(e, "lpp_reduce");
            DM_TRY_CUDA(reduce_launch(r, e.stream, &ctx->launches));
        }
        ProfScope ps(e, "lpp_apply");
        DM_TRY_CUDA(lpp_apply_launch(t, p->X, n, d, p->ldx, p->mu, r.res, p->p, kk,
                                     static_cast<unsigned char*>(out) + (size_t)j0 * out_size(t), ldo,
                                     ctx->num_sms, e.stream, &ctx->launches));
    }
    return DM_OK;
}

// ||x - y||_p^p for odd p (Theorem "odd_p"): out is zeroed, then the tile
// sums of the p + 1 weights per column, the scan over tiles and the
// evaluation, which adds every coordinate's share into out.
dm_status lpp_odd_run(const Exec& e, dm_plan* p, const void* Z, int64_t k, int64_t ldz, void* out,
                      int64_t ldo) {
    dm_ctx* ctx = e.ctx;
    const size_t es = out_size(p->dtype);
    DM_TRY_CUDA(ldo == k ? cudaMemsetAsync(out, 0, (size_t)p->n * k * es, e.stream)
                         : cudaMemset2DAsync(out, (size_t)ldo * es, 0, (size_t)k * es, (size_t)p->n, e.stream));
    OddArgs a{};
    a.dtype = p->dtype;
    a.n = p->n; a.d = p->d;
    a.xs = p->xs; a.perm = p->perm;
    a.Z = Z; a.ldz = ldz; a.k = k;
    a.p = p->p;
    a.out = out; a.ldo = ldo;
    a.scratch = e.scratch;
    static const char* const names[3] = {"lpp_odd_tiles", "lpp_odd_scan", "lpp_odd_eval"};
    for (int stage = 0; stage < 3; ++stage) {
        ProfScope ps(e, names[stage]);
        DM_TRY_CUDA(oddp_launch(a, stage, e.stream, &ctx->launches));
    }
    return DM_OK;
}

dm_status matmat_run(const Exec& e, dm_plan* p, const void* Z, int64_t k, int64_t ldz, void* out,
                     int64_t ldo) {
    dm_ctx* ctx = e.ctx;
    const dm_dtype t = p->dtype;
    const int64_t n = p->n, d = p->d;
    if (e.scratch_bytes < matmat_scratch(p, k)) return DM_ERR_INTERNAL;

    if (lpp_odd(p)) return lpp_odd_run(e, p, Z, k, ldz, out, ldo);
    if (p->metric == DM_LPP) return lpp_run(e, p, Z, k, ldz, out, ldo);
    if (sorted_metric(p->metric)) {
        // R^T Z, 1^T Z and the group-major copy of Z, then the sorted part
        // (Algorithm 2).
        L1QueryArgs q{};
        q.dtype = t;
        q.xs = p->xs; q.perm = p->perm; q.n = n; q.d = d;
        q.R = p->R;
        q.mu = static_cast<unsigned char*>(p->xs) + (size_t)(n / 2) * dtype_size(t);
        q.mu_stride = n;
        q.Z = Z; q.k = k; q.ldz = ldz;
        q.out = out; q.ldo = ldo;
        q.scratch = e.scratch;
        q.err = ctx->err;
        q.num_sms = ctx->num_sms;
        q.deterministic = ctx->deterministic;
        q.spin_limit = ctx->spin_limit;
        {
            ProfScope ps(e, "l1_prologue");
            DM_TRY_CUDA(l1_prologue_launch(q, e.stream, &ctx->launches));
        }
        {
            ProfScope ps(e, "l1_aggregate");
            DM_TRY_CUDA(l1_aggregate_launch(q, e.stream, &ctx->launches));
        }
        {
            ProfScope ps(e, "l1_query");
            DM_TRY_CUDA(l1_query_launch(q, e.stream, &ctx->launches));
        }
        if (!q.deterministic) {
            ProfScope ps(e, "l1_finalize");
            DM_TRY_CUDA(l1_finalize_launch(q, e.stream, &ctx->launches));
        }
        if (p->metric == DM_TV) {   // TV(x, y) = ||x - y||_1 / 2
            ProfScope ps(e, "tv_scale");
            DM_TRY_CUDA(scale_launch(t, out, n, k, ldo, 0.5, ctx->num_sms, e.stream, &ctx->launches));
        }
        return DM_OK;
    }

    const int64_t kc = l2_chunk(p, k);
    if (kc < 1) return DM_ERR_UNSUPPORTED;
    for (int64_t j0 = 0; j0 < k; j0 += kc) {
        const int64_t kk = std::min<int64_t>(kc, k - j0);
        ReduceArgs r{};
        r.dtype = t;
        r.n = n; r.d = d;
        r.Z = static_cast<const unsigned char*>(Z) + (size_t)j0 * dtype_size(t);
        r.k = kk; r.ldz = ldz;
        r.num_sms = ctx->num_sms;
        r.err = ctx->err;
        r.engine = ctx->engine;
        r.spin_limit = ctx->spin_limit;
        const int blocks = reduce_blocks(r);
        const size_t o_res = up16((size_t)blocks * (d + 2) * kk * 8);
        unsigned char* base = e.scratch;
        r.partial = base;
        r.res = base + o_res;
        r.X = p->X; r.ldx = p->ldx; r.x_acc = false;
        r.mu = p->mu; r.mu_stride = 1;
        r.with_s = true;
        {
            ProfScope ps(e, "l2_reduce");
            DM_TRY_CUDA(reduce_launch(r, e.stream, &ctx->launches));
        }
        L2ApplyArgs ap{};
        ap.dtype = t;
        ap.X = p->X; ap.n = n; ap.d = d; ap.ldx = p->ldx;
        ap.mu = p->mu; ap.res = r.res; ap.k = kk;
        ap.out = static_cast<unsigned char*>(out) + (size_t)j0 * out_size(t);
        ap.ldo = ldo;
        ap.num_sms = ctx->num_sms;
        ap.engine = ctx->engine;
        ap.err = ctx->err;
        ap.spin_limit = ctx->spin_limit;
        ProfScope ps(e, "l2_apply");
        DM_TRY_CUDA(l2apply_launch(ap, e.stream, &ctx->launches));
    }
    return DM_OK;
}

dm_status matmat_impl(dm_plan* p, const void* Z, int64_t k, int64_t ldz, void* out, int64_t ldo) {
    if (p->metric == DM_L2SQ && l2_chunk(p, k) < 1) return DM_ERR_UNSUPPORTED;
    const bool even = p->metric == DM_LPP && !lpp_odd(p);
    if (even && reduce_max_k(p->dtype, p->d * p->p) < 1) return DM_ERR_UNSUPPORTED;
    if (lpp_odd(p) && (p->d * (p->p + 1) * k > INT_MAX ||
                       p->d * ((p->n + 1023) / 1024) > INT_MAX))
        return DM_ERR_UNSUPPORTED;
    if (even && lpp_apply_smem(p->dtype, p->d, p->p, std::min<int64_t>(k, reduce_max_k(p->dtype, p->d * p->p))) > 200 * 1024)
        return DM_ERR_UNSUPPORTED;
    DM_TRY(ensure_arena(p->ctx, matmat_scratch(p, k)));
    return matmat_run(ctx_exec(p->ctx), p, Z, k, ldz, out, ldo);
}

// --------------------------------------------------------------- gradient
dm_status grad_impl(dm_plan* p, const void* W, int64_t ldw, const void* Z, int64_t ldz, int64_t k,
                    void* G, int64_t ldg) {
    dm_ctx* ctx = p->ctx;
    const dm_dtype t = p->dtype;
    const int64_t n = p->n, d = p->d;
    GradArgs a{};
    a.dtype = t;
    a.n = n; a.d = d;
    a.W = W; a.ldw = ldw; a.Z = Z; a.ldz = ldz; a.k = k;
    a.G = G; a.ldg = ldg;
    a.num_sms = ctx->num_sms;
    const size_t gbytes = up16(grad_scratch_bytes(t, n, d, k));
    if (p->metric == DM_LPP || p->metric == DM_L2_EMBED) return DM_ERR_UNSUPPORTED;
    if (p->metric == DM_L1 || p->metric == DM_TV) {
        DM_TRY(ensure_arena(ctx, gbytes));
        a.scratch = ctx->arena;
        a.xs = p->xs; a.perm = p->perm;
        {
            ProfScope ps(ctx, "grad_pack");
            DM_TRY_CUDA(grad_pack_launch(a, ctx->stream, &ctx->launches));
        }
        {
            ProfScope ps(ctx, "grad_l1_tiles");
            DM_TRY_CUDA(grad_l1_launch(a, 0, ctx->stream, &ctx->launches));
        }
        {
            ProfScope ps(ctx, "grad_l1_scan");
            DM_TRY_CUDA(grad_l1_launch(a, 1, ctx->stream, &ctx->launches));
        }
        {
            ProfScope ps(ctx, "grad_l1_eval");
            DM_TRY_CUDA(grad_l1_launch(a, 2, ctx->stream, &ctx->launches));
        }
        {
            ProfScope ps(ctx, "grad_l1_transpose");
            DM_TRY_CUDA(grad_l1_launch(a, 3, ctx->stream, &ctx->launches));
        }
        if (p->metric == DM_TV) {
            ProfScope ps(ctx, "tv_scale");
            DM_TRY_CUDA(scale_launch(t, G, n, d, ldg, 0.5, ctx->num_sms, ctx->stream, &ctx->launches));
        }
        return DM_OK;
    }
    // squared l2: [X - mu, 1]^T [z_q, w_q] by the reduce kernel, then the closed form
    if (reduce_max_k(t, d) < 2 * k) return DM_ERR_UNSUPPORTED;
    ReduceArgs r{};
    r.dtype = t;
    r.n = n; r.d = d;
    r.k = 2 * k; r.ldz = 2 * k;
    r.num_sms = ctx->num_sms;
    r.err = ctx->err;
    r.engine = ctx->engine;
    r.spin_limit = ctx->spin_limit;
    const int blocks = reduce_blocks(r);
    const size_t o_res = up16(gbytes + (size_t)blocks * (d + 2) * 2 * k * 8);
    DM_TRY(ensure_arena(ctx, up16(o_res + (size_t)(d + 2) * 2 * k * 8)));
    unsigned char* base = static_cast<unsigned char*>(ctx->arena);
    a.scratch = base;
    r.partial = base + gbytes;
    r.res = base + o_res;
    r.Z = grad_packed(a);
    r.X = p->X; r.ldx = p->ldx; r.x_acc = false;
    r.mu = p->mu; r.mu_stride = 1;
    r.with_s = false;
    a.X = p->X; a.ldx = p->ldx; a.mu = p->mu; a.res = r.res;
    {
        ProfScope ps(ctx, "grad_pack");
        DM_TRY_CUDA(grad_pack_launch(a, ctx->stream, &ctx->launches));
    }
    {
        ProfScope ps(ctx, "grad_l2_reduce");
        DM_TRY_CUDA(reduce_launch(r, ctx->stream, &ctx->launches));
    }
    ProfScope ps(ctx, "grad_l2_apply");
    DM_TRY_CUDA(grad_l2_apply_launch(a, ctx->stream, &ctx->launches));
    return DM_OK;
}

// ------------------------------------------------------------------ batch
// Tear down the lanes and the graph (the plans stay).
void batch_release_graph(dm_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    for (auto st : b->streams) cudaStreamDestroy(st);
    for (auto p : b->scratch) cudaFree(p);
    for (auto ev : b->joins) cudaEventDestroy(ev);
    b->streams.clear();
    b->scratch.clear();
    b->scratch_bytes.clear();
    b->joins.clear();
    b->lanes = 0;
}

// Spread the sets over L lanes (largest first, each to the least loaded
// lane), give every lane a scratch buffer for its largest set, and capture
// prepare + product of every set into one graph: the lanes fork from the
// origin stream and join back into it.
dm_status batch_build(dm_batch* b, int L) {
    dm_ctx* ctx = b->ctx;
    batch_release_graph(b);
    std::vector<size_t> order(b->sets.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t x, size_t y) { return b->sets[x].cost > b->sets[y].cost; });
    std::vector<double> load((size_t)L, 0.0);
    std::vector<size_t> need((size_t)L, 16);
    for (size_t i : order) {
        auto& st = b->sets[i];
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        st.lane = l;
        load[(size_t)l] += st.cost;
        dm_plan* p = st.plan;
        const size_t prep = sorted_metric(p->metric) ? sort_layout(p->dtype, p->n, p->d).total : prepare_l2_scratch(p);
        need[(size_t)l] = std::max(need[(size_t)l], std::max(prep, matmat_scratch(p, st.k)));
    }
    for (int l = 0; l < L; ++l) {
        cudaStream_t st = nullptr;
        void* buf = nullptr;
        cudaEvent_t ev = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            if (st) cudaStreamDestroy(st);
            batch_release_graph(b);
            return DM_ERR_CUDA;
        }
        b->streams.push_back(st);
        b->joins.push_back(ev);
        if (cudaMalloc(&buf, need[(size_t)l]) != cudaSuccess) {
            cudaGetLastError();
            batch_release_graph(b);
            return DM_ERR_OOM;
        }
        b->scratch.push_back(buf);
        b->scratch_bytes.push_back(need[(size_t)l]);
    }
    b->lanes = L;

    const int64_t launches0 = ctx->launches;
    DM_TRY_CUDA(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed));
    dm_status s = from_cuda(cudaEventRecord(b->fork, b->origin));
    for (int l = 0; l < L && s == DM_OK; ++l) s = from_cuda(cudaStreamWaitEvent(b->streams[(size_t)l], b->fork, 0));
    for (size_t i = 0; i < b->sets.size() && s == DM_OK; ++i) {
        auto& st = b->sets[i];
        const Exec e{ctx, b->streams[(size_t)st.lane], static_cast<unsigned char*>(b->scratch[(size_t)st.lane]),
                     b->scratch_bytes[(size_t)st.lane], true};
        s = sorted_metric(st.plan->metric) ? prepare_l1_run(e, st.plan, st.X, st.ldx)
                                           : prepare_l2_run(e, st.plan, st.X, st.ldx);
        if (s == DM_OK) s = matmat_run(e, st.plan, st.Z, st.k, st.ldz, st.out, st.ldo);
    }
    for (int l = 0; l < L && s == DM_OK; ++l) {
        s = from_cuda(cudaEventRecord(b->joins[(size_t)l], b->streams[(size_t)l]));
        if (s == DM_OK) s = from_cuda(cudaStreamWaitEvent(b->origin, b->joins[(size_t)l], 0));
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->origin, &g);
    if (s == DM_OK) s = from_cuda(ee);
    if (s != DM_OK) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        batch_release_graph(b);
        return s;
    }
    b->graph = g;
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
        cudaGetLastError();
        batch_release_graph(b);
        return DM_ERR_CUDA;
    }
    b->launches_per_run = ctx->launches - launches0;
    ctx->launches = launches0;
    return DM_OK;
}

dm_status batch_launch(dm_batch* b) {
    dm_ctx* ctx = b->ctx;
    DM_TRY_CUDA(cudaEventRecord(b->done, ctx->stream));
    DM_TRY_CUDA(cudaStreamWaitEvent(b->origin, b->done, 0));
    DM_TRY_CUDA(cudaGraphLaunch(b->exec, b->origin));
    DM_TRY_CUDA(cudaEventRecord(b->done, b->origin));
    DM_TRY_CUDA(cudaStreamWaitEvent(ctx->stream, b->done, 0));
    ctx->launches += b->launches_per_run;
    return DM_OK;
}

// The autotuner's choices, by batch shape (process-wide, shared by threads).
std::map<std::string, int>& lane_cache() {
    static std::map<std::string, int> m;
    return m;
}
std::mutex& lane_cache_mutex() {
    static std::mutex mu;
    return mu;
}

bool lane_cache_find(const std::string& key, int* lanes) {
    std::lock_guard<std::mutex> lock(lane_cache_mutex());
    auto it = lane_cache().find(key);
    if (it == lane_cache().end()) return false;
    *lanes = it->second;
    return true;
}

void lane_cache_store(const std::string& key, int lanes) {
    std::lock_guard<std::mutex> lock(lane_cache_mutex());
    lane_cache()[key] = lanes;
}

std::string batch_key(const dm_batch* b) {
    double sn = 0, snd = 0, snk = 0;
    int64_t mx = 0;
    for (auto& st : b->sets) {
        sn += (double)st.plan->n;
        snd += (double)st.plan->n * (double)st.plan->d;
        snk += (double)st.plan->n * (double)st.k;
        mx = std::max(mx, st.plan->n * st.plan->d);
    }
    char buf[256];
    snprintf(buf, sizeof(buf), "%d/%d/%d/%.0f/%.0f/%.0f/%lld/%d", (int)b->metric, (int)b->dtype,
             (int)b->sets.size(), sn, snd, snk, (long long)mx, b->ctx->deterministic);
    return buf;
}

// Time each candidate lane count on the batch (one warm-up and three timed
// replays of its graph) and keep the fastest.
dm_status batch_autotune(dm_batch* b) {
    const std::string key = batch_key(b);
    int cached = 0;
    if (lane_cache_find(key, &cached)) return batch_build(b, cached);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    DM_TRY_CUDA(cudaEventCreate(&t0));
    if (cudaEventCreate(&t1) != cudaSuccess) { cudaEventDestroy(t0); return DM_ERR_CUDA; }
    int best = 1;
    float best_ms = -1.0f;
    dm_status s = DM_OK;
    for (int L : {1, 2, 4, 8, 16}) {
        if (L > (int)b->sets.size() && L > 1) break;
        s = batch_build(b, L);
        if (s != DM_OK) break;
        s = batch_launch(b);
        if (s == DM_OK) s = from_cuda(cudaEventRecord(t0, b->ctx->stream));
        for (int r = 0; r < 3 && s == DM_OK; ++r) s = batch_launch(b);
        if (s == DM_OK) s = from_cuda(cudaEventRecord(t1, b->ctx->stream));
        if (s == DM_OK) s = from_cuda(cudaEventSynchronize(t1));
        float ms = 0;
        if (s == DM_OK) s = from_cuda(cudaEventElapsedTime(&ms, t0, t1));
        if (s != DM_OK) break;
        if (best_ms < 0 || ms < best_ms) { best_ms = ms; best = L; }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (s != DM_OK) return s;
    lane_cache_store(key, best);
    return batch_build(b, best);
}

void batch_free(dm_batch* b) {
    if (b->origin) cudaStreamSynchronize(b->origin);
    if (b->ctx && !b->ctx->destroyed) cudaStreamSynchronize(b->ctx->stream);
    batch_release_graph(b);
    for (auto& st : b->sets) {
        if (st.plan) { free_plan_buffers(st.plan); delete st.plan; }
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->done) cudaEventDestroy(b->done);
    if (b->origin) cudaStreamDestroy(b->origin);
    delete b;
}

// Release everything a context owns.  The caller has synchronized its
// stream (dm_destroy) or the stream may be gone already (the last child of a
// destroyed context): only device-wide waits are used here.
void ctx_free(dm_ctx* ctx) {
    for (size_t i = 0; i < ctx->peers.size(); ++i) {
        dm_destroy(ctx->peers[i]);             // no plans outlive a host call
        cudaStreamDestroy(ctx->peer_streams[i]);
    }
    if (ctx->x_done) cudaEventDestroy(ctx->x_done);
    if (ctx->arena) cudaFree(ctx->arena);
    for (auto& b : ctx->pool) cudaFree(b.p);
    if (ctx->hx) cudaFree(ctx->hx);
    if (ctx->hz) cudaFree(ctx->hz);
    if (ctx->ho) cudaFree(ctx->ho);
    if (ctx->aux) { cudaStreamSynchronize(ctx->aux); cudaStreamDestroy(ctx->aux); }
    if (ctx->aux_done) cudaEventDestroy(ctx->aux_done);
    if (ctx->err) cudaFree(ctx->err);
    if (ctx->host_err) cudaFreeHost(ctx->host_err);
    if (ctx->host_hist) cudaFreeHost(ctx->host_hist);
    for (auto& p : ctx->pending) { cudaEventDestroy(p.start); cudaEventDestroy(p.stop); }
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    delete ctx;
}

// A plan or batch of `ctx` is gone; the context follows it when it was
// destroyed already and this was its last child.
void child_released(dm_ctx* ctx) {
    if (--ctx->children == 0 && ctx->destroyed) ctx_free(ctx);
}

}  // namespace

// ===================================================================== ABI
extern "C" {

const char* dm_status_string(dm_status s) {
    switch (s) {
        case DM_OK: return "DM_OK";
        case DM_ERR_INVALID_ARG: return "DM_ERR_INVALID_ARG";
        case DM_ERR_UNSUPPORTED: return "DM_ERR_UNSUPPORTED";
        case DM_ERR_NONFINITE: return "DM_ERR_NONFINITE";
        case DM_ERR_OOM: return "DM_ERR_OOM";
        case DM_ERR_CUDA: return "DM_ERR_CUDA";
        case DM_ERR_TIMEOUT: return "DM_ERR_TIMEOUT";
        case DM_ERR_INTERNAL: return "DM_ERR_INTERNAL";
    }
    return "DM_ERR_UNKNOWN";
}

dm_status dm_create(dm_ctx** out, int device, void* stream) {
    if (!out) return DM_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) { cudaGetLastError(); return DM_ERR_CUDA; }
    if (device < 0 || device >= count) return DM_ERR_INVALID_ARG;
    DeviceGuard g(device);
    dm_ctx* ctx = new (std::nothrow) dm_ctx();
    if (!ctx) return DM_ERR_OOM;
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(stream);
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc(reinterpret_cast<void**>(&ctx->err), 4) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&ctx->host_err), 4) != cudaSuccess ||
        cudaMemset(ctx->err, 0, 4) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->err) cudaFree(ctx->err);
        if (ctx->host_err) cudaFreeHost(ctx->host_err);
        delete ctx;
        return DM_ERR_OOM;
    }
    *out = ctx;
    return DM_OK;
}

void dm_destroy(dm_ctx* ctx) {
    if (!ctx || ctx->destroyed) return;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    ctx->destroyed = true;
    if (ctx->children == 0) ctx_free(ctx);
}

dm_status dm_set_deterministic(dm_ctx* ctx, int on) {
    if (!ctx || ctx->destroyed) return DM_ERR_INVALID_ARG;
    ctx->deterministic = on ? 1 : 0;
    return DM_OK;
}

dm_status dm_set_wait_limit(dm_ctx* ctx, uint32_t rounds) {
    if (!ctx || ctx->destroyed) return DM_ERR_INVALID_ARG;
    ctx->spin_limit = rounds ? rounds : dm::kSpinLimit;
    return DM_OK;
}

dm_status dm_test_unpublished_wait(dm_ctx* ctx) {
    if (!ctx || ctx->destroyed) return DM_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    const int64_t n = 2 * (int64_t)sort_tile_f32();
    const SortLayout L = sort_layout(DM_F32, n, 1);
    DM_TRY(ensure_arena(ctx, L.total));
    unsigned char* base = static_cast<unsigned char*>(ctx->arena);
    SortArgs a{};
    a.dtype = DM_F32;
    a.n = n; a.d = 1; a.ldx = 1;
    a.keys_a = base + L.ka; a.keys_b = base + L.kb;
    a.vals_a = reinterpret_cast<int32_t*>(base + L.va);
    a.vals_b = reinterpret_cast<int32_t*>(base + L.vb);
    a.hist = reinterpret_cast<uint32_t*>(base + L.hist);
    a.counters = reinterpret_cast<uint32_t*>(base + L.cnt);
    a.lookback = reinterpret_cast<uint32_t*>(base + L.lb);
    a.err = ctx->err;
    a.spin_limit = ctx->spin_limit;
    // zero keys, histograms and look-back words; the tile counter starts at 1
    DM_TRY_CUDA(cudaMemsetAsync(base, 0, L.kb, ctx->stream));
    DM_TRY_CUDA(cudaMemsetAsync(a.counters, 1, 1, ctx->stream));
    DM_TRY_CUDA(sort_launch_unpublished_wait(a, ctx->stream, &ctx->launches));
    return DM_OK;
}

dm_status dm_set_engine(dm_ctx* ctx, dm_engine engine) {
    if (!ctx || ctx->destroyed || (engine != DM_ENGINE_AUTO && engine != DM_ENGINE_CUDA_CORES && engine != DM_ENGINE_TENSOR_CORES))
        return DM_ERR_INVALID_ARG;
    ctx->engine = engine;
    return DM_OK;
}

dm_status dm_set_stream(dm_ctx* ctx, void* stream) {
    if (!ctx || ctx->destroyed) return DM_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);   // pooled buffers may be in use on the old stream
    ctx->stream = static_cast<cudaStream_t>(stream);
    return DM_OK;
}

int64_t dm_launch_count(const dm_ctx* ctx) { return ctx ? ctx->launches : 0; }

dm_status dm_profile_enable(dm_ctx* ctx, int enable) {
    if (!ctx || ctx->destroyed) return DM_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    DM_TRY(resolve_profile(ctx));
    ctx->stats.clear();
    ctx->profiling = enable != 0;
    return DM_OK;
}

dm_status dm_profile_read(dm_ctx* ctx, int max, int* count, char* names, int64_t* launches,
                          double* total_ms) {
    if (!ctx || ctx->destroyed || !count || max < 0 || (max > 0 && (!names || !launches || !total_ms)))
        return DM_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    DM_TRY(resolve_profile(ctx));
    int i = 0;
    for (const auto& kv : ctx->stats) {
        if (i >= max) break;
        std::memset(names + 32 * i, 0, 32);
        std::strncpy(names + 32 * i, kv.first.c_str(), 31);
        launches[i] = kv.second.launches;
        total_ms[i] = kv.second.ms;
        ++i;
    }
    *count = i;
    return DM_OK;
}

dm_status dm_prepare(dm_ctx* ctx, dm_metric metric, dm_dtype dtype, const void* X, int64_t n,
                     int64_t d, int64_t ldx, dm_plan** plan) {
    if (!plan) return DM_ERR_INVALID_ARG;
    *plan = nullptr;
    if (!ctx || ctx->destroyed || !X || !(valid_metric(metric) || metric == DM_TV) || !valid_dtype(dtype))
        return DM_ERR_INVALID_ARG;
    if (metric == DM_TV && dtype == DM_I32) return DM_ERR_UNSUPPORTED;   // half-integer results
    if (n < 1 || n > kMaxN || d < 1 || ldx < d) return DM_ERR_INVALID_ARG;
    if ((double)n * (double)d >= 2147483648.0) return DM_ERR_UNSUPPORTED;
    DeviceGuard g(ctx->device);
    dm_plan* p = new (std::nothrow) dm_plan();
    if (!p) return DM_ERR_OOM;
    p->ctx = ctx;
    p->metric = metric;
    p->dtype = dtype;
    p->n = n;
    p->d = d;
    const dm_status s = sorted_metric(metric) ? prepare_l1(ctx, p, X, ldx) : prepare_l2(ctx, p, X, ldx);
    if (s != DM_OK) {
        cudaStreamSynchronize(ctx->stream);
        cudaGetLastError();
        free_plan_buffers(p);
        delete p;
        return s;
    }
    ++ctx->children;
    *plan = p;
    return DM_OK;
}

dm_status dm_prepare_lpp(dm_ctx* ctx, dm_dtype dtype, const void* X, int64_t n, int64_t d, int64_t ldx,
                         int pw, dm_plan** plan) {
    if (!plan) return DM_ERR_INVALID_ARG;
    *plan = nullptr;
    const bool odd = (pw & 1) != 0;
    if (!ctx || !X || !valid_dtype(dtype) || pw < 2 || pw > (odd ? 15 : 16)) return DM_ERR_INVALID_ARG;
    if (n < 1 || n > kMaxN || d < 1 || ldx < d) return DM_ERR_INVALID_ARG;
    if (odd && (double)n * (double)d >= 2147483648.0) return DM_ERR_UNSUPPORTED;
    if (!odd && (double)n * (double)d * pw >= 2147483648.0) return DM_ERR_UNSUPPORTED;
    if (!odd && (reduce_max_k(dtype, d * pw) < 1 || lpp_apply_smem(dtype, d, pw, 1) > 200 * 1024))
        return DM_ERR_UNSUPPORTED;
    if (ctx->destroyed) return DM_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    dm_plan* p = new (std::nothrow) dm_plan();
    if (!p) return DM_ERR_OOM;
    p->ctx = ctx; p->metric = DM_LPP; p->dtype = dtype; p->n = n; p->d = d; p->p = pw;
    // even p: X and its column means; odd p: the sorted coordinates (Algorithm 1)
    const dm_status s = odd ? prepare_l1(ctx, p, X, ldx) : prepare_l2(ctx, p, X, ldx);
    if (s != DM_OK) {
        cudaStreamSynchronize(ctx->stream);
        cudaGetLastError();
        free_plan_buffers(p);
        delete p;
        return s;
    }
    ++ctx->children;
    *plan = p;
    return DM_OK;
}

dm_status dm_prepare_l2_embed(dm_ctx* ctx, dm_dtype dtype, const void* X, int64_t n, int64_t d,
                              int64_t ldx, const void* G, int64_t m, dm_plan** plan) {
    if (!plan) return DM_ERR_INVALID_ARG;
    *plan = nullptr;
    if (!ctx || ctx->destroyed || !X || !G || (dtype != DM_F32 && dtype != DM_F64) || m < 1)
        return DM_ERR_INVALID_ARG;
    if (n < 1 || n > kMaxN || d < 1 || ldx < d) return DM_ERR_INVALID_ARG;
    if ((double)n * (double)m >= 2147483648.0) return DM_ERR_UNSUPPORTED;
    if (project_smem(dtype, d, m) > 200 * 1024) return DM_ERR_UNSUPPORTED;
    DeviceGuard g(ctx->device);
    dm_plan* p = new (std::nothrow) dm_plan();
    if (!p) return DM_ERR_OOM;
    p->ctx = ctx; p->metric = DM_L2_EMBED; p->dtype = dtype; p->n = n; p->d = m; p->d_in = d;
    // T(X) into a buffer of the plan, the l1 plan of T(X), then the buffer
    // goes back to the context (the plan keeps only the sorted coordinates).
    void* Xp = nullptr;
    dm_status s = plan_alloc(p, (size_t)n * m * dtype_size(dtype), &Xp);
    if (s == DM_OK) {
        ProfScope ps(ctx, "l2_embed_project");
        s = from_cuda(project_launch(dtype, X, n, d, ldx, G, m, Xp, ctx->num_sms, ctx->stream, &ctx->launches));
    }
    if (s == DM_OK) s = prepare_l1(ctx, p, Xp, m);
    if (s == DM_OK) {
        for (size_t i = 0; i < p->owned.size(); ++i) {
            if (p->owned[i].first == Xp) {
                if (ctx->pool_bytes + p->owned[i].second <= kPoolCap) {
                    ctx->pool.push_back({Xp, p->owned[i].second});
                    ctx->pool_bytes += p->owned[i].second;
                } else {
                    cudaStreamSynchronize(ctx->stream);
                    cudaFree(Xp);
                }
                p->owned.erase(p->owned.begin() + (long)i);
                break;
            }
        }
    }
    if (s != DM_OK) {
        cudaStreamSynchronize(ctx->stream);
        cudaGetLastError();
        free_plan_buffers(p);
        delete p;
        return s;
    }
    ++ctx->children;
    *plan = p;
    return DM_OK;
}

void dm_plan_destroy(dm_plan* p) {
    if (!p) return;
    dm_ctx* ctx = p->ctx;
    DeviceGuard g(ctx->device);
    free_plan_buffers(p);   // stream-ordered reuse: no wait needed
    delete p;
    child_released(ctx);
}

dm_status dm_matmat(dm_plan* p, const void* Z, int64_t k, int64_t ldz, void* out, int64_t ldo) {
    if (!p || p->ctx->destroyed || !Z || !out || k < 1 || ldz < k || ldo < k) return DM_ERR_INVALID_ARG;
    DeviceGuard g(p->ctx->device);
    return matmat_impl(p, Z, k, ldz, out, ldo);
}

dm_status dm_grad(dm_plan* p, const void* W, int64_t ldw, const void* Z, int64_t ldz, int64_t k,
                  void* G, int64_t ldg) {
    if (!p || p->ctx->destroyed || !W || !Z || !G || k < 1 || k > 64 || ldw < k || ldz < k || ldg < p->d)
        return DM_ERR_INVALID_ARG;
    DeviceGuard g(p->ctx->device);
    return grad_impl(p, W, ldw, Z, ldz, k, G, ldg);
}

dm_status dm_batch_create(dm_ctx* ctx, dm_metric metric, dm_dtype dtype, int64_t nsets,
                          const int64_t* n, const int64_t* d, const void* const* X,
                          const int64_t* ldx, const int64_t* k, const void* const* Z,
                          const int64_t* ldz, void* const* out, const int64_t* ldo, int lanes,
                          dm_batch** batch) {
    if (!batch) return DM_ERR_INVALID_ARG;
    *batch = nullptr;
    if (!ctx || ctx->destroyed || !(valid_metric(metric) || metric == DM_TV) || !valid_dtype(dtype) || nsets < 1 || lanes < 0 ||
        lanes > 64 ||
        !n || !d || !X || !ldx || !k || !Z || !ldz || !out || !ldo)
        return DM_ERR_INVALID_ARG;
    for (int64_t i = 0; i < nsets; ++i) {
        if (!X[i] || !Z[i] || !out[i] || n[i] < 1 || n[i] > kMaxN || d[i] < 1 || ldx[i] < d[i] ||
            k[i] < 1 || ldz[i] < k[i] || ldo[i] < k[i])
            return DM_ERR_INVALID_ARG;
        if ((double)n[i] * (double)d[i] >= 2147483648.0) return DM_ERR_UNSUPPORTED;
        if (metric == DM_L2SQ && reduce_max_k(dtype, d[i]) < 1) return DM_ERR_UNSUPPORTED;
    }
    DeviceGuard g(ctx->device);
    dm_batch* b = new (std::nothrow) dm_batch();
    if (!b) return DM_ERR_OOM;
    b->ctx = ctx;
    b->metric = metric;
    b->dtype = dtype;
    dm_status s = DM_OK;
    if (cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        s = DM_ERR_CUDA;
    }
    for (int64_t i = 0; i < nsets && s == DM_OK; ++i) {
        dm_plan* p = new (std::nothrow) dm_plan();
        if (!p) { s = DM_ERR_OOM; break; }
        p->ctx = ctx; p->metric = metric; p->dtype = dtype; p->n = n[i]; p->d = d[i];
        const double es = (double)dtype_size(dtype);
        if (metric == DM_TV && dtype == DM_I32) { s = DM_ERR_UNSUPPORTED; delete p; break; }
        const double cost = sorted_metric(metric) ? (double)n[i] * d[i] * (8.0 + 8.0 * k[i] + 64.0)
                                            : (double)n[i] * (2.0 * d[i] * es + 2.0 * k[i] * es);
        b->sets.push_back({p, X[i], ldx[i], Z[i], k[i], ldz[i], out[i], ldo[i], cost, 0});
        s = sorted_metric(metric) ? alloc_l1_plan(p) : plan_alloc(p, (size_t)d[i] * dtype_size(dtype), &p->mu);
        if (metric == DM_L2SQ) { p->X = X[i]; p->ldx = ldx[i]; }
    }
    if (s == DM_OK) s = lanes > 0 ? batch_build(b, (int)std::min<int64_t>(lanes, nsets)) : batch_autotune(b);
    if (s != DM_OK) {
        batch_free(b);
        return s;
    }
    ++ctx->children;
    *batch = b;
    return DM_OK;
}

dm_status dm_batch_run(dm_batch* b) {
    if (!b || !b->exec || b->ctx->destroyed) return DM_ERR_INVALID_ARG;
    DeviceGuard g(b->ctx->device);
    return batch_launch(b);
}

int dm_batch_lanes(const dm_batch* b) { return b ? b->lanes : 0; }

void dm_batch_destroy(dm_batch* b) {
    if (!b) return;
    dm_ctx* ctx = b->ctx;
    DeviceGuard g(ctx->device);
    batch_free(b);
    child_released(ctx);
}

dm_status dm_matvec_l1(dm_plan* p, const void* z, void* out) {
    if (!p || p->metric != DM_L1) return DM_ERR_INVALID_ARG;
    return dm_matmat(p, z, 1, 1, out, 1);
}

dm_status dm_matvec_l2sq(dm_plan* p, const void* z, void* out) {
    if (!p || p->metric != DM_L2SQ) return DM_ERR_INVALID_ARG;
    return dm_matmat(p, z, 1, 1, out, 1);
}

dm_status dm_dense_tn(dm_ctx* ctx, const float* A, int64_t n, int64_t m, int64_t lda, const float* B,
                      int64_t k, int64_t ldb, float* C, int64_t ldc, float alpha) {
    if (!ctx || ctx->destroyed || !A || !B || !C || n < 1 || m < 1 || k < 1 || lda < m || ldb < k || ldc < k)
        return DM_ERR_INVALID_ARG;
    if (m > INT_MAX / 2 || k > INT_MAX / 2) return DM_ERR_UNSUPPORTED;
    DeviceGuard g(ctx->device);
    int chunks = 0;
    int64_t rpc = 0;
    dense_tn_plan(n, m, k, ctx->num_sms, &chunks, &rpc);
    DM_TRY(ensure_arena(ctx, (size_t)chunks * (size_t)m * (size_t)k * sizeof(float)));
    ProfScope ps(ctx, "dense_tn");
    DM_TRY_CUDA(dense_tn_launch(A, n, m, lda, B, k, ldb, C, ldc, alpha, static_cast<float*>(ctx->arena),
                                ctx->num_sms, ctx->stream, &ctx->launches));
    return DM_OK;
}

dm_status dm_dense_nn(dm_ctx* ctx, const float* A, int64_t n, int64_t m, int64_t lda, const float* T,
                      int64_t k, int64_t ldt, float* C, int64_t ldc, float alpha, float beta) {
    if (!ctx || ctx->destroyed || !A || !T || !C || n < 1 || m < 1 || k < 1 || lda < m || ldt < k || ldc < k)
        return DM_ERR_INVALID_ARG;
    if (k > 64 || m > INT_MAX / 2) return DM_ERR_UNSUPPORTED;
    DeviceGuard g(ctx->device);
    ProfScope ps(ctx, "dense_nn");
    DM_TRY_CUDA(dense_nn_launch(A, n, m, lda, T, k, ldt, C, ldc, alpha, beta, ctx->stream, &ctx->launches));
    return DM_OK;
}

dm_status dm_sync(dm_ctx* ctx) {
    if (!ctx || ctx->destroyed) return DM_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return from_cuda(e);
    return take_device_error(ctx);
}

dm_status dm_plan_export(dm_plan* p, void* sorted_values, int32_t* perm) {
    if (!p || p->ctx->destroyed || !(sorted_metric(p->metric) || lpp_odd(p)) || !sorted_values || !perm)
        return DM_ERR_INVALID_ARG;
    DeviceGuard g(p->ctx->device);
    const size_t nd = (size_t)p->n * (size_t)p->d;
    DM_TRY_CUDA(cudaMemcpyAsync(sorted_values, p->xs, nd * dtype_size(p->dtype),
                                cudaMemcpyDeviceToDevice, p->ctx->stream));
    DM_TRY_CUDA(cudaMemcpyAsync(perm, p->perm, nd * 4, cudaMemcpyDeviceToDevice, p->ctx->stream));
    return DM_OK;
}

dm_status dm_bruteforce(dm_ctx* ctx, dm_metric metric, dm_dtype dtype, const void* X, int64_t n,
                        int64_t d, int64_t ldx, const void* Z, int64_t k, int64_t ldz, void* out,
                        int64_t ldo) {
    if (!ctx || ctx->destroyed || !X || !Z || !out || !valid_metric(metric) || !valid_dtype(dtype))
        return DM_ERR_INVALID_ARG;
    if (n < 1 || n > kMaxN || d < 1 || ldx < d || k < 1 || ldz < k || ldo < k) return DM_ERR_INVALID_ARG;
    if (d > 64) return DM_ERR_UNSUPPORTED;
    DeviceGuard g(ctx->device);
    BruteArgs a{};
    a.dtype = dtype; a.metric = metric;
    a.X = X; a.n = n; a.d = d; a.ldx = ldx;
    a.Z = Z; a.k = k; a.ldz = ldz;
    a.out = out; a.ldo = ldo;
    ProfScope ps(ctx, "bruteforce");
    DM_TRY_CUDA(brute_launch(a, ctx->stream, &ctx->launches));
    return DM_OK;
}

}  // extern "C"

namespace {

// Order of the host-to-device copies of concurrent dm_matmat_host calls on
// one device: each call's copies of X and Z wait for the previous call's
// copies, so the calls take the host link one after the other at its full
// rate instead of sharing it (the first call's preprocessing then starts
// after its own copies, not after everyone's).  One event per device, moved
// under the mutex.
struct LinkOrder {
    std::mutex mu;
    std::map<int, cudaEvent_t> last_h2d;
};
LinkOrder& link_order() {
    static LinkOrder* L = new LinkOrder();   // never destroyed: calls may run at exit
    return *L;
}

// The copies, preprocessing, product and copy back of dm_matmat_host,
// issued on the context's streams without waiting for them.
dm_status matmat_host_issue(dm_ctx* ctx, dm_metric metric, dm_dtype dtype, const void* Xh, int64_t n,
                            int64_t d, int64_t ldx, const void* Zh, int64_t k, int64_t ldz, void* outh,
                            int64_t ldo) {
    if (!ctx || ctx->destroyed || !Xh || !Zh || !outh || !valid_metric(metric) || !valid_dtype(dtype))
        return DM_ERR_INVALID_ARG;
    if (n < 1 || n > kMaxN || d < 1 || ldx < d || k < 1 || ldz < k || ldo < k) return DM_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    const size_t es = dtype_size(dtype), os = out_size(dtype);
    DM_TRY(ensure_buffer(ctx, &ctx->hx, &ctx->hx_bytes, (size_t)n * d * es));
    if (ctx->aux) DM_TRY_CUDA(cudaStreamSynchronize(ctx->aux));   // an earlier copy may still target hz
    DM_TRY(ensure_buffer(ctx, &ctx->hz, &ctx->hz_bytes, (size_t)n * k * es));
    DM_TRY(ensure_buffer(ctx, &ctx->ho, &ctx->ho_bytes, (size_t)n * k * os));
    if (!ctx->aux) {
        DM_TRY_CUDA(cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking));
        DM_TRY_CUDA(cudaEventCreateWithFlags(&ctx->aux_done, cudaEventDisableTiming));
    }
    // X crosses the host link first, alone and at the link's full rate, so
    // preprocessing starts as early as possible; Z follows on the second
    // stream while X is preprocessed, and the product waits for it.  (The
    // second stream waits for the X copy, and with it for earlier work on the
    // context's stream, which may still read the previous Z.)
    {
        LinkOrder& L = link_order();
        std::lock_guard<std::mutex> lock(L.mu);
        cudaEvent_t& last = L.last_h2d[ctx->device];
        if (!last) DM_TRY_CUDA(cudaEventCreateWithFlags(&last, cudaEventDisableTiming));
        else DM_TRY_CUDA(cudaStreamWaitEvent(ctx->stream, last, 0));
        DM_TRY_CUDA(cudaMemcpy2DAsync(ctx->hx, d * es, Xh, ldx * es, d * es, n, cudaMemcpyHostToDevice,
                                      ctx->stream));
        DM_TRY_CUDA(cudaEventRecord(ctx->aux_done, ctx->stream));
        DM_TRY_CUDA(cudaStreamWaitEvent(ctx->aux, ctx->aux_done, 0));
        DM_TRY_CUDA(cudaMemcpy2DAsync(ctx->hz, k * es, Zh, ldz * es, k * es, n, cudaMemcpyHostToDevice,
                                      ctx->aux));
        DM_TRY_CUDA(cudaEventRecord(ctx->aux_done, ctx->aux));
        DM_TRY_CUDA(cudaEventRecord(last, ctx->aux));
    }
    dm_plan* p = nullptr;
    DM_TRY(dm_prepare(ctx, metric, dtype, ctx->hx, n, d, d, &p));
    DM_TRY_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->aux_done, 0));
    dm_status s = dm_matmat(p, ctx->hz, k, k, ctx->ho, k);
    if (s == DM_OK) {
        cudaError_t e = cudaMemcpy2DAsync(outh, ldo * os, ctx->ho, k * os, k * os, n,
                                          cudaMemcpyDeviceToHost, ctx->stream);
        s = from_cuda(e);
    }
    // the plan's buffers go back to the context's pool: later use of them is
    // ordered after this product on the same stream
    dm_plan_destroy(p);
    return s;
}

}  // namespace

extern "C" {

dm_status dm_matmat_host(dm_ctx* ctx, dm_metric metric, dm_dtype dtype, const void* Xh, int64_t n,
                         int64_t d, int64_t ldx, const void* Zh, int64_t k, int64_t ldz,
                         void* outh, int64_t ldo) {
    dm_status s = matmat_host_issue(ctx, metric, dtype, Xh, n, d, ldx, Zh, k, ldz, outh, ldo);
    if (s == DM_OK) s = dm_sync(ctx);
    return s;
}

dm_status dm_matmat_host_async(dm_ctx* ctx, dm_metric metric, dm_dtype dtype, const void* Xh, int64_t n,
                               int64_t d, int64_t ldx, const void* Zh, int64_t k, int64_t ldz,
                               void* outh, int64_t ldo) {
    return matmat_host_issue(ctx, metric, dtype, Xh, n, d, ldx, Zh, k, ldz, outh, ldo);
}

dm_status dm_matmat_host_multi(dm_ctx* ctx, int count, const dm_metric* metrics, dm_dtype dtype,
                               const void* Xh, int64_t n, int64_t d, int64_t ldx, const void* Zh,
                               int64_t k, int64_t ldz, void* const* outh, int64_t ldo) {
    if (!ctx || ctx->destroyed || !metrics || !Xh || !Zh || !outh || !valid_dtype(dtype) || count < 1 ||
        count > kMaxHostProducts)
        return DM_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i)
        if (!valid_metric(metrics[i]) || !outh[i]) return DM_ERR_INVALID_ARG;
    if (n < 1 || n > kMaxN || d < 1 || ldx < d || k < 1 || ldz < k || ldo < k) return DM_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    const size_t es = dtype_size(dtype), os = out_size(dtype);
    const size_t out_bytes = (size_t)n * k * os;
    DM_TRY(ensure_buffer(ctx, &ctx->hx, &ctx->hx_bytes, (size_t)n * d * es));
    if (ctx->aux) DM_TRY_CUDA(cudaStreamSynchronize(ctx->aux));
    DM_TRY(ensure_buffer(ctx, &ctx->hz, &ctx->hz_bytes, (size_t)n * k * es));
    DM_TRY(ensure_buffer(ctx, &ctx->ho, &ctx->ho_bytes, out_bytes * count));
    if (!ctx->aux) {
        DM_TRY_CUDA(cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking));
        DM_TRY_CUDA(cudaEventCreateWithFlags(&ctx->aux_done, cudaEventDisableTiming));
    }
    if (!ctx->x_done) DM_TRY_CUDA(cudaEventCreateWithFlags(&ctx->x_done, cudaEventDisableTiming));
    // one context per product: the call's own for the first, peers for the rest
    while ((int)ctx->peers.size() < count - 1) {
        cudaStream_t ps = nullptr;
        DM_TRY_CUDA(cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking));
        dm_ctx* peer = nullptr;
        const dm_status cs = dm_create(&peer, ctx->device, ps);
        if (cs != DM_OK) { cudaStreamDestroy(ps); return cs; }
        ctx->peers.push_back(peer);
        ctx->peer_streams.push_back(ps);
    }
    // X and Z cross the host link once for all products, in the device's
    // link order (X alone first, Z on the second stream behind it)
    {
        LinkOrder& L = link_order();
        std::lock_guard<std::mutex> lock(L.mu);
        cudaEvent_t& last = L.last_h2d[ctx->device];
        if (!last) DM_TRY_CUDA(cudaEventCreateWithFlags(&last, cudaEventDisableTiming));
        else DM_TRY_CUDA(cudaStreamWaitEvent(ctx->stream, last, 0));
        DM_TRY_CUDA(cudaMemcpy2DAsync(ctx->hx, d * es, Xh, ldx * es, d * es, n, cudaMemcpyHostToDevice,
                                      ctx->stream));
        DM_TRY_CUDA(cudaEventRecord(ctx->x_done, ctx->stream));
        DM_TRY_CUDA(cudaStreamWaitEvent(ctx->aux, ctx->x_done, 0));
        DM_TRY_CUDA(cudaMemcpy2DAsync(ctx->hz, k * es, Zh, ldz * es, k * es, n, cudaMemcpyHostToDevice,
                                      ctx->aux));
        DM_TRY_CUDA(cudaEventRecord(ctx->aux_done, ctx->aux));
        DM_TRY_CUDA(cudaEventRecord(last, ctx->aux));
    }
    // Issue order: products whose preprocessing does not wait on the host
    // first (an l1 plan reads its key histograms back), each on its context.
    int order[kMaxHostProducts];
    int m = 0;
    for (int pass = 0; pass < 2; ++pass)
        for (int i = 0; i < count; ++i)
            if (sorted_metric(metrics[i]) == (pass == 1)) order[m++] = i;
    dm_status s = DM_OK;
    int used = 0;
    for (int j = 0; j < count && s == DM_OK; ++j) {
        used = j + 1;
        const int i = order[j];
        dm_ctx* e = j == 0 ? ctx : ctx->peers[j - 1];
        if (j > 0) {
            e->deterministic = ctx->deterministic;
            e->spin_limit = ctx->spin_limit;
            e->engine = ctx->engine;
            s = from_cuda(cudaStreamWaitEvent(e->stream, ctx->x_done, 0));
            if (s != DM_OK) break;
        }
        const int64_t before = e->launches;
        dm_plan* p = nullptr;
        s = dm_prepare(e, metrics[i], dtype, ctx->hx, n, d, d, &p);
        if (s != DM_OK) break;
        void* oi = static_cast<unsigned char*>(ctx->ho) + out_bytes * i;
        s = from_cuda(cudaStreamWaitEvent(e->stream, ctx->aux_done, 0));
        if (s == DM_OK) s = dm_matmat(p, ctx->hz, k, k, oi, k);
        if (s == DM_OK)
            s = from_cuda(cudaMemcpy2DAsync(outh[i], ldo * os, oi, k * os, k * os, n,
                                            cudaMemcpyDeviceToHost, e->stream));
        dm_plan_destroy(p);
        if (j > 0) ctx->launches += e->launches - before;
    }
    // wait for every product issued; the first error wins
    for (int j = 0; j < used; ++j) {
        const dm_status t = dm_sync(j == 0 ? ctx : ctx->peers[j - 1]);
        if (s == DM_OK) s = t;
    }
    return s;
}

}  // extern "C"
