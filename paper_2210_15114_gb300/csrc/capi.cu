// C ABI of libdm: contexts, plans, argument checks, scratch management and
// the launch sequences of each call.  Host code only; kernels live in the
// other translation units.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
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
    // Device buffers of dm_matmat_host (grown on demand).
    void* hx = nullptr; size_t hx_bytes = 0;
    void* hz = nullptr; size_t hz_bytes = 0;
    void* ho = nullptr; size_t ho_bytes = 0;
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
    // squared l2
    const void* X = nullptr;
    int64_t ldx = 0;
    void* mu = nullptr;
};

namespace {

using namespace dm;

constexpr int64_t kMaxN = (int64_t(1) << 30) - 1;

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

// Brackets one group of launches with events when timing is enabled.
struct ProfScope {
    dm_ctx* ctx;
    const char* name;
    cudaEvent_t start = nullptr;
    int64_t before = 0;
    ProfScope(dm_ctx* c, const char* n) : ctx(c), name(n) {
        if (!ctx->profiling) return;
        start = pool_event(ctx);
        before = ctx->launches;
        if (start) cudaEventRecord(start, ctx->stream);
    }
    ~ProfScope() {
        if (!ctx->profiling || !start) return;
        cudaEvent_t stop = pool_event(ctx);
        if (!stop) { ctx->event_pool.push_back(start); return; }
        cudaEventRecord(stop, ctx->stream);
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

// Hand a plan's buffers back to the context pool (freed beyond the cap).
void plan_release(dm_plan* p) {
    dm_ctx* ctx = p->ctx;
    for (auto& ob : p->owned) {
        if (ctx->pool_bytes + ob.second <= kPoolCap) {
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
dm_status prepare_l1(dm_ctx* ctx, dm_plan* p, const void* X, int64_t ldx) {
    const dm_dtype t = p->dtype;
    const int64_t n = p->n, d = p->d;
    const size_t nd = (size_t)n * (size_t)d;
    const size_t key_bytes = key_bits(t) / 8;
    const int P = sort_passes(t);
    const size_t hist_words = sort_hist_words(t, d);
    const size_t lb_words = sort_lookback_words(t, n, d);

    DM_TRY(plan_alloc(p, nd * dtype_size(t), &p->xs));
    DM_TRY(plan_alloc(p, nd * 4, reinterpret_cast<void**>(&p->perm)));

    // arena: [hist | counters | lookback] (zeroed) then keys_a, keys_b, vals_a, vals_b
    const size_t o_hist = 0;
    const size_t o_cnt = up16(o_hist + hist_words * 4);
    const size_t o_lb = up16(o_cnt + 4 * (size_t)P);
    const size_t zero_bytes = up16(o_lb + lb_words * 4);
    const size_t o_ka = zero_bytes;
    const size_t o_kb = up16(o_ka + nd * key_bytes);
    const size_t o_va = up16(o_kb + nd * key_bytes);
    const size_t o_vb = up16(o_va + nd * 4);
    const size_t total = up16(o_vb + nd * 4);
    DM_TRY(ensure_arena(ctx, total));
    unsigned char* base = static_cast<unsigned char*>(ctx->arena);

    SortArgs a{};
    a.dtype = t;
    a.X = X; a.n = n; a.d = d; a.ldx = ldx;
    a.keys_a = base + o_ka; a.keys_b = base + o_kb;
    a.vals_a = reinterpret_cast<int32_t*>(base + o_va);
    a.vals_b = reinterpret_cast<int32_t*>(base + o_vb);
    a.hist = reinterpret_cast<uint32_t*>(base + o_hist);
    a.counters = reinterpret_cast<uint32_t*>(base + o_cnt);
    a.lookback = reinterpret_cast<uint32_t*>(base + o_lb);
    a.sorted_out = p->xs;
    a.perm_out = p->perm;
    a.err = ctx->err;

    DM_TRY_CUDA(cudaMemsetAsync(base, 0, zero_bytes, ctx->stream));
    {
        ProfScope ps(ctx, "sort_keygen_hist");
        DM_TRY_CUDA(sort_launch_keygen(a, ctx->stream, &ctx->launches));
    }

    // Read the histograms back: skip digit positions that are constant in
    // every column (a stable pass over a constant digit is the identity).
    if (ctx->host_hist_words < hist_words) {
        if (ctx->host_hist) cudaFreeHost(ctx->host_hist);
        ctx->host_hist = nullptr;
        ctx->host_hist_words = 0;
        DM_TRY_CUDA(cudaMallocHost(reinterpret_cast<void**>(&ctx->host_hist), hist_words * 4));
        ctx->host_hist_words = hist_words;
    }
    DM_TRY_CUDA(cudaMemcpyAsync(ctx->host_hist, a.hist, hist_words * 4, cudaMemcpyDeviceToHost,
                                ctx->stream));
    DM_TRY(take_device_error(ctx));   // synchronizes
    std::vector<int> passes;
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
    {
        ProfScope ps(ctx, "sort_onesweep");
        DM_TRY_CUDA(sort_launch_passes(a, passes.data(), (int)passes.size(), ctx->stream,
                                       &ctx->launches));
    }
    // R_i for the part of the query that is linear in the point (shift: the
    // median of each column, xs[c * n + n / 2]).
    DM_TRY(plan_alloc(p, (size_t)n * acc_size(t), &p->R));
    {
        ProfScope ps(ctx, "l1_rowsum");
        DM_TRY_CUDA(rowsum_launch(t, X, n, d, ldx,
                                  static_cast<unsigned char*>(p->xs) + (size_t)(n / 2) * dtype_size(t),
                                  n, p->R, ctx->stream, &ctx->launches));
    }
    return DM_OK;
}

// ------------------------------------------------------------- l2 prepare
dm_status prepare_l2(dm_ctx* ctx, dm_plan* p, const void* X, int64_t ldx) {
    const dm_dtype t = p->dtype;
    p->X = X;
    p->ldx = ldx;
    DM_TRY(plan_alloc(p, (size_t)p->d * dtype_size(t), &p->mu));
    L2PrepArgs a{};
    a.dtype = t;
    a.X = X; a.n = p->n; a.d = p->d; a.ldx = ldx;
    a.mu = p->mu; a.err = ctx->err;
    const int blocks = l2prep_blocks(a);
    DM_TRY(ensure_arena(ctx, (size_t)blocks * p->d * 8 + 16));
    a.partial = ctx->arena;
    {
        ProfScope ps(ctx, "l2_prepare");
        DM_TRY_CUDA(l2prep_launch(a, ctx->stream, &ctx->launches));
    }
    return DM_OK;
}

void free_plan_buffers(dm_plan* p) {
    plan_release(p);
    p->xs = nullptr; p->perm = nullptr; p->R = nullptr; p->mu = nullptr;
}

// ------------------------------------------------------------------ query
dm_status matmat_impl(dm_plan* p, const void* Z, int64_t k, int64_t ldz, void* out, int64_t ldo) {
    dm_ctx* ctx = p->ctx;
    const dm_dtype t = p->dtype;
    const int64_t n = p->n, d = p->d;

    if (p->metric == DM_L1) {
        // R^T Z, 1^T Z and the group-major copy of Z, then the sorted part
        // (Algorithm 2).
        DM_TRY(ensure_arena(ctx, l1_query_scratch_bytes(t, n, d, k, ctx->num_sms)));
        L1QueryArgs q{};
        q.dtype = t;
        q.xs = p->xs; q.perm = p->perm; q.n = n; q.d = d;
        q.R = p->R;
        q.mu = static_cast<unsigned char*>(p->xs) + (size_t)(n / 2) * dtype_size(t);
        q.mu_stride = n;
        q.Z = Z; q.k = k; q.ldz = ldz;
        q.out = out; q.ldo = ldo;
        q.scratch = ctx->arena;
        q.err = ctx->err;
        q.num_sms = ctx->num_sms;
        q.deterministic = ctx->deterministic;
        {
            ProfScope ps(ctx, "l1_prologue");
            DM_TRY_CUDA(l1_prologue_launch(q, ctx->stream, &ctx->launches));
        }
        {
            ProfScope ps(ctx, "l1_aggregate");
            DM_TRY_CUDA(l1_aggregate_launch(q, ctx->stream, &ctx->launches));
        }
        {
            ProfScope ps(ctx, "l1_query");
            DM_TRY_CUDA(l1_query_launch(q, ctx->stream, &ctx->launches));
        }
        if (!q.deterministic) {
            ProfScope ps(ctx, "l1_finalize");
            DM_TRY_CUDA(l1_finalize_launch(q, ctx->stream, &ctx->launches));
        }
        return DM_OK;
    }

    if (!reduce_supported(d, k)) return DM_ERR_UNSUPPORTED;
    ReduceArgs r{};
    r.dtype = t;
    r.n = n; r.d = d;
    r.Z = Z; r.k = k; r.ldz = ldz;
    r.num_sms = ctx->num_sms;
    const int blocks = reduce_blocks(r);
    const size_t o_res = up16((size_t)blocks * (d + 2) * k * 8);
    DM_TRY(ensure_arena(ctx, up16(o_res + (size_t)(d + 2) * k * 8)));
    unsigned char* base = static_cast<unsigned char*>(ctx->arena);
    r.partial = base;
    r.res = base + o_res;
    r.X = p->X; r.ldx = p->ldx; r.x_acc = false;
    r.mu = p->mu; r.mu_stride = 1;
    r.with_s = true;
    {
        ProfScope ps(ctx, "l2_reduce");
        DM_TRY_CUDA(reduce_launch(r, ctx->stream, &ctx->launches));
    }
    L2ApplyArgs ap{};
    ap.dtype = t;
    ap.X = p->X; ap.n = n; ap.d = d; ap.ldx = p->ldx;
    ap.mu = p->mu; ap.res = r.res; ap.k = k;
    ap.out = out; ap.ldo = ldo;
    ap.num_sms = ctx->num_sms;
    ProfScope ps(ctx, "l2_apply");
    DM_TRY_CUDA(l2apply_launch(ap, ctx->stream, &ctx->launches));
    return DM_OK;
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
    if (p->metric == DM_L1) {
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
        ProfScope ps(ctx, "grad_l1_transpose");
        DM_TRY_CUDA(grad_l1_launch(a, 3, ctx->stream, &ctx->launches));
        return DM_OK;
    }
    // squared l2: [X - mu, 1]^T [z_q, w_q] by the reduce kernel, then the closed form
    if (!reduce_supported(d, 2 * k)) return DM_ERR_UNSUPPORTED;
    ReduceArgs r{};
    r.dtype = t;
    r.n = n; r.d = d;
    r.k = 2 * k; r.ldz = 2 * k;
    r.num_sms = ctx->num_sms;
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
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->arena) cudaFree(ctx->arena);
    for (auto& b : ctx->pool) cudaFree(b.p);
    if (ctx->hx) cudaFree(ctx->hx);
    if (ctx->hz) cudaFree(ctx->hz);
    if (ctx->ho) cudaFree(ctx->ho);
    if (ctx->err) cudaFree(ctx->err);
    if (ctx->host_err) cudaFreeHost(ctx->host_err);
    if (ctx->host_hist) cudaFreeHost(ctx->host_hist);
    for (auto& p : ctx->pending) { cudaEventDestroy(p.start); cudaEventDestroy(p.stop); }
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    delete ctx;
}

dm_status dm_set_deterministic(dm_ctx* ctx, int on) {
    if (!ctx) return DM_ERR_INVALID_ARG;
    ctx->deterministic = on ? 1 : 0;
    return DM_OK;
}

dm_status dm_set_stream(dm_ctx* ctx, void* stream) {
    if (!ctx) return DM_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);   // pooled buffers may be in use on the old stream
    ctx->stream = static_cast<cudaStream_t>(stream);
    return DM_OK;
}

int64_t dm_launch_count(const dm_ctx* ctx) { return ctx ? ctx->launches : 0; }

dm_status dm_profile_enable(dm_ctx* ctx, int enable) {
    if (!ctx) return DM_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    DM_TRY(resolve_profile(ctx));
    ctx->stats.clear();
    ctx->profiling = enable != 0;
    return DM_OK;
}

dm_status dm_profile_read(dm_ctx* ctx, int max, int* count, char* names, int64_t* launches,
                          double* total_ms) {
    if (!ctx || !count || max < 0 || (max > 0 && (!names || !launches || !total_ms)))
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
    if (!ctx || !X || !valid_metric(metric) || !valid_dtype(dtype)) return DM_ERR_INVALID_ARG;
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
    const dm_status s = metric == DM_L1 ? prepare_l1(ctx, p, X, ldx) : prepare_l2(ctx, p, X, ldx);
    if (s != DM_OK) {
        cudaStreamSynchronize(ctx->stream);
        cudaGetLastError();
        free_plan_buffers(p);
        delete p;
        return s;
    }
    *plan = p;
    return DM_OK;
}

void dm_plan_destroy(dm_plan* p) {
    if (!p) return;
    DeviceGuard g(p->ctx->device);
    free_plan_buffers(p);   // stream-ordered reuse: no wait needed
    delete p;
}

dm_status dm_matmat(dm_plan* p, const void* Z, int64_t k, int64_t ldz, void* out, int64_t ldo) {
    if (!p || !Z || !out || k < 1 || ldz < k || ldo < k) return DM_ERR_INVALID_ARG;
    DeviceGuard g(p->ctx->device);
    return matmat_impl(p, Z, k, ldz, out, ldo);
}

dm_status dm_grad(dm_plan* p, const void* W, int64_t ldw, const void* Z, int64_t ldz, int64_t k,
                  void* G, int64_t ldg) {
    if (!p || !W || !Z || !G || k < 1 || k > 64 || ldw < k || ldz < k || ldg < p->d)
        return DM_ERR_INVALID_ARG;
    DeviceGuard g(p->ctx->device);
    return grad_impl(p, W, ldw, Z, ldz, k, G, ldg);
}

dm_status dm_matvec_l1(dm_plan* p, const void* z, void* out) {
    if (!p || p->metric != DM_L1) return DM_ERR_INVALID_ARG;
    return dm_matmat(p, z, 1, 1, out, 1);
}

dm_status dm_matvec_l2sq(dm_plan* p, const void* z, void* out) {
    if (!p || p->metric != DM_L2SQ) return DM_ERR_INVALID_ARG;
    return dm_matmat(p, z, 1, 1, out, 1);
}

dm_status dm_sync(dm_ctx* ctx) {
    if (!ctx) return DM_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return from_cuda(e);
    return take_device_error(ctx);
}

dm_status dm_plan_export(dm_plan* p, void* sorted_values, int32_t* perm) {
    if (!p || p->metric != DM_L1 || !sorted_values || !perm) return DM_ERR_INVALID_ARG;
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
    if (!ctx || !X || !Z || !out || !valid_metric(metric) || !valid_dtype(dtype)) return DM_ERR_INVALID_ARG;
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

dm_status dm_matmat_host(dm_ctx* ctx, dm_metric metric, dm_dtype dtype, const void* Xh, int64_t n,
                         int64_t d, int64_t ldx, const void* Zh, int64_t k, int64_t ldz,
                         void* outh, int64_t ldo) {
    if (!ctx || !Xh || !Zh || !outh || !valid_metric(metric) || !valid_dtype(dtype)) return DM_ERR_INVALID_ARG;
    if (n < 1 || n > kMaxN || d < 1 || ldx < d || k < 1 || ldz < k || ldo < k) return DM_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    const size_t es = dtype_size(dtype), os = out_size(dtype);
    DM_TRY(ensure_buffer(ctx, &ctx->hx, &ctx->hx_bytes, (size_t)n * d * es));
    DM_TRY(ensure_buffer(ctx, &ctx->hz, &ctx->hz_bytes, (size_t)n * k * es));
    DM_TRY(ensure_buffer(ctx, &ctx->ho, &ctx->ho_bytes, (size_t)n * k * os));
    DM_TRY_CUDA(cudaMemcpy2DAsync(ctx->hx, d * es, Xh, ldx * es, d * es, n, cudaMemcpyHostToDevice,
                                  ctx->stream));
    DM_TRY_CUDA(cudaMemcpy2DAsync(ctx->hz, k * es, Zh, ldz * es, k * es, n, cudaMemcpyHostToDevice,
                                  ctx->stream));
    dm_plan* p = nullptr;
    DM_TRY(dm_prepare(ctx, metric, dtype, ctx->hx, n, d, d, &p));
    dm_status s = dm_matmat(p, ctx->hz, k, k, ctx->ho, k);
    if (s == DM_OK) {
        cudaError_t e = cudaMemcpy2DAsync(outh, ldo * os, ctx->ho, k * os, k * os, n,
                                          cudaMemcpyDeviceToHost, ctx->stream);
        s = from_cuda(e);
    }
    if (s == DM_OK) s = dm_sync(ctx);
    dm_plan_destroy(p);
    return s;
}

}  // extern "C"
