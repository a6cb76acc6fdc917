// Gradient of L = sum_q w_q^T A(X) z_q with respect to the points X.
//
// The paper states no gradient.  By the chain rule on the definition of A,
//
//     dL/dx_i(c) = sum_q sum_j (w_iq z_jq + z_iq w_jq) phi'(x_i(c) - x_j(c)),
//
// phi' = sgn for l1 (sgn(0) = 0: tied coordinates contribute nothing) and
// phi'(t) = 2t for squared l2.
//
// l1 reuses the plan's sorted coordinates (Algorithm 1).  For the point at
// sorted position r of coordinate c, inside the tie group of positions a..b,
//
//     sum_j y_j sgn(x_r - x_j) = E_y(a) + I_y(b) - T_y,
//
// with E / I the exclusive / inclusive prefix sums of y in sorted order (as in
// Algorithm 2) and T the total.  Three passes over tiles of sorted positions:
//   grad_tile_kernel<aggregate>: per tile, the sums of z and w, the exclusive
//       prefix at the tile's last tie-group head and the inclusive prefix at
//       its first tie-group end, and the head / end positions;
//   grad_scan_kernel: per (coordinate, column), the tile prefixes, E at the
//       head of the group entering each tile and I at the end of the group
//       leaving it (forward and backward scans over the tiles);
//   grad_tile_kernel<eval>: in-tile scans, the head and end of every
//       position's tie group, and Gt[c, perm[r]] = sum_q w S_z + z S_w;
//   grad_transpose_kernel: Gt (d x n) into the caller's G (n x d).
// Tiles are claimed coordinate by coordinate, so the scattered writes of the
// evaluation pass fall in one column of Gt at a time (a few MB, held in L2
// until every sector is complete).  Only the per-tile scan works in FP64
// (the FP64 pipe is narrow); it hands the evaluation pass its per-tile
// constants already in the accumulation type.
//
// Squared l2: with u = 1^T y and Y = (X - mu)^T y for y = z_q, w_q (the
// reduce kernel on the packed columns), the sum over j expands to
//     dL/dx_i = 2 sum_q [(x_i - mu)(w_iq u_zq + z_iq u_wq) - w_iq Y_zq - z_iq Y_wq].
#include <algorithm>
#include <climits>
#include <cstring>

#include "dm_internal.h"

namespace dm {
namespace {

constexpr int kGT = 256;                // threads per block
constexpr int kGI = 4;                  // sorted positions per thread
constexpr int kGTile = kGT * kGI;       // sorted positions per tile
constexpr int kGW = kGT / 32;           // warps per block
constexpr int kNone = INT_MAX;

__device__ __forceinline__ float to_a(float v, float) { return v; }
__device__ __forceinline__ double to_a(double v, double) { return v; }
__device__ __forceinline__ long long to_a(int32_t v, long long) { return (long long)v; }

// ---------------------------------------------------------------- scans
// Exclusive prefix sum of one value per thread; t receives the block total.
template <class A>
__device__ __forceinline__ A block_excl_sum1(A v, A* ws, A& t) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    A iv = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const A a = __shfl_up_sync(0xffffffffu, iv, o);
        if (lane >= o) iv += a;
    }
    if (lane == 31) ws[warp] = iv;
    __syncthreads();
    if (warp == 0) {
        A x = lane < kGW ? ws[lane] : A(0);
#pragma unroll
        for (int o = 1; o < kGW; o <<= 1) {
            const A a = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += a;
        }
        ws[32 + lane] = x;
    }
    __syncthreads();
    const A b = warp > 0 ? ws[32 + warp - 1] : A(0);
    t = ws[32 + kGW - 1];
    __syncthreads();
    return b + iv - v;
}

// Maximum over the threads before this one (-1 if none); *all = block max.
__device__ __forceinline__ int block_excl_max(int v, int* ws, int* all) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int iv = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, iv, o);
        if (lane >= o) iv = max(iv, a);
    }
    if (lane == 31) ws[warp] = iv;
    __syncthreads();
    int before = -1;
    for (int w = 0; w < warp; ++w) before = max(before, ws[w]);
    int tot = -1;
    for (int w = 0; w < kGW; ++w) tot = max(tot, ws[w]);
    const int prev = __shfl_up_sync(0xffffffffu, iv, 1);
    const int ex = max(before, lane > 0 ? prev : -1);
    __syncthreads();
    *all = tot;
    return ex;
}

// Minimum over the threads after this one (kNone if none); *all = block min.
__device__ __forceinline__ int block_excl_suffix_min(int v, int* ws, int* all) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int iv = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_down_sync(0xffffffffu, iv, o);
        if (lane + o < 32) iv = min(iv, a);
    }
    if (lane == 0) ws[warp] = iv;
    __syncthreads();
    int after = kNone;
    for (int w = warp + 1; w < kGW; ++w) after = min(after, ws[w]);
    int tot = kNone;
    for (int w = 0; w < kGW; ++w) tot = min(tot, ws[w]);
    const int next = __shfl_down_sync(0xffffffffu, iv, 1);
    const int ex = min(after, lane < 31 ? next : kNone);
    __syncthreads();
    *all = tot;
    return ex;
}

// ---------------------------------------------------------------- kernels
template <dm_dtype DT>
struct GradParams {
    using V = typename Types<DT>::V;
    using Wide = typename Types<DT>::Wide;
    using Out = typename Types<DT>::Out;
    const V* xs; const int32_t* perm; int64_t n; int d;
    const V* P; int k;          // packed (z_q, w_q) pairs, n x 2k
    using Acc = typename Types<DT>::Acc;
    int64_t T;                  // tiles per coordinate
    int4* flags;                // d x T: first head, last head, first end, last end
    Acc* summ;                  // d x T x 2k x 3: sum, prefix at last head, at first end
    const Acc* cst;             // d x T x 2k x 4: E + I - T for (head, end) outside/inside
    Out* Gt;                    // d x n
    bool pvec;                  // 16-byte loads of P's row chunks
};

// In-tile inclusive prefixes in shared memory: one padding element per 32
// positions (a thread's positions are 4 apart; without it a warp's reads of
// them fall in 8 banks).
constexpr int kPadTile = kGTile + kGTile / 32;


// Which of this thread's items sits at tile position pos (-1: none).
__device__ __forceinline__ int own_item(int pos, int base) {
    const int j = pos - base;
    return (j >= 0 && j < kGI) ? j : -1;
}

// x[j][v] for a run-time j (register selects, no local memory).
template <class A, int N>
__device__ __forceinline__ A pick(const A (&x)[kGI][N], int j, int v) {
    A r = x[0][v];
#pragma unroll
    for (int i = 1; i < kGI; ++i) if (j == i) r = x[i][v];
    return r;
}
template <class A>
__device__ __forceinline__ A pick1(const A (&x)[kGI], int j) {
    A r = x[0];
#pragma unroll
    for (int i = 1; i < kGI; ++i) if (j == i) r = x[i];
    return r;
}

template <class V, bool VEC>
__device__ __forceinline__ void load_items(const V* __restrict__ src, int valid, int base, V* v) {
    if (VEC && base + kGI <= valid) {
        constexpr int E = 16 / (int)sizeof(V);
#pragma unroll
        for (int j = 0; j < kGI; j += E) {
            const uint4 raw = __ldg(reinterpret_cast<const uint4*>(src + base + j));
            memcpy(&v[j], &raw, 16);
        }
    } else {
#pragma unroll
        for (int j = 0; j < kGI; ++j) v[j] = base + j < valid ? src[base + j] : V(0);
    }
}

// Exclusive prefix sums over the block (thread order) of N values per
// thread.  ws: N * kGW entries, 16-byte aligned.
template <class A, int N>
__device__ __forceinline__ void block_excl_sumN(A (&v)[N], A* ws) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    A iv[N];
#pragma unroll
    for (int u = 0; u < N; ++u) iv[u] = v[u];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int u = 0; u < N; ++u) {
            const A t = __shfl_up_sync(0xffffffffu, iv[u], o);
            if (lane >= o) iv[u] += t;
        }
    }
    if (lane == 31) {
#pragma unroll
        for (int u = 0; u < N; ++u) ws[warp * N + u] = iv[u];
    }
    __syncthreads();
    A before[N];
#pragma unroll
    for (int u = 0; u < N; ++u) before[u] = A(0);
    for (int w = 0; w < warp; ++w) {
        if constexpr ((N * sizeof(A)) % 16 == 0) {
            A t[N];
#pragma unroll
            for (int h = 0; h < (int)(N * sizeof(A) / 16); ++h) {
                const uint4 raw = reinterpret_cast<const uint4*>(ws + w * N)[h];
                memcpy(reinterpret_cast<unsigned char*>(t) + 16 * h, &raw, 16);
            }
#pragma unroll
            for (int u = 0; u < N; ++u) before[u] += t[u];
        } else {
#pragma unroll
            for (int u = 0; u < N; ++u) before[u] += ws[w * N + u];
        }
    }
#pragma unroll
    for (int u = 0; u < N; ++u) v[u] = before[u] + iv[u] - v[u];
    __syncthreads();
}

// CQ consecutive elements of one row (zeros past the kq valid ones).
template <class V, class A, int CQ>
__device__ __forceinline__ void load_zrow(const V* __restrict__ z, int kq, bool vec, A (&y)[CQ]) {
    if (vec && kq == CQ) {
        V r[CQ];
        if constexpr (sizeof(V) * CQ == 16) {
            const uint4 raw = __ldg(reinterpret_cast<const uint4*>(z));
            memcpy(r, &raw, 16);
        } else {
            static_assert(sizeof(V) * CQ == 8, "row chunk of 8 or 16 bytes");
            const uint2 raw = __ldg(reinterpret_cast<const uint2*>(z));
            memcpy(r, &raw, 8);
        }
#pragma unroll
        for (int u = 0; u < CQ; ++u) y[u] = to_a(r[u], A());
    } else {
#pragma unroll
        for (int u = 0; u < CQ; ++u) y[u] = u < kq ? to_a(z[u], A()) : A(0);
    }
}

// NV: (z, w) values per row chunk -- 16 bytes of them, or one (z, w) pair
// when k = 1.
template <dm_dtype DT, bool EVAL, bool VEC, int NV>
__global__ void __launch_bounds__(kGT) grad_tile_kernel(GradParams<DT> p) {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    using Wide = typename Types<DT>::Wide;
    using Out = typename Types<DT>::Out;
    constexpr int GQ = NV / 2;                 // query columns per chunk
    __shared__ Acc Ip[EVAL ? NV : 1][EVAL ? kPadTile : 1];
    __shared__ Acc kc[EVAL ? NV * 4 : 1];      // the chunk's scan constants
    __shared__ __align__(16) Acc ws[NV * kGW];
    __shared__ int wsi[32];
    __shared__ int red[4];

    const int c = (int)(blockIdx.x / p.T);             // coordinate-major claim order
    const int64_t t = blockIdx.x - (int64_t)c * p.T;
    const int64_t ts = t * kGTile;
    const int valid = (int)min64(kGTile, p.n - ts);
    const int base = threadIdx.x * kGI;
    const V* xc = p.xs + (int64_t)c * p.n + ts;
    const int32_t* pc = p.perm + (int64_t)c * p.n + ts;

    V x[kGI];
    int32_t pi[kGI];
    load_items<V, VEC>(xc, valid, base, x);
    load_items<int32_t, VEC>(pc, valid, base, pi);
    const V prevv = (ts + base > 0 && base < valid) ? xc[base - 1] : x[0];
    const V nextv = (ts + base + kGI < p.n) ? xc[base + kGI] : x[kGI - 1];

    // Tie-group heads and ends (equal values, -0 and +0 included, are a tie).
    bool hd[kGI], en[kGI];
#pragma unroll
    for (int j = 0; j < kGI; ++j) {
        const bool in = base + j < valid;
        const int64_t r = ts + base + j;
        const V left = j > 0 ? x[j - 1] : prevv;
        const V right = j + 1 < kGI ? x[j + 1] : nextv;
        hd[j] = in && (r == 0 || x[j] != left);
        en[j] = in && (r == p.n - 1 || x[j] != right);
    }
    int lh = -1, fe = kNone;
#pragma unroll
    for (int j = 0; j < kGI; ++j) if (hd[j]) lh = base + j;
#pragma unroll
    for (int j = kGI - 1; j >= 0; --j) if (en[j]) fe = base + j;

    int a[kGI], b[kGI];
    int last_head, first_end;
    {
        int run = block_excl_max(lh, wsi, &last_head);
#pragma unroll
        for (int j = 0; j < kGI; ++j) { if (hd[j]) run = base + j; a[j] = run; }
        run = block_excl_suffix_min(fe, wsi, &first_end);
#pragma unroll
        for (int j = kGI - 1; j >= 0; --j) { if (en[j]) run = base + j; b[j] = run; }
    }
    if (!EVAL) {
        int fh = kNone, le = -1;
#pragma unroll
        for (int j = 0; j < kGI; ++j) {
            if (hd[j]) fh = min(fh, base + j);
            if (en[j]) le = max(le, base + j);
        }
        if (threadIdx.x == 0) { red[0] = kNone; red[1] = -1; }
        __syncthreads();
        if (fh != kNone) atomicMin(&red[0], fh);
        if (le >= 0) atomicMax(&red[1], le);
        __syncthreads();
        if (threadIdx.x == 0)
            p.flags[(int64_t)c * p.T + t] = make_int4(red[0], last_head, first_end, red[1]);
    }

    const int K2 = 2 * p.k;
    Acc g[kGI];
#pragma unroll
    for (int j = 0; j < kGI; ++j) g[j] = Acc(0);
    // the items holding the tile's last position, last head and first end
    // (three threads of the block store the tile sums)
    const int jv = own_item(valid - 1, base), jh = own_item(last_head, base), jf = own_item(first_end, base);
    const bool owner = threadIdx.x == 0 || jv >= 0 || jh >= 0 || jf >= 0;

    for (int q0 = 0; q0 < p.k; q0 += GQ) {
        const int kq = min(GQ, p.k - q0);
        // (z, w) of columns q0 .. q0 + GQ - 1, their in-thread inclusive
        // prefixes, then the block's exclusive offsets
        Acc y[kGI][NV], ip[kGI][NV], off[NV];
#pragma unroll
        for (int j = 0; j < kGI; ++j) {
            if (base + j < valid) {
                load_zrow<V, Acc, NV>(p.P + (int64_t)pi[j] * K2 + 2 * q0, 2 * kq, p.pvec, y[j]);
            } else {
#pragma unroll
                for (int v = 0; v < NV; ++v) y[j][v] = Acc(0);
            }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            Acc run = 0;
#pragma unroll
            for (int j = 0; j < kGI; ++j) { run += y[j][v]; ip[j][v] = run; }
            off[v] = run;
        }
        block_excl_sumN<Acc, NV>(off, ws);
#pragma unroll
        for (int j = 0; j < kGI; ++j)
#pragma unroll
            for (int v = 0; v < NV; ++v) ip[j][v] += off[v];

        const int64_t slot0 = ((int64_t)c * p.T + t) * K2 + 2 * q0;
        if (!EVAL) {
            // per (column, z or w): the sum, the exclusive prefix at the last
            // head, the inclusive prefix at the first end.  The tile sum is
            // the inclusive prefix at the tile's last position (not the block
            // total, which sums in another order): a group that runs to the
            // end of the tile then cancels exactly.  Stored in the
            // accumulation type (the values are formed in it): the scan over
            // tiles widens them as it reads, so this kernel issues no
            // conversions on the narrow FP64 pipe.
            if (owner) {
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    if (v >= 2 * kq) continue;
                    Acc* sm = p.summ + (slot0 + v) * 3;
                    if (threadIdx.x == 0) {
                        if (last_head < 0) sm[1] = 0;
                        if (first_end == kNone) sm[2] = 0;
                    }
                    if (jv >= 0) sm[0] = pick(ip, jv, v);
                    if (jh >= 0) sm[1] = pick(ip, jh, v) - pick(y, jh, v);
                    if (jf >= 0) sm[2] = pick(ip, jf, v);
                }
            }
        } else {
            const int pb = base + (base >> 5);   // a thread's 4 positions share one 32-group
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
                for (int j = 0; j < kGI; ++j) Ip[v][pb + j] = ip[j][v];
            // E(a) + I(b) - T with the parts that lie outside the tile taken
            // from the scan: (head outside, end outside), (outside, inside),
            // (inside, outside), (inside, inside)
            if (threadIdx.x < NV * 4)
                kc[threadIdx.x] = (threadIdx.x >> 2) < 2 * kq ? p.cst[slot0 * 4 + threadIdx.x] : Acc(0);
            __syncthreads();
#pragma unroll
            for (int j = 0; j < kGI; ++j) {
                if (base + j >= valid) continue;
                // a point alone in its tie group: both prefixes are this
                // thread's own (the exclusive one is the previous item's)
                const bool single = a[j] == base + j && b[j] == base + j;
                const bool ain = a[j] >= 0, bin = b[j] != kNone;
                const int sel = (ain ? 2 : 0) + (bin ? 1 : 0);
                const int ah = a[j] - 1 + ((a[j] - 1) >> 5), bh = b[j] + (b[j] >> 5);
#pragma unroll
                for (int u = 0; u < GQ; ++u) {
                    Acc Sz = kc[8 * u + sel], Sw = kc[8 * u + 4 + sel];
                    if (single) {
                        Sz += (j > 0 ? ip[j - 1][2 * u] : off[2 * u]) + ip[j][2 * u];
                        Sw += (j > 0 ? ip[j - 1][2 * u + 1] : off[2 * u + 1]) + ip[j][2 * u + 1];
                    } else {
                        if (ain && a[j] > 0) { Sz += Ip[2 * u][ah]; Sw += Ip[2 * u + 1][ah]; }
                        if (bin) { Sz += Ip[2 * u][bh]; Sw += Ip[2 * u + 1][bh]; }
                    }
                    g[j] += y[j][2 * u + 1] * Sz + y[j][2 * u] * Sw;
                }
            }
            // (Ip and kc are next written after the next chunk's block scan,
            // whose barriers order those writes after these reads)
        }
    }
    if (EVAL) {
#pragma unroll
        for (int j = 0; j < kGI; ++j)
            if (base + j < valid) p.Gt[(int64_t)c * p.n + pi[j]] = (Out)g[j];
    }
}

// ||x - y||_p^p for odd p (Theorem "odd_p"), on the same tiling: with
// x~ = x - median (translation invariance), for the point at sorted position r
// in the tie group a..b,
//     sum_j y_j |x~ - x~_j|^p = sum_s C(p, s) x~^(p-s) S_s,
//     S_s = E_s(a) + I_s(b) - T_s over the weights y (-x~)^s, s = 0..p
// (E, I, T as for the gradient; ties contribute nothing).  Query columns are
// taken CQ at a time (16 bytes of accumulator: one vector load of each
// point's row of Z), the weights two powers at a time: one block scan of
// 2 CQ values per pair.  Each coordinate's share of the CQ columns is added
// into out with one reduction per point.
template <dm_dtype DT>
struct OddParams {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    using Wide = typename Types<DT>::Wide;
    using Out = typename Types<DT>::Out;
    const V* xs; const int32_t* perm; int64_t n; int d;
    const V* Z; int64_t ldz; int k; int pw;   // pw: the odd power
    int64_t T;
    int4* flags;
    Acc* summ;                  // d x T x Q x 3, Q = k (pw + 1)
    const Acc* cst;             // d x T x Q x 4
    Out* out; int64_t ldo;
    bool zvec, ovec;            // vector loads of Z rows / reductions into out
    Acc coef[16];               // C(pw, s), s = 0..pw
};

template <dm_dtype DT>
struct OddCq { static constexpr int value = 16 / (int)sizeof(typename Types<DT>::Acc); };

__device__ __forceinline__ void out_add(float* p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void out_add(double* p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void out_add(long long* p, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}

template <class Out, int CQ>
__device__ __forceinline__ void add_orow(Out* o, int kq, bool vec, const Out (&g)[CQ]) {
    if constexpr (CQ == 4 && sizeof(Out) == 4) {
        if (vec && kq == CQ) {
            asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};"
                         :: "l"(o), "f"(g[0]), "f"(g[1]), "f"(g[2]), "f"(g[3]) : "memory");
            return;
        }
    }
#pragma unroll
    for (int u = 0; u < CQ; ++u)
        if (u < kq) out_add(o + u, g[u]);
}

// CQ: query columns per chunk.  The FP32 tile-sum pass fits 3 blocks per SM
// in registers; the evaluation pass (more state per column) runs 2.
template <dm_dtype DT, bool EVAL, bool VEC, int CQ>
__global__ void __launch_bounds__(kGT, (!EVAL && sizeof(typename Types<DT>::Acc) == 4) ? 3 : 2)
oddp_tile_kernel(OddParams<DT> p) {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    using Wide = typename Types<DT>::Wide;
    using Out = typename Types<DT>::Out;
    __shared__ Acc Ia[EVAL ? CQ : 1][EVAL ? kPadTile : 1];
    __shared__ Acc Ib[EVAL ? CQ : 1][EVAL ? kPadTile : 1];
    __shared__ Acc kc[EVAL ? CQ * 8 : 1];     // the pair's scan constants per column
    __shared__ __align__(16) Acc ws[2 * CQ * kGW];
    __shared__ int wsi[32];
    __shared__ int red[4];

    const int c = (int)(blockIdx.x / p.T);
    const int64_t t = blockIdx.x - (int64_t)c * p.T;
    const int64_t ts = t * kGTile;
    const int valid = (int)min64(kGTile, p.n - ts);
    const int base = threadIdx.x * kGI;
    const V* xc = p.xs + (int64_t)c * p.n + ts;
    const int32_t* pc = p.perm + (int64_t)c * p.n + ts;
    const Acc med = to_a(p.xs[(int64_t)c * p.n + p.n / 2], Acc());

    V x[kGI];
    int32_t pi[kGI];
    load_items<V, VEC>(xc, valid, base, x);
    load_items<int32_t, VEC>(pc, valid, base, pi);
    const V prevv = (ts + base > 0 && base < valid) ? xc[base - 1] : x[0];
    const V nextv = (ts + base + kGI < p.n) ? xc[base + kGI] : x[kGI - 1];

    bool hd[kGI], en[kGI];
#pragma unroll
    for (int j = 0; j < kGI; ++j) {
        const bool in = base + j < valid;
        const int64_t r = ts + base + j;
        const V left = j > 0 ? x[j - 1] : prevv;
        const V right = j + 1 < kGI ? x[j + 1] : nextv;
        hd[j] = in && (r == 0 || x[j] != left);
        en[j] = in && (r == p.n - 1 || x[j] != right);
    }
    int lh = -1, fe = kNone;
#pragma unroll
    for (int j = 0; j < kGI; ++j) if (hd[j]) lh = base + j;
#pragma unroll
    for (int j = kGI - 1; j >= 0; --j) if (en[j]) fe = base + j;
    int a[kGI], b[kGI];
    int last_head, first_end;
    {
        int run = block_excl_max(lh, wsi, &last_head);
#pragma unroll
        for (int j = 0; j < kGI; ++j) { if (hd[j]) run = base + j; a[j] = run; }
        run = block_excl_suffix_min(fe, wsi, &first_end);
#pragma unroll
        for (int j = kGI - 1; j >= 0; --j) { if (en[j]) run = base + j; b[j] = run; }
    }
    if (!EVAL) {
        int fh = kNone, le = -1;
#pragma unroll
        for (int j = 0; j < kGI; ++j) {
            if (hd[j]) fh = min(fh, base + j);
            if (en[j]) le = max(le, base + j);
        }
        if (threadIdx.x == 0) { red[0] = kNone; red[1] = -1; }
        __syncthreads();
        if (fh != kNone) atomicMin(&red[0], fh);
        if (le >= 0) atomicMax(&red[1], le);
        __syncthreads();
        if (threadIdx.x == 0)
            p.flags[(int64_t)c * p.T + t] = make_int4(red[0], last_head, first_end, red[1]);
    }

    const int P1 = p.pw + 1;
    const int Q = p.k * P1;
    Acc xt[kGI];
#pragma unroll
    for (int j = 0; j < kGI; ++j) xt[j] = base + j < valid ? to_a(x[j], Acc()) - med : Acc(0);
    const int jv = own_item(valid - 1, base), jh = own_item(last_head, base), jf = own_item(first_end, base);
    const bool owner = threadIdx.x == 0 || jv >= 0 || jh >= 0 || jf >= 0;

    for (int q0 = 0; q0 < p.k; q0 += CQ) {
        const int kq = min(CQ, p.k - q0);
        Acc y[kGI][CQ];
#pragma unroll
        for (int j = 0; j < kGI; ++j) {
            if (base + j < valid) {
                load_zrow<V, Acc, CQ>(p.Z + (int64_t)pi[j] * p.ldz + q0, kq, p.zvec, y[j]);
            } else {
#pragma unroll
                for (int u = 0; u < CQ; ++u) y[j][u] = Acc(0);
            }
        }
        Acc g[kGI][CQ];
#pragma unroll
        for (int j = 0; j < kGI; ++j)
#pragma unroll
            for (int u = 0; u < CQ; ++u) g[j][u] = Acc(0);
        Acc pwa[kGI];                          // (-x~)^s0
#pragma unroll
        for (int j = 0; j < kGI; ++j) pwa[j] = Acc(1);
        for (int s0 = 0; s0 < P1; s0 += 2) {
            // inclusive in-thread prefixes of y (-x~)^s0 and y (-x~)^(s0+1)
            Acc ia[kGI][CQ], ib[kGI][CQ];
            Acc off[2 * CQ];
#pragma unroll
            for (int u = 0; u < CQ; ++u) {
                Acc sa = 0, sb = 0;
#pragma unroll
                for (int j = 0; j < kGI; ++j) {
                    const Acc va = y[j][u] * pwa[j];
                    sa += va;
                    sb -= va * xt[j];
                    ia[j][u] = sa;
                    ib[j][u] = sb;
                }
                off[u] = sa;
                off[CQ + u] = sb;
            }
            block_excl_sumN<Acc, 2 * CQ>(off, ws);
#pragma unroll
            for (int j = 0; j < kGI; ++j)
#pragma unroll
                for (int u = 0; u < CQ; ++u) { ia[j][u] += off[u]; ib[j][u] += off[CQ + u]; }
            if (!EVAL) {
                if (owner) {
#pragma unroll
                    for (int u = 0; u < CQ; ++u) {
                        if (u >= kq) continue;
                        const int64_t slot = ((int64_t)c * p.T + t) * Q + (int64_t)(q0 + u) * P1 + s0;
                        Acc* sm = p.summ + slot * 3;
                        if (threadIdx.x == 0) {
                            if (last_head < 0) { sm[1] = 0; sm[4] = 0; }
                            if (first_end == kNone) { sm[2] = 0; sm[5] = 0; }
                        }
                        if (jv >= 0) { sm[0] = pick(ia, jv, u); sm[3] = pick(ib, jv, u); }
                        if (jh >= 0) {
                            const Acc va = pick(y, jh, u) * pick1(pwa, jh);
                            sm[1] = pick(ia, jh, u) - va;
                            sm[4] = pick(ib, jh, u) + va * pick1(xt, jh);
                        }
                        if (jf >= 0) { sm[2] = pick(ia, jf, u); sm[5] = pick(ib, jf, u); }
                    }
                }
            } else {
                const int pb = base + (base >> 5);   // a thread's 4 positions share one 32-group
#pragma unroll
                for (int u = 0; u < CQ; ++u)
#pragma unroll
                    for (int j = 0; j < kGI; ++j) { Ia[u][pb + j] = ia[j][u]; Ib[u][pb + j] = ib[j][u]; }
                if (threadIdx.x < CQ * 8) {
                    const int u = threadIdx.x >> 3;
                    kc[threadIdx.x] = u < kq ? p.cst[(((int64_t)c * p.T + t) * Q + (int64_t)(q0 + u) * P1 + s0) * 4 +
                                                     (threadIdx.x & 7)]
                                             : Acc(0);
                }
                __syncthreads();
                const Acc ca = p.coef[s0], cb = p.coef[s0 + 1];
#pragma unroll
                for (int j = 0; j < kGI; ++j) {
                    if (base + j >= valid) continue;
                    const bool ain = a[j] >= 0, bin = b[j] != kNone;
                    const int sel = (ain ? 2 : 0) + (bin ? 1 : 0);
                    // C(p, s) x~^(p - s) for s = s0 and s0 + 1
                    Acc e1 = 1;
                    for (int u = 0; u < p.pw - s0 - 1; ++u) e1 *= xt[j];
                    const Acc w0 = ca * e1 * xt[j], w1 = cb * e1;
                    const int ah = a[j] - 1 + ((a[j] - 1) >> 5), bh = b[j] + (b[j] >> 5);
#pragma unroll
                    for (int u = 0; u < CQ; ++u) {
                        Acc S0 = kc[u * 8 + sel], S1 = kc[u * 8 + 4 + sel];
                        if (ain && a[j] > 0) { S0 += Ia[u][ah]; S1 += Ib[u][ah]; }
                        if (bin) { S0 += Ia[u][bh]; S1 += Ib[u][bh]; }
                        g[j][u] += w0 * S0 + w1 * S1;
                    }
                }
                // (Ia, Ib and kc are next written after the next pair's block
                // scan, whose barriers order those writes after these reads)
            }
            // next pair: (-x~)^(s0 + 2)
#pragma unroll
            for (int j = 0; j < kGI; ++j) pwa[j] *= xt[j] * xt[j];
        }
        if (EVAL) {
#pragma unroll
            for (int j = 0; j < kGI; ++j) {
                if (base + j >= valid) continue;
                Out o[CQ];
#pragma unroll
                for (int u = 0; u < CQ; ++u) o[u] = (Out)g[j][u];
                add_orow<Out, CQ>(p.out + (int64_t)pi[j] * p.ldo + q0, kq, p.ovec, o);
            }
        }
    }
}

// One block per (coordinate, column, z or w): forward scan of the tile sums
// (tile prefixes, E at the head of the group entering each tile), then a
// backward scan (I at the end of the group leaving each tile).
template <class W, class A>
__global__ void __launch_bounds__(kGT) grad_scan_kernel(const int4* __restrict__ flags,
                                                        const A* __restrict__ summ, W* pre,
                                                        A* __restrict__ cst, int64_t n, int64_t T,
                                                        int K2) {
    __shared__ W vals[kGT];
    __shared__ W ws[64];
    __shared__ int wsi[32];
    const int c = blockIdx.x / K2;
    const int qy = blockIdx.x - c * K2;
    const int tid = threadIdx.x;
    W carry_tp = 0, carry_e = 0;
    for (int64_t c0 = 0; c0 < T; c0 += kGT) {
        const int64_t t = c0 + tid;
        const bool in = t < T;
        const int64_t slot = ((int64_t)c * T + t) * K2 + qy;
        const int4 f = in ? flags[(int64_t)c * T + t] : make_int4(kNone, -1, kNone, -1);
        const W sum = in ? (W)summ[slot * 3] : W(0);
        W chunk;
        const W tp = carry_tp + block_excl_sum1(sum, ws, chunk);
        const bool has_head = in && f.y >= 0;
        vals[tid] = tp + (in ? (W)summ[slot * 3 + 1] : W(0));
        int last;
        const int idx = block_excl_max(has_head ? tid : -1, wsi, &last);
        const W el = (in && f.x == 0) ? tp : (idx >= 0 ? vals[idx] : carry_e);
        if (in) { pre[slot * 3] = tp; pre[slot * 3 + 1] = el; }
        if (last >= 0) carry_e = vals[last];
        carry_tp += chunk;
        __syncthreads();
    }
    const W total = carry_tp;
    W carry_i = 0;
    for (int64_t c0 = ((T - 1) / kGT) * kGT; c0 >= 0; c0 -= kGT) {
        const int64_t t = c0 + tid;
        const bool in = t < T;
        const int64_t slot = ((int64_t)c * T + t) * K2 + qy;
        const int4 f = in ? flags[(int64_t)c * T + t] : make_int4(kNone, -1, kNone, -1);
        const W tp = in ? pre[slot * 3] : W(0);
        const bool has_end = in && f.z != kNone;
        vals[tid] = tp + (in ? (W)summ[slot * 3 + 2] : W(0));
        int first;
        const int idx = block_excl_suffix_min(has_end ? tid : kNone, wsi, &first);
        const int valid = in ? (int)min64(kGTile, n - t * kGTile) : 0;
        const bool end_at_last = in && f.w == valid - 1;
        const W ir = end_at_last ? tp + (W)summ[slot * 3] : (idx != kNone ? vals[idx] : carry_i);
        if (in) {
            const W el = pre[slot * 3 + 1];
            A* k4 = cst + slot * 4;
            k4[0] = (A)(el + ir - total);
            k4[1] = (A)(el + tp - total);
            k4[2] = (A)(tp + ir - total);
            k4[3] = (A)(2 * tp - total);
        }
        if (first != kNone) carry_i = vals[first];
        __syncthreads();
    }
}

// G (n x d, leading dimension ldg) = Gt^T (Gt: d x n), through 32 x 32 tiles
// in shared memory: coalesced reads of Gt rows and writes of G rows.  Each
// block moves two tiles along n, so every thread has 8 loads in flight.
template <class Out>
__global__ void __launch_bounds__(256) grad_transpose_kernel(const Out* __restrict__ Gt, int64_t n, int d,
                                                             Out* __restrict__ G, int64_t ldg) {
    __shared__ Out tile[2][32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 64;
    const int c0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int r = ty; r < 32; r += 8) {
            const int c = c0 + r;
            const int64_t i = i0 + 32 * h + tx;
            if (c < d && i < n) tile[h][r][tx] = Gt[(int64_t)c * n + i];
        }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int r = ty; r < 32; r += 8) {
            const int64_t i = i0 + 32 * h + r;
            const int c = c0 + tx;
            if (c < d && i < n) G[i * ldg + c] = tile[h][tx][r];
        }
}

// P[i, 2q] = Z[i, q], P[i, 2q + 1] = W[i, q].
template <class V>
__global__ void grad_pack_kernel(const V* __restrict__ W, int64_t ldw, const V* __restrict__ Z,
                                 int64_t ldz, int64_t n, int k, V* __restrict__ P) {
    const int64_t total = n * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / k;
        const int q = (int)(e - i * k);
        P[i * 2 * k + 2 * q] = Z[i * ldz + q];
        P[i * 2 * k + 2 * q + 1] = W[i * ldw + q];
    }
}

// Squared l2: one warp per row, lanes over the coordinates.
template <dm_dtype DT>
__global__ void __launch_bounds__(kGT)
grad_l2_apply_kernel(const typename Types<DT>::V* __restrict__ X, int64_t n, int d, int64_t ldx,
                     const typename Types<DT>::V* __restrict__ mu,
                     const typename Types<DT>::Wide* __restrict__ res,
                     const typename Types<DT>::V* __restrict__ P, int k,
                     typename Types<DT>::Out* __restrict__ G, int64_t ldg) {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    using Out = typename Types<DT>::Out;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int K2 = 2 * k;
    Acc* Y = reinterpret_cast<Acc*>(smem_raw);   // d x 2k: (X - mu)^T z_q, (X - mu)^T w_q
    Acc* u = Y + (size_t)d * K2;                 // 2k: 1^T z_q, 1^T w_q
    Acc* m = u + K2;                             // d
    for (int e = threadIdx.x; e < d * K2; e += blockDim.x) Y[e] = (Acc)res[e];
    for (int e = threadIdx.x; e < K2; e += blockDim.x) u[e] = (Acc)res[(size_t)d * K2 + e];
    for (int e = threadIdx.x; e < d; e += blockDim.x) m[e] = to_a(mu[e], Acc());
    __syncthreads();
    // U rows per warp step, every load of the step issued before the
    // arithmetic (enough bytes in flight to keep HBM busy).
    constexpr int U = 8;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i0 = gw * U; i0 < n; i0 += nw * U) {
        for (int c = lane; c - lane < d; c += 32) {
            Acc xc[U];
#pragma unroll
            for (int u2 = 0; u2 < U; ++u2) {
                const int64_t i = i0 + u2;
                xc[u2] = (i < n && c < d) ? to_a(X[i * ldx + c], Acc()) - m[c] : Acc(0);
            }
            Acc g[U];
#pragma unroll
            for (int u2 = 0; u2 < U; ++u2) g[u2] = 0;
            for (int q = 0; q < k; ++q) {
                const Acc yz = c < d ? Y[c * K2 + 2 * q] : Acc(0);
                const Acc yw = c < d ? Y[c * K2 + 2 * q + 1] : Acc(0);
#pragma unroll
                for (int u2 = 0; u2 < U; ++u2) {
                    const int64_t i = min64(i0 + u2, n - 1);
                    const Acc zq = to_a(P[i * K2 + 2 * q], Acc()), wq = to_a(P[i * K2 + 2 * q + 1], Acc());
                    g[u2] += xc[u2] * (wq * u[2 * q] + zq * u[2 * q + 1]) - wq * yz - zq * yw;
                }
            }
#pragma unroll
            for (int u2 = 0; u2 < U; ++u2) {
                const int64_t i = i0 + u2;
                if (i < n && c < d) G[i * ldg + c] = (Out)(2 * g[u2]);
            }
        }
    }
}

struct GradLayout {
    int64_t T;
    size_t p, flags, summ, pre, cst, gt, total;
};

constexpr size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

GradLayout grad_layout(dm_dtype t, int64_t n, int64_t d, int64_t k) {
    GradLayout L;
    L.T = (n + kGTile - 1) / kGTile;
    const size_t K2 = 2 * (size_t)k;
    L.p = 0;
    L.flags = al256(L.p + (size_t)n * K2 * dtype_size(t));
    L.summ = al256(L.flags + 16 * (size_t)(d * L.T));
    L.pre = al256(L.summ + 8 * 3 * K2 * (size_t)(d * L.T));
    L.cst = al256(L.pre + 8 * 3 * K2 * (size_t)(d * L.T));
    L.gt = al256(L.cst + 8 * 4 * K2 * (size_t)(d * L.T));
    L.total = al256(L.gt + out_size(t) * (size_t)n * (size_t)d);
    return L;
}

template <dm_dtype DT>
cudaError_t grad_pack_t(const GradArgs& a, cudaStream_t s, int64_t* launches) {
    using V = typename Types<DT>::V;
    const GradLayout L = grad_layout(a.dtype, a.n, a.d, a.k);
    V* P = reinterpret_cast<V*>(static_cast<unsigned char*>(a.scratch) + L.p);
    const int64_t total = a.n * a.k;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 8 * (int64_t)a.num_sms));
    grad_pack_kernel<V><<<blocks, 256, 0, s>>>(static_cast<const V*>(a.W), a.ldw,
                                               static_cast<const V*>(a.Z), a.ldz, a.n, (int)a.k, P);
    *launches += 1;
    return cudaGetLastError();
}

template <dm_dtype DT>
GradParams<DT> make_params(const GradArgs& a) {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    using Wide = typename Types<DT>::Wide;
    using Out = typename Types<DT>::Out;
    const GradLayout L = grad_layout(a.dtype, a.n, a.d, a.k);
    unsigned char* sc = static_cast<unsigned char*>(a.scratch);
    GradParams<DT> p;
    p.xs = static_cast<const V*>(a.xs);
    p.perm = a.perm;
    p.n = a.n;
    p.d = (int)a.d;
    p.P = reinterpret_cast<const V*>(sc + L.p);
    p.k = (int)a.k;
    p.T = L.T;
    p.flags = reinterpret_cast<int4*>(sc + L.flags);
    p.summ = reinterpret_cast<Acc*>(sc + L.summ);
    p.cst = reinterpret_cast<const Acc*>(sc + L.cst);
    p.Gt = reinterpret_cast<Out*>(sc + L.gt);
    p.pvec = (2 * a.k * (int64_t)sizeof(V)) % 16 == 0;   // P is 256-byte aligned in the scratch
    return p;
}

template <dm_dtype DT>
cudaError_t grad_l1_stage_t(const GradArgs& a, int stage, cudaStream_t s, int64_t* launches) {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    using Wide = typename Types<DT>::Wide;
    using Out = typename Types<DT>::Out;
    GradParams<DT> p = make_params<DT>(a);
    const GradLayout L = grad_layout(a.dtype, a.n, a.d, a.k);
    unsigned char* sc = static_cast<unsigned char*>(a.scratch);
    const int64_t blocks = a.d * L.T;
    if (blocks > INT_MAX) return cudaErrorInvalidConfiguration;
    // row chunks of 16 bytes, or of one (z, w) pair for a single column (its
    // rows of 2 sizeof(V) bytes are aligned to that size)
    constexpr int kNV = 16 / (int)sizeof(V);
    const bool narrow = a.k == 1;
    if (narrow) p.pvec = true;
    // 16-byte loads of the sorted column need every column start aligned
    const bool vec = (a.n % (16 / (int64_t)sizeof(V))) == 0 && (a.n % 4) == 0 &&
                     reinterpret_cast<uintptr_t>(a.xs) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(a.perm) % 16 == 0;
    if (stage == 0) {
        if (narrow) {
            if (vec) grad_tile_kernel<DT, false, true, 2><<<(unsigned)blocks, kGT, 0, s>>>(p);
            else grad_tile_kernel<DT, false, false, 2><<<(unsigned)blocks, kGT, 0, s>>>(p);
        } else {
            if (vec) grad_tile_kernel<DT, false, true, kNV><<<(unsigned)blocks, kGT, 0, s>>>(p);
            else grad_tile_kernel<DT, false, false, kNV><<<(unsigned)blocks, kGT, 0, s>>>(p);
        }
    } else if (stage == 1) {
        grad_scan_kernel<Wide, Acc><<<(unsigned)(a.d * 2 * a.k), kGT, 0, s>>>(
            p.flags, p.summ, reinterpret_cast<Wide*>(sc + L.pre), reinterpret_cast<Acc*>(sc + L.cst),
            a.n, L.T, (int)(2 * a.k));
    } else if (stage == 2) {
        if (narrow) {
            if (vec) grad_tile_kernel<DT, true, true, 2><<<(unsigned)blocks, kGT, 0, s>>>(p);
            else grad_tile_kernel<DT, true, false, 2><<<(unsigned)blocks, kGT, 0, s>>>(p);
        } else {
            if (vec) grad_tile_kernel<DT, true, true, kNV><<<(unsigned)blocks, kGT, 0, s>>>(p);
            else grad_tile_kernel<DT, true, false, kNV><<<(unsigned)blocks, kGT, 0, s>>>(p);
        }
    } else {
        const int64_t bx = (a.n + 63) / 64;
        if (bx > INT_MAX) return cudaErrorInvalidConfiguration;
        dim3 grid((unsigned)bx, (unsigned)((a.d + 31) / 32));
        grad_transpose_kernel<Out><<<grid, 256, 0, s>>>(p.Gt, a.n, (int)a.d, static_cast<Out*>(a.G), a.ldg);
    }
    *launches += 1;
    return cudaGetLastError();
}

template <dm_dtype DT>
cudaError_t grad_l2_apply_t(const GradArgs& a, cudaStream_t s, int64_t* launches) {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    using Wide = typename Types<DT>::Wide;
    using Out = typename Types<DT>::Out;
    const GradLayout L = grad_layout(a.dtype, a.n, a.d, a.k);
    const V* P = reinterpret_cast<const V*>(static_cast<unsigned char*>(a.scratch) + L.p);
    const size_t smem = sizeof(Acc) * ((size_t)a.d * 2 * a.k + 2 * a.k + a.d);
    auto kern = grad_l2_apply_kernel<DT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t warps = (a.n + 7) / 8;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((warps + kGW - 1) / kGW, 8 * (int64_t)a.num_sms));
    kern<<<blocks, kGT, smem, s>>>(static_cast<const V*>(a.X), a.n, (int)a.d, a.ldx,
                                   static_cast<const V*>(a.mu), static_cast<const Wide*>(a.res), P,
                                   (int)a.k, static_cast<Out*>(a.G), a.ldg);
    *launches += 1;
    return cudaGetLastError();
}

struct OddLayout {
    int64_t T, Q;
    size_t flags, summ, pre, cst, total;
};

OddLayout oddp_layout(int64_t n, int64_t d, int64_t k, int pw) {
    OddLayout L;
    L.T = (n + kGTile - 1) / kGTile;
    L.Q = k * (pw + 1);
    const size_t dt = (size_t)(d * L.T);
    L.flags = 0;
    L.summ = al256(16 * dt);
    L.pre = al256(L.summ + 8 * 3 * (size_t)L.Q * dt);
    L.cst = al256(L.pre + 8 * 3 * (size_t)L.Q * dt);
    L.total = al256(L.cst + 8 * 4 * (size_t)L.Q * dt);
    return L;
}

template <dm_dtype DT>
cudaError_t oddp_stage_t(const OddArgs& a, int stage, cudaStream_t s, int64_t* launches) {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    using Wide = typename Types<DT>::Wide;
    using Out = typename Types<DT>::Out;
    const OddLayout L = oddp_layout(a.n, a.d, a.k, a.p);
    unsigned char* sc = static_cast<unsigned char*>(a.scratch);
    OddParams<DT> p;
    p.xs = static_cast<const V*>(a.xs);
    p.perm = a.perm;
    p.n = a.n;
    p.d = (int)a.d;
    p.Z = static_cast<const V*>(a.Z);
    p.ldz = a.ldz;
    p.k = (int)a.k;
    p.pw = a.p;
    p.T = L.T;
    p.flags = reinterpret_cast<int4*>(sc + L.flags);
    p.summ = reinterpret_cast<Acc*>(sc + L.summ);
    p.cst = reinterpret_cast<const Acc*>(sc + L.cst);
    p.out = static_cast<Out*>(a.out);
    p.ldo = a.ldo;
    // 16 bytes of accumulator per chunk in both passes (2 FP32 columns per
    // chunk in the evaluation pass measured slower: twice the block scans)
    constexpr int CQ = OddCq<DT>::value;
    const int cq = CQ;
    const size_t zrow = sizeof(V) * cq;   // bytes of one vector load of a row chunk
    p.zvec = a.ldz % cq == 0 && reinterpret_cast<uintptr_t>(a.Z) % zrow == 0;
    p.ovec = a.ldo % cq == 0 && reinterpret_cast<uintptr_t>(a.out) % (sizeof(Out) * cq) == 0;
    long long cb = 1;
    for (int t = 0; t < 16; ++t) {
        p.coef[t] = t <= a.p ? (Acc)cb : Acc(0);
        if (t < a.p) cb = cb * (a.p - t) / (t + 1);
    }
    const int64_t blocks = a.d * L.T;
    if (blocks > INT_MAX || L.Q * a.d > INT_MAX) return cudaErrorInvalidConfiguration;
    const bool vec = (a.n % (16 / (int64_t)sizeof(V))) == 0 && (a.n % 4) == 0 &&
                     reinterpret_cast<uintptr_t>(a.xs) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(a.perm) % 16 == 0;
    if (stage == 0) {
        if (vec) oddp_tile_kernel<DT, false, true, CQ><<<(unsigned)blocks, kGT, 0, s>>>(p);
        else oddp_tile_kernel<DT, false, false, CQ><<<(unsigned)blocks, kGT, 0, s>>>(p);
    } else if (stage == 1) {
        grad_scan_kernel<Wide, Acc><<<(unsigned)(a.d * L.Q), kGT, 0, s>>>(
            p.flags, p.summ, reinterpret_cast<Wide*>(sc + L.pre), reinterpret_cast<Acc*>(sc + L.cst),
            a.n, L.T, (int)L.Q);
    } else {
        if (vec) oddp_tile_kernel<DT, true, true, CQ><<<(unsigned)blocks, kGT, 0, s>>>(p);
        else oddp_tile_kernel<DT, true, false, CQ><<<(unsigned)blocks, kGT, 0, s>>>(p);
    }
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace

size_t oddp_scratch_bytes(int64_t n, int64_t d, int64_t k, int p) {
    return oddp_layout(n, d, k, p).total;
}

cudaError_t oddp_launch(const OddArgs& a, int stage, cudaStream_t s, int64_t* launches) {
    switch (a.dtype) {
        case DM_F32: return oddp_stage_t<DM_F32>(a, stage, s, launches);
        case DM_F64: return oddp_stage_t<DM_F64>(a, stage, s, launches);
        default: return oddp_stage_t<DM_I32>(a, stage, s, launches);
    }
}

size_t grad_scratch_bytes(dm_dtype t, int64_t n, int64_t d, int64_t k) {
    return grad_layout(t, n, d, k).total;
}

const void* grad_packed(const GradArgs& a) {
    return static_cast<const unsigned char*>(a.scratch) + grad_layout(a.dtype, a.n, a.d, a.k).p;
}

cudaError_t grad_pack_launch(const GradArgs& a, cudaStream_t s, int64_t* launches) {
    switch (a.dtype) {
        case DM_F32: return grad_pack_t<DM_F32>(a, s, launches);
        case DM_F64: return grad_pack_t<DM_F64>(a, s, launches);
        default: return grad_pack_t<DM_I32>(a, s, launches);
    }
}

cudaError_t grad_l1_launch(const GradArgs& a, int stage, cudaStream_t s, int64_t* launches) {
    switch (a.dtype) {
        case DM_F32: return grad_l1_stage_t<DM_F32>(a, stage, s, launches);
        case DM_F64: return grad_l1_stage_t<DM_F64>(a, stage, s, launches);
        default: return grad_l1_stage_t<DM_I32>(a, stage, s, launches);
    }
}

cudaError_t grad_l2_apply_launch(const GradArgs& a, cudaStream_t s, int64_t* launches) {
    switch (a.dtype) {
        case DM_F32: return grad_l2_apply_t<DM_F32>(a, s, launches);
        case DM_F64: return grad_l2_apply_t<DM_F64>(a, s, launches);
        default: return grad_l2_apply_t<DM_I32>(a, s, launches);
    }
}

}  // namespace dm
