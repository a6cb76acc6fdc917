// Query of the l1 product (Algorithm 2, Section 2; Theorem "p=1").
//
// For coordinate c with sorted values xs_c and order perm_c, Algorithm 2 adds
// to point k at sorted position r
//     x_r (S3 - S4) + S2 - S1
//       = 2 (x_r P_z[r] - P_xz[r]) + (T_xz - x_r T_z),
// with P the exclusive prefix sums of z and x.z in sorted order (S3 and S1)
// and T their totals (S3 + S4 and S1 + S2).  The second term is linear in
// x_r, so its sum over the coordinates needs no sort:
//     sum_c (T_xz[c] - x_k(c) T_z) = R^T Z - R_k (1^T Z),  R_k = sum_c x_k(c)
// (any per-coordinate shift mu_c cancels; the plan uses each column's median
// and stores R_k = sum_c (x_k(c) - mu_c)).  So the query is
//     out[k,:] = R^T Z - R_k 1^T Z + sum_c 2 (x_r P_z[r] - P_xz[r]).
//
// Kernels, in launch order:
//
// l1_prologue (+ finalize): one pass over the query block computes R^T Z and
//   1^T Z (FP32 partial sums, added in FP64, fixed-order finalize) and writes
//   a column-group-major copy Zg[g][i][0:KC] of Z (KC = 8 FP32 columns = one
//   32-byte sector per row, or 4 when one group's copies outgrow L2; a
//   partial last group is zero-padded).
//
// The sorted part: the k columns are processed one group of KC at a time,
//   all coordinates of group g before group g+1, so the random-access working
//   set of a group -- the gathered rows of Zg[g] and the partial output
//   outg[g], n*KC elements each (32 + 32 MiB at n = 2^20) -- stays resident
//   in L2 while the sorted columns stream past it.  Work unit: a tile of
//   TILE_E consecutive sorted positions of one coordinate of one group,
//   claimed by one warp from an atomic counter (persistent CTAs whose warps
//   never wait on one another) and walked in 8 sub-tiles of SUB_E positions.
//   Per sub-tile:
//   A. each thread takes SEG_LEN consecutive positions: x - b (b = the tile's
//      first sorted value), the checked permutation and the gathered QW-wide
//      slices of the rows Zg[g][perm[r]];
//   B. in-tile exclusive prefix sums Lz, Lxz of z and (x - b) z (FP32 for
//      FP32 data): in-thread, then across the warp by shuffles, plus the
//      running sums of the tile's earlier sub-tiles (carried in registers);
//   C. from the tile's exclusive prefix Pt over the earlier tiles of its
//      (group, coordinate), two per-column constants formed in FP64 once per
//      tile:
//        alpha = Pt_z,   gamma = Pt_xz - (b - mu) Pt_z,
//      so that 2 (x_r P_z[r] - P_xz[r]) = 2 ((x_r - b)(alpha + Lz_r) - (gamma + Lxz_r)):
//      the large terms are combined in FP64 once per tile and each element
//      works on tile-local values;
//   D. the values are summed over the coordinates into a partial output.
//
// Kernels of the sorted part (reduce-then-scan):
//   l1_aggregate + l1_tile_scan form every tile's sums of z and (x - mu) z
//   (one warp per tile, 256-bit row loads) and their exclusive scan over the
//   tiles of each (group, coordinate) in FP64: Pt.
//   l1_query (claims in (group, coordinate, tile) order, the next
//   sub-tile's permutation and coordinates loaded while the current one is
//   evaluated) does steps A-D; a thread takes SEG_LEN consecutive positions
//   and one 16-byte slice (QW columns) of their rows, the rest of a row on
//   the adjacent lane.  No shared memory and no block barrier.
//   Step D, default mode: every value is added into the Acc-type outg with
//   vector reductions in L2 (no waits; the order of the d additions per
//   element varies from run to run); l1_finalize then writes
//   out = outg + R^T Z - R_k 1^T Z in the caller's layout.
//   Step D, ordered mode (dm_set_deterministic): a tile of coordinate c waits
//   (bounded spin) until every tile of coordinate c-1 of its group is done,
//   then adds its values into the FP64 partial output outw with plain loads
//   and stores, in coordinate order; the last coordinate writes out.
// Every wait is on tiles claimed earlier by running warps (a warp claims its
// next tile before finishing the current one, never before starting it): the
// unfinished tile claimed first waits on nothing unfinished, so no deadlock.
// Integer data run the same steps exactly in int64.
#include <algorithm>

#include "dm_internal.h"

namespace dm {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

template <dm_dtype DT, int KC>
struct QCfg {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    // Thread (seg, quad) owns QW adjacent columns (one 16-byte vector of a Zg
    // row, or the whole row when narrower) of SEG_LEN consecutive sorted
    // positions; a column group of KC columns is NQ = KC / QW threads wide.
    // The tile lives in registers: no shared-memory staging.
    static constexpr int QW = (16 / (int)sizeof(V)) < KC ? (16 / (int)sizeof(V)) : KC;
    static constexpr int NQ = KC / QW;
    static constexpr int SEGS = 32 / NQ;                       // segments per sub-tile (one warp)
    static constexpr int SEG_LEN = sizeof(Acc) == 8 ? 4 : 8;
    static constexpr int SUB_E = SEGS * SEG_LEN;               // sorted positions per sub-tile
    static constexpr int TILE_E = 8 * SUB_E;                   // sorted positions per tile
    static constexpr int NV = 2 * KC;                          // scanned quantities
    static_assert(KC % QW == 0, "tile shape");
};

template <class V, class Acc, class Wide>
struct QParams {
    const V* xs; const int32_t* perm; int64_t n; int d;
    const Acc* R;                     // R_k = sum_c (x_k(c) - mu_c)
    const V* Zg;                      // G x n x KC, group-major copy of Z
    int k;
    const Wide* res;                  // R^T Z (k), then 1^T Z (k)
    const V* mu; int64_t mu_stride;
    Acc* outg;                        // G x n x KC partial sums (L2-reduction mode)
    Wide* outw;                       // G x n x KC partial sums (ordered mode)
    void* out; int64_t ldo;
    uint32_t* counter; uint32_t* done;
    const Wide* pre;                  // G x d x T x 2KC exclusive tile prefixes
    uint32_t* err;
    int T, G;
    uint32_t spin_limit;              // rounds of the ordered mode's wait
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ float diff(float a, float b) { return a - b; }
__device__ __forceinline__ double diff(double a, double b) { return a - b; }
__device__ __forceinline__ long long diff(int32_t a, int32_t b) { return (long long)a - (long long)b; }

__device__ __forceinline__ float fmac(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmac(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ long long fmac(long long a, long long b, long long c) {
    return (long long)((unsigned long long)a * (unsigned long long)b + (unsigned long long)c);
}

__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ long long ldcg(const long long* p) { return __ldcg(p); }
__device__ __forceinline__ void stcg(float* p, float v) { __stcg(p, v); }
__device__ __forceinline__ void stcg(double* p, double v) { __stcg(p, v); }
__device__ __forceinline__ void stcg(long long* p, long long v) { __stcg(p, v); }

// N consecutive elements (N * sizeof(T) in {4, 8, 16, 32}) moved as vectors.
template <class T, int N>
__device__ __forceinline__ void ld_vec(const T* p, T (&v)[N]) {
    constexpr int B = N * (int)sizeof(T);
    if constexpr (B % 16 == 0) {
#pragma unroll
        for (int h = 0; h < B / 16; ++h) {
            const uint4 u = *reinterpret_cast<const uint4*>(reinterpret_cast<const char*>(p) + 16 * h);
            memcpy(reinterpret_cast<char*>(v) + 16 * h, &u, 16);
        }
    } else if constexpr (B == 8) {
        const uint2 u = *reinterpret_cast<const uint2*>(p);
        memcpy(v, &u, 8);
    } else {
#pragma unroll
        for (int q = 0; q < N; ++q) v[q] = p[q];
    }
}

template <class T, int N>
__device__ __forceinline__ void ldcg_vec(const T* p, T (&v)[N]) {
    constexpr int B = N * (int)sizeof(T);
    if constexpr (B % 16 == 0) {
#pragma unroll
        for (int h = 0; h < B / 16; ++h) {
            const uint4 u = __ldcg(reinterpret_cast<const uint4*>(reinterpret_cast<const char*>(p) + 16 * h));
            memcpy(reinterpret_cast<char*>(v) + 16 * h, &u, 16);
        }
    } else {
#pragma unroll
        for (int q = 0; q < N; ++q) v[q] = ldcg(p + q);
    }
}

template <class T, int N>
__device__ __forceinline__ void stcg_vec(T* p, const T (&v)[N]) {
    constexpr int B = N * (int)sizeof(T);
    if constexpr (B % 16 == 0) {
#pragma unroll
        for (int h = 0; h < B / 16; ++h) {
            uint4 u;
            memcpy(&u, reinterpret_cast<const char*>(v) + 16 * h, 16);
            __stcg(reinterpret_cast<uint4*>(reinterpret_cast<char*>(p) + 16 * h), u);
        }
    } else {
#pragma unroll
        for (int q = 0; q < N; ++q) stcg(p + q, v[q]);
    }
}

// One row of N elements (N * sizeof(T) == 32 bytes) in a single 256-bit
// global load; other sizes fall back to ld_vec.
template <class T, int N>
__device__ __forceinline__ void ld_row(const T* p, T (&v)[N]) {
    if constexpr (N * sizeof(T) == 32) {
        uint32_t r[8];
        asm volatile("ld.global.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                       "=r"(r[6]), "=r"(r[7])
                     : "l"(p));
        memcpy(v, r, 32);
    } else {
        ld_vec<T, N>(p, v);
    }
}

// Reductions in L2 (relaxed, gpu scope): vector form for FP32.
template <int N>
__device__ __forceinline__ void red_add(float* p, const float (&v)[N]) {
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int h = 0; h < N / 4; ++h)
            asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};"
                         :: "l"(p + 4 * h), "f"(v[4 * h]), "f"(v[4 * h + 1]), "f"(v[4 * h + 2]),
                            "f"(v[4 * h + 3]) : "memory");
    } else if constexpr (N == 2) {
        asm volatile("red.relaxed.gpu.global.add.v2.f32 [%0], {%1, %2};"
                     :: "l"(p), "f"(v[0]), "f"(v[1]) : "memory");
    } else {
#pragma unroll
        for (int q = 0; q < N; ++q) atomicAdd(p + q, v[q]);
    }
}
template <int N>
__device__ __forceinline__ void red_add(double* p, const double (&v)[N]) {
#pragma unroll
    for (int q = 0; q < N; ++q) atomicAdd(p + q, v[q]);
}
template <int N>
__device__ __forceinline__ void red_add(long long* p, const long long (&v)[N]) {
#pragma unroll
    for (int q = 0; q < N; ++q)
        atomicAdd(reinterpret_cast<unsigned long long*>(p + q), (unsigned long long)v[q]);
}

// Bounded wait until *p >= target (acquire).  Returns false on timeout.
__device__ __forceinline__ bool wait_geq(const uint32_t* p, uint32_t target, uint32_t* err,
                                         uint32_t spin_limit) {
    uint32_t spins = 0;
    while (ld_acquire(p) < target) {
        if (++spins > spin_limit) { set_error(err, kErrTimeout); return false; }
        __nanosleep(128);
    }
    return true;
}

// ---------------------------------------------------------------- kernel
template <dm_dtype DT, int KC, bool ORDERED>
__global__ void __launch_bounds__(kThreads)
l1_query_kernel(QParams<typename Types<DT>::V, typename Types<DT>::Acc, typename Types<DT>::Wide> p) {
    using Cfg = QCfg<DT, KC>;
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    using Wide = typename Types<DT>::Wide;
    using Out = typename Types<DT>::Out;
    constexpr int SEG_LEN = Cfg::SEG_LEN, SUB_E = Cfg::SUB_E, TILE_E = Cfg::TILE_E, NV = Cfg::NV;
    constexpr int QW = Cfg::QW, NQ = Cfg::NQ, SPW = Cfg::SEGS;
    constexpr unsigned kFull = 0xffffffffu;

    // Every warp works alone (no block barrier): it claims whole tiles from
    // the counter and walks each in sub-tiles of SUB_E positions, carrying
    // the running in-tile sums from one sub-tile to the next.
    const int lane = threadIdx.x & 31;
    const int quad = lane % NQ, seg = lane / NQ;
    const int col0 = quad * QW;                 // first column of this thread
    const int d = p.d, T = p.T, k = p.k;
    const uint32_t total_tiles = (uint32_t)p.G * (uint32_t)d * (uint32_t)T;
    const int i0 = seg * SEG_LEN;

    // The permutation and coordinates of the next sub-tile (of this tile or
    // of the next claimed one) are loaded while the current one is evaluated.
    int32_t pe[SEG_LEN];
    V xv[SEG_LEN];
    auto load_sub = [&](uint32_t claim, int s, int32_t (&pv)[SEG_LEN], V (&xw)[SEG_LEN]) {
        const int t = (int)(claim % (uint32_t)T);
        const int c = (int)((claim / (uint32_t)T) % (uint32_t)d);
        const int64_t e0 = (int64_t)t * TILE_E;
        const int ne = (int)min64(TILE_E, p.n - e0);
        const int64_t sbase = (int64_t)c * p.n + e0 + s * SUB_E + i0;
        const int lim = ne - s * SUB_E - i0;
#pragma unroll
        for (int i = 0; i < SEG_LEN; ++i) {
            pv[i] = -1;
            xw[i] = V(0);
            if (i < lim) { pv[i] = __ldcs(p.perm + sbase + i); xw[i] = __ldcs(p.xs + sbase + i); }
        }
    };
    uint32_t mine = 0;
    if (lane == 0) mine = atomicAdd(p.counter, 1u);
    uint32_t claim = __shfl_sync(kFull, mine, 0);
    if (claim < total_tiles) load_sub(claim, 0, pe, xv);
    bool bad = false;

    while (claim < total_tiles) {
        if (lane == 0) mine = atomicAdd(p.counter, 1u);     // the next tile
        const int t = (int)(claim % (uint32_t)T);
        const int c = (int)((claim / (uint32_t)T) % (uint32_t)d);
        const int g = (int)(claim / ((uint32_t)T * (uint32_t)d));
        const int64_t e0 = (int64_t)t * TILE_E;
        const int ne = (int)min64(TILE_E, p.n - e0);
        const int nsub = (ne + SUB_E - 1) / SUB_E;
        const int64_t sbase = (int64_t)c * p.n + e0;
        const V b = __ldcs(p.xs + sbase);
        // C. the tile's exclusive prefix Pt over the earlier tiles (from the
        // tile scan), this thread's columns -> alpha, gamma (formed in Wide)
        Acc al[QW], gm[QW];
        {
            const Wide* pr = p.pre + (((int64_t)g * d + c) * T + t) * NV;
            const Wide bm = (Wide)b - (Wide)p.mu[(int64_t)c * p.mu_stride];
#pragma unroll
            for (int q = 0; q < QW; ++q) {
                const Wide Pz = pr[col0 + q], Pxz = pr[KC + col0 + q];
                al[q] = (Acc)Pz;
                gm[q] = (Acc)(Pxz - bm * Pz);
            }
        }
        Acc Cz[QW], Cxz[QW];                    // in-tile sums of the earlier sub-tiles
#pragma unroll
        for (int q = 0; q < QW; ++q) { Cz[q] = 0; Cxz[q] = 0; }
        uint32_t next = 0;

        for (int s = 0; s < nsub; ++s) {
            const int lim = ne - s * SUB_E - i0;
            // A. this thread's positions: x - b, checked permutation, gathered columns
            Acc dx[SEG_LEN];
#pragma unroll
            for (int i = 0; i < SEG_LEN; ++i) {
                if (i < lim && (uint32_t)pe[i] >= (uint32_t)p.n) { bad = true; pe[i] = -1; }   // never for a valid plan
                dx[i] = i < lim ? diff(xv[i], b) : Acc(0);
            }
            V zv[SEG_LEN][QW];
            {
                const V* zg = p.Zg + (int64_t)g * p.n * KC + col0;
#pragma unroll
                for (int i = 0; i < SEG_LEN; ++i) {
                    if (pe[i] >= 0) ld_vec<V, QW>(zg + (int64_t)pe[i] * KC, zv[i]);
                    else {
#pragma unroll
                        for (int q = 0; q < QW; ++q) zv[i][q] = V(0);
                    }
                }
            }
            // B. exclusive in-tile prefix Lz, Lxz of this thread's segment:
            // in-thread sums, a shuffle scan over the warp's segments, plus
            // the carry of the earlier sub-tiles
            Acc Lz[QW], Lxz[QW];
#pragma unroll
            for (int q = 0; q < QW; ++q) {
                Acc sz = 0, sxz = 0;
#pragma unroll
                for (int i = 0; i < SEG_LEN; ++i) {
                    const Acc z = (Acc)zv[i][q];
                    sz += z;
                    sxz = fmac(dx[i], z, sxz);
                }
                Acc iz = sz, ixz = sxz;
#pragma unroll
                for (int o = 1; o < SPW; o <<= 1) {
                    const Acc a = __shfl_up_sync(kFull, iz, o * NQ);
                    const Acc bb = __shfl_up_sync(kFull, ixz, o * NQ);
                    if (lane >= o * NQ) { iz += a; ixz += bb; }
                }
                Lz[q] = Cz[q] + (iz - sz);
                Lxz[q] = Cxz[q] + (ixz - sxz);
            }
            // D. (ordered) coordinate order: wait for every tile of coordinate c-1
            if (ORDERED && s == 0) {
                if (c > 0 && lane == 0) wait_geq(p.done + (int64_t)g * d + c - 1, (uint32_t)T, p.err, p.spin_limit);
                __syncwarp();
            }
            int32_t pe_n[SEG_LEN];
            V xv_n[SEG_LEN];
            if (s + 1 < nsub) {
                load_sub(claim, s + 1, pe_n, xv_n);
            } else {
                next = __shfl_sync(kFull, mine, 0);
                if (next < total_tiles) load_sub(next, 0, pe_n, xv_n);
            }

            // E. evaluate and accumulate
            if constexpr (!ORDERED) {
                // every value added into outg with a vector reduction in L2
                Acc* og = p.outg + (int64_t)g * p.n * KC + col0;
#pragma unroll
                for (int i = 0; i < SEG_LEN; ++i) {
                    Acc val[QW];
#pragma unroll
                    for (int q = 0; q < QW; ++q) {
                        val[q] = Acc(2) * fmac(dx[i], al[q] + Lz[q], -(gm[q] + Lxz[q]));
                        const Acc z = (Acc)zv[i][q];
                        Lz[q] += z;
                        Lxz[q] = fmac(dx[i], z, Lxz[q]);
                    }
                    if (pe[i] >= 0) red_add<QW>(og + (int64_t)pe[i] * KC, val);
                }
            } else {
                // Wide-type partial sums: the sum over the coordinates runs in
                // the Wide type (FP64 for FP32 data), each term added once
                const bool first = c == 0, final_ = c == d - 1;
                const int kg = min(KC, k - g * KC);
                Wide* ow = p.outw + (int64_t)g * p.n * KC + col0;
                Out* oc = static_cast<Out*>(p.out) + (int64_t)g * KC + col0;
                Wide old[SEG_LEN][QW];
#pragma unroll
                for (int i = 0; i < SEG_LEN; ++i) {
                    if (pe[i] >= 0 && !first) {
                        ldcg_vec<Wide, QW>(ow + (int64_t)pe[i] * KC, old[i]);
                    } else if (pe[i] >= 0) {
                        // coordinate 0 starts from R^T Z - R_k 1^T Z
                        const Wide Rk = (Wide)p.R[pe[i]];
#pragma unroll
                        for (int q = 0; q < QW; ++q) {
                            const int gc = g * KC + col0 + q;
                            old[i][q] = gc < k ? p.res[gc] - Rk * p.res[k + gc] : Wide(0);
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < QW; ++q) old[i][q] = 0;
                    }
                }
#pragma unroll
                for (int i = 0; i < SEG_LEN; ++i) {
                    Wide sum[QW];
#pragma unroll
                    for (int q = 0; q < QW; ++q) {
                        const Acc v = fmac(dx[i], al[q] + Lz[q], -(gm[q] + Lxz[q]));
                        sum[q] = old[i][q] + Wide(2) * (Wide)v;
                        const Acc z = (Acc)zv[i][q];
                        Lz[q] += z;
                        Lxz[q] = fmac(dx[i], z, Lxz[q]);
                    }
                    if (pe[i] >= 0) {
                        if (!final_) {
                            stcg_vec<Wide, QW>(ow + (int64_t)pe[i] * KC, sum);
                        } else {
#pragma unroll
                            for (int q = 0; q < QW; ++q)
                                if (col0 + q < kg) stcg(oc + (int64_t)pe[i] * p.ldo + q, (Out)sum[q]);
                        }
                    }
                }
            }
            // the running sums through this sub-tile, from its last segment
#pragma unroll
            for (int q = 0; q < QW; ++q) {
                Cz[q] = __shfl_sync(kFull, Lz[q], (SPW - 1) * NQ + quad);
                Cxz[q] = __shfl_sync(kFull, Lxz[q], (SPW - 1) * NQ + quad);
            }
#pragma unroll
            for (int i = 0; i < SEG_LEN; ++i) { pe[i] = pe_n[i]; xv[i] = xv_n[i]; }
        }
        if (ORDERED) {
            // F. this tile's values are in place before it is counted
            __threadfence();
            __syncwarp();
            if (lane == 0) red_release_add(p.done + (int64_t)g * d + c, 1u);
        }
        claim = next;
    }
    if (bad) set_error(p.err, kErrInternal);
}

// Tile aggregates (the reduce half of reduce-then-scan): one warp per tile
// of the query kernel's tiling, sum_r z[perm[r]] and sum_r (x_r - mu) z[perm[r]]
// over the tile, formed as (b - mu) sum z + sum (x - b) z with b the tile's
// first sorted value (FP32 partial sums per lane, warp tree, FP64 frame
// shift).  No shared memory and no barriers: a pure stream of loads.
// FP32 with 8-column groups: four CTAs per SM (64 registers) measured 4%
// faster than three; with 4-column groups the same bound made it 43% slower.
template <dm_dtype DT, int KC>
__global__ void __launch_bounds__(kThreads, DT == DM_F32 && KC == 8 ? 4 : 1)
l1_aggregate_kernel(const typename Types<DT>::V* __restrict__ xs, const int32_t* __restrict__ perm,
                    int64_t n, int d, const typename Types<DT>::V* __restrict__ Zg,
                    const typename Types<DT>::V* __restrict__ mu, int64_t mu_stride,
                    typename Types<DT>::Wide* __restrict__ agg, int T, int G, uint32_t* err) {
    using Cfg = QCfg<DT, KC>;
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    using Wide = typename Types<DT>::Wide;
    constexpr int TILE_E = Cfg::TILE_E, NV = Cfg::NV, U = 4;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * kThreads) >> 5;
    const int64_t total = (int64_t)G * d * T;
    for (int64_t tile = gw; tile < total; tile += nw) {
        const int t = (int)(tile % T);
        const int c = (int)((tile / T) % d);
        const int g = (int)(tile / ((int64_t)T * d));
        const int64_t e0 = (int64_t)t * TILE_E;
        const int ne = (int)min64(TILE_E, n - e0);
        const int64_t sbase = (int64_t)c * n + e0;
        const V b = xs[sbase];
        const V* zg = Zg + (int64_t)g * n * KC;
        Acc sz[KC], sxz[KC];
#pragma unroll
        for (int q = 0; q < KC; ++q) { sz[q] = 0; sxz[q] = 0; }
        bool bad = false;
        // Software pipeline: the permutation of block j+1 is loaded while the
        // rows of block j are gathered and summed.
        int32_t pe[U];
        Acc dx[U];
        auto load_block = [&](int e, int32_t (&pv)[U], Acc (&dv)[U]) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int ee = e + 32 * u;
                pv[u] = -1;
                dv[u] = 0;
                if (ee < ne) { pv[u] = __ldcs(perm + sbase + ee); dv[u] = diff(__ldcs(xs + sbase + ee), b); }
                if (ee < ne && (uint32_t)pv[u] >= (uint32_t)n) { bad = true; pv[u] = -1; }
            }
        };
        load_block(lane, pe, dx);
        for (int e = lane; e < ne; e += 32 * U) {
            V zv[U][KC];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (pe[u] >= 0) ld_row<V, KC>(zg + (int64_t)pe[u] * KC, zv[u]);
                else {
#pragma unroll
                    for (int q = 0; q < KC; ++q) zv[u][q] = V(0);
                }
            }
            int32_t pe_n[U];
            Acc dx_n[U];
            load_block(e + 32 * U, pe_n, dx_n);
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int q = 0; q < KC; ++q) {
                    const Acc z = (Acc)zv[u][q];
                    sz[q] += z;
                    sxz[q] = fmac(dx[u], z, sxz[q]);
                }
#pragma unroll
            for (int u = 0; u < U; ++u) { pe[u] = pe_n[u]; dx[u] = dx_n[u]; }
        }
        if (bad) set_error(err, kErrInternal);
        // Reduce-scatter over the warp: each halving step trades half of the
        // NV sums with the lane o apart, after which lane L holds the warp
        // total of quantity L >> (5 - H) (sums of z first, then of (x - b) z).
        constexpr int H = NV == 16 ? 4 : NV == 8 ? 3 : NV == 4 ? 2 : 1;
        static_assert((1 << H) == NV, "NV is a power of two up to 16");
        Acc v[NV];
#pragma unroll
        for (int q = 0; q < KC; ++q) { v[q] = sz[q]; v[KC + q] = sxz[q]; }
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const int o = 16 >> h, half = NV >> (h + 1);
            const bool up = lane & o;
#pragma unroll
            for (int j = 0; j < half; ++j) {
                const Acc keep = up ? v[j + half] : v[j];
                const Acc send = up ? v[j] : v[j + half];
                v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
        Acc tot = v[0];
#pragma unroll
        for (int o = 16 >> H; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
        const int qi = lane >> (5 - H);                       // the quantity this lane holds
        const Acc tz = __shfl_sync(0xffffffffu, tot, (qi % KC) << (5 - H));   // sum z of its column
        if ((lane & ((1 << (5 - H)) - 1)) == 0) {
            Wide mine;
            if (qi < KC) {
                mine = (Wide)tot;
            } else {
                const Wide bm = (Wide)b - (Wide)mu[(int64_t)c * mu_stride];
                mine = bm * (Wide)tz + (Wide)tot;
            }
            agg[tile * NV + qi] = mine;
        }
    }
}

// Exclusive scan of the tile aggregates of each (group, coordinate) segment,
// in place (the scan half): thread (value v, chunk ch) sums its chunk of
// tiles, chunk bases are added in chunk order, then the chunk is rewritten
// as running prefixes.  Fixed order: reproducible.
template <class Wide>
__global__ void __launch_bounds__(kThreads)
l1_tile_scan_kernel(Wide* __restrict__ agg, int T, int NV) {
    __shared__ Wide cs[kThreads];
    Wide* a = agg + (int64_t)blockIdx.x * T * NV;
    const int CH = kThreads / NV;
    const int v = threadIdx.x % NV, ch = threadIdx.x / NV;
    const int per = (T + CH - 1) / CH;
    const int t0 = ch < CH ? min(T, ch * per) : T, t1 = ch < CH ? min(T, t0 + per) : T;
    Wide sum = 0;
    for (int t = t0; t < t1; ++t) sum += a[(int64_t)t * NV + v];
    cs[threadIdx.x] = sum;
    __syncthreads();
    Wide run = 0;
    for (int j = 0; j < ch && j < CH; ++j) run += cs[j * NV + v];
    for (int t = t0; t < t1; ++t) {
        const Wide x = a[(int64_t)t * NV + v];
        a[(int64_t)t * NV + v] = run;
        run += x;
    }
}

// out[i, j] = outg[j / KC][i][j % KC] + R^T Z[j] - R_i 1^T Z[j]  (atomic mode).
// Thread per (row, VEC adjacent columns); VEC = 4 needs k % 4 == 0, ldo % 4 == 0
// and an aligned out.
template <dm_dtype DT, int KC, int VEC>
__global__ void __launch_bounds__(kThreads)
l1_finalize_kernel(const typename Types<DT>::Acc* __restrict__ outg,
                   const typename Types<DT>::Acc* __restrict__ R,
                   const typename Types<DT>::Wide* __restrict__ res, int64_t n, int k,
                   typename Types<DT>::Out* __restrict__ out, int64_t ldo) {
    using Acc = typename Types<DT>::Acc;
    using Out = typename Types<DT>::Out;
    // The per-column terms R^T Z and 1^T Z, converted once per block (a
    // conversion from the wide type is an FP64-pipe instruction).
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Acc* rs = reinterpret_cast<Acc*>(smem_raw);      // [0, k): R^T Z, [k, 2k): 1^T Z
    for (int j = threadIdx.x; j < 2 * k; j += kThreads) rs[j] = (Acc)res[j];
    __syncthreads();
    const int nv = (k + VEC - 1) / VEC;
    const int64_t total = n * nv;
    for (int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * kThreads) {
        const int64_t i = idx / nv;
        const int j0 = (int)(idx - i * nv) * VEC;
        const Acc Ri = R[i];
        Acc v[VEC];
        if constexpr (VEC == 4 && KC % 4 == 0) {
            ldcg_vec<Acc, 4>(outg + ((int64_t)(j0 / KC) * n + i) * KC + (j0 % KC), v);
        } else {
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
                const int j = j0 + q;
                v[q] = j < k ? __ldcs(outg + ((int64_t)(j / KC) * n + i) * KC + (j % KC)) : Acc(0);
            }
        }
        Out o[VEC];
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
            const int j = min(j0 + q, k - 1);
            o[q] = (Out)(v[q] + (rs[j] - Ri * rs[k + j]));
        }
        if constexpr (VEC == 4 && sizeof(Out) == 4) {
            *reinterpret_cast<float4*>(out + i * ldo + j0) = make_float4(o[0], o[1], o[2], o[3]);
        } else {
#pragma unroll
            for (int q = 0; q < VEC; ++q)
                if (j0 + q < k) out[i * ldo + j0 + q] = o[q];
        }
    }
}

// ---------------------------------------------------------------- prologue
// R^T Z and 1^T Z (per-block partials) and the group-major copy Zg of Z.
// Thread (row group rg, column vector jv): VEC adjacent padded columns
// j = jv*VEC .. +VEC of rows rg, rg + RGS, ..., U rows per step with all loads
// issued first.  VEC = 4 needs k % 4 == 0, ldz % 4 == 0 and an aligned Z.
template <dm_dtype DT, int KC, int VEC>
__global__ void __launch_bounds__(kThreads)
l1_prologue_kernel(const typename Types<DT>::V* __restrict__ Z, int64_t n, int k, int64_t ldz,
                   const typename Types<DT>::Acc* __restrict__ R,
                   typename Types<DT>::V* __restrict__ Zg, int JW,
                   typename Types<DT>::Wide* __restrict__ partial, int64_t rows_per_block) {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    using Wide = typename Types<DT>::Wide;
    constexpr int U = 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Wide* red = reinterpret_cast<Wide*>(smem_raw);      // [RGS][2][JC]
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min64(n, r0 + rows_per_block);
    const int NJV = JW / VEC;                              // column vectors per row
    const int JC = NJV < kThreads ? NJV : kThreads;        // vectors per sweep
    const int RGS = kThreads / JC;
    const int rg = threadIdx.x / JC, jl = threadIdx.x % JC;
    for (int jb = 0; jb < NJV; jb += JC) {
        const int jv = jb + jl;
        const bool active = rg < RGS && jv < NJV;
        const int j0 = jv * VEC;
        const int g = j0 / KC, q0 = j0 % KC;
        Wide wu[VEC], wr[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) { wu[v] = 0; wr[v] = 0; }
        if (active) {
            Acc cu[VEC], cr[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) { cu[v] = 0; cr[v] = 0; }
            int cnt = 0;
            for (int64_t r = r0 + rg; r < r1; r += (int64_t)RGS * U) {
                V z[U][VEC];
                Acc rr[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t ru = r + (int64_t)u * RGS;
                    rr[u] = ru < r1 ? R[ru] : Acc(0);
                    if constexpr (VEC == 4) {
                        // k % 4 == 0: a vector is wholly inside [0, k) or wholly padding
                        if (ru < r1 && j0 < k) ld_vec<V, 4>(Z + ru * ldz + j0, z[u]);
                        else {
#pragma unroll
                            for (int v = 0; v < VEC; ++v) z[u][v] = V(0);
                        }
                    } else {
#pragma unroll
                        for (int v = 0; v < VEC; ++v) z[u][v] = (ru < r1 && j0 + v < k) ? Z[ru * ldz + j0 + v] : V(0);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t ru = r + (int64_t)u * RGS;
                    if (ru >= r1) continue;
                    V* dst = Zg + ((int64_t)g * n + ru) * KC + q0;
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        dst[v] = z[u][v];
                        cu[v] += (Acc)z[u][v];
                        cr[v] += rr[u] * (Acc)z[u][v];
                    }
                }
                if (++cnt == 32) {
#pragma unroll
                    for (int v = 0; v < VEC; ++v) { wu[v] += (Wide)cu[v]; wr[v] += (Wide)cr[v]; cu[v] = 0; cr[v] = 0; }
                    cnt = 0;
                }
            }
#pragma unroll
            for (int v = 0; v < VEC; ++v) { wu[v] += (Wide)cu[v]; wr[v] += (Wide)cr[v]; }
        }
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            __syncthreads();
            if (rg < RGS) { red[(rg * 2 + 0) * JC + jl] = wu[v]; red[(rg * 2 + 1) * JC + jl] = wr[v]; }
            __syncthreads();
            const int j = j0 + v;
            if (rg == 0 && jv < NJV && j < k) {
                Wide tu = 0, tr = 0;
                for (int t = 0; t < RGS; ++t) { tu += red[(t * 2) * JC + jl]; tr += red[(t * 2 + 1) * JC + jl]; }
                Wide* out = partial + (int64_t)blockIdx.x * 2 * k;
                out[j] = tr;       // R^T Z
                out[k + j] = tu;   // 1^T Z
            }
        }
    }
}

// One warp per result entry: lanes stride over the block partials, then a
// fixed-order warp tree (reproducible).
template <class Wide>
__global__ void l1_prologue_finalize(const Wide* __restrict__ partial, int blocks, int k2,
                                     Wide* __restrict__ res) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= k2) return;
    Wide t = 0;
    for (int b = lane; b < blocks; b += 32) t += partial[(int64_t)b * k2 + w];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) res[w] = t;
}

int full_kc(dm_dtype t) { return t == DM_F64 ? 4 : 8; }

// Column-group width: one 32-byte sector of a Zg row (8 FP32 / 4 FP64
// columns), or half of it when one group's Zg and outg copies
// ((element + accumulator) n kc bytes) exceed what L2 keeps: the random row
// gathers and reductions then go to DRAM, and narrower rows halve that
// working set at the cost of one more pass over the sorted data per group
// (measured at n = 2^22, d = 16: k = 8 / 16 / 40 ran 13 / 11 / 1% faster).
constexpr size_t kGroupL2Bytes = size_t(96) << 20;

int pick_kc(dm_dtype t, int64_t n, int64_t k) {
    const int full = full_kc(t);
    const size_t row = dtype_size(t) + (t == DM_F32 ? 4 : 8);
    const int cap = (size_t)n * row * full > kGroupL2Bytes ? full / 2 : full;
    if (k >= cap) return cap;
    int kc = 1;
    while (kc < k) kc <<= 1;
    return kc;
}

template <dm_dtype DT>
int tile_elems_rt(int kc) {
    switch (kc) {
        case 1: return QCfg<DT, 1>::TILE_E;
        case 2: return QCfg<DT, 2>::TILE_E;
        case 4: return QCfg<DT, 4>::TILE_E;
        default: return QCfg<DT, DT == DM_F64 ? 4 : 8>::TILE_E;
    }
}

int tile_elems_dt(dm_dtype t, int kc) {
    switch (t) {
        case DM_F32: return tile_elems_rt<DM_F32>(kc);
        case DM_F64: return tile_elems_rt<DM_F64>(kc);
        default: return tile_elems_rt<DM_I32>(kc);
    }
}

int prologue_blocks(int64_t n, int num_sms) {
    const int64_t want = (n + 2047) / 2048;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, 2 * (int64_t)std::max(num_sms, 1)));
}

struct ScratchLayout {
    int kc; int64_t G, T;
    size_t counter, done, memset_bytes, pre, partial, res, zg, outg, total;
};

// Every region starts on a 256-byte boundary (the arena itself comes from
// cudaMalloc): the 256-bit row loads from Zg need 32-byte alignment.
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

ScratchLayout scratch_layout(dm_dtype t, int64_t n, int64_t d, int64_t k, int num_sms) {
    ScratchLayout L;
    L.kc = pick_kc(t, n, k);
    L.G = (k + L.kc - 1) / L.kc;
    const int64_t tile = tile_elems_dt(t, L.kc);
    L.T = (n + tile - 1) / tile;
    const size_t wide = 8, vsz = dtype_size(t), acc = (t == DM_F32) ? 4 : 8;
    const size_t tiles = (size_t)(L.G * d * L.T);
    L.counter = 0;
    L.done = 16;
    L.memset_bytes = align256(L.done + 4 * (size_t)(L.G * d));
    L.pre = L.memset_bytes;                                   // tile sums, then exclusive prefixes
    L.partial = align256(L.pre + wide * tiles * 2 * L.kc);
    L.res = align256(L.partial + wide * (size_t)prologue_blocks(n, num_sms) * 2 * k);
    L.zg = align256(L.res + wide * 2 * (size_t)k);
    L.outg = align256(L.zg + vsz * (size_t)(L.G * n * L.kc));
    L.total = align256(L.outg + std::max(acc, wide) * (size_t)(L.G * n * L.kc));
    return L;
}

template <dm_dtype DT, int KC>
cudaError_t launch_kc(const L1QueryArgs& a, cudaStream_t st, int64_t* launches, int stage) {
    using Cfg = QCfg<DT, KC>;
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    using Wide = typename Types<DT>::Wide;
    const ScratchLayout L = scratch_layout(a.dtype, a.n, a.d, a.k, a.num_sms);
    unsigned char* sc = static_cast<unsigned char*>(a.scratch);
    // 256-bit loads of Zg rows and 16-byte accesses to outg need aligned bases.
    if ((reinterpret_cast<uintptr_t>(sc + L.zg) % 32) != 0 ||
        (reinterpret_cast<uintptr_t>(sc + L.outg) % 32) != 0)
        return cudaErrorMisalignedAddress;
    cudaError_t e;
    const bool atomic = !a.deterministic;
    if (stage == 2) {   // finalize (L2-reduction mode only)
        if (!atomic) return cudaSuccess;
        const bool vec = (a.k % 4 == 0) && (a.ldo % 4 == 0) && sizeof(typename Types<DT>::Out) == 4 &&
                         (reinterpret_cast<uintptr_t>(a.out) % 16 == 0);
        const int64_t total = a.n * ((a.k + 3) / 4);
        const int64_t fb = std::max<int64_t>(1, std::min<int64_t>((total + kThreads - 1) / kThreads,
                                                                   8 * (int64_t)a.num_sms));
        auto kern = vec ? l1_finalize_kernel<DT, KC, 4> : l1_finalize_kernel<DT, KC, 1>;
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(2 * a.k * sizeof(Acc)))) != cudaSuccess)
            return e;
        kern<<<(unsigned)fb, kThreads, 2 * (size_t)a.k * sizeof(Acc), st>>>(
            reinterpret_cast<const Acc*>(sc + L.outg), static_cast<const Acc*>(a.R),
            reinterpret_cast<const Wide*>(sc + L.res), a.n, (int)a.k,
            static_cast<typename Types<DT>::Out*>(a.out), a.ldo);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++*launches;
        return cudaSuccess;
    }
    if (stage == 0) {
        const int blocks = prologue_blocks(a.n, a.num_sms);
        const int64_t rpb = (a.n + blocks - 1) / blocks;
        const int JW = (int)(L.G * KC);
        const bool vec = (a.k % 4 == 0) && (a.ldz % 4 == 0) && sizeof(V) == 4 && KC % 4 == 0 &&
                         (reinterpret_cast<uintptr_t>(a.Z) % 16 == 0);
        const int VEC = vec ? 4 : 1;
        const int NJV = JW / VEC;
        const int JC = NJV < kThreads ? NJV : kThreads;
        const size_t smem = sizeof(Wide) * 2 * (size_t)(kThreads / JC) * JC;
        auto kern = vec ? l1_prologue_kernel<DT, KC, 4> : l1_prologue_kernel<DT, KC, 1>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<blocks, kThreads, smem, st>>>(
            static_cast<const V*>(a.Z), a.n, (int)a.k, a.ldz, static_cast<const Acc*>(a.R),
            reinterpret_cast<V*>(sc + L.zg), JW, reinterpret_cast<Wide*>(sc + L.partial), rpb);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int k2 = (int)(2 * a.k);
        l1_prologue_finalize<Wide><<<(k2 + 7) / 8, 256, 0, st>>>(
            reinterpret_cast<const Wide*>(sc + L.partial), blocks, k2,
            reinterpret_cast<Wide*>(sc + L.res));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        *launches += 2;
        return cudaSuccess;
    }

    if (stage == 3) {   // tile aggregates + per-segment exclusive scan
        auto kern = l1_aggregate_kernel<DT, KC>;
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, 0);
        if (e != cudaSuccess) return e;
        const int64_t warps = L.G * a.d * L.T;
        const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(
            (warps + kWarps - 1) / kWarps, (int64_t)std::max(occ, 1) * a.num_sms));
        kern<<<(unsigned)blocks, kThreads, 0, st>>>(
            static_cast<const V*>(a.xs), a.perm, a.n, (int)a.d, reinterpret_cast<const V*>(sc + L.zg),
            static_cast<const V*>(a.mu), a.mu_stride, reinterpret_cast<Wide*>(sc + L.pre), (int)L.T,
            (int)L.G, a.err);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        l1_tile_scan_kernel<Wide><<<(unsigned)(L.G * a.d), kThreads, 0, st>>>(
            reinterpret_cast<Wide*>(sc + L.pre), (int)L.T, 2 * KC);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        *launches += 2;
        return cudaSuccess;
    }

    e = cudaMemsetAsync(sc, 0, L.memset_bytes, st);
    if (e != cudaSuccess) return e;
    if (atomic) {
        e = cudaMemsetAsync(sc + L.outg, 0, sizeof(Acc) * (size_t)(L.G * a.n * KC), st);
        if (e != cudaSuccess) return e;
    }
    QParams<V, Acc, Wide> p;
    p.xs = static_cast<const V*>(a.xs);
    p.perm = a.perm;
    p.n = a.n;
    p.d = (int)a.d;
    p.R = static_cast<const Acc*>(a.R);
    p.Zg = reinterpret_cast<const V*>(sc + L.zg);
    p.k = (int)a.k;
    p.res = reinterpret_cast<const Wide*>(sc + L.res);
    p.mu = static_cast<const V*>(a.mu);
    p.mu_stride = a.mu_stride;
    p.outg = reinterpret_cast<Acc*>(sc + L.outg);
    p.outw = reinterpret_cast<Wide*>(sc + L.outg);   // the same region: one mode per call
    p.out = a.out;
    p.ldo = a.ldo;
    p.counter = reinterpret_cast<uint32_t*>(sc + L.counter);
    p.done = reinterpret_cast<uint32_t*>(sc + L.done);
    p.pre = reinterpret_cast<const Wide*>(sc + L.pre);
    p.err = a.err;
    p.T = (int)L.T;
    p.G = (int)L.G;
    p.spin_limit = a.spin_limit;

    auto kern = atomic ? l1_query_kernel<DT, KC, false> : l1_query_kernel<DT, KC, true>;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, 0);
    if (e != cudaSuccess) return e;
    // a warp per claimed tile; every CTA resident (the ordered mode's waits
    // are on tiles claimed by running warps)
    const int64_t total_tiles = (int64_t)p.G * p.d * p.T;
    const int64_t blocks = std::max<int64_t>(
        1, std::min<int64_t>((total_tiles + kWarps - 1) / kWarps, (int64_t)std::max(occ, 1) * a.num_sms));
    kern<<<(unsigned)blocks, kThreads, 0, st>>>(p);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*launches;
    return cudaSuccess;
}

template <dm_dtype DT>
cudaError_t launch_dt(const L1QueryArgs& a, cudaStream_t st, int64_t* launches, int stage) {
    constexpr int FULL = DT == DM_F64 ? 4 : 8;
    switch (pick_kc(a.dtype, a.n, a.k)) {
        case 1: return launch_kc<DT, 1>(a, st, launches, stage);
        case 2: return launch_kc<DT, 2>(a, st, launches, stage);
        case 4: return launch_kc<DT, 4>(a, st, launches, stage);
        default: return launch_kc<DT, FULL>(a, st, launches, stage);
    }
}

cudaError_t launch_any(const L1QueryArgs& a, cudaStream_t s, int64_t* launches, int stage) {
    switch (a.dtype) {
        case DM_F32: return launch_dt<DM_F32>(a, s, launches, stage);
        case DM_F64: return launch_dt<DM_F64>(a, s, launches, stage);
        default: return launch_dt<DM_I32>(a, s, launches, stage);
    }
}

}  // namespace

size_t l1_query_scratch_bytes(dm_dtype t, int64_t n, int64_t d, int64_t k, int num_sms) {
    return scratch_layout(t, n, d, k, num_sms).total;
}

cudaError_t l1_prologue_launch(const L1QueryArgs& a, cudaStream_t s, int64_t* launches) {
    return launch_any(a, s, launches, 0);
}

cudaError_t l1_query_launch(const L1QueryArgs& a, cudaStream_t s, int64_t* launches) {
    return launch_any(a, s, launches, 1);
}

cudaError_t l1_finalize_launch(const L1QueryArgs& a, cudaStream_t s, int64_t* launches) {
    return launch_any(a, s, launches, 2);
}

cudaError_t l1_aggregate_launch(const L1QueryArgs& a, cudaStream_t s, int64_t* launches) {
    return launch_any(a, s, launches, 3);
}

}  // namespace dm
