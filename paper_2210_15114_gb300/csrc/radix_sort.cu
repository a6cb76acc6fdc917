// Preprocessing of the l1 product (Algorithm 1, Section 2): sort every
// coordinate column of X ascending, keeping the sorting permutation.
//
// Stable LSD radix sort with 8-bit digits over d independent column segments:
//   keygen_hist   -- one read of row-major X: order-preserving unsigned keys
//                    written column-major (d x n) plus the digit histograms of
//                    every digit position of every column, in one pass.
//   onesweep_pass -- one digit position: each CTA ranks a tile of keys by the
//                    digit (ballot peer masks + per-warp counters, stable), publishes
//                    its digit counts and finds the counts of all earlier tiles
//                    of its column through a decoupled look-back (bounded
//                    spin), then scatters keys and payload through shared
//                    memory so that runs of equal digits are written
//                    contiguously.  The last pass writes the sorted values (in
//                    the input element type) and the permutation.
// Ties keep index order (LSD is stable), so the permutation equals a stable
// argsort of each column.  -0.0 sorts before +0.0 (they differ in key, not in
// value; either order gives the same product).
#include <algorithm>

#include "dm_internal.h"

namespace dm {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRadix = 256;

// ------------------------------------------------------------ key mapping
__device__ __forceinline__ uint32_t to_key(float v) {
    uint32_t u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ unsigned long long to_key(double v) {
    unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | (1ull << 63));
}
__device__ __forceinline__ uint32_t to_key(int32_t v) { return (uint32_t)v ^ 0x80000000u; }

__device__ __forceinline__ void from_key(uint32_t k, float* v) {
    *v = __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}
__device__ __forceinline__ void from_key(unsigned long long k, double* v) {
    *v = __longlong_as_double((long long)((k >> 63) ? (k & ~(1ull << 63)) : ~k));
}
__device__ __forceinline__ void from_key(uint32_t k, int32_t* v) { *v = (int32_t)(k ^ 0x80000000u); }

__device__ __forceinline__ bool finite_val(float v) { return isfinite(v); }
__device__ __forceinline__ bool finite_val(double v) { return isfinite(v); }
__device__ __forceinline__ bool finite_val(int32_t) { return true; }

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Lanes of the warp holding the same 8-bit digit as this lane, from eight
// ballots (one per digit bit): a lane is a peer when it agrees on every bit.
// Every lane holds a key (positions past n carry the all-ones padding key),
// so the match starts from the full warp.  All 32 lanes must call it.
__device__ __forceinline__ uint32_t digit_peers(uint32_t digit) {
    uint32_t peers = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const bool bit = (digit >> b) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bal : ~bal;
    }
    return peers;
}

// Exclusive scan of one value per thread over the 256 threads of the CTA.
// `warp_tot` is kWarps words of shared memory.  Returns the exclusive prefix;
// *total receives the sum over the CTA.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tot,
                                                         uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    uint32_t before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        uint32_t t = warp_tot[w];
        if (w < warp) before += t;
        all += t;
    }
    __syncthreads();
    *total = all;
    return before + inc - v;
}

// ------------------------------------------------------------ keygen + hist
// CTA = RB rows x DB columns of X.  All loads of a thread are issued first
// (RB*DB/256 values in registers), the keys go to a padded shared tile, then
// each warp histograms one column's keys into a private shared histogram
// (no contention between warps; lanes of one warp that hit the same bin --
// frequent in the two highest digit positions, where sign and exponent bits
// collide -- are serialized by the shared-memory unit, which costs less than
// forming peer masks on the saturated integer pipe), and finally the tile is
// written column-major and the histograms are added to the global counts.
template <dm_dtype DT>
struct KeygenCfg {
    using Ty = Types<DT>;
    using Key = typename Ty::Key;
    static constexpr int P = (int)sizeof(Key);           // digit positions
    static constexpr int DB = sizeof(Key) == 4 ? 8 : 4;  // columns per CTA
    static constexpr int RB = 1024;                      // rows per CTA
    static constexpr int TS = RB + 8;                    // padded row stride of the tile
    static constexpr int WPC = kWarps / DB;              // warps per column
    static constexpr int PER = RB * DB / kThreads;       // loads per thread
    static constexpr size_t hist_bytes = (size_t)kWarps * P * kRadix * 4;
    static constexpr size_t smem = hist_bytes + (size_t)DB * TS * sizeof(Key);
};

template <dm_dtype DT>
__global__ void __launch_bounds__(kThreads)
keygen_hist_kernel(const typename Types<DT>::V* __restrict__ X, int64_t n, int64_t d, int64_t ldx,
                   typename Types<DT>::Key* __restrict__ keys, uint32_t* __restrict__ hist,
                   uint32_t* err) {
    using Cfg = KeygenCfg<DT>;
    using Key = typename Cfg::Key;
    using V = typename Types<DT>::V;
    constexpr int P = Cfg::P, DB = Cfg::DB, RB = Cfg::RB, TS = Cfg::TS, PER = Cfg::PER;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t* h = reinterpret_cast<uint32_t*>(smem_raw);                    // [warp][P][256]
    Key* tile = reinterpret_cast<Key*>(smem_raw + Cfg::hist_bytes);         // [DB][TS]

    // Persistent over row blocks (one histogram flush per CTA instead of one
    // per row block); blockIdx.x is the column block, so the CTAs that share
    // the rows' cache lines run side by side.
    const int64_t c0 = (int64_t)blockIdx.x * DB;
    const int nd = (int)min64(DB, d - c0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nrb = (n + RB - 1) / RB;

    for (int i = threadIdx.x; i < kWarps * P * kRadix; i += kThreads) h[i] = 0;

    bool bad = false;
    for (int64_t rb = blockIdx.y; rb < nrb; rb += gridDim.y) {
        const int64_t row0 = rb * RB;
        const int nr = (int)min64(RB, n - row0);
        V v[PER];
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int idx = threadIdx.x + j * kThreads;
            const int r = idx / DB, c = idx % DB;
            v[j] = (r < nr && c < nd) ? X[(row0 + r) * ldx + c0 + c] : V(0);
        }
        __syncthreads();   // the previous block's tile has been written out
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int idx = threadIdx.x + j * kThreads;
            const int r = idx / DB, c = idx % DB;
            if (r < nr && c < nd) bad |= !finite_val(v[j]);
            tile[c * TS + r] = to_key(v[j]);
        }
        __syncthreads();
        {
            const int c = warp % DB, part = warp / DB;
            uint32_t* hw = h + warp * P * kRadix;
            const int rows_per = RB / Cfg::WPC;
            const int rbeg = part * rows_per;
            const bool colok = c < nd;
            for (int r = rbeg + lane; r < rbeg + rows_per; r += 32) {
                const bool ok = colok && r < nr;
                const Key key = ok ? tile[c * TS + r] : Key(0);
                if (ok) {
#pragma unroll
                    for (int q = 0; q < P; ++q)
                        atomicAdd(&hw[q * kRadix + ((uint32_t)(key >> (8 * q)) & 0xffu)], 1u);
                }
            }
        }
        for (int i = threadIdx.x; i < nd * RB; i += kThreads) {
            const int cc = i / RB, r = i % RB;
            if (r < nr) keys[(c0 + cc) * n + row0 + r] = tile[cc * TS + r];
        }
    }
    if (bad) set_error(err, kErrNonfinite);
    __syncthreads();
    for (int i = threadIdx.x; i < nd * P * kRadix; i += kThreads) {
        const int c = i / (P * kRadix), rest = i % (P * kRadix);
        uint32_t tot = 0;
#pragma unroll
        for (int part = 0; part < Cfg::WPC; ++part) tot += h[(part * DB + c) * P * kRadix + rest];
        if (tot) atomicAdd(&hist[(c0 + c) * P * kRadix + rest], tot);
    }
}

// ------------------------------------------------------------ onesweep pass
// Keys per thread: 20 for 4-byte keys in large passes (measured best of 8-32
// at n = 2^20, d = 32: 0.191 ms per pass against 0.212 with 12), 12 where so
// few keys would leave the GPU short of tiles (sets of a batch with n d below
// 2^24: 58 against 64 ms for the whole batch with 20); 8 for 8-byte keys.
template <dm_dtype DT, bool WIDE>
struct PassCfg {
    using Key = typename Types<DT>::Key;
    static constexpr int ITEMS = sizeof(Key) == 4 ? (WIDE ? 20 : 12) : 8;
    static constexpr int TILE = kThreads * ITEMS;
    // the tile's keys and payload, staged for the scatter (dynamic shared memory)
    static constexpr size_t smem = (size_t)TILE * (sizeof(Key) + sizeof(int32_t));
};

bool wide_tiles(dm_dtype t, int64_t n, int64_t d) {
    return t != DM_F64 && n * d >= (int64_t(1) << 24);
}

template <dm_dtype DT, bool WIDE>
cudaError_t onesweep_smem_attr();

constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1;

template <dm_dtype DT, bool WIDE>
__global__ void __launch_bounds__(kThreads, 3)
onesweep_kernel(const typename Types<DT>::Key* __restrict__ keys_in,
                const int32_t* __restrict__ vals_in,            // null on the first pass
                typename Types<DT>::Key* __restrict__ keys_out,
                int32_t* __restrict__ vals_out,
                typename Types<DT>::V* __restrict__ sorted_out,  // last pass only
                int32_t* __restrict__ perm_out,                   // last pass only
                const uint32_t* __restrict__ hist, uint32_t* lookback, uint32_t* counter,
                int64_t n, int D, int pass, int P, int T, int first, int last, uint32_t* err,
                uint32_t spin_limit) {
    using Key = typename Types<DT>::Key;
    using V = typename Types<DT>::V;
    constexpr int ITEMS = PassCfg<DT, WIDE>::ITEMS, TILE = PassCfg<DT, WIDE>::TILE;

    __shared__ uint32_t s_tile;
    __shared__ uint32_t wcount[kWarps][kRadix];
    __shared__ uint32_t tile_start[kRadix];
    __shared__ uint32_t gbase[kRadix];
    __shared__ uint32_t warp_tot[kWarps];
    extern __shared__ __align__(16) unsigned char os_smem[];
    Key* sk = reinterpret_cast<Key*>(os_smem);                             // [TILE]
    int32_t* sv = reinterpret_cast<int32_t*>(os_smem + (size_t)TILE * sizeof(Key));   // [TILE]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(counter, 1u);
    for (int i = tid; i < kWarps * kRadix; i += kThreads) (&wcount[0][0])[i] = 0;
    __syncthreads();
    // Claims interleave the columns (column fastest), so the look-back
    // chains of all d columns advance side by side and each chain has only a
    // few tiles in flight.
    const uint32_t g = s_tile;
    const int64_t c = g % (uint32_t)D;
    const int t = (int)(g / (uint32_t)D);
    const int64_t seg = c * n;
    const int64_t tile0 = (int64_t)t * TILE;
    const int shift = 8 * pass;

    // Segment-level start of every digit from the upfront histogram.
    uint32_t seg_total;
    const uint32_t digit_start =
        block_exclusive_scan(hist[(c * P + pass) * kRadix + tid], warp_tot, &seg_total);

    // Load a warp-striped tile: item j of lane l sits at tile position
    // warp*32*ITEMS + j*32 + l, so ranking items in (j, lane) order is the
    // original order.  Positions past n get digit 255 and land after every
    // real key of the tile; their global positions are >= n and are dropped.
    // Tile-relative indices in 32 bits (n < 2^30): base pointers of the column
    // and of the tile are formed once.
    const uint32_t n32 = (uint32_t)n;
    const uint32_t rem = (uint32_t)(n - tile0);           // positions left in the column
    const uint32_t lbase = (uint32_t)(warp * 32 * ITEMS + lane);
    const Key* kin = keys_in + seg + tile0;
    Key key[ITEMS];
    uint32_t rank[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t li = lbase + 32u * j;
        key[j] = li < rem ? kin[li] : ~(Key)0;
    }
    // Stable ranks within the warp: item j of every lane is ranked after all
    // items j' < j of the warp and after lower lanes' item j.  All matches are
    // issued first; then the lowest lane of each group of equal digits adds the
    // group size to the warp's counter with an atomic that returns the prior
    // count (one warp's shared atomics take effect in program order, so the
    // counts stay in item order) and hands it to its peers.
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint32_t peers[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) peers[j] = digit_peers((uint32_t)(key[j] >> shift) & 0xffu);
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t dg = (uint32_t)(key[j] >> shift) & 0xffu;
        rank[j] = 0;
        if ((peers[j] & lt_mask) == 0) rank[j] = atomicAdd(&wcount[warp][dg], (uint32_t)__popc(peers[j]));
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j)
        rank[j] = __shfl_sync(0xffffffffu, rank[j], __ffs(peers[j]) - 1) + __popc(peers[j] & lt_mask);
    __syncthreads();

    // Per digit: exclusive offsets of the warps, and the tile's count.
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const uint32_t x = wcount[w][tid];
        wcount[w][tid] = cnt;
        cnt += x;
    }

    // Decoupled look-back over the earlier tiles of this column.
    uint32_t* lb = lookback + (int64_t)c * T * kRadix;
    uint32_t excl = 0;
    if (t == 0) {
        st_relaxed(&lb[tid], kFlagInc | cnt);
    } else {
        st_relaxed(&lb[(int64_t)t * kRadix + tid], kFlagAgg | cnt);
        // Predecessors are read W at a time (one round trip per window); a
        // tile that has not published yet is waited for (bounded), and the
        // walk stops at the first inclusive count.
        constexpr int W = 8;
        int base = t - 1;
        uint32_t spins = 0;
        bool done = false;
        while (!done) {
            uint32_t sv[W];
#pragma unroll
            for (int u = 0; u < W; ++u)
                sv[u] = base - u >= 0 ? ld_relaxed(&lb[(int64_t)(base - u) * kRadix + tid]) : kFlagInc;
#pragma unroll
            for (int u = 0; u < W; ++u) {
                if (!done) {
                    uint32_t sq = sv[u];
                    while ((sq & ~kValMask) == 0) {
                        if (++spins > spin_limit) { set_error(err, kErrTimeout); sq = kFlagInc; break; }
                        __nanosleep(64);
                        sq = ld_relaxed(&lb[(int64_t)(base - u) * kRadix + tid]);
                    }
                    excl += sq & kValMask;
                    if ((sq & ~kValMask) == kFlagInc) done = true;
                }
            }
            base -= W;
        }
        st_relaxed(&lb[(int64_t)t * kRadix + tid], kFlagInc | (excl + cnt));
    }

    uint32_t tile_total;
    const uint32_t ts = block_exclusive_scan(cnt, warp_tot, &tile_total);
    tile_start[tid] = ts;
    gbase[tid] = digit_start + excl - ts;   // global = gbase[digit] + tile position
    __syncthreads();

    // Tile positions; the payload is read only now, straight to its slot.
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t dg = (uint32_t)(key[j] >> shift) & 0xffu;
        rank[j] += tile_start[dg] + wcount[warp][dg];
        sk[rank[j]] = key[j];
    }
    const int32_t* vin = first ? nullptr : vals_in + seg + tile0;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t li = lbase + 32u * j;
        sv[rank[j]] = li < rem ? (first ? (int32_t)(tile0 + li) : vin[li]) : -1;
    }
    __syncthreads();

    Key* kout = last ? nullptr : keys_out + seg;
    int32_t* vout = last ? perm_out + seg : vals_out + seg;
    V* sout = last ? sorted_out + seg : nullptr;
#pragma unroll 4
    for (int pos = tid; pos < TILE; pos += kThreads) {
        const Key k = sk[pos];
        const uint32_t dg = (uint32_t)(k >> shift) & 0xffu;
        const uint32_t gp = gbase[dg] + (uint32_t)pos;
        if (gp < n32) {
            if (last) {
                V v;
                from_key(k, &v);
                sout[gp] = v;
            } else {
                kout[gp] = k;
            }
            vout[gp] = sv[pos];
        }
    }
}

template <dm_dtype DT, bool WIDE>
cudaError_t onesweep_smem_attr() {
    cudaError_t e = cudaFuncSetAttribute(onesweep_kernel<DT, WIDE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)PassCfg<DT, WIDE>::smem);
    if (e != cudaSuccess || !WIDE) return e;
    // wide tiles: three CTAs of 50 KB per SM.  (Not for the narrow tiling: a
    // batch's lanes run other kernels beside the passes, and an SM split
    // fixed at the maximum kept them apart: 67 against 58 ms for the batch.)
    return cudaFuncSetAttribute(onesweep_kernel<DT, WIDE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                cudaSharedmemCarveoutMaxShared);
}

template <dm_dtype DT>
cudaError_t launch_keygen_t(const SortArgs& a, cudaStream_t s) {
    using Cfg = KeygenCfg<DT>;
    auto kern = keygen_hist_kernel<DT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Cfg::smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t cb = (a.d + Cfg::DB - 1) / Cfg::DB;
    const int64_t nrb = (a.n + Cfg::RB - 1) / Cfg::RB;
    const int64_t per_col = std::max<int64_t>(1, std::min<int64_t>(nrb, (3 * (int64_t)sms + cb - 1) / cb));
    dim3 grid((unsigned)cb, (unsigned)per_col);
    kern<<<grid, kThreads, Cfg::smem, s>>>(
        static_cast<const typename Types<DT>::V*>(a.X), a.n, a.d, a.ldx,
        static_cast<typename Types<DT>::Key*>(a.keys_a), a.hist, a.err);
    return cudaGetLastError();
}

template <dm_dtype DT, bool WIDE>
cudaError_t launch_passes_w(const SortArgs& a, const int* pass_list, int npass, cudaStream_t s,
                            int64_t* launches) {
    using Key = typename Types<DT>::Key;
    using V = typename Types<DT>::V;
    constexpr int TILE = PassCfg<DT, WIDE>::TILE;
    const int T = (int)((a.n + TILE - 1) / TILE);
    const int P = (int)sizeof(Key);
    const Key* kin = static_cast<const Key*>(a.keys_a);
    const int32_t* vin = nullptr;
    Key* kbuf[2] = {static_cast<Key*>(a.keys_b), static_cast<Key*>(a.keys_a)};
    int32_t* vbuf[2] = {a.vals_b, a.vals_a};
    const size_t lb_stride = (size_t)a.d * T * kRadix;
    cudaError_t ea = onesweep_smem_attr<DT, WIDE>();
    if (ea != cudaSuccess) return ea;
    for (int i = 0; i < npass; ++i) {
        const int first = i == 0, last = i == npass - 1;
        Key* kout = kbuf[i & 1];
        int32_t* vout = vbuf[i & 1];
        onesweep_kernel<DT, WIDE><<<(unsigned)(a.d * T), kThreads, PassCfg<DT, WIDE>::smem, s>>>(
            kin, vin, kout, vout, static_cast<V*>(a.sorted_out), a.perm_out, a.hist,
            a.lookback + i * lb_stride, a.counters + i, a.n, (int)a.d, pass_list[i], P, T, first,
            last, a.err, a.spin_limit);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        ++*launches;
        kin = kout;
        vin = vout;
    }
    return cudaSuccess;
}

template <dm_dtype DT>
cudaError_t launch_passes_t(const SortArgs& a, const int* pass_list, int npass, cudaStream_t s,
                            int64_t* launches) {
    if constexpr (sizeof(typename Types<DT>::Key) == 4) {
        if (wide_tiles(DT, a.n, a.d)) return launch_passes_w<DT, true>(a, pass_list, npass, s, launches);
    }
    return launch_passes_w<DT, false>(a, pass_list, npass, s, launches);
}

}  // namespace

// The tile of a one-column FP32 pass (the narrow tiling: n d below 2^24 for
// the two-tile column of the unpublished-wait test).
int sort_tile_f32() { return PassCfg<DM_F32, false>::TILE; }

cudaError_t sort_launch_unpublished_wait(const SortArgs& a, cudaStream_t s, int64_t* launches) {
    using Key = Types<DM_F32>::Key;
    constexpr int TILE = PassCfg<DM_F32, false>::TILE;
    if (a.dtype != DM_F32 || a.d != 1 || a.n != 2 * TILE) return cudaErrorInvalidValue;
    // One CTA; it claims ticket 1 = (column 0, tile 1) and waits for tile 0.
    // First pass (no payload read), not the last (keys_b / vals_b written).
    cudaError_t ea = onesweep_smem_attr<DM_F32, false>();
    if (ea != cudaSuccess) return ea;
    onesweep_kernel<DM_F32, false><<<1, kThreads, PassCfg<DM_F32, false>::smem, s>>>(
        static_cast<const Key*>(a.keys_a), nullptr, static_cast<Key*>(a.keys_b), a.vals_b, nullptr,
        nullptr, a.hist, a.lookback, a.counters, a.n, 1, 0, sort_passes(DM_F32), 2, 1, 0, a.err,
        a.spin_limit);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) ++*launches;
    return e;
}

int sort_passes(dm_dtype t) { return key_bits(t) / 8; }

size_t sort_hist_words(dm_dtype t, int64_t d) { return (size_t)d * sort_passes(t) * kRadix; }

size_t sort_lookback_words(dm_dtype t, int64_t n, int64_t d) {
    // sized for the narrower tiling (more tiles)
    const int tile = (t == DM_F64) ? PassCfg<DM_F64, false>::TILE : PassCfg<DM_F32, false>::TILE;
    const int64_t T = (n + tile - 1) / tile;
    return (size_t)sort_passes(t) * d * T * kRadix;
}

cudaError_t sort_launch_keygen(const SortArgs& a, cudaStream_t s, int64_t* launches) {
    cudaError_t e;
    switch (a.dtype) {
        case DM_F32: e = launch_keygen_t<DM_F32>(a, s); break;
        case DM_F64: e = launch_keygen_t<DM_F64>(a, s); break;
        default: e = launch_keygen_t<DM_I32>(a, s); break;
    }
    if (e == cudaSuccess) ++*launches;
    return e;
}

cudaError_t sort_launch_passes(const SortArgs& a, const int* pass_list, int npass, cudaStream_t s,
                               int64_t* launches) {
    switch (a.dtype) {
        case DM_F32: return launch_passes_t<DM_F32>(a, pass_list, npass, s, launches);
        case DM_F64: return launch_passes_t<DM_F64>(a, pass_list, npass, s, launches);
        default: return launch_passes_t<DM_I32>(a, pass_list, npass, s, launches);
    }
}

}  // namespace dm
