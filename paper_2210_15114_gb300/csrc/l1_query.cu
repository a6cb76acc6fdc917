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
// One persistent kernel does the sorted part for all coordinates.  Work unit:
// a tile of TILE_E consecutive sorted positions of one coordinate and one
// group of KC query columns.  Per tile:
//   A. stage perm, x - b (b = the tile's first sorted value) and gather the
//      k-wide query rows Z[perm[r], :] into shared memory (cp.async);
//   B. in-tile exclusive prefix sums Lz, Lxz of z and (x - b) z (FP32 for
//      FP32 data);
//   C. decoupled look-back over the earlier tiles of the same coordinate for
//      the tile's exclusive prefix Pt (FP64 for FP32 data, bounded spin), and
//      two per-column constants in FP64:
//        alpha = Pt_z,   gamma = Pt_xz - (b - mu) Pt_z,
//      so that 2 (x_r P_z[r] - P_xz[r]) = 2 ((x_r - b)(alpha + Lz_r) - (gamma + Lxz_r)):
//      the large terms are combined in FP64 once per tile and each element
//      works on tile-local values;
//   D. wait until every tile of coordinate c-1 (same column group) has added
//      its values (bounded spin on a counter), so each output element receives
//      its d contributions in coordinate order: the result is deterministic;
//   E. coordinate 0 stores value + R^T Z - R_k 1^T Z; later coordinates add;
//   F. publish "tile done" for coordinate c.
// Tiles are claimed from an atomic counter in (group, coordinate, tile) order,
// so every wait is on work claimed earlier by a running CTA: no deadlock.
// Integer data run the same steps exactly in int64.
#include <algorithm>

#include "dm_internal.h"

namespace dm {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

template <dm_dtype DT, int KC>
struct QCfg {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    static constexpr int SEGS = kThreads / KC;                 // thread segments per column
    static constexpr int SEG_LEN = sizeof(V) == 4 ? (8 * KC < 48 ? 8 * KC : 48)
                                                  : (4 * KC < 24 ? 4 * KC : 24);
    static constexpr int TILE_E = SEGS * SEG_LEN;              // sorted positions per tile
    static constexpr int SEG_STRIDE = (SEG_LEN + 1) * KC;      // padded (bank spread)
    static constexpr int NV = 2 * KC;                          // scanned quantities
    static constexpr size_t dx_off = align16((size_t)SEGS * SEG_STRIDE * sizeof(V));
    static constexpr size_t perm_off = dx_off + align16((size_t)TILE_E * sizeof(Acc));
    static constexpr size_t smem = perm_off + (size_t)TILE_E * 4;
    static constexpr int BATCH = SEG_LEN < 8 ? SEG_LEN : 8;   // RMW loads in flight per thread
};

template <class V, class Acc, class Wide>
struct QParams {
    const V* xs; const int32_t* perm; int64_t n; int d;
    const Acc* R;                     // R_k = sum_c (x_k(c) - mu_c)
    const V* Z; int64_t ldz; int k;
    const Wide* res;                  // R^T Z (k), then 1^T Z (k)
    const V* mu; int64_t mu_stride;
    void* out; int64_t ldo;
    uint32_t* counter; uint32_t* done; uint32_t* flags;
    Wide* agg; Wide* inc;
    uint32_t* err;
    int T, G, vw;
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ void cp_async16(void* s, const void* g, int src) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(sa), "l"(g), "r"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* s, const void* g, int src) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" :: "r"(sa), "l"(g), "r"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* s, const void* g, int src) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" :: "r"(sa), "l"(g), "r"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

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

// Bounded wait until *p >= target (acquire).  Returns false on timeout.
__device__ __forceinline__ bool wait_geq(const uint32_t* p, uint32_t target, uint32_t* err) {
    uint32_t spins = 0;
    while (ld_acquire(p) < target) {
        if (++spins > kSpinLimit) { set_error(err, kErrTimeout); return false; }
        __nanosleep(128);
    }
    return true;
}

// Gather the query rows of the tile into shared memory: z_s[seg][i][col].
template <dm_dtype DT, int KC>
__device__ __forceinline__ void gather_rows(typename Types<DT>::V* z_s, const int32_t* perm_s,
                                            const typename Types<DT>::V* Zg, int64_t ldz, int kg,
                                            int vw) {
    using Cfg = QCfg<DT, KC>;
    using V = typename Types<DT>::V;
    constexpr int ROWB = KC * (int)sizeof(V);
    if constexpr (ROWB % 16 == 0) {
        if (vw == 16 && kg == KC) {
            constexpr int VPC = 16 / (int)sizeof(V), CPR = ROWB / 16;
            for (int j = threadIdx.x; j < Cfg::TILE_E * CPR; j += kThreads) {
                const int e = j / CPR, q = j % CPR;
                const int32_t pe = perm_s[e];
                V* dst = z_s + (e / Cfg::SEG_LEN) * Cfg::SEG_STRIDE + (e % Cfg::SEG_LEN) * KC + q * VPC;
                const V* src = Zg + (int64_t)(pe < 0 ? 0 : pe) * ldz + q * VPC;
                cp_async16(dst, src, pe >= 0 ? 16 : 0);
            }
            return;
        }
    }
    if constexpr (ROWB % 8 == 0 && sizeof(V) <= 8) {
        if (vw == 8 && kg == KC) {
            constexpr int VPC = 8 / (int)sizeof(V), CPR = ROWB / 8;
            for (int j = threadIdx.x; j < Cfg::TILE_E * CPR; j += kThreads) {
                const int e = j / CPR, q = j % CPR;
                const int32_t pe = perm_s[e];
                V* dst = z_s + (e / Cfg::SEG_LEN) * Cfg::SEG_STRIDE + (e % Cfg::SEG_LEN) * KC + q * VPC;
                const V* src = Zg + (int64_t)(pe < 0 ? 0 : pe) * ldz + q * VPC;
                cp_async8(dst, src, pe >= 0 ? 8 : 0);
            }
            return;
        }
    }
    for (int j = threadIdx.x; j < Cfg::TILE_E * KC; j += kThreads) {
        const int e = j / KC, q = j % KC;
        const int32_t pe = perm_s[e];
        V* dst = z_s + (e / Cfg::SEG_LEN) * Cfg::SEG_STRIDE + (e % Cfg::SEG_LEN) * KC + q;
        const V* src = Zg + (int64_t)(pe < 0 ? 0 : pe) * ldz + (q < kg ? q : 0);
        const int bytes = (pe >= 0 && q < kg) ? (int)sizeof(V) : 0;
        if constexpr (sizeof(V) == 8) cp_async8(dst, src, bytes);
        else cp_async4(dst, src, bytes);
    }
}

// ---------------------------------------------------------------- kernel
template <dm_dtype DT, int KC>
__global__ void __launch_bounds__(kThreads)
l1_query_kernel(QParams<typename Types<DT>::V, typename Types<DT>::Acc, typename Types<DT>::Wide> p) {
    using Cfg = QCfg<DT, KC>;
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    using Wide = typename Types<DT>::Wide;
    using Out = typename Types<DT>::Out;
    constexpr int SEG_LEN = Cfg::SEG_LEN, TILE_E = Cfg::TILE_E, NV = Cfg::NV;
    constexpr int SPW = 32 / KC;   // segments of one column per warp

    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* z_s = reinterpret_cast<V*>(smem_raw);
    Acc* dx_s = reinterpret_cast<Acc*>(smem_raw + Cfg::dx_off);
    int32_t* perm_s = reinterpret_cast<int32_t*>(smem_raw + Cfg::perm_off);
    __shared__ Acc wt[kWarps][NV];
    __shared__ Acc tile_tot[NV];
    __shared__ Acc ag_s[4][KC];
    __shared__ uint32_t s_claim;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int col = tid % KC, seg = tid / KC;
    const int d = p.d, T = p.T, k = p.k;
    const uint32_t total_tiles = (uint32_t)p.G * (uint32_t)d * (uint32_t)T;

    while (true) {
        if (tid == 0) s_claim = atomicAdd(p.counter, 1u);
        __syncthreads();
        const uint32_t claim = s_claim;
        if (claim >= total_tiles) break;
        const int t = (int)(claim % (uint32_t)T);
        const int c = (int)((claim / (uint32_t)T) % (uint32_t)d);
        const int g = (int)(claim / ((uint32_t)T * (uint32_t)d));
        const int64_t e0 = (int64_t)t * TILE_E;
        const int ne = (int)min64(TILE_E, p.n - e0);
        const int64_t sbase = (int64_t)c * p.n + e0;
        const V b = p.xs[sbase];
        const int kg = min(KC, k - g * KC);

        // A. stage the tile
        for (int e = tid; e < TILE_E; e += kThreads) {
            int32_t pe = -1;
            Acc dx = 0;
            if (e < ne) {
                pe = p.perm[sbase + e];
                dx = diff(p.xs[sbase + e], b);
                if ((uint32_t)pe >= (uint32_t)p.n) {   // never for a valid plan
                    set_error(p.err, kErrInternal);
                    pe = -1;
                }
            }
            perm_s[e] = pe;
            dx_s[e] = dx;
        }
        __syncthreads();
        gather_rows<DT, KC>(z_s, perm_s, p.Z + (int64_t)g * KC, p.ldz, kg, p.vw);
        cp_async_wait_all();
        __syncthreads();

        // B. in-tile exclusive prefix of this thread's segment
        const V* zcol = z_s + seg * Cfg::SEG_STRIDE + col;
        const Acc* dxs = dx_s + seg * SEG_LEN;
        Acc sz = 0, sxz = 0;
#pragma unroll 8
        for (int i = 0; i < SEG_LEN; ++i) {
            const Acc z = (Acc)zcol[i * KC];
            sz += z;
            sxz = fmac(dxs[i], z, sxz);
        }
        Acc iz = sz, ixz = sxz;
#pragma unroll
        for (int o = 1; o < SPW; o <<= 1) {
            const Acc a = __shfl_up_sync(0xffffffffu, iz, o * KC);
            const Acc bb = __shfl_up_sync(0xffffffffu, ixz, o * KC);
            if (lane >= o * KC) { iz += a; ixz += bb; }
        }
        Acc ez = __shfl_up_sync(0xffffffffu, iz, KC);
        Acc exz = __shfl_up_sync(0xffffffffu, ixz, KC);
        if (lane < KC) { ez = 0; exz = 0; }
        if (lane >= 32 - KC) { wt[warp][col] = iz; wt[warp][KC + col] = ixz; }
        __syncthreads();
        Acc pz = 0, pxz = 0, tz = 0, txz = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const Acc a = wt[w][col], bb = wt[w][KC + col];
            if (w < warp) { pz += a; pxz += bb; }
            tz += a;
            txz += bb;
        }
        Acc Lz = pz + ez, Lxz = pxz + exz;
        if (tid < KC) { tile_tot[tid] = tz; tile_tot[KC + tid] = txz; }
        __syncthreads();

        // C. look-back for the tile's exclusive prefix, then alpha / gamma
        if (warp == 0) {
            const Wide bm = (Wide)b - (Wide)p.mu[(int64_t)c * p.mu_stride];
            const int64_t dimt = ((int64_t)g * d + c) * T;
            uint32_t* fl = p.flags + dimt;
            Wide* ag = p.agg + dimt * NV;
            Wide* in = p.inc + dimt * NV;
            Wide agg = 0, excl = 0;
            if (lane < NV) {
                const int cc = lane % KC;
                agg = (lane < KC) ? (Wide)tile_tot[cc]
                                  : bm * (Wide)tile_tot[cc] + (Wide)tile_tot[KC + cc];
            }
            if (t == 0) {
                if (lane < NV) in[lane] = agg;
                __threadfence();
                __syncwarp();
                if (lane == 0) st_release(&fl[0], 2u);
            } else {
                if (lane < NV) ag[(int64_t)t * NV + lane] = agg;
                __threadfence();
                __syncwarp();
                if (lane == 0) st_release(&fl[t], 1u);
                int pred = t - 1;
                while (true) {
                    uint32_t f = 0;
                    if (lane == 0) {
                        uint32_t spins = 0;
                        while ((f = ld_acquire(&fl[pred])) == 0u) {
                            if (++spins > kSpinLimit) { set_error(p.err, kErrTimeout); f = 2u; break; }
                            __nanosleep(32);
                        }
                    }
                    f = __shfl_sync(0xffffffffu, f, 0);
                    __syncwarp();
                    if (lane < NV) excl += ldcg((f == 2u ? in : ag) + (int64_t)pred * NV + lane);
                    if (f == 2u || pred == 0) break;
                    --pred;
                }
                if (lane < NV) in[(int64_t)t * NV + lane] = excl + agg;
                __threadfence();
                __syncwarp();
                if (lane == 0) st_release(&fl[t], 2u);
            }
            const Wide pxz_l = __shfl_sync(0xffffffffu, excl, (lane + KC) & 31);
            if (lane < KC) {
                const Wide Pz = excl, Pxz = pxz_l;
                ag_s[0][lane] = (Acc)Pz;
                ag_s[1][lane] = (Acc)(Pxz - bm * Pz);
                if (c == 0) {
                    const int gc = g * KC + lane;
                    ag_s[2][lane] = gc < k ? (Acc)p.res[gc] : Acc(0);       // R^T Z
                    ag_s[3][lane] = gc < k ? (Acc)p.res[k + gc] : Acc(0);   // 1^T Z
                }
            }
        }

        // D. coordinate order: wait for every tile of coordinate c-1
        if (c > 0 && tid == 0) wait_geq(p.done + (int64_t)g * d + c - 1, (uint32_t)T, p.err);
        __syncthreads();

        // E. evaluate and accumulate into the output rows
        {
            const Acc al = ag_s[0][col], gm = ag_s[1][col];
            const Acc rz = ag_s[2][col], uz = ag_s[3][col];
            const bool colok = col < kg;
            Out* ocol = static_cast<Out*>(p.out) + (int64_t)g * KC + col;
            const int32_t* ps = perm_s + seg * SEG_LEN;
            constexpr int B = Cfg::BATCH;
            for (int i0 = 0; i0 < SEG_LEN; i0 += B) {
                int32_t pr[B];
                Acc old[B];
#pragma unroll
                for (int q = 0; q < B; ++q) {
                    pr[q] = ps[i0 + q];
                    old[q] = 0;
                    if (colok && pr[q] >= 0) {
                        if (c > 0) old[q] = (Acc)ldcg(ocol + (int64_t)pr[q] * p.ldo);
                        else old[q] = rz - p.R[pr[q]] * uz;
                    }
                }
#pragma unroll
                for (int q = 0; q < B; ++q) {
                    const int i = i0 + q;
                    const Acc z = (Acc)zcol[i * KC];
                    const Acc dx = dxs[i];
                    const Acc v = fmac(dx, al + Lz, -(gm + Lxz));
                    if (colok && pr[q] >= 0) stcg(ocol + (int64_t)pr[q] * p.ldo, (Out)fmac(Acc(2), v, old[q]));
                    Lz += z;
                    Lxz = fmac(dx, z, Lxz);
                }
            }
        }

        // F. this tile's values are in place
        __threadfence();
        __syncthreads();
        if (tid == 0) red_release_add(p.done + (int64_t)g * d + c, 1u);
    }
}

template <dm_dtype DT, int KC>
int tile_elems() { return QCfg<DT, KC>::TILE_E; }

int pick_kc(int64_t k) {
    if (k >= 16) return 16;
    int kc = 1;
    while (kc < k) kc <<= 1;
    return kc;
}

template <dm_dtype DT>
int tile_elems_rt(int kc) {
    switch (kc) {
        case 1: return tile_elems<DT, 1>();
        case 2: return tile_elems<DT, 2>();
        case 4: return tile_elems<DT, 4>();
        case 8: return tile_elems<DT, 8>();
        default: return tile_elems<DT, 16>();
    }
}

int tile_elems_dt(dm_dtype t, int kc) {
    switch (t) {
        case DM_F32: return tile_elems_rt<DM_F32>(kc);
        case DM_F64: return tile_elems_rt<DM_F64>(kc);
        default: return tile_elems_rt<DM_I32>(kc);
    }
}

struct ScratchLayout {
    size_t counter, done, flags, agg, inc, memset_bytes, total;
};

ScratchLayout scratch_layout(dm_dtype t, int64_t n, int64_t d, int64_t k) {
    const int kc = pick_kc(k);
    const int64_t G = (k + kc - 1) / kc;
    const int64_t T = (n + tile_elems_dt(t, kc) - 1) / tile_elems_dt(t, kc);
    const size_t wide = 8;
    ScratchLayout L;
    L.counter = 0;
    L.done = 16;
    L.flags = align16(L.done + 4 * (size_t)(G * d));
    L.memset_bytes = align16(L.flags + 4 * (size_t)(G * d * T));
    L.agg = L.memset_bytes;
    L.inc = align16(L.agg + wide * (size_t)(G * d * T) * 2 * kc);
    L.total = align16(L.inc + wide * (size_t)(G * d * T) * 2 * kc);
    return L;
}

template <dm_dtype DT, int KC>
cudaError_t launch_kc(const L1QueryArgs& a, cudaStream_t st, int64_t* launches) {
    using Cfg = QCfg<DT, KC>;
    using V = typename Types<DT>::V;
    using Wide = typename Types<DT>::Wide;
    const ScratchLayout L = scratch_layout(a.dtype, a.n, a.d, a.k);
    unsigned char* sc = static_cast<unsigned char*>(a.scratch);
    cudaError_t e = cudaMemsetAsync(sc, 0, L.memset_bytes, st);
    if (e != cudaSuccess) return e;

    QParams<V, typename Types<DT>::Acc, Wide> p;
    p.xs = static_cast<const V*>(a.xs);
    p.R = static_cast<const typename Types<DT>::Acc*>(a.R);
    p.perm = a.perm;
    p.n = a.n;
    p.d = (int)a.d;
    p.Z = static_cast<const V*>(a.Z);
    p.ldz = a.ldz;
    p.k = (int)a.k;
    p.res = static_cast<const Wide*>(a.res);
    p.mu = static_cast<const V*>(a.mu);
    p.mu_stride = a.mu_stride;
    p.out = a.out;
    p.ldo = a.ldo;
    p.counter = reinterpret_cast<uint32_t*>(sc + L.counter);
    p.done = reinterpret_cast<uint32_t*>(sc + L.done);
    p.flags = reinterpret_cast<uint32_t*>(sc + L.flags);
    p.agg = reinterpret_cast<Wide*>(sc + L.agg);
    p.inc = reinterpret_cast<Wide*>(sc + L.inc);
    p.err = a.err;
    p.T = (int)((a.n + Cfg::TILE_E - 1) / Cfg::TILE_E);
    p.G = (int)((a.k + KC - 1) / KC);
    // Widest cp.async the query rows allow.
    p.vw = (int)sizeof(V);
    const size_t rowb = (size_t)KC * sizeof(V);
    for (int cand : {16, 8}) {
        if (rowb % cand == 0 && (reinterpret_cast<uintptr_t>(a.Z) % cand) == 0 &&
            (a.ldz * sizeof(V)) % cand == 0) {
            p.vw = cand;
            break;
        }
    }

    auto kern = l1_query_kernel<DT, KC>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, Cfg::smem);
    if (e != cudaSuccess) return e;
    const int64_t total_tiles = (int64_t)p.G * p.d * p.T;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(total_tiles, (int64_t)std::max(occ, 1) * a.num_sms));
    kern<<<(unsigned)blocks, kThreads, Cfg::smem, st>>>(p);
    e = cudaGetLastError();
    if (e == cudaSuccess) ++*launches;
    return e;
}

template <dm_dtype DT>
cudaError_t launch_dt(const L1QueryArgs& a, cudaStream_t st, int64_t* launches) {
    switch (pick_kc(a.k)) {
        case 1: return launch_kc<DT, 1>(a, st, launches);
        case 2: return launch_kc<DT, 2>(a, st, launches);
        case 4: return launch_kc<DT, 4>(a, st, launches);
        case 8: return launch_kc<DT, 8>(a, st, launches);
        default: return launch_kc<DT, 16>(a, st, launches);
    }
}

}  // namespace

size_t l1_query_scratch_bytes(dm_dtype t, int64_t n, int64_t d, int64_t k) {
    return scratch_layout(t, n, d, k).total;
}

cudaError_t l1_query_launch(const L1QueryArgs& a, cudaStream_t s, int64_t* launches) {
    switch (a.dtype) {
        case DM_F32: return launch_dt<DM_F32>(a, s, launches);
        case DM_F64: return launch_dt<DM_F64>(a, s, launches);
        default: return launch_dt<DM_I32>(a, s, launches);
    }
}

}  // namespace dm
