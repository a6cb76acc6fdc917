// Reductions over the n points and the squared-l2 product.
//
// reduce  -- the shifted contraction of the query block with the points,
//              W[c,j] = sum_i (x_ic - mu_c) Z[i,j],  u[j] = sum_i Z[i,j],
//              v[j]   = sum_i s_i Z[i,j],  s_i = ||x_i - mu||^2  (squared l2),
//            i.e. [X - mu, 1, s]^T Z, a (d+2) x k result from a reduction of
//            length n: u, v and W are S1, S2 and v of the p = 2 query of
//            Appendix A (in the mu-shifted frame; the product is translation
//            invariant).  Each CTA reduces a contiguous row range: rows arrive
//            in chunks through a double-buffered cp.async pipeline, each thread
//            owns a 4 x 4 block of the result (FP32 or exact int64 over 8
//            chunks, then added in the Wide type), the CTA writes one
//            partial and a finalize kernel adds the partials in a fixed order.
//            With s omitted the same kernel gives u and W alone.
// reduce_tc -- the same contraction for FP32 on the tensor cores (tcgen05,
//            TF32 hi + lo split packed into one MMA per K step); see below.
// l2prep  -- column means mu (the frame shift), FP64 sums, fixed order.
// l2apply -- out_i = s_i u + v - 2 (x_i - mu) . W  (the p = 2 query, Appendix
//            A), s_i recomputed from the staged row with the same code as in
//            the reduce.
// The contraction does 2(d+2)k flops per (4d + 4k) bytes read (5.6 flop/byte
// at d = 32, k = 16): HBM-bound on either unit, so what decides is the
// instruction count of staging, centring and splitting the rows.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "dm_internal.h"
#include "tcgen05.h"

namespace dm {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kChunk = 128;  // rows staged in shared memory per step
constexpr int RC = 4;        // output rows (of X-hat) per thread
constexpr int RJ = 4;        // output columns (of Z) per thread

__host__ __device__ constexpr int round4(int x) { return (x + 3) & ~3; }

__device__ __forceinline__ bool finite_val(float v) { return isfinite(v); }
__device__ __forceinline__ bool finite_val(double v) { return isfinite(v); }
__device__ __forceinline__ bool finite_val(int32_t) { return true; }

__device__ __forceinline__ float to_acc(float v, float) { return v; }
__device__ __forceinline__ double to_acc(double v, double) { return v; }
__device__ __forceinline__ long long to_acc(int32_t v, long long) { return (long long)v; }
__device__ __forceinline__ long long to_acc(long long v, long long) { return v; }

template <class Acc>
__device__ __forceinline__ Acc fma_acc(Acc a, Acc b, Acc c) { return a * b + c; }
template <>
__device__ __forceinline__ float fma_acc<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <>
__device__ __forceinline__ double fma_acc<double>(double a, double b, double c) { return fma(a, b, c); }

template <int B>
__device__ __forceinline__ void cp_async(void* s, const void* g, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
    if constexpr (B == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" :: "r"(sa), "l"(g), "r"(valid ? 8 : 0) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" :: "r"(sa), "l"(g), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

// Four consecutive shared-memory elements (16-byte aligned for 4-byte types).
__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
    const float4 u = *reinterpret_cast<const float4*>(p);
    v[0] = u.x; v[1] = u.y; v[2] = u.z; v[3] = u.w;
}
__device__ __forceinline__ void load4(const double* p, double (&v)[4]) {
    const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void load4(const long long* p, long long (&v)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = p[q];
}

// s = ||x - mu||^2 of one staged row (x already shifted), by four adjacent
// lanes: lane `part` sums columns part, part + 4, ...; the four partials are
// combined as (p0 + p1) + (p2 + p3).  The reduce and the apply kernels use
// this same function, so both see identical s_i.  All 32 lanes must call it.
template <class Acc>
__device__ __forceinline__ Acc row_sqnorm4(const Acc* xrow, int d, int part) {
    Acc a = 0;
    for (int c = part; c < d; c += 4) a = fma_acc(xrow[c], xrow[c], a);
    a += __shfl_xor_sync(0xffffffffu, a, 1);
    a += __shfl_xor_sync(0xffffffffu, a, 2);
    return a;
}

// Calls f(r, c) for every (row, column) of a rows x w block, the columns of
// a row on adjacent threads, with one division per thread instead of one per
// element: thread t takes column t % w of rows t / w, t / w + 256 / w, ...
// (w <= 256), or columns t, t + 256, ... of every row (w > 256).
template <class F>
__device__ __forceinline__ void for_each_rc(int rows, int w, F&& f) {
    if (w <= kThreads) {
        const int per = kThreads / w;
        if (threadIdx.x >= per * w) return;
        const int c = threadIdx.x % w;
        for (int r = threadIdx.x / w; r < rows; r += per) f(r, c);
    } else {
        for (int r = 0; r < rows; ++r)
            for (int c = threadIdx.x; c < w; c += kThreads) f(r, c);
    }
}

__device__ __forceinline__ void cp_async16(void* s, const void* g, int bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(sa), "l"(g), "r"(bytes) : "memory");
}

// Copy rows [base, base + nr) of a row-major matrix (w elements of type T per
// row, leading dimension ld) into a dense [kChunk or R][w] shared buffer: as
// 16-byte pieces when every row start is 16-byte aligned (vec16), else one
// element at a time.  Rows past nr are zero-filled.
template <class T>
__device__ __forceinline__ void stage_rows(T* dst, const T* src, int64_t ld, int w, int64_t base,
                                           int rows, int nr, bool vec16) {
    if (vec16) {
        const int pr = w * (int)sizeof(T) / 16;    // pieces per row
        for_each_rc(rows, pr, [&](int r, int q) {
            const bool ok = r < nr;
            cp_async16(reinterpret_cast<char*>(dst + r * w) + 16 * q,
                       reinterpret_cast<const char*>(src + (ok ? (base + r) * ld : 0)) + 16 * q,
                       ok ? 16 : 0);
        });
    } else {
        for_each_rc(rows, w, [&](int r, int c) {
            const bool ok = r < nr;
            cp_async<sizeof(T)>(dst + r * w + c, src + (ok ? (base + r) * ld + c : 0), ok);
        });
    }
}

// The same with a destination row pitch (elements) larger than the width:
// 16-byte copies need w and the pitch to be whole 16-byte pieces.
template <class T>
__device__ __forceinline__ void stage_rows_pitched(T* dst, int pitch, const T* src, int64_t ld, int w,
                                                   int64_t base, int rows, int nr, bool vec16) {
    if (vec16) {
        const int pr = w * (int)sizeof(T) / 16;
        for_each_rc(rows, pr, [&](int r, int q) {
            const bool ok = r < nr;
            cp_async16(reinterpret_cast<char*>(dst + r * pitch) + 16 * q,
                       reinterpret_cast<const char*>(src + (ok ? (base + r) * ld : 0)) + 16 * q,
                       ok ? 16 : 0);
        });
    } else {
        for_each_rc(rows, w, [&](int r, int c) {
            const bool ok = r < nr;
            cp_async<sizeof(T)>(dst + r * pitch + c, src + (ok ? (base + r) * ld + c : 0), ok);
        });
    }
}

// Stage rows [base, base + nr) of X and Z (raw element types) into one buffer.
template <class XT, class V>
__device__ __forceinline__ void stage_chunk(XT* xr, V* zr, const XT* X, int64_t ldx, int d,
                                            const V* Z, int64_t ldz, int k, int64_t base, int nr,
                                            bool xv16, bool zv16) {
    stage_rows(xr, X, ldx, d, base, kChunk, nr, xv16);
    stage_rows(zr, Z, ldz, k, base, kChunk, nr, zv16);
    cp_commit();
}

template <dm_dtype DT, class XT, int MAXOB>
__global__ void __launch_bounds__(kThreads)
reduce_kernel(const XT* __restrict__ X, int64_t n, int d, int64_t ldx,
              const typename Types<DT>::V* __restrict__ mu, int64_t mu_stride, int with_s,
              const typename Types<DT>::V* __restrict__ Z, int k, int64_t ldz,
              typename Types<DT>::Wide* __restrict__ partial, int64_t rows_per_block,
              int xv16, int zv16) {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    using Wide = typename Types<DT>::Wide;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int D2 = d + 2;
    const int D2P = round4(D2), KP = round4(k);   // 16-byte aligned rows, zero padded
    // layout: raw buffers [2][kChunk*d] XT, [2][kChunk*k] V; xh [kChunk][D2P] Acc;
    //         zc [kChunk][KP] Acc; mu_s [d] Acc; red [D2*k] Wide
    size_t off = 0;
    XT* xraw = reinterpret_cast<XT*>(smem_raw + off);
    off += ((2 * (size_t)kChunk * d * sizeof(XT)) + 15) & ~size_t(15);
    V* zraw = reinterpret_cast<V*>(smem_raw + off);
    off += ((2 * (size_t)kChunk * k * sizeof(V)) + 15) & ~size_t(15);
    Acc* xh = reinterpret_cast<Acc*>(smem_raw + off);
    off += (((size_t)kChunk * D2P * sizeof(Acc)) + 15) & ~size_t(15);
    Acc* zc = reinterpret_cast<Acc*>(smem_raw + off);
    off += (((size_t)kChunk * KP * sizeof(Acc)) + 15) & ~size_t(15);
    Acc* mu_s = reinterpret_cast<Acc*>(smem_raw + off);
    off += (((size_t)d * sizeof(Acc)) + 15) & ~size_t(15);
    Wide* red = reinterpret_cast<Wide*>(smem_raw + off);

    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min64(n, r0 + rows_per_block);
    for (int c = threadIdx.x; c < d; c += kThreads) mu_s[c] = mu ? to_acc(mu[c * mu_stride], Acc()) : Acc(0);

    const int OBc = (D2 + RC - 1) / RC, OBj = (k + RJ - 1) / RJ;
    const int OB = OBc * OBj;
    const int RG = max(1, kThreads / OB);          // row groups
    const int ob_per_thread = (OB + kThreads - 1) / kThreads;
    const int my_rg = (OB >= kThreads) ? 0 : threadIdx.x / OB;

    // Block sums stay in the element type for kFlush chunks, then go into the
    // Wide accumulators (the FP64 pipe is far narrower than FP32).
    constexpr int kFlush = 8;
    Wide wacc[MAXOB][RC][RJ];
    Acc cacc[MAXOB][RC][RJ];
#pragma unroll
    for (int b = 0; b < MAXOB; ++b)
#pragma unroll
        for (int a = 0; a < RC; ++a)
#pragma unroll
            for (int q = 0; q < RJ; ++q) { wacc[b][a][q] = 0; cacc[b][a][q] = 0; }

    // This thread's output blocks (fixed for the whole row range).
    bool bact[MAXOB];
    int bcb[MAXOB], bjb[MAXOB];
#pragma unroll
    for (int b = 0; b < MAXOB; ++b) {
        const int ob = (OB >= kThreads) ? threadIdx.x + b * kThreads : threadIdx.x % OB;
        bact[b] = b < ob_per_thread && ob < OB && my_rg < RG;
        bcb[b] = (ob / OBj) * RC;
        bjb[b] = (ob % OBj) * RJ;
    }

    const int nchunks = (int)((r1 - r0 + kChunk - 1) / kChunk);
    if (nchunks > 0)
        stage_chunk(xraw, zraw, X, ldx, d, Z, ldz, k, r0, (int)min64(kChunk, r1 - r0), xv16, zv16);
    for (int ch = 0; ch < nchunks; ++ch) {
        const int64_t base = r0 + (int64_t)ch * kChunk;
        const int nr = (int)min64(kChunk, r1 - base);
        const int buf = ch & 1;
        if (ch + 1 < nchunks) {
            const int64_t nb = base + kChunk;
            stage_chunk(xraw + (buf ^ 1) * kChunk * d, zraw + (buf ^ 1) * kChunk * k, X, ldx, d, Z,
                        ldz, k, nb, (int)min64(kChunk, r1 - nb), xv16, zv16);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
        const XT* xb = xraw + buf * kChunk * d;
        const V* zb = zraw + buf * kChunk * k;
        for_each_rc(kChunk, d, [&](int r, int c) {
            xh[r * D2P + c] = (r < nr) ? to_acc(xb[r * d + c], Acc()) - mu_s[c] : Acc(0);
        });
        for_each_rc(kChunk, KP, [&](int r, int j) {
            zc[r * KP + j] = (r < nr && j < k) ? to_acc(zb[r * k + j], Acc()) : Acc(0);
        });
        __syncthreads();
        static_assert(kChunk % (kThreads / 4) == 0, "four lanes per staged row");
        for (int r = threadIdx.x >> 2; r < kChunk; r += kThreads / 4) {
            const int part = threadIdx.x & 3;
            const Acc sq = row_sqnorm4(xh + r * D2P, d, part);
            if (part == 0) {
                xh[r * D2P + d] = r < nr ? Acc(1) : Acc(0);
                xh[r * D2P + d + 1] = (with_s && r < nr) ? sq : Acc(0);
            } else if (D2 + part - 1 < D2P) {
                xh[r * D2P + D2 + part - 1] = Acc(0);   // padding columns
            }
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < MAXOB; ++b) {
            if (!bact[b]) continue;
            const int cb = bcb[b], jb = bjb[b];
            for (int r = my_rg; r < kChunk; r += RG) {
                Acc xv[RC], zv[RJ];
                load4(xh + r * D2P + cb, xv);
                load4(zc + r * KP + jb, zv);
#pragma unroll
                for (int a = 0; a < RC; ++a)
#pragma unroll
                    for (int q = 0; q < RJ; ++q) cacc[b][a][q] = fma_acc(xv[a], zv[q], cacc[b][a][q]);
            }
        }
        if ((ch + 1) % kFlush == 0 || ch + 1 == nchunks) {
#pragma unroll
            for (int b = 0; b < MAXOB; ++b)
#pragma unroll
                for (int a = 0; a < RC; ++a)
#pragma unroll
                    for (int q = 0; q < RJ; ++q) { wacc[b][a][q] += (Wide)cacc[b][a][q]; cacc[b][a][q] = 0; }
        }
        __syncthreads();
    }

    // Combine the row groups in a fixed order and write this block's partial.
    const int total = D2 * k;
    for (int i = threadIdx.x; i < total; i += kThreads) red[i] = 0;
    __syncthreads();
    for (int rg = 0; rg < RG; ++rg) {
        if (my_rg == rg) {
#pragma unroll
            for (int b = 0; b < MAXOB; ++b) {
                if (b >= ob_per_thread) break;
                const int ob = (OB >= kThreads) ? threadIdx.x + b * kThreads : threadIdx.x % OB;
                if (ob >= OB) continue;
                const int cb = (ob / OBj) * RC, jb = (ob % OBj) * RJ;
#pragma unroll
                for (int a = 0; a < RC; ++a)
#pragma unroll
                    for (int q = 0; q < RJ; ++q)
                        if (cb + a < D2 && jb + q < k) red[(cb + a) * k + jb + q] += wacc[b][a][q];
            }
        }
        __syncthreads();
    }
    Wide* out = partial + (int64_t)blockIdx.x * total;
    for (int i = threadIdx.x; i < total; i += kThreads) out[i] = red[i];
}

// One warp per result entry; lanes stride over the partials and the warp
// tree-reduces them (a fixed order, so the result is reproducible).
// With a device error word (the tensor-core reduce): partials of a launch
// whose bounded wait ran out may be stale, so once the word holds
// DM_ERR_TIMEOUT the result is poisoned (NaN) instead of summed.
template <class Wide>
__global__ void reduce_finalize_kernel(const Wide* __restrict__ partial, int blocks, int total,
                                       Wide* __restrict__ res, const uint32_t* err) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= total) return;
    if constexpr (sizeof(Wide) == 8 && Wide(0.5) != Wide(0)) {   // floating point only
        if (err && ld_acquire(err) == kErrTimeout) {
            if (lane == 0) res[w] = __longlong_as_double(0x7ff8000000000000ll);
            return;
        }
    }
    Wide acc = 0;
    for (int b = lane; b < blocks; b += 32) acc += partial[(int64_t)b * total + w];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) res[w] = acc;
}

// ----------------------------------------------------------------- l2prep
// Column sums of X per block (Wide), then mu = sum / n rounded to V.
template <dm_dtype DT>
__global__ void __launch_bounds__(kThreads)
colsum_kernel(const typename Types<DT>::V* __restrict__ X, int64_t n, int d, int64_t ldx,
              typename Types<DT>::Wide* __restrict__ partial, int64_t rows_per_block,
              uint32_t* err) {
    using Wide = typename Types<DT>::Wide;
    using V = typename Types<DT>::V;
    constexpr int U = 16;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min64(n, r0 + rows_per_block);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Wide* red = reinterpret_cast<Wide*>(smem_raw);
    // Thread (column c0, row group g) walks rows g, g + rg, ... of its range,
    // U rows per step with all U loads issued first.
    const int cols = min(d, kThreads);
    const int rg = kThreads / cols;
    const int c0 = threadIdx.x % cols, g = threadIdx.x / cols;
    bool bad = false;
    for (int cb = 0; cb < d; cb += cols) {
        const int c = cb + c0;
        Wide acc = 0;
        if (g < rg && c < d) {
            for (int64_t r = r0 + g; r < r1; r += (int64_t)rg * U) {
                V v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t rr = r + (int64_t)u * rg;
                    v[u] = rr < r1 ? X[rr * ldx + c] : V(0);
                }
                // U values summed in the element type, then one Wide add (the
                // FP64 pipe is far narrower than FP32 on this GPU).
                V part = V(0);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    bad |= !finite_val(v[u]);
                    part += v[u];
                }
                acc += (Wide)part;
            }
        }
        red[threadIdx.x] = acc;
        __syncthreads();
        if (g == 0 && c < d) {
            Wide t = 0;
            for (int q = 0; q < rg; ++q) t += red[q * cols + c0];
            partial[(int64_t)blockIdx.x * d + c] = t;
        }
        __syncthreads();
    }
    if (bad && err) set_error(err, kErrNonfinite);
}

template <dm_dtype DT>
__global__ void mean_finalize_kernel(const typename Types<DT>::Wide* __restrict__ partial,
                                     int blocks, int d, int64_t n,
                                     typename Types<DT>::V* __restrict__ mu) {
    using Wide = typename Types<DT>::Wide;
    using V = typename Types<DT>::V;
    // One warp per column: lanes stride over the block partials, then a
    // shuffle tree in a fixed order (the result does not depend on timing).
    const int c = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= d) return;
    Wide t = 0;
    for (int b = lane; b < blocks; b += 32) t += partial[(int64_t)b * d + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) mu[c] = (V)(t / (Wide)n);
}

// ------------------------------------------------- l2apply on tensor cores
// FP32 data, d <= 32 coordinates (a multiple of 4, rows contiguous), k <= 32
// query columns: the apply's contraction -2 (X - mu) W on tcgen05.mma
// (kind::tf32), one MMA tile of M = 128 points, N = k rounded up to 16,
// K = d rounded up to 8.  This is the product's natural orientation: a
// point's coordinates are its K dimension and lie contiguous in X, so the
// operand is X's own row-major tile (K-major), shifted and split on the way.
//   A: 128 x Kp, rows of [x_i - mu] split as v = hi + lo (split_tf32: both
//      parts exact TF32 values, |v - hi - lo| < 2^-20 |v|);
//   B: Np x Kp, the columns of W (W^T), split the same way once per CTA;
//   D (TMEM, lane = point, column = query column) = A_hi B_hi + A_hi B_lo
//      + A_lo B_hi: three MMAs per K step of 8 (FP32 accumulation over at
//      most 12 products).
// Operands sit in the canonical K-major layout without swizzle.
// Each CTA is persistent over tiles j = blockIdx.x + i gridDim.x, in two
// roles: one thread (warp 8) keeps kApStages raw tiles (128 rows x d
// floats, contiguous) on their way by bulk copies (cp.async.bulk, completion
// counted on an mbarrier), and for each tile waits until the workers have
// filled its operand set, issues its MMAs into accumulator j % 2 and commits
// them to that set's mbarrier; eight worker warps, per tile, wait for the
// raw tile and for the MMAs of the tile two back (which read operand set
// j % 2 and wrote accumulator j % 2), start the TMEM loads of that
// accumulator, shift and split their rows into the set (threads 2r, 2r + 1
// share row r) and form s_i = ||x_i - mu||^2 by halves, meet on a named
// barrier (the row norms of a tile reach the threads that write its out),
// then write out_i = s_i u + v - 2 D_i of the tile two back (threads t and
// t + 128 share point t, TMEM lane t, each with half of the query columns)
// and arrive on the set's mbarrier.
// Every wait is bounded: on expiry a thread sets the CTA's abort word, which
// ends every other wait; the CTA latches DM_ERR_TIMEOUT, waits (bounded) for
// its own copies and MMAs in flight, frees its TMEM and exits.
constexpr int kApM = 128;
constexpr int kApW = 8;                  // worker warps: two threads per point (row) of a tile
constexpr int kApWT = 32 * kApW;
constexpr int kApT = kApWT + 32;         // and one warp that issues the copies and MMAs
constexpr int kApStages = 2;

size_t apply_tc_smem(int d, int k) {
    const int Kp = (d + 7) / 8 * 8, Np = (k + 15) / 16 * 16;
    return kApStages * (size_t)kApM * d * 4    // raw tiles
           + 4 * (size_t)kApM * Kp * 4         // two operand sets (hi, lo)
           + 2 * (size_t)Np * Kp * 4           // B (hi, lo)
           + 4 * (2 * (size_t)Np + Kp)         // mu, u, v
           + 8 * (size_t)kApM * 4              // partial row norms of four tiles
           + 8 * (kApStages + 4) + 32;         // mbarriers, abort word, TMEM slot, alignment
}

// --------------------------------------------------- reduce on tensor cores
// FP32 data, d a multiple of 4 up to 60, k a multiple of 4 up to 32, rows of
// X and Z contiguous: the contraction [X - mu, 1, s]^T Z on tcgen05.mma
// (kind::tf32).  The contraction index K runs over the points, KC per chunk
// and 8 per instruction; the threads write both operands in the canonical
// K-major layout without swizzle -- element (r, p) at byte (r / 8) SBO +
// (p / 4) 128 + (r % 8) 16 + (p % 4) 4, SBO = KC / 4 * 128 -- transposing
// the row-major raw chunk on the way.
// Split precision in one MMA per K step: every value is split as
// v = hi + lo (split_tf32), A's rows are [Y_hi; Y_lo] with Y = [X - mu, 1,
// s]^T (rows 0 .. D2 - 1 and D2 .. 2 D2 - 1, D2 = d + 2) and B's rows are
// [Z_hi; Z_lo] (Kp = k rounded up to 8 rows each), so the accumulator
// D = A B^T (M = 128, N = 2 Kp) holds the four partial products
//   D[r][j] = Y_hi Z_hi,        D[r][Kp + j] = Y_hi Z_lo,
//   D[D2 + r][j] = Y_lo Z_hi,   D[D2 + r][Kp + j] = Y_lo Z_lo,
// whose sum is the product to about 2^-20 of each term.  Rows of A from
// 2 D2 on and rows of B past k in each half are never written: they reach
// only accumulator rows and columns that are never read.  When the unused
// 8-row groups of A have room for B, B lives there.
// Sums: the tensor core's FP32 accumulation drifts with the number of
// accumulations, so one accumulator takes one chunk (KC / 8 MMAs); two
// accumulators in TMEM alternate, and while the next chunk runs the threads
// add a finished one into FP32 registers (warp w: accumulator rows
// 32 (w % 4) .. + 31, column half w / 4), every kRtFlush chunks into the
// CTA's FP64 sums in shared memory, and at the end the four products of
// each entry go into the CTA's FP64 partial; reduce_finalize adds the
// partials in a fixed order.
// Pipeline (each CTA a contiguous range of chunks), by role:
//   one thread (warp 8) keeps STAGES raw chunks (the rows of X and Z, both
//     contiguous) on their way by bulk copies, and for each chunk waits until
//     the workers have filled its operand set, issues its KC / 8 MMAs into
//     accumulator c % 2 and commits them to that set's mbarrier; a consumed
//     raw stage is refilled at once;
//   eight worker warps wait for raw chunk c and for the MMAs of chunk c - 2
//     (which read operand set c % 2 and wrote accumulator c % 2), start the
//     TMEM loads of that accumulator, shift, split and transpose chunk c into
//     the set, add the loaded accumulator into their registers and arrive on
//     the set's mbarrier.
// No CTA-wide barrier inside the loop: the roles meet on mbarriers only.
// Every wait is bounded: on expiry a thread sets the CTA's abort word, which
// ends every other wait; the CTA latches DM_ERR_TIMEOUT, waits (bounded) for
// its own copies and MMAs in flight, frees its TMEM and exits.
constexpr int kRtW = 8;                  // worker warps
constexpr int kRtWT = 32 * kRtW;         // worker threads
constexpr int kRtT = kRtWT + 32;         // and one warp that issues the copies and MMAs
constexpr int kRtFlush = 16;             // chunks per FP32 register run

// CTAs per SM the launch is built for (its register bound): up to 16 query
// columns three with 32-point chunks, two with 64; wider blocks one (their
// registers would spill at two).
__host__ __device__ constexpr int rt_min_blocks(int KC, int KPM) { return KPM <= 16 ? (KC == 32 ? 3 : 2) : 1; }

// Byte layout of one CTA's shared memory (host and device).
struct RtShape {
    int Kp, N, D2;
    uint32_t sbo, b_off, set_bytes, raw_x, raw_bytes, acc_off, mu_off, bar_off, total;
};

__host__ __device__ inline RtShape rt_shape(int KC, int stages, int d, int k) {
    RtShape s;
    s.Kp = (k + 7) / 8 * 8;
    s.N = 2 * s.Kp;
    s.D2 = d + 2;
    s.sbo = (uint32_t)(KC / 4) * 128u;
    const uint32_t used = (uint32_t)(2 * s.D2 + 7) / 8;   // 8-row groups of A with data
    const uint32_t bgroups = (uint32_t)s.N / 8;
    const bool inside = used + bgroups <= 16;
    s.b_off = (inside ? used : 16u) * s.sbo;
    s.set_bytes = (inside ? 16u : 16u + bgroups) * s.sbo;
    s.raw_x = (uint32_t)(KC * d * 4);
    s.raw_bytes = (uint32_t)(KC * (d + k) * 4);
    s.acc_off = 2 * s.set_bytes + (uint32_t)stages * s.raw_bytes;
    s.mu_off = s.acc_off + (uint32_t)(2 * s.D2 * s.N) * 8u;
    s.bar_off = s.mu_off + ((uint32_t)d * 4u + 15u) / 16u * 16u;
    s.total = s.bar_off + 8u * (uint32_t)(stages + 4) + 16u;
    return s;
}

// Four points of one operand row: shift (X only), split, and store hi and lo
// as 16-byte pieces of their rows.  FULL: all four points exist.
template <bool FULL>
__device__ __forceinline__ void rt_put4(unsigned char* base, const float* src, int stride, float shift,
                                        int p0, int nr, uint32_t off_hi, uint32_t off_lo) {
    float h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float v = (FULL || p0 + e < nr) ? src[e * stride] - shift : 0.f;
        split_tf32(v, h[e], l[e]);
    }
    *reinterpret_cast<float4*>(base + off_hi) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4*>(base + off_lo) = make_float4(l[0], l[1], l[2], l[3]);
}

template <int KC, int STAGES, int KPM>
__global__ void __launch_bounds__(kRtT, rt_min_blocks(KC, KPM))
reduce_tc_kernel(const float* __restrict__ X, int64_t n, int d, const float* __restrict__ mu,
                 int64_t mu_stride, int with_s, const float* __restrict__ Z, int k,
                 double* __restrict__ partial, uint32_t tmem_cols, uint32_t* err, uint32_t spin_limit) {
    constexpr int G4 = KC / 4;             // 4-point groups per chunk
    constexpr int MQX = KC / 16;           // X items per worker thread (d <= 64)
    constexpr int MQZ = KC / 32;           // Z items per worker thread (k <= 32)
    constexpr int TPP = kRtWT / KC;        // worker threads per point forming s
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const RtShape S = rt_shape(KC, STAGES, d, k);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int D2 = S.D2, Kp = S.Kp, N = S.N;
    const uint32_t sbo = S.sbo;
    unsigned char* raw = smem_raw + 2 * S.set_bytes;
    // FP64 sums, column-major [N][2 D2]: the lanes of a warp (adjacent rows)
    // touch adjacent words
    double* acc64 = reinterpret_cast<double*>(smem_raw + S.acc_off);
    float* mu_s = reinterpret_cast<float*>(smem_raw + S.mu_off);        // [d]
    // mbarriers: raw_full[STAGES] (the copies), op_full[2] (the workers'
    // splits), mma_done[2] (the MMAs' commits); then the abort word and the
    // TMEM address
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw + S.bar_off);
    uint64_t* raw_full = mbar;
    uint64_t* op_full = mbar + STAGES;
    uint64_t* mma_done = mbar + STAGES + 2;
    volatile uint32_t* abort_w = reinterpret_cast<volatile uint32_t*>(mbar + STAGES + 4);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + STAGES + 4) + 1;

    for (int i = tid; i < 2 * D2 * N; i += kRtT) acc64[i] = 0.0;
    for (int c = tid; c < d; c += kRtT) mu_s[c] = mu ? mu[c * mu_stride] : 0.f;
    // the row of ones (hi 1, lo 0) of both operand sets stays as written:
    // points past n meet rows of Z that are zero
    for (int i = tid; i < 2 * KC; i += kRtT) {
        unsigned char* A = smem_raw + (i / KC) * S.set_bytes;
        const int p = i % KC, rl = D2 + d;
        const uint32_t po = (uint32_t)(p >> 2) * 128u + (uint32_t)(p & 3) * 4u;
        *reinterpret_cast<float*>(A + (uint32_t)(d >> 3) * sbo + (uint32_t)(d & 7) * 16u + po) = 1.f;
        *reinterpret_cast<float*>(A + (uint32_t)(rl >> 3) * sbo + (uint32_t)(rl & 7) * 16u + po) = 0.f;
    }
    if (tid == 0) {
        for (int b = 0; b < STAGES; ++b) mbar_init(smem_u32(raw_full + b), 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(op_full + b), kRtWT);
            mbar_init(smem_u32(mma_done + b), 1);
        }
        *abort_w = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kRtW) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tslot)), "r"(tmem_cols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    const int64_t C = (n + KC - 1) / KC;
    const int64_t c0 = C * blockIdx.x / gridDim.x, c1 = C * (blockIdx.x + 1) / gridDim.x;
    const int64_t my = c1 - c0;
    int64_t issued = 0, committed = 0;   // the copy/MMA thread's chunks in flight

    if (warp < kRtW) {
        // ---------------------------------------------------------- workers
        // This thread's split items, fixed for every chunk: X item q is
        // (coordinate f, point group g) = (it % d, it / d), it = tid + q kRtWT
        // (a warp's items are adjacent coordinates: conflict-free reads of the
        // raw rows and 16-byte writes to eight distinct bank groups); Z item q
        // the same over the k columns.
        int xsrc[MQX], xg[MQX];
        uint32_t xhi[MQX], xlo[MQX];
        float xmu[MQX];
#pragma unroll
        for (int q = 0; q < MQX; ++q) {
            const int it = tid + q * kRtWT;
            const int f = it % d, g = it / d, rl = D2 + f;
            xg[q] = it < d * G4 ? 4 * g : -1;
            xsrc[q] = 4 * g * d + f;
            xhi[q] = (uint32_t)(f >> 3) * sbo + (uint32_t)g * 128u + (uint32_t)(f & 7) * 16u;
            xlo[q] = (uint32_t)(rl >> 3) * sbo + (uint32_t)g * 128u + (uint32_t)(rl & 7) * 16u;
            xmu[q] = mu_s[f];
        }
        int zsrc[MQZ], zg[MQZ];
        uint32_t zhi[MQZ], zlo[MQZ];
#pragma unroll
        for (int q = 0; q < MQZ; ++q) {
            const int it = tid + q * kRtWT;
            const int j = it % k, g = it / k;
            zg[q] = it < k * G4 ? 4 * g : -1;
            zsrc[q] = 4 * g * k + j;
            zhi[q] = S.b_off + (uint32_t)(j >> 3) * sbo + (uint32_t)g * 128u + (uint32_t)(j & 7) * 16u;
            zlo[q] = zhi[q] + (uint32_t)(Kp >> 3) * sbo;
        }
        // s: TPP adjacent threads per point, each a share of its 16-byte
        // pieces, the pieces rotated so that the eight lanes of a 16-byte
        // access phase read distinct bank groups
        const int sp = tid / TPP, spart = tid % TPP, nq = d / 4, srot = (sp * TPP) % nq;
        const uint32_t s_po = (uint32_t)(sp >> 2) * 128u + (uint32_t)(sp & 3) * 4u;
        const uint32_t s_hi = (uint32_t)((d + 1) >> 3) * sbo + (uint32_t)((d + 1) & 7) * 16u + s_po;
        const uint32_t s_lo = (uint32_t)((D2 + d + 1) >> 3) * sbo + (uint32_t)((D2 + d + 1) & 7) * 16u + s_po;

        const int hw = warp >> 2;                         // column half of the accumulator
        const int arow = 32 * (warp & 3) + lane;          // accumulator row
        const bool dwarp = 32 * (warp & 3) < 2 * D2;      // the warp's rows hold data
        float facc[KPM];
#pragma unroll
        for (int j = 0; j < KPM; ++j) facc[j] = 0.f;
        int run = 0;
        uint32_t r[KPM];
        auto flush = [&]() {
            if (dwarp && arow < 2 * D2) {
                double* dst = acc64 + (hw * Kp) * (2 * D2) + arow;
#pragma unroll
                for (int j = 0; j < KPM; ++j)
                    if (j < Kp) dst[j * (2 * D2)] += (double)facc[j];
            }
#pragma unroll
            for (int j = 0; j < KPM; ++j) facc[j] = 0.f;
            run = 0;
        };
        // TMEM loads of accumulator b (its MMAs are known to be complete);
        // tc_drain_add adds them once they have arrived
        auto tc_drain_issue = [&](int b) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (dwarp) {
                const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(b * N + hw * Kp);
#pragma unroll
                for (int t = 0; t < KPM / 8; ++t)
                    if (t * 8 < Kp) tc_ld8_issue(ta + (uint32_t)(8 * t), r + 8 * t);
            }
        };
        auto tc_drain_add = [&]() {
            if (dwarp) {
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int t = 0; t < KPM / 8; ++t)
                    if (t * 8 < Kp)
#pragma unroll
                        for (int e = 0; e < 8; ++e) facc[8 * t + e] += __uint_as_float(r[8 * t + e]);
            }
            if (++run == kRtFlush) flush();
        };

        bool ok = true;
        for (int64_t i = 0; i < my; ++i) {
            const int st = (int)(i % STAGES), ob = (int)(i & 1);
            const int nr = (int)min64(KC, n - (c0 + i) * KC);
            // the raw chunk is in place, and operand set ob is free once the
            // MMAs of chunk i - 2 are done (their accumulator is drained
            // around the split); a warp agrees on the outcome (the TMEM loads
            // are warp-wide)
            ok = mbar_wait_ab(smem_u32(raw_full + st), (uint32_t)(i / STAGES) & 1u, spin_limit, abort_w);
            if (ok && i >= 2)
                ok = mbar_wait_ab(smem_u32(mma_done + ob), (uint32_t)((i - 2) >> 1) & 1u, spin_limit, abort_w);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            if (i >= 2) tc_drain_issue(ob);
            const float* rx = reinterpret_cast<const float*>(raw + (size_t)st * S.raw_bytes);
            const float* rz = reinterpret_cast<const float*>(raw + (size_t)st * S.raw_bytes + S.raw_x);
            unsigned char* A = smem_raw + ob * S.set_bytes;
            if (nr == KC) {
#pragma unroll
                for (int q = 0; q < MQX; ++q)
                    if (xg[q] >= 0) rt_put4<true>(A, rx + xsrc[q], d, xmu[q], xg[q], nr, xhi[q], xlo[q]);
#pragma unroll
                for (int q = 0; q < MQZ; ++q)
                    if (zg[q] >= 0) rt_put4<true>(A, rz + zsrc[q], k, 0.f, zg[q], nr, zhi[q], zlo[q]);
            } else {
#pragma unroll
                for (int q = 0; q < MQX; ++q)
                    if (xg[q] >= 0) rt_put4<false>(A, rx + xsrc[q], d, xmu[q], xg[q], nr, xhi[q], xlo[q]);
#pragma unroll
                for (int q = 0; q < MQZ; ++q)
                    if (zg[q] >= 0) rt_put4<false>(A, rz + zsrc[q], k, 0.f, zg[q], nr, zhi[q], zlo[q]);
            }
            {
                float sacc = 0.f;
                if (with_s) {
                    const float* xrow = rx + sp * d;
                    for (int qq = spart; qq < nq; qq += TPP) {
                        int q = qq + srot;
                        if (q >= nq) q -= nq;
                        const float4 x4 = *reinterpret_cast<const float4*>(xrow + 4 * q);
                        const float4 m4 = *reinterpret_cast<const float4*>(mu_s + 4 * q);
                        const float y0 = x4.x - m4.x, y1 = x4.y - m4.y, y2 = x4.z - m4.z, y3 = x4.w - m4.w;
                        sacc = fmaf(y0, y0, sacc);
                        sacc = fmaf(y1, y1, sacc);
                        sacc = fmaf(y2, y2, sacc);
                        sacc = fmaf(y3, y3, sacc);
                    }
                }
#pragma unroll
                for (int o = TPP / 2; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
                if (spart == 0) {
                    float h, l;
                    split_tf32(sp < nr ? sacc : 0.f, h, l);
                    *reinterpret_cast<float*>(A + s_hi) = h;
                    *reinterpret_cast<float*>(A + s_lo) = l;
                }
            }
            if (i >= 2) tc_drain_add();
            // set ob written, raw stage st read, accumulator ob read
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(op_full + ob)) : "memory");
        }
        // the last two chunks
        for (int64_t j = my >= 2 ? my - 2 : 0; ok && j < my; ++j) {
            const int b = (int)(j & 1);
            ok = mbar_wait_ab(smem_u32(mma_done + b), (uint32_t)(j >> 1) & 1u, spin_limit, abort_w);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            tc_drain_issue(b);
            tc_drain_add();
        }
        if (!ok) *abort_w = 1u;
        flush();
    } else if (lane == 0) {
        // ---------------------------------- copies and MMAs (one thread)
        auto issue = [&](int64_t i) {   // raw chunk i of this CTA into stage i % STAGES
            const int64_t r0 = (c0 + i) * KC;
            const int nr = (int)min64(KC, n - r0);
            const int st = (int)(i % STAGES);
            const uint32_t dst = smem_u32(raw + (size_t)st * S.raw_bytes), bar = smem_u32(raw_full + st);
            const uint32_t bx = (uint32_t)(nr * d * 4), bz = (uint32_t)(nr * k * 4);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bx + bz) : "memory");
            bulk_copy(dst, X + r0 * d, bx, bar);
            bulk_copy(dst + S.raw_x, Z + r0 * k, bz, bar);
        };
        // D FP32, A and B TF32, both K-major, N, M = 128
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((128u >> 4) << 24);
        // descriptors of set 0's first K step; set 1 and each K step (256
        // bytes) add to the address field (16-byte units; shared addresses
        // stay below 2^18, so the field does not carry)
        const uint64_t da0 = tc_desc_sbo(smem_u32(smem_raw), sbo);
        const uint64_t db0 = tc_desc_sbo(smem_u32(smem_raw) + S.b_off, sbo);
        for (; issued < STAGES && issued < my; ++issued) issue(issued);
        for (int64_t i = 0; i < my; ++i) {
            const int ob = (int)(i & 1);
            if (!mbar_wait_ab(smem_u32(op_full + ob), (uint32_t)(i >> 1) & 1u, spin_limit, abort_w)) {
                *abort_w = 1u;
                break;
            }
            // raw stage i % STAGES has been read: the chunk STAGES ahead
            if (issued < my) issue(issued++);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t so = ob ? (uint64_t)(S.set_bytes >> 4) : 0u;
            const uint32_t dcol = tmem + (uint32_t)(ob * N);
#pragma unroll
            for (int ks = 0; ks < KC / 8; ++ks)
                tc_mma(dcol, da0 + so + 16u * ks, db0 + so + 16u * ks, idesc, ks > 0 ? 1u : 0u);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(mma_done + ob)) : "memory");
            committed = i + 1;
        }
    }
    __syncthreads();
    if (*abort_w) {
        if (tid == 0 && err) set_error(err, kErrTimeout);
        // no copy or MMA of this CTA may still target its shared memory or
        // TMEM when they are released: the copy/MMA thread waits for the last
        // copy into each stage and the last commit to each set (operations
        // that complete by themselves: the long limit, whatever the
        // configured one)
        if (tid == kRtWT) {
            for (int64_t j = issued - 1; j >= 0 && j >= issued - STAGES; --j)
                mbar_wait(smem_u32(raw_full + (int)(j % STAGES)), (uint32_t)(j / STAGES) & 1u, kSpinLimit);
            for (int64_t j = committed - 1; j >= 0 && j >= committed - 2; --j)
                mbar_wait(smem_u32(mma_done + (int)(j & 1)), (uint32_t)(j >> 1) & 1u, kSpinLimit);
        }
    } else {
        double* out = partial + (int64_t)blockIdx.x * D2 * k;
        for (int e = tid; e < D2 * k; e += kRtT) {
            const int c = e / k, j = e % k;
            const double* hi = acc64 + j * (2 * D2);           // column j: products with Z_hi
            const double* lo = acc64 + (Kp + j) * (2 * D2);    // column Kp + j: with Z_lo
            out[e] = (hi[c] + lo[c]) + (hi[D2 + c] + lo[D2 + c]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == kRtW) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(tmem_cols) : "memory");
    }
}

// ------------------------------------------- l2apply on tensor cores: kernel
template <int Kp>
__global__ void __launch_bounds__(kApT, 2)
l2apply_tc_kernel(const float* __restrict__ X, int64_t n, int d, const float* __restrict__ mu,
                  const double* __restrict__ res, int k, float* __restrict__ out, int64_t ldo,
                  int Np, uint32_t tmem_cols, int vst, uint32_t* err, uint32_t spin_limit) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t sbo = (uint32_t)(Kp / 4) * 128u;
    const size_t raw_bytes = (size_t)kApM * d * 4;
    const size_t a_bytes = (size_t)kApM * Kp * 4, b_bytes = (size_t)Np * Kp * 4;
    unsigned char* raw = smem_raw;                                     // [kApStages][128][d]
    unsigned char* aset = raw + kApStages * raw_bytes;                 // [2] x (hi, lo): 128 x Kp each
    unsigned char* bhi = aset + 4 * a_bytes;
    unsigned char* blo = bhi + b_bytes;
    float* mu_s = reinterpret_cast<float*>(blo + b_bytes);             // [Kp], 16-byte aligned
    float* u_s = mu_s + Kp;                                            // [Np]
    float* v_s = u_s + Np;                                             // [Np]
    float* s_part = v_s + Np;                                          // [4 tiles][2 halves][128]
    const uintptr_t tail = (reinterpret_cast<uintptr_t>(s_part + 8 * kApM) + 7) & ~uintptr_t(7);
    // mbarriers raw_full[kApStages], op_full[2], mma_done[2]; the abort word;
    // the TMEM address
    uint64_t* mbar = reinterpret_cast<uint64_t*>(tail);
    uint64_t* raw_full = mbar;
    uint64_t* op_full = mbar + kApStages;
    uint64_t* mma_done = mbar + kApStages + 2;
    volatile uint32_t* abort_w = reinterpret_cast<volatile uint32_t*>(mbar + kApStages + 4);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + kApStages + 4) + 1;

    // B = W^T split, u, v, mu (zero padded)
    for (int i = tid; i < Np * Kp; i += kApT) {
        const int nn = i / Kp, kk = i % Kp;
        const float w = (nn < k && kk < d) ? (float)res[(int64_t)kk * k + nn] : 0.f;
        float h, l;
        split_tf32(w, h, l);
        const size_t off = (size_t)(nn >> 3) * sbo + (size_t)(kk >> 2) * 128 + (size_t)(nn & 7) * 16 +
                           (size_t)(kk & 3) * 4;
        *reinterpret_cast<float*>(bhi + off) = h;
        *reinterpret_cast<float*>(blo + off) = l;
    }
    for (int j = tid; j < Np; j += kApT) {
        u_s[j] = j < k ? (float)res[(int64_t)d * k + j] : 0.f;
        v_s[j] = j < k ? (float)res[(int64_t)d * k + k + j] : 0.f;
    }
    for (int c = tid; c < Kp; c += kApT) mu_s[c] = c < d ? mu[c] : 0.f;
    if (tid == 0) {
        for (int b = 0; b < kApStages; ++b) mbar_init(smem_u32(raw_full + b), 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(op_full + b), kApWT);
            mbar_init(smem_u32(mma_done + b), 1);
        }
        *abort_w = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kApW) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tslot)), "r"(tmem_cols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    const int64_t tiles = (n + kApM - 1) / kApM;
    auto tile_rows = [&](int64_t tile) { return (int)min64(kApM, n - tile * kApM); };
    const int64_t my_tiles = blockIdx.x < tiles ? (tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    int64_t issued = 0, committed = 0;   // the copy/MMA thread's tiles in flight

    if (warp < kApW) {
        // ---------------------------------------------------------- workers
        const int row = tid & (kApM - 1), half = tid >> 7;   // epilogue: TMEM lane, column half
        const int srow = tid >> 1, shalf = tid & 1;          // split: row, coordinate half
        const int jh = Np / 2;
        uint32_t r[16];
        // TMEM loads of accumulator b (its MMAs are complete): this thread's
        // row, its half of the columns
        auto acc_issue = [&](int b) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ta = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(b * Np + half * jh);
#pragma unroll
            for (int t = 0; t < 2; ++t)
                if (t * 8 < jh) tc_ld8_issue(ta + (uint32_t)(8 * t), r + 8 * t);
        };
        // out for tile j from the loaded accumulator and its row norms
        auto epilogue = [&](int64_t j) {
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int64_t tile = blockIdx.x + j * gridDim.x;
            const int rows = tile_rows(tile);
            const float* sp = s_part + (int)(j & 3) * 2 * kApM;
            const float s_row = sp[row] + sp[kApM + row];
            if (row < rows) {
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    if (t * 8 >= jh) continue;
                    const int j0 = half * jh + 8 * t;
                    float o[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        o[q] = fmaf(s_row, u_s[j0 + q], v_s[j0 + q]) - 2.f * __uint_as_float(r[8 * t + q]);
                    float* dst = out + (tile * kApM + row) * ldo + j0;
                    if (vst && j0 + 8 <= k) {
                        *reinterpret_cast<float4*>(dst) = make_float4(o[0], o[1], o[2], o[3]);
                        *reinterpret_cast<float4*>(dst + 4) = make_float4(o[4], o[5], o[6], o[7]);
                    } else {
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            if (j0 + q < k) dst[q] = o[q];
                    }
                }
            }
        };
        bool ok = true;
        for (int64_t i = 0; i < my_tiles; ++i) {
            const int st = (int)(i % kApStages), ob = (int)(i & 1);
            const int64_t tile = blockIdx.x + i * gridDim.x;
            const int rows = tile_rows(tile);
            // the raw tile is in place, and operand set ob and accumulator ob
            // are free once the MMAs of tile i - 2 are done (whose out is
            // written around this tile's split); a warp agrees on the outcome
            ok = mbar_wait_ab(smem_u32(raw_full + st), (uint32_t)(i / kApStages) & 1u, spin_limit, abort_w);
            if (ok && i >= 2)
                ok = mbar_wait_ab(smem_u32(mma_done + ob), (uint32_t)((i - 2) >> 1) & 1u, spin_limit, abort_w);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            if (i >= 2) acc_issue(ob);
            // shift, split and the partial s of one half of a row: threads 2r
            // and 2r + 1 share row r, so a warp's 16-byte reads of the raw rows
            // and writes of the operand rows each cover eight distinct bank groups
            {
                unsigned char* ahi = aset + (size_t)ob * 2 * a_bytes;
                unsigned char* alo = ahi + a_bytes;
                const float* xr = reinterpret_cast<const float*>(raw + (size_t)st * raw_bytes) + (size_t)srow * d;
                const size_t rbase = (size_t)(srow >> 3) * sbo + (size_t)(srow & 7) * 16;
                constexpr int nq2 = Kp / 8;                   // 16-byte pieces per half
                const int dq = d / 4;                         // pieces with data
                float sp = 0.f;
#pragma unroll
                for (int qq = 0; qq < nq2; ++qq) {
                    const int q = shalf * nq2 + (srow + qq) % nq2;
                    float v[4] = {0.f, 0.f, 0.f, 0.f};
                    if (srow < rows && q < dq) {
                        const float4 x4 = *reinterpret_cast<const float4*>(xr + 4 * q);
                        const float4 m4 = *reinterpret_cast<const float4*>(mu_s + 4 * q);
                        v[0] = x4.x - m4.x;
                        v[1] = x4.y - m4.y;
                        v[2] = x4.z - m4.z;
                        v[3] = x4.w - m4.w;
                    }
                    float h[4], l[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        sp = fmaf(v[e], v[e], sp);
                        split_tf32(v[e], h[e], l[e]);
                    }
                    const size_t off = rbase + (size_t)q * 128;
                    *reinterpret_cast<float4*>(ahi + off) = make_float4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<float4*>(alo + off) = make_float4(l[0], l[1], l[2], l[3]);
                }
                s_part[(int)(i & 3) * 2 * kApM + shalf * kApM + srow] = sp;
            }
            // the workers' row norms of this tile are visible to every worker
            // before its out is written (two tiles later)
            asm volatile("bar.sync 1, %0;" :: "n"(kApWT) : "memory");
            if (i >= 2) epilogue(i - 2);
            // set ob written, raw stage st read, accumulator ob read
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(op_full + ob)) : "memory");
        }
        // the last two tiles
        for (int64_t j = my_tiles >= 2 ? my_tiles - 2 : 0; ok && j < my_tiles; ++j) {
            const int b = (int)(j & 1);
            ok = mbar_wait_ab(smem_u32(mma_done + b), (uint32_t)(j >> 1) & 1u, spin_limit, abort_w);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            acc_issue(b);
            epilogue(j);
        }
        if (!ok) *abort_w = 1u;
    } else if ((tid & 31) == 0) {
        // ---------------------------------- copies and MMAs (one thread)
        auto issue = [&](int64_t i) {   // raw tile i of this CTA into stage i % kApStages
            const int64_t tile = blockIdx.x + i * gridDim.x;
            const int st = (int)(i % kApStages);
            bulk_load(smem_u32(raw + (size_t)st * raw_bytes), X + tile * kApM * d,
                      (uint32_t)(tile_rows(tile) * d * 4), smem_u32(raw_full + st));
        };
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(Np >> 3) << 17) |
                               ((uint32_t)(kApM >> 4) << 24);
        // descriptors of set 0's first K step (hi, lo) and of B; set 1 and
        // each K step (256 bytes) add to the address field (16-byte units)
        const uint64_t dah = tc_desc_sbo(smem_u32(aset), sbo), dal = tc_desc_sbo(smem_u32(aset) + (uint32_t)a_bytes, sbo);
        const uint64_t dbh = tc_desc_sbo(smem_u32(bhi), sbo), dbl = tc_desc_sbo(smem_u32(blo), sbo);
        const uint64_t set_step = (uint64_t)((2 * a_bytes) >> 4);
        for (; issued < kApStages && issued < my_tiles; ++issued) issue(issued);
        for (int64_t i = 0; i < my_tiles; ++i) {
            const int ob = (int)(i & 1);
            if (!mbar_wait_ab(smem_u32(op_full + ob), (uint32_t)(i >> 1) & 1u, spin_limit, abort_w)) {
                *abort_w = 1u;
                break;
            }
            // raw stage i % kApStages has been read: the tile kApStages ahead
            if (issued < my_tiles) issue(issued++);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t so = ob ? set_step : 0u;
            const uint32_t dcol = tmem + (uint32_t)(ob * Np);
#pragma unroll
            for (int ks = 0; ks < Kp / 8; ++ks) {
                const uint64_t o = 16u * ks;
                tc_mma(dcol, dah + so + o, dbh + o, idesc, ks > 0 ? 1u : 0u);
                tc_mma(dcol, dah + so + o, dbl + o, idesc, 1u);
                tc_mma(dcol, dal + so + o, dbh + o, idesc, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(mma_done + ob)) : "memory");
            committed = i + 1;
        }
    }
    __syncthreads();
    if (*abort_w) {
        if (tid == 0 && err) set_error(err, kErrTimeout);
        // no copy or MMA of this CTA may still target its shared memory or
        // TMEM when they are released (the long limit: these complete by
        // themselves)
        if (tid == kApWT) {
            for (int64_t j = issued - 1; j >= 0 && j >= issued - kApStages; --j)
                mbar_wait(smem_u32(raw_full + (int)(j % kApStages)), (uint32_t)(j / kApStages) & 1u, kSpinLimit);
            for (int64_t j = committed - 1; j >= 0 && j >= committed - 2; --j)
                mbar_wait(smem_u32(mma_done + (int)(j & 1)), (uint32_t)(j >> 1) & 1u, kSpinLimit);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == kApW) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(tmem_cols) : "memory");
    }
}

// ----------------------------------------------------------------- l2apply
// Persistent CTAs over tiles of R rows; each tile of X arrives by cp.async
// into a double buffer (rows at a padded pitch: conflict-free reads) while
// the previous tile is computed.  Thread (row quad, column quad) forms, in
// one sweep over the coordinates, x_i - mu on the fly, its squared norm s_i
// and -2 (x_i - mu) . W for four rows (q, q + R/4, q + R/2, q + 3R/4: the
// items of a warp read consecutive rows) and four columns, then writes
// s_i u + v - 2 (x_i - mu) . W.  XV4: rows are whole 16-byte pieces (read as
// vectors at pitch d + 4, so eight consecutive rows fall in distinct banks);
// otherwise scalar reads at pitch d + 1.
template <dm_dtype DT, bool VST, bool XV4>
__global__ void __launch_bounds__(kThreads)
l2apply_kernel(const typename Types<DT>::V* __restrict__ X, int64_t n, int d, int64_t ldx,
               const typename Types<DT>::V* __restrict__ mu,
               const typename Types<DT>::Wide* __restrict__ res, int k,
               typename Types<DT>::Out* __restrict__ out, int64_t ldo, int R) {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    using Out = typename Types<DT>::Out;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int XP = XV4 ? d + 4 : d + 1;
    const int KP = round4(k), DR = round4(d);
    auto up = [](size_t x) { return (x + 15) & ~size_t(15); };
    size_t off = 0;
    V* xraw = reinterpret_cast<V*>(smem_raw);                      // [2][R][XP]
    off += up(2 * (size_t)R * XP * sizeof(V));
    Acc* Wm2 = reinterpret_cast<Acc*>(smem_raw + off);             // -2 W, DR x KP (zero padded)
    off += up((size_t)DR * KP * sizeof(Acc));
    Acc* uv = reinterpret_cast<Acc*>(smem_raw + off);              // u (KP), v (KP)
    off += up((size_t)2 * KP * sizeof(Acc));
    Acc* mu_s = reinterpret_cast<Acc*>(smem_raw + off);            // DR (zero padded)

    for (int i = threadIdx.x; i < DR * KP; i += kThreads) {
        const int c = i / KP, j = i % KP;
        Wm2[i] = (j < k && c < d) ? (Acc)(-2 * res[c * k + j]) : Acc(0);
    }
    for (int i = threadIdx.x; i < 2 * KP; i += kThreads) {
        const int h = i / KP, j = i % KP;
        uv[i] = j < k ? (Acc)res[d * k + h * k + j] : Acc(0);
    }
    for (int c = threadIdx.x; c < DR; c += kThreads) mu_s[c] = c < d ? to_acc(mu[c], Acc()) : Acc(0);

    const int64_t tiles = (n + R - 1) / R;
    auto stage = [&](int64_t tile, int buf) {
        const int64_t row0 = tile * R;
        const int nr = (int)min64(R, n - row0);
        stage_rows_pitched(xraw + (size_t)buf * R * XP, XP, X, ldx, d, row0, R, nr, XV4);
        cp_commit();
    };
    int64_t tile = blockIdx.x;
    if (tile < tiles) stage(tile, 0);
    int buf = 0;
    const int QJ = KP / 4;                            // column quads
    const int RQ = R / 4;                             // row quads; row h of quad q is q + h * RQ
    const int items = RQ * QJ;
    for (; tile < tiles; tile += gridDim.x, buf ^= 1) {
        const int64_t next = tile + gridDim.x;
        if (next < tiles) { stage(next, buf ^ 1); cp_wait<1>(); }
        else cp_wait<0>();
        __syncthreads();
        const int64_t row0 = tile * R;
        const int nr = (int)min64(R, n - row0);
        const V* xb = xraw + (size_t)buf * R * XP;
        for (int it = threadIdx.x; it < items; it += kThreads) {
            const int rq = it % RQ, jb = (it / RQ) * 4;
            Acc acc[4][4], sq[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                sq[h] = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[h][q] = 0;
            }
            for (int c0 = 0; c0 < DR; c0 += 4) {
                Acc xv[4][4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const V* xr = xb + (rq + h * RQ) * XP + c0;
                    if constexpr (XV4) {
                        V raw[4];
                        const uint4 u = *reinterpret_cast<const uint4*>(xr);
                        static_assert(sizeof(V) == 4 || !XV4 || true, "");
                        if constexpr (sizeof(V) == 4) {
                            memcpy(raw, &u, 16);
                        } else {
                            const uint4 u2 = *reinterpret_cast<const uint4*>(xr + 2);
                            memcpy(raw, &u, 16);
                            memcpy(raw + 2, &u2, 16);
                        }
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) xv[h][cc] = to_acc(raw[cc], Acc()) - mu_s[c0 + cc];
                    } else {
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc)
                            xv[h][cc] = c0 + cc < d ? to_acc(xr[cc], Acc()) - mu_s[c0 + cc] : Acc(0);
                    }
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) sq[h] = fma_acc(xv[h][cc], xv[h][cc], sq[h]);
                }
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    Acc wv[4];
                    load4(Wm2 + (c0 + cc) * KP + jb, wv);
#pragma unroll
                    for (int h = 0; h < 4; ++h)
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[h][q] = fma_acc(xv[h][cc], wv[q], acc[h][q]);
                }
            }
            Acc u4[4], v4[4];
            load4(uv + jb, u4);
            load4(uv + KP + jb, v4);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int r = rq + h * RQ;
                if (r >= nr) continue;
                Acc o[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) o[q] = fma_acc(sq[h], u4[q], v4[q]) + acc[h][q];
                Out* dst = out + (row0 + r) * ldo + jb;
                if constexpr (VST) {
                    *reinterpret_cast<float4*>(dst) = make_float4(o[0], o[1], o[2], o[3]);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (jb + q < k) dst[q] = (Out)o[q];
                }
            }
        }
        __syncthreads();
    }
}

template <dm_dtype DT, class XT>
size_t reduce_smem(int d, int k) {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    using Wide = typename Types<DT>::Wide;
    auto up = [](size_t x) { return (x + 15) & ~size_t(15); };
    const int D2 = d + 2;
    return up(2 * (size_t)kChunk * d * sizeof(XT)) + up(2 * (size_t)kChunk * k * sizeof(V)) +
           up((size_t)kChunk * round4(D2) * sizeof(Acc)) + up((size_t)kChunk * round4(k) * sizeof(Acc)) +
           up((size_t)d * sizeof(Acc)) + sizeof(Wide) * (size_t)D2 * k;
}

int sm_count(int hint) {
    if (hint > 0) return hint;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

bool rows16(const void* p, int64_t ld, int64_t w, size_t es) {
    return reinterpret_cast<uintptr_t>(p) % 16 == 0 && (ld * es) % 16 == 0 && (w * es) % 16 == 0;
}

template <dm_dtype DT, class XT, int MAXOB>
cudaError_t reduce_launch_t(const ReduceArgs& a, cudaStream_t st, int64_t* launches) {
    using V = typename Types<DT>::V;
    using Wide = typename Types<DT>::Wide;
    const size_t smem = reduce_smem<DT, XT>((int)a.d, (int)a.k);
    auto kern = reduce_kernel<DT, XT, MAXOB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    // One wave: no tail of partially filled SMs (at most reduce_blocks()).
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(
        reduce_blocks(a), (int64_t)std::max(occ, 1) * sm_count(a.num_sms)));
    const int64_t rpb = (a.n + blocks - 1) / blocks;
    kern<<<blocks, kThreads, smem, st>>>(
        static_cast<const XT*>(a.X), a.n, (int)a.d, a.ldx, static_cast<const V*>(a.mu), a.mu_stride,
        a.with_s ? 1 : 0, static_cast<const V*>(a.Z), (int)a.k, a.ldz, static_cast<Wide*>(a.partial),
        rpb, rows16(a.X, a.ldx, a.d, sizeof(XT)) ? 1 : 0, rows16(a.Z, a.ldz, a.k, sizeof(V)) ? 1 : 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int total = (int)((a.d + 2) * a.k);
    const int warps_per_block = 8;
    reduce_finalize_kernel<Wide><<<(total + warps_per_block - 1) / warps_per_block, 32 * warps_per_block,
                                   0, st>>>(static_cast<const Wide*>(a.partial), blocks, total,
                                            static_cast<Wide*>(a.res), nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *launches += 2;
    return cudaSuccess;
}

template <dm_dtype DT, class XT>
cudaError_t reduce_launch_ob(const ReduceArgs& a, cudaStream_t st, int64_t* launches) {
    const int64_t OB = ((a.d + 2 + RC - 1) / RC) * ((a.k + RJ - 1) / RJ);
    if (OB <= kThreads) return reduce_launch_t<DT, XT, 1>(a, st, launches);
    return reduce_launch_t<DT, XT, 4>(a, st, launches);
}

template <dm_dtype DT>
cudaError_t reduce_launch_dt(const ReduceArgs& a, cudaStream_t st, int64_t* launches) {
    if (a.x_acc) return reduce_launch_ob<DT, typename Types<DT>::Acc>(a, st, launches);
    return reduce_launch_ob<DT, typename Types<DT>::V>(a, st, launches);
}

// R_i = sum_c (x_ic - mu_c): one warp per row, lanes over the coordinates,
// U rows per warp step with all loads issued first.
template <dm_dtype DT>
__global__ void __launch_bounds__(kThreads)
rowsum_kernel(const typename Types<DT>::V* __restrict__ X, int64_t n, int d, int64_t ldx,
              const typename Types<DT>::V* __restrict__ mu, int64_t mu_stride,
              typename Types<DT>::Acc* __restrict__ R) {
    using Acc = typename Types<DT>::Acc;
    using V = typename Types<DT>::V;
    constexpr int U = 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Acc* mu_s = reinterpret_cast<Acc*>(smem_raw);
    for (int c = threadIdx.x; c < d; c += kThreads) mu_s[c] = to_acc(mu[c * mu_stride], Acc());
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * kThreads) >> 5;
    for (int64_t i0 = gw * U; i0 < n; i0 += nw * U) {
        Acc acc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) acc[u] = 0;
        for (int cb = 0; cb < d; cb += 32) {
            const int c = cb + lane;
            V v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = (c < d && i0 + u < n) ? X[(i0 + u) * ldx + c] : V(0);
#pragma unroll
            for (int u = 0; u < U; ++u) acc[u] += (c < d) ? to_acc(v[u], Acc()) - mu_s[c] : Acc(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            Acc x = acc[u];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0 && i0 + u < n) R[i0 + u] = x;
        }
    }
}

template <dm_dtype DT>
cudaError_t l2prep_launch_t(const L2PrepArgs& a, cudaStream_t st, int64_t* launches) {
    using V = typename Types<DT>::V;
    using Wide = typename Types<DT>::Wide;
    const int blocks = l2prep_blocks(a);
    const int64_t rpb = (a.n + blocks - 1) / blocks;
    colsum_kernel<DT><<<blocks, kThreads, kThreads * sizeof(Wide), st>>>(
        static_cast<const V*>(a.X), a.n, (int)a.d, a.ldx, static_cast<Wide*>(a.partial), rpb, a.err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mean_finalize_kernel<DT><<<(unsigned)((a.d + 3) / 4), 128, 0, st>>>(
        static_cast<const Wide*>(a.partial), blocks, (int)a.d, a.n, static_cast<V*>(a.mu));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *launches += 2;
    return cudaSuccess;
}

template <dm_dtype DT>
cudaError_t l2apply_launch_t(const L2ApplyArgs& a, cudaStream_t st, int64_t* launches, int num_sms) {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    using Wide = typename Types<DT>::Wide;
    using Out = typename Types<DT>::Out;
    auto up = [](size_t x) { return (x + 15) & ~size_t(15); };
    const bool xv4 = (a.d % 4 == 0) && rows16(a.X, a.ldx, a.d, sizeof(V));
    const int XP = xv4 ? (int)a.d + 4 : (int)a.d + 1;
    const int KP = round4((int)a.k);
    const int DR = round4((int)a.d);
    // Rows per tile: the double buffer within about 96 KB, a multiple of 4.
    int R = (int)std::min<int64_t>(256, (96 * 1024) / (2 * (int64_t)XP * (int64_t)sizeof(V)));
    R = std::max(4, R & ~3);
    const size_t smem = up(2 * (size_t)R * XP * sizeof(V)) + up((size_t)DR * KP * sizeof(Acc)) +
                        up(2 * (size_t)KP * sizeof(Acc)) + up((size_t)DR * sizeof(Acc));
    const bool vst = sizeof(Out) == 4 && a.k % 4 == 0 && a.ldo % 4 == 0 &&
                     reinterpret_cast<uintptr_t>(a.out) % 16 == 0;
    auto kern = vst ? (xv4 ? l2apply_kernel<DT, true, true> : l2apply_kernel<DT, true, false>)
                    : (xv4 ? l2apply_kernel<DT, false, true> : l2apply_kernel<DT, false, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (a.n + R - 1) / R;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)std::max(occ, 1) * num_sms));
    kern<<<(unsigned)blocks, kThreads, smem, st>>>(
        static_cast<const V*>(a.X), a.n, (int)a.d, a.ldx, static_cast<const V*>(a.mu),
        static_cast<const Wide*>(a.res), (int)a.k, static_cast<Out*>(a.out), a.ldo, R);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *launches += 1;
    return cudaSuccess;
}

}  // namespace

// Largest number of query columns one reduce launch takes for d coordinates
// of element type t (0 when even one column does not fit): the launch's
// output blocks and its shared memory (the kernel's own layout) bound it.
int64_t reduce_max_k(dm_dtype t, int64_t d) {
    if (d < 1 || d > 4096) return 0;
    int64_t best = 0;
    for (int64_t k = 1; k <= 4096; ++k) {
        const int64_t OB = ((d + 2 + RC - 1) / RC) * ((k + RJ - 1) / RJ);
        if (OB > 4 * kThreads) break;
        size_t smem = 0;
        switch (t) {
            case DM_F32: smem = reduce_smem<DM_F32, float>((int)d, (int)k); break;
            case DM_F64: smem = reduce_smem<DM_F64, double>((int)d, (int)k); break;
            default: smem = reduce_smem<DM_I32, int32_t>((int)d, (int)k); break;
        }
        if (smem > 220 * 1024) break;
        best = k;
    }
    return best;
}

bool reduce_supported(int64_t d, int64_t k) {
    const int64_t OB = ((d + 2 + RC - 1) / RC) * ((k + RJ - 1) / RJ);
    if (OB > 4 * kThreads || d > 4096 || k > 4096) return false;
    // shared memory of the reduce kernel (FP64/int64 worst case)
    const size_t smem = 2 * (size_t)kChunk * d * 8 + 2 * (size_t)kChunk * k * 8 +
                        (size_t)kChunk * (d + 6) * 8 + (size_t)kChunk * (k + 4) * 8 + (size_t)d * 8 +
                        8 * (size_t)(d + 2) * k + 96;
    return smem <= 220 * 1024;
}

// The tensor-core reduce: FP32 points (or precomputed FP32 features), d a
// multiple of 4 with the 2 (d + 2) rows of [Y_hi; Y_lo] within M = 128,
// k a multiple of 4 up to 32, rows of X and Z contiguous and 16-byte
// aligned (whole bulk copies per chunk).  Taken when the context asks for
// it, or automatically where it measured faster than the CUDA-core kernel.
bool tc_shape_ok(const ReduceArgs& a) {
    return a.dtype == DM_F32 && a.d >= 4 && a.d % 4 == 0 && 2 * (a.d + 2) <= 128 && a.k >= 4 &&
           a.k % 4 == 0 && a.k <= 32 && a.ldx == a.d && a.ldz == a.k && a.X != nullptr && a.Z != nullptr &&
           reinterpret_cast<uintptr_t>(a.X) % 16 == 0 && reinterpret_cast<uintptr_t>(a.Z) % 16 == 0;
}

// Measured (n = 2^20, CUDA-core vs tensor-core reduce + finalize, ms):
// d 32 k 16: 0.150 / 0.121; d 32 k 4: 0.123 / 0.108; d 16 k 16: 0.110 /
// 0.105; d 8 k 8: 0.124 / 0.093; d 60 k 32: 0.456 / 0.275; but d 32 k 32:
// 0.195 / 0.216.
bool tc_auto(const ReduceArgs& a) { return a.k <= 16 || a.d >= 48; }

bool tc_ok(const ReduceArgs& a) {
    if (!tc_shape_ok(a) || a.engine == DM_ENGINE_CUDA_CORES) return false;
    return a.engine == DM_ENGINE_TENSOR_CORES || tc_auto(a);
}

// Points per chunk of the tensor-core reduce and its raw stages (64-point
// chunks at two CTAs per SM measured faster than 32-point chunks at three:
// 0.121 vs 0.165 ms at n = 2^20, d = 32, k = 16, in the earlier lockstep form).
constexpr int kRtKC = 64;
constexpr int kRtStages = kRtKC == 32 ? 3 : 2;

// Partials of the CUDA-core reduce: one per CTA, at most 3 per SM, a CTA
// per 1024 rows at least.  Scratch sized from this count holds the partials
// of either kernel.
int reduce_blocks_cc(const ReduceArgs& a) {
    const int sms = sm_count(a.num_sms);
    int64_t cap = 3 * (int64_t)sms;
    if (a.max_blocks > 0) cap = std::min<int64_t>(cap, a.max_blocks);
    const int64_t want = (a.n + 1023) / 1024;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, cap));
}

uint32_t rt_tmem_cols(int k) {
    const uint32_t N = 2u * (uint32_t)((k + 7) / 8 * 8);
    uint32_t cols = 32;
    while (cols < 2u * N) cols <<= 1;     // two accumulators
    return cols;
}

// CTAs of the tensor-core reduce (one partial each): all resident at once,
// shared memory (227 KB per SM, 1 KB reserved per CTA), TMEM and the
// register bound of the launch limiting the CTAs per SM; never more than the
// CUDA-core kernel's count.
int rt_grid(const ReduceArgs& a) {
    const RtShape S = rt_shape(kRtKC, kRtStages, (int)a.d, (int)a.k);
    int per_sm = (int)((227 * 1024) / (S.total + 1024));
    per_sm = std::min(per_sm, (int)(512 / rt_tmem_cols((int)a.k)));
    per_sm = std::max(1, std::min(per_sm, rt_min_blocks(kRtKC, (a.k + 7) / 8 * 8 <= 16 ? 16 : 32)));
    const int64_t chunks = (a.n + kRtKC - 1) / kRtKC;
    const int64_t g = std::min<int64_t>(chunks, (int64_t)per_sm * sm_count(a.num_sms));
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, reduce_blocks_cc(a)));
}

cudaError_t reduce_tc_launch(const ReduceArgs& a, cudaStream_t st, int64_t* launches) {
    const int d = (int)a.d, k = (int)a.k;
    const RtShape S = rt_shape(kRtKC, kRtStages, d, k);
    const uint32_t cols = rt_tmem_cols(k);
    auto kern = S.Kp <= 16 ? reduce_tc_kernel<kRtKC, kRtStages, 16> : reduce_tc_kernel<kRtKC, kRtStages, 32>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.total);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    const int blocks = rt_grid(a);
    kern<<<blocks, kRtT, S.total, st>>>(
        static_cast<const float*>(a.X), a.n, d, static_cast<const float*>(a.mu), a.mu_stride,
        a.with_s ? 1 : 0, static_cast<const float*>(a.Z), k, static_cast<double*>(a.partial), cols, a.err,
        a.spin_limit);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int total = (d + 2) * k;
    const int warps_per_block = 8;
    reduce_finalize_kernel<double><<<(total + warps_per_block - 1) / warps_per_block, 32 * warps_per_block,
                                     0, st>>>(static_cast<const double*>(a.partial), blocks, total,
                                              static_cast<double*>(a.res), a.err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *launches += 2;
    return cudaSuccess;
}

int reduce_blocks(const ReduceArgs& a) { return tc_ok(a) ? rt_grid(a) : reduce_blocks_cc(a); }

int l2prep_blocks(const L2PrepArgs& a) {
    const int sms = sm_count(0);
    int64_t cap = 4 * (int64_t)sms;
    if (a.max_blocks > 0) cap = std::min<int64_t>(cap, a.max_blocks);
    const int64_t want = (a.n + 1023) / 1024;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, cap));
}

cudaError_t reduce_launch(const ReduceArgs& a, cudaStream_t s, int64_t* launches) {
    if (tc_ok(a)) return reduce_tc_launch(a, s, launches);
    switch (a.dtype) {
        case DM_F32: return reduce_launch_dt<DM_F32>(a, s, launches);
        case DM_F64: return reduce_launch_dt<DM_F64>(a, s, launches);
        default: return reduce_launch_dt<DM_I32>(a, s, launches);
    }
}

// The same row sums for rows of whole 16-byte vectors (d * sizeof(V) a
// multiple of 16, rows 16-byte aligned, VPR = vectors per row a power of two
// <= 32): a warp reads 32 / VPR consecutive rows with one 16-byte load per
// lane, U such loads in flight, and reduces each row over its VPR lanes.
template <dm_dtype DT, int VPR>
__global__ void __launch_bounds__(kThreads)
rowsum_vec_kernel(const typename Types<DT>::V* __restrict__ X, int64_t n, int64_t ldx,
                  const typename Types<DT>::V* __restrict__ mu, int64_t mu_stride,
                  typename Types<DT>::Acc* __restrict__ R) {
    using Acc = typename Types<DT>::Acc;
    using V = typename Types<DT>::V;
    constexpr int E = 16 / (int)sizeof(V);       // elements per vector
    constexpr int RPW = 32 / VPR;                // rows per warp load
    constexpr int U = 4;
    const int lane = threadIdx.x & 31;
    const int sub = lane % VPR, rw = lane / VPR;
    Acc m[E];
#pragma unroll
    for (int e = 0; e < E; ++e) m[e] = to_acc(mu[(int64_t)(sub * E + e) * mu_stride], Acc());
    const int64_t gw = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * kThreads) >> 5;
    for (int64_t i0 = gw * (U * RPW); i0 < n; i0 += nw * (U * RPW)) {
        V v[U][E];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + u * RPW + rw;
            if (i < n) {
                const uint4 raw = *reinterpret_cast<const uint4*>(X + i * ldx + sub * E);
                memcpy(&v[u][0], &raw, 16);
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) v[u][e] = V(0);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            Acc x = 0;
#pragma unroll
            for (int e = 0; e < E; ++e) x += to_acc(v[u][e], Acc()) - m[e];
#pragma unroll
            for (int o = VPR / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            const int64_t i = i0 + u * RPW + rw;
            if (sub == 0 && i < n) R[i] = x;
        }
    }
}

template <dm_dtype DT, int VPR>
cudaError_t rowsum_vec_launch(const void* X, int64_t n, int64_t ldx, const void* mu,
                              int64_t mu_stride, void* R, cudaStream_t s) {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    const int64_t rows_per_warp_step = 4 * (32 / VPR);
    const int64_t warps = (n + rows_per_warp_step - 1) / rows_per_warp_step;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, 8 * (int64_t)sm_count(0)));
    rowsum_vec_kernel<DT, VPR><<<(unsigned)blocks, kThreads, 0, s>>>(
        static_cast<const V*>(X), n, ldx, static_cast<const V*>(mu), mu_stride, static_cast<Acc*>(R));
    return cudaGetLastError();
}

template <dm_dtype DT>
cudaError_t rowsum_launch_t(const void* X, int64_t n, int64_t d, int64_t ldx, const void* mu,
                            int64_t mu_stride, void* R, cudaStream_t s) {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    if (rows16(X, ldx, d, sizeof(V))) {
        const int64_t vpr = d * (int64_t)sizeof(V) / 16;
        switch (vpr) {
            case 1: return rowsum_vec_launch<DT, 1>(X, n, ldx, mu, mu_stride, R, s);
            case 2: return rowsum_vec_launch<DT, 2>(X, n, ldx, mu, mu_stride, R, s);
            case 4: return rowsum_vec_launch<DT, 4>(X, n, ldx, mu, mu_stride, R, s);
            case 8: return rowsum_vec_launch<DT, 8>(X, n, ldx, mu, mu_stride, R, s);
            case 16: return rowsum_vec_launch<DT, 16>(X, n, ldx, mu, mu_stride, R, s);
            case 32: return rowsum_vec_launch<DT, 32>(X, n, ldx, mu, mu_stride, R, s);
            default: break;
        }
    }
    const size_t smem = sizeof(Acc) * (size_t)d;
    auto kern = rowsum_kernel<DT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t warps = (n + 3) / 4;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, 8 * (int64_t)sm_count(0)));
    kern<<<(unsigned)blocks, kThreads, smem, s>>>(
        static_cast<const V*>(X), n, (int)d, ldx, static_cast<const V*>(mu), mu_stride,
        static_cast<Acc*>(R));
    return cudaGetLastError();
}

cudaError_t rowsum_launch(dm_dtype t, const void* X, int64_t n, int64_t d, int64_t ldx,
                          const void* mu, int64_t mu_stride, void* R, cudaStream_t s,
                          int64_t* launches) {
    cudaError_t e;
    switch (t) {
        case DM_F32: e = rowsum_launch_t<DM_F32>(X, n, d, ldx, mu, mu_stride, R, s); break;
        case DM_F64: e = rowsum_launch_t<DM_F64>(X, n, d, ldx, mu, mu_stride, R, s); break;
        default: e = rowsum_launch_t<DM_I32>(X, n, d, ldx, mu, mu_stride, R, s); break;
    }
    if (e == cudaSuccess) ++*launches;
    return e;
}

cudaError_t l2prep_launch(const L2PrepArgs& a, cudaStream_t s, int64_t* launches) {
    switch (a.dtype) {
        case DM_F32: return l2prep_launch_t<DM_F32>(a, s, launches);
        case DM_F64: return l2prep_launch_t<DM_F64>(a, s, launches);
        default: return l2prep_launch_t<DM_I32>(a, s, launches);
    }
}

namespace {
// DM_ENGINE_AUTO picks the tensor-core apply where it measured at least as
// fast as the CUDA-core kernel (n = 2^20, tensor / CUDA cores: d = 32,
// k = 16: 0.060 / 0.061 ms; d = 32, k = 32: 0.090 / 0.113 ms; d = 16,
// k = 32: 0.076 / 0.076 ms).  Its time has a floor of about 0.055 ms at
// d = 32 whatever k (reading, shifting and splitting X), so narrower blocks
// stay on the CUDA cores (d = 24, k = 16: 0.055 / 0.053 ms).
bool apply_tc_auto(const L2ApplyArgs& a) { return a.k >= 16 && a.d * a.k >= 512; }
}  // namespace

// The apply on the tensor cores: FP32, d a multiple of 4 up to 32, k up to
// 32, rows of X contiguous (ldx = d) and 16-byte aligned.
bool apply_tc_shape_ok(const L2ApplyArgs& a) {
    return a.dtype == DM_F32 && a.d % 4 == 0 && a.d >= 4 && a.d <= 32 && a.k >= 1 && a.k <= 32 &&
           a.ldx == a.d && reinterpret_cast<uintptr_t>(a.X) % 16 == 0;
}

cudaError_t l2apply_tc_launch(const L2ApplyArgs& a, cudaStream_t st, int64_t* launches, int num_sms) {
    const int d = (int)a.d, k = (int)a.k;
    const int Kp = (d + 7) / 8 * 8, Np = (k + 15) / 16 * 16;
    uint32_t cols = 32;
    while (cols < (uint32_t)(2 * Np)) cols <<= 1;
    const size_t smem = apply_tc_smem(d, k);
    auto kern = Kp == 8 ? l2apply_tc_kernel<8> : Kp == 16 ? l2apply_tc_kernel<16>
              : Kp == 24 ? l2apply_tc_kernel<24> : l2apply_tc_kernel<32>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    // CTAs per SM: shared memory (227 KB usable, 1 KB reserved per CTA) and
    // TMEM (every resident CTA holds `cols` of the SM's 512 columns) bound it
    int occ = (int)((227 * 1024) / (smem + 1024));
    occ = std::max(1, std::min(occ, std::min(2, (int)(512 / cols))));   // 2: the launch's register bound
    const int64_t tiles = (a.n + kApM - 1) / kApM;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)occ * num_sms));
    const bool vst = a.k % 4 == 0 && a.ldo % 4 == 0 && reinterpret_cast<uintptr_t>(a.out) % 16 == 0;
    kern<<<(unsigned)blocks, kApT, smem, st>>>(
        static_cast<const float*>(a.X), a.n, d, static_cast<const float*>(a.mu),
        static_cast<const double*>(a.res), k, static_cast<float*>(a.out), a.ldo, Np, cols,
        vst ? 1 : 0, a.err, a.spin_limit);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *launches += 1;
    return cudaSuccess;
}

cudaError_t l2apply_launch(const L2ApplyArgs& a, cudaStream_t s, int64_t* launches) {
    const int sms = sm_count(a.num_sms);
    if (a.engine != DM_ENGINE_CUDA_CORES && apply_tc_shape_ok(a) &&
        (a.engine == DM_ENGINE_TENSOR_CORES || apply_tc_auto(a)))
        return l2apply_tc_launch(a, s, launches, sms);
    switch (a.dtype) {
        case DM_F32: return l2apply_launch_t<DM_F32>(a, s, launches, sms);
        case DM_F64: return l2apply_launch_t<DM_F64>(a, s, launches, sms);
        default: return l2apply_launch_t<DM_I32>(a, s, launches, sms);
    }
}

}  // namespace dm

// ===================================================================
// Squared-l2 product without allocation (dm_l2sq_matmat_noalloc).
//
// Some callers cannot allocate device memory when they call in: code that
// runs inside a memory pool or arena it does not own, callers that forbid
// allocation on their hot path (a cudaMalloc can synchronize the device), or
// setups whose memory is fully reserved up front.  This entry point runs the
// column means, the reduce and the apply of the squared-l2 product with all
// of its scratch in one file-scope device array of fixed size.
namespace dm {
namespace {

constexpr int kNoAllocMaxD = 32;
constexpr int kNoAllocMaxK = 32;
constexpr int kNoAllocMaxBlocks = 320;
constexpr size_t kNoAllocColsum = 0;
constexpr size_t kNoAllocMu = (kNoAllocColsum + 8 * (size_t)kNoAllocMaxBlocks * kNoAllocMaxD + 255) & ~size_t(255);
constexpr size_t kNoAllocPartial = (kNoAllocMu + 8 * (size_t)kNoAllocMaxD + 255) & ~size_t(255);
constexpr size_t kNoAllocRes =
    (kNoAllocPartial + 8 * (size_t)kNoAllocMaxBlocks * (kNoAllocMaxD + 2) * kNoAllocMaxK + 255) & ~size_t(255);
constexpr size_t kNoAllocBytes = (kNoAllocRes + 8 * (size_t)(kNoAllocMaxD + 2) * kNoAllocMaxK + 255) & ~size_t(255);
static_assert(kNoAllocBytes <= (size_t(3) << 20), "static scratch stays under 3 MiB");

// The scratch itself: every GPU that loads this library holds it until the
// process exits.  Host code must not pass this name to a kernel (on the host
// it is only a stand-in); it uses the device address below.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (with that device current).
cudaError_t noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace dm

extern "C" dm_status dm_l2sq_matmat_noalloc(dm_dtype dtype, const void* X, int64_t n, int64_t d,
                                            int64_t ldx, const void* Z, int64_t k, int64_t ldz,
                                            void* out, int64_t ldo, void* cuda_stream) {
    using namespace dm;
    if (!X || !Z || !out) return DM_ERR_INVALID_ARG;
    if (dtype != DM_F32 && dtype != DM_F64 && dtype != DM_I32) return DM_ERR_INVALID_ARG;
    if (n < 1 || n >= (int64_t(1) << 30) || d < 1 || ldx < d || k < 1 || ldz < k || ldo < k)
        return DM_ERR_INVALID_ARG;
    if (d > kNoAllocMaxD || k > kNoAllocMaxK || !reduce_supported(d, k)) return DM_ERR_UNSUPPORTED;
    void* base = nullptr;
    if (noalloc_scratch(&base) != cudaSuccess) { cudaGetLastError(); return DM_ERR_CUDA; }
    unsigned char* sc = static_cast<unsigned char*>(base);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int64_t launches = 0;

    L2PrepArgs pa{};
    pa.dtype = dtype;
    pa.X = X; pa.n = n; pa.d = d; pa.ldx = ldx;
    pa.partial = sc + kNoAllocColsum;
    pa.mu = sc + kNoAllocMu;
    pa.err = nullptr;
    pa.max_blocks = kNoAllocMaxBlocks;
    if (l2prep_launch(pa, st, &launches) != cudaSuccess) { cudaGetLastError(); return DM_ERR_CUDA; }

    ReduceArgs r{};
    r.dtype = dtype;
    r.X = X; r.n = n; r.d = d; r.ldx = ldx; r.x_acc = false;
    r.mu = sc + kNoAllocMu; r.mu_stride = 1; r.with_s = true;
    r.Z = Z; r.k = k; r.ldz = ldz;
    r.partial = sc + kNoAllocPartial;
    r.res = sc + kNoAllocRes;
    r.max_blocks = kNoAllocMaxBlocks;
    if (reduce_launch(r, st, &launches) != cudaSuccess) { cudaGetLastError(); return DM_ERR_CUDA; }

    L2ApplyArgs ap{};
    ap.dtype = dtype;
    ap.X = X; ap.n = n; ap.d = d; ap.ldx = ldx;
    ap.mu = sc + kNoAllocMu; ap.res = sc + kNoAllocRes; ap.k = k;
    ap.out = out; ap.ldo = ldo;
    if (l2apply_launch(ap, st, &launches) != cudaSuccess) { cudaGetLastError(); return DM_ERR_CUDA; }
    return DM_OK;
}
