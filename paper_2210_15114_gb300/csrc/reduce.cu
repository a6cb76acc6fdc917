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
// l2prep  -- column means mu (the frame shift), FP64 sums, fixed order.
// l2apply -- out_i = s_i u + v - 2 (x_i - mu) . W  (the p = 2 query, Appendix
//            A), s_i recomputed from the staged row with the same code as in
//            the reduce.
// These kernels are HBM-bound at the shapes of interest (d, k <= 64): the
// contraction does 2(d+2)k flops per (4d + 4k) bytes read, below the FP32
// ALU ridge, so they run on the CUDA cores.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "dm_internal.h"

namespace dm {
namespace {

constexpr int kThreads = 256;
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
template <class Wide>
__global__ void reduce_finalize_kernel(const Wide* __restrict__ partial, int blocks, int total,
                                       Wide* __restrict__ res) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= total) return;
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
                                            static_cast<Wide*>(a.res));
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

int reduce_blocks(const ReduceArgs& a) {
    const int sms = sm_count(a.num_sms);
    int64_t cap = 3 * (int64_t)sms;
    if (a.max_blocks > 0) cap = std::min<int64_t>(cap, a.max_blocks);
    const int64_t want = (a.n + 1023) / 1024;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, cap));
}

int l2prep_blocks(const L2PrepArgs& a) {
    const int sms = sm_count(0);
    int64_t cap = 4 * (int64_t)sms;
    if (a.max_blocks > 0) cap = std::min<int64_t>(cap, a.max_blocks);
    const int64_t want = (a.n + 1023) / 1024;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, cap));
}

cudaError_t reduce_launch(const ReduceArgs& a, cudaStream_t s, int64_t* launches) {
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

cudaError_t l2apply_launch(const L2ApplyArgs& a, cudaStream_t s, int64_t* launches) {
    const int sms = sm_count(a.num_sms);
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
