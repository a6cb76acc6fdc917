// Reductions over the n points and the squared-l2 product.
//
// reduce  -- the shifted contraction of the query block with the points,
//              W[c,j] = sum_i (x_ic - mu_c) Z[i,j],  u[j] = sum_i Z[i,j],
//              v[j]   = sum_i s_i Z[i,j]             (squared l2 only),
//            i.e. [X - mu, 1, s]^T Z, a (d+2) x k result from a reduction of
//            length n.  The l1 query uses u and W as the totals T_z and T_xz
//            of its prefix sums; the squared-l2 query uses u, v and W as
//            S1, S2 and v of the p = 2 query (Appendix A).
//            Each CTA accumulates a contiguous row range (FP32 or exact int64
//            within a 64-row chunk, the chunk sums added in the Wide type),
//            writes one partial; a finalize kernel adds the partials in a
//            fixed order (deterministic for a given device).
// l2prep  -- column means mu (the frame shift; the product is translation
//            invariant) and s_i = ||x_i - mu||^2.
// l2apply -- out_i = s_i u + v - 2 (x_i - mu) . W  (Appendix A, in the
//            mu-shifted frame of the Gram decomposition of Section 1.2).
// These kernels are HBM-bound at the shapes of interest (d, k <= 64): the
// contraction does 2(d+2)k flops per (4d + 4k) bytes read, below the FP32
// ALU ridge, so they run on the CUDA cores.
#include <algorithm>

#include "dm_internal.h"

namespace dm {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 64;   // rows staged in shared memory per step
constexpr int RC = 2;        // output rows (of X-hat) per thread
constexpr int RJ = 4;        // output columns (of Z) per thread

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

// Shared-memory layout of one staged chunk: xh[kChunk][D2P] (the augmented
// row [x - mu, 1, s]) and zc[kChunk][KP].
template <dm_dtype DT, class XT>
__global__ void __launch_bounds__(kThreads)
reduce_kernel(const XT* __restrict__ X, int64_t n, int d, int64_t ldx,
              const typename Types<DT>::V* __restrict__ mu, int64_t mu_stride,
              const typename Types<DT>::Acc* __restrict__ s,
              const typename Types<DT>::V* __restrict__ Z, int k, int64_t ldz,
              typename Types<DT>::Wide* __restrict__ partial, int64_t rows_per_block) {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    using Wide = typename Types<DT>::Wide;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int D2 = d + 2;
    const int D2P = D2 + 1, KP = k + 1;
    Acc* mu_s = reinterpret_cast<Acc*>(smem_raw);
    Acc* xh = mu_s + d;
    Acc* zc = xh + kChunk * D2P;
    size_t red_off = sizeof(Acc) * ((size_t)d + (size_t)kChunk * D2P + (size_t)kChunk * KP);
    red_off = (red_off + 15) & ~size_t(15);
    Wide* red = reinterpret_cast<Wide*>(smem_raw + red_off);   // final combine

    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min64(n, r0 + rows_per_block);
    for (int c = threadIdx.x; c < d; c += kThreads) mu_s[c] = mu ? to_acc(mu[c * mu_stride], Acc()) : Acc(0);

    const int OBc = (D2 + RC - 1) / RC, OBj = (k + RJ - 1) / RJ;
    const int OB = OBc * OBj;
    const int RG = max(1, kThreads / OB);          // row groups
    const int ob_per_thread = (OB + kThreads - 1) / kThreads;

    // Each thread owns up to ob_per_thread output blocks of RC x RJ.
    constexpr int MAXOB = 4;
    Wide wacc[MAXOB][RC][RJ];
#pragma unroll
    for (int b = 0; b < MAXOB; ++b)
#pragma unroll
        for (int a = 0; a < RC; ++a)
#pragma unroll
            for (int q = 0; q < RJ; ++q) wacc[b][a][q] = 0;

    const int my_rg = (OB >= kThreads) ? 0 : threadIdx.x / OB;
    __syncthreads();

    for (int64_t base = r0; base < r1; base += kChunk) {
        const int nr = (int)min64(kChunk, r1 - base);
        __syncthreads();
        for (int i = threadIdx.x; i < kChunk * D2; i += kThreads) {
            const int r = i / D2, c = i % D2;
            Acc v = 0;
            if (r < nr) {
                if (c < d) v = to_acc(X[(base + r) * ldx + c], Acc()) - mu_s[c];
                else if (c == d) v = 1;
                else v = s ? s[base + r] : Acc(0);
            }
            xh[r * D2P + c] = v;
        }
        for (int i = threadIdx.x; i < kChunk * k; i += kThreads) {
            const int r = i / k, j = i % k;
            zc[r * KP + j] = (r < nr) ? to_acc(Z[(base + r) * ldz + j], Acc()) : Acc(0);
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < MAXOB; ++b) {
            if (b >= ob_per_thread) break;
            const int ob = (OB >= kThreads) ? threadIdx.x + b * kThreads : threadIdx.x % OB;
            if (ob >= OB || my_rg >= RG) continue;
            const int cb = (ob / OBj) * RC, jb = (ob % OBj) * RJ;
            Acc acc[RC][RJ];
#pragma unroll
            for (int a = 0; a < RC; ++a)
#pragma unroll
                for (int q = 0; q < RJ; ++q) acc[a][q] = 0;
            for (int r = my_rg; r < kChunk; r += RG) {
                Acc xv[RC], zv[RJ];
#pragma unroll
                for (int a = 0; a < RC; ++a) xv[a] = (cb + a < D2) ? xh[r * D2P + cb + a] : Acc(0);
#pragma unroll
                for (int q = 0; q < RJ; ++q) zv[q] = (jb + q < k) ? zc[r * KP + jb + q] : Acc(0);
#pragma unroll
                for (int a = 0; a < RC; ++a)
#pragma unroll
                    for (int q = 0; q < RJ; ++q) acc[a][q] = fma_acc(xv[a], zv[q], acc[a][q]);
            }
#pragma unroll
            for (int a = 0; a < RC; ++a)
#pragma unroll
                for (int q = 0; q < RJ; ++q) wacc[b][a][q] += (Wide)acc[a][q];
        }
    }
    __syncthreads();

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
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min64(n, r0 + rows_per_block);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Wide* red = reinterpret_cast<Wide*>(smem_raw);
    // Thread (column c0, row group g) walks rows g, g + rg, ... of its range.
    const int cols = min(d, kThreads);
    const int rg = kThreads / cols;
    const int c0 = threadIdx.x % cols, g = threadIdx.x / cols;
    bool bad = false;
    for (int cb = 0; cb < d; cb += cols) {
        const int c = cb + c0;
        Wide acc = 0;
        if (g < rg && c < d) {
            for (int64_t r = r0 + g; r < r1; r += rg) {
                const auto v = X[r * ldx + c];
                bad |= !finite_val(v);
                acc += (Wide)v;
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
    if (bad) set_error(err, kErrNonfinite);
}

template <dm_dtype DT>
__global__ void mean_finalize_kernel(const typename Types<DT>::Wide* __restrict__ partial,
                                     int blocks, int d, int64_t n,
                                     typename Types<DT>::V* __restrict__ mu) {
    using Wide = typename Types<DT>::Wide;
    using V = typename Types<DT>::V;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d) return;
    Wide t = 0;
    for (int b = 0; b < blocks; ++b) t += partial[(int64_t)b * d + c];
    mu[c] = (V)(t / (Wide)n);
}

template <dm_dtype DT>
__global__ void __launch_bounds__(kThreads)
sqnorm_kernel(const typename Types<DT>::V* __restrict__ X, int64_t n, int d, int64_t ldx,
              const typename Types<DT>::V* __restrict__ mu, typename Types<DT>::Acc* __restrict__ s) {
    using Acc = typename Types<DT>::Acc;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Acc acc = 0;
    for (int c = 0; c < d; ++c) {
        const Acc t = to_acc(X[i * ldx + c], Acc()) - to_acc(mu[c], Acc());
        acc = fma_acc(t, t, acc);
    }
    s[i] = acc;
}

// ----------------------------------------------------------------- l2apply
// Block: kApplyRows rows x all k columns.  Thread (row pair, column quad).
constexpr int kApplyRows = 128;
template <dm_dtype DT>
__global__ void __launch_bounds__(kThreads)
l2apply_kernel(const typename Types<DT>::V* __restrict__ X, int64_t n, int d, int64_t ldx,
               const typename Types<DT>::V* __restrict__ mu, const typename Types<DT>::Acc* __restrict__ s,
               const typename Types<DT>::Wide* __restrict__ res, int k,
               typename Types<DT>::Out* __restrict__ out, int64_t ldo) {
    using Acc = typename Types<DT>::Acc;
    constexpr int R = kApplyRows;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int DP = d + 1;
    Acc* Wm2 = reinterpret_cast<Acc*>(smem_raw);   // -2 W, d x k
    Acc* uv = Wm2 + d * k;                          // u (k), v (k)
    Acc* xt = uv + 2 * k;                           // R x DP shifted rows
    Acc* mu_s = xt + R * DP;

    for (int i = threadIdx.x; i < d * k; i += kThreads) Wm2[i] = (Acc)(-2 * res[i]);
    for (int i = threadIdx.x; i < 2 * k; i += kThreads) uv[i] = (Acc)res[d * k + i];
    for (int c = threadIdx.x; c < d; c += kThreads) mu_s[c] = to_acc(mu[c], Acc());
    __syncthreads();

    const int64_t row0 = (int64_t)blockIdx.x * R;
    const int nr = (int)min64(R, n - row0);
    for (int i = threadIdx.x; i < R * d; i += kThreads) {
        const int r = i / d, c = i % d;
        xt[r * DP + c] = (r < nr) ? to_acc(X[(row0 + r) * ldx + c], Acc()) - mu_s[c] : Acc(0);
    }
    __syncthreads();

    const int QJ = (k + RJ - 1) / RJ;                 // column quads
    for (int w = threadIdx.x; w < (R / 2) * QJ; w += kThreads) {
        const int rp = w / QJ, jq = w % QJ;
        const int ra = 2 * rp, jb = jq * RJ;
        Acc acc[2][RJ];
#pragma unroll
        for (int q = 0; q < RJ; ++q) {
            const int j = min(jb + q, k - 1);
            const Acc base = uv[k + j];
            acc[0][q] = (ra < nr) ? fma_acc(s[row0 + ra], uv[j], base) : Acc(0);
            acc[1][q] = (ra + 1 < nr) ? fma_acc(s[row0 + ra + 1], uv[j], base) : Acc(0);
        }
        for (int c = 0; c < d; ++c) {
            const Acc x0 = xt[ra * DP + c], x1 = xt[(ra + 1) * DP + c];
#pragma unroll
            for (int q = 0; q < RJ; ++q) {
                const Acc wv = Wm2[c * k + min(jb + q, k - 1)];
                acc[0][q] = fma_acc(x0, wv, acc[0][q]);
                acc[1][q] = fma_acc(x1, wv, acc[1][q]);
            }
        }
#pragma unroll
        for (int q = 0; q < RJ; ++q) {
            if (jb + q >= k) break;
            if (ra < nr) out[(row0 + ra) * ldo + jb + q] = acc[0][q];
            if (ra + 1 < nr) out[(row0 + ra + 1) * ldo + jb + q] = acc[1][q];
        }
    }
}

template <dm_dtype DT>
size_t reduce_smem(int d, int k) {
    using Acc = typename Types<DT>::Acc;
    using Wide = typename Types<DT>::Wide;
    const int D2 = d + 2;
    size_t a = sizeof(Acc) * ((size_t)d + kChunk * (D2 + 1) + (size_t)kChunk * (k + 1));
    a = (a + 15) & ~size_t(15);
    return a + sizeof(Wide) * (size_t)D2 * k;
}

template <dm_dtype DT, class XT>
cudaError_t reduce_launch_t(const ReduceArgs& a, cudaStream_t st, int64_t* launches) {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    using Wide = typename Types<DT>::Wide;
    const int blocks = reduce_blocks(a);
    const int64_t rpb = (a.n + blocks - 1) / blocks;
    const size_t smem = reduce_smem<DT>((int)a.d, (int)a.k);
    auto kern = reduce_kernel<DT, XT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<blocks, kThreads, smem, st>>>(
        static_cast<const XT*>(a.X), a.n, (int)a.d, a.ldx, static_cast<const V*>(a.mu), a.mu_stride,
        static_cast<const Acc*>(a.s), static_cast<const V*>(a.Z), (int)a.k, a.ldz,
        static_cast<Wide*>(a.partial), rpb);
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

template <dm_dtype DT>
cudaError_t reduce_launch_dt(const ReduceArgs& a, cudaStream_t st, int64_t* launches) {
    if (a.x_acc) return reduce_launch_t<DT, typename Types<DT>::Acc>(a, st, launches);
    return reduce_launch_t<DT, typename Types<DT>::V>(a, st, launches);
}

// R_i = sum_c (x_ic - mu_c), one thread per point.
template <dm_dtype DT>
__global__ void __launch_bounds__(kThreads)
rowsum_kernel(const typename Types<DT>::V* __restrict__ X, int64_t n, int d, int64_t ldx,
              const typename Types<DT>::V* __restrict__ mu, int64_t mu_stride,
              typename Types<DT>::Acc* __restrict__ R) {
    using Acc = typename Types<DT>::Acc;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Acc* mu_s = reinterpret_cast<Acc*>(smem_raw);
    for (int c = threadIdx.x; c < d; c += kThreads) mu_s[c] = to_acc(mu[c * mu_stride], Acc());
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    Acc acc = 0;
    for (int c = 0; c < d; ++c) acc += to_acc(X[i * ldx + c], Acc()) - mu_s[c];
    R[i] = acc;
}

template <dm_dtype DT>
cudaError_t l2prep_launch_t(const L2PrepArgs& a, cudaStream_t st, int64_t* launches) {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    using Wide = typename Types<DT>::Wide;
    const int blocks = l2prep_blocks(a);
    const int64_t rpb = (a.n + blocks - 1) / blocks;
    colsum_kernel<DT><<<blocks, kThreads, kThreads * sizeof(Wide), st>>>(
        static_cast<const V*>(a.X), a.n, (int)a.d, a.ldx, static_cast<Wide*>(a.partial), rpb, a.err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mean_finalize_kernel<DT><<<(unsigned)((a.d + 127) / 128), 128, 0, st>>>(
        static_cast<const Wide*>(a.partial), blocks, (int)a.d, a.n, static_cast<V*>(a.mu));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    sqnorm_kernel<DT><<<(unsigned)((a.n + kThreads - 1) / kThreads), kThreads, 0, st>>>(
        static_cast<const V*>(a.X), a.n, (int)a.d, a.ldx, static_cast<const V*>(a.mu),
        static_cast<Acc*>(a.s));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *launches += 3;
    return cudaSuccess;
}

template <dm_dtype DT>
cudaError_t l2apply_launch_t(const L2ApplyArgs& a, cudaStream_t st, int64_t* launches) {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    using Wide = typename Types<DT>::Wide;
    using Out = typename Types<DT>::Out;
    const size_t smem = sizeof(Acc) * ((size_t)a.d * a.k + 2 * a.k + kApplyRows * (a.d + 1) + a.d);
    auto kern = l2apply_kernel<DT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)((a.n + kApplyRows - 1) / kApplyRows), kThreads, smem, st>>>(
        static_cast<const V*>(a.X), a.n, (int)a.d, a.ldx, static_cast<const V*>(a.mu),
        static_cast<const Acc*>(a.s), static_cast<const Wide*>(a.res), (int)a.k,
        static_cast<Out*>(a.out), a.ldo);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *launches += 1;
    return cudaSuccess;
}

}  // namespace

bool reduce_supported(int64_t d, int64_t k) {
    const int64_t OB = ((d + 2 + RC - 1) / RC) * ((k + RJ - 1) / RJ);
    return OB <= 4 * kThreads && d <= 4096 && k <= 4096;
}

int reduce_blocks(const ReduceArgs& a) {
    int sms = a.num_sms;
    if (sms <= 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const int64_t want = (a.n + 1023) / 1024;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, 2 * sms));
}

int l2prep_blocks(const L2PrepArgs& a) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (a.n + 1023) / 1024;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, 2 * sms));
}

cudaError_t reduce_launch(const ReduceArgs& a, cudaStream_t s, int64_t* launches) {
    switch (a.dtype) {
        case DM_F32: return reduce_launch_dt<DM_F32>(a, s, launches);
        case DM_F64: return reduce_launch_dt<DM_F64>(a, s, launches);
        default: return reduce_launch_dt<DM_I32>(a, s, launches);
    }
}

template <dm_dtype DT>
cudaError_t rowsum_launch_t(const void* X, int64_t n, int64_t d, int64_t ldx, const void* mu,
                            int64_t mu_stride, void* R, cudaStream_t s) {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    const size_t smem = sizeof(Acc) * (size_t)d;
    auto kern = rowsum_kernel<DT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, smem, s>>>(
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
    switch (a.dtype) {
        case DM_F32: return l2apply_launch_t<DM_F32>(a, s, launches);
        case DM_F64: return l2apply_launch_t<DM_F64>(a, s, launches);
        default: return l2apply_launch_t<DM_I32>(a, s, launches);
    }
}

}  // namespace dm
