// The plain method: out[i,:] = sum_j f(x_i, x_j) Z[j,:] with every distance
// computed on the fly, O(n^2 (d + k)) work -- the naive baseline of Section 4
// without materializing A (which the paper could not do at n = 1.2e6 either).
//
// CTA = 128 threads x RPT query rows each; the points x_j and their query
// rows stream through shared memory in chunks of JC.  Each distance is
// computed once per (i, j) pair and reused for all k columns of the chunk.
// Coordinates beyond d are zero-padded up to the compile-time DMAX (they add
// |0 - 0| = 0).  Columns are processed KMAX at a time.
#include <algorithm>

#include "dm_internal.h"

namespace dm {
namespace {

constexpr int kThreads = 128;
constexpr int JC = 32;

__device__ __forceinline__ float to_acc(float v, float) { return v; }
__device__ __forceinline__ double to_acc(double v, double) { return v; }
__device__ __forceinline__ long long to_acc(int32_t v, long long) { return (long long)v; }

__device__ __forceinline__ float absd(float v) { return fabsf(v); }
__device__ __forceinline__ double absd(double v) { return fabs(v); }
__device__ __forceinline__ long long absd(long long v) { return v < 0 ? -v : v; }

template <dm_dtype DT, int METRIC, int DMAX, int KMAX, int RPT>
__global__ void __launch_bounds__(kThreads)
brute_kernel(const typename Types<DT>::V* __restrict__ X, int64_t n, int d, int64_t ldx,
             const typename Types<DT>::V* __restrict__ Z, int k, int64_t ldz,
             typename Types<DT>::Out* __restrict__ out, int64_t ldo) {
    using Acc = typename Types<DT>::Acc;
    __shared__ __align__(16) Acc xj[JC][DMAX];
    __shared__ __align__(16) Acc zj[JC][KMAX];

    const int col0 = blockIdx.y * KMAX;
    const int kc = min(KMAX, k - col0);
    const int64_t i0 = ((int64_t)blockIdx.x * kThreads + threadIdx.x) * RPT;

    Acc xi[RPT][DMAX];
    Acc acc[RPT][KMAX];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int64_t i = i0 + q;
#pragma unroll
        for (int c = 0; c < DMAX; ++c)
            xi[q][c] = (i < n && c < d) ? to_acc(X[i * ldx + c], Acc()) : Acc(0);
#pragma unroll
        for (int m = 0; m < KMAX; ++m) acc[q][m] = 0;
    }

    for (int64_t jb = 0; jb < n; jb += JC) {
        __syncthreads();
        for (int t = threadIdx.x; t < JC * DMAX; t += kThreads) {
            const int r = t / DMAX, c = t % DMAX;
            const int64_t j = jb + r;
            xj[r][c] = (j < n && c < d) ? to_acc(X[j * ldx + c], Acc()) : Acc(0);
        }
        for (int t = threadIdx.x; t < JC * KMAX; t += kThreads) {
            const int r = t / KMAX, m = t % KMAX;
            const int64_t j = jb + r;
            zj[r][m] = (j < n && m < kc) ? to_acc(Z[j * ldz + col0 + m], Acc()) : Acc(0);
        }
        __syncthreads();
#pragma unroll 2
        for (int r = 0; r < JC; ++r) {
            Acc dist[RPT];
#pragma unroll
            for (int q = 0; q < RPT; ++q) dist[q] = 0;
#pragma unroll
            for (int c = 0; c < DMAX; ++c) {
                const Acc y = xj[r][c];
#pragma unroll
                for (int q = 0; q < RPT; ++q) {
                    const Acc t = xi[q][c] - y;
                    dist[q] += (METRIC == DM_L1) ? absd(t) : t * t;
                }
            }
#pragma unroll
            for (int m = 0; m < KMAX; ++m) {
                const Acc w = zj[r][m];
#pragma unroll
                for (int q = 0; q < RPT; ++q) acc[q][m] += dist[q] * w;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int64_t i = i0 + q;
        if (i >= n) continue;
#pragma unroll
        for (int m = 0; m < KMAX; ++m)
            if (m < kc) out[i * ldo + col0 + m] = acc[q][m];
    }
}

template <dm_dtype DT, int METRIC, int DMAX, int KMAX>
cudaError_t launch4(const BruteArgs& a, cudaStream_t s) {
    using V = typename Types<DT>::V;
    using Out = typename Types<DT>::Out;
    constexpr int RPT = (sizeof(typename Types<DT>::Acc) == 4 && DMAX <= 32) ? 2 : 1;
    const int64_t rows_per_block = (int64_t)kThreads * RPT;
    dim3 grid((unsigned)((a.n + rows_per_block - 1) / rows_per_block), (unsigned)((a.k + KMAX - 1) / KMAX));
    brute_kernel<DT, METRIC, DMAX, KMAX, RPT><<<grid, kThreads, 0, s>>>(
        static_cast<const V*>(a.X), a.n, (int)a.d, a.ldx, static_cast<const V*>(a.Z), (int)a.k, a.ldz,
        static_cast<Out*>(a.out), a.ldo);
    return cudaGetLastError();
}

template <dm_dtype DT, int METRIC>
cudaError_t launch_m(const BruteArgs& a, cudaStream_t s) {
    const bool k1 = a.k == 1;
    if (a.d <= 8) return k1 ? launch4<DT, METRIC, 8, 1>(a, s) : launch4<DT, METRIC, 8, 16>(a, s);
    if (a.d <= 32) return k1 ? launch4<DT, METRIC, 32, 1>(a, s) : launch4<DT, METRIC, 32, 16>(a, s);
    return k1 ? launch4<DT, METRIC, 64, 1>(a, s) : launch4<DT, METRIC, 64, 16>(a, s);
}

template <dm_dtype DT>
cudaError_t launch_dt(const BruteArgs& a, cudaStream_t s) {
    return a.metric == DM_L1 ? launch_m<DT, DM_L1>(a, s) : launch_m<DT, DM_L2SQ>(a, s);
}

}  // namespace

cudaError_t brute_launch(const BruteArgs& a, cudaStream_t s, int64_t* launches) {
    cudaError_t e;
    switch (a.dtype) {
        case DM_F32: e = launch_dt<DM_F32>(a, s); break;
        case DM_F64: e = launch_dt<DM_F64>(a, s); break;
        default: e = launch_dt<DM_I32>(a, s); break;
    }
    if (e == cudaSuccess) ++*launches;
    return e;
}

}  // namespace dm
