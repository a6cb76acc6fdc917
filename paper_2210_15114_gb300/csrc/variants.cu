// Variants of the product on the same machinery (Appendix A):
//   total variation  TV(x, y) = ||x - y||_1 / 2 (Theorem "tv"): the l1 product
//                    followed by scale_kernel;
//   ||x - y||_p^p for even p ("General p"): with x~ = x - mu (the product is
//                    translation invariant) and M_{c,s} = sum_j y_j x~_j(c)^s,
//                    (Ay)_k = sum_c sum_{t=0}^{p} C(p,t) (-1)^(p-t) x~_k(c)^t M_{c,p-t}.
//                    lpp_features_kernel writes the powers x~^s (s = 1..p), the
//                    reduce kernel forms M, lpp_apply_kernel evaluates the sum
//                    (Horner in x~ per coordinate, the binomial coefficients and
//                    signs folded into the coefficients);
//   approximate l2 ("Approximate Matrix-Vector Query for l2"): the points are
//                    mapped by T(x) = G x / (beta m), beta = sqrt(2/pi), G an
//                    m x d Gaussian matrix given by the caller (Theorem
//                    "l2embed"), in project_kernel, and the l1 product of the
//                    mapped points is the approximation.
#include <algorithm>

#include "dm_internal.h"

namespace dm {
namespace {

constexpr int kVT = 256;

__device__ __forceinline__ float to_v(float v, float) { return v; }
__device__ __forceinline__ double to_v(double v, double) { return v; }
__device__ __forceinline__ long long to_v(int32_t v, long long) { return (long long)v; }

template <class Out>
__global__ void scale_kernel(Out* __restrict__ out, int64_t n, int64_t k, int64_t ldo, Out s) {
    const int64_t total = n * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / k, j = e - (e / k) * k;
        out[i * ldo + j] *= s;
    }
}

// F[i, c*p + s - 1] = (x_ic - mu_c)^s, s = 1..p (accumulation type).
template <dm_dtype DT>
__global__ void lpp_features_kernel(const typename Types<DT>::V* __restrict__ X, int64_t n, int d,
                                    int64_t ldx, const typename Types<DT>::V* __restrict__ mu, int p,
                                    typename Types<DT>::Acc* __restrict__ F) {
    using Acc = typename Types<DT>::Acc;
    const int64_t total = n * d;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / d;
        const int c = (int)(e - i * d);
        const Acc x = to_v(X[i * ldx + c], Acc()) - to_v(mu[c], Acc());
        Acc* f = F + e * p;
        Acc v = x;
        for (int s = 0; s < p; ++s) {
            f[s] = v;
            v *= x;
        }
    }
}

// out[i, j] = sum_c sum_t x~_ic^t K[c][t][j] with
// K[c][t][j] = C(p,t) (-1)^(p-t) M_{c,p-t,j}; M_{c,0,j} = 1^T z_j, M_{c,s,j}
// for s >= 1 from the reduce: res[(c*p + s - 1) * k + j], then 1^T Z at
// res[d*p*k + j].  One thread per (row, column); K in shared memory.
template <dm_dtype DT>
__global__ void __launch_bounds__(kVT)
lpp_apply_kernel(const typename Types<DT>::V* __restrict__ X, int64_t n, int d, int64_t ldx,
                 const typename Types<DT>::V* __restrict__ mu,
                 const typename Types<DT>::Wide* __restrict__ res, int p, int k,
                 typename Types<DT>::Out* __restrict__ out, int64_t ldo) {
    using Acc = typename Types<DT>::Acc;
    using Wide = typename Types<DT>::Wide;
    using Out = typename Types<DT>::Out;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Acc* K = reinterpret_cast<Acc*>(smem_raw);          // [d][p+1][k]
    Acc* m = K + (size_t)d * (p + 1) * k;               // [d]
    const int P1 = p + 1;
    for (int e = threadIdx.x; e < d * P1 * k; e += blockDim.x) {
        const int c = e / (P1 * k), r = e - c * (P1 * k), t = r / k, j = r - t * k;
        const int s = p - t;                             // power of -x_j in the moment
        Wide binom = 1;
        for (int u = 0; u < t; ++u) binom = binom * (Wide)(p - u) / (Wide)(u + 1);
        const Wide M = s == 0 ? res[(size_t)d * p * k + j] : res[((size_t)c * p + s - 1) * k + j];
        K[e] = (Acc)(((s & 1) ? -binom : binom) * M);
    }
    for (int c = threadIdx.x; c < d; c += blockDim.x) m[c] = to_v(mu[c], Acc());
    __syncthreads();
    const int64_t total = n * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / k;
        const int j = (int)(e - i * k);
        Acc acc = 0;
        for (int c = 0; c < d; ++c) {
            const Acc x = to_v(X[i * ldx + c], Acc()) - m[c];
            const Acc* kc = K + (size_t)c * P1 * k + j;
            Acc h = kc[(size_t)p * k];
            for (int t = p - 1; t >= 0; --t) h = h * x + kc[(size_t)t * k];
            acc += h;
        }
        out[i * ldo + j] = (Out)acc;
    }
}

// Xp[i, c] = scale * sum_t X[i, t] G[c, t]: 64-row tiles, each thread a 4 x 4
// block of outputs, G and the row tile in shared memory.
constexpr int kPR = 64;     // rows per block
constexpr int kPC = 64;     // output columns per pass

template <class V>
__global__ void __launch_bounds__(kVT)
project_kernel(const V* __restrict__ X, int64_t n, int d, int64_t ldx, const V* __restrict__ G, int m,
               V scale, V* __restrict__ Xp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* Gs = reinterpret_cast<V*>(smem_raw);             // [m][d + 1] (padded: no bank conflicts)
    V* Xs = Gs + (size_t)m * (d + 1);                    // [kPR][d + 1]
    for (int e = threadIdx.x; e < m * d; e += blockDim.x) Gs[(e / d) * (d + 1) + e % d] = G[e];
    const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;   // 16 x 16 threads, 4 x 4 each
    for (int64_t r0 = (int64_t)blockIdx.x * kPR; r0 < n; r0 += (int64_t)gridDim.x * kPR) {
        __syncthreads();
        for (int e = threadIdx.x; e < kPR * d; e += blockDim.x) {
            const int r = e / d, t = e - r * d;
            Xs[r * (d + 1) + t] = r0 + r < n ? X[(r0 + r) * ldx + t] : V(0);
        }
        __syncthreads();
        for (int c0 = 0; c0 < m; c0 += kPC) {
            V acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = V(0);
            for (int t = 0; t < d; ++t) {
                V xv[4], gv[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) xv[a] = Xs[(tr * 4 + a) * (d + 1) + t];
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int c = c0 + tc + 16 * b;
                    gv[b] = c < m ? Gs[(size_t)c * (d + 1) + t] : V(0);
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] += xv[a] * gv[b];
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int64_t r = r0 + tr * 4 + a;
                if (r >= n) continue;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int c = c0 + tc + 16 * b;
                    if (c < m) Xp[r * m + c] = acc[a][b] * scale;
                }
            }
        }
    }
}

int grid_for(int64_t work, int num_sms) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + kVT - 1) / kVT, 8 * (int64_t)num_sms));
}

}  // namespace

cudaError_t scale_launch(dm_dtype t, void* out, int64_t n, int64_t k, int64_t ldo, double s,
                         int num_sms, cudaStream_t st, int64_t* launches) {
    const int g = grid_for(n * k, num_sms);
    switch (t) {
        case DM_F32: scale_kernel<float><<<g, kVT, 0, st>>>(static_cast<float*>(out), n, k, ldo, (float)s); break;
        case DM_F64: scale_kernel<double><<<g, kVT, 0, st>>>(static_cast<double*>(out), n, k, ldo, s); break;
        default: return cudaErrorInvalidValue;
    }
    ++*launches;
    return cudaGetLastError();
}

size_t lpp_feature_bytes(dm_dtype t, int64_t n, int64_t d, int p) {
    return (size_t)n * (size_t)d * (size_t)p * (t == DM_F32 ? 4 : 8);
}

template <dm_dtype DT>
cudaError_t lpp_features_t(const void* X, int64_t n, int64_t d, int64_t ldx, const void* mu, int p,
                           void* F, int num_sms, cudaStream_t st) {
    using V = typename Types<DT>::V;
    using Acc = typename Types<DT>::Acc;
    lpp_features_kernel<DT><<<grid_for(n * d, num_sms), kVT, 0, st>>>(
        static_cast<const V*>(X), n, (int)d, ldx, static_cast<const V*>(mu), p, static_cast<Acc*>(F));
    return cudaGetLastError();
}

cudaError_t lpp_features_launch(dm_dtype t, const void* X, int64_t n, int64_t d, int64_t ldx,
                                const void* mu, int p, void* F, int num_sms, cudaStream_t st,
                                int64_t* launches) {
    cudaError_t e;
    switch (t) {
        case DM_F32: e = lpp_features_t<DM_F32>(X, n, d, ldx, mu, p, F, num_sms, st); break;
        case DM_F64: e = lpp_features_t<DM_F64>(X, n, d, ldx, mu, p, F, num_sms, st); break;
        default: e = lpp_features_t<DM_I32>(X, n, d, ldx, mu, p, F, num_sms, st); break;
    }
    if (e == cudaSuccess) ++*launches;
    return e;
}

size_t lpp_apply_smem(dm_dtype t, int64_t d, int p, int64_t k) {
    return ((size_t)d * (p + 1) * k + d) * (t == DM_F32 ? 4 : 8);
}

template <dm_dtype DT>
cudaError_t lpp_apply_t(const void* X, int64_t n, int64_t d, int64_t ldx, const void* mu,
                        const void* res, int p, int64_t k, void* out, int64_t ldo, int num_sms,
                        cudaStream_t st) {
    using V = typename Types<DT>::V;
    using Wide = typename Types<DT>::Wide;
    using Out = typename Types<DT>::Out;
    const size_t smem = lpp_apply_smem(DT, d, p, k);
    auto kern = lpp_apply_kernel<DT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid_for(n * k, num_sms), kVT, smem, st>>>(static_cast<const V*>(X), n, (int)d, ldx,
                                                     static_cast<const V*>(mu), static_cast<const Wide*>(res),
                                                     p, (int)k, static_cast<Out*>(out), ldo);
    return cudaGetLastError();
}

cudaError_t lpp_apply_launch(dm_dtype t, const void* X, int64_t n, int64_t d, int64_t ldx,
                             const void* mu, const void* res, int p, int64_t k, void* out, int64_t ldo,
                             int num_sms, cudaStream_t st, int64_t* launches) {
    cudaError_t e;
    switch (t) {
        case DM_F32: e = lpp_apply_t<DM_F32>(X, n, d, ldx, mu, res, p, k, out, ldo, num_sms, st); break;
        case DM_F64: e = lpp_apply_t<DM_F64>(X, n, d, ldx, mu, res, p, k, out, ldo, num_sms, st); break;
        default: e = lpp_apply_t<DM_I32>(X, n, d, ldx, mu, res, p, k, out, ldo, num_sms, st); break;
    }
    if (e == cudaSuccess) ++*launches;
    return e;
}

size_t project_smem(dm_dtype t, int64_t d, int64_t m) {
    return ((size_t)m * (d + 1) + (size_t)kPR * (d + 1)) * dtype_size(t);
}

cudaError_t project_launch(dm_dtype t, const void* X, int64_t n, int64_t d, int64_t ldx, const void* G,
                           int64_t m, void* Xp, int num_sms, cudaStream_t st, int64_t* launches) {
    const size_t smem = project_smem(t, d, m);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + kPR - 1) / kPR, 2 * (int64_t)num_sms));
    const double beta = 0.79788456080286535588;   // sqrt(2 / pi)
    const double scale = 1.0 / (beta * (double)m);
    cudaError_t e;
    if (t == DM_F32) {
        auto kern = project_kernel<float>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<blocks, kVT, smem, st>>>(static_cast<const float*>(X), n, (int)d, ldx,
                                        static_cast<const float*>(G), (int)m, (float)scale,
                                        static_cast<float*>(Xp));
    } else if (t == DM_F64) {
        auto kern = project_kernel<double>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<blocks, kVT, smem, st>>>(static_cast<const double*>(X), n, (int)d, ldx,
                                        static_cast<const double*>(G), (int)m, scale,
                                        static_cast<double*>(Xp));
    } else {
        return cudaErrorInvalidValue;
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) ++*launches;
    return e;
}

}  // namespace dm
