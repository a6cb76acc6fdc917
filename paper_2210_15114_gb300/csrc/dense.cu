// Dense products on tall-skinny FP32 blocks: the steps between distance-matrix
// products of the block Krylov iteration (Appendix C, Theorems "musco" and
// "singular_values_system"): projections W - P (P^T W), Gram matrices of
// Cholesky QR, the Rayleigh-Ritz matrix Q^T (A Q) and the Ritz vectors Q V.
// Two shapes cover them, every block n x (small) with n in the millions:
//
// dense_tn -- C (m x k) = alpha A^T B, A n x m, B n x k.  The output is split
//   into tiles of 128 x TN (TN = 4 TNT columns); the n rows are split into
//   chunks, one CTA per (tile, chunk).  A CTA stages 32 rows of its A and B
//   columns at a time in shared memory (cp.async, double-buffered) and every
//   thread accumulates an 8 x 4 block of its tile in FP32 registers (32 FMAs
//   per 12 loaded values).  The CTAs write FP32 partial tiles; a finalize
//   kernel adds the chunks' partials in FP64, in chunk order (reproducible).
// dense_nn -- C (n x k) = beta C + alpha A T, A n x m, T m x k.  One CTA per
//   128 rows, all k columns: m is taken 32 at a time, the rows' chunk of A
//   and T's chunk staged in shared memory, every thread accumulating an
//   8 x 4 block of the CTA's rows and columns.
// Both keep FP32 arithmetic (the iteration measured too much pollution of
// late Krylov blocks with TF32 products); they are bound by FP32 FMA issue
// and shared-memory bandwidth.
#include <algorithm>
#include <type_traits>

#include "dm_internal.h"

namespace dm {
namespace {

constexpr int kRowsChunk = 32;   // rows staged per step
constexpr int kTM = 128;         // output rows of a dense_tn tile / rows of a dense_nn CTA

__device__ __forceinline__ void cp4(float* s, const float* g, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" :: "r"(sa), "l"(g), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp16(float* s, const float* g, int bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(sa), "l"(g), "r"(bytes) : "memory");
}
__device__ __forceinline__ void commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void wait_groups() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

// Stage rows [r0, r0 + 32) (below r1), columns [c0, c0 + w) (below cols) of a
// row-major matrix into dst[32][pitch]; everything outside is zero.  VEC:
// 16-byte copies (cols, ld and the base are multiples of 4 floats / 16 bytes).
template <bool VEC, int NT>
__device__ __forceinline__ void stage(float* dst, int pitch, const float* src, int64_t ld, int64_t r0,
                                      int64_t r1, int64_t c0, int w, int64_t cols) {
    if constexpr (VEC) {
        const int pr = w / 4;   // 16-byte pieces per row
        for (int i = threadIdx.x; i < kRowsChunk * pr; i += NT) {
            const int r = i / pr, q = i % pr;
            const int64_t row = r0 + r, col = c0 + 4 * q;
            const bool ok = row < r1 && col < cols;
            cp16(dst + r * pitch + 4 * q, ok ? src + row * ld + col : src, ok ? 16 : 0);
        }
    } else {
        for (int i = threadIdx.x; i < kRowsChunk * w; i += NT) {
            const int r = i / w, c = i % w;
            const int64_t row = r0 + r, col = c0 + c;
            const bool ok = row < r1 && col < cols;
            cp4(dst + r * pitch + c, ok ? src + row * ld + col : src, ok);
        }
    }
}

// --------------------------------------------------------------- A^T B
// Tile TM x TN = 8 TMT x 4 TNT, TMT x TNT threads.
template <int TMT, int TNT, bool VEC>
__global__ void __launch_bounds__(TMT * TNT)
dense_tn_kernel(const float* __restrict__ A, int64_t n, int m, int64_t lda, const float* __restrict__ B,
                int k, int64_t ldb, float* __restrict__ part, int64_t rows_per_chunk) {
    constexpr int NT = TMT * TNT, TN = 4 * TNT, TM = 8 * TMT;
    constexpr int PA = TM + 4, PB = TN + 4;    // padded pitches (16-byte rows)
    extern __shared__ __align__(16) float smem_f[];
    float (*As)[kRowsChunk][PA] = reinterpret_cast<float (*)[kRowsChunk][PA]>(smem_f);
    float (*Bs)[kRowsChunk][PB] = reinterpret_cast<float (*)[kRowsChunk][PB]>(smem_f + 2 * kRowsChunk * PA);
    const int tx = threadIdx.x % TNT, ty = threadIdx.x / TNT;
    const int64_t m0 = (int64_t)blockIdx.x * TM, k0 = (int64_t)blockIdx.y * TN;
    const int64_t r_begin = (int64_t)blockIdx.z * rows_per_chunk;
    const int64_t r_end = min64(n, r_begin + rows_per_chunk);
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    auto load = [&](int buf, int64_t r0) {
        stage<VEC, NT>(&As[buf][0][0], PA, A, lda, r0, r_end, m0, TM, m);
        stage<VEC, NT>(&Bs[buf][0][0], PB, B, ldb, r0, r_end, k0, TN, k);
        commit();
    };
    int buf = 0;
    if (r_begin < r_end) load(0, r_begin);
    for (int64_t r0 = r_begin; r0 < r_end; r0 += kRowsChunk, buf ^= 1) {
        if (r0 + kRowsChunk < r_end) {
            load(buf ^ 1, r0 + kRowsChunk);
            wait_groups<1>();
        } else {
            wait_groups<0>();
        }
        __syncthreads();
#pragma unroll 4
        for (int r = 0; r < kRowsChunk; ++r) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][r][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][r][ty * 8 + 4]);
            const float4 b = *reinterpret_cast<const float4*>(&Bs[buf][r][tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();   // the buffer is refilled next round
    }
    // partial tile of this chunk: part[chunk][m][k]
    float* p = part + (int64_t)blockIdx.z * m * k;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t row = m0 + ty * 8 + i;
        if (row >= m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t col = k0 + tx * 4 + j;
            if (col < k) p[row * k + col] = acc[i][j];
        }
    }
}

// C = alpha * (sum over chunks of the partials), added in FP64 in chunk order.
__global__ void dense_tn_finalize(const float* __restrict__ part, int chunks, int m, int k, float alpha,
                                  float* __restrict__ C, int64_t ldc) {
    const int64_t total = (int64_t)m * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < chunks; ++c) s += (double)part[(int64_t)c * total + e];
        const int64_t i = e / k, j = e - i * k;
        C[i * ldc + j] = (float)((double)alpha * s);
    }
}

// --------------------------------------------------------------- A T
template <int CT, bool VEC>
__global__ void __launch_bounds__(16 * CT)
dense_nn_kernel(const float* __restrict__ A, int64_t n, int m, int64_t lda, const float* __restrict__ Tm,
                int k, int64_t ldt, float* __restrict__ C, int64_t ldc, float alpha, float beta) {
    constexpr int NT = 16 * CT, KP = 4 * CT;
    constexpr int PA = kRowsChunk + 1;    // rows of A, one per row of the CTA (odd pitch)
    constexpr int PT = KP + 4;
    extern __shared__ __align__(16) float smem_f[];
    float (*Ts)[kRowsChunk][PT] = reinterpret_cast<float (*)[kRowsChunk][PT]>(smem_f);
    float (*As)[kTM][PA] = reinterpret_cast<float (*)[kTM][PA]>(smem_f + 2 * kRowsChunk * PT);
    const int tx = threadIdx.x % CT, ty = threadIdx.x / CT;
    const int64_t row0 = (int64_t)blockIdx.x * kTM;
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    // A: 128 rows x 32 columns per chunk, read as 16-byte pieces into
    // registers (a warp covers 4 whole 128-byte row segments) and stored at the
    // odd pitch (the 32 lanes of a store fall in distinct banks); T by cp.async.
    constexpr int PIECES = kTM * kRowsChunk / 4;              // 16-byte pieces per chunk
    constexpr int PER = (PIECES + NT - 1) / NT;
    const bool avec = VEC && (reinterpret_cast<uintptr_t>(A) % 16 == 0) && lda % 4 == 0 && m % 4 == 0;
    float4 ra[PER];
    auto fetch = [&](int c0) {
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int i = threadIdx.x + j * NT;
            const int r = i / (kRowsChunk / 4), q = i % (kRowsChunk / 4);
            const int64_t row = row0 + r;
            const int col = c0 + 4 * q;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < PIECES && row < n) {
                if (avec) {
                    if (col < m) v = __ldg(reinterpret_cast<const float4*>(A + row * lda + col));
                } else {
                    const float* src = A + row * lda;
                    v.x = col < m ? __ldg(src + col) : 0.f;
                    v.y = col + 1 < m ? __ldg(src + col + 1) : 0.f;
                    v.z = col + 2 < m ? __ldg(src + col + 2) : 0.f;
                    v.w = col + 3 < m ? __ldg(src + col + 3) : 0.f;
                }
            }
            ra[j] = v;
        }
    };
    auto put = [&](int buf) {
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int i = threadIdx.x + j * NT;
            if (i >= PIECES) continue;
            const int r = i / (kRowsChunk / 4), q = i % (kRowsChunk / 4);
            float* d = &As[buf][r][4 * q];
            d[0] = ra[j].x; d[1] = ra[j].y; d[2] = ra[j].z; d[3] = ra[j].w;
        }
    };
    auto load_t = [&](int buf, int c0) {
        stage<VEC, NT>(&Ts[buf][0][0], PT, Tm, ldt, c0, m, 0, KP, k);
        commit();
    };
    int buf = 0;
    fetch(0);
    load_t(0, 0);
    put(0);
    for (int c0 = 0; c0 < m; c0 += kRowsChunk, buf ^= 1) {
        const bool more = c0 + kRowsChunk < m;
        if (more) {
            fetch(c0 + kRowsChunk);          // in flight while this chunk is computed
            load_t(buf ^ 1, c0 + kRowsChunk);
            wait_groups<1>();
        } else {
            wait_groups<0>();
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kRowsChunk; ++kk) {
            float av[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) av[i] = As[buf][ty * 8 + i][kk];
            const float4 b = *reinterpret_cast<const float4*>(&Ts[buf][kk][tx * 4]);
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (more) put(buf ^ 1);              // the other buffer was last read before the previous barrier
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t row = row0 + ty * 8 + i;
        if (row >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int col = tx * 4 + j;
            if (col < k) {
                float* dst = C + row * ldc + col;
                *dst = beta == 0.f ? alpha * acc[i][j] : fmaf(beta, *dst, alpha * acc[i][j]);
            }
        }
    }
}

bool vec_ok(const void* p, int64_t ld, int64_t w) {
    return reinterpret_cast<uintptr_t>(p) % 16 == 0 && ld % 4 == 0 && w % 4 == 0;
}

template <int TMT, int TNT>
cudaError_t tn_launch(const float* A, int64_t n, int m, int64_t lda, const float* B, int k, int64_t ldb,
                      float* part, int chunks, int64_t rpc, bool vec, cudaStream_t st) {
    constexpr int TM = 8 * TMT, TN = 4 * TNT;
    const dim3 grid((unsigned)((m + TM - 1) / TM), (unsigned)((k + TN - 1) / TN), (unsigned)chunks);
    const size_t smem = 2 * (size_t)kRowsChunk * ((TM + 4) + (TN + 4)) * sizeof(float);
    auto kern = vec ? dense_tn_kernel<TMT, TNT, true> : dense_tn_kernel<TMT, TNT, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, TMT * TNT, smem, st>>>(A, n, m, lda, B, k, ldb, part, rpc);
    return cudaGetLastError();
}

template <int CT>
cudaError_t nn_launch(const float* A, int64_t n, int m, int64_t lda, const float* T, int k, int64_t ldt,
                      float* C, int64_t ldc, float alpha, float beta, bool vec, cudaStream_t st) {
    const unsigned grid = (unsigned)((n + kTM - 1) / kTM);
    const size_t smem = 2 * ((size_t)kRowsChunk * (4 * CT + 4) + (size_t)kTM * (kRowsChunk + 1)) * sizeof(float);
    auto kern = vec ? dense_nn_kernel<CT, true> : dense_nn_kernel<CT, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 16 * CT, smem, st>>>(A, n, m, lda, T, k, ldt, C, ldc, alpha, beta);
    return cudaGetLastError();
}

}  // namespace

// Row chunks of dense_tn for an (m, k) output: enough CTAs to fill the GPU a
// few times over, chunks of a multiple of 32 rows.
// Output tile rows TM in {64, 96, 128}: the fewest padded rows for m (ties:
// the larger tile).
int tn_tile_rows(int64_t m) {
    int best = 128;
    int64_t waste = (m + 127) / 128 * 128 - m;
    for (int tm : {96, 64}) {
        const int64_t w = (m + tm - 1) / tm * tm - m;
        if (w < waste) { waste = w; best = tm; }
    }
    return best;
}

void dense_tn_plan(int64_t n, int64_t m, int64_t k, int num_sms, int* chunks, int64_t* rows_per_chunk) {
    const int TN = k <= 48 ? 48 : 64;
    const int TM = tn_tile_rows(m);
    const int64_t tiles = ((m + TM - 1) / TM) * ((k + TN - 1) / TN);
    const int64_t want = std::max<int64_t>(1, (4 * (int64_t)std::max(num_sms, 1) + tiles - 1) / tiles);
    const int64_t max_chunks = std::max<int64_t>(1, (n + 255) / 256);
    const int64_t c = std::min(want, max_chunks);
    int64_t rpc = (n + c - 1) / c;
    rpc = (rpc + kRowsChunk - 1) / kRowsChunk * kRowsChunk;
    *rows_per_chunk = std::max<int64_t>(kRowsChunk, rpc);
    *chunks = (int)((n + *rows_per_chunk - 1) / *rows_per_chunk);
}

cudaError_t dense_tn_launch(const float* A, int64_t n, int64_t m, int64_t lda, const float* B, int64_t k,
                            int64_t ldb, float* C, int64_t ldc, float alpha, float* part, int num_sms,
                            cudaStream_t st, int64_t* launches) {
    int chunks = 0;
    int64_t rpc = 0;
    dense_tn_plan(n, m, k, num_sms, &chunks, &rpc);
    const bool vec = vec_ok(A, lda, m) && vec_ok(B, ldb, k);
    const int TM = tn_tile_rows(m);
    cudaError_t e;
    auto go = [&](auto tmt, auto tnt) {
        return tn_launch<decltype(tmt)::value, decltype(tnt)::value>(A, n, (int)m, lda, B, (int)k, ldb, part,
                                                                   chunks, rpc, vec, st);
    };
    using I8 = std::integral_constant<int, 8>;
    using I12 = std::integral_constant<int, 12>;
    using I16 = std::integral_constant<int, 16>;
    if (k <= 48) e = TM == 64 ? go(I8{}, I12{}) : TM == 96 ? go(I12{}, I12{}) : go(I16{}, I12{});
    else e = TM == 64 ? go(I8{}, I16{}) : TM == 96 ? go(I12{}, I16{}) : go(I16{}, I16{});
    if (e != cudaSuccess) return e;
    const int64_t total = m * k;
    const unsigned fb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 4 * (int64_t)num_sms));
    dense_tn_finalize<<<fb, 256, 0, st>>>(part, chunks, (int)m, (int)k, alpha, C, ldc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *launches += 2;
    return cudaSuccess;
}

cudaError_t dense_nn_launch(const float* A, int64_t n, int64_t m, int64_t lda, const float* T, int64_t k,
                            int64_t ldt, float* C, int64_t ldc, float alpha, float beta, cudaStream_t st,
                            int64_t* launches) {
    const bool vec = vec_ok(T, ldt, k);
    cudaError_t e;
    if (k <= 32) e = nn_launch<8>(A, n, (int)m, lda, T, (int)k, ldt, C, ldc, alpha, beta, vec, st);
    else if (k <= 48) e = nn_launch<12>(A, n, (int)m, lda, T, (int)k, ldt, C, ldc, alpha, beta, vec, st);
    else e = nn_launch<16>(A, n, (int)m, lda, T, (int)k, ldt, C, ldc, alpha, beta, vec, st);
    if (e == cudaSuccess) ++*launches;
    return e;
}

}  // namespace dm
