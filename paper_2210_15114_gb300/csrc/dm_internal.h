// Internal declarations shared by the CUDA translation units of libdm.
#pragma once

#include <cstdint>
#include <cstddef>
#include <cuda_runtime.h>

#include "../../include/dm.h"

namespace dm {

// ------------------------------------------------------------------ errors
// Device error word values (first error wins, see set_error()).
enum : uint32_t { kErrNone = 0, kErrNonfinite = DM_ERR_NONFINITE, kErrTimeout = DM_ERR_TIMEOUT,
                  kErrInternal = DM_ERR_INTERNAL };

// Default iteration cap of every device-side spin wait (with a short
// __nanosleep per round, about a second in total).  On expiry the waiting
// kernel latches DM_ERR_TIMEOUT, stops waiting and finishes its tile with
// what it has.  A context can lower it (dm_set_wait_limit); the radix passes
// and the ordered l1 query take the context's value as a launch argument.
constexpr uint32_t kSpinLimit = 1u << 20;

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ void set_error(uint32_t* err, uint32_t code) {
    atomicCAS(err, 0u, code);
}

// ----------------------------------------------------------- memory order
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_release_add(uint32_t* p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// ------------------------------------------------------------ element types
template <dm_dtype DT> struct Types;
template <> struct Types<DM_F32> {
    using V = float;      // coordinate / query element
    using Acc = float;    // per-element and in-tile arithmetic
    using Wide = double;  // per-tile and cross-tile arithmetic
    using Out = float;    // result element
    using Key = uint32_t; // radix key
};
template <> struct Types<DM_F64> {
    using V = double; using Acc = double; using Wide = double; using Out = double;
    using Key = unsigned long long;
};
template <> struct Types<DM_I32> {
    using V = int32_t; using Acc = long long; using Wide = long long; using Out = long long;
    using Key = uint32_t;
};

inline size_t dtype_size(dm_dtype t) { return t == DM_F64 ? 8 : 4; }
inline size_t out_size(dm_dtype t) { return t == DM_F32 ? 4 : 8; }
inline int key_bits(dm_dtype t) { return t == DM_F64 ? 64 : 32; }

// ---------------------------------------------------------------- launches
// Radix sort of every coordinate column (Algorithm 1).
struct SortArgs {
    dm_dtype dtype;
    const void* X; int64_t n, d, ldx;
    void* keys_a; void* keys_b;          // d x n keys (ping-pong)
    int32_t* vals_a; int32_t* vals_b;    // d x n payload (ping-pong)
    uint32_t* hist;                      // d x passes x 256 digit counts
    uint32_t* lookback;                  // passes x d x tiles x 256 status words
    uint32_t* counters;                  // passes tile counters
    void* sorted_out; int32_t* perm_out; // plan outputs, d x n
    uint32_t* err;
    uint32_t spin_limit = kSpinLimit;    // rounds of a look-back wait before DM_ERR_TIMEOUT
};
size_t sort_hist_words(dm_dtype t, int64_t d);
size_t sort_lookback_words(dm_dtype t, int64_t n, int64_t d);
int sort_passes(dm_dtype t);
// Launch the keygen + histogram kernel.
cudaError_t sort_launch_keygen(const SortArgs& a, cudaStream_t s, int64_t* launches);
// Launch the radix passes listed in pass_list (digit positions, ascending).
cudaError_t sort_launch_passes(const SortArgs& a, const int* pass_list, int npass,
                               cudaStream_t s, int64_t* launches);
// Test of the bounded look-back wait: one CTA of the first FP32 radix pass
// over one column of two tiles, started as the column's second tile (the
// caller sets *counters to 1 and zeroes the histogram and look-back words),
// so its predecessor never publishes.  Writes stay inside the first tile of
// keys_b / vals_b; the wait runs out after a.spin_limit rounds.
cudaError_t sort_launch_unpublished_wait(const SortArgs& a, cudaStream_t s, int64_t* launches);
int sort_tile_f32();

// Column sums of the query block and the shifted contraction:
//   u[j]   = sum_i Z[i,j]
//   W[c,j] = sum_i (X[i,c] - mu[c]) Z[i,j]      (mu == nullptr: no shift)
//   v[j]   = sum_i s_i Z[i,j],  s_i = ||x_i - mu||^2   (with_s; else 0)
// Result layout in `res` (Wide type): W (d x k), then u (k), then v (k).
// X holds V elements, or Acc elements when x_acc is set.
struct ReduceArgs {
    dm_dtype dtype;
    const void* X; int64_t n, d, ldx;
    bool x_acc;
    const void* mu; int64_t mu_stride;   // shift mu[c] = mu[c * mu_stride] (V type)
    bool with_s;
    const void* Z; int64_t k, ldz;
    void* partial;                       // scratch: blocks x (d+2) x k Wide
    void* res;                           // (d+2) x k Wide
    int num_sms;
    int max_blocks;                      // 0: no cap beyond the default
    uint32_t* err;                       // device error word (may be null)
    int engine;                          // dm_engine: the contraction's units
    uint32_t spin_limit = kSpinLimit;    // rounds of a tensor-core wait before DM_ERR_TIMEOUT
};
bool reduce_supported(int64_t d, int64_t k);   // any element type (FP64 worst case)
int64_t reduce_max_k(dm_dtype t, int64_t d);   // columns per launch for this type
int reduce_blocks(const ReduceArgs& a);
cudaError_t reduce_launch(const ReduceArgs& a, cudaStream_t s, int64_t* launches);

// R_i = sum_c (X[i,c] - mu_c) (Acc type), mu_c = mu[c * mu_stride] (V type).
cudaError_t rowsum_launch(dm_dtype t, const void* X, int64_t n, int64_t d, int64_t ldx,
                          const void* mu, int64_t mu_stride, void* R, cudaStream_t s,
                          int64_t* launches);

// Column means mu (V type, rounded): the frame shift of the squared-l2 plan.
struct L2PrepArgs {
    dm_dtype dtype;
    const void* X; int64_t n, d, ldx;
    void* partial;                       // scratch: blocks x d Wide
    void* mu;                            // d entries, V type
    uint32_t* err;                       // may be null (non-finite input not reported)
    int max_blocks;                      // 0: no cap beyond the default
};
int l2prep_blocks(const L2PrepArgs& a);
cudaError_t l2prep_launch(const L2PrepArgs& a, cudaStream_t s, int64_t* launches);

// out_i = s_i u + v - 2 (x_i - mu) . W,  s_i = ||x_i - mu||^2
struct L2ApplyArgs {
    dm_dtype dtype;
    const void* X; int64_t n, d, ldx;
    const void* mu;
    const void* res;                     // W, u, v as produced by the reduce
    int64_t k;
    void* out; int64_t ldo;
    int num_sms;
    int engine = DM_ENGINE_AUTO;         // dm_engine: the contraction's units
    uint32_t* err = nullptr;             // device error word (bounded waits)
    uint32_t spin_limit = kSpinLimit;
};
cudaError_t l2apply_launch(const L2ApplyArgs& a, cudaStream_t s, int64_t* launches);

// l1 query: scan + evaluate + cross-coordinate accumulation (Algorithm 2),
// launched in order on one stream with the same arguments and scratch:
// l1_prologue_launch (R^T Z, 1^T Z, group-major copy of Z),
// l1_aggregate_launch (tile sums and their per-coordinate exclusive scan),
// l1_query_launch (the sorted pass), l1_finalize_launch (L2-reduction mode).
struct L1QueryArgs {
    dm_dtype dtype;
    const void* xs; const int32_t* perm; int64_t n, d;   // plan (d x n each)
    const void* R;                       // plan: R_i = sum_c (x_i(c) - mu_c), Acc type
    const void* mu;  int64_t mu_stride;  // the shift mu_c (V type)
    const void* Z; int64_t k, ldz;
    void* out; int64_t ldo;
    void* scratch;                       // l1_query_scratch_bytes()
    uint32_t* err;
    int num_sms;
    int deterministic;                   // 1: ordered accumulation, 0: L2 reductions
    uint32_t spin_limit = kSpinLimit;    // rounds of the ordered mode's wait
};
size_t l1_query_scratch_bytes(dm_dtype t, int64_t n, int64_t d, int64_t k, int num_sms);
cudaError_t l1_prologue_launch(const L1QueryArgs& a, cudaStream_t s, int64_t* launches);
cudaError_t l1_query_launch(const L1QueryArgs& a, cudaStream_t s, int64_t* launches);
cudaError_t l1_finalize_launch(const L1QueryArgs& a, cudaStream_t s, int64_t* launches);
cudaError_t l1_aggregate_launch(const L1QueryArgs& a, cudaStream_t s, int64_t* launches);

// Plain on-the-fly product (baseline).
struct BruteArgs {
    dm_dtype dtype; dm_metric metric;
    const void* X; int64_t n, d, ldx;
    const void* Z; int64_t k, ldz;
    void* out; int64_t ldo;
};
cudaError_t brute_launch(const BruteArgs& a, cudaStream_t s, int64_t* launches);

// Gradient of L = sum_q w_q^T A(X) z_q with respect to X (grad.cu).
struct GradArgs {
    dm_dtype dtype;
    int64_t n, d;
    const void* W; int64_t ldw;          // n x k
    const void* Z; int64_t ldz;          // n x k
    int64_t k;
    void* G; int64_t ldg;                // n x d result (Out type)
    void* scratch;                       // grad_scratch_bytes()
    int num_sms;
    // l1 plan
    const void* xs; const int32_t* perm;
    // squared-l2 plan
    const void* X; int64_t ldx; const void* mu; const void* res;
};
size_t grad_scratch_bytes(dm_dtype t, int64_t n, int64_t d, int64_t k);
const void* grad_packed(const GradArgs& a);   // the packed (z_q, w_q) pairs, n x 2k
cudaError_t grad_pack_launch(const GradArgs& a, cudaStream_t s, int64_t* launches);
// stage 0: tile sums, 1: scan over tiles, 2: evaluation and scatter into a
// coordinate-major copy, 3: transpose of that copy into G
cudaError_t grad_l1_launch(const GradArgs& a, int stage, cudaStream_t s, int64_t* launches);
cudaError_t grad_l2_apply_launch(const GradArgs& a, cudaStream_t s, int64_t* launches);

// ||x - y||_p^p for odd p through the sorted order (grad.cu): stage 0 tile
// sums of the p + 1 weights y (-x~)^s, 1 scan over tiles, 2 evaluation,
// added into out (which the caller zeroes first).
struct OddArgs {
    dm_dtype dtype;
    int64_t n, d;
    const void* xs; const int32_t* perm;  // the l1 plan's sorted coordinates
    const void* Z; int64_t ldz; int64_t k;
    int p;                                // odd, 3..15
    void* out; int64_t ldo;
    void* scratch;                        // oddp_scratch_bytes()
};
size_t oddp_scratch_bytes(int64_t n, int64_t d, int64_t k, int p);
cudaError_t oddp_launch(const OddArgs& a, int stage, cudaStream_t s, int64_t* launches);

// Dense products on tall-skinny FP32 blocks (dense.cu), for the block Krylov
// iteration.  dense_tn: C (m x k) = alpha A^T B (A n x m, B n x k), partial
// tiles in `part` (dense_tn_plan's chunks x m x k floats), then added in FP64.
// dense_nn: C (n x k) = beta C + alpha A T (A n x m, T m x k), k <= 64.
void dense_tn_plan(int64_t n, int64_t m, int64_t k, int num_sms, int* chunks, int64_t* rows_per_chunk);
cudaError_t dense_tn_launch(const float* A, int64_t n, int64_t m, int64_t lda, const float* B, int64_t k,
                            int64_t ldb, float* C, int64_t ldc, float alpha, float* part, int num_sms,
                            cudaStream_t st, int64_t* launches);
cudaError_t dense_nn_launch(const float* A, int64_t n, int64_t m, int64_t lda, const float* T, int64_t k,
                            int64_t ldt, float* C, int64_t ldc, float alpha, float beta, cudaStream_t st,
                            int64_t* launches);

// Variants (variants.cu).
cudaError_t scale_launch(dm_dtype t, void* out, int64_t n, int64_t k, int64_t ldo, double s,
                         int num_sms, cudaStream_t st, int64_t* launches);
size_t lpp_feature_bytes(dm_dtype t, int64_t n, int64_t d, int p);
cudaError_t lpp_features_launch(dm_dtype t, const void* X, int64_t n, int64_t d, int64_t ldx,
                                const void* mu, int p, void* F, int num_sms, cudaStream_t st,
                                int64_t* launches);
size_t lpp_apply_smem(dm_dtype t, int64_t d, int p, int64_t k);
cudaError_t lpp_apply_launch(dm_dtype t, const void* X, int64_t n, int64_t d, int64_t ldx,
                             const void* mu, const void* res, int p, int64_t k, void* out, int64_t ldo,
                             int num_sms, cudaStream_t st, int64_t* launches);
size_t project_smem(dm_dtype t, int64_t d, int64_t m);
cudaError_t project_launch(dm_dtype t, const void* X, int64_t n, int64_t d, int64_t ldx, const void* G,
                           int64_t m, void* Xp, int num_sms, cudaStream_t st, int64_t* launches);

}  // namespace dm
