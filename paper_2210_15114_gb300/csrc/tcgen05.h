// Device helpers of the kernels that use the 5th-generation tensor cores
// (tcgen05), the bulk-copy engine and shared-memory mbarriers (the squared-l2
// reduce and apply).  Every wait here is bounded by an explicit round limit.
#pragma once

#include <cstdint>

namespace dm {
namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// One tcgen05.mma (kind::tf32, one CTA); accumulate = 0 overwrites D.
__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}

// v = hi + lo with hi = v with its 13 low mantissa bits cleared and lo the
// same of v - hi (both exact TF32 values, whatever conversion the tensor
// core applies to its inputs): |v - hi - lo| < 2^-20 |v|.
__device__ __forceinline__ void split_tf32(float v, float& hi, float& lo) {
    hi = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
    lo = __uint_as_float(__float_as_uint(v - hi) & 0xFFFFE000u);
}

__device__ __forceinline__ void tc_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "r"(taddr) : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}

// tcgen05.ld of 8 columns without the wait (the caller waits once for all).
__device__ __forceinline__ void tc_ld8_issue(uint32_t taddr, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "r"(taddr) : "memory");
}

__device__ __forceinline__ uint64_t tc_desc_sbo(uint32_t saddr, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((128u >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(mbar), "r"(count) : "memory");
}

// One try_wait on an mbarrier phase: the thread is suspended until the
// phase completes or a hardware time limit passes, so a waiting warp takes
// no issue slots.
__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
    return done != 0;
}

// Bounded wait on an mbarrier phase with an explicit round limit.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try(mbar, parity)) return true;
    return false;
}

// One bulk copy global -> shared of `bytes` (a multiple of 16, both addresses
// 16-byte aligned), completion counted on mbar (the caller's arrive carries
// the transaction count).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mbar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}

// Bounded wait on an mbarrier phase that also gives up once the CTA's abort
// word is set (another thread's wait ran out).
__device__ __forceinline__ bool mbar_wait_ab(uint32_t mbar, uint32_t parity, uint32_t limit,
                                             volatile uint32_t* abort_w) {
    for (uint32_t i = 0; i < limit; ++i) {
        if (mbar_try(mbar, parity)) return true;
        if (*abort_w) return false;
    }
    return false;
}

// Bulk copy global -> shared without an arrive (the caller has set the
// transaction count of the whole stage on mbar).
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}

}  // namespace
}  // namespace dm
