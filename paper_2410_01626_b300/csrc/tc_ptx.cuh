// Inline-PTX helpers for the 5th-generation tensor cores (tcgen05), TMEM, mbarriers and
// bulk asynchronous copies on sm_100-family GPUs (compiled for sm_103a).
#pragma once
#include <cstdint>

namespace fmmcph {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- mbarrier ----
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Non-blocking test of the phase with the given parity (try_wait may suspend the thread).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with the given parity; false after `limit` clock cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
    if (mbar_try_wait(bar, parity)) return true;  // fast path: no clock read
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}
// Bounded wait by every lane of a warp; the result is warp-uniform, so that a timeout seen by
// one lane can never leave the warp divergent before a whole-warp (elect.sync) instruction.
__device__ __forceinline__ bool mbar_wait_all(uint64_t* bar, uint32_t parity, long long limit) {
    return __all_sync(0xffffffffu, mbar_wait(bar, parity, limit));
}
// The same bounded wait for warps that are not latency critical: between polls the thread
// sleeps (32 ns doubling to 512 ns), so that it leaves the issue slots of its SM sub-partition
// to the single-thread producer and MMA issuer.
__device__ __forceinline__ bool mbar_wait_backoff(uint64_t* bar, uint32_t parity, long long limit) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    unsigned ns = 32;
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
        __nanosleep(ns);
        if (ns < 512) ns <<= 1;
    }
    return true;
}

// Bounded waits that also give up when another role of the CTA has set the shared abort flag
// (read only while the barrier is not yet complete, so the fast path is unchanged).  They
// return true only when the phase has completed.
__device__ __forceinline__ bool mbar_wait_abort(uint64_t* bar, uint32_t parity, long long limit,
                                                const volatile int* abort) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort || clock64() - t0 > limit) return false;
    }
    return true;
}
__device__ __forceinline__ bool mbar_wait_all_abort(uint64_t* bar, uint32_t parity, long long limit,
                                                    const volatile int* abort) {
    return __all_sync(0xffffffffu, mbar_wait_abort(bar, parity, limit, abort));
}
__device__ __forceinline__ bool mbar_wait_backoff_abort(uint64_t* bar, uint32_t parity, long long limit,
                                                        const volatile int* abort) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    unsigned ns = 32;
    while (!mbar_try_wait(bar, parity)) {
        if (*abort || clock64() - t0 > limit) return false;
        __nanosleep(ns);
        if (ns < 512) ns <<= 1;
    }
    return true;
}

// ---- bulk asynchronous copy global -> shared (16-byte aligned, size multiple of 16) ----
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---- tensor memory ----
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem desc] x B[smem desc]^T, TF32 inputs, FP32 accumulate; single thread.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// D[tmem] (+)= A x B^T with BF16 inputs (kind::f16), FP32 accumulate; single thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Arrive on `bar` once every previously issued tcgen05 operation of this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// Whole-warp forms: every lane of the warp executes the instruction and one elected lane issues
// it.  Keeping the issuing loop warp-wide keeps its descriptors warp-uniform, which makes each
// MMA issue much cheaper than from a lone thread inside a divergent branch (measured on the M2L:
// 0.76 -> 0.64 ms at 500k atoms).
__device__ __forceinline__ void mma_bf16_w(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
        " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_tf32_w(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
        " @e tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit_w(uint64_t* bar) {
    asm volatile(
        "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
        " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}" ::"r"(smem_u32(bar))
        : "memory");
}

// One K step of a split product (hi*hi + hi*lo + lo*hi) into D, all three MMAs issued by one
// elected lane of the warp, optionally followed by a commit to `bar`: one election per K step
// keeps the issuing loop short enough for the tensor pipe never to wait on it (N = 192).
template <bool BF16, bool COMMIT>
__device__ __forceinline__ void mma3_w(uint32_t d_tmem, uint64_t a, uint64_t b, uint64_t alo, uint64_t blo,
                                       uint32_t idesc, uint32_t accumulate, uint64_t* bar) {
    if (BF16) {
        if (COMMIT)
            asm volatile(
                "{\n .reg .pred p, e;\n setp.ne.b32 p, %6, 0;\n elect.sync _|e, 0xffffffff;\n"
                " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %5, p;\n"
                " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %4, %5, 1;\n"
                " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %3, %2, %5, 1;\n"
                " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%7];\n}" ::"r"(d_tmem),
                "l"(a), "l"(b), "l"(alo), "l"(blo), "r"(idesc), "r"(accumulate), "r"(smem_u32(bar))
                : "memory");
        else
            asm volatile(
                "{\n .reg .pred p, e;\n setp.ne.b32 p, %6, 0;\n elect.sync _|e, 0xffffffff;\n"
                " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %5, p;\n"
                " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %4, %5, 1;\n"
                " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %3, %2, %5, 1;\n}" ::"r"(d_tmem),
                "l"(a), "l"(b), "l"(alo), "l"(blo), "r"(idesc), "r"(accumulate)
                : "memory");
    } else {
        if (COMMIT)
            asm volatile(
                "{\n .reg .pred p, e;\n setp.ne.b32 p, %6, 0;\n elect.sync _|e, 0xffffffff;\n"
                " @e tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %5, p;\n"
                " @e tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %4, %5, 1;\n"
                " @e tcgen05.mma.cta_group::1.kind::tf32 [%0], %3, %2, %5, 1;\n"
                " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%7];\n}" ::"r"(d_tmem),
                "l"(a), "l"(b), "l"(alo), "l"(blo), "r"(idesc), "r"(accumulate), "r"(smem_u32(bar))
                : "memory");
        else
            asm volatile(
                "{\n .reg .pred p, e;\n setp.ne.b32 p, %6, 0;\n elect.sync _|e, 0xffffffff;\n"
                " @e tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %5, p;\n"
                " @e tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %4, %5, 1;\n"
                " @e tcgen05.mma.cta_group::1.kind::tf32 [%0], %3, %2, %5, 1;\n}" ::"r"(d_tmem),
                "l"(a), "l"(b), "l"(alo), "l"(blo), "r"(idesc), "r"(accumulate)
                : "memory");
    }
}
// N (1 to 3) kind::f16 products (a0, b0) .. into D by one elected lane, then a commit to
// `bar`, in one instruction group with a non-blocking test of the phase `parity` of `probe_bar`
// (returned, 1 = complete): the test's latency passes while the MMAs issue, instead of before
// the next wait.  The first product accumulates when `accumulate` is nonzero, the others always.
template <int N>
__device__ __forceinline__ uint32_t mma_f16_n_probe_w(uint32_t d_tmem, uint64_t a0, uint64_t b0, uint64_t a1,
                                                      uint64_t b1, uint64_t a2, uint64_t b2, uint32_t idesc,
                                                      uint32_t accumulate, uint64_t* bar, uint64_t* probe_bar,
                                                      uint32_t parity) {
    static_assert(N >= 1 && N <= 3, "1 to 3 products");
    uint32_t ready;
    if (N == 1)
        asm volatile(
            "{\n .reg .pred p, e, q;\n mbarrier.test_wait.parity.shared::cta.b64 q, [%6], %7;\n"
            " setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
            " @e tcgen05.mma.cta_group::1.kind::f16 [%1], %2, %3, %8, p;\n"
            " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%5];\n"
            " selp.u32 %0, 1, 0, q;\n}"
            : "=r"(ready)
            : "r"(d_tmem), "l"(a0), "l"(b0), "r"(accumulate), "r"(smem_u32(bar)), "r"(smem_u32(probe_bar)),
              "r"(parity), "r"(idesc)
            : "memory");
    else if (N == 2)
        asm volatile(
            "{\n .reg .pred p, e, q;\n mbarrier.test_wait.parity.shared::cta.b64 q, [%9], %10;\n"
            " setp.ne.b32 p, %7, 0;\n elect.sync _|e, 0xffffffff;\n"
            " @e tcgen05.mma.cta_group::1.kind::f16 [%1], %2, %3, %6, p;\n"
            " @e tcgen05.mma.cta_group::1.kind::f16 [%1], %4, %5, %6, 1;\n"
            " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%8];\n"
            " selp.u32 %0, 1, 0, q;\n}"
            : "=r"(ready)
            : "r"(d_tmem), "l"(a0), "l"(b0), "l"(a1), "l"(b1), "r"(idesc), "r"(accumulate), "r"(smem_u32(bar)),
              "r"(smem_u32(probe_bar)), "r"(parity)
            : "memory");
    else
        asm volatile(
            "{\n .reg .pred p, e, q;\n mbarrier.test_wait.parity.shared::cta.b64 q, [%11], %12;\n"
            " setp.ne.b32 p, %9, 0;\n elect.sync _|e, 0xffffffff;\n"
            " @e tcgen05.mma.cta_group::1.kind::f16 [%1], %2, %3, %8, p;\n"
            " @e tcgen05.mma.cta_group::1.kind::f16 [%1], %4, %5, %8, 1;\n"
            " @e tcgen05.mma.cta_group::1.kind::f16 [%1], %6, %7, %8, 1;\n"
            " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%10];\n"
            " selp.u32 %0, 1, 0, q;\n}"
            : "=r"(ready)
            : "r"(d_tmem), "l"(a0), "l"(b0), "l"(a1), "l"(b1), "l"(a2), "l"(b2), "r"(idesc), "r"(accumulate),
              "r"(smem_u32(bar)), "r"(smem_u32(probe_bar)), "r"(parity)
            : "memory");
    return ready;
}

// One TF32 MMA by one elected lane, optionally followed by a commit to `bar`.
template <bool COMMIT>
__device__ __forceinline__ void mma1_tf32_w(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate,
                                            uint64_t* bar) {
    if (COMMIT)
        asm volatile(
            "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
            " @e tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
            " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%5];\n}" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate), "r"(smem_u32(bar))
            : "memory");
    else
        asm volatile(
            "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
            " @e tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
            : "memory");
}

// 32 lanes x 32 bits, 16 consecutive columns per thread: thread t of warp w reads
// TMEM lane (32 w + t), columns [col, col + 16).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor, K-major, no swizzle (core matrices of 8 rows x 16 bytes):
//   lbo = byte distance between core matrices adjacent in K,
//   sbo = byte distance between core matrices adjacent in M (or N).
__host__ __device__ constexpr uint64_t smem_desc_kmajor(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major, dense.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor: kind::f16, D = F32, A = B = BF16, both K-major, dense.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor: kind::f16, D = F32, A = B = FP16, both K-major, dense.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float round_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

}  // namespace tc
}  // namespace fmmcph
