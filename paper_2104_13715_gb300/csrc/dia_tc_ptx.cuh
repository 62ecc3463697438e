// Inline-PTX building blocks of the tcgen05 kernels (sm_103a): shared-memory
// matrix and instruction descriptors, the MMA, mbarriers and a bounded wait.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dia {

constexpr long long kTcWaitCycles = 2000000000LL;   // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t su32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// No-swizzle shared-memory matrix descriptor (version 1): start address,
// leading byte offset = stride between core matrices (8 rows x 16 bytes)
// along K, stride byte offset = stride between core matrices along M / N.
// The same assignment holds for K-major and MN-major operands; in an MN-major
// operand a core matrix's 16-byte rows run along K and hold 8 M / N elements.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::f16 with float32 accumulators: A and B both
// bf16 (f16 = 0) or both f16 (f16 = 1); a_mn / b_mn = 1 for an MN-major
// operand (else K-major); M, N the MMA shape.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N, int a_mn = 0, int b_mn = 0,
                                               int f16 = 0) {
    return (1u << 4) | ((f16 ? 0u : 1u) << 7) | ((f16 ? 0u : 1u) << 10) |
           ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t taddr, uint64_t a, uint64_t b, uint32_t idesc,
                                       int acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                 :: "r"(taddr), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// the same MMA accumulating unconditionally (no predicate set-up: the issue
// loop's cost per MMA bounds small-N products)
__device__ __forceinline__ void tc_mma_acc(uint32_t taddr, uint64_t a, uint64_t b, uint32_t idesc) {
    asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 1;"
                 :: "r"(taddr), "l"(a), "l"(b), "r"(idesc));
}

__device__ __forceinline__ void mbar_init(uint64_t *b, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(su32(b)) : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(su32(b)));
}

// Wait for the phase with parity `ph`; false after `limit` SM clock cycles or
// once the other role has aborted (*other != 0).
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t ph, const int *other,
                                        long long limit = kTcWaitCycles) {
    const long long t0 = clock64();
    const volatile int *ab = other;
    for (;;) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n" : "=r"(done) : "r"(su32(bar)), "r"(ph));
        if (done) return true;
        if (*ab != 0 || clock64() - t0 > limit) return false;
    }
}

// A kernel's own bounds check failed: status[0] <- code (2 forward pass, 3
// weight gradient), status[1] <- the low bits of the offending index; the
// access itself is skipped.
__device__ __forceinline__ void tc_report_bad(int *status, int code, size_t idx) {
    atomicExch(status, code);
    atomicExch(status + 1, (int)(idx & 0x7fffffff));
}

}  // namespace dia
