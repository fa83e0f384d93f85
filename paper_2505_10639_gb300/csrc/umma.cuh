// 5th-generation tensor-core (tcgen05) helpers shared by the modal
// projections: shared-memory operand descriptors, the kind::f16 instruction
// descriptor, the MMA itself and the three-plane BF16 products.
#pragma once

#include <cstdint>

namespace mfbd_dev {
namespace umma {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory descriptor of a no-swizzle, K-major operand: core matrices
// of 8 rows x 16 bytes; `lbo` bytes between core matrices adjacent along K,
// `sbo` bytes between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, absolute LBO mode, layout 0 = no swizzle
}

// kind::f16 instruction descriptor: BF16 A and B, both K-major, FP32 D,
// an m x n tile.
__host__ __device__ constexpr uint32_t instr_desc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// The MMAs of one tile or chunk from one thread: the plane pairs of weight
// >= 2^-16 in decreasing weight (one pair with one plane), `ksteps` K-steps of
// 16 each. da0 / db0 describe plane 0 of A / B; a plane is a_plane / b_plane
// bytes further and a K-step 256 bytes (two core matrices along K, 128 bytes
// apart; the descriptor's address field counts 16-byte units, and no
// shared-memory address overflows it).
__device__ __forceinline__ void issue_mmas(uint32_t tmem_d, uint64_t da0, uint64_t db0, uint32_t a_plane,
                                           uint32_t b_plane, int ksteps, int planes, uint32_t idesc, bool accumulate) {
    const uint32_t pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
    const int npairs = planes == 3 ? 6 : 1;
    uint32_t acc = accumulate ? 1u : 0u;
    for (int pp = 0; pp < npairs; ++pp) {
        const uint64_t da = da0 + ((pa[pp] * a_plane) >> 4), db = db0 + ((pb[pp] * b_plane) >> 4);
        for (int s = 0; s < ksteps; ++s) {
            mma_bf16(tmem_d, da + (uint64_t)(s * 16), db + (uint64_t)(s * 16), idesc, acc);
            acc = 1u;
        }
    }
}

// One arrival on `mbar` once every tcgen05 operation this thread issued
// before has completed.
__device__ __forceinline__ void commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(mbar))
                 : "memory");
}

__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

}  // namespace umma
}  // namespace mfbd_dev
