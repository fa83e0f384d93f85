// Tensor-memory-accelerator (TMA) tile loads with an mbarrier, and the host
// side that encodes their tensor maps (cuTensorMapEncodeTiled, reached
// through the runtime's driver entry point so the library links no libcuda).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace mfbd_dev {
namespace tma {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Bounded polls of an mbarrier phase (each try_wait may suspend the thread
// for a while): about a second or more before a wait gives up.
constexpr long long kWaitPolls = 1ll << 22;

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    // make the initialised barrier visible to the asynchronous proxy
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One arrival that also announces `bytes` of asynchronous transactions.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// true once the phase with this parity has completed; false when the
// bounded poll gives up
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (long long it = 0; it < kWaitPolls; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Generic-proxy accesses of shared memory before asynchronous-proxy writes
// (a TMA load into a buffer that was just read).
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 2-D tiled load of the box at (x, y) (x in elements of the innermost
// dimension; x times the element size a multiple of 16 bytes) into `dst`,
// completing `bytes` transactions on `bar`.
__device__ __forceinline__ void load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Host: a 2-D tensor map over a row-major float32 array of `rows` rows of
// `cols` elements (row pitch `cols` elements), boxes of box_rows x box_cols,
// 128-byte swizzle (box_cols * 4 must be 128). Returns false when the driver
// entry point is missing or the encoding is refused (alignment, sizes).
bool encode_f32_2d_swizzle128(CUtensorMap* map, const float* base, uint64_t cols, uint64_t rows, uint32_t box_cols,
                              uint32_t box_rows);

}  // namespace tma
}  // namespace mfbd_dev
