// Host side of the batched persistent kernel (batch_kernels.cuh): shared-memory
// size and the dispatch over its two register variants.
#include "batch_internal.h"

#include <algorithm>

namespace mfbd_dev {

size_t batch_smem(int es_small, int es_large) {
    // four 64-pixel warps, one 128-pixel unit, or the P item's coefficient tile
    const size_t small = (size_t)(kBT / 32) * 64 * es_small * sizeof(float2);
    const size_t large = (size_t)128 * es_large * sizeof(float2);
    const size_t proj = (size_t)kJC * 256 * sizeof(float);
    return std::max(std::max(small, large), proj);
}

int batch_max_ctas_per_sm(size_t smem, int variant) {
    return variant == 1 ? batch_max_ctas_variant<3>(smem) : batch_max_ctas_variant<2>(smem);
}

cudaError_t launch_batch(const BatchParams& prm, int ctas, size_t smem, int variant, cudaStream_t s) {
    if (prm.n_items == 0) return cudaSuccess;
    return variant == 1 ? launch_batch_variant<3>(prm, ctas, smem, s) : launch_batch_variant<2>(prm, ctas, smem, s);
}

}  // namespace mfbd_dev
