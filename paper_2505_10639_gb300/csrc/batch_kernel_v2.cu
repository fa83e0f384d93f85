// The batch kernel of batch_kernels.cuh compiled for 2 CTAs per SM
// (up to 255 registers a thread).
// scalar complex adds in this kernel (see fft_reg.cuh)
#define MFBD_SCALAR_COMPLEX_ADD 1
#include "batch_kernels.cuh"

namespace mfbd_dev {

template int batch_max_ctas_variant<2>(size_t smem);
template cudaError_t launch_batch_variant<2>(const BatchParams& prm, int ctas, size_t smem, cudaStream_t s);

}  // namespace mfbd_dev
