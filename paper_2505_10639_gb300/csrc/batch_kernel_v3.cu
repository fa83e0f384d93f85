// The batch kernel of batch_kernels.cuh compiled for 3 CTAs per SM
// (up to 170 registers a thread; the 96 and 128 px passes spill).
// scalar complex adds in this kernel (see fft_reg.cuh)
#define MFBD_SCALAR_COMPLEX_ADD 1
#include "batch_kernels.cuh"

namespace mfbd_dev {

template int batch_max_ctas_variant<3>(size_t smem);
template cudaError_t launch_batch_variant<3>(const BatchParams& prm, int ctas, size_t smem, cudaStream_t s);

}  // namespace mfbd_dev
