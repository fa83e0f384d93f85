// Pass kernels of 128 px patches (the CTA-per-unit kernels of generic_kernels.cuh).
#include "generic_kernels.cuh"

namespace mfbd_dev {

template int generic_adjoint_ctas_n<128>(int es, int sms);
template cudaError_t launch_generic_forward_n<128>(const GenericParams& prm, int sms, cudaStream_t s);
template cudaError_t launch_generic_adjoint_n<128>(const GenericParams& prm, int sms, cudaStream_t s);

}  // namespace mfbd_dev
