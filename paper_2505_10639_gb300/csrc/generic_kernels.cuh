// Pass kernels of one problem for patch sizes other than 64 (48, 96, 128),
// and for 64 on request: one CTA per unit (patch, object, frame),
// persistent over the units; for N <= 64 the CTA is one warp. The passes
// themselves (Sec. 3.1, Eqs. 20-22 and their adjoint) are in unit_passes.cuh.
// Each patch size is instantiated in a translation unit of its own
// (generic_n48.cu ... generic_n128.cu) so that they compile in parallel.
#pragma once

#include <algorithm>
#include "mfbd_internal.h"
#include "unit_passes.cuh"

namespace mfbd_dev {

namespace generic_detail {

namespace {

using namespace unitpass;

template <int N>
__device__ __forceinline__ UnitPtr unit_ptr(const GenericParams& prm, long long u) {
    const int J = prm.J, K = prm.K;
    const int j = (int)(u % J);
    const long long pk = u / J;
    const int k = (int)(pk % K);
    const long long p = pk / K;
    const GenericObj& ob = prm.obj[k];
    const long long img = (p * J + j) * (long long)ob.W * ob.W;
    UnitPtr q;
    q.phi = prm.phi + ob.phi_off + img;
    q.gphi = prm.gphi + ob.phi_off + img;
    q.h = prm.gscr + (size_t)u * N * Geo<N>::NH;
    q.pf = prm.pscr ? prm.pscr + (size_t)u * N * N : nullptr;
    q.pp = prm.uscr ? prm.uscr + (size_t)u * prm.ustride : nullptr;
    q.mask = ob.mask;
    q.mw = ob.mw;
    q.W = ob.W;
    q.inv_z = ob.inv_z;
    q.supp = ob.supp;
    q.sw = prm.sw;
    q.cmask = ob.cmask;
    q.csupp = ob.csupp;
    return q;
}

// Threads of a CTA: N <= 64, one warp working on one unit at a time (32
// lines per round, no CTA barrier); N = 96, 128, 128 threads on one unit (64
// lines of two lanes per round).
template <int N>
struct Cta {
    static constexpr bool WARP = N <= 64;
    static constexpr int THREADS = WARP ? 32 : Geo<N>::THREADS;
    static constexpr int LINES = WARP ? 32 : Geo<N>::LINES;
    static constexpr int MIN_CTAS = WARP ? 12 : 1;  // 12 warps per SM: at most 170 registers a thread
};

template <int N>
__global__ void __launch_bounds__(Cta<N>::THREADS, Cta<N>::MIN_CTAS) generic_forward_kernel(const GenericParams prm) {
    extern __shared__ __align__(16) unsigned char gsm[];
    float2* E = reinterpret_cast<float2*>(gsm);
    const long long units = (long long)prm.P * prm.K * prm.J;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        constexpr int L = Cta<N>::LINES;
        if constexpr (Cta<N>::WARP) unit_forward_rounds<N, L>(unit_ptr<N>(prm, u), E, prm.es, threadIdx.x, WarpBar{});
        else unit_forward<N, L>(unit_ptr<N>(prm, u), E, prm.es, threadIdx.x, CtaBar{});
    }
}

template <int N, bool RECOMPUTE>
__global__ void __launch_bounds__(Cta<N>::THREADS, Cta<N>::MIN_CTAS) generic_adjoint_kernel(const GenericParams prm) {
    extern __shared__ __align__(16) unsigned char gsm[];
    float2* E = reinterpret_cast<float2*>(gsm);
    // RECOMPUTE: the column transforms of P, in this CTA's global buffer (kept
    // in L2) so that shared memory holds one exchange buffer
    float2* E2 = RECOMPUTE ? prm.e2scr + (size_t)blockIdx.x * N * prm.es2 : nullptr;
    const long long units = (long long)prm.P * prm.K * prm.J;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        constexpr int L = Cta<N>::LINES;
        if constexpr (Cta<N>::WARP)
            unit_adjoint<N, L, RECOMPUTE>(unit_ptr<N>(prm, u), E, prm.es, E2, prm.es2, threadIdx.x, WarpBar{});
        else
            unit_adjoint<N, L, RECOMPUTE>(unit_ptr<N>(prm, u), E, prm.es, E2, prm.es2, threadIdx.x, CtaBar{});
    }
}

template <class Kern>
cudaError_t persistent_ctas(Kern kern, int threads, size_t smem, int sms, long long* ctas) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *ctas = (long long)sms * per_sm;
    return cudaSuccess;
}

template <class Kern>
cudaError_t launch_persistent(Kern kern, int threads, size_t smem, long long units, int sms, const GenericParams& prm,
                              cudaStream_t s, int max_ctas = 0) {
    long long ctas = 0;
    cudaError_t e = persistent_ctas(kern, threads, smem, sms, &ctas);
    if (e != cudaSuccess) return e;
    if (max_ctas > 0 && ctas > max_ctas) ctas = max_ctas;
    if (ctas > units) ctas = units;
    kern<<<(int)ctas, threads, smem, s>>>(prm);
    return cudaGetLastError();
}

}  // namespace

}  // namespace generic_detail

template <int N>
int generic_adjoint_ctas_n(int es, int sms) {
    using namespace generic_detail;
    const size_t smem = generic_smem(N, es, 0, true);
    long long c = 0;
    const cudaError_t e = persistent_ctas(generic_adjoint_kernel<N, true>, Cta<N>::THREADS, smem, sms, &c);
    return e == cudaSuccess ? (int)c : 0;
}

template <int N>
cudaError_t launch_generic_forward_n(const GenericParams& prm, int sms, cudaStream_t s) {
    using namespace generic_detail;
    const long long units = (long long)prm.P * prm.K * prm.J;
    const size_t smem = generic_smem(prm.N, prm.es, prm.es2, false);
    return launch_persistent(generic_forward_kernel<N>, Cta<N>::THREADS, smem, units, sms, prm, s);
}

template <int N>
cudaError_t launch_generic_adjoint_n(const GenericParams& prm, int sms, cudaStream_t s) {
    using namespace generic_detail;
    const long long units = (long long)prm.P * prm.K * prm.J;
    const bool rec = prm.pscr == nullptr;
    const size_t smem = generic_smem(prm.N, prm.es, prm.es2, rec);
    return rec ? launch_persistent(generic_adjoint_kernel<N, true>, Cta<N>::THREADS, smem, units, sms, prm, s,
                                   prm.e2_ctas)
               : launch_persistent(generic_adjoint_kernel<N, false>, Cta<N>::THREADS, smem, units, sms, prm, s);
}

}  // namespace mfbd_dev
