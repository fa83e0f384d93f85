// Frame reduction of the CTA-per-unit kernels (any patch size) and the
// size dispatch of their pass kernels, which are instantiated per patch
// size in generic_n48.cu ... generic_n128.cu (generic_kernels.cuh).
#include <algorithm>

#include "mfbd_internal.h"
#include "unit_passes.cuh"

namespace mfbd_dev {

namespace {

using namespace unitpass;

// One CTA per patch (persistent over patches), one warp per object; the
// patch loss sums the objects in order.
__global__ void __launch_bounds__(32 * kMaxObjects) generic_reduce_kernel(const GenericParams prm) {
    __shared__ double sobj[kMaxObjects];
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int N = prm.N, half = N * (N / 2 + 1), J = prm.J;
    const size_t dstride = (size_t)N * prm.spec_ld;
    const int S = (prm.rsplit > 1 && prm.lpart) ? prm.rsplit : 1;
    const long long work = (long long)prm.P * S;
    for (long long u = blockIdx.x; u < work; u += gridDim.x) {
        const int p = (int)(u / S), sp = (int)(u - (long long)p * S);
        const size_t unit0 = ((size_t)p * prm.K + k) * J;
        RedPtr r;
        r.N = N;
        r.J = J;
        r.spec_ld = prm.spec_ld;
        r.gamma = prm.gamma;
        r.d = prm.spectra + unit0 * dstride;
        r.h = prm.gscr + unit0 * half;
        r.w = prm.weights + (size_t)k * J;
        r.supp = prm.obj[k].supp;
        r.sw = prm.sw;
        r.obj = prm.object ? prm.object + ((size_t)p * prm.K + k) * dstride : nullptr;
        r.oin = prm.oin ? prm.oin + ((size_t)p * prm.K + k) * dstride : nullptr;
        r.gobj = prm.gobj ? prm.gobj + ((size_t)p * prm.K + k) * dstride : nullptr;
        const double v = reduce_warp(r, lane, 32 * sp, 32 * S);
        if (lane == 0) sobj[k] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int i = 0; i < prm.K; ++i) tot += sobj[i];
            if (S == 1)
                prm.loss[p] = tot;
            else
                prm.lpart[u] = tot;
        }
        __syncthreads();
    }
}

__global__ void loss_combine_kernel(const double* __restrict__ lpart, int S, double* __restrict__ loss, int P) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    double tot = 0.0;
    for (int i = 0; i < S; ++i) tot += lpart[(size_t)p * S + i];
    loss[p] = tot;
}

}  // namespace

size_t generic_smem(int N, int es, int es2, bool recompute) {
    (void)es2;
    (void)recompute;  // the recompute buffer is in global memory (e2scr)
    return (size_t)N * es * sizeof(float2);
}

int generic_adjoint_ctas(int N, int es, int sms) {
    switch (N) {
        case 48: return generic_adjoint_ctas_n<48>(es, sms);
        case 64: return generic_adjoint_ctas_n<64>(es, sms);
        case 96: return generic_adjoint_ctas_n<96>(es, sms);
        case 128: return generic_adjoint_ctas_n<128>(es, sms);
        default: return 0;
    }
}

cudaError_t launch_generic_forward(const GenericParams& prm, int sms, cudaStream_t s) {
    const long long units = (long long)prm.P * prm.K * prm.J;
    if (units == 0) return cudaSuccess;
    switch (prm.N) {
        case 48: return launch_generic_forward_n<48>(prm, sms, s);
        case 64: return launch_generic_forward_n<64>(prm, sms, s);
        case 96: return launch_generic_forward_n<96>(prm, sms, s);
        case 128: return launch_generic_forward_n<128>(prm, sms, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_generic_adjoint(const GenericParams& prm, int sms, cudaStream_t s) {
    const long long units = (long long)prm.P * prm.K * prm.J;
    if (units == 0) return cudaSuccess;
    const bool rec = prm.pscr == nullptr;
    if (rec && (!prm.e2scr || prm.e2_ctas < 1)) return cudaErrorInvalidValue;
    switch (prm.N) {
        case 48: return launch_generic_adjoint_n<48>(prm, sms, s);
        case 64: return launch_generic_adjoint_n<64>(prm, sms, s);
        case 96: return launch_generic_adjoint_n<96>(prm, sms, s);
        case 128: return launch_generic_adjoint_n<128>(prm, sms, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_generic_reduction(const GenericParams& prm, int sms, cudaStream_t s) {
    if (prm.P == 0) return cudaSuccess;
    const int threads = 32 * prm.K;
    const int S = (prm.rsplit > 1 && prm.lpart) ? prm.rsplit : 1;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, generic_reduce_kernel, threads, 0);
    if (e != cudaSuccess) return e;
    long long ctas = (long long)sms * (per_sm > 0 ? per_sm : 1);
    if (ctas > (long long)prm.P * S) ctas = (long long)prm.P * S;
    generic_reduce_kernel<<<(int)ctas, threads, 0, s>>>(prm);
    if ((e = cudaGetLastError()) != cudaSuccess || S == 1) return e;
    return launch_loss_combine(prm.lpart, S, prm.loss, prm.P, s);
}

int reduction_split(int P, int K, int N, int sms) {
    const long long warps = (long long)P * K, want = 8LL * sms;
    if (warps <= 0 || warps >= want) return 1;
    const long long smax = std::max(1, N * (N / 2 + 1) / 128);
    return (int)std::min((want + warps - 1) / warps, smax);
}

cudaError_t launch_loss_combine(const double* lpart, int S, double* loss, int P, cudaStream_t s) {
    if (P == 0) return cudaSuccess;
    loss_combine_kernel<<<(P + 127) / 128, 128, 0, s>>>(lpart, S, loss, P);
    return cudaGetLastError();
}

}  // namespace mfbd_dev
