// Pass and reduction kernels of one problem for the patch sizes other than
// 64 (48, 96, 128), and for 64 on request: one CTA per unit (patch, object,
// frame), persistent over the units; for N <= 64 the CTA is one warp. The passes themselves (Sec. 3.1,
// Eqs. 20-22 and their adjoint) are in unit_passes.cuh.
#include <algorithm>

#include "mfbd_internal.h"
#include "unit_passes.cuh"

namespace mfbd_dev {

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

size_t generic_smem(int N, int es, int es2, bool recompute) {
    (void)es2;
    (void)recompute;  // the recompute buffer is in global memory (e2scr)
    return (size_t)N * es * sizeof(float2);
}

int generic_adjoint_ctas(int N, int es, int sms) {
    const size_t smem = generic_smem(N, es, 0, true);
    long long c = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (N) {
        case 48: e = persistent_ctas(generic_adjoint_kernel<48, true>, Cta<48>::THREADS, smem, sms, &c); break;
        case 64: e = persistent_ctas(generic_adjoint_kernel<64, true>, Cta<64>::THREADS, smem, sms, &c); break;
        case 96: e = persistent_ctas(generic_adjoint_kernel<96, true>, Cta<96>::THREADS, smem, sms, &c); break;
        case 128: e = persistent_ctas(generic_adjoint_kernel<128, true>, Cta<128>::THREADS, smem, sms, &c); break;
        default: break;
    }
    return e == cudaSuccess ? (int)c : 0;
}

cudaError_t launch_generic_forward(const GenericParams& prm, int sms, cudaStream_t s) {
    const long long units = (long long)prm.P * prm.K * prm.J;
    if (units == 0) return cudaSuccess;
    const size_t smem = generic_smem(prm.N, prm.es, prm.es2, false);
    switch (prm.N) {
        case 48: return launch_persistent(generic_forward_kernel<48>, Cta<48>::THREADS, smem, units, sms, prm, s);
        case 64: return launch_persistent(generic_forward_kernel<64>, Cta<64>::THREADS, smem, units, sms, prm, s);
        case 96: return launch_persistent(generic_forward_kernel<96>, Cta<96>::THREADS, smem, units, sms, prm, s);
        case 128: return launch_persistent(generic_forward_kernel<128>, Cta<128>::THREADS, smem, units, sms, prm, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_generic_adjoint(const GenericParams& prm, int sms, cudaStream_t s) {
    const long long units = (long long)prm.P * prm.K * prm.J;
    if (units == 0) return cudaSuccess;
    const bool rec = prm.pscr == nullptr;
    if (rec && (!prm.e2scr || prm.e2_ctas < 1)) return cudaErrorInvalidValue;
    const size_t smem = generic_smem(prm.N, prm.es, prm.es2, rec);
#define MFBD_ADJ(NN)                                                                                            \
    case NN:                                                                                                    \
        return rec ? launch_persistent(generic_adjoint_kernel<NN, true>, Cta<NN>::THREADS, smem, units, sms, prm, s, \
                                       prm.e2_ctas)                                                              \
                   : launch_persistent(generic_adjoint_kernel<NN, false>, Cta<NN>::THREADS, smem, units, sms, prm, s);
    switch (prm.N) {
        MFBD_ADJ(48)
        MFBD_ADJ(64)
        MFBD_ADJ(96)
        MFBD_ADJ(128)
        default: return cudaErrorInvalidValue;
    }
#undef MFBD_ADJ
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
