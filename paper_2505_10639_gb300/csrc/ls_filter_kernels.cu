// The Lofdahl-Scharmer Fourier filter of the objects (Sec. 4.1.1, Eq. 25).
//
// Per patch and object k, from the frames' data spectra D_kj and OTFs S_kj:
//   H_k(u) = 1 - nu sum_j w_j |S_kj(u)|^2 / |sum_j w_j D_kj(u) conj(S_kj(u))|^2,
// H < 0.2 -> 0 and H > 1 -> 1, a 3 x 3 median over the periodic frequency
// plane, and every nonzero value not 4-connected (periodically) to the zero
// frequency set to zero; the object is multiplied by H.
//
// One CTA per (patch, object), persistent. The full N x N plane of H lives in
// shared memory: the half spectrum kx <= N/2 is evaluated from the inputs
// (columns 0 and N/2 from their own data) and mirrored to -u for
// 0 < kx < N/2, where the sums are the conjugates of those at u. The
// connectivity is a fixed-point sweep: a nonzero pixel with a reached
// 4-neighbour becomes reached, until a sweep changes nothing (at most one
// sweep per pixel of the plane; each sweep that continues adds one).
//
// Arithmetic: FP32 in a fixed order with every product and sum rounded on its
// own (__fmul_rn / __fadd_rn / __fsub_rn / __fdiv_rn, no fused multiply-add),
// so that the threshold decisions can be reproduced exactly:
//   t_re = d_re s_re + d_im s_im,  t_im = d_im s_re - d_re s_im,
//   n += w t,  q += w (s_re s_re + s_im s_im)   (frames in order),
//   H = 1 - (nu q) / (n_re n_re + n_im n_im).
// A zero denominator gives -inf or NaN, both 0 after the threshold.
#include "mfbd_internal.h"

namespace mfbd_dev {

namespace {

constexpr int kLsThreads = 256;

// 5th smallest of 9 (the median): selection of the five smallest values.
__device__ __forceinline__ float median9(float v[9]) {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
#pragma unroll
        for (int j = i + 1; j < 9; ++j) {
            const float a = v[i], b = v[j];
            v[i] = fminf(a, b);
            v[j] = fmaxf(a, b);
        }
    }
    return v[4];
}

template <int N>
__global__ void __launch_bounds__(kLsThreads) ls_filter_kernel(const LsFilterParams prm) {
    constexpr int NH = N / 2 + 1, HALF = N * NH, NN = N * N;
    extern __shared__ __align__(16) unsigned char lsm[];
    float* hraw = reinterpret_cast<float*>(lsm);
    float* hmed = hraw + NN;
    volatile unsigned char* reach = reinterpret_cast<unsigned char*>(hmed + NN);
    const int tid = threadIdx.x, J = prm.J;
    const float nu = prm.noise_power;
    const long long planes = (long long)prm.P * prm.K;
    for (long long pk = blockIdx.x; pk < planes; pk += gridDim.x) {
        const int k = (int)(pk % prm.K);
        const float* w = prm.weights + (size_t)k * J;
        const float2* dbase = prm.spectra + (size_t)pk * J * N * prm.spec_ld;
        const float2* sbase = prm.otf + (size_t)pk * J * HALF;
        // H on the half spectrum, thresholded, mirrored
        for (int f = tid; f < HALF; f += kLsThreads) {
            const int ky = f / NH, kx = f - ky * NH;
            const float2* dp = dbase + (size_t)ky * prm.spec_ld + kx;
            const float2* sp = sbase + f;
            float nr = 0.f, ni = 0.f, q = 0.f;
#pragma unroll 4
            for (int j = 0; j < J; ++j) {
                const float2 d = dp[(size_t)j * N * prm.spec_ld];
                const float2 s = sp[(size_t)j * HALF];
                const float wj = w[j];
                const float tr = __fadd_rn(__fmul_rn(d.x, s.x), __fmul_rn(d.y, s.y));
                const float ti = __fsub_rn(__fmul_rn(d.y, s.x), __fmul_rn(d.x, s.y));
                nr = __fadd_rn(nr, __fmul_rn(wj, tr));
                ni = __fadd_rn(ni, __fmul_rn(wj, ti));
                q = __fadd_rn(q, __fmul_rn(wj, __fadd_rn(__fmul_rn(s.x, s.x), __fmul_rn(s.y, s.y))));
            }
            const float n2 = __fadd_rn(__fmul_rn(nr, nr), __fmul_rn(ni, ni));
            float h = __fsub_rn(1.0f, __fdiv_rn(__fmul_rn(nu, q), n2));
            h = h >= 0.2f ? fminf(h, 1.0f) : 0.0f;  // NaN -> 0
            hraw[ky * N + kx] = h;
            if (kx > 0 && kx < N / 2) hraw[(ky == 0 ? 0 : N - ky) * N + (N - kx)] = h;
        }
        __syncthreads();
        // 3 x 3 median, periodic
        for (int i = tid; i < NN; i += kLsThreads) {
            const int y = i / N, x = i - y * N;
            const int ym = y == 0 ? N - 1 : y - 1, yp = y == N - 1 ? 0 : y + 1;
            const int xm = x == 0 ? N - 1 : x - 1, xp = x == N - 1 ? 0 : x + 1;
            float v[9] = {hraw[ym * N + xm], hraw[ym * N + x], hraw[ym * N + xp],
                          hraw[y * N + xm],  hraw[y * N + x],  hraw[y * N + xp],
                          hraw[yp * N + xm], hraw[yp * N + x], hraw[yp * N + xp]};
            hmed[i] = median9(v);
            reach[i] = 0;
        }
        __syncthreads();
        if (tid == 0) reach[0] = hmed[0] > 0.f ? 1 : 0;
        __syncthreads();
        // the component of the zero frequency
        for (int sweep = 0; sweep < NN; ++sweep) {
            int changed = 0;
            for (int i = tid; i < NN; i += kLsThreads) {
                if (reach[i] || !(hmed[i] > 0.f)) continue;
                const int y = i / N, x = i - y * N;
                const int ym = y == 0 ? N - 1 : y - 1, yp = y == N - 1 ? 0 : y + 1;
                const int xm = x == 0 ? N - 1 : x - 1, xp = x == N - 1 ? 0 : x + 1;
                if (reach[ym * N + x] | reach[yp * N + x] | reach[y * N + xm] | reach[y * N + xp]) {
                    reach[i] = 1;
                    changed = 1;
                }
            }
            if (!__syncthreads_or(changed)) break;
        }
        // H out; the object multiplied in place
        if (prm.filter) {
            float* fo = prm.filter + (size_t)pk * HALF;
            for (int f = tid; f < HALF; f += kLsThreads) {
                const int ky = f / NH, kx = f - ky * NH, i = ky * N + kx;
                fo[f] = reach[i] ? hmed[i] : 0.f;
            }
        }
        if (prm.object) {
            float2* ob = prm.object + (size_t)pk * N * prm.obj_ld;
            const int cols = prm.obj_ld;  // N / 2 + 1 or N
            for (int e = tid; e < N * cols; e += kLsThreads) {
                const int y = e / cols, x = e - y * cols, i = y * N + x;
                const float h = reach[i] ? hmed[i] : 0.f;
                const float2 o = ob[e];
                ob[e] = make_float2(__fmul_rn(o.x, h), __fmul_rn(o.y, h));
            }
        }
        __syncthreads();
    }
}

template <int N>
cudaError_t launch_ls(const LsFilterParams& prm, int sms, cudaStream_t s) {
    const size_t smem = ls_filter_smem(N);
    auto* kern = ls_filter_kernel<N>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLsThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long ctas = (long long)sms * per_sm;
    const long long planes = (long long)prm.P * prm.K;
    if (ctas > planes) ctas = planes;
    kern<<<(int)ctas, kLsThreads, smem, s>>>(prm);
    return cudaGetLastError();
}

}  // namespace

size_t ls_filter_smem(int N) { return (size_t)N * N * (2 * sizeof(float) + 1); }

cudaError_t launch_ls_filter(const LsFilterParams& prm, int sms, cudaStream_t s) {
    if ((long long)prm.P * prm.K == 0) return cudaSuccess;
    switch (prm.N) {
        case 48: return launch_ls<48>(prm, sms, s);
        case 64: return launch_ls<64>(prm, sms, s);
        case 96: return launch_ls<96>(prm, sms, s);
        case 128: return launch_ls<128>(prm, sms, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mfbd_dev
