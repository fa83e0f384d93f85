// The Lofdahl-Scharmer Fourier filter of the objects (Sec. 4.1.1, Eq. 25).
//
// Per patch and object k, from the frames' data spectra D_kj and OTFs S_kj:
//   H_k(u) = 1 - nu sum_j w_j |S_kj(u)|^2 / |sum_j w_j D_kj(u) conj(S_kj(u))|^2,
// H < 0.2 -> 0 and H > 1 -> 1, a 3 x 3 median over the periodic frequency
// plane, and every nonzero value not 4-connected (periodically) to the zero
// frequency set to zero; the object is multiplied by H.
//
// Two kernels: a streaming pass, one thread per half-spectrum frequency,
// writes the thresholded H (to the filter output, or plan scratch); then one
// CTA per (patch, object), persistent, holds the full N x N plane in shared
// memory: the half spectrum kx <= N/2 as evaluated (columns 0 and N/2 from
// their own data), mirrored to -u for 0 < kx < N/2, where the sums are the
// conjugates of those at u. The values
// are >= 0, so a 3 x 3 median is nonzero exactly where at least 5 of the 9
// neighbours are: the median's nonzero pattern comes from bit rows of the
// thresholded plane by bit-sliced counting, and the median itself is
// evaluated only where the filter keeps it. The connectivity works on bit
// rows: the nonzero pixels of each row and of each column as N-bit rings; one thread per row fills the reached bits along its
// row's runs of nonzero pixels (a logarithmic fill with rotations, so runs
// wrap around), the rows are transposed to columns and filled the same way,
// and the two alternate until a column fill adds nothing (each round that
// continues adds a pixel: at most N^2 rounds, a handful in practice).
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

// An N-bit ring (N <= 128) in two words: bit b of the ring is bit b of lo
// (b < 64) or bit b - 64 of hi.
struct Ring {
    unsigned long long lo, hi;
};

__device__ __forceinline__ Ring ring_and(Ring a, Ring b) { return {a.lo & b.lo, a.hi & b.hi}; }
__device__ __forceinline__ Ring ring_or(Ring a, Ring b) { return {a.lo | b.lo, a.hi | b.hi}; }
__device__ __forceinline__ bool ring_eq(Ring a, Ring b) { return a.lo == b.lo && a.hi == b.hi; }

// Logical shifts of the 128-bit pair, 0 <= k < 128.
__device__ __forceinline__ Ring shl128(Ring a, int k) {
    if (k == 0) return a;
    if (k >= 64) return {0ull, a.lo << (k - 64)};
    return {a.lo << k, (a.hi << k) | (a.lo >> (64 - k))};
}
__device__ __forceinline__ Ring shr128(Ring a, int k) {
    if (k == 0) return a;
    if (k >= 64) return {a.hi >> (k - 64), 0ull};
    return {(a.lo >> k) | (a.hi << (64 - k)), a.hi >> k};
}

template <int N>
__device__ __forceinline__ Ring ring_full() {
    if constexpr (N <= 64) return {N == 64 ? ~0ull : (1ull << N) - 1ull, 0ull};
    else return {~0ull, N == 128 ? ~0ull : (1ull << (N - 64)) - 1ull};
}

// Rotations of the N-bit ring by 0 < k < N.
template <int N>
__device__ __forceinline__ Ring ring_up(Ring a, int k) {
    return ring_and(ring_or(shl128(a, k), shr128(a, N - k)), ring_full<N>());
}
template <int N>
__device__ __forceinline__ Ring ring_down(Ring a, int k) {
    return ring_and(ring_or(shr128(a, k), shl128(a, N - k)), ring_full<N>());
}

// The bits of m in runs (around the ring) that hold a bit of seeds & m:
// Kogge-Stone occluded fills up and down with steps 1, 2, 4, ... < N.
template <int N>
__device__ __forceinline__ Ring ring_fill(Ring m, Ring seeds) {
    Ring gu = ring_and(seeds, m), gd = gu, pu = m, pd = m;
#pragma unroll
    for (int k = 1; k < N; k <<= 1) {
        gu = ring_or(gu, ring_and(pu, ring_up<N>(gu, k)));
        pu = ring_and(pu, ring_up<N>(pu, k));
        gd = ring_or(gd, ring_and(pd, ring_down<N>(gd, k)));
        pd = ring_and(pd, ring_down<N>(pd, k));
    }
    return ring_or(gu, gd);
}

__device__ __forceinline__ Ring ring_xor(Ring a, Ring b) { return {a.lo ^ b.lo, a.hi ^ b.hi}; }

// Bit-sliced full adder: sum and carry of three rings.
__device__ __forceinline__ void full_add(Ring a, Ring b, Ring c, Ring& sum, Ring& carry) {
    const Ring ab = ring_xor(a, b);
    sum = ring_xor(ab, c);
    carry = ring_or(ring_and(a, b), ring_and(c, ab));
}

// Bits where at least 5 of the 3 x 3 neighbourhood (rows up, mid, down of
// the periodic plane, each with its left and right neighbours) are set.
template <int N>
__device__ __forceinline__ Ring at_least_5_of_9(Ring up, Ring mid, Ring down) {
    Ring s1, k1, s2, k2, s3, k3, s0, k4;
    full_add(ring_up<N>(up, 1), up, ring_down<N>(up, 1), s1, k1);
    full_add(ring_up<N>(mid, 1), mid, ring_down<N>(mid, 1), s2, k2);
    full_add(ring_up<N>(down, 1), down, ring_down<N>(down, 1), s3, k3);
    full_add(s1, s2, s3, s0, k4);           // count bit 0: s0; weight-2 carries k1..k4
    Ring t1, u1;
    full_add(k1, k2, k3, t1, u1);           // weight 2: t1, weight 4: u1
    const Ring t2 = ring_xor(t1, k4), u2 = ring_and(t1, k4);
    const Ring v = ring_xor(u1, u2), w8 = ring_and(u1, u2);
    // count = s0 + 2 t2 + 4 v + 8 w8 >= 5
    return ring_or(w8, ring_and(v, ring_or(t2, s0)));
}

__device__ __forceinline__ int ring_bit(const Ring& a, int b) {
    return (int)((b < 64 ? a.lo >> b : a.hi >> (b - 64)) & 1ull);
}

// out[i] = the ring whose bit j is bit i of in[j] (i, j < N): thread i reads
// every in[j] (one address for all threads: broadcast).
template <int N>
__device__ __forceinline__ Ring ring_transpose(const Ring* in, int i) {
    Ring acc{0ull, 0ull};
    const int sh = i < 64 ? i : i - 64;
    const bool upper = i >= 64;
#pragma unroll 8
    for (int j = 0; j < (N < 64 ? N : 64); ++j) {
        const Ring r = in[j];
        acc.lo |= (((upper ? r.hi : r.lo) >> sh) & 1ull) << j;
    }
    if constexpr (N > 64) {
#pragma unroll 8
        for (int j = 64; j < N; ++j) {
            const Ring r = in[j];
            acc.hi |= (((upper ? r.hi : r.lo) >> sh) & 1ull) << (j - 64);
        }
    }
    return acc;
}

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

// The median of the periodic 3 x 3 neighbourhood of (y, x).
template <int N>
__device__ __forceinline__ float median_at(const float* h, int y, int x) {
    const int ym = y == 0 ? N - 1 : y - 1, yp = y == N - 1 ? 0 : y + 1;
    const int xm = x == 0 ? N - 1 : x - 1, xp = x == N - 1 ? 0 : x + 1;
    float v[9] = {h[ym * N + xm], h[ym * N + x], h[ym * N + xp],
                  h[y * N + xm],  h[y * N + x],  h[y * N + xp],
                  h[yp * N + xm], h[yp * N + x], h[yp * N + xp]};
    return median9(v);
}

// Thresholded H on the half spectra of every (patch, object), one thread per
// frequency: a streaming pass over D and S.
template <int N>
__global__ void __launch_bounds__(kLsThreads) ls_raw_kernel(const LsFilterParams prm) {
    constexpr int NH = N / 2 + 1, HALF = N * NH;
    const int J = prm.J;
    const float nu = prm.noise_power;
    const long long total = (long long)prm.P * prm.K * HALF;
    for (long long e = (long long)blockIdx.x * kLsThreads + threadIdx.x; e < total;
         e += (long long)gridDim.x * kLsThreads) {
        const long long pk = e / HALF;
        const int f = (int)(e - pk * HALF);
        const int k = (int)(pk % prm.K), ky = f / NH, kx = f - ky * NH;
        const float* w = prm.weights + (size_t)k * J;
        const float2* dp = prm.spectra + (size_t)pk * J * N * prm.spec_ld + (size_t)ky * prm.spec_ld + kx;
        const float2* sp = prm.otf + (size_t)pk * J * HALF + f;
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
        const float h = __fsub_rn(1.0f, __fdiv_rn(__fmul_rn(nu, q), n2));
        prm.raw[e] = h >= 0.2f ? fminf(h, 1.0f) : 0.0f;  // NaN -> 0
    }
}

template <int N>
__global__ void __launch_bounds__(kLsThreads) ls_filter_kernel(const LsFilterParams prm) {
    constexpr int NH = N / 2 + 1, HALF = N * NH, NN = N * N;
    extern __shared__ __align__(16) unsigned char lsm[];
    Ring* raw = reinterpret_cast<Ring*>(lsm);   // [N] nonzero thresholded pixels of row y
    Ring* mrow = raw + N;                       // [N] nonzero medians of row y
    Ring* mcol = mrow + N;                      // [N] nonzero medians of column x
    Ring* rrow = mcol + N;                      // [N] reached pixels of row y
    Ring* rcol = rrow + N;                      // [N] reached pixels of column x
    float* hraw = reinterpret_cast<float*>(rcol + N);
    const int tid = threadIdx.x;
    const long long planes = (long long)prm.P * prm.K;
    for (long long pk = blockIdx.x; pk < planes; pk += gridDim.x) {
        // the thresholded half plane, mirrored to -u
        const float* rp = prm.raw + (size_t)pk * HALF;
        for (int f = tid; f < HALF; f += kLsThreads) {
            const int ky = f / NH, kx = f - ky * NH;
            const float h = rp[f];
            hraw[ky * N + kx] = h;
            if (kx > 0 && kx < N / 2) hraw[(ky == 0 ? 0 : N - ky) * N + (N - kx)] = h;
        }
        __syncthreads();
        // nonzero rows by warp ballots (a warp per row, 32 columns per ballot)
        for (int y = tid >> 5; y < N; y += kLsThreads / 32) {
            Ring m{0ull, 0ull};
            const int lane = tid & 31;
#pragma unroll
            for (int c = 0; c < (N + 31) / 32; ++c) {
                const int x = c * 32 + lane;
                const unsigned b = __ballot_sync(0xffffffffu, x < N && hraw[y * N + (x < N ? x : 0)] > 0.f);
                if (c < 2) m.lo |= (unsigned long long)b << (32 * c);
                else m.hi |= (unsigned long long)b << (32 * (c - 2));
            }
            if (lane == 0) raw[y] = m;
        }
        __syncthreads();
        // nonzero medians; the seed is the zero frequency
        if (tid < N) {
            const int y = tid;
            const Ring m = at_least_5_of_9<N>(raw[y == 0 ? N - 1 : y - 1], raw[y], raw[y == N - 1 ? 0 : y + 1]);
            mrow[y] = m;
            rrow[y] = Ring{y == 0 ? (m.lo & 1ull) : 0ull, 0ull};
        }
        __syncthreads();
        if (tid < N) mcol[tid] = ring_transpose<N>(mrow, tid);
        __syncthreads();
        // the component of the zero frequency: row fills and column fills in turn
        for (int round = 0; round < NN; ++round) {
            if (tid < N) rrow[tid] = ring_fill<N>(mrow[tid], rrow[tid]);
            __syncthreads();
            int changed = 0;
            if (tid < N) {
                const Ring c = ring_transpose<N>(rrow, tid);
                const Ring f = ring_fill<N>(mcol[tid], c);
                changed = !ring_eq(f, c);
                rcol[tid] = f;
            }
            if (!__syncthreads_or(changed)) break;
            if (tid < N) rrow[tid] = ring_transpose<N>(rcol, tid);
            __syncthreads();
        }
        // H out; the object multiplied in place
        if (prm.filter) {
            float* fo = prm.filter + (size_t)pk * HALF;
            for (int f = tid; f < HALF; f += kLsThreads) {
                const int ky = f / NH, kx = f - ky * NH;
                fo[f] = ring_bit(rcol[kx], ky) ? median_at<N>(hraw, ky, kx) : 0.f;
            }
        }
        if (prm.object) {
            float2* ob = prm.object + (size_t)pk * N * prm.obj_ld;
            const int cols = prm.obj_ld;  // N / 2 + 1 or N
            for (int e = tid; e < N * cols; e += kLsThreads) {
                const int y = e / cols, x = e - y * cols;
                const float h = ring_bit(rcol[x], y) ? median_at<N>(hraw, y, x) : 0.f;
                const float2 o = ob[e];
                ob[e] = make_float2(__fmul_rn(o.x, h), __fmul_rn(o.y, h));
            }
        }
        __syncthreads();
    }
}

template <int N>
cudaError_t launch_ls(const LsFilterParams& prm, int sms, cudaStream_t s) {
    {
        const long long total = (long long)prm.P * prm.K * N * (N / 2 + 1);
        long long blocks = (total + kLsThreads - 1) / kLsThreads;
        if (blocks > 16ll * sms) blocks = 16ll * sms;
        ls_raw_kernel<N><<<(int)blocks, kLsThreads, 0, s>>>(prm);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
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

size_t ls_filter_smem(int N) { return (size_t)N * (5 * sizeof(Ring) + N * sizeof(float)); }

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
