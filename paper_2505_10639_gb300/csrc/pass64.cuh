// Building blocks of the 64 px warp-per-frame pass kernels, shared by the
// three-kernel path (mfbd_kernels.cu) and the fused per-(patch, object)
// kernel (fused_kernels.cu): asynchronous copies, L2 prefetch, mask bits,
// and the quarter-line 64-point transform.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "fft_reg.cuh"
#include "mfbd_device.cuh"
#include "mfbd_internal.h"

namespace mfbd_dev {
namespace pass64 {

using fftreg::cadd;
using fftreg::cconj;
using fftreg::cmul;
using fftreg::cscale;
using fftreg::csub;

// Asynchronous global -> shared copy of 8 bytes (both addresses 8-byte
// aligned); complete for the issuing thread after cp_async_wait.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(__cvta_generic_to_global(gmem))
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// L2 prefetch of [ptr, ptr + bytes) (bulk prefetch needs 16-byte alignment
// and a multiple of 16 bytes; the range is widened to that).
__device__ __forceinline__ void prefetch_l2(const void* ptr, size_t bytes) {
    uintptr_t a = reinterpret_cast<uintptr_t>(ptr);
    uintptr_t b = (a + bytes + 15) & ~uintptr_t(15);
    a &= ~uintptr_t(15);
    if (b > a)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(
                         reinterpret_cast<const void*>(a))),
                     "r"((unsigned)(b - a))
                     : "memory");
}

// The same with an L2 access policy (createpolicy) for the prefetched lines.
__device__ __forceinline__ void prefetch_l2_hint(const void* ptr, size_t bytes, uint64_t pol) {
    uintptr_t a = reinterpret_cast<uintptr_t>(ptr);
    uintptr_t b = (a + bytes + 15) & ~uintptr_t(15);
    a &= ~uintptr_t(15);
    if (b > a)
        asm volatile("cp.async.bulk.prefetch.L2.global.L2::cache_hint [%0], %1, %2;" ::"l"(__cvta_generic_to_global(
                         reinterpret_cast<const void*>(a))),
                     "r"((unsigned)(b - a)), "l"(pol)
                     : "memory");
}

__device__ __forceinline__ bool bit(uint64_t w, int b) { return (w >> b) & 1ull; }

// ----------------------------------------------- quarter-line transforms

// Boxes 33..40 px wide leave 1..8 columns after the first round of 32. Those
// are transformed by 4 lanes each instead of one lane per column (in the
// PUPIL pass): lane
// l = lane & 3 holds a[n] = x[4 n + l] (n < 16), transforms it with a 16-point
// FFT, multiplies A_l[k] by exp(-2 pi i l k / 64), and the 4-point DFT over
// the lanes (two xor-shuffle stages) leaves X[k + 16 q] in lane l, with
// q = ((l & 1) << 1) | (l >> 1). Forward transform.
constexpr int kSplitMaxW = 40;

__device__ __forceinline__ int split_q(int l) { return ((l & 1) << 1) | (l >> 1); }

__device__ __forceinline__ void fft64_quarters(float2 (&a)[kN / 4], int l) {
    fftreg::fft4<kN / 4, -1>(a);
    fftreg::static_for<1, kN / 4>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        constexpr fftreg::SinCos w1 = fftreg::sincos_2pi(-k, kN), w2 = fftreg::sincos_2pi(-2 * k, kN),
                                 w3 = fftreg::sincos_2pi(-3 * k, kN);
        const float c = l == 0 ? 1.f : l == 1 ? (float)w1.c : l == 2 ? (float)w2.c : (float)w3.c;
        const float sn = l == 0 ? 0.f : l == 1 ? (float)w1.s : l == 2 ? (float)w2.s : (float)w3.s;
        a[k] = make_float2(a[k].x * c - a[k].y * sn, a[k].x * sn + a[k].y * c);
    });
    const float s2 = (l & 2) ? -1.f : 1.f, s1 = (l & 1) ? -1.f : 1.f;
    const bool rot = l == 3;
#pragma unroll
    for (int k = 0; k < kN / 4; ++k) {
        // lanes l and l ^ 2: l < 2 keeps the sum, l >= 2 the difference (times -i for l = 3)
        const float ox = __shfl_xor_sync(0xffffffffu, a[k].x, 2), oy = __shfl_xor_sync(0xffffffffu, a[k].y, 2);
        const float tx = fmaf(s2, a[k].x, ox), ty = fmaf(s2, a[k].y, oy);
        const float ux = rot ? ty : tx, uy = rot ? -tx : ty;
        // lanes l and l ^ 1: even l the sum, odd l the difference
        const float px = __shfl_xor_sync(0xffffffffu, ux, 1), py = __shfl_xor_sync(0xffffffffu, uy, 1);
        a[k] = make_float2(fmaf(s1, ux, px), fmaf(s1, uy, py));
    }
}

// --------------------------------------------------------- L2 cache hints

// Access policies for the L2: evict_first for data read once (the spectra),
// evict_last for scratch that is written and read back soon (the fused
// kernel's field slots), so that the stream of the one does not push the
// other out.
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ float2 ld_hint(const float2* a, uint64_t pol) {
    float2 v;
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
                 : "=f"(v.x), "=f"(v.y)
                 : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ float4 ld_hint(const float4* a, uint64_t pol) {
    float4 v;
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_hint(float* a, float v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_hint(float4* a, float4 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(a), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w), "l"(pol)
                 : "memory");
}

// ------------------------------------------------------- frame reduction

// Frame reduction of one (patch, object): per frequency u,
// N = sum_j w D conj(H), Q = sum_j w |H|^2 + gamma, O = N / Q, the loss term
// t(u) = sum_j w |D - O H|^2 + gamma |O|^2 and the adjoint seeds
// G_j = -w conj(O)(D - O H) (written over H_j). The residual is formed in
// FP32. Where the fit leaves little residual energy (sum_j w|r_j|^2 <
// kCancel sum_j w|D_j|^2, estimated from E - |N|^2/Q) it cancels badly in
// FP32 (for J = 1, r = D gamma / Q everywhere the OTF is large), so such a
// frequency is redone with N, Q, O and r_j in FP64 -- except DC, whose seed
// is zero and whose loss term is exact enough in FP32. Each thread sums its
// loss terms with Kahan compensation and returns them in FP64 (the callers
// combine the threads' sums in a fixed order). The thread takes the
// frequencies fstart, fstart + fstep, ... < N (N/2 + 1); hbase points at the
// pair's first frame of H (frames kHalf elements apart, global or shared
// memory).
// JM > 0: J <= JM, the J spectra and OTFs of a frequency are loaded once, all
// at once, into registers. JM == 0: any J, streamed from memory twice.
// MODE: 0 takes the object-inferring branch when prm.oin is set, 1 compiles
// the Wiener loss only, 2 the object-inferring loss only. STREAM: the
// spectra are read with an L2 evict-first hint (JM > 0).
template <int JM, int MODE = 0, bool STREAM = false>
__device__ __forceinline__ double reduce_frequencies(const FusedParams& prm, int p, int k, float2* hbase,
                                                     int fstart, int fstep) {
    const int J = prm.J;
    const size_t unit0 = ((size_t)p * prm.K + k) * J;
    const size_t dstride = (size_t)kN * prm.spec_ld;
    const float2* dbase = prm.spectra + unit0 * dstride;
    const float* w = prm.weights + (size_t)k * J;
    const uint64_t* supp = prm.obj[k].supp;
    const float gam = (float)prm.gamma;
    float wv[JM > 0 ? JM : 1];
    if constexpr (JM > 0) {
#pragma unroll
        for (int j = 0; j < JM; ++j) wv[j] = (j < J) ? w[j] : 0.f;
    }
    const uint64_t pol = STREAM ? l2_evict_first() : 0;
    KahanSum acc;
    for (int f = fstart; f < kHalf; f += fstep) {
        const int ky = f / kNH, kx = f - ky * kNH;
        const size_t doff = (size_t)ky * prm.spec_ld + kx;
        const float2* dp = dbase + doff;
        float2* hp = hbase + f;
        const bool seed = (f != 0) && bit(supp[ky], kx);
        if (MODE == 2 || (MODE == 0 && prm.oin)) {  // object-inferring loss: the object is given
            const size_t ooff = ((size_t)p * prm.K + k) * dstride;
            float2 g;
            const float t = explicit_frequency(J, dp, dstride, hp, kHalf, w, prm.gamma, seed, prm.oin[ooff + doff], g);
            acc.add((kx == 0 || kx == kN / 2) ? t : 2.0f * t);
            if (prm.gobj) {
                prm.gobj[ooff + doff] = g;
                if (prm.spec_ld == kN && kx > 0 && kx < kN / 2)
                    prm.gobj[ooff + (size_t)((kN - ky) % kN) * kN + (kN - kx)] = cconj(g);
            }
            continue;
        }
        float2 num = make_float2(0.f, 0.f), o;
        float e = 0.f, q = 0.f, t;
        if constexpr (JM > 0) {
            float2 d[JM], h[JM];
#pragma unroll
            for (int j = 0; j < JM; ++j) {
                if constexpr (STREAM)
                    d[j] = (j < J) ? ld_hint(dp + (size_t)j * dstride, pol) : make_float2(0.f, 0.f);
                else
                    d[j] = (j < J) ? dp[(size_t)j * dstride] : make_float2(0.f, 0.f);
                h[j] = (j < J) ? hp[(size_t)j * kHalf] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int j = 0; j < JM; ++j) {
                num.x += wv[j] * (d[j].x * h[j].x + d[j].y * h[j].y);
                num.y += wv[j] * (d[j].y * h[j].x - d[j].x * h[j].y);
                e += wv[j] * (d[j].x * d[j].x + d[j].y * d[j].y);
                q += wv[j] * (h[j].x * h[j].x + h[j].y * h[j].y);
            }
            q += gam;
            const float invq = 1.0f / q;
            o = cscale(num, invq);
            const float t_est = e - (num.x * num.x + num.y * num.y) * invq;
            if (f != 0 && t_est < kCancel * e) {
                fp64_frequency(J, dp, dstride, hp, kHalf, w, prm.gamma, seed, t, o);
            } else {
                float tsum = 0.f;
#pragma unroll
                for (int j = 0; j < JM; ++j) {
                    const float2 r = csub(d[j], cmul(o, h[j]));
                    tsum += wv[j] * (r.x * r.x + r.y * r.y);
                    if (j < J)
                        hp[(size_t)j * kHalf] = seed ? cscale(cmul(cconj(o), r), -wv[j]) : make_float2(0.f, 0.f);
                }
                t = tsum + gam * (o.x * o.x + o.y * o.y);
            }
        } else {
#pragma unroll 4
            for (int j = 0; j < J; ++j) {
                const float2 d = dp[(size_t)j * dstride];
                const float2 h = hp[(size_t)j * kHalf];
                const float wj = w[j];
                num.x += wj * (d.x * h.x + d.y * h.y);
                num.y += wj * (d.y * h.x - d.x * h.y);
                e += wj * (d.x * d.x + d.y * d.y);
                q += wj * (h.x * h.x + h.y * h.y);
            }
            q += gam;
            const float invq = 1.0f / q;
            o = cscale(num, invq);
            const float t_est = e - (num.x * num.x + num.y * num.y) * invq;
            if (f != 0 && t_est < kCancel * e) {
                fp64_frequency(J, dp, dstride, hp, kHalf, w, prm.gamma, seed, t, o);
            } else {
                float tsum = 0.f;
#pragma unroll 4
                for (int j = 0; j < J; ++j) {
                    const float2 d = dp[(size_t)j * dstride];
                    const float2 h = hp[(size_t)j * kHalf];
                    const float wj = w[j];
                    const float2 r = csub(d, cmul(o, h));
                    tsum += wj * (r.x * r.x + r.y * r.y);
                    hp[(size_t)j * kHalf] = seed ? cscale(cmul(cconj(o), r), -wj) : make_float2(0.f, 0.f);
                }
                t = tsum + gam * (o.x * o.x + o.y * o.y);
            }
        }
        acc.add((kx == 0 || kx == kN / 2) ? t : 2.0f * t);
        if (prm.object) {
            float2* ob = prm.object + ((size_t)p * prm.K + k) * dstride;
            ob[doff] = o;
            if (prm.spec_ld == kN && kx > 0 && kx < kN / 2)
                ob[(size_t)((kN - ky) % kN) * kN + (kN - kx)] = cconj(o);
        }
    }
    return (double)acc.s - (double)acc.c;
}

}  // namespace pass64
}  // namespace mfbd_dev
