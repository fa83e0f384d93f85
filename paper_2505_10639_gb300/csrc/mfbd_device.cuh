// Device helpers shared by the pass and reduction kernels of every patch size.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace mfbd_dev {

// exp(i phi): reduction to [-pi, pi] by a two-constant Cody-Waite step
// (2 pi = 6.2831854820251465 - 1.7484556e-7), then the SFU sine/cosine.
__device__ __forceinline__ float2 expi(float ph) {
    const float n = rintf(ph * 0.159154943091895336f);
    float r = fmaf(n, -6.28318548202514648f, ph);
    r = fmaf(n, 1.74845553e-7f, r);
    float s, c;
    __sincosf(r, &s, &c);
    return make_float2(c, s);
}

// Where the fit leaves little residual energy (sum_j w |r_j|^2 below kCancel
// of sum_j w |D_j|^2) the FP32 residual cancels badly: such a frequency is
// redone in FP64 (fp64_frequency).
constexpr float kCancel = 1e-3f;

struct KahanSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// One frequency in FP64: N, Q, O = N / Q, the residuals r_j = D_j - O H_j,
// the loss term t = sum_j w |r_j|^2 + gamma |O|^2 and the adjoint seeds
// -w conj(O) r_j (0 when `seed` is false) written over H_j. dp / hp point at
// frame 0; frames are dstride / hstride complex elements apart.
__device__ __forceinline__ void fp64_frequency(int J, const float2* dp, size_t dstride, float2* hp, size_t hstride,
                                               const float* w, double gamma, bool seed, float& t, float2& o) {
    double nx = 0.0, ny = 0.0, qd = gamma;
    for (int j = 0; j < J; ++j) {
        const float2 d = dp[(size_t)j * dstride];
        const float2 h = hp[(size_t)j * hstride];
        const double wj = w[j];
        nx += wj * ((double)d.x * h.x + (double)d.y * h.y);
        ny += wj * ((double)d.y * h.x - (double)d.x * h.y);
        qd += wj * ((double)h.x * h.x + (double)h.y * h.y);
    }
    const double ox = nx / qd, oy = ny / qd;
    double tsum = 0.0;
    for (int j = 0; j < J; ++j) {
        const float2 d = dp[(size_t)j * dstride];
        const float2 h = hp[(size_t)j * hstride];
        const double wj = w[j];
        const double rx = (double)d.x - (ox * h.x - oy * h.y);
        const double ry = (double)d.y - (ox * h.y + oy * h.x);
        tsum += wj * (rx * rx + ry * ry);
        hp[(size_t)j * hstride] = seed ? make_float2((float)(-wj * (ox * rx + oy * ry)), (float)(-wj * (ox * ry - oy * rx)))
                                       : make_float2(0.f, 0.f);
    }
    t = (float)(tsum + gamma * (ox * ox + oy * oy));
    o = make_float2((float)ox, (float)oy);
}

// One frequency of the object-inferring loss (the object o given): the
// residuals r_j = D_j - o H_j, the loss term t = sum_j w |r_j|^2 + gamma |o|^2
// (returned), the adjoint seeds -w conj(o) r_j (0 when `seed` is false)
// written over H_j, and g = gamma o - sum_j w conj(H_j) r_j, the derivative
// of the loss with respect to conj(O) at this frequency. FP32; redone in FP64
// where the residual energy is below kCancel of the data's.
__device__ __forceinline__ float explicit_frequency(int J, const float2* dp, size_t dstride, float2* hp,
                                                    size_t hstride, const float* w, double gamma, bool seed,
                                                    float2 o, float2& g) {
    float tsum = 0.f, e = 0.f;
#pragma unroll 4
    for (int j = 0; j < J; ++j) {
        const float2 d = dp[(size_t)j * dstride];
        const float2 h = hp[(size_t)j * hstride];
        const float wj = w[j];
        const float rx = d.x - (o.x * h.x - o.y * h.y), ry = d.y - (o.x * h.y + o.y * h.x);
        tsum += wj * (rx * rx + ry * ry);
        e += wj * (d.x * d.x + d.y * d.y);
    }
    if (tsum >= kCancel * e) {
        const float gam = (float)gamma;
        float gx = 0.f, gy = 0.f;
#pragma unroll 4
        for (int j = 0; j < J; ++j) {
            const float2 d = dp[(size_t)j * dstride];
            const float2 h = hp[(size_t)j * hstride];
            const float wj = w[j];
            const float rx = d.x - (o.x * h.x - o.y * h.y), ry = d.y - (o.x * h.y + o.y * h.x);
            gx += wj * (h.x * rx + h.y * ry);
            gy += wj * (h.x * ry - h.y * rx);
            hp[(size_t)j * hstride] = seed ? make_float2(-wj * (o.x * rx + o.y * ry), -wj * (o.x * ry - o.y * rx))
                                           : make_float2(0.f, 0.f);
        }
        g = make_float2(gam * o.x - gx, gam * o.y - gy);
        return tsum + gam * (o.x * o.x + o.y * o.y);
    }
    const double ox = o.x, oy = o.y;
    double ts = 0.0, gx = 0.0, gy = 0.0;
    for (int j = 0; j < J; ++j) {
        const float2 d = dp[(size_t)j * dstride];
        const float2 h = hp[(size_t)j * hstride];
        const double wj = w[j];
        const double rx = (double)d.x - (ox * h.x - oy * h.y), ry = (double)d.y - (ox * h.y + oy * h.x);
        ts += wj * (rx * rx + ry * ry);
        gx += wj * ((double)h.x * rx + (double)h.y * ry);
        gy += wj * ((double)h.x * ry - (double)h.y * rx);
        hp[(size_t)j * hstride] = seed ? make_float2((float)(-wj * (ox * rx + oy * ry)), (float)(-wj * (ox * ry - oy * rx)))
                                       : make_float2(0.f, 0.f);
    }
    g = make_float2((float)(gamma * ox - gx), (float)(gamma * oy - gy));
    return (float)(ts + gamma * (ox * ox + oy * oy));
}

}  // namespace mfbd_dev
