// Register-resident FFTs with compile-time twiddles.
//
// One thread owns one whole line (N complex values in registers) and
// transforms it with a fully unrolled radix-2 decimation-in-time network.
// Every index and every twiddle factor is a compile-time constant, so the
// twiddles become instruction immediates and the trivial ones (1, -1, +-i)
// cost nothing. Transform convention (unnormalised):
//   DIR = -1:  X[k] = sum_n x[n] exp(-2 pi i n k / N)   (forward)
//   DIR = +1:  x[n] = sum_k X[k] exp(+2 pi i n k / N)   (adjoint, F^H)
// The functions are __host__ __device__ so the same arithmetic can be
// exercised on the CPU.
#pragma once

#include <cuda_runtime.h>

#define MFBD_HD __host__ __device__ __forceinline__

namespace fftreg {

template <int I>
struct IC {
    static constexpr int value = I;
};

template <int B, int E, class F>
MFBD_HD void static_for(F&& f) {
    if constexpr (B < E) {
        f(IC<B>{});
        static_for<B + 1, E>(f);
    }
}

// ---- compile-time sin/cos of 2 pi k / n (Taylor series after an exact
// integer reduction to the first octant) ----
constexpr double kPi = 3.14159265358979323846264338327950288;

constexpr double taylor_sin(double x) {
    double x2 = x * x, term = x, sum = x;
    for (int i = 1; i < 16; ++i) {
        term *= -x2 / ((2.0 * i) * (2.0 * i + 1.0));
        sum += term;
    }
    return sum;
}

constexpr double taylor_cos(double x) {
    double x2 = x * x, term = 1.0, sum = 1.0;
    for (int i = 1; i < 16; ++i) {
        term *= -x2 / ((2.0 * i - 1.0) * (2.0 * i));
        sum += term;
    }
    return sum;
}

struct SinCos {
    double s, c;
};

constexpr SinCos sincos_2pi(long k, long n) {
    k = ((k % n) + n) % n;
    const long q = (4 * k) / n;    // quadrant
    const long r = 4 * k - q * n;  // angle within the quadrant = (pi/2) r / n
    double sa = 0, ca = 0;
    if (2 * r > n) {
        const double b = (kPi / 2) * (double)(n - r) / (double)n;
        sa = taylor_cos(b);
        ca = taylor_sin(b);
    } else {
        const double a = (kPi / 2) * (double)r / (double)n;
        sa = taylor_sin(a);
        ca = taylor_cos(a);
    }
    switch (q) {
        case 0: return SinCos{sa, ca};
        case 1: return SinCos{ca, -sa};
        case 2: return SinCos{-sa, -ca};
        default: return SinCos{-ca, sa};
    }
}

template <int N>
constexpr int ilog2() {
    int l = 0;
    while ((1 << l) < N) ++l;
    return l;
}

template <int N>
constexpr int bitrev(int i) {
    int r = 0;
    for (int b = 0; b < ilog2<N>(); ++b)
        if ((i >> b) & 1) r |= 1 << (ilog2<N>() - 1 - b);
    return r;
}

// Complex add and subtract. On sm_100 and later each is one paired FP32
// instruction (FADD2: two round-to-nearest adds, the same results as two
// scalar adds) instead of two: the butterflies issue fewer instructions. A
// translation unit that defines MFBD_SCALAR_COMPLEX_ADD before including
// this header keeps the scalar adds (the batch kernel, measured 3 % faster
// with them; the 128 px field 3 % faster with the paired ones).
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000) && !defined(MFBD_SCALAR_COMPLEX_ADD)
#define MFBD_PAIRED_ADD 1
#endif
MFBD_HD float2 cadd(float2 a, float2 b) {
#if defined(MFBD_PAIRED_ADD)
    return __fadd2_rn(a, b);
#else
    return make_float2(a.x + b.x, a.y + b.y);
#endif
}
MFBD_HD float2 csub(float2 a, float2 b) {
#if defined(MFBD_PAIRED_ADD)
    return __fadd2_rn(a, make_float2(-b.x, -b.y));
#else
    return make_float2(a.x - b.x, a.y - b.y);
#endif
}
MFBD_HD float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
MFBD_HD float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
MFBD_HD float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// v * exp(DIR * 2 pi i K / L)
template <int L, int K, int DIR>
MFBD_HD float2 twmul(float2 v) {
    constexpr int k = ((K % L) + L) % L;
    if constexpr (k == 0) {
        return v;
    } else if constexpr (2 * k == L) {
        return make_float2(-v.x, -v.y);
    } else if constexpr (4 * k == L) {  // exp(DIR i pi/2) = DIR * i
        if constexpr (DIR < 0) return make_float2(v.y, -v.x);
        else return make_float2(-v.y, v.x);
    } else if constexpr (4 * k == 3 * L) {
        if constexpr (DIR < 0) return make_float2(-v.y, v.x);
        else return make_float2(v.y, -v.x);
    } else {
        constexpr SinCos sc = sincos_2pi(k, L);
        constexpr float c = (float)sc.c;
        constexpr float s = (float)(DIR * sc.s);
        return make_float2(c * v.x - s * v.y, c * v.y + s * v.x);
    }
}

// In-place length-N complex FFT of a register array (natural order in/out).
template <int N, int DIR>
MFBD_HD void fft(float2 (&a)[N]) {
    float2 b[N];
    static_for<0, N>([&](auto i) { b[decltype(i)::value] = a[bitrev<N>(decltype(i)::value)]; });
    static_for<0, ilog2<N>()>([&](auto s) {
        constexpr int m = 1 << decltype(s)::value;
        static_for<0, N / 2>([&](auto t) {
            constexpr int T = decltype(t)::value;
            constexpr int i0 = (T / m) * 2 * m + (T % m);
            constexpr int i1 = i0 + m;
            const float2 o = twmul<2 * m, T % m, DIR>(b[i1]);
            const float2 e = b[i0];
            b[i0] = cadd(e, o);
            b[i1] = csub(e, o);
        });
    });
    static_for<0, N>([&](auto i) { a[decltype(i)::value] = b[decltype(i)::value]; });
}

template <int N>
constexpr int ilog4() {
    int l = 0;
    while ((1 << (2 * l)) < N) ++l;
    return l;
}

// base-4 digit reversal of i for N = 4^k
template <int N>
constexpr int digitrev4(int i) {
    int r = 0;
    for (int d = 0; d < ilog4<N>(); ++d) {
        r = (r << 2) | (i & 3);
        i >>= 2;
    }
    return r;
}

// In-place radix-4 decimation-in-time FFT for N = 4^k (natural order in and
// out). Each butterfly twiddles inputs 1..3 by W_{4L}^{qk} and applies the
// 4-point DFT with t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3, t3 = a1 - a3:
// X0 = t0 + t2, X2 = t0 - t2, X1 = t1 + DIR i t3, X3 = t1 - DIR i t3.
template <int N, int DIR>
MFBD_HD void fft4(float2 (&a)[N]) {
    static_assert((1 << (2 * ilog4<N>())) == N, "fft4 needs N = 4^k");
    float2 b[N];
    static_for<0, N>([&](auto i) { b[decltype(i)::value] = a[digitrev4<N>(decltype(i)::value)]; });
    static_for<0, ilog4<N>()>([&](auto s) {
        constexpr int L = 1 << (2 * decltype(s)::value);
        static_for<0, N / 4>([&](auto t) {
            constexpr int T = decltype(t)::value;
            constexpr int k = T % L;
            constexpr int i0 = (T / L) * 4 * L + k;
            const float2 a0 = b[i0];
            const float2 a1 = twmul<4 * L, k, DIR>(b[i0 + L]);
            const float2 a2 = twmul<4 * L, 2 * k, DIR>(b[i0 + 2 * L]);
            const float2 a3 = twmul<4 * L, 3 * k, DIR>(b[i0 + 3 * L]);
            const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
            const float2 t2 = cadd(a1, a3), t3 = csub(a1, a3);
            b[i0] = cadd(t0, t2);
            b[i0 + 2 * L] = csub(t0, t2);
            // t1 +- DIR i t3: the rotation swaps the parts, so these stay
            // scalar adds (a paired add would need the swapped pair first)
            if constexpr (DIR < 0) {
                b[i0 + L] = make_float2(t1.x + t3.y, t1.y - t3.x);
                b[i0 + 3 * L] = make_float2(t1.x - t3.y, t1.y + t3.x);
            } else {
                b[i0 + L] = make_float2(t1.x - t3.y, t1.y + t3.x);
                b[i0 + 3 * L] = make_float2(t1.x + t3.y, t1.y - t3.x);
            }
        });
    });
    static_for<0, N>([&](auto i) { a[decltype(i)::value] = b[decltype(i)::value]; });
}

// In-place 48-point FFT (natural order in and out): three 16-point FFTs of
// x[3n + r], each output twiddled by exp(DIR 2 pi i r k / 48), then a 3-point
// DFT over r: X[k + 16 q] = sum_r W3^(r q) (W48^(r k) A_r[k]).
template <int DIR>
MFBD_HD void fft48(float2 (&a)[48]) {
    float2 b[3][16];
    static_for<0, 48>([&](auto i) {
        constexpr int I = decltype(i)::value;
        b[I % 3][I / 3] = a[I];
    });
    fft4<16, DIR>(b[0]);
    fft4<16, DIR>(b[1]);
    fft4<16, DIR>(b[2]);
    constexpr float c3 = -0.5f;
    constexpr float s3 = (float)(DIR * 0.86602540378443864676);  // DIR sin(2 pi / 3)
    static_for<0, 16>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        const float2 x0 = b[0][k];
        const float2 x1 = twmul<48, k, DIR>(b[1][k]);
        const float2 x2 = twmul<48, 2 * k, DIR>(b[2][k]);
        const float2 sum = cadd(x1, x2), dif = csub(x1, x2);
        a[k] = cadd(x0, sum);
        const float2 m = make_float2(x0.x + c3 * sum.x, x0.y + c3 * sum.y);
        const float2 r = make_float2(-s3 * dif.y, s3 * dif.x);  // i s3 (x1 - x2)
        a[k + 16] = cadd(m, r);
        a[k + 32] = csub(m, r);
    });
}

// Length-L line FFT for the line lengths used (48, 64).
template <int L, int DIR>
MFBD_HD void fft_line(float2 (&a)[L]) {
    if constexpr (L == 48) fft48<DIR>(a);
    else fft4<L, DIR>(a);
}

// Real-to-complex forward FFT of N real samples -> X[0..N/2] (X[0], X[N/2]
// real), by one N/2-point complex FFT of z[n] = r[2n] + i r[2n+1]:
//   E[k] = (Z[k] + conj Z[H-k]) / 2,  O[k] = (Z[k] - conj Z[H-k]) / (2i),
//   X[k] = E[k] + exp(-2 pi i k / N) O[k].
template <int N>
MFBD_HD void rfft(const float (&r)[N], float2 (&X)[N / 2 + 1]) {
    constexpr int H = N / 2;
    float2 z[H];
    static_for<0, H>([&](auto n) {
        constexpr int i = decltype(n)::value;
        z[i] = make_float2(r[2 * i], r[2 * i + 1]);
    });
    fft<H, -1>(z);
    X[0] = make_float2(z[0].x + z[0].y, 0.f);
    X[H] = make_float2(z[0].x - z[0].y, 0.f);
    static_for<1, H>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        const float2 zk = z[k];
        const float2 zc = cconj(z[H - k]);
        const float2 e = cscale(cadd(zk, zc), 0.5f);
        const float2 d = cscale(csub(zk, zc), 0.5f);
        const float2 o = make_float2(d.y, -d.x);  // d / i
        X[k] = cadd(e, twmul<N, k, -1>(o));
    });
}

// Complex-to-real adjoint FFT: X[0..N/2] (Hermitian half, X[0] and X[N/2]
// taken as real) -> y[n] = sum_{k<N} Xfull[k] exp(+2 pi i k n / N), by one
// N/2-point inverse FFT of C[k] = A[k] + i B[k] with
//   A[k] = X[k] + conj X[H-k],  B[k] = (X[k] - conj X[H-k]) exp(+2 pi i k / N),
// whose output is y[2n] + i y[2n+1].
template <int N>
MFBD_HD void irfft(const float2 (&X)[N / 2 + 1], float (&y)[N]) {
    constexpr int H = N / 2;
    float2 c[H];
    c[0] = make_float2(X[0].x + X[H].x, X[0].x - X[H].x);
    static_for<1, H>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        const float2 xk = X[k];
        const float2 xc = cconj(X[H - k]);
        const float2 a = cadd(xk, xc);
        const float2 b = twmul<N, k, +1>(csub(xk, xc));
        c[k] = make_float2(a.x - b.y, a.y + b.x);
    });
    fft<H, +1>(c);
    static_for<0, H>([&](auto n) {
        constexpr int i = decltype(n)::value;
        y[2 * i] = c[i].x;
        y[2 * i + 1] = c[i].y;
    });
}

}  // namespace fftreg
