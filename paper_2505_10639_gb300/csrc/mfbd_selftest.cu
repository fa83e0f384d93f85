// Host-side execution of the register FFTs (see include/mfbd_testing.h).
#include "../../include/mfbd_testing.h"
#include "fft_reg.cuh"

extern "C" int mfbd_test_fft_host(int kind, const float* in, float* out) {
    if (!in || !out) return 1;
    switch (kind) {
        case 0:
        case 1: {
            float2 a[64];
            for (int i = 0; i < 64; ++i) a[i] = make_float2(in[2 * i], in[2 * i + 1]);
            if (kind == 0) fftreg::fft<64, -1>(a);
            else fftreg::fft<64, +1>(a);
            for (int i = 0; i < 64; ++i) { out[2 * i] = a[i].x; out[2 * i + 1] = a[i].y; }
            return 0;
        }
        case 2: {
            float r[64];
            float2 x[33];
            for (int i = 0; i < 64; ++i) r[i] = in[i];
            fftreg::rfft<64>(r, x);
            for (int i = 0; i < 33; ++i) { out[2 * i] = x[i].x; out[2 * i + 1] = x[i].y; }
            return 0;
        }
        case 3: {
            float2 x[33];
            float y[64];
            for (int i = 0; i < 33; ++i) x[i] = make_float2(in[2 * i], in[2 * i + 1]);
            fftreg::irfft<64>(x, y);
            for (int i = 0; i < 64; ++i) out[i] = y[i];
            return 0;
        }
        case 4: {
            float2 a[32];
            for (int i = 0; i < 32; ++i) a[i] = make_float2(in[2 * i], in[2 * i + 1]);
            fftreg::fft<32, -1>(a);
            for (int i = 0; i < 32; ++i) { out[2 * i] = a[i].x; out[2 * i + 1] = a[i].y; }
            return 0;
        }
        case 5:
        case 6: {
            float2 a[64];
            for (int i = 0; i < 64; ++i) a[i] = make_float2(in[2 * i], in[2 * i + 1]);
            if (kind == 5) fftreg::fft4<64, -1>(a);
            else fftreg::fft4<64, +1>(a);
            for (int i = 0; i < 64; ++i) { out[2 * i] = a[i].x; out[2 * i + 1] = a[i].y; }
            return 0;
        }
        case 7:
        case 8: {
            float2 a[48];
            for (int i = 0; i < 48; ++i) a[i] = make_float2(in[2 * i], in[2 * i + 1]);
            if (kind == 7) fftreg::fft48<-1>(a);
            else fftreg::fft48<+1>(a);
            for (int i = 0; i < 48; ++i) { out[2 * i] = a[i].x; out[2 * i + 1] = a[i].y; }
            return 0;
        }
        default:
            return 1;
    }
}
