// Pass and reduction kernels for the patch sizes other than 64 (48, 96, 128).
//
// The same passes as the 64-pixel pass machine (Sec. 3.1, Eqs. 20-22 and
// their adjoint), organised for lines that do not fit one thread: a line of
// N points is held by S = 1 (N <= 64) or S = 2 (N = 96, 128) lanes, L = N / S
// points each. A line transform runs a register FFT of L points on the
// decimated samples x[S n + s] of each lane s and, for S = 2, one radix-2
// stage across the lane pair by shuffles, leaving X[s L + k] in lane s
// (decimation in time); the decimation-in-frequency twin takes X in that
// blocked order and leaves x[S m + s]. One CTA works on one unit (patch,
// object, frame) at a time, 64 lines per round, with the 2-D transforms
// exchanged through an N x es buffer in shared memory and the passes
// separated by CTA barriers; CTAs are persistent over the units.
//
// RECOMPUTE (the adjoint kernel's template flag): the field p = F P and the
// pupil phasors are not kept by the forward passes; the adjoint recomputes
// the column transforms of P into a second buffer and each row of p just
// before it is needed.
#include "mfbd_internal.h"
#include "fft_reg.cuh"
#include "mfbd_device.cuh"

namespace mfbd_dev {

using fftreg::cadd;
using fftreg::cconj;
using fftreg::cmul;
using fftreg::cscale;
using fftreg::csub;

namespace {

template <int N>
struct Geo {
    static constexpr int S = N > 64 ? 2 : 1;  // lanes per line
    static constexpr int L = N / S;           // points per lane
    static constexpr int NH = N / 2 + 1;
    static constexpr int LINES = 64;          // lines per round
    static constexpr int THREADS = LINES * S;
};

__device__ __forceinline__ bool wbit(const uint32_t* rows, int words, int r, int c) {
    return (rows[r * words + (c >> 5)] >> (c & 31)) & 1u;
}

__device__ __forceinline__ float2 shfl_xor2(float2 v, int m) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// Forward (DIR = -1) line transform, decimation in time: lane s holds
// x[S n + s] on entry and X[s L + k] on exit.
template <int N, int DIR>
__device__ __forceinline__ void line_fft(float2 (&v)[Geo<N>::L], int sub) {
    constexpr int S = Geo<N>::S, L = Geo<N>::L;
    fftreg::fft_line<L, DIR>(v);
    if constexpr (S == 2) {
        fftreg::static_for<0, L>([&](auto kk) {
            constexpr int k = decltype(kk)::value;
            const float2 t = sub ? fftreg::twmul<N, k, DIR>(v[k]) : v[k];  // lane 1: W^k O[k]
            const float2 o = shfl_xor2(t, 1);
            v[k] = sub ? csub(o, t) : cadd(t, o);
        });
    }
}

// Decimation in frequency: lane s holds X[s L + k] on entry and the
// transform's x[S m + s] on exit.
template <int N, int DIR>
__device__ __forceinline__ void line_fft_dif(float2 (&v)[Geo<N>::L], int sub) {
    constexpr int S = Geo<N>::S, L = Geo<N>::L;
    if constexpr (S == 2) {
        fftreg::static_for<0, L>([&](auto kk) {
            constexpr int k = decltype(kk)::value;
            const float2 o = shfl_xor2(v[k], 1);
            v[k] = sub ? fftreg::twmul<N, k, DIR>(csub(o, v[k])) : cadd(v[k], o);
        });
    }
    fftreg::fft_line<L, DIR>(v);
}

// Conjugate partner Z[(N - kx) mod N] of the element k of lane `sub` (which
// holds kx = sub L + k after line_fft), for every k.
template <int N>
__device__ __forceinline__ void conj_partners(const float2 (&v)[Geo<N>::L], float2 (&pc)[Geo<N>::L], int sub) {
    constexpr int S = Geo<N>::S, L = Geo<N>::L;
    fftreg::static_for<0, L>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        if constexpr (S == 1) {
            pc[k] = cconj(v[(L - k) % L]);
        } else if constexpr (k == 0) {
            pc[k] = cconj(v[0]);  // kx = 0 or N/2: its own partner
        } else {
            pc[k] = cconj(shfl_xor2(v[L - k], 1));
        }
    });
    (void)sub;
}

template <int N>
struct UnitPtr {
    const float* phi;  // [W][W] box phase
    float* gphi;
    float2* h;         // [N][NH]
    float2* pf;        // [N x N] field [x][y] or null
    float2* pp;        // [W][W] phasors or null
    const uint32_t* mask;
    int mw;
    int W;
    float inv_z;
};

template <int N>
__device__ __forceinline__ UnitPtr<N> unit_ptr(const GenericParams& prm, long long u) {
    const int J = prm.J, K = prm.K;
    const int j = (int)(u % J);
    const long long pk = u / J;
    const int k = (int)(pk % K);
    const long long p = pk / K;
    const GenericObj& ob = prm.obj[k];
    const long long img = (p * J + j) * (long long)ob.W * ob.W;
    UnitPtr<N> q;
    q.phi = prm.phi + ob.phi_off + img;
    q.gphi = prm.gphi + ob.phi_off + img;
    q.h = prm.gscr + (size_t)u * N * Geo<N>::NH;
    q.pf = prm.pscr ? prm.pscr + (size_t)u * N * N : nullptr;
    q.pp = prm.uscr ? prm.uscr + (size_t)u * prm.ustride : nullptr;
    q.mask = ob.mask;
    q.mw = ob.mw;
    q.W = ob.W;
    q.inv_z = ob.inv_z;
    return q;
}

// PUPIL: the W box columns of P = exp(i phi) (zero-padded to N rows),
// transformed along y into columns c of B (row stride bs); phasors kept
// when `keep` and the unit has a buffer.
template <int N>
__device__ __forceinline__ void pass_pupil(const UnitPtr<N>& q, float2* B, int bs, bool keep) {
    constexpr int S = Geo<N>::S, L = Geo<N>::L;
    const int t = threadIdx.x, sub = t % S, li = t / S;
    for (int c0 = 0; c0 < q.W; c0 += Geo<N>::LINES) {
        const int c = c0 + li;
        const bool act = c < q.W;
        float2 v[L];
#pragma unroll
        for (int n = 0; n < L; ++n) {
            const int y = S * n + sub;
            float2 val = make_float2(0.f, 0.f);
            if (act && y < q.W) {
                if (wbit(q.mask, q.mw, y, c)) val = expi(q.phi[y * q.W + c]);
                if (keep && q.pp) q.pp[y * q.W + c] = val;
            }
            v[n] = val;
        }
        line_fft<N, -1>(v, sub);
        if (act) {
#pragma unroll
            for (int k = 0; k < L; ++k) B[(sub * L + k) * bs + c] = v[k];
        }
    }
}

// ------------------------------------------------------------------ forward

template <int N>
__global__ void __launch_bounds__(Geo<N>::THREADS) generic_forward_kernel(const GenericParams prm) {
    constexpr int S = Geo<N>::S, L = Geo<N>::L, NH = Geo<N>::NH;
    extern __shared__ __align__(16) unsigned char gsm[];
    float2* E = reinterpret_cast<float2*>(gsm);
    float* Ef = reinterpret_cast<float*>(gsm);
    const int es = prm.es;
    const int t = threadIdx.x, sub = t % S, li = t / S;
    const long long units = (long long)prm.P * prm.K * prm.J;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        const UnitPtr<N> q = unit_ptr<N>(prm, u);
        const int k_obj = (int)((u / prm.J) % prm.K);
        const uint32_t* supp = prm.obj[k_obj].supp;
        pass_pupil<N>(q, E, es, true);
        __syncthreads();
        // FIELD rows: p = F P along x; the PSF row |p|^2 / (N^2 n_pup) as floats
        for (int y0 = 0; y0 < N; y0 += Geo<N>::LINES) {
            const int y = y0 + li;
            const bool act = y < N;
            float2 v[L];
#pragma unroll
            for (int n = 0; n < L; ++n) {
                const int x = S * n + sub;
                v[n] = (act && x < q.W) ? E[y * es + x] : make_float2(0.f, 0.f);
            }
            line_fft<N, -1>(v, sub);
            __syncwarp();  // both lanes of the line have read row y
            if (act) {
#pragma unroll
                for (int k = 0; k < L; ++k) {
                    const int kx = sub * L + k;
                    if (q.pf) q.pf[(size_t)kx * N + y] = v[k];
                    Ef[(size_t)y * 2 * es + kx] = (v[k].x * v[k].x + v[k].y * v[k].y) * q.inv_z;
                }
            }
        }
        __syncthreads();
        // PSF rows y and y + N/2 as one complex line; split into the two
        // half spectra (kx <= N/2)
        for (int y0 = 0; y0 < N / 2; y0 += Geo<N>::LINES) {
            const int y = y0 + li;
            const bool act = y < N / 2;
            float2 v[L], pc[L];
#pragma unroll
            for (int n = 0; n < L; ++n) {
                const int x = S * n + sub;
                v[n] = act ? make_float2(Ef[(size_t)y * 2 * es + x], Ef[(size_t)(y + N / 2) * 2 * es + x])
                           : make_float2(0.f, 0.f);
            }
            line_fft<N, -1>(v, sub);
            conj_partners<N>(v, pc, sub);
            __syncwarp();
            if (act) {
#pragma unroll
                for (int k = 0; k < L; ++k) {
                    const int kx = sub * L + k;
                    if (kx <= N / 2) {
                        const float2 a = cscale(cadd(v[k], pc[k]), 0.5f);
                        const float2 d = cscale(csub(v[k], pc[k]), 0.5f);
                        E[y * es + kx] = a;
                        E[(y + N / 2) * es + kx] = make_float2(d.y, -d.x);
                    }
                }
            }
        }
        __syncthreads();
        // OTF columns kx = 1 .. N/2 - 1; line 0 packs the real columns 0 and N/2
        for (int l0 = 0; l0 < N / 2; l0 += Geo<N>::LINES) {
            const int line = l0 + li;
            const bool act = line < N / 2;
            const int kx = line;
            float2 v[L], pc[L];
#pragma unroll
            for (int n = 0; n < L; ++n) {
                const int ky = S * n + sub;
                if (!act) v[n] = make_float2(0.f, 0.f);
                else if (kx == 0) v[n] = make_float2(E[ky * es].x, E[ky * es + N / 2].x);
                else v[n] = E[ky * es + kx];
            }
            line_fft<N, -1>(v, sub);
            conj_partners<N>(v, pc, sub);
            if (act) {
#pragma unroll
                for (int k = 0; k < L; ++k) {
                    const int ky = sub * L + k;
                    if (kx > 0) {
                        q.h[ky * NH + kx] = wbit(supp, prm.sw, ky, kx) ? v[k] : make_float2(0.f, 0.f);
                    } else {
                        float2 h0 = cscale(cadd(v[k], pc[k]), 0.5f);
                        const float2 d = cscale(csub(v[k], pc[k]), 0.5f);
                        float2 hn = make_float2(d.y, -d.x);
                        if (!wbit(supp, prm.sw, ky, 0)) h0 = make_float2(0.f, 0.f);
                        if (!wbit(supp, prm.sw, ky, N / 2)) hn = make_float2(0.f, 0.f);
                        if (ky == 0) h0 = make_float2(1.f, 0.f);
                        q.h[ky * NH] = h0;
                        q.h[ky * NH + N / 2] = hn;
                    }
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ adjoint

template <int N, bool RECOMPUTE>
__global__ void __launch_bounds__(Geo<N>::THREADS) generic_adjoint_kernel(const GenericParams prm) {
    constexpr int S = Geo<N>::S, L = Geo<N>::L, NH = Geo<N>::NH;
    extern __shared__ __align__(16) unsigned char gsm[];
    float2* E = reinterpret_cast<float2*>(gsm);
    float* Ef = reinterpret_cast<float*>(gsm);
    const int es = prm.es, es2 = prm.es2;
    float2* E2 = E + (size_t)N * es;  // RECOMPUTE: column transforms of P
    const int t = threadIdx.x, sub = t % S, li = t / S;
    const long long units = (long long)prm.P * prm.K * prm.J;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        const UnitPtr<N> q = unit_ptr<N>(prm, u);
        // SEED: conj of the columns of G; line 0 packs the columns 0 and N/2
        for (int l0 = 0; l0 < N / 2; l0 += Geo<N>::LINES) {
            const int line = l0 + li;
            const bool act = line < N / 2;
            const int kx = line;
            float2 v[L];
#pragma unroll
            for (int n = 0; n < L; ++n) {
                const int ky = S * n + sub;
                float2 g = make_float2(0.f, 0.f);
                if (act) {
                    if (kx == 0) {
                        const float2 a = q.h[ky * NH], b = q.h[ky * NH + N / 2];
                        g = make_float2(a.x - b.y, a.y + b.x);  // a + i b
                    } else {
                        g = q.h[ky * NH + kx];
                    }
                }
                v[n] = cconj(g);
            }
            line_fft<N, -1>(v, sub);
            if (act) {
#pragma unroll
                for (int k = 0; k < L; ++k) E[(sub * L + k) * es + kx] = cconj(v[k]);  // kx = 0: (T_0, T_N/2), both real
            }
        }
        __syncthreads();
        // C2R rows y and y + N/2: conj of T_y + i T_(y+N/2), Hermitian-extended
        // along x; g_q rows (2 Re / (N^2 n_pup)) as floats
        for (int y0 = 0; y0 < N / 2; y0 += Geo<N>::LINES) {
            const int y = y0 + li;
            const bool act = y < N / 2;
            float2 v[L];
#pragma unroll
            for (int n = 0; n < L; ++n) {
                const int x = S * n + sub;
                float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
                if (act) {
                    if (x == 0) {
                        a = make_float2(E[y * es].x, 0.f);
                        b = make_float2(E[(y + N / 2) * es].x, 0.f);
                    } else if (x == N / 2) {
                        a = make_float2(E[y * es].y, 0.f);
                        b = make_float2(E[(y + N / 2) * es].y, 0.f);
                    } else if (x < N / 2) {
                        a = E[y * es + x];
                        b = E[(y + N / 2) * es + x];
                    } else {
                        a = cconj(E[y * es + N - x]);
                        b = cconj(E[(y + N / 2) * es + N - x]);
                    }
                }
                v[n] = make_float2(a.x - b.y, -(a.y + b.x));  // conj(a + i b)
            }
            line_fft<N, -1>(v, sub);
            __syncwarp();
            if (act) {
                const float sc = 2.0f * q.inv_z;
#pragma unroll
                for (int k = 0; k < L; ++k) {
                    const int x = sub * L + k;
                    Ef[(size_t)y * 2 * es + x] = v[k].x * sc;
                    Ef[(size_t)(y + N / 2) * 2 * es + x] = -v[k].y * sc;
                }
            }
        }
        __syncthreads();
        if constexpr (RECOMPUTE) {
            pass_pupil<N>(q, E2, es2, false);
            __syncthreads();
        }
        // rows of F^H(g_q p), kept on the box columns x < W
        for (int y0 = 0; y0 < N; y0 += Geo<N>::LINES) {
            const int y = y0 + li;
            const bool act = y < N;
            float2 v[L];
            int pos_mul, pos_add;  // output element k sits at x = pos_mul k + pos_add
            if constexpr (!RECOMPUTE) {
#pragma unroll
                for (int n = 0; n < L; ++n) {
                    const int x = S * n + sub;
                    float2 w = make_float2(0.f, 0.f);
                    if (act) {
                        const float g = Ef[(size_t)y * 2 * es + x];
                        const float2 pv = q.pf[(size_t)x * N + y];
                        w = make_float2(g * pv.x, -g * pv.y);  // conj(g_q p)
                    }
                    v[n] = w;
                }
                line_fft<N, -1>(v, sub);
                pos_mul = 1;
                pos_add = sub * L;
            } else {
                // p row y from the recomputed columns (blocked order kx = sub L + k)
#pragma unroll
                for (int n = 0; n < L; ++n) {
                    const int x = S * n + sub;
                    v[n] = (act && x < q.W) ? E2[y * es2 + x] : make_float2(0.f, 0.f);
                }
                line_fft<N, -1>(v, sub);
#pragma unroll
                for (int k = 0; k < L; ++k) {
                    const int kx = sub * L + k;
                    const float g = act ? Ef[(size_t)y * 2 * es + kx] : 0.f;
                    v[k] = make_float2(g * v[k].x, -g * v[k].y);
                }
                line_fft_dif<N, -1>(v, sub);
                pos_mul = S;
                pos_add = sub;
            }
            __syncwarp();
            if (act) {
#pragma unroll
                for (int k = 0; k < L; ++k) {
                    const int x = pos_mul * k + pos_add;
                    if (x < q.W) E[y * es + x] = cconj(v[k]);
                }
            }
        }
        __syncthreads();
        // ADJ: box columns of F^H along y; dL/dphi = 2 Im(conj(P) G_P) on the pupil
        for (int c0 = 0; c0 < q.W; c0 += Geo<N>::LINES) {
            const int c = c0 + li;
            const bool act = c < q.W;
            float2 v[L];
#pragma unroll
            for (int n = 0; n < L; ++n) {
                const int y = S * n + sub;
                v[n] = act ? cconj(E[y * es + c]) : make_float2(0.f, 0.f);
            }
            line_fft<N, -1>(v, sub);
            if (act) {
#pragma unroll
                for (int k = 0; k < L; ++k) {
                    const int y = sub * L + k;
                    if (y < q.W) {
                        float gv = 0.f;
                        if (wbit(q.mask, q.mw, y, c)) {
                            const float2 pv = q.pp ? q.pp[y * q.W + c] : expi(q.phi[y * q.W + c]);
                            const float2 g = cconj(v[k]);
                            gv = 2.0f * (pv.x * g.y - pv.y * g.x);
                        }
                        q.gphi[y * q.W + c] = gv;
                    }
                }
            }
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------- reduction

// Frame reduction of one (patch, object) by one warp for any patch size (the
// same arithmetic as the 64-pixel reduction: residual form in FP32, FP64
// where it would cancel, Kahan sums per lane, FP64 warp combine).
__device__ double generic_reduce_warp(const GenericParams& prm, int p, int k) {
    const int lane = threadIdx.x & 31;
    const int N = prm.N, NH = N / 2 + 1, half = N * NH, J = prm.J;
    const size_t unit0 = ((size_t)p * prm.K + k) * J;
    const size_t dstride = (size_t)N * prm.spec_ld;
    const float2* dbase = prm.spectra + unit0 * dstride;
    float2* hbase = prm.gscr + unit0 * half;
    const float* w = prm.weights + (size_t)k * J;
    const uint32_t* supp = prm.obj[k].supp;
    const float gam = (float)prm.gamma;
    KahanSum acc;
    for (int f = lane; f < half; f += 32) {
        const int ky = f / NH, kx = f - ky * NH;
        const size_t doff = (size_t)ky * prm.spec_ld + kx;
        const float2* dp = dbase + doff;
        float2* hp = hbase + f;
        const bool seed = (f != 0) && wbit(supp, prm.sw, ky, kx);
        float2 num = make_float2(0.f, 0.f), o;
        float e = 0.f, qs = 0.f, tval;
        for (int j = 0; j < J; ++j) {
            const float2 d = dp[(size_t)j * dstride];
            const float2 h = hp[(size_t)j * half];
            const float wj = w[j];
            num.x += wj * (d.x * h.x + d.y * h.y);
            num.y += wj * (d.y * h.x - d.x * h.y);
            e += wj * (d.x * d.x + d.y * d.y);
            qs += wj * (h.x * h.x + h.y * h.y);
        }
        qs += gam;
        const float invq = 1.0f / qs;
        o = cscale(num, invq);
        const float t_est = e - (num.x * num.x + num.y * num.y) * invq;
        if (f != 0 && t_est < kCancel * e) {
            fp64_frequency(J, dp, dstride, hp, half, w, prm.gamma, seed, tval, o);
        } else {
            float tsum = 0.f;
            for (int j = 0; j < J; ++j) {
                const float2 d = dp[(size_t)j * dstride];
                const float2 h = hp[(size_t)j * half];
                const float wj = w[j];
                const float2 r = csub(d, cmul(o, h));
                tsum += wj * (r.x * r.x + r.y * r.y);
                hp[(size_t)j * half] = seed ? cscale(cmul(cconj(o), r), -wj) : make_float2(0.f, 0.f);
            }
            tval = tsum + gam * (o.x * o.x + o.y * o.y);
        }
        acc.add((kx == 0 || kx == N / 2) ? tval : 2.0f * tval);
        if (prm.object) {
            float2* ob = prm.object + ((size_t)p * prm.K + k) * dstride;
            ob[doff] = o;
            if (prm.spec_ld == N && kx > 0 && kx < N / 2) ob[(size_t)((N - ky) % N) * N + (N - kx)] = cconj(o);
        }
    }
    double v = (double)acc.s - (double)acc.c;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}

__global__ void __launch_bounds__(32 * kMaxObjects) generic_reduce_kernel(const GenericParams prm) {
    __shared__ double sobj[kMaxObjects];
    const int k = threadIdx.x >> 5;
    for (int p = blockIdx.x; p < prm.P; p += gridDim.x) {
        const double v = generic_reduce_warp(prm, p, k);
        if ((threadIdx.x & 31) == 0) sobj[k] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int i = 0; i < prm.K; ++i) tot += sobj[i];
            prm.loss[p] = tot;
        }
        __syncthreads();
    }
}

template <class Kern>
cudaError_t launch_persistent(Kern kern, int threads, size_t smem, long long units, int sms, const GenericParams& prm,
                              cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long ctas = (long long)sms * per_sm;
    if (ctas > units) ctas = units;
    kern<<<(int)ctas, threads, smem, s>>>(prm);
    return cudaGetLastError();
}

}  // namespace

size_t generic_smem(int N, int es, int es2, bool recompute) {
    return (size_t)N * es * sizeof(float2) + (recompute ? (size_t)N * es2 * sizeof(float2) : 0);
}

cudaError_t launch_generic_forward(const GenericParams& prm, int sms, cudaStream_t s) {
    const long long units = (long long)prm.P * prm.K * prm.J;
    if (units == 0) return cudaSuccess;
    const size_t smem = generic_smem(prm.N, prm.es, prm.es2, false);
    switch (prm.N) {
        case 48: return launch_persistent(generic_forward_kernel<48>, Geo<48>::THREADS, smem, units, sms, prm, s);
        case 64: return launch_persistent(generic_forward_kernel<64>, Geo<64>::THREADS, smem, units, sms, prm, s);
        case 96: return launch_persistent(generic_forward_kernel<96>, Geo<96>::THREADS, smem, units, sms, prm, s);
        case 128: return launch_persistent(generic_forward_kernel<128>, Geo<128>::THREADS, smem, units, sms, prm, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_generic_adjoint(const GenericParams& prm, int sms, cudaStream_t s) {
    const long long units = (long long)prm.P * prm.K * prm.J;
    if (units == 0) return cudaSuccess;
    const bool rec = prm.pscr == nullptr;
    const size_t smem = generic_smem(prm.N, prm.es, prm.es2, rec);
#define MFBD_ADJ(NN)                                                                                            \
    case NN:                                                                                                    \
        return rec ? launch_persistent(generic_adjoint_kernel<NN, true>, Geo<NN>::THREADS, smem, units, sms, prm, s) \
                   : launch_persistent(generic_adjoint_kernel<NN, false>, Geo<NN>::THREADS, smem, units, sms, prm, s);
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
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, generic_reduce_kernel, threads, 0);
    if (e != cudaSuccess) return e;
    long long ctas = (long long)sms * (per_sm > 0 ? per_sm : 1);
    if (ctas > prm.P) ctas = prm.P;
    generic_reduce_kernel<<<(int)ctas, threads, 0, s>>>(prm);
    return cudaGetLastError();
}

}  // namespace mfbd_dev
