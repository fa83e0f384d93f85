// Per-unit passes of the CTA-per-unit kernels (patch sizes 48, 64, 96, 128),
// shared by the single-problem kernels (generic_kernels.cu) and the batched
// persistent kernel (batch_kernels.cu).
//
// The passes are those of Sec. 3.1, Eqs. 20-22 and their adjoint: a line of
// N points is held by S = 1 (N <= 64) or S = 2 (N = 96, 128) lanes, L = N / S
// points each. A line transform runs a register FFT of L points on the
// decimated samples x[S n + s] of each lane s and, for S = 2, one radix-2
// stage across the lane pair by shuffles, leaving X[s L + k] in lane s
// (decimation in time); the decimation-in-frequency twin takes X in that
// blocked order and leaves x[S m + s]. A group of LINES * S threads works on
// one unit (patch, object, frame), LINES lines per round, with the 2-D
// transforms exchanged through an N x es buffer in shared memory and the
// passes separated by the group's barrier: one warp (LINES = 32, N <= 64,
// __syncwarp), or 128 threads (LINES = 64, N = 96, 128: the CTA's barrier or
// a named barrier).
//
// RECOMPUTE (the adjoint's template flag): the field p = F P and the pupil
// phasors are not kept by the forward passes; the adjoint recomputes the
// column transforms of P into a second buffer and each row of p just before
// it is needed.
#pragma once

#include <cstdint>

#include "fft_reg.cuh"
#include "mfbd_device.cuh"

namespace mfbd_dev {
namespace unitpass {

using fftreg::cadd;
using fftreg::cconj;
using fftreg::cmul;
using fftreg::cscale;
using fftreg::csub;

template <int N>
struct Geo {
    static constexpr int S = N > 64 ? 2 : 1;  // lanes per line
    static constexpr int L = N / S;           // points per lane
    static constexpr int NH = N / 2 + 1;
    static constexpr int LINES = 64;          // lines per round of a 64 S-thread group
    static constexpr int THREADS = LINES * S;
};

// Barrier of the threads that work on one unit: the whole CTA, or the named
// barrier `id` of a group of n threads (n a multiple of 32).
struct CtaBar {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct WarpBar {  // a group of one warp (32 lines per round, N <= 64)
    __device__ __forceinline__ void operator()() const { __syncwarp(); }
};
struct GroupBar {
    int id, n;
    __device__ __forceinline__ void operator()() const {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
    }
};

__device__ __forceinline__ bool wbit(const uint32_t* rows, int words, int r, int c) {
    return (rows[r * words + (c >> 5)] >> (c & 31)) & 1u;
}

// Bit i (< 128) of a column held as two 64-bit words.
__device__ __forceinline__ bool cbit(uint64_t w0, uint64_t w1, int i) {
    return ((i < 64 ? w0 >> i : w1 >> (i - 64)) & 1ull) != 0;
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

// Conjugate partner conj Z[(N - kx) mod N] of element K of this lane (which
// holds kx = sub L + K after line_fft). With S = 2 it comes from the pair
// lane by a shuffle that every lane of the warp executes; the callers take
// one partner at a time so that no second register array is live.
template <int N, int K>
__device__ __forceinline__ float2 conj_partner(const float2 (&v)[Geo<N>::L]) {
    constexpr int S = Geo<N>::S, L = Geo<N>::L;
    if constexpr (S == 1) return cconj(v[(L - K) % L]);
    else if constexpr (K == 0) return cconj(v[0]);  // kx = 0 or N/2: its own partner
    else return cconj(shfl_xor2(v[L - K], 1));
}

// Everything one unit's passes touch.
struct UnitPtr {
    const float* phi;       // [W][W] box phase
    float* gphi;            // [W][W] dL/dphi (0 outside the pupil)
    float2* h;              // [N][N/2+1]: OTF, then the adjoint seed
    float2* pf;             // [N x N] field [x][y], or null (recomputed)
    float2* pp;             // [W][W] phasors, or null (recomputed / not kept)
    const uint32_t* mask;   // [W][mw] box rows, bit c = pupil pixel at box column c
    int mw;
    int W;
    float inv_z;            // 1 / (N^2 n_pup)
    const uint32_t* supp;   // [N][sw] OTF-support rows over kx <= N/2
    int sw;
    const uint64_t* cmask;  // [W][2] box column c: bit y = pupil pixel at box (y, c)
    const uint64_t* csupp;  // [N/2+1][2] column kx: bit ky = OTF support
};

// PUPIL: the W box columns of P = exp(i phi) (zero-padded to N rows),
// transformed along y into columns c of B (row stride bs); phasors kept
// when `keep` and the unit has a buffer. t: thread index in the group.
template <int N, int LINES>
__device__ __forceinline__ void pass_pupil(const UnitPtr& q, float2* B, int bs, bool keep, int t) {
    constexpr int S = Geo<N>::S, L = Geo<N>::L;
    const int sub = t % S, li = t / S;
    for (int c0 = 0; c0 < q.W; c0 += LINES) {
        const int c = c0 + li;
        const bool act = c < q.W;
        const uint64_t m0 = act ? q.cmask[2 * c] : 0ull, m1 = act ? q.cmask[2 * c + 1] : 0ull;
        float2 v[L];
#pragma unroll
        for (int n = 0; n < L; ++n) {
            const int y = S * n + sub;
            float2 val = make_float2(0.f, 0.f);
            if (act && y < q.W) {
                if (cbit(m0, m1, y)) val = expi(q.phi[y * q.W + c]);
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

// Forward passes of one unit: PUPIL, FIELD (field kept when q.pf), PSF rows,
// OTF columns -> q.h (masked by the OTF support, H(0) = 1). E: the group's
// N x es exchange buffer. Ends with the group's barrier.
template <int N, int LINES, class Bar>
__device__ __forceinline__ void unit_forward(const UnitPtr& q, float2* E, int es, int t, Bar bar) {
    constexpr int S = Geo<N>::S, L = Geo<N>::L, NH = Geo<N>::NH;
    float* Ef = reinterpret_cast<float*>(E);
    const int sub = t % S, li = t / S;
    pass_pupil<N, LINES>(q, E, es, true, t);
    bar();
    // FIELD rows: p = F P along x; the PSF row |p|^2 / (N^2 n_pup) as floats
    for (int y0 = 0; y0 < N; y0 += LINES) {
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
    bar();
    // PSF rows y and y + N/2 as one complex line; split into the two
    // half spectra (kx <= N/2)
    for (int y0 = 0; y0 < N / 2; y0 += LINES) {
        const int y = y0 + li;
        const bool act = y < N / 2;
        float2 v[L];
#pragma unroll
        for (int n = 0; n < L; ++n) {
            const int x = S * n + sub;
            v[n] = act ? make_float2(Ef[(size_t)y * 2 * es + x], Ef[(size_t)(y + N / 2) * 2 * es + x])
                       : make_float2(0.f, 0.f);
        }
        line_fft<N, -1>(v, sub);
        __syncwarp();
        fftreg::static_for<0, L>([&](auto kk) {
            constexpr int k = decltype(kk)::value;
            const float2 pc = conj_partner<N, k>(v);
            const int kx = sub * L + k;
            if (act && kx <= N / 2) {
                const float2 a = cscale(cadd(v[k], pc), 0.5f);
                const float2 d = cscale(csub(v[k], pc), 0.5f);
                E[y * es + kx] = a;
                E[(y + N / 2) * es + kx] = make_float2(d.y, -d.x);
            }
        });
    }
    bar();
    // OTF columns kx = 1 .. N/2 - 1; line 0 packs the real columns 0 and N/2
    for (int l0 = 0; l0 < N / 2; l0 += LINES) {
        const int line = l0 + li;
        const bool act = line < N / 2;
        const int kx = line;
        float2 v[L];
#pragma unroll
        for (int n = 0; n < L; ++n) {
            const int ky = S * n + sub;
            if (!act) v[n] = make_float2(0.f, 0.f);
            else if (kx == 0) v[n] = make_float2(E[ky * es].x, E[ky * es + N / 2].x);
            else v[n] = E[ky * es + kx];
        }
        line_fft<N, -1>(v, sub);
        const uint64_t s0 = act ? q.csupp[2 * kx] : 0ull, s1 = act ? q.csupp[2 * kx + 1] : 0ull;
        const uint64_t n0 = act && kx == 0 ? q.csupp[N] : 0ull, n1 = act && kx == 0 ? q.csupp[N + 1] : 0ull;
        fftreg::static_for<0, L>([&](auto kk) {
            constexpr int k = decltype(kk)::value;
            const float2 pc = conj_partner<N, k>(v);
            const int ky = sub * L + k;
            if (act) {
                if (kx > 0) {
                    q.h[ky * NH + kx] = cbit(s0, s1, ky) ? v[k] : make_float2(0.f, 0.f);
                } else {
                    float2 h0 = cscale(cadd(v[k], pc), 0.5f);
                    const float2 d = cscale(csub(v[k], pc), 0.5f);
                    float2 hn = make_float2(d.y, -d.x);
                    if (!cbit(s0, s1, ky)) h0 = make_float2(0.f, 0.f);
                    if (!cbit(n0, n1, ky)) hn = make_float2(0.f, 0.f);
                    if (ky == 0) h0 = make_float2(1.f, 0.f);
                    q.h[ky * NH] = h0;
                    q.h[ky * NH + N / 2] = hn;
                }
            }
        });
    }
    bar();
}

// Adjoint passes of one unit: SEED (columns of the seed G in q.h), C2R rows
// -> g_q, rows of F^H(g_q p), ADJ columns -> q.gphi = 2 Im(conj(P) G_P) on
// the pupil (0 elsewhere in the box). E2 (row stride es2): RECOMPUTE's
// buffer for the column transforms of P. Ends with the group's barrier.
template <int N, int LINES, bool RECOMPUTE, class Bar>
__device__ __forceinline__ void unit_adjoint(const UnitPtr& q, float2* E, int es, float2* E2, int es2, int t,
                                             Bar bar) {
    constexpr int S = Geo<N>::S, L = Geo<N>::L, NH = Geo<N>::NH;
    float* Ef = reinterpret_cast<float*>(E);
    const int sub = t % S, li = t / S;
    // SEED: conj of the columns of G; line 0 packs the columns 0 and N/2
    for (int l0 = 0; l0 < N / 2; l0 += LINES) {
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
    bar();
    // C2R rows y and y + N/2: conj of T_y + i T_(y+N/2), Hermitian-extended
    // along x; g_q rows (2 Re / (N^2 n_pup)) as floats
    for (int y0 = 0; y0 < N / 2; y0 += LINES) {
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
    bar();
    if constexpr (RECOMPUTE) {
        pass_pupil<N, LINES>(q, E2, es2, false, t);
        bar();
    }
    // rows of F^H(g_q p), kept on the box columns x < W
    for (int y0 = 0; y0 < N; y0 += LINES) {
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
    bar();
    // ADJ: box columns of F^H along y; dL/dphi = 2 Im(conj(P) G_P) on the pupil
    for (int c0 = 0; c0 < q.W; c0 += LINES) {
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
            const uint64_t m0 = q.cmask[2 * c], m1 = q.cmask[2 * c + 1];
#pragma unroll
            for (int k = 0; k < L; ++k) {
                const int y = sub * L + k;
                if (y < q.W) {
                    float gv = 0.f;
                    if (cbit(m0, m1, y)) {
                        const float2 pv = q.pp ? q.pp[y * q.W + c] : expi(q.phi[y * q.W + c]);
                        const float2 g = cconj(v[k]);
                        gv = 2.0f * (pv.x * g.y - pv.y * g.x);
                    }
                    q.gphi[y * q.W + c] = gv;
                }
            }
        }
    }
    bar();
}

// The passes of one unit. Forward: PUPIL (box columns of P = exp(i phi),
// zero-padded, along y), FIELD (rows of p = F P along x; the field is kept
// when q.pf; the PSF rows |p|^2 / (N^2 n_pup) as floats), PSF (rows y and
// y + N/2 of the PSF as one complex line, split into two half spectra), OTF
// (half-spectrum columns -> q.h, masked by the OTF support, H(0) = 1; line 0
// packs the real columns 0 and N/2). Adjoint: SEED (conj of the columns of
// the seed G in q.h), C2R (rows y and y + N/2, Hermitian-extended -> the g_q
// rows 2 Re / (N^2 n_pup) as floats), RPUPIL (recompute only: PUPIL into the
// second buffer E2), GP (rows of F^H(g_q p) on the box columns), ADJ (box
// columns of F^H along y -> q.gphi = 2 Im(conj(P) G_P) on the pupil, 0
// elsewhere in the box).
enum Pass : int { PS_PUPIL = 0, PS_FIELD, PS_PSF, PS_OTF, PS_SEED, PS_C2R, PS_RPUPIL, PS_GP, PS_ADJ };

__device__ __forceinline__ int pass_lines(int ps, int N, int W) {
    return (ps == PS_PUPIL || ps == PS_RPUPIL || ps == PS_ADJ) ? W : (ps == PS_FIELD || ps == PS_GP) ? N : N / 2;
}

// The same forward passes as rounds of LINES lines: each round loads one
// line per lane group (a branch on the pass), runs the one register FFT of
// this function and stores (a branch on the pass), so the unrolled FFT
// exists once in the code: smaller code, at the price of pass-generic
// register allocation. Measured on GB300: faster for N <= 64 forward passes
// and inside the batched kernel; slower for N = 96, 128 and for the N <= 64
// adjoint on their own kernels. E: the group's N x es exchange buffer; t: thread index in the
// group. Each pass ends with the group's barrier.
template <int N, int LINES, class Bar>
__device__ __forceinline__ void unit_forward_rounds(const UnitPtr& q, float2* E, int es, int t, Bar bar) {
    constexpr int S = Geo<N>::S, L = Geo<N>::L, NH = Geo<N>::NH;
    float* Ef = reinterpret_cast<float*>(E);
    const int sub = t % S, li = t / S;
    const int W = q.W;
#pragma unroll 1
    for (int ps = PS_PUPIL; ps <= PS_OTF; ++ps) {
        const int lines = pass_lines(ps, N, W);
#pragma unroll 1
        for (int l0 = 0; l0 < lines; l0 += LINES) {
            const int line = l0 + li;
            const bool act = line < lines;
            float2 v[L];
            if (ps == PS_PUPIL) {
                const uint64_t m0 = act ? q.cmask[2 * line] : 0ull, m1 = act ? q.cmask[2 * line + 1] : 0ull;
#pragma unroll
                for (int n = 0; n < L; ++n) {
                    const int y = S * n + sub;
                    float2 val = make_float2(0.f, 0.f);
                    if (act && y < W) {
                        if (cbit(m0, m1, y)) val = expi(q.phi[y * W + line]);
                        if (q.pp) q.pp[y * W + line] = val;
                    }
                    v[n] = val;
                }
            } else if (ps == PS_FIELD) {
#pragma unroll
                for (int n = 0; n < L; ++n) {
                    const int x = S * n + sub;
                    v[n] = (act && x < W) ? E[line * es + x] : make_float2(0.f, 0.f);
                }
            } else if (ps == PS_PSF) {
#pragma unroll
                for (int n = 0; n < L; ++n) {
                    const int x = S * n + sub;
                    v[n] = act ? make_float2(Ef[(size_t)line * 2 * es + x], Ef[(size_t)(line + N / 2) * 2 * es + x])
                               : make_float2(0.f, 0.f);
                }
            } else {  // PS_OTF
#pragma unroll
                for (int n = 0; n < L; ++n) {
                    const int ky = S * n + sub;
                    if (!act) v[n] = make_float2(0.f, 0.f);
                    else if (line == 0) v[n] = make_float2(E[ky * es].x, E[ky * es + N / 2].x);
                    else v[n] = E[ky * es + line];
                }
            }
            line_fft<N, -1>(v, sub);
            __syncwarp();  // every lane of the line has read it before any store
            if (ps == PS_PUPIL) {
                if (act) {
#pragma unroll
                    for (int k = 0; k < L; ++k) E[(sub * L + k) * es + line] = v[k];
                }
            } else if (ps == PS_FIELD) {
                if (act) {
#pragma unroll
                    for (int k = 0; k < L; ++k) {
                        const int kx = sub * L + k;
                        if (q.pf) q.pf[(size_t)kx * N + line] = v[k];
                        Ef[(size_t)line * 2 * es + kx] = (v[k].x * v[k].x + v[k].y * v[k].y) * q.inv_z;
                    }
                }
            } else if (ps == PS_PSF) {
                fftreg::static_for<0, L>([&](auto kk) {
                    constexpr int k = decltype(kk)::value;
                    const float2 pc = conj_partner<N, k>(v);
                    const int kx = sub * L + k;
                    if (act && kx <= N / 2) {
                        const float2 a = cscale(cadd(v[k], pc), 0.5f);
                        const float2 d = cscale(csub(v[k], pc), 0.5f);
                        E[line * es + kx] = a;
                        E[(line + N / 2) * es + kx] = make_float2(d.y, -d.x);
                    }
                });
            } else {  // PS_OTF
                const int kx = line;
                const uint64_t s0 = act ? q.csupp[2 * kx] : 0ull, s1 = act ? q.csupp[2 * kx + 1] : 0ull;
                const uint64_t n0 = act && kx == 0 ? q.csupp[N] : 0ull, n1 = act && kx == 0 ? q.csupp[N + 1] : 0ull;
                fftreg::static_for<0, L>([&](auto kk) {
                    constexpr int k = decltype(kk)::value;
                    const float2 pc = conj_partner<N, k>(v);
                    const int ky = sub * L + k;
                    if (act) {
                        if (kx > 0) {
                            q.h[ky * NH + kx] = cbit(s0, s1, ky) ? v[k] : make_float2(0.f, 0.f);
                        } else {
                            float2 h0 = cscale(cadd(v[k], pc), 0.5f);
                            const float2 d = cscale(csub(v[k], pc), 0.5f);
                            float2 hn = make_float2(d.y, -d.x);
                            if (!cbit(s0, s1, ky)) h0 = make_float2(0.f, 0.f);
                            if (!cbit(n0, n1, ky)) hn = make_float2(0.f, 0.f);
                            if (ky == 0) h0 = make_float2(1.f, 0.f);
                            q.h[ky * NH] = h0;
                            q.h[ky * NH + N / 2] = hn;
                        }
                    }
                });
            }
        }
        bar();
    }
}

// The adjoint passes (SEED, C2R, RPUPIL when RECOMPUTE, GP, ADJ) as rounds
// with one register FFT (and, for RECOMPUTE, its decimation-in-
// frequency twin in GP). E2 (row stride es2): RECOMPUTE's buffer for the
// column transforms of P. Each pass ends with the group's barrier.
template <int N, int LINES, bool RECOMPUTE, class Bar>
__device__ __forceinline__ void unit_adjoint_rounds(const UnitPtr& q, float2* E, int es, float2* E2, int es2, int t,
                                             Bar bar) {
    constexpr int S = Geo<N>::S, L = Geo<N>::L, NH = Geo<N>::NH;
    float* Ef = reinterpret_cast<float*>(E);
    const int sub = t % S, li = t / S;
    const int W = q.W;
#pragma unroll 1
    for (int ps = PS_SEED; ps <= PS_ADJ; ++ps) {
        if (!RECOMPUTE && ps == PS_RPUPIL) continue;
        const int lines = pass_lines(ps, N, W);
#pragma unroll 1
        for (int l0 = 0; l0 < lines; l0 += LINES) {
            const int line = l0 + li;
            const bool act = line < lines;
            float2 v[L];
            if (ps == PS_SEED) {
#pragma unroll
                for (int n = 0; n < L; ++n) {
                    const int ky = S * n + sub;
                    float2 g = make_float2(0.f, 0.f);
                    if (act) {
                        if (line == 0) {
                            const float2 a = q.h[ky * NH], b = q.h[ky * NH + N / 2];
                            g = make_float2(a.x - b.y, a.y + b.x);  // a + i b
                        } else {
                            g = q.h[ky * NH + line];
                        }
                    }
                    v[n] = cconj(g);
                }
            } else if (ps == PS_C2R) {
#pragma unroll
                for (int n = 0; n < L; ++n) {
                    const int x = S * n + sub, y = line;
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
            } else if (ps == PS_RPUPIL) {
                const uint64_t m0 = act ? q.cmask[2 * line] : 0ull, m1 = act ? q.cmask[2 * line + 1] : 0ull;
#pragma unroll
                for (int n = 0; n < L; ++n) {
                    const int y = S * n + sub;
                    v[n] = (act && y < W && cbit(m0, m1, y)) ? expi(q.phi[y * W + line]) : make_float2(0.f, 0.f);
                }
            } else if (ps == PS_GP) {
                if constexpr (!RECOMPUTE) {
#pragma unroll
                    for (int n = 0; n < L; ++n) {
                        const int x = S * n + sub;
                        float2 w = make_float2(0.f, 0.f);
                        if (act) {
                            const float g = Ef[(size_t)line * 2 * es + x];
                            const float2 pv = q.pf[(size_t)x * N + line];
                            w = make_float2(g * pv.x, -g * pv.y);  // conj(g_q p)
                        }
                        v[n] = w;
                    }
                } else {  // the field row from the recomputed columns, transformed below
#pragma unroll
                    for (int n = 0; n < L; ++n) {
                        const int x = S * n + sub;
                        v[n] = (act && x < W) ? E2[line * es2 + x] : make_float2(0.f, 0.f);
                    }
                }
            } else {  // PS_ADJ
#pragma unroll
                for (int n = 0; n < L; ++n) {
                    const int y = S * n + sub;
                    v[n] = act ? cconj(E[y * es + line]) : make_float2(0.f, 0.f);
                }
            }
            line_fft<N, -1>(v, sub);
            bool dif = false;
            if constexpr (RECOMPUTE) {
                if (ps == PS_GP) {
                    // conj(g_q p) on the row (blocked order kx = sub L + k), then F^H by the DIF twin
#pragma unroll
                    for (int k = 0; k < L; ++k) {
                        const int kx = sub * L + k;
                        const float g = act ? Ef[(size_t)line * 2 * es + kx] : 0.f;
                        v[k] = make_float2(g * v[k].x, -g * v[k].y);
                    }
                    line_fft_dif<N, -1>(v, sub);
                    dif = true;
                }
            }
            __syncwarp();  // every lane of the line has read it before any store
            if (ps == PS_SEED) {
                if (act) {
#pragma unroll
                    for (int k = 0; k < L; ++k)
                        E[(sub * L + k) * es + line] = cconj(v[k]);  // line 0: (T_0, T_N/2), both real
                }
            } else if (ps == PS_C2R) {
                if (act) {
                    const float sc = 2.0f * q.inv_z;
#pragma unroll
                    for (int k = 0; k < L; ++k) {
                        const int x = sub * L + k;
                        Ef[(size_t)line * 2 * es + x] = v[k].x * sc;
                        Ef[(size_t)(line + N / 2) * 2 * es + x] = -v[k].y * sc;
                    }
                }
            } else if (ps == PS_RPUPIL) {
                if (act) {
#pragma unroll
                    for (int k = 0; k < L; ++k) E2[(sub * L + k) * es2 + line] = v[k];
                }
            } else if (ps == PS_GP) {
                if (act) {
#pragma unroll
                    for (int k = 0; k < L; ++k) {
                        const int x = dif ? S * k + sub : sub * L + k;
                        if (x < W) E[line * es + x] = cconj(v[k]);
                    }
                }
            } else {  // PS_ADJ
                if (act) {
                    const uint64_t m0 = q.cmask[2 * line], m1 = q.cmask[2 * line + 1];
#pragma unroll
                    for (int k = 0; k < L; ++k) {
                        const int y = sub * L + k;
                        if (y < W) {
                            float gv = 0.f;
                            if (cbit(m0, m1, y)) {
                                const float2 pv = q.pp ? q.pp[y * W + line] : expi(q.phi[y * W + line]);
                                const float2 g = cconj(v[k]);
                                gv = 2.0f * (pv.x * g.y - pv.y * g.x);
                            }
                            q.gphi[y * W + line] = gv;
                        }
                    }
                }
            }
        }
        bar();
    }
}

// Frame reduction of one (patch, object) by one warp, any patch size: the
// residual form of Eq. 12 in FP32 with FP64 where it would cancel, Kahan sums
// per lane and an FP64 warp combine; writes the object (Eq. 11) when `obj`
// is not null and the adjoint seeds G_j = -w_j conj(O) (D_j - O H_j) over H_j.
// Returns the (patch, object) loss on every lane.
struct RedPtr {
    int N, J, spec_ld;      // spectra / object row stride: N/2 + 1 or N
    double gamma;
    const float2* d;        // frame 0 of D; frames N spec_ld apart
    float2* h;              // frame 0 of H; frames N (N/2 + 1) apart
    const float* w;         // [J] frame weights
    const uint32_t* supp;   // [N][sw] OTF support rows
    int sw;
    float2* obj = nullptr;           // [N][spec_ld] or null
    const float2* oin = nullptr;     // object-inferring loss: the given object [N][spec_ld], else null
    float2* gobj = nullptr;          // with oin: dL/dconj(O) [N][spec_ld], or null
};

// Lanes take the frequencies f0 + lane, f0 + lane + fstep, ... (fstep a
// multiple of 32: several warps can share one (patch, object)); the returned
// sum covers this warp's frequencies.
__device__ __forceinline__ double reduce_warp(const RedPtr& r, int lane, int f0 = 0, int fstep = 32) {
    const int N = r.N, NH = N / 2 + 1, half = N * NH, J = r.J;
    const size_t dstride = (size_t)N * r.spec_ld;
    const float gam = (float)r.gamma;
    KahanSum acc;
    for (int f = f0 + lane; f < half; f += fstep) {
        const int ky = f / NH, kx = f - ky * NH;
        const size_t doff = (size_t)ky * r.spec_ld + kx;
        const float2* dp = r.d + doff;
        float2* hp = r.h + f;
        const bool seed = (f != 0) && wbit(r.supp, r.sw, ky, kx);
        if (r.oin) {  // object-inferring loss: the object is given
            float2 g;
            const float t = explicit_frequency(J, dp, dstride, hp, half, r.w, r.gamma, seed, r.oin[doff], g);
            acc.add((kx == 0 || kx == N / 2) ? t : 2.0f * t);
            if (r.gobj) {
                r.gobj[doff] = g;
                if (r.spec_ld == N && kx > 0 && kx < N / 2) r.gobj[(size_t)((N - ky) % N) * N + (N - kx)] = cconj(g);
            }
            continue;
        }
        float2 num = make_float2(0.f, 0.f), o;
        float e = 0.f, qs = 0.f, tval;
#pragma unroll 4
        for (int j = 0; j < J; ++j) {
            const float2 d = dp[(size_t)j * dstride];
            const float2 h = hp[(size_t)j * half];
            const float wj = r.w[j];
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
            fp64_frequency(J, dp, dstride, hp, half, r.w, r.gamma, seed, tval, o);
        } else {
            float tsum = 0.f;
#pragma unroll 4
            for (int j = 0; j < J; ++j) {
                const float2 d = dp[(size_t)j * dstride];
                const float2 h = hp[(size_t)j * half];
                const float wj = r.w[j];
                const float2 res = csub(d, cmul(o, h));
                tsum += wj * (res.x * res.x + res.y * res.y);
                hp[(size_t)j * half] = seed ? cscale(cmul(cconj(o), res), -wj) : make_float2(0.f, 0.f);
            }
            tval = tsum + gam * (o.x * o.x + o.y * o.y);
        }
        acc.add((kx == 0 || kx == N / 2) ? tval : 2.0f * tval);
        if (r.obj) {
            r.obj[doff] = o;
            if (r.spec_ld == N && kx > 0 && kx < N / 2) r.obj[(size_t)((N - ky) % N) * N + (N - kx)] = cconj(o);
        }
    }
    double v = (double)acc.s - (double)acc.c;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

}  // namespace unitpass
}  // namespace mfbd_dev
