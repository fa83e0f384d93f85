// sm_103a fused kernel of the MOMFBD hot path (N = 64 patches).
//
// Three launches per evaluation: a forward pass kernel and an adjoint pass
// kernel in which every warp carries one frame (unit) at a time through a
// sequence of passes over its own 64 x es complex exchange buffer in shared
// memory, synchronising with __syncwarp only, and between them a
// frequency-parallel frame-reduction kernel. In every pass a lane owns one whole 64-point line in
// registers and transforms it with the single register FFT instance of the
// kernel, a radix-4 network (adjoint transforms use F^H x = conj(F conj x)).
//
// The pupil's W x W bounding box is placed at the origin of the grid: the
// PSF |F P|^2 does not depend on where the pupil sits, so every quantity
// that leaves the kernel is unchanged, and the nonzero rows and columns of
// the pupil transforms are [0, W).
//
// Forward passes (Sec. 3.1, Eqs. 20-22):
//   PUPIL  W columns: P = A exp(i phi) -> column FFT
//   FIELD  rows: p = F P (stored for the adjoint), s = |p|^2 / (N^2 n_pup)
//          (Parseval: sum |p|^2 = N^2 n_pup for a phase-only pupil); a third
//          round transforms two real rows of s packed as one complex line
//   OTF    columns: H = F s on the half spectrum (columns 0 and N/2 packed),
//          H(0) := 1, H := 0 outside the exact OTF support
// Frame reduction per object (Sec. 2.2.1, Eqs. 11-12), all warps:
//   N = sum_j w D conj(H), Q = sum_j w |H|^2 + gamma, O = N / Q,
//   t(u) = sum_j w |D - O H|^2 + gamma |O|^2 (the summand of Eq. 12 at
//   O = N/Q without its cancellation), loss summed over u in FP64,
//   G_j = dL/dconj(H_j) = -w conj(O)(D - O H) with G(0) := 0 and G := 0
//   outside the support; frequencies whose residual cancels are redone
//   in FP64.
// Adjoint passes:
//   SEED   columns: F^H along ky of G (columns 0 and N/2 packed)
//   C2R    rows: g = F^H G (two Hermitian rows packed as one line),
//          g_q = 2 g / (N^2 n_pup); then per row G_p = g_q p -> row F^H,
//          keeping the W box columns
//   ADJ    W columns: column F^H -> G_P, dL/dphi = 2 Im(conj(P) G_P)
#include "mfbd_internal.h"
#include "fft_reg.cuh"
#include "mfbd_device.cuh"
#include "pass64.cuh"

namespace mfbd_dev {

using fftreg::cadd;
using fftreg::cconj;
using fftreg::cmul;
using fftreg::cscale;
using fftreg::csub;

namespace {

using namespace pass64;

constexpr int kWarps = 6;
constexpr int kThreads = 32 * kWarps;

enum Pass : int { P_PUPIL = 0, P_FIELD = 1, P_OTF = 2, P_SEED = 3, P_C2R = 4, P_ADJ = 5, P_END = 6 };

// Per-unit pointers of the warp's current unit, kept in shared memory (one
// per warp) so they do not occupy registers across the transforms; every
// pass reads the ones it needs once.
struct Unit {
    const float* phi;  // first box pixel of the unit's phase image (row stride ld)
    float* gphi;       // same for dL/dphi
    float2* pp;        // pupil phasors exp(i phi) on the box, [W][W]
    float2* h;         // [N][N/2+1]: H (forward), then the adjoint seed G
    float2* pf;        // field p = F P, [x][y]; null: not kept
    const float2* hn;  // adjoint seed of the warp's next unit (L2 prefetch); null: none
    int W, ld;
    float inv_z;
};

__device__ __forceinline__ int pass_rounds(int pass, int W) {
    switch (pass) {
        case P_PUPIL:
        case P_ADJ: return (W + 31) >> 5;
        case P_FIELD:
        case P_C2R: return 3;
        default: return 1;
    }
}


// ------------------------------------------------------------ load stages

// Pupil column c of the box: P = exp(i phi) where the column mask `cm` has
// bit y (zero outside the pupil and for c >= W); the phasors are also kept
// for the adjoint when the unit has a phasor buffer. R >= W is the
// compile-time bound on the box side.
template <int R>
__device__ __forceinline__ void load_pupil(const volatile Unit* su, uint64_t cm, int W, int c, float2 (&v)[kN]) {
    const float* ph = (const float*)su->phi + c;
    float2* pp = (float2*)su->pp;
    const int ld = su->ld;
    float phv[R];  // every phase load of the column is issued before use
#pragma unroll
    for (int yy = 0; yy < R; ++yy) phv[yy] = (c < W && yy < W) ? ph[yy * ld] : 0.f;
#pragma unroll
    for (int yy = 0; yy < kN; ++yy) {
        if (yy < R) {
            v[yy] = bit(cm, yy) ? expi(phv[yy]) : make_float2(0.f, 0.f);
            if (pp != nullptr && c < W && yy < W) pp[yy * W + c] = v[yy];
        } else {
            v[yy] = make_float2(0.f, 0.f);
        }
    }
}

// Second PUPIL round of a box 33..40 px wide: columns 32..W-1, four lanes
// per column (lane >> 2 picks the column). (The ADJ pass keeps the generic
// second round: the quarter transform there pushes the adjoint kernel past
// its register budget.)
template <int ES>
__device__ __forceinline__ void quarter_round_pupil(const volatile Unit* su, float2* __restrict__ E,
                                                    const uint64_t* __restrict__ cmask, int W, int lane) {
    const int l = lane & 3, q = split_q(l), c = 32 + (lane >> 2);
    const bool active = c < W;
    const int ld = su->ld;
    const float* ph = (const float*)su->phi + c;
    float2* pp = (float2*)su->pp;
    const uint64_t cm = active ? cmask[c] : 0ull;
    float2 a[kN / 4];
    float phv[kN / 4];  // exp(i phi) on rows 4 n + l of column c
#pragma unroll
    for (int n = 0; n < kN / 4; ++n) phv[n] = (active && 4 * n + l < W) ? ph[(4 * n + l) * ld] : 0.f;
#pragma unroll
    for (int n = 0; n < kN / 4; ++n) {
        const int y = 4 * n + l;
        a[n] = bit(cm, y) ? expi(phv[n]) : make_float2(0.f, 0.f);
        if (pp != nullptr && active && y < W) pp[y * W + c] = a[n];
    }
    fft64_quarters(a, l);
    if (active) {
#pragma unroll
        for (int k = 0; k < kN / 4; ++k) E[(k + 16 * q) * ES + c] = a[k];
    }
}

// ----------------------------------------------------------- the machine

// Runs passes [FIRST, LAST) of one unit on the calling warp.
// Inactive warps (no unit left) only take part in the CTA barrier that ends
// every pass: the CTA's warps run the same pass at a time.
template <int FIRST, int LAST, int ES>
__device__ __forceinline__ void run_passes(const volatile Unit* su, float2* __restrict__ E,
                                           const uint64_t* __restrict__ cmask, const uint64_t* __restrict__ csupp,
                                           bool active) {
    constexpr int R = ES < kN ? ES : kN;  // the box side W is at most R
    const int lane = threadIdx.x & 31;
    const int W = active ? su->W : 0;
#pragma unroll 1
    for (int pass = FIRST; pass < LAST; ++pass) {
        const int nr = active ? pass_rounds(pass, W) : 0;
        if (FIRST >= P_SEED && lane == 0 && active) {  // L2 prefetch about one pass ahead of use
            if (pass == P_C2R && su->pp) prefetch_l2((const void*)su->pp, (size_t)W * W * sizeof(float2));
            if (pass == P_ADJ && su->hn) prefetch_l2((const void*)su->hn, (size_t)kHalf * sizeof(float2));
        }
#pragma unroll 1
        for (int r = 0; r < nr; ++r) {
            if constexpr (FIRST <= P_PUPIL && P_PUPIL < LAST) {
                if (pass == P_PUPIL && r == 1 && W <= kSplitMaxW) {
                    quarter_round_pupil<ES>(su, E, cmask, W, lane);
                    continue;
                }
            }
            float2 v[kN];
            // ------------------------------------------------------ load
            if constexpr (FIRST <= P_PUPIL && P_PUPIL < LAST) {
                if (pass == P_PUPIL) load_pupil<R>(su, cmask[lane + 32 * r], W, lane + 32 * r, v);
            }
            if constexpr (FIRST <= P_FIELD && P_FIELD < LAST) {
                if (pass == P_FIELD) {
                    if (r < 2) {  // row y of the pupil's column transform (box columns [0, W))
                        const int y = lane + 32 * r;
#pragma unroll
                        for (int x = 0; x < kN; ++x) v[x] = (x < R && x < W) ? E[y * ES + x] : make_float2(0.f, 0.f);
                    } else {  // two real PSF rows as one complex line
#pragma unroll
                        for (int i = 0; i < kN / 2; ++i) {
                            const float2 a = E[lane * ES + i], b = E[(lane + 32) * ES + i];
                            v[2 * i] = make_float2(a.x, b.x);
                            v[2 * i + 1] = make_float2(a.y, b.y);
                        }
                    }
                }
            }
            if constexpr (FIRST <= P_OTF && P_OTF < LAST) {
                if (pass == P_OTF) {  // column lane; lane 0: real columns 0 and N/2 packed
#pragma unroll
                    for (int ky = 0; ky < kN; ++ky) v[ky] = E[ky * ES + lane];
                }
            }
            if constexpr (FIRST <= P_SEED && P_SEED < LAST) {
                if (pass == P_SEED) {  // conj of column lane of G; lane 0: columns 0 and N/2 as a + i b
                    const float2* h = (const float2*)su->h;
#pragma unroll
                    for (int ky = 0; ky < kN; ++ky) {
                        const float2 a = h[ky * kNH + lane];
                        const float2 b = lane == 0 ? h[ky * kNH + 32] : make_float2(0.f, 0.f);
                        v[ky] = make_float2(a.x - b.y, -(a.y + b.x));
                    }
                }
            }
            if constexpr (FIRST <= P_C2R && P_C2R < LAST) {
                if (pass == P_C2R) {
                    if (r == 0) {  // conj of T_lane + i T_(lane+32), Hermitian-extended rows
#pragma unroll
                        for (int k = 0; k < kN; ++k) {
                            float2 a, b;
                            if (k == 0) {
                                a = make_float2(E[lane * ES].x, 0.f);
                                b = make_float2(E[(lane + 32) * ES].x, 0.f);
                            } else if (k == kN / 2) {
                                a = make_float2(E[lane * ES].y, 0.f);
                                b = make_float2(E[(lane + 32) * ES].y, 0.f);
                            } else if (k < kN / 2) {
                                a = E[lane * ES + k];
                                b = E[(lane + 32) * ES + k];
                            } else {
                                a = cconj(E[lane * ES + (kN - k)]);
                                b = cconj(E[(lane + 32) * ES + (kN - k)]);
                            }
                            v[k] = make_float2(a.x - b.y, -(a.y + b.x));
                        }
                    } else {  // conj(g_q p) of row y
                        const int y = lane + 32 * (r - 1);
                        const float2* pf = (const float2*)su->pf;
#pragma unroll
                        for (int i = 0; i < kN / 2; ++i) {
                            const float2 g = E[y * ES + i];  // g_q at x = 2i, 2i+1
                            const float2 p0 = pf[(2 * i) * kN + y], p1 = pf[(2 * i + 1) * kN + y];
                            v[2 * i] = make_float2(g.x * p0.x, -g.x * p0.y);
                            v[2 * i + 1] = make_float2(g.y * p1.x, -g.y * p1.y);
                        }
                    }
                }
            }
            if constexpr (FIRST <= P_ADJ && P_ADJ < LAST) {
                if (pass == P_ADJ) {
                    // conj of box column c; an inactive lane transforms a
                    // column that no lane overwrites in this round
                    const int c = lane + 32 * r;
                    const int cc = c < W ? c : (c < ES ? c : c - 32);
#pragma unroll
                    for (int y = 0; y < kN; ++y) v[y] = cconj(E[y * ES + cc]);
                    const float2* pp = (const float2*)su->pp;
                    if (c < W && pp != nullptr) {
                        // the column's kept phasors are copied into it while
                        // the transform runs
#pragma unroll
                        for (int yy = 0; yy < kN; ++yy)
                            if (yy < R && yy < W) cp_async8(&E[yy * ES + c], pp + yy * W + c);
                    }
                }
            }
            // --------------------------------------------------- transform
            fftreg::fft4<kN, -1>(v);
            if (pass >= P_SEED) {
#pragma unroll
                for (int i = 0; i < kN; ++i) v[i].y = -v[i].y;
            }
            // ----------------------------------------------------- store
            if constexpr (FIRST <= P_PUPIL && P_PUPIL < LAST) {
                if (pass == P_PUPIL) {
                    const int c = lane + 32 * r;
                    if (c < W) {
#pragma unroll
                        for (int ky = 0; ky < kN; ++ky) E[ky * ES + c] = v[ky];
                    }
                }
            }
            if constexpr (FIRST <= P_FIELD && P_FIELD < LAST) {
                if (pass == P_FIELD) {
                    if (r < 2) {  // keep the field row; PSF row s = |p|^2 / (N^2 n_pup) as float pairs
                        const int y = lane + 32 * r;
                        float2* pf = (float2*)su->pf;
                        if (pf) {
#pragma unroll
                            for (int x = 0; x < kN; ++x) pf[x * kN + y] = v[x];
                        }
                        const float iz = su->inv_z;
#pragma unroll
                        for (int i = 0; i < kN / 2; ++i)
                            E[y * ES + i] = make_float2((v[2 * i].x * v[2 * i].x + v[2 * i].y * v[2 * i].y) * iz,
                                                        (v[2 * i + 1].x * v[2 * i + 1].x + v[2 * i + 1].y * v[2 * i + 1].y) * iz);
                    } else {
                        // split the transform of s_lane + i s_(lane+32); the real
                        // columns kx = 0 and N/2 share slot 0 as (S[0], S[N/2])
#pragma unroll
                        for (int k = 0; k <= kN / 2; ++k) {
                            const float2 z = v[k];
                            const float2 zc = cconj(v[(kN - k) % kN]);
                            const float2 a = cscale(cadd(z, zc), 0.5f);
                            const float2 d = cscale(csub(z, zc), 0.5f);
                            const float2 b = make_float2(d.y, -d.x);
                            if (k == 0) {
                                E[lane * ES] = make_float2(a.x, 0.f);
                                E[(lane + 32) * ES] = make_float2(b.x, 0.f);
                            } else if (k == kN / 2) {
                                E[lane * ES].y = a.x;
                                E[(lane + 32) * ES].y = b.x;
                            } else {
                                E[lane * ES + k] = a;
                                E[(lane + 32) * ES + k] = b;
                            }
                        }
                    }
                }
            }
            if constexpr (FIRST <= P_OTF && P_OTF < LAST) {
                if (pass == P_OTF) {
                    // every lane writes its OTF column (lane 0 the packed
                    // Z = F(s_col0 + i s_colN/2), replaced below) and keeps a
                    // copy in shared memory for the split of column 0
                    float2* h = (float2*)su->h;
                    const uint64_t cs = lane == 0 ? ~0ull : csupp[lane];
#pragma unroll
                    for (int ky = 0; ky < kN; ++ky) {
                        h[ky * kNH + lane] = bit(cs, ky) ? v[ky] : make_float2(0.f, 0.f);
                        E[ky * ES + lane] = v[ky];
                    }
                    __syncwarp();
                    const uint64_t cs0 = csupp[0], cs32 = csupp[kN / 2];
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const int ky = lane + 32 * i;
                        const float2 z = E[ky * ES];
                        const float2 zc = cconj(E[((kN - ky) & (kN - 1)) * ES]);
                        float2 h0 = cscale(cadd(z, zc), 0.5f);
                        const float2 d = cscale(csub(z, zc), 0.5f);
                        float2 h32 = make_float2(d.y, -d.x);
                        if (!bit(cs0, ky)) h0 = make_float2(0.f, 0.f);
                        if (!bit(cs32, ky)) h32 = make_float2(0.f, 0.f);
                        if (ky == 0) h0 = make_float2(1.f, 0.f);
                        h[ky * kNH] = h0;
                        h[ky * kNH + 32] = h32;
                    }
                }
            }
            if constexpr (FIRST <= P_SEED && P_SEED < LAST) {
                if (pass == P_SEED) {  // lane 0 keeps (T_0, T_N/2), both real, packed
#pragma unroll
                    for (int y = 0; y < kN; ++y) E[y * ES + lane] = v[y];
                }
            }
            if constexpr (FIRST <= P_C2R && P_C2R < LAST) {
                if (pass == P_C2R) {
                    if (r == 0) {  // g_q rows lane and lane+32 as float pairs
                        const float sc = 2.0f * su->inv_z;
#pragma unroll
                        for (int i = 0; i < kN / 2; ++i) {
                            E[lane * ES + i] = make_float2(v[2 * i].x * sc, v[2 * i + 1].x * sc);
                            E[(lane + 32) * ES + i] = make_float2(v[2 * i].y * sc, v[2 * i + 1].y * sc);
                        }
                    } else {  // box columns of the row's F^H
                        const int y = lane + 32 * (r - 1);
#pragma unroll
                        for (int x = 0; x < kN; ++x)
                            if (x < R && x < W) E[y * ES + x] = v[x];
                    }
                }
            }
            if constexpr (FIRST <= P_ADJ && P_ADJ < LAST) {
                if (pass == P_ADJ) {  // dL/dphi = 2 Im(conj(P) G_P) on the pupil
                    const int c = lane + 32 * r;
                    if (c < W) {
                        float* gph = (float*)su->gphi + c;
                        const int ld = su->ld;
                        const uint64_t cm = cmask[c];
                        cp_async_wait();
                        if (su->pp) {
#pragma unroll
                            for (int yy = 0; yy < kN; ++yy) {
                                if (yy < R && yy < W) {
                                    const float2 pv = E[yy * ES + c];
                                    gph[yy * ld] = bit(cm, yy) ? 2.0f * fmaf(pv.x, v[yy].y, -(pv.y * v[yy].x)) : 0.f;
                                }
                            }
                        } else {  // no phasor buffer: G_P parked, phasors from the phase (compact loop)
#pragma unroll
                            for (int yy = 0; yy < kN; ++yy)
                                if (yy < R && yy < W) E[yy * ES + c] = v[yy];
                            const float* ph = (const float*)su->phi + c;
#pragma unroll 4
                            for (int yy = 0; yy < W; ++yy) {
                                const float2 pv = expi(ph[yy * ld]);
                                const float2 g = E[yy * ES + c];
                                gph[yy * ld] = bit(cm, yy) ? 2.0f * fmaf(pv.x, g.y, -(pv.y * g.x)) : 0.f;
                            }
                        }
                    }
                }
            }
        }
        __syncwarp();
        __syncthreads();
    }
}

// Frame reduction of one (patch, object) by one warp (reduce_frequencies,
// pass64.cuh); the warp combines its lanes' sums in FP64. Valid in lane 0.
template <int JM>
__device__ double reduce_object_warp(const FusedParams& prm, int p, int k, int f0, int fstep) {
    const int lane = threadIdx.x & 31;
    float2* hbase = prm.gscr + ((size_t)p * prm.K + k) * prm.J * kHalf;
    double v = reduce_frequencies<JM>(prm, p, k, hbase, f0 + lane, fstep);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}

// One warp per unit (patch, object, frame), persistent over the units;
// FIRST..LAST selects the forward (PUPIL, FIELD, OTF) or adjoint (SEED,
// C2R, ADJ) passes. A CTA barrier ends every pass, so the CTA's warps run
// the same pass's code at a time.
template <int FIRST, int LAST, int ES>
__global__ void __launch_bounds__(kThreads, 2) mfbd_pass_kernel(const FusedParams prm) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Unit sunit[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    float2* E = reinterpret_cast<float2*>(smem) + (size_t)warp * kN * ES;
    volatile Unit* su = &sunit[warp];
    const int J = prm.J, K = prm.K;
    const long long units = (long long)prm.P * K * J;
    const long long stride = (long long)gridDim.x * nwarps;
    // a uniform trip count over the CTA (the passes end in CTA barriers)
    for (long long base = (long long)blockIdx.x * nwarps; base < units; base += stride) {
        const long long u = base + warp;
        const bool active = u < units;
        const long long ua = active ? u : 0;
        const int j = (int)(ua % J);
        const long long pk = ua / J;
        const int k = (int)(pk % K);
        const long long p = pk / K;
        const ObjParams& ob = prm.obj[k];
        const long long pj = p * J + j;  // index of the unit's phase image
        __syncwarp();
        if (lane == 0 && active) {
            su->W = ob.W;
            su->ld = ob.phi_ld;
            su->inv_z = ob.inv_z;
            su->phi = prm.phi + ob.phi_off + pj * ob.phi_unit + ob.phi_org;
            su->gphi = FIRST >= P_SEED ? prm.gphi + ob.phi_off + pj * ob.phi_unit + ob.phi_org : nullptr;
            su->h = prm.gscr + (size_t)u * kHalf;
            su->pf = prm.pscr ? prm.pscr + (size_t)u * kN * kN : nullptr;
            su->pp = prm.uscr ? prm.uscr + (size_t)u * prm.ustride : nullptr;
            su->hn = FIRST == P_SEED && u + stride < units ? prm.gscr + (size_t)(u + stride) * kHalf : nullptr;
            if (FIRST == P_SEED && prm.pscr)  // this unit's field, used from the second C2R round on
                prefetch_l2(prm.pscr + (size_t)u * kN * kN, (size_t)kN * kN * sizeof(float2));
            if (FIRST == P_PUPIL && u + stride < units) {  // next unit's phase into L2
                const long long un = u + stride;
                const int jn = (int)(un % J), kn = (int)((un / J) % K);
                const long long pn = un / J / K;
                const ObjParams& on = prm.obj[kn];
                prefetch_l2(prm.phi + on.phi_off + (pn * J + jn) * on.phi_unit + on.phi_org,
                            ((size_t)(on.W - 1) * on.phi_ld + on.W) * 4);
            }
        }
        __syncwarp();
        run_passes<FIRST, LAST, ES>(su, E, ob.cmask, ob.csupp, active);
    }
}

// Frame reduction: one CTA per (patch, split), warp k reduces the split's
// frequencies of object k (32-wide blocks s, s + S, s + 2S, ...); the CTA
// sums the objects in order, and with S > 1 a second kernel sums the splits
// in order (deterministic for a given S).
template <int JM>
__global__ void __launch_bounds__(32 * kMaxObjects) mfbd_reduce_kernel(const FusedParams prm) {
    __shared__ double sobj[kMaxObjects];
    const int k = threadIdx.x >> 5;
    const int S = (prm.rsplit > 1 && prm.lpart) ? prm.rsplit : 1;
    const long long work = (long long)prm.P * S;
    for (long long u = blockIdx.x; u < work; u += gridDim.x) {
        const int p = (int)(u / S), sp = (int)(u - (long long)p * S);
        const double v = reduce_object_warp<JM>(prm, p, k, 32 * sp, 32 * S);
        if ((threadIdx.x & 31) == 0) sobj[k] = v;
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

}  // namespace

FusedGeometry fused_geometry(int max_box) {
    FusedGeometry g;
    // exchange-buffer row strides compiled in (odd, >= N/2 + 1)
    g.xs = max_box <= 33 ? 33 : max_box <= 37 ? 37 : max_box <= 45 ? 45 : 65;
    // up to kWarps warps, two CTAs per SM when their buffers fit in 227 KB
    const size_t per_warp = (size_t)kN * g.xs * sizeof(float2);
    int warps = (int)(((size_t)113 * 1024) / per_warp);
    if (warps < 1) warps = 1;
    g.slots = warps < kWarps ? warps : kWarps;
    g.smem_bytes = (size_t)g.slots * per_warp;
    return g;
}

template <int FIRST, int LAST>
cudaError_t launch_pass(const FusedParams& prm, const FusedGeometry& g, int sms, cudaStream_t s) {
    auto* kern = g.xs == 33 ? mfbd_pass_kernel<FIRST, LAST, 33>
                 : g.xs == 37 ? mfbd_pass_kernel<FIRST, LAST, 37>
                 : g.xs == 45 ? mfbd_pass_kernel<FIRST, LAST, 45>
                              : mfbd_pass_kernel<FIRST, LAST, 65>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem_bytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, g.slots * 32, g.smem_bytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long units = (long long)prm.P * prm.K * prm.J;
    long long ctas = (long long)sms * per_sm;
    const long long need = (units + g.slots - 1) / g.slots;
    if (ctas > need) ctas = need;
    kern<<<(int)ctas, g.slots * 32, g.smem_bytes, s>>>(prm);
    return cudaGetLastError();
}

template <int JM>
cudaError_t launch_reduction_jm(const FusedParams& prm, int sms, cudaStream_t s) {
    const int threads = 32 * prm.K;
    const int S = (prm.rsplit > 1 && prm.lpart) ? prm.rsplit : 1;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mfbd_reduce_kernel<JM>, threads, 0);
    if (e != cudaSuccess) return e;
    long long ctas = (long long)sms * (per_sm > 0 ? per_sm : 1);
    if (ctas > (long long)prm.P * S) ctas = (long long)prm.P * S;
    mfbd_reduce_kernel<JM><<<(int)ctas, threads, 0, s>>>(prm);
    if ((e = cudaGetLastError()) != cudaSuccess || S == 1) return e;
    return launch_loss_combine(prm.lpart, S, prm.loss, prm.P, s);
}

cudaError_t launch_reduction(const FusedParams& prm, int sms, cudaStream_t s) {
    if (prm.P == 0) return cudaSuccess;
    return prm.J <= 16 ? launch_reduction_jm<16>(prm, sms, s) : launch_reduction_jm<0>(prm, sms, s);
}

cudaError_t launch_forward_passes(const FusedParams& prm, const FusedGeometry& g, int sms, cudaStream_t s) {
    if (prm.P == 0) return cudaSuccess;
    return launch_pass<P_PUPIL, P_OTF + 1>(prm, g, sms, s);
}

cudaError_t launch_adjoint_passes(const FusedParams& prm, const FusedGeometry& g, int sms, cudaStream_t s) {
    if (prm.P == 0) return cudaSuccess;
    return launch_pass<P_SEED, P_END>(prm, g, sms, s);
}

int max_ctas_per_sm(const FusedGeometry& g) {
    auto* kern = g.xs == 33 ? mfbd_pass_kernel<P_PUPIL, P_OTF + 1, 33>
                 : g.xs == 37 ? mfbd_pass_kernel<P_PUPIL, P_OTF + 1, 37>
                 : g.xs == 45 ? mfbd_pass_kernel<P_PUPIL, P_OTF + 1, 45>
                              : mfbd_pass_kernel<P_PUPIL, P_OTF + 1, 65>;
    int n = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem_bytes) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, g.slots * 32, g.smem_bytes) != cudaSuccess)
        return 0;
    return n;
}

// mode FWD: forward passes + reduction; BWD: adjoint passes; FUSED: all
// three launches; OTF: forward passes only. `sms` is the SM count.
cudaError_t launch_fused(const FusedParams& prm, int mode, const FusedGeometry& g, int sms, cudaStream_t s) {
    if (prm.P == 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (mode != MODE_BWD) {
        e = launch_forward_passes(prm, g, sms, s);
        if (e != cudaSuccess || mode == MODE_OTF) return e;
        e = launch_reduction(prm, sms, s);
        if (e != cudaSuccess || mode == MODE_FWD) return e;
    }
    return launch_adjoint_passes(prm, g, sms, s);
}

}  // namespace mfbd_dev
