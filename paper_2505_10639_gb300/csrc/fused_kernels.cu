// Fused evaluation of the MOMFBD loss and gradient for 64 px patches: one
// persistent kernel in which a CTA carries one (patch, object) pair at a
// time through the whole chain of Sec. 3.1 (Eqs. 20-22), the frame
// reduction of Sec. 2.2.1 (Eqs. 11-12) and the adjoint of both, so that
// nothing but the inputs (phases, spectra) and the outputs (loss, object,
// dL/dphi) crosses HBM.
//
// A CTA has 12 warps, one per frame of the pair (J <= 12), and holds one
// 64 x ES complex exchange buffer per warp in shared memory (227 KB at
// ES = 37). Per pair:
//   forward passes, each warp on its frame (one register FFT instance):
//     PUPIL  W columns: P = A exp(i phi) -> column FFT
//     FIELD  rows: p = F P (kept for the adjoint: rows 0..31 in the
//            warp's tensor-memory columns, rows 32..63 in the frame's slot
//            of a global buffer of 12 x 16 KB per CTA that stays in L2, x
//            pairs of a row as one 16-byte access),
//            s = |p|^2 / (N^2 n_pup); two real PSF rows per complex line
//     OTF    columns: H = F s (half spectrum, columns 0 and N/2 packed),
//            written into shared memory over the exchange buffers: the
//            J OTFs of the pair, [J][N][N/2+1]
//   frame reduction by all 384 threads, each on a set of frequencies with
//     the J frames of each in registers: N, Q, O = N / Q, the loss term and
//     the adjoint seeds G_j = -w conj(O)(D_j - O H_j) written over H_j
//     (reduce_frequencies, the arithmetic of the three-kernel path)
//   adjoint passes, each warp on its frame:
//     SEED   columns of G_j from shared memory -> F^H along ky
//     C2R    rows: g_q = 2 Re F^H G / (N^2 n_pup); G_p = g_q p with the
//            field from the frame's slot -> row F^H
//     ADJ    W columns: column F^H -> G_P; dL/dphi = 2 Im(conj(P) G_P) with
//            P = exp(i phi) recomputed from the phase, which is copied into
//            the column's shared-memory slots while the transform runs
// CTA barriers stand only where the data cross warps: after the OTF pass (the
// reduction reads every frame's OTF) and after the reduction (every seed is
// written); the named barrier of the frame warps orders the OTF and SEED
// passes against the exchange buffers they overlap.
// The pair's loss (the threads' Kahan sums, combined in a fixed order) goes
// to lpair[p][k]; the CTA that completes a patch's last object (a per-patch
// counter, reset after use) sums its objects' losses in object order.
#include "mfbd_internal.h"
#include "fft_reg.cuh"
#include "mfbd_device.cuh"
#include "pass64.cuh"

namespace mfbd_dev {

namespace {

using namespace pass64;

constexpr int kFW = kFusedFrames;  // warps per CTA: the frames of a pair in flight
constexpr int kFT = 32 * kFW;

enum FusedPass : int { F_PUPIL = 0, F_FIELD = 1, F_OTF = 2, F_SEED = 3, F_C2R = 4, F_ADJ = 5, F_END = 6 };

// Per-warp pointers of the frame it carries, kept in shared memory so that
// they occupy no registers across the transforms.
struct FrameSlot {
    const float* phi;  // first box pixel of the frame's phase image (row stride phi_ld)
    float* gphi;       // same for dL/dphi
};

__device__ __forceinline__ int fused_rounds(int pass, int W) {
    switch (pass) {
        case F_PUPIL:
        case F_ADJ: return (W + 31) >> 5;
        case F_FIELD:
        case F_C2R: return 3;
        default: return 1;
    }
}

// Barrier of the warps that carry a frame (named barrier 1): the OTF and
// SEED passes move data between the exchange buffers and the OTF area,
// which overlap.
__device__ __forceinline__ void frames_barrier(int nthreads) {
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Tensor memory as a store for half of each frame's field: warp w owns the
// TMEM lanes of its quarter (32 (w mod 4) ..) and 128 columns (w / 4) * 128 ..
// of them, one lane per field row. tmem_st32 / tmem_ld32 move 32 consecutive
// 32-bit columns of the calling thread's lane.
constexpr uint32_t kTmemCols = 512;

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float (&v)[32]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]), "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]), "f"(v[16]), "f"(v[17]), "f"(v[18]), "f"(v[19]), "f"(v[20]), "f"(v[21]), "f"(v[22]), "f"(v[23]), "f"(v[24]), "f"(v[25]), "f"(v[26]), "f"(v[27]), "f"(v[28]), "f"(v[29]), "f"(v[30]), "f"(v[31])
                 : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]), "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15]), "=f"(v[16]), "=f"(v[17]), "=f"(v[18]), "=f"(v[19]), "=f"(v[20]), "=f"(v[21]), "=f"(v[22]), "=f"(v[23]), "=f"(v[24]), "=f"(v[25]), "=f"(v[26]), "=f"(v[27]), "=f"(v[28]), "=f"(v[29]), "=f"(v[30]), "=f"(v[31])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 4-byte asynchronous global -> shared copy.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(__cvta_generic_to_global(gmem))
                 : "memory");
}

// Pupil column c of the box: P = exp(i phi) where the column mask has bit y.
template <int R>
__device__ __forceinline__ void fused_load_pupil(const float* ph, int ld, uint64_t cm, int W, int c,
                                                 float2 (&v)[kN]) {
    float phv[R];  // every phase load of the column is issued before use
#pragma unroll
    for (int yy = 0; yy < R; ++yy) phv[yy] = (c < W && yy < W) ? ph[yy * ld + c] : 0.f;
#pragma unroll
    for (int yy = 0; yy < kN; ++yy) v[yy] = (yy < R && bit(cm, yy)) ? expi(phv[yy]) : make_float2(0.f, 0.f);
}

// Second PUPIL round of a box 33..40 px wide: columns 32..W-1, four lanes
// per column (fft64_quarters). Out of line: the pass loop's code stays
// smaller (the kernel's instruction fetch is one of its stalls; measured
// 1 % faster than inlined).
template <int ES>
__device__ __noinline__ void fused_quarter_pupil(const float* ph, int ld, float2* __restrict__ E,
                                                    const uint64_t* __restrict__ cmask, int W, int lane) {
    const int l = lane & 3, q = split_q(l), c = 32 + (lane >> 2);
    const bool active = c < W;
    const uint64_t cm = active ? cmask[c] : 0ull;
    float2 a[kN / 4];
    float phv[kN / 4];
#pragma unroll
    for (int n = 0; n < kN / 4; ++n) phv[n] = (active && 4 * n + l < W) ? ph[(4 * n + l) * ld + c] : 0.f;
#pragma unroll
    for (int n = 0; n < kN / 4; ++n) a[n] = bit(cm, 4 * n + l) ? expi(phv[n]) : make_float2(0.f, 0.f);
    fft64_quarters(a, l);
    if (active) {
#pragma unroll
        for (int k = 0; k < kN / 4; ++k) E[(k + 16 * q) * ES + c] = a[k];
    }
}

// EXPL: the object-inferring loss (the objects given), else the Wiener loss.
template <int ES, bool EXPL>
__global__ void __launch_bounds__(kFT, 1) fused_pair_kernel(const FusedParams prm) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ FrameSlot slot[kFW];
    __shared__ double swarp[kFW];
    __shared__ uint32_t s_tmem;
    constexpr int R = ES < kN ? ES : kN;  // the box side W is at most R
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* const E = reinterpret_cast<float2*>(smem) + (size_t)warp * kN * ES;
    float2* const HA = reinterpret_cast<float2*>(smem);  // [J][N][N/2+1]: OTFs, then seeds
    // the frame's field: rows 0 .. N/2-1 in the warp's tensor-memory columns
    // (x pairs as 32-bit columns re, im), rows N/2 .. N-1 in its global slot,
    // [x / 2][y - N/2] pairs (p[y][x], p[y][x + 1]), one 16-byte access per
    // pair (recomputed where used rather than held in registers)
    auto field_slot = [&]() {
        return reinterpret_cast<float4*>(prm.fscr) +
               ((size_t)blockIdx.x * kFW + (threadIdx.x >> 5)) * (kN / 2) * (kN / 2);
    };
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (unsigned)__cvta_generic_to_shared(&s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem_base = s_tmem;
    auto tmem_row = [&]() {  // this lane's row of the warp's columns
        return tmem_base + ((uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16) + (uint32_t)((threadIdx.x >> 7) * 128);
    };
    const int J = prm.J, K = prm.K;
    const long long P = prm.P, pairs = P * K;
    const bool active = warp < J;
    const int nframe_threads = 32 * (J < kFW ? J : kFW);
    const size_t dstride = (size_t)kN * prm.spec_ld;
    // Pairs in object order prm.korder (widest pupil box first, the costliest
    // pairs first), patch by patch. A CTA starts on pair blockIdx.x and takes
    // each next pair from a ticket counter when it starts the current one
    // (longest-first greedy dealing); the ticket goes through shared memory,
    // two slots used in turn, and is read after the CTA barrier that follows
    // the OTF pass.
    __shared__ long long s_next[2];
    int par = 0;
    for (long long i = blockIdx.x; i < pairs; par ^= 1) {
        if (threadIdx.x == 0) s_next[par] = (long long)gridDim.x + atomicAdd(prm.fticket, 1);
        const int k = prm.korder[(int)(i / P)];
        const long long p = i % P;
        const ObjParams& ob = prm.obj[k];
        const int W = ob.W;
        long long next = pairs;
        if (lane == 0 && active) {
            const long long img = (p * J + warp) * ob.phi_unit + ob.phi_org;
            slot[warp].phi = prm.phi + ob.phi_off + img;
            slot[warp].gphi = prm.gphi + ob.phi_off + img;
            // this frame's spectrum into L2 for the reduction
            prefetch_l2_hint(prm.spectra + (((size_t)p * K + k) * J + warp) * dstride, dstride * sizeof(float2),
                             l2_evict_first());
        }
        __syncwarp();
#pragma unroll 1
        for (int pass = F_PUPIL; pass < F_END; ++pass) {
            if (pass == F_SEED) {
                // frame reduction over the J OTFs in shared memory (every
                // OTF pass ended in the CTA barrier below)
                double v = reduce_frequencies<kFW, EXPL ? 2 : 1, true>(prm, (int)p, k, HA, threadIdx.x, kFT);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
                if (lane == 0) swarp[warp] = v;
                __syncthreads();
                if (threadIdx.x == 0) {
                    double tot = 0.0;
                    for (int w = 0; w < kFW; ++w) tot += swarp[w];
                    prm.lpair[p * K + k] = tot;
                    // the CTA that finishes the patch's last object sums the
                    // objects' losses in object order and resets the count
                    __threadfence();
                    if (atomicAdd(&prm.lcnt[p], 1) == K - 1) {
                        __threadfence();
                        double sum = 0.0;
                        for (int kk = 0; kk < K; ++kk) sum += __ldcg(&prm.lpair[p * K + kk]);
                        prm.loss[p] = sum;
                        prm.lcnt[p] = 0;
                    }
                }
            }
            const int nr = active ? fused_rounds(pass, W) : 0;
#pragma unroll 1
            for (int r = 0; r < nr; ++r) {
                if (pass == F_PUPIL && r == 1 && W <= kSplitMaxW) {
                    fused_quarter_pupil<ES>(slot[warp].phi, ob.phi_ld, E, ob.cmask, W, lane);
                    continue;
                }
                float2 v[kN];
                // ------------------------------------------------------ load
                if (pass == F_PUPIL) {
                    const int c = lane + 32 * r;
                    fused_load_pupil<R>(slot[warp].phi, ob.phi_ld, ob.cmask[c], W, c, v);
                } else if (pass == F_FIELD) {
                    if (r < 2) {  // row y of the pupil's column transform (box columns [0, W))
                        const int y = lane + 32 * r;
#pragma unroll
                        for (int x = 0; x < kN; ++x) v[x] = (x < R && x < W) ? E[y * ES + x] : make_float2(0.f, 0.f);
                    } else {  // two real PSF rows as one complex line
#pragma unroll
                        for (int i2 = 0; i2 < kN / 2; ++i2) {
                            const float2 a = E[lane * ES + i2], b = E[(lane + 32) * ES + i2];
                            v[2 * i2] = make_float2(a.x, b.x);
                            v[2 * i2 + 1] = make_float2(a.y, b.y);
                        }
                    }
                } else if (pass == F_OTF) {  // column lane; lane 0: real columns 0 and N/2 packed
#pragma unroll
                    for (int ky = 0; ky < kN; ++ky) v[ky] = E[ky * ES + lane];
                } else if (pass == F_SEED) {  // conj of column lane of G; lane 0: columns 0 and N/2 as a + i b
                    const float2* g = HA + (size_t)warp * kHalf;
#pragma unroll
                    for (int ky = 0; ky < kN; ++ky) {
                        const float2 a = g[ky * kNH + lane];
                        const float2 b = lane == 0 ? g[ky * kNH + 32] : make_float2(0.f, 0.f);
                        v[ky] = make_float2(a.x - b.y, -(a.y + b.x));
                    }
                } else if (pass == F_C2R) {
                    if (r == 0) {
                        // conj of T_lane + i T_(lane+32), Hermitian-extended
                        // rows; the buffer holds conj(T) (the SEED pass stores
                        // its transform unconjugated)
#pragma unroll
                        for (int kk = 0; kk < kN; ++kk) {
                            if (kk == 0) {
                                v[kk] = make_float2(E[lane * ES].x, -E[(lane + 32) * ES].x);
                            } else if (kk == kN / 2) {
                                v[kk] = make_float2(-E[lane * ES].y, E[(lane + 32) * ES].y);
                            } else if (kk < kN / 2) {
                                const float2 a = E[lane * ES + kk], b = E[(lane + 32) * ES + kk];
                                v[kk] = make_float2(a.x + b.y, a.y - b.x);
                            } else {
                                const float2 a = E[lane * ES + (kN - kk)], b = E[(lane + 32) * ES + (kN - kk)];
                                v[kk] = make_float2(a.x - b.y, -(a.y + b.x));
                            }
                        }
                    } else if (r == 1) {  // conj(g_q p) of row y = lane, p from tensor memory
                        const int y = lane;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            float t[32];
                            tmem_ld32(tmem_row() + 32 * q, t);
                            tmem_wait_ld();
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                const int i2 = 8 * q + i;
                                const float2 g = E[y * ES + i2];  // g_q at x = 2 i2, 2 i2 + 1
                                v[2 * i2] = make_float2(g.x * t[4 * i], -g.x * t[4 * i + 1]);
                                v[2 * i2 + 1] = make_float2(g.y * t[4 * i + 2], -g.y * t[4 * i + 3]);
                            }
                        }
                    } else {  // conj(g_q p) of row y = lane + N/2, p from the global slot
                        const int y = lane + 32;
                        const uint64_t keep = l2_evict_last();  // the slot is written again by the next pair
                        const float4* pf = field_slot();
#pragma unroll
                        for (int i2 = 0; i2 < kN / 2; ++i2) {
                            const float2 g = E[y * ES + i2];  // g_q at x = 2 i2, 2 i2 + 1
                            const float4 pp = ld_hint(pf + i2 * (kN / 2) + lane, keep);  // p at x = 2 i2, 2 i2 + 1
                            v[2 * i2] = make_float2(g.x * pp.x, -g.x * pp.y);
                            v[2 * i2 + 1] = make_float2(g.y * pp.z, -g.y * pp.w);
                        }
                    }
                } else {  // F_ADJ: conj of box column c (the C2R pass left conj(G_P) in the
                          // buffer); an inactive lane transforms a column no lane writes
                    const int c = lane + 32 * r;
                    const int cc = c < W ? c : (c < ES ? c : c - 32);
#pragma unroll
                    for (int y = 0; y < kN; ++y) v[y] = E[y * ES + cc];
                    if (c < W) {  // the column's phases are copied into it while the transform runs
                        const float* ph = slot[warp].phi + c;
#pragma unroll
                        for (int yy = 0; yy < kN; ++yy)
                            if (yy < R && yy < W) cp_async4(&E[yy * ES + c], ph + yy * ob.phi_ld);
                    }
                }
                // --------------------------------------------------- transform
                // adjoint passes: F^H x = conj(F conj x); the loads above
                // conjugate, and the outer conjugation is left to the next
                // consumer (the stores below keep the transform as it is)
                fftreg::fft4<kN, -1>(v);
                // ----------------------------------------------------- store
                if (pass == F_PUPIL) {
                    const int c = lane + 32 * r;
                    if (c < W) {
#pragma unroll
                        for (int ky = 0; ky < kN; ++ky) E[ky * ES + c] = v[ky];
                    }
                } else if (pass == F_FIELD) {
                    if (r < 2) {  // keep the field row; PSF row s = |p|^2 / (N^2 n_pup) as float pairs
                        const int y = lane + 32 * r;
                        if (r == 0) {  // rows 0 .. N/2-1 into tensor memory
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                float t[32];
#pragma unroll
                                for (int i = 0; i < 16; ++i) {
                                    t[2 * i] = v[16 * q + i].x;
                                    t[2 * i + 1] = v[16 * q + i].y;
                                }
                                tmem_st32(tmem_row() + 32 * q, t);
                            }
                            tmem_wait_st();
                        } else {  // rows N/2 .. N-1 into the global slot, kept in L2 until C2R
                            const uint64_t keep = l2_evict_last();
                            float4* pf = field_slot();
#pragma unroll
                            for (int i2 = 0; i2 < kN / 2; ++i2)
                                st_hint(pf + i2 * (kN / 2) + lane,
                                        make_float4(v[2 * i2].x, v[2 * i2].y, v[2 * i2 + 1].x, v[2 * i2 + 1].y), keep);
                        }
                        const float iz = ob.inv_z;
#pragma unroll
                        for (int i2 = 0; i2 < kN / 2; ++i2)
                            E[y * ES + i2] = make_float2((v[2 * i2].x * v[2 * i2].x + v[2 * i2].y * v[2 * i2].y) * iz,
                                                         (v[2 * i2 + 1].x * v[2 * i2 + 1].x +
                                                          v[2 * i2 + 1].y * v[2 * i2 + 1].y) * iz);
                    } else {
                        // split the transform of s_lane + i s_(lane+32); the real
                        // columns kx = 0 and N/2 share slot 0 as (S[0], S[N/2])
#pragma unroll
                        for (int kk = 0; kk <= kN / 2; ++kk) {
                            const float2 z = v[kk];
                            const float2 zc = cconj(v[(kN - kk) % kN]);
                            const float2 a = cscale(cadd(z, zc), 0.5f);
                            const float2 d = cscale(csub(z, zc), 0.5f);
                            const float2 b = make_float2(d.y, -d.x);
                            if (kk == 0) {
                                E[lane * ES] = make_float2(a.x, 0.f);
                                E[(lane + 32) * ES] = make_float2(b.x, 0.f);
                            } else if (kk == kN / 2) {
                                E[lane * ES].y = a.x;
                                E[(lane + 32) * ES].y = b.x;
                            } else {
                                E[lane * ES + kk] = a;
                                E[(lane + 32) * ES + kk] = b;
                            }
                        }
                    }
                } else if (pass == F_OTF) {
                    // every frame warp has read its buffer: the OTF area over
                    // the buffers is free. Column lane (lane 0: the packed
                    // Z = F(s_col0 + i s_colN/2)), masked by the support.
                    frames_barrier(nframe_threads);
                    float2* h = HA + (size_t)warp * kHalf;
                    const uint64_t cs = lane == 0 ? ~0ull : ob.csupp[lane];
#pragma unroll
                    for (int ky = 0; ky < kN; ++ky) h[ky * kNH + lane] = bit(cs, ky) ? v[ky] : make_float2(0.f, 0.f);
                    __syncwarp();
                    const uint64_t cs0 = ob.csupp[0], cs32 = ob.csupp[kN / 2];
                    float2 h0[2], h32[2];
#pragma unroll
                    for (int i2 = 0; i2 < 2; ++i2) {
                        const int ky = lane + 32 * i2;
                        const float2 z = h[ky * kNH];
                        const float2 zc = cconj(h[((kN - ky) & (kN - 1)) * kNH]);
                        h0[i2] = cscale(cadd(z, zc), 0.5f);
                        const float2 d = cscale(csub(z, zc), 0.5f);
                        h32[i2] = make_float2(d.y, -d.x);
                        if (!bit(cs0, ky)) h0[i2] = make_float2(0.f, 0.f);
                        if (!bit(cs32, ky)) h32[i2] = make_float2(0.f, 0.f);
                        if (ky == 0) h0[i2] = make_float2(1.f, 0.f);
                    }
                    __syncwarp();
#pragma unroll
                    for (int i2 = 0; i2 < 2; ++i2) {
                        const int ky = lane + 32 * i2;
                        h[ky * kNH] = h0[i2];
                        h[ky * kNH + 32] = h32[i2];
                    }
                } else if (pass == F_SEED) {
                    // every frame warp has read its seed: the buffers over
                    // the seed area are free again. conj(T) (lane 0: of
                    // T_0 + i T_N/2)
                    frames_barrier(nframe_threads);
#pragma unroll
                    for (int y = 0; y < kN; ++y) E[y * ES + lane] = v[y];
                } else if (pass == F_C2R) {
                    if (r == 0) {  // g_q rows lane and lane+32 (the real and imaginary parts of conj v)
                        const float sc = 2.0f * ob.inv_z;
#pragma unroll
                        for (int i2 = 0; i2 < kN / 2; ++i2) {
                            E[lane * ES + i2] = make_float2(v[2 * i2].x * sc, v[2 * i2 + 1].x * sc);
                            E[(lane + 32) * ES + i2] = make_float2(v[2 * i2].y * -sc, v[2 * i2 + 1].y * -sc);
                        }
                    } else {  // box columns of the row's conj(F^H)
                        const int y = lane + 32 * (r - 1);
#pragma unroll
                        for (int x = 0; x < kN; ++x)
                            if (x < R && x < W) E[y * ES + x] = v[x];
                    }
                } else {  // F_ADJ: dL/dphi = 2 Im(conj(P) G_P) on the pupil, P = exp(i phi), G_P = conj(v)
                    const int c = lane + 32 * r;
                    if (c < W) {
                        float* gph = slot[warp].gphi + c;
                        const uint64_t cm = ob.cmask[c];
                        const uint64_t stream = l2_evict_first();  // read once, by the modal adjoint
                        cp_async_wait();
#pragma unroll
                        for (int yy = 0; yy < kN; ++yy) {
                            if (yy < R && yy < W) {
                                const float2 pv = expi(E[yy * ES + c].x);
                                st_hint(gph + yy * ob.phi_ld,
                                        bit(cm, yy) ? 2.0f * fmaf(pv.x, -v[yy].y, -(pv.y * v[yy].x)) : 0.f, stream);
                            }
                        }
                    }
                }
            }
            // the reduction needs every frame's OTF; the other passes work on
            // the warp's own buffer
            __syncwarp();
            if (pass == F_OTF) {
                __syncthreads();
                // the next pair (its ticket is visible after the barrier), and
                // its phase into L2 for its PUPIL pass
                next = s_next[par];
                if (lane == 0 && active && next < pairs) {
                    const int kn = prm.korder[(int)(next / P)];
                    const long long pn = next % P;
                    const ObjParams& on = prm.obj[kn];
                    prefetch_l2(prm.phi + on.phi_off + (pn * J + warp) * on.phi_unit + on.phi_org,
                                ((size_t)(on.W - 1) * on.phi_ld + on.W) * sizeof(float));
                }
            }
        }
        i = next;
    }
    // the last CTA out resets the counters for the next launch
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(prm.fticket + 1, 1) == (int)gridDim.x - 1) {
            prm.fticket[0] = 0;
            prm.fticket[1] = 0;
            __threadfence();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols));
}

template <int ES, bool EXPL>
cudaError_t launch_pairs_es(const FusedParams& prm, int ctas, cudaStream_t s) {
    const size_t smem = fused_pair_smem(ES);
    cudaError_t e = cudaFuncSetAttribute(fused_pair_kernel<ES, EXPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    fused_pair_kernel<ES, EXPL><<<ctas, kFT, smem, s>>>(prm);
    return cudaGetLastError();
}

template <int ES>
int pair_ctas_per_sm_es() {
    const size_t smem = fused_pair_smem(ES);
    if (cudaFuncSetAttribute(fused_pair_kernel<ES, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_pair_kernel<ES, false>, kFT, smem) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace

size_t fused_pair_smem(int es) { return (size_t)kFW * kN * es * sizeof(float2); }

bool fused_pair_supported(int J, int es) { return J >= 1 && J <= kFW && (es == 33 || es == 37); }

int fused_pair_ctas_per_sm(int es) {
    switch (es) {
        case 33: return pair_ctas_per_sm_es<33>();
        case 37: return pair_ctas_per_sm_es<37>();
        default: return 0;
    }
}

cudaError_t launch_fused_pairs(const FusedParams& prm, int es, int ctas, cudaStream_t s) {
    const long long pairs = (long long)prm.P * prm.K;
    if (pairs == 0) return cudaSuccess;
    if (!fused_pair_supported(prm.J, es) || !prm.fscr || !prm.lpair || !prm.lcnt || !prm.fticket)
        return cudaErrorInvalidValue;
    if (ctas > pairs) ctas = (int)pairs;
    const bool expl = prm.oin != nullptr;
    cudaError_t e = es == 33 ? (expl ? launch_pairs_es<33, true>(prm, ctas, s) : launch_pairs_es<33, false>(prm, ctas, s))
                             : (expl ? launch_pairs_es<37, true>(prm, ctas, s) : launch_pairs_es<37, false>(prm, ctas, s));
    return e;
}

}  // namespace mfbd_dev
