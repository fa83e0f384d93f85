// Batched persistent kernel: the whole loss + gradient of an uneven batch of
// problems (patch sizes 48, 64, 96, 128; objects, frames and modes per
// problem) in one launch.
//
// The work is a list of items, each of one kind (BatchKind): P, the phases
// phi = c_k B_k a of every object and frame of a patch (Sec. 3.1, Eq. 22);
// F, the forward passes of a unit (Eqs. 20-21 and the OTF); R, the frame
// reduction of a patch (Sec. 2.2.1, Eqs. 11-12, and the adjoint seeds); A,
// the adjoint passes of a unit (-> dL/dphi); G, the modal adjoint of a patch
// (dL/da = sum_k c_k B_k^T dL/dphi_k). CTAs (128 threads) take items in list
// order from a ticket counter. In one-launch mode an item first waits for
// the items it depends on (P -> F -> R -> A -> G of the same patch), which
// all come earlier in the list: the holder of the smallest unfinished ticket
// never waits, so the launch always progresses. Every wait is bounded: on
// giving up it sets the error flag and the item is skipped. In staged mode
// the host launches each kind's range of the list separately and nothing
// waits.
//
// F and A items of patches of N <= 64 px cover up to four consecutive units
// (k J + j) of one patch: each of the CTA's four warps runs one unit on its own
// exchange buffer with warp synchronisation only. Larger patches use all 128
// threads on one unit. Every pass runs as rounds with one register FFT per
// (patch size, direction) (unit_forward_rounds, unit_adjoint_rounds): the
// kernel holds all patch sizes and both directions, and the smaller code was
// measured faster here (18.7 against 20.7 ms on the 2000-problem batch).
//
// Data written by one CTA and read by another inside the launch (phases,
// OTFs and seeds, fields, dL/dphi) is published by the writer's barrier,
// fence and counter increment and acquired by the reader's thread 0
// (ld.acquire.gpu, fence) before its CTA barrier: the PTX memory model then
// orders the readers' plain loads after the writes. Every per-unit and
// per-patch scratch block also starts on a 256-byte boundary, so no cache
// line is shared by blocks of different writers.
//
// The kernel is instantiated for its two register budgets in
// batch_kernel_v2.cu and batch_kernel_v3.cu, which compile in parallel.
#pragma once

#include "batch_internal.h"
#include "unit_passes.cuh"

#include <algorithm>


namespace mfbd_dev {

namespace {

using namespace unitpass;

constexpr long long kSpinLimit = 1ll << 22; // polls of a dependency counter (~1 s)

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0: wait until *c >= target. false (and the error flag set) when the
// wait gives up or another CTA has given up already.
__device__ bool wait_ctr(const int* c, int target, int* err) {
    for (long long it = 0; it < kSpinLimit; ++it) {
        if (ld_acquire(c) >= target) {
            __threadfence();
            return true;
        }
        if (*(volatile int*)err) return false;
        __nanosleep(200);
    }
    atomicExch(err, 1);
    return false;
}

__device__ __forceinline__ long long unit_stride_phi(int W) { return ((long long)W * W + 63) & ~63ll; }

// Pointers of unit (patch p, object k, frame j) of problem pr.
template <int N>
__device__ __forceinline__ UnitPtr batch_unit(const BatchParams& prm, const BatchProblem& pr, int p, int k, int j) {
    const BatchObj& ob = pr.obj[k];
    const long long u = ((long long)p * pr.K + k) * pr.J + j;
    const long long phi = pr.phi_off + (long long)p * pr.phi_patch + ob.phi_koff + (long long)j * unit_stride_phi(ob.W);
    UnitPtr q;
    q.phi = prm.phi + phi;
    q.gphi = prm.gphi + phi;
    q.h = prm.gscr + pr.gscr_off + u * N * Geo<N>::NH;
    q.pf = prm.pscr + pr.pscr_off + u * N * N;
    q.pp = nullptr;  // exp(i phi) is recomputed from the phase in the adjoint
    q.mask = ob.mask;
    q.mw = ob.mw;
    q.W = ob.W;
    q.inv_z = ob.inv_z;
    q.supp = ob.supp;
    q.sw = pr.sw;
    q.cmask = ob.cmask;
    q.csupp = ob.csupp;
    return q;
}

// F or A item: one unit per warp (N <= 64: up to four units of one patch,
// 32 lines per round, warp synchronisation only) or one unit on the
// whole CTA (N = 96, 128: 64 lines of two lanes per round, CTA barriers).
template <int N, bool ADJ>
__device__ void item_unit(const BatchParams& prm, const BatchProblem& pr, const BatchItem& it, float2* smem) {
    const int t = threadIdx.x;
    if constexpr (N <= 64) {
        const int w = t >> 5, lane = t & 31;
        if (w > it.extra) return;
        const int kj = it.kj + w, k = kj / pr.J, j = kj - k * pr.J;
        const UnitPtr q = batch_unit<N>(prm, pr, it.patch, k, j);
        float2* E = smem + (size_t)w * N * prm.es_small;
        if constexpr (ADJ) unit_adjoint_rounds<N, 32, false>(q, E, prm.es_small, nullptr, 0, lane, WarpBar{});
        else unit_forward_rounds<N, 32>(q, E, prm.es_small, lane, WarpBar{});
    } else {
        const int k = it.kj / pr.J, j = it.kj - k * pr.J;
        const UnitPtr q = batch_unit<N>(prm, pr, it.patch, k, j);
        if constexpr (ADJ) unit_adjoint_rounds<N, 64, false>(q, smem, prm.es_large, nullptr, 0, t, CtaBar{});
        else unit_forward_rounds<N, 64>(q, smem, prm.es_large, t, CtaBar{});
    }
}

// P item: phi_kj[i] = c_k sum_m a_j[m] B_k[m][i] on every box pixel i, for
// every object and frame of the patch; kJC frames per register tile with
// their coefficients staged in shared memory mode-major ([m][kJC]: two
// 16-byte loads per mode).
__device__ void item_proj(const BatchParams& prm, const BatchProblem& pr, int p, float* sa) {
    const int t = threadIdx.x, J = pr.J, M = pr.M;
    const float* a = prm.coeffs + pr.coeff_off + (size_t)p * J * M;
    for (int jc = 0; jc < J; jc += kJC) {
        const int nj = min(kJC, J - jc);
        __syncthreads();
        for (int e = t; e < kJC * M; e += kBT) {
            const int m = e / kJC, jj = e - m * kJC;
            sa[e] = jj < nj ? a[(size_t)(jc + jj) * M + m] : 0.f;
        }
        __syncthreads();
        const float4* sa4 = reinterpret_cast<const float4*>(sa);
        for (int k = 0; k < pr.K; ++k) {
            const BatchObj& ob = pr.obj[k];
            const int npix = ob.W * ob.W;
            const long long us = unit_stride_phi(ob.W);
            float* phi = prm.phi + pr.phi_off + (long long)p * pr.phi_patch + ob.phi_koff + jc * us;
            for (int i = t; i < npix; i += kBT) {
                float acc[kJC];
#pragma unroll
                for (int jj = 0; jj < kJC; ++jj) acc[jj] = 0.f;
                for (int m = 0; m < M; ++m) {
                    const float b = ob.bm[(size_t)m * npix + i];
                    const float4 c0 = sa4[2 * m], c1 = sa4[2 * m + 1];
                    acc[0] = fmaf(c0.x, b, acc[0]);
                    acc[1] = fmaf(c0.y, b, acc[1]);
                    acc[2] = fmaf(c0.z, b, acc[2]);
                    acc[3] = fmaf(c0.w, b, acc[3]);
                    acc[4] = fmaf(c1.x, b, acc[4]);
                    acc[5] = fmaf(c1.y, b, acc[5]);
                    acc[6] = fmaf(c1.z, b, acc[6]);
                    acc[7] = fmaf(c1.w, b, acc[7]);
                }
#pragma unroll
                for (int jj = 0; jj < kJC; ++jj)
                    if (jj < nj) phi[jj * us + i] = ob.scale * acc[jj];
            }
        }
    }
}

// G item: grad[j][m] = sum_k c_k sum_i dL/dphi_kj[i] B_k[m][i], the objects
// added in order; one thread per (mode, tile of kJC frames). (Staging
// dL/dphi and basis chunks in shared memory was measured slower: 5.7 against
// 2.0 ms for the 2000-problem batch.)
__device__ void item_grad(const BatchParams& prm, const BatchProblem& pr, int p) {
    const int t = threadIdx.x, J = pr.J, M = pr.M;
    const int tiles = (J + kJC - 1) / kJC;
    float* grad = prm.grad + pr.coeff_off + (size_t)p * J * M;
    for (int idx = t; idx < M * tiles; idx += kBT) {
        const int m = idx % M, jc = (idx / M) * kJC, nj = min(kJC, J - jc);
        float acc[kJC];
#pragma unroll
        for (int jj = 0; jj < kJC; ++jj) acc[jj] = 0.f;
        for (int k = 0; k < pr.K; ++k) {
            const BatchObj& ob = pr.obj[k];
            const int npix = ob.W * ob.W;
            const long long us = unit_stride_phi(ob.W);
            const float* g = prm.gphi + pr.phi_off + (long long)p * pr.phi_patch + ob.phi_koff + jc * us;
            const float* row[kJC];
#pragma unroll
            for (int jj = 0; jj < kJC; ++jj) row[jj] = g + min(jj, nj - 1) * us;
            float part[kJC];
#pragma unroll
            for (int jj = 0; jj < kJC; ++jj) part[jj] = 0.f;
            // four pixels per step: one 16-byte load of each frame's dL/dphi
            // (rows are 256-byte aligned), then the tail
            const int n4 = npix & ~3;
            for (int i = 0; i < n4; i += 4) {
                const float b0 = ob.bt[(size_t)i * ob.ldt + m], b1 = ob.bt[(size_t)(i + 1) * ob.ldt + m];
                const float b2 = ob.bt[(size_t)(i + 2) * ob.ldt + m], b3 = ob.bt[(size_t)(i + 3) * ob.ldt + m];
#pragma unroll
                for (int jj = 0; jj < kJC; ++jj) {
                    const float4 gv = *reinterpret_cast<const float4*>(row[jj] + i);
                    float x = fmaf(gv.x, b0, part[jj]);
                    x = fmaf(gv.y, b1, x);
                    x = fmaf(gv.z, b2, x);
                    part[jj] = fmaf(gv.w, b3, x);
                }
            }
            for (int i = n4; i < npix; ++i) {
                const float b = ob.bt[(size_t)i * ob.ldt + m];
#pragma unroll
                for (int jj = 0; jj < kJC; ++jj) part[jj] = fmaf(row[jj][i], b, part[jj]);
            }
#pragma unroll
            for (int jj = 0; jj < kJC; ++jj) acc[jj] = fmaf(ob.scale, part[jj], acc[jj]);
        }
#pragma unroll
        for (int jj = 0; jj < kJC; ++jj)
            if (jj < nj) grad[(size_t)(jc + jj) * M + m] = acc[jj];
    }
}

// R item: the four warps share each object's frequencies (warp w takes
// f = 32 w + lane + 128 i); the patch loss adds the warps' sums of an object
// in warp order, then the objects in order.
__device__ void item_reduce(const BatchParams& prm, const BatchProblem& pr, int p, double* sobj) {
    constexpr int kW = kBT / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int N = pr.N, NH = N / 2 + 1, J = pr.J;
    const size_t dstride = (size_t)N * NH;
    for (int k = 0; k < pr.K; ++k) {
        const size_t unit0 = ((size_t)p * pr.K + k) * J;
        RedPtr r;
        r.N = N;
        r.J = J;
        r.spec_ld = NH;
        r.gamma = pr.gamma;
        r.d = prm.spectra + pr.spec_off + unit0 * dstride;
        r.h = prm.gscr + pr.gscr_off + unit0 * dstride;
        r.w = pr.weights + (size_t)k * J;
        r.supp = pr.obj[k].supp;
        r.sw = pr.sw;
        r.obj = prm.object ? prm.object + pr.obj_off + ((size_t)p * pr.K + k) * dstride : nullptr;
        const double v = reduce_warp(r, lane, 32 * warp, 32 * kW);
        if (lane == 0) sobj[k * kW + warp] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int k = 0; k < pr.K; ++k) {
            double tk = 0.0;
            for (int w = 0; w < kW; ++w) tk += sobj[k * kW + w];
            tot += tk;
        }
        prm.loss[pr.loss_off + p] = tot;
    }
}

template <bool ADJ>
__device__ void dispatch_unit(const BatchParams& prm, const BatchProblem& pr, const BatchItem& it, float2* smem) {
    switch (pr.N) {
        case 48: item_unit<48, ADJ>(prm, pr, it, smem); break;
        case 64: item_unit<64, ADJ>(prm, pr, it, smem); break;
        case 96: item_unit<96, ADJ>(prm, pr, it, smem); break;
        default: item_unit<128, ADJ>(prm, pr, it, smem); break;
    }
}

// MINB: CTAs per SM the register budget is set for (2: up to 255 registers a
// thread; 3: up to 170, the 96 and 128 px passes then spill). The autotuner
// picks one.
template <int MINB>
__global__ void __launch_bounds__(kBT, MINB) batch_kernel(const BatchParams prm) {
    extern __shared__ __align__(16) unsigned char bsm[];
    float2* smem = reinterpret_cast<float2*>(bsm);
    __shared__ int s_item, s_ok;
    __shared__ double sobj[kMaxObjects * (kBT / 32)];
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(prm.ticket, 1);
        __syncthreads();
        const int i = s_item;
        if (i >= prm.n_items) break;
        const BatchItem it = prm.items[prm.item0 + i];
        const BatchProblem& pr = prm.probs[it.prob];
        int* ctr = prm.ctr + (pr.ctr_off + it.patch) * BC_COUNT;
        if (threadIdx.x == 0) {
            bool ok = true;
            if (prm.wait) {
                const int units = pr.K * pr.J;
                switch (it.kind) {
                    case BK_FWD: ok = wait_ctr(ctr + BC_PROJ, 1, prm.err); break;
                    case BK_RED: ok = wait_ctr(ctr + BC_FWD, units, prm.err); break;
                    case BK_ADJ: ok = wait_ctr(ctr + BC_RED, 1, prm.err); break;
                    case BK_GRAD: ok = wait_ctr(ctr + BC_ADJ, units, prm.err); break;
                    default: break;
                }
            }
            s_ok = ok;
        }
        __syncthreads();
        if (s_ok && ((prm.kinds >> it.kind) & 1)) {
            switch (it.kind) {
                case BK_PROJ: item_proj(prm, pr, it.patch, reinterpret_cast<float*>(bsm)); break;
                case BK_FWD: dispatch_unit<false>(prm, pr, it, smem); break;
                case BK_RED: item_reduce(prm, pr, it.patch, sobj); break;
                case BK_ADJ: dispatch_unit<true>(prm, pr, it, smem); break;
                default: item_grad(prm, pr, it.patch); break;
            }
        }
        __syncthreads();  // the item's writes precede the signal; s_item is free again
        if (prm.wait && threadIdx.x == 0 && it.kind != BK_GRAD) {
            __threadfence();
            const int n = (it.kind == BK_FWD || it.kind == BK_ADJ) ? 1 + it.extra : 1;
            const int slot = it.kind == BK_PROJ ? BC_PROJ : it.kind == BK_FWD ? BC_FWD : it.kind == BK_RED ? BC_RED
                                                                                                      : BC_ADJ;
            atomicAdd(ctr + slot, n);
        }
    }
}

}  // namespace

template <int MINB>
int batch_max_ctas_variant(size_t smem) {
    if (cudaFuncSetAttribute(batch_kernel<MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<MINB>, kBT, smem) != cudaSuccess)
        return 0;
    return per_sm;
}

template <int MINB>
cudaError_t launch_batch_variant(const BatchParams& prm, int ctas, size_t smem, cudaStream_t s) {
    batch_kernel<MINB><<<ctas, kBT, smem, s>>>(prm);
    return cudaGetLastError();
}

}  // namespace mfbd_dev
