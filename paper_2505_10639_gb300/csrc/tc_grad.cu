// Modal adjoint on the 5th-generation tensor cores (Sec. 3.1, the transpose
// of Eq. 22; the chain rule of Sec. 3.3 from the phase to the modal
// coefficients):
//   part_k[z][u][m] = sum_{i in pixel chunk z of object k} dL/dphi_k[u][i] B_k[m][i]
// and grad[u][m] = sum_k c_k sum_z part_k[z][u][m] (grad_combine_kernel).
//
// D[u][m] is a tile of 128 units (MMA M, TMEM lanes) x Mp modes (MMA N, TMEM
// columns); the pixels are the contraction, streamed in stages of 32:
//   - a producer warp loads each stage's FP32 dL/dphi tile (128 units x 32
//     pixels, 16 KB) with a TMA tile copy (128-byte swizzle) and the stage's
//     basis planes (3 x Mp x 32 BF16, laid out by the plan in the MMA's
//     K-major core-matrix layout) with a bulk copy, both on one mbarrier;
//   - eight converter warps split the FP32 tile into three BF16 planes,
//     x = x0 + x1 + x2 (each the BF16 rounding of what is left), written to
//     shared memory in the core-matrix layout (double buffered);
//   - one thread of an MMA warp issues the six plane products of weight
//     >= 2^-16 (a0 b0, a0 b1, a1 b0, a0 b2, a1 b1, a2 b0) per K-step of 16,
//     FP32 accumulation in tensor memory, and commits each stage to the
//     barriers that free its ring slot and its plane buffer;
//   - after a chunk's last stage the converter warps read the accumulator
//     (two TMEM accumulators: the next chunk's MMAs run meanwhile) and write
//     the partial sums of the chunk.
// A CTA (one per SM) takes the work items (unit tile, object, pixel chunk)
// blockIdx.x, blockIdx.x + gridDim.x, ... and streams their stages through
// one ring, so loads run ahead across items. The chunks are fixed by the
// plan for all P*J units: the summation order of a unit's gradient does not
// depend on which call or CTA computes it.
//
// Every mbarrier wait is bounded: a wait that gives up sets the error flag
// and a CTA-wide abort flag that ends the other roles' loops; the CTA then
// waits (bounded) for its copies and MMAs in flight and frees its tensor
// memory before it returns.
#include "mfbd_internal.h"
#include "tma.cuh"
#include "umma.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

namespace mfbd_dev {

namespace {

constexpr int kGS = 32;                       // pixels per stage (one 128-byte FP32 TMA row)
constexpr int kGR = 128;                      // units per tile (MMA M)
constexpr int kGConv = 8;                     // converter / epilogue warps
constexpr int kGThreads = (kGConv + 2) * 32;  // + a producer warp and an MMA warp
constexpr int kGMaxRing = 8;
constexpr uint32_t kFBytes = kGR * kGS * 4;   // FP32 tile of a stage
constexpr uint32_t kAPlane = kGR * kGS * 2;   // one BF16 plane of it
constexpr long long kGWait = 1ll << 22;       // bounded mbarrier polls
constexpr size_t kGSmemLimit = 227 * 1024;

using umma::smem_addr;

struct GradMmaParams {
    CUtensorMap gmap[kMaxObjects];      // dL/dphi_k [rows][npix_k] FP32, box 32 x 128, 128-byte swizzle
    const uint16_t* bpl[kMaxObjects];   // B_k planes per stage [stage][3][Mp x 32]
    float* part[kMaxObjects];           // [splits_k][U][M], row 0 = the call's first unit
    int nst[kMaxObjects];               // stages of object k (ceil(npix_k / 32))
    int cst[kMaxObjects];               // stages per chunk
    int split0[kMaxObjects + 1];        // prefix sums of the chunk counts
    int K, U, M, Mp, row0, n_items, ring, acc_cols;
    int* err;
};

struct Item {
    int k, t, z, s0, ns;
};

__device__ __forceinline__ Item item_of(const GradMmaParams& q, int i) {
    const int ipt = q.split0[q.K];
    Item it;
    it.t = i / ipt;
    const int r = i - it.t * ipt;
    int k = 0;
    while (k + 1 < q.K && r >= q.split0[k + 1]) ++k;
    it.k = k;
    it.z = r - q.split0[k];
    it.s0 = it.z * q.cst[k];
    const int e = it.s0 + q.cst[k] < q.nst[k] ? it.s0 + q.cst[k] : q.nst[k];
    it.ns = e - it.s0;
    return it;
}

__device__ __forceinline__ bool try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; false when the CTA aborts (this wait gave up, or another did)
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err) {
    for (long long n = 0; n < kGWait; ++n) {
        if (try_wait(bar, parity)) return true;
        if ((n & 63) == 63 && *abort_flag) return false;
    }
    *abort_flag = 1;
    atomicExch(err, 1);
    return false;
}

// mbarrier init without the fence (one fence after all of them)
__device__ __forceinline__ void bar_init(uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// two FP32 values -> their BF16 roundings as a pair (x in the low half) and
// the exact remainders
__device__ __forceinline__ uint32_t split_pair(float& x, float& y) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(x, y);
    const uint32_t u = *reinterpret_cast<const uint32_t*>(&b);
    x -= __uint_as_float(u << 16);
    y -= __uint_as_float(u & 0xFFFF0000u);
    return u;
}

__global__ void __launch_bounds__(kGThreads, 1) grad_mma_kernel(const __grid_constant__ GradMmaParams q) {
    extern __shared__ __align__(16) unsigned char g_dyn[];
    __shared__ __align__(8) uint64_t full[kGMaxRing], empty[kGMaxRing];
    __shared__ __align__(8) uint64_t conv[2], afree[2], accf[2], accfree[2], fin;
    __shared__ uint32_t tmem_s;
    __shared__ int abort_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = q.ring, Mp = q.Mp;
    const uint32_t bst = (uint32_t)Mp * kGS * 2 * 3;  // basis bytes of a stage
    // 1024-byte aligned FP32 tiles (the swizzle pattern repeats every 1024 bytes)
    unsigned char* g_smem = g_dyn + ((1024 - (smem_addr(g_dyn) & 1023)) & 1023);
    unsigned char* sF = g_smem;
    unsigned char* sB = g_smem + (size_t)S * kFBytes;
    unsigned char* sA = g_smem + (((size_t)S * (kFBytes + bst) + 1023) & ~(size_t)1023);
    volatile int* abort_flag = &abort_s;

    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            bar_init(&full[i], 1);
            bar_init(&empty[i], 1);
        }
        for (int b = 0; b < 2; ++b) {
            bar_init(&conv[b], kGConv);
            bar_init(&afree[b], 1);
            bar_init(&accf[b], 1);
            bar_init(&accfree[b], kGConv);
        }
        bar_init(&fin, 1);
        // the initialised barriers, visible to the asynchronous proxy
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_s = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_s)),
                     "r"(q.acc_cols * 2));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = tmem_s;

    if (warp == kGConv) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            uint32_t n = 0;
            bool ok = true;
            for (int i = blockIdx.x; ok && i < q.n_items; i += gridDim.x) {
                const Item it = item_of(q, i);
                const int y = q.row0 + it.t * kGR;
                for (int s = 0; s < it.ns; ++s, ++n) {
                    const int slot = (int)(n % (uint32_t)S);
                    if (n >= (uint32_t)S && !wait_or_abort(&empty[slot], (n / S - 1) & 1, abort_flag, q.err)) {
                        ok = false;
                        break;
                    }
                    tma::mbar_arrive_expect_tx(&full[slot], kFBytes + bst);
                    tma::load_2d(sF + (size_t)slot * kFBytes, &q.gmap[it.k], (it.s0 + s) * kGS, y, &full[slot]);
                    bulk_load(sB + (size_t)slot * bst, q.bpl[it.k] + (size_t)(it.s0 + s) * (bst / 2), bst,
                              &full[slot]);
                }
            }
            // copies still in flight (an abort): wait for them before the
            // shared memory is released
            const uint32_t first = n > (uint32_t)S ? n - S : 0;
            for (uint32_t m = first; m < n; ++m) {
                const int slot = (int)(m % (uint32_t)S);
                for (long long w = 0; w < kGWait && !try_wait(&full[slot], (m / S) & 1); ++w) {
                }
            }
        }
    } else if (warp == kGConv + 1) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            const uint32_t idesc = umma::instr_desc_bf16(kGR, Mp);
            uint32_t n = 0;
            int c = 0;
            bool ok = true;
            for (int i = blockIdx.x; ok && i < q.n_items; i += gridDim.x, ++c) {
                const Item it = item_of(q, i);
                const int a = c & 1;
                if (c >= 2 && !wait_or_abort(&accfree[a], ((c >> 1) - 1) & 1, abort_flag, q.err)) break;
                umma::fence_after_sync();
                for (int s = 0; s < it.ns; ++s, ++n) {
                    const int slot = (int)(n % (uint32_t)S), b = (int)(n & 1);
                    if (!wait_or_abort(&conv[b], (n >> 1) & 1, abort_flag, q.err)) {
                        ok = false;
                        break;
                    }
                    umma::fence_after_sync();
                    // A: the units' planes, B: the modes' planes; K-major, core
                    // matrices 128 bytes apart along K, 8-row groups 512 bytes apart
                    umma::issue_mmas(tmem + (uint32_t)(a * q.acc_cols),
                                     umma::smem_desc(smem_addr(sA + (size_t)b * 3 * kAPlane), 128, 512),
                                     umma::smem_desc(smem_addr(sB + (size_t)slot * bst), 128, 512), kAPlane,
                                     (uint32_t)Mp * kGS * 2, kGS / 16, 3, idesc, s > 0);
                    umma::commit(&empty[slot]);
                    umma::commit(&afree[b]);
                }
                if (ok) umma::commit(&accf[a]);
            }
            // every MMA issued has completed before the tensor memory is freed
            umma::commit(&fin);
            for (long long w = 0; w < kGWait && !try_wait(&fin, 0); ++w) {
            }
        }
    } else {
        // ---------------------------------------- converters and epilogue
        const int lq = warp & 3, half = warp >> 2;
        auto epilogue = [&](int c, const Item& it) -> bool {
            const int a = c & 1;
            if (!__all_sync(0xFFFFFFFFu, wait_or_abort(&accf[a], (c >> 1) & 1, abort_flag, q.err))) return false;
            umma::fence_after_sync();
            const int u = it.t * kGR + lq * 32 + lane;
            float* prow = q.part[it.k] + ((size_t)it.z * q.U + u) * q.M;
            // columns in groups of 16, alternately to the two warps of a lane quarter
            for (int g = half; g < Mp / 16; g += 2) {
                uint32_t v[16];
                const uint32_t taddr = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(a * q.acc_cols + g * 16);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (u < q.U) {
                    const int m0 = g * 16;
                    if ((q.M & 3) == 0) {
#pragma unroll
                        for (int e = 0; e < 16; e += 4)
                            if (m0 + e < q.M)
                                *reinterpret_cast<float4*>(prow + m0 + e) =
                                    make_float4(__uint_as_float(v[e]), __uint_as_float(v[e + 1]),
                                                __uint_as_float(v[e + 2]), __uint_as_float(v[e + 3]));
                    } else {
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            if (m0 + e < q.M) prow[m0 + e] = __uint_as_float(v[e]);
                    }
                }
            }
            umma::fence_before_sync();
            __syncwarp();
            if (lane == 0) arrive(&accfree[a]);
            return true;
        };

        uint32_t n = 0;
        int c = 0;
        bool ok = true;
        Item prev{};
        for (int i = blockIdx.x; ok && i < q.n_items; i += gridDim.x, ++c) {
            const Item it = item_of(q, i);
            for (int s = 0; s < it.ns; ++s, ++n) {
                const int slot = (int)(n % (uint32_t)S), b = (int)(n & 1);
                bool w = wait_or_abort(&full[slot], (n / S) & 1, abort_flag, q.err);
                if (w && n >= 2) w = wait_or_abort(&afree[b], ((n >> 1) - 1) & 1, abort_flag, q.err);
                // the outcome is warp-uniform: one elected lane arrives for the warp
                if (!__all_sync(0xFFFFFFFFu, w)) {
                    ok = false;
                    break;
                }
                const unsigned char* f = sF + (size_t)slot * kFBytes;
                unsigned char* ab = sA + (size_t)b * 3 * kAPlane;
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int idx = tid + kGConv * 32 * j;
                    const int r = idx & (kGR - 1), kg = idx >> 7;  // unit row, 8-pixel group
                    // 128-byte swizzle: 16-byte chunk c of row r sits at chunk c ^ (r mod 8)
                    const float4 lo =
                        *reinterpret_cast<const float4*>(f + r * 128 + (((2 * kg) ^ (r & 7)) << 4));
                    const float4 hi =
                        *reinterpret_cast<const float4*>(f + r * 128 + (((2 * kg + 1) ^ (r & 7)) << 4));
                    float x[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
                    uint32_t pl[3][4];
#pragma unroll
                    for (int p = 0; p < 3; ++p)
#pragma unroll
                        for (int e = 0; e < 4; ++e) pl[p][e] = split_pair(x[2 * e], x[2 * e + 1]);
                    const int off = (r >> 3) * 512 + kg * 128 + (r & 7) * 16;
#pragma unroll
                    for (int p = 0; p < 3; ++p)
                        *reinterpret_cast<uint4*>(ab + p * kAPlane + off) =
                            make_uint4(pl[p][0], pl[p][1], pl[p][2], pl[p][3]);
                }
                tma::fence_proxy_async_smem();  // the planes -> the tensor core's reads
                __syncwarp();
                if (lane == 0) arrive(&conv[b]);
                if (s == 0 && c >= 1 && !epilogue(c - 1, prev)) {
                    ok = false;
                    break;
                }
            }
            prev = it;
        }
        if (ok && c >= 1) epilogue(c - 1, prev);
    }

    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(q.acc_cols * 2));
}

uint16_t bf16_bits(float x) {  // round to nearest even (x finite)
    uint32_t u;
    std::memcpy(&u, &x, 4);
    return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}

float bf16_value(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float x;
    std::memcpy(&x, &u, 4);
    return x;
}

}  // namespace

size_t grad_mma_smem(int M, int ring) {
    const size_t Mp = (size_t)(M + 15) / 16 * 16;
    const size_t bst = Mp * kGS * 2 * 3;
    // + 1024 bytes to align the base
    return 1024 + (((size_t)ring * (kFBytes + bst) + 1023) & ~(size_t)1023) + 2 * 3 * kAPlane;
}

int grad_mma_ring(int M) {
    const int Mp = (M + 15) / 16 * 16;
    if (M < 1 || Mp > 256) return 0;
    int ring = kGMaxRing > 6 ? 6 : kGMaxRing;
    while (ring >= 2 && grad_mma_smem(M, ring) > kGSmemLimit) --ring;
    return ring >= 2 ? ring : 0;
}

size_t grad_mma_basis_elems(int npix, int M) {
    const size_t Mp = (size_t)(M + 15) / 16 * 16;
    return (size_t)((npix + kGS - 1) / kGS) * 3 * Mp * kGS;
}

void grad_mma_basis(const float* basis, int npix, int M, uint16_t* out) {
    const int Mp = (M + 15) / 16 * 16, nst = (npix + kGS - 1) / kGS;
    std::fill(out, out + grad_mma_basis_elems(npix, M), (uint16_t)0);
    for (int s = 0; s < nst; ++s)
        for (int m = 0; m < M; ++m)
            for (int c = 0; c < kGS; ++c) {
                const int i = s * kGS + c;
                if (i >= npix) break;
                float left = basis[(size_t)m * npix + i];
                for (int p = 0; p < 3; ++p) {
                    const uint16_t b = bf16_bits(left);
                    left -= bf16_value(b);
                    // [stage][plane][mode group][pixel group][mode mod 8][pixel mod 8]
                    const size_t off = (((size_t)s * 3 + p) * (Mp / 8) + m / 8) * 256 + (size_t)(c / 8) * 64 +
                                       (size_t)(m % 8) * 8 + (c % 8);
                    out[off] = b;
                }
            }
}

void grad_mma_layout(int K, const int* npix, int M, int U, int sms, int* chunk, int* splits) {
    // Chunk lengths (in stages) of about equal size for all objects, chosen
    // to even out the stages the CTAs stream (items dealt round robin), with
    // each chunk's partial-sum write (128 x M floats) counted as stages.
    const int n_tiles = (U + kGR - 1) / kGR > 0 ? (U + kGR - 1) / kGR : 1;
    int nst[kMaxObjects], most = 1;
    for (int k = 0; k < K; ++k) {
        nst[k] = (npix[k] + kGS - 1) / kGS;
        if (nst[k] > most) most = nst[k];
    }
    const double write_cost = (double)M * 4.0 / (kGS * 4.0);  // a partial row against a stage row
    double best = 1e300;
    int best_l = most;
    for (int L = 1; L <= most; ++L) {
        std::vector<int> sizes;
        for (int k = 0; k < K; ++k)
            for (int s0 = 0; s0 < nst[k]; s0 += L) sizes.push_back(std::min(L, nst[k] - s0));
        const long long items = (long long)n_tiles * (long long)sizes.size();
        const int G = (int)std::min<long long>(items, sms);
        std::vector<double> load(G, 0.0);
        for (long long i = 0; i < items; ++i) load[i % G] += sizes[i % sizes.size()] + write_cost;
        double worst = 0;
        for (double v : load) worst = std::max(worst, v);
        if (worst < best * 0.999) {
            best = worst;
            best_l = L;
        }
    }
    for (int k = 0; k < K; ++k) {
        chunk[k] = best_l * kGS;
        splits[k] = nst[k] > 0 ? (nst[k] + best_l - 1) / best_l : 1;
    }
}

bool encode_grad_map(CUtensorMap* map, const float* gphi, int npix, long long rows) {
    if (npix % 4 != 0 || (reinterpret_cast<uintptr_t>(gphi) & 15) != 0 || rows < 1) return false;
    return tma::encode_f32_2d_swizzle128(map, gphi, (uint64_t)npix, (uint64_t)rows, kGS, kGR);
}

cudaError_t launch_grad_mma(const GradMmaJob& job, int sms, cudaStream_t s) {
    if (job.U == 0) return cudaSuccess;
    if (job.K < 1 || job.K > kMaxObjects) return cudaErrorInvalidValue;
    GradMmaParams q;
    std::memset(&q, 0, sizeof q);
    q.K = job.K;
    q.U = job.U;
    q.M = job.M;
    q.Mp = (job.M + 15) / 16 * 16;
    q.row0 = job.row0;
    q.ring = grad_mma_ring(job.M);
    if (q.ring < 2) return cudaErrorInvalidConfiguration;
    int cols = 32;
    while (cols < q.Mp) cols *= 2;
    q.acc_cols = cols;  // two accumulators of acc_cols columns (a power of two, <= 256)
    q.err = job.err;
    q.split0[0] = 0;
    for (int k = 0; k < job.K; ++k) {
        q.gmap[k] = *job.gmap[k];
        q.bpl[k] = job.bpl[k];
        q.part[k] = job.part[k];
        q.nst[k] = (job.npix[k] + kGS - 1) / kGS;
        q.cst[k] = job.chunk[k] / kGS;
        if (q.cst[k] < 1 || job.chunk[k] % kGS != 0) return cudaErrorInvalidValue;
        q.split0[k + 1] = q.split0[k] + (q.nst[k] + q.cst[k] - 1) / q.cst[k];
    }
    const long long items = (long long)((job.U + kGR - 1) / kGR) * q.split0[job.K];
    if (items >= (1ll << 31)) return cudaErrorInvalidValue;
    q.n_items = (int)items;
    const size_t smem = grad_mma_smem(job.M, q.ring);
    cudaError_t e = cudaFuncSetAttribute(grad_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<long long>(items, sms);
    grad_mma_kernel<<<grid, kGThreads, smem, s>>>(q);
    return cudaGetLastError();
}

}  // namespace mfbd_dev
