// Modal phase projection on the 5th-generation tensor cores (Sec. 3.1,
// Eq. 22): phi[u][i] = c_k sum_m a[u][m] B_k[m][i], u = patch * J + frame,
// i a pixel of object k's pupil box.
//
// tcgen05.mma (kind::f16, BF16 operands, FP32 accumulation in tensor memory)
// computes the transposed product D[i][u] = sum_m B[m][i] a[u][m] on tiles
// of 128 pixels (MMA M, TMEM lanes) x 128 units (MMA N, TMEM columns), the
// modes being the contraction:
//   - FP32 precision: every operand is split into three BF16 planes,
//     x = x0 + x1 + x2 (each the BF16 rounding of what is left), and the six
//     plane products of weight >= 2^-16 are accumulated: a0 b0 + a0 b1 +
//     a1 b0 + a0 b2 + a1 b1 + a2 b0; the dropped ones are below 2^-24 of |a b|.
//   - BF16-phase precision: one plane each (a0 b0).
// Operands live in shared memory in the no-swizzle K-major core-matrix
// layout (8 rows x 16 bytes per core matrix, core matrices adjacent along K
// 128 bytes apart, 8-row groups Mp * 16 bytes apart); both come from global
// memory already in that layout (the basis from the plan, the coefficients
// from a split kernel), so staging is a plain asynchronous copy. A CTA keeps
// one pixel tile of the basis and loops over unit tiles with two coefficient
// buffers and two TMEM accumulators: one thread of a ninth warp issues the
// MMAs of tile n (the issue itself takes about as long as the MMAs) while the
// eight epilogue warps drain tile n - 1 from the other accumulator and the
// copy of tile n + 1 is in flight. In the epilogue a lane holds one pixel, so each store
// instruction writes 32 consecutive pixels of one unit's phase row.
#include "mfbd_internal.h"
#include "umma.cuh"

#include <cstdint>

namespace mfbd_dev {

namespace {

constexpr int kEpiWarps = 8;              // epilogue warps: two per TMEM lane quarter
constexpr int kTcThreads = 32 * (kEpiWarps + 1);  // + a warp that issues the MMAs
constexpr int kTile = 128;                // pixels (MMA M) and units (MMA N) per tile
constexpr long long kWaitLimit = 1ll << 22;  // bounded mbarrier polls

using umma::smem_addr;
using umma::smem_desc;
using umma::instr_desc_bf16;
using umma::issue_mmas;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem)), "l"(__cvta_generic_to_global(gmem))
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// all but the most recent group complete
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// true once the mbarrier's phase with this parity has completed (bounded poll)
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity) {
    uint32_t done = 0;
    for (long long n = 0; n < kWaitLimit && !done; ++n)
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(mbar)), "r"(parity)
            : "memory");
    return done != 0;
}

// x = x0 + x1 + x2 + r: each plane the BF16 rounding (to nearest even, by
// integer arithmetic on the bits; x finite) of what the previous planes
// leave; every subtraction is exact.
__device__ __forceinline__ uint32_t bf16_round_bits(float x) {
    const uint32_t u = __float_as_uint(x);
    return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
}

__device__ __forceinline__ void bf16_split3(float x, uint32_t& b0, uint32_t& b1, uint32_t& b2) {
    b0 = bf16_round_bits(x);
    const float r1 = x - __uint_as_float(b0 << 16);
    b1 = bf16_round_bits(r1);
    b2 = bf16_round_bits(r1 - __uint_as_float(b1 << 16));
}

// Coefficients [U][M] float -> BF16 planes in the MMA layout,
// [n_tiles][planes][128 units x Mp modes]; one thread per (unit, 8 modes).
__global__ void __launch_bounds__(256) split_coeffs_kernel(const float* __restrict__ a, int U, int M, int Mp,
                                                           int planes, uint16_t* __restrict__ out) {
    const int kcs = Mp / 8;
    const int n_tiles = (U + kTile - 1) / kTile;
    const long long total = (long long)n_tiles * kTile * kcs;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int kc = (int)(idx % kcs);
        const long long u = idx / kcs;
        uint32_t h[3][8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int m = kc * 8 + e;
            bf16_split3((u < U && m < M) ? a[u * M + m] : 0.f, h[0][e], h[1][e], h[2][e]);
        }
        const long long t = u / kTile;
        const int r = (int)(u % kTile);
        const size_t off = (size_t)(r >> 3) * Mp * 8 + (size_t)kc * 64 + (size_t)(r & 7) * 8;  // elements
        for (int p = 0; p < planes; ++p) {
            uint4 v;
            v.x = h[p][0] | (h[p][1] << 16);
            v.y = h[p][2] | (h[p][3] << 16);
            v.z = h[p][4] | (h[p][5] << 16);
            v.w = h[p][6] | (h[p][7] << 16);
            *reinterpret_cast<uint4*>(out + ((size_t)t * planes + p) * kTile * Mp + off) = v;
        }
    }
}

struct PhaseMmaParams {
    const uint16_t* at;                 // coefficient planes [n_utiles][planes][128 x Mp]
    int U, Mp, planes, K;
    int groups;                         // CTAs per pixel tile (the unit tiles are dealt among them)
    const uint16_t* bt[kMaxObjects];    // basis planes of object k [n_itiles_k][planes][128 x Mp]
    int npix[kMaxObjects], n_itiles[kMaxObjects];
    int cta0[kMaxObjects + 1];          // first CTA of object k
    float scale[kMaxObjects];
    float* out[kMaxObjects];            // [U][npix_k]
    int* err;                           // set to 1 when an MMA wait gives up
};

__global__ void __launch_bounds__(kTcThreads, 1) phase_mma_kernel(const PhaseMmaParams q) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Mp = q.Mp, planes = q.planes;
    const uint32_t plane_bytes = (uint32_t)kTile * Mp * 2;
    const uint32_t tile_bytes = plane_bytes * planes;
    unsigned char* sP = tc_smem;                   // basis (pixels) tile
    unsigned char* sU[2] = {tc_smem + tile_bytes, tc_smem + 2 * tile_bytes};  // coefficient (units) tiles
    const uint32_t sbo = (uint32_t)Mp * 16;

    int k = 0;
    while (k + 1 < q.K && (int)blockIdx.x >= q.cta0[k + 1]) ++k;
    const int local = (int)blockIdx.x - q.cta0[k];
    const int npix = q.npix[k];
    const float scale = q.scale[k];
    float* const out = q.out[k];
    const int it = local % q.n_itiles[k];
    const int g0 = local / q.n_itiles[k], gs = q.groups;
    const int n_utiles = (q.U + kTile - 1) / kTile;
    const int i0 = it * kTile;
    const int n_tiles = g0 < n_utiles ? (n_utiles - g0 + gs - 1) / gs : 0;  // this CTA's unit tiles

    auto copy_tile = [&](unsigned char* dst, const uint16_t* src) {
        const uint4* s4 = reinterpret_cast<const uint4*>(src);
        uint4* d4 = reinterpret_cast<uint4*>(dst);
        for (int i = tid; i < (int)(tile_bytes / 16); i += kTcThreads) cp_async16(d4 + i, s4 + i);
    };
    auto unit_src = [&](int n) { return q.at + (size_t)(g0 + n * gs) * planes * kTile * Mp; };

    copy_tile(sP, q.bt[k] + (size_t)it * planes * kTile * Mp);
    if (n_tiles > 0) copy_tile(sU[0], unit_src(0));
    cp_async_commit();
    if (n_tiles > 1) copy_tile(sU[1], unit_src(1));
    cp_async_commit();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base_s)),
                     "r"(2 * kTile));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[1])));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_s;
    const uint32_t idesc = instr_desc_bf16(kTile, kTile);
    const int lq = warp & 3, ch = warp >> 2;  // TMEM lane quarter (pixels), unit-column half

    // D[pixel][unit] of tile n (accumulator buf) -> phases
    auto epilogue = [&](int n, int buf) {
        const int u0 = (g0 + n * gs) * kTile;
        const int pix = lq * 32 + lane;
        float* ocol = out + i0 + pix;
        const bool pix_ok = i0 + pix < npix;
        for (int c0 = ch * (kTile / 2); c0 < (ch + 1) * (kTile / 2); c0 += 32) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(buf * kTile + c0);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (pix_ok) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int u = u0 + c0 + j;
                    if (u < q.U) ocol[(size_t)u * npix] = scale * __uint_as_float(v[j]);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    };

    bool ok = true;
    for (int n = 0; n < n_tiles; ++n) {
        const int buf = n & 1;
        cp_async_wait_prior();  // tile n (and the basis) landed; tile n + 1 may still be in flight
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // copies -> tensor core reads
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (warp == kEpiWarps && lane == 0) {
            // A: basis (pixel rows), B: coefficients (unit rows); a fresh accumulator per tile
            issue_mmas(tmem + (uint32_t)(buf * kTile), smem_desc(smem_addr(sP), 128, sbo),
                       smem_desc(smem_addr(sU[buf]), 128, sbo), plane_bytes, plane_bytes, Mp / 16, planes, idesc,
                       false);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(&mbar[buf]))
                         : "memory");
        }
        if (n >= 1 && warp < kEpiWarps) epilogue(n - 1, buf ^ 1);  // overlaps the MMAs of tile n
        const bool done = mbar_wait(&mbar[buf], (uint32_t)((n >> 1) & 1));
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (__syncthreads_or(!done)) {  // an MMA never completed: report, stop
            if (tid == 0) atomicExch(q.err, 1);
            ok = false;
            break;
        }
        // tile n's coefficients are consumed: prefetch tile n + 2 into them
        if (n + 2 < n_tiles) copy_tile(sU[buf], unit_src(n + 2));
        cp_async_commit();
    }
    if (ok && n_tiles > 0 && warp < kEpiWarps) epilogue(n_tiles - 1, (n_tiles - 1) & 1);
    cp_async_wait_all();
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTile));
}

}  // namespace

size_t phase_mma_smem(int M, int planes) {
    const size_t Mp = (size_t)(M + 15) / 16 * 16;
    return (size_t)3 * kTile * Mp * 2 * planes;  // basis tile + two coefficient tiles
}

size_t split_coeffs_elems(int U, int M, int planes) {
    const size_t Mp = (size_t)(M + 15) / 16 * 16;
    return (size_t)((U + kTile - 1) / kTile) * planes * kTile * Mp;
}

cudaError_t launch_split_coeffs(const float* a, int U, int M, int planes, uint16_t* at, cudaStream_t s) {
    if (U == 0) return cudaSuccess;
    const int Mp = (M + 15) / 16 * 16;
    const long long total = (long long)((U + kTile - 1) / kTile) * kTile * (Mp / 8);
    long long blocks = (total + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    split_coeffs_kernel<<<(int)blocks, 256, 0, s>>>(a, U, M, Mp, planes, at);
    return cudaGetLastError();
}

cudaError_t launch_phase_mma(const uint16_t* at, int U, int M, int K, const uint16_t* const* bt, const int* npix,
                             int planes, const float* scale, float* const* phase, int* err, int sms, cudaStream_t s) {
    if (U == 0 || K == 0) return cudaSuccess;
    if (K > kMaxObjects) return cudaErrorInvalidValue;
    PhaseMmaParams q;
    q.at = at;
    q.U = U;
    q.Mp = (M + 15) / 16 * 16;
    q.planes = planes;
    q.K = K;
    q.err = err;
    int total_itiles = 0;
    for (int k = 0; k < K; ++k) {
        q.bt[k] = bt[k];
        q.npix[k] = npix[k];
        q.n_itiles[k] = (npix[k] + kTile - 1) / kTile;
        q.scale[k] = scale[k];
        q.out[k] = phase[k];
        total_itiles += q.n_itiles[k];
    }
    // tensor memory holds 512 columns per SM and a CTA takes 256: the dynamic
    // shared memory is padded until at most two CTAs fit on an SM, so that
    // every resident CTA's allocation succeeds at once
    const int cap = 512 / (2 * kTile);
    size_t smem = phase_mma_smem(M, planes);
    int per_sm = 0;
    cudaError_t e = cudaFuncSetAttribute(phase_mma_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    for (int tries = 0; tries < 64; ++tries) {
        e = cudaFuncSetAttribute(phase_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, phase_mma_kernel, kTcThreads, smem);
        if (e != cudaSuccess) return e;
        if (per_sm <= cap) break;
        smem += 4096;
    }
    if (per_sm < 1 || per_sm > cap) return cudaErrorInvalidConfiguration;
    // one wave: every pixel tile of every object gets the same number of
    // CTAs, and all CTAs are resident at once
    const int n_utiles = (U + kTile - 1) / kTile;
    int groups = sms * per_sm / total_itiles;
    if (groups > n_utiles) groups = n_utiles;
    if (groups < 1) groups = 1;
    q.groups = groups;
    q.cta0[0] = 0;
    for (int k = 0; k < K; ++k) q.cta0[k + 1] = q.cta0[k] + groups * q.n_itiles[k];
    phase_mma_kernel<<<q.cta0[K], kTcThreads, smem, s>>>(q);
    return cudaGetLastError();
}

}  // namespace mfbd_dev
