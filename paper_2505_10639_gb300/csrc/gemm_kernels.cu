// SIMT FP32 GEMMs of the modal projections (Sec. 3.1, Eq. 22):
//   phi[u][i]  = c_k sum_m a[u][m] B_k[m][i]          (u = patch*J + frame)
//   g_a[u][m] (+)= c_k sum_i dL/dphi[u][i] B_k[m][i]
// Register-tiled SIMT kernels with the operands staged in shared memory.
#include "mfbd_internal.h"

#include <cstdint>

namespace mfbd_dev {

namespace {

// ---------------------------------------------------------------- GEMMs

// phase[u][i] = scale * sum_m a[u][m] basis[m][i]: 128 x 128 output tile per
// CTA of 256 threads, 8 x 8 per thread (two 4 x 4 quadrants 64 apart, so
// that the stores of a row are contiguous across threads), the modes in
// chunks of 16 staged in shared memory (rows padded to 132 floats).
constexpr int kPT = 128, kPK = 16, kPS = kPT + 4;

__global__ void __launch_bounds__(256, 2) phase_gemm_kernel(const float* __restrict__ a, int U, int M,
                                                            const float* __restrict__ basis, int npix, float scale,
                                                            float* __restrict__ out, int vec_store) {
    __shared__ __align__(16) float As[kPK][kPS];  // [m][u]
    __shared__ __align__(16) float Bs[kPK][kPS];  // [m][i]
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int u0 = blockIdx.y * kPT, i0 = blockIdx.x * kPT;
    float acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
    for (int m0 = 0; m0 < M; m0 += kPK) {
#pragma unroll
        for (int t = 0; t < kPT * kPK / 256; ++t) {
            const int idx = threadIdx.x + 256 * t;
            const int mm = idx & (kPK - 1), uu = idx >> 4;  // a: 16 consecutive modes of one row
            const int u = u0 + uu, m = m0 + mm;
            As[mm][uu] = (u < U && m < M) ? a[(size_t)u * M + m] : 0.f;
            const int ii = idx & (kPT - 1), mb = idx >> 7;  // basis: 128 consecutive pixels of one mode
            const int i = i0 + ii, mbm = m0 + mb;
            Bs[mb][ii] = (i < npix && mbm < M) ? basis[(size_t)mbm * npix + i] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kPK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[k][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[k][64 + tx * 4]);
            const float ar[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float br[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(ar[r], br[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int u = u0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + r - 4);
        if (u >= U) continue;
        float* row = out + (size_t)u * npix;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = i0 + h * 64 + tx * 4;
            if (vec_store) {  // npix % 4 == 0 and a 16-byte aligned output: whole float4 in or out
                if (i < npix)
                    *reinterpret_cast<float4*>(row + i) =
                        make_float4(scale * acc[r][4 * h], scale * acc[r][4 * h + 1], scale * acc[r][4 * h + 2],
                                    scale * acc[r][4 * h + 3]);
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (i + c < npix) row[i + c] = scale * acc[r][4 * h + c];
            }
        }
    }
}

// part[z][u][m] = sum_{i in chunk z} gphi[u][i] basis[m][i]: 128 x 48 output
// tile per CTA of 128 threads, 8 x 6 per thread, pixels in steps of 32 staged
// in shared memory (two buffers; the next step's operands are loaded into
// registers while the current one is computed). A thread loads row u = t of
// the dL/dphi step and stores it transposed, As[i][u]: the 32 lanes of a warp
// write 32 consecutive u of one i (no bank conflicts). Every object's pixel
// range is split into chunks; blockIdx.z runs over all (object, chunk).
constexpr int kGU = 128, kGM = 48, kGK = 32, kGT = 128;

__global__ void __launch_bounds__(kGT, 3) grad_gemm_kernel(const GradJob job, int U, int M) {
    __shared__ __align__(16) float As[2][kGK][kGU + 4];  // [i][u]
    __shared__ __align__(16) float Bs[2][kGK][kGM + 4];  // [i][m]
    int k = 0;
    while (k + 1 < job.K && (int)blockIdx.z >= job.split0[k + 1]) ++k;
    const float* __restrict__ gphi = job.gphi[k];
    const float* __restrict__ basis = job.basis[k];
    const int npix = job.npix[k], chunk = job.chunk[k], vec = job.vec[k];
    const int z = (int)blockIdx.z - job.split0[k];
    float* __restrict__ part = job.part[k];
    const int t = threadIdx.x;
    const int tx = t & 7, ty = t >> 3;  // 8 x 6 outputs: u = ty * 8 .., m = tx * 6 ..
    const int u0 = blockIdx.y * kGU, m0 = blockIdx.x * kGM;
    const int ib = z * chunk;
    const int ie = ib + chunk < npix ? ib + chunk : npix;
    float ra[kGK];      // row u0 + t of the next step
    float rb[3][4];     // (m, 4 pixels) groups of the next step's basis
    auto load = [&](int i0) {
        const int u = u0 + t;
        const float* g = gphi + (size_t)u * npix + i0;
        if (vec && u < U && i0 + kGK <= ie) {
#pragma unroll
            for (int q = 0; q < kGK / 4; ++q) {
                const float4 v = *reinterpret_cast<const float4*>(g + 4 * q);
                ra[4 * q] = v.x;
                ra[4 * q + 1] = v.y;
                ra[4 * q + 2] = v.z;
                ra[4 * q + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < kGK; ++i) ra[i] = (u < U && i0 + i < ie) ? g[i] : 0.f;
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int idx = t + kGT * r;  // < 384 = 48 modes x 8 groups of 4 pixels
            const int mm = idx % kGM, q = idx / kGM;
            const int m = m0 + mm, i = i0 + 4 * q;
            const float* bsrc = basis + (size_t)m * npix + i;
#pragma unroll
            for (int e = 0; e < 4; ++e) rb[r][e] = (m < M && i + e < ie) ? bsrc[e] : 0.f;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int i = 0; i < kGK; ++i) As[buf][i][t] = ra[i];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int idx = t + kGT * r;
            const int mm = idx % kGM, q = idx / kGM;
#pragma unroll
            for (int e = 0; e < 4; ++e) Bs[buf][4 * q + e][mm] = rb[r][e];
        }
    };
    float acc[8][6];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[r][c] = 0.f;
    if (ib < ie) {
        load(ib);
        store(0);
    }
    __syncthreads();
    int buf = 0;
    for (int i0 = ib; i0 < ie; i0 += kGK) {
        const bool more = i0 + kGK < ie;
        if (more) load(i0 + kGK);  // in flight during this step's FMAs
#pragma unroll 8
        for (int k = 0; k < kGK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 8 + 4]);
            const float2 b0 = *reinterpret_cast<const float2*>(&Bs[buf][k][tx * 6]);
            const float2 b1 = *reinterpret_cast<const float2*>(&Bs[buf][k][tx * 6 + 2]);
            const float2 b2 = *reinterpret_cast<const float2*>(&Bs[buf][k][tx * 6 + 4]);
            const float ar[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float br[6] = {b0.x, b0.y, b1.x, b1.y, b2.x, b2.y};
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 6; ++c) acc[r][c] = fmaf(ar[r], br[c], acc[r][c]);
        }
        if (more) store(buf ^ 1);  // the other buffer was last read before the previous barrier
        __syncthreads();
        buf ^= 1;
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int u = u0 + ty * 8 + r;
        if (u >= U) continue;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const int m = m0 + tx * 6 + c;
            if (m < M) part[((size_t)z * U + u) * M + m] = acc[r][c];
        }
    }
}

// grad[e] = sum_k scale_k sum_z part_k[z][e], in a fixed order
__global__ void __launch_bounds__(256) grad_combine_kernel(const GradParts gp, size_t n, float* __restrict__ grad) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        float v = 0.f;
        for (int k = 0; k < gp.K; ++k) {
            float t = 0.f;
            for (int z = 0; z < gp.splits[k]; ++z) t += gp.part[k][(size_t)z * n + e];
            v = fmaf(gp.scale[k], t, v);
        }
        grad[e] = v;
    }
}

}  // namespace

void grad_layout(int K, const int* npix, int U, int sms, int* chunk, int* splits) {
    // about one wave of CTAs (3 per SM) over all objects, the chunks of every
    // object about equally long (a multiple of the 32-pixel step)
    const int n_ut = (U + kGU - 1) / kGU > 0 ? (U + kGU - 1) / kGU : 1;
    long long total = 0;
    for (int k = 0; k < K; ++k) total += npix[k];
    long long want = 3LL * sms / n_ut;
    if (want < K) want = K;
    for (int k = 0; k < K; ++k) {
        long long sk = total > 0 ? (npix[k] * want + total / 2) / total : 1;
        if (sk < 1) sk = 1;
        long long c = (npix[k] + sk - 1) / sk;
        c = (c + kGK - 1) / kGK * kGK;
        if (c < kGK) c = kGK;
        chunk[k] = (int)c;
        splits[k] = npix[k] > 0 ? (int)((npix[k] + c - 1) / c) : 1;
    }
}

// phase[u][i] += div[u mod J][i]: the known diversity phase of frame j
// added to every patch's phase (phase diversity, Sec. 2.1).
__global__ void __launch_bounds__(256) add_diversity_kernel(float* __restrict__ phase,
                                                            const float* __restrict__ div, long long n, int J,
                                                            int npix) {
    const long long per = (long long)J * npix;
    for (long long e = blockIdx.x * 256ll + threadIdx.x; e < n; e += (long long)gridDim.x * 256)
        phase[e] += div[e % per];
}

cudaError_t launch_add_diversity(float* phase, const float* div, int U, int J, int npix, int sms, cudaStream_t s) {
    const long long n = (long long)U * npix;
    if (n == 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 8ll * sms) blocks = 8ll * sms;
    add_diversity_kernel<<<(int)blocks, 256, 0, s>>>(phase, div, n, J, npix);
    return cudaGetLastError();
}

cudaError_t launch_phase_gemm(const float* a, int U, int M, const float* basis, int npix, float scale,
                              float* phase, cudaStream_t s) {
    if (U == 0) return cudaSuccess;
    const int vec = (npix % 4 == 0) && (reinterpret_cast<uintptr_t>(phase) % 16 == 0);
    dim3 grid((npix + kPT - 1) / kPT, (U + kPT - 1) / kPT);
    phase_gemm_kernel<<<grid, 256, 0, s>>>(a, U, M, basis, npix, scale, phase, vec);
    return cudaGetLastError();
}

cudaError_t launch_grad_gemm(GradJob job, int U, int M, cudaStream_t s) {
    if (U == 0) return cudaSuccess;
    job.split0[0] = 0;
    for (int k = 0; k < job.K; ++k) {
        job.split0[k + 1] = job.split0[k] + job.splits[k];
        // whole float4 steps need 16-byte aligned rows
        job.vec[k] = (job.npix[k] % 4 == 0) && (reinterpret_cast<uintptr_t>(job.gphi[k]) % 16 == 0);
    }
    dim3 grid((M + kGM - 1) / kGM, (U + kGU - 1) / kGU, job.split0[job.K]);
    grad_gemm_kernel<<<grid, kGT, 0, s>>>(job, U, M);
    return cudaGetLastError();
}

cudaError_t launch_grad_combine(const GradParts& gp, int U, int M, float* grad, cudaStream_t s) {
    const size_t n = (size_t)U * M;
    if (n == 0) return cudaSuccess;
    size_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    grad_combine_kernel<<<(int)blocks, 256, 0, s>>>(gp, n, grad);
    return cudaGetLastError();
}

}  // namespace mfbd_dev
