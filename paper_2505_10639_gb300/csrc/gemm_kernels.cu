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

// part[z][u][m] = sum_{i in chunk z} gphi[u][i] basis[m][i]: 64 x 48 output
// tile per CTA of 64 threads, 8 x 6 per thread, pixels in chunks of 32
// staged in shared memory; the pixel range is split over blockIdx.z.
constexpr int kGU = 64, kGM = 48, kGK = 32;

__global__ void __launch_bounds__(64) grad_gemm_kernel(const float* __restrict__ gphi, int U, int npix,
                                                       const float* __restrict__ basis, int M, int chunk,
                                                       float* __restrict__ part) {
    __shared__ __align__(16) float As[kGK][kGU + 4];  // [i][u]
    __shared__ __align__(16) float Bs[kGK][kGM + 4];  // [i][m]
    const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
    const int u0 = blockIdx.y * kGU, m0 = blockIdx.x * kGM;
    const int ib = blockIdx.z * chunk;
    const int ie = ib + chunk < npix ? ib + chunk : npix;
    float acc[8][6];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[r][c] = 0.f;
    for (int i0 = ib; i0 < ie; i0 += kGK) {
#pragma unroll 8
        for (int t = 0; t < kGK * kGU / 64; ++t) {  // 32 consecutive pixels of one row per 32 threads
            const int idx = threadIdx.x + 64 * t;
            const int ii = idx & (kGK - 1), rr = idx >> 5;
            const int u = u0 + rr, i = i0 + ii;
            As[ii][rr] = (u < U && i < ie) ? gphi[(size_t)u * npix + i] : 0.f;
        }
#pragma unroll 8
        for (int t = 0; t < kGK * kGM / 64; ++t) {
            const int idx = threadIdx.x + 64 * t;
            const int ii = idx & (kGK - 1), rr = idx >> 5;
            const int m = m0 + rr, i = i0 + ii;
            Bs[ii][rr] = (m < M && i < ie) ? basis[(size_t)m * npix + i] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kGK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[k][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[k][ty * 8 + 4]);
            const float2 b0 = *reinterpret_cast<const float2*>(&Bs[k][tx * 6]);
            const float2 b1 = *reinterpret_cast<const float2*>(&Bs[k][tx * 6 + 2]);
            const float2 b2 = *reinterpret_cast<const float2*>(&Bs[k][tx * 6 + 4]);
            const float ar[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float br[6] = {b0.x, b0.y, b1.x, b1.y, b2.x, b2.y};
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 6; ++c) acc[r][c] = fmaf(ar[r], br[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int u = u0 + ty * 8 + r;
        if (u >= U) continue;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const int m = m0 + tx * 6 + c;
            if (m < M) part[((size_t)blockIdx.z * U + u) * M + m] = acc[r][c];
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

int grad_splits(int npix, int* chunk) {
    // pixel chunks of about 160 (a multiple of the 32-pixel staging step)
    int splits = (npix + 80) / 160;
    if (splits < 1) splits = 1;
    int c = (npix + splits - 1) / splits;
    c = (c + kGK - 1) / kGK * kGK;
    *chunk = c;
    return (npix + c - 1) / c;
}

cudaError_t launch_phase_gemm(const float* a, int U, int M, const float* basis, int npix, float scale,
                              float* phase, cudaStream_t s) {
    if (U == 0) return cudaSuccess;
    const int vec = (npix % 4 == 0) && (reinterpret_cast<uintptr_t>(phase) % 16 == 0);
    dim3 grid((npix + kPT - 1) / kPT, (U + kPT - 1) / kPT);
    phase_gemm_kernel<<<grid, 256, 0, s>>>(a, U, M, basis, npix, scale, phase, vec);
    return cudaGetLastError();
}

cudaError_t launch_grad_gemm(const float* gphi, int U, int npix, const float* basis, int M, float* part,
                             cudaStream_t s) {
    if (U == 0) return cudaSuccess;
    int chunk = 0;
    const int splits = grad_splits(npix, &chunk);
    dim3 grid((M + kGM - 1) / kGM, (U + kGU - 1) / kGU, splits);
    grad_gemm_kernel<<<grid, 64, 0, s>>>(gphi, U, npix, basis, M, chunk, part);
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
