// SIMT FP32 GEMMs of the modal projections (Sec. 3.1, Eq. 22):
//   phi[u][i]  = c_k sum_m a[u][m] B_k[m][i]          (u = patch*J + frame)
//   g_a[u][m] (+)= c_k sum_i dL/dphi[u][i] B_k[m][i]
// 64 x 64 output tiles, 4 x 4 per thread, operands staged in shared memory.
#include "mfbd_internal.h"

namespace mfbd_dev {

namespace {

// ---------------------------------------------------------------- GEMMs

// phase[u][i] = scale * sum_m a[u][m] basis[m][i]; 64x64 tiles, 4x4 per thread
__global__ void __launch_bounds__(256) phase_gemm_kernel(const float* __restrict__ a, int U, int M,
                                                         const float* __restrict__ basis, int npix, float scale,
                                                         float* __restrict__ out) {
    __shared__ float As[16][68];
    __shared__ float Bs[16][68];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int u0 = blockIdx.y * 64, i0 = blockIdx.x * 64;
    float acc[4][4] = {};
    for (int m0 = 0; m0 < M; m0 += 16) {
        for (int idx = threadIdx.x; idx < 16 * 64; idx += 256) {
            const int uu = idx >> 4, mm = idx & 15;
            const int u = u0 + uu, m = m0 + mm;
            As[mm][uu] = (u < U && m < M) ? a[(size_t)u * M + m] : 0.f;
            const int ii = idx & 63, mb = idx >> 6;
            const int i = i0 + ii, mbm = m0 + mb;
            Bs[mb][ii] = (i < npix && mbm < M) ? basis[(size_t)mbm * npix + i] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int mm = 0; mm < 16; ++mm) {
            float ar[4], br[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) ar[r] = As[mm][ty * 4 + r];
#pragma unroll
            for (int c = 0; c < 4; ++c) br[c] = Bs[mm][tx * 4 + c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(ar[r], br[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int u = u0 + ty * 4 + r;
        if (u >= U) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int i = i0 + tx * 4 + c;
            if (i < npix) out[(size_t)u * npix + i] = scale * acc[r][c];
        }
    }
}

// part[z][u][m] = sum_{i in chunk z} gphi[u][i] basis[m][i]  (split over i)
__global__ void __launch_bounds__(256) grad_gemm_kernel(const float* __restrict__ gphi, int U, int npix,
                                                        const float* __restrict__ basis, int M, int chunk,
                                                        float* __restrict__ part) {
    __shared__ float As[16][68];
    __shared__ float Bs[16][68];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int u0 = blockIdx.y * 64, m0 = blockIdx.x * 64;
    const int ib = blockIdx.z * chunk;
    const int ie = ib + chunk < npix ? ib + chunk : npix;
    float acc[4][4] = {};
    for (int i0 = ib; i0 < ie; i0 += 16) {
        for (int idx = threadIdx.x; idx < 16 * 64; idx += 256) {
            const int rr = idx >> 4, ii = idx & 15;
            const int u = u0 + rr, m = m0 + rr, i = i0 + ii;
            As[ii][rr] = (u < U && i < ie) ? gphi[(size_t)u * npix + i] : 0.f;
            Bs[ii][rr] = (m < M && i < ie) ? basis[(size_t)m * npix + i] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int ii = 0; ii < 16; ++ii) {
            float ar[4], br[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) ar[r] = As[ii][ty * 4 + r];
#pragma unroll
            for (int c = 0; c < 4; ++c) br[c] = Bs[ii][tx * 4 + c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(ar[r], br[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int u = u0 + ty * 4 + r;
        if (u >= U) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int m = m0 + tx * 4 + c;
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
    int splits = (npix + 255) / 256;
    if (splits < 1) splits = 1;
    int c = (npix + splits - 1) / splits;
    c = (c + 15) / 16 * 16;
    *chunk = c;
    return (npix + c - 1) / c;
}

cudaError_t launch_phase_gemm(const float* a, int U, int M, const float* basis, int npix, float scale,
                              float* phase, cudaStream_t s) {
    if (U == 0) return cudaSuccess;
    dim3 grid((npix + 63) / 64, (U + 63) / 64);
    phase_gemm_kernel<<<grid, 256, 0, s>>>(a, U, M, basis, npix, scale, phase);
    return cudaGetLastError();
}

cudaError_t launch_grad_gemm(const float* gphi, int U, int npix, const float* basis, int M, float* part,
                             cudaStream_t s) {
    if (U == 0) return cudaSuccess;
    int chunk = 0;
    const int splits = grad_splits(npix, &chunk);
    dim3 grid((M + 63) / 64, (U + 63) / 64, splits);
    grad_gemm_kernel<<<grid, 256, 0, s>>>(gphi, U, npix, basis, M, chunk, part);
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
