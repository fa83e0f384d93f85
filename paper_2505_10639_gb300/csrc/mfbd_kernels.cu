// sm_103a kernels of the MOMFBD hot path (N = 64 patches).
//
// Fused kernel (one persistent CTA per patch at a time, S frame slots of 64
// threads each; one thread owns one 64-point line in registers):
//   forward per frame (Sec. 3.1, Eqs. 20-22):
//     F1  pupil columns:  P = A exp(i phi) on the pupil's bounding box,
//                         column FFTs (only the W box columns are nonzero)
//     F2  rows:           row FFTs -> field p; s = |p|^2 / (N^2 n_pup)
//                         (Parseval: sum |p|^2 = N^2 n_pup for a phase-only
//                         pupil); real-to-complex row FFTs of s
//     F3  columns:        column FFTs -> H = F s on the half spectrum;
//                         H(0) := 1, H := 0 outside the exact OTF support
//   reduction per object (Sec. 2.2.1, Eqs. 11-12), per frequency u:
//     N = sum_j w D conj(H) (FP32), Q = sum_j w |H|^2 + gamma (FP64),
//     O = N / Q, t(u) = sum_j w |D - O H|^2 + gamma |O|^2 (equal to the
//     summand of Eq. 12 at O = N/Q, without its cancellation), loss summed
//     over u in FP64; adjoint seed G_j = dL/dconj(H_j) = -w conj(O)(D - O H)
//     with G(0) := 0 and G := 0 outside the support (exact: H(0) == 1 and
//     H == 0 there for every wavefront)
//   backward per frame:
//     B1/B2  C2R of G:    g_s = 2 Re F^H G,  g_q = g_s / (N^2 n_pup)
//     F1r/F2r             recompute p, G_p = g_q p, row F^H
//     B3                  column F^H on the box columns -> G_P,
//                         dL/dphi = 2 Im(conj(P) G_P) on pupil pixels
// The modal projections phi = c B a and dL/da = sum_k c_k B_k^T dL/dphi are
// separate GEMM kernels.
#include "mfbd_internal.h"
#include "fft_reg.cuh"

namespace mfbd_dev {

using fftreg::cadd;
using fftreg::cconj;
using fftreg::cmul;
using fftreg::cscale;
using fftreg::csub;

namespace {

constexpr int kMaxSlots = 6;
constexpr int kThreadsMax = 64 * kMaxSlots;

__device__ __forceinline__ void slot_sync(int slot) {
    asm volatile("bar.sync %0, 64;" ::"r"(slot + 1) : "memory");
}

__device__ __forceinline__ float2 pupil_value(float ph) {
    float s, c;
    sincosf(ph, &s, &c);
    return make_float2(c, s);
}

// F1 / F1r: column t of the pupil's box -> column FFT -> X[:, t]
__device__ __forceinline__ void pupil_columns(const ObjParams& ob, const float* phi, const uint64_t* smask,
                                              float2* X, int xs, int t) {
    const int W = ob.W, x0 = ob.x0;
    for (int yy = 0; yy < W; ++yy) {
        float2 v = make_float2(0.f, 0.f);
        if ((smask[yy] >> t) & 1ull) v = pupil_value(phi[yy * ob.phi_ld + t]);
        X[(x0 + yy) * xs + t] = v;
    }
    float2 col[kN];
#pragma unroll
    for (int y = 0; y < kN; ++y)
        col[y] = ((unsigned)(y - x0) < (unsigned)W) ? X[y * xs + t] : make_float2(0.f, 0.f);
    fftreg::fft<kN, -1>(col);
#pragma unroll
    for (int y = 0; y < kN; ++y) X[y * xs + t] = col[y];
}

// row t of the field p = F P (box columns of X are the only nonzero inputs)
__device__ __forceinline__ void field_row(const ObjParams& ob, const float2* X, int xs, int t, float2 (&row)[kN]) {
    const int W = ob.W, x0 = ob.x0;
#pragma unroll
    for (int x = 0; x < kN; ++x)
        row[x] = ((unsigned)(x - x0) < (unsigned)W) ? X[t * xs + (x - x0)] : make_float2(0.f, 0.f);
    fftreg::fft<kN, -1>(row);
}

__device__ void forward_unit(const FusedParams& prm, const ObjParams& ob, long long unit, float2* hout,
                             const uint64_t* smask, const uint64_t* ssupp, float2* X, float2* Y, int xs,
                             int t, int slot) {
    const float* phi = prm.phi + ob.phi_off + unit * ob.phi_unit + ob.phi_org;
    if (t < ob.W) pupil_columns(ob, phi, smask, X, xs, t);
    slot_sync(slot);
    {
        float2 row[kN];
        field_row(ob, X, xs, t, row);
        float s[kN];
#pragma unroll
        for (int x = 0; x < kN; ++x) s[x] = (row[x].x * row[x].x + row[x].y * row[x].y) * ob.inv_z;
        float2 sh[kNH];
        fftreg::rfft<kN>(s, sh);
#pragma unroll
        for (int kx = 0; kx < kNH; ++kx) Y[t * kNH + kx] = sh[kx];
    }
    slot_sync(slot);
    if (t < 32) {
        float2 col[kN];
        if (t == 0) {
#pragma unroll
            for (int ky = 0; ky < kN; ++ky) col[ky] = make_float2(Y[ky * kNH].x, Y[ky * kNH + 32].x);
        } else {
#pragma unroll
            for (int ky = 0; ky < kN; ++ky) col[ky] = Y[ky * kNH + t];
        }
        fftreg::fft<kN, -1>(col);
        if (t == 0) {
            // split the transform of (real col 0) + i (real col 32)
#pragma unroll
            for (int ky = 0; ky < kN; ++ky) {
                const float2 a = col[ky];
                const float2 b = cconj(col[(kN - ky) % kN]);
                float2 h0 = cscale(cadd(a, b), 0.5f);
                const float2 d = cscale(csub(a, b), 0.5f);
                float2 h32 = make_float2(d.y, -d.x);
                if (!((ssupp[ky] >> 0) & 1ull)) h0 = make_float2(0.f, 0.f);
                if (!((ssupp[ky] >> 32) & 1ull)) h32 = make_float2(0.f, 0.f);
                if (ky == 0) h0 = make_float2(1.f, 0.f);
                hout[ky * kNH] = h0;
                hout[ky * kNH + 32] = h32;
            }
        } else {
#pragma unroll
            for (int ky = 0; ky < kN; ++ky) {
                float2 h = col[ky];
                if (!((ssupp[ky] >> t) & 1ull)) h = make_float2(0.f, 0.f);
                hout[ky * kNH + t] = h;
            }
        }
    }
}

__device__ void backward_unit(const FusedParams& prm, const ObjParams& ob, long long unit, const float2* gin,
                              const uint64_t* smask, float2* X, float2* Y, int xs, int t, int slot) {
    const int W = ob.W, x0 = ob.x0;
    const float* phi = prm.phi + ob.phi_off + unit * ob.phi_unit + ob.phi_org;
    float* gphi = prm.gphi + ob.phi_off + unit * ob.phi_unit + ob.phi_org;
    // B1: inverse column transforms of G (columns 0 and 32 packed)
    if (t < 32) {
        float2 col[kN];
        if (t == 0) {
#pragma unroll
            for (int ky = 0; ky < kN; ++ky) {
                const float2 a = gin[ky * kNH], b = gin[ky * kNH + 32];
                col[ky] = make_float2(a.x - b.y, a.y + b.x);
            }
        } else {
#pragma unroll
            for (int ky = 0; ky < kN; ++ky) col[ky] = gin[ky * kNH + t];
        }
        fftreg::fft<kN, +1>(col);
        if (t == 0) {
#pragma unroll
            for (int y = 0; y < kN; ++y) {
                Y[y * kNH] = make_float2(col[y].x, 0.f);
                Y[y * kNH + 32] = make_float2(col[y].y, 0.f);
            }
        } else {
#pragma unroll
            for (int y = 0; y < kN; ++y) Y[y * kNH + t] = col[y];
        }
    }
    slot_sync(slot);
    // B2: complex-to-real row transforms -> g_q = 2 Re F^H G / (N^2 n_pup),
    // written over the thread's own row of Y as float pairs
    {
        float2 xh[kNH];
#pragma unroll
        for (int kx = 0; kx < kNH; ++kx) xh[kx] = Y[t * kNH + kx];
        float g[kN];
        fftreg::irfft<kN>(xh, g);
        const float sc = 2.0f * ob.inv_z;
#pragma unroll
        for (int i = 0; i < kN / 2; ++i) Y[t * kNH + i] = make_float2(g[2 * i] * sc, g[2 * i + 1] * sc);
    }
    // F1r: recompute the pupil column transforms
    if (t < W) pupil_columns(ob, phi, smask, X, xs, t);
    slot_sync(slot);
    // F2r: field row, G_p = g_q p, inverse row transform, keep box columns
    {
        float2 row[kN];
        field_row(ob, X, xs, t, row);
#pragma unroll
        for (int i = 0; i < kN / 2; ++i) {
            const float2 q = Y[t * kNH + i];
            row[2 * i] = cscale(row[2 * i], q.x);
            row[2 * i + 1] = cscale(row[2 * i + 1], q.y);
        }
        fftreg::fft<kN, +1>(row);
#pragma unroll
        for (int x = 0; x < kN; ++x)
            if ((unsigned)(x - x0) < (unsigned)W) X[t * xs + (x - x0)] = row[x];
    }
    slot_sync(slot);
    // B3: inverse column transforms on box columns -> dL/dphi on the pupil
    if (t < W) {
        float2 col[kN];
#pragma unroll
        for (int ky = 0; ky < kN; ++ky) col[ky] = X[ky * xs + t];
        fftreg::fft<kN, +1>(col);
#pragma unroll
        for (int y = 0; y < kN; ++y) X[y * xs + t] = col[y];
        for (int yy = 0; yy < W; ++yy) {
            float gv = 0.f;
            if ((smask[yy] >> t) & 1ull) {
                const float2 pv = pupil_value(phi[yy * ob.phi_ld + t]);
                const float2 gp = X[(x0 + yy) * xs + t];
                gv = 2.0f * (pv.x * gp.y - pv.y * gp.x);
            }
            gphi[yy * ob.phi_ld + t] = gv;
        }
    }
}

// Per-object frame reduction: O, loss terms, adjoint seeds G_j (over H_j).
// The residual r_j = D_j - O H_j is formed in FP32. Where the fit leaves
// little residual energy (sum_j w|r_j|^2 < kCancel sum_j w|D_j|^2, estimated
// from E - |N|^2/Q), r_j cancels badly in FP32 (for J = 1, r = D gamma / Q
// everywhere the OTF is large), so that frequency is redone with N, O and
// r_j in FP64. With several frames this triggers at DC and little else.
constexpr float kCancel = 1e-3f;

__device__ double reduce_object(const FusedParams& prm, int p, int k, const uint64_t* ssupp, float2* hbase) {
    const int J = prm.J;
    const size_t unit0 = ((size_t)p * prm.K + k) * J;
    const size_t dstride = (size_t)kN * prm.spec_ld;
    const float2* dbase = prm.spectra + unit0 * dstride;
    const float* w = prm.weights + (size_t)k * J;
    double acc = 0.0;
    for (int f = threadIdx.x; f < kHalf; f += blockDim.x) {
        const int ky = f / kNH, kx = f - ky * kNH;
        const size_t doff = (size_t)ky * prm.spec_ld + kx;
        const float2* dp = dbase + doff;
        float2* hp = hbase + f;
        float2 num = make_float2(0.f, 0.f);
        float e = 0.f;
        double q = 0.0;
#pragma unroll 4
        for (int j = 0; j < J; ++j) {
            const float2 d = dp[(size_t)j * dstride];
            const float2 h = hp[(size_t)j * kHalf];
            const float wj = w[j];
            num.x += wj * (d.x * h.x + d.y * h.y);
            num.y += wj * (d.y * h.x - d.x * h.y);
            e += wj * (d.x * d.x + d.y * d.y);
            q += (double)wj * ((double)h.x * h.x + (double)h.y * h.y);
        }
        q += prm.gamma;
        const float invq = (float)(1.0 / q);
        float2 o = cscale(num, invq);
        const bool seed = (f != 0) && ((ssupp[ky] >> kx) & 1ull);
        const float t_est = e - (num.x * num.x + num.y * num.y) * invq;
        float t;
        if (!(t_est < kCancel * e)) {
            float tsum = 0.f;
#pragma unroll 4
            for (int j = 0; j < J; ++j) {
                const float2 d = dp[(size_t)j * dstride];
                const float2 h = hp[(size_t)j * kHalf];
                const float wj = w[j];
                const float2 r = csub(d, cmul(o, h));
                tsum += wj * (r.x * r.x + r.y * r.y);
                hp[(size_t)j * kHalf] = seed ? cscale(cmul(cconj(o), r), -wj) : make_float2(0.f, 0.f);
            }
            t = tsum + (float)prm.gamma * (o.x * o.x + o.y * o.y);
        } else {
            double nx = 0.0, ny = 0.0;
            for (int j = 0; j < J; ++j) {
                const float2 d = dp[(size_t)j * dstride];
                const float2 h = hp[(size_t)j * kHalf];
                const double wj = w[j];
                nx += wj * ((double)d.x * h.x + (double)d.y * h.y);
                ny += wj * ((double)d.y * h.x - (double)d.x * h.y);
            }
            const double ox = nx / q, oy = ny / q;
            double tsum = 0.0;
            for (int j = 0; j < J; ++j) {
                const float2 d = dp[(size_t)j * dstride];
                const float2 h = hp[(size_t)j * kHalf];
                const double wj = w[j];
                const double rx = (double)d.x - (ox * h.x - oy * h.y);
                const double ry = (double)d.y - (ox * h.y + oy * h.x);
                tsum += wj * (rx * rx + ry * ry);
                // G = -w conj(O) r
                hp[(size_t)j * kHalf] =
                    seed ? make_float2((float)(-wj * (ox * rx + oy * ry)), (float)(-wj * (ox * ry - oy * rx)))
                         : make_float2(0.f, 0.f);
            }
            t = (float)(tsum + prm.gamma * (ox * ox + oy * oy));
            o = make_float2((float)ox, (float)oy);
        }
        const double wt = (kx == 0 || kx == kN / 2) ? 1.0 : 2.0;
        acc += wt * (double)t;
        if (prm.object) {
            float2* ob = prm.object + ((size_t)p * prm.K + k) * dstride;
            ob[doff] = o;
            if (prm.spec_ld == kN && kx > 0 && kx < kN / 2)
                ob[(size_t)((kN - ky) % kN) * kN + (kN - kx)] = cconj(o);
        }
    }
    return acc;
}

__device__ double block_sum(double v, double* sred) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sred[warp] = v;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += sred[i];
    return tot;
}

__global__ void __launch_bounds__(kThreadsMax, 1)
    mfbd_fused_kernel(const FusedParams prm, int mode, int xs) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t smask[kN];
    __shared__ uint64_t ssupp[kN];
    __shared__ double sred[32];
    const int tid = threadIdx.x;
    const int slot = tid >> 6, t = tid & 63;
    const int slots = blockDim.x >> 6;
    const size_t slot_bytes = (size_t)kN * xs * sizeof(float2) + (size_t)kN * kNH * sizeof(float2);
    float2* X = reinterpret_cast<float2*>(smem + slot * slot_bytes);
    float2* Y = X + kN * xs;
    const int J = prm.J;

    for (int p = blockIdx.x; p < prm.P; p += gridDim.x) {
        double lacc = 0.0;
        for (int k = 0; k < prm.K; ++k) {
            const ObjParams& ob = prm.obj[k];
            __syncthreads();
            if (tid < kN) {
                smask[tid] = tid < ob.W ? ob.mask[tid] : 0ull;
                ssupp[tid] = ob.supp[tid];
            }
            __syncthreads();
            const size_t unit0 = ((size_t)p * prm.K + k) * J;
            float2* hscr = prm.scratch_ring ? prm.gscr + (size_t)blockIdx.x * J * kHalf : prm.gscr + unit0 * kHalf;
            if (mode != MODE_BWD) {
                for (int j0 = 0; j0 < J; j0 += slots) {
                    const int j = j0 + slot;
                    if (j < J)
                        forward_unit(prm, ob, (long long)p * J + j, hscr + (size_t)j * kHalf, smask, ssupp,
                                     X, Y, xs, t, slot);
                }
                __syncthreads();
                if (mode != MODE_OTF) lacc += reduce_object(prm, p, k, ssupp, hscr);
                __syncthreads();
            }
            if (mode == MODE_BWD || mode == MODE_FUSED) {
                for (int j0 = 0; j0 < J; j0 += slots) {
                    const int j = j0 + slot;
                    if (j < J)
                        backward_unit(prm, ob, (long long)p * J + j, hscr + (size_t)j * kHalf, smask, X, Y,
                                      xs, t, slot);
                }
            }
        }
        if (mode == MODE_FWD || mode == MODE_FUSED) {
            const double tot = block_sum(lacc, sred);
            if (tid == 0) prm.loss[p] = tot;
        }
    }
}

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

// grad[u][m] (+)= scale * sum_i gphi[u][i] basis[m][i]
__global__ void __launch_bounds__(256) grad_gemm_kernel(const float* __restrict__ gphi, int U, int npix,
                                                        const float* __restrict__ basis, int M, float scale,
                                                        int accumulate, float* __restrict__ grad) {
    __shared__ float As[16][68];
    __shared__ float Bs[16][68];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int u0 = blockIdx.y * 64, m0 = blockIdx.x * 64;
    float acc[4][4] = {};
    for (int i0 = 0; i0 < npix; i0 += 16) {
        for (int idx = threadIdx.x; idx < 16 * 64; idx += 256) {
            const int rr = idx >> 4, ii = idx & 15;
            const int u = u0 + rr, m = m0 + rr, i = i0 + ii;
            As[ii][rr] = (u < U && i < npix) ? gphi[(size_t)u * npix + i] : 0.f;
            Bs[ii][rr] = (m < M && i < npix) ? basis[(size_t)m * npix + i] : 0.f;
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
            if (m >= M) continue;
            float v = scale * acc[r][c];
            if (accumulate) v += grad[(size_t)u * M + m];
            grad[(size_t)u * M + m] = v;
        }
    }
}

}  // namespace

FusedGeometry fused_geometry(int max_box) {
    FusedGeometry g;
    g.xs = max_box | 1;
    const size_t slot_bytes = (size_t)kN * g.xs * sizeof(float2) + (size_t)kN * kNH * sizeof(float2);
    int slots = (int)((216u * 1024u) / slot_bytes);
    if (slots > kMaxSlots) slots = kMaxSlots;
    if (slots < 1) slots = 1;
    g.slots = slots;
    g.smem_bytes = slot_bytes * slots;
    return g;
}

int max_ctas_per_sm(const FusedGeometry& g) {
    int n = 0;
    if (cudaFuncSetAttribute(mfbd_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)g.smem_bytes) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, mfbd_fused_kernel, g.slots * 64, g.smem_bytes) !=
        cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_fused(const FusedParams& prm, int mode, const FusedGeometry& g, int ctas, cudaStream_t s) {
    if (prm.P == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(mfbd_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)g.smem_bytes);
    if (e != cudaSuccess) return e;
    mfbd_fused_kernel<<<ctas, g.slots * 64, g.smem_bytes, s>>>(prm, mode, g.xs);
    return cudaGetLastError();
}

cudaError_t launch_phase_gemm(const float* a, int U, int M, const float* basis, int npix, float scale,
                              float* phase, cudaStream_t s) {
    if (U == 0) return cudaSuccess;
    dim3 grid((npix + 63) / 64, (U + 63) / 64);
    phase_gemm_kernel<<<grid, 256, 0, s>>>(a, U, M, basis, npix, scale, phase);
    return cudaGetLastError();
}

cudaError_t launch_grad_gemm(const float* gphi, int U, int npix, const float* basis, int M, float scale,
                             int accumulate, float* grad, cudaStream_t s) {
    if (U == 0) return cudaSuccess;
    dim3 grid((M + 63) / 64, (U + 63) / 64);
    grad_gemm_kernel<<<grid, 256, 0, s>>>(gphi, U, npix, basis, M, scale, accumulate, grad);
    return cudaGetLastError();
}

}  // namespace mfbd_dev
