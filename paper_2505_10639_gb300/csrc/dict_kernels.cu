// The spatially variant PSF model on a dictionary (Sec. 2.2.2, "Spatially
// variant convolution"): the PSF at object point r' is sum_i a_i(r') phi_i,
// the image of object k in frame j is sum_i (o_k a_ikj) * phi_i, and the data
// term of the log-posterior in the Fourier domain is
//   L = sum_kj gamma_kj sum_u |I_kj(u) - sum_i F(o_k a_ikj)(u) Phi_i(u)|^2
// (full frequency plane). With R_kj = I_kj - sum_i F(o_k a_ikj) Phi_i and
// g_ikj = Re F^H[conj(Phi_i) (-2 gamma_kj R_kj)] (F^H unnormalised):
//   dL/da_ikj = o_k g_ikj,  dL/do_k = sum_j sum_i a_ikj g_ikj.
//
// dict_unit_kernel: one warp per unit (patch, object, frame), N = 64.
//   Forward, per atom i: lane y forms rows y and y + N/2 of o a_i as one
//   complex line (16-byte loads), transforms it and splits it into the two
//   rows' half spectra (the real columns 0 and N/2 stored packed as one
//   complex column); lane kx transforms half-spectrum column kx (lane 0 the
//   packed column, which it leaves in shared memory for all lanes to split,
//   two rows each) and accumulates X_i Phi_i into the unit's model spectrum
//   in shared memory. Then the residual, the unit's loss (FP64 sums of FP32
//   terms; columns 0 and N/2 once, the others twice) and G = -2 gamma R in
//   place of the model.
//   Backward, per atom i: the inverse of the half spectrum conj(Phi_i) G
//   (columns along ky, 0 and N/2 packed, then Hermitian-extended row pairs,
//   as the mosaic's object images) gives rows y and y + N/2 of g_i in lane
//   y: dL/da_i = o g_i is stored (16-byte stores), and a_i g_i accumulated
//   into the unit's share of dL/do in shared memory, written out at the end.
// dict_combine_kernel: dL/do_k = the units' shares summed over frames in
// frame order; the patch loss = the units' losses summed over (k, j) in order.
#include "../../include/mfbd.h"
#include "mfbd_internal.h"
#include "unit_passes.cuh"

#include <cuda_runtime.h>

#include <cstdint>

using namespace mfbd_dev;

namespace {

using namespace mfbd_dev::unitpass;

constexpr int kDN = 64, kDNH = kDN / 2 + 1, kDES = kDNH;  // exchange stride 33 (odd)
constexpr int kDoLd = kDN + 1;                             // dL/do rows, padded
// shared memory of one unit: exchange buffer, model / G spectrum, dL/do share,
// lane 0's packed column
constexpr size_t kDictSmem = 2 * (size_t)kDN * kDES * sizeof(float2) + (size_t)kDN * kDoLd * sizeof(float) +
                             (size_t)kDN * sizeof(float2);

struct DictParams {
    int P, K, J, M;
    const float2* atom_otf;  // [M][N][NH]
    const float* gamma;      // [K][J]
    const float* object;     // [P][K][N][N]
    const float* coeff;      // [P][K][J][M][N][N]
    const float2* spectra;   // [P][K][J][N][NH]
    float* grad_coeff;       // [P][K][J][M][N][N] or null
    float* unit_gobj;        // [P][K][J][N][N] or null (workspace)
    double* unit_loss;       // [P][K][J] (workspace)
};

// rows y and y + N/2 of o a (a = 0: o alone is not needed) as one complex line
__device__ __forceinline__ void load_product_rows(const float* o, const float* a, int y, float2 (&v)[kDN]) {
    const float4* o0 = reinterpret_cast<const float4*>(o + y * kDN);
    const float4* o1 = reinterpret_cast<const float4*>(o + (y + kDN / 2) * kDN);
    const float4* a0 = reinterpret_cast<const float4*>(a + y * kDN);
    const float4* a1 = reinterpret_cast<const float4*>(a + (y + kDN / 2) * kDN);
#pragma unroll
    for (int c = 0; c < kDN / 4; ++c) {
        const float4 p = o0[c], q = o1[c], s = a0[c], t = a1[c];
        v[4 * c] = make_float2(p.x * s.x, q.x * t.x);
        v[4 * c + 1] = make_float2(p.y * s.y, q.y * t.y);
        v[4 * c + 2] = make_float2(p.z * s.z, q.z * t.z);
        v[4 * c + 3] = make_float2(p.w * s.w, q.w * t.w);
    }
}

}  // namespace

namespace {

__global__ void __launch_bounds__(32) dict_unit_kernel(const DictParams prm) {
    extern __shared__ __align__(16) unsigned char dsm[];
    float2* E = reinterpret_cast<float2*>(dsm);             // [N][33] exchange
    float2* A = E + kDN * kDES;                               // [N][33] model spectrum, then G
    float* DO = reinterpret_cast<float*>(A + kDN * kDES);     // [N][65] the unit's share of dL/do
    float2* Z = reinterpret_cast<float2*>(DO + kDN * kDoLd);  // [N] a packed column
    const int lane = threadIdx.x;
    const long long units = (long long)prm.P * prm.K * prm.J;
    const bool backward = prm.grad_coeff != nullptr || prm.unit_gobj != nullptr;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        const int j = (int)(u % prm.J);
        const long long pk = u / prm.J;
        const int k = (int)(pk % prm.K);
        const float* o = prm.object + (size_t)pk * kDN * kDN;
        const float* a = prm.coeff + (size_t)u * prm.M * kDN * kDN;
        const float2* I = prm.spectra + (size_t)u * kDN * kDNH;
        const float gam = prm.gamma[k * prm.J + j];
        for (int e = lane; e < kDN * kDES; e += 32) A[e] = make_float2(0.f, 0.f);
        __syncwarp();
        // ------------------------------------------- model: sum_i F(o a_i) Phi_i
        for (int i = 0; i < prm.M; ++i) {
            const float2* Phi = prm.atom_otf + (size_t)i * kDN * kDNH;
            float2 v[kDN];
            load_product_rows(o, a + (size_t)i * kDN * kDN, lane, v);
            line_fft<kDN, -1>(v, 0);
            // rows y, y + N/2: their half spectra; columns 0 and N/2 packed in column 0
            E[lane * kDES] = make_float2(v[0].x, v[kDN / 2].x);
            E[(lane + kDN / 2) * kDES] = make_float2(v[0].y, v[kDN / 2].y);
            fftreg::static_for<1, kDN / 2>([&](auto kk) {
                constexpr int kq = decltype(kk)::value;
                const float2 pc = conj_partner<kDN, kq>(v);
                const float2 ra = cscale(cadd(v[kq], pc), 0.5f);
                const float2 d = cscale(csub(v[kq], pc), 0.5f);
                E[lane * kDES + kq] = ra;
                E[(lane + kDN / 2) * kDES + kq] = make_float2(d.y, -d.x);
            });
            __syncwarp();
#pragma unroll
            for (int ky = 0; ky < kDN; ++ky) v[ky] = E[ky * kDES + lane];
            __syncwarp();
            line_fft<kDN, -1>(v, 0);
            // lanes 1 .. 31 accumulate their column; lane 0 leaves the packed one
#pragma unroll
            for (int ky = 0; ky < kDN; ++ky) {
                const float2 ph = Phi[ky * kDNH + lane];
                if (lane > 0) {
                    float2* acc = &A[ky * kDES + lane];
                    *acc = cadd(*acc, cmul(v[ky], ph));
                } else {
                    Z[ky] = v[ky];
                }
            }
            __syncwarp();
            // X(ky, 0) = (Z[ky] + conj Z[-ky]) / 2, X(ky, N/2) = (Z[ky] - conj Z[-ky]) / (2i)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int ky = lane + h * (kDN / 2);
                const float2 z = Z[ky], zp = cconj(Z[(kDN - ky) & (kDN - 1)]);
                const float2 x0 = cscale(cadd(z, zp), 0.5f);
                const float2 d = cscale(csub(z, zp), 0.5f);
                const float2 xh = make_float2(d.y, -d.x);
                A[ky * kDES] = cadd(A[ky * kDES], cmul(x0, Phi[ky * kDNH]));
                A[ky * kDES + kDN / 2] = cadd(A[ky * kDES + kDN / 2], cmul(xh, Phi[ky * kDNH + kDN / 2]));
            }
            __syncwarp();
        }
        // --------------------------------- residual, loss, G = -2 gamma R in A
        double lacc = 0.0;
        if (lane > 0) {
#pragma unroll 8
            for (int ky = 0; ky < kDN; ++ky) {
                const float2 d = I[ky * kDNH + lane], m = A[ky * kDES + lane];
                const float2 r = make_float2(d.x - m.x, d.y - m.y);
                lacc += 2.0 * (double)(r.x * r.x + r.y * r.y);
                A[ky * kDES + lane] = cscale(r, -2.f * gam);
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int ky = lane + h * (kDN / 2);
#pragma unroll
            for (int c = 0; c <= kDN / 2; c += kDN / 2) {
                const float2 d = I[ky * kDNH + c], m = A[ky * kDES + c];
                const float2 r = make_float2(d.x - m.x, d.y - m.y);
                lacc += (double)(r.x * r.x + r.y * r.y);
                A[ky * kDES + c] = cscale(r, -2.f * gam);
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) lacc += __shfl_xor_sync(0xffffffffu, lacc, off);
        if (lane == 0) prm.unit_loss[u] = (double)gam * lacc;
        __syncwarp();
        if (!backward) continue;
        // ------------------------------ g_i = F^H[conj(Phi_i) G] (real), per atom
        float* const gobj = prm.unit_gobj;
        if (gobj)
            for (int e = lane; e < kDN * kDoLd; e += 32) DO[e] = 0.f;
        for (int i = 0; i < prm.M; ++i) {
            const float2* Phi = prm.atom_otf + (size_t)i * kDN * kDNH;
            const float* ai = a + (size_t)i * kDN * kDN;
            // the packed real columns: conj(V(ky, 0) + i V(ky, N/2)), two rows a lane
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int ky = lane + h * (kDN / 2);
                const float2 va = cmul(cconj(Phi[ky * kDNH]), A[ky * kDES]);
                const float2 vb = cmul(cconj(Phi[ky * kDNH + kDN / 2]), A[ky * kDES + kDN / 2]);
                Z[ky] = make_float2(va.x - vb.y, -(va.y + vb.x));
            }
            __syncwarp();
            // columns along ky: F^H x = conj(F conj x); lane 0 the packed columns
            float2 v[kDN];
#pragma unroll
            for (int ky = 0; ky < kDN; ++ky) {
                const float2 vv = cmul(cconj(Phi[ky * kDNH + lane]), A[ky * kDES + lane]);
                const float2 zz = Z[ky];
                v[ky] = lane > 0 ? cconj(vv) : zz;
            }
            line_fft<kDN, -1>(v, 0);
#pragma unroll
            for (int ky = 0; ky < kDN; ++ky) E[ky * kDES + lane] = cconj(v[ky]);
            __syncwarp();
            // rows y and y + N/2: F^H of the Hermitian-extended rows, packed as
            // T_y + i T_(y+N/2) (both results real)
            const int y = lane;
#pragma unroll
            for (int x = 0; x < kDN; ++x) {
                float2 p, q;
                if (x == 0) {
                    p = make_float2(E[y * kDES].x, 0.f);
                    q = make_float2(E[(y + kDN / 2) * kDES].x, 0.f);
                } else if (x == kDN / 2) {
                    p = make_float2(E[y * kDES].y, 0.f);
                    q = make_float2(E[(y + kDN / 2) * kDES].y, 0.f);
                } else if (x < kDN / 2) {
                    p = E[y * kDES + x];
                    q = E[(y + kDN / 2) * kDES + x];
                } else {
                    p = cconj(E[y * kDES + kDN - x]);
                    q = cconj(E[(y + kDN / 2) * kDES + kDN - x]);
                }
                v[x] = make_float2(p.x - q.y, -(p.y + q.x));  // conj(p + i q)
            }
            line_fft<kDN, -1>(v, 0);
            // v[x].x = g_i(y, x), -v[x].y = g_i(y + N/2, x)
            const float4* o0 = reinterpret_cast<const float4*>(o + y * kDN);
            const float4* o1 = reinterpret_cast<const float4*>(o + (y + kDN / 2) * kDN);
            const float4* a0 = reinterpret_cast<const float4*>(ai + y * kDN);
            const float4* a1 = reinterpret_cast<const float4*>(ai + (y + kDN / 2) * kDN);
            float4* gc0 = prm.grad_coeff ? reinterpret_cast<float4*>(prm.grad_coeff + ((size_t)u * prm.M + i) * kDN * kDN + y * kDN) : nullptr;
            float4* gc1 = gc0 ? gc0 + (kDN / 2) * kDN / 4 : nullptr;
#pragma unroll
            for (int c = 0; c < kDN / 4; ++c) {
                const float g0[4] = {v[4 * c].x, v[4 * c + 1].x, v[4 * c + 2].x, v[4 * c + 3].x};
                const float g1[4] = {-v[4 * c].y, -v[4 * c + 1].y, -v[4 * c + 2].y, -v[4 * c + 3].y};
                if (gc0) {
                    const float4 p = o0[c], q = o1[c];
                    gc0[c] = make_float4(p.x * g0[0], p.y * g0[1], p.z * g0[2], p.w * g0[3]);
                    gc1[c] = make_float4(q.x * g1[0], q.y * g1[1], q.z * g1[2], q.w * g1[3]);
                }
                if (gobj) {
                    const float4 s = a0[c], t = a1[c];
                    float* d0 = DO + y * kDoLd + 4 * c;
                    float* d1 = DO + (y + kDN / 2) * kDoLd + 4 * c;
                    d0[0] = fmaf(s.x, g0[0], d0[0]);
                    d0[1] = fmaf(s.y, g0[1], d0[1]);
                    d0[2] = fmaf(s.z, g0[2], d0[2]);
                    d0[3] = fmaf(s.w, g0[3], d0[3]);
                    d1[0] = fmaf(t.x, g1[0], d1[0]);
                    d1[1] = fmaf(t.y, g1[1], d1[1]);
                    d1[2] = fmaf(t.z, g1[2], d1[2]);
                    d1[3] = fmaf(t.w, g1[3], d1[3]);
                }
            }
            __syncwarp();  // E and Z free for the next atom
        }
        if (gobj) {
            float* out = gobj + (size_t)u * kDN * kDN;
            for (int e = lane; e < kDN * kDN; e += 32) out[e] = DO[(e / kDN) * kDoLd + (e % kDN)];
        }
        __syncwarp();
    }
}

// dL/do_k = sum_j of the units' shares (frame order); loss_p = sum_kj of the
// units' losses (in order). One CTA per patch.
__global__ void __launch_bounds__(256) dict_combine_kernel(int K, int J, const double* __restrict__ unit_loss,
                                                           const float* __restrict__ unit_gobj,
                                                           float* __restrict__ grad_object, double* __restrict__ loss) {
    const int p = blockIdx.x;
    if (grad_object) {
        const int per = K * kDN * kDN;
        for (int e = threadIdx.x; e < per; e += blockDim.x) {
            const int k = e / (kDN * kDN), r = e - k * kDN * kDN;
            const float* src = unit_gobj + (((size_t)p * K + k) * J) * kDN * kDN + r;
            float s = 0.f;
            for (int j = 0; j < J; ++j) s += src[(size_t)j * kDN * kDN];
            grad_object[(size_t)p * per + e] = s;
        }
    }
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int e = 0; e < K * J; ++e) s += unit_loss[(size_t)p * K * J + e];
        loss[p] = s;
    }
}

}  // namespace

namespace {

// workspace: the units' losses, then (256-byte aligned) their dL/do shares
size_t dict_gobj_offset(long long units) { return ((size_t)units * sizeof(double) + 255) & ~(size_t)255; }

int dict_check_desc(const mfbd_dict_desc* d) {
    if (!d) return set_error(MFBD_ERR_INVALID_ARG, "dictionary descriptor is NULL");
    if (d->n_patches < 0 || d->n_objects < 1 || d->n_frames < 1 || d->n_atoms < 1)
        return set_error(MFBD_ERR_INVALID_ARG, "dictionary sizes: n_patches >= 0, n_objects, n_frames, n_atoms >= 1");
    if (d->n != kDN) return set_error(MFBD_ERR_UNSUPPORTED, "the dictionary model supports n = 64");
    if ((long long)d->n_patches * d->n_objects * d->n_frames * d->n_atoms > (1ll << 40))
        return set_error(MFBD_ERR_INVALID_ARG, "dictionary problem too large");
    return MFBD_OK;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

}  // namespace

extern "C" size_t mfbd_dict_workspace_bytes(const mfbd_dict_desc* desc) {
    if (dict_check_desc(desc) != MFBD_OK) return 0;
    const long long units = (long long)desc->n_patches * desc->n_objects * desc->n_frames;
    return dict_gobj_offset(units) + (size_t)units * kDN * kDN * sizeof(float);
}

extern "C" int mfbd_dict_loss_grad(const mfbd_dict_desc* desc, const void* atom_otf, const float* gamma,
                                   const float* object, const float* coeff, const void* spectra, void* workspace,
                                   double* loss, float* grad_object, float* grad_coeff, void* stream) {
    int st = dict_check_desc(desc);
    if (st != MFBD_OK) return st;
    const long long units = (long long)desc->n_patches * desc->n_objects * desc->n_frames;
    if (units == 0) return MFBD_OK;
    if (!atom_otf || !gamma || !object || !coeff || !spectra || !workspace || !loss)
        return set_error(MFBD_ERR_INVALID_ARG, "a required dictionary-model pointer is NULL");
    if (!aligned(object, 16) || !aligned(coeff, 16) || (grad_coeff && !aligned(grad_coeff, 16)) ||
        !aligned(workspace, 16) || !aligned(atom_otf, 8) || !aligned(spectra, 8) || !aligned(loss, 8) ||
        (grad_object && !aligned(grad_object, 4)))
        return set_error(MFBD_ERR_INVALID_ARG,
                         "object, coeff, grad_coeff and workspace need 16-byte alignment; atom_otf, spectra, loss 8");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(dict_unit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDictSmem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dict_unit_kernel, 32, kDictSmem);
    if (e != cudaSuccess) return set_cuda_error(e, "mfbd_dict_loss_grad setup");
    if (per_sm < 1) return set_error(MFBD_ERR_UNSUPPORTED, "the dictionary kernel does not fit an SM");
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    DictParams prm;
    prm.P = desc->n_patches;
    prm.K = desc->n_objects;
    prm.J = desc->n_frames;
    prm.M = desc->n_atoms;
    prm.atom_otf = static_cast<const float2*>(atom_otf);
    prm.gamma = gamma;
    prm.object = object;
    prm.coeff = coeff;
    prm.spectra = static_cast<const float2*>(spectra);
    prm.grad_coeff = grad_coeff;
    prm.unit_loss = reinterpret_cast<double*>(ws);
    prm.unit_gobj = grad_object ? reinterpret_cast<float*>(ws + dict_gobj_offset(units)) : nullptr;
    long long ctas = (long long)sms * per_sm;
    if (ctas > units) ctas = units;
    dict_unit_kernel<<<(int)ctas, 32, kDictSmem, s>>>(prm);
    if ((e = cudaGetLastError()) != cudaSuccess) return set_cuda_error(e, "dict_unit_kernel launch");
    dict_combine_kernel<<<desc->n_patches, 256, 0, s>>>(prm.K, prm.J, prm.unit_loss, prm.unit_gobj, grad_object,
                                                        loss);
    if ((e = cudaGetLastError()) != cudaSuccess) return set_cuda_error(e, "dict_combine_kernel launch");
    return MFBD_OK;
}
