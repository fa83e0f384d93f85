// Internal launch interface between the C-ABI layer and the kernels.
#pragma once

#include <cuda.h>  // CUtensorMap
#include <cuda_runtime.h>
#include <cstdint>

namespace mfbd_dev {

constexpr int kMaxObjects = 8;
constexpr int kN = 64;                  // patch size supported by the fused kernel
constexpr int kNH = kN / 2 + 1;         // 33 half-spectrum columns
constexpr int kHalf = kN * kNH;         // 2112 half-spectrum frequencies
constexpr int kFusedFrames = 12;        // frames of a (patch, object) pair the fused kernel holds

// Fused-kernel modes.
enum Mode : int { MODE_FWD = 0, MODE_BWD = 1, MODE_FUSED = 2, MODE_OTF = 3 };

struct ObjParams {
    int W;                   // side of the pupil's bounding box
    int x0;                  // first row/column of the box
    float inv_z;             // 1 / (N^2 n_pup): PSF normalisation (Parseval)
    long long phi_off;       // float offset of this object's phase block
    long long phi_unit;      // floats per (patch, frame) phase image: W*W (box) or N*N (full grid)
    int phi_org;             // offset of the box's first pixel in that image: 0 or x0*N + x0
    int phi_ld;              // row stride of that image: W or N
    const uint64_t* mask;    // [W] rows, bit t = pupil pixel at box column t
    const uint64_t* supp;    // [N] rows, bit kx = OTF support (kx <= N/2)
    const uint64_t* cmask;   // [N] box columns c, bit y = pupil pixel at box (y, c); 0 for c >= W
    const uint64_t* csupp;   // [N] columns kx <= N/2, bit ky = OTF support; the rest 0
};

struct FusedParams {
    int P, K, J, M;
    double gamma;
    const float* weights;     // [K][J]
    const float* phi;         // phases, per object [P*J][W*W] at phi_off
    float* gphi;              // dL/dphi, same layout
    float2* gscr;             // [P][K][J][N][N/2+1]: OTF, then dL/dconj(H)
    float2* pscr;             // [P][K][J][N x N]: field p = F P, stored [x][y] (null: not kept)
    float2* uscr;             // [P][K][J][ustride]: pupil phasors exp(i phi) on the box (null: not kept)
    int ustride;              // complex elements per unit in uscr (>= W_k^2 for every object)
    const float2* spectra;    // D
    int spec_ld;              // row stride of D and O in complex elements (33 or 64)
    double* loss;             // [P]
    float2* object;           // [P][K][N][spec_ld] or null
    int rsplit;               // warps per (patch, object) of the frame reduction (<= 1: one)
    double* lpart;            // rsplit > 1: per-split patch losses [P][rsplit]
    const float2* oin;        // object-inferring loss: the given objects [P][K][N][spec_ld], else null
    float2* gobj;             // with oin: dL/dconj(O) [P][K][N][spec_ld], or null
    float2* fscr;             // fused kernel: per CTA and frame slot rows N/2.. of the field p [ctas][kFusedFrames][N x N/2]
    double* lpair;            // fused kernel: per (patch, object) losses [P][K]
    int* lcnt;                // fused kernel: per patch, the objects done [P] (0 between calls)
    int* fticket;             // fused kernel: [0] next-pair ticket, [1] CTAs done (0 between calls)
    int korder[kMaxObjects];  // fused kernel: objects in the order their pairs are dealt
    ObjParams obj[kMaxObjects];
};

// Fused kernel geometry for the largest pupil box of a plan.
struct FusedGeometry {
    int slots;          // warps per CTA of the pass kernels; each works on one frame at a time
    size_t smem_bytes;  // dynamic shared memory per CTA
    int xs;             // row stride (complex elements) of a warp's exchange buffer
};

FusedGeometry fused_geometry(int max_box);

// The three kernels of an evaluation (`sms` is the device's SM count):
// forward passes (OTF, field), frame reduction (loss, object, adjoint
// seeds), adjoint passes (dL/dphi).
cudaError_t launch_forward_passes(const FusedParams& prm, const FusedGeometry& g, int sms, cudaStream_t s);
cudaError_t launch_reduction(const FusedParams& prm, int sms, cudaStream_t s);
cudaError_t launch_adjoint_passes(const FusedParams& prm, const FusedGeometry& g, int sms, cudaStream_t s);
// The kernels of `mode` in order (FWD: forward + reduction; BWD: adjoint;
// FUSED: all three; OTF: forward only).
cudaError_t launch_fused(const FusedParams& prm, int mode, const FusedGeometry& g, int sms, cudaStream_t s);

// The fused evaluation (fused_kernels.cu): one persistent launch in which
// a CTA of kFusedFrames warps carries one (patch, object) pair at a time
// through the forward passes, the frame reduction and the adjoint passes,
// then a small kernel sums the pair losses per patch. Needs J <= kFusedFrames
// and an exchange-buffer stride es of 33 or 37 (pupil boxes up to 37 px);
// fscr holds ctas x kFusedFrames fields, lpair P x K losses.
size_t fused_pair_smem(int es);
bool fused_pair_supported(int J, int es);
int fused_pair_ctas_per_sm(int es);
cudaError_t launch_fused_pairs(const FusedParams& prm, int es, int ctas, cudaStream_t s);

// phase[u][i] += div[u mod J][i] for U units (U a multiple of J): the
// known diversity phases of the J frames added to every patch's phases.
cudaError_t launch_add_diversity(float* phase, const float* div, int U, int J, int npix, int sms, cudaStream_t s);

// phase[u][i] = scale * sum_m a[u][m] basis[m][i]  (u < U, i < npix)
cudaError_t launch_phase_gemm(const float* a, int U, int M, const float* basis, int npix,
                              float scale, float* phase, cudaStream_t s);

// The same on the tensor cores (tcgen05, BF16 operands, FP32 accumulation).
// launch_split_coeffs writes the coefficients as `planes` BF16 planes (3:
// FP32-accurate split, 1: BF16) in the MMA tile layout (split_coeffs_elems
// elements); bt holds the basis the same way in 128-pixel tiles; err is set
// when an MMA wait gives up. phase_mma_smem: dynamic shared memory of a CTA.
size_t phase_mma_smem(int M, int planes);
size_t split_coeffs_elems(int U, int M, int planes);
cudaError_t launch_split_coeffs(const float* a, int U, int M, int planes, uint16_t* at, cudaStream_t s);
// One launch for the K objects: bt[k] the basis planes of object k (npix[k]
// pixels), phase[k] its [U][npix[k]] output, scaled by scale[k].
cudaError_t launch_phase_mma(const uint16_t* at, int U, int M, int K, const uint16_t* const* bt, const int* npix,
                             int planes, const float* scale, float* const* phase, int* err, int sms, cudaStream_t s);

// Modal adjoint, one launch for all objects: part_k[z][u][m] = sum over
// pixel chunk z of object k of gphi_k[u][i] basis_k[m][i]. grad_layout picks
// the chunk length and the number of chunks of every object for U units on
// `sms` SMs (the partial-sum buffers hold splits[k] x U x M floats).
struct GradJob {
    int K;
    const float* gphi[kMaxObjects];
    const float* basis[kMaxObjects];
    int npix[kMaxObjects];
    int chunk[kMaxObjects];
    int splits[kMaxObjects];
    float* part[kMaxObjects];
    int split0[kMaxObjects + 1];  // filled by launch_grad_gemm
    int vec[kMaxObjects];         // filled by launch_grad_gemm
};
void grad_layout(int K, const int* npix, int U, int sms, int* chunk, int* splits);
cudaError_t launch_grad_gemm(GradJob job, int U, int M, cudaStream_t s);

// The modal adjoint on the tensor cores (tc_grad.cu): dL/dphi read in FP32
// through a TMA tensor map per object (encode_grad_map: rows P*J of npix
// pixels; npix a multiple of 4 and the base 16-byte aligned), split into
// three BF16 planes on the fly; the basis comes from the plan as BF16 planes
// per 32-pixel stage (grad_mma_basis, grad_mma_basis_elems elements). chunk
// (pixels, a multiple of 32) and splits come from grad_mma_layout; the
// partial sums have the layout of the SIMT kernel's. grad_mma_ring: the
// pipeline depth for M modes, 0 when the kernel does not fit.
struct GradMmaJob {
    int K, U, M;
    int row0;                          // the call's first unit among the tensor maps' rows
    const CUtensorMap* gmap[kMaxObjects];
    const uint16_t* bpl[kMaxObjects];
    float* part[kMaxObjects];
    int npix[kMaxObjects];
    int chunk[kMaxObjects];
    int* err;                          // set to 1 when a wait gives up
};
int grad_mma_ring(int M);
size_t grad_mma_smem(int M, int ring);
size_t grad_mma_basis_elems(int npix, int M);
void grad_mma_basis(const float* basis, int npix, int M, uint16_t* out);
void grad_mma_layout(int K, const int* npix, int M, int U, int sms, int* chunk, int* splits);
bool encode_grad_map(CUtensorMap* map, const float* gphi, int npix, long long rows);
cudaError_t launch_grad_mma(const GradMmaJob& job, int sms, cudaStream_t s);

// grad[u][m] = sum_k scale_k sum_z part_k[z][u][m] (fixed summation order)
struct GradParts {
    int K;
    int splits[kMaxObjects];
    float scale[kMaxObjects];
    const float* part[kMaxObjects];
};
cudaError_t launch_grad_combine(const GradParts& gp, int U, int M, float* grad, cudaStream_t s);

int max_ctas_per_sm(const FusedGeometry& g);

// ------------------------------------------------- patch sizes 48, 96, 128
// (and 64 on request): CTA-per-unit kernels, generic_kernels.cu.
struct GenericObj {
    int W;                  // side of the pupil's bounding box
    long long phi_off;      // float offset of this object's [P*J][W*W] phase block
    float inv_z;            // 1 / (N^2 n_pup)
    const uint32_t* mask;   // [W][mw] box rows, bit c = pupil pixel at box column c
    int mw;                 // words per mask row
    const uint32_t* supp;   // [N][sw] OTF support rows over kx <= N/2
    const uint64_t* cmask;  // [W][2] box columns: bit y = pupil pixel
    const uint64_t* csupp;  // [N/2+1][2] half-spectrum columns: bit ky = OTF support
};

struct GenericParams {
    int P, K, J, N;
    int sw;                 // words per support row
    double gamma;
    const float* weights;   // [K][J]
    const float* phi;       // box phases, per object at phi_off
    float* gphi;            // dL/dphi, same layout
    float2* gscr;           // [P][K][J][N][N/2+1]: OTF, then dL/dconj(H)
    float2* pscr;           // [P][K][J][N x N] field p [x][y]; null: recomputed by the adjoint
    float2* uscr;           // [P][K][J][ustride] pupil phasors; null: recomputed
    int ustride;
    const float2* spectra;  // D
    int spec_ld;            // N/2 + 1 or N
    double* loss;           // [P]
    float2* object;         // [P][K][N][spec_ld] or null
    int es, es2;            // row strides (complex) of the exchange buffers
    float2* e2scr;          // recompute: per-CTA second buffers [ctas][N * es2] in global memory (L2)
    int e2_ctas;            // CTAs e2scr has room for
    int rsplit;             // warps per (patch, object) of the frame reduction (<= 1: one)
    double* lpart;          // rsplit > 1: per-split patch losses [P][rsplit]
    const float2* oin;      // object-inferring loss: the given objects [P][K][N][spec_ld], else null
    float2* gobj;           // with oin: dL/dconj(O) [P][K][N][spec_ld], or null
    GenericObj obj[kMaxObjects];
};

size_t generic_smem(int N, int es, int es2, bool recompute);
// CTAs of the recompute adjoint launch on `sms` SMs (the size of e2scr).
int generic_adjoint_ctas(int N, int es, int sms);
cudaError_t launch_generic_forward(const GenericParams& prm, int sms, cudaStream_t s);
cudaError_t launch_generic_reduction(const GenericParams& prm, int sms, cudaStream_t s);
cudaError_t launch_generic_adjoint(const GenericParams& prm, int sms, cudaStream_t s);
// The same per patch size, defined in generic_kernels.cuh and instantiated
// in generic_n<N>.cu (one translation unit per size).
template <int N> int generic_adjoint_ctas_n(int es, int sms);
template <int N> cudaError_t launch_generic_forward_n(const GenericParams& prm, int sms, cudaStream_t s);
template <int N> cudaError_t launch_generic_adjoint_n(const GenericParams& prm, int sms, cudaStream_t s);

// Warps per (patch, object) of a frame reduction over P patches of K objects
// at N px: one while the patches alone give every SM 8 warps, more (each lane
// keeping at least 4 frequencies) when they are few. A plan fixes it from its
// patch count, so chunked calls sum the loss in the same order.
int reduction_split(int P, int K, int N, int sms);
// loss[p] = sum over s < S of lpart[p][s], in order.
cudaError_t launch_loss_combine(const double* lpart, int S, double* loss, int P, cudaStream_t s);

// ----------------------------------------- data front and back end of a field
struct FrontParams {
    int N, P, K, J;
    int H, Wimg;            // frame / mosaic size
    int nx, stride;         // patches per row, patch stride (N - overlap)
    int border;             // window transition, px
    int es;                 // exchange-buffer row stride (complex), >= N/2 + 1
    const float* frames;    // [K][J][H][Wimg]
    float2* spectra;        // [P][K][J][N][N/2+1]
    const float2* object;   // [P][K][N][N/2+1]
    float* oimg;            // [P][K][N][N] patch objects in the image domain (scratch)
    float* image;           // [K][H][Wimg]
    int* err;               // set when a bounded wait of a kernel gives up (TMA form of the spectra)
};
struct FilterParams {
    int N, P, K, ld;        // ld: N / 2 + 1 (half spectra) or N
    float2* object;         // [P][K][N][ld]
    float inv_diam[kMaxObjects], f_lower[kMaxObjects], f_upper[kMaxObjects];
};
cudaError_t launch_filter_objects(const FilterParams& prm, int sms, cudaStream_t s);

// Lofdahl-Scharmer filter (Sec. 4.1.1, Eq. 25): one CTA per (patch, object).
struct LsFilterParams {
    int N, P, K, J;
    int spec_ld, obj_ld;    // row strides (complex) of D and of the object: N / 2 + 1 or N
    float noise_power;      // nu, the noise power of one frame's spectrum per frequency
    const float2* spectra;  // D [P][K][J][N][spec_ld]
    const float2* otf;      // S [P][K][J][N][N/2+1]
    const float* weights;   // [K][J]
    float2* object;         // [P][K][N][obj_ld], multiplied in place, or null
    float* filter;          // [P][K][N][N/2+1] receives H, or null
    float* raw;             // [P][K][N][N/2+1] thresholded H before the median (filter or plan scratch)
};
size_t ls_filter_smem(int N);
cudaError_t launch_ls_filter(const LsFilterParams& prm, int sms, cudaStream_t s);
size_t front_smem(int N, int es);
// Spectra from frames; 64 px patches on 16-byte column boundaries take the
// TMA-staged kernel (spectra_tma_eligible), the rest the plain one.
bool spectra_tma_eligible(const FrontParams& prm);
cudaError_t launch_spectra_from_frames(const FrontParams& prm, int sms, cudaStream_t s);
cudaError_t launch_merge_objects(const FrontParams& prm, int sms, cudaStream_t s);

// Record an error for mfbd_last_error() (fixed-size buffer, no allocation).
int set_error(int status, const char* why);
int set_cuda_error(cudaError_t e, const char* where);

}  // namespace mfbd_dev
