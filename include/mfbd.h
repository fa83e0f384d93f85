/*
 * mfbd.h -- C ABI of the GB300 (sm_103a) MOMFBD hot path.
 *
 * Method: Asensio Ramos et al., "torchmfbd: a flexible multi-object
 * multi-frame blind deconvolution code" (arXiv:2505.10639).
 *   Sec. 3.1, Eq. 22  wavefront  phi_kj = c_k sum_m a_jm B_km, c_k = lambda_0/lambda_k
 *   Sec. 3.1, Eq. 20  pupil      P_kj   = A_k exp(i phi_kj)
 *   Sec. 3.1, Eq. 21  PSF        s_kj   = |F P_kj|^2 / sum |F P_kj|^2   (forward FFT)
 *                     OTF        H_kj   = F s_kj
 *   Sec. 2.2.1, Eq. 11  Wiener object  O_k = sum_j w D conj(H) / (sum_j w |H|^2 + gamma)
 *   Sec. 2.2.1, Eq. 12  loss  L_p = sum_k sum_u [ sum_j w |D|^2
 *                                    - |sum_j w D conj(H)|^2 / (sum_j w |H|^2 + gamma) ]
 *   and dL/da by the adjoint of Eqs. 20-22 and 12.
 * Index names: p patch, k object, j frame (diversity channels folded in,
 * Sec. 2.1), m mode, u frequency.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named "dev" are device memory owned by the caller; they must stay
 *   valid until the stream reaches the call. Pointers named "host" are read
 *   during the call only.
 * - Every compute call is asynchronous on the given stream (a cudaStream_t
 *   passed as void*; NULL means the legacy default stream) and never
 *   synchronises, allocates or frees after mfbd_plan_create.
 * - Every function returns an mfbd_status. Errors are returned, never thrown.
 *   A failed launch or CUDA error returns MFBD_ERR_CUDA and marks the plan
 *   failed: later compute calls on it return MFBD_ERR_STATE.
 * - There is no CPU fallback: without a usable CUDA device the compute calls
 *   return MFBD_ERR_UNSUPPORTED (or MFBD_ERR_CUDA) and compute nothing.
 * - Grids: the patch size N (n_pix) is 48, 64, 96 or 128. Images are
 *   [row y][column x], row-major. Spectra are unnormalised forward DFTs
 *   X[ky][kx] = sum_{y,x} x[y][x] exp(-2 pi i (ky y + kx x) / N), stored as
 *   interleaved complex64 (float re, float im). A "half spectrum" is the
 *   columns kx = 0..N/2 of every row: [N][N/2+1] (the layout of a real-to-
 *   complex 2-D FFT); a "full spectrum" is [N][N].
 * - Pupil sampling: centre at ((N-1)/2, (N-1)/2); pixel (y, x) is inside iff
 *   (x-c)^2 + (y-c)^2 <= (D_p/2)^2 (minus a central obscuration), computed in
 *   double from the float diameter.
 */
#ifndef MFBD_H
#define MFBD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MFBD_ABI_VERSION 1

typedef enum {
    MFBD_OK = 0,
    MFBD_ERR_INVALID_ARG = 1, /* bad descriptor, NULL pointer, size mismatch */
    MFBD_ERR_UNSUPPORTED = 2, /* valid request the library cannot run (N, no GPU) */
    MFBD_ERR_OOM = 3,         /* device or host allocation failed in create */
    MFBD_ERR_CUDA = 4,        /* a CUDA call or kernel launch failed */
    MFBD_ERR_STATE = 5,       /* wrong call order or a failed plan */
    MFBD_ERR_TIMEOUT = 6      /* a bounded device-side wait gave up */
} mfbd_status;

typedef enum {
    MFBD_BASIS_ZERNIKE = 0, /* Noll modes 2..M+1 (Noll 1976 normalisation) */
    MFBD_BASIS_KL = 1,      /* Karhunen-Loeve modes of Kolmogorov turbulence */
    MFBD_BASIS_USER = 2     /* caller-supplied basis, see user_basis */
} mfbd_basis;

typedef enum {
    MFBD_PREC_FP32 = 0,      /* FFTs, adjoint in FP32; the phase projection on the
                              * tensor cores with every operand split into three
                              * BF16 planes (FP32-accurate), or on the SIMT kernel */
    MFBD_PREC_BF16_PHASE = 1 /* phase projection phi = B a on the tensor cores with
                              * BF16 operands and FP32 accumulation; the rest as
                              * MFBD_PREC_FP32 */
} mfbd_precision;

/* flags */
#define MFBD_FLAG_FULL_SPECTRUM 0x1u /* spectra/object are [N][N], else [N][N/2+1] */
#define MFBD_FLAG_SIMT_PROJECTION 0x2u /* FP32 phase projection and modal adjoint on the
                                        * SIMT kernels instead of the tensor cores
                                        * (comparison runs; not with MFBD_PREC_BF16_PHASE) */
#define MFBD_FLAG_RECOMPUTE_BACKWARD 0x4u /* the adjoint recomputes the field F P and the
                                           * pupil phasors instead of keeping them from
                                           * the forward pass: 8 N^2 + 8 W^2 fewer bytes of
                                           * device memory per (patch, object, frame), about
                                           * 40 % more adjoint work */
#define MFBD_FLAG_GENERIC_KERNELS 0x8u /* run N = 64 on the kernels of the other patch
                                        * sizes (one CTA per unit) instead of the 64-pixel
                                        * pass machine (comparison runs) */
#define MFBD_FLAG_SPLIT_PASSES 0x10u /* N = 64: run mfbd_loss_grad (and the explicit and
                                      * host-buffer calls) as three kernels that exchange
                                      * the OTFs, seeds, fields and phasors through the
                                      * plan's workspaces, instead of the fused kernel
                                      * that keeps them on chip (comparison runs) */

typedef struct {
    int n_pix;      /* N, patch size in pixels: 48, 64, 96 or 128 */
    int n_patches;  /* P >= 0 (0: every compute call is a no-op) */
    int n_objects;  /* K, 1..8 */
    int n_frames;   /* J, 1..1024 (frames x diversity channels) */
    int n_modes;    /* M, 1..256 */
    const float* pupil_diam_px; /* host [K], D_p in pixels, 0 < D_p <= N */
    const double* wavelength;   /* host [K], any unit; c_k = wavelength[0]/wavelength[k] */
    float central_obscuration;  /* fraction of the diameter, 0 <= e < 1 */
    int basis;                  /* mfbd_basis */
    const float* user_basis;    /* host [K][M][N][N] when basis == MFBD_BASIS_USER, else NULL */
    double gamma;               /* Wiener constant S_n/S_0 (Eq. 11), > 0 */
    const float* frame_weight;  /* host [K][J] weights w_kj >= 0 (Eq. 2), or NULL for 1 */
    int precision;              /* mfbd_precision */
    unsigned flags;             /* MFBD_FLAG_* */
} mfbd_plan_desc;

typedef struct mfbd_plan* mfbd_plan_t;

typedef struct {
    int n_pix, n_patches, n_objects, n_frames, n_modes;
    int pupil_pixels[8];   /* n_pup,k: pixels inside pupil k */
    int pupil_box[8];      /* W_k: side of the pupil's bounding box */
    size_t workspace_bytes; /* device memory owned by the plan */
    int slots_per_cta;      /* frames a CTA of the fused kernel works on at once */
    int ctas;               /* CTAs of the fused kernel */
    int reduction_split;    /* warps per (patch, object) of the frame reduction; > 1 adds a
                               second launch that sums the per-split losses in order */
    int fused_ctas;         /* CTAs of the fused per-(patch, object) kernel that
                               mfbd_loss_grad runs (one per SM), or 0 when it runs the
                               three-kernel path (N != 64, J > 12, a pupil box wider
                               than 37 px, or MFBD_FLAG_SPLIT_PASSES) */
    int tc_projection;      /* 1: the phase projection phi = c B a runs on the tensor cores */
    int tc_adjoint;         /* 1: the modal adjoint dL/da = c B^T dL/dphi runs on the tensor
                               cores (dL/dphi and the basis split into three BF16 planes,
                               FP32 accumulation); 0: on the SIMT kernel
                               (MFBD_FLAG_SIMT_PROJECTION, an odd pupil box side, or more
                               than 256 modes) */
} mfbd_plan_info;

/* Create a plan: validates the descriptor, samples pupils, builds the modal
 * bases (double precision, on the host) and the exact OTF supports, uploads
 * them and allocates every workspace. Runs the uploads on `stream` and
 * synchronises it once. *out receives the plan (NULL on failure). */
int mfbd_plan_create(mfbd_plan_t* out, const mfbd_plan_desc* desc, void* stream);

/* Release a plan and its device memory (synchronises the device). NULL is OK. */
int mfbd_plan_destroy(mfbd_plan_t plan);

int mfbd_plan_get_info(mfbd_plan_t plan, mfbd_plan_info* info);

/* Synchronise `stream`, then MFBD_ERR_TIMEOUT if a bounded device-side wait
 * of an earlier call on this plan gave up (the tensor-core phase
 * projection's MMA completion, the TMA loads of mfbd_spectra_from_frames):
 * the outputs of the calls since the last check are then invalid. The flag
 * is cleared. MFBD_OK otherwise. The paper has no counterpart (device-side
 * failure detection of this library). */
int mfbd_plan_check(mfbd_plan_t plan, void* stream);

/* Forward pass (Eqs. 20-22, 11, 12).
 *   coeffs  dev [P][J][M] float: a_pjm, radians at wavelength[0].
 *   spectra dev [P][K][J][N][N/2+1] complex64 (or [N][N] with
 *           MFBD_FLAG_FULL_SPECTRUM): D_pkj, the FFTs of the observed frames.
 *   loss    dev [P] double: L_p = sum over objects and all N^2 frequencies.
 *   object  dev [P][K][N][N/2+1] (or [N][N]) complex64: O_pk (Eq. 11), or NULL.
 * Also keeps what mfbd_backward needs (the adjoint seeds dL/dconj(H) and the
 * wavefronts) in the plan. */
int mfbd_forward(mfbd_plan_t plan, const float* coeffs, const void* spectra,
                 double* loss, void* object, void* stream);

/* Backward pass: grad dev [P][J][M] float = dL_p/da_pjm for the coefficients
 * and spectra of the last mfbd_forward on this plan (MFBD_ERR_STATE if there
 * was none, or if an mfbd_loss_grad, mfbd_loss_grad_explicit or
 * mfbd_loss_grad_host came after it). */
int mfbd_backward(mfbd_plan_t plan, float* grad, void* stream);

/* Forward and backward in one call: loss, object (or NULL) and grad as
 * above. For N = 64 with J <= 12 and pupil boxes up to 37 px the pass work is
 * one fused launch (the fused per-(patch, object) kernel: forward passes,
 * frame reduction and adjoint passes of a pair in one CTA, the OTFs and seeds
 * in shared memory, the fields in a per-CTA buffer that stays in L2) plus a
 * small loss-combine kernel, between the modal phase projection and the
 * modal adjoint; otherwise the three-kernel path. Keeps nothing for
 * mfbd_backward on the fused path. */
int mfbd_loss_grad(mfbd_plan_t plan, const float* coeffs, const void* spectra,
                   double* loss, void* object, float* grad, void* stream);

/* mfbd_loss_grad (loss of Sec. 2.2.1, Eq. 12, object of Eq. 11 and dL/da)
 * from HOST buffers, with the copies overlapped with the
 * kernels: the patches go through in n_chunks chunks (n_chunks <= 0: about
 * 120 patches per chunk, 1 to 16 chunks); the
 * spectra of chunk c + 1 are copied to the device while chunk c is computed
 * (a chunk's phases and forward passes run while its own spectra are still
 * in flight: only the frame reduction reads them), and the loss, grad (and
 * object) of each chunk are copied back while later chunks are computed.
 * Same layouts as mfbd_loss_grad, all four (five)
 * pointers host memory; page-locked (cudaHostAlloc / pinned) buffers are
 * needed for the copies to overlap, pageable ones work but serialise. The
 * results are the same bits as mfbd_loss_grad's on the same inputs (every
 * kernel works per patch or per unit).
 * Asynchronous like the other calls: the host buffers may be read or
 * written until `stream` has completed the work queued by this call, which
 * covers the last copy back. The plan keeps device staging (coefficients,
 * loss and gradient of all patches, two chunks of spectra, the object when
 * asked for, two copy streams) from the first call on; a later call needing
 * larger staging synchronises the device and rebuilds it. Calls on one plan
 * from different streams must be ordered by the caller. After this call
 * mfbd_backward reports MFBD_ERR_STATE (the plan's per-unit buffers hold only
 * the last chunk). Errors: MFBD_ERR_INVALID_ARG for a NULL plan, coeffs,
 * spectra, loss or grad; a failed CUDA call returns its error and marks the
 * plan failed. */
int mfbd_loss_grad_host(mfbd_plan_t plan, const float* coeffs, const void* spectra,
                        double* loss, void* object, float* grad, int n_chunks, void* stream);

/* Forward model only: otf dev [P][K][J][N][N/2+1] complex64 = H_pkj
 * (Sec. 3.1, Eqs. 20-22, then H = F s), e.g. to synthesise data. */
int mfbd_otf(mfbd_plan_t plan, const float* coeffs, void* otf, void* stream);

/* Phase diversity (Sec. 2.1): a known phase theta_kj added to the wavefront
 * of object k in frame (diversity channel) j of every patch,
 * phi_kj = c_k B_k a_j + theta_kj, e.g. a defocus in the diversity channels.
 *   diversity host [K][J][N][N] float, radians, on the same grid as the pupil
 *             (read on pupil pixels only); NULL removes it.
 * Applies to every later evaluation and mfbd_otf on this plan (the forward
 * model, the loss, the object and dL/da; theta does not depend on a). The
 * first call allocates K x J x W_k^2 floats of device memory. Synchronises
 * `stream` (before and after the upload). */
int mfbd_plan_set_diversity(mfbd_plan_t plan, const float* diversity, void* stream);

/* Data front end of a field (Sec. 5.2): the plan's spectra from frames.
 *   frames  dev [K][J][height][width] float, the observed frames of every
 *           object and frame.
 * The field is cut into patches of n_pix px at stride n_pix - overlap, as
 * many as fit from the first row and column (their number must be the
 * plan's n_patches; patch p at row p / nx, column p % nx of the grid). In
 * every patch and frame the patch mean is subtracted, the modified Hanning
 * window applied (1 inside, a raised-cosine transition of `border` px at
 * each edge evaluated at pixel centres: w[x] = (1 - cos(pi (x + 1/2) /
 * border)) / 2 within `border` of an edge) and the mean added back;
 *   spectra dev [P][K][J][N][N/2+1] complex64 receives the unnormalised DFT
 *           of the result, in the layout mfbd_loss_grad reads.
 * Half-spectrum plans only (MFBD_ERR_UNSUPPORTED otherwise);
 * MFBD_ERR_INVALID_ARG for overlap outside [0, n_pix), border outside
 * [0, n_pix / 2], a field smaller than a patch or a patch count that is not
 * the plan's. Asynchronous; allocates nothing. */
int mfbd_spectra_from_frames(mfbd_plan_t plan, const float* frames, int height, int width, int overlap,
                             int border, void* spectra, void* stream);

/* Back end (Sec. 5.2): the mosaic of the patch objects.
 *   object dev [P][K][N][N/2+1] complex64, e.g. the Wiener objects of
 *          mfbd_forward / mfbd_loss_grad;
 *   image  dev [K][height][width] float receives, per pixel, the average of
 *          the patches covering it (patch grid as mfbd_spectra_from_frames),
 *          each patch object taken to the image domain by the inverse DFT
 *          normalised by 1 / N^2 and weighted by the window of `border` px;
 *          0 where no patch covers the pixel.
 * Same argument checks as mfbd_spectra_from_frames. The first call
 * allocates P x K x N^2 floats of plan scratch; later calls allocate
 * nothing. Asynchronous. */
int mfbd_merge_objects(mfbd_plan_t plan, const void* object, int height, int width, int overlap, int border,
                       float* image, void* stream);

/* Fourier filter of the objects (Sec. 4.1.1, the top-hat filter with a
 * cosine transition): O_k(u) *= H_k(u) in place, H = 1 for f <= f_lower[k],
 * 0 for f >= f_upper[k], (1 + cos(pi (f - f_lower) / (f_upper - f_lower))) / 2
 * between, f = |u| / D_p,k the frequency in units of object k's diffraction
 * limit (|u| in frequency bins of the N x N grid, D_p,k its pupil diameter
 * in px).
 *   object           dev [P][K][N][N/2+1] (or [N][N]) complex64, as
 *                    mfbd_forward returns it;
 *   f_lower, f_upper host [K], 0 <= f_lower < f_upper.
 * Asynchronous; allocates nothing. */
int mfbd_filter_objects(mfbd_plan_t plan, void* object, const float* f_lower, const float* f_upper, void* stream);

/* The object-inferring loss (Sec. 2.2.1, Eq. 8 with the regulariser
 * R = sum_k sum_u |O_k|^2 and beta = gamma, under which the Wiener object of
 * Eq. 11 is the exact minimiser) for given objects, and its gradients:
 *   L_p = sum_k sum_u [ sum_j w_kj |D_kj - O_k H_kj|^2 + gamma |O_k|^2 ]
 * (sum over the full frequency plane, from the half spectrum: columns 0 and
 * N/2 once, the others twice).
 *   coeffs, spectra, loss, grad  as mfbd_loss_grad (grad = dL/da with the
 *                                objects held fixed);
 *   object       dev [P][K][N][N/2+1] (or [N][N]) complex64, the given
 *                objects (Hermitian spectra of real images: the columns
 *                kx <= N/2 are read);
 *   grad_object  dev, the layout of object, receives dL/dconj(O(u)) per
 *                frequency: gamma O - sum_j w conj(H_j) (D_j - O H_j); NULL
 *                to skip.
 * FP32 with a frequency redone in FP64 where its residual energy falls
 * below 1e-3 of the data's. A following mfbd_backward returns
 * MFBD_ERR_STATE. Asynchronous; allocates nothing. */
int mfbd_loss_grad_explicit(mfbd_plan_t plan, const float* coeffs, const void* spectra, const void* object,
                            double* loss, float* grad, void* grad_object, void* stream);

/* The Lofdahl-Scharmer filter of the objects (Sec. 4.1.1, Eq. 25), per patch
 * and object k:
 *   H_k(u) = 1 - nu sum_j w_kj |S_kj(u)|^2 / |sum_j w_kj D_kj(u) conj(S_kj(u))|^2,
 * values below 0.2 set to 0 and above 1 to 1, a 3 x 3 median over the
 * periodic frequency plane, and every nonzero value not 4-connected to the
 * zero frequency (periodically) set to 0; then O_k *= H_k.
 *   spectra      dev D [P][K][J][N][N/2+1] (or [N][N]) complex64, the plan's
 *                layout, as passed to mfbd_forward;
 *   otf          dev S [P][K][J][N][N/2+1] complex64, as mfbd_otf writes it;
 *   noise_power  nu, the noise power of one frame's spectrum per frequency in
 *                the units of |D|^2 (N^2 sigma^2 for white noise of variance
 *                sigma^2 per pixel); 1 gives the printed form; finite;
 *   object       dev [P][K][N][N/2+1] (or [N][N]) complex64, multiplied in
 *                place, or NULL;
 *   filter       dev [P][K][N][N/2+1] float receives H, or NULL (not both
 *                NULL).
 * The frame weights are the plan's w_kj. FP32 with each product and sum
 * rounded on its own in a fixed order (no fused multiply-add). One CTA per
 * (patch, object) with the N x N plane in shared memory (4 N^2 + 80 N bytes),
 * after a streaming pass that writes the thresholded H to `filter` (or, when
 * `filter` is NULL, to P x K x N x (N/2+1) floats of plan scratch allocated
 * by the first such call). Asynchronous. */
int mfbd_ls_filter_objects(mfbd_plan_t plan, const void* spectra, const void* otf, float noise_power, void* object,
                           float* filter, void* stream);

/* Host-only plan-time data (no GPU needed), for inspection and tests:
 *   mask     host [N][N] uint8, pupil k (1 inside), or NULL
 *   basis    host [M][N][N] float, modes of object k (0 outside pupil), or NULL
 *   variance host [M] double, Kolmogorov variance of each mode in units of
 *            (D/r0)^(5/3) rad^2 (Zernike: Noll covariance diagonal; KL:
 *            eigenvalues; USER: zeros), or NULL
 *   support  host [N][N/2+1] uint8, exact OTF support of pupil k, or NULL */
int mfbd_describe_object(const mfbd_plan_desc* desc, int object, unsigned char* mask,
                         float* basis, double* variance, unsigned char* support);

/* Kernel timing. When enabled, every compute call records a CUDA event pair
 * on its stream around each stage it launches (per object for the phase
 * projection), from a pool of max_launches pairs created here (enable = 0
 * destroys the pool). Calls made while the pool is full are not timed. */
int mfbd_plan_set_profiling(mfbd_plan_t plan, int enable, int max_launches);

/* Waits for the recorded events, then returns the summed device time in ms
 * and the number of kernels launched inside the timed pairs, per kind,
 * arrays of 6: [0] modal phase
 * projection, [1] forward passes (pupil -> OTF), [2] frame reduction (loss,
 * object, adjoint seeds), [3] adjoint passes (-> dL/dphi), [4] modal adjoint
 * projection, [5] the fused per-(patch, object) kernel (forward passes,
 * reduction and adjoint passes in one launch, with its loss combine). With
 * reset != 0 the pool is emptied for reuse. Arrays may be NULL. */
int mfbd_plan_read_profile(mfbd_plan_t plan, double* ms, long long* launches, int reset);

/* Allocation-free variant of the fused kernel, for callers that cannot
 * allocate device memory (a plugin whose host framework owns all device
 * memory, code where the CUDA allocator is off limits, a fixed memory
 * budget): such callers cannot create a plan, because mfbd_plan_create
 * allocates workspaces. The paper has no counterpart; this is library
 * plumbing. No plan is needed and nothing is allocated: the caller passes
 * the inputs and outputs, and the kernel's working memory is one 16 MiB
 * array compiled into the library, held by every GPU that loads it until
 * the process exits.
 *   desc        host: n_pix (64 only), n_patches, n_objects, n_frames, pupil
 *               diameters, obscuration, gamma, frame weights and flags are
 *               used; n_modes, basis, user_basis, wavelength and precision
 *               are ignored (the wavefront is given as a phase).
 *   phase       dev [K][P][J][N][N] float: phi_kpj on the full grid, radians
 *               (read on pupil pixels only)
 *   spectra     dev as in mfbd_forward
 *   loss        dev [P] double, as in mfbd_forward
 *   object      dev as in mfbd_forward, or NULL
 *   grad_phase  dev [K][P][J][N][N] float: dL/dphi (0 outside the pupil)
 * Limits: n_objects x n_frames <= 336 per call (MFBD_ERR_INVALID_ARG beyond
 * that: the scratch of one patch, K x J x (N x (N/2+1) + N x N) complex64,
 * must fit); the patches are processed in batches that fit the array (14
 * patches per batch at 2 objects x 12 frames), so this path is slower than
 * the plan path for large fields.
 * The first call on each device looks up the array's device address (with
 * that device current) and caches it; make that first call before any
 * stream capture. The cached address belongs to the device's context of
 * that moment: after cudaDeviceReset on a device, do not call this entry
 * point on that device again in the same process. Each call uploads its small constants with one
 * cudaMemcpyAsync from pageable host memory (which may wait for the
 * stream's earlier work) and clears grad_phase with cudaMemsetAsync.
 * Calls are serialised on the host, but every call shares the one array
 * and it keeps the last call's contents: calls whose work overlaps on the
 * GPU (other streams, other host threads) race and give wrong results.
 * Nothing in the array needs to start at zero: each element a call reads
 * is written earlier in the same call. */
int mfbd_phase_loss_grad_noalloc(const mfbd_plan_desc* desc, const float* phase, const void* spectra,
                                 double* loss, void* object, float* grad_phase, void* stream);

/* ------------------------------------------------------------------------
 * Uneven batches: many problems of different sizes in one persistent launch
 * ------------------------------------------------------------------------
 * A batch holds n problems, each described by an mfbd_plan_desc of its own
 * (patch size 48, 64, 96 or 128, patches, objects, frames, modes, pupils,
 * wavelengths, basis, gamma, weights; FP32 precision, half spectra and no
 * flags). Its loss, Wiener object and dL/da are those of Sec. 2.2.1
 * (Eqs. 11, 12) with the forward model of Sec. 3.1 (Eqs. 20-22), computed per
 * problem as mfbd_loss_grad computes them for a plan.
 *
 * Caller buffers are the problems' buffers of mfbd_loss_grad packed one after
 * the other in problem order (mfbd_batch_get_offsets gives each problem's
 * start, in elements):
 *   coeffs  dev float      [sum_i P_i J_i M_i]
 *   spectra dev complex64  [sum_i P_i K_i J_i N_i (N_i/2+1)]
 *   loss    dev double     [sum_i P_i]
 *   object  dev complex64  [sum_i P_i K_i N_i (N_i/2+1)] or NULL
 *   grad    dev float      like coeffs
 *
 * One evaluation is one launch of a persistent kernel over a list of work
 * items (per patch: phases, forward passes per frame, frame reduction,
 * adjoint passes per frame, modal adjoint), in which an item waits (bounded)
 * for the items of its patch that it depends on; or, in the staged schedule,
 * five launches (one per kind of item) that never wait. The schedule (mode,
 * window of units over which the kinds of item are interleaved, CTAs per SM)
 * is set by mfbd_batch_set_schedule or chosen by timing in
 * mfbd_batch_autotune. mfbd_batch_loss_grad does no host synchronisation and
 * no allocation, so it can be captured in a CUDA graph (a memset node and the
 * kernel node(s)). Evaluations of one batch must not overlap on the GPU (they
 * share the batch's scratch and counters). */
#define MFBD_BATCH_ONE_LAUNCH 0 /* one launch; items wait for their dependencies */
#define MFBD_BATCH_STAGED 1     /* one launch per kind of item; no waits */

typedef struct mfbd_batch* mfbd_batch_t;

typedef struct {
    int n_problems;
    long long n_patches, n_units, n_items;
    long long coeff_floats, spectra_complex, loss_doubles, object_complex;  /* packed sizes */
    size_t workspace_bytes;  /* device memory owned by the batch */
    int mode;                /* MFBD_BATCH_ONE_LAUNCH or MFBD_BATCH_STAGED */
    int window_units;        /* one-launch interleaving window, 64 px units (0: kind-major) */
    int ctas_per_sm, max_ctas_per_sm, ctas;
    int smem_bytes;          /* dynamic shared memory per CTA */
    int variant;             /* kernel variant (register budget), see mfbd_batch_set_schedule */
} mfbd_batch_info;

/* Create a batch from n_problems host descriptors: validates each (as
 * mfbd_plan_create), builds the pupils, bases (shared between problems with
 * the same sampling; Zernike sets are shared across mode counts) and OTF
 * supports on the host, uploads them, allocates the scratch (per unit: OTF
 * and seed N (N/2+1), field N^2 complex64; phases and dL/dphi on the pupil
 * box) and the work list, and synchronises `stream` once. The default
 * schedule is one launch with windows of 8192 units and the most CTAs per
 * SM that fit. Errors: MFBD_ERR_INVALID_ARG / MFBD_ERR_UNSUPPORTED for a bad
 * or unsupported descriptor (mfbd_last_error names it), MFBD_ERR_OOM,
 * MFBD_ERR_CUDA without a usable device. */
int mfbd_batch_create(mfbd_batch_t* out, const mfbd_plan_desc* problems, int n_problems, void* stream);

/* Release a batch (synchronises the device). NULL is OK. */
int mfbd_batch_destroy(mfbd_batch_t batch);

int mfbd_batch_get_info(mfbd_batch_t batch, mfbd_batch_info* info);

/* Start of each problem in the packed buffers, host arrays [n_problems] of
 * element offsets (any may be NULL). */
int mfbd_batch_get_offsets(mfbd_batch_t batch, long long* coeffs, long long* spectra, long long* loss,
                           long long* object);

/* Set the schedule: mode MFBD_BATCH_ONE_LAUNCH or MFBD_BATCH_STAGED,
 * window_units (one launch: the kinds of item of about this many 64 px units
 * are interleaved with the next window's; <= 0: all items of a kind before
 * the next kind), ctas_per_sm (1..max_ctas_per_sm of the variant, 0: the
 * maximum), variant (0: the kernel compiled with up to 255 registers a
 * thread, 2 CTAs of 128 threads per SM; 1: up to 170 registers, 3 CTAs per
 * SM, the 96 and 128 px passes spilling). Synchronises the device (the work
 * list is rewritten). */
int mfbd_batch_set_schedule(mfbd_batch_t batch, int mode, int window_units, int ctas_per_sm, int variant);

/* Loss, object (or NULL) and dL/da of every problem (layouts above),
 * asynchronous on `stream`. A dependency wait that gives up (it cannot in a
 * correct launch; the bound guards against a fault elsewhere) sets the
 * batch's error flag, reported by mfbd_batch_check. */
int mfbd_batch_loss_grad(mfbd_batch_t batch, const float* coeffs, const void* spectra, double* loss,
                         void* object, float* grad, void* stream);

/* Forward model only (Sec. 3.1, Eqs. 20-22, then H = F s) of every problem:
 * otf dev complex64, packed like spectra (the same offsets), = H_pkj, e.g. to
 * synthesise data. Runs the phase and forward-pass items of the schedule. */
int mfbd_batch_otf(mfbd_batch_t batch, const float* coeffs, void* otf, void* stream);

/* Synchronise `stream`, then MFBD_ERR_TIMEOUT if a wait of an earlier
 * evaluation gave up (the flag is cleared), else MFBD_OK. */
int mfbd_batch_check(mfbd_batch_t batch, void* stream);

/* Autotuner: times each candidate schedule (one launch with windows of 0,
 * 2048, 8192 and 32768 units, and staged; each kernel variant at its most
 * CTAs per SM) on these inputs, `reps` evaluations each after one warm-up, keeps
 * the fastest and returns. Synchronises; outputs hold the last evaluation. */
int mfbd_batch_autotune(mfbd_batch_t batch, const float* coeffs, const void* spectra, double* loss,
                        void* object, float* grad, int reps, void* stream);

/* ---- Spatially variant PSF on a dictionary (Sec. 2.2.2, "Spatially variant
 * convolution"; the PSF expansion, the image as a sum of convolutions and the
 * Fourier-domain log-posterior). Plan-free: the PSF at object point r' is
 * sum_i a_i(r') phi_i(r), and per patch the data term is
 *   L_p = sum_k sum_j gamma_kj sum_u |I_kj(u) - sum_i F(o_k a_ikj)(u) Phi_i(u)|^2
 * over the full N x N frequency plane (from the half spectrum: columns 0 and
 * N/2 once, the others twice), F unnormalised, Phi_i = F(phi_i). The
 * regulariser of the paper's log-posterior is left to the caller. ---- */
typedef struct {
    int n;          /* patch size N; 64 */
    int n_patches;  /* P >= 0 */
    int n_objects;  /* K >= 1 */
    int n_frames;   /* J >= 1 */
    int n_atoms;    /* M >= 1, dictionary functions */
} mfbd_dict_desc;

/* Bytes of device workspace mfbd_dict_loss_grad needs for `desc`
 * (P K J doubles and P K J N^2 floats, with alignment padding); 0 for an
 * invalid descriptor. */
size_t mfbd_dict_workspace_bytes(const mfbd_dict_desc* desc);

/* L_p and its gradients for given objects and coefficient maps:
 *   dL/da_ikj = o_k g_ikj,  dL/do_k = sum_j sum_i a_ikj g_ikj,
 *   g_ikj = Re F^H[conj(Phi_i) (-2 gamma_kj R_kj)],
 *   R_kj = I_kj - sum_i F(o_k a_ikj) Phi_i.
 *   atom_otf     dev [M][N][N/2+1] complex64, Phi_i (half spectra of the real
 *                dictionary functions phi_i), 8-byte aligned;
 *   gamma        dev [K][J] float, the frame weights gamma_kj;
 *   object       dev [P][K][N][N] float, o_k (image domain), 16-byte aligned;
 *   coeff        dev [P][K][J][M][N][N] float, a_ikj(r'), 16-byte aligned;
 *   spectra      dev [P][K][J][N][N/2+1] complex64, I_kj, half spectra of
 *                real images (the plan's spectra layout), 8-byte aligned;
 *   workspace    dev, mfbd_dict_workspace_bytes(desc) bytes, 16-byte aligned,
 *                owned by the caller, contents undefined on return;
 *   loss         dev [P] double, L_p;
 *   grad_object  dev [P][K][N][N] float, dL/do, or NULL to skip;
 *   grad_coeff   dev [P][K][J][M][N][N] float, dL/da, 16-byte aligned, or
 *                NULL to skip.
 * FP32 transforms and products; the loss sums each frame's terms in FP64,
 * and both sums over frames and objects run in a fixed order. Errors:
 * MFBD_ERR_INVALID_ARG (descriptor, NULL or misaligned pointer),
 * MFBD_ERR_UNSUPPORTED (n other than 64), MFBD_ERR_CUDA. Asynchronous on
 * `stream`; allocates nothing. */
int mfbd_dict_loss_grad(const mfbd_dict_desc* desc, const void* atom_otf, const float* gamma, const float* object,
                        const float* coeff, const void* spectra, void* workspace, double* loss, float* grad_object,
                        float* grad_coeff, void* stream);

/* Static description of a status code (never NULL). */
const char* mfbd_status_string(int status);

/* Detail of the last error raised on the calling host thread (never NULL). */
const char* mfbd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MFBD_H */
