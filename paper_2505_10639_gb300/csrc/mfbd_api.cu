// C ABI of the MOMFBD hot path: plans, validation, workspaces, launches.
// The arithmetic lives in mfbd_kernels.cu (device) and optics_host.cpp
// (plan-time host math); this file only validates, allocates and schedules.
#include "../../include/mfbd.h"
#include "mfbd_internal.h"
#include "optics_host.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <string>
#include <vector>

using namespace mfbd_dev;

namespace {

constexpr int kProfileKinds = 6;  // see mfbd_plan_read_profile

thread_local char g_last_error[512] = "no error";

int fail(int status, const char* why) {
    std::snprintf(g_last_error, sizeof g_last_error, "%s", why);
    return status;
}

int fail(int status, const std::string& why) { return fail(status, why.c_str()); }

int cuda_fail(cudaError_t e, const char* where) {
    std::snprintf(g_last_error, sizeof g_last_error, "%s: %s", where, cudaGetErrorString(e));
    return MFBD_ERR_CUDA;
}

struct ObjectData {
    int W = 0, x0 = 0, npup = 0;
    float diam = 0.f;            // pupil diameter in px (the diffraction limit in frequency bins)
    float scale = 1.f, inv_z = 0.f;
    long long phi_off = 0;
    long long part_off = 0;     // offset of this object's modal-adjoint partial sums
    int g_chunk = 0, g_splits = 0;  // modal-adjoint pixel chunks for all P*J units (sizes part buffer)
    float* d_basis = nullptr;   // [M][W*W]
    uint64_t* d_mask = nullptr; // [W] box rows, then [N] box columns
    uint32_t* d_gmask = nullptr;  // general sizes: [W][mw] box mask rows
    uint32_t* d_gsupp = nullptr;  // general sizes: [N][sw] OTF-support rows
    uint64_t* d_gcol = nullptr;   // general sizes: [W][2] box-column mask words, then [N/2+1][2] support columns
    int mw = 0;
    uint64_t* d_supp = nullptr; // [N] rows, then [N] columns of the OTF support
    // tensor-core phase projection: the box basis as BF16 planes in the MMA
    // tile layout, [n_tiles][planes][Nt * Mp]; planes == 0: SIMT kernel
    uint16_t* d_basis_tc = nullptr;
    int tc_planes = 0;
    // tensor-core modal adjoint: the box basis as BF16 planes per 32-pixel
    // stage, and the TMA map of this object's dL/dphi (all P*J units)
    uint16_t* d_gbasis_tc = nullptr;
    CUtensorMap gmap{};
    float* d_div = nullptr;       // known diversity phases [J][W*W] (phase diversity), or null
    float* d_div_buf = nullptr;   // their buffer, allocated by the first mfbd_plan_set_diversity
};

}  // namespace

struct mfbd_plan {
    int N = 0, P = 0, K = 0, J = 0, M = 0;
    unsigned flags = 0;
    int precision = MFBD_PREC_FP32;
    bool generic = false;       // CTA-per-unit kernels (N != 64, recompute, or on request)
    bool fused = false;         // mfbd_loss_grad runs the fused per-(patch, object) kernel
    int fused_ctas = 0;         // its CTAs (one per SM)
    float2* d_fscr = nullptr;   // its field slots [fused_ctas][kFusedFrames][N*N/2] (rows N/2..N-1)
    double* d_lpair = nullptr;  // its per-(patch, object) losses [P][K]
    int* d_lcnt = nullptr;      // its per-patch counts of finished objects [P], 0 between calls
    int* d_fticket = nullptr;   // its pair ticket and count of finished CTAs, 0 between calls
    int es = 0, es2 = 0, sw = 0;  // their exchange-buffer strides and support-row words
    double gamma = 0;
    int* d_err = nullptr;       // set by a tensor-core kernel whose MMA wait gave up
    uint16_t* d_acoef = nullptr;  // coefficients as BF16 planes in the MMA tile layout
    bool tc_grad = false;         // the modal adjoint runs on the tensor cores
    int device = 0;
    ObjectData obj[kMaxObjects];
    float* d_weights = nullptr;
    float* d_phi = nullptr;
    float* d_gphi = nullptr;
    float* d_gpart = nullptr;   // modal-adjoint partial sums [K][splits][P*J][M]
    float2* d_gscr = nullptr;   // per unit [P][K][J][N][N/2+1]: OTF, then adjoint seed
    float2* d_pscr = nullptr;   // per unit [P][K][J][N*N]: field
    float2* d_uscr = nullptr;   // per unit [P][K][J][ustride]: pupil phasors on the box
    float* d_oimg = nullptr;    // mfbd_merge_objects: patch objects in the image domain [P][K][N][N]
    float* d_lsraw = nullptr;   // mfbd_ls_filter_objects without a filter output: [P][K][N][N/2+1]
    float2* d_e2scr = nullptr;  // recompute, CTA-per-unit kernels: per-CTA second buffers [e2_ctas][N * es2]
    int e2_ctas = 0;
    const void* x_oin = nullptr;  // mfbd_loss_grad_explicit: the given objects, during that call only
    void* x_gobj = nullptr;       // and dL/dconj(O)
    int rsplit = 1;             // warps per (patch, object) of the frame reduction
    double* d_lpart = nullptr;  // rsplit > 1: per-split patch losses [P][rsplit]
    int ustride = 0;
    long long phi_floats = 0;
    size_t workspace = 0;
    FusedGeometry geo{};
    int ctas = 0;   // CTAs of a pass kernel
    int sms = 0;
    bool failed = false;
    bool have_forward = false;
    std::vector<void*> allocations;
    // host-buffer pipeline (mfbd_loss_grad_host), created on first use
    struct HostPipe {
        bool ready = false;
        int chunk_patches = 0;            // patches per staging buffer
        bool with_object = false;
        float* d_coeffs = nullptr;        // [P][J][M]
        void* d_spec[2] = {nullptr, nullptr};
        double* d_loss = nullptr;         // [P]
        float* d_grad = nullptr;          // [P][J][M]
        void* d_object = nullptr;         // [P][K][N][ld] or null
        cudaStream_t h2d = nullptr, d2h = nullptr;
        cudaEvent_t ev_start = nullptr, ev_coeffs = nullptr, ev_end = nullptr, ev_done = nullptr;
        cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_consumed[2] = {nullptr, nullptr};
        std::vector<void*> allocations;
    } host;
    // kernel timing (mfbd_plan_set_profiling)
    std::vector<cudaEvent_t> ev;    // 2 per pair
    std::vector<int> ev_kind;       // kind of each used pair
    std::vector<int> ev_nk;         // kernels launched inside each used pair
    int ev_used = 0;
};

namespace {

int validate(const mfbd_plan_desc* d) {
    if (!d) return fail(MFBD_ERR_INVALID_ARG, "descriptor is NULL");
    if (d->n_pix <= 0) return fail(MFBD_ERR_INVALID_ARG, "n_pix must be positive");
    if (d->n_patches < 0) return fail(MFBD_ERR_INVALID_ARG, "n_patches must be >= 0");
    if (d->n_objects < 1 || d->n_objects > kMaxObjects)
        return fail(MFBD_ERR_INVALID_ARG, "n_objects must be in 1..8");
    if (d->n_frames < 1 || d->n_frames > 1024) return fail(MFBD_ERR_INVALID_ARG, "n_frames must be in 1..1024");
    if (d->n_modes < 1 || d->n_modes > 256) return fail(MFBD_ERR_INVALID_ARG, "n_modes must be in 1..256");
    if (!d->pupil_diam_px) return fail(MFBD_ERR_INVALID_ARG, "pupil_diam_px is NULL");
    if (!d->wavelength) return fail(MFBD_ERR_INVALID_ARG, "wavelength is NULL");
    for (int k = 0; k < d->n_objects; ++k) {
        float dp = d->pupil_diam_px[k];
        if (!(dp > 0.f) || !(dp <= (float)d->n_pix))
            return fail(MFBD_ERR_INVALID_ARG, "pupil diameter must be in (0, n_pix]");
        if (!(d->wavelength[k] > 0.0) || !std::isfinite(d->wavelength[k]))
            return fail(MFBD_ERR_INVALID_ARG, "wavelength must be positive and finite");
    }
    if (!(d->central_obscuration >= 0.f) || !(d->central_obscuration < 1.f))
        return fail(MFBD_ERR_INVALID_ARG, "central_obscuration must be in [0, 1)");
    if (d->basis != MFBD_BASIS_ZERNIKE && d->basis != MFBD_BASIS_KL && d->basis != MFBD_BASIS_USER)
        return fail(MFBD_ERR_INVALID_ARG, "unknown basis");
    if (d->basis == MFBD_BASIS_USER && !d->user_basis)
        return fail(MFBD_ERR_INVALID_ARG, "user_basis is NULL for MFBD_BASIS_USER");
    if (!(d->gamma > 0.0) || !std::isfinite(d->gamma)) return fail(MFBD_ERR_INVALID_ARG, "gamma must be > 0");
    if (d->frame_weight)
        for (int i = 0; i < d->n_objects * d->n_frames; ++i)
            if (!(d->frame_weight[i] >= 0.f) || !std::isfinite(d->frame_weight[i]))
                return fail(MFBD_ERR_INVALID_ARG, "frame weights must be finite and >= 0");
    if (d->precision != MFBD_PREC_FP32 && d->precision != MFBD_PREC_BF16_PHASE)
        return fail(MFBD_ERR_INVALID_ARG, "unknown precision");
    if (d->flags & ~(MFBD_FLAG_FULL_SPECTRUM | MFBD_FLAG_SIMT_PROJECTION | MFBD_FLAG_RECOMPUTE_BACKWARD |
                     MFBD_FLAG_GENERIC_KERNELS | MFBD_FLAG_SPLIT_PASSES))
        return fail(MFBD_ERR_INVALID_ARG, "unknown flags");
    if (d->n_pix != 48 && d->n_pix != 64 && d->n_pix != 96 && d->n_pix != 128)
        return fail(MFBD_ERR_UNSUPPORTED, "n_pix must be 48, 64, 96 or 128");
    if (d->precision == MFBD_PREC_BF16_PHASE && (d->flags & MFBD_FLAG_SIMT_PROJECTION))
        return fail(MFBD_ERR_INVALID_ARG, "the BF16 phase projection runs on the tensor cores only");
    return MFBD_OK;
}

// BF16 bits of x, rounded to nearest even (finite x).
uint16_t bf16_round(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

float bf16_float(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float x;
    std::memcpy(&x, &u, 4);
    return x;
}

// Tensor-core layout of object o's box basis `hb` ([M][W^2] float): for each
// tile of 128 pixels and each BF16 plane (x = x0 + x1 + x2, each plane
// the rounding of what the previous ones leave; one plane for the BF16 phase
// path), the 128 x Mp operand in the no-swizzle K-major core-matrix order
// (8 pixels x 8 modes per 128-byte core matrix, core matrices along the modes
// 128 bytes apart, 8-pixel groups Mp * 16 bytes apart). Returns false (SIMT
// kernel) when the projection is forced onto the SIMT kernel or its tiles do
// not fit in shared memory.
bool tc_projection_layout(const mfbd_plan* p, ObjectData& o, const std::vector<float>& hb,
                          std::vector<uint16_t>* out) {
    if (p->flags & MFBD_FLAG_SIMT_PROJECTION) return false;
    const int planes = p->precision == MFBD_PREC_BF16_PHASE ? 1 : 3;
    const int Mp = (p->M + 15) / 16 * 16, npix = o.W * o.W;
    if (phase_mma_smem(p->M, planes) > (size_t)200 * 1024) return false;
    const int nt = 128;  // pixels per tile (the MMA's M)
    const int tiles = (npix + nt - 1) / nt;
    out->assign((size_t)tiles * planes * nt * Mp, 0);
    for (int t = 0; t < tiles; ++t)
        for (int r = 0; r < nt; ++r) {
            const int i = t * nt + r;
            if (i >= npix) break;
            for (int m = 0; m < p->M; ++m) {
                const float x = hb[(size_t)m * npix + i];
                float left = x;
                for (int q = 0; q < planes; ++q) {
                    const uint16_t b = bf16_round(left);
                    left -= bf16_float(b);
                    const size_t off = (size_t)(r / 8) * Mp * 8 + (size_t)(m / 8) * 64 + (size_t)(r % 8) * 8 + (m % 8);
                    (*out)[((size_t)t * planes + q) * nt * Mp + off] = b;
                }
            }
        }
    o.tc_planes = planes;
    return true;
}

// full-grid double basis [M][N][N] of object k
std::vector<double> object_basis(const mfbd_plan_desc* d, int k, std::vector<double>* variance) {
    const int n = d->n_pix, m = d->n_modes;
    if (d->basis == MFBD_BASIS_USER) {
        std::vector<double> b((size_t)m * n * n);
        const float* src = d->user_basis + (size_t)k * m * n * n;
        for (size_t i = 0; i < b.size(); ++i) b[i] = src[i];
        if (variance) variance->assign(m, 0.0);
        return b;
    }
    mfbd_host::ModalBasis mb = d->basis == MFBD_BASIS_ZERNIKE
                                   ? mfbd_host::zernike_basis(n, d->pupil_diam_px[k], d->central_obscuration, m)
                                   : mfbd_host::kl_basis(n, d->pupil_diam_px[k], d->central_obscuration, m);
    if (variance) *variance = mb.variance;
    return mb.modes;
}

template <class T>
int dev_alloc(mfbd_plan* p, T** ptr, size_t count) {
    *ptr = nullptr;
    if (count == 0) return MFBD_OK;
    void* raw = nullptr;
    cudaError_t e = cudaMalloc(&raw, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(MFBD_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    p->allocations.push_back(raw);
    p->workspace += count * sizeof(T);
    *ptr = static_cast<T*>(raw);
    return MFBD_OK;
}

void release(mfbd_plan* p) {
    for (void* a : p->allocations) cudaFree(a);
    p->allocations.clear();
}

// Kernel parameters for patches [p0, p0 + np): spectra, loss and object
// point at patch p0; the per-unit scratch is reused from its start.
FusedParams fused_params(const mfbd_plan* p, int p0, int np, const void* spectra, double* loss, void* object,
                         float2* gscr, float2* pscr, float2* uscr) {
    FusedParams f{};
    f.P = np;
    f.K = p->K;
    f.J = p->J;
    f.M = p->M;
    f.gamma = p->gamma;
    f.weights = p->d_weights;
    f.phi = p->d_phi;
    f.gphi = p->d_gphi;
    f.gscr = gscr;
    f.pscr = pscr;
    f.uscr = uscr;
    f.ustride = uscr ? p->ustride : 0;
    f.spectra = static_cast<const float2*>(spectra);
    f.spec_ld = (p->flags & MFBD_FLAG_FULL_SPECTRUM) ? p->N : p->N / 2 + 1;
    f.loss = loss;
    f.object = static_cast<float2*>(object);
    f.rsplit = p->rsplit;
    f.lpart = p->d_lpart;
    f.oin = static_cast<const float2*>(p->x_oin);
    f.gobj = static_cast<float2*>(p->x_gobj);
    for (int k = 0; k < p->K; ++k) {
        f.obj[k].W = p->obj[k].W;
        f.obj[k].x0 = p->obj[k].x0;
        f.obj[k].inv_z = p->obj[k].inv_z;
        f.obj[k].phi_off = p->obj[k].phi_off + (long long)p0 * p->J * p->obj[k].W * p->obj[k].W;
        f.obj[k].phi_unit = (long long)p->obj[k].W * p->obj[k].W;
        f.obj[k].phi_org = 0;
        f.obj[k].phi_ld = p->obj[k].W;
        f.obj[k].mask = p->obj[k].d_mask;
        f.obj[k].supp = p->obj[k].d_supp;
        f.obj[k].cmask = p->obj[k].d_mask + p->obj[k].W;
        f.obj[k].csupp = p->obj[k].d_supp + p->N;
    }
    return f;
}

int check_plan(mfbd_plan_t p) {
    if (!p) return fail(MFBD_ERR_INVALID_ARG, "plan is NULL");
    if (p->failed) return fail(MFBD_ERR_STATE, "plan failed earlier");
    return MFBD_OK;
}

int set_device(mfbd_plan_t p) {
    cudaError_t e = cudaSetDevice(p->device);
    if (e != cudaSuccess) {
        p->failed = true;
        return cuda_fail(e, "cudaSetDevice");
    }
    return MFBD_OK;
}

// event pair around one launch when profiling: returns the pair index or -1
int prof_begin(mfbd_plan_t p, int kind, cudaStream_t s) {
    if (p->ev.empty() || p->ev_used * 2 >= (int)p->ev.size()) return -1;
    const int i = p->ev_used++;
    p->ev_kind[i] = kind;
    cudaEventRecord(p->ev[2 * i], s);
    return i;
}

void prof_end(mfbd_plan_t p, int i, cudaStream_t s, int kernels) {
    if (i < 0) return;
    p->ev_nk[i] = kernels;
    cudaEventRecord(p->ev[2 * i + 1], s);
}

// Phases of patches [p0, p0 + np); coeffs points at patch p0.
int run_phase(mfbd_plan_t p, const float* coeffs, cudaStream_t s, int p0, int np) {
    const int U = np * p->J;
    if (p->obj[0].tc_planes > 0) {  // tensor cores: one split, one launch for all objects
        const uint16_t* bt[kMaxObjects];
        int npix[kMaxObjects];
        float scale[kMaxObjects];
        float* out[kMaxObjects];
        int ndiv = 0;
        for (int k = 0; k < p->K; ++k) {
            const ObjectData& o = p->obj[k];
            bt[k] = o.d_basis_tc;
            npix[k] = o.W * o.W;
            scale[k] = o.scale;
            out[k] = p->d_phi + o.phi_off + (size_t)p0 * p->J * o.W * o.W;
            ndiv += o.d_div ? 1 : 0;
        }
        const int pi = prof_begin(p, 0, s);
        cudaError_t e = launch_split_coeffs(coeffs, U, p->M, p->obj[0].tc_planes, p->d_acoef, s);
        if (e == cudaSuccess)
            e = launch_phase_mma(p->d_acoef, U, p->M, p->K, bt, npix, p->obj[0].tc_planes, scale, out, p->d_err,
                                 p->sms, s);
        for (int k = 0; k < p->K && e == cudaSuccess; ++k)  // phi_kj = c_k B_k a_j + theta_kj
            if (p->obj[k].d_div) e = launch_add_diversity(out[k], p->obj[k].d_div, U, p->J, npix[k], p->sms, s);
        prof_end(p, pi, s, 2 + ndiv);
        if (e != cudaSuccess) {
            p->failed = true;
            return cuda_fail(e, "phase projection");
        }
        return MFBD_OK;
    }
    for (int k = 0; k < p->K; ++k) {
        const ObjectData& o = p->obj[k];
        const int pi = prof_begin(p, 0, s);
        float* out = p->d_phi + o.phi_off + (size_t)p0 * p->J * o.W * o.W;
        cudaError_t e = launch_phase_gemm(coeffs, U, p->M, o.d_basis, o.W * o.W, o.scale, out, s);
        if (e == cudaSuccess && o.d_div)  // phi_kj = c_k B_k a_j + theta_kj
            e = launch_add_diversity(out, o.d_div, U, p->J, o.W * o.W, p->sms, s);
        prof_end(p, pi, s, 1 + (o.d_div ? 1 : 0));
        if (e != cudaSuccess) {
            p->failed = true;
            return cuda_fail(e, "phase projection");
        }
    }
    return MFBD_OK;
}

// dL/da of patches [p0, p0 + np); grad points at patch p0.
int run_grad(mfbd_plan_t p, float* grad, cudaStream_t s, int p0, int np) {
    const int U = np * p->J;
    GradJob job{};
    job.K = p->K;
    // The plan's pixel chunks (laid out for all P*J units at create), for
    // every call: the summation order of dL/da then does not depend on how
    // many patches a call covers, so a chunked host-buffer call gives the
    // same bits as one device call.
    int npix[kMaxObjects], chunk[kMaxObjects], splits[kMaxObjects];
    for (int k = 0; k < p->K; ++k) {
        npix[k] = p->obj[k].W * p->obj[k].W;
        chunk[k] = p->obj[k].g_chunk;
        splits[k] = p->obj[k].g_splits;
    }
    GradParts gp{};
    gp.K = p->K;
    for (int k = 0; k < p->K; ++k) {
        const ObjectData& o = p->obj[k];
        job.gphi[k] = p->d_gphi + o.phi_off + (size_t)p0 * p->J * o.W * o.W;
        job.basis[k] = o.d_basis;
        job.npix[k] = npix[k];
        job.chunk[k] = chunk[k];
        job.splits[k] = splits[k];
        job.part[k] = p->d_gpart + o.part_off;
        gp.splits[k] = splits[k];
        gp.scale[k] = o.scale;
        gp.part[k] = job.part[k];
    }
    const int pi = prof_begin(p, 4, s);
    cudaError_t e;
    if (p->tc_grad) {
        GradMmaJob mj{};
        mj.K = p->K;
        mj.U = U;
        mj.M = p->M;
        mj.row0 = p0 * p->J;
        mj.err = p->d_err;
        for (int k = 0; k < p->K; ++k) {
            mj.gmap[k] = &p->obj[k].gmap;
            mj.bpl[k] = p->obj[k].d_gbasis_tc;
            mj.part[k] = job.part[k];
            mj.npix[k] = npix[k];
            mj.chunk[k] = chunk[k];
        }
        e = launch_grad_mma(mj, p->sms, s);
    } else {
        e = launch_grad_gemm(job, U, p->M, s);
    }
    if (e == cudaSuccess) e = launch_grad_combine(gp, U, p->M, grad, s);
    prof_end(p, pi, s, 2);
    if (e != cudaSuccess) {
        p->failed = true;
        return cuda_fail(e, "modal adjoint");
    }
    return MFBD_OK;
}

// Kernels of an evaluation, selected by bit: the forward passes, the frame
// reduction, the adjoint passes; OTF_ONLY writes the OTFs to `gscr` and keeps
// nothing for the adjoint.
enum Stage : int { ST_FWD = 1, ST_RED = 2, ST_ADJ = 4, ST_OTF_ONLY = 8 };

// General patch sizes: the same stages on the CTA-per-unit kernels.
int run_generic(mfbd_plan_t p, int stages, const void* spectra, double* loss, void* object, float2* gscr,
                cudaStream_t s, int p0, int np) {
    GenericParams g{};
    g.P = np;
    g.K = p->K;
    g.J = p->J;
    g.N = p->N;
    g.sw = p->sw;
    g.gamma = p->gamma;
    g.weights = p->d_weights;
    g.phi = p->d_phi;
    g.gphi = p->d_gphi;
    const bool otf_only = (stages & ST_OTF_ONLY) != 0;
    g.gscr = otf_only ? gscr : p->d_gscr;
    g.pscr = otf_only ? nullptr : p->d_pscr;
    g.uscr = otf_only ? nullptr : p->d_uscr;
    g.ustride = p->ustride;
    g.spectra = static_cast<const float2*>(spectra);
    g.spec_ld = (p->flags & MFBD_FLAG_FULL_SPECTRUM) ? p->N : p->N / 2 + 1;
    g.loss = loss;
    g.object = static_cast<float2*>(object);
    g.es = p->es;
    g.es2 = p->es2;
    g.e2scr = p->d_e2scr;
    g.e2_ctas = p->e2_ctas;
    g.rsplit = p->rsplit;
    g.lpart = p->d_lpart;
    g.oin = static_cast<const float2*>(p->x_oin);
    g.gobj = static_cast<float2*>(p->x_gobj);
    for (int k = 0; k < p->K; ++k) {
        const ObjectData& o = p->obj[k];
        g.obj[k].W = o.W;
        g.obj[k].phi_off = o.phi_off + (long long)p0 * p->J * o.W * o.W;
        g.obj[k].inv_z = o.inv_z;
        g.obj[k].mask = o.d_gmask;
        g.obj[k].mw = o.mw;
        g.obj[k].supp = o.d_gsupp;
        g.obj[k].cmask = o.d_gcol;
        g.obj[k].csupp = o.d_gcol ? o.d_gcol + 2 * o.W : nullptr;
    }
    cudaError_t e = cudaSuccess;
    if (stages & ST_FWD) {
        const int pi = prof_begin(p, 1, s);
        e = launch_generic_forward(g, p->sms, s);
        prof_end(p, pi, s, 1);
    }
    if (e == cudaSuccess && (stages & ST_RED)) {
        const int pr = prof_begin(p, 2, s);
        e = launch_generic_reduction(g, p->sms, s);
        prof_end(p, pr, s, p->rsplit > 1 && p->d_lpart ? 2 : 1);  // + the loss combine
    }
    if (e == cudaSuccess && (stages & ST_ADJ)) {
        const int pb = prof_begin(p, 3, s);
        e = launch_generic_adjoint(g, p->sms, s);
        prof_end(p, pb, s, 1);
    }
    if (e != cudaSuccess) {
        p->failed = true;
        return cuda_fail(e, "pass or reduction kernel");
    }
    return MFBD_OK;
}

// Pass and reduction kernels of `stages` for patches [p0, p0 + np).
int run_fused(mfbd_plan_t p, int stages, const void* spectra, double* loss, void* object, float2* gscr,
              cudaStream_t s, int p0, int np) {
    if (p->generic) return run_generic(p, stages, spectra, loss, object, gscr, s, p0, np);
    FusedParams f = (stages & ST_OTF_ONLY)
                        ? fused_params(p, p0, np, spectra, loss, object, gscr, nullptr, nullptr)
                        : fused_params(p, p0, np, spectra, loss, object, p->d_gscr, p->d_pscr, p->d_uscr);
    cudaError_t e = cudaSuccess;
    if (stages & ST_FWD) {
        const int pi = prof_begin(p, 1, s);
        e = launch_forward_passes(f, p->geo, p->sms, s);
        prof_end(p, pi, s, 1);
    }
    if (e == cudaSuccess && (stages & ST_RED)) {
        const int pr = prof_begin(p, 2, s);
        e = launch_reduction(f, p->sms, s);
        prof_end(p, pr, s, p->rsplit > 1 && p->d_lpart ? 2 : 1);  // + the loss combine
    }
    if (e == cudaSuccess && (stages & ST_ADJ)) {
        const int pb = prof_begin(p, 3, s);
        e = launch_adjoint_passes(f, p->geo, p->sms, s);
        prof_end(p, pb, s, 1);
    }
    if (e != cudaSuccess) {
        p->failed = true;
        return cuda_fail(e, "pass or reduction kernel");
    }
    return MFBD_OK;
}

// The fused per-(patch, object) kernel for patches [p0, p0 + np): loss,
// object and dL/dphi of the chunk in one launch (plus the loss combine).
int run_pairs(mfbd_plan_t p, const void* spectra, double* loss, void* object, cudaStream_t s, int p0, int np) {
    FusedParams f = fused_params(p, p0, np, spectra, loss, object, nullptr, nullptr, nullptr);
    f.fscr = p->d_fscr;
    f.lpair = p->d_lpair + (size_t)p0 * p->K;
    f.lcnt = p->d_lcnt + p0;
    f.fticket = p->d_fticket;
    // pairs of the widest pupil boxes (the costliest) are dealt first
    for (int k = 0; k < p->K; ++k) f.korder[k] = k;
    std::stable_sort(f.korder, f.korder + p->K, [&](int a, int b) { return p->obj[a].W > p->obj[b].W; });
    const int pi = prof_begin(p, 5, s);
    const cudaError_t e = launch_fused_pairs(f, p->geo.xs, p->fused_ctas, s);
    prof_end(p, pi, s, 1);
    if (e != cudaSuccess) {
        p->failed = true;
        return cuda_fail(e, "fused kernel");
    }
    return MFBD_OK;
}

// ------------------------------------------------------- host-buffer pipeline

void host_release(mfbd_plan* p) {
    auto& h = p->host;
    for (cudaStream_t st : {h.h2d, h.d2h})
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : {h.ev_start, h.ev_coeffs, h.ev_end, h.ev_done, h.ev_copied[0], h.ev_copied[1],
                          h.ev_consumed[0], h.ev_consumed[1]})
        if (e) cudaEventDestroy(e);
    for (void* a : h.allocations) cudaFree(a);
    h = mfbd_plan::HostPipe{};
}

size_t spectrum_patch_bytes(const mfbd_plan* p) {
    const int ld = (p->flags & MFBD_FLAG_FULL_SPECTRUM) ? p->N : p->N / 2 + 1;
    return (size_t)p->K * p->J * p->N * ld * sizeof(float2);
}

size_t object_patch_bytes(const mfbd_plan* p) {
    const int ld = (p->flags & MFBD_FLAG_FULL_SPECTRUM) ? p->N : p->N / 2 + 1;
    return (size_t)p->K * p->N * ld * sizeof(float2);
}

// Device staging of the host pipeline for `chunk` patches per buffer; kept
// across calls and rebuilt (after a device synchronisation) only when a call
// needs more.
int host_setup(mfbd_plan* p, int chunk, bool with_object) {
    auto& h = p->host;
    if (h.ready && h.chunk_patches >= chunk && (h.with_object || !with_object)) return MFBD_OK;
    cudaDeviceSynchronize();
    host_release(p);
    auto alloc = [&](void** ptr, size_t bytes) -> cudaError_t {
        cudaError_t e = cudaMalloc(ptr, bytes > 0 ? bytes : 16);
        if (e == cudaSuccess) h.allocations.push_back(*ptr);
        return e;
    };
    const size_t cm = (size_t)p->P * p->J * p->M;
    cudaError_t e = cudaSuccess;
    if ((e = alloc((void**)&h.d_coeffs, cm * sizeof(float))) || (e = alloc((void**)&h.d_grad, cm * sizeof(float))) ||
        (e = alloc((void**)&h.d_loss, (size_t)p->P * sizeof(double))) ||
        (e = alloc(&h.d_spec[0], (size_t)chunk * spectrum_patch_bytes(p))) ||
        (e = alloc(&h.d_spec[1], (size_t)chunk * spectrum_patch_bytes(p))) ||
        (with_object && (e = alloc(&h.d_object, (size_t)p->P * object_patch_bytes(p)))) ||
        (e = cudaStreamCreateWithFlags(&h.h2d, cudaStreamNonBlocking)) ||
        (e = cudaStreamCreateWithFlags(&h.d2h, cudaStreamNonBlocking))) {
        host_release(p);
        return cuda_fail(e, "host pipeline setup");
    }
    for (cudaEvent_t* ev : {&h.ev_start, &h.ev_coeffs, &h.ev_end, &h.ev_done, &h.ev_copied[0], &h.ev_copied[1],
                            &h.ev_consumed[0], &h.ev_consumed[1]})
        if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming))) {
            host_release(p);
            return cuda_fail(e, "host pipeline events");
        }
    h.ready = true;
    h.chunk_patches = chunk;
    h.with_object = with_object;
    return MFBD_OK;
}

}  // namespace

namespace mfbd_dev {
int validate_desc(const mfbd_plan_desc* d) { return validate(d); }
int set_error(int status, const char* why) { return fail(status, why); }
int set_cuda_error(cudaError_t e, const char* where) { return cuda_fail(e, where); }
}  // namespace mfbd_dev

extern "C" {

const char* mfbd_status_string(int status) {
    switch (status) {
        case MFBD_OK: return "MFBD_OK";
        case MFBD_ERR_INVALID_ARG: return "MFBD_ERR_INVALID_ARG: invalid argument";
        case MFBD_ERR_UNSUPPORTED: return "MFBD_ERR_UNSUPPORTED: not supported by the library or the device";
        case MFBD_ERR_OOM: return "MFBD_ERR_OOM: allocation failed";
        case MFBD_ERR_CUDA: return "MFBD_ERR_CUDA: CUDA error";
        case MFBD_ERR_STATE: return "MFBD_ERR_STATE: wrong call order or failed plan";
        case MFBD_ERR_TIMEOUT: return "MFBD_ERR_TIMEOUT: device wait gave up";
        default: return "unknown mfbd status";
    }
}

const char* mfbd_last_error(void) { return g_last_error; }

int mfbd_describe_object(const mfbd_plan_desc* desc, int object, unsigned char* mask, float* basis,
                         double* variance, unsigned char* support) {
    int st = validate(desc);
    if (st == MFBD_ERR_UNSUPPORTED && desc && desc->n_pix > 0 && desc->n_pix <= 256 && desc->n_pix % 2 == 0)
        st = MFBD_OK;  // host data is defined for any even N
    if (st != MFBD_OK) return st;
    if (object < 0 || object >= desc->n_objects) return fail(MFBD_ERR_INVALID_ARG, "object index out of range");
    try {
        const int n = desc->n_pix;
        std::vector<uint8_t> m = mfbd_host::pupil_mask(n, desc->pupil_diam_px[object], desc->central_obscuration);
        if (mask) std::memcpy(mask, m.data(), m.size());
        if (basis || variance) {
            std::vector<double> var;
            std::vector<double> b = object_basis(desc, object, &var);
            if (basis)
                for (size_t i = 0; i < b.size(); ++i) basis[i] = (float)b[i];
            if (variance)
                for (int i = 0; i < desc->n_modes; ++i) variance[i] = var[i];
        }
        if (support) {
            std::vector<uint8_t> s = mfbd_host::otf_support_half(m, n);
            std::memcpy(support, s.data(), s.size());
        }
    } catch (const std::exception& e) {
        return fail(MFBD_ERR_INVALID_ARG, e.what());
    }
    return MFBD_OK;
}

int mfbd_plan_create(mfbd_plan_t* out, const mfbd_plan_desc* d, void* stream) {
    if (!out) return fail(MFBD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int st = validate(d);
    if (st != MFBD_OK) return st;

    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(MFBD_ERR_UNSUPPORTED, "no CUDA device (there is no CPU fallback)");
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
    if (prop.major * 10 + prop.minor != 103)
        return fail(MFBD_ERR_UNSUPPORTED, "the library targets sm_103a (GB300)");

    mfbd_plan* p = new (std::nothrow) mfbd_plan();
    if (!p) return fail(MFBD_ERR_OOM, "host allocation failed");
    p->N = d->n_pix;
    p->P = d->n_patches;
    p->K = d->n_objects;
    p->J = d->n_frames;
    p->M = d->n_modes;
    p->flags = d->flags;
    p->precision = d->precision;
    p->generic = d->n_pix != kN || (d->flags & (MFBD_FLAG_RECOMPUTE_BACKWARD | MFBD_FLAG_GENERIC_KERNELS));
    p->gamma = d->gamma;
    p->device = dev;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n = p->N;

    try {
        std::vector<float> w((size_t)p->K * p->J, 1.0f);
        if (d->frame_weight) std::memcpy(w.data(), d->frame_weight, w.size() * sizeof(float));
        if ((st = dev_alloc(p, &p->d_weights, w.size()))) throw st;
        if ((e = cudaMemcpyAsync(p->d_weights, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice, s)))
            throw cuda_fail(e, "upload weights");

        std::vector<std::vector<float>> hb(p->K);
        std::vector<std::vector<uint16_t>> htc(p->K);
        if ((st = dev_alloc(p, &p->d_err, 1))) throw st;
        if ((e = cudaMemsetAsync(p->d_err, 0, sizeof(int), s))) throw cuda_fail(e, "clear error flag");
        std::vector<std::vector<uint64_t>> hm(p->K), hs(p->K);
        std::vector<std::vector<uint32_t>> gm(p->K), gs(p->K);
        std::vector<std::vector<uint64_t>> gc(p->K);
        long long phi_floats = 0;
        int max_box = 1;
        for (int k = 0; k < p->K; ++k) {
            ObjectData& o = p->obj[k];
            std::vector<uint8_t> mask = mfbd_host::pupil_mask(n, d->pupil_diam_px[k], d->central_obscuration);
            int lo = n, hi = -1, npup = 0;
            for (int y = 0; y < n; ++y)
                for (int x = 0; x < n; ++x)
                    if (mask[(size_t)y * n + x]) {
                        ++npup;
                        lo = std::min(lo, std::min(x, y));
                        hi = std::max(hi, std::max(x, y));
                    }
            if (npup == 0) throw fail(MFBD_ERR_INVALID_ARG, "pupil has no pixel");
            o.npup = npup;
            o.diam = d->pupil_diam_px[k];
            o.x0 = lo;
            o.W = hi - lo + 1;
            max_box = std::max(max_box, o.W);
            o.scale = (float)(d->wavelength[0] / d->wavelength[k]);
            o.inv_z = (float)(1.0 / ((double)n * n * npup));
            o.phi_off = phi_floats;
            phi_floats += (long long)p->P * p->J * o.W * o.W;
            std::vector<double> full = object_basis(d, k, nullptr);
            hb[k].assign((size_t)p->M * o.W * o.W, 0.f);
            for (int m = 0; m < p->M; ++m)
                for (int yy = 0; yy < o.W; ++yy)
                    for (int xx = 0; xx < o.W; ++xx) {
                        size_t src = (size_t)m * n * n + (size_t)(o.x0 + yy) * n + (o.x0 + xx);
                        if (mask[(size_t)(o.x0 + yy) * n + (o.x0 + xx)])
                            hb[k][(size_t)m * o.W * o.W + (size_t)yy * o.W + xx] = (float)full[src];
                    }
            std::vector<uint8_t> sup = mfbd_host::otf_support_half(mask, n);
            if (!p->generic) {
                // bit rows, then the same bits by column (a lane's column in one word)
                hm[k].assign(o.W + n, 0);
                for (int yy = 0; yy < o.W; ++yy)
                    for (int xx = 0; xx < o.W; ++xx)
                        if (mask[(size_t)(o.x0 + yy) * n + (o.x0 + xx)]) {
                            hm[k][yy] |= 1ull << xx;
                            hm[k][o.W + xx] |= 1ull << yy;
                        }
                hs[k].assign(2 * n, 0);
                for (int ky = 0; ky < n; ++ky)
                    for (int kx = 0; kx <= n / 2; ++kx)
                        if (sup[(size_t)ky * (n / 2 + 1) + kx]) {
                            hs[k][ky] |= 1ull << kx;
                            hs[k][n + kx] |= 1ull << ky;
                        }
            } else {
                // 32-bit words: box rows [W][mw], support rows [N][sw]
                o.mw = (o.W + 31) / 32;
                p->sw = (n / 2 + 1 + 31) / 32;
                gm[k].assign((size_t)o.W * o.mw, 0u);
                for (int yy = 0; yy < o.W; ++yy)
                    for (int xx = 0; xx < o.W; ++xx)
                        if (mask[(size_t)(o.x0 + yy) * n + (o.x0 + xx)]) gm[k][yy * o.mw + xx / 32] |= 1u << (xx % 32);
                gs[k].assign((size_t)n * p->sw, 0u);
                for (int ky = 0; ky < n; ++ky)
                    for (int kx = 0; kx <= n / 2; ++kx)
                        if (sup[(size_t)ky * (n / 2 + 1) + kx]) gs[k][ky * p->sw + kx / 32] |= 1u << (kx % 32);
                gc[k].assign((size_t)2 * o.W + 2 * (n / 2 + 1), 0ull);
                for (int yy = 0; yy < o.W; ++yy)
                    for (int xx = 0; xx < o.W; ++xx)
                        if (mask[(size_t)(o.x0 + yy) * n + (o.x0 + xx)]) gc[k][2 * xx + yy / 64] |= 1ull << (yy % 64);
                for (int ky = 0; ky < n; ++ky)
                    for (int kx = 0; kx <= n / 2; ++kx)
                        if (sup[(size_t)ky * (n / 2 + 1) + kx]) gc[k][2 * o.W + 2 * kx + ky / 64] |= 1ull << (ky % 64);
                if ((st = dev_alloc(p, &o.d_gcol, gc[k].size()))) throw st;
                if ((e = cudaMemcpyAsync(o.d_gcol, gc[k].data(), gc[k].size() * 8, cudaMemcpyHostToDevice, s)))
                    throw cuda_fail(e, "upload column masks");
                if ((st = dev_alloc(p, &o.d_gmask, gm[k].size()))) throw st;
                if ((st = dev_alloc(p, &o.d_gsupp, gs[k].size()))) throw st;
                if ((e = cudaMemcpyAsync(o.d_gmask, gm[k].data(), gm[k].size() * 4, cudaMemcpyHostToDevice, s)) ||
                    (e = cudaMemcpyAsync(o.d_gsupp, gs[k].data(), gs[k].size() * 4, cudaMemcpyHostToDevice, s)))
                    throw cuda_fail(e, "upload masks");
            }
            if ((st = dev_alloc(p, &o.d_basis, hb[k].size()))) throw st;
            if (tc_projection_layout(p, o, hb[k], &htc[k])) {
                if ((st = dev_alloc(p, &o.d_basis_tc, htc[k].size()))) throw st;
                if ((e = cudaMemcpyAsync(o.d_basis_tc, htc[k].data(), htc[k].size() * 2, cudaMemcpyHostToDevice, s)))
                    throw cuda_fail(e, "upload tensor-core basis");
            }
            if ((e = cudaMemcpyAsync(o.d_basis, hb[k].data(), hb[k].size() * sizeof(float), cudaMemcpyHostToDevice,
                                     s)))
                throw cuda_fail(e, "upload plan data");
            if (!p->generic) {
                if ((st = dev_alloc(p, &o.d_mask, hm[k].size()))) throw st;
                if ((st = dev_alloc(p, &o.d_supp, hs[k].size()))) throw st;
                if ((e = cudaMemcpyAsync(o.d_mask, hm[k].data(), hm[k].size() * 8, cudaMemcpyHostToDevice, s)) ||
                    (e = cudaMemcpyAsync(o.d_supp, hs[k].data(), hs[k].size() * 8, cudaMemcpyHostToDevice, s)))
                    throw cuda_fail(e, "upload plan data");
            }
        }
        p->phi_floats = phi_floats;
        if (p->obj[0].tc_planes > 0 &&
            (st = dev_alloc(p, &p->d_acoef, split_coeffs_elems(p->P * p->J, p->M, p->obj[0].tc_planes))))
            throw st;
        // the modal adjoint on the tensor cores: every pupil box of an even
        // side (rows of whole 16-byte groups for the TMA maps), M <= 256
        p->tc_grad = !(p->flags & MFBD_FLAG_SIMT_PROJECTION) && grad_mma_ring(p->M) >= 2;
        for (int k = 0; k < p->K; ++k)
            if ((p->obj[k].W * p->obj[k].W) % 4 != 0) p->tc_grad = false;
        if (p->tc_grad)
            for (int k = 0; k < p->K; ++k) {
                ObjectData& o = p->obj[k];
                std::vector<uint16_t> hg(grad_mma_basis_elems(o.W * o.W, p->M));
                grad_mma_basis(hb[k].data(), o.W * o.W, p->M, hg.data());
                if ((st = dev_alloc(p, &o.d_gbasis_tc, hg.size()))) throw st;
                if ((e = cudaMemcpyAsync(o.d_gbasis_tc, hg.data(), hg.size() * 2, cudaMemcpyHostToDevice, s)))
                    throw cuda_fail(e, "upload tensor-core adjoint basis");
            }
        long long part_floats = 0;
        {
            int npix[kMaxObjects], chunk[kMaxObjects], splits[kMaxObjects];
            for (int k = 0; k < p->K; ++k) npix[k] = p->obj[k].W * p->obj[k].W;
            if (p->tc_grad)  // chunks of whole 32-pixel stages, which the SIMT kernel also takes
                grad_mma_layout(p->K, npix, p->M, p->P * p->J, prop.multiProcessorCount, chunk, splits);
            else
                grad_layout(p->K, npix, p->P * p->J, prop.multiProcessorCount, chunk, splits);
            for (int k = 0; k < p->K; ++k) {
                p->obj[k].g_chunk = chunk[k];
                p->obj[k].g_splits = splits[k];
                p->obj[k].part_off = part_floats;
                part_floats += (long long)splits[k] * p->P * p->J * p->M;
            }
        }
        if ((st = dev_alloc(p, &p->d_gpart, (size_t)part_floats))) throw st;
        if ((st = dev_alloc(p, &p->d_phi, (size_t)phi_floats))) throw st;
        if ((st = dev_alloc(p, &p->d_gphi, (size_t)phi_floats))) throw st;
        for (int k = 0; k < p->K && p->tc_grad; ++k) {
            ObjectData& o = p->obj[k];
            if (!encode_grad_map(&o.gmap, p->d_gphi + o.phi_off, o.W * o.W, (long long)p->P * p->J))
                p->tc_grad = false;  // the SIMT kernel takes the same chunks
        }
        const bool keep = !(p->flags & MFBD_FLAG_RECOMPUTE_BACKWARD);
        if ((st = dev_alloc(p, &p->d_gscr, (size_t)p->P * p->K * p->J * n * (n / 2 + 1)))) throw st;
        if (keep && (st = dev_alloc(p, &p->d_pscr, (size_t)p->P * p->K * p->J * n * n))) throw st;
        p->ustride = (max_box * max_box + 31) & ~31;  // 256-byte aligned units
        if (keep && (st = dev_alloc(p, &p->d_uscr, (size_t)p->P * p->K * p->J * p->ustride))) throw st;

        p->sms = prop.multiProcessorCount;
        p->rsplit = reduction_split(p->P, p->K, n, p->sms);
        if (p->rsplit > 1 && (st = dev_alloc(p, &p->d_lpart, (size_t)p->P * p->rsplit))) throw st;
        if (!p->generic) {
            p->geo = fused_geometry(max_box);
            int per_sm = max_ctas_per_sm(p->geo);
            if (per_sm < 1) throw fail(MFBD_ERR_UNSUPPORTED, "fused kernel does not fit on this device");
            p->ctas = prop.multiProcessorCount * per_sm;
            // the fused per-(patch, object) kernel for mfbd_loss_grad when the
            // frames and the pupil boxes fit its shared memory
            if (!(p->flags & MFBD_FLAG_SPLIT_PASSES) && fused_pair_supported(p->J, p->geo.xs)) {
                const int fper = fused_pair_ctas_per_sm(p->geo.xs);
                if (fper >= 1) {
                    p->fused = true;
                    p->fused_ctas = prop.multiProcessorCount * fper;
                    if ((st = dev_alloc(p, &p->d_fscr, (size_t)p->fused_ctas * kFusedFrames * n * n / 2))) throw st;
                    if ((st = dev_alloc(p, &p->d_lpair, (size_t)std::max(1, p->P * p->K)))) throw st;
                    if ((st = dev_alloc(p, &p->d_lcnt, (size_t)std::max(1, p->P)))) throw st;
                    if ((st = dev_alloc(p, &p->d_fticket, 2))) throw st;
                    if ((e = cudaMemsetAsync(p->d_lcnt, 0, (size_t)std::max(1, p->P) * sizeof(int), s)) ||
                        (e = cudaMemsetAsync(p->d_fticket, 0, 2 * sizeof(int), s)))
                        throw cuda_fail(e, "clear fused-kernel counters");
                }
            }
        } else {
            // odd row strides: column accesses do not conflict in shared memory
            p->es = std::max(n / 2 + 1, max_box) | 1;
            p->es2 = max_box | 1;
            if (generic_smem(n, p->es, p->es2, !keep) > (size_t)227 * 1024)
                throw fail(MFBD_ERR_UNSUPPORTED, "the pupil box is too large for the shared-memory buffers");
            if (!keep) {
                p->e2_ctas = generic_adjoint_ctas(n, p->es, prop.multiProcessorCount);
                if (p->e2_ctas < 1) throw fail(MFBD_ERR_UNSUPPORTED, "the adjoint kernel does not fit on this device");
                if ((st = dev_alloc(p, &p->d_e2scr, (size_t)p->e2_ctas * n * p->es2))) throw st;
            }
            p->geo = FusedGeometry{};
            p->ctas = prop.multiProcessorCount;
        }
        if ((e = cudaStreamSynchronize(s))) throw cuda_fail(e, "plan upload");
    } catch (int status) {
        release(p);
        delete p;
        return status;
    } catch (const std::exception& ex) {
        release(p);
        delete p;
        return fail(MFBD_ERR_INVALID_ARG, ex.what());
    }
    *out = p;
    return MFBD_OK;
}

int mfbd_plan_set_profiling(mfbd_plan_t p, int enable, int max_launches) {
    if (!p) return fail(MFBD_ERR_INVALID_ARG, "plan is NULL");
    cudaSetDevice(p->device);
    for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
    p->ev.clear();
    p->ev_kind.clear();
    p->ev_nk.clear();
    p->ev_used = 0;
    if (!enable) return MFBD_OK;
    if (max_launches < 1 || max_launches > 1 << 16) return fail(MFBD_ERR_INVALID_ARG, "max_launches out of range");
    p->ev.resize((size_t)2 * max_launches);
    p->ev_kind.assign(max_launches, 0);
    p->ev_nk.assign(max_launches, 0);
    for (size_t i = 0; i < p->ev.size(); ++i) {
        cudaError_t e = cudaEventCreate(&p->ev[i]);
        if (e != cudaSuccess) {
            for (size_t j = 0; j < i; ++j) cudaEventDestroy(p->ev[j]);
            p->ev.clear();
            p->ev_kind.clear();
            p->ev_nk.clear();
            return cuda_fail(e, "cudaEventCreate");
        }
    }
    return MFBD_OK;
}

int mfbd_plan_read_profile(mfbd_plan_t p, double* ms, long long* launches, int reset) {
    if (!p) return fail(MFBD_ERR_INVALID_ARG, "plan is NULL");
    double acc[kProfileKinds] = {};
    long long cnt[kProfileKinds] = {};
    for (int i = 0; i < p->ev_used; ++i) {
        cudaError_t e = cudaEventSynchronize(p->ev[2 * i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
        float t = 0.f;
        if ((e = cudaEventElapsedTime(&t, p->ev[2 * i], p->ev[2 * i + 1])) != cudaSuccess)
            return cuda_fail(e, "cudaEventElapsedTime");
        acc[p->ev_kind[i]] += t;
        cnt[p->ev_kind[i]] += p->ev_nk[i];
    }
    for (int k = 0; k < kProfileKinds; ++k) {
        if (ms) ms[k] = acc[k];
        if (launches) launches[k] = cnt[k];
    }
    if (reset) p->ev_used = 0;
    return MFBD_OK;
}

int mfbd_plan_destroy(mfbd_plan_t p) {
    if (!p) return MFBD_OK;
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
    host_release(p);
    release(p);
    delete p;
    return MFBD_OK;
}

int mfbd_plan_set_diversity(mfbd_plan_t p, const float* diversity, void* stream) {
    int st = check_plan(p);
    if (st) return st;
    if ((st = set_device(p))) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(s);  // no queued evaluation may be reading the old phases
    if (e != cudaSuccess) return cuda_fail(e, "synchronise before setting the diversity");
    for (int k = 0; k < p->K; ++k) {
        ObjectData& o = p->obj[k];
        if (!diversity) {
            o.d_div = nullptr;  // the buffer stays with the plan's allocations
            continue;
        }
        const int n = p->N, W = o.W;
        std::vector<float> hb((size_t)p->J * W * W, 0.f);
        for (int j = 0; j < p->J; ++j)
            for (int yy = 0; yy < W; ++yy)
                for (int xx = 0; xx < W; ++xx) {
                    const size_t g = (size_t)(o.x0 + yy) * n + (o.x0 + xx);
                    hb[((size_t)j * W + yy) * W + xx] = diversity[((size_t)k * p->J + j) * n * n + g];
                }
        if (!o.d_div_buf && (st = dev_alloc(p, &o.d_div_buf, hb.size()))) return st;
        if ((e = cudaMemcpyAsync(o.d_div_buf, hb.data(), hb.size() * sizeof(float), cudaMemcpyHostToDevice, s)))
            return cuda_fail(e, "upload diversity");
        o.d_div = o.d_div_buf;
    }
    if ((e = cudaStreamSynchronize(s))) return cuda_fail(e, "upload diversity");
    return MFBD_OK;
}

namespace {

// Field geometry of the front and back end: patches of N px at stride
// N - overlap that fit in height x width must number the plan's P.
int front_params(mfbd_plan_t p, int height, int width, int overlap, int border, FrontParams* f) {
    if (p->flags & MFBD_FLAG_FULL_SPECTRUM)
        return fail(MFBD_ERR_UNSUPPORTED, "the field front and back end use half spectra");
    const int n = p->N;
    if (overlap < 0 || overlap >= n) return fail(MFBD_ERR_INVALID_ARG, "overlap must be in [0, n_pix)");
    if (border < 0 || 2 * border > n) return fail(MFBD_ERR_INVALID_ARG, "border must be in [0, n_pix / 2]");
    if (height < n || width < n) return fail(MFBD_ERR_INVALID_ARG, "the field is smaller than a patch");
    const int st = n - overlap;
    const long long ny = (height - n) / st + 1, nx = (width - n) / st + 1;
    if (ny * nx != p->P)
        return fail(MFBD_ERR_INVALID_ARG, "the plan's n_patches differs from the patches that fit in the field");
    *f = FrontParams{};
    f->N = n;
    f->P = p->P;
    f->K = p->K;
    f->J = p->J;
    f->H = height;
    f->Wimg = width;
    f->nx = (int)nx;
    f->stride = st;
    f->border = border;
    f->es = (n / 2 + 1) | 1;
    return MFBD_OK;
}

}  // namespace

int mfbd_spectra_from_frames(mfbd_plan_t p, const float* frames, int height, int width, int overlap, int border,
                             void* spectra, void* stream) {
    int st = check_plan(p);
    if (st) return st;
    if (!frames || !spectra) return fail(MFBD_ERR_INVALID_ARG, "frames and spectra must not be NULL");
    FrontParams f;
    if ((st = front_params(p, height, width, overlap, border, &f))) return st;
    if ((st = set_device(p))) return st;
    f.frames = frames;
    f.spectra = static_cast<float2*>(spectra);
    f.err = p->d_err;
    cudaError_t e = launch_spectra_from_frames(f, p->sms, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        p->failed = true;
        return cuda_fail(e, "spectra from frames");
    }
    return MFBD_OK;
}

int mfbd_merge_objects(mfbd_plan_t p, const void* object, int height, int width, int overlap, int border,
                       float* image, void* stream) {
    int st = check_plan(p);
    if (st) return st;
    if (!object || !image) return fail(MFBD_ERR_INVALID_ARG, "object and image must not be NULL");
    FrontParams f;
    if ((st = front_params(p, height, width, overlap, border, &f))) return st;
    if ((st = set_device(p))) return st;
    if (!p->d_oimg && (st = dev_alloc(p, &p->d_oimg, (size_t)p->P * p->K * p->N * p->N))) return st;
    f.object = static_cast<const float2*>(object);
    f.oimg = p->d_oimg;
    f.image = image;
    cudaError_t e = launch_merge_objects(f, p->sms, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        p->failed = true;
        return cuda_fail(e, "merge objects");
    }
    return MFBD_OK;
}

int mfbd_filter_objects(mfbd_plan_t p, void* object, const float* f_lower, const float* f_upper, void* stream) {
    int st = check_plan(p);
    if (st) return st;
    if (!object || !f_lower || !f_upper) return fail(MFBD_ERR_INVALID_ARG, "object and cutoffs must not be NULL");
    FilterParams f{};
    f.N = p->N;
    f.P = p->P;
    f.K = p->K;
    f.ld = (p->flags & MFBD_FLAG_FULL_SPECTRUM) ? p->N : p->N / 2 + 1;
    f.object = static_cast<float2*>(object);
    for (int k = 0; k < p->K; ++k) {
        if (!(f_lower[k] >= 0.f) || !(f_upper[k] > f_lower[k]) || !std::isfinite(f_upper[k]))
            return fail(MFBD_ERR_INVALID_ARG, "cutoffs must satisfy 0 <= f_lower < f_upper");
        f.inv_diam[k] = 1.0f / p->obj[k].diam;
        f.f_lower[k] = f_lower[k];
        f.f_upper[k] = f_upper[k];
    }
    if ((st = set_device(p))) return st;
    cudaError_t e = launch_filter_objects(f, p->sms, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        p->failed = true;
        return cuda_fail(e, "filter objects");
    }
    return MFBD_OK;
}

int mfbd_ls_filter_objects(mfbd_plan_t p, const void* spectra, const void* otf, float noise_power, void* object,
                           float* filter, void* stream) {
    int st = check_plan(p);
    if (st) return st;
    if (!spectra || !otf) return fail(MFBD_ERR_INVALID_ARG, "spectra and otf must not be NULL");
    if (!object && !filter) return fail(MFBD_ERR_INVALID_ARG, "object or filter must be given");
    if (!std::isfinite(noise_power)) return fail(MFBD_ERR_INVALID_ARG, "noise_power must be finite");
    LsFilterParams f{};
    f.N = p->N;
    f.P = p->P;
    f.K = p->K;
    f.J = p->J;
    f.spec_ld = (p->flags & MFBD_FLAG_FULL_SPECTRUM) ? p->N : p->N / 2 + 1;
    f.obj_ld = f.spec_ld;
    f.noise_power = noise_power;
    f.spectra = static_cast<const float2*>(spectra);
    f.otf = static_cast<const float2*>(otf);
    f.weights = p->d_weights;
    f.object = static_cast<float2*>(object);
    f.filter = filter;
    if ((st = set_device(p))) return st;
    if (!filter && !p->d_lsraw && (st = dev_alloc(p, &p->d_lsraw, (size_t)p->P * p->K * p->N * (p->N / 2 + 1))))
        return st;
    f.raw = filter ? filter : p->d_lsraw;
    cudaError_t e = launch_ls_filter(f, p->sms, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        p->failed = true;
        return cuda_fail(e, "Lofdahl-Scharmer filter");
    }
    return MFBD_OK;
}

int mfbd_plan_check(mfbd_plan_t p, void* stream) {
    int st = check_plan(p);
    if (st) return st;
    if ((st = set_device(p))) return st;
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        p->failed = true;
        return cuda_fail(e, "plan stream");
    }
    int flag = 0;
    if ((e = cudaMemcpy(&flag, p->d_err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "read the plan's error flag");
    if (flag) {
        cudaMemset(p->d_err, 0, sizeof(int));
        return fail(MFBD_ERR_TIMEOUT, "a bounded device-side wait gave up; the results of the calls since the "
                                      "last check are invalid");
    }
    return MFBD_OK;
}

int mfbd_plan_get_info(mfbd_plan_t p, mfbd_plan_info* info) {
    if (!p || !info) return fail(MFBD_ERR_INVALID_ARG, "NULL argument");
    std::memset(info, 0, sizeof *info);
    info->n_pix = p->N;
    info->n_patches = p->P;
    info->n_objects = p->K;
    info->n_frames = p->J;
    info->n_modes = p->M;
    for (int k = 0; k < p->K; ++k) {
        info->pupil_pixels[k] = p->obj[k].npup;
        info->pupil_box[k] = p->obj[k].W;
    }
    info->workspace_bytes = p->workspace;
    info->slots_per_cta = p->generic ? 0 : p->geo.slots;
    info->reduction_split = p->rsplit;
    info->ctas = p->ctas;
    info->fused_ctas = p->fused ? p->fused_ctas : 0;
    info->tc_projection = p->obj[0].tc_planes > 0 ? 1 : 0;
    info->tc_adjoint = p->tc_grad ? 1 : 0;
    return MFBD_OK;
}

int mfbd_forward(mfbd_plan_t p, const float* coeffs, const void* spectra, double* loss, void* object,
                 void* stream) {
    int st = check_plan(p);
    if (st) return st;
    if (p->P == 0) {
        p->have_forward = true;
        return MFBD_OK;
    }
    if (!coeffs || !spectra || !loss) return fail(MFBD_ERR_INVALID_ARG, "coeffs, spectra and loss are required");
    if ((st = set_device(p))) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((st = run_phase(p, coeffs, s, 0, p->P))) return st;
    if ((st = run_fused(p, ST_FWD | ST_RED, spectra, loss, object, p->d_gscr, s, 0, p->P))) return st;
    p->have_forward = true;
    return MFBD_OK;
}

int mfbd_backward(mfbd_plan_t p, float* grad, void* stream) {
    int st = check_plan(p);
    if (st) return st;
    if (!p->have_forward) return fail(MFBD_ERR_STATE, "mfbd_backward needs a preceding mfbd_forward");
    if (p->P == 0) return MFBD_OK;
    if (!grad) return fail(MFBD_ERR_INVALID_ARG, "grad is NULL");
    if ((st = set_device(p))) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((st = run_fused(p, ST_ADJ, nullptr, nullptr, nullptr, p->d_gscr, s, 0, p->P))) return st;
    return run_grad(p, grad, s, 0, p->P);
}

int mfbd_loss_grad(mfbd_plan_t p, const float* coeffs, const void* spectra, double* loss, void* object,
                   float* grad, void* stream) {
    int st = check_plan(p);
    if (st) return st;
    if (p->P == 0) return MFBD_OK;
    if (!coeffs || !spectra || !loss || !grad)
        return fail(MFBD_ERR_INVALID_ARG, "coeffs, spectra, loss and grad are required");
    if ((st = set_device(p))) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((st = run_phase(p, coeffs, s, 0, p->P))) return st;
    if (p->fused) {  // one launch; nothing is kept for mfbd_backward
        p->have_forward = false;
        if ((st = run_pairs(p, spectra, loss, object, s, 0, p->P))) return st;
        return run_grad(p, grad, s, 0, p->P);
    }
    if ((st = run_fused(p, ST_FWD | ST_RED | ST_ADJ, spectra, loss, object, p->d_gscr, s, 0, p->P))) return st;
    if ((st = run_grad(p, grad, s, 0, p->P))) return st;
    p->have_forward = true;
    return MFBD_OK;
}

int mfbd_loss_grad_explicit(mfbd_plan_t p, const float* coeffs, const void* spectra, const void* object,
                            double* loss, float* grad, void* grad_object, void* stream) {
    int st = check_plan(p);
    if (st) return st;
    if (p->P == 0) return MFBD_OK;
    if (!coeffs || !spectra || !object || !loss || !grad)
        return fail(MFBD_ERR_INVALID_ARG, "coeffs, spectra, object, loss and grad are required");
    if ((st = set_device(p))) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    p->have_forward = false;  // the seeds will belong to the given objects
    if ((st = run_phase(p, coeffs, s, 0, p->P))) return st;
    p->x_oin = object;
    p->x_gobj = grad_object;
    st = p->fused ? run_pairs(p, spectra, loss, nullptr, s, 0, p->P)
                  : run_fused(p, ST_FWD | ST_RED | ST_ADJ, spectra, loss, nullptr, p->d_gscr, s, 0, p->P);
    p->x_oin = nullptr;
    p->x_gobj = nullptr;
    if (st) return st;
    return run_grad(p, grad, s, 0, p->P);
}

int mfbd_loss_grad_host(mfbd_plan_t p, const float* coeffs, const void* spectra, double* loss, void* object,
                        float* grad, int n_chunks, void* stream) {
    int st = check_plan(p);
    if (st) return st;
    if (p->P == 0) return MFBD_OK;
    if (!coeffs || !spectra || !loss || !grad)
        return fail(MFBD_ERR_INVALID_ARG, "coeffs, spectra, loss and grad are required");
    if ((st = set_device(p))) return st;
    const int P = p->P, J = p->J, M = p->M;
    if (n_chunks <= 0) {
        // ~120 patches per chunk: the last chunk's kernels, which no copy
        // overlaps, stay short (measured on the 961-patch field: 3 chunks
        // 2.22 ms, 8 chunks 2.05 ms per evaluation, the host link bounding it)
        n_chunks = P / 120;
        n_chunks = n_chunks < 1 ? 1 : (n_chunks > 16 ? 16 : n_chunks);
    }
    if (n_chunks > P) n_chunks = P;
    const int cp = (P + n_chunks - 1) / n_chunks;  // patches per chunk (the last may have fewer)
    n_chunks = (P + cp - 1) / cp;
    if ((st = host_setup(p, cp, object != nullptr))) {
        p->failed = true;
        return st;
    }
    auto& h = p->host;
    const size_t sp = spectrum_patch_bytes(p), op = object_patch_bytes(p);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
#define MFBD_HOST_TRY(call)                        \
    if ((e = (call)) != cudaSuccess) {             \
        p->failed = true;                          \
        return cuda_fail(e, "host pipeline");      \
    }
    // the copies start after the work already queued on `stream`
    MFBD_HOST_TRY(cudaEventRecord(h.ev_start, s));
    MFBD_HOST_TRY(cudaStreamWaitEvent(h.h2d, h.ev_start, 0));
    MFBD_HOST_TRY(cudaStreamWaitEvent(h.d2h, h.ev_start, 0));
    MFBD_HOST_TRY(cudaMemcpyAsync(h.d_coeffs, coeffs, (size_t)P * J * M * sizeof(float), cudaMemcpyHostToDevice,
                                  h.h2d));
    MFBD_HOST_TRY(cudaEventRecord(h.ev_coeffs, h.h2d));
    MFBD_HOST_TRY(cudaStreamWaitEvent(s, h.ev_coeffs, 0));
    for (int c = 0; c < n_chunks; ++c) {
        const int b = c & 1, p0 = c * cp, np = P - p0 < cp ? P - p0 : cp;
        // chunk c's spectra go into the buffer chunk c - 2 read; its
        // reduction kernel is the only reader
        if (c >= 2) MFBD_HOST_TRY(cudaStreamWaitEvent(h.h2d, h.ev_consumed[b], 0));
        MFBD_HOST_TRY(cudaMemcpyAsync(h.d_spec[b], static_cast<const char*>(spectra) + (size_t)p0 * sp,
                                      (size_t)np * sp, cudaMemcpyHostToDevice, h.h2d));
        MFBD_HOST_TRY(cudaEventRecord(h.ev_copied[b], h.h2d));
        void* obj = object && h.d_object ? static_cast<char*>(h.d_object) + (size_t)p0 * op : nullptr;
        // phases and forward passes need only the coefficients: they run
        // while the chunk's spectra are still in flight
        if ((st = run_phase(p, h.d_coeffs + (size_t)p0 * J * M, s, p0, np))) return st;
        if (p->fused) {  // the fused kernel reads the spectra from its first pass on
            MFBD_HOST_TRY(cudaStreamWaitEvent(s, h.ev_copied[b], 0));
            if ((st = run_pairs(p, h.d_spec[b], h.d_loss + p0, obj, s, p0, np))) return st;
            MFBD_HOST_TRY(cudaEventRecord(h.ev_consumed[b], s));
        } else {
            if ((st = run_fused(p, ST_FWD, nullptr, nullptr, nullptr, p->d_gscr, s, p0, np))) return st;
            MFBD_HOST_TRY(cudaStreamWaitEvent(s, h.ev_copied[b], 0));
            if ((st = run_fused(p, ST_RED, h.d_spec[b], h.d_loss + p0, obj, p->d_gscr, s, p0, np))) return st;
            MFBD_HOST_TRY(cudaEventRecord(h.ev_consumed[b], s));
            if ((st = run_fused(p, ST_ADJ, nullptr, nullptr, nullptr, p->d_gscr, s, p0, np))) return st;
        }
        if ((st = run_grad(p, h.d_grad + (size_t)p0 * J * M, s, p0, np))) return st;
        MFBD_HOST_TRY(cudaEventRecord(h.ev_done, s));
        MFBD_HOST_TRY(cudaStreamWaitEvent(h.d2h, h.ev_done, 0));
        MFBD_HOST_TRY(cudaMemcpyAsync(loss + p0, h.d_loss + p0, (size_t)np * sizeof(double), cudaMemcpyDeviceToHost,
                                      h.d2h));
        MFBD_HOST_TRY(cudaMemcpyAsync(grad + (size_t)p0 * J * M, h.d_grad + (size_t)p0 * J * M,
                                      (size_t)np * J * M * sizeof(float), cudaMemcpyDeviceToHost, h.d2h));
        if (obj)
            MFBD_HOST_TRY(cudaMemcpyAsync(static_cast<char*>(object) + (size_t)p0 * op, obj, (size_t)np * op,
                                          cudaMemcpyDeviceToHost, h.d2h));
    }
    // `stream` completes only after the last read-back
    MFBD_HOST_TRY(cudaEventRecord(h.ev_end, h.d2h));
    MFBD_HOST_TRY(cudaStreamWaitEvent(s, h.ev_end, 0));
#undef MFBD_HOST_TRY
    p->have_forward = false;  // the per-unit buffers hold the last chunk only
    return MFBD_OK;
}

int mfbd_otf(mfbd_plan_t p, const float* coeffs, void* otf, void* stream) {
    int st = check_plan(p);
    if (st) return st;
    if (p->P == 0) return MFBD_OK;
    if (!coeffs || !otf) return fail(MFBD_ERR_INVALID_ARG, "coeffs and otf are required");
    if ((st = set_device(p))) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    p->have_forward = false;  // the phases now belong to these coefficients
    if ((st = run_phase(p, coeffs, s, 0, p->P))) return st;
    return run_fused(p, ST_FWD | ST_OTF_ONLY, nullptr, nullptr, nullptr, static_cast<float2*>(otf), s, 0, p->P);
}

}  // extern "C"
