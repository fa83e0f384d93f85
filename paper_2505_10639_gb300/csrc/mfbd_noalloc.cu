// Allocation-free entry point: mfbd_phase_loss_grad_noalloc (see mfbd.h).
//
// Some callers cannot allocate device memory at all: a plugin whose host
// framework owns every allocation, code running where the CUDA allocator is
// off limits, or a program with a fixed device-memory budget decided up
// front. Such a caller cannot create a plan (mfbd_plan_create allocates its
// workspaces), so this entry point runs the fused kernel without a plan: the
// caller passes the phases, spectra and output buffers, and every byte of
// working memory the kernel needs comes from one fixed array compiled into
// this library, which each GPU that loads the library keeps until exit.
#include "../../include/mfbd.h"
#include "mfbd_internal.h"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

using namespace mfbd_dev;

// 16 MiB per device: 64 KiB of per-call constants (pupil and OTF-support
// bits by row and by column, frame weights) followed by the per-unit scratch of one batch of
// patches: [Pb][K][J][N][N/2+1] complex64 OTFs / adjoint seeds, then
// [Pb][K][J][N][N] complex64 fields.
static __device__ __align__(256) unsigned char g_static_workspace[(size_t)16 << 20];

namespace {

constexpr size_t kStaticBytes = sizeof(g_static_workspace);
constexpr size_t kConstBytes = (size_t)64 << 10;
constexpr size_t kBitsBytes = (size_t)kMaxObjects * 4 * kN * sizeof(uint64_t);  // 16 KiB
constexpr int kMaxDevices = 64;

std::mutex g_mu;
void* g_device_ptr[kMaxDevices] = {};                   // device address of the array, per device
alignas(16) unsigned char g_host_consts[kConstBytes];   // staging of the constants (under g_mu)

// Device address of the static array on the current device. The host-side
// name g_static_workspace is only a stand-in for the symbol, so it is looked
// up once per device (with that device current) and cached.
int static_workspace(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return set_error(MFBD_ERR_UNSUPPORTED, "device index too large");
    if (!g_device_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_workspace);
        if (e != cudaSuccess) return set_cuda_error(e, "cudaGetSymbolAddress");
        g_device_ptr[dev] = p;
    }
    *out = g_device_ptr[dev];
    return MFBD_OK;
}

int check_desc(const mfbd_plan_desc* d) {
    if (!d) return set_error(MFBD_ERR_INVALID_ARG, "descriptor is NULL");
    if (d->n_patches < 0) return set_error(MFBD_ERR_INVALID_ARG, "n_patches must be >= 0");
    if (d->n_objects < 1 || d->n_objects > kMaxObjects)
        return set_error(MFBD_ERR_INVALID_ARG, "n_objects must be in 1..8");
    if (d->n_frames < 1 || d->n_frames > 1024)
        return set_error(MFBD_ERR_INVALID_ARG, "n_frames must be in 1..1024");
    if (!d->pupil_diam_px) return set_error(MFBD_ERR_INVALID_ARG, "pupil_diam_px is NULL");
    if (d->n_pix != kN) return set_error(MFBD_ERR_UNSUPPORTED, "n_pix must be 64");
    for (int k = 0; k < d->n_objects; ++k)
        if (!(d->pupil_diam_px[k] > 0.f) || !(d->pupil_diam_px[k] <= (float)kN))
            return set_error(MFBD_ERR_INVALID_ARG, "pupil diameter must be in (0, n_pix]");
    if (!(d->central_obscuration >= 0.f) || !(d->central_obscuration < 1.f))
        return set_error(MFBD_ERR_INVALID_ARG, "central_obscuration must be in [0, 1)");
    if (!(d->gamma > 0.0) || !std::isfinite(d->gamma))
        return set_error(MFBD_ERR_INVALID_ARG, "gamma must be > 0");
    if (d->frame_weight)
        for (int i = 0; i < d->n_objects * d->n_frames; ++i)
            if (!(d->frame_weight[i] >= 0.f) || !std::isfinite(d->frame_weight[i]))
                return set_error(MFBD_ERR_INVALID_ARG, "frame weights must be finite and >= 0");
    if (d->flags & ~MFBD_FLAG_FULL_SPECTRUM) return set_error(MFBD_ERR_INVALID_ARG, "unknown flags");
    return MFBD_OK;
}

// Pupil bit rows over the full grid (bit x of row y), the same sampling rule
// as the plan path: centre (N-1)/2, inside iff r^2 <= (D/2)^2 in double.
void pupil_rows(float diam, float obsc, uint64_t (&rows)[kN]) {
    const double c = (kN - 1) / 2.0, r = (double)diam * 0.5, ro = (double)obsc * r;
    for (int y = 0; y < kN; ++y) {
        rows[y] = 0;
        for (int x = 0; x < kN; ++x) {
            const double dx = x - c, dy = y - c, r2 = dx * dx + dy * dy;
            bool in = r2 <= r * r;
            if (obsc > 0.f) in = in && r2 >= ro * ro;
            if (in) rows[y] |= 1ull << x;
        }
    }
}

// Exact OTF support on the half spectrum: u is in it iff some pupil pixel v
// has v + u (mod N) inside the pupil as well.
void support_rows(const uint64_t (&rows)[kN], uint64_t (&supp)[kN]) {
    for (int dy = 0; dy < kN; ++dy) {
        supp[dy] = 0;
        for (int dx = 0; dx <= kN / 2; ++dx) {
            bool any = false;
            for (int y = 0; y < kN && !any; ++y) {
                const uint64_t a = rows[y];
                const uint64_t b = rows[(y + dy) % kN];
                const uint64_t bs = dx == 0 ? b : ((b >> dx) | (b << (kN - dx)));
                any = (a & bs) != 0;
            }
            if (any) supp[dy] |= 1ull << dx;
        }
    }
}

}  // namespace

extern "C" int mfbd_phase_loss_grad_noalloc(const mfbd_plan_desc* desc, const float* phase, const void* spectra,
                                            double* loss, void* object, float* grad_phase, void* stream) {
    int st = check_desc(desc);
    if (st != MFBD_OK) return st;
    const int P = desc->n_patches, K = desc->n_objects, J = desc->n_frames;
    const size_t per_patch = (size_t)K * J * (kHalf + kN * kN) * sizeof(float2);
    if (per_patch > kStaticBytes - kConstBytes)
        return set_error(MFBD_ERR_INVALID_ARG,
                         "n_objects x n_frames exceeds the static workspace (at most 336 per call)");
    if (P == 0) return MFBD_OK;
    if (!phase || !spectra || !loss || !grad_phase)
        return set_error(MFBD_ERR_INVALID_ARG, "phase, spectra, loss and grad_phase are required");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaGetDevice");
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return set_cuda_error(e, "cudaDeviceGetAttribute");
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    std::lock_guard<std::mutex> lock(g_mu);
    void* ws = nullptr;
    if ((st = static_workspace(dev, &ws)) != MFBD_OK) return st;
    unsigned char* base = static_cast<unsigned char*>(ws);

    // per-call constants: bit rows of every object, then the frame weights
    std::memset(g_host_consts, 0, kBitsBytes + (size_t)K * J * sizeof(float));
    uint64_t* bits = reinterpret_cast<uint64_t*>(g_host_consts);
    float* wts = reinterpret_cast<float*>(g_host_consts + kBitsBytes);
    FusedParams f{};
    int max_box = 1;
    for (int k = 0; k < K; ++k) {
        uint64_t rows[kN], supp[kN];
        pupil_rows(desc->pupil_diam_px[k], desc->central_obscuration, rows);
        int lo = kN, hi = -1, npup = 0;
        for (int y = 0; y < kN; ++y)
            for (int x = 0; x < kN; ++x)
                if ((rows[y] >> x) & 1ull) {
                    ++npup;
                    lo = lo < x ? lo : x;
                    lo = lo < y ? lo : y;
                    hi = hi > x ? hi : x;
                    hi = hi > y ? hi : y;
                }
        if (npup == 0) return set_error(MFBD_ERR_INVALID_ARG, "pupil has no pixel");
        support_rows(rows, supp);
        const int W = hi - lo + 1;
        max_box = max_box > W ? max_box : W;
        // per object: pupil rows of the box, OTF-support rows, then the
        // same bits by column (box columns; support columns kx <= N/2)
        uint64_t* mk = bits + (size_t)k * 4 * kN;
        for (int yy = 0; yy < W; ++yy) mk[yy] = rows[lo + yy] >> lo;
        if (W < 64)
            for (int yy = 0; yy < W; ++yy) mk[yy] &= (1ull << W) - 1;
        std::memcpy(mk + kN, supp, sizeof supp);
        for (int yy = 0; yy < W; ++yy)
            for (int xx = 0; xx < W; ++xx)
                if ((mk[yy] >> xx) & 1ull) mk[2 * kN + xx] |= 1ull << yy;
        for (int ky = 0; ky < kN; ++ky)
            for (int kx = 0; kx <= kN / 2; ++kx)
                if ((supp[ky] >> kx) & 1ull) mk[3 * kN + kx] |= 1ull << ky;
        ObjParams& ob = f.obj[k];
        ob.W = W;
        ob.x0 = lo;
        ob.inv_z = (float)(1.0 / ((double)kN * kN * npup));
        ob.phi_off = (long long)k * P * J * kN * kN;
        ob.phi_unit = (long long)kN * kN;
        ob.phi_org = lo * kN + lo;
        ob.phi_ld = kN;
        ob.mask = reinterpret_cast<const uint64_t*>(base) + (size_t)k * 4 * kN;
        ob.supp = ob.mask + kN;
        ob.cmask = ob.mask + 2 * kN;
        ob.csupp = ob.mask + 3 * kN;
    }
    for (int i = 0; i < K * J; ++i) wts[i] = desc->frame_weight ? desc->frame_weight[i] : 1.0f;
    if ((e = cudaMemcpyAsync(base, g_host_consts, kBitsBytes + (size_t)K * J * sizeof(float),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return set_cuda_error(e, "constant upload");
    // dL/dphi is written on each pupil's box only; the rest of the grid is 0
    if ((e = cudaMemsetAsync(grad_phase, 0, (size_t)K * P * J * kN * kN * sizeof(float), s)) != cudaSuccess)
        return set_cuda_error(e, "cudaMemsetAsync");

    f.K = K;
    f.J = J;
    f.M = 0;
    f.gamma = desc->gamma;
    f.weights = reinterpret_cast<const float*>(base + kBitsBytes);
    f.spec_ld = (desc->flags & MFBD_FLAG_FULL_SPECTRUM) ? kN : kN / 2 + 1;
    const FusedGeometry g = fused_geometry(max_box);
    if (max_ctas_per_sm(g) < 1) return set_error(MFBD_ERR_UNSUPPORTED, "pass kernel does not fit on this device");
    // the patches go through in batches whose scratch fits the array
    const int batch = (int)((kStaticBytes - kConstBytes) / per_patch);
    float2* gscr = reinterpret_cast<float2*>(base + kConstBytes);
    for (int p0 = 0; p0 < P; p0 += batch) {
        const int pb = P - p0 < batch ? P - p0 : batch;
        const size_t img = (size_t)p0 * J * kN * kN;
        f.P = pb;
        f.phi = phase + img;
        f.gphi = grad_phase + img;
        f.gscr = gscr;
        f.pscr = gscr + (size_t)pb * K * J * kHalf;
        f.spectra = static_cast<const float2*>(spectra) + (size_t)p0 * K * J * kN * f.spec_ld;
        f.loss = loss + p0;
        f.object = object ? static_cast<float2*>(object) + (size_t)p0 * K * kN * f.spec_ld : nullptr;
        if ((e = launch_fused(f, MODE_FUSED, g, sms, s)) != cudaSuccess) return set_cuda_error(e, "kernels");
    }
    return MFBD_OK;
}
