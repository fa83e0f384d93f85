// C ABI of uneven batches (mfbd_batch_*): validation, shared plan-time data,
// packed layouts, the item list of a schedule, launches and the autotuner.
// The arithmetic is in batch_kernels.cu and unit_passes.cuh.
#include "../../include/mfbd_testing.h"
#include "batch_internal.h"
#include "optics_host.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <exception>
#include <map>
#include <string>
#include <tuple>
#include <vector>

using namespace mfbd_dev;

namespace {

constexpr int kMaxSchedules = 16;

long long round_up(long long x, long long a) { return (x + a - 1) / a * a; }
long long phi_stride(int W) { return round_up((long long)W * W, 64); }

// Plan-time data shared by every (problem, object) with the same sampling.
struct SharedObj {
    int W = 0, x0 = 0, npup = 0, mw = 0, M = 0;
    float* bm = nullptr;       // [M][W*W]
    float* bt = nullptr;       // [W*W][M]
    uint32_t* mask = nullptr;  // [W][mw]
    uint32_t* supp = nullptr;  // [N][sw]
    uint64_t* cmask = nullptr; // [W][2] box columns
    uint64_t* csupp = nullptr; // [N/2+1][2] support columns
};

}  // namespace

struct mfbd_batch {
    int device = 0, sms = 0;
    int n = 0;                          // problems
    std::vector<BatchProblem> probs;    // host copy of the device table
    std::vector<long long> coeff_off, spec_off, loss_off, obj_off;
    long long coeff_floats = 0, spec_complex = 0, loss_doubles = 0, obj_complex = 0;
    long long patches = 0, units = 0;
    int es_small = 33, es_large = 65;
    size_t smem = 0;
    int max_per_sm_v[2] = {0, 0};       // CTAs per SM of each kernel variant
    // schedule
    int mode = MFBD_BATCH_ONE_LAUNCH, window_units = 0, ctas_per_sm = 0, variant = 0;
    std::vector<int> stage_begin;       // staged mode: first item of each kind, then the end
    long long n_items = 0;
    // device memory
    BatchProblem* d_probs = nullptr;
    BatchItem* d_items = nullptr;
    int* d_ctr = nullptr;               // [patches][BC_COUNT], then 8 tickets, then the error flag
    float* d_phi = nullptr;
    float* d_gphi = nullptr;
    float2* d_gscr = nullptr;
    float2* d_pscr = nullptr;
    size_t workspace = 0;
    std::vector<void*> allocations;
    bool failed = false;
};

namespace {

template <class T>
int balloc(mfbd_batch* b, T** ptr, size_t count) {
    *ptr = nullptr;
    if (count == 0) return MFBD_OK;
    void* raw = nullptr;
    cudaError_t e = cudaMalloc(&raw, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(MFBD_ERR_OOM, (std::string("cudaMalloc: ") + cudaGetErrorString(e)).c_str());
    }
    b->allocations.push_back(raw);
    b->workspace += count * sizeof(T);
    *ptr = static_cast<T*>(raw);
    return MFBD_OK;
}

void batch_release(mfbd_batch* b) {
    for (void* a : b->allocations) cudaFree(a);
    b->allocations.clear();
}

// Relative cost of a unit of size N (for ordering items, largest first).
int unit_cost(int N) { return N * N; }

// The item list of a schedule. Per patch: P, the F items (units k J + j in
// fours when N <= 64), R, the A items, G. Staged: all P, all F, all R, all A, all
// G (each a launch). One launch: the patches are cut into windows of about
// `window` 64 px units (0: one window) and window w's kind s goes into block
// w + s, each block listing its older windows first, so an item's
// dependencies sit about one block earlier in the list; within a window the
// larger patches come first.
std::vector<BatchItem> build_items(const mfbd_batch* b, int mode, int window, std::vector<int>* stage_begin) {
    struct PatchRef {
        int prob, patch;
    };
    std::vector<PatchRef> order;
    for (int i = 0; i < b->n; ++i)
        for (int p = 0; p < b->probs[i].P; ++p) order.push_back({i, p});
    auto items_of = [&](const PatchRef& r, int kind, std::vector<BatchItem>& out) {
        const BatchProblem& pr = b->probs[r.prob];
        BatchItem it{};
        it.kind = kind;
        it.prob = r.prob;
        it.patch = r.patch;
        if (kind == BK_FWD || kind == BK_ADJ) {
            const int units = pr.K * pr.J;  // (k, j) flattened: a group of four may span two objects
            for (int u = 0; u < units;) {
                it.kj = u;
                it.extra = pr.N <= 64 ? std::min(3, units - 1 - u) : 0;
                out.push_back(it);
                u += 1 + it.extra;
            }
        } else {
            out.push_back(it);
        }
    };
    std::vector<std::vector<PatchRef>> windows;
    if (mode == MFBD_BATCH_STAGED || window <= 0) {
        windows.push_back(order);
    } else {
        long long acc = 0;
        windows.emplace_back();
        for (const PatchRef& r : order) {
            const BatchProblem& pr = b->probs[r.prob];
            const long long u = (long long)pr.K * pr.J * unit_cost(pr.N) / (64 * 64);
            if (acc > 0 && acc + u > window) {
                windows.emplace_back();
                acc = 0;
            }
            windows.back().push_back(r);
            acc += u;
        }
    }
    for (auto& w : windows)
        std::stable_sort(w.begin(), w.end(), [&](const PatchRef& x, const PatchRef& y) {
            return unit_cost(b->probs[x.prob].N) > unit_cost(b->probs[y.prob].N);
        });
    std::vector<BatchItem> items;
    const int kinds[5] = {BK_PROJ, BK_FWD, BK_RED, BK_ADJ, BK_GRAD};
    if (stage_begin) stage_begin->clear();
    if (mode == MFBD_BATCH_STAGED) {
        for (int s = 0; s < 5; ++s) {
            if (stage_begin) stage_begin->push_back((int)items.size());
            for (const PatchRef& r : windows[0]) items_of(r, kinds[s], items);
        }
        if (stage_begin) stage_begin->push_back((int)items.size());
        return items;
    }
    const int nw = (int)windows.size();
    for (int blk = 0; blk < nw + 4; ++blk)
        for (int s = 4; s >= 0; --s) {  // the oldest window's kind first
            const int w = blk - s;
            if (w < 0 || w >= nw) continue;
            for (const PatchRef& r : windows[w]) items_of(r, kinds[s], items);
        }
    return items;
}

int apply_schedule(mfbd_batch* b, int mode, int window, int ctas_per_sm, int variant) {
    if (mode != MFBD_BATCH_ONE_LAUNCH && mode != MFBD_BATCH_STAGED)
        return set_error(MFBD_ERR_INVALID_ARG, "unknown batch schedule mode");
    if (variant != 0 && variant != 1) return set_error(MFBD_ERR_INVALID_ARG, "unknown batch kernel variant");
    if (b->max_per_sm_v[variant] < 1)
        return set_error(MFBD_ERR_UNSUPPORTED, "this batch kernel variant does not fit on this device");
    if (ctas_per_sm < 0 || ctas_per_sm > b->max_per_sm_v[variant])
        return set_error(MFBD_ERR_INVALID_ARG, "ctas_per_sm out of range for this batch");
    std::vector<int> sb;
    std::vector<BatchItem> items = build_items(b, mode, window, &sb);
    if ((long long)items.size() != b->n_items) return set_error(MFBD_ERR_STATE, "item count changed");
    if (!items.empty()) {
        cudaError_t e =
            cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return set_cuda_error(e, "upload batch items");
    }
    b->mode = mode;
    b->window_units = mode == MFBD_BATCH_STAGED ? 0 : std::max(0, window);
    b->ctas_per_sm = ctas_per_sm == 0 ? b->max_per_sm_v[variant] : ctas_per_sm;
    b->variant = variant;
    b->stage_begin = sb;
    return MFBD_OK;
}

int check_batch(mfbd_batch_t b) {
    if (!b) return set_error(MFBD_ERR_INVALID_ARG, "batch is NULL");
    if (b->failed) return set_error(MFBD_ERR_STATE, "batch failed earlier");
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaSetDevice");
    return MFBD_OK;
}

// One evaluation: the kinds of item in the bit set `kinds` run (all five for
// loss + gradient; phases and forward passes for the OTF only, with the OTFs
// written to `gscr`).
int run_batch(mfbd_batch_t b, const float* coeffs, const void* spectra, double* loss, void* object, float* grad,
              float2* gscr, int kinds, cudaStream_t s) {
    if (b->n_items == 0) return MFBD_OK;
    const size_t ctr_ints = (size_t)b->patches * BC_COUNT + 8;
    cudaError_t e = cudaMemsetAsync(b->d_ctr, 0, ctr_ints * sizeof(int), s);
    BatchParams prm{};
    prm.probs = b->d_probs;
    prm.items = b->d_items;
    prm.kinds = kinds;
    prm.es_small = b->es_small;
    prm.es_large = b->es_large;
    prm.ctr = b->d_ctr;
    prm.err = b->d_ctr + ctr_ints;
    prm.coeffs = coeffs;
    prm.spectra = static_cast<const float2*>(spectra);
    prm.loss = loss;
    prm.object = static_cast<float2*>(object);
    prm.grad = grad;
    prm.gscr = gscr;
    prm.pscr = b->d_pscr;
    prm.phi = b->d_phi;
    prm.gphi = b->d_gphi;
    const long long cap = (long long)b->sms * b->ctas_per_sm;
    if (b->mode == MFBD_BATCH_ONE_LAUNCH) {
        prm.item0 = 0;
        prm.n_items = (int)b->n_items;
        prm.wait = 1;
        prm.ticket = b->d_ctr + (size_t)b->patches * BC_COUNT;
        if (e == cudaSuccess)
            e = launch_batch(prm, (int)std::min<long long>(cap, b->n_items), b->smem, b->variant, s);
    } else {
        for (int st = 0; st < 5 && e == cudaSuccess; ++st) {
            if (!((kinds >> st) & 1)) continue;
            prm.item0 = b->stage_begin[st];
            prm.n_items = b->stage_begin[st + 1] - b->stage_begin[st];
            prm.wait = 0;
            prm.ticket = b->d_ctr + (size_t)b->patches * BC_COUNT + st;
            e = launch_batch(prm, (int)std::min<long long>(cap, std::max(1, prm.n_items)), b->smem, b->variant, s);
        }
    }
    if (e != cudaSuccess) {
        b->failed = true;
        return set_cuda_error(e, "batch kernel");
    }
    return MFBD_OK;
}

constexpr int kAllKinds = 0x1f;
constexpr int kOtfKinds = (1 << BK_PROJ) | (1 << BK_FWD);

int run_loss_grad(mfbd_batch_t b, const float* coeffs, const void* spectra, double* loss, void* object, float* grad,
                  cudaStream_t s) {
    if (!coeffs || !spectra || !loss || !grad)
        return set_error(MFBD_ERR_INVALID_ARG, "coeffs, spectra, loss and grad must not be NULL");
    return run_batch(b, coeffs, spectra, loss, object, grad, b->d_gscr, kAllKinds, s);
}

}  // namespace

extern "C" {

int mfbd_batch_create(mfbd_batch_t* out, const mfbd_plan_desc* problems, int n_problems, void* stream) {
    if (!out) return set_error(MFBD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_problems < 0 || (n_problems > 0 && !problems))
        return set_error(MFBD_ERR_INVALID_ARG, "problems must be an array of n_problems >= 0 descriptors");
    for (int i = 0; i < n_problems; ++i) {
        const mfbd_plan_desc* d = problems + i;
        int st = validate_desc(d);
        if (st != MFBD_OK) return st;
        if (d->precision != MFBD_PREC_FP32 || d->flags != 0)
            return set_error(MFBD_ERR_UNSUPPORTED, "batch problems take FP32 precision, half spectra and no flags");
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_cuda_error(e, "no CUDA device");
    cudaDeviceProp prop{};
    if ((e = cudaGetDeviceProperties(&prop, dev))) return set_cuda_error(e, "cudaGetDeviceProperties");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    mfbd_batch* b = new mfbd_batch();
    b->device = dev;
    b->sms = prop.multiProcessorCount;
    b->n = n_problems;
    try {
        int st;
        typedef std::tuple<int, uint32_t, uint32_t, int, int> Key;
        // shared (problem, object) data keyed by sampling and basis; Zernike
        // sets are shared across mode counts (modes 2..M+1 are a prefix)
        std::map<Key, SharedObj> shared;
        std::map<Key, int> want_m;
        auto key_of = [&](const mfbd_plan_desc* d, int k) {
            uint32_t db, ob;
            std::memcpy(&db, &d->pupil_diam_px[k], 4);
            std::memcpy(&ob, &d->central_obscuration, 4);
            const int mkey = d->basis == MFBD_BASIS_ZERNIKE ? 0 : d->n_modes;
            return std::make_tuple(d->n_pix, db, ob, d->basis, mkey);
        };
        for (int i = 0; i < n_problems; ++i) {
            const mfbd_plan_desc* d = problems + i;
            if (d->basis == MFBD_BASIS_USER) continue;
            for (int k = 0; k < d->n_objects; ++k) {
                Key key = key_of(d, k);
                want_m[key] = std::max(want_m[key], d->n_modes);
            }
        }
        std::vector<std::vector<char>> staging;  // host buffers alive until the stream syncs
        auto upload = [&](const void* src, void* dst, size_t bytes) {
            cudaError_t ee = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
            if (ee != cudaSuccess) throw set_cuda_error(ee, "upload batch data");
        };
        auto make_shared = [&](const mfbd_plan_desc* d, int k, int M, const std::vector<double>* user) {
            SharedObj so;
            const int n = d->n_pix;
            std::vector<uint8_t> mask = mfbd_host::pupil_mask(n, d->pupil_diam_px[k], d->central_obscuration);
            int lo = n, hi = -1, npup = 0;
            for (int y = 0; y < n; ++y)
                for (int x = 0; x < n; ++x)
                    if (mask[(size_t)y * n + x]) {
                        ++npup;
                        lo = std::min(lo, std::min(x, y));
                        hi = std::max(hi, std::max(x, y));
                    }
            if (npup == 0) throw set_error(MFBD_ERR_INVALID_ARG, "pupil has no pixel");
            so.W = hi - lo + 1;
            so.x0 = lo;
            so.npup = npup;
            so.M = M;
            std::vector<double> full;
            if (user) {
                full = *user;
            } else {
                mfbd_host::ModalBasis mb =
                    d->basis == MFBD_BASIS_ZERNIKE
                        ? mfbd_host::zernike_basis(n, d->pupil_diam_px[k], d->central_obscuration, M)
                        : mfbd_host::kl_basis(n, d->pupil_diam_px[k], d->central_obscuration, M);
                full = std::move(mb.modes);
            }
            const int W = so.W, npix = W * W;
            staging.emplace_back((size_t)2 * M * npix * sizeof(float));
            float* hb = reinterpret_cast<float*>(staging.back().data());
            float* ht = hb + (size_t)M * npix;
            for (int m = 0; m < M; ++m)
                for (int yy = 0; yy < W; ++yy)
                    for (int xx = 0; xx < W; ++xx) {
                        const size_t g = (size_t)(lo + yy) * n + (lo + xx);
                        const float v = mask[g] ? (float)full[(size_t)m * n * n + g] : 0.f;
                        hb[(size_t)m * npix + yy * W + xx] = v;
                        ht[(size_t)(yy * W + xx) * M + m] = v;
                    }
            so.mw = (W + 31) / 32;
            const int sw = (n / 2 + 1 + 31) / 32;
            const size_t mwords = (size_t)W * so.mw + (size_t)n * sw;
            staging.emplace_back(mwords * sizeof(uint32_t), 0);
            uint32_t* hm = reinterpret_cast<uint32_t*>(staging.back().data());
            uint32_t* hs = hm + (size_t)W * so.mw;
            for (int yy = 0; yy < W; ++yy)
                for (int xx = 0; xx < W; ++xx)
                    if (mask[(size_t)(lo + yy) * n + (lo + xx)]) hm[yy * so.mw + xx / 32] |= 1u << (xx % 32);
            std::vector<uint8_t> sup = mfbd_host::otf_support_half(mask, n);
            for (int ky = 0; ky < n; ++ky)
                for (int kx = 0; kx <= n / 2; ++kx)
                    if (sup[(size_t)ky * (n / 2 + 1) + kx]) hs[ky * sw + kx / 32] |= 1u << (kx % 32);
            if ((st = balloc(b, &so.bm, (size_t)2 * M * npix))) throw st;
            so.bt = so.bm + (size_t)M * npix;
            upload(hb, so.bm, (size_t)2 * M * npix * sizeof(float));
            if ((st = balloc(b, &so.mask, mwords))) throw st;
            so.supp = so.mask + (size_t)W * so.mw;
            upload(hm, so.mask, mwords * sizeof(uint32_t));
            const size_t cwords = (size_t)2 * W + 2 * (n / 2 + 1);
            staging.emplace_back(cwords * sizeof(uint64_t), 0);
            uint64_t* hc = reinterpret_cast<uint64_t*>(staging.back().data());
            for (int yy = 0; yy < W; ++yy)
                for (int xx = 0; xx < W; ++xx)
                    if (mask[(size_t)(lo + yy) * n + (lo + xx)]) hc[2 * xx + yy / 64] |= 1ull << (yy % 64);
            for (int ky = 0; ky < n; ++ky)
                for (int kx = 0; kx <= n / 2; ++kx)
                    if (sup[(size_t)ky * (n / 2 + 1) + kx]) hc[2 * W + 2 * kx + ky / 64] |= 1ull << (ky % 64);
            if ((st = balloc(b, &so.cmask, cwords))) throw st;
            so.csupp = so.cmask + 2 * W;
            upload(hc, so.cmask, cwords * sizeof(uint64_t));
            return so;
        };

        b->probs.resize(n_problems);
        b->coeff_off.resize(n_problems);
        b->spec_off.resize(n_problems);
        b->loss_off.resize(n_problems);
        b->obj_off.resize(n_problems);
        long long gscr = 0, pscr = 0, phi = 0, ctr = 0;
        int max_small = 0, max_large = 0;
        std::vector<std::vector<float>> weights(n_problems);
        std::vector<long long> w_off(n_problems);
        long long w_total = 0;
        for (int i = 0; i < n_problems; ++i) {
            const mfbd_plan_desc* d = problems + i;
            BatchProblem& pr = b->probs[i];
            const int n = d->n_pix, nh = n / 2 + 1;
            pr.N = n;
            pr.P = d->n_patches;
            pr.K = d->n_objects;
            pr.J = d->n_frames;
            pr.M = d->n_modes;
            pr.sw = (nh + 31) / 32;
            pr.gamma = d->gamma;
            pr.coeff_off = b->coeff_off[i] = b->coeff_floats;
            pr.spec_off = b->spec_off[i] = b->spec_complex;
            pr.loss_off = b->loss_off[i] = b->loss_doubles;
            pr.obj_off = b->obj_off[i] = b->obj_complex;
            b->coeff_floats += (long long)pr.P * pr.J * pr.M;
            b->spec_complex += (long long)pr.P * pr.K * pr.J * n * nh;
            b->loss_doubles += pr.P;
            b->obj_complex += (long long)pr.P * pr.K * n * nh;
            pr.gscr_off = gscr;
            gscr += (long long)pr.P * pr.K * pr.J * n * nh;
            pr.pscr_off = pscr;
            pscr += (long long)pr.P * pr.K * pr.J * n * n;
            pr.ctr_off = ctr;
            ctr += pr.P;
            b->patches += pr.P;
            b->units += (long long)pr.P * pr.K * pr.J;
            weights[i].assign((size_t)pr.K * pr.J, 1.0f);
            if (d->frame_weight) std::memcpy(weights[i].data(), d->frame_weight, weights[i].size() * sizeof(float));
            w_off[i] = w_total;
            w_total += (long long)weights[i].size();
            long long koff = 0;
            for (int k = 0; k < pr.K; ++k) {
                SharedObj so;
                if (d->basis == MFBD_BASIS_USER) {
                    std::vector<double> ub((size_t)pr.M * n * n);
                    const float* src = d->user_basis + (size_t)k * pr.M * n * n;
                    for (size_t q = 0; q < ub.size(); ++q) ub[q] = src[q];
                    so = make_shared(d, k, pr.M, &ub);
                } else {
                    Key key = key_of(d, k);
                    auto f = shared.find(key);
                    if (f == shared.end()) f = shared.emplace(key, make_shared(d, k, want_m[key], nullptr)).first;
                    so = f->second;
                }
                BatchObj& ob = pr.obj[k];
                ob.W = so.W;
                ob.mw = so.mw;
                ob.ldt = so.M;
                ob.scale = (float)(d->wavelength[0] / d->wavelength[k]);
                ob.inv_z = (float)(1.0 / ((double)n * n * so.npup));
                ob.bm = so.bm;
                ob.bt = so.bt;
                ob.mask = so.mask;
                ob.supp = so.supp;
                ob.cmask = so.cmask;
                ob.csupp = so.csupp;
                ob.phi_koff = koff;
                koff += (long long)pr.J * phi_stride(so.W);
                if (n <= 64) max_small = std::max(max_small, so.W);
                else max_large = std::max(max_large, so.W);
            }
            pr.phi_patch = koff;
            pr.phi_off = phi;
            phi += (long long)pr.P * koff;
        }
        b->es_small = std::max(33, max_small) | 1;
        b->es_large = std::max(65, max_large) | 1;
        b->smem = batch_smem(b->es_small, b->es_large);
        if (b->smem > (size_t)227 * 1024)
            throw set_error(MFBD_ERR_UNSUPPORTED, "a pupil box is too large for the batch kernel's shared memory");
        b->max_per_sm_v[0] = batch_max_ctas_per_sm(b->smem, 0);
        b->max_per_sm_v[1] = batch_max_ctas_per_sm(b->smem, 1);
        if (b->max_per_sm_v[0] < 1)
            throw set_error(MFBD_ERR_UNSUPPORTED, "the batch kernel does not fit on this device");
        // weights, problem table, scratch
        float* d_w = nullptr;
        if ((st = balloc(b, &d_w, (size_t)std::max(1ll, w_total)))) throw st;
        staging.emplace_back((size_t)std::max(1ll, w_total) * sizeof(float));
        float* hw = reinterpret_cast<float*>(staging.back().data());
        for (int i = 0; i < n_problems; ++i) {
            std::memcpy(hw + w_off[i], weights[i].data(), weights[i].size() * sizeof(float));
            b->probs[i].weights = d_w + w_off[i];
        }
        if (w_total > 0) upload(hw, d_w, (size_t)w_total * sizeof(float));
        if ((st = balloc(b, &b->d_probs, (size_t)std::max(1, n_problems)))) throw st;
        if (n_problems > 0) upload(b->probs.data(), b->d_probs, (size_t)n_problems * sizeof(BatchProblem));
        if ((st = balloc(b, &b->d_phi, (size_t)phi))) throw st;
        if ((st = balloc(b, &b->d_gphi, (size_t)phi))) throw st;
        if ((st = balloc(b, &b->d_gscr, (size_t)gscr))) throw st;
        if ((st = balloc(b, &b->d_pscr, (size_t)pscr))) throw st;
        if ((st = balloc(b, &b->d_ctr, (size_t)b->patches * BC_COUNT + 9))) throw st;
        if ((e = cudaMemsetAsync(b->d_ctr, 0, ((size_t)b->patches * BC_COUNT + 9) * sizeof(int), s)))
            throw set_cuda_error(e, "clear batch counters");
        b->n_items = (long long)build_items(b, MFBD_BATCH_ONE_LAUNCH, 0, nullptr).size();
        if (b->n_items > (1ll << 30)) throw set_error(MFBD_ERR_UNSUPPORTED, "too many work items in one batch");
        if ((st = balloc(b, &b->d_items, (size_t)std::max(1ll, b->n_items)))) throw st;
        if ((e = cudaStreamSynchronize(s))) throw set_cuda_error(e, "batch upload");
        staging.clear();
        // default schedule: one launch, windows of about 8192 64 px units
        if ((st = apply_schedule(b, MFBD_BATCH_ONE_LAUNCH, 8192, 0, 0))) throw st;
    } catch (int status) {
        batch_release(b);
        delete b;
        return status;
    } catch (const std::exception& ex) {
        batch_release(b);
        delete b;
        return set_error(MFBD_ERR_INVALID_ARG, ex.what());
    }
    *out = b;
    return MFBD_OK;
}

int mfbd_batch_destroy(mfbd_batch_t b) {
    if (!b) return MFBD_OK;
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    batch_release(b);
    delete b;
    return MFBD_OK;
}

int mfbd_batch_get_info(mfbd_batch_t b, mfbd_batch_info* info) {
    if (!b || !info) return set_error(MFBD_ERR_INVALID_ARG, "batch or info is NULL");
    info->n_problems = b->n;
    info->n_patches = b->patches;
    info->n_units = b->units;
    info->n_items = b->n_items;
    info->coeff_floats = b->coeff_floats;
    info->spectra_complex = b->spec_complex;
    info->loss_doubles = b->loss_doubles;
    info->object_complex = b->obj_complex;
    info->workspace_bytes = b->workspace;
    info->mode = b->mode;
    info->window_units = b->window_units;
    info->ctas_per_sm = b->ctas_per_sm;
    info->max_ctas_per_sm = b->max_per_sm_v[b->variant];
    info->variant = b->variant;
    info->ctas = b->sms * b->ctas_per_sm;
    info->smem_bytes = (int)b->smem;
    return MFBD_OK;
}

int mfbd_batch_get_offsets(mfbd_batch_t b, long long* coeffs, long long* spectra, long long* loss, long long* object) {
    if (!b) return set_error(MFBD_ERR_INVALID_ARG, "batch is NULL");
    for (int i = 0; i < b->n; ++i) {
        if (coeffs) coeffs[i] = b->coeff_off[i];
        if (spectra) spectra[i] = b->spec_off[i];
        if (loss) loss[i] = b->loss_off[i];
        if (object) object[i] = b->obj_off[i];
    }
    return MFBD_OK;
}

int mfbd_batch_set_schedule(mfbd_batch_t b, int mode, int window_units, int ctas_per_sm, int variant) {
    int st = check_batch(b);
    if (st) return st;
    cudaError_t e = cudaDeviceSynchronize();  // no launch may be reading the item list
    if (e != cudaSuccess) return set_cuda_error(e, "synchronise before a schedule change");
    return apply_schedule(b, mode, window_units, ctas_per_sm, variant);
}

int mfbd_batch_loss_grad(mfbd_batch_t b, const float* coeffs, const void* spectra, double* loss, void* object,
                         float* grad, void* stream) {
    int st = check_batch(b);
    if (st) return st;
    return run_loss_grad(b, coeffs, spectra, loss, object, grad, static_cast<cudaStream_t>(stream));
}

int mfbd_batch_otf(mfbd_batch_t b, const float* coeffs, void* otf, void* stream) {
    int st = check_batch(b);
    if (st) return st;
    if (!coeffs || !otf) return set_error(MFBD_ERR_INVALID_ARG, "coeffs and otf must not be NULL");
    return run_batch(b, coeffs, nullptr, nullptr, nullptr, nullptr, static_cast<float2*>(otf), kOtfKinds,
                     static_cast<cudaStream_t>(stream));
}

int mfbd_batch_check(mfbd_batch_t b, void* stream) {
    int st = check_batch(b);
    if (st) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        b->failed = true;
        return set_cuda_error(e, "batch stream");
    }
    int flag = 0;
    int* d_err = b->d_ctr + (size_t)b->patches * BC_COUNT + 8;
    if ((e = cudaMemcpy(&flag, d_err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return set_cuda_error(e, "read the batch error flag");
    if (flag) {
        cudaMemset(d_err, 0, sizeof(int));
        return set_error(MFBD_ERR_TIMEOUT, "a dependency wait of the batch kernel gave up; the results are invalid");
    }
    return MFBD_OK;
}

int mfbd_test_batch_items(const int* sizes, int n, int mode, int window_units, int* items, long long cap,
                          long long* count) {
    if (!sizes || n < 0 || !count || (cap > 0 && !items)) return MFBD_ERR_INVALID_ARG;
    if (mode != MFBD_BATCH_ONE_LAUNCH && mode != MFBD_BATCH_STAGED) return MFBD_ERR_INVALID_ARG;
    mfbd_batch b;
    b.n = n;
    b.probs.resize(n);
    for (int i = 0; i < n; ++i) {
        BatchProblem& pr = b.probs[i];
        pr.N = sizes[4 * i];
        pr.P = sizes[4 * i + 1];
        pr.K = sizes[4 * i + 2];
        pr.J = sizes[4 * i + 3];
        if (pr.N < 1 || pr.P < 0 || pr.K < 1 || pr.K > kMaxObjects || pr.J < 1) return MFBD_ERR_INVALID_ARG;
    }
    std::vector<BatchItem> v = build_items(&b, mode, window_units, nullptr);
    *count = (long long)v.size();
    for (long long i = 0; i < (long long)v.size() && i < cap; ++i) {
        int* r = items + 5 * i;
        r[0] = v[i].kind;
        r[1] = v[i].prob;
        r[2] = v[i].patch;
        r[3] = v[i].kj;
        r[4] = v[i].extra;
    }
    return MFBD_OK;
}

int mfbd_batch_autotune(mfbd_batch_t b, const float* coeffs, const void* spectra, double* loss, void* object,
                        float* grad, int reps, void* stream) {
    int st = check_batch(b);
    if (st) return st;
    if (reps < 1) reps = 2;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    struct Cand {
        int mode, window, cps, variant;
    };
    std::vector<Cand> cands;
    for (int v = 0; v < 2; ++v) {
        const int mx = b->max_per_sm_v[v];
        if (mx < 1) continue;
        for (int w : {0, 2048, 8192, 32768}) cands.push_back({MFBD_BATCH_ONE_LAUNCH, w, mx, v});
        cands.push_back({MFBD_BATCH_STAGED, 0, mx, v});
    }
    if ((int)cands.size() > kMaxSchedules) cands.resize(kMaxSchedules);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    Cand best_c = {b->mode, b->window_units, b->ctas_per_sm, b->variant};
    for (const Cand& c : cands) {
        if ((st = mfbd_batch_set_schedule(b, c.mode, c.window, c.cps, c.variant))) break;
        if ((st = run_loss_grad(b, coeffs, spectra, loss, object, grad, s))) break;  // warm-up
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && !st; ++r) st = run_loss_grad(b, coeffs, spectra, loss, object, grad, s);
        cudaEventRecord(e1, s);
        if (st) break;
        if ((st = mfbd_batch_check(b, stream))) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_c = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    return mfbd_batch_set_schedule(b, best_c.mode, best_c.window, best_c.cps, best_c.variant);
}

}  // extern "C"
