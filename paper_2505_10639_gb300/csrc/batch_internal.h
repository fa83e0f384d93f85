// Launch interface of the batched persistent kernel (uneven batches of
// problems: patch sizes 48-128, objects, frames and modes per problem).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "../../include/mfbd.h"
#include "mfbd_internal.h"

namespace mfbd_dev {

// Descriptor checks of mfbd_plan_create (MFBD_OK or the status, with the
// reason recorded for mfbd_last_error).
int validate_desc(const mfbd_plan_desc* d);

// One (problem, object): plan-time data on the device.
struct BatchObj {
    int W;                  // side of the pupil's bounding box
    int mw;                 // 32-bit words per box mask row
    int ldt;                // row stride of bt (>= M: bases are shared between problems)
    float scale;            // c_k = lambda_0 / lambda_k
    float inv_z;            // 1 / (N^2 n_pup)
    const float* bm;        // [M][W*W] basis on the box (0 outside the pupil)
    const float* bt;        // [W*W][ldt] the same, transposed
    const uint32_t* mask;   // [W][mw] box rows
    const uint32_t* supp;   // [N][sw] OTF-support rows over kx <= N/2
    const uint64_t* cmask;  // [W][2] box columns: bit y = pupil pixel
    const uint64_t* csupp;  // [N/2+1][2] half-spectrum columns: bit ky = OTF support
    long long phi_koff;     // floats from a patch's phase block to this object's [J][stride(W)]
};

// One problem of the batch: its sizes and where its data sit in the packed
// caller buffers and in the batch's scratch.
struct BatchProblem {
    int N, P, K, J, M, sw;
    double gamma;
    const float* weights;   // [K][J]
    long long coeff_off;    // floats: [P][J][M] in coeffs and grad
    long long spec_off;     // complex: [P][K][J][N][N/2+1] in spectra
    long long loss_off;     // doubles: [P] in loss
    long long obj_off;      // complex: [P][K][N][N/2+1] in object
    long long gscr_off;     // complex: per unit (p K + k) J + j, N (N/2+1) each
    long long pscr_off;     // complex: per unit, N^2 each (the field)
    long long phi_off;      // floats: per patch phi_patch floats, then per object phi_koff
    long long phi_patch;    // J * sum_k stride(W_k)
    long long ctr_off;      // index of patch 0's dependency counters
    BatchObj obj[kMaxObjects];
};

// Work items. F and A cover one unit (patch, object, frame), or up to four
// consecutive units k J + j of one patch when N <= 64 (one warp per unit);
// P, R and G cover one patch.
enum BatchKind : int {
    BK_PROJ = 0,   // phases of every object and frame of a patch (Eq. 22)
    BK_FWD = 1,    // forward passes of a unit (Eqs. 20-21, OTF)
    BK_RED = 2,    // frame reduction of a patch (Eqs. 11-12, adjoint seeds)
    BK_ADJ = 3,    // adjoint passes of a unit (-> dL/dphi)
    BK_GRAD = 4    // modal adjoint of a patch (dL/da)
};

struct BatchItem {
    int kind;       // BatchKind
    int prob;       // problem index
    int patch;      // patch within the problem
    int kj;         // F, A: k * J + j of the first unit; P, R, G: 0
    int extra;      // F, A: further units kj + 1 .. kj + extra in the item (N <= 64: 0..3)
    int pad[3];
};

// Dependency counters of a patch (cleared before every launch).
enum BatchCtr : int { BC_PROJ = 0, BC_FWD = 1, BC_RED = 2, BC_ADJ = 3, BC_COUNT = 4 };

struct BatchParams {
    const BatchProblem* probs;
    const BatchItem* items;
    int n_items;
    int item0;              // first item of this launch (staged mode)
    int wait;               // 1: check dependencies (one launch over all kinds)
    int kinds;              // bit k set: items of kind k run (the others are skipped, and signalled)
    int es_small, es_large; // exchange-buffer row strides (complex) for N <= 64 and N > 64
    int* ctr;               // [patches][BC_COUNT] counters
    int* ticket;            // next item to take
    int* err;               // set when a dependency wait gives up
    const float* coeffs;
    const float2* spectra;
    double* loss;
    float2* object;         // or null
    float* grad;
    float2* gscr;
    float2* pscr;
    float* phi;
    float* gphi;
};

constexpr int kBT = 128;  // threads per CTA of the batch kernel
constexpr int kJC = 8;    // frames per register tile of its P and G items

size_t batch_smem(int es_small, int es_large);
// Kernel variants: 0, a register budget of up to 255 a thread (2 CTAs per
// SM); 1, up to 170 (3 CTAs per SM). Also sets the variant's dynamic
// shared-memory limit to `smem` (required before launch_batch).
int batch_max_ctas_per_sm(size_t smem, int variant);
// One launch of `ctas` CTAs over items [item0, item0 + n_items).
cudaError_t launch_batch(const BatchParams& prm, int ctas, size_t smem, int variant, cudaStream_t s);
// The same per register budget (MINB CTAs per SM), defined in
// batch_kernels.cuh and instantiated in batch_kernel_v2.cu / batch_kernel_v3.cu.
template <int MINB> int batch_max_ctas_variant(size_t smem);
template <int MINB> cudaError_t launch_batch_variant(const BatchParams& prm, int ctas, size_t smem, cudaStream_t s);

}  // namespace mfbd_dev
