// Data front and back end of a field (Sec. 5.2, "Division in patches and
// apodization"): the data spectra of every patch and frame from the frames,
// and the mosaic of the patch objects.
//
// Spectra: one CTA per unit (patch, object, frame), persistent. The patch is
// staged in shared memory by coalesced row loads; its mean is subtracted,
// the modified Hanning window w[y] w[x] applied and the mean added back; rows y and y + N/2 are transformed as one complex line
// and split into two half spectra, then the half-spectrum columns (columns
// 0 and N/2, real after the row transforms, packed as one line) are
// transformed along y: the unnormalised 2-D DFT of the apodised patch,
// kx <= N/2.
//
// Mosaic: (1) per (patch, object) the inverse 2-D DFT of the object's half
// spectrum, normalised by 1/N^2: columns along ky (0 and N/2 packed, both
// transforms real), then row pairs Hermitian-extended along kx; (2) per
// mosaic pixel, the average of the patches covering it weighted by the
// window, summed in patch order (deterministic); a CTA per mosaic row.
//
// Object filter: the top-hat filter with a cosine transition of Sec. 4.1.1
// applied to objects in place (one thread per frequency).
//
// Spectra of 64 px patches whose columns start on 16-byte boundaries (patch
// stride and frame width multiples of 4) take the TMA form: the patch comes
// into shared memory as two 64 x 32 float boxes of a 2-D tensor map over the
// frames (128-byte swizzle, so that a lane reading its row with 16-byte loads
// meets no bank conflict); the half spectra between the row and column
// passes go to the same bytes, and the next unit's patch is requested into
// them as soon as the lanes hold their columns in registers. 18 KB of shared
// memory and at most 168 registers per warp give twelve warps per SM; its
// arrival is awaited on an mbarrier with a bounded wait.
//
// The window (a raised-cosine transition of `border` px at each edge,
// evaluated at pixel centres) is computed per CTA in shared memory with
// cosf.
#include "mfbd_internal.h"
#include "tma.cuh"
#include "unit_passes.cuh"

#include <cmath>

namespace mfbd_dev {

namespace {

using namespace unitpass;

// Threads per CTA: one warp for N <= 64 (32 lines per round, every lane
// busy in the N/2-line passes), 128 for N = 96, 128 (64 lines of two lanes).
template <int N>
struct FrontCta {
    static constexpr int THREADS = N <= 64 ? 32 : Geo<N>::THREADS;
    static constexpr int LINES = N <= 64 ? 32 : Geo<N>::LINES;
};

__device__ void window_to_smem(float* w, int n, int border) {
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
        const int e = x < n - 1 - x ? x : n - 1 - x;  // distance to the nearer edge
        w[x] = e < border ? 0.5f * (1.0f - cosf(3.14159265358979f * ((float)e + 0.5f) / (float)border)) : 1.0f;
    }
}

template <int N>
__global__ void __launch_bounds__(FrontCta<N>::THREADS) spectra_kernel(const FrontParams prm) {
    constexpr int S = Geo<N>::S, L = Geo<N>::L, NH = Geo<N>::NH, LINES = FrontCta<N>::LINES;
    constexpr int T = FrontCta<N>::THREADS;
    extern __shared__ __align__(16) unsigned char fsm[];
    float* win = reinterpret_cast<float*>(fsm);                     // [N]
    double* red = reinterpret_cast<double*>(fsm + 16 * ((N * 4 + 15) / 16));  // [THREADS / 32]
    float2* E = reinterpret_cast<float2*>(fsm + 16 * ((N * 4 + 15) / 16) + 16 * 8);
    float* Ef = reinterpret_cast<float*>(E);
    const int es = prm.es;
    const int t = threadIdx.x, sub = t % S, li = t / S;
    window_to_smem(win, N, prm.border);  // read after the first barrier below
    const long long units = (long long)prm.P * prm.K * prm.J;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        const int j = (int)(u % prm.J);
        const long long pk = u / prm.J;
        const int k = (int)(pk % prm.K);
        const int p = (int)(pk / prm.K);
        const int y0 = (p / prm.nx) * prm.stride, x0 = (p % prm.nx) * prm.stride;
        const float* F = prm.frames + ((size_t)k * prm.J + j) * prm.H * prm.Wimg + (size_t)y0 * prm.Wimg + x0;
        // the patch into shared memory (coalesced rows; float rows 2 es
        // apart, in the exchange buffer) and its mean
        __syncthreads();  // the previous unit's column pass has read E
        // per-thread FP32 partial sums over four interleaved accumulators
        // (fixed order), combined across the CTA in FP64
        constexpr int kPer = N * N / T;
        float part[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int e = t + i * T;
            const int y = e / N, x = e - y * N;
            const float v = F[(size_t)y * prm.Wimg + x];
            Ef[(size_t)y * 2 * es + x] = v;
            part[i & 3] += v;
        }
        double acc = ((double)part[0] + (double)part[1]) + ((double)part[2] + (double)part[3]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if ((t & 31) == 0) red[t >> 5] = acc;
        __syncthreads();
        double tot = 0.0;
        for (int w = 0; w < T / 32; ++w) tot += red[w];
        const float m = (float)(tot / (N * N));
        // rows y and y + N/2 of the apodised patch as one complex line; the
        // line's lanes read both rows before any of them writes the two half
        // spectra over them
        // (every lane of a warp runs every round, inactive ones on zeros, so
        // that the warp-wide __syncwarp and shuffles see all lanes)
        for (int y0 = 0; y0 < N / 2; y0 += LINES) {
            const int y = y0 + li;
            const bool act = y < N / 2;
            float2 v[L];
#pragma unroll
            for (int n = 0; n < L; ++n) {
                const int x = S * n + sub;
                float a = 0.f, b = 0.f;
                if (act) {
                    a = (Ef[(size_t)y * 2 * es + x] - m) * win[y] * win[x] + m;
                    b = (Ef[(size_t)(y + N / 2) * 2 * es + x] - m) * win[y + N / 2] * win[x] + m;
                }
                v[n] = make_float2(a, b);
            }
            line_fft<N, -1>(v, sub);
            __syncwarp();
            fftreg::static_for<0, L>([&](auto kk) {
                constexpr int kq = decltype(kk)::value;
                const float2 pc = conj_partner<N, kq>(v);
                const int kx = sub * L + kq;
                if (act && kx <= N / 2) {
                    const float2 ra = cscale(cadd(v[kq], pc), 0.5f);
                    const float2 d = cscale(csub(v[kq], pc), 0.5f);
                    E[y * es + kx] = ra;
                    E[(y + N / 2) * es + kx] = make_float2(d.y, -d.x);
                }
            });
        }
        __syncthreads();
        // columns kx = 1 .. N/2 - 1; line 0 packs the real columns 0 and N/2
        float2* D = prm.spectra + (size_t)u * N * NH;
        for (int l0 = 0; l0 < N / 2; l0 += LINES) {
            const int kx = l0 + li;
            const bool act = kx < N / 2;
            float2 v[L];
#pragma unroll
            for (int n = 0; n < L; ++n) {
                const int ky = S * n + sub;
                v[n] = !act ? make_float2(0.f, 0.f)
                            : kx == 0 ? make_float2(E[ky * es].x, E[ky * es + N / 2].x) : E[ky * es + kx];
            }
            line_fft<N, -1>(v, sub);
            fftreg::static_for<0, L>([&](auto kk) {
                constexpr int kq = decltype(kk)::value;
                const float2 pc = conj_partner<N, kq>(v);
                const int ky = sub * L + kq;
                if (!act) {
                } else if (kx > 0) {
                    D[ky * NH + kx] = v[kq];
                } else {
                    const float2 d0 = cscale(cadd(v[kq], pc), 0.5f);
                    const float2 d = cscale(csub(v[kq], pc), 0.5f);
                    D[ky * NH] = d0;
                    D[ky * NH + N / 2] = make_float2(d.y, -d.x);
                }
            });
        }
        __syncthreads();
    }
}

constexpr int kTmaBoxCols = 32;                            // 128 bytes of float: the swizzle span
constexpr uint32_t kTmaTileBytes = 64 * 64 * sizeof(float);  // one 64 x 64 patch, two boxes

// Shared memory of the TMA form: one area (1024-byte aligned) that holds the
// swizzled patch and then, once the lanes hold their rows, the exchange
// buffer of the half spectra; the mbarrier.
__host__ __device__ inline size_t tma_front_area(int es) {
    const size_t ex = ((size_t)64 * es * sizeof(float2) + 15) & ~(size_t)15;
    const size_t z = kTmaTileBytes + 64 * sizeof(float2);  // the tile and, past it, one packed column
    return ex > z ? ex : z;
}
size_t tma_front_smem(int es) { return 1024 + tma_front_area(es) + 16; }

// Row y of the swizzled patch as float4 chunks: chunk c (floats 4c..4c+3 of
// the row) of the box `half` (columns 32 half .. 32 half + 31).
__device__ __forceinline__ float4 tile_chunk(const float* tile, int half, int y, int c) {
    const unsigned char* b = reinterpret_cast<const unsigned char*>(tile) + half * (kTmaTileBytes / 2) + y * 128 +
                             ((c ^ (y & 7)) << 4);
    return *reinterpret_cast<const float4*>(b);
}

// The window of the TMA form, from the host: w[x] for the 64 columns (the
// same factors serve the rows).
struct Window64 {
    float w[64];
};

// Apodisation (p - m) w_y w_x + m as a transform of (p - m) w_x along x,
// the factor w_y applied to each row's half spectrum, and the transform of
// the constant m (m N^2 at frequency 0) added to the DC term.
__global__ void __launch_bounds__(32, 12) spectra_tma_kernel(const FrontParams prm, const __grid_constant__ CUtensorMap map,
                                                             const Window64 win) {
    constexpr int N = 64, NH = N / 2 + 1;
    extern __shared__ __align__(16) unsigned char fsm[];
    unsigned char* base = fsm + ((1024 - (tma::smem_u32(fsm) & 1023)) & 1023);
    const int es = prm.es, lane = threadIdx.x;
    const size_t area = tma_front_area(es);
    float* tile = reinterpret_cast<float*>(base);
    float2* E = reinterpret_cast<float2*>(base);  // the same bytes as the tile
    // lane 0's packed column, past the bytes the next patch's TMA load fills
    float2* Z = reinterpret_cast<float2*>(base + kTmaTileBytes);
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + area);
    const long long units = (long long)prm.P * prm.K * prm.J;
    // frame row and column of unit u's patch in the tensor map
    auto request = [&](long long u) {
        const int j = (int)(u % prm.J);
        const long long pk = u / prm.J;
        const int k = (int)(pk % prm.K);
        const int p = (int)(pk / prm.K);
        const int x0 = (p % prm.nx) * prm.stride;
        const int row = (k * prm.J + j) * prm.H + (p / prm.nx) * prm.stride;
        tma::mbar_arrive_expect_tx(bar, kTmaTileBytes);
        tma::load_2d(tile, &map, x0, row, bar);
        tma::load_2d(tile + kTmaTileBytes / 8, &map, x0 + kTmaBoxCols, row, bar);
    };
    if (lane == 0) {
        tma::mbar_init(bar, 1);
        if ((long long)blockIdx.x < units) request(blockIdx.x);
    }
    __syncwarp();
    // half the window factors of this lane's rows (the row split's 1/2)
    const float ha = 0.5f * win.w[lane], hb = 0.5f * win.w[lane + N / 2];
    uint32_t parity = 0;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        if (!tma::mbar_wait(bar, parity)) {  // the copy never arrived: flag it and stop
            if (lane == 0) atomicExch(prm.err, 1);
            return;
        }
        parity ^= 1;
        // rows lane and lane + N/2 of the patch as the real and imaginary
        // parts of one line, with per-lane FP32 sums for the mean
        float2 v[N];
        float part[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float4 a = tile_chunk(tile, h, lane, c), b = tile_chunk(tile, h, lane + N / 2, c);
                const int x = 32 * h + 4 * c;
                v[x] = make_float2(a.x, b.x);
                v[x + 1] = make_float2(a.y, b.y);
                v[x + 2] = make_float2(a.z, b.z);
                v[x + 3] = make_float2(a.w, b.w);
                part[c & 3] += (a.x + a.y) + (a.z + a.w) + ((b.x + b.y) + (b.z + b.w));
            }
        }
        __syncwarp();  // every lane holds its rows: the half spectra may overwrite the tile
        double acc = ((double)part[0] + (double)part[1]) + ((double)part[2] + (double)part[3]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        const float m = (float)(acc / (N * N));
        const float2 nm = make_float2(-m, -m);
#pragma unroll
        for (int x = 0; x < N; ++x) v[x] = __fmul2_rn(__fadd2_rn(v[x], nm), make_float2(win.w[x], win.w[x]));
        float2* D = prm.spectra + (size_t)u * N * NH;
        const int kx = lane;
        // pass 0 transforms the row pairs, pass 1 the half-spectrum columns:
        // one copy of the transform's code serves both
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            line_fft<N, -1>(v, 0);
            if (pass == 0) {
                // rows: split the line's transform into the two rows' half
                // spectra, each times its w_y; columns 0 and N/2 (real) are
                // stored packed as one complex column in column 0
                E[lane * es] = make_float2(v[0].x * (2.f * ha), v[N / 2].x * (2.f * ha));
                E[(lane + N / 2) * es] = make_float2(v[0].y * (2.f * hb), v[N / 2].y * (2.f * hb));
                fftreg::static_for<1, N / 2>([&](auto kk) {
                    constexpr int k = decltype(kk)::value;
                    const float2 pc = conj_partner<N, k>(v);
                    const float2 ra = cscale(cadd(v[k], pc), ha);
                    const float2 d = cscale(csub(v[k], pc), hb);
                    E[lane * es + k] = ra;
                    E[(lane + N / 2) * es + k] = make_float2(d.y, -d.x);
                });
                __syncwarp();
                // columns kx = 1 .. N/2 - 1, and in lane 0 the packed real columns
#pragma unroll
                for (int ky = 0; ky < N; ++ky) v[ky] = E[ky * es + kx];
                __syncwarp();
                // every lane holds its column: the next unit's patch may land
                // in the area, under this unit's column transforms and stores
                if (lane == 0 && u + gridDim.x < units) {
                    tma::fence_proxy_async_smem();
                    request(u + gridDim.x);
                }
            } else {
                // lane 0 keeps the transform of the packed columns in shared memory
#pragma unroll
                for (int ky = 0; ky < N; ++ky) {
                    if (kx > 0) D[ky * NH + kx] = v[ky];
                    else Z[ky] = v[ky];
                }
            }
        }
        __syncwarp();
        // split the packed columns' transform Z into kx = 0 and N/2:
        // X0 = (Z[ky] + conj Z[-ky]) / 2, X(N/2) = (Z[ky] - conj Z[-ky]) / (2i);
        // lane l takes ky = l and l + N/2
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int ky = lane + h * (N / 2);
            const float2 z = Z[ky], zp = cconj(Z[(N - ky) & (N - 1)]);
            float2 d0 = cscale(cadd(z, zp), 0.5f);
            const float2 d = cscale(csub(z, zp), 0.5f);
            if (ky == 0) d0.x += m * (float)(N * N);  // the constant's transform
            D[ky * NH] = d0;
            D[ky * NH + N / 2] = make_float2(d.y, -d.x);
        }
        __syncwarp();
    }
}

template <int N>
__global__ void __launch_bounds__(FrontCta<N>::THREADS) object_image_kernel(const FrontParams prm) {
    constexpr int S = Geo<N>::S, L = Geo<N>::L, NH = Geo<N>::NH, LINES = FrontCta<N>::LINES;
    extern __shared__ __align__(16) unsigned char fsm[];
    float2* E = reinterpret_cast<float2*>(fsm);
    const int es = prm.es;
    const int t = threadIdx.x, sub = t % S, li = t / S;
    const float sc = 1.0f / (float)(N * N);
    const long long units = (long long)prm.P * prm.K;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        const float2* O = prm.object + (size_t)u * N * NH;
        // columns along ky: F^H of O[:, kx]; line 0 packs the columns 0 and
        // N/2 (both inverse transforms are real)
        for (int l0 = 0; l0 < N / 2; l0 += LINES) {
            const int kx = l0 + li;
            const bool act = kx < N / 2;
            float2 v[L];
#pragma unroll
            for (int n = 0; n < L; ++n) {
                const int ky = S * n + sub;
                float2 z = make_float2(0.f, 0.f);
                if (!act) {
                } else if (kx == 0) {
                    const float2 a = O[ky * NH], b = O[ky * NH + N / 2];
                    z = make_float2(a.x - b.y, a.y + b.x);  // a + i b
                } else {
                    z = O[ky * NH + kx];
                }
                v[n] = cconj(z);
            }
            line_fft<N, -1>(v, sub);
            if (act) {
#pragma unroll
                for (int q = 0; q < L; ++q) E[(sub * L + q) * es + kx] = cconj(v[q]);
            }
        }
        __syncthreads();
        // rows y and y + N/2: F^H of the Hermitian-extended rows of T, packed
        // as T_y + i T_(y+N/2); both results real
        float* img = prm.oimg + (size_t)u * N * N;
        for (int y0 = 0; y0 < N / 2; y0 += LINES) {
            const int y = y0 + li;
            const bool act = y < N / 2;
            float2 v[L];
#pragma unroll
            for (int n = 0; n < L; ++n) {
                const int x = S * n + sub;
                float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
                if (!act) {
                } else if (x == 0) {
                    a = make_float2(E[y * es].x, 0.f);
                    b = make_float2(E[(y + N / 2) * es].x, 0.f);
                } else if (x == N / 2) {
                    a = make_float2(E[y * es].y, 0.f);
                    b = make_float2(E[(y + N / 2) * es].y, 0.f);
                } else if (x < N / 2) {
                    a = E[y * es + x];
                    b = E[(y + N / 2) * es + x];
                } else {
                    a = cconj(E[y * es + N - x]);
                    b = cconj(E[(y + N / 2) * es + N - x]);
                }
                v[n] = make_float2(a.x - b.y, -(a.y + b.x));  // conj(a + i b)
            }
            line_fft<N, -1>(v, sub);
            if (act) {  // 16-byte stores: four consecutive pixels of a row
                static_assert(L % 4 == 0, "rows are stored four pixels at a time");
                float4* ra = reinterpret_cast<float4*>(img + (size_t)y * N + sub * L);
                float4* rb = reinterpret_cast<float4*>(img + (size_t)(y + N / 2) * N + sub * L);
#pragma unroll
                for (int q = 0; q < L; q += 4) {
                    ra[q / 4] = make_float4(v[q].x * sc, v[q + 1].x * sc, v[q + 2].x * sc, v[q + 3].x * sc);
                    rb[q / 4] = make_float4(-v[q].y * sc, -v[q + 1].y * sc, -v[q + 2].y * sc, -v[q + 3].y * sc);
                }
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) merge_kernel(const FrontParams prm) {
    extern __shared__ __align__(16) unsigned char fsm[];
    float* win = reinterpret_cast<float*>(fsm);
    const int N = prm.N, s = prm.stride;
    window_to_smem(win, N, prm.border);
    __syncthreads();
    const int ny = prm.P / prm.nx;
    // one mosaic row (object k, row Y) per CTA iteration: the patch rows
    // covering it are the same for the whole row
    const long long rows = (long long)prm.K * prm.H;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int k = (int)(row / prm.H), Y = (int)(row - (long long)k * prm.H);
        const int iy0 = Y >= N ? (Y - N + s) / s : 0, iy1 = min(ny - 1, Y / s);
        float* out = prm.image + (size_t)row * prm.Wimg;
        for (int X = threadIdx.x; X < prm.Wimg; X += 256) {
            const int ix0 = X >= N ? (X - N + s) / s : 0, ix1 = min(prm.nx - 1, X / s);
            float num = 0.f, den = 0.f;
            for (int iy = iy0; iy <= iy1; ++iy) {
                const int dy = Y - iy * s;
                if (dy >= N) continue;
                for (int ix = ix0; ix <= ix1; ++ix) {
                    const int dx = X - ix * s;
                    if (dx >= N) continue;
                    const float w = win[dy] * win[dx];
                    const int p = iy * prm.nx + ix;
                    num = fmaf(w, prm.oimg[(((size_t)p * prm.K + k) * N + dy) * N + dx], num);
                    den += w;
                }
            }
            out[X] = den > 0.f ? num / den : 0.f;
        }
    }
}

// Object filter (Sec. 4.1.1): O_k(u) *= H_k(u), 1 below f_lower, 0 above
// f_upper, a cosine transition between, f = |u| / D_p,k.
__global__ void __launch_bounds__(256) filter_kernel(const FilterParams prm) {
    const int N = prm.N, ld = prm.ld;
    const long long per = (long long)N * ld;
    const long long n = (long long)prm.P * prm.K * per;
    for (long long e = blockIdx.x * 256ll + threadIdx.x; e < n; e += (long long)gridDim.x * 256) {
        const int k = (int)((e / per) % prm.K);
        const long long r = e % per;
        const int ky = (int)(r / ld), kx = (int)(r - (long long)ky * ld);
        const float fy = (float)(ky <= N / 2 ? ky : ky - N), fx = (float)(kx <= N / 2 ? kx : kx - N);
        const float f = sqrtf(fy * fy + fx * fx) * prm.inv_diam[k];
        const float lo = prm.f_lower[k], hi = prm.f_upper[k];
        float h = f <= lo ? 1.0f : 0.0f;
        if (f > lo && f < hi) h = 0.5f * (1.0f + cosf(3.14159265358979f * (f - lo) / (hi - lo)));
        const float2 o = prm.object[e];
        prm.object[e] = make_float2(o.x * h, o.y * h);
    }
}

template <class Kern>
cudaError_t launch_persistent_front(Kern kern, int threads, size_t smem, long long work, int sms, const FrontParams& prm,
                                    cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long ctas = (long long)sms * per_sm;
    if (ctas > work) ctas = work;
    kern<<<(int)ctas, threads, smem, s>>>(prm);
    return cudaGetLastError();
}

}  // namespace

size_t front_smem(int N, int es) { return (size_t)16 * ((N * 4 + 15) / 16) + 16 * 8 + (size_t)N * es * sizeof(float2); }

namespace tma {

bool encode_f32_2d_swizzle128(CUtensorMap* map, const float* base, uint64_t cols, uint64_t rows, uint32_t box_cols,
                              uint32_t box_rows) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    if (box_cols * sizeof(float) != 128) return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * sizeof(float)};
    const cuuint32_t box[2] = {box_cols, box_rows};
    const cuuint32_t elem[2] = {1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, elem,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tma

bool spectra_tma_eligible(const FrontParams& prm) {
    return prm.N == 64 && prm.stride % 4 == 0 && prm.Wimg % 4 == 0 &&
           (reinterpret_cast<uintptr_t>(prm.frames) & 15) == 0 && prm.err != nullptr &&
           (long long)prm.K * prm.J * prm.H < (1ll << 31);
}

cudaError_t launch_spectra_from_frames(const FrontParams& prm, int sms, cudaStream_t s) {
    const long long units = (long long)prm.P * prm.K * prm.J;
    if (units == 0) return cudaSuccess;
    if (spectra_tma_eligible(prm)) {
        CUtensorMap map;
        if (tma::encode_f32_2d_swizzle128(&map, prm.frames, (uint64_t)prm.Wimg,
                                          (uint64_t)prm.K * prm.J * prm.H, kTmaBoxCols, 64)) {
            const size_t smem = tma_front_smem(prm.es);
            cudaError_t e = cudaFuncSetAttribute(spectra_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
            int per_sm = 0;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spectra_tma_kernel, 32, smem)) !=
                cudaSuccess)
                return e;
            if (per_sm < 1) return cudaErrorInvalidConfiguration;
            long long ctas = (long long)sms * per_sm;
            if (ctas > units) ctas = units;
            Window64 win;  // the window of window_to_smem, evaluated in double
            for (int x = 0; x < 64; ++x) {
                const int e = x < 63 - x ? x : 63 - x;
                win.w[x] = e < prm.border ? (float)(0.5 * (1.0 - std::cos(3.14159265358979323846 * (e + 0.5) /
                                                                          prm.border)))
                                          : 1.0f;
            }
            spectra_tma_kernel<<<(int)ctas, 32, smem, s>>>(prm, map, win);
            return cudaGetLastError();
        }
    }
    const size_t smem = front_smem(prm.N, prm.es);
    switch (prm.N) {
        case 48: return launch_persistent_front(spectra_kernel<48>, FrontCta<48>::THREADS, smem, units, sms, prm, s);
        case 64: return launch_persistent_front(spectra_kernel<64>, FrontCta<64>::THREADS, smem, units, sms, prm, s);
        case 96: return launch_persistent_front(spectra_kernel<96>, FrontCta<96>::THREADS, smem, units, sms, prm, s);
        case 128: return launch_persistent_front(spectra_kernel<128>, FrontCta<128>::THREADS, smem, units, sms, prm, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_filter_objects(const FilterParams& prm, int sms, cudaStream_t s) {
    const long long n = (long long)prm.P * prm.K * prm.N * prm.ld;
    if (n == 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 8ll * sms) blocks = 8ll * sms;
    filter_kernel<<<(int)blocks, 256, 0, s>>>(prm);
    return cudaGetLastError();
}

cudaError_t launch_merge_objects(const FrontParams& prm, int sms, cudaStream_t s) {
    const long long units = (long long)prm.P * prm.K;
    if (units > 0) {
        const size_t smem = (size_t)prm.N * prm.es * sizeof(float2);
        cudaError_t e = cudaErrorInvalidValue;
        switch (prm.N) {
            case 48: e = launch_persistent_front(object_image_kernel<48>, FrontCta<48>::THREADS, smem, units, sms, prm, s); break;
            case 64: e = launch_persistent_front(object_image_kernel<64>, FrontCta<64>::THREADS, smem, units, sms, prm, s); break;
            case 96: e = launch_persistent_front(object_image_kernel<96>, FrontCta<96>::THREADS, smem, units, sms, prm, s); break;
            case 128: e = launch_persistent_front(object_image_kernel<128>, FrontCta<128>::THREADS, smem, units, sms, prm, s); break;
            default: break;
        }
        if (e != cudaSuccess) return e;
    }
    const long long rows = (long long)prm.H * prm.K;
    if (rows == 0 || prm.Wimg == 0) return cudaSuccess;
    long long blocks = rows;  // one mosaic row per CTA
    if (blocks > 16ll * sms) blocks = 16ll * sms;
    merge_kernel<<<(int)blocks, 256, (size_t)prm.N * sizeof(float), s>>>(prm);
    return cudaGetLastError();
}

}  // namespace mfbd_dev
