/*
 * mfbd_testing.h -- host-side self-test hooks of the MOMFBD library.
 *
 * These entry points run the library's register-FFT building blocks on the
 * HOST CPU (they are compiled __host__ __device__), so their arithmetic can
 * be checked without a GPU. They are not part of the compute path and the
 * paper has no counterpart; they exist for testing only.
 */
#ifndef MFBD_TESTING_H
#define MFBD_TESTING_H

#ifdef __cplusplus
extern "C" {
#endif

/* kind selects the transform (length 64 unless stated), unnormalised:
 *   0  complex forward  in: 64 complex (128 floats)  out: 64 complex
 *   1  complex adjoint  in: 64 complex               out: 64 complex
 *   2  real-to-complex  in: 64 floats                out: 33 complex (66 floats)
 *   3  complex-to-real  in: 33 complex (Hermitian)   out: 64 floats
 *   4  complex forward, length 32
 *   5  complex forward, length 64, radix-4 network
 *   6  complex adjoint, length 64, radix-4 network
 *   7  complex forward, length 48 (three 16-point FFTs and a radix-3 stage)
 *   8  complex adjoint, length 48
 * Forward: X[k] = sum x[n] exp(-2 pi i n k / N); adjoint uses exp(+...).
 * Returns 0 (MFBD_OK) or 1 (MFBD_ERR_INVALID_ARG) for an unknown kind or
 * NULL pointers. */
int mfbd_test_fft_host(int kind, const float* in, float* out);

/* The work list of a batch schedule, built on the host exactly as
 * mfbd_batch_create / mfbd_batch_set_schedule build it, for problems of
 * sizes[i] = {N, P, K, J} (n problems), mode MFBD_BATCH_ONE_LAUNCH or
 * MFBD_BATCH_STAGED and window_units. Writes up to `cap` items as rows of 5
 * ints {kind (0 phases, 1 forward, 2 reduction, 3 adjoint, 4 modal adjoint),
 * problem, patch, k * J + j of the first unit, the number e of further
 * units (k J + j) + 1 .. (k J + j) + e it covers} and the total in *count. Returns 0, or 1 for bad arguments. */
int mfbd_test_batch_items(const int* sizes, int n, int mode, int window_units, int* items, long long cap,
                          long long* count);

/* Throughput probe of the fused multiply-add pipe on the current device
 * (a measurement hook of the benchmark; it runs on the GPU, unlike the
 * hooks above). fp64 = 0 times FP32 FMAs, 1 FP64 FMAs: 8 CTAs of 256
 * threads per SM, each thread 8 independent chains of 16 x iters FMAs, one
 * untimed warm-up launch and one launch timed with CUDA events on `stream`
 * (a cudaStream_t as void*). Writes the flops of the timed launch (2 per
 * FMA) to *flops and its time to *ms; synchronises the stream. Returns 0,
 * MFBD_ERR_INVALID_ARG (NULL pointers, iters < 1), MFBD_ERR_UNSUPPORTED (no
 * device) or MFBD_ERR_CUDA. */
int mfbd_probe_fma_rate(int fp64, long long iters, void* stream, double* flops, float* ms);

#ifdef __cplusplus
}
#endif

#endif /* MFBD_TESTING_H */
