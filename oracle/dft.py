"""Discrete Fourier transforms for the oracle (test infrastructure only).

Conventions (used throughout the oracle):
  forward  X[k] = sum_n x[n] exp(-2 pi i n k / N)   (sign = -1, unnormalised)
  adjoint  x[n] = sum_k X[k] exp(+2 pi i n k / N)   (sign = +1, unnormalised, F^H)

The paper (Sec. 2.2.1) evaluates its convolutions with FFTs. This module is
the oracle's own implementation: an iterative radix-2 decimation-in-time FFT
for power-of-two lengths, a naive O(N^2) DFT (product with the DFT matrix)
for any length, and a direct O(N^4) 2-D DFT used as brute force on tiny grids.
"""

import numpy as np


def _bit_reverse_permutation(n):
    bits = n.bit_length() - 1
    idx = np.arange(n)
    rev = np.zeros(n, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    return rev


def dft_matrix(n, sign=-1):
    """The n x n DFT matrix W[k, m] = exp(sign * 2 pi i k m / n)."""
    k = np.arange(n)
    # reduce k*m modulo n before scaling so the angle stays small and exact
    km = np.mod(np.outer(k, k), n)
    return np.exp(sign * 2j * np.pi * km / n)


def dft_naive(x, axis=-1, sign=-1):
    """1-D DFT along ``axis`` by a product with the DFT matrix, O(N^2)."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    w = dft_matrix(x.shape[-1], sign)
    y = x @ w.T
    return np.moveaxis(y, -1, axis)


def fft_radix2(x, axis=-1, sign=-1):
    """1-D FFT along ``axis``: iterative radix-2 decimation in time.

    Input is put in bit-reversed order, then log2(N) butterfly stages combine
    pairs of half-length transforms: X[k] = E[k] + w^k O[k] and
    X[k+m] = E[k] - w^k O[k], with w = exp(sign * i pi / m).
    """
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    n = x.shape[-1]
    if n & (n - 1) or n == 0:
        raise ValueError("fft_radix2 needs a power-of-two length, got %d" % n)
    lead = x.shape[:-1]
    a = x[..., _bit_reverse_permutation(n)]
    m = 1
    while m < n:
        w = np.exp(sign * 1j * np.pi * np.arange(m) / m)
        a = a.reshape(lead + (n // (2 * m), 2, m))
        e = a[..., 0, :]
        o = a[..., 1, :] * w
        a = np.stack((e + o, e - o), axis=-2).reshape(lead + (n,))
        m *= 2
    return np.moveaxis(a, -1, axis)


def fft1(x, axis=-1, sign=-1):
    """1-D transform: radix-2 for powers of two, the naive DFT otherwise."""
    n = np.shape(x)[axis]
    if n > 0 and (n & (n - 1)) == 0:
        return fft_radix2(x, axis, sign)
    return dft_naive(x, axis, sign)


def fft2(x, sign=-1):
    """2-D transform over the last two axes ([..., y, x])."""
    return fft1(fft1(x, -1, sign), -2, sign)


def ifft2_unnormalised(x):
    """F^H over the last two axes (no 1/N^2 factor)."""
    return fft2(x, sign=+1)


def dft2_direct(x, sign=-1):
    """Brute-force 2-D DFT over the last two axes, O(N^4): every output
    frequency is an explicit double sum over every input pixel."""
    x = np.asarray(x, dtype=np.complex128)
    ny, nx = x.shape[-2:]
    ky = np.arange(ny)[:, None, None, None]
    kx = np.arange(nx)[None, :, None, None]
    yy = np.arange(ny)[None, None, :, None]
    xx = np.arange(nx)[None, None, None, :]
    phase = sign * 2j * np.pi * (np.mod(ky * yy, ny) / ny + np.mod(kx * xx, nx) / nx)
    kern = np.exp(phase)  # [ky, kx, y, x]
    return np.einsum("kqyx,...yx->...kq", kern, x)
