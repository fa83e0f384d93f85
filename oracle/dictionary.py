"""The spatially variant PSF model on a dictionary (Sec. 2.2.2, "Spatially
variant convolution": the PSF expansion over a dictionary, the image as a sum
of convolutions, and the Fourier-domain log-posterior), in FP64 (test
infrastructure only: nothing in the library imports this module).

The PSF at object point r' is s(r', r) = sum_i a_i(r') phi_i(r); the image of
object k in frame j is i_kj = sum_i (o_k a_ikj) * phi_i (circular convolution
on the N x N patch), and the data term of the log-posterior is

  L = sum_k sum_j gamma_kj sum_u |I_kj(u) - sum_i F(o_k a_ikj)(u) Phi_i(u)|^2

with Phi_i = F(phi_i) and the sum over the full N x N frequency plane.

Gradients (real o, a; F unnormalised, F^H its adjoint, sum_u exp(+2 pi i u r / N)):

  g_ikj(r) = -2 gamma_kj Re F^H[conj(Phi_i) R_kj](r),  R_kj = I_kj - sum_i F(o_k a_ikj) Phi_i
  dL/da_ikj = o_k g_ikj,  dL/do_k = sum_j sum_i a_ikj g_ikj

Readings (the text leaves these open):
* The regulariser beta R(o, s) is left to the caller: L is the data term.
* gamma_kj weights frame j of object k (the loss's frame weights).
* The patch is periodic: the convolution is circular, as the Fourier form
  makes it.

Every function is pinned in tests/test_oracle_dictionary.py: the Fourier
model against a real-space sum over object points, the spatially invariant
case against a single PSF sum_i c_i phi_i, the gradients against central
differences, and a zero residual.
"""

import numpy as np


def model_image_direct(obj, coeff, atoms):
    """i(r) = sum_r' o(r') sum_i a_i(r') phi_i(r - r') by brute force
    (periodic), for small N: obj [N, N], coeff [M, N, N], atoms [M, N, N]."""
    n = obj.shape[0]
    out = np.zeros((n, n))
    for yp in range(n):
        for xp in range(n):
            psf = np.tensordot(coeff[:, yp, xp], atoms, axes=1)  # s(r', .) on the patch
            # the PSF of point r' centred on r': psf(r - r')
            out += obj[yp, xp] * np.roll(np.roll(psf, yp, axis=0), xp, axis=1)
    return out


def model_spectrum(obj, coeff, atom_otf):
    """sum_i F(o a_i) Phi_i: obj [N, N], coeff [M, N, N], atom_otf [M, N, N]."""
    return np.sum(np.fft.fft2(obj[None] * coeff) * atom_otf, axis=0)


def loss_grad(obj, coeff, atom_otf, spectra, gamma):
    """Data term and gradients for one patch.

    obj [K, N, N] real, coeff [K, J, M, N, N] real, atom_otf [M, N, N]
    complex (full plane), spectra [K, J, N, N] complex (full plane),
    gamma [K, J]. Returns (L, dL/do [K, N, N], dL/da [K, J, M, N, N])."""
    obj = np.asarray(obj, np.float64)
    coeff = np.asarray(coeff, np.float64)
    K, J, M, n, _ = coeff.shape
    loss = 0.0
    g_obj = np.zeros((K, n, n))
    g_coeff = np.zeros_like(coeff)
    for k in range(K):
        for j in range(J):
            r = spectra[k, j] - model_spectrum(obj[k], coeff[k, j], atom_otf)
            loss += gamma[k, j] * np.sum(np.abs(r) ** 2)
            g = -2.0 * gamma[k, j] * np.real(np.fft.ifft2(np.conj(atom_otf) * r[None]) * (n * n))
            g_coeff[k, j] = obj[k][None] * g
            g_obj[k] += np.sum(coeff[k, j] * g, axis=0)
    return loss, g_obj, g_coeff
