"""Division of frames into apodised patches and merging of patch objects
into a mosaic (Sec. 5.2 of the paper, "Division in patches and
apodization"), in FP64 (test infrastructure only).

Readings (the paper describes these steps in words only):
* Patch grid: patches of n x n px at stride n - overlap, as many as fit
  entirely in the frame, starting at the frame's first row and column
  (a 1024 px frame, 64 px patches, overlap 32: 31 x 31 patches).
* Modified Hanning window: 1 inside, a raised-cosine transition over
  `border` px at each edge, evaluated at pixel centres:
  w[x] = (1 - cos(pi (x + 1/2) / border)) / 2 for x < border, mirrored at
  the other edge (border = 0: all ones). The 2-D window is w[y] w[x].
* Apodisation: the patch mean is subtracted, the window applied and the
  mean added back.
* Data spectra: the unnormalised forward DFT of the apodised patch.
* Merge: each patch object goes back to the image domain by the inverse DFT
  (normalised by 1/n^2) and the mosaic is the weighted average of the
  patches covering a pixel, with the same raised-cosine window (its own
  border) as the weight; pixels no patch covers are 0.
"""

import numpy as np

from . import dft


def hanning_window(n, border):
    """The 1-D modified Hanning window of length n."""
    w = np.ones(n)
    b = int(border)
    for x in range(min(b, n)):
        v = 0.5 * (1.0 - np.cos(np.pi * (x + 0.5) / b))
        w[x] = min(w[x], v)
        w[n - 1 - x] = min(w[n - 1 - x], v)
    return w


def patch_grid(height, width, n, overlap):
    """Origins (y0, x0) of the patches, row by row."""
    s = n - overlap
    ny = (height - n) // s + 1
    nx = (width - n) // s + 1
    return [(iy * s, ix * s) for iy in range(ny) for ix in range(nx)]


def apodize(tile, border):
    """(tile - mean) * window + mean."""
    n = tile.shape[-1]
    w1 = hanning_window(n, border)
    win = np.outer(w1, w1)
    m = tile.mean()
    return (tile - m) * win + m


def spectra_from_frames(frames, n, overlap, border):
    """frames [K, J, H, W] -> D [P, K, J, n, n] (full spectra)."""
    frames = np.asarray(frames, np.float64)
    K, J, H, W = frames.shape
    out = []
    for y0, x0 in patch_grid(H, W, n, overlap):
        dk = np.zeros((K, J, n, n), np.complex128)
        for k in range(K):
            for j in range(J):
                dk[k, j] = dft.fft2(apodize(frames[k, j, y0:y0 + n, x0:x0 + n], border))
        out.append(dk)
    return np.array(out)


def object_images(objects):
    """Patch objects [P, K, n, n] (full spectra) -> real images, the inverse
    DFT normalised by 1/n^2."""
    n = objects.shape[-1]
    return (dft.ifft2_unnormalised(np.asarray(objects, np.complex128)) / (n * n)).real


def merge(images, height, width, overlap, border):
    """Patch images [P, K, n, n] -> mosaic [K, H, W]: the weighted average of
    the patches covering each pixel."""
    images = np.asarray(images, np.float64)
    P, K, n, _ = images.shape
    w1 = hanning_window(n, border)
    win = np.outer(w1, w1)
    num = np.zeros((K, height, width))
    den = np.zeros((height, width))
    for p, (y0, x0) in enumerate(patch_grid(height, width, n, overlap)):
        num[:, y0:y0 + n, x0:x0 + n] += win[None] * images[p]
        den[y0:y0 + n, x0:x0 + n] += win
    out = np.zeros_like(num)
    covered = den > 0
    out[:, covered] = num[:, covered] / den[covered]
    return out


def tophat_cosine_filter(n, diam_px, f_lower, f_upper):
    """The low-pass filter of the object (Sec. 4.1.1, "Fourier filtering"),
    on the full n x n frequency grid [ky, kx]: 1 below f_lower, 0 above
    f_upper, (1 + cos(pi (f - f_lower) / (f_upper - f_lower))) / 2 between,
    f = |u| / D_p the frequency in units of the diffraction limit (the OTF of
    a D_p px pupil reaches |u| = D_p frequency bins)."""
    k = np.fft.fftfreq(n) * n  # signed frequency index
    f = np.hypot(k[:, None], k[None, :]) / float(diam_px)
    h = np.where(f <= f_lower, 1.0, 0.0)
    mid = (f > f_lower) & (f < f_upper)
    h[mid] = 0.5 * (1.0 + np.cos(np.pi * (f[mid] - f_lower) / (f_upper - f_lower)))
    return h
