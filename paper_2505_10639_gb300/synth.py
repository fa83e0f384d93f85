"""Seeded synthetic inputs for the MOMFBD hot path.

This module only draws random numbers and shapes them into the statistical
structure of the paper's workloads (solar granulation-like objects,
Kolmogorov wavefront coefficients, detector noise). It contains none of the
method's arithmetic (no pupil, PSF, OTF, Wiener filter or loss), so both the
CUDA path and the FP64 oracle may use it as their common source of inputs.

All draws use numpy's Philox4x32-10 counter-based generator, keyed by an
integer seed and a stream tag, so every array is reproducible on any host.

Input recipe (the paper's data are not available, Sec. 6):
* object: positive Gaussian random field with a k^-3 power spectrum, mean 1
  and rms contrast 10 %: white complex noise times |k|^(-3/2) (k != 0), real
  part of the inverse DFT, rescaled to the target mean and contrast, clamped
  at 1e-3;
* wavefront coefficients: independent N(0, var_m (D/r0)^(5/3)) per mode, with
  the per-mode Kolmogorov variances var_m supplied by the caller;
* noise: white Gaussian, sigma = 1e-3 times the object mean, image domain.
"""

import numpy as np

_STREAMS = {"object": 1, "coeff": 2, "noise": 3, "misc": 4}


def rng(seed, stream="misc", sub=0):
    """Philox generator for (seed, stream, sub) -- independent streams."""
    key = (int(seed) & 0xFFFFFFFFFFFFFFFF)
    ctr = [_STREAMS.get(stream, 0), int(sub), 0, 0]
    return np.random.Generator(np.random.Philox(key=key, counter=ctr))


def object_field(seed, shape, mean=1.0, contrast=0.1, slope=-3.0, sub=0):
    """Real field(s) of shape [..., ny, nx] with power spectrum |k|^slope."""
    g = rng(seed, "object", sub)
    ny, nx = shape[-2:]
    white = g.standard_normal(shape) + 1j * g.standard_normal(shape)
    ky = np.fft.fftfreq(ny)[:, None]
    kx = np.fft.fftfreq(nx)[None, :]
    k = np.hypot(ky, kx)
    amp = np.zeros_like(k)
    amp[k > 0] = k[k > 0] ** (slope / 2.0)
    field = np.fft.ifft2(white * amp).real
    field -= field.mean(axis=(-2, -1), keepdims=True)
    field /= field.std(axis=(-2, -1), keepdims=True)
    field = mean * (1.0 + contrast * field)
    return np.maximum(field, 1e-3 * mean)


def patches_from_field(field, n_pix, stride):
    """Cut [..., H, W] into overlapping [..., n_py * n_px, n_pix, n_pix]."""
    h, w = field.shape[-2:]
    ny = (h - n_pix) // stride + 1
    nx = (w - n_pix) // stride + 1
    out = []
    for iy in range(ny):
        for ix in range(nx):
            out.append(field[..., iy * stride: iy * stride + n_pix,
                             ix * stride: ix * stride + n_pix])
    return np.stack(out, axis=-3)


def kolmogorov_coeffs(seed, variances, d_over_r0, shape, sub=0):
    """Coefficients [..., M] ~ N(0, variances * (D/r0)^(5/3)), rad at lambda_0.

    ``variances`` are per-mode variances in units of (D/r0)^(5/3)."""
    var = np.asarray(variances, np.float64)
    g = rng(seed, "coeff", sub)
    z = g.standard_normal(tuple(shape) + (var.size,))
    return z * np.sqrt(var * d_over_r0 ** (5.0 / 3.0))


def noise(seed, shape, sigma, sub=0):
    """White Gaussian image-domain noise with standard deviation sigma."""
    return rng(seed, "noise", sub).standard_normal(shape) * sigma


def uniform(seed, shape, lo=0.0, hi=1.0, sub=0):
    return rng(seed, "misc", sub).uniform(lo, hi, shape)


def noise_torch(seed, shape, sigma, sub=0, device="cuda"):
    """White Gaussian noise drawn on `device` by torch's seeded generator
    (for fields too large to draw on the host), keyed by (seed, sub)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed((int(seed) * 1000003 + 7919 * int(sub) + _STREAMS["noise"]) & 0x7FFFFFFFFFFFFFFF)
    return torch.randn(shape, generator=g, device=device, dtype=torch.float64) * sigma


def uneven_problems(seed, n, sizes=(48, 64, 96, 128), objects=(1, 3), frames=(8, 24), modes=(20, 66),
                    pupil_frac=(0.35, 0.5), wavelength0=6563.0):
    """Sizes of an uneven batch of n problems (one patch each), drawn
    uniformly: patch size from `sizes`, objects, frames and modes from the
    inclusive ranges; each object's pupil diameter 2 round(U(pupil_frac) N / 2)
    px and its wavelength wavelength0 * D_0 / D_k (pupil diameter in pixels
    inversely proportional to the wavelength)."""
    g = rng(seed, "misc", 7)
    out = []
    for _ in range(n):
        npx = int(sizes[g.integers(0, len(sizes))])
        k = int(g.integers(objects[0], objects[1] + 1))
        j = int(g.integers(frames[0], frames[1] + 1))
        m = int(g.integers(modes[0], modes[1] + 1))
        diams = [float(2 * round(g.uniform(*pupil_frac) * npx / 2)) for _ in range(k)]
        wls = [wavelength0 * diams[0] / d for d in diams]
        out.append(dict(n_pix=npx, n_objects=k, n_frames=j, n_modes=m, diams=diams, wavelengths=wls))
    return out


def dictionary_case(seed, n_patches, n_objects, n_frames, n_atoms, n=64):
    """Inputs of the spatially variant dictionary model (Sec. 2.2.2).

    Recipe (the paper's NMF dictionary, learned from simulated PSFs, is not
    available): atoms phi_i are periodic elliptical Gaussians centred near the
    origin, widths 0.8-4 px, normalised to unit sum (non-negative, unit
    integral, as the expansion requires); coefficient maps a_ikj(r') are
    uniform draws in [0.1, 1.1) normalised so that sum_i a_i = 1 at every
    point; objects are k^-3 granulation-like fields (object_field); the data
    are half spectra of further k^-3 fields (the loss is defined for any
    data), made exactly Hermitian in the columns 0 and n/2; gamma = 1 / J.

    Returns float32 / complex64 arrays: atoms [M, n, n], atom_otf [M, n,
    n/2+1], gamma [K, J], obj [P, K, n, n], coeff [P, K, J, M, n, n],
    spectra [P, K, J, n, n/2+1]."""
    g = rng(seed, "misc", 77)
    atoms = np.empty((n_atoms, n, n))
    for i in range(n_atoms):
        sy, sx = g.uniform(0.8, 4.0, size=2)
        cy, cx = g.uniform(-1.5, 1.5, size=2)
        dy = np.minimum(np.abs(np.arange(n) - cy), n - np.abs(np.arange(n) - cy))
        dx = np.minimum(np.abs(np.arange(n) - cx), n - np.abs(np.arange(n) - cx))
        atoms[i] = np.exp(-0.5 * (dy[:, None] / sy) ** 2 - 0.5 * (dx[None, :] / sx) ** 2)
        atoms[i] /= atoms[i].sum()
    coeff = g.uniform(0.1, 1.1, size=(n_patches, n_objects, n_frames, n_atoms, n, n))
    coeff /= coeff.sum(axis=3, keepdims=True)
    obj = object_field(seed, (n_patches, n_objects, n, n), sub=7)
    data = object_field(seed, (n_patches, n_objects, n_frames, n, n), sub=8)

    def half(x):
        h = np.fft.rfft2(x).astype(np.complex64)
        for c in (0, n // 2):  # exactly Hermitian along ky
            col = h[..., :, c].astype(np.complex128)
            mirror = np.conj(np.roll(col[..., ::-1], 1, axis=-1))
            h[..., :, c] = (0.5 * (col + mirror)).astype(np.complex64)
        return h

    gamma = np.full((n_objects, n_frames), 1.0 / n_frames, np.float32)
    return (atoms.astype(np.float32), half(atoms), gamma, obj.astype(np.float32), coeff.astype(np.float32),
            half(data))
