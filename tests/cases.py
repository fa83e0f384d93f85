"""Seeded test cases built with the FP64 oracle (inputs from ``synth``).

A case holds the per-object plan data (pupil masks, sampled bases, phase
scales, weights, gamma), the true coefficients used to synthesise the data,
the data spectra D and an evaluation point a_eval = a_true + 0.3 * delta,
with delta an independent Kolmogorov draw (the optimiser's trajectory passes
through such points; at a_true the gradient is noise-dominated).

Workload readings: image-domain noise sigma = 1e-3 * mean(o) = 1e-3 and the
Wiener constant gamma = 1e-3 * N^2 sigma^2 (the per-frequency noise variance
of D, scaled by 1e-3).
"""

import numpy as np

from oracle import mfbd, optics
from paper_2505_10639_gb300 import synth

SEED_C1 = 20250516  # seed of the single-patch 64 px workload


def make_setup(n_pix, diams, wavelengths, n_frames, n_modes, basis="zernike",
               obscuration=0.0, weights=None, gamma=None, noise_sigma=1e-3):
    masks, bases = [], []
    for d in diams:
        masks.append(optics.pupil_mask(n_pix, d, obscuration))
        if basis == "zernike":
            bases.append(optics.zernike_basis(n_pix, d, range(2, n_modes + 2), obscuration))
        else:
            bases.append(optics.kl_basis(n_pix, d, n_modes, obscuration)[0])
    scales = np.array([wavelengths[0] / wl for wl in wavelengths])
    k = len(diams)
    w = np.ones((k, n_frames)) if weights is None else np.asarray(weights, np.float64)
    if gamma is None:
        gamma = 1e-3 * n_pix * n_pix * noise_sigma ** 2
    return mfbd.Setup(masks, bases, scales, w, gamma)


def make_case(n_pix=64, diams=(32.0,), wavelengths=(8542.0,), n_frames=8,
              n_modes=20, basis="zernike", n_patches=1, d_over_r0=5.0,
              seed=SEED_C1, noise_sigma=1e-3, gamma=None, weights=None,
              obscuration=0.0, perturb=0.3):
    setup = make_setup(n_pix, diams, wavelengths, n_frames, n_modes, basis,
                       obscuration, weights, gamma, noise_sigma)
    var = optics.mode_variances(basis, n_modes)
    k = len(diams)
    a_true = synth.kolmogorov_coeffs(seed, var, d_over_r0, (n_patches, n_frames))
    delta = synth.kolmogorov_coeffs(seed, var, d_over_r0, (n_patches, n_frames), sub=1)
    a_eval = a_true + perturb * delta
    objs = synth.object_field(seed, (n_patches, k, n_pix, n_pix))
    noise = synth.noise(seed, (n_patches, k, n_frames, n_pix, n_pix), noise_sigma)
    d = np.array([mfbd.synth_spectra(setup, a_true[p], objs[p], noise[p])
                  for p in range(n_patches)])
    return dict(setup=setup, a_true=a_true, a_eval=a_eval, d=d, objects=objs,
                n_pix=n_pix, diams=tuple(diams), wavelengths=tuple(wavelengths),
                n_frames=n_frames, n_modes=n_modes, basis=basis,
                obscuration=obscuration, variances=var)


def single_patch_64px():
    """1 patch, 64 px, 1 object, 8 frames, 32 px pupil, Zernike Noll 2-21,
    D/r0 = 5."""
    return make_case()
