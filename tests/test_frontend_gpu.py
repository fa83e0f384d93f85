"""GPU parity of the field front and back end (Sec. 5.2): the plan's spectra
from frames (patches, mean-subtracted modified-Hanning apodisation, DFT) and
the mosaic of patch objects, against the FP64 oracle (`oracle.patches`), and
a small field taken from frames through the loss, object and dL/da to the
mosaic.

Tolerances: spectra and mosaics 1e-5 relative (max-norm); loss, dL/da and
object as the FP32 path elsewhere (1e-5, 1e-4, 1e-4).
"""

import numpy as np
import pytest
import torch

from oracle import mfbd as omfbd
from oracle import optics
from oracle import patches as opatches
from paper_2505_10639_gb300 import synth

pytestmark = pytest.mark.gpu


def _plan(n, n_patches, diams, n_frames, n_modes=8, gamma=1e-3, basis="zernike"):
    from paper_2505_10639_gb300.mfbd import Plan
    wl = [6563.0 * diams[0] / d for d in diams]
    return Plan(n, n_patches, list(diams), wl, n_frames, n_modes, basis=basis, gamma=gamma)


@pytest.mark.parametrize("n,h,w,overlap,border", [(64, 160, 224, 32, 6), (48, 120, 100, 16, 5),
                                                  (96, 192, 160, 32, 8), (128, 128, 256, 64, 0),
                                                  (64, 164, 230, 30, 6), (64, 130, 222, 32, 6)])
def test_spectra_from_frames(n, h, w, overlap, border):
    """64 px patches at a stride and width that are multiples of 4 columns
    take the TMA-staged kernel; stride 34 (overlap 30) and a 222 px wide
    frame take the plain one; every call reports no failed wait."""
    g = np.random.default_rng(n + w)
    frames = (1.0 + 0.1 * g.standard_normal((2, 3, h, w))).astype(np.float32)
    grid = opatches.patch_grid(h, w, n, overlap)
    plan = _plan(n, len(grid), (0.4 * n, 0.3 * n), 3)
    d = plan.spectra_from_frames(torch.from_numpy(frames).cuda(), overlap, border).cpu().numpy()
    plan.check()
    ref = opatches.spectra_from_frames(frames.astype(np.float64), n, overlap, border)
    refh = omfbd.half_spectrum(ref)
    err = np.abs(d - refh).max() / np.abs(refh).max()
    assert err <= 1e-5, err


@pytest.mark.parametrize("n,h,w,overlap,border", [(64, 160, 224, 32, 6), (48, 120, 100, 16, 5),
                                                  (128, 200, 256, 64, 12)])
def test_merge_objects(n, h, w, overlap, border):
    g = np.random.default_rng(100 + n)
    grid = opatches.patch_grid(h, w, n, overlap)
    imgs = g.standard_normal((len(grid), 2, n, n))
    half = np.fft.rfft2(imgs).astype(np.complex64)  # Hermitian half spectra of real patch images
    plan = _plan(n, len(grid), (0.4 * n, 0.3 * n), 2)
    m = plan.merge_objects(torch.from_numpy(half).cuda(), h, w, overlap, border).cpu().numpy()
    full = omfbd.full_from_half(half.astype(np.complex128), n)
    ref = opatches.merge(opatches.object_images(full), h, w, overlap, border)
    err = np.abs(m - ref).max() / np.abs(ref).max()
    assert err <= 1e-5, err
    bad = plan.merge_objects
    with pytest.raises(Exception):
        bad(torch.from_numpy(half).cuda(), h + n, w, overlap, border)  # another patch count


def test_field_from_frames_to_mosaic():
    """A 96 x 96 field of 64 px patches at overlap 32 (2 x 2 patches), two
    objects, four frames: spectra from frames, loss, dL/da and the Wiener
    objects against the oracle on the oracle's own spectra, then the mosaic
    of the objects."""
    n, h, w, ov, bd = 64, 96, 96, 32, 6
    seed = 20250560
    field = synth.object_field(seed, (2, h, w))
    frames = (field[:, None] + synth.noise(seed, (2, 4, h, w), 1e-2)).astype(np.float32)
    grid = opatches.patch_grid(h, w, n, ov)
    diams = (26.0, 20.0)
    plan = _plan(n, len(grid), diams, 4, n_modes=10, gamma=4e-6)
    var = optics.mode_variances("zernike", 10)
    a32 = synth.kolmogorov_coeffs(seed, var, 5.0, (len(grid), 4)).astype(np.float32)
    d_gpu = plan.spectra_from_frames(torch.from_numpy(frames).cuda(), ov, bd)
    loss, grad, obj = plan.loss_grad(torch.from_numpy(a32).cuda(), d_gpu, want_object=True)
    mosaic = plan.merge_objects(obj, h, w, ov, bd).cpu().numpy()
    loss, grad, obj = loss.cpu().numpy(), grad.cpu().numpy(), obj.cpu().numpy()
    d_or = opatches.spectra_from_frames(frames.astype(np.float64), n, ov, bd)
    masks = [optics.pupil_mask(n, d) for d in diams]
    bases = [optics.zernike_basis(n, d, range(2, 12)) for d in diams]
    setup = omfbd.Setup(masks, bases, [1.0, diams[1] / diams[0]], np.ones((2, 4)), 4e-6)
    lo, oo, go = omfbd.loss_object_grad(setup, a32.astype(np.float64), d_or)
    for p in range(len(grid)):
        assert abs(loss[p] - lo[p]) <= 1e-5 * abs(lo[p]), (p, loss[p], lo[p])
        assert np.linalg.norm(grad[p] - go[p]) <= 1e-4 * np.linalg.norm(go[p]), p
        for k in range(2):
            supp = optics.otf_support(masks[k])
            of = omfbd.full_from_half(obj[p, k].astype(np.complex128), n)
            assert np.linalg.norm((of - oo[p][k])[supp]) <= 1e-4 * np.linalg.norm(oo[p][k][supp]), (p, k)
    ref = opatches.merge(opatches.object_images(oo), h, w, ov, bd)
    err = np.abs(mosaic - ref).max() / np.abs(ref).max()
    assert err <= 1e-4, err


@pytest.mark.parametrize("n,full", [(64, False), (64, True), (96, False)])
def test_filter_objects(n, full):
    """The top-hat / cosine Fourier filter of the objects in place, against
    the oracle's filter, per object with its own pupil and cutoffs."""
    from paper_2505_10639_gb300.mfbd import Plan
    g = np.random.default_rng(n + full)
    diams = (0.5 * n, 0.4 * n)
    plan = Plan(n, 3, list(diams), [6563.0, 6563.0 * diams[0] / diams[1]], 2, 6, basis="zernike", gamma=1e-3,
                full_spectrum=full)
    cols = n if full else n // 2 + 1
    o = (g.standard_normal((3, 2, n, cols)) + 1j * g.standard_normal((3, 2, n, cols))).astype(np.complex64)
    t = torch.from_numpy(o).cuda()
    plan.filter_objects(t, [0.7, 0.6], [0.8, 0.75])
    got = t.cpu().numpy()
    for k, (d, lo, hi) in enumerate(zip(diams, (0.7, 0.6), (0.8, 0.75))):
        h = opatches.tophat_cosine_filter(n, d, lo, hi)[:, :cols]
        assert np.abs(got[:, k] - o[:, k] * h[None]).max() <= 1e-6 * np.abs(o).max()
