"""Pins of the dictionary PSF model's oracle (Sec. 2.2.2, "Spatially variant
convolution") against what the mathematics fixes: the real-space definition
of the spatially variant convolution, the spatially invariant special case,
flux conservation for unit-integral atoms and coefficients summing to one,
central differences of the loss, and a zero residual."""

import numpy as np

from oracle import dictionary as od


def _rand_case(seed, K=2, J=2, M=3, n=6):
    rng = np.random.default_rng(seed)
    obj = 1.0 + 0.3 * rng.standard_normal((K, n, n))
    coeff = rng.random((K, J, M, n, n))
    atoms = rng.random((M, n, n))
    atoms /= atoms.sum(axis=(1, 2), keepdims=True)
    spectra = rng.standard_normal((K, J, n, n)) + 1j * rng.standard_normal((K, J, n, n))
    gamma = 0.5 + rng.random((K, J))
    return obj, coeff, atoms, np.fft.fft2(atoms), spectra, gamma


def test_fourier_model_is_the_spatially_variant_convolution():
    obj, coeff, atoms, otf, _, _ = _rand_case(1)
    direct = od.model_image_direct(obj[0], coeff[0, 1], atoms)
    fourier = np.fft.ifft2(od.model_spectrum(obj[0], coeff[0, 1], otf))
    assert np.abs(fourier.imag).max() < 1e-12
    assert np.allclose(fourier.real, direct, rtol=0, atol=1e-12)


def test_point_source_images_its_own_psf():
    # a unit point at r' images to s(r', r - r') = sum_i a_i(r') phi_i(r - r')
    _, coeff, atoms, otf, _, _ = _rand_case(2, n=5)
    obj = np.zeros((5, 5))
    obj[3, 1] = 1.0
    img = np.fft.ifft2(od.model_spectrum(obj, coeff[0, 0], otf)).real
    psf = np.tensordot(coeff[0, 0][:, 3, 1], atoms, axes=1)
    assert np.allclose(img, np.roll(np.roll(psf, 3, axis=0), 1, axis=1), atol=1e-13)


def test_constant_coefficients_reduce_to_one_invariant_psf():
    obj, _, atoms, otf, _, _ = _rand_case(3)
    c = np.array([0.2, 0.5, 0.3])
    coeff = np.broadcast_to(c[:, None, None], (3, 6, 6))
    spec = od.model_spectrum(obj[1], coeff, otf)
    assert np.allclose(spec, np.fft.fft2(obj[1]) * np.tensordot(c, otf, axes=1), atol=1e-12)


def test_flux_is_conserved_for_unit_atoms_and_coefficients_summing_to_one():
    obj, coeff, atoms, otf, _, _ = _rand_case(4)
    a = coeff[0, 0] / coeff[0, 0].sum(axis=0, keepdims=True)
    img = np.fft.ifft2(od.model_spectrum(obj[0], a, otf)).real
    assert abs(img.sum() - obj[0].sum()) < 1e-11 * abs(obj[0].sum())


def test_zero_residual_gives_zero_loss_and_gradients():
    obj, coeff, atoms, otf, _, gamma = _rand_case(5)
    K, J = gamma.shape
    spectra = np.array([[od.model_spectrum(obj[k], coeff[k, j], otf) for j in range(J)] for k in range(K)])
    loss, go, ga = od.loss_grad(obj, coeff, otf, spectra, gamma)
    assert loss < 1e-20 and np.abs(go).max() < 1e-10 and np.abs(ga).max() < 1e-10


def test_gradients_match_central_differences():
    obj, coeff, atoms, otf, spectra, gamma = _rand_case(6, K=2, J=2, M=2, n=4)
    loss, go, ga = od.loss_grad(obj, coeff, otf, spectra, gamma)
    h = 1e-6
    rng = np.random.default_rng(0)
    for _ in range(6):
        idx = tuple(int(rng.integers(s)) for s in obj.shape)
        op, om = obj.copy(), obj.copy()
        op[idx] += h
        om[idx] -= h
        fd = (od.loss_grad(op, coeff, otf, spectra, gamma)[0] - od.loss_grad(om, coeff, otf, spectra, gamma)[0]) / (2 * h)
        assert abs(fd - go[idx]) <= 1e-6 * max(1.0, abs(go[idx])), (idx, fd, go[idx])
    for _ in range(6):
        idx = tuple(int(rng.integers(s)) for s in coeff.shape)
        cp, cm = coeff.copy(), coeff.copy()
        cp[idx] += h
        cm[idx] -= h
        fd = (od.loss_grad(obj, cp, otf, spectra, gamma)[0] - od.loss_grad(obj, cm, otf, spectra, gamma)[0]) / (2 * h)
        assert abs(fd - ga[idx]) <= 1e-6 * max(1.0, abs(ga[idx])), (idx, fd, ga[idx])


def test_loss_is_the_weighted_residual_energy():
    # one frame, one atom phi = delta (Phi = 1), a = 1: the model is F(o)
    rng = np.random.default_rng(7)
    obj = rng.standard_normal((1, 4, 4))
    spectra = rng.standard_normal((1, 1, 4, 4)) + 1j * rng.standard_normal((1, 1, 4, 4))
    loss, _, _ = od.loss_grad(obj, np.ones((1, 1, 1, 4, 4)), np.ones((1, 4, 4), complex), spectra, np.array([[2.5]]))
    assert abs(loss - 2.5 * np.sum(np.abs(spectra[0, 0] - np.fft.fft2(obj[0])) ** 2)) < 1e-10
