"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties the oracle to something other than itself: brute force,
closed forms, invariants stated in the paper (Sec. 3.1: the even-mode sign
ambiguity; Sec. 2.2.1: Eq. 12 does not depend on the object), published
tables (Noll 1976) and independent numerical routes (quadrature, central
differences). No GPU is used.
"""

import math
import os

import numpy as np
import pytest
from scipy import integrate, special

from oracle import dft, mfbd, optics
from paper_2505_10639_gb300 import synth
from tests import cases

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------- transforms

@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 64, 128])
def test_radix2_fft_matches_naive_dft_and_numpy(n):
    g = synth.rng(1, sub=n)
    x = g.standard_normal((3, n)) + 1j * g.standard_normal((3, n))
    ref = np.fft.fft(x)
    assert np.allclose(dft.fft_radix2(x), dft.dft_naive(x), atol=1e-12 * n)
    assert np.allclose(dft.fft_radix2(x), ref, atol=1e-12 * n)
    assert np.allclose(dft.fft_radix2(x, sign=+1), np.fft.ifft(x) * n, atol=1e-12 * n)


@pytest.mark.parametrize("n", [6, 12, 48])
def test_naive_dft_non_power_of_two(n):
    g = synth.rng(2, sub=n)
    x = g.standard_normal((2, n)) + 1j * g.standard_normal((2, n))
    assert np.allclose(dft.fft1(x), np.fft.fft(x), atol=1e-11 * n)


def test_direct_2d_dft_matches_fft2():
    g = synth.rng(3)
    x = g.standard_normal((2, 8, 8)) + 1j * g.standard_normal((2, 8, 8))
    assert np.allclose(dft.dft2_direct(x), dft.fft2(x), atol=1e-12)
    assert np.allclose(dft.dft2_direct(x, +1), dft.ifft2_unnormalised(x), atol=1e-12)


# ------------------------------------------------------- P1: brute force

def _brute_force_loss(masks, bases, scales, w, gamma, coeffs, d):
    """Eqs. 20-22 and 12 written with explicit O(N^4) DFTs and explicit
    frequency loops (tiny grids only)."""
    total = 0.0
    for k in range(len(masks)):
        n = masks[k].shape[0]
        hs = []
        for j in range(coeffs.shape[0]):
            phi = np.zeros((n, n))
            for m in range(coeffs.shape[1]):
                phi += scales[k] * coeffs[j, m] * bases[k][m]
            pup = np.where(masks[k], np.cos(phi) + 1j * np.sin(phi), 0)
            field = dft.dft2_direct(pup)
            inten = np.abs(field) ** 2
            hs.append(dft.dft2_direct(inten / inten.sum()))
        for ky in range(n):
            for kx in range(n):
                e = sum(w[k, j] * abs(d[k, j, ky, kx]) ** 2 for j in range(len(hs)))
                num = sum(w[k, j] * d[k, j, ky, kx] * np.conj(hs[j][ky, kx]) for j in range(len(hs)))
                den = sum(w[k, j] * abs(hs[j][ky, kx]) ** 2 for j in range(len(hs))) + gamma
                total += e - abs(num) ** 2 / den
    return total


def _tiny_case():
    # 8 x 8 grid, pupil diameter 4 px, 3 frames, 5 Zernike modes, 2 objects
    return cases.make_case(n_pix=8, diams=(4.0, 5.0), wavelengths=(5000.0, 6000.0),
                           n_frames=3, n_modes=5, seed=11, noise_sigma=1e-2,
                           weights=[[1.0, 0.5, 2.0], [0.7, 1.0, 1.3]])


def test_brute_force_loss_8x8():
    c = _tiny_case()
    s = c["setup"]
    a = c["a_eval"][0]
    ref = _brute_force_loss(s.masks, s.bases, s.scales, s.weights, s.gamma, a, c["d"][0])
    got = mfbd.loss_patch(s, a, c["d"][0])
    assert abs(got - ref) <= 1e-12 * abs(ref)


def test_brute_force_gradient_8x8():
    c = _tiny_case()
    s = c["setup"]
    a = c["a_eval"][0]
    _, _, g = mfbd.loss_object_grad_patch(s, a, c["d"][0])
    h = 1e-5
    fd = np.zeros_like(a)
    for j in range(a.shape[0]):
        for m in range(a.shape[1]):
            ap, am = a.copy(), a.copy()
            ap[j, m] += h
            am[j, m] -= h
            fd[j, m] = (_brute_force_loss(s.masks, s.bases, s.scales, s.weights, s.gamma, ap, c["d"][0])
                        - _brute_force_loss(s.masks, s.bases, s.scales, s.weights, s.gamma, am, c["d"][0])) / (2 * h)
    assert np.abs(g - fd).max() <= 1e-6 * np.abs(fd).max()


# --------------------------------------------------- P2/P3: normalisation

def test_parseval_and_psf_normalisation():
    c = cases.single_patch_64px()
    s = c["setup"]
    inter = mfbd.otf_patch(s, c["a_eval"][0])[0]
    n = c["n_pix"]
    npup = s.masks[0].sum()
    # sum_x |F P|^2 = N^2 sum_v |P|^2 = N^2 n_pup (phase-only pupil)
    assert np.allclose(inter["z"].ravel(), n * n * npup, rtol=1e-13)
    # sum_u |H|^2 = N^2 sum_x s^2
    lhs = (np.abs(inter["H"]) ** 2).sum(axis=(-2, -1))
    rhs = n * n * (inter["s"] ** 2).sum(axis=(-2, -1))
    assert np.allclose(lhs, rhs, rtol=1e-12)
    assert np.allclose(inter["H"][:, 0, 0], 1.0, atol=1e-14)
    assert (inter["s"] >= 0).all()


def test_aberration_free_psf_peak():
    n, dp = 64, 32.0
    mask = optics.pupil_mask(n, dp)
    _, _, _, s = mfbd.psf_from_pupil(mfbd.pupil_function(mask, np.zeros((n, n))))
    npup = mask.sum()
    assert abs(s[0, 0] - npup / n ** 2) <= 1e-15
    assert s[0, 0] == s.max()


# ------------------------------------------------------------- P4: Airy

def test_aberration_free_psf_is_airy():
    n, dp, over = 64, 32.0, 8
    mask = optics.pupil_mask(n, dp)
    big = np.zeros((n * over, n * over))
    big[:n, :n] = mask  # zero-padding samples the PSF every 1/over px
    field = dft.fft2(big)
    prof = np.abs(field[0, : 4 * over]) ** 2
    prof /= prof[0]
    r = np.arange(4 * over) / over
    arg = np.pi * dp * r / n
    airy = np.ones_like(arg)
    airy[1:] = (2 * special.j1(arg[1:]) / arg[1:]) ** 2
    core = r <= 2.0
    assert np.abs(prof[core] - airy[core]).max() < 0.02
    first_min = r[np.argmin(prof[: 3 * over + 1])]
    assert abs(first_min - 1.2197 * n / dp) <= 0.1


# --------------------------------------------------------- P5: tip-tilt

@pytest.mark.parametrize("shift", [1, 3, -2])
def test_tip_tilt_shifts_psf(shift):
    n, dp = 64, 32.0
    r = dp / 2
    basis = optics.zernike_basis(n, dp, [2, 3])
    mask = optics.pupil_mask(n, dp)
    _, _, _, s0 = mfbd.psf_from_pupil(mfbd.pupil_function(mask, np.zeros((n, n))))
    a2 = np.pi * r * shift / n  # Z2 = 2 rho cos(theta): phase ramp 2 pi shift x / N
    for mode, axis in ((0, 1), (1, 0)):  # Z2 shifts along x (columns), Z3 along y
        coef = np.zeros(2)
        coef[mode] = a2
        phi = mfbd.phase(basis, coef, 1.0)
        _, _, _, s = mfbd.psf_from_pupil(mfbd.pupil_function(mask, phi))
        assert np.abs(s - np.roll(s0, shift, axis=axis)).max() < 1e-14


# ----------------------------------------------------------- P6: piston

def test_piston_invariance():
    c = cases.single_patch_64px()
    s = c["setup"]
    a = c["a_eval"][0]
    piston = np.ones((1,) + s.bases[0].shape[1:]) * s.masks[0]
    s2 = mfbd.Setup(s.masks, [np.concatenate([s.bases[0], piston])], s.scales, s.weights, s.gamma)
    a0 = np.concatenate([a, np.zeros((a.shape[0], 1))], axis=1)
    a1 = np.concatenate([a, np.full((a.shape[0], 1), 0.731)], axis=1)
    l0, o0, g0 = mfbd.loss_object_grad_patch(s2, a0, c["d"][0])
    l1, o1, g1 = mfbd.loss_object_grad_patch(s2, a1, c["d"][0])
    # FP64 floor of Eq. 12: sum_u E ~ 1e8 cancels down to L ~ 1e4
    assert abs(l1 - l0) <= 1e-10 * l0
    assert np.abs(o1 - o0).max() <= 1e-10 * np.abs(o0).max()
    assert np.abs(g1 - g0).max() <= 1e-9 * np.abs(g0).max()
    assert np.abs(g0[:, -1]).max() <= 1e-8 * np.abs(g0).max()  # dL/d(piston) = 0


# ---------------------------------------------- phase diversity (Sec. 2.1)

def _diversity_case():
    return cases.make_case(n_pix=32, diams=(14.0, 11.0), wavelengths=(6563.0, 8542.0), n_frames=3,
                           n_modes=6, basis="zernike", seed=20250541)


def test_modal_diversity_equals_shifted_coefficients():
    """A diversity theta_kj = c_k B_k delta_j is the wavefront of delta_j:
    the loss, object and dL/da at a equal those at a + delta with no
    diversity (checks that theta is added, per object, unscaled)."""
    c = _diversity_case()
    s = c["setup"]
    a = c["a_eval"][0]
    delta = synth.kolmogorov_coeffs(7, np.ones(6), 5.0, (3,))
    theta = [mfbd.phase(s.bases[k], delta, s.scales[k]) for k in range(2)]
    sd = mfbd.Setup(s.masks, s.bases, s.scales, s.weights, s.gamma, diversity=theta)
    l1, o1, g1 = mfbd.loss_object_grad_patch(sd, a, c["d"][0])
    l0, o0, g0 = mfbd.loss_object_grad_patch(s, a + delta, c["d"][0])
    assert abs(l1 - l0) <= 1e-11 * abs(l0)
    assert np.abs(o1 - o0).max() <= 1e-10 * np.abs(o0).max()
    assert np.abs(g1 - g0).max() <= 1e-9 * np.abs(g0).max()
    # and it is not the same as no diversity, or as the diversity subtracted
    lm, _, _ = mfbd.loss_object_grad_patch(s, a - delta, c["d"][0])
    ln, _, _ = mfbd.loss_object_grad_patch(s, a, c["d"][0])
    assert abs(lm - l1) > 1e-3 * abs(l1) and abs(ln - l1) > 1e-3 * abs(l1)


def test_piston_diversity_changes_nothing():
    c = _diversity_case()
    s = c["setup"]
    a = c["a_eval"][0]
    theta = [np.full((3,) + s.masks[k].shape, 0.3 + 0.7 * k) for k in range(2)]
    sd = mfbd.Setup(s.masks, s.bases, s.scales, s.weights, s.gamma, diversity=theta)
    l1, o1, g1 = mfbd.loss_object_grad_patch(sd, a, c["d"][0])
    l0, o0, g0 = mfbd.loss_object_grad_patch(s, a, c["d"][0])
    assert abs(l1 - l0) <= 1e-11 * abs(l0)
    assert np.abs(o1 - o0).max() <= 1e-10 * np.abs(o0).max()
    assert np.abs(g1 - g0).max() <= 1e-9 * np.abs(g0).max()


# ---------------------------------------------- P7: even-mode sign flip

@pytest.mark.parametrize("basis", ["zernike", "kl"])
def test_even_mode_sign_flip(basis):
    """Sec. 3.1: the PSF is unchanged when all even modes change sign."""
    c = cases.make_case(n_frames=3, n_modes=14, basis=basis, seed=5)
    s = c["setup"]
    ms = optics.mode_parity_m(basis, 14)
    t = np.where(ms % 2 == 0, -1.0, 1.0)
    a = c["a_eval"][0]
    l0, o0, g0 = mfbd.loss_object_grad_patch(s, a, c["d"][0])
    l1, o1, g1 = mfbd.loss_object_grad_patch(s, a * t, c["d"][0])
    h0 = mfbd.otf_patch(s, a)[0]["s"]
    h1 = mfbd.otf_patch(s, a * t)[0]["s"]
    assert np.abs(h1 - h0).max() < 1e-15
    assert abs(l1 - l0) <= 1e-10 * l0  # FP64 floor of the Eq. 12 cancellation
    assert np.abs(g1 - g0 * t).max() <= 1e-9 * np.abs(g0).max()
    # a plain sign flip of all modes is NOT a symmetry (odd modes matter)
    l2 = mfbd.loss_patch(s, -a, c["d"][0])
    assert abs(l2 - l0) > 1e-3 * l0


# --------------------------------------- P8/P9: Wiener algebra (Eq. 11-12)

def test_loss_terms_nonnegative_and_lagrange_identity():
    c = cases.make_case(n_frames=4, seed=7, weights=[[1.0, 0.3, 2.0, 0.9]])
    s = c["setup"]
    h = mfbd.otf_patch(s, c["a_eval"][0])[0]["H"]
    d = c["d"][0, 0]
    w = s.weights[0]
    t = mfbd.loss_terms(d, h, w, s.gamma)
    num, den, ene = mfbd.wiener_sums(d, h, w, s.gamma)
    # E Q - |N|^2 = sum_{j<l} w_j w_l |D_j H_l - D_l H_j|^2 + gamma E
    lag = s.gamma * ene
    for j in range(4):
        for l in range(j + 1, 4):
            lag = lag + w[j] * w[l] * np.abs(d[j] * h[l] - d[l] * h[j]) ** 2
    assert np.allclose(t * den, lag, rtol=1e-8, atol=1e-8 * np.abs(lag).max())
    assert (t >= -1e-9 * ene).all()


def test_wiener_object_minimises_joint_loss():
    """Eq. 12 equals Eq. 8 (with R = gamma |O|^2) at O = Eq. 11, and any
    other object gives a larger value."""
    c = cases.make_case(n_frames=4, seed=8, weights=[[1.0, 0.3, 2.0, 0.9]])
    s = c["setup"]
    h = mfbd.otf_patch(s, c["a_eval"][0])[0]["H"]
    d = c["d"][0, 0]
    w = s.weights[0][:, None, None]

    def joint(o):
        return (w * np.abs(d - o[None] * h) ** 2).sum() + s.gamma * (np.abs(o) ** 2).sum()

    o = mfbd.wiener_object(d, h, s.weights[0], s.gamma)
    l12 = mfbd.loss_terms(d, h, s.weights[0], s.gamma).sum()
    assert abs(joint(o) - l12) <= 1e-9 * l12
    g = synth.rng(9)
    for _ in range(3):
        dlt = (g.standard_normal(o.shape) + 1j * g.standard_normal(o.shape)) * 1e-3 * np.abs(o).mean()
        assert joint(o + dlt) > joint(o)


# --------------------------------------------------- P10/P11: gamma -> 0

def test_single_frame_noiseless_loss_vanishes_linearly_in_gamma():
    c = cases.make_case(n_frames=1, noise_sigma=0.0, gamma=1.0, seed=12)
    s = c["setup"]
    a = c["a_true"][0]
    h = mfbd.otf_patch(s, a)[0]["H"][0]
    supp = optics.otf_support(s.masks[0])
    fo = dft.fft2(c["objects"][0, 0])
    target = (np.abs(fo[supp]) ** 2).sum()
    ratios = []
    for gam in (1e-4, 1e-6, 1e-8):
        s.gamma = gam
        ratios.append(mfbd.loss_patch(s, a, c["d"][0]) / gam)
    # L / gamma -> sum over the support of |O_true|^2 (weighted by
    # |H|^2/(|H|^2+gamma) -> 1)
    assert abs(ratios[-1] - target) <= 1e-3 * target
    assert abs(ratios[-1] - target) < abs(ratios[0] - target)


def test_true_coefficients_are_stationary_as_gamma_vanishes():
    c = cases.make_case(n_frames=4, noise_sigma=0.0, gamma=1.0, seed=13)
    s = c["setup"]
    vals = []
    for gam in (1e-6, 1e-7):
        s.gamma = gam
        l, _, g = mfbd.loss_object_grad_patch(s, c["a_true"][0], c["d"][0])
        vals.append((l, np.linalg.norm(g)))
    # both scale ~ linearly with gamma
    assert 5.0 < vals[0][0] / vals[1][0] < 20.0
    assert 5.0 < vals[0][1] / vals[1][1] < 20.0
    s.gamma = 1e-7
    _, _, g_off = mfbd.loss_object_grad_patch(s, c["a_eval"][0], c["d"][0])
    assert np.linalg.norm(g_off) > 1e3 * vals[1][1]


# ------------------------------------------ P12: gradient vs central FD

def _fd4(f, a, h=2e-4):
    """Fourth-order central differences. The step balances truncation
    (O(h^4)) against the FP64 cancellation floor of Eq. 12 (~1e-12 L)."""
    out = np.zeros_like(a)
    for idx in np.ndindex(a.shape):
        vals = []
        for step in (2, 1, -1, -2):
            x = a.copy()
            x[idx] += step * h
            vals.append(f(x))
        out[idx] = (-vals[0] + 8 * vals[1] - 8 * vals[2] + vals[3]) / (12 * h)
    return out


def test_gradient_central_differences_single_patch():
    c = cases.single_patch_64px()
    s = c["setup"]
    a = c["a_eval"][0]
    _, _, g = mfbd.loss_object_grad_patch(s, a, c["d"][0])
    fd = _fd4(lambda x: mfbd.loss_patch(s, x, c["d"][0]), a)
    assert np.abs(g - fd).max() <= 1e-6 * np.abs(g).max()
    assert np.linalg.norm(g - fd) <= 3e-7 * np.linalg.norm(g)


def test_gradient_central_differences_two_objects_weights():
    c = cases.make_case(n_pix=32, diams=(12.0, 15.0), wavelengths=(6563.0, 8542.0),
                        n_frames=3, n_modes=8, basis="kl", seed=14,
                        weights=[[1.0, 0.5, 1.5], [0.8, 1.2, 1.0]])
    s = c["setup"]
    a = c["a_eval"][0]
    _, _, g = mfbd.loss_object_grad_patch(s, a, c["d"][0])
    fd = _fd4(lambda x: mfbd.loss_patch(s, x, c["d"][0]), a)
    assert np.linalg.norm(g - fd) <= 3e-7 * np.linalg.norm(g)


# ------------------------------------------------- P13: F versus F^-1

def test_forward_and_inverse_psf_are_reflections():
    c = cases.single_patch_64px()
    s = c["setup"]
    phi = mfbd.phase(s.bases[0], c["a_eval"][0, 0], 1.0)
    pup = mfbd.pupil_function(s.masks[0], phi)
    _, _, _, sf = mfbd.psf_from_pupil(pup, sign=-1)
    _, _, _, si = mfbd.psf_from_pupil(pup, sign=+1)
    n = c["n_pix"]
    idx = (-np.arange(n)) % n
    assert np.abs(sf - si[np.ix_(idx, idx)]).max() < 1e-15


# ----------------------------------------- OTF support and its mask

def test_otf_vanishes_outside_exact_support_and_masking_is_exact():
    c = cases.make_case(diams=(28.0,), n_frames=4, seed=15, gamma=1e-9)
    s = c["setup"]
    h = mfbd.otf_patch(s, c["a_eval"][0])[0]["H"]
    supp = optics.otf_support(s.masks[0])
    assert np.abs(h[:, ~supp]).max() < 1e-15
    assert np.abs(h[:, supp]).min() >= 0
    # restricting the loss sum to the support and H to its mask changes it
    # only by the (pure-data) out-of-support energy term
    d = c["d"][0, 0]
    w = s.weights[0]
    t_full = mfbd.loss_terms(d, h, w, s.gamma)
    t_mask = mfbd.loss_terms(d, h * supp, w, s.gamma)
    assert np.abs(t_full - t_mask).sum() <= 1e-12 * t_full.sum()
    e_out = (np.abs(d[:, ~supp]) ** 2).sum()
    assert abs(t_full[~supp].sum() - e_out) <= 1e-6 * e_out


# ----------------------------------------------- Zernike / Noll / KL

def test_noll_indexing_and_low_order_closed_forms():
    assert [optics.noll_to_nm(j) for j in range(1, 12)] == [
        (0, 0), (1, 1), (1, 1), (2, 0), (2, 2), (2, 2), (3, 1), (3, 1), (3, 3), (3, 3), (4, 0)]
    g = synth.rng(16)
    rho = g.uniform(0, 1, 50)
    th = g.uniform(-np.pi, np.pi, 50)
    closed = {
        2: 2 * rho * np.cos(th), 3: 2 * rho * np.sin(th),
        4: math.sqrt(3) * (2 * rho ** 2 - 1),
        5: math.sqrt(6) * rho ** 2 * np.sin(2 * th), 6: math.sqrt(6) * rho ** 2 * np.cos(2 * th),
        7: math.sqrt(8) * (3 * rho ** 3 - 2 * rho) * np.sin(th),
        8: math.sqrt(8) * (3 * rho ** 3 - 2 * rho) * np.cos(th),
        11: math.sqrt(5) * (6 * rho ** 4 - 6 * rho ** 2 + 1),
    }
    for j, ref in closed.items():
        assert np.allclose(optics.zernike(j, rho, th), ref, atol=1e-13)


def test_zernike_orthonormal_in_the_continuum_limit():
    n = 1024
    b = optics.zernike_basis(n, n - 2.0, range(2, 12))
    mask = optics.pupil_mask(n, n - 2.0)
    v = b[:, mask]
    gram = v @ v.T / mask.sum()
    assert np.abs(gram - np.eye(10)).max() < 5e-3


def _noll_table():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "noll1976_table4.txt"))
            if l.strip() and not l.startswith("#")]
    return {int(a): float(b) for a, b in rows}


def _piston_removed_variance():
    """Delta_1 by quadrature of W(f) (1 - |2 J1(pi D f)/(pi D f)|^2) for
    D = r0 = 1 (an independent route to the covariance's scale)."""
    a = optics.kolmogorov_psd_constant()

    def f(x):
        arg = np.pi * x
        return a * x ** (-11.0 / 3.0) * (1 - (2 * special.j1(arg) / arg) ** 2) * 2 * np.pi * x

    edges = np.r_[1e-9, np.arange(0.5, 3000.5, 0.5)]
    body = sum(integrate.quad(f, lo, hi, limit=200)[0] for lo, hi in zip(edges[:-1], edges[1:]))
    # tail: 1 - (...)^2 -> 1, so int_X^inf a f^(-8/3) 2 pi df
    return body + a * 2 * np.pi * 3000.0 ** (-5.0 / 3.0) / (5.0 / 3.0)


def test_noll_covariance_closed_form_matches_quadrature():
    a = optics.kolmogorov_psd_constant()
    rr = 0.5  # D = 1

    def cov_quad(n, n2):
        def f(x):
            arg = 2 * np.pi * rr * x
            q = (special.jv(n + 1, arg) * special.jv(n2 + 1, arg)) / (np.pi * rr * x) ** 2
            return a * x ** (-11.0 / 3.0) * q * 2 * np.pi * x
        edges = np.r_[1e-9, np.arange(0.5, 400.5, 0.5)]
        v = sum(integrate.quad(f, lo, hi, limit=200)[0] for lo, hi in zip(edges[:-1], edges[1:]))
        return v * math.sqrt((n + 1) * (n2 + 1))

    cov = optics.noll_covariance([2, 4, 8, 11, 16, 22])
    # (j, j') = (2,2) n=1; (4,4) n=2; (2,8) n=1,3 m=1 cos; (4,11) n=2,4 m=0
    assert abs(cov[0, 0] - cov_quad(1, 1)) < 1e-9
    assert abs(cov[1, 1] - cov_quad(2, 2)) < 1e-9
    assert abs(cov[0, 2] - (-1) * cov_quad(1, 3)) < 1e-9
    assert abs(cov[1, 3] - (-1) * cov_quad(2, 4)) < 1e-9
    assert cov[0, 1] == 0.0 and cov[2, 3] == 0.0


def test_noll_covariance_against_noll_table():
    tab = _noll_table()
    d1 = _piston_removed_variance()
    var = np.diag(optics.noll_covariance(range(2, 22)))
    ours = d1 - np.cumsum(var)  # Delta_2 .. Delta_21
    for j in range(2, 22):
        # shape: residuals relative to Delta_1 agree to the table's rounding
        assert abs(ours[j - 2] / d1 - tab[j] / tab[1]) < 6e-4, j
    # scale: Noll's Delta_1 is 0.24 % below the exact Kolmogorov constant's
    assert abs(d1 / tab[1] - 1.0) < 5e-3


def test_kl_basis_diagonalises_covariance_and_is_orthonormal():
    coef, var, ms = optics.kl_modes(20)
    jmax = coef.shape[1] + 1
    cov = optics.noll_covariance(range(2, jmax + 1))
    proj = coef @ cov @ coef.T
    assert np.allclose(proj, np.diag(var), atol=1e-12)
    assert np.allclose(coef @ coef.T, np.eye(20), atol=1e-12)
    assert (np.diff(var) <= 1e-15).all()
    assert var.sum() <= np.trace(cov) + 1e-12
    b, _, _ = optics.kl_basis(64, 28.0, 20)
    mask = optics.pupil_mask(64, 28.0)
    v = b[:, mask]
    assert np.allclose(v @ v.T / mask.sum(), np.eye(20), atol=1e-12)
    # the first KL pair is the (Zernike) tip-tilt pair
    assert set(ms[:2]) == {1}


def test_kolmogorov_generator_variances():
    var = optics.mode_variances("zernike", 20)
    a = synth.kolmogorov_coeffs(20250515, var, 5.0, (10000,))
    target = var * 5.0 ** (5.0 / 3.0)
    sample = a.var(axis=0)
    # 10^4 draws: relative sampling std of a variance is sqrt(2/1e4) = 1.4 %
    assert np.all(np.abs(sample / target - 1.0) < 0.06)
    assert abs(sample.sum() / target.sum() - 1.0) < 0.03


# --------------------------------------------- spectrum layout helpers

def test_half_and_full_spectrum_roundtrip():
    g = synth.rng(17)
    img = g.standard_normal((2, 16, 16))
    full = dft.fft2(img)
    half = mfbd.half_spectrum(full)
    assert half.shape == (2, 16, 9)
    assert np.allclose(mfbd.full_from_half(half, 16), full, atol=1e-12)


# ---------------------------------------------- patches, apodisation, merge (Sec. 5.2)

def test_hanning_window_shape():
    from oracle import patches
    assert np.array_equal(patches.hanning_window(64, 0), np.ones(64))
    for n, b in ((64, 6), (48, 5), (128, 12)):
        w = patches.hanning_window(n, b)
        assert np.allclose(w, w[::-1], rtol=0, atol=1e-15)          # symmetric
        assert np.all(w[b:n - b] == 1.0) and np.all((w > 0) & (w <= 1))
        assert np.allclose(w[:b] + w[:b][::-1], 1.0, rtol=0, atol=1e-14)  # raised-cosine transition
        assert np.all(np.diff(w[:b]) > 0)


def test_patch_grid_of_the_961_patch_field():
    from oracle import patches
    g = patches.patch_grid(1024, 1024, 64, 32)
    assert len(g) == 31 * 31 and g[0] == (0, 0) and g[-1] == (960, 960) and g[1] == (0, 32)
    assert len(patches.patch_grid(4096, 4096, 128, 64)) == 63 * 63


def test_spectra_from_frames_is_the_fft_of_the_apodised_patch():
    from oracle import patches
    g = np.random.default_rng(3)
    frames = 1.0 + 0.1 * g.standard_normal((2, 3, 80, 112))
    d = patches.spectra_from_frames(frames, 48, 16, 5)
    grid = patches.patch_grid(80, 112, 48, 16)
    assert d.shape == (len(grid), 2, 3, 48, 48)
    w1 = patches.hanning_window(48, 5)
    win = np.outer(w1, w1)
    for p in (0, len(grid) - 1):
        y0, x0 = grid[p]
        tile = frames[1, 2, y0:y0 + 48, x0:x0 + 48]
        apod = (tile - tile.mean()) * win + tile.mean()
        assert np.allclose(d[p, 1, 2], np.fft.fft2(apod), rtol=0, atol=1e-10)
    flat = np.full((1, 1, 64, 64), 3.25)
    assert np.allclose(patches.apodize(flat[0, 0], 6), 3.25, rtol=0, atol=1e-14)  # a flat patch is unchanged


def test_merge_of_unprocessed_patches_is_the_image():
    """Patches cut from an image, taken to the Fourier domain and back
    (object_images), merge into the same image wherever a patch covers it
    (the weights form a partition of unity), and 0 elsewhere."""
    from oracle import patches
    g = np.random.default_rng(4)
    img = g.standard_normal((2, 100, 90))
    n, ov, b = 32, 16, 6
    grid = patches.patch_grid(100, 90, n, ov)
    tiles = np.array([[img[k, y0:y0 + n, x0:x0 + n] for k in range(2)] for y0, x0 in grid])
    back = patches.object_images(np.fft.fft2(tiles))
    assert np.allclose(back, tiles, rtol=0, atol=1e-12)
    m = patches.merge(back, 100, 90, ov, b)
    hmax = grid[-1][0] + n
    wmax = grid[-1][1] + n
    assert np.allclose(m[:, :hmax, :wmax], img[:, :hmax, :wmax], rtol=0, atol=1e-12)
    assert np.all(m[:, hmax:, :] == 0) and np.all(m[:, :, wmax:] == 0)


def test_tophat_cosine_filter():
    """1 at the zero frequency and below f_l, 0 beyond f_u, the cosine
    transition at its midpoint 1/2, even (a real object stays real), and
    monotone along an axis."""
    from oracle import patches
    n, d = 64, 32.0
    h = patches.tophat_cosine_filter(n, d, 0.7, 0.8)
    assert h[0, 0] == 1.0 and h[0, int(0.7 * d)] == 1.0 and h[0, int(0.8 * d) + 1] == 0.0
    k = np.fft.fftfreq(n) * n
    f = np.hypot(k[:, None], k[None, :]) / d
    assert np.all(h[f >= 0.8] == 0.0) and np.all(h[f <= 0.7] == 1.0)
    assert np.allclose(h, np.roll(np.flip(h, (0, 1)), 1, (0, 1)))  # h(-u) = h(u)
    assert np.all(np.diff(h[0, : n // 2]) <= 0)
    hm = patches.tophat_cosine_filter(64, 40.0, 0.5, 0.7)
    assert abs(hm[0, 24] - 0.5) < 1e-12  # f = 0.6, the midpoint
