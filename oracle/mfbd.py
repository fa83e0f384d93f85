"""The MOMFBD forward model, loss, Wiener object and gradient in FP64
(test infrastructure only).

Notation: k = object, j = frame (frames and diversity channels folded
together, Sec. 2.1), u = frequency, x = image pixel, v = pupil pixel,
m = mode. Spectra are full N x N complex arrays in the forward-FFT
convention of ``oracle.dft`` (index [ky][kx], unnormalised).

Per object k and frame j (Sec. 3.1):
  phi_kj(v) = c_k sum_m a_jm B_km(v) [+ theta_kj(v)]      (Eq. 22; theta: the known
                                                           diversity phase, Sec. 2.1)
  P_kj      = A_k exp(i phi_kj)                           (Eq. 20)
  s_kj      = |F P_kj|^2 / sum_x |F P_kj|^2               (Eq. 21, normalised)
  H_kj      = F s_kj
Per object k (Sec. 2.2.1), with weights w_kj (Eq. 2's gamma_kj) and the
Wiener constant gamma (S_n / S_0 = C):
  O_k  = sum_j w D conj(H) / (sum_j w |H|^2 + gamma)      (Eq. 11)
  L    = sum_k sum_u [ sum_j w |D|^2
                       - |sum_j w D conj(H)|^2 / (sum_j w |H|^2 + gamma) ]   (Eq. 12)

Readings (the paper leaves them open):
* The PSF uses the forward FFT of the pupil. Eq. 21 writes the inverse
  transform; the two PSFs are reflections of one another (tested), so the
  choice only fixes the sign convention, and the synthetic data use the same
  one.
* c_k = lambda_0 / lambda_k: coefficients are phases in radians at the
  wavelength of object 0 (Eq. 22 divides by lambda_k).
* The gradient is dL/da computed by the chain rule through Eqs. 20-22 and 12,
  where O is held at its optimum (the derivative of Eq. 12 with respect to
  O vanishes there). No support mask, no H(0) override and no G(0) zeroing is
  applied here: this is the plain definition.
"""

import numpy as np

from . import dft


def phase(basis, coeffs, scale):
    """phi[..., y, x] = scale * sum_m coeffs[..., m] basis[m, y, x] (Eq. 22)."""
    return scale * np.tensordot(np.asarray(coeffs, np.float64), basis, axes=(-1, 0))


def pupil_function(mask, phi):
    """P = A exp(i phi) (Eq. 20)."""
    return np.where(mask, np.exp(1j * phi), 0.0)


def psf_from_pupil(pupil, sign=-1):
    """Field p = F P, intensity q = |p|^2, PSF s = q / sum q (Eq. 21).

    Returns (p, q, z, s) with z = sum_x q the normalisation per frame."""
    p = dft.fft2(pupil, sign=sign)
    q = (p * p.conj()).real
    z = q.sum(axis=(-2, -1), keepdims=True)
    return p, q, z, q / z


def otf(psf):
    """H = F s."""
    return dft.fft2(psf)


def wiener_sums(d, h, w, gamma):
    """N = sum_j w D conj(H), Q = sum_j w |H|^2 + gamma, E = sum_j w |D|^2.

    d, h: [J, N, N] complex; w: [J]."""
    w = np.asarray(w, np.float64)[:, None, None]
    num = (w * d * h.conj()).sum(axis=0)
    den = (w * (h * h.conj()).real).sum(axis=0) + gamma
    ene = (w * (d * d.conj()).real).sum(axis=0)
    return num, den, ene


def wiener_object(d, h, w, gamma):
    """O = N / Q (Eq. 11)."""
    num, den, _ = wiener_sums(d, h, w, gamma)
    return num / den


def loss_terms(d, h, w, gamma):
    """t(u) = E - |N|^2 / Q per frequency (the summand of Eq. 12)."""
    num, den, ene = wiener_sums(d, h, w, gamma)
    return ene - (num * num.conj()).real / den


class Setup:
    """Per-object plan data: masks, sampled bases, phase scales, weights, and
    optionally the known diversity phases theta [K][J, N, N] (radians) added
    to the wavefront of object k in frame j (phase diversity, Sec. 2.1)."""

    def __init__(self, masks, bases, scales, weights, gamma, diversity=None):
        self.masks = [np.asarray(m, bool) for m in masks]
        self.bases = [np.asarray(b, np.float64) for b in bases]
        self.scales = np.asarray(scales, np.float64)
        self.weights = np.asarray(weights, np.float64)  # [K, J]
        self.gamma = float(gamma)
        self.diversity = None if diversity is None else [np.asarray(t, np.float64) for t in diversity]

    @property
    def n_objects(self):
        return len(self.masks)


def otf_patch(setup, coeffs):
    """H[k, j] for one patch, coeffs [J, M]. Also returns the intermediates
    (P, p, z, s) per object for the gradient."""
    out = []
    for k in range(setup.n_objects):
        phi = phase(setup.bases[k], coeffs, setup.scales[k])
        if setup.diversity is not None:
            phi = phi + setup.diversity[k]  # phi_kj = c_k B_k a_j + theta_kj
        pup = pupil_function(setup.masks[k], phi)
        p, q, z, s = psf_from_pupil(pup)
        out.append(dict(P=pup, p=p, z=z, s=s, H=otf(s)))
    return out


def loss_patch(setup, coeffs, d):
    """Loss (Eq. 12) of one patch: coeffs [J, M], d [K, J, N, N]."""
    inter = otf_patch(setup, coeffs)
    total = 0.0
    for k in range(setup.n_objects):
        total += loss_terms(d[k], inter[k]["H"], setup.weights[k], setup.gamma).sum()
    return total


def loss_object_grad_patch(setup, coeffs, d):
    """(loss, objects [K, N, N], dL/da [J, M]) of one patch.

    Gradient chain (derived from Eqs. 12, 21, 20, 22):
      G_j   = dL/d conj(H_j) = -w_j conj(O) (D_j - O H_j)
      g_s   = 2 Re F^H G_j                      (dL/ds, H = F s)
      g_q   = (g_s - sum_x g_s s) / z           (s = q / z, z = sum q)
      G_P   = F^H (g_q p)                       (q = |p|^2, p = F P)
      g_phi = 2 Im(conj(P) G_P)                 (P = A exp(i phi))
      g_a   = sum_k c_k sum_v B_k(v) g_phi,k(v)
    """
    coeffs = np.asarray(coeffs, np.float64)
    inter = otf_patch(setup, coeffs)
    total = 0.0
    objs = []
    grad = np.zeros_like(coeffs)
    for k in range(setup.n_objects):
        it = inter[k]
        h = it["H"]
        w = setup.weights[k]
        num, den, ene = wiener_sums(d[k], h, w, setup.gamma)
        total += (ene - (num * num.conj()).real / den).sum()
        o = num / den
        objs.append(o)
        g_h = -w[:, None, None] * o.conj()[None] * (d[k] - o[None] * h)
        g_s = 2.0 * dft.ifft2_unnormalised(g_h).real
        g_q = (g_s - (g_s * it["s"]).sum(axis=(-2, -1), keepdims=True)) / it["z"]
        g_pp = dft.ifft2_unnormalised(g_q * it["p"])
        g_phi = 2.0 * (it["P"].conj() * g_pp).imag
        g_phi = np.where(setup.masks[k], g_phi, 0.0)
        grad += setup.scales[k] * np.tensordot(g_phi, setup.bases[k], axes=([1, 2], [1, 2]))
    return total, np.array(objs), grad


def explicit_loss_grad_patch(setup, coeffs, d, objects):
    """The object-inferring loss of one patch (Sec. 2.2.1, Eq. 8, with the
    regulariser R = sum_k sum_u |O_k|^2 and beta = gamma, under which the
    Wiener object of Eq. 11 is its exact minimiser) for given objects:

      L = sum_k sum_u [ sum_j w_kj |D_kj - O_k H_kj|^2 + gamma |O_k|^2 ]

    coeffs [J, M], d [K, J, N, N], objects [K, N, N] (full spectra). Returns
    (loss, dL/da [J, M], g_O [K, N, N]) with g_O(u) = dL/dconj(O(u)) per
    frequency: gamma O - sum_j w conj(H_j) (D_j - O H_j).
    dL/da follows the chain of loss_object_grad_patch from
    G_j = dL/dconj(H_j) = -w_j conj(O) (D_j - O H_j) with O held fixed."""
    coeffs = np.asarray(coeffs, np.float64)
    objects = np.asarray(objects, np.complex128)
    inter = otf_patch(setup, coeffs)
    total = 0.0
    grad = np.zeros_like(coeffs)
    g_obj = []
    for k in range(setup.n_objects):
        it = inter[k]
        h = it["H"]
        w = setup.weights[k][:, None, None]
        o = objects[k]
        res = d[k] - o[None] * h
        total += (w * (res * res.conj()).real).sum() + setup.gamma * (o * o.conj()).real.sum()
        g_obj.append(setup.gamma * o - (w * h.conj() * res).sum(axis=0))
        g_h = -w * o.conj()[None] * res
        g_s = 2.0 * dft.ifft2_unnormalised(g_h).real
        g_q = (g_s - (g_s * it["s"]).sum(axis=(-2, -1), keepdims=True)) / it["z"]
        g_pp = dft.ifft2_unnormalised(g_q * it["p"])
        g_phi = 2.0 * (it["P"].conj() * g_pp).imag
        g_phi = np.where(setup.masks[k], g_phi, 0.0)
        grad += setup.scales[k] * np.tensordot(g_phi, setup.bases[k], axes=([1, 2], [1, 2]))
    return total, grad, np.array(g_obj)


def loss_object_grad(setup, coeffs, d):
    """Batched over patches: coeffs [P, J, M], d [P, K, J, N, N]."""
    losses, objs, grads = [], [], []
    for p in range(coeffs.shape[0]):
        l, o, g = loss_object_grad_patch(setup, coeffs[p], d[p])
        losses.append(l)
        objs.append(o)
        grads.append(g)
    return np.array(losses), np.array(objs), np.array(grads)


def synth_spectra(setup, coeffs_true, objects, noise):
    """Data D_kj = F(o_k (*) s_kj + n_kj) (Eq. 6 with circular convolution):
    coeffs_true [J, M], objects [K, N, N] real, noise [K, J, N, N] real."""
    inter = otf_patch(setup, coeffs_true)
    d = []
    for k in range(setup.n_objects):
        fo = dft.fft2(objects[k])
        d.append(fo[None] * inter[k]["H"] + dft.fft2(noise[k]))
    return np.array(d)


def half_spectrum(x):
    """[..., N, N] -> [..., N, N/2 + 1] (the columns kx = 0..N/2)."""
    n = x.shape[-1]
    return x[..., : n // 2 + 1]


def full_from_half(xh, n):
    """Inverse of half_spectrum for Hermitian spectra of real images:
    X[ky, kx] = conj(X[-ky, -kx]) for kx > N/2."""
    xh = np.asarray(xh)
    out = np.zeros(xh.shape[:-1] + (n,), dtype=np.complex128)
    out[..., : n // 2 + 1] = xh
    ky = (-np.arange(n)) % n
    for kx in range(n // 2 + 1, n):
        out[..., :, kx] = np.conj(xh[..., ky, n - kx])
    return out
