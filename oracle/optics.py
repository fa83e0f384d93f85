"""Pupil geometry and modal bases for the oracle (test infrastructure only).

Readings of the paper used here (Sec. 3.1 defines the generalised pupil and
the modal wavefront but fixes no sampling convention):

* Grid [row y][column x], N x N. The pupil centre sits between pixels at
  c = (N - 1) / 2 on both axes, so the mask is point-symmetric under
  n -> N - 1 - n. A pixel is inside iff (x - c)^2 + (y - c)^2 <= R^2 with
  R = D_p / 2 (D_p = pupil diameter in pixels); a central obscuration of
  fraction e removes pixels with (x - c)^2 + (y - c)^2 < (e R)^2.
* rho = r / R, theta = atan2(y - c, x - c) (measured from +x).
* Zernike modes in Noll's (1976) ordering and normalisation (unit rms on the
  disk): Z_j = sqrt(n+1) R_n^m(rho) for m = 0, and
  sqrt(2(n+1)) R_n^m(rho) cos(m theta) (j even) / sin(m theta) (j odd).
* Kolmogorov statistics of the Zernike coefficients follow Noll (1976): the
  covariance below is written out from the Kolmogorov phase spectrum
  W(f) = A r0^(-5/3) f^(-11/3) and the Weber-Schafheitlin integral; A is fixed
  by the phase structure function D(r) = 2 ((24/5) Gamma(6/5))^(5/6) (r/r0)^(5/3).
* The Karhunen-Loeve basis (Sec. 3.1: diagonalise the Zernike covariance) is
  built from Zernike modes 2..J_max, where J_max closes the smallest complete
  radial order with at least 4 M + 1 modes. The covariance is block diagonal
  in (m, cos/sin); each block is diagonalised separately (so degenerate
  cos/sin pairs never mix), each eigenvector's largest-magnitude component is
  made positive, the modes are sorted by decreasing eigenvalue (ties: smaller
  m first, cos before sin), the first M are sampled on the pupil and then
  re-orthonormalised on the discrete pupil by modified Gram-Schmidt in that
  order, with the inner product <f, g> = mean over pupil pixels of f g.
"""

import math
import numpy as np
from scipy.special import gamma as _gamma


# ---------------------------------------------------------------- pupil ---

def pupil_mask(n, diam_px, obscuration=0.0):
    """Binary aperture A_k on the N x N grid (Sec. 3.1, Eq. 20)."""
    c = (n - 1) / 2.0
    r = float(np.float32(diam_px)) * 0.5
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    r2 = (x - c) ** 2 + (y - c) ** 2
    inside = r2 <= r * r
    if obscuration > 0.0:
        ro = float(np.float32(obscuration)) * r
        inside &= r2 >= ro * ro
    return inside


def polar_coords(n, diam_px):
    """(rho, theta) of every pixel, rho normalised to the pupil radius."""
    c = (n - 1) / 2.0
    r = float(np.float32(diam_px)) * 0.5
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    return np.hypot(x - c, y - c) / r, np.arctan2(y - c, x - c)


# -------------------------------------------------------------- Zernike ---

def noll_to_nm(j):
    """Noll index j >= 1 -> (n, m >= 0). Within radial order n the |m|
    values increase; even j carries cos(m theta), odd j sin(m theta)."""
    if j < 1:
        raise ValueError("Noll index starts at 1")
    n = 0
    while (n + 1) * (n + 2) // 2 < j:
        n += 1
    p = j - n * (n + 1) // 2 - 1
    if n % 2 == 0:
        m = 2 * ((p + 1) // 2)
    else:
        m = 2 * (p // 2) + 1
    return n, m


def zernike_radial(n, m, rho):
    """R_n^m(rho) = sum_s (-1)^s (n-s)! / (s! ((n+m)/2-s)! ((n-m)/2-s)!) rho^(n-2s)."""
    out = np.zeros_like(rho, dtype=np.float64)
    for s in range((n - m) // 2 + 1):
        coef = ((-1) ** s * math.factorial(n - s)
                / (math.factorial(s) * math.factorial((n + m) // 2 - s)
                   * math.factorial((n - m) // 2 - s)))
        out += coef * rho ** (n - 2 * s)
    return out


def zernike(j, rho, theta):
    """Noll-normalised Zernike mode Z_j evaluated at (rho, theta)."""
    n, m = noll_to_nm(j)
    rad = zernike_radial(n, m, rho)
    if m == 0:
        return math.sqrt(n + 1) * rad
    ang = np.cos(m * theta) if j % 2 == 0 else np.sin(m * theta)
    return math.sqrt(2 * (n + 1)) * rad * ang


def zernike_basis(n_pix, diam_px, noll_indices, obscuration=0.0):
    """[M, N, N] Zernike modes sampled on the pupil, zero outside it."""
    mask = pupil_mask(n_pix, diam_px, obscuration)
    rho, th = polar_coords(n_pix, diam_px)
    out = np.zeros((len(noll_indices), n_pix, n_pix))
    for i, j in enumerate(noll_indices):
        out[i] = np.where(mask, zernike(j, rho, th), 0.0)
    return out


# ------------------------------------------------- Kolmogorov statistics ---

def kolmogorov_psd_constant():
    """A in W(f) = A r0^(-5/3) f^(-11/3) (f in cycles per unit length).

    Fixed by D(r) = 2 int W(f) (1 - cos 2 pi f.r) d^2f = 6.8839 (r/r0)^(5/3):
    with mu = 8/3, int_0^inf u^-mu (1 - J0(u)) du = -Gamma((1-mu)/2) /
    (2^mu Gamma((1+mu)/2)), so D(r) = 4 pi A (2 pi)^(5/3) I r^(5/3)."""
    mu = 8.0 / 3.0
    integral = -_gamma((1 - mu) / 2) / (2 ** mu * _gamma((1 + mu) / 2))
    d_coef = 2.0 * ((24.0 / 5.0) * _gamma(6.0 / 5.0)) ** (5.0 / 6.0)
    return d_coef / (4 * math.pi * (2 * math.pi) ** (5.0 / 3.0) * integral)


def noll_covariance(noll_indices):
    """Covariance <a_j a_j'> of Noll-normalised Zernike coefficients of a
    Kolmogorov phase screen, in units of (D/r0)^(5/3) rad^2 (Noll 1976).

    Nonzero only for equal m and, for m > 0, both cos (even j) or both sin
    (odd j). Value:
      K (-1)^((n+n'-2m)/2) sqrt((n+1)(n'+1)) Gamma((n+n'-5/3)/2)
        / (Gamma((n-n'+17/3)/2) Gamma((n'-n+17/3)/2) Gamma((n+n'+23/3)/2))
    with K = A 8 pi^(8/3) Gamma(14/3) / 2^(14/3): the angular integral gives
    2 pi, the radial one is the Weber-Schafheitlin integral of
    J_{n+1} J_{n'+1} x^(-14/3), and (R/r0)^(5/3) = 2^(-5/3) (D/r0)^(5/3).
    """
    a = kolmogorov_psd_constant()
    k = a * 8.0 * math.pi ** (8.0 / 3.0) * _gamma(14.0 / 3.0) / 2 ** (14.0 / 3.0)
    js = list(noll_indices)
    cov = np.zeros((len(js), len(js)))
    for u, j in enumerate(js):
        n, m = noll_to_nm(j)
        for v, jp in enumerate(js):
            n2, m2 = noll_to_nm(jp)
            if m != m2:
                continue
            if m != 0 and (j % 2) != (jp % 2):
                continue
            sign = (-1) ** ((n + n2 - 2 * m) // 2)
            cov[u, v] = (k * sign * math.sqrt((n + 1) * (n2 + 1))
                         * _gamma((n + n2 - 5.0 / 3.0) / 2)
                         / (_gamma((n - n2 + 17.0 / 3.0) / 2)
                            * _gamma((n2 - n + 17.0 / 3.0) / 2)
                            * _gamma((n + n2 + 23.0 / 3.0) / 2)))
    return cov


# ------------------------------------------------------------------- KL ---

def kl_jmax(n_modes):
    """Last Noll index used to build M KL modes: closes the smallest
    complete radial order n with (n+1)(n+2)/2 >= 4 M + 1."""
    n = 0
    while (n + 1) * (n + 2) // 2 < 4 * n_modes + 1:
        n += 1
    return (n + 1) * (n + 2) // 2


def kl_modes(n_modes):
    """Karhunen-Loeve modes as combinations of Zernike modes 2..J_max.

    Returns (coef [M, J_max-1], variance [M], m_of_mode [M]): KL_i =
    sum_j coef[i, j-2] Z_j, with variance in units of (D/r0)^(5/3).
    """
    jmax = kl_jmax(n_modes)
    js = np.arange(2, jmax + 1)
    cov = noll_covariance(js)
    blocks = {}
    for idx, j in enumerate(js):
        n, m = noll_to_nm(int(j))
        kind = 0 if (m == 0 or j % 2 == 0) else 1  # 0: cos / radial, 1: sin
        blocks.setdefault((m, kind), []).append(idx)
    entries = []
    for (m, kind), idxs in blocks.items():
        sub = cov[np.ix_(idxs, idxs)]
        evals, evecs = np.linalg.eigh(sub)
        for e in range(len(idxs)):
            vec = evecs[:, e].copy()
            big = np.argmax(np.abs(vec))
            if vec[big] < 0:
                vec = -vec
            full = np.zeros(len(js))
            full[idxs] = vec
            entries.append((float(evals[e]), m, kind, full))
    entries.sort(key=lambda t: (-float("%.9e" % t[0]), t[1], t[2]))
    entries = entries[:n_modes]
    coef = np.array([t[3] for t in entries])
    var = np.array([t[0] for t in entries])
    ms = np.array([t[1] for t in entries])
    return coef, var, ms


def kl_basis(n_pix, diam_px, n_modes, obscuration=0.0):
    """[M, N, N] KL modes sampled on the pupil and re-orthonormalised on the
    discrete pupil (modified Gram-Schmidt, unit mean square)."""
    coef, var, ms = kl_modes(n_modes)
    jmax = coef.shape[1] + 1
    zb = zernike_basis(n_pix, diam_px, range(2, jmax + 1), obscuration)
    mask = pupil_mask(n_pix, diam_px, obscuration)
    npup = mask.sum()
    vecs = np.tensordot(coef, zb, axes=(1, 0))[:, mask]  # [M, n_pup]
    q = np.zeros_like(vecs)
    for i in range(vecs.shape[0]):
        v = vecs[i].copy()
        for p in range(i):
            v -= (np.dot(q[p], v) / npup) * q[p]
        v /= math.sqrt(np.dot(v, v) / npup)
        q[i] = v
    out = np.zeros((n_modes, n_pix, n_pix))
    out[:, mask] = q
    return out, var, ms


def mode_parity_m(basis_kind, n_modes):
    """Azimuthal order m of every mode (Zernike: Noll 2..M+1)."""
    if basis_kind == "zernike":
        return np.array([noll_to_nm(j)[1] for j in range(2, n_modes + 2)])
    return kl_modes(n_modes)[2]


def mode_variances(basis_kind, n_modes):
    """Kolmogorov variance of each coefficient in units of (D/r0)^(5/3)."""
    if basis_kind == "zernike":
        return np.diag(noll_covariance(range(2, n_modes + 2))).copy()
    return kl_modes(n_modes)[1]


# -------------------------------------------------------------- support ---

def otf_support(mask):
    """Exact support of the OTF: frequencies u (on the N x N torus) at which
    the circular autocorrelation of the binary pupil is nonzero. Computed by
    brute force over pairs of pupil pixels (integer arithmetic)."""
    n = mask.shape[0]
    ys, xs = np.nonzero(mask)
    supp = np.zeros((n, n), dtype=bool)
    dy = np.mod(ys[:, None] - ys[None, :], n)
    dx = np.mod(xs[:, None] - xs[None, :], n)
    supp[dy.ravel(), dx.ravel()] = True
    return supp
