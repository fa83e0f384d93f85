"""The Lofdahl-Scharmer Fourier filter of the object (Sec. 4.1.1, "Fourier
filtering", Eq. 25), in FP64 (test infrastructure only).

Per patch and object k, from the frames' data spectra D_kj and OTFs S_kj:

  H_k(u) = 1 - nu sum_j w_j |S_kj(u)|^2 / |sum_j w_j D_kj(u) conj(S_kj(u))|^2

then H < 0.2 -> 0 and H > 1 -> 1, a 3 x 3 median, and every nonzero value not
connected to the zero frequency set to zero. The filtered object is H_k O_k.

Readings (the printed equation and text leave these open):
* nu, the noise power of one frame's spectrum per frequency, multiplies the
  printed ratio (nu = 1 is the printed form): without it the ratio has the
  units of 1 / |D|^2. The cross spectrum conjugates S (the least-squares
  object estimate is sum_j D_j conj(S_j) / sum_j |S_j|^2), and the frame
  weights w_j of the loss enter both sums (w = 1 is the printed form).
* |n|^2 = 0 gives H = -inf (or NaN), i.e. 0 after the threshold.
* Precision: the paper does not fix it; the threshold decides which values
  survive, so the oracle evaluates H in the precision it is given with the
  operations in a fixed order (float32 for parity with the FP32 kernel,
  float64 for the closed-form pins); the median and the connectivity are
  exact in either.
* The frequency plane is periodic: the median window and the connectivity
  wrap around at the edges. Connectivity is 4-neighbour.
* The half spectrum fixes the plane: a frequency with 0 < kx < N/2 and its
  mirror -u have the same H (the sums at -u are the conjugates of those at
  u); the columns kx = 0 and N/2 are evaluated from their own data.
"""

from collections import deque

import numpy as np


def ls_filter_raw(d, s, weights, noise_power, dtype=np.float64):
    """H before the threshold, [N, N], from d, s [J, N, N] complex (full
    spectra) and weights [J], computed in `dtype` with each product and sum
    rounded on its own, in this order (frames in order):
      t_re = d_re s_re + d_im s_im,  t_im = d_im s_re - d_re s_im,
      n += w t,  q += w (s_re s_re + s_im s_im),
      H = 1 - (nu q) / (n_re n_re + n_im n_im).
    float32 takes the threshold decisions in the kernel's precision."""
    f = np.dtype(dtype).type
    d = np.asarray(d)
    s = np.asarray(s)
    dr, di = np.real(d).astype(dtype), np.imag(d).astype(dtype)
    sr, si = np.real(s).astype(dtype), np.imag(s).astype(dtype)
    w = np.asarray(weights).astype(dtype)
    nr = np.zeros(d.shape[1:], dtype)
    ni = np.zeros(d.shape[1:], dtype)
    q = np.zeros(d.shape[1:], dtype)
    for j in range(d.shape[0]):
        tr = dr[j] * sr[j] + di[j] * si[j]
        ti = di[j] * sr[j] - dr[j] * si[j]
        nr = nr + w[j] * tr
        ni = ni + w[j] * ti
        q = q + w[j] * (sr[j] * sr[j] + si[j] * si[j])
    n2 = nr * nr + ni * ni
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        return f(1) - (f(noise_power) * q) / n2


def threshold(h):
    """H < 0.2 -> 0 (NaN too), H > 1 -> 1, in the precision of h."""
    h = np.asarray(h)
    f = h.dtype.type
    with np.errstate(invalid="ignore"):
        out = np.where(h >= f(0.2), h, f(0))
    return np.minimum(out, f(1))


def median3x3_periodic(h):
    """The median of each pixel's 3 x 3 neighbourhood, wrapping at the edges."""
    h = np.asarray(h, np.float64)
    ny, nx = h.shape
    out = np.empty_like(h)
    for y in range(ny):
        for x in range(nx):
            vals = sorted(h[(y + dy) % ny, (x + dx) % nx] for dy in (-1, 0, 1) for dx in (-1, 0, 1))
            out[y, x] = vals[4]
    return out


def connected_to_zero(mask):
    """Pixels of `mask` (bool [N, N]) 4-connected, on the periodic plane, to
    the pixel [0, 0] (empty if mask[0, 0] is False): a breadth-first search."""
    mask = np.asarray(mask, bool)
    ny, nx = mask.shape
    reach = np.zeros_like(mask)
    if not mask[0, 0]:
        return reach
    reach[0, 0] = True
    todo = deque([(0, 0)])
    while todo:
        y, x = todo.popleft()
        for yy, xx in (((y + 1) % ny, x), ((y - 1) % ny, x), (y, (x + 1) % nx), (y, (x - 1) % nx)):
            if mask[yy, xx] and not reach[yy, xx]:
                reach[yy, xx] = True
                todo.append((yy, xx))
    return reach


def lofdahl_scharmer_filter(d, s, weights, noise_power, dtype=np.float64):
    """The filter H_k [N, N] of one patch and object: d, s [J, N, N]; H
    evaluated in `dtype`, the median and the connectivity exact."""
    h = median3x3_periodic(threshold(ls_filter_raw(d, s, weights, noise_power, dtype)))
    return np.where(connected_to_zero(h > 0), h, 0.0)
