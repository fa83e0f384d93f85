"""Pins of the FP64 oracle's Lofdahl-Scharmer filter (Sec. 4.1.1, Eq. 25)
against closed forms, library routines and brute force (CPU only)."""

import numpy as np
import pytest

from oracle import filters

scipy_ndimage = pytest.importorskip("scipy.ndimage")


def _const_planes(n, d_vals, s_vals):
    d = np.array([np.full((n, n), v, np.complex128) for v in d_vals])
    s = np.array([np.full((n, n), v, np.complex128) for v in s_vals])
    return d, s


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_raw_filter_closed_form(dtype):
    """Constant spectra: H = 1 - nu sum w |s|^2 / |sum w d conj(s)|^2."""
    d_vals = [3.0 + 1.0j, -2.0 + 0.5j, 1.5 - 2.0j]
    s_vals = [0.8 - 0.1j, 0.5 + 0.3j, 0.2 + 0.6j]
    w = [1.0, 0.5, 2.0]
    nu = 0.7
    d, s = _const_planes(8, d_vals, s_vals)
    num = sum(wj * abs(sj) ** 2 for wj, sj in zip(w, s_vals))
    cross = sum(wj * dj * np.conj(sj) for wj, dj, sj in zip(w, d_vals, s_vals))
    want = 1.0 - nu * num / abs(cross) ** 2
    h = filters.ls_filter_raw(d, s, w, nu, dtype)
    assert h.dtype == dtype
    tol = 1e-14 if dtype == np.float64 else 1e-6
    assert np.allclose(h, want, rtol=tol, atol=tol)


def test_raw_filter_is_the_printed_form_for_unit_noise_and_weights():
    """nu = 1, w = 1: H = 1 - sum |S|^2 / |sum D conj(S)|^2 elementwise."""
    rng = np.random.default_rng(5)
    d = rng.standard_normal((4, 6, 6)) + 1j * rng.standard_normal((4, 6, 6))
    s = rng.standard_normal((4, 6, 6)) + 1j * rng.standard_normal((4, 6, 6))
    want = 1.0 - np.sum(np.abs(s) ** 2, 0) / np.abs(np.sum(d * np.conj(s), 0)) ** 2
    assert np.allclose(filters.ls_filter_raw(d, s, np.ones(4), 1.0), want, rtol=1e-12)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_threshold(dtype):
    h = np.array([np.nan, -np.inf, -1.0, 0.1999, 0.2, 0.5, 1.0, 1.5, np.inf], dtype)
    want = np.array([0, 0, 0, 0, 0.2, 0.5, 1.0, 1.0, 1.0], dtype)
    out = filters.threshold(h)
    assert out.dtype == dtype and np.array_equal(out, want)


def test_median_matches_scipy_wrap():
    rng = np.random.default_rng(7)
    for shape in ((8, 8), (12, 10), (48, 48)):
        h = rng.integers(0, 6, shape).astype(np.float64) / 5.0  # many ties
        want = scipy_ndimage.median_filter(h, size=3, mode="wrap")
        assert np.array_equal(filters.median3x3_periodic(h), want)


def test_median_removes_isolated_pixels_and_keeps_blocks():
    h = np.zeros((16, 16))
    h[3, 3] = 1.0                 # isolated: removed
    h[8:11, 8:11] = 0.5           # a 3 x 3 block: its centre survives
    h[0, 0:3] = 0.7               # a line across the wrap: removed
    m = filters.median3x3_periodic(h)
    assert m[3, 3] == 0.0 and m[9, 9] == 0.5 and m[0, 1] == 0.0


def test_connected_to_zero_matches_scipy_label_off_the_edges():
    """Masks whose components stay away from the edges of the centred
    (fftshifted) plane: the periodic component of frequency 0 is scipy's
    label of the centre pixel."""
    rng = np.random.default_rng(11)
    n = 32
    for _ in range(20):
        m = rng.random((n, n)) < 0.55
        m[:2, :] = m[-2:, :] = False
        m[:, :2] = m[:, -2:] = False
        m[n // 2, n // 2] = True
        lab, _ = scipy_ndimage.label(m)  # 4-connectivity
        want_c = lab == lab[n // 2, n // 2]
        got = filters.connected_to_zero(np.fft.ifftshift(m))
        assert np.array_equal(np.fft.fftshift(got), want_c)


def test_connected_to_zero_on_the_torus_matches_label_with_wrapped_merges():
    """Dense random masks (components cross the edges): scipy's planar label
    with the labels that touch across an edge merged (union-find) gives the
    periodic components."""
    rng = np.random.default_rng(13)
    for n in (6, 9, 16):
        for _ in range(30):
            m = rng.random((n, n)) < 0.5
            lab, nl = scipy_ndimage.label(m)
            parent = list(range(nl + 1))

            def find(a):
                while parent[a] != a:
                    parent[a] = parent[parent[a]]
                    a = parent[a]
                return a

            for i in range(n):
                for a, b in ((lab[0, i], lab[n - 1, i]), (lab[i, 0], lab[i, n - 1])):
                    if a and b:
                        parent[find(a)] = find(b)
            got = filters.connected_to_zero(m)
            if not m[0, 0]:
                assert not got.any()
                continue
            root = find(lab[0, 0])
            want = np.array([[lab[y, x] != 0 and find(lab[y, x]) == root for x in range(n)] for y in range(n)])
            assert np.array_equal(got, want)


def test_connected_to_zero_brute_force_tiny():
    """Every 3 x 3 mask: the component by repeated dilation."""
    for bits in range(1 << 9):
        m = np.array([(bits >> i) & 1 for i in range(9)], bool).reshape(3, 3)
        r = np.zeros_like(m)
        r[0, 0] = m[0, 0]
        for _ in range(9):
            grow = r | np.roll(r, 1, 0) | np.roll(r, -1, 0) | np.roll(r, 1, 1) | np.roll(r, -1, 1)
            r = grow & m
        assert np.array_equal(filters.connected_to_zero(m), r)


def _island_case(n=32):
    """J = 1, S = 1: H = 1 - nu / |D|^2. |D| large on a disk around frequency
    0 (radius 6) and on a 5 x 5 island centred at (+-12, +-12), small
    elsewhere (H < 0.2 there); Hermitian."""
    k = np.fft.fftfreq(n) * n
    ky, kx = np.meshgrid(k, k, indexing="ij")
    big = (ky ** 2 + kx ** 2 <= 36) | ((np.abs(np.abs(ky) - 12) <= 2) & (np.abs(np.abs(kx) - 12) <= 2))
    d = np.where(big, 10.0, 1.0).astype(np.complex128)[None]
    s = np.ones_like(d)
    return d, s, 4.0  # H = 0.96 on the big set, -3 elsewhere


def test_filter_removes_peaks_not_connected_to_zero():
    d, s, nu = _island_case()
    h = filters.lofdahl_scharmer_filter(d, s, [1.0], nu)
    m = filters.median3x3_periodic(filters.threshold(filters.ls_filter_raw(d, s, [1.0], nu)))
    assert m[12, 12] > 0 and m[-12, 12] > 0          # the island survives the median ...
    assert h[12, 12] == 0 and h[-12, -12] == 0       # ... but is not connected to 0
    assert h[0, 0] == pytest.approx(0.96) and h[3, 3] == pytest.approx(0.96)
    assert h[10, 0] == 0                              # outside the disk


@pytest.mark.parametrize("nu,want", [(0.5, 0.5), (0.9, 0.0), (-1.0, 1.0)])
def test_filter_constant_data(nu, want):
    """D = S = 1 everywhere (one frame): H = 1 - nu before the threshold."""
    d, s = _const_planes(16, [1.0], [1.0])
    h = filters.lofdahl_scharmer_filter(d, s, [1.0], nu)
    assert np.allclose(h, want, atol=1e-15)


def test_filter_is_symmetric_for_spectra_of_real_images():
    """D and S from real images (made exactly Hermitian): H(-u) = H(u) bit
    for bit."""
    rng = np.random.default_rng(17)
    n, j = 16, 3
    img = 1.0 + 0.2 * rng.standard_normal((j, n, n))
    psf = rng.random((j, n, n)) ** 8
    psf /= psf.sum(axis=(1, 2), keepdims=True)
    d, s = np.fft.fft2(img), np.fft.fft2(psf)
    neg = (-np.arange(n)) % n
    d = 0.5 * (d + np.conj(d[:, neg][:, :, neg]))  # exactly Hermitian
    s = 0.5 * (s + np.conj(s[:, neg][:, :, neg]))
    noise = float(np.median(np.abs(d) ** 2)) * 0.05
    for dtype in (np.float64, np.float32):
        h = filters.lofdahl_scharmer_filter(d, s, np.ones(j), noise, dtype)
        mirror = h[(-np.arange(n)) % n][:, (-np.arange(n)) % n]
        assert np.array_equal(h, mirror)
        assert h[0, 0] > 0.9
