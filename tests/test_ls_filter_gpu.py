"""GPU parity of the Lofdahl-Scharmer object filter (mfbd_ls_filter_objects,
Sec. 4.1.1, Eq. 25) against the oracle, bit for bit.

The kernel's inputs are the oracle's: data spectra D from the oracle's
forward model and OTFs S from `oracle.mfbd.otf_patch`, both rounded to
complex64. The oracle evaluates H in float32 with the kernel's order of
operations (the threshold decisions are then the same); the median and the
connectivity are exact, so the filters agree bit for bit and the filtered
object is the input object times the filter.
"""

import numpy as np
import pytest
import torch

from oracle import filters
from oracle import mfbd as omfbd
from tests import cases

pytestmark = pytest.mark.gpu


def _case(n_pix, diams, n_frames, n_patches, seed):
    wl = (6563.0, 8542.0, 5000.0)[:len(diams)]
    return cases.make_case(n_pix=n_pix, diams=diams, wavelengths=wl, n_frames=n_frames, n_modes=12, basis="kl",
                           n_patches=n_patches, seed=seed)


def _plan(case, full_spectrum=False, weights=None):
    from paper_2505_10639_gb300.mfbd import Plan
    s = case["setup"]
    return Plan(case["n_pix"], case["d"].shape[0], list(case["diams"]), list(case["wavelengths"]),
                case["n_frames"], case["n_modes"], basis=case["basis"], gamma=s.gamma,
                weights=s.weights if weights is None else weights, full_spectrum=full_spectrum)


def _inputs(case):
    """D (complex64, half or full layout chosen later) and S (complex64 half
    spectra) from the oracle."""
    n = case["n_pix"]
    a = case["a_eval"]
    s_half = np.array([[omfbd.half_spectrum(o["H"]) for o in omfbd.otf_patch(case["setup"], a[p])]
                       for p in range(a.shape[0])]).astype(np.complex64)
    return case["d"].astype(np.complex64), s_half, n


def _oracle_filters(case, d64, s_half, nu, weights):
    n = case["n_pix"]
    P, K = s_half.shape[:2]
    out = np.zeros((P, K, n, n))
    for p in range(P):
        for k in range(K):
            d_full = omfbd.full_from_half(omfbd.half_spectrum(d64[p, k]).astype(np.complex128), n)
            s_full = omfbd.full_from_half(s_half[p, k].astype(np.complex128), n)
            out[p, k] = filters.lofdahl_scharmer_filter(d_full, s_full, weights[k], nu, np.float32)
    return out


def _noise_power(case, factor):
    n = case["n_pix"]
    return factor * n * n * 1e-6  # sigma = 1e-3 per pixel


@pytest.mark.parametrize("n_pix,diams,n_frames,n_patches,factor",
                         [(64, (36.0, 28.0), 12, 3, 200.0), (48, (22.0,), 5, 2, 50.0),
                          (96, (40.0, 30.0), 4, 1, 100.0), (128, (56.0,), 3, 1, 400.0)])
def test_ls_filter_matches_oracle_bits(n_pix, diams, n_frames, n_patches, factor):
    case = _case(n_pix, diams, n_frames, n_patches, 20250521 + n_pix)
    d64, s_half, n = _inputs(case)
    nu = _noise_power(case, factor)
    weights = np.asarray(case["setup"].weights, np.float32)
    want = _oracle_filters(case, d64, s_half, nu, weights)
    plan = _plan(case)
    d = torch.from_numpy(np.ascontiguousarray(omfbd.half_spectrum(d64))).cuda()
    s = torch.from_numpy(s_half).cuda()
    rng = np.random.default_rng(3)
    obj0 = (rng.standard_normal(plan.object_shape()) + 1j * rng.standard_normal(plan.object_shape())).astype(
        np.complex64)
    obj = torch.from_numpy(obj0).cuda()
    h = plan.ls_filter_objects(d, s, nu, obj=obj)
    torch.cuda.synchronize()
    h = h.cpu().numpy()
    want_half = want[..., : n // 2 + 1]
    zeros = np.mean(want_half == 0)
    print("N=%d: %.1f %% of the half plane filtered out" % (n, 100 * zeros))
    assert 0.01 < zeros < 0.99  # the threshold matters here
    assert np.array_equal(h.astype(np.float64), want_half)
    got = obj.cpu().numpy()
    assert np.array_equal(got.real, obj0.real * h) and np.array_equal(got.imag, obj0.imag * h)


def test_ls_filter_full_spectrum_layout_and_weights():
    """Full N x N spectra and objects, unequal frame weights: the object is
    multiplied by the full plane of H (its mirror for kx > N/2)."""
    case = _case(64, (32.0, 26.0), 6, 2, 20250530)
    d64, s_half, n = _inputs(case)
    w = np.array([[1.0, 0.5, 2.0, 1.0, 0.25, 1.5], [0.7, 1.0, 1.0, 3.0, 0.5, 1.0]], np.float32)
    nu = _noise_power(case, 200.0)
    want = _oracle_filters(case, d64, s_half, nu, w)
    plan = _plan(case, full_spectrum=True, weights=w)
    # the kernel reads D's full rows: give it the exactly Hermitian full planes the oracle used
    d_full = np.array([[omfbd.full_from_half(omfbd.half_spectrum(d64[p, k]).astype(np.complex128), n)
                        for k in range(d64.shape[1])] for p in range(d64.shape[0])]).astype(np.complex64)
    obj0 = np.ones(plan.object_shape(), np.complex64) * (1.0 + 2.0j)
    obj = torch.from_numpy(obj0).cuda()
    h = plan.ls_filter_objects(torch.from_numpy(d_full).cuda(), torch.from_numpy(s_half).cuda(), nu, obj=obj)
    torch.cuda.synchronize()
    assert np.array_equal(h.cpu().numpy().astype(np.float64), want[..., : n // 2 + 1])
    got = obj.cpu().numpy()
    assert np.array_equal(got.real, (1.0 * want).astype(np.float32))
    assert np.array_equal(got.imag, (2.0 * want).astype(np.float32))
    # without a filter output (plan scratch holds the thresholded H): the same object
    obj2 = torch.from_numpy(obj0).cuda()
    assert plan.ls_filter_objects(torch.from_numpy(d_full).cuda(), torch.from_numpy(s_half).cuda(), nu, obj=obj2,
                                  want_filter=False) is None
    torch.cuda.synchronize()
    assert np.array_equal(obj2.cpu().numpy(), got)


def test_ls_filter_argument_errors():
    from paper_2505_10639_gb300 import _lib
    case = _case(48, (22.0,), 3, 1, 20250531)
    plan = _plan(case)
    d = torch.zeros(plan.spectra_shape(), dtype=torch.complex64, device="cuda")
    s = torch.zeros(plan.otf_shape(), dtype=torch.complex64, device="cuda")
    with pytest.raises(_lib.MFBDError):
        plan.ls_filter_objects(d, s, float("nan"))
    with pytest.raises(ValueError):
        plan.ls_filter_objects(d, s, 1.0, obj=None, want_filter=False)
    # all-zero data: every |n|^2 = 0, so H = 0 everywhere
    h = plan.ls_filter_objects(d, s, 1.0)
    torch.cuda.synchronize()
    assert not h.cpu().numpy().any()


@pytest.mark.parametrize("n_pix,diams,n_frames,n_patches,factor",
                         [(64, (36.0, 28.0), 12, 3, 200.0), (128, (56.0,), 3, 1, 400.0)])
def test_ls_filter_against_fp64_definition(n_pix, diams, n_frames, n_patches, factor):
    """The FP32 kernel against Eq. 25 evaluated in FP64. The threshold turns
    H into a decision, so the two may decide differently only where the FP64
    H lies within the FP32 rounding error of 0.2 (the error of nu q / |n|^2
    bounded per frequency from the sizes of the summed terms). Running the
    FP64 pipeline with the FP32 decisions at exactly those frequencies must
    then give the kernel's filter: the same zero pattern and the same values
    to FP32 rounding."""
    case = _case(n_pix, diams, n_frames, n_patches, 20250521 + n_pix)
    d64, s_half, n = _inputs(case)
    nu = _noise_power(case, factor)
    weights = np.asarray(case["setup"].weights, np.float32)
    plan = _plan(case)
    d = torch.from_numpy(np.ascontiguousarray(omfbd.half_spectrum(d64))).cuda()
    h = plan.ls_filter_objects(d, torch.from_numpy(s_half).cuda(), nu)
    torch.cuda.synchronize()
    h = h.cpu().numpy().astype(np.float64)
    eps = 2.0 ** -24
    ambiguous_total = 0
    for p in range(s_half.shape[0]):
        for k in range(s_half.shape[1]):
            dd = omfbd.full_from_half(omfbd.half_spectrum(d64[p, k]).astype(np.complex128), n)
            ss = omfbd.full_from_half(s_half[p, k].astype(np.complex128), n)
            w = weights[k].astype(np.float64)
            h64 = filters.ls_filter_raw(dd, ss, w, nu, np.float64)
            h32 = filters.ls_filter_raw(dd, ss, w, nu, np.float32).astype(np.float64)
            # FP32 error bound of H = 1 - r, r = nu q / |n|^2: q sums J
            # positive terms (relative error <= (J + 2) eps); n sums J terms
            # whose sizes add up to sum |w d s| (absolute error <= (J + 2)
            # eps sum |w d s|, doubled in |n|^2); one more eps for the ratio
            J = len(w)
            nabs = np.abs(np.tensordot(w, dd * np.conj(ss), axes=1))
            tsum = np.tensordot(np.abs(w), np.abs(dd) * np.abs(ss), axes=1)
            with np.errstate(divide="ignore", invalid="ignore"):
                bound = np.abs(1.0 - h64) * eps * ((J + 3.0) + 2.0 * (J + 2.0) * tsum / nabs)
            dec64 = np.nan_to_num(h64, nan=-1.0, neginf=-1.0) >= 0.2
            dec32 = np.nan_to_num(h32, nan=-1.0, neginf=-1.0) >= 0.2
            amb = np.abs(h64 - 0.2) <= 2.0 * np.nan_to_num(bound, nan=np.inf, posinf=np.inf)
            assert not np.any((dec32 != dec64) & ~amb), (p, k)
            ambiguous_total += int(np.sum(dec32 != dec64))
            t = np.minimum(np.where(dec32, np.nan_to_num(h64), 0.0), 1.0)
            med = filters.median3x3_periodic(t)
            want = np.where(filters.connected_to_zero(med > 0), med, 0.0)[:, : n // 2 + 1]
            got = h[p, k]
            assert np.array_equal(got == 0, want == 0), (p, k)
            assert np.allclose(got, want, rtol=1e-5, atol=0), (p, k, np.max(np.abs(got - want)))
    print("N=%d: %d threshold decisions differ between FP32 and FP64, all within the rounding bound"
          % (n, ambiguous_total))
