"""Host-side tests of the C ABI (no GPU): the library builds, loads and
exports every declared symbol; descriptors are validated; compute calls
refuse to run without a GPU (no CPU fallback); plan-time pupil, support and
modal bases built by the library's C++ agree with the independent oracle;
the library's register FFTs (run on the host) agree with the oracle's FFT.
"""

import ctypes
import glob
import os
import re

import numpy as np
import pytest
import torch

from oracle import dft, optics
from paper_2505_10639_gb300 import _lib, mfbd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    return _lib.load()


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(mfbd_\w+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert "mfbd_plan_create" in names and "mfbd_loss_grad" in names
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    for code in range(7):
        assert lib.mfbd_status_string(code).decode().startswith("MFBD_")
    assert b"unknown" in lib.mfbd_status_string(99)


def _desc(**kw):
    args = dict(n_pix=64, n_patches=1, diams=[32.0], wavelengths=[8542.0], n_frames=8, n_modes=20,
                basis="zernike", gamma=1e-3, weights=None, obscuration=0.0, user_basis=None,
                precision="fp32", full_spectrum=False)
    args.update(kw)
    return mfbd._Desc(**args)


@pytest.mark.parametrize("bad", [
    dict(n_objects_override=0), dict(n_frames=0), dict(n_modes=0), dict(n_modes=300),
    dict(diams=[0.0]), dict(diams=[65.0]), dict(wavelengths=[-1.0]), dict(gamma=0.0),
    dict(gamma=float("nan")), dict(obscuration=1.0), dict(n_patches=-1),
    dict(weights=[[1.0] * 7 + [-1.0]]), dict(basis="user"),
])
def test_invalid_descriptors_are_rejected(lib, bad):
    bad = dict(bad)
    k0 = bad.pop("n_objects_override", None)
    d = _desc(**bad)
    if k0 is not None:
        d.desc.n_objects = k0
    out = ctypes.c_void_p()
    st = lib.mfbd_plan_create(ctypes.byref(out), ctypes.byref(d.desc), None)
    assert st == _lib.MFBD_ERR_INVALID_ARG, lib.mfbd_last_error()
    assert out.value is None
    st = lib.mfbd_describe_object(ctypes.byref(d.desc), 0, None, None, None, None)
    assert st == _lib.MFBD_ERR_INVALID_ARG


def test_unsupported_size_and_null_arguments(lib):
    d = _desc(n_pix=80, diams=[40.0])  # patch sizes: 48, 64, 96, 128
    out = ctypes.c_void_p()
    assert lib.mfbd_plan_create(ctypes.byref(out), ctypes.byref(d.desc), None) == _lib.MFBD_ERR_UNSUPPORTED
    assert lib.mfbd_plan_create(None, ctypes.byref(d.desc), None) == _lib.MFBD_ERR_INVALID_ARG
    assert lib.mfbd_forward(None, None, None, None, None, None) == _lib.MFBD_ERR_INVALID_ARG
    assert lib.mfbd_backward(None, None, None) == _lib.MFBD_ERR_INVALID_ARG
    assert lib.mfbd_loss_grad_host(None, None, None, None, None, None, 4, None) == _lib.MFBD_ERR_INVALID_ARG
    assert lib.mfbd_plan_destroy(None) == _lib.MFBD_OK


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU behaviour")
def test_no_cpu_fallback_without_gpu(lib):
    d = _desc()
    out = ctypes.c_void_p()
    st = lib.mfbd_plan_create(ctypes.byref(out), ctypes.byref(d.desc), None)
    assert st == _lib.MFBD_ERR_UNSUPPORTED
    assert b"no CUDA device" in lib.mfbd_last_error()
    assert out.value is None


@pytest.mark.parametrize("diam,obs", [(32.0, 0.0), (28.0, 0.0), (36.0, 0.0), (21.4, 0.0), (33.0, 0.25)])
def test_pupil_and_support_match_oracle_exactly(diam, obs):
    mask, _, _, sup = mfbd.describe_object(0, 64, [diam], [5000.0], 4, 5, basis="zernike", obscuration=obs)
    om = optics.pupil_mask(64, diam, obs)
    assert np.array_equal(mask.astype(bool), om)
    osup = optics.otf_support(om)[:, :33]
    assert np.array_equal(sup.astype(bool), osup)


def test_zernike_basis_matches_oracle():
    _, bas, var, _ = mfbd.describe_object(0, 64, [28.0], [6563.0], 4, 20, basis="zernike")
    ob = optics.zernike_basis(64, 28.0, range(2, 22))
    assert np.abs(bas - ob).max() <= 4e-7 * np.abs(ob).max()
    assert np.allclose(var, optics.mode_variances("zernike", 20), rtol=1e-12)


@pytest.mark.parametrize("diam,m", [(28.0, 44), (36.0, 44), (32.0, 20)])
def test_kl_basis_matches_oracle(diam, m):
    _, bas, var, _ = mfbd.describe_object(0, 64, [diam], [6563.0], 4, m, basis="kl")
    ob, ovar, _ = optics.kl_basis(64, diam, m)
    assert np.allclose(var, ovar, rtol=1e-10)
    assert np.abs(bas - ob).max() <= 1e-6 * np.abs(ob).max()


def test_user_basis_is_passed_through():
    g = np.random.default_rng(0)
    ub = g.standard_normal((1, 3, 64, 64)).astype(np.float32)
    _, bas, var, _ = mfbd.describe_object(0, 64, [30.0], [5000.0], 2, 3, basis="user", user_basis=ub)
    assert np.array_equal(bas, ub[0])
    assert np.all(var == 0)


# ------------------------------------------ register FFTs run on the host

def _host_fft(lib, kind, x, nout):
    xin = np.ascontiguousarray(x, np.float32)
    out = np.zeros(nout, np.float32)
    assert lib.mfbd_test_fft_host(kind, xin.ctypes.data, out.ctypes.data) == 0
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_register_ffts_match_oracle(lib, seed):
    g = np.random.default_rng(seed)
    z = (g.standard_normal(64) + 1j * g.standard_normal(64)).astype(np.complex64)
    zin = np.stack([z.real, z.imag], -1).ravel()
    for kind, sign in ((0, -1), (1, +1), (5, -1), (6, +1)):
        o = _host_fft(lib, kind, zin, 128)
        ref = dft.fft_radix2(z.astype(np.complex128), sign=sign)
        got = o[0::2] + 1j * o[1::2]
        assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max()
    for kind, sign in ((7, -1), (8, +1)):  # 48 points: radix-3 stage over radix-4 16-point FFTs
        o = _host_fft(lib, kind, zin[:96], 96)
        ref = dft.dft_naive(z[:48].astype(np.complex128), sign=sign)
        assert np.abs(o[0::2] + 1j * o[1::2] - ref).max() <= 2e-6 * np.abs(ref).max()
    o = _host_fft(lib, 4, zin[:64], 64)
    ref = dft.fft_radix2(z[:32].astype(np.complex128))
    assert np.abs(o[0::2] + 1j * o[1::2] - ref).max() <= 2e-6 * np.abs(ref).max()
    r = g.standard_normal(64).astype(np.float32)
    o = _host_fft(lib, 2, r, 66)
    ref = dft.fft_radix2(r.astype(np.complex128))[:33]
    assert np.abs(o[0::2] + 1j * o[1::2] - ref).max() <= 2e-6 * np.abs(ref).max()
    # complex-to-real adjoint of a Hermitian half spectrum
    img = g.standard_normal(64)
    half = dft.fft_radix2(img.astype(np.complex128))[:33]
    hin = np.stack([half.real, half.imag], -1).ravel()
    o = _host_fft(lib, 3, hin, 64)
    full = np.concatenate([half, np.conj(half[1:32][::-1])])
    ref = dft.fft_radix2(full, sign=+1).real
    assert np.abs(o - ref).max() <= 2e-6 * np.abs(ref).max()


def test_noalloc_entry_point_checks_arguments_on_host(lib):
    """Argument checks of mfbd_phase_loss_grad_noalloc run before any CUDA
    call: bad descriptors and frame counts beyond its fixed workspace are
    rejected with MFBD_ERR_INVALID_ARG."""
    f = lib.mfbd_phase_loss_grad_noalloc
    assert f(None, None, None, None, None, None, None) == _lib.MFBD_ERR_INVALID_ARG
    d = _desc(n_frames=337)  # 1 object x 337 frames
    assert f(ctypes.byref(d.desc), None, None, None, None, None, None) == _lib.MFBD_ERR_INVALID_ARG
    assert b"static workspace" in lib.mfbd_last_error()
    d = _desc(gamma=-1.0)
    assert f(ctypes.byref(d.desc), None, None, None, None, None, None) == _lib.MFBD_ERR_INVALID_ARG
    d = _desc(n_patches=0)
    assert f(ctypes.byref(d.desc), None, None, None, None, None, None) == _lib.MFBD_OK
    d = _desc()
    assert f(ctypes.byref(d.desc), None, None, None, None, None, None) == _lib.MFBD_ERR_INVALID_ARG


# ------------------------------------------------------------ batches

def _batch_items(lib, sizes, mode, window):
    s = np.ascontiguousarray(np.array(sizes, np.int32).reshape(-1, 4))
    count = ctypes.c_longlong()
    assert lib.mfbd_test_batch_items(s.ctypes.data, len(s), mode, window, None, 0, ctypes.byref(count)) == 0
    out = np.zeros((count.value, 5), np.int32)
    assert lib.mfbd_test_batch_items(s.ctypes.data, len(s), mode, window, out.ctypes.data, count.value,
                                     ctypes.byref(count)) == 0
    return out


@pytest.mark.parametrize("mode,window", [(_lib.MFBD_BATCH_ONE_LAUNCH, 0), (_lib.MFBD_BATCH_ONE_LAUNCH, 40),
                                         (_lib.MFBD_BATCH_ONE_LAUNCH, 1), (_lib.MFBD_BATCH_STAGED, 0)])
def test_batch_work_list_covers_every_unit_once_after_its_dependencies(lib, mode, window):
    """The batch work list: one phase, reduction and modal-adjoint item per
    patch, every unit in exactly one forward and one adjoint item (groups of
    up to four units only for N <= 64 and only within one patch), and in
    one-launch mode every
    item after the items it waits for (the progress argument of the kernel)."""
    sizes = [(48, 2, 1, 5), (64, 1, 2, 4), (96, 3, 1, 3), (128, 1, 3, 2), (64, 2, 1, 1), (128, 0, 2, 3)]
    items = _batch_items(lib, sizes, mode, window)
    pos, seen_f, seen_a = {}, {}, {}
    for idx, (kind, prob, patch, kj, pair) in enumerate(items):
        n, p, k_, j_ = sizes[prob]
        assert 0 <= patch < p
        if kind in (1, 3):
            assert 0 <= pair <= 3
            if pair:
                assert n <= 64 and kj + pair < k_ * j_
            for u in range(kj, kj + 1 + pair):
                d = seen_f if kind == 1 else seen_a
                assert (prob, patch, u) not in d
                d[(prob, patch, u)] = idx
        else:
            assert (kind, prob, patch) not in pos
            pos[(kind, prob, patch)] = idx
    for prob, (n, p, k_, j_) in enumerate(sizes):
        for patch in range(p):
            for kind in (0, 2, 4):
                assert (kind, prob, patch) in pos
            for u in range(k_ * j_):
                f, a = seen_f[(prob, patch, u)], seen_a[(prob, patch, u)]
                if mode == _lib.MFBD_BATCH_ONE_LAUNCH:
                    assert pos[(0, prob, patch)] < f < pos[(2, prob, patch)] < a < pos[(4, prob, patch)]
    assert len(seen_f) == sum(p * k * j for _, p, k, j in sizes) == len(seen_a)
    if mode == _lib.MFBD_BATCH_STAGED:
        assert list(items[:, 0]) == sorted(items[:, 0])


def test_batch_create_validates_without_gpu(lib):
    out = ctypes.c_void_p()
    assert lib.mfbd_batch_create(None, None, 0, None) == _lib.MFBD_ERR_INVALID_ARG
    bad = _desc(n_pix=80, diams=[30.0])
    assert lib.mfbd_batch_create(ctypes.byref(out), ctypes.byref(bad.desc), 1, None) == _lib.MFBD_ERR_UNSUPPORTED
    bf = _desc(precision="bf16_phase")
    assert lib.mfbd_batch_create(ctypes.byref(out), ctypes.byref(bf.desc), 1, None) == _lib.MFBD_ERR_UNSUPPORTED
    fs = _desc(full_spectrum=True)
    assert lib.mfbd_batch_create(ctypes.byref(out), ctypes.byref(fs.desc), 1, None) == _lib.MFBD_ERR_UNSUPPORTED
    if not torch.cuda.is_available():
        ok = _desc()
        st = lib.mfbd_batch_create(ctypes.byref(out), ctypes.byref(ok.desc), 1, None)
        assert st in (_lib.MFBD_ERR_CUDA, _lib.MFBD_ERR_UNSUPPORTED) and not out.value


def test_uneven_problem_draws():
    from paper_2505_10639_gb300 import synth
    probs = synth.uneven_problems(20250518, 400)
    assert {p["n_pix"] for p in probs} == {48, 64, 96, 128}
    for p in probs:
        assert 1 <= p["n_objects"] <= 3 and 8 <= p["n_frames"] <= 24 and 20 <= p["n_modes"] <= 66
        assert len(p["diams"]) == p["n_objects"]
        for d, wl in zip(p["diams"], p["wavelengths"]):
            assert d % 2 == 0 and 0.35 * p["n_pix"] - 1 <= d <= 0.5 * p["n_pix"] + 1
            assert abs(d * wl - p["diams"][0] * p["wavelengths"][0]) < 1e-6 * d * wl
    assert probs == synth.uneven_problems(20250518, 400)


def test_field_front_end_refuses_without_a_plan(lib):
    assert lib.mfbd_spectra_from_frames(None, None, 96, 96, 32, 6, None, None) == _lib.MFBD_ERR_INVALID_ARG
    assert lib.mfbd_merge_objects(None, None, 96, 96, 32, 6, None, None) == _lib.MFBD_ERR_INVALID_ARG
    assert lib.mfbd_filter_objects(None, None, None, None, None) == _lib.MFBD_ERR_INVALID_ARG
    assert lib.mfbd_ls_filter_objects(None, None, None, 1.0, None, None, None) == _lib.MFBD_ERR_INVALID_ARG
    assert lib.mfbd_loss_grad_explicit(None, None, None, None, None, None, None, None) == _lib.MFBD_ERR_INVALID_ARG


def test_dictionary_model_descriptor_and_workspace(lib):
    """mfbd_dict_workspace_bytes / mfbd_dict_loss_grad validate before any
    device call: bad sizes and n != 64 are refused, an empty problem is a
    no-op, and the workspace holds P K J doubles and P K J N^2 floats."""
    d = _lib.DictDesc(64, 3, 2, 5, 4)
    units = 3 * 2 * 5
    nbytes = lib.mfbd_dict_workspace_bytes(ctypes.byref(d))
    assert nbytes >= units * 8 + units * 64 * 64 * 4 and nbytes % 4 == 0
    for bad in (_lib.DictDesc(64, -1, 2, 5, 4), _lib.DictDesc(64, 3, 0, 5, 4), _lib.DictDesc(64, 3, 2, 0, 4),
                _lib.DictDesc(64, 3, 2, 5, 0)):
        assert lib.mfbd_dict_workspace_bytes(ctypes.byref(bad)) == 0
        assert lib.mfbd_dict_loss_grad(ctypes.byref(bad), *([None] * 10)) == 1  # MFBD_ERR_INVALID_ARG
    assert lib.mfbd_dict_loss_grad(None, *([None] * 10)) == 1
    assert lib.mfbd_dict_loss_grad(ctypes.byref(_lib.DictDesc(48, 3, 2, 5, 4)), *([None] * 10)) == 2  # UNSUPPORTED
    assert lib.mfbd_dict_loss_grad(ctypes.byref(_lib.DictDesc(64, 0, 2, 5, 4)), *([None] * 10)) == 0  # empty
    assert lib.mfbd_dict_loss_grad(ctypes.byref(d), *([None] * 10)) == 1  # NULL inputs
