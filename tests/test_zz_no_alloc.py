"""The allocation-free entry point mfbd_phase_loss_grad_noalloc.

It serves callers that cannot allocate device memory and so cannot create a
plan; its working memory is a fixed array inside the library. This test
calls it through the C ABI twice in a row and checks both results against
the plan-based mfbd_loss_grad on the same problem: the loss and the object
directly, and dL/dphi by projecting it onto the modes (dL/da = sum_k c_k
B_k^T dL/dphi_k) with the library's own basis.

The file is named to be collected last, so that a failure here cannot stop a
run before the other tests.
"""

import ctypes

import numpy as np
import pytest
import torch

from oracle import mfbd as omfbd
from paper_2505_10639_gb300 import _lib
from paper_2505_10639_gb300.mfbd import Plan, _Desc, describe_object
from tests import cases

pytestmark = pytest.mark.gpu


def _full_grid_phase(a32, diams, wavelengths, n_frames, n_modes, basis):
    """phi[k, p, j] = c_k sum_m a[p, j, m] B_k[m] on the 64 x 64 grid."""
    phis, bases = [], []
    for k in range(len(diams)):
        _, b, _, _ = describe_object(k, 64, list(diams), list(wavelengths), n_frames, n_modes, basis=basis)
        c = wavelengths[0] / wavelengths[k]
        phis.append(c * np.tensordot(a32.astype(np.float64), b.astype(np.float64), axes=(-1, 0)))
        bases.append((c, b.astype(np.float64)))
    return np.ascontiguousarray(np.array(phis), dtype=np.float32), bases


def _noalloc(d, phase, spectra, want_object):
    lib = _lib.load()
    P = d.desc.n_patches
    K, J = d.desc.n_objects, d.desc.n_frames
    loss = torch.full((P,), float("nan"), dtype=torch.float64, device="cuda")
    gphi = torch.full((K, P, J, 64, 64), float("nan"), dtype=torch.float32, device="cuda")
    obj = torch.zeros((P, K, 64, 33), dtype=torch.complex64, device="cuda") if want_object else None
    st = lib.mfbd_phase_loss_grad_noalloc(
        ctypes.byref(d.desc), ctypes.c_void_p(phase.data_ptr()), ctypes.c_void_p(spectra.data_ptr()),
        ctypes.c_void_p(loss.data_ptr()), ctypes.c_void_p(obj.data_ptr()) if obj is not None else None,
        ctypes.c_void_p(gphi.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == _lib.MFBD_OK, lib.mfbd_last_error()
    torch.cuda.synchronize()
    return loss.cpu().numpy(), gphi.cpu().numpy(), (obj.cpu().numpy() if obj is not None else None)


@pytest.mark.parametrize("kind", ["two_objects_kl", "single_patch", "two_objects_20_patches",
                                  "one_object_300_frames"])
def test_noalloc_matches_plan_path_twice(kind):
    """The patches go through the static array in batches: 14 patches per
    batch at 2 objects x 12 frames, so 20 patches take two batches (14 + 6),
    and one patch per batch at 1 object x 300 frames, so 3 patches take
    three; both check every per-batch offset against the one-launch plan."""
    if kind == "single_patch":
        case = cases.single_patch_64px()
    elif kind == "one_object_300_frames":
        case = cases.make_case(diams=(32.0,), wavelengths=(8542.0,), n_frames=300, n_modes=20,
                               basis="zernike", n_patches=3, seed=20250519)
    else:
        case = cases.make_case(diams=(36.0, 28.0), wavelengths=(6563.0, 8542.0), n_frames=12, n_modes=44,
                               basis="kl", n_patches=20 if kind == "two_objects_20_patches" else 3,
                               seed=20250517)
    s = case["setup"]
    P, K, J, M = case["d"].shape[0], len(case["diams"]), case["n_frames"], case["n_modes"]
    a32 = case["a_eval"].astype(np.float32)
    d32 = omfbd.half_spectrum(case["d"]).astype(np.complex64)
    a = torch.from_numpy(a32).cuda()
    dd = torch.from_numpy(d32).cuda()

    plan = Plan(64, P, list(case["diams"]), list(case["wavelengths"]), J, M, basis=case["basis"],
                gamma=s.gamma)
    l_ref, g_ref, o_ref = plan.loss_grad(a, dd, want_object=True)
    torch.cuda.synchronize()
    l_ref, g_ref, o_ref = l_ref.cpu().numpy(), g_ref.cpu().numpy(), o_ref.cpu().numpy()
    plan.close()

    phase_np, bases = _full_grid_phase(a32, case["diams"], case["wavelengths"], J, M, case["basis"])
    phase = torch.from_numpy(phase_np).cuda()
    d = _Desc(64, P, list(case["diams"]), list(case["wavelengths"]), J, M, case["basis"], s.gamma, None,
              0.0, None, "fp32", False)
    for call in range(2):
        loss, gphi, obj = _noalloc(d, phase, dd, want_object=True)
        assert np.all(np.isfinite(loss)) and np.all(np.isfinite(gphi)), call
        assert np.all(np.abs(loss - l_ref) <= 1e-5 * np.abs(l_ref)), (call, loss, l_ref)
        for k, mask in enumerate(s.masks):
            assert np.all(gphi[k][:, :, ~mask] == 0.0)
            num = np.linalg.norm(obj[:, k] - o_ref[:, k])
            assert num <= 1e-4 * np.linalg.norm(o_ref[:, k]), (call, k)
        g_a = sum(c * np.tensordot(gphi[k].astype(np.float64), b, axes=([2, 3], [1, 2]))
                  for k, (c, b) in enumerate(bases))
        for p in range(P):
            err = np.linalg.norm(g_a[p] - g_ref[p]) / np.linalg.norm(g_ref[p])
            assert err <= 1e-4, (call, p, err)
