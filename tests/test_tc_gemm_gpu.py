"""The two modal projections on the tensor cores (phase projection phi =
c_k B_k a, Eq. 22, and the modal adjoint dL/da = sum_k c_k B_k^T dL/dphi)
at the edges of their tiling, against the SIMT kernels and the oracle.

Cases: three objects in one launch with 21 modes (the tensor-core tiles pad
the modes to 32, and the adjoint's epilogue takes the scalar path because
21 is not a multiple of 4); 100 modes over 360 units (three unit tiles, the
last ragged) with a 40 px pupil (a box too wide for the fused kernel: the
three-kernel path); 250 modes (the widest MMA tile, N = 256, and the
shallowest pipeline); one patch of 6 units (one unit tile, mostly empty).
In FP32 the phase projection's three-plane tiles fit shared memory up to 80
modes; beyond, it runs on the SIMT kernel while the adjoint stays on the
tensor cores.
"""

import numpy as np
import pytest
import torch

from oracle import mfbd as omfbd
from oracle import optics
from tests import cases

pytestmark = pytest.mark.gpu

# tensor-core (three BF16 planes) against SIMT FP32 projections: the same
# bounds as the projection test of test_parity_gpu.py
PROJ_LOSS_RTOL = 1e-5
PROJ_GRAD_RTOL = 1e-4
# against the FP64 oracle (the FP32 path's bounds)
LOSS_RTOL = 1e-5
GRAD_RTOL = 1e-4
OBJ_RTOL = 1e-4


def _plans(diams, n_modes, n_patches, n_frames):
    from paper_2505_10639_gb300.mfbd import Plan
    wl = [6563.0 * diams[0] / d for d in diams]  # pupil diameter inversely proportional to the wavelength
    args = (64, n_patches, list(diams), wl, n_frames, n_modes)
    return Plan(*args, basis="zernike"), Plan(*args, basis="zernike", projection="simt")


def _random_inputs(plan, seed):
    """Seeded coefficients (0.1 rad per mode) and complex spectra; the loss
    and its gradient are defined for any data."""
    g = torch.Generator().manual_seed(seed)
    a = 0.1 * torch.randn(plan.coeff_shape(), generator=g, dtype=torch.float32)
    shape = plan.spectra_shape()
    d = torch.complex(torch.randn(shape, generator=g), torch.randn(shape, generator=g)).to(torch.complex64)
    return a.cuda(), d.cuda()


@pytest.mark.parametrize("diams,n_modes,n_patches,n_frames", [
    ((36.0, 30.0, 24.0), 21, 11, 5),
    ((40.0,), 100, 30, 12),
    ((32.0, 26.0), 250, 4, 8),
    ((36.0,), 64, 1, 6),
])
def test_tensor_core_projections_match_simt(diams, n_modes, n_patches, n_frames):
    pt, ps = _plans(diams, n_modes, n_patches, n_frames)
    it, is_ = pt.info(), ps.info()
    assert it["tc_projection"] == (1 if n_modes <= 80 else 0) and it["tc_adjoint"] == 1
    assert is_["tc_projection"] == 0 and is_["tc_adjoint"] == 0
    a, d = _random_inputs(pt, seed=20250601 + n_modes)
    lt, gt, _ = pt.loss_grad(a, d)
    ls, gs, _ = ps.loss_grad(a, d)
    torch.cuda.synchronize()
    lt, gt, ls, gs = lt.cpu().numpy(), gt.cpu().numpy(), ls.cpu().numpy(), gs.cpu().numpy()
    assert np.all(np.isfinite(gt)) and np.all(np.isfinite(lt))
    el = np.max(np.abs(lt - ls) / np.abs(ls))
    eg = max(np.linalg.norm(gt[p] - gs[p]) / np.linalg.norm(gs[p]) for p in range(n_patches))
    print("%s modes %d: tensor vs SIMT loss %.2e grad %.2e" % (diams, n_modes, el, eg))
    assert el <= PROJ_LOSS_RTOL and eg <= PROJ_GRAD_RTOL, (el, eg)


def test_three_objects_in_one_launch_against_oracle():
    """Three objects (36, 30 and 24 px pupils) of 21 Zernike modes through
    the tensor-core projections, against the FP64 oracle."""
    case = cases.make_case(diams=(36.0, 30.0, 24.0), wavelengths=(6563.0, 7876.0, 9845.0), n_frames=5,
                           n_modes=21, basis="zernike", n_patches=3, seed=20250602)
    from paper_2505_10639_gb300.mfbd import Plan
    s = case["setup"]
    plan = Plan(64, 3, list(case["diams"]), list(case["wavelengths"]), case["n_frames"], case["n_modes"],
                basis="zernike", gamma=s.gamma, weights=s.weights)
    assert plan.info()["tc_projection"] == 1 and plan.info()["tc_adjoint"] == 1
    a32 = case["a_eval"].astype(np.float32)
    d32 = omfbd.half_spectrum(case["d"]).astype(np.complex64)
    d_or = omfbd.full_from_half(d32.astype(np.complex128), 64)
    loss, grad, obj = plan.loss_grad(torch.from_numpy(a32).cuda(), torch.from_numpy(d32).cuda(), want_object=True)
    torch.cuda.synchronize()
    loss, grad = loss.cpu().numpy(), grad.cpu().numpy()
    obj = obj.cpu().numpy().astype(np.complex128)
    lo, oo, go = omfbd.loss_object_grad(s, a32.astype(np.float64), d_or)
    for p in range(3):
        assert abs(loss[p] - lo[p]) <= LOSS_RTOL * abs(lo[p]), (p, loss[p], lo[p])
        err = np.linalg.norm(grad[p] - go[p]) / np.linalg.norm(go[p])
        assert err <= GRAD_RTOL, (p, err)
        for k, mask in enumerate(s.masks):
            supp = optics.otf_support(mask)
            of = omfbd.full_from_half(obj[p, k], 64)
            e = np.linalg.norm((of - oo[p][k])[supp]) / np.linalg.norm(oo[p][k][supp])
            assert e <= OBJ_RTOL, (p, k, e)
