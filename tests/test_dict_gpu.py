"""The spatially variant dictionary PSF model (Sec. 2.2.2, "Spatially variant
convolution") through the C ABI (mfbd_dict_loss_grad) against the FP64
oracle, on the same seeded inputs (synth.dictionary_case; the library's
complex64 half spectra of the atoms and data, Hermitian-extended for the
oracle).

Bounds (FP32 transforms of 64 x 64 planes, FP64 loss sums): the patch loss
within 1e-5 relative; every gradient element within 2e-5 of the largest
magnitude of its (patch, object[, frame, atom]) block."""

import numpy as np
import pytest
import torch

from oracle import dictionary as od
from oracle import mfbd as omfbd
from paper_2505_10639_gb300 import synth

pytestmark = pytest.mark.gpu

LOSS_RTOL = 1e-5
GRAD_TOL = 2e-5


def _run(case, want_obj=True, want_coeff=True):
    from paper_2505_10639_gb300.mfbd import dict_loss_grad
    atoms, atom_otf, gamma, obj, coeff, spectra = case
    t = [torch.from_numpy(x).cuda() for x in (atom_otf, gamma, obj, coeff, spectra)]
    loss, go, ga = dict_loss_grad(*t, want_grad_object=want_obj, want_grad_coeff=want_coeff)
    torch.cuda.synchronize()
    return (loss.cpu().numpy(), go.cpu().numpy() if go is not None else None,
            ga.cpu().numpy() if ga is not None else None)


def _oracle(case, p):
    atoms, atom_otf, gamma, obj, coeff, spectra = case
    phi = omfbd.full_from_half(atom_otf.astype(np.complex128), 64)
    data = omfbd.full_from_half(spectra[p].astype(np.complex128), 64)
    return od.loss_grad(obj[p].astype(np.float64), coeff[p].astype(np.float64), phi, data,
                        gamma.astype(np.float64))


def _check(p, loss, go, ga, ref):
    lo, goo, gao = ref
    assert abs(loss[p] - lo) <= LOSS_RTOL * abs(lo), (p, loss[p], lo)
    if go is not None:
        for k in range(goo.shape[0]):
            err = np.abs(go[p, k] - goo[k]).max() / np.abs(goo[k]).max()
            assert err <= GRAD_TOL, ("dL/do", p, k, err)
    if ga is not None:
        K, J, M = gao.shape[:3]
        for k in range(K):
            for j in range(J):
                for i in range(M):
                    err = np.abs(ga[p, k, j, i] - gao[k, j, i]).max() / np.abs(gao[k, j, i]).max()
                    assert err <= GRAD_TOL, ("dL/da", p, k, j, i, err)


@pytest.mark.parametrize("P,K,J,M", [(3, 2, 3, 4), (1, 1, 1, 1), (2, 3, 2, 7)])
def test_dictionary_model_matches_oracle(P, K, J, M):
    case = synth.dictionary_case(20260101 + 7 * M + P, P, K, J, M)
    loss, go, ga = _run(case)
    assert np.all(np.isfinite(loss)) and np.all(np.isfinite(go)) and np.all(np.isfinite(ga))
    for p in range(P):
        _check(p, loss, go, ga, _oracle(case, p))


def test_dictionary_model_optional_outputs():
    """The loss alone, and each gradient alone, equal the full call's."""
    case = synth.dictionary_case(20260102, 2, 2, 2, 3)
    full = _run(case)
    only_loss = _run(case, want_obj=False, want_coeff=False)
    only_obj = _run(case, want_coeff=False)
    only_coeff = _run(case, want_obj=False)
    assert np.array_equal(only_loss[0], full[0])
    assert np.array_equal(only_obj[1], full[1]) and np.array_equal(only_coeff[2], full[2])


def test_dictionary_model_zero_residual():
    """Data made from the model itself (by the oracle, in FP64): the loss is
    at the FP32 rounding level of the data energy and the gradients small."""
    case = list(synth.dictionary_case(20260103, 1, 1, 2, 3))
    atoms, atom_otf, gamma, obj, coeff, spectra = case
    phi = omfbd.full_from_half(atom_otf.astype(np.complex128), 64)
    for j in range(2):
        spec = od.model_spectrum(obj[0, 0].astype(np.float64), coeff[0, 0, j].astype(np.float64), phi)
        spectra[0, 0, j] = spec[:, :33].astype(np.complex64)
    loss, go, ga = _run(tuple(case))
    energy = float(np.sum(np.abs(spectra.astype(np.complex128)) ** 2))
    assert loss[0] <= 1e-10 * energy, (loss[0], energy)
