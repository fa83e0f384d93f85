"""GPU parity of uneven batches (mfbd_batch_*): several problems of
different patch sizes, objects, frames and modes in one persistent launch,
against the FP64 oracle problem by problem, and against the single-problem
plan path on a larger batch drawn like the 2000-problem workload.

Tolerances are those of the plan path: loss 1e-5 relative per patch, dL/da
1e-4 norm-wise per patch, object 1e-4 norm-wise over the OTF support.
"""

import numpy as np
import pytest
import torch

from oracle import mfbd as omfbd
from oracle import optics
from paper_2505_10639_gb300 import synth
from tests import cases

pytestmark = pytest.mark.gpu

LOSS_RTOL = 1e-5
GRAD_RTOL = 1e-4
OBJ_RTOL = 1e-4

# (n_pix, diams, wavelengths, frames, modes, basis, patches, weights)
SMALL = [
    (48, (20.0,), (8542.0,), 3, 8, "zernike", 2, None),
    (64, (28.0, 24.0), (6563.0, 8542.0), 4, 10, "kl", 1, None),
    (96, (40.0,), (6563.0,), 3, 12, "zernike", 1, None),
    (128, (56.0, 44.0), (6563.0, 8542.0), 2, 9, "zernike", 1, None),
    (64, (30.0,), (8542.0,), 5, 7, "zernike", 1, np.array([[1.0, 0.5, 2.0, 1.5, 0.75]])),
]


@pytest.fixture(scope="module")
def small_batch():
    data = []
    for i, (n, diams, wl, j, m, basis, p, w) in enumerate(SMALL):
        case = cases.make_case(n_pix=n, diams=diams, wavelengths=wl, n_frames=j, n_modes=m, basis=basis,
                               n_patches=p, weights=w, seed=20250530 + i)
        a32 = case["a_eval"].astype(np.float32)
        d32 = omfbd.half_spectrum(case["d"]).astype(np.complex64)
        d_or = omfbd.full_from_half(d32.astype(np.complex128), n)
        ref = omfbd.loss_object_grad(case["setup"], a32.astype(np.float64), d_or)
        data.append((case, a32, d32, ref))
    return data


def _make_batch(data):
    from paper_2505_10639_gb300.mfbd import Batch, Problem
    probs = [Problem(c["n_pix"], a.shape[0], c["diams"], c["wavelengths"], c["n_frames"], c["n_modes"],
                     basis=c["basis"], gamma=c["setup"].gamma,
                     weights=None if np.all(c["setup"].weights == 1) else c["setup"].weights)
             for c, a, d, _ in data]
    b = Batch(probs)
    coeffs = Batch.pack([torch.from_numpy(a).cuda() for _, a, _, _ in data])
    spectra = Batch.pack([torch.from_numpy(d).cuda() for _, _, d, _ in data])
    return b, coeffs, spectra


def _run(b, coeffs, spectra):
    loss, grad, obj = b.loss_grad(coeffs, spectra, want_object=True)
    b.check()
    return loss, grad, obj


def test_small_uneven_batch_against_oracle(small_batch):
    b, coeffs, spectra = _make_batch(small_batch)
    loss, grad, obj = _run(b, coeffs, spectra)
    ls, gs, os_ = b.unpack(loss, "loss"), b.unpack(grad, "grad"), b.unpack(obj, "object")
    for i, (case, a32, d32, (lo, oo, go)) in enumerate(small_batch):
        n = case["n_pix"]
        l, g, o = ls[i].cpu().numpy(), gs[i].cpu().numpy(), os_[i].cpu().numpy()
        for p in range(a32.shape[0]):
            assert abs(l[p] - lo[p]) <= LOSS_RTOL * abs(lo[p]), (i, p, l[p], lo[p])
            eg = np.linalg.norm(g[p] - go[p]) / np.linalg.norm(go[p])
            assert eg <= GRAD_RTOL, (i, p, eg)
            for k, mask in enumerate(case["setup"].masks):
                supp = optics.otf_support(mask)
                of = omfbd.full_from_half(o[p, k].astype(np.complex128), n)
                eo = np.linalg.norm((of - oo[p][k])[supp]) / np.linalg.norm(oo[p][k][supp])
                assert eo <= OBJ_RTOL, (i, p, k, eo)


def test_schedules_graph_and_autotune_give_the_same_bits(small_batch):
    """Every item computes the same arithmetic whatever the schedule: one
    launch with any window, staged launches, either kernel variant (register
    budget), a CUDA-graph replay and the autotuned schedule all give
    identical bits."""
    b, coeffs, spectra = _make_batch(small_batch)
    ref = [t.cpu() for t in _run(b, coeffs, spectra)]
    for mode, window, cps, var in (("one_launch", 0, 0, 0), ("one_launch", 1, 1, 0), ("one_launch", 100000, 0, 0),
                                   ("staged", 0, 0, 0), ("one_launch", 8192, 0, 1), ("staged", 0, 0, 1)):
        b.set_schedule(mode, window, cps, var)
        out = _run(b, coeffs, spectra)
        for x, y in zip(out, ref):
            assert torch.equal(x.cpu(), y), (mode, window, cps, var)
    loss, grad, obj = b.outputs(want_object=True)
    graph = b.capture(coeffs, spectra, loss, grad, obj)
    for _ in range(2):
        loss.zero_()
        graph.replay()
    b.check()
    assert torch.equal(loss.cpu(), ref[0]) and torch.equal(grad.cpu(), ref[1]) and torch.equal(obj.cpu(), ref[2])
    info = b.autotune(coeffs, spectra, loss, grad, obj, reps=1)
    assert info["mode"] in (0, 1)
    out = _run(b, coeffs, spectra)
    assert torch.equal(out[0].cpu(), ref[0]) and torch.equal(out[1].cpu(), ref[1])


def test_batch_otf_matches_plan_otf(small_batch):
    from paper_2505_10639_gb300.mfbd import Plan
    b, coeffs, _ = _make_batch(small_batch)
    hs = b.unpack(b.otf(coeffs), "spectra")
    for i, (case, a32, _, _) in enumerate(small_batch):
        plan = Plan(case["n_pix"], a32.shape[0], list(case["diams"]), list(case["wavelengths"]),
                    case["n_frames"], case["n_modes"], basis=case["basis"], gamma=case["setup"].gamma)
        hp = plan.otf(torch.from_numpy(a32).cuda())
        assert (hs[i] - hp).abs().max().item() <= 2e-6, i


def test_batch_of_uneven_draws_against_plans():
    """24 problems drawn like the 2000-problem workload (patch sizes 48-128,
    1-3 objects, 8-24 frames, 20-66 Zernike modes), spectra from the
    library's own OTFs: each problem's loss, dL/da and object against a plan
    of that problem alone (SIMT FP32 phase projection, like the batch), within
    the oracle tolerances."""
    from paper_2505_10639_gb300.mfbd import Batch, Plan, Problem
    spec = synth.uneven_problems(20250518, 24)
    probs = [Problem(s["n_pix"], 1, s["diams"], s["wavelengths"], s["n_frames"], s["n_modes"], basis="zernike",
                     gamma=1e-3 * s["n_pix"] ** 2 * 1e-6) for s in spec]
    b = Batch(probs)
    coeffs, spectra = [], []
    for i, (s, pr) in enumerate(zip(spec, probs)):
        var = optics.mode_variances("zernike", s["n_modes"])
        a_true = synth.kolmogorov_coeffs(20250518, var, 5.0, (1, s["n_frames"]), sub=2 * i).astype(np.float32)
        a_eval = a_true + 0.3 * synth.kolmogorov_coeffs(20250518, var, 5.0, (1, s["n_frames"]), sub=2 * i + 1)
        plan = Plan(s["n_pix"], 1, s["diams"], s["wavelengths"], s["n_frames"], s["n_modes"], basis="zernike",
                    gamma=pr.gamma)
        h = plan.otf(torch.from_numpy(a_true).cuda())
        o = torch.from_numpy(synth.object_field(20250518, (1, pr.n_objects, s["n_pix"], s["n_pix"]), sub=i)).cuda()
        nz = torch.from_numpy(synth.noise(20250518, (1, pr.n_objects, s["n_frames"], s["n_pix"], s["n_pix"]), 1e-3,
                                          sub=i)).cuda()
        d = (torch.fft.rfft2(o)[:, :, None] * h + torch.fft.rfft2(nz)).to(torch.complex64)
        coeffs.append(torch.from_numpy(a_eval.astype(np.float32)).cuda())
        spectra.append(d.contiguous())
    loss, grad, obj = _run(b, Batch.pack(coeffs), Batch.pack(spectra))
    ls, gs, os_ = b.unpack(loss, "loss"), b.unpack(grad, "grad"), b.unpack(obj, "object")
    for i, (s, pr) in enumerate(zip(spec, probs)):
        plan = Plan(s["n_pix"], 1, s["diams"], s["wavelengths"], s["n_frames"], s["n_modes"], basis="zernike",
                    gamma=pr.gamma, projection="simt")
        lp, gp, op = plan.loss_grad(coeffs[i], spectra[i], want_object=True)
        assert abs(ls[i].item() - lp.item()) <= LOSS_RTOL * abs(lp.item()), i
        assert (gs[i] - gp).norm().item() <= GRAD_RTOL * gp.norm().item(), i
        assert (os_[i] - op).abs().max().item() <= OBJ_RTOL * op.abs().max().item(), i
    assert b.info()["n_units"] == sum(pr.n_objects * pr.n_frames for pr in probs)


def test_empty_batch_and_patchless_problem():
    from paper_2505_10639_gb300.mfbd import Batch, Problem
    b = Batch([])
    assert b.info()["n_items"] == 0
    b2 = Batch([Problem(64, 0, [30.0], [8542.0], 4, 6), Problem(48, 1, [20.0], [8542.0], 2, 5)])
    inf = b2.info()
    assert inf["n_patches"] == 1 and inf["n_units"] == 2
