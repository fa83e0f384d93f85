"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (FP32 path): loss relative 1e-5 per patch; dL/da norm-wise 1e-4
per patch; Wiener object norm-wise 1e-4 over the OTF support; OTF absolute
2e-6 (H(0) = 1). The oracle sees exactly the rounded inputs the GPU gets
(float32 coefficients, complex64 spectra).
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
# tensor-core (three BF16 planes) against SIMT FP32 phase projection
PROJ_LOSS_RTOL = 1e-5
PROJ_GRAD_RTOL = 1e-4
# BF16 phase projection (BF16 coefficients and basis, FP32 accumulation)
# (measured on the 3-patch, 2-object, 12-frame KL slice: loss 4.3e-3, dL/da
# 7.8e-3, object 5.0e-4; the bound is twice that)
BF16_LOSS_RTOL = 1e-2
BF16_GRAD_RTOL = 2e-2
BF16_OBJ_RTOL = 1e-3


def _plan_for(case, n_patches=None, full_spectrum=False, weights=None, **kw):
    from paper_2505_10639_gb300.mfbd import Plan
    s = case["setup"]
    return Plan(case["n_pix"], n_patches if n_patches is not None else case["d"].shape[0],
                list(case["diams"]), list(case["wavelengths"]), case["n_frames"], case["n_modes"],
                basis=case["basis"], gamma=s.gamma,
                weights=s.weights if weights is None else weights,
                obscuration=case["obscuration"], full_spectrum=full_spectrum, **kw)


def _inputs(case, full_spectrum=False):
    a32 = case["a_eval"].astype(np.float32)
    dfull = case["d"]
    n = case["n_pix"]
    if full_spectrum:
        d32 = dfull.astype(np.complex64)
        d_or = d32.astype(np.complex128)
    else:
        d32 = omfbd.half_spectrum(dfull).astype(np.complex64)
        d_or = omfbd.full_from_half(d32.astype(np.complex128), n)
    return a32, d32, d_or


def _oracle(case, a32, d_or):
    return omfbd.loss_object_grad(case["setup"], a32.astype(np.float64), d_or)


def _check(case, loss, grad, obj, ref, full_spectrum=False, patches=None):
    lo, oo, go = ref
    patches = range(len(lo)) if patches is None else patches
    n = case["n_pix"]
    for i, p in enumerate(patches):
        assert abs(loss[p] - lo[i]) <= LOSS_RTOL * abs(lo[i]), (p, loss[p], lo[i])
        err = np.linalg.norm(grad[p] - go[i]) / np.linalg.norm(go[i])
        assert err <= GRAD_RTOL, (p, err)
        if obj is not None:
            for k, mask in enumerate(case["setup"].masks):
                supp = optics.otf_support(mask)
                ofull = obj[p, k] if full_spectrum else omfbd.full_from_half(obj[p, k], n)
                e = np.linalg.norm((ofull - oo[i][k])[supp]) / np.linalg.norm(oo[i][k][supp])
                assert e <= OBJ_RTOL, (p, k, e)


def _run_fused(plan, a32, d32, want_object=True):
    a = torch.from_numpy(a32).cuda()
    d = torch.from_numpy(d32).cuda()
    loss, grad, obj = plan.loss_grad(a, d, want_object=want_object)
    torch.cuda.synchronize()
    return (loss.cpu().numpy(), grad.cpu().numpy(),
            obj.cpu().numpy().astype(np.complex128) if obj is not None else None)


@pytest.fixture(scope="module")
def c1():
    return cases.single_patch_64px()


@pytest.fixture(scope="module")
def c2_slice():
    # the 961-patch field's shapes: 2 objects (6563 A: 36 px pupil, 8542 A: 28 px), 12
    # frames, 44 KL modes; three patches
    return cases.make_case(diams=(36.0, 28.0), wavelengths=(6563.0, 8542.0), n_frames=12, n_modes=44,
                           basis="kl", n_patches=3, seed=20250517)


def test_single_patch_loss_object_grad(c1):
    a32, d32, d_or = _inputs(c1)
    ref = _oracle(c1, a32, d_or)
    plan = _plan_for(c1)
    loss, grad, obj = _run_fused(plan, a32, d32)
    _check(c1, loss, grad, obj, ref)


def test_single_patch_otf(c1):
    a32, _, _ = _inputs(c1)
    plan = _plan_for(c1)
    h = plan.otf(torch.from_numpy(a32).cuda()).cpu().numpy()
    inter = omfbd.otf_patch(c1["setup"], a32[0].astype(np.float64))
    href = omfbd.half_spectrum(inter[0]["H"])
    assert np.abs(h[0, 0] - href).max() <= 2e-6


def test_field_slice_loss_object_grad(c2_slice):
    a32, d32, d_or = _inputs(c2_slice)
    ref = _oracle(c2_slice, a32, d_or)
    plan = _plan_for(c2_slice)
    loss, grad, obj = _run_fused(plan, a32, d32)
    _check(c2_slice, loss, grad, obj, ref)


def test_split_forward_backward_equals_one_call(c2_slice):
    """mfbd_forward + mfbd_backward (the three kernels with the plan's
    workspaces) give the bits of mfbd_loss_grad on the same three kernels."""
    a32, d32, _ = _inputs(c2_slice)
    plan = _plan_for(c2_slice, split=True)
    assert plan.info()["fused_ctas"] == 0
    lf, gf, of = _run_fused(plan, a32, d32)
    a = torch.from_numpy(a32).cuda()
    d = torch.from_numpy(d32).cuda()
    loss, obj = plan.forward(a, d)
    grad = plan.backward()
    torch.cuda.synchronize()
    assert np.array_equal(loss.cpu().numpy(), lf)
    assert np.array_equal(grad.cpu().numpy(), gf)
    assert np.array_equal(obj.cpu().numpy().astype(np.complex128), of)


@pytest.mark.parametrize("case_name", ["c1", "c2_slice", "weights", "two_frames"])
def test_fused_kernel_matches_three_kernel_path(case_name, c1, c2_slice):
    """The fused per-(patch, object) kernel and the three-kernel path do the
    same arithmetic per frequency and per line: the object and dL/da agree
    bit for bit; the loss sums the same FP32 terms with another split into
    per-thread Kahan sums (agreement to 1e-6; up to 1.7e-8 measured at J = 2)."""
    if case_name == "c1":
        case = c1
    elif case_name == "c2_slice":
        case = c2_slice
    elif case_name == "weights":
        case = cases.make_case(diams=(36.0, 28.0), wavelengths=(6563.0, 8542.0), n_frames=7, n_modes=30,
                               basis="kl", n_patches=5, seed=20250523,
                               weights=np.linspace(0.5, 1.5, 14).reshape(2, 7))
    else:
        case = cases.make_case(diams=(30.0,), wavelengths=(8542.0,), n_frames=2, n_modes=12, n_patches=4,
                               seed=20250524)
    a32, d32, d_or = _inputs(case)
    fused = _plan_for(case)
    assert fused.info()["fused_ctas"] > 0
    split = _plan_for(case, split=True)
    lf, gf, of = _run_fused(fused, a32, d32)
    ls, gs, os_ = _run_fused(split, a32, d32)
    assert np.array_equal(gf, gs)
    assert np.array_equal(of, os_)
    assert np.all(np.abs(lf - ls) <= 1e-6 * np.abs(ls)), (lf, ls)
    _check(case, lf, gf, of, _oracle(case, a32, d_or))


def test_full_spectrum_layout(c1):
    a32, d32, d_or = _inputs(c1, full_spectrum=True)
    ref = _oracle(c1, a32, d_or)
    plan = _plan_for(c1, full_spectrum=True)
    loss, grad, obj = _run_fused(plan, a32, d32)
    _check(c1, loss, grad, obj, ref, full_spectrum=True)


@pytest.mark.parametrize("variant", ["one_frame", "weights", "ragged_pupil", "obscured", "one_mode",
                                     "many_frames"])
def test_edge_cases(variant):
    kw = dict(n_frames=4, seed=31)
    if variant == "one_frame":
        kw.update(n_frames=1)
    elif variant == "many_frames":  # more frames than the register-resident reduction holds
        kw.update(n_frames=20, n_modes=10)
    elif variant == "weights":
        kw.update(weights=[[1.0, 0.0, 2.5, 0.3]])
    elif variant == "ragged_pupil":
        kw.update(diams=(21.4,), n_modes=9)
    elif variant == "obscured":
        kw.update(diams=(40.0,), obscuration=0.3)
    elif variant == "one_mode":
        kw.update(n_modes=1)
    case = cases.make_case(**kw)
    a32, d32, d_or = _inputs(case)
    ref = _oracle(case, a32, d_or)
    plan = _plan_for(case)
    loss, grad, obj = _run_fused(plan, a32, d32)
    _check(case, loss, grad, obj, ref)


def test_zero_patches_is_a_noop():
    from paper_2505_10639_gb300.mfbd import Plan
    plan = Plan(64, 0, [32.0], [5000.0], 4, 5, basis="zernike", gamma=1e-3)
    a = torch.zeros((0, 4, 5), device="cuda")
    d = torch.zeros((0, 1, 4, 64, 33), dtype=torch.complex64, device="cuda")
    loss, grad, _ = plan.loss_grad(a, d)
    assert loss.numel() == 0 and grad.numel() == 0


def test_more_units_than_warps_and_determinism(c2_slice):
    """A ragged persistent schedule (units = patches x objects x frames not a
    multiple of the warps resident, several units per warp): every copy of a
    patch gives the same bits."""
    a32, d32, d_or = _inputs(c2_slice)
    ref = _oracle(c2_slice, a32, d_or)
    reps = 107  # 321 patches, 7704 units
    plan = _plan_for(c2_slice, n_patches=3 * reps)
    info = plan.info()
    units = 3 * reps * len(c2_slice["diams"]) * c2_slice["n_frames"]
    assert 2 * info["ctas"] * info["slots_per_cta"] < units
    assert units % (info["ctas"] * info["slots_per_cta"]) != 0
    aa = np.tile(a32, (reps, 1, 1))
    dd = np.tile(d32, (reps, 1, 1, 1, 1))
    loss, grad, obj = _run_fused(plan, aa, dd)
    loss2, grad2, _ = _run_fused(plan, aa, dd, want_object=False)
    assert np.array_equal(loss, loss2) and np.array_equal(grad, grad2)
    for r in range(reps):
        assert np.array_equal(loss[3 * r:3 * r + 3], loss[:3])
        assert np.array_equal(grad[3 * r:3 * r + 3], grad[:3])
    _check(c2_slice, loss[:3], grad[:3], obj[:3], ref)


def test_autograd_function(c1):
    from paper_2505_10639_gb300.mfbd import momfbd_loss
    a32, d32, _ = _inputs(c1)
    plan = _plan_for(c1)
    a = torch.from_numpy(a32).cuda().requires_grad_(True)
    d = torch.from_numpy(d32).cuda()
    loss = momfbd_loss(a, d, plan)
    (3.0 * loss.sum()).backward()
    _, g, _ = _run_fused(plan, a32, d32, want_object=False)
    assert np.allclose(a.grad.cpu().numpy(), 3.0 * g, rtol=1e-6, atol=0)


def test_autograd_two_forwards_before_one_backward(c2_slice):
    """Two evaluations on one plan before one backward (a loss summed over
    two evaluations): each node's gradient is that of its own inputs, not
    of the plan's last evaluation."""
    from paper_2505_10639_gb300.mfbd import momfbd_loss
    a32, d32, _ = _inputs(c2_slice)
    b32 = (a32 + 0.05 * np.sin(np.arange(a32.size, dtype=np.float32)).reshape(a32.shape)).astype(np.float32)
    plan = _plan_for(c2_slice)
    d = torch.from_numpy(d32).cuda()
    a = torch.from_numpy(a32).cuda().requires_grad_(True)
    b = torch.from_numpy(b32).cuda().requires_grad_(True)
    total = 2.0 * momfbd_loss(a, d, plan).sum() + momfbd_loss(b, d, plan).sum()
    total.backward()
    _, ga, _ = _run_fused(plan, a32, d32, want_object=False)
    _, gb, _ = _run_fused(plan, b32, d32, want_object=False)
    assert not np.allclose(ga, gb)
    assert np.array_equal(a.grad.cpu().numpy(), (2.0 * torch.from_numpy(ga)).numpy())
    assert np.array_equal(b.grad.cpu().numpy(), gb)


def test_gradient_central_differences_on_gpu(c1):
    """dL/da of the CUDA path against central differences of its own loss
    (FP32 internals: a 1e-2 rad step, 1e-2 relative agreement)."""
    a32, d32, _ = _inputs(c1)
    plan = _plan_for(c1)
    _, g, _ = _run_fused(plan, a32, d32, want_object=False)
    d = torch.from_numpy(d32).cuda()
    idx = np.argsort(-np.abs(g[0]).ravel())[:6]
    h = 1e-2
    for flat in idx:
        j, m = np.unravel_index(flat, g[0].shape)
        vals = []
        for sgn in (+1, -1):
            a = a32.copy()
            a[0, j, m] += sgn * h
            loss, _ = plan.forward(torch.from_numpy(a).cuda(), d, want_object=False)
            vals.append(loss.cpu().numpy()[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g[0, j, m]) <= 1e-2 * abs(g[0, j, m]), (j, m, fd, g[0, j, m])


@pytest.mark.parametrize("n_chunks", [1, 4, 0])
def test_host_pipeline_equals_device_call(c2_slice, n_chunks):
    """mfbd_loss_grad_host (pinned host buffers, chunked copies overlapped with
    the kernels; 10 patches in chunks of 10, 3 + 3 + 3 + 1, or the default)
    gives the bits of mfbd_loss_grad, and mfbd_backward is refused after it."""
    a32, d32, _ = _inputs(c2_slice)
    reps = 4
    aa = np.ascontiguousarray(np.tile(a32, (reps, 1, 1))[:10])
    dd = np.ascontiguousarray(np.tile(d32, (reps, 1, 1, 1, 1))[:10])
    plan = _plan_for(c2_slice, n_patches=10)
    loss, grad, obj = _run_fused(plan, aa, dd)
    ah = torch.from_numpy(aa).pin_memory()
    dh = torch.from_numpy(dd).pin_memory()
    lh, gh, oh = plan.loss_grad_host(ah, dh, want_object=True, n_chunks=n_chunks)
    torch.cuda.current_stream().synchronize()
    assert np.array_equal(lh.numpy(), loss)
    assert np.array_equal(gh.numpy(), grad)
    assert np.array_equal(oh.numpy().astype(np.complex128), obj)
    from paper_2505_10639_gb300._lib import MFBDError
    with pytest.raises(MFBDError):
        plan.backward()
    # a second call on the same plan (staging reused) without the object
    lh2, gh2, _ = plan.loss_grad_host(ah, dh, n_chunks=n_chunks)
    torch.cuda.current_stream().synchronize()
    assert np.array_equal(lh2.numpy(), loss) and np.array_equal(gh2.numpy(), grad)


def test_host_pipeline_bits_at_larger_field(c2_slice):
    """160 patches in 4 host chunks of 40: a chunk covers a quarter of the
    units, so a modal-adjoint pixel-chunk layout chosen per call would sum
    dL/da in another order than the one-call path; the plan's fixed layout
    keeps the bits equal."""
    a32, d32, _ = _inputs(c2_slice)
    reps = 54
    aa = np.ascontiguousarray(np.tile(a32, (reps, 1, 1))[:160])
    dd = np.ascontiguousarray(np.tile(d32, (reps, 1, 1, 1, 1))[:160])
    plan = _plan_for(c2_slice, n_patches=160)
    loss, grad, _ = _run_fused(plan, aa, dd, want_object=False)
    lh, gh, _ = plan.loss_grad_host(torch.from_numpy(aa).pin_memory(), torch.from_numpy(dd).pin_memory(),
                                    n_chunks=4)
    torch.cuda.current_stream().synchronize()
    assert np.array_equal(lh.numpy(), loss)
    assert np.array_equal(gh.numpy(), grad)


def test_tensor_projection_matches_simt_projection(c2_slice):
    """The FP32 phase projection and modal adjoint on the tensor cores (three
    BF16 planes per operand) and on the SIMT kernels give the same loss and
    gradient to FP32 rounding."""
    a32, d32, _ = _inputs(c2_slice)
    pt, ps = _plan_for(c2_slice), _plan_for(c2_slice, projection="simt")
    assert pt.info()["tc_projection"] == 1 and pt.info()["tc_adjoint"] == 1
    assert ps.info()["tc_projection"] == 0 and ps.info()["tc_adjoint"] == 0
    lt, gt, _ = _run_fused(pt, a32, d32, want_object=False)
    ls, gs, _ = _run_fused(ps, a32, d32, want_object=False)
    el = np.max(np.abs(lt - ls) / np.abs(ls))
    eg = max(np.linalg.norm(gt[p] - gs[p]) / np.linalg.norm(gs[p]) for p in range(len(ls)))
    print("tensor vs SIMT projection: loss %.3e grad %.3e" % (el, eg))
    assert el <= PROJ_LOSS_RTOL and eg <= PROJ_GRAD_RTOL


def test_bf16_phase_error_against_oracle(c2_slice):
    """BF16 phase projection: errors against the FP64 oracle (printed) within
    the bounds stated for the BF16-phase path."""
    a32, d32, d_or = _inputs(c2_slice)
    lo, oo, go = _oracle(c2_slice, a32, d_or)
    loss, grad, obj = _run_fused(_plan_for(c2_slice, precision="bf16_phase"), a32, d32)
    el = np.max(np.abs(loss - lo) / np.abs(lo))
    eg = max(np.linalg.norm(grad[p] - go[p]) / np.linalg.norm(go[p]) for p in range(len(lo)))
    eo = 0.0
    n = c2_slice["n_pix"]
    for p in range(len(lo)):
        for k, mask in enumerate(c2_slice["setup"].masks):
            supp = optics.otf_support(mask)
            of = omfbd.full_from_half(obj[p, k], n)
            eo = max(eo, np.linalg.norm((of - oo[p][k])[supp]) / np.linalg.norm(oo[p][k][supp]))
    print("bf16 phase: loss %.3e grad %.3e object %.3e" % (el, eg, eo))
    assert el <= BF16_LOSS_RTOL and eg <= BF16_GRAD_RTOL and eo <= BF16_OBJ_RTOL


@pytest.mark.parametrize("recompute", [False, True])
@pytest.mark.parametrize("n_pix,diams", [(48, (22.0,)), (96, (40.0, 30.0)), (128, (56.0, 44.0))])
def test_general_patch_sizes(n_pix, diams, recompute):
    """Patch sizes 48, 96 and 128 (one CTA per unit, lines over one or two
    lanes), keeping or recomputing the field for the adjoint."""
    wl = (6563.0, 8542.0)[:len(diams)]
    case = cases.make_case(n_pix=n_pix, diams=diams, wavelengths=wl, n_frames=3, n_modes=12, basis="kl",
                           n_patches=2, seed=20250518 + n_pix)
    a32, d32, d_or = _inputs(case)
    ref = _oracle(case, a32, d_or)
    plan = _plan_for(case, recompute=recompute)
    assert plan.info()["slots_per_cta"] == 0  # the general-size kernels
    loss, grad, obj = _run_fused(plan, a32, d32)
    _check(case, loss, grad, obj, ref)


@pytest.mark.parametrize("n_pix,diams", [(64, (36.0, 28.0)), (96, (40.0, 30.0))])
def test_split_frame_reduction(n_pix, diams):
    """A plan of one patch splits its frame reduction over several warps per
    object (and sums the per-split losses in a second kernel); a plan of 640
    patches does not. Patch 0 gets the same object bits from both (every
    frequency is reduced by one lane either way) and the same loss and dL/da
    to FP32 summation order."""
    case = cases.make_case(n_pix=n_pix, diams=diams, wavelengths=(6563.0, 8542.0), n_frames=3, n_modes=12,
                           basis="kl", n_patches=1, seed=20250519 + n_pix)
    a32, d32, d_or = _inputs(case)
    ref = _oracle(case, a32, d_or)
    one = _plan_for(case)
    many = _plan_for(case, n_patches=640)
    assert one.info()["reduction_split"] > 1 and many.info()["reduction_split"] == 1
    l1, g1, o1 = _run_fused(one, a32, d32)
    lm, gm, om = _run_fused(many, np.ascontiguousarray(np.tile(a32, (640, 1, 1))),
                            np.ascontiguousarray(np.tile(d32, (640, 1, 1, 1, 1))))
    assert np.array_equal(o1[0], om[0]) and np.array_equal(om[0], om[639])
    assert abs(l1[0] - lm[0]) <= 1e-6 * abs(lm[0])
    assert np.linalg.norm(g1[0] - gm[0]) <= 1e-5 * np.linalg.norm(gm[0])
    _check(case, l1, g1, o1, ref)


def test_general_kernels_match_64px_pass_machine(c2_slice):
    """N = 64 on the general-size kernels (with and without recompute)
    against the 64-pixel pass machine."""
    a32, d32, _ = _inputs(c2_slice)
    lf, gf, of = _run_fused(_plan_for(c2_slice), a32, d32)
    for rec in (False, True):
        lg, gg, og = _run_fused(_plan_for(c2_slice, generic=True, recompute=rec), a32, d32)
        assert np.all(np.abs(lg - lf) <= 2e-6 * np.abs(lf))
        for p in range(len(lf)):
            assert np.linalg.norm(gg[p] - gf[p]) <= 2e-5 * np.linalg.norm(gf[p])
        assert np.abs(og - of).max() <= 1e-5 * np.abs(of).max()


@pytest.mark.parametrize("n_pix,diams,generic", [(64, (32.0, 26.0), False), (64, (32.0, 26.0), True),
                                                 (48, (22.0,), False), (96, (40.0,), False)])
def test_phase_diversity(n_pix, diams, generic):
    """Phase diversity: a known defocus (Noll Z4, 1.5 rad) on frames 2 and 3 of
    every object, the data synthesised with it; loss, object, dL/da and the
    OTF against the oracle with the same diversity; removing it gives back the
    plain plan's bits."""
    wl = (6563.0, 8542.0)[:len(diams)]
    seed = 20250550 + n_pix
    case = cases.make_case(n_pix=n_pix, diams=diams, wavelengths=wl, n_frames=4, n_modes=10, basis="zernike",
                           n_patches=2, seed=seed)
    s = case["setup"]
    theta = []
    for d in diams:
        t = np.zeros((4, n_pix, n_pix))
        t[2:] = 1.5 * optics.zernike_basis(n_pix, d, [4])[0]
        theta.append(t)
    sd = omfbd.Setup(s.masks, s.bases, s.scales, s.weights, s.gamma, diversity=theta)
    noise = synth.noise(seed, (2, len(diams), 4, n_pix, n_pix), 1e-3)
    d = np.array([omfbd.synth_spectra(sd, case["a_true"][p], case["objects"][p], noise[p]) for p in range(2)])
    a32 = case["a_eval"].astype(np.float32)
    d32 = omfbd.half_spectrum(d).astype(np.complex64)
    d_or = omfbd.full_from_half(d32.astype(np.complex128), n_pix)
    ref = omfbd.loss_object_grad(sd, a32.astype(np.float64), d_or)
    plan = _plan_for(case, generic=generic)
    _, _, _ = _run_fused(plan, a32, d32)
    plain = _run_fused(plan, a32, d32)
    plan.set_diversity(np.array(theta, np.float32))
    loss, grad, obj = _run_fused(plan, a32, d32)
    _check(dict(case, setup=sd), loss, grad, obj, ref)
    h = plan.otf(torch.from_numpy(a32).cuda()).cpu().numpy()
    for p in range(2):
        inter = omfbd.otf_patch(sd, a32[p].astype(np.float64))
        for k in range(len(diams)):
            supp = optics.otf_support(s.masks[k])
            hk = omfbd.full_from_half(h[p, k].astype(np.complex128), n_pix)
            assert np.abs((hk - inter[k]["H"])[:, supp]).max() <= 2e-6
    plan.set_diversity(None)
    again = _run_fused(plan, a32, d32)
    for x, y in zip(again, plain):
        assert np.array_equal(x, y)


def test_lbfgs_driven_from_the_host(c2_slice):
    """torch's L-BFGS, driven from the host through the autograd function
    (the optimiser of the 961-patch workload's description), lowers the loss
    of every patch and its gradient from the evaluation point."""
    from paper_2505_10639_gb300.mfbd import momfbd_loss
    a32, d32, _ = _inputs(c2_slice)
    plan = _plan_for(c2_slice)
    d = torch.from_numpy(d32).cuda()
    a = torch.from_numpy(a32).cuda().requires_grad_(True)
    opt = torch.optim.LBFGS([a], lr=1.0, max_iter=50, history_size=10, line_search_fn="strong_wolfe")
    l0 = momfbd_loss(a, d, plan).detach().clone()

    def closure():
        opt.zero_grad()
        loss = momfbd_loss(a, d, plan).sum()
        loss.backward()
        return loss

    opt.step(closure)
    l1 = momfbd_loss(a, d, plan).detach()
    assert torch.all(l1 < 0.9 * l0), (l0, l1)


@pytest.mark.parametrize("split", [False, True])
def test_profile_counts_the_kernels_of_a_step(c2_slice, split):
    """The profiling pairs count every kernel a step launches: the
    coefficient split and one tensor-core phase projection for all objects; then
    the fused kernel (which also sums each patch's object losses), or the forward passes, the frame
    reduction and, when it is split, the loss combine, and the adjoint
    passes; and the modal adjoint GEMM and combine."""
    a32, d32, _ = _inputs(c2_slice)
    plan = _plan_for(c2_slice, split=split)
    assert plan.info()["reduction_split"] > 1  # three patches
    plan.set_profiling(True, max_launches=64)
    _run_fused(plan, a32, d32, want_object=False)
    prof = plan.read_profile(reset=True)
    counts = {k: v[1] for k, v in prof.items()}
    want = [2, 1, 2, 1, 2, 0] if split else [2, 0, 0, 0, 2, 1]
    assert list(counts.values()) == want, counts
    plan.set_profiling(False)
