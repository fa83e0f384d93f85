"""Python binding of the MOMFBD C ABI (argument marshalling only).

Every call forwards torch tensors' device pointers and the current CUDA
stream to ``libmfbd.so``; all arithmetic runs in the library's kernels.
Names follow the C ABI: ``Plan.forward`` -> ``mfbd_forward`` and so on.
"""

import ctypes

import numpy as np
import torch

from . import _lib

_BASIS = {"zernike": _lib.MFBD_BASIS_ZERNIKE, "kl": _lib.MFBD_BASIS_KL, "user": _lib.MFBD_BASIS_USER}
_PREC = {"fp32": _lib.MFBD_PREC_FP32, "bf16_phase": _lib.MFBD_PREC_BF16_PHASE}
KERNEL_KINDS = ("phase", "forward", "reduction", "adjoint", "grad", "fused")


def _fptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype)) if a is not None else None


class _Desc:
    """A PlanDesc plus the host arrays it points into (kept alive)."""

    def __init__(self, n_pix, n_patches, diams, wavelengths, n_frames, n_modes, basis, gamma,
                 weights, obscuration, user_basis, precision, full_spectrum, projection="tensor",
                 recompute=False, generic=False, split=False):
        if projection not in ("tensor", "simt"):
            raise ValueError("projection must be 'tensor' or 'simt'")
        k = len(diams)
        self.diams = np.ascontiguousarray(diams, dtype=np.float32)
        self.wl = np.ascontiguousarray(wavelengths, dtype=np.float64)
        self.weights = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32).reshape(k, n_frames)
        self.user = None if user_basis is None else np.ascontiguousarray(user_basis, dtype=np.float32)
        self.desc = _lib.PlanDesc(
            n_pix=n_pix, n_patches=n_patches, n_objects=k, n_frames=n_frames, n_modes=n_modes,
            pupil_diam_px=_fptr(self.diams, ctypes.c_float), wavelength=_fptr(self.wl, ctypes.c_double),
            central_obscuration=obscuration, basis=_BASIS[basis],
            user_basis=_fptr(self.user, ctypes.c_float), gamma=gamma,
            frame_weight=_fptr(self.weights, ctypes.c_float), precision=_PREC[precision],
            flags=(_lib.MFBD_FLAG_FULL_SPECTRUM if full_spectrum else 0)
            | (_lib.MFBD_FLAG_SIMT_PROJECTION if projection == "simt" else 0)
            | (_lib.MFBD_FLAG_RECOMPUTE_BACKWARD if recompute else 0)
            | (_lib.MFBD_FLAG_GENERIC_KERNELS if generic else 0)
            | (_lib.MFBD_FLAG_SPLIT_PASSES if split else 0))


def describe_object(obj, n_pix, diams, wavelengths, n_frames, n_modes, basis="kl", gamma=1e-3,
                    obscuration=0.0, user_basis=None):
    """Host-only plan-time data of object ``obj`` (mfbd_describe_object):
    (mask [N,N] uint8, basis [M,N,N] float32, variance [M], support [N,N/2+1])."""
    lib = _lib.load()
    d = _Desc(n_pix, 1, diams, wavelengths, n_frames, n_modes, basis, gamma, None, obscuration,
              user_basis, "fp32", False)
    mask = np.zeros((n_pix, n_pix), np.uint8)
    bas = np.zeros((n_modes, n_pix, n_pix), np.float32)
    var = np.zeros(n_modes, np.float64)
    sup = np.zeros((n_pix, n_pix // 2 + 1), np.uint8)
    _lib.check(lib.mfbd_describe_object(ctypes.byref(d.desc), obj, mask.ctypes.data, bas.ctypes.data,
                                        var.ctypes.data, sup.ctypes.data), "mfbd_describe_object")
    return mask, bas, var, sup


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _host(t, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or t.device.type != "cpu":
        raise ValueError("%s must be a CPU tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


def _dev(t, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """An mfbd plan: fixed sizes, pupils, bases and workspaces on one GPU.

    coeffs  [P, J, M] float32 (radians at wavelengths[0])
    spectra [P, K, J, N, N//2+1] complex64 (or [.., N, N] with full_spectrum)
    """

    def __init__(self, n_pix, n_patches, diams, wavelengths, n_frames, n_modes, basis="kl",
                 gamma=1e-3, weights=None, obscuration=0.0, user_basis=None, precision="fp32",
                 full_spectrum=False, projection="tensor", recompute=False, generic=False, split=False,
                 stream=None):
        self._lib = _lib.load()
        self._d = _Desc(n_pix, n_patches, diams, wavelengths, n_frames, n_modes, basis, gamma, weights,
                        obscuration, user_basis, precision, full_spectrum, projection, recompute, generic, split)
        self.n_pix, self.n_patches, self.n_objects = n_pix, n_patches, len(diams)
        self.n_frames, self.n_modes = n_frames, n_modes
        self.full_spectrum = full_spectrum
        self.device = torch.device("cuda", torch.cuda.current_device())
        handle = ctypes.c_void_p()
        _lib.check(self._lib.mfbd_plan_create(ctypes.byref(handle), ctypes.byref(self._d.desc),
                                              _stream(stream)), "mfbd_plan_create")
        self._h = handle

    # ------------------------------------------------------------ shapes
    @property
    def spec_cols(self):
        return self.n_pix if self.full_spectrum else self.n_pix // 2 + 1

    def coeff_shape(self):
        return (self.n_patches, self.n_frames, self.n_modes)

    def spectra_shape(self):
        return (self.n_patches, self.n_objects, self.n_frames, self.n_pix, self.spec_cols)

    def object_shape(self):
        return (self.n_patches, self.n_objects, self.n_pix, self.spec_cols)

    def otf_shape(self):
        return (self.n_patches, self.n_objects, self.n_frames, self.n_pix, self.n_pix // 2 + 1)

    def info(self):
        inf = _lib.PlanInfo()
        _lib.check(self._lib.mfbd_plan_get_info(self._h, ctypes.byref(inf)), "mfbd_plan_get_info")
        k = self.n_objects
        return dict(pupil_pixels=list(inf.pupil_pixels[:k]), pupil_box=list(inf.pupil_box[:k]),
                    workspace_bytes=inf.workspace_bytes, slots_per_cta=inf.slots_per_cta, ctas=inf.ctas,
                    reduction_split=inf.reduction_split, fused_ctas=inf.fused_ctas,
                    tc_projection=inf.tc_projection, tc_adjoint=inf.tc_adjoint)

    # ------------------------------------------------------------ calls
    def forward(self, coeffs, spectra, loss=None, obj=None, want_object=True, stream=None):
        """mfbd_forward -> (loss [P] float64, object or None)."""
        if loss is None:
            loss = torch.empty(self.n_patches, dtype=torch.float64, device=self.device)
        if obj is None and want_object:
            obj = torch.empty(self.object_shape(), dtype=torch.complex64, device=self.device)
        _lib.check(self._lib.mfbd_forward(
            self._h, _dev(coeffs, torch.float32, self.coeff_shape(), "coeffs"),
            _dev(spectra, torch.complex64, self.spectra_shape(), "spectra"),
            _dev(loss, torch.float64, (self.n_patches,), "loss"),
            _dev(obj, torch.complex64, self.object_shape(), "object") if obj is not None else None,
            _stream(stream)), "mfbd_forward")
        return loss, obj

    def backward(self, grad=None, stream=None):
        """mfbd_backward -> dL/da [P, J, M] float32."""
        if grad is None:
            grad = torch.empty(self.coeff_shape(), dtype=torch.float32, device=self.device)
        _lib.check(self._lib.mfbd_backward(self._h, _dev(grad, torch.float32, self.coeff_shape(), "grad"),
                                           _stream(stream)), "mfbd_backward")
        return grad

    def loss_grad(self, coeffs, spectra, loss=None, grad=None, obj=None, want_object=False, stream=None):
        """mfbd_loss_grad -> (loss, grad, object or None)."""
        if loss is None:
            loss = torch.empty(self.n_patches, dtype=torch.float64, device=self.device)
        if grad is None:
            grad = torch.empty(self.coeff_shape(), dtype=torch.float32, device=self.device)
        if obj is None and want_object:
            obj = torch.empty(self.object_shape(), dtype=torch.complex64, device=self.device)
        _lib.check(self._lib.mfbd_loss_grad(
            self._h, _dev(coeffs, torch.float32, self.coeff_shape(), "coeffs"),
            _dev(spectra, torch.complex64, self.spectra_shape(), "spectra"),
            _dev(loss, torch.float64, (self.n_patches,), "loss"),
            _dev(obj, torch.complex64, self.object_shape(), "object") if obj is not None else None,
            _dev(grad, torch.float32, self.coeff_shape(), "grad"), _stream(stream)), "mfbd_loss_grad")
        return loss, grad, obj

    def loss_grad_explicit(self, coeffs, spectra, obj, loss=None, grad=None, grad_obj=None, want_grad_object=True,
                           stream=None):
        """mfbd_loss_grad_explicit: the object-inferring loss for the given
        objects -> (loss [P], dL/da [P, J, M], dL/dconj(O) or None)."""
        if loss is None:
            loss = torch.empty(self.n_patches, dtype=torch.float64, device=self.device)
        if grad is None:
            grad = torch.empty(self.coeff_shape(), dtype=torch.float32, device=self.device)
        if grad_obj is None and want_grad_object:
            grad_obj = torch.empty(self.object_shape(), dtype=torch.complex64, device=self.device)
        _lib.check(self._lib.mfbd_loss_grad_explicit(
            self._h, _dev(coeffs, torch.float32, self.coeff_shape(), "coeffs"),
            _dev(spectra, torch.complex64, self.spectra_shape(), "spectra"),
            _dev(obj, torch.complex64, self.object_shape(), "object"),
            _dev(loss, torch.float64, (self.n_patches,), "loss"),
            _dev(grad, torch.float32, self.coeff_shape(), "grad"),
            _dev(grad_obj, torch.complex64, self.object_shape(), "grad_object") if grad_obj is not None else None,
            _stream(stream)), "mfbd_loss_grad_explicit")
        return loss, grad, grad_obj

    def loss_grad_host(self, coeffs, spectra, loss=None, grad=None, obj=None, want_object=False, n_chunks=0,
                       stream=None):
        """mfbd_loss_grad_host: the same outputs from CPU tensors (pin them for
        the copies to overlap with the kernels). Asynchronous: synchronise
        `stream` before reading the outputs or reusing the inputs."""
        pin = torch.cuda.is_available()
        if loss is None:
            loss = torch.empty(self.n_patches, dtype=torch.float64, pin_memory=pin)
        if grad is None:
            grad = torch.empty(self.coeff_shape(), dtype=torch.float32, pin_memory=pin)
        if obj is None and want_object:
            obj = torch.empty(self.object_shape(), dtype=torch.complex64, pin_memory=pin)
        _lib.check(self._lib.mfbd_loss_grad_host(
            self._h, _host(coeffs, torch.float32, self.coeff_shape(), "coeffs"),
            _host(spectra, torch.complex64, self.spectra_shape(), "spectra"),
            _host(loss, torch.float64, (self.n_patches,), "loss"),
            _host(obj, torch.complex64, self.object_shape(), "object") if obj is not None else None,
            _host(grad, torch.float32, self.coeff_shape(), "grad"), ctypes.c_int(int(n_chunks)),
            _stream(stream)), "mfbd_loss_grad_host")
        return loss, grad, obj

    def capture(self, coeffs, spectra, loss, grad, obj=None):
        """A CUDA graph of one mfbd_loss_grad on these buffers (the modal
        phase projection, the pass kernels and the modal adjoint);
        replay() re-runs it."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.loss_grad(coeffs, spectra, loss=loss, grad=grad, obj=obj, stream=side)  # warm-up
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self.loss_grad(coeffs, spectra, loss=loss, grad=grad, obj=obj)
        return graph

    def otf(self, coeffs, out=None, stream=None):
        """mfbd_otf -> H [P, K, J, N, N//2+1] complex64."""
        if out is None:
            out = torch.empty(self.otf_shape(), dtype=torch.complex64, device=self.device)
        _lib.check(self._lib.mfbd_otf(self._h, _dev(coeffs, torch.float32, self.coeff_shape(), "coeffs"),
                                      _dev(out, torch.complex64, self.otf_shape(), "otf"), _stream(stream)),
                   "mfbd_otf")
        return out

    def spectra_from_frames(self, frames, overlap, border, out=None, stream=None):
        """mfbd_spectra_from_frames: frames [K, J, H, W] float32 (device) ->
        the plan's spectra [P, K, J, N, N//2+1] (patches, mean-subtracted
        modified-Hanning apodisation, DFT)."""
        if not isinstance(frames, torch.Tensor) or frames.dim() != 4:
            raise ValueError("frames must be a [K, J, H, W] tensor")
        h, w = int(frames.shape[2]), int(frames.shape[3])
        if out is None:
            out = torch.empty(self.spectra_shape(), dtype=torch.complex64, device=self.device)
        _lib.check(self._lib.mfbd_spectra_from_frames(
            self._h, _dev(frames, torch.float32, (self.n_objects, self.n_frames, h, w), "frames"), h, w,
            int(overlap), int(border), _dev(out, torch.complex64, self.spectra_shape(), "spectra"), _stream(stream)),
            "mfbd_spectra_from_frames")
        return out

    def filter_objects(self, obj, f_lower, f_upper, stream=None):
        """mfbd_filter_objects: the top-hat / cosine Fourier filter of every
        object in place; cutoffs per object in units of the diffraction limit."""
        lo = np.ascontiguousarray(np.broadcast_to(np.asarray(f_lower, np.float32), (self.n_objects,)))
        hi = np.ascontiguousarray(np.broadcast_to(np.asarray(f_upper, np.float32), (self.n_objects,)))
        _lib.check(self._lib.mfbd_filter_objects(
            self._h, _dev(obj, torch.complex64, self.object_shape(), "object"), ctypes.c_void_p(lo.ctypes.data),
            ctypes.c_void_p(hi.ctypes.data), _stream(stream)), "mfbd_filter_objects")
        return obj

    def ls_filter_objects(self, spectra, otf, noise_power, obj=None, want_filter=True, stream=None):
        """mfbd_ls_filter_objects: the Lofdahl-Scharmer filter of every patch
        and object from the data spectra and the OTFs (mfbd_otf); multiplies
        `obj` in place when given and returns H [P, K, N, N//2+1] float32 (or
        None when want_filter is False)."""
        flt = None
        if want_filter:
            flt = torch.empty(self.object_shape()[:3] + (self.n_pix // 2 + 1,), dtype=torch.float32,
                              device=self.device)
        if obj is None and flt is None:
            raise ValueError("give obj or ask for the filter")
        _lib.check(self._lib.mfbd_ls_filter_objects(
            self._h, _dev(spectra, torch.complex64, self.spectra_shape(), "spectra"),
            _dev(otf, torch.complex64, self.otf_shape(), "otf"), ctypes.c_float(float(noise_power)),
            _dev(obj, torch.complex64, self.object_shape(), "object") if obj is not None else None,
            _dev(flt, torch.float32, tuple(flt.shape), "filter") if flt is not None else None, _stream(stream)),
            "mfbd_ls_filter_objects")
        return flt

    def merge_objects(self, obj, height, width, overlap, border, out=None, stream=None):
        """mfbd_merge_objects: patch objects [P, K, N, N//2+1] -> mosaic
        [K, height, width] float32."""
        if out is None:
            out = torch.empty((self.n_objects, height, width), dtype=torch.float32, device=self.device)
        _lib.check(self._lib.mfbd_merge_objects(
            self._h, _dev(obj, torch.complex64, self.object_shape(), "object"), int(height), int(width), int(overlap),
            int(border), _dev(out, torch.float32, (self.n_objects, height, width), "image"), _stream(stream)),
            "mfbd_merge_objects")
        return out

    def set_diversity(self, diversity, stream=None):
        """mfbd_plan_set_diversity: known phases theta [K, J, N, N] (radians,
        host array) added to every patch's wavefronts, or None to remove them."""
        if diversity is None:
            ptr, keep = None, None
        else:
            keep = np.ascontiguousarray(diversity, dtype=np.float32)
            if keep.shape != (self.n_objects, self.n_frames, self.n_pix, self.n_pix):
                raise ValueError("diversity must have shape %s" % ((self.n_objects, self.n_frames, self.n_pix,
                                                                    self.n_pix),))
            ptr = ctypes.c_void_p(keep.ctypes.data)
        _lib.check(self._lib.mfbd_plan_set_diversity(self._h, ptr, _stream(stream)), "mfbd_plan_set_diversity")

    def check(self, stream=None):
        """mfbd_plan_check: synchronise, then raise MFBDError
        (MFBD_ERR_TIMEOUT) if a bounded device-side wait gave up since the
        last check."""
        _lib.check(self._lib.mfbd_plan_check(self._h, _stream(stream)), "mfbd_plan_check")

    def set_profiling(self, enable=True, max_launches=4096):
        """mfbd_plan_set_profiling: time every kernel with CUDA events."""
        _lib.check(self._lib.mfbd_plan_set_profiling(self._h, int(enable), int(max_launches)),
                   "mfbd_plan_set_profiling")

    def read_profile(self, reset=True):
        """mfbd_plan_read_profile -> {kind: (ms, launches)} for KERNEL_KINDS."""
        ms = np.zeros(len(KERNEL_KINDS), np.float64)
        n = np.zeros(len(KERNEL_KINDS), np.int64)
        _lib.check(self._lib.mfbd_plan_read_profile(self._h, ms.ctypes.data, n.ctypes.data, int(reset)),
                   "mfbd_plan_read_profile")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_KINDS)}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mfbd_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def phase_loss_grad_noalloc(phase, spectra, n_patches, diams, n_frames, gamma, weights=None,
                            obscuration=0.0, full_spectrum=False, loss=None, grad_phase=None, obj=None,
                            want_object=False, stream=None):
    """mfbd_phase_loss_grad_noalloc: loss [P], dL/dphi [K, P, J, 64, 64] (and
    optionally the object) from full-grid phases [K, P, J, 64, 64], without a
    plan and without any device allocation by the library (the output
    tensors are the caller's)."""
    lib = _lib.load()
    k = len(diams)
    d = _Desc(64, n_patches, diams, [1.0] * k, n_frames, 1, "zernike", gamma, weights, obscuration, None,
              "fp32", full_spectrum)
    dev = phase.device
    if loss is None:
        loss = torch.empty(n_patches, dtype=torch.float64, device=dev)
    if grad_phase is None:
        grad_phase = torch.empty_like(phase)
    cols = 64 if full_spectrum else 33
    if obj is None and want_object:
        obj = torch.empty((n_patches, k, 64, cols), dtype=torch.complex64, device=dev)
    shape = (k, n_patches, n_frames, 64, 64)
    _lib.check(lib.mfbd_phase_loss_grad_noalloc(
        ctypes.byref(d.desc), _dev(phase, torch.float32, shape, "phase"),
        _dev(spectra, torch.complex64, (n_patches, k, n_frames, 64, cols), "spectra"),
        _dev(loss, torch.float64, (n_patches,), "loss"),
        _dev(obj, torch.complex64, (n_patches, k, 64, cols), "object") if obj is not None else None,
        _dev(grad_phase, torch.float32, shape, "grad_phase"), _stream(stream)), "mfbd_phase_loss_grad_noalloc")
    return loss, grad_phase, obj


def dict_loss_grad(atom_otf, gamma, obj, coeff, spectra, want_grad_object=True, want_grad_coeff=True,
                   loss=None, grad_object=None, grad_coeff=None, workspace=None, stream=None):
    """mfbd_dict_loss_grad: the spatially variant dictionary model's data term
    L [P] (float64) and its gradients dL/do [P, K, 64, 64], dL/da
    [P, K, J, M, 64, 64] for atom_otf [M, 64, 33] complex64, gamma [K, J],
    obj [P, K, 64, 64], coeff [P, K, J, M, 64, 64] float32 and spectra
    [P, K, J, 64, 33] complex64, all on the device (plan-free; the workspace
    is allocated here unless given)."""
    lib = _lib.load()
    n_atoms = int(atom_otf.shape[0])
    n_patches, k, j = int(coeff.shape[0]), int(coeff.shape[1]), int(coeff.shape[2])
    desc = _lib.DictDesc(64, n_patches, k, j, n_atoms)
    dev = coeff.device
    if loss is None:
        loss = torch.empty(n_patches, dtype=torch.float64, device=dev)
    if grad_object is None and want_grad_object:
        grad_object = torch.empty((n_patches, k, 64, 64), dtype=torch.float32, device=dev)
    if grad_coeff is None and want_grad_coeff:
        grad_coeff = torch.empty_like(coeff)
    if workspace is None:
        nbytes = int(lib.mfbd_dict_workspace_bytes(ctypes.byref(desc)))
        workspace = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=dev)
    cshape = (n_patches, k, j, n_atoms, 64, 64)
    _lib.check(lib.mfbd_dict_loss_grad(
        ctypes.byref(desc), _dev(atom_otf, torch.complex64, (n_atoms, 64, 33), "atom_otf"),
        _dev(gamma, torch.float32, (k, j), "gamma"), _dev(obj, torch.float32, (n_patches, k, 64, 64), "object"),
        _dev(coeff, torch.float32, cshape, "coeff"),
        _dev(spectra, torch.complex64, (n_patches, k, j, 64, 33), "spectra"),
        ctypes.c_void_p(workspace.data_ptr()), _dev(loss, torch.float64, (n_patches,), "loss"),
        _dev(grad_object, torch.float32, (n_patches, k, 64, 64), "grad_object") if grad_object is not None else None,
        _dev(grad_coeff, torch.float32, cshape, "grad_coeff") if grad_coeff is not None else None,
        _stream(stream)), "mfbd_dict_loss_grad")
    return loss, grad_object, grad_coeff


def probe_fma_rate(fp64=False, iters=None, stream=None):
    """mfbd_probe_fma_rate: the FP32 (or FP64) fused multiply-add rate of the
    current device, one timed launch that fills every SM; returns
    (TFLOP/s, ms, flops)."""
    lib = _lib.load()
    if iters is None:
        iters = 4000 if fp64 else 200000
    flops = ctypes.c_double(0.0)
    ms = ctypes.c_float(0.0)
    _lib.check(lib.mfbd_probe_fma_rate(1 if fp64 else 0, int(iters), _stream(stream), ctypes.byref(flops),
                                       ctypes.byref(ms)), "mfbd_probe_fma_rate")
    return flops.value / (ms.value * 1e-3) / 1e12, ms.value, flops.value


class Problem:
    """One problem of a Batch: the arguments of Plan (FP32, half spectra)."""

    def __init__(self, n_pix, n_patches, diams, wavelengths, n_frames, n_modes, basis="zernike",
                 gamma=1e-3, weights=None, obscuration=0.0, user_basis=None):
        self.n_pix, self.n_patches, self.n_frames, self.n_modes = n_pix, n_patches, n_frames, n_modes
        self.diams, self.wavelengths = list(diams), list(wavelengths)
        self.n_objects = len(diams)
        self.basis, self.gamma, self.weights, self.obscuration = basis, gamma, weights, obscuration
        self.user_basis = user_basis

    def desc(self):
        return _Desc(self.n_pix, self.n_patches, self.diams, self.wavelengths, self.n_frames, self.n_modes,
                     self.basis, self.gamma, self.weights, self.obscuration, self.user_basis, "fp32", False)

    def coeff_shape(self):
        return (self.n_patches, self.n_frames, self.n_modes)

    def spectra_shape(self):
        return (self.n_patches, self.n_objects, self.n_frames, self.n_pix, self.n_pix // 2 + 1)

    def object_shape(self):
        return (self.n_patches, self.n_objects, self.n_pix, self.n_pix // 2 + 1)


class Batch:
    """An uneven batch (mfbd_batch_*): many problems, one persistent launch.

    Buffers are flat tensors holding the problems' buffers one after the
    other (``pack`` / ``unpack`` convert from and to per-problem tensors):
    coeffs and grad float32 [coeff_floats], spectra complex64
    [spectra_complex], loss float64 [loss_doubles], object complex64
    [object_complex] (sizes from ``info()``)."""

    def __init__(self, problems, stream=None):
        self._lib = _lib.load()
        self.problems = list(problems)
        self._descs = [p.desc() for p in self.problems]
        arr = (_lib.PlanDesc * max(1, len(self._descs)))()
        for i, d in enumerate(self._descs):
            arr[i] = d.desc
        self.device = torch.device("cuda", torch.cuda.current_device())
        handle = ctypes.c_void_p()
        _lib.check(self._lib.mfbd_batch_create(ctypes.byref(handle), arr, len(self._descs), _stream(stream)),
                   "mfbd_batch_create")
        self._h = handle
        n = len(self.problems)
        self.offsets = {k: np.zeros(max(1, n), np.int64) for k in ("coeffs", "spectra", "loss", "object")}
        _lib.check(self._lib.mfbd_batch_get_offsets(self._h, self.offsets["coeffs"].ctypes.data,
                                                    self.offsets["spectra"].ctypes.data,
                                                    self.offsets["loss"].ctypes.data,
                                                    self.offsets["object"].ctypes.data), "mfbd_batch_get_offsets")
        self._info = self.info()

    def info(self):
        inf = _lib.BatchInfo()
        _lib.check(self._lib.mfbd_batch_get_info(self._h, ctypes.byref(inf)), "mfbd_batch_get_info")
        return {name: getattr(inf, name) for name, _ in _lib.BatchInfo._fields_}

    # ------------------------------------------------------------ packing
    @staticmethod
    def pack(tensors, kind=None):
        """Concatenate per-problem tensors (coeffs or spectra) into one flat tensor."""
        return torch.cat([t.reshape(-1) for t in tensors]).contiguous()

    def unpack(self, flat, kind):
        """Split a flat buffer (coeffs, grad, spectra, loss, object) into per-problem views."""
        shape_of = {"coeffs": Problem.coeff_shape, "grad": Problem.coeff_shape,
                    "spectra": Problem.spectra_shape, "object": Problem.object_shape,
                    "loss": lambda p: (p.n_patches,)}[kind]
        off = self.offsets["coeffs" if kind == "grad" else kind]
        out = []
        for i, p in enumerate(self.problems):
            shp = shape_of(p)
            n = int(np.prod(shp))
            out.append(flat[int(off[i]):int(off[i]) + n].view(shp))
        return out

    # ------------------------------------------------------------ calls
    def _bufs(self, coeffs, spectra, loss, grad, obj):
        inf = self._info
        return (_dev(coeffs, torch.float32, (inf["coeff_floats"],), "coeffs"),
                _dev(spectra, torch.complex64, (inf["spectra_complex"],), "spectra"),
                _dev(loss, torch.float64, (inf["loss_doubles"],), "loss"),
                _dev(obj, torch.complex64, (inf["object_complex"],), "object") if obj is not None else None,
                _dev(grad, torch.float32, (inf["coeff_floats"],), "grad"))

    def outputs(self, want_object=False):
        inf = self._info
        loss = torch.empty(inf["loss_doubles"], dtype=torch.float64, device=self.device)
        grad = torch.empty(inf["coeff_floats"], dtype=torch.float32, device=self.device)
        obj = (torch.empty(inf["object_complex"], dtype=torch.complex64, device=self.device)
               if want_object else None)
        return loss, grad, obj

    def loss_grad(self, coeffs, spectra, loss=None, grad=None, obj=None, want_object=False, stream=None):
        """mfbd_batch_loss_grad -> (loss, grad, object or None), flat."""
        if loss is None or grad is None or (want_object and obj is None):
            l2, g2, o2 = self.outputs(want_object and obj is None)
            loss = l2 if loss is None else loss
            grad = g2 if grad is None else grad
            obj = o2 if obj is None else obj
        a, d, lo, ob, g = self._bufs(coeffs, spectra, loss, grad, obj)
        _lib.check(self._lib.mfbd_batch_loss_grad(self._h, a, d, lo, ob, g, _stream(stream)),
                   "mfbd_batch_loss_grad")
        return loss, grad, obj

    def otf(self, coeffs, out=None, stream=None):
        """mfbd_batch_otf -> H of every problem, flat, packed like the spectra."""
        inf = self._info
        if out is None:
            out = torch.empty(inf["spectra_complex"], dtype=torch.complex64, device=self.device)
        _lib.check(self._lib.mfbd_batch_otf(self._h, _dev(coeffs, torch.float32, (inf["coeff_floats"],), "coeffs"),
                                            _dev(out, torch.complex64, (inf["spectra_complex"],), "otf"),
                                            _stream(stream)), "mfbd_batch_otf")
        return out

    def check(self, stream=None):
        """mfbd_batch_check: synchronise and raise if a dependency wait gave up."""
        _lib.check(self._lib.mfbd_batch_check(self._h, _stream(stream)), "mfbd_batch_check")

    def set_schedule(self, mode="one_launch", window_units=0, ctas_per_sm=0, variant=0):
        m = {"one_launch": _lib.MFBD_BATCH_ONE_LAUNCH, "staged": _lib.MFBD_BATCH_STAGED}[mode]
        _lib.check(self._lib.mfbd_batch_set_schedule(self._h, m, int(window_units), int(ctas_per_sm), int(variant)),
                   "mfbd_batch_set_schedule")
        self._info = self.info()

    def autotune(self, coeffs, spectra, loss, grad, obj=None, reps=2, stream=None):
        """mfbd_batch_autotune: time the candidate schedules, keep the fastest."""
        a, d, lo, ob, g = self._bufs(coeffs, spectra, loss, grad, obj)
        _lib.check(self._lib.mfbd_batch_autotune(self._h, a, d, lo, ob, g, int(reps), _stream(stream)),
                   "mfbd_batch_autotune")
        self._info = self.info()
        return self._info

    def capture(self, coeffs, spectra, loss, grad, obj=None):
        """A CUDA graph of one evaluation on these buffers (the counter
        memset and the launch(es) of the current schedule); replay() re-runs
        it."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.loss_grad(coeffs, spectra, loss=loss, grad=grad, obj=obj, stream=side)  # warm-up
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self.loss_grad(coeffs, spectra, loss=loss, grad=grad, obj=obj)
        return graph

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mfbd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MOMFBDLoss(torch.autograd.Function):
    """loss[P] = MOMFBD loss of every patch as a differentiable function of
    the modal coefficients (spectra are data: no gradient).

    The forward runs mfbd_loss_grad (the fused path) and keeps dL/da with
    the node; the backward scales it by the incoming gradient. No node
    depends on the plan's state after its forward, so any number of
    evaluations on one plan may precede the backward."""

    @staticmethod
    def forward(ctx, coeffs, spectra, plan):
        loss, grad, _ = plan.loss_grad(coeffs.detach().contiguous(), spectra.detach().contiguous())
        ctx.save_for_backward(grad)
        return loss

    @staticmethod
    def backward(ctx, grad_loss):
        (g,) = ctx.saved_tensors
        return g * grad_loss.to(g.dtype)[:, None, None], None, None


def momfbd_loss(coeffs, spectra, plan):
    return MOMFBDLoss.apply(coeffs, spectra, plan)
