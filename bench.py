#!/usr/bin/env python
"""Benchmark of the MOMFBD loss+gradient hot path on GB300.

Workload (one "step" = one loss+gradient evaluation of the whole field):
a 1024 x 1024 px field of view cut into 64 x 64 px patches at 50 % overlap
(31 x 31 = 961 patches), 2 objects (6563 A with a 36 px pupil, 8542 A with a
28 px pupil, sharing the wavefront), 12 frames, 44 KL modes, FP32 path,
through ``mfbd_loss_grad``. Inputs are seeded and synthetic: a k^-3
granulation-like object, Kolmogorov (D/r0 = 5) wavefronts, image-domain noise
sigma = 1e-3, data D = F(o (*) s + n). The spectra (390 MB) are larger than
the 129 MB L2, so no flush is needed between steps.

Metric: loss+grad evaluations per second, counted in (patch x object x frame)
units at 64 px. ``--gpus N`` runs N replicas (one per rank, each its own
field): there is no data-path collective; the value is the units all ranks
processed divided by the slowest rank's time.

``--impl reference`` times the FP64 CPU oracle on the host cores instead
(a bounded sample of the same workload).
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Workloads: the 961-patch field of 64 px patches (the headline) and the
# 3969-patch field of 128 px patches (4 objects, 32 frames, 100 KL modes,
# BF16 phase projection, field and phasors recomputed in the backward pass).
WORKLOADS = {
    "fov1024_64px": dict(workload="fov1024_64px_961patches_2obj_12frames_44kl", seed=20250517, fov=1024,
                         n_pix=64, stride=32, n_patches=961, diams=[36.0, 28.0], wavelengths=[6563.0, 8542.0],
                         n_frames=12, n_modes=44, basis="kl", d_over_r0=5.0, noise_sigma=1e-3,
                         precision="fp32", recompute=False, device_noise=False, cpu_patches=300),
    "fov4096_128px": dict(workload="fov4096_128px_3969patches_4obj_32frames_100kl", seed=20250520, fov=4096,
                          n_pix=128, stride=64, n_patches=3969, diams=[40.0, 48.0, 56.0, 64.0],
                          wavelengths=[8542.0, 8542.0 * 40 / 48, 8542.0 * 40 / 56, 8542.0 * 40 / 64],
                          n_frames=32, n_modes=100, basis="kl", d_over_r0=10.0, noise_sigma=1e-3,
                          precision="bf16_phase", recompute=True, device_noise=True, cpu_patches=16),
    "batched2000": dict(workload="batched_2000problems_48to128px_1to3obj_8to24frames_20to66zernike",
                        seed=20250518, n_problems=2000, basis="zernike", d_over_r0=5.0, noise_sigma=1e-3,
                        n_pix=64, precision="fp32", recompute=False, cpu_patches=32),
}
WORKLOAD = dict(WORKLOADS["fov1024_64px"])
SEED = WORKLOAD["seed"]  # 20250515 + workload index
FP32_LANES_PER_SM = 128
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per unit of each
# kernel of the 64 px three-kernel path, from one ncu capture of the first
# 400 patches of the 961-patch workload (9600 units), and of the fused
# kernel; a launch's traffic is this times its units (the traffic is per
# unit: no cross-unit reuse)
NCU_DRAM_BYTES_PER_UNIT = {"forward_passes": (71857152 + 503112704) / 9600,
                           "adjoint_passes": (643635200 + 32342272) / 9600,
                           "reduction": (324495360 + 115700480) / 9600,
                           # the fused kernel (pairs dealt by ticket, patch losses
                           # summed in the kernel), one capture of the full 961-patch
                           # field (23,064 units)
                           "fused_pairs": (499180288 + 113483776) / 23064}
# the same for the 128 px CTA-per-unit kernels with the field recomputed in
# the adjoint, from one capture (--metrics dram__bytes_read.sum,
# dram__bytes_write.sum) of the first 48 patches of the 3969-patch field
# (6144 units, 409 MB of spectra: larger than L2)
NCU_DRAM_BYTES_PER_UNIT_128 = {"forward_passes": (67911680 + 344916992) / 6144,
                               "adjoint_passes": (481574144 + 66861568) / 6144,
                               "reduction": (818419968 + 364834048) / 6144}
# DRAM bytes per launch of the front-end kernels on the 961-patch 64 px field
# (one ncu capture of the full launch each): spectra_tma_kernel (MemoryWorkload
# section: 3.734345 TB/s x 121.088 us); object_image_kernel + merge_kernel
# (none since the object images are stored 16 bytes at a time);
# ls_raw_kernel + ls_filter_kernel (dram__bytes_read.sum + dram__bytes_write.sum)
NCU_FRONT_DRAM_BYTES = {"spectra_from_frames": int(3.734345e12 * 121.088e-6),
                        "merge_objects": None,
                        "ls_filter_objects": 779402496 + 16724480 + 48732416 + 3328}
# DRAM bytes of the batch kernel per 64 px-equivalent unit, from one ncu
# capture of the first 200 problems of the 2000-problem batch (13869 units)
# under the schedule the autotuner picks there (one launch, window 0, the
# 170-register variant)
NCU_BATCH_DRAM_BYTES_PER_UNIT64 = (1142750976 + 911612160) / 13868.964937802688
NCU_BATCH_SCHEDULE = (0, 0, 1)  # mode, window_units, variant of that capture
METRIC = "loss+grad evals/s (patch*obj*frame units at 64px)"
UNIT = "units/s"


def gamma_of(w):
    return 1e-3 * w["n_pix"] ** 2 * w["noise_sigma"] ** 2


def units_of(w):
    return w["n_patches"] * len(w["diams"]) * w["n_frames"]


def unit_weight_64(n_pix):
    """Work of one unit at n_pix relative to one at 64 px, N^2 log2 N^2."""
    return (n_pix * n_pix * math.log2(n_pix * n_pix)) / (64 * 64 * 12.0)


def units64_of(w):
    return units_of(w) * unit_weight_64(w["n_pix"])


# ------------------------------------------------------------ distributed

def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def aggregate(local_ms, local_units, world, reduce_max=None, reduce_sum=None):
    """Whole-job figures: time = max over ranks, units = sum over ranks."""
    ms = reduce_max(local_ms) if (world > 1 and reduce_max) else local_ms
    units = reduce_sum(local_units) if (world > 1 and reduce_sum) else local_units
    return ms, units, (units / (ms * 1e-3) if ms > 0 else 0.0)


def torch_reducers():
    import torch
    import torch.distributed as dist

    dev = torch.device("cuda") if torch.cuda.is_available() and dist.get_backend() == "nccl" else torch.device("cpu")

    def rmax(v):
        t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def rsum(v):
        t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())

    return rmax, rsum


# ------------------------------------------------------------ inputs

def per_patch_draws(w, seed, p, variances):
    from paper_2505_10639_gb300 import synth
    a_true = synth.kolmogorov_coeffs(seed, variances, w["d_over_r0"], (w["n_frames"],), sub=2 * p)
    delta = synth.kolmogorov_coeffs(seed, variances, w["d_over_r0"], (w["n_frames"],), sub=2 * p + 1)
    return a_true, a_true + 0.3 * delta


def object_patches(w, seed):
    from paper_2505_10639_gb300 import synth
    field = synth.object_field(seed, (len(w["diams"]), w["fov"], w["fov"]))
    pat = synth.patches_from_field(field, w["n_pix"], w["stride"])  # [K, P, N, N]
    return np.ascontiguousarray(np.swapaxes(pat, 0, 1))[: w["n_patches"]]


def make_gpu_inputs(w, seed, chunk=256):
    """Synthetic spectra built on the GPU with the library's own OTF, chunk
    by chunk of patches (a plan of `chunk` patches makes each chunk's OTFs):
    D = F(o) H_true + F(n). The 961-patch workload draws its noise with the
    numpy generator of `synth`; the 3969-patch one (8.3e9 noise samples)
    with the seeded torch generator of `synth.noise_torch` on the device."""
    import torch
    from paper_2505_10639_gb300 import synth
    from paper_2505_10639_gb300.mfbd import Plan, describe_object
    _, _, var, _ = describe_object(0, w["n_pix"], w["diams"], w["wavelengths"], w["n_frames"],
                                   w["n_modes"], basis=w["basis"])
    P, K, J, N = w["n_patches"], len(w["diams"]), w["n_frames"], w["n_pix"]
    a_true = np.zeros((P, J, w["n_modes"]), np.float32)
    a_eval = np.zeros_like(a_true)
    for p in range(P):
        a_true[p], a_eval[p] = per_patch_draws(w, seed, p, var)
    dev = torch.device("cuda", torch.cuda.current_device())
    objs = object_patches(w, seed)
    spec = torch.empty((P, K, J, N, N // 2 + 1), dtype=torch.complex64, device=dev)
    chunk = min(chunk, P) if P > 0 else 1
    dplan = Plan(N, chunk, w["diams"], w["wavelengths"], J, w["n_modes"], basis=w["basis"], gamma=gamma_of(w))
    for p0 in range(0, P, chunk):
        n = min(chunk, P - p0)
        at = np.zeros((chunk, J, w["n_modes"]), np.float32)
        at[:n] = a_true[p0:p0 + n]
        h = dplan.otf(torch.from_numpy(at).to(dev))[:n]
        obj = torch.from_numpy(objs[p0:p0 + n]).to(dev)
        sp = torch.fft.rfft2(obj.to(torch.float64)).to(torch.complex64)[:, :, None] * h
        del h
        for q in range(n):
            p = p0 + q
            if w.get("device_noise"):
                nz = synth.noise_torch(seed, (K, J, N, N), w["noise_sigma"], sub=p, device=dev)
            else:
                nz = torch.from_numpy(synth.noise(seed, (K, J, N, N), w["noise_sigma"], sub=p)).to(dev)
            sp[q] += torch.fft.rfft2(nz).to(torch.complex64)
        spec[p0:p0 + n] = sp
        del sp
    dplan.close()
    torch.cuda.synchronize()
    return torch.from_numpy(a_eval).to(dev), spec


# ------------------------------------------------------------ clocks

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
            os.unlink(self.path)
        except Exception:
            pass
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i]
                          and not r[5 + i].startswith("Not")})
        out.update(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=reasons, samples=len(rows))
        return out


# ------------------------------------------------------------ roofline

def pass_flops_per_unit(n_pix, npup):
    """Algorithmic FP32 flops per (patch, object, frame) of the two pass
    kernels, with 2-D transforms counted at 5 N^2 log2(N^2) (complex) or half
    that (real):
      forward: pupil -> field (complex) + PSF -> OTF (real) + PSF 3 N^2;
      adjoint: OTF seed -> PSF (real) + field -> pupil (complex)
               + g_q scaling N^2 + G_p = g_q p 2 N^2 + dL/dphi 4 n_pup."""
    n2 = n_pix * n_pix
    c2 = 5.0 * n2 * math.log2(n2)
    fwd = c2 + c2 / 2 + 3 * n2
    adj = c2 / 2 + c2 + 3 * n2 + 4 * npup
    return fwd, adj


def reduction_flops_per_unit(n_pix):
    """Algorithmic FP32 flops per unit of the frame reduction, per
    half-spectrum frequency: N += w D conj(H) (8), Q += w |H|^2 (4),
    E += w |D|^2 (4), r = D - O H (8), w |r|^2 (4), seed -w conj(O) r (8)."""
    return 36.0 * n_pix * (n_pix // 2 + 1)


def reduction_bytes_per_unit(n_pix, n_frames, spec_cols):
    """Algorithmic bytes per unit of the frame reduction: D read, H read,
    G written (complex64 half spectra), object written once per J frames."""
    half = n_pix * (n_pix // 2 + 1) * 8
    return n_pix * spec_cols * 8 + 2 * half + half / n_frames


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def fp32_peak_tflops(n_sm, sm_mhz):
    return n_sm * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def probe_peaks(local_rank):
    """FP32 and FP64 fused multiply-add rates of this GPU, measured by the
    library's probe kernel (every SM full of independent FMA chains, one
    launch timed with CUDA events) with nvidia-smi clocks sampled during
    the probe. Outside any timed region."""
    from paper_2505_10639_gb300 import mfbd
    mfbd.probe_fma_rate(False, iters=20000)  # warm the clocks
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.2)
    fp32, ms32, _ = mfbd.probe_fma_rate(False)
    fp64, ms64, _ = mfbd.probe_fma_rate(True)
    clk = clocks.stop()
    return {"fp32_tflops": fp32, "fp32_ms": ms32, "fp64_tflops": fp64, "fp64_ms": ms64, "clocks": clk,
            "how": "library probe mfbd_probe_fma_rate: 8 CTAs x 256 threads per SM, 8 independent FMA "
                   "chains a thread, one launch timed with CUDA events"}


# ------------------------------------------------------------ CPU oracle leg

def _oracle_worker(args):
    """Generate this worker's patches (untimed), wait at the barrier, then
    time the oracle's loss+object+gradient on them."""
    (w, seed, patch_ids, objs, barrier, queue) = args
    from oracle import mfbd as omfbd
    from oracle import optics
    from paper_2505_10639_gb300 import synth
    masks = [optics.pupil_mask(w["n_pix"], d) for d in w["diams"]]
    bases, var = [], None
    for d in w["diams"]:
        b, v, _ = optics.kl_basis(w["n_pix"], d, w["n_modes"])
        bases.append(b)
        var = v
    scales = [w["wavelengths"][0] / x for x in w["wavelengths"]]
    setup = omfbd.Setup(masks, bases, scales, np.ones((len(w["diams"]), w["n_frames"])), gamma_of(w))
    data = []
    K, J, N = len(w["diams"]), w["n_frames"], w["n_pix"]
    for i, p in enumerate(patch_ids):
        a_true, a_eval = per_patch_draws(w, seed, p, var)
        noise = synth.noise(seed, (K, J, N, N), w["noise_sigma"], sub=p)
        d = omfbd.synth_spectra(setup, a_true, objs[i], noise)
        data.append((a_eval.astype(np.float32).astype(np.float64), d.astype(np.complex64).astype(np.complex128)))
    barrier.wait()
    t0 = time.time()
    for a, d in data:
        omfbd.loss_object_grad_patch(setup, a, d)
    t1 = time.time()
    queue.put((t0, t1, len(patch_ids)))


def run_oracle_config1(min_seconds=2.0):
    """The FP64 oracle on the single-patch workload (64 px, 1 object, 8
    frames, 32 px pupil, Noll 2-21, D/r0 = 5, seed 20250516) on one host
    core: loss, object and gradient repeated for at least min_seconds;
    returns (units/s, seconds, evaluations)."""
    from oracle import mfbd as omfbd
    from oracle import optics
    from paper_2505_10639_gb300 import synth
    n, diam, J, M, seed = 64, 32.0, 8, 20, 20250516
    setup = omfbd.Setup([optics.pupil_mask(n, diam)], [optics.zernike_basis(n, diam, range(2, M + 2))], [1.0],
                        np.ones((1, J)), 1e-3 * n * n * 1e-6)
    var = optics.mode_variances("zernike", M)
    a_true = synth.kolmogorov_coeffs(seed, var, 5.0, (1, J))
    a_eval = a_true + 0.3 * synth.kolmogorov_coeffs(seed, var, 5.0, (1, J), sub=1)
    obj = synth.object_field(seed, (1, 1, n, n))
    noise = synth.noise(seed, (1, 1, J, n, n), 1e-3)
    d = omfbd.synth_spectra(setup, a_true[0], obj[0], noise[0])
    a = a_eval[0].astype(np.float32).astype(np.float64)
    dd = d.astype(np.complex64).astype(np.complex128)
    count, t0 = 0, time.time()
    while True:
        omfbd.loss_object_grad_patch(setup, a, dd)
        count += 1
        t = time.time() - t0
        if t >= min_seconds:
            return count * J / t, t, count


def run_oracle_sample(w, seed, n_patches, cores):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    ids = list(range(n_patches))
    chunks = [ids[i::cores] for i in range(cores)]
    chunks = [c for c in chunks if c]
    objs = object_patches(w, seed)  # the field once, in this process
    barrier = ctx.Barrier(len(chunks))
    queue = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=((w, seed, c, objs[c], barrier, queue),)) for c in chunks]
    for p in procs:
        p.start()
    res = [queue.get() for _ in procs]
    for p in procs:
        p.join()
    t0 = min(r[0] for r in res)
    t1 = max(r[1] for r in res)
    n = sum(r[2] for r in res)
    units = n * len(w["diams"]) * w["n_frames"]
    return units / (t1 - t0), t1 - t0, n, len(chunks)


# ------------------------------------------------------------ GPU leg

def time_replays(graph, steps, stream, world, local_rank):
    """Replays a captured step `steps` times on `stream`, every replay
    between two CUDA events, with nvidia-smi clocks sampled meanwhile and a
    barrier plus synchronisation on both sides; returns the mean (the K
    steps' total / K), the per-step times and the clock record."""
    import torch
    import torch.distributed as dist
    clocks = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    clocks.start()
    time.sleep(0.2)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record(stream)
    for i in range(steps):
        graph.replay()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    return ev[0].elapsed_time(ev[steps]) / steps, per, clk


def step_stats(per):
    return {"median_ms": statistics.median(per), "min_ms": min(per), "max_ms": max(per), "replays": len(per)}


def profile_steps(plan, steps, run):
    """Per-kernel CUDA-event times of `steps` evaluations (the library's
    profiling pairs), outside the timed region."""
    import torch
    plan.set_profiling(True, max_launches=8 * (steps + 2) * (2 * plan.n_objects + 4))
    plan.read_profile(reset=True)
    for _ in range(steps):
        run()
    torch.cuda.synchronize()
    prof = plan.read_profile(reset=True)
    plan.set_profiling(False)
    return prof


def make_plan(w, precision, projection, recompute, kernels):
    from paper_2505_10639_gb300.mfbd import Plan
    return Plan(w["n_pix"], w["n_patches"], w["diams"], w["wavelengths"], w["n_frames"], w["n_modes"],
                basis=w["basis"], gamma=gamma_of(w), precision=precision, projection=projection,
                recompute=recompute, generic=(kernels == "generic"), split=(kernels == "split"))


def time_field(args, w, seed, local_rank, world, peaks):
    """Inputs, plan, captured step, timed replays and the profiled kernel
    pass of one field workload; returns (line, plan, buffers)."""
    import torch
    coeffs, spectra = make_gpu_inputs(w, seed)  # the data always come from the FP32 forward model
    plan = make_plan(w, args.precision, args.projection, args.recompute, args.kernels)
    info = plan.info()
    loss = torch.empty(w["n_patches"], dtype=torch.float64, device=plan.device)
    grad = torch.empty(plan.coeff_shape(), dtype=torch.float32, device=plan.device)
    stream = torch.cuda.current_stream()
    graph = plan.capture(coeffs, spectra, loss, grad)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    if not np.isfinite(loss.cpu().numpy()).all():
        raise RuntimeError("non-finite loss")
    local_ms, per, clk = time_replays(graph, args.steps, stream, world, local_rank)
    del graph
    prof = profile_steps(plan, args.steps, lambda: plan.loss_grad(coeffs, spectra, loss=loss, grad=grad))
    rmax, rsum = (torch_reducers() if world > 1 else (None, None))
    ms, units, value = aggregate(local_ms, units64_of(w), world, rmax, rsum)
    line = finish_line(args, plan, info, w, world, ms, value, None, prof, clk, peaks)
    line["timing"] = dict(step_stats(per), how="CUDA graph of one mfbd_loss_grad replayed per step, CUDA events "
                                               "between replays on the launching stream; kernel times from a "
                                               "separate profiled pass of the same number of steps")
    return line, plan, (coeffs, spectra, loss, grad, stream, rmax, rsum, local_ms)


def run_gpu(args, rank, local_rank, world, peaks):
    import torch

    torch.cuda.set_device(local_rank)
    w = WORKLOAD
    line, plan, bufs = time_field(args, w, SEED + rank, local_rank, world, peaks)
    coeffs, spectra, loss, grad, stream, rmax, rsum, local_ms = bufs
    if world == 1 and not args.no_extras and w["n_pix"] == 64 and args.precision == "fp32":
        line["bf16_phase"] = run_bf16_arm(args, w, plan, coeffs, spectra, local_rank, local_ms)
        line["dictionary_model"] = run_dictionary(args, w)
    if not args.no_e2e:
        line["e2e"] = run_e2e(args, plan, coeffs, spectra, loss, grad, stream, world, rmax, rsum, w)
    if not args.no_frontend:
        # (the front end writes its own spectra over the workload's: last)
        line["object_inferring_loss"] = run_explicit(args, plan, coeffs, spectra, w)
        line["frontend"] = run_frontend(args, plan, coeffs, spectra, w)
    plan.close()
    return line


def compact(line):
    """The figures of a workload's own line that another line carries."""
    keep = ("value", "unit", "ms_per_step", "timing", "roofline", "step_roofline", "kernels_ms_per_step",
            "gpu_launches", "clocks", "e2e")
    out = {k: line[k] for k in keep if k in line}
    out["workload"] = line["config"]["workload"]
    for k in ("problems_per_s", "units_per_step", "units64_per_step", "precision", "recompute", "schedule"):
        if k in line["config"]:
            out[k] = line["config"][k]
    return out


def run_extras(args, local_rank, peaks):
    """The other configurations of the benchmark in the same process, after
    the headline: the 2000-problem uneven batch and the 128 px field (its
    own precision and recompute settings), each timed like the headline."""
    import copy
    import torch
    out = {}
    a = copy.copy(args)
    a.no_e2e, a.no_frontend = True, True
    w = dict(WORKLOADS["batched2000"])
    out["batched2000"] = compact(run_gpu_batch(a, 0, local_rank, 1, w=w, peaks=peaks))
    torch.cuda.empty_cache()
    w = dict(WORKLOADS["fov4096_128px"])
    if args.extra_128px_patches:
        w["n_patches"] = args.extra_128px_patches
        w["workload"] += "_first%d" % args.extra_128px_patches
    w["workload"] += "_bf16phase"
    a.precision, a.recompute, a.projection, a.kernels = w["precision"], w["recompute"], "tensor", "pass"
    line, plan, bufs = time_field(a, w, w["seed"], local_rank, 1, peaks)
    plan.close()
    del bufs
    torch.cuda.empty_cache()
    out["fov4096_128px"] = compact(line)
    return out


def run_bf16_arm(args, w, plan32, coeffs, spectra, local_rank, fp32_ms):
    """The BF16-phase form of the same workload (the phase projection with
    BF16 operands on the tensor cores, the rest as FP32) on the same inputs
    in the same process: time per step as for the FP32 line, and its
    difference from the FP32 results (max relative loss difference over the
    patches, worst per-patch relative L2 difference of dL/da)."""
    import torch
    loss32, grad32, _ = plan32.loss_grad(coeffs, spectra)  # the FP32 results on these inputs
    plan = make_plan(w, "bf16_phase", "tensor", args.recompute, args.kernels)
    loss = torch.empty_like(loss32)
    grad = torch.empty_like(grad32)
    stream = torch.cuda.current_stream()
    graph = plan.capture(coeffs, spectra, loss, grad)
    for _ in range(args.warmup):
        graph.replay()
    ms, per, clk = time_replays(graph, args.steps, stream, 1, local_rank)
    prof = profile_steps(plan, args.steps, lambda: plan.loss_grad(coeffs, spectra, loss=loss, grad=grad))
    l32, g32 = loss32.cpu().numpy(), grad32.cpu().numpy()
    l16, g16 = loss.cpu().numpy(), grad.cpu().numpy()
    dl = float(np.max(np.abs(l16 - l32) / np.abs(l32)))
    num = np.linalg.norm((g16 - g32).reshape(len(l32), -1), axis=1)
    den = np.linalg.norm(g32.reshape(len(l32), -1), axis=1)
    dg = float(np.max(num / den))
    del graph
    plan.close()
    return {"workload": w["workload"] + "_bf16phase", "ms_per_step": ms, "value": units64_of(w) / (ms * 1e-3),
            "unit": UNIT, "speedup_vs_fp32": fp32_ms / ms, "timing": step_stats(per), "clocks": clk,
            "kernels_ms_per_step": {k: v[0] / max(1, args.steps) for k, v in prof.items()},
            "difference_from_fp32": {"loss_max_rel": dl, "grad_max_rel_l2": dg},
            "accuracy": "errors against the FP64 oracle are bounded by the -m gpu tests (loss 1e-2, dL/da 2e-2, "
                        "object 1e-3 relative)"}


def run_explicit(args, plan, coeffs, spectra, w):
    """The object-inferring loss (mfbd_loss_grad_explicit) on the same inputs
    with the Wiener objects given back (dL/da and dL/dconj(O) both
    computed): CUDA-event time per call and the same metric (not part of a
    step)."""
    import torch
    loss, grad, obj = plan.loss_grad(coeffs, spectra, want_object=True)
    gobj = torch.empty_like(obj)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        plan.loss_grad_explicit(coeffs, spectra, obj, loss=loss, grad=grad, grad_obj=gobj)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.loss_grad_explicit(coeffs, spectra, obj, loss=loss, grad=grad, grad_obj=gobj)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / args.steps
    return {"ms": t, "value": units64_of(w) / (t * 1e-3), "unit": UNIT}


DICT_ATOMS = 8


def run_dictionary(args, w):
    """The spatially variant dictionary model (mfbd_dict_loss_grad, Sec.
    2.2.2) on the workload's patches, objects and frames with an 8-atom
    dictionary, both gradients computed (not part of a step): the inputs of
    synth.dictionary_case drawn for 31 patches and tiled over the field's
    patches (timing does not depend on the values); CUDA-event time per call,
    units (patch, object, frame) per second, and the HBM roofline of the unit
    kernel's algorithmic bytes (coefficient maps read, their gradient written,
    spectra read: 2 M N^2 4 + N (N/2+1) 8 bytes per unit)."""
    import torch
    from paper_2505_10639_gb300 import synth
    from paper_2505_10639_gb300.mfbd import dict_loss_grad
    P, K, J, N, M = w["n_patches"], len(w["diams"]), w["n_frames"], w["n_pix"], DICT_ATOMS
    blk = 31
    atoms, atom_otf, gamma, obj, coeff, spectra = synth.dictionary_case(SEED, blk, K, J, M, n=N)
    rep = (P + blk - 1) // blk

    def tiled(x):
        t = torch.from_numpy(x).cuda()
        return t.repeat((rep,) + (1,) * (t.dim() - 1))[:P].contiguous()

    t_otf, t_gamma = torch.from_numpy(atom_otf).cuda(), torch.from_numpy(gamma).cuda()
    t_obj, t_coeff, t_spec = tiled(obj), tiled(coeff), tiled(spectra)
    loss, go, ga = dict_loss_grad(t_otf, t_gamma, t_obj, t_coeff, t_spec)
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup - 1, 0)):
        dict_loss_grad(t_otf, t_gamma, t_obj, t_coeff, t_spec, loss=loss, grad_object=go, grad_coeff=ga)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        dict_loss_grad(t_otf, t_gamma, t_obj, t_coeff, t_spec, loss=loss, grad_object=go, grad_coeff=ga)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / args.steps
    units = P * K * J
    nbytes = units * (2 * M * N * N * 4 + N * (N // 2 + 1) * 8)
    hbm = measured_peaks().get("hbm_gbs", 6800.0)
    out = {"ms": t, "value": units / (t * 1e-3), "unit": "units/s (patch*obj*frame, %d atoms)" % M,
           "workload": "fov1024_64px_961patches_2obj_12frames_%datoms" % M,
           "roofline": {"bound": "hbm", "achieved": nbytes / (t * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                        "frac": nbytes / (t * 1e-3) / 1e9 / hbm, "traffic": None,
                        "algorithmic_bytes": nbytes},
           "gpu_launches": 2}
    del t_coeff, ga
    torch.cuda.empty_cache()
    return out


def run_frontend(args, plan, coeffs, spectra, w):
    """The field front and back end on the workload's field (not part of a
    step): mfbd_spectra_from_frames over K x J seeded frames of fov^2 px
    (overlap N/2, border 6), mfbd_merge_objects of the Wiener objects and
    mfbd_ls_filter_objects (the Lofdahl-Scharmer filter from the spectra and
    the OTFs); CUDA-event times of each and their algorithmic HBM bytes per
    launch (frames read + spectra written; objects read, patch images written
    and read, mosaic written; spectra and OTFs read, filter written, objects
    read and written)."""
    import torch
    K, J, N, P, fov = len(w["diams"]), w["n_frames"], w["n_pix"], w["n_patches"], w["fov"]
    if P != ((fov - N) // (N // 2) + 1) ** 2:
        return None  # a partial field (--patches)
    g = torch.Generator(device=plan.device)
    g.manual_seed(w["seed"])
    frames = 1.0 + 0.1 * torch.randn((K, J, fov, fov), generator=g, device=plan.device)
    _, _, obj = plan.loss_grad(coeffs, spectra, want_object=True)
    image = torch.empty((K, fov, fov), dtype=torch.float32, device=plan.device)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        plan.spectra_from_frames(frames, N // 2, 6, out=spectra)
        plan.merge_objects(obj, fov, fov, N // 2, 6, out=image)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(stream)
    for _ in range(args.steps):
        plan.spectra_from_frames(frames, N // 2, 6, out=spectra)
    ev[1].record(stream)
    ev[2].record(stream)
    for _ in range(args.steps):
        plan.merge_objects(obj, fov, fov, N // 2, 6, out=image)
    ev[3].record(stream)
    torch.cuda.synchronize()
    t_spec = ev[0].elapsed_time(ev[1]) / args.steps
    t_merge = ev[2].elapsed_time(ev[3]) / args.steps
    # the Lofdahl-Scharmer filter of the objects from D and the OTFs, noise
    # power N^2 sigma^2 (the synthetic noise's)
    otf = plan.otf(coeffs)
    nu = N * N * w["noise_sigma"] ** 2
    flt = None
    for _ in range(args.warmup):
        flt = plan.ls_filter_objects(spectra, otf, nu, obj=obj)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(args.steps):
        plan.ls_filter_objects(spectra, otf, nu, obj=obj)
    ev[1].record(stream)
    torch.cuda.synchronize()
    t_ls = ev[0].elapsed_time(ev[1]) / args.steps
    b_ls = spectra.numel() * 8 + otf.numel() * 8 + flt.numel() * 4 + 2 * obj.numel() * 8
    del otf
    b_spec = frames.numel() * 4 + spectra.numel() * 8
    b_merge = obj.numel() * 8 + 2 * P * K * N * N * 4 + image.numel() * 4
    hbm = measured_peaks().get("hbm_gbs", 6800.0)
    captured = N == 64 and P == 961  # the field of the ncu capture
    return {"bound": "hbm", "peak_gbs": hbm,
            "spectra_from_frames": {"ms": t_spec, "bytes": b_spec, "gbs": b_spec / (t_spec * 1e-3) / 1e9,
                                    "frac": b_spec / (t_spec * 1e-3) / 1e9 / hbm,
                                    "traffic": NCU_FRONT_DRAM_BYTES["spectra_from_frames"] if captured else None},
            "merge_objects": {"ms": t_merge, "bytes": b_merge, "gbs": b_merge / (t_merge * 1e-3) / 1e9,
                              "frac": b_merge / (t_merge * 1e-3) / 1e9 / hbm,
                              "traffic": NCU_FRONT_DRAM_BYTES["merge_objects"] if captured else None},
            "ls_filter_objects": {"ms": t_ls, "bytes": b_ls, "gbs": b_ls / (t_ls * 1e-3) / 1e9,
                                  "frac": b_ls / (t_ls * 1e-3) / 1e9 / hbm,
                                  "traffic": NCU_FRONT_DRAM_BYTES["ls_filter_objects"] if captured else None},
            "field": "%d x %d px, %d patches of %d px, overlap %d, border 6" % (fov, fov, P, N, N // 2)}


def run_e2e(args, plan, coeffs, spectra, loss, grad, stream, world, rmax, rsum, w):
    """Same metric through the public host-buffer call (mfbd_loss_grad_host):
    every step copies its coefficients and spectra from pinned host memory
    and reads loss and grad back, chunk by chunk, overlapped with the
    kernels of other chunks."""
    import torch
    import torch.distributed as dist
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    a_host = torch.empty(coeffs.shape, dtype=coeffs.dtype, pin_memory=True)
    a_host.copy_(coeffs)
    d_host = torch.empty(spectra.shape, dtype=spectra.dtype, pin_memory=True)
    d_host.copy_(spectra)
    l_host = torch.empty_like(loss, device="cpu").pin_memory()
    g_host = torch.empty_like(grad, device="cpu").pin_memory()

    def e2e_step():
        plan.loss_grad_host(a_host, d_host, loss=l_host, grad=g_host, n_chunks=args.e2e_chunks, stream=stream)

    for _ in range(max(1, args.warmup)):
        e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    # the host-buffer results are the device call's bits
    plan.loss_grad(coeffs, spectra, loss=loss, grad=grad)
    torch.cuda.synchronize()
    if not (torch.equal(loss.cpu(), l_host) and torch.equal(grad.cpu(), g_host)):
        raise RuntimeError("host-buffer call differs from the device call")
    e2e_local = e0.elapsed_time(e1) / args.steps
    e2e_ms, _, e2e_value = aggregate(e2e_local, units64_of(w), world, rmax, rsum)
    h2d = coeffs.numel() * 4 + spectra.numel() * 8
    d2h = loss.numel() * 8 + grad.numel() * 4
    return {"value": e2e_value, "unit": UNIT, "ms_per_step": e2e_ms, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "chunks": args.e2e_chunks}


def alu_peak_of(peaks, n_sm):
    """FP32 peak for the ALU-bound kernels: the probe's measured FMA rate
    when there is one, else SMs x 128 lanes x 2 flop x the maximum clock."""
    mp = measured_peaks()
    derived = fp32_peak_tflops(n_sm, mp.get("sm_max_mhz", 2070.0))
    if peaks and peaks.get("fp32_tflops"):
        basis = ("measured: FP32 FMA probe (mfbd_probe_fma_rate), %.1f TFLOP/s at %s MHz median SM clock; "
                 "derived %d SMs x %d lanes x 2 flop x %.0f MHz = %.1f"
                 % (peaks["fp32_tflops"], peaks["clocks"].get("sm_mhz"), n_sm, FP32_LANES_PER_SM,
                    mp.get("sm_max_mhz", 2070.0), derived))
        return peaks["fp32_tflops"], basis, derived
    return derived, ("derived: %d SMs x %d lanes x 2 flop x %.0f MHz (max SM clock)"
                     % (n_sm, FP32_LANES_PER_SM, mp.get("sm_max_mhz", 2070.0))), derived


def step_flops_per_unit(n_pix, npup, n_modes):
    """Algorithmic FP32 flops of one unit of a whole step: the two pass
    directions, the frame reduction, and the modal projection and its adjoint
    on the pupil's pixels (2 n_pup M each)."""
    f, a = pass_flops_per_unit(n_pix, npup)
    return f + a + reduction_flops_per_unit(n_pix) + 4.0 * npup * n_modes


def finish_line(args, plan, info, w, world, ms, value, e2e, prof, clk, peaks):
    import torch
    local_rank = dist_env()[1]
    # roofline: every kernel against its bound; the dominant one is reported
    npup = info["pupil_pixels"]
    per_obj = [pass_flops_per_unit(w["n_pix"], npup[k]) for k in range(len(npup))]
    units_obj = w["n_patches"] * w["n_frames"]
    fwd_flops = sum(f for f, _ in per_obj) * units_obj
    adj_flops = sum(a for _, a in per_obj) * units_obj
    red_bytes = reduction_bytes_per_unit(w["n_pix"], w["n_frames"], w["n_pix"] // 2 + 1) * units_of(w)
    mp = measured_peaks()
    n_sm = torch.cuda.get_device_properties(local_rank).multi_processor_count
    alu_peak, alu_basis, alu_derived = alu_peak_of(peaks, n_sm)
    hbm_peak = mp.get("hbm_gbs", 6800.0)

    def per_launch(kind):
        # one launch of each stage per step (the reduction and fused stages
        # include their loss-combine kernel)
        return prof[kind][0] / max(1, args.steps)

    # DRAM traffic from the committed ncu captures of the 64 px kernels and
    # of the 128 px kernels with recompute; not measured for the others
    ncu_tab, ncu_basis = None, "not captured for this kernel family"
    if w["n_pix"] == 64 and args.kernels in ("pass", "split") and not args.recompute:
        ncu_tab, ncu_basis = NCU_DRAM_BYTES_PER_UNIT, "ncu DRAM bytes per unit (400-patch capture) x units per launch"
    elif w["n_pix"] == 128 and args.recompute:
        ncu_tab, ncu_basis = NCU_DRAM_BYTES_PER_UNIT_128, "ncu DRAM bytes per unit (48-patch capture) x units per launch"
    kernels = {}
    if prof.get("fused", (0.0, 0))[1] > 0:
        # the fused per-(patch, object) kernel: the pass flops of both
        # directions plus the frame reduction's, against the FP32 peak
        red_flops = reduction_flops_per_unit(w["n_pix"]) * units_of(w)
        work = fwd_flops + adj_flops + red_flops
        t = per_launch("fused")
        a = work / (t * 1e-3) / 1e12 if t > 0 else 0.0
        tr = NCU_DRAM_BYTES_PER_UNIT.get("fused_pairs") if ncu_tab else None
        if tr:
            ncu_basis = "ncu DRAM bytes per unit (capture of the full 961-patch launch) x units per launch"
        kernels["fused_pairs"] = {"bound": "alu", "ms": t, "achieved": a, "peak": alu_peak, "unit": "TFLOP/s",
                                  "frac": a / alu_peak, "frac_of_derived_peak": a / alu_derived,
                                  "work_per_launch": work, "traffic": tr * units_of(w) if tr else None}
    for name, kind, work in (("forward_passes", "forward", fwd_flops), ("adjoint_passes", "adjoint", adj_flops)):
        if prof.get(kind, (0.0, 0))[1] == 0:
            continue
        t = per_launch(kind)
        a = work / (t * 1e-3) / 1e12 if t > 0 else 0.0
        kernels[name] = {"bound": "alu", "ms": t, "achieved": a, "peak": alu_peak, "unit": "TFLOP/s",
                         "frac": a / alu_peak, "frac_of_derived_peak": a / alu_derived, "work_per_launch": work,
                         "traffic": ncu_tab[name] * units_of(w) if ncu_tab else None}
    if prof.get("reduction", (0.0, 0))[1] > 0:
        t = per_launch("reduction")
        a = red_bytes / (t * 1e-3) / 1e9 if t > 0 else 0.0
        kernels["reduction"] = {"bound": "hbm", "ms": t, "achieved": a, "peak": hbm_peak, "unit": "GB/s",
                                "frac": a / hbm_peak, "work_per_launch": red_bytes,
                                "traffic": ncu_tab["reduction"] * units_of(w) if ncu_tab else None}
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    dk = kernels[dom]
    roofline = {"bound": dk["bound"], "kernel": dom, "achieved": dk["achieved"], "peak": dk["peak"],
                "unit": dk["unit"], "frac": dk["frac"], "traffic": dk["traffic"],
                "traffic_basis": ncu_basis,
                "peak_basis": alu_basis if dk["bound"] == "alu" else "HBM copy bandwidth of MEASURED_PEAKS.json",
                "work_per_launch": dk["work_per_launch"], "kernel_ms": dk["ms"]}
    # the whole step against the binding pipe (FP32: the FP64 and HBM work
    # per unit bind later)
    step_flops = sum(step_flops_per_unit(w["n_pix"], npup[k], w["n_modes"]) for k in range(len(npup))) * units_obj
    step_tf = step_flops / (ms * 1e-3) / 1e12
    step_roofline = {"bound": "alu", "achieved": step_tf, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": step_tf / alu_peak, "work_per_step": step_flops,
                     "work_per_unit": step_flops / units_of(w),
                     "basis": "pass flops of both directions + frame reduction + modal projection and adjoint "
                              "(4 n_pup M) per unit, over ms_per_step"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w["workload"], "patch_px": w["n_pix"], "patches": w["n_patches"],
                   "objects": len(w["diams"]), "frames": w["n_frames"], "modes": w["n_modes"],
                   "basis": w["basis"], "pupil_px": w["diams"], "d_over_r0": w["d_over_r0"],
                   "precision": args.precision, "projection": args.projection, "recompute": args.recompute,
                   "kernels": args.kernels, "units_per_step": units_of(w),
                   "unit_weight_at_64px": unit_weight_64(w["n_pix"]),
                   "l2": "inputs larger than L2 (%.0f MB spectra)"
                         % (units_of(w) * w["n_pix"] * (w["n_pix"] // 2 + 1) * 8 / 1e6),
                   "parallelism": "replicas" if world > 1 else "single"},
        "e2e": e2e,
        "roofline": roofline,
        "step_roofline": step_roofline,
        "kernels": kernels,
        "kernels_ms_per_step": {k: v[0] / max(1, args.steps) for k, v in prof.items()},
        "gpu_launches": int(sum(v[1] for v in prof.values())),  # kernels, counted by the library
        "clocks": clk,
        "peaks_measured": peaks,
        "plan": info,
    }
    return line


# ------------------------------------------------------------ uneven batch

def batch_problems(w):
    from paper_2505_10639_gb300 import synth
    return synth.uneven_problems(w["seed"], 2000)[: w["n_problems"]]


def batch_gamma(n_pix, w):
    return 1e-3 * n_pix ** 2 * w["noise_sigma"] ** 2


def batch_units64(probs):
    return sum(p["n_objects"] * p["n_frames"] * unit_weight_64(p["n_pix"]) for p in probs)


def batch_flops(probs):
    """Algorithmic FP32 flops of one evaluation: the pass flops of every unit
    (pass_flops_per_unit) plus the phase projection and modal adjoint,
    2 n_box M flops each per unit (n_box = W^2, the pupil's box)."""
    from paper_2505_10639_gb300.mfbd import describe_object
    tot = 0.0
    cache = {}
    for p in probs:
        for k, d in enumerate(p["diams"]):
            key = (p["n_pix"], d)
            if key not in cache:
                mask, _, _, _ = describe_object(0, p["n_pix"], [d], [1.0], 1, 1, basis="zernike")
                ys, xs = np.nonzero(mask)
                w_box = int(max(ys.max() - ys.min(), xs.max() - xs.min()) + 1)
                cache[key] = (int(mask.sum()), w_box)
            npup, w_box = cache[key]
            f, a = pass_flops_per_unit(p["n_pix"], npup)
            tot += p["n_frames"] * (f + a + 4.0 * w_box * w_box * p["n_modes"])
    return tot


def make_batch_inputs(batch, probs, w):
    """Coefficients (Kolmogorov draws at the evaluation point) and spectra
    D = F(o) H_true + F(n), built on the device with the batch's own OTF."""
    import torch
    from paper_2505_10639_gb300 import synth
    from paper_2505_10639_gb300.mfbd import Batch, describe_object
    _, _, var, _ = describe_object(0, 64, [32.0], [1.0], 1, 66, basis="zernike")  # Noll variances, a prefix per M
    dev = batch.device
    a_true, a_eval = [], []
    for i, p in enumerate(probs):
        v = var[:p["n_modes"]]
        t = synth.kolmogorov_coeffs(w["seed"], v, w["d_over_r0"], (1, p["n_frames"]), sub=2 * i)
        e = t + 0.3 * synth.kolmogorov_coeffs(w["seed"], v, w["d_over_r0"], (1, p["n_frames"]), sub=2 * i + 1)
        a_true.append(torch.from_numpy(t.astype(np.float32)))
        a_eval.append(torch.from_numpy(e.astype(np.float32)))
    h = batch.otf(Batch.pack(a_true).to(dev))
    hs = batch.unpack(h, "spectra")
    for i, p in enumerate(probs):
        n, k, j = p["n_pix"], p["n_objects"], p["n_frames"]
        o = torch.from_numpy(synth.object_field(w["seed"], (1, k, n, n), sub=i)).to(dev)
        nz = synth.noise_torch(w["seed"], (1, k, j, n, n), w["noise_sigma"], sub=i, device=dev)
        hs[i].mul_(torch.fft.rfft2(o).to(torch.complex64)[:, :, None]).add_(torch.fft.rfft2(nz).to(torch.complex64))
    torch.cuda.synchronize()
    return Batch.pack(a_eval).to(dev), h


def _oracle_batch_worker(args):
    (w, items, barrier, queue) = args
    from oracle import mfbd as omfbd
    from oracle import optics
    from paper_2505_10639_gb300 import synth
    data = []
    for i, p in items:
        n, k, j, m = p["n_pix"], p["n_objects"], p["n_frames"], p["n_modes"]
        masks = [optics.pupil_mask(n, d) for d in p["diams"]]
        bases = [optics.zernike_basis(n, d, range(2, m + 2)) for d in p["diams"]]
        scales = [p["wavelengths"][0] / x for x in p["wavelengths"]]
        setup = omfbd.Setup(masks, bases, scales, np.ones((k, j)), batch_gamma(n, w))
        var = optics.mode_variances("zernike", m)
        t = synth.kolmogorov_coeffs(w["seed"], var, w["d_over_r0"], (1, j), sub=2 * i)
        e = t + 0.3 * synth.kolmogorov_coeffs(w["seed"], var, w["d_over_r0"], (1, j), sub=2 * i + 1)
        o = synth.object_field(w["seed"], (1, k, n, n), sub=i)
        nz = synth.noise(w["seed"], (k, j, n, n), w["noise_sigma"], sub=i)
        d = omfbd.synth_spectra(setup, t[0], o[0], nz)
        data.append((setup, e[0].astype(np.float32).astype(np.float64), d.astype(np.complex64).astype(np.complex128),
                     k * j * unit_weight_64(n)))
    barrier.wait()
    t0 = time.time()
    for setup, a, d, _ in data:
        omfbd.loss_object_grad_patch(setup, a, d)
    t1 = time.time()
    queue.put((t0, t1, len(items), sum(x[3] for x in data)))


def run_oracle_batch_sample(w, n_problems, cores):
    """The FP64 oracle on the first n_problems problems, spread over the
    host cores (spawned workers); returns 64 px units/s, seconds, problems,
    workers."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    probs = batch_problems(w)[:n_problems]
    items = list(enumerate(probs))
    chunks = [c for c in (items[i::cores] for i in range(cores)) if c]
    barrier = ctx.Barrier(len(chunks))
    queue = ctx.Queue()
    procs = [ctx.Process(target=_oracle_batch_worker, args=((w, c, barrier, queue),)) for c in chunks]
    for p in procs:
        p.start()
    res = [queue.get() for _ in procs]
    for p in procs:
        p.join()
    t0, t1 = min(r[0] for r in res), max(r[1] for r in res)
    units = sum(r[3] for r in res)
    return units / (t1 - t0), t1 - t0, sum(r[2] for r in res), len(chunks)


def run_gpu_batch(args, rank, local_rank, world, w=None, peaks=None):
    """One evaluation of the 2000-problem uneven batch per step: the captured
    CUDA graph of mfbd_batch_loss_grad (counter memset + one persistent
    launch, or the autotuner's schedule) replayed, inputs resident."""
    import torch
    from paper_2505_10639_gb300.mfbd import Batch, Problem

    torch.cuda.set_device(local_rank)
    w = dict(WORKLOAD if w is None else w)
    w["seed"] = w["seed"] + rank
    probs = batch_problems(w)
    batch = Batch([Problem(p["n_pix"], 1, p["diams"], p["wavelengths"], p["n_frames"], p["n_modes"],
                           basis="zernike", gamma=batch_gamma(p["n_pix"], w)) for p in probs])
    coeffs, spectra = make_batch_inputs(batch, probs, w)
    loss, grad, _ = batch.outputs()
    if args.batch_schedule == "auto":
        batch.autotune(coeffs, spectra, loss, grad, reps=2)
    else:
        parts = args.batch_schedule.split(":") + ["0", "0"]
        batch.set_schedule(parts[0], int(parts[1]), 0, int(parts[2]))
    info = batch.info()
    graph = batch.capture(coeffs, spectra, loss, grad)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        graph.replay()
    batch.check()
    if not np.isfinite(loss.cpu().numpy()).all():
        raise RuntimeError("non-finite loss")
    local_ms, per, clk = time_replays(graph, args.steps, stream, world, local_rank)
    batch.check()
    rmax, rsum = (torch_reducers() if world > 1 else (None, None))
    u64 = batch_units64(probs)
    ms, _, value = aggregate(local_ms, u64, world, rmax, rsum)

    e2e = None
    if not args.no_e2e:
        # through the public API from pinned host buffers: H2D of coefficients
        # and spectra, the evaluation, D2H of loss and gradient, every step
        a_h = torch.empty(coeffs.shape, dtype=coeffs.dtype, pin_memory=True)
        a_h.copy_(coeffs)
        d_h = torch.empty(spectra.shape, dtype=spectra.dtype, pin_memory=True)
        d_h.copy_(spectra)
        l_h = torch.empty(loss.shape, dtype=loss.dtype, pin_memory=True)
        g_h = torch.empty(grad.shape, dtype=grad.dtype, pin_memory=True)
        a_d, d_d = torch.empty_like(coeffs), torch.empty_like(spectra)

        def e2e_step():
            a_d.copy_(a_h, non_blocking=True)
            d_d.copy_(d_h, non_blocking=True)
            batch.loss_grad(a_d, d_d, loss=loss, grad=grad)
            l_h.copy_(loss, non_blocking=True)
            g_h.copy_(grad, non_blocking=True)

        for _ in range(max(1, args.warmup)):
            e2e_step()
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        f1.record(stream)
        torch.cuda.synchronize()
        e2e_ms, _, e2e_value = aggregate(f0.elapsed_time(f1) / args.steps, u64, world, rmax, rsum)
        e2e = {"value": e2e_value, "unit": UNIT, "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": coeffs.numel() * 4 + spectra.numel() * 8,
               "d2h_bytes_per_step": loss.numel() * 8 + grad.numel() * 4}

    n_sm = torch.cuda.get_device_properties(local_rank).multi_processor_count
    alu_peak, alu_basis, alu_derived = alu_peak_of(peaks, n_sm)
    flops = batch_flops(probs)
    achieved = flops / (local_ms * 1e-3) / 1e12
    units = sum(p["n_objects"] * p["n_frames"] for p in probs)
    captured = (info["mode"], info["window_units"], info["variant"]) == NCU_BATCH_SCHEDULE
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w["workload"], "problems": len(probs), "units_per_step": units,
                   "units64_per_step": u64, "problems_per_s": len(probs) / (ms * 1e-3),
                   "patch_px": sorted({p["n_pix"] for p in probs}), "basis": "zernike",
                   "schedule": {"mode": ["one_launch", "staged"][info["mode"]], "window_units": info["window_units"],
                                "ctas_per_sm": info["ctas_per_sm"], "kernel_variant": info["variant"],
                                "autotuned": args.batch_schedule == "auto"},
                   "graph": "captured CUDA graph replayed per step",
                   "l2": "inputs larger than L2 (%.0f MB spectra)" % (spectra.numel() * 8 / 1e6),
                   "parallelism": "replicas" if world > 1 else "single"},
        "e2e": e2e,
        "roofline": {"bound": "alu", "kernel": "batch_kernel", "achieved": achieved, "peak": alu_peak,
                     "unit": "TFLOP/s", "frac": achieved / alu_peak,
                     "traffic": NCU_BATCH_DRAM_BYTES_PER_UNIT64 * u64 if captured else None,
                     "traffic_basis": ("ncu DRAM bytes per 64 px-equivalent unit (first 200 problems, same "
                                       "schedule) x units of the launch" if captured
                                       else "not captured for this schedule"),
                     "peak_basis": alu_basis, "frac_of_derived_peak": achieved / alu_derived,
                     "work_per_launch": flops, "kernel_ms": local_ms},
        "gpu_launches": args.steps * (1 if info["mode"] == 0 else 5),
        "clocks": clk,
        "timing": dict(step_stats(per), how="CUDA graph of one batch evaluation replayed per step, CUDA events "
                                            "between replays"),
        "peaks_measured": peaks,
        "batch": {k: info[k] for k in ("n_items", "workspace_bytes", "ctas", "smem_bytes", "max_ctas_per_sm")},
    }
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-patches", type=int, default=0)
    ap.add_argument("--patches", type=int, default=0,
                    help="use only the first N patches of the field (smaller profiling cases)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-frontend", action="store_true",
                    help="skip timing the field front end (spectra from frames) and back end (mosaic)")
    ap.add_argument("--precision", default=None, choices=["fp32", "bf16_phase"],
                    help="bf16_phase: the phase projection with BF16 operands on the tensor cores")
    ap.add_argument("--projection", default="tensor", choices=["tensor", "simt"],
                    help="FP32 phase projection on the tensor cores (three BF16 planes) or the SIMT kernel")
    ap.add_argument("--e2e-chunks", type=int, default=0,
                    help="patch chunks of the host-buffer call (copies overlap the kernels of other chunks)")
    ap.add_argument("--workload", default="fov1024_64px", choices=sorted(WORKLOADS),
                    help="fov1024_64px: 961 patches of 64 px (default); fov4096_128px: 3969 patches of "
                         "128 px; batched2000: 2000 uneven problems in one persistent launch")
    ap.add_argument("--kernels", default="pass", choices=["pass", "split", "generic"],
                    help="64 px: the fused per-(patch, object) kernel (pass; the three-kernel path when the "
                         "plan cannot fuse), the three-kernel path (split), or the CTA-per-unit kernels of the "
                         "other sizes (generic)")
    ap.add_argument("--recompute", default=None, choices=["on", "off"],
                    help="recompute the field and phasors in the backward pass (default: the workload's)")
    ap.add_argument("--problems", type=int, default=0,
                    help="batched2000: use only the first N problems (smaller profiling cases)")
    ap.add_argument("--no-extras", action="store_true",
                    help="time only the chosen workload (by default the 64 px field's line also carries the "
                         "BF16-phase form, the 2000-problem batch and the 128 px field)")
    ap.add_argument("--extra-128px-patches", type=int, default=0,
                    help="time only the first N patches of the 128 px field in the extras (0: all 3969)")
    ap.add_argument("--probe-peaks", action="store_true",
                    help="only measure and print the FP32 and FP64 FMA rates of the GPU")
    ap.add_argument("--batch-schedule", default="auto",
                    help="batched2000: auto (autotuner) or <one_launch|staged>:<window units>:<kernel variant>")
    args = ap.parse_args()
    WORKLOAD.clear()
    WORKLOAD.update(WORKLOADS[args.workload])
    global SEED
    SEED = WORKLOAD["seed"]
    if args.precision is None:
        args.precision = WORKLOAD["precision"]
    args.recompute = WORKLOAD["recompute"] if args.recompute is None else (args.recompute == "on")
    if args.problems and args.workload == "batched2000":
        WORKLOAD["n_problems"] = args.problems
        WORKLOAD["workload"] += "_first%d" % args.problems
    if args.patches:
        WORKLOAD["n_patches"] = args.patches
        WORKLOAD["workload"] += "_first%d" % args.patches
    if args.precision == "bf16_phase":
        WORKLOAD["workload"] += "_bf16phase"
    elif args.projection == "simt":
        WORKLOAD["workload"] += "_simtphase"
    if args.recompute != WORKLOAD["recompute"]:
        WORKLOAD["workload"] += "_recompute" if args.recompute else "_keep"
    if args.kernels == "generic":
        WORKLOAD["workload"] += "_ctaperunit"
    elif args.kernels == "split":
        WORKLOAD["workload"] += "_threekernels"
    args.warmup = max(3, args.warmup)
    rank, local_rank, world = dist_env()

    if args.impl == "reference" and args.workload == "batched2000":
        if rank != 0:
            return 0
        cores = os.cpu_count() or 1
        n = args.cpu_patches or WORKLOAD["cpu_patches"]
        total_t, total_u = 0.0, 0.0
        for _ in range(args.steps):
            rate, t, nprob, used = run_oracle_batch_sample(WORKLOAD, n, cores)
            total_t += t
            total_u += rate * t
        value = total_u / total_t
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": WORKLOAD["workload"], "precision": "fp64 oracle"},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                                 "sample": "the first %d of %d problems per step" % (n, WORKLOAD["n_problems"])},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0
    if args.impl == "reference":
        if rank != 0:
            return 0
        cores = os.cpu_count() or 1
        n = args.cpu_patches or WORKLOAD["cpu_patches"]
        total_t, total_u, rates = 0.0, 0, []
        for _ in range(args.warmup):
            pass  # the oracle has no warm state; warm-up steps are not needed
        for _ in range(args.steps):
            rate, t, npat, used = run_oracle_sample(WORKLOAD, SEED, n, cores)
            rates.append(rate)
            total_t += t
            total_u += npat * len(WORKLOAD["diams"]) * WORKLOAD["n_frames"] * unit_weight_64(WORKLOAD["n_pix"])
        value = total_u / total_t
        sample = "%d of %d patches (all %d objects x %d frames) per step" % (
            n, WORKLOAD["n_patches"], len(WORKLOAD["diams"]), WORKLOAD["n_frames"])
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": WORKLOAD["workload"], "patch_px": WORKLOAD["n_pix"],
                           "precision": "fp64 oracle"},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    if args.probe_peaks:
        import torch
        torch.cuda.set_device(local_rank)
        print(json.dumps(probe_peaks(local_rank)))
        return 0
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import torch
    torch.cuda.set_device(local_rank)
    peaks = probe_peaks(local_rank)
    if args.workload == "batched2000":
        line = run_gpu_batch(args, rank, local_rank, world, peaks=peaks)
        if rank == 0:
            if world == 1 and not args.no_cpu_baseline:
                n = args.cpu_patches or WORKLOAD["cpu_patches"]
                rate, t, nprob, used = run_oracle_batch_sample(WORKLOAD, n, os.cpu_count() or 1)
                line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": used, "kind": "oracle",
                                        "sample": "the first %d of %d problems, %.1f s wall"
                                                  % (nprob, WORKLOAD["n_problems"], t)}
            print(json.dumps(line))
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0
    line = run_gpu(args, rank, local_rank, world, peaks)
    if world == 1 and not args.no_extras and args.workload == "fov1024_64px" and args.kernels == "pass" \
            and args.precision == "fp32" and not args.patches:
        line["configs"] = run_extras(args, local_rank, peaks)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            cores = os.cpu_count() or 1
            n = args.cpu_patches or WORKLOAD["cpu_patches"]
            rate, t, npat, used = run_oracle_sample(WORKLOAD, SEED, n, cores)
            line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": used, "kind": "oracle",
                                    "sample": "%d of %d patches (%d objects x %d frames each), %.1f s wall"
                                              % (npat, WORKLOAD["n_patches"], len(WORKLOAD["diams"]),
                                                 WORKLOAD["n_frames"], t)}
            line["cpu_baseline"]["value"] *= unit_weight_64(WORKLOAD["n_pix"])
            r1, t1, n1 = run_oracle_config1()
            line["cpu_baseline"]["config1_single_thread"] = {
                "value": r1, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": "%d evaluations of the single-patch workload (1 patch, 1 object, 8 frames, 64 px, "
                          "Noll 2-21), %.1f s" % (n1, t1)}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
