"""Benchmark: cubic B-spline interpolation (BSI) of FFD control grids on GB300.

One step = one pass of the whole hot path over one CT-shaped volume
(512 x 512 x 300 voxels, control spacing 5 x 5 x 5, smooth Gaussian random
control displacements): the forward field (Eq. 1) and the adjoint gather of a
voxel gradient back onto the control grid -- what every iteration of the FFD
registration loop computes.  ``value`` is voxels per second of that step,
summed over ranks (independent volumes per rank: weak scaling, no collective
on the data path).

Reported alongside (same run): forward-only FP32 and BF16, the adjoint alone,
the 512^3 spacing sweep, the 64-volume uneven batch (forward + adjoint, one
CUDA-graph replay per step), the end-to-end rate through the public API with
host buffers, the roofline of the dominant kernel against the measured HBM
peak, GPU clocks sampled during the timed region, and the FP64 CPU oracle
timed on the host cores on a bounded slab of the same workload.

``--impl reference`` times the FP64 oracle (the only reference this method
has: the paper ships no code) on the same workload and metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import pathlib
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = pathlib.Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "deformation-field Gvoxels/s (fwd, fwd+adjoint, batched) and % HBM roofline"
UNIT = "Gvoxels/s"
CT_SHAPE, CT_SPACING = (300, 512, 512), (5, 5, 5)
WORKLOAD = ("CT-shaped 512x512x300 voxels, spacing 5x5x5, FP32 control grid 106x106x63x3 "
            "(smooth Gaussian random field, std 3 voxels), forward + adjoint per step")


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)   # ~1 s timed: several clock samples
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-extras", action="store_true", help="main step only (profiling runs)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU-oracle leg")
    ap.add_argument("--section", choices=["resample", "batched", "rational"], default=None,
                    help="run only this extra measurement (profiling runs) and print its JSON")
    return ap.parse_args()


# ------------------------------------------------------------------ distributed

def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            import torch

            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, ws, device=None):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock / throttle samples in the background (200 ms period)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), [v.strip() for v in line.split(",")]))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self, t0, t1):
        rows = [s for (t, s) in self.samples if t0 <= t <= t1 and len(s) >= 9]
        window = "timed region"
        if not rows:  # short timed region: fall back to the whole sampled span
            rows = [s for (_, s) in self.samples if len(s) >= 9]
            window = "whole run (timed region shorter than one sample)"
        if not rows:
            return None

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "window": window,
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


# ------------------------------------------------------------------ helpers

def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_sources_sha():
    h = hashlib.sha256()
    for name in ("bsi_kernels.cuh", "bsi_async.cuh", "bsi_forward.cu", "bsi_adjoint.cu", "bsi_geometry.h",
                 "bsi_weights.cuh", "bsi_abi.cu", "bsi_launch.h"):
        h.update((ROOT / "paper_2004_05962_gb300" / "csrc" / name).read_bytes())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary and
    whether that capture was taken on the current kernel sources: (bytes, True),
    (bytes of an older capture, False) or (None, False)."""
    p = ROOT / "profiles" / "dram_traffic.md"
    if not p.exists():
        return None, False
    sha = kernel_sources_sha()
    old = None
    for line in p.read_text().splitlines():
        m = re.match(r"\|\s*(\S+)\s*\|\s*(\S+)\s*\|\s*([0-9.eE+]+)\s*\|\s*([0-9a-f]+)\s*\|", line)
        if m and m.group(1) == kernel:
            if m.group(4) == sha:
                return float(m.group(3)), True
            old = float(m.group(3))
    return old, False


def traffic_fields(kernels):
    """roofline.traffic (summed over `kernels`, null unless every capture is on
    the current sources) and a note that says which case applies."""
    got = [ncu_traffic(k) for k in kernels]
    if all(v is not None and fresh for v, fresh in got):
        return sum(v for v, _ in got), "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, profiles/dram_traffic.md"
    if all(v is not None for v, _ in got):
        return None, ("stale: the committed ncu capture (%.0f B) predates the current kernel sources %s"
                      % (sum(v for v, _ in got), kernel_sources_sha()))
    return None, "no ncu capture committed for these kernels"


# ------------------------------------------------------------------ our arm

def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    from paper_2004_05962_gb300 import build as pbuild

    pbuild.build()
    import paper_2004_05962_gb300 as P
    from paper_2004_05962_gb300 import model, synth

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    s = torch.cuda.current_stream(dev)
    shape, spacing = CT_SHAPE, CT_SPACING
    nvox = int(np.prod(shape))

    phi = torch.from_numpy(synth.gaussian_random_phi(shape, spacing, 3.0, 2.0, seed=2 + rank)).to(dev)
    grad = torch.from_numpy(synth.normal_field(shape, seed=4 + rank)).to(dev)
    field = torch.empty(shape + (3,), device=dev)
    dphi = torch.empty_like(phi)
    wsb = P.bsi_adjoint_workspace_bytes(shape, spacing)
    work = torch.empty(wsb, dtype=torch.uint8, device=dev)

    def step(ev=None):
        if ev is not None:
            ev[0].record(s)
        P.bsi_field_forward(phi, shape, spacing, out=field)
        if ev is not None:
            ev[1].record(s)
        P.bsi_field_adjoint(grad, spacing, out=dphi, workspace=work)
        if ev is not None:
            ev[2].record(s)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)

    def timed(with_events):
        barrier(ws)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for k in range(args.steps):
            step(evs[k] if with_events else None)
        e1.record(s)
        torch.cuda.synchronize()
        barrier(ws)
        return max_over_ranks(e0.elapsed_time(e1), ws, dev)

    # Timed region A, the throughput: K steps with nothing between the kernels,
    # so each launch may be scheduled while the previous one drains
    # (programmatic dependent launches).  Timed region B, the per-kernel split
    # the roofline reports: the same K steps with an event between the forward
    # and the adjoint -- an event between two kernels forgoes that overlap, so
    # B's steps run slower than A's.
    t0 = time.time()
    ms_total = timed(False)
    ms_total_b = timed(True)
    t1 = time.time()
    clk.stop()
    ms_step = ms_total / args.steps
    fwd_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    adj_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    value = ws * nvox / (ms_step * 1e-3) / 1e9
    launches = 3 * args.steps  # forward, adjoint partials, adjoint reduce per step (timed region A)

    hbm_peak, peak_kind = measured_peaks()
    fwd_bytes = model.forward_bytes(shape, spacing)
    adj_bytes = model.adjoint_bytes(shape, spacing)
    fwd_gbs = fwd_bytes / (fwd_ms * 1e-3) / 1e9
    adj_gbs = adj_bytes / (adj_ms * 1e-3) / 1e9
    dominant = "bsi_forward_kernel" if fwd_ms >= adj_ms else "bsi_field_adjoint (partials + reduce)"
    if fwd_ms >= adj_ms:
        tr, note = traffic_fields(["bsi_forward_kernel"])
        roof = {"kernel": "bsi_forward_kernel", "bound": "hbm", "achieved": round(fwd_gbs, 1),
                "peak": hbm_peak, "unit": "GB/s", "frac": round(fwd_gbs / hbm_peak, 4),
                "traffic": tr, "traffic_note": note,
                "algorithmic_bytes_per_launch": fwd_bytes, "avg_launch_ms": round(fwd_ms, 5),
                "peak_kind": f"{peak_kind} HBM copy (MEASURED_PEAKS.json hbm_gbs)"}
    else:
        # X % 4 == 0 and dx <= 8: the adjoint's tensor-copy partials kernel runs
        pk = "bsi_adjoint_partials_tma_kernel" if shape[2] % 4 == 0 and spacing[2] <= 8 else \
            "bsi_adjoint_partials_kernel"
        tr, note = traffic_fields([pk, "bsi_adjoint_reduce_kernel"])
        roof = {"kernel": f"{pk} + bsi_adjoint_reduce_kernel (one bsi_field_adjoint call)",
                "bound": "hbm", "achieved": round(adj_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(adj_gbs / hbm_peak, 4), "traffic": tr, "traffic_note": note,
                "algorithmic_bytes_per_launch": adj_bytes, "avg_launch_ms": round(adj_ms, 5),
                "peak_kind": f"{peak_kind} HBM copy (MEASURED_PEAKS.json hbm_gbs)"}

    # both kernels of the step, timed inside it (the dominant one is the roofline above)
    roof["in_step_how"] = ("CUDA events between the kernels over %d steps (timed region B: %.5f ms per step; "
                           "region A without the events: %.5f ms)" % (args.steps, ms_total_b / args.steps, ms_step))
    roof["in_step"] = {
        "forward": {"kernel": "bsi_forward_kernel", "ms": round(fwd_ms, 5), "gbs": round(fwd_gbs, 1),
                    "frac": round(fwd_gbs / hbm_peak, 4), "algorithmic_bytes": fwd_bytes},
        "adjoint": {"kernel": "bsi_field_adjoint (partials + reduce)", "ms": round(adj_ms, 5),
                    "gbs": round(adj_gbs, 1), "frac": round(adj_gbs / hbm_peak, 4), "algorithmic_bytes": adj_bytes}}

    extras = {}
    if not args.no_extras:
        extras = run_extras(args, P, synth, model, dev, s, phi, grad, field, dphi, work, hbm_peak)
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "volume_zyx": list(shape), "spacing_zyx": list(spacing),
                   "voxels_per_step_per_gpu": nvox, "step": "bsi_field_forward + bsi_field_adjoint",
                   "l2": "inputs larger than L2 (field 944 MB written, voxel gradient 944 MB read per step)",
                   "parallelism": f"{ws} independent volume(s), one per GPU"},
        "fwd_ms": round(fwd_ms, 5), "adjoint_ms": round(adj_ms, 5),
        "fwd_gbs": round(fwd_gbs, 1), "adjoint_gbs": round(adj_gbs, 1), "dominant_kernel": dominant,
        "roofline": roof, "gpu_launches": launches,
        "clocks": clk.summary(t0, t1),
    }
    out.update(extras)
    if "e2e" not in out:
        out["e2e"] = None

    def gpu_fields():
        """The step's FP32 field and its BF16 variant, for the oracle leg's error report."""
        f32 = P.bsi_field_forward(phi, shape, spacing)
        b16 = P.bsi_field_forward(phi, shape, spacing, out_dtype=torch.bfloat16)
        torch.cuda.synchronize()
        return f32, b16

    return out, gpu_fields


def time_fn(fn, s, iters, warm=3):
    import torch

    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(iters):
        fn()
    b.record(s)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / iters


def measure_resample(P, synth, model, dev, s, phi, field, dphi, hbm_peak, iters):
    """BSI fused with the resampling of a floating image on the CT volume: value
    and gradient with respect to phi; unfused context: our field, then torch's
    grid_sample."""
    import numpy as np
    import torch
    import torch.nn.functional as TF

    shape, spacing = CT_SHAPE, CT_SPACING
    nvox = int(np.prod(shape))

    F = torch.zeros(shape, device=dev)
    Z, Y, X = shape
    for c, sg, a in synth.blob_params(shape, seed=6):   # separable blobs, evaluated on the device
        ez = torch.exp(-((torch.arange(Z, device=dev) - c[0]) ** 2) / (2 * sg * sg))
        ey = torch.exp(-((torch.arange(Y, device=dev) - c[1]) ** 2) / (2 * sg * sg))
        ex = torch.exp(-((torch.arange(X, device=dev) - c[2]) ** 2) / (2 * sg * sg))
        F += a * ez[:, None, None] * ey[None, :, None] * ex[None, None, :]
    Wt = torch.empty(shape, device=dev)
    ms_rs = time_fn(lambda: P.bsi_resample_forward(phi, shape, spacing, F, out=Wt), s, iters)
    gW = torch.randn(shape, device=dev)
    wsr = torch.empty(P.bsi_resample_backward_workspace_bytes(shape, spacing), dtype=torch.uint8, device=dev)
    ms_rsb = time_fn(lambda: P.bsi_resample_backward(phi, shape, spacing, F, gW, out=dphi, workspace=wsr), s, 20)
    base = torch.stack(torch.meshgrid(torch.arange(X, device=dev), torch.arange(Y, device=dev),
                                      torch.arange(Z, device=dev), indexing="xy"), -1).float()
    base = base.permute(2, 0, 1, 3).contiguous()            # [Z, Y, X, 3] as (x, y, z)
    norm = torch.tensor([2.0 / (X - 1), 2.0 / (Y - 1), 2.0 / (Z - 1)], device=dev)

    def unfused():
        P.bsi_field_forward(phi, shape, spacing, out=field)
        grid = (base + field) * norm - 1.0
        return TF.grid_sample(F[None, None], grid[None], mode="bilinear", padding_mode="zeros", align_corners=True)

    ms_unf = time_fn(unfused, s, 10)
    agree = float((unfused()[0, 0] - P.bsi_resample_forward(phi, shape, spacing, F, out=Wt)).abs().max())
    rb = model.resample_bytes(shape, spacing)
    rbb = model.resample_backward_bytes(shape, spacing)
    return {
        "fwd_ms": round(ms_rs, 5), "fwd_gvox_s": round(nvox / ms_rs / 1e6, 2),
        "fwd_gbs": round(rb / ms_rs / 1e6, 1), "fwd_frac_of_hbm": round(rb / ms_rs / 1e6 / hbm_peak, 4),
        "fwd_algorithmic_bytes": rb,
        "bwd_ms": round(ms_rsb, 5), "bwd_gvox_s": round(nvox / ms_rsb / 1e6, 2),
        "bwd_gbs_algorithmic": round(rbb / ms_rsb / 1e6, 1),
        # the algorithmic bytes plus the voxel gradient G, written and read back once
        "bwd_bytes_moved": rbb + 24 * nvox,
        "bwd_bytes_moved_over_algorithmic": round((rbb + 24 * nvox) / rbb, 3),
        "unfused_field_plus_torch_grid_sample_ms": round(ms_unf, 5),
        "unfused_max_abs_diff": agree,
        "image": "sum of 8 Gaussian blobs (sigma 8-20 voxels), seed 6; phi = the bench's CT control grid"}


def batch_launches(shapes, spacings, max_batch=64):
    """Kernel launches of one batched forward + adjoint, by the library's grouping:
    forward -- x-spacing <= 8 and > 8 groups; adjoint -- tensor-copy (X % 4 == 0,
    dx <= 8; torch buffers are 16-byte aligned), row-copy (dx <= 8) and generic
    groups, each a partials and a reduce launch; at most 64 instances a launch."""
    def groups(keys):
        return sum(-(-keys.count(k) // max_batch) for k in set(keys))
    fwd = [sp[2] > 8 for sp in spacings]
    adj = [("tma" if (sh[2] % 4 == 0 and sp[2] <= 8) else ("row" if sp[2] <= 8 else "generic"))
           for sh, sp in zip(shapes, spacings)]
    return groups(fwd) + 2 * groups(adj)


def run_extras(args, P, synth, model, dev, s, phi, grad, field, dphi, work, hbm_peak):
    import numpy as np
    import torch

    shape, spacing = CT_SHAPE, CT_SPACING
    nvox = int(np.prod(shape))
    res = {}
    iters = 50

    # write-only HBM denominator: the library's own 2 GiB fill through the
    # forward's store path (bsi_probe_fill), best of 10
    buf = torch.empty(2 << 30, dtype=torch.uint8, device=dev)
    wbest = min(time_fn(lambda: P.bsi_probe_fill(buf, 7), s, 3, warm=1) for _ in range(10))
    write_peak = buf.numel() / wbest / 1e6
    del buf
    res["hbm_write_peak"] = {"gbs": round(write_peak, 1), "how": "bsi_probe_fill of 2 GiB, best of 10 x 3 launches",
                             "nominal_gbs": 7900.0}

    # forward-only FP32 / BF16 and adjoint-only on the CT volume
    ms = time_fn(lambda: P.bsi_field_forward(phi, shape, spacing, out=field), s, iters)
    b16 = torch.empty(shape + (3,), dtype=torch.bfloat16, device=dev)
    ms16 = time_fn(lambda: P.bsi_field_forward(phi, shape, spacing, out=b16), s, iters)
    msa = time_fn(lambda: P.bsi_field_adjoint(grad, spacing, out=dphi, workspace=work), s, iters)
    res["components"] = {
        "fwd_f32": {"gvox_s": round(nvox / ms / 1e6, 2), "ms": round(ms, 5),
                    "gbs": round(model.forward_bytes(shape, spacing) / ms / 1e6, 1),
                    "frac_of_write_peak": round(model.forward_bytes(shape, spacing) / ms / 1e6 / write_peak, 4),
                    "frac_of_nominal": round(model.forward_bytes(shape, spacing) / ms / 1e6 / 7900.0, 4)},
        "fwd_bf16": {"gvox_s": round(nvox / ms16 / 1e6, 2), "ms": round(ms16, 5),
                     "gbs": round(model.forward_bytes(shape, spacing, 2) / ms16 / 1e6, 1)},
        "adjoint": {"gvox_s": round(nvox / msa / 1e6, 2), "ms": round(msa, 5),
                    "gbs": round(model.adjoint_bytes(shape, spacing) / msa / 1e6, 1)},
    }
    del b16

    res["resample"] = measure_resample(P, synth, model, dev, s, phi, field, dphi, hbm_peak, iters)

    # the paper's thread-per-tile formulations (TT, TTLI) on the same volume
    pv = {}
    for v in ("tt", "ttli"):
        t = time_fn(lambda: P.bsi_field_forward_variant(phi, shape, spacing, v, out=field), s, 5)
        pv[v] = {"ms": round(t, 5), "gvox_s": round(nvox / t / 1e6, 2)}
    pv["separable_ms"] = res["components"]["fwd_f32"]["ms"]
    res["paper_tile_variants"] = pv

    res["rational_forward"] = measure_rational(P, model, dev, s, shape, field, hbm_peak, iters)

    # scalar BSI: a 4x zoom of a 128 x 128 x 75 image (its samples as control
    # points, one border sample below and two above) into the 512 x 512 x 300 volume
    zshape, zsp = (300, 512, 512), (4, 4, 4)
    img = torch.from_numpy(synth.blob_image(synth.grid_shape(zshape, zsp), seed=7)).to(dev)
    zout = torch.empty(zshape, device=dev)
    ms_z = time_fn(lambda: P.bsi_scalar_forward(img, zshape, zsp, out=zout), s, iters)
    zb = 4 * int(np.prod(zshape)) + 4 * img.numel()
    res["scalar_zoom"] = {"ms": round(ms_z, 5), "gvox_s": round(nvox / ms_z / 1e6, 2), "gbs": round(zb / ms_z / 1e6, 1),
                          "frac_of_hbm": round(zb / ms_z / 1e6 / hbm_peak, 4),
                          "workload": "4x zoom of a 78 x 131 x 131 grid (128 x 128 x 75 image + border) to 512 x 512 x 300, FP32"}
    del img, zout

    # 512^3 spacing sweep (forward FP32)
    sweep = {}
    big = (512, 512, 512)
    out = torch.empty(big + (3,), device=dev)
    for sp in [(3, 3, 3), (5, 5, 5), (6, 5, 4), (8, 8, 8)]:
        ph = torch.from_numpy(synth.uniform_phi(big, sp, -4, 4, seed=3)).to(dev)
        t = time_fn(lambda: P.bsi_field_forward(ph, big, sp, out=out), s, 20)
        gbs = model.forward_bytes(big, sp) / t / 1e6
        sweep["x".join(str(v) for v in sp[::-1])] = {
            "gvox_s": round(512 ** 3 / t / 1e6, 2), "ms": round(t, 5), "gbs": round(gbs, 1),
            "frac_of_copy_peak": round(gbs / hbm_peak, 4), "frac_of_write_probe": round(gbs / write_peak, 4),
            "frac_of_nominal": round(gbs / 7900.0, 4)}
    res["sweep_512cubed_fwd"] = sweep
    del out

    # 512^3 spacing sweep (adjoint)
    sweep = {}
    g = torch.randn(big + (3,), device=dev)
    for sp in [(3, 3, 3), (5, 5, 5), (6, 5, 4), (8, 8, 8)]:
        d_ = torch.empty(synth.grid_shape(big, sp) + (3,), device=dev)
        w_ = torch.empty(P.bsi_adjoint_workspace_bytes(big, sp), dtype=torch.uint8, device=dev)
        t = time_fn(lambda: P.bsi_field_adjoint(g, sp, out=d_, workspace=w_), s, 20)
        gbs = model.adjoint_bytes(big, sp) / t / 1e6
        sweep["x".join(str(v) for v in sp[::-1])] = {
            "gvox_s": round(512 ** 3 / t / 1e6, 2), "ms": round(t, 5), "gbs": round(gbs, 1),
            "frac_of_copy_peak": round(gbs / hbm_peak, 4), "frac_of_nominal": round(gbs / 7900.0, 4)}
        del d_, w_
    res["sweep_512cubed_adj"] = sweep
    del g

    # 64-volume uneven batch, forward + adjoint, replayed as one CUDA graph
    geoms = synth.batch_geometries(64, seed=5)
    shapes = [g[0] for g in geoms]
    spacings = [g[1] for g in geoms]
    bvox = sum(int(np.prod(x)) for x in shapes)
    phis = [torch.from_numpy(synth.uniform_phi(a, b, -3, 3, seed=500 + i)).to(dev) for i, (a, b) in enumerate(geoms)]
    grads = [torch.randn(a + (3,), device=dev) for a in shapes]
    outs = [torch.empty(a + (3,), device=dev) for a in shapes]
    dps = [torch.empty_like(p) for p in phis]
    bws = torch.empty(P.bsi_batched_adjoint_workspace_bytes(shapes, spacings), dtype=torch.uint8, device=dev)

    def bstep():
        P.bsi_field_forward_batched(phis, shapes, spacings, outs=outs)
        P.bsi_field_adjoint_batched(grads, spacings, outs=dps, workspace=bws)

    # untuned (library defaults), then ONE launch shape tuned for the whole batch
    # (timed in this run: the tuner's cache is bypassed)
    from paper_2004_05962_gb300 import tune

    t_default = time_fn(bstep, s, 10)
    t_tune0 = time.time()
    tuned = tune.tune_batched(shapes, spacings, iters=5, retune=True)
    tune_s = time.time() - t_tune0
    bws = torch.empty(P.bsi_batched_adjoint_workspace_bytes(shapes, spacings), dtype=torch.uint8, device=dev)

    side = torch.cuda.Stream(dev)
    side.wait_stream(s)
    with torch.cuda.stream(side):
        bstep()
    s.wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bstep()
    tb = time_fn(g.replay, s, 20)
    tbf = time_fn(lambda: P.bsi_field_forward_batched(phis, shapes, spacings, outs=outs), s, 20)
    res["batched_64"] = {"gvox_s_fwd_adj": round(bvox / tb / 1e6, 2), "ms_fwd_adj": round(tb, 5),
                         "gvox_s_fwd": round(bvox / tbf / 1e6, 2), "voxels": bvox,
                         "vs_single_volume_fwd": round((bvox / tbf) / (nvox / ms), 3),
                         "vs_single_volume_fwd_adj": round((bvox / tb) / (nvox / (ms + msa)), 3),
                         "launches_per_step": batch_launches(shapes, spacings), "cuda_graph": True,
                         "autotuned": {k: v for k, v in tuned.items() if k not in ("dx", "dy", "dz")},
                         "autotuned_scope": "one launch shape for the whole batch, timed in this run",
                         "spacing_classes": len(set(map(tuple, spacings))),
                         "tuning_s": round(tune_s, 1), "gvox_s_fwd_adj_untuned": round(bvox / t_default / 1e6, 2)}
    P.bsi_set_tile_configs([])
    del phis, grads, outs, dps, bws, g

    # end to end through the public API with host buffers.  Every step uploads
    # its inputs (phi and the voxel gradient, pinned host memory), runs forward +
    # adjoint, and reads its result -- the control-grid gradient, what a
    # registration step hands back -- to the host; the field stays on the device
    # (the next step of the registration consumes it there).  Steps are
    # pipelined as a user would: the upload of step k+1 and the read-back of
    # step k-1 overlap step k's kernels (double-buffered inputs and results,
    # ordered by events).  Timed from the first upload to the last read-back.
    phi_h = phi.cpu().pin_memory()
    grad_h = grad.cpu().pin_memory()
    dphi_h = [torch.empty(dphi.shape, dtype=dphi.dtype).pin_memory() for _ in range(2)]
    phi_d = [torch.empty_like(phi) for _ in range(2)]
    grad_d = [torch.empty_like(grad) for _ in range(2)]
    dphi_d = [torch.empty_like(dphi) for _ in range(2)]
    s_up, s_down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def e2e_run(nsteps):
        ev_up = [torch.cuda.Event() for _ in range(nsteps)]
        ev_comp = [torch.cuda.Event() for _ in range(nsteps)]
        ev_down = [torch.cuda.Event() for _ in range(nsteps)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(s)
        s_up.wait_event(t0)
        for k in range(nsteps):
            b = k % 2
            if k >= 2:
                s_up.wait_event(ev_comp[k - 2])      # buffer b's last readers are done
            with torch.cuda.stream(s_up):
                phi_d[b].copy_(phi_h, non_blocking=True)
                grad_d[b].copy_(grad_h, non_blocking=True)
                ev_up[k].record(s_up)
            s.wait_event(ev_up[k])
            if k >= 2:
                s.wait_event(ev_down[k - 2])         # dphi_d[b] has been read back
            P.bsi_field_forward(phi_d[b], shape, spacing, out=field, stream=s)
            P.bsi_field_adjoint(grad_d[b], spacing, out=dphi_d[b], workspace=work, stream=s)
            ev_comp[k].record(s)
            s_down.wait_event(ev_comp[k])
            with torch.cuda.stream(s_down):
                dphi_h[b].copy_(dphi_d[b], non_blocking=True)
                ev_down[k].record(s_down)
        s.wait_event(ev_down[nsteps - 1])
        t1.record(s)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / nsteps

    e2e_run(3)
    te = min(e2e_run(10), e2e_run(10))
    h2d = phi_h.numel() * 4 + grad_h.numel() * 4
    d2h = dphi_h[0].numel() * 4
    assert torch.equal(dphi_h[1].to(dev), P.bsi_field_adjoint(grad, spacing, workspace=work))
    # the host link's own rates, the e2e denominator: one pinned copy of the
    # step's largest input (the voxel gradient) host -> device and back, each
    # timed alone on a copy stream, best of 5
    back_h = torch.empty(grad.shape, dtype=grad.dtype).pin_memory()

    def copy_ms(fn, st):
        best = float("inf")
        for _ in range(6):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(st)
            with torch.cuda.stream(st):
                fn()
            b.record(st)
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        return best

    nb = grad_h.numel() * 4
    h2d_gbs = nb / copy_ms(lambda: grad_d[0].copy_(grad_h, non_blocking=True), s_up) / 1e6
    d2h_gbs = nb / copy_ms(lambda: back_h.copy_(grad_d[0], non_blocking=True), s_down) / 1e6
    # copies of one direction share a link direction; the two directions overlap
    bound_ms = max(h2d / h2d_gbs, d2h / d2h_gbs) / 1e6
    del back_h
    res["e2e"] = {"value": round(nvox / te / 1e6, 3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                  "d2h_bytes_per_step": d2h, "ms_per_step": round(te, 4),
                  "link": {"h2d_gbs": round(h2d_gbs, 1), "d2h_gbs": round(d2h_gbs, 1),
                           "how": f"one pinned {nb / 1e6:.0f} MB copy each way, best of 6",
                           "bound_gvox_s": round(nvox / bound_ms / 1e6, 3),
                           "frac_of_link_bound": round(bound_ms / te, 4)},
                  "how": "pinned host inputs uploaded every step, dL/dphi read back every step, field kept on "
                         "the device; uploads / read-backs of neighbouring steps overlap the kernels (2 copy streams)"}
    return res


# ------------------------------------------------------------------ oracle legs

def oracle_slab_rate(budget_s, shape=CT_SHAPE, spacing=CT_SPACING, seed=2, gpu_fields=None):
    """Times the FP64 oracle (forward + adjoint, all host cores) on a z-slab of the
    workload sized to ~budget_s seconds (planes [0, zs); the whole volume when it
    fits); returns (gvox_s, cores, sample text, errors).  With ``gpu_fields`` (a
    function returning the library's FP32 and BF16 fields of the same control
    grid, on the device), ``errors`` holds their max / mean absolute error
    against the oracle's forward over the timed planes (else None)."""
    import numpy as np

    import oracle
    from paper_2004_05962_gb300 import synth

    Z, Y, X = shape
    dz = spacing[0]
    phi = synth.gaussian_random_phi(shape, spacing, 3.0, 2.0, seed=seed)
    rng = np.random.default_rng(seed)

    def run(zs, keep=False):
        sub = (zs, Y, X)
        nzs = -(-zs // dz) + 3
        ph = np.ascontiguousarray(phi[:nzs])
        g = rng.standard_normal(sub + (3,), dtype=np.float32)
        t = time.perf_counter()
        f = oracle.forward(ph, sub, spacing)
        oracle.adjoint(g, spacing)
        return time.perf_counter() - t, (f if keep else None)

    t1, _ = run(1)
    zs = int(max(1, min(Z, budget_s / max(t1, 1e-6))))
    t, want = run(zs, keep=gpu_fields is not None)
    vox = zs * Y * X
    cores = oracle.threads()
    sample = f"forward + adjoint of a {X}x{Y}x{zs} z-slab (of {Z}) of the same workload, {t:.1f} s"
    errors = None
    if gpu_fields is not None:
        # planes [0, zs) of the whole volume's field need only grid planes
        # [0, ceil(zs / dz) + 3): the slab's forward is the volume's, voxel for voxel
        amax = float(np.abs(phi).max())
        errors = {}
        for name, dev_field in zip(("fwd_f32", "fwd_bf16"), gpu_fields()):
            mx, tot, over = 0.0, 0.0, 0
            for z0 in range(0, zs, 32):
                z1 = min(zs, z0 + 32)
                got = dev_field[z0:z1].float().cpu().numpy().astype(np.float64)
                w = want[z0:z1]
                d = np.abs(got - w)
                mx = max(mx, float(d.max()))
                tot += float(d.sum())
                if name == "fwd_bf16":
                    over += int(np.count_nonzero(d > 2.0 ** -8 * np.abs(w) + (1 + 2.0 ** -8) * 1e-5 * amax))
                else:
                    over += int(np.count_nonzero(d > 1e-5 * amax))
            e = {"max_abs": mx, "mean_abs": tot / (3.0 * vox), "max_abs_over_max_phi": mx / amax,
                 "voxels": vox, "beyond_bound": over}
            e["bound"] = ("|err| <= 2^-8 |T| + (1 + 2^-8) 1e-5 max|phi| (RNE of the FP32 field)" if name == "fwd_bf16"
                          else "|err| <= 1e-5 max|phi|")
            errors[name] = e
    return vox / t / 1e9, cores, sample, errors


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    import numpy as np

    import oracle
    from paper_2004_05962_gb300 import synth

    shape, spacing = CT_SHAPE, CT_SPACING
    Z, Y, X = shape
    # each step a z-slab sized so the whole run takes about 150 s of oracle time,
    # and no step more than --cpu-seconds
    per_step = min(args.cpu_seconds, max(0.5, 150.0 / max(1, args.steps + args.warmup)))
    phi = synth.gaussian_random_phi(shape, spacing, 3.0, 2.0, seed=2)
    rng = np.random.default_rng(4)

    def run(zs):
        sub = (zs, Y, X)
        nzs = -(-zs // spacing[0]) + 3
        g = rng.standard_normal(sub + (3,), dtype=np.float32)
        t = time.perf_counter()
        oracle.forward(np.ascontiguousarray(phi[:nzs]), sub, spacing)
        oracle.adjoint(g, spacing)
        return time.perf_counter() - t

    t1 = run(1)
    zs = int(max(1, min(Z, per_step / max(t1, 1e-6))))
    for _ in range(args.warmup):
        run(zs)
    times = [run(zs) for _ in range(args.steps)]
    tot = sum(times)
    vox = zs * Y * X
    value = args.steps * vox / tot / 1e9
    cores = oracle.threads()
    sample = f"forward + adjoint of a {X}x{Y}x{zs} z-slab (of {Z}) per step"
    return {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * tot / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "volume_zyx": list(shape), "spacing_zyx": list(spacing),
                       "reference": "FP64 CPU oracle of Eq. 1 and its transpose (the paper ships no code)"},
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}


def measure_rational(P, model, dev, s, shape, field, hbm_peak, iters):
    """Non-integer, non-aligned spacing: 4.7 voxels per axis, lattice shifted by
    0.3 / 0 / 0.9 voxels (z, y, x), on the 512 x 512 x 300 volume."""
    import torch

    nvox = shape[0] * shape[1] * shape[2]
    rn, rd, ro = (47, 47, 47), (10, 10, 10), (3, 0, 9)
    rgrid = P.rational_grid_shape(shape, rn, rd, ro)
    rphi = torch.rand(rgrid + (3,), device=dev) * 6.0 - 3.0
    ms_r = time_fn(lambda: P.bsi_field_forward_rational(rphi, shape, rn, rd, ro, out=field), s, iters)
    rb = model.forward_bytes(shape, (5, 5, 5)) - 12 * model.grid_points(shape, (5, 5, 5)) + 12 * rphi.numel() // 3
    # its transpose: the field buffer as the voxel gradient, dL/dphi into a grid-shaped buffer
    rdphi = torch.empty_like(rphi)
    rws = torch.empty(P.bsi_rational_adjoint_workspace_bytes(shape, rn, rd, ro), dtype=torch.uint8, device=dev)
    ms_a = time_fn(lambda: P.bsi_field_adjoint_rational(field, rn, rd, ro, out=rdphi, workspace=rws), s, iters)
    return {"ms": round(ms_r, 5), "gvox_s": round(nvox / ms_r / 1e6, 2),
            "gbs": round(rb / ms_r / 1e6, 1), "frac_of_hbm": round(rb / ms_r / 1e6 / hbm_peak, 4),
            "adjoint_ms": round(ms_a, 5), "adjoint_gvox_s": round(nvox / ms_a / 1e6, 2),
            "adjoint_gbs": round(rb / ms_a / 1e6, 1), "adjoint_frac_of_hbm": round(rb / ms_a / 1e6 / hbm_peak, 4),
            "adjoint_workspace_mb": round(rws.numel() / 1e6, 1),
            "workload": "512x512x300, spacing 4.7 voxels, lattice shift (0.3, 0, 0.9) (z, y, x), FP32"}


def run_section_rational(args):
    import torch

    from paper_2004_05962_gb300 import build as pbuild

    pbuild.build()
    import paper_2004_05962_gb300 as P
    from paper_2004_05962_gb300 import model

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    s = torch.cuda.current_stream(dev)
    field = torch.empty(CT_SHAPE + (3,), device=dev)
    hbm_peak, _ = measured_peaks()
    return {"section": "rational", "rational_forward": measure_rational(P, model, dev, s, CT_SHAPE, field, hbm_peak,
                                                                        args.steps)}


def run_section_resample(args):
    import torch

    from paper_2004_05962_gb300 import build as pbuild

    pbuild.build()
    import paper_2004_05962_gb300 as P
    from paper_2004_05962_gb300 import model, synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    s = torch.cuda.current_stream(dev)
    phi = torch.from_numpy(synth.gaussian_random_phi(CT_SHAPE, CT_SPACING, 3.0, 2.0, seed=2)).to(dev)
    field = torch.empty(CT_SHAPE + (3,), device=dev)
    dphi = torch.empty_like(phi)
    hbm_peak, _ = measured_peaks()
    return {"section": "resample", "workload": WORKLOAD,
            "resample": measure_resample(P, synth, model, dev, s, phi, field, dphi, hbm_peak, args.steps)}


def run_section_batched(args):
    """The 64-volume batch's forward + adjoint with library defaults, --steps
    times (profiling runs)."""
    import numpy as np
    import torch

    from paper_2004_05962_gb300 import build as pbuild

    pbuild.build()
    import paper_2004_05962_gb300 as P
    from paper_2004_05962_gb300 import synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    geoms = synth.batch_geometries(64, seed=5)
    shapes = [g[0] for g in geoms]
    spacings = [g[1] for g in geoms]
    phis = [torch.from_numpy(synth.uniform_phi(a, b, -3, 3, seed=500 + i)).to(dev) for i, (a, b) in enumerate(geoms)]
    grads = [torch.randn(a + (3,), device=dev) for a in shapes]
    outs = [torch.empty(a + (3,), device=dev) for a in shapes]
    dps = [torch.empty_like(p) for p in phis]
    bws = torch.empty(P.bsi_batched_adjoint_workspace_bytes(shapes, spacings), dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream(dev)

    def bstep():
        P.bsi_field_forward_batched(phis, shapes, spacings, outs=outs)
        P.bsi_field_adjoint_batched(grads, spacings, outs=dps, workspace=bws)

    ms = time_fn(bstep, s, args.steps)
    bvox = sum(int(np.prod(x)) for x in shapes)
    return {"section": "batched", "ms_fwd_adj": round(ms, 5), "gvox_s_fwd_adj": round(bvox / ms / 1e6, 2),
            "launches_per_step": batch_launches(shapes, spacings)}


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        out = run_reference(args, ws, rank)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if args.section == "resample":
        print(json.dumps(run_section_resample(args)), flush=True)
        return
    if args.section == "batched":
        print(json.dumps(run_section_batched(args)), flush=True)
        return
    if args.section == "rational":
        print(json.dumps(run_section_rational(args)), flush=True)
        return
    out, gpu_fields = run_ours(args, ws, rank, local)
    if rank == 0:
        if ws == 1 and not args.no_extras:
            v, cores, sample, errors = oracle_slab_rate(args.cpu_seconds, gpu_fields=gpu_fields)
            out["cpu_baseline"] = {"value": round(v, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
                                   "sample": sample}
            for name, e in (errors or {}).items():
                out["components"][name]["err_vs_oracle"] = e
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
