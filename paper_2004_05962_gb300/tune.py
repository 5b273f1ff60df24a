"""Autotuner of the kernels' launch shapes (``bsi_tile_config``) per spacing class.

For one spacing (dz, dy, dx) it times candidate shapes on a representative
volume with CUDA events -- forward: tiles per warp strip and warps per CTA;
adjoint: tile-planes per warp unit and warps per CTA -- keeps the fastest of
each, and returns one table entry.  The paper picked its block shape by hand
for each GPU (Sec. 3.4, Sec. 5.2); here the choice is measured on the GPU at
hand and cached in a JSON file keyed by GPU name, SM count, spacing and output
dtype, so later processes load it instead of re-timing.

Every candidate is a valid launch shape (the library checks the ranges), so
tuning changes speed only: the results of both kernels do not depend on the
shape except through FP32 summation order in the adjoint (parity tests run
under tuned shapes too).
"""
from __future__ import annotations

import json
import os
import pathlib

import torch

from . import bsi as B
from . import synth

DEFAULT_CACHE = pathlib.Path(__file__).resolve().parent / "_build" / "tile_configs.json"

FWD_STRIPS = (0, 24, 20, 16)          # 0: the library's aligned default (28 or 29)
ADJ_ZCHUNKS = (3, 4, 5, 6, 8)
WARPS = (0, 4)                        # forward, 0: as many as shared memory allows (8)
ADJ_WARPS = (0, 2)                    # adjoint, 0: the default 4


def _key(spacing, dtype, dev):
    p = torch.cuda.get_device_properties(dev)
    dz, dy, dx = spacing
    return f"{p.name}|sm{p.multi_processor_count}|{dx}x{dy}x{dz}|{str(dtype).replace('torch.', '')}"


def _time(fn, iters, stream):
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(iters):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / iters


def representative_shape(spacing, shapes=None, max_voxels=40_000_000):
    """The largest of ``shapes`` (those of a batch with this spacing), else a
    CT-like 160 x 256 x 256 volume; capped at ``max_voxels``."""
    cands = [tuple(s) for s in (shapes or [])]
    shape = max(cands, key=lambda s: s[0] * s[1] * s[2]) if cands else (160, 256, 256)
    Z, Y, X = shape
    while Z * Y * X > max_voxels and Z > 8:
        Z //= 2
    return (Z, Y, X)


def tune_spacing(spacing, shape=None, dtype=torch.float32, iters=10, device=None, seed=0):
    """Times the candidates for one spacing on a volume of ``shape`` and returns
    the chosen table entry (a dict), with the measured times under "_ms"."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    shape = tuple(shape) if shape is not None else representative_shape(spacing)
    dz, dy, dx = (int(s) for s in spacing)
    stream = torch.cuda.current_stream(dev)
    phi = torch.from_numpy(synth.uniform_phi(shape, spacing, -2, 2, seed)).to(dev)
    out = torch.empty(shape + (3,), dtype=dtype, device=dev)
    grad = torch.randn(shape + (3,), device=dev)
    dphi = torch.empty_like(phi)
    saved = B.bsi_tile_configs()
    base = {"dx": dx, "dy": dy, "dz": dz}
    times = {}
    try:
        best_f, best_f_ms = None, float("inf")
        for strip in FWD_STRIPS:
            for w in WARPS:
                cfg = dict(base, fwd_strip_tiles=strip, fwd_warps=w)
                B.bsi_set_tile_configs([cfg])
                ms = _time(lambda: B.bsi_field_forward(phi, shape, spacing, out=out), iters, stream)
                times[f"fwd strip={strip} warps={w}"] = ms
                if ms < best_f_ms:
                    best_f, best_f_ms = cfg, ms
        best_a, best_a_ms = None, float("inf")
        for zc in ADJ_ZCHUNKS:
            for w in ADJ_WARPS:
                cfg = dict(base, adj_zchunk=zc, adj_warps=w)
                B.bsi_set_tile_configs([cfg])
                ws = torch.empty(B.bsi_adjoint_workspace_bytes(shape, spacing), dtype=torch.uint8, device=dev)
                ms = _time(lambda: B.bsi_field_adjoint(grad, spacing, out=dphi, workspace=ws), iters, stream)
                times[f"adj zchunk={zc} warps={w}"] = ms
                if ms < best_a_ms:
                    best_a, best_a_ms = cfg, ms
    finally:
        B.bsi_set_tile_configs(saved)
    entry = dict(base, adj_zchunk=best_a["adj_zchunk"], adj_warps=best_a["adj_warps"],
                 fwd_strip_tiles=best_f["fwd_strip_tiles"], fwd_warps=best_f["fwd_warps"])
    entry["_ms"] = {"fwd": best_f_ms, "adj": best_a_ms, "shape_zyx": list(shape), "candidates": times}
    return entry


def load_cache(path=DEFAULT_CACHE):
    p = pathlib.Path(path)
    return json.loads(p.read_text()) if p.exists() else {}


def save_cache(cache, path=DEFAULT_CACHE):
    p = pathlib.Path(path)
    p.parent.mkdir(parents=True, exist_ok=True)
    tmp = p.with_name(p.name + f".tmp{os.getpid()}")
    tmp.write_text(json.dumps(cache, indent=1, sort_keys=True))
    os.replace(tmp, p)


def _batch_key(shapes, spacings, dtype, dev):
    import hashlib

    p = torch.cuda.get_device_properties(dev)
    h = hashlib.sha256(repr((list(map(tuple, shapes)), list(map(tuple, spacings)))).encode()).hexdigest()[:16]
    return f"{p.name}|sm{p.multi_processor_count}|batch{len(shapes)}:{h}|{str(dtype).replace('torch.', '')}"


def tune_batched(shapes, spacings, dtype=torch.float32, cache_path=DEFAULT_CACHE, retune=False, iters=5,
                 apply=True, seed=0):
    """Tunes ONE launch shape for a whole batch by timing the batched forward and
    adjoint themselves (all instances share a launch, so per-volume optima do not
    compose: one class asking for fewer warps slows every volume of its launch).
    Installs (with ``apply``) and returns the single wildcard table entry."""
    dev = torch.device("cuda", torch.cuda.current_device())
    cache = load_cache(cache_path) if cache_path else {}
    k = _batch_key(shapes, spacings, dtype, dev)
    if retune or k not in cache:
        stream = torch.cuda.current_stream(dev)
        shapes = [tuple(int(v) for v in s) for s in shapes]
        phis = [torch.from_numpy(synth.uniform_phi(s, d, -2, 2, seed + i)).to(dev)
                for i, (s, d) in enumerate(zip(shapes, spacings))]
        outs = [torch.empty(s + (3,), dtype=dtype, device=dev) for s in shapes]
        grads = [torch.randn(s + (3,), device=dev) for s in shapes]
        dps = [torch.empty_like(p) for p in phis]
        saved = B.bsi_tile_configs()
        times = {}
        try:
            best_f, best_f_ms = None, float("inf")
            for strip in FWD_STRIPS:
                for w in WARPS:
                    cfg = {"fwd_strip_tiles": strip, "fwd_warps": w}
                    B.bsi_set_tile_configs([cfg])
                    ms = _time(lambda: B.bsi_field_forward_batched(phis, shapes, spacings, outs=outs), iters, stream)
                    times[f"fwd strip={strip} warps={w}"] = ms
                    if ms < best_f_ms:
                        best_f, best_f_ms = cfg, ms
            best_a, best_a_ms = None, float("inf")
            for zc in ADJ_ZCHUNKS:
                for w in ADJ_WARPS:
                    cfg = {"adj_zchunk": zc, "adj_warps": w}
                    B.bsi_set_tile_configs([cfg])
                    ws = torch.empty(B.bsi_batched_adjoint_workspace_bytes(shapes, spacings), dtype=torch.uint8,
                                     device=dev)
                    ms = _time(lambda: B.bsi_field_adjoint_batched(grads, spacings, outs=dps, workspace=ws),
                               iters, stream)
                    times[f"adj zchunk={zc} warps={w}"] = ms
                    if ms < best_a_ms:
                        best_a, best_a_ms = cfg, ms
        finally:
            B.bsi_set_tile_configs(saved)
        entry = {"dx": 0, "dy": 0, "dz": 0, **best_f, **best_a}
        entry["_ms"] = {"fwd": best_f_ms, "adj": best_a_ms, "candidates": times}
        cache[k] = entry
        if cache_path:
            save_cache(cache, cache_path)
    e = {f: cache[k].get(f, 0) for f in B.BsiTileConfig.FIELDS}
    if apply:
        B.bsi_set_tile_configs([e])
    return e


def tune(spacings, shapes=None, dtype=torch.float32, cache_path=DEFAULT_CACHE, retune=False, iters=10,
         apply=True):
    """Tunes (or loads from the cache) every distinct spacing of a workload of
    single-volume calls and, with ``apply``, installs the table in the library.
    ``shapes`` (parallel to ``spacings``) picks the representative volume of each
    spacing.  Returns the table entries (cache bookkeeping keys stripped).  For
    batched calls use tune_batched."""
    dev = torch.device("cuda", torch.cuda.current_device())
    cache = load_cache(cache_path) if cache_path else {}
    by_spacing = {}
    for i, sp in enumerate(spacings):
        by_spacing.setdefault(tuple(int(v) for v in sp), []).append(shapes[i] if shapes is not None else None)
    entries, dirty = [], False
    for sp, shs in by_spacing.items():
        k = _key(sp, dtype, dev)
        if retune or k not in cache:
            shape = representative_shape(sp, [s for s in shs if s is not None])
            cache[k] = tune_spacing(sp, shape, dtype=dtype, iters=iters, device=dev)
            dirty = True
        entries.append({f: cache[k][f] for f in B.BsiTileConfig.FIELDS})
    if dirty and cache_path:
        save_cache(cache, cache_path)
    if apply:
        B.bsi_set_tile_configs(entries)
    return entries
