"""Python binding of the C ABI in include/bsi.h (ctypes; argument marshalling only).

Every computation runs in the sm_103a kernels of ``_build/libbsi_gb300.so``;
this module only checks tensor shapes and dtypes, builds the C structs and
passes raw device pointers and the current CUDA stream.  PyTorch supplies
device memory and streams.  There is no CPU fallback: if the library is
missing every call raises ``BsiLibraryMissing``.

Python shapes follow array order: ``shape = (Z, Y, X)`` voxels and
``spacing = (dz, dy, dx)`` voxels; a control grid is a float32 tensor
``[nz, ny, nx, 3]`` and a field ``[Z, Y, X, 3]`` (float32 or bfloat16).
The function names are those of the C entry points.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

BSI_F32, BSI_BF16 = 0, 1
STATUS = {
    0: "BSI_OK", 1: "BSI_ERR_NULL", 2: "BSI_ERR_DIMS", 3: "BSI_ERR_SPACING",
    4: "BSI_ERR_GRID_MISMATCH", 5: "BSI_ERR_DTYPE", 6: "BSI_ERR_ALIGN", 7: "BSI_ERR_WORKSPACE",
    8: "BSI_ERR_CUDA", 9: "BSI_ERR_DEVICE_STATUS", 10: "BSI_ERR_BATCH", 11: "BSI_ERR_SCRATCH_LIMIT",
}


class BsiLibraryMissing(RuntimeError):
    pass


class BsiError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {STATUS.get(status, status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


class BsiGeom(ctypes.Structure):
    _fields_ = [("X", ctypes.c_int64), ("Y", ctypes.c_int64), ("Z", ctypes.c_int64),
                ("dx", ctypes.c_int32), ("dy", ctypes.c_int32), ("dz", ctypes.c_int32),
                ("reserved", ctypes.c_int32),
                ("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64)]


class BsiGeomRational(ctypes.Structure):
    _fields_ = [("X", ctypes.c_int64), ("Y", ctypes.c_int64), ("Z", ctypes.c_int64),
                ("num", ctypes.c_int32 * 3), ("den", ctypes.c_int32 * 3), ("off", ctypes.c_int32 * 3),
                ("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64)]


class BsiInstance(ctypes.Structure):
    _fields_ = [("geom", BsiGeom), ("phi", ctypes.c_void_p), ("field", ctypes.c_void_p),
                ("grad_field", ctypes.c_void_p), ("grad_phi", ctypes.c_void_p)]


class BsiTileConfig(ctypes.Structure):
    _fields_ = [("dx", ctypes.c_int32), ("dy", ctypes.c_int32), ("dz", ctypes.c_int32),
                ("adj_zchunk", ctypes.c_int32), ("adj_warps", ctypes.c_int32),
                ("fwd_strip_tiles", ctypes.c_int32), ("fwd_warps", ctypes.c_int32)]

    FIELDS = ("dx", "dy", "dz", "adj_zchunk", "adj_warps", "fwd_strip_tiles", "fwd_warps")

    def as_dict(self):
        return {k: int(getattr(self, k)) for k in self.FIELDS}


_LIBS: dict = {}
_USE_CHECKED = os.environ.get("BSI_CHECKED", "0") == "1"


def set_checked(flag: bool) -> None:
    """Routes the entry points of this module to the bounds-checked build
    (``True``) or the release build (``False``)."""
    global _USE_CHECKED
    _USE_CHECKED = bool(flag)


def library(checked: bool | None = None) -> ctypes.CDLL:
    """The loaded C library.  ``checked`` (default: env BSI_CHECKED=1, or the last
    ``set_checked``) selects the bounds-checked build."""
    if checked is None:
        checked = _USE_CHECKED
    if checked in _LIBS:
        return _LIBS[checked]
    path = _build.lib_path(checked)
    if not path.exists():
        raise BsiLibraryMissing(
            f"{path} not found: build it with `python -m paper_2004_05962_gb300.build"
            f"{' --checked' if checked else ''}` (or __graft_entry__.build()).  "
            "There is no CPU fallback.")
    lib = ctypes.CDLL(str(path))
    vp, i32, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    G = ctypes.POINTER(BsiGeom)
    I = ctypes.POINTER(BsiInstance)
    sig = {
        "bsi_geom_init": (i32, [G, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                ctypes.c_int32, ctypes.c_int32]),
        "bsi_field_forward": (i32, [G, vp, vp, i32, vp]),
        "bsi_adjoint_workspace_bytes": (sz, [G]),
        "bsi_field_adjoint": (i32, [G, vp, vp, vp, sz, vp]),
        "bsi_field_forward_batched": (i32, [I, i32, i32, vp]),
        "bsi_batched_adjoint_workspace_bytes": (sz, [I, i32]),
        "bsi_field_adjoint_batched": (i32, [I, i32, vp, sz, vp]),
        "bsi_status_string": (ctypes.c_char_p, [i32]),
        "bsi_last_cuda_error": (ctypes.c_char_p, []),
        "bsi_check_device_status": (i32, [vp, ctypes.POINTER(ctypes.c_uint32)]),
        "bsi_version": (i32, []),
        "bsi_selfcheck_ranges": (i32, [I, i32, i32, i32, ctypes.c_char_p, sz]),
        "bsi_field_adjoint_noalloc": (i32, [G, vp, vp, vp]),
        "bsi_set_tile_configs": (i32, [ctypes.POINTER(BsiTileConfig), i32]),
        "bsi_get_tile_config": (i32, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.POINTER(BsiTileConfig)]),
        "bsi_probe_fill": (i32, [vp, sz, ctypes.c_uint32, vp]),
        "bsi_selftest_lost_copy": (i32, [vp]),
        "bsi_scalar_forward": (i32, [G, vp, vp, i32, vp]),
        "bsi_field_forward_variant": (i32, [G, vp, vp, ctypes.c_int32, vp]),
        "bsi_geom_rational_init": (i32, [ctypes.POINTER(BsiGeomRational), ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_int64, vp, vp, vp]),
        "bsi_field_forward_rational": (i32, [ctypes.POINTER(BsiGeomRational), vp, vp, vp]),
        "bsi_rational_adjoint_workspace_bytes": (sz, [ctypes.POINTER(BsiGeomRational)]),
        "bsi_field_adjoint_rational": (i32, [ctypes.POINTER(BsiGeomRational), vp, vp, vp, sz, vp]),
        "bsi_resample_forward": (i32, [G, vp, vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, vp, vp]),
        "bsi_resample_backward_workspace_bytes": (sz, [G]),
        "bsi_resample_backward": (i32, [G, vp, vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, vp, vp, vp,
                                        sz, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIBS[checked] = lib
    return lib


def exported_symbols():
    return ["bsi_geom_init", "bsi_field_forward", "bsi_adjoint_workspace_bytes", "bsi_field_adjoint",
            "bsi_field_forward_batched", "bsi_batched_adjoint_workspace_bytes",
            "bsi_field_adjoint_batched", "bsi_status_string", "bsi_last_cuda_error",
            "bsi_check_device_status", "bsi_version", "bsi_selfcheck_ranges",
            "bsi_field_adjoint_noalloc", "bsi_set_tile_configs", "bsi_get_tile_config", "bsi_probe_fill",
            "bsi_resample_forward", "bsi_resample_backward_workspace_bytes", "bsi_resample_backward",
            "bsi_scalar_forward", "bsi_field_forward_variant", "bsi_geom_rational_init",
            "bsi_field_forward_rational", "bsi_rational_adjoint_workspace_bytes", "bsi_field_adjoint_rational",
            "bsi_selftest_lost_copy"]


def bsi_set_tile_configs(configs) -> None:
    """Replaces the library's launch-shape table with ``configs`` (a list of dicts
    with keys dx, dy, dz, adj_zchunk, adj_warps, fwd_strip_tiles, fwd_warps;
    missing keys are 0 = default / wildcard)."""
    global _TILE_TABLE
    arr = (BsiTileConfig * max(1, len(configs)))()
    for i, c in enumerate(configs):
        for k in BsiTileConfig.FIELDS:
            setattr(arr[i], k, int(c.get(k, 0)))
    _check(library().bsi_set_tile_configs(arr, len(configs)), "bsi_set_tile_configs")
    _TILE_TABLE = [{k: int(c.get(k, 0)) for k in BsiTileConfig.FIELDS} for c in configs]


_TILE_TABLE: list = []


def bsi_tile_configs() -> list:
    """The table last installed through this module (a copy)."""
    return [dict(c) for c in _TILE_TABLE]


def bsi_get_tile_config(spacing) -> dict:
    """The launch shape the library uses for spacing (dz, dy, dx)."""
    dz, dy, dx = (int(s) for s in spacing)
    c = BsiTileConfig()
    _check(library().bsi_get_tile_config(dx, dy, dz, ctypes.byref(c)), "bsi_get_tile_config")
    return c.as_dict()


# ---------------------------------------------------------------- helpers

def grid_shape(shape, spacing):
    """Control-grid dims (nz, ny, nx) = ceil(N/d) + 3 per axis."""
    Z, Y, X = (int(s) for s in shape)
    dz, dy, dx = (int(s) for s in spacing)
    return (-(-Z // dz) + 3, -(-Y // dy) + 3, -(-X // dx) + 3)


def make_geom(shape, spacing) -> BsiGeom:
    Z, Y, X = (int(s) for s in shape)
    dz, dy, dx = (int(s) for s in spacing)
    g = BsiGeom()
    st = library().bsi_geom_init(ctypes.byref(g), X, Y, Z, dx, dy, dz)
    if st:
        raise BsiError(st, "bsi_geom_init", f"shape={shape} spacing={spacing}")
    return g


def _stream(stream, device) -> int:
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return int(stream.cuda_stream)


def _check(st, where):
    if st:
        detail = library().bsi_last_cuda_error().decode() if st == 8 else ""
        raise BsiError(st, where, detail)


def _need(t, name, dtype, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _out_dtype_code(dtype):
    if dtype == torch.float32:
        return BSI_F32
    if dtype == torch.bfloat16:
        return BSI_BF16
    raise ValueError(f"field dtype must be float32 or bfloat16, got {dtype}")


# ---------------------------------------------------------------- entry points

def bsi_field_forward(phi, shape, spacing, out=None, out_dtype=torch.float32, stream=None):
    """Dense field [Z, Y, X, 3] from the control grid ``phi`` [nz, ny, nx, 3] (Eq. 1)."""
    shape = tuple(int(s) for s in shape)
    _need(phi, "phi", torch.float32, grid_shape(shape, spacing) + (3,))
    if out is None:
        out = torch.empty(shape + (3,), dtype=out_dtype, device=phi.device)
    _need(out, "out", out.dtype, shape + (3,))
    g = make_geom(shape, spacing)
    st = library().bsi_field_forward(ctypes.byref(g), phi.data_ptr(), out.data_ptr(),
                                     _out_dtype_code(out.dtype), _stream(stream, phi.device))
    _check(st, "bsi_field_forward")
    return out


def bsi_adjoint_workspace_bytes(shape, spacing) -> int:
    g = make_geom(shape, spacing)
    return int(library().bsi_adjoint_workspace_bytes(ctypes.byref(g)))


def _workspace(nbytes, device, workspace):
    if nbytes == 0:
        return workspace, 0
    if workspace is None:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
    if not workspace.is_cuda or workspace.numel() * workspace.element_size() < nbytes:
        raise ValueError(f"workspace must be a CUDA tensor of at least {nbytes} bytes")
    return workspace, workspace.numel() * workspace.element_size()


def bsi_field_adjoint(grad_field, spacing, out=None, workspace=None, stream=None):
    """Transpose of Eq. 1: control-grid gradient [nz, ny, nx, 3] from a voxel
    gradient [Z, Y, X, 3] (float32).  ``workspace`` (uint8 CUDA tensor) is
    allocated through PyTorch when not given."""
    _need(grad_field, "grad_field", torch.float32)
    if grad_field.dim() != 4 or grad_field.shape[3] != 3:
        raise ValueError("grad_field must be [Z, Y, X, 3]")
    shape = tuple(grad_field.shape[:3])
    grid = grid_shape(shape, spacing)
    if out is None:
        out = torch.empty(grid + (3,), dtype=torch.float32, device=grad_field.device)
    _need(out, "out", torch.float32, grid + (3,))
    g = make_geom(shape, spacing)
    need = int(library().bsi_adjoint_workspace_bytes(ctypes.byref(g)))
    ws, wsb = _workspace(need, grad_field.device, workspace)
    st = library().bsi_field_adjoint(ctypes.byref(g), grad_field.data_ptr(), out.data_ptr(),
                                     ws.data_ptr() if ws is not None else None, wsb,
                                     _stream(stream, grad_field.device))
    _check(st, "bsi_field_adjoint")
    return out


def bsi_field_adjoint_noalloc(grad_field, spacing, out=None, stream=None):
    """``bsi_field_adjoint`` without a workspace argument: the partial sums go to
    a fixed 64 MiB device array inside the library, for callers that cannot
    allocate device memory.  Calls that overlap on the GPU race on that array."""
    _need(grad_field, "grad_field", torch.float32)
    if grad_field.dim() != 4 or grad_field.shape[3] != 3:
        raise ValueError("grad_field must be [Z, Y, X, 3]")
    shape = tuple(grad_field.shape[:3])
    grid = grid_shape(shape, spacing)
    if out is None:
        out = torch.empty(grid + (3,), dtype=torch.float32, device=grad_field.device)
    _need(out, "out", torch.float32, grid + (3,))
    g = make_geom(shape, spacing)
    st = library().bsi_field_adjoint_noalloc(ctypes.byref(g), grad_field.data_ptr(), out.data_ptr(),
                                             _stream(stream, grad_field.device))
    _check(st, "bsi_field_adjoint_noalloc")
    return out


def _instances(shapes, spacings, phis=None, fields=None, grads=None, dphis=None):
    n = len(shapes)
    arr = (BsiInstance * max(n, 1))()
    for i in range(n):
        arr[i].geom = make_geom(shapes[i], spacings[i])
        arr[i].phi = phis[i].data_ptr() if phis is not None else None
        arr[i].field = fields[i].data_ptr() if fields is not None else None
        arr[i].grad_field = grads[i].data_ptr() if grads is not None else None
        arr[i].grad_phi = dphis[i].data_ptr() if dphis is not None else None
    return arr


def bsi_field_forward_batched(phis, shapes, spacings, outs=None, out_dtype=torch.float32, stream=None):
    """Forward over a batch of volumes of uneven size and spacing (persistent launch)."""
    n = len(phis)
    shapes = [tuple(int(s) for s in sh) for sh in shapes]
    for i in range(n):
        _need(phis[i], f"phis[{i}]", torch.float32, grid_shape(shapes[i], spacings[i]) + (3,))
    if outs is None:
        outs = [torch.empty(shapes[i] + (3,), dtype=out_dtype, device=phis[i].device) for i in range(n)]
    dt = outs[0].dtype if n else out_dtype
    for i in range(n):
        _need(outs[i], f"outs[{i}]", dt, shapes[i] + (3,))
    arr = _instances(shapes, spacings, phis=phis, fields=outs)
    dev = phis[0].device if n else torch.device("cuda")
    st = library().bsi_field_forward_batched(arr, n, _out_dtype_code(dt), _stream(stream, dev))
    _check(st, "bsi_field_forward_batched")
    return outs


def bsi_batched_adjoint_workspace_bytes(shapes, spacings) -> int:
    arr = _instances([tuple(s) for s in shapes], spacings)
    return int(library().bsi_batched_adjoint_workspace_bytes(arr, len(shapes)))


def bsi_field_adjoint_batched(grads, spacings, outs=None, workspace=None, stream=None):
    """Adjoint over a batch: one partial-sum launch over all volumes, one reduce."""
    n = len(grads)
    shapes = []
    for i in range(n):
        _need(grads[i], f"grads[{i}]", torch.float32)
        shapes.append(tuple(grads[i].shape[:3]))
    if outs is None:
        outs = [torch.empty(grid_shape(shapes[i], spacings[i]) + (3,), dtype=torch.float32,
                            device=grads[i].device) for i in range(n)]
    for i in range(n):
        _need(outs[i], f"outs[{i}]", torch.float32, grid_shape(shapes[i], spacings[i]) + (3,))
    arr = _instances(shapes, spacings, grads=grads, dphis=outs)
    dev = grads[0].device if n else torch.device("cuda")
    need = int(library().bsi_batched_adjoint_workspace_bytes(arr, n))
    ws, wsb = _workspace(need, dev, workspace)
    st = library().bsi_field_adjoint_batched(arr, n, ws.data_ptr() if ws is not None else None, wsb,
                                             _stream(stream, dev))
    _check(st, "bsi_field_adjoint_batched")
    return outs


def make_geom_rational(shape, num, den, off):
    """bsi_geom_rational for a (Z, Y, X) volume; num, den, off in (z, y, x) order."""
    Z, Y, X = (int(v) for v in shape)
    arr = lambda a: (ctypes.c_int32 * 3)(*[int(v) for v in tuple(a)[::-1]])   # to (x, y, z)
    g = BsiGeomRational()
    st = library().bsi_geom_rational_init(ctypes.byref(g), X, Y, Z, arr(num), arr(den), arr(off))
    _check(st, "bsi_geom_rational_init")
    return g


def rational_grid_shape(shape, num, den, off):
    """Stored grid (nz, ny, nx) for spacing num/den and lattice shift off/den voxels
    per axis ((z, y, x) order): floor(((N - 1) den + off) / num) + 4."""
    return tuple(((int(N) - 1) * int(d) + int(o)) // int(n) + 4 if int(N) > 0 else 4
                 for N, n, d, o in zip(shape, num, den, off))


def bsi_field_forward_rational(phi, shape, num, den, off=(0, 0, 0), out=None, stream=None):
    """Eq. 1 with non-integer spacing num/den and lattice shift off/den voxels per
    axis ((z, y, x) order like ``shape``): FP32 field [Z, Y, X, 3]."""
    shape = tuple(int(s) for s in shape)
    _need(phi, "phi", torch.float32, rational_grid_shape(shape, num, den, off) + (3,))
    if out is None:
        out = torch.empty(shape + (3,), dtype=torch.float32, device=phi.device)
    _need(out, "out", torch.float32, shape + (3,))
    g = make_geom_rational(shape, num, den, off)
    st = library().bsi_field_forward_rational(ctypes.byref(g), phi.data_ptr(), out.data_ptr(),
                                              _stream(stream, phi.device))
    _check(st, "bsi_field_forward_rational")
    return out


def bsi_rational_adjoint_workspace_bytes(shape, num, den, off=(0, 0, 0)) -> int:
    return int(library().bsi_rational_adjoint_workspace_bytes(ctypes.byref(make_geom_rational(shape, num, den, off))))


def bsi_field_adjoint_rational(grad_field, num, den, off=(0, 0, 0), out=None, workspace=None, stream=None):
    """Transpose of bsi_field_forward_rational: dphi [nz, ny, nx, 3] from
    grad_field [Z, Y, X, 3] (FP32); num, den, off in (z, y, x) order."""
    _need(grad_field, "grad_field", torch.float32)
    if grad_field.dim() != 4 or grad_field.shape[3] != 3:
        raise ValueError("grad_field must be [Z, Y, X, 3]")
    shape = tuple(int(s) for s in grad_field.shape[:3])
    grid = rational_grid_shape(shape, num, den, off)
    if out is None:
        out = torch.empty(grid + (3,), dtype=torch.float32, device=grad_field.device)
    _need(out, "out", torch.float32, grid + (3,))
    g = make_geom_rational(shape, num, den, off)
    nbytes = int(library().bsi_rational_adjoint_workspace_bytes(ctypes.byref(g)))
    ws, wsb = _workspace(nbytes, grad_field.device, workspace)
    st = library().bsi_field_adjoint_rational(ctypes.byref(g), grad_field.data_ptr(), out.data_ptr(),
                                              ws.data_ptr() if ws is not None else None, wsb,
                                              _stream(stream, grad_field.device))
    _check(st, "bsi_field_adjoint_rational")
    return out


VARIANTS = {"separable": 0, "tt": 1, "ttli": 2}


def bsi_field_forward_variant(phi, shape, spacing, variant="ttli", out=None, stream=None):
    """Dense FP32 field by one of the paper's GPU formulations ("tt": thread per
    tile, "ttli": thread per tile with trilinear interpolations) or the
    separable kernel ("separable")."""
    shape = tuple(int(s) for s in shape)
    _need(phi, "phi", torch.float32, grid_shape(shape, spacing) + (3,))
    if out is None:
        out = torch.empty(shape + (3,), dtype=torch.float32, device=phi.device)
    _need(out, "out", torch.float32, shape + (3,))
    g = make_geom(shape, spacing)
    st = library().bsi_field_forward_variant(ctypes.byref(g), phi.data_ptr(), out.data_ptr(), VARIANTS[variant],
                                             _stream(stream, phi.device))
    _check(st, "bsi_field_forward_variant")
    return out


def bsi_scalar_forward(coeff, shape, spacing, out=None, out_dtype=torch.float32, stream=None):
    """Scalar BSI (image interpolation / zooming): [Z, Y, X] from a one-channel
    control grid ``coeff`` [nz, ny, nx] (Eq. 1 with one channel)."""
    shape = tuple(int(s) for s in shape)
    _need(coeff, "coeff", torch.float32, grid_shape(shape, spacing))
    if out is None:
        out = torch.empty(shape, dtype=out_dtype, device=coeff.device)
    _need(out, "out", out.dtype, shape)
    g = make_geom(shape, spacing)
    st = library().bsi_scalar_forward(ctypes.byref(g), coeff.data_ptr(), out.data_ptr(), _out_dtype_code(out.dtype),
                                      _stream(stream, coeff.device))
    _check(st, "bsi_scalar_forward")
    return out


def _floating(image):
    _need(image, "image", torch.float32, tuple(image.shape))
    if image.dim() != 3:
        raise ValueError("the floating image is [fZ, fY, fX]")
    fZ, fY, fX = (int(v) for v in image.shape)
    return fX, fY, fZ


def bsi_resample_forward(phi, shape, spacing, image, out=None, stream=None):
    """Floating ``image`` [fZ, fY, fX] sampled at x + T(x) (T: Eq. 1 from ``phi``),
    trilinear with zeros outside the image: warped [Z, Y, X], without storing T."""
    shape = tuple(int(s) for s in shape)
    _need(phi, "phi", torch.float32, grid_shape(shape, spacing) + (3,))
    fX, fY, fZ = _floating(image)
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=phi.device)
    _need(out, "out", torch.float32, shape)
    g = make_geom(shape, spacing)
    st = library().bsi_resample_forward(ctypes.byref(g), phi.data_ptr(), image.data_ptr(), fX, fY, fZ,
                                        out.data_ptr(), _stream(stream, phi.device))
    _check(st, "bsi_resample_forward")
    return out


def bsi_resample_backward_workspace_bytes(shape, spacing) -> int:
    g = make_geom(shape, spacing)
    return int(library().bsi_resample_backward_workspace_bytes(ctypes.byref(g)))


def bsi_resample_backward(phi, shape, spacing, image, grad_warped, out=None, workspace=None, stream=None):
    """dL/dphi [nz, ny, nx, 3] for dL/dwarped = ``grad_warped`` [Z, Y, X]."""
    shape = tuple(int(s) for s in shape)
    _need(phi, "phi", torch.float32, grid_shape(shape, spacing) + (3,))
    _need(grad_warped, "grad_warped", torch.float32, shape)
    fX, fY, fZ = _floating(image)
    if out is None:
        out = torch.empty_like(phi)
    _need(out, "out", torch.float32, tuple(phi.shape))
    g = make_geom(shape, spacing)
    need = int(library().bsi_resample_backward_workspace_bytes(ctypes.byref(g)))
    ws, wsb = _workspace(need, phi.device, workspace)
    st = library().bsi_resample_backward(ctypes.byref(g), phi.data_ptr(), image.data_ptr(), fX, fY, fZ,
                                         grad_warped.data_ptr(), out.data_ptr(),
                                         ws.data_ptr() if ws is not None else None, wsb,
                                         _stream(stream, phi.device))
    _check(st, "bsi_resample_backward")
    return out


def bsi_probe_fill(buf: torch.Tensor, value: int = 0, stream=None) -> None:
    """Fills a contiguous device tensor (size and address multiples of 16 bytes)
    with a 32-bit pattern through the forward kernel's store path: the
    write-only HBM peak probe."""
    if not buf.is_cuda or not buf.is_contiguous():
        raise ValueError("bsi_probe_fill wants a contiguous CUDA tensor")
    st = library().bsi_probe_fill(buf.data_ptr(), buf.numel() * buf.element_size(), value & 0xFFFFFFFF,
                                  _stream(stream, buf.device))
    _check(st, "bsi_probe_fill")


DEVICE_FLAG_TIMEOUT = 128


def bsi_selftest_lost_copy(stream=None, device=None) -> None:
    """Enqueues the failure-detection self-test: a wait for a copy that never
    comes runs out (<= ~2 s) and records DEVICE_FLAG_TIMEOUT; read it with
    bsi_check_device_status."""
    st = library().bsi_selftest_lost_copy(_stream(stream, device))
    _check(st, "bsi_selftest_lost_copy")


def bsi_check_device_status(stream=None, device=None) -> int:
    """Synchronises the stream and returns (and clears) the kernel error word."""
    flags = ctypes.c_uint32(0)
    st = library().bsi_check_device_status(_stream(stream, device), ctypes.byref(flags))
    if st not in (0, 9):
        _check(st, "bsi_check_device_status")
    return int(flags.value)


def bsi_selfcheck_ranges(shapes, spacings, op: str = "forward", cover: bool = True):
    """Host-only range check of every kernel access for a planned call (no GPU).
    ``op`` is "forward", "forward_bf16", "adjoint", "resample", "resample_grad", "scalar" or
    "scalar_bf16".
    Returns (violations, message)."""
    code = {"forward": 0, "forward_bf16": 1, "adjoint": 2, "resample": 3, "resample_grad": 4, "scalar": 5,
            "scalar_bf16": 6}[op]
    arr = _instances([tuple(s) for s in shapes], spacings)
    buf = ctypes.create_string_buffer(256)
    n = library().bsi_selfcheck_ranges(arr, len(shapes), code, int(cover), buf, 256)
    return int(n), buf.value.decode()
