"""FP64 CPU oracle for cubic B-spline interpolation (BSI) -- test infrastructure.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding in ``paper_2004_05962_gb300``) never does, and the two share no
code: the oracle is plain C in ``bsi_oracle.c``, built with gcc, loaded here
through ctypes.

Every function evaluates Eq. 1 (Sec. 2.1) or its transpose literally in FP64;
see ``bsi_oracle.c`` for the readings of the paper it encodes.
"""
from __future__ import annotations

import ctypes
import os
import pathlib
import subprocess

import numpy as np

_DIR = pathlib.Path(__file__).resolve().parent
_SRC = _DIR / "bsi_oracle.c"
_BUILD = _DIR / "_build"
_LIB_NAME = "libbsi_oracle.so"

_lib = None


def build(out_dir: pathlib.Path | None = None, mutant: int = 0, quiet: bool = True) -> pathlib.Path:
    """Compiles the oracle with gcc into a shared library and returns its path.

    ``mutant`` plants one known mistake (see ORACLE_MUTANT in the C source);
    it exists only for the test that checks the pins catch such mistakes.
    FP contraction is off so that x86 and Arm builds round identically.
    """
    out_dir = pathlib.Path(out_dir) if out_dir is not None else _BUILD
    out_dir.mkdir(parents=True, exist_ok=True)
    name = _LIB_NAME if mutant == 0 else f"libbsi_oracle_m{mutant}.so"
    out = out_dir / name
    tmp = out_dir / (name + f".tmp{os.getpid()}")
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
           f"-DORACLE_MUTANT={int(mutant)}", "-o", str(tmp), str(_SRC), "-lm"]
    subprocess.run(cmd, check=True, capture_output=quiet)
    os.replace(tmp, out)
    return out


def _bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    i64, i32, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
    geom = [i64, i64, i64, i32, i32, i32]
    lib.bsi_oracle_threads.argtypes = [i32]
    lib.bsi_oracle_threads.restype = i32
    lib.bsi_oracle_forward.argtypes = geom + [vp, i32, vp, i32]
    lib.bsi_oracle_forward_points.argtypes = geom + [vp, i32, vp, i64, vp, i32]
    lib.bsi_oracle_adjoint.argtypes = geom + [vp, i32, vp, i32]
    lib.bsi_oracle_adjoint_points.argtypes = geom + [vp, i32, vp, i64, vp, i32]
    lib.bsi_oracle_resample.argtypes = geom + [vp, i32, vp, i32, i64, i64, i64, vp, i32]
    lib.bsi_oracle_resample_grad.argtypes = geom + [vp, i32, vp, i32, i64, i64, i64, vp, i32, vp, i32]
    lib.bsi_oracle_forward_rational.argtypes = [i64, i64, i64, vp, vp, vp, vp, i32, vp]
    lib.bsi_oracle_resample_points.argtypes = geom + [vp, i32, vp, i32, i64, i64, i64, vp, i64, vp, vp]
    lib.bsi_oracle_forward_rational_points.argtypes = [i64, i64, i64, vp, vp, vp, vp, i32, vp, i64, vp]
    lib.bsi_oracle_adjoint_rational.argtypes = [i64, i64, i64, vp, vp, vp, vp, i32, vp]
    lib.bsi_oracle_adjoint_rational_points.argtypes = [i64, i64, i64, vp, vp, vp, vp, i32, vp, i64, vp]
    for f in ("bsi_oracle_forward", "bsi_oracle_forward_points", "bsi_oracle_adjoint",
              "bsi_oracle_adjoint_points", "bsi_oracle_resample", "bsi_oracle_resample_grad",
              "bsi_oracle_forward_rational", "bsi_oracle_resample_points", "bsi_oracle_forward_rational_points"):
        getattr(lib, f).restype = i32
    return lib


def load(path: pathlib.Path | None = None) -> ctypes.CDLL:
    """Loads (building first if needed) the oracle library; cached for the default build."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(str(path)))
    if _lib is None:
        p = _BUILD / _LIB_NAME
        if not p.exists() or p.stat().st_mtime < _SRC.stat().st_mtime:
            build()
        _lib = _bind(ctypes.CDLL(str(p)))
    return _lib


def grid_shape(shape, spacing):
    """Stored control-grid dims (nz, ny, nx) for a volume (Z, Y, X): ceil(N/d) + 3."""
    Z, Y, X = shape
    dz, dy, dx = spacing
    return (-(-Z // dz) + 3, -(-Y // dy) + 3, -(-X // dx) + 3)


def _in(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.float32:
        return a, 1
    if a.dtype != np.float64:
        a = a.astype(np.float64)
    return a, 0


def _geom(shape, spacing):
    Z, Y, X = (int(s) for s in shape)
    dz, dy, dx = (int(s) for s in spacing)
    return [X, Y, Z, dx, dy, dz]


class OracleError(RuntimeError):
    pass


def forward(phi, shape, spacing, nthreads: int = 0, lib=None) -> np.ndarray:
    """Dense field [Z, Y, X, 3] (FP64) from phi [nz, ny, nx, 3] (FP32 or FP64).

    ``shape`` is (Z, Y, X) voxels, ``spacing`` is (dz, dy, dx) voxels.
    """
    lib = lib or load()
    Z, Y, X = (int(s) for s in shape)
    assert phi.shape == grid_shape(shape, spacing) + (3,), (phi.shape, shape, spacing)
    p, f32 = _in(phi)
    out = np.empty((Z, Y, X, 3), np.float64)
    rc = lib.bsi_oracle_forward(*_geom(shape, spacing), p.ctypes.data, f32, out.ctypes.data, nthreads)
    if rc:
        raise OracleError("bsi_oracle_forward: bad arguments")
    return out


def forward_points(phi, shape, spacing, xyz, nthreads: int = 0, lib=None) -> np.ndarray:
    """Eq. 1 at voxels ``xyz`` [n, 3] given as (x, y, z); returns [n, 3] FP64."""
    lib = lib or load()
    assert phi.shape == grid_shape(shape, spacing) + (3,)
    p, f32 = _in(phi)
    q = np.ascontiguousarray(xyz, dtype=np.int64).reshape(-1, 3)
    out = np.empty((q.shape[0], 3), np.float64)
    rc = lib.bsi_oracle_forward_points(*_geom(shape, spacing), p.ctypes.data, f32, q.ctypes.data,
                                       q.shape[0], out.ctypes.data, nthreads)
    if rc:
        raise OracleError("bsi_oracle_forward_points: bad arguments")
    return out


def adjoint(grad, spacing, nthreads: int = 0, lib=None) -> np.ndarray:
    """Transpose of Eq. 1: dphi [nz, ny, nx, 3] (FP64) from grad [Z, Y, X, 3]."""
    lib = lib or load()
    Z, Y, X = grad.shape[:3]
    g, f32 = _in(grad)
    out = np.empty(grid_shape((Z, Y, X), spacing) + (3,), np.float64)
    rc = lib.bsi_oracle_adjoint(*_geom((Z, Y, X), spacing), g.ctypes.data, f32, out.ctypes.data,
                                nthreads)
    if rc:
        raise OracleError("bsi_oracle_adjoint: bad arguments")
    return out


def adjoint_points(grad, spacing, gxyz, nthreads: int = 0, lib=None) -> np.ndarray:
    """Transpose of Eq. 1 at stored control points ``gxyz`` [n, 3] as (gx, gy, gz)."""
    lib = lib or load()
    Z, Y, X = grad.shape[:3]
    g, f32 = _in(grad)
    q = np.ascontiguousarray(gxyz, dtype=np.int64).reshape(-1, 3)
    out = np.empty((q.shape[0], 3), np.float64)
    rc = lib.bsi_oracle_adjoint_points(*_geom((Z, Y, X), spacing), g.ctypes.data, f32,
                                       q.ctypes.data, q.shape[0], out.ctypes.data, nthreads)
    if rc:
        raise OracleError("bsi_oracle_adjoint_points: bad arguments")
    return out


def rational_grid_shape(shape, num, den, off):
    """Stored grid (nz, ny, nx) for spacing num/den and lattice shift off/den per
    axis; num, den, off are given (z, y, x) like shape."""
    return tuple(((int(N) - 1) * int(d) + int(o)) // int(n) + 4 if int(N) > 0 else 4
                 for N, n, d, o in zip(shape, num, den, off))


def forward_rational(phi, shape, num, den, off, lib=None) -> np.ndarray:
    """Eq. 1 with spacing num/den and lattice shift off/den voxels per axis
    ((z, y, x) order like ``shape``): field [Z, Y, X, 3] (FP64)."""
    lib = lib or load()
    Z, Y, X = (int(s) for s in shape)
    assert phi.shape == rational_grid_shape(shape, num, den, off) + (3,), (phi.shape, shape)
    p, f32 = _in(phi)
    to_xyz = lambda a: np.ascontiguousarray(np.array(a, np.int64)[::-1])
    n3, d3, o3 = to_xyz(num), to_xyz(den), to_xyz(off)
    out = np.empty((Z, Y, X, 3), np.float64)
    rc = lib.bsi_oracle_forward_rational(X, Y, Z, n3.ctypes.data, d3.ctypes.data, o3.ctypes.data, p.ctypes.data,
                                         f32, out.ctypes.data)
    if rc:
        raise OracleError("bsi_oracle_forward_rational: bad arguments")
    return out


def forward_rational_points(phi, shape, num, den, off, xyz, lib=None) -> np.ndarray:
    """forward_rational at voxels ``xyz`` [n, 3] given as (x, y, z); returns [n, 3]."""
    lib = lib or load()
    Z, Y, X = (int(s) for s in shape)
    assert phi.shape == rational_grid_shape(shape, num, den, off) + (3,)
    p, f32 = _in(phi)
    to_xyz = lambda a: np.ascontiguousarray(np.array(a, np.int64)[::-1])
    n3, d3, o3 = to_xyz(num), to_xyz(den), to_xyz(off)
    q = np.ascontiguousarray(xyz, dtype=np.int64).reshape(-1, 3)
    out = np.empty((q.shape[0], 3), np.float64)
    rc = lib.bsi_oracle_forward_rational_points(X, Y, Z, n3.ctypes.data, d3.ctypes.data, o3.ctypes.data,
                                                p.ctypes.data, f32, q.ctypes.data, q.shape[0], out.ctypes.data)
    if rc:
        raise OracleError("bsi_oracle_forward_rational_points: bad arguments")
    return out


def adjoint_rational(grad, num, den, off, lib=None) -> np.ndarray:
    """Transpose of forward_rational: dphi [nz, ny, nx, 3] (FP64) from grad
    [Z, Y, X, 3]; num, den, off are (z, y, x)."""
    lib = lib or load()
    Z, Y, X = (int(s) for s in grad.shape[:3])
    g, f32 = _in(grad)
    to_xyz = lambda a: np.ascontiguousarray(np.array(a, np.int64)[::-1])
    n3, d3, o3 = to_xyz(num), to_xyz(den), to_xyz(off)
    out = np.empty(rational_grid_shape((Z, Y, X), num, den, off) + (3,), np.float64)
    rc = lib.bsi_oracle_adjoint_rational(X, Y, Z, n3.ctypes.data, d3.ctypes.data, o3.ctypes.data, g.ctypes.data,
                                         f32, out.ctypes.data)
    if rc:
        raise OracleError("bsi_oracle_adjoint_rational: bad arguments")
    return out


def adjoint_rational_points(grad, num, den, off, gxyz, lib=None) -> np.ndarray:
    """adjoint_rational at stored control points ``gxyz`` [n, 3] as (gx, gy, gz)."""
    lib = lib or load()
    Z, Y, X = (int(s) for s in grad.shape[:3])
    g, f32 = _in(grad)
    to_xyz = lambda a: np.ascontiguousarray(np.array(a, np.int64)[::-1])
    n3, d3, o3 = to_xyz(num), to_xyz(den), to_xyz(off)
    q = np.ascontiguousarray(gxyz, dtype=np.int64).reshape(-1, 3)
    out = np.empty((q.shape[0], 3), np.float64)
    rc = lib.bsi_oracle_adjoint_rational_points(X, Y, Z, n3.ctypes.data, d3.ctypes.data, o3.ctypes.data,
                                                g.ctypes.data, f32, q.ctypes.data, q.shape[0], out.ctypes.data)
    if rc:
        raise OracleError("bsi_oracle_adjoint_rational_points: bad arguments")
    return out


def resample_points(phi, shape, spacing, image, xyz, lib=None):
    """resample at voxels ``xyz`` [n, 3] (x, y, z): (values [n], interpolant
    gradients [n, 3]) in FP64."""
    lib = lib or load()
    assert phi.shape == grid_shape(shape, spacing) + (3,)
    p, f32 = _in(phi)
    im, if32 = _in(image)
    fZ, fY, fX = im.shape
    q = np.ascontiguousarray(xyz, dtype=np.int64).reshape(-1, 3)
    val = np.empty(q.shape[0], np.float64)
    grad = np.empty((q.shape[0], 3), np.float64)
    rc = lib.bsi_oracle_resample_points(*_geom(shape, spacing), p.ctypes.data, f32, im.ctypes.data, if32, fX, fY, fZ,
                                        q.ctypes.data, q.shape[0], val.ctypes.data, grad.ctypes.data)
    if rc:
        raise OracleError("bsi_oracle_resample_points: bad arguments")
    return val, grad


def resample(phi, shape, spacing, image, nthreads: int = 0, lib=None) -> np.ndarray:
    """Floating ``image`` [fZ, fY, fX] sampled at x + T(x) (trilinear, zeros
    outside the image): warped [Z, Y, X] (FP64)."""
    lib = lib or load()
    Z, Y, X = (int(s) for s in shape)
    assert phi.shape == grid_shape(shape, spacing) + (3,)
    p, f32 = _in(phi)
    im, if32 = _in(image)
    fZ, fY, fX = im.shape
    out = np.empty((Z, Y, X), np.float64)
    rc = lib.bsi_oracle_resample(*_geom(shape, spacing), p.ctypes.data, f32, im.ctypes.data, if32, fX, fY, fZ,
                                 out.ctypes.data, nthreads)
    if rc:
        raise OracleError("bsi_oracle_resample: bad arguments")
    return out


def resample_grad(phi, shape, spacing, image, dwarped, nthreads: int = 0, lib=None) -> np.ndarray:
    """Voxel gradient G [Z, Y, X, 3] = dwarped * grad F~(x + T(x)) (FP64)."""
    lib = lib or load()
    Z, Y, X = (int(s) for s in shape)
    assert phi.shape == grid_shape(shape, spacing) + (3,) and tuple(dwarped.shape) == (Z, Y, X)
    p, f32 = _in(phi)
    im, if32 = _in(image)
    dw, df32 = _in(dwarped)
    fZ, fY, fX = im.shape
    out = np.empty((Z, Y, X, 3), np.float64)
    rc = lib.bsi_oracle_resample_grad(*_geom(shape, spacing), p.ctypes.data, f32, im.ctypes.data, if32, fX, fY,
                                      fZ, dw.ctypes.data, df32, out.ctypes.data, nthreads)
    if rc:
        raise OracleError("bsi_oracle_resample_grad: bad arguments")
    return out


def resample_backward(phi, shape, spacing, image, dwarped, nthreads: int = 0, lib=None) -> np.ndarray:
    """dL/dphi [nz, ny, nx, 3] for dL/dwarped = ``dwarped``: the transpose of
    Eq. 1 applied to resample_grad."""
    return adjoint(resample_grad(phi, shape, spacing, image, dwarped, nthreads, lib), spacing, nthreads, lib)


def threads(nthreads: int = 0, lib=None) -> int:
    """Thread count the oracle uses for a request of ``nthreads`` (0: all host cores)."""
    lib = lib or load()
    return int(lib.bsi_oracle_threads(nthreads))
