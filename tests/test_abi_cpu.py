"""The C-ABI library on the CPU: it loads, exports every symbol include/bsi.h
declares, rejects bad arguments before touching CUDA, and every planned
kernel access lies inside its buffer (host-only range self-check)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2004_05962_gb300 as P
from paper_2004_05962_gb300 import bsi as B
from paper_2004_05962_gb300 import build as Bd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    Bd.build()
    return B.library()


def header_symbols():
    src = open(os.path.join(ROOT, "include", "bsi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bsi_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_what_binding_binds():
    assert header_symbols() == sorted(B.exported_symbols())


def test_library_exports_every_declared_symbol(lib):
    for name in header_symbols():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_status_strings(lib):
    for code, name in B.STATUS.items():
        assert lib.bsi_status_string(code).decode().startswith(name)
    assert lib.bsi_version() >= 100


def _geom(X, Y, Z, dx, dy, dz):
    g = B.BsiGeom()
    st = B.library().bsi_geom_init(ctypes.byref(g), X, Y, Z, dx, dy, dz)
    return g, st


def test_geom_init_and_limits(lib):
    g, st = _geom(64, 64, 64, 5, 5, 5)
    assert st == 0 and (g.nx, g.ny, g.nz) == (16, 16, 16)
    g, st = _geom(512, 512, 300, 5, 5, 5)
    assert (g.nx, g.ny, g.nz) == (106, 106, 63)
    assert _geom(-1, 4, 4, 2, 2, 2)[1] == 2
    assert _geom(4, 4, (1 << 20) + 1, 2, 2, 2)[1] == 2
    assert _geom(4, 4, 4, 0, 2, 2)[1] == 3
    assert _geom(4, 4, 4, 2, 65, 2)[1] == 3
    assert lib.bsi_geom_init(None, 4, 4, 4, 1, 1, 1) == 1
    g, st = _geom(0, 7, 7, 3, 3, 3)
    assert st == 0 and g.nx == 3


FAKE_DEV = 0x7F0000000000  # never dereferenced: every call below fails validation first


def test_forward_validation_before_cuda(lib):
    g, _ = _geom(10, 10, 10, 3, 3, 3)
    assert lib.bsi_field_forward(None, FAKE_DEV, FAKE_DEV, 0, None) == 1
    assert lib.bsi_field_forward(ctypes.byref(g), None, FAKE_DEV, 0, None) == 1
    assert lib.bsi_field_forward(ctypes.byref(g), FAKE_DEV, None, 0, None) == 1
    assert lib.bsi_field_forward(ctypes.byref(g), FAKE_DEV, FAKE_DEV, 7, None) == 5
    assert lib.bsi_field_forward(ctypes.byref(g), FAKE_DEV + 2, FAKE_DEV, 0, None) == 6
    assert lib.bsi_field_forward(ctypes.byref(g), FAKE_DEV, FAKE_DEV + 2, 0, None) == 6
    assert lib.bsi_field_forward(ctypes.byref(g), FAKE_DEV, FAKE_DEV + 1, 1, None) == 6
    bad = B.BsiGeom.from_buffer_copy(g)
    bad.nx += 1
    assert lib.bsi_field_forward(ctypes.byref(bad), FAKE_DEV, FAKE_DEV, 0, None) == 4
    bad = B.BsiGeom.from_buffer_copy(g)
    bad.dy = 0
    assert lib.bsi_field_forward(ctypes.byref(bad), FAKE_DEV, FAKE_DEV, 0, None) == 3


def test_adjoint_validation_before_cuda(lib):
    g, _ = _geom(40, 30, 20, 5, 4, 3)
    need = lib.bsi_adjoint_workspace_bytes(ctypes.byref(g))
    assert need > 0 and need % 16 == 0
    assert lib.bsi_field_adjoint(ctypes.byref(g), FAKE_DEV, FAKE_DEV, FAKE_DEV, need - 4, None) == 7
    assert lib.bsi_field_adjoint(ctypes.byref(g), FAKE_DEV, FAKE_DEV, None, need, None) == 7
    assert lib.bsi_field_adjoint(ctypes.byref(g), FAKE_DEV, FAKE_DEV, FAKE_DEV + 4, need, None) == 6
    assert lib.bsi_field_adjoint(ctypes.byref(g), None, FAKE_DEV, FAKE_DEV, need, None) == 1
    assert lib.bsi_field_adjoint(ctypes.byref(g), FAKE_DEV, None, FAKE_DEV, need, None) == 1
    e, _ = _geom(0, 30, 20, 5, 4, 3)
    assert lib.bsi_adjoint_workspace_bytes(ctypes.byref(e)) == 0


def test_batched_validation_before_cuda(lib):
    assert lib.bsi_field_forward_batched(None, 3, 0, None) == 10
    assert lib.bsi_field_forward_batched(None, -1, 0, None) == 10
    arr = (B.BsiInstance * 2)()
    g, _ = _geom(10, 10, 10, 3, 3, 3)
    arr[0].geom = g
    arr[1].geom = g
    arr[0].phi = arr[0].field = arr[1].phi = FAKE_DEV
    assert lib.bsi_field_forward_batched(arr, 2, 0, None) == 1  # arr[1].field is NULL
    arr[1].field = FAKE_DEV
    arr[1].geom.nz = 99
    assert lib.bsi_field_forward_batched(arr, 2, 0, None) == 4
    assert lib.bsi_batched_adjoint_workspace_bytes(arr, 2) == 0  # invalid geometry -> 0


def test_no_gpu_means_cuda_error_not_fallback(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    g, _ = _geom(10, 10, 10, 3, 3, 3)
    st = lib.bsi_field_forward(ctypes.byref(g), FAKE_DEV, FAKE_DEV, 0, None)
    assert st == 8
    assert lib.bsi_last_cuda_error().decode()


def test_binding_fails_loudly_when_library_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(B, "_LIBS", {})
    monkeypatch.setattr(Bd, "BUILD", tmp_path)
    with pytest.raises(B.BsiLibraryMissing):
        B.library()


# ------------------------------------------------------------ range self-check

EDGE_CASES = [
    ((64, 64, 64), (5, 5, 5)),
    ((1, 1, 1), (1, 1, 1)),
    ((1, 1, 1), (64, 64, 64)),
    ((3, 5, 7), (1, 2, 3)),
    ((17, 1, 33), (4, 1, 8)),
    ((9, 13, 300), (2, 3, 9)),       # generic x-spacing, long row
    ((5, 6, 1000), (3, 3, 7)),       # several x-groups
    ((7, 11, 29 * 8 + 1), (2, 2, 8)),  # ragged last x-group
    ((4, 4, 87), (3, 3, 3)),         # exactly 29 tiles per row
    ((30, 20, 130), (6, 5, 64)),     # spacing 64
    ((12, 40, 60), (16, 4, 13)),
    ((0, 10, 10), (3, 3, 3)),
    ((10, 0, 10), (3, 3, 3)),
    ((10, 10, 0), (3, 3, 3)),
]


@pytest.mark.parametrize("op", ["forward", "forward_bf16", "adjoint", "resample", "resample_grad", "scalar",
                                "scalar_bf16"])
def test_selfcheck_edge_cases(lib, op):
    for shape, spacing in EDGE_CASES:
        n, msg = P.bsi_selfcheck_ranges([shape], [spacing], op, cover=True)
        assert n == 0, (shape, spacing, msg)


# Single volumes whose forward rows leave by tensor stores in blocks (16-byte
# rows and strips): FP32 at x-spacings <= 4, BF16 at even x-spacings and (24-tile
# strips) odd ones >= 5, one and three channels, block heights 2..8, the CT and
# 512^3 bench shapes.
TENSOR_STORE = [
    ((300, 512, 512), (5, 5, 5)),
    ((512, 512, 512), (3, 3, 3)),
    ((512, 512, 512), (4, 4, 4)),
    ((512, 512, 512), (8, 8, 8)),
    ((512, 512, 512), (6, 5, 4)),
    ((7, 13, 64), (2, 3, 1)),
    ((9, 22, 120), (3, 4, 2)),
    ((10, 17, 252), (4, 6, 3)),
    ((5, 30, 236), (2, 8, 4)),
    ((6, 23, 248), (2, 5, 5)),
    ((4, 17, 464), (2, 8, 8)),
    ((7, 30, 64), (2, 6, 2)),
    ((5, 18, 336), (2, 3, 6)),
]


@pytest.mark.parametrize("op", ["forward", "forward_bf16", "scalar", "scalar_bf16"])
def test_selfcheck_tensor_store_blocks(lib, op):
    for shape, spacing in TENSOR_STORE:
        n, msg = P.bsi_selfcheck_ranges([shape], [spacing], op, cover=shape[0] * shape[1] * shape[2] < 1e8)
        assert n == 0, (shape, spacing, msg)


def test_selfcheck_two_row_adjoint_units(lib):
    """Single volumes at y-spacings 4..6 plan units of two tile-rows on the
    tensor-copy path: every partial write and read in range, every read written
    first, and the plan inside the documented (and the no-alloc) workspace bound."""
    cases = [((40, 18, 48), (3, 5, 4)), ((8, 40, 64), (2, 6, 4)), ((13, 24, 100), (5, 4, 3)),
             ((11, 13, 40), (3, 5, 2)), ((20, 21, 4), (5, 5, 5)), ((7, 9, 96), (2, 4, 8))]
    for shape, spacing in cases:
        n, msg = P.bsi_selfcheck_ranges([shape], [spacing], "adjoint", cover=True)
        assert n == 0, (shape, spacing, msg)
    for shape, spacing in [((300, 512, 512), (5, 5, 5)), ((512, 512, 512), (6, 5, 4))]:
        n, msg = P.bsi_selfcheck_ranges([shape], [spacing], "adjoint", cover=False)
        assert n == 0, (shape, spacing, msg)


@pytest.mark.parametrize("op", ["forward", "adjoint", "resample", "resample_grad", "scalar", "scalar_bf16"])
def test_selfcheck_random_geometries(lib, op):
    rng = np.random.default_rng(7)
    for _ in range(60):
        shape = tuple(int(v) for v in rng.integers(1, 90, 3))
        spacing = tuple(int(v) for v in rng.integers(1, 12, 3))
        n, msg = P.bsi_selfcheck_ranges([shape], [spacing], op, cover=True)
        assert n == 0, (shape, spacing, msg)


@pytest.mark.parametrize("op", ["forward", "adjoint"])
def test_selfcheck_batches(lib, op):
    from paper_2004_05962_gb300 import synth

    geoms = synth.batch_geometries(64, seed=5)
    geoms += [((20, 30, 40), (3, 4, 11)), ((0, 3, 3), (2, 2, 2)), ((5, 5, 5), (9, 9, 9))]
    geoms += synth.batch_geometries(70, seed=9, xy_range=(8, 40), z_range=(8, 30), spacing_range=(1, 10))
    n, msg = P.bsi_selfcheck_ranges([g[0] for g in geoms], [g[1] for g in geoms], op, cover=True)
    assert n == 0, msg


@pytest.mark.parametrize("spacing", [(3, 3, 3), (5, 5, 5), (6, 5, 4), (8, 8, 8)])
def test_selfcheck_full_size_volumes(lib, spacing):
    for op in ("forward", "adjoint"):
        n, msg = P.bsi_selfcheck_ranges([(512, 512, 512)], [spacing], op, cover=False)
        assert n == 0, msg
    n, msg = P.bsi_selfcheck_ranges([(300, 512, 512)], [(5, 5, 5)], "forward_bf16", cover=False)
    assert n == 0, msg


def test_selfcheck_detects_a_bad_plan(lib):
    """The checker itself is not vacuous: an invalid geometry is reported."""
    arr = (B.BsiInstance * 1)()
    g, _ = _geom(10, 10, 10, 3, 3, 3)
    g.nx = 2
    arr[0].geom = g
    buf = ctypes.create_string_buffer(256)
    assert lib.bsi_selfcheck_ranges(arr, 1, 0, 1, buf, 256) > 0


def test_probe_fill_validation_before_cuda(lib):
    fake = 0x7F0000000000  # never dereferenced: validation fails first
    assert lib.bsi_probe_fill(None, 0, 0, None) == 0
    assert lib.bsi_probe_fill(None, 16, 0, None) == 1
    assert lib.bsi_probe_fill(fake + 4, 16, 0, None) == 6
    assert lib.bsi_probe_fill(fake, 20, 0, None) == 6


def test_resample_validation_before_cuda(lib):
    fake = 0x7F0000000000  # never dereferenced: validation fails first
    g, _ = _geom(40, 30, 20, 5, 4, 3)
    rf = lib.bsi_resample_forward
    assert rf(ctypes.byref(g), fake, fake, 0, 30, 20, fake, None) == 2          # empty floating image
    assert rf(ctypes.byref(g), fake, fake, 1 << 20, 1 << 12, 1, fake, None) == 2   # 2^32 elements: too many
    assert rf(ctypes.byref(g), fake, None, 1 << 20, (1 << 12) - 1, 1, fake, None) == 1   # 2^32 - 2^20: admitted
    assert rf(ctypes.byref(g), fake, None, 40, 30, 20, fake, None) == 1         # floating NULL
    assert rf(ctypes.byref(g), fake, fake + 2, 40, 30, 20, fake, None) == 6     # floating misaligned
    assert rf(ctypes.byref(g), None, fake, 40, 30, 20, fake, None) == 1
    assert rf(ctypes.byref(g), fake, fake, 40, 30, 20, fake + 2, None) == 6
    need = lib.bsi_resample_backward_workspace_bytes(ctypes.byref(g))
    assert need >= 12 * 40 * 30 * 20 + lib.bsi_adjoint_workspace_bytes(ctypes.byref(g))
    rb = lib.bsi_resample_backward
    assert rb(ctypes.byref(g), fake, fake, 40, 30, 20, fake, fake, fake, need - 16, None) == 7
    assert rb(ctypes.byref(g), fake, fake, 40, 30, 20, fake, fake, fake + 4, need, None) == 6
    assert rb(ctypes.byref(g), fake, fake, 40, 30, 20, None, fake, fake, need, None) == 1
    assert rb(ctypes.byref(g), fake, fake, 40, 30, 20, fake, None, fake, need, None) == 1
    e, _ = _geom(0, 30, 20, 5, 4, 3)
    assert lib.bsi_resample_backward_workspace_bytes(ctypes.byref(e)) == 0


def test_scalar_validation_before_cuda(lib):
    fake = 0x7F0000000000  # never dereferenced: validation fails first
    g, _ = _geom(40, 30, 20, 5, 4, 3)
    sf = lib.bsi_scalar_forward
    assert sf(ctypes.byref(g), None, fake, 0, None) == 1
    assert sf(ctypes.byref(g), fake, None, 0, None) == 1
    assert sf(ctypes.byref(g), fake + 2, fake, 0, None) == 6
    assert sf(ctypes.byref(g), fake, fake + 2, 0, None) == 6
    assert sf(ctypes.byref(g), fake, fake, 7, None) == 5
    e, _ = _geom(0, 30, 20, 5, 4, 3)
    assert sf(ctypes.byref(e), None, None, 0, None) == 0


def test_variant_validation_before_cuda(lib):
    fake = 0x7F0000000000  # never dereferenced: validation fails first
    g, _ = _geom(40, 30, 20, 5, 4, 3)
    fv = lib.bsi_field_forward_variant
    assert fv(ctypes.byref(g), fake, fake, 7, None) == 5
    assert fv(ctypes.byref(g), None, fake, 1, None) == 1
    assert fv(ctypes.byref(g), fake, fake + 2, 2, None) == 6
    big, _ = _geom(40, 30, 20, 33, 4, 3)
    assert fv(ctypes.byref(big), fake, fake, 2, None) == 3


def test_rational_geometry_and_validation_before_cuda(lib):
    import oracle

    for shape, num, den, off in [((7, 9, 11), (5, 7, 9), (2, 2, 2), (0, 3, 1)), ((300, 512, 512), (47, 47, 47),
                                                                                 (10, 10, 10), (3, 0, 9))]:
        g = B.make_geom_rational(shape, num, den, off)
        assert (g.nz, g.ny, g.nx) == B.rational_grid_shape(shape, num, den, off) == \
            oracle.rational_grid_shape(shape, num, den, off)
    fake = 0x7F0000000000  # never dereferenced: validation fails first
    g = B.make_geom_rational((7, 9, 11), (5, 7, 9), (2, 2, 2), (0, 3, 1))
    fr = lib.bsi_field_forward_rational
    assert fr(ctypes.byref(g), None, fake, None) == 1
    assert fr(ctypes.byref(g), fake + 2, fake, None) == 6
    g.nx += 1
    assert fr(ctypes.byref(g), fake, fake, None) == 4
    for bad in [((1, 1, 1), (2, 1, 1), (0, 0, 0)),          # spacing below 1
                ((5, 5, 5), (2, 2, 2), (0, 5, 0)),          # shift of a whole cell
                ((5, 5, 5), (2000, 2, 2), (0, 0, 0))]:      # denominator beyond the limit
        with pytest.raises(B.BsiError):
            B.make_geom_rational((7, 9, 11), *bad)


def test_rational_adjoint_workspace_and_validation_before_cuda(lib):
    """The adjoint's workspace: per unit (zc z-cells x one y-cell x a strip of up
    to 29 x-cells) zc + 3 grid planes of 4 rows x 32 columns x 3 floats; zc = 4,
    halved while there are fewer than 6000 units or a unit has more than 64
    voxel planes.  The argument checks come before any CUDA call."""
    fake = 0x7F0000000000  # never dereferenced: validation fails first
    cases = [((300, 512, 512), (47, 47, 47), (10, 10, 10), (3, 0, 9)),
             ((7, 9, 11), (5, 7, 9), (2, 2, 2), (0, 3, 1)),
             ((10, 10, 33), (640, 13, 23), (10, 5, 7), (639, 4, 22))]
    for shape, num, den, off in cases:
        g = B.make_geom_rational(shape, num, den, off)
        ncell = [((N - 1) * d + o) // n + 1 for N, n, d, o in zip(shape, num, den, off)]   # (z, y, x)
        cmax = -(-num[2] // den[2])
        sc = min(29, 232 // cmax)
        nsx = -(-ncell[2] // sc)
        zc, zmax = 4, -(-num[0] // den[0])
        while zc > 1 and (-(-ncell[0] // zc) * ncell[1] * nsx < 6000 or zc * zmax > 64):
            zc //= 2
        want = -(-ncell[0] // zc) * ncell[1] * nsx * (zc + 3) * 4 * 32 * 3 * 4
        assert lib.bsi_rational_adjoint_workspace_bytes(ctypes.byref(g)) == want, (shape, num)
    g = B.make_geom_rational((7, 9, 11), (5, 7, 9), (2, 2, 2), (0, 3, 1))
    need = lib.bsi_rational_adjoint_workspace_bytes(ctypes.byref(g))
    ar = lib.bsi_field_adjoint_rational
    assert ar(ctypes.byref(g), fake, None, fake, need, None) == 1          # grad_phi NULL
    assert ar(ctypes.byref(g), fake, fake + 2, fake, need, None) == 6      # grad_phi misaligned
    assert ar(ctypes.byref(g), None, fake, fake, need, None) == 1          # grad_field NULL
    assert ar(ctypes.byref(g), fake + 2, fake, fake, need, None) == 6      # grad_field misaligned
    assert ar(ctypes.byref(g), fake, fake, None, need, None) == 7          # no workspace
    assert ar(ctypes.byref(g), fake, fake, fake, need - 4, None) == 7      # short workspace
    assert ar(ctypes.byref(g), fake, fake, fake + 4, need, None) == 6      # workspace misaligned
    g.nx += 1
    assert ar(ctypes.byref(g), fake, fake, fake, need, None) == 4
    assert lib.bsi_rational_adjoint_workspace_bytes(ctypes.byref(g)) == 0
