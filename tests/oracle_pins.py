"""Checks that pin the FP64 oracle to facts other than itself.

Each ``pin_*`` function takes an oracle library handle and returns
(max_error, tolerance).  tests/test_oracle_pins.py asserts every pin holds for
the real oracle; tests/test_oracle_mutants.py builds the oracle with planted
mistakes and asserts that each one breaks at least one pin.

What pins what:
  * partition of unity (sum_l B_l = 1): constant grid -> constant field;
  * affine reproduction (sum_l l B_l(t) = 1 + t): an affine grid
    phi_g = A p_g + b, p_g = ((gx-1)dx, (gy-1)dy, (gz-1)dz), gives the affine
    field A x + b -- pins the basis order, the index origin and the axis order;
  * knot values from tests/golden (textbook values of the cubic B-spline);
  * brute force: the global sum over ALL grid points of
    phi_g beta3(x/dx - gx + 1) beta3(y/dy - gy + 1) beta3(z/dz - gz + 1),
    with the centred cubic B-spline beta3 -- a different formulation from
    the oracle's local 4x4x4 neighbourhood sum;
  * scipy's tensor-product B-spline (NdBSpline) with uniform knots;
  * the adjoint: brute-force transpose, dot-product identity, and central
    differences of the linear functional <W, T(phi)>.
"""
from __future__ import annotations

import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def beta3(t):
    """Centred cubic B-spline (support [-2, 2])."""
    a = np.abs(np.asarray(t, dtype=np.float64))
    return np.where(a < 1.0, 2.0 / 3.0 - a * a + 0.5 * a ** 3,
                    np.where(a < 2.0, (2.0 - a) ** 3 / 6.0, 0.0))


def weight_matrix(N, d):
    """W[x, g] = beta3(x/d - g + 1) for voxels x < N and stored points g < ceil(N/d)+3."""
    n = -(-N // d) + 3
    x = np.arange(N, dtype=np.float64)[:, None]
    g = np.arange(n, dtype=np.float64)[None, :]
    return beta3(x / d - g + 1.0)


def brute_forward(phi, shape, spacing):
    """Global sum over every stored grid point (matrix form of the brute force)."""
    Z, Y, X = shape
    dz, dy, dx = spacing
    Wz, Wy, Wx = weight_matrix(Z, dz), weight_matrix(Y, dy), weight_matrix(X, dx)
    return np.einsum("zc,yb,xa,cbad->zyxd", Wz, Wy, Wx, phi.astype(np.float64), optimize=True)


def brute_forward_loops(phi, shape, spacing):
    """The same global sum with explicit loops over voxels and grid points."""
    Z, Y, X = shape
    dz, dy, dx = spacing
    nz, ny, nx = phi.shape[:3]
    out = np.zeros((Z, Y, X, 3))
    for z in range(Z):
        for y in range(Y):
            for x in range(X):
                acc = np.zeros(3)
                for gz in range(nz):
                    wz = float(beta3(z / dz - gz + 1))
                    if wz == 0.0:
                        continue
                    for gy in range(ny):
                        wy = float(beta3(y / dy - gy + 1))
                        if wy == 0.0:
                            continue
                        for gx in range(nx):
                            wx = float(beta3(x / dx - gx + 1))
                            if wx != 0.0:
                                acc += wz * wy * wx * phi[gz, gy, gx].astype(np.float64)
                out[z, y, x] = acc
    return out


def brute_adjoint(grad, spacing):
    Z, Y, X = grad.shape[:3]
    dz, dy, dx = spacing
    Wz, Wy, Wx = weight_matrix(Z, dz), weight_matrix(Y, dy), weight_matrix(X, dx)
    return np.einsum("zc,yb,xa,zyxd->cbad", Wz, Wy, Wx, grad.astype(np.float64), optimize=True)


# shapes (Z, Y, X) and spacings (dz, dy, dx) with ragged tails and anisotropy
SMALL_CASES = [
    ((7, 9, 11), (2, 3, 4)),
    ((12, 10, 8), (5, 3, 2)),
    ((5, 6, 13), (1, 2, 5)),
    ((10, 10, 10), (4, 4, 4)),
    ((3, 11, 7), (3, 5, 1)),
]


def _rng(seed):
    return np.random.default_rng(seed)


def pin_partition_of_unity(lib):
    worst = 0.0
    for shape, spacing in SMALL_CASES:
        k = np.array([1.75, -3.5, 0.3125])
        phi = np.broadcast_to(k, oracle.grid_shape(shape, spacing) + (3,)).copy()
        T = oracle.forward(phi, shape, spacing, lib=lib)
        worst = max(worst, float(np.max(np.abs(T - k))))
    return worst, 1e-14 * 3.5


def pin_affine_reproduction(lib):
    rng = _rng(11)
    worst, scale = 0.0, 1.0
    for shape, spacing in SMALL_CASES:
        A = rng.uniform(-2, 2, (3, 3))
        b = rng.uniform(-5, 5, 3)
        nz, ny, nx = oracle.grid_shape(shape, spacing)
        dz, dy, dx = spacing
        gz, gy, gx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        p = np.stack([(gx - 1) * dx, (gy - 1) * dy, (gz - 1) * dz], axis=-1).astype(np.float64)
        phi = p @ A.T + b
        T = oracle.forward(phi, shape, spacing, lib=lib)
        Z, Y, X = shape
        z, y, x = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
        q = np.stack([x, y, z], axis=-1).astype(np.float64)
        want = q @ A.T + b
        worst = max(worst, float(np.max(np.abs(T - want))))
        scale = max(scale, float(np.max(np.abs(want))))
    return worst, 1e-13 * scale


def load_knots():
    rows = []
    with open(os.path.join(GOLDEN, "bspline_basis_values.txt")) as f:
        for line in f:
            line = line.split("#")[0].split()
            if not line:
                continue
            tn, td, b0, b1, b2, b3, den = (int(v) for v in line)
            rows.append((tn / td, np.array([b0, b1, b2, b3], np.float64) / den))
    return rows


def pin_knot_values(lib):
    """One-hot grid: T at voxels with fractional offset t in every axis equals
    the tensor product of the golden knot values."""
    worst = 0.0
    for t, Bt in load_knots():
        d = 4 if t == 0.5 else 3
        spacing = (d, d, d)
        shape = (5 * d, 5 * d, 5 * d)
        nz, ny, nx = oracle.grid_shape(shape, spacing)
        g = (4, 3, 5)  # stored (gz, gy, gx) of the one-hot point
        phi = np.zeros((nz, ny, nx, 3))
        phi[g[0], g[1], g[2], 1] = 1.0
        pts, want = [], []
        r = int(round(t * d))
        for fz in range(5):
            for fy in range(5):
                for fx in range(5):
                    lz, ly, lx = g[0] - fz, g[1] - fy, g[2] - fx
                    if not (0 <= lz < 4 and 0 <= ly < 4 and 0 <= lx < 4):
                        continue
                    pts.append([fx * d + r, fy * d + r, fz * d + r])
                    want.append(Bt[lx] * Bt[ly] * Bt[lz])
        T = oracle.forward_points(phi, shape, spacing, np.array(pts), lib=lib)
        worst = max(worst, float(np.max(np.abs(T[:, 1] - np.array(want)))))
        worst = max(worst, float(np.max(np.abs(T[:, [0, 2]]))))
    return worst, 1e-15


def pin_brute_force(lib):
    rng = _rng(12)
    worst = 0.0
    for shape, spacing in SMALL_CASES:
        phi = rng.uniform(-2, 2, oracle.grid_shape(shape, spacing) + (3,))
        T = oracle.forward(phi, shape, spacing, lib=lib)
        worst = max(worst, float(np.max(np.abs(T - brute_forward(phi, shape, spacing)))))
    # the literal loop form on one tiny anisotropic case
    shape, spacing = (4, 5, 6), (2, 3, 4)
    phi = rng.uniform(-2, 2, oracle.grid_shape(shape, spacing) + (3,))
    T = oracle.forward(phi, shape, spacing, lib=lib)
    worst = max(worst, float(np.max(np.abs(T - brute_forward_loops(phi, shape, spacing)))))
    return worst, 1e-13


def pin_scipy_tensor_bspline(lib):
    from scipy.interpolate import NdBSpline

    rng = _rng(13)
    worst = 0.0
    for shape, spacing in SMALL_CASES:
        nz, ny, nx = oracle.grid_shape(shape, spacing)
        phi = rng.uniform(-2, 2, (nz, ny, nx, 3))
        knots = tuple(np.arange(n + 4, dtype=np.float64) - 3.0 for n in (nz, ny, nx))
        spl = NdBSpline(knots, phi, 3)
        Z, Y, X = shape
        dz, dy, dx = spacing
        z, y, x = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
        xi = np.stack([z / dz, y / dy, x / dx], axis=-1).reshape(-1, 3)
        want = spl(xi).reshape(Z, Y, X, 3)
        T = oracle.forward(phi, shape, spacing, lib=lib)
        worst = max(worst, float(np.max(np.abs(T - want))))
    return worst, 1e-12


def pin_scipy_1d_curve(lib):
    """A grid that varies along x only gives the textbook 1-D cubic B-spline curve."""
    from scipy.interpolate import BSpline

    rng = _rng(14)
    worst = 0.0
    for X, dx in ((23, 3), (40, 5), (17, 8)):
        shape, spacing = (3, 4, X), (2, 2, dx)
        nz, ny, nx = oracle.grid_shape(shape, spacing)
        c = rng.uniform(-3, 3, (nx, 3))
        phi = np.broadcast_to(c, (nz, ny, nx, 3)).copy()
        curve = BSpline(np.arange(nx + 4, dtype=np.float64) - 3.0, c, 3)
        want = curve(np.arange(X) / dx)
        T = oracle.forward(phi, shape, spacing, lib=lib)
        worst = max(worst, float(np.max(np.abs(T - want[None, None]))))
    return worst, 1e-12


def pin_adjoint_brute(lib):
    rng = _rng(15)
    worst, scale = 0.0, 1.0
    for shape, spacing in SMALL_CASES:
        G = rng.normal(size=shape + (3,))
        got = oracle.adjoint(G, spacing, lib=lib)
        want = brute_adjoint(G, spacing)
        worst = max(worst, float(np.max(np.abs(got - want))))
        scale = max(scale, float(np.max(np.abs(want))))
    return worst, 1e-13 * scale


def pin_adjoint_dot_product(lib):
    """<T(phi), W> == <phi, T^T(W)> to FP64 rounding."""
    rng = _rng(16)
    worst = 0.0
    for shape, spacing in SMALL_CASES:
        phi = rng.uniform(-2, 2, oracle.grid_shape(shape, spacing) + (3,))
        W = rng.normal(size=shape + (3,))
        lhs = float(np.sum(oracle.forward(phi, shape, spacing, lib=lib) * W))
        rhs = float(np.sum(phi * oracle.adjoint(W, spacing, lib=lib)))
        worst = max(worst, abs(lhs - rhs) / max(1.0, abs(lhs)))
    return worst, 1e-12


def pin_adjoint_finite_difference(lib):
    """L(phi) = <W, T(phi)> is linear, so a central difference on any grid entry
    equals the adjoint entry up to FP64 rounding."""
    rng = _rng(17)
    shape, spacing = (9, 8, 10), (3, 2, 4)
    phi = rng.uniform(-2, 2, oracle.grid_shape(shape, spacing) + (3,))
    W = rng.normal(size=shape + (3,))
    adj = oracle.adjoint(W, spacing, lib=lib)
    worst = 0.0
    eps = 1e-3
    for _ in range(12):
        idx = tuple(int(rng.integers(0, s)) for s in phi.shape)
        p1, p2 = phi.copy(), phi.copy()
        p1[idx] += eps
        p2[idx] -= eps
        fd = (np.sum(W * oracle.forward(p1, shape, spacing, lib=lib))
              - np.sum(W * oracle.forward(p2, shape, spacing, lib=lib))) / (2 * eps)
        worst = max(worst, abs(fd - adj[idx]))
    return worst, 1e-9


def pin_points_match_dense(lib):
    """The point-sampled entry points agree with the dense ones."""
    rng = _rng(18)
    worst = 0.0
    for shape, spacing in SMALL_CASES[:3]:
        grid = oracle.grid_shape(shape, spacing)
        phi = rng.uniform(-2, 2, grid + (3,))
        T = oracle.forward(phi, shape, spacing, lib=lib)
        Z, Y, X = shape
        pts = np.stack([rng.integers(0, X, 50), rng.integers(0, Y, 50), rng.integers(0, Z, 50)], 1)
        Tp = oracle.forward_points(phi, shape, spacing, pts, lib=lib)
        worst = max(worst, float(np.max(np.abs(Tp - T[pts[:, 2], pts[:, 1], pts[:, 0]]))))
        G = rng.normal(size=shape + (3,))
        A = oracle.adjoint(G, spacing, lib=lib)
        nz, ny, nx = grid
        gp = np.stack([rng.integers(0, nx, 50), rng.integers(0, ny, 50), rng.integers(0, nz, 50)], 1)
        Ap = oracle.adjoint_points(G, spacing, gp, lib=lib)
        worst = max(worst, float(np.max(np.abs(Ap - A[gp[:, 2], gp[:, 1], gp[:, 0]]))))
    return worst, 1e-12


# ---------------------------------------------------------------- resampling
# The floating image sampled at x + T(x), trilinear with zeros outside (the FFD
# step after BSI that Sec. 8 proposes to merge with it), and its gradient.

RESAMPLE_CASES = [  # (shape, spacing, floating image shape): equal and unequal image sizes
    ((7, 9, 11), (2, 3, 4), (7, 9, 11)),
    ((6, 8, 10), (3, 2, 2), (9, 5, 13)),
]


def _grid_points(shape):
    Z, Y, X = shape
    return np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")


def pin_resample_identity(lib):
    """phi = 0: every sample lands on its own voxel, W = F exactly."""
    rng = _rng(31)
    worst = 0.0
    for shape, spacing, _ in RESAMPLE_CASES:
        F = rng.normal(size=shape)
        phi = np.zeros(oracle.grid_shape(shape, spacing) + (3,))
        worst = max(worst, float(np.max(np.abs(oracle.resample(phi, shape, spacing, F, lib=lib) - F))))
    return worst, 1e-15


def pin_resample_integer_shift(lib):
    """phi = integer constant (a, b, c): W(x) = F(x + a, y + b, z + c), and 0 where
    that voxel lies outside the floating image (of another size than the volume)."""
    rng = _rng(32)
    worst = 0.0
    for shape, spacing, fshape in RESAMPLE_CASES:
        F = rng.normal(size=fshape)
        for shift in [(2, -1, 3), (-3, 2, -1), (0, 4, 0)]:
            phi = np.broadcast_to(np.array(shift, np.float64), oracle.grid_shape(shape, spacing) + (3,)).copy()
            W = oracle.resample(phi, shape, spacing, F, lib=lib)
            z, y, x = _grid_points(shape)
            xs, ys, zs = x + shift[0], y + shift[1], z + shift[2]
            fZ, fY, fX = fshape
            inside = (xs >= 0) & (xs < fX) & (ys >= 0) & (ys < fY) & (zs >= 0) & (zs < fZ)
            want = np.where(inside, F[np.clip(zs, 0, fZ - 1), np.clip(ys, 0, fY - 1), np.clip(xs, 0, fX - 1)], 0.0)
            worst = max(worst, float(np.max(np.abs(W - want))))
    return worst, 1e-12


def _scipy_sample(F, px, py, pz):
    """scipy's order-1 spline interpolation with zeros beyond the edges (a library
    routine for the trilinear interpolant extended by zeros)."""
    from scipy import ndimage

    return ndimage.map_coordinates(F, [pz.ravel(), py.ravel(), px.ravel()], order=1, mode="grid-constant",
                                   cval=0.0).reshape(px.shape)


def pin_resample_scipy(lib):
    """Random displacements of several voxels (many samples fall outside the
    image): W equals scipy.ndimage.map_coordinates(order=1, mode='grid-constant')
    at x + T(x), T from the (pinned) forward."""
    rng = _rng(33)
    worst, scale = 0.0, 1.0
    for shape, spacing, fshape in RESAMPLE_CASES:
        F = rng.normal(size=fshape)
        phi = rng.uniform(-4, 4, oracle.grid_shape(shape, spacing) + (3,))
        T = oracle.forward(phi, shape, spacing, lib=lib)
        z, y, x = _grid_points(shape)
        want = _scipy_sample(F, x + T[..., 0], y + T[..., 1], z + T[..., 2])
        W = oracle.resample(phi, shape, spacing, F, lib=lib)
        worst = max(worst, float(np.max(np.abs(W - want))))
        scale = max(scale, float(np.max(np.abs(F))))
    return worst, 1e-12 * scale


def pin_resample_affine_image(lib):
    """F affine in the voxel coordinates and every sample inside the image:
    trilinear interpolation reproduces it, W(x) = k . (x + T(x)) + c."""
    rng = _rng(34)
    worst, scale = 0.0, 1.0
    shape, spacing = (10, 11, 12), (3, 2, 4)
    Z, Y, X = shape
    k, c0 = rng.uniform(-2, 2, 3), 0.7
    z, y, x = _grid_points(shape)
    F = k[0] * x + k[1] * y + k[2] * z + c0
    phi = rng.uniform(-0.9, 0.9, oracle.grid_shape(shape, spacing) + (3,))
    T = oracle.forward(phi, shape, spacing, lib=lib)
    p = np.stack([x + T[..., 0], y + T[..., 1], z + T[..., 2]], -1)
    inside = np.all((p >= 0) & (p <= np.array([X - 1, Y - 1, Z - 1])), axis=-1)
    W = oracle.resample(phi, shape, spacing, F, lib=lib)
    want = p @ k + c0
    worst = float(np.max(np.abs(W - want)[inside]))
    scale = float(np.max(np.abs(want)))
    assert inside.mean() > 0.5
    return worst, 1e-13 * scale


def pin_resample_grad_scipy_fd(lib):
    """G / dW is the gradient of the interpolant at x + T(x): central differences
    of scipy's interpolant (samples with any coordinate within 1e-3 of an
    integer, where the interpolant has a kink, are left out)."""
    rng = _rng(35)
    worst, scale = 0.0, 1.0
    for shape, spacing, fshape in RESAMPLE_CASES:
        F = rng.normal(size=fshape)
        phi = rng.uniform(-3, 3, oracle.grid_shape(shape, spacing) + (3,))
        dW = rng.normal(size=shape)
        G = oracle.resample_grad(phi, shape, spacing, F, dW, lib=lib)
        T = oracle.forward(phi, shape, spacing, lib=lib)
        z, y, x = _grid_points(shape)
        p = [x + T[..., 0], y + T[..., 1], z + T[..., 2]]
        frac = np.stack([q - np.floor(q) for q in p], -1)
        ok = np.all((frac > 1e-3) & (frac < 1 - 1e-3), axis=-1)
        h = 1e-6
        for ch in range(3):
            hi = [q + (h if i == ch else 0.0) for i, q in enumerate(p)]
            lo = [q - (h if i == ch else 0.0) for i, q in enumerate(p)]
            fd = (_scipy_sample(F, *hi) - _scipy_sample(F, *lo)) / (2 * h)
            worst = max(worst, float(np.max(np.abs(G[..., ch] - dW * fd)[ok])))
        scale = max(scale, float(np.max(np.abs(G))))
    return worst, 1e-7 * scale


def pin_resample_backward_fd(lib):
    """dL/dphi (adjoint of G) against central differences of
    L(phi) = sum dW * W(phi) through the oracle's own resampling."""
    rng = _rng(36)
    shape, spacing, fshape = (8, 7, 9), (3, 2, 3), (9, 8, 10)
    F = rng.normal(size=fshape)
    phi = rng.uniform(-2, 2, oracle.grid_shape(shape, spacing) + (3,))
    dW = rng.normal(size=shape)
    grad = oracle.resample_backward(phi, shape, spacing, F, dW, lib=lib)
    worst = 0.0
    eps = 1e-7
    for _ in range(12):
        idx = tuple(int(rng.integers(0, s)) for s in phi.shape)
        p1, p2 = phi.copy(), phi.copy()
        p1[idx] += eps
        p2[idx] -= eps
        fd = (np.sum(dW * oracle.resample(p1, shape, spacing, F, lib=lib))
              - np.sum(dW * oracle.resample(p2, shape, spacing, F, lib=lib))) / (2 * eps)
        worst = max(worst, abs(fd - grad[idx]))
    return worst, 1e-5 * max(1.0, float(np.max(np.abs(grad))))


# ---------------------------------------------------------------- non-integer spacing
# Spacing num/den and lattice shift off/den voxels per axis ((z, y, x) order):
# u = (x den + off) / num (Sec. 8's grids not aligned to the voxel grid).

RATIONAL_CASES = [  # (shape, num, den, off)
    ((7, 9, 11), (5, 7, 9), (2, 2, 2), (0, 3, 1)),        # spacings 2.5, 3.5, 4.5
    ((6, 10, 13), (4, 3, 10), (3, 1, 3), (2, 0, 7)),       # 1.33, 3, 3.33; shifted lattices
    ((5, 8, 9), (1, 9, 7), (1, 4, 5), (0, 8, 6)),          # 1, 2.25, 1.4
]


def _rat_u(N, n, d, o):
    return (np.arange(N, dtype=np.float64) * d + o) / n


def pin_rational_integer_case(lib):
    """den = 1, off = 0 is integer spacing: the same values as the integer oracle."""
    rng = _rng(41)
    worst = 0.0
    for shape, spacing in SMALL_CASES[:4]:
        phi = rng.uniform(-2, 2, oracle.grid_shape(shape, spacing) + (3,))
        a = oracle.forward(phi, shape, spacing, lib=lib)
        b = oracle.forward_rational(phi, shape, spacing, (1, 1, 1), (0, 0, 0), lib=lib)
        worst = max(worst, float(np.max(np.abs(a - b))))
    return worst, 0.0


def pin_rational_brute_force(lib):
    """The global sum over all grid points of phi_g beta3(u - g + 1) per axis."""
    rng = _rng(42)
    worst = 0.0
    for shape, num, den, off in RATIONAL_CASES:
        grid = oracle.rational_grid_shape(shape, num, den, off)
        phi = rng.uniform(-2, 2, grid + (3,))
        W = [beta3(_rat_u(N, n, d, o)[:, None] - np.arange(g, dtype=np.float64)[None, :] + 1.0)
             for N, n, d, o, g in zip(shape, num, den, off, grid)]
        want = np.einsum("zc,yb,xa,cbad->zyxd", W[0], W[1], W[2], phi, optimize=True)
        T = oracle.forward_rational(phi, shape, num, den, off, lib=lib)
        worst = max(worst, float(np.max(np.abs(T - want))))
    return worst, 1e-13


def pin_rational_scipy(lib):
    """scipy's tensor-product cubic B-spline (knots at the integers, starting at
    -3) evaluated at the lattice coordinates u."""
    from scipy.interpolate import NdBSpline

    rng = _rng(43)
    worst = 0.0
    for shape, num, den, off in RATIONAL_CASES:
        grid = oracle.rational_grid_shape(shape, num, den, off)
        phi = rng.uniform(-2, 2, grid + (3,))
        spl = NdBSpline(tuple(np.arange(g + 4, dtype=np.float64) - 3.0 for g in grid), phi, 3)
        uz, uy, ux = (_rat_u(N, n, d, o) for N, n, d, o in zip(shape, num, den, off))
        Z, Y, X = shape
        z, y, x = np.meshgrid(uz, uy, ux, indexing="ij")
        want = spl(np.stack([z, y, x], -1).reshape(-1, 3)).reshape(Z, Y, X, 3)
        T = oracle.forward_rational(phi, shape, num, den, off, lib=lib)
        worst = max(worst, float(np.max(np.abs(T - want))))
    return worst, 1e-12


def pin_rational_affine(lib):
    """Control point g at voxel coordinate (g - 1) num/den - off/den per axis and
    phi affine in it: T(x) = A x + b exactly (the index origin and the shift)."""
    rng = _rng(44)
    worst, scale = 0.0, 1.0
    for shape, num, den, off in RATIONAL_CASES:
        grid = oracle.rational_grid_shape(shape, num, den, off)
        A, b = rng.uniform(-2, 2, (3, 3)), rng.uniform(-5, 5, 3)
        pos = [(np.arange(g, dtype=np.float64) - 1.0) * n / d - o / d for g, n, d, o in zip(grid, num, den, off)]
        gz, gy, gx = np.meshgrid(*pos, indexing="ij")
        phi = np.stack([gx, gy, gz], -1) @ A.T + b
        T = oracle.forward_rational(phi, shape, num, den, off, lib=lib)
        Z, Y, X = shape
        z, y, x = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
        want = np.stack([x, y, z], -1).astype(np.float64) @ A.T + b
        worst = max(worst, float(np.max(np.abs(T - want))))
        scale = max(scale, float(np.max(np.abs(want))))
    return worst, 1e-13 * scale


def pin_rational_adjoint_brute_force(lib):
    """The transpose of the explicit weight matrices of pin_rational_brute_force:
    dphi = sum over voxels of beta3 products times grad."""
    rng = _rng(46)
    worst, scale = 0.0, 1.0
    for shape, num, den, off in RATIONAL_CASES:
        grid = oracle.rational_grid_shape(shape, num, den, off)
        G = rng.normal(size=shape + (3,))
        W = [beta3(_rat_u(N, n, d, o)[:, None] - np.arange(g, dtype=np.float64)[None, :] + 1.0)
             for N, n, d, o, g in zip(shape, num, den, off, grid)]
        want = np.einsum("zc,yb,xa,zyxd->cbad", W[0], W[1], W[2], G, optimize=True)
        got = oracle.adjoint_rational(G, num, den, off, lib=lib)
        worst = max(worst, float(np.max(np.abs(got - want))))
        scale = max(scale, float(np.max(np.abs(want))))
    return worst, 1e-13 * scale


def pin_rational_adjoint_dot_product(lib):
    """<forward_rational(phi), G> = <phi, adjoint_rational(G)>, and den = 1,
    off = 0 gives the integer adjoint."""
    rng = _rng(47)
    worst = 0.0
    for shape, num, den, off in RATIONAL_CASES:
        phi = rng.uniform(-2, 2, oracle.rational_grid_shape(shape, num, den, off) + (3,))
        G = rng.normal(size=shape + (3,))
        lhs = float(np.sum(oracle.forward_rational(phi, shape, num, den, off, lib=lib) * G))
        rhs = float(np.sum(phi * oracle.adjoint_rational(G, num, den, off, lib=lib)))
        worst = max(worst, abs(lhs - rhs) / max(abs(lhs), 1.0))
    for shape, spacing in SMALL_CASES[:3]:
        G = rng.normal(size=shape + (3,))
        a = oracle.adjoint(G, spacing, lib=lib)
        b = oracle.adjoint_rational(G, spacing, (1, 1, 1), (0, 0, 0), lib=lib)
        worst = max(worst, float(np.max(np.abs(a - b))) / max(float(np.max(np.abs(a))), 1.0))
    return worst, 1e-12


def pin_new_points_match_dense(lib):
    """The point-wise resampling and non-integer-spacing functions agree with the
    dense ones (value and interpolant gradient)."""
    rng = _rng(45)
    worst = 0.0
    shape, spacing, fshape = RESAMPLE_CASES[1]
    F = rng.normal(size=fshape)
    phi = rng.uniform(-3, 3, oracle.grid_shape(shape, spacing) + (3,))
    dW = np.ones(shape)
    W = oracle.resample(phi, shape, spacing, F, lib=lib)
    G = oracle.resample_grad(phi, shape, spacing, F, dW, lib=lib)
    pts = synth_points(shape, 60, rng)
    v, g = oracle.resample_points(phi, shape, spacing, F, pts, lib=lib)
    worst = max(worst, float(np.max(np.abs(v - W[pts[:, 2], pts[:, 1], pts[:, 0]]))),
                float(np.max(np.abs(g - G[pts[:, 2], pts[:, 1], pts[:, 0]]))))
    for shape, num, den, off in RATIONAL_CASES:
        phi = rng.uniform(-2, 2, oracle.rational_grid_shape(shape, num, den, off) + (3,))
        T = oracle.forward_rational(phi, shape, num, den, off, lib=lib)
        pts = synth_points(shape, 40, rng)
        Tp = oracle.forward_rational_points(phi, shape, num, den, off, pts, lib=lib)
        worst = max(worst, float(np.max(np.abs(Tp - T[pts[:, 2], pts[:, 1], pts[:, 0]]))))
        G = rng.normal(size=shape + (3,))
        D = oracle.adjoint_rational(G, num, den, off, lib=lib)
        gp = synth_points(D.shape[:3], 40, rng)
        Dp = oracle.adjoint_rational_points(G, num, den, off, gp, lib=lib)
        worst = max(worst, float(np.max(np.abs(Dp - D[gp[:, 2], gp[:, 1], gp[:, 0]]))))
    return worst, 1e-12


def synth_points(shape, n, rng):
    Z, Y, X = shape
    return np.stack([rng.integers(0, X, n), rng.integers(0, Y, n), rng.integers(0, Z, n)], 1).astype(np.int64)


ALL_PINS = [
    pin_partition_of_unity,
    pin_affine_reproduction,
    pin_knot_values,
    pin_brute_force,
    pin_scipy_tensor_bspline,
    pin_scipy_1d_curve,
    pin_adjoint_brute,
    pin_adjoint_dot_product,
    pin_adjoint_finite_difference,
    pin_points_match_dense,
    pin_resample_identity,
    pin_resample_integer_shift,
    pin_resample_scipy,
    pin_resample_affine_image,
    pin_resample_grad_scipy_fd,
    pin_resample_backward_fd,
    pin_rational_integer_case,
    pin_rational_brute_force,
    pin_rational_scipy,
    pin_rational_affine,
    pin_rational_adjoint_brute_force,
    pin_rational_adjoint_dot_product,
    pin_new_points_match_dense,
]


def failed_pins(lib):
    """Names of the pins that do not hold for ``lib``."""
    bad = []
    for pin in ALL_PINS:
        try:
            err, tol = pin(lib)
        except oracle.OracleError:   # the oracle refused its own arithmetic (an index out of range)
            bad.append(pin.__name__)
            continue
        if not (err <= tol):
            bad.append(pin.__name__)
    return bad
