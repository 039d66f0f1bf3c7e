"""Independent textbook formulas used to pin the oracle (not oracle code).

The piecewise-polynomial forms of the centred B-splines of degree 0..3 and a
few closed-form geometric quantities, each written out from its classic
definition.
"""
import numpy as np


def bspline(n, x):
    """Centred B-spline of degree n (piecewise form); beta^0 on [-1/2, 1/2)."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    if n == 0:
        return ((x >= -0.5) & (x < 0.5)).astype(np.float64)
    if n == 1:
        return np.maximum(0.0, 1.0 - a)
    if n == 2:
        return np.where(a < 0.5, 0.75 - a * a, np.where(a < 1.5, 0.5 * (a - 1.5) ** 2, 0.0))
    if n == 3:
        return np.where(a < 1.0, 2.0 / 3.0 - a * a + 0.5 * a ** 3, np.where(a < 2.0, (2.0 - a) ** 3 / 6.0, 0.0))
    raise ValueError(n)


def box_chord(lo, hi, s, w):
    """Length of the line s + t w inside the box [lo, hi] (slab method)."""
    t0, t1 = -np.inf, np.inf
    for d in range(3):
        if w[d] == 0.0:
            if not (lo[d] <= s[d] <= hi[d]):
                return 0.0
            continue
        a, b = (lo[d] - s[d]) / w[d], (hi[d] - s[d]) / w[d]
        t0, t1 = max(t0, min(a, b)), min(t1, max(a, b))
    return max(0.0, t1 - t0)


def pair_set(n, dims, origin, s, w):
    """Every grid index k (linear, C-order [z][y][x]) whose open support cube
    [k - W, k + W]^3 meets the line in a segment of positive length, by
    brute force over the whole grid."""
    W = 0.5 * (n + 1)
    nx, ny, nz = dims
    kz, ky, kx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ctr = np.stack([origin[0] + kx, origin[1] + ky, origin[2] + kz], axis=-1).reshape(-1, 3)
    t0 = np.full(ctr.shape[0], -np.inf)
    t1 = np.full(ctr.shape[0], np.inf)
    ok = np.ones(ctr.shape[0], dtype=bool)
    for d in range(3):
        p = s[d] - ctr[:, d]
        if w[d] == 0.0:
            ok &= bspline(n, p) != 0.0
            continue
        a, b = (-W - p) / w[d], (W - p) / w[d]
        t0 = np.maximum(t0, np.minimum(a, b))
        t1 = np.minimum(t1, np.maximum(a, b))
    ok &= t1 > t0
    return set(np.nonzero(ok)[0].tolist())


def spline_on_points(n, c, origin, X):
    """f(x) = sum_k c_k prod_d beta^n(x_d - origin_d - k_d) at points X [P,3],
    c in C-order [z][y][x]."""
    nz, ny, nx = c.shape
    Bx = bspline(n, X[:, 0:1] - origin[0] - np.arange(nx)[None, :])
    By = bspline(n, X[:, 1:2] - origin[1] - np.arange(ny)[None, :])
    Bz = bspline(n, X[:, 2:3] - origin[2] - np.arange(nz)[None, :])
    return np.einsum("zyx,pz,py,px->p", c, Bz, By, Bx, optimize=True)
